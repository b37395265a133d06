"""Multi-process host logic of the replica (one process per GPU) bench path,
run as world_size-2 gloo ranks on the CPU: each rank renders its own replica
(distinct random stream), the job time is the slowest rank's, and the job
throughput counts every rank's samples."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench

    class A:
        size, spp, workload = 64, 16, "procedural"
    scene, view = bench.workload(A, rank)
    ms = 100.0 + 50.0 * rank  # rank 1 is the slow replica
    t_max = bench.reduce_max(ms, world)
    value = bench.job_throughput(view["width"] * view["height"] * view["spp"], t_max, world)
    q.put((rank, view["view_index"], t_max, value, len(scene["tri_mat"])))
    dist.barrier()
    dist.destroy_process_group()


def test_two_replicas_gloo():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=300)
        assert p.exitcode == 0
    res = sorted(q.get(timeout=10) for _ in range(2))
    assert [r[1] for r in res] == [0, 1]          # distinct random streams
    assert all(r[2] == 150.0 for r in res)        # max over ranks
    samples = 64 * 64 * 16
    assert all(abs(r[3] - 2 * samples / 0.150 / 1e6) < 1e-9 for r in res)
    assert res[0][4] == res[1][4]                 # the same scene on every rank


def test_reference_arm_other_ranks_exit_without_work(monkeypatch):
    """Under torchrun only rank 0 runs the oracle reference arm."""
    import bench
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")

    class A:
        size, spp, steps, warmup, gpus, workload = 64, 16, 1, 1, 2, "procedural"
    assert bench.run_reference(A) is None
