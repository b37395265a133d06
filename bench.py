#!/usr/bin/env python
"""Throughput of backward generalized-ray path tracing on one GB300 (or N
independent replicas), in path samples per second.

Workload (default): the procedural scene -- ground plane plus 64 objects,
~92k triangles, rough Gaussian-statistics conductors and gratings, 1-4
partially coherent emissive quads -- seen by a 512x512 camera at 256 samples
per pixel, 32 spectral bins (400-700 nm), full Stokes vector, up to 3
interactions, next-event estimation with MIS.  One step renders all
512*512*256 = 67.1M path samples.  Inputs are synthetic (seeded generator); the
paper's own scenes are not available.

Prints one JSON line (rank 0).  At N = 1 the line also carries, under
`extras`, the other workloads' measurements, each run after the timed region
and bounded to seconds (--no-extras skips them): the glass workload (f2) on a
crop where the glass decides most pixel-bins, hero-wavelength MIS (f1) with its
variance and efficiency, anisotropic footprints (f4), the batched form
(config 4) against the plain per-view form with and without a graph, the
progressive serving loop (config 5) with p50/p99 frame latency, the order-table
precision form (configs 1 and 3) and the double slit at scale (f3), each
against the FP64 oracle where it has an image.  `--impl reference` times the
FP64 CPU oracle on a bounded crop of the same workload instead.
"""
import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "gen-ray path Msamples/s at <=1e-3 rel-L2 vs FP64 oracle; p50/p99 frame ms"
UNIT = "Msamples/s"
FP32_PEAK_TFLOPS = 2 * 152 * 128 * 2.070e9 / 1e12  # nominal: FMA = 2 FLOP, 152 SMs x 128 lanes at 2070 MHz
# Algorithmic FP32 FLOPs (FMA = 2) of the traversal units, counted from the
# operations the closest-hit query needs: a node visit tests two child boxes
# (6 slab FMAs + 11 min/max + 3 for the far-distance widening, compare and
# clip = 26 per box); a watertight triangle test (9 subtractions, 6 shear
# FMAs, 3 edge functions of 1 mul + 1 FMA, 2 adds, 3 mul + 2 FMA for T, 1
# division) = 41.
FLOP_PER_NODE = 52
FLOP_PER_TRI = 41
# a 4-wide quantised node: per child 6 slab FMAs + 11 min/max + 4 for widening
# and compare (25), plus 9 for the node's affine decode (3 mul, 3 sub, 3 mul)
FLOP_PER_WNODE = 109
KERNELS = ["k_regen", "k_trace", "k_shade", "k_shadow"]
# DRAM traffic of the dominant kernel per unit (ray) from one ncu capture:
# dram__bytes_read.sum + dram__bytes_write.sum of the second k_trace launch of
# the 256x256 x 64 spp case (162.50 + 7.37 MB), divided by the rays it traced
# (the full default pool: one slot per ticket, 2,097,152 slots, all live in
# the second iteration, plus about a thousand next-event rays, not counted);
# traffic grows with the rays a launch processes.  Valid only for the
# traversal sources whose hash (source_hash) is recorded with it (else
# reported null).
NCU_TRAFFIC_PER_RAY = {("k_trace", "374dc2e6c0ef425d"): (162.498816e6 + 7.366912e6) / 2097152}
# the glass workload: a constant environment of this radiance lets paths
# refracted through the glass reach a light, and the oracle crop (x0, y0,
# side) is where the glass decides the most pixel-bins of the 512^2 view
GLASS_ENV = 0.05
GLASS_CROP = (0, 144, 96)


def source_hash():
    """Hash of what k_trace's DRAM bytes per ray depend on: the device header
    (traversal, BVH layout), the slot-pool layout, the BVH builder (node
    order) and the trace section of the render source (the queue schedule and
    the kernel)."""
    csrc = os.path.join(ROOT, "paper_2303_15762_gb300", "csrc")
    h = hashlib.sha256()
    for f in ["gr_device.cuh", "gr_build.h", "gr_bvh.cu"]:
        with open(os.path.join(csrc, f), "rb") as fh:
            h.update(fh.read())
    with open(os.path.join(csrc, "gr_render.cu"), "rb") as fh:
        text = fh.read()
    start = text.index(b"// ------------------------------------------------------------------ trace")
    end = text.index(b"// ------------------------------------------------------------------ footprint")
    h.update(text[start:end])
    return h.hexdigest()[:16]


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--spp", type=int, default=256)
    ap.add_argument("--size", type=int, default=512)
    ap.add_argument("--table", default="f32", choices=["f32", "f16", "bf16"])
    ap.add_argument("--pool", type=int, default=0)
    ap.add_argument("--wide", action="store_true", help="traverse the 4-wide quantised BVH")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true", help="skip the other workloads' legs of the default run")
    ap.add_argument("--extras", default="dielectric,hero,aniso,batched,serving,precision,doubleslit,aperture3d",
                    help="legs of the default run (comma list)")
    ap.add_argument("--cpu-crop", type=int, default=128, help="side of the oracle's centre crop")
    ap.add_argument("--e2e-steps", type=int, default=2)
    ap.add_argument("--workload", choices=["procedural", "batched", "serving", "precision", "dielectric",
                                           "doubleslit", "hero", "aniso", "aperture3d"],
                    default="procedural",
                    help="procedural: the headline single-view workload; batched: 64 views/scenes, plain "
                         "per-view FP32 form vs the autotuned single-graph form; serving: "
                         "Poisson-arriving progressive requests; precision: FP32/FP16/BF16 order tables, "
                         "image and per-quantity errors vs the FP64 oracle; dielectric: the procedural "
                         "workload with refracting glass slabs; doubleslit: footprint-resolved generalized "
                         "rays through two slits at scale; hero: the procedural workload with "
                         "hero-wavelength spectral MIS vs without (throughput, variance, efficiency); "
                         "aniso: the procedural workload with anisotropic footprints vs the scalar model")
    ap.add_argument("--views", type=int, default=64)
    ap.add_argument("--rate", type=float, default=20.0)
    ap.add_argument("--rates", default="5,50,100", help="serving: further arrival rates to sweep (req/s)")
    ap.add_argument("--requests", type=int, default=24)
    ap.add_argument("--frames", type=int, default=64)
    return ap.parse_args()


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def reduce_max(value, world):
    """Max over ranks (the slowest replica sets the whole job's time)."""
    if world <= 1:
        return float(value)
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(value)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(samples_per_rank, t_max_ms, world):
    """Whole-job Msamples/s: every rank renders its own replica (weak scaling)."""
    return world * samples_per_rank / (t_max_ms * 1e-3) / 1e6


def workload(args, rank):
    from paper_2303_15762_gb300 import scenegen as sg
    scene = sg.procedural_scene(seed=2)
    if args.workload == "dielectric":
        scene = sg.add_glass(scene, env_radiance=GLASS_ENV)
    view = sg.procedural_view(width=args.size, height=args.size, spp=args.spp, view_index=rank)
    return scene, view


def workload_name(args, scene):
    glass = (" with 8 dispersive glass slabs (n = 1.5 + 0.0042/lambda^2) and a constant environment of radiance %g"
             % GLASS_ENV) if args.workload == "dielectric" else ""
    return ("procedural scene%s, %d tris, %dx%d, %d spp, 32 bins 400-700 nm, 4 Stokes, depth<=3, NEE+MIS"
            % (glass, len(scene["tri_mat"]), args.size, args.size, args.spp))


class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.p = None
        self.gpu = gpu_index
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(gpu_index), "--query-gpu=" + self.FIELDS,
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.p = None

    def stop(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        try:
            out, _ = self.p.communicate(timeout=5)
        except Exception:
            self.p.kill()
            out = ""
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


def run_reference(args):
    """FP64 CPU oracle on a bounded crop of the same workload."""
    world, rank, _ = dist_setup()
    if rank != 0:
        return
    from oracle import oracle as orc
    scene, view = workload(args, 0)
    S = orc.Scene(scene)
    crop = 32
    x0 = args.size // 2 - crop // 2
    box = (x0, x0, x0 + crop, x0 + crop)
    samples = crop * crop * args.spp
    cores = os.cpu_count() or 1
    for _ in range(args.warmup):
        S.render(view, 2, orc.FLAG_NEE, crop=box, n_threads=cores)
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        S.render(view, 2, orc.FLAG_NEE, crop=box, n_threads=cores)
        times.append(time.perf_counter() - t0)
    ms = 1e3 * statistics.mean(times)
    value = samples / (ms * 1e-3) / 1e6
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": workload_name(args, scene), "sample": "%dx%d centre crop" % (crop, crop)},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": "%dx%d centre crop x %d spp per step" % (crop, crop, args.spp)},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def _timed(fn, flush, stream):
    """Device time of fn() in ms (CUDA events on the render stream, L2 flushed first)."""
    import torch
    flush.zero_()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    fn()
    e1.record(stream)
    e1.synchronize()
    return e0.elapsed_time(e1)


def run_batched(args):
    """64 seeded views/scenes: the plain per-view FP32 form (one gr_render per
    view with the library's default pool, timed both with the host-driven
    iteration loop and as one graph launch per view) against one autotuned
    render of all views as a single graph launch."""
    import numpy as np
    import torch
    import paper_2303_15762_gb300 as gr
    from paper_2303_15762_gb300 import autotune
    from paper_2303_15762_gb300 import scenegen as sg
    gr.load()
    t0 = time.perf_counter()
    scenes, views = sg.batch_views(seed=4, n_views=args.views)
    gen_s = time.perf_counter() - t0
    t0 = time.perf_counter()
    S = [gr.Scene(s) for s in scenes]
    torch.cuda.synchronize()
    build_s = time.perf_counter() - t0
    samples = sum(v["width"] * v["height"] * v["spp"] for v in views)
    flags = gr.FLAG_NEE | gr.FLAG_RR
    stream = torch.cuda.current_stream()
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")
    steps, warmup = max(1, args.steps), max(1, args.warmup)
    plain_frames = [gr.Frame([dict(v, scene_index=0)]) for v in views]

    def plain(graph):
        def run():
            for i, v in enumerate(views):
                plain_frames[i].reset()
                gr.render([S[i]], [dict(v, scene_index=0)], plain_frames[i], seed=2, flags=flags, table_dtype="f32",
                          use_graph=graph)
        return run
    res = {}
    for name, graph in (("plain_host_loop", False), ("plain_graph", True)):
        for _ in range(warmup):
            plain(graph)()
        res[name] = statistics.mean([_timed(plain(graph), flush, stream) for _ in range(steps)])
    best, trials = autotune.autotune(gr, S, views, dict(seed=2, flags=flags, table_dtype="f32", use_graph=True),
                                     probe_spp=max(1, views[0]["spp"] // 4))
    F = gr.Frame(views)

    def batched():
        F.reset()
        gr.render(S, views, F, **best)
    for _ in range(warmup):
        batched()
    res["batched"] = statistics.mean([_timed(batched, flush, stream) for _ in range(steps)])
    val = {k: samples / (ms * 1e-3) / 1e6 for k, ms in res.items()}
    # accuracy: batched vs the oracle on the four smallest views (full images;
    # an image whose oracle norm is below 1e-20 is dark -- FP32 cannot carry
    # the 1e-30-scale tails that remain there -- and is reported as null)
    from oracle import oracle as orc
    rels = {}
    for i in sorted(range(len(views)), key=lambda k: views[k]["width"] * views[k]["height"])[:4]:
        ref = orc.Scene(scenes[i]).render(views[i], 2, orc.FLAG_NEE | orc.FLAG_RR)
        nr = float(np.linalg.norm(ref))
        got = F.readback(i).astype(np.float64)
        rels[i] = ({"rel_l2": float(np.linalg.norm(got - ref) / nr),
                    "max_elem_err_over_max": float(np.max(np.abs(got - ref)) / np.max(np.abs(ref)))}
                   if nr >= 1e-20 else None)
    identical = all(np.array_equal(F.readback(i), plain_frames[i].readback(0)) for i in range(len(views)))
    st = F.stats()
    for f in plain_frames:
        f.close()
    F.close()
    for s_ in S:
        s_.close()
    tabs = {t[0]["table_dtype"] for t in trials}
    return {"workload": "batched (config 4)", "metric": METRIC, "unit": UNIT, "value": val["batched"],
            "plain_graph_value": val["plain_graph"], "plain_host_loop_value": val["plain_host_loop"],
            "speedup_vs_plain_graph": val["batched"] / val["plain_graph"],
            "speedup_vs_plain_host_loop": val["batched"] / val["plain_host_loop"],
            "ms": res, "samples_per_step": samples, "n_views": len(views), "steps": steps, "warmup": warmup,
            "plain_form": "one gr_render per view, FP32 tables, the library's default pool (one slot per ticket)",
            "tris_range": [min(len(s["tri_mat"]) for s in scenes), max(len(s["tri_mat"]) for s in scenes)],
            "side_range": [min(v["width"] for v in views), max(v["width"] for v in views)],
            "autotuned": {k: best[k] for k in ("pool_size", "block", "regen_threshold_pct", "table_dtype")},
            "tables_tried": sorted(tabs),
            "autotune_trials": [[t[0]["pool_size"], t[0]["block"], t[0]["regen_threshold_pct"], t[0]["table_dtype"],
                                 round(t[1], 3)] for t in trials],
            "oracle_four_smallest_views": rels, "batched_equals_per_view_bitwise": identical,
            "graph_launches_per_render": 1, "iterations": st["iterations"],
            "scene_gen_s": gen_s, "scene_build_s": build_s,
            "l2": "flushed before every timed step (256 MB write)"}


def run_serving(args, rates=None):
    """Poisson-arriving progressive requests (config 5): p50/p99 inter-frame
    and first-frame latency, throughput over wall time and over device-busy
    time, at the headline arrival rate and optionally a sweep."""
    import numpy as np
    import paper_2303_15762_gb300 as gr
    from paper_2303_15762_gb300 import scenegen as sg
    from paper_2303_15762_gb300 import serving
    gr.load()

    def make(rng):
        return [serving.Request(k + 1, *sg.serving_request(rng, k + 1), args.frames) for k in range(args.requests)]
    opts = dict(seed=1, flags=0, table_dtype="f32", use_graph=True)
    # warm-up pass (graph builds, allocator) on a few requests
    srv = serving.ProgressiveServer(gr, render_opts=opts)
    serving.run_poisson(gr, make(np.random.default_rng(5))[:3], 1000.0, srv)
    srv.close()
    rates = [args.rate] if rates is None else rates
    runs = {}
    for rate in rates:
        srv = serving.ProgressiveServer(gr, render_opts=opts)
        runs[rate] = serving.run_poisson(gr, make(np.random.default_rng(5)), rate, srv, seed=6)
        srv.close()
    res = dict(runs[rates[0]])
    keys = ("msamples_per_s", "msamples_per_busy_s", "p50_frame_ms", "p99_frame_ms", "p50_first_frame_ms",
            "p99_first_frame_ms", "p50_arrival_to_first_frame_ms", "p99_arrival_to_first_frame_ms", "device_frames",
            "wall_s")
    res.update({"workload": "serving (config 5)", "metric": METRIC, "unit": UNIT, "value": res["msamples_per_s"],
                "value_basis": "samples over wall-clock time of the run (msamples_per_busy_s: over device-busy time)",
                "rate_req_per_s": rates[0], "frames_per_request": args.frames, "requests_submitted": args.requests,
                "resolutions": "256^2, 512^2, 1280x720, 1920x1080, 16 bins, 1 spp per frame"})
    if len(rates) > 1:
        res["rate_sweep"] = [dict(rate_req_per_s=r, **{k: runs[r][k] for k in keys}) for r in sorted(runs)]
    return res


def run_precision(args):
    """Planar-grating workload (config 1) with FP32 / FP16 / BF16 order tables
    (config 3): image rel-L2 vs the FP64 oracle and vs the FP32-table image,
    and per-quantity errors vs FP64 (stored order weights a_j; beta^2 and rho
    along three-segment chains) through the library's inspection calls."""
    import math
    import numpy as np
    import torch
    import paper_2303_15762_gb300 as gr
    from paper_2303_15762_gb300 import scenegen as sg
    from oracle import oracle as orc
    gr.load()
    scene, view = sg.grating_scene(), sg.grating_view()
    cores = os.cpu_count() or 1
    t0 = time.perf_counter()
    ref = orc.Scene(scene).render(view, 1, 0, n_threads=cores)
    oracle_s = time.perf_counter() - t0
    samples = view["width"] * view["height"] * view["spp"]
    S = gr.Scene(scene)
    F = gr.Frame([view])
    stream = torch.cuda.current_stream()
    out = {}
    img32 = None
    for dt in ("f32", "f16", "bf16"):
        times = []
        for r in range(args.warmup + args.steps):
            F.reset()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            gr.render([S], [view], F, seed=1, table_dtype=dt)
            e1.record(stream)
            e1.synchronize()
            if r >= args.warmup:
                times.append(e0.elapsed_time(e1))
        img = F.readback(0).astype(np.float64)
        if img32 is None:
            img32 = img
        # order weights of the workload's 16 bins: relative error where the
        # type is normal, absolute error where it is not (FP16 below 2^-14)
        tiny = {"f32": 1.2e-38, "f16": 6.1e-5, "bf16": 1.2e-38}[dt]
        worst_rel = worst_abs = 0.0
        for b in range(view["n_bins"]):
            lam = 0.4 + 0.3 * b / (view["n_bins"] - 1)
            jmax = int(2 * 1.6 / lam) + 2
            got = gr.debug_order_table(0.2, lam, jmax, dt).astype(np.float64)
            x = math.pi * float(np.float32(0.2)) / lam
            a = np.array([orc.bessel_j(j, x) ** 2 for j in range(jmax + 1)])
            nrm = a >= tiny
            if nrm.any():
                worst_rel = max(worst_rel, float(np.max(np.abs(got - a)[nrm] / a[nrm])))
            if (~nrm).any():
                worst_abs = max(worst_abs, float(np.max(np.abs(got - a)[~nrm])))
        out[dt] = {"rel_l2_vs_oracle": float(np.linalg.norm(img - ref) / np.linalg.norm(ref)),
                   "max_elem_err_over_max": float(np.max(np.abs(img - ref)) / np.max(np.abs(ref))),
                   "rel_l2_vs_f32_tables": float(np.linalg.norm(img - img32) / np.linalg.norm(img32)),
                   "max_rel_err_a_j_normal_range": worst_rel, "max_abs_err_a_j_below_normal": worst_abs,
                   "ms_per_render": statistics.mean(times),
                   "msamples_per_s": samples / (statistics.mean(times) * 1e-3) / 1e6}
    # footprint: three segments of 0.05-5 m from a camera footprint (beta0 = 1 um)
    rng = np.random.default_rng(11)
    n = 2000
    seg = rng.uniform(0.05, 5.0, (n, 3)).astype(np.float32)
    kw = (2 * math.pi / rng.uniform(0.4, 0.7, n)).astype(np.float32)
    st = np.stack([np.ones(n, np.float32), np.zeros(n, np.float32)], axis=1)
    rf = [(1.0, 0.0)] * n
    for k in range(3):
        st = gr.debug_footprint(np.stack([st[:, 0], st[:, 1], seg[:, k], kw], axis=1))
        rf = [orc.propagate(b, r, float(seg[i, k]) * 1e6 / float(kw[i])) for i, (b, r) in enumerate(rf)]
    rf = np.array(rf)
    F.close()
    S.close()
    return {"workload": "precision (configs 1 and 3)", "metric": METRIC, "unit": UNIT,
            "value": out["f32"]["msamples_per_s"],
            "config": "planar grating 64x64, 64 spp, 16 bins 400-700 nm, 1 interaction, S0",
            "tables": out,
            "cpu_baseline": {"value": samples / oracle_s / 1e6, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": "the full workload (%d samples), %.2f s" % (samples, oracle_s)},
            "footprint_fp32_vs_fp64_3_segments": {
                "max_rel_err_beta2": float(np.max(np.abs(st[:, 0] - rf[:, 0]) / rf[:, 0])),
                "max_rel_err_rho": float(np.max(np.abs(st[:, 1] - rf[:, 1]) / np.abs(rf[:, 1])))}}


def run_doubleslit(args):
    """Double slit at scale (Sec. 5.1-5.2 with the footprint-resolved
    propagation of Sec. 6): 4001 detector elements across +-2000 wavelengths,
    d = 400, b = 40, z = 10^4, every element integrated over its ~8300
    directions, each overlapped with 800 aperture samples.  Unit: generalized
    rays (element x direction) per second; the oracle's FP64 computation of
    the same sums on a bounded sample of elements is the CPU baseline."""
    import numpy as np
    import paper_2303_15762_gb300 as gr
    from paper_2303_15762_gb300 import scenegen as sg
    from oracle import doubleslit as ds
    gr.load()
    s = sg.double_slit_setup(d=400.0, x0=np.linspace(-2000.0, 2000.0, 4001))
    th = lambda x0: int(np.ceil((np.arctan((x0 + s["reach"]) / s["z"]) - np.arctan((x0 - s["reach"]) / s["z"]))
                                / s["dtheta"]))
    rays = sum(th(x) for x in s["x0"])
    args_ = (s["x0"], s["x_ap"], s["w_ap"], s["beta"], s["z"], s["k"], s["reach"], s["dtheta"], s["rho_cut"])
    for _ in range(args.warmup):
        gr.aperture_backward_2d(*args_)
    times, walls = [], []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        out, ms = gr.aperture_backward_2d(*args_)
        walls.append(time.perf_counter() - t0)
        times.append(ms)
    ms = statistics.mean(times)
    # FP64 oracle on 5 elements, scaled per ray
    sub = s["x0"][::1000]
    t0 = time.perf_counter()
    ref = ds.backward_generalized_rays(sub, 400.0, s["beta"], rho_cut=s["rho_cut"])
    cpu_s = time.perf_counter() - t0
    cpu_rays = sum(th(x) for x in sub)
    err = float(np.max(np.abs(out[::1000] - ref)) / np.max(ref))
    return {"workload": "doubleslit (f3)", "metric": "generalized rays (element x direction) per second, each "
            "overlapped with the aperture samples", "unit": "Mrays/s", "value": rays / (ms * 1e-3) / 1e6,
            "ms_per_step": ms, "wall_ms_per_call": 1e3 * statistics.mean(walls), "steps": args.steps,
            "warmup": args.warmup, "config": {"elements": len(s["x0"]), "rays": rays, "aperture_samples": len(s["x_ap"]),
                                             "d": 400, "b": 40, "z": 1e4, "beta": s["beta"], "rho_cut": s["rho_cut"]},
            "overlaps_per_s": rays * len(s["x_ap"]) / (ms * 1e-3),
            "max_err_vs_oracle_over_peak": err,
            "cpu_baseline": {"value": cpu_rays / cpu_s / 1e6, "unit": "Mrays/s", "cores": 1, "kind": "oracle",
                             "sample": "%d of the elements (%d rays), numpy FP64, %.1f s" % (len(sub), cpu_rays, cpu_s)}}


def run_aperture3d(args):
    """Footprint-resolved generalized rays through a disk aperture in a 3D
    world onto a 48 x 48 screen of detector elements (the double-slit
    validation of Sec. 5.1-5.2 taken to a plane aperture, with the Sec. 6
    truncation): generalized rays (element x direction) per second, and one
    element against the oracle's FP64 sums and against exact 3D
    Rayleigh-Sommerfeld diffraction."""
    import numpy as np
    import paper_2303_15762_gb300 as gr
    from paper_2303_15762_gb300 import scenegen as sg
    from oracle import aperture3d as a3
    gr.load()
    s = sg.aperture3d_setup("disk")
    n_t = int(np.ceil(2 * s["reach"] / (s["z"] * s["dt"])))
    rays = len(s["x0"]) * n_t * n_t
    args_ = (s["x0"], s["x_ap"], s["w_ap"], s["beta"], s["z"], s["k"], s["reach"], s["dt"], s["rho_cut"])
    for _ in range(max(1, args.warmup)):
        gr.aperture_backward_3d(*args_)
    times = []
    for _ in range(max(1, args.steps)):
        out, ms = gr.aperture_backward_3d(*args_)
        times.append(ms)
    ms = statistics.mean(times)
    i0 = int(np.argmin(np.abs(s["x0"][:, 0] - 30.0) + np.abs(s["x0"][:, 1] + 30.0)))
    x0 = s["x0"][i0:i0 + 1]
    t0 = time.perf_counter()
    ref = a3.backward_generalized_rays(x0, s["z"], s["k"], s["x_ap"], s["w_ap"], s["beta"], s["reach"], s["dt"],
                                       s["rho_cut"])
    cpu_s = time.perf_counter() - t0
    exact = a3.forward_exact(x0, s["z"], s["k"], s["x_ap"], s["w_ap"], s["beta"])
    return {"workload": "aperture3d (f3, plane aperture in a 3D world)",
            "metric": "generalized rays (element x direction) per second, each overlapped with the aperture samples",
            "unit": "Mrays/s", "value": rays / (ms * 1e-3) / 1e6, "ms_per_step": ms, "steps": max(1, args.steps),
            "config": {"aperture": "disk of radius 12 wavelengths, %d samples" % len(s["x_ap"]),
                       "elements": len(s["x0"]), "screen": "48 x 48 over +-240", "directions_per_element": n_t * n_t,
                       "z": s["z"], "beta": s["beta"], "beta_at_aperture": s["beta_ap"], "rho_cut": s["rho_cut"]},
            "overlaps_per_s": rays * len(s["x_ap"]) / (ms * 1e-3),
            "element": [float(v) for v in x0[0]],
            "rel_err_vs_oracle_sums": float(abs(out[i0] - ref[0]) / ref[0]),
            "rel_err_vs_exact_rayleigh_sommerfeld": float(abs(out[i0] - exact[0]) / exact[0]),
            "cpu_baseline": {"value": n_t * n_t / cpu_s / 1e6, "unit": "Mrays/s", "cores": 1, "kind": "oracle",
                             "sample": "one element (%d rays), numpy FP64, %.1f s" % (n_t * n_t, cpu_s)}}


def time_modes(args, S, F, view, modes, clock_mode, steps=None, warmup=None):
    """Device time per step (CUDA events, L2 flushed) and per-kernel time of
    each named flag set; nvidia-smi clocks are sampled during `clock_mode`.
    Returns ms, kernel ms per step, clocks and each mode's last image."""
    import torch
    import paper_2303_15762_gb300 as gr
    steps = args.steps if steps is None else steps
    warmup = max(3, args.warmup) if warmup is None else warmup
    stream = torch.cuda.current_stream()
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")  # 256 MB > 129 MB L2

    def step(flags, profile=False):
        F.reset()
        gr.render([S], [view], F, seed=2, flags=flags, table_dtype=args.table, pool_size=args.pool, profile=profile)

    ms, kernel_ms, clk, imgs = {}, {}, None, {}
    for name, flags in modes.items():
        for _ in range(warmup):
            step(flags)
        torch.cuda.synchronize()
        clocks = ClockSampler(0) if name == clock_mode else None
        times, kms = [], [0.0] * 4
        for _ in range(steps):
            times.append(_timed(lambda: step(flags, profile=True), flush, stream))
            st = F.stats()
            for k in range(4):
                kms[k] += st["kernel_ms"][k] / steps
        if clocks is not None:
            clk = clocks.stop()
        ms[name] = statistics.mean(times)
        kernel_ms[name] = {KERNELS[k]: kms[k] for k in range(4)}
        imgs[name] = F.readback(0)
    return ms, kernel_ms, clk, imgs


def _centre_crop(args, side):
    c = min(side, args.size)
    x0 = args.size // 2 - c // 2
    return (x0, x0, x0 + c, x0 + c)


def _crop_parity(img, ref, box):
    import numpy as np
    x0, y0, x1, y1 = box
    got = img[y0:y1, x0:x1].astype(np.float64)
    return {"rel_l2": float(np.linalg.norm(got - ref) / max(np.linalg.norm(ref), 1e-300)),
            "max_elem_err_over_max": float(np.max(np.abs(got - ref)) / max(np.max(np.abs(ref)), 1e-300)),
            "crop": "x %d-%d, y %d-%d of the %dx%d view" % (x0, x1, y0, y1, img.shape[1], img.shape[0])}


def run_aniso(args, steps=None, warmup=None, crop=128):
    """Anisotropic footprints (beta and rho as 2x2 matrices, Sec. 3.1) on the
    headline procedural workload: throughput with and without the flag,
    per-kernel device time, rel-L2 against the oracle's anisotropic model on
    a centre crop, and how far the anisotropic image moves from the scalar
    model's."""
    import numpy as np
    import paper_2303_15762_gb300 as gr
    gr.load()
    scene, view = workload(args, 0)
    samples = view["width"] * view["height"] * view["spp"]
    S = gr.Scene(scene)
    F = gr.Frame([view])
    modes = {"scalar": gr.FLAG_NEE, "aniso": gr.FLAG_NEE | gr.FLAG_ANISO}
    ms, kernel_ms, clk, imgs = time_modes(args, S, F, view, modes, "aniso", steps, warmup)
    st = F.stats()
    a, b = imgs["aniso"].astype(np.float64), imgs["scalar"].astype(np.float64)
    par = None
    if not args.no_cpu_baseline:
        from oracle import oracle as orc
        box = _centre_crop(args, crop)
        ref = orc.Scene(scene).render(view, 2, orc.FLAG_NEE | orc.FLAG_ANISO, crop=box)
        par = _crop_parity(imgs["aniso"], ref, box)
    F.close()
    S.close()
    return {"workload": "aniso (f4)", "metric": METRIC, "unit": UNIT, "value": samples / (ms["aniso"] * 1e-3) / 1e6,
            "scalar_value": samples / (ms["scalar"] * 1e-3) / 1e6, "ms_aniso": ms["aniso"], "ms_scalar": ms["scalar"],
            "kernel_ms_per_step": kernel_ms, "steps": steps or args.steps, "higher_is_better": True,
            "dtype": "f32", "data": "synthetic",
            "config": {"workload": workload_name(args, scene) + ", anisotropic footprints",
                       "l2": "flushed before every timed step (256 MB write)"},
            "vs_oracle_aniso": par,
            "rel_change_vs_scalar_model": float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)),
            "clocks": clk, "stats": {"iterations": st["iterations"], "segments": st["segments"],
                                     "shadow_rays": st["shadow_rays"]}}


def run_hero(args, steps=None, warmup=None, crop=128):
    """Hero-wavelength spectral MIS (Sec. 7.2) on the headline procedural
    workload: throughput with and without the flag, with per-kernel device
    time; rel-L2 of the hero image against the oracle's hero estimator on a
    centre crop; and the variance of both estimators across independent
    seeds at equal samples per pixel, so that efficiency = (variance x time
    per sample) of the plain estimator over that of the hero estimator (> 1:
    hero MIS reaches a given noise sooner)."""
    import numpy as np
    import paper_2303_15762_gb300 as gr
    from paper_2303_15762_gb300 import scenegen as sg
    gr.load()
    scene, view = workload(args, 0)
    samples = view["width"] * view["height"] * view["spp"]
    S = gr.Scene(scene)
    F = gr.Frame([view])
    modes = {"plain": gr.FLAG_NEE, "hero": gr.FLAG_NEE | gr.FLAG_HERO}
    ms, kernel_ms, clk, imgs = time_modes(args, S, F, view, modes, "hero", steps, warmup)
    st = F.stats()
    par = None
    if not args.no_cpu_baseline:
        from oracle import oracle as orc
        box = _centre_crop(args, crop)
        ref = orc.Scene(scene).render(view, 2, orc.FLAG_NEE | orc.FLAG_HERO, crop=box)
        par = _crop_parity(imgs["hero"], ref, box)
    # variance across seeds at equal samples (a smaller view of the same camera)
    vv = sg.procedural_view(width=128, height=128, spp=32)
    Fv = gr.Frame([vv])
    var = {}
    n_seeds = 8
    for name, flags in modes.items():
        ims = []
        for sd in range(n_seeds):
            Fv.reset()
            gr.render([S], [vv], Fv, seed=100 + sd, flags=flags)
            ims.append(Fv.readback(0).astype(np.float64))
        a = np.stack(ims)
        v = np.var(a, axis=0, ddof=1)
        var[name] = {"total": float(v[..., 0].sum()), "mean_intensity": float(a[..., 0].mean())}
    vratio = var["plain"]["total"] / max(var["hero"]["total"], 1e-300)
    Fv.close()
    F.close()
    S.close()
    return {"workload": "hero (f1)", "metric": METRIC, "unit": UNIT, "value": samples / (ms["hero"] * 1e-3) / 1e6,
            "plain_value": samples / (ms["plain"] * 1e-3) / 1e6, "ms_hero": ms["hero"], "ms_plain": ms["plain"],
            "kernel_ms_per_step": kernel_ms, "steps": steps or args.steps, "higher_is_better": True,
            "dtype": "f32", "data": "synthetic",
            "config": {"workload": workload_name(args, scene) + ", hero-wavelength MIS over classes of 4 bins",
                       "l2": "flushed before every timed step (256 MB write)"},
            "vs_oracle_hero": par,
            "variance_ratio_plain_over_hero": vratio,
            "efficiency_plain_over_hero": vratio * ms["plain"] / ms["hero"],
            "variance": {"view": "128x128, 32 spp, 32 bins, intensity (Stokes I), %d seeds per estimator" % n_seeds,
                         **var},
            "clocks": clk, "stats": {"iterations": st["iterations"], "segments": st["segments"],
                                     "shadow_rays": st["shadow_rays"]}}


def run_dielectric(args, steps=None, warmup=None):
    """The glass workload (f2): throughput, and parity with the oracle on the
    crop where the glass decides the most pixel-bins; the fraction of the
    crop's pixel-bins whose oracle value depends on the glass (it differs from
    the same render with the glass removed) says how much of the comparison
    exercises refraction."""
    import numpy as np
    import paper_2303_15762_gb300 as gr
    from paper_2303_15762_gb300 import scenegen as sg
    gr.load()
    a2 = argparse.Namespace(**dict(vars(args), workload="dielectric"))
    scene, view = workload(a2, 0)
    samples = view["width"] * view["height"] * view["spp"]
    S = gr.Scene(scene)
    F = gr.Frame([view])
    ms, kernel_ms, clk, imgs = time_modes(a2, S, F, view, {"glass": gr.FLAG_NEE}, "glass", steps, warmup)
    par = frac = None
    if not args.no_cpu_baseline:
        from oracle import oracle as orc
        x0, y0, c = GLASS_CROP
        box = (x0, y0, x0 + c, y0 + c)
        cores = os.cpu_count() or 1
        ref = orc.Scene(scene).render(view, 2, orc.FLAG_NEE, crop=box, n_threads=cores)
        bare = orc.Scene(sg.env_only(sg.procedural_scene(seed=2), GLASS_ENV)).render(view, 2, orc.FLAG_NEE, crop=box,
                                                                                     n_threads=cores)
        par = _crop_parity(imgs["glass"], ref, box)
        frac = float(np.any(ref != bare, axis=3).mean())
    st = F.stats()
    F.close()
    S.close()
    return {"workload": "dielectric (f2)", "metric": METRIC, "unit": UNIT, "value": samples / (ms["glass"] * 1e-3) / 1e6,
            "ms_per_step": ms["glass"], "kernel_ms_per_step": kernel_ms["glass"], "steps": steps or args.steps,
            "config": {"workload": workload_name(a2, scene), "l2": "flushed before every timed step (256 MB write)"},
            "vs_oracle": par, "glass_fraction_of_crop_pixel_bins": frac,
            "glass_fraction_note": "pixel-bins of the crop whose oracle value changes when the glass is removed",
            "clocks": clk, "stats": {"iterations": st["iterations"], "segments": st["segments"]}}


def run_extras(args):
    """The other workloads' legs, after the headline's timed region: each
    bounded (1 warm-up and 2 timed steps where it times a render) and isolated
    (an error is reported in its place)."""
    legs = {"dielectric": lambda: run_dielectric(args, steps=2, warmup=1),
            "hero": lambda: run_hero(args, steps=2, warmup=1, crop=64),
            "aniso": lambda: run_aniso(args, steps=2, warmup=1, crop=64),
            "batched": lambda: run_batched(argparse.Namespace(**dict(vars(args), steps=1, warmup=1))),
            "serving": lambda: run_serving(args),
            "precision": lambda: run_precision(argparse.Namespace(**dict(vars(args), steps=3, warmup=2))),
            "doubleslit": lambda: run_doubleslit(argparse.Namespace(**dict(vars(args), steps=3, warmup=1))),
            "aperture3d": lambda: run_aperture3d(argparse.Namespace(**dict(vars(args), steps=2, warmup=1)))}
    out = {}
    for name in [x for x in args.extras.split(",") if x]:
        t0 = time.perf_counter()
        try:
            out[name] = legs[name]()
        except Exception as e:  # a failing leg must not lose the headline line
            out[name] = {"error": repr(e)[:400]}
        out[name]["leg_wall_s"] = round(time.perf_counter() - t0, 2)
    return out


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
        return
    legs = {"batched": lambda: run_batched(args),
            "serving": lambda: run_serving(args, [args.rate] + [float(r) for r in args.rates.split(",")
                                                              if r and float(r) != args.rate]),
            "precision": lambda: run_precision(args), "doubleslit": lambda: run_doubleslit(args),
            "aperture3d": lambda: run_aperture3d(args),
            "hero": lambda: run_hero(args), "aniso": lambda: run_aniso(args),
            "dielectric": lambda: run_dielectric(args)}
    if args.workload in legs:
        print(json.dumps(legs[args.workload]()))
        return
    world, rank, local = dist_setup()
    import numpy as np
    import torch
    assert torch.cuda.is_available(), "bench.py needs a CUDA device"
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", init_method="env://")
    import paper_2303_15762_gb300 as gr
    gr.load()
    scene, view = workload(args, rank)
    samples = view["width"] * view["height"] * view["spp"]
    flags = gr.FLAG_NEE | (gr.FLAG_WIDE_BVH if args.wide else 0)
    S = gr.Scene(scene)
    F = gr.Frame([view])
    stream = torch.cuda.current_stream()
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")  # 256 MB > 129 MB L2

    def step(profile):
        F.reset()
        gr.render([S], [view], F, seed=2, flags=flags, table_dtype=args.table, pool_size=args.pool, profile=profile)

    for _ in range(max(3, args.warmup)):
        step(False)
    torch.cuda.synchronize()
    # FP32 FMA throughput of this GPU (the traversal kernels' roofline
    # denominator), measured after warm-up and outside the timed region
    peak_tflops, peak_ms = gr.measure_fp32_peak()
    launches0 = F.stats()["kernel_launches"]
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    step_ms, kms, kcnt = [], [0.0] * 4, [0] * 4
    visits = tests = 0
    for _ in range(args.steps):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        step(True)
        e1.record(stream)
        e1.synchronize()
        step_ms.append(e0.elapsed_time(e1))
        st = F.stats()
        for k in range(4):
            kms[k] += st["kernel_ms"][k]
            kcnt[k] += st["kernel_count"][k]
        visits += st["node_visits"]
        tests += st["tri_tests"]
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    clk = clocks.stop()
    stats = F.stats()
    launches = stats["kernel_launches"] - launches0
    mean_ms = statistics.mean(step_ms)
    # the same steps as one graph launch each (no per-kernel events), after the timed region
    graph_ms = None
    if world == 1:
        def gstep():
            F.reset()
            gr.render([S], [view], F, seed=2, flags=flags, table_dtype=args.table, pool_size=args.pool, use_graph=True)
        gstep()
        graph_ms = statistics.mean([_timed(gstep, flush, stream) for _ in range(max(1, min(args.steps, 5)))])
    t_max = reduce_max(mean_ms, world)
    value = job_throughput(samples, t_max, world)
    img = F.readback(0)

    # ---- CPU oracle baseline on a centre crop, the accuracy of this run there,
    # and the traversal work per closest-hit query of the oracle's SAH tree
    cpu = None
    rel = elem = None
    ref_work = None
    if rank == 0 and not args.no_cpu_baseline:
        from oracle import oracle as orc
        c = min(args.cpu_crop, args.size)
        x0 = args.size // 2 - c // 2
        O = orc.Scene(scene)
        cores = os.cpu_count() or 1
        orc.work_reset()
        t0 = time.perf_counter()
        ref = O.render(view, 2, orc.FLAG_NEE, crop=(x0, x0, x0 + c, x0 + c), n_threads=cores)
        dt = time.perf_counter() - t0
        ref_work = orc.work_counters()
        cpu = {"value": c * c * view["spp"] / dt / 1e6, "unit": UNIT, "cores": cores, "kind": "oracle",
               "sample": "%dx%d centre crop of the same view, %d spp (%d samples), %.1f s" % (
                   c, c, view["spp"], c * c * view["spp"], dt)}
        crop = img[x0:x0 + c, x0:x0 + c].astype(np.float64)
        rel = float(np.linalg.norm(crop - ref) / max(np.linalg.norm(ref), 1e-300))
        elem = float(np.max(np.abs(crop - ref)) / max(np.max(np.abs(ref)), 1e-300))

    # ---- roofline of the dominant kernel (device time share from live events)
    dom = int(np.argmax(kms))
    per_launch_ms = kms[dom] / max(1, kcnt[dom])
    if dom in (1, 3):
        # traversal kernels, ALU/latency-bound.  Work = closest-hit queries of
        # this step (segments + next-event rays) x the FLOPs a query needs
        # through the oracle's binned-SAH reference tree (its node visits and
        # triangle tests per query, counted on the oracle's crop), so that the
        # work does not depend on the GPU's own tree; the kernels' own counts
        # are reported beside it.
        per_node = FLOP_PER_WNODE if args.wide else FLOP_PER_NODE
        trav_ms = (kms[1] + kms[3]) / args.steps
        queries = (stats["segments"] + stats["shadow_rays"])
        flops_kernel = (visits * per_node + tests * FLOP_PER_TRI) / args.steps
        achieved_kernel = flops_kernel / (trav_ms * 1e-3) / 1e12
        if ref_work and ref_work["queries"] > 0:
            vq = ref_work["node_visits"] / ref_work["queries"]
            tq = ref_work["tri_tests"] / ref_work["queries"]
            flops = queries * (vq * FLOP_PER_NODE + tq * FLOP_PER_TRI)
            basis = ("closest-hit queries per step (%d segments + next-event rays) x (%.2f node visits x %d + %.2f "
                     "triangle tests x %d FLOP) per query of the oracle's binned-SAH binary tree (ordered traversal, "
                     "counted over its %d queries on the centre crop)" % (queries, vq, FLOP_PER_NODE, tq, FLOP_PER_TRI,
                                                                         ref_work["queries"]))
        else:
            flops = flops_kernel
            basis = "the kernels' own node visits and triangle tests (no oracle run)"
        achieved = flops / (trav_ms * 1e-3) / 1e12
        roof = {"bound": "alu", "kernel": KERNELS[dom] + "+k_shadow" if dom == 1 else KERNELS[dom],
                "achieved": achieved, "peak": peak_tflops, "unit": "TFLOP/s",
                "frac": achieved / peak_tflops, "work_basis": basis,
                "achieved_kernel_counts": achieved_kernel,
                "kernel_counts": "%.2f node visits and %.2f triangle tests per query in the GPU's PLOC tree" % (
                    visits / args.steps / max(queries, 1), tests / args.steps / max(queries, 1)),
                "peak_source": "measured: FP32 FMA-chain microbenchmark, gr_measure_fp32_peak (best of 3, %.2f ms); "
                               "nominal 152 SM x 128 lanes x 2 FLOP x 2070 MHz = %.1f" % (peak_ms, FP32_PEAK_TFLOPS),
                "traffic": None, "per_launch_ms": per_launch_ms}
        tpr = NCU_TRAFFIC_PER_RAY.get((KERNELS[dom], source_hash()))
        if tpr is not None:
            rays_per_launch = stats["segments"] / max(1, stats["iterations"])
            roof["traffic"] = tpr * rays_per_launch
            roof["traffic_note"] = "ncu DRAM bytes per ray of a full-queue k_trace launch x rays per launch"
    else:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))) if os.path.exists(
            os.path.join(ROOT, "MEASURED_PEAKS.json")) else {"hbm_gbs": 6800.0}
        roof = {"bound": "hbm", "kernel": KERNELS[dom], "achieved": None, "peak": peaks.get("hbm_gbs", 6800.0),
                "unit": "GB/s", "frac": None, "traffic": None,
                "per_launch_ms": per_launch_ms, "note": "bytes per launch not yet derived"}
    roof["kernel_ms_share"] = {KERNELS[k]: kms[k] / max(sum(kms), 1e-9) for k in range(4)}

    # ---- end to end through the C ABI with pinned host buffers
    e2e = None
    if rank == 0 and args.e2e_steps > 0:
        pinned = {}
        for key in ("verts", "tri_mat", "mats", "lights"):
            a = np.ascontiguousarray(scene[key])
            t = torch.from_numpy(a.copy()).pin_memory()
            pinned[key] = t.numpy()
        h2d = sum(pinned[k].nbytes for k in pinned) + 100  # + one view descriptor
        host_img = torch.empty(img.size, dtype=torch.float32).pin_memory().numpy().reshape(img.shape)
        d2h = host_img.nbytes
        times = []
        for i in range(args.e2e_steps + 1):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            s2 = gr.Scene(pinned)
            f2 = gr.Frame([view])
            gr.render([s2], [view], f2, seed=2, flags=flags, table_dtype=args.table, pool_size=args.pool)
            _lib = gr.lib_handle()
            from paper_2303_15762_gb300 import _native as nat
            nat._check(_lib.gr_readback(f2.handle, 0, host_img.ctypes.data_as(nat.ctypes.c_void_p),
                                        host_img.nbytes, 0, nat.current_stream()))
            f2.close()
            s2.close()
            torch.cuda.synchronize()
            if i > 0:
                times.append(time.perf_counter() - t0)
        e2e_ms = 1e3 * statistics.mean(times)
        # the same calls once more with a synchronisation between phases, so
        # that scene build and readback are timed on their own
        ph = {"scene_upload_build_ms": [], "frame_alloc_render_ms": [], "readback_ms": []}
        for i in range(2):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            s2 = gr.Scene(pinned)
            torch.cuda.synchronize()
            t1 = time.perf_counter()
            f2 = gr.Frame([view])
            gr.render([s2], [view], f2, seed=2, flags=flags, table_dtype=args.table, pool_size=args.pool)
            torch.cuda.synchronize()
            t2 = time.perf_counter()
            nat._check(_lib.gr_readback(f2.handle, 0, host_img.ctypes.data_as(nat.ctypes.c_void_p),
                                        host_img.nbytes, 0, nat.current_stream()))
            torch.cuda.synchronize()
            t3 = time.perf_counter()
            f2.close()
            s2.close()
            ph["scene_upload_build_ms"].append(1e3 * (t1 - t0))
            ph["frame_alloc_render_ms"].append(1e3 * (t2 - t1))
            ph["readback_ms"].append(1e3 * (t3 - t2))
        e2e = {"value": world * samples / (e2e_ms * 1e-3) / 1e6, "unit": UNIT, "h2d_bytes_per_step": int(h2d),
               "d2h_bytes_per_step": int(d2h), "ms_per_step": e2e_ms,
               "includes": "scene upload + BVH build, frame alloc, render, readback to pinned host",
               "phases": {k: statistics.mean(v) for k, v in ph.items()}}

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": mean_ms, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": {"workload": workload_name(args, scene), "tables": args.table,
                           "parallelism": "replicas x%d" % world,
                           "l2": "flushed before every timed step (256 MB write)",
                           "pool": "library default (one slot per ticket)" if not args.pool else args.pool,
                           "step_ms_p50": float(np.percentile(step_ms, 50)),
                           "step_ms_p99": float(np.percentile(step_ms, 99))},
                "rel_l2_vs_oracle": rel, "max_elem_err_over_max_vs_oracle": elem,
                "oracle_crop": "%dx%d centre crop" % (min(args.cpu_crop, args.size), min(args.cpu_crop, args.size)),
                "graph_value": samples / (graph_ms * 1e-3) / 1e6 if graph_ms else None,
                "graph_value_note": "the same render as one CUDA graph launch per step (CUDA events, L2 flushed), "
                                    "timed after the timed region",
                "roofline": roof, "cpu_baseline": cpu, "e2e": e2e,
                "gpu_launches": int(launches), "clocks": clk,
                "stats": {"iterations_per_step": stats["iterations"], "segments": stats["segments"],
                          "shadow_rays": stats["shadow_rays"], "refine64_hits": stats["refine64_hits"],
                          "refine64_lobes": stats["refine64_lobes"],
                          "node_visits_per_step": visits / args.steps, "tri_tests_per_step": tests / args.steps}}
        if world == 1 and not args.no_extras:
            line["extras"] = run_extras(args)
        print(json.dumps(line))
    if world > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
