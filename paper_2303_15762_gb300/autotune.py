"""Autotuner for the wavefront render's launch parameters.

Coordinate descent over the slot-pool size, the block size, the
regeneration threshold and the order-table precision on a reduced-sample probe
of the actual workload (the same scenes and views, fewer samples per pixel),
timed with CUDA events on the render stream.  The result is a dict of
gr_render options.  Pool sizes are tried as fractions of the probe's tickets
(one ticket = a pixel's samples in one wavelength bin) and the winning
fraction is applied to the full workload's tickets: the probe has fewer
tickets than the render it stands for, so an absolute pool size would not
transfer.  Table precision is a tuning choice because a narrower
table widens the window around a CDF boundary inside which a grating order is
re-decided in FP64, and FP64 throughput is low on this part: FP16 tables trade
shared-memory footprint for roughly ten times as many FP64 re-decisions.
"""
import math
import statistics

POOL_FRACTIONS = (1 / 128, 1 / 64, 1 / 32, 1 / 16, 1 / 8, 1 / 4)
POOL_MIN, POOL_MAX = 1 << 18, 1 << 26  # 2^26 slots = 16 GB of slot state
BLOCKS = (128, 256)
THRESHOLDS = (0, 25, 50, 75)
TABLES = ("f32", "f16")


def _time_render(gr, scenes, views, frame, opts, repeats=2):
    import torch
    stream = torch.cuda.current_stream()
    times = []
    for r in range(repeats + 1):
        frame.reset()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        gr.render(scenes, views, frame, **opts)
        e1.record(stream)
        e1.synchronize()
        if r > 0:  # the first run builds and caches the render graph
            times.append(e0.elapsed_time(e1))
    return statistics.median(times)


def tickets(views):
    """Tickets of a view set: pixels x the bins that receive samples."""
    return sum(v["width"] * v["height"] * min(v["spp"], v["n_bins"]) for v in views)


def pool_for(fraction, n_tickets):
    """A power-of-two pool of about fraction x n_tickets slots, clamped."""
    p = 1 << max(0, int(round(math.log2(max(1.0, fraction * n_tickets)))))
    return int(min(POOL_MAX, max(POOL_MIN, p)))


def autotune(gr, scenes, views, base_opts, probe_spp=None, pool_fractions=POOL_FRACTIONS, blocks=BLOCKS,
             thresholds=THRESHOLDS, tables=TABLES, log=None):
    """Return (best_opts, trials).  base_opts are fixed options (seed, flags,
    use_graph; table_dtype is the starting point of its coordinate);
    probe_spp reduces every view's samples.  The returned pool_size is the
    winning fraction of the probe's tickets applied to the full views'."""
    probe = [dict(v, spp=probe_spp if probe_spp else v["spp"]) for v in views]
    frame = gr.Frame(probe)
    trials = []
    n_probe, n_full = tickets(probe), tickets(views)
    pools = sorted({pool_for(f, n_probe) for f in pool_fractions})
    best = dict(base_opts, pool_size=pool_for(1 / 16, n_probe), block=256, regen_threshold_pct=0)
    best.setdefault("table_dtype", "f32")

    def run(cand):
        ms = _time_render(gr, scenes, probe, frame, cand)
        trials.append((dict(pool_size=cand["pool_size"], block=cand["block"],
                            regen_threshold_pct=cand["regen_threshold_pct"], table_dtype=cand["table_dtype"]), ms))
        if log:
            log("autotune pool=%d block=%d thr=%d table=%s: %.2f ms" % (
                cand["pool_size"], cand["block"], cand["regen_threshold_pct"], cand["table_dtype"], ms))
        return ms

    best_ms = run(best)
    for key, values in (("pool_size", pools), ("block", blocks), ("regen_threshold_pct", thresholds),
                        ("table_dtype", tables)):
        for v in values:
            if v == best[key]:
                continue
            cand = dict(best, **{key: v})
            ms = run(cand)
            if ms < best_ms:
                best, best_ms = cand, ms
    frame.close()
    best = dict(best, pool_size=pool_for(best["pool_size"] / max(1, n_probe), n_full))
    return best, trials
