"""Progressive-render service with continuous batching.

Requests (a scene + a camera) arrive over time and each asks for a number of
progressive frames at 1 sample per pixel per frame.  The service

* admits a waiting request as soon as its resident accumulators (width x
  height x bins x Stokes x 8 bytes for sum + compensation) and its scene fit in
  the device-memory budget -- requests that arrive while others are on the GPU
  join the next device frame;
* renders one device frame for every active request in ONE launch
  (gr_render_multi: the views of all active requests share one wavefront slot
  pool, so their paths overlap on the device);
* keeps each request's accumulators resident between frames and retires the
  request, returning its mean image, when it has its frames;
* records per-request frame completion times, from which p50/p99 inter-frame
  latency and admission-to-first-frame latency are reported.

A request's image depends only on its own random stream (its view index), so
it is the same alone and in any mix.
"""
import time

import numpy as np


class Request:
    def __init__(self, rid, scene, view, frames, arrival_s=0.0):
        self.id = rid
        self.scene = scene
        self.view = dict(view, spp=1, view_index=rid)
        self.frames = frames
        self.arrival = arrival_s
        # runtime state
        self.gscene = None
        self.frame = None
        self.done = 0
        self.admitted_at = None
        self.frame_times = []
        self.image = None

    def accum_bytes(self):
        v = self.view
        return v["width"] * v["height"] * v["n_bins"] * v["n_stokes"] * 8

    def scene_bytes(self):
        return int(self.scene["verts"].nbytes * 2 + self.scene["tri_mat"].nbytes * 2 + 4096)


class ProgressiveServer:
    def __init__(self, gr, memory_budget_bytes=None, render_opts=None, clock=time.perf_counter):
        import torch
        self.gr = gr
        self.clock = clock
        if memory_budget_bytes is None:
            free, _ = torch.cuda.mem_get_info()
            memory_budget_bytes = int(free * 0.5)
        self.budget = memory_budget_bytes
        self.used = 0
        self.waiting = []
        self.active = []
        self.finished = []
        self.opts = dict(seed=1, flags=0, table_dtype="f32") if render_opts is None else dict(render_opts)
        # a permanent 1x1 view with no samples owns the slot pool, counters and
        # render graph of every device frame
        self._work_view = dict(eye=(0.0, 0.0, 1.0), look_at=(0.0, 0.0, 0.0), up=(0.0, 1.0, 0.0), vfov_deg=10.0,
                               width=1, height=1, p_pix_um=2.0, f_beta=0.5, lambda_min_um=0.5, lambda_max_um=0.5,
                               n_bins=1, n_stokes=1, max_depth=0, spp=0, first_sample=0, view_index=0,
                               scene_index=0, ortho=0, ortho_half_m=0.0)
        self._work = gr.Frame([self._work_view])
        self.samples = 0
        self.device_frames = 0

    def submit(self, req):
        self.waiting.append(req)

    def admit(self):
        """Admit waiting requests (in arrival order) while memory allows."""
        still = []
        for r in self.waiting:
            need = r.accum_bytes() + r.scene_bytes()
            if self.used + need <= self.budget:
                r.gscene = self.gr.Scene(r.scene)
                r.frame = self.gr.Frame([r.view])
                r.admitted_at = self.clock()
                self.used += need
                self.active.append(r)
            else:
                still.append(r)
        self.waiting = still

    def step(self):
        """One device frame: 1 spp for every active request, one launch."""
        if not self.active:
            return 0
        import torch
        n_stokes = self.active[0].view["n_stokes"]
        scenes = [self.active[0].gscene]
        views = [dict(self._work_view, n_stokes=n_stokes)] if n_stokes == 1 else []
        frames = [self._work] if n_stokes == 1 else []
        fview = [0] if n_stokes == 1 else []
        for i, r in enumerate(self.active):
            if i > 0:
                scenes.append(r.gscene)
            views.append(dict(r.view, first_sample=r.done, scene_index=i))
            frames.append(r.frame)
            fview.append(0)
        self.gr.render_multi(scenes, views, frames, fview, **self.opts)
        torch.cuda.current_stream().synchronize()
        now = self.clock()
        n = 0
        keep = []
        for r in self.active:
            r.done += 1
            r.frame_times.append(now)
            n += r.view["width"] * r.view["height"]
            if r.done >= r.frames:
                r.image = r.frame.readback(0)
                r.frame.close()
                r.gscene.close()
                self.used -= r.accum_bytes() + r.scene_bytes()
                self.finished.append(r)
            else:
                keep.append(r)
        self.active = keep
        self.samples += n
        self.device_frames += 1
        return n

    def close(self):
        for r in self.active:
            r.frame.close()
            r.gscene.close()
        self.active = []
        self._work.close()


def run_poisson(gr, requests, rate_hz, server, seed=0, time_limit_s=600.0):
    """Replay `requests` with Poisson arrivals of the given rate (requests
    per second) in real time; returns latency and throughput statistics."""
    rng = np.random.default_rng(seed)
    t = 0.0
    for r in requests:
        t += rng.exponential(1.0 / rate_hz)
        r.arrival = t
    pending = sorted(requests, key=lambda r: r.arrival)
    t0 = server.clock()
    busy = 0.0
    while (pending or server.waiting or server.active) and server.clock() - t0 < time_limit_s:
        now = server.clock() - t0
        while pending and pending[0].arrival <= now:
            server.submit(pending.pop(0))
        server.admit()
        if server.active:
            s = server.clock()
            server.step()
            busy += server.clock() - s
        elif pending:
            time.sleep(max(0.0, min(0.01, pending[0].arrival - (server.clock() - t0))))
    wall = server.clock() - t0
    inter, first = [], []
    for r in server.finished:
        first.append(r.frame_times[0] - r.admitted_at)
        inter += list(np.diff(r.frame_times))
    q = lambda a, p: float(np.percentile(a, p)) * 1e3 if len(a) else None  # noqa: E731
    return {"requests": len(server.finished), "device_frames": server.device_frames,
            "samples": server.samples, "wall_s": wall, "busy_s": busy,
            "msamples_per_s": server.samples / max(busy, 1e-9) / 1e6,
            "p50_frame_ms": q(inter, 50), "p99_frame_ms": q(inter, 99),
            "p50_first_frame_ms": q(first, 50), "p99_first_frame_ms": q(first, 99)}
