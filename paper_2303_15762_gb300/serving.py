"""Progressive-render service with continuous batching.

Requests (a scene + a camera) arrive over time and each asks for a number of
progressive frames at 1 sample per pixel per frame.  The service

* prepares arriving requests on a host thread of their own, on a CUDA stream
  of their own: the scene upload and BVH build and the creation of the
  request's resident accumulators run while the device renders the active
  requests' frames, so an arrival does not stall them;
* admits a request only while the device memory it accounts for stays within
  the budget.  The accounting is the library's: a scene's and a frame's
  device bytes (gr_scene_bytes, gr_frame_bytes), and the shared wavefront
  scratch of every device frame (gr_render_scratch_bytes; the slot pool is
  sized explicitly, one slot per ticket of the active requests up to a cap, so
  a request's share of it is known before it joins).  Before a scene exists
  its size is bounded from its triangle, material and light counts; the bound
  is replaced by the actual size once the scene is built;
* renders one device frame for the active requests in ONE launch per Stokes
  count (gr_render_multi: the views of all active requests share one
  wavefront slot pool, so their paths overlap on the device; requests with 1
  and with 4 Stokes components form two groups, each with its own pool);
* keeps each request's accumulators resident between frames and retires the
  request, returning its mean image, when it has its frames;
* records per-request frame completion times, from which p50/p99 inter-frame
  latency and arrival- and admission-to-first-frame latency are reported,
  with throughput over wall-clock time and over device-busy time.

A request's image depends only on its own random stream (its view index), so
it is the same alone and in any mix.
"""
import collections
import threading
import time

import numpy as np

# device bytes per slot of the wavefront pool (the render's slot state, queues
# and state byte), and an allowance for the view and order-table descriptors
SLOT_BYTES = 265
DESCRIPTOR_ALLOWANCE = 1 << 20


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
        self.arrived_at = None
        self.admitted_at = None
        self.frame_times = []
        self.image = None
        self.held = 0          # device bytes accounted to this request

    def accum_bytes(self):
        v = self.view
        return v["width"] * v["height"] * v["n_bins"] * v["n_stokes"] * 8

    def tickets(self):
        """Wavefront tickets of one progressive frame (1 sample per pixel)."""
        return self.view["width"] * self.view["height"]

    def scene_bytes_bound(self):
        """Upper bound of gr_scene_bytes for this scene: per triangle its
        vertices (48 B), material (4), binary nodes (64 + 32 in FP16), 4-wide
        nodes (64), Morton key (8) and, for emitters, a vertex copy (48); per
        material 64 + 4 B and an emitter record (96); per light 32 B; 256 B of
        alignment for each of the 13 arrays."""
        n = len(self.scene["tri_mat"])
        m = len(self.scene["mats"])
        L = len(self.scene["lights"])
        return n * (48 + 4 + 64 + 32 + 64 + 8 + 48) + m * (64 + 4 + 96) + L * 32 + 13 * 256 + 4096


class ProgressiveServer:
    def __init__(self, gr, memory_budget_bytes=None, render_opts=None, clock=time.perf_counter,
                 pool_slots_max=1 << 24):
        import torch
        self.gr = gr
        self.clock = clock
        self.device = torch.cuda.current_device()
        if memory_budget_bytes is None:
            free, _ = torch.cuda.mem_get_info()
            memory_budget_bytes = int(free * 0.5)
        self.budget = memory_budget_bytes
        self.pool_slots_max = int(pool_slots_max)
        self.opts = dict(seed=1, flags=0, table_dtype="f32") if render_opts is None else dict(render_opts)
        self.opts.pop("pool_size", None)
        self._lock = threading.Condition()
        self.used = 0            # accounted device bytes: requests + shared scratch
        self.peak_used = 0
        self.waiting = collections.deque()   # submitted, not yet prepared
        self.ready = []          # prepared (scene and frame built), not yet rendering
        self.active = []
        self.finished = []
        self.rejected = []       # requests that can never fit the budget
        self._building = []      # taken from `waiting`, scene and frame being built
        # a permanent 1x1 view with no samples per Stokes count owns the slot
        # pool, counters and render graph of that group's device frames
        self._work_view = dict(eye=(0.0, 0.0, 1.0), look_at=(0.0, 0.0, 0.0), up=(0.0, 1.0, 0.0), vfov_deg=10.0,
                               width=1, height=1, p_pix_um=2.0, f_beta=0.5, lambda_min_um=0.5, lambda_max_um=0.5,
                               n_bins=1, n_stokes=1, max_depth=0, spp=0, first_sample=0, view_index=0,
                               scene_index=0, ortho=0, ortho_half_m=0.0)
        self._work, self._work_base = {}, {}
        for ns in (1, 4):
            self._new_work(ns)
            self.used += self._work_base[ns]
        self._scratch = {1: 0, 4: 0}     # accounted shared scratch per group
        self.samples = 0
        self.device_frames = 0
        self._stop = False
        self._side = torch.cuda.Stream()
        self._thread = threading.Thread(target=self._prepare_loop, daemon=True)
        self._thread.start()

    def _new_work(self, ns):
        f = self.gr.Frame([dict(self._work_view, n_stokes=ns)])
        self._work[ns] = f
        self._work_base[ns] = f.device_bytes()   # accumulators and counters, no scratch yet

    def _held_scratch(self, ns):
        return self._work[ns].device_bytes() - self._work_base[ns]

    # ---------------------------------------------------------- accounting
    def _account(self, delta):
        self.used += delta
        self.peak_used = max(self.peak_used, self.used)

    def _group(self, ns):
        return [r for r in self.active + self.ready if r.view["n_stokes"] == ns]

    def _scratch_need(self, reqs):
        slots = min(self.pool_slots_max, sum(r.tickets() for r in reqs))
        return slots * SLOT_BYTES + DESCRIPTOR_ALLOWANCE if reqs else 0

    # ---------------------------------------------------------- preparation thread
    def submit(self, req):
        with self._lock:
            req.arrived_at = self.clock()
            self.waiting.append(req)
            self._lock.notify_all()

    def _prepare_loop(self):
        import ctypes
        import torch
        torch.cuda.set_device(self.device)
        side = ctypes.c_void_p(self._side.cuda_stream)
        while True:
            with self._lock:
                while not self._stop and not self._next_fits():
                    self._lock.wait(0.05)
                if self._stop:
                    return
                r = self.waiting.popleft()
                self._building.append(r)
                ns = r.view["n_stokes"]
                grow = max(0, self._scratch_need(self._group(ns) + [r]) - self._scratch[ns])
                frame_bytes = r.accum_bytes() + 256
                bound = r.scene_bytes_bound() + frame_bytes
                r.held = bound
                self._account(bound)
                self._scratch[ns] += grow
                self._account(grow)
            # build outside the lock: the device keeps rendering meanwhile
            gscene = self.gr.Scene(r.scene, stream=side)
            frame = self.gr.Frame([r.view], stream=side)
            self._side.synchronize()
            actual = gscene.device_bytes() + frame.device_bytes()
            with self._lock:
                r.gscene, r.frame = gscene, frame
                self._account(actual - r.held)
                r.held = actual
                self._building.remove(r)
                self.ready.append(r)
                self._lock.notify_all()

    def _next_fits(self):
        """Whether the first waiting request fits the budget now (requests are
        prepared in arrival order; one that can never fit is set aside)."""
        while self.waiting:
            r = self.waiting[0]
            ns = r.view["n_stokes"]
            need = r.scene_bytes_bound() + r.accum_bytes() + 256 + self._scratch_need([r])
            if need + sum(self._work_base.values()) > self.budget:
                self.rejected.append(self.waiting.popleft())
                continue
            grow = max(0, self._scratch_need(self._group(ns) + [r]) - self._scratch[ns])
            return self.used + r.scene_bytes_bound() + r.accum_bytes() + 256 + grow <= self.budget
        return False

    # ---------------------------------------------------------- device frames
    def admit(self):
        """Requests whose scene and frame are built join the next device frame."""
        with self._lock:
            now = self.clock()
            for r in self.ready:
                r.admitted_at = now
            self.active += self.ready
            self.ready = []

    def idle(self):
        with self._lock:
            return not (self.waiting or self.ready or self.active)

    def wait_prepared(self, timeout_s=60.0):
        """Block until the preparation thread has built every waiting request
        that fits the budget now (for deterministic tests)."""
        t0 = time.perf_counter()
        with self._lock:
            while self.waiting and self._next_fits() and time.perf_counter() - t0 < timeout_s:
                self._lock.wait(0.01)
            # a request popped from `waiting` may still be building
            while any(r.gscene is None for r in self._building) and time.perf_counter() - t0 < timeout_s:
                self._lock.wait(0.01)

    def step(self):
        """One device frame: 1 spp for every active request, one launch per
        Stokes count."""
        if not self.active:
            return 0
        import torch
        for ns in (1, 4):
            group = [r for r in self.active if r.view["n_stokes"] == ns]
            if not group:
                continue
            slots = min(self.pool_slots_max, sum(r.tickets() for r in group))
            scenes, views = [], [dict(self._work_view, n_stokes=ns)]
            frames, fview = [self._work[ns]], [0]
            for i, r in enumerate(group):
                scenes.append(r.gscene)
                views.append(dict(r.view, first_sample=r.done, scene_index=i))
                frames.append(r.frame)
                fview.append(0)
            self.gr.render_multi(scenes, views, frames, fview, pool_size=slots, **self.opts)
        torch.cuda.current_stream().synchronize()
        now = self.clock()
        n = 0
        keep, gone = [], []
        for r in self.active:
            r.done += 1
            r.frame_times.append(now)
            n += r.tickets()
            if r.done >= r.frames:
                r.image = r.frame.readback(0)
                gone.append(r)
            else:
                keep.append(r)
        with self._lock:
            self.active = keep
            for r in gone:
                r.frame.close()
                r.gscene.close()
                self._account(-r.held)
                r.held = 0
                self.finished.append(r)
            for ns in (1, 4):
                # the scratch a device frame left in the group's work frame is
                # accounted at least at its actual size; a group left with no
                # request releases it (a new work frame holds none)
                held = self._held_scratch(ns)
                if held > self._scratch[ns]:
                    self._account(held - self._scratch[ns])
                    self._scratch[ns] = held
                if not self._group(ns) and self._scratch[ns] > 0:
                    self._work[ns].close()
                    self._new_work(ns)
                    self._account(-self._scratch[ns])
                    self._scratch[ns] = 0
            self._lock.notify_all()
        self.samples += n
        self.device_frames += 1
        return n

    def close(self):
        with self._lock:
            self._stop = True
            self._lock.notify_all()
        self._thread.join()
        for r in self.active + self.ready:
            r.frame.close()
            r.gscene.close()
        self.active, self.ready = [], []
        for f in self._work.values():
            f.close()


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
    while (pending or not server.idle()) and server.clock() - t0 < time_limit_s:
        now = server.clock() - t0
        while pending and pending[0].arrival <= now:
            server.submit(pending.pop(0))
        server.admit()
        if server.active:
            s = server.clock()
            server.step()
            busy += server.clock() - s
        else:
            nxt = pending[0].arrival - (server.clock() - t0) if pending else 0.002
            time.sleep(max(0.0, min(0.002, nxt)))
    wall = server.clock() - t0
    inter, first_adm, first_arr = [], [], []
    for r in server.finished:
        first_adm.append(r.frame_times[0] - r.admitted_at)
        first_arr.append(r.frame_times[0] - r.arrived_at)
        inter += list(np.diff(r.frame_times))
    q = lambda a, p: float(np.percentile(a, p)) * 1e3 if len(a) else None  # noqa: E731
    return {"requests": len(server.finished), "device_frames": server.device_frames,
            "samples": server.samples, "wall_s": wall, "busy_s": busy,
            "msamples_per_s": server.samples / max(wall, 1e-9) / 1e6,
            "msamples_per_busy_s": server.samples / max(busy, 1e-9) / 1e6,
            "p50_frame_ms": q(inter, 50), "p99_frame_ms": q(inter, 99),
            "p50_first_frame_ms": q(first_adm, 50), "p99_first_frame_ms": q(first_adm, 99),
            "p50_arrival_to_first_frame_ms": q(first_arr, 50), "p99_arrival_to_first_frame_ms": q(first_arr, 99),
            "peak_accounted_bytes": server.peak_used, "budget_bytes": server.budget}
