"""Many frames on one GPU: batched frames and a continuously batched serving loop.

Every frame slot owns one reconstruction context (its grids, FFT workspaces,
brick tables and mesh stay resident in HBM), one CUDA stream, device staging
buffers for the frame's points and RGB-D views, and device texture outputs.
A submitted frame is copied in from pinned host memory and queued on the
slot's stream as per-camera point ingests (or, for RGB-D frames, the raw
reconstruction of the depth maps on the device) followed by one CUDA-graph
replay of the whole reconstruction (``ftr_frame_launch``); frames on
different slots run concurrently on the device.  Nothing here does reconstruction arithmetic:
it only moves buffers and orders calls into the C ABI.

* ``run_batch``: B frames of mixed grid sizes, one slot each, all submitted at
  once; throughput against the same frames one after another.  Each slot's
  FFT tile plan is autotuned for its grid size when the slot is created
  (``ftr_autotune``, cached per grid, so only the first slot of a size pays).
* ``Server``: live sessions (each a camera rig with a grid size) are admitted
  while their device memory fits an HBM budget; frames arrive per session as
  a Poisson process; a frame is dispatched as soon as its session's slot is
  free, so frames that arrive while others are on the GPU join the work in
  flight (continuous batching); per-frame latency = completion - arrival.
"""

import gc
import time
from dataclasses import dataclass, field

import numpy as np

from . import ftr


def _torch():
    import torch
    if not torch.cuda.is_available():
        raise RuntimeError("the serving runtime needs a CUDA device")
    return torch


@dataclass
class FrameInput:
    """One frame in pinned host memory: oriented points with their views, or
    (rgbd) only the RGB-D images, whose points, normals and confidence maps
    the device computes (Sec. III-A, ftr_splat_depth_async)."""
    points: object
    normals: object
    weights: object
    per_camera: list
    views: list          # dicts: depth, conf, rgb (pinned tensors), K, world_to_cam, K_rgb, world_to_rgb
    n_points: int = 0
    rgbd: bool = False

    @classmethod
    def from_frame(cls, fr, rgbd=False):
        torch = _torch()

        def pin(a):
            return torch.from_numpy(np.ascontiguousarray(a)).pin_memory()
        views = []
        for v in fr["views"]:
            d = {k: v[k] for k in ("K", "world_to_cam", "K_rgb", "world_to_rgb")}
            d["depth"], d["rgb"] = pin(v["depth"]), pin(v["rgb"])
            d["conf"] = None if rgbd else pin(v["conf"])
            views.append(d)
        if rgbd:
            return cls(None, None, None, [], views, 0, True)
        return cls(pin(fr["points"]), pin(fr["normals"]), pin(fr["weights"]), list(fr["per_camera"]), views,
                   int(len(fr["points"])))

    def h2d_bytes(self):
        b = 0 if self.rgbd else 4 * (self.points.numel() + self.normals.numel() + self.weights.numel())
        for v in self.views:
            b += 4 * v["depth"].numel() + v["rgb"].numel() + (0 if self.rgbd else 4 * v["conf"].numel())
        return b


class Slot:
    """A resident context with its stream, staging buffers and texture outputs."""

    def __init__(self, grid_n, bbox, template, point_cap, mesh_cap=None, device=0):
        torch = _torch()
        self.torch = torch
        self.dev = torch.device("cuda", device)
        self.grid_n = tuple(grid_n)
        self.bbox = tuple(bbox)
        self.stream = torch.cuda.Stream(device=self.dev)
        self.ctx = ftr.Context(grid_n, bbox, stream=self.stream.cuda_stream)
        self.ctx.autotune()           # tile plans: timed once per grid size, then cached
        self.point_cap = int(point_cap)
        self.rgbd = template.rgbd
        z = dict(dtype=torch.float32, device=self.dev)
        self.P = torch.empty((max(1, self.point_cap), 3), **z)
        self.N = torch.empty((max(1, self.point_cap), 3), **z)
        self.W = torch.empty((max(1, self.point_cap),), **z)
        self.views = []
        for v in template.views:
            d = {k: v[k] for k in ("K", "world_to_cam", "K_rgb", "world_to_rgb")}
            d["depth"] = torch.empty_like(v["depth"], device=self.dev)
            d["conf"] = torch.empty(tuple(v["depth"].shape), **z)   # rgbd: written by the raw stage
            d["rgb"] = torch.empty_like(v["rgb"], device=self.dev)
            self.views.append(d)
        K = len(self.views)
        nx, ny, nz = self.grid_n
        self.cap = int(mesh_cap or max(1 << 16, (nx * ny * nz) // 64))
        self.out_w = torch.empty((self.cap, K), **z)
        self.out_uv = torch.empty((self.cap, K, 2), **z)
        self.out_rgb = torch.empty((self.cap, 3), dtype=torch.uint8, device=self.dev)
        self.out_tex = torch.empty((self.cap,), dtype=torch.uint8, device=self.dev)
        self.done = torch.cuda.Event()
        self.fetched = torch.cuda.Event()
        self.nv = self.nt = 0
        self.busy = False
        self.tag = None
        tol_h = max((bbox[3 + a] - bbox[a]) / grid_n[a] for a in range(3))
        self.tol = float(np.float32(max(3.0 * tol_h, 0.02)))

    def device_bytes(self):
        t = self.torch
        staged = sum(x.numel() * x.element_size() for x in (self.P, self.N, self.W, self.out_w, self.out_uv,
                                                               self.out_rgb, self.out_tex))
        for v in self.views:
            staged += sum(v[k].numel() * v[k].element_size() for k in ("depth", "conf", "rgb"))
        del t
        return ftr.ftr_device_bytes(self.ctx.h) + staged

    def submit(self, fin, tag=None):
        """Queue one frame (copies in, ingests, graph replay); returns immediately."""
        if fin.n_points > self.point_cap:
            raise ValueError("frame has more points than the slot holds")
        if fin.rgbd != self.rgbd or len(fin.views) != len(self.views) or any(
                tuple(v["depth"].shape) != tuple(d["depth"].shape) or tuple(v["rgb"].shape) != tuple(d["rgb"].shape)
                for d, v in zip(self.views, fin.views)):
            raise ValueError("frame does not match the slot's cameras")
        torch = self.torch
        n = fin.n_points
        with torch.cuda.stream(self.stream):
            if not fin.rgbd:
                self.P[:n].copy_(fin.points, non_blocking=True)
                self.N[:n].copy_(fin.normals, non_blocking=True)
                self.W[:n].copy_(fin.weights, non_blocking=True)
            for d, v in zip(self.views, fin.views):
                for k in ("K", "world_to_cam", "K_rgb", "world_to_rgb"):
                    d[k] = v[k]          # the frame's calibration (updated in the frame graph)
                d["depth"].copy_(v["depth"], non_blocking=True)
                if not fin.rgbd:
                    d["conf"].copy_(v["conf"], non_blocking=True)
                d["rgb"].copy_(v["rgb"], non_blocking=True)
            self.ctx.reset()
            if fin.rgbd:
                # points, normals and the confidence maps from the depth maps, on the device
                ftr.ftr_splat_depth(self.ctx.h, self.views, conf_out=[d["conf"] for d in self.views], wait=False)
            if fin.per_camera:        # every camera's points in one ingest launch
                ftr.ftr_splat_sets(self.ctx.h, [(self.P[s:s + c], self.N[s:s + c], self.W[s:s + c])
                                                for (s, c) in fin.per_camera])
            ftr.ftr_frame_launch(self.ctx.h, self.views, self.tol, self.out_w, self.out_uv, self.out_rgb,
                                 self.out_tex, self.cap)
            self.done.record(self.stream)
        self.busy = True
        self.tag = tag

    def ready(self):
        return self.done.query()

    def finish(self):
        """Complete the frame; returns (n_vertices, n_tris)."""
        m = ftr.ftr_frame_finish(self.ctx.h)
        self.busy = False
        self.nv, self.nt = int(m.n_vertices), int(m.n_tris)
        return self.nv, self.nt

    def host_buffers(self):
        """Page-locked host buffers for ``fetch_async`` at this slot's capacity."""
        torch = self.torch
        K = len(self.views)

        def pin(shape, dtype):
            return torch.empty(shape, dtype=dtype).pin_memory()
        return {"vertices": pin((self.cap, 3), torch.float32), "normals": pin((self.cap, 3), torch.float32),
                "tris": pin((2 * self.cap, 3), torch.int32), "weights": pin((self.cap, K), torch.float32),
                "uv": pin((self.cap, K, 2), torch.float32), "rgb": pin((self.cap, 3), torch.uint8),
                "textured": pin((self.cap,), torch.uint8)}

    def fetch_async(self, host):
        """Enqueue, on the slot's stream, the copies of the last finished
        frame's mesh and texture data into ``host`` (``host_buffers()``); they
        are done when ``self.fetched`` has completed.  Returns the bytes."""
        nv, nt = self.nv, self.nt
        if nv > host["vertices"].shape[0] or nt > host["tris"].shape[0] or nv > self.cap:
            raise ValueError("host buffers smaller than the frame's mesh")
        torch = self.torch
        ftr.ftr_mesh_copy_async(self.ctx.h, host["vertices"], host["normals"], host["tris"])
        with torch.cuda.stream(self.stream):
            for key, src in (("weights", self.out_w), ("uv", self.out_uv), ("rgb", self.out_rgb),
                             ("textured", self.out_tex)):
                host[key][:nv].copy_(src[:nv], non_blocking=True)
            self.fetched.record(self.stream)
        K = len(self.views)
        return nv * (24 + 12 * K + 4) + nt * 12

    def mesh(self):
        m = ftr.ftr_frame_info(self.ctx.h)
        v = np.zeros((m["n_vertices"], 3), np.float32)
        t = np.zeros((m["n_tris"], 3), np.int32)
        ftr.ftr_mesh_copy(self.ctx.h, v, None, t)
        return v, t

    def results(self):
        """The last finished frame's mesh and texture data as host arrays:
        dict(vertices, tris, weights, uv, rgb, textured)."""
        v, t = self.mesh()
        nv = len(v)
        return {"vertices": v, "tris": t, "weights": self.out_w[:nv].cpu().numpy(),
                "uv": self.out_uv[:nv].cpu().numpy(), "rgb": self.out_rgb[:nv].cpu().numpy(),
                "textured": self.out_tex[:nv].cpu().numpy()}

    def close(self):
        self.ctx.close()


def run_batch(frames, grids, bboxes, sequential=False, rounds=3, results=False):
    """Reconstruct ``frames`` (FrameInput list) on one slot each, all queued at
    once (or one after another), ``rounds`` times; returns (median seconds per
    round, [(n_vertices, n_tris)]), or with ``results`` (median seconds, per
    frame ``Slot.results()`` of the last round: mesh and texture data)."""
    torch = _torch()
    slots = [Slot(g, b, f, f.n_points) for f, g, b in zip(frames, grids, bboxes)]
    # warm-up, twice: the first round sizes every slot's buffers (growing them
    # invalidates the slot's graph), the second captures the final graphs
    for _ in range(2):
        for s, f in zip(slots, frames):
            s.submit(f)
        for s in slots:
            s.finish()
    torch.cuda.synchronize()
    times, out = [], []
    gc.disable()
    for _ in range(rounds):
        t0 = time.perf_counter()
        out = []
        if sequential:
            for s, f in zip(slots, frames):
                s.submit(f)
                out.append(s.finish())
        else:
            for s, f in zip(slots, frames):
                s.submit(f)
            out = [s.finish() for s in slots]
        torch.cuda.synchronize()
        times.append(time.perf_counter() - t0)
    gc.enable()
    if results:
        out = [s.results() for s in slots]
    for s in slots:
        s.close()
    return float(np.median(times)), out


@dataclass
class Session:
    """A live capture rig: grid, bbox and a cycle of frames (continuous motion).

    ``start_s`` / ``stop_s``: when the session joins and leaves the serving
    loop (seconds after its start; ``stop_s`` None = until the end);
    ``n_slots``: resident slots of the session, so that up to that many of
    its frames can be on the device at once."""
    sid: int
    grid_n: tuple
    bbox: tuple
    frames: list
    rate_hz: float = 30.0
    slot: object = None
    queue: list = field(default_factory=list)
    start_s: float = 0.0
    stop_s: object = None
    n_slots: int = 1
    slots: list = field(default_factory=list)
    nbytes: int = 0


def slot_estimate_bytes(sess):
    """Device bytes a session's slots will hold, from its grid, frames and
    cameras alone (nothing is allocated): the library's estimate of a
    context at the largest frame's point count and the mesh capacity, plus
    the slot's staging and texture outputs."""
    nx, ny, nz = sess.grid_n
    pts = max(int(f.n_points) for f in sess.frames)
    t = sess.frames[0]
    pixels = sum(int(v["depth"].numel()) for v in t.views)
    rgb = sum(int(v["rgb"].numel()) for v in t.views)
    cap = max(1 << 16, (nx * ny * nz) // 64)
    K = len(t.views)
    ctx = ftr.ftr_estimate_bytes(sess.grid_n, pts, pixels if t.rgbd else 0, cap, 2 * cap)
    staged = 28 * max(1, pts) + 8 * pixels + rgb + cap * (12 * K + 4)
    return sess.n_slots * (ctx + staged)


class Server:
    """Continuous-batching request loop over resident per-session slots.

    Sessions join and leave while the loop runs: a session is admitted when
    its device memory fits the HBM budget (checked on an estimate before
    anything is allocated, then on the slots' real size after they have run
    each of the session's frames once); one that does not fit waits and is
    admitted when a departing session has freed enough.  A frame is
    dispatched as soon as one of its session's slots is free, so frames that
    arrive while others are on the GPU join the work in flight."""

    def __init__(self, hbm_budget_bytes, slot_factory=None, sync=None, estimate=None):
        """``slot_factory(session)`` makes one of a session's slots (default:
        a resident ``Slot``); ``estimate(session)`` its bytes before any
        allocation (default ``slot_estimate_bytes``); ``sync()`` waits for
        the device (default ``torch.cuda.synchronize``).  They exist so that
        the scheduling can be exercised without a device."""
        self.budget = int(hbm_budget_bytes)
        self.used = 0
        self.sessions = []
        self.rejected = []
        self.waiting = []
        self.events = []
        self.slot_factory = slot_factory or (
            lambda sess: Slot(sess.grid_n, sess.bbox, sess.frames[0], max(f.n_points for f in sess.frames)))
        self.estimate = estimate or slot_estimate_bytes
        self.sync = sync

    def admit(self, sess):
        """Make the session's slots if they fit the budget; False if not."""
        if self.used + self.estimate(sess) > self.budget:
            self.rejected.append(sess.sid)
            return False
        slots = [self.slot_factory(sess) for _ in range(max(1, sess.n_slots))]
        # every frame once per slot: the buffers reach their final size (and
        # the frame graphs are captured) before the memory is counted
        for sl in slots:
            for f in sess.frames:
                sl.submit(f)
                sl.finish()
        need = sum(sl.device_bytes() for sl in slots)
        if self.used + need > self.budget:
            for sl in slots:
                sl.close()
            self.rejected.append(sess.sid)
            return False
        self.used += need
        sess.nbytes = need
        sess.slots = slots
        sess.slot = slots[0]
        self.sessions.append(sess)
        return True

    def _depart(self, sess):
        for sl in sess.slots:
            sl.close()
        self.used -= sess.nbytes
        sess.nbytes = 0
        sess.slots = []
        sess.slot = None
        self.sessions.remove(sess)

    def run(self, duration_s, seed=0, saturate=False, keep_meshes=None, late=()):
        """Serve the admitted sessions, and the ``late`` ones from their
        ``start_s``, for ``duration_s`` seconds of arrivals (Poisson, rate_hz
        each, within [start_s, stop_s); ``saturate`` makes every frame of the
        admitted sessions available at t = 0).  Returns latency and
        throughput statistics, overall and per grid size."""
        sync = self.sync or _torch().cuda.synchronize
        rng = np.random.default_rng(seed)
        everyone = list(self.sessions) + [s for s in late if s not in self.sessions]
        arrivals = []
        for s in everyone:
            t = 0.0 if saturate else float(s.start_s)
            end = duration_s if s.stop_s is None else min(duration_s, float(s.stop_s))
            k = 0
            while True:
                t += 0.0 if saturate else rng.exponential(1.0 / s.rate_hz)
                if (not saturate and t > end) or (saturate and k >= int(duration_s * s.rate_hz)):
                    break
                arrivals.append((t, s.sid, k))
                k += 1
        arrivals.sort()
        by_id = {s.sid: s for s in everyone}
        # warm-up of the admitted sessions: every frame on every slot, twice
        # (the first pass sizes the buffers, which frees memory and waits for
        # the whole device, and invalidates the frame graphs; the second
        # captures the final graphs before arrivals start)
        for _ in range(2):
            for s in self.sessions:
                for sl in s.slots:
                    for f in s.frames:
                        sl.submit(f)
                        sl.finish()
        sync()
        pending_join = sorted((s for s in everyone if s not in self.sessions), key=lambda s: s.start_s)
        self.events = []
        lat, qwait, grid_of, done_frames, meshes = [], [], [], 0, {}
        host_submit, host_finish, worst = [], [], []
        dropped = 0
        nxt = 0
        pending = len(arrivals)
        gc.disable()                  # no collector pauses inside the loop
        t0 = time.perf_counter()
        while pending:
            now = time.perf_counter() - t0
            # joins: admitted now if the budget allows, else they wait for a departure
            while pending_join and pending_join[0].start_s <= now:
                s = pending_join.pop(0)
                ta = time.perf_counter()
                ok = self.admit(s)
                self.events.append(("join", s.sid, round(now, 4), ok, round(1e3 * (time.perf_counter() - ta), 2)))
                if not ok:
                    self.waiting.append(s)
            while nxt < len(arrivals) and arrivals[nxt][0] <= now:
                ta, sid, k = arrivals[nxt]
                by_id[sid].queue.append((ta, k))
                nxt += 1
            for s in list(self.sessions):
                for sl in s.slots:
                    if sl.busy and sl.ready():
                        tf = time.perf_counter()
                        nv, nt = sl.finish()
                        host_finish.append(time.perf_counter() - tf)
                        ta, td, k = sl.tag
                        t_end = time.perf_counter() - t0
                        lat.append(t_end - ta)
                        qwait.append(td - ta)
                        grid_of.append(s.grid_n[0])
                        worst.append((t_end - ta, s.sid, k, round(1e3 * ta, 3), round(1e3 * (td - ta), 3),
                                      round(1e3 * (t_end - td), 3)))
                        done_frames += 1
                        pending -= 1
                        if keep_meshes is not None and (s.sid, k) in keep_meshes:
                            meshes[(s.sid, k)] = sl.mesh()
                    if not sl.busy and s.queue:
                        ta, k = s.queue.pop(0)
                        ts = time.perf_counter()
                        sl.submit(s.frames[k % len(s.frames)], tag=(ta, ts - t0, k))
                        host_submit.append(time.perf_counter() - ts)
                # departure: past stop_s with nothing queued or in flight
                if (s.stop_s is not None and now >= s.stop_s and not s.queue
                        and not any(sl.busy for sl in s.slots)):
                    self._depart(s)
                    self.events.append(("leave", s.sid, round(now, 4)))
                    for w in list(self.waiting):
                        if self.admit(w):
                            self.waiting.remove(w)
                            self.events.append(("join", w.sid, round(time.perf_counter() - t0, 4), True, None))
            # frames of sessions that never got in are not served
            for w in self.waiting:
                dropped += len(w.queue)
                pending -= len(w.queue)
                w.queue.clear()
        wall = time.perf_counter() - t0
        gc.enable()
        lat_ms = np.array(lat) * 1e3
        q_ms = np.array(qwait) * 1e3
        grids = np.array(grid_of)

        def pct(a, q):
            return float(np.percentile(a, q)) if len(a) else float("nan")
        per_grid = {}
        for g in sorted(set(grid_of)):
            m = grids == g
            per_grid[int(g)] = {"frames": int(m.sum()), "p50_ms": pct(lat_ms[m], 50), "p99_ms": pct(lat_ms[m], 99),
                                "max_ms": float(lat_ms[m].max())}
        return {"frames": done_frames, "seconds": wall, "frames_per_s": done_frames / wall,
                "p50_ms": pct(lat_ms, 50), "p99_ms": pct(lat_ms, 99),
                "max_ms": float(lat_ms.max()) if len(lat_ms) else float("nan"),
                "mean_ms": float(lat_ms.mean()) if len(lat_ms) else float("nan"),
                "queue_p99_ms": pct(q_ms, 99), "per_grid": per_grid,
                "host_submit_ms": {"p50": pct(np.array(host_submit) * 1e3, 50), "p99": pct(np.array(host_submit) * 1e3, 99),
                                   "max": float(np.max(host_submit) * 1e3) if host_submit else float("nan")},
                "host_finish_ms": {"p50": pct(np.array(host_finish) * 1e3, 50), "p99": pct(np.array(host_finish) * 1e3, 99),
                                   "max": float(np.max(host_finish) * 1e3) if host_finish else float("nan")},
                "slowest": [list(w[1:]) for w in sorted(worst, reverse=True)[:5]],
                "sessions": len(self.sessions), "rejected": list(self.rejected),
                "not_served": dropped, "events": list(self.events),
                "hbm_bytes": self.used, "meshes": meshes}

    def close(self):
        for s in self.sessions:
            for sl in s.slots:
                sl.close()
            s.slots = []
            s.slot = None
        self.sessions = []
