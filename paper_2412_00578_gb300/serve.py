"""Serving loop with continuous batching over resident scenes.

Scenes stay resident on the device.  Render requests (scene, camera pose,
resolution) arrive over time.  A fixed number of execution slots, each with
its own CUDA stream and its own batch frame, run batches concurrently on the
GPU.  Whenever a slot finishes, the scheduler fills it at once with the
requests waiting at that moment:
- the oldest request's scene first;
- FIFO within a scene;
- at most ``max_batch`` requests;
- and only if the batch's buffers fit the device-memory budget.
So requests that arrive while other work is on the GPU join the next free
slot and their work overlaps with the batches in flight.  That is continuous
batching, not a drain-then-refill queue.

Every request's image is the batch renderer's output for its camera, which
equals a standalone render of that camera bit for bit (the batch path
computes each camera exactly as the single-camera path does).

``Scheduler`` holds the policy and is plain Python (tested on the CPU with a
fake executor); ``GpuExecutor`` runs batches with ``raster.BatchRenderer``.
"""
from __future__ import annotations

import collections
import statistics
import time
from dataclasses import dataclass, field
from typing import Callable


@dataclass
class Request:
    rid: int
    scene: str
    camera: object
    arrival: float                 # seconds, on the serving clock
    start: float | None = None     # when its batch was launched
    done: float | None = None      # when its result was observed complete
    result: object = None
    batch: int | None = None
    deadline: float | None = None  # seconds after arrival by which it must have started
    status: str = "pending"        # pending | done | expired | cancelled

    @property
    def latency(self) -> float:
        return self.done - self.arrival


def batch_bytes(n: int, cams, tile: int = 16, keys_per_pixel: float = 4.0) -> int:
    """Estimate of the device memory of one batch frame: per-(camera,
    Gaussian) 2D state and counts, keys at a keys-per-pixel ratio (ping-pong
    buffers), per-tile ranges and per-pixel outputs."""
    pixels = sum(c.width * c.height for c in cams)
    tiles = sum(((c.width + tile - 1) // tile) * ((c.height + tile - 1) // tile) for c in cams)
    keys = int(keys_per_pixel * pixels) + (1 << 16)
    return len(cams) * n * (48 + 4) + keys * 24 + tiles * 8 + pixels * 20


@dataclass
class Scheduler:
    """Continuous-batching policy: which waiting requests go into a free slot."""
    scene_sizes: dict                 # scene name -> Gaussian count
    max_batch: int = 16
    memory_budget: int = 1 << 34      # bytes available to in-flight batch frames
    size_fn: Callable = batch_bytes
    waiting: collections.OrderedDict = field(default_factory=collections.OrderedDict)
    in_use: int = 0                   # bytes held by in-flight batches

    def submit(self, req: Request):
        self.waiting[req.rid] = req

    def cancel(self, rid: int) -> bool:
        """Withdraw a waiting request (False if it is not waiting: already in a
        batch on the GPU, finished, or unknown)."""
        r = self.waiting.pop(rid, None)
        if r is None:
            return False
        r.status = "cancelled"
        return True

    def expire(self, now: float):
        """Drop the waiting requests whose deadline has passed at time ``now``."""
        gone = [r for r in self.waiting.values() if r.deadline is not None and now > r.arrival + r.deadline]
        for r in gone:
            del self.waiting[r.rid]
            r.status = "expired"
        return gone

    def next_batch(self):
        """Requests for one batch (same scene), or [] if nothing is admissible."""
        if not self.waiting:
            return [], 0
        oldest = next(iter(self.waiting.values()))
        scene = oldest.scene
        chosen = []
        for r in self.waiting.values():
            if r.scene != scene:
                continue
            trial = chosen + [r]
            need = self.size_fn(self.scene_sizes[scene], [q.camera for q in trial])
            if self.in_use + need > self.memory_budget:
                break
            chosen = trial
            if len(chosen) >= self.max_batch:
                break
        if not chosen:
            return [], 0
        need = self.size_fn(self.scene_sizes[scene], [q.camera for q in chosen])
        for r in chosen:
            del self.waiting[r.rid]
        self.in_use += need
        return chosen, need

    def release(self, nbytes: int):
        self.in_use -= nbytes


class GpuExecutor:
    """``slots`` concurrent batch renderers, each on its own CUDA stream."""

    def __init__(self, scenes: dict, device=None, slots: int = 3, tile: int = 16, mode: str = "accutile",
                 keep_results: bool = True):
        import torch

        from . import raster

        self.torch = torch
        self.device = torch.device(device or "cuda")
        self.scenes = scenes
        self.streams = [torch.cuda.Stream(self.device) for _ in range(slots)]
        self.renderers = []
        for s in self.streams:
            r = raster.BatchRenderer(self.device, tile=tile, mode=mode)
            r.rast.set_stream(s)
            self.renderers.append(r)
        self.busy = [None] * slots  # (requests, nbytes, event, batch id) per slot
        self.raster = raster
        # keep_results: clone each finished image for the caller (device
        # memory per request); otherwise only its completion is recorded
        self.keep_results = keep_results

    def free_slots(self):
        return [k for k, b in enumerate(self.busy) if b is None]

    def launch(self, slot: int, reqs, nbytes: int, batch_id: int):
        torch = self.torch
        r = self.renderers[slot]
        stream = self.streams[slot]
        scene = self.scenes[reqs[0].scene]
        cams = [q.camera for q in reqs]
        with torch.cuda.stream(stream):
            n = int(scene.means.shape[1])
            r.ensure(n, cams, min_keys=int(4.5 * sum(c.width * c.height for c in cams)))
            r._launch(scene, cams)
            ev = torch.cuda.Event()
            ev.record(stream)
        self.busy[slot] = (reqs, nbytes, ev, batch_id)

    def poll(self):
        """Completed (slot, requests, nbytes, batch id) tuples; results copied out."""
        torch = self.torch
        out = []
        for k, b in enumerate(self.busy):
            if b is None or not b[2].query():
                continue
            reqs, nbytes, _, bid = b
            r = self.renderers[k]
            cams = [q.camera for q in reqs]
            K, flags = r.rast.gs_batch_status(r.frame, raise_on_error=False)
            if flags & self.raster.FLAG_CAPACITY:  # rare: grow and re-run this batch on its slot
                scene = self.scenes[reqs[0].scene]
                with torch.cuda.stream(self.streams[k]):
                    r.ensure(int(scene.means.shape[1]), cams, min_keys=int(K * r.headroom) + 1)
                    r._launch(scene, cams)
                    ev = torch.cuda.Event()
                    ev.record(self.streams[k])
                self.busy[k] = (reqs, nbytes, ev, bid)
                continue
            if flags:
                r.rast.gs_batch_status(r.frame, raise_on_error=True)
            if self.keep_results:
                with torch.cuda.stream(self.streams[k]):
                    imgs = r.frame.images(cams)
                    for q, im in zip(reqs, imgs):
                        q.result = im.clone()
                self.streams[k].synchronize()
            self.busy[k] = None
            out.append((k, reqs, nbytes, bid))
        return out


def serve(requests, scheduler: Scheduler, executor, clock=time.perf_counter, idle_sleep=5e-5, cancels=()):
    """Run the request stream to completion in real time.  ``requests`` are
    sorted by arrival (seconds after start).  A request with a ``deadline``
    that has not started within it is dropped (expired); ``cancels`` lists
    (time, rid) withdrawals, honoured while the request still waits.  Returns
    the finished requests and a stats dict."""
    pending = collections.deque(sorted(requests, key=lambda r: r.arrival))
    cancel_q = collections.deque(sorted(cancels))
    finished = []
    expired, cancelled = [], []
    t0 = clock()
    batch_id = 0
    max_inflight = 0
    sizes = []
    while pending or scheduler.waiting or any(b is not None for b in executor.busy):
        now = clock() - t0
        while pending and pending[0].arrival <= now:
            scheduler.submit(pending.popleft())
        while cancel_q and cancel_q[0][0] <= now:
            rid = cancel_q.popleft()[1]
            if scheduler.cancel(rid):
                cancelled.append(rid)
        expired.extend(scheduler.expire(now))
        for k, reqs, nbytes, _ in executor.poll():
            t = clock() - t0
            for q in reqs:
                q.done = t
                q.status = "done"
            finished.extend(reqs)
            scheduler.release(nbytes)
        for slot in executor.free_slots():
            reqs, nbytes = scheduler.next_batch()
            if not reqs:
                break
            t = clock() - t0
            for q in reqs:
                q.start = t
                q.batch = batch_id
            executor.launch(slot, reqs, nbytes, batch_id)
            sizes.append(len(reqs))
            batch_id += 1
        max_inflight = max(max_inflight, sum(b is not None for b in executor.busy))
        if idle_sleep:
            time.sleep(idle_sleep)
    span = clock() - t0
    lat = sorted(q.latency for q in finished)
    stats = {
        "requests": len(finished),
        "batches": batch_id,
        "mean_batch": statistics.mean(sizes) if sizes else 0.0,
        "max_inflight_batches": max_inflight,
        "p50_ms": 1e3 * lat[len(lat) // 2] if lat else None,
        "p99_ms": 1e3 * lat[min(len(lat) - 1, int(0.99 * len(lat)))] if lat else None,
        "frames_per_s": len(finished) / span if span > 0 else None,
        "span_s": span,
        "expired": len(expired),
        "cancelled": len(cancelled),
    }
    return finished, stats


def poisson_requests(rate: float, duration: float, scenes: list, cam_fn, seed: int = 7):
    """Poisson arrivals at ``rate`` per second for ``duration`` seconds; each
    request picks a scene uniformly and a camera from ``cam_fn(gen)``."""
    import torch

    gen = torch.Generator().manual_seed(seed)
    t, rid, out = 0.0, 0, []
    while True:
        u = float(torch.rand(1, generator=gen, dtype=torch.float64))
        t += -math_log(1.0 - u) / rate
        if t > duration:
            break
        k = int(torch.randint(len(scenes), (1,), generator=gen))
        out.append(Request(rid, scenes[k], cam_fn(gen), t))
        rid += 1
    return out


def math_log(x: float) -> float:
    import math

    return math.log(max(x, 1e-300))
