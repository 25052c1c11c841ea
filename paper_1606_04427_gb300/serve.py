"""Continuous-batching render server over particle sets resident on the GPU.

Requests (set, camera) arrive at any time.  A request is admitted when a slot (a
worker thread with its own CUDA stream) is free and its device footprint fits in the
remaining HBM budget; admitted requests render concurrently on their streams, so a
request that arrives while others are on the GPU starts as soon as a slot and memory
free up.  Latency is arrival to completion; the server reports throughput and p50 / p99.

Admission is a reservation of exactly what the library will allocate, never an
estimate.  A request first reserves the count phase's workspace and its image (both
known before any GPU work), runs the count phase (splotch_frame_prepare), which reports
the exact bytes of its tile lists, and reserves those before the library allocates
them.  When they do not fit, the request releases everything and waits in the queue
with its full footprint known; the next admission reserves all of it at once.  The sum
of reservations stays within the budget, except for a request admitted with nothing
else in flight (so that the queue always drains) whose footprint alone exceeds it.

The paper's analogue is several MPI tasks sharing one coprocessor to keep it busy
(Section 3.2.1, Section 4.2.1); here the tasks are streams of one process.
"""
from __future__ import annotations

import threading
import time
from collections import deque
from dataclasses import dataclass, field
from typing import Callable, Dict, List, Optional, Sequence

import numpy as np
import torch

from . import render


@dataclass
class Completed:
    request_id: int
    set_index: int
    width: int
    height: int
    arrival: float
    start: float
    finish: float
    pairs: int
    reserved_bytes: int
    allocated_bytes: int = 0
    image: Optional[torch.Tensor] = None

    @property
    def latency(self) -> float:
        return self.finish - self.arrival


@dataclass
class _Pending:
    request_id: int
    set_index: int
    camera: object
    arrival: float
    first: int = 0           # count-phase workspace + image: known at submission
    lists: Optional[int] = None  # tile lists and split scratch, once a count phase ran
    bypassed: int = 0

    @property
    def need(self) -> int:
        return self.first + (self.lists or 0)


class _CudaDevice:
    """Streams and image buffers of the server's workers on the current CUDA device."""

    def __init__(self):
        self.index = torch.cuda.current_device()

    def bind(self):
        torch.cuda.set_device(self.index)

    def free_bytes(self) -> int:
        return torch.cuda.mem_get_info()[0]

    def stream(self):
        return torch.cuda.Stream()

    def image(self, height: int, width: int, stream):
        with torch.cuda.stream(stream):
            return torch.empty((height, width, 3), dtype=torch.float32, device="cuda")

    def synchronize(self, stream):
        stream.synchronize()


class Server:
    """``scenes``: resident :class:`render.Scene` objects.  ``slots``: concurrent
    requests (one CUDA stream each).  ``hbm_budget``: bytes the in-flight requests may
    reserve (default 80 % of the free device memory at construction).  ``device``: where
    the workers' streams and images live (the current CUDA device by default; the host
    tests of the admission logic pass a stand-in)."""

    def __init__(self, scenes: Sequence[render.Scene], slots: int = 4, hbm_budget: Optional[int] = None,
                 params: Optional[render.RenderParams] = None, keep_images: bool = False,
                 max_bypass: int = 8, device=None):
        self.scenes = list(scenes)
        self.slots = slots
        self.dev = device if device is not None else _CudaDevice()
        if hbm_budget is None:
            hbm_budget = int(0.8 * self.dev.free_bytes())
        self.budget = int(hbm_budget)
        self.params = params or render.RenderParams()
        self.keep_images = keep_images
        self.max_bypass = max_bypass
        self.reserved = 0
        self.peak_reserved = 0
        self.requeued = 0
        self.cv = threading.Condition()
        self.queue: deque = deque()
        self.done: List[Completed] = []
        self.errors: List[str] = []
        self.in_flight = 0
        self.next_id = 0
        self.stop = False
        self.t0 = time.perf_counter()
        self.streams = [self.dev.stream() for _ in range(slots)]
        self.threads = [threading.Thread(target=self._worker, args=(k,), daemon=True) for k in range(slots)]
        for t in self.threads:
            t.start()

    # ---------------------------------------------------------------------------------
    def submit(self, set_index: int, cam, arrival: Optional[float] = None) -> int:
        sc = self.scenes[set_index]
        first = sc.frame_fixed_bytes(cam, self.params) + int(cam.width) * int(cam.height) * 12
        with self.cv:
            rid = self.next_id
            self.next_id += 1
            p = _Pending(rid, set_index, cam, self.now() if arrival is None else arrival, first)
            self.queue.append(p)
            self.cv.notify_all()
            return rid

    def now(self) -> float:
        return time.perf_counter() - self.t0

    def _pick(self) -> Optional[_Pending]:
        """Earliest queued request whose known footprint fits the free budget; a request
        passed over `max_bypass` times blocks later ones until it fits.  With nothing in
        flight the head is admitted whatever its footprint (so no request waits forever)."""
        free = self.budget - self.reserved
        for k, p in enumerate(self.queue):
            if p.need <= free or self.in_flight == 0:
                for q in list(self.queue)[:k]:
                    q.bypassed += 1
                del self.queue[k]
                return p
            if p.bypassed >= self.max_bypass:
                return None
        return None

    def _reserve(self, n: int) -> None:
        self.reserved += n
        self.peak_reserved = max(self.peak_reserved, self.reserved)

    def _worker(self, k: int):
        self.dev.bind()
        stream = self.streams[k]
        while True:
            with self.cv:
                p = None
                while not self.stop:
                    p = self._pick()
                    if p is not None:
                        break
                    self.cv.wait(timeout=0.05)
                if p is None:
                    return
                held = p.need  # the first part, and the lists when a count phase already ran
                self._reserve(held)
                self.in_flight += 1
            start = self.now()
            frame = None
            img = None
            requeue = False
            try:
                sc = self.scenes[p.set_index]
                cam = p.camera
                frame = sc.prepare(cam, self.params, stream=stream)
                with self.cv:
                    if p.lists is not None and frame.var_bytes > p.lists:
                        # cannot happen (the count phase is deterministic); stay exact anyway
                        self._reserve(frame.var_bytes - p.lists)
                        held += frame.var_bytes - p.lists
                    if p.lists is None:
                        # the count phase's exact list bytes: reserve them now if they
                        # fit, else give everything back and wait with the full footprint.
                        # Past the budget only while this request is the only one in flight
                        # (others admitted during its count phase took the free budget).
                        alone = self.in_flight == 1
                        if self.reserved + frame.var_bytes <= self.budget or alone:
                            self._reserve(frame.var_bytes)
                            held += frame.var_bytes
                        else:
                            requeue = True
                    p.lists = frame.var_bytes
                if not requeue:
                    img = self.dev.image(int(cam.height), int(cam.width), stream)
                    frame.render(img, stream=stream)
                    self.dev.synchronize(stream)
            except Exception as e:  # a failed request is reported, the server keeps going
                with self.cv:
                    self.errors.append(f"request {p.request_id}: {e}")
            finally:
                if frame is not None:
                    fixed, var, pairs = frame.fixed_bytes, frame.var_bytes, frame.pairs
                    frame.close()
                    self.dev.synchronize(stream)
            finish = self.now()
            with self.cv:
                self.reserved -= held
                self.in_flight -= 1
                if requeue:
                    p.bypassed = 0
                    self.queue.appendleft(p)
                    self.requeued += 1
                elif frame is not None:
                    self.done.append(Completed(p.request_id, p.set_index, int(p.camera.width),
                                               int(p.camera.height), p.arrival, start, finish, pairs, held,
                                               fixed + var + int(p.camera.width) * int(p.camera.height) * 12,
                                               img if (self.keep_images and img is not None) else None))
                self.cv.notify_all()

    def wait_all(self, timeout: Optional[float] = None) -> None:
        t_end = None if timeout is None else time.perf_counter() + timeout
        with self.cv:
            while self.queue or self.in_flight:
                left = None if t_end is None else t_end - time.perf_counter()
                if left is not None and left <= 0:
                    raise TimeoutError("server did not drain")
                self.cv.wait(timeout=0.05 if left is None else min(0.05, left))

    def close(self):
        with self.cv:
            self.stop = True
            self.cv.notify_all()
        for t in self.threads:
            t.join(timeout=10)

    # ---------------------------------------------------------------------------------
    def run_trace(self, requests: Sequence, time_scale: float = 1.0) -> dict:
        """Replay requests (objects with set_index, camera, arrival_s) in real time,
        wait for all and return the statistics of this trace."""
        first = len(self.done)
        t_base = self.now()
        for r in requests:
            t_arr = t_base + r.arrival_s * time_scale
            dt = t_arr - self.now()
            if dt > 0:
                time.sleep(dt)
            self.submit(r.set_index, r.camera, arrival=t_arr)
        self.wait_all()
        return stats(self.done[first:], [self.scenes[i].n for i in range(len(self.scenes))])


def stats(done: Sequence[Completed], set_sizes: Sequence[int]) -> dict:
    if not done:
        return {"requests": 0}
    lat = np.array([d.latency for d in done])
    t0 = min(d.arrival for d in done)
    t1 = max(d.finish for d in done)
    parts = sum(set_sizes[d.set_index] for d in done)
    span = max(t1 - t0, 1e-9)
    return {"requests": len(done), "seconds": span, "requests_per_s": len(done) / span,
            "mparticles_per_s": parts / span / 1e6, "p50_ms": 1e3 * float(np.percentile(lat, 50)),
            "p99_ms": 1e3 * float(np.percentile(lat, 99)), "mean_ms": 1e3 * float(lat.mean()),
            "max_ms": 1e3 * float(lat.max()),
            "pairs_per_request": float(np.mean([d.pairs for d in done]))}
