"""Continuous-batching request loop for light-field frames.

Requests (frames of any size, camera count, D and iteration count) arrive
over time.  Each is admitted once a slot is free and its device buffers fit
the free HBM (``torch.cuda.mem_get_info`` minus a reserve, or an explicit
byte budget); on admission its inputs are copied to the device on a copy
stream and stay there until its results are read back.  Admitted requests are
batched as they become ready: up to ``inflight`` batches (``lf.Batch``, each
on its own stream, each one CUDA graph) run at once, so requests arriving
while others are on the GPU are admitted, copied and launched without
waiting for them.  Completion is polled with CUDA events; per-request latency
is completion minus arrival.

``mode="plain"`` is the reference path: one frame per launch through
``lf.Context`` (float32 maps), in arrival order, inputs copied to the device
per request.
"""
from __future__ import annotations

import collections
import dataclasses
import time
from typing import List, Optional

import numpy as np

from . import lf


@dataclasses.dataclass
class Request:
    """One frame to process.  Host arrays as ``scenes.Scene`` holds them."""

    rid: int
    baselines: np.ndarray
    images: np.ndarray
    seg_prior: np.ndarray
    points: np.ndarray
    d_min: float
    d_max: float
    D: int
    iters: int
    arrival: float = 0.0          # seconds, on the server's clock
    admitted: float = -1.0
    launched: float = -1.0
    done: float = -1.0
    result: Optional[dict] = None  # host numpy outputs
    # device state while admitted
    dev: Optional[dict] = None
    copy_event: object = None
    nbytes: int = 0

    @classmethod
    def from_scene(cls, rid: int, scene, arrival: float = 0.0) -> "Request":
        return cls(rid, scene.baselines, scene.images, scene.seg_prior, scene.points, scene.d_min, scene.d_max,
                   scene.D, scene.iters, arrival)

    @property
    def K(self):
        return int(self.images.shape[0])

    @property
    def H(self):
        return int(self.images.shape[1])

    @property
    def W(self):
        return int(self.images.shape[2])

    @property
    def C(self):
        return 1 if self.images.ndim == 3 else int(self.images.shape[3])

    @property
    def latency(self) -> float:
        return self.done - self.arrival

    def device_bytes(self) -> int:
        """Inputs, outputs and the batch's per-frame workspace (prior map,
        staging) -- what admission reserves."""
        K, H, W, C = self.K, self.H, self.W, self.C
        HW = H * W
        inputs = self.images.nbytes + self.seg_prior.nbytes
        outputs = HW * (4 + 4 + 2) + K * HW * 4 + HW * C * 4
        workspace = HW * 4 + inputs + 64 * 1024
        return inputs + outputs + workspace


def _pinned(torch, arr):
    """A page-locked CPU tensor over arr (no copy if arr already is one)."""
    t = arr if isinstance(arr, torch.Tensor) else torch.from_numpy(np.ascontiguousarray(arr))
    return t if t.is_pinned() else t.pin_memory()


def percentiles(latencies: List[float]) -> dict:
    if not latencies:
        return {"p50_ms": None, "p95_ms": None, "p99_ms": None}
    a = np.asarray(latencies) * 1e3
    return {"p50_ms": float(np.percentile(a, 50)), "p95_ms": float(np.percentile(a, 95)),
            "p99_ms": float(np.percentile(a, 99))}


class Server:
    """The request loop.  ``mode`` is "batched" (continuous batching) or
    "plain" (one frame per launch, float32)."""

    def __init__(self, params: Optional[lf.Params] = None, *, mode: str = "batched", max_batch: int = 32,
                 inflight: int = 2, max_slots: int = 256, hbm_reserve: int = 4 << 30,
                 hbm_budget: Optional[int] = None):
        import torch
        self.torch = torch
        self.mode = mode
        self.params = params if params is not None else lf.default_params()
        self.max_batch = max_batch
        self.max_slots = max_slots
        self.hbm_reserve = hbm_reserve
        self.hbm_budget = hbm_budget      # explicit cap on admitted bytes (tests), else free HBM
        self.admitted_bytes = 0
        self.copy_stream = torch.cuda.Stream()
        self.pending: collections.deque = collections.deque()
        self.ready: List[Request] = []
        self.inflight = []                # (batch index, requests, done event)
        self.draining = []                # (requests, event of their result copies)
        self.completed: List[Request] = []
        self.t0 = time.perf_counter()
        self.peak_admitted = 0
        self.batches_run = 0
        if mode == "batched":
            self.streams = [torch.cuda.Stream() for _ in range(inflight)]
            self.batches = [lf.Batch(self.params, stream=s) for s in self.streams]
            self.free_batches = list(range(inflight))
        elif mode == "plain":
            self.stream = torch.cuda.current_stream()
        else:
            raise ValueError(mode)

    # ------------------------------------------------------------ plumbing
    def now(self) -> float:
        return time.perf_counter() - self.t0

    def submit(self, req: Request):
        self.pending.append(req)

    def _fits(self, need: int) -> bool:
        if self.hbm_budget is not None:
            return self.admitted_bytes + need <= self.hbm_budget
        free, _ = self.torch.cuda.mem_get_info()
        return free - need >= self.hbm_reserve

    def _admit(self):
        torch = self.torch
        n_admitted = len(self.ready) + sum(len(r) for _, r, _ in self.inflight) + \
            sum(len(r) for r, _ in self.draining)
        while self.pending and n_admitted < self.max_slots:
            req = self.pending[0]
            need = req.device_bytes()
            if not self._fits(need):
                break                      # head-of-line: keep arrival order
            self.pending.popleft()
            req.nbytes = need
            self.admitted_bytes += need
            with torch.cuda.stream(self.copy_stream):
                img = _pinned(torch, req.images).to("cuda", non_blocking=True)
                seg = _pinned(torch, req.seg_prior).to("cuda", non_blocking=True)
                out = lf.device_outputs(req.K, req.H, req.W, req.C)
                ev = torch.cuda.Event()
                ev.record(self.copy_stream)
            req.dev = {"img": img, "seg": seg, "out": out}
            req.copy_event = ev
            req.admitted = self.now()
            self.ready.append(req)
            n_admitted += 1
        self.peak_admitted = max(self.peak_admitted, n_admitted)

    def _launch(self):
        torch = self.torch
        while self.ready and self.free_batches:
            bi = self.free_batches.pop(0)
            b, s = self.batches[bi], self.streams[bi]
            reqs = self.ready[:self.max_batch]
            self.ready = self.ready[self.max_batch:]
            b.clear()
            for r in reqs:
                s.wait_event(r.copy_event)
                b.add(r.baselines, r.d_min, r.d_max, r.D, r.iters, r.dev["img"], r.dev["seg"], r.points,
                      r.dev["out"])
                r.launched = self.now()
            b.run()
            ev = torch.cuda.Event()
            ev.record(s)
            self.inflight.append((bi, reqs, ev))
            self.batches_run += 1

    def _complete(self):
        torch = self.torch
        still = []
        for bi, reqs, ev in self.inflight:
            if not ev.query():
                still.append((bi, reqs, ev))
                continue
            self.batches[bi].synchronize()   # surfaces device errors of this batch
            # results to page-locked host buffers on the copy stream; the
            # batch object is free again at once
            self.copy_stream.wait_event(ev)
            with torch.cuda.stream(self.copy_stream):
                for r in reqs:
                    r.result = {k: torch.empty(v.shape, dtype=v.dtype, pin_memory=True).copy_(v, non_blocking=True)
                                for k, v in r.dev["out"].items()}
                done = torch.cuda.Event()
                done.record(self.copy_stream)
            self.draining.append((reqs, done))
            self.free_batches.append(bi)
        self.inflight = still
        keep = []
        for reqs, done in self.draining:
            if not done.query():
                keep.append((reqs, done))
                continue
            t = self.now()
            for r in reqs:
                r.result = {k: v.numpy() for k, v in r.result.items()}
                r.done = t
                r.dev = None
                self.admitted_bytes -= r.nbytes
                self.completed.append(r)
        self.draining = keep

    def _plain_one(self, req: Request):
        torch = self.torch
        req.admitted = req.launched = self.now()
        p = lf.default_params(precision=lf.LF_PREC_F32)
        for f in ("beta", "gamma", "sigma", "seg_threshold", "eps", "mstep_seg_term", "median", "early_exit"):
            setattr(p, f, getattr(self.params, f))
        with lf.Context(req.baselines, req.H, req.W, req.d_min, req.d_max, req.D, p) as ctx:
            ctx.set_stream(self.stream)
            img = _pinned(torch, req.images).to("cuda", non_blocking=True)
            seg = _pinned(torch, req.seg_prior).to("cuda", non_blocking=True)
            ctx.set_inputs(img, seg, req.points)
            out = ctx.run(req.iters, device=True)
            ctx.synchronize()
            req.result = {k: v.cpu().numpy() for k, v in out.items()}
        req.done = self.now()
        self.completed.append(req)

    # ------------------------------------------------------------ loops
    def step(self):
        """One pass of the batched loop (non-blocking)."""
        self._complete()
        self._admit()
        self._launch()

    def drain(self, timeout_s: float = 600.0):
        """Run until every submitted request is complete."""
        t_end = time.perf_counter() + timeout_s
        if self.mode == "plain":
            while self.pending:
                self._plain_one(self.pending.popleft())
            return
        while self.pending or self.ready or self.inflight or self.draining:
            self.step()
            if time.perf_counter() > t_end:
                raise TimeoutError("server did not drain")
            if self.inflight and not self.ready and (not self.pending or not self.free_batches):
                time.sleep(0.0002)

    def run_arrivals(self, requests: List[Request], timeout_s: float = 600.0) -> dict:
        """Replay requests at their arrival times (seconds from now) and
        report latency percentiles and throughput."""
        self.t0 = time.perf_counter()
        order = sorted(requests, key=lambda r: r.arrival)
        i = 0
        t_end = time.perf_counter() + timeout_s
        while i < len(order) or self.pending or self.ready or \
                (self.mode == "batched" and (self.inflight or self.draining)):
            now = self.now()
            while i < len(order) and order[i].arrival <= now:
                self.submit(order[i])
                i += 1
            if self.mode == "plain":
                if self.pending:
                    self._plain_one(self.pending.popleft())
                elif i < len(order):
                    time.sleep(max(0.0, min(order[i].arrival - self.now(), 0.001)))
            else:
                self.step()
                if not self.ready and not (self.pending and self.free_batches):
                    time.sleep(0.0002)
            if time.perf_counter() > t_end:
                raise TimeoutError("arrival replay did not finish")
        lat = [r.latency for r in self.completed]
        span = max(r.done for r in self.completed) - min(r.arrival for r in self.completed)
        out = {"requests": len(self.completed), "frames_per_s": len(self.completed) / span if span > 0 else None,
               "batches": self.batches_run, "peak_admitted": self.peak_admitted}
        out.update(percentiles(lat))
        return out

    def close(self):
        if self.mode == "batched":
            for b in self.batches:
                b.close()


def poisson_arrivals(rate_hz: float, duration_s: float, seed: int) -> np.ndarray:
    """Arrival times of a Poisson process of the given rate over duration_s."""
    rng = np.random.default_rng(seed)
    t, out = 0.0, []
    while True:
        t += rng.exponential(1.0 / rate_hz)
        if t >= duration_s:
            return np.asarray(out)
        out.append(t)
