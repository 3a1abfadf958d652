"""Continuous-batching request loop for light-field frames.

Requests (frames of any size, camera count, D and iteration count) arrive
over time.  Each is admitted once a slot is free and its device buffers fit
the server's share of HBM; on admission its inputs are copied to the device
on a copy stream and stay there until its results are read back.  Admitted
requests are batched as they become ready: up to ``inflight`` batches
(``lf.Batch``, each on its own stream, each one CUDA graph) run at once, so
requests arriving while others are on the GPU are admitted, copied and
launched without waiting for them.  Completion is polled with CUDA events;
per-request latency is completion (results on the host) minus arrival.

Memory.  The loop allocates nothing once it runs.  At start the server takes
one device block (``hbm_budget`` bytes, by default the free HBM minus
``hbm_reserve``, capped at ``max_arena``) and one page-locked host block for
results, and carves every request's buffers out of them with a first-fit
``Arena``: admission by free HBM is then admission by free arena space,
without allocator calls (each of which can synchronise the device) or a
free-memory query that drifts with other allocators' caches.  A request that
can never fit is rejected at ``submit``; a request still waiting for
admission (or admitted but not launched) can be cancelled, which returns its
bytes.  Results are numpy views of the host block, valid until ``release``.

``mode="plain"`` is the reference path: one frame per launch through
``lf.Context`` with float32 maps, in arrival order; one context per frame
signature, created on first use and kept.
"""
from __future__ import annotations

import bisect
import collections
import dataclasses
import time
from typing import List, Optional, Tuple

import numpy as np

from . import lf

_ALIGN = 256


class Arena:
    """First-fit allocation of byte ranges in [0, capacity) (host logic; the
    server maps ranges onto one device block and one host block).  Blocks
    are aligned to ``align`` bytes; freed neighbours merge."""

    def __init__(self, capacity: int, align: int = _ALIGN):
        self.capacity = int(capacity) // align * align
        self.align = align
        self.free_list: List[Tuple[int, int]] = [(0, self.capacity)] if self.capacity > 0 else []  # (offset, size)
        self.used: dict = {}
        self.bytes_used = 0
        self.peak = 0

    def size_of(self, nbytes: int) -> int:
        return max(self.align, (int(nbytes) + self.align - 1) // self.align * self.align)

    def fits_ever(self, nbytes: int) -> bool:
        return self.size_of(nbytes) <= self.capacity

    def alloc(self, nbytes: int) -> Optional[int]:
        need = self.size_of(nbytes)
        for i, (off, size) in enumerate(self.free_list):
            if size >= need:
                if size == need:
                    self.free_list.pop(i)
                else:
                    self.free_list[i] = (off + need, size - need)
                self.used[off] = need
                self.bytes_used += need
                self.peak = max(self.peak, self.bytes_used)
                return off
        return None

    def free(self, off: int):
        size = self.used.pop(off)
        self.bytes_used -= size
        i = bisect.bisect_left(self.free_list, (off, 0))
        self.free_list.insert(i, (off, size))
        # merge with the next and the previous free range
        if i + 1 < len(self.free_list) and off + size == self.free_list[i + 1][0]:
            self.free_list[i] = (off, size + self.free_list[i + 1][1])
            self.free_list.pop(i + 1)
        if i > 0 and self.free_list[i - 1][0] + self.free_list[i - 1][1] == off:
            poff, psize = self.free_list[i - 1]
            self.free_list[i - 1] = (poff, psize + self.free_list[i][1])
            self.free_list.pop(i)


@dataclasses.dataclass
class Request:
    """One frame to process.  Host arrays as ``scenes.Scene`` holds them (or
    page-locked torch tensors)."""

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
    status: str = "new"           # pending, admitted, launched, done, rejected, cancelled
    error: str = ""
    result: Optional[dict] = None  # host numpy outputs (views of the server's host block)
    # device state while admitted
    dev: Optional[dict] = None
    dev_off: Optional[int] = None
    host_off: Optional[int] = None
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
        return 1 if len(self.images.shape) == 3 else int(self.images.shape[3])

    @property
    def latency(self) -> float:
        return self.done - self.arrival

    def output_layout(self) -> List[Tuple[str, tuple, object]]:
        """(name, shape, numpy dtype) of every output, in block order."""
        K, H, W, C = self.K, self.H, self.W, self.C
        return [("d_idx", (H, W), np.int32), ("d", (H, W), np.float32), ("post", (K, H, W), np.float32),
                ("labels", (H, W), np.int16), ("refocus", (H, W, C) if C > 1 else (H, W), np.float32)]

    def output_bytes(self) -> int:
        return sum(_aligned(int(np.prod(s)) * np.dtype(t).itemsize) for _, s, t in self.output_layout())

    def device_bytes(self) -> int:
        """Inputs and outputs in the device block -- what admission reserves
        there (the batch's own per-frame workspace is sized at warm-up)."""
        return _aligned(_nbytes(self.images)) + _aligned(_nbytes(self.seg_prior)) + self.output_bytes()


def _aligned(n: int) -> int:
    return (int(n) + _ALIGN - 1) // _ALIGN * _ALIGN


def _nbytes(a) -> int:
    return int(a.nbytes) if hasattr(a, "nbytes") else int(a.numel() * a.element_size())


def percentiles(latencies: List[float]) -> dict:
    if not latencies:
        return {"p50_ms": None, "p95_ms": None, "p99_ms": None}
    a = np.asarray(latencies) * 1e3
    return {"p50_ms": float(np.percentile(a, 50)), "p95_ms": float(np.percentile(a, 95)),
            "p99_ms": float(np.percentile(a, 99))}


def _torch_dtype(torch, dt):
    return {np.dtype(np.int32): torch.int32, np.dtype(np.float32): torch.float32, np.dtype(np.int16): torch.int16,
            np.dtype(np.uint8): torch.uint8, np.dtype(np.float16): torch.float16}[np.dtype(dt)]


def _np_dtype(a):
    return a.dtype if isinstance(a, np.ndarray) else a.numpy().dtype


class Server:
    """The request loop.  ``mode`` is "batched" (continuous batching) or
    "plain" (one frame per launch, float32)."""

    def __init__(self, params: Optional[lf.Params] = None, *, mode: str = "batched", max_batch: int = 32,
                 inflight: int = 2, max_slots: int = 256, hbm_reserve: int = 4 << 30,
                 hbm_budget: Optional[int] = None, max_arena: int = 16 << 30, host_budget: Optional[int] = None):
        import torch
        self.torch = torch
        self.mode = mode
        self.params = params if params is not None else lf.default_params()
        self.max_batch = max_batch
        self.max_slots = max_slots
        if mode == "plain":
            hbm_budget = 0                # the cached contexts own the device buffers
        elif hbm_budget is None:
            free, _ = torch.cuda.mem_get_info()
            hbm_budget = max(0, min(free - hbm_reserve, max_arena))
        self.dev_arena = Arena(hbm_budget)
        self.host_arena = Arena(host_budget if host_budget is not None else 2 << 30)
        self.dev_block = torch.empty(max(self.dev_arena.capacity, _ALIGN), dtype=torch.uint8, device="cuda")
        self.host_block = torch.empty(max(self.host_arena.capacity, _ALIGN), dtype=torch.uint8, pin_memory=True)
        self.copy_stream = torch.cuda.Stream()
        self.pending: collections.deque = collections.deque()
        self.ready: List[Request] = []
        self.inflight = []                # (batch index, requests, done event)
        self.draining = []                # (requests, event of their result copies)
        self.completed: List[Request] = []
        self.rejected: List[Request] = []
        self.keep_results = True
        self.t0 = time.perf_counter()
        self.peak_admitted = 0
        self.batches_run = 0
        self.contexts = {}                # plain mode: one context per frame signature
        if mode == "batched":
            self.streams = [torch.cuda.Stream() for _ in range(inflight)]
            self.batches = [lf.Batch(self.params, stream=s) for s in self.streams]
            self.free_batches = list(range(inflight))
        elif mode == "plain":
            self.stream = torch.cuda.current_stream()
        else:
            raise ValueError(mode)

    @property
    def admitted_bytes(self) -> int:
        return self.dev_arena.bytes_used

    # ------------------------------------------------------------ plumbing
    def now(self) -> float:
        return time.perf_counter() - self.t0

    def submit(self, req: Request) -> bool:
        """Queue a request; False (and status "rejected") if it can never fit
        the server's device or host block."""
        need_dev = req.device_bytes() if self.mode == "batched" else 0
        if (need_dev and not self.dev_arena.fits_ever(need_dev)) or not self.host_arena.fits_ever(req.output_bytes()):
            req.status = "rejected"
            req.error = (f"needs {need_dev} device bytes and {req.output_bytes()} host bytes; the server holds "
                         f"{self.dev_arena.capacity} and {self.host_arena.capacity}")
            req.done = self.now()
            self.rejected.append(req)
            return False
        req.status = "pending"
        self.pending.append(req)
        return True

    def cancel(self, req: Request) -> bool:
        """Withdraw a request that waits for admission or for its launch; its
        bytes are returned.  False once it is on the GPU or finished."""
        if req.status == "pending":
            self.pending.remove(req)
        elif req.status == "admitted" and req in self.ready:
            self.ready.remove(req)
            self._free(req, keep_result=False)
        else:
            return False
        req.status = "cancelled"
        return True

    def release(self, req: Request):
        """Return the host bytes of a completed request's results (they are
        views of the server's host block and become invalid)."""
        if req.host_off is not None:
            self.host_arena.free(req.host_off)
            req.host_off = None
        req.result = None

    def _free(self, req: Request, keep_result: bool):
        if req.dev_off is not None:
            self.dev_arena.free(req.dev_off)
            req.dev_off = None
        req.dev = None
        if not keep_result:
            self.release(req)

    def _host_views(self, req: Request, torch_views: bool):
        out, off = {}, req.host_off
        for name, shape, dt in req.output_layout():
            n = int(np.prod(shape)) * np.dtype(dt).itemsize
            v = self.host_block[off:off + n]
            out[name] = v.view(_torch_dtype(self.torch, dt)).view(shape) if torch_views else \
                v.numpy().view(dt).reshape(shape)
            off += _aligned(n)
        return out

    def _device_views(self, req: Request):
        """Device input and output views of an admitted request, carved out
        of the device block."""
        torch = self.torch
        off = req.dev_off
        n = _nbytes(req.images)
        img = self.dev_block[off:off + n].view(_torch_dtype(torch, _np_dtype(req.images))).view(tuple(req.images.shape))
        off += _aligned(n)
        n = _nbytes(req.seg_prior)
        seg = self.dev_block[off:off + n].view(torch.float32).view(tuple(req.seg_prior.shape))
        off += _aligned(n)
        out = {}
        for name, shape, dt in req.output_layout():
            n = int(np.prod(shape)) * np.dtype(dt).itemsize
            out[name] = self.dev_block[off:off + n].view(_torch_dtype(torch, dt)).view(shape)
            off += _aligned(n)
        return img, seg, out

    def _admit(self):
        torch = self.torch
        n_admitted = len(self.ready) + sum(len(r) for _, r, _ in self.inflight) + \
            sum(len(r) for r, _ in self.draining)
        while self.pending and n_admitted < self.max_slots:
            req = self.pending[0]
            doff = self.dev_arena.alloc(req.device_bytes())
            if doff is None:
                break                      # head-of-line: keep arrival order
            hoff = self.host_arena.alloc(req.output_bytes())
            if hoff is None:
                self.dev_arena.free(doff)
                break
            self.pending.popleft()
            req.dev_off, req.host_off = doff, hoff
            req.nbytes = req.device_bytes()
            img, seg, out = self._device_views(req)
            with torch.cuda.stream(self.copy_stream):
                img.copy_(_as_tensor(torch, req.images), non_blocking=True)
                seg.copy_(_as_tensor(torch, req.seg_prior), non_blocking=True)
                ev = torch.cuda.Event()
                ev.record(self.copy_stream)
            req.dev = {"img": img, "seg": seg, "out": out, "host": self._host_views(req, True)}
            req.copy_event = ev
            req.admitted = self.now()
            req.status = "admitted"
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
                r.status = "launched"
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
            # results to the page-locked host block on the copy stream; the
            # batch object is free again at once
            self.copy_stream.wait_event(ev)
            with torch.cuda.stream(self.copy_stream):
                for r in reqs:
                    for k, v in r.dev["out"].items():
                        r.dev["host"][k].copy_(v, non_blocking=True)
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
                self._finish(r, t)
        self.draining = keep

    def _finish(self, r: Request, t: float):
        r.result = self._host_views(r, False)
        r.result["labels"] = r.result["labels"].view(np.uint16)
        r.done = t
        r.status = "done"
        self._free(r, keep_result=self.keep_results)
        self.completed.append(r)

    def _plain_one(self, req: Request):
        req.admitted = req.launched = self.now()
        key = (tuple(np.asarray(req.baselines, np.float32).tolist()), req.H, req.W, float(req.d_min),
               float(req.d_max), req.D)
        ctx = self.contexts.get(key)
        if ctx is None:
            p = lf.default_params(precision=lf.LF_PREC_F32)
            for f in ("beta", "gamma", "sigma", "seg_threshold", "eps", "mstep_seg_term", "median", "early_exit"):
                setattr(p, f, getattr(self.params, f))
            ctx = lf.Context(req.baselines, req.H, req.W, req.d_min, req.d_max, req.D, p)
            ctx.set_stream(self.stream)
            self.contexts[key] = ctx
        hoff = self.host_arena.alloc(req.output_bytes())
        if hoff is None:
            raise MemoryError("the host block is full: release completed results")
        req.host_off = hoff
        host = self._host_views(req, False)
        host["labels"] = host["labels"].view(np.uint16)
        ctx.set_inputs(_as_host(req.images), _as_host(req.seg_prior), req.points)
        ctx.run(req.iters, out=host)
        req.result = host
        req.done = self.now()
        req.status = "done"
        if not self.keep_results:
            self.release(req)
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

    def run_arrivals(self, requests: List[Request], timeout_s: float = 600.0,
                     keep_results: bool = True) -> dict:
        """Replay requests at their arrival times (seconds from now) and
        report latency percentiles and throughput.  keep_results=False
        releases every result at completion (long runs)."""
        self.keep_results = keep_results
        self.t0 = time.perf_counter()
        order = sorted(requests, key=lambda r: r.arrival)
        i = 0
        t_end = time.perf_counter() + timeout_s
        last, max_gap = time.perf_counter(), 0.0
        while i < len(order) or self.pending or self.ready or \
                (self.mode == "batched" and (self.inflight or self.draining)):
            tnow = time.perf_counter()
            max_gap = max(max_gap, tnow - last)
            last = tnow
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
        self.keep_results = True
        lat = [r.latency for r in self.completed]
        span = max(r.done for r in self.completed) - min(r.arrival for r in self.completed) if self.completed else 0
        out = {"requests": len(self.completed), "rejected": len(self.rejected),
               "frames_per_s": len(self.completed) / span if span > 0 else None,
               "batches": self.batches_run, "peak_admitted": self.peak_admitted,
               # HBM the admitted requests held at most (device block bytes, since the server started)
               "peak_device_bytes": self.dev_arena.peak,
               "max_loop_gap_ms": 1e3 * max_gap}
        out.update(percentiles(lat))
        # where the time goes: queueing for admission, admitted to launch,
        # launch to results on the host (p50 / p99 of each, ms)
        for name, a, b in (("wait", "arrival", "admitted"), ("ready", "admitted", "launched"),
                           ("run", "launched", "done")):
            x = np.asarray([getattr(r, b) - getattr(r, a) for r in self.completed]) * 1e3
            if x.size:
                out[f"{name}_p50_ms"] = float(np.percentile(x, 50))
                out[f"{name}_p99_ms"] = float(np.percentile(x, 99))
        if self.mode == "batched":
            out["graph_captures"] = sum(b.stats()["graph_captures"] for b in self.batches)
        return out

    def close(self):
        if self.mode == "batched":
            for b in self.batches:
                b.close()
        for c in self.contexts.values():
            c.close()
        self.contexts = {}


def _as_tensor(torch, a):
    return a if isinstance(a, torch.Tensor) else torch.from_numpy(np.ascontiguousarray(a))


def _as_host(a):
    """A numpy view of a host array or CPU tensor (no copy)."""
    return a if isinstance(a, np.ndarray) else a.numpy()


def poisson_arrivals(rate_hz: float, duration_s: float, seed: int) -> np.ndarray:
    """Arrival times of a Poisson process of the given rate over duration_s."""
    rng = np.random.default_rng(seed)
    t, out = 0.0, []
    while True:
        t += rng.exponential(1.0 / rate_hz)
        if t >= duration_s:
            return np.asarray(out)
        out.append(t)
