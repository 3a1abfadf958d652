"""Python binding of the C ABI in ``include/lf.h`` (ctypes; marshalling only).

Every step of the path runs in the library's CUDA kernels.  Loading fails
loudly when the in-tree ``_lib/liblf.so`` is missing -- there is no CPU
fallback.  Host inputs are numpy arrays; device inputs are torch CUDA tensors
(torch is only imported when such a tensor is passed), whose data pointers are
handed to the library together with the current torch stream.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional

import numpy as np

LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "_lib", "liblf.so")

LF_OK, LF_EINVAL, LF_ENOMEM, LF_ECUDA, LF_ESTATE, LF_ETIMEOUT = range(6)
LF_U8, LF_F32, LF_F16, LF_BF16 = 0, 1, 2, 3
LF_PREC_F32, LF_PREC_F16, LF_PREC_BF16 = 0, 1, 2
LF_EM_HARD, LF_EM_SOFT, LF_EM_JOINT = 0, 1, 2

EXPORTS = ("lf_default_params", "lf_create", "lf_set_stream", "lf_set_inputs", "lf_run_em",
           "lf_synchronize", "lf_get_prior", "lf_get_stats", "lf_last_error", "lf_destroy",
           "lf_triangulate", "lf_set_timing", "lf_run_em_static", "lf_batch_create", "lf_batch_set_stream",
           "lf_batch_add", "lf_batch_run", "lf_batch_synchronize", "lf_batch_clear", "lf_batch_get_stats",
           "lf_batch_destroy", "lf_set_tile", "lf_create_calibrated", "lf_default_support_params",
           "lf_set_support_params", "lf_get_support_points", "lf_selftest_bounded_wait", "lf_host_alloc",
           "lf_host_free", "lf_inject_alloc_failure")
LF_DETECT_SUPPORT = -1
LF_HOST_ASYNC = 2


class LfError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"lf status {status}: {msg}")
        self.status = status


class Params(ctypes.Structure):
    _fields_ = [("beta", ctypes.c_float), ("gamma", ctypes.c_float), ("sigma", ctypes.c_float),
                ("seg_threshold", ctypes.c_float), ("eps", ctypes.c_float),
                ("mstep_seg_term", ctypes.c_int), ("median", ctypes.c_int), ("precision", ctypes.c_int),
                ("early_exit", ctypes.c_int), ("dynamic_only", ctypes.c_int),
                ("em_mode", ctypes.c_int), ("prune", ctypes.c_int)]


class SupportParams(ctypes.Structure):
    """lf_support_params (support-point detection, see include/lf.h)."""
    _fields_ = [("grid", ctypes.c_int), ("ratio_pct", ctypes.c_int), ("texture", ctypes.c_int),
                ("window", ctypes.c_int), ("delta", ctypes.c_float), ("min_support", ctypes.c_int)]


class Stats(ctypes.Structure):
    _fields_ = [("runs", ctypes.c_uint64), ("nominal_ray_samples", ctypes.c_uint64),
                ("executed_ray_samples", ctypes.c_uint64),
                ("halo_left", ctypes.c_int), ("halo_right", ctypes.c_int),
                ("tile_rows", ctypes.c_int), ("tile_cols", ctypes.c_int),
                ("kernels_launched", ctypes.c_int),
                ("ms_prior", ctypes.c_float), ("ms_sweep", ctypes.c_float), ("ms_refocus", ctypes.c_float),
                ("ms_median", ctypes.c_float), ("graph_captures", ctypes.c_int),
                ("tuned_signatures", ctypes.c_int), ("ms_support", ctypes.c_float),
                ("ms_set_inputs", ctypes.c_float), ("executed_static_ray_samples", ctypes.c_uint64),
                ("executed_pixel_iterations", ctypes.c_uint64)]


_lib = None


def load(path: str = LIB_PATH) -> ctypes.CDLL:
    """Load the in-tree library (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"{path} is missing: build it with `python -c 'import __graft_entry__ as g; g.build()'`")
    lib = ctypes.CDLL(path)
    P = ctypes.c_void_p
    I = ctypes.c_int
    lib.lf_default_params.argtypes = [ctypes.POINTER(Params)]
    lib.lf_default_params.restype = None
    lib.lf_create.argtypes = [ctypes.POINTER(P), I, P, I, I, ctypes.c_float, ctypes.c_float, I,
                              ctypes.POINTER(Params)]
    lib.lf_create_calibrated.argtypes = lib.lf_create.argtypes
    lib.lf_default_support_params.argtypes = [ctypes.POINTER(SupportParams)]
    lib.lf_default_support_params.restype = None
    lib.lf_set_support_params.argtypes = [P, ctypes.POINTER(SupportParams)]
    lib.lf_set_support_params.restype = I
    lib.lf_get_support_points.argtypes = [P, P, I, ctypes.POINTER(I)]
    lib.lf_get_support_points.restype = I
    lib.lf_set_stream.argtypes = [P, P]
    lib.lf_set_inputs.argtypes = [P, P, I, I, P, P, I, I]
    lib.lf_run_em.argtypes = [P, I, P, P, P, P, P, I]
    lib.lf_synchronize.argtypes = [P]
    lib.lf_get_prior.argtypes = [P, P, I]
    lib.lf_get_stats.argtypes = [P, ctypes.POINTER(Stats)]
    lib.lf_set_timing.argtypes = [P, I]
    lib.lf_set_tile.argtypes = [P, I, I]
    lib.lf_set_tile.restype = I
    lib.lf_last_error.argtypes = [P]
    lib.lf_last_error.restype = ctypes.c_char_p
    lib.lf_destroy.argtypes = [P]
    lib.lf_destroy.restype = None
    lib.lf_run_em_static.argtypes = [I, P, I, I, ctypes.c_float, ctypes.c_float, I, ctypes.POINTER(Params), I,
                                     P, I, I, P, P, P, P, P, P, P]
    lib.lf_run_em_static.restype = I
    lib.lf_batch_create.argtypes = [ctypes.POINTER(P), ctypes.POINTER(Params), I]
    lib.lf_batch_set_stream.argtypes = [P, P]
    lib.lf_batch_add.argtypes = [P, I, P, I, I, ctypes.c_float, ctypes.c_float, I, I, P, I, I, P, P, I,
                                 P, P, P, P, P, ctypes.POINTER(I)]
    lib.lf_batch_run.argtypes = [P]
    lib.lf_batch_synchronize.argtypes = [P]
    lib.lf_batch_clear.argtypes = [P]
    lib.lf_batch_get_stats.argtypes = [P, ctypes.POINTER(Stats)]
    lib.lf_batch_destroy.argtypes = [P]
    lib.lf_batch_destroy.restype = None
    for name in ("lf_batch_create", "lf_batch_set_stream", "lf_batch_add", "lf_batch_run",
                 "lf_batch_synchronize", "lf_batch_clear", "lf_batch_get_stats"):
        getattr(lib, name).restype = I
    lib.lf_triangulate.argtypes = [P, I, P, I]
    lib.lf_triangulate.restype = I
    lib.lf_host_alloc.argtypes = [ctypes.POINTER(P), ctypes.c_size_t]
    lib.lf_host_alloc.restype = I
    lib.lf_host_free.argtypes = [P]
    lib.lf_host_free.restype = None
    lib.lf_inject_alloc_failure.argtypes = [I]
    lib.lf_inject_alloc_failure.restype = None
    lib.lf_selftest_bounded_wait.argtypes = [ctypes.c_ulonglong]
    lib.lf_selftest_bounded_wait.restype = I
    for name in ("lf_create", "lf_create_calibrated", "lf_set_stream", "lf_set_inputs", "lf_run_em", "lf_synchronize",
                 "lf_get_prior", "lf_get_stats", "lf_set_timing"):
        getattr(lib, name).restype = I
    _lib = lib
    return lib


def default_support_params(**overrides) -> SupportParams:
    p = SupportParams()
    load().lf_default_support_params(ctypes.byref(p))
    for k, v in overrides.items():
        setattr(p, k, v)
    return p


def default_params(**overrides) -> Params:
    p = Params()
    load().lf_default_params(ctypes.byref(p))
    for k, v in overrides.items():
        setattr(p, k, v)
    return p


def _check(status: int):
    if status != LF_OK:
        msg = load().lf_last_error(None)
        raise LfError(status, msg.decode() if msg else "")


def selftest_bounded_wait(timeout_ns: int) -> int:
    """Run the device's bounded-wait self-test (one CTA waits for bytes no
    copy delivers); returns the status, LF_ETIMEOUT when the expiry was
    detected and reported."""
    return int(load().lf_selftest_bounded_wait(int(timeout_ns)))


def triangulate(points: np.ndarray) -> np.ndarray:
    """Delaunay triangles of the (u, v) of [M,3] points (host utility)."""
    pts = np.ascontiguousarray(points, np.float32).reshape(-1, 3)
    M = pts.shape[0]
    cap = max(2 * M + 8, 8)
    out = np.zeros((cap, 3), np.int32)
    n = load().lf_triangulate(pts.ctypes.data, M, out.ctypes.data, cap)
    if n < 0:
        raise LfError(LF_EINVAL, "invalid points")
    return out[:n].copy()


def run_em_static(baselines, d_min: float, d_max: float, D: int, iters: int, images, seg_prior, mu,
                  out: dict, params: Optional[Params] = None, stream=None) -> dict:
    """The allocation-free sweep on caller-owned torch CUDA tensors.

    images [K,H,W] / [K,H,W,3] uint8 or float32, seg_prior [K,H,W] float32,
    mu [H,W] float32 (NaN outside the triangulation); out holds preallocated
    tensors "d_idx" (int32, required) and optionally "d", "post", "labels".
    The library allocates nothing; the call waits for ``stream``."""
    import torch
    b = np.ascontiguousarray(baselines, np.float32)
    K, H, W = images.shape[:3]
    C = 1 if images.dim() == 3 else int(images.shape[3])
    dt = LF_U8 if images.dtype == torch.uint8 else LF_F32
    ptr = lambda k: out[k].data_ptr() if k in out else None
    handle = getattr(stream, "cuda_stream", stream)
    _check(load().lf_run_em_static(int(K), b.ctypes.data, int(H), int(W), float(d_min), float(d_max), int(D),
                                   ctypes.byref(params) if params is not None else None, int(iters),
                                   images.data_ptr(), C, dt, seg_prior.data_ptr(), mu.data_ptr(),
                                   ptr("d_idx"), ptr("d"), ptr("post"), ptr("labels"),
                                   ctypes.c_void_p(handle or 0)))
    return out


class HostArray(np.ndarray):
    """A numpy array over page-locked memory from lf_host_alloc (freed with
    the array), for the LF_HOST_ASYNC transfer mode."""

    def __array_finalize__(self, obj):
        if obj is not None and getattr(self, "_lf_block", None) is None:
            self._lf_block = getattr(obj, "_lf_block", None)


class _HostBlock:
    def __init__(self, nbytes: int):
        ptr = ctypes.c_void_p()
        _check(load().lf_host_alloc(ctypes.byref(ptr), max(int(nbytes), 1)))
        self.ptr = ptr.value

    def __del__(self):
        if getattr(self, "ptr", None):
            load().lf_host_free(ctypes.c_void_p(self.ptr))
            self.ptr = None


def host_array(shape, dtype) -> np.ndarray:
    """Page-locked host array allocated by the library (lf_host_alloc)."""
    dt = np.dtype(dtype)
    n = int(np.prod(shape)) * dt.itemsize
    blk = _HostBlock(n)
    buf = (ctypes.c_uint8 * max(n, 1)).from_address(blk.ptr)
    a = np.frombuffer(buf, dtype=dt, count=int(np.prod(shape))).reshape(shape).view(HostArray)
    a._lf_block = blk
    return a


def _is_torch(x) -> bool:
    return type(x).__module__.startswith("torch")


class Context:
    """One camera array / image size; owns the library's device buffers.
    ``cameras`` ([K,3,4]): a calibrated, non-rectified array (lf_create_calibrated);
    the baselines are then not used (may be None)."""

    def __init__(self, baselines, H: int, W: int, d_min: float, d_max: float, D: int,
                 params: Optional[Params] = None, stream=None, cameras=None):
        lib = load()
        self.H, self.W, self.D = int(H), int(W), int(D)
        h = ctypes.c_void_p()
        prm = ctypes.byref(params) if params is not None else None
        if cameras is not None:
            cams = np.ascontiguousarray(cameras, np.float32).reshape(-1, 3, 4)
            self.K = int(cams.shape[0])
            _check(lib.lf_create_calibrated(ctypes.byref(h), self.K, cams.ctypes.data, self.H, self.W,
                                            float(d_min), float(d_max), self.D, prm))
        else:
            self.K = len(baselines)
            b = np.ascontiguousarray(baselines, np.float32)
            _check(lib.lf_create(ctypes.byref(h), self.K, b.ctypes.data, self.H, self.W, float(d_min),
                                 float(d_max), self.D, prm))
        self._h = h
        self.C = None
        if stream is not None:
            self.set_stream(stream)

    # -- plumbing
    def set_stream(self, stream):
        """stream: a torch.cuda.Stream, a raw cudaStream_t integer, or None."""
        handle = getattr(stream, "cuda_stream", stream)
        _check(load().lf_set_stream(self._h, ctypes.c_void_p(handle or 0)))

    def close(self):
        if getattr(self, "_h", None):
            load().lf_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # -- the path
    def set_inputs(self, images, seg_prior, points, host_async: bool = False):
        """images [K,H,W] / [K,H,W,3] uint8, float32, float16 or bfloat16
        (the library reads each type as it is); seg_prior [K,H,W] float32
        P(dynamic); points [M,3] float32 (host), or None to detect the
        support points on the device (LF_DETECT_SUPPORT).  numpy arrays and
        CPU torch tensors are host inputs, torch CUDA tensors device inputs.
        host_async: host inputs copied asynchronously on the context's stream
        (LF_HOST_ASYNC); keep them unchanged until synchronize()."""
        detect = points is None
        pts = np.zeros((0, 3), np.float32) if detect else np.ascontiguousarray(points, np.float32).reshape(-1, 3)
        pptr = None if detect else pts.ctypes.data
        M = LF_DETECT_SUPPORT if detect else pts.shape[0]
        if _is_torch(images):
            import torch
            images = images.contiguous()
            C = 1 if images.dim() == 3 else int(images.shape[3])
            dt = {torch.uint8: LF_U8, torch.float32: LF_F32, torch.float16: LF_F16,
                  torch.bfloat16: LF_BF16}[images.dtype]
            if images.is_cuda:
                assert seg_prior.is_cuda and seg_prior.is_contiguous() and seg_prior.dtype == torch.float32
                self._keep = (images, seg_prior)
                _check(load().lf_set_inputs(self._h, images.data_ptr(), C, dt, seg_prior.data_ptr(), pptr, M, 1))
            else:  # host tensor: copied by the library within the call
                seg = np.ascontiguousarray(seg_prior.numpy() if _is_torch(seg_prior) else seg_prior, np.float32)
                _check(load().lf_set_inputs(self._h, images.data_ptr(), C, dt, seg.ctypes.data, pptr, M, 0))
        else:
            imgs = np.ascontiguousarray(images)
            dts = {np.dtype(np.uint8): LF_U8, np.dtype(np.float32): LF_F32, np.dtype(np.float16): LF_F16}
            if imgs.dtype not in dts:
                raise TypeError(f"images must be uint8, float32 or float16 (got {imgs.dtype}); "
                                "pass bfloat16 images as a torch tensor")
            C = 1 if imgs.ndim == 3 else int(imgs.shape[3])
            dt = dts[imgs.dtype]
            seg = np.ascontiguousarray(seg_prior, np.float32)
            if host_async:
                self._keep = (imgs, seg)
            _check(load().lf_set_inputs(self._h, imgs.ctypes.data, C, dt, seg.ctypes.data, pptr, M,
                                        LF_HOST_ASYNC if host_async else 0))
        self.C = C

    def run(self, iters: int, *, posteriors: bool = True, refocus: bool = True, disparity: bool = True,
            labels: bool = True, out: Optional[dict] = None, device: bool = False,
            host_async: bool = False) -> dict:
        """Run the hot path.  device=False: numpy outputs (the call waits).
        device=True: torch CUDA outputs written on the context's stream (pass
        preallocated tensors in ``out`` to avoid allocation).  host_async:
        numpy outputs in ``out`` (page-locked, e.g. host_array) written by
        asynchronous copies (LF_HOST_ASYNC); valid after synchronize()."""
        lib = load()
        K, H, W, C = self.K, self.H, self.W, self.C
        if C is None:
            raise LfError(LF_ESTATE, "set_inputs first")
        if device:
            import torch
            if out is None:
                dev = torch.device("cuda")
                out = {"d_idx": torch.empty((H, W), dtype=torch.int32, device=dev)}
                if disparity:
                    out["d"] = torch.empty((H, W), dtype=torch.float32, device=dev)
                if posteriors:
                    out["post"] = torch.empty((K, H, W), dtype=torch.float32, device=dev)
                if labels:
                    out["labels"] = torch.empty((H, W), dtype=torch.int16, device=dev)
                if refocus:
                    out["refocus"] = torch.empty((H, W, C) if C > 1 else (H, W), dtype=torch.float32, device=dev)
            ptr = lambda k: out[k].data_ptr() if k in out else None
            _check(lib.lf_run_em(self._h, int(iters), ptr("d_idx"), ptr("d"), ptr("post"), ptr("labels"),
                                 ptr("refocus"), 1))
            return out
        if out is not None:
            res = out
        else:
            res = {"d_idx": np.zeros((H, W), np.int32)}
            if disparity:
                res["d"] = np.zeros((H, W), np.float32)
            if posteriors:
                res["post"] = np.zeros((K, H, W), np.float32)
            if labels:
                res["labels"] = np.zeros((H, W), np.uint16)
            if refocus:
                res["refocus"] = np.zeros((H, W, C) if C > 1 else (H, W), np.float32)
        ptr = lambda k: res[k].ctypes.data if k in res else None
        _check(lib.lf_run_em(self._h, int(iters), ptr("d_idx"), ptr("d"), ptr("post"), ptr("labels"),
                             ptr("refocus"), LF_HOST_ASYNC if host_async else 0))
        return res

    def set_support_params(self, params: Optional[SupportParams] = None):
        _check(load().lf_set_support_params(self._h, ctypes.byref(params) if params is not None else None))

    def support_points(self) -> np.ndarray:
        """[M,3] (u, v, d) of the last detection."""
        n = ctypes.c_int(0)
        _check(load().lf_get_support_points(self._h, None, 0, ctypes.byref(n)))
        out = np.zeros((n.value, 3), np.float32)
        if n.value:
            _check(load().lf_get_support_points(self._h, out.ctypes.data, n.value, ctypes.byref(n)))
        return out

    def set_tile(self, tile_rows: int, tile_cols: int):
        _check(load().lf_set_tile(self._h, int(tile_rows), int(tile_cols)))

    def set_timing(self, enable: bool = True):
        _check(load().lf_set_timing(self._h, int(enable)))

    def synchronize(self):
        _check(load().lf_synchronize(self._h))

    def prior(self) -> np.ndarray:
        mu = np.zeros((self.H, self.W), np.float32)
        _check(load().lf_get_prior(self._h, mu.ctypes.data, 0))
        return mu

    def stats(self) -> dict:
        s = Stats()
        _check(load().lf_get_stats(self._h, ctypes.byref(s)))
        return {f: getattr(s, f) for f, _ in Stats._fields_}


class Batch:
    """Uneven batch of frames on device buffers (torch CUDA tensors), run as
    one CUDA graph (see lf_batch_* in include/lf.h)."""

    def __init__(self, params: Optional[Params] = None, stream=None, autotune: bool = False):
        h = ctypes.c_void_p()
        _check(load().lf_batch_create(ctypes.byref(h), ctypes.byref(params) if params is not None else None,
                                      int(autotune)))
        self._h = h
        self._keep = []
        if stream is not None:
            self.set_stream(stream)

    def set_stream(self, stream):
        handle = getattr(stream, "cuda_stream", stream)
        _check(load().lf_batch_set_stream(self._h, ctypes.c_void_p(handle or 0)))

    def add(self, baselines, d_min, d_max, D, iters, images, seg_prior, points, out: dict) -> int:
        """images / seg_prior: torch CUDA tensors; out: preallocated torch
        CUDA tensors ("d_idx" required; "d", "post", "labels", "refocus")."""
        import torch
        b = np.ascontiguousarray(baselines, np.float32)
        pts = np.ascontiguousarray(points, np.float32).reshape(-1, 3)
        K, H, W = images.shape[:3]
        C = 1 if images.dim() == 3 else int(images.shape[3])
        dt = {torch.uint8: LF_U8, torch.float32: LF_F32, torch.float16: LF_F16, torch.bfloat16: LF_BF16}[images.dtype]
        ptr = lambda k: out[k].data_ptr() if k in out else None
        idx = ctypes.c_int(-1)
        _check(load().lf_batch_add(self._h, int(K), b.ctypes.data, int(H), int(W), float(d_min), float(d_max),
                                   int(D), int(iters), images.data_ptr(), C, dt, seg_prior.data_ptr(),
                                   pts.ctypes.data, pts.shape[0], ptr("d_idx"), ptr("d"), ptr("post"),
                                   ptr("labels"), ptr("refocus"), ctypes.byref(idx)))
        self._keep.append((images, seg_prior, out))
        return idx.value

    def run(self):
        _check(load().lf_batch_run(self._h))

    def synchronize(self):
        _check(load().lf_batch_synchronize(self._h))

    def clear(self):
        _check(load().lf_batch_clear(self._h))
        self._keep = []

    def stats(self) -> dict:
        s = Stats()
        _check(load().lf_batch_get_stats(self._h, ctypes.byref(s)))
        return {f: getattr(s, f) for f, _ in Stats._fields_}

    def close(self):
        if getattr(self, "_h", None):
            load().lf_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def device_outputs(K: int, H: int, W: int, C: int, device=None) -> dict:
    """Preallocated torch CUDA output tensors for one frame."""
    import torch
    dev = device or torch.device("cuda")
    return {"d_idx": torch.empty((H, W), dtype=torch.int32, device=dev),
            "d": torch.empty((H, W), dtype=torch.float32, device=dev),
            "post": torch.empty((K, H, W), dtype=torch.float32, device=dev),
            "labels": torch.empty((H, W), dtype=torch.int16, device=dev),
            "refocus": torch.empty((H, W, C) if C > 1 else (H, W), dtype=torch.float32, device=dev)}


def run_scene(scene, params: Optional[Params] = None, iters: Optional[int] = None,
              support: Optional[SupportParams] = None, detect_support: bool = False, **kw) -> dict:
    """Convenience: one frame of a ``scenes.Scene`` through host buffers.
    detect_support: support points detected on the device instead of the
    scene's points (``support`` = their parameters)."""
    with Context(scene.baselines, scene.H, scene.W, scene.d_min, scene.d_max, scene.D, params,
                 cameras=getattr(scene, "cameras", None)) as ctx:
        if support is not None:
            ctx.set_support_params(support)
        ctx.set_inputs(scene.images, scene.seg_prior, None if detect_support else scene.points)
        if detect_support:
            out_pts = ctx.support_points()
        out = ctx.run(scene.iters if iters is None else iters, **kw)
        out["stats"] = ctx.stats()
        out["mu"] = ctx.prior()
        if detect_support:
            out["support_points"] = out_pts
    return out
