"""FP64 CPU oracle: Python driver for the C core plus the triangulation prior.

TEST INFRASTRUCTURE ONLY.  Only the tests, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline / reference leg may import this module.  It shares
no code with the CUDA path and imports nothing from the library package.

Pieces:

* ``prior_raster`` -- the piecewise-planar disparity prior (Sec. III-C
  "Disparity Prior"): a Delaunay triangulation of the sparse support points
  (scipy's Qhull as the library primitive) and, per integer pixel centre, the
  barycentric interpolation of the vertex disparities in the triangle that
  contains it.  Containment uses double-precision orientation tests with
  "on an edge" counting as inside; pixels in no triangle are outside the
  prior (uniform).  Repeated (u, v) positions keep their first occurrence.
* ``run`` -- the per-pixel EM, features, posteriors and refocus (the C core,
  ``lf_oracle.c``; see its header for the step-by-step statement).
* ``median3`` -- the 3x3 median of Sec. III-E.
"""
from __future__ import annotations

import ctypes
import dataclasses
import os
import subprocess
from typing import Optional

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "lf_oracle.c")
SUPPORT_SRC = os.path.join(HERE, "support_oracle.c")
BUILD_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD_DIR, "liblf_oracle.so")


@dataclasses.dataclass
class Params:
    """Model constants (the paper names beta, gamma, sigma and the 0.7
    threshold but prints values only for the threshold; the others are
    runtime parameters with these defaults)."""

    beta: float = 200.0
    gamma: float = 0.1
    sigma: float = 2.0
    seg_threshold: float = 0.7
    eps: float = 1e-4
    mstep_seg_term: int = 1
    em_mode: int = 0          # 0 hard EM (the paper's), 1 soft EM, 2 joint MAP


class _CParams(ctypes.Structure):
    _fields_ = [("beta", ctypes.c_double), ("gamma", ctypes.c_double), ("sigma", ctypes.c_double),
                ("seg_threshold", ctypes.c_double), ("eps", ctypes.c_double),
                ("mstep_seg_term", ctypes.c_int), ("em_mode", ctypes.c_int)]


@dataclasses.dataclass
class SupportParams:
    """Support-point detection (see support_oracle.c for the reading)."""

    grid: int = 5
    ratio_pct: int = 85
    texture: int = 120
    window: int = 3
    delta: float = 3.0
    min_support: int = 2
    seg_threshold: float = 0.7


class _CSupport(ctypes.Structure):
    _fields_ = [("grid", ctypes.c_int), ("ratio_pct", ctypes.c_int), ("texture", ctypes.c_int),
                ("window", ctypes.c_int), ("delta", ctypes.c_double), ("min_support", ctypes.c_int),
                ("seg_threshold", ctypes.c_float)]


def build(force: bool = False) -> str:
    """Compile the C core with gcc (OpenMP when available).  FP contraction is
    off so that x86 and Arm builds round identically."""
    os.makedirs(BUILD_DIR, exist_ok=True)
    if not force and os.path.exists(LIB) and all(os.path.getmtime(LIB) >= os.path.getmtime(s)
                                                  for s in (SRC, SUPPORT_SRC)):
        return LIB
    base = ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared", SRC, SUPPORT_SRC,
            "-o", LIB + ".tmp", "-lm"]
    try:
        subprocess.run(base[:1] + ["-fopenmp"] + base[1:], check=True, capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base, check=True, capture_output=True)
    os.replace(LIB + ".tmp", LIB)
    return LIB


_lib = None


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        P = ctypes.c_void_p
        lib.orc_run.restype = ctypes.c_int
        lib.orc_run.argtypes = [ctypes.c_int, P, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                P, P, P, P, ctypes.c_float, ctypes.c_float, ctypes.c_int, ctypes.c_int,
                                ctypes.POINTER(_CParams), ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                P, P, P, P, P, P, P, P, P]
        lib.orc_run_general.restype = ctypes.c_int
        lib.orc_run_general.argtypes = lib.orc_run.argtypes
        lib.orc_support_points.restype = ctypes.c_int
        lib.orc_support_points.argtypes = [ctypes.c_int, P, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                           P, P, ctypes.c_float, ctypes.c_float, ctypes.c_int,
                                           ctypes.POINTER(_CSupport), P, P, P, P]
        lib.orc_max_threads.restype = ctypes.c_int
        lib.orc_objective_at.restype = ctypes.c_double
        lib.orc_objective_at.argtypes = [ctypes.c_int, P, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                         P, P, ctypes.POINTER(_CParams), ctypes.c_int, ctypes.c_int,
                                         ctypes.c_double, ctypes.c_double, ctypes.c_int, ctypes.c_uint,
                                         ctypes.c_int]
        lib.orc_features.argtypes = [ctypes.c_int] * 5 + [P, P]
        lib.orc_median3.argtypes = [ctypes.c_int] * 3 + [P, P]
        lib.orc_sample.restype = ctypes.c_double
        lib.orc_sample.argtypes = [P, ctypes.c_int, ctypes.c_double]
        _lib = lib
    return _lib


def _ptr(a: np.ndarray):
    return ctypes.c_void_p(a.ctypes.data)


def _cparams(p: Optional[Params]) -> _CParams:
    p = p or Params()
    return _CParams(p.beta, p.gamma, p.sigma, p.seg_threshold, p.eps, p.mstep_seg_term, p.em_mode)


def max_threads() -> int:
    return int(_load().orc_max_threads())


# --------------------------------------------------------------- the prior

def _orient(ax, ay, bx, by, px, py):
    """Twice the signed area of (a, b, p); > 0 when p is left of a->b."""
    return (bx - ax) * (py - ay) - (by - ay) * (px - ax)


def triangulate(points: np.ndarray) -> np.ndarray:
    """Delaunay triangles (index triples into the de-duplicated point list,
    counter-clockwise) of the (u, v) support points, plus the kept points.
    Returns (tris [T,3] int, pts [M',3] float64)."""
    pts = np.asarray(points, np.float64).reshape(-1, 3)
    if pts.shape[0] == 0:
        return np.zeros((0, 3), np.int64), pts
    _, first = np.unique(pts[:, :2], axis=0, return_index=True)
    pts = pts[np.sort(first)]
    if pts.shape[0] < 3:
        return np.zeros((0, 3), np.int64), pts
    from scipy.spatial import Delaunay, QhullError
    try:
        tri = Delaunay(pts[:, :2])
    except QhullError:
        return np.zeros((0, 3), np.int64), pts
    t = tri.simplices.astype(np.int64)
    a, b, c = pts[t[:, 0]], pts[t[:, 1]], pts[t[:, 2]]
    area = _orient(a[:, 0], a[:, 1], b[:, 0], b[:, 1], c[:, 0], c[:, 1])
    t = t[area != 0.0]
    flip = _orient(pts[t[:, 0], 0], pts[t[:, 0], 1], pts[t[:, 1], 0], pts[t[:, 1], 1],
                   pts[t[:, 2], 0], pts[t[:, 2], 1]) < 0
    t[flip] = t[flip][:, [0, 2, 1]]
    return t, pts


def prior_raster(points: np.ndarray, H: int, W: int):
    """Per-pixel interpolated disparity mu [H,W] (float64) and inside flag
    [H,W] (uint8) of the piecewise-planar prior (Sec. III-C)."""
    mu = np.zeros((H, W), np.float64)
    inside = np.zeros((H, W), np.uint8)
    tris, pts = triangulate(points)
    for t in tris:
        a, b, c = pts[t[0]], pts[t[1]], pts[t[2]]
        u0 = max(0, int(np.ceil(min(a[0], b[0], c[0]))))
        u1 = min(W - 1, int(np.floor(max(a[0], b[0], c[0]))))
        v0 = max(0, int(np.ceil(min(a[1], b[1], c[1]))))
        v1 = min(H - 1, int(np.floor(max(a[1], b[1], c[1]))))
        if u1 < u0 or v1 < v0:
            continue
        vv, uu = np.meshgrid(np.arange(v0, v1 + 1, dtype=np.float64),
                             np.arange(u0, u1 + 1, dtype=np.float64), indexing="ij")
        la = _orient(b[0], b[1], c[0], c[1], uu, vv)
        lb = _orient(c[0], c[1], a[0], a[1], uu, vv)
        lc = _orient(a[0], a[1], b[0], b[1], uu, vv)
        hit = (la >= 0) & (lb >= 0) & (lc >= 0)
        sub_in = inside[v0:v1 + 1, u0:u1 + 1]
        new = hit & (sub_in == 0)
        if not new.any():
            continue
        s = la + lb + lc
        val = (la * a[2] + lb * b[2] + lc * c[2]) / s
        mu[v0:v1 + 1, u0:u1 + 1][new] = val[new]
        sub_in[new] = 1
    return mu, inside


# ------------------------------------------------------------------ the EM

def run(images: np.ndarray, seg_prior: np.ndarray, baselines: np.ndarray, points: np.ndarray,
        d_min: float, d_max: float, D: int, iters: int, params: Optional[Params] = None,
        rows: Optional[tuple] = None, threads: int = 0, mu=None, inside=None, cameras=None) -> dict:
    """Run the oracle on one frame.

    images: [K,H,W] or [K,H,W,C] uint8 (scaled 1/255) or float32 in [0,1].
    seg_prior: [K,H,W] P(dynamic).  baselines: [K], one entry 0.
    rows: optional (begin, end) subset of rows (other rows stay zero).
    cameras: optional [K,3,4] matrices of a calibrated array (Eq. 1 in
    generalized disparity space); then the baselines are not used.
    """
    lib = _load()
    imgs = np.ascontiguousarray(images)
    if imgs.dtype == np.uint8:
        dtype = 0
    elif imgs.dtype == np.float32:
        dtype = 1
    else:
        raise TypeError("images must be uint8 or float32")
    K, H, W = imgs.shape[:3]
    C = 1 if imgs.ndim == 3 else imgs.shape[3]
    seg = np.ascontiguousarray(seg_prior, dtype=np.float32)
    b = np.ascontiguousarray(baselines, dtype=np.float32)
    if mu is None:
        mu, inside = prior_raster(points, H, W)
    mu = np.ascontiguousarray(mu, np.float64)
    inside = np.ascontiguousarray(inside, np.uint8)
    r0, r1 = (0, H) if rows is None else rows
    out = {
        "d_idx": np.zeros((H, W), np.int32),
        "d": np.zeros((H, W), np.float64),
        "labels": np.zeros((H, W), np.uint16),
        "post": np.zeros((K, H, W), np.float64),
        "refocus": np.zeros((H, W, C), np.float64),
        "m_margin": np.zeros((iters, H, W), np.float64),
        "e_margin": np.zeros((iters, H, W), np.float64),
        "J_t": np.zeros((iters, H, W), np.float64),
        "init_margin": np.zeros((H, W), np.float64),
    }
    cp = _cparams(params)
    if cameras is not None:
        cams = np.ascontiguousarray(cameras, dtype=np.float32).reshape(K, 3, 4)
        fn, geo = lib.orc_run_general, cams
    else:
        fn, geo = lib.orc_run, b
    rc = fn(K, _ptr(geo), H, W, C, dtype, _ptr(imgs), _ptr(seg), _ptr(mu), _ptr(inside),
                     float(d_min), float(d_max), int(D), int(iters), ctypes.byref(cp), int(r0), int(r1),
                     int(threads), _ptr(out["d_idx"]), _ptr(out["d"]), _ptr(out["labels"]),
                     _ptr(out["post"]), _ptr(out["refocus"]), _ptr(out["m_margin"]),
                     _ptr(out["e_margin"]), _ptr(out["J_t"]), _ptr(out["init_margin"]))
    if rc != 0:
        raise ValueError("oracle rejected the arguments")
    if C == 1:
        out["refocus"] = out["refocus"][..., 0]
    out["mu"], out["inside"] = mu, inside
    return out


def run_scene(scene, params: Optional[Params] = None, rows=None, threads: int = 0, iters=None) -> dict:
    return run(scene.images, scene.seg_prior, scene.baselines, scene.points, scene.d_min, scene.d_max,
               scene.D, scene.iters if iters is None else iters, params, rows, threads,
               cameras=getattr(scene, "cameras", None))


def support_points(images, seg_prior, baselines, d_min: float, d_max: float, D: int,
                   params: Optional[SupportParams] = None) -> dict:
    """Support points of the disparity prior (Sec. III-C).  Returns the
    per-cell arrays (cell_j: candidate index or -1, cell_src: source camera,
    cell_u / cell_v: reference coordinates) and ``points`` [M,3] (u, v, d) in
    cell raster order."""
    lib = _load()
    sp = params or SupportParams()
    imgs = np.ascontiguousarray(images)
    dtype = 0 if imgs.dtype == np.uint8 else 1
    if dtype == 1 and imgs.dtype != np.float32:
        imgs = imgs.astype(np.float32)
    K, H, W = imgs.shape[:3]
    C = 1 if imgs.ndim == 3 else imgs.shape[3]
    seg = np.ascontiguousarray(seg_prior, np.float32)
    b = np.ascontiguousarray(baselines, np.float32)
    nx, ny = (W + sp.grid - 1) // sp.grid, (H + sp.grid - 1) // sp.grid
    out = {"cell_j": np.zeros((ny, nx), np.int32), "cell_src": np.zeros((ny, nx), np.int32),
           "cell_u": np.zeros((ny, nx), np.float64), "cell_v": np.zeros((ny, nx), np.float64)}
    cs = _CSupport(sp.grid, sp.ratio_pct, sp.texture, sp.window, sp.delta, sp.min_support, sp.seg_threshold)
    n = lib.orc_support_points(K, _ptr(b), H, W, C, dtype, _ptr(imgs), _ptr(seg), float(d_min), float(d_max),
                               int(D), ctypes.byref(cs), _ptr(out["cell_j"]), _ptr(out["cell_src"]),
                               _ptr(out["cell_u"]), _ptr(out["cell_v"]))
    if n < 0:
        raise ValueError("oracle rejected the arguments")
    dval = np.array([float(d_min)] if D == 1 else
                    [float(d_min) + j * ((float(d_max) - float(d_min)) / (D - 1)) for j in range(D)])
    m = out["cell_j"] >= 0
    # points sit at their cell's position plus a fixed sub-pixel offset per
    # cell (at most 0.01 px) that keeps grid points off common circles: the
    # Delaunay triangulation of the prior is then unique
    cj, ci = np.nonzero(m)
    ju = 0.01 * ((7 * ci + 13 * cj) % 17 + 1).astype(np.float64) / 18.0
    jv = 0.01 * ((11 * ci + 5 * cj) % 19 + 1).astype(np.float64) / 20.0
    out["points"] = np.stack([out["cell_u"][m] + ju, out["cell_v"][m] + jv, dval[out["cell_j"][m]]], 1)
    assert out["points"].shape[0] == n
    return out


def features(images: np.ndarray) -> np.ndarray:
    """[K,3,H,W] descriptor maps [Y, Sobel-x/8, Sobel-y/8] (float64)."""
    lib = _load()
    imgs = np.ascontiguousarray(images)
    dtype = 0 if imgs.dtype == np.uint8 else 1
    K, H, W = imgs.shape[:3]
    C = 1 if imgs.ndim == 3 else imgs.shape[3]
    out = np.zeros((K, 3, H, W), np.float64)
    lib.orc_features(K, H, W, C, dtype, _ptr(imgs), _ptr(out))
    return out


def objective_at(images, seg_prior, baselines, u, v, d, S, mu=0.0, inside=0, params=None,
                 with_seg=1) -> float:
    """J(d, S) of pixel (u, v) (complete-data objective)."""
    lib = _load()
    imgs = np.ascontiguousarray(images)
    dtype = 0 if imgs.dtype == np.uint8 else 1
    K, H, W = imgs.shape[:3]
    C = 1 if imgs.ndim == 3 else imgs.shape[3]
    seg = np.ascontiguousarray(seg_prior, dtype=np.float32)
    b = np.ascontiguousarray(baselines, dtype=np.float32)
    cp = _cparams(params)
    return float(lib.orc_objective_at(K, _ptr(b), H, W, C, dtype, _ptr(imgs), _ptr(seg), ctypes.byref(cp),
                                      int(u), int(v), float(d), float(mu), int(inside), int(S), int(with_seg)))


def sample(row: np.ndarray, x: float) -> float:
    """Clamp-to-edge linear sample of a 1-D row at continuous position x."""
    r = np.ascontiguousarray(row, np.float64)
    return float(_load().orc_sample(_ptr(r), int(r.shape[0]), float(x)))


def median3(img: np.ndarray) -> np.ndarray:
    """3x3 per-channel median, border replicated (Sec. III-E)."""
    lib = _load()
    a = np.ascontiguousarray(img, np.float64)
    squeeze = a.ndim == 2
    if squeeze:
        a = a[..., None]
    H, W, C = a.shape
    out = np.zeros_like(a)
    lib.orc_median3(H, W, C, _ptr(a), _ptr(out))
    return out[..., 0] if squeeze else out


def excused(out: dict, tau_rel: float = 1e-4, tau_init: float = 1e-5) -> np.ndarray:
    """Pixels whose result the oracle itself cannot decide robustly: an M- or
    E-step arg-max margin below tau_rel * (1 + |J|) at any iteration, or an
    initial-threshold sample within tau_init of the 0.7 threshold."""
    J = np.abs(out["J_t"])
    tau = tau_rel * (1.0 + J)
    bad = np.any(out["m_margin"] < tau, axis=0) | np.any(out["e_margin"] < tau, axis=0)
    return bad | (out["init_margin"] < tau_init)
