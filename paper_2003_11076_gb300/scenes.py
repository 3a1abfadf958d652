"""Seeded synthetic light-field scenes for a rectified linear camera array.

This module renders inputs only. It holds none of the method's arithmetic (no
features, variances, priors or EM steps); both the CUDA path and the FP64 oracle
consume what it produces.

Geometry (Sec. III-A, Eq. 1 specialised to a rectified linear array): a
fronto-parallel surface at disparity ``d`` seen at reference column ``u``
appears in camera ``k`` at column ``u - d * b_k`` on the same row, where
``b_k`` is camera k's signed position relative to the reference camera
(``b_ref = 0``).  Rendering inverts that map: view pixel ``(u_k, v)`` shows the
nearest surface whose reference-coordinate footprint contains
``(u_k + d * b_k, v)``.

Scenes are layered: static textured planes (the background the method must
recover) and "dynamic" occluders (the people the segmentation prior flags).
Per view the generator returns the image, the segmentation prior
P(dynamic), and, for the reference view, the ground-truth static disparity and
the static image that refocusing should recover.

Workloads (seed = workload id * 1000 + frame index):

* ``small_gray`` -- 5 cameras at 0, +-0.1, +-0.2, 64x48 gray float32, planes
  at disparity 4 and 9 with value-noise texture, one occluder at disparity 20
  with per-pixel uniform-noise texture drawn only in the three central views,
  Gaussian noise 0.01, P = 0.9 / 0.05 +- U(0.03), 40 sparse points with
  N(0, 0.3^2) disparity noise, D = 32 (0..31), 5 EM iterations.
* ``street_rgb`` -- 5 cameras at 0, +-0.1, +-0.2, 960x600 RGB uint8, three
  depth planes, 1-4 person-sized boxes covering 10-35 % of the reference view
  that move between views by parallax only, P ~ Beta(8,2) on occluder pixels
  and Beta(1,15) elsewhere, 300 sparse points with N(0, 0.5^2) noise,
  D = 64 (0..63), 10 EM iterations.
* ``random_frame`` -- the uneven-batch / serving generator: size, camera
  count, baselines and D drawn from a seeded generator, scene as small_gray.
"""
from __future__ import annotations

import dataclasses
from typing import List, Optional, Sequence

import numpy as np

__all__ = [
    "Surface",
    "Scene",
    "value_noise",
    "render_scene",
    "small_gray",
    "street_rgb",
    "random_frame",
    "plane_scene",
    "calibrated_cameras",
]


# --------------------------------------------------------------------------
# procedural textures (Perlin-style value noise, written for this project)
# --------------------------------------------------------------------------

def _fade(t: np.ndarray) -> np.ndarray:
    return t * t * (3.0 - 2.0 * t)


def value_noise(rng: np.random.Generator, cells: Sequence[float], weights: Sequence[float],
                extent: tuple, lo: float = 0.1, hi: float = 0.9):
    """Return ``tex(u, v)``: a sum of smoothly interpolated random lattices.

    ``cells`` are lattice spacings in pixels, ``weights`` their amplitudes and
    ``extent`` = (u0, v0, u1, v1) the reference-coordinate box the texture must
    cover (with a margin).  Values are mapped affinely into [lo, hi].
    """
    u0, v0, u1, v1 = extent
    lattices = []
    for c in cells:
        nu = int(np.ceil((u1 - u0) / c)) + 3
        nv = int(np.ceil((v1 - v0) / c)) + 3
        lattices.append(rng.random((nv, nu)))
    wsum = float(np.sum(weights))

    def tex(u: np.ndarray, v: np.ndarray) -> np.ndarray:
        out = np.zeros(np.broadcast(u, v).shape, dtype=np.float64)
        for c, w, g in zip(cells, weights, lattices):
            x = (np.asarray(u, np.float64) - u0) / c + 1.0
            y = (np.asarray(v, np.float64) - v0) / c + 1.0
            x = np.clip(x, 0.0, g.shape[1] - 1.000001)
            y = np.clip(y, 0.0, g.shape[0] - 1.000001)
            ix = np.floor(x).astype(np.int64)
            iy = np.floor(y).astype(np.int64)
            fx = _fade(x - ix)
            fy = _fade(y - iy)
            a = g[iy, ix] * (1 - fx) + g[iy, ix + 1] * fx
            b = g[iy + 1, ix] * (1 - fx) + g[iy + 1, ix + 1] * fx
            out += w * (a * (1 - fy) + b * fy)
        return lo + (hi - lo) * out / wsum

    return tex


def pixel_noise(rng: np.random.Generator, extent: tuple, lo: float = 0.0, hi: float = 1.0):
    """Return ``tex(u, v)``: i.i.d. uniform values on the unit pixel lattice
    (nearest-cell lookup), i.e. an uncorrelated per-pixel noise texture."""
    u0, v0, u1, v1 = extent
    nu = int(np.ceil(u1 - u0)) + 2
    nv = int(np.ceil(v1 - v0)) + 2
    g = lo + (hi - lo) * rng.random((nv, nu))

    def tex(u: np.ndarray, v: np.ndarray) -> np.ndarray:
        x = np.clip(np.floor(np.asarray(u, np.float64) - u0 + 1e-9).astype(np.int64), 0, nu - 1)
        y = np.clip(np.floor(np.asarray(v, np.float64) - v0 + 1e-9).astype(np.int64), 0, nv - 1)
        return g[y, x]

    return tex


# --------------------------------------------------------------------------
# layered scene model
# --------------------------------------------------------------------------

@dataclasses.dataclass
class Surface:
    """A fronto-parallel rectangle in reference coordinates.

    ``rect`` = (u0, v0, u1, v1), half-open, or ``None`` for "everywhere".
    ``tex`` maps reference coordinates to one value per channel (a list of
    C callables).  ``dynamic`` surfaces are occluders flagged by the prior;
    ``views`` restricts in which cameras a dynamic surface is drawn
    (``None`` = all, moving by parallax only).
    """

    disparity: float
    rect: Optional[tuple]
    tex: list
    dynamic: bool = False
    views: Optional[Sequence[int]] = None

    def covers(self, u: np.ndarray, v: np.ndarray) -> np.ndarray:
        if self.rect is None:
            return np.ones(np.broadcast(u, v).shape, dtype=bool)
        u0, v0, u1, v1 = self.rect
        return (u >= u0) & (u < u1) & (v >= v0) & (v < v1)


@dataclasses.dataclass
class Scene:
    """Inputs and ground truth of one light-field frame."""

    name: str
    seed: int
    baselines: np.ndarray        # [K] float32, one entry exactly 0
    images: np.ndarray           # [K,H,W] float32 in [0,1]  or  [K,H,W,3] uint8
    seg_prior: np.ndarray        # [K,H,W] float32, P(dynamic)
    points: np.ndarray           # [M,3] float32 (u, v, d) in the reference view
    d_min: float
    d_max: float
    D: int
    iters: int
    gt_disparity: np.ndarray     # [H,W] float32, static background in the ref view
    gt_static: np.ndarray        # [H,W] or [H,W,3] float32 in [0,1]
    dynamic_mask: np.ndarray     # [K,H,W] bool, pixels showing a dynamic surface
    halo: int = 0                # border (px) affected by rays leaving the image
    cameras: Optional[np.ndarray] = None  # [K,3,4] calibrated (non-rectified) array, else None

    @property
    def K(self) -> int:
        return int(self.baselines.shape[0])

    @property
    def H(self) -> int:
        return int(self.images.shape[1])

    @property
    def W(self) -> int:
        return int(self.images.shape[2])

    @property
    def C(self) -> int:
        return 1 if self.images.ndim == 3 else int(self.images.shape[3])

    @property
    def ref(self) -> int:
        return int(np.flatnonzero(self.baselines == 0)[0])

    @property
    def nominal_ray_samples(self) -> int:
        return self.H * self.W * self.K * self.D * self.iters


def _ref_coords(cam: np.ndarray, d: float, uu: np.ndarray, vv: np.ndarray):
    """Reference coordinates of the point at disparity d that the calibrated
    camera ``cam`` (3x4, (u, v, 1, d) -> homogeneous pixel) sees at (uu, vv):
    the inverse of the homography of the plane at disparity d."""
    G = np.asarray(cam, np.float64)[:, :3].copy()
    G[:, 2] += d * np.asarray(cam, np.float64)[:, 3]
    Gi = np.linalg.inv(G)
    X = Gi[0, 0] * uu + Gi[0, 1] * vv + Gi[0, 2]
    Y = Gi[1, 0] * uu + Gi[1, 1] * vv + Gi[1, 2]
    Z = Gi[2, 0] * uu + Gi[2, 1] * vv + Gi[2, 2]
    return X / Z, Y / Z


def calibrated_cameras(rng: np.random.Generator, baselines, H: int, W: int, rot_deg: float = 0.6,
                       shift_y: float = 0.02, shift_z: float = 0.03, focal_jitter: float = 0.01) -> np.ndarray:
    """[K,3,4] camera matrices of a calibrated, non-rectified array in
    generalized disparity space (Eq. 1): camera k at (b_k, ty, tz) relative
    to the reference with a small random rotation and its own intrinsics, so
    that a reference pixel (u, v) at disparity d = f / depth appears at
    M_k (u, v, 1, d).  The reference matrix is exactly [I | 0]; with no
    rotation, equal intrinsics and ty = tz = 0 the matrix reduces to the
    rectified shift u - d b_k."""
    b = np.asarray(baselines, np.float64)
    f = 1.2 * W
    Kr = np.array([[f, 0.0, (W - 1) / 2.0], [0.0, f, (H - 1) / 2.0], [0.0, 0.0, 1.0]])
    Kr_inv = np.linalg.inv(Kr)
    out = np.zeros((len(b), 3, 4))
    for k, bk in enumerate(b):
        if bk == 0.0:
            out[k, :, :3] = np.eye(3)
            continue
        fk = f * (1.0 + rng.uniform(-focal_jitter, focal_jitter))
        Kk = np.array([[fk, 0.0, (W - 1) / 2.0 + rng.uniform(-1, 1)],
                       [0.0, fk, (H - 1) / 2.0 + rng.uniform(-1, 1)], [0.0, 0.0, 1.0]])
        ax, ay, az = np.deg2rad(rng.uniform(-rot_deg, rot_deg, size=3))
        Rx = np.array([[1, 0, 0], [0, np.cos(ax), -np.sin(ax)], [0, np.sin(ax), np.cos(ax)]])
        Ry = np.array([[np.cos(ay), 0, np.sin(ay)], [0, 1, 0], [-np.sin(ay), 0, np.cos(ay)]])
        Rz = np.array([[np.cos(az), -np.sin(az), 0], [np.sin(az), np.cos(az), 0], [0, 0, 1]])
        t = np.array([-bk, rng.uniform(-shift_y, shift_y), rng.uniform(-shift_z, shift_z)])
        out[k, :, :3] = Kk @ (Rz @ Ry @ Rx) @ Kr_inv
        out[k, :, 3] = Kk @ t / f
    return out.astype(np.float32)


def render_scene(surfaces: List[Surface], baselines: np.ndarray, H: int, W: int, C: int, cameras=None):
    """Render every view by parallax (or, with ``cameras``, through the
    inverse plane homographies of a calibrated array).

    Returns (images [K,H,W,C] float64, dynamic mask [K,H,W], static reference
    image [H,W,C], static reference disparity [H,W]).
    """
    K = len(baselines)
    order = sorted(range(len(surfaces)), key=lambda i: -surfaces[i].disparity)
    vv, uu = np.meshgrid(np.arange(H, dtype=np.float64), np.arange(W, dtype=np.float64), indexing="ij")
    images = np.zeros((K, H, W, C))
    dyn = np.zeros((K, H, W), dtype=bool)
    ref = int(np.flatnonzero(np.asarray(baselines) == 0)[0])
    st_img = np.zeros((H, W, C))
    st_disp = np.zeros((H, W))
    for k in range(K):
        done = np.zeros((H, W), dtype=bool)
        st_done = np.zeros((H, W), dtype=bool)
        for i in order:
            s = surfaces[i]
            if cameras is None:
                ur, vr = uu + s.disparity * float(baselines[k]), vv
            else:
                ur, vr = _ref_coords(cameras[k], s.disparity, uu, vv)
            hit = s.covers(ur, vr)
            drawn = s.views is None or k in s.views
            if drawn:
                m = hit & ~done
                if m.any():
                    for c in range(C):
                        images[k, :, :, c][m] = s.tex[c](ur[m], vr[m])
                    dyn[k][m] = s.dynamic
                    done |= m
            if k == ref and not s.dynamic:
                m = hit & ~st_done
                if m.any():
                    for c in range(C):
                        st_img[:, :, c][m] = s.tex[c](ur[m], vr[m])
                    st_disp[m] = s.disparity
                    st_done |= m
        assert done.all(), "scene must have a background surface covering every ray"
    return images, dyn, st_img, st_disp


def _static_disparity_at(surfaces: List[Surface], u: np.ndarray, v: np.ndarray) -> np.ndarray:
    """Disparity of the nearest static surface at continuous ref coords."""
    out = np.full(u.shape, np.nan)
    for s in sorted(surfaces, key=lambda s: -s.disparity):
        if s.dynamic:
            continue
        m = s.covers(u, v) & np.isnan(out)
        out[m] = s.disparity
    return out


def _sparse_points(rng, surfaces, H, W, M, sigma):
    """Support points: continuous (u, v) uniform over the reference image with
    the static background disparity there plus Gaussian noise.  Points on
    dynamic objects are dropped and the background behind them is observed
    from other views (Sec. III-C), which this stands in for."""
    u = rng.uniform(0.0, W - 1.0, size=M)
    v = rng.uniform(0.0, H - 1.0, size=M)
    d = _static_disparity_at(surfaces, u, v) + rng.normal(0.0, sigma, size=M)
    return np.stack([u, v, d], axis=1).astype(np.float32)


def _finish(name, seed, rng, surfaces, baselines, H, W, C, u8, noise, prior_fn,
            M, point_sigma, d_min, d_max, D, iters, cameras=None):
    images, dyn, st_img, st_disp = render_scene(surfaces, baselines, H, W, C, cameras)
    if noise > 0:
        images = images + rng.normal(0.0, noise, size=images.shape)
    images = np.clip(images, 0.0, 1.0)
    if u8:
        images_out = np.clip(np.rint(images * 255.0), 0, 255).astype(np.uint8)
    else:
        images_out = images.astype(np.float32)
    if C == 1:
        images_out = images_out[..., 0]
        st_img = st_img[..., 0]
    seg = prior_fn(rng, dyn).astype(np.float32)
    pts = _sparse_points(rng, surfaces, H, W, M, point_sigma)
    bmax = float(np.max(np.abs(baselines)))
    halo = int(np.ceil(bmax * max(abs(d_min), abs(d_max)))) + 2
    return Scene(name=name if cameras is None else name + "_calibrated", seed=seed,
                 baselines=np.asarray(baselines, np.float32),
                 images=images_out, seg_prior=seg, points=pts, d_min=float(d_min),
                 d_max=float(d_max), D=int(D), iters=int(iters),
                 gt_disparity=st_disp.astype(np.float32), gt_static=st_img.astype(np.float32),
                 dynamic_mask=dyn, halo=halo, cameras=cameras)


def _two_level_prior(p_dyn, p_static, jitter):
    def f(rng, dyn):
        p = np.where(dyn, p_dyn, p_static) + rng.uniform(-jitter, jitter, size=dyn.shape)
        return np.clip(p, 0.0, 1.0)
    return f


def _beta_prior(a_dyn, b_dyn, a_st, b_st):
    def f(rng, dyn):
        return np.where(dyn, rng.beta(a_dyn, b_dyn, size=dyn.shape), rng.beta(a_st, b_st, size=dyn.shape))
    return f


FIVE_CAMERAS = np.array([-0.2, -0.1, 0.0, 0.1, 0.2], dtype=np.float32)


def small_gray(frame: int = 0, *, H: int = 48, W: int = 64, baselines=None, D: int = 32,
               iters: int = 5, noise: float = 0.01, occluder: bool = True,
               planes=(4.0, 9.0), occluder_disparity: float = 20.0, M: int = 40,
               point_sigma: float = 0.3, calibrated: bool = False, rot_deg: float = 1.5) -> Scene:
    """5 cameras, gray float32, two planes + one occluder seen by 3 of 5 views.
    calibrated: a non-rectified array (``calibrated_cameras``, rotations up to
    rot_deg), cameras drawn from their own seeded stream."""
    seed = 1 * 1000 + frame
    rng = np.random.default_rng(seed)
    b = FIVE_CAMERAS if baselines is None else np.asarray(baselines, np.float32)
    margin = 64.0 + float(np.max(np.abs(b))) * max(planes + (occluder_disparity,))
    ext = (-margin, -4.0, W + margin, H + 4.0)
    far = Surface(planes[0], None, [value_noise(rng, (8.0, 4.0, 2.0), (0.5, 0.3, 0.2), ext)])
    split = 0.45 * W
    near = Surface(planes[1], (-1e9, -1e9, split, 1e9), [value_noise(rng, (8.0, 4.0, 2.0), (0.5, 0.3, 0.2), ext)])
    surfaces = [far, near]
    if occluder:
        ow, oh = max(4, int(0.22 * W)), max(4, int(0.45 * H))
        ou = int(0.5 * W - ow / 2)
        ov = int(0.5 * H - oh / 2)
        central = [k for k in range(len(b)) if abs(float(b[k])) <= 0.1 + 1e-6]
        surfaces.append(Surface(occluder_disparity, (ou, ov, ou + ow, ov + oh),
                                [pixel_noise(rng, (ou - 2, ov - 2, ou + ow + 2, ov + oh + 2))],
                                dynamic=True, views=central))
    cams = calibrated_cameras(np.random.default_rng(seed + 500), b, H, W, rot_deg) if calibrated else None
    return _finish("small_gray", seed, rng, surfaces, b, H, W, 1, False, noise,
                   _two_level_prior(0.9, 0.05, 0.03), M, point_sigma, 0.0, float(D - 1), D, iters, cams)


def plane_scene(seed: int, *, H: int, W: int, baselines, planes, D: int, d_min: float = 0.0,
                d_max: Optional[float] = None, iters: int = 5, noise: float = 0.0,
                M: int = 40, point_sigma: float = 0.0, texture_cells=(6.0, 3.0, 1.5),
                p_static: float = 0.05, cameras=None) -> Scene:
    """Occluder-free scene: a far plane everywhere plus nearer planes as
    vertical bands.  ``planes`` = disparities, far first."""
    rng = np.random.default_rng(seed)
    b = np.asarray(baselines, np.float32)
    margin = 64.0 + float(np.max(np.abs(b))) * max(planes)
    ext = (-margin, -4.0, W + margin, H + 4.0)
    surfaces = [Surface(planes[0], None, [value_noise(rng, texture_cells, (0.5, 0.3, 0.2), ext)])]
    n = len(planes) - 1
    for i, d in enumerate(planes[1:]):
        u0 = W * i / max(n, 1) * 0.5
        u1 = u0 + W * 0.35
        surfaces.append(Surface(d, (u0, -1e9, u1, 1e9), [value_noise(rng, texture_cells, (0.5, 0.3, 0.2), ext)]))
    dm = float(D - 1) if d_max is None else float(d_max)
    return _finish("plane_scene", seed, rng, surfaces, b, H, W, 1, False, noise,
                   _two_level_prior(0.9, p_static, 0.0), M, point_sigma, d_min, dm, D, iters, cameras)


def street_rgb(frame: int = 0, *, H: int = 600, W: int = 960, baselines=None, D: int = 64,
               iters: int = 10, noise: float = 0.01, M: int = 300, point_sigma: float = 0.5,
               n_boxes: Optional[int] = None, calibrated: bool = False, rot_deg: float = 0.6) -> Scene:
    """Paper-shaped frame: 5 cameras, RGB uint8, 3 planes, 1-4 person boxes.
    calibrated: the same scene seen by a non-rectified array."""
    seed = 2 * 1000 + frame
    rng = np.random.default_rng(seed)
    b = FIVE_CAMERAS if baselines is None else np.asarray(baselines, np.float32)
    dmax = float(D - 1)
    margin = 64.0 + float(np.max(np.abs(b))) * dmax
    ext = (-margin, -4.0, W + margin, H + 4.0)

    def rgb_tex(cells):
        return [value_noise(rng, cells, (0.5, 0.3, 0.2), ext, 0.08, 0.92) for _ in range(3)]

    # three fronto-parallel depth planes: far wall, a mid-depth side wall and a
    # near low structure (bench / railing), all static.
    sc = dmax / 63.0
    d_far, d_mid, d_near = sc * (6.0 + 4.0 * rng.random()), sc * (14.0 + 6.0 * rng.random()), \
        sc * (24.0 + 6.0 * rng.random())
    surfaces = [
        Surface(d_far, None, rgb_tex((24.0, 9.0, 3.0))),
        Surface(d_mid, (-1e9, -1e9, 0.3 * W, 1e9), rgb_tex((16.0, 6.0, 2.0))),
        Surface(d_near, (0.55 * W, 0.72 * H, 1e9, 1e9), rgb_tex((12.0, 5.0, 2.0))),
    ]
    # 1-4 person-sized boxes covering 10-35 % of the reference view.
    for _attempt in range(1000):
        nb = int(rng.integers(1, 5)) if n_boxes is None else int(n_boxes)
        boxes = []
        cover = np.zeros((H, W), dtype=bool)
        for _ in range(nb):
            bh = int(rng.uniform(0.45, 0.9) * H)
            bw = int(bh * rng.uniform(0.28, 0.42))
            u0 = int(rng.uniform(0.02 * W, W - bw - 0.02 * W))
            v0 = int(rng.uniform(0.05 * H, H - bh))
            d = float(rng.uniform(0.54 * dmax, 0.92 * dmax))
            boxes.append((u0, v0, u0 + bw, v0 + bh, d))
            cover[v0:v0 + bh, u0:u0 + bw] = True
        frac = cover.mean()
        if 0.10 <= frac <= 0.35:
            break
    for (u0, v0, u1, v1, d) in boxes:
        surfaces.append(Surface(d, (u0, v0, u1, v1), rgb_tex((10.0, 4.0, 1.5)), dynamic=True))
    cams = calibrated_cameras(np.random.default_rng(seed + 500), b, H, W, rot_deg) if calibrated else None
    return _finish("street_rgb", seed, rng, surfaces, b, H, W, 3, True, noise,
                   _beta_prior(8.0, 2.0, 1.0, 15.0), M, point_sigma, 0.0, dmax, D, iters, cams)


def random_frame(index: int, *, workload_id: int = 3, size_range=((320, 240), (1280, 1024)),
                 cams=(3, 5, 7, 9), Ds=(32, 64, 128), iters: int = 5, scale: float = 1.0) -> Scene:
    """Uneven frame for batched / served runs: resolution uniform in
    ``size_range`` (scaled by ``scale``), K from ``cams`` on a linear array
    with adjacent spacings U(0.05, 0.25) about a centre reference camera,
    D from ``Ds`` (levels 0..D-1), scene as ``small_gray``."""
    seed = workload_id * 1000 + index
    rng = np.random.default_rng(seed)
    (w0, h0), (w1, h1) = size_range
    W = max(8, int(rng.integers(w0, w1 + 1) * scale))
    H = max(8, int(rng.integers(h0, h1 + 1) * scale))
    K = int(rng.choice(cams))
    D = int(rng.choice(Ds))
    half = K // 2
    steps_r = np.cumsum(rng.uniform(0.05, 0.25, size=K - 1 - half))
    steps_l = -np.cumsum(rng.uniform(0.05, 0.25, size=half))
    b = np.concatenate([steps_l[::-1], [0.0], steps_r]).astype(np.float32)
    bmax = float(np.max(np.abs(b)))
    # keep the largest shift inside the image: disparities scaled to the width
    dmax = float(D - 1)
    margin = 64.0 + bmax * dmax
    ext = (-margin, -4.0, W + margin, H + 4.0)
    d_far = rng.uniform(0.1, 0.2) * dmax
    d_near = rng.uniform(0.25, 0.4) * dmax
    d_occ = rng.uniform(0.6, 0.9) * dmax
    surfaces = [
        Surface(d_far, None, [value_noise(rng, (8.0, 4.0, 2.0), (0.5, 0.3, 0.2), ext)]),
        Surface(d_near, (-1e9, -1e9, 0.45 * W, 1e9), [value_noise(rng, (8.0, 4.0, 2.0), (0.5, 0.3, 0.2), ext)]),
    ]
    ow, oh = max(4, int(0.22 * W)), max(4, int(0.45 * H))
    ou, ov = int(0.5 * W - ow / 2), int(0.5 * H - oh / 2)
    central = [k for k in range(K) if abs(k - (K // 2)) <= 1]
    surfaces.append(Surface(d_occ, (ou, ov, ou + ow, ov + oh),
                            [pixel_noise(rng, (ou - 2, ov - 2, ou + ow + 2, ov + oh + 2))],
                            dynamic=True, views=central))
    M = max(10, int(40 * (H * W) / (64 * 48) ** 1.0 * 0.05))
    return _finish("random_frame", seed, rng, surfaces, b, H, W, 1, False, 0.01,
                   _two_level_prior(0.9, 0.05, 0.03), M, 0.3, 0.0, dmax, D, iters)
