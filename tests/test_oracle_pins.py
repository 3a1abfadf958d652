"""Pins of the FP64 oracle against facts fixed outside it (CPU only).

Each test ties one oracle function to a closed form, a special case that
reduces to a textbook or library routine, brute force, or ground truth that
the scene construction fixes, so that a dropped term, a wrong sign or index,
or a transposed operand anywhere in the oracle fails at least one of them.
"""
import itertools

import numpy as np
import pytest
from scipy import ndimage

from oracle import bruteforce as BF
from oracle import oracle as O
from paper_2003_11076_gb300 import scenes

rng0 = np.random.default_rng(12345)


# ------------------------------------------------------------------ features

def test_sobel_of_linear_ramp_is_its_gradient():
    """Sobel/8 of Y = a*u + b*v is exactly (a, b) away from the border and half
    of it on the replicated border (Sec. III-C descriptors)."""
    H, W = 7, 9
    a, b = 0.03, -0.02
    vv, uu = np.meshgrid(np.arange(H), np.arange(W), indexing="ij")
    Y = (0.2 + a * uu + b * vv).astype(np.float32)[None]
    f = O.features(Y)
    assert np.allclose(f[0, 0], Y[0], atol=0)
    assert np.allclose(f[0, 1, :, 1:-1], a, atol=1e-12)
    assert np.allclose(f[0, 2, 1:-1, :], b, atol=1e-12)
    assert np.allclose(f[0, 1, :, 0], a / 2, atol=1e-12)
    assert np.allclose(f[0, 1, :, -1], a / 2, atol=1e-12)
    assert np.allclose(f[0, 2, 0, :], b / 2, atol=1e-12)


@pytest.mark.parametrize("rgb", [False, True])
def test_features_match_scipy_correlate(rgb):
    """Descriptors equal scipy's 'nearest'-mode correlation with the Sobel
    kernels on the BT.601 luminance (library routine)."""
    if rgb:
        imgs = rng0.integers(0, 256, size=(3, 6, 11, 3), dtype=np.uint8)
    else:
        imgs = rng0.random((3, 6, 11)).astype(np.float32)
    assert np.allclose(O.features(imgs), BF.descriptors(imgs), atol=1e-13, rtol=0)


def test_golden_sobel_fixture():
    """Hand-computed 3x4 fixture (tests/golden/sobel_3x4.txt)."""
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "sobel_3x4.txt")
    rows = [line.split() for line in open(path) if line.strip() and not line.startswith("#")]
    vals = np.array([[float(x) for x in r] for r in rows])
    Y = vals[0:3].astype(np.float32)
    gx = vals[3:6]
    gy = vals[6:9]
    f = O.features(Y[None])
    assert np.allclose(f[0, 1], gx, atol=1e-6)
    assert np.allclose(f[0, 2], gy, atol=1e-6)


def test_sampling_is_clamped_linear_interpolation():
    row = rng0.random(13)
    for x in np.concatenate([np.linspace(-3, 16, 97), [0.0, 12.0, 5.5, 11.999]]):
        assert O.sample(row, x) == pytest.approx(np.interp(x, np.arange(13.0), row), abs=1e-15)


# ----------------------------------------------------------------- objective

def _tiny_frame(K, H, W, seed, baselines=None, P=None):
    rng = np.random.default_rng(seed)
    imgs = rng.random((K, H, W)).astype(np.float32)
    seg = rng.uniform(0.02, 0.98, size=(K, H, W)).astype(np.float32) if P is None else \
        np.full((K, H, W), P, np.float32)
    if baselines is None:
        baselines = np.concatenate([[0.0], rng.uniform(-0.6, 0.6, size=K - 1)]).astype(np.float32)
    return imgs, seg, np.asarray(baselines, np.float32)


def test_two_ray_variance_closed_form():
    """Var of two static rays = |f1 - f2|^2 / 4 (population variance)."""
    imgs, seg, b = _tiny_frame(2, 5, 9, 7, baselines=[0.0, 0.37])
    p = O.Params()
    f = BF.descriptors(imgs)
    ls, ld = np.log(np.maximum(1 - seg.astype(np.float64), p.eps)), np.log(np.maximum(seg.astype(np.float64), p.eps))
    u, v, d = 6, 2, 3.3
    xs = [u - d * float(b[k]) for k in range(2)]
    f1 = np.array([np.interp(xs[0], np.arange(9.0), f[0, c, v]) for c in range(3)])
    f2 = np.array([np.interp(xs[1], np.arange(9.0), f[1, c, v]) for c in range(3)])
    seg_both = sum(np.interp(xs[k], np.arange(9.0), ls[k, v]) for k in range(2))
    expect = -p.beta * np.sum((f1 - f2) ** 2) / 4.0 + seg_both
    got = O.objective_at(imgs, seg, b, u, v, d, S=0b11)
    assert got == pytest.approx(expect, abs=1e-11)
    # one static ray: no variance, one static and one dynamic log-prior
    expect1 = np.interp(xs[0], np.arange(9.0), ls[0, v]) + np.interp(xs[1], np.arange(9.0), ld[1, v])
    assert O.objective_at(imgs, seg, b, u, v, d, S=0b01) == pytest.approx(expect1, abs=1e-12)


def test_log_prior_closed_form():
    """K = 1: J(d, static) = log(gamma + exp(-(d-mu)^2/(2 sigma^2))) + log(1-P);
    at d = mu this is log(gamma + 1) + log(1 - P)."""
    imgs, seg, b = _tiny_frame(1, 3, 4, 3, P=0.25)
    p = O.Params(gamma=0.1, sigma=2.0)
    mu = 5.25
    assert O.objective_at(imgs, seg, b, 1, 1, mu, 1, mu=mu, inside=1, params=p) == \
        pytest.approx(np.log(1.1) + np.log(0.75), abs=1e-14)
    d = 8.0
    expect = np.log(0.1 + np.exp(-(d - mu) ** 2 / 8.0)) + np.log(0.75)
    assert O.objective_at(imgs, seg, b, 1, 1, d, 1, mu=mu, inside=1, params=p) == pytest.approx(expect, abs=1e-14)
    # outside the triangulation the prior is uniform (0)
    assert O.objective_at(imgs, seg, b, 1, 1, d, 1, mu=mu, inside=0, params=p) == pytest.approx(np.log(0.75), abs=1e-14)


def test_single_camera_posterior_is_one_minus_P():
    """K = 1: the variance vanishes, so q(static) = (1-P) / ((1-P) + P)."""
    rng = np.random.default_rng(5)
    imgs = rng.random((1, 4, 6)).astype(np.float32)
    seg = rng.uniform(0.01, 0.99, size=(1, 4, 6)).astype(np.float32)
    out = O.run(imgs, seg, np.zeros(1, np.float32), np.zeros((0, 3), np.float32), 0, 3, 4, 2)
    assert np.allclose(out["post"][0], 1.0 - seg[0].astype(np.float64), atol=1e-12)
    assert np.array_equal(out["labels"] & 1, (seg[0] < 0.5).astype(np.uint16))


def test_two_camera_posteriors_closed_form():
    """K = 2: the four label vectors' objectives written out by hand give the
    marginals; they also lie in [0, 1]."""
    imgs, seg, b = _tiny_frame(2, 4, 8, 11, baselines=[0.0, -0.45])
    p = O.Params()
    out = O.run(imgs, seg, b, np.zeros((0, 3), np.float32), 0.0, 5.0, 6, 3, params=p)
    f = BF.descriptors(imgs)
    P = seg.astype(np.float64)
    ls, ld = np.log(np.maximum(1 - P, p.eps)), np.log(np.maximum(P, p.eps))
    grid = np.arange(8.0)
    for v in range(4):
        for u in range(8):
            d = out["d"][v, u]
            xs = [u - d * float(b[k]) for k in range(2)]
            fk = [np.array([np.interp(xs[k], grid, f[k, c, v]) for c in range(3)]) for k in range(2)]
            s_ = [np.interp(xs[k], grid, ls[k, v]) for k in range(2)]
            d_ = [np.interp(xs[k], grid, ld[k, v]) for k in range(2)]
            J00 = d_[0] + d_[1]
            J10 = s_[0] + d_[1]
            J01 = d_[0] + s_[1]
            J11 = s_[0] + s_[1] - p.beta * np.sum((fk[0] - fk[1]) ** 2) / 4.0
            e = np.exp(np.array([J00, J10, J01, J11]) - max(J00, J10, J01, J11))
            Z = e.sum()
            assert out["post"][0, v, u] == pytest.approx((e[1] + e[3]) / Z, abs=1e-12)
            assert out["post"][1, v, u] == pytest.approx((e[2] + e[3]) / Z, abs=1e-12)
    assert np.all((out["post"] >= 0) & (out["post"] <= 1))


# ------------------------------------------------------------- brute force

@pytest.mark.parametrize("seed,K,H,W,D", [(1, 3, 4, 6, 5), (2, 4, 3, 5, 6), (3, 2, 4, 6, 6),
                                          (4, 4, 2, 6, 4), (5, 3, 3, 7, 1), (6, 1, 4, 6, 5)])
def test_em_matches_exhaustive_enumeration(seed, K, H, W, D):
    """Every M-step and E-step arg-max, the posteriors and the refocus agree
    with the exhaustive J[d, S] table (pairwise-variance formula), and the EM
    objective never exceeds the joint maximum over (d, S)."""
    imgs, seg, b = _tiny_frame(K, H, W, seed)
    rng = np.random.default_rng(seed + 100)
    pts = np.stack([rng.uniform(-1, W, 6), rng.uniform(-1, H, 6), rng.uniform(0, 4, 6)], 1).astype(np.float32)
    p = O.Params(beta=30.0)
    iters = 4
    out = O.run(imgs, seg, b, pts, 0.0, 4.0, D, iters, params=p)
    bf = BF.run(imgs, seg, b, out["mu"], out["inside"], 0.0, 4.0, D, iters, p)
    ok = ~O.excused(out, tau_rel=1e-9, tau_init=1e-9)
    assert ok.sum() >= 6   # clamped border columns and K = 1 can tie exactly
    assert np.array_equal(out["d_idx"][ok], bf["d_idx"][ok])
    assert np.array_equal(out["labels"][ok].astype(np.int64), bf["labels"][ok])
    assert np.allclose(out["post"][:, ok], bf["post"][:, ok], atol=1e-11)
    assert np.allclose(out["refocus"][ok], bf["refocus"][ok], atol=1e-12)
    assert np.allclose(out["J_t"][-1][ok], bf["J_final"][ok], atol=1e-10)
    assert np.all(out["J_t"][-1] <= bf["joint_max"] + 1e-10)


@pytest.mark.parametrize("seed,K,H,W,D", [(1, 3, 4, 6, 5), (2, 4, 3, 5, 6), (3, 2, 4, 6, 6), (6, 1, 4, 6, 5)])
def test_soft_em_matches_exhaustive_table(seed, K, H, W, D):
    """Soft EM: after the first iteration the M-step maximises the table's
    rows averaged under the previous E-step's softmax (J @ q); the oracle's
    arg-maxes, posteriors and log marginals agree with the table's."""
    imgs, seg, b = _tiny_frame(K, H, W, seed)
    rng = np.random.default_rng(seed + 100)
    pts = np.stack([rng.uniform(-1, W, 6), rng.uniform(-1, H, 6), rng.uniform(0, 4, 6)], 1).astype(np.float32)
    p = O.Params(beta=30.0, em_mode=1)
    iters = 4
    out = O.run(imgs, seg, b, pts, 0.0, 4.0, D, iters, params=p)
    bf = BF.run(imgs, seg, b, out["mu"], out["inside"], 0.0, 4.0, D, iters, p, mode="soft")
    ok = ~O.excused(out, tau_rel=1e-9, tau_init=1e-9)
    assert ok.sum() >= 6
    assert np.array_equal(out["d_idx"][ok], bf["d_idx"][ok])
    assert np.array_equal(out["labels"][ok].astype(np.int64), bf["labels"][ok])
    assert np.allclose(out["post"][:, ok], bf["post"][:, ok], atol=1e-11)
    assert np.allclose(out["J_t"][:, ok], bf["L_t"][:, ok], atol=1e-10)
    hard = O.run(imgs, seg, b, pts, 0.0, 4.0, D, iters, params=O.Params(beta=30.0))
    if K > 1:  # the two EMs are different algorithms: some pixel must differ
        assert not np.array_equal(out["J_t"], hard["J_t"])


@pytest.mark.parametrize("seed,K,H,W,D", [(1, 3, 4, 6, 5), (2, 4, 3, 5, 6), (5, 3, 3, 7, 1), (6, 1, 4, 6, 5)])
def test_joint_map_matches_exhaustive_table(seed, K, H, W, D):
    """Joint MAP is the arg-max of the whole table (lowest d, then smallest
    mask); its objective is the table maximum at every pixel, tie or not."""
    imgs, seg, b = _tiny_frame(K, H, W, seed)
    rng = np.random.default_rng(seed + 100)
    pts = np.stack([rng.uniform(-1, W, 6), rng.uniform(-1, H, 6), rng.uniform(0, 4, 6)], 1).astype(np.float32)
    p = O.Params(beta=30.0, em_mode=2)
    out = O.run(imgs, seg, b, pts, 0.0, 4.0, D, 2, params=p)
    bf = BF.run(imgs, seg, b, out["mu"], out["inside"], 0.0, 4.0, D, 2, p, mode="joint")
    assert np.allclose(out["J_t"][0], bf["joint_max"], atol=1e-10)
    assert np.array_equal(out["J_t"][0], out["J_t"][1])
    ok = ~O.excused(out, tau_rel=1e-9, tau_init=1e-9)
    assert ok.sum() >= 6
    assert np.array_equal(out["d_idx"][ok], bf["d_idx"][ok])
    assert np.array_equal(out["labels"][ok].astype(np.int64), bf["labels"][ok])
    assert np.allclose(out["post"][:, ok], bf["post"][:, ok], atol=1e-11)
    assert np.allclose(out["refocus"][ok], bf["refocus"][ok], atol=1e-12)
    hard = O.run(imgs, seg, b, pts, 0.0, 4.0, D, 4, params=O.Params(beta=30.0))
    assert np.all(hard["J_t"][-1] <= out["J_t"][0] + 1e-10)


def test_soft_em_pin_catches_planted_uniform_posterior(monkeypatch):
    """The soft-EM pin is sensitive: averaging the rows under a uniform
    instead of the E-step's posterior changes the result somewhere."""
    imgs, seg, b = _tiny_frame(3, 4, 6, 1)
    p = O.Params(beta=30.0, em_mode=1)
    out = O.run(imgs, seg, b, np.zeros((0, 3), np.float32), 0.0, 4.0, 5, 4, params=p)
    good = BF.run(imgs, seg, b, out["mu"], out["inside"], 0.0, 4.0, 5, 4, p, mode="soft")
    assert np.allclose(good["L_t"], out["J_t"], atol=1e-10)
    monkeypatch.setattr(BF, "_softmax", lambda row: np.full(row.shape, 1.0 / row.size))
    bad = BF.run(imgs, seg, b, out["mu"], out["inside"], 0.0, 4.0, 5, 4, p, mode="soft")
    assert not np.allclose(bad["L_t"], out["J_t"], atol=1e-10)


def test_brute_force_catches_planted_sign_error(monkeypatch):
    """The brute force is sensitive enough: flipping the sign of the variance
    term in the exhaustive table changes the arg-max somewhere."""
    imgs, seg, b = _tiny_frame(3, 4, 6, 1)
    p = O.Params(beta=30.0)
    out = O.run(imgs, seg, b, np.zeros((0, 3), np.float32), 0.0, 4.0, 5, 3, params=p)
    good = BF.run(imgs, seg, b, out["mu"], out["inside"], 0.0, 4.0, 5, 3, p)
    orig = BF.pairwise_variance
    monkeypatch.setattr(BF, "pairwise_variance", lambda f: -orig(f))
    bad = BF.run(imgs, seg, b, out["mu"], out["inside"], 0.0, 4.0, 5, 3, p)
    assert not np.array_equal(good["d_idx"], bad["d_idx"]) or not np.array_equal(good["labels"], bad["labels"])


# ----------------------------------------------------------- EM invariants

def test_objective_never_decreases():
    """J(d_t, S_t) >= J(d_{t-1}, S_{t-1}) at every pixel (M-step and E-step
    are both maximisations of the same complete-data objective)."""
    s = scenes.small_gray(0)
    out = O.run_scene(s, iters=6)
    J = out["J_t"]
    assert np.all(J[1:] >= J[:-1] - 1e-12)
    post = out["post"]
    assert np.all((post >= 0) & (post <= 1))


def test_soft_em_log_marginal_never_decreases():
    """Soft EM never decreases log sum_S exp J(d_t, S) (Jensen's bound: the
    M-step raises the expected objective under the exact posterior at
    d_{t-1}, which lower-bounds the log marginal and touches it at d_{t-1})."""
    s = scenes.small_gray(0)
    out = O.run_scene(s, params=O.Params(em_mode=1), iters=6)
    L = out["J_t"]
    assert np.all(L[1:] >= L[:-1] - 1e-9 * (1 + np.abs(L[:-1])))
    hard = O.run_scene(s, iters=6)
    assert not np.array_equal(out["d_idx"], hard["d_idx"]) or not np.array_equal(L[-1], hard["J_t"][-1])


def test_joint_map_bounds_both_ems():
    """The joint maximum over (d, S) is at least the final objective of the
    hard EM at every pixel."""
    s = scenes.small_gray(1)
    joint = O.run_scene(s, params=O.Params(em_mode=2), iters=1)
    hard = O.run_scene(s, iters=5)
    assert np.all(hard["J_t"][-1] <= joint["J_t"][0] + 1e-9)


def test_occluder_free_integer_shift_scene_is_exact():
    """Noise-free fronto-parallel planes, dyadic baselines so the true shifts
    are whole pixels, uniform prior: away from the image border and the plane
    boundary the recovered disparity is the ground-truth plane, every ray is
    static and the refocus reproduces the static texture exactly."""
    b = [-0.25, -0.125, 0.0, 0.125, 0.25]
    for seed in (11, 12):
        s = scenes.plane_scene(seed, H=32, W=64, baselines=b, planes=(8.0, 16.0), D=32, M=0)
        out = O.run_scene(s)
        mask = np.zeros((s.H, s.W), bool)
        mask[1:-1, s.halo:s.W - s.halo] = True
        u = np.arange(s.W)
        for ub in (0.0, 0.35 * s.W):
            mask[:, np.abs(u - ub) <= 5] = False
        assert mask.sum() > 500
        assert np.array_equal(out["d"][mask], s.gt_disparity[mask].astype(np.float64))
        assert np.all(out["labels"][mask] == 0b11111)
        assert np.array_equal(out["refocus"][mask], s.gt_static[mask].astype(np.float64))


def test_occluder_free_noisy_fractional_scene_is_close():
    """sigma = 0.01 noise and baselines 0.1 / 0.2 (fractional shifts): the
    disparity is within 2 levels of the ground truth on >= 99 % of interior
    pixels and every ray stays static."""
    b = [-0.2, -0.1, 0.0, 0.1, 0.2]
    s = scenes.plane_scene(12, H=40, W=72, baselines=b, planes=(4.0, 9.0), D=32, noise=0.01, M=0)
    out = O.run_scene(s)
    mask = np.zeros((s.H, s.W), bool)
    mask[1:-1, s.halo:s.W - s.halo] = True
    u = np.arange(s.W)
    for ub in (0.0, 0.35 * s.W):
        mask[:, np.abs(u - ub) <= 4] = False
    err = np.abs(out["d"] - s.gt_disparity)[mask]
    assert np.mean(err <= 2) >= 0.99
    assert np.all(out["labels"][mask] == 0b11111)


def test_beta_zero_picks_candidate_nearest_prior():
    """beta = 0 and a constant segmentation prior: the objective reduces to
    the disparity prior, maximised by the candidate nearest mu (lower index on
    a tie); outside the triangulation every candidate ties -> index 0."""
    imgs, seg, b = _tiny_frame(3, 12, 16, 9, P=0.2)
    pts = np.array([[1.3, 0.7, 3.1], [14.6, 1.2, 7.9], [7.7, 10.9, 12.4]], np.float32)
    p = O.Params(beta=0.0)
    D = 32
    out = O.run(imgs, seg, b, pts, 0.0, 15.5, D, 2, params=p)
    dvals = np.arange(D) * (15.5 / (D - 1))
    ins = out["inside"] == 1
    assert ins.sum() > 20 and (~ins).sum() > 20
    expect = np.argmin(np.abs(dvals[None, :] - out["mu"][ins][:, None]), axis=1)
    assert np.array_equal(out["d_idx"][ins], expect)
    assert np.all(out["d_idx"][~ins] == 0)


def test_large_gamma_is_plain_multibaseline_stereo():
    """gamma -> infinity (flat prior), all rays static with a constant prior:
    the M-step is the arg-min over d of the sum of squared deviations of the
    sampled descriptors across views (plain multi-baseline stereo)."""
    imgs, seg, b = _tiny_frame(4, 6, 20, 21, baselines=[0.0, 0.3, -0.25, 0.55], P=0.05)
    pts = np.array([[0, 0, 1], [19, 0, 2], [0, 5, 3], [19, 5, 1.5]], np.float32)
    p = O.Params(gamma=1e12)
    D = 12
    out = O.run(imgs, seg, b, pts, 0.0, 11.0, D, 1, params=p)
    f = BF.descriptors(imgs)
    grid = np.arange(20.0)
    for v in range(6):
        for u in range(20):
            ssd = []
            for j in range(D):
                samp = np.array([[np.interp(u - j * float(b[k]), grid, f[k, c, v]) for c in range(3)]
                                 for k in range(4)])
                ssd.append(np.sum((samp - samp.mean(axis=0)) ** 2))
            ssd = np.array(ssd)
            order = np.sort(ssd)
            if order[1] - order[0] > 1e-12:
                assert out["d_idx"][v, u] == int(np.argmin(ssd))


# ------------------------------------------------------------------- prior

def test_prior_is_exact_at_vertices_and_planar_inside_triangles():
    """mu equals the vertex disparity on a vertex pixel, is the plane through
    the triangle's three vertices elsewhere (a 3x3 solve), and pixels outside
    the hull are flagged outside."""
    pts = np.array([[2.0, 3.0, 5.0], [20.0, 1.0, 9.0], [11.0, 17.0, 2.0], [25.0, 15.0, 6.5]], np.float32)
    H, W = 20, 30
    mu, inside = O.prior_raster(pts, H, W)
    for (u, v, d) in pts:
        assert inside[int(v), int(u)] == 1
        assert mu[int(v), int(u)] == pytest.approx(d, abs=1e-12)
    tris, P = O.triangulate(pts)
    assert len(tris) == 2
    vv, uu = np.meshgrid(np.arange(H), np.arange(W), indexing="ij")
    covered = np.zeros((H, W), bool)
    # barycentric coordinates by a linear solve, independent of the raster
    for t in tris:
        A = np.c_[P[t, 0], P[t, 1], np.ones(3)]
        coef = np.linalg.solve(A, P[t, 2])
        lam = np.linalg.solve(A.T, np.stack([uu.ravel(), vv.ravel(), np.ones(uu.size)]))
        strict = np.all(lam > 1e-9, axis=0).reshape(H, W)
        assert np.all(inside[strict] == 1)
        plane = coef[0] * uu + coef[1] * vv + coef[2]
        assert np.allclose(mu[strict], plane[strict], atol=1e-10)
        covered |= np.all(lam >= -1e-9, axis=0).reshape(H, W)
    assert np.all(inside[~covered] == 0)


def test_prior_degenerate_point_sets_are_uniform():
    for pts in (np.zeros((0, 3)), np.array([[1, 1, 2], [5, 5, 3]]), np.array([[0, 0, 1], [1, 1, 2], [2, 2, 3], [3, 3, 1]])):
        mu, inside = O.prior_raster(np.asarray(pts, np.float32), 6, 6)
        assert inside.sum() == 0


# ------------------------------------------------------------------ refocus

def test_refocus_all_static_is_mean_of_samples_and_empty_is_reference():
    """Eq. 2: with every ray static the refocus is the plain mean of the K
    interpolated samples at the final disparity; with none static the
    reference pixel is kept."""
    imgs, _, b = _tiny_frame(3, 4, 10, 17, baselines=[0.0, 0.4, -0.3])
    seg = np.full((3, 4, 10), 0.01, np.float32)
    out = O.run(imgs, seg, b, np.zeros((0, 3), np.float32), 0.0, 3.0, 4, 2, params=O.Params(beta=1e-3))
    assert np.all(out["labels"] == 0b111)
    grid = np.arange(10.0)
    for v in range(4):
        for u in range(10):
            d = out["d"][v, u]
            m = np.mean([np.interp(u - d * float(b[k]), grid, imgs[k, v].astype(np.float64)) for k in range(3)])
            assert out["refocus"][v, u] == pytest.approx(m, abs=1e-15)
    seg_dyn = np.full((3, 4, 10), 0.99, np.float32)
    out = O.run(imgs, seg_dyn, b, np.zeros((0, 3), np.float32), 0.0, 3.0, 4, 2)
    assert np.all(out["labels"] == 0)
    assert np.array_equal(out["refocus"], imgs[0].astype(np.float64))


def test_refocus_rgb_uint8_scaling():
    rng = np.random.default_rng(8)
    imgs = rng.integers(0, 256, size=(2, 3, 7, 3), dtype=np.uint8)
    seg = np.full((2, 3, 7), 0.99, np.float32)
    out = O.run(imgs, seg, np.array([0.0, 0.5], np.float32), np.zeros((0, 3), np.float32), 0.0, 2.0, 3, 1)
    assert np.allclose(out["refocus"], imgs[0] / 255.0, atol=1e-15)


def test_median3_matches_scipy():
    rng = np.random.default_rng(2)
    img = rng.random((9, 13, 3))
    ref = np.stack([ndimage.median_filter(img[..., c], size=3, mode="nearest") for c in range(3)], -1)
    assert np.array_equal(O.median3(img), ref)
