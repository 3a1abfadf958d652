"""The oracle's decision margins, which the GPU parity rule uses to excuse
pixels, against the brute-force J[d, S] table (CPU only).

The parity tests excuse a GPU/oracle mismatch only at a pixel whose M-step
or E-step arg-max the oracle itself wins by less than 1e-4 (1 + |J|), or
whose first-iteration threshold test (Sec. III-F) sits within 1e-5 of the
threshold.  Those margins come from the C oracle; here they are recomputed
from the exhaustive table of `oracle/bruteforce.py` (pairwise variance,
`np.interp` sampling) under the EM schedule of Sec. III-B to III-D, so that a
margin the oracle overstates or understates (and with it an excusal rule that
hides real mismatches or rejects exact ties) fails.
"""
import numpy as np
import pytest

from oracle import bruteforce as BF
from oracle import oracle as O
from paper_2003_11076_gb300 import scenes


def _tiny_frame(K, H, W, seed):
    rng = np.random.default_rng(seed)
    imgs = rng.random((K, H, W)).astype(np.float32)
    seg = rng.uniform(0.02, 0.98, size=(K, H, W)).astype(np.float32)
    b = np.concatenate([[0.0], rng.uniform(-0.6, 0.6, size=K - 1)]).astype(np.float32)
    pts = np.stack([rng.uniform(-1, W, 6), rng.uniform(-1, H, 6), rng.uniform(0, 4, 6)], 1).astype(np.float32)
    return imgs, seg, b, pts


def _top_two_gap(x):
    s = np.sort(np.asarray(x, np.float64))
    return s[-1] - s[-2] if s.size > 1 else np.inf


@pytest.mark.parametrize("seed,K,H,W,D", [(21, 3, 4, 7, 6), (22, 4, 3, 6, 5), (23, 2, 4, 8, 7), (24, 5, 2, 6, 4)])
def test_margins_match_the_brute_force_table(seed, K, H, W, D):
    imgs, seg, b, pts = _tiny_frame(K, H, W, seed)
    p = O.Params(beta=30.0)
    iters = 3
    out = O.run(imgs, seg, b, pts, 0.0, 4.0, D, iters, params=p)
    feat = BF.descriptors(imgs)
    P = seg.astype(np.float64)
    ls = np.log(np.maximum(1.0 - P, p.eps))
    ld = np.log(np.maximum(P, p.eps))
    dvals = [j * 4.0 / (D - 1) for j in range(D)]
    log_thr = np.log(p.seg_threshold / (1.0 - p.seg_threshold))
    cols = np.arange(W, dtype=np.float64)
    for v in range(H):
        for u in range(W):
            J, S_init = BF.em_pixel_table(feat, ls, ld, imgs, b, u, v, dvals, out["mu"][v, u],
                                          out["inside"][v, u], p)
            tol = 1e-9 * (1.0 + np.abs(J).max())
            S = None
            for t in range(iters):
                col = J[np.arange(D), S_init] if t == 0 else J[:, S]
                j = int(np.argmax(col))
                assert out["m_margin"][t, v, u] == pytest.approx(_top_two_gap(col), abs=tol)
                row = J[j]
                S = int(np.argmax(row))
                assert out["e_margin"][t, v, u] == pytest.approx(_top_two_gap(row), abs=tol)
                assert out["J_t"][t, v, u] == pytest.approx(row[S], abs=tol)
            # first-iteration threshold test: the closest any ray's sample
            # comes to it, over every candidate and camera
            z = [abs(np.interp(u - d * float(b[k]), cols, ld[k, v]) - np.interp(u - d * float(b[k]), cols, ls[k, v])
                     - log_thr) for d in dvals for k in range(K)]
            assert out["init_margin"][v, u] == pytest.approx(min(z), abs=1e-12)


def test_excusal_follows_its_margins_and_is_rare():
    """excused() = some margin below its bound, nothing else; on the 64x48
    frame it excuses few pixels, so the parity rule stays tight."""
    s = scenes.small_gray(0)
    out = O.run_scene(s)
    tau = 1e-4 * (1.0 + np.abs(out["J_t"]))
    expect = np.any(out["m_margin"] < tau, axis=0) | np.any(out["e_margin"] < tau, axis=0) | \
        (out["init_margin"] < 1e-5)
    assert np.array_equal(O.excused(out), expect)
    assert 0 < expect.mean() < 0.02
    # a looser rule excuses a superset, a tighter one a subset
    assert np.all(O.excused(out, tau_rel=1e-3) >= expect) and np.all(O.excused(out, tau_rel=1e-6) <= expect)


@pytest.mark.parametrize("seed,K,H,W,D", [(31, 3, 4, 6, 5), (32, 4, 3, 5, 6)])
def test_calibrated_margins_match_the_brute_force_table(seed, K, H, W, D):
    """The same for a calibrated (non-rectified) array: the table's rays are
    sampled by scipy.ndimage.map_coordinates at the cameras' positions."""
    from scipy import ndimage
    rng = np.random.default_rng(seed)
    imgs = rng.random((K, H, W)).astype(np.float32)
    seg = rng.uniform(0.02, 0.98, size=(K, H, W)).astype(np.float32)
    b = np.concatenate([[0.0], rng.uniform(-0.6, 0.6, size=K - 1)]).astype(np.float32)
    cams = scenes.calibrated_cameras(rng, b, H, W, rot_deg=4.0, shift_y=0.3, shift_z=0.1, focal_jitter=0.05)
    pts = np.stack([rng.uniform(-1, W, 6), rng.uniform(-1, H, 6), rng.uniform(0, 4, 6)], 1).astype(np.float32)
    p = O.Params(beta=30.0)
    iters = 3
    out = O.run(imgs, seg, b, pts, 0.0, 4.0, D, iters, params=p, cameras=cams)
    feat = BF.descriptors(imgs)
    P = seg.astype(np.float64)
    ls = np.log(np.maximum(1.0 - P, p.eps))
    ld = np.log(np.maximum(P, p.eps))
    dvals = [j * 4.0 / (D - 1) for j in range(D)]
    log_thr = np.log(p.seg_threshold / (1.0 - p.seg_threshold))
    for v in range(H):
        for u in range(W):
            J, S_init = BF.em_pixel_table(feat, ls, ld, imgs, b, u, v, dvals, out["mu"][v, u],
                                          out["inside"][v, u], p, cameras=cams)
            tol = 1e-9 * (1.0 + np.abs(J).max())
            S = None
            for t in range(iters):
                col = J[np.arange(D), S_init] if t == 0 else J[:, S]
                j = int(np.argmax(col))
                assert out["m_margin"][t, v, u] == pytest.approx(_top_two_gap(col), abs=tol)
                S = int(np.argmax(J[j]))
                assert out["e_margin"][t, v, u] == pytest.approx(_top_two_gap(J[j]), abs=tol)
            z = []
            for d in dvals:
                for k in range(K):
                    X = np.asarray(cams[k], np.float64) @ np.array([u, v, 1.0, d])
                    xy = [[X[1] / X[2]], [X[0] / X[2]]]
                    z.append(abs(ndimage.map_coordinates(ld[k], xy, order=1, mode="nearest")[0]
                                 - ndimage.map_coordinates(ls[k], xy, order=1, mode="nearest")[0] - log_thr))
            assert out["init_margin"][v, u] == pytest.approx(min(z), abs=1e-12)


@pytest.mark.parametrize("seed,K,H,W,D", [(41, 3, 4, 6, 5), (42, 4, 3, 5, 6)])
def test_soft_em_margins_match_the_brute_force_table(seed, K, H, W, D):
    """Soft EM (reading R23): after the first iteration the M-step column is
    Q(d) = sum_S q(S) J(d, S) with q the softmax of the previous E-step's
    row; the recorded objective is the row's log-sum-exp (the log marginal)."""
    imgs, seg, b, pts = _tiny_frame(K, H, W, seed)
    p = O.Params(beta=30.0, em_mode=1)
    iters = 3
    out = O.run(imgs, seg, b, pts, 0.0, 4.0, D, iters, params=p)
    feat = BF.descriptors(imgs)
    P = seg.astype(np.float64)
    ls = np.log(np.maximum(1.0 - P, p.eps))
    ld = np.log(np.maximum(P, p.eps))
    dvals = [j * 4.0 / (D - 1) for j in range(D)]
    for v in range(H):
        for u in range(W):
            J, S_init = BF.em_pixel_table(feat, ls, ld, imgs, b, u, v, dvals, out["mu"][v, u],
                                          out["inside"][v, u], p)
            tol = 1e-9 * (1.0 + np.abs(J).max())
            q = None
            for t in range(iters):
                col = J[np.arange(D), S_init] if t == 0 else J @ q
                j = int(np.argmax(col))
                assert out["m_margin"][t, v, u] == pytest.approx(_top_two_gap(col), abs=tol)
                row = J[j]
                assert out["e_margin"][t, v, u] == pytest.approx(_top_two_gap(row), abs=tol)
                m = row.max()
                q = np.exp(row - m)
                assert out["J_t"][t, v, u] == pytest.approx(m + np.log(q.sum()), abs=tol)
                q /= q.sum()


@pytest.mark.parametrize("seed,K,H,W,D", [(51, 3, 4, 6, 5), (52, 2, 3, 7, 6)])
def test_joint_map_margins_match_the_brute_force_table(seed, K, H, W, D):
    """Joint MAP (reading R24): the M margin is the gap between the two best
    candidates' row maxima, the E margin the gap inside the winning row, the
    recorded objective the joint maximum, in every diagnostic slot."""
    imgs, seg, b, pts = _tiny_frame(K, H, W, seed)
    p = O.Params(beta=30.0, em_mode=2)
    iters = 2
    out = O.run(imgs, seg, b, pts, 0.0, 4.0, D, iters, params=p)
    feat = BF.descriptors(imgs)
    P = seg.astype(np.float64)
    ls = np.log(np.maximum(1.0 - P, p.eps))
    ld = np.log(np.maximum(P, p.eps))
    dvals = [j * 4.0 / (D - 1) for j in range(D)]
    for v in range(H):
        for u in range(W):
            J, _ = BF.em_pixel_table(feat, ls, ld, imgs, b, u, v, dvals, out["mu"][v, u], out["inside"][v, u], p)
            tol = 1e-9 * (1.0 + np.abs(J).max())
            rowmax = J.max(axis=1)
            j = int(np.argmax(rowmax))
            for t in range(iters):
                assert out["m_margin"][t, v, u] == pytest.approx(_top_two_gap(rowmax), abs=tol)
                assert out["e_margin"][t, v, u] == pytest.approx(_top_two_gap(J[j]), abs=tol)
                assert out["J_t"][t, v, u] == pytest.approx(J.max(), abs=tol)
