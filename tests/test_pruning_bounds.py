"""The bounds behind the exact pruning, checked in FP64 on the brute-force
table (CPU only).

The GPU path skips candidates of an M-step (and, from seven cameras, blocks
of label vectors of an E-step) whose upper bound is below an objective it has
already computed; the GPU tests compare it bit for bit with full sweeps.
These tests check the algebra the skipping rests on, independently of the
kernel, on the exhaustive J[d, S] table of `oracle/bruteforce.py` under the
EM schedule of Sec. III-B to III-D:

* every objective is at most log prior(d) + seg_max, seg_max being the sum
  over cameras of the largest max(log p(static), log p(dynamic)) among the
  texels the camera's ray interpolates over the candidate range (the
  variance term -beta Var is never positive);
* with J* the objective of one candidate of the M-step's own column, every
  candidate outside (d - mu)^2 <= -2 sigma^2 log(exp(J* - seg_max) - gamma)
  has an objective below J*, so the column's arg-max (lowest index on ties)
  lies inside;
* an E-step block of label vectors sharing their high cameras has every
  objective at most the block's base plus the positive parts of its low
  cameras' log-odds, so a block below the all-static vector's objective
  holds no arg-max.
"""
import numpy as np
import pytest

from oracle import bruteforce as BF
from oracle import oracle as O


def _frame(K, H, W, seed):
    rng = np.random.default_rng(seed)
    imgs = rng.random((K, H, W)).astype(np.float32)
    # P(dynamic) with both tails, so max(log p(static), log p(dynamic))
    # comes from either map
    seg = np.where(rng.random((K, H, W)) < 0.3, rng.uniform(0.6, 0.99, (K, H, W)),
                   rng.uniform(0.01, 0.4, (K, H, W))).astype(np.float32)
    b = np.concatenate([[0.0], rng.uniform(-0.5, 0.5, size=K - 1)]).astype(np.float32)
    return imgs, seg, b, rng


def _log_maps(seg, eps):
    P = seg.astype(np.float64)
    return np.log(np.maximum(1.0 - P, eps)), np.log(np.maximum(P, eps))


def _seg_max(ls, ld, b, u, v, dvals, W):
    """Sum over cameras of the largest max(ls, ld) over the texels between the
    ray's leftmost and rightmost sample positions (both ends clamped)."""
    total = 0.0
    for k in range(ls.shape[0]):
        xs = [u - d * float(b[k]) for d in dvals]
        lo = int(np.clip(np.floor(min(xs)), 0, W - 1))
        hi = int(np.clip(np.ceil(max(xs)), 0, W - 1))
        total += float(np.max(np.maximum(ls[k, v, lo:hi + 1], ld[k, v, lo:hi + 1])))
    return total


def _log_prior(d, mu, inside, gamma, sigma):
    return BF.log_prior(d, mu, inside, gamma, sigma)


def _interval(Js, seg_ub, mu, gamma, sigma, dvals):
    """Candidates whose bound log prior + seg_ub can reach Js (exact
    arithmetic, no slack): |d - mu| <= r with gamma + exp(-r^2 / 2 sigma^2)
    = exp(Js - seg_ub); all of them when exp(Js - seg_ub) <= gamma."""
    e = np.exp(Js - seg_ub)
    if not np.isfinite(Js) or e <= gamma:
        return np.ones(len(dvals), bool)
    r2 = -2.0 * sigma * sigma * np.log(e - gamma)
    return (np.asarray(dvals) - mu) ** 2 <= r2


CASES = [
    # K, H, W, D, d range, beta, gamma, sigma, seed
    (2, 4, 14, 17, (-2.0, 6.0), 200.0, 0.1, 2.0, 1),
    (3, 4, 14, 13, (0.0, 9.0), 200.0, 0.0, 1.0, 2),
    (4, 3, 12, 9, (-3.0, 3.0), 5.0, 0.5, 0.7, 3),
    (5, 3, 12, 11, (0.0, 5.0), 50.0, 0.01, 3.0, 4),
    (3, 3, 16, 21, (-4.0, 4.0), 2000.0, 0.1, 0.4, 5),
]


@pytest.mark.filterwarnings("ignore:divide by zero")   # log(gamma) at gamma = 0 is -inf, as intended
@pytest.mark.parametrize("K,H,W,D,dr,beta,gamma,sigma,seed", CASES)
def test_candidate_interval_holds_every_m_step_argmax(K, H, W, D, dr, beta, gamma, sigma, seed):
    imgs, seg, b, rng = _frame(K, H, W, seed)
    p = O.Params(beta=beta, gamma=gamma, sigma=sigma)
    feat = BF.descriptors(imgs)
    ls, ld = _log_maps(seg, p.eps)
    d0, d1 = dr
    dvals = [d0 + j * (d1 - d0) / (D - 1) for j in range(D)]
    iters = 4
    pruned = 0
    total = 0
    for v in range(H):
        for u in range(W):
            # a prior centre anywhere from below the range to above it
            mu = float(rng.uniform(d0 - 3.0, d1 + 3.0))
            inside = 1
            J, S_init = BF.em_pixel_table(feat, ls, ld, imgs, b, u, v, dvals, mu, inside, p)
            seg_ub = _seg_max(ls, ld, b, u, v, dvals, W)
            lp = np.array([_log_prior(d, mu, inside, gamma, sigma) for d in dvals])
            # the per-candidate bound covers every label vector
            assert np.all(J <= lp[:, None] + seg_ub + 1e-12)
            j_prev = None
            S = None
            for t in range(iters):
                col = J[np.arange(D), S_init] if t == 0 else J[:, S]
                if t == 0:
                    # reference candidate: the one nearest mu, lowest index on a tie
                    j_ref = int(np.argmin([abs(d - mu) for d in dvals]))
                else:
                    j_ref = j_prev
                Js = col[j_ref]
                keep = _interval(Js, seg_ub, mu, gamma, sigma, dvals)
                keep[j_ref] = True
                j = int(np.argmax(col))
                assert keep[j], (u, v, t)
                # everything skipped is strictly below the reference objective
                assert np.all(col[~keep] < Js)
                pruned += int(np.count_nonzero(~keep))
                total += D
                S = int(np.argmax(J[j]))
                j_prev = j
    # the rule is not vacuous on these frames
    assert pruned > 0


def test_interval_rejects_a_planted_sign_error():
    """The same check with the prior's exponent sign flipped in the bound
    (exp(+r^2 / 2 sigma^2)) keeps the wrong candidates, and some column's
    arg-max falls outside: the check can fail."""
    K, H, W, D = 3, 3, 14, 17
    imgs, seg, b, rng = _frame(K, H, W, 9)
    p = O.Params(beta=200.0, gamma=0.1, sigma=1.5)
    feat = BF.descriptors(imgs)
    ls, ld = _log_maps(seg, p.eps)
    dvals = [j * 0.5 for j in range(D)]
    missed = 0
    for v in range(H):
        for u in range(W):
            mu = float(rng.uniform(-2.0, 10.0))
            J, S_init = BF.em_pixel_table(feat, ls, ld, imgs, b, u, v, dvals, mu, 1, p)
            seg_ub = _seg_max(ls, ld, b, u, v, dvals, W)
            col = J[np.arange(D), S_init]
            j_ref = int(np.argmin([abs(d - mu) for d in dvals]))
            Js = col[j_ref]
            e = np.exp(Js - seg_ub)
            if e <= p.gamma:
                continue
            r2_wrong = 2.0 * p.sigma ** 2 * np.log(e - p.gamma)     # sign dropped
            keep = (np.asarray(dvals) - mu) ** 2 <= r2_wrong
            keep[j_ref] = True
            missed += int(not keep[int(np.argmax(col))])
    assert missed > 0


@pytest.mark.parametrize("K,beta,seed", [(7, 5.0, 11), (8, 5.0, 12), (7, 20.0, 13)])
def test_label_block_bound_never_skips_the_e_step_argmax(K, beta, seed):
    """From seven cameras the E-step runs 2^(K-6) blocks of 64 label vectors
    sharing cameras 6..K-1.  A block's objectives are at most
    base + sum over its high static cameras of a_k + sum over cameras 0..5 of
    max(a_k, 0), with a_k = log p(static) - log p(dynamic) of ray k and base
    = log prior + sum_k log p(dynamic); blocks below the all-static vector's
    objective never hold the row's arg-max."""
    H, W, D = 2, 8, 5
    imgs, seg, b, rng = _frame(K, H, W, seed)
    # (a small beta keeps the all-static vector's variance term small, so
    # the bound skips blocks and the check is not vacuous)
    p = O.Params(beta=beta, gamma=0.1, sigma=2.0)
    feat = BF.descriptors(imgs)
    ls, ld = _log_maps(seg, p.eps)
    dvals = [j * 1.0 for j in range(D)]
    cols = np.arange(W, dtype=np.float64)
    skipped = 0
    for v in range(H):
        for u in range(W):
            mu = float(rng.uniform(-1.0, 5.0))
            J, _ = BF.em_pixel_table(feat, ls, ld, imgs, b, u, v, dvals, mu, 1, p)
            for j, d in enumerate(dvals):
                row = J[j]
                xs = [u - d * float(b[k]) for k in range(K)]
                sls = np.array([np.interp(xs[k], cols, ls[k, v]) for k in range(K)])
                sld = np.array([np.interp(xs[k], cols, ld[k, v]) for k in range(K)])
                a = sls - sld
                base = _log_prior(d, mu, 1, p.gamma, p.sigma) + float(np.sum(sld))
                seed_obj = row[(1 << K) - 1]
                best = int(np.argmax(row))
                low_pos = float(np.sum(np.maximum(a[:6], 0.0)))
                for h in range(1 << (K - 6)):
                    hi_sum = float(sum(a[6 + i] for i in range(K - 6) if h >> i & 1))
                    bound = base + hi_sum + low_pos
                    block = np.arange(h << 6, (h + 1) << 6)
                    assert np.all(row[block] <= bound + 1e-12)
                    if bound < seed_obj:
                        skipped += 1
                        assert not (block[0] <= best < block[-1] + 1)
    assert skipped > 0


def _interval_f32(mu, Js, seg_ub, gamma, inv2s2, d0, inv_step, D, js):
    """The candidate interval in float32 with the slacks the sweep applies:
    J* lowered by 2^-18 (1 + |J*|) and 1e-3 (the hardware exp2 / log2 of the
    prior), the radius widened by 0.1 % + 1e-3, one more candidate each side,
    the reference candidate always kept; everything when theta is below
    -87 (exp(theta) would leave float32's normal range, where its log is no
    longer theta), exp(theta) - gamma is not in (0, 1) or J* is not
    finite."""
    f = np.float32
    if not abs(Js) <= f(3.0e38):
        return 0, D - 1
    th = f(f(f(Js - f(f(1) + f(abs(Js))) * f(2.0 ** -18)) - seg_ub) - f(1e-3))
    if not th >= f(-87.0):
        return 0, D - 1
    A = f(np.exp(th, dtype=np.float32) - gamma)
    if not (A > 0 and A < 1):
        return 0, D - 1
    r = f(f(np.sqrt(f(-np.log(A, dtype=np.float32) / inv2s2), dtype=np.float32)) * f(1.001) + f(1e-3))
    flo = max(f(f(mu - r - d0) * inv_step), f(-2))
    fhi = min(f(f(mu + r - d0) * inv_step), f(D) + f(1))
    return min(max(int(np.floor(flo)) - 1, 0), js), max(min(int(np.ceil(fhi)) + 1, D - 1), js)


@pytest.mark.parametrize("flush", [True, False])
def test_float32_interval_keeps_every_candidate_that_can_reach_the_reference(flush):
    """Random candidate grids (|d| up to 1000, the finest spacing pruning is
    enabled for, 2^-12 max(1, |d|), up to 1024 candidates), sigma from 1e-3
    to 100, gamma 0 or 1e-6 to 10, prior centres far outside the grid: no
    candidate whose float32 bound (log prior, raised by 1e-5 for the
    hardware exp2 / log2, plus seg_max) reaches J* falls outside the
    interval, whether the prior's exponential flushes results below the
    normal float32 range to 0 (the rectified sweep's exp2) or keeps them
    as denormals."""
    f = np.float32
    tiny = np.finfo(np.float32).tiny
    rng = np.random.default_rng(20)
    cases = 0
    pruned = 0.0
    while cases < 20000:
        D = int(rng.integers(2, 1025))
        dmag = 10 ** rng.uniform(-1, 3)
        d0 = rng.uniform(-dmag, dmag)
        step = 10 ** rng.uniform(np.log10(max(1.0, abs(d0)) / 4096.0), np.log10(max(1.0, abs(d0)) / 4096.0) + 4)
        d1 = d0 + step * (D - 1)
        if step < max(1.0, abs(d0), abs(d1)) / 4096.0:
            continue
        dval = (d0 + np.arange(D) * ((d1 - d0) / (D - 1))).astype(np.float32)
        sigma = 10 ** rng.uniform(-3, 2)
        inv2s2 = f(1.0 / (2.0 * sigma * sigma))
        gamma = f(0.0) if rng.random() < 0.2 else f(10 ** rng.uniform(-6, 1))
        mu = f(rng.uniform(float(dval[0]) - 50 * sigma, float(dval[-1]) + 50 * sigma))
        seg_ub = f(rng.uniform(-20, 0))
        t = (dval - mu).astype(np.float32)
        e = np.exp(-(t * t) * inv2s2, dtype=np.float32)
        if flush:
            e = np.where(e < tiny, f(0), e)
        with np.errstate(divide="ignore"):
            prior = np.log(gamma + e, dtype=np.float32).astype(np.float64)
        js = int(np.argmin(np.abs(t))) if rng.random() < 0.7 else int(rng.integers(0, D))
        if not np.isfinite(prior[js]):
            continue
        Js = f(prior[js] + float(seg_ub) - rng.exponential(0.5))
        lo, hi = _interval_f32(mu, Js, seg_ub, gamma, inv2s2, f(dval[0]), f(1.0 / ((d1 - d0) / (D - 1))), D, js)
        outside = np.ones(D, bool)
        outside[lo:hi + 1] = False
        assert not np.any(outside & (prior + 1e-5 + float(seg_ub) >= float(Js))), (D, d0, step, sigma, gamma, mu)
        pruned += outside.mean()
        cases += 1
    assert pruned / cases > 0.1
