"""Brute-force restatement of the per-pixel EM for tiny inputs.

TEST INFRASTRUCTURE ONLY (imported by the CPU test-suite).  It pins the C
oracle from outside: every quantity is computed by a different route than the
C core uses --

* descriptors: Sobel through ``scipy.ndimage.correlate`` (mode 'nearest');
* ray sampling: ``numpy.interp``, whose end-point clamping is the
  clamp-to-edge reading of out-of-image rays; for a calibrated array,
  ``scipy.ndimage.map_coordinates`` (order 1, mode 'nearest') at positions
  from the camera matrices;
* variance of the static rays: the pairwise form
  ``Var = (1 / n^2) * sum_{i<j} |f_i - f_j|^2`` instead of mean-then-deviations;
* disparity prior: ``logaddexp(log gamma, -(d - mu)^2 / (2 sigma^2))``;
* the EM: the full table J[d, S] over every candidate and every label vector
  is formed first; the M-step is an arg-max down a column, the E-step an
  arg-max along a row (Sec. III-B schedule, Eqs. e-step / m-step).
"""
from __future__ import annotations

import itertools

import numpy as np
from scipy import ndimage

SOBEL_X = np.array([[-1.0, 0.0, 1.0], [-2.0, 0.0, 2.0], [-1.0, 0.0, 1.0]])


def descriptors(images: np.ndarray) -> np.ndarray:
    """[K,3,H,W] = [Y, Sobel-x/8, Sobel-y/8]."""
    imgs = np.asarray(images)
    x = imgs.astype(np.float64) / (255.0 if imgs.dtype == np.uint8 else 1.0)
    if x.ndim == 4:
        Y = x @ np.array([0.299, 0.587, 0.114])
    else:
        Y = x
    out = np.zeros((Y.shape[0], 3) + Y.shape[1:])
    for k in range(Y.shape[0]):
        out[k, 0] = Y[k]
        out[k, 1] = ndimage.correlate(Y[k], SOBEL_X, mode="nearest") / 8.0
        out[k, 2] = ndimage.correlate(Y[k], SOBEL_X.T, mode="nearest") / 8.0
    return out


def _interp(row: np.ndarray, x: float) -> float:
    return float(np.interp(x, np.arange(row.shape[0], dtype=np.float64), row))


def _interp2(img: np.ndarray, x: float, y: float) -> float:
    return float(ndimage.map_coordinates(img, [[y], [x]], order=1, mode="nearest")[0])


def _position(cam, u, v, d):
    """(x, y) in a calibrated camera: dehomogenised cam @ (u, v, 1, d)."""
    X = np.asarray(cam, np.float64) @ np.array([u, v, 1.0, d])
    return X[0] / X[2], X[1] / X[2]


def pairwise_variance(f: np.ndarray) -> float:
    n = f.shape[0]
    if n <= 1:
        return 0.0
    acc = 0.0
    for i in range(n):
        for j in range(i + 1, n):
            acc += float(np.sum((f[i] - f[j]) ** 2))
    return acc / (n * n)


def log_prior(d, mu, inside, gamma, sigma):
    if not inside:
        return 0.0
    return float(np.logaddexp(np.log(gamma), -((d - mu) ** 2) / (2.0 * sigma * sigma)))


def em_pixel_table(feat, ls, ld, images, baselines, u, v, dvals, mu, inside, p, cameras=None):
    """J[d_j, S] for every candidate and every label vector, plus the
    per-candidate initial label vector S(d_j) and the sampled images."""
    K = feat.shape[0]
    D = len(dvals)
    nS = 1 << K
    J = np.zeros((D, nS))
    S_init = np.zeros(D, dtype=np.int64)
    thr = p.seg_threshold
    for j, d in enumerate(dvals):
        if cameras is None:
            xs = [u - d * float(baselines[k]) for k in range(K)]
            f = np.array([[_interp(feat[k, c, v], xs[k]) for c in range(3)] for k in range(K)])
            sls = np.array([_interp(ls[k, v], xs[k]) for k in range(K)])
            sld = np.array([_interp(ld[k, v], xs[k]) for k in range(K)])
        else:
            pos = [_position(cameras[k], u, v, d) for k in range(K)]
            f = np.array([[_interp2(feat[k, c], *pos[k]) for c in range(3)] for k in range(K)])
            sls = np.array([_interp2(ls[k], *pos[k]) for k in range(K)])
            sld = np.array([_interp2(ld[k], *pos[k]) for k in range(K)])
        lp = log_prior(d, mu, inside, p.gamma, p.sigma)
        # initial threshold: static iff the normalised dynamic probability of
        # the two interpolated log-priors is below thr
        pd = np.exp(sld) / (np.exp(sld) + np.exp(sls))
        S_init[j] = sum(1 << k for k in range(K) if pd[k] < thr)
        for S in range(nS):
            members = [k for k in range(K) if S >> k & 1]
            var = pairwise_variance(f[members]) if members else 0.0
            seg = sum(sls[k] if S >> k & 1 else sld[k] for k in range(K))
            J[j, S] = -p.beta * var + lp + seg
    return J, S_init


def _softmax(row: np.ndarray) -> np.ndarray:
    q = np.exp(row - row.max())
    return q / q.sum()


def run(images, seg_prior, baselines, mu, inside, d_min, d_max, D, iters, p, mode: str = "hard",
        cameras=None):
    """EM on every pixel of a tiny frame from the full J[d, S] table.

    mode "hard": the paper's EM (M-step down the column of the current S,
    E-step along the row of the current d).  "soft": after the first
    iteration the M-step maximises the table's rows averaged under the
    previous row's softmax, ``J @ q``.  "joint": the arg-max of the whole
    table.  Returns dict like the oracle's (d_idx, labels, post, refocus)
    plus ``joint_max`` = max over (d, S) and, per iteration, ``L_t`` = the
    log-sum-exp of the row of d_t.  ``cameras`` ([K,3,4]): a calibrated array
    (the reference is the camera whose matrix is [I | 0])."""
    imgs = np.asarray(images)
    K, H, W = imgs.shape[:3]
    feat = descriptors(imgs)
    P = np.asarray(seg_prior, np.float64)
    ls = np.log(np.maximum(1.0 - P, p.eps))
    ld = np.log(np.maximum(P, p.eps))
    dvals = [float(d_min)] if D == 1 else [float(d_min) + j * ((float(d_max) - float(d_min)) / (D - 1))
                                            for j in range(D)]
    x = imgs.astype(np.float64) / (255.0 if imgs.dtype == np.uint8 else 1.0)
    if x.ndim == 3:
        x = x[..., None]
    C = x.shape[3]
    if cameras is None:
        ref = int(np.flatnonzero(np.asarray(baselines) == 0)[0])
    else:
        eye = np.hstack([np.eye(3), np.zeros((3, 1))])
        ref = next(k for k in range(K) if np.array_equal(np.asarray(cameras[k], np.float64), eye))
    out = {k: None for k in ("d_idx", "labels", "post", "refocus", "J_final", "joint_max")}
    d_idx = np.zeros((H, W), np.int64)
    labels = np.zeros((H, W), np.int64)
    post = np.zeros((K, H, W))
    refocus = np.zeros((H, W, C))
    J_final = np.zeros((H, W))
    joint = np.zeros((H, W))
    L_t = np.zeros((iters, H, W))
    for v in range(H):
        for u in range(W):
            J, S_init = em_pixel_table(feat, ls, ld, imgs, baselines, u, v, dvals, mu[v, u], inside[v, u], p,
                                       cameras)
            if not p.mstep_seg_term:
                raise NotImplementedError
            S = None
            q = None
            if mode == "joint":
                j, S = (int(i) for i in np.unravel_index(int(np.argmax(J)), J.shape))  # row-major first maximum
            else:
                for t in range(iters):
                    if t == 0:
                        col = J[np.arange(len(dvals)), S_init]
                    elif mode == "soft":
                        col = J @ q
                    else:
                        col = J[:, S]
                    j = int(np.argmax(col))          # first maximum = lowest index
                    S = int(np.argmax(J[j]))          # first maximum = smallest mask
                    q = _softmax(J[j])
                    L_t[t, v, u] = np.log(np.sum(np.exp(J[j] - J[j].max()))) + J[j].max()
            d_idx[v, u], labels[v, u] = j, S
            J_final[v, u] = J[j, S]
            joint[v, u] = J.max()
            row = J[j]
            q = np.exp(row - row.max())
            q /= q.sum()
            for k in range(K):
                post[k, v, u] = sum(q[s] for s in range(1 << K) if s >> k & 1)
            members = [k for k in range(K) if S >> k & 1]
            if not members:
                refocus[v, u] = x[ref, v, u]
            elif cameras is None:
                for c in range(C):
                    refocus[v, u, c] = np.mean([_interp(x[k, v, :, c], u - dvals[j] * float(baselines[k]))
                                                for k in members])
            else:
                for c in range(C):
                    refocus[v, u, c] = np.mean([_interp2(x[k, :, :, c], *_position(cameras[k], u, v, dvals[j]))
                                                for k in members])
    out.update(d_idx=d_idx, labels=labels, post=post, refocus=refocus[..., 0] if C == 1 else refocus,
               J_final=J_final, joint_max=joint, L_t=L_t)
    return out


def all_label_vectors(K):
    return list(itertools.product((0, 1), repeat=K))


# ------------------------------------------------------------ support points

def support_points(images, seg_prior, baselines, d_min, d_max, D, sp):
    """The support points of support_oracle.c restated with array operations
    (scipy integer Sobel, padded descriptor windows, the whole cost table per
    point).  Returns the per-cell arrays like ``oracle.support_points``."""
    imgs = np.asarray(images)
    K, H, W = imgs.shape[:3]
    if imgs.dtype == np.uint8:
        q = imgs.astype(np.int64)
    else:
        q = np.clip(np.rint(np.float32(255.0) * imgs.astype(np.float32)), 0, 255).astype(np.int64)
    Y = q if q.ndim == 3 else (77 * q[..., 0] + 150 * q[..., 1] + 29 * q[..., 2] + 128) >> 8
    kx = np.array([[-1, 0, 1], [-2, 0, 2], [-1, 0, 1]])
    gx = np.stack([ndimage.correlate(Y[k], kx, mode="nearest") for k in range(K)])
    gy = np.stack([ndimage.correlate(Y[k], kx.T, mode="nearest") for k in range(K)])
    # descriptor windows: [K, H, W, 18]
    pad = lambda a: np.pad(a, ((0, 0), (1, 1), (1, 1)), mode="edge")
    gxp, gyp = pad(gx), pad(gy)
    desc = np.concatenate([np.stack([gxp[:, 1 + dy:1 + dy + H, 1 + dx:1 + dx + W] for dy in (-1, 0, 1)
                                     for dx in (-1, 0, 1)], -1),
                           np.stack([gyp[:, 1 + dy:1 + dy + H, 1 + dx:1 + dx + W] for dy in (-1, 0, 1)
                                     for dx in (-1, 0, 1)], -1)], -1)
    tex = np.abs(desc).sum(-1)
    P = np.asarray(seg_prior, np.float32)
    Pp = np.pad(P, ((0, 0), (1, 1), (1, 1)), mode="edge")
    win_static = np.all(np.stack([Pp[:, 1 + dy:1 + dy + H, 1 + dx:1 + dx + W] for dy in (-1, 0, 1)
                                  for dx in (-1, 0, 1)], -1) < np.float32(sp.seg_threshold), -1)
    b = np.asarray(baselines, np.float32).astype(np.float64)
    ref = int(np.flatnonzero(b == 0)[0])
    dval = np.array([float(d_min)] if D == 1 else
                    [float(d_min) + j * ((float(d_max) - float(d_min)) / (D - 1)) for j in range(D)])
    step = (float(d_max) - float(d_min)) / (D - 1) if D > 1 else 0.0
    g, h = sp.grid, sp.grid // 2
    nx, ny = (W + g - 1) // g, (H + g - 1) // g
    cell_j = np.full((ny, nx), -1, np.int64)
    cell_src = np.full((ny, nx), -1, np.int64)
    cell_u = np.zeros((ny, nx))
    cell_v = np.zeros((ny, nx))

    def match(s, targets, u, v):
        if tex[s, v, u] < sp.texture or D < 2 or step <= 0:
            return -1
        bmax = max(abs(b[t] - b[s]) for t in targets)
        if bmax <= 0:
            return -1
        delta = int(np.ceil(1.0 / (bmax * step)))
        costs = np.full(D, -1, np.int64)
        for j in range(D):
            xs = [u + int(np.floor(-dval[j] * (b[t] - b[s]) + 0.5)) for t in targets]
            if any(x < 0 or x > W - 1 for x in xs):
                continue
            costs[j] = sum(int(np.abs(desc[s, v, u] - desc[t, v, x]).sum()) for t, x in zip(targets, xs))
        valid = np.flatnonzero(costs >= 0)
        if valid.size == 0:
            return -1
        best = int(valid[np.argmin(costs[valid])])      # first minimum
        far = valid[np.abs(valid - best) >= delta]
        if far.size == 0:
            return -1
        return best if 100 * costs[best] < sp.ratio_pct * costs[far].min() else -1

    others = [t for t in range(K) if t != ref]
    for cj in range(ny):
        for ci in range(nx):
            u, v = g * ci + h, g * cj + h
            if u > W - 1 or v > H - 1 or not win_static[ref, v, u]:
                continue
            j = match(ref, others, u, v)
            if j >= 0:
                cell_j[cj, ci], cell_src[cj, ci], cell_u[cj, ci], cell_v[cj, ci] = j, ref, u, v
    for s in others:
        targets = [t for t in others if t != s]
        if not targets:
            continue
        for cj in range(ny):
            for ci in range(nx):
                u, v = g * ci + h, g * cj + h
                if u > W - 1 or v > H - 1 or not win_static[s, v, u]:
                    continue
                j = match(s, targets, u, v)
                if j < 0:
                    continue
                ur = u + dval[j] * b[s]
                if ur < 0 or ur > W - 1 or P[ref, v, int(np.floor(ur + 0.5))] < np.float32(sp.seg_threshold):
                    continue
                c = (cj, int(np.floor(ur / g)))
                if cell_j[c] >= 0:
                    continue
                cell_j[c], cell_src[c], cell_u[c], cell_v[c] = j, s, ur, v
    keep = np.zeros_like(cell_j, bool)
    for cj in range(ny):
        for ci in range(nx):
            if cell_j[cj, ci] < 0:
                continue
            win = cell_j[max(cj - sp.window, 0):cj + sp.window + 1, max(ci - sp.window, 0):ci + sp.window + 1]
            near = win[win >= 0]
            agree = np.sum(np.abs(dval[near] - dval[cell_j[cj, ci]]) <= sp.delta) - 1  # not itself
            keep[cj, ci] = agree >= sp.min_support
    cell_j[~keep] = -1
    cell_src[~keep] = -1
    cell_u[~keep] = 0.0
    cell_v[~keep] = 0.0
    return {"cell_j": cell_j, "cell_src": cell_src, "cell_u": cell_u, "cell_v": cell_v}
