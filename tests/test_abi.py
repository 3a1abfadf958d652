"""The C-ABI library loads, exports every symbol its header declares, and its
host-only logic behaves (CPU; no compute call touches a GPU here)."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2003_11076_gb300 import build, lf
    build.build()
    return lf.load()


def _declared_functions():
    text = open(os.path.join(ROOT, "include", "lf.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(lf_[a-z_]+)\s*\(", text)))


def test_header_symbols_are_exported(lib):
    names = _declared_functions()
    assert len(names) >= 10
    for n in names:
        assert hasattr(lib, n), n
    from paper_2003_11076_gb300 import lf
    assert set(lf.EXPORTS) == set(names)


def test_library_is_built_for_sm_103a_only():
    from paper_2003_11076_gb300 import build
    assert build.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]


def test_default_params(lib):
    from paper_2003_11076_gb300 import lf
    p = lf.default_params()
    assert (p.beta, p.gamma, p.sigma, p.eps) == (200.0, pytest.approx(0.1), 2.0, pytest.approx(1e-4))
    assert p.seg_threshold == pytest.approx(0.7) and p.mstep_seg_term == 1 and p.early_exit == 1
    assert p.median == 0 and p.precision == lf.LF_PREC_F32
    assert p.em_mode == lf.LF_EM_HARD and p.dynamic_only == 0 and p.prune == 1


def test_params_and_stats_layouts_match_the_header():
    """The binding's ctypes structures list the fields of lf_params and
    lf_stats in the header's order (a field added on one side only would shift
    every field after it)."""
    from paper_2003_11076_gb300 import lf
    hdr = open(os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "lf.h")).read()
    hdr = re.sub(r"/\*.*?\*/", " ", hdr, flags=re.S)  # comments out
    for struct, cls in (("lf_params", lf.Params), ("lf_stats", lf.Stats)):
        body = hdr[hdr.index("typedef struct " + struct + " {") + len("typedef struct " + struct + " {"):]
        body = body[:body.index("} " + struct + ";")]
        names = []
        for decl in body.split(";"):
            words = decl.split()
            if words:  # "<type> a, b"
                names += [n for n in " ".join(words[1:]).replace(" ", "").split(",") if n]
        assert [f for f, _ in cls._fields_] == names, struct


@pytest.mark.parametrize("kw,expect", [
    (dict(K=0), "n_cams"), (dict(K=13), "n_cams"), (dict(b0=0.3), "reference"),
    (dict(H=2), "H and W"), (dict(D=0), "D must"), (dict(D=2000), "D must"),
    (dict(dmin=5.0, dmax=1.0), "d_min"),
])
def test_create_rejects_invalid_arguments(lib, kw, expect):
    from paper_2003_11076_gb300 import lf
    K = kw.get("K", 3)
    b = np.zeros(max(K, 1), np.float32)
    b[1:] = np.linspace(0.1, 0.3, max(K, 1) - 1)
    if "b0" in kw:
        b[0] = kw["b0"]
    h = ctypes.c_void_p()
    s = lib.lf_create(ctypes.byref(h), K, b.ctypes.data, kw.get("H", 16), 16, kw.get("dmin", 0.0),
                      kw.get("dmax", 7.0), kw.get("D", 8), None)
    assert s == lf.LF_EINVAL
    assert not h.value
    assert expect in lib.lf_last_error(None).decode()


def test_null_context_calls_fail_cleanly(lib):
    from paper_2003_11076_gb300 import lf
    assert lib.lf_run_em(None, 3, None, None, None, None, None, 0) == lf.LF_EINVAL
    assert lib.lf_synchronize(None) == lf.LF_EINVAL
    lib.lf_destroy(None)


def _tri_set(tris):
    return {tuple(sorted(t)) for t in np.asarray(tris).tolist()}


@pytest.mark.parametrize("seed,M", [(0, 3), (1, 10), (2, 40), (3, 300), (4, 1000)])
def test_host_delaunay_matches_qhull(lib, seed, M):
    """The library's Bowyer-Watson triangulation equals scipy's Qhull
    Delaunay triangulation (general position: the triangulation is unique)."""
    from scipy.spatial import Delaunay
    from paper_2003_11076_gb300 import lf
    rng = np.random.default_rng(seed)
    pts = np.stack([rng.uniform(0, 960, M), rng.uniform(0, 600, M), rng.uniform(0, 60, M)], 1).astype(np.float32)
    got = lf.triangulate(pts)
    ref = Delaunay(pts[:, :2].astype(np.float64)).simplices
    assert _tri_set(got) == _tri_set(ref)
    # counter-clockwise
    a, b, c = pts[got[:, 0], :2], pts[got[:, 1], :2], pts[got[:, 2], :2]
    area = (b[:, 0] - a[:, 0]) * (c[:, 1] - a[:, 1]) - (b[:, 1] - a[:, 1]) * (c[:, 0] - a[:, 0])
    assert np.all(area > 0)


def test_host_delaunay_degenerate_inputs(lib):
    from paper_2003_11076_gb300 import lf
    assert len(lf.triangulate(np.zeros((0, 3), np.float32))) == 0
    assert len(lf.triangulate(np.array([[0, 0, 1], [1, 1, 1]], np.float32))) == 0
    collinear = np.array([[0, 0, 1], [1, 1, 1], [2, 2, 1], [5, 5, 2]], np.float32)
    assert len(lf.triangulate(collinear)) == 0
    # repeated points keep their first occurrence; result as without repeats
    pts = np.array([[0, 0, 1], [10, 0, 2], [0, 10, 3], [10, 0, 9], [7, 8, 4]], np.float32)
    t = lf.triangulate(pts)
    assert 3 not in t
    sub = lf.triangulate(pts[[0, 1, 2, 4]])
    remap = np.array([0, 1, 2, 4])
    assert _tri_set(t) == _tri_set(remap[sub])
    assert lib.lf_triangulate(None, 3, None, 0) == -1


def test_package_never_imports_the_oracle():
    """The product path neither imports nor links the oracle."""
    pkg = os.path.join(ROOT, "paper_2003_11076_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".cpp", ".h")):
                src = open(os.path.join(dirpath, f)).read()
                assert not re.search(r"^\s*(from|import)\s+oracle", src, re.M), f
                assert "lf_oracle" not in src and "orc_" not in src, f


def _rect_cams(b):
    cams = np.zeros((len(b), 3, 4), np.float32)
    for k, bk in enumerate(b):
        cams[k, :, :3] = np.eye(3)
        cams[k, 0, 3] = -bk
    return cams


@pytest.mark.parametrize("case,expect", [
    ("no_reference", "[I | 0]"), ("nan", "non-finite"), ("behind", "behind the camera"),
    ("soft", "hard EM"), ("f16", "hard EM"), ("huge", "2^31"),
])
def test_create_calibrated_rejects_invalid_arguments(lib, case, expect):
    """Argument checks of lf_create_calibrated run before any device work."""
    from paper_2003_11076_gb300 import lf
    cams = _rect_cams([-0.2, 0.0, 0.2])
    p = lf.default_params()
    if case == "no_reference":
        cams[1, 0, 3] = 0.01
    elif case == "nan":
        cams[2, 1, 1] = np.nan
    elif case == "behind":
        cams[2, 2, 3] = -1.0  # Z = 1 - d: negative for d > 1
    elif case == "soft":
        p = lf.default_params(em_mode=lf.LF_EM_SOFT)
    elif case == "f16":
        p = lf.default_params(precision=lf.LF_PREC_F16)
    H = W = 16
    if case == "huge":  # 3 x 27000 x 27000 texels: past 32-bit map indices
        H = W = 27000
    h = ctypes.c_void_p()
    s = lib.lf_create_calibrated(ctypes.byref(h), 3, np.ascontiguousarray(cams).ctypes.data, H, W, 0.0, 7.0, 8,
                                 ctypes.byref(p))
    assert s == lf.LF_EINVAL
    assert not h.value
    assert expect in lib.lf_last_error(None).decode()
    assert lib.lf_create_calibrated(ctypes.byref(h), 3, None, 16, 16, 0.0, 7.0, 8, None) == lf.LF_EINVAL


def test_host_delaunay_of_grid_support_points_matches_qhull(lib):
    """Support points sit on a regular grid plus a fixed per-cell sub-pixel
    offset; with the offset the triangulation is unique, so the library's
    host Delaunay and Qhull agree on it."""
    from scipy.spatial import Delaunay
    from oracle import oracle as O
    from paper_2003_11076_gb300 import lf, scenes
    s = scenes.street_rgb(1, H=240, W=384, D=64, M=20)
    pts = O.support_points(s.images, s.seg_prior, s.baselines, s.d_min, s.d_max, s.D)["points"].astype(np.float32)
    assert pts.shape[0] > 1000
    assert _tri_set(lf.triangulate(pts)) == _tri_set(Delaunay(pts[:, :2].astype(np.float64)).simplices)


def _check_delaunay_valid(pts_xy, tris):
    """Exact validity of a Delaunay triangulation of integer points: every
    triangle counter-clockwise and non-degenerate, no input point strictly
    inside any circumcircle, triangle areas summing to the convex hull's,
    every edge shared by at most two triangles (hull edges by one)."""
    from scipy.spatial import ConvexHull
    P = [(int(x), int(y)) for x, y in pts_xy]
    uniq = sorted(set(P))
    area2 = 0
    edges = {}
    for a, b, c in np.asarray(tris).tolist():
        (ax, ay), (bx, by), (cx, cy) = P[a], P[b], P[c]
        o = (bx - ax) * (cy - ay) - (by - ay) * (cx - ax)
        assert o > 0, "triangle not counter-clockwise"
        area2 += o
        for dx, dy in uniq:
            adx, ady, bdx, bdy, cdx, cdy = ax - dx, ay - dy, bx - dx, by - dy, cx - dx, cy - dy
            det = ((adx * adx + ady * ady) * (bdx * cdy - cdx * bdy) + (bdx * bdx + bdy * bdy) * (cdx * ady - adx * cdy)
                   + (cdx * cdx + cdy * cdy) * (adx * bdy - bdx * ady))
            assert det <= 0, f"point {(dx, dy)} strictly inside the circumcircle of {(P[a], P[b], P[c])}"
        for e in ((a, b), (b, c), (c, a)):
            key = tuple(sorted((P[e[0]], P[e[1]])))
            edges[key] = edges.get(key, 0) + 1
    assert all(n <= 2 for n in edges.values())
    hull = ConvexHull(np.array(uniq, np.float64))
    assert area2 == int(round(2 * hull.volume))
    used = {P[i] for t in np.asarray(tris).tolist() for i in t}
    assert used == set(uniq)


@pytest.mark.parametrize("case", ["lattice", "lattice_holes", "circle", "lattice_repeats", "collinear_rows"])
def test_host_delaunay_degenerate_sets_are_valid(lib, case):
    """Sets whose Delaunay triangulation is not unique (cocircular lattice
    squares, lattice points on one circle, repeats, long collinear runs on
    the hull): the host triangulation is a valid one, checked exactly."""
    from paper_2003_11076_gb300 import lf
    rng = np.random.default_rng(7)
    if case == "lattice":
        xy = [(x, y) for y in range(0, 60, 5) for x in range(0, 90, 5)]
    elif case == "lattice_holes":
        xy = [(x, y) for y in range(0, 60, 5) for x in range(0, 90, 5) if rng.uniform() > 0.3]
    elif case == "circle":  # the 12 lattice points at distance 5 from the origin, the origin, a far point
        xy = [(5, 0), (4, 3), (3, 4), (0, 5), (-3, 4), (-4, 3), (-5, 0), (-4, -3), (-3, -4), (0, -5), (3, -4),
              (4, -3), (0, 0), (20, 1)]
    elif case == "lattice_repeats":
        base = [(x, y) for y in range(0, 40, 4) for x in range(0, 40, 4)]
        xy = base + [base[i] for i in rng.integers(0, len(base), 30)]
    else:
        xy = [(x, 0) for x in range(0, 100, 2)] + [(x, 50) for x in range(0, 100, 2)] + [(50, 25), (10, 30)]
    pts = np.array([(x, y, 1.0) for x, y in xy], np.float32)
    tris = lf.triangulate(pts)
    assert len(tris) > 0
    _check_delaunay_valid(pts[:, :2], tris)


def test_delaunay_validity_check_catches_a_wrong_flip():
    """The exact checker above rejects a triangulation with a non-Delaunay
    edge (the long diagonal of a thin quadrilateral)."""
    xy = np.array([(0, 0), (10, 0), (12, 3), (0, 2)], np.float64)
    good = np.array([(0, 1, 3), (1, 2, 3)])   # diagonal 1-3 (short)
    bad = np.array([(0, 1, 2), (0, 2, 3)])    # diagonal 0-2 (long)
    _check_delaunay_valid(xy, good)
    with pytest.raises(AssertionError):
        _check_delaunay_valid(xy, bad)


@pytest.mark.parametrize("field,value,expect", [
    ("sigma", 0.0, "sigma"), ("sigma", 1e-20, "sigma too small"),
    ("seg_threshold", 1.0, "seg_threshold"), ("seg_threshold", 0.0, "seg_threshold"),
    ("eps", 0.0, "eps"), ("gamma", -1.0, "gamma"), ("beta", float("nan"), "non-finite"),
    ("precision", 7, "precision"), ("em_mode", 9, "em_mode"),
])
def test_create_and_static_entry_check_params_alike(lib, field, value, expect):
    """lf_create and the allocation-free lf_run_em_static share one parameter
    check; both reject before any device work (so this runs without a GPU)."""
    from paper_2003_11076_gb300 import lf
    p = lf.default_params()
    setattr(p, field, value)
    b = np.array([-0.1, 0.0, 0.1], np.float32)
    h = ctypes.c_void_p()
    assert lib.lf_create(ctypes.byref(h), 3, b.ctypes.data, 16, 16, 0.0, 7.0, 8, ctypes.byref(p)) == lf.LF_EINVAL
    assert not h.value and expect in lib.lf_last_error(None).decode()
    img = np.zeros((3, 16, 16), np.float32)  # host stand-ins: never dereferenced on this path
    mu = np.zeros((16, 16), np.float32)
    didx = np.zeros((16, 16), np.int32)
    s = lib.lf_run_em_static(3, b.ctypes.data, 16, 16, 0.0, 7.0, 8, ctypes.byref(p), 3, img.ctypes.data, 1,
                             lf.LF_F32, img.ctypes.data, mu.ctypes.data, didx.ctypes.data, None, None, None, None)
    assert s == lf.LF_EINVAL
    assert expect in lib.lf_last_error(None).decode()


def test_static_entry_rejects_dynamic_only(lib):
    from paper_2003_11076_gb300 import lf
    p = lf.default_params(dynamic_only=1)
    b = np.array([-0.1, 0.0, 0.1], np.float32)
    img = np.zeros((3, 16, 16), np.float32)
    mu = np.zeros((16, 16), np.float32)
    didx = np.zeros((16, 16), np.int32)
    s = lib.lf_run_em_static(3, b.ctypes.data, 16, 16, 0.0, 7.0, 8, ctypes.byref(p), 3, img.ctypes.data, 1,
                             lf.LF_F32, img.ctypes.data, mu.ctypes.data, didx.ctypes.data, None, None, None, None)
    assert s == lf.LF_EINVAL and "dynamic_only" in lib.lf_last_error(None).decode()


def test_host_alloc_rejects_bad_arguments(lib):
    from paper_2003_11076_gb300 import lf
    p = ctypes.c_void_p()
    assert lib.lf_host_alloc(ctypes.byref(p), 0) == lf.LF_EINVAL and not p.value
    assert lib.lf_host_alloc(None, 64) == lf.LF_EINVAL
    lib.lf_host_free(None)  # a no-op


def test_binding_fails_loudly_without_the_library(monkeypatch, tmp_path):
    """No fallback: with the library absent every entry of the binding raises
    instead of computing anything on the host."""
    from paper_2003_11076_gb300 import lf
    monkeypatch.setattr(lf, "_lib", None)
    missing = str(tmp_path / "liblf.so")
    with pytest.raises(ImportError, match="missing"):
        lf.load(missing)
    monkeypatch.setattr(lf, "LIB_PATH", missing)
    monkeypatch.setattr(lf.load, "__defaults__", (missing,))
    with pytest.raises(ImportError, match="missing"):
        lf.Context(np.array([-0.1, 0.0, 0.1], np.float32), 16, 16, 0.0, 7.0, 8)
