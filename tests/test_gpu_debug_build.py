"""The debug build (-DLF_DEBUG): every index into the sweep's shared-memory
carve-up is checked against its region (a violation is reported as LF_ECUDA
and the access clamped, so nothing leaves shared memory).  A small set of
frames covering the camera counts, tile shapes, staging paths, precisions
and modes runs through it in a separate process; every run must come back
without a violation and with the release build's results."""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CASES = r'''
import json, sys
import numpy as np
sys.path.insert(0, {root!r})
from paper_2003_11076_gb300 import lf, scenes
lf.load({lib!r})
cases = [
    ("small_gray", scenes.small_gray(0), {{}}),
    ("rgb", scenes.street_rgb(1, H=72, W=130, D=32, iters=5, M=40), {{}}),
    ("K1", scenes.small_gray(3, H=20, W=40, baselines=[0.0], D=8, iters=3, M=10), {{}}),
    ("K9", scenes.small_gray(4, H=24, W=70, baselines=[-0.4, -0.3, -0.2, -0.1, 0.0, 0.1, 0.2, 0.3, 0.4], D=24,
                             iters=4, M=15), {{}}),
    ("K12_ref0", scenes.small_gray(5, H=16, W=48, baselines=[0.0, 0.05, 0.1, 0.15, 0.2, 0.25, 0.3, 0.35, 0.4, 0.45,
                                                              0.5, 0.55], D=12, iters=3, M=10), {{}}),
    ("ragged", scenes.small_gray(6, H=37, W=75, M=12), {{}}),
    ("halo48", scenes.small_gray(7, H=40, W=160, baselines=[-1.0, -0.5, 0.0, 0.5, 1.0], D=48, iters=3), {{}}),
    ("D1024", scenes.small_gray(8, H=16, W=40, D=1024, iters=2, M=10), {{}}),
    ("f16", scenes.small_gray(9), {{"precision": 1}}),
    ("bf16", scenes.small_gray(10), {{"precision": 2}}),
    ("dynamic_only", scenes.small_gray(11), {{"dynamic_only": 1}}),
    ("soft", scenes.small_gray(12), {{"em_mode": 1}}),
    ("joint", scenes.small_gray(13), {{"em_mode": 2}}),
]
out = {{}}
for name, s, kw in cases:
    r = lf.run_scene(s, params=lf.default_params(**kw))
    out[name] = r["d_idx"].tolist()
print("RESULT " + json.dumps(out))
'''


def test_debug_build_checks_every_shared_memory_index():
    from paper_2003_11076_gb300 import build
    release = build.build()
    debug = build.build(debug=True)
    res = {}
    for lib in (release, debug):
        r = subprocess.run([sys.executable, "-c", CASES.format(root=ROOT, lib=lib)], capture_output=True,
                           text=True, timeout=900)
        assert r.returncode == 0, r.stdout[-3000:] + r.stderr[-3000:]
        line = [l for l in r.stdout.splitlines() if l.startswith("RESULT ")]
        res[lib] = json.loads(line[-1][len("RESULT "):])
    for name in res[release]:
        assert np.array_equal(np.asarray(res[release][name]), np.asarray(res[debug][name])), name
