"""Source hygiene of the committed tree (CPU only): nothing here may name
the batched-copy calls that faulted GPUs of this model's predecessor, change
a GPU setting, or run ncu with locked clocks."""
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _tracked_files():
    try:
        out = subprocess.run(["git", "ls-files"], cwd=ROOT, capture_output=True, text=True, check=True).stdout
    except (OSError, subprocess.CalledProcessError):
        pytest.skip("not a git checkout")
    here = os.path.relpath(os.path.abspath(__file__), ROOT)
    return [f for f in out.splitlines() if f and f != here and os.path.isfile(os.path.join(ROOT, f))]


def _text(path):
    with open(os.path.join(ROOT, path), "rb") as fh:
        data = fh.read()
    return data.decode("utf-8", errors="replace") if b"\0" not in data else None


def test_no_batched_copy_calls():
    # the names are assembled here so that this file does not spell them out
    names = [p + "Memcpy" + d + "BatchAsync" for p in ("cuda", "cu") for d in ("", "3D")]
    hits = []
    for f in _tracked_files():
        if f.endswith(".md"):
            continue
        t = _text(f)
        if t is not None:
            hits += [f"{f}: {n}" for n in names if n in t]
    assert not hits, hits


def test_no_gpu_setting_is_changed():
    """nvidia-smi only queries; no NVML setter; every ncu command line keeps
    the clocks unlocked."""
    setters = re.compile(r"nvidia-smi[^\n]*\s(-lgc|-rgc|-lmc|-rmc|-ac|-rac|-pm|-pl|-r|--gpu-reset|-mig|-c|-e)\b"
                         r"|nvmlDeviceSet|nvmlDeviceReset|cudaDeviceSetLimit\(cudaLimitPersisting")
    bad = []
    for f in _tracked_files():
        if f.endswith(".md"):
            continue
        t = _text(f)
        if t is None:
            continue
        bad += [f"{f}: {m.group(0)}" for m in setters.finditer(t)]
        for line in t.splitlines():
            s = line.strip().lstrip("#").strip()
            if re.match(r"^(ncu|.*&&\s*ncu)\s", s) and "--clock-control none" not in s:
                bad.append(f"{f}: ncu without --clock-control none: {s[:80]}")
    assert not bad, bad
