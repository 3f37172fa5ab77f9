"""The C oracle under AddressSanitizer and UndefinedBehaviorSanitizer: a
small forward and backward (projection, binning, compositing, analytic
backward, pose twist) runs with no out-of-bounds access, use after free or
undefined arithmetic. CPU only; skipped where gcc has no sanitizer runtime."""
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

SCRIPT = r"""
import sys
sys.path.insert(0, {root!r})
import numpy as np
from oracle import oracle as O
O._LIB = {lib!r}
from paper_2509_25191_gb300 import synth
sc, vw = synth.uneven_scenes(seeds=(1, 2), sizes=(300, 200), views_per_scene=2,
                             resolutions=((45, 31), (64, 48)))
fwd = O.forward(sc, vw, 16, 16)
ups = [np.random.default_rng(v).standard_normal(f["image"].shape) for v, f in enumerate(fwd)]
grads, dRt, tw, _ = O.backward(sc, vw, fwd, ups, 16, 16)
assert O.lib()._name == {lib!r}
maps = open("/proc/self/maps").read()
assert "libasan" in maps and "liboracle_san" in maps
assert all(np.isfinite(f["image"]).all() for f in fwd)
assert all(np.isfinite(g).all() for g in grads.values()) and np.isfinite(dRt).all() and np.isfinite(tw).all()
print("sanitized oracle ok")
"""


def test_oracle_runs_clean_under_asan_and_ubsan(tmp_path):
    asan = subprocess.run(["gcc", "-print-file-name=libasan.so"], capture_output=True, text=True).stdout.strip()
    if not os.path.isabs(asan) or not os.path.exists(asan):
        pytest.skip("gcc has no AddressSanitizer runtime here")
    lib = str(tmp_path / "liboracle_san.so")
    subprocess.check_call(["gcc", "-std=c11", "-O1", "-g", "-ffp-contract=off", "-fno-fast-math",
                           "-fsanitize=address,undefined", "-fno-sanitize-recover=undefined",
                           "-fno-omit-frame-pointer", "-fPIC", "-shared", "-o", lib,
                           os.path.join(ROOT, "oracle", "gs_oracle.c"), "-lm"])
    env = dict(os.environ, LD_PRELOAD=asan, ASAN_OPTIONS="detect_leaks=0:abort_on_error=0",
               UBSAN_OPTIONS="print_stacktrace=1:halt_on_error=1")
    r = subprocess.run([sys.executable, "-c", SCRIPT.format(root=ROOT, lib=lib)], env=env,
                       capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-4000:]
    assert "sanitized oracle ok" in r.stdout
    assert "AddressSanitizer" not in r.stderr and "runtime error" not in r.stderr, r.stderr[-4000:]
