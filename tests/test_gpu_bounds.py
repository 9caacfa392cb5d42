"""Bounds-check build: the library compiled with -DLBM_BOUNDS_CHECK checks
every population access of the step kernels against the handle's buffers
(an access outside is skipped and counted, nothing traps).  The cases of
tests/bounds_cases.py -- the 8^3 and 16x4 boxes, stage A by quads of x nodes
and its scalar fallback, ghost and wall fills, the multi-pass and batched
steps -- run in a child process on that build: no access may fall outside,
and the fields must agree with the regular build's to the rounding of each
case's precision (the two builds contract multiply-adds differently)."""
import os
import subprocess
import sys

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

P = pytest.importorskip("paper_2510_14712_gb300")
HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2510_14712_gb300 import build
    build.build()
    P.load()


def test_bounds_check_build_finds_no_out_of_buffer_access(tmp_path):
    from paper_2510_14712_gb300 import build
    lib_bc = build.build(bounds_check=True)
    out = str(tmp_path / "bc.npz")
    env = dict(os.environ, LBM_LIBRARY=lib_bc)
    r = subprocess.run([sys.executable, os.path.join(HERE, "bounds_cases.py"), out], env=env,
                       capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stderr[-3000:]
    got = np.load(out)
    assert int(got["violations"]) == 0, "population accesses outside the buffers: %d" % int(got["violations"])
    assert P.lbm_debug_bounds_violations() == -1        # the regular build has no checks
    import bounds_cases
    want = bounds_cases.run_all(P)
    # the checks change no arithmetic, but the code around each access changes
    # shape, and with it the compiler's choice of fused multiply-adds: results
    # agree to the rounding of the build's precision, not bit for bit (FP32:
    # 1e-4 over 12 steps of boxes with 1% noise, where u is small)
    for k, v in want.items():
        tol = 1e-12 if "fp64" in k else (1e-3 if "fp16" in k else 1e-4)
        err = np.linalg.norm((got[k] - v).ravel()) / max(np.linalg.norm(v.ravel()), 1e-300)
        assert err <= tol, (k, err)
