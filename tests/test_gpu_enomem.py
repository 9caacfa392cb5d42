"""Out-of-memory paths of the C interface, with the failure injected by the
library's own test hook (lbm_debug_fail_alloc) instead of exhausting the
GPU's memory: every device allocation of create + init + shock capturing, and
of a batch, is failed in turn; each failure must come back as LBM_ENOMEM, leave
no device memory behind, and leave the library usable."""
import numpy as np
import pytest

import inputs

pytestmark = pytest.mark.gpu

P = pytest.importorskip("paper_2510_14712_gb300")


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2510_14712_gb300 import build
    build.build()
    P.load()


def free_bytes():
    import torch
    torch.cuda.synchronize()
    return torch.cuda.mem_get_info()[0]


def handle_lifecycle(case):
    s = P.Solver(case, precision="fp32")
    try:
        P.lbm_set_shock_capturing(s.h, 0.1, 0.0, 0.1)       # allocates the shock-capturing planes
        s.init().step(2)
        return s.fields()
    finally:
        s.close()


def test_every_handle_allocation_failure_is_enomem_without_leak():
    case = inputs.add_noise(inputs.tgv(shape=(24, 16, 12)), 1)
    want = handle_lifecycle(case)
    base = free_bytes()
    failures = 0
    for k in range(1, 40):
        P.lbm_debug_fail_alloc(k)
        try:
            handle_lifecycle(case)
            P.lbm_debug_fail_alloc(0)
            break                                          # k is past the last allocation
        except P.LbmError as e:
            P.lbm_debug_fail_alloc(0)
            assert e.code == P.LBM_ENOMEM, (k, e.code, str(e))
            failures += 1
        assert free_bytes() == base, "device memory left behind after failing allocation %d" % k
    assert failures >= 8                                   # partials, totals, status, 2 x populations, scratch, io, shock
    got = handle_lifecycle(case)                           # the library still works and gives the same result
    for key in ("rho", "u", "T"):
        assert np.array_equal(got[key], want[key])


def batch_lifecycle(cases):
    b = P.Batch(cases, precision="fp32")
    try:
        b.init()
        b.step(2)
    finally:
        b.close()


def test_every_batch_allocation_failure_is_enomem_without_leak():
    cases = inputs.batch(3)
    batch_lifecycle(cases)
    base = free_bytes()
    failures = 0
    for k in range(1, 60):
        P.lbm_debug_fail_alloc(k)
        try:
            batch_lifecycle(cases)
            P.lbm_debug_fail_alloc(0)
            break
        except P.LbmError as e:
            P.lbm_debug_fail_alloc(0)
            assert e.code == P.LBM_ENOMEM, (k, e.code, str(e))
            failures += 1
        assert free_bytes() == base, "device memory left behind after failing allocation %d" % k
    assert failures >= 3 * 7


def test_fail_alloc_rejects_negative():
    with pytest.raises(P.LbmError):
        P.lbm_debug_fail_alloc(-1)
