"""The C interface library builds, loads and exports every symbol include/lbm.h declares.

Runs without a GPU: argument validation happens before any CUDA call, so
invalid arguments must come back as LBM_EINVAL with a message.
"""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2510_14712_gb300 import build
    build.build()
    import paper_2510_14712_gb300 as P
    return P.load()


def declared_symbols():
    names = set()
    inc = os.path.join(ROOT, "include")
    for f in sorted(os.listdir(inc)):
        if f.endswith(".h"):
            src = re.sub(r"/\*.*?\*/", "", open(os.path.join(inc, f)).read(), flags=re.S)
            names.update(re.findall(r"\b(lbm_[a-z0-9_]+)\s*\(", src))
    return sorted(names)


def test_header_declares_expected_entry_points():
    names = declared_symbols()
    for core in ("lbm_create", "lbm_init", "lbm_step", "lbm_moments", "lbm_destroy"):
        assert core in names


def test_every_declared_symbol_is_exported(lib):
    import paper_2510_14712_gb300 as P
    for name in declared_symbols():
        assert hasattr(lib, name), name
    assert sorted(P.EXPORTS) == declared_symbols()


def test_invalid_arguments_rejected_without_gpu(lib):
    import paper_2510_14712_gb300 as P
    e = P.lbm_eos(kind=0, a=0.3, b=1 / 3, R=8 / 3, kappa=0.01, eta_over_mu=1.0, rho_ref=0.6, T_ref=0.15,
                  precision=1, closure=0)
    h = ctypes.c_void_p()
    assert lib.lbm_create(ctypes.byref(h), 10, 8, 8, 1, ctypes.byref(e), 0.1, 0.7, 8.0) == P.LBM_EINVAL
    assert b"lattice" in lib.lbm_last_error()
    assert lib.lbm_create(ctypes.byref(h), 9, 8, 8, 2, ctypes.byref(e), 0.1, 0.7, 8.0) == P.LBM_EINVAL
    assert lib.lbm_create(ctypes.byref(h), 27, 0, 8, 8, ctypes.byref(e), 0.1, 0.7, 8.0) == P.LBM_EINVAL
    assert lib.lbm_create(ctypes.byref(h), 27, 8, 8, 8, ctypes.byref(e), -1.0, 0.7, 8.0) == P.LBM_EINVAL
    e.b = 2.0
    assert lib.lbm_create(ctypes.byref(h), 27, 8, 8, 8, ctypes.byref(e), 0.1, 0.7, 8.0) == P.LBM_EINVAL
    e.b, e.kind = 1 / 3, 1
    assert lib.lbm_create(ctypes.byref(h), 27, 8, 8, 8, ctypes.byref(e), 0.1, 0.7, 8.0) == P.LBM_EINVAL
    e.kind, e.precision = 0, 7
    assert lib.lbm_create(ctypes.byref(h), 27, 8, 8, 8, ctypes.byref(e), 0.1, 0.7, 8.0) == P.LBM_EINVAL
    assert lib.lbm_create(None, 27, 8, 8, 8, ctypes.byref(e), 0.1, 0.7, 8.0) == P.LBM_EINVAL
    assert lib.lbm_destroy(None) == P.LBM_OK
    assert lib.lbm_step(None, 1) == P.LBM_EINVAL
    assert lib.lbm_moments(None, None, None, None, None) == P.LBM_EINVAL
    assert lib.lbm_population_bytes(None) == 0
    assert lib.lbm_tile_count(None) == P.LBM_EINVAL
    assert lib.lbm_set_tile(None, 0) == P.LBM_EINVAL
    assert lib.lbm_version().startswith(b"gb300")


def test_product_path_does_not_import_the_oracle():
    """The package and its sources never name the oracle (no CPU fallback)."""
    pkg = os.path.join(ROOT, "paper_2510_14712_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                text = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in text and "from oracle" not in text, f


def test_mlp_invalid_arguments_rejected_without_gpu(lib):
    import paper_2510_14712_gb300 as P
    h = ctypes.c_void_p()
    assert lib.lbm_mlp_create(None, 0.25, 1 / 3, 8 / 3, 8.0, 1) == P.LBM_EINVAL
    assert lib.lbm_mlp_create(ctypes.byref(h), 0.25, 1 / 3, -1.0, 8.0, 1) == P.LBM_EINVAL
    assert b"R > 0" in lib.lbm_mlp_last_error()
    assert lib.lbm_mlp_set_scaling(None, None) == P.LBM_EINVAL
    assert lib.lbm_mlp_attach(None, None) == P.LBM_EINVAL
    assert lib.lbm_mlp_loss_grad(None, None, None, 1, None, None) == P.LBM_EINVAL
    assert lib.lbm_mlp_train(None, None, None, 1, 64, 1, 1e-3, 1e-4, 0.0, 0, None) == P.LBM_EINVAL
    assert lib.lbm_get_closure(None) == P.LBM_CLOSURE_EXACT
    assert lib.lbm_mlp_destroy(None) == P.LBM_OK
