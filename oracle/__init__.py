"""FP64 CPU oracle of the non-ideal compressible LBM (test infrastructure).

Only tests/, __graft_entry__.smoke() and bench.py's cpu_baseline and
--impl reference legs may import this package; oracle/write_scenarios.py uses
it to write stored scalar constants.  The CUDA product path never imports it.
"""
from . import thermo, lbm  # noqa: F401
