"""Python binding of the GB300 non-ideal compressible LBM library (include/lbm.h).

Argument marshalling only: every step of the method runs in the CUDA
kernels of ``_build/liblbm.so``.  The functions carry the names of the C
entry points; ``Solver`` is a small convenience wrapper around one handle.
Importing this package fails loudly when the library has not been built
(``python -m paper_2510_14712_gb300.build``); there is no CPU fallback.

Field arrays follow the C convention: interior nodes in the order
n = x + Nx (y + Ny z); as numpy arrays of shape ([Nz,] Ny, Nx).
"""
import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
# LBM_LIBRARY selects another build of the library (the bounds-check build,
# _build/liblbm_bc.so, of tests/test_gpu_bounds.py)
LIB_PATH = os.environ.get("LBM_LIBRARY") or os.path.join(_HERE, "_build", "liblbm.so")

LBM_D2Q9, LBM_D3Q27 = 9, 27
LBM_OK, LBM_EINVAL, LBM_ENOMEM, LBM_ECUDA, LBM_EUNSTABLE, LBM_ESTATE = 0, -1, -2, -3, -4, -5
LBM_FP64, LBM_FP32, LBM_FP16DEV = 0, 1, 2
LBM_CLOSURE_EXACT, LBM_CLOSURE_MLP = 0, 1
LBM_BC_PERIODIC, LBM_BC_OUTFLOW, LBM_BC_INFLOW, LBM_BC_WALL = 0, 1, 2, 3
LBM_EOS_VDW, LBM_EOS_PR = 0, 1
LBM_FACE_XLO, LBM_FACE_XHI = 0, 1
LBM_FLAG_NONFINITE, LBM_FLAG_NEGATIVE, LBM_FLAG_THETA, LBM_FLAG_PRESSURE = 1, 2, 4, 8
LBM_STEP_FUSED, LBM_STEP_MULTIPASS = 0, 1
PRECISIONS = {"fp64": LBM_FP64, "fp32": LBM_FP32, "fp16dev": LBM_FP16DEV}

# every symbol include/lbm.h declares (checked by tests/test_abi.py)
EXPORTS = ("lbm_create", "lbm_set_boundary", "lbm_set_stream", "lbm_init", "lbm_init_device",
           "lbm_step", "lbm_step_async", "lbm_sync", "lbm_moments", "lbm_moments_device",
           "lbm_get_flags", "lbm_population_bytes", "lbm_get_populations", "lbm_set_populations",
           "lbm_set_step_kernel", "lbm_autotune", "lbm_autotune_times", "lbm_tile_count", "lbm_set_tile",
           "lbm_set_graphs", "lbm_set_temperature_fp64", "lbm_get_temperature_fp64",
           "lbm_set_shock_capturing", "lbm_launch_count",
           "lbm_destroy",
           "lbm_last_error", "lbm_version", "lbm_debug_fail_alloc", "lbm_debug_bounds_violations",
           "lbm_totals_noalloc", "lbm_totals_noalloc_error",
           "lbm_batch_create", "lbm_batch_set_boundary", "lbm_batch_set_shock_capturing", "lbm_batch_set_stream",
           "lbm_batch_init",
           "lbm_batch_step", "lbm_batch_step_async", "lbm_batch_sync", "lbm_batch_moments", "lbm_batch_flags",
           "lbm_batch_autotune", "lbm_batch_nodes", "lbm_batch_launch_count", "lbm_batch_destroy",
           "lbm_batch_last_error",
           # include/lbm_mlp.h
           "lbm_mlp_create", "lbm_mlp_set_stream", "lbm_mlp_collect", "lbm_mlp_fit_scaling", "lbm_mlp_get_scaling",
           "lbm_mlp_set_scaling", "lbm_mlp_get_params", "lbm_mlp_set_params", "lbm_mlp_loss_grad", "lbm_mlp_train",
           "lbm_mlp_predict", "lbm_mlp_attach", "lbm_get_closure", "lbm_mlp_destroy", "lbm_mlp_last_error",
           "lbm_mlp_set_mma", "lbm_mlp_get_mma")
LBM_MLP_NPARAM, LBM_MLP_NSCALE = 4547, 10


class LbmError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("lbm error %d: %s" % (code, msg))
        self.code = code


class lbm_eos(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("a", ctypes.c_double), ("b", ctypes.c_double),
                ("R", ctypes.c_double), ("kappa", ctypes.c_double), ("eta_over_mu", ctypes.c_double),
                ("rho_ref", ctypes.c_double), ("T_ref", ctypes.c_double),
                ("precision", ctypes.c_int), ("closure", ctypes.c_int),
                ("Tc", ctypes.c_double), ("m", ctypes.c_double)]


_lib = None


def load():
    """The loaded shared library (raises ImportError when it is not built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError("CUDA library not built (%s missing): run "
                          "`python -m paper_2510_14712_gb300.build`" % LIB_PATH)
    lib = ctypes.CDLL(LIB_PATH)
    P, I, D, S = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_size_t
    dp = ctypes.POINTER(ctypes.c_double)
    sig = {
        "lbm_create": (I, [ctypes.POINTER(P), I, I, I, I, ctypes.POINTER(lbm_eos), D, D, D]),
        "lbm_set_boundary": (I, [P, I, I, dp]),
        "lbm_set_stream": (I, [P, P]),
        "lbm_init": (I, [P, P, P, P]),
        "lbm_init_device": (I, [P, P, P, P]),
        "lbm_step": (I, [P, I]),
        "lbm_step_async": (I, [P, I]),
        "lbm_sync": (I, [P]),
        "lbm_moments": (I, [P, P, P, P, P]),
        "lbm_moments_device": (I, [P, P, P, P, P]),
        "lbm_get_flags": (I, [P, ctypes.POINTER(ctypes.c_uint)]),
        "lbm_population_bytes": (S, [P]),
        "lbm_get_populations": (I, [P, P, S]),
        "lbm_set_populations": (I, [P, P, S]),
        "lbm_set_step_kernel": (I, [P, I]),
        "lbm_autotune": (I, [P, I, ctypes.POINTER(I), ctypes.POINTER(ctypes.c_float)]),
        "lbm_autotune_times": (I, [P, P, I]),
        "lbm_tile_count": (I, [P]),
        "lbm_set_tile": (I, [P, I]),
        "lbm_set_graphs": (I, [P, I]),
        "lbm_set_temperature_fp64": (I, [P, I]),
        "lbm_get_temperature_fp64": (I, [P]),
        "lbm_set_shock_capturing": (I, [P, D, D, D]),
        "lbm_launch_count": (ctypes.c_longlong, [P]),
        "lbm_destroy": (I, [P]),
        "lbm_last_error": (ctypes.c_char_p, []),
        "lbm_version": (ctypes.c_char_p, []),
        "lbm_debug_fail_alloc": (I, [I]),
        "lbm_debug_bounds_violations": (ctypes.c_longlong, []),
        "lbm_totals_noalloc": (I, [I, ctypes.c_longlong, P, P, P, D, D, P, P]),
        "lbm_totals_noalloc_error": (ctypes.c_char_p, []),
        "lbm_batch_create": (I, [ctypes.POINTER(P), I, I, P, P, P, ctypes.POINTER(lbm_eos), D, D, D]),
        "lbm_batch_set_boundary": (I, [P, I, I, I, dp]),
        "lbm_batch_set_stream": (I, [P, P]),
        "lbm_batch_set_shock_capturing": (I, [P, I, D, D, D]),
        "lbm_batch_init": (I, [P, I, P, P, P]),
        "lbm_batch_step": (I, [P, I]),
        "lbm_batch_step_async": (I, [P, I]),
        "lbm_batch_sync": (I, [P]),
        "lbm_batch_moments": (I, [P, I, P, P, P, P]),
        "lbm_batch_flags": (I, [P, I, ctypes.POINTER(ctypes.c_uint)]),
        "lbm_batch_autotune": (I, [P, I, ctypes.POINTER(I), ctypes.POINTER(ctypes.c_float)]),
        "lbm_batch_nodes": (ctypes.c_longlong, [P]),
        "lbm_batch_launch_count": (ctypes.c_longlong, [P]),
        "lbm_batch_destroy": (I, [P]),
        "lbm_batch_last_error": (ctypes.c_char_p, []),
        "lbm_mlp_create": (I, [ctypes.POINTER(P), D, D, D, D, ctypes.c_uint64]),
        "lbm_mlp_set_stream": (I, [P, P]),
        "lbm_mlp_collect": (I, [P, P, P, D]),
        "lbm_mlp_fit_scaling": (I, [P, P, P, ctypes.c_longlong]),
        "lbm_mlp_get_scaling": (I, [P, P]),
        "lbm_mlp_set_scaling": (I, [P, P]),
        "lbm_mlp_get_params": (I, [P, P]),
        "lbm_mlp_set_params": (I, [P, P]),
        "lbm_mlp_loss_grad": (I, [P, P, P, I, dp, P]),
        "lbm_mlp_train": (I, [P, P, P, ctypes.c_longlong, I, I, D, D, D, ctypes.c_uint64, P]),
        "lbm_mlp_predict": (I, [P, P, P, ctypes.c_longlong, P]),
        "lbm_mlp_attach": (I, [P, P]),
        "lbm_get_closure": (I, [P]),
        "lbm_mlp_destroy": (I, [P]),
        "lbm_mlp_set_mma": (I, [P, I]),
        "lbm_mlp_get_mma": (I, [P]),
        "lbm_mlp_last_error": (ctypes.c_char_p, []),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype, fn.argtypes = res, args
    _lib = lib
    return lib


def _check(rc):
    if rc != LBM_OK:
        raise LbmError(rc, load().lbm_last_error().decode())
    return rc


def _ptr(a):
    """Host pointer of a C-contiguous float64 numpy array (or None)."""
    if a is None:
        return None
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(ctypes.c_void_p)


def _dptr(t):
    """Device pointer of a torch CUDA tensor (float64, contiguous) or None."""
    if t is None:
        return None
    assert t.is_cuda and t.dtype.itemsize == 8 and t.is_contiguous()
    return ctypes.c_void_p(t.data_ptr())


# ---- entry points (same names as the C interface) ---------------------------

def lbm_create(lattice, Nx, Ny, Nz, eos, tau, Pr, cv, precision="fp64", closure=LBM_CLOSURE_EXACT):
    lib = load()
    pr = eos.get("kind", "vdw") == "pr"
    e = lbm_eos(kind=LBM_EOS_PR if pr else LBM_EOS_VDW, a=eos["a"], b=eos["b"], R=eos["R"], kappa=eos["kappa"],
                eta_over_mu=eos["eta_over_mu"], rho_ref=eos["rho_ref"], T_ref=eos["T_ref"],
                precision=PRECISIONS.get(precision, precision), closure=closure,
                Tc=eos["Tc"] if pr else 0.0, m=eos["m"] if pr else 0.0)
    h = ctypes.c_void_p()
    _check(lib.lbm_create(ctypes.byref(h), lattice, Nx, Ny, Nz, ctypes.byref(e), tau, Pr, cv))
    return h


def face_args(spec, D):
    """(LBM_BC_* type, state or None) of an x-face spec: "outflow",
    ("inflow", (rho, u, T)) or ("wall", (u, T))."""
    if spec == "outflow":
        return LBM_BC_OUTFLOW, None
    kind, state = spec
    if kind == "inflow":
        rb, ub, Tb = state
        return LBM_BC_INFLOW, [rb] + list(ub)[:D] + [Tb]
    if kind == "wall":
        uw, Tw = state
        return LBM_BC_WALL, list(uw)[:D] + [Tw]
    raise ValueError("unknown face spec %r" % (spec,))


def lbm_set_boundary(h, face, bctype, state=None):
    st = None
    if state is not None:
        arr = np.ascontiguousarray(state, dtype=np.float64)
        st = arr.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    _check(load().lbm_set_boundary(h, face, bctype, st))


def lbm_set_stream(h, stream_ptr):
    _check(load().lbm_set_stream(h, ctypes.c_void_p(stream_ptr) if stream_ptr else None))


def lbm_init(h, rho, u, T):
    rho = np.ascontiguousarray(rho, dtype=np.float64)
    u = np.ascontiguousarray(u, dtype=np.float64)
    T = np.ascontiguousarray(T, dtype=np.float64)
    _check(load().lbm_init(h, _ptr(rho), _ptr(u), _ptr(T)))


def lbm_init_device(h, rho, u, T):
    _check(load().lbm_init_device(h, _dptr(rho), _dptr(u), _dptr(T)))


def lbm_step(h, n):
    _check(load().lbm_step(h, n))


def lbm_step_async(h, n):
    _check(load().lbm_step_async(h, n))


def lbm_sync(h):
    _check(load().lbm_sync(h))


def lbm_moments(h, shape, D, want=("rho", "u", "T", "totals")):
    """Host outputs as numpy arrays of the given ([Nz,] Ny, Nx) shape."""
    out = {}
    rho = np.empty(shape) if "rho" in want else None
    u = np.empty((D,) + tuple(shape)) if "u" in want else None
    T = np.empty(shape) if "T" in want else None
    tot = np.empty(D + 2) if "totals" in want else None
    _check(load().lbm_moments(h, _ptr(rho), _ptr(u), _ptr(T), _ptr(tot)))
    for k, v in (("rho", rho), ("u", u), ("T", T), ("totals", tot)):
        if v is not None:
            out[k] = v
    return out


def lbm_moments_device(h, rho=None, u=None, T=None, totals=None):
    _check(load().lbm_moments_device(h, _dptr(rho), _dptr(u), _dptr(T), _ptr(totals)))


def lbm_get_flags(h):
    f = ctypes.c_uint()
    _check(load().lbm_get_flags(h, ctypes.byref(f)))
    return f.value


def lbm_population_bytes(h):
    return load().lbm_population_bytes(h)


def lbm_get_populations(h):
    n = lbm_population_bytes(h)
    buf = np.empty(n, dtype=np.uint8)
    _check(load().lbm_get_populations(h, buf.ctypes.data_as(ctypes.c_void_p), n))
    return buf


def lbm_set_populations(h, buf):
    buf = np.ascontiguousarray(buf, dtype=np.uint8)
    _check(load().lbm_set_populations(h, buf.ctypes.data_as(ctypes.c_void_p), buf.size))


def lbm_set_step_kernel(h, kind):
    _check(load().lbm_set_step_kernel(h, kind))


def lbm_autotune(h, reps=3):
    """Pick the fastest fused-kernel tile shape; returns (index, ms per step)."""
    c, ms = ctypes.c_int(), ctypes.c_float()
    _check(load().lbm_autotune(h, reps, ctypes.byref(c), ctypes.byref(ms)))
    return c.value, ms.value


def lbm_set_shock_capturing(h, C_mu=0.1, C_eta=0.0, C_k=0.1):
    _check(load().lbm_set_shock_capturing(h, C_mu, C_eta, C_k))


def lbm_set_graphs(h, on=True):
    _check(load().lbm_set_graphs(h, 1 if on else 0))


def lbm_set_temperature_fp64(h, on=True):
    """FP64 temperature inversion in the FP32 / FP16-deviation kernels (default off)."""
    _check(load().lbm_set_temperature_fp64(h, 1 if on else 0))


def lbm_get_temperature_fp64(h):
    return bool(load().lbm_get_temperature_fp64(h))


def lbm_debug_fail_alloc(k):
    """Test hook: the k-th device allocation of the library from now on fails (0 disarms)."""
    _check(load().lbm_debug_fail_alloc(int(k)))


def lbm_debug_bounds_violations():
    """Out-of-buffer population accesses so far (bounds-check builds; -1 otherwise)."""
    return int(load().lbm_debug_bounds_violations())


def lbm_tile_count(h):
    """Number of tile shapes of the fused step for this handle."""
    n = load().lbm_tile_count(h)
    if n < 0:
        _check(n)
    return n


def lbm_set_tile(h, index):
    """Use tile shape `index` of the fused step until the next init / autotune."""
    _check(load().lbm_set_tile(h, int(index)))


def lbm_autotune_times(h):
    """ms per step of every tile candidate at the last lbm_autotune."""
    ms = np.zeros(16, dtype=np.float32)
    n = load().lbm_autotune_times(h, ms.ctypes.data_as(ctypes.c_void_p), 16)
    if n < 0:
        _check(n)
    return ms[:min(n, 16)].tolist()


def lbm_launch_count(h):
    return load().lbm_launch_count(h)


def lbm_destroy(h):
    if h:
        load().lbm_destroy(h)


def lbm_totals_noalloc(lattice, n, rho, u, T, a, cv, totals, stream_ptr=None):
    """Totals of device fields into the device tensor ``totals`` without allocating (see include/lbm.h)."""
    rc = load().lbm_totals_noalloc(lattice, n, _dptr(rho), _dptr(u), _dptr(T), a, cv, _dptr(totals),
                                   ctypes.c_void_p(stream_ptr) if stream_ptr else None)
    if rc != LBM_OK:
        raise LbmError(rc, load().lbm_totals_noalloc_error().decode())


def lbm_version():
    return load().lbm_version().decode()


# ---- batches ----------------------------------------------------------------------

def _bcheck(rc):
    if rc != LBM_OK:
        raise LbmError(rc, load().lbm_batch_last_error().decode())
    return rc


class Batch:
    """Several ``inputs.Case`` instances (same lattice, fluid and precision) stepped together."""

    def __init__(self, cases, precision="fp32"):
        lib = load()
        c0 = cases[0]
        self.cases = list(cases)
        self.D = c0.D
        n = len(cases)
        Nx = (ctypes.c_int * n)(*[c.shape[0] for c in cases])
        Ny = (ctypes.c_int * n)(*[c.shape[1] for c in cases])
        Nz = (ctypes.c_int * n)(*[(c.shape[2] if c.D == 3 else 1) for c in cases])
        e = c0.eos
        eos = lbm_eos(kind=LBM_EOS_PR if e.get("kind", "vdw") == "pr" else LBM_EOS_VDW, a=e["a"], b=e["b"], R=e["R"],
                      kappa=e["kappa"], eta_over_mu=e["eta_over_mu"],
                      rho_ref=e["rho_ref"], T_ref=e["T_ref"], precision=PRECISIONS.get(precision, precision),
                      closure=LBM_CLOSURE_EXACT)
        self.b = ctypes.c_void_p()
        _bcheck(lib.lbm_batch_create(ctypes.byref(self.b), c0.lattice, n, Nx, Ny, Nz, ctypes.byref(eos),
                                     c0.tau, c0.Pr, c0.cv))
        for k, c in enumerate(cases):
            for face, spec in ((LBM_FACE_XLO, c.x_low), (LBM_FACE_XHI, c.x_high)):
                if spec == "periodic":
                    continue
                bctype, state = face_args(spec, self.D)
                arr = None if state is None else np.ascontiguousarray(state, dtype=np.float64)
                st = None if arr is None else arr.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
                _bcheck(lib.lbm_batch_set_boundary(self.b, k, face, bctype, st))

    def init(self):
        lib = load()
        for k, c in enumerate(self.cases):
            rho = np.ascontiguousarray(c.rho, dtype=np.float64)
            u = np.ascontiguousarray(np.stack(c.u), dtype=np.float64)
            T = np.ascontiguousarray(c.T, dtype=np.float64)
            _bcheck(lib.lbm_batch_init(self.b, k, _ptr(rho), _ptr(u), _ptr(T)))
        return self

    def step(self, n=1):
        _bcheck(load().lbm_batch_step(self.b, n))
        return self

    def set_shock_capturing(self, C_mu, C_eta, C_k, k=-1):
        """Shock capturing for instance k (every instance with k = -1)."""
        _bcheck(load().lbm_batch_set_shock_capturing(self.b, k, C_mu, C_eta, C_k))
        return self

    def step_async(self, n=1):
        _bcheck(load().lbm_batch_step_async(self.b, n))

    def sync(self):
        _bcheck(load().lbm_batch_sync(self.b))

    def autotune(self, reps=3):
        c, ms = ctypes.c_int(), ctypes.c_float()
        _bcheck(load().lbm_batch_autotune(self.b, reps, ctypes.byref(c), ctypes.byref(ms)))
        return c.value, ms.value

    def fields(self, k):
        c = self.cases[k]
        shape = tuple(reversed(c.shape))
        rho, u, T, tot = np.empty(shape), np.empty((c.D,) + shape), np.empty(shape), np.empty(c.D + 2)
        _bcheck(load().lbm_batch_moments(self.b, k, _ptr(rho), _ptr(u), _ptr(T), _ptr(tot)))
        return dict(rho=rho, u=u, T=T, totals=tot)

    def flags(self, k):
        f = ctypes.c_uint()
        _bcheck(load().lbm_batch_flags(self.b, k, ctypes.byref(f)))
        return f.value

    def nodes(self):
        return load().lbm_batch_nodes(self.b)

    def launches(self):
        return load().lbm_batch_launch_count(self.b)

    def close(self):
        if self.b:
            load().lbm_batch_destroy(self.b)
            self.b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ---- learned closure (include/lbm_mlp.h) ----------------------------------------

def _mcheck(rc):
    if rc != LBM_OK:
        raise LbmError(rc, load().lbm_mlp_last_error().decode())
    return rc


def _f32(a, n):
    a = np.ascontiguousarray(a, dtype=np.float32)
    assert a.size == n
    return a


def lbm_mlp_create(a, b, R, cv, seed):
    h = ctypes.c_void_p()
    _mcheck(load().lbm_mlp_create(ctypes.byref(h), a, b, R, cv, ctypes.c_uint64(seed)))
    return h


def lbm_mlp_set_stream(net, stream_ptr):
    _mcheck(load().lbm_mlp_set_stream(net, ctypes.c_void_p(stream_ptr)))


def lbm_mlp_collect(h, rho, e, e_scale=1.0):
    """Solver state -> (rho, e) samples in the device tensors rho, e (float64, Nx Ny Nz each)."""
    _mcheck(load().lbm_mlp_collect(h, _dptr(rho), _dptr(e), e_scale))


def lbm_mlp_fit_scaling(net, rho, e):
    _mcheck(load().lbm_mlp_fit_scaling(net, _dptr(rho), _dptr(e), rho.numel()))


def lbm_mlp_get_scaling(net):
    s = np.zeros(LBM_MLP_NSCALE)
    _mcheck(load().lbm_mlp_get_scaling(net, _ptr(s)))
    return s


def lbm_mlp_set_scaling(net, scale):
    s = np.ascontiguousarray(scale, dtype=np.float64)
    assert s.size == LBM_MLP_NSCALE
    _mcheck(load().lbm_mlp_set_scaling(net, _ptr(s)))


def lbm_mlp_get_params(net):
    th = np.zeros(LBM_MLP_NPARAM, dtype=np.float32)
    _mcheck(load().lbm_mlp_get_params(net, th.ctypes.data_as(ctypes.c_void_p)))
    return th


def lbm_mlp_set_params(net, theta):
    th = _f32(theta, LBM_MLP_NPARAM)
    _mcheck(load().lbm_mlp_set_params(net, th.ctypes.data_as(ctypes.c_void_p)))


def lbm_mlp_loss_grad(net, x, y):
    """(loss, gradient) of the network on host samples x (n, 2), y (n, 3)."""
    n = int(np.asarray(x).shape[0])
    xs, ys = _f32(x, 2 * n), _f32(y, 3 * n)
    g = np.zeros(LBM_MLP_NPARAM, dtype=np.float32)
    loss = ctypes.c_double()
    _mcheck(load().lbm_mlp_loss_grad(net, xs.ctypes.data_as(ctypes.c_void_p), ys.ctypes.data_as(ctypes.c_void_p),
                                     n, ctypes.byref(loss), g.ctypes.data_as(ctypes.c_void_p)))
    return loss.value, g


def lbm_mlp_train(net, rho, e, batch, steps, lr0, lr1, wd=0.0, seed=0):
    """AdamW steps on the device samples (rho, e); returns the per-step minibatch losses."""
    losses = np.zeros(max(steps, 1), dtype=np.float32)
    _mcheck(load().lbm_mlp_train(net, _dptr(rho), _dptr(e), rho.numel(), batch, steps, lr0, lr1, wd,
                                 ctypes.c_uint64(seed), losses.ctypes.data_as(ctypes.c_void_p)))
    return losses[:steps]


def lbm_mlp_predict(net, rho, e, out):
    """out (device float64, n x 4): T, P, c_s^2, network used (1) or exact (0)."""
    _mcheck(load().lbm_mlp_predict(net, _dptr(rho), _dptr(e), rho.numel(), _dptr(out)))


def lbm_mlp_attach(h, net):
    _mcheck(load().lbm_mlp_attach(h, net))


def lbm_get_closure(h):
    return load().lbm_get_closure(h)


LBM_MLP_MMA_WARP, LBM_MLP_MMA_TCGEN05 = 0, 1


def lbm_mlp_set_mma(net, kind):
    """Contraction path of the training kernels (LBM_MLP_MMA_TCGEN05 default, or LBM_MLP_MMA_WARP)."""
    _mcheck(load().lbm_mlp_set_mma(net, int(kind)))


def lbm_mlp_get_mma(net):
    return int(load().lbm_mlp_get_mma(net))


def lbm_mlp_destroy(net):
    return load().lbm_mlp_destroy(net)


# ---- convenience wrapper -------------------------------------------------------

class Solver:
    """One handle set up from an ``inputs.Case``-like description."""

    def __init__(self, case, precision="fp64", stream=None, step_kernel=LBM_STEP_FUSED, t_fp64=None):
        """t_fp64: FP64 temperature inversion of the FP32 / FP16-deviation kernels
        (None keeps the library default, off)."""
        self.case = case
        self.D = case.D
        Nx, Ny = case.shape[0], case.shape[1]
        Nz = case.shape[2] if case.D == 3 else 1
        self.arr_shape = tuple(reversed(case.shape))
        self.h = lbm_create(case.lattice, Nx, Ny, Nz, case.eos, case.tau, case.Pr, case.cv, precision)
        if stream:
            lbm_set_stream(self.h, stream)
        lbm_set_step_kernel(self.h, step_kernel)
        if t_fp64 is not None:
            lbm_set_temperature_fp64(self.h, t_fp64)
        for face, spec in ((LBM_FACE_XLO, case.x_low), (LBM_FACE_XHI, case.x_high)):
            if spec == "periodic":
                continue
            lbm_set_boundary(self.h, face, *face_args(spec, self.D))

    def init(self, rho=None, u=None, T=None):
        c = self.case
        rho = c.rho if rho is None else rho
        u = c.u if u is None else u
        T = c.T if T is None else T
        lbm_init(self.h, np.asarray(rho, dtype=np.float64), np.stack([np.asarray(x, dtype=np.float64) for x in u]),
                 np.asarray(T, dtype=np.float64))
        return self

    def step(self, n=1):
        lbm_step(self.h, n)
        return self

    def fields(self):
        return lbm_moments(self.h, self.arr_shape, self.D)

    def close(self):
        lbm_destroy(self.h)
        self.h = None

    def __del__(self):
        try:
            if self.h:
                self.close()
        except Exception:
            pass


# ---- learned closure wrapper ---------------------------------------------------

class Closure:
    """One learned-closure network (an lbm_mlp handle); device data are torch tensors."""

    def __init__(self, a, b, R, cv, seed=1, stream=None):
        self.eos = (a, b, R, cv)
        self.net = lbm_mlp_create(a, b, R, cv, seed)
        if stream:
            lbm_mlp_set_stream(self.net, stream)

    def collect(self, solver, e_scale=1.0):
        """(rho, e) of the solver's current interior state as two device tensors."""
        import torch
        n = int(np.prod(solver.arr_shape))
        rho = torch.empty(n, dtype=torch.float64, device="cuda")
        e = torch.empty(n, dtype=torch.float64, device="cuda")
        lbm_mlp_collect(solver.h, rho, e, e_scale)
        return rho, e

    def collect_runs(self, runs, snapshots, every, precision="fp64", shock_capturing=None):
        """Run each (case, e_scale) for snapshots * every steps and collect every `every` steps
        (optionally with shock capturing (C_mu, C_eta, C_k))."""
        import torch
        rs, es = [], []
        for case, e_scale in runs:
            s = Solver(case, precision)
            if shock_capturing:
                lbm_set_shock_capturing(s.h, *shock_capturing)
            s.init()
            for _ in range(snapshots):
                s.step(every)
                r, e = self.collect(s, e_scale)
                rs.append(r)
                es.append(e)
            s.close()
        return torch.cat(rs), torch.cat(es)

    def fit_scaling(self, rho, e):
        lbm_mlp_fit_scaling(self.net, rho, e)

    @property
    def scaling(self):
        return lbm_mlp_get_scaling(self.net)

    @scaling.setter
    def scaling(self, s):
        lbm_mlp_set_scaling(self.net, s)

    @property
    def params(self):
        return lbm_mlp_get_params(self.net)

    @params.setter
    def params(self, theta):
        lbm_mlp_set_params(self.net, theta)

    @property
    def mma(self):
        """Contraction path of training: LBM_MLP_MMA_TCGEN05 or LBM_MLP_MMA_WARP."""
        return lbm_mlp_get_mma(self.net)

    @mma.setter
    def mma(self, kind):
        lbm_mlp_set_mma(self.net, kind)

    def loss_grad(self, x, y):
        return lbm_mlp_loss_grad(self.net, x, y)

    def train(self, rho, e, batch=8192, steps=1000, lr0=3e-3, lr1=3e-5, wd=0.0, seed=0):
        return lbm_mlp_train(self.net, rho, e, batch, steps, lr0, lr1, wd, seed)

    def predict(self, rho, e):
        """(n, 4) device tensor: T, P, c_s^2, 1 where the network was used."""
        import torch
        out = torch.empty((rho.numel(), 4), dtype=torch.float64, device="cuda")
        lbm_mlp_predict(self.net, rho, e, out)
        return out

    def attach(self, solver):
        lbm_mlp_attach(solver.h, self.net)

    @staticmethod
    def detach(solver):
        lbm_mlp_attach(solver.h, None)

    def close(self):
        if self.net:
            lbm_mlp_destroy(self.net)
        self.net = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
