"""Python binding of libhdgdg (ctypes): argument marshalling only, same names as the C ABI.

Every step of the hot path runs in the CUDA library; there is no Python or CPU fallback.
If the shared library is missing this module raises at first use.
"""
import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libhdgdg.so")

OK, EINVAL, ENOMEM, ECUDA, ENOTCONVERGED, ENONFINITE, ESTATE = range(7)
STATUS_NAMES = ["OK", "EINVAL", "ENOMEM", "ECUDA", "ENOTCONVERGED", "ENONFINITE", "ESTATE"]
SCHEMES = {"ars2": 0, "ars3": 1, "rk2": 2, "rk3": 3}
PRECISIONS = {"fp64": 0, "mixed": 1}
LOCAL_PRECISIONS = {"fp64": 0, "fp32": 1, "bf16": 2, "f32x2": 3, "bf16split": 4}
BOUNDARIES = {"periodic": 0, "wall": 1, "vortex": 2}
DG_PRECISIONS = {"default": 0, "bf16": 1}

EXPORTS = ["hdgdg_bytes_required", "hdgdg_node_coords", "hdgdg_create", "hdgdg_set_state",
           "hdgdg_step", "hdgdg_get_state", "hdgdg_get_stats", "hdgdg_last_error", "hdgdg_destroy",
           "hdgdg_update_state", "hdgdg_eval_nl", "hdgdg_condense_rhs", "hdgdg_trace_apply", "hdgdg_set_trace_tile", "hdgdg_set_local_tiles",
           "hdgdg_stage_solve",
           "hdgdg_measure_fp64_tflops", "hdgdg_measure_conversion_rates", "hdgdg_set_kernel_timing", "hdgdg_kernel_time",
           "hdgdg_mass_noalloc", "hdgdg_gll", "hdgdg_checkpoint_bytes", "hdgdg_save_checkpoint",
           "hdgdg_load_checkpoint", "hdgdg_ensemble_create", "hdgdg_ensemble_set_state", "hdgdg_ensemble_step",
           "hdgdg_ensemble_get_state", "hdgdg_ensemble_get_stats", "hdgdg_ensemble_last_error",
           "hdgdg_ensemble_destroy"]
KERNEL_CLASSES = ["spmv", "ortho", "condense", "recover", "dg", "combine", "residual", "guess", "precond"]


class HdgdgError(RuntimeError):
    def __init__(self, status, message):
        self.status = status
        name = STATUS_NAMES[status] if 0 <= status < len(STATUS_NAMES) else str(status)
        super().__init__(f"hdgdg {name}: {message}")


class Config(ctypes.Structure):
    _fields_ = [("n_side", ctypes.c_int), ("degree_k", ctypes.c_int), ("g", ctypes.c_double),
                ("H0", ctypes.c_double), ("scheme", ctypes.c_int), ("dt", ctypes.c_double),
                ("precision", ctypes.c_int), ("krylov_rtol", ctypes.c_double),
                ("krylov_restart", ctypes.c_int), ("krylov_maxit", ctypes.c_int),
                ("linear_only", ctypes.c_int), ("boundary", ctypes.c_int), ("x0", ctypes.c_double),
                ("length", ctypes.c_double), ("bc_params", ctypes.c_double * 5),
                ("batch", ctypes.c_int), ("dt_per_instance", ctypes.POINTER(ctypes.c_double)),
                ("local_precision", ctypes.c_int), ("krylov_guess", ctypes.c_int), ("spmv_kernel", ctypes.c_int),
                ("krylov_ortho", ctypes.c_int), ("residual_f32x2", ctypes.c_int),
                ("local_dense", ctypes.c_int), ("trace_operator", ctypes.c_int),
                ("host_steps", ctypes.c_int), ("dg_precision", ctypes.c_int), ("krylov_guess_ls", ctypes.c_int)]


class Stats(ctypes.Structure):
    _fields_ = [("steps", ctypes.c_longlong), ("krylov_iterations", ctypes.c_longlong),
                ("last_krylov_iterations", ctypes.c_int), ("last_rel_residual", ctypes.c_double),
                ("mass", ctypes.c_double), ("kernel_launches", ctypes.c_longlong), ("time", ctypes.c_double),
                ("last_guess_order", ctypes.c_int), ("local_tile_condense", ctypes.c_int),
                ("local_tile_recover", ctypes.c_int), ("trace_tile", ctypes.c_int),
                ("trace_tile_prefetch", ctypes.c_int)]


_lib = None
_P = ctypes.POINTER(ctypes.c_double)


def lib():
    """Load libhdgdg.so (built in-tree by ``paper_1711_02751_gb300.build``); raise if absent."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with `python -m paper_1711_02751_gb300.build`")
        L = ctypes.CDLL(LIB_PATH)
        L.hdgdg_bytes_required.restype = ctypes.c_size_t
        L.hdgdg_bytes_required.argtypes = [ctypes.POINTER(Config)]
        L.hdgdg_node_coords.argtypes = [ctypes.POINTER(Config), _P, _P]
        L.hdgdg_gll.argtypes = [ctypes.c_int, _P, _P]
        L.hdgdg_create.argtypes = [ctypes.POINTER(Config), _P, ctypes.c_void_p, ctypes.POINTER(ctypes.c_void_p)]
        L.hdgdg_set_state.argtypes = [ctypes.c_void_p, _P, _P, _P]
        L.hdgdg_update_state.argtypes = [ctypes.c_void_p, _P, _P, _P]
        L.hdgdg_checkpoint_bytes.restype = ctypes.c_size_t
        L.hdgdg_checkpoint_bytes.argtypes = [ctypes.c_void_p]
        L.hdgdg_save_checkpoint.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t]
        L.hdgdg_load_checkpoint.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t]
        L.hdgdg_step.argtypes = [ctypes.c_void_p, ctypes.c_int]
        L.hdgdg_get_state.argtypes = [ctypes.c_void_p, _P, _P, _P]
        L.hdgdg_get_stats.argtypes = [ctypes.c_void_p, ctypes.POINTER(Stats)]
        L.hdgdg_last_error.restype = ctypes.c_char_p
        L.hdgdg_last_error.argtypes = [ctypes.c_void_p]
        L.hdgdg_destroy.restype = None
        L.hdgdg_destroy.argtypes = [ctypes.c_void_p]
        L.hdgdg_eval_nl.argtypes = [ctypes.c_void_p, _P, _P]
        L.hdgdg_condense_rhs.argtypes = [ctypes.c_void_p, _P, _P]
        L.hdgdg_trace_apply.argtypes = [ctypes.c_void_p, _P, _P]
        L.hdgdg_set_trace_tile.argtypes = [ctypes.c_void_p, ctypes.c_int]
        L.hdgdg_set_local_tiles.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int]
        L.hdgdg_stage_solve.argtypes = [ctypes.c_void_p, _P, _P, _P, ctypes.POINTER(ctypes.c_int)]
        L.hdgdg_measure_fp64_tflops.argtypes = [_P]
        L.hdgdg_measure_conversion_rates.argtypes = [_P, _P]
        L.hdgdg_set_kernel_timing.argtypes = [ctypes.c_void_p, ctypes.c_int]
        L.hdgdg_kernel_time.argtypes = [ctypes.c_void_p, ctypes.c_int, _P, ctypes.POINTER(ctypes.c_longlong)]
        L.hdgdg_mass_noalloc.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_void_p,
                                         ctypes.c_void_p, ctypes.c_void_p]
        L.hdgdg_ensemble_create.argtypes = [ctypes.POINTER(Config), ctypes.c_int, ctypes.POINTER(ctypes.c_int),
                                            ctypes.POINTER(ctypes.c_int), _P, ctypes.POINTER(_P), ctypes.c_void_p,
                                            ctypes.POINTER(ctypes.c_void_p)]
        L.hdgdg_ensemble_set_state.argtypes = [ctypes.c_void_p, ctypes.c_int, _P, _P, _P]
        L.hdgdg_ensemble_get_state.argtypes = [ctypes.c_void_p, ctypes.c_int, _P, _P, _P]
        L.hdgdg_ensemble_step.argtypes = [ctypes.c_void_p, ctypes.c_int]
        L.hdgdg_ensemble_get_stats.argtypes = [ctypes.c_void_p, ctypes.POINTER(Stats)]
        L.hdgdg_ensemble_last_error.restype = ctypes.c_char_p
        L.hdgdg_ensemble_last_error.argtypes = [ctypes.c_void_p]
        L.hdgdg_ensemble_destroy.restype = None
        L.hdgdg_ensemble_destroy.argtypes = [ctypes.c_void_p]
        for name in EXPORTS:
            getattr(L, name).restype = getattr(L, name).restype or ctypes.c_int
        _lib = L
    return _lib


def _ptr(a):
    return a.ctypes.data_as(_P)


def _f64(a, shape=None):
    a = np.ascontiguousarray(a, dtype=np.float64)
    if shape is not None and a.size != int(np.prod(shape)):
        raise ValueError(f"expected {int(np.prod(shape))} values, got {a.size}")
    return a


def make_config(N, k, dt, g=1.0, H0=1.0, scheme="ars2", krylov_rtol=0.0, krylov_restart=0,
                krylov_maxit=0, linear_only=False, precision="fp64", boundary="periodic", x0=0.0,
                length=1.0, bc_params=(0.0, 0.0, 0.0, 0.0, 0.0), batch=1, dt_per_instance=None,
                local_precision="fp64", krylov_guess=0, spmv_kernel=0, krylov_ortho=0, residual_f32x2=False,
                local_dense=False, trace_operator=0, host_steps=False, dg_precision="default", krylov_guess_ls=False):
    """bc_params (boundary='vortex'): beta, u_inf, v_inf, x_c, y_c of the moving vortex.
    batch > 1: that many instances in one handle; dt_per_instance (length batch) overrides dt
    instance by instance (dt then only sets the scale the factors are taken against)."""
    dts = None
    if dt_per_instance is not None:
        dts = np.ascontiguousarray(dt_per_instance, dtype=np.float64).reshape(-1)
        if dts.size != int(batch):
            raise ValueError("dt_per_instance needs one time step per instance")
    cfg = Config(int(N), int(k), float(g), float(H0), SCHEMES[scheme], float(dt), PRECISIONS[precision],
                 float(krylov_rtol), int(krylov_restart), int(krylov_maxit), int(bool(linear_only)),
                 BOUNDARIES[boundary], float(x0), float(length), (ctypes.c_double * 5)(*bc_params),
                 int(batch), _ptr(dts) if dts is not None else None, LOCAL_PRECISIONS[local_precision],
                 int(krylov_guess), int(spmv_kernel), int(krylov_ortho), int(bool(residual_f32x2)),
                 int(bool(local_dense)), int(trace_operator), int(bool(host_steps)),
                 DG_PRECISIONS[dg_precision], int(bool(krylov_guess_ls)))
    cfg._dts = dts                     # keeps the array alive as long as the config
    return cfg


def bytes_required(cfg):
    return int(lib().hdgdg_bytes_required(ctypes.byref(cfg)))


def node_coords(N, k, boundary="periodic", x0=0.0, length=1.0):
    """GLL node coordinates (x, y), each [N*N, (k+1)^2], from the library's own tables."""
    cfg = make_config(N, k, 1.0, boundary=boundary, x0=x0, length=length)
    x = np.empty((N * N, (k + 1) ** 2))
    y = np.empty_like(x)
    st = lib().hdgdg_node_coords(ctypes.byref(cfg), _ptr(x), _ptr(y))
    if st != OK:
        raise HdgdgError(st, "node_coords")
    return x, y


def mass_noalloc(n_side, degree_k, phi_eta_dev_ptr, mass_dev_ptr, stream=None, length=1.0):
    """hdgdg_mass_noalloc on caller-owned device buffers (raw addresses); returns the status."""
    return lib().hdgdg_mass_noalloc(int(n_side), int(degree_k), float(length), ctypes.c_void_p(phi_eta_dev_ptr),
                                    ctypes.c_void_p(mass_dev_ptr), ctypes.c_void_p(stream) if stream else None)


def gll(k):
    """The library's GLL nodes and weights of degree k."""
    x = np.empty(k + 1)
    w = np.empty(k + 1)
    st = lib().hdgdg_gll(int(k), _ptr(x), _ptr(w))
    if st != OK:
        raise HdgdgError(st, "gll")
    return x, w


def measure_conversion_rates():
    """(hardware, integer-pipe) FP64<->FP32 conversions per second on the current device."""
    hw, it = ctypes.c_double(0.0), ctypes.c_double(0.0)
    st = lib().hdgdg_measure_conversion_rates(ctypes.byref(hw), ctypes.byref(it))
    if st != OK:
        raise HdgdgError(st, "measure_conversion_rates")
    return hw.value, it.value


def measure_fp64_tflops():
    out = ctypes.c_double(0.0)
    st = lib().hdgdg_measure_fp64_tflops(ctypes.byref(out))
    if st != OK:
        raise HdgdgError(st, "measure_fp64_tflops")
    return out.value


class Sim:
    """One simulation handle (hdgdg_create ... hdgdg_destroy)."""

    def __init__(self, N, k, dt, bottom=None, g=1.0, H0=1.0, scheme="ars2", stream=None,
                 krylov_rtol=0.0, krylov_restart=0, krylov_maxit=0, linear_only=False, precision="fp64",
                 boundary="periodic", x0=0.0, length=1.0, bc_params=(0.0, 0.0, 0.0, 0.0, 0.0),
                 batch=1, dt_per_instance=None, local_precision="fp64", krylov_guess=0, spmv_kernel=0,
                 krylov_ortho=0, residual_f32x2=False, local_dense=False, trace_operator=0, host_steps=False,
                 dg_precision="default", krylov_guess_ls=False):
        """batch > 1 holds that many independent instances of the mesh (one launch per kernel
        per stage covers all of them); arrays are then [batch * N * N, (k+1)^2], instance-major,
        and the bottom and the time step (dt_per_instance) may differ from instance to instance."""
        self.N, self.k, self.P = int(N), int(k), int(k) + 1
        self.batch = int(batch)
        self.n_el, self.Np = self.batch * self.N * self.N, self.P * self.P
        self.n_edges = self.batch * (2 * self.N * (self.N + 1) if boundary != "periodic" else 2 * self.N * self.N)
        self.cfg = make_config(N, k, dt, g, H0, scheme, krylov_rtol, krylov_restart, krylov_maxit,
                               linear_only, precision, boundary, x0, length, bc_params, batch,
                               dt_per_instance, local_precision, krylov_guess, spmv_kernel, krylov_ortho,
                               residual_f32x2, local_dense, trace_operator, host_steps, dg_precision,
                               krylov_guess_ls)
        self._h = ctypes.c_void_p(None)
        b = None if bottom is None else _f64(bottom, (self.n_el, self.Np))
        st = lib().hdgdg_create(ctypes.byref(self.cfg), None if b is None else _ptr(b),
                                ctypes.c_void_p(stream) if stream else None, ctypes.byref(self._h))
        if st != OK:
            msg = self.last_error() if self._h else "create"
            self.close()
            raise HdgdgError(st, msg)

    # -- lifecycle --------------------------------------------------------------------
    def close(self):
        if self._h:
            lib().hdgdg_destroy(self._h)
            self._h = ctypes.c_void_p(None)

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def last_error(self):
        return lib().hdgdg_last_error(self._h).decode()

    def _check(self, st):
        if st != OK:
            raise HdgdgError(st, self.last_error())

    # -- state ------------------------------------------------------------------------
    def set_state(self, h, hu, hv):
        sh = (self.n_el, self.Np)
        h, hu, hv = _f64(h, sh), _f64(hu, sh), _f64(hv, sh)
        self._check(lib().hdgdg_set_state(self._h, _ptr(h), _ptr(hu), _ptr(hv)))

    def set_state_ptrs(self, h_ptr, hu_ptr, hv_ptr):
        """set_state from raw host addresses (e.g. pinned buffers); sizes as in set_state."""
        self._check(lib().hdgdg_set_state(self._h, ctypes.cast(h_ptr, _P), ctypes.cast(hu_ptr, _P),
                                          ctypes.cast(hv_ptr, _P)))

    def update_state(self, h, hu, hv):
        """Replace the state of the running trajectory (time, counters and solver history kept)."""
        sh = (self.n_el, self.Np)
        h, hu, hv = _f64(h, sh), _f64(hu, sh), _f64(hv, sh)
        self._check(lib().hdgdg_update_state(self._h, _ptr(h), _ptr(hu), _ptr(hv)))

    def update_state_ptrs(self, h_ptr, hu_ptr, hv_ptr):
        """update_state from raw host addresses (e.g. pinned buffers)."""
        self._check(lib().hdgdg_update_state(self._h, ctypes.cast(h_ptr, _P), ctypes.cast(hu_ptr, _P),
                                             ctypes.cast(hv_ptr, _P)))

    def save_checkpoint(self):
        """The state, time, counters and solver history as bytes (see hdgdg_save_checkpoint)."""
        n = int(lib().hdgdg_checkpoint_bytes(self._h))
        if n == 0:
            raise HdgdgError(ESTATE, "save_checkpoint before set_state")
        buf = ctypes.create_string_buffer(n)
        self._check(lib().hdgdg_save_checkpoint(self._h, buf, n))
        return buf.raw

    def load_checkpoint(self, data):
        """Continue from bytes written by save_checkpoint (same configuration and bottom)."""
        buf = ctypes.create_string_buffer(bytes(data), len(data))
        self._check(lib().hdgdg_load_checkpoint(self._h, buf, len(data)))

    def step(self, n_steps=1):
        self._check(lib().hdgdg_step(self._h, int(n_steps)))

    def get_state(self):
        out = [np.empty((self.n_el, self.Np)) for _ in range(3)]
        self._check(lib().hdgdg_get_state(self._h, *[_ptr(a) for a in out]))
        return tuple(out)

    def get_state_ptrs(self, h_ptr, hu_ptr, hv_ptr):
        self._check(lib().hdgdg_get_state(self._h, ctypes.cast(h_ptr, _P), ctypes.cast(hu_ptr, _P),
                                          ctypes.cast(hv_ptr, _P)))

    def stats(self):
        s = Stats()
        self._check(lib().hdgdg_get_stats(self._h, ctypes.byref(s)))
        return {f: getattr(s, f) for f, _ in Stats._fields_}

    def set_kernel_timing(self, on=True):
        self._check(lib().hdgdg_set_kernel_timing(self._h, int(bool(on))))

    def kernel_times(self):
        """{class: (total_ms, launch groups)} of the per-kernel-class timers."""
        out = {}
        for c, name in enumerate(KERNEL_CLASSES):
            ms, n = ctypes.c_double(0.0), ctypes.c_longlong(0)
            self._check(lib().hdgdg_kernel_time(self._h, c, ctypes.byref(ms), ctypes.byref(n)))
            out[name] = (ms.value, n.value)
        return out

    # -- row-level entry points --------------------------------------------------------
    def eval_nl(self, q):
        q = _f64(q, (3, self.n_el, self.Np))
        out = np.empty((3, self.n_el, self.Np))
        self._check(lib().hdgdg_eval_nl(self._h, _ptr(q), _ptr(out)))
        return out

    def condense_rhs(self, R1):
        R1 = _f64(R1, (3, self.n_el, self.Np))
        out = np.empty((self.n_edges, 3, self.P))
        self._check(lib().hdgdg_condense_rhs(self._h, _ptr(R1), _ptr(out)))
        return out

    def trace_apply(self, x):
        x = _f64(x, (self.n_edges, 3, self.P))
        out = np.empty((self.n_edges, 3, self.P))
        self._check(lib().hdgdg_trace_apply(self._h, _ptr(x), _ptr(out)))
        return out

    def set_trace_tile(self, tile):
        """Select the inner cycles' element-pass tile (0 the default, 1..8 at degrees 2..4)."""
        self._check(lib().hdgdg_set_trace_tile(self._h, int(tile)))

    def set_local_tiles(self, condense, recover):
        """Select the Schur condensation and recovery tiles (0 the default, 1..2, 3 staged at k = 3)."""
        self._check(lib().hdgdg_set_local_tiles(self._h, int(condense), int(recover)))

    def stage_solve(self, R1):
        R1 = _f64(R1, (3, self.n_el, self.Np))
        Q = np.empty((3, self.n_el, self.Np))
        lam = np.empty((self.n_edges, 3, self.P))
        its = ctypes.c_int(0)
        self._check(lib().hdgdg_stage_solve(self._h, _ptr(R1), _ptr(Q), _ptr(lam), ctypes.byref(its)))
        return Q, lam, its.value


class Ensemble:
    """Uneven ensemble (hdgdg_ensemble_create ... hdgdg_ensemble_destroy): members of different
    mesh sizes and degrees advanced together, one persistent launch per kernel class per stage."""

    def __init__(self, sides, degrees, dts, bottoms=None, g=1.0, H0=1.0, scheme="ars2", stream=None,
                 krylov_rtol=0.0, krylov_restart=0, krylov_maxit=0, krylov_guess=0):
        self.sides = [int(v) for v in sides]
        self.degrees = [int(v) for v in degrees]
        n = len(self.sides)
        base = make_config(2, 2, 1.0, g, H0, scheme, krylov_rtol, krylov_restart, krylov_maxit,
                           precision="mixed", local_precision="f32x2", krylov_guess=krylov_guess,
                           trace_operator=1)
        ns = (ctypes.c_int * n)(*self.sides)
        ks = (ctypes.c_int * n)(*self.degrees)
        d = _f64(dts, (n,))
        self._bots = [None if bottoms is None or bottoms[i] is None else
                      _f64(bottoms[i], (self.sides[i] ** 2, (self.degrees[i] + 1) ** 2)) for i in range(n)]
        barr = (_P * n)(*[(_ptr(b) if b is not None else _P()) for b in self._bots])
        self._h = ctypes.c_void_p(None)
        st = lib().hdgdg_ensemble_create(ctypes.byref(base), n, ns, ks, _ptr(d), barr,
                                         ctypes.c_void_p(stream) if stream else None, ctypes.byref(self._h))
        if st != OK:
            msg = self.last_error() if self._h else "ensemble_create"
            self.close()
            raise HdgdgError(st, msg)

    def close(self):
        if self._h:
            lib().hdgdg_ensemble_destroy(self._h)
            self._h = ctypes.c_void_p(None)

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def last_error(self):
        return lib().hdgdg_ensemble_last_error(self._h).decode()

    def _check(self, st):
        if st != OK:
            raise HdgdgError(st, self.last_error())

    def _shape(self, m):
        return (self.sides[m] ** 2, (self.degrees[m] + 1) ** 2)

    def set_state(self, m, h, hu, hv):
        sh = self._shape(m)
        h, hu, hv = _f64(h, sh), _f64(hu, sh), _f64(hv, sh)
        self._check(lib().hdgdg_ensemble_set_state(self._h, int(m), _ptr(h), _ptr(hu), _ptr(hv)))

    def step(self, n_steps=1):
        self._check(lib().hdgdg_ensemble_step(self._h, int(n_steps)))

    def get_state(self, m):
        out = [np.empty(self._shape(m)) for _ in range(3)]
        self._check(lib().hdgdg_ensemble_get_state(self._h, int(m), *[_ptr(a) for a in out]))
        return tuple(out)

    def stats(self):
        s = Stats()
        self._check(lib().hdgdg_ensemble_get_stats(self._h, ctypes.byref(s)))
        return {f: getattr(s, f) for f, _ in Stats._fields_}
