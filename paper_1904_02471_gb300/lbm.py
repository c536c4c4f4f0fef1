"""ctypes binding of liblbm.so (the C ABI of include/lbm.h).

Argument marshalling only: every step of the CS and FD updates runs in the
library's CUDA kernels. Loading fails loudly when the library has not been
built; there is no CPU fallback.

Low-level functions keep the C names (``lbm_create``, ``lbm_step``, ...);
``Lattice`` and ``Batch`` wrap them for numpy arrays.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
# LBM_LIBRARY selects another build of the same library (e.g. the
# bounds-checked one in _build_bounds/)
LIB_PATH = os.environ.get("LBM_LIBRARY") or os.path.join(HERE, "_build", "liblbm.so")

LBM_OK, LBM_EINVAL, LBM_ECFL, LBM_ESTIFF, LBM_ENOMEM, LBM_ECUDA = 0, 1, 2, 3, 4, 5
LBM_ENOTREADY, LBM_ETIMEOUT, LBM_EBUSY, LBM_ENONFINITE, LBM_ECANCELLED, LBM_ENOTFOUND = 6, 7, 8, 9, 10, 11
LBM_CS, LBM_FD = 0, 1
LBM_FP64, LBM_FP32_DEV = 0, 1


class lbm_obs(ctypes.Structure):
    _fields_ = [("step", ctypes.c_int64), ("time", ctypes.c_double), ("mass", ctypes.c_double),
                ("mom_x", ctypes.c_double), ("mom_y", ctypes.c_double), ("amp", ctypes.c_double),
                ("nonfinite", ctypes.c_int32), ("reserved", ctypes.c_int32)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_ if f != "reserved"}


class lbm_spec(ctypes.Structure):
    _fields_ = [("model", ctypes.c_int), ("q_per_axis", ctypes.c_int), ("nx", ctypes.c_int), ("ny", ctypes.c_int),
                ("precision", ctypes.c_int), ("storage", ctypes.c_int), ("tau", ctypes.c_double),
                ("dt", ctypes.c_double), ("dx", ctypes.c_double), ("rho0", ctypes.c_double),
                ("scheme", ctypes.c_int), ("reserved", ctypes.c_int)]


class lbm_view(ctypes.Structure):
    _fields_ = [("base", ctypes.c_void_p), ("plane", ctypes.c_int64), ("pitch", ctypes.c_int32),
                ("elem_bytes", ctypes.c_int32), ("cs_pull_phase", ctypes.c_int32), ("reserved", ctypes.c_int32)]


class lbm_request(ctypes.Structure):
    _fields_ = [("spec", lbm_spec), ("steps", ctypes.c_int64), ("init", ctypes.c_int), ("obs_every", ctypes.c_int),
                ("keep_moments", ctypes.c_int), ("reserved", ctypes.c_int),
                ("U", ctypes.c_double), ("rho_l", ctypes.c_double), ("rho_r", ctypes.c_double),
                ("user_tag", ctypes.c_uint64)]


class lbm_result(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int), ("reserved", ctypes.c_int), ("user_tag", ctypes.c_uint64),
                ("steps", ctypes.c_int64), ("first", lbm_obs), ("last", lbm_obs), ("nu_fit", ctypes.c_double),
                ("t_submit", ctypes.c_double), ("t_admit", ctypes.c_double), ("t_done", ctypes.c_double),
                ("n_series", ctypes.c_int64)]

    def as_dict(self):
        d = {f: getattr(self, f) for f, _ in self._fields_ if f not in ("reserved", "first", "last")}
        d["first"] = self.first.as_dict()
        d["last"] = self.last.as_dict()
        return d


class LbmError(RuntimeError):
    def __init__(self, code: int, what: str):
        self.code = code
        super().__init__(f"{what}: {strerror(code)} ({code}): {last_error()}")


_lib: Optional[ctypes.CDLL] = None

_P = ctypes.c_void_p
_D = ctypes.POINTER(ctypes.c_double)
_i, _d, _i64, _sz = ctypes.c_int, ctypes.c_double, ctypes.c_int64, ctypes.c_size_t

# (name, restype, argtypes)
_SIGS = [
    ("lbm_version", ctypes.c_char_p, []),
    ("lbm_strerror", ctypes.c_char_p, [_i]),
    ("lbm_last_error", ctypes.c_char_p, []),
    ("lbm_nu", _d, [_i, _d, _d]),
    ("lbm_tau_lu_from_fd", _d, [_i, _d]),
    ("lbm_tau_fd_from_lu", _d, [_i, _d]),
    ("lbm_tau_star", _d, [_d]),
    ("lbm_fd_max_dt", _d, [_i, _d, _d]),
    ("lbm_velocity_set", _i, [_i, _D, _D, _D]),
    ("lbm_fit_decay", _i, [_D, _D, _i64, _d, _D, _D]),
    ("lbm_create", _i, [ctypes.POINTER(_P), _i, _i, _i, _i, _d, _d, _d, _i, _d, _P]),
    ("lbm_create_spec", _i, [ctypes.POINTER(_P), ctypes.POINTER(lbm_spec), _P]),
    ("lbm_spec_from_nu", _i, [ctypes.POINTER(lbm_spec), _d, _i, _i, ctypes.POINTER(lbm_spec)]),
    ("lbm_create_nu", _i, [ctypes.POINTER(_P), ctypes.POINTER(lbm_spec), _d, _i, _i, _P]),
    ("lbm_destroy", None, [_P]),
    ("lbm_get_spec", _i, [_P, ctypes.POINTER(lbm_spec)]),
    ("lbm_set_weno_eps", _i, [_P, _d]),
    ("lbm_inject_wait_timeout", _i, [_P, _i]),
    ("lbm_batch_inject_wait_timeout", _i, [_P, _i]),
    ("lbm_server_inject_wait_timeout", _i, [_P, _i]),
    ("lbm_init", _i, [_P, _D, _D, _D]),
    ("lbm_set_populations", _i, [_P, _D]),
    ("lbm_step", _i, [_P, _i64]),
    ("lbm_sync", _i, [_P]),
    ("lbm_steps_done", _i64, [_P]),
    ("lbm_moments", _i, [_P, _D, _D, _D]),
    ("lbm_populations", _i, [_P, _D]),
    ("lbm_populations_region", _i, [_P, _i, _i, _i, _i, _D]),
    ("lbm_set_probe", _i, [_P, _i, _D, _D, _d]),
    ("lbm_observables", _i, [_P, ctypes.POINTER(lbm_obs)]),
    ("lbm_record", _i, [_P, _i64, _i64]),
    ("lbm_series", _i, [_P, ctypes.POINTER(lbm_obs), _i64, ctypes.POINTER(_i64)]),
    ("lbm_checkpoint_size", _sz, [_P]),
    ("lbm_save", _i, [_P, _P, _sz]),
    ("lbm_load", _i, [_P, _P, _sz]),
    ("lbm_device_view", _i, [_P, ctypes.POINTER(lbm_view)]),
    ("lbm_batch_create", _i, [ctypes.POINTER(_P), ctypes.POINTER(lbm_spec), _i, _P]),
    ("lbm_batch_destroy", None, [_P]),
    ("lbm_batch_size", _i, [_P]),
    ("lbm_batch_init", _i, [_P, _i, _D, _D, _D]),
    ("lbm_batch_set_budget", _i, [_P, _i, _i64]),
    ("lbm_batch_step", _i, [_P, _i64]),
    ("lbm_batch_sync", _i, [_P]),
    ("lbm_batch_steps_done", _i64, [_P, _i]),
    ("lbm_batch_moments", _i, [_P, _i, _D, _D, _D]),
    ("lbm_batch_populations", _i, [_P, _i, _D]),
    ("lbm_batch_populations_region", _i, [_P, _i, _i, _i, _i, _i, _D]),
    ("lbm_batch_set_probe", _i, [_P, _i, _i, _D, _D, _d]),
    ("lbm_batch_observables", _i, [_P, _i, ctypes.POINTER(lbm_obs)]),
    ("lbm_batch_record", _i, [_P, _i, _i64, _i64]),
    ("lbm_batch_series", _i, [_P, _i, ctypes.POINTER(lbm_obs), _i64, ctypes.POINTER(_i64)]),
    ("lbm_batch_groups", _i, [_P, ctypes.POINTER(_i), ctypes.POINTER(_i), ctypes.POINTER(_i), _i]),
    ("lbm_batch_step_profiled", _i, [_P, _i64, _D, _i, _D]),
    ("lbm_batch_config", _i, [_P, _i, _i, _i]),
    ("lbm_config", _i, [_P, _i, _i]),
    ("lbm_n_tiles", _i, [_i]),
    ("lbm_batch_kernel_launches", _i64, [_P]),
    ("lbm_kernel_launches", _i64, [_P]),
    ("lbm_batch_tune", _i, [_P, _i, ctypes.c_char_p, _sz]),
    ("lbm_server_create", _i, [ctypes.POINTER(_P), _sz, _i, _i, _P]),
    ("lbm_submit", _i, [_P, ctypes.POINTER(lbm_request), ctypes.POINTER(ctypes.c_uint64)]),
    ("lbm_poll", _i, [_P, ctypes.c_uint64, ctypes.POINTER(lbm_result)]),
    ("lbm_result_series", _i, [_P, ctypes.c_uint64, ctypes.POINTER(lbm_obs), _i64, ctypes.POINTER(_i64)]),
    ("lbm_cancel", _i, [_P, ctypes.c_uint64]),
    ("lbm_probe_fp32", _i, [_i, _D, ctypes.POINTER(_i), _D]),
    ("lbm_result_moments", _i, [_P, ctypes.c_uint64, _D, _D, _D]),
    ("lbm_release", _i, [_P, ctypes.c_uint64]),
    ("lbm_server_drain", _i, [_P, _d]),
    ("lbm_server_stats", _i, [_P, ctypes.POINTER(_i64), ctypes.POINTER(_i64), ctypes.POINTER(_i64),
                              ctypes.POINTER(_sz)]),
    ("lbm_server_destroy", None, [_P]),
    ("lbm_server_plan_round", _i, [ctypes.POINTER(lbm_spec), ctypes.POINTER(_i64), _i, _i, ctypes.POINTER(_i64)]),
    ("lbm_footprint", _i, [ctypes.POINTER(lbm_spec), ctypes.POINTER(ctypes.c_size_t)]),
    ("lbm_observables_noalloc", _i, [_i, _i, _i, _i, _i, _P, _i64, ctypes.c_int32, ctypes.c_int32, _d, _i, _P, _P,
                                     _d, _i64, _d, _P, _P]),
]


def lib() -> ctypes.CDLL:
    """The loaded library; raises if it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"CUDA library not built ({LIB_PATH} missing): run "
                               "`python -c 'import __graft_entry__ as g; g.build()'` (needs nvcc)")
        L = ctypes.CDLL(LIB_PATH)
        for name, res, args in _SIGS:
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def lbm_n_tiles(model):
    return lib().lbm_n_tiles(MODELS[model] if isinstance(model, str) else model)


def exported_names():
    return [n for n, _, _ in _SIGS]


def strerror(code: int) -> str:
    return lib().lbm_strerror(code).decode()


def last_error() -> str:
    return lib().lbm_last_error().decode()


def check(rc: int, what: str):
    if rc != LBM_OK:
        raise LbmError(rc, what)


def _dp(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(_D)


def _f64(a, shape=None) -> np.ndarray:
    a = np.ascontiguousarray(a, dtype=np.float64)
    if shape is not None and a.shape != tuple(shape):
        raise ValueError(f"expected shape {shape}, got {a.shape}")
    return a


# ---- unit helpers ----------------------------------------------------------
def lbm_nu(model, tau, dt):
    return lib().lbm_nu(model, tau, dt)


def lbm_tau_lu_from_fd(n, tau_fd):
    return lib().lbm_tau_lu_from_fd(n, tau_fd)


def lbm_tau_fd_from_lu(n, tau_lu):
    return lib().lbm_tau_fd_from_lu(n, tau_lu)


def lbm_tau_star(tau_lu):
    return lib().lbm_tau_star(tau_lu)


def lbm_fd_max_dt(q, dx, tau):
    return lib().lbm_fd_max_dt(q, dx, tau)


def lbm_velocity_set(q):
    K = q * q
    vx, vy, w = np.zeros(K), np.zeros(K), np.zeros(K)
    check(lib().lbm_velocity_set(q, _dp(vx), _dp(vy), _dp(w)), "lbm_velocity_set")
    return vx, vy, w


def lbm_fit_decay(t, a, t_skip=0.0):
    t, a = _f64(t), _f64(a)
    g, a0 = ctypes.c_double(), ctypes.c_double()
    check(lib().lbm_fit_decay(_dp(t), _dp(a), len(t), t_skip, ctypes.byref(g), ctypes.byref(a0)), "lbm_fit_decay")
    return g.value, a0.value


def probe_fp32(packed=True):
    """Measured FP32 rate of the current device (lbm_probe_fp32): (flops/s,
    SM count, ms per probe launch)."""
    f, n, ms = ctypes.c_double(), ctypes.c_int(), ctypes.c_double()
    check(lib().lbm_probe_fp32(1 if packed else 0, ctypes.byref(f), ctypes.byref(n), ctypes.byref(ms)),
          "lbm_probe_fp32")
    return f.value, n.value, ms.value


MODELS = {"cs": LBM_CS, "fd": LBM_FD}
PRECISIONS = {"fp64": LBM_FP64, "fp32": LBM_FP32_DEV, "fp32dev": LBM_FP32_DEV}
LBM_STORE_AB, LBM_STORE_INPLACE = 0, 1
STORAGES = {"ab": LBM_STORE_AB, "inplace": LBM_STORE_INPLACE}
LBM_TS_RK3, LBM_TS_IMEX, LBM_TS_RK3_FUSED = 0, 1, 2
SCHEMES = {"rk3": LBM_TS_RK3, "imex": LBM_TS_IMEX, "rk3_fused": LBM_TS_RK3_FUSED}


def make_spec(model, q, nx, ny, tau, dt=0.0, dx=0.0, precision="fp64", rho0=0.0, storage="ab",
              scheme="rk3") -> lbm_spec:
    s = lbm_spec()
    s.model = MODELS[model] if isinstance(model, str) else model
    s.q_per_axis = q
    s.nx, s.ny = nx, ny
    s.precision = PRECISIONS[precision] if isinstance(precision, str) else precision
    s.storage = STORAGES[storage] if isinstance(storage, str) else storage
    s.scheme = SCHEMES[scheme] if isinstance(scheme, str) else scheme
    s.tau, s.dt, s.dx, s.rho0 = tau, dt, dx, rho0
    return s


def _stream_ptr(stream):
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream
    return int(stream.cuda_stream)  # torch.cuda.Stream


def spec_from_nu(model, q, nx, ny, nu, nu_model=None, n_ref=0, dt=0.0, dx=0.0, precision="fp64", rho0=0.0,
                 storage="ab", scheme="rk3") -> lbm_spec:
    """lbm_spec_from_nu: the resolved spec of a lattice given its viscosity
    (in the units of nu_model, default the lattice's own model)."""
    s = make_spec(model, q, nx, ny, 0.0, dt, dx, precision, rho0, storage, scheme)
    nm = s.model if nu_model is None else (MODELS[nu_model] if isinstance(nu_model, str) else nu_model)
    out = lbm_spec()
    check(lib().lbm_spec_from_nu(ctypes.byref(s), nu, nm, n_ref, ctypes.byref(out)), "lbm_spec_from_nu")
    return out


class Lattice:
    """One lattice context (lbm_create ... lbm_destroy). With nu given instead
    of tau (tau=None) the context is made by lbm_create_nu."""

    def __init__(self, model, q, nx, ny, tau, dt=0.0, dx=0.0, precision="fp64", rho0=0.0, stream=None, storage="ab",
                 nu=None, nu_model=None, n_ref=0, scheme="rk3"):
        self._h = ctypes.c_void_p()
        if tau is None:
            spec = make_spec(model, q, nx, ny, 0.0, dt, dx, precision, rho0, storage, scheme)
            nm = spec.model if nu_model is None else (MODELS[nu_model] if isinstance(nu_model, str) else nu_model)
            check(lib().lbm_create_nu(ctypes.byref(self._h), ctypes.byref(spec), nu, nm, n_ref,
                                      _stream_ptr(stream)), "lbm_create_nu")
        else:
            spec = make_spec(model, q, nx, ny, tau, dt, dx, precision, rho0, storage, scheme)
            check(lib().lbm_create_spec(ctypes.byref(self._h), ctypes.byref(spec), _stream_ptr(stream)),
                  "lbm_create")
        out = lbm_spec()
        check(lib().lbm_get_spec(self._h, ctypes.byref(out)), "lbm_get_spec")
        self.spec = out
        self.nx, self.ny, self.q = nx, ny, q
        self.K = q * q

    def close(self):
        if self._h:
            lib().lbm_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    @property
    def handle(self):
        return self._h

    def set_weno_eps(self, eps):
        check(lib().lbm_set_weno_eps(self._h, eps), "lbm_set_weno_eps")

    def inject_wait_timeout(self, microseconds):
        """Test injection: the next CS bulk-copy launches run a wait out (see lbm.h)."""
        check(lib().lbm_inject_wait_timeout(self._h, int(microseconds)), "lbm_inject_wait_timeout")

    def init(self, rho, ux, uy):
        shp = (self.ny, self.nx)
        r, u, v = _f64(rho, shp), _f64(ux, shp), _f64(uy, shp)
        check(lib().lbm_init(self._h, _dp(r), _dp(u), _dp(v)), "lbm_init")

    def set_populations(self, f):
        f = _f64(f, (self.K, self.ny, self.nx))
        check(lib().lbm_set_populations(self._h, _dp(f)), "lbm_set_populations")

    def step(self, n):
        check(lib().lbm_step(self._h, int(n)), "lbm_step")

    def sync(self):
        check(lib().lbm_sync(self._h), "lbm_sync")

    @property
    def steps_done(self):
        return lib().lbm_steps_done(self._h)

    def moments(self):
        r = np.empty((self.ny, self.nx))
        u = np.empty_like(r)
        v = np.empty_like(r)
        check(lib().lbm_moments(self._h, _dp(r), _dp(u), _dp(v)), "lbm_moments")
        return r, u, v

    def populations(self):
        f = np.empty((self.K, self.ny, self.nx))
        check(lib().lbm_populations(self._h, _dp(f)), "lbm_populations")
        return f

    def populations_region(self, x0, y0, wx, wy):
        f = np.empty((self.K, wy, wx))
        check(lib().lbm_populations_region(self._h, x0, y0, wx, wy, _dp(f)), "lbm_populations_region")
        return f

    def set_probe(self, comp, px, py, norm):
        px, py = _f64(px, (self.nx,)), _f64(py, (self.ny,))
        check(lib().lbm_set_probe(self._h, comp, _dp(px), _dp(py), norm), "lbm_set_probe")

    def observables(self):
        o = lbm_obs()
        check(lib().lbm_observables(self._h, ctypes.byref(o)), "lbm_observables")
        return o.as_dict()

    def record(self, every, capacity):
        check(lib().lbm_record(self._h, int(every), int(capacity)), "lbm_record")

    def series(self, cap=None):
        n = ctypes.c_int64()
        check(lib().lbm_series(self._h, None, 0, ctypes.byref(n)), "lbm_series")
        m = n.value if cap is None else min(cap, n.value)
        arr = (lbm_obs * max(m, 1))()
        check(lib().lbm_series(self._h, arr, m, ctypes.byref(n)), "lbm_series")
        return [arr[i].as_dict() for i in range(m)]

    def save(self) -> bytes:
        size = lib().lbm_checkpoint_size(self._h)
        buf = ctypes.create_string_buffer(size)
        check(lib().lbm_save(self._h, ctypes.cast(buf, ctypes.c_void_p), size), "lbm_save")
        return buf.raw

    def load(self, data: bytes):
        buf = ctypes.create_string_buffer(data, len(data))
        check(lib().lbm_load(self._h, ctypes.cast(buf, ctypes.c_void_p), len(data)), "lbm_load")

    @property
    def kernel_launches(self):
        return lib().lbm_kernel_launches(self._h)

    def config(self, tile, grid=0):
        check(lib().lbm_config(self._h, tile, grid), "lbm_config")

    def device_view(self):
        v = lbm_view()
        check(lib().lbm_device_view(self._h, ctypes.byref(v)), "lbm_device_view")
        return v


class Batch:
    """Many lattices advanced together (lbm_batch_*)."""

    def __init__(self, specs, stream=None):
        arr = (lbm_spec * len(specs))(*specs)
        self._h = ctypes.c_void_p()
        check(lib().lbm_batch_create(ctypes.byref(self._h), arr, len(specs), _stream_ptr(stream)), "lbm_batch_create")
        self.specs = list(specs)

    def close(self):
        if self._h:
            lib().lbm_batch_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __len__(self):
        return lib().lbm_batch_size(self._h)

    def _shape(self, i):
        s = self.specs[i]
        return s.ny, s.nx

    def init(self, i, rho, ux, uy):
        shp = self._shape(i)
        r, u, v = _f64(rho, shp), _f64(ux, shp), _f64(uy, shp)
        check(lib().lbm_batch_init(self._h, i, _dp(r), _dp(u), _dp(v)), "lbm_batch_init")

    def set_budget(self, i, steps):
        check(lib().lbm_batch_set_budget(self._h, i, int(steps)), "lbm_batch_set_budget")

    def step(self, n):
        check(lib().lbm_batch_step(self._h, int(n)), "lbm_batch_step")

    def inject_wait_timeout(self, microseconds):
        """Test injection: the next CS bulk-copy launches run a wait out (see lbm.h)."""
        check(lib().lbm_batch_inject_wait_timeout(self._h, int(microseconds)), "lbm_batch_inject_wait_timeout")

    def sync(self):
        check(lib().lbm_batch_sync(self._h), "lbm_batch_sync")

    def steps_done(self, i):
        return lib().lbm_batch_steps_done(self._h, i)

    def moments(self, i):
        ny, nx = self._shape(i)
        r, u, v = np.empty((ny, nx)), np.empty((ny, nx)), np.empty((ny, nx))
        check(lib().lbm_batch_moments(self._h, i, _dp(r), _dp(u), _dp(v)), "lbm_batch_moments")
        return r, u, v

    def populations(self, i):
        ny, nx = self._shape(i)
        K = self.specs[i].q_per_axis ** 2
        f = np.empty((K, ny, nx))
        check(lib().lbm_batch_populations(self._h, i, _dp(f)), "lbm_batch_populations")
        return f

    def populations_region(self, i, x0, y0, wx, wy):
        K = self.specs[i].q_per_axis ** 2
        f = np.empty((K, wy, wx))
        check(lib().lbm_batch_populations_region(self._h, i, x0, y0, wx, wy, _dp(f)), "lbm_batch_populations_region")
        return f

    def set_probe(self, i, comp, px, py, norm):
        ny, nx = self._shape(i)
        px, py = _f64(px, (nx,)), _f64(py, (ny,))
        check(lib().lbm_batch_set_probe(self._h, i, comp, _dp(px), _dp(py), norm), "lbm_batch_set_probe")

    def observables(self, i):
        o = lbm_obs()
        check(lib().lbm_batch_observables(self._h, i, ctypes.byref(o)), "lbm_batch_observables")
        return o.as_dict()

    def record(self, i, every, capacity):
        check(lib().lbm_batch_record(self._h, i, int(every), int(capacity)), "lbm_batch_record")

    def series(self, i, cap=None):
        n = ctypes.c_int64()
        check(lib().lbm_batch_series(self._h, i, None, 0, ctypes.byref(n)), "lbm_batch_series")
        m = n.value if cap is None else min(cap, n.value)
        arr = (lbm_obs * max(m, 1))()
        check(lib().lbm_batch_series(self._h, i, arr, m, ctypes.byref(n)), "lbm_batch_series")
        return [arr[k].as_dict() for k in range(m)]

    def groups(self):
        G = lib().lbm_batch_groups(self._h, None, None, None, 0)
        m, q, p = (ctypes.c_int * G)(), (ctypes.c_int * G)(), (ctypes.c_int * G)()
        lib().lbm_batch_groups(self._h, m, q, p, G)
        return [dict(model=m[g], q=q[g], precision=p[g]) for g in range(G)]

    def config(self, group, tile, grid=0):
        check(lib().lbm_batch_config(self._h, group, tile, grid), "lbm_batch_config")

    def step_profiled(self, n):
        """Returns (per-group list of {kind: ms}, total ms)."""
        G = len(self.groups())
        ms = np.zeros(4 * max(G, 1))
        tot = ctypes.c_double()
        check(lib().lbm_batch_step_profiled(self._h, int(n), _dp(ms), 4 * G, ctypes.byref(tot)),
              "lbm_batch_step_profiled")
        return ms.reshape(-1, 4), tot.value

    @property
    def kernel_launches(self):
        return lib().lbm_batch_kernel_launches(self._h)

    def tune(self, trial_steps=3):
        buf = ctypes.create_string_buffer(4096)
        check(lib().lbm_batch_tune(self._h, trial_steps, buf, 4096), "lbm_batch_tune")
        return buf.value.decode()


INITS = {"tg": 0, "taylor_green": 0, "shear": 1, "shock": 2}


def make_request(spec: lbm_spec, steps, init="tg", U=0.01, obs_every=0, rho_l=1.1, rho_r=0.9, tag=0,
                 keep_moments=False) -> lbm_request:
    r = lbm_request()
    r.spec = spec
    r.steps = int(steps)
    r.init = INITS[init] if isinstance(init, str) else init
    r.obs_every = int(obs_every)
    r.keep_moments = 1 if keep_moments else 0
    r.U, r.rho_l, r.rho_r = U, rho_l, rho_r
    r.user_tag = tag
    return r


def plan_round(specs, left, chunk_steps):
    """Steps each run advances in one server round (lbm_server_plan_round)."""
    n = len(specs)
    arr = (lbm_spec * max(n, 1))(*specs)
    lft = (_i64 * max(n, 1))(*[int(v) for v in left])
    out = (_i64 * max(n, 1))()
    check(lib().lbm_server_plan_round(arr, lft, n, int(chunk_steps), out), "lbm_server_plan_round")
    return [int(out[i]) for i in range(n)]


def footprint(spec):
    """Device bytes a lattice of this spec holds (lbm_footprint)."""
    out = ctypes.c_size_t()
    check(lib().lbm_footprint(ctypes.byref(spec), ctypes.byref(out)), "lbm_footprint")
    return out.value


class Server:
    """Continuous-batching run server (lbm_server_*)."""

    def __init__(self, hbm_budget_bytes, max_slots=64, chunk_steps=256, stream=None):
        self._h = ctypes.c_void_p()
        check(lib().lbm_server_create(ctypes.byref(self._h), int(hbm_budget_bytes), max_slots, chunk_steps,
                                      _stream_ptr(stream)), "lbm_server_create")

    def close(self):
        if self._h:
            lib().lbm_server_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def submit(self, req: lbm_request) -> int:
        t = ctypes.c_uint64()
        check(lib().lbm_submit(self._h, ctypes.byref(req), ctypes.byref(t)), "lbm_submit")
        return t.value

    def poll(self, ticket):
        r = lbm_result()
        rc = lib().lbm_poll(self._h, ticket, ctypes.byref(r))
        if rc == LBM_ENOTREADY:
            return None
        check(rc, "lbm_poll")
        return r.as_dict()

    def series(self, ticket):
        n = ctypes.c_int64()
        check(lib().lbm_result_series(self._h, ticket, None, 0, ctypes.byref(n)), "lbm_result_series")
        arr = (lbm_obs * max(n.value, 1))()
        check(lib().lbm_result_series(self._h, ticket, arr, n.value, ctypes.byref(n)), "lbm_result_series")
        return [arr[i].as_dict() for i in range(n.value)]

    def moments(self, ticket, nx, ny):
        """Kept final fields of a finished run (lbm_result_moments)."""
        r, u, v = np.empty((ny, nx)), np.empty((ny, nx)), np.empty((ny, nx))
        check(lib().lbm_result_moments(self._h, ticket, _dp(r), _dp(u), _dp(v)), "lbm_result_moments")
        return r, u, v

    def release(self, ticket):
        check(lib().lbm_release(self._h, ticket), "lbm_release")

    def cancel(self, ticket):
        check(lib().lbm_cancel(self._h, ticket), "lbm_cancel")

    def inject_wait_timeout(self, microseconds):
        """Test injection from the next round on (see lbm.h)."""
        check(lib().lbm_server_inject_wait_timeout(self._h, int(microseconds)), "lbm_server_inject_wait_timeout")

    def drain(self, timeout_s=600.0):
        check(lib().lbm_server_drain(self._h, timeout_s), "lbm_server_drain")

    def stats(self):
        q, r, f, b = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64(), ctypes.c_size_t()
        check(lib().lbm_server_stats(self._h, ctypes.byref(q), ctypes.byref(r), ctypes.byref(f), ctypes.byref(b)),
              "lbm_server_stats")
        return dict(queued=q.value, running=r.value, finished=f.value, resident_bytes=b.value)
