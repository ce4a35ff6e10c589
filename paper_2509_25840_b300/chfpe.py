"""Thin ctypes binding of libchfpe.so (include/chfpe.h): argument marshalling only.

Every numerical step runs in the library's CUDA kernels.  Loading fails loudly when the library
is missing or cannot be opened; there is no CPU fallback.  Device buffers are passed as raw
pointers (e.g. ``tensor.data_ptr()`` of a contiguous torch CUDA tensor of the handle's dtype).
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import inputs

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libchfpe.so")

OK, EINVAL, ENOMEM, ECUDA, EUNSTABLE, ETIMEOUT, ESTATE = range(7)
STAGE_VARIANTS = 18
_NAMES = {0: "CHFPE_OK", 1: "CHFPE_EINVAL", 2: "CHFPE_ENOMEM", 3: "CHFPE_ECUDA",
          4: "CHFPE_EUNSTABLE", 5: "CHFPE_ETIMEOUT", 6: "CHFPE_ESTATE"}


class ChfpeError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{_NAMES.get(status, status)}: {message}")
        self.status = status


class chfpe_model(ctypes.Structure):
    _fields_ = [("nmodes", ctypes.c_int), ("kT", ctypes.c_double),
                ("m", ctypes.c_double * 3), ("omega", ctypes.c_double * 3),
                ("g3", ctypes.c_double * 3), ("g4", ctypes.c_double * 3),
                ("g2", (ctypes.c_double * 3) * 3), ("g_s2s", (ctypes.c_double * 3) * 3),
                ("g_ss2", (ctypes.c_double * 3) * 3),
                ("zeta", ctypes.c_double * 3), ("gamma", ctypes.c_double * 3),
                ("V_LL", ctypes.c_double * 3), ("V_SL", ctypes.c_double * 3)]


class chfpe_optical(ctypes.Structure):
    _fields_ = [("lin", ctypes.c_double * 3), ("quad", (ctypes.c_double * 3) * 3)]


class chfpe_grid(ctypes.Structure):
    _fields_ = [("nq", ctypes.c_int * 3), ("np", ctypes.c_int * 3),
                ("qmin", ctypes.c_double * 3), ("qmax", ctypes.c_double * 3),
                ("pmin", ctypes.c_double * 3), ("pmax", ctypes.c_double * 3)]


class chfpe_options(ctypes.Structure):
    _fields_ = [("depth", ctypes.c_int), ("precision", ctypes.c_int), ("dt", ctypes.c_double),
                ("max_batch", ctypes.c_int), ("stream", ctypes.c_void_p), ("bf16_tier", ctypes.c_int),
                ("truncation", ctypes.c_int), ("p_basis", ctypes.c_int), ("q_scheme", ctypes.c_int)]


class chfpe_stats(ctypes.Structure):
    _fields_ = [("kernel_launches", ctypes.c_longlong), ("stage_launches", ctypes.c_longlong),
                ("stage_ms", ctypes.c_double), ("stage_bytes", ctypes.c_double),
                ("cell_updates", ctypes.c_double)]


_lib = None
_DP = ctypes.POINTER(ctypes.c_double)
_FP = ctypes.POINTER(ctypes.c_float)
_VP = ctypes.c_void_p
_H = ctypes.c_void_p


def load(path: str = LIB_PATH):
    """Open libchfpe.so (once).  Raises if it is missing: build it with
    ``python -m paper_2509_25840_b300.build`` or ``__graft_entry__.build()``."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"libchfpe.so not found at {path}; build it first "
                           "(python -m paper_2509_25840_b300.build)")
    lib = ctypes.CDLL(path)
    S = ctypes.c_int
    sig = {
        "chfpe_create": ([ctypes.POINTER(chfpe_model), ctypes.POINTER(chfpe_grid),
                          ctypes.POINTER(chfpe_options), ctypes.POINTER(_H)], S),
        "chfpe_destroy": ([_H], None),
        "chfpe_equilibrate": ([_H, ctypes.c_long, ctypes.c_double, ctypes.c_long,
                               ctypes.POINTER(ctypes.c_long), _DP], S),
        "chfpe_set_equilibrium": ([_H, _DP], S),
        "chfpe_get_equilibrium": ([_H, _DP], S),
        "chfpe_set_state": ([_H, _DP], S),
        "chfpe_get_state": ([_H, _DP], S),
        "chfpe_propagate": ([_H, ctypes.c_long], S),
        "chfpe_response1": ([_H, ctypes.POINTER(chfpe_optical), ctypes.POINTER(chfpe_optical),
                             ctypes.c_int, ctypes.c_int, _DP], S),
        "chfpe_response2": ([_H, ctypes.POINTER(chfpe_optical), ctypes.POINTER(chfpe_optical),
                             ctypes.POINTER(chfpe_optical), ctypes.c_int, ctypes.c_int,
                             ctypes.c_int, _DP], S),
        "chfpe_response3": ([_H, ctypes.POINTER(chfpe_optical), ctypes.POINTER(chfpe_optical),
                             ctypes.POINTER(chfpe_optical), ctypes.POINTER(chfpe_optical),
                             ctypes.c_int, ctypes.c_long, ctypes.c_int, ctypes.c_int, _DP], S),
        "chfpe_save_equilibrium": ([_H, ctypes.c_char_p], S),
        "chfpe_load_equilibrium": ([_H, ctypes.c_char_p], S),
        "chfpe_sizes": ([_H, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_long)], S),
        "chfpe_rhs_device": ([_H, _VP, _VP, ctypes.c_int], S),
        "chfpe_rk4_device": ([_H, _VP, ctypes.c_int, ctypes.c_long], S),
        "chfpe_insert_device": ([_H, ctypes.POINTER(chfpe_optical), _VP, _VP, ctypes.c_int], S),
        "chfpe_observe_device": ([_H, ctypes.POINTER(chfpe_optical), _VP, ctypes.c_int, _VP], S),
        "chfpe_sample_device": ([_H, ctypes.POINTER(chfpe_optical), _VP, ctypes.c_int, ctypes.c_int,
                                 ctypes.c_int, _VP, ctypes.c_long], S),
        "chfpe_observe_noalloc": ([ctypes.POINTER(chfpe_model), ctypes.POINTER(chfpe_grid),
                                   ctypes.c_int, ctypes.c_int, ctypes.POINTER(chfpe_optical),
                                   _VP, ctypes.c_int, _VP, _VP], S),
        "chfpe_create_batch": ([ctypes.c_int, ctypes.POINTER(chfpe_model), ctypes.POINTER(chfpe_grid),
                                ctypes.POINTER(chfpe_options), ctypes.POINTER(_H)], S),
        "chfpe_batch_instance": ([_H, ctypes.c_int, ctypes.POINTER(_H)], S),
        "chfpe_time_step": ([_H, _DP], S),
        "chfpe_batch_equilibrate": ([_H, ctypes.c_long, ctypes.c_double, ctypes.c_long, _DP], S),
        "chfpe_batch_response1": ([_H, ctypes.POINTER(chfpe_optical), ctypes.POINTER(chfpe_optical),
                                   ctypes.c_int, ctypes.c_int, _DP], S),
        "chfpe_batch_response2": ([_H, ctypes.POINTER(chfpe_optical), ctypes.POINTER(chfpe_optical),
                                   ctypes.POINTER(chfpe_optical), ctypes.c_int, ctypes.c_int,
                                   ctypes.c_int, _DP], S),
        "chfpe_spectrum1": ([_DP, ctypes.c_int, ctypes.c_double, ctypes.c_int, ctypes.c_double,
                             _DP, _VP], S),
        "chfpe_spectrum2": ([_DP, ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_int,
                             ctypes.c_int, ctypes.c_double, _DP, _VP], S),
        "chfpe_spectrum3": ([_DP, ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_int,
                             ctypes.c_int, ctypes.c_double, _DP, _VP], S),
        "chfpe_stats_reset": ([_H, ctypes.c_int], S),
        "chfpe_stats_get": ([_H, ctypes.POINTER(chfpe_stats)], S),
        "chfpe_alu_peak": ([ctypes.c_int, _VP, ctypes.POINTER(ctypes.c_double)], S),
        "chfpe_last_error": ([], ctypes.c_char_p),
        "chfpe_stage_tuning": ([_H, ctypes.POINTER(ctypes.c_int), _DP], S),
        "chfpe_surrogate_param_count": ([], ctypes.c_longlong),
        "chfpe_surrogate_create": ([ctypes.c_int, ctypes.c_ulonglong, _VP, ctypes.POINTER(_H)], S),
        "chfpe_surrogate_destroy": ([_H], None),
        "chfpe_surrogate_get_params": ([_H, _FP], S),
        "chfpe_surrogate_set_params": ([_H, _FP], S),
        "chfpe_surrogate_infer": ([_H, _VP, ctypes.c_int, _VP, _VP], S),
        "chfpe_surrogate_gradients": ([_H, _VP, _VP, _VP, ctypes.c_int, ctypes.c_float, _DP, _FP], S),
        "chfpe_surrogate_train": ([_H, _VP, _VP, _VP, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                   ctypes.c_float, ctypes.c_float, ctypes.c_float,
                                   ctypes.c_ulonglong, _DP], S),
        "chfpe_surrogate_gemm": ([_VP, ctypes.c_int, ctypes.c_int, _VP, ctypes.c_int, ctypes.c_int,
                                  _VP, _VP, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                  _VP], S),
    }
    for name, (args, res) in sig.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = res
    _lib = lib
    return lib


def alu_peak(precision: int, stream: int | None = None) -> float:
    """chfpe_alu_peak: measured FMA throughput of the FP64 or FP32 ALUs in FLOP/s."""
    out = ctypes.c_double(0.0)
    _check(load().chfpe_alu_peak(int(precision), stream, ctypes.byref(out)))
    return out.value


def last_error() -> str:
    return load().chfpe_last_error().decode()


def _check(status: int):
    if status != OK:
        raise ChfpeError(status, last_error())


def _fill(arr, vals, n=3):
    vals = list(vals) + [0] * n
    for i in range(n):
        arr[i] = vals[i]


def make_model(model: "inputs.Model") -> chfpe_model:
    m = chfpe_model()
    m.nmodes = int(model.nmodes)
    m.kT = float(model.kT)
    for name in ("m", "omega", "g3", "g4", "zeta", "gamma", "V_LL", "V_SL"):
        _fill(getattr(m, name), [float(x) for x in getattr(model, name)])
    for name in ("g2", "g_s2s", "g_ss2"):
        src = np.asarray(getattr(model, name), dtype=np.float64)
        dst = getattr(m, name)
        for i in range(3):
            for j in range(3):
                dst[i][j] = float(src[i, j]) if i < src.shape[0] and j < src.shape[1] else 0.0
    return m


def make_grid(grid: "inputs.Grid") -> chfpe_grid:
    g = chfpe_grid()
    _fill(g.nq, [int(x) for x in grid.nq])
    _fill(g.np, [int(x) for x in grid.np])
    for name in ("qmin", "qmax", "pmin", "pmax"):
        _fill(getattr(g, name), [float(x) for x in getattr(grid, name)])
    return g


def make_optical(X: "inputs.Optical") -> chfpe_optical:
    o = chfpe_optical()
    _fill(o.lin, [float(x) for x in X.lin])
    q = np.asarray(X.quad, dtype=np.float64)
    for i in range(3):
        for j in range(3):
            o.quad[i][j] = float(q[i, j]) if i < q.shape[0] and j < q.shape[1] else 0.0
    return o


def _dptr(a: np.ndarray):
    return a.ctypes.data_as(_DP)


def observe_noalloc(model, grid, depth: int, precision: int, C, states_ptr: int, batch: int,
                    R_ptr: int, stream: int | None = None):
    """chfpe_observe_noalloc: the observable of `batch` device states into device doubles at
    R_ptr, without any device allocation (fixed 256 KB reduction scratch inside the library)."""
    m, g, c = make_model(model), make_grid(grid), make_optical(C)
    _check(load().chfpe_observe_noalloc(ctypes.byref(m), ctypes.byref(g), int(depth),
                                        int(precision), ctypes.byref(c), states_ptr, int(batch),
                                        R_ptr, stream))


def frequencies(L: int, dtau: float) -> np.ndarray:
    """The centred frequency grid of the spectra: w_j = 2 pi (j - L/2) / (L dtau)."""
    return 2.0 * np.pi * (np.arange(L) - L // 2) / (L * dtau)


def spectrum1(R1, dtau: float, L: int, eta: float = 0.0, stream: int | None = None) -> np.ndarray:
    """chfpe_spectrum1 (Eq. 1DIR_Raman): I[j] on frequencies(L, dtau)."""
    R = np.ascontiguousarray(R1, dtype=np.float64)
    out = np.empty(int(L))
    _check(load().chfpe_spectrum1(_dptr(R), R.shape[0], float(dtau), int(L), float(eta),
                                  _dptr(out), stream))
    return out


def spectrum2(R2, dtau: float, L1: int, L2: int, eta: float = 0.0,
              stream: int | None = None) -> np.ndarray:
    """chfpe_spectrum2 (Eq. 2DThz_Raman): I[w1][w2] from R2[t1][t2]."""
    R = np.ascontiguousarray(R2, dtype=np.float64)
    out = np.empty((int(L1), int(L2)))
    _check(load().chfpe_spectrum2(_dptr(R), R.shape[0], R.shape[1], float(dtau), int(L1), int(L2),
                                  float(eta), _dptr(out), stream))
    return out


def spectrum3(R3, dtau: float, L1: int, L3: int, eta: float = 0.0,
              stream: int | None = None) -> np.ndarray:
    """chfpe_spectrum3 (Eq. noncorrelation at one t2): I[w1][w3] from R3[t1][t3]."""
    R = np.ascontiguousarray(R3, dtype=np.float64)
    out = np.empty((int(L1), int(L3)))
    _check(load().chfpe_spectrum3(_dptr(R), R.shape[0], R.shape[1], float(dtau), int(L1), int(L3),
                                  float(eta), _dptr(out), stream))
    return out


class Handle:
    """One model on one grid: owns the device arenas of libchfpe."""

    def __init__(self, model, grid, depth: int, dt: float, precision: int = 32,
                 max_batch: int = 1, stream: int | None = None, bf16_tier: int = 0,
                 p_basis: int = 0, q_scheme: int = 0):
        """p_basis = 1: momenta in grid.np[s] Hermite functions (states hold coefficients);
        q_scheme = 1 (with p_basis = 1): compact q-derivatives solved by PCR; 2: their
        skew-symmetric part."""
        lib = load()
        self._m, self._g = make_model(model), make_grid(grid)
        self._o = chfpe_options(depth=int(depth), precision=int(precision), dt=float(dt),
                                max_batch=int(max_batch), stream=stream, bf16_tier=int(bf16_tier),
                                p_basis=int(p_basis), q_scheme=int(q_scheme))
        h = _H()
        _check(lib.chfpe_create(ctypes.byref(self._m), ctypes.byref(self._g),
                                ctypes.byref(self._o), ctypes.byref(h)))
        self._h = h
        M, P = ctypes.c_int(), ctypes.c_long()
        _check(lib.chfpe_sizes(h, ctypes.byref(M), ctypes.byref(P)))
        self.members, self.points = M.value, P.value
        self.shape = tuple(grid.nq) + tuple(grid.np)
        self.precision = int(precision)
        self.max_batch = int(max_batch)

    @classmethod
    def _borrowed(cls, h, grid, precision: int):
        """Wrap an instance handle owned by a batch (closing the wrapper does not destroy it)."""
        self = cls.__new__(cls)
        self._h = h
        self._owner = False
        M, P = ctypes.c_int(), ctypes.c_long()
        _check(load().chfpe_sizes(h, ctypes.byref(M), ctypes.byref(P)))
        self.members, self.points = M.value, P.value
        self.shape = tuple(grid.nq) + tuple(grid.np)
        self.precision = int(precision)
        self.max_batch = 0
        return self

    # -- lifetime -------------------------------------------------------------------------
    def close(self):
        if getattr(self, "_h", None):
            if getattr(self, "_owner", True):
                load().chfpe_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    @property
    def state_shape(self):
        return (self.members,) + self.shape

    def _host(self, a) -> np.ndarray:
        a = np.ascontiguousarray(a, dtype=np.float64)
        if a.size != self.members * self.points:
            raise ValueError(f"state has {a.size} values, expected {self.members * self.points}")
        return a

    # -- equilibrium and states -------------------------------------------------------------
    def equilibrate(self, max_steps: int, tol: float, check_every: int = 100):
        steps, res = ctypes.c_long(), ctypes.c_double()
        _check(load().chfpe_equilibrate(self._h, int(max_steps), float(tol), int(check_every),
                                        ctypes.byref(steps), ctypes.byref(res)))
        return steps.value, res.value

    def set_equilibrium(self, W):
        a = self._host(W)
        _check(load().chfpe_set_equilibrium(self._h, _dptr(a)))

    def get_equilibrium(self) -> np.ndarray:
        out = np.empty(self.state_shape)
        _check(load().chfpe_get_equilibrium(self._h, _dptr(out)))
        return out

    def set_state(self, W):
        a = self._host(W)
        _check(load().chfpe_set_state(self._h, _dptr(a)))

    def get_state(self) -> np.ndarray:
        out = np.empty(self.state_shape)
        _check(load().chfpe_get_state(self._h, _dptr(out)))
        return out

    def time_step(self) -> float:
        """chfpe_time_step: this handle's RK4 step (dt / nsub_i for a batch instance)."""
        v = ctypes.c_double()
        _check(load().chfpe_time_step(self._h, ctypes.byref(v)))
        return v.value

    def propagate(self, nsteps: int):
        _check(load().chfpe_propagate(self._h, int(nsteps)))

    def save_equilibrium(self, path: str):
        _check(load().chfpe_save_equilibrium(self._h, os.fsencode(path)))

    def load_equilibrium(self, path: str):
        _check(load().chfpe_load_equilibrium(self._h, os.fsencode(path)))

    # -- responses ----------------------------------------------------------------------------
    def response1(self, A, C, nt: int, stride: int, out: np.ndarray | None = None) -> np.ndarray:
        R = np.empty(nt) if out is None else out
        a, c = make_optical(A), make_optical(C)
        _check(load().chfpe_response1(self._h, ctypes.byref(a), ctypes.byref(c), int(nt),
                                      int(stride), _dptr(R)))
        return R

    def response2(self, A, B, C, nt1: int, nt2: int, stride: int,
                  out: np.ndarray | None = None) -> np.ndarray:
        R = np.empty((nt1, nt2)) if out is None else out
        a, b, c = make_optical(A), make_optical(B), make_optical(C)
        _check(load().chfpe_response2(self._h, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c),
                                      int(nt1), int(nt2), int(stride), _dptr(R)))
        return R

    def response3(self, A, B, C, D, nt1: int, n2: int, nt3: int, stride: int,
                  out: np.ndarray | None = None) -> np.ndarray:
        """chfpe_response3 (Eq. 3Dresponse) at waiting time n2 dt: R[t1][t3]."""
        R = np.empty((nt1, nt3)) if out is None else out
        a, b, c, d = make_optical(A), make_optical(B), make_optical(C), make_optical(D)
        _check(load().chfpe_response3(self._h, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c),
                                      ctypes.byref(d), int(nt1), int(n2), int(nt3), int(stride),
                                      _dptr(R)))
        return R

    def stage_tuning(self):
        """(chosen launch shape, microseconds per stage launch of each shape or -1)."""
        v = ctypes.c_int()
        us = np.zeros(STAGE_VARIANTS)
        _check(load().chfpe_stage_tuning(self._h, ctypes.byref(v), _dptr(us)))
        return v.value, us

    # -- device buffers -------------------------------------------------------------------------
    def rhs_device(self, in_ptr: int, out_ptr: int, batch: int = 1):
        _check(load().chfpe_rhs_device(self._h, in_ptr, out_ptr, int(batch)))

    def rk4_device(self, ptr: int, batch: int, nsteps: int):
        _check(load().chfpe_rk4_device(self._h, ptr, int(batch), int(nsteps)))

    def insert_device(self, X, in_ptr: int, out_ptr: int, batch: int = 1):
        x = make_optical(X)
        _check(load().chfpe_insert_device(self._h, ctypes.byref(x), in_ptr, out_ptr, int(batch)))

    def observe_device(self, C, in_ptr: int, batch: int, R_ptr: int):
        c = make_optical(C)
        _check(load().chfpe_observe_device(self._h, ctypes.byref(c), in_ptr, int(batch), R_ptr))

    def sample_device(self, C, states_ptr: int, batch: int, nsamples: int, stride: int,
                      R_ptr: int, ld: int | None = None):
        """chfpe_sample_device: observe C every `stride` RK4 steps of `batch` device states
        (nsamples samples, the states advance in place) into device doubles R[b * ld + k]."""
        c = make_optical(C)
        _check(load().chfpe_sample_device(self._h, ctypes.byref(c), states_ptr, int(batch),
                                          int(nsamples), int(stride), R_ptr,
                                          int(nsamples if ld is None else ld)))

    # -- counters ---------------------------------------------------------------------------------
    def stats_reset(self, time_stages: bool = False):
        _check(load().chfpe_stats_reset(self._h, int(bool(time_stages))))

    def stats(self) -> dict:
        st = chfpe_stats()
        _check(load().chfpe_stats_get(self._h, ctypes.byref(st)))
        return {k: getattr(st, k) for k, _ in chfpe_stats._fields_}


class Batch(Handle):
    """chfpe_create_batch: n instances (models, grids) advanced together by one launch per RK4
    stage; instance(i) gives the borrowed per-instance handle."""

    def __init__(self, models, grids, depth: int, dt: float, precision: int = 32,
                 stream: int | None = None, bf16_tier: int = 0, max_batch: int = 0):
        lib = load()
        n = len(models)
        self._ms = (chfpe_model * n)(*[make_model(m) for m in models])
        self._gs = (chfpe_grid * n)(*[make_grid(g) for g in grids])
        self._o = chfpe_options(depth=int(depth), precision=int(precision), dt=float(dt),
                                max_batch=int(max_batch), stream=stream, bf16_tier=int(bf16_tier))
        h = _H()
        _check(lib.chfpe_create_batch(n, self._ms, self._gs, ctypes.byref(self._o), ctypes.byref(h)))
        self._h = h
        self._owner = True
        self.n = n
        self.grids = list(grids)
        self.precision = int(precision)
        self._inst = [None] * n

    def instance(self, i: int) -> Handle:
        if self._inst[i] is None:
            h = _H()
            _check(load().chfpe_batch_instance(self._h, int(i), ctypes.byref(h)))
            self._inst[i] = Handle._borrowed(h, self.grids[i], self.precision)
        return self._inst[i]

    def equilibrate_all(self, max_steps: int, tol: float, check_every: int = 100) -> np.ndarray:
        r = np.zeros(self.n)
        _check(load().chfpe_batch_equilibrate(self._h, int(max_steps), float(tol), int(check_every),
                                              _dptr(r)))
        return r

    def response1_all(self, A, C, nt: int, stride: int) -> np.ndarray:
        R = np.empty((self.n, nt))
        a, c = make_optical(A), make_optical(C)
        _check(load().chfpe_batch_response1(self._h, ctypes.byref(a), ctypes.byref(c), int(nt),
                                            int(stride), _dptr(R)))
        return R

    def response2_all(self, A, B, C, nt1: int, nt2: int, stride: int) -> np.ndarray:
        """chfpe_batch_response2: R[i, a, b] of every instance (branches batched across the
        instances, max_batch t1 rows per chunk)."""
        R = np.empty((self.n, nt1, nt2))
        a, b, c = make_optical(A), make_optical(B), make_optical(C)
        _check(load().chfpe_batch_response2(self._h, ctypes.byref(a), ctypes.byref(b),
                                            ctypes.byref(c), int(nt1), int(nt2), int(stride),
                                            _dptr(R)))
        return R

    def close(self):
        for w in getattr(self, "_inst", []) or []:
            if w is not None:
                w._h = None
        super().close()


# ------------------------------------------------------------------------------------------
# learned surrogate (chfpe_surrogate_*): device pointers are passed as integers
# ------------------------------------------------------------------------------------------

SURROGATE_NIN, SURROGATE_NOUT = 12, 4096


def surrogate_param_count() -> int:
    return int(load().chfpe_surrogate_param_count())


def surrogate_gemm(A_ptr: int, ta: bool, lda: int, B_ptr: int, tb: bool, ldb: int, C_ptr: int,
                   bias_ptr: int | None, M: int, N: int, K: int, splits: int = 1,
                   stream: int | None = None):
    """chfpe_surrogate_gemm: the BF16 tensor-core GEMM alone (BF16 A, B; FP32 C and bias)."""
    _check(load().chfpe_surrogate_gemm(A_ptr, int(bool(ta)), int(lda), B_ptr, int(bool(tb)),
                                       int(ldb), C_ptr, bias_ptr, int(M), int(N), int(K),
                                       int(splits), stream))


class Surrogate:
    """chfpe_surrogate: the 12 -> 64 x 64 network, its training and inference on the device."""

    def __init__(self, max_batch: int = 256, seed: int = 1, stream: int | None = None):
        h = _H()
        _check(load().chfpe_surrogate_create(int(max_batch), int(seed), stream, ctypes.byref(h)))
        self._h = h
        self.max_batch = int(max_batch)
        self.stream = stream          # cudaStream_t the calls run on (None: the handle's own)
        self.nparam = surrogate_param_count()

    def close(self):
        if getattr(self, "_h", None):
            load().chfpe_surrogate_destroy(self._h)
            self._h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def get_params(self) -> np.ndarray:
        out = np.empty(self.nparam, dtype=np.float32)
        _check(load().chfpe_surrogate_get_params(self._h, out.ctypes.data_as(_FP)))
        return out

    def set_params(self, flat: np.ndarray):
        a = np.ascontiguousarray(flat, dtype=np.float32)
        if a.size != self.nparam:
            raise ValueError(f"expected {self.nparam} parameters, got {a.size}")
        _check(load().chfpe_surrogate_set_params(self._h, a.ctypes.data_as(_FP)))

    def infer(self, X_ptr: int, n: int, Y_ptr: int, S_ptr: int):
        _check(load().chfpe_surrogate_infer(self._h, X_ptr, int(n), Y_ptr, S_ptr))

    def gradients(self, X_ptr: int, T_ptr: int, TS_ptr: int, n: int, w_scale: float = 1.0,
                  want_grads: bool = True):
        loss = ctypes.c_double()
        g = np.empty(self.nparam, dtype=np.float32) if want_grads else None
        _check(load().chfpe_surrogate_gradients(self._h, X_ptr, T_ptr, TS_ptr, int(n),
                                                float(w_scale), ctypes.byref(loss),
                                                g.ctypes.data_as(_FP) if want_grads else None))
        return loss.value, g

    def train(self, X_ptr: int, T_ptr: int, TS_ptr: int, n: int, batch: int, epochs: int,
              lr: float, weight_decay: float = 0.0, w_scale: float = 1.0, seed: int = 0):
        losses = np.zeros(max(int(epochs), 1), dtype=np.float64)
        _check(load().chfpe_surrogate_train(self._h, X_ptr, T_ptr, TS_ptr, int(n), int(batch),
                                            int(epochs), float(lr), float(weight_decay),
                                            float(w_scale), int(seed), _dptr(losses)))
        return losses[:int(epochs)]
