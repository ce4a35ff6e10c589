"""FP64 CPU oracle for the CHFPE hot path -- TEST INFRASTRUCTURE.

This package wraps ``chfpe_oracle.c``, a plain, slow, obviously-correct FP64 restatement of the
multimode classical hierarchical Fokker-Planck equations of arXiv 2509.25840 (Eq. HEOM with
Eqs. CL_liouville, Phi, Theta; insertion Eq. Opticalexc; responses Eqs. 1Dresponse and
2Dresponse).  States hold the symmetrised members g^(n) = W^(n) exp(H/2kT) / lambda_n (the
exp(-H/2kT) prefactor of Appendix A); ``to_density`` maps them back to W^(n).  It exists to check the CUDA library against.  Only the tests, the smoke check and
the benchmark's CPU-baseline / reference leg may import it; the product path never does.

It shares no code with the CUDA library: its own C source, its own ctypes structs, its own
build command.  Model parameters come in as the plain containers of
``paper_2509_25840_b300.inputs`` (which hold numbers only, no arithmetic of the method).

Parity status per function (what pins it; the pins live in ``tests/test_oracle_pins.py``):
  deriv1d      Taylor exactness on polynomials of degree <= 6, antisymmetry, 6th-order rate
  potential,   symbolic differentiation (sympy) of the paper's polynomial
  dUdq
  rhs          Boltzmann stationarity (any U, any V_LL/V_SL) at 6th order, norm conservation of
               W^(0), closed-form R1/R2 of the harmonic Brownian oscillator, moment closure
               (multimode harmonic + bilinear coupling), classical-trajectory R1 (anharmonic,
               zeta = 0), separability, reciprocity of equilibrium correlations (LL + SL)
  rk4          the RK4 stability polynomial applied to the extracted generator
  insert       analytic derivative of the Boltzmann distribution; zero total mass
  observe      Gaussian moments of the sampled Boltzmann distribution
  residual     zero on an exact null vector of the extracted generator, invariance under scaling,
               sixth-order decay on the sampled Boltzmann state
  equilibrate  stationarity of its result; agreement with the sampled Boltzmann to O(h^6)
  response1/2  closed forms and moment closure above
  response3    the moment closure (one mode, deep hierarchy, linear and quadratic optics) and
               the vanishing third-order response of the harmonic / all-linear case
  h_*          (Hermite-function momenta, Appendix A) the antisymmetry of the ladder generator,
               Boltzmann stationarity, the Brownian closed form, the moment closure, and the
               grid representation's responses on the same model; with qscheme = 1 (compact q
               derivatives, Sec. III B) the Brownian closed form and Boltzmann stationarity;
               with qscheme = 2 (its skew-symmetric part) also the antisymmetry of the generator
  compact_deriv1d  exactness on polynomials of degree <= 6 away from the ends, the scheme's
               closed-form Fourier symbol, the truncation-error constant against the explicit
               stencil (1/9 of it), decay of the end effect at the rate of A's Green's function
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "chfpe_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (OpenMP on, no fast-math, no FMA contraction: IEEE FP64)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-fPIC", "-shared", "-fopenmp", "-fno-fast-math",
               "-ffp-contract=off", "-std=c11", _SRC, "-o", tmp, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


class _Problem(ctypes.Structure):
    _fields_ = [
        ("d", ctypes.c_int), ("depth", ctypes.c_int), ("kT", ctypes.c_double),
        ("m", ctypes.c_double * 3), ("omega", ctypes.c_double * 3),
        ("g3", ctypes.c_double * 3), ("g4", ctypes.c_double * 3),
        ("g2", (ctypes.c_double * 3) * 3), ("g_s2s", (ctypes.c_double * 3) * 3),
        ("g_ss2", (ctypes.c_double * 3) * 3),
        ("zeta", ctypes.c_double * 3), ("gamma", ctypes.c_double * 3),
        ("V_LL", ctypes.c_double * 3), ("V_SL", ctypes.c_double * 3),
        ("nq", ctypes.c_int * 3), ("np", ctypes.c_int * 3),
        ("qmin", ctypes.c_double * 3), ("qmax", ctypes.c_double * 3),
        ("pmin", ctypes.c_double * 3), ("pmax", ctypes.c_double * 3),
        ("qscheme", ctypes.c_int),
    ]


class _Optical(ctypes.Structure):
    _fields_ = [("lin", ctypes.c_double * 3), ("quad", (ctypes.c_double * 3) * 3)]


_DP = ctypes.POINTER(ctypes.c_double)


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            P = ctypes.POINTER(_Problem)
            O = ctypes.POINTER(_Optical)
            lib.orc_threads.restype = ctypes.c_int
            lib.orc_members.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_int)]
            lib.orc_member_count.argtypes = [ctypes.c_int, ctypes.c_int]
            lib.orc_points.argtypes = [P]
            lib.orc_points.restype = ctypes.c_long
            lib.orc_potential.argtypes = [P, _DP]
            lib.orc_potential.restype = ctypes.c_double
            lib.orc_dUdq.argtypes = [P, _DP, ctypes.c_int]
            lib.orc_dUdq.restype = ctypes.c_double
            lib.orc_deriv1d.argtypes = [ctypes.c_long, ctypes.c_double, _DP, _DP]
            lib.orc_compact_deriv1d.argtypes = [ctypes.c_long, ctypes.c_double, _DP, _DP]
            lib.orc_compact_skew_deriv1d.argtypes = [ctypes.c_long, ctypes.c_double, _DP, _DP]
            lib.orc_rhs.argtypes = [P, _DP, _DP]
            lib.orc_rk4.argtypes = [P, _DP, ctypes.c_double, ctypes.c_long]
            lib.orc_insert.argtypes = [P, O, _DP, _DP]
            lib.orc_observe.argtypes = [P, O, _DP]
            lib.orc_observe.restype = ctypes.c_double
            lib.orc_boltzmann.argtypes = [P, _DP]
            lib.orc_to_density.argtypes = [P, _DP, _DP]
            lib.orc_residual.argtypes = [P, _DP]
            lib.orc_residual.restype = ctypes.c_double
            lib.orc_equilibrate.argtypes = [P, _DP, ctypes.c_double, ctypes.c_long,
                                            ctypes.c_double, ctypes.c_long, _DP]
            lib.orc_equilibrate.restype = ctypes.c_long
            lib.orc_response1.argtypes = [P, O, O, _DP, ctypes.c_double, ctypes.c_int,
                                          ctypes.c_long, _DP]
            lib.orc_response2.argtypes = [P, O, O, O, _DP, ctypes.c_double, ctypes.c_int,
                                          ctypes.c_int, ctypes.c_long, _DP]
            lib.orc_h_rhs.argtypes = [P, _DP, _DP]
            lib.orc_h_rk4.argtypes = [P, _DP, ctypes.c_double, ctypes.c_long]
            lib.orc_h_insert.argtypes = [P, O, _DP, _DP]
            lib.orc_h_observe.argtypes = [P, O, _DP]
            lib.orc_h_observe.restype = ctypes.c_double
            lib.orc_h_boltzmann.argtypes = [P, _DP]
            _lib = lib
    return _lib


def threads() -> int:
    """OpenMP threads the oracle uses (OMP_NUM_THREADS, else all cores)."""
    return int(_load().orc_threads())


def members(d: int, depth: int) -> np.ndarray:
    """Member multi-indices n (shape [M, d]) in storage order: by tier, then lexicographic."""
    lib = _load()
    M = lib.orc_member_count(d, depth)
    out = (ctypes.c_int * (3 * M))()
    lib.orc_members(d, depth, out)
    return np.array(out, dtype=np.int64).reshape(M, 3)[:, :d]


class Problem:
    """One model on one grid with one hierarchy depth, as the oracle sees it."""

    def __init__(self, model, grid, depth: int, qscheme: int = 0):
        d = int(model.nmodes)
        s = _Problem()
        s.qscheme = int(qscheme)
        s.d = d
        s.depth = int(depth)
        s.kT = float(model.kT)
        for name in ("m", "omega", "g3", "g4", "zeta", "gamma", "V_LL", "V_SL"):
            vals = list(getattr(model, name)) + [0.0] * 3
            arr = getattr(s, name)
            for i in range(3):
                arr[i] = float(vals[i])
        for name in ("g2", "g_s2s", "g_ss2"):
            mat = np.zeros((3, 3))
            src = np.asarray(getattr(model, name), dtype=np.float64)
            mat[: src.shape[0], : src.shape[1]] = src
            arr = getattr(s, name)
            for i in range(3):
                for j in range(3):
                    arr[i][j] = float(mat[i, j])
        for name in ("nq", "np"):
            vals = list(getattr(grid, name)) + [1] * 3
            arr = getattr(s, name)
            for i in range(3):
                arr[i] = int(vals[i])
        for name in ("qmin", "qmax", "pmin", "pmax"):
            vals = list(getattr(grid, name)) + [0.0] * 3
            arr = getattr(s, name)
            for i in range(3):
                arr[i] = float(vals[i])
        self._s = s
        self.d = d
        self.depth = int(depth)
        self.members = members(d, depth)
        self.M = len(self.members)
        self.shape = tuple(int(grid.nq[i]) for i in range(d)) + tuple(int(grid.np[i]) for i in range(d))
        self.P = int(np.prod(self.shape))

    @property
    def state_shape(self):
        return (self.M,) + self.shape

    def zeros(self) -> np.ndarray:
        return np.zeros(self.state_shape, dtype=np.float64)

    def _ptr(self):
        return ctypes.byref(self._s)


def _optical(X) -> _Optical:
    o = _Optical()
    lin = list(X.lin) + [0.0] * 3
    quad = np.zeros((3, 3))
    src = np.asarray(X.quad, dtype=np.float64)
    quad[: src.shape[0], : src.shape[1]] = src
    for i in range(3):
        o.lin[i] = float(lin[i])
        for j in range(3):
            o.quad[i][j] = float(quad[i, j])
    return o


def _as_state(pb: Problem, W) -> np.ndarray:
    W = np.ascontiguousarray(W, dtype=np.float64)
    if W.size != pb.M * pb.P:
        raise ValueError(f"state has {W.size} values, expected {pb.M * pb.P}")
    return W.reshape(pb.state_shape)


def _p(a: np.ndarray):
    return a.ctypes.data_as(_DP)


def deriv1d(f, h: float) -> np.ndarray:
    f = np.ascontiguousarray(f, dtype=np.float64)
    out = np.empty_like(f)
    _load().orc_deriv1d(f.size, float(h), _p(f), _p(out))
    return out


def compact_deriv1d(f, h: float) -> np.ndarray:
    """The compact sixth-order first derivative of Sec. III B (tridiagonal solve, zero values
    outside the array; constants alpha = 1/3, a = 7/9, b = 1/36)."""
    f = np.ascontiguousarray(f, dtype=np.float64)
    out = np.empty_like(f)
    _load().orc_compact_deriv1d(f.size, float(h), _p(f), _p(out))
    return out


def compact_skew_deriv1d(f, h: float) -> np.ndarray:
    """The skew-symmetric part (A^{-1} B + B A^{-1}) f / 2h of the compact derivative."""
    f = np.ascontiguousarray(f, dtype=np.float64)
    out = np.empty_like(f)
    _load().orc_compact_skew_deriv1d(f.size, float(h), _p(f), _p(out))
    return out


def potential(pb: Problem, q) -> float:
    q = np.ascontiguousarray(list(q) + [0.0] * 3, dtype=np.float64)
    return float(_load().orc_potential(pb._ptr(), _p(q)))


def dUdq(pb: Problem, q, s: int) -> float:
    q = np.ascontiguousarray(list(q) + [0.0] * 3, dtype=np.float64)
    return float(_load().orc_dUdq(pb._ptr(), _p(q), int(s)))


def rhs(pb: Problem, W) -> np.ndarray:
    W = _as_state(pb, W)
    K = np.empty_like(W)
    if _load().orc_rhs(pb._ptr(), _p(W), _p(K)):
        raise RuntimeError("orc_rhs failed")
    return K


def rk4(pb: Problem, W, dt: float, nsteps: int) -> np.ndarray:
    Y = _as_state(pb, W).copy()
    if _load().orc_rk4(pb._ptr(), _p(Y), float(dt), int(nsteps)):
        raise RuntimeError("orc_rk4 failed")
    return Y


def insert(pb: Problem, X, W) -> np.ndarray:
    W = _as_state(pb, W)
    out = np.empty_like(W)
    o = _optical(X)
    if _load().orc_insert(pb._ptr(), ctypes.byref(o), _p(W), _p(out)):
        raise RuntimeError("orc_insert failed")
    return out


def observe(pb: Problem, C, W) -> float:
    W = _as_state(pb, W)
    o = _optical(C)
    return float(_load().orc_observe(pb._ptr(), ctypes.byref(o), _p(W)))


def boltzmann(pb: Problem) -> np.ndarray:
    W = pb.zeros()
    if _load().orc_boltzmann(pb._ptr(), _p(W)):
        raise RuntimeError("orc_boltzmann failed")
    return W


def to_density(pb: Problem, G) -> np.ndarray:
    """W^(n) = lambda_n exp(-H/2kT) g^(n): the distributions of Eq. HEOM from a stored state."""
    G = _as_state(pb, G)
    W = np.empty_like(G)
    if _load().orc_to_density(pb._ptr(), _p(G), _p(W)):
        raise RuntimeError("orc_to_density failed")
    return W


def residual(pb: Problem, W) -> float:
    W = _as_state(pb, W)
    return float(_load().orc_residual(pb._ptr(), _p(W)))


def equilibrate(pb: Problem, dt: float, max_steps: int, tol: float, check_every: int = 100,
                W0=None):
    """Returns (W_eq, steps, residual).  Starts from the sampled Boltzmann unless W0 given."""
    W = boltzmann(pb) if W0 is None else _as_state(pb, W0).copy()
    r = ctypes.c_double(0.0)
    steps = _load().orc_equilibrate(pb._ptr(), _p(W), float(dt), int(max_steps), float(tol),
                                    int(check_every), ctypes.byref(r))
    if steps < 0:
        raise RuntimeError("orc_equilibrate failed")
    return W, int(steps), float(r.value)


def response1(pb: Problem, A, C, Weq, dt: float, nt: int, stride: int) -> np.ndarray:
    Weq = _as_state(pb, Weq)
    R = np.zeros(nt)
    a, c = _optical(A), _optical(C)
    if _load().orc_response1(pb._ptr(), ctypes.byref(a), ctypes.byref(c), _p(Weq), float(dt),
                             int(nt), int(stride), _p(R)):
        raise RuntimeError("orc_response1 failed")
    return R


def response2(pb: Problem, A, B, C, Weq, dt: float, nt1: int, nt2: int, stride: int) -> np.ndarray:
    Weq = _as_state(pb, Weq)
    R = np.zeros((nt1, nt2))
    a, b, c = _optical(A), _optical(B), _optical(C)
    if _load().orc_response2(pb._ptr(), ctypes.byref(a), ctypes.byref(b), ctypes.byref(c),
                             _p(Weq), float(dt), int(nt1), int(nt2), int(stride), _p(R)):
        raise RuntimeError("orc_response2 failed")
    return R


def response3(pb: Problem, A, B, C, D, Weq, dt: float, nt1: int, n2: int, nt3: int,
              stride: int) -> np.ndarray:
    """Eq. 3Dresponse at one waiting time t2 = n2 dt:
    R[a][c] = integral D G(c stride dt) C^x G(n2 dt) B^x G(a stride dt) A^x W_eq,
    a = 0..nt1-1 (t1), c = 0..nt3-1 (t3); each t1 branch propagated on its own, in the order
    the equation applies its operators (insert, rk4 and observe are the C oracle's)."""
    W = insert(pb, A, _as_state(pb, Weq))
    R = np.zeros((nt1, nt3))
    for a in range(nt1):
        X = rk4(pb, insert(pb, B, W), dt, n2)
        X = insert(pb, C, X)
        for c in range(nt3):
            R[a, c] = observe(pb, D, X)
            if c + 1 < nt3:
                X = rk4(pb, X, dt, stride)
        if a + 1 < nt1:
            W = rk4(pb, W, dt, stride)
    return R


# ------------------------------------------------------------------------------------------
# Hermite-function representation of the momenta (Sec. III A, Appendix A, Eq. HEOM2FP-H):
# states [member][q_1..q_d][k_1..k_d]; the grid's np[s] is the number K_s of Hermite functions
# ------------------------------------------------------------------------------------------

def h_rhs(pb: Problem, C) -> np.ndarray:
    C = _as_state(pb, C)
    out = np.empty_like(C)
    if _load().orc_h_rhs(pb._ptr(), _p(C), _p(out)):
        raise RuntimeError("orc_h_rhs failed")
    return out


def h_rk4(pb: Problem, C, dt: float, nsteps: int) -> np.ndarray:
    y = _as_state(pb, C).copy()
    if _load().orc_h_rk4(pb._ptr(), _p(y), float(dt), int(nsteps)):
        raise RuntimeError("orc_h_rk4 failed")
    return y


def h_insert(pb: Problem, X, C) -> np.ndarray:
    C = _as_state(pb, C)
    out = np.empty_like(C)
    x = _optical(X)
    if _load().orc_h_insert(pb._ptr(), ctypes.byref(x), _p(C), _p(out)):
        raise RuntimeError("orc_h_insert failed")
    return out


def h_observe(pb: Problem, Cop, C) -> float:
    C = _as_state(pb, C)
    x = _optical(Cop)
    return float(_load().orc_h_observe(pb._ptr(), ctypes.byref(x), _p(C)))


def h_boltzmann(pb: Problem) -> np.ndarray:
    out = pb.zeros()
    if _load().orc_h_boltzmann(pb._ptr(), _p(out)):
        raise RuntimeError("orc_h_boltzmann failed")
    return out


def h_response1(pb: Problem, A, C, Ceq, dt: float, nt: int, stride: int) -> np.ndarray:
    """Eq. 1Dresponse in the Hermite representation: insert, then observe every stride steps."""
    X = h_insert(pb, A, Ceq)
    R = np.zeros(nt)
    for k in range(nt):
        R[k] = h_observe(pb, C, X)
        if k + 1 < nt:
            X = h_rk4(pb, X, dt, stride)
    return R


def h_response2(pb: Problem, A, B, C, Ceq, dt: float, nt1: int, nt2: int, stride: int) -> np.ndarray:
    """Eq. 2Dresponse in the Hermite representation, each t1 branch propagated on its own."""
    W = h_insert(pb, A, Ceq)
    R = np.zeros((nt1, nt2))
    for i in range(nt1):
        X = h_insert(pb, B, W)
        for j in range(nt2):
            R[i, j] = h_observe(pb, C, X)
            if j + 1 < nt2:
                X = h_rk4(pb, X, dt, stride)
        if i + 1 < nt1:
            W = h_rk4(pb, W, dt, stride)
    return R
