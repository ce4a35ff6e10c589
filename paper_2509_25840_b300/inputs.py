"""Seeded, synthetic inputs for the CHFPE hot path.

Plain parameter containers (model, grid, optical operator), a counter-based random generator
(SplitMix64) and the named workloads the tests and the benchmark run.  This module holds no
arithmetic of the method itself: no potential derivatives, no finite differences, no hierarchy
couplings.  It is the one module that both the CUDA path's callers and the FP64 oracle's callers
import.

Workloads (dimensionless units, omega, m and kT as given):
  one_mode_64      1 harmonic mode, 64x64 on [-6,6]^2, Drude zeta=0.2, gamma=1, kT=1,
                   linear-linear coupling only, depth 5, dt=0.005, mu = q, R1 over 2000 steps
  two_mode_32      2 coupled anharmonic modes on a 32^4 grid, g4 = (0.01, 0.05), a cubic mode
                   coupling whose q1 q2^2 coefficient is 0.02, LL + SL (V_SL/V_LL = 0.3), depth 4
                   (15 members), dt=0.005, R2 on 64x64 (t1, t2) with dtau = 0.2
  three_mode_20    3 water-like intermolecular modes, omega = (0.5, 1.0, 1.6), 20^6 grid, depth 2
                   (10 members), dt=0.002, TRT R2 on 128x128 with dtau = 0.1
  sweep            256 two-mode instances with seeded uniform parameters, grids 24..48 per axis
"""
from __future__ import annotations

import dataclasses
import math
from typing import Sequence

import numpy as np

MASK64 = (1 << 64) - 1


# ------------------------------------------------------------------------------------------
# containers
# ------------------------------------------------------------------------------------------

@dataclasses.dataclass
class Model:
    """System and bath parameters (Sec. II A).  Pair terms are read for s < s' only."""
    nmodes: int
    kT: float = 1.0
    m: Sequence[float] = (1.0, 1.0, 1.0)
    omega: Sequence[float] = (1.0, 1.0, 1.0)
    g3: Sequence[float] = (0.0, 0.0, 0.0)
    g4: Sequence[float] = (0.0, 0.0, 0.0)
    g2: np.ndarray = dataclasses.field(default_factory=lambda: np.zeros((3, 3)))
    g_s2s: np.ndarray = dataclasses.field(default_factory=lambda: np.zeros((3, 3)))
    g_ss2: np.ndarray = dataclasses.field(default_factory=lambda: np.zeros((3, 3)))
    zeta: Sequence[float] = (0.0, 0.0, 0.0)
    gamma: Sequence[float] = (1.0, 1.0, 1.0)
    V_LL: Sequence[float] = (1.0, 1.0, 1.0)
    V_SL: Sequence[float] = (0.0, 0.0, 0.0)

    def __post_init__(self):
        for name in ("m", "omega", "g3", "g4", "zeta", "gamma", "V_LL", "V_SL"):
            v = list(getattr(self, name)) + [0.0] * 3
            setattr(self, name, tuple(float(x) for x in v[:3]))
        for name in ("g2", "g_s2s", "g_ss2"):
            a = np.zeros((3, 3))
            src = np.asarray(getattr(self, name), dtype=np.float64)
            a[: src.shape[0], : src.shape[1]] = src
            setattr(self, name, a)

    def replace(self, **kw) -> "Model":
        return dataclasses.replace(self, **kw)


@dataclasses.dataclass
class Grid:
    """Uniform grid per axis, both end points included."""
    nq: Sequence[int]
    np: Sequence[int]
    qmin: Sequence[float]
    qmax: Sequence[float]
    pmin: Sequence[float]
    pmax: Sequence[float]

    def __post_init__(self):
        for name in ("nq", "np"):
            setattr(self, name, tuple(int(x) for x in getattr(self, name)))
        for name in ("qmin", "qmax", "pmin", "pmax"):
            setattr(self, name, tuple(float(x) for x in getattr(self, name)))

    @property
    def d(self) -> int:
        return len(self.nq)

    @property
    def shape(self):
        return tuple(self.nq) + tuple(self.np)

    @property
    def points(self) -> int:
        return int(np.prod(self.shape))


@dataclasses.dataclass
class Optical:
    """X(q) = sum_s lin_s q_s + 1/2 sum_{s,s'} quad_ss' q_s q_s'  (Eqs. NLdip / NLpol)."""
    lin: Sequence[float]
    quad: np.ndarray = dataclasses.field(default_factory=lambda: np.zeros((3, 3)))

    def __post_init__(self):
        v = list(self.lin) + [0.0] * 3
        self.lin = tuple(float(x) for x in v[:3])
        a = np.zeros((3, 3))
        src = np.asarray(self.quad, dtype=np.float64)
        a[: src.shape[0], : src.shape[1]] = src
        self.quad = a


@dataclasses.dataclass
class Workload:
    name: str
    model: Model
    grid: Grid
    depth: int
    dt: float
    stride: int          # RK4 steps between two time samples
    nt1: int             # samples along t1 (R1 length, or R2 rows)
    nt2: int             # samples along t2 (0 for a linear response)
    A: Optical
    B: Optical
    C: Optical

    @property
    def members(self) -> int:
        return member_count(self.grid.d, self.depth)

    @property
    def cells(self) -> int:
        return self.members * self.grid.points

    def r2_state_steps(self) -> int:
        """RK4 steps of one state summed over the t1 chain and all t2 branches."""
        return (self.nt1 - 1) * self.stride + self.nt1 * (self.nt2 - 1) * self.stride


def member_count(d: int, depth: int) -> int:
    """Members n in N^d with n_1+..+n_d <= depth: C(depth+d, d)."""
    return math.comb(depth + d, d)


# ------------------------------------------------------------------------------------------
# SplitMix64 (Steele, Lea & Flood 2014): counter-based, x_k = mix(seed + k * golden)
# ------------------------------------------------------------------------------------------

def splitmix64(seed: int, counter: int) -> int:
    z = (seed + (counter + 1) * 0x9E3779B97F4A7C15) & MASK64
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK64
    return z ^ (z >> 31)


def uniform(seed: int, counter: int, lo: float = 0.0, hi: float = 1.0) -> float:
    """Uniform double in [lo, hi) from the top 53 bits of draw number `counter`."""
    u = (splitmix64(seed, counter) >> 11) * (1.0 / (1 << 53))
    return lo + (hi - lo) * u


def uniform_array(seed: int, n: int, lo: float = -1.0, hi: float = 1.0) -> np.ndarray:
    """n uniform doubles, vectorised SplitMix64 (identical to `uniform` element by element)."""
    k = np.arange(1, n + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(seed & MASK64) + k * np.uint64(0x9E3779B97F4A7C15)
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        z = z ^ (z >> np.uint64(31))
    u = (z >> np.uint64(11)).astype(np.float64) * (1.0 / (1 << 53))
    return lo + (hi - lo) * u


# ------------------------------------------------------------------------------------------
# grid domains
# ------------------------------------------------------------------------------------------

def _single_mode_energy(m: float, omega: float, g3: float, g4: float, q: float) -> float:
    return 0.5 * m * omega * omega * q * q + g3 * q ** 3 / 6.0 + g4 * q ** 4 / 24.0


def q_extent(m: float, omega: float, g3: float, g4: float, kT: float, cut: float = 18.0) -> float:
    """Half-width L with min(U_s(L), U_s(-L)) = cut * kT (bisection); the grid is [-L, L]."""
    target = cut * kT

    def lowest(L):
        return min(_single_mode_energy(m, omega, g3, g4, L), _single_mode_energy(m, omega, g3, g4, -L))

    hi = math.sqrt(2.0 * target / (m * omega * omega))
    lo = 0.0
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if lowest(mid) < target:
            lo = mid
        else:
            hi = mid
    return 0.5 * (lo + hi)


def p_extent(m: float, kT: float, nsigma: float = 6.0) -> float:
    return nsigma * math.sqrt(m * kT)


def default_grid(model: Model, n: Sequence[int], nsigma: float = 6.0, cut: float = 18.0) -> Grid:
    """q_s in [-L_s, L_s] with U_s(+-L_s) >= cut kT; p_s in +-nsigma sqrt(m_s kT)."""
    d = model.nmodes
    n = list(n)
    if len(n) == 1:
        n = n * (2 * d)
    elif len(n) == d:
        n = n + n
    L = [q_extent(model.m[s], model.omega[s], model.g3[s], model.g4[s], model.kT, cut) for s in range(d)]
    Pm = [p_extent(model.m[s], model.kT, nsigma) for s in range(d)]
    return Grid(nq=n[:d], np=n[d:], qmin=[-x for x in L], qmax=L, pmin=[-x for x in Pm], pmax=Pm)


# ------------------------------------------------------------------------------------------
# named workloads
# ------------------------------------------------------------------------------------------

def one_mode_64(nt: int = 2001, stride: int = 1, n: int = 64) -> Workload:
    model = Model(nmodes=1, kT=1.0, m=(1.0,), omega=(1.0,), zeta=(0.2,), gamma=(1.0,),
                  V_LL=(1.0,), V_SL=(0.0,))
    grid = Grid(nq=(n,), np=(n,), qmin=(-6.0,), qmax=(6.0,), pmin=(-6.0,), pmax=(6.0,))
    mu = Optical(lin=(1.0,))
    return Workload("one_mode_64", model, grid, depth=5, dt=0.005, stride=stride, nt1=nt, nt2=0,
                    A=mu, B=mu, C=mu)


def two_mode_model() -> Model:
    g_ss2 = np.zeros((3, 3))
    g_ss2[0, 1] = 0.12          # (1/6) g_{12^2} q1 q2^2 with coefficient 0.02
    return Model(nmodes=2, kT=1.0, m=(1.0, 1.0), omega=(1.0, 1.0), g4=(0.01, 0.05),
                 g_ss2=g_ss2, zeta=(0.2, 0.2), gamma=(1.0, 1.0), V_LL=(1.0, 1.0),
                 V_SL=(0.3, 0.3))


def two_mode_32(n: int = 32, nt: int = 64, stride: int = 40) -> Workload:
    model = two_mode_model()
    grid = default_grid(model, [n])
    mu = Optical(lin=(1.0, 1.0))
    return Workload("two_mode_32", model, grid, depth=4, dt=0.005, stride=stride, nt1=nt, nt2=nt,
                    A=mu, B=mu, C=mu)


def three_mode_model() -> Model:
    g_s2s = np.zeros((3, 3))
    g_ss2 = np.zeros((3, 3))
    for a in range(3):
        for b in range(a + 1, 3):
            g_s2s[a, b] = 0.12      # q_a^2 q_b / 6 and q_a q_b^2 / 6 with coefficient 0.02
            g_ss2[a, b] = 0.12
    return Model(nmodes=3, kT=1.0, m=(1.0, 1.0, 1.0), omega=(0.5, 1.0, 1.6),
                 g4=(0.02, 0.02, 0.02), g_s2s=g_s2s, g_ss2=g_ss2, zeta=(0.2, 0.2, 0.2),
                 gamma=(0.5, 1.0, 1.5), V_LL=(1.0, 1.0, 1.0), V_SL=(0.3, 0.3, 0.3))


def three_mode_optics():
    mu_q = np.zeros((3, 3))
    pi_q = np.zeros((3, 3))
    for (a, b), v in {(0, 1): 0.02, (0, 2): 0.02, (1, 2): -0.05}.items():
        mu_q[a, b] = mu_q[b, a] = v
    for (a, b), v in {(0, 1): 0.01, (0, 2): 0.01, (1, 2): 0.04}.items():
        pi_q[a, b] = pi_q[b, a] = v
    pi_q[0, 0] = -1.0
    mu = Optical(lin=(2.0, 4.0, 1.5), quad=mu_q)
    Pi = Optical(lin=(2.0, 6.3, 2.5), quad=pi_q)
    return mu, Pi


def three_mode_20(n: int = 20, nt: int = 128, stride: int = 50) -> Workload:
    model = three_mode_model()
    grid = default_grid(model, [n])
    mu, Pi = three_mode_optics()
    return Workload("three_mode_20", model, grid, depth=2, dt=0.002, stride=stride, nt1=nt, nt2=nt,
                    A=mu, B=Pi, C=mu)


def sweep_instance(seed: int, nmin: int = 24, nmax: int = 48) -> Workload:
    """Seeded two-mode instance of the parameter sweep (uniform draws, SplitMix64)."""
    u = lambda k, lo, hi: uniform(seed, k, lo, hi)
    omega = (u(0, 0.5, 2.0), u(1, 0.5, 2.0))
    g4 = (u(2, 0.0, 0.05), u(3, 0.0, 0.05))
    zeta = (u(4, 0.05, 1.0), u(5, 0.05, 1.0))
    gamma = (u(6, 0.5, 3.0), u(7, 0.5, 3.0))
    kT = u(8, 0.5, 2.0)
    g_ss2 = np.zeros((3, 3))
    g_ss2[0, 1] = u(9, 0.0, 0.3)
    ratio = u(10, 0.0, 0.5)
    model = Model(nmodes=2, kT=kT, m=(1.0, 1.0), omega=omega, g4=g4, g_ss2=g_ss2, zeta=zeta,
                  gamma=gamma, V_LL=(1.0, 1.0), V_SL=(ratio, ratio))
    n = [nmin + int(u(11 + a, 0.0, 1.0) * (nmax - nmin + 1)) for a in range(4)]
    grid = default_grid(model, n)
    mu = Optical(lin=(1.0, 1.0))
    return Workload(f"sweep_{seed}", model, grid, depth=4, dt=0.005, stride=40, nt1=64, nt2=64,
                    A=mu, B=mu, C=mu)


# ------------------------------------------------------------------------------------------
# seeded states for operator-level parity
# ------------------------------------------------------------------------------------------

def random_state(grid: Grid, nmembers: int, seed: int, smooth: bool = True) -> np.ndarray:
    """A seeded state [member][q...][p...]: a Gaussian envelope times uniform noise in [-1, 1]
    (smooth=True multiplies in a slowly varying random quadratic instead of raw noise)."""
    d = grid.d
    axes = [np.linspace(grid.qmin[s], grid.qmax[s], grid.nq[s]) for s in range(d)]
    axes += [np.linspace(grid.pmin[s], grid.pmax[s], grid.np[s]) for s in range(d)]
    mesh = np.meshgrid(*axes, indexing="ij")
    out = np.empty((nmembers,) + grid.shape)
    for i in range(nmembers):
        env = np.ones(grid.shape)
        for a, X in enumerate(mesh):
            w = 0.25 * (axes[a][-1] - axes[a][0])
            env = env * np.exp(-0.5 * (X / w) ** 2)
        if smooth:
            c = uniform_array(seed * 1000003 + i, 2 * len(mesh) + 1)
            poly = c[0] + sum(c[1 + 2 * a] * X / axes[a][-1] + c[2 + 2 * a] * (X / axes[a][-1]) ** 2
                              for a, X in enumerate(mesh))
            out[i] = env * poly
        else:
            out[i] = env * uniform_array(seed * 1000003 + i, grid.points).reshape(grid.shape)
    return out


# ------------------------------------------------------------------------------------------
# the surrogate's parameter space: the sweep's uniform ranges, 12 parameters per instance
# ------------------------------------------------------------------------------------------

SURROGATE_NAMES = ("omega_1", "omega_2", "g4_1", "g4_2", "zeta_1", "zeta_2", "gamma_1",
                   "gamma_2", "kT", "g_12^2", "V_SL/V_LL_1", "V_SL/V_LL_2")
SURROGATE_LO = np.array([0.5, 0.5, 0.0, 0.0, 0.05, 0.05, 0.5, 0.5, 0.5, 0.0, 0.0, 0.0])
SURROGATE_HI = np.array([2.0, 2.0, 0.05, 0.05, 1.0, 1.0, 3.0, 3.0, 2.0, 0.3, 0.5, 0.5])


def surrogate_params(seed: int) -> np.ndarray:
    """Seeded draw of the 12 parameters, each uniform in its range (SplitMix64 stream `seed`)."""
    u = uniform_array(seed * 7919 + 17, 12, 0.0, 1.0)
    return SURROGATE_LO + u * (SURROGATE_HI - SURROGATE_LO)


def surrogate_model(x) -> Model:
    """The two-mode model of a 12-parameter vector (m = 1, V_LL = 1, the other couplings 0)."""
    x = [float(v) for v in x]
    g_ss2 = np.zeros((3, 3))
    g_ss2[0, 1] = x[9]
    return Model(nmodes=2, kT=x[8], m=(1.0, 1.0), omega=(x[0], x[1]), g4=(x[2], x[3]),
                 g_ss2=g_ss2, zeta=(x[4], x[5]), gamma=(x[6], x[7]), V_LL=(1.0, 1.0),
                 V_SL=(x[10], x[11]))
