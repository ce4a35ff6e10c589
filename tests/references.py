"""Independent references that pin the FP64 oracle (none of them calls the oracle).

* ``brownian_matrix`` / ``brownian_r1_continuum``: the harmonic Brownian oscillator with a Drude
  bath and linear-linear coupling.  Its first moments (<q>_0, <p>_0, integral of W^(1)) close
  exactly under the hierarchy of Eq. HEOM, so R1 of Eq. 1Dresponse with mu = q is a 3x3 matrix
  exponential; the continuum form is a sum over the roots of
  s^3 + gamma s^2 + (omega^2 + zeta gamma V_LL^2) s + gamma omega^2.
* ``MomentClosure``: the same idea for d modes, bilinear mode coupling and linear/quadratic
  optical operators: polynomial observables of bounded (tier + degree) form an invariant space
  of the adjoint hierarchy generator, obtained by integrating Eq. HEOM by parts; responses of
  Eqs. 1Dresponse / 2Dresponse then follow from small matrix powers.  Time stepping is mirrored
  exactly with the RK4 stability polynomial.
* ``trajectory_r1``: zeta = 0 makes the bath drop out, so R1 is a classical-trajectory average
  (Gauss quadrature over the Boltzmann weight, ODE integration of Hamilton's equations).
* ``boltzmann_grid``: exp(-H/kT) on grid nodes, normalised, written from Eqs. "sec: System
  Hamiltonian", "sec: Potenentials" (+ quartic) and "sec: Potential ss'"; ``boltzmann_sym`` is
  the same in the symmetrised variable g = W exp(H/2kT) that stored states hold.
"""
from __future__ import annotations

import itertools
import math

import numpy as np
import scipy.integrate


# ------------------------------------------------------------------------------------------
# RK4
# ------------------------------------------------------------------------------------------

def rk4_poly(Z: np.ndarray) -> np.ndarray:
    """Stability polynomial of classical RK4: 1 + Z + Z^2/2 + Z^3/6 + Z^4/24."""
    I = np.eye(Z.shape[0])
    Z2 = Z @ Z
    Z3 = Z2 @ Z
    return I + Z + Z2 / 2.0 + Z3 / 6.0 + Z3 @ Z / 24.0


# ------------------------------------------------------------------------------------------
# potential and Boltzmann distribution (test's own restatement of Sec. II A)
# ------------------------------------------------------------------------------------------

def potential(model, q):
    d = model.nmodes
    U = 0.0
    for s in range(d):
        U = U + 0.5 * model.m[s] * model.omega[s] ** 2 * q[s] ** 2 + model.g3[s] * q[s] ** 3 / 6.0 \
            + model.g4[s] * q[s] ** 4 / 24.0
    for a in range(d):
        for b in range(a + 1, d):
            U = U + model.g2[a, b] * q[a] * q[b] + (model.g_s2s[a, b] * q[a] ** 2 * q[b]
                                                     + model.g_ss2[a, b] * q[a] * q[b] ** 2) / 6.0
    return U


def grid_axes(grid):
    d = grid.d
    return ([np.linspace(grid.qmin[s], grid.qmax[s], grid.nq[s]) for s in range(d)]
            + [np.linspace(grid.pmin[s], grid.pmax[s], grid.np[s]) for s in range(d)])


def cell_volume(grid):
    return float(np.prod([(a[-1] - a[0]) / (len(a) - 1) for a in grid_axes(grid)]))


def boltzmann_grid(model, grid) -> np.ndarray:
    d = model.nmodes
    mesh = np.meshgrid(*grid_axes(grid), indexing="ij")
    H = potential(model, mesh[:d])
    for s in range(d):
        H = H + mesh[d + s] ** 2 / (2.0 * model.m[s])
    W = np.exp(-(H - H.min()) / model.kT)
    return W / (W.sum() * cell_volume(grid))


def sym_weight(model, grid) -> np.ndarray:
    """exp(-H/2kT) on the grid nodes: W^(0) = sym_weight * g^(0)."""
    d = model.nmodes
    mesh = np.meshgrid(*grid_axes(grid), indexing="ij")
    H = potential(model, mesh[:d])
    for s in range(d):
        H = H + mesh[d + s] ** 2 / (2.0 * model.m[s])
    return np.exp(-H / (2.0 * model.kT))


def boltzmann_sym(model, grid) -> np.ndarray:
    """The normalised Boltzmann distribution in the symmetrised variable g = W exp(H/2kT)."""
    return boltzmann_grid(model, grid) / sym_weight(model, grid)


def hierarchy_state(W0: np.ndarray, nmembers: int) -> np.ndarray:
    out = np.zeros((nmembers,) + W0.shape)
    out[0] = W0
    return out


# ------------------------------------------------------------------------------------------
# single harmonic Brownian oscillator, LL coupling
# ------------------------------------------------------------------------------------------

def brownian_matrix(m, omega, zeta, gamma, V):
    """d/dt (<q>_0, <p>_0, int W^(1)) for the harmonic mode with V(q) = V q."""
    return np.array([[0.0, 1.0 / m, 0.0],
                     [-m * omega ** 2, 0.0, -V],
                     [0.0, zeta * gamma * V, -gamma]])


def g_discrete(Amat, dt, nsteps_list):
    """[R4(dt A)^k]_{01} for each k."""
    P = rk4_poly(dt * Amat)
    out = []
    cur = np.eye(3)
    done = 0
    for k in nsteps_list:
        while done < k:
            cur = P @ cur
            done += 1
        out.append(cur[0, 1])
    return np.array(out)


def brownian_r1_continuum(m, omega, zeta, gamma, V, t):
    """-[exp(A t)]_{01} = -(1/m) sum_r (r + gamma) e^{r t} / P'(r)."""
    coeffs = [1.0, gamma, omega ** 2 + zeta * gamma * V ** 2, gamma * omega ** 2]
    roots = np.roots(coeffs)
    dP = np.polyder(np.poly1d(coeffs))
    t = np.asarray(t, dtype=np.float64)
    g = sum((r + gamma) * np.exp(r * t) / dP(r) for r in roots) / m
    return -np.real(g)


# ------------------------------------------------------------------------------------------
# moment closure (adjoint of Eq. HEOM on polynomial observables)
# ------------------------------------------------------------------------------------------

class MomentClosure:
    """Exact response functions for harmonic modes with bilinear coupling g2 and LL bath
    coupling (V_SL = 0, g3 = g4 = g_s2s = g_ss2 = 0), any depth, any linear/quadratic optics.

    An observable is f = (f_n(q,p))_n, acting as <f, W> = sum_n integral f_n W^(n).  Integrating
    the right-hand side of Eq. HEOM by parts gives the adjoint generator
      (M'f)_k = -sum_s F_s d f_k/dp_s + sum_s (p_s/m_s) d f_k/dq_s - (sum_s k_s gamma_s) f_k
                - sum_s V_s' d f_{k-e_s}/dp_s
                + sum_s (k_s+1) zeta_s gamma_s V_s' (p_s f_{k+e_s} - m_s kT d f_{k+e_s}/dp_s)
    and for an insertion X^x:  ((X^x)'f)_k = -sum_s dX/dq_s d f_k/dp_s.
    Observables with tier |k| + polynomial degree <= K stay in that space.
    """

    def __init__(self, model, depth: int, K: int = 2):
        d = model.nmodes
        for name in ("g3", "g4", "V_SL"):
            assert all(abs(x) == 0.0 for x in getattr(model, name)[:d]), name
        assert not np.any(model.g_s2s[:d, :d]) and not np.any(model.g_ss2[:d, :d])
        self.model, self.d, self.depth, self.K = model, d, depth, K
        self.members = [n for t in range(depth + 1) for n in self._tier(d, t)]
        self.mindex = {n: i for i, n in enumerate(self.members)}
        self.basis = []
        for k in self.members:
            t = sum(k)
            if t > K:
                continue
            for e in itertools.product(range(K - t + 1), repeat=2 * d):
                if sum(e) <= K - t:
                    self.basis.append((k, e))
        self.index = {b: i for i, b in enumerate(self.basis)}
        self.M = self._generator()

    @staticmethod
    def _tier(d, t):
        return [n for n in itertools.product(range(t + 1), repeat=d) if sum(n) == t]

    def _add(self, vec, k, e, c):
        key = (k, tuple(e))
        if c != 0.0 and key in self.index:
            vec[self.index[key]] += c
        elif c != 0.0 and k in self.mindex and sum(k) + sum(e) <= self.K:
            raise AssertionError("closure broken")

    def _force_coeffs(self, s):
        """F_s = sum_b c_b q_b (harmonic + bilinear coupling)."""
        md = self.model
        c = np.zeros(self.d)
        c[s] = md.m[s] * md.omega[s] ** 2
        for b in range(self.d):
            if b > s:
                c[b] += md.g2[s, b]
            elif b < s:
                c[b] += md.g2[b, s]
        return c

    def _generator(self):
        md, d = self.model, self.d
        nb = len(self.basis)
        M = np.zeros((nb, nb))
        for j, (k, e) in enumerate(self.basis):
            col = np.zeros(nb)
            e = list(e)
            # Liouvillian and damping on member k
            for s in range(d):
                ip = d + s
                if e[ip] > 0:                      # -F_s d/dp_s
                    fc = self._force_coeffs(s)
                    for b in range(d):
                        if fc[b] != 0.0:
                            e2 = e.copy(); e2[ip] -= 1; e2[b] += 1
                            self._add(col, k, e2, -fc[b] * e[ip])
                if e[s] > 0:                       # (p_s/m_s) d/dq_s
                    e2 = e.copy(); e2[s] -= 1; e2[ip] += 1
                    self._add(col, k, e2, e[s] / md.m[s])
            damp = sum(k[s] * md.gamma[s] for s in range(d))
            self._add(col, k, e, -damp)
            for s in range(d):
                ip = d + s
                Vp = md.V_LL[s]
                # to member k + e_s:  -V' d/dp_s f_k
                up = tuple(k[r] + (1 if r == s else 0) for r in range(d))
                if up in self.mindex and e[ip] > 0:
                    e2 = e.copy(); e2[ip] -= 1
                    self._add(col, up, e2, -Vp * e[ip])
                # to member k - e_s:  k_s zeta gamma V' (p_s f_k - m kT d f_k/dp_s)
                if k[s] >= 1:
                    dn = tuple(k[r] - (1 if r == s else 0) for r in range(d))
                    zg = md.zeta[s] * md.gamma[s] * k[s] * Vp
                    e2 = e.copy(); e2[ip] += 1
                    self._add(col, dn, e2, zg)
                    if e[ip] > 0:
                        e3 = e.copy(); e3[ip] -= 1
                        self._add(col, dn, e3, -zg * md.m[s] * md.kT * e[ip])
            M[:, j] = col
        return M

    def insertion(self, X):
        """Matrix of (X^x)' on the basis."""
        d = self.d
        nb = len(self.basis)
        T = np.zeros((nb, nb))
        Q = 0.5 * (np.asarray(X.quad)[:d, :d] + np.asarray(X.quad)[:d, :d].T)
        for j, (k, e) in enumerate(self.basis):
            col = np.zeros(nb)
            e = list(e)
            for s in range(d):
                ip = d + s
                if e[ip] == 0:
                    continue
                e2 = e.copy(); e2[ip] -= 1
                self._add(col, k, e2, -X.lin[s] * e[ip])
                for b in range(d):
                    if Q[s, b] != 0.0:
                        e3 = e2.copy(); e3[b] += 1
                        self._add(col, k, e3, -Q[s, b] * e[ip])
            T[:, j] = col
        return T

    def observable(self, X):
        """Coefficient vector of X(q) placed on member 0."""
        d = self.d
        v = np.zeros(len(self.basis))
        k0 = tuple([0] * d)
        for s in range(d):
            e = [0] * (2 * d); e[s] = 1
            self._add(v, k0, e, X.lin[s])
        for a in range(d):
            for b in range(d):
                e = [0] * (2 * d); e[a] += 1; e[b] += 1
                self._add(v, k0, e, 0.5 * X.quad[a][b])
        return v

    def equilibrium_moments(self, W0: np.ndarray, grid) -> np.ndarray:
        """<basis_i, W_eq> for W_eq = (W0, 0, 0, ...), sums over the grid nodes."""
        mesh = np.meshgrid(*grid_axes(grid), indexing="ij")
        vol = cell_volume(grid)
        k0 = tuple([0] * self.d)
        out = np.zeros(len(self.basis))
        for i, (k, e) in enumerate(self.basis):
            if k != k0:
                continue
            f = np.ones_like(W0)
            for a, ea in enumerate(e):
                if ea:
                    f = f * mesh[a] ** ea
            out[i] = vol * np.sum(f * W0)
        return out

    def response1(self, A, C, W0, grid, dt, nt, stride):
        P = np.linalg.matrix_power(rk4_poly(dt * self.M), stride)
        Ax = self.insertion(A)
        meq = self.equilibrium_moments(W0, grid)
        f = self.observable(C)
        out = []
        for _ in range(nt):
            out.append(meq @ (Ax @ f))
            f = P @ f
        return np.array(out)

    def response2(self, A, B, C, W0, grid, dt, nt1, nt2, stride):
        P = np.linalg.matrix_power(rk4_poly(dt * self.M), stride)
        Ax, Bx = self.insertion(A), self.insertion(B)
        meq = self.equilibrium_moments(W0, grid)
        row = meq @ Ax                       # functional applied after the t1 propagation
        rows = []
        for _ in range(nt1):
            rows.append(row)
            row = row @ P
        f = self.observable(C)
        R = np.zeros((nt1, nt2))
        for j in range(nt2):
            h = Bx @ f
            for i in range(nt1):
                R[i, j] = rows[i] @ h
            f = P @ f
        return R


    def response3(self, A, B, C, D, W0, grid, dt, nt1, n2, nt3, stride):
        """Eq. 3Dresponse at one waiting time n2 dt: R[a][c] with t1 = a stride dt and
        t3 = c stride dt, from the adjoint chain D <- (C^x)' <- G(n2) <- (B^x)' <- G(t1) <- (A^x)'."""
        P = np.linalg.matrix_power(rk4_poly(dt * self.M), stride)
        P2 = np.linalg.matrix_power(rk4_poly(dt * self.M), n2)
        Ax, Bx, Cx = self.insertion(A), self.insertion(B), self.insertion(C)
        meq = self.equilibrium_moments(W0, grid)
        row = meq @ Ax
        rows = []
        for _ in range(nt1):
            rows.append(row)
            row = row @ P
        f = self.observable(D)
        R = np.zeros((nt1, nt3))
        for c in range(nt3):
            h = Bx @ (P2 @ (Cx @ f))
            for a in range(nt1):
                R[a, c] = rows[a] @ h
            f = P @ f
        return R


# ------------------------------------------------------------------------------------------
# classical trajectories (zeta = 0)
# ------------------------------------------------------------------------------------------

def exact_force(model, q):
    """dU/dq for one mode, differentiated by hand from the test's own potential above."""
    m, w = model.m[0], model.omega[0]
    return m * w * w * q + model.g3[0] * q * q / 2.0 + model.g4[0] * q ** 3 / 6.0


def trajectory_r1(model, mu_lin, times, nq=60, npq=40, rtol=1e-12, atol=1e-13):
    """R1(t) = integral mu(q(t)) mu^x W_B = -(1/kT) integral mu(q_t(x)) (mu' p/m) W_B dx
    for a single mode (d = 1) with zeta = 0, by quadrature and trajectory integration.
    q-quadrature: Gauss-Legendre on +-9 sigma with the Boltzmann weight; p: Gauss-Hermite."""
    assert model.nmodes == 1
    m, kT = model.m[0], model.kT
    U = lambda q: potential(model, [q])
    L = 9.0 * math.sqrt(kT / (m * model.omega[0] ** 2))
    xq, wq = np.polynomial.legendre.leggauss(nq)
    qs = L * xq
    Uq = np.array([U(q) for q in qs])
    wqs = L * wq * np.exp(-(Uq - Uq.min()) / kT)
    xp, wp = np.polynomial.hermite.hermgauss(npq)   # weight exp(-x^2): p = sqrt(2 m kT) x
    ps = math.sqrt(2.0 * m * kT) * xp
    Z = wqs.sum() * wp.sum() * math.sqrt(2.0 * m * kT)
    times = np.asarray(times)
    R = np.zeros_like(times, dtype=np.float64)

    def rhs(t, y):
        q, p = y
        return [p / m, -exact_force(model, q)]

    for i, q0 in enumerate(qs):
        for j, p0 in enumerate(ps):
            sol = scipy.integrate.solve_ivp(rhs, (0.0, times[-1]), [q0, p0], t_eval=times,
                                            method="DOP853", rtol=rtol, atol=atol)
            qt = sol.y[0]
            weight = wqs[i] * wp[j] * math.sqrt(2.0 * m * kT) / Z
            R += weight * (mu_lin * qt) * (-(mu_lin * p0 / m) / kT)
    return R
