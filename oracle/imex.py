"""IMEX Runge-Kutta tableaux and Algorithm 1 (IMEX HDG-DG) -- oracle.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

The paper uses ARS2(2,3,2) and ARS3(4,4,3) of Ascher, Ruuth and Spiteri (1997), cited in
Sec. 6 but not printed.  They are written here in the padded (s+1)-stage form of eq.
IMEXRKi, where the explicit first stage has a_11 = 0 (Algorithm 1, "if a_ii = 0").
ARS2(2,3,2): gamma = 1 - 1/sqrt(2), delta = -2 sqrt(2)/3.
ARS3(4,4,3): implicit diagonal 1/2.
Their order conditions are pinned in the tests.
"""
import math

import numpy as np

from . import swe
from .hdg import Condensed, solve_unreduced


def ars2():
    g = 1.0 - 1.0 / math.sqrt(2.0)
    d = -2.0 * math.sqrt(2.0) / 3.0
    A = np.array([[0.0, 0.0, 0.0], [g, 0.0, 0.0], [d, 1.0 - d, 0.0]])
    At = np.array([[0.0, 0.0, 0.0], [0.0, g, 0.0], [0.0, 1.0 - g, g]])
    b = np.array([0.0, 1.0 - g, g])
    return A, At, b, b.copy()


def ars3():
    A = np.array([[0, 0, 0, 0, 0],
                  [1 / 2, 0, 0, 0, 0],
                  [11 / 18, 1 / 18, 0, 0, 0],
                  [5 / 6, -5 / 6, 1 / 2, 0, 0],
                  [1 / 4, 7 / 4, 3 / 4, -7 / 4, 0]], dtype=float)
    At = np.array([[0, 0, 0, 0, 0],
                   [0, 1 / 2, 0, 0, 0],
                   [0, 1 / 6, 1 / 2, 0, 0],
                   [0, -1 / 2, 1 / 2, 1 / 2, 0],
                   [0, 3 / 2, -3 / 2, 1 / 2, 1 / 2]], dtype=float)
    return A, At, A[-1].copy(), At[-1].copy()


SCHEMES = {"ars2": ars2, "ars3": ars3}


class Stepper:
    """Algorithm 1 of the paper for a fixed mesh, bottom and dt.

    solver: 'unreduced' (dense direct solve of the coupled system every stage), or a
    ``hdg.Condensed`` solver kind ('lu', 'dense', 'gmres').  ``linear_only`` drops NL
    (the linear-wave tests).
    """

    def __init__(self, mesh, phiB, dt, scheme="ars2", solver="lu", linear_only=False, rtol=1e-14,
                 bc=None):
        """bc(t) -> prescribed boundary states [3, e, 4, P] at time t (Dirichlet meshes only)."""
        self.mesh, self.phiB, self.dt = mesh, phiB, dt
        self.bc = bc
        self.t = 0.0
        self.A, self.At, self.b, self.bt = SCHEMES[scheme]()
        self.s = len(self.b)
        self.tau_e = mesh.face_tau_hat(phiB)
        self.solver = solver
        self.linear_only = linear_only
        diag = sorted({float(a) for a in np.diag(self.At) if a != 0.0})
        if len(diag) != 1:
            raise ValueError("the stage operators are shared only for a constant implicit diagonal")
        self.a_ii = diag[0]
        self.cond = None if solver == "unreduced" else Condensed(mesh, phiB, self.tau_e, dt * self.a_ii,
                                                                 solver=solver, rtol=rtol)
        self.last = {}

    def nl(self, Q):
        if self.linear_only:
            return np.zeros_like(Q)
        return swe.NL(self.mesh, Q, self.phiB)

    def lin(self, Q, lam_g):
        return swe.L(self.mesh, Q, self.mesh.element_traces(lam_g), self.phiB, self.tau_e)

    def stage_solve(self, R1, R2=None):
        if self.cond is None:
            return solve_unreduced(self.mesh, self.phiB, self.tau_e, self.dt * self.a_ii, R1, R2)
        return self.cond.solve(R1, R2)

    def _boundary_at(self, t):
        """Set the prescribed boundary states for stage time t; returns the trace rows' R2."""
        if self.bc is None:
            return None
        self.mesh.bc_q = self.bc(t)
        return swe.dirichlet_R2(self.mesh, self.mesh.bc_q)

    def step(self, q):
        """One step q^n -> q^{n+1} of Algorithm 1 (stage i at time t + c_i dt, c = A 1)."""
        m, dt = self.mesh, self.dt
        c = self.A.sum(axis=1)
        NLs, Ls, Qs, R1s, lams = [None] * self.s, [None] * self.s, [None] * self.s, [None] * self.s, [None] * self.s
        for i in range(self.s):
            R2 = self._boundary_at(self.t + c[i] * dt)
            if self.At[i, i] == 0.0:
                Q = q
                # L(Q^(i)) is needed only if some later coefficient multiplies it.
                if np.any(self.At[i + 1:, i] != 0.0) or self.bt[i] != 0.0:
                    lam = swe.trace_from_conservation(m, Q, self.phiB, self.tau_e, R2)
                    Ls[i] = self.lin(Q, lam)
                    lams[i] = lam
            else:
                acc = np.zeros_like(q)
                for j in range(i):
                    if self.A[i, j] != 0.0:
                        acc = acc + self.A[i, j] * NLs[j]
                    if self.At[i, j] != 0.0:
                        acc = acc + self.At[i, j] * Ls[j]
                R1 = q + dt * swe.minv(m, acc)
                Q, lam = self.stage_solve(R1, R2)
                Ls[i] = self.lin(Q, lam)
                R1s[i], lams[i] = R1, lam
            Qs[i] = Q
            NLs[i] = self.nl(Q)
        acc = np.zeros_like(q)
        for i in range(self.s):
            if self.b[i] != 0.0:
                acc = acc + self.b[i] * NLs[i]
            if self.bt[i] != 0.0:
                acc = acc + self.bt[i] * Ls[i]
        self.last = {"Q": Qs, "R1": R1s, "L": Ls, "NL": NLs, "lam": lams}
        self.t += dt
        return q + dt * swe.minv(m, acc)

    def run(self, q, n_steps):
        for _ in range(n_steps):
            q = self.step(q)
        return q


# -- explicit RK DG (the comparison scheme of Sec. 7) ------------------------------------------
class ExplicitRK:
    """Explicit strong-stability-preserving Runge-Kutta on the full DG residual: 'rk2' is Heun's
    two-stage method, 'rk3' the three-stage method of Shu and Osher -- the RK2 DG / RK3 DG the
    paper compares IMEX HDG-DG against (Sec. 7.1, 7.2)."""

    def __init__(self, mesh, phiB, dt, scheme="rk2", bc=None):
        self.mesh, self.phiB, self.dt, self.scheme = mesh, phiB, dt, scheme
        self.bc = bc
        self.t = 0.0

    def rhs(self, q, t):
        if self.bc is not None:
            self.mesh.bc_q = self.bc(t)
        return swe.minv(self.mesh, swe.DG_full(self.mesh, q, self.phiB))

    def step(self, q):
        dt, t = self.dt, self.t
        self.t += dt
        if self.scheme == "rk2":
            q1 = q + dt * self.rhs(q, t)
            return 0.5 * q + 0.5 * (q1 + dt * self.rhs(q1, t + dt))
        if self.scheme == "rk3":
            q1 = q + dt * self.rhs(q, t)
            q2 = 0.75 * q + 0.25 * (q1 + dt * self.rhs(q1, t + dt))
            return q / 3.0 + 2.0 / 3.0 * (q2 + dt * self.rhs(q2, t + 0.5 * dt))
        raise ValueError(self.scheme)

    def run(self, q, n_steps):
        for _ in range(n_steps):
            q = self.step(q)
        return q


# -- diagnostics ------------------------------------------------------------------------------
def mass(mesh, q):
    """Total mass integral of phi_eta (GLL quadrature): sum_e J sum_ij w_i w_j phi_eta."""
    return float(np.sum(mesh.mass[None, :, :] * q[0]))


def energy_linear(mesh, q, phiB):
    """E_h = ||phi_eta||^2 + ||U||^2_{phi_B^-1} (semi-discrete energy of the linear part)."""
    return float(np.sum(mesh.mass[None, :, :] * (q[0] ** 2 + (q[1] ** 2 + q[2] ** 2) / phiB)))


def rel_l2(mesh, a, ref):
    """GLL-weighted relative L2 distance ||a - ref|| / ||ref|| of one nodal field [e, j, i]."""
    wgt = mesh.mass[None, :, :]
    num = np.sqrt(np.sum(wgt * (a - ref) ** 2))
    den = np.sqrt(np.sum(wgt * ref ** 2))
    return float(num / den) if den > 0 else float(num)
