"""Planar shallow water on a periodic quad mesh: fluxes and DG / HDG residuals -- oracle.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).  Literal FP64 restatement of the
paper's Sec. 3.1 and Sec. 4:

* state q = (phi_eta, U, V) with phi = phi_eta + phi_B, phi_B = g B (eq. psweGov);
* full flux F (eq. psweFluxTensor), linear flux F_L (eq. psweLinearFluxTensor),
  source s = (0, phi_eta d_x phi_B, phi_eta d_y phi_B), F_NL = F - F_L;
* NL(q)     = (F_NL, grad v) - <F*_NL . n, v>  with F*_NL = F* - F_L*, the Rusanov
  fluxes of eq. Full_russanov / Linear_russanov (Sec. 4.3);
* L(q, qh)  = (F_L, grad v) + (s, v) - <Fhat_L . n, v>, Fhat_L of eq. linear_hdgflux3
  with tau_hat = tau_L* = max(sqrt(phi_B^+), sqrt(phi_B^-));
* Flx(q, qh) = <[[Fhat_L . n]], mu> on the skeleton (eq. HDGcont).

Readings where the paper is silent (all listed in the design notes):
* quadrature: collocated tensor-product GLL, k+1 points per direction, so the mass
  matrix is J w_i w_j per node and face integrals use the k+1 face nodes;
* jump: [[q (x) n]] = q^- (x) n^- + q^+ (x) n^+ (the printed "[[v]] := 2{v}" is garbled);
* grad phi_B: nodal derivative of the nodal phi_B;
* trace space: nodal P^k on each edge at the GLL points, i.e. the element face nodes.

Mesh conventions (periodic unit square by default; see ``Mesh`` for walls): N x N
elements, element e = ey*N + ex, node (i, j) with
i along x fastest at GLL points xi_i: x = (ex + (1 + xi_i)/2)/N.  Local faces
0 = x-minus (left), 1 = x-plus (right), 2 = y-minus (bottom), 3 = y-plus (top).  Edge r < N^2
is the right face of element r; edge N^2 + r is the top face of element r.  Arrays of
nodal fields are [field c][element e][j][i].
"""
import numpy as np

from .gll import gll_nodes_weights, lagrange_derivative_matrix

FACE_NORMALS = np.array([[-1.0, 0.0], [1.0, 0.0], [0.0, -1.0], [0.0, 1.0]])
OPPOSITE_FACE = np.array([1, 0, 3, 2])


class Mesh:
    """Uniform N x N quadrilateral mesh of [x0, x0+L]^2 with degree-k GLL nodes.

    boundary='periodic' (default): the unit-square torus; edge r < N^2 is the right face of
    element r and edge N^2 + r its top face.  boundary='wall': reflecting walls on the four
    sides (Sec. 4.3, eq. reflection); x-edges are numbered ey*(N+1) + ix (ix = 0..N) and
    y-edges N(N+1) + iy*N + ex (iy = 0..N); a face on the wall has no neighbour (-1) and sees
    the mirror state of its own element instead.  boundary='dirichlet': the same numbering,
    and a boundary face sees a prescribed state (``bc_q``, set by the caller for the current
    time) while its trace equals that state (the exact-solution boundary conditions of the
    paper's moving-vortex test, Sec. 7.1).
    """

    def __init__(self, N, k, boundary="periodic", x0=0.0, length=1.0):
        if boundary == "periodic" and N < 2:
            raise ValueError("periodic mesh needs N >= 2")
        if boundary not in ("periodic", "wall", "dirichlet"):
            raise ValueError(boundary)
        self.bc_q = None
        self.N, self.k, self.P = N, k, k + 1
        self.boundary = boundary
        self.n_el = N * N
        self.h = length / N
        self.xi, self.w = gll_nodes_weights(k)
        self.D = lagrange_derivative_matrix(self.xi)
        self.J = (self.h / 2.0) ** 2          # area Jacobian of the reference map
        self.dxi_dx = 2.0 / self.h            # d(xi)/dx = d(eta)/dy
        self.face_jac = self.h / 2.0          # length Jacobian of every face
        e = np.arange(self.n_el)
        ex, ey = e % N, e // N
        self.x = np.broadcast_to(x0 + (ex[:, None, None] + (1.0 + self.xi[None, None, :]) / 2.0) * self.h,
                                 (self.n_el, self.P, self.P)).copy()
        self.y = np.broadcast_to(x0 + (ey[:, None, None] + (1.0 + self.xi[None, :, None]) / 2.0) * self.h,
                                 (self.n_el, self.P, self.P)).copy()
        if boundary == "periodic":
            left = ey * N + (ex - 1) % N
            right = ey * N + (ex + 1) % N
            bottom = ((ey - 1) % N) * N + ex
            top = ((ey + 1) % N) * N + ex
            self.nbr = np.stack([left, right, bottom, top], axis=1)            # [e, f]
            self.edge_of_face = np.stack([left, e, N * N + bottom, N * N + e], axis=1)
            self.n_edges = 2 * N * N
        else:
            left = np.where(ex > 0, ey * N + ex - 1, -1)
            right = np.where(ex < N - 1, ey * N + ex + 1, -1)
            bottom = np.where(ey > 0, (ey - 1) * N + ex, -1)
            top = np.where(ey < N - 1, (ey + 1) * N + ex, -1)
            self.nbr = np.stack([left, right, bottom, top], axis=1)
            nx = N * (N + 1)
            self.edge_of_face = np.stack([ey * (N + 1) + ex, ey * (N + 1) + ex + 1,
                                          nx + ey * N + ex, nx + (ey + 1) * N + ex], axis=1)
            self.n_edges = 2 * N * (N + 1)
        # mass-matrix diagonal per node (tensor-product GLL): J w_i w_j, shape [j, i]
        self.mass = self.J * np.outer(self.w, self.w)

    # -- face access -----------------------------------------------------------------
    def face_values(self, u, f):
        """Values of nodal field(s) u[..., e, j, i] on local face f, ordered along the face."""
        P = self.P
        return [u[..., :, :, 0], u[..., :, :, P - 1], u[..., :, 0, :], u[..., :, P - 1, :]][f]

    def add_to_face(self, r, f, val):
        """r[..., e, face nodes of f] += val[..., e, b]."""
        P = self.P
        if f == 0:
            r[..., :, :, 0] += val
        elif f == 1:
            r[..., :, :, P - 1] += val
        elif f == 2:
            r[..., :, 0, :] += val
        else:
            r[..., :, P - 1, :] += val

    def wall(self, f):
        """Boolean [e]: face f of the element lies on a wall."""
        return self.nbr[:, f] < 0

    def neighbour_face_values(self, u, f):
        """Scalar field u seen from the other side of face f (the neighbour's opposite face; on a
        wall, the element's own value)."""
        nb = np.where(self.nbr[:, f] < 0, np.arange(self.n_el), self.nbr[:, f])
        other = self.face_values(u[..., nb, :, :], OPPOSITE_FACE[f])
        own = self.face_values(u, f)
        return np.where(self.wall(f)[:, None], own, other)

    def neighbour_state(self, q, f):
        """State q = (phi_eta, U, V) across face f; on a wall the mirror state of eq. reflection:
        phi^+ = phi^-, U^+ = U^- - 2 (U^- . n) n; on a Dirichlet boundary the prescribed state."""
        qp = np.stack([self.neighbour_face_values(q[c], f) for c in range(3)])
        if self.boundary == "dirichlet":
            return np.where(self.wall(f)[None, :, None], self.bc_q[:, :, f, :], qp)
        return np.where(self.wall(f)[None, :, None], reflect(self.face_values(q, f), FACE_NORMALS[f]), qp)

    # -- trace vectors ---------------------------------------------------------------
    def element_traces(self, lam_g):
        """Global trace lam_g[edge, c, b] -> element view [c, e, f, b]."""
        return np.transpose(lam_g[self.edge_of_face], (2, 0, 1, 3))

    def assemble_edges(self, val_e):
        """Sum element-face contributions val_e[c, e, f, b] into a global [edge, c, b] vector."""
        out = np.zeros((self.n_edges, 3, self.P))
        np.add.at(out, self.edge_of_face, np.transpose(val_e, (1, 2, 0, 3)))
        return out

    def face_tau_hat(self, phiB):
        """tau_hat = tau_L* = max over both sides of sqrt(phi_B) at every face node, [e, f, b]."""
        t = np.zeros((self.n_el, 4, self.P))
        for f in range(4):
            t[:, f, :] = np.maximum(np.sqrt(self.face_values(phiB, f)),
                                    np.sqrt(self.neighbour_face_values(phiB, f)))
        return t


def reflect(q_face, n):
    """Mirror state across a wall with unit normal n (eq. reflection)."""
    ph, U, V = q_face
    un = U * n[0] + V * n[1]
    return np.stack([ph, U - 2.0 * un * n[0], V - 2.0 * un * n[1]])


# -- fluxes (Sec. 3.1) ------------------------------------------------------------------
def flux_full(q, phiB):
    """F = (F_x, F_y) of eq. psweFluxTensor; each is [3, ...]."""
    ph, U, V = q
    phi = ph + phiB
    Fx = np.stack([U, U * U / phi + 0.5 * ph * ph + ph * phiB, U * V / phi])
    Fy = np.stack([V, V * U / phi, V * V / phi + 0.5 * ph * ph + ph * phiB])
    return Fx, Fy


def flux_linear(q, phiB):
    """F_L of eq. psweLinearFluxTensor: rows (U, V), (phi_eta phi_B, 0), (0, phi_eta phi_B)."""
    ph, U, V = q
    z = np.zeros_like(ph)
    Fx = np.stack([U, ph * phiB, z])
    Fy = np.stack([V, z, ph * phiB])
    return Fx, Fy


def flux_nonlinear(q, phiB):
    """F_NL := F - F_L."""
    Fx, Fy = flux_full(q, phiB)
    Lx, Ly = flux_linear(q, phiB)
    return Fx - Lx, Fy - Ly


# -- element integrals ---------------------------------------------------------------------
def volume_flux_term(mesh, Fx, Fy):
    """(F, grad v)_K for every nodal test function v = l_i(xi) l_j(eta), by GLL quadrature.

    sum_{a,b} J w_a w_b [F_x(a,b) d_x v(a,b) + F_y(a,b) d_y v(a,b)], where
    d_x v_ij(a,b) = (2/h) l_i'(xi_a) delta_jb and d_y v_ij(a,b) = (2/h) delta_ia l_j'(eta_b).
    """
    w, D, c = mesh.w, mesh.D, mesh.J * mesh.dxi_dx
    tx = c * np.einsum('j,a,ai,ceja->ceji', w, w, D, Fx)
    ty = c * np.einsum('i,b,bj,cebi->ceji', w, w, D, Fy)
    return tx + ty


def nodal_gradient(mesh, u):
    """(d_x u, d_y u) of a nodal field u[e, j, i] by differentiating its interpolant."""
    dx = mesh.dxi_dx * np.einsum('ia,eja->eji', mesh.D, u)
    dy = mesh.dxi_dx * np.einsum('jb,ebi->eji', mesh.D, u)
    return dx, dy


def face_integral_to_nodes(mesh, r, f, fn):
    """r -= <fn, v>_face f: the face-node value times face Jacobian times GLL weight."""
    mesh.add_to_face(r, f, -mesh.face_jac * mesh.w * fn)


# -- DG residual of the nonlinear part (eq. SemiDiscretizedForm_ode, NL) -----------------
def rusanov_nl_normal_flux(mesh, q, phiB, f):
    """F*_NL . n on face f of every element, n the element's outward normal; [3, e, b].

    F* = {F} + tau*/2 [[q (x) n]], F_L* = {F_L} + tau_L*/2 [[q (x) n]], F*_NL = F* - F_L*,
    tau* = max_pm (|u.n| + sqrt(phi)), tau_L* = max_pm sqrt(phi_B).
    """
    n = FACE_NORMALS[f]
    qm = mesh.face_values(q, f)
    qp = mesh.neighbour_state(q, f)
    bm = mesh.face_values(phiB, f)
    bp = mesh.neighbour_face_values(phiB, f)
    Fxm, Fym = flux_full(qm, bm)
    Fxp, Fyp = flux_full(qp, bp)
    Lxm, Lym = flux_linear(qm, bm)
    Lxp, Lyp = flux_linear(qp, bp)
    # jump of q (x) n, dotted with this element's normal: q^- (n^-.n) + q^+ (n^+.n), n^+ = -n
    jump_n = qm * (n @ n) + qp * ((-n) @ n)
    phim, phip = qm[0] + bm, qp[0] + bp
    un_m = (qm[1] * n[0] + qm[2] * n[1]) / phim
    un_p = (qp[1] * n[0] + qp[2] * n[1]) / phip
    tau_star = np.maximum(np.abs(un_m) + np.sqrt(phim), np.abs(un_p) + np.sqrt(phip))
    tau_L = np.maximum(np.sqrt(bm), np.sqrt(bp))
    Fstar_n = 0.5 * ((Fxm + Fxp) * n[0] + (Fym + Fyp) * n[1]) + 0.5 * tau_star * jump_n
    FLstar_n = 0.5 * ((Lxm + Lxp) * n[0] + (Lym + Lyp) * n[1]) + 0.5 * tau_L * jump_n
    return Fstar_n - FLstar_n


def NL(mesh, q, phiB):
    """NL(q) = (F_NL(q), grad v) - <F*_NL(q^+-) . n, v> as a nodal weak-form vector [3, e, j, i]."""
    Fx, Fy = flux_nonlinear(q, phiB)
    r = volume_flux_term(mesh, Fx, Fy)
    for f in range(4):
        face_integral_to_nodes(mesh, r, f, rusanov_nl_normal_flux(mesh, q, phiB, f))
    return r


# -- explicit DG residual of the full system (the RK-DG comparison of Sec. 7) ---------------
def rusanov_full_normal_flux(mesh, q, phiB, f):
    """F* . n of eq. Full_russanov on face f of every element: {F} . n + tau*/2 (q^- - q^+)."""
    n = FACE_NORMALS[f]
    qm = mesh.face_values(q, f)
    qp = mesh.neighbour_state(q, f)
    bm = mesh.face_values(phiB, f)
    bp = mesh.neighbour_face_values(phiB, f)
    Fxm, Fym = flux_full(qm, bm)
    Fxp, Fyp = flux_full(qp, bp)
    jump_n = qm * (n @ n) + qp * ((-n) @ n)
    phim, phip = qm[0] + bm, qp[0] + bp
    un_m = (qm[1] * n[0] + qm[2] * n[1]) / phim
    un_p = (qp[1] * n[0] + qp[2] * n[1]) / phip
    tau_star = np.maximum(np.abs(un_m) + np.sqrt(phim), np.abs(un_p) + np.sqrt(phip))
    return 0.5 * ((Fxm + Fxp) * n[0] + (Fym + Fyp) * n[1]) + 0.5 * tau_star * jump_n


def DG_full(mesh, q, phiB):
    """(F(q), grad v) + (s(q), v) - <F*(q^+-) . n, v> of eq. WeakForm_DG for the whole flux;
    a nodal weak-form vector [3, e, j, i] (the explicit RK DG scheme the paper compares with)."""
    Fx, Fy = flux_full(q, phiB)
    r = volume_flux_term(mesh, Fx, Fy)
    dBx, dBy = nodal_gradient(mesh, phiB)
    s = np.stack([np.zeros_like(q[0]), q[0] * dBx, q[0] * dBy])
    r = r + mesh.mass[None, None, :, :] * s
    for f in range(4):
        face_integral_to_nodes(mesh, r, f, rusanov_full_normal_flux(mesh, q, phiB, f))
    return r


# -- HDG residual of the linear part and the conservation condition ------------------------
def hdg_normal_flux(q_face, lam_face, phiB_face, tau_face, n):
    """n . Fhat_L(q, qhat) of eq. linear_hdgflux3 at face nodes; all [3 or 1, e, b]."""
    ph, U, V = q_face
    ph_h, U_h, V_h = lam_face
    return np.stack([n[0] * U + n[1] * V + tau_face * (ph - ph_h),
                     n[0] * phiB_face * ph + tau_face * (U - U_h),
                     n[1] * phiB_face * ph + tau_face * (V - V_h)])


def L(mesh, Q, lam_e, phiB, tau_e):
    """L(q, qhat) = (F_L(q), grad v) + (s(q), v) - <Fhat_L(q, qhat) . n, v>; [3, e, j, i].

    lam_e is the element view of the trace, [3, e, f, b]; tau_e is [e, f, b].
    """
    Fx, Fy = flux_linear(Q, phiB)
    r = volume_flux_term(mesh, Fx, Fy)
    dBx, dBy = nodal_gradient(mesh, phiB)
    s = np.stack([np.zeros_like(Q[0]), Q[0] * dBx, Q[0] * dBy])
    r = r + mesh.mass[None, None, :, :] * s
    for f in range(4):
        fn = hdg_normal_flux(mesh.face_values(Q, f), lam_e[:, :, f, :], mesh.face_values(phiB, f),
                             tau_e[:, f, :], FACE_NORMALS[f])
        face_integral_to_nodes(mesh, r, f, fn)
    return r


def flux_contributions(mesh, Q, lam_e, phiB, tau_e):
    """Each element's share of Flx: <Fhat_L . n_K, mu> on its four faces, [3, e, f, b].

    Summing the two shares that meet on an edge (``Mesh.assemble_edges``) gives
    <[[Fhat_L . n]], mu>_e of eq. HDGcont at every trace node.  On a wall the second share is
    the mirror element's (eq. reflection with eq. HDGcont, which yields eq. reflectionBC).
    """
    out = np.zeros((3, mesh.n_el, 4, mesh.P))
    for f in range(4):
        n = FACE_NORMALS[f]
        qf, bf = mesh.face_values(Q, f), mesh.face_values(phiB, f)
        fn = hdg_normal_flux(qf, lam_e[:, :, f, :], bf, tau_e[:, f, :], n)
        if mesh.boundary == "dirichlet":
            # a Dirichlet trace row is qhat = q_bc: its left side is qhat (q_bc goes to R2)
            out[:, :, f, :] = np.where(mesh.wall(f)[None, :, None], lam_e[:, :, f, :],
                                       mesh.face_jac * mesh.w * fn)
            continue
        # on a wall the mirror element (eq. reflection) contributes its share with normal -n
        ghost = hdg_normal_flux(reflect(qf, n), lam_e[:, :, f, :], bf, tau_e[:, f, :], -n)
        fn = fn + np.where(mesh.wall(f)[None, :, None], ghost, 0.0)
        out[:, :, f, :] = mesh.face_jac * mesh.w * fn
    return out


def Flx(mesh, Q, lam_g, phiB, tau_e):
    """Global conservation residual Flx(Q, Qhat) at every trace node, [edge, c, b]."""
    return mesh.assemble_edges(flux_contributions(mesh, Q, mesh.element_traces(lam_g), phiB, tau_e))


def minv(mesh, r):
    """Apply the inverse of the (diagonal, collocated GLL) mass matrix to a weak-form vector."""
    return r / mesh.mass[None, None, :, :]


def trace_from_conservation(mesh, Q, phiB, tau_e, R2=None):
    """The trace that makes Flx(Q, qhat) = R2 (0 by default) for a given volume state Q.

    With collocated face quadrature the conservation rows are node-local and diagonal in
    qhat, so qhat = (R2 - Flx(Q, 0)) / Flx(0, 1) node by node.  Used where Algorithm 1 asks
    for L(Q^(i)) with no trace (an explicit first stage).
    """
    z = np.zeros((mesh.n_edges, 3, mesh.P))
    num = Flx(mesh, Q, z, phiB, tau_e)
    den = Flx(mesh, np.zeros_like(Q), np.ones_like(z), phiB, tau_e)
    return ((0.0 if R2 is None else R2) - num) / den


def dirichlet_R2(mesh, bc_face):
    """Right side of the trace rows for prescribed boundary states bc_face [3, e, f, b]: the
    boundary value on Dirichlet edges, 0 on every conservation row; global [edge, c, b]."""
    val = np.where(np.stack([mesh.wall(f) for f in range(4)], axis=1)[None, :, :, None], bc_face, 0.0)
    return mesh.assemble_edges(val)


# -- boundary conversions ------------------------------------------------------------------
def to_state(h, hu, hv, b, g, H0):
    """(h, hu, hv, b) on nodes [e, Np] -> q = (phi_eta, U, V) [3, e, j, i] and phi_B.

    B = H0 - b is the depth below the reference level, phi_B = g B, phi_eta = g (h - B),
    U = g hu, V = g hv (phi = g H and U = phi u, Sec. 3).
    """
    n_el, Np = np.shape(h)
    P = int(round(np.sqrt(Np)))
    sh = (n_el, P, P)
    B = H0 - np.reshape(b, sh)
    q = np.stack([g * (np.reshape(h, sh) - B), g * np.reshape(hu, sh), g * np.reshape(hv, sh)])
    return q, g * B


def from_state(q, phiB, g):
    """Inverse of ``to_state``: returns (h, hu, hv) as [e, Np]."""
    n_el = q.shape[1]
    B = phiB / g
    h = q[0] / g + B
    return h.reshape(n_el, -1), (q[1] / g).reshape(n_el, -1), (q[2] / g).reshape(n_el, -1)
