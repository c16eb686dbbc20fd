"""The implicit HDG stage system and its static condensation -- oracle.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).  Sec. 6 of the paper: an implicit
IMEX stage with diagonal coefficient a = a_ii solves, for (Q, Qhat),

    Res(Q, Qhat) = Q - dt a M^{-1} L(Q, Qhat) - R1 = 0      (eq. IMEXRKDiscretizedForm)
    Flx(Q, Qhat) = <[[Fhat_L(Q, Qhat) . n]], mu>   = 0

which is linear, i.e. [[A, B], [C, D]] [Q; Qhat] = [R1; 0] (eq. linearizedHDGsystem) with
A = I - dt a M^{-1} dL/dQ, B = -dt a M^{-1} dL/dQhat, C = dFlx/dQ, D = dFlx/dQhat.

Two independent routes:
* ``solve_unreduced``: every column of the global operator is obtained by applying the
  residuals above to a unit vector, then one dense solve of the whole coupled system.
* ``Condensed``: element blocks A_e, B_e, C_e, D_e from unit vectors applied to the
  element-local residuals; Schur complement (D - C A^{-1} B) Qhat = -C A^{-1} R1
  (eq. linearizedHDGsystem_schur), factorised ONCE and reused for every stage and step as
  the paper does with its one-time LU (Sec. 7.1); then element-wise recovery
  Q = A^{-1}(R1 - B Qhat) (eq. recover_volume_unknowns).
"""
import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from . import swe


def _stage_residual_global(mesh, phiB, tau_e, dta, Q, lam_g):
    """(Q - dt a M^{-1} L(Q, Qhat), Flx(Q, Qhat)) flattened; the LHS of the stage system."""
    lam_e = mesh.element_traces(lam_g)
    rv = Q - dta * swe.minv(mesh, swe.L(mesh, Q, lam_e, phiB, tau_e))
    rt = swe.Flx(mesh, Q, lam_g, phiB, tau_e)
    return np.concatenate([rv.ravel(), rt.ravel()])


def unreduced_matrix(mesh, phiB, tau_e, dta):
    """Dense [[A, B], [C, D]] of the whole mesh, one unit vector per column (tiny meshes)."""
    nv = 3 * mesh.n_el * mesh.P ** 2
    nt = mesh.n_edges * 3 * mesh.P
    K = np.zeros((nv + nt, nv + nt))
    Qshape = (3, mesh.n_el, mesh.P, mesh.P)
    Lshape = (mesh.n_edges, 3, mesh.P)
    for col in range(nv + nt):
        u = np.zeros(nv + nt)
        u[col] = 1.0
        K[:, col] = _stage_residual_global(mesh, phiB, tau_e, dta,
                                           u[:nv].reshape(Qshape), u[nv:].reshape(Lshape))
    return K, nv, nt


def solve_unreduced(mesh, phiB, tau_e, dta, R1, R2=None):
    """Direct dense solve of the coupled (Q, Qhat) system; returns (Q [3,e,j,i], Qhat [edge,c,b]).
    R2 [edge, c, b] is the right side of the trace rows (0 except prescribed boundary values)."""
    K, nv, nt = unreduced_matrix(mesh, phiB, tau_e, dta)
    r2 = np.zeros(nt) if R2 is None else R2.ravel()
    sol = np.linalg.solve(K, np.concatenate([R1.ravel(), r2]))
    return sol[:nv].reshape(R1.shape), sol[nv:].reshape(mesh.n_edges, 3, mesh.P)


def _elem_major(u):
    """[3, e, ...] -> [e, 3 * ...] (element-local vector, field slowest)."""
    return np.moveaxis(u, 1, 0).reshape(u.shape[1], -1)


def _field_major(u, shape):
    """Inverse of ``_elem_major``: [e, n] -> [3, e, ...] with ... = shape."""
    return np.moveaxis(u.reshape((u.shape[0], 3) + tuple(shape)), 0, 1)


def local_blocks(mesh, phiB, tau_e, dta):
    """Per-element A_e, B_e, C_e, D_e of the stage system, by unit vectors.

    Local volume vector: (c, j, i) of one element, n_v = 3 P^2.  Local trace vector:
    (c, f, b) over the element's four faces, n_t = 12 P.  Because the element-local
    residuals depend only on the element's own Q and the traces on its own faces, a unit
    vector placed at the same local slot of every element probes all elements at once.
    """
    P, E = mesh.P, mesh.n_el
    nvl, ntl = 3 * P * P, 12 * P
    A = np.zeros((E, nvl, nvl))
    B = np.zeros((E, nvl, ntl))
    C = np.zeros((E, ntl, nvl))
    D = np.zeros((E, ntl, ntl))
    zq = np.zeros((3, E, P, P))
    zl = np.zeros((3, E, 4, P))
    for d in range(nvl):
        u = np.zeros((E, nvl))
        u[:, d] = 1.0
        Q = _field_major(u, (P, P))
        rv = Q - dta * swe.minv(mesh, swe.L(mesh, Q, zl, phiB, tau_e))
        A[:, :, d] = _elem_major(rv)
        C[:, :, d] = _elem_major(swe.flux_contributions(mesh, Q, zl, phiB, tau_e))
    for t in range(ntl):
        u = np.zeros((E, ntl))
        u[:, t] = 1.0
        lam = _field_major(u, (4, P))
        rv = -dta * swe.minv(mesh, swe.L(mesh, zq, lam, phiB, tau_e))
        B[:, :, t] = _elem_major(rv)
        D[:, :, t] = _elem_major(swe.flux_contributions(mesh, zq, lam, phiB, tau_e))
    return A, B, C, D


def local_trace_index(mesh):
    """Global trace index of every element-local trace slot (c, f, b), shape [e, 12P].

    Global trace vector layout is [edge][c][b].
    """
    P = mesh.P
    c = np.arange(3)[:, None, None]
    b = np.arange(P)[None, None, :]
    edge = mesh.edge_of_face[:, None, :, None]            # [e, 1, f, 1]
    return ((edge * 3 + c[None]) * P + b[None]).reshape(mesh.n_el, -1)


class Condensed:
    """Static condensation of the stage system, set up once for a given dt * a_ii.

    solver: 'lu' (sparse LU of the trace matrix, reused), 'dense' (dense LU), or
    'gmres' (scipy GMRES with the trace matrix's edge-block-diagonal inverse as
    preconditioner, relative residual ``rtol``) for meshes too large to factorise.
    """

    def __init__(self, mesh, phiB, tau_e, dta, solver="lu", rtol=1e-14):
        self.mesh, self.dta, self.solver, self.rtol = mesh, dta, solver, rtol
        A, B, C, D = local_blocks(mesh, phiB, tau_e, dta)
        self.Ainv = np.linalg.inv(A)
        self.B, self.C = B, C
        S_loc = D - C @ self.Ainv @ B                           # [e, nt, nt]
        gi = local_trace_index(mesh)
        rows = np.broadcast_to(gi[:, :, None], S_loc.shape).ravel()
        cols = np.broadcast_to(gi[:, None, :], S_loc.shape).ravel()
        n = mesh.n_edges * 3 * mesh.P
        self.S = sp.csr_matrix((S_loc.ravel(), (rows, cols)), shape=(n, n))
        self.gi = gi
        self.n = n
        if solver == "dense":
            self.lu = sla.lu_factor(self.S.toarray())
        elif solver == "lu":
            self.lu = spla.splu(self.S.tocsc())
        elif solver == "gmres":
            nb = 3 * mesh.P
            blocks = self.S.toarray() if n <= 4096 else None
            self.Minv = self._block_jacobi(nb, blocks)
        else:
            raise ValueError(solver)
        self.last_iterations = 0

    def _block_jacobi(self, nb, dense):
        n_blocks = self.n // nb
        if dense is not None:
            diag = np.stack([dense[r * nb:(r + 1) * nb, r * nb:(r + 1) * nb] for r in range(n_blocks)])
        else:
            Sc = self.S.tocoo()
            keep = (Sc.row // nb) == (Sc.col // nb)
            diag = np.zeros((n_blocks, nb, nb))
            np.add.at(diag, (Sc.row[keep] // nb, Sc.row[keep] % nb, Sc.col[keep] % nb), Sc.data[keep])
        inv = np.linalg.inv(diag)
        return sp.block_diag([sp.coo_matrix(b) for b in inv], format="csr")

    def rhs(self, R1, R2=None):
        """R2 - C A^{-1} R1 assembled on the skeleton (R2 = 0 except prescribed boundary values)."""
        R1e = _elem_major(R1)
        loc = -np.einsum('etv,ev->et', self.C, np.einsum('evw,ew->ev', self.Ainv, R1e))
        g = np.bincount(self.gi.ravel(), weights=loc.ravel(), minlength=self.n)
        return g if R2 is None else g + R2.ravel()

    def solve_trace(self, g):
        if self.solver == "dense":
            return sla.lu_solve(self.lu, g)
        if self.solver == "lu":
            return self.lu.solve(g)
        its = [0]

        def count(_):
            its[0] += 1
        x, info = spla.gmres(self.S, g, rtol=self.rtol, atol=0.0, restart=60, maxiter=2000,
                             M=self.Minv, callback=count, callback_type="pr_norm")
        if info != 0:
            raise RuntimeError(f"oracle GMRES did not converge (info={info})")
        self.last_iterations = its[0]
        return x

    def recover(self, R1, lam):
        """Q = A^{-1} (R1 - B Qhat), element by element (eq. recover_volume_unknowns)."""
        R1e = _elem_major(R1)
        lam_loc = lam[self.gi]                                   # [e, nt]
        Qe = np.einsum('evw,ew->ev', self.Ainv, R1e - np.einsum('evt,et->ev', self.B, lam_loc))
        return _field_major(Qe, R1.shape[2:])

    def solve(self, R1, R2=None):
        g = self.rhs(R1, R2)
        lam = self.solve_trace(g)
        Q = self.recover(R1, lam)
        return Q, lam.reshape(self.mesh.n_edges, 3, self.mesh.P)
