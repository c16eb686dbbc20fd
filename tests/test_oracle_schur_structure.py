"""The block structure the Schur-complement local solves rest on, checked on the oracle's own
element operators (no GPU).

The implicit stage's element operator A = I - dt a M^{-1} dL/dQ (eq. linearizedHDGsystem) is
built here by the oracle from unit vectors (oracle.hdg.local_blocks).  With collocated GLL nodes
its velocity blocks are diagonal and equal to the phi block's diagonal, so U and V can be
eliminated node by node:  S phi = x_phi - A_phiU d^{-1} x_U - A_phiV d^{-1} x_V with
S = diag(d) - A_phiU d^{-1} A_Uphi - A_phiV d^{-1} A_Vphi, and S^{-1} is the (phi, phi) block of
A^{-1}.  The couplings are A_phiU = alpha Dhat_x + kk diag(n_x) and
A_Uphi = alpha Dhat_x diag(phi_B) + diag(alpha d_x phi_B + kk n_x phi_B), with
alpha = -dt a (2/h), kk = dt a (2/h) / w_0, Dhat the weak-form derivative (w_a / w_i) D_ai and
n_x the outward x-normal of the element's faces through the node (y alike) -- the terms the
kernels rebuild from phi_B, tau and Dhat instead of storing A^{-1}.
"""
import numpy as np
import pytest

from oracle import hdg

from _common import oracle_state, user_state


def _operators(N, k, kind, dta):
    m, h, hu, hv, b = user_state(N, k, kind)
    q, phiB = oracle_state(m, h, hu, hv, b)
    tau = m.face_tau_hat(phiB)
    A = hdg.local_blocks(m, phiB, tau, dta)[0]
    return m, phiB, A


@pytest.mark.parametrize("N,k,kind", [(3, 3, "large"), (4, 2, "large"), (3, 1, "large"), (3, 4, "bump8")])
def test_velocity_blocks_are_the_phi_diagonal(N, k, kind):
    m, phiB, A = _operators(N, k, kind, 0.07)
    Np = m.P ** 2
    for e in range(m.n_el):
        Ae = A[e]
        blk = lambda r, c: Ae[r * Np:(r + 1) * Np, c * Np:(c + 1) * Np]  # noqa: E731
        d = np.diag(blk(0, 0))
        assert np.abs(blk(0, 0) - np.diag(d)).max() == 0.0
        for c in (1, 2):
            assert np.abs(blk(c, c) - np.diag(d)).max() <= 1e-15 * np.abs(d).max()
        assert np.abs(blk(1, 2)).max() == 0.0 and np.abs(blk(2, 1)).max() == 0.0
        assert d.min() >= 1.0   # 1 + kk sum tau >= 1: the node-by-node elimination never divides by 0


@pytest.mark.parametrize("N,k,kind", [(3, 3, "large"), (4, 2, "large"), (3, 4, "bump8")])
def test_schur_route_reproduces_the_local_solve(N, k, kind):
    rng = np.random.Generator(np.random.PCG64(1711))
    m, phiB, A = _operators(N, k, kind, 0.07)
    Np = m.P ** 2
    for e in range(m.n_el):
        Ae = A[e]
        blk = lambda r, c: Ae[r * Np:(r + 1) * Np, c * Np:(c + 1) * Np]  # noqa: E731
        rd = 1.0 / np.diag(blk(0, 0))
        S = blk(0, 0) - blk(0, 1) @ (rd[:, None] * blk(1, 0)) - blk(0, 2) @ (rd[:, None] * blk(2, 0))
        Ainv = np.linalg.inv(Ae)
        assert np.abs(np.linalg.inv(S) - Ainv[:Np, :Np]).max() <= 1e-12 * np.abs(Ainv[:Np, :Np]).max()
        x = rng.standard_normal(3 * Np)
        xp, xu, xv = x[:Np], x[Np:2 * Np], x[2 * Np:]
        phi = np.linalg.solve(S, xp - blk(0, 1) @ (rd * xu) - blk(0, 2) @ (rd * xv))
        U = rd * (xu - blk(1, 0) @ phi)
        V = rd * (xv - blk(2, 0) @ phi)
        ref = np.linalg.solve(Ae, x)
        got = np.concatenate([phi, U, V])
        assert np.abs(got - ref).max() <= 1e-12 * np.abs(ref).max()


@pytest.mark.parametrize("N,k", [(3, 3), (4, 2)])
def test_couplings_are_the_rebuilt_terms(N, k):
    """The coefficients the kernels rebuild (per instance E = alpha Dhat + kk diag(n) and
    G = alpha Dhat; per node d, c_x, c_y) against the oracle's A entry by entry."""
    dta = 0.07
    m, phiB, A = _operators(N, k, "large", dta)
    P, Np = m.P, m.P ** 2
    th = 2.0 / m.h
    alpha, kk = -dta * th, dta * th / m.w[0]
    Dhat = (m.w[None, :] / m.w[:, None]) * m.D.T          # Dhat[i, a] = (w_a / w_i) D[a, i]
    nv = np.zeros(P)
    nv[0], nv[-1] = -1.0, 1.0
    E = alpha * Dhat + kk * np.diag(nv)
    I = np.eye(P)
    Ex = np.kron(I, E)          # acts along i (x) for node index j * P + i
    Ey = np.kron(E, I)          # along j (y)
    G = alpha * Dhat
    Gx, Gy = np.kron(I, G), np.kron(G, I)
    Dx, Dy = np.kron(I, m.D), np.kron(m.D, I)
    nx = np.tile(nv, P)                   # x-normal of the face through node (i, j)
    ny = np.repeat(nv, P)
    scale = np.abs(A).max()
    for e in range(m.n_el):
        Ae = A[e]
        pb = phiB[e].reshape(-1)
        blk = lambda r, c: Ae[r * Np:(r + 1) * Np, c * Np:(c + 1) * Np]  # noqa: E731
        assert np.abs(blk(0, 1) - Ex).max() <= 1e-13 * scale
        assert np.abs(blk(0, 2) - Ey).max() <= 1e-13 * scale
        cx = alpha * (Dx @ pb) + kk * nx * pb
        cy = alpha * (Dy @ pb) + kk * ny * pb
        assert np.abs(blk(1, 0) - (Gx * pb[None, :] + np.diag(cx))).max() <= 1e-13 * scale
        assert np.abs(blk(2, 0) - (Gy * pb[None, :] + np.diag(cy))).max() <= 1e-13 * scale
