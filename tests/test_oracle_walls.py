"""Pins of the oracle's reflecting walls (Sec. 4.3, eq. reflection and eq. reflectionBC)."""
import math

import numpy as np
import pytest

from oracle import hdg, imex, swe
from paper_1711_02751_gb300 import workloads as W

rng = np.random.Generator(np.random.PCG64(19))


def _walled(N, k, kind="large", x0=0.0, length=1.0):
    m = swe.Mesh(N, k, boundary="wall", x0=x0, length=length)
    x, y = m.x.reshape(m.n_el, -1), m.y.reshape(m.n_el, -1)
    h, hu, hv, b = W.make_state(kind, x, y)
    q, phiB = swe.to_state(h, hu, hv, b, W.G, W.H0)
    return m, q, phiB


def test_wall_mesh_counts():
    m = swe.Mesh(3, 2, boundary="wall")
    assert m.n_edges == 2 * 3 * 4                     # 2 n (n+1) edges of the walled n x n mesh
    assert np.count_nonzero(m.nbr < 0) == 4 * 3       # 4n wall faces
    # every interior edge is shared by exactly two element faces, every wall edge by one
    counts = np.bincount(m.edge_of_face.ravel(), minlength=m.n_edges)
    assert sorted(set(counts.tolist())) == [1, 2] and np.count_nonzero(counts == 1) == 12


@pytest.mark.parametrize("N,k", [(2, 1), (3, 2), (2, 3), (4, 2)])
def test_condensed_equals_unreduced_with_walls(N, k):
    m, q, phiB = _walled(N, k)
    tau = m.face_tau_hat(phiB)
    R1 = q + 0.01 * rng.standard_normal(q.shape)
    Qu, lu = hdg.solve_unreduced(m, phiB, tau, 0.05, R1)
    Qc, lc = hdg.Condensed(m, phiB, tau, 0.05, solver="dense").solve(R1)
    assert np.abs(Qu - Qc).max() < 1e-12 * max(1.0, np.abs(Qu).max())
    assert np.abs(lu - lc).max() < 1e-12 * max(1.0, np.abs(lu).max())


def test_wall_trace_is_eq_reflectionBC():
    """On a wall: phi_hat = phi + U.n / tau, U_hat . n = 0, tangential U_hat = U^t."""
    m, q, phiB = _walled(3, 2)
    q = q + 0.01 * rng.standard_normal(q.shape)
    tau = m.face_tau_hat(phiB)
    lam_e = m.element_traces(swe.trace_from_conservation(m, q, phiB, tau))
    for f in range(4):
        w = m.wall(f)
        n = swe.FACE_NORMALS[f]
        qf = m.face_values(q, f)[:, w]
        lf = lam_e[:, w, f, :]
        t = tau[w, f, :]
        un = qf[1] * n[0] + qf[2] * n[1]
        np.testing.assert_allclose(lf[0], qf[0] + un / t, atol=1e-15)
        np.testing.assert_allclose(lf[1] * n[0] + lf[2] * n[1], 0.0, atol=1e-16)
        np.testing.assert_allclose(lf[1] * n[1] - lf[2] * n[0], qf[1] * n[1] - qf[2] * n[0], atol=1e-16)


def test_walls_conserve_mass_and_keep_lake_at_rest():
    m, q, phiB = _walled(4, 3)
    m0 = imex.mass(m, q)
    q1 = imex.Stepper(m, phiB, 0.02, solver="lu").run(q, 4)
    assert abs(imex.mass(m, q1) - m0) < 1e-15 + 1e-14 * abs(m0)
    ml, ql, pl = _walled(4, 3, kind="lake")
    assert np.all(imex.Stepper(ml, pl, 0.05, solver="lu").run(ql, 3) == 0.0)


@pytest.mark.parametrize("k", [1, 2])
def test_standing_wave_with_walls_converges(k):
    """Closed-form linear standing wave in the walled box: error falls at about k+1 in h."""
    T = 0.25
    errs = []
    for N in (4, 8, 16):
        m = swe.Mesh(N, k, boundary="wall")
        x, y = m.x.reshape(m.n_el, -1), m.y.reshape(m.n_el, -1)
        h, hu, hv, b = W.standing_wave_walls_state(x, y)
        q, phiB = swe.to_state(h, hu, hv, b, W.G, W.H0)
        q = imex.Stepper(m, phiB, T / 100, scheme="ars3", solver="lu", linear_only=True).run(q, 100)
        ht, _, _, _ = W.standing_wave_walls_state(x, y, t=T)
        qt, _ = swe.to_state(ht, hu * 0, hv * 0, b, W.G, W.H0)
        errs.append(imex.rel_l2(m, q[0], qt[0]))
    rates = [math.log2(errs[i] / errs[i + 1]) for i in range(2)]
    assert rates[-1] > k + 0.6, (errs, rates)


def test_centred_perturbation_is_symmetric_in_the_box():
    m = swe.Mesh(6, 2, boundary="wall", x0=-1.0, length=2.0)
    x, y = m.x.reshape(m.n_el, -1), m.y.reshape(m.n_el, -1)
    h, hu, hv, b = W.perturbation_state(x, y, H_inf=1.0, sigma=0.3)
    q, phiB = swe.to_state(h, hu, hv, b, W.G, W.H0)
    q = imex.Stepper(m, phiB, 0.02, solver="lu").run(q, 3)
    g = q.reshape(3, 6, 6, 3, 3)
    gx = g[:, :, ::-1, :, ::-1]
    np.testing.assert_allclose(g[0], gx[0], atol=1e-14)
    np.testing.assert_allclose(g[1], -gx[1], atol=1e-14)
