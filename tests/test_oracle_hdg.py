"""Pins of the oracle's implicit HDG stage, static condensation and Algorithm 1 stepping."""
import math

import numpy as np
import pytest

from oracle import hdg, imex, swe
from paper_1711_02751_gb300 import workloads as W

rng = np.random.Generator(np.random.PCG64(11))


def _mesh_state(N, k, kind="large"):
    m = swe.Mesh(N, k)
    x, y = m.x.reshape(m.n_el, -1), m.y.reshape(m.n_el, -1)
    h, hu, hv, b = W.make_state(kind, x, y)
    q, phiB = swe.to_state(h, hu, hv, b, W.G, W.H0)
    return m, q, phiB


@pytest.mark.parametrize("N,k", [(2, 1), (2, 2), (3, 1), (3, 3), (4, 2), (4, 4), (2, 4)])
def test_condensed_equals_unreduced_direct_solve(N, k):
    """Static condensation + recovery reproduces the direct solve of the whole coupled system."""
    m, q, phiB = _mesh_state(N, k)
    tau = m.face_tau_hat(phiB)
    dta = 0.07
    R1 = q + 0.01 * rng.standard_normal(q.shape)
    Qu, lu = hdg.solve_unreduced(m, phiB, tau, dta, R1)
    Qc, lc = hdg.Condensed(m, phiB, tau, dta, solver="dense").solve(R1)
    assert np.abs(Qu - Qc).max() < 1e-12 * max(1.0, np.abs(Qu).max())
    assert np.abs(lu - lc).max() < 1e-12 * max(1.0, np.abs(lu).max())
    # the unreduced solution satisfies both residual equations
    rv = Qu - dta * swe.minv(m, swe.L(m, Qu, m.element_traces(lu), phiB, tau)) - R1
    rt = swe.Flx(m, Qu, lu, phiB, tau)
    assert np.abs(rv).max() < 1e-12 and np.abs(rt).max() < 1e-12


def test_trace_count_and_blocks():
    """Periodic n x n mesh: 2 n^2 edges of (k+1) nodes per field (the non-periodic count of
    Sec. 6 is 2 n (n+1)(p+1)); D = dFlx/dQhat is diagonal node by node (collocated faces)."""
    m, q, phiB = _mesh_state(3, 2)
    assert m.n_edges * m.P == 2 * 3 * 3 * 3
    tau = m.face_tau_hat(phiB)
    A, B, C, D = hdg.local_blocks(m, phiB, tau, 0.1)
    for e in range(m.n_el):
        assert np.count_nonzero(D[e] - np.diag(np.diag(D[e]))) == 0
    # B couples each trace node to exactly one volume node of the same field
    assert np.all(np.count_nonzero(B, axis=1) == 1)
    # A is non-singular and well conditioned for a dissipative L
    assert np.linalg.cond(A[0]) < 1e4


def test_trace_matrix_is_not_symmetric():
    """The condensed trace matrix is non-symmetric, so the Krylov solver is GMRES, not CG."""
    m, q, phiB = _mesh_state(4, 2, kind="bump8")
    tau = m.face_tau_hat(phiB)
    S = hdg.Condensed(m, phiB, tau, 0.2, solver="dense").S.toarray()
    assert np.linalg.norm(S - S.T) / np.linalg.norm(S) > 0.1


def test_linear_residual_identity():
    """L_i = M (Q^(i) - R1) / (dt a_ii) for the recovered stage state (local rows are exact)."""
    m, q, phiB = _mesh_state(3, 3)
    st = imex.Stepper(m, phiB, 0.05, solver="dense")
    st.step(q)
    for i in (1, 2):
        lhs = swe.minv(m, st.last["L"][i])
        rhs = (st.last["Q"][i] - st.last["R1"][i]) / (0.05 * st.a_ii)
        assert np.abs(lhs - rhs).max() < 1e-10 * np.abs(lhs).max()


def test_gmres_route_matches_lu_route():
    m, q, phiB = _mesh_state(6, 3)
    a = imex.Stepper(m, phiB, 0.04, solver="lu").run(q, 2)
    b = imex.Stepper(m, phiB, 0.04, solver="gmres", rtol=1e-14).run(q, 2)
    for c in range(3):
        assert imex.rel_l2(m, b[c], a[c]) < 1e-12


def test_lake_at_rest_is_bitwise_steady():
    m, q, phiB = _mesh_state(4, 3, kind="lake")
    assert np.all(q == 0.0)
    q1 = imex.Stepper(m, phiB, 0.1, solver="lu").run(q, 3)
    assert np.all(q1 == 0.0)


@pytest.mark.parametrize("scheme", ["ars2", "ars3"])
def test_mass_conserved_to_round_off(scheme):
    m, q, phiB = _mesh_state(4, 3)
    m0 = imex.mass(m, q)
    q1 = imex.Stepper(m, phiB, 0.05, scheme=scheme, solver="lu").run(q, 5)
    assert abs(imex.mass(m, q1) - m0) < 1e-15 * 10 + 1e-14 * abs(m0)


def test_linear_energy_non_increasing():
    """Linear part only (NL dropped): the discrete energy never grows (Lemma of Sec. 5)."""
    m, q, phiB = _mesh_state(4, 3)
    st = imex.Stepper(m, phiB, 0.05, solver="lu", linear_only=True)
    e = [imex.energy_linear(m, q, phiB)]
    for _ in range(10):
        q = st.step(q)
        e.append(imex.energy_linear(m, q, phiB))
    assert all(e[i + 1] <= e[i] * (1 + 1e-14) for i in range(len(e) - 1)), e
    assert e[-1] < e[0]


def _standing_wave_error(N, k, scheme, n_steps, T):
    m = swe.Mesh(N, k)
    x, y = m.x.reshape(m.n_el, -1), m.y.reshape(m.n_el, -1)
    h, hu, hv, b = W.standing_wave_state(x, y)
    q, phiB = swe.to_state(h, hu, hv, b, W.G, W.H0)
    q = imex.Stepper(m, phiB, T / n_steps, scheme=scheme, solver="lu", linear_only=True).run(q, n_steps)
    ht, hut, hvt, _ = W.standing_wave_state(x, y, t=T)
    qt, _ = swe.to_state(ht, hut, hvt, b, W.G, W.H0)
    return imex.rel_l2(m, q[0], qt[0])


@pytest.mark.parametrize("k", [1, 2])
def test_standing_wave_spatial_order(k):
    """Linear standing wave (closed form of the linear PDE): error falls at about k+1 in h."""
    T = 0.25
    errs = [_standing_wave_error(N, k, "ars3", 100, T) for N in (4, 8, 16)]
    rates = [math.log2(errs[i] / errs[i + 1]) for i in range(2)]
    assert rates[-1] > k + 0.6, (errs, rates)


@pytest.mark.parametrize("scheme,order", [("ars2", 2), ("ars3", 3)])
def test_standing_wave_temporal_order(scheme, order):
    """Fine space (k = 6), coarse steps: error falls at the scheme's order in dt."""
    T = 0.3
    errs = [_standing_wave_error(4, 6, scheme, n, T) for n in (6, 12, 24)]
    rates = [math.log2(errs[i] / errs[i + 1]) for i in range(2)]
    assert min(rates) > order - 0.3, (errs, rates)


def test_centred_bump_keeps_its_symmetries():
    """The 8x8 centred-bump workload is symmetric under x -> 1-x, y -> 1-y and x <-> y."""
    m, q, phiB = _mesh_state(8, 2, kind="bump8")
    dt = W.advective_dt(m.x.reshape(m.n_el, -1), *swe.from_state(q, phiB, W.G), n_side=8)
    q = imex.Stepper(m, phiB, dt, solver="lu").run(q, 3)
    N, P = 8, 3
    g = q.reshape(3, N, N, P, P)                     # [c, ey, ex, j, i]
    gx = g[:, :, ::-1, :, ::-1]                      # mirror in x
    np.testing.assert_allclose(g[0], gx[0], atol=1e-14)
    np.testing.assert_allclose(g[1], -gx[1], atol=1e-14)
    np.testing.assert_allclose(g[2], gx[2], atol=1e-14)
    gt = np.transpose(g, (0, 2, 1, 4, 3))           # swap x and y
    np.testing.assert_allclose(g[0], gt[0], atol=1e-14)
    np.testing.assert_allclose(g[1], gt[2], atol=1e-14)
