"""Pins of the oracle's Dirichlet boundaries with the paper's moving vortex (Sec. 7.1)."""
import json
import math
import os

import numpy as np
import pytest

from oracle import hdg, imex, swe
from paper_1711_02751_gb300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "vortex_errors.json")
V = W.VORTEX


def vortex_problem(N, k):
    m = swe.Mesh(N, k, boundary="dirichlet", x0=-2.0, length=4.0)
    x, y = m.x.reshape(m.n_el, -1), m.y.reshape(m.n_el, -1)
    h, hu, hv, b = W.vortex_state(x, y, 0.0, **V)
    q, phiB = swe.to_state(h, hu, hv, b, V["g"], V["H_inf"])
    P = m.P

    def bc(t):
        hh, uu, vv, bb = W.vortex_state(m.x.reshape(m.n_el, -1), m.y.reshape(m.n_el, -1), t, **V)
        qq, _ = swe.to_state(hh, uu, vv, bb, V["g"], V["H_inf"])
        return np.stack([m.face_values(qq, f) for f in range(4)], axis=2)   # [3, e, 4, P]
    return m, q, phiB, bc


def eta_errors(m, q, t):
    """L1, L2 and Linf errors of eta against the exact vortex (GLL quadrature, nodal max)."""
    x, y = m.x.reshape(m.n_el, -1), m.y.reshape(m.n_el, -1)
    h, _, _, _ = W.vortex_state(x, y, t, **V)
    e = q[0] / V["g"] - (h.reshape(m.x.shape) - V["H_inf"])
    w = m.mass[None]
    return float(np.sum(w * np.abs(e))), float(np.sqrt(np.sum(w * e * e))), float(np.abs(e).max())


def test_condensed_equals_unreduced_with_dirichlet_traces():
    m, q, phiB, bc = vortex_problem(3, 2)
    m.bc_q = bc(0.1)
    R2 = swe.dirichlet_R2(m, m.bc_q)
    tau = m.face_tau_hat(phiB)
    R1 = q + 0.01 * np.random.default_rng(1).standard_normal(q.shape)
    Qu, lu = hdg.solve_unreduced(m, phiB, tau, 0.01, R1, R2)
    Qc, lc = hdg.Condensed(m, phiB, tau, 0.01, solver="dense").solve(R1, R2)
    assert np.abs(Qu - Qc).max() < 1e-12 * np.abs(Qu).max()
    assert np.abs(lu - lc.reshape(lu.shape)).max() < 1e-12 * np.abs(lu).max()
    # the boundary traces are the prescribed states
    lam_e = m.element_traces(lu)
    for f in range(4):
        wmask = m.wall(f)
        np.testing.assert_allclose(lam_e[:, wmask, f, :], m.bc_q[:, wmask, f, :], atol=1e-13)


def test_vortex_translates_and_converges():
    """ARS3 HDG-DG with exact-solution traces: the vortex error at t = 0.2 falls with h."""
    errs = []
    for N in (4, 8):
        m, q, phiB, bc = vortex_problem(N, 2)
        st = imex.Stepper(m, phiB, 0.005, scheme="ars3", solver="lu", bc=bc)
        q = st.run(q, 40)
        errs.append(eta_errors(m, q, 0.2)[1])
    assert errs[1] < errs[0] / 3.0, errs


@pytest.mark.slow_oracle
def test_vortex_error_matches_papers_table():
    """p = 2 at T = 2 on 4x4 and 8x8 (Table tab:tc_mv_hconv_hdg3): the L1 and L2 errors of eta
    agree with the printed values to within 15% (measured: 7% and 4% on 4x4, 3% and 3% on 8x8).
    The printed Linf is not pinned: the paper does not say at which points it takes the maximum
    (this oracle's nodal maximum includes the element-edge nodes of a discontinuous field)."""
    gold = json.load(open(GOLDEN))["eta"]["2"]
    for N in (4, 8):
        m, q, phiB, bc = vortex_problem(N, 2)
        st = imex.Stepper(m, phiB, 0.005, scheme="ars3", solver="lu", bc=bc)
        q = st.run(q, 400)
        l1, l2, _ = eta_errors(m, q, 2.0)
        ref = gold[str(N)]
        assert abs(l1 - ref[0]) <= 0.15 * ref[0], (N, l1, ref[0])
        assert abs(l2 - ref[1]) <= 0.15 * ref[1], (N, l2, ref[1])


@pytest.mark.slow_oracle
@pytest.mark.parametrize("k,dt", [(2, 0.005), (3, 0.0025)])
def test_vortex_error_on_16x16_matches_papers_table_to_two_percent(k, dt):
    """p = 2 and 3 at T = 2 on 16 x 16 (Table tab:tc_mv_hconv_hdg3): on a mesh that resolves the
    vortex, the L1 and L2 errors of eta agree with the printed values to within 2% (measured:
    0.3% for p = 2, 0.05% for p = 3).  This pins the Rusanov dissipation coefficient tau* of the
    explicit part against the paper's own numbers: with tau* = sqrt(phi) (|u.n| dropped) the p = 2
    errors move by -8.9% / -4.4%, with |U.n| not divided by phi by +10% / +13%, while on 4 x 4 and
    8 x 8 the second slip stays within the 15% of the test above.  (The sharp pin of tau* is the
    flux Jacobian's spectrum in test_oracle_swe.)"""
    gold = json.load(open(GOLDEN))["eta"][str(k)]["16"]
    m, q, phiB, bc = vortex_problem(16, k)
    st = imex.Stepper(m, phiB, dt, scheme="ars3", solver="lu", bc=bc)
    q = st.run(q, int(round(2.0 / dt)))
    l1, l2, _ = eta_errors(m, q, 2.0)
    assert abs(l1 - gold[0]) <= 0.02 * gold[0], (l1, gold[0])
    assert abs(l2 - gold[1]) <= 0.02 * gold[1], (l2, gold[1])
