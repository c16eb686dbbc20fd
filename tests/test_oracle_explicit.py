"""Pins of the oracle's explicit RK DG (the paper's comparison scheme)."""
import math

import numpy as np
import pytest

from oracle import imex, swe
from paper_1711_02751_gb300 import workloads as W


def test_full_residual_is_nl_plus_linear_with_conserving_trace():
    """F = F_NL + F_L and F* = F*_NL + F_L*, with Fhat_L at the conserving trace equal to F_L*
    on a polygonal mesh (footnote of Sec. 4.3): DG_full = NL + L(q, qhat*)."""
    m = swe.Mesh(4, 3)
    rng = np.random.Generator(np.random.PCG64(3))
    q = 0.02 * rng.standard_normal((3,) + m.x.shape)
    phiB = 1.0 + 0.1 * np.sin(2 * np.pi * m.x) * np.sin(2 * np.pi * m.y)
    tau = m.face_tau_hat(phiB)
    lam = swe.trace_from_conservation(m, q, phiB, tau)
    a = swe.DG_full(m, q, phiB)
    b = swe.NL(m, q, phiB) + swe.L(m, q, m.element_traces(lam), phiB, tau)
    assert np.abs(a - b).max() <= 1e-14 * np.abs(a).max()


@pytest.mark.parametrize("scheme,order", [("rk2", 2), ("rk3", 3)])
def test_explicit_rk_converges_on_the_linear_wave(scheme, order):
    """Standing wave of amplitude 1e-6 (nonlinear terms negligible): temporal order 2 / 3."""
    m = swe.Mesh(4, 6)
    x, y = m.x.reshape(m.n_el, -1), m.y.reshape(m.n_el, -1)
    h, hu, hv, b = W.standing_wave_state(x, y, eps=1e-6)
    q0, phiB = swe.to_state(h, hu, hv, b, W.G, W.H0)
    T = 0.05
    ref = imex.ExplicitRK(m, phiB, T / 400, scheme).run(q0, 400)
    errs = []
    for n in (25, 50, 100):
        qa = imex.ExplicitRK(m, phiB, T / n, scheme).run(q0, n)
        errs.append(np.sqrt(np.sum(m.mass * (qa[0] - ref[0]) ** 2)))
    rates = [math.log2(errs[i] / errs[i + 1]) for i in range(2)]
    assert min(rates) > order - 0.3, (errs, rates)


def test_stability_contrast_with_imex():
    """Sec. 7: the explicit RK2 DG blows up once the gravity Courant number is well above its
    limit (the paper: above Cr ~ 0.28), while ARS2 HDG-DG stays bounded at the same large dt."""
    m = swe.Mesh(8, 2)
    x, y = m.x.reshape(m.n_el, -1), m.y.reshape(m.n_el, -1)
    h, hu, hv, b = W.bump8_state(x, y)
    q0, phiB = swe.to_state(h, hu, hv, b, W.G, W.H0)
    dx_min = (1 / 8) / 2 * np.diff(m.xi).min()
    dt_big = 4.0 * dx_min            # gravity Courant 4
    dt_small = 0.1 * dx_min          # gravity Courant 0.1
    with np.errstate(all="ignore"):
        qe = imex.ExplicitRK(m, phiB, dt_big, "rk2").run(q0, 40)
    assert not np.all(np.isfinite(qe)) or np.abs(qe).max() > 1.0
    qs = imex.ExplicitRK(m, phiB, dt_small, "rk2").run(q0, 40)
    assert np.abs(qs[0]).max() < 0.011
    qi = imex.Stepper(m, phiB, dt_big, solver="lu").run(q0, 40)
    assert np.all(np.isfinite(qi)) and np.abs(qi[0]).max() < 0.011
