"""Pins of the oracle's DG / HDG residuals against exact integrals, identities and limits."""
import math

import numpy as np
import pytest
import sympy as sym
from numpy.polynomial import Polynomial
from numpy.polynomial.legendre import leggauss

from oracle import swe
from oracle.gll import gll_nodes_weights

rng = np.random.Generator(np.random.PCG64(7))


def _basis(k):
    x, _ = gll_nodes_weights(k)
    ls = []
    for j in range(k + 1):
        others = np.delete(x, j)
        ls.append(Polynomial.fromroots(others) / np.prod(x[j] - others))
    return ls


@pytest.mark.parametrize("k", [1, 2, 3, 4])
def test_volume_term_equals_exact_integral(k):
    """(F, grad v)_K equals the exact integral when the integrand is within GLL exactness.

    F_x = p(x) r(y) with deg p <= k, deg r <= k-1 (and F_y with the roles swapped):
    integrand degrees stay <= 2k-1, so the collocated quadrature must be exact.
    Reference: 12-point Gauss-Legendre of the analytic polynomials on one element.
    """
    N = 3
    m = swe.Mesh(N, k)
    px = Polynomial(rng.standard_normal(k + 1))
    ry = Polynomial(rng.standard_normal(k))
    Fx = np.zeros((3, m.n_el, k + 1, k + 1))
    Fy = np.zeros_like(Fx)
    xi = m.xi
    Fx[1] = (ry(xi)[:, None] * px(xi)[None, :])[None]          # [j, i] -> p(xi_i) r(eta_j)
    Fy[2] = (px(xi)[:, None] * ry(xi)[None, :])[None]          # p(eta_j) r(xi_i)
    got = swe.volume_flux_term(m, Fx, Fy)
    t, wt = leggauss(12)
    ls = _basis(k)
    h = m.h
    for j in range(k + 1):
        for i in range(k + 1):
            # d/dx = (2/h) d/dxi ; dK = (h/2)^2 dxi deta
            ex_x = (h / 2) ** 2 * (2 / h) * np.sum(wt[:, None] * wt[None, :] *
                                                  (px(t)[None, :] * ry(t)[:, None]) *
                                                  (ls[i].deriv()(t)[None, :] * ls[j](t)[:, None]))
            ex_y = (h / 2) ** 2 * (2 / h) * np.sum(wt[:, None] * wt[None, :] *
                                                  (px(t)[:, None] * ry(t)[None, :]) *
                                                  (ls[i](t)[None, :] * ls[j].deriv()(t)[:, None]))
            assert abs(got[1, 0, j, i] - ex_x) < 1e-12
            assert abs(got[2, 0, j, i] - ex_y) < 1e-12


def _smooth_fields():
    x, y = sym.symbols("x y")
    two_pi = 2 * sym.pi
    ph = sym.Rational(1, 10) * sym.sin(two_pi * x) * sym.cos(two_pi * y) + sym.Rational(1, 20) * sym.cos(two_pi * y)
    U = sym.Rational(1, 20) * sym.cos(two_pi * x + 1) + sym.Rational(1, 50) * sym.sin(two_pi * y)
    V = sym.Rational(3, 100) * sym.sin(two_pi * y + sym.Rational(1, 2)) * sym.cos(two_pi * x)
    pB = 1 + sym.Rational(1, 10) * sym.sin(two_pi * x) * sym.sin(two_pi * y)
    return x, y, ph, U, V, pB


def _eval(expr, xs, ys):
    f = sym.lambdify(sym.symbols("x y"), expr, "numpy")
    return np.broadcast_to(f(xs, ys), xs.shape).astype(float)


def _state(m, exprs):
    x, y, ph, U, V, pB = exprs
    q = np.stack([_eval(ph, m.x, m.y), _eval(U, m.x, m.y), _eval(V, m.x, m.y)])
    return q, _eval(pB, m.x, m.y)


def test_nl_converges_to_minus_divergence():
    """For a smooth state M^{-1} NL(q) -> -div F_NL at the nodes, at rate ~k."""
    ex = _smooth_fields()
    x, y, ph, U, V, pB = ex
    phi = ph + pB
    div = [sym.Integer(0),
           sym.diff(U * U / phi + ph ** 2 / 2, x) + sym.diff(U * V / phi, y),
           sym.diff(U * V / phi, x) + sym.diff(V * V / phi + ph ** 2 / 2, y)]
    k = 2
    errs = []
    for N in (8, 16, 32):
        m = swe.Mesh(N, k)
        q, phiB = _state(m, ex)
        r = swe.minv(m, swe.NL(m, q, phiB))
        ref = np.stack([np.zeros_like(m.x)] + [-_eval(d, m.x, m.y) for d in div[1:]])
        errs.append(np.sqrt(np.mean((r - ref) ** 2)) / np.sqrt(np.mean(ref ** 2)))
    rates = [math.log2(errs[i] / errs[i + 1]) for i in range(2)]
    assert errs[-1] < 2e-2 and min(rates) > k - 0.3, (errs, rates)


def test_linear_residual_converges_to_pde():
    """M^{-1} L(q, qhat*) -> -div F_L + s for a smooth state, qhat* the conservation trace."""
    ex = _smooth_fields()
    x, y, ph, U, V, pB = ex
    rhs = [-(sym.diff(U, x) + sym.diff(V, y)),
           -sym.diff(ph * pB, x) + ph * sym.diff(pB, x),
           -sym.diff(ph * pB, y) + ph * sym.diff(pB, y)]
    k = 3
    errs = []
    for N in (4, 8, 16):
        m = swe.Mesh(N, k)
        q, phiB = _state(m, ex)
        tau = m.face_tau_hat(phiB)
        lam = swe.trace_from_conservation(m, q, phiB, tau)
        r = swe.minv(m, swe.L(m, q, m.element_traces(lam), phiB, tau))
        ref = np.stack([_eval(e, m.x, m.y) for e in rhs])
        errs.append(np.sqrt(np.mean((r - ref) ** 2)) / np.sqrt(np.mean(ref ** 2)))
    rates = [math.log2(errs[i] / errs[i + 1]) for i in range(2)]
    assert min(rates) > k - 0.3, (errs, rates)


@pytest.mark.parametrize("k", [2, 3])
def test_continuous_state_gives_strong_form(k):
    """Summation by parts of GLL collocation: for a state continuous across faces the weak
    form equals minus the nodal derivative of the nodal flux, exactly up to round-off."""
    ex = _smooth_fields()
    m = swe.Mesh(4, k)
    q, phiB = _state(m, ex)
    Fx, Fy = swe.flux_nonlinear(q, phiB)
    strong = np.zeros_like(q)
    for c in range(3):
        dx, _ = swe.nodal_gradient(m, Fx[c])
        _, dy = swe.nodal_gradient(m, Fy[c])
        strong[c] = -(dx + dy)
    np.testing.assert_allclose(swe.minv(m, swe.NL(m, q, phiB)), strong, atol=1e-12)


def test_lake_at_rest_residuals_vanish_exactly():
    m = swe.Mesh(4, 3)
    phiB = 1.0 + 0.1 * np.sin(2 * np.pi * m.x) * np.sin(2 * np.pi * m.y)
    q = np.zeros((3,) + m.x.shape)
    tau = m.face_tau_hat(phiB)
    assert np.all(swe.NL(m, q, phiB) == 0.0)
    lam = np.zeros((m.n_edges, 3, m.P))
    assert np.all(swe.L(m, q, m.element_traces(lam), phiB, tau) == 0.0)


def test_free_stream_preserved():
    """Uniform state over a flat bottom: both residuals vanish to round-off."""
    m = swe.Mesh(3, 3)
    phiB = np.full(m.x.shape, 1.3)
    q = np.stack([np.full(m.x.shape, 0.02), np.full(m.x.shape, 0.07), np.full(m.x.shape, -0.04)])
    tau = m.face_tau_hat(phiB)
    assert np.abs(swe.minv(m, swe.NL(m, q, phiB))).max() < 1e-13
    lam = swe.trace_from_conservation(m, q, phiB, tau)
    assert np.abs(swe.minv(m, swe.L(m, q, m.element_traces(lam), phiB, tau))).max() < 1e-13


def test_conservation_of_mass_and_momentum():
    """Discontinuous random state: sum over the mesh of the weak residual is zero for mass
    (any bottom) and momentum (flat bottom), i.e. the face fluxes are single valued."""
    m = swe.Mesh(4, 2)
    q = 0.02 * rng.standard_normal((3,) + m.x.shape)
    for phiB in (np.ones(m.x.shape), 1 + 0.1 * np.sin(2 * np.pi * m.x) * np.sin(2 * np.pi * m.y)):
        r = swe.NL(m, q, phiB)
        assert abs(r[0].sum()) < 1e-15
        tau = m.face_tau_hat(phiB)
        lam = swe.trace_from_conservation(m, q, phiB, tau)
        rl = swe.L(m, q, m.element_traces(lam), phiB, tau)
        assert abs(rl[0].sum()) < 1e-15
    phiB = np.ones(m.x.shape)
    r = swe.NL(m, q, phiB)
    assert abs(r[1].sum()) < 1e-15 and abs(r[2].sum()) < 1e-15


def test_hybridised_flux_equals_linear_rusanov():
    """Footnote of Sec. 4.3: on a polygonal mesh, Fhat_L . n evaluated at the conserving trace
    equals the linear Rusanov flux {F_L} . n + tau_L*/2 (q^- - q^+), face by face."""
    m = swe.Mesh(3, 3)
    q = 0.05 * rng.standard_normal((3,) + m.x.shape)
    phiB = 1 + 0.2 * rng.uniform(size=m.x.shape)
    tau = m.face_tau_hat(phiB)
    lam_e = m.element_traces(swe.trace_from_conservation(m, q, phiB, tau))
    for f in range(4):
        n = swe.FACE_NORMALS[f]
        qm, qp = m.face_values(q, f), m.neighbour_face_values(q, f)
        bm, bp = m.face_values(phiB, f), m.neighbour_face_values(phiB, f)
        hyb = swe.hdg_normal_flux(qm, lam_e[:, :, f, :], bm, tau[:, f, :], n)
        Lxm, Lym = swe.flux_linear(qm, bm)
        Lxp, Lyp = swe.flux_linear(qp, bp)
        rus = 0.5 * ((Lxm + Lxp) * n[0] + (Lym + Lyp) * n[1]) + 0.5 * tau[:, f, :] * (qm - qp)
        # equal where phi_B is continuous across the face (the momentum rows carry phi_B^-)
        cont = np.isclose(bm, bp)
        np.testing.assert_allclose(hyb[0], rus[0], atol=1e-15)
        np.testing.assert_allclose(np.where(cont, hyb[1:], 0), np.where(cont, rus[1:], 0), atol=1e-15)


def test_conserving_trace_closed_form():
    """qhat = avg(q) + jump terms / (2 tau): phi_hat = (phi^- + phi^+)/2 + n.(U^- - U^+)/(2 tau),
    U_hat = (U^- + U^+)/2 + n phi_B (phi^- - phi^+)/(2 tau) (phi_B continuous)."""
    m = swe.Mesh(3, 2)
    q = 0.05 * rng.standard_normal((3,) + m.x.shape)
    phiB = np.full(m.x.shape, 1.7)
    tau = m.face_tau_hat(phiB)
    lam_e = m.element_traces(swe.trace_from_conservation(m, q, phiB, tau))
    t = math.sqrt(1.7)
    for f in range(4):
        n = swe.FACE_NORMALS[f]
        qm, qp = m.face_values(q, f), m.neighbour_face_values(q, f)
        ph = 0.5 * (qm[0] + qp[0]) + (n[0] * (qm[1] - qp[1]) + n[1] * (qm[2] - qp[2])) / (2 * t)
        U = 0.5 * (qm[1] + qp[1]) + n[0] * 1.7 * (qm[0] - qp[0]) / (2 * t)
        V = 0.5 * (qm[2] + qp[2]) + n[1] * 1.7 * (qm[0] - qp[0]) / (2 * t)
        np.testing.assert_allclose(lam_e[:, :, f, :], np.stack([ph, U, V]), atol=1e-15)


def test_boundary_conversion_roundtrip():
    m = swe.Mesh(2, 2)
    h = 1 + 0.1 * rng.uniform(size=(m.n_el, 9))
    hu, hv, b = rng.standard_normal((3, m.n_el, 9)) * 0.01
    q, phiB = swe.to_state(h, hu, hv, b, 9.81, 2.0)
    np.testing.assert_allclose(phiB.reshape(m.n_el, 9), 9.81 * (2.0 - b))
    np.testing.assert_allclose(q[0].reshape(m.n_el, 9), 9.81 * (h - 2.0 + b))
    out = swe.from_state(q, phiB, 9.81)
    for a, r in zip(out, (h, hu, hv)):
        np.testing.assert_allclose(a, r, rtol=1e-14, atol=1e-16)


# -- the Rusanov dissipation coefficients, pinned by the flux Jacobian's spectrum ----------------
def _spectral_radius(flux, q, phiB, n):
    """max |lambda| of d(F(q) . n)/dq at every node, F = flux(q, phiB) -> (F_x, F_y) each [3, ...].

    The Jacobian is taken by central differences of the flux function and its eigenvalues by
    numpy.linalg.eigvals, so nothing here restates the wave-speed formula (|u.n| + sqrt(phi)
    for the full flux, sqrt(phi_B) for the linear one) that the oracle writes out.
    """
    q = np.asarray(q, dtype=float)
    shape = q.shape[1:]
    J = np.zeros(shape + (3, 3))
    for c in range(3):
        step = 1e-6 * (1.0 + np.abs(q[c]))
        qp, qm = q.copy(), q.copy()
        qp[c] += step
        qm[c] -= step
        Fxp, Fyp = flux(qp, phiB)
        Fxm, Fym = flux(qm, phiB)
        dF = ((Fxp - Fxm) * n[0] + (Fyp - Fym) * n[1]) / (2.0 * step)   # [3, ...]
        J[..., :, c] = np.moveaxis(dF, 0, -1)
    return np.abs(np.linalg.eigvals(J)).max(axis=-1)


def _discontinuous_state(m, speed):
    """phi_B in [1.5, 3] (so that phi differs from 1), depth perturbations of 0.2 and velocities of
    `speed` that jump across every face (independent nodal noise, no continuity)."""
    r = np.random.Generator(np.random.PCG64(11))
    shape = (m.n_el, m.P, m.P)
    phiB = 1.5 + 1.5 * r.random(shape)
    q = np.stack([0.2 * r.standard_normal(shape),
                  speed * phiB * r.standard_normal(shape),
                  speed * phiB * r.standard_normal(shape)])
    return q, phiB


@pytest.mark.parametrize("f", [0, 1, 2, 3])
def test_rusanov_coefficients_are_the_jacobian_spectral_radii(f):
    """Eq. Full_russanov / Linear_russanov: tau* is the largest |eigenvalue| of the normal flux
    Jacobian over the two sides of the face, and tau_L* the same for the linear flux.  The
    oracle's F*_NL . n minus its central part {F_NL} . n must equal (tau* - tau_L*)/2 (q^- - q^+)
    with both coefficients taken from the numerically computed spectra.  A dissipation
    coefficient that drops |u.n|, forgets to divide U.n by phi, or uses phi_B in place of phi
    moves the result by O(jump) and fails here."""
    m = swe.Mesh(3, 2)
    q, phiB = _discontinuous_state(m, 0.4)
    n = swe.FACE_NORMALS[f]
    qm, qp = m.face_values(q, f), m.neighbour_state(q, f)
    bm, bp = m.face_values(phiB, f), m.neighbour_face_values(phiB, f)
    Fxm, Fym = swe.flux_nonlinear(qm, bm)
    Fxp, Fyp = swe.flux_nonlinear(qp, bp)
    central = 0.5 * ((Fxm + Fxp) * n[0] + (Fym + Fyp) * n[1])
    got = swe.rusanov_nl_normal_flux(m, q, phiB, f) - central
    tau = np.maximum(_spectral_radius(swe.flux_full, qm, bm, n), _spectral_radius(swe.flux_full, qp, bp, n))
    tau_L = np.maximum(_spectral_radius(swe.flux_linear, qm, bm, n), _spectral_radius(swe.flux_linear, qp, bp, n))
    want = 0.5 * (tau - tau_L)[None] * (qm - qp)
    scale = np.abs(want).max()
    assert scale > 0.05                      # the dissipation term is not negligible in this state
    assert np.abs(got - want).max() <= 1e-7 * scale
    # the full flux of the explicit RK DG comparison uses the same tau*
    Fxm, Fym = swe.flux_full(qm, bm)
    Fxp, Fyp = swe.flux_full(qp, bp)
    got_full = swe.rusanov_full_normal_flux(m, q, phiB, f) - 0.5 * ((Fxm + Fxp) * n[0] + (Fym + Fyp) * n[1])
    want_full = 0.5 * tau[None] * (qm - qp)
    assert np.abs(got_full - want_full).max() <= 1e-7 * np.abs(want_full).max()


def test_jacobian_spectrum_of_the_shallow_water_flux():
    """Sanity of the numerical spectrum itself on one state where the textbook answer is known:
    a resting lake (U = V = 0) has normal-flux eigenvalues 0, +-sqrt(phi)."""
    phi_eta, phiB = np.array([0.44]), np.array([2.0])
    q = np.stack([phi_eta, np.zeros(1), np.zeros(1)])
    rho = _spectral_radius(swe.flux_full, q, phiB, np.array([1.0, 0.0]))
    assert abs(rho[0] - math.sqrt(2.44)) <= 1e-8
    rho_L = _spectral_radius(swe.flux_linear, q, phiB, np.array([0.0, 1.0]))
    assert abs(rho_L[0] - math.sqrt(2.0)) <= 1e-8
