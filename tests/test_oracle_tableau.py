"""Pins of the ARS IMEX-RK tableaux: order conditions and observed order on a split ODE."""
import math

import numpy as np
import pytest
from scipy.integrate import solve_ivp

from oracle.imex import ars2, ars3


def _conditions(A, At, b, bt):
    c, ct = A.sum(1), At.sum(1)
    one = np.ones_like(b)
    return c, ct, one


@pytest.mark.parametrize("scheme,order", [(ars2, 2), (ars3, 3)])
def test_order_conditions(scheme, order):
    A, At, b, bt = scheme()
    c, ct, _ = _conditions(A, At, b, bt)
    np.testing.assert_allclose(c, ct, atol=1e-15)            # same abscissae (c = c~)
    assert np.allclose(np.triu(A), 0.0)                      # explicit part is strictly lower
    assert np.allclose(np.triu(At, 1), 0.0)                  # implicit part is diagonally implicit
    for bb in (b, bt):
        assert abs(bb.sum() - 1.0) < 1e-14
        assert abs(bb @ c - 0.5) < 1e-14
    if order >= 3:
        for bb in (b, bt):
            assert abs(bb @ c ** 2 - 1 / 3) < 1e-14
        for bb in (b, bt):
            for M in (A, At):
                assert abs(bb @ M @ c - 1 / 6) < 1e-14


def test_ars2_constants():
    A, At, b, bt = ars2()
    g = 1 - 1 / math.sqrt(2)
    assert abs(At[1, 1] - g) < 1e-16 and abs(At[2, 2] - g) < 1e-16
    assert abs(A[2, 0] + 2 * math.sqrt(2) / 3) < 1e-15
    np.testing.assert_array_equal(bt, At[-1])                # stiffly accurate implicit part


def test_ars3_stiffly_accurate():
    A, At, b, bt = ars3()
    np.testing.assert_array_equal(b, A[-1])
    np.testing.assert_array_equal(bt, At[-1])
    assert set(np.diag(At)[1:]) == {0.5}


def _imex_scalar(scheme, lam_s, f, y0, T, n):
    """IMEX-RK on y' = f(y) + lam_s y (f explicit, lam_s y implicit)."""
    A, At, b, bt = scheme()
    s = len(b)
    dt = T / n
    y = y0
    for _ in range(n):
        F, G = np.zeros(s), np.zeros(s)
        for i in range(s):
            r = y + dt * sum(A[i, j] * F[j] + At[i, j] * G[j] for j in range(i))
            Y = r / (1 - dt * At[i, i] * lam_s)
            F[i], G[i] = f(Y), lam_s * Y
        y = y + dt * (b @ F + bt @ G)
    return y


@pytest.mark.parametrize("scheme,order", [(ars2, 2), (ars3, 3)])
def test_observed_order_on_split_ode(scheme, order):
    lam_s = -20.0
    f = lambda y: math.sin(y) + 0.5           # noqa: E731
    T, y0 = 1.0, 0.3
    ref = solve_ivp(lambda t, y: f(y[0]) + lam_s * y[0], (0, T), [y0], rtol=1e-13, atol=1e-15,
                    method="DOP853").y[0, -1]
    errs = [abs(_imex_scalar(scheme, lam_s, f, y0, T, n) - ref) for n in (80, 160, 320)]
    rates = [math.log2(errs[i] / errs[i + 1]) for i in range(2)]
    assert min(rates) > order - 0.25, rates
