"""The delayed second Gram-Schmidt pass of the FP32 inner cycles, in exact-enough arithmetic.

The matrix-free form's Arnoldi step j leaves v_{j+1} = (w1 - V h2) / hn unformed and takes the
next product of w1; the fused pass then forms v_{j+1} and A v_{j+1} = (A w1 - V_{j+2} c) / hn with
c = H h2 over the unrotated Hessenberg columns (the Arnoldi relation A V_{j+1} = V_{j+2} H).  This
restates that sequence in FP64 numpy, step for step as the kernels order it (first-pass dots, the
update with its second-pass dots and hn = sqrt(|w1|^2 - |h2|^2), c, the fused pass), and checks it
against classical Gram-Schmidt twice done in place: the same basis and Hessenberg matrix, an
orthonormal basis, and the Arnoldi relation.  In FP64 the second pass is of rounding size, so the
first pass's dots are also perturbed on purpose (by d_j, the same in both): the second pass then
carries an O(1) correction, and a slip in c or in the fused pass shows at O(1).  No GPU."""
import numpy as np
import pytest


def _in_place(A, r, m, d):
    n = A.shape[0]
    V = np.zeros((n, m + 1))
    H = np.zeros((m + 1, m))
    V[:, 0] = r / np.linalg.norm(r)
    for j in range(m):
        w = A @ V[:, j]
        h1 = V[:, : j + 1].T @ w + d[j][: j + 1]
        w1 = w - V[:, : j + 1] @ h1
        h2 = V[:, : j + 1].T @ w1
        hn = np.sqrt(w1 @ w1 - h2 @ h2)
        H[: j + 1, j] = h1 + h2
        H[j + 1, j] = hn
        V[:, j + 1] = (w1 - V[:, : j + 1] @ h2) / hn
    return V, H


def _delayed(A, r, m, d):
    n = A.shape[0]
    V = np.zeros((n, m + 1))
    H = np.zeros((m + 1, m))
    V[:, 0] = r / np.linalg.norm(r)
    w = A @ V[:, 0]                       # step 0: the product of v_0 and its first-pass dots
    h1 = V[:, :1].T @ w
    for j in range(m):
        h1 = h1 + d[j][: j + 1]
        w1 = w - V[:, : j + 1] @ h1       # the update: w1, second-pass dots, hn, Hessenberg column
        h2 = V[:, : j + 1].T @ w1
        hn = np.sqrt(w1 @ w1 - h2 @ h2)
        H[: j + 1, j] = h1 + h2
        H[j + 1, j] = hn
        c = np.array([sum(H[i, k] * h2[k] for k in range(max(0, i - 1), j + 1)) for i in range(j + 2)])
        if j == m - 1:
            V[:, j + 1] = (w1 - V[:, : j + 1] @ h2) / hn
            break
        z = A @ w1                        # the next product, of w1
        v = (w1 - V[:, : j + 1] @ h2) / hn   # the fused pass: v_{j+1}, A v_{j+1}, next dots
        V[:, j + 1] = v
        w = (z - V[:, : j + 1] @ c[: j + 1] - c[j + 1] * v) / hn
        h1 = V[:, : j + 2].T @ w
    return V, H


@pytest.mark.parametrize("n,m,seed,eps", [(60, 10, 1, 0.0), (200, 10, 2, 0.0), (120, 20, 3, 0.0),
                                          (60, 10, 4, 0.3), (200, 10, 5, 0.3)])
def test_delayed_pass_equals_the_in_place_passes(n, m, seed, eps):
    rng = np.random.default_rng(seed)
    # a nonsymmetric operator with a spread spectrum, like the preconditioned trace system
    A = np.eye(n) + 0.3 * rng.standard_normal((n, n)) / np.sqrt(n) + np.diag(rng.uniform(0.0, 2.0, n))
    r = rng.standard_normal(n)
    d = eps * rng.standard_normal((m, m))
    V0, H0 = _in_place(A, r, m, d)
    V1, H1 = _delayed(A, r, m, d)
    assert np.abs(V1 - V0).max() <= 1e-11
    assert np.abs(H1 - H0).max() <= 1e-11 * np.abs(H0).max()
    assert np.abs(V1.T @ V1 - np.eye(m + 1)).max() <= 1e-13
    assert np.abs(A @ V1[:, :m] - V1 @ H1).max() <= 1e-12 * np.abs(A).max()


def test_the_correction_is_of_the_second_pass_size():
    """c = H h2 is as small as h2 (the second pass's dots, of the size of the first pass's
    rounding): the product of v reached through the Arnoldi relation differs from the direct one
    by rounding alone."""
    rng = np.random.default_rng(7)
    n, m = 150, 10
    A = np.eye(n) + np.diag(rng.uniform(0.0, 3.0, n)) + 0.2 * rng.standard_normal((n, n)) / np.sqrt(n)
    V, H = _in_place(A, rng.standard_normal(n), m, np.zeros((m, m)))
    for j in range(1, m):
        w = A @ V[:, j]
        h1 = V[:, : j + 1].T @ w
        w1 = w - V[:, : j + 1] @ h1
        h2 = V[:, : j + 1].T @ w1
        hn = np.sqrt(w1 @ w1 - h2 @ h2)
        v = (w1 - V[:, : j + 1] @ h2) / hn
        c = H[: j + 2, : j + 1] @ h2
        via = (A @ w1 - V[:, : j + 2] @ c) / hn
        assert np.abs(h2).max() <= 1e-12 * np.linalg.norm(w)
        assert np.abs(via - A @ v).max() <= 1e-12 * np.abs(A @ v).max()
