"""Gauss-Lobatto-Legendre (GLL) collocation tables -- oracle (test infrastructure only).

The spatial discretisation (Sec. 4.2, eq. WeakForm_DG / WeakForm_HDG) uses a nodal
tensor-product basis on each quadrilateral.  The paper does not fix the quadrature;
the reading taken here is collocated GLL quadrature of degree k (k+1 points per
direction), the standard nodal-DG choice of the works the paper cites for its DG
discretisation.  This module is the textbook definition:

* nodes: -1, +1 and the k-1 roots of P_k'(x) (P_k the Legendre polynomial);
* weights: w_i = 2 / (k (k+1) P_k(x_i)^2);
* derivative matrix D[i, j] = l_j'(x_i) of the Lagrange basis l_j on the nodes,
  from barycentric weights.
"""
import numpy as np
from numpy.polynomial import legendre as _leg


def gll_nodes_weights(k):
    """Return (nodes, weights) of the (k+1)-point GLL rule on [-1, 1], ascending."""
    if k < 1:
        raise ValueError("GLL rule needs degree k >= 1")
    Pk = _leg.Legendre.basis(k)
    interior = np.sort(np.real(Pk.deriv().roots())) if k > 1 else np.zeros(0)
    x = np.concatenate(([-1.0], interior, [1.0]))
    # Polish the interior roots with Newton on P_k' (roots() is an eigenvalue solve).
    dP, d2P = Pk.deriv(), Pk.deriv(2)
    for _ in range(3):
        x[1:-1] -= dP(x[1:-1]) / d2P(x[1:-1])
    w = 2.0 / (k * (k + 1) * Pk(x) ** 2)
    return x, w


def lagrange_derivative_matrix(x):
    """D[i, j] = d/dx l_j (x_i) for the Lagrange basis on nodes x (barycentric form)."""
    n = len(x)
    lam = np.array([1.0 / np.prod([x[j] - x[m] for m in range(n) if m != j]) for j in range(n)])
    D = np.zeros((n, n))
    for i in range(n):
        for j in range(n):
            if i != j:
                D[i, j] = (lam[j] / lam[i]) / (x[i] - x[j])
        D[i, i] = -np.sum(D[i, :])   # the derivative of the constant 1 = sum_j l_j is zero
    return D


def lagrange_eval(x, j, t):
    """Plain product formula of the j-th Lagrange basis polynomial on nodes x at points t."""
    t = np.asarray(t, dtype=float)
    out = np.ones_like(t)
    for m in range(len(x)):
        if m != j:
            out = out * (t - x[m]) / (x[j] - x[m])
    return out
