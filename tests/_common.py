"""Shared set-up for tests: seeded workloads evaluated on the oracle's node coordinates."""
import numpy as np

from oracle import imex, swe
from paper_1711_02751_gb300 import workloads as W


def user_state(N, k, kind):
    """(mesh, h, hu, hv, b) of a named workload on the oracle's GLL nodes, arrays [n_el, Np]."""
    m = swe.Mesh(N, k)
    x, y = m.x.reshape(m.n_el, -1), m.y.reshape(m.n_el, -1)
    h, hu, hv, b = W.make_state(kind, x, y)
    return m, h, hu, hv, b


def oracle_state(m, h, hu, hv, b):
    return swe.to_state(h, hu, hv, b, W.G, W.H0)


def flat(q):
    """Oracle [3, e, j, i] -> library [3, e, Np]."""
    return q.reshape(3, q.shape[1], -1)


def rel_l2_fields(m, a, o):
    """Relative L2 of (eta, hu, hv) between two (h, hu, hv) triples [e, Np]; eta = h - B."""
    out = []
    for c in range(3):
        out.append(imex.rel_l2(m, a[c].reshape(m.x.shape), o[c].reshape(m.x.shape)))
    return out


def dt_of(m, h, hu, hv):
    return W.advective_dt(m.x.reshape(m.n_el, -1), h, hu, hv, m.N)
