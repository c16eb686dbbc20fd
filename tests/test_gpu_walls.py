"""Reflecting walls (Sec. 4.3, eq. reflection / eq. reflectionBC) on the GPU against the oracle."""
import numpy as np
import pytest

from oracle import imex, swe
from paper_1711_02751_gb300 import workloads as W

pytestmark = pytest.mark.gpu
hd = pytest.importorskip("paper_1711_02751_gb300.hdgdg")
rng = np.random.Generator(np.random.PCG64(404))


def _walled(N, k, kind="large", x0=0.0, length=1.0, **kw):
    m = swe.Mesh(N, k, boundary="wall", x0=x0, length=length)
    x, y = m.x.reshape(m.n_el, -1), m.y.reshape(m.n_el, -1)
    if kind == "perturbation":
        h, hu, hv, b = W.perturbation_state(x, y, **kw)
    else:
        h, hu, hv, b = W.make_state(kind, x, y)
    q, phiB = swe.to_state(h, hu, hv, b, W.G, W.H0)
    return m, (h, hu, hv, b), q, phiB


def _sim(m, b, dt, **kw):
    return hd.Sim(m.N, m.k, dt, bottom=b, g=W.G, H0=W.H0, boundary="wall", x0=m.x.min(),
                  length=m.h * m.N, **kw)


def _flat(q):
    return q.reshape(3, q.shape[1], -1)


def test_wall_node_coordinates():
    m = swe.Mesh(5, 3, boundary="wall", x0=-1.0, length=2.0)
    x, y = hd.node_coords(5, 3, boundary="wall", x0=-1.0, length=2.0)
    np.testing.assert_allclose(x, m.x.reshape(m.n_el, -1), atol=1e-15)
    np.testing.assert_allclose(y, m.y.reshape(m.n_el, -1), atol=1e-15)


@pytest.mark.parametrize("N,k", [(5, 3), (4, 2), (1, 2), (7, 1)])
def test_wall_eval_nl_matches_oracle(N, k):
    m, (h, hu, hv, b), q, phiB = _walled(N, k)
    q = q + 0.003 * rng.standard_normal(q.shape)
    ref = _flat(swe.minv(m, swe.NL(m, q, phiB)))
    with _sim(m, b, 0.01) as s:
        got = s.eval_nl(_flat(q))
    assert np.abs(got - ref).max() <= 1e-12 * np.abs(ref).max()


@pytest.mark.parametrize("N,k", [(3, 2), (4, 3), (2, 1)])
def test_wall_trace_system_matches_oracle(N, k):
    m, (h, hu, hv, b), q, phiB = _walled(N, k)
    dt = 0.3 / N
    st = imex.Stepper(m, phiB, dt, solver="dense")
    R1 = q + 0.01 * rng.standard_normal(q.shape)
    wgt = (m.face_jac * m.w)[None, None, :]
    ref_g = st.cond.rhs(R1).reshape(m.n_edges, 3, m.P) / wgt
    x = rng.standard_normal(m.n_edges * 3 * m.P)
    ref_y = (st.cond.S.toarray() @ x).reshape(m.n_edges, 3, m.P) / wgt
    Qo, lo = st.cond.solve(R1)
    with _sim(m, b, dt) as s:
        g = s.condense_rhs(_flat(R1))
        y = s.trace_apply(x.reshape(m.n_edges, 3, m.P))
        Q, lam, _ = s.stage_solve(_flat(R1))
    assert np.abs(g - ref_g).max() <= 1e-12 * np.abs(ref_g).max()
    assert np.abs(y - ref_y).max() <= 1e-12 * np.abs(ref_y).max()
    for c in range(3):
        assert imex.rel_l2(m, Q[c].reshape(m.x.shape), Qo[c]) <= 1e-11


@pytest.mark.parametrize("scheme,precision,tol", [("ars2", "fp64", 1e-11), ("ars3", "fp64", 1e-11),
                                                  ("ars2", "mixed", 1e-7), ("rk2", "fp64", 1e-11)])
def test_wall_steps_match_oracle(scheme, precision, tol):
    m, (h, hu, hv, b), q, phiB = _walled(6, 3)
    dt = W.advective_dt(m.x.reshape(m.n_el, -1), h, hu, hv, 6)
    if scheme == "rk2":
        dt *= 0.2
        qo = imex.ExplicitRK(m, phiB, dt, "rk2").run(q, 5)
    else:
        qo = imex.Stepper(m, phiB, dt, scheme=scheme, solver="lu").run(q, 5)
    with _sim(m, b, dt, scheme=scheme, precision=precision) as s:
        s.set_state(h, hu, hv)
        s.step(5)
        qa, _ = swe.to_state(*s.get_state(), b, W.G, W.H0)
    for c in range(3):
        assert imex.rel_l2(m, qa[c], qo[c]) <= tol


def test_walls_conserve_mass_on_gpu():
    m, (h, hu, hv, b), q, phiB = _walled(16, 3)
    with _sim(m, b, 0.005) as s:
        s.set_state(h, hu, hv)
        m0 = s.stats()["mass"]
        s.step(10)
        m1 = s.stats()["mass"]
    assert abs(m1 - m0) <= 1e-12 * abs(m0)


def test_perturbation_in_the_box_is_symmetric():
    """The paper's water-height perturbation (Sec. 7.2) on [-1,1]^2 with walls, H_inf = 100:
    mirror symmetric in x and y after 20 ARS2 steps at gravity Courant ~4."""
    m, (h, hu, hv, b), q, phiB = _walled(10, 3, kind="perturbation", x0=-1.0, length=2.0)
    with _sim(m, b, 0.002) as s:
        s.set_state(h, hu, hv)
        s.step(20)
        qa, _ = swe.to_state(*s.get_state(), b, W.G, W.H0)
    g = qa.reshape(3, 10, 10, 4, 4)
    gx = g[:, :, ::-1, :, ::-1]
    scale = np.abs(g[0]).max()
    assert np.abs(g[0] - gx[0]).max() <= 1e-10 * scale


@pytest.mark.parametrize("k", [6, 8])
def test_high_degree_walls_match_oracle(k):
    """k = 6 and 8 (the local inverses built in a global workspace): DG residual, one implicit
    stage and two whole steps against the oracle on a 3 x 3 walled box."""
    m, (h, hu, hv, b), q, phiB = _walled(3, k, kind="perturbation", x0=-1.0, length=2.0, H_inf=1.0,
                                         sigma=0.4)
    dt = 0.01
    st = imex.Stepper(m, phiB, dt, solver="dense")
    R1 = q + 0.001 * rng.standard_normal(q.shape)
    Qo, _ = st.cond.solve(R1)
    qo = st.run(q, 2)
    ref_nl = _flat(swe.minv(m, swe.NL(m, R1, phiB)))
    with _sim(m, b, dt) as s:
        nl = s.eval_nl(_flat(R1))
        Q, _, _ = s.stage_solve(_flat(R1))
        s.set_state(h, hu, hv)
        s.step(2)
        qa, _ = swe.to_state(*s.get_state(), b, W.G, W.H0)
    assert np.abs(nl - ref_nl).max() <= 1e-11 * np.abs(ref_nl).max()
    for c in range(3):
        assert imex.rel_l2(m, Q[c].reshape(m.x.shape), Qo[c]) <= 1e-10
        assert imex.rel_l2(m, qa[c], qo[c]) <= 1e-10
