"""The matrix-free trace operator (trace_operator = 1) against the oracle and the assembled matrix.

S x = D x - C A^{-1} B x is applied element by element (the Schur-complement local solve between
the lift B and the extraction C, each edge row summed from its two elements).  Checks:
* the operator itself (row-level entry point, FP64-class arithmetic) against the oracle's
  assembled condensed matrix, on periodic, walled and prescribed-trace (moving vortex) meshes,
  batches with per-instance time steps, degrees 1..5 and ragged element counts;
* stage solves and whole steps of the mixed form against the oracle (<= 1e-6 per field) and
  against the same form on the assembled matrix;
* bitwise reproducibility: the order in which an edge's two elements finish does not change a
  bit of the result.
"""
import numpy as np
import pytest

from oracle import imex, swe
from paper_1711_02751_gb300 import workloads as W

from _common import dt_of, flat, oracle_state, user_state
from test_oracle_vortex import vortex_problem

pytestmark = pytest.mark.gpu
hd = pytest.importorskip("paper_1711_02751_gb300.hdgdg")
rng = np.random.Generator(np.random.PCG64(4242))

MF = dict(precision="mixed", local_precision="f32x2", trace_operator=1)
ASSEMBLED = dict(precision="mixed", local_precision="f32x2", residual_f32x2=True)


@pytest.mark.parametrize("N,k", [(2, 2), (3, 3), (5, 2), (4, 4), (7, 1), (3, 5)])
def test_operator_matches_oracle_periodic(N, k):
    m, h, hu, hv, b = user_state(N, k, "large")
    q, phiB = oracle_state(m, h, hu, hv, b)
    dt = 0.4 / N
    st = imex.Stepper(m, phiB, dt, solver="dense")
    S = st.cond.S.toarray()
    Wt = np.tile(m.face_jac * m.w, m.n_edges * 3)
    x = rng.standard_normal(m.n_edges * 3 * m.P)
    ref = (S @ x) / Wt                                   # the library's rows are pointwise
    with hd.Sim(N, k, dt, bottom=b, g=W.G, H0=W.H0, **MF) as s:
        got = s.trace_apply(x.reshape(m.n_edges, 3, m.P)).ravel()
        again = s.trace_apply(x.reshape(m.n_edges, 3, m.P)).ravel()
    assert np.abs(got - ref).max() <= 1e-12 * np.abs(ref).max()
    assert np.array_equal(got, again)                    # tickets were left at zero


@pytest.mark.parametrize("N,k", [(3, 2), (4, 3)])
def test_operator_matches_oracle_walls(N, k):
    m = swe.Mesh(N, k, boundary="wall")
    x_, y_ = m.x.reshape(m.n_el, -1), m.y.reshape(m.n_el, -1)
    h, hu, hv, b = W.large_state(x_, y_)
    q, phiB = swe.to_state(h, hu, hv, b, W.G, W.H0)
    dt = 0.3 / N
    st = imex.Stepper(m, phiB, dt, solver="dense")
    S = st.cond.S.toarray()
    Wt = np.tile(m.face_jac * m.w, m.n_edges * 3)
    x = rng.standard_normal(m.n_edges * 3 * m.P)
    ref = (S @ x) / Wt
    with hd.Sim(N, k, dt, bottom=b, g=W.G, H0=W.H0, boundary="wall", **MF) as s:
        got = s.trace_apply(x.reshape(m.n_edges, 3, m.P)).ravel()
    assert np.abs(got - ref).max() <= 1e-12 * np.abs(ref).max()


def test_operator_matches_assembled_on_prescribed_traces():
    """Moving vortex: prescribed boundary rows are the identity; interior rows keep their
    couplings to the prescribed traces.  Same product as the assembled FP64 matrix."""
    m, q, phiB, bc = vortex_problem(4, 3)
    V = W.VORTEX
    kw = dict(bottom=np.zeros((m.n_el, m.P ** 2)), g=V["g"], H0=V["H_inf"], boundary="vortex", x0=-2.0,
              length=4.0, bc_params=(V["beta"], V["u_inf"], V["v_inf"], V["xc"], V["yc"]), scheme="ars3")
    x = rng.standard_normal((m.n_edges, 3, m.P))
    with hd.Sim(4, 3, 0.01, **kw) as s:
        ref = s.trace_apply(x)
    with hd.Sim(4, 3, 0.01, **kw, **MF) as s:
        got = s.trace_apply(x)
    assert np.abs(got - ref).max() <= 1e-12 * np.abs(ref).max()


def test_operator_on_a_batch_with_per_instance_steps():
    N, k, B = 4, 3, 3
    m, h, hu, hv, b = user_state(N, k, "large")
    dts = np.array([0.05, 0.08, 0.11])
    x = rng.standard_normal((B * m.n_edges, 3, m.P))
    bb = np.concatenate([b, 0.5 * b, 0.0 * b])
    with hd.Sim(N, k, 0.11, bottom=bb, g=W.G, H0=W.H0, batch=B, dt_per_instance=dts) as s:
        ref = s.trace_apply(x)
    with hd.Sim(N, k, 0.11, bottom=bb, g=W.G, H0=W.H0, batch=B, dt_per_instance=dts, **MF) as s:
        got = s.trace_apply(x)
    assert np.abs(got - ref).max() <= 1e-12 * np.abs(ref).max()


@pytest.mark.parametrize("N,k,dt", [(8, 2, 0.25), (6, 3, 0.05), (11, 3, 0.02)])
def test_stage_solve_matches_oracle(N, k, dt):
    m, h, hu, hv, b = user_state(N, k, "large" if N != 8 else "bump8")
    q, phiB = oracle_state(m, h, hu, hv, b)
    st = imex.Stepper(m, phiB, dt, solver="lu")
    R1 = q + 0.01 * rng.standard_normal(q.shape)
    Qo, lo = st.cond.solve(R1)
    with hd.Sim(N, k, dt, bottom=b, g=W.G, H0=W.H0, **MF) as s:
        Q, lam, its = s.stage_solve(flat(R1))
    assert its > 0
    for c in range(3):
        assert imex.rel_l2(m, Q[c].reshape(m.x.shape), Qo[c]) <= 1e-8
    assert np.abs(lam - lo).max() <= 1e-8 * np.abs(lo).max()


def _steps(kind, N, k, n, **kw):
    m, h, hu, hv, b = user_state(N, k, kind)
    dt = dt_of(m, h, hu, hv)
    with hd.Sim(N, k, dt, bottom=b, g=W.G, H0=W.H0, **kw) as s:
        s.set_state(h, hu, hv)
        s.step(n)
        out = s.get_state()
    return m, swe.to_state(*out, b, W.G, W.H0)[0], (h, hu, hv, b, dt)


def test_bump8_two_hundred_steps_against_the_oracle():
    m, qa, (h, hu, hv, b, dt) = _steps("bump8", 8, 2, 200, **MF)
    q, phiB = oracle_state(m, h, hu, hv, b)
    qo = imex.Stepper(m, phiB, dt, solver="lu").run(q, 200)
    rel = [imex.rel_l2(m, qa[c], qo[c]) for c in range(3)]
    print(f"bump8 matrix-free mixed, 200 steps: {rel}")
    assert max(rel) <= 1e-6


@pytest.mark.parametrize("N,k,n", [(16, 3, 5), (12, 4, 3), (9, 2, 6)])
def test_matches_the_assembled_route(N, k, n):
    m, qa, _ = _steps("large", N, k, n, **MF)
    _, qb, _ = _steps("large", N, k, n, **ASSEMBLED)
    for c in range(3):
        assert imex.rel_l2(m, qa[c], qb[c]) <= 1e-7


def _steps_its(N, k, n, **kw):
    m, h, hu, hv, b = user_state(N, k, "large")
    dt = dt_of(m, h, hu, hv)
    with hd.Sim(N, k, dt, bottom=b, g=W.G, H0=W.H0, **kw) as s:
        s.set_state(h, hu, hv)
        s.step(n)
        out, its = s.get_state(), s.stats()["krylov_iterations"]
    return m, swe.to_state(*out, b, W.G, W.H0)[0], its


@pytest.mark.parametrize("N,k,n", [(64, 3, 6), (20, 3, 12), (9, 3, 4)])
def test_delayed_gram_schmidt(N, k, n):
    """The matrix-free FP32 cycles run Gram-Schmidt twice with the second pass delayed into the
    next Arnoldi step: the product is taken of the once-projected vector and corrected through
    the Arnoldi relation (A v = (A w1 - V H h2) / hn).  Over several steps, on meshes whose last
    reduction blocks are partial, that needs the inner iterations of Gram-Schmidt twice done in
    place (the assembled route, whose cycles keep it) to within one per stage, and of the single
    pass (krylov_ortho = 1, matrix-free), and the states agree within the solver tolerance."""
    m, q_del, its_del = _steps_its(N, k, n, **MF)
    _, q_in, its_in = _steps_its(N, k, n, **ASSEMBLED)
    _, q_one, its_one = _steps_its(N, k, n, krylov_ortho=1, **MF)
    stages = 2 * n
    print(f"delayed {its_del}, in place {its_in}, single pass {its_one} iterations over {stages} stages")
    assert abs(its_del - its_in) <= stages and abs(its_del - its_one) <= stages
    for c in range(3):
        assert imex.rel_l2(m, q_del[c], q_in[c]) <= 1e-7
        assert imex.rel_l2(m, q_del[c], q_one[c]) <= 1e-7


def test_walls_and_vortex_steps_against_the_oracle():
    m = swe.Mesh(6, 3, boundary="wall")
    x_, y_ = m.x.reshape(m.n_el, -1), m.y.reshape(m.n_el, -1)
    h, hu, hv, b = W.standing_wave_walls_state(x_, y_)
    q, phiB = swe.to_state(h, hu, hv, b, W.G, W.H0)
    qo = imex.Stepper(m, phiB, 0.02, solver="lu").run(q, 5)
    with hd.Sim(6, 3, 0.02, bottom=b, g=W.G, H0=W.H0, boundary="wall", **MF) as s:
        s.set_state(h, hu, hv)
        s.step(5)
        qa = swe.to_state(*s.get_state(), b, W.G, W.H0)[0]
    assert max(imex.rel_l2(m, qa[c], qo[c]) for c in range(3)) <= 1e-6
    m, q, phiB, bc = vortex_problem(4, 2)
    V = W.VORTEX
    qo = imex.Stepper(m, phiB, 0.005, scheme="ars3", solver="lu", bc=bc).run(q, 4)
    user = swe.from_state(q, np.full(m.x.shape, V["g"] * V["H_inf"]), V["g"])
    with hd.Sim(4, 2, 0.005, bottom=np.zeros((m.n_el, 9)), g=V["g"], H0=V["H_inf"], boundary="vortex", x0=-2.0,
                length=4.0, bc_params=(V["beta"], V["u_inf"], V["v_inf"], V["xc"], V["yc"]), scheme="ars3",
                **MF) as s:
        s.set_state(*[a.reshape(m.n_el, -1) for a in user])
        s.step(4)
        out = s.get_state()
    qa = swe.to_state(*out, np.zeros((m.n_el, 9)), V["g"], V["H_inf"])[0]
    assert max(imex.rel_l2(m, qa[c], qo[c]) for c in range(3)) <= 1e-6


def test_bitwise_reproducible():
    outs = []
    for _ in range(2):
        m, qa, _ = _steps("large", 32, 3, 3, **MF)
        outs.append(qa)
    assert np.array_equal(outs[0], outs[1])


def test_autotuned_tiles_change_no_result():
    """On a mesh of >= 4096 elements the element pass's tile and the Schur kernels' tiles are picked
    at create by timing.  Whichever tiles win, the operator matches the assembled FP64 matrix and
    three mixed-form steps stay within the solver tolerance of the assembled route."""
    N, k = 64, 3
    m, h, hu, hv, b = user_state(N, k, "large")
    x = rng.standard_normal((m.n_edges, 3, m.P))
    with hd.Sim(N, k, 0.01, bottom=b, g=W.G, H0=W.H0, **MF) as s:
        st = s.stats()
        assert st["trace_tile"] in (8, 16, 32) and st["trace_tile_prefetch"] in (0, 1)
        assert st["local_tile_condense"] in (8, 16, 32) and st["local_tile_recover"] in (8, 16, 32)
        got = s.trace_apply(x)
        s.set_state(h, hu, hv)
        s.step(3)
        tuned = s.get_state()
    with hd.Sim(N, k, 0.01, bottom=b, g=W.G, H0=W.H0) as s:
        ref = s.trace_apply(x)
    assert np.abs(got - ref).max() <= 1e-12 * np.abs(ref).max()
    with hd.Sim(N, k, 0.01, bottom=b, g=W.G, H0=W.H0, **ASSEMBLED) as s:
        s.set_state(h, hu, hv)
        s.step(3)
        assembled = s.get_state()
    B = W.H0 - b
    for a_, c_ in zip((tuned[0] - B, tuned[1], tuned[2]), (assembled[0] - B, assembled[1], assembled[2])):
        assert np.linalg.norm(a_ - c_) <= 1e-7 * np.linalg.norm(c_)


def test_every_inner_tile_gives_the_same_steps():
    """The inner cycles' element pass in each of its tiles -- blocks of 128, 256 and 512 threads,
    with and without the S^{-1} row loaded ahead into registers, under different register caps --
    gives the same three mixed-form steps bit for bit on a mesh of 4356 elements (N = 66, k = 3),
    whose last block is partial in every tile."""
    N, k = 66, 3
    m, h, hu, hv, b = user_state(N, k, "large")
    results = {}
    with hd.Sim(N, k, 0.01, bottom=b, g=W.G, H0=W.H0, **MF) as s:
        for t in range(9):
            s.set_trace_tile(t)
            st = s.stats()
            assert st["trace_tile_prefetch"] in (0, 1)
            s.set_state(h, hu, hv)
            s.step(3)
            results[t] = s.get_state()
        with pytest.raises(hd.HdgdgError):
            s.set_trace_tile(9)
    for t in range(1, 9):
        for a_, c_ in zip(results[t], results[0]):
            assert np.array_equal(a_, c_), t

