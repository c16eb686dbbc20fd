"""Local solves through the Schur complement on phi (local_dense = 0, the default) against the
dense per-element A^{-1} (local_dense = 1) and the oracle.

With collocated GLL nodes the velocity blocks of the element operator A are diagonal, so the
condensation Z = A^{-1} R1 and the recovery A^{-1}(tau qhat) (eq. linearizedHDGsystem_schur,
recover_volume_unknowns) can eliminate U and V node by node and keep only the (phi, phi) block of
A^{-1}.  Both routes compute the same A^{-1} x; they differ only by rounding.  A dropped coupling
term, a transposed derivative or a wrong boundary diagonal would be O(1) off, and the cases cover
k = 1 ... 8 (one to 64 elements per block, ragged tails), walls, prescribed vortex traces and
batches with per-instance time steps.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu
hd = pytest.importorskip("paper_1711_02751_gb300.hdgdg")
from paper_1711_02751_gb300 import workloads as W  # noqa: E402

from _common import flat, oracle_state, user_state  # noqa: E402
from oracle import imex  # noqa: E402

rng = np.random.Generator(np.random.PCG64(1711))


def _rows(N, k, dt, R1, b, **kw):
    with hd.Sim(N, k, dt, bottom=b, g=W.G, H0=W.H0, **kw) as s:
        g = s.condense_rhs(R1)
        Q, lam, its = s.stage_solve(R1)
    return g, Q, lam


def _close(a, b, tol):
    return np.abs(a - b).max() <= tol * max(np.abs(b).max(), 1e-300)


@pytest.mark.parametrize("N,k", [(6, 1), (5, 3), (7, 2), (3, 5), (2, 7), (2, 8), (17, 3)])
@pytest.mark.parametrize("local", ["fp64", "f32x2"])
def test_schur_rows_equal_dense_rows(N, k, local):
    """Condensation right-hand side and a whole stage solve, Schur route vs dense A^{-1}."""
    m, h, hu, hv, b = user_state(N, k, "large")
    q, _ = oracle_state(m, h, hu, hv, b)
    R1 = flat(q + 0.01 * rng.standard_normal(q.shape))
    dt = 0.4 / N
    gs, Qs, ls = _rows(N, k, dt, R1, b, local_precision=local)
    gd, Qd, ld = _rows(N, k, dt, R1, b, local_precision=local, local_dense=True)
    tol = 1e-13 if local == "fp64" else 1e-12
    assert _close(gs, gd, tol)
    assert _close(Qs, Qd, tol)
    assert _close(ls, ld, tol)


@pytest.mark.parametrize("N,k,dt", [(4, 3, 0.1), (5, 2, 0.05), (3, 4, 0.1)])
@pytest.mark.parametrize("local", ["fp64", "f32x2"])
def test_schur_stage_solve_matches_oracle(N, k, dt, local):
    """The Schur route's stage solve against the oracle's dense local solves."""
    m, h, hu, hv, b = user_state(N, k, "large")
    q, phiB = oracle_state(m, h, hu, hv, b)
    R1 = q + 0.01 * rng.standard_normal(q.shape)
    Qo, lo = imex.Stepper(m, phiB, dt, solver="lu").cond.solve(R1)
    with hd.Sim(N, k, dt, bottom=b, g=W.G, H0=W.H0, local_precision=local) as s:
        Q, lam, its = s.stage_solve(flat(R1))
    for c in range(3):
        assert imex.rel_l2(m, Q[c].reshape(m.x.shape), Qo[c]) <= 1e-11
    assert np.abs(lam - lo).max() <= 1e-10 * np.abs(lo).max()


def _steps(N, k, steps, boundary, **kw):
    x, y = hd.node_coords(N, k, boundary=boundary)
    h, hu, hv, b = W.large_state(x, y, seed=21, n_bumps=2, umax=0.05)
    if boundary != "periodic":
        hu, hv = 0.0 * hu, 0.0 * hv
    dt = 0.5 * W.advective_dt(x, h, hu, hv, N)
    out = {}
    for dense in (False, True):
        with hd.Sim(N, k, dt, bottom=b, g=W.G, H0=W.H0, boundary=boundary, local_dense=dense, **kw) as s:
            s.set_state(h, hu, hv)
            s.step(steps)
            out[dense] = s.get_state()
    return out


@pytest.mark.parametrize("boundary", ["periodic", "wall"])
@pytest.mark.parametrize("kw", [{}, {"precision": "mixed", "local_precision": "f32x2", "residual_f32x2": True},
                                {"scheme": "ars3"}])
def test_schur_steps_equal_dense_steps(boundary, kw):
    out = _steps(10, 3, 6, boundary, **kw)
    tol = 1e-12 if not kw.get("precision") else 1e-7   # mixed: each within its 1e-9 refinement tolerance
    for a, b in zip(out[False], out[True]):
        assert _close(a, b, tol)


def test_schur_vortex_traces_equal_dense():
    """Prescribed exact-solution traces (moving vortex, Sec. 7.1): same steps either way."""
    V = W.VORTEX
    bc = (V["beta"], V["u_inf"], V["v_inf"], V["xc"], V["yc"])
    N, k = 6, 3
    x, y = hd.node_coords(N, k, boundary="vortex", x0=-2.0, length=4.0)
    h, hu, hv, b = W.vortex_state(x, y, 0.0, H_inf=V["H_inf"], u_inf=V["u_inf"], v_inf=V["v_inf"],
                                  beta=V["beta"], g=V["g"], xc=V["xc"], yc=V["yc"])
    out = []
    for dense in (False, True):
        with hd.Sim(N, k, 0.005, bottom=b, g=V["g"], H0=V["H_inf"], boundary="vortex", x0=-2.0, length=4.0,
                    bc_params=bc, scheme="ars3", local_dense=dense) as s:
            s.set_state(h, hu, hv)
            s.step(4)
            out.append(s.get_state())
    for a, b in zip(out[0], out[1]):
        assert _close(a, b, 1e-12)


def test_schur_batch_with_per_instance_time_steps():
    """Each instance's time step scales its own coupling terms and diagonal."""
    N, k, B = 6, 3, 3
    x, y = hd.node_coords(N, k)
    hs, bs = [], []
    for i in range(B):
        h, hu, hv, b = W.large_state(x, y, seed=40 + i, n_bumps=1, umax=0.05)
        hs.append((h, hu, hv))
        bs.append(b)
    dts = np.array([0.01, 0.02, 0.005])
    cat = lambda j: np.concatenate([s[j] for s in hs])  # noqa: E731
    out = []
    for dense in (False, True):
        with hd.Sim(N, k, 0.02, bottom=np.concatenate(bs), g=W.G, H0=W.H0, batch=B, dt_per_instance=dts,
                    local_dense=dense) as s:
            s.set_state(cat(0), cat(1), cat(2))
            s.step(3)
            out.append(s.get_state())
    for a, b in zip(out[0], out[1]):
        assert _close(a, b, 1e-12)


@pytest.mark.parametrize("boundary", ["periodic", "wall"])
@pytest.mark.parametrize("kw", [{}, {"precision": "mixed", "local_precision": "f32x2", "trace_operator": 1}])
def test_every_schur_tile_gives_the_same_steps(boundary, kw):
    """The condensation and recovery kernels in each tile -- 256, 128 and 512 threads, and 128
    threads with the element operators staged in shared memory by bulk asynchronous copies -- give
    the same three steps bit for bit, in the FP64 form (FP64 Schur operators) and in the mixed
    form (FP32-pair operators), on a mesh of 4356 elements (N = 66, k = 3) whose last block is
    partial in every tile."""
    N, k = 66, 3
    m, h, hu, hv, b = user_state(N, k, "large")
    out = {}
    with hd.Sim(N, k, 0.01, bottom=b, g=W.G, H0=W.H0, boundary=boundary, **kw) as s:
        for t in range(4):
            s.set_local_tiles(t, t)
            s.set_state(h, hu, hv)
            s.step(3)
            out[t] = s.get_state()
        with pytest.raises(hd.HdgdgError):
            s.set_local_tiles(4, 0)
    for t in range(1, 4):
        for a_, c_ in zip(out[t], out[0]):
            assert np.array_equal(a_, c_), t
