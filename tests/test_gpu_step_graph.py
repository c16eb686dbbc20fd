"""Whole-step CUDA graphs (host_steps = 0, the default) against host-driven steps (host_steps = 1).

A replayed step takes every decision of the trace solve on the device -- the start (zero or the
extrapolation order with the smallest residual), the restart cycles inside a conditional while
node, the stop tests -- in the host driver's order and arithmetic, so the two paths must agree
bit for bit, with the same iteration counts, over enough steps for the initial-guess history to
fill and its buffers to rotate through every cached graph.
"""
import numpy as np
import pytest

from oracle import swe
from paper_1711_02751_gb300 import workloads as W

from _common import dt_of, user_state

pytestmark = pytest.mark.gpu
hd = pytest.importorskip("paper_1711_02751_gb300.hdgdg")

MF = dict(precision="mixed", local_precision="f32x2", trace_operator=1)
ASSEMBLED = dict(precision="mixed", local_precision="f32x2", residual_f32x2=True)


def _run(N, k, kind, steps, host_steps, boundary="periodic", **kw):
    if boundary == "wall":
        m = swe.Mesh(N, k, boundary="wall")
        x, y = m.x.reshape(m.n_el, -1), m.y.reshape(m.n_el, -1)
        h, hu, hv, b = W.standing_wave_walls_state(x, y)
        dt = 0.02
    else:
        m, h, hu, hv, b = user_state(N, k, kind)
        dt = dt_of(m, h, hu, hv)
    with hd.Sim(N, k, dt, bottom=b, g=W.G, H0=W.H0, boundary=boundary, host_steps=host_steps, **kw) as s:
        s.set_state(h, hu, hv)
        guesses = []
        for _ in range(steps):
            s.step(1)
            guesses.append(s.stats()["last_guess_order"])
        out = s.get_state()
        st = s.stats()
    return out, st, guesses


@pytest.mark.parametrize("name,N,k,kind,steps,kw", [
    ("fp64", 16, 3, "large", 9, {}),
    ("mixed_assembled", 16, 3, "large", 9, ASSEMBLED),
    ("mixed_matrix_free", 16, 3, "large", 9, MF),
    ("mixed_fp64_local", 12, 2, "large", 7, dict(precision="mixed")),
    ("ars3", 10, 3, "large", 7, dict(scheme="ars3")),
    ("linear_only", 8, 3, "standing", 6, dict(linear_only=True)),
    ("bump8_stiff_guess3", 8, 2, "bump8", 8, dict(krylov_guess=3)),
    ("mixed_matrix_free_ls", 16, 3, "large", 9, dict(MF, krylov_guess_ls=True)),
    ("mixed_assembled_ls_guess2", 12, 3, "large", 7, dict(ASSEMBLED, krylov_guess_ls=True, krylov_guess=2)),
])
def test_graph_steps_equal_host_driven_steps(name, N, k, kind, steps, kw):
    a, sa, ga = _run(N, k, kind, steps, False, **kw)
    b, sb, gb = _run(N, k, kind, steps, True, **kw)
    for x, y in zip(a, b):
        assert np.array_equal(x, y), name
    assert sa["krylov_iterations"] == sb["krylov_iterations"] > 0
    assert sa["last_krylov_iterations"] == sb["last_krylov_iterations"]
    assert sa["last_rel_residual"] == sb["last_rel_residual"]
    assert ga == gb
    assert sa["steps"] == sb["steps"] == steps
    assert sa["kernel_launches"] > 0


def test_graph_steps_on_walls_and_batches():
    a, sa, _ = _run(6, 3, None, 6, False, boundary="wall", **MF)
    b, sb, _ = _run(6, 3, None, 6, True, boundary="wall", **MF)
    for x, y in zip(a, b):
        assert np.array_equal(x, y)
    N, k, B = 8, 3, 3
    m, h, hu, hv, b0 = user_state(N, k, "large")
    dts = np.array([0.01, 0.015, 0.02])
    outs = []
    for host in (False, True):
        with hd.Sim(N, k, 0.02, bottom=np.concatenate([b0, 0.5 * b0, 0 * b0]), batch=B, dt_per_instance=dts,
                    host_steps=host, **MF) as s:
            s.set_state(*[np.concatenate([v] * B) for v in (h, hu, hv)])
            s.step(6)
            outs.append(s.get_state())
    for x, y in zip(*outs):
        assert np.array_equal(x, y)


def test_graph_step_after_set_state_and_checkpoint():
    """set_state drops the solver history (new cached graphs with shorter histories); a checkpoint
    restores it; both continue exactly as the uninterrupted run."""
    m, h, hu, hv, b = user_state(12, 3, "large")
    dt = dt_of(m, h, hu, hv)
    with hd.Sim(12, 3, dt, bottom=b, **MF) as s:
        s.set_state(h, hu, hv)
        s.step(4)
        ck = s.save_checkpoint()
        s.step(5)
        ref = s.get_state()
        s.set_state(h, hu, hv)
        s.step(4)
        s.load_checkpoint(ck)
        s.step(5)
        again = s.get_state()
    for x, y in zip(ref, again):
        assert np.array_equal(x, y)
