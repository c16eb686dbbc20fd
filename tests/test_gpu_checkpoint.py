"""Checkpoint / resume: a run checkpointed part-way and continued in a fresh handle (same
configuration and bottom) matches the uninterrupted run bit for bit -- the checkpoint carries
the state, the simulated time, the counters and the trace solve's initial-guess history -- and
checkpoints of other configurations or truncated buffers are rejected."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu
hd = pytest.importorskip("paper_1711_02751_gb300.hdgdg")
from paper_1711_02751_gb300 import workloads as W  # noqa: E402

FAST = {"precision": "mixed", "local_precision": "f32x2", "residual_f32x2": True}


def _setup(case):
    if case == "vortex":
        V = W.VORTEX
        kw = dict(boundary="vortex", x0=-2.0, length=4.0, g=V["g"], H0=V["H_inf"], scheme="ars3",
                  bc_params=(V["beta"], V["u_inf"], V["v_inf"], V["xc"], V["yc"]))
        x, y = hd.node_coords(8, 3, boundary="vortex", x0=-2.0, length=4.0)
        h, hu, hv, b = W.vortex_state(x, y, 0.0, **V)
        return 8, 3, 0.02, (h, hu, hv, b), kw
    x, y = hd.node_coords(12, 3)
    h, hu, hv, b = W.large_state(x, y, seed=5)
    return 12, 3, W.advective_dt(x, h, hu, hv, 12), (h, hu, hv, b), (FAST if case == "mixed" else {})


@pytest.mark.parametrize("case", ["fp64", "mixed", "vortex"])
def test_resume_is_bit_identical(case):
    N, k, dt, (h, hu, hv, b), kw = _setup(case)
    with hd.Sim(N, k, dt, bottom=b, **kw) as s:
        s.set_state(h, hu, hv)
        s.step(8)
        ref, st_ref = s.get_state(), s.stats()
    with hd.Sim(N, k, dt, bottom=b, **kw) as s:
        s.set_state(h, hu, hv)
        s.step(3)
        ck = s.save_checkpoint()
    with hd.Sim(N, k, dt, bottom=b, **kw) as s:      # a fresh handle
        s.load_checkpoint(ck)
        assert s.stats()["steps"] == 3
        s.step(5)
        got, st = s.get_state(), s.stats()
    for a, r in zip(got, ref):
        assert np.array_equal(a, r)
    assert st["steps"] == st_ref["steps"] and st["time"] == st_ref["time"]
    assert st["krylov_iterations"] == st_ref["krylov_iterations"]


def test_checkpoint_rejections():
    N, k, dt, (h, hu, hv, b), kw = _setup("fp64")
    with hd.Sim(N, k, dt, bottom=b) as s:
        with pytest.raises(hd.HdgdgError):
            s.save_checkpoint()                         # no state yet
        s.set_state(h, hu, hv)
        s.step(2)
        ck = s.save_checkpoint()
        with pytest.raises(hd.HdgdgError):
            s.load_checkpoint(ck[:len(ck) // 2])        # truncated
        with pytest.raises(hd.HdgdgError):
            s.load_checkpoint(b"not a checkpoint" * 64)
    with hd.Sim(N, k, 0.5 * dt, bottom=b) as s:         # another time step
        with pytest.raises(hd.HdgdgError):
            s.load_checkpoint(ck)
    with hd.Sim(N, k, dt, bottom=b, precision="mixed") as s:   # another arithmetic
        with pytest.raises(hd.HdgdgError):
            s.load_checkpoint(ck)


def test_batch_checkpoint_checks_the_time_steps():
    x, y = hd.node_coords(8, 2)
    h, hu, hv, b = W.large_state(x, y, seed=3)
    dt = W.advective_dt(x, h, hu, hv, 8)
    cat = lambda a: np.concatenate([a, a])  # noqa: E731
    with hd.Sim(8, 2, dt, bottom=cat(b), batch=2, dt_per_instance=[dt, 0.5 * dt]) as s:
        s.set_state(cat(h), cat(hu), cat(hv))
        s.step(2)
        ck = s.save_checkpoint()
        ref = None
        s.step(2)
        ref = s.get_state()
    with hd.Sim(8, 2, dt, bottom=cat(b), batch=2, dt_per_instance=[0.5 * dt, dt]) as s:
        with pytest.raises(hd.HdgdgError):
            s.load_checkpoint(ck)
    with hd.Sim(8, 2, dt, bottom=cat(b), batch=2, dt_per_instance=[dt, 0.5 * dt]) as s:
        s.load_checkpoint(ck)
        s.step(2)
        for a, r in zip(s.get_state(), ref):
            assert np.array_equal(a, r)
