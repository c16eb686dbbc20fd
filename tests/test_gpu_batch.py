"""Batched handles: B instances of one mesh in one handle (one launch per kernel per stage for
all of them) advance exactly as each instance does alone, with its own bottom, state and time
step; one instance is also checked against the oracle directly."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu
hd = pytest.importorskip("paper_1711_02751_gb300.hdgdg")
from paper_1711_02751_gb300 import workloads as W  # noqa: E402

from _common import oracle_state  # noqa: E402


def _instances(N, k, B, boundary="periodic", seed0=300):
    x, y = hd.node_coords(N, k, boundary=boundary)
    out = []
    for i in range(B):
        h, hu, hv, b = W.large_state(x, y, seed=seed0 + i, n_bumps=1, umax=0.05)
        amp = 0.02 * (i + 1)                       # each instance its own bottom amplitude
        bump, u, v = h - (W.H0 - b), hu / h, hv / h
        b = b * (amp / 0.1)
        h = W.H0 - b + bump
        if boundary != "periodic":                 # at rest against the walls
            u, v = 0.0 * u, 0.0 * v
        out.append((h, h * u, h * v, b, W.advective_dt(x, h, h * u, h * v, N)))
    return out


def _run_alone(N, k, inst, steps, **kw):
    h, hu, hv, b, dt = inst
    with hd.Sim(N, k, dt, bottom=b, **kw) as s:
        s.set_state(h, hu, hv)
        s.step(steps)
        return s.get_state()


def _run_batched(N, k, insts, steps, **kw):
    B = len(insts)
    cat = lambda j: np.concatenate([x[j] for x in insts])  # noqa: E731
    dts = np.array([x[4] for x in insts])
    with hd.Sim(N, k, float(dts.max()), bottom=cat(3), batch=B, dt_per_instance=dts, **kw) as s:
        s.set_state(cat(0), cat(1), cat(2))
        s.step(steps)
        st = s.get_state()
        stats = s.stats()
    n = N * N
    return [tuple(a[i * n:(i + 1) * n] for a in st) for i in range(B)], stats


def _rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


@pytest.mark.parametrize("scheme", ["ars2", "ars3", "rk2"])
def test_batched_fp64_equals_alone(scheme):
    N, k, B, steps = 12, 3, 4, 10
    insts = _instances(N, k, B)
    if scheme == "rk2":                            # explicit: a stable step for every instance
        insts = [x[:4] + (0.05 * x[4],) for x in insts]   # gravity Courant ~0.13
    res, _ = _run_batched(N, k, insts, steps, scheme=scheme)
    for inst, got in zip(insts, res):
        ref = _run_alone(N, k, inst, steps, scheme=scheme)
        for a, b in zip(got, ref):
            assert _rel(a, b) <= 1e-12


def test_batched_time_steps_really_differ():
    N, k = 8, 2
    insts = _instances(N, k, 2)
    insts = [insts[0][:4] + (insts[0][4],), insts[0][:4] + (0.5 * insts[0][4],)]   # same state, dt / 2
    res, _ = _run_batched(N, k, insts, 6)
    assert _rel(res[0][0], res[1][0]) > 1e-6       # different times reached
    for inst, got in zip(insts, res):
        ref = _run_alone(N, k, inst, 6)
        assert _rel(got[0], ref[0]) <= 1e-12


def test_batched_walls_equal_alone():
    N, k, B = 8, 3, 3
    insts = _instances(N, k, B, boundary="wall")
    res, _ = _run_batched(N, k, insts, 8, boundary="wall")
    for inst, got in zip(insts, res):
        ref = _run_alone(N, k, inst, 8, boundary="wall")
        for a, b in zip(got, ref):
            assert _rel(a, b) <= 1e-12 or np.abs(a - b).max() <= 1e-14


def test_batched_mixed_within_1e6_of_fp64():
    N, k, B, steps = 16, 3, 4, 20
    insts = _instances(N, k, B)
    res, stats = _run_batched(N, k, insts, steps, precision="mixed")
    for inst, got in zip(insts, res):
        ref = _run_alone(N, k, inst, steps)
        for a, b in zip(got, ref):
            assert _rel(a, b) <= 1e-6
    assert stats["steps"] == steps


def test_batched_instance_matches_oracle():
    """The last instance of a batch against the FP64 oracle, two ARS2 steps."""
    from oracle import imex, swe
    N, k, B = 6, 3, 3
    insts = _instances(N, k, B)
    res, _ = _run_batched(N, k, insts, 2)
    h, hu, hv, b, dt = insts[-1]
    m = swe.Mesh(N, k)
    q, phiB = oracle_state(m, h, hu, hv, b)
    qn = imex.Stepper(m, phiB, dt, "ars2").run(q, 2)
    ref = swe.from_state(qn, phiB, W.G)
    for a, r in zip(res[-1], ref):
        assert _rel(a, r) <= 1e-11


def test_batched_bytes_and_bad_time_step():
    c1 = hd.make_config(16, 3, 1e-3)
    c4 = hd.make_config(16, 3, 1e-3, batch=4)
    assert hd.bytes_required(c4) > 3 * hd.bytes_required(c1)
    with pytest.raises(hd.HdgdgError):
        hd.Sim(4, 2, 1e-3, batch=2, dt_per_instance=[1e-3, -1e-3])
    with pytest.raises(ValueError):
        hd.make_config(4, 2, 1e-3, batch=3, dt_per_instance=[1e-3, 1e-3])
