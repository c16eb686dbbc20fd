"""Uneven ensembles: members of different mesh sizes and degrees advanced together, every
geometry-dependent kernel of a step one persistent launch over all (N, k) groups.

Each member must match its lone run (the same mixed form on a single handle) to the solver
tolerance -- the ensemble's trace systems are solved together as one block-diagonal system, so
the stop test sees the whole ensemble's residual -- and one member is checked against the oracle.
"""
import numpy as np
import pytest

from oracle import imex, swe
from paper_1711_02751_gb300 import workloads as W

from _common import oracle_state, user_state

pytestmark = pytest.mark.gpu
hd = pytest.importorskip("paper_1711_02751_gb300.hdgdg")

MF = dict(precision="mixed", local_precision="f32x2", trace_operator=1)
MEMBERS = [(8, 2, "large"), (12, 3, "large"), (8, 2, "bump8"), (6, 4, "large"), (16, 3, "large"), (12, 3, "standing")]


def _member(N, k, kind):
    m, h, hu, hv, b = user_state(N, k, kind)
    dt = W.advective_dt(m.x.reshape(m.n_el, -1), h, hu, hv, N) if kind != "standing" else 0.01
    return m, h, hu, hv, b, dt


def _rel(a, b, B):
    out = []
    for x, y in ((a[0] - B, b[0] - B), (a[1], b[1]), (a[2], b[2])):
        den = np.linalg.norm(y)
        out.append(np.linalg.norm(x - y) / den if den > 0 else np.linalg.norm(x))
    return out


def test_members_match_their_lone_runs():
    data = [_member(*mk) for mk in MEMBERS]
    steps = 5
    with hd.Ensemble([d[0].N for d in data], [d[0].k for d in data], [d[5] for d in data],
                     bottoms=[d[4] for d in data], g=W.G, H0=W.H0) as ens:
        for i, d in enumerate(data):
            ens.set_state(i, d[1], d[2], d[3])
        ens.step(steps)
        st = ens.stats()
        outs = [ens.get_state(i) for i in range(len(data))]
    assert st["steps"] == steps and st["krylov_iterations"] > 0 and st["kernel_launches"] > 0
    for (m, h, hu, hv, b, dt), got in zip(data, outs):
        with hd.Sim(m.N, m.k, dt, bottom=b, g=W.G, H0=W.H0, **MF) as s:
            s.set_state(h, hu, hv)
            s.step(steps)
            ref = s.get_state()
        rel = _rel(got, ref, W.H0 - b)
        print(f"member N={m.N} k={m.k}: rel to lone run {rel}")
        assert max(rel) <= 1e-6


def test_member_against_the_oracle():
    data = [_member(*mk) for mk in MEMBERS[:4]]
    with hd.Ensemble([d[0].N for d in data], [d[0].k for d in data], [d[5] for d in data],
                     bottoms=[d[4] for d in data], g=W.G, H0=W.H0) as ens:
        for i, d in enumerate(data):
            ens.set_state(i, d[1], d[2], d[3])
        ens.step(3)
        got = ens.get_state(1)
    m, h, hu, hv, b, dt = data[1]
    q, phiB = oracle_state(m, h, hu, hv, b)
    qo = imex.Stepper(m, phiB, dt, solver="lu").run(q, 3)
    qa, _ = swe.to_state(*got, b, W.G, W.H0)
    assert max(imex.rel_l2(m, qa[c], qo[c]) for c in range(3)) <= 1e-6


def test_ensemble_rejects_unsupported_configurations():
    with pytest.raises(hd.HdgdgError) as ei:
        hd.Ensemble([8, 8], [1, 2], [0.01, 0.01])          # k = 1 is outside the ensemble kernels' degrees
    assert ei.value.status == hd.EINVAL
