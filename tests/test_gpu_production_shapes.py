"""Whole-step parity with the oracle at the kernels' production launch shapes.

A 64 x 64, k = 3 mesh (4096 elements, 8192 edges) puts every kernel past its small-mesh launch
shapes: the local kernels run hundreds of blocks, the trace SpMV and the Gram-Schmidt / norm
reductions finish over multi-block partials, and the dense tile autotuner's threshold (4096
elements) is reached.  Four steps of the large recipe (variable bottom, bumps, streamfunction
flow) run in the FP64 form and in the benchmark's mixed configuration (FP32 Krylov cycles with
FP32-pair refinement residual and FP32-pair local solves); the stiff variant (gravity Courant
number ~14) runs on 32 x 32.  The oracle's trace solve is its FP64 GMRES to rtol 1e-14 on 64 x 64
(it agrees with the oracle's sparse LU to 5e-14 there; the LU's setup alone takes minutes) and
its LU on 32 x 32.
Bars: FP64 form <= 1e-10, mixed form <= 1e-6 (relative L2 per field; eta = h - B, hu, hv).
"""
import numpy as np
import pytest

from oracle import imex, swe
from paper_1711_02751_gb300 import workloads as W

from _common import oracle_state, user_state

pytestmark = pytest.mark.gpu
hd = pytest.importorskip("paper_1711_02751_gb300.hdgdg")

MIXED = {"assembled_mixed": dict(precision="mixed", local_precision="f32x2", residual_f32x2=True),
         "bench_mixed": dict(precision="mixed", local_precision="f32x2", trace_operator=1)}


def _oracle_run(kind, N, k, steps, solver, **kw):
    m, h, hu, hv, b = user_state(N, k, kind)
    q, phiB = oracle_state(m, h, hu, hv, b)
    floor = W.STIFF_FLOOR if kind == "stiff" else 0.05
    dt = W.advective_dt(m.x.reshape(m.n_el, -1), h, hu, hv, N, floor=floor)
    qo = imex.Stepper(m, phiB, dt, solver=solver, **kw).run(q, steps)
    return m, (h, hu, hv, b), dt, qo


def _gpu_run(m, state, dt, steps, **kw):
    h, hu, hv, b = state
    with hd.Sim(m.N, m.k, dt, bottom=b, g=W.G, H0=W.H0, **kw) as s:
        s.set_state(h, hu, hv)
        s.step(steps)
        out = s.get_state()
        st = s.stats()
    qa, _ = swe.to_state(*out, b, W.G, W.H0)
    return qa, st


@pytest.fixture(scope="module")
def large64():
    return _oracle_run("large", 64, 3, 4, "gmres", rtol=1e-14)


@pytest.fixture(scope="module")
def stiff32():
    return _oracle_run("stiff", 32, 3, 4, "lu")


FORMS = [("fp64", 1e-10), ("assembled_mixed", 1e-6), ("bench_mixed", 1e-6)]


@pytest.mark.parametrize("form,bound", FORMS)
def test_64x64_four_steps_against_the_oracle(large64, form, bound):
    m, state, dt, qo = large64
    kw = MIXED.get(form, {})
    qa, st = _gpu_run(m, state, dt, 4, **kw)
    rel = [imex.rel_l2(m, qa[c], qo[c]) for c in range(3)]
    print(f"64x64 k=3 {form}: rel L2 eta {rel[0]:.2e} hu {rel[1]:.2e} hv {rel[2]:.2e}, "
          f"{st['krylov_iterations'] / 8:.1f} GMRES iterations per stage")
    assert st["steps"] == 4
    assert max(rel) <= bound


@pytest.mark.parametrize("form,bound", FORMS)
def test_stiff_regime_against_the_oracle(stiff32, form, bound):
    """The stiff variant: gravity Courant number ~14 with the explicit part inside its bound."""
    m, state, dt, qo = stiff32
    h, hu, hv, b = state
    dx_min = m.h / 2 * np.diff(m.xi).min()
    assert np.sqrt(W.G * h).max() * dt / dx_min >= 10.0
    kw = MIXED.get(form, {})
    qa, st = _gpu_run(m, state, dt, 4, **kw)
    rel = [imex.rel_l2(m, qa[c], qo[c]) for c in range(3)]
    print(f"stiff 32x32 k=3 {form}: rel L2 eta {rel[0]:.2e} hu {rel[1]:.2e} hv {rel[2]:.2e}, "
          f"{st['krylov_iterations'] / 8:.1f} GMRES iterations per stage")
    assert max(rel) <= bound
