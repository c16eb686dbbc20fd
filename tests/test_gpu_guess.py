"""Initial guesses of the trace solve (krylov_guess: the same stage's solutions of the previous
steps extrapolated in time -- constant, linear or quadratic -- or -1, zero): the stop test is
unchanged, so a run matches the oracle as closely as one started from zero, in fewer Krylov
iterations."""
import pytest

pytestmark = pytest.mark.gpu
hd = pytest.importorskip("paper_1711_02751_gb300.hdgdg")
from paper_1711_02751_gb300 import workloads as W  # noqa: E402

from _common import dt_of, oracle_state, user_state  # noqa: E402
from oracle import imex, swe  # noqa: E402


def _run(N, k, kind, steps, guess, precision="fp64", scheme="ars2"):
    m, h, hu, hv, b = user_state(N, k, kind)
    dt = dt_of(m, h, hu, hv)
    with hd.Sim(N, k, dt, bottom=b, g=W.G, H0=W.H0, krylov_guess=guess, precision=precision, scheme=scheme) as s:
        s.set_state(h, hu, hv)
        s.step(steps)
        out = s.get_state()
        st = s.stats()
    return m, h, hu, hv, b, dt, swe.to_state(*out, b, W.G, W.H0)[0], st


@pytest.mark.parametrize("guess,scheme", [(1, "ars2"), (2, "ars2"), (3, "ars2"), (4, "ars2"), (6, "ars2"), (2, "ars3"),
                                          (4, "ars3"), (0, "ars2")])
def test_guess_matches_oracle(guess, scheme):
    m, h, hu, hv, b, dt, qa, st = _run(12, 3, "large", 8, guess, scheme=scheme)
    q, phiB = oracle_state(m, h, hu, hv, b)
    qo = imex.Stepper(m, phiB, dt, scheme=scheme, solver="lu").run(q, 8)
    assert max(imex.rel_l2(m, qa[c], qo[c]) for c in range(3)) <= 1e-10
    _, _, _, _, _, _, _, st0 = _run(12, 3, "large", 8, -1, scheme=scheme)
    assert st["krylov_iterations"] < st0["krylov_iterations"]


def test_guess_restarts_with_set_state():
    """set_state starts a new trajectory: the guess history is dropped, so a second run from the
    same state repeats the first exactly."""
    m, h, hu, hv, b = user_state(8, 2, "large")
    dt = dt_of(m, h, hu, hv)
    with hd.Sim(8, 2, dt, bottom=b, krylov_guess=2) as s:
        s.set_state(h, hu, hv)
        s.step(4)
        a = s.get_state()
        s.set_state(h, hu, hv)
        s.step(4)
        c = s.get_state()
    for x, y in zip(a, c):
        assert (x == y).all()


def test_guess_mixed_within_1e6():
    _, _, _, _, _, _, q1, st1 = _run(16, 3, "large", 20, 2, precision="mixed")
    m, _, _, _, _, _, q0, _ = _run(16, 3, "large", 20, -1, precision="fp64")
    assert max(imex.rel_l2(m, q1[c], q0[c]) for c in range(3)) <= 1e-6


def test_update_state_continues_the_trajectory():
    """update_state replaces the state but keeps time, counters and the guess history: a run
    that is read back and re-entered half-way matches the uninterrupted run to round-off."""
    import numpy as np
    m, h, hu, hv, b = user_state(8, 3, "large")
    dt = dt_of(m, h, hu, hv)
    with hd.Sim(8, 3, dt, bottom=b) as s:
        with pytest.raises(hd.HdgdgError):
            s.update_state(h, hu, hv)              # no trajectory yet
        s.set_state(h, hu, hv)
        s.step(6)
        ref = s.get_state()
        s.set_state(h, hu, hv)
        s.step(3)
        mid = s.get_state()
        s.update_state(*mid)
        s.step(3)
        got = s.get_state()
        st = s.stats()
    assert st["steps"] == 6 and abs(st["time"] - 6 * dt) <= 1e-15
    for a, r in zip(got, ref):
        assert np.abs(a - r).max() <= 1e-12 * max(np.abs(r).max(), 1.0)


def test_single_pass_gram_schmidt_in_the_inner_cycles():
    """krylov_ortho = 1 (classical Gram-Schmidt once in the mixed form's FP32 cycles): the FP64
    refinement keeps the result within 1e-6 of the FP64 form."""
    import numpy as np  # noqa: F401
    m, h, hu, hv, b = user_state(16, 3, "large")
    dt = dt_of(m, h, hu, hv)
    outs = []
    for kw in ({"precision": "mixed", "krylov_ortho": 1}, {"precision": "fp64"}):
        with hd.Sim(16, 3, dt, bottom=b, **kw) as s:
            s.set_state(h, hu, hv)
            s.step(20)
            outs.append(swe.to_state(*s.get_state(), b, W.G, W.H0)[0])
    assert max(imex.rel_l2(m, outs[0][c], outs[1][c]) for c in range(3)) <= 1e-6


def test_fp32_pair_refinement_residual():
    """residual_f32x2: the mixed form's refinement residual in FP64-class arithmetic on the FP32
    pipes (~1e-13 relative) gives the same iteration counts and stays within 1e-6 of the FP64
    form.  Against the mixed form with an FP64 residual the bound is 1e-7: both stop at the
    refinement tolerance 1e-9 per solve, so they differ by that tolerance accumulated over the
    40 stage solves (2.2e-8 measured)."""
    m, h, hu, hv, b = user_state(16, 3, "large")
    dt = dt_of(m, h, hu, hv)
    outs, its = [], []
    for kw in ({"precision": "mixed", "residual_f32x2": True, "local_precision": "f32x2"},
               {"precision": "mixed"}, {"precision": "fp64"}):
        with hd.Sim(16, 3, dt, bottom=b, **kw) as s:
            s.set_state(h, hu, hv)
            s.step(20)
            outs.append(swe.to_state(*s.get_state(), b, W.G, W.H0)[0])
            its.append(s.stats()["krylov_iterations"])
    assert its[0] == its[1]
    assert max(imex.rel_l2(m, outs[0][c], outs[2][c]) for c in range(3)) <= 1e-6
    assert max(imex.rel_l2(m, outs[0][c], outs[1][c]) for c in range(3)) <= 1e-7


@pytest.mark.parametrize("case", ["walls", "vortex", "batch", "k1", "k7"])
def test_bench_mixed_form_across_configurations(case):
    """The mixed form as bench.py and the serving loop run it (FP32 Krylov cycles and DG residual,
    FP32-pair local contractions and refinement residual) against the FP64 form: <= 1e-6 after
    10 steps on walls, prescribed vortex traces, a batch with unequal time steps, k = 1 and k = 7."""
    import numpy as np
    fast = {"precision": "mixed", "local_precision": "f32x2", "residual_f32x2": True}
    kw, N, k, B = {}, 8, 3, 1
    if case == "k1":
        N, k = 16, 1
    if case == "k7":
        N, k = 4, 7
    if case == "vortex":
        V = W.VORTEX
        kw = dict(boundary="vortex", x0=-2.0, length=4.0, g=V["g"], H0=V["H_inf"],
                  bc_params=(V["beta"], V["u_inf"], V["v_inf"], V["xc"], V["yc"]))
        x, y = hd.node_coords(N, k, boundary="vortex", x0=-2.0, length=4.0)
        h, hu, hv, b = W.vortex_state(x, y, 0.0, **V)
        dt = 0.02
    else:
        bnd = "wall" if case == "walls" else "periodic"
        kw = dict(boundary=bnd)
        x, y = hd.node_coords(N, k, boundary=bnd)
        h, hu, hv, b = W.large_state(x, y, seed=21)
        if case == "walls":
            hu, hv = 0.0 * hu, 0.0 * hv
        dt = W.advective_dt(x, h, hu, hv, N)
    if case == "batch":
        B = 3
        kw["batch"], kw["dt_per_instance"] = B, [dt, 0.7 * dt, 0.4 * dt]
        h, hu, hv, b = (np.concatenate([a] * B) for a in (h, hu, hv, b))
    outs = []
    for form in (fast, {"precision": "fp64"}):
        with hd.Sim(N, k, dt, bottom=b, **form, **kw) as s:
            s.set_state(h, hu, hv)
            s.step(10)
            outs.append(s.get_state())
    B0 = (kw.get("H0", W.H0)) - b
    for a, r, base in zip(outs[0], outs[1], (B0, 0.0, 0.0)):
        ra, rr = a - base, r - base
        assert np.linalg.norm(ra - rr) <= 1e-6 * np.linalg.norm(rr)


def test_adaptive_guess_order():
    """Each solve starts from the extrapolation order (<= krylov_guess) or zero whose residual is
    smallest: the order reported stays in range, and on the coarse, under-resolved bump case -- where
    high fixed orders extrapolate the unresolved oscillation and lose to a zero start -- the run
    needs no more Krylov iterations than starting from zero."""
    m, h, hu, hv, b = user_state(12, 3, "large")
    dt = dt_of(m, h, hu, hv)
    its = {}
    for guess in (-1, 6):
        with hd.Sim(12, 3, dt, bottom=b, krylov_guess=guess) as s:
            s.set_state(h, hu, hv)
            orders = []
            for _ in range(8):
                s.step(1)
                orders.append(s.stats()["last_guess_order"])
            its[guess] = s.stats()["krylov_iterations"]
        assert all(0 <= o <= max(guess, 0) for o in orders)
    assert its[6] <= its[-1]


@pytest.mark.parametrize("kw", [dict(local_precision="f32x2", trace_operator=1), dict(local_precision="f32x2")])
def test_least_squares_start_matches_oracle(kw):
    """The least-squares start (krylov_guess_ls): the projection of the trace solution on the affine
    span of the stored solutions, chosen when its residual beats the zero start.  The stop test is
    unchanged, so the mixed form stays within its tolerance of the oracle; each polynomial
    extrapolation is a candidate of the projection, so the solves take no more Krylov iterations
    than from the best polynomial start (two spare for rounding of the FP32 Gram sums)."""
    N, k, steps = 12, 3, 10
    m, h, hu, hv, b = user_state(N, k, "large")
    dt = dt_of(m, h, hu, hv)
    res = {}
    for ls in (False, True):
        with hd.Sim(N, k, dt, bottom=b, g=W.G, H0=W.H0, precision="mixed", krylov_guess_ls=ls, **kw) as s:
            s.set_state(h, hu, hv)
            s.step(steps)
            res[ls] = (swe.to_state(*s.get_state(), b, W.G, W.H0)[0], s.stats())
    q, phiB = oracle_state(m, h, hu, hv, b)
    qo = imex.Stepper(m, phiB, dt, solver="lu").run(q, steps)
    assert max(imex.rel_l2(m, res[True][0][c], qo[c]) for c in range(3)) <= 1e-6
    assert res[True][1]["krylov_iterations"] <= res[False][1]["krylov_iterations"] + 2
    with pytest.raises(hd.HdgdgError):   # the FP64 form keeps the polynomial candidates
        hd.Sim(N, k, dt, bottom=b, g=W.G, H0=W.H0, krylov_guess_ls=True)

