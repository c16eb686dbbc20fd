"""Precision variants of the local contractions -- condensation Z = A^{-1} R1 and recovery
A^{-1}(tau qhat) (eq. linearizedHDGsystem_schur, recover_volume_unknowns):

* local_precision='fp32': per-element FP32 copies of A^{-1}, FP32 products and sums;
* local_precision='bf16': one operator shared by all elements (flat bottom), applied to all
  elements as one product on the tensor cores with BF16 inputs and FP32 accumulation.

The tensor-core product is checked sharply against a host emulation of the same arithmetic:
the oracle's A^{-1} and the inputs rounded to BF16 (round to nearest even, 8 significant bits),
exact products and sums (the device's FP32 accumulation adds ~1e-7 relative).  A wrong tile
layout, a transposed operator or a misplaced row would be O(1) off; the BF16 rounding itself is
~1e-3, so each test also checks that it really differs from the FP64 path by that much.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu
hd = pytest.importorskip("paper_1711_02751_gb300.hdgdg")
from paper_1711_02751_gb300 import workloads as W  # noqa: E402

from _common import dt_of, flat, oracle_state, user_state  # noqa: E402
from oracle import imex, swe  # noqa: E402

rng = np.random.Generator(np.random.PCG64(77))


def bf16(x):
    """Round FP64 values to BF16 (8 significant bits, nearest even)."""
    m, e = np.frexp(np.asarray(x, dtype=np.float64))
    return np.ldexp(np.rint(m * 256.0) / 256.0, e)


def _flat_case(N, k):
    """The 8x8 bump recipe (flat bottom) on an N x N mesh, with a small seeded velocity."""
    m = swe.Mesh(N, k)
    x, y = m.x.reshape(m.n_el, -1), m.y.reshape(m.n_el, -1)
    h, hu, hv, b = W.make_state("bump8", x, y)
    hu = hu + 0.01 * np.sin(2 * np.pi * y)
    hv = hv + 0.01 * np.cos(2 * np.pi * x)
    return m, h, hu, hv, b


def _elem(u):
    """[3, e, ...] -> [e, 3 * ...]"""
    return np.moveaxis(np.asarray(u), 1, 0).reshape(np.shape(u)[1], -1)


@pytest.mark.parametrize("N,k", [(6, 3), (12, 2), (5, 1), (4, 4), (17, 3)])
def test_tensor_core_condensation_matches_bf16_emulation(N, k):
    m, h, hu, hv, b = _flat_case(N, k)
    q, phiB = oracle_state(m, h, hu, hv, b)
    dt = 0.4 / N
    st = imex.Stepper(m, phiB, dt, solver="dense")
    R1 = q + 0.01 * rng.standard_normal(q.shape)
    Ainv, C = st.cond.Ainv, st.cond.C
    Zb = np.einsum("evw,ew->ev", bf16(Ainv), bf16(_elem(R1)))          # emulated tensor-core product
    loc = -np.einsum("etv,ev->et", C, Zb)
    ref = np.bincount(st.cond.gi.ravel(), weights=loc.ravel(), minlength=st.cond.n)
    ref = ref.reshape(m.n_edges, 3, m.P) / (m.face_jac * m.w)[None, None, :]
    with hd.Sim(N, k, dt, bottom=b, g=W.G, H0=W.H0, local_precision="bf16") as s:
        got = s.condense_rhs(flat(R1))
    with hd.Sim(N, k, dt, bottom=b, g=W.G, H0=W.H0) as s:
        g64 = s.condense_rhs(flat(R1))
    scale = np.abs(ref).max()
    err = np.abs(got - ref).max()
    assert err <= 2e-6 * scale
    assert np.abs(g64 - ref).max() >= 20 * max(err, 1e-300)   # the BF16 rounding is really there


@pytest.mark.parametrize("N,k", [(6, 3), (12, 2), (4, 4)])
def test_tensor_core_recovery_matches_bf16_emulation(N, k):
    """Q = Z + beta A^{-1}(tau qhat) from the library's own stage solve (its qhat), emulated on
    the host from the oracle's A^{-1} and B (B qhat = -beta tau qhat on the boundary nodes,
    beta = dt a_ii (2/h)/w_0)."""
    m, h, hu, hv, b = _flat_case(N, k)
    q, phiB = oracle_state(m, h, hu, hv, b)
    dt = 0.4 / N
    st = imex.Stepper(m, phiB, dt, solver="dense")
    R1 = q + 0.01 * rng.standard_normal(q.shape)
    with hd.Sim(N, k, dt, bottom=b, g=W.G, H0=W.H0, local_precision="bf16") as s:
        Q, lam, _ = s.stage_solve(flat(R1))
    Ainv, B = st.cond.Ainv, st.cond.B
    lam_loc = lam.ravel()[st.cond.gi]
    v = -np.einsum("evt,et->ev", B, lam_loc)                          # = beta * tau qhat (gathered)
    w0 = 2.0 / (k * (k + 1))
    beta = dt * st.a_ii * (2.0 * N) / w0
    Zb = np.einsum("evw,ew->ev", bf16(Ainv), bf16(_elem(R1)))
    Qb = Zb + beta * np.einsum("evw,ew->ev", bf16(Ainv), bf16(v / beta))
    Q64 = np.einsum("evw,ew->ev", Ainv, _elem(R1) + v)
    got = _elem(Q)
    scale = np.abs(Qb).max()
    err = np.abs(got - Qb).max()
    assert err <= 2e-6 * scale
    assert np.abs(Q64 - Qb).max() >= 20 * max(err, 1e-300)


@pytest.mark.parametrize("N,k", [(6, 3), (9, 2)])
def test_fp32_local_operators_match_fp64_to_fp32_rounding(N, k):
    m, h, hu, hv, b = user_state(N, k, "large")      # variable bottom: per-element operators
    q, phiB = oracle_state(m, h, hu, hv, b)
    dt = 0.4 / N
    R1 = q + 0.01 * rng.standard_normal(q.shape)
    with hd.Sim(N, k, dt, bottom=b, g=W.G, H0=W.H0, local_precision="fp32") as s:
        g32 = s.condense_rhs(flat(R1))
        Q32, lam32, _ = s.stage_solve(flat(R1))
    with hd.Sim(N, k, dt, bottom=b, g=W.G, H0=W.H0) as s:
        g64 = s.condense_rhs(flat(R1))
        Q64, lam64, _ = s.stage_solve(flat(R1))
    d = np.abs(g32 - g64).max() / np.abs(g64).max()
    assert 1e-10 < d <= 1e-5
    assert np.abs(Q32 - Q64).max() <= 1e-5 * np.abs(Q64).max()


def test_bf16_needs_a_shared_operator():
    m, h, hu, hv, b = user_state(4, 2, "large")          # variable bottom
    with pytest.raises(hd.HdgdgError):
        hd.Sim(4, 2, 0.01, bottom=b, local_precision="bf16")
    with pytest.raises(hd.HdgdgError):
        hd.Sim(4, 5, 0.01, local_precision="bf16")        # tensor-core tiles cover k <= 4
    with pytest.raises(hd.HdgdgError):
        hd.Sim(4, 2, 0.01, batch=2, dt_per_instance=[0.01, 0.02], local_precision="bf16")


def _energy_rel(m, qa, qo, phiB):
    w = m.mass[None]
    num = np.sum(w * ((qa[0] - qo[0]) ** 2 + ((qa[1] - qo[1]) ** 2 + (qa[2] - qo[2]) ** 2) / phiB))
    den = np.sum(w * (qo[0] ** 2 + (qo[1] ** 2 + qo[2] ** 2) / phiB))
    return float(np.sqrt(num / den))


def _bump8_run(local, n_steps):
    m, h, hu, hv, b = user_state(8, 2, "bump8")
    q, phiB = oracle_state(m, h, hu, hv, b)
    dt = dt_of(m, h, hu, hv)
    qo = imex.Stepper(m, phiB, dt, solver="lu").run(q, n_steps)
    with hd.Sim(8, 2, dt, bottom=b, g=W.G, H0=W.H0, precision="mixed", local_precision=local) as s:
        s.set_state(h, hu, hv)
        s.step(n_steps)
        out = s.get_state()
    qa, _ = swe.to_state(*out, b, W.G, W.H0)
    return _energy_rel(m, qa, qo, phiB), max(imex.rel_l2(m, qa[c], qo[c]) for c in range(3))


@pytest.mark.parametrize("local,bound", [("fp32", 1e-6), ("bf16", 2e-2)])
def test_precision_variant_one_step(local, bound):
    """One step of the 8x8, k = 2 bump in the mixed form with FP32 or BF16 (tensor-core) local
    contractions: error against the FP64 oracle at the operands' rounding level (FP32: ~1e-7;
    BF16: ~1e-3) -- and not below it, so the variant really ran."""
    e, r_max = _bump8_run(local, 1)
    print(f"local {local}, 1 step: energy-norm rel {e:.3e}, largest field rel {r_max:.3e}")
    assert e <= bound and r_max <= bound
    assert e >= bound * 1e-4


def test_fp32_variant_of_the_8x8_bump_200_steps():
    """The precision variant of the 8x8 bump over its 200 steps with FP32 local contractions:
    measured 2.7e-5 (eta), 1.2e-5 (hu), 1.4e-5 (hv) against the FP64 oracle; every field and the
    energy norm are gated at 1e-4.  The error grows while the L-stable implicit part damps the
    bump: every stage rounds R1 -- the state itself -- to FP32, and the damped solution shrinks
    below the injected rounding.  (With BF16 operands the same mechanism leaves no accuracy after
    200 steps: 1.04 measured; bench.py --precision-table reports it.)"""
    e, r_max = _bump8_run("fp32", 200)
    print(f"local fp32, 200 steps: energy-norm rel {e:.3e}, largest field rel {r_max:.3e}")
    assert e <= 1e-4 and r_max <= 1e-4


@pytest.mark.parametrize("N,k", [(6, 3), (9, 2), (5, 4)])
def test_f32x2_local_operators_are_fp64_class(N, k):
    """HDGDG_LOCAL_F32X2 (FP32-pair operator, compensated Dot2 sums): condensation and a whole
    stage solve agree with the FP64 local operators to ~1e-13, far below FP32's ~1e-7."""
    m, h, hu, hv, b = user_state(N, k, "large")
    q, phiB = oracle_state(m, h, hu, hv, b)
    dt = 0.4 / N
    R1 = q + 0.01 * rng.standard_normal(q.shape)
    with hd.Sim(N, k, dt, bottom=b, g=W.G, H0=W.H0, local_precision="f32x2") as s:
        gx = s.condense_rhs(flat(R1))
        Qx, _, _ = s.stage_solve(flat(R1))
    with hd.Sim(N, k, dt, bottom=b, g=W.G, H0=W.H0) as s:
        g64 = s.condense_rhs(flat(R1))
        Q64, _, _ = s.stage_solve(flat(R1))
    assert np.abs(gx - g64).max() <= 1e-12 * np.abs(g64).max()
    assert np.abs(Qx - Q64).max() <= 1e-12 * np.abs(Q64).max()


def test_f32x2_mixed_bump8_200_steps_against_the_oracle():
    """The mixed form with FP32-pair local contractions over the 8x8 bump's 200 steps stays as
    close to the FP64 oracle as the mixed form with FP64 local contractions (energy norm and
    every field <= 1e-6; FP32 local contractions end at 2.7e-5)."""
    e, r_max = _bump8_run("f32x2", 200)
    print(f"local f32x2, 200 steps: energy-norm rel {e:.3e}, largest field rel {r_max:.3e}")
    assert e <= 1e-6 and r_max <= 1e-6


def test_f32x2_autotuned_tile():
    """On a mesh of >= 4096 elements the dense FP32-pair local kernels' tile (elements per block)
    is picked at create by timing the candidates; whichever wins, the condensation and stage solve
    stay within 1e-12 of the FP64 local operators (the tile does not change any row's sums).  The
    Schur-complement kernels (the default) are tuned too: 8, 16 or 32 elements per block at k = 3."""
    N, k = 64, 3
    x, y = hd.node_coords(N, k)
    h, hu, hv, b = W.large_state(x, y, seed=9)
    q = np.stack([W.G * (h - (W.H0 - b)), W.G * hu, W.G * hv])
    R1 = q + 0.01 * rng.standard_normal(q.shape)
    dt = 0.4 / N
    with hd.Sim(N, k, dt, bottom=b, g=W.G, H0=W.H0, local_precision="f32x2") as s:
        st = s.stats()
        assert st["local_tile_condense"] in (8, 16, 32) and st["local_tile_recover"] in (8, 16, 32)
    with hd.Sim(N, k, dt, bottom=b, g=W.G, H0=W.H0, local_precision="f32x2", local_dense=True) as s:
        st = s.stats()
        assert st["local_tile_condense"] in (1, 2, 4, 5, 8) and st["local_tile_recover"] in (1, 2, 4, 5, 8)
        gx = s.condense_rhs(R1)
        Qx, _, _ = s.stage_solve(R1)
    with hd.Sim(N, k, dt, bottom=b, g=W.G, H0=W.H0, local_dense=True) as s:
        g64 = s.condense_rhs(R1)
        Q64, _, _ = s.stage_solve(R1)
    assert np.abs(gx - g64).max() <= 1e-12 * np.abs(g64).max()
    assert np.abs(Qx - Q64).max() <= 1e-12 * np.abs(Q64).max()


# ---- FP64-class products on the tensor cores: BF16 slices (Ozaki splitting) ----------------------
SLICES = 5


def _exp_above(v):
    """e with |v| < 2^e for the largest |v| (numpy frexp), -1074 for all zeros."""
    m = np.abs(v).max(axis=-1)
    _, e = np.frexp(m)
    return np.where(m == 0.0, -1074, e)


def _slices(v, e):
    """Seven-bit integer slices t_i of v / 2^e, rounding to nearest even, as the device cuts them."""
    u = np.ldexp(v, -np.where(e < -1000, 0, e)[..., None])
    out = []
    for _ in range(SLICES):
        w = u * 128.0
        r = np.rint(w)
        out.append(r.astype(np.int64))
        u = w - r
    return out


def _split_product(X, B):
    """X @ B^T with the device's arithmetic, emulated exactly: rows of X (elements) and rows of B
    (outputs; B[r][k] = (A^{-1})_{rk}) scaled and sliced, D_s = sum_{i+j=s} t_i s_j^T in integers,
    combined and scaled by powers of two."""
    er = _exp_above(X)                                   # [rows]
    ec = _exp_above(B)                                   # [outputs]
    tx = _slices(X, er)
    tb = _slices(B, ec)
    acc = np.zeros((X.shape[0], B.shape[0]), dtype=object)
    for s in range(SLICES):
        D = sum(tx[i].astype(object) @ tb[s - i].astype(object).T for i in range(s + 1))
        acc = acc * 128 + D
    scale = (er[:, None] + ec[None, :] - 7 * (SLICES + 1))
    out = np.array([[float(np.ldexp(float(acc[a, b]), int(scale[a, b]))) for b in range(acc.shape[1])]
                    for a in range(acc.shape[0])])
    zero = (er[:, None] < -1000) | (ec[None, :] < -1000)
    return np.where(zero, 0.0, out)


@pytest.mark.parametrize("N,k", [(6, 3), (12, 2), (4, 4), (17, 3)])
def test_split_tensor_core_condensation_matches_exact_emulation(N, k):
    """Condensation with the sliced operator on the tensor cores: Z equals the exact emulation of the
    slices' products (so g = -C Z equals it to the FP64 rounding of C), and Z is FP64-class: its
    distance to the FP64 route is below 1e-9 of the field, 1e4 times below the BF16 variant's."""
    m, h, hu, hv, b = _flat_case(N, k)
    q, phiB = oracle_state(m, h, hu, hv, b)
    dt = 0.4 / N
    st = imex.Stepper(m, phiB, dt, solver="dense")
    R1 = q + 0.01 * rng.standard_normal(q.shape)
    Ainv, C = st.cond.Ainv, st.cond.C
    Z = _split_product(_elem(R1), Ainv[0])               # the shared operator: every element's is the same
    loc = -np.einsum("etv,ev->et", C, Z)
    ref = np.bincount(st.cond.gi.ravel(), weights=loc.ravel(), minlength=st.cond.n)
    ref = ref.reshape(m.n_edges, 3, m.P) / (m.face_jac * m.w)[None, None, :]
    with hd.Sim(N, k, dt, bottom=b, g=W.G, H0=W.H0, local_precision="bf16split") as s:
        got = s.condense_rhs(flat(R1))
    with hd.Sim(N, k, dt, bottom=b, g=W.G, H0=W.H0) as s:
        g64 = s.condense_rhs(flat(R1))
    scale = np.abs(ref).max()
    assert np.abs(got - ref).max() <= 1e-13 * scale
    assert np.abs(got - g64).max() <= 1e-9 * scale


@pytest.mark.parametrize("N,k", [(6, 3), (12, 2)])
def test_split_tensor_core_stage_solve_is_fp64_class(N, k):
    m, h, hu, hv, b = _flat_case(N, k)
    q, phiB = oracle_state(m, h, hu, hv, b)
    dt = 0.4 / N
    R1 = q + 0.01 * rng.standard_normal(q.shape)
    with hd.Sim(N, k, dt, bottom=b, g=W.G, H0=W.H0, local_precision="bf16split") as s:
        Qs, lams, _ = s.stage_solve(flat(R1))
    with hd.Sim(N, k, dt, bottom=b, g=W.G, H0=W.H0) as s:
        Q64, lam64, _ = s.stage_solve(flat(R1))
    assert np.abs(Qs - Q64).max() <= 1e-9 * np.abs(Q64).max()


def test_split_tensor_core_bump8_200_steps_against_the_oracle():
    """The precision variant of the 8x8 bump with the local contractions on the tensor cores as BF16
    slices: every field within 1e-6 of the FP64 oracle after the 200 steps (BF16 operands: 1.0;
    FP32 CUDA-core operands: 2.7e-5)."""
    e, r_max = _bump8_run("bf16split", 200)
    print(f"local bf16split, 200 steps: energy-norm rel {e:.3e}, largest field rel {r_max:.3e}")
    assert e <= 1e-6 and r_max <= 1e-6


def test_bf16_input_dg_residual_variant():
    """The mixed form with the DG residual's inputs rounded to BF16 (FP32 arithmetic): its error
    against the FP64 oracle after one step sits at the BF16 rounding of the nonlinear increment --
    above the FP32 residual's and below 1e-3.  Over the 200 steps the error grows as the damped
    solution shrinks below the rounding each stage injects (measured 0.23, against 1.04 for BF16
    local contractions): the run stays finite and bounded, but this variant does not keep 1e-6."""
    m, h, hu, hv, b = user_state(8, 2, "bump8")
    hu = hu + 0.01 * np.sin(2 * np.pi * m.y.reshape(m.n_el, -1))    # a flow, so that the NL term is not zero
    q, phiB = oracle_state(m, h, hu, hv, b)
    dt = dt_of(m, h, hu, hv)
    errs = {}
    for dgp in ("default", "bf16"):
        with hd.Sim(8, 2, dt, bottom=b, g=W.G, H0=W.H0, precision="mixed", local_precision="f32x2",
                    trace_operator=1, dg_precision=dgp) as s:
            s.set_state(h, hu, hv)
            s.step(1)
            one = swe.to_state(*s.get_state(), b, W.G, W.H0)[0]
            s.step(199)
            two = swe.to_state(*s.get_state(), b, W.G, W.H0)[0]
        errs[dgp] = (one, two)
    st = imex.Stepper(m, phiB, dt, solver="lu")
    q1 = st.step(q)
    q200 = st.run(q1, 199)
    e1 = {k_: max(imex.rel_l2(m, v[0][c], q1[c]) for c in range(3)) for k_, v in errs.items()}
    e200 = {k_: max(imex.rel_l2(m, v[1][c], q200[c]) for c in range(3)) for k_, v in errs.items()}
    print(f"DG residual variants, 1 step: {e1}; 200 steps: {e200}")
    assert e1["bf16"] <= 1e-3 and e1["bf16"] >= 10 * e1["default"]
    assert all(np.isfinite(a).all() for a in errs["bf16"][1]) and e200["bf16"] < 1.0
