"""bench.py's algorithmic model -- the numerators of every roofline fraction it reports -- against
the per-unit counts written out by hand from the layouts (no GPU):

* SpMV: per edge the six off-diagonal n_f x n_f blocks of S~ (the block-Jacobi-preconditioned
  trace matrix, identity diagonal not stored), six int32 column indices, x and y once; 2 n_f^2 + n_f
  flops per row (the identity adds x).
* Schur-complement local solves: per element the (phi, phi) block of A^{-1} ((k+1)^4 numbers)
  and four numbers per node, R1 in and Z out (condensation) or Z, R1 in and Q, L out
  (recovery), eight bytes each -- Q four in the mixed form, whose DG residual reads it in FP32 --
  plus the trace traffic per edge.
* dense route: the whole (3 (k+1)^2)^2 A^{-1} for the condensation and its boundary columns for
  the recovery.
"""
import importlib.util
import os

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def bench():
    pytest.importorskip("torch")
    spec = importlib.util.spec_from_file_location("bench_model_mod", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_spmv_bytes_and_flops(bench):
    N, k = 512, 3
    edges, nf = 2 * N * N, 3 * (k + 1)
    b64, f = bench._algorithmic(N, k, "spmv", "fp64")
    b32, f32 = bench._algorithmic(N, k, "spmv", "mixed")
    assert b64 == edges * 7128 and b32 == edges * 3576          # 6*144*8 + 24 + 192 ; 6*144*4 + 24 + 96
    assert b32 == 1874853888                                     # the figure bench.py reports
    assert f == f32 == edges * nf * (12 * nf + 1)


@pytest.mark.parametrize("k", [1, 3, 5])
def test_local_solve_bytes(bench, k):
    N = 64
    P, n_el, edges = k + 1, N * N, 2 * N * N
    Np, NV, NF = P * P, 3 * P * P, 3 * P
    sc, _ = bench._algorithmic(N, k, "condense", "mixed", dense=False, local="f32x2")
    sr, _ = bench._algorithmic(N, k, "recover", "mixed", dense=False, local="f32x2")
    assert sc == n_el * ((Np * Np + 4 * Np) * 8 + 2 * NV * 8) + edges * NF * 8 * 3
    # forming R1 from q and two terms on average: q, the terms and R1 out replace R1 in
    sf, ff = bench._algorithmic(N, k, "condense", "mixed", dense=False, local="f32x2", r1_terms=2.0)
    assert sf == sc + n_el * NV * 8 * 3 and ff == n_el * Np * 12 + n_el * NV * 4
    assert bench.ARS2_R1_TERMS == 2.0
    assert sr == n_el * ((Np * Np + 4 * Np) * 8 + 3 * NV * 8 + NV * 4) + edges * NF * 8
    dc, _ = bench._algorithmic(N, k, "condense", "fp64", dense=True)
    dr, _ = bench._algorithmic(N, k, "recover", "fp64", dense=True)
    nb = 3 * (4 * P - 4)                                          # boundary columns of A^{-1}
    assert dc == n_el * (NV * NV * 8 + 2 * NV * 8) + edges * NF * 8 * 3
    assert dr == n_el * (NV * nb * 8 + 4 * NV * 8) + edges * NF * 8
    assert dc > (5 if k >= 3 else 2) * sc      # the Schur route's point (vectors dominate at k = 1)


def test_fp32_pair_schur_is_hbm_bound_in_the_model(bench):
    """The FP32-pair Schur kernels count only their FP64 operations against the FP64 rate, so the
    model calls them HBM bound at the measured peaks; the FP64 versions are FP64-rate bound."""
    N, k = 512, 3
    for cls in ("condense", "recover"):
        b, f = bench._algorithmic(N, k, cls, "mixed", dense=False, local="f32x2")
        assert b / 6679.8e9 > f / 1.25e12
        b, f = bench._algorithmic(N, k, cls, "fp64", dense=False, local="fp64")
        assert b / 6679.8e9 < f / 1.25e12


def test_matrix_free_operator_bytes(bench):
    """Matrix-free trace operator (FP32 arithmetic): per edge its FP16 M^{-1} block (n_f^2 halves)
    and its scale (one float), tau (P floats), x and y (n_f floats each); per element the FP32 Schur
    operators ((k+1)^4 + 4 (k+1)^2 floats).  At k = 3 that is 404 B per edge + 1280 B per element:
    3.4x below the assembled FP32 product's 3576 B per edge."""
    N, k = 512, 3
    edges, n_el = 2 * N * N, N * N
    b, f = bench._algorithmic(N, k, "spmv", "mixed", dense=False, local="f32x2", mf=True)
    assert b == edges * (144 * 2 + 4 + 4 * 4 + 2 * 12 * 4) + n_el * (256 + 64) * 4 == 547356672
    b32, _ = bench._algorithmic(N, k, "spmv", "mixed")
    assert b32 / b > 3.3
    assert f > 0
