"""The C-ABI library loads and exports every symbol its header declares (no GPU needed)."""
import os
import re
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "hdgdg.h")


def _declared():
    text = open(HEADER).read()
    return sorted(set(re.findall(r"\b(hdgdg_[a-z0-9_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def libmod():
    from paper_1711_02751_gb300 import build, hdgdg
    if not os.path.exists(hdgdg.LIB_PATH):
        build.build()
    return hdgdg


def test_header_declares_the_binding_names(libmod):
    assert _declared() == sorted(libmod.EXPORTS)


def test_library_exports_every_declared_symbol(libmod):
    L = libmod.lib()
    for name in _declared():
        assert hasattr(L, name), name
    out = subprocess.run(["nm", "-D", "--defined-only", libmod.LIB_PATH], capture_output=True, text=True).stdout
    exported = set(re.findall(r" T (hdgdg_\w+)", out))
    assert set(_declared()) <= exported


def test_host_only_entry_points(libmod):
    """bytes_required and node_coords make no GPU call."""
    cfg = libmod.make_config(8, 2, 0.625)
    assert libmod.bytes_required(cfg) > 0
    assert libmod.bytes_required(libmod.make_config(1, 2, 0.1)) == 0      # N < 2 rejected
    assert libmod.bytes_required(libmod.make_config(4, 9, 0.1)) == 0      # k > 8 rejected
    x, y = libmod.node_coords(4, 3)
    from oracle import swe
    m = swe.Mesh(4, 3)
    np.testing.assert_allclose(x, m.x.reshape(16, -1), atol=1e-15)
    np.testing.assert_allclose(y, m.y.reshape(16, -1), atol=1e-15)


def test_large_workload_fits_one_gpu(libmod):
    cfg = libmod.make_config(512, 3, 5.4e-3)
    assert libmod.bytes_required(cfg) < 60e9


def test_schur_local_operators_need_less_memory(libmod):
    """The Schur-complement local solves keep the (phi, phi) block of A^{-1} instead of an FP32
    pair of the whole A^{-1}: (k+1)^4 + 4 (k+1)^2 eight-byte numbers per element (and two
    (k+1) x (k+1) matrices per instance) instead of 9 (k+1)^4 FP32 pairs."""
    s = libmod.bytes_required(libmod.make_config(64, 3, 5e-3, local_precision="f32x2"))
    d = libmod.bytes_required(libmod.make_config(64, 3, 5e-3, local_precision="f32x2", local_dense=True))
    n_el, Np = 64 * 64, 16
    assert d - s == n_el * 8 * (3 * Np) ** 2 - (n_el * (Np * Np + 4 * Np) + 2 * Np) * 8
    bad = libmod.make_config(8, 2, 0.1)
    bad.local_dense = 2
    assert libmod.bytes_required(bad) == 0
