"""The allocation-free mass entry point agrees with the mass that hdgdg_get_stats reports.

hdgdg_mass_noalloc serves callers that cannot allocate device memory; its partial sums live
in the library's static device memory.  It is called twice in a row through the C ABI on
caller-owned device buffers, and each result must match the handle's mass within the FP64
tolerance of the other parity tests.
"""
import numpy as np
import pytest

from _common import user_state
from paper_1711_02751_gb300 import workloads as W

pytestmark = pytest.mark.gpu

hd = pytest.importorskip("paper_1711_02751_gb300.hdgdg")
torch = pytest.importorskip("torch")


def test_mass_noalloc_matches_get_stats_twice():
    N, k = 16, 3
    m, h, hu, hv, b = user_state(N, k, "large")
    with hd.Sim(N, k, 0.01, bottom=b, g=W.G, H0=W.H0) as s:
        s.set_state(h, hu, hv)
        ref = s.stats()["mass"]
    phi_eta = W.G * (h - (W.H0 - b))
    d_phi = torch.tensor(phi_eta, dtype=torch.float64, device="cuda")
    for _ in range(2):
        d_out = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")
        torch.cuda.synchronize()
        assert hd.mass_noalloc(N, k, d_phi.data_ptr(), d_out.data_ptr()) == hd.OK
        torch.cuda.synchronize()
        got = float(d_out.item())
        assert abs(got - ref) <= 1e-14 * abs(ref) + 1e-18


def test_mass_noalloc_rejects_sizes_beyond_its_scratch():
    d = torch.zeros(16, dtype=torch.float64, device="cuda")
    assert hd.mass_noalloc(1025, 3, d.data_ptr(), d.data_ptr()) == hd.EINVAL
    assert hd.mass_noalloc(4, 9, d.data_ptr(), d.data_ptr()) == hd.EINVAL
