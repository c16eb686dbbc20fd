"""The allocation-free mass entry point agrees with the mass that hdgdg_get_stats reports.

hdgdg_mass_noalloc serves callers that cannot allocate device memory (code inside another
framework's fixed memory pool, a real-time loop kept out of the CUDA allocator, a host callback);
its partial sums live in the library's static device memory.  It is called twice in a row through
the C ABI on caller-owned device buffers, on the unit square and on the moving vortex's 4 x 4
domain, and each result must match the handle's mass within the FP64 tolerance of the other
parity tests.  (This file is collected last so that a run stopping at its first failure has run
every other test first.)
"""
import numpy as np
import pytest

from _common import user_state
from paper_1711_02751_gb300 import workloads as W

pytestmark = pytest.mark.gpu

hd = pytest.importorskip("paper_1711_02751_gb300.hdgdg")
torch = pytest.importorskip("torch")


def _twice(N, k, phi_eta, ref, length):
    d_phi = torch.tensor(np.ascontiguousarray(phi_eta), dtype=torch.float64, device="cuda")
    for _ in range(2):
        d_out = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")
        torch.cuda.synchronize()
        assert hd.mass_noalloc(N, k, d_phi.data_ptr(), d_out.data_ptr(), length=length) == hd.OK
        torch.cuda.synchronize()
        got = float(d_out.item())
        assert abs(got - ref) <= 1e-14 * abs(ref) + 1e-18, (got, ref)


def test_mass_noalloc_matches_get_stats_twice():
    N, k = 16, 3
    m, h, hu, hv, b = user_state(N, k, "large")
    with hd.Sim(N, k, 0.01, bottom=b, g=W.G, H0=W.H0) as s:
        s.set_state(h, hu, hv)
        ref = s.stats()["mass"]
    _twice(N, k, W.G * (h - (W.H0 - b)), ref, 1.0)


def test_mass_noalloc_on_a_domain_of_side_four():
    """The moving vortex's [-2, 2]^2 domain: J = (4 / (2N))^2, sixteen times the unit square's."""
    V = W.VORTEX
    N, k = 6, 2
    x, y = hd.node_coords(N, k, boundary="vortex", x0=-2.0, length=4.0)
    h, hu, hv, b = W.vortex_state(x, y, 0.0, **V)
    bc = (V["beta"], V["u_inf"], V["v_inf"], V["xc"], V["yc"])
    with hd.Sim(N, k, 0.01, bottom=b, g=V["g"], H0=V["H_inf"], boundary="vortex", x0=-2.0, length=4.0,
                bc_params=bc) as s:
        s.set_state(h, hu, hv)
        ref = s.stats()["mass"]
    phi_eta = V["g"] * (h - (V["H_inf"] - b))
    assert abs(ref) > 1e-3
    _twice(N, k, phi_eta, ref, 4.0)


def test_mass_noalloc_rejects_sizes_beyond_its_scratch():
    d = torch.zeros(16, dtype=torch.float64, device="cuda")
    assert hd.mass_noalloc(1025, 3, d.data_ptr(), d.data_ptr()) == hd.EINVAL
    assert hd.mass_noalloc(4, 9, d.data_ptr(), d.data_ptr()) == hd.EINVAL
    assert hd.mass_noalloc(4, 2, d.data_ptr(), d.data_ptr(), length=float("nan")) == hd.EINVAL
