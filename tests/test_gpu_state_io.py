"""State transfers through pinned host buffers (read and written by the conversion kernels over the
host link) against pageable host arrays (staged through device memory): the same states bit for
bit, for set_state, update_state and get_state, on a batch of two instances."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu
hd = pytest.importorskip("paper_1711_02751_gb300.hdgdg")
torch = pytest.importorskip("torch")
from paper_1711_02751_gb300 import workloads as W  # noqa: E402

from _common import user_state  # noqa: E402


def _pinned(a):
    t = torch.empty(a.size, dtype=torch.float64, pin_memory=True)
    t.numpy()[:] = a.ravel()
    return t


@pytest.mark.parametrize("kw", [{}, {"precision": "mixed", "local_precision": "f32x2", "trace_operator": 1}])
def test_pinned_buffers_equal_pageable(kw):
    N, k = 12, 3
    m, h, hu, hv, b = user_state(N, k, "large")
    h2, hu2, hv2, b2 = (np.concatenate([a, a[::-1]]) for a in (h, hu, hv, b))
    dts = [0.004, 0.003]
    out = {}
    for mode in ("pageable", "pinned"):
        with hd.Sim(N, k, max(dts), bottom=b2, g=W.G, H0=W.H0, batch=2, dt_per_instance=dts, **kw) as s:
            if mode == "pageable":
                s.set_state(h2, hu2, hv2)
                s.step(2)
                mid = s.get_state()
                s.update_state(*mid)
                s.step(2)
                out[mode] = s.get_state()
            else:
                src = [_pinned(a) for a in (h2, hu2, hv2)]
                dst = [torch.empty(h2.size, dtype=torch.float64, pin_memory=True) for _ in range(3)]
                s.set_state_ptrs(*(t.data_ptr() for t in src))
                s.step(2)
                s.get_state_ptrs(*(t.data_ptr() for t in dst))
                s.update_state_ptrs(*(t.data_ptr() for t in dst))
                s.step(2)
                res = [torch.empty(h2.size, dtype=torch.float64, pin_memory=True) for _ in range(3)]
                s.get_state_ptrs(*(t.data_ptr() for t in res))
                out[mode] = [t.numpy().reshape(h2.shape).copy() for t in res]
    for a_, c_ in zip(out["pinned"], out["pageable"]):
        assert np.array_equal(a_, c_)
