"""Kernel-class timers: recorded inside the captured GMRES cycle graph (external event-record
nodes), they leave the results bit-identical and read back a positive time for every class the
step runs."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu
hd = pytest.importorskip("paper_1711_02751_gb300.hdgdg")

from _common import dt_of, user_state  # noqa: E402


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_timers_on_and_off_give_the_same_steps(precision):
    m, h, hu, hv, b = user_state(16, 3, "large")
    dt = dt_of(m, h, hu, hv)
    outs = []
    for timing in (False, True):
        with hd.Sim(16, 3, dt, bottom=b, precision=precision) as s:
            s.set_kernel_timing(timing)
            s.set_state(h, hu, hv)
            s.step(5)
            outs.append(s.get_state())
            kt = s.kernel_times()
        if timing:
            for cls in ("spmv", "ortho", "condense", "recover", "dg", "combine", "residual", "guess", "precond"):
                assert kt[cls][0] > 0.0 and kt[cls][1] > 0, cls
        else:
            assert all(v[1] == 0 for v in kt.values())
    for a, c in zip(*outs):
        assert np.array_equal(a, c)
