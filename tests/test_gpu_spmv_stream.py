"""The pipelined FP32 trace-matrix product (spmv_kernel = 1: bulk copies into shared memory,
two stages on mbarriers, persistent CTAs) against the default kernel (spmv_kernel = 0): the same summation order, so whole
mixed-form steps are identical bit for bit.  The sizes give every CTA several tiles, so both
stages are reused, and end on a ragged last tile (k = 2: 28 edges per tile)."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu
hd = pytest.importorskip("paper_1711_02751_gb300.hdgdg")
from paper_1711_02751_gb300 import workloads as W  # noqa: E402


@pytest.mark.parametrize("N,k,boundary", [(96, 3, "periodic"), (128, 2, "periodic"), (40, 1, "wall"),
                                          (24, 4, "periodic")])
def test_stream_spmv_bit_identical(N, k, boundary):
    x, y = hd.node_coords(N, k, boundary=boundary)
    h, hu, hv, b = W.large_state(x, y, seed=11)
    if boundary != "periodic":
        hu, hv = 0.0 * hu, 0.0 * hv
    dt = W.advective_dt(x, h, hu, hv, N)
    outs, its = [], []
    for kernel in (0, 1):
        with hd.Sim(N, k, dt, bottom=b, precision="mixed", spmv_kernel=kernel, boundary=boundary) as s:
            s.set_state(h, hu, hv)
            s.step(3)
            outs.append(s.get_state())
            its.append(s.stats()["krylov_iterations"])
    assert its[0] == its[1]
    for a, c in zip(*outs):
        assert np.array_equal(a, c)
