"""Continuous-batching request loop: every request's result is the same alone and in the mix."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu
hd = pytest.importorskip("paper_1711_02751_gb300.hdgdg")
from paper_1711_02751_gb300 import serving  # noqa: E402


def _requests(precision):
    rs = serving.poisson_requests(6, rate_per_s=50.0, seed=77, n_range=(12, 32), degrees=(2, 3),
                                  steps_range=(10, 30), precision=precision)
    return rs


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_results_same_alone_and_in_the_mix(precision):
    reqs = _requests(precision)
    budget = 4 * max(serving.bytes_of(r) for r in reqs)
    srv = serving.Server(hbm_budget=budget, max_slots=3, chunk=5)
    summary = srv.serve(reqs, time_scale=1.0)
    assert summary["completed"] == len(reqs) and not summary["errors"]
    assert summary["max_running"] >= 2                  # the work really overlapped
    for r in reqs:
        alone = serving.run_one(r, chunk=7)
        for a, b in zip(r.result, alone):
            assert np.array_equal(a, b)
    assert summary["tts_p50_s"] <= summary["tts_p99_s"]


def test_admission_respects_the_memory_budget():
    reqs = _requests("fp64")
    sizes = [serving.bytes_of(r) for r in reqs]
    srv = serving.Server(hbm_budget=max(sizes), max_slots=8, chunk=5)
    summary = srv.serve(reqs)
    assert summary["completed"] == len(reqs)
    for e in srv.log:
        assert e["hbm_used"] <= max(sizes)
    too_big = serving.Request(99, 64, 4, 5, 1, 0.0, "fp64")
    srv2 = serving.Server(hbm_budget=1000, max_slots=2)
    s2 = srv2.serve([too_big])
    assert s2["completed"] == 0 and s2["errors"] == ["exceeds the memory budget"]


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("mixed", 1e-6)])
def test_batched_units_match_lone_runs(precision, tol):
    """Requests grouped into batched handles give each member its lone result (to the solver
    tolerance: a batch's trace systems are solved together)."""
    reqs = serving.ensemble_requests(n=10, sides=(8, 12), degrees=(2, 3), steps=12, precision=precision)
    units = serving.batch_requests(reqs, max_batch=3)
    assert any(len(u.members) > 1 for u in units)
    budget = sum(serving.bytes_of(u) for u in units)
    summary = serving.Server(hbm_budget=budget, max_slots=4, chunk=5).serve(units)
    assert summary["completed"] == len(reqs) and not summary["errors"]
    for r in reqs:
        alone = serving.run_one(r, chunk=12)
        for a, b in zip(r.result, alone):
            assert np.linalg.norm(a - b) <= tol * np.linalg.norm(b)
