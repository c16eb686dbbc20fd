"""Pins of the workload definitions: the paper's Courant numbers and the generators' shapes."""
import json
import math
import os

import numpy as np

from oracle.gll import gll_nodes_weights
from paper_1711_02751_gb300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "courant_pairs.json")


def _dx_min(domain, n, p):
    x, _ = gll_nodes_weights(p)
    return (domain / n) / 2.0 * np.diff(x).min()


def _half_digit(v):
    """Half a unit in the second significant digit of a printed value."""
    return 0.5 * 10.0 ** (math.floor(math.log10(v)) - 1)


def test_courant_definition_reproduces_printed_pairs():
    """Cr = (max|u| + sqrt(phi)) dt / dx_min, dx_min the smallest physical GLL gap, gives the
    (dt, Cr) pairs the paper prints for its two planar tests, to two significant digits."""
    gold = json.load(open(GOLDEN))
    p = gold["perturbation"]
    dxm = _dx_min(p["domain"], p["n"], p["p"])
    c = math.sqrt(p["g"] * p["H_inf"])
    for dt, cr in p["pairs"]:
        assert abs(W.courant(dxm, dt, c) - cr) <= _half_digit(cr)
    v = gold["vortex"]
    dxm = _dx_min(v["domain"], v["n"], v["p"])
    # max |u|: u_inf plus the vortex's peak swirl beta/(2 pi) max_r r e^{1 - r^2} = beta/(2 pi) e^{1/2}/sqrt 2
    umax = v["u_inf"] + v["beta"] / (2 * math.pi) * math.exp(0.5) / math.sqrt(2)
    c = umax + math.sqrt(v["g"] * v["H_inf"])
    for dt, cr in v["pairs"]:
        assert abs(W.courant(dxm, dt, c) - cr) <= _half_digit(cr)


def test_advective_dt_of_the_two_workloads():
    """dt = 0.5 h / ((2k+1) * 2 max|u|), floored speed 0.05 at rest: bump8 0.25, large512 with
    its 0.05 peak speed 0.5 / (512 * 7 * 0.1)."""
    for N, k, umax, expect in [(8, 2, 0.0, 0.5 / (8 * 5 * 0.05)), (512, 3, 0.05, 0.5 / (512 * 7 * 0.1))]:
        shape = (4, (k + 1) ** 2)
        h = np.ones(shape)
        hu = np.full(shape, umax)
        z = np.zeros(shape)
        assert abs(W.advective_dt(z, h, hu, z, N) - expect) < 1e-12 * expect


def test_explicit_step_stays_below_the_papers_explicit_limit():
    """In the paper's Courant definition (smallest GLL gap), the explicit part's speed 2|u| and
    this dt give 0.26 on large512: below the Cr ~ 0.28 at which the paper reports its explicit
    RK2 DG blowing up (Sec. 7.1)."""
    k, N = 3, 512
    dx_min = _dx_min(1.0, N, k)
    dt = W.advective_dt(np.zeros((1, 16)), np.ones((1, 16)), np.full((1, 16), 0.05), np.zeros((1, 16)), N)
    assert W.courant(dx_min, dt, 0.1) < 0.28


def test_large_state_is_seeded_and_bounded():
    x = np.random.default_rng(0).uniform(size=(64, 16))
    y = np.random.default_rng(1).uniform(size=(64, 16))
    a = W.large_state(x, y)
    b = W.large_state(x, y)
    for u, v in zip(a, b):
        np.testing.assert_array_equal(u, v)
    h, hu, hv, bot = a
    assert np.all(h > 0.8)
    assert np.sqrt((hu / h) ** 2 + (hv / h) ** 2).max() <= 0.05 + 1e-15
    assert np.abs(bot).max() <= 0.1
