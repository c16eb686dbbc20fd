"""Seeded synthetic workloads (initial states, bottoms, time steps) for the shallow-water runs.

This module holds input generation only: it evaluates closed-form initial conditions at
node coordinates that the caller supplies, and the time-step rule below.  It contains
none of the discretisation's arithmetic and is shared by the tests, the benchmark and
the oracle-side checks so that both sides see identical inputs.

All states are returned as (h, hu, hv, b) arrays of shape [n_el, (k+1)^2] in the node
order of the library (element e = ey*N + ex, node n = j*(k+1) + i, i along x).

Workloads (unit square, periodic, g = 1, H0 = 1):

* ``bump8``      8 x 8 quads, k = 2, flat bottom, h = 1 + 0.01 exp(-r^2 / 0.01) centred
                 at (0.5, 0.5), u = v = 0, 100 steps.
* ``large512``   512 x 512 quads, k = 3, b = 0.1 sin(2 pi x) sin(2 pi y), h = 1 - b + 16
                 seeded Gaussian bumps (amplitude U[0.005, 0.02], width U[0.02, 0.08],
                 centre U[0,1]^2, minimum-image distance), velocity from a seeded smooth
                 random streamfunction scaled to max |u| = 0.05, 200 steps.
* ``large512_stiff`` the large512 recipe with a slower flow, max |u| = 0.01 (same seeds), and
                 the rest-state floor of the time-step rule lowered to 0.01 sqrt(g H0): the
                 explicit part keeps its Courant number while the gravity Courant number of
                 the implicit part rises to about 14 (the stiff regime of the method).
* ``sized(N, k)`` the large512 recipe on another mesh (parity cases that span several
                 tiles and a ragged tail).

Time step (the advective CFL 0.5 of the workload definition): dt = 0.5 h_e / ((2k+1)
lambda_NL), the standard explicit DG bound with the spectral radius lambda_NL = 2 max|u| of
the nonlinear flux Jacobian (floored at 0.05 sqrt(g H0)).  In the paper's own Courant number
Cr = (max|u| + sqrt(phi)) dt / dx_min (dx_min the smallest GLL gap) this gives a gravity
Courant number of about 2.7 on large512 and 4 on bump8.
"""
import math

import numpy as np

G = 1.0
H0 = 1.0


def _min_image(d):
    return d - np.round(d)


def gaussian_bumps(x, y, rng, n_bumps):
    """Sum of n_bumps seeded periodic Gaussian bumps a exp(-d^2 / w^2)."""
    out = np.zeros_like(x)
    for _ in range(n_bumps):
        cx, cy = rng.uniform(0.0, 1.0, size=2)
        amp = rng.uniform(0.005, 0.02)
        wid = rng.uniform(0.02, 0.08)
        d2 = _min_image(x - cx) ** 2 + _min_image(y - cy) ** 2
        out += amp * np.exp(-d2 / wid ** 2)
    return out


def streamfunction_velocity(x, y, rng, umax=0.05, kmax=4):
    """Divergence-free (u, v) = (d_y psi, -d_x psi) of a seeded smooth periodic psi.

    psi = sum_{(m,n) != 0, |m|,|n| <= kmax} a_mn sin(2 pi (m x + n y) + theta_mn),
    a_mn ~ N(0,1) / (m^2 + n^2), theta ~ U[0, 2 pi); scaled so max over nodes |u| = umax.
    """
    u = np.zeros_like(x)
    v = np.zeros_like(x)
    for m in range(-kmax, kmax + 1):
        for n in range(-kmax, kmax + 1):
            if m == 0 and n == 0:
                continue
            a = rng.standard_normal() / (m * m + n * n)
            th = rng.uniform(0.0, 2.0 * math.pi)
            c = np.cos(2.0 * math.pi * (m * x + n * y) + th)
            u += a * 2.0 * math.pi * n * c
            v -= a * 2.0 * math.pi * m * c
    speed = np.sqrt(u * u + v * v).max()
    return u * (umax / speed), v * (umax / speed)


def bump8_state(x, y):
    """The 8 x 8, k = 2 flat-bottom workload at node coordinates x, y [n_el, Np]."""
    b = np.zeros_like(x)
    h = 1.0 + 0.01 * np.exp(-((x - 0.5) ** 2 + (y - 0.5) ** 2) / 0.01)
    return h, np.zeros_like(x), np.zeros_like(x), b


def large_state(x, y, seed=2000, n_bumps=16, umax=0.05):
    """The variable-bottom workload (bumps + streamfunction velocity) at nodes x, y."""
    rng = np.random.Generator(np.random.PCG64(seed))
    b = 0.1 * np.sin(2.0 * math.pi * x) * np.sin(2.0 * math.pi * y)
    h = H0 - b + gaussian_bumps(x, y, rng, n_bumps)
    u, v = streamfunction_velocity(x, y, rng, umax=umax)
    return h, h * u, h * v, b


def bump_at_rest_state(x, y, seed, bottom_amp=0.0):
    """Ensemble and serving requests: one seeded Gaussian bump (centre U[0,1]^2, amplitude
    U[0.005, 0.02], width U[0.02, 0.08], minimum-image distance) on a lake at rest (u = v = 0)
    over the bottom b = bottom_amp sin(2 pi x) sin(2 pi y) (0: flat, as the 8 x 8 bump)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    b = bottom_amp * np.sin(2.0 * math.pi * x) * np.sin(2.0 * math.pi * y)
    h = H0 - b + gaussian_bumps(x, y, rng, 1)
    return h, np.zeros_like(x), np.zeros_like(x), b


def lake_at_rest_state(x, y, amp=0.1):
    """Still water over the sinusoidal bottom: h = H0 - b, u = v = 0."""
    b = amp * np.sin(2.0 * math.pi * x) * np.sin(2.0 * math.pi * y)
    return H0 - b, np.zeros_like(x), np.zeros_like(x), b


def standing_wave_state(x, y, eps=1e-3, t=0.0):
    """Linear standing gravity wave on a flat bottom (closed form of the linear PDE).

    phi_eta = eps cos(2 pi x) cos(2 pi y) cos(w t), U = eps/sqrt2 sin cos sin(w t),
    V = eps/sqrt2 cos sin sin(w t), w = 2 pi sqrt(2), with g = H0 = 1.
    """
    w = 2.0 * math.pi * math.sqrt(2.0)
    cx, sx = np.cos(2 * math.pi * x), np.sin(2 * math.pi * x)
    cy, sy = np.cos(2 * math.pi * y), np.sin(2 * math.pi * y)
    eta = eps * cx * cy * math.cos(w * t)
    U = eps / math.sqrt(2.0) * sx * cy * math.sin(w * t)
    V = eps / math.sqrt(2.0) * cx * sy * math.sin(w * t)
    return H0 + eta / G, U / G, V / G, np.zeros_like(x)


def standing_wave_walls_state(x, y, eps=1e-3, t=0.0):
    """Linear standing gravity wave in the walled unit square (flat bottom, g = H0 = 1):
    phi_eta = eps cos(pi x) cos(pi y) cos(w t), U = eps/sqrt2 sin(pi x) cos(pi y) sin(w t),
    V = eps/sqrt2 cos(pi x) sin(pi y) sin(w t), w = pi sqrt(2); U.n = 0 on the walls."""
    w = math.pi * math.sqrt(2.0)
    cx, sx = np.cos(math.pi * x), np.sin(math.pi * x)
    cy, sy = np.cos(math.pi * y), np.sin(math.pi * y)
    eta = eps * cx * cy * math.cos(w * t)
    U = eps / math.sqrt(2.0) * sx * cy * math.sin(w * t)
    V = eps / math.sqrt(2.0) * cx * sy * math.sin(w * t)
    return H0 + eta / G, U / G, V / G, np.zeros_like(x)


def perturbation_state(x, y, H_inf=100.0, sigma=0.1):
    """The paper's water-height perturbation (Sec. 7.2) on [-1, 1]^2: H = H_inf +
    exp(-(x^2 + y^2) / (2 sigma^2)), u = v = 0, flat bottom (b = H0 - H_inf with H0 = 1 so
    that B = H_inf).  The paper does not print sigma; 0.1 is this library's reading."""
    b = np.full_like(x, H0 - H_inf)
    h = H_inf + np.exp(-(x * x + y * y) / (2.0 * sigma * sigma))
    return h, np.zeros_like(x), np.zeros_like(x), b


VORTEX = {"H_inf": 1.0, "u_inf": 1.0, "v_inf": 0.0, "beta": 5.0, "g": 2.0, "xc": 0.0, "yc": 0.0}


def vortex_state(x, y, t, H_inf=1.0, u_inf=1.0, v_inf=0.0, beta=5.0, g=2.0, xc=0.0, yc=0.0):
    """The moving vortex of the paper's Sec. 7.1 (eq. tc_vortex_ic) at time t, as (h, hu, hv, b)
    with a flat bottom b = 0 and H0 = H_inf.  The depth is H_inf - beta^2/(16 pi^2 g)
    e^{-2(r^2-1)}, which is the cyclostrophic balance of the printed swirl and equals the printed
    beta^2/(32 pi^2) at the paper's g = 2."""
    xt = x - xc - u_inf * t
    yt = y - yc - v_inf * t
    r2 = xt * xt + yt * yt
    e = np.exp(-(r2 - 1.0))
    H = H_inf - beta * beta / (16.0 * math.pi ** 2 * g) * e * e
    u = u_inf - beta / (2.0 * math.pi) * e * yt
    v = v_inf + beta / (2.0 * math.pi) * e * xt
    return H, H * u, H * v, np.zeros_like(x)


def advective_dt(x, h, hu, hv, n_side, cfl=0.5, g=G, H0_=H0, floor=0.05):
    """Explicit-part time step dt = cfl * h_e / ((2k+1) * lambda_NL) for states [n_el, (k+1)^2].

    h_e = 1/n_side is the element size and h_e/(2k+1) the standard explicit DG length scale
    for degree k.  lambda_NL is the spectral radius of the nonlinear flux Jacobian dF_NL/dq,
    whose largest eigenvalue is 2|u| (from d(U^2/phi)/dU), floored at `floor` sqrt(g H0) for
    states at rest (0.05 unless a workload states otherwise).  x is unused beyond its shape.
    """
    k = int(round(np.sqrt(np.shape(x)[1]))) - 1
    speed = np.sqrt(hu ** 2 + hv ** 2) / h
    lam = max(2.0 * float(speed.max()), floor * math.sqrt(g * H0_))
    return cfl * (1.0 / n_side) / ((2 * k + 1) * lam)


def courant(dx_min, dt, max_speed_plus_celerity):
    """The paper's Courant number (max|u| + sqrt(phi)) dt / dx_min."""
    return max_speed_plus_celerity * dt / dx_min


STIFF_UMAX = 0.01    # large512_stiff: max |u| of the streamfunction flow
STIFF_FLOOR = 0.01   # large512_stiff: rest-state floor of the time-step rule, in units of sqrt(g H0)


def stiff_state(x, y, seed=2000):
    """large512_stiff: the large recipe with the flow slowed to max |u| = STIFF_UMAX."""
    return large_state(x, y, seed=seed, umax=STIFF_UMAX)


WORKLOADS = {
    "bump8": {"N": 8, "k": 2, "steps": 100, "state": "bump8"},
    "large512": {"N": 512, "k": 3, "steps": 200, "state": "large"},
    "large512_stiff": {"N": 512, "k": 3, "steps": 200, "state": "stiff", "dt_floor": STIFF_FLOOR},
}


def make_state(name, x, y, seed=None):
    """Dispatch to a state generator by workload name."""
    kind = WORKLOADS[name]["state"] if name in WORKLOADS else name
    if kind == "bump8":
        return bump8_state(x, y)
    if kind == "large":
        return large_state(x, y, seed=2000 if seed is None else seed)
    if kind == "stiff":
        return stiff_state(x, y, seed=2000 if seed is None else seed)
    if kind == "lake":
        return lake_at_rest_state(x, y)
    if kind == "standing":
        return standing_wave_state(x, y)
    if kind == "standing_walls":
        return standing_wave_walls_state(x, y)
    raise KeyError(name)
