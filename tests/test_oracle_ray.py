"""Pins of the oracle's curved-ray propagator (reading RB) against facts other than
its own Snell-invariant quadrature: the closed-form rays of a medium with n^2
linear in height, a shooting integration of the vector ray equation, Fermat's
exact second-order form of the time saved against the straight line, the
constant-index limit and the weak-refraction scaling."""
import math

import mpmath as mp
import numpy as np
import pytest

import oracle

C = 299792458.0
AIR_RAY = {"kind": "exponential_ray", "N0": 3.25e-4, "H": 8000.0}
AIR_FLAT = {"kind": "exponential", "N0": 3.25e-4, "H": 8000.0}

GEOMETRIES = [  # (x_e, x_a): near-vertical, the inclined shower's, long and off-axis, below the antenna
    ([10.0, -20.0, 4000.0], [300.0, 0.0, 0.0]),
    ([-7000.0, 0.0, 4000.0], [0.0, 0.0, 0.0]),
    ([-17000.0, 300.0, 10000.0], [200.0, -50.0, 0.0]),
    ([0.0, 0.0, 500.0], [2500.0, 1000.0, 3000.0]),
]


@pytest.mark.parametrize("ze,za,p", [(4000.0, 0.0, 0.5), (9000.0, 100.0, 0.93), (600.0, 20.0, 0.2),
                                     (100.0, 3000.0, 0.7)])
def test_linear_n2_profile_matches_closed_form(ze, za, p):
    """n(z)^2 = n0^2 + g z: the ray is x(z) = (2p/g) sqrt(q(z)) + const with
    q = n^2 - p^2, and c T = (2/(3g)) q^(3/2) + (2 p^2/g) sqrt(q) between the ends."""
    n0, g = 1.0003, -5e-8
    med = {"kind": "ray_linear_n2", "n": n0, "dn2dz": g}
    # the closed forms in 30-digit arithmetic (their differences cancel in FP64)
    mp.mp.dps = 30
    q = lambda z: mp.mpf(n0) ** 2 + mp.mpf(g) * z - mp.mpf(p) ** 2
    lo, hi = min(ze, za), max(ze, za)
    gm = mp.mpf(g)
    rho = float((2 * mp.mpf(p) / gm) * (mp.sqrt(q(hi)) - mp.sqrt(q(lo))))
    cT = float((2 / (3 * gm)) * (q(hi) ** 1.5 - q(lo) ** 1.5)
               + (2 * mp.mpf(p) ** 2 / gm) * (mp.sqrt(q(hi)) - mp.sqrt(q(lo))))
    xe = [0.0, 0.0, ze]
    xa = [rho * 0.6, rho * 0.8, za]
    R, n_src, n_avg, delay = oracle.propagate(med, xe, xa)
    assert n_src == pytest.approx(math.sqrt(n0 * n0 + g * ze), rel=1e-15)
    assert delay * C == pytest.approx(cT, rel=1e-13)
    rh = oracle.emission_direction(med, xe, xa)
    s_e = p / math.sqrt(n0 * n0 + g * ze)
    want = np.array([0.6 * s_e, 0.8 * s_e, (1.0 if za > ze else -1.0) * math.sqrt(1 - s_e * s_e)])
    assert np.abs(rh - want).max() < 1e-13


def test_constant_index_gives_the_straight_line():
    med = {"kind": "ray_linear_n2", "n": 1.78, "dn2dz": 0.0}
    for xe, xa in GEOMETRIES:
        R, n_src, n_avg, delay = oracle.propagate(med, xe, xa)
        d = np.array(xa) - np.array(xe)
        assert R == pytest.approx(np.linalg.norm(d), rel=1e-15)
        assert delay == pytest.approx(1.78 * R / C, rel=1e-14)
        assert np.abs(oracle.emission_direction(med, xe, xa) - d / R).max() < 1e-14


def _shoot(medium, x_e, u0, z_stop, ds=0.5):
    """Integrate the ray equation d/ds (n t) = grad n (t the unit tangent) with
    classical RK4 in the state (x, n t) from x_e along u0 until z = z_stop;
    returns the end point and the optical path (integral of n ds)."""
    N0, H = medium["N0"], medium["H"]

    def n(z):
        return 1.0 + N0 * math.exp(-z / H)

    def dn(z):
        return -N0 / H * math.exp(-z / H)

    def f(y):
        x, v = y[:3], y[3:6]  # v = n t
        nz = n(x[2])
        return np.concatenate([v / nz, [0.0, 0.0, dn(x[2])], [nz]])

    y = np.concatenate([np.array(x_e, float), n(x_e[2]) * np.array(u0, float), [0.0]])
    down = u0[2] < 0
    while True:
        k1 = f(y)
        k2 = f(y + 0.5 * ds * k1)
        k3 = f(y + 0.5 * ds * k2)
        k4 = f(y + ds * k3)
        y2 = y + ds / 6.0 * (k1 + 2 * k2 + 2 * k3 + k4)
        if (y2[2] <= z_stop) if down else (y2[2] >= z_stop):
            # last partial step to the stopping height (linear in s at this resolution)
            frac = (z_stop - y[2]) / (y2[2] - y[2])
            h = frac * ds
            k1 = f(y)
            k2 = f(y + 0.5 * h * k1)
            k3 = f(y + 0.5 * h * k2)
            k4 = f(y + h * k3)
            y = y + h / 6.0 * (k1 + 2 * k2 + 2 * k3 + k4)
            return y[:3], y[6]
        y = y2


@pytest.mark.parametrize("k", range(len(GEOMETRIES)))
def test_shooting_the_ray_equation_hits_the_antenna(k):
    """Launched from x_e along the oracle's emission direction, the ray of the
    eikonal equation (no Snell invariant used) reaches the antenna's height at the
    antenna, with the oracle's optical path."""
    xe, xa = GEOMETRIES[k]
    u0 = oracle.emission_direction(AIR_RAY, xe, xa)
    end, opt = _shoot(AIR_RAY, xe, u0, xa[2])
    R, _, _, delay = oracle.propagate(AIR_RAY, xe, xa)
    assert np.linalg.norm(end[:2] - np.array(xa[:2])) < 1e-6 * R
    assert opt == pytest.approx(delay * C, rel=1e-11)


@pytest.mark.parametrize("k", range(len(GEOMETRIES)))
def test_time_saved_equals_fermat_second_order_form(k):
    """With theta_s the straight line's angle from the vertical, theta(z) the
    ray's and C = cos(theta_s), the ray's optical path is the straight one minus
    the integral over z of 2 n sin^2((theta - theta_s)/2)/C (exact; it follows
    from n sin(theta) = p and the shared end points).  Evaluated with mpmath at
    30 digits, with p from the ray's end-point condition solved there too."""
    xe, xa = GEOMETRIES[k]
    mp.mp.dps = 30
    N0, H = mp.mpf(AIR_RAY["N0"]), mp.mpf(AIR_RAY["H"])
    n = lambda z: 1 + N0 * mp.exp(-z / H)
    d = [mp.mpf(b) - mp.mpf(a) for a, b in zip(xe, xa)]
    rho = mp.sqrt(d[0] ** 2 + d[1] ** 2)
    R = mp.sqrt(rho ** 2 + d[2] ** 2)
    lo, hi = sorted([mp.mpf(xe[2]), mp.mpf(xa[2])])
    S, Cs = rho / R, abs(d[2]) / R
    n_top = n(hi)
    p = mp.findroot(lambda pp: mp.quad(lambda z: pp / mp.sqrt(n(z) ** 2 - pp ** 2), [lo, hi]) - rho,
                    (0.5 * S * n_top, min(n_top * (1 - mp.mpf(10) ** -9), 2 * S * n_top)), solver="illinois")
    th_s = mp.asin(S)
    saved = mp.quad(lambda z: 2 * n(z) * mp.sin((mp.asin(p / n(z)) - th_s) / 2) ** 2 / Cs, [lo, hi])
    R_, _, _, d_ray = oracle.propagate(AIR_RAY, xe, xa)
    _, _, _, d_flat = oracle.propagate(AIR_FLAT, xe, xa)
    got = (d_flat - d_ray) * C  # metres of optical path saved
    assert saved > 0
    assert got == pytest.approx(float(saved), rel=1e-6, abs=1e-12)


def test_weak_refraction_scaling():
    """Halving the refractivity halves the bending at the source and quarters the
    time saved (both to first order in N0)."""
    xe, xa = GEOMETRIES[2]
    half = dict(AIR_RAY, N0=AIR_RAY["N0"] / 2)
    flat_half = dict(AIR_FLAT, N0=AIR_FLAT["N0"] / 2)
    d = (np.array(xa) - np.array(xe)) / np.linalg.norm(np.array(xa) - np.array(xe))
    ang = lambda med: math.acos(min(1.0, float(oracle.emission_direction(med, xe, xa) @ d)))
    saved = lambda med, flat: oracle.propagate(flat, xe, xa)[3] - oracle.propagate(med, xe, xa)[3]
    assert ang(half) / ang(AIR_RAY) == pytest.approx(0.5, rel=2e-3)
    assert saved(half, flat_half) / saved(AIR_RAY, AIR_FLAT) == pytest.approx(0.25, rel=2e-3)
    assert saved(AIR_RAY, AIR_FLAT) > 0


def test_vertical_and_near_horizontal_paths_stay_straight():
    for xe, xa in [([5.0, 5.0, 4000.0], [5.0, 5.0, 0.0]), ([0.0, 0.0, 10.0], [20000.0, 0.0, 0.0])]:
        rh = oracle.emission_direction(AIR_RAY, xe, xa)
        d = np.array(xa) - np.array(xe)
        assert np.abs(rh - d / np.linalg.norm(d)).max() < 1e-15
        # the delay is the integral of n along the straight line
        assert oracle.propagate(AIR_RAY, xe, xa)[3] == pytest.approx(oracle.propagate(AIR_FLAT, xe, xa)[3],
                                                                   rel=1e-13)
