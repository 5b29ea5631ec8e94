"""Pins of the FP64 oracle against things other than itself.

Each test fixes part of the oracle with an independent fact: a closed form
derived by hand for one geometry and evaluated in 50-digit mpmath, a brute-force
integration of the textbook Lienard-Wiechert radiation field, a quadrature, an
exact identity between two different code paths (Endpoint forced to the
midpoint vs the ZHS potential sampled at bin edges), or an invariant
(superposition, charge sign, rotation, time shift, collinear split, filter).
Central finite differences pin the hand-written adjoint.
"""
import math

import mpmath as mp
import numpy as np
import pytest

import oracle
from _util import AIR_EXP, AIR_UNIFORM, NEAR_CHERENKOV_CASES, near_cherenkov_pair

FIELDS = oracle.FIELDS
C = 299792458.0
QE = 1.602176634e-19
EPS0 = 8.8541878128e-12
MU0 = 1.0 / (EPS0 * C * C)


def one_track(x0, x1, t0, t1, beta, q=-1.0):
    vals = list(x0) + list(x1) + [t0, t1] + list(beta) + [q]
    return {f: np.array([float(v)], dtype=np.float64) for f, v in zip(FIELDS, vals)}


def cat(*ts):
    return {f: np.concatenate([t[f] for t in ts]) for f in FIELDS}


def rel_l2(a, b):
    d = np.linalg.norm((np.asarray(a) - np.asarray(b)).ravel())
    n = np.linalg.norm(np.asarray(b).ravel())
    return d / n if n > 0 else d


UNIFORM_AIR = {"kind": "uniform", "n": 1.000292}
EXP_AIR = {"kind": "exponential", "N0": 3.25e-4, "H": 8000.0}
ICE = {"kind": "uniform", "n": 1.78}


def random_tracks(n, seed, spread_deg=5.0, hmin=500.0, hmax=6000.0, L=(0.5, 5.0), gmin=10.0):
    rng = np.random.default_rng(seed)
    h = rng.uniform(hmin, hmax, n)
    r = rng.exponential(30.0, n)
    ph = rng.uniform(0, 2 * np.pi, n)
    ax = rng.normal(0, np.radians(spread_deg), n)
    ay = rng.normal(0, np.radians(spread_deg), n)
    u = np.stack([-np.cos(ax) * np.sin(ay), np.sin(ax), -np.cos(ax) * np.cos(ay)], 1)
    u /= np.linalg.norm(u, axis=1)[:, None]
    ln = rng.uniform(*L, n)
    g = np.exp(rng.uniform(np.log(gmin), np.log(1e4), n))
    b = np.sqrt(1 - 1 / g ** 2) * 0.9999999
    x0 = np.stack([r * np.cos(ph), r * np.sin(ph), h], 1)
    x1 = x0 + u * ln[:, None]
    t0 = (10000.0 - h) / C
    t1 = t0 + ln / (b * C)
    beta = u * b[:, None]
    q = np.where(rng.uniform(size=n) < 0.55, -1.0, 1.0)
    return {"x0": x0[:, 0], "y0": x0[:, 1], "z0": x0[:, 2], "x1": x1[:, 0], "y1": x1[:, 1], "z1": x1[:, 2],
            "t0": t0, "t1": t1, "bx": beta[:, 0], "by": beta[:, 1], "bz": beta[:, 2], "q": q}


def ground_antennas(radii, angles_deg):
    return np.array([[r * math.cos(math.radians(a)), r * math.sin(math.radians(a)), 0.0]
                     for r in radii for a in angles_deg])


def t_ref_for(ant, lead=50e-9):
    return np.full(len(ant), 10000.0 / C - lead)


# ---------------------------------------------------------------------------
# closed form: vertical track seen by one ground antenna, uniform medium
# ---------------------------------------------------------------------------
def closed_form_vertical(h, L, b, n, d, q, t0, dt, t_ref):
    """Hand-derived deposits of a track from (0,0,h) to (0,0,h-L) with beta=(0,0,-b),
    antenna at (d,0,0): R_j = sqrt(d^2+z_j^2), beta.rhat = b z_j/R_j,
    V = (b z_j d / R_j^2, 0, b d^2 / R_j^2), D_j = 1 - n b z_j / R_j."""
    mp.mp.dps = 50
    h, L, b, n, d, q, t0, dt, t_ref = map(mp.mpf, (h, L, b, n, d, q, t0, dt, t_ref))
    c, e, eps0 = mp.mpf(C), mp.mpf(QE), mp.mpf(EPS0)
    K = q * e / (4 * mp.pi * eps0 * c)
    z1 = h - L
    t1 = t0 + L / (b * c)
    out = []
    for s, z, t in ((1, h, t0), (-1, z1, t1)):
        R = mp.sqrt(d * d + z * z)
        D = 1 - n * b * z / R
        amp = s * K / (D * R * dt)
        u = (t - t_ref + n * R / c) / dt
        out.append((int(mp.floor(u)), amp * b * z * d / R ** 2, amp * b * d * d / R ** 2, D, u))
    return out


@pytest.mark.parametrize("n,d,b", [(1.000292, 1000.0, 0.99999), (1.78, 2000.0, 0.999), (1.0, 150.0, 0.95)])
def test_endpoint_closed_form_vertical(n, d, b):
    h, L, q, dt = 3000.0, 5.0, -1.0, 0.2e-9
    t0 = 0.0
    t1 = t0 + L / (b * C)
    R0 = math.hypot(d, h)
    t_ref = t0 + n * R0 / C - 100.3 * dt
    ref = closed_form_vertical(h, L, b, n, d, q, t0, dt, t_ref)
    assert all(abs(r[3]) > 2e-3 for r in ref)  # two-endpoint branch (eps_C = 1e-3)
    assert ref[0][0] != ref[1][0]
    tr = one_track((0, 0, h), (0, 0, h - L), t0, t1, (0, 0, -b), q)
    out, kept = oracle.forward(tr, [[d, 0, 0]], [t_ref], 4096, dt, {"kind": "uniform", "n": n})
    assert kept == 1
    for k, ex, ez, D, u in ref:
        assert 0 <= k < 4096
        frac = float(u - mp.floor(u))
        assert 1e-6 < frac < 1 - 1e-6
        assert out[0, 0, k] == pytest.approx(float(ex), rel=1e-13)
        assert out[0, 1, k] == 0.0
        assert out[0, 2, k] == pytest.approx(float(ez), rel=1e-13)
    mask = np.ones(4096, bool)
    mask[[ref[0][0], ref[1][0]]] = False
    assert not out[0][:, mask].any()


def test_endpoint_matches_lienard_wiechert_radiation():
    """Time integral of the textbook radiation field of a charge that ramps smoothly
    from rest to beta* (vacuum) equals the Endpoint start deposit times dt."""
    h, d, bstar, q, dt = 3000.0, 800.0, 0.9, -1.0, 0.2e-9
    tau = 1e-12
    u_hat = np.array([0.0, 0.0, -1.0])
    xs = np.array([0.0, 0.0, h])
    xa = np.array([d, 0.0, 0.0])
    s = np.linspace(0.0, 1.0, 200001)
    beta_s = bstar * (3 * s ** 2 - 2 * s ** 3)
    dbeta_s = bstar * (6 * s - 6 * s ** 2) / tau
    path = bstar * (s ** 3 - s ** 4 / 2) * tau * C
    x = xs[None, :] + path[:, None] * u_hat[None, :]
    dvec = xa[None, :] - x
    R = np.linalg.norm(dvec, axis=1)
    nh = dvec / R[:, None]
    beta = beta_s[:, None] * u_hat[None, :]
    bdot = dbeta_s[:, None] * u_hat[None, :]
    one_m = 1.0 - np.einsum("ij,ij->i", beta, nh)
    inner = np.cross(nh - beta, bdot)
    E_rad = q * QE / (4 * np.pi * EPS0 * C) * np.cross(nh, inner) / (one_m ** 3 * R)[:, None]
    integrand = E_rad * one_m[:, None]  # dt_obs = (1 - beta.n) dt'
    from scipy.integrate import simpson
    integral = np.array([simpson(integrand[:, k], x=s * tau) for k in range(3)])
    # Endpoint: a track that starts at xs with beta*, ends 3 m further down
    L = 3.0
    t1 = L / (bstar * C)
    R0 = np.linalg.norm(xa - xs)
    t_ref = R0 / C - 50.5 * dt
    tr = one_track(xs, xs + L * u_hat, 0.0, t1, bstar * u_hat, q)
    out, _ = oracle.forward(tr, [xa], [t_ref], 4096, dt, {"kind": "uniform", "n": 1.0})
    k0 = 50
    got = out[0, :, k0] * dt
    assert np.linalg.norm(got - integral) / np.linalg.norm(integral) < 1e-5
    assert got[0] != 0.0 and np.sign(got[0]) == np.sign(integral[0])


# ---------------------------------------------------------------------------
# ZHS
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("medium,d,b,L", [
    (UNIFORM_AIR, 300.0, 0.99999, 2.0),     # off-Cherenkov, a few bins
    (UNIFORM_AIR, 66.4, 0.9999999, 2.0),    # near-Cherenkov: single bin
    (ICE, 2000.0, 0.999, 3.0),              # inside the cone (D < 0), many bins
    (ICE, 5000.0, 0.999, 1.0),
])
def test_zhs_time_integral_closed_form(medium, d, b, L):
    """sum_k A_k dt = K_A |beta_perp| dt_e / R_m for a track inside the window, any D."""
    h, q, dt = 3000.0, 1.0, 0.2e-9
    n = medium["n"]
    zm = h - L / 2
    Rm = math.hypot(d, zm)
    t1 = L / (b * C)
    t_ref = 0.5 * t1 + n * Rm / C - 2000 * dt
    tr = one_track((0, 0, h), (0, 0, h - L), 0.0, t1, (0, 0, -b), q)
    out, _ = oracle.forward(tr, [[d, 0, 0]], [t_ref], 4096, dt, medium, formalism=oracle.ZHS)
    mp.mp.dps = 40
    KA = mp.mpf(MU0) * q * mp.mpf(QE) * mp.mpf(C) / (4 * mp.pi)
    R = mp.sqrt(mp.mpf(d) ** 2 + mp.mpf(zm) ** 2)
    # beta_perp = beta - (beta.rhat) rhat with rhat = (d, 0, -zm)/R, beta = (0,0,-b):
    bperp_x = -(b * zm / R) * d / R
    bperp_z = -b + (b * zm / R) * zm / R
    ex = float(KA * bperp_x * mp.mpf(t1) / R)
    ez = float(KA * bperp_z * mp.mpf(t1) / R)
    assert out[0, 0].sum() * dt == pytest.approx(ex, rel=1e-12)
    assert out[0, 2].sum() * dt == pytest.approx(ez, rel=1e-12)
    assert out[0, 1].sum() == 0.0


def test_zhs_matches_brute_force_sampling():
    """Bin averages of the midpoint step potential sampled on 1e4 points per bin."""
    tr = random_tracks(6, 7, spread_deg=25.0, L=(2.0, 5.0))
    ant = ground_antennas([200.0, 1500.0], [0.0, 120.0])
    dt, N = 0.2e-9, 4096
    t_ref = np.array([tr["t0"].min() + 1.78 * np.linalg.norm(a - [0, 0, 3000.0]) / C - 3000 * dt for a in ant])
    out, _ = oracle.forward(tr, ant, t_ref, N, dt, ICE, formalism=oracle.ZHS)
    br, u = oracle.arrivals(tr, ant, t_ref, N, dt, ICE, formalism=oracle.ZHS)
    KA = MU0 * QE * C / (4 * np.pi)
    sub = 10000
    for a in range(len(ant)):
        bf = np.zeros((3, N))
        for i in range(len(tr["x0"])):
            xm = np.array([tr["x0"][i] + tr["x1"][i], tr["y0"][i] + tr["y1"][i], tr["z0"][i] + tr["z1"][i]]) / 2
            beta = np.array([tr["bx"][i], tr["by"][i], tr["bz"][i]])
            dv = ant[a] - xm
            R = np.linalg.norm(dv)
            rh = dv / R
            D = 1 - ICE["n"] * beta @ rh
            bperp = beta - (beta @ rh) * rh
            height = tr["q"][i] * KA * bperp / (R * abs(D))
            ulo, uhi = u[i, a]
            for k in range(int(np.floor(ulo)), int(np.floor(uhi)) + 1):
                if not 0 <= k < N:
                    continue
                ts = k + (np.arange(sub) + 0.5) / sub
                frac = np.count_nonzero((ts >= ulo) & (ts < uhi)) / sub
                bf[:, k] += height * frac
        assert rel_l2(out[a], bf) < 1e-4


# ---------------------------------------------------------------------------
# exact identity between the two formalisms
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("medium", [UNIFORM_AIR, ICE, EXP_AIR])
def test_endpoint_midpoint_equals_minus_zhs_edge_difference(medium):
    """E_k = -(A(e_{k+1}) - A(e_k))/dt exactly, for Endpoint forced to midpoint form."""
    ant = ground_antennas([30.0, 150.0, 400.0], [0.0, 45.0, 200.0])
    dt, N = 0.2e-9, 4096
    if medium is ICE:  # dense medium: keep heights close so the arrivals fit one window
        tr = random_tracks(400, 11, spread_deg=8.0, hmin=2990.0, hmax=3010.0)
        t_ref = np.full(len(ant), (7000.0 + 1.78 * 3000.0) / C - 100e-9)
    else:
        tr = random_tracks(400, 11, spread_deg=8.0)
        t_ref = t_ref_for(ant)
    E, _ = oracle.forward(tr, ant, t_ref, N, dt, medium, oracle.ENDPOINT, mode=oracle.MODE_FORCE_MIDPOINT)
    A, _ = oracle.forward(tr, ant, t_ref, N, dt, medium, oracle.ZHS, mode=oracle.MODE_ZHS_EDGE_SAMPLED)
    E_from_A = -(A[:, :, 1:] - A[:, :, :-1]) / dt
    assert np.abs(E).max() > 0
    assert rel_l2(E[:, :, :-1], E_from_A) < 1e-12


def test_endpoint_vs_zhs_physical_agreement_off_cherenkov():
    """Production Endpoint (per-endpoint geometry) vs production ZHS (midpoint,
    bin-averaged) away from the Cherenkov angle: -dt*cumsum(E) tracks A within the
    O(L/R) geometry difference plus one-bin edge terms."""
    # long tracks: pulses ~60 bins wide, so the one-bin edge terms are a few per cent
    tr = random_tracks(200, 21, spread_deg=1.0, L=(15.0, 20.0), hmin=2995.0, hmax=3005.0)
    ant = ground_antennas([2500.0], [30.0])  # ~40 deg off axis: |D| ~ 0.2
    dt, N = 0.2e-9, 4096
    t_ref = np.array([(7000.0 + 1.000292 * math.hypot(2500.0, 3000.0)) / C - 1500 * dt])
    E, _ = oracle.forward(tr, ant, t_ref, N, dt, UNIFORM_AIR, oracle.ENDPOINT)
    A, _ = oracle.forward(tr, ant, t_ref, N, dt, UNIFORM_AIR, oracle.ZHS)
    br, u = oracle.arrivals(tr, ant, t_ref, N, dt, UNIFORM_AIR, oracle.ENDPOINT)
    assert (br == 0).all()
    assert (u > 0).all() and (u < N - 10).all()
    fromE = -dt * np.cumsum(E[0], axis=1)
    box = np.ones(5) / 5
    sm = lambda x: np.stack([np.convolve(x[c], box, mode="same") for c in range(3)])
    assert rel_l2(sm(fromE), sm(A[0])) < 5e-2


# ---------------------------------------------------------------------------
# invariants
# ---------------------------------------------------------------------------
def test_charge_flip_negates_exactly():
    tr = random_tracks(300, 3)
    ant = ground_antennas([50.0, 300.0], [0.0, 90.0])
    t_ref = t_ref_for(ant)
    for f in (oracle.ENDPOINT, oracle.ZHS):
        a, _ = oracle.forward(tr, ant, t_ref, 4096, 0.2e-9, EXP_AIR, f)
        tr2 = dict(tr)
        tr2["q"] = -tr["q"]
        b, _ = oracle.forward(tr2, ant, t_ref, 4096, 0.2e-9, EXP_AIR, f)
        assert np.array_equal(a, -b)


def test_superposition():
    tr = random_tracks(500, 4)
    ant = ground_antennas([50.0, 300.0], [0.0, 90.0])
    t_ref = t_ref_for(ant)
    A = {f: tr[f][:200] for f in FIELDS}
    B = {f: tr[f][200:] for f in FIELDS}
    for f in (oracle.ENDPOINT, oracle.ZHS):
        ab, _ = oracle.forward(tr, ant, t_ref, 4096, 0.2e-9, EXP_AIR, f)
        a, _ = oracle.forward(A, ant, t_ref, 4096, 0.2e-9, EXP_AIR, f)
        b, _ = oracle.forward(B, ant, t_ref, 4096, 0.2e-9, EXP_AIR, f)
        assert rel_l2(a + b, ab) < 1e-13


def test_rotation_about_vertical_axis():
    tr = random_tracks(300, 8)
    ant = ground_antennas([60.0, 250.0], [10.0, 100.0, 250.0])
    t_ref = t_ref_for(ant)
    phi = 0.7
    c, s = math.cos(phi), math.sin(phi)
    rot = lambda x, y: (c * x - s * y, s * x + c * y)
    tr2 = dict(tr)
    for p in ("0", "1"):
        tr2["x" + p], tr2["y" + p] = rot(tr["x" + p], tr["y" + p])
    tr2["bx"], tr2["by"] = rot(tr["bx"], tr["by"])
    ant2 = ant.copy()
    ant2[:, 0], ant2[:, 1] = rot(ant[:, 0], ant[:, 1])
    for f in (oracle.ENDPOINT, oracle.ZHS):
        br, u = oracle.arrivals(tr, ant, t_ref, 4096, 0.2e-9, EXP_AIR, f)
        fr = u - np.floor(u)
        assert (np.minimum(fr, 1 - fr)[br >= 0] > 1e-9).all()  # no edge-ambiguous deposit
        a, _ = oracle.forward(tr, ant, t_ref, 4096, 0.2e-9, EXP_AIR, f)
        b, _ = oracle.forward(tr2, ant2, t_ref, 4096, 0.2e-9, EXP_AIR, f)
        ax, ay = rot(a[:, 0], a[:, 1])
        assert rel_l2(np.stack([ax, ay, a[:, 2]], 1), b) < 1e-11


def test_time_shift_by_whole_bins_shifts_trace():
    tr = random_tracks(300, 9)
    ant = ground_antennas([60.0, 250.0], [10.0, 100.0])
    dt = 0.2e-9
    t_ref = t_ref_for(ant)
    m = 37
    tr2 = dict(tr)
    tr2["t0"] = tr["t0"] + m * dt
    tr2["t1"] = tr["t1"] + m * dt
    for f in (oracle.ENDPOINT, oracle.ZHS):
        br, u = oracle.arrivals(tr, ant, t_ref, 4096, dt, EXP_AIR, f)
        fr = u - np.floor(u)
        assert (np.minimum(fr, 1 - fr)[br >= 0] > 1e-9).all()
        assert (u[br >= 0] < 4096 - m - 1).all()
        a, _ = oracle.forward(tr, ant, t_ref, 4096, dt, EXP_AIR, f)
        b, _ = oracle.forward(tr2, ant, t_ref, 4096, dt, EXP_AIR, f)
        # Endpoint amplitudes do not depend on time; a ZHS interval split across a
        # bin edge moves with the last bits of the shifted arrival time
        assert rel_l2(b[:, :, m:], a[:, :, :-m]) < (1e-14 if f == oracle.ENDPOINT else 1e-9)
        assert not b[:, :, :m].any()


def test_collinear_split_leaves_endpoint_trace_unchanged():
    """Splitting a track at an interior point (same beta) cancels the interior pair."""
    tr = random_tracks(50, 12, spread_deg=1.0, hmin=2995.0, hmax=3005.0)
    ant = ground_antennas([1500.0], [0.0, 90.0])  # far off axis: two-endpoint branch everywhere
    t_ref = np.full(2, (7000.0 + 1.000292 * math.hypot(1500.0, 3000.0)) / C - 1500 * 0.2e-9)
    f = 0.37
    a_tr = dict(tr)
    b_tr = dict(tr)
    for c in "xyz":
        mid = tr[c + "0"] + f * (tr[c + "1"] - tr[c + "0"])
        a_tr[c + "1"] = mid
        b_tr[c + "0"] = mid
    tmid = tr["t0"] + f * (tr["t1"] - tr["t0"])
    a_tr["t1"] = tmid
    b_tr["t0"] = tmid
    whole, _ = oracle.forward(tr, ant, t_ref, 4096, 0.2e-9, UNIFORM_AIR)
    split, _ = oracle.forward(cat(a_tr, b_tr), ant, t_ref, 4096, 0.2e-9, UNIFORM_AIR)
    for t in (tr, a_tr, b_tr):
        br, _ = oracle.arrivals(t, ant, t_ref, 4096, 0.2e-9, UNIFORM_AIR)
        assert (br == 0).all()
    assert np.abs(whole).max() > 0
    assert rel_l2(split, whole) < 1e-12


def test_filter_drops_and_counts():
    good = one_track((0, 0, 3000), (0, 0, 2998), 0.0, 1e-8, (0, 0, -0.9), -1)
    bad = [
        one_track((0, 0, 3000), (0, 0, 2998), 0.0, 1e-8, (0, 0, -0.9), 0.0),       # neutral
        one_track((0, 0, 3000), (0, 0, 3000), 0.0, 1e-8, (0, 0, -0.9), -1),        # zero length
        one_track((0, 0, 3000), (0, 0, 2998), 0.0, 1e-8, (0, 0, -1.0), -1),        # |beta| = 1
        one_track((0, 0, 3000), (0, 0, 2998), 0.0, 1e-8, (0, 0, 0.0), -1),         # |beta| = 0
        one_track((0, 0, 3000), (0, 0, 2998), 1e-8, 1e-8, (0, 0, -0.9), -1),       # t1 == t0
        one_track((0, 0, np.nan), (0, 0, 2998), 0.0, 1e-8, (0, 0, -0.9), -1),      # NaN
        one_track((0, 0, 3000), (0, 0, 2998), 0.0, np.inf, (0, 0, -0.9), -1),      # inf
    ]
    ant = [[100.0, 0, 0]]
    t_ref = [3000.0 / C - 100e-9]
    ref, kept = oracle.forward(good, ant, t_ref, 4096, 0.2e-9, UNIFORM_AIR)
    assert kept == 1
    allt = cat(good, *bad)
    out, kept = oracle.forward(allt, ant, t_ref, 4096, 0.2e-9, UNIFORM_AIR)
    assert kept == 1
    assert np.array_equal(out, ref)
    assert oracle.keep_mask(allt).tolist() == [True] + [False] * len(bad)


def test_bins_outside_window_are_dropped():
    tr = one_track((0, 0, 3000), (0, 0, 2990), 0.0, 10 / (0.99 * C), (0, 0, -0.99), -1)
    ant = [[500.0, 0, 0]]
    R0 = math.hypot(500.0, 3000.0)
    dt = 0.2e-9
    # start arrives 0.5 bin before the window, end inside
    t_ref = [1.000292 * R0 / C + 0.5 * dt]
    out, _ = oracle.forward(tr, ant, t_ref, 4096, dt, UNIFORM_AIR)
    br, u = oracle.arrivals(tr, ant, t_ref, 4096, dt, UNIFORM_AIR)
    assert br[0, 0] == 0 and -1 < u[0, 0, 0] < 0 and 0 <= u[0, 0, 1] < 4096
    nz = np.nonzero(out[0].any(axis=0))[0]
    assert nz.tolist() == [int(np.floor(u[0, 0, 1]))]
    # both outside: nothing
    out2, _ = oracle.forward(tr, ant, [t_ref[0] - 1e-6], 4096, dt, UNIFORM_AIR)
    assert not out2.any()


# ---------------------------------------------------------------------------
# propagator
# ---------------------------------------------------------------------------
def test_uniform_propagation_delay():
    R, ns, na, delay = oracle.propagate(UNIFORM_AIR, [10.0, -20.0, 3000.0], [100.0, 50.0, 0.0])
    exp_R = math.sqrt(90.0 ** 2 + 70.0 ** 2 + 3000.0 ** 2)
    assert R == pytest.approx(exp_R, rel=1e-15)
    assert ns == na == 1.000292
    assert delay == pytest.approx(1.000292 * exp_R / C, rel=1e-15)


@pytest.mark.parametrize("ze,za", [(4000.0, 0.0), (9500.0, 100.0), (600.0, 580.0), (50.0, 1200.0)])
def test_exponential_path_average_matches_quadrature(ze, za):
    N0, H = EXP_AIR["N0"], EXP_AIR["H"]
    xe, xa = [30.0, 10.0, ze], [-200.0, 40.0, za]
    R, ns, na, delay = oracle.propagate(EXP_AIR, xe, xa)
    s = np.linspace(0.0, 1.0, 100001)
    z = ze + (za - ze) * s
    f = N0 * np.exp(-z / H)
    trap = (f[0] / 2 + f[1:-1].sum() + f[-1] / 2) * (s[1] - s[0])
    assert na - 1.0 == pytest.approx(trap, rel=1e-10)
    assert ns - 1.0 == pytest.approx(N0 * math.exp(-ze / H), rel=1e-14)
    assert delay == pytest.approx(na * R / C, rel=1e-15)


def test_exponential_path_average_continuous_at_equal_altitude():
    z = 1234.5
    vals = [oracle.propagate(EXP_AIR, [0, 0, z], [100.0, 0, z + dz])[2] - 1.0 for dz in (-1e-7, 0.0, 1e-7)]
    local = EXP_AIR["N0"] * math.exp(-z / EXP_AIR["H"])
    for v in vals:
        assert v == pytest.approx(local, rel=1e-10)


# ---------------------------------------------------------------------------
# reading MS: the exponential atmosphere over a spherical Earth
# ---------------------------------------------------------------------------
SPH_AIR = dict(kind="exponential_spherical", N0=3.25e-4, H=8000.0, R_E=6371e3)


def _sphere_h(x, R_E):
    x = [mp.mpf(float(v)) for v in x]
    return mp.sqrt(x[0] ** 2 + x[1] ** 2 + (x[2] + R_E) ** 2) - R_E


def test_spherical_emission_index_closed_form():
    mp.mp.dps = 40
    for xe in ([0.0, 0.0, 4000.0], [10000.0, 0.0, 0.0], [15000.0, -7000.0, 2500.0]):
        h = _sphere_h(xe, mp.mpf(SPH_AIR["R_E"]))
        n_src = 1 + mp.mpf(SPH_AIR["N0"]) * mp.exp(-h / SPH_AIR["H"])
        got = oracle.propagate(SPH_AIR, xe, [0.0, 0.0, 0.0])[1]
        assert abs(got - float(n_src)) <= 1e-15 * float(n_src)


def test_spherical_path_integral_against_mpmath_quadrature():
    mp.mp.dps = 30
    R_E, N0, H = mp.mpf(SPH_AIR["R_E"]), mp.mpf(SPH_AIR["N0"]), mp.mpf(SPH_AIR["H"])
    for xe, xa in (([9000.0, 3000.0, 5000.0], [120.0, -40.0, 0.0]), ([-20000.0, 500.0, 9000.0], [300.0, 800.0, 10.0])):
        d = [mp.mpf(b) - mp.mpf(a) for a, b in zip(xe, xa)]
        R = mp.sqrt(sum(v * v for v in d))

        def f(s):
            x = [mp.mpf(xe[k]) + s * d[k] / R for k in range(3)]
            return N0 * mp.exp(-(mp.sqrt(x[0] ** 2 + x[1] ** 2 + (x[2] + R_E) ** 2) - R_E) / H)

        F = mp.quad(f, [0, R / 2, R])
        got = oracle.propagate(SPH_AIR, xe, xa)
        assert got[0] == pytest.approx(float(R), rel=1e-15)
        assert (got[2] - 1.0) * got[0] == pytest.approx(float(F), rel=1e-12)


def test_spherical_radial_path_equals_flat_closed_form():
    """Along a vertical line through the sphere's centre the altitude is z itself,
    so the spherical path integral equals the flat closed form."""
    flat = dict(kind="exponential", N0=SPH_AIR["N0"], H=SPH_AIR["H"])
    for ze, za in ((500.0, 0.0), (4000.0, 0.0), (9000.0, 1200.0), (100.0, 3000.0)):
        a = oracle.propagate(flat, [0.0, 0.0, ze], [0.0, 0.0, za])
        b = oracle.propagate(SPH_AIR, [0.0, 0.0, ze], [0.0, 0.0, za])
        assert b[2] - 1.0 == pytest.approx(a[2] - 1.0, rel=1e-13)
        assert b[1] == pytest.approx(a[1], rel=1e-15)


def test_spherical_reduces_to_flat_for_a_large_radius():
    flat = dict(kind="exponential", N0=SPH_AIR["N0"], H=SPH_AIR["H"])
    big = dict(SPH_AIR, R_E=1e13)
    for xe, xa in (([9000.0, 3000.0, 5000.0], [120.0, -40.0, 0.0]), ([-20000.0, 500.0, 9000.0], [300.0, 800.0, 10.0])):
        a = oracle.propagate(flat, xe, xa)
        b = oracle.propagate(big, xe, xa)
        c = oracle.propagate(SPH_AIR, xe, xa)
        assert abs(b[2] - a[2]) <= 1e-9 * (a[2] - 1.0)
        assert abs(c[2] - a[2]) > 1e-5 * (a[2] - 1.0)  # at the real radius the curvature shows


def test_spherical_path_integral_symmetric_and_additive():
    xa, xb = np.array([-15000.0, 4000.0, 8000.0]), np.array([200.0, -100.0, 0.0])
    fwd = oracle.propagate(SPH_AIR, xa, xb)
    rev = oracle.propagate(SPH_AIR, xb, xa)
    assert rev[2] == pytest.approx(fwd[2], rel=1e-15)
    F = (fwd[2] - 1.0) * fwd[0]
    for lam in (0.2, 0.5, 0.77):
        xm = xa + lam * (xb - xa)
        p1 = oracle.propagate(SPH_AIR, xa, xm)
        p2 = oracle.propagate(SPH_AIR, xm, xb)
        # the quadrature is good to ~1e-13 (pinned against mpmath above); a sum of
        # two adds their errors
        assert (p1[2] - 1.0) * p1[0] + (p2[2] - 1.0) * p2[0] == pytest.approx(F, rel=2e-12)


# ---------------------------------------------------------------------------
# adjoint vs central finite differences
# ---------------------------------------------------------------------------
def _loss(tr, ant, t_ref, medium, G, dt, N):
    out, _ = oracle.forward(tr, ant, t_ref, N, dt, medium)
    return float((out * G).sum())


@pytest.mark.parametrize("medium", [EXP_AIR, UNIFORM_AIR])
def test_adjoint_matches_central_differences(medium):
    tr = random_tracks(5, 31, spread_deg=6.0)
    ant = ground_antennas([40.0, 200.0], [0.0, 130.0])
    dt, N = 0.2e-9, 4096
    t_ref = t_ref_for(ant)
    rng = np.random.default_rng(2)
    out, _ = oracle.forward(tr, ant, t_ref, N, dt, medium)
    G = rng.normal(size=out.shape) * (np.abs(out) > 0)
    G += 0.1 * rng.normal(size=out.shape)
    tg, ag, dN = oracle.backward(tr, ant, t_ref, N, dt, medium, G)
    br0, u0 = oracle.arrivals(tr, ant, t_ref, N, dt, medium)
    assert (br0 == 1).any() and (br0 == 0).any()  # both branches exercised

    def same_bins(t2, a2=ant, m2=medium):
        br, u = oracle.arrivals(t2, a2, t_ref, N, dt, m2)
        return np.array_equal(br, br0) and np.array_equal(np.floor(u), np.floor(u0))

    # absolute FD rounding noise of the summed loss at step h: ~eps * sum|trace*G| / h
    l1 = float(np.abs(out * G).sum())

    gscale = {"pos": np.abs(np.concatenate([tg[:, :6].ravel(), ag.ravel()])).max(), "beta": np.abs(tg[:, 8:]).max()}

    def close(fd, adj, h, kind="pos"):
        # at step 1e-6 the FD quotient carries ~1e-6..1e-4 of rounding noise (the
        # traces are sums of large start/end deposits that nearly cancel); the noise
        # scales with the loss's overall sensitivity, so the floor uses the largest
        # gradient component of the same kind
        return abs(fd - adj) <= 1e-4 * abs(adj) + 1e-6 * gscale[kind] + 100 * 2.2e-16 * l1 / h

    checked = skipped = 0
    names = ["x0", "y0", "z0", "x1", "y1", "z1", "t0", "t1", "bx", "by", "bz"]
    for i in range(len(tr["x0"])):
        for j, f in enumerate(names):
            v = tr[f][i]
            h = 1e-6 * max(abs(v), 1e-3) if f[0] != "t" else 1e-6 * 1e-9
            tp, tm = dict(tr), dict(tr)
            tp[f] = tr[f].copy(); tp[f][i] = v + h
            tm[f] = tr[f].copy(); tm[f][i] = v - h
            if not (same_bins(tp) and same_bins(tm)):
                skipped += 1
                continue
            fd = (_loss(tp, ant, t_ref, medium, G, dt, N) - _loss(tm, ant, t_ref, medium, G, dt, N)) / (2 * h)
            if f[0] == "t":
                assert fd == 0.0 and tg[i, j] == 0.0
            else:
                assert close(fd, tg[i, j], h, "beta" if f[0] == "b" else "pos"), (i, f, fd, tg[i, j])
            checked += 1
    for a in range(len(ant)):
        for k in range(3):
            h = 1e-6 * max(np.linalg.norm(ant[a]), 1.0)  # relative to the antenna's distance
            ap, am = ant.copy(), ant.copy()
            ap[a, k] += h
            am[a, k] -= h
            if not (same_bins(tr, ap) and same_bins(tr, am)):
                skipped += 1
                continue
            fd = (_loss(tr, ap, t_ref, medium, G, dt, N) - _loss(tr, am, t_ref, medium, G, dt, N)) / (2 * h)
            assert close(fd, ag[a, k], h), (a, k, fd, ag[a, k])
            checked += 1
    key = "N0" if medium["kind"] == "exponential" else "n"
    h = 1e-6 * (medium[key] if key == "N0" else medium["n"] - 1)
    mp_, mm_ = dict(medium), dict(medium)
    mp_[key] += h
    mm_[key] -= h
    if same_bins(tr, ant, mp_) and same_bins(tr, ant, mm_):
        fd = (_loss(tr, ant, t_ref, mp_, G, dt, N) - _loss(tr, ant, t_ref, mm_, G, dt, N)) / (2 * h)
        assert close(fd, dN, h), (fd, dN)
        checked += 1
    assert checked > 5 * skipped


def _loss_zhs(tr, ant, t_ref, medium, G, dt, N):
    out, _ = oracle.forward(tr, ant, t_ref, N, dt, medium, oracle.ZHS)
    return float((out * G).sum())


@pytest.mark.parametrize("medium", [EXP_AIR, UNIFORM_AIR])
def test_zhs_adjoint_matches_central_differences(medium):
    """Reading GZ: with the bins of the interval ends held fixed the ZHS traces are
    smooth in every input, times included; central differences that keep those
    bins pin every component of the hand-written gradient."""
    tr = random_tracks(5, 37, spread_deg=6.0)
    ant = ground_antennas([40.0, 200.0], [0.0, 130.0])
    dt, N = 0.2e-9, 4096
    t_ref = t_ref_for(ant)
    rng = np.random.default_rng(3)
    out, _ = oracle.forward(tr, ant, t_ref, N, dt, medium, oracle.ZHS)
    G = rng.normal(size=out.shape) * (np.abs(out) > 0)
    G += 0.1 * rng.normal(size=out.shape)
    tg, ag, dN = oracle.backward(tr, ant, t_ref, N, dt, medium, G, formalism=oracle.ZHS)
    br0, u0 = oracle.arrivals(tr, ant, t_ref, N, dt, medium, oracle.ZHS)
    assert (br0 == 3).any()  # multi-bin intervals: the weights vary with the times

    def same_bins(t2, a2=ant, m2=medium):
        br, u = oracle.arrivals(t2, a2, t_ref, N, dt, m2, oracle.ZHS)
        return np.array_equal(br, br0) and np.array_equal(np.floor(u), np.floor(u0))

    l1 = float(np.abs(out * G).sum())
    gs = {"pos": np.abs(np.concatenate([tg[:, :6].ravel(), ag.ravel()])).max(), "t": np.abs(tg[:, 6:8]).max(),
          "beta": np.abs(tg[:, 8:]).max()}
    assert gs["t"] > 0  # the times do get gradients

    def close(fd, adj, h, kind):
        return abs(fd - adj) <= 1e-5 * abs(adj) + 1e-7 * gs[kind] + 100 * 2.2e-16 * l1 / h

    checked = skipped = 0
    names = ["x0", "y0", "z0", "x1", "y1", "z1", "t0", "t1", "bx", "by", "bz"]
    for i in range(len(tr["x0"])):
        for j, f in enumerate(names):
            v = tr[f][i]
            h = 1e-6 * max(abs(v), 1e-3) if f[0] != "t" else 1e-6 * 1e-9
            tp, tm = dict(tr), dict(tr)
            tp[f] = tr[f].copy(); tp[f][i] = v + h
            tm[f] = tr[f].copy(); tm[f][i] = v - h
            if not (same_bins(tp) and same_bins(tm)):
                skipped += 1
                continue
            fd = (_loss_zhs(tp, ant, t_ref, medium, G, dt, N) - _loss_zhs(tm, ant, t_ref, medium, G, dt, N)) / (2 * h)
            kind = {"t": "t", "b": "beta"}.get(f[0], "pos")
            assert close(fd, tg[i, j], h, kind), (i, f, fd, tg[i, j])
            checked += 1
    for a in range(len(ant)):
        for k in range(3):
            h = 1e-6 * max(np.linalg.norm(ant[a]), 1.0)
            ap, am = ant.copy(), ant.copy()
            ap[a, k] += h
            am[a, k] -= h
            if not (same_bins(tr, ap) and same_bins(tr, am)):
                skipped += 1
                continue
            fd = (_loss_zhs(tr, ap, t_ref, medium, G, dt, N) - _loss_zhs(tr, am, t_ref, medium, G, dt, N)) / (2 * h)
            assert close(fd, ag[a, k], h, "pos"), (a, k, fd, ag[a, k])
            checked += 1
    key = "N0" if medium["kind"] == "exponential" else "n"
    h = 1e-6 * (medium[key] if key == "N0" else medium["n"] - 1)
    mp_, mm_ = dict(medium), dict(medium)
    mp_[key] += h
    mm_[key] -= h
    if same_bins(tr, ant, mp_) and same_bins(tr, ant, mm_):
        fd = (_loss_zhs(tr, ant, t_ref, mp_, G, dt, N) - _loss_zhs(tr, ant, t_ref, mm_, G, dt, N)) / (2 * h)
        assert abs(fd - dN) <= 1e-5 * abs(dN) + 100 * 2.2e-16 * l1 / h, (fd, dN)
        checked += 1
    assert checked > 5 * skipped


def test_abs_mode_bounds_the_signed_traces():
    """MODE_ABS sums |deposit|: it bounds |trace| bin by bin and equals it where a
    bin holds a single deposit."""
    tr = random_tracks(50, 41)
    ant = ground_antennas([60.0, 300.0], [0.0, 90.0])
    t_ref = t_ref_for(ant)
    for f in (oracle.ENDPOINT, oracle.ZHS):
        s, _ = oracle.forward(tr, ant, t_ref, 4096, 0.2e-9, EXP_AIR, f)
        a, _ = oracle.forward(tr, ant, t_ref, 4096, 0.2e-9, EXP_AIR, f, mode=oracle.MODE_ABS)
        assert (a >= np.abs(s) * (1 - 1e-12)).all()
        one = {k: v[:1] for k, v in tr.items()}
        s1, _ = oracle.forward(one, ant[:1], t_ref[:1], 4096, 0.2e-9, EXP_AIR, f)
        a1, _ = oracle.forward(one, ant[:1], t_ref[:1], 4096, 0.2e-9, EXP_AIR, f, mode=oracle.MODE_ABS)
        br, u = oracle.arrivals(one, ant[:1], t_ref[:1], 4096, 0.2e-9, EXP_AIR, f)
        if f == oracle.ENDPOINT and br[0, 0] == 0 and np.floor(u[0, 0, 0]) != np.floor(u[0, 0, 1]):
            assert np.array_equal(a1, np.abs(s1))


# ---------------------------------------------------------------------------
# constructed near-Cherenkov pairs (the branch of reading C), one-bin deposit
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("medium_name,D,place", NEAR_CHERENKOV_CASES)
def test_constructed_near_cherenkov_pairs(medium_name, D, place):
    """A track at D_m = +-1e-4 or +-1e-6 from one antenna: the Endpoint pair
    takes the midpoint branch; with both linearised arrivals in one bin it gives
    exactly 0, otherwise +-K V/(D R dt) in the two bins, equal to the negative
    time difference of the edge-sampled ZHS potential; the ZHS deposit over the
    same tiny interval keeps the closed-form time integral K_A |beta_perp|
    (t1 - t0)/R_m, in one bin or split evenly over the two bins at the edge."""
    medium = AIR_UNIFORM if medium_name == "uniform" else AIR_EXP
    N, K, dtn = 64, 32, 0.2
    trn, ant, t_start = near_cherenkov_pair(D, place, medium, n_bins=N, K=K, dt_ns=dtn)
    tr = oracle.tracks_from_ns(trn)
    dt, t_ref = dtn * 1e-9, t_start * 1e-9
    br, u = oracle.arrivals(tr, ant, t_ref, N, dt, medium, oracle.ENDPOINT)
    assert br[0, 0] == 1
    du = abs(u[0, 0, 1] - u[0, 0, 0])
    assert du == pytest.approx(abs(D) * (tr["t1"][0] - tr["t0"][0]) / dt, rel=1e-3)
    E, _ = oracle.forward(tr, ant, t_ref, N, dt, medium, oracle.ENDPOINT)
    A_edge, _ = oracle.forward(tr, ant, t_ref, N, dt, medium, oracle.ZHS, mode=oracle.MODE_ZHS_EDGE_SAMPLED)
    if place == "same":
        assert not E.any()
    else:
        nz = np.flatnonzero(np.abs(E[0]).sum(axis=0))
        assert list(nz) == [K - 1, K]
        np.testing.assert_array_equal(E[0, :, K - 1], -E[0, :, K])
        E_from_A = -(A_edge[:, :, 1:] - A_edge[:, :, :-1]) / dt
        assert rel_l2(E[:, :, :-1], E_from_A) < 1e-12
    # ZHS: the time integral in closed form (50 digits), one bin or two halves
    Z, _ = oracle.forward(tr, ant, t_ref, N, dt, medium, oracle.ZHS)
    mp.mp.dps = 50
    KA = mp.mpf(MU0) * 1 * mp.mpf(QE) * mp.mpf(C) / (4 * mp.pi)  # |q| = 1; q = -1 flips the sign
    zm = (mp.mpf(tr["z0"][0]) + mp.mpf(tr["z1"][0])) / 2
    dx = mp.mpf(ant[0, 0])
    R = mp.sqrt(dx ** 2 + zm ** 2)
    b = -mp.mpf(tr["bz"][0])
    dte = mp.mpf(tr["t1"][0]) - mp.mpf(tr["t0"][0])
    # beta = (0, 0, -b), rhat = (dx, 0, -zm)/R: beta_perp = beta - (beta.rhat) rhat
    bpx = -(b * zm / R) * dx / R
    bpz = -b + (b * zm / R) * zm / R
    ex, ez = float(-KA * bpx * dte / R), float(-KA * bpz * dte / R)
    assert Z[0, 0].sum() * dt == pytest.approx(ex, rel=1e-12)
    assert Z[0, 2].sum() * dt == pytest.approx(ez, rel=1e-12)
    nz = np.flatnonzero(np.abs(Z[0]).sum(axis=0))
    if place == "same":
        assert list(nz) == [K]
    else:
        assert list(nz) == [K - 1, K]
        # the interval is split by the edge in halves (to the placement's rounding, ~1e-12 bin)
        assert Z[0, 2, K - 1] == pytest.approx(Z[0, 2, K], rel=1e-12 / du + 1e-12)
