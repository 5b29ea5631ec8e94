"""Pins of the oracle's linear (two-bin) deposit, reading LD, against things other
than itself.

Spreading a deposit evenly over one bin width centred on its arrival is the
same as averaging the one-bin (reading T) traces over window starts shifted by
s dt, s uniform in [-1/2, 1/2]: a deposit at u lands in bin floor(u - s), and
the measure of the shifts that put it in bin k is the linear weight of bin k.
So the linear traces of both formalisms, the near-Cherenkov branch included,
are pinned by integrating the one-bin oracle over s exactly (it is piecewise
constant in s for Endpoint and piecewise linear for ZHS, with breakpoints where
an arrival crosses a bin edge, so the midpoint rule on each piece is exact).
The near-Cherenkov Endpoint form is also pinned by an identity with the one-bin
ZHS potential on a grid shifted by half a bin, and the adjoints by central
differences (the times now have informative gradients).
"""
import numpy as np
import pytest

import oracle
from test_oracle_pins import EXP_AIR, ICE, UNIFORM_AIR, cat, ground_antennas, random_tracks, rel_l2, t_ref_for

LIN, BIN = oracle.DEPOSIT_LINEAR, oracle.DEPOSIT_BIN


def case(medium, spread, seed, n, ant, dt, lead_bins=250):
    """Random tracks and per-antenna window starts lead_bins before the first
    arrival; in ice (n = 1.78) the tracks start 100-130 m up so that their
    arrivals fit a window of a few thousand bins."""
    if medium is ICE:
        tr = random_tracks(n, seed, spread_deg=spread, hmin=100.0, hmax=130.0)
    else:
        tr = random_tracks(n, seed, spread_deg=spread)
    _, u = oracle.arrivals(tr, ant, np.zeros(len(ant)), 1, dt, medium, oracle.ZHS)
    return tr, u.min(axis=(0, 2)) * dt - lead_bins * dt


def _breakpoints(tr, ant, t_ref, N, dt, medium, formalism, eps_C):
    """Shifts s in (-1/2, 1/2) at which some arrival of the one-bin evaluation
    crosses a bin edge (u - s integer)."""
    _, u = oracle.arrivals(tr, ant, t_ref, N, dt, medium, formalism, eps_C)
    u = u.ravel()
    f = u - np.floor(u)  # in [0, 1): crossings at s = f and s = f - 1
    s = np.concatenate([f, f - 1.0])
    return np.unique(s[(s > -0.5) & (s < 0.5)])


def shift_average(tr, ant, t_ref, N, dt, medium, formalism, eps_C=1e-3, mode=oracle.MODE_NORMAL):
    """Integral over s in [-1/2, 1/2] of the one-bin traces with the window start
    moved by s dt, piece by piece between the breakpoints."""
    edges = np.concatenate([[-0.5], _breakpoints(tr, ant, t_ref, N, dt, medium, formalism, eps_C), [0.5]])
    acc = 0.0
    for a, b in zip(edges[:-1], edges[1:]):
        if b - a < 1e-12:
            continue
        s = 0.5 * (a + b)
        out, _ = oracle.forward(tr, ant, np.asarray(t_ref) + s * dt, N, dt, medium, formalism, eps_C, mode, BIN)
        acc = acc + (b - a) * out
    return acc


@pytest.mark.parametrize("formalism", [oracle.ENDPOINT, oracle.ZHS])
@pytest.mark.parametrize("medium,spread", [(EXP_AIR, 5.0), (UNIFORM_AIR, 5.0), (ICE, 40.0)])
def test_linear_equals_one_bin_averaged_over_window_shifts(formalism, medium, spread):
    ant = ground_antennas([25.0, 120.0, 300.0], [0.0, 200.0])
    dt, N = 0.2e-9, 4096
    tr, t_ref = case(medium, spread, 71, 6, ant, dt)
    eps_C = 0.05 if medium is ICE else 1e-3  # in ice: many pairs in the near-Cherenkov branch
    lin, _ = oracle.forward(tr, ant, t_ref, N, dt, medium, formalism, eps_C, deposit=LIN)
    avg = shift_average(tr, ant, t_ref, N, dt, medium, formalism, eps_C)
    assert np.abs(lin).max() > 0
    assert rel_l2(lin, avg) < 1e-11
    br, _ = oracle.arrivals(tr, ant, t_ref, N, dt, medium, formalism, eps_C)
    if medium is ICE and formalism == oracle.ENDPOINT:
        assert (br == 1).any()  # the near-Cherenkov branch is part of the check


def test_linear_near_cherenkov_pairs_average_over_shifts():
    """Tracks built to sit at the Cherenkov angle of an antenna (D_m from 1e-4 to
    1e-7, both signs), with their arrivals both between the same two bin centres
    (the exact limit) and on either side of one (the two spread deposits)."""
    ant = np.array([[0.0, 0.0, 0.0]])
    dt, N = 0.2e-9, 2048
    C = 299792458.0
    rng = np.random.default_rng(12)
    tr = near_cherenkov_tracks([1e-4, -1e-4, 1e-6, -1e-6, 3e-5, -2e-7, 1e-7, 5e-5], 0.1, 6, rng)
    t_ref = [1e-7 + 100.0 * 1.78 / C - 50e-9]
    # move every other track in time so that its two arrivals straddle a bin centre
    _, u = oracle.arrivals(tr, ant, t_ref, N, dt, ICE, oracle.ENDPOINT)
    um, du = u[:, 0].mean(axis=1), np.abs(u[:, 0, 1] - u[:, 0, 0])
    move = (np.floor(um) + 0.5 + rng.uniform(-0.4, 0.4, len(um)) * du - um) * dt
    move[::2] = 0.0
    tr["t0"] = tr["t0"] + move
    tr["t1"] = tr["t1"] + move
    br, u = oracle.arrivals(tr, ant, t_ref, N, dt, ICE, oracle.ENDPOINT)
    assert (br == 1).all()
    same = np.floor(u[..., 0] + 0.5) == np.floor(u[..., 1] + 0.5)
    assert same.any() and (~same).any()
    # track by track: the shift average integrates +/-K V/(D R dt) over shifts
    # whose range is the arrival separation |du|, itself a difference of
    # arrivals ~500 bins from the window start (rounding ~1e-13 bin), so it
    # carries a relative error ~1e-13/|du|; the linear form has no such division
    for i in range(len(tr["x0"])):
        one = {f: tr[f][i:i + 1] for f in oracle.FIELDS}
        lin, _ = oracle.forward(one, ant, t_ref, N, dt, ICE, oracle.ENDPOINT, deposit=LIN)
        avg = shift_average(one, ant, t_ref, N, dt, ICE, oracle.ENDPOINT)
        du = abs(u[i, 0, 1] - u[i, 0, 0])
        assert np.abs(lin).max() > 0
        assert rel_l2(lin, avg) < 1e-12 + 4e-13 / du, (i, du)


@pytest.mark.parametrize("medium", [ICE, EXP_AIR])
def test_linear_midpoint_endpoint_equals_minus_half_shifted_zhs_difference(medium):
    """Endpoint forced to its midpoint form with the linear deposit gives
    E_k = -(A'_{k+1} - A'_k)/dt, where A' is the one-bin ZHS potential on the
    grid whose bin j covers [k - 1/2, k + 1/2) of the original bins."""
    ant = ground_antennas([30.0, 150.0], [0.0, 90.0, 250.0])
    dt, N = 0.2e-9, 4096
    tr, t_ref = case(medium, 35.0 if medium is ICE else 5.0, 5, 60, ant, dt)
    _, u = oracle.arrivals(tr, ant, t_ref, N, dt, medium, oracle.ZHS)
    W = u[..., 1] - u[..., 0]  # interval widths in bins, [track, antenna]
    for i in range(len(tr["x0"])):
        one = {f: tr[f][i:i + 1] for f in oracle.FIELDS}
        E, _ = oracle.forward(one, ant, t_ref, N, dt, medium, oracle.ENDPOINT, mode=oracle.MODE_FORCE_MIDPOINT,
                              deposit=LIN)
        A, _ = oracle.forward(one, ant, np.asarray(t_ref) - 0.5 * dt, N + 1, dt, medium, oracle.ZHS)
        rhs = -(A[..., 1:] - A[..., :-1]) / dt
        assert np.abs(E).max() > 0
        # both sides place the interval ends (times ~4e-7 s, ulp ~3e-13 bin, a
        # few roundings on each side: ~1e-12 bin) and divide by its width W in
        # different orders; the one-bin ZHS overlaps of whole bins,
        # (k + 1) dt - k dt, are dt to a few ulps
        err = np.abs(E - rhs).max() / np.abs(E).max()
        assert err < 4e-12 + 4e-12 / W[i].min(), (i, W[i].min(), err)


@pytest.mark.parametrize("formalism", [oracle.ENDPOINT, oracle.ZHS])
def test_linear_keeps_the_time_integral(formalism):
    """Spreading moves no weight out of the window: for tracks whose deposits stay
    clear of the window ends the sum over bins equals the one-bin sum."""
    tr = random_tracks(10, 9)
    ant = ground_antennas([50.0, 250.0], [0.0, 45.0])
    dt, N = 0.2e-9, 8192
    t_ref = t_ref_for(ant, lead=300e-9)
    lin, _ = oracle.forward(tr, ant, t_ref, N, dt, EXP_AIR, formalism, deposit=LIN)
    one, _ = oracle.forward(tr, ant, t_ref, N, dt, EXP_AIR, formalism)
    _, u = oracle.arrivals(tr, ant, t_ref, N, dt, EXP_AIR, formalism)
    assert u.min() > 2 and u.max() < N - 2
    mag, _ = oracle.forward(tr, ant, t_ref, N, dt, EXP_AIR, formalism, mode=oracle.MODE_ABS)
    assert np.abs(lin.sum(-1) - one.sum(-1)).max() <= 1e-13 * mag.sum(-1).max()
    assert not np.array_equal(lin, one)


def _loss(tr, ant, t_ref, medium, G, dt, N, formalism, eps_C):
    out, _ = oracle.forward(tr, ant, t_ref, N, dt, medium, formalism, eps_C, deposit=LIN)
    return float((out * G).sum())


def _fd_check(tr, ant, t_ref, N, dt, medium, formalism, eps_C, seed):
    """Central differences of the linear-deposit loss against the oracle's
    adjoint, for every track field, antenna coordinate and N0; steps whose
    arrivals would cross a bin centre (a kink of the linear weights) or change
    the branch are left out.  Returns (branch codes, checked, skipped)."""
    rng = np.random.default_rng(seed)
    out, _ = oracle.forward(tr, ant, t_ref, N, dt, medium, formalism, eps_C, deposit=LIN)
    G = rng.normal(size=out.shape) * (np.abs(out) > 0)
    G += 0.1 * rng.normal(size=out.shape)
    tg, ag, dN = oracle.backward(tr, ant, t_ref, N, dt, medium, G, eps_C, formalism=formalism, deposit=LIN)
    br0, u0 = oracle.arrivals(tr, ant, t_ref, N, dt, medium, formalism, eps_C)

    def cells(u):
        return np.floor(u - 0.5), np.floor(u + 0.5)

    c0 = cells(u0)

    def same_cells(t2, a2=ant, m2=medium):
        br, u = oracle.arrivals(t2, a2, t_ref, N, dt, m2, formalism, eps_C)
        c = cells(u)
        return np.array_equal(br == 1, br0 == 1) and all(np.array_equal(x, y) for x, y in zip(c, c0))

    def loss(t2, a2=ant, m2=medium):
        o, _ = oracle.forward(t2, a2, t_ref, N, dt, m2, formalism, eps_C, deposit=LIN)
        return float((o * G).sum())

    l1 = float(np.abs(out * G).sum())
    gs = {"pos": np.abs(np.concatenate([tg[:, :6].ravel(), ag.ravel()])).max(), "t": np.abs(tg[:, 6:8]).max(),
          "beta": np.abs(tg[:, 8:]).max()}
    assert gs["t"] > 0  # the times get gradients

    def close(fd, adj, h, kind):
        return abs(fd - adj) <= 1e-4 * abs(adj) + 1e-6 * gs[kind] + 100 * 2.2e-16 * l1 / h

    checked = skipped = 0
    names = ["x0", "y0", "z0", "x1", "y1", "z1", "t0", "t1", "bx", "by", "bz"]
    for i in range(len(tr["x0"])):
        for j, f in enumerate(names):
            v = tr[f][i]
            h = 1e-6 * max(abs(v), 1e-3) if f[0] != "t" else 1e-6 * 1e-9
            tp, tm = dict(tr), dict(tr)
            tp[f] = tr[f].copy(); tp[f][i] = v + h
            tm[f] = tr[f].copy(); tm[f][i] = v - h
            if not (same_cells(tp) and same_cells(tm)):
                skipped += 1
                continue
            fd = (loss(tp) - loss(tm)) / (2 * h)
            kind = {"t": "t", "b": "beta"}.get(f[0], "pos")
            assert close(fd, tg[i, j], h, kind), (i, f, fd, tg[i, j])
            checked += 1
    for a in range(len(ant)):
        for k in range(3):
            h = 1e-6 * max(np.linalg.norm(ant[a]), 1.0)
            ap, am = ant.copy(), ant.copy()
            ap[a, k] += h
            am[a, k] -= h
            if not (same_cells(tr, ap) and same_cells(tr, am)):
                skipped += 1
                continue
            fd = (loss(tr, ap) - loss(tr, am)) / (2 * h)
            assert close(fd, ag[a, k], h, "pos"), (a, k, fd, ag[a, k])
            checked += 1
    key = "N0" if medium["kind"] == "exponential" else "n"
    h = 1e-6 * (medium[key] if key == "N0" else medium["n"] - 1)
    mp_, mm_ = dict(medium), dict(medium)
    mp_[key] += h
    mm_[key] -= h
    if same_cells(tr, ant, mp_) and same_cells(tr, ant, mm_):
        fd = (loss(tr, ant, mp_) - loss(tr, ant, mm_)) / (2 * h)
        assert close(fd, dN, h, "pos"), (fd, dN)
        checked += 1
    return br0, u0, checked, skipped


@pytest.mark.parametrize("formalism", [oracle.ENDPOINT, oracle.ZHS])
@pytest.mark.parametrize("medium,spread", [(EXP_AIR, 6.0), (UNIFORM_AIR, 6.0), (ICE, 40.0)])
def test_linear_adjoint_matches_central_differences(formalism, medium, spread):
    """The hand-written adjoint of the linear deposit against central differences."""
    ant = ground_antennas([40.0, 200.0], [0.0, 130.0])
    dt, N = 0.2e-9, 4096
    tr, t_ref = case(medium, spread, 43, 5, ant, dt)
    eps_C = 0.05 if medium is ICE else 1e-3
    br0, _, checked, skipped = _fd_check(tr, ant, t_ref, N, dt, medium, formalism, eps_C, 4)
    if formalism == oracle.ENDPOINT and medium is ICE:
        assert (br0 == 1).any()
    assert checked > 5 * skipped


def near_cherenkov_tracks(D_values, L, per_D, rng, n=1.78, b=0.9995, R=100.0):
    """Downward tracks whose midpoint sees the antenna at the origin at an angle
    with 1 - n b cos(theta) = D."""
    C = 299792458.0
    trs = []
    for D in D_values:
        for _ in range(per_D):
            cos_t = (1.0 - D) / (n * b)
            sin_t = np.sqrt(1.0 - cos_t ** 2)
            Rk = R + rng.uniform(0, 0.3)
            xm = np.array([-Rk * sin_t, 0.0, Rk * cos_t])  # rhat = (sin theta, 0, -cos theta)
            u = np.array([0.0, 0.0, -1.0])
            x0, x1 = xm - 0.5 * L * u, xm + 0.5 * L * u
            t0 = 1e-7 + rng.uniform(0, 1e-9)
            t1 = t0 + L / (b * C)
            vals = list(x0) + list(x1) + [t0, t1] + list(b * u) + [-1.0]
            trs.append({f: np.array([v]) for f, v in zip(oracle.FIELDS, vals)})
    return cat(*trs)


def test_linear_near_cherenkov_adjoint_matches_central_differences():
    """Near-Cherenkov Endpoint pairs of both kinds (arrivals between the same two
    bin centres, and on either side of one) under central differences."""
    rng = np.random.default_rng(21)
    ant = np.array([[0.0, 0.0, 0.0]])
    dt, N, eps_C = 0.2e-9, 2048, 0.05
    tr = near_cherenkov_tracks([0.03, -0.03, 0.02, -0.02, 0.01], 1.0, 4, rng)
    t_ref = [1e-7 + 100.0 * 1.78 / 299792458.0 - 50e-9]
    _, u = oracle.arrivals(tr, ant, t_ref, N, dt, ICE, oracle.ENDPOINT, eps_C)
    um, du = u[:, 0].mean(axis=1), np.abs(u[:, 0, 1] - u[:, 0, 0])
    move = (np.floor(um) + 0.5 + rng.uniform(-0.3, 0.3, len(um)) * du - um) * dt
    move[::2] = 0.0
    tr["t0"] = tr["t0"] + move
    tr["t1"] = tr["t1"] + move
    br0, u0, checked, skipped = _fd_check(tr, ant, t_ref, N, dt, ICE, oracle.ENDPOINT, eps_C, 6)
    assert (br0 == 1).all()
    same = np.floor(u0[..., 0] + 0.5) == np.floor(u0[..., 1] + 0.5)
    assert same.sum() >= 4 and (~same).sum() >= 4
    assert checked > 5 * skipped
