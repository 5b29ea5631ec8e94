"""Host check (numpy FP32) of the error bound of the mixed Endpoint kernels'
FP32 arrival: the arrival from shifted times T = t/dt + k z in its split and
direct forms of x = R - (z_e - z_a), and the bound the kernels hold a bin edge
against before they take a bin from it (any endpoint whose bound reaches an
edge goes to the float-float arrival instead).  Every step is emulated as the
kernels state it, rounded once per operation, with the reciprocal square root
and the fast quotients perturbed within their 2-ulp error (both extremes and
random draws), and compared with the oracle's FP64 arrivals.  Like
test_numerics, this checks the arithmetic and its bound, not the CUDA code;
the GPU parity tests compare the kernels' bins with the oracle's."""
import numpy as np
import pytest

import oracle
from paper_2309_03717_gb300 import synth

F32 = np.float32
F64 = np.float64
U = 2.0 ** -24
ULP2 = 2.0 ** -22  # 2 ulp, relative
C_M_PER_NS = 0.299792458


def r(x):
    return np.asarray(x, F64).astype(F32)


def fma(a, b, c):
    return r(np.asarray(a, F64) * np.asarray(b, F64) + np.asarray(c, F64))


def split(x):
    h = r(x)
    return h, r(np.asarray(x, F64) - h.astype(F64))


def perturb(x, mode, rng):
    """An approximate result within 2 ulp of x: +2 ulp, -2 ulp or random."""
    x = np.asarray(x, F64)
    if mode == "up":
        f = np.full_like(x, ULP2)
    elif mode == "down":
        f = np.full_like(x, -ULP2)
    else:
        f = rng.uniform(-ULP2, ULP2, size=x.shape)
    return r(x * (1.0 + f))


def emulated_arrivals(w, tracks, split_form, mode, rng):
    """(uf, eps) per endpoint, [2][n_tracks, n_ant]: the FP32 arrival and its
    bound as the kernels form them, from the antenna constants as the host
    forms them."""
    dt = w["dt_ns"]
    med = w["medium"]
    expo = med["kind"] == "exponential"
    kc = 1.0 / (C_M_PER_NS * dt)
    if expo:
        N0, H = med["N0"], med["H"]
        kh, kl = split(kc)
        cNh, _ = split(N0 * H * kc)
        invHh, _ = split(1.0 / H)
        nmax = 1.0 + N0
    else:
        kh, kl = split(med["n"] * kc)
        nmax = med["n"]
    kff = F64(kh) + F64(kl)
    A = np.asarray(w["ant_xyz"], F64)
    Axh, Axl = split(A[:, 0])
    Ayh, Ayl = split(A[:, 1])
    Azh, Azl = split(A[:, 2])
    Ta = np.asarray(w["t_start_ns"], F64) / dt + kff * A[:, 2]
    Tah, Tal = split(Ta)
    al = np.sqrt(Axl.astype(F64) ** 2 + Ayl.astype(F64) ** 2 + Azl.astype(F64) ** 2)
    fb_abs = r(2.02 * nmax * kc * al + 16.0 * U * U * np.abs(Ta) + 1e-6)
    fb_rel_v = r(1.01 * np.abs(Azl.astype(F64)) / (0.999e-3 * H)) if expo else np.zeros(len(A), F32)
    if expo:
        Eah, Eal = split(np.exp(-A[:, 2] / H))
    out = []
    for xs, ys, zs, ts in (("x0", "y0", "z0", "t0"), ("x1", "y1", "z1", "t1")):
        px = tracks[xs].astype(F32)[:, None]
        py = tracks[ys].astype(F32)[:, None]
        pz = tracks[zs].astype(F32)[:, None]
        Teh, Tel = split(tracks[ts].astype(F64) / dt + kff * tracks[zs].astype(F64))
        Teh, Tel = Teh[:, None], Tel[:, None]
        s0, s1, s2 = r(Axh[None] - px), r(Ayh[None] - py), r(Azh[None] - pz)
        rho2 = fma(s0, s0, r(s1.astype(F64) * s1))
        S = fma(s2, s2, rho2)
        with np.errstate(divide="ignore", invalid="ignore"):
            y = perturb(1.0 / np.sqrt(S.astype(F64)), mode, rng)
            R0 = r(S.astype(F64) * y)
            if split_form:
                R = R0
                xa = perturb(rho2.astype(F64) / r(R.astype(F64) - s2).astype(F64), mode, rng)
                x = np.where(s2 < 0, xa, r(R.astype(F64) + s2))
            else:
                res = fma(-R0, R0, S)
                R = fma(res, r(0.5 * y.astype(F64)), R0)
                x = r(R.astype(F64) + s2)
            q = r(x.astype(F64) * kh)
            Td = r(r(Teh.astype(F64) - Tah[None]).astype(F64) + r(Tel.astype(F64) - Tal[None]))
            if expo:
                Eeh, Eel = split(np.exp(-tracks[zs].astype(F64) / H))
                Eeh, Eel = Eeh[:, None], Eel[:, None]
                xq = r(s2.astype(F64) * invHh)
                num = r(r(Eeh.astype(F64) - Eah[None]).astype(F64) + r(Eel.astype(F64) - Eal[None]))
                qv_big = perturb(num.astype(F64) / s2, mode, rng)
                f = r(xq.astype(F64) * fma(xq, fma(xq, r(-1.0 / 24.0), r(1.0 / 6.0)), r(-0.5)))
                qv_small = r(r(Eeh.astype(F64) * invHh).astype(F64) * r(1.0 + f.astype(F64)))
                qv = np.where(np.abs(xq) > F32(1e-3), qv_big, qv_small)
                v = r(r(qv.astype(F64) * R).astype(F64) * cNh)
            else:
                v = np.zeros_like(q)
            uf = r(r(Td.astype(F64) + q).astype(F64) + v)
            tail = fma(r(2.25 * U), np.abs(Td),
                       fma(fma(r(22.0 if split_form else 17.0), r(U), fb_rel_v[None]), np.abs(v),
                           fma(r(3.25 * U), np.abs(uf), fb_abs[None])))
            if split_form:
                eps = fma(r(19.0 * U), q, tail)
            else:
                eps = fma(r(6.25 * U), q, fma(r(2.5 * U * F64(kh)), R, tail))
        out.append((uf, eps))
    return out


def workload(name):
    if name == "vertical":
        w = synth.workload(1, n_tracks=1500)
    elif name == "inclined":
        w = synth.workload(2, n_tracks=1500, n_ant=64)
    elif name == "uniform":
        w = synth.workload(0, n_tracks=1500)
    else:  # a dense uniform medium (n = 1.78), the windows placed around the arrivals
        w = synth.workload(0, n_tracks=1500)
        w["medium"] = {"kind": "uniform", "n": 1.78}
    w["dtype"] = np.float32
    tracks = synth.workload_tracks(w)
    if name == "dense":
        _, u0 = oracle.arrivals(oracle.tracks_from_ns(tracks), w["ant_xyz"], np.zeros(len(w["ant_xyz"])), 1,
                                w["dt_ns"] * 1e-9, w["medium"], oracle.ENDPOINT)
        w["t_start_ns"] = np.median(u0[..., 0], axis=0) * w["dt_ns"] - 300.0
    return w, tracks


@pytest.mark.parametrize("name", ["vertical", "inclined", "uniform", "dense"])
@pytest.mark.parametrize("split_form", [True, False], ids=["split", "direct"])
def test_fp32_arrival_within_its_bound(name, split_form):
    w, tracks = workload(name)
    br, u = oracle.arrivals(oracle.tracks_from_ns(tracks), w["ant_xyz"], w["t_start_ns"] * 1e-9, w["n_bins"],
                            w["dt_ns"] * 1e-9, w["medium"], oracle.ENDPOINT)
    two = br == 0  # the pairs evaluated at their two endpoints (near-Cherenkov ones take the midpoint)
    assert two.mean() > 0.5
    rng = np.random.default_rng(7)
    worst = 0.0
    for mode in ("up", "down", "random", "random"):
        for j, (uf, eps) in enumerate(emulated_arrivals(w, tracks, split_form, mode, rng)):
            err = np.abs(uf.astype(F64) - u[..., j])[two]
            ratio = err / eps.astype(F64)[two]
            assert np.all(np.isfinite(ratio))
            worst = max(worst, float(ratio.max()))
    assert worst <= 1.0, f"the FP32 arrival left its bound: error / bound = {worst:.3f}"


def test_split_form_bound_is_small_on_a_vertical_shower():
    """Where the split form pays (emission points high above the array), its
    bound leaves almost every in-window endpoint decided: the float-float
    arrival is needed only within the bound of an edge."""
    w, tracks = workload("vertical")
    br, u = oracle.arrivals(oracle.tracks_from_ns(tracks), w["ant_xyz"], w["t_start_ns"] * 1e-9, w["n_bins"],
                            w["dt_ns"] * 1e-9, w["medium"], oracle.ENDPOINT)
    rng = np.random.default_rng(3)
    uf, eps = emulated_arrivals(w, tracks, True, "random", rng)[0]
    inwin = (br == 0) & (u[..., 0] > 0) & (u[..., 0] < w["n_bins"])
    assert inwin.mean() > 0.3
    undecided = np.floor(uf - eps) != np.floor(uf + eps)
    assert float(np.median(eps[inwin])) < 1e-2
    assert undecided[inwin].mean() < 0.01


# ---------------------------------------------------------------------------
# The near-Cherenkov zero decision.  A pair whose two linearised arrivals
# u_m -/+ D_m (t1 - t0)/(2 dt) fall in one bin (or both before, or both after,
# the window) contributes exactly 0 (reading C).  The kernels settle most such
# pairs from FP32 midpoint geometry with a bound, and leave the rest to the
# float-float evaluation; a pair settled as zero must be zero for the oracle.
# ---------------------------------------------------------------------------
def emulated_field_D(sx, sy, sz, R, invR, bx, by, bz, bmag, om, n, mode, rng):
    """D = 1 - n beta.rhat in FP32 as the kernels' field arithmetic forms it
    (the cancellation-free form when beta.d >= 0)."""
    wx = fma(sy, bz, -r(sz.astype(F64) * by))
    wy = fma(sz, bx, -r(sx.astype(F64) * bz))
    wz = fma(sx, by, -r(sy.astype(F64) * bx))
    bd = fma(bx, sx, fma(by, sy, r(bz.astype(F64) * sz)))
    w2 = fma(wx, wx, fma(wy, wy, r(wz.astype(F64) * wz)))
    den = r(R.astype(F64) * fma(bmag, R, bd))
    with np.errstate(divide="ignore", invalid="ignore"):
        Dp = r(om.astype(F64) + perturb(r(n.astype(F64) * w2).astype(F64) / den, mode, rng))
    Dn = r(1.0 - r(r(n.astype(F64) * bd).astype(F64) * invR))
    return np.where(bd >= 0, Dp, Dn)


def emulated_near_zero(w, tracks, split_form, mode, rng):
    """[n_tracks, n_ant] bool: the kernels' FP32 decision that a near-Cherenkov
    pair contributes zero, from the tile fields as the ingest forms them."""
    dt = w["dt_ns"]
    med = w["medium"]
    expo = med["kind"] == "exponential"
    N = w["n_bins"]
    kc = 1.0 / (C_M_PER_NS * dt)
    if expo:
        N0, H = med["N0"], med["H"]
        kh, kl = split(kc)
        cNh, _ = split(N0 * H * kc)
        invHh, _ = split(1.0 / H)
        nmax = 1.0 + N0
    else:
        kh, kl = split(med["n"] * kc)
        nmax = med["n"]
    kff = F64(kh) + F64(kl)
    A = np.asarray(w["ant_xyz"], F64)
    Axh, Axl = split(A[:, 0])
    Ayh, Ayl = split(A[:, 1])
    Azh, Azl = split(A[:, 2])
    Ta = np.asarray(w["t_start_ns"], F64) / dt + kff * A[:, 2]
    Tah, Tal = split(Ta)
    al = np.sqrt(Axl.astype(F64) ** 2 + Ayl.astype(F64) ** 2 + Azl.astype(F64) ** 2)
    fb_abs = r(2.02 * nmax * kc * al + 16.0 * U * U * np.abs(Ta) + 1e-6)[None]
    fb_rel_v = (r(1.01 * np.abs(Azl.astype(F64)) / (0.999e-3 * H)) if expo else np.zeros(len(A), F32))[None]
    # tile fields
    c = lambda k: tracks[k].astype(F32)[:, None]
    x0, y0, z0, x1, y1, z1 = (c(k) for k in ("x0", "y0", "z0", "x1", "y1", "z1"))
    bx, by, bz = c("bx"), c("by"), c("bz")
    Sb = bx.astype(F64) ** 2 + by.astype(F64) ** 2 + bz.astype(F64) ** 2
    bmag = r(np.sqrt(r(Sb).astype(F64)))
    omb = r(r(1.0 - Sb).astype(F64) / r(1.0 + bmag.astype(F64)))
    t0, t1 = tracks["t0"].astype(F64)[:, None], tracks["t1"].astype(F64)[:, None]
    dtau = r((t1 - t0) / dt)
    zm = 0.5 * (z0.astype(F64) + z1.astype(F64))
    # the midpoint geometry from the endpoints' FP32 differences
    a0x, a0y, a0z = r(Axh[None] - x0), r(Ayh[None] - y0), r(Azh[None] - z0)
    a1x, a1y, a1z = r(Axh[None] - x1), r(Ayh[None] - y1), r(Azh[None] - z1)
    sx = r(0.5 * r(a0x.astype(F64) + a1x))
    sy = r(0.5 * r(a0y.astype(F64) + a1y))
    sz = r(0.5 * r(a0z.astype(F64) + a1z))
    rho2 = fma(sx, sx, r(sy.astype(F64) * sy))
    S = fma(sz, sz, rho2)
    with np.errstate(divide="ignore", invalid="ignore"):
        y = perturb(1.0 / np.sqrt(S.astype(F64)), mode, rng)
        R0 = r(S.astype(F64) * y)
        L1 = r(r(np.abs(r(a0x.astype(F64) - a1x)).astype(F64) + np.abs(r(a0y.astype(F64) - a1y)))
               .astype(F64) + np.abs(r(a0z.astype(F64) - a1z)))
        if expo:
            Eh, El = split(np.exp(-zm / H))
            nm1 = r(F64(r(N0)) * Eh)
        else:
            Eh, El = np.ones_like(zm, F32), np.zeros_like(zm, F32)
            nm1 = np.full_like(zm, r(med["n"] - 1.0), F32)
        om = r(omb.astype(F64) - r(nm1.astype(F64) * bmag))
        n1 = r(1.0 + nm1.astype(F64))
        D = emulated_field_D(sx, sy, sz, R0, y, bx, by, bz, bmag, om, n1, mode, rng)
        Tmh, Tml = split(0.5 * (t0 + t1) / dt + kff * zm)
        # the FP32 arrival of the midpoint, its d carrying three more roundings
        if split_form:
            R = R0
            xa = perturb(rho2.astype(F64) / r(R.astype(F64) - sz).astype(F64), mode, rng)
            x = np.where(sz < 0, xa, r(R.astype(F64) + sz))
        else:
            res = fma(-R0, R0, S)
            R = fma(res, r(0.5 * y.astype(F64)), R0)
            x = r(R.astype(F64) + sz)
        q = r(x.astype(F64) * kh)
        Td = r(r(Tmh.astype(F64) - Tah[None]).astype(F64) + r(Tml.astype(F64) - Tal[None]))
        if expo:
            xq = r(sz.astype(F64) * invHh)
            Eah, Eal = split(np.exp(-A[:, 2] / H))
            num = r(r(Eh.astype(F64) - Eah[None]).astype(F64) + r(El.astype(F64) - Eal[None]))
            qv_big = perturb(num.astype(F64) / sz, mode, rng)
            f = r(xq.astype(F64) * fma(xq, fma(xq, r(-1.0 / 24.0), r(1.0 / 6.0)), r(-0.5)))
            qv_small = r(r(Eh.astype(F64) * invHh).astype(F64) * r(1.0 + f.astype(F64)))
            qv = np.where(np.abs(xq) > F32(1e-3), qv_big, qv_small)
            v = r(r(qv.astype(F64) * R).astype(F64) * cNh)
        else:
            v = np.zeros_like(q)
        uf = r(r(Td.astype(F64) + q).astype(F64) + v)
        tail = fma(r(2.25 * U), np.abs(Td),
                   fma(fma(r(22.0 if split_form else 17.0), r(U), fb_rel_v), np.abs(v),
                       fma(r(3.25 * U), np.abs(uf), fb_abs)))
        if split_form:
            eps_a = fma(fma(r(3.0), r(U), r(19.0 * U)), q, tail)
        else:
            eps_a = fma(fma(r(3.0), r(U), r(6.25 * U)), q, fma(r(2.5 * U * F64(kh)), R, tail))
        eps_u = fma(r(2.0 * U * F64(kh)), L1, eps_a)
        aD = np.abs(D)
        h = r(0.5 * r(aD.astype(F64) * dtau))
        dh = r(fma(r(16.0 * U), aD, r(8.0 * U * n1.astype(F64))).astype(F64) * dtau)
        e = r(r(eps_u.astype(F64) + dh).astype(F64) + r(2.0 * U * r(np.abs(uf).astype(F64) + h)))
        lo = r(r(uf.astype(F64) - h).astype(F64) - e)
        hi = r(r(uf.astype(F64) + h).astype(F64) + e)
        zero = (hi < 0) | (lo >= F32(N)) | (np.floor(lo) == np.floor(hi))
    return zero & (R0 > 0)


@pytest.mark.parametrize("name", ["vertical", "inclined", "uniform"])
@pytest.mark.parametrize("split_form", [True, False], ids=["split", "direct"])
def test_near_cherenkov_zero_decision_is_exact(name, split_form):
    w, tracks = workload(name)
    br, u = oracle.arrivals(oracle.tracks_from_ns(tracks), w["ant_xyz"], w["t_start_ns"] * 1e-9, w["n_bins"],
                            w["dt_ns"] * 1e-9, w["medium"], oracle.ENDPOINT)
    mid = br == 1  # the oracle's near-Cherenkov pairs (midpoint form)
    assert mid.sum() > 100
    N = w["n_bins"]
    clamp = lambda k: np.where(k < 0, -1, np.where(k >= N, N, k))
    oracle_zero = clamp(np.floor(u[..., 0])) == clamp(np.floor(u[..., 1]))
    rng = np.random.default_rng(11)
    for mode in ("up", "down", "random"):
        zero = emulated_near_zero(w, tracks, split_form, mode, rng)
        wrong = zero & mid & ~oracle_zero
        assert not wrong.any(), f"{wrong.sum()} near-Cherenkov pairs settled as zero are not zero"
        # most of the oracle's zero pairs are settled without the float-float
        # path (97-100 % on these workloads in the form the kernels pick for
        # them, 70-80 % on the 60-degree array)
        assert (zero & mid).sum() >= 0.6 * (oracle_zero & mid).sum()


# ---------------------------------------------------------------------------
# The float-float Doppler factor.  The ZHS interval ends u_m -/+ |D_m| (t1 -
# t0)/(2 dt) and the near-Cherenkov Endpoint arrivals need D = 1 - n beta.rhat
# to ~1e-9 absolute (half-widths reach ~1e2 bins); the kernels form it from the
# float-float midpoint geometry with error-free transformations, to ~1e-10
# (set by n - 1 rounded to FP32).
# ---------------------------------------------------------------------------
def two_sum(a, b):
    a, b = a.astype(F32), b.astype(F32)
    s = (a + b).astype(F32)
    bb = (s - a).astype(F32)
    return s, ((a - (s - bb).astype(F32)).astype(F32) + (b - bb).astype(F32)).astype(F32)


def two_prod(a, b):
    p = r(a.astype(F64) * b)
    return p, r(a.astype(F64) * b - p)  # the product's error is an FP32 number


def emulated_doppler_ff(w, tracks, mode, rng):
    """D at the track midpoints as the ZHS kernel forms it, float-float, and
    the FP64 value of the same formula from the exact inputs."""
    med = w["medium"]
    N0, H = med["N0"], med["H"]
    A = np.asarray(w["ant_xyz"], F64)
    Axh, Axl = split(A[:, 0])
    Ayh, Ayl = split(A[:, 1])
    Azh, Azl = split(A[:, 2])
    c = lambda k: tracks[k].astype(F32)[:, None]
    x0, y0, z0, x1, y1, z1 = (c(k) for k in ("x0", "y0", "z0", "x1", "y1", "z1"))
    bx, by, bz = c("bx"), c("by"), c("bz")
    # midpoint (x0 + x1)/2, exact in float-float
    m = []
    for p0, p1 in ((x0, x1), (y0, y1), (z0, z1)):
        h, l = two_sum(p0, p1)
        m.append((r(0.5 * h.astype(F64)), r(0.5 * l.astype(F64))))
    # geo_lite: d = a - m as float-float
    s, e = [], []
    for (ah, al_), (mh, ml) in zip(((Axh, Axl), (Ayh, Ayl), (Azh, Azl)), m):
        sh, sl = two_sum(np.broadcast_to(ah[None], (len(mh), len(ah))), np.broadcast_to(-mh, (len(mh), len(ah))))
        s.append(sh)
        e.append(r(sl.astype(F64) + r(al_[None].astype(F64) - ml)))
    S = fma(s[2], s[2], fma(s[0], s[0], r(s[1].astype(F64) * s[1])))
    y = perturb(1.0 / np.sqrt(S.astype(F64)), mode, rng)
    R0 = r(S.astype(F64) * y)
    # geo_refine: R = R0 + R1
    (p0, q0), (p1, q1), (p2, q2) = (two_prod(s[k], s[k]) for k in range(3))
    S1, E1 = two_sum(p0, p1)
    S2, E2 = two_sum(S1, p2)
    cross = fma(s[0], e[0], fma(s[1], e[1], r(s[2].astype(F64) * e[2])))
    lo = r(r(r(q0.astype(F64) + q1).astype(F64) + r(q2.astype(F64) + E1)).astype(F64)
           + r(E2.astype(F64) + r(2.0 * cross.astype(F64))))
    rq, rqe = two_prod(R0, R0)
    rho = r(r(r(S2.astype(F64) - rq).astype(F64) - rqe).astype(F64) + lo)
    R1 = r(r(rho.astype(F64) * 0.5).astype(F64) * y)
    # doppler_ff
    (p0, q0), (p1, q1), (p2, q2) = two_prod(bx, s[0]), two_prod(by, s[1]), two_prod(bz, s[2])
    S1, E1 = two_sum(p0, p1)
    S2, E2 = two_sum(S1, p2)
    be = fma(bx, e[0], fma(by, e[1], r(bz.astype(F64) * e[2])))
    lo = r(r(r(q0.astype(F64) + q1).astype(F64) + r(q2.astype(F64) + E1)).astype(F64) + r(E2.astype(F64) + be))
    qh = r(S2.astype(F64) * y)
    ph, pl = two_prod(qh, R0)
    res = r(r(r(r(S2.astype(F64) - ph).astype(F64) - pl).astype(F64) + lo).astype(F64) - r(qh.astype(F64) * R1))
    ql = r(res.astype(F64) * y)
    zm = 0.5 * (z0.astype(F64) + z1.astype(F64))
    Emh, _ = split(np.exp(-zm / H))
    nm1 = r(F64(r(N0)) * Emh)
    nh, nl = two_sum(qh, r(nm1.astype(F64) * qh))
    nl = r(nl.astype(F64) + ql)
    dh, dl = two_sum(np.ones_like(nh), -nh)
    dl = r(dl.astype(F64) - nl)
    D = dh.astype(F64) + dl.astype(F64)
    # FP64: the same formula from the exact midpoint and antenna positions
    mx = 0.5 * (x0.astype(F64) + x1.astype(F64))
    my = 0.5 * (y0.astype(F64) + y1.astype(F64))
    dx, dy, dz = A[None, :, 0] - mx, A[None, :, 1] - my, A[None, :, 2] - zm
    R = np.sqrt(dx * dx + dy * dy + dz * dz)
    n = 1.0 + N0 * np.exp(-zm / H)
    D64 = 1.0 - n * (bx.astype(F64) * dx + by.astype(F64) * dy + bz.astype(F64) * dz) / R
    return D, D64


@pytest.mark.parametrize("name", ["vertical", "inclined"])
def test_float_float_doppler_factor(name):
    w, tracks = workload(name)
    rng = np.random.default_rng(5)
    for mode in ("up", "down", "random"):
        D, D64 = emulated_doppler_ff(w, tracks, mode, rng)
        err = np.abs(D - D64)
        # ~1.2e-10 at most on these workloads (n - 1 rounded to FP32, and the
        # FP32 low parts of the float-float steps); the interval ends need 1e-9
        assert float(err.max()) < 3e-10, float(err.max())
        # an FP32 D would be off by up to ~u |D|
        assert float(np.abs(D64).max()) > 0.05
