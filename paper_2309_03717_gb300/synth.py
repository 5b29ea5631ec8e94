"""Seeded synthetic shower workloads (inputs only; none of the radio arithmetic).

The paper measures on CORSIKA 8 electron showers and on detector arrays of 160
to 10 000 antennas (§5).  Neither the shower simulation nor its tracks are
available here, so these generators stand in for them with tracks that have the
shape of a shower's charged-particle tracks:

* start height h ~ Normal(4 km, 1.5 km), truncated to [0.5, 10] km by rejection;
* lateral offset from the axis r ~ Exp(30 m) with uniform azimuth;
* direction: straight down, tilted by independent Normal(0, 5 deg) angles about
  the x and y axes (one reading of "Gaussian 5 deg spread");
* track length L ~ U[0.5, 5] m, Lorentz factor log-uniform on [10, 1e4];
* charge -1 with probability 0.55, else +1;
* emission time t0 = (10 km - h)/c, t1 = t0 + L / (|beta| c), x1 = x0 + L u.

An inclined shower is the vertical sample rotated about the core by the zenith
angle (azimuth 0); altitude is then the rotated z and the 10 km epoch is
measured along the axis.

Storage is FP32-exact: every position (m), time (ns, offset from t = 0) and
velocity component is rounded to float32 and beta is scaled down until its
float32 norm is below 1, so both the CUDA path and the FP64 oracle consume the
same exact values.  ``dtype=np.float64`` keeps the unrounded FP64 values.

Every antenna's trace starts 50 ns before the plane shower front reaches it;
the front moves at c along the axis from the 10 km axis point.
"""
from __future__ import annotations

import math

import numpy as np

C_LIGHT = 299792458.0          # m/s
C_M_PER_NS = C_LIGHT * 1e-9    # m/ns
FIELDS = ("x0", "y0", "z0", "x1", "y1", "z1", "t0", "t1", "bx", "by", "bz", "q")

AIR_UNIFORM = {"kind": "uniform", "n": 1.000292}
AIR_EXPONENTIAL = {"kind": "exponential", "N0": 3.25e-4, "H": 8000.0}
# the same atmosphere over a spherical Earth (mean radius 6371 km)
AIR_SPHERICAL = {"kind": "exponential_spherical", "N0": 3.25e-4, "H": 8000.0, "R_E": 6.371e6}


def _rot_y(theta):
    c, s = math.cos(theta), math.sin(theta)
    return np.array([[c, 0.0, s], [0.0, 1.0, 0.0], [-s, 0.0, c]])


def shower_axis_up(zenith_deg: float) -> np.ndarray:
    """Unit vector pointing up the shower axis (towards where the shower comes from)."""
    return _rot_y(math.radians(zenith_deg)) @ np.array([0.0, 0.0, 1.0])


def make_tracks(n: int, seed: int, zenith_deg: float = 0.0, dtype=np.float32) -> dict:
    """n seeded shower-like tracks as a dict of SoA arrays (times in ns)."""
    rng = np.random.default_rng(seed)
    n = int(n)
    h = np.empty(0)
    while h.size < n:
        cand = rng.normal(4000.0, 1500.0, size=max(2 * (n - h.size), 16))
        h = np.concatenate([h, cand[(cand >= 500.0) & (cand <= 10000.0)]])
    h = h[:n]
    r = rng.exponential(30.0, size=n)
    phi = rng.uniform(0.0, 2.0 * math.pi, size=n)
    ax = rng.normal(0.0, math.radians(5.0), size=n)
    ay = rng.normal(0.0, math.radians(5.0), size=n)
    L = rng.uniform(0.5, 5.0, size=n)
    gamma = np.exp(rng.uniform(math.log(10.0), math.log(1e4), size=n))
    q = np.where(rng.uniform(size=n) < 0.55, -1.0, 1.0)

    # direction: -z tilted about x by ax, then about y by ay
    ux = -np.cos(ax) * np.sin(ay)
    uy = np.sin(ax)
    uz = -np.cos(ax) * np.cos(ay)
    norm = np.sqrt(ux * ux + uy * uy + uz * uz)
    u = np.stack([ux / norm, uy / norm, uz / norm], axis=1)
    x0 = np.stack([r * np.cos(phi), r * np.sin(phi), h], axis=1)
    if zenith_deg:
        Rz = _rot_y(math.radians(zenith_deg))
        x0 = x0 @ Rz.T
        u = u @ Rz.T
    bmag = np.sqrt(1.0 - 1.0 / (gamma * gamma))
    beta = u * bmag[:, None]
    x1 = x0 + u * L[:, None]

    if dtype == np.float32:
        beta = beta.astype(np.float32)
        for _ in range(64):
            b = np.sqrt((beta.astype(np.float64) ** 2).sum(axis=1))
            bad = b >= 1.0
            if not bad.any():
                break
            beta[bad] = (beta[bad].astype(np.float64) * (1.0 - 2e-7)).astype(np.float32)
        else:  # pragma: no cover - the loop converges in a few passes
            raise RuntimeError("could not bring |beta| below 1 in float32")
        x0 = x0.astype(np.float32)
        x1 = x1.astype(np.float32)
    bnorm = np.sqrt((beta.astype(np.float64) ** 2).sum(axis=1))
    t0 = (10000.0 - h) / C_M_PER_NS
    t1 = t0 + L / (bnorm * C_M_PER_NS)
    out = {
        "x0": x0[:, 0], "y0": x0[:, 1], "z0": x0[:, 2],
        "x1": x1[:, 0], "y1": x1[:, 1], "z1": x1[:, 2],
        "t0": t0, "t1": t1,
        "bx": beta[:, 0], "by": beta[:, 1], "bz": beta[:, 2],
        "q": q,
    }
    return {k: np.ascontiguousarray(v, dtype=dtype) for k, v in out.items()}


def antennas_line(count: int = 16, spacing: float = 25.0) -> np.ndarray:
    """East line at spacing, 2*spacing, ... on the ground."""
    x = spacing * np.arange(1, count + 1, dtype=np.float64)
    return np.stack([x, np.zeros_like(x), np.zeros_like(x)], axis=1)


def antennas_star(arms: int = 8, radii=None, n_radii: int = 20, r_min: float = 10.0, r_max: float = 400.0,
                  limit: int | None = None) -> np.ndarray:
    """Star pattern: arms at 360/arms degree steps, radii linspace(r_min, r_max)."""
    if radii is None:
        radii = np.linspace(r_min, r_max, n_radii)
    pos = []
    for k in range(arms):
        a = 2.0 * math.pi * k / arms
        for rr in radii:
            pos.append((rr * math.cos(a), rr * math.sin(a), 0.0))
    pos = np.array(pos, dtype=np.float64)
    return pos if limit is None else pos[:limit]


def antennas_grid(side: int, spacing: float = 50.0, limit: int | None = None) -> np.ndarray:
    """side x side ground grid centred on the core."""
    c = (np.arange(side) - (side - 1) / 2.0) * spacing
    X, Y = np.meshgrid(c, c, indexing="ij")
    pos = np.stack([X.ravel(), Y.ravel(), np.zeros(side * side)], axis=1)
    return pos if limit is None else pos[:limit]


def trace_start_ns(ant_xyz: np.ndarray, zenith_deg: float = 0.0, lead_ns: float = 50.0) -> np.ndarray:
    """Start time (ns) of every antenna's trace: plane-front arrival minus lead_ns."""
    s = np.asarray(ant_xyz, dtype=np.float64) @ shower_axis_up(zenith_deg)
    return (10000.0 - s) / C_M_PER_NS - lead_ns


def workload(cfg: int, n_tracks: int | None = None, n_ant: int | None = None, seed_offset: int = 0) -> dict:
    """One of the five benchmark workloads, optionally cut down.

    0: Endpoint FP64, 1e5 tracks, 16 antennas (east line), uniform n, 4096 x 0.2 ns.
    1: Endpoint + ZHS, 2e7 tracks, 160 antennas (star 8 x 20), exponential n, 4096 x 0.2 ns.
    2: inclined (60 deg), 1e8 tracks in 4e6 chunks, 32 x 32 grid at 50 m, 8192 x 0.1 ns.
    4: differentiable Endpoint, 1e6 tracks, star 8 x 8, exponential n, 2048 x 0.2 ns.
    (3, the batched set of 64 showers, is ``batched_workload``.)
    """
    seed = 1000 + cfg + seed_offset
    if cfg == 0:
        ant = antennas_line(16, 25.0)
        w = dict(n_tracks=100_000, zenith=0.0, medium=dict(AIR_UNIFORM), n_bins=4096, dt_ns=0.2,
                 dtype=np.float64, formalisms=("endpoint",), precision="fp64")
    elif cfg == 1:
        ant = antennas_star(8, n_radii=20)
        w = dict(n_tracks=20_000_000, zenith=0.0, medium=dict(AIR_EXPONENTIAL), n_bins=4096, dt_ns=0.2,
                 dtype=np.float32, formalisms=("endpoint", "zhs"), precision="mixed")
    elif cfg == 2:
        ant = antennas_grid(32, 50.0)
        w = dict(n_tracks=100_000_000, zenith=60.0, medium=dict(AIR_EXPONENTIAL), n_bins=8192, dt_ns=0.1,
                 dtype=np.float32, formalisms=("endpoint",), precision="mixed", chunk=4_000_000)
    elif cfg == 4:
        ant = antennas_star(8, n_radii=8)
        w = dict(n_tracks=1_000_000, zenith=0.0, medium=dict(AIR_EXPONENTIAL), n_bins=2048, dt_ns=0.2,
                 dtype=np.float32, formalisms=("endpoint",), precision="mixed")
    else:
        raise ValueError(f"no single-shower workload {cfg}")
    if n_ant is not None:
        ant = ant[:n_ant]
    if n_tracks is not None:
        w["n_tracks"] = int(n_tracks)
    w["ant_xyz"] = ant
    w["t_start_ns"] = trace_start_ns(ant, w["zenith"])
    w["seed"] = seed
    w["cfg"] = cfg
    return w


def workload_tracks(w: dict, n: int | None = None, chunk_index: int = 0) -> dict:
    """Tracks of workload w (chunk_index > 0 draws an independent chunk of a streamed set)."""
    n = w["n_tracks"] if n is None else int(n)
    seed = w["seed"] if chunk_index == 0 else w["seed"] * 1_000_003 + chunk_index
    return make_tracks(n, seed, w["zenith"], w["dtype"])


def perturbed_target_tracks(tracks: dict, seed: int, rel: float = 0.01) -> dict:
    """Each endpoint coordinate moved by Normal(0, (rel * L)^2); times and beta kept."""
    rng = np.random.default_rng(seed)
    dt = tracks["x0"].dtype
    x0 = np.stack([tracks["x0"], tracks["y0"], tracks["z0"]], 1).astype(np.float64)
    x1 = np.stack([tracks["x1"], tracks["y1"], tracks["z1"]], 1).astype(np.float64)
    L = np.linalg.norm(x1 - x0, axis=1)
    x0 = x0 + rng.normal(size=x0.shape) * (rel * L)[:, None]
    x1 = x1 + rng.normal(size=x1.shape) * (rel * L)[:, None]
    out = dict(tracks)
    for k, c in enumerate("xyz"):
        out[c + "0"] = x0[:, k].astype(dt)
        out[c + "1"] = x1[:, k].astype(dt)
    return out


def batched_workload(n_showers: int = 64, seed: int = 1003, track_scale: float = 1.0,
                     max_tracks: int | None = None) -> list[dict]:
    """64 uneven showers: zenith U[0, 65] deg, tracks log-uniform [1e5, 1e7],
    antennas U{16..512}; star layout (8 arms) for even showers, 50 m grid for odd."""
    rng = np.random.default_rng(seed)
    out = []
    for s in range(n_showers):
        zen = rng.uniform(0.0, 65.0)
        T = int(round(math.exp(rng.uniform(math.log(1e5), math.log(1e7))) * track_scale))
        if max_tracks is not None:
            T = min(T, max_tracks)
        A = int(rng.integers(16, 513))
        if s % 2 == 0:
            ant = antennas_star(8, n_radii=int(math.ceil(A / 8)), limit=A)
        else:
            side = int(math.ceil(math.sqrt(A)))
            ant = antennas_grid(side, 50.0, limit=A)
        out.append(dict(shower=s, zenith=zen, n_tracks=max(T, 1), ant_xyz=ant,
                        t_start_ns=trace_start_ns(ant, zen), seed=seed * 1000 + s,
                        medium=dict(AIR_EXPONENTIAL), n_bins=4096, dt_ns=0.2, dtype=np.float32))
    return out


# ---------------------------------------------------------------------------
# Counter-based shower generator: the same distributions as make_tracks, with
# every track drawn from its own Philox4x32-10 blocks (Salmon, Moraes, Dror &
# Shaw, SC'11), so any range of tracks of a shower can be generated on its own
# and on the device (c8r_generate_tracks) with the same values.  All transforms
# are FP64 with one rounding per operation, in the order written here.
# ---------------------------------------------------------------------------
_PHILOX_M0, _PHILOX_M1 = 0xD2511F53, 0xCD9E8D57
_PHILOX_W0, _PHILOX_W1 = 0x9E3779B9, 0xBB67AE85
PHILOX_TAG = 0x63387237  # fourth counter word of every block
H_ATTEMPTS = 16          # rejection attempts for the start height


def philox4x32_10(c0, c1, c2, c3, k0, k1):
    """Vectorised Philox4x32-10 (uint64 arrays holding 32-bit words)."""
    c0, c1, c2, c3 = (np.asarray(v, dtype=np.uint64) for v in (c0, c1, c2, c3))
    k0 = np.asarray(k0, dtype=np.uint64) + np.zeros_like(c0)
    k1 = np.asarray(k1, dtype=np.uint64) + np.zeros_like(c0)
    mask = np.uint64(0xFFFFFFFF)
    for _ in range(10):
        p0 = np.uint64(_PHILOX_M0) * c0
        p1 = np.uint64(_PHILOX_M1) * c2
        c0, c1, c2, c3 = (p1 >> np.uint64(32)) ^ c1 ^ k0, p1 & mask, (p0 >> np.uint64(32)) ^ c3 ^ k1, p0 & mask
        k0 = (k0 + np.uint64(_PHILOX_W0)) & mask
        k1 = (k1 + np.uint64(_PHILOX_W1)) & mask
    return c0, c1, c2, c3


def _u01(w):
    return (w.astype(np.float64) + 0.5) * (1.0 / 4294967296.0)


def make_tracks_counter(first: int, n: int, seed: int, zenith_deg: float = 0.0) -> dict:
    """Tracks first .. first+n-1 of the counter-based synthetic shower `seed`
    (FP32 SoA).  Block b of track g is philox(counter = (g lo, g hi, b, tag),
    key = (seed lo, seed hi)); U(w) = (w + 1/2) / 2^32.
      block 0: r = -30 ln U, phi = 2 pi U, L = 0.5 + 4.5 U, gamma = exp(ln 10 + ln(1e3) U);
      block 1: q = -1 if U < 0.55 else +1; two Box-Muller normals of 5 deg: ax, ay;
      blocks 2 .. 17: start height h = 4000 + 1500 N(0,1), the first in [500, 10000]
      (4000 if none); then the geometry of make_tracks."""
    g = np.arange(first, first + n, dtype=np.uint64)
    lo, hi = g & np.uint64(0xFFFFFFFF), g >> np.uint64(32)
    k0, k1 = np.uint64(seed & 0xFFFFFFFF), np.uint64((seed >> 32) & 0xFFFFFFFF)

    def block(b, sel=slice(None)):
        m = lo[sel].size
        return philox4x32_10(lo[sel], hi[sel], np.full(m, b, dtype=np.uint64), np.full(m, PHILOX_TAG, dtype=np.uint64),
                             k0, k1)

    w = block(0)
    r = -30.0 * np.log(_u01(w[0]))
    phi = (2.0 * math.pi) * _u01(w[1])
    L = 0.5 + 4.5 * _u01(w[2])
    gamma = np.exp(math.log(10.0) + (math.log(1e4) - math.log(10.0)) * _u01(w[3]))
    w = block(1)
    q = np.where(_u01(w[0]) < 0.55, -1.0, 1.0)
    rad = np.sqrt(-2.0 * np.log(_u01(w[1])))
    ang = (2.0 * math.pi) * _u01(w[2])
    sig = 5.0 * math.pi / 180.0
    ax = sig * (rad * np.cos(ang))
    ay = sig * (rad * np.sin(ang))
    h = np.full(n, 4000.0)
    todo = np.arange(n)  # tracks still without a height (attempts only for them)
    for j in range(H_ATTEMPTS):
        if todo.size == 0:
            break
        w = block(2 + j, todo)
        z = np.sqrt(-2.0 * np.log(_u01(w[0]))) * np.cos((2.0 * math.pi) * _u01(w[1]))
        hj = 4000.0 + 1500.0 * z
        take = (hj >= 500.0) & (hj <= 10000.0)
        h[todo[take]] = hj[take]
        todo = todo[~take]
    ux = -(np.cos(ax) * np.sin(ay))
    uy = np.sin(ax)
    uz = -(np.cos(ax) * np.cos(ay))
    un = np.sqrt((ux * ux + uy * uy) + uz * uz)
    ux, uy, uz = ux / un, uy / un, uz / un
    x, y, zz = r * np.cos(phi), r * np.sin(phi), h
    if zenith_deg:
        c, s = math.cos(math.radians(zenith_deg)), math.sin(math.radians(zenith_deg))
        x, zz = c * x + s * zz, c * zz - s * x
        ux, uz = c * ux + s * uz, c * uz - s * ux
    bmag = np.sqrt(1.0 - 1.0 / (gamma * gamma))
    b = [(ux * bmag).astype(np.float32), (uy * bmag).astype(np.float32), (uz * bmag).astype(np.float32)]
    for _ in range(64):
        b2 = (b[0].astype(np.float64) * b[0] + b[1].astype(np.float64) * b[1]) + b[2].astype(np.float64) * b[2]
        bad = b2 >= 1.0
        if not bad.any():
            break
        for k in range(3):
            b[k] = np.where(bad, (b[k].astype(np.float64) * (1.0 - 2e-7)).astype(np.float32), b[k])
    b2 = (b[0].astype(np.float64) * b[0] + b[1].astype(np.float64) * b[1]) + b[2].astype(np.float64) * b[2]
    t0 = (10000.0 - h) / C_M_PER_NS
    t1 = t0 + L / (np.sqrt(b2) * C_M_PER_NS)
    f32 = np.float32
    return {"x0": x.astype(f32), "y0": y.astype(f32), "z0": zz.astype(f32),
            "x1": (x + ux * L).astype(f32), "y1": (y + uy * L).astype(f32), "z1": (zz + uz * L).astype(f32),
            "t0": t0.astype(f32), "t1": t1.astype(f32), "bx": b[0], "by": b[1], "bz": b[2], "q": q.astype(f32)}
