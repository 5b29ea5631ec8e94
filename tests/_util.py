"""Helpers shared by the tests: building the library, moving synthetic tracks to
the GPU, and comparing CUDA-path results with the oracle."""
import numpy as np

import oracle
from paper_2309_03717_gb300 import synth

FIELDS = oracle.FIELDS


def built_lib():
    from paper_2309_03717_gb300 import build
    return build.build()


def to_device(tracks, dtype=None):
    import torch
    out = {}
    for f in FIELDS:
        a = np.ascontiguousarray(tracks[f])
        t = torch.from_numpy(a)
        if dtype is not None:
            t = t.to(dtype)
        out[f] = t.cuda()
    return out


def medium_for_oracle(m):
    return dict(m)


def rel_l2(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    n = np.linalg.norm(b.ravel())
    d = np.linalg.norm((a - b).ravel())
    return d / n if n > 0 else d


def oracle_traces(tracks, ant, t_start_ns, n_bins, dt_ns, medium, formalism, eps_C=1e-3):
    tr = oracle.tracks_from_ns(tracks)
    out, kept = oracle.forward(tr, ant, np.asarray(t_start_ns) * 1e-9, n_bins, dt_ns * 1e-9, medium,
                               oracle.ENDPOINT if formalism == "endpoint" else oracle.ZHS, eps_C)
    return out, kept


def oracle_abs_traces(tracks, ant, t_start_ns, n_bins, dt_ns, medium, formalism, eps_C=1e-3):
    """Sum of |deposit| per bin and component: the magnitude of the summed terms."""
    tr = oracle.tracks_from_ns(tracks)
    out, _ = oracle.forward(tr, ant, np.asarray(t_start_ns) * 1e-9, n_bins, dt_ns * 1e-9, medium,
                            oracle.ENDPOINT if formalism == "endpoint" else oracle.ZHS, eps_C, oracle.MODE_ABS)
    return out


def cond_err(got, ref, absref):
    """Error relative to the magnitude of the summed deposits (condition-aware):
    a trace whose start and end deposits nearly cancel has a tiny norm, and
    relative to it any rounding looks large."""
    return np.linalg.norm((np.asarray(got, np.float64) - ref).ravel()) / np.linalg.norm(absref.ravel())


def oracle_arrivals(tracks, ant, t_start_ns, n_bins, dt_ns, medium, formalism, eps_C=1e-3):
    tr = oracle.tracks_from_ns(tracks)
    return oracle.arrivals(tr, ant, np.asarray(t_start_ns) * 1e-9, n_bins, dt_ns * 1e-9, medium,
                           oracle.ENDPOINT if formalism == "endpoint" else oracle.ZHS, eps_C)


def edge_ambiguous(u, tol):
    """Mask of arrival positions within tol of a bin edge."""
    fr = u - np.floor(u)
    return np.minimum(fr, 1.0 - fr) < tol


def compare_bins(gpu_branch, gpu_bin, gpu_frac, ora_branch, ora_u, n_bins, tol=1e-6):
    """Branch and bin of every (track, antenna) arrival must agree with the oracle
    except where the oracle's arrival lies within tol of a bin edge (there either
    neighbouring bin is correct).  Returns (n_compared, n_ambiguous)."""
    gb = np.asarray(gpu_branch)
    assert gb.shape == ora_branch.shape
    kept = ora_branch >= 0
    assert np.array_equal(gb >= 0, kept), "filter decisions differ"
    ob = np.floor(ora_u)
    ob = np.where(ob < 0, -1, np.where(ob >= n_bins, n_bins, ob)).astype(np.int64)
    amb = edge_ambiguous(ora_u, tol)
    both = kept[..., None] & np.ones_like(amb)
    gbin = np.asarray(gpu_bin).astype(np.int64)
    # the GPU's arrival position where both sides agree on the bin: bin + fraction
    gu = gbin + np.asarray(gpu_frac, dtype=np.float64)
    inside = both & (gbin == ob) & (ob >= 0) & (ob < n_bins)
    du = np.abs(gu - ora_u)[inside]
    worst = float(du.max()) if du.size else 0.0
    # branch: compare where no arrival of the pair is ambiguous and the pair
    # reaches the window (outside it the listing clamps bins to -1 / n_bins, so a
    # ZHS interval wholly before or after the window reads as one bin there)
    pair_amb = amb.any(axis=-1)
    outside = (ora_u < 0).all(axis=-1) | (ora_u >= n_bins).all(axis=-1)
    sel = kept & ~pair_amb & ~outside
    nb = int((gb[sel] != ora_branch[sel]).sum())
    assert nb == 0, f"branch decisions differ for {nb} pairs (largest arrival difference {worst:.2e} bin)"
    same_branch = kept & (gb == ora_branch)
    m = both & same_branch[..., None] & ~amb
    bad = m & (gbin != ob)
    assert not bad.any(), f"{int(bad.sum())} bins differ away from edges, e.g. {np.argwhere(bad)[:5]}"
    off = both & same_branch[..., None] & amb & (np.abs(gbin - ob) > 1)
    assert not off.any(), "an edge-ambiguous arrival landed more than one bin away"
    return int(m.sum()), int((both & amb).sum())


def drop_tracks(tracks, keep_mask):
    return {f: np.ascontiguousarray(tracks[f][keep_mask]) for f in FIELDS}


def unambiguous(tracks, ant, t_start_ns, n_bins, dt_ns, medium, formalism, tol=1e-6):
    """Tracks none of whose arrival positions (Endpoint deposits, ZHS interval
    ends) lies within tol bin of a bin edge."""
    _, u = oracle_arrivals(tracks, ant, t_start_ns, n_bins, dt_ns, medium, formalism)
    return ~edge_ambiguous(u, tol).any(axis=-1).any(axis=-1)


def endpoint_unambiguous(tracks, ant, t_start_ns, n_bins, dt_ns, medium, tol=1e-6, eps_C=1e-3):
    """Tracks none of whose Endpoint arrivals (the two endpoint arrivals, or the
    two linearised midpoint arrivals near the Cherenkov angle) lies within tol
    bin of a bin edge at any antenna: their traces do not depend on which of two
    bins an edge-ambiguous deposit takes."""
    _, u = oracle_arrivals(tracks, ant, t_start_ns, n_bins, dt_ns, medium, "endpoint", eps_C)
    amb = edge_ambiguous(u, tol).any(axis=-1).any(axis=-1)
    return ~amb


def either_bin_reference(gpu, ref, tracks, ant, t_start_ns, n_bins, dt_ns, medium, tol=1e-6, eps_C=1e-3):
    """The oracle's Endpoint traces `ref` with every deposit whose arrival lies
    within tol bin of an edge placed in whichever of its two neighbouring bins
    the GPU's traces agree with better (reading P: there either bin is correct).

    For each (track, antenna) pair with such an arrival the pair's contribution
    is evaluated by the oracle twice, with the antenna's window as given and with
    it moved by a fraction of a bin that carries the arrival across its edge
    (the deposit amplitudes do not depend on the window), and the pair keeps the
    version nearer the GPU at that antenna.  Only the oracle computes values."""
    _, u = oracle_arrivals(tracks, ant, t_start_ns, n_bins, dt_ns, medium, "endpoint", eps_C)
    amb = edge_ambiguous(u, tol)
    ref = np.array(ref, dtype=np.float64, copy=True)
    gpu = np.asarray(gpu, dtype=np.float64)
    ts = np.asarray(t_start_ns, dtype=np.float64)
    for i, a in np.argwhere(amb.any(axis=-1)):
        j = int(np.argmax(amb[i, a]))
        fr = u[i, a, j] - np.floor(u[i, a, j])
        # moving the window start by s bins moves every arrival of the pair by -s
        s = (fr + 2 * tol) if fr < 0.5 else -(1.0 - fr + 2 * tol)
        one = {f: tracks[f][i:i + 1] for f in FIELDS}
        c0, _ = oracle_traces(one, ant[a:a + 1], ts[a:a + 1], n_bins, dt_ns, medium, "endpoint", eps_C)
        c1, _ = oracle_traces(one, ant[a:a + 1], ts[a:a + 1] + s * dt_ns, n_bins, dt_ns, medium, "endpoint", eps_C)
        alt = ref[a] - c0[0] + c1[0]
        if np.linalg.norm(gpu[a] - alt) < np.linalg.norm(gpu[a] - ref[a]):
            ref[a] = alt
    return ref


AIR_UNIFORM = {"kind": "uniform", "n": 1.000292}
AIR_EXP = {"kind": "exponential", "N0": 3.25e-4, "H": 8000.0}


def near_cherenkov_pair(D, place, medium, h=1000.0, L=2.0, dt_ns=0.2, n_bins=64, K=32):
    """One track and one antenna built so that the antenna sees the track's
    midpoint at the Doppler factor D_m = D (the near-Cherenkov branch of the
    Endpoint formalism, |D| << eps_C at both endpoints).

    A vertical down-going track from (0, 0, h + L/2) to (0, 0, h - L/2) with
    beta = (0, 0, -b), b = 1 - 2^-20, and a ground antenna at (d, 0, 0) with
    h / R = cos(theta) = (1 - D) / (n_m b), n_m the index at the midpoint.  All
    inputs are FP32-exact (times in ns).  The antenna's window start is placed,
    from the oracle's own arrival of the midpoint, so that the midpoint arrival
    u_m lies at K + 1/2 (place 'same': both linearised arrivals
    u_m -/+ D (t1 - t0)/(2 dt) inside bin K, so the Endpoint pair gives exactly
    0 and the ZHS interval is one bin) or exactly on the edge K ('straddle': the
    arrivals in bins K - 1 and K).  Returns (tracks, ant [1, 3], t_start_ns [1])."""
    b = float(np.float32(1.0 - 2.0 ** -20))
    if medium["kind"] == "uniform":
        n = medium["n"]
    else:
        n = 1.0 + medium["N0"] * np.exp(-h / medium["H"])
    cos_t = (1.0 - D) / (n * b)
    d = float(np.float32(h * np.sqrt(1.0 - cos_t ** 2) / cos_t))
    c_ns = 0.299792458
    t0 = 100.0
    t1 = float(np.float32(t0 + L / (b * c_ns)))
    vals = [0.0, 0.0, h + L / 2, 0.0, 0.0, h - L / 2, t0, t1, 0.0, 0.0, -b, -1.0]
    tracks = {f: np.array([v], dtype=np.float64) for f, v in zip(FIELDS, vals)}
    for f in FIELDS:
        assert float(np.float32(tracks[f][0])) == tracks[f][0]
    ant = np.array([[d, 0.0, 0.0]])
    br, u = oracle_arrivals(tracks, ant, np.zeros(1), n_bins, dt_ns, medium, "endpoint")
    assert br[0, 0] == 1, "not in the near-Cherenkov branch"
    um = 0.5 * (u[0, 0, 0] + u[0, 0, 1])
    f = 0.5 if place == "same" else 0.0
    t_start = np.array([(um - (K + f)) * dt_ns])
    return tracks, ant, t_start


NEAR_CHERENKOV_CASES = [(m, D, place) for m in ("uniform", "exponential") for D in (1e-4, -1e-4, 1e-6, -1e-6)
                        for place in ("same", "straddle")]
