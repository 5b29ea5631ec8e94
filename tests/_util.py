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
    """Tracks whose Endpoint deposits are all away from bin edges and whose branch
    decision is away from the threshold (so the trace is a continuous function of
    the inputs within the mixed path's rounding)."""
    br, u = oracle_arrivals(tracks, ant, t_start_ns, n_bins, dt_ns, medium, "endpoint", eps_C)
    amb = edge_ambiguous(u, tol).any(axis=-1).any(axis=-1)
    return ~amb
