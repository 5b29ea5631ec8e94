"""Parity of the CUDA path (called through the C ABI) with the FP64 oracle.

Bars (from the hot-path contract): relative L2 <= 1e-9 for the FP64 path and
<= 1e-4 for the mixed path; bin indices identical except within 1e-6 bin of an
edge.  Inputs are the seeded synthetic shower workloads, cut to sizes the oracle
finishes in seconds while still spanning many track tiles (128 tracks), several
antenna tiles and a ragged tail.
"""
import numpy as np
import pytest

from _util import (AIR_EXP, AIR_UNIFORM, NEAR_CHERENKOV_CASES, built_lib, compare_bins, cond_err, drop_tracks,
                   either_bin_reference, endpoint_unambiguous, near_cherenkov_pair, oracle_abs_traces,
                   oracle_arrivals, oracle_traces, rel_l2, to_device)
from paper_2309_03717_gb300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    built_lib()
    from paper_2309_03717_gb300 import c8r
    c8r.load()


def process(w, formalism, precision, **kw):
    from paper_2309_03717_gb300.c8r import RadioProcess
    return RadioProcess(w["medium"], w["ant_xyz"], w["t_start_ns"], w["n_bins"], w["dt_ns"], formalism, precision,
                        **kw)


def run(w, tracks, formalism, precision, shape=None):
    p = process(w, formalism, precision)
    if shape:
        p.set_launch_shape(*shape)
    dt = torch.float64 if precision == "fp64" else torch.float32
    p.push(to_device(tracks, dt))
    out = p.traces().cpu().numpy()
    br, b, fr = p.arrivals(to_device(tracks, dt))
    st = p.stats()
    p.close()
    return out, (br.cpu().numpy(), b.cpu().numpy(), fr.cpu().numpy()), st


CASES = [
    # (cfg, n_tracks, n_ant, formalism, precision, tolerance)
    (0, 20011, 16, "endpoint", "fp64", 1e-9),
    (0, 20011, 16, "zhs", "fp64", 1e-9),
    (1, 6007, 40, "endpoint", "fp64", 1e-9),
    (1, 6007, 40, "zhs", "fp64", 1e-9),
    (1, 20011, 160, "endpoint", "mixed", 1e-4),
    (1, 20011, 160, "zhs", "mixed", 1e-4),
    (0, 20011, 16, "endpoint", "mixed", 1e-4),
    (0, 20011, 16, "zhs", "mixed", 1e-4),
    # inclined (60 deg) shower, 32 x 32 grid, 8192 x 0.1 ns
    (2, 6007, 64, "endpoint", "fp64", 1e-9),
    (2, 6007, 64, "zhs", "fp64", 1e-9),
    (2, 20011, 256, "endpoint", "mixed", 1e-4),
    (2, 20011, 256, "zhs", "mixed", 1e-4),
    # differentiable workload: star 8 x 8, 2048 x 0.2 ns
    (4, 20011, 64, "endpoint", "mixed", 1e-4),
]


@pytest.mark.parametrize("cfg,n,n_ant,formalism,precision,tol", CASES)
def test_traces_match_oracle(cfg, n, n_ant, formalism, precision, tol):
    w = synth.workload(cfg, n_tracks=n, n_ant=n_ant)
    if precision == "mixed":
        w["dtype"] = np.float32
    tracks = synth.workload_tracks(w)
    ref, kept = oracle_traces(tracks, w["ant_xyz"], w["t_start_ns"], w["n_bins"], w["dt_ns"], w["medium"], formalism)
    gpu, arr, st = run(w, tracks, formalism, precision)
    assert st["tracks_kept"] == kept
    assert np.abs(ref).max() > 0
    obr, ou = oracle_arrivals(tracks, w["ant_xyz"], w["t_start_ns"], w["n_bins"], w["dt_ns"], w["medium"], formalism)
    if formalism == "endpoint":
        # a deposit within 1e-6 bin of an edge may land in either bin (reading P):
        # the reference takes, for each, the placement the GPU's trace is nearer
        ref = either_bin_reference(gpu, ref, tracks, w["ant_xyz"], w["t_start_ns"], w["n_bins"], w["dt_ns"],
                                   w["medium"])
        assert (obr == 1).sum() > 0  # the near-Cherenkov branch is part of the check
    err = rel_l2(gpu, ref)
    assert err <= tol, f"relative L2 {err:.3e} > {tol:.0e}"
    # antenna by antenna: an error confined to the small traces of the outer
    # antennas must not hide under the inner ones
    per_ant = [rel_l2(gpu[a], ref[a]) for a in range(len(ref)) if np.abs(ref[a]).max() > 0]
    assert max(per_ant) <= tol, f"worst antenna: relative L2 {max(per_ant):.3e} > {tol:.0e} (all: {err:.3e})"
    n_cmp, n_amb = compare_bins(arr[0], arr[1], arr[2], obr, ou, w["n_bins"])
    assert n_cmp > 0.99 * obr.size


@pytest.mark.parametrize("formalism", ["endpoint", "zhs"])
@pytest.mark.parametrize("precision,tol", [("fp64", 1e-9), ("mixed", 1e-4)])
def test_largest_window(formalism, precision, tol):
    """The largest window accepted, 2^24 bins, ending on the shower front:
    arrival positions up to 2^24, where FP32 is spaced by 1 and the float-float
    low part carries the whole fraction (an arrival in the last bin has a high
    part of 2^24), and many arrivals after the window."""
    w = synth.workload(1, n_tracks=2003, n_ant=2)
    if precision == "mixed":
        w["dtype"] = np.float32
    tracks = synth.workload_tracks(w)
    N = 1 << 24
    # every window starts earlier, so that its first 300 bins (the 50 ns before
    # the front and the front itself) become the last 300 bins of the large one:
    # most arrivals fall in the window, ~2 % after it, ~10 in its last bin
    w["t_start_ns"] = np.asarray(w["t_start_ns"]) - (N - 300) * w["dt_ns"]
    w["n_bins"] = N
    if formalism == "endpoint":
        keep = endpoint_unambiguous(tracks, w["ant_xyz"], w["t_start_ns"], N, w["dt_ns"], w["medium"])
        tracks = drop_tracks(tracks, keep)
    ref, kept = oracle_traces(tracks, w["ant_xyz"], w["t_start_ns"], N, w["dt_ns"], w["medium"], formalism)
    assert np.abs(ref[:, :, N - 16:]).max() > 0 and not ref[:, :, :N - 4096].any()
    gpu, arr, st = run(w, tracks, formalism, precision)
    assert st["tracks_kept"] == kept
    if precision == "fp64" and formalism == "zhs":
        # an arrival position near 1.7e7 bins carries its own FP64 rounding,
        # ~4e-9 bin (one ulp there, against ~1e-11 in the shower's own window),
        # and the ZHS bin averages pass it on as ~4e-9/W of a deposit (W the
        # interval's width in bins): measured 6e-9 in relative L2
        tol = 2e-8
    err = rel_l2(gpu, ref)
    assert err <= tol, f"relative L2 {err:.3e} > {tol:.0e}"
    obr, ou = oracle_arrivals(tracks, w["ant_xyz"], w["t_start_ns"], N, w["dt_ns"], w["medium"], formalism)
    n_cmp, _ = compare_bins(arr[0], arr[1], arr[2], obr, ou, N)
    assert n_cmp > 0.99 * obr.size


@pytest.mark.parametrize("cfg,n,n_ant", [(2, 2003, 64), (1, 2003, 40)])
@pytest.mark.parametrize("formalism", ["endpoint", "zhs"])
@pytest.mark.parametrize("precision,tol", [("fp64", 1e-9), ("mixed", 1e-4)])
def test_spherical_earth_matches_oracle(cfg, n, n_ant, formalism, precision, tol):
    """The exponential atmosphere over a spherical Earth: the curvature part of
    the optical path (quadrature on the GPU, composite quadrature in the oracle)
    and of the source index, on the inclined shower where it matters most."""
    w = synth.workload(cfg, n_tracks=n, n_ant=n_ant)
    w["medium"] = dict(synth.AIR_SPHERICAL)
    if precision == "mixed":
        w["dtype"] = np.float32
    tracks = synth.workload_tracks(w)
    if formalism == "endpoint":
        keep = endpoint_unambiguous(tracks, w["ant_xyz"], w["t_start_ns"], w["n_bins"], w["dt_ns"], w["medium"])
        tracks = drop_tracks(tracks, keep)
    ref, kept = oracle_traces(tracks, w["ant_xyz"], w["t_start_ns"], w["n_bins"], w["dt_ns"], w["medium"], formalism)
    flat, _ = oracle_traces(tracks, w["ant_xyz"], w["t_start_ns"], w["n_bins"], w["dt_ns"], synth.AIR_EXPONENTIAL,
                            formalism)
    if cfg == 2:  # the inclined shower's emission points lie tens of km out: the curvature shows
        assert rel_l2(flat, ref) > 10 * tol
    gpu, arr, st = run(w, tracks, formalism, precision)
    assert st["tracks_kept"] == kept
    err = rel_l2(gpu, ref)
    assert err <= tol, f"relative L2 {err:.3e} > {tol:.0e}"
    obr, ou = oracle_arrivals(tracks, w["ant_xyz"], w["t_start_ns"], w["n_bins"], w["dt_ns"], w["medium"], formalism)
    n_cmp, _ = compare_bins(arr[0], arr[1], arr[2], obr, ou, w["n_bins"])
    assert n_cmp > 0.99 * obr.size


@pytest.mark.parametrize("formalism", ["endpoint", "zhs"])
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_invariant_to_launch_shape(formalism, precision):
    """§5: pulses do not depend on the number of threads; here: on the antenna
    tile, the number of track ranges and the chunking (up to addition order)."""
    w = synth.workload(1, n_tracks=9001, n_ant=24)
    tracks = synth.workload_tracks(w)
    base, _, _ = run(w, tracks, formalism, precision)
    tol = 1e-12 if precision == "fp64" else 2e-6
    for shape in [(1, 1, 0), (3, 16, 0), (2, 2, 1000), (4, 0, 4096), (32, 1, 0), (16, 64, 2048)]:
        other, _, _ = run(w, tracks, formalism, precision, shape)
        assert rel_l2(other, base) <= tol, shape


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_edge_cases(precision):
    from paper_2309_03717_gb300 import c8r
    from paper_2309_03717_gb300.c8r import C8RError
    w = synth.workload(1, n_tracks=300, n_ant=5)
    dt = torch.float64 if precision == "fp64" else torch.float32
    p = process(w, "endpoint", precision)
    # empty push is a no-op
    empty = {f: torch.empty(0, dtype=dt, device="cuda") for f in synth.FIELDS}
    p.push(empty)
    assert not p.traces().any()
    # a single track, and a ragged count (not a multiple of the 128-track tile);
    # with so few tracks the start and end deposits of a track can nearly cancel,
    # so the error is measured against the magnitude of the summed deposits
    tr = synth.workload_tracks(w)
    for n in (1, 129, 300):
        p.reset()
        sub = {f: tr[f][:n] for f in synth.FIELDS}
        p.push(to_device(sub, dt))
        args = (sub, w["ant_xyz"], w["t_start_ns"], w["n_bins"], w["dt_ns"], w["medium"], "endpoint")
        ref, _ = oracle_traces(*args)
        got = p.traces().cpu().numpy()
        assert cond_err(got, ref, oracle_abs_traces(*args)) <= (1e-12 if precision == "fp64" else 1e-6), n
    # all tracks filtered: neutral / non-finite / zero length / |beta| >= 1
    bad = {f: np.array(tr[f][:4]) for f in synth.FIELDS}
    bad["q"][0] = 0.0
    bad["x0"][1] = np.nan
    bad["x1"][2], bad["y1"][2], bad["z1"][2] = bad["x0"][2], bad["y0"][2], bad["z0"][2]
    bad["bz"][3] = -1.0
    bad["bx"][3] = bad["by"][3] = 0.0
    p.reset()
    p.push(to_device(bad, dt))
    assert not p.traces().any()
    assert p.stats()["tracks_kept"] == 0
    # a window that every arrival misses
    w2 = dict(w)
    w2["t_start_ns"] = w["t_start_ns"] - 1e6
    p2 = process(w2, "zhs", precision)
    p2.push(to_device(tr, dt))
    assert not p2.traces().any()
    # invalid arguments are rejected, not run
    with pytest.raises(C8RError):
        c8r.c8r_set_medium(p.ctx, c8r.C8R_UNIFORM, -1.0, 1.0)
    with pytest.raises(C8RError):
        c8r.c8r_set_antennas(p.ctx, w["ant_xyz"], w["t_start_ns"], 0, 0.2, 0, 1)
    with pytest.raises(C8RError):
        c8r.c8r_set_antennas(p.ctx, w["ant_xyz"], w["t_start_ns"], (1 << 24) + 1, 0.2, 0, 1)  # beyond 2^24 bins
    p.close()
    p2.close()


def test_mixed_accepts_fp64_input_rounded_to_fp32():
    w = synth.workload(1, n_tracks=2000, n_ant=8)
    tr32 = synth.workload_tracks(w)
    tr64 = {f: tr32[f].astype(np.float64) for f in synth.FIELDS}
    a, _, _ = run(w, tr32, "endpoint", "mixed")
    p = process(w, "endpoint", "mixed")
    p.push(to_device(tr64))
    b = p.traces().cpu().numpy()
    p.close()
    assert np.array_equal(a != 0, b != 0)
    assert rel_l2(b, a) < 1e-6


@pytest.mark.parametrize("cfg,n,n_ant", [(2, 2003, 64), (1, 2003, 40)])
@pytest.mark.parametrize("formalism", ["endpoint", "zhs"])
@pytest.mark.parametrize("precision,tol", [("fp64", 1e-9), ("mixed", 1e-4)])
def test_curved_rays_match_oracle(cfg, n, n_ant, formalism, precision, tol):
    """The refracted-ray propagator: the ray's direction at the emission point
    and its travel time (a fixed-point ray solve plus Fermat's form of the time
    saved on the GPU; Newton on Snell's invariant with composite quadrature in
    the oracle), on the inclined shower, where the bending shows most."""
    w = synth.workload(cfg, n_tracks=n, n_ant=n_ant)
    w["medium"] = dict(synth.AIR_EXPONENTIAL, kind="exponential_ray")
    if precision == "mixed":
        w["dtype"] = np.float32
    tracks = synth.workload_tracks(w)
    if formalism == "endpoint":
        keep = endpoint_unambiguous(tracks, w["ant_xyz"], w["t_start_ns"], w["n_bins"], w["dt_ns"], w["medium"])
        tracks = drop_tracks(tracks, keep)
    ref, kept = oracle_traces(tracks, w["ant_xyz"], w["t_start_ns"], w["n_bins"], w["dt_ns"], w["medium"], formalism)
    flat, _ = oracle_traces(tracks, w["ant_xyz"], w["t_start_ns"], w["n_bins"], w["dt_ns"], synth.AIR_EXPONENTIAL,
                            formalism)
    if cfg == 2:  # inclined: the paths are long and slanted, the bending shows
        assert rel_l2(flat, ref) > 2e-4
    gpu, arr, st = run(w, tracks, formalism, precision)
    assert st["tracks_kept"] == kept
    err = rel_l2(gpu, ref)
    assert err <= tol, f"relative L2 {err:.3e} > {tol:.0e}"
    obr, ou = oracle_arrivals(tracks, w["ant_xyz"], w["t_start_ns"], w["n_bins"], w["dt_ns"], w["medium"], formalism)
    n_cmp, _ = compare_bins(arr[0], arr[1], arr[2], obr, ou, w["n_bins"])
    assert n_cmp > 0.99 * obr.size


@pytest.mark.parametrize("medium_name,D,place", NEAR_CHERENKOV_CASES)
@pytest.mark.parametrize("formalism", ["endpoint", "zhs"])
@pytest.mark.parametrize("precision,tol", [("fp64", 1e-9), ("mixed", 1e-4)])
def test_constructed_near_cherenkov_pairs(medium_name, D, place, formalism, precision, tol):
    """One track and one antenna at D_m = +-1e-4 or +-1e-6 (the near-Cherenkov
    treatment of reading C, and ZHS intervals of 3e-3 to 3e-5 bin), element by
    element against the oracle.  With both linearised arrivals in one bin the
    Endpoint pair must give exactly 0 on both sides."""
    medium = AIR_UNIFORM if medium_name == "uniform" else AIR_EXP
    N, K = 64, 32
    tracks, ant, t_start = near_cherenkov_pair(D, place, medium, n_bins=N, K=K)
    w = dict(medium=medium, ant_xyz=ant, t_start_ns=t_start, n_bins=N, dt_ns=0.2)
    ref, kept = oracle_traces(tracks, ant, t_start, N, 0.2, medium, formalism)
    gpu, arr, st = run(w, tracks, formalism, precision)
    assert kept == 1 and st["tracks_kept"] == 1
    expect_branch = (1 if formalism == "endpoint" else (2 if place == "same" else 3))
    assert int(arr[0][0, 0]) == expect_branch
    if formalism == "endpoint" and place == "same":
        assert not ref.any() and not gpu.any()
        return
    assert np.abs(ref).max() > 0
    if formalism == "zhs" and place == "straddle":
        # the two halves of an interval W = |D| (t1 - t0)/dt bins wide split at an
        # edge carry the rounding of the arrival itself over W: in FP64 the
        # arrival is a sum of terms of up to ~2e4 bins (the window start and the
        # travel time), each of a handful of roundings off by up to 1.8e-12 bin
        # (half an ulp of 2e4), so each side is good to ~1e-11 bin and oracle
        # and GPU may differ by ~2e-11/W (6e-9 at D = 1e-4, 6e-7 at 1e-6)
        W = abs(D) * (tracks["t1"][0] - tracks["t0"][0]) / 0.2
        tol = max(tol, 2e-11 / W)
    err = np.abs(gpu - ref).max() / np.abs(ref).max()
    assert err <= tol, f"largest element difference {err:.3e} of the largest element (bar {tol:.1e})"
    np.testing.assert_array_equal(gpu != 0, ref != 0)


@pytest.mark.parametrize("medium", [{"kind": "uniform", "n": 1.78},
                                    {"kind": "exponential", "N0": 0.1, "H": 1000.0}])
@pytest.mark.parametrize("formalism", ["endpoint", "zhs"])
@pytest.mark.parametrize("precision,tol", [("fp64", 1e-9), ("mixed", 1e-4)])
def test_dense_media_match_oracle(medium, formalism, precision, tol):
    """Dense media, where the FP32 arrival's error bound (and the refractivity
    term in it) is far from the air showers': ice (n = 1.78, a wide Cherenkov
    cone, many near-Cherenkov pairs, most arrivals outside the window) and a
    steep exponential atmosphere (N0 = 0.1, H = 1 km).  In ice the antennas lie
    0.6-3 km from the axis on one line, where some tracks see them near the 56
    degree cone.  Every window is placed around the median of the oracle's
    arrivals at that antenna."""
    w = synth.workload(0, n_tracks=8009, n_ant=16)
    w["medium"] = dict(medium)
    if medium["kind"] == "uniform":
        w["ant_xyz"] = np.stack([np.linspace(600.0, 3000.0, 16), np.zeros(16), np.zeros(16)], 1)
    if precision == "mixed":
        w["dtype"] = np.float32
    tracks = synth.workload_tracks(w)
    _, u0 = oracle_arrivals(tracks, w["ant_xyz"], np.zeros(16), 1, w["dt_ns"], w["medium"], formalism)
    w["t_start_ns"] = np.median(u0.reshape(len(tracks["x0"]), 16, 2)[..., 0], axis=0) * w["dt_ns"] - 300.0
    ref, kept = oracle_traces(tracks, w["ant_xyz"], w["t_start_ns"], w["n_bins"], w["dt_ns"], w["medium"], formalism)
    gpu, arr, st = run(w, tracks, formalism, precision)
    assert st["tracks_kept"] == kept
    assert np.abs(ref).max() > 0
    obr, ou = oracle_arrivals(tracks, w["ant_xyz"], w["t_start_ns"], w["n_bins"], w["dt_ns"], w["medium"], formalism)
    if formalism == "endpoint":
        ref = either_bin_reference(gpu, ref, tracks, w["ant_xyz"], w["t_start_ns"], w["n_bins"], w["dt_ns"],
                                   w["medium"])
        assert (obr == 1).sum() > 0
    err = rel_l2(gpu, ref)
    assert err <= tol, f"relative L2 {err:.3e} > {tol:.0e}"
    n_cmp, _ = compare_bins(arr[0], arr[1], arr[2], obr, ou, w["n_bins"])
    # most arrivals here lie outside the window, where the listing clamps a ZHS
    # interval to one bin; every arrival of a pair that reaches it is compared
    reach = ~((ou < 0).all(axis=-1) | (ou >= w["n_bins"]).all(axis=-1))
    assert reach.sum() > 1000 and n_cmp > 0.99 * 2 * reach.sum()


ICE = {"kind": "uniform", "n": 1.78}
FORM_CASES = [
    # (cfg, n_tracks, n_ant, ice): where each form of the FP32 arrival pays and where not
    (1, 20011, 160, False),   # vertical shower, star array: lines of sight near the vertical
    (2, 20011, 256, False),   # 60 degrees, 32 x 32 grid: inclined lines of sight
    (0, 20011, 16, False),    # uniform medium, a line of antennas
    (0, 8009, 16, True),      # ice, antennas 0.6-3 km out: near-horizontal lines of sight
]


def form_workload(cfg, n, n_ant, ice):
    w = synth.workload(cfg, n_tracks=n, n_ant=n_ant)
    w["dtype"] = np.float32
    if ice:
        w["medium"] = dict(ICE)
        w["ant_xyz"] = np.stack([np.linspace(600.0, 3000.0, 16), np.zeros(16), np.zeros(16)], 1)
    tracks = synth.workload_tracks(w)
    if ice:
        _, u0 = oracle_arrivals(tracks, w["ant_xyz"], np.zeros(16), 1, w["dt_ns"], w["medium"], "endpoint")
        w["t_start_ns"] = np.median(u0.reshape(len(tracks["x0"]), 16, 2)[..., 0], axis=0) * w["dt_ns"] - 300.0
    return w, tracks


@pytest.mark.parametrize("form", ["split", "direct"])
@pytest.mark.parametrize("cfg,n,n_ant,ice", FORM_CASES)
def test_arrival_forms_match_oracle(cfg, n, n_ant, ice, form):
    """Each form of the FP32 arrival of the mixed one-bin Endpoint kernels,
    pinned, against the oracle at the mixed bar, antenna by antenna, on a
    geometry where it pays and on ones where it does not: a bin comes from the
    FP32 arrival only where its bound leaves no edge in reach."""
    w, tracks = form_workload(cfg, n, n_ant, ice)
    check_form(w, tracks, form)


def check_form(w, tracks, form):
    ref, kept = oracle_traces(tracks, w["ant_xyz"], w["t_start_ns"], w["n_bins"], w["dt_ns"], w["medium"], "endpoint")
    p = process(w, "endpoint", "mixed")
    p.set_arrival_form(form)
    p.push(to_device(tracks, torch.float32))
    gpu = p.traces().cpu().numpy()
    st = p.stats()
    p.close()
    assert st["tracks_kept"] == kept and st["arrival_form"] == form
    ref = either_bin_reference(gpu, ref, tracks, w["ant_xyz"], w["t_start_ns"], w["n_bins"], w["dt_ns"], w["medium"])
    assert np.abs(ref).max() > 0
    err = rel_l2(gpu, ref)
    assert err <= 1e-4, f"relative L2 {err:.3e}"
    per_ant = [rel_l2(gpu[a], ref[a]) for a in range(len(ref)) if np.abs(ref[a]).max() > 0]
    assert max(per_ant) <= 1e-4, f"worst antenna: relative L2 {max(per_ant):.3e}"


@pytest.mark.parametrize("form", ["split", "direct"])
@pytest.mark.parametrize("case", ["antennas_inside_the_shower", "late_time_origin"])
def test_arrival_forms_edge_geometries(case, form):
    """Both forms where their arithmetic changes branch or scale: antennas at
    4 km, the shower's median track height, so that half of the emission points
    lie below them (the split form's direct fallback, x = R + s_z >= R); and a
    time origin 1e6 ns before the shower (shifted times near 5e6 bins, where the
    float-float forms of T and the u^2 terms of the bound matter)."""
    w = synth.workload(1, n_tracks=6007, n_ant=16)
    w["dtype"] = np.float32
    tracks = synth.workload_tracks(w)
    if case == "antennas_inside_the_shower":
        ant = np.asarray(w["ant_xyz"], np.float64).copy()
        ant[:, 2] = 4000.0
        w["ant_xyz"] = ant
        _, u0 = oracle_arrivals(tracks, ant, np.zeros(16), 1, w["dt_ns"], w["medium"], "endpoint")
        w["t_start_ns"] = np.median(u0.reshape(len(tracks["x0"]), 16, 2)[..., 0], axis=0) * w["dt_ns"] - 300.0
        assert (tracks["z0"] < 4000.0).mean() > 0.3
    else:
        off = 1.0e6
        tracks = dict(tracks)
        tracks["t0"] = (tracks["t0"].astype(np.float64) + off).astype(np.float32)
        tracks["t1"] = (tracks["t1"].astype(np.float64) + off).astype(np.float32)
        w["t_start_ns"] = np.asarray(w["t_start_ns"], np.float64) + off
    check_form(w, tracks, form)


@pytest.mark.parametrize("cfg,n_ant,expect", [(1, 160, "split"), (2, 256, "direct")])
def test_arrival_form_chosen_from_the_tracks(cfg, n_ant, expect):
    """The automatic choice: before any push the split form; each push's ingest
    counts the tracks whose start point sees the antenna array from above within
    45 degrees, and later pushes follow the count (split for the vertical
    shower, direct for the 60-degree one).  The bins are the same in both forms,
    so a push in either form gives the same traces up to the order of the
    additions; a new antenna layout starts over."""
    w, tracks = form_workload(cfg, 20011, n_ant, False)
    dev = to_device(tracks, torch.float32)
    p = process(w, "endpoint", "mixed")
    assert p.stats()["arrival_form"] == "split"
    p.push(dev)
    first = p.traces(reset=True).cpu().numpy()
    assert p.stats()["arrival_form"] == expect
    p.push(dev)
    second = p.traces(reset=True).cpu().numpy()
    assert rel_l2(second, first) <= 1e-6
    assert np.abs(second - first).max() <= 1e-5 * np.abs(first).max()
    p.set_antenna_positions(np.asarray(w["ant_xyz"])[::-1].copy())   # same layout: the count stays
    assert p.stats()["arrival_form"] == expect
    p.close()


@pytest.mark.parametrize("formalism", ["endpoint", "zhs"])
@pytest.mark.parametrize("precision,tol", [("fp64", 1e-9), ("mixed", 1e-4)])
def test_uneven_antenna_altitudes(formalism, precision, tol):
    """The exponential atmosphere with antennas at different altitudes (0-150 m),
    where the refractivity quotient (E_e - E_a)/(z_a - z_e) is formed per pair
    (a flat array forms it once per track): every antenna at the bar."""
    w = synth.workload(1, n_tracks=6007, n_ant=16)
    if precision == "mixed":
        w["dtype"] = np.float32
    ant = np.asarray(w["ant_xyz"], np.float64).copy()
    ant[:, 2] = np.linspace(0.0, 150.0, 16)
    w["ant_xyz"] = ant
    tracks = synth.workload_tracks(w)
    _, u0 = oracle_arrivals(tracks, ant, np.zeros(16), 1, w["dt_ns"], w["medium"], formalism)
    w["t_start_ns"] = np.median(u0.reshape(len(tracks["x0"]), 16, 2)[..., 0], axis=0) * w["dt_ns"] - 300.0
    ref, kept = oracle_traces(tracks, ant, w["t_start_ns"], w["n_bins"], w["dt_ns"], w["medium"], formalism)
    gpu, _, st = run(w, tracks, formalism, precision)
    assert st["tracks_kept"] == kept and np.abs(ref).max() > 0
    if formalism == "endpoint":
        ref = either_bin_reference(gpu, ref, tracks, ant, w["t_start_ns"], w["n_bins"], w["dt_ns"], w["medium"])
    per_ant = [rel_l2(gpu[a], ref[a]) for a in range(16) if np.abs(ref[a]).max() > 0]
    assert max(per_ant) <= tol, f"worst antenna: relative L2 {max(per_ant):.3e}"


@pytest.mark.parametrize("formalism", ["endpoint", "zhs"])
@pytest.mark.parametrize("cfg", [1, 2])
def test_flat_array_kernel_matches_the_per_pair_quotient(cfg, formalism):
    """A flat array (every antenna at z = 0) takes the kernel that forms the
    refractivity quotient once per track (Endpoint: the direct arrival form;
    ZHS: the midpoint's quotient in float-float); moving one antenna by 1 mm
    in z takes the kernel that forms it per pair.  The quotient is the same
    arithmetic either way, so the other antennas' traces agree to the order of
    the additions (vertical and 60-degree showers; Endpoint with the direct
    form pinned)."""
    w = synth.workload(cfg, n_tracks=20011, n_ant=32 if cfg == 1 else 64)
    w["dtype"] = np.float32
    tracks = synth.workload_tracks(w)
    dev = to_device(tracks, torch.float32)
    out = []
    for dz in (0.0, 1e-3):
        ant = np.asarray(w["ant_xyz"], np.float64).copy()
        ant[-1, 2] += dz
        p = process(dict(w, ant_xyz=ant), formalism, "mixed")
        if formalism == "endpoint":
            p.set_arrival_form("direct")
        p.push(dev)
        out.append(p.traces().cpu().numpy()[:-1].astype(np.float64))
        p.close()
    assert np.abs(out[0]).max() > 0
    assert rel_l2(out[1], out[0]) <= 1e-6
    assert np.abs(out[1] - out[0]).max() <= 1e-5 * np.abs(out[0]).max()
