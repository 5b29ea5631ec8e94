"""The linear (two-bin) deposit on the GPU (c8r_set_deposit) against the oracle:
traces of both formalisms in both precisions (bars 1e-9 / 1e-4 relative L2, as
for the one-bin deposit), and the adjoints, whose time gradients are now
informative.  The linear traces are continuous in the arrival times, so the
forward comparison needs no edge exclusions; the gradients hold the cell of
each deposit fixed and change at the bin centres, so tracks with an arrival
within 1e-6 bin of a bin centre are left out of the gradient comparison."""
import numpy as np
import pytest

import oracle
from _util import built_lib, drop_tracks, oracle_arrivals, rel_l2, to_device
from paper_2309_03717_gb300 import synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

ICE = {"kind": "uniform", "n": 1.78}


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    built_lib()


def _oracle_form(formalism):
    return oracle.ENDPOINT if formalism == "endpoint" else oracle.ZHS


def oracle_linear(tracks, w, formalism, eps_C=1e-3, medium=None):
    out, kept = oracle.forward(oracle.tracks_from_ns(tracks), w["ant_xyz"], np.asarray(w["t_start_ns"]) * 1e-9,
                               w["n_bins"], w["dt_ns"] * 1e-9, medium or w["medium"], _oracle_form(formalism), eps_C,
                               deposit=oracle.DEPOSIT_LINEAR)
    return out, kept


def gpu_linear(tracks, w, formalism, precision, eps_C=None, medium=None, shape=None):
    from paper_2309_03717_gb300.c8r import RadioProcess
    p = RadioProcess(medium or w["medium"], w["ant_xyz"], w["t_start_ns"], w["n_bins"], w["dt_ns"], formalism,
                     precision, eps_C=eps_C, deposit="linear")
    if shape:
        p.set_launch_shape(*shape)
    p.push(to_device(tracks, torch.float64 if precision == "fp64" else torch.float32))
    out = p.traces().cpu().numpy()
    st = p.stats()
    p.close()
    return out, st


CASES = [
    (0, 20011, 16, "endpoint", "fp64", 1e-9),
    (0, 20011, 16, "zhs", "fp64", 1e-9),
    (1, 6007, 40, "endpoint", "fp64", 1e-9),
    (1, 6007, 40, "zhs", "fp64", 1e-9),
    (1, 20011, 160, "endpoint", "mixed", 1e-4),
    (1, 20011, 160, "zhs", "mixed", 1e-4),
    (2, 6007, 64, "endpoint", "fp64", 1e-9),
    (2, 20011, 256, "zhs", "mixed", 1e-4),
    (2, 20011, 256, "endpoint", "mixed", 1e-4),
]


@pytest.mark.parametrize("cfg,n,n_ant,formalism,precision,tol", CASES)
def test_linear_traces_match_oracle(cfg, n, n_ant, formalism, precision, tol):
    w = synth.workload(cfg, n_tracks=n, n_ant=n_ant)
    if precision == "mixed":
        w["dtype"] = np.float32
    tracks = synth.workload_tracks(w)
    ref, kept = oracle_linear(tracks, w, formalism)
    gpu, st = gpu_linear(tracks, w, formalism, precision)
    assert st["tracks_kept"] == kept
    assert np.abs(ref).max() > 0
    err = rel_l2(gpu, ref)
    assert err <= tol, f"relative L2 {err:.3e} > {tol:.0e}"
    # the one-bin traces differ: the deposit shape is in effect
    one, _ = oracle.forward(oracle.tracks_from_ns(tracks), w["ant_xyz"], np.asarray(w["t_start_ns"]) * 1e-9,
                            w["n_bins"], w["dt_ns"] * 1e-9, w["medium"], _oracle_form(formalism))
    assert rel_l2(one, ref) > 100 * tol


@pytest.mark.parametrize("formalism", ["endpoint", "zhs"])
@pytest.mark.parametrize("precision,tol", [("fp64", 1e-9), ("mixed", 1e-4)])
def test_linear_near_cherenkov_in_ice(formalism, precision, tol):
    """A dense medium with a wide near-Cherenkov band (eps_C = 0.05): most
    Endpoint pairs take the midpoint branch, in both of its linear forms."""
    w = synth.workload(0, n_tracks=3001, n_ant=16)
    if precision == "mixed":
        w["dtype"] = np.float32  # FP32-exact tracks (beta renormalised below 1 after rounding)
    tracks = synth.workload_tracks(w)
    # start the tracks 100-130 m up, so that in ice their arrivals fit the window
    h = 100.0 + 30.0 * (np.arange(len(tracks["z0"])) % 97) / 97.0
    dz = (h - tracks["z0"]).astype(np.float32)
    tracks["z0"] = (tracks["z0"] + dz).astype(np.float32)
    tracks["z1"] = (tracks["z1"] + dz).astype(np.float32)
    dur = tracks["t1"].astype(np.float64) - tracks["t0"]
    tracks["t0"] = np.zeros_like(tracks["t0"])
    tracks["t1"] = dur.astype(np.float32)
    w2 = dict(w)
    br, u = oracle.arrivals(oracle.tracks_from_ns(tracks), w["ant_xyz"], np.zeros(16), 1, w["dt_ns"] * 1e-9, ICE,
                            oracle.ZHS)
    w2["t_start_ns"] = (u.min(axis=(0, 2)) - 200.0) * w["dt_ns"]
    ref, kept = oracle_linear(tracks, w2, formalism, 0.05, ICE)
    gpu, st = gpu_linear(tracks, w2, formalism, precision, eps_C=0.05, medium=ICE)
    assert st["tracks_kept"] == kept
    if formalism == "endpoint":
        obr, _ = oracle.arrivals(oracle.tracks_from_ns(tracks), w2["ant_xyz"], np.asarray(w2["t_start_ns"]) * 1e-9,
                                 w2["n_bins"], w2["dt_ns"] * 1e-9, ICE, oracle.ENDPOINT, 0.05)
        assert (obr == 1).mean() > 0.05
    err = rel_l2(gpu, ref)
    assert err <= tol, f"relative L2 {err:.3e} > {tol:.0e}"


@pytest.mark.parametrize("formalism", ["endpoint", "zhs"])
def test_linear_invariant_to_launch_shape(formalism):
    w = synth.workload(1, n_tracks=9001, n_ant=24)
    tracks = synth.workload_tracks(w)
    base, _ = gpu_linear(tracks, w, formalism, "mixed")
    for shape in [(1, 1, 0), (3, 16, 1000), (32, 2, 0)]:
        other, _ = gpu_linear(tracks, w, formalism, "mixed", shape=shape)
        assert rel_l2(other, base) <= 2e-6, shape


def _cells_clear(tracks, w, formalism, tol):
    """Tracks none of whose arrivals lies within tol bin of a bin centre (where
    the cell of a deposit, and with it the gradient, changes)."""
    _, u = oracle_arrivals(tracks, w["ant_xyz"], w["t_start_ns"], w["n_bins"], w["dt_ns"], w["medium"], formalism)
    v = u + 0.5
    fr = v - np.floor(v)
    return ~(np.minimum(fr, 1.0 - fr) < tol).any(axis=-1).any(axis=-1), u


@pytest.mark.parametrize("formalism", ["endpoint", "zhs"])
@pytest.mark.parametrize("precision,tol", [("fp64", 1e-9), ("mixed", 1e-4)])
def test_linear_adjoint_matches_oracle_gradient(formalism, precision, tol):
    from paper_2309_03717_gb300 import c8r
    w = synth.workload(4, n_tracks=3001, n_ant=16)
    tracks = synth.workload_tracks(w)
    keep, u = _cells_clear(tracks, w, formalism, 1e-6)
    # an interval (ZHS, or the two near-Cherenkov Endpoint arrivals) across a
    # bin centre: its gradient goes through the fractions of the interval on
    # either side, slopes 1/W, so the FP64 rounding of the arrival (~4e-11 bin)
    # reaches it as ~4e-11/W; such narrow straddling intervals are left out
    v = u + 0.5
    straddle = np.floor(v[..., 0]) != np.floor(v[..., 1])
    narrow = np.abs(u[..., 1] - u[..., 0]) < 0.05
    if formalism == "endpoint":
        br, _ = oracle_arrivals(tracks, w["ant_xyz"], w["t_start_ns"], w["n_bins"], w["dt_ns"], w["medium"],
                                "endpoint")
        straddle &= br == 1
    keep &= ~(straddle & narrow).any(axis=1)
    assert keep.mean() > 0.8
    tracks = drop_tracks(tracks, keep)
    dt = torch.float64 if precision == "fp64" else torch.float32
    p = c8r.RadioProcess(w["medium"], w["ant_xyz"], w["t_start_ns"], w["n_bins"], w["dt_ns"], formalism, precision,
                         deposit="linear")
    dev = to_device(tracks, dt)
    p.push(dev)
    # dL/dtrace of the squared misfit against perturbed endpoints and N0 x 1.02,
    # from the oracle's traces, scaled to order one
    tgt_tracks = synth.perturbed_target_tracks(tracks, 77)
    med2 = dict(w["medium"])
    med2["N0"] *= 1.02
    diff = oracle_linear(tracks, w, formalism)[0] - oracle_linear(tgt_tracks, w, formalism, medium=med2)[0]
    G = torch.from_numpy(2.0 * diff / np.abs(diff).max()).to(dt).cuda()
    n = tracks["x0"].size
    tg = {f: torch.zeros(n, dtype=dt, device="cuda") for f in c8r.GRAD_FIELDS}
    ag = torch.zeros((len(w["ant_xyz"]), 3), dtype=torch.float64, device="cuda")
    dn = torch.zeros(1, dtype=torch.float64, device="cuda")
    c8r.c8r_backward(p.ctx, dev, G, tg, ag, dn)
    torch.cuda.synchronize()
    p.close()
    tg_ref, ag_ref, dn_ref = oracle.backward(oracle.tracks_from_ns(tracks), w["ant_xyz"], w["t_start_ns"] * 1e-9,
                                             w["n_bins"], w["dt_ns"] * 1e-9, w["medium"], G.double().cpu().numpy(),
                                             formalism=_oracle_form(formalism), deposit=oracle.DEPOSIT_LINEAR)
    got = np.stack([tg[f].double().cpu().numpy() for f in c8r.GRAD_FIELDS], axis=1)
    # the times get gradients (the oracle's per second, ours per ns)
    assert np.abs(tg_ref[:, 6:8]).max() > 0
    assert rel_l2(got[:, 6:8], tg_ref[:, 6:8] * 1e-9) <= tol
    assert rel_l2(got[:, 0:6], tg_ref[:, 0:6]) <= tol
    assert rel_l2(got[:, 8:11], tg_ref[:, 8:11]) <= tol
    assert rel_l2(ag.cpu().numpy(), ag_ref) <= tol
    assert abs(dn.item() - dn_ref) <= tol * abs(dn_ref)


def test_linear_autograd_uses_the_context_deposit():
    from paper_2309_03717_gb300 import c8r
    w = synth.workload(4, n_tracks=1500, n_ant=8, seed_offset=3)
    tracks = synth.workload_tracks(w)
    p = c8r.RadioProcess(w["medium"], w["ant_xyz"], w["t_start_ns"], w["n_bins"], w["dt_ns"], "endpoint", "mixed",
                         deposit="linear")
    dev = to_device(tracks)
    leaves = {f: dev[f].clone().requires_grad_(f != "q") for f in synth.FIELDS}
    ant = torch.tensor(w["ant_xyz"], device="cuda", requires_grad=True)
    N0 = torch.tensor(w["medium"]["N0"], dtype=torch.float64, device="cuda", requires_grad=True)
    out = c8r.RadioTraces.apply(p, N0, *[leaves[f] for f in synth.FIELDS], ant)
    (out * torch.randn_like(out)).sum().backward()
    assert leaves["t0"].grad.abs().max() > 0 and leaves["t1"].grad.abs().max() > 0
    p.close()


@pytest.mark.parametrize("formalism", ["endpoint", "zhs"])
@pytest.mark.parametrize("precision,tol", [("fp64", 1e-9), ("mixed", 1e-4)])
def test_linear_window_edges(formalism, precision, tol):
    """A short window (48 bins) whose start sits just after the first arrivals:
    spread deposits and ZHS intervals are cut by both window ends (cells -1, 0,
    N and N + 1 of the linear deposit)."""
    w = synth.workload(0, n_tracks=4001, n_ant=16)
    if precision == "mixed":
        w["dtype"] = np.float32
    tracks = synth.workload_tracks(w)
    _, u = oracle_arrivals(tracks, w["ant_xyz"], np.zeros(16), 1, w["dt_ns"], w["medium"], formalism)
    w = dict(w)
    w["n_bins"] = 48
    w["t_start_ns"] = (np.median(u.reshape(-1, 16, 2)[..., 0], axis=0) - 24.3) * w["dt_ns"]
    ref, kept = oracle_linear(tracks, w, formalism)
    gpu, st = gpu_linear(tracks, w, formalism, precision)
    assert st["tracks_kept"] == kept
    _, u2 = oracle_arrivals(tracks, w["ant_xyz"], w["t_start_ns"], w["n_bins"], w["dt_ns"], w["medium"], formalism)
    assert ((u2 > -1) & (u2 < 0.5)).any() and ((u2 > 47.5) & (u2 < 49)).any()  # both edges are crossed
    assert np.abs(ref).max() > 0
    err = rel_l2(gpu, ref)
    assert err <= tol, f"relative L2 {err:.3e} > {tol:.0e}"


@pytest.mark.parametrize("kind", ["exponential_spherical", "exponential_ray"])
@pytest.mark.parametrize("formalism", ["endpoint", "zhs"])
@pytest.mark.parametrize("precision,tol", [("fp64", 1e-9), ("mixed", 1e-4)])
def test_linear_deposit_with_spherical_and_curved_ray_media(kind, formalism, precision, tol):
    """The linear deposit combined with the two heavier propagators, on the
    inclined shower."""
    w = synth.workload(2, n_tracks=2003, n_ant=48)
    w["medium"] = dict(synth.AIR_SPHERICAL) if kind == "exponential_spherical" else dict(synth.AIR_EXPONENTIAL,
                                                                                         kind="exponential_ray")
    if precision == "mixed":
        w["dtype"] = np.float32
    tracks = synth.workload_tracks(w)
    ref, kept = oracle_linear(tracks, w, formalism)
    gpu, st = gpu_linear(tracks, w, formalism, precision)
    assert st["tracks_kept"] == kept
    assert np.abs(ref).max() > 0
    err = rel_l2(gpu, ref)
    assert err <= tol, f"relative L2 {err:.3e} > {tol:.0e}"
