"""The hand-written adjoints (Endpoint and ZHS) on the GPU against the oracle's
FP64 reverse gradients (which the CPU tests pin with central finite
differences).  Bars: relative L2 <= 1e-9 (FP64 path), <= 1e-4 (mixed path), per
gradient group."""
import numpy as np
import pytest

import oracle
from _util import built_lib, drop_tracks, oracle_arrivals, rel_l2, to_device, unambiguous
from paper_2309_03717_gb300 import synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    built_lib()


def setup(precision, n=3001, n_ant=16, seed_off=0, formalism="endpoint", uneven=False):
    from paper_2309_03717_gb300 import c8r
    w = synth.workload(4, n_tracks=n, n_ant=n_ant, seed_offset=seed_off)
    tracks = synth.workload_tracks(w)
    if uneven:
        # antennas at 0-150 m: the refractivity quotient is formed per pair (a
        # flat array forms it once per track); each trace window is placed
        # around the antenna's median arrival
        ant = np.asarray(w["ant_xyz"], np.float64).copy()
        ant[:, 2] = np.linspace(0.0, 150.0, n_ant)
        w["ant_xyz"] = ant
        _, u0 = oracle_arrivals(tracks, ant, np.zeros(n_ant), 1, w["dt_ns"], w["medium"], formalism)
        w["t_start_ns"] = np.median(u0.reshape(len(tracks["x0"]), n_ant, 2)[..., 0], axis=0) * w["dt_ns"] - 200.0
    # away from the kinks (an arrival within 1e-6 bin of an edge may take either bin)
    keep = unambiguous(tracks, w["ant_xyz"], w["t_start_ns"], w["n_bins"], w["dt_ns"], w["medium"], formalism)
    if formalism == "zhs":
        # The ZHS gradients go through the fractions of the interval [u_lo, u_hi]
        # in its end bins, whose slopes are 1/W, W = u_hi - u_lo.  The rounding of
        # the arrival itself (~4e-11 bin in FP64: it is a difference of ~1e5-bin
        # terms) therefore reaches the gradient as ~4e-11/W relative: ~2e-8 for
        # the narrow edge-straddling intervals near the Cherenkov angle, where the
        # oracle and the GPU differ at that level, both off the exact value (an
        # mpmath check of one such pair).  Tracks with an edge-straddling interval
        # narrower than 0.05 bin at any antenna (about 1 in 10) are left out.
        br, u = oracle_arrivals(tracks, w["ant_xyz"], w["t_start_ns"], w["n_bins"], w["dt_ns"], w["medium"], "zhs")
        narrow = (br == 3) & (u[..., 1] - u[..., 0] < 0.05)
        keep &= ~narrow.any(axis=1)
        assert keep.mean() > 0.8
    tracks = drop_tracks(tracks, keep)
    p = c8r.RadioProcess(w["medium"], w["ant_xyz"], w["t_start_ns"], w["n_bins"], w["dt_ns"], formalism, precision)
    return c8r, w, tracks, p


@pytest.mark.parametrize("formalism", ["endpoint", "zhs"])
@pytest.mark.parametrize("precision,tol", [("fp64", 1e-9), ("mixed", 1e-4)])
def test_adjoint_matches_oracle_gradient(precision, tol, formalism):
    check_adjoint(precision, tol, formalism)


def test_mixed_zhs_adjoint_with_a_constant_gradient_part():
    """The mixed ZHS adjoint sums dL/dtrace over the whole bins of an interval
    as a difference of running sums over the 2048 bins.  A constant part of
    dL/dtrace (here twice the size of the varying part) makes the sums grow with
    the bin index to ~4e3, where FP32 rounds at ~2e-4, while a run of a few bins
    sums to ~1; the float-float sums keep the bar."""
    check_adjoint("mixed", 1e-4, "zhs", offset=2.0)


def check_adjoint(precision, tol, formalism, offset=0.0, form=None, uneven=False):
    c8r, w, tracks, p = setup(precision, formalism=formalism, uneven=uneven)
    if form:
        p.set_arrival_form(form)
    dt = torch.float64 if precision == "fp64" else torch.float32
    dev = to_device(tracks, dt)
    # loss = sum (trace - target)^2 against traces of 1%-perturbed endpoints and
    # N0 x 1.02; dL/dtrace is formed from the oracle's traces (an input of both
    # adjoints) and scaled to order one, as in FP32 training: unscaled, a squared
    # loss of ZHS potentials (~1e-19 V s/m) has gradients near 1e-38, below FP32
    tgt_tracks = synth.perturbed_target_tracks(tracks, 77)
    med2 = dict(w["medium"])
    med2["N0"] *= 1.02
    form = oracle.ZHS if formalism == "zhs" else oracle.ENDPOINT
    args = (w["ant_xyz"], w["t_start_ns"] * 1e-9, w["n_bins"], w["dt_ns"] * 1e-9)
    diff = (oracle.forward(oracle.tracks_from_ns(tracks), *args, w["medium"], form)[0]
            - oracle.forward(oracle.tracks_from_ns(tgt_tracks), *args, med2, form)[0])
    G = torch.from_numpy(2.0 * diff / np.abs(diff).max() + offset).to(dt).cuda()
    n = tracks["x0"].size
    tg = {f: torch.zeros(n, dtype=dt, device="cuda") for f in c8r.GRAD_FIELDS}
    ag = torch.zeros((len(w["ant_xyz"]), 3), dtype=torch.float64, device="cuda")
    dn = torch.zeros(1, dtype=torch.float64, device="cuda")
    c8r.c8r_backward(p.ctx, dev, G, tg, ag, dn)
    torch.cuda.synchronize()
    p.close()
    tg_ref, ag_ref, dn_ref = oracle.backward(oracle.tracks_from_ns(tracks), w["ant_xyz"], w["t_start_ns"] * 1e-9,
                                             w["n_bins"], w["dt_ns"] * 1e-9, w["medium"], G.double().cpu().numpy(),
                                             formalism=oracle.ZHS if formalism == "zhs" else oracle.ENDPOINT)
    got = np.stack([tg[f].double().cpu().numpy() for f in c8r.GRAD_FIELDS], axis=1)
    if formalism == "endpoint":
        # bins fixed: the Endpoint deposits do not depend on the times
        assert np.all(got[:, 6:8] == 0.0) and np.all(tg_ref[:, 6:8] == 0.0)
    else:
        # the oracle's time gradients are per second, ours per ns
        assert np.abs(tg_ref[:, 6:8]).max() > 0
        assert rel_l2(got[:, 6:8], tg_ref[:, 6:8] * 1e-9) <= tol
    assert rel_l2(got[:, 0:6], tg_ref[:, 0:6]) <= tol
    assert rel_l2(got[:, 8:11], tg_ref[:, 8:11]) <= tol
    assert rel_l2(ag.cpu().numpy(), ag_ref) <= tol
    assert abs(dn.item() - dn_ref) <= tol * abs(dn_ref)


@pytest.mark.parametrize("formalism", ["endpoint", "zhs"])
@pytest.mark.parametrize("precision,tol", [("fp64", 1e-9), ("mixed", 1e-4)])
def test_adjoint_with_uneven_antenna_altitudes(precision, tol, formalism):
    """The adjoints for an array that is not flat (antennas at 0-150 m), where
    the mixed kernels form the refractivity quotient per pair rather than once
    per track."""
    check_adjoint(precision, tol, formalism, uneven=True)


@pytest.mark.parametrize("form", ["split", "direct"])
def test_mixed_endpoint_adjoint_in_both_arrival_forms(form):
    """The Endpoint adjoint takes its bins as the forward kernel does, from the
    FP32 arrival in the pinned form where its bound leaves no edge in reach."""
    check_adjoint("mixed", 1e-4, "endpoint", form=form)


@pytest.mark.parametrize("formalism", ["endpoint", "zhs"])
def test_autograd_function_routes_to_the_adjoint(formalism):
    c8r, w, tracks, p = setup("mixed", n=1500, n_ant=8, seed_off=3, formalism=formalism)
    dev = to_device(tracks)
    leaves = {f: dev[f].clone().requires_grad_(f != "q") for f in synth.FIELDS}
    ant = torch.tensor(w["ant_xyz"], device="cuda", requires_grad=True)
    N0 = torch.tensor(w["medium"]["N0"], dtype=torch.float64, device="cuda", requires_grad=True)
    out = c8r.RadioTraces.apply(p, N0, *[leaves[f] for f in synth.FIELDS], ant)
    G = torch.randn_like(out)
    (out * G).sum().backward()
    tg = {f: torch.zeros(tracks["x0"].size, dtype=torch.float32, device="cuda") for f in c8r.GRAD_FIELDS}
    ag = torch.zeros((len(w["ant_xyz"]), 3), dtype=torch.float64, device="cuda")
    dn = torch.zeros(1, dtype=torch.float64, device="cuda")
    c8r.c8r_backward(p.ctx, dev, G, tg, ag, dn)
    # a track's gradients are summed with FP32 reductions (one per antenna tile,
    # and one per endpoint evaluated after the main pass) whose order differs
    # between two runs: equal to FP32 rounding of the largest terms
    for f in c8r.GRAD_FIELDS:
        assert torch.allclose(leaves[f].grad, tg[f], rtol=1e-5, atol=1e-6 * float(tg[f].abs().max())), f
    # antenna and N0 gradients are summed with shared-memory atomics in FP32: the
    # order, and so the last bits, differ between two runs
    assert torch.allclose(ant.grad, ag, rtol=1e-5, atol=1e-6 * float(ag.abs().max()))
    assert torch.allclose(N0.grad, dn.reshape(()), rtol=1e-5, atol=0)
    p.close()


def test_autograd_function_follows_n0_and_antenna_positions():
    """RadioTraces is a function of every tensor it differentiates: moving one
    antenna by 1 m, or scaling N0 by 1.02 (the differentiable workload's target),
    changes the forward traces to those of a process configured that way."""
    from paper_2309_03717_gb300 import c8r
    w = synth.workload(4, n_tracks=3001, n_ant=8, seed_offset=5)
    w["dtype"] = np.float32
    tracks = to_device(synth.workload_tracks(w))
    args = [tracks[f] for f in synth.FIELDS]
    p = c8r.RadioProcess(w["medium"], w["ant_xyz"], w["t_start_ns"], w["n_bins"], w["dt_ns"], "endpoint", "mixed")
    N0 = torch.tensor(w["medium"]["N0"], dtype=torch.float64, device="cuda")
    ant = torch.tensor(w["ant_xyz"], dtype=torch.float64, device="cuda")
    base = c8r.RadioTraces.apply(p, N0, *args, ant).cpu().numpy()

    def fresh(medium, pos):
        q = c8r.RadioProcess(medium, pos, w["t_start_ns"], w["n_bins"], w["dt_ns"], "endpoint", "mixed")
        q.push(tracks)
        out = q.traces().cpu().numpy()
        q.close()
        return out

    moved = ant.clone()
    moved[3, 0] += 1.0
    got = c8r.RadioTraces.apply(p, N0, *args, moved).cpu().numpy()
    ref = fresh(w["medium"], moved.cpu().numpy())
    assert rel_l2(got[3], base[3]) > 1e-2  # the moved antenna's trace changed
    assert rel_l2(got, ref) < 1e-5
    assert rel_l2(np.delete(got, 3, 0), np.delete(base, 3, 0)) < 1e-5
    med = dict(w["medium"], N0=w["medium"]["N0"] * 1.02)
    got = c8r.RadioTraces.apply(p, N0 * 1.02, *args, ant).cpu().numpy()
    assert rel_l2(got, base) > 1e-2
    assert rel_l2(got, fresh(med, w["ant_xyz"])) < 1e-5
    p.close()


@pytest.mark.parametrize("formalism", ["endpoint", "zhs"])
def test_autograd_matches_central_differences_fp64(formalism):
    """Central differences of a loss through RadioTraces (FP64 path, a tiny
    case) against its backward: N0, every antenna coordinate and a few track
    coordinates.  Tracks with an arrival (or ZHS interval end) within 2e-3 bin of
    an edge are left out, so that no step moves a bin."""
    from paper_2309_03717_gb300 import c8r
    w = synth.workload(4, n_tracks=400, n_ant=3, seed_offset=9)
    w["dtype"] = np.float64
    tracks = synth.workload_tracks(w)
    keep = unambiguous(tracks, w["ant_xyz"], w["t_start_ns"], w["n_bins"], w["dt_ns"], w["medium"], formalism,
                       tol=2e-3)
    tracks = drop_tracks(tracks, keep)
    n = tracks["x0"].size
    assert n > 300
    dev = to_device(tracks)
    p = c8r.RadioProcess(w["medium"], w["ant_xyz"], w["t_start_ns"], w["n_bins"], w["dt_ns"], formalism, "fp64")
    leaves = {f: dev[f].clone().requires_grad_(f != "q") for f in synth.FIELDS}
    ant = torch.tensor(w["ant_xyz"], dtype=torch.float64, device="cuda", requires_grad=True)
    N0 = torch.tensor(w["medium"]["N0"], dtype=torch.float64, device="cuda", requires_grad=True)
    out = c8r.RadioTraces.apply(p, N0, *[leaves[f] for f in synth.FIELDS], ant)
    G = torch.from_numpy(np.random.default_rng(3).normal(size=tuple(out.shape))).cuda()
    scale = 1.0 / float(out.detach().abs().max())
    (out * G).sum().mul(scale).backward()

    def loss(N0v, antv, trk):
        with torch.no_grad():
            o = c8r.RadioTraces.apply(p, N0v, *[trk[f] for f in synth.FIELDS], antv)
            return float((o * G).sum()) * scale

    base = {f: dev[f].clone() for f in synth.FIELDS}
    checks = []
    h = 1e-6 * w["medium"]["N0"]
    fd = (loss(N0.detach() + h, ant.detach(), base) - loss(N0.detach() - h, ant.detach(), base)) / (2 * h)
    checks.append(("N0", fd, float(N0.grad)))
    for a in range(3):
        for c in range(3):
            hp = 2e-5  # m: moves an arrival by ~3e-4 bin
            ap, am = ant.detach().clone(), ant.detach().clone()
            ap[a, c] += hp
            am[a, c] -= hp
            fd = (loss(N0.detach(), ap, base) - loss(N0.detach(), am, base)) / (2 * hp)
            checks.append((f"ant[{a},{c}]", fd, float(ant.grad[a, c])))
    # beta does not move the arrivals: a step of 2e-7 changes D by ~1e-7 of
    # its size (>= 1e-3); tracks with 1 - |beta| > 1e-5 stay below 1 under it
    bmag = np.sqrt(tracks["bx"] ** 2 + tracks["by"] ** 2 + tracks["bz"] ** 2)
    slow = np.flatnonzero(1.0 - bmag > 1e-5)
    for i, ib in zip((0, n // 2, n - 1), (slow[0], slow[len(slow) // 2], slow[-1])):
        for f in ("x0", "z1", "bx"):
            if f == "bx":
                i = ib
            hp = 2e-5 if f != "bx" else 2e-7
            tp = {k: v.clone() for k, v in base.items()}
            tm = {k: v.clone() for k, v in base.items()}
            tp[f][i] += hp
            tm[f][i] -= hp
            fd = (loss(N0.detach(), ant.detach(), tp) - loss(N0.detach(), ant.detach(), tm)) / (2 * hp)
            checks.append((f"{f}[{i}]", fd, float(leaves[f].grad[i])))
    floor = 1e-6 * max(abs(c[2]) for c in checks if c[0].startswith("ant"))
    bad = [c for c in checks if abs(c[1] - c[2]) > 1e-5 * abs(c[2]) + floor]
    assert not bad, bad
    p.close()
