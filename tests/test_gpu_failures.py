"""Failure detection without a GPU fault: every bounded wait of the kernels can
be made to give up at once (c8r_set_wait_limit(0)), after which the kernels
drain their copies in flight, set their status word and return, and the calls
report C8R_ECANCELLED; and device allocations can be made to fail on the host
(c8r_inject_alloc_failures), after which the calls report C8R_ENOMEM and the
library stays usable.  The paper's only fault mechanism is the thread pool's
stop token (§3); these are the GPU counterparts."""
import numpy as np
import pytest

from _util import built_lib, rel_l2, to_device
from paper_2309_03717_gb300 import synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    built_lib()


@pytest.fixture(autouse=True)
def _knobs_cleared():
    from paper_2309_03717_gb300 import c8r
    c8r.c8r_set_wait_limit(-1)
    c8r.c8r_inject_alloc_failures(0, 0)
    yield
    c8r.c8r_set_wait_limit(-1)
    c8r.c8r_inject_alloc_failures(0, 0)


def small():
    w = synth.workload(1, n_tracks=5003, n_ant=24)
    w["dtype"] = np.float32
    return w, to_device(synth.workload_tracks(w))


def process(w, formalism="endpoint", precision="mixed"):
    from paper_2309_03717_gb300.c8r import RadioProcess
    return RadioProcess(w["medium"], w["ant_xyz"], w["t_start_ns"], w["n_bins"], w["dt_ns"], formalism, precision)


@pytest.mark.parametrize("formalism", ["endpoint", "zhs"])
@pytest.mark.parametrize("precision", ["mixed", "fp64"])
def test_forward_wait_give_up_is_reported_and_recoverable(formalism, precision):
    from paper_2309_03717_gb300 import c8r
    w, tr = small()
    if precision == "fp64":
        tr = {k: v.double() for k, v in tr.items()}
    ref = process(w, formalism, precision)
    ref.push(tr)
    good = ref.traces().cpu().numpy()
    ref.close()
    p = process(w, formalism, precision)
    c8r.c8r_set_wait_limit(0)
    p.push(tr)
    with pytest.raises(c8r.C8RError) as ei:
        p.stats()
    assert ei.value.code == c8r.C8R_ECANCELLED
    torch.cuda.synchronize()  # the context (and the device) stay usable
    c8r.c8r_set_wait_limit(-1)
    p.reset()
    p.push(tr)
    assert p.stats()["tracks_kept"] > 0
    assert rel_l2(p.traces().cpu().numpy(), good) < 1e-5
    p.close()


def test_adjoint_wait_give_up_is_reported():
    from paper_2309_03717_gb300 import c8r
    w, tr = small()
    p = process(w)
    p.push(tr)
    g = torch.ones((len(w["ant_xyz"]), 3, w["n_bins"]), dtype=torch.float32, device="cuda")
    n = tr["x0"].numel()
    tg = {f: torch.zeros(n, dtype=torch.float32, device="cuda") for f in c8r.GRAD_FIELDS}
    ag = torch.zeros((len(w["ant_xyz"]), 3), dtype=torch.float64, device="cuda")
    dn = torch.zeros(1, dtype=torch.float64, device="cuda")
    p.stats()
    c8r.c8r_set_wait_limit(0)
    c8r.c8r_backward(p.ctx, tr, g, tg, ag, dn)
    with pytest.raises(c8r.C8RError) as ei:
        p.stats()
    assert ei.value.code == c8r.C8R_ECANCELLED
    c8r.c8r_set_wait_limit(-1)
    ag.zero_()
    c8r.c8r_backward(p.ctx, tr, g, tg, ag, dn)
    p.stats()
    assert torch.isfinite(ag).all() and ag.abs().sum() > 0
    p.close()


def test_batch_wait_give_up_is_reported():
    from paper_2309_03717_gb300 import c8r
    showers = synth.batched_workload(n_showers=3, seed=7, track_scale=0.002)
    tracks = [synth.make_tracks(s["n_tracks"], s["seed"], s["zenith"]) for s in showers]
    cat = to_device({f: np.concatenate([t[f] for t in tracks]) for f in synth.FIELDS})
    c8r.c8r_set_wait_limit(0)
    b = c8r.Batch(showers, synth.AIR_EXPONENTIAL, 4096, 0.2)
    out = b.new_output()
    b.run(cat, out, use_graph=False)
    with pytest.raises(c8r.C8RError) as ei:
        b.sync()
    assert ei.value.code == c8r.C8R_ECANCELLED
    b.close()
    c8r.c8r_set_wait_limit(-1)
    b = c8r.Batch(showers, synth.AIR_EXPONENTIAL, 4096, 0.2)
    out = b.new_output()
    b.run(cat, out, use_graph=False)
    b.sync()
    assert out.abs().sum() > 0
    b.close()


def test_injected_allocation_failures_leave_the_library_usable():
    import ctypes
    from paper_2309_03717_gb300 import c8r
    lib = c8r.load()
    w, tr = small()
    # context creation
    c8r.c8r_inject_alloc_failures(0, 1)
    h = ctypes.c_void_p()
    assert lib.c8r_create(ctypes.byref(h), 0) == c8r.C8R_ENOMEM and h.value is None
    # antenna state: the first (antenna table) or the second (accumulator) allocation fails
    p = process(w)
    ref_p = process(w)
    ref_p.push(tr)
    good = ref_p.traces().cpu().numpy()
    ref_p.close()
    for skip in (0, 1):
        # a new layout (one antenna fewer), so that the call allocates
        c8r.c8r_inject_alloc_failures(skip, 1)
        with pytest.raises(c8r.C8RError) as ei:
            c8r.c8r_set_antennas(p.ctx, w["ant_xyz"][:-1], w["t_start_ns"][:-1], w["n_bins"], w["dt_ns"],
                                 c8r.C8R_ENDPOINT, c8r.C8R_MIXED)
        assert ei.value.code == c8r.C8R_ENOMEM
        with pytest.raises(c8r.C8RError) as ei:  # unconfigured until the next successful call
            p.push(tr)
        assert ei.value.code == c8r.C8R_ESTATE
    c8r.c8r_set_antennas(p.ctx, w["ant_xyz"], w["t_start_ns"], w["n_bins"], w["dt_ns"], c8r.C8R_ENDPOINT,
                         c8r.C8R_MIXED)
    # the derived-track scratch (first push) and the adjoint's gradient buffer
    c8r.c8r_inject_alloc_failures(0, 1)
    with pytest.raises(c8r.C8RError) as ei:
        p.push(tr)
    assert ei.value.code == c8r.C8R_ENOMEM
    p.push(tr)
    assert rel_l2(p.traces().cpu().numpy(), good) < 1e-5
    n = tr["x0"].numel()
    g = torch.ones((len(w["ant_xyz"]), 3, w["n_bins"]), dtype=torch.float32, device="cuda")
    tg = {f: torch.zeros(n, dtype=torch.float32, device="cuda") for f in c8r.GRAD_FIELDS}
    ag = torch.zeros((len(w["ant_xyz"]), 3), dtype=torch.float64, device="cuda")
    dn = torch.zeros(1, dtype=torch.float64, device="cuda")
    c8r.c8r_inject_alloc_failures(0, 1)
    with pytest.raises(c8r.C8RError) as ei:
        c8r.c8r_backward(p.ctx, tr, g, tg, ag, dn)
    assert ei.value.code == c8r.C8R_ENOMEM
    c8r.c8r_backward(p.ctx, tr, g, tg, ag, dn)
    p.stats()
    assert ag.abs().sum() > 0
    # the host-copy staging buffer
    c8r.c8r_inject_alloc_failures(0, 1)
    host = torch.empty((len(w["ant_xyz"]), 3, w["n_bins"]), dtype=torch.float32)
    with pytest.raises(c8r.C8RError) as ei:
        c8r.c8r_fetch_traces(p.ctx, host)
    assert ei.value.code == c8r.C8R_ENOMEM
    c8r.c8r_fetch_traces(p.ctx, host)
    assert rel_l2(host.numpy(), good) < 1e-5
    p.close()


def test_failed_antenna_allocations_do_not_leak():
    """A failing c8r_set_antennas frees what it allocated before the failure:
    many failures with a large antenna table leave the device's free memory
    unchanged (to allocation granularity)."""
    from paper_2309_03717_gb300 import c8r
    w, _ = small()
    p = process(w)
    n_ant = 200_000  # 19 MB antenna table; the accumulator (second allocation) fails
    pos = np.zeros((n_ant, 3))
    pos[:, 0] = np.arange(n_ant)
    ts = np.zeros(n_ant)
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for _ in range(10):
        c8r.c8r_inject_alloc_failures(1, 1)
        with pytest.raises(c8r.C8RError):
            c8r.c8r_set_antennas(p.ctx, pos, ts, 8, 0.2, c8r.C8R_ENDPOINT, c8r.C8R_MIXED)
    torch.cuda.synchronize()
    free1 = torch.cuda.mem_get_info()[0]
    assert free0 - free1 < 32 << 20, f"{(free0 - free1) / 2**20:.1f} MB lost over 10 failed calls"
    p.close()
