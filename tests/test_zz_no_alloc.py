"""c8r_traces_noalloc: the forward pass for callers that cannot allocate device
memory (it keeps its scratch in fixed-size device arrays instead of a context).
Its output must match the context path's (c8r_push_tracks) within the FP32
addition-order tolerance the other launch-shape tests use, on two calls in a row
that reuse the same scratch.  This file is collected last on purpose."""
import ctypes

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


def noalloc(c8r, tracks_dev, w, formalism, out):
    lib = c8r.load()
    s = c8r.tracks_struct(tracks_dev)
    pos = np.ascontiguousarray(w["ant_xyz"], dtype=np.float64)
    ts = np.ascontiguousarray(w["t_start_ns"], dtype=np.float64)
    med = w["medium"]
    kind = c8r.C8R_EXPONENTIAL if med["kind"] == "exponential" else c8r.C8R_UNIFORM
    a = med["N0"] if kind == c8r.C8R_EXPONENTIAL else med["n"]
    H = med.get("H", 1.0)
    dp = ctypes.POINTER(ctypes.c_double)
    return lib.c8r_traces_noalloc(ctypes.byref(s), tracks_dev["x0"].numel(), len(pos), pos.ctypes.data_as(dp),
                                  ts.ctypes.data_as(dp), w["n_bins"], w["dt_ns"],
                                  c8r.C8R_ENDPOINT if formalism == "endpoint" else c8r.C8R_ZHS, kind, a, H,
                                  ctypes.c_void_p(out.data_ptr()),
                                  ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))


def context_traces(c8r, tracks_dev, w, formalism):
    p = c8r.RadioProcess(w["medium"], w["ant_xyz"], w["t_start_ns"], w["n_bins"], w["dt_ns"], formalism, "mixed")
    p.push(tracks_dev)
    out = p.traces().cpu().numpy()
    p.close()
    return out


@pytest.mark.parametrize("dtype", [np.float32, np.float64])
@pytest.mark.parametrize("formalism", ["endpoint", "zhs"])
def test_noalloc_matches_context_path_on_two_calls(formalism, dtype):
    from paper_2309_03717_gb300 import c8r
    # first call: 70001 tracks (two internal chunks, ragged tail), 40 antennas;
    # second call: fewer tracks and antennas in a uniform medium, so stale
    # scratch from the first call would show.  FP64 input tracks are rounded to
    # FP32 by the ingest of both paths (and read with 8-byte chunk offsets).
    cases = [synth.workload(1, n_tracks=70001, n_ant=40), synth.workload(0, n_tracks=3001, n_ant=9)]
    for w in cases:
        w["dtype"] = np.float32
        tr = to_device(synth.workload_tracks(w))
        if dtype == np.float64:
            tr = {k: v.double() for k, v in tr.items()}
        ref = context_traces(c8r, tr, w, formalism)
        out = torch.zeros((len(w["ant_xyz"]), 3, w["n_bins"]), dtype=torch.float32, device="cuda")
        assert noalloc(c8r, tr, w, formalism, out) == c8r.C8R_OK
        got = out.cpu().numpy()
        assert np.abs(ref).max() > 0
        assert rel_l2(got, ref) < 1e-5


def test_noalloc_rejects_sizes_beyond_its_scratch():
    from paper_2309_03717_gb300 import c8r
    w = synth.workload(1, n_tracks=10, n_ant=1)
    w["ant_xyz"] = np.zeros((1025, 3))
    w["t_start_ns"] = np.zeros(1025)
    tr = to_device(synth.workload_tracks(w))
    out = torch.zeros(1, dtype=torch.float32, device="cuda")
    assert noalloc(c8r, tr, w, "endpoint", out) == c8r.C8R_ETOOBIG
    assert not out.any()
    w = synth.workload(1, n_tracks=10, n_ant=1)
    w["n_bins"] = (1 << 24) + 1
    assert noalloc(c8r, tr, w, "endpoint", out) == c8r.C8R_ETOOBIG
    assert not out.any()


def test_noalloc_without_tracks_is_a_no_op():
    from paper_2309_03717_gb300 import c8r
    w = synth.workload(1, n_tracks=10, n_ant=3)
    w["dtype"] = np.float32
    tr = {k: v[:0] for k, v in to_device(synth.workload_tracks(w)).items()}
    out = torch.zeros((3, 3, w["n_bins"]), dtype=torch.float32, device="cuda")
    assert noalloc(c8r, tr, w, "endpoint", out) == c8r.C8R_OK
    assert not out.any()


def test_noalloc_reports_a_given_up_wait():
    """A kernel that gives up a bounded wait (here made to give up at once by the
    test knob) returns early; the call reports it as C8R_ECANCELLED instead of
    returning incomplete traces as a success, and the next call is whole."""
    from paper_2309_03717_gb300 import c8r
    w = synth.workload(1, n_tracks=4001, n_ant=16)
    w["dtype"] = np.float32
    tr = to_device(synth.workload_tracks(w))
    out = torch.zeros((16, 3, w["n_bins"]), dtype=torch.float32, device="cuda")
    c8r.c8r_set_wait_limit(0)
    try:
        assert noalloc(c8r, tr, w, "endpoint", out) == c8r.C8R_ECANCELLED
    finally:
        c8r.c8r_set_wait_limit(-1)
    out.zero_()
    assert noalloc(c8r, tr, w, "endpoint", out) == c8r.C8R_OK
    ref = context_traces(c8r, tr, w, "endpoint")
    assert rel_l2(out.cpu().numpy(), ref) < 1e-5
