"""Parity at full size, in the launch configuration bench.py times.

The 2e7-track shower (exponential atmosphere, 160-antenna star, 4096 x 0.2 ns)
goes through the default launch shape for both formalisms in mixed precision;
the inclined 1024-antenna workload (8192 x 0.1 ns) streams 8e6 tracks in its
4e6-track chunks.  The CUDA path computes every antenna; the oracle, which
cannot, evaluates all tracks for a sample of antennas, one antenna at a time.
Bar: the mixed-precision relative L2 of 1e-4 on each sampled antenna.

As in the smaller parity tests, the tracks with an Endpoint deposit within
1e-6 bin of an edge at a sampled antenna (a few hundred of the 2e7) are left
out of the input: either bin is correct for them, and at this size one of them
moves ~2e-4 of a trace, because a trace is ~1e3 times smaller than the sum of
the magnitudes of its deposits.  The bin test at smaller sizes covers them."""
import numpy as np
import pytest

from _util import built_lib, drop_tracks, edge_ambiguous, oracle_arrivals, oracle_traces, rel_l2, to_device
from paper_2309_03717_gb300 import synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    built_lib()


def sampled_check(w, tracks, formalisms, sample, chunk=0):
    from paper_2309_03717_gb300.c8r import RadioProcess
    amb = np.zeros(len(tracks["x0"]), dtype=bool)
    for a in sample:
        _, u = oracle_arrivals(tracks, w["ant_xyz"][a:a + 1], w["t_start_ns"][a:a + 1], w["n_bins"], w["dt_ns"],
                               w["medium"], "endpoint")
        amb |= edge_ambiguous(u, 1e-6).reshape(len(amb), -1).any(axis=1)
    assert amb.mean() < 1e-4
    tracks = drop_tracks(tracks, ~amb)
    dev = to_device(tracks)
    for formalism in formalisms:
        p = RadioProcess(w["medium"], w["ant_xyz"], w["t_start_ns"], w["n_bins"], w["dt_ns"], formalism, "mixed")
        if chunk:
            p.set_launch_shape(0, 0, chunk)
        p.push(dev)
        got = p.traces().cpu().numpy()
        kept = p.stats()["tracks_kept"]
        p.close()
        for a in sample:
            ref, okept = oracle_traces(tracks, w["ant_xyz"][a:a + 1], w["t_start_ns"][a:a + 1], w["n_bins"],
                                       w["dt_ns"], w["medium"], formalism)
            assert okept == kept
            assert np.abs(ref).max() > 0
            err = rel_l2(got[a:a + 1], ref)
            assert err <= 1e-4, f"{formalism} antenna {a}: relative L2 {err:.3e}"


def test_shower_2e7_tracks_star_160_antennas():
    w = synth.workload(1)
    assert w["n_tracks"] == 20_000_000 and len(w["ant_xyz"]) == 160
    tracks = synth.workload_tracks(w)
    # innermost, a middle radius and the outermost antenna, on different arms
    sample = [0, 8 * 10 + 3, 159]
    sampled_check(w, tracks, ("endpoint", "zhs"), sample)


def test_inclined_1024_antennas_streamed_in_4e6_track_chunks():
    w = synth.workload(2, n_tracks=8_000_000)
    assert len(w["ant_xyz"]) == 1024 and w["n_bins"] == 8192 and w["chunk"] == 4_000_000
    tracks = synth.workload_tracks(w)
    sample = [0, 527, 1023]
    sampled_check(w, tracks, ("endpoint", "zhs"), sample, chunk=w["chunk"])


def test_differentiable_workload_adjoint_full_size():
    """The differentiable workload at its full size (1e6 tracks x 64 antennas,
    2048 x 0.2 ns), forward and Endpoint adjoint in the default launch shape,
    every gradient against the oracle's."""
    import oracle
    from paper_2309_03717_gb300 import c8r
    w = synth.workload(4)
    assert w["n_tracks"] == 1_000_000 and len(w["ant_xyz"]) == 64 and w["n_bins"] == 2048
    tracks = synth.workload_tracks(w)
    _, u = oracle_arrivals(tracks, w["ant_xyz"], w["t_start_ns"], w["n_bins"], w["dt_ns"], w["medium"], "endpoint")
    amb = edge_ambiguous(u, 1e-6).reshape(len(tracks["x0"]), -1).any(axis=1)
    assert amb.mean() < 1e-2
    tracks = drop_tracks(tracks, ~amb)
    args = (w["ant_xyz"], w["t_start_ns"] * 1e-9, w["n_bins"], w["dt_ns"] * 1e-9)
    tgt = synth.perturbed_target_tracks(tracks, 77)
    med2 = dict(w["medium"], N0=w["medium"]["N0"] * 1.02)
    ref, kept = oracle.forward(oracle.tracks_from_ns(tracks), *args, w["medium"], oracle.ENDPOINT)
    diff = ref - oracle.forward(oracle.tracks_from_ns(tgt), *args, med2, oracle.ENDPOINT)[0]
    G = 2.0 * diff / np.abs(diff).max()
    p = c8r.RadioProcess(w["medium"], w["ant_xyz"], w["t_start_ns"], w["n_bins"], w["dt_ns"], "endpoint", "mixed")
    dev = to_device(tracks)
    p.push(dev)
    assert rel_l2(p.traces().cpu().numpy(), ref) <= 1e-4
    assert p.stats()["tracks_kept"] == kept
    n = tracks["x0"].size
    tg = {f: torch.zeros(n, dtype=torch.float32, device="cuda") for f in c8r.GRAD_FIELDS}
    ag = torch.zeros((len(w["ant_xyz"]), 3), dtype=torch.float64, device="cuda")
    dn = torch.zeros(1, dtype=torch.float64, device="cuda")
    c8r.c8r_backward(p.ctx, dev, torch.from_numpy(G.astype(np.float32)).cuda(), tg, ag, dn)
    torch.cuda.synchronize()
    p.close()
    tg_ref, ag_ref, dn_ref = oracle.backward(oracle.tracks_from_ns(tracks), *args, w["medium"],
                                             G.astype(np.float32).astype(np.float64))
    got = np.stack([tg[f].double().cpu().numpy() for f in c8r.GRAD_FIELDS], axis=1)
    assert rel_l2(got[:, 0:6], tg_ref[:, 0:6]) <= 1e-4
    assert rel_l2(got[:, 8:11], tg_ref[:, 8:11]) <= 1e-4
    assert rel_l2(ag.cpu().numpy(), ag_ref) <= 1e-4
    assert abs(dn.item() - dn_ref) <= 1e-4 * abs(dn_ref)


def test_inclined_shower_1e8_tracks_generated_on_the_device():
    """The whole inclined shower as the benchmark runs it: 1e8 tracks drawn on
    the device by the counter-based generator, 4e6 per chunk, each pushed as it
    is made, against the oracle at three antennas (the oracle's tracks come from
    the generator's host twin, chunk by chunk in spawned worker processes)."""
    import multiprocessing as mp
    import os

    from _chunk_oracle import chunk_job
    from paper_2309_03717_gb300 import c8r
    w = synth.workload(2, n_tracks=1000)
    n_full, chunk, seed, zenith = 100_000_000, w["chunk"], 2309, w["zenith"]
    assert zenith == 60.0 and len(w["ant_xyz"]) == 1024
    sample = [0, 527, 1023]
    jobs = [(first, min(chunk, n_full - first), seed, zenith, np.ascontiguousarray(w["ant_xyz"][sample]),
             w["t_start_ns"][sample], w["n_bins"], w["dt_ns"], w["medium"], "endpoint")
            for first in range(0, n_full, chunk)]
    with mp.get_context("spawn").Pool(max(1, min(len(jobs), os.cpu_count() or 1))) as pool:
        results = pool.map(chunk_job, jobs)
    drop = np.concatenate([r[0] for r in results])
    ref = sum(r[1] for r in results)
    okept = sum(r[2] for r in results)
    assert drop.size < 1e-4 * n_full
    p = c8r.RadioProcess(w["medium"], w["ant_xyz"], w["t_start_ns"], w["n_bins"], w["dt_ns"], "endpoint", "mixed")
    p.set_launch_shape(0, 0, chunk)
    drop_dev = torch.from_numpy(drop).cuda()
    for first in range(0, n_full, chunk):
        m = min(chunk, n_full - first)
        tr = c8r.c8r_generate_tracks(seed, first, m, zenith)
        sel = drop_dev[(drop_dev >= first) & (drop_dev < first + m)] - first
        tr["q"][sel] = 0.0
        p.push(tr)
    got = p.traces().cpu().numpy()
    kept = p.stats()["tracks_kept"]
    p.close()
    assert kept == okept
    for j, a in enumerate(sample):
        assert np.abs(ref[j]).max() > 0
        err = rel_l2(got[a], ref[j])
        assert err <= 1e-4, f"antenna {a}: relative L2 {err:.3e}"
