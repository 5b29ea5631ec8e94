"""The batched persistent launches against separate launches per shower (the
same bins and deposits in either arrival form, so equal up to FP32 addition
order), graph replay, and the cancel word."""
import numpy as np
import pytest

from _util import built_lib, oracle_traces, rel_l2, to_device
from paper_2309_03717_gb300 import synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    built_lib()


def small_batch():
    showers = synth.batched_workload(n_showers=7, seed=11, max_tracks=6000)
    for k, s in enumerate(showers):
        s["n_tracks"] = [300, 5000, 1, 129, 6000, 2048, 777][k]
        s["ant_xyz"] = s["ant_xyz"][: [5, 17, 3, 40, 9, 1, 23][k]]
        s["t_start_ns"] = s["t_start_ns"][: len(s["ant_xyz"])]
    tracks = [synth.make_tracks(s["n_tracks"], s["seed"], s["zenith"]) for s in showers]
    cat = {f: np.concatenate([t[f] for t in tracks]) for f in synth.FIELDS}
    return showers, tracks, cat


@pytest.mark.parametrize("formalism", ["endpoint", "zhs"])
def test_batch_equals_separate_launches(formalism):
    from paper_2309_03717_gb300 import c8r
    showers, tracks, cat = small_batch()
    med = synth.AIR_EXPONENTIAL
    b = c8r.Batch(showers, med, 4096, 0.2, formalism)
    out = b.new_output()
    b.run(to_device(cat), out, use_graph=False)
    b.sync()
    got = out.cpu().numpy()
    off = 0
    for s, t in zip(showers, tracks):
        p = c8r.RadioProcess(med, s["ant_xyz"], s["t_start_ns"], 4096, 0.2, formalism, "mixed")
        p.push(to_device(t))
        ref = p.traces().cpu().numpy()
        p.close()
        A = len(s["ant_xyz"])
        if np.abs(ref).max() > 0:
            assert rel_l2(got[off:off + A], ref) < 2e-6
        else:
            assert not got[off:off + A].any()
        off += A
    # one shower against the oracle as well
    s, t = showers[3], tracks[3]
    ref, _ = oracle_traces(t, s["ant_xyz"], s["t_start_ns"], 4096, 0.2, med, formalism)
    a0 = sum(len(x["ant_xyz"]) for x in showers[:3])
    if np.abs(ref).max() > 0:
        assert rel_l2(got[a0:a0 + len(s["ant_xyz"])], ref) < 1e-4
    b.close()


def test_graph_replay_accumulates_and_cancel_word_stops_work():
    from paper_2309_03717_gb300 import c8r
    showers, tracks, cat = small_batch()
    b = c8r.Batch(showers, synth.AIR_EXPONENTIAL, 4096, 0.2, "endpoint")
    dev = to_device(cat)
    once = b.new_output()
    b.run(dev, once, use_graph=False)
    b.sync()
    twice = b.new_output()
    b.run(dev, twice, use_graph=True)   # captures, then launches
    b.run(dev, twice, use_graph=True)   # replays
    b.sync()
    assert rel_l2(twice.cpu().numpy(), 2 * once.cpu().numpy()) < 2e-6
    b.set_cancel(True)
    cancelled = b.new_output()
    b.run(dev, cancelled, use_graph=False)
    with pytest.raises(c8r.C8RError) as ei:
        b.sync()
    assert ei.value.code == c8r.C8R_ECANCELLED
    assert not cancelled.any()
    b.set_cancel(False)
    again = b.new_output()
    b.run(dev, again, use_graph=False)
    b.sync()
    assert rel_l2(again.cpu().numpy(), once.cpu().numpy()) < 2e-6
    b.close()


def test_full_batched_workload_sampled_against_oracle():
    """The 64 uneven showers at their stated sizes (1e5-1e7 tracks, 16-512
    antennas, zenith 0-65 deg; ~1.4e8 tracks generated on the device, one seed
    per shower), in the graph-captured persistent launches the benchmark times:
    the smallest, the median and the largest shower against the oracle at their
    first, middle and last antenna, over all their tracks (the oracle's tracks
    from the generator's host twin, chunk by chunk in spawned workers).  Tracks
    with an arrival within 1e-6 bin of an edge at a sampled antenna get charge 0
    on both sides."""
    import multiprocessing as mp
    import os

    from _chunk_oracle import chunk_job
    from paper_2309_03717_gb300 import c8r
    showers = synth.batched_workload(64)
    n_tr = np.array([s["n_tracks"] for s in showers])
    order = np.argsort(n_tr)
    picks = [int(order[0]), int(order[len(order) // 2]), int(order[-1])]
    assert n_tr[picks[0]] < 2e5 and n_tr[picks[2]] > 5e6
    off = np.concatenate([[0], np.cumsum(n_tr)[:-1]])
    total = int(n_tr.sum())
    cat = {f: torch.empty(total, dtype=torch.float32, device="cuda") for f in synth.FIELDS}
    for s, sh in enumerate(showers):
        t = c8r.c8r_generate_tracks(sh["seed"], 0, int(sh["n_tracks"]), sh["zenith"])
        for f in synth.FIELDS:
            cat[f][off[s]:off[s] + n_tr[s]].copy_(t[f])
        del t
    chunk = 1_000_000
    jobs, owner = [], []
    for s in picks:
        sh = showers[s]
        A = len(sh["ant_xyz"])
        sample = sorted({0, A // 2, A - 1})
        for first in range(0, int(n_tr[s]), chunk):
            jobs.append((first, min(chunk, int(n_tr[s]) - first), sh["seed"], sh["zenith"],
                         np.ascontiguousarray(sh["ant_xyz"][sample]), np.asarray(sh["t_start_ns"])[sample], 4096, 0.2,
                         sh["medium"], "endpoint"))
            owner.append((s, sample))
    with mp.get_context("spawn").Pool(max(1, min(len(jobs), os.cpu_count() or 1))) as pool:
        results = pool.map(chunk_job, jobs)
    refs = {}
    for (s, sample), (drop, out, _) in zip(owner, results):
        q = cat["q"][off[s]:off[s] + n_tr[s]]
        if drop.size:
            q[torch.from_numpy(drop).cuda()] = 0.0
        refs[s] = (sample, refs[s][1] + out if s in refs else out)
    b = c8r.Batch(showers, synth.AIR_EXPONENTIAL, 4096, 0.2, "endpoint")
    out = b.new_output()
    b.run(cat, out, use_graph=True)
    b.sync()
    got = out.cpu().numpy()
    b.close()
    a_off = np.concatenate([[0], np.cumsum([len(s["ant_xyz"]) for s in showers])[:-1]])
    for s in picks:
        sample, ref = refs[s]
        for j, a in enumerate(sample):
            assert np.abs(ref[j]).max() > 0
            err = rel_l2(got[a_off[s] + a], ref[j])
            assert err <= 1e-4, f"shower {s} ({n_tr[s]} tracks) antenna {a}: relative L2 {err:.3e}"
