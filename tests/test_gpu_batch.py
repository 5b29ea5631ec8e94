"""The batched persistent launch against separate launches per shower (the
same kernels' arithmetic, so equal up to FP32 addition order), graph replay,
and the cancel word."""
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
