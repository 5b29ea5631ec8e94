"""The benchmark's multi-rank path on CPU: two gloo ranks, each with its own
seeded shower (weak scaling: the showers are independent, so nothing is
exchanged on the data path), the time taken as the maximum over the ranks, and
the job's rate as all ranks' units over that time."""
import socket

import numpy as np
import pytest

import oracle
from paper_2309_03717_gb300 import synth

torch = pytest.importorskip("torch")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_two_gloo_ranks_weak_scaling(tmp_path):
    import torch.multiprocessing as tmp

    from _multirank_worker import rank_main
    import bench
    local = [0.010, 0.030]  # per-rank step times: the job's time is the slower one
    tmp.spawn(rank_main, args=(2, _free_port(), str(tmp_path), local), nprocs=2, join=True)
    r = [np.load(tmp_path / f"rank{k}.npz") for k in range(2)]
    assert float(r[0]["t_max"]) == float(r[1]["t_max"]) == max(local)
    assert not np.array_equal(r[0]["x0"], r[1]["x0"])  # different showers
    units = int(r[0]["kept"]) * 4
    assert int(r[0]["kept"]) == int(r[1]["kept"]) == 300
    assert float(r[0]["value"]) == pytest.approx(2 * units / max(local))
    # each rank's result is its own shower's, as one process computes it
    w = synth.workload(0, n_tracks=300, n_ant=4)
    for k in range(2):
        tr = bench.host_tracks(w, 300, k)
        ref, _ = oracle.forward(oracle.tracks_from_ns(tr), w["ant_xyz"], w["t_start_ns"] * 1e-9, w["n_bins"],
                                w["dt_ns"] * 1e-9, w["medium"], oracle.ENDPOINT)
        assert np.array_equal(r[k]["traces"], ref)


def test_single_process_needs_no_collective():
    import bench
    assert bench.max_over_ranks(0.25, None, "cpu") == 0.25
    assert bench.whole_job_rate(1000, 5, 1, 2.0) == 2500.0
