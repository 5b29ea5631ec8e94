"""Rank body of the two-rank CPU test of the benchmark's multi-process path (a
module of its own so that spawned ranks import it without the GPU stack)."""
import os

import numpy as np


def rank_main(rank, world, port, out_dir, local_seconds):
    import torch.distributed as dist

    import bench
    import oracle
    from paper_2309_03717_gb300 import synth
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        # each rank takes its own seeded shower (weak scaling, no data-path collective)
        w = synth.workload(0, n_tracks=300, n_ant=4)
        tr = bench.host_tracks(w, 300, rank)
        out, kept = oracle.forward(oracle.tracks_from_ns(tr), w["ant_xyz"], w["t_start_ns"] * 1e-9, w["n_bins"],
                                   w["dt_ns"] * 1e-9, w["medium"], oracle.ENDPOINT)
        t_max = bench.max_over_ranks(local_seconds[rank], dist, "cpu")
        value = bench.whole_job_rate(kept * len(w["ant_xyz"]), 1, world, t_max)
        np.savez(os.path.join(out_dir, f"rank{rank}.npz"), x0=tr["x0"], traces=out, kept=kept, t_max=t_max,
                 value=value)
        dist.barrier()
    finally:
        dist.destroy_process_group()
