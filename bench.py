#!/usr/bin/env python3
"""Benchmark of the track x antenna radio hot path on GB300.

One step = one pass of the hot path over the 2e7-track shower of the
160-antenna star array (exponential atmosphere, 4096 bins of 0.2 ns): track
ingest + filter, then the Endpoint and the ZHS radio processes (the two
formalisms the paper runs side by side on one shower), mixed precision.  The
headline is track-antenna pairs per second over both formalisms.

Also reported: the FP64 path on the same workload (a sample of it), the adjoint
/ forward time ratio on the differentiable 1e6-track x 64-antenna workload, the
batched persistent launches against separate launches (64 uneven showers at
their stated sizes, and scaled down), the ALU roofline of the dominant kernel, the oracle timed on
the host cores, and GPU clocks during the timed region.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Under torchrun each rank takes its own seeded shower (weak scaling); there is no
collective on the data path, only a barrier and a max over the ranks' times.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")
SM_COUNT = 152
FP32_LANES_PER_SM = 128
# algorithmic FP32-pipe operations per Endpoint pair, counted from the plain
# formula (two endpoints: propagator, Doppler factor, arrival bin, field vector
# and amplitude): 56 arithmetic + 6 special-function operations
ALG_OPS_PER_ENDPOINT_PAIR = 62
# DRAM bytes (read + write) per pair of the Endpoint forward kernel: one ncu
# capture of a 4e6-track x 160-antenna launch (6.4e8 pairs, default launch
# shape, the split arrival form the vertical shower takes) read 407.7 MB and
# wrote 5.3 MB; the traffic is the staged track tiles, so it scales with the
# pairs at a fixed antenna count.  Set to None when the kernel changes.
DRAM_BYTES_PER_ENDPOINT_PAIR = (407675648 + 5301504) / 6.4e8
# The same capture: warp instructions issued per pair and the share of issue
# slots busy (smsp__issue_active).  Set to None when the kernel changes.
ENDPOINT_WARP_INST_PER_PAIR = 6.417611830e9 / 6.4e8
ENDPOINT_ISSUE_ACTIVE_NCU = 0.5998
# Algorithmic work per pair of the other kernels, counted from their plain
# formulas: ZHS one midpoint evaluation (distance, Doppler factor, transverse
# beta, arrival, interval ends, their bins and weights, up to four deposits):
# 48 arithmetic + 6 special-function operations; the Endpoint adjoint (per
# endpoint: the forward geometry and bin, the deposit's chain rule and the
# accumulation into the track, antenna and N0 gradients): 174 + 10.
ALG_OPS_PER_ZHS_PAIR = 54
ALG_OPS_PER_ENDPOINT_ADJOINT_PAIR = 184
# Per pair, from one ncu capture of each kernel (4e6-track shower x 160
# antennas for the forward kernels; the differentiable workload for the
# adjoint): global float4 reductions (lts__t_requests_srcunit_tex_op_red) and
# DRAM bytes (read + write).  None where not captured.
RED_PER_PAIR = {"endpoint": 565344812 / 6.4e8, "zhs": 649034623 / 6.4e8, "adjoint": None}
DRAM_BYTES_PER_PAIR = {"endpoint": DRAM_BYTES_PER_ENDPOINT_PAIR, "zhs": (424902144 + 10217984) / 6.4e8,
                       "adjoint": None}
# algorithmic bytes per track of the whole path: the 48-byte FP32 track record
ALG_BYTES_PER_TRACK = 48.0


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--tracks", type=int, default=None, help="override the track count (testing only)")
    ap.add_argument("--no-extras", action="store_true")
    ap.add_argument("--fp64-only", type=int, default=0, metavar="TRACKS",
                    help="time only the FP64 path on TRACKS tracks of the shower (a small case for profiling)")
    ap.add_argument("--adjoint-only", choices=["endpoint", "zhs"], default=None,
                    help="time only the forward pass and the adjoint of one formalism on the differentiable "
                         "workload (1e6 tracks x 64 antennas; a small case for profiling)")
    ap.add_argument("--cpu-sample-tracks", type=int, default=400000)
    return ap.parse_args()


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""

    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (OSError, ValueError):
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for n, v in zip(names, parts[3:7]):
                if v.lower() in ("active", "1"):
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def peaks():
    try:
        with open(PEAKS_FILE) as f:
            return json.load(f), "measured"
    except (OSError, ValueError):
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


def roofline_bounds(pairs_per_s, ops_per_pair, red_per_pair, dram_per_pair, fp64_ops_per_pair, rates, pk):
    """The bounds of a pair kernel (pairs/s each), the binding one (the lowest)
    and the achieved fraction of it: (i) FP32 issue, the algorithmic FP32-pipe
    operations per pair against 152 SMs x 128 lanes x the maximum SM clock (the
    FFMA probe's rate beside it); (ii) FP64 issue, the FP64 operations per pair
    against the probe's DFMA rate; (iii) global float4 reductions per pair
    against the probe's rate of scattered reductions into an L2-resident buffer;
    (iv) HBM, the DRAM bytes per pair against the measured copy bandwidth."""
    mhz = pk.get("sm_max_mhz", 2070.0)
    lane_peak = SM_COUNT * FP32_LANES_PER_SM * mhz * 1e6
    b = {"fp32_issue": {"pairs_per_s": lane_peak / ops_per_pair, "peak_lane_ops_per_s": lane_peak,
                        "ops_per_pair": ops_per_pair, "probe_ffma_lane_ops_per_s": rates.get("ffma_per_s")}}
    if fp64_ops_per_pair:
        b["fp64_issue"] = {"pairs_per_s": rates["dfma_per_s"] / fp64_ops_per_pair, "ops_per_pair": fp64_ops_per_pair,
                           "probe_dfma_per_s": rates.get("dfma_per_s")}
    else:
        b["fp64_issue"] = {"pairs_per_s": None, "ops_per_pair": 0, "probe_dfma_per_s": rates.get("dfma_per_s"),
                           "note": "no FP64 operation per pair"}
    if red_per_pair and rates.get("global_red_f32x4_per_s"):
        b["global_reductions"] = {"pairs_per_s": rates["global_red_f32x4_per_s"] / red_per_pair,
                                  "per_pair": red_per_pair, "probe_red_f32x4_per_s": rates["global_red_f32x4_per_s"]}
    if dram_per_pair:
        b["hbm"] = {"pairs_per_s": pk.get("hbm_gbs", 6800.0) * 1e9 / dram_per_pair, "bytes_per_pair": dram_per_pair,
                    "peak_gbs": pk.get("hbm_gbs", 6800.0)}
    live = {k: v for k, v in b.items() if v.get("pairs_per_s")}
    binding = min(live, key=lambda k: live[k]["pairs_per_s"])
    return {"bounds": b, "binding": binding, "pairs_per_s": pairs_per_s,
            "frac_of_binding": pairs_per_s / live[binding]["pairs_per_s"]}


def max_over_ranks(x, dist, device):
    """The largest of the ranks' values (timing: the job ends with its slowest
    rank); x itself when not distributed."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank_step, steps, world, seconds):
    """Weak scaling: every rank processes its own units each step, so the job's
    rate is all ranks' units over the slowest rank's time."""
    return units_per_rank_step * steps * world / seconds


def host_tracks(w, n, seed_offset):
    from paper_2309_03717_gb300 import synth
    w = dict(w)
    w["seed"] = w["seed"] + 7919 * seed_offset
    return synth.workload_tracks(w, n)


def to_dev(tracks, torch, pinned=False):
    out = {}
    for k, v in tracks.items():
        t = torch.from_numpy(np.ascontiguousarray(v))
        out[k] = t.pin_memory() if pinned else t.cuda()
    return out


_CPU_TRACKS = None


def _cpu_init(n_tracks, seed, zenith):
    """Worker set-up (untimed): the same seeded track sample in every process."""
    global _CPU_TRACKS
    import oracle
    from paper_2309_03717_gb300 import synth
    _CPU_TRACKS = oracle.tracks_from_ns(synth.make_tracks(n_tracks, seed, zenith, np.float32))


def _cpu_part(job):
    import oracle
    ant, t_start_s, n_bins, dt_s, medium, formalism = job
    oracle.forward(_CPU_TRACKS, ant, t_start_s, n_bins, dt_s, medium, formalism)
    return len(ant)


class OraclePool:
    """The oracle as it stands in one process per host core, each taking a
    contiguous slice of the antennas (the paper's antenna-bunch split).  The
    workers are spawned (never forked) and set up their track sample untimed."""

    def __init__(self, w, n_tracks, formalisms):
        import multiprocessing as mp
        import oracle
        oracle.build()
        self.w, self.n_tracks, self.formalisms = w, n_tracks, formalisms
        A = len(w["ant_xyz"])
        self.P = P = max(1, min(os.cpu_count() or 1, A))
        bounds = np.linspace(0, A, P + 1).astype(int)
        self.jobs = [(np.ascontiguousarray(w["ant_xyz"][bounds[i]:bounds[i + 1]]),
                      w["t_start_ns"][bounds[i]:bounds[i + 1]] * 1e-9, w["n_bins"], w["dt_ns"] * 1e-9, w["medium"],
                      oracle.ENDPOINT if f == "endpoint" else oracle.ZHS)
                     for f in formalisms for i in range(P)]
        self.pool = mp.get_context("spawn").Pool(P, initializer=_cpu_init,
                                                 initargs=(n_tracks, w["seed"] + 17, w["zenith"]))
        self.pool.map(_cpu_part, [(j[0][:1], j[1][:1], 16, j[3], j[4], j[5]) for j in self.jobs[:P]])  # warm-up

    def run(self):
        """One timed pass over the sample: returns (pairs/s, seconds)."""
        t0 = time.perf_counter()
        self.pool.map(_cpu_part, self.jobs, chunksize=1)
        dt = time.perf_counter() - t0
        return self.n_tracks * len(self.w["ant_xyz"]) * len(self.formalisms) / dt, dt

    def describe(self, dt):
        A = len(self.w["ant_xyz"])
        pairs = self.n_tracks * A * len(self.formalisms)
        return (f"{self.n_tracks} tracks x {A} antennas x {len(self.formalisms)} formalisms ({pairs:.3g} pairs, "
                f"{dt:.2f} s wall, FP64 C oracle, {self.P} processes each on 1/{self.P} of the antennas)")

    def close(self):
        self.pool.close()
        self.pool.join()


def cpu_baseline_all_cores(w, n_tracks, formalisms):
    op = OraclePool(w, n_tracks, formalisms)
    try:
        v, dt = op.run()
        return {"value": v, "unit": "pairs/s", "cores": op.P, "kind": "oracle", "sample": op.describe(dt)}
    finally:
        op.close()


def cpu_baseline(w, n_tracks, formalisms):
    """The FP64 oracle as it stands, single-threaded, on a sample of the workload."""
    import oracle
    from paper_2309_03717_gb300 import synth
    tr = synth.make_tracks(n_tracks, w["seed"] + 17, w["zenith"], np.float32)
    trs = oracle.tracks_from_ns(tr)
    pairs = 0
    t0 = time.perf_counter()
    for f in formalisms:
        oracle.forward(trs, w["ant_xyz"], w["t_start_ns"] * 1e-9, w["n_bins"], w["dt_ns"] * 1e-9, w["medium"],
                       oracle.ENDPOINT if f == "endpoint" else oracle.ZHS)
        pairs += n_tracks * len(w["ant_xyz"])
    dt = time.perf_counter() - t0
    return {"value": pairs / dt, "unit": "pairs/s", "cores": 1, "kind": "oracle",
            "sample": f"{n_tracks} tracks x {len(w['ant_xyz'])} antennas x {len(formalisms)} formalisms "
                      f"({pairs:.3g} pairs, {dt:.1f} s, FP64 C oracle, one thread)"}


def run_reference(args):
    """Reference arm: the oracle, timed on all host cores on bounded samples."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    from paper_2309_03717_gb300 import synth
    w = synth.workload(1)
    n = args.cpu_sample_tracks
    op = OraclePool(w, n, ("endpoint", "zhs"))
    try:
        for _ in range(args.warmup):
            op.run()
        vals = []
        t0 = time.perf_counter()
        for _ in range(args.steps):
            vals.append(op.run())
        elapsed = time.perf_counter() - t0
    finally:
        op.close()
    pairs_per_step = 2 * n * len(w["ant_xyz"])
    v = pairs_per_step * args.steps / sum(dt for _, dt in vals)
    line = {
        "impl": "reference", "metric": "track-antenna pairs/sec (Endpoint, ZHS) on 1 GB300; backward/forward time ratio",
        "value": v, "unit": "pairs/s", "n_gpus": 0, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * elapsed / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": "shower 2e7 tracks (sampled), star 8x20 antennas, exp. atmosphere, 4096 x 0.2 ns",
                   "sample_tracks_per_step": n, "pairs_per_step": pairs_per_step},
        "cpu_baseline": {"value": v, "kind": "oracle", "cores": op.P, "sample": op.describe(vals[0][1])},
        "e2e": {"value": v, "unit": "pairs/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
        return
    import torch
    import torch.distributed as dist

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)

    from paper_2309_03717_gb300 import build, c8r, synth
    if rank == 0:
        build.build()
    c8r.load()
    rates = c8r.c8r_measure_peaks(local)  # the units' measured rates (a few ms)
    if args.fp64_only:
        c8r.load()
        print(json.dumps({"fp64_only": fp64_timing(torch, c8r, synth.workload(1), args.fp64_only)}))
        return
    if args.adjoint_only:
        c8r.load()
        w4 = synth.workload(4)
        d4 = {k: torch.from_numpy(v).cuda() for k, v in synth.workload_tracks(w4).items()}
        fwd_ms, bwd_ms = adjoint_timing(torch, c8r, w4, d4, args.adjoint_only)
        print(json.dumps({"adjoint_only": {"formalism": args.adjoint_only, "fwd_ms": fwd_ms, "bwd_ms": bwd_ms,
                                           "bwd_fwd_ratio": bwd_ms / fwd_ms}}))
        return
    if world > 1:
        dist.barrier()
    c8r.load()

    w = synth.workload(1)
    T = args.tracks or w["n_tracks"]
    A = len(w["ant_xyz"])
    tracks_h = host_tracks(w, T, rank)
    dev = to_dev(tracks_h, torch)
    procs = {f: c8r.RadioProcess(w["medium"], w["ant_xyz"], w["t_start_ns"], w["n_bins"], w["dt_ns"], f, "mixed")
             for f in ("endpoint", "zhs")}
    outs = {f: torch.empty((A, 3, w["n_bins"]), dtype=torch.float32, device="cuda") for f in procs}
    stream = torch.cuda.current_stream()

    def step():
        for f, p in procs.items():
            p.reset()
            p.push(dev)
            p.traces(out=outs[f])

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    for _ in range(args.warmup):
        step()
    kept = procs["endpoint"].stats()["tracks_kept"]
    pairs_per_step = 2 * kept * A
    c8r.c8r_profile(procs["endpoint"].ctx, True)
    c8r.c8r_profile(procs["zhs"].ctx, True)
    barrier()
    with ClockSampler(local) as clk:
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.steps):
            step()
        e1.record(stream)
        barrier()
    ms = e0.elapsed_time(e1)
    prof_e = c8r.c8r_profile_read(procs["endpoint"].ctx)
    prof_z = c8r.c8r_profile_read(procs["zhs"].ctx)
    c8r.c8r_profile(procs["endpoint"].ctx, False)
    c8r.c8r_profile(procs["zhs"].ctx, False)
    t_max = max_over_ranks(ms, dist if world > 1 else None, "cuda")
    value = whole_job_rate(pairs_per_step, args.steps, world, t_max * 1e-3)

    # end to end through the public API: pinned host tracks in, host traces out
    pinned = to_dev(tracks_h, torch, pinned=True)
    # the pinned host -> device copy bandwidth of this machine, for reading the end-to-end figure
    probe = torch.empty_like(pinned["x0"], device="cuda")
    probe.copy_(pinned["x0"], non_blocking=True)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(3):
        probe.copy_(pinned["x0"], non_blocking=True)
    e1.record()
    torch.cuda.synchronize()
    h2d_gbs = 3 * probe.numel() * probe.element_size() / (e0.elapsed_time(e1) * 1e-3) / 1e9
    del probe
    host_out = {f: torch.empty((A, 3, w["n_bins"]), dtype=torch.float32).pin_memory() for f in procs}
    h2d = sum(v.numel() * v.element_size() for v in pinned.values())
    d2h = sum(v.numel() * v.element_size() for v in host_out.values())

    # the host->device copy of chunk c+1 (copy stream) overlaps the radio
    # processes' work on chunk c (compute stream); the traces come back at the end.
    # Chunks grow (1/32, 3/32, 1/4, 1/4, 3/8 of the tracks) so that only the
    # small first copy is exposed: a chunk's compute takes several times longer
    # than the copy of the next, larger one.
    bounds = np.unique((T * np.array([0.0, 1 / 32, 1 / 8, 3 / 8, 5 / 8, 1.0])).astype(np.int64))
    n_chunks = len(bounds) - 1
    copy_stream = torch.cuda.Stream()
    dev_buf = {k: torch.empty(v.shape, dtype=v.dtype, device="cuda") for k, v in pinned.items()}

    def step_e2e():
        for p in procs.values():
            p.reset()
        for c in range(n_chunks):
            lo, hi = int(bounds[c]), int(bounds[c + 1])
            with torch.cuda.stream(copy_stream):
                for k, v in pinned.items():
                    dev_buf[k][lo:hi].copy_(v[lo:hi], non_blocking=True)
                ev = torch.cuda.Event()
                ev.record(copy_stream)
            stream.wait_event(ev)
            chunk = {k: v[lo:hi] for k, v in dev_buf.items()}
            for p in procs.values():
                p.push(chunk)
        for f, p in procs.items():
            p.traces(out=host_out[f])

    step_e2e()
    barrier()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        step_e2e()
    barrier()
    e2e_s = time.perf_counter() - t0
    e2e_s = max_over_ranks(e2e_s, dist if world > 1 else None, "cuda")
    e2e_value = whole_job_rate(pairs_per_step, args.steps, world, e2e_s)
    e2e_check = max(float(torch.linalg.vector_norm(host_out[f].cuda() - outs[f]) / torch.linalg.vector_norm(outs[f]))
                    for f in procs)

    # dominant kernel: the Endpoint pair kernel (one launch per chunk)
    pk, pk_src = peaks()
    clocks = clk.summary()
    kernel_ms = prof_e["pair_ms"] / max(prof_e["pair_launches"], 1)
    pairs_per_launch = kept * A / max(prof_e["pair_launches"] / args.steps, 1)
    alg_ops = ALG_OPS_PER_ENDPOINT_PAIR * pairs_per_launch
    achieved = alg_ops / (kernel_ms * 1e-3) / 1e9
    peak_alu = SM_COUNT * FP32_LANES_PER_SM * pk.get("sm_max_mhz", 2070.0) * 1e6 / 1e9
    result = {
        "metric": "track-antenna pairs/sec (Endpoint, ZHS) on 1 GB300; backward/forward time ratio",
        "value": value, "unit": "pairs/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": t_max / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32+ff (mixed)", "data": "synthetic",
        "config": {"workload": f"shower {T:.3g} tracks x star 8x20 antennas, exponential atmosphere, "
                               f"Endpoint + ZHS, 4096 bins x 0.2 ns, mixed precision",
                   "tracks_per_gpu": T, "antennas": A, "n_bins": w["n_bins"], "formalisms": ["endpoint", "zhs"],
                   "l2": "inputs larger than L2 (tracks %.2f GB per GPU)" % (T * 48 / 1e9),
                   "parallelism": f"{world} independent showers (weak)"},
        "e2e": {"value": e2e_value, "unit": "pairs/s", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                "note": f"pinned host tracks copied in {n_chunks} growing chunks on a second stream, overlapping the "
                        f"processes' work on the previous chunk; traces copied back to pinned host memory",
                "traces_vs_device_path_rel_l2": e2e_check, "pinned_h2d_gbs": h2d_gbs},
        "gpu_launches": int(prof_e["pair_launches"] + prof_e["ingest_launches"] + prof_z["pair_launches"]
                            + prof_z["ingest_launches"]),
        "roofline": {"bound": "alu", "kernel": "k_forward<OpsMixed<Endpoint, exponential>>",
                     "achieved": achieved, "peak": peak_alu, "unit": "Gop/s (FP32 lane ops)",
                     "frac": achieved / peak_alu,
                     "traffic": (DRAM_BYTES_PER_ENDPOINT_PAIR * pairs_per_launch
                                 if DRAM_BYTES_PER_ENDPOINT_PAIR and A == 160 else None),
                     "traffic_note": "DRAM bytes per launch: ncu capture of a 4e6-track launch, scaled by pairs",
                     "issue": ({"warp_inst_per_pair_ncu": ENDPOINT_WARP_INST_PER_PAIR,
                                "achieved_warp_inst_per_s": ENDPOINT_WARP_INST_PER_PAIR * pairs_per_launch
                                / (kernel_ms * 1e-3),
                                "peak_warp_inst_per_s": SM_COUNT * 4 * pk.get("sm_max_mhz", 2070.0) * 1e6,
                                "issue_slots_busy_ncu": ENDPOINT_ISSUE_ACTIVE_NCU}
                               if ENDPOINT_WARP_INST_PER_PAIR else None),
                     "peak_source": f"152 SMs x 128 FP32 lanes x {pk.get('sm_max_mhz', 2070.0):.0f} MHz "
                                    f"({pk_src} max SM clock)",
                     "ops_per_pair": ALG_OPS_PER_ENDPOINT_PAIR, "kernel_ms": kernel_ms,
                     "pairs_per_launch": pairs_per_launch,
                     "traffic_over_algorithmic": (DRAM_BYTES_PER_ENDPOINT_PAIR * A / ALG_BYTES_PER_TRACK
                                                  if DRAM_BYTES_PER_ENDPOINT_PAIR and A == 160 else None),
                     **roofline_bounds(pairs_per_launch / (kernel_ms * 1e-3), ALG_OPS_PER_ENDPOINT_PAIR,
                                       RED_PER_PAIR["endpoint"], DRAM_BYTES_PER_PAIR["endpoint"], 0, rates, pk)},
        "roofline_kernels": {
            "k_forward<OpsMixed<ZHS, exponential>>":
                roofline_bounds(kept * A * args.steps / (prof_z["pair_ms"] * 1e-3), ALG_OPS_PER_ZHS_PAIR,
                                RED_PER_PAIR["zhs"], DRAM_BYTES_PER_PAIR["zhs"], 0, rates, pk)},
        "peaks_measured": rates,
        "kernels": {"endpoint_pair_ms_per_step": prof_e["pair_ms"] / args.steps,
                    "zhs_pair_ms_per_step": prof_z["pair_ms"] / args.steps,
                    "ingest_ms_per_step": (prof_e["ingest_ms"] + prof_z["ingest_ms"]) / args.steps,
                    "endpoint_pairs_per_s": kept * A * args.steps / (prof_e["pair_ms"] * 1e-3),
                    "zhs_pairs_per_s": kept * A * args.steps / (prof_z["pair_ms"] * 1e-3)},
        "clocks": clocks,
    }
    for p in procs.values():
        p.close()
    del dev, pinned

    if rank == 0 and world == 1 and not args.no_extras:
        result["extras"] = extras(torch, c8r, synth, w)
        # the metric's second part: adjoint / forward time on the differentiable workload
        result["bwd_fwd_ratio"] = result["extras"]["bwd_fwd_ratio"]
        # the Endpoint adjoint's bounds, from its time per pass (ingest and the
        # gradient's layout included) on the 1e6-track x 64-antenna workload
        result["roofline_kernels"]["k_backward<OpsMixed<Endpoint, exponential>>"] = roofline_bounds(
            6.4e7 / (result["extras"]["diff_bwd_ms"] * 1e-3), ALG_OPS_PER_ENDPOINT_ADJOINT_PAIR,
            RED_PER_PAIR["adjoint"], DRAM_BYTES_PER_PAIR["adjoint"], 0, rates, pk)
        single = cpu_baseline(w, args.cpu_sample_tracks, ("endpoint", "zhs"))
        result["cpu_baseline"] = cpu_baseline_all_cores(w, 5 * args.cpu_sample_tracks // 2, ("endpoint", "zhs"))
        result["cpu_baseline"]["single_core"] = {k: single[k] for k in ("value", "cores", "sample")}
    if rank == 0:
        print(json.dumps(result))
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()


def fp64_timing(torch, c8r, w, n64, reps=2, formalisms=("endpoint", "zhs"), tag="fp64"):
    """The FP64 path on n64 tracks of workload w (drawn on the device by the
    counter-based generator, FP32-exact values passed as FP64), each formalism:
    pairs/s."""
    out = {}
    gen = c8r.c8r_generate_tracks(99, 0, n64, w["zenith"])
    d64 = {k: v.double() for k, v in gen.items()}
    del gen
    A = len(w["ant_xyz"])
    for f in formalisms:
        p = c8r.RadioProcess(w["medium"], w["ant_xyz"], w["t_start_ns"], w["n_bins"], w["dt_ns"], f, "fp64")
        p.push(d64)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            p.push(d64)
        e1.record()
        torch.cuda.synchronize()
        out[f"{tag}_{f}_pairs_per_s"] = reps * n64 * A / (e0.elapsed_time(e1) * 1e-3)
        p.close()
    return out


def extras(torch, c8r, synth, w):
    A = len(w["ant_xyz"])
    # the FP64 path on the whole 2e7-track shower (one timed pass per formalism)
    out = fp64_timing(torch, c8r, w, w["n_tracks"], reps=1)
    out["fp64_workload"] = f"{w['n_tracks']:.3g} tracks x star 8x20, exponential atmosphere, 4096 x 0.2 ns, FP64"
    # the 16-antenna FP64 Endpoint workload: 1e5 tracks, east line 25-400 m, uniform n
    w0 = synth.workload(0)
    out.update(fp64_timing(torch, c8r, w0, w0["n_tracks"], reps=20, formalisms=("endpoint",), tag="line16"))
    out["line16_workload"] = "1e5 tracks x 16-antenna line (25-400 m), uniform n = 1.000292, 4096 x 0.2 ns, FP64 Endpoint"
    # the linear (two-bin) deposit, mixed precision, on 4e6 tracks of the same
    # shower (drawn on the device by the counter-based generator) and array
    n_lin = 4_000_000
    d_lin = c8r.c8r_generate_tracks(98, 0, n_lin, w["zenith"])
    for f in ("endpoint", "zhs"):
        p = c8r.RadioProcess(w["medium"], w["ant_xyz"], w["t_start_ns"], w["n_bins"], w["dt_ns"], f, "mixed",
                             deposit="linear")
        p.push(d_lin)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(3):
            p.push(d_lin)
        e1.record()
        torch.cuda.synchronize()
        out[f"linear_{f}_pairs_per_s"] = 3 * n_lin * A / (e0.elapsed_time(e1) * 1e-3)
        p.close()
    del d_lin
    # adjoint / forward on the differentiable workload (1e6 tracks x 64 antennas,
    # 2048 bins): the Endpoint adjoint the workload names, and the ZHS one
    w4 = synth.workload(4)
    tr4 = synth.workload_tracks(w4)
    d4 = {k: torch.from_numpy(v).cuda() for k, v in tr4.items()}
    for f, tag, dep in (("endpoint", "diff", "bin"), ("zhs", "diff_zhs", "bin"),
                        ("endpoint", "diff_linear", "linear"), ("zhs", "diff_zhs_linear", "linear")):
        fwd_ms, bwd_ms = adjoint_timing(torch, c8r, w4, d4, f, dep)
        out[f"{tag}_fwd_ms"] = fwd_ms
        out[f"{tag}_bwd_ms"] = bwd_ms
        out[f"{tag}_bwd_fwd_ratio"] = bwd_ms / fwd_ms
    out["bwd_fwd_ratio"] = out["diff_bwd_fwd_ratio"]
    out["diff_workload"] = "1e6 tracks x star 8x8, 2048 x 0.2 ns, exponential atmosphere, mixed precision"
    del d4

    # large inclined array: 60 deg shower, 32 x 32 grid (1024 antennas), 8192 x 0.1 ns,
    # tracks streamed through the context in 4e6-track chunks (a sample of 8e6 tracks)
    w2 = synth.workload(2, n_tracks=8_000_000)
    d2 = {k: torch.from_numpy(v).cuda() for k, v in synth.workload_tracks(w2).items()}
    p = c8r.RadioProcess(w2["medium"], w2["ant_xyz"], w2["t_start_ns"], w2["n_bins"], w2["dt_ns"], "endpoint", "mixed")
    p.set_launch_shape(0, 0, w2["chunk"])
    o2 = torch.empty((len(w2["ant_xyz"]), 3, w2["n_bins"]), dtype=torch.float32, device="cuda")

    def step2():
        p.reset()
        p.push(d2)
        p.traces(out=o2)

    step2()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(3):
        step2()
    e1.record()
    torch.cuda.synchronize()
    out["inclined_pairs_per_s"] = 3 * 8_000_000 * len(w2["ant_xyz"]) / (e0.elapsed_time(e1) * 1e-3)
    out["inclined_workload"] = ("8e6 tracks (2 chunks of 4e6) x 32x32 grid, 60 deg, 8192 x 0.1 ns, exponential "
                                "atmosphere, Endpoint mixed")
    p.close()
    # the same with the atmosphere over a spherical Earth (curvature quadrature per pair)
    for f in ("endpoint", "zhs"):
        p = c8r.RadioProcess(synth.AIR_SPHERICAL, w2["ant_xyz"], w2["t_start_ns"], w2["n_bins"], w2["dt_ns"], f,
                             "mixed")
        p.set_launch_shape(0, 0, w2["chunk"])
        step2()
        torch.cuda.synchronize()
        e0.record()
        for _ in range(3):
            step2()
        e1.record()
        torch.cuda.synchronize()
        out[f"inclined_spherical_{f}_pairs_per_s"] = 3 * 8_000_000 * len(w2["ant_xyz"]) / (e0.elapsed_time(e1) * 1e-3)
        p.close()
    # the same with curved rays (a ray solve per emission point and antenna)
    for f in ("endpoint", "zhs"):
        p = c8r.RadioProcess(dict(w2["medium"], kind="exponential_ray"), w2["ant_xyz"], w2["t_start_ns"],
                             w2["n_bins"], w2["dt_ns"], f, "mixed")
        p.set_launch_shape(0, 0, w2["chunk"])
        step2()
        torch.cuda.synchronize()
        e0.record()
        for _ in range(3):
            step2()
        e1.record()
        torch.cuda.synchronize()
        out[f"inclined_ray_{f}_pairs_per_s"] = 3 * 8_000_000 * len(w2["ant_xyz"]) / (e0.elapsed_time(e1) * 1e-3)
        p.close()
    del d2
    # the whole inclined shower: 1e8 tracks generated on the device by the
    # counter-based generator, 4e6 at a time, each chunk pushed as it is made
    n_full, chunk = 100_000_000, w2["chunk"]
    p = c8r.RadioProcess(w2["medium"], w2["ant_xyz"], w2["t_start_ns"], w2["n_bins"], w2["dt_ns"], "endpoint", "mixed")
    p.set_launch_shape(0, 0, chunk)

    def full_pass(n):
        p.reset()
        for first in range(0, n, chunk):
            p.push(c8r.c8r_generate_tracks(2309, first, min(chunk, n - first), 60.0))
        p.traces(out=o2)

    full_pass(chunk)
    torch.cuda.synchronize()
    e0.record()
    full_pass(n_full)
    e1.record()
    torch.cuda.synchronize()
    out["inclined_full_generated_pairs_per_s"] = n_full * len(w2["ant_xyz"]) / (e0.elapsed_time(e1) * 1e-3)
    out["inclined_full_generated_s"] = e0.elapsed_time(e1) * 1e-3
    e0.record()
    for first in range(0, n_full, chunk):
        c8r.c8r_generate_tracks(2309, first, chunk, 60.0)
    e1.record()
    torch.cuda.synchronize()
    out["generate_tracks_per_s"] = n_full / (e0.elapsed_time(e1) * 1e-3)
    out["inclined_full_workload"] = ("1e8 tracks generated on the device in 25 chunks of 4e6 x 32x32 grid, 60 deg, "
                                     "8192 x 0.1 ns, exponential atmosphere, Endpoint mixed")
    p.close()
    del o2

    # batched uneven showers: the graph-captured persistent launches (one per
    # arrival form of the Endpoint evaluation) against one launch per shower (64 showers at their stated track counts, 1e5-1e7 each,
    # drawn on the device by the counter-based generator; and with the track
    # counts scaled by 0.01, where per-launch costs show)
    for scale, tag in ((1.0, "batched"), (0.01, "batched_small")):
        r = batched_vs_separate(torch, c8r, synth, scale)
        out[f"{tag}_pairs_per_s"] = r["batched"]
        out[f"{tag}_separate_launches_pairs_per_s"] = r["separate"]
        out[f"{tag}_workload"] = r["workload"]
    return out


def adjoint_timing(torch, c8r, w4, d4, formalism, deposit="bin"):
    """(forward ms, adjoint ms) per pass; both include their ingest."""
    p = c8r.RadioProcess(w4["medium"], w4["ant_xyz"], w4["t_start_ns"], w4["n_bins"], w4["dt_ns"], formalism, "mixed",
                         deposit=deposit)
    n4 = d4["x0"].numel()
    g = torch.randn((len(w4["ant_xyz"]), 3, w4["n_bins"]), device="cuda")
    tg = {f: torch.zeros(n4, dtype=torch.float32, device="cuda") for f in c8r.GRAD_FIELDS}
    ag = torch.zeros((len(w4["ant_xyz"]), 3), dtype=torch.float64, device="cuda")
    dn = torch.zeros(1, dtype=torch.float64, device="cuda")

    def fwd():
        p.reset()
        p.push(d4)

    def bwd():
        c8r.c8r_backward(p.ctx, d4, g, tg, ag, dn)

    for fn in (fwd, bwd):
        fn()
    torch.cuda.synchronize()
    times = {}
    for name, fn in (("fwd", fwd), ("bwd", bwd)):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(3):
            fn()
        e1.record()
        torch.cuda.synchronize()
        times[name] = e0.elapsed_time(e1) / 3
    p.close()
    return times["fwd"], times["bwd"]


def batched_tracks(torch, c8r, showers):
    """The showers' tracks, each drawn on the device by the counter-based
    generator (seed and zenith of the shower), concatenated in order."""
    total = int(sum(sh["n_tracks"] for sh in showers))
    cat = {f: torch.empty(total, dtype=torch.float32, device="cuda") for f in c8r.TRACK_FIELDS}
    off = 0
    for sh in showers:
        n = int(sh["n_tracks"])
        t = c8r.c8r_generate_tracks(sh["seed"], 0, n, sh["zenith"])
        for f in cat:
            cat[f][off:off + n].copy_(t[f])
        off += n
        del t
    return cat


def batched_vs_separate(torch, c8r, synth, scale):
    showers = synth.batched_workload(64, track_scale=scale)
    cat = batched_tracks(torch, c8r, showers)
    pairs = float(sum(sh["n_tracks"] * len(sh["ant_xyz"]) for sh in showers))
    b = c8r.Batch(showers, synth.AIR_EXPONENTIAL, 4096, 0.2, "endpoint")
    bo = b.new_output()
    for _ in range(2):
        bo.zero_()
        b.run(cat, bo, use_graph=True)
    b.sync()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(3):
        bo.zero_()
        b.run(cat, bo, use_graph=True)
    e1.record()
    b.sync()
    torch.cuda.synchronize()
    t_batch = e0.elapsed_time(e1) / 3
    b.close()
    procs = []
    off = 0
    for sh in showers:
        n = sh["n_tracks"]
        sub = {f: cat[f][off:off + n] for f in synth.FIELDS}
        off += n
        pr = c8r.RadioProcess(synth.AIR_EXPONENTIAL, sh["ant_xyz"], sh["t_start_ns"], 4096, 0.2, "endpoint", "mixed")
        procs.append((pr, sub, torch.empty((len(sh["ant_xyz"]), 3, 4096), dtype=torch.float32, device="cuda")))

    def separate():
        for pr, sub, o in procs:
            pr.reset()
            pr.push(sub)
            pr.traces(out=o)

    separate()
    torch.cuda.synchronize()
    e0.record()
    for _ in range(3):
        separate()
    e1.record()
    torch.cuda.synchronize()
    t_sep = e0.elapsed_time(e1) / 3
    for pr, _, _ in procs:
        pr.close()
    return {"batched": pairs / (t_batch * 1e-3), "separate": pairs / (t_sep * 1e-3),
            "workload": (f"64 showers, {int(sum(sh['n_tracks'] for sh in showers)):.3g} tracks (generated on the "
                         f"device), {pairs:.3g} pairs, antennas 16-512, zenith 0-65 deg, exponential atmosphere, "
                         f"4096 x 0.2 ns, Endpoint mixed")}


if __name__ == "__main__":
    main()
