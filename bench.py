#!/usr/bin/env python
"""Benchmark of the EMC hot path: pattern.rotation pairs/s per EMC iteration.

One step = one whole EMC iteration (Algorithm 2.1: expansion, both E-step
passes, M-step update, compression and the final division) over the frames
resident in HBM, through libemc's emc_iteration. Default workload "emc64":
64^3 grid, 64x64 detector with 10% of pixels masked, n=10 rotation sampling
(50100 rotations), 20000 Poisson frames at 1 photon/pixel.

value  = M_rot * M_data / (seconds per iteration), summed over GPUs (replicas)
e2e    = the same metric through the public API with the frames copied from
         pinned host memory and the new model read back every step
roofline (dominant kernel), cpu_baseline (the FP64 oracle on host cores),
clocks sampled during the timed region, per-form results (FP32 SIMT, BF16,
BF16 split) are added to the single JSON line rank 0 prints.

--impl reference times the FP64 CPU oracle (the only other implementation of
the method here) on bounded samples of the same workload.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "pattern·rotation pairs/s per EMC iteration: FP32 vs BF16-split vs learned"
WORKLOAD_TEXT = {
    "emc32": "32^3 grid, 32x32 detector, n=4 -> 3240 rotations, 1000 Poisson frames, "
             "0.5 photons/pixel",
    "emc64": "64^3 grid, 64x64 detector (10% masked), n=10 -> 50100 rotations, 20000 Poisson "
             "frames, 1 photon/pixel",
    "emc128": "128^3 grid, 128x128 detector, n=16 -> 204960 rotations, 100000 Poisson frames, "
              "0.3 photons/pixel",
    "emc160": "160^3 grid, 160x160 detector, n=20 -> 400200 rotations, 200000 Poisson frames, "
              "0.2 photons/pixel, log-normal fluence (sigma 0.3)",
}
DTYPE = {"fp32": "f32", "bf16": "bf16", "bf16_split": "bf16x3", "fp16_split": "f16x2"}
LEARNED_FORMS = ("learned",)
ADAPTIVE_FORMS = ("adaptive",)
GAUSS_FORMS = ("gaussian",)
FLUENCE_FORMS = ("poisson_fluence",)
RECON_FORMS = ("reconstruct", "reconstruct_learned")
SPARSE_K_FORMS = ("sparse_k",)
# other workloads' own configurations (their own seeded data, built once)
SCALE_FORMS = {"emc128_recompute": "emc128", "learned128": "emc128"}


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="bf16_split", choices=list(DTYPE))
    ap.add_argument("--workload", default="emc64", choices=list(WORKLOAD_TEXT))
    ap.add_argument("--n-data", type=int, default=None, help="override the frame count")
    ap.add_argument("--n-quat", type=int, default=None, help="override the rotation sampling n")
    ap.add_argument("--forms",
                    default="fp32,bf16,fp16_split,learned,adaptive,gaussian,poisson_fluence,"
                            "sparse_k,emc128_recompute,learned128",
                    help="other forms to time briefly (comma list, or 'none')")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--learned-iters", type=int, default=30,
                    help="iterations of the learned-vs-dense model comparison (0 to skip)")
    ap.add_argument("--recon-iters", type=int, default=10,
                    help="iterations of the reconstruct form")
    ap.add_argument("--adaptive-iters", type=int, default=12,
                    help="iterations of the adaptive-sampling schedule")
    ap.add_argument("--sigma", type=float, default=1.0,
                    help="sigma of the Gaussian noise model form (photon units)")
    ap.add_argument("--learned-sparse-k", type=int, default=1,
                    help="sparse Maximize reads the frames' non-zero pixel lists (1) or rows (0)")
    ap.add_argument("--n-cand", type=int, default=512, help="candidate rotations per frame")
    ap.add_argument("--recompute", action="store_true",
                    help="two-pass streamed E-step (pass 2 recomputes the scores) instead of "
                         "keeping the pass-1 scores in HBM")
    return ap.parse_args()


# ---------------------------------------------------------------------------
# workload
# ---------------------------------------------------------------------------

def workload(args, device):
    from paper_1409_4256_gb300 import synth
    cfg = dict(synth.WORKLOADS[args.workload])
    if args.n_data:
        cfg["n_data"] = args.n_data
    if args.n_quat:
        cfg["n_quat"] = args.n_quat
    ds = synth.make_dataset(cfg["N"], cfg["D"], cfg["n_data"], cfg["mean_photons"],
                            masked_fraction=cfg["masked_fraction"],
                            fluence_sigma=cfg["fluence_sigma"], device=device)
    return cfg, ds


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.rows = []
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([x.strip() for x in line.split(",")])

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        if not self.rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(r[1]) for r in self.rows if len(r) > 8 and r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in self.rows if len(r) > 8 and r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = set()
        for r in self.rows:
            if len(r) > 8:
                for n, v in zip(names, r[5:9]):
                    if v.strip().lower() == "active":
                        reasons.add(n)
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": sorted(reasons),
                "samples": len(self.rows)}


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
        return d, "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0,
            "sm_max_mhz": 2070.0}, "fallback"


def max_over_ranks(dist, x: float, device) -> float:
    """The largest x over all ranks (x itself without a process group): the
    slowest replica's time is the job's time."""
    if not dist:
        return x
    import torch
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(world: int, pairs_per_rank: int, ms: float) -> float:
    """pairs/s of the whole job: every rank's pairs over the slowest rank's time."""
    return world * pairs_per_rank / (ms * 1e-3)


# ---------------------------------------------------------------------------
# CPU oracle timing (cpu_baseline leg and --impl reference)
# ---------------------------------------------------------------------------

def oracle_sample(cfg, ds, quat, w, n_rot_s, n_data_s):
    """Time one oracle EMC iteration on a bounded sample; returns pairs/s."""
    from oracle import oracle
    oracle.build()
    idx = np.linspace(0, quat.shape[0] - 1, n_rot_s).astype(np.int64)
    q_s, w_s = quat[idx], w[idx] / w[idx].sum()
    K = ds.K[:n_data_s].astype(np.float64)
    grid = ds.model_start.astype(np.float32).astype(np.float64)
    floor = 1e-10 * float(grid.mean())
    t0 = time.perf_counter()
    oracle.iteration(grid, q_s, w_s, ds.q, K, floor)
    dt = time.perf_counter() - t0
    return n_rot_s * n_data_s / dt, dt, oracle.num_threads()


def sample_sizes(cfg, ds, n_rot):
    # about 10-20 s of oracle work on 16 host cores (~1e6 pairs/s at 4096 pixels)
    target_pairs = 1.2e7 * 2732.0 / max(ds.q.shape[0], 1)
    n_data_s = min(ds.K.shape[0], 4000)
    n_rot_s = int(min(n_rot, max(64, target_pairs / n_data_s)))
    return n_rot_s, n_data_s


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    from paper_1409_4256_gb300 import synth
    from oracle import oracle
    cfg, ds = workload(args, "cpu")
    oracle.build()
    quat, w = oracle.quat_generate(cfg["n_quat"])
    n_rot_s, n_data_s = sample_sizes(cfg, ds, quat.shape[0])
    n_rot_s = max(64, n_rot_s // 4)  # each step a quarter of the baseline sample
    for _ in range(args.warmup):
        oracle_sample(cfg, ds, quat, w, max(32, n_rot_s // 8), min(500, n_data_s))
    times = []
    for _ in range(args.steps):
        v, dt, cores = oracle_sample(cfg, ds, quat, w, n_rot_s, n_data_s)
        times.append(dt)
    tot = sum(times)
    value = args.steps * n_rot_s * n_data_s / tot
    sample = (f"{n_rot_s} of {quat.shape[0]} rotations x {n_data_s} of {cfg['n_data']} frames "
              f"per step, one full FP64 oracle iteration each")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "pairs/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * tot / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"{args.workload}: {WORKLOAD_TEXT[args.workload]}",
                       "precision": "fp64 oracle"},
            "cpu_baseline": {"value": value, "unit": "pairs/s", "cores": cores, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": "pairs/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------

def time_form(torch, emc, ctx, grid, steps, warmup, stream, dist=None):
    """Warm up, then time `steps` iterations with CUDA events on `stream`.
    Consecutive iterations of one reconstruction: each output model is the next
    iteration's input (two buffers in turn), from the start model on. The timed
    iterations run without statistics (no host wait inside the loop); the
    phase times come from `steps` more iterations with statistics after it.
    Returns (ms per iteration, phases, kernels, last loglik, the model reached)."""
    a, b = grid.clone(), torch.empty_like(grid)
    phases = {k: 0.0 for k in ("ms_expand", "ms_loglik", "ms_normalize", "ms_update",
                                "ms_compress")}
    kernels = 0
    tiles = [0, 0, 0, 0, 0]  # pass-1 tiles, exact, bound-pruned steps, incremental, hi pairs
    with torch.cuda.stream(stream):
        for _ in range(warmup):
            ctx.iteration(a, b, stats=True, stream=stream)
            a, b = b, a
        stream.synchronize()
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            ctx.iteration(a, b, stats=False, stream=stream)
            a, b = b, a
        e1.record(stream)
        e1.synchronize()
        torch.cuda.synchronize()
        lls = []
        for _ in range(steps):
            _, st = ctx.iteration(a, b, stats=True, stream=stream)
            a, b = b, a
            for k in phases:
                phases[k] += st[k]
            kernels += st["kernels"]
            tiles[0] += st["pass1_tiles"]
            tiles[1] += st["pass1_exact"]
            tiles[2] += st["pass1_pruned"]
            tiles[3] += st["pass1_delta"]
            tiles[4] += st["pass1_bound_pairs"]
            lls.append(st["loglik"])
            if st["device_status"] != 0:
                raise RuntimeError(f"device status {st['device_status']}")
    ms = e0.elapsed_time(e1) / steps
    ph = {k: v / steps for k, v in phases.items()}
    ph["pass1_exact_tile_fraction"] = tiles[1] / tiles[0] if tiles[0] else None
    ph["pass1_bound_pruned_steps"] = tiles[2]
    ph["pass1_incremental_bound_steps"] = tiles[3]
    ph["pass1_hi_bound_pairs_per_step"] = tiles[4] / steps
    return ms, ph, kernels, lls[-1], a


def e2e_timed(torch, ctx, K_host, K_dev, cur, nxt, steps, stream):
    """End to end through the public API: every step copies its frames from
    pinned host memory (emc_set_frames then reads them) and its new model back
    to pinned host memory. The copies run on a second stream into two frame
    buffers and two host buffers in turn, so that step n+1's frames arrive
    while step n computes; each waits only for what it needs (a frame buffer
    once emc_set_frames has consumed it, a model buffer once its iteration has
    written it). One untimed step first; the timed region spans every copy of
    the timed steps. Returns (ms per step, bytes read back per step)."""
    cs = torch.cuda.Stream(device=K_dev.device)
    kbuf = [K_dev, torch.empty_like(K_dev)]
    outh = [torch.empty(cur.shape, dtype=torch.float32).pin_memory() for _ in range(2)]
    with torch.cuda.stream(stream):  # untimed step: the plain sequence
        kbuf[0].copy_(K_host, non_blocking=True)
        ctx.set_frames(kbuf[0], stream=stream)
        ctx.iteration(cur, nxt, stats=False, stream=stream)
        outh[0].copy_(nxt, non_blocking=True)
        cur, nxt = nxt, cur
    stream.synchronize()
    ev = lambda: torch.cuda.Event()  # noqa: E731
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    cs.wait_event(e0)
    h2d, consumed, d2h = [None] * steps, [None] * steps, [None] * steps
    with torch.cuda.stream(cs):
        kbuf[0].copy_(K_host, non_blocking=True)
        h2d[0] = ev()
        h2d[0].record(cs)
    for n in range(steps):
        stream.wait_event(h2d[n])
        ctx.set_frames(kbuf[n % 2], stream=stream)
        consumed[n] = ev()
        consumed[n].record(stream)
        if n + 1 < steps:  # the other buffer was consumed by step n - 1
            if n >= 1:
                cs.wait_event(consumed[n - 1])
            with torch.cuda.stream(cs):
                kbuf[(n + 1) % 2].copy_(K_host, non_blocking=True)
                h2d[n + 1] = ev()
                h2d[n + 1].record(cs)
        if n >= 2:  # this step overwrites the model step n - 2 wrote; read back by now
            stream.wait_event(d2h[n - 2])
        ctx.iteration(cur, nxt, stats=False, stream=stream)
        done = ev()
        done.record(stream)
        cs.wait_event(done)
        with torch.cuda.stream(cs):
            outh[n % 2].copy_(nxt, non_blocking=True)
            d2h[n] = ev()
            d2h[n].record(cs)
        cur, nxt = nxt, cur
    stream.wait_event(d2h[steps - 1])
    e1.record(stream)
    e1.synchronize()
    return e0.elapsed_time(e1) / steps, int(outh[0].numel() * 4)


def rot_chunk_for(n_rot: int, n_data: int, cap: float = 8e9) -> int:
    """Rotations per pass-2 chunk keeping the P chunk (2 x 2 B per pair) below
    `cap` bytes; 0 (one chunk) when everything fits."""
    ld_data = -(-n_data // 256) * 256
    rows = -(-n_rot // 128) * 128
    if 4.0 * ld_data * rows <= cap:
        return 0
    return max(128, int(cap // (4 * ld_data)) // 128 * 128)


def learned_form(torch, emc, args, cfg, ds, quat, w, grid, K_dev, stream, dist, world,
                 iters=None, max_cycles=None):
    """Learned proposal + sparse Maximize with a dense fallback every 5th
    iteration. Untimed set-up: 2 dense iterations from the start model give the
    soft targets (top 32 per frame), the MLP trains on 90% of the frames. Each
    frame's candidate set is the top R = 32 rotations of the last dense E-step
    followed by the network's best rotations not among them (M in all); every
    dense fallback refreshes the dense part. Reported separately: the mass the
    network's own top M captures on held-out and training frames, and the same
    schedule with the network's part of each set replaced by random rotations,
    or with the whole set taken from the dense E-step's top M (the schedule
    without the network), each against the dense iterations."""
    from paper_1409_4256_gb300 import learned
    n_rot, n_data = quat.shape[0], ds.K.shape[0]
    M = min(args.n_cand, n_rot)
    R = min(32, M)
    iters = args.learned_iters if iters is None else iters
    floor = 1e-10 * float(ds.model_start.mean())
    ctx = emc.Context(cfg["N"], ds.q, quat, w, n_data, precision="bf16_split", w_floor=floor,
                      store_scores=True, n_cand=M, device=str(grid.device), stream=stream,
                      rot_chunk=rot_chunk_for(n_rot, n_data), sparse_k=args.learned_sparse_k)
    ctx.set_frames(K_dev, stream=stream)
    ctx.collect(min(256, n_rot))  # the dense steps' non-zero P: the missed mass summed directly

    def refresh_net(net):
        # candidates = top R of the last dense E-step + the network's best others
        ti, _ = ctx.targets_from_scores(R, stream=stream)
        ctx.set_candidates(emc.merge_candidates(ti, net, M, stream=stream), stream=stream)

    # the network's part replaced by random rotations (distinct per frame: a
    # seeded frame offset plus M fixed distinct offsets, modulo n_rot)
    rng = np.random.default_rng(1008)
    offs = np.sort(rng.choice(n_rot, M, replace=False))
    rand = torch.as_tensor(((rng.integers(0, n_rot, size=n_data)[:, None] + offs[None, :]) %
                            n_rot).astype(np.int32), device=grid.device)

    def refresh_random():
        ti, _ = ctx.targets_from_scores(R, stream=stream)
        ctx.set_candidates(emc.merge_candidates(ti, rand, M, stream=stream), stream=stream)

    # the dense E-step's own top M (no network): its responsibilities, top M per frame
    frames = torch.arange(n_data, dtype=torch.int32, device=grid.device)
    dense_cand = torch.empty((n_data, M), dtype=torch.int32, device=grid.device)
    fb = max(1, min(n_data, int(4e9 // (4 * n_rot))))

    def refresh_dense_top():
        for f0 in range(0, n_data, fb):
            b = min(fb, n_data - f0)
            Pf = ctx.responsibilities(frames[f0:f0 + b], stream=stream)
            emc.topm(Pf, b, n_rot, n_rot, M, dense_cand[f0:f0 + b], stream=stream)
        ctx.set_candidates(dense_cand, stream=stream)

    with torch.cuda.stream(stream):
        t0 = time.perf_counter()
        g1, _ = ctx.iteration(grid, stream=stream)
        g2, _ = ctx.iteration(g1, stream=stream)
        tidx, tprob = ctx.targets_from_scores(32, stream=stream)
        feat = ctx.features(stream=stream)
        train, test = learned.split_rows(n_data)
        prop = learned.Proposal(n_rot, device=str(grid.device))
        hist = prop.train(feat, tidx, tprob, train, epochs=8, batch=512, lr=1e-3, stream=stream)
        net = prop.propose(feat, M, n_data, stream=stream)
        # recall at the current model: the network's own sets, then the merged ones
        ctx.set_candidates(net, stream=stream)
        ctx.iteration(g2, stream=stream)  # dense E-step on the current model
        mm_net = ctx.missed_mass(stream=stream).cpu().numpy()
        refresh_net(net)
        mm = ctx.missed_mass(stream=stream).cpu().numpy()
        stream.synchronize()
        setup_s = time.perf_counter() - t0
        # timed: cycles of 4 sparse iterations, 1 dense fallback and the refresh
        out = torch.empty_like(grid)
        for _ in range(2):
            ctx.sparse_iteration(g2, out, stats=False, stream=stream)
        stream.synchronize()
        if dist:
            dist.barrier()
        cycles = max(1, args.steps // 5 + 1)
        if max_cycles:
            cycles = min(cycles, max_cycles)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(cycles):
            for _ in range(4):
                ctx.sparse_iteration(g2, out, stats=False, stream=stream)
            ctx.iteration(g2, out, stats=False, stream=stream)
            refresh_net(net)
        e1.record(stream)
        e1.synchronize()
        ms = e0.elapsed_time(e1) / (5 * cycles)
        e0.record(stream)
        for _ in range(5):
            ctx.sparse_iteration(g2, out, stats=False, stream=stream)
        e1.record(stream)
        e1.synchronize()
        ms_sparse = e0.elapsed_time(e1) / 5
    res = {"value": world * n_rot * n_data / (ms * 1e-3), "ms_per_step": ms,
           "ms_sparse_iteration": ms_sparse,
           "evaluated_pairs_per_s": world * M * n_data / (ms_sparse * 1e-3),
           "candidates": M, "dense_top_kept": R, "frames_as_nonzero_lists": bool(args.learned_sparse_k),
           "schedule": "4 sparse + 1 dense per 5 iterations; candidates = dense top 32 + "
                       "network's best others, refreshed at every dense step",
           "train_loss_first_last": [hist[0], hist[-1]],
           "network_heldout_captured_mass": float(1.0 - mm_net[test].mean()),
           "network_train_captured_mass": float(1.0 - mm_net[train].mean()),
           "random_sets_captured_mass_expected": M / n_rot,
           "merged_heldout_captured_mass": float(1.0 - mm[test].mean()),
           "merged_train_captured_mass": float(1.0 - mm[train].mean()), "setup_s": setup_s}
    if iters > 0:
        # model after `iters` iterations, each candidate schedule vs dense, same start
        dense_ctx = emc.Context(cfg["N"], ds.q, quat, w, n_data, precision="bf16_split",
                                w_floor=floor, store_scores=False, device=str(grid.device),
                                stream=stream, rot_chunk=rot_chunk_for(n_rot, n_data))
        dense_ctx.set_frames(K_dev, stream=stream)
        truth = torch.as_tensor(ds.model_true, device=grid.device)
        with torch.cuda.stream(stream):
            a, b = g2.clone(), torch.empty_like(g2)
            for _ in range(iters):
                dense_ctx.iteration(a, b, stats=False, stream=stream)
                a, b = b, a
            stream.synchronize()
        del dense_ctx
        ref = a.double()

        def rel(x, y):
            return float(torch.linalg.norm(x - y) / torch.linalg.norm(y))

        variants = {"network": lambda: refresh_net(net), "random_filler": refresh_random,
                    "dense_top_m": refresh_dense_top}
        res["schedules_vs_dense"] = {}
        for name, refresh in variants.items():
            with torch.cuda.stream(stream):
                ctx.iteration(g2, stream=stream)  # each schedule starts from a dense E-step's sets
                refresh()
                c, d = g2.clone(), torch.empty_like(g2)
                missed, direct = [], []
                t1 = time.perf_counter()
                for it in range(iters):
                    if it % 5 == 4:
                        ctx.iteration(c, d, stats=False, stream=stream)
                        missed.append(float(ctx.missed_mass(stream=stream).mean().item()))
                        _, _, mmd = ctx.collected_targets(32, missed=True, stream=stream)
                        direct.append(float(mmd.mean().item()))
                        refresh()
                    else:
                        ctx.sparse_iteration(c, d, stats=False, stream=stream)
                    c, d = d, c
                stream.synchronize()
                wall = time.perf_counter() - t1
            if ctx.status() != 0:
                raise RuntimeError("device status set in the learned schedule")
            res["schedules_vs_dense"][name] = {
                "rel_model_diff_vs_dense": rel(c.double(), ref),
                "rel_model_err_vs_truth": rel(c.double(), truth),
                # 1 - sum over the set in FP32 (its floor is FP32 rounding), and the
                # recorded P outside the set summed directly
                "mean_missed_mass_at_dense_steps": missed,
                "mean_missed_mass_direct_at_dense_steps": direct, "wall_s": wall}
        res["iters_compared"] = iters
        res["rel_model_err_vs_truth_dense"] = rel(ref, truth)
        nv = res["schedules_vs_dense"]["network"]
        res["rel_model_diff_vs_dense"] = nv["rel_model_diff_vs_dense"]
        res["mean_missed_mass_at_dense_steps"] = nv["mean_missed_mass_at_dense_steps"]
        res["mean_missed_mass_direct_at_dense_steps"] = nv["mean_missed_mass_direct_at_dense_steps"]
    del ctx
    return res


def truth_error(torch, N, ds, dev):
    """The model's relative L2 error against the true intensity over the voxels
    the detector's q-range reaches, after a least-squares scale (the fluence
    model fixes the model only up to one)."""
    ax = torch.arange(N, device=dev, dtype=torch.float64) - N // 2
    r2 = ax[:, None, None] ** 2 + ax[None, :, None] ** 2 + ax[None, None, :] ** 2
    inside = r2 <= (N / 2 - 1) ** 2
    truth = torch.as_tensor(ds.model_true, device=dev)[inside]

    def err(g):
        x = g.double()[inside]
        sc = float((x * truth).sum() / (x * x).sum())
        return float(torch.linalg.norm(sc * x - truth) / torch.linalg.norm(truth))
    return err


def reconstruct_form(torch, args, cfg, ds, grid, stream, make_ctx, n_rot):
    """Consecutive iterations from the start model in the workload's noise model
    (the Poisson-fluence model where frames carry a random fluence): time per
    iteration and the model's relative L2 error against the true intensity over
    the voxels the detector's q-range reaches, after a least-squares scale (the
    fluence model fixes the model only up to one)."""
    model = "poisson_fluence" if cfg.get("fluence_sigma", 0.0) > 0 else "poisson"
    prec = args.precision if args.precision in ("bf16_split", "fp16_split") else "bf16_split"
    ctx = make_ctx(prec, model=model)
    err = truth_error(torch, cfg["N"], ds, grid.device)

    errs, ms, tiles, phases = [err(grid)], [], [], []
    a, b = grid.clone(), torch.empty_like(grid)
    with torch.cuda.stream(stream):
        for _ in range(args.recon_iters):
            _, st = ctx.iteration(a, b, stats=True, stream=stream)
            if st["device_status"] != 0:
                raise RuntimeError(f"device status {st['device_status']}")
            ms.append(st["ms_total"])
            tiles.append(st["pass1_exact"] / st["pass1_tiles"])
            phases.append({k: round(st[k], 2) for k in ("ms_expand", "ms_loglik", "ms_normalize",
                                                        "ms_update", "ms_compress")} |
                          {"bound_pairs": st["pass1_bound_pairs"],
                           "incremental_bound": st["pass1_delta"]})
            errs.append(err(b))
            a, b = b, a
    del ctx
    # pairs/s over the iterations after the first (which has no frame order yet
    # and runs the dense pass 1)
    later = ms[1:] if len(ms) > 1 else ms
    return {"model": model, "precision": prec, "iterations": args.recon_iters,
            "ms_per_iteration": ms, "pass1_exact_tile_fraction": tiles, "phases_ms": phases,
            "rel_err_vs_truth_after_scale_fit": errs,
            "value": n_rot * ds.K.shape[0] / (sum(later) / len(later) * 1e-3)}


def reconstruct_learned_form(torch, emc, args, cfg, ds, quat, w, grid, K_dev, stream, n_rot,
                             iters=30):
    """The learned schedule as a reconstruction in the workload's noise model:
    `iters` iterations from the start model, the first two dense (their
    recorded responsibilities give the network's soft targets, top 32 per
    frame, and it trains on 90% of the frames), then cycles of 4 sparse
    iterations over the candidate sets and a dense fallback, which measures the
    sets' missed mass and refreshes them (dense top 32 + the network's best
    others). The dense iterations record their non-zero responsibilities, so no
    scores are stored (pass 2 recomputes them where they do not fit). Reported
    per iteration: time and the model's error against the true intensity after a
    scale fit; beside it the same number of dense iterations from the same start."""
    from paper_1409_4256_gb300 import learned
    model = "poisson_fluence" if cfg.get("fluence_sigma", 0.0) > 0 else "poisson"
    n_data = ds.K.shape[0]
    M, R = min(args.n_cand, n_rot), 32
    floor = 1e-10 * float(ds.model_start.mean())
    wide = bool(ds.K.max() > 256)
    dev = grid.device

    def make(n_cand):
        c = emc.Context(cfg["N"], ds.q, quat, w, n_data, precision="bf16_split", w_floor=floor,
                        store_scores=not args.recompute, model=model, n_cand=n_cand,
                        device=str(dev), stream=stream, rot_chunk=rot_chunk_for(n_rot, n_data),
                        wide_counts=wide, sparse_k=bool(args.learned_sparse_k and n_cand))
        c.set_frames(K_dev, stream=stream)
        return c

    err = truth_error(torch, cfg["N"], ds, dev)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]

    def timed(fn, *a):
        ev[0].record(stream)
        fn(*a, stats=False, stream=stream)
        ev[1].record(stream)
        ev[1].synchronize()
        return ev[0].elapsed_time(ev[1])

    ctx = make(M)
    ctx.collect(256)  # entries per frame: the rotations with a non-zero P, a few at most
    kinds, ms, errs, missed = [], [], [err(grid)], []
    bufs = [grid.clone(), torch.empty_like(grid)]
    with torch.cuda.stream(stream):
        for it in range(2):
            ms.append(timed(ctx.iteration, bufs[0], bufs[1]))
            kinds.append("dense")
            bufs.reverse()
            errs.append(err(bufs[0]))
        t0 = time.perf_counter()
        tidx, tprob = ctx.collected_targets(R, stream=stream)
        feat = ctx.features(stream=stream)
        train, _ = learned.split_rows(n_data)
        prop = learned.Proposal(n_rot, device=str(dev))
        hist = prop.train(feat, tidx, tprob, train, epochs=8, batch=512, lr=1e-3, stream=stream)
        net = prop.propose(feat, M, n_data, stream=stream)
        ctx.set_candidates(emc.merge_candidates(tidx, net, M, stream=stream), stream=stream)
        stream.synchronize()
        setup_s = time.perf_counter() - t0
        for it in range(2, iters):
            if it % 5 == 4:
                ms.append(timed(ctx.iteration, bufs[0], bufs[1]))
                kinds.append("dense")
                ti, _, mm = ctx.collected_targets(R, missed=True, stream=stream)
                missed.append(float(mm.mean().item()))
                ctx.set_candidates(emc.merge_candidates(ti, net, M, stream=stream),
                                   stream=stream)
            else:
                ms.append(timed(ctx.sparse_iteration, bufs[0], bufs[1]))
                kinds.append("sparse")
            bufs.reverse()
            errs.append(err(bufs[0]))
        if ctx.status() != 0:
            raise RuntimeError("device status set in the learned reconstruction")
        learned_grid = bufs[0].clone()
    del ctx, prop
    torch.cuda.empty_cache()
    dctx = make(0)
    dms, derrs = [], [err(grid)]
    bufs = [grid.clone(), torch.empty_like(grid)]
    with torch.cuda.stream(stream):
        for it in range(iters):
            dms.append(timed(dctx.iteration, bufs[0], bufs[1]))
            bufs.reverse()
            derrs.append(err(bufs[0]))
    diff = float(torch.linalg.norm(learned_grid.double() - bufs[0].double()) /
                 torch.linalg.norm(bufs[0].double()))
    del dctx
    sched = ms[2:]
    return {"model": model, "iterations": iters, "candidates": M, "dense_top_kept": R,
            "schedule": "2 dense (targets), then 4 sparse + 1 dense per 5 iterations; "
                        "candidates = dense top 32 + the network's best others",
            "ms_per_iteration": [round(x, 2) for x in ms], "kinds": kinds,
            "rel_err_vs_truth_after_scale_fit": errs,
            "mean_missed_mass_at_dense_steps": missed,
            "train_loss_first_last": [hist[0], hist[-1]], "setup_s": setup_s,
            "value": n_rot * n_data / (sum(sched) / len(sched) * 1e-3),
            "dense_schedule": {"ms_per_iteration": [round(x, 2) for x in dms],
                               "rel_err_vs_truth_after_scale_fit": derrs,
                               "value": n_rot * n_data / (sum(dms[2:]) / len(dms[2:]) * 1e-3)},
            "rel_model_diff_learned_vs_dense": diff}


def sparse_k_form(torch, emc, cfg, ds, quat, w, grid, K_dev, stream, tensor_pass1_ms):
    """E-step pass 1 gathered over each frame's non-zero pixels (FP32 log W),
    timed beside the same pass as a dense FP32 SIMT contraction and the
    tensor-core pass of the headline form."""
    n_rot, n_data = quat.shape[0], ds.K.shape[0]
    floor = 1e-10 * float(ds.model_start.mean())
    ctx = emc.Context(cfg["N"], ds.q, quat, w, n_data, precision="fp32", w_floor=floor,
                      sparse_k=True, device=str(grid.device), stream=stream)
    ctx.set_frames(K_dev, stream=stream)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
    with torch.cuda.stream(stream):
        L, bias = ctx.expand(grid, 0, n_rot, stream=stream)
        m, s_ = ctx.loglik_sparse_k(L, bias, n_rot, stream=stream)  # warm-up
        ev[0].record(stream)
        for _ in range(2):
            ctx.loglik_sparse_k(L, bias, n_rot, m, s_, stream=stream)
        ev[1].record(stream)
        md, sd = ctx.loglik(L, bias, n_rot, stream=stream)
        ev[2].record(stream)
        ctx.loglik(L, bias, n_rot, md, sd, stream=stream)
        ev[3].record(stream)
        ev[3].synchronize()
    if ctx.status() != 0:
        raise RuntimeError("device status set by the sparse-K pass")
    ms = ev[0].elapsed_time(ev[1]) / 2
    ms_dense = ev[2].elapsed_time(ev[3])
    lse_diff = float((m + torch.log(s_) - md - torch.log(sd))[:n_data].abs().max())
    nz = float(np.count_nonzero(ds.K)) / ds.K.size
    res = {"ms_pass1": ms, "pairs_per_s": n_rot * n_data / (ms * 1e-3),
           "nonzero_fraction": nz, "fp32_dense_pass1_ms": ms_dense,
           "tensor_pass1_ms": tensor_pass1_ms, "max_lse_diff_vs_dense_fp32": lse_diff,
           # cost scales with the non-zero count: the density where it would match the
           # tensor-core pass on this geometry
           "break_even_nonzero_fraction": nz * tensor_pass1_ms / ms}
    del ctx, L, bias
    return res


def adaptive_form(torch, args, cfg, ds, grid, K_dev, stream, ctx, fixed_ms):
    """Adaptive rotation sampling (Sec. 3.4, Eq. 3.1) from the start model:
    d rises from n_quat - 5 to n_quat as the likelihood settles. Reports every
    level's iterations and device time, against the same number of iterations
    at the final d (fixed_ms each), and the likelihoods both schedules reach."""
    from paper_1409_4256_gb300 import adaptive
    d_max = cfg["n_quat"]
    d0 = max(1, d_max - 5)
    iters = args.adaptive_iters
    floor = 1e-10 * float(ds.model_start.mean())
    t0 = time.perf_counter()
    g, hist = adaptive.run(cfg["N"], ds.q, K_dev, grid, d0, d_max, iters, precision=args.precision,
                           w_floor=floor, store_scores=not args.recompute, device=str(grid.device),
                           K_host=ds.K, stream=stream)
    wall = time.perf_counter() - t0
    levels = {}
    for h in hist:
        lv = levels.setdefault(h.d, {"d": h.d, "rotations": h.n_rot, "iterations": 0, "ms": 0.0})
        lv["iterations"] += 1
        lv["ms"] += h.ms
    for lv in levels.values():
        lv["pairs_per_s"] = lv["rotations"] * ds.K.shape[0] * lv["iterations"] / (lv["ms"] * 1e-3)
    # the same number of iterations at the final d (the benchmark's context)
    const = adaptive.log_factorial_sum(ds.K)
    fixed_ll = []
    with torch.cuda.stream(stream):
        a, b = grid.clone(), torch.empty_like(grid)
        for _ in range(iters):
            _, st = ctx.iteration(a, b, stream=stream)
            fixed_ll.append(st["loglik"] - const)
            a, b = b, a
    return {"schedule": f"d {d0} -> {d_max}, refine when |dL| <= 0.01 |L|", "iterations": iters,
            "levels": list(levels.values()), "device_ms_total": sum(h.ms for h in hist),
            "fixed_d_ms_total": iters * fixed_ms, "wall_s_with_setup": wall,
            "loglik_per_iteration": [h.loglik for h in hist], "reached_d": hist[-1].d,
            "fixed_d_loglik_per_iteration": fixed_ll}


# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) per launch of the
# steady iterations, from the one-pass ncu launch-list capture of this exact
# configuration (emc64, BF16 split, 20000 frames, stored scores; the full-size
# workload; its summary is kept with the other profiles)
MEASURED_TRAFFIC_EMC64 = {
    # pass 1 of a steady pruned iteration: the increments' product, the
    # hi-plane bound over the few listed pairs and the exact pass over the
    # live tiles; dense: the single three-plane launch of the first iteration
    "pass1_pruned": 0.331e9 + 0.0002e9 + 2.02e9,
    "pass1_dense": 6.650e9 + 4.247e9,
    "compress": 0.325e9,
    "expand": 1.668e9,
}


def traffic_for(workload, precision, n_rot, n_data, recompute, phases, kernel="pass1"):
    """DRAM bytes per launch (pass 1: per iteration) of one phase's kernels from
    the ncu capture of this exact configuration; None where no capture of the
    configuration exists."""
    if not (workload == "emc64" and precision == "bf16_split" and n_data == 20000
            and n_rot == 50100 and not recompute):
        return None
    if kernel == "pass1":
        pruned = bool(phases.get("pass1_bound_pruned_steps"))
        return MEASURED_TRAFFIC_EMC64["pass1_pruned" if pruned else "pass1_dense"]
    return MEASURED_TRAFFIC_EMC64.get(kernel)


def pass1_roofline(precision, n_pix, n_rot, n_data, phases, traffic):
    """Roofline line of E-step pass 1, the dominant step: algorithmic FLOPs
    (2 n_pix per pair over every pair) over its CUDA-event time per iteration."""
    pk, pk_src = peaks()
    dom_ms = phases["ms_loglik"]
    flops = 2.0 * n_pix * n_rot * n_data  # score contraction sum_i K_ik log W_ij
    if precision == "fp32":
        peak = 152 * 128 * 2 * pk.get("sm_max_mhz", 2070.0) * 1e6 / 1e12
        roof = {"bound": "alu", "peak_source": "derived: 152 SM x 128 FP32 lanes x 2 x max clock"}
    else:
        peak = pk["bf16_tflops_sustained"]
        roof = {"bound": "tensor", "peak_source": f"{pk_src} bf16 sustained"}
    achieved = flops / (dom_ms * 1e-3) / 1e12
    planes = 3 if precision == "bf16_split" else 2 if precision == "fp16_split" else 1
    pruned = bool(phases.get("pass1_bound_pruned_steps"))
    exact = phases.get("pass1_exact_tile_fraction")
    # executed tensor work: every plane over every tile; or (pruned) every plane
    # over the tiles left live, the hi plane over the pairs of row tiles the
    # hi-plane bound covered (256 x 256 per pair and frame tile), and the
    # incremental bound's product (3 rows per row tile, 1/128 of the hi plane)
    if pruned:
        steps = max(1, phases.get("pass1_bound_pruned_steps", 1))
        inc = phases.get("pass1_incremental_bound_steps", 0) / steps
        hi_pairs = phases.get("pass1_hi_bound_pairs_per_step", 0.0)
        executed = (flops * planes * exact + hi_pairs * 256 * 256 * 2.0 * n_pix +
                    inc * flops * 3 / 128)
    else:
        executed = flops * planes
    # pruned, the pass skips most of the dense work: its roofline counts the
    # tensor work it executes, and the dense-equivalent rate is reported beside
    done = executed / (dom_ms * 1e-3) / 1e12
    roof.update({"kernel": ("E-step pass 1: incremental and hi-plane bounds, exact "
                            "contraction of the tiles they leave live, online log-sum-exp"
                            if pruned else "E-step pass 1 (scores + online log-sum-exp)"),
                 "achieved": done if pruned else achieved, "peak": peak, "unit": "TFLOP/s",
                 "frac": (done if pruned else achieved) / peak,
                 "dense_equivalent_achieved": achieved,
                 "dense_equivalent_frac": achieved / peak,
                 "traffic": traffic,
                 "traffic_unit": ("bytes per iteration's pass 1 (increments, bound and exact "
                                  "launches)" if pruned else "bytes per launch"),
                 "traffic_source": ("ncu capture of this configuration" if traffic is not None
                                    else "unmeasured for this configuration"),
                 "algorithmic_flops_per_launch": flops, "executed_flops_per_launch": executed,
                 "executed_frac": executed / (dom_ms * 1e-3) / 1e12 / peak,
                 "exact_tile_fraction": exact,
                 "frac_basis": ("executed: every plane over the live tiles, the hi plane "
                                "where the hi-plane bound ran, the incremental bound's "
                                "product; dense_equivalent_*: 2 n_pix per pair over every "
                                "pair" if pruned else
                                "2 n_pix per pair over every pair (the split forms execute it "
                                "once per plane)")})
    return roof


def phase_rooflines(precision, n_pix, ld_pix, n_rot, n_data, phases, pass1_roof):
    """Roofline of every phase of the iteration (CUDA-event times per iteration
    inside emc_iteration), and the dominant one. Expansion and compression are
    measured against the copy bandwidth on the bytes the method itself must move
    (L written; Num read), the passes on the tensor cores against the BF16 peak."""
    pk, pk_src = peaks()
    hbm = pk["hbm_gbs"]
    planes = 3 if precision == "bf16_split" else 2 if precision == "fp16_split" else 1
    esz = 4 if precision == "fp32" else 2
    pairs = n_rot * n_data
    out = {}
    ms = phases["ms_expand"]
    b = planes * esz * n_rot * ld_pix  # L written
    out["expand"] = {"bound": "hbm", "unit": "GB/s", "achieved": b / (ms * 1e-3) / 1e9,
                     "peak": hbm, "peak_source": f"{pk_src} copy bandwidth", "ms": ms,
                     "algorithmic_bytes": b, "per_unit": f"{planes * esz} B of L per (i, j)",
                     "limiter": "instruction issue and gather latency",
                     "limiter_source": "ncu, 8192-frame case: 64% issue-active, long-scoreboard "
                                       "stalls first, DRAM at 17%"}
    ms = phases["ms_compress"]
    b = 4 * n_rot * ld_pix  # Num read
    out["compress"] = {"bound": "hbm", "unit": "GB/s", "achieved": b / (ms * 1e-3) / 1e9,
                       "peak": hbm, "peak_source": f"{pk_src} copy bandwidth", "ms": ms,
                       "algorithmic_bytes": b, "per_unit": "4 B of Num per (i, j)",
                       "limiter": "L1 / shared-memory (LSU) wavefronts of the corner merging "
                                  "and the L2 reductions",
                       "limiter_frac": 0.86,
                       "limiter_source": "ncu l1tex__data_pipe_lsu_wavefronts, 8192-frame case "
                                         "(DRAM at 2%, FP64 pipe 70% for the conversions)"}
    out["pass1"] = dict(pass1_roof, ms=phases["ms_loglik"])
    for k in ("expand", "compress"):
        out[k]["frac"] = out[k]["achieved"] / out[k]["peak"]
    out["normalize"] = {"ms": phases["ms_normalize"]}
    out["update"] = {"ms": phases["ms_update"]}
    dom = max(("expand", "pass1", "normalize", "update", "compress"), key=lambda k: out[k]["ms"])
    return out, dom


def scale_form(torch, emc, args, form, cache, stream, dist, world, local):
    """Another workload's own configuration with its own seeded data:
    emc128_recompute -- the two-pass streamed Maximize (pass 2 recomputes the
    scores of the live tiles, rotation chunks) at 128^3, 3 timed consecutive
    iterations after 2 warm-up ones; learned128 -- the learned proposal at
    128^3 (204960 rotations, top 512), 10 iterations per schedule."""
    from paper_1409_4256_gb300 import synth
    name = SCALE_FORMS[form]
    if name not in cache:
        c = dict(synth.WORKLOADS[name])
        t0 = time.perf_counter()
        d = synth.make_dataset(c["N"], c["D"], c["n_data"], c["mean_photons"],
                               masked_fraction=c["masked_fraction"],
                               fluence_sigma=c["fluence_sigma"], device=f"cuda:{local}")
        q, w = emc.quat_generate(c["n_quat"])
        cache[name] = (c, d, q, w, time.perf_counter() - t0)
    cfg, ds, quat, w, gen_s = cache[name]
    dev = torch.device("cuda", local)
    grid = torch.as_tensor(ds.model_start.astype(np.float32), device=dev)
    K_dev = torch.as_tensor(ds.K, device=dev)
    n_rot, n_data, n_pix = quat.shape[0], ds.K.shape[0], ds.q.shape[0]
    if form == "learned128":
        res = learned_form(torch, emc, args, cfg, ds, quat, w, grid, K_dev, stream, dist, world,
                           iters=10, max_cycles=2)
    else:
        floor = 1e-10 * float(ds.model_start.mean())
        ctx = emc.Context(cfg["N"], ds.q, quat, w, n_data, precision="bf16_split",
                          w_floor=floor, store_scores=False, device=str(dev), stream=stream,
                          rot_chunk=rot_chunk_for(n_rot, n_data), wide_counts=bool(ds.K.max() > 256))
        ctx.set_frames(K_dev, stream=stream)
        with ClockSampler(local) as clk:
            ms, ph, kernels, ll, _ = time_form(torch, emc, ctx, grid, 3, 2, stream, dist)
        del ctx
        res = {"value": world * n_rot * n_data / (ms * 1e-3), "ms_per_step": ms, "loglik": ll,
               "estep": "recompute", "rot_chunk": rot_chunk_for(n_rot, n_data),
               "phases_ms": ph, "gpu_launches": kernels, "clocks": clk.summary(),
               "roofline": pass1_roofline("bf16_split", n_pix, n_rot, n_data, ph,
                                          traffic_for(name, "bf16_split", n_rot, n_data, True,
                                                      ph))}
    res["workload"] = f"{name}: {WORKLOAD_TEXT[name]}"
    res["data_gen_s"] = gen_s
    del K_dev
    return res


def run_ours(args):
    import torch

    from paper_1409_4256_gb300 import build as libbuild
    from paper_1409_4256_gb300 import emc

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    libbuild.build()

    cfg, ds = workload(args, str(dev))
    quat, w = emc.quat_generate(cfg["n_quat"])
    n_rot, n_data, n_pix = quat.shape[0], ds.K.shape[0], ds.q.shape[0]
    pairs = n_rot * n_data
    grid = torch.as_tensor(ds.model_start.astype(np.float32), device=dev)
    floor = 1e-10 * float(ds.model_start.mean())
    K_dev = torch.as_tensor(ds.K, device=dev)
    stream = torch.cuda.Stream(device=dev)

    wide = bool(ds.K.max() > 256)  # counts above 256 (160^3): duplicate pixel columns

    def make_ctx(prec, **kw):
        c = emc.Context(cfg["N"], ds.q, quat, w, n_data, precision=prec, w_floor=floor,
                        store_scores=not args.recompute, device=str(dev), stream=stream,
                        rot_chunk=rot_chunk_for(n_rot, n_data), wide_counts=wide, **kw)
        c.set_frames(K_dev, stream=stream)
        return c

    ctx = make_ctx(args.precision)
    with ClockSampler(local) as clk:
        ms, phases, kernels, loglik, g_last = time_form(torch, emc, ctx, grid, args.steps,
                                                        args.warmup, stream, dist)
    clocks = clk.summary()
    ms = max_over_ranks(dist, ms, dev)
    value = whole_job_rate(world, pairs, ms)

    # ---- e2e: host frames in, new model out, through the public API ----------
    K_host = torch.as_tensor(ds.K).pin_memory()
    cur, nxt = g_last.clone(), torch.empty_like(grid)  # the reconstruction goes on
    e2e_steps = max(2, min(args.steps, 5))
    e2e_ms, out_bytes = e2e_timed(torch, ctx, K_host, K_dev, cur, nxt, e2e_steps, stream)
    e2e_ms = max_over_ranks(dist, e2e_ms, dev)
    e2e = {"value": whole_job_rate(world, pairs, e2e_ms), "unit": "pairs/s",
           "h2d_bytes_per_step": int(ds.K.nbytes), "d2h_bytes_per_step": out_bytes,
           "copies": "every step's frames from pinned host memory and its model back to "
                     "pinned host memory, on a copy stream overlapped with the neighbouring "
                     "iterations, all inside the timed region"}

    # ---- roofline of the dominant kernel ------------------------------------
    roof1 = pass1_roofline(args.precision, n_pix, n_rot, n_data, phases,
                           traffic_for(args.workload, args.precision, n_rot, n_data,
                                       args.recompute, phases))
    rooflines, dominant = phase_rooflines(args.precision, n_pix,
                                          ctx.buffer_sizes(n_rot).ld_pix, n_rot, n_data,
                                          phases, roof1)
    # the roofline line is the dominant phase's; the others follow in "rooflines"
    traffic_src = ("ncu dram__bytes_read.sum + dram__bytes_write.sum of one full-size launch "
                   "(one-pass launch-list capture of this configuration)")
    for k, name in (("compress", "compress_kernel (c-step, Eq. 2.12): trilinear scatter of the "
                                 "slices into the grid, corner terms merged in shared memory, "
                                 "FP64 reductions in L2"),
                    ("expand", "expand_tile_kernel (e-step, Eq. 2.9): trilinear gather of the "
                               "slices, log W split into planes, increments of the bound")):
        tr = traffic_for(args.workload, args.precision, n_rot, n_data, args.recompute, phases, k)
        rooflines[k].update({"kernel": name, "traffic": tr,
                             "traffic_source": traffic_src if tr is not None
                             else "unmeasured for this configuration"})
    roof = dict(rooflines[dominant], phase=dominant)

    # ---- other precision forms, briefly --------------------------------------
    forms = {args.precision: {"value": value, "ms_per_step": ms, "loglik": loglik}}
    others = [x for x in args.forms.split(",") if x and x not in (args.precision, "none")]
    for f in [x for x in others if x in ADAPTIVE_FORMS]:  # the one form that reuses ctx
        try:
            forms[f] = adaptive_form(torch, args, cfg, ds, grid, K_dev, stream, ctx, ms)
        except Exception as e:
            forms[f] = {"error": str(e)[:300]}
    del ctx  # every other form builds its own context
    torch.cuda.empty_cache()
    scale_data = {}
    for f in [x for x in others if x in SCALE_FORMS]:
        try:
            forms[f] = scale_form(torch, emc, args, f, scale_data, stream, dist, world, local)
        except Exception as e:
            forms[f] = {"error": str(e)[:300]}
        torch.cuda.empty_cache()
    scale_data.clear()
    torch.cuda.empty_cache()
    for f in [x for x in others if x not in ADAPTIVE_FORMS and x not in SCALE_FORMS]:
        if f in RECON_FORMS:
            try:
                if f == "reconstruct_learned":
                    forms[f] = reconstruct_learned_form(torch, emc, args, cfg, ds, quat, w, grid,
                                                        K_dev, stream, n_rot)
                else:
                    forms[f] = reconstruct_form(torch, args, cfg, ds, grid, stream, make_ctx,
                                                n_rot)
            except Exception as e:
                forms[f] = {"error": str(e)[:300]}
            continue
        if f in SPARSE_K_FORMS:
            try:
                forms[f] = sparse_k_form(torch, emc, cfg, ds, quat, w, grid, K_dev, stream,
                                         phases["ms_loglik"])
            except Exception as e:
                forms[f] = {"error": str(e)[:300]}
            continue
        if f in LEARNED_FORMS:
            try:
                forms[f] = learned_form(torch, emc, args, cfg, ds, quat, w, grid, K_dev, stream,
                                        dist, world)
            except Exception as e:
                forms[f] = {"error": str(e)[:300]}
            continue
        try:
            gauss, flu = f in GAUSS_FORMS, f in FLUENCE_FORMS
            c2 = (make_ctx(None, model="gaussian", sigma=args.sigma) if gauss else
                  make_ctx("bf16_split", model="poisson_fluence") if flu else make_ctx(f))
            fms, fph, _, fll, _ = time_form(torch, emc, c2, grid, 2, 3, stream, dist)
            forms[f] = {"value": world * pairs / (fms * 1e-3), "ms_per_step": fms, "loglik": fll,
                        "ms_loglik": fph["ms_loglik"]}
            if gauss:
                forms[f].update({"model": "Gaussian, per-(j,k) fluence (Eqs. 2.2-2.6)",
                                 "sigma": args.sigma, "phases_ms": fph})
            if flu:
                forms[f].update({"model": "Poisson, per-(j,k) maximum-likelihood fluence, "
                                          "BF16 split", "phases_ms": fph})
            del c2
        except Exception as e:  # a form that is not built yet is reported, not hidden
            forms[f] = {"error": str(e)[:200]}

    # ---- CPU oracle baseline (rank 0, N = 1) --------------------------------
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        from oracle import oracle
        oracle.build()
        quat_o, w_o = oracle.quat_generate(cfg["n_quat"])  # the oracle's own sampling
        n_rot_s, n_data_s = sample_sizes(cfg, ds, n_rot)
        v, dt, cores = oracle_sample(cfg, ds, quat_o, w_o, n_rot_s, n_data_s)
        cpu = {"value": v, "unit": "pairs/s", "cores": cores, "kind": "oracle",
               "sample": f"one FP64 oracle iteration over {n_rot_s} of {n_rot} rotations x "
                         f"{n_data_s} of {n_data} frames ({dt:.1f} s)"}

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": "pairs/s", "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": DTYPE[args.precision], "data": "synthetic",
                "config": {"workload": f"{args.workload}: {WORKLOAD_TEXT[args.workload]}",
                           "precision": args.precision, "rotations": n_rot, "frames": n_data,
                           "estep": "recompute" if args.recompute else "stored scores",
                           "pixels_used": n_pix, "parallelism": "replicas",
                           "l2": "inputs larger than L2 (log W and frames re-read every step)"},
                "phases_ms": phases, "roofline": roof, "rooflines": rooflines,
                "cpu_baseline": cpu, "e2e": e2e,
                "clocks": clocks, "gpu_launches": kernels, "forms": forms, "loglik": loglik}
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


def main():
    args = parse_args()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
