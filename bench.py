#!/usr/bin/env python3
"""Benchmark: simulated cells/s of the CCWSIM best-match search on GB300.

A step is one whole simulation call (data events, their Haar approximation,
the masked CCF over every candidate, top-K, Philox draw, Inverse-DWT paste,
for every patch of the raster path) on the workload named by --workload.
The default (c5: 256 realizations 512x512 of the 250x250 binary ribbon TI,
template 48, overlap 12, level 2) times the plain full-CCF batched form and
then the learned+batched form (the encoder is trained on the GPU first,
outside the timed region) on the same batch: `value` is the learned form,
`plain` the full search, with the pattern statistics of both ensembles as
the equal-accuracy evidence. Other workloads (--workload c2: one 2000x2000
3-facies realization with 400 hard data, top-5; c3, c4, t2_*) time one form.
Inputs are synthetic and seeded (workloads/configs.py).

Prints one JSON line. `value` is device-timed (CUDA events on the launching
stream, inputs resident, L2 flushed by a 256 MiB write between steps);
`e2e` is the same metric through the public API with host buffers (hard data
copied in from pinned memory, and the realizations copied back to pinned host
memory by the library, band by band as the wavefronts finish them, inside the
timed region). `--impl reference` times the CPU oracle instead, on a bounded
sample of patches per step.

Multi-GPU (torchrun, or --gpus N alone, which starts the ranks): realizations
are independent, so each rank simulates its own realizations with no exchange
(weak scaling); the time is the max over ranks.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

# FP32 FMA roofline of GB300: 152 SMs x 128 FP32 lanes x 2 flop x 2.07 GHz
# (maximum SM clock), for the CCF kernel on the FP32 lanes.
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.070e9 / 1e12


def hbm_peak_gbs():
    """Measured copy bandwidth of this GPU pool (MEASURED_PEAKS.json hbm_gbs)."""
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            return float(json.load(f)["hbm_gbs"]), "measured (MEASURED_PEAKS.json hbm_gbs)"
    except Exception:
        return 6800.0, "fallback (6.8 TB/s)"


def tensor_peak_tflops():
    """Measured dense BF16 GEMM throughput of this GPU pool (FP16 runs at the
    same dense rate): the roofline of the tensor-core CCF kernel."""
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            return float(json.load(f)["bf16_tflops"]), "measured (MEASURED_PEAKS.json bf16_tflops)"
    except Exception:
        return 1900.0, "fallback (1.9 PFLOP/s dense bf16)"

# workloads whose default run times the learned proposal beside the plain
# full search (the metric's comparison)
LEARNED_COMPARE = ("c5",)

WORKLOAD_TEXT = {
    "c1": "2D binary ribbon TI 250x250; 1 realization 250x250; T40 OR10 J1; no hard data; K=1",
    "c2": "2D 3-facies channel/lens TI 1000x1000; 1 realization 2000x2000; T64 OR16 J2; "
          "400 hard data; K=5",
    "c3": "2D binary ribbon TI 250x250; 64 realizations 1000x1000; T64 OR16 J2; K=1",
    "c4a": "3D 4-facies TI 180x150x120; 8 realizations 200x200x100; T24 OR6 J1; 1000 hard "
           "data; K=5",
    "c4b": "3D 4-facies TI 180x150x120; 8 realizations 100x100x100; T24 OR6 J1; 1000 hard "
           "data; K=5",
    "c4": "3D 4-facies TI 180x150x120; one batch of 8 realizations 200x200x100 and 8 of "
          "100x100x100; T24 OR6 J1; 1000 hard data per grid size; K=5",
    "c5": "2D binary ribbon TI 250x250; 256 realizations 512x512; T48 OR12 J2; K=1",
}
for _j in (1, 2, 3):
    for _g in (128, 256, 512, 768, 1024):
        WORKLOAD_TEXT[f"sw_j{_j}_g{_g}"] = (
            f"level sweep over grid sizes: 2D binary ribbon TI 250x250; 20 realizations "
            f"{_g}x{_g}; T32 OR8 J{_j}; hard data at 1000 per 512^2; K=5")
for _j in (1, 2, 3):
    for _h in (1000, 2000):
        WORKLOAD_TEXT[f"t2_j{_j}_h{_h}"] = (
            f"Table 2 level sweep: 2D binary ribbon TI 250x250; 20 realizations 512x512; T32 "
            f"OR8 J{_j}; {_h} hard data; K=5")


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="c5", choices=sorted(WORKLOAD_TEXT))
    ap.add_argument("--plain-only", action="store_true",
                    help="on the learned-proposal workload, time the plain full-CCF form only")
    ap.add_argument("--cpu-seconds", type=float, default=15.0,
                    help="target CPU time of the oracle baseline sample")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-cpu-parallel", action="store_true",
                    help="skip the realization-parallel oracle run on all host cores")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--precision", type=int, default=None,
                    help="0 FP32 FMA lanes, 1 FP16 tensor cores, 2 BF16 tensor cores "
                         "(default: 1 for 2D workloads, 0 for 3D)")
    ap.add_argument("--autotune", action="store_true",
                    help="pick the CCF tiling by timing every accepted one (outside the timed "
                         "region) instead of the committed per-workload table")
    ap.add_argument("--no-autotune", action="store_true",
                    help="the library's own tiling heuristic (ccf_tile 0)")
    ap.add_argument("--ccf-tile", type=lambda v: int(v, 0), default=None,
                    help="force this ccw_params.ccf_tile (implies --no-autotune)")
    ap.add_argument("--vt-ext", type=int, default=0,
                    help="non-causal conditioning: hard data up to this many cells beyond the "
                         "template's forward edges join the mismatch count (0 = off)")
    ap.add_argument("--all-shift", action="store_true",
                    help="all-shift (polyphase) candidates: every fine offset of the TI, "
                         "not only block-aligned ones (2D, tensor cores)")
    ap.add_argument("--boundary-cut", action="store_true",
                    help="paste through the minimum-error boundary cuts (2D)")
    ap.add_argument("--learned", action="store_true",
                    help="learned proposal (2D): train the encoder on pairs from plain runs "
                         "before timing, calibrate the gap threshold on held-out pairs")
    ap.add_argument("--train-real", type=int, default=1024,
                    help="plain realizations that generate the training pairs")
    ap.add_argument("--train-steps", type=int, default=600)
    ap.add_argument("--target-miss", type=float, default=0.02)
    return ap.parse_args()


def profiled_traffic(kernel: str, workload: str, tile: int, items_per_launch: float):
    """DRAM bytes of an average launch of `kernel` in the timed call, from the
    committed ncu summary (profiles/traffic.txt: bytes per launch over a few
    mid-call launches and the data events those launches processed), scaled
    to the timed call's mean data events per launch; None unless the capture
    was taken on this workload and tiling with the current kernel source."""
    import hashlib
    if items_per_launch <= 0:
        return None
    src = {"k_ccf_tc": "tc.cu", "k_ccf_tcs": "tcs.cu", "k_ccf_simt": "ccf_simt.cu",
           "k_nnsel_tc": "proposal.cu", "k_encode_tc": "encoder_tc.cu"}[kernel]
    path = os.path.join(ROOT, "paper_2404_00441_gb300", "csrc", src)
    try:
        with open(path, "rb") as f:
            sha = hashlib.sha256(f.read()).hexdigest()[:16]
        with open(os.path.join(ROOT, "profiles", "traffic.txt")) as f:
            for line in f:
                parts = line.split()
                if len(parts) >= 6 and not line.startswith("#") and parts[0] == kernel and \
                        parts[1] == workload and int(parts[2], 0) == tile and parts[3] == sha:
                    return int(float(parts[4]) * items_per_launch / float(parts[5]))
    except (OSError, ValueError, ZeroDivisionError):
        pass
    return None


def shard_real_base(rank: int, total_real: int, group_base: int) -> int:
    """First realization id of a group on `rank`: ranks own disjoint id
    ranges [rank * total_real, (rank + 1) * total_real), so every rank draws
    different Philox streams and no exchange is needed."""
    return rank * total_real + group_base


def max_over_ranks(values, world: int, device: str):
    """Element-wise max of a list of floats over all ranks (the job's time is
    that of its slowest rank)."""
    import torch
    t = torch.tensor(values, dtype=torch.float64, device=device)
    if world > 1:
        import torch.distributed as dist
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(v) for v in t.tolist()]


def wavefronts_of(grid, T, O):
    """Wavefront steps of the raster-equivalent schedule: a patch (ix, iy, iz)
    runs at step ix + 2 iy + 4 iz."""
    S = T - O
    n = [1 + (max(g - T, 0) + S - 1) // S for g in grid]
    n += [1] * (3 - len(n))
    return (n[0] - 1) + 2 * (n[1] - 1) + 4 * (n[2] - 1) + 1


def n_patches_of(grid, T, O):
    S = T - O
    n = 1
    for g in grid:
        n *= 1 + (max(g - T, 0) + S - 1) // S
    return n


def cells_of(grid):
    c = 1
    for g in grid:
        c *= g
    return c


# --------------------------------------------------------------- oracle ---
def oracle_sample(w, target_s, r=0):
    """Run the CPU oracle on the first patches of one realization's raster
    path until about target_s seconds have passed. Returns (patches, seconds,
    candidate evaluations)."""
    from oracle import oracle as O
    o = O.OracleTI(w["ti"], w["F"], w["J"])
    hd = w["hd"]
    kw = dict(K=w["K"], hd_cells=None if hd is None else hd[0],
              hd_vals=None if hd is None else hd[1], seed=w["seed"], r=r, want_log=False)
    # calibrate on a few patches, then run a sample sized to target_s
    n_total = n_patches_of(w["grid"], w["T"], w["O"])
    probe = min(n_total, 8)
    t0 = time.perf_counter()
    o.simulate(w["grid"], w["T"], w["O"], max_patches=probe, **kw)
    dt = time.perf_counter() - t0
    n = max(probe, min(n_total, int(probe * target_s / max(dt, 1e-6))))
    t0 = time.perf_counter()
    o.simulate(w["grid"], w["T"], w["O"], max_patches=n, **kw)
    dt = time.perf_counter() - t0
    return n, dt, n * o.num_candidates(w["T"])


_barrier = None


def _oracle_worker_init(barrier):
    global _barrier
    _barrier = barrier


def _oracle_worker(job):
    """One realization's first n patches on the oracle, in a worker process:
    the TI is prepared first, then every worker starts the clock together
    (a barrier) and returns its (start, end) on the host's monotonic clock."""
    try:
        from oracle import oracle as O
        w, r, n = job
        o = O.OracleTI(w["ti"], w["F"], w["J"])
        hd = w["hd"]
        kw = dict(K=w["K"], hd_cells=None if hd is None else hd[0],
                  hd_vals=None if hd is None else hd[1], seed=w["seed"], r=r, want_log=False)
    except BaseException:
        _barrier.abort()   # release the other workers at once
        raise
    _barrier.wait(timeout=120)
    t0 = time.monotonic()
    o.simulate(w["grid"], w["T"], w["O"], max_patches=n, **kw)
    return t0, time.monotonic()


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


class OraclePool:
    """The oracle realization-parallel over `procs` host cores: one spawned
    process per realization (0 .. procs-1), each running the first n patches
    of its raster path; run(n) returns the wall seconds from the first start
    to the last end (TI preparation and process start-up excluded)."""

    def __init__(self, w, procs):
        import multiprocessing as mp
        ctx = mp.get_context("spawn")   # no fork after CUDA is initialised
        keys = ("ti", "F", "J", "grid", "T", "O", "K", "hd", "seed")
        self.w = {k: w[k] for k in keys}
        self.procs = procs
        self.pool = ctx.Pool(procs, initializer=_oracle_worker_init,
                             initargs=(ctx.Barrier(procs),))

    def run(self, n):
        spans = self.pool.map(_oracle_worker, [(self.w, r, n) for r in range(self.procs)],
                              chunksize=1)
        return max(e for _, e in spans) - min(s0 for s0, _ in spans)

    def close(self):
        self.pool.close()
        self.pool.join()


def oracle_parallel(w, n, procs):
    """One realization-parallel run of the oracle (OraclePool) on `procs`
    cores; returns its wall seconds."""
    pool = OraclePool(w, procs)
    try:
        return pool.run(n)
    finally:
        pool.close()


# ------------------------------------------------------------- clocks -----
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index):
        self.proc = None
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200", "-i", str(device_index)],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except Exception:
            self.proc.kill()
            out, _ = self.proc.communicate()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.splitlines():
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx),
                "reasons": sorted(reasons), "samples": len(sm)}


# ------------------------------------------------------------ reference ---
def run_reference(args, rank, world):
    if rank != 0:
        return
    from workloads import configs
    w = configs.workload(args.workload)
    if w.get("groups"):
        w = dict(w, grid=w["groups"][0]["grid"], hd=w["groups"][0]["hd"])
    per_step = max(0.5, min(args.cpu_seconds, 45.0 / max(1, args.steps + args.warmup)))
    n_tot = n_patches_of(w["grid"], w["T"], w["O"])
    cells_per_patch = cells_of(w["grid"]) / n_tot
    # single thread: sizes the sample (about per_step seconds) and gives the
    # one-core figure
    n, dt1, ce1 = oracle_sample(w, per_step)
    single = {"value": n * cells_per_patch / dt1, "unit": "cells/s", "cores": 1,
              "sample": f"first {n} of {n_tot} patches of realization 0, {dt1:.1f} s"}
    procs = host_cores()
    vals, evs, ts = [], [], []
    try:
        # every step: the same sample on every host core at once, one
        # realization per core (realizations are independent, Algorithm 1)
        pool = OraclePool(w, procs)
        try:
            for _ in range(args.warmup):
                pool.run(max(1, n // 4))
            for _ in range(args.steps):
                wall = pool.run(n)
                vals.append(procs * n * cells_per_patch / wall)
                evs.append(procs * ce1 / wall)
                ts.append(wall)
        finally:
            pool.close()
        cores = procs
        sample = (f"first {n} of {n_tot} patches of realizations 0..{procs - 1} per step, "
                  f"one process per host core")
    except Exception as e:   # fall back to one core
        vals, evs, ts = [], [], []
        for _ in range(args.steps):
            n, dt, ce = oracle_sample(w, per_step)
            vals.append(n * cells_per_patch / dt)
            evs.append(ce / dt)
            ts.append(dt)
        cores = 1
        sample = (f"first {n} of {n_tot} patches of realization 0 per step, single thread "
                  f"(the all-core run failed: {type(e).__name__})")
    value = statistics.median(vals)
    line = {
        "impl": "reference", "metric": "simulated cells/s", "value": value,
        "unit": "cells/s", "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * statistics.median(ts), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "int64", "data": "synthetic",
        "cand_evals_per_s": statistics.median(evs),
        "config": {"workload": f"{args.workload}: {WORKLOAD_TEXT[args.workload]}",
                   "sample": sample},
        "cpu_baseline": {"value": value, "unit": "cells/s", "cores": cores, "kind": "oracle",
                         "sample": sample, "single_thread": single},
        "e2e": {"value": value, "unit": "cells/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------ ours ---
def train_proposal(args, ti, w, grid):
    """Trains the proposal encoder on the GPU from plain runs of the same
    geometry (not timed) and attaches it with a calibrated gap threshold."""
    import torch

    import paper_2404_00441_gb300 as ccw
    from paper_2404_00441_gb300 import proposal as PR
    t0 = time.time()
    tj = w["T"] // (2 ** w["J"])
    cnt_tr, best_tr = PR.generate_pairs(ti, grid, args.train_real, seed=1000)
    cnt_te, best_te = PR.generate_pairs(ti, grid, max(args.train_real // 16, 8), seed=2000)
    net = ccw.Net(w["F"], tj, seed=1)
    losses = PR.train(ti, net, cnt_tr, best_tr, args.train_steps, log_every=max(
        args.train_steps // 4, 1))
    ti.attach_proposal(net, 64, 0.0)
    hit, gap, _ = PR.proposal_hits(ti, cnt_te, best_te)
    theta = PR.calibrate_gap(hit, gap, args.target_miss)
    ti.attach_proposal(net, 64, theta)
    ok = gap >= 0
    settled = ok & (gap >= theta)
    miss = float((~hit[settled]).float().mean().item()) if settled.any() else 0.0
    torch.cuda.synchronize()
    return {"train_pairs": int(cnt_tr.shape[0]), "train_steps": args.train_steps,
            "loss_first_last": [losses[0], losses[-1]], "n_prop": 64, "theta": theta,
            "target_miss": args.target_miss, "held_out_miss_of_settled": miss,
            "held_out_settled_frac": float(settled.float().mean().item()),
            "prep_s": time.time() - t0}


def encoder_macs(C, tj):
    """Multiply-adds of one encoder pass (3 x 3 convolutions C -> 32, 32 -> 32
    stride 2, 32 -> 32 stride 2, linear -> 64) on a C x tj x tj input."""
    h2 = (tj - 1) // 2 + 1
    h3 = (h2 - 1) // 2 + 1
    return 32 * C * 9 * tj * tj + 32 * 32 * 9 * (h2 * h2 + h3 * h3) + 64 * 32 * h3 * h3


def ours_line(args, world, m):
    """The benchmark's JSON line from the measurements `m` (see run_ours)."""
    cells = m["cells_per_step"] * world * args.steps
    total_ms, kern_ms = m["total_ms"], m["kern_ms"]
    value = cells / (total_ms / 1e3)
    achieved = 2.0 * m["macs"] / (kern_ms / 1e3) / 1e12 if kern_ms > 0 else 0.0
    precision, tile = m["precision"], m["tile"]
    if precision == 0:
        bound, peak, peak_src = "alu", FP32_PEAK_TFLOPS, \
            "derived: 152 SMs x 128 FP32 lanes x 2 flop x 2070 MHz"
        kernel, kname = "k_ccf_simt", "k_ccf_simt (masked CCF on the FP32 lanes, per-tile top-K)"
    else:
        bound = "tensor"
        peak, peak_src = tensor_peak_tflops()
        if m["ndim"] == 3 or (tile >> 25) & 1:
            kernel = "k_ccf_tcs"
            kname = ("k_ccf_tcs (masked CCF on tcgen05 tensor cores, operands streamed through "
                     "shared-memory stages, per-CTA top-K)")
        else:
            kernel = "k_ccf_tc"
            kname = "k_ccf_tc (masked CCF on tcgen05 tensor cores, per-CTA top-K)"
    line = {
        "metric": "simulated cells/s", "value": value, "unit": "cells/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": total_ms / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": {0: "f32", 1: "f16", 2: "bf16"}[precision], "data": "synthetic",
        "cand_evals_per_s": m["cand_evals"] * world / (total_ms / 1e3),
        "config": {"workload": f"{args.workload}: {WORKLOAD_TEXT[args.workload]}",
                   "realizations_per_gpu": m["total_real"], "precision": precision,
                   "wavefronts": m.get("wavefronts"),
                   "ms_per_wavefront": (total_ms / args.steps / m["wavefronts"]
                                        if m.get("wavefronts") else None),
                   "ccf_tile": tile,
                   "l2": "flushed by a 256 MiB write between timed steps",
                   "parallelism": f"realizations sharded over {world} GPU(s), no exchange"},
        "roofline": {"bound": bound, "kernel": kname, "achieved": achieved, "peak": peak,
                     "unit": "TFLOP/s", "frac": achieved / peak,
                     "traffic": profiled_traffic(
                         kernel, args.workload, tile,
                         m.get("items_per_step", 0) * args.steps / max(m["n_launch"], 1)),
                     "traffic_note": "cold-cache DRAM bytes (read + write) per launch: ncu's "
                                     "bytes per data event over a few mid-call launches "
                                     "(profiles/traffic.txt) times the call's mean data events "
                                     "per launch; null unless taken on this workload, tiling "
                                     "and kernel source",
                     "launches": m["n_launch"],
                     "kernel_ms_per_step": kern_ms / args.steps,
                     "instrumented_ms_per_step": m["instr_ms"] / args.steps,
                     "timing": "CUDA events around every CCF launch on its stream, over a "
                               "second pass of the same K steps",
                     "peak_source": peak_src,
                     "work": "2 x (data-holding level-J cells x channels) flop per candidate"},
        "gpu_launches": int(m["launches"]),
        "clocks": m["clocks"],
    }
    if m.get("learned") is not None:
        line["config"]["learned"] = m["learned"]
    if m.get("prop_ms") and any(m["prop_ms"]):
        # the learned form: its dominant kernel may be the encoder or the
        # nearest-window selector rather than the CCF. Both run their
        # contractions on the tcgen05 tensor cores (BF16), so they are
        # measured against the BF16 peak with their algorithmic flops: the
        # encoder's multiply-adds per data event, 64 per (data event, TI
        # window) for the selector (which also ranks and re-ranks)
        items = m["items_per_step"] * world
        enc_ms, sel_ms = (v / args.steps for v in m["prop_ms"])
        enc_flop = 2.0 * encoder_macs(m["F"], m["Tj"]) * items
        sel_flop = 2.0 * 64 * m["n_cand"] * items
        parts = {"k_encode_tc": (enc_ms, enc_flop), "k_nnsel_tc": (sel_ms, sel_flop),
                 kernel: (kern_ms / args.steps, 2.0 * m["macs"] / args.steps)}
        line["learned_kernels"] = {
            k: {"ms_per_step": v[0], "flop_per_step": v[1],
                "tflops": v[1] / (v[0] / 1e3) / 1e12 if v[0] > 0 else 0.0}
            for k, v in parts.items()}
        line["learned_kernels"]["note"] = (
            "CUDA events around the encoder and around the selector (with its re-rank) inside "
            "the captured graph, second pass of the same K steps; flop = algorithmic work")
        top = max(parts, key=lambda k: parts[k][0])
        if top != kernel:
            ms, fl = parts[top]
            tpeak, tsrc = tensor_peak_tflops()
            ach = fl / (ms / 1e3) / 1e12 if ms > 0 else 0.0
            line["roofline"] = {
                "bound": "tensor", "kernel": top + (" (encoder of the data events, tcgen05 "
                                                    "implicit GEMMs)" if top == "k_encode_tc"
                                                    else " (nearest TI windows by embedding "
                                                    "on tcgen05, selection and exact "
                                                    "re-rank)"),
                "achieved": ach, "peak": tpeak, "unit": "TFLOP/s", "frac": ach / tpeak,
                # one launch per wavefront
                "traffic": profiled_traffic(top, args.workload, tile,
                                            m["items_per_step"] / max(m.get("wavefronts") or 1,
                                                                      1)),
                "traffic_note": "cold-cache DRAM bytes (read + write) per launch: ncu's bytes "
                                "per data event (profiles/traffic.txt) times the call's mean "
                                "data events per launch; null unless taken on this workload, "
                                "tiling and kernel source",
                "kernel_ms_per_step": ms,
                "timing": "CUDA events around the proposal kernels inside the captured graph, "
                          "second pass of the same K steps",
                "peak_source": tsrc,
                "work": "encoder: 2 x its multiply-adds per data event; selector: 2 x 64 "
                        "flop per (data event, TI window)"}
    # the library runs the learned form and the one-kernel form in one lane
    lanes = 1 if (tile >> 30) & 1 or m.get("learned") is not None else ((tile >> 20) & 7) + 1
    if lanes > 1:
        line["config"]["realization_lanes"] = lanes
        line["roofline"]["timing"] += (
            f"; with {lanes} realization lanes the launches of different lanes overlap, so "
            "the summed launch durations exceed the kernel's busy time and the fraction is a "
            "lower bound")
    if getattr(args, "vt_ext", 0):
        line["config"]["vt_ext"] = args.vt_ext
    if getattr(args, "boundary_cut", False):
        line["config"]["boundary_cut"] = 1
    if getattr(args, "all_shift", False):
        line["config"]["all_shift"] = 1
    if m.get("autotune") is not None:
        line["config"]["autotune"] = m["autotune"]
    if m.get("e2e_ms"):
        line["e2e"] = {"value": cells / (m["e2e_ms"] / 1e3), "unit": "cells/s",
                       "h2d_bytes_per_step": m["h2d"], "d2h_bytes_per_step": m["d2h"]}
    if m.get("phase_ms"):
        # the other two kernels of a wavefront step against the HBM roofline:
        # algorithmic bytes per data event / pasted patch
        hbm, hbm_src = hbm_peak_gbs()
        ndim = m["ndim"]
        td, tjd = m["T"] ** ndim, m["Tj"] ** ndim
        items = m["items_per_step"] * world
        per = {"k_events": td * (2 if m["has_hd"] else 1) + 4 * (m["F"] - 1) * tjd,
               "k_finish": 3 * td}
        kern = {}
        ev_ms = m["phase_ms"][0]
        if m.get("prop_ms"):
            # the events phase of the learned form spans the encoder and selector
            ev_ms = max(ev_ms - sum(m["prop_ms"]), 0.0)
        for name, ms in (("k_events", ev_ms), ("k_finish", m["phase_ms"][2])):
            ms_step = ms / args.steps
            by = items * per[name]
            gbs = by / (ms_step / 1e3) / 1e9 if ms_step > 0 else 0.0
            kern[name] = {"bound": "hbm", "ms_per_step": ms_step, "bytes_per_step": by,
                          "achieved": gbs, "peak": hbm, "unit": "GB/s", "frac": gbs / hbm}
        kern["note"] = ("bytes per item: events = template window (+ hard-data overlay) read + "
                        "level-J weights written; finish = pattern written + its 16-bit "
                        "coefficients read; times from the instrumented pass; peak " + hbm_src)
        line["kernels"] = kern
    return line


def run_ours(args, rank, world, local_rank, learned=None, cpu=True, keep=False):
    """Measures one form of the simulation (learned proposal on or off) and
    returns (JSON line or None off rank 0, the realizations when `keep`)."""
    import torch
    import torch.distributed as dist

    import paper_2404_00441_gb300 as ccw
    from workloads import configs

    torch.cuda.set_device(local_rank)
    w = configs.workload(args.workload)
    ti_t = torch.from_numpy(w["ti"]).cuda()
    g = ccw.TI(ti_t, w["F"], w["J"], w["T"], w["O"])
    # one or several grid sizes; each rank simulates its own realizations
    specs = w.get("groups") or [dict(grid=w["grid"], n_real=w["n_real"], hd=w["hd"],
                                     real_base=0)]
    total_real = sum(s["n_real"] for s in specs)
    groups = []
    for s in specs:
        hd = s["hd"]
        groups.append(dict(
            grid=tuple(s["grid"]), n_real=s["n_real"],
            real_base=shard_real_base(rank, total_real, s.get("real_base", 0)),
            hd_cells=None if hd is None else torch.from_numpy(hd[0]).cuda(),
            hd_vals=None if hd is None else torch.from_numpy(hd[1]).cuda(),
            hd_host=hd))
    ndim = len(groups[0]["grid"])
    bench_prec, bench_tile = configs.bench_tile(args.workload)
    precision = args.precision if args.precision is not None else bench_prec
    cells_per_step = sum(gr["n_real"] * cells_of(gr["grid"]) for gr in groups)
    learned = args.learned if learned is None else learned
    learned_info = None
    if learned:
        learned_info = train_proposal(args, g, w, groups[0]["grid"])
    # CCF tiling: the autotuner times every accepted (precision, tile) pair on
    # this batch (outside the timed region); results do not depend on it
    tile, tune_info = 0, None
    if args.ccf_tile is not None:
        tile = args.ccf_tile
    elif args.no_autotune:
        tile = 0
    elif not args.autotune:
        # the committed table (what the parity tests run)
        tile = bench_tile if precision == bench_prec else 0
        tune_info = {"chosen": f"p{precision}/{tile:#x}",
                     "source": "committed per-workload table (workloads/configs.py BENCH_TILE), "
                               "parity-tested at full size"}
    else:
        from paper_2404_00441_gb300 import autotune
        precs = ((precision,) if args.precision is not None
                 else (0, 1, 2))
        tg = [dict(grid=gr["grid"], n_real=gr["n_real"], real_base=gr["real_base"],
                   hd_cells=gr["hd_cells"], hd_vals=gr["hd_vals"]) for gr in groups]
        precision, tile, times = autotune.tune(g, tg, topk=w["K"], seed=w["seed"],
                                               precisions=precs, use_cache=False,
                                               vt_ext=args.vt_ext,
                                               boundary_cut=int(args.boundary_cut))
        tune_info = {"chosen": f"p{precision}/{tile:#x}", "timed_candidates": len(times),
                     "ms": {k: round(v, 3) for k, v in sorted(times.items(),
                                                                key=lambda kv: kv[1])[:6]}}
    outs = [torch.empty((gr["n_real"],) + gr["grid"][::-1], dtype=torch.uint8, device="cuda")
            for gr in groups]
    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device="cuda")
    stream = torch.cuda.current_stream()

    def run(hd_dev=None, host=None):
        hd_dev = hd_dev or [(gr["hd_cells"], gr["hd_vals"]) for gr in groups]
        host = host or [None] * len(groups)
        if len(groups) == 1:
            gr = groups[0]
            ccw.simulate(g, gr["grid"], n_real=gr["n_real"], topk=w["K"], seed=w["seed"],
                         hd_cells=hd_dev[0][0], hd_vals=hd_dev[0][1],
                         real_base=gr["real_base"], out=outs[0], precision=precision,
                         learned=1 if learned else 0, ccf_tile=tile,
                         vt_ext=args.vt_ext, boundary_cut=int(args.boundary_cut),
                         all_shift=int(getattr(args, "all_shift", False)), out_host=host[0])
            return outs
        res = ccw.simulate_groups(
            g, [dict(grid=gr["grid"], n_real=gr["n_real"], real_base=gr["real_base"],
                     hd_cells=h[0], hd_vals=h[1], out=o, out_host=ho)
                for gr, h, o, ho in zip(groups, hd_dev, outs, host)],
            topk=w["K"], seed=w["seed"], precision=precision,
            learned=1 if learned else 0, ccf_tile=tile, vt_ext=args.vt_ext,
            boundary_cut=int(args.boundary_cut), all_shift=int(getattr(args, "all_shift", False)))
        return [r[0] for r in res]

    for _ in range(max(args.warmup, 0)):
        run()
    torch.cuda.synchronize()

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    clocks = ClockSampler(local_rank)
    launches0 = ccw.launch_count()

    def timed_steps():
        barrier()
        ms = 0.0
        for _ in range(args.steps):
            flush.fill_(1)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            run()
            e1.record(stream)
            e1.synchronize()
            ms += e0.elapsed_time(e1)
        barrier()
        return ms

    total_ms = timed_steps()
    launches = ccw.launch_count() - launches0
    if learned_info is not None:
        n_known, n_prop, n_settled = g.proposal_stats()
        learned_info["settled_frac"] = n_settled / max(n_known, 1)
        learned_info["with_proposals_frac"] = n_prop / max(n_known, 1)
    # the same K steps again with a CUDA event pair recorded on the launching
    # stream around every CCF launch (inside the captured graph): the
    # kernel's own duration for the roofline. The events split the
    # programmatic launch overlap, so `value` comes from the pass above.
    ccw.profile_enable(True)
    run()   # captures the instrumented graph (not timed)
    torch.cuda.synchronize()
    ccw.profile_read()           # drop the capture call's counters
    ccw.profile_read_phases()
    ccw.profile_read_proposal()
    instr_ms = timed_steps()
    ccw.profile_enable(False)
    n_launch, kern_ms, cand_evals, macs = ccw.profile_read()
    phase_ms = ccw.profile_read_phases()
    prop_ms = ccw.profile_read_proposal()
    clk = clocks.stop()

    # end to end through the public API with host buffers: the hard data come
    # in from pinned host memory and the library copies the realizations back
    # to pinned host memory (band by band while the later wavefronts run)
    e2e_ms = None
    h2d = d2h = 0
    if not args.no_e2e:
        host_outs = [torch.empty(o.shape, dtype=torch.uint8).pin_memory() for o in outs]
        pinned, dev_hd = [], []
        for gr in groups:
            hd = gr["hd_host"]
            if hd is None:
                pinned.append(None)
                dev_hd.append((None, None))
                continue
            pc = torch.from_numpy(hd[0]).pin_memory()
            pv = torch.from_numpy(hd[1]).pin_memory()
            pinned.append((pc, pv))
            dev_hd.append((torch.empty_like(pc, device="cuda"), torch.empty_like(pv, device="cuda")))
            h2d += pc.numel() * 4 + pv.numel()
        d2h = sum(o.numel() for o in outs)
        run(dev_hd, host_outs)   # builds the read-back graph for these buffers (not timed)
        barrier()
        e2e_ms = 0.0
        for _ in range(args.steps):
            flush.fill_(1)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for p, dv in zip(pinned, dev_hd):
                if p is not None:
                    dv[0].copy_(p[0], non_blocking=True)
                    dv[1].copy_(p[1], non_blocking=True)
            run(dev_hd, host_outs)
            e1.record(stream)
            e1.synchronize()
            e2e_ms += e0.elapsed_time(e1)
        barrier()

    total_ms, e2e_ms_max, kern_ms_max = max_over_ranks([total_ms, e2e_ms or 0.0, kern_ms], world,
                                                       "cuda")
    if rank != 0:
        return None, (outs if keep else None)
    line = ours_line(args, world, dict(
        total_ms=total_ms, kern_ms=kern_ms, instr_ms=instr_ms, macs=macs, cand_evals=cand_evals,
        n_launch=n_launch, launches=launches, clocks=clk, precision=precision, tile=tile,
        ndim=ndim, total_real=total_real, cells_per_step=cells_per_step,
        e2e_ms=e2e_ms_max if e2e_ms else None, h2d=h2d, d2h=d2h, learned=learned_info,
        autotune=tune_info, phase_ms=phase_ms, prop_ms=prop_ms if learned else None,
        n_cand=g.n_cand,
        items_per_step=sum(gr["n_real"] * n_patches_of(gr["grid"], w["T"], w["O"])
                           for gr in groups),
        T=w["T"], Tj=w["T"] // (2 ** w["J"]), F=w["F"],
        wavefronts=max(wavefronts_of(gr["grid"], w["T"], w["O"]) for gr in groups),
        has_hd=any(gr["hd_host"] is not None for gr in groups)))
    if cpu and not args.no_cpu_baseline and world == 1:
        w0 = dict(w, grid=groups[0]["grid"], hd=groups[0]["hd_host"])
        n, dt, ce = oracle_sample(w0, args.cpu_seconds)
        grid = groups[0]["grid"]
        n_tot = n_patches_of(grid, w["T"], w["O"])
        line["cpu_baseline"] = {"value": n * cells_of(grid) / n_tot / dt, "unit": "cells/s",
                                "cores": 1, "kind": "oracle",
                                "sample": f"first {n} of {n_tot} patches of one realization, "
                                          f"{dt:.1f} s, single thread",
                                "cand_evals_per_s": ce / dt}
        if not args.no_cpu_parallel:
            procs = host_cores()
            try:
                wall = oracle_parallel(w0, n, procs)
                line["cpu_baseline"]["parallel"] = {
                    "value": procs * n * cells_of(grid) / n_tot / wall, "unit": "cells/s",
                    "cores": procs, "kind": "oracle",
                    "sample": f"first {n} of {n_tot} patches of realizations 0..{procs - 1}, "
                              f"one process per host core, {wall:.1f} s wall"}
            except Exception as e:   # the single-thread figure above stands
                line["cpu_baseline"]["parallel"] = {"unavailable": f"{type(e).__name__}: {e}"}
    return line, (outs if keep else None)


def ensemble_statistics(outs, ti, F):
    """Pattern-reproduction statistics of an ensemble of 2D realizations on
    the GPU (Sec. 5.2-5.3): facies-1 proportion, E-W indicator variogram and
    probability of connection of facies 1, 4 x 4 pattern histograms at full
    and half resolution."""
    import torch

    from paper_2404_00441_gb300 import evaluate as ev
    reals = torch.cat([o.reshape((-1,) + tuple(o.shape[-2:])) for o in outs])
    lags = (1, 2, 4, 8, 16, 32)
    plags = (8, 32, 64)
    return dict(
        n=int(reals.shape[0]),
        prop=ev.proportions(reals, F).numpy()[:, 1],
        vario=ev.variogram(reals, 1, 0, lags).numpy(),
        conn=ev.connection_probability(reals, 1, plags, 0),
        hist=[ev.pattern_histogram(reals, F, 4, d) for d in (1, 2)],
        lags=lags, plags=plags)


def compare_ensembles(a, b, ti_stats):
    """Equal-accuracy evidence between two ensembles (means with 95 % half
    widths, and the Jensen-Shannon divergence of their pattern histograms;
    the same divergence of each against the TI)."""
    import math

    import numpy as np

    from paper_2404_00441_gb300 import evaluate as ev

    def ci(x):
        x = np.asarray(x, np.float64)
        return [float(np.nanmean(x, 0).round(6)) if x.ndim == 1 else
                [round(float(v), 6) for v in np.nanmean(x, 0)],
                float((1.96 * np.nanstd(x, 0, ddof=1) / math.sqrt(len(x))).max())]
    out = {"realizations": [a["n"], b["n"]]}
    for k in ("prop", "vario", "conn"):
        out[k] = {"plain": ci(a[k]), "learned": ci(b[k])}
    out["variogram_lags"] = list(a["lags"])
    out["connection_lags"] = list(a["plags"])
    out["js_learned_vs_plain"] = [round(ev.js_divergence(x, y), 5)
                                  for x, y in zip(a["hist"], b["hist"])]
    out["js_vs_ti"] = {"plain": [round(ev.js_divergence(x, y), 5)
                                 for x, y in zip(a["hist"], ti_stats["hist"])],
                       "learned": [round(ev.js_divergence(x, y), 5)
                                   for x, y in zip(b["hist"], ti_stats["hist"])]}
    out["note"] = ("means over the ensembles with 95 % half widths; JS divergence of 4x4 "
                   "pattern histograms at down 1 and 2")
    return out


def rank_command(argv, n):
    """The torchrun command that runs this benchmark on n local ranks (one per
    GPU, rendezvous on 127.0.0.1 at a free port) with the same arguments."""
    import socket
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    return [sys.executable, "-m", "torch.distributed.run", "--nnodes=1",
            f"--nproc-per-node={n}", "--master-addr", "127.0.0.1", "--master-port", str(port),
            os.path.abspath(__file__)] + list(argv)


def main():
    args = parse_args()
    if args.gpus > 1 and "WORLD_SIZE" not in os.environ:
        # `--gpus N` without a launcher: start the N ranks here (rank 0 prints
        # the line; n_gpus is the number of ranks that ran)
        sys.exit(subprocess.call(rank_command(sys.argv[1:], args.gpus)))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(local_rank)
        dist.init_process_group("nccl")
    if args.workload in LEARNED_COMPARE and not args.plain_only and not args.learned:
        # the metric's comparison: the plain full-CCF batched form, then the
        # learned+batched form of the same batch (value = the latter)
        plain, plain_outs = run_ours(args, rank, world, local_rank, learned=False, cpu=False,
                                     keep=True)
        line, outs = run_ours(args, rank, world, local_rank, learned=True, cpu=True, keep=True)
        if rank == 0:
            import torch
            from workloads import configs
            w = configs.workload(args.workload)
            ti_t = torch.from_numpy(w["ti"]).cuda()[None]
            line["plain"] = {k: plain[k] for k in ("value", "ms_per_step", "cand_evals_per_s",
                                                   "e2e", "roofline", "gpu_launches", "config",
                                                   "kernels")
                             if k in plain}
            line["learned_vs_plain"] = line["value"] / plain["value"]
            line["accuracy"] = compare_ensembles(
                ensemble_statistics(plain_outs, w["ti"], w["F"]),
                ensemble_statistics(outs, w["ti"], w["F"]),
                ensemble_statistics([ti_t], w["ti"], w["F"]))
            line["metric"] = "simulated cells/s (learned+batched; plain full-CCF in 'plain')"
            print(json.dumps(line), flush=True)
    else:
        line, _ = run_ours(args, rank, world, local_rank)
        if rank == 0:
            print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
