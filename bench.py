#!/usr/bin/env python
"""Benchmark of the DartMinHash hot path on GB300.

One step = one dm_sketch_bbit call over workload W1 (1,000,000 weighted sets, 256 distinct
elements each over d = 2^20, Exp(1) weights): k = 256 uint64 minhash keys plus the 1-bit
packed sketch (4 words) per set, inputs and outputs resident in HBM (2 GB in, 2 GB out: far
larger than the 129 MB L2, so no flush between steps).  Prints one JSON line (rank 0).  The same
run then times the heavy-tailed W2 batch (200,000 sets, k = 1024) in the batched and the plain
per-set forms and reports it under "w2" in that line (--no-w2 skips it).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl dm|reference] [--sets N]

Under torchrun (N > 1) every rank sketches its own W1 batch on its own GPU (weak scaling,
no data-path collective); the barrier and the max-over-ranks time use torch.distributed.
--impl reference times the oracle (plain single-threaded C per set, run over all host cores)
on the same workload, as the reference arm.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

K_SLOTS = 256
B_BITS = 1
SEED = 1
METRIC = "weighted sets/s (k=256 minhashes + 1-bit sketch, bit-exact)"

# Algorithmic integer work per unit (32-bit lane operations), counted from the method's own
# arithmetic: SplitMix64's output function = 3 xor-shifts of a 64-bit word (4 ops each) + 2
# 64-bit multiplies by constants (3 ops each) = 18.
OPS_MIX = 18
OPS_PER_AREA = 2 + OPS_MIX + 2              # counter step, hash, Poisson inversion (E[X]+1 compares)
OPS_PER_DART = 2 + OPS_MIX + 3 + 1 + 4 + 4 + 1   # counter, hash, U/V, weight test, rank, code, compare
OPS_PER_KEPT = OPS_MIX + 1 + 1 + 1          # bucket/fingerprint hash, fastrange, key, min
INT_LANES_PER_SM = 128                      # 4 schedulers x 32 lanes, one integer op per lane per clock


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["dm", "reference"], default="dm")
    ap.add_argument("--sets", type=int, default=None, help="prefix of the workload (profiling only)")
    ap.add_argument("--workload", choices=["W1", "W2", "W3", "W4", "W1B", "CMP", "W3S", "IDX", "T1"], default="W1",
                    help="W1 (default, the headline): k=256 keys + 1-bit words; W2: k=1024 heavy-tailed batch; "
                         "W3: (L, K) = (64, 8) LSH; W4: serving loop on a Poisson request trace; "
                         "W1B: bottom-k sketches (k=256) of the W1 sets; CMP: similarity counts of sketch pairs; "
                         "W3S: W3 with each set's weight class normalised to ||x||_1 in [1, 2); "
                         "IDX: LSH-table index build and query over the W3 values; "
                         "T1: Table 1's sets (1,024 elements, 64-bit ids, binary64 weights, k=256) at "
                         "||x||_1 = 1, 2^64, 2^-64, 2^512, 2^-512 through dm_sketch_f64")
    ap.add_argument("--duration", type=float, default=60.0, help="W4: seconds of 50,000/s arrivals to replay")
    ap.add_argument("--norm-exp", type=int, default=2,
                    help="W3S: normalise each weight class to ||x||_1 in [2^e, 2^(e+1)) (2: first limit below 1)")
    ap.add_argument("--form", choices=["batched", "plain", "persistent"], default="batched",
                    help="launch form (the plain form is the one-warp-per-set reference)")
    ap.add_argument("--large-nnz", type=int, default=None, help="batched form: element count of a large set")
    ap.add_argument("--phi0", type=float, default=None, help="initial phi (launch setting; with --autotune off)")
    ap.add_argument("--wpb", type=int, default=None, help="warps per block (launch setting; with --autotune off)")
    ap.add_argument("--autotune", choices=["on", "off"], default="on",
                    help="dm_autotune on a prefix of the batch before the warm-up (launch settings only)")
    ap.add_argument("--no-graph", action="store_true", help="plain launches instead of CUDA-graph replay")
    ap.add_argument("--no-plain", action="store_true", help="skip the plain per-set form measured beside")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-w2", action="store_true", help="W1: skip the heavy-tailed batch timed beside it")
    return ap.parse_args()


# ------------------------------------------------------------------------------------------
# distributed plumbing (host logic; covered by gloo tests)
# ------------------------------------------------------------------------------------------
def dist_env():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)), int(os.environ.get("LOCAL_RANK", 0))


def dist_init(world: int, use_cuda: bool):
    if world <= 1:
        return None
    import torch.distributed as dist
    if not dist.is_initialized():
        dist.init_process_group(backend="nccl" if use_cuda else "gloo")
    return dist


def barrier(dist, use_cuda: bool):
    import torch
    if use_cuda:
        torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()


def max_over_ranks(dist, value: float, use_cuda: bool) -> float:
    if dist is None:
        return value
    import torch
    t = torch.tensor([value], dtype=torch.float64, device="cuda" if use_cuda else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(dist, value: float, use_cuda: bool) -> float:
    if dist is None:
        return value
    import torch
    t = torch.tensor([value], dtype=torch.float64, device="cuda" if use_cuda else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


# ------------------------------------------------------------------------------------------
# clocks during the timed region
# ------------------------------------------------------------------------------------------
CLOCK_QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
               "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
               "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")


class ClockSampler:
    def __init__(self, gpu: int):
        self.gpu = gpu
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={CLOCK_QUERY}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        time.sleep(0.25)

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        self.proc.wait()
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        os.unlink(self.path)
        return summarize_clocks(rows)


def summarize_clocks(rows):
    import statistics
    names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
    sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
    mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
    reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
    return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
            "reasons": reasons, "samples": len(rows)}


# ------------------------------------------------------------------------------------------
# traffic from the committed ncu capture (valid only for the kernel source it was taken on)
# ------------------------------------------------------------------------------------------
def kernel_fingerprint() -> str:
    """Hash of the kernel sources (device code only) with comments and blank space removed, so
    that a change of wording does not retire a capture but any change of code does."""
    import hashlib
    import re
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2005_11547_gb300", "csrc")
    for f in ("dm_sketch.cu", "dm_device.cuh"):
        text = open(os.path.join(csrc, f), encoding="utf-8").read()
        text = re.sub(r"/\*.*?\*/", " ", text, flags=re.S)
        text = re.sub(r"//[^\n]*", " ", text)
        h.update(" ".join(text.split()).encode())
    return h.hexdigest()[:16]


def mix_ceiling(dmx, props, peak_ops, stream):
    """What pure hashing reaches: SplitMix64 chains alone (dm_mix64_burn, full occupancy), in the
    same op count per mix as the roofline's work model, against the same peak."""
    import torch
    blocks, iters = props.multi_processor_count * 8, 20000
    out = dmx.dm_mix64_burn(blocks, 100, stream=stream)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    ev[0].record(stream)
    dmx.dm_mix64_burn(blocks, iters, out=out, stream=stream)
    ev[1].record(stream)
    torch.cuda.synchronize()
    s = ev[0].elapsed_time(ev[1]) / 1e3
    mixes = 4 * iters * 256 * blocks
    return {"kernel": "dm_mix64_burn", "mix64_per_s": mixes / s, "gop_per_s": mixes * OPS_MIX / s / 1e9,
            "frac_of_peak": mixes * OPS_MIX / s / peak_ops}


# ------------------------------------------------------------------------------------------
# CPU oracle timing (cpu_baseline leg and the reference arm)
# ------------------------------------------------------------------------------------------
def traffic_per_set(wl: str):
    """DRAM bytes per set of the workload's dominant kernel, from its committed ncu capture
    (profiles/traffic_<workload>.json: read + write bytes of one launch over a prefix of the batch,
    divided by the sets it processed).  None when the workload has no capture or the kernel source
    changed since it was taken."""
    path = os.path.join(ROOT, "profiles", f"traffic_{wl.lower()}.json")
    if not os.path.exists(path):
        return None
    d = json.load(open(path))
    if d.get("workload") != wl or d.get("kernel_fingerprint") != kernel_fingerprint():
        return None
    return d.get("dram_bytes_per_set")


def time_oracle(batch, n_sample: int, cores: int):
    import oracle
    sub = batch.rows(range(min(n_sample, batch.n_sets)))
    oracle.build()
    t0 = time.perf_counter()
    oracle.sketch_bbit(sub.indptr, sub.indices, sub.weights, K_SLOTS, B_BITS, SEED, keys=True, threads=cores)
    dt = time.perf_counter() - t0
    return sub.n_sets / dt, sub.n_sets, dt


WL_DESC = {
    "W1": "W1: 1,000,000 sets x 256 distinct elements (d=2^20), Exp(1) fp32 weights; k=256 uint64 keys + 1-bit words",
    "W2": "W2: 200,000 heavy-tailed sets (nnz log-normal median 100, sigma 1.5, clipped to [1, 1e5]; ||x||_1 "
          "log-uniform 1e-3..1e3), d=2^24; k=1024 uint64 keys",
    "W3": "W3: 1,000,000 tf-idf-like sets (Zipf(1.1) tokens, nnz U{200..2000}), d=2^20; (L, K) = (64, 8) LSH uint32 "
          "values",
    "W1B": "W1 sets (1,000,000 x 256 elements, Exp(1) weights); bottom-k sketches, k=256 sorted uint64 keys",
}


def reference_arm(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    import workloads
    b = workloads.workload1(min(args.sets or 1_000_000, 200_000))
    cores = os.cpu_count() or 1
    per_step = 4000 * cores
    sets = []
    for s in range(args.warmup + args.steps):
        lo = (s * per_step) % max(1, b.n_sets - per_step)
        sub = b.rows(range(lo, lo + per_step))
        v, n, dt = time_oracle(sub, per_step, cores)
        if s >= args.warmup:
            sets.append((n, dt))
    n_tot = sum(n for n, _ in sets)
    t_tot = sum(dt for _, dt in sets)
    value = n_tot / t_tot
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "sets/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t_tot / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int64",
        "data": "synthetic", "minhashes_per_s": value * K_SLOTS,
        "config": {"workload": "W1: 1,000,000 sets x 256 distinct elements (d=2^20), Exp(1) fp32 weights; "
                               "k=256 uint64 keys + 1-bit words", "k": K_SLOTS, "b": B_BITS,
                   "step": f"{per_step} sets of W1 per step (bounded sample)"},
        "cpu_baseline": {"value": value, "unit": "sets/s", "cores": cores, "kind": "oracle",
                         "sample": f"{per_step} W1 sets per step x {args.steps} steps"},
        "e2e": {"value": value, "unit": "sets/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------------------------------
# GPU arm
# ------------------------------------------------------------------------------------------
def measure(args, wl, local, dist, props, full):
    """Time one batch workload (W1, W2, W3, W1B, W3S) on this rank's GPU: autotune, graph replay,
    W warm-up steps, K steps between barriers with CUDA events on the launching stream (max over
    ranks), the unit counts of one launch, the plain per-set form beside it.  full: also the
    end-to-end leg through the host-buffer entry (W1), the hash ceiling and the CPU oracle."""
    import numpy as np
    import torch

    import paper_2005_11547_gb300 as dmx
    import workloads

    rank, world, _ = dist_env()
    # every rank sketches a batch of its own, drawn from the same distribution (rank 0's is the
    # workload itself): independent problems, no data-path collective
    if wl in ("W1", "W1B"):
        b = workloads.workload1(args.sets or 1_000_000, shard=rank)
    elif wl == "W2":
        b = workloads.workload2(args.sets or 200_000, shard=rank)
    else:
        b = workloads.workload3(args.sets or 1_000_000, shard=rank)
    lsh_kind = wl in ("W3", "W3S")
    n = b.n_sets
    kk = {"W1": K_SLOTS, "W2": 1024, "W3": 64, "W1B": K_SLOTS, "W3S": 64}[wl]
    words = (K_SLOTS * B_BITS + 63) // 64
    ip = torch.from_numpy(b.indptr).cuda()
    ix = torch.from_numpy(b.indices.view(np.int32)).cuda()
    w = torch.from_numpy(b.weights).cuda()
    if lsh_kind:
        keys = torch.empty((n, 64), dtype=torch.int32, device="cuda")
        outw = None
    else:
        keys = torch.empty((n, kk), dtype=torch.int64, device="cuda")
        outw = torch.empty((n, words), dtype=torch.int64, device="cuda") if wl == "W1" else None
    cls = torch.empty(n, dtype=torch.int32, device="cuda")
    scl = torch.empty(n, dtype=torch.int32, device="cuda")
    form_id = {"batched": dmx.FORM_BATCHED, "plain": dmx.FORM_PLAIN, "persistent": dmx.FORM_PERSISTENT}[args.form]

    def manual_settings(c):
        dmx.dm_set_option(c, dmx.OPT_FORM, form_id)
        if args.large_nnz is not None:
            dmx.dm_set_option(c, dmx.OPT_LARGE_NNZ, args.large_nnz)
        if args.phi0 is not None:
            dmx.dm_set_option(c, dmx.OPT_LSH_PHI0 if lsh_kind else dmx.OPT_PHI0, int(round(args.phi0 * 1024)))
        if args.wpb is not None:
            dmx.dm_set_option(c, dmx.OPT_WARPS_PER_BLOCK, args.wpb)

    ctx = dmx.dm_create(local)
    manual_settings(ctx)
    stream = torch.cuda.current_stream()

    def launch(c):
        if wl == "W1":
            dmx.dm_sketch_bbit(c, ip, ix, w, K_SLOTS, B_BITS, SEED, out_words=outw, out_keys=keys, stream=stream)
        elif wl == "W2":
            dmx.dm_sketch(c, ip, ix, w, 1024, SEED, out=keys, stream=stream)
        elif wl == "W1B":
            dmx.dm_bottomk(c, ip, ix, w, K_SLOTS, SEED, out=keys, stream=stream)
        elif wl == "W3S":
            # classes, then the class-normalised values (both inside the step)
            dmx.dm_weight_classes(c, ip, w, out=cls, scale_out=scl, norm_exp=args.norm_exp, stream=stream)
            dmx.dm_lsh_scaled(c, ip, ix, w, 64, 8, SEED, scl, out=keys, stream=stream)
        else:
            dmx.dm_lsh(c, ip, ix, w, 64, 8, SEED, out=keys, stream=stream)

    # launch settings: the autotuner on a prefix of the batch (results never depend on them)
    tuning = None
    if args.autotune == "on" and args.form == "batched":
        if wl == "W1":
            tuning = dmx.dm_autotune(ctx, ip, ix, w, K_SLOTS, SEED, b=B_BITS, stream=stream)
        elif wl == "W2":
            tuning = dmx.dm_autotune(ctx, ip, ix, w, 1024, SEED, max_sets=n, stream=stream)
        elif wl == "W1B":
            tuning = dmx.dm_autotune(ctx, ip, ix, w, K_SLOTS, SEED, bottomk=True, stream=stream)
        elif wl == "W3":
            tuning = dmx.dm_autotune(ctx, ip, ix, w, 64, SEED, lsh_K=8, stream=stream)
    if not args.no_graph:
        dmx.dm_set_option(ctx, dmx.OPT_GRAPH, 1)

    # work units of one launch (untimed counting launch with the same settings; counters never
    # change output bits)
    cnt = torch.zeros(4, dtype=torch.int64, device="cuda")
    cctx = dmx.dm_create(local)
    dmx.dm_set_option(cctx, dmx.OPT_COUNTERS, cnt.data_ptr())
    manual_settings(cctx)
    if tuning:
        dmx.dm_set_option(cctx, dmx.OPT_FORM, tuning["form"])
        dmx.dm_set_option(cctx, dmx.OPT_WARPS_PER_BLOCK, tuning["warps_per_block"])
        dmx.dm_set_option(cctx, dmx.OPT_LARGE_NNZ, tuning["large_nnz"])
        dmx.dm_set_option(cctx, dmx.OPT_LARGE_WORK, tuning["large_work"])
        dmx.dm_set_option(cctx, dmx.OPT_LSH_PHI0 if lsh_kind else dmx.OPT_PHI0, tuning["phi0_1024"])
    launch(cctx)
    dmx.dm_sync_status(cctx)
    areas, darts, kept, passes = [int(v) for v in cnt.cpu().tolist()]
    cctx.close()

    for _ in range(max(3, args.warmup)):
        launch(ctx)
    dmx.dm_sync_status(ctx)
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    sampler = ClockSampler(local)
    sampler.start()
    barrier(dist, True)
    t_wall = time.perf_counter()
    for i in range(args.steps):
        starts[i].record(stream)
        launch(ctx)
        ends[i].record(stream)
    barrier(dist, True)
    t_wall = time.perf_counter() - t_wall
    clocks = sampler.stop()
    dmx.dm_sync_status(ctx)
    per_launch_ms = [starts[i].elapsed_time(ends[i]) for i in range(args.steps)]
    total_ms = starts[0].elapsed_time(ends[-1])
    t_max = max_over_ranks(dist, total_ms / 1e3, True)
    all_sets = sum_over_ranks(dist, float(n * args.steps), True)
    value = all_sets / t_max

    # the plain per-set form (one warp per set in input order, static grid) on the same batch
    plain = None
    if not args.no_plain and args.form == "batched":
        pctx = dmx.dm_create(local)
        dmx.dm_set_option(pctx, dmx.OPT_FORM, dmx.FORM_PLAIN)
        launch(pctx)
        pe = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
        barrier(dist, True)
        pe[0].record(stream)
        for _ in range(3):
            launch(pctx)
        pe[1].record(stream)
        barrier(dist, True)
        dmx.dm_sync_status(pctx)
        pctx.close()
        p_max = max_over_ranks(dist, pe[0].elapsed_time(pe[1]) / 3 / 1e3, True)
        plain = {"ms_per_step": p_max * 1e3, "value": all_sets / args.steps / p_max, "unit": "sets/s",
                 "batched_over_plain": value / (all_sets / args.steps / p_max)}

    # the one-kernel-per-set form: every set of a sample is its own dm_sketch call (plain form,
    # one set), so each set pays its own launches; timed on the device over the sample, and each
    # set's keys checked against the batched call's
    per_set = None
    if wl == "W2" and plain is not None:
        sctx = dmx.dm_create(local)
        dmx.dm_set_option(sctx, dmx.OPT_FORM, dmx.FORM_PLAIN)
        ns = min(n, 2000)
        got = torch.empty((ns, kk), dtype=torch.int64, device="cuda")

        def one(i):
            dmx.dm_sketch(sctx, ip[i:i + 2], ix, w, kk, SEED, out=got[i], stream=stream)

        for i in range(min(ns, 64)):
            one(i)
        se = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
        barrier(dist, True)
        se[0].record(stream)
        for i in range(ns):
            one(i)
        se[1].record(stream)
        barrier(dist, True)
        dmx.dm_sync_status(sctx)
        sctx.close()
        if not torch.equal(got, keys[:ns]):
            raise RuntimeError("per-set calls differ from the batched call's keys")
        s_max = max_over_ranks(dist, se[0].elapsed_time(se[1]) / 1e3, True)
        rate = world * ns / s_max
        per_set = {"value": rate, "unit": "sets/s", "ms_per_step_extrapolated": n / (ns / s_max) * 1e3,
                   "sample": f"first {ns} sets, one dm_sketch call (plain form, one set) each, device time",
                   "batched_over_per_set": value / rate}

    # end to end through the host-buffer C-ABI entry (copies inside the timed region)
    e2e = None
    if full and not args.no_e2e and wl == "W1":
        hip = torch.from_numpy(b.indptr).pin_memory()
        hix = torch.from_numpy(b.indices.view(np.int32)).pin_memory()
        hw = torch.from_numpy(b.weights).pin_memory()
        hk = torch.empty((n, K_SLOTS), dtype=torch.int64).pin_memory()
        hwd = torch.empty((n, words), dtype=torch.int64).pin_memory()
        e2e_steps = max(2, min(args.steps, 5))
        ref_keys = keys.cpu().numpy()

        def host_rate(mode):
            dmx.dm_set_option(ctx, dmx.OPT_HOST_MODE, mode)
            hk.fill_(0)
            dmx.dm_sketch_host(ctx, hip, hix, hw, K_SLOTS, SEED, out_keys=hk, b=B_BITS, out_words=hwd)
            if not np.array_equal(hk.numpy(), ref_keys):
                raise RuntimeError("host-entry keys differ from the device-resident run")
            barrier(dist, True)
            t0 = time.perf_counter()
            for _ in range(e2e_steps):
                dmx.dm_sketch_host(ctx, hip, hix, hw, K_SLOTS, SEED, out_keys=hk, b=B_BITS, out_words=hwd)
            barrier(dist, True)
            return world * n * e2e_steps / max_over_ranks(dist, time.perf_counter() - t0, True)

        staged = host_rate(dmx.HOST_STAGED)
        in_place = host_rate(dmx.HOST_AUTO)          # the library default: page-locked arrays are used in place
        dmx.dm_set_option(ctx, dmx.OPT_HOST_MODE, dmx.HOST_AUTO)
        h2d = b.indptr.nbytes + b.indices.nbytes + b.weights.nbytes
        d2h = hk.numel() * 8 + hwd.numel() * 8
        e2e = {"value": in_place, "unit": "sets/s", "h2d_bytes_per_step": int(h2d),
               "d2h_bytes_per_step": int(d2h), "copies_declared": True,
               "transfer": "dm_sketch_host from page-locked host arrays; the kernels read the CSR and write the "
                           "keys and words through the host link inside the timed region (in place, the default)",
               "staged": {"value": staged, "unit": "sets/s",
                          "transfer": "chunked cudaMemcpyAsync to device buffers, overlapped with the kernels"}}
        del hip, hix, hw, hk, hwd

    # roofline of the dominant kernel of the step (integer issue; see the work model above)
    mean_launch_s = sum(per_launch_ms) / len(per_launch_ms) / 1e3
    ops = areas * OPS_PER_AREA + darts * OPS_PER_DART + kept * OPS_PER_KEPT
    out_bytes = keys.numel() * keys.element_size() + (outw.numel() * 8 if outw is not None else 0)
    sm_max = clocks.get("sm_max_mhz") or 2070.0
    peak_ops = props.multi_processor_count * INT_LANES_PER_SM * sm_max * 1e6
    achieved = ops / mean_launch_s
    tps = traffic_per_set(wl) if args.sets is None else None
    roofline = {"bound": "alu", "achieved": achieved / 1e9, "peak": peak_ops / 1e9, "unit": "Gop/s",
                "frac": achieved / peak_ops, "traffic": (tps * n if tps is not None else None),
                "traffic_source": (f"profiles/traffic_{wl.lower()}.json" if tps is not None else
                                   "none for the current kernel source"),
                "ops_per_launch": ops, "units_per_launch": {"areas": areas, "darts": darts, "kept": kept,
                                                            "passes": passes},
                "hbm_gbs_algorithmic": (b.indptr.nbytes + b.indices.nbytes + b.weights.nbytes
                                        + out_bytes) / mean_launch_s / 1e9,
                "peak_source": f"{props.multi_processor_count} SMs x {INT_LANES_PER_SM} int32 lanes x "
                               f"{sm_max:.0f} MHz (max SM clock)"}
    if full:
        roofline["peak_check"] = mix_ceiling(dmx, props, peak_ops, stream)
        roofline["peak_check"]["kernel_frac_of_ceiling"] = achieved / (roofline["peak_check"]["gop_per_s"] * 1e9)

    cpu_baseline = None
    if full and rank == 0 and world == 1 and not args.no_cpu_baseline and wl == "W1":
        cores = os.cpu_count() or 1
        v, ns, dt = time_oracle(b, 8000 * cores, cores)         # about 30 core-seconds
        v1, ns1, dt1 = time_oracle(b, 40000, 1)                 # about 10 seconds
        cpu_baseline = {"value": v, "unit": "sets/s", "cores": cores, "kind": "oracle",
                        "sample": f"first {ns} sets of W1 ({dt:.1f} s wall on {cores} threads)",
                        "single_thread": {"value": v1, "unit": "sets/s", "cores": 1,
                                          "sample": f"first {ns1} sets of W1 ({dt1:.1f} s wall on 1 thread)"}}
    # kernels per step: fast + general; the batched form adds classify, scan, scatter, a second
    # general launch (the fast kernel's deferrals) and, for sketches with a large-set threshold,
    # the block-per-set kernel; W3S adds the class kernel
    eff = tuning or {"form": form_id, "large_nnz": 2048 if args.large_nnz is None else args.large_nnz,
                     "large_work": 0}
    large_on = wl in ("W1", "W2") and (eff["large_nnz"] > 0 or eff["large_work"] > 0)
    launches_per_step = (2 if eff["form"] != dmx.FORM_BATCHED else 6 + (1 if large_on else 0)) \
        + (1 if wl == "W3S" else 0)
    ctx.close()
    return {"value": value, "t_max": t_max, "n": n, "kk": kk, "roofline": roofline, "plain_form": plain,
            "per_set_form": per_set,
            "e2e": e2e, "cpu_baseline": cpu_baseline, "clocks": clocks, "tuning": tuning,
            "gpu_launches": launches_per_step * args.steps, "wall_s_timed": t_wall}


def gpu_arm(args):
    import torch

    import paper_2005_11547_gb300 as dmx

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dist = dist_init(world, True)
    dmx.build()
    dmx.load()
    props = torch.cuda.get_device_properties(local)
    wl = args.workload
    r = measure(args, wl, local, dist, props, full=True)
    # the heavy-tailed batch (k = 1024) is part of the default run: its batched (autotuned,
    # graph) and plain forms are timed on the same GPU after the headline workload
    w2 = None
    if wl == "W1" and args.sets is None and not args.no_w2:
        import gc
        gc.collect()
        torch.cuda.empty_cache()
        r2 = measure(args, "W2", local, dist, props, full=False)
        w2 = {"workload": WL_DESC["W2"], "value": r2["value"], "unit": "sets/s",
              "ms_per_step": r2["t_max"] * 1e3 / args.steps, "minhashes_per_s": r2["value"] * 1024,
              "plain_form": r2["plain_form"], "per_set_form": r2["per_set_form"], "roofline": r2["roofline"],
              "tuning": r2["tuning"],
              "clocks": r2["clocks"], "gpu_launches": r2["gpu_launches"]}
    desc = dict(WL_DESC)
    desc["W3S"] = (f"W3 sets with each set's weight class normalised to ||x||_1 in [2^{args.norm_exp}, "
                   f"2^{args.norm_exp + 1}) (Section 3); (L, K) = (64, 8) LSH uint32 values")
    if rank == 0:
        line = {
            "metric": METRIC if wl == "W1" else f"weighted sets/s ({wl})",
            "value": r["value"], "unit": "sets/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": r["t_max"] * 1e3 / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "int64", "data": "synthetic",
            "minhashes_per_s": r["value"] * r["kk"],
            "config": {"workload": desc[wl] if args.sets is None else f"{wl} prefix of {r['n']} sets",
                       "n_sets": r["n"], "k": r["kk"], "b": B_BITS if wl == "W1" else None, "seed": SEED,
                       "form": args.form + ("" if args.no_graph else " + CUDA graph")
                               + (" + autotuned" if r["tuning"] else ""),
                       "l2": "inputs and outputs of a step are GBs, > 129 MB L2: no flush needed"},
            "roofline": r["roofline"], "cpu_baseline": r["cpu_baseline"], "e2e": r["e2e"], "clocks": r["clocks"],
            "plain_form": r["plain_form"], "per_set_form": r["per_set_form"], "tuning": r["tuning"],
            "gpu_launches": r["gpu_launches"] + (w2["gpu_launches"] if w2 else 0),
            "wall_s_timed": r["wall_s_timed"], "w2": w2,
        }
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


# ------------------------------------------------------------------------------------------
# W4: the serving loop on a request trace
# ------------------------------------------------------------------------------------------
def serve_arm(args):
    """Requests of one set each (nnz = min(1e5, floor(Pareto(1.2) + 1)), weights U(0, 5],
    d = 2^24, k uniform over {64, 256, 1024}) arriving as a Poisson process at 50,000/s, played in
    real time through dm_server_replay from host memory (copies in and out are part of every
    request's latency).  Reported: latency percentiles from arrival to result ready and the
    sustained rate at that load, the closed-loop capacity (all requests queued at once), and the
    same for the plain per-request form (one request per launch on one stream)."""
    import numpy as np
    import torch

    import paper_2005_11547_gb300 as dmx
    import workloads

    rank, world, local = dist_env()
    if rank != 0:
        return
    torch.cuda.set_device(local)
    dmx.build()
    dmx.load()
    arrivals, b, ks = workloads.workload4_requests(rate=50_000.0, seconds=args.duration)
    n = b.n_sets
    arr_ns = np.ascontiguousarray((arrivals - arrivals[0]) * 1e9, dtype=np.int64)
    seeds = np.full(n, SEED, dtype=np.uint64)
    ip = b.indptr

    def prefix(m):
        return np.ascontiguousarray(ip[: m + 1])

    # sample check: the server's keys equal dm_sketch's on the same rows (device entry, one call per k)
    m = min(n, 20000)
    srv = dmx.Server(local, lanes=4)
    out, _, st = srv.replay(prefix(m), b.indices, b.weights, ks[:m], seeds[:m], np.zeros(m, np.int64))
    srv.close()
    if np.any(st != 0):
        raise RuntimeError("serving sample: a request failed")
    ctx = dmx.dm_create(local)
    off = np.concatenate([[0], np.cumsum(ks[:m].astype(np.int64))])
    for k in (64, 256, 1024):
        sel = np.nonzero(ks[:m] == k)[0]
        sub = b.rows(sel)
        d_ip = torch.from_numpy(sub.indptr).cuda()
        d_ix = torch.from_numpy(sub.indices.view(np.int32)).cuda()
        d_w = torch.from_numpy(sub.weights).cuda()
        ref = dmx.dm_sketch(ctx, d_ip, d_ix, d_w, k, SEED).cpu().numpy().view(np.uint64)
        got = np.stack([out[off[i]:off[i + 1]] for i in sel])
        if not np.array_equal(got, ref):
            raise RuntimeError(f"serving sample: keys differ from dm_sketch (k={k})")
    ctx.close()

    def pct(lat_ns):
        v = np.sort(lat_ns) / 1e3
        return {"p50_us": float(np.percentile(v, 50)), "p99_us": float(np.percentile(v, 99)),
                "max_us": float(v[-1])}

    def run(per_request, lanes, m_open, m_closed):
        srv = dmx.Server(local, lanes=lanes, mem_budget_bytes=8 << 30, per_request=per_request)
        w0 = min(n, 3000)                                     # warm-up: lanes, contexts, kernels
        srv.replay(prefix(w0), b.indices, b.weights, ks[:w0], seeds[:w0], np.zeros(w0, np.int64), deliver=False)
        srv.reset_stats()
        sampler = ClockSampler(local)
        sampler.start()
        t0 = time.perf_counter()
        _, lat, st = srv.replay(prefix(m_open), b.indices, b.weights, ks[:m_open], seeds[:m_open],
                                arr_ns[:m_open], deliver=False)
        wall_open = time.perf_counter() - t0
        stats = srv.stats()
        srv.reset_stats()
        t0 = time.perf_counter()
        srv.replay(prefix(m_closed), b.indices, b.weights, ks[:m_closed], seeds[:m_closed],
                   np.zeros(m_closed, np.int64), deliver=False)
        wall_closed = time.perf_counter() - t0
        stats_closed = srv.stats()
        clocks = sampler.stop()
        srv.close()
        if np.any(st != 0):
            raise RuntimeError("serving run: a request failed")
        nnz = int(ip[m_open])
        return {"requests": m_open, "offered_per_s": 50_000.0, "sustained_per_s": m_open / wall_open,
                **pct(lat), "mean_batch": stats["mean_batch"], "batches": stats["batches"],
                "gpu_launches": stats["kernel_launches"] + stats_closed["kernel_launches"],
                "capacity_per_s": m_closed / wall_closed, "capacity_requests": m_closed,
                "h2d_bytes": 8 * (m_open + 1) + 8 * nnz, "d2h_bytes": 8 * int(ks[:m_open].astype(np.int64).sum()),
                "clocks": clocks}

    batched = run(False, 4, n, min(n, 500_000))
    plain = run(True, 1, min(n, 250_000), min(n, 100_000))
    line = {
        "metric": "W4 serving: requests/s sustained at 50,000/s Poisson arrivals (p50/p99 latency)",
        "value": batched["sustained_per_s"], "unit": "requests/s", "n_gpus": 1, "steps": 1, "warmup": 1,
        "ms_per_step": 1e3 * n / batched["sustained_per_s"], "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "int64", "data": "synthetic",
        "config": {"workload": f"W4: {n} requests over {args.duration:g} s (Poisson 50,000/s), nnz = min(1e5, "
                               "floor(Pareto(1.2)+1)), weights U(0,5], d=2^24, k uniform {64,256,1024}; 8 GiB "
                               "admission budget, 4 lanes", "l2": "host-resident trace; no reuse across requests"},
        "latency_us": {k: batched[k] for k in ("p50_us", "p99_us", "max_us")},
        "capacity_requests_per_s": batched["capacity_per_s"],
        "batched": batched, "plain_per_request": plain,
        "e2e": {"value": batched["sustained_per_s"], "unit": "requests/s",
                "h2d_bytes_per_step": batched["h2d_bytes"], "d2h_bytes_per_step": batched["d2h_bytes"]},
        "gpu_launches": batched["gpu_launches"], "clocks": batched["clocks"], "cpu_baseline": None, "roofline": None,
    }
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------------------------------
# CMP: similarity counts of sketches (dm_compare)
# ------------------------------------------------------------------------------------------
def compare_arm(args):
    """Row-aligned pairs of k = 256 key sketches (1,000,000 pairs: 4.1 GB read per step, HBM
    bound), plus the cross form of 2,048 query rows against 131,072 rows (k = 256 keys and 1-bit
    words).  Sketch values are random: the counts do not depend on where the keys came from."""
    import numpy as np
    import torch

    import paper_2005_11547_gb300 as dmx

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dist = dist_init(world, True)
    dmx.build()
    dmx.load()
    n, k = args.sets or 1_000_000, 256
    g = torch.Generator(device="cuda").manual_seed(5)
    a = torch.randint(-2 ** 62, 2 ** 62, (n, k), device="cuda", dtype=torch.int64, generator=g)
    c = a.clone()
    flip = torch.rand((n, k), device="cuda", generator=g) < 0.5
    c[flip] ^= 1 << 40
    out = torch.empty(n, dtype=torch.int32, device="cuda")
    ctx = dmx.dm_create(local)
    stream = torch.cuda.current_stream()
    for _ in range(max(3, args.warmup)):
        dmx.dm_compare(ctx, a, c, k, out=out, stream=stream)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    sampler = ClockSampler(local)
    sampler.start()
    barrier(dist, True)
    ev[0].record(stream)
    for _ in range(args.steps):
        dmx.dm_compare(ctx, a, c, k, out=out, stream=stream)
    ev[1].record(stream)
    barrier(dist, True)
    clocks = sampler.stop()
    t = max_over_ranks(dist, ev[0].elapsed_time(ev[1]) / 1e3, True)
    per = t / args.steps
    bytes_launch = 2 * n * k * 8 + n * 4
    peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))) if os.path.exists(
        os.path.join(ROOT, "MEASURED_PEAKS.json")) else {}
    hbm = peaks.get("hbm_gbs", 6800.0)
    value = sum_over_ranks(dist, float(n * args.steps), True) / t
    # cross form
    qa, qc = a[:2048].contiguous(), c[:131072].contiguous()
    cross = torch.empty((2048, 131072), dtype=torch.int32, device="cuda")
    dmx.dm_compare(ctx, qa, qc, k, cross=True, out=cross, stream=stream)
    e2 = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    e2[0].record(stream)
    for _ in range(3):
        dmx.dm_compare(ctx, qa, qc, k, cross=True, out=cross, stream=stream)
    e2[1].record(stream)
    torch.cuda.synchronize()
    cross_s = e2[0].elapsed_time(e2[1]) / 3e3
    wa = torch.randint(-2 ** 62, 2 ** 62, (2048, 4), device="cuda", dtype=torch.int64, generator=g)
    wc = torch.randint(-2 ** 62, 2 ** 62, (131072, 4), device="cuda", dtype=torch.int64, generator=g)
    dmx.dm_compare(ctx, wa, wc, k, bits=1, cross=True, out=cross, stream=stream)
    e2[0].record(stream)
    for _ in range(3):
        dmx.dm_compare(ctx, wa, wc, k, bits=1, cross=True, out=cross, stream=stream)
    e2[1].record(stream)
    torch.cuda.synchronize()
    cross1_s = e2[0].elapsed_time(e2[1]) / 3e3
    # top-10 neighbours of each query row among the 131,072 rows (dm_compare_topk), keys and 1-bit
    topk_s = {}
    for name, qq, cc, bits in (("keys", qa, qc, 0), ("one_bit", wa, wc, 1)):
        dmx.dm_compare_topk(ctx, qq, cc, k, 10, bits=bits, stream=stream)
        e2[0].record(stream)
        for _ in range(3):
            dmx.dm_compare_topk(ctx, qq, cc, k, 10, bits=bits, stream=stream)
        e2[1].record(stream)
        torch.cuda.synchronize()
        topk_s[name] = e2[0].elapsed_time(e2[1]) / 3e3
    ctx.close()
    if rank == 0:
        line = {
            "metric": "sketch pairs compared/s (k=256 uint64 keys, row-aligned pairs)", "value": value,
            "unit": "pairs/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": per * 1e3, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "int64", "data": "synthetic",
            "config": {"workload": f"CMP: {n} pairs of k=256 uint64 key rows (random, half the slots agreeing)",
                       "l2": "4.1 GB read per step, > 129 MB L2: no flush needed"},
            "roofline": {"bound": "hbm", "achieved": bytes_launch / per / 1e9, "peak": hbm, "unit": "GB/s",
                         "frac": bytes_launch / per / 1e9 / hbm, "traffic": None,
                         "peak_source": "MEASURED_PEAKS.json hbm_gbs" if peaks else "fallback 6.8 TB/s"},
            "cross": {"keys_pairs_per_s": 2048 * 131072 / cross_s, "one_bit_pairs_per_s": 2048 * 131072 / cross1_s,
                      "shape": "2,048 x 131,072 rows, k = 256"},
            "topk": {"k_neighbours": 10, "shape": "2,048 queries x 131,072 rows, k = 256",
                     "keys_queries_per_s": 2048 / topk_s["keys"], "keys_pairs_per_s": 2048 * 131072 / topk_s["keys"],
                     "one_bit_queries_per_s": 2048 / topk_s["one_bit"],
                     "one_bit_pairs_per_s": 2048 * 131072 / topk_s["one_bit"]},
            "cpu_baseline": None, "e2e": None, "clocks": clocks, "gpu_launches": args.steps,
        }
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


# ------------------------------------------------------------------------------------------
# IDX: LSH tables (dm_lsh_index_*) over the W3 LSH values
# ------------------------------------------------------------------------------------------
def index_arm(args):
    """Insert the (64, 8) LSH values of the 1,000,000 W3 sets into the tables, then query the
    values of 200,000 of them (each finds itself and its collisions), 64 candidates per query."""
    import numpy as np
    import torch

    import paper_2005_11547_gb300 as dmx
    import workloads

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dist = dist_init(world, True)
    dmx.build()
    dmx.load()
    b = workloads.workload3(args.sets or 1_000_000)
    n, L, m, cmax = b.n_sets, 64, min(b.n_sets, 200_000), 64
    ip = torch.from_numpy(b.indptr).cuda()
    ix = torch.from_numpy(b.indices.view(np.int32)).cuda()
    w = torch.from_numpy(b.weights).cuda()
    ctx = dmx.dm_create(local)
    vals = dmx.dm_lsh(ctx, ip, ix, w, L, 8, SEED)
    ctx.close()
    stream = torch.cuda.current_stream()
    q = vals[:m].contiguous()
    ins, qry = [], []
    sampler = ClockSampler(local)
    sampler.start()
    for step in range(args.warmup + args.steps):
        index = dmx.LshIndex(L, n, local)
        e = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
        barrier(dist, True)
        e[0].record(stream)
        index.insert(vals, stream=stream)
        e[1].record(stream)
        counts, ids = index.query(q, cmax, stream=stream)
        e[2].record(stream)
        torch.cuda.synchronize()
        if index.status() != 0:
            raise RuntimeError("index insertion error")
        if step >= args.warmup:
            ins.append(e[0].elapsed_time(e[1]) / 1e3)
            qry.append(e[1].elapsed_time(e[2]) / 1e3)
        index.close()
    clocks = sampler.stop()
    found = (ids[:, 0] >= 0).float().mean().item()
    raw = float(counts.clamp(min=0).sum().item())
    t_ins = max_over_ranks(dist, sum(ins) / len(ins), True)
    t_q = max_over_ranks(dist, sum(qry) / len(qry), True)
    peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))) if os.path.exists(
        os.path.join(ROOT, "MEASURED_PEAKS.json")) else {}
    hbm = peaks.get("hbm_gbs", 6800.0)
    # algorithmic bytes of the queries: values read, one key and one head per table, the ids of
    # the distinct candidates (a lower bound on the chain walk), counts and ids written
    qbytes = m * (L * 4 + L * 12 + 4 + cmax * 8) + raw * 12
    if rank == 0:
        line = {
            "metric": "LSH-index queries/s ((64, 8) values of W3 sets, 64 candidates per query)",
            "value": sum_over_ranks(dist, float(m), True) / t_q, "unit": "queries/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * (t_ins + t_q), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "int64", "data": "synthetic",
            "config": {"workload": f"IDX: {n} W3 sets' LSH values inserted, {m} of them queried",
                       "l2": "index of 1.5 GB per step, > 129 MB L2: no flush needed"},
            "insert_points_per_s": n / t_ins, "query_ms": t_q * 1e3, "insert_ms": t_ins * 1e3,
            "queries_with_a_candidate": found,
            "roofline": {"bound": "hbm", "achieved": qbytes / t_q / 1e9, "peak": hbm, "unit": "GB/s",
                         "frac": qbytes / t_q / 1e9 / hbm, "traffic": None,
                         "note": "random 32-byte sector accesses: latency-bound chains, not streaming"},
            "cpu_baseline": None, "e2e": None, "clocks": clocks, "gpu_launches": 2 * args.steps,
        }
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


T1_NORMS = [("1", 1.0), ("2^64", 2.0 ** 64), ("2^-64", 2.0 ** -64), ("2^512", 2.0 ** 512),
            ("2^-512", 2.0 ** -512)]


def wide_arm(args):
    """Table 1's workload through the wide-range entry: per norm, n sets of 1,024 elements on the
    simplex scaled to ||x||_1 (Section 4's recipe, 64-bit ids), k = 256.  A step sketches the
    whole batch (all norms) in one call; each norm is also timed alone."""
    import numpy as np
    import torch

    import paper_2005_11547_gb300 as dmx
    import workloads

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dist = dist_init(world, True)
    dmx.build()
    dmx.load()
    props = torch.cuda.get_device_properties(local)
    per, nnz, k = args.sets or 8000, 1024, K_SLOTS
    parts = [workloads.table1_batch(per, nnz, l1, 700 + i + 16 * rank) for i, (_, l1) in enumerate(T1_NORMS)]
    ip = torch.from_numpy(np.concatenate([[0]] + [p.indptr[1:] + nnz * per * i for i, p in enumerate(parts)])).cuda()
    ix = torch.from_numpy(np.concatenate([p.indices for p in parts]).view(np.int64)).cuda()
    w = torch.from_numpy(np.concatenate([p.weights for p in parts])).cuda()
    n = per * len(parts)
    out = torch.empty((n, k), dtype=torch.int64, device="cuda")
    stream = torch.cuda.current_stream()
    ctx = dmx.dm_create(local)

    # work counts of one launch (counting kernel variant, outside the timed region)
    cnt = torch.zeros(4, dtype=torch.int64, device="cuda")
    cctx = dmx.dm_create(local)
    dmx.dm_set_option(cctx, dmx.OPT_COUNTERS, cnt.data_ptr())
    dmx.dm_sketch_f64(cctx, ip, ix, w, k, SEED, out=out)
    dmx.dm_sync_status(cctx)
    areas, darts, kept, passes = [int(v) for v in cnt.cpu().tolist()]
    cctx.close()

    def timed(lo, hi, steps):
        sub_ip = ip[lo:hi + 1] if lo == 0 else (ip[lo:hi + 1] - ip[lo]).contiguous()
        e0 = ip[lo].item()
        sub_ix, sub_w = ix[e0:].contiguous() if lo else ix, w[e0:].contiguous() if lo else w
        sub_out = out[lo:hi]
        for _ in range(max(3, args.warmup)):
            dmx.dm_sketch_f64(ctx, sub_ip, sub_ix, sub_w, k, SEED, out=sub_out)
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
        barrier(dist, True)
        ev[0].record(stream)
        for _ in range(steps):
            dmx.dm_sketch_f64(ctx, sub_ip, sub_ix, sub_w, k, SEED, out=sub_out)
        ev[1].record(stream)
        barrier(dist, True)
        dmx.dm_sync_status(ctx)
        return ev[0].elapsed_time(ev[1]) / 1e3 / steps

    sampler = ClockSampler(local)
    sampler.start()
    t_step = timed(0, n, args.steps)
    clocks = sampler.stop()
    per_norm = {}
    for i, (name, _) in enumerate(T1_NORMS):
        t = timed(i * per, (i + 1) * per, max(1, min(args.steps, 3)))
        per_norm[name] = {"sets_per_s": per / t, "us_per_set_per_gpu": t / per * 1e6}
    t_max = max_over_ranks(dist, t_step, True)
    all_sets = sum_over_ranks(dist, float(n), True)
    ops = areas * OPS_PER_AREA + darts * OPS_PER_DART + kept * OPS_PER_KEPT
    sm_max = clocks.get("sm_max_mhz") or 2070.0
    peak_ops = props.multi_processor_count * INT_LANES_PER_SM * sm_max * 1e6
    if rank == 0:
        line = {
            "metric": "weighted sets/s (Table 1 norms, k=256 wide-range minhash keys, bit-exact)",
            "value": all_sets / t_max, "unit": "sets/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": t_max * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "int64", "data": "synthetic",
            "config": {"workload": f"T1: {per} sets per norm x 5 norms (1, 2^64, 2^-64, 2^512, 2^-512), "
                                   f"{nnz} distinct 64-bit ids per set, binary64 simplex weights scaled to the norm",
                       "k": k, "seed": SEED,
                       "l2": f"inputs {n * nnz * 16 / 1e6:.0f} MB per step, > 129 MB L2: no flush needed"},
            "per_norm": per_norm,
            "roofline": {"bound": "alu", "achieved": ops / t_step / 1e9, "peak": peak_ops / 1e9, "unit": "Gop/s",
                         "frac": ops / t_step / peak_ops, "traffic": None, "ops_per_launch": ops,
                         "units_per_launch": {"areas": areas, "darts": darts, "kept": kept, "passes": passes},
                         "peak_source": f"{props.multi_processor_count} SMs x {INT_LANES_PER_SM} int32 lanes x "
                                        f"{sm_max:.0f} MHz (max SM clock)"},
            "cpu_baseline": None, "e2e": None, "clocks": clocks, "gpu_launches": args.steps,
        }
        print(json.dumps(line), flush=True)
    ctx.close()
    if dist is not None:
        dist.destroy_process_group()


def main():
    args = parse()
    if args.impl == "reference":
        reference_arm(args)
    elif args.workload == "W4":
        serve_arm(args)
    elif args.workload == "CMP":
        compare_arm(args)
    elif args.workload == "IDX":
        index_arm(args)
    elif args.workload == "T1":
        wide_arm(args)
    else:
        gpu_arm(args)


if __name__ == "__main__":
    main()
