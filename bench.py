"""Benchmark: syndromes decoded per second by the GB300 blockBP decoder.

Workload (one step = one batch through the whole hot path): the distance-11
planar surface code under depolarizing noise p = 0.10, 10^4 seeded synthetic
syndromes per GPU, blockBP with 4x4-node blocks, bond D = 8, max-iter 20,
delta0 = 1e-4, delta1 = 1e-2, eta = 0.1 (Sec. IV parameters).  The headline
path is the FP32 kernel (tensors, QR and SVD in float; logs, Delta and the
read-out in double); the plain FP64 kernel is timed beside it on a subset.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

One JSON line is printed by rank 0.  Under torchrun every rank decodes its own
shot range (weak scaling); only the timing is reduced (max over ranks).
``--impl reference`` times the CPU FP64 oracle instead (rank 0 only).
"""

from __future__ import annotations

import argparse
import json
import math
import multiprocessing as mp
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import synth  # noqa: E402

METRIC = "syndromes decoded/s at d=11 p=0.10 D=8: learned+mixed vs plain FP64 GPU"
D_CODE, P_NOISE, K_BLOCK, D_BOND = 11, 0.10, 4, 8
MAX_ITER, DELTA0, DELTA1, ETA = 20, 1e-4, 1e-2, 0.1
SEED = synth.workload_seed(2, 2)        # d = 11 workload, p index 2 of {0.05, 0.08, 0.10, 0.13, 0.15}
WORKLOAD = (f"planar surface code d={D_CODE}, depolarizing p={P_NOISE:.2f}, blockBP k={K_BLOCK} "
            f"(4x4-node blocks), D={D_BOND}, max_iter={MAX_ITER}, delta0={DELTA0:g}, "
            f"delta1={DELTA1:g}, eta={ETA:g}")
N_SM = 152
SM_MAX_MHZ = 2070.0
# ALU peaks derived from unit counts: 128 FP32 FMA lanes per SM; FP64 at
# 1/64 of that (2 DFMA per clock per SM, the nominal 1.25 TFLOP/s of GB300).
FP32_FMA_PER_SM_CLK = 128
FP64_FMA_PER_SM_CLK = 2


def oracle_one(args):
    """Oracle decode of one shot (runs in a spawned worker)."""
    s, max_iter, delta0 = args
    from oracle import blockbp as bb
    P = bb.Params(d=D_CODE, k=K_BLOCK, D=D_BOND, p=P_NOISE, max_iter=max_iter, eta=ETA,
                  delta0=delta0, delta1=DELTA1)
    r = bb.decode(np.asarray(s, dtype=np.uint8), P)
    return r["stats"].flops, int(r["decision"]), [int(x) for x in r["iters"]]


def run_oracle_sample(first_shot: int, n: int, procs: int):
    """Decode n shots of the workload with the oracle on ``procs`` processes."""
    _, _, S = synth.sample_syndromes(SEED, first_shot, n, D_CODE, P_NOISE)
    ctx = mp.get_context("spawn")
    with ctx.Pool(procs) as pool:
        pool.map(int, range(procs))                 # workers up before the clock starts
        t0 = time.perf_counter()
        res = pool.map(oracle_one, [(S[b].tolist(), MAX_ITER, DELTA0) for b in range(n)], chunksize=1)
        dt = time.perf_counter() - t0
    return dt, res


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during a region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.idx), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (OSError, ValueError):
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def reference_arm(args):
    """CPU FP64 oracle timed on the host cores (rank 0 only)."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    procs = args.cpu_procs or min(os.cpu_count() or 1, 32)
    n = procs
    for w in range(args.warmup):
        run_oracle_sample(w * n, n, procs)
    times = []
    for s in range(args.steps):
        dt, _ = run_oracle_sample((args.warmup + s) * n, n, procs)
        times.append(dt)
    tot = sum(times)
    value = n * args.steps / tot
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "syndromes/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * tot / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "batch_per_step": n},
        "cpu_baseline": {"value": value, "unit": "syndromes/s", "cores": procs, "kind": "oracle",
                         "sample": f"{n} shots of the workload per step, one process per core"},
        "e2e": {"value": value, "unit": "syndromes/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def ours(args):
    import torch

    import paper_2402_04834_gb300 as pkg
    from paper_2402_04834_gb300 import _lib
    if not os.path.exists(_lib.LIB_PATH):
        from paper_2402_04834_gb300.build import build
        build()

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    B = args.batch
    prm = pkg.DecoderParams(d=D_CODE, k=K_BLOCK, D=D_BOND, p=P_NOISE, max_iter=MAX_ITER, eta=ETA,
                            delta0=DELTA0, delta1=DELTA1, precision=args.precision)
    first = rank * B
    _, _, S = synth.sample_syndromes(SEED, first, B, D_CODE, P_NOISE)
    S_host = torch.from_numpy(S).pin_memory()
    S_dev = S_host.to(dev)
    ws = pkg.Workspace()
    out = None
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream(dev)

    for _ in range(args.warmup):
        out = pkg.decode(S_dev, prm, workspace=ws, out=out)
    barrier()

    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    with ClockSampler(local) as clk:
        barrier()
        t0 = time.perf_counter()
        for i in range(args.steps):
            flush.fill_(float(i))                   # evict L2 before every step
            starts[i].record(stream)
            out = pkg.decode(S_dev, prm, workspace=ws, out=out)
            ends[i].record(stream)
        barrier()
        wall = time.perf_counter() - t0
    step_ms = [s.elapsed_time(e) for s, e in zip(starts, ends)]
    dev_ms = sum(step_ms)
    t = torch.tensor([dev_ms], dtype=torch.float64, device=dev)
    if dist is not None:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dev_ms_max = float(t.item())
    value = world * B * args.steps / (dev_ms_max / 1e3)
    iters_mean = float(out["iters"].double().mean().item())
    decisions = out["decision"].cpu().numpy()

    # End to end through the host entry point: H2D syndromes, decode, D2H results.
    hout = {"logp": np.empty((B, 4)), "delta": None, "iters": None, "flags": None,
            "decision": np.empty(B, dtype=np.int8)}
    hsyn = S_host.numpy()
    pkg.decode_host(hsyn, prm, workspace=ws, out=hout, device=dev)
    barrier()
    e2e_t = []
    for _ in range(args.steps):
        t1 = time.perf_counter()
        pkg.decode_host(hsyn, prm, workspace=ws, out=hout, device=dev)
        e2e_t.append(time.perf_counter() - t1)
    te = torch.tensor([sum(e2e_t)], dtype=torch.float64, device=dev)
    if dist is not None:
        dist.all_reduce(te, op=dist.ReduceOp.MAX)
    e2e_value = world * B * args.steps / float(te.item())

    # Plain FP64 GPU blockBP on a subset of the same workload.
    fp64 = None
    if args.fp64_batch > 0:
        B64 = min(args.fp64_batch, B)
        p64 = pkg.DecoderParams(d=D_CODE, k=K_BLOCK, D=D_BOND, p=P_NOISE, max_iter=MAX_ITER, eta=ETA,
                                delta0=DELTA0, delta1=DELTA1, precision="fp64")
        s64 = S_dev[:B64].contiguous()
        o64 = pkg.decode(s64, p64, workspace=ws)
        barrier()
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
        ms64 = 0.0
        for i in range(2):
            flush.fill_(float(i))
            ev[2 * i].record(stream)
            o64 = pkg.decode(s64, p64, workspace=ws, out=o64)
            ev[2 * i + 1].record(stream)
        barrier()
        ms64 = ev[0].elapsed_time(ev[1]) + ev[2].elapsed_time(ev[3])
        fp64_val = 2 * B64 / (ms64 / 1e3)
        agree = float(np.mean(o64["decision"].cpu().numpy() == decisions[:B64]))
        fp64 = {"value": fp64_val, "unit": "syndromes/s", "batch": B64,
                "mean_iters": float(o64["iters"].double().mean().item()),
                "decision_agreement_with_headline": agree,
                "headline_speedup": value / world / fp64_val}

    if rank != 0:
        if dist is not None:
            dist.destroy_process_group()
        return

    # Oracle on a bounded sample: CPU baseline and the algorithmic flop count.
    cpu = None
    flops_per_synd = None
    if args.cpu_baseline and world == 1:
        procs = args.cpu_procs or min(os.cpu_count() or 1, 32)
        dt, res = run_oracle_sample(0, procs, procs)
        flops_per_synd = float(np.mean([r[0] for r in res]))
        agree = float(np.mean([r[1] == int(decisions[i]) for i, r in enumerate(res)]))
        cpu = {"value": procs / dt, "unit": "syndromes/s", "cores": procs, "kind": "oracle",
               "sample": f"shots 0..{procs - 1} of the workload, one per process ({dt:.1f} s)",
               "decision_agreement": agree}

    fp = 1 if args.precision == "fp32" else 0
    per_clk = FP32_FMA_PER_SM_CLK if fp else FP64_FMA_PER_SM_CLK
    peak = 2.0 * per_clk * N_SM * SM_MAX_MHZ * 1e6 / 1e12
    roof = None
    if flops_per_synd is not None:
        kern_s = (dev_ms / args.steps) / 1e3
        achieved = flops_per_synd * B / kern_s / 1e12
        roof = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "frac": achieved / peak, "traffic": None,
                "kernel": "decode_kernel", "peak_source": ("FP32 FMA lanes x 2 x SMs x max clock"
                                                          if fp else "FP64 DFMA/clk/SM x 2 x SMs x max clock"),
                "flops_per_syndrome": flops_per_synd}

    line = {
        "metric": METRIC, "value": value, "unit": "syndromes/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": dev_ms_max / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32" if fp else "f64",
        "data": "synthetic: seeded i.i.d. depolarizing errors (SplitMix64 counter RNG) and their syndromes",
        "config": {"workload": WORKLOAD, "batch_per_gpu": B, "precision": args.precision,
                   "l2": "256 MB buffer written before every timed step; message arena larger than L2",
                   "mean_iters": iters_mean, "wall_s": wall},
        "clocks": clk.summary(),
        "e2e": {"value": e2e_value, "unit": "syndromes/s", "h2d_bytes_per_step": int(B * S.shape[1]),
                "d2h_bytes_per_step": int(B * (1 + 32))},
        "gpu_launches": 2 * args.steps,
        "roofline": roof, "cpu_baseline": cpu, "fp64_gpu": fp64,
    }
    print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--batch", type=int, default=10000)
    ap.add_argument("--precision", default="fp32", choices=["fp32", "fp64"])
    ap.add_argument("--fp64-batch", type=int, default=1024)
    ap.add_argument("--cpu-procs", type=int, default=0)
    ap.add_argument("--no-cpu-baseline", dest="cpu_baseline", action="store_false")
    args = ap.parse_args()
    if args.impl == "reference":
        reference_arm(args)
    else:
        ours(args)


if __name__ == "__main__":
    main()
