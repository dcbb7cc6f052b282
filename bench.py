"""Benchmark: syndromes decoded per second by the GB300 blockBP decoder.

Workload (one step = one batch through the whole hot path): the distance-11
planar surface code under depolarizing noise p = 0.10, 10^4 seeded synthetic
syndromes per GPU, blockBP with 4x4-node blocks, max-iter 20, delta0 = 1e-4,
delta1 = 1e-2, eta = 0.1 (Sec. IV parameters), D = 8 for the MPS form.
The headline decoder is the learned + mixed-precision one: features of
the distinct message rows (as bits), the warm-start network on the tensor
cores (trained first, untimed, on converged messages of seeded decodes)
and the expansion of its proposals to every coset, then the fused-block
form of Remark 9 (the form the paper ran for k = 4) in FP32 with an FP64
read-out, started from the proposals.  Timed beside it on the same
batch: the same decoder from the uniform start (cold), the plain FP64
blockBP in the fused form (the like-for-like denominator of the metric:
same algorithm, same results), the FP64 MPS form (a change of algorithm
as well as of precision, reported under its own label) and the FP32 MPS
form; then a mixed-distance batch (4096 syndromes,
d in {7, 9, 13, 17, 21}) in one autotuned persistent launch replayed from
a CUDA graph, against one launch per distance.  ``--no-warm`` makes the
cold decoder the headline.

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
SM_MAX_MHZ = 2070.0
# ALU peaks derived from unit counts: 128 FP32 FMA lanes per SM; FP64 at
# 1/64 of that (2 DFMA per clock per SM, the nominal 1.25 TFLOP/s of GB300).
FP32_FMA_PER_SM_CLK = 128
FP64_FMA_PER_SM_CLK = 2
# Warm-start network: 256 -> 256 -> 256 -> 16, two flops per multiply-add.
MLP_FLOPS_PER_ROW = 2 * (256 * 256 + 256 * 256 + 256 * 16)
# DRAM bytes read + written per unit, from ncu captures (dram__bytes_read.sum
# + dram__bytes_write.sum) of the current kernels at d = 11 (4 cosets per
# CTA, the register-form-only variant sized for 4 CTAs per SM).  The timed
# launches of the benchmark step (one-pass capture of the NVTX range
# "timed", 10^4 syndromes, mean of its two launches): the decode from the
# network's proposals moved 310.29 MB + 1.35 MB (it reads every proposed
# message: 4 cosets x 120 messages x 16 floats per syndrome), the network
# kernel fed by feature bits 55.78 MB + 39.71 MB for its 1.54 M rows.  The
# decode from the uniform start moved 362.0 KB + 0 for 1024 syndromes.
FUSED_DRAM_BYTES_PER_SYNDROME_WARM = (310.29e6 + 1.35e6) / 10000
FUSED_DRAM_BYTES_PER_SYNDROME = (361.984e3 + 0.0) / 1024
NETWORK_DRAM_BYTES_PER_ROW = (55.78e6 + 39.71e6) / 1540000


def oracle_one(args):
    """Oracle decode of one shot (runs in a spawned worker).

    ``fused`` selects the dense fused-block oracle (Remark 9), otherwise the
    MPS blockBP oracle; both apply the decision rule of Algorithm 1."""
    s, max_iter, delta0, algorithm = args
    s = np.asarray(s, dtype=np.uint8)
    from oracle import blockbp as bb
    if algorithm == "fused":
        from oracle.lattice import Lattice
        from oracle.naive import run_naive
        from oracle.tn import coset_network
        lat = Lattice(D_CODE)
        lp, dl, its = [], [], []
        for L in range(4):
            a, b, it, _ = run_naive(coset_network(lat, s, L, P_NOISE), K_BLOCK, max_iter, ETA, delta0)
            lp.append(a)
            dl.append(b)
            its.append(it)
        flags = [0 if x < DELTA1 else 1 for x in dl]
        return None, int(bb.decide(lp, dl, flags)), its, [float(x) for x in lp]
    P = bb.Params(d=D_CODE, k=K_BLOCK, D=D_BOND, p=P_NOISE, max_iter=max_iter, eta=ETA,
                  delta0=delta0, delta1=DELTA1)
    r = bb.decode(s, P)
    return r["stats"].flops, int(r["decision"]), [int(x) for x in r["iters"]], [float(x) for x in r["logp"]]


def run_oracle_sample(first_shot: int, n: int, procs: int, algorithm: str):
    """Decode n shots of the workload with the oracle on ``procs`` processes."""
    _, _, S = synth.sample_syndromes(SEED, first_shot, n, D_CODE, P_NOISE)
    ctx = mp.get_context("spawn")
    with ctx.Pool(procs) as pool:
        pool.map(int, range(procs))                 # workers up before the clock starts
        t0 = time.perf_counter()
        res = pool.map(oracle_one, [(S[b].tolist(), MAX_ITER, DELTA0, algorithm) for b in range(n)],
                       chunksize=1)
        dt = time.perf_counter() - t0
    return dt, res


# Multiply-adds of the 4 x 4 register form per (row, coset): column 0's two
# butterflies 6; per upper leg a0 of column 0 (two): column 1's upper-qubit
# butterflies 4 and lower-qubit products 4, the upper side message's
# entries 4, column 2's butterflies and data column 16; the lower side
# message's data column 8; column 3 6.  Only the entries with column 3's
# upper leg e equal to the row's bit r0 (the check at its top ties them)
# are formed.
REGISTER_FORM_MADDS = 76


def fused_flops(d: int, k: int):
    """Algorithmic arithmetic of the fused-block update (multiply-adds count 2), per coset.

    Returns (per BP iteration, read-out).  A 4 x 4 block counts the register
    form of its update (see the kernel); every other block is contracted
    towards each neighbour in the kernel's order: per column, the side message's data
    column (a dense contraction over the legs recorded so far), then the
    column's nodes, then the closing sums of the other side message.  Only
    the qubit nodes do arithmetic: their tensor pi(f + (x, z)) is a 2 x 2
    XOR convolution, four multiply-adds per entry of the state.  Check nodes
    are copy tensors (Sec. III.A): they move entries and cost nothing.  Then
    normalisation, damping and overlaps per message, and the Lemma 1
    read-out (4 x 4 blocks in register form; the others node by node with
    per-column renormalisation; closing dots, edge overlaps)."""
    W = 2 * d - 1
    rng = [(a, min(a + k, W)) for a in range(0, W, k)]
    nb = len(rng)

    def sweep(qubits_per_col, h, has_a, has_b, readout):
        nc = len(qubits_per_col)
        fl = 0.0
        ab = bb = 0
        sd, nf = nc >> 1, nc - (nc >> 1) - 1
        for t in range(nc):
            nab = 0 if not has_a else (ab + 1 if t < sd else (nf if t == sd else ab - 1))
            size = 2 ** (nab + h + bb + 1)
            if has_a and t == sd:
                fl += 2.0 * size * 2 ** ab
            ab = nab
            fl += qubits_per_col[t] * 8.0 * size
            nbb = 0 if not has_b else (bb + 1 if t < sd else (nf if t == sd else bb - 1))
            size_b = 2 ** (ab + h + nbb)
            if has_b and t == sd:
                fl += 2.0 * size_b * 2 ** (bb + 1)
            elif has_b and t > sd:
                fl += 1.0 * size_b
            bb = nbb
            if readout:
                fl += 3.0 * 2 ** (ab + h + bb)
        return fl

    def qubits(lines):
        # lines: the grid positions of each swept column, in sweep order
        return [sum(1 for (i, j) in col if (i + j) % 2 == 0) for col in lines]

    per_iter = 0.0
    readout = 0.0
    for I in range(nb):
        for J in range(nb):
            r0, r1 = rng[I]
            c0, c1 = rng[J]
            rows, cols = range(r0, r1), range(c0, c1)
            for dr, (di, dj) in enumerate(((0, 1), (0, -1), (1, 0), (-1, 0))):
                if not (0 <= I + di < nb and 0 <= J + dj < nb):
                    continue
                if dr < 2:      # right / left: columns of the block, left to right or back
                    order = cols if dr == 0 else reversed(cols)
                    lines = [[(i, j) for i in rows] for j in order]
                    h, ha, hb = r1 - r0, I > 0, I + 1 < nb
                else:           # down / up: rows of the block, top to bottom or back
                    order = rows if dr == 2 else reversed(rows)
                    lines = [[(i, j) for j in cols] for i in order]
                    h, ha, hb = c1 - c0, J > 0, J + 1 < nb
                if h == 4 and len(lines) == 4:
                    # 4 x 4 blocks: the register form of the update (butterflies
                    # over single row bits, side messages contracted where their
                    # legs enter), 76 multiply-adds per (row, coset) entry
                    # whichever node column 0 starts with (a chain starting with
                    # a check is read bottom to top).
                    per_iter += 2.0 * 16 * REGISTER_FORM_MADDS + 12.0 * 2 ** h
                else:
                    per_iter += sweep(qubits(lines), h, ha, hb, False) + 12.0 * 2 ** h
                if dr in (0, 2):
                    readout += 2.0 * 2 ** h
            lines = [[(i, j) for i in rows] for j in cols]
            if r1 - r0 == 4 and c1 - c0 == 4:      # the read-out's register form, then the closing dot
                readout += 2.0 * 16 * REGISTER_FORM_MADDS + 2.0 * 16
            else:
                readout += sweep(qubits(lines), r1 - r0, I > 0, I + 1 < nb, True) + 2.0 * 2 ** (r1 - r0)
    return per_iter, readout


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


MIXED_DISTANCES = (7, 9, 13, 17, 21)


def mixed_batch_leg(args, dev, pkg):
    """Batching: ``args.mixed_batch`` syndromes of distances drawn uniformly
    from MIXED_DISTANCES (p = 0.10, k = 4) in one persistent launch, launch
    shape from the autotuner, captured in a CUDA graph and replayed; against
    one launch per distance on the same syndromes.  Group j (distance
    MIXED_DISTANCES[j]) holds consecutive shots of seed workload_seed(3, j);
    the batch is packed in a seeded random order."""
    import torch

    from paper_2402_04834_gb300 import autotune
    from paper_2402_04834_gb300.decoder import decode_mixed, pack_mixed
    n = args.mixed_batch
    rng = np.random.default_rng(synth.workload_seed(3, 9))
    counts = np.bincount(rng.integers(0, len(MIXED_DISTANCES), size=n), minlength=len(MIXED_DISTANCES))
    shots, ds = [], []
    for j, (d, c) in enumerate(zip(MIXED_DISTANCES, counts)):
        if c:
            _, _, S = synth.sample_syndromes(synth.workload_seed(3, j), 0, int(c), d, P_NOISE)
            shots += list(S)
            ds += [d] * int(c)
    perm = rng.permutation(n)
    shots = [shots[i] for i in perm]
    ds = np.asarray(ds)[perm]
    packed, offsets, d_of = pack_mixed(shots, device=dev)
    prm = pkg.DecoderParams(d=0, k=K_BLOCK, p=P_NOISE, max_iter=MAX_ITER, eta=ETA, delta0=DELTA0, delta1=DELTA1,
                            precision="fp32", algorithm="fused")
    # Every distance here is odd, so the register-form-only kernels are candidates too.
    lean = ((8, 4, 3), (8, 2, 3)) if all(d % 2 == 1 for d in MIXED_DISTANCES) else ()
    prm, table = autotune.tune_mixed(packed, offsets, d_of, prm,
                                     shapes=lean + ((8, 4, 1), (8, 4, 2), (8, 2, 1), (8, 2, 2), (4, 2, 1), (4, 4, 1)),
                                     ctas=(0, 1, 2))
    order = torch.argsort(d_of, descending=True, stable=True).to(torch.int32)
    d_max = int(max(MIXED_DISTANCES))
    counter = torch.empty(256 + pkg.workspace_bytes(pkg.DecoderParams(**{**prm.__dict__, "d": d_max}), n),
                          dtype=torch.uint8, device=dev)
    out = decode_mixed(packed, offsets, d_of, prm, counter=counter, order=order, d_max=d_max)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    side = torch.cuda.Stream(dev)
    side.wait_stream(torch.cuda.current_stream(dev))
    with torch.cuda.stream(side):
        with torch.cuda.graph(g, stream=side):
            decode_mixed(packed, offsets, d_of, prm, counter=counter, order=order, d_max=d_max, out=out,
                         stream=side)
    torch.cuda.current_stream(dev).wait_stream(side)
    torch.cuda.synchronize()
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    reps, ms = 3, 0.0
    for i in range(reps):
        flush.fill_(float(i))
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        g.replay()
        b.record()
        torch.cuda.synchronize()
        ms += a.elapsed_time(b)
    mixed_val = reps * n / (ms / 1e3)
    # One launch per distance (default shapes), the same syndromes.
    groups = [(d, np.nonzero(ds == d)[0]) for d in MIXED_DISTANCES]
    dev_groups = [(d, idx, torch.from_numpy(np.stack([shots[i] for i in idx])).to(dev)) for d, idx in groups
                  if len(idx)]
    outs = {}
    for d, idx, S in dev_groups:
        outs[d] = pkg.decode(S, pkg.DecoderParams(**{**prm.__dict__, "d": d, "warps": 0, "cosets": 0,
                                                     "ctas_per_sm": 0, "messages": 0}))
    torch.cuda.synchronize()
    ms2 = 0.0
    for i in range(reps):
        flush.fill_(float(i))
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        for d, idx, S in dev_groups:
            pkg.decode(S, pkg.DecoderParams(**{**prm.__dict__, "d": d, "warps": 0, "cosets": 0, "ctas_per_sm": 0,
                                               "messages": 0}), out=outs[d])
        b.record()
        torch.cuda.synchronize()
        ms2 += a.elapsed_time(b)
    per_d_val = reps * n / (ms2 / 1e3)
    dec = out["decision"].cpu().numpy()
    agree = float(np.mean(np.concatenate([dec[idx] == outs[d]["decision"].cpu().numpy()
                                          for d, idx, _ in dev_groups])))
    return {"value": mixed_val, "unit": "syndromes/s", "batch": n, "distances": list(MIXED_DISTANCES),
            "counts": [int(c) for c in counts], "p": P_NOISE, "precision": "fp32", "algorithm": "fused",
            "launch": "one persistent launch, largest distance first, replayed from a CUDA graph",
            "shape": {"warps": prm.warps, "cosets": prm.cosets,
                      "messages": {1: "shared", 2: "workspace", 3: "shared, register form only"}[prm.messages],
                      "ctas_per_sm": prm.ctas_per_sm},
            "autotune_candidates": len(table),
            "mean_iters": float(out["iters"].double().mean().item()),
            "per_distance_launches": {"value": per_d_val, "unit": "syndromes/s", "launches": len(dev_groups)},
            "speedup_vs_per_distance": mixed_val / per_d_val, "decision_agreement_with_per_distance": agree}


def reference_arm(args):
    """CPU FP64 oracle timed on the host cores (rank 0 only)."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    procs = args.cpu_procs or min(os.cpu_count() or 1, 32)
    n = procs
    for w in range(args.warmup):
        run_oracle_sample(w * n, n, procs, args.algorithm)
    times = []
    for s in range(args.steps):
        dt, _ = run_oracle_sample((args.warmup + s) * n, n, procs, args.algorithm)
        times.append(dt)
    tot = sum(times)
    value = n * args.steps / tot
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "syndromes/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * tot / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "batch_per_step": n, "algorithm": args.algorithm},
        "cpu_baseline": {"value": value, "unit": "syndromes/s", "cores": procs, "kind": "oracle",
                         "sample": f"{n} shots of the workload per step, one process per core, "
                                   f"{'dense fused-block' if args.algorithm == 'fused' else 'MPS'} oracle"},
        "e2e": {"value": value, "unit": "syndromes/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def ours(args):
    import torch

    import paper_2402_04834_gb300 as pkg
    from paper_2402_04834_gb300 import _lib
    from paper_2402_04834_gb300 import warmstart as wsm
    from paper_2402_04834_gb300.sharding import reduce_max, shot_range
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
                            delta0=DELTA0, delta1=DELTA1, precision=args.precision,
                            algorithm=args.algorithm)
    first, _ = shot_range(rank, world, B)
    _, _, S = synth.sample_syndromes(SEED, first, B, D_CODE, P_NOISE)
    S_host = torch.from_numpy(S).pin_memory()
    S_dev = S_host.to(dev)
    ws = pkg.Workspace()
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream(dev)
    learned = args.warm and args.algorithm == "fused"

    # The learned warm start is trained first, untimed, on converged messages
    # of seeded d = 11 and d = 15 decodes at p in [0.05, 0.15].
    net, train_info = None, None
    if learned:
        t_w = time.perf_counter()
        Ftr, Ttr, Ltr = wsm.build_training_set(device=dev)
        net = wsm.WarmStart(device=dev, seed=0)
        hist = net.train(Ftr, Ttr, Ltr, epochs=12, batch=8192, lr=3e-3)
        hist += net.train(Ftr, Ttr, Ltr, epochs=8, batch=8192, lr=5e-4, seed=1)
        torch.cuda.synchronize()
        train_info = {"training_rows": int(Ftr.shape[0]), "train_s": time.perf_counter() - t_w,
                      "final_loss": hist[-1]}
        del Ftr, Ttr, Ltr

    # One step = the whole decoder over the batch.  Learned: features of the
    # distinct message rows (cosets that agree on the logical strings a
    # message's window sees share its row) -> tensor-core network ->
    # expansion to every (coset, message) -> fused decode from the
    # proposals; events around the network and around the decode kernel.
    M = wsm.message_count(prm)
    rows = B * (wsm.message_classes(prm)[1].numel() if learned else 4 * M)
    ev_mlp = []
    ev_dec = []

    def step(out, record=False):
        if not learned:
            a = torch.cuda.Event(enable_timing=True) if record else None
            b = torch.cuda.Event(enable_timing=True) if record else None
            if record:
                a.record(stream)
            out = pkg.decode(S_dev, prm, workspace=ws, out=out)
            if record:
                b.record(stream)
                ev_dec.append((a, b))
            return out
        evs = [torch.cuda.Event(enable_timing=True) for _ in range(4)] if record else None
        bits, lens = wsm.feature_bits_rows(S_dev, prm)
        if record:
            evs[0].record(stream)
        init = wsm.expand_rows(net.infer_bits(bits, lens, prm.p, alpha=wsm.DEFAULT_ALPHA), B, prm)
        if record:
            evs[1].record(stream)
            evs[2].record(stream)
        out = wsm.decode_ex(S_dev, prm, init_msgs=init, out=out)
        if record:
            evs[3].record(stream)
            ev_mlp.append((evs[0], evs[1]))
            ev_dec.append((evs[2], evs[3]))
        return out

    out = None
    for _ in range(args.warmup):
        out = step(out)
    barrier()

    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    with ClockSampler(local) as clk:
        barrier()
        torch.cuda.nvtx.range_push("timed")        # lets a profiler select the timed steps
        t0 = time.perf_counter()
        for i in range(args.steps):
            flush.fill_(float(i))                   # evict L2 before every step
            starts[i].record(stream)
            out = step(out, record=True)
            ends[i].record(stream)
        barrier()
        wall = time.perf_counter() - t0
        torch.cuda.nvtx.range_pop()
    step_ms = [s.elapsed_time(e) for s, e in zip(starts, ends)]
    dev_ms = sum(step_ms)
    dev_ms_max = reduce_max(dev_ms, dist, dev)
    value = world * B * args.steps / (dev_ms_max / 1e3)
    dec_ms = sum(a.elapsed_time(b) for a, b in ev_dec) / args.steps
    mlp_ms = sum(a.elapsed_time(b) for a, b in ev_mlp) / args.steps if ev_mlp else None
    iters_mean = float(out["iters"].double().mean().item())
    decisions = out["decision"].cpu().numpy()

    # End to end through the public API with host buffers: H2D syndromes,
    # the decoder, D2H decisions and log P, every step.
    hsyn = S_host
    e2e_t = []
    if learned:
        hout = wsm.decode_warm_host(hsyn, prm, net)
        barrier()
        for _ in range(args.steps):
            t1 = time.perf_counter()
            wsm.decode_warm_host(hsyn, prm, net, out=hout)
            e2e_t.append(time.perf_counter() - t1)
    else:
        hout = {"logp": np.empty((B, 4)), "delta": None, "iters": None, "flags": None,
                "decision": np.empty(B, dtype=np.int8)}
        pkg.decode_host(hsyn.numpy(), prm, workspace=ws, out=hout, device=dev)
        barrier()
        for _ in range(args.steps):
            t1 = time.perf_counter()
            pkg.decode_host(hsyn.numpy(), prm, workspace=ws, out=hout, device=dev)
            e2e_t.append(time.perf_counter() - t1)
    e2e_value = world * B * args.steps / reduce_max(sum(e2e_t), dist, dev)

    # Comparison legs on the same batch: cold start (uniform messages,
    # Remark 2), the plain FP64 blockBP with MPS messages (the denominator of
    # the metric) and the other combinations.
    outs_kept = {}

    def leg(alg, prec, nshots, cold=False):
        if nshots <= 0:
            return None
        nshots = min(nshots, B)
        pp = pkg.DecoderParams(d=D_CODE, k=K_BLOCK, D=D_BOND, p=P_NOISE, max_iter=MAX_ITER, eta=ETA,
                               delta0=DELTA0, delta1=DELTA1, precision=prec, algorithm=alg)
        sub = S_dev[:nshots].contiguous()
        o = pkg.decode(sub, pp, workspace=ws)
        barrier()
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
        for i in range(2):
            flush.fill_(float(i))
            ev[2 * i].record(stream)
            o = pkg.decode(sub, pp, workspace=ws, out=o)
            ev[2 * i + 1].record(stream)
        barrier()
        ms = ev[0].elapsed_time(ev[1]) + ev[2].elapsed_time(ev[3])
        val = 2 * nshots / (ms / 1e3)
        outs_kept[(alg, prec)] = o
        agree = float(np.mean(o["decision"].cpu().numpy() == decisions[:nshots]))
        return {"value": val, "unit": "syndromes/s", "batch": nshots, "algorithm": alg, "precision": prec,
                "mean_iters": float(o["iters"].double().mean().item()),
                "decision_agreement_with_headline": agree, "headline_speedup": value / world / val}

    cold = leg("fused", args.precision, B) if learned else None
    mixed = mixed_batch_leg(args, dev, pkg) if args.mixed_batch > 0 and args.algorithm == "fused" else None
    # The metric's denominator, like for like: the same algorithm (the fused
    # form of Remark 9, which gives the same results at this workload) in
    # FP64.  The MPS form in FP64 also changes the algorithm; it is reported
    # separately with that label.
    fp64_fused = leg("fused", "fp64", args.other_batch)
    legs = {"fp64_mps": leg("mps", "fp64", args.fp64_batch),
            "fp32_mps": leg("mps", "fp32", args.other_batch // 4)}
    if legs["fp64_mps"] is not None:
        legs["fp64_mps"]["label"] = ("MPS messages (Sec. III.D) in FP64: a different algorithm and precision "
                                     "from the headline, not its like-for-like denominator")
    speedup = None
    if fp64_fused is not None:
        speedup = {"like_for_like": value / world / fp64_fused["value"],
                   "denominator": "fused-block blockBP (Remark 9) in FP64, same shots, same results",
                   "target": 10.0,
                   "met": value / world / fp64_fused["value"] >= 10.0}
        if legs["fp64_mps"] is not None:
            speedup["vs_fp64_mps_change_of_algorithm"] = value / world / legs["fp64_mps"]["value"]

    if rank != 0:
        if dist is not None:
            dist.destroy_process_group()
        return

    # Oracle on a bounded sample of the same workload: the CPU baseline.
    cpu = None
    if args.cpu_baseline and world == 1:
        procs = args.cpu_procs or min(os.cpu_count() or 1, 32)
        # About 200 shots of the dense oracle (10-30 s on the host cores); the
        # MPS oracle is far slower, so one shot per process there.
        n_cpu = procs * max(1, -(-200 // procs)) if args.algorithm == "fused" else procs
        dt, res = run_oracle_sample(0, n_cpu, procs, args.algorithm)
        agree = float(np.mean([r[1] == int(decisions[i]) for i, r in enumerate(res)]))
        # Parity of the GPU decoder on these shots, element by element: the
        # cold-start FP32 decoder (the oracle starts cold) against the FP64
        # oracle.  Both exit at Delta < delta0, so a coset whose Delta sits
        # within rounding of delta0 may stop one iteration apart.
        ref = outs_kept.get(("fused", args.precision)) if learned else out
        parity = None
        if ref is not None and args.algorithm == "fused":
            got = ref["logp"][:n_cpu].cpu().numpy()
            err = np.abs(got - np.array([r[3] for r in res]))
            parity = {"max_abs_dlogp": float(err.max()), "n_cosets": int(err.size),
                      "n_above_1e-3": int((err > 1e-3).sum()),
                      "gpu_leg": "fused FP32 cold start", "oracle": "dense fused-block FP64"}
        cpu = {"value": n_cpu / dt, "unit": "syndromes/s", "cores": procs, "kind": "oracle",
               "sample": (f"shots 0..{n_cpu - 1} of the workload on {procs} processes ({dt:.1f} s), "
                          f"{'dense fused-block' if args.algorithm == 'fused' else 'MPS'} oracle, cold start"),
               "decision_agreement": agree, "parity": parity}

    # Roofline of the dominant kernel (the fused decode): its arithmetic per
    # launch over its event-timed duration; and of the network on the tensor cores.
    fp = 1 if args.precision == "fp32" else 0
    per_clk = FP32_FMA_PER_SM_CLK if fp else FP64_FMA_PER_SM_CLK
    n_sm = torch.cuda.get_device_properties(dev).multi_processor_count
    clocks = clk.summary()
    sm_mhz = clocks["sm_max_mhz"] or SM_MAX_MHZ
    peak = 2.0 * per_clk * n_sm * sm_mhz * 1e6 / 1e12
    roof = roof_mlp = None
    if args.algorithm == "fused":
        f_it, f_ro = fused_flops(D_CODE, K_BLOCK)
        flops = float(out["iters"].double().sum().item()) * f_it + B * 4 * f_ro
        achieved = flops / (dec_ms / 1e3) / 1e12
        warm_launch = mlp_ms is not None            # the decode reads the network's proposals
        per_syn = FUSED_DRAM_BYTES_PER_SYNDROME_WARM if warm_launch else FUSED_DRAM_BYTES_PER_SYNDROME
        traffic = per_syn * B
        roof = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "frac": achieved / peak, "traffic": traffic, "kernel": "fused_kernel",
                "traffic_source": ("ncu DRAM bytes of the timed 10^4-syndrome launch reading the proposals, "
                                   "per syndrome, scaled to the batch" if warm_launch else
                                   "ncu DRAM bytes of a 1024-syndrome launch from the uniform start, "
                                   "scaled to the batch"),
                "launch_ms": dec_ms,
                "peak_source": (f"derived: {per_clk} {'FP32 lanes' if fp else 'FP64 FMA/clk'} per SM x 2 x "
                                f"{n_sm} SMs x {sm_mhz:.0f} MHz (max SM clock)"),
                "flop_model": "4x4 blocks: the multiply-adds of the register form (76 per row and "
                              "coset); other blocks: qubit nodes as 2x2 XOR convolutions (4 multiply-adds "
                              "per state entry), check nodes as zero-flop copy tensors, side-message data "
                              "columns; normalise/damp/overlap; Lemma 1 read-out (register form for 4x4 blocks)",
                "flops_per_syndrome": flops / B}
    if mlp_ms is not None:
        bf16_peak, src = 1900.0, "fallback"
        try:
            with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
                bf16_peak, src = float(json.load(f)["bf16_tflops"]), "measured (burst)"
        except (OSError, KeyError, ValueError):
            pass
        mf = rows * MLP_FLOPS_PER_ROW / (mlp_ms / 1e3) / 1e12
        roof_mlp = {"bound": "tensor", "achieved": mf, "peak": bf16_peak, "unit": "TFLOP/s", "frac": mf / bf16_peak,
                    "traffic": None if NETWORK_DRAM_BYTES_PER_ROW is None else NETWORK_DRAM_BYTES_PER_ROW * rows,
                    "traffic_source": ("ncu DRAM bytes of the timed 1.54 M-row launch, scaled to the step's rows"
                                       if NETWORK_DRAM_BYTES_PER_ROW is not None else
                                       "no capture of the current kernel"),
                    "kernel": "mlp_tc_kernel (+ weight preparation and the expansion to every coset)",
                    "launch_ms": mlp_ms,
                    "rows": rows, "peak_source": src}

    # Learned warm start against cold start on the same shots: iterations and
    # the logical error rate (Wilson 95 % intervals).
    learned_info = None
    if learned and world == 1:
        ev = wsm.evaluate(net, d=D_CODE, p=P_NOISE, shots=B, k=K_BLOCK, seed=SEED, device=dev,
                          max_iter=MAX_ITER, delta0=DELTA0, alpha=wsm.DEFAULT_ALPHA)
        learned_info = {**train_info, "alpha": ev["alpha"], "cold": ev["cold"], "warm": ev["warm"],
                        "iterations_saved_fraction": ev["iterations_saved_fraction"],
                        "decision_agreement": ev["decision_agreement"]}

    chunks = -(-rows // _lib.WARM_MAX_ROWS)
    per_step = (1 + 2 * chunks + 3) if learned else 2     # features, (weights, network) per chunk, expansion, decode, decision
    line = {
        "metric": METRIC, "value": value, "unit": "syndromes/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": dev_ms_max / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32" if fp else "f64",
        "data": "synthetic: seeded i.i.d. depolarizing errors (SplitMix64 counter RNG) and their syndromes",
        "config": {"workload": WORKLOAD, "batch_per_gpu": B, "precision": args.precision,
                   "algorithm": args.algorithm,
                   "decoder": ("learned warm start (tensor-core network over the distinct message rows, "
                               "alpha=%g) + fused FP32 blockBP" % wsm.DEFAULT_ALPHA)
                   if learned else "fused blockBP, cold start",
                   "l2": "flushed: a 256 MB buffer is written before every timed step",
                   "mean_iters": iters_mean, "wall_s": wall},
        "clocks": clocks,
        "e2e": {"value": e2e_value, "unit": "syndromes/s", "h2d_bytes_per_step": int(B * S.shape[1]),
                "d2h_bytes_per_step": int(B * (1 + 32))},
        "gpu_launches": per_step * args.steps,
        "roofline": roof, "roofline_network": roof_mlp, "cpu_baseline": cpu,
        "speedup": speedup,
        "cold_start": cold, "plain_fp64_gpu": fp64_fused, "other_paths": legs, "mixed_batch": mixed,
        "learned_warm_start": learned_info,
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
    ap.add_argument("--algorithm", default="fused", choices=["fused", "mps"])
    ap.add_argument("--fp64-batch", type=int, default=512)
    ap.add_argument("--other-batch", type=int, default=4096)
    ap.add_argument("--mixed-batch", type=int, default=4096,
                    help="syndromes of the mixed-distance batching leg (0 skips it)")
    ap.add_argument("--cpu-procs", type=int, default=0)
    ap.add_argument("--no-cpu-baseline", dest="cpu_baseline", action="store_false")
    ap.add_argument("--no-warm", dest="warm", action="store_false")
    args = ap.parse_args()
    if args.impl == "reference":
        reference_arm(args)
    else:
        ours(args)


if __name__ == "__main__":
    main()
