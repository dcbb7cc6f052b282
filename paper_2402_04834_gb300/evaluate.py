"""Logical error rate and throughput of the decoder on seeded syndromes.

P_L is estimated as in Sec. IV: errors are drawn on the device
(``decoder.sample``, which also returns each error's true logical class), the
decoder picks a coset, and a shot fails when the pick is not the true
class; the 95 % interval is Wilson's.  Throughput is timed with CUDA events
around the decode calls of the whole batch.  The paper observes that BP
converges faster at low noise, so max-iter can be lowered there (Sec. IV,
last paragraph); ``sweep`` measures that trade-off.

    python -m paper_2402_04834_gb300.evaluate --d 11 --p 0.05 0.10 --max-iter 5 10 20 --shots 10000
    # d = 31 with 6 x 6 blocks, 10^5 shots per noise level (seeds 5000, 5001)
    python -m paper_2402_04834_gb300.evaluate --d 31 --k 6 --p 0.12 0.15 --max-iter 20 --shots 100000 \
        --seed-base 5000 --seed-per-d 0
"""

from __future__ import annotations

import argparse
import json

import torch

from ._lib import DecoderParams
from .decoder import decode, sample
from .warmstart import wilson


def logical_error_rate(d: int, p: float, shots: int, seed: int, chunk: int = 16384, first_shot: int = 0,
                       **params) -> dict:
    """Decode ``shots`` seeded syndromes, ``chunk`` per call after one
    untimed warm-up call; P_L with its Wilson 95 % interval, mean iterations
    over cosets, syndromes per second (device time of the decode calls) and
    a histogram of the final Delta of every coset by decade."""
    # Shots first_shot .. first_shot + shots - 1 of the seed's counter-based
    # stream: a run resumes, or splits into parts, by shot index.
    _, _, s, tc = sample(seed, first_shot, shots, d, p, with_errors=False)
    prm = DecoderParams(d=d, p=p, **params)
    decode(s[:min(shots, 64)], prm)
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    dec, its, dls = [], [], []
    a.record()
    for c0 in range(0, shots, chunk):
        out = decode(s[c0:c0 + chunk], prm)
        dec.append(out["decision"])
        its.append(out["iters"])
        dls.append(out["delta"])
    b.record()
    torch.cuda.synchronize()
    ms = a.elapsed_time(b)
    fails = int((torch.cat(dec).to(torch.int64) != tc.to(torch.int64)).sum().item())
    lo, hi = wilson(fails, shots)
    # Final Delta of every coset in decades: [0, 1e-8), [1e-8, 1e-7), ..., [1e-1, inf).
    dl = torch.cat(dls).double().clamp_min(1e-300).log10().floor().clamp(-9, -1).cpu()
    hist = [int((dl == e).sum().item()) for e in range(-9, 0)]
    return {"d": d, "p": p, "shots": shots, "first_shot": first_shot, **params, "failures": fails,
            "P_L": fails / shots,
            "P_L_wilson95": [lo, hi], "mean_iters": float(torch.cat(its).double().mean().item()),
            "syndromes_per_s": shots / ms * 1e3,
            "delta_decades": {"edges": [0.0] + [10.0 ** e for e in range(-8, 0)] + ["inf"], "counts": hist}}


def sweep(d_list, p_list, max_iters, shots, k=4, precision="fp32", algorithm="fused", seed_base=7000,
          seed_per_d=100, first_shot=0):
    """Seeds: seed_base + seed_per_d * d + (index of p in p_list)."""
    rows = []
    for d in d_list:
        for ip, p in enumerate(p_list):
            for mi in max_iters:
                rows.append(logical_error_rate(d, p, shots, seed_base + seed_per_d * d + ip, k=k, max_iter=mi,
                                               precision=precision, algorithm=algorithm, first_shot=first_shot))
    return rows


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--d", type=int, nargs="+", default=[11])
    ap.add_argument("--p", type=float, nargs="+", default=[0.05, 0.10])
    ap.add_argument("--max-iter", type=int, nargs="+", default=[5, 10, 20])
    ap.add_argument("--shots", type=int, default=10000)
    ap.add_argument("--precision", default="fp32", choices=["fp32", "fp64"])
    ap.add_argument("--algorithm", default="fused", choices=["fused", "mps"])
    ap.add_argument("--k", type=int, default=4, help="block side (6: the d = 31 scheme of Sec. IV)")
    ap.add_argument("--seed-base", type=int, default=7000)
    ap.add_argument("--seed-per-d", type=int, default=100)
    ap.add_argument("--first-shot", type=int, default=0, help="resume or split a run by shot index")
    args = ap.parse_args()
    for r in sweep(args.d, args.p, args.max_iter, args.shots, k=args.k, precision=args.precision,
                   algorithm=args.algorithm, seed_base=args.seed_base, seed_per_d=args.seed_per_d,
                   first_shot=args.first_shot):
        print(json.dumps(r), flush=True)


if __name__ == "__main__":
    main()
