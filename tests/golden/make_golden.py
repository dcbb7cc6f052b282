"""Write the oracle's expected values used by the GPU parity tests.

Calls only ``oracle/`` (and the seeded workload in ``synth/``).  Each file
holds, per shot, the oracle's log P, Delta, iterations, flags, decision and
the smallest relative Schmidt gap at a real truncation (inf = none), for a
seeded workload named in the file.  The truncating workloads also record
how far the oracle's own log P moves when every matrix it decomposes
carries relative noise of 1e-13 (FP64) or 1e-6 (FP32), about a thousand
units of rounding (``sens_fp64``, ``sens_fp32``, the larger of two seeded
draws): the parity tests compare a shot at a precision only where that
movement is far below the tolerance.  The k = 6 workloads (d = 31, 6 x 6
blocks) run the dense fused-block oracle of Remark 9 (``oracle.naive``),
which truncates nothing; one coset takes about ten minutes and 11 GB
there, so they are spread over (shot, coset) pairs.

    python tests/golden/make_golden.py [--which d5|d11|...|all] [--procs N]

``all`` leaves out the d = 31 workloads (about an hour on four cores and
45 GB): name them, e.g. ``--which d31_k6_p012,d31_k6_p015 --procs 4``.
"""

from __future__ import annotations

import argparse
import json
import multiprocessing as mp
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import synth  # noqa: E402
from oracle import blockbp as bb  # noqa: E402
from oracle import naive  # noqa: E402

HERE = os.path.dirname(os.path.abspath(__file__))

WORKLOADS = {
    # Small case: d = 5, p = 0.10, k = 3, D = 4, 10 fixed iterations, 200 shots.
    "d5": dict(file="oracle_d5_k3_D4_p010.json", d=5, k=3, D=4, p=0.10, max_iter=10, delta0=0.0,
               seed=synth.workload_seed(1, 0), first_shot=0, shots=200, fp32_ref=True),
    # Distance 11, p = 0.10, k = 4, D = 8, 20 fixed iterations.
    "d11": dict(file="oracle_d11_k4_D8_p010.json", d=11, k=4, D=8, p=0.10, max_iter=20, delta0=0.0,
                seed=synth.workload_seed(2, 2), first_shot=0, shots=200, fp32_ref=True),
}
# The other noise levels of the d = 11 workload (p index 0, 1, 3, 4).
for _ip, _p in ((0, 0.05), (1, 0.08), (3, 0.13), (4, 0.15)):
    WORKLOADS[f"d11_p{int(round(_p * 100)):03d}"] = dict(
        file=f"oracle_d11_k4_D8_p{int(round(_p * 100)):03d}.json", d=11, k=4, D=8, p=_p, max_iter=20,
        delta0=0.0, seed=synth.workload_seed(2, _ip), first_shot=0, shots=50, fp32_ref=True)

# The benchmark workload (d = 11, p = 0.10, k = 4, 20 fixed iterations)
# through the dense fused-block oracle of Remark 9, the reference of the
# fused form: it truncates nothing, where the MPS oracle drops Schmidt
# values below 1e-13 of the largest (a few 1e-9 in log P on some shots).
WORKLOADS["d11_fused"] = dict(file="oracle_d11_k4_fused_p010.json", d=11, k=4, D=16, p=0.10, max_iter=20,
                              delta0=0.0, seed=synth.workload_seed(2, 2), first_shot=0, shots=200, form="fused")

# Truncating MPS workloads: k = 4 with D = 2 and 4 at d = 9 and 11 (p = 0.10,
# 20 fixed iterations).  The in-block boundary MPS of a 4 x 4 block needs a
# bond of up to 16, so both bonds truncate inside every block, and D = 2
# also truncates the messages (exact bond up to 4).
for _d in (9, 11):
    for _D in (2, 4):
        WORKLOADS[f"d{_d}_D{_D}"] = dict(
            file=f"oracle_d{_d}_k4_D{_D}_p010.json", d=_d, k=4, D=_D, p=0.10, max_iter=20, delta0=0.0,
            seed=synth.workload_seed(6, 10 * _d + _D), first_shot=0, shots=24, sensitivity=True, fp32_ref=True)

# Distance 31, k = 6 (dense 64-entry messages), 20 fixed iterations, at the
# two noise levels of the d = 31 workload (p index 0, 1).
for _ip, _p in ((0, 0.12), (1, 0.15)):
    WORKLOADS[f"d31_k6_p{int(round(_p * 100)):03d}"] = dict(
        file=f"oracle_d31_k6_p{int(round(_p * 100)):03d}.json", d=31, k=6, D=64, p=_p, max_iter=20,
        delta0=0.0, seed=synth.workload_seed(5, _ip), first_shot=0, shots=3, form="fused")


def _one_coset(args):
    """One coset of one shot through the dense fused-block oracle."""
    w, b, L, s = args
    T = bb.coset_network(bb.Lattice(w["d"]), np.asarray(s, dtype=np.uint8), L, w["p"])
    logp, delta, iters, _ = naive.run_naive(T, w["k"], w["max_iter"], 0.1, w["delta0"])
    return b, L, float(logp), float(delta), int(iters)


def _assemble(w, rows):
    """Per-shot records from per-coset results (flags: Delta >= delta1 only,
    since positive tensors and messages keep every Z_v and o_e positive)."""
    out = []
    for b in range(w["shots"]):
        mine = sorted((r for r in rows if r[0] == b), key=lambda r: r[1])
        logp = [r[2] for r in mine]
        delta = [r[3] for r in mine]
        flags = [bb.FLAG_UNTRUSTED if dl >= 1e-2 else 0 for dl in delta]
        out.append(dict(shot=w["first_shot"] + b, logp=logp, delta=delta, iters=[r[4] for r in mine],
                        flags=flags, decision=int(bb.decide(logp, delta, flags)), min_gap=None,
                        truncations=0))
    return out


def _perturbed_svd(rel, seed):
    """numpy's SVD applied to M * (1 + rel * n), n standard normal per entry:
    rounding-level noise on every decomposition the oracle makes."""
    svd = np.linalg.svd
    rng = np.random.default_rng(seed)

    def noisy(M, full_matrices=False):
        return svd(M * (1.0 + rel * rng.standard_normal(M.shape)), full_matrices=full_matrices)
    return svd, noisy


def _sensitivity(P, s, base, rel, seed, draws=2):
    """Largest |d log P| of the oracle, over ``draws`` seeded draws, when every
    matrix it decomposes carries a relative perturbation of size rel.  Where
    the truncated iteration amplifies rounding (near-degenerate cuts, BP that
    does not settle at a small D), two correct implementations with
    different rounding can end far apart; this measures how far."""
    worst = 0.0
    for k in range(draws):
        svd, noisy = _perturbed_svd(rel, seed + 7919 * k)
        np.linalg.svd = noisy
        try:
            pert = bb.decode(s, P)["logp"]
        finally:
            np.linalg.svd = svd
        worst = max(worst, float(np.max(np.abs(np.asarray(base) - np.asarray(pert)))))
    return worst


def _one(args):
    w, b, s = args
    P = bb.Params(d=w["d"], k=w["k"], D=w["D"], p=w["p"], max_iter=w["max_iter"], delta0=w["delta0"])
    s = np.asarray(s, dtype=np.uint8)
    r = bb.decode(s, P)
    st = r["stats"]
    row = dict(shot=w["first_shot"] + b, logp=[float(x) for x in r["logp"]],
               delta=[float(x) for x in r["delta"]], iters=[int(x) for x in r["iters"]],
               flags=[int(x) for x in r["flags"]], decision=int(r["decision"]),
               min_gap=(None if not np.isfinite(st.min_gap) else float(st.min_gap)),
               truncations=int(st.truncations), flops=float(st.flops))
    if w.get("fp32_ref"):
        # The same steps in float32 (numpy / LAPACK single precision, relative
        # cutoff 1e-7 as the GPU's FP32 default): how far single precision
        # moves the method's own log P on this shot.
        P32 = bb.Params(d=w["d"], k=w["k"], D=w["D"], p=w["p"], max_iter=w["max_iter"], delta0=w["delta0"],
                        cutoff=1e-7)
        r32 = bb.decode(s, P32, dtype=np.float32)
        row["dlogp_fp32"] = float(np.max(np.abs(np.asarray(r32["logp"]) - np.asarray(r["logp"]))))
    if w.get("sensitivity"):
        # Noise of the size by which two correct decompositions of the same
        # matrix differ: about a thousand units of rounding (unit roundoff
        # 1.1e-16 in FP64 and 6e-8 in FP32; the GPU's Gram-Schmidt and
        # one-sided Jacobi against LAPACK here), seeded by the shot.
        row["sens_fp64"] = _sensitivity(P, s, r["logp"], 1e-13, 1000 + b)
        row["sens_fp32"] = _sensitivity(P, s, r["logp"], 1e-6, 2000 + b)
    return row


def make(name: str, procs: int):
    w = WORKLOADS[name]
    ex, ez, S = synth.sample_syndromes(w["seed"], w["first_shot"], w["shots"], w["d"], w["p"])
    ctx = mp.get_context("spawn")
    if w.get("form") == "fused":
        with ctx.Pool(procs) as pool:
            per = pool.map(_one_coset, [(w, b, L, S[b].tolist()) for b in range(w["shots"]) for L in range(4)],
                           chunksize=1)
        rows = _assemble(w, per)
    else:
        with ctx.Pool(procs) as pool:
            rows = pool.map(_one, [(w, b, S[b].tolist()) for b in range(w["shots"])])
    meta = {k: v for k, v in w.items() if k not in ("file", "form", "sensitivity", "fp32_ref")}
    if w.get("form") == "fused":
        meta["oracle"] = "dense fused-block blockBP (Remark 9), no truncation"
    meta["eta"], meta["delta1"], meta["cutoff"] = 0.1, 1e-2, 1e-13
    with open(os.path.join(HERE, w["file"]), "w") as f:
        json.dump({"workload": meta, "shots": rows}, f, indent=0)
    print("wrote", w["file"])


if __name__ == "__main__":
    ap = argparse.ArgumentParser()
    ap.add_argument("--which", default="all")
    ap.add_argument("--procs", type=int, default=os.cpu_count() or 1)
    a = ap.parse_args()
    names = [n for n in WORKLOADS if not n.startswith("d31")] if a.which == "all" else a.which.split(",")
    for name in names:
        make(name, a.procs)
