"""Write the oracle's expected values used by the GPU parity tests.

Calls only ``oracle/`` (and the seeded workload in ``synth/``).  Each file
holds, per shot, the oracle's log P, Delta, iterations, flags, decision and
the smallest relative Schmidt gap at a real truncation (inf = none), for a
seeded workload named in the file.

    python tests/golden/make_golden.py [--which d5|d11|all] [--procs N]
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

HERE = os.path.dirname(os.path.abspath(__file__))

WORKLOADS = {
    # Small case: d = 5, p = 0.10, k = 3, D = 4, 10 fixed iterations, 200 shots.
    "d5": dict(file="oracle_d5_k3_D4_p010.json", d=5, k=3, D=4, p=0.10, max_iter=10, delta0=0.0,
               seed=synth.workload_seed(1, 0), first_shot=0, shots=200),
    # Distance 11, p = 0.10, k = 4, D = 8, 20 fixed iterations.
    "d11": dict(file="oracle_d11_k4_D8_p010.json", d=11, k=4, D=8, p=0.10, max_iter=20, delta0=0.0,
                seed=synth.workload_seed(2, 2), first_shot=0, shots=12),
}
# The other noise levels of the d = 11 workload (p index 0, 1, 3, 4).
for _ip, _p in ((0, 0.05), (1, 0.08), (3, 0.13), (4, 0.15)):
    WORKLOADS[f"d11_p{int(round(_p * 100)):03d}"] = dict(
        file=f"oracle_d11_k4_D8_p{int(round(_p * 100)):03d}.json", d=11, k=4, D=8, p=_p, max_iter=20,
        delta0=0.0, seed=synth.workload_seed(2, _ip), first_shot=0, shots=4)


def _one(args):
    w, b, s = args
    P = bb.Params(d=w["d"], k=w["k"], D=w["D"], p=w["p"], max_iter=w["max_iter"], delta0=w["delta0"])
    r = bb.decode(np.asarray(s, dtype=np.uint8), P)
    st = r["stats"]
    return dict(shot=w["first_shot"] + b, logp=[float(x) for x in r["logp"]],
                delta=[float(x) for x in r["delta"]], iters=[int(x) for x in r["iters"]],
                flags=[int(x) for x in r["flags"]], decision=int(r["decision"]),
                min_gap=(None if not np.isfinite(st.min_gap) else float(st.min_gap)),
                truncations=int(st.truncations), flops=float(st.flops))


def make(name: str, procs: int):
    w = WORKLOADS[name]
    ex, ez, S = synth.sample_syndromes(w["seed"], w["first_shot"], w["shots"], w["d"], w["p"])
    ctx = mp.get_context("spawn")
    with ctx.Pool(procs) as pool:
        rows = pool.map(_one, [(w, b, S[b].tolist()) for b in range(w["shots"])])
    meta = {k: v for k, v in w.items() if k != "file"}
    meta["eta"], meta["delta1"], meta["cutoff"] = 0.1, 1e-2, 1e-13
    with open(os.path.join(HERE, w["file"]), "w") as f:
        json.dump({"workload": meta, "shots": rows}, f, indent=0)
    print("wrote", w["file"])


if __name__ == "__main__":
    ap = argparse.ArgumentParser()
    ap.add_argument("--which", default="all")
    ap.add_argument("--procs", type=int, default=os.cpu_count() or 1)
    a = ap.parse_args()
    for name in (WORKLOADS if a.which == "all" else [a.which]):
        make(name, a.procs)
