"""GPU check of the logical-error-rate estimator: its failure count equals
the count obtained from the oracle's true logical class of the same seeded
errors (the CPU sampler and the device sampler draw identical errors)."""

import numpy as np
import pytest

import paper_2402_04834_gb300 as pkg
import synth
from oracle.lattice import Lattice
from paper_2402_04834_gb300 import evaluate
from paper_2402_04834_gb300.build import build

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu


def test_failure_count_matches_oracle_true_class():
    build()
    d, p, shots, seed = 5, 0.12, 300, 4242
    r = evaluate.logical_error_rate(d, p, shots, seed, k=4, max_iter=10, precision="fp32", algorithm="fused")
    ex, ez, S = synth.sample_syndromes(seed, 0, shots, d, p)
    lat = Lattice(d)
    tc = np.array([lat.true_class(ex[b], ez[b], S[b]) for b in range(shots)])
    out = pkg.decode(torch.from_numpy(S).cuda(), pkg.DecoderParams(d=d, k=4, p=p, max_iter=10, precision="fp32",
                                                                    algorithm="fused"))
    fails = int(np.sum(out["decision"].cpu().numpy() != tc))
    assert r["failures"] == fails
    lo, hi = r["P_L_wilson95"]
    assert lo <= r["P_L"] <= hi and r["mean_iters"] <= 10


def test_runs_split_by_shot_index_add_up():
    # The sampler is counter-based: shots 0 .. 399 decoded in two parts give
    # the failures and iterations of one run over all of them.
    build()
    kw = dict(k=4, max_iter=10, precision="fp32", algorithm="fused")
    whole = evaluate.logical_error_rate(7, 0.12, 400, 77, **kw)
    a = evaluate.logical_error_rate(7, 0.12, 150, 77, first_shot=0, **kw)
    b = evaluate.logical_error_rate(7, 0.12, 250, 77, first_shot=150, **kw)
    assert a["failures"] + b["failures"] == whole["failures"]
    assert abs(a["mean_iters"] * 150 + b["mean_iters"] * 250 - whole["mean_iters"] * 400) < 1e-6
