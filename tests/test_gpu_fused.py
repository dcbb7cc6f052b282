"""GPU parity of the fused-block path (Remark 9) against the dense oracle.

The fused path carries dense messages and truncates nothing, so its oracle
is ``oracle.naive`` (the same rule written with whole-block tensors); FP64
must agree to 1e-9 in every coset's log P and FP32 to 1e-3.  Where the MPS
form truncates nothing (d = 11, k = 4, D = 8 on these shots) the fused path
also reproduces the MPS oracle's golden values.
"""

import json
import os

import numpy as np
import pytest

import paper_2402_04834_gb300 as pkg
import synth
from oracle import blockbp as bb
from oracle.lattice import Lattice
from oracle.naive import run_naive
from oracle.tn import coset_network
from paper_2402_04834_gb300.build import build

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu
HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def dev():
    build()
    pkg.lib()
    return torch.device("cuda:0")


def gpu(S, prm, dev):
    out = pkg.decode(torch.from_numpy(np.ascontiguousarray(S)).to(dev), prm)
    torch.cuda.synchronize()
    return {k: v.cpu().numpy() for k, v in out.items()}


_naive_cache = {}


def naive_logp(S, d, k, p, iters, delta0=0.0):
    key = (S.tobytes(), d, k, p, iters, delta0)
    if key in _naive_cache:
        return _naive_cache[key]
    lat = Lattice(d)
    out = []
    for s in S:
        row = []
        for L in range(4):
            lp, dl, it, _ = run_naive(coset_network(lat, s, L, p), k, iters, 0.1, delta0)
            row.append((lp, dl, it))
        out.append(row)
    _naive_cache[key] = out
    return out


# Every compiled launch shape (warps per CTA, cosets per CTA) of each precision.
SHAPES = [(prec, w, c) for prec, shapes in pkg.FUSED_SHAPES.items() for (w, c) in shapes]


@pytest.mark.parametrize("d,k,iters,p", [
    (5, 3, 8, 0.10),      # 3 x 3 blocks of 3
    (5, 4, 6, 0.10),      # blocks 4, 4, 1
    (7, 4, 5, 0.08),      # blocks 4, 4, 4, 1
    (3, 2, 6, 0.12),      # blocks 2, 2, 1
    (4, 1, 4, 0.10),      # one node per block (plain BP on the network)
    (2, 3, 3, 0.20),      # one block, no messages
])
@pytest.mark.parametrize("precision,warps,cosets", SHAPES, ids=[f"{a}-w{b}-g{c}" for a, b, c in SHAPES])
def test_fused_matches_dense_oracle(dev, d, k, iters, p, precision, warps, cosets):
    _, _, S = synth.sample_syndromes(515, 0, 3, d, p)
    prm = pkg.DecoderParams(d=d, k=k, p=p, max_iter=iters, delta0=0.0, precision=precision,
                            algorithm="fused", warps=warps, cosets=cosets)
    out = gpu(S, prm, dev)
    ref = naive_logp(S, d, k, p, iters)
    tol = 1e-9 if precision == "fp64" else 1e-3
    for b in range(S.shape[0]):
        for L in range(4):
            lp, dl, it = ref[b][L]
            assert abs(out["logp"][b][L] - lp) <= tol, (b, L, out["logp"][b][L], lp)
            assert abs(out["delta"][b][L] - dl) <= (1e-7 if precision == "fp64" else 1e-4)
            if d > 2:
                assert out["iters"][b][L] == iters


SHAPES_K6 = [(prec, w, c) for prec, shapes in pkg.FUSED_SHAPES_K6.items() for (w, c) in shapes]


@pytest.mark.parametrize("d,k,iters,p", [
    (7, 6, 4, 0.08),      # blocks 6, 6, 1: an interior 6 x 6 block with all four side messages
    (4, 6, 4, 0.10),      # blocks 6, 1
    (9, 5, 3, 0.10),      # blocks 5, 5, 5, 2
])
@pytest.mark.parametrize("precision,warps,cosets", SHAPES_K6, ids=[f"{a}-w{b}-g{c}" for a, b, c in SHAPES_K6])
def test_fused_k6_matches_dense_oracle(dev, d, k, iters, p, precision, warps, cosets):
    # Block sides 5 and 6 (dense messages of 32 and 64, states of up to 2^12
    # entries): FP64 to 1e-9 and FP32 to 1e-3 against the dense oracle.
    _, _, S = synth.sample_syndromes(515, 0, 2, d, p)
    prm = pkg.DecoderParams(d=d, k=k, p=p, max_iter=iters, delta0=0.0, precision=precision,
                            algorithm="fused", warps=warps, cosets=cosets)
    out = gpu(S, prm, dev)
    ref = naive_logp(S, d, k, p, iters)
    tol = 1e-9 if precision == "fp64" else 1e-3
    for b in range(S.shape[0]):
        for L in range(4):
            lp, dl, it = ref[b][L]
            assert abs(out["logp"][b][L] - lp) <= tol, (b, L, out["logp"][b][L], lp)
            assert abs(out["delta"][b][L] - dl) <= (1e-7 if precision == "fp64" else 1e-4)
            assert out["iters"][b][L] == iters


def test_fused_k6_large_distances(dev):
    # d = 13 with 6 x 6 blocks: FP32 against FP64.  d = 31 (the largest
    # configuration; FP64 messages would not fit in shared memory): finite
    # log-probabilities below 0, valid decisions, bitwise-repeatable results.
    _, _, S13 = synth.sample_syndromes(4013, 0, 6, 13, 0.10)
    r = {prec: gpu(S13, pkg.DecoderParams(d=13, k=6, p=0.10, max_iter=8, delta0=0.0, precision=prec,
                                           algorithm="fused"), dev) for prec in ("fp32", "fp64")}
    assert np.max(np.abs(r["fp32"]["logp"] - r["fp64"]["logp"])) < 1e-3
    assert np.array_equal(r["fp32"]["decision"], r["fp64"]["decision"])
    _, _, S31 = synth.sample_syndromes(4031, 0, 4, 31, 0.12)
    prm = pkg.DecoderParams(d=31, k=6, p=0.12, max_iter=6, delta0=0.0, precision="fp32", algorithm="fused")
    a, b = gpu(S31, prm, dev), gpu(S31, prm, dev)
    assert np.all(np.isfinite(a["logp"])) and np.all(a["logp"] < 0)
    assert np.all((a["decision"] >= 0) & (a["decision"] < 4))
    for key in ("logp", "delta", "iters", "decision"):
        assert np.array_equal(a[key], b[key]), key


def test_fused_equals_mps_golden_at_d11(dev):
    with open(os.path.join(HERE, "golden", "oracle_d11_k4_D8_p010.json")) as f:
        g = json.load(f)
    w = g["workload"]
    _, _, S = synth.sample_syndromes(w["seed"], w["first_shot"], w["shots"], w["d"], w["p"])
    prm = pkg.DecoderParams(d=w["d"], k=w["k"], p=w["p"], max_iter=w["max_iter"], delta0=w["delta0"],
                            precision="fp64", algorithm="fused")
    out = gpu(S, prm, dev)
    for r in g["shots"]:
        assert r["truncations"] == 0          # the MPS form truncated nothing here
        b = r["shot"] - w["first_shot"]
        np.testing.assert_allclose(out["logp"][b], r["logp"], rtol=0, atol=1e-9)
        assert int(out["decision"][b]) == r["decision"]


@pytest.mark.parametrize("precision,warps,cosets", [("fp64", 8, 1), ("fp64", 4, 2), ("fp64", 8, 2), ("fp64", 4, 4),
                                                    ("fp32", 8, 4), ("fp32", 8, 2)])
def test_fused_early_exit_and_decision(dev, precision, warps, cosets):
    # delta0 = 1e-4: the cosets of one syndrome stop at different
    # iterations; a CTA that decodes several of them freezes each one when
    # it converges, so iterations and log P match a coset decoded alone.
    d, k, p = 7, 4, 0.06
    _, _, S = synth.sample_syndromes(77, 0, 4, d, p)
    prm = pkg.DecoderParams(d=d, k=k, p=p, max_iter=40, delta0=1e-4, algorithm="fused", precision=precision,
                            warps=warps, cosets=cosets)
    out = gpu(S, prm, dev)
    lat = Lattice(d)
    margin, tol = (1e-6, 1e-9) if precision == "fp64" else (1e-5, 1e-3)
    its = set()
    for b in range(4):
        lps, dls = [], []
        for L in range(4):
            lp, dl, it, _ = run_naive(coset_network(lat, S[b], L, p), k, 40, 0.1, 1e-4)
            lps.append(lp)
            dls.append(dl)
            its.add(it)
            if abs(dl - 1e-4) > margin:
                assert out["iters"][b][L] == it
                assert abs(out["logp"][b][L] - lp) < tol
        flags = [0 if x < 1e-2 else 1 for x in dls]
        assert int(out["decision"][b]) == bb.decide(lps, dls, flags)
    assert len(its) > 1          # the cosets really stop at different iterations


def test_fused_needs_no_workspace(dev):
    prm = pkg.DecoderParams(d=11, k=4, algorithm="fused")
    assert pkg.workspace_bytes(prm, 1000) == 0
