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
# ... with the messages in shared memory (1) and, where compiled, in workspace slots (2).
SHAPES = ([(prec, w, c, 1) for prec, shapes in pkg.FUSED_SHAPES.items() for (w, c) in shapes] +
          [(prec, w, c, 2) for prec, shapes in pkg.FUSED_SHAPES_WS.items() for (w, c) in shapes])


@pytest.mark.parametrize("d,k,iters,p", [
    (5, 3, 8, 0.10),      # 3 x 3 blocks of 3
    (5, 4, 6, 0.10),      # blocks 4, 4, 1
    (7, 4, 5, 0.08),      # blocks 4, 4, 4, 1
    (3, 2, 6, 0.12),      # blocks 2, 2, 1
    (4, 1, 4, 0.10),      # one node per block (plain BP on the network)
    (2, 3, 3, 0.20),      # one block, no messages
])
@pytest.mark.parametrize("precision,warps,cosets,messages", SHAPES,
                         ids=[f"{a}-w{b}-g{c}-m{m}" for a, b, c, m in SHAPES])
def test_fused_matches_dense_oracle(dev, d, k, iters, p, precision, warps, cosets, messages):
    _, _, S = synth.sample_syndromes(515, 0, 3, d, p)
    prm = pkg.DecoderParams(d=d, k=k, p=p, max_iter=iters, delta0=0.0, precision=precision,
                            algorithm="fused", warps=warps, cosets=cosets, messages=messages)
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


@pytest.mark.parametrize("d,p,B,iters", [(13, 0.10, 6, 8), (31, 0.12, 2, 6)])
def test_fused_k6_fp32_against_fp64(dev, d, p, B, iters):
    # 6 x 6 blocks at the larger distances: FP32 within 1e-3 of FP64, same
    # decisions, and bitwise-repeatable results; log P finite and below 0.
    _, _, S = synth.sample_syndromes(4000 + d, 0, B, d, p)
    r = {prec: gpu(S, pkg.DecoderParams(d=d, k=6, p=p, max_iter=iters, delta0=0.0, precision=prec,
                                        algorithm="fused"), dev) for prec in ("fp32", "fp64")}
    assert np.max(np.abs(r["fp32"]["logp"] - r["fp64"]["logp"])) < 1e-3
    assert np.array_equal(r["fp32"]["decision"], r["fp64"]["decision"])
    assert np.all(np.isfinite(r["fp64"]["logp"])) and np.all(r["fp64"]["logp"] < 0)
    again = gpu(S, pkg.DecoderParams(d=d, k=6, p=p, max_iter=iters, delta0=0.0, precision="fp32",
                                     algorithm="fused"), dev)
    for key in ("logp", "delta", "iters", "decision"):
        assert np.array_equal(again[key], r["fp32"][key]), key


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_fused_k6_persistent_grid_takes_every_item(dev, precision):
    # k = 6 runs a persistent grid with one message slot per CTA: 1200 items
    # in one call (several per CTA, slots reused) give bitwise the results
    # of small calls, early exit included.
    d, p = 7, 0.10
    _, _, S = synth.sample_syndromes(707, 0, 300, d, p)
    prm = pkg.DecoderParams(d=d, k=6, p=p, max_iter=12, delta0=1e-4, precision=precision, algorithm="fused")
    whole = gpu(S, prm, dev)
    for b0 in range(0, 300, 37):
        part = gpu(S[b0:b0 + 37], prm, dev)
        for key in ("logp", "delta", "iters", "flags", "decision"):
            assert np.array_equal(part[key], whole[key][b0:b0 + 37]), (b0, key)


def test_fused_k6_mixed_launch_equals_per_distance_decodes(dev):
    from paper_2402_04834_gb300.decoder import decode_mixed, pack_mixed
    p = 0.10
    rng = np.random.default_rng(66)
    ds = rng.choice([4, 7, 13], size=40)
    shots = [synth.sample_syndromes(66, b, 1, int(d), p)[2][0] for b, d in enumerate(ds)]
    packed, offsets, d_of = pack_mixed(shots, device=dev)
    prm = pkg.DecoderParams(d=0, k=6, p=p, max_iter=8, delta0=1e-4, precision="fp32", algorithm="fused")
    out = decode_mixed(packed, offsets, d_of, prm)
    torch.cuda.synchronize()
    for d in sorted(set(ds.tolist())):
        idx = np.nonzero(ds == d)[0]
        ref = gpu(np.stack([shots[i] for i in idx]), pkg.DecoderParams(**{**prm.__dict__, "d": int(d)}), dev)
        for key in ("logp", "delta", "iters", "flags", "decision"):
            assert np.array_equal(out[key].cpu().numpy()[idx], ref[key]), (d, key)


@pytest.mark.parametrize("name", ["oracle_d31_k6_p012.json", "oracle_d31_k6_p015.json"])
def test_fused_k6_d31_matches_oracle_golden(dev, name):
    # The d = 31, k = 6 workload (20 fixed iterations) against stored values
    # of the dense fused-block oracle: FP32 within 1e-3 per coset, FP64 within
    # 1e-9, decisions equal where the oracle's margin exceeds 1e-2.
    path = os.path.join(HERE, "golden", name)
    if not os.path.exists(path):
        pytest.skip(f"{name} not generated")
    with open(path) as f:
        g = json.load(f)
    w = g["workload"]
    _, _, S = synth.sample_syndromes(w["seed"], w["first_shot"], len(g["shots"]), w["d"], w["p"])
    for precision, tol in (("fp32", 1e-3), ("fp64", 1e-9)):
        prm = pkg.DecoderParams(d=w["d"], k=w["k"], p=w["p"], max_iter=w["max_iter"], delta0=w["delta0"],
                                precision=precision, algorithm="fused")
        out = gpu(S, prm, dev)
        for r in g["shots"]:
            b = r["shot"] - w["first_shot"]
            np.testing.assert_allclose(out["logp"][b], r["logp"], rtol=0, atol=tol)
            np.testing.assert_allclose(out["delta"][b], r["delta"], rtol=0, atol=1e-4 if precision == "fp32" else 1e-7)
            assert list(out["iters"][b]) == r["iters"]
            lp = sorted(r["logp"][L] for L in range(4) if r["flags"][L] == 0)
            if len(lp) < 2 or lp[-1] - lp[-2] > 1e-2:
                assert int(out["decision"][b]) == r["decision"], (precision, b)


def test_fused_equals_mps_golden_at_d11(dev):
    # The MPS form truncates nothing on these shots (D = 8); its oracle drops
    # Schmidt values below 1e-13 of the largest, which moves log P by a few
    # 1e-9 at most: the fused form matches it to 1e-8 and the dense
    # fused-block oracle to 1e-9 (test_gpu_parity).
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
        np.testing.assert_allclose(out["logp"][b], r["logp"], rtol=0, atol=1e-8)
        assert int(out["decision"][b]) == r["decision"]


@pytest.mark.parametrize("precision,warps,cosets,messages", [
    ("fp64", 8, 1, 1), ("fp64", 4, 2, 1), ("fp64", 8, 2, 1), ("fp64", 4, 4, 1), ("fp64", 4, 2, 2),
    ("fp32", 8, 4, 1), ("fp32", 8, 2, 1), ("fp32", 8, 4, 2), ("fp32", 8, 2, 2)])
def test_fused_early_exit_and_decision(dev, precision, warps, cosets, messages):
    # delta0 = 1e-4: the cosets of one syndrome stop at different
    # iterations; a CTA that decodes several of them freezes each one when
    # it converges, so iterations and log P match a coset decoded alone.
    d, k, p = 7, 4, 0.06
    _, _, S = synth.sample_syndromes(77, 0, 4, d, p)
    prm = pkg.DecoderParams(d=d, k=k, p=p, max_iter=40, delta0=1e-4, algorithm="fused", precision=precision,
                            warps=warps, cosets=cosets, messages=messages)
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
    # The benchmark's shape keeps its messages in shared memory.
    prm = pkg.DecoderParams(d=11, k=4, algorithm="fused", precision="fp32")
    assert pkg.workspace_bytes(prm, 1000) == 0
    assert pkg.workspace_bytes(pkg.DecoderParams(d=11, k=4, algorithm="fused", messages=2, precision="fp32"),
                               1000) > 0


@pytest.mark.parametrize("d,precision,warps,cosets", [(11, "fp32", 8, 4), (13, "fp32", 8, 2), (21, "fp32", 8, 4),
                                                      (11, "fp64", 4, 2), (13, "fp64", 4, 2)])
def test_messages_in_workspace_or_shared_memory_give_the_same_bits(dev, d, precision, warps, cosets):
    # Where the messages live (shared memory, or a workspace slot of a
    # persistent CTA reused by several items) changes no bit of any output,
    # early exit, initial messages and exported messages included.
    from paper_2402_04834_gb300 import warmstart as wsm
    _, _, S = synth.sample_syndromes(1300 + d, 0, 400, d, 0.1)
    s = torch.from_numpy(S).to(dev)
    M = wsm.message_count(pkg.DecoderParams(d=d, k=4, algorithm="fused"))
    init = torch.rand((400 * 4 * M, 16), generator=torch.Generator().manual_seed(d)).to(dev) + 0.01
    res = {}
    for mem in (1, 2):
        prm = pkg.DecoderParams(d=d, k=4, p=0.1, max_iter=15, delta0=1e-4, precision=precision, algorithm="fused",
                                warps=warps, cosets=cosets, messages=mem)
        final = torch.empty_like(init)
        res[mem] = (wsm.decode_ex(s, prm), wsm.decode_ex(s, prm, init_msgs=init, final_msgs=final), final)
    torch.cuda.synchronize()
    for i in range(2):
        for key in ("logp", "delta", "iters", "flags", "decision"):
            assert torch.equal(res[1][i][key], res[2][i][key]), (i, key)
    assert torch.equal(res[1][2], res[2][2])


@pytest.mark.parametrize("d,precision", [(9, "fp64"), (11, "fp64"), (11, "fp32")])
def test_four_coset_passes_give_the_two_coset_bits(dev, d, precision):
    # With four cosets per CTA the register forms run one pass over the
    # three or four iterating cosets of a message (8 lanes per coset, two
    # rows per lane), and passes of two once one or two iterate; with one or
    # two cosets per CTA every pass holds two coset jobs of 16 lanes each.
    # delta0 = 1e-4 lets the cosets of a syndrome stop at different
    # iterations, so every pass width runs, and odd d brings in the edge
    # blocks' forms: every output of every compiled shape is the same bits.
    _, _, S = synth.sample_syndromes(1700 + d, 0, 256, d, 0.1)
    s = torch.from_numpy(S).to(dev)
    res = {}
    for w, c in pkg.FUSED_SHAPES[precision]:
        prm = pkg.DecoderParams(d=d, k=4, p=0.1, max_iter=15, delta0=1e-4, precision=precision,
                                algorithm="fused", warps=w, cosets=c, messages=1)
        res[(w, c)] = pkg.decode(s, prm)
    torch.cuda.synchronize()
    shapes = list(res)
    assert any(c == 4 for _, c in shapes) and any(c < 4 for _, c in shapes)
    ref = res[shapes[0]]
    for sh in shapes[1:]:
        for key in ("logp", "delta", "iters", "flags", "decision"):
            assert torch.equal(res[sh][key], ref[key]), (sh, key)
    its = ref["iters"].view(-1, 4)
    assert bool((its.max(1).values != its.min(1).values).any())   # cosets stop at different iterations


@pytest.mark.parametrize("d,precision,messages", [(46, "fp32", 1), (34, "fp64", 1), (58, "fp32", 0), (54, "fp64", 0)])
def test_fused_k4_at_the_largest_distance(dev, d, precision, messages):
    # The largest distances with the messages in shared memory (46 / 34) and
    # in the workspace (58 / 54): finite log-probabilities below 0, valid
    # decisions, repeatable bit for bit.
    _, _, S = synth.sample_syndromes(4800 + d, 0, 2, d, 0.1)
    prm = pkg.DecoderParams(d=d, k=4, p=0.1, max_iter=3, delta0=0.0, precision=precision, algorithm="fused",
                            messages=messages)
    a, b = gpu(S, prm, dev), gpu(S, prm, dev)
    assert np.all(np.isfinite(a["logp"])) and np.all(a["logp"] < 0)
    assert np.all((a["decision"] >= 0) & (a["decision"] < 4))
    for key in ("logp", "delta", "iters", "decision"):
        assert np.array_equal(a[key], b[key]), key


@pytest.mark.parametrize("p", [0.002, 0.3, 0.6])
def test_fused_fp32_against_fp64_at_extreme_noise(dev, p):
    # Noise far from the benchmark's: the qubit tables span pi(I) = 0.998 to
    # pi(X) = 6.7e-4 at p = 0.002, and pi(I) < pi(X) + pi(Y) + pi(Z) at
    # p = 0.6.  FP32 stays within 1e-3 of FP64 per coset, with the same
    # decisions wherever the FP64 margin exceeds 1e-2.
    d = 11
    _, _, S = synth.sample_syndromes(6600 + int(p * 1000), 0, 64, d, p)
    r = {prec: gpu(S, pkg.DecoderParams(d=d, k=4, p=p, max_iter=20, delta0=0.0, precision=prec,
                                        algorithm="fused"), dev) for prec in ("fp32", "fp64")}
    assert np.all(np.isfinite(r["fp64"]["logp"]))
    assert np.max(np.abs(r["fp32"]["logp"] - r["fp64"]["logp"])) < 1e-3
    lp = np.sort(np.where(r["fp64"]["flags"] == 0, r["fp64"]["logp"], -np.inf), axis=1)
    sure = (lp[:, -1] - lp[:, -2]) > 1e-2
    assert np.array_equal(r["fp32"]["decision"][sure], r["fp64"]["decision"][sure])


@pytest.mark.parametrize("d,precision,warps,cosets", [(11, "fp32", 8, 4), (13, "fp32", 8, 4), (13, "fp32", 8, 2),
                                                      (5, "fp32", 8, 4), (11, "fp64", 4, 2), (9, "fp64", 8, 2)])
def test_register_form_only_kernels_give_the_same_bits(dev, d, precision, warps, cosets):
    # The register-form-only variants (messages = 3: small per-warp buffers,
    # more CTAs per SM, no node-by-node code) run the same block updates as
    # the full kernel: every output bit for bit, early exit, initial and
    # exported messages included.  FP32 (8, 4) takes its 4-CTA variant at
    # d = 5 and 11 and its 3-CTA variant at d = 13 (shared memory).
    from paper_2402_04834_gb300 import warmstart as wsm
    _, _, S = synth.sample_syndromes(1500 + d, 0, 300, d, 0.1)
    s = torch.from_numpy(S).to(dev)
    M = wsm.message_count(pkg.DecoderParams(d=d, k=4, algorithm="fused"))
    init = torch.rand((300 * 4 * M, 16), generator=torch.Generator().manual_seed(d)).to(dev) + 0.01
    res = {}
    for mem in (1, 3):
        prm = pkg.DecoderParams(d=d, k=4, p=0.1, max_iter=15, delta0=1e-4, precision=precision, algorithm="fused",
                                warps=warps, cosets=cosets, messages=mem)
        final = torch.empty_like(init)
        res[mem] = (wsm.decode_ex(s, prm), wsm.decode_ex(s, prm, init_msgs=init, final_msgs=final), final)
    torch.cuda.synchronize()
    for i in range(2):
        for key in ("logp", "delta", "iters", "flags", "decision"):
            assert torch.equal(res[1][i][key], res[3][i][key]), (i, key)
    assert torch.equal(res[1][2], res[3][2])
    assert not torch.any(res[3][0]["flags"] & (1 << 16))     # no block outside the register forms
