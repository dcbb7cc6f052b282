"""GPU parity: the CUDA path through the C ABI against the CPU oracle.

Tolerances (written from the arithmetic): FP64 |d log P| <= 1e-9 per coset
(the target of the decoder); Delta within 1e-7 absolute (Delta is
sqrt(sum 2 - 2<a|b>^2)/M, which cancels near convergence and carries
~sqrt(M eps)/M of rounding); decisions identical wherever the oracle's
log-likelihood margin among eligible cosets exceeds 1e-2.  FP32
|d log P| <= 1e-3.  Shots whose oracle run met a near-degenerate truncation
(relative Schmidt gap <= 1e-8) may legitimately keep a different subspace
and are only checked for validity.
"""

import json
import math
import os

import numpy as np
import pytest

import paper_2402_04834_gb300 as pkg
import synth
from oracle import blockbp as bb
from oracle.lattice import Lattice
from paper_2402_04834_gb300.build import build

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu
HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def dev():
    build()
    pkg.lib()
    return torch.device("cuda:0")


def load_golden(name):
    with open(os.path.join(HERE, "golden", name)) as f:
        return json.load(f)


def margin(logp, flags):
    el = sorted((logp[i] for i in range(4) if flags[i] == 0), reverse=True)
    return el[0] - el[1] if len(el) >= 2 else math.inf


def gpu_decode(S, prm, dev):
    out = pkg.decode(torch.from_numpy(np.ascontiguousarray(S)).to(dev), prm)
    torch.cuda.synchronize()
    return {k: v.cpu().numpy() for k, v in out.items()}


def compare(out, rows, offset, tol_logp, check_iters=True, tol_delta=1e-7):
    n_checked = 0
    for r in rows:
        b = r["shot"] - offset
        gap = r["min_gap"]
        degenerate = gap is not None and gap <= 1e-8
        lp = np.array(r["logp"])
        if not degenerate:
            np.testing.assert_allclose(out["logp"][b], lp, rtol=0, atol=tol_logp, err_msg=f"shot {r['shot']}")
            np.testing.assert_allclose(out["delta"][b], r["delta"], rtol=0, atol=tol_delta)
            if check_iters:
                assert list(out["iters"][b]) == r["iters"]
            if margin(r["logp"], r["flags"]) > 1e-2 and list(out["flags"][b]) == r["flags"]:
                assert int(out["decision"][b]) == r["decision"], f"shot {r['shot']}"
            n_checked += 1
        assert 0 <= int(out["decision"][b]) < 4
    return n_checked


def test_sampler_bit_exact_with_workload_module(dev):
    for d in (3, 5, 11):
        ex, ez, s, tc = pkg.sample(1234, 7, 64, d, 0.1, device=dev)
        torch.cuda.synchronize()
        rx, rz, rs = synth.sample_syndromes(1234, 7, 64, d, 0.1)
        assert np.array_equal(ex.cpu().numpy(), rx)
        assert np.array_equal(ez.cpu().numpy(), rz)
        assert np.array_equal(s.cpu().numpy(), rs)
        lat = Lattice(d)
        tcn = tc.cpu().numpy()
        for b in range(16):
            assert tcn[b] == lat.true_class(rx[b], rz[b], rs[b])


def test_fp64_parity_d5_config(dev):
    g = load_golden("oracle_d5_k3_D4_p010.json")
    w = g["workload"]
    _, _, S = synth.sample_syndromes(w["seed"], w["first_shot"], w["shots"], w["d"], w["p"])
    prm = pkg.DecoderParams(d=w["d"], k=w["k"], D=w["D"], p=w["p"], max_iter=w["max_iter"],
                            delta0=w["delta0"], precision="fp64")
    out = gpu_decode(S, prm, dev)
    assert compare(out, g["shots"], w["first_shot"], 1e-9) == w["shots"]


def test_fp64_parity_d11_config(dev):
    g = load_golden("oracle_d11_k4_D8_p010.json")
    w = g["workload"]
    _, _, S = synth.sample_syndromes(w["seed"], w["first_shot"], w["shots"], w["d"], w["p"])
    prm = pkg.DecoderParams(d=w["d"], k=w["k"], D=w["D"], p=w["p"], max_iter=w["max_iter"],
                            delta0=w["delta0"], precision="fp64")
    out = gpu_decode(S, prm, dev)
    assert compare(out, g["shots"], w["first_shot"], 1e-9) >= len(g["shots"]) - 1


@pytest.mark.parametrize("d,k,D,iters,p", [
    (3, 2, 4, 5, 0.1),     # W = 5: blocks 2, 2, 1 (ragged tail)
    (4, 3, 2, 4, 0.12),    # W = 7: blocks 3, 3, 1; D = 2 truncates
    (5, 4, 8, 5, 0.1),     # W = 9: blocks 4, 4, 1
    (7, 4, 2, 4, 0.08),    # W = 13: blocks 4, 4, 4, 1; D = 2 truncates
    (7, 3, 2, 3, 0.08),    # W = 13: blocks 3, 3, 3, 3, 1
    (2, 3, 4, 3, 0.2),     # W = 3: one block, no messages (bMPS limit)
])
def test_fp64_parity_ragged_live_oracle(dev, d, k, D, iters, p):
    _, _, S = synth.sample_syndromes(4242, 0, 3, d, p)
    prm = pkg.DecoderParams(d=d, k=k, D=D, p=p, max_iter=iters, delta0=0.0)
    out = gpu_decode(S, prm, dev)
    rows = []
    for b in range(S.shape[0]):
        r = bb.decode(S[b], bb.Params(d=d, k=k, D=D, p=p, max_iter=iters, delta0=0.0))
        st = r["stats"]
        rows.append(dict(shot=b, logp=list(r["logp"]), delta=list(r["delta"]), iters=list(r["iters"]),
                         flags=list(r["flags"]), decision=r["decision"],
                         min_gap=None if not np.isfinite(st.min_gap) else st.min_gap))
    assert compare(out, rows, 0, 1e-9) >= 1


def test_fp64_early_exit_matches_oracle(dev):
    d, k, D, p = 5, 3, 4, 0.06
    _, _, S = synth.sample_syndromes(99, 0, 4, d, p)
    prm = pkg.DecoderParams(d=d, k=k, D=D, p=p, max_iter=40, delta0=1e-4)
    out = gpu_decode(S, prm, dev)
    for b in range(4):
        r = bb.decode(S[b], bb.Params(d=d, k=k, D=D, p=p, max_iter=40, delta0=1e-4))
        for L in range(4):
            # Delta is compared against delta0 on both sides; only a Delta within
            # rounding of delta0 could exit on a different iteration.
            if abs(r["cosets"][L].delta - 1e-4) > 1e-6:
                assert out["iters"][b][L] == r["iters"][L]
                assert abs(out["logp"][b][L] - r["logp"][L]) < 1e-9


def mps_fp32_bar(r):
    """Per-shot cap of the FP32 MPS form: 1e-2, or four times how far the
    same steps run in float32 (numpy / LAPACK single precision) end from the
    float64 oracle, where that is larger.  The MPS form compresses every
    message by QR and SVD; in single precision the compressed messages keep
    directions only down to a few units of rounding of their largest Schmidt
    value, and where a read-out overlap is small that reaches 1e-3 in log P
    and more for any single-precision implementation of the method (the
    float32 oracle misses 1e-3 on 3 of the 200 benchmark shots, and by up to
    2.6e-2 at p = 0.08, and on 4 of 50 shots at p = 0.05).  The 1e-3 bar
    itself is required on 90 % of the shots (MPS_FP32_SHARE); the fused
    form, the decoder of the benchmark, meets it on every shot."""
    return max(1e-2, 4.0 * r["dlogp_fp32"])


MPS_FP32_SHARE = 0.90


def test_fp32_within_reduced_precision_tolerance(dev):
    for name in ("oracle_d5_k3_D4_p010.json", "oracle_d11_k4_D8_p010.json"):
        g = load_golden(name)
        w = g["workload"]
        _, _, S = synth.sample_syndromes(w["seed"], w["first_shot"], w["shots"], w["d"], w["p"])
        prm = pkg.DecoderParams(d=w["d"], k=w["k"], D=w["D"], p=w["p"], max_iter=w["max_iter"],
                                delta0=w["delta0"], precision="fp32")
        out = gpu_decode(S, prm, dev)
        n_strict = 0
        for r in g["shots"]:
            b = r["shot"] - w["first_shot"]
            err = np.max(np.abs(out["logp"][b] - np.array(r["logp"])))
            assert err <= mps_fp32_bar(r), (name, r["shot"], err, r["dlogp_fp32"])
            n_strict += err <= 1e-3
            if margin(r["logp"], r["flags"]) > 1e-2 and list(out["flags"][b]) == r["flags"]:
                assert int(out["decision"][b]) == r["decision"]
        assert n_strict >= MPS_FP32_SHARE * len(g["shots"]), (name, n_strict)


def test_host_entry_point_matches_device_entry_point(dev):
    _, _, S = synth.sample_syndromes(5, 0, 9, 5, 0.1)
    prm = pkg.DecoderParams(d=5, k=3, D=4, p=0.1, max_iter=6, delta0=0.0)
    a = gpu_decode(S, prm, dev)
    h = pkg.decode_host(S, prm, device=dev)
    for key in ("logp", "delta", "iters", "flags", "decision"):
        assert np.array_equal(a[key], h[key]), key


def test_deterministic_reruns(dev):
    _, _, S = synth.sample_syndromes(6, 0, 16, 7, 0.1)
    prm = pkg.DecoderParams(d=7, k=4, D=8, p=0.1, max_iter=5, delta0=0.0)
    a = gpu_decode(S, prm, dev)
    b = gpu_decode(S, prm, dev)
    for key in a:
        assert np.array_equal(a[key], b[key]), key


def test_zero_syndrome_and_single_shot(dev):
    d = 5
    S = np.zeros((1, 2 * d * (d - 1)), dtype=np.uint8)
    prm = pkg.DecoderParams(d=d, k=3, D=4, p=0.05, max_iter=8, delta0=0.0)
    out = gpu_decode(S, prm, dev)
    assert int(out["decision"][0]) == 0
    r = bb.decode(S[0], bb.Params(d=d, k=3, D=4, p=0.05, max_iter=8, delta0=0.0))
    np.testing.assert_allclose(out["logp"][0], r["logp"], rtol=0, atol=1e-9)


def test_full_size_batch_in_bench_configuration(dev):
    # The benchmark's batch and kernel: 10^4 syndromes at d = 11, p = 0.10,
    # k = 4, decoded by the fused FP32 kernel in one launch (the launch shape
    # the benchmark times); the first 200 shots are compared with the oracle.
    g = load_golden("oracle_d11_k4_D8_p010.json")
    w = g["workload"]
    B = 10000
    _, _, S = synth.sample_syndromes(w["seed"], 0, B, w["d"], w["p"])
    prm = pkg.DecoderParams(d=w["d"], k=w["k"], D=w["D"], p=w["p"], max_iter=w["max_iter"],
                            delta0=w["delta0"], precision="fp32", algorithm="fused")
    out = gpu_decode(S, prm, dev)
    for r in g["shots"]:
        b = r["shot"]
        assert np.max(np.abs(out["logp"][b] - np.array(r["logp"]))) <= 1e-3
    # Properties at any size: valid decisions, probabilities <= 1, finite logs.
    assert np.all((out["decision"] >= 0) & (out["decision"] < 4))
    assert np.all(out["iters"] == w["max_iter"])
    fin = np.isfinite(out["logp"])
    assert fin.mean() > 0.999
    lse = np.log(np.sum(np.exp(np.where(fin, out["logp"], -np.inf)), axis=1))
    assert np.all(lse < 1e-6)


_NOISE_CASES = [(pn, prec, alg, tol) for pn in ("p005", "p008", "p013", "p015")
                for prec, alg, tol in (("fp64", "mps", 1e-9), ("fp32", "mps", 1e-3), ("fp32", "fused", 1e-3))]


@pytest.mark.parametrize("pname,prec,alg,tol", _NOISE_CASES, ids=[f"{c[0]}-{c[1]}-{c[2]}" for c in _NOISE_CASES])
def test_d11_other_noise_levels(dev, pname, prec, alg, tol):
    # d = 11 workload at the other noise levels against the FP64 oracle:
    # FP64 MPS to 1e-9, the FP32 forms to 1e-3.
    g = load_golden(f"oracle_d11_k4_D8_{pname}.json")
    w = g["workload"]
    _, _, S = synth.sample_syndromes(w["seed"], w["first_shot"], w["shots"], w["d"], w["p"])
    prm = pkg.DecoderParams(d=w["d"], k=w["k"], D=w["D"], p=w["p"], max_iter=w["max_iter"],
                            delta0=w["delta0"], precision=prec, algorithm=alg)
    out = gpu_decode(S, prm, dev)
    n_strict = n = 0
    for r in g["shots"]:
        if r["truncations"] and alg == "fused":
            continue          # the fused form equals the MPS form only without truncation
        b = r["shot"] - w["first_shot"]
        err = np.max(np.abs(out["logp"][b] - np.array(r["logp"])))
        bar = mps_fp32_bar(r) if (prec, alg) == ("fp32", "mps") else tol
        assert err <= bar, (pname, prec, alg, r["shot"], err)
        n_strict += err <= tol
        n += 1
    if (prec, alg) == ("fp32", "mps"):
        assert n_strict >= MPS_FP32_SHARE * n, (pname, n_strict, n)


def test_headline_workload_every_form_on_200_shots(dev):
    # The benchmark's workload (d = 11, p = 0.10, k = 4, 20 fixed
    # iterations) on 200 shots of the dense fused-block oracle (Remark 9),
    # element by element: the fused form in FP64 to 1e-9 and in FP32 to
    # 1e-3, decisions wherever the oracle's margin exceeds 1e-2.
    g = load_golden("oracle_d11_k4_fused_p010.json")
    w = g["workload"]
    assert w["shots"] >= 200
    _, _, S = synth.sample_syndromes(w["seed"], w["first_shot"], w["shots"], w["d"], w["p"])
    for prec, tol, tol_delta in (("fp64", 1e-9, 1e-7), ("fp32", 1e-3, 1e-4)):
        prm = pkg.DecoderParams(d=w["d"], k=w["k"], D=w["D"], p=w["p"], max_iter=w["max_iter"],
                                delta0=w["delta0"], precision=prec, algorithm="fused")
        out = gpu_decode(S, prm, dev)
        assert compare(out, g["shots"], w["first_shot"], tol, tol_delta=tol_delta) == w["shots"], prec


# Truncating MPS workloads: a 4 x 4 block needs an in-block bond of up to 16,
# so D = 4 truncates inside every block and D = 2 also truncates the
# messages.  Whether two correct implementations can agree closely there
# depends on the shot: near-degenerate cuts, and at D = 2 a BP iteration
# that does not settle, amplify rounding.  The golden file records how far
# the oracle's own log P moves when every matrix it decomposes carries
# relative noise of 1e-13 (sens_fp64) or 1e-6 (sens_fp32), about what
# separates two correct decompositions in each precision.  A shot is compared
# at 1e-9 in FP64 where sens_fp64 <= 1e-10, and at 1e-3 in FP32 where both
# sens_fp32 and sens_fp64 are <= 1e-4 (a chaotic shot can move far under
# either noise); every other shot is checked for validity (a decision among
# the four cosets).
_TRUNC = [(d, D, prec) for d in (9, 11) for D in (2, 4) for prec in ("fp64", "fp32")]
# Shots of each golden file that meet the bar (a count of the oracle's own
# records): at D = 4 nearly all; at D = 2 the truncated iteration does not
# settle within 20 iterations and only a few shots are stable under noise.
MIN_COMPARED = {(9, 2, "fp64"): 1, (9, 2, "fp32"): 4, (11, 2, "fp64"): 0, (11, 2, "fp32"): 1,
                (9, 4, "fp64"): 24, (9, 4, "fp32"): 17, (11, 4, "fp64"): 24, (11, 4, "fp32"): 19}


@pytest.mark.parametrize("d,D,prec", _TRUNC, ids=[f"d{c[0]}-D{c[1]}-{c[2]}" for c in _TRUNC])
def test_truncating_mps_parity(dev, d, D, prec):
    g = load_golden(f"oracle_d{d}_k4_D{D}_p010.json")
    w = g["workload"]
    _, _, S = synth.sample_syndromes(w["seed"], w["first_shot"], w["shots"], w["d"], w["p"])
    prm = pkg.DecoderParams(d=w["d"], k=w["k"], D=w["D"], p=w["p"], max_iter=w["max_iter"],
                            delta0=w["delta0"], precision=prec)
    out = gpu_decode(S, prm, dev)
    assert all(r["truncations"] > 0 for r in g["shots"])
    sens, bar, tol = ("sens_fp64", 1e-10, 1e-9) if prec == "fp64" else ("sens_fp32", 1e-4, 1e-3)
    n = 0
    for r in g["shots"]:
        b = r["shot"] - w["first_shot"]
        assert 0 <= int(out["decision"][b]) < 4
        if max(r[sens], r["sens_fp64"]) > bar:
            continue
        err = np.max(np.abs(out["logp"][b] - np.array(r["logp"])))
        assert err <= (tol if prec == "fp64" else mps_fp32_bar(r)), (r["shot"], err, r[sens])
        n += 1
    assert n >= MIN_COMPARED[(d, D, prec)], n
