"""The library built with device bounds checks (-DBLOCKBP_CHECKS): every
table index the kernels derive is tested before use, a failure flagged
(BBP_FLAG_CHECK) and the access skipped.  On valid workloads of every path
no check fires and the results are those of the default build.  Also the
always-on guard of mixed batches against a distance outside 2..d_max."""

import numpy as np
import pytest

import paper_2402_04834_gb300 as pkg
import synth
from paper_2402_04834_gb300 import _lib
from paper_2402_04834_gb300 import warmstart as wsm
from paper_2402_04834_gb300.build import build
from paper_2402_04834_gb300.decoder import decode_mixed, pack_mixed

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def libs():
    default, checked = build(), build(checks=True)
    yield default, checked
    _lib.use_library(None)


def both(libs, fn):
    res = []
    for path in libs:
        _lib.use_library(path)
        out = fn()
        torch.cuda.synchronize()
        res.append({k: v.cpu().numpy() for k, v in out.items()})
    assert b"checks" in _lib.lib().bbp_version()
    _lib.use_library(None)
    assert b"checks" not in _lib.lib().bbp_version()
    return res


def same(a, b, precision):
    assert not np.any(b["flags"] & _lib.FLAG_CHECK)
    assert not np.any(a["flags"] & _lib.FLAG_CHECK)
    if precision == "fp64":
        assert np.array_equal(a["iters"], b["iters"])
        assert np.max(np.abs(a["logp"] - b["logp"])) < 1e-10
    else:
        eq = a["iters"] == b["iters"]
        assert eq.mean() > 0.99
        assert np.max(np.abs(a["logp"][eq] - b["logp"][eq])) < 1e-4
    assert np.mean(a["decision"] == b["decision"]) > 0.99


CASES = [  # d, k, precision, algorithm, D, messages, warps, cosets
    (11, 4, "fp32", "fused", 8, 0, 0, 0), (13, 4, "fp32", "fused", 8, 0, 0, 0), (12, 4, "fp32", "fused", 8, 0, 0, 0),
    (11, 4, "fp32", "fused", 8, 1, 8, 4), (11, 4, "fp32", "fused", 8, 2, 8, 2), (9, 4, "fp64", "fused", 8, 0, 0, 0),
    (7, 4, "fp64", "fused", 8, 1, 4, 4), (7, 6, "fp32", "fused", 8, 0, 0, 0), (6, 2, "fp32", "fused", 8, 0, 0, 0),
    (4, 1, "fp64", "fused", 8, 0, 0, 0), (7, 4, "fp64", "mps", 8, 0, 0, 0), (5, 3, "fp32", "mps", 4, 0, 0, 0),
]


@pytest.mark.parametrize("d,k,precision,algorithm,D,messages,warps,cosets", CASES)
def test_no_check_fires_and_results_agree(libs, d, k, precision, algorithm, D, messages, warps, cosets):
    dev = torch.device("cuda:0")
    B = 64 if algorithm == "mps" else 500
    _, _, S = synth.sample_syndromes(9100 + d, 0, B, d, 0.1)
    s = torch.from_numpy(S).to(dev)
    prm = pkg.DecoderParams(d=d, k=k, D=D, p=0.1, max_iter=20, delta0=1e-4, precision=precision,
                            algorithm=algorithm, messages=messages, warps=warps, cosets=cosets)
    a, b = both(libs, lambda: pkg.decode(s, prm))
    same(a, b, precision)


def test_mixed_batch_and_learned_decoder_under_checks(libs):
    dev = torch.device("cuda:0")
    rng = np.random.default_rng(91)
    ds = rng.choice([7, 9, 13], size=120)
    shots = [synth.sample_syndromes(91, i, 1, int(d), 0.1)[2][0] for i, d in enumerate(ds)]
    packed, offsets, d_of = pack_mixed(shots, device=dev)
    prm = pkg.DecoderParams(d=0, k=4, p=0.1, max_iter=20, delta0=1e-4, precision="fp32", algorithm="fused")
    a, b = both(libs, lambda: decode_mixed(packed, offsets, d_of, prm))
    same(a, b, "fp32")
    _, _, S = synth.sample_syndromes(92, 0, 200, 11, 0.1)
    s = torch.from_numpy(S).to(dev)
    prm11 = pkg.DecoderParams(d=11, k=4, p=0.1, max_iter=20, delta0=1e-4, precision="fp32", algorithm="fused")
    net = wsm.WarmStart(device=dev, seed=5)
    a, b = both(libs, lambda: wsm.decode_warm(s, prm11, net, alpha=0.3))
    same(a, b, "fp32")


def test_mixed_batch_distance_beyond_d_max_is_flagged(libs):
    # The shared memory of a mixed launch is sized for d_max; a syndrome
    # whose distance (in a device buffer) exceeds it is not decoded: its rows
    # carry BBP_FLAG_CHECK and NaN, every other syndrome is decoded as usual.
    dev = torch.device("cuda:0")
    ds = [7, 9, 13, 9, 7, 13]
    shots = [synth.sample_syndromes(93, i, 1, d, 0.1)[2][0] for i, d in enumerate(ds)]
    packed, offsets, d_of = pack_mixed(shots, device=dev)
    prm = pkg.DecoderParams(d=0, k=4, p=0.1, max_iter=20, delta0=1e-4, precision="fp32", algorithm="fused")
    good = decode_mixed(packed, offsets, d_of, prm)
    cut = decode_mixed(packed, offsets, d_of, prm, d_max=9)
    torch.cuda.synchronize()
    big = np.array(ds) > 9
    fl = cut["flags"].cpu().numpy()
    assert np.all(fl[big] & _lib.FLAG_CHECK)
    assert np.all(np.isnan(cut["logp"].cpu().numpy()[big]))
    assert not np.any(fl[~big] & _lib.FLAG_CHECK)
    # the other syndromes: the same values (the launch shape is the one of d_max = 9, results do not depend on it)
    for key in ("logp", "delta", "iters", "decision"):
        assert np.array_equal(cut[key].cpu().numpy()[~big], good[key].cpu().numpy()[~big]), key
