"""Batching: mixed distances in one persistent launch, CUDA-graph capture,
autotuned launch shapes.  Results must not depend on any of them."""

import numpy as np
import pytest

import paper_2402_04834_gb300 as pkg
import synth
from oracle.lattice import Lattice
from oracle.naive import run_naive
from oracle.tn import coset_network
from paper_2402_04834_gb300 import autotune
from paper_2402_04834_gb300.build import build
from paper_2402_04834_gb300.decoder import decode_mixed, pack_mixed

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dev():
    build()
    pkg.lib()
    return torch.device("cuda:0")


def mixed_batch(B, dists, p, seed):
    rng = np.random.default_rng(seed)
    ds = rng.choice(dists, size=B)
    shots = []
    for b, d in enumerate(ds):
        _, _, S = synth.sample_syndromes(seed, b, 1, int(d), p)
        shots.append(S[0])
    return ds, shots


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_mixed_batch_equals_per_distance_decodes(dev, precision):
    p = 0.1
    ds, shots = mixed_batch(96, [3, 5, 7, 9, 11], p, 17)
    packed, offsets, d_of = pack_mixed(shots, device=dev)
    prm = pkg.DecoderParams(d=0, k=4, p=p, max_iter=8, delta0=1e-4, precision=precision, algorithm="fused")
    for largest_first in (True, False):
        out = decode_mixed(packed, offsets, d_of, prm, largest_first=largest_first)
        torch.cuda.synchronize()
        for d in sorted(set(ds.tolist())):
            idx = np.nonzero(ds == d)[0]
            S = np.stack([shots[i] for i in idx])
            ref = pkg.decode(torch.from_numpy(S).to(dev), pkg.DecoderParams(**{**prm.__dict__, "d": int(d)}))
            torch.cuda.synchronize()
            for key in ("logp", "delta", "iters", "flags", "decision"):
                assert torch.equal(out[key][torch.from_numpy(idx).to(dev)], ref[key]), (d, key)


def test_mixed_batch_matches_dense_oracle_on_a_sample(dev):
    p = 0.1
    ds, shots = mixed_batch(16, [3, 5, 7], p, 23)
    packed, offsets, d_of = pack_mixed(shots, device=dev)
    prm = pkg.DecoderParams(d=0, k=4, p=p, max_iter=5, delta0=0.0, precision="fp64", algorithm="fused")
    out = decode_mixed(packed, offsets, d_of, prm)
    torch.cuda.synchronize()
    for b in (0, 5, 11):
        d = int(ds[b])
        lat = Lattice(d)
        for L in range(4):
            lp, _, _, _ = run_naive(coset_network(lat, shots[b], L, p), 4, 5, 0.1, 0.0)
            assert abs(out["logp"][b, L].item() - lp) < 1e-9


def test_cuda_graph_capture_replays_the_decode(dev):
    d, p = 11, 0.1
    prm = pkg.DecoderParams(d=d, k=4, p=p, max_iter=20, delta0=1e-4, precision="fp32", algorithm="fused")
    _, _, S1 = synth.sample_syndromes(31, 0, 512, d, p)
    _, _, S2 = synth.sample_syndromes(32, 0, 512, d, p)
    s_static = torch.from_numpy(S1).to(dev)
    out = pkg.decode(s_static, prm)                      # warm up: buffers exist before capture
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    stream = torch.cuda.Stream()
    stream.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(stream):
        with torch.cuda.graph(g, stream=stream):
            pkg.decode(s_static, prm, out=out, stream=stream)
    torch.cuda.current_stream().wait_stream(stream)
    for S in (S2, S1):
        s_static.copy_(torch.from_numpy(S).to(dev))
        g.replay()
        torch.cuda.synchronize()
        ref = pkg.decode(torch.from_numpy(S).to(dev), prm)
        torch.cuda.synchronize()
        for key in ("logp", "iters", "decision"):
            assert torch.equal(out[key], ref[key]), key


def test_cuda_graph_capture_replays_the_mixed_decode(dev):
    # The persistent mixed-distance launch (counter reset, kernel, decision)
    # captured once and replayed on new syndromes of the same shapes.
    p = 0.1
    ds, shots1 = mixed_batch(64, [5, 7, 9, 11], p, 61)
    shots2 = [synth.sample_syndromes(62, b, 1, int(d), p)[2][0] for b, d in enumerate(ds)]
    packed, offsets, d_of = pack_mixed(shots1, device=dev)
    packed2, _, _ = pack_mixed(shots2, device=dev)
    prm = pkg.DecoderParams(d=0, k=4, p=p, max_iter=12, delta0=1e-4, precision="fp32", algorithm="fused")
    order = torch.argsort(d_of, descending=True, stable=True).to(torch.int32)
    counter = torch.empty(256, dtype=torch.uint8, device=dev)
    out = decode_mixed(packed, offsets, d_of, prm, counter=counter, order=order, d_max=11)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    stream = torch.cuda.Stream()
    stream.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(stream):
        with torch.cuda.graph(g, stream=stream):
            decode_mixed(packed, offsets, d_of, prm, counter=counter, order=order, d_max=11, out=out, stream=stream)
    torch.cuda.current_stream().wait_stream(stream)
    src = packed.clone()
    for new in (packed2, src):
        packed.copy_(new)
        g.replay()
        torch.cuda.synchronize()
        ref = decode_mixed(new, offsets, d_of, prm)
        torch.cuda.synchronize()
        for key in ("logp", "delta", "iters", "flags", "decision"):
            assert torch.equal(out[key], ref[key]), key


def test_autotuned_shapes_give_identical_results(dev):
    d, p = 9, 0.1
    _, _, S = synth.sample_syndromes(41, 0, 256, d, p)
    s = torch.from_numpy(S).to(dev)
    prm = pkg.DecoderParams(d=d, k=4, p=p, max_iter=10, precision="fp32", algorithm="fused")
    best, table = autotune.tune_uniform(s, prm)
    cands = autotune.candidates(prm)
    assert len(table) == len(cands) and (best.warps, best.cosets, best.messages) in cands
    ref = pkg.decode(s, prm)
    for w, c, mem in cands:
        got = pkg.decode(s, pkg.DecoderParams(**{**prm.__dict__, "warps": w, "cosets": c, "messages": mem}))
        torch.cuda.synchronize()
        for key in ("logp", "delta", "iters", "flags"):
            assert torch.equal(got[key], ref[key]), (w, c, mem, key)
    ds, shots = mixed_batch(128, [7, 9, 13], p, 5)
    packed, offsets, d_of = pack_mixed(shots, device=dev)
    mp = pkg.DecoderParams(d=0, k=4, p=p, max_iter=10, precision="fp32", algorithm="fused")
    best, table = autotune.tune_mixed(packed, offsets, d_of, mp, shapes=((8, 4, 1), (8, 4, 2), (8, 2, 1), (8, 1, 1)),
                                      ctas=(0, 2))
    assert len(table) >= 2
    a = decode_mixed(packed, offsets, d_of, best)
    b = decode_mixed(packed, offsets, d_of, mp)
    torch.cuda.synchronize()
    assert torch.equal(a["logp"], b["logp"])


def test_mixed_workload_4096_over_five_distances(dev):
    # 4096 syndromes, d uniform over {7, 9, 13, 17, 21}, p = 0.10, one
    # persistent launch with the autotuned shape, captured in a CUDA graph.
    p = 0.10
    ds, shots = mixed_batch(4096, [7, 9, 13, 17, 21], p, 3000)
    packed, offsets, d_of = pack_mixed(shots, device=dev)
    prm = pkg.DecoderParams(d=0, k=4, p=p, max_iter=20, delta0=1e-4, precision="fp32", algorithm="fused")
    best, table = autotune.tune_mixed(packed, offsets, d_of, prm, shapes=((8, 4, 1), (8, 4, 2), (8, 2, 1), (8, 1, 1)),
                                      ctas=(0, 2))
    out = decode_mixed(packed, offsets, d_of, best)
    torch.cuda.synchronize()
    counter = torch.empty(256 + pkg.workspace_bytes(pkg.DecoderParams(**{**best.__dict__, "d": 21}), len(shots)),
                          dtype=torch.uint8, device=dev)
    g = torch.cuda.CUDAGraph()
    stream = torch.cuda.Stream()
    stream.wait_stream(torch.cuda.current_stream())
    order = torch.argsort(d_of, descending=True, stable=True).to(torch.int32)
    d_max = int(d_of.max().item())
    with torch.cuda.stream(stream):
        graph_out = decode_mixed(packed, offsets, d_of, best, stream=stream, counter=counter, order=order,
                                 d_max=d_max)
        torch.cuda.current_stream(dev).synchronize()
        with torch.cuda.graph(g, stream=stream):
            decode_mixed(packed, offsets, d_of, best, stream=stream, out=graph_out, counter=counter, order=order,
                         d_max=d_max)
    torch.cuda.current_stream().wait_stream(stream)
    g.replay()
    torch.cuda.synchronize()
    for key in ("logp", "iters", "decision"):
        assert torch.equal(graph_out[key], out[key]), key
    # Per-distance decodes give the same bits.
    for d in (7, 21):
        idx = np.nonzero(ds == d)[0][:64]
        S = np.stack([shots[i] for i in idx])
        ref = pkg.decode(torch.from_numpy(S).to(dev), pkg.DecoderParams(**{**best.__dict__, "d": d, "ctas_per_sm": 0}))
        torch.cuda.synchronize()
        assert torch.equal(out["logp"][torch.from_numpy(idx).to(dev)], ref["logp"])
    assert (out["decision"] >= 0).all() and (out["decision"] < 4).all()


@pytest.mark.parametrize("precision,warps,cosets", [("fp32", 8, 4), ("fp32", 8, 2), ("fp64", 4, 2)])
def test_register_form_only_mixed_batch_of_odd_distances(dev, precision, warps, cosets):
    # A batch whose distances are all odd may take the register-form-only
    # kernels (launch_messages = 3): the same bits as per-distance decodes.
    p = 0.1
    ds, shots = mixed_batch(120, [5, 7, 9, 11, 13], p, 41)
    packed, offsets, d_of = pack_mixed(shots, device=dev)
    prm = pkg.DecoderParams(d=0, k=4, p=p, max_iter=12, delta0=1e-4, precision=precision, algorithm="fused",
                            warps=warps, cosets=cosets, messages=3)
    out = decode_mixed(packed, offsets, d_of, prm)
    torch.cuda.synchronize()
    for d in sorted(set(ds.tolist())):
        idx = np.nonzero(ds == d)[0]
        S = np.stack([shots[i] for i in idx])
        ref = pkg.decode(torch.from_numpy(S).to(dev), pkg.DecoderParams(**{**prm.__dict__, "d": int(d),
                                                                            "messages": 0, "warps": 0, "cosets": 0}))
        torch.cuda.synchronize()
        for key in ("logp", "delta", "iters", "flags", "decision"):
            assert torch.equal(out[key][torch.from_numpy(idx).to(dev)], ref[key]), (d, key)


def test_register_form_only_mixed_batch_flags_an_even_distance(dev):
    # The caller vouches for odd distances; a syndrome of even distance in
    # such a batch is flagged (BBP_FLAG_CAPACITY), the others are decoded as
    # usual; an even d_max is refused on the host.
    from paper_2402_04834_gb300 import _lib
    p = 0.1
    ds = [7, 8, 9, 7, 9, 8]
    shots = [synth.sample_syndromes(43, i, 1, d, p)[2][0] for i, d in enumerate(ds)]
    packed, offsets, d_of = pack_mixed(shots, device=dev)
    lean = pkg.DecoderParams(d=0, k=4, p=p, max_iter=12, delta0=1e-4, precision="fp32", algorithm="fused",
                             messages=3)
    out = decode_mixed(packed, offsets, d_of, lean)
    full = decode_mixed(packed, offsets, d_of, pkg.DecoderParams(**{**lean.__dict__, "messages": 0}))
    torch.cuda.synchronize()
    even = np.array(ds) % 2 == 0
    fl = out["flags"].cpu().numpy()
    assert np.all(fl[even] & _lib.FLAG_CAPACITY)
    assert not np.any(fl[~even] & _lib.FLAG_CAPACITY)
    for key in ("logp", "delta", "iters", "decision"):
        assert np.array_equal(out[key].cpu().numpy()[~even], full[key].cpu().numpy()[~even]), key
    with pytest.raises(pkg.BbpError):
        decode_mixed(packed, offsets, d_of, lean, d_max=10)
