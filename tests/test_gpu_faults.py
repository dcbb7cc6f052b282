"""Failure handling, injected from the host (no GPU fault): unusable initial
messages (NaN, all zero) fall back to the uniform start of Remark 2 per
(coset, message); a coset that never meets Delta < delta1 is flagged and the
decision falls back to the smallest Delta (Remark 6)."""

import numpy as np
import pytest

import paper_2402_04834_gb300 as pkg
import synth
from paper_2402_04834_gb300 import warmstart as wsm
from paper_2402_04834_gb300.build import build

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

FLAG_UNTRUSTED = 1          # BBP_FLAG_UNTRUSTED


@pytest.fixture(scope="module")
def dev():
    build()
    pkg.lib()
    return torch.device("cuda:0")


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_unusable_initial_messages_fall_back_to_uniform(dev, precision):
    d, p, B = 7, 0.1, 8
    _, _, S = synth.sample_syndromes(4242, 0, B, d, p)
    s = torch.from_numpy(S).to(dev)
    prm = pkg.DecoderParams(d=d, k=4, p=p, max_iter=12, delta0=0.0, precision=precision, algorithm="fused")
    M = wsm.message_count(prm)
    cold = wsm.decode_ex(s, prm)
    nan = torch.full((B * 4 * M, 16), float("nan"), device=dev)
    zero = torch.zeros((B * 4 * M, 16), device=dev)
    for init in (nan, zero):
        out = wsm.decode_ex(s, prm, init_msgs=init)
        for key in ("logp", "delta", "iters", "flags", "decision"):
            assert torch.equal(out[key], cold[key]), key
    # Some rows unusable among usable ones: NaN and zero rows take the same path.
    g = torch.Generator(device="cpu").manual_seed(5)
    prop = torch.rand((B * 4 * M, 16), generator=g).to(dev) + 0.05
    bad = torch.rand(B * 4 * M, generator=g) < 0.3
    with_nan, with_zero = prop.clone(), prop.clone()
    with_nan[bad.to(dev)] = float("nan")
    with_zero[bad.to(dev)] = 0.0
    a = wsm.decode_ex(s, prm, init_msgs=with_nan)
    b = wsm.decode_ex(s, prm, init_msgs=with_zero)
    torch.cuda.synchronize()
    for key in ("logp", "delta", "iters", "flags", "decision"):
        assert torch.equal(a[key], b[key]), key
    assert torch.isfinite(a["logp"]).all()


def test_untrusted_cosets_are_flagged_and_decided_by_smallest_delta(dev):
    # One iteration cannot bring Delta below delta1 = 1e-6 anywhere: every
    # coset is flagged untrusted, and the decision is the coset of smallest Delta.
    d, p, B = 9, 0.12, 32
    _, _, S = synth.sample_syndromes(4343, 0, B, d, p)
    prm = pkg.DecoderParams(d=d, k=4, p=p, max_iter=1, delta0=0.0, delta1=1e-6, precision="fp32",
                            algorithm="fused")
    out = pkg.decode(torch.from_numpy(S).to(dev), prm)
    torch.cuda.synchronize()
    flags = out["flags"].cpu().numpy()
    delta = out["delta"].cpu().numpy()
    assert np.all(flags & FLAG_UNTRUSTED)
    assert np.array_equal(out["decision"].cpu().numpy(), np.argmin(delta, axis=1))
