"""bbp_decode_batch_static: the decode for callers that cannot allocate.

Real-time decoding loops that must not take the allocator's locks or run
out of memory mid-run, and hosts that own only the input and output buffers,
cannot give the decoder a workspace.  This
entry point keeps the message arena in a fixed device array inside the
library instead.  Here it is called through the C ABI and must reproduce the
workspace-taking entry point on two calls in a row (the second call reuses
the array the first one left behind), and refuse a batch that does not fit.
The file is named so that pytest collects it last.
"""

import ctypes

import numpy as np
import pytest

import paper_2402_04834_gb300 as pkg
import synth
from paper_2402_04834_gb300 import _lib
from paper_2402_04834_gb300.build import build

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu


def _static_decode(S_dev, prm):
    """Call bbp_decode_batch_static with caller-owned device buffers only."""
    B = S_dev.shape[0]
    dev = S_dev.device
    out = {
        "logp": torch.empty(B, 4, dtype=torch.float64, device=dev),
        "delta": torch.empty(B, 4, dtype=torch.float64, device=dev),
        "iters": torch.empty(B, 4, dtype=torch.int32, device=dev),
        "flags": torch.empty(B, 4, dtype=torch.int32, device=dev),
        "decision": torch.empty(B, dtype=torch.int8, device=dev),
    }
    cp = prm.c()
    rc = pkg.lib().bbp_decode_batch_static(
        S_dev.data_ptr(), B, ctypes.byref(cp), out["logp"].data_ptr(), out["delta"].data_ptr(),
        out["iters"].data_ptr(), out["flags"].data_ptr(), out["decision"].data_ptr(),
        torch.cuda.current_stream(dev).cuda_stream)
    return rc, out


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_static_entry_point_matches_workspace_entry_point(precision):
    build()
    dev = torch.device("cuda:0")
    d, p = 11, 0.10
    prm = pkg.DecoderParams(d=d, k=4, D=8, p=p, max_iter=6, delta0=0.0, precision=precision)
    _, _, S = synth.sample_syndromes(synth.workload_seed(2, 2), 0, 96, d, p)
    S_dev = torch.from_numpy(S).to(dev)
    ref = pkg.decode(S_dev, prm)
    torch.cuda.synchronize()
    ref = {k: v.cpu().numpy() for k, v in ref.items()}
    for call in range(2):
        rc, out = _static_decode(S_dev, prm)
        assert rc == 0, pkg.lib().bbp_strerror(rc)
        torch.cuda.synchronize()
        got = {k: v.cpu().numpy() for k, v in out.items()}
        tol = 1e-9 if precision == "fp64" else 1e-3
        np.testing.assert_allclose(got["logp"], ref["logp"], rtol=0, atol=tol, err_msg=f"call {call}")
        np.testing.assert_allclose(got["delta"], ref["delta"], rtol=0, atol=1e-7)
        assert np.array_equal(got["iters"], ref["iters"])
        assert np.array_equal(got["flags"], ref["flags"])
        assert np.array_equal(got["decision"], ref["decision"])


def test_static_entry_point_refuses_batches_beyond_its_array():
    build()
    dev = torch.device("cuda:0")
    prm = pkg.DecoderParams(d=11, k=4, D=8, p=0.1, max_iter=2, precision="fp64")
    B = 1024                                    # needs 127 MiB > 32 MiB
    assert pkg.workspace_bytes(prm, B) > _lib.STATIC_WORKSPACE_BYTES
    S_dev = torch.zeros(B, prm.m, dtype=torch.uint8, device=dev)
    rc, _ = _static_decode(S_dev, prm)
    assert rc == _lib.BBP_ETOOLARGE


def test_static_entry_point_takes_the_shared_memory_shape_when_slots_do_not_fit():
    # Fused k = 4 at d = 19: the default shape keeps its messages in
    # workspace slots (600 syndromes: 512 slots of 4 x 360 x 16 floats =
    # 47.2 MB > 32 MiB), so the static entry point takes the shape that
    # keeps them in shared memory; the results are those of the allocating
    # entry point bit for bit.
    build()
    dev = torch.device("cuda:0")
    d, B = 19, 600
    prm = pkg.DecoderParams(d=d, k=4, p=0.1, max_iter=6, delta0=1e-4, precision="fp32", algorithm="fused")
    assert pkg.workspace_bytes(prm, B) > _lib.STATIC_WORKSPACE_BYTES
    _, _, S = synth.sample_syndromes(2121, 0, B, d, 0.1)
    S_dev = torch.from_numpy(S).to(dev)
    ref = pkg.decode(S_dev, prm)
    rc, out = _static_decode(S_dev, prm)
    assert rc == 0, pkg.lib().bbp_strerror(rc)
    torch.cuda.synchronize()
    for key in ("logp", "delta", "iters", "flags", "decision"):
        assert torch.equal(out[key], ref[key]), key
