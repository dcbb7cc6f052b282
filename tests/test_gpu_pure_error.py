"""The pure error f_s on the device (Algorithm 1, first step) against the
oracle's construction, bit for bit, and the defining property s(f_s) = s."""

import numpy as np
import pytest

import paper_2402_04834_gb300 as pkg
import synth
from oracle.lattice import Lattice
from paper_2402_04834_gb300.build import build

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dev():
    build()
    pkg.lib()
    return torch.device("cuda:0")


@pytest.mark.parametrize("d,B", [(2, 16), (3, 64), (5, 40), (11, 12), (31, 3)])
def test_pure_error_equals_oracle_and_reproduces_the_syndrome(dev, d, B):
    rng = np.random.default_rng(900 + d)
    S = rng.integers(0, 2, size=(B, 2 * d * (d - 1)), dtype=np.uint8)    # arbitrary syndromes
    fx, fz = pkg.pure_error(torch.from_numpy(S).to(dev), d)
    torch.cuda.synchronize()
    fx, fz = fx.cpu().numpy(), fz.cpu().numpy()
    lat = Lattice(d)
    for b in range(B):
        ox, oz = lat.pure_error(S[b])
        assert np.array_equal(fx[b], ox) and np.array_equal(fz[b], oz), b
    assert np.array_equal(synth.syndromes_of(fx, fz, d), S)


def test_pure_error_of_sampled_syndromes_and_the_true_class(dev):
    # e f_s is in the centraliser: its syndrome vanishes, and its logical
    # part is the sampler's true class.
    d = 9
    ex, ez, s, tc = pkg.sample(77, 0, 256, d, 0.12, device=dev)
    fx, fz = pkg.pure_error(s, d)
    torch.cuda.synchronize()
    cx = (ex ^ fx).cpu().numpy()
    cz = (ez ^ fz).cpu().numpy()
    assert not synth.syndromes_of(cx, cz, d).any()
    lat = Lattice(d)
    xb, zb = lat.logical_bits()
    for b in range(256):
        bx = int(np.dot(cx[b].astype(int), zb) & 1)     # X-bar part: anticommutes with Z-bar
        bz = int(np.dot(cz[b].astype(int), xb) & 1)
        want = (2 if bz else 1) if bx else (3 if bz else 0)
        assert want == int(tc[b].item()), b


def test_pure_error_empty_batch(dev):
    s = torch.empty(0, 40, dtype=torch.uint8, device=dev)
    fx, fz = pkg.pure_error(s, 5)
    assert fx.shape == (0, 41) and fz.shape == (0, 41)
