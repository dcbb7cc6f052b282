"""CPU float64 oracle of the learned warm start's network and loss.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

The network maps the features of one directed block edge to an initial
message for it (the paper starts from uniform messages, Remark 2, and points
to learned techniques as a way to improve BP, Sec. V).  It is a multilayer
perceptron F -> H -> H -> O with the GELU activation
gelu(x) = x Phi(x) = x (1 + erf(x / sqrt 2)) / 2.  Its O outputs o are turned
into a non-negative unit vector over the 2^w configurations of the message
(w sites): m_i = exp(o_i - max_j o_j) for i < 2^w and 0 otherwise,
u = m / ||m||.  The loss against a converged message t (unit norm) is the
per-message term of Delta (Remark 4), L = 1 - <u, t>^2, averaged over the
batch.

Parameters are one flat vector laid out as W1 (F x H, row-major), b1 (H),
W2 (H x H), b2 (H), W3 (H x O), b3 (O).

Parity status: pinned by central finite differences of the loss
(tests/test_oracle_mlp.py) and by the closed-form values of gelu at 0 and
the loss at u = t.
"""

from __future__ import annotations

import math

import numpy as np
from scipy.special import erf

F_IN, HIDDEN, OUT = 256, 256, 16


def sizes(F=F_IN, H=HIDDEN, O=OUT):
    return [(F, H), (H,), (H, H), (H,), (H, O), (O,)]


def n_params(F=F_IN, H=HIDDEN, O=OUT):
    return sum(int(np.prod(s)) for s in sizes(F, H, O))


def unpack(theta, F=F_IN, H=HIDDEN, O=OUT):
    out, o = [], 0
    for s in sizes(F, H, O):
        n = int(np.prod(s))
        out.append(np.asarray(theta[o:o + n], dtype=np.float64).reshape(s))
        o += n
    return out


def gelu(x):
    return 0.5 * x * (1.0 + erf(x / math.sqrt(2.0)))


def gelu_grad(x):
    return 0.5 * (1.0 + erf(x / math.sqrt(2.0))) + x * np.exp(-0.5 * x * x) / math.sqrt(2.0 * math.pi)


def forward(theta, X, F=F_IN, H=HIDDEN, O=OUT):
    """Logits [N, O] and the cached pre-activations."""
    W1, b1, W2, b2, W3, b3 = unpack(theta, F, H, O)
    z1 = X @ W1 + b1
    a1 = gelu(z1)
    z2 = a1 @ W2 + b2
    a2 = gelu(z2)
    o = a2 @ W3 + b3
    return o, (z1, a1, z2, a2)


def message_from_logits(o, lens):
    """Unit non-negative messages [N, O] from logits; lens = 2^w per row."""
    N, O = o.shape
    mask = np.arange(O)[None, :] < np.asarray(lens)[:, None]
    oo = np.where(mask, o, -np.inf)
    m = np.where(mask, np.exp(oo - oo.max(axis=1, keepdims=True)), 0.0)
    return m / np.linalg.norm(m, axis=1, keepdims=True), m


def loss(theta, X, T, lens, F=F_IN, H=HIDDEN, O=OUT):
    o, _ = forward(theta, X, F, H, O)
    u, _ = message_from_logits(o, lens)
    c = np.sum(u * T, axis=1)
    return float(np.mean(1.0 - c * c))


def loss_and_grad(theta, X, T, lens, F=F_IN, H=HIDDEN, O=OUT):
    """Loss and its gradient with respect to the flat parameter vector."""
    W1, b1, W2, b2, W3, b3 = unpack(theta, F, H, O)
    o, (z1, a1, z2, a2) = forward(theta, X, F, H, O)
    u, m = message_from_logits(o, lens)
    N = X.shape[0]
    c = np.sum(u * T, axis=1)
    L = float(np.mean(1.0 - c * c))
    # dL/du = -2 c t / N; through u = m / ||m|| and m = exp(o - max) (masked).
    gu = (-2.0 * c / N)[:, None] * T
    nm = np.linalg.norm(m, axis=1, keepdims=True)
    gm = (gu - np.sum(gu * u, axis=1, keepdims=True) * u) / nm
    go = gm * m
    gW3 = a2.T @ go
    gb3 = go.sum(axis=0)
    ga2 = go @ W3.T
    gz2 = ga2 * gelu_grad(z2)
    gW2 = a1.T @ gz2
    gb2 = gz2.sum(axis=0)
    ga1 = gz2 @ W2.T
    gz1 = ga1 * gelu_grad(z1)
    gW1 = X.T @ gz1
    gb1 = gz1.sum(axis=0)
    g = np.concatenate([x.reshape(-1) for x in (gW1, gb1, gW2, gb2, gW3, gb3)])
    return L, g


def adam(theta, g, m, v, step, lr, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update (Kingma & Ba 2015), in place; returns theta."""
    m[:] = b1 * m + (1.0 - b1) * g
    v[:] = b2 * v + (1.0 - b2) * g * g
    mh = m / (1.0 - b1 ** step)
    vh = v / (1.0 - b2 ** step)
    theta -= lr * mh / (np.sqrt(vh) + eps)
    return theta
