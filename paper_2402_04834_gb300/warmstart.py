"""Learned warm start for the fused-block decoder (argument marshalling only).

A network proposes the initial message of every directed block edge from
local features; it is trained on messages that the GPU decoder itself
produces at convergence.  Features, training steps, inference and decoding
all run in libblockbp (include/blockbp.h); PyTorch provides device memory.
Cold start (uniform messages, Remark 2) stays the default and the fallback.
"""

from __future__ import annotations

import ctypes
import math

import numpy as np
import torch

from ._lib import (WARM_F, WARM_H, WARM_INFER_WS_BYTES, WARM_MAX_ROWS, WARM_O, WARM_STATUS_OFFSET as STATUS_OFFSET,
                   DecoderParams, check, lib, workspace_bytes)
from .decoder import Workspace, _ptr, _stream, decode


def message_count(prm: DecoderParams) -> int:
    M = ctypes.c_int32(0)
    cp = prm.c()
    check(lib().bbp_message_count(ctypes.byref(cp), ctypes.byref(M)))
    return int(M.value)


def features(syndromes: torch.Tensor, prm: DecoderParams, stream=None):
    """Features [B*4*M, 256] (float32) and message lengths [B*4*M] (int32)."""
    B = syndromes.shape[0]
    M = message_count(prm)
    N = B * 4 * M
    feats = torch.empty(N, WARM_F, dtype=torch.float32, device=syndromes.device)
    lens = torch.empty(N, dtype=torch.int32, device=syndromes.device)
    cp = prm.c()
    check(lib().bbp_message_features(_ptr(syndromes.contiguous()), B, ctypes.byref(cp), _ptr(feats), _ptr(lens),
                                     _stream(stream)))
    return feats, lens


_classes: dict = {}


def message_classes(prm: DecoderParams, device=None):
    """Distinct feature rows of a syndrome (bbp_message_classes): (uniq_of
    [4*M], row_key [U]) int32, on ``device`` if given; cached per geometry.
    Cosets that agree on the logical strings a message's window sees share
    one row (d = 11, k = 4: 154 of 480 rows)."""
    key = (prm.d, prm.k, str(device))
    if key not in _classes:
        M = message_count(prm)
        uniq = np.empty(4 * M, dtype=np.int32)
        rk = np.empty(4 * M, dtype=np.int32)
        U = ctypes.c_int32(0)
        cp = prm.c()
        check(lib().bbp_message_classes(ctypes.byref(cp), uniq.ctypes.data, rk.ctypes.data, ctypes.byref(U)))
        uq, rk = torch.from_numpy(uniq), torch.from_numpy(rk[:U.value].copy())
        _classes[key] = (uq.to(device), rk.to(device)) if device is not None else (uq, rk)
    return _classes[key]


def features_rows(syndromes: torch.Tensor, prm: DecoderParams, stream=None):
    """Features [B*U, 256] and lengths [B*U] of the distinct rows only
    (``message_classes``); row b*U + u is (coset, message) = row_key[u]."""
    B = syndromes.shape[0]
    _, rk = message_classes(prm, syndromes.device)
    U = rk.numel()
    feats = torch.empty(B * U, WARM_F, dtype=torch.float32, device=syndromes.device)
    lens = torch.empty(B * U, dtype=torch.int32, device=syndromes.device)
    cp = prm.c()
    check(lib().bbp_message_features_rows(_ptr(syndromes.contiguous()), B, ctypes.byref(cp), _ptr(rk), U,
                                          _ptr(feats), _ptr(lens), _stream(stream)))
    return feats, lens


def feature_bits_rows(syndromes: torch.Tensor, prm: DecoderParams, stream=None):
    """The rows of ``features_rows`` as bits [B*U, 8] int32 (bit q % 32 of word
    q // 32 set where feature q is not zero; feature 253 stands for 10 p)
    and the lengths [B*U]."""
    B = syndromes.shape[0]
    _, rk = message_classes(prm, syndromes.device)
    U = rk.numel()
    bits = torch.empty(B * U, WARM_F // 32, dtype=torch.int32, device=syndromes.device)
    lens = torch.empty(B * U, dtype=torch.int32, device=syndromes.device)
    cp = prm.c()
    check(lib().bbp_message_feature_bits_rows(_ptr(syndromes.contiguous()), B, ctypes.byref(cp), _ptr(rk), U,
                                              _ptr(bits), _ptr(lens), _stream(stream)))
    return bits, lens


def expand_rows(rows: torch.Tensor, B: int, prm: DecoderParams, out=None, stream=None):
    """Messages [B*4*M, 16] (rows ordered syndrome, coset, message) from the
    distinct rows [B*U, 16]."""
    uq, rk = message_classes(prm, rows.device)
    M = message_count(prm)
    out = out if out is not None else torch.empty(B * 4 * M, WARM_O, dtype=torch.float32, device=rows.device)
    check(lib().bbp_expand_rows(_ptr(rows), B, rk.numel(), _ptr(uq), M, _ptr(out), _stream(stream)))
    return out


def _ws_bytes(N: int) -> int:
    out = ctypes.c_size_t(0)
    check(lib().bbp_warm_workspace_bytes(N, ctypes.byref(out)))
    return int(out.value)


class WarmStart:
    """Parameters and Adam state of the network, on one device."""

    def __init__(self, device="cuda", seed: int = 0):
        n = int(lib().bbp_warm_param_count())
        g = torch.Generator(device="cpu").manual_seed(seed)
        parts = []
        for fan_in, fan_out in ((WARM_F, WARM_H), (WARM_H, WARM_H), (WARM_H, WARM_O)):
            w = torch.randn(fan_in, fan_out, generator=g) * math.sqrt(2.0 / (fan_in + fan_out))
            parts += [w.reshape(-1), torch.zeros(fan_out)]
        theta = torch.cat(parts)
        assert theta.numel() == n
        self.device = torch.device(device)
        self.theta = theta.to(self.device, torch.float32).contiguous()
        self.m = torch.zeros_like(self.theta)
        self.v = torch.zeros_like(self.theta)
        self.grad = torch.zeros_like(self.theta)
        self.loss = torch.zeros(1, dtype=torch.float32, device=self.device)
        self.step = 0
        self.ws = Workspace()
        self.infer_ws = Workspace()

    def train_step(self, feats, targets, lens, lr=1e-3, stream=None) -> float:
        """One Adam step on a minibatch; returns the mean loss before the step."""
        N = feats.shape[0]
        ws = self.ws.get(_ws_bytes(N), self.device)
        self.step += 1
        check(lib().bbp_warm_train_step(_ptr(self.theta), _ptr(self.m), _ptr(self.v), self.step, lr, _ptr(feats),
                                        _ptr(targets), _ptr(lens), N, _ptr(self.grad), _ptr(self.loss), _ptr(ws),
                                        ws.numel(), _stream(stream)))
        return float(self.loss.item()) / N

    def gradient(self, feats, targets, lens, stream=None):
        """Loss and gradient without an update (used by the gradient check)."""
        N = feats.shape[0]
        ws = self.ws.get(_ws_bytes(N), self.device)
        check(lib().bbp_warm_train_step(_ptr(self.theta), None, None, 0, 0.0, _ptr(feats), _ptr(targets),
                                        _ptr(lens), N, _ptr(self.grad), _ptr(self.loss), _ptr(ws), ws.numel(),
                                        _stream(stream)))
        torch.cuda.synchronize(self.device)
        return float(self.loss.item()) / N, self.grad.clone()

    def infer(self, feats, lens, out=None, stream=None, alpha=1.0):
        """Initial messages [N, 16] for the given feature rows (chunked),
        blended with the uniform start by ``alpha``."""
        N = feats.shape[0]
        out = out if out is not None else torch.empty(N, WARM_O, dtype=torch.float32, device=feats.device)
        step = max(1, min(N, WARM_MAX_ROWS))
        ws = self.infer_ws.get(WARM_INFER_WS_BYTES, self.device)
        for a in range(0, N, step):
            b = min(N, a + step)
            check(lib().bbp_warm_infer(_ptr(self.theta), _ptr(feats[a:b]), _ptr(lens[a:b]), b - a, alpha,
                                       _ptr(out[a:b]), _ptr(ws), ws.numel(), _stream(stream)))
        return out

    def infer_bits(self, bits, lens, p, out=None, stream=None, alpha=1.0):
        """``infer`` from feature bits [N, 8] (``feature_bits_rows``) and the
        noise rate of feature 253: the same messages bit for bit."""
        N = bits.shape[0]
        out = out if out is not None else torch.empty(N, WARM_O, dtype=torch.float32, device=bits.device)
        step = max(1, min(N, WARM_MAX_ROWS))
        ws = self.infer_ws.get(WARM_INFER_WS_BYTES, self.device)
        for a in range(0, N, step):
            b = min(N, a + step)
            check(lib().bbp_warm_infer_bits(_ptr(self.theta), _ptr(bits[a:b]), _ptr(lens[a:b]), b - a, p, alpha,
                                            _ptr(out[a:b]), _ptr(ws), ws.numel(), _stream(stream)))
        return out

    def infer_syndromes(self, syndromes, prm: DecoderParams, out=None, stream=None, alpha=1.0):
        """Initial messages [B*4*M, 16] for every message of the syndromes
        [B, m], the features computed inside the tensor-core kernel."""
        B = syndromes.shape[0]
        N = B * 4 * message_count(prm)
        out = out if out is not None else torch.empty(N, WARM_O, dtype=torch.float32, device=syndromes.device)
        ws = self.infer_ws.get(WARM_INFER_WS_BYTES, self.device)
        cp = prm.c()
        check(lib().bbp_warm_infer_syndromes(_ptr(self.theta), _ptr(syndromes.contiguous()), B, ctypes.byref(cp),
                                             alpha, _ptr(out), _ptr(ws), ws.numel(), _stream(stream)))
        return out

    def status(self) -> int:
        """Status word of the last inference (0 = every device wait completed)."""
        torch.cuda.synchronize(self.device)
        buf = self.infer_ws.buf
        if buf is None or buf.numel() < STATUS_OFFSET + 4:
            return 0
        return int(buf[STATUS_OFFSET:STATUS_OFFSET + 4].view(torch.int32).item())

    def train(self, feats, targets, lens, epochs=4, batch=8192, lr=1e-3, seed=0, log=None):
        N = feats.shape[0]
        g = torch.Generator(device="cpu").manual_seed(seed)
        hist = []
        for ep in range(epochs):
            perm = torch.randperm(N, generator=g).to(feats.device)
            tot, cnt = 0.0, 0
            for a in range(0, N - batch + 1, batch):
                idx = perm[a:a + batch]
                lo = self.train_step(feats[idx].contiguous(), targets[idx].contiguous(), lens[idx].contiguous(), lr)
                tot += lo
                cnt += 1
            hist.append(tot / max(cnt, 1))
            if log:
                log(f"epoch {ep}: mean loss {hist[-1]:.4e}")
        return hist


def decode_ex(syndromes, prm: DecoderParams, init_msgs=None, final_msgs=None, workspace=None, stream=None,
              out=None):
    """Fused-path decode with optional initial messages and message export."""
    B = syndromes.shape[0]
    dev = syndromes.device
    if out is None:
        out = {
            "logp": torch.empty(B, 4, dtype=torch.float64, device=dev),
            "delta": torch.empty(B, 4, dtype=torch.float64, device=dev),
            "iters": torch.empty(B, 4, dtype=torch.int32, device=dev),
            "flags": torch.empty(B, 4, dtype=torch.int32, device=dev),
            "decision": torch.empty(B, dtype=torch.int8, device=dev),
        }
    cp = prm.c()
    ws = (workspace or Workspace()).get(max(256, workspace_bytes(prm, B)), dev)
    check(lib().bbp_decode_batch_ex(_ptr(syndromes), B, ctypes.byref(cp),
                                    _ptr(init_msgs) if init_msgs is not None else None,
                                    _ptr(final_msgs) if final_msgs is not None else None,
                                    _ptr(out["logp"]), _ptr(out["delta"]), _ptr(out["iters"]), _ptr(out["flags"]),
                                    _ptr(out["decision"]), _ptr(ws), ws.numel(), _stream(stream)))
    return out


DEFAULT_ALPHA = 0.1     # blend weight of the proposal (measured: larger weights raise P_L)


def propose(syndromes, prm: DecoderParams, net: WarmStart, stream=None, alpha=DEFAULT_ALPHA):
    """Initial messages [B*4*M, 16] from the network: features of the
    distinct rows, the network on the tensor cores over those rows, and the
    expansion to every (coset, message); equal bit for bit to the network
    over every row."""
    feats, lens = features_rows(syndromes, prm, stream)
    rows = net.infer(feats, lens, stream=stream, alpha=alpha)
    return expand_rows(rows, syndromes.shape[0], prm, stream=stream)


def decode_warm_workspace_bytes(prm: DecoderParams, B: int, include_io: bool = False) -> int:
    out = ctypes.c_size_t(0)
    cp = prm.c()
    check(lib().bbp_decode_warm_workspace_bytes(ctypes.byref(cp), B, int(include_io), ctypes.byref(out)))
    return int(out.value)


def decode_warm(syndromes, prm: DecoderParams, net: WarmStart, stream=None, out=None, alpha=DEFAULT_ALPHA,
                workspace=None):
    """Learned warm start in one library call (bbp_decode_warm): features of
    the distinct rows, the network on the tensor cores, the expansion to
    every (coset, message), then the fused decode from the proposals; equal
    bit for bit to ``propose`` followed by ``decode_ex``."""
    B = syndromes.shape[0]
    dev = syndromes.device
    if out is None:
        out = {
            "logp": torch.empty(B, 4, dtype=torch.float64, device=dev),
            "delta": torch.empty(B, 4, dtype=torch.float64, device=dev),
            "iters": torch.empty(B, 4, dtype=torch.int32, device=dev),
            "flags": torch.empty(B, 4, dtype=torch.int32, device=dev),
            "decision": torch.empty(B, dtype=torch.int8, device=dev),
        }
    ws = (workspace or net.infer_ws).get(decode_warm_workspace_bytes(prm, B), dev)
    cp = prm.c()
    check(lib().bbp_decode_warm(_ptr(net.theta), _ptr(syndromes.contiguous()), B, ctypes.byref(cp), alpha,
                                _ptr(out["logp"]), _ptr(out["delta"]), _ptr(out["iters"]), _ptr(out["flags"]),
                                _ptr(out["decision"]), _ptr(ws), ws.numel(), _stream(stream)))
    return out


def decode_warm_host(syndromes, prm: DecoderParams, net: WarmStart, out=None, alpha=DEFAULT_ALPHA, stream=None,
                     workspace=None):
    """The learned decoder from host memory in one library call
    (bbp_decode_warm_host): syndromes [B, m] uint8 (numpy or CPU tensor,
    pinned for asynchronous copies) in, decisions [B] and log P [B, 4] back
    in host memory; the call synchronises the stream."""
    syn = torch.as_tensor(syndromes).contiguous()
    B = syn.shape[0]
    if out is None:
        out = {"decision": torch.empty(B, dtype=torch.int8, pin_memory=True),
               "logp": torch.empty(B, 4, dtype=torch.float64, pin_memory=True)}
    ws = (workspace or net.infer_ws).get(decode_warm_workspace_bytes(prm, B, include_io=True), net.device)
    cp = prm.c()
    st = stream or torch.cuda.current_stream(net.device)
    check(lib().bbp_decode_warm_host(_ptr(net.theta), syn.data_ptr(), B, ctypes.byref(cp), alpha,
                                     out["logp"].data_ptr() if out.get("logp") is not None else None,
                                     out["delta"].data_ptr() if out.get("delta") is not None else None,
                                     out["iters"].data_ptr() if out.get("iters") is not None else None,
                                     out["flags"].data_ptr() if out.get("flags") is not None else None,
                                     out["decision"].data_ptr(), _ptr(ws), ws.numel(), _stream(st)))
    return out


def collect(syndromes, prm: DecoderParams, max_delta=1e-3):
    """Training rows from one batch: features and the decoder's converged
    messages, keeping the (syndrome, coset) pairs whose final Delta is below
    ``max_delta`` (converged)."""
    B = syndromes.shape[0]
    M = message_count(prm)
    final = torch.empty(B * 4 * M, WARM_O, dtype=torch.float32, device=syndromes.device)
    out = decode_ex(syndromes, prm, final_msgs=final)
    feats, lens = features(syndromes, prm)
    ok = (out["delta"] < max_delta).reshape(-1).repeat_interleave(M)
    return feats[ok], final[ok], lens[ok]


def wilson(k: int, n: int, z: float = 1.959963984540054):
    """Wilson score interval of a binomial proportion k / n (95% by default)."""
    if n == 0:
        return (0.0, 1.0)
    ph = k / n
    den = 1 + z * z / n
    c = (ph + z * z / (2 * n)) / den
    h = z * math.sqrt(ph * (1 - ph) / n + z * z / (4 * n * n)) / den
    return (max(0.0, c - h), min(1.0, c + h))


def build_training_set(device="cuda", d_list=(11, 15), shots=(1500, 800), p_grid=(0.05, 0.075, 0.10, 0.125, 0.15),
                       k=4, seed_base=4000, max_rows=1_000_000):
    """Converged messages of seeded decodes (the decoder labels its own data)."""
    feats, targets, lens = [], [], []
    for d, n in zip(d_list, shots):
        per_p = max(1, n // len(p_grid))
        for ip, p in enumerate(p_grid):
            prm = DecoderParams(d=d, k=k, p=p, max_iter=40, delta0=1e-6, precision="fp32", algorithm="fused")
            from .decoder import sample
            _, _, s, _ = sample(seed_base + 100 * d + ip, 0, per_p, d, p, device=device, with_errors=False)
            f, t, ln = collect(s, prm)
            feats.append(f)
            targets.append(t)
            lens.append(ln)
    F = torch.cat(feats)[:max_rows].contiguous()
    T = torch.cat(targets)[:max_rows].contiguous()
    L = torch.cat(lens)[:max_rows].contiguous()
    return F, T, L


def evaluate(net: WarmStart, d=13, p=0.10, shots=10000, k=4, seed=5000, device="cuda", max_iter=20, delta0=1e-4,
             alpha=DEFAULT_ALPHA):
    """Cold versus warm start on fresh syndromes: iterations, P_L, throughput."""
    from .decoder import sample
    _, _, s, tc = sample(seed, 0, shots, d, p, device=device, with_errors=False)
    prm = DecoderParams(d=d, k=k, p=p, max_iter=max_iter, delta0=delta0, precision="fp32", algorithm="fused")
    res = {"alpha": alpha}
    for name in ("cold", "warm"):
        run = (lambda: decode(s, prm)) if name == "cold" else (lambda: decode_warm(s, prm, net, alpha=alpha))
        out = run()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        out = run()
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        fails = int((out["decision"].to(torch.int64) != tc.to(torch.int64)).sum().item())
        lo, hi = wilson(fails, shots)
        res[name] = {"mean_iters": float(out["iters"].double().mean().item()), "failures": fails, "shots": shots,
                     "P_L": fails / shots, "P_L_wilson95": [lo, hi], "ms": ms, "syndromes_per_s": shots / ms * 1e3}
        res[name + "_decision"] = out["decision"]
    agree = float((res["cold_decision"] == res["warm_decision"]).double().mean().item())
    for key in ("cold_decision", "warm_decision"):
        res.pop(key)
    res["decision_agreement"] = agree
    res["iterations_saved_fraction"] = 1.0 - res["warm"]["mean_iters"] / res["cold"]["mean_iters"]
    return res


def time_inference(syndromes_n=2500, d=11, p=0.10, k=4, seed=5000, reps=3):
    """Features, tensor-core inference from them, and inference with the
    features computed in its kernel, for an untrained network over the
    messages of ``syndromes_n`` seeded syndromes (4 M rows per syndrome);
    then the same for the distinct rows only, from FP32 rows and from
    feature bits; returns the rows and the best times in ms."""
    from .decoder import sample
    dev = torch.device("cuda")
    _, _, s, _ = sample(seed, 0, syndromes_n, d, p, device=dev, with_errors=False)
    prm = DecoderParams(d=d, k=k, p=p, precision="fp32", algorithm="fused")
    net = WarmStart(device=dev, seed=0)
    feats, lens = features(s, prm)
    out = net.infer(feats, lens)
    # The distinct rows only (what the decoder runs), as FP32 rows and as bits.
    rfeats, rlens = features_rows(s, prm)
    bits, blens = feature_bits_rows(s, prm)
    rout = net.infer(rfeats, rlens)
    res = {"rows": int(feats.shape[0]), "distinct_rows": int(rfeats.shape[0])}
    for name, fn in (("features_ms", lambda: features(s, prm)), ("infer_ms", lambda: net.infer(feats, lens, out=out)),
                     ("infer_from_syndromes_ms", lambda: net.infer_syndromes(s, prm, out=out)),
                     ("features_rows_ms", lambda: features_rows(s, prm)),
                     ("infer_rows_ms", lambda: net.infer(rfeats, rlens, out=rout)),
                     ("feature_bits_rows_ms", lambda: feature_bits_rows(s, prm)),
                     ("infer_bits_ms", lambda: net.infer_bits(bits, blens, p, out=rout))):
        best = float("inf")
        for _ in range(reps):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            fn()
            b.record()
            torch.cuda.synchronize()
            best = min(best, a.elapsed_time(b))
        res[name] = best
    res["status"] = net.status()
    return res


def main():
    import json
    import sys
    import time
    if len(sys.argv) > 2 and sys.argv[1] == "--time-inference":
        print(json.dumps(time_inference(int(sys.argv[2]))))
        return
    dev = torch.device("cuda")
    t0 = time.time()
    F, T, L = build_training_set(device=dev)
    t1 = time.time()
    net = WarmStart(device=dev, seed=0)
    hist = net.train(F, T, L, epochs=12, batch=8192, lr=3e-3)
    hist += net.train(F, T, L, epochs=8, batch=8192, lr=5e-4, seed=1)
    torch.cuda.synchronize()
    t2 = time.time()
    evs = [evaluate(net, device=dev, alpha=a) for a in (0.1, 0.25, 0.5, 1.0)]
    print(json.dumps({"training_rows": int(F.shape[0]), "data_s": t1 - t0, "train_s": t2 - t1,
                      "loss_per_epoch": hist, "evaluation_d13_p010": evs}))


if __name__ == "__main__":
    main()
