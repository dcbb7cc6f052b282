"""The C-ABI library: loads, exports every declared symbol, validates arguments (no GPU)."""

import ctypes
import os
import re

import pytest

import paper_2402_04834_gb300 as pkg
from paper_2402_04834_gb300 import _lib
from paper_2402_04834_gb300.build import build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    build()
    return pkg.lib()


def declared_functions():
    with open(os.path.join(ROOT, "include", "blockbp.h")) as f:
        text = f.read()
    return sorted(set(re.findall(r"^(?:int|const char\*)\s+(bbp_\w+)\s*\(", text, flags=re.M)))


def test_every_declared_symbol_is_exported(L):
    names = declared_functions()
    assert len(names) >= 6
    for n in names:
        assert hasattr(L, n), n
    assert set(names) == set(_lib.SYMBOLS)


def test_version_and_strerror(L):
    assert b"sm_103a" in L.bbp_version()
    for code in (0, -1, -2, -3, -4):
        assert len(L.bbp_strerror(code)) > 0


def test_workspace_sizes_scale_with_batch(L):
    p = pkg.DecoderParams(d=11, k=4, D=8)
    a = pkg.workspace_bytes(p, 100)
    b = pkg.workspace_bytes(p, 200)
    assert b >= 2 * a - 256 and a > 0
    p32 = pkg.DecoderParams(d=11, k=4, D=8, precision="fp32")
    assert pkg.workspace_bytes(p32, 100) < a
    assert pkg.workspace_bytes(p, 100, include_io=True) > a


@pytest.mark.parametrize("field,val", [("d", 1), ("k", 0), ("D", 0), ("p", 0.0), ("p", 0.8),
                                       ("eta", 1.0), ("precision", 7), ("max_iter", -1),
                                       ("launch_warps", 5), ("launch_cosets", 3), ("launch_messages", 4)])
def test_invalid_parameters_rejected(L, field, val):
    c = pkg.DecoderParams(d=5, k=3, D=4).c()
    setattr(c, field, val)
    out = ctypes.c_size_t(0)
    assert L.bbp_workspace_bytes(ctypes.byref(c), 10, 0, ctypes.byref(out)) == -1


def test_unsupported_sizes_reported(L):
    c = pkg.DecoderParams(d=11, k=9, D=8).c()
    out = ctypes.c_size_t(0)
    assert L.bbp_workspace_bytes(ctypes.byref(c), 10, 0, ctypes.byref(out)) == -4


def test_fused_launch_shapes_checked_on_the_host(L):
    # Compiled shapes are accepted; uncompiled ones, and shapes whose shared
    # memory cannot fit one CTA, are reported before any CUDA call.
    out = ctypes.c_size_t(0)
    for prec, shapes in pkg.FUSED_SHAPES.items():
        for w, g in shapes:
            c = pkg.DecoderParams(d=7, k=4, precision=prec, algorithm="fused", warps=w, cosets=g).c()
            assert L.bbp_workspace_bytes(ctypes.byref(c), 10, 0, ctypes.byref(out)) == 0, (prec, w, g)
    c = pkg.DecoderParams(d=7, k=4, precision="fp64", algorithm="fused", warps=16, cosets=4).c()
    assert L.bbp_workspace_bytes(ctypes.byref(c), 10, 0, ctypes.byref(out)) == -4
    c = pkg.DecoderParams(d=31, k=4, precision="fp64", algorithm="fused", warps=4, cosets=4).c()
    assert L.bbp_workspace_bytes(ctypes.byref(c), 10, 0, ctypes.byref(out)) == -4
    c = pkg.DecoderParams(d=31, k=4, precision="fp64", algorithm="fused").c()
    assert L.bbp_workspace_bytes(ctypes.byref(c), 10, 0, ctypes.byref(out)) == 0
    for prec, shapes in pkg.FUSED_SHAPES_K6.items():
        for w, g in shapes:
            c = pkg.DecoderParams(d=31, k=6, precision=prec, algorithm="fused", warps=w, cosets=g).c()
            assert L.bbp_workspace_bytes(ctypes.byref(c), 10, 0, ctypes.byref(out)) == 0, (prec, w, g)
    c = pkg.DecoderParams(d=31, k=6, precision="fp64", algorithm="fused", warps=4, cosets=1).c()
    assert L.bbp_workspace_bytes(ctypes.byref(c), 10, 0, ctypes.byref(out)) == -4
    for prec, shapes in pkg.FUSED_SHAPES_WS.items():
        for w, g in shapes:
            c = pkg.DecoderParams(d=13, k=4, precision=prec, algorithm="fused", warps=w, cosets=g, messages=2).c()
            assert L.bbp_workspace_bytes(ctypes.byref(c), 10, 0, ctypes.byref(out)) == 0 and out.value > 0
    c = pkg.DecoderParams(d=13, k=4, precision="fp32", algorithm="fused", warps=4, cosets=4, messages=2).c()
    assert L.bbp_workspace_bytes(ctypes.byref(c), 10, 0, ctypes.byref(out)) == -4   # not compiled
    c = pkg.DecoderParams(d=13, k=6, precision="fp32", algorithm="fused", messages=1).c()
    assert L.bbp_workspace_bytes(ctypes.byref(c), 10, 0, ctypes.byref(out)) == -4   # k = 6: workspace only


def test_fused_k6_workspace_holds_one_message_slot_per_resident_cta(L):
    # k <= 4 keeps the messages in shared memory; k = 5, 6 keep them in
    # min(4B, 512) slots of 64 M scalars (d = 31: M = 440 directed edges).
    assert pkg.workspace_bytes(pkg.DecoderParams(d=31, k=4, precision="fp32", algorithm="fused", messages=1),
                               1000) == 0
    # k = 4 at d = 31: the default shape (8 warps, 2 cosets; with 4 cosets the
    # per-message tables alone leave room for one CTA per SM) keeps its
    # messages in min(2B, 512) slots of 2 x M x 16 scalars (M = 4 * 16 * 15).
    assert pkg.workspace_bytes(pkg.DecoderParams(d=31, k=4, precision="fp32", algorithm="fused"), 1000) == \
        512 * 2 * 960 * 16 * 4
    for B, prec, size in ((10, "fp32", 4), (10, "fp64", 8), (1000, "fp32", 4)):
        slots = min(4 * B, 512)
        want = -(-slots * 440 * 64 * size // 256) * 256
        assert pkg.workspace_bytes(pkg.DecoderParams(d=31, k=6, precision=prec, algorithm="fused"), B) == want


def test_decode_null_pointers_rejected_before_any_cuda_call(L):
    c = pkg.DecoderParams(d=5, k=3, D=4).c()
    rc = L.bbp_decode_batch(None, 4, ctypes.byref(c), None, None, None, None, None, None, 0, None)
    assert rc == -1
    rc = L.bbp_decode_batch_host(None, 4, ctypes.byref(c), None, None, None, None, None, None, 0, None)
    assert rc == -1
    assert L.bbp_sample(1, 0, 4, 1, 0.1, None, None, None, None, None) == -1


def test_pure_error_arguments_checked_on_the_host(L):
    big = ctypes.c_void_p(256)                      # never dereferenced: every call below returns first
    assert L.bbp_pure_error(1, big, 4, big, big, None) == -1
    assert L.bbp_pure_error(65, big, 4, big, big, None) == -1
    assert L.bbp_pure_error(5, None, 4, big, big, None) == -1
    assert L.bbp_pure_error(5, big, 4, None, big, None) == -1
    assert L.bbp_pure_error(5, big, -1, big, big, None) == -1
    assert L.bbp_pure_error(5, None, 0, None, None, None) == 0


def test_empty_batch_is_a_no_op(L):
    c = pkg.DecoderParams(d=5, k=3, D=4).c()
    assert L.bbp_decode_batch(None, 0, ctypes.byref(c), None, None, None, None, None, None, 0, None) == 0


def test_warm_start_arguments_checked_on_the_host(L):
    # Argument errors of the warm-start entry points are reported before any
    # CUDA call; an empty batch is a no-op.
    vp = ctypes.c_void_p
    c = pkg.DecoderParams(d=11, k=4, precision="fp32", algorithm="fused").c()
    big = vp(256)                                   # never dereferenced: every call below returns first
    assert L.bbp_warm_infer_syndromes(None, big, 4, ctypes.byref(c), 0.1, big, big, 1 << 20, None) == -1
    assert L.bbp_warm_infer_syndromes(big, big, 4, ctypes.byref(c), 1.5, big, big, 1 << 20, None) == -1
    assert L.bbp_warm_infer_syndromes(big, big, 4, ctypes.byref(c), 0.1, big, big, 1024, None) == -3
    assert L.bbp_warm_infer_syndromes(big, big, 0, ctypes.byref(c), 0.1, big, None, 0, None) == 0
    c5 = pkg.DecoderParams(d=11, k=5, precision="fp32", algorithm="fused").c()
    assert L.bbp_warm_infer_syndromes(big, big, 4, ctypes.byref(c5), 0.1, big, big, 1 << 20, None) == -1
    assert L.bbp_warm_infer(big, big, big, 10, 0.1, big, big, _lib.WARM_INFER_WS_BYTES - 1, None) == -3
    assert L.bbp_warm_infer(big, big, big, _lib.WARM_MAX_ROWS + 1, 0.1, big, big, 1 << 20, None) == -1
    assert L.bbp_warm_infer(big, big, big, 0, 0.1, big, None, 0, None) == 0
    # the feature-bits forms
    assert L.bbp_warm_infer_bits(big, None, big, 10, 0.1, 0.1, big, big, 1 << 20, None) == -1
    assert L.bbp_warm_infer_bits(big, big, big, 10, 0.0, 0.1, big, big, 1 << 20, None) == -1     # p outside (0, 0.75)
    assert L.bbp_warm_infer_bits(big, big, big, 10, 0.1, 1.5, big, big, 1 << 20, None) == -1     # alpha
    assert L.bbp_warm_infer_bits(big, big, big, _lib.WARM_MAX_ROWS + 1, 0.1, 0.1, big, big, 1 << 20, None) == -1
    assert L.bbp_warm_infer_bits(big, big, big, 10, 0.1, 0.1, big, big, _lib.WARM_INFER_WS_BYTES - 1, None) == -3
    assert L.bbp_warm_infer_bits(big, big, big, 0, 0.1, 0.1, big, None, 0, None) == 0
    assert L.bbp_message_feature_bits_rows(big, 4, ctypes.byref(c), big, 10, None, big, None) == -1
    assert L.bbp_message_feature_bits_rows(big, 4, ctypes.byref(c), big, 4 * 120 + 1, big, big, None) == -1
    assert L.bbp_message_feature_bits_rows(big, 0, ctypes.byref(c), big, 10, big, big, None) == 0


def _window_logicals(d, k, I, J, dr):
    """Independent restatement: which logical strings the 7 x 7 window of
    message (I, J, dr) in its rotated frame (chain rows -1 .. 5, the last 7
    columns) sees: bit 0 for a horizontal-edge qubit (even, even) of grid
    row 0 (X-bar), bit 1 for one of grid column 0 (Z-bar)."""
    W = 2 * d - 1
    rg = [(a, min(a + k, W)) for a in range(0, W, k)]
    r0, r1 = rg[I]
    c0, c1 = rg[J]
    ncols = (c1 - c0) if dr in (0, 1) else (r1 - r0)
    seen = 0
    for t in range(ncols - 7, ncols):
        for sp in range(-1, 6):
            i, j = {0: (r0 + sp, c0 + t), 1: (r0 + sp, c1 - 1 - t), 2: (r0 + t, c0 + sp),
                    3: (r1 - 1 - t, c0 + sp)}[dr]
            if 0 <= i < W and 0 <= j < W and i % 2 == 0 and j % 2 == 0:
                seen |= (1 if i == 0 else 0) | (2 if j == 0 else 0)
    return seen


@pytest.mark.parametrize("d,k", [(11, 4), (13, 4), (3, 4), (7, 3), (5, 2)])
def test_message_classes_on_the_host(L, d, k):
    # Cosets (bx, bz) that agree on the logical strings a window sees share
    # a row: one row when it sees neither, two for one string, four for
    # both; d = 11, k = 4: 90 / 14 / 14 / 2 messages, 154 rows.
    c = pkg.DecoderParams(d=d, k=k, precision="fp32", algorithm="fused").c()
    M = ctypes.c_int32(0)
    assert L.bbp_message_count(ctypes.byref(c), ctypes.byref(M)) == 0
    M = M.value
    uq = (ctypes.c_int32 * (4 * M))()
    rk = (ctypes.c_int32 * (4 * M))()
    U = ctypes.c_int32(0)
    assert L.bbp_message_classes(ctypes.byref(c), uq, rk, ctypes.byref(U)) == 0
    nb = -(-(2 * d - 1) // k)
    msgs = [(I, J, dr) for I in range(nb) for J in range(nb) for dr, (di, dj) in
            enumerate(((0, 1), (0, -1), (1, 0), (-1, 0))) if 0 <= I + di < nb and 0 <= J + dj < nb]
    assert len(msgs) == M
    seen = [_window_logicals(d, k, *m) for m in msgs]
    assert U.value == sum({0: 1, 1: 2, 2: 2, 3: 4}[x] for x in seen)
    if (d, k) == (11, 4):
        assert [seen.count(x) for x in range(4)] == [90, 14, 14, 2] and U.value == 154
    for i, x in enumerate(seen):
        assert len({uq[c2 * M + i] for c2 in range(4)}) == {0: 1, 1: 2, 2: 2, 3: 4}[x]
        for c2 in range(4):
            bx = c2 in (1, 2) and bool(x & 1)
            bz = c2 in (2, 3) and bool(x & 2)
            rep = (2 if bz else 1) if bx else (3 if bz else 0)
            key = rk[uq[c2 * M + i]]
            assert key % M == i and key // M == rep
    bad = pkg.DecoderParams(d=d, k=5, precision="fp32", algorithm="fused").c()
    assert L.bbp_message_classes(ctypes.byref(bad), uq, rk, ctypes.byref(U)) == -1


@pytest.mark.parametrize("alg,prec,k,messages,d_max", [
    ("fused", "fp32", 4, 1, 46), ("fused", "fp64", 4, 1, 34), ("fused", "fp32", 4, 0, 58), ("fused", "fp64", 4, 0, 54),
    ("fused", "fp32", 2, 0, 36), ("fused", "fp32", 1, 0, 19), ("fused", "fp32", 2, 1, 25), ("fused", "fp32", 1, 1, 13),
    ("fused", "fp32", 6, 0, 64), ("fused", "fp64", 6, 0, 64), ("mps", "fp64", 4, 0, 64), ("mps", "fp32", 4, 0, 64)])
def test_largest_supported_distance(L, alg, prec, k, messages, d_max):
    # Fused k <= 4 with its messages in shared memory is bounded by them (the
    # messages of k < 4 are padded to 16 entries); with the messages in
    # workspace slots by the per-message tables that stay in shared memory;
    # k = 6 and the MPS form take the API's d <= 64.  Past the bound the call
    # is refused on the host.
    out = ctypes.c_size_t(0)
    c = pkg.DecoderParams(d=d_max, k=k, D=8, precision=prec, algorithm=alg, messages=messages).c()
    assert L.bbp_workspace_bytes(ctypes.byref(c), 4, 0, ctypes.byref(out)) == 0
    c = pkg.DecoderParams(d=d_max + 1, k=k, D=8, precision=prec, algorithm=alg, messages=messages).c()
    assert L.bbp_workspace_bytes(ctypes.byref(c), 4, 0, ctypes.byref(out)) == (-4 if d_max < 64 else -1)


def test_learned_decoder_entry_points_check_arguments_on_the_host(L):
    # bbp_decode_warm / _host: every argument is checked before any CUDA call.
    vp = ctypes.c_void_p
    fused = pkg.DecoderParams(d=11, k=4, p=0.1, precision="fp32", algorithm="fused")
    cp = fused.c()
    out = ctypes.c_size_t(0)
    assert L.bbp_decode_warm_workspace_bytes(ctypes.byref(cp), 100, 0, ctypes.byref(out)) == 0
    dev_bytes = out.value
    assert L.bbp_decode_warm_workspace_bytes(ctypes.byref(cp), 100, 1, ctypes.byref(out)) == 0
    assert out.value > dev_bytes
    # Room for the feature bits of the distinct rows (154 per syndrome, 32
    # bytes each), their proposals (16 floats) and the expanded initial
    # messages (480 x 16 floats per syndrome); no FP32 feature rows.
    assert dev_bytes >= 100 * (154 * (32 + 64) + 480 * 64)
    assert dev_bytes < 100 * (154 * 1024 + 480 * 64)
    for bad in (pkg.DecoderParams(d=11, k=4, algorithm="mps"),
                pkg.DecoderParams(d=11, k=6, precision="fp32", algorithm="fused"),
                pkg.DecoderParams(d=1, k=4, algorithm="fused")):
        c = bad.c()
        assert L.bbp_decode_warm_workspace_bytes(ctypes.byref(c), 100, 0, ctypes.byref(out)) == -1
    assert L.bbp_decode_warm_workspace_bytes(ctypes.byref(cp), 100, 0, None) == -1
    fake = vp(256)
    for fn in (L.bbp_decode_warm, L.bbp_decode_warm_host):
        # null parameter vector, syndromes, decision, workspace
        assert fn(None, fake, 4, ctypes.byref(cp), 0.1, fake, fake, fake, fake, fake, fake, 1 << 40, None) == -1
        assert fn(fake, None, 4, ctypes.byref(cp), 0.1, fake, fake, fake, fake, fake, fake, 1 << 40, None) == -1
        assert fn(fake, fake, 4, ctypes.byref(cp), 0.1, fake, fake, fake, fake, None, fake, 1 << 40, None) == -1
        assert fn(fake, fake, 4, ctypes.byref(cp), 0.1, fake, fake, fake, fake, fake, None, 1 << 40, None) == -1
        # alpha outside [0, 1], negative batch, misaligned or short workspace
        assert fn(fake, fake, 4, ctypes.byref(cp), 1.5, fake, fake, fake, fake, fake, fake, 1 << 40, None) == -1
        assert fn(fake, fake, -1, ctypes.byref(cp), 0.1, fake, fake, fake, fake, fake, fake, 1 << 40, None) == -1
        assert fn(fake, fake, 4, ctypes.byref(cp), 0.1, fake, fake, fake, fake, fake, vp(257), 1 << 40, None) == -1
        assert fn(fake, fake, 4, ctypes.byref(cp), 0.1, fake, fake, fake, fake, fake, fake, 1024, None) == -3
        assert fn(fake, fake, 0, ctypes.byref(cp), 0.1, None, None, None, None, None, None, 0, None) == 0


def test_register_form_only_shapes_chosen_where_every_block_has_one(L):
    # messages = 3 (every block update in register form) exists for k = 4
    # at odd d (the last block row / column one node wide); at even d the
    # 3-wide last blocks need the node-by-node path.  bbp_decode_mixed takes
    # it only on request, and refuses the request for an even d_max or
    # k != 4 before any CUDA call.
    out = ctypes.c_size_t(0)
    for d in (5, 11, 13, 21):
        c = pkg.DecoderParams(d=d, k=4, precision="fp32", algorithm="fused", messages=3).c()
        assert L.bbp_workspace_bytes(ctypes.byref(c), 10, 0, ctypes.byref(out)) == 0, d
        assert out.value == 0
    for d in (6, 12):
        c = pkg.DecoderParams(d=d, k=4, precision="fp32", algorithm="fused", messages=3).c()
        assert L.bbp_workspace_bytes(ctypes.byref(c), 10, 0, ctypes.byref(out)) == -4, d
    c = pkg.DecoderParams(d=11, k=3, precision="fp32", algorithm="fused", messages=3).c()
    assert L.bbp_workspace_bytes(ctypes.byref(c), 10, 0, ctypes.byref(out)) == -4
    c = pkg.DecoderParams(d=11, k=4, precision="fp32", algorithm="fused", messages=3).c()
    vp = ctypes.c_void_p
    fake = vp(256)                                  # never dereferenced: both calls return first
    assert L.bbp_decode_mixed(fake, fake, fake, None, 4, 12, ctypes.byref(c), fake, fake, fake, fake, fake, fake,
                              1 << 20, None) == -4
    c3 = pkg.DecoderParams(d=11, k=3, precision="fp32", algorithm="fused", messages=3).c()
    assert L.bbp_decode_mixed(fake, fake, fake, None, 4, 11, ctypes.byref(c3), fake, fake, fake, fake, fake, fake,
                              1 << 20, None) == -4
