// C ABI of the blockBP decoder: argument checks, workspace sizing and the
// kernel launches.  See include/blockbp.h for the contract of each call.
#include <cuda_runtime.h>
#include <math.h>
#include <stddef.h>
#include <stdint.h>

#include "../../include/blockbp.h"
#include "bbp_launch.h"

namespace {

using bbp::Geo;

size_t align256(size_t x) { return (x + 255) / 256 * 256; }

// Launch shape of the fused kernel for this request at geometry g; *gm is
// set when its messages live in the workspace.
// *lean: 0, or the CTAs per SM the register-form-only kernel is sized for.
bool shape_of(const bbp_params* p, const Geo& g, int M, int* warps, int* cosets, bool* gm, int* lean = nullptr,
              bool allow_lean = true) {
  *warps = p->launch_warps;
  *cosets = p->launch_cosets;
  int messages = p->launch_messages, lb = 0;
  const bool ok = bbp::fused_shape(p->precision, g, M, warps, cosets, &messages, allow_lean, &lb);
  *gm = messages == 2;
  if (lean) *lean = messages == 3 ? lb : 0;
  return ok;
}

int check_params(const bbp_params* p) {
  if (!p) return BBP_EINVAL;
  if (p->d < 2 || p->d > 64) return BBP_EINVAL;
  if (p->k < 1 || p->D < 1 || p->max_iter < 0 || p->max_iter > 100000) return BBP_EINVAL;
  if (!(p->p > 0.0 && p->p < 0.75)) return BBP_EINVAL;
  if (!(p->eta >= 0.0 && p->eta < 1.0)) return BBP_EINVAL;
  if (!(p->delta0 >= 0.0) || !(p->delta1 >= 0.0) || !(p->cutoff >= 0.0 && p->cutoff < 1.0)) return BBP_EINVAL;
  if (p->precision != BBP_FP64 && p->precision != BBP_FP32) return BBP_EINVAL;
  if (p->algorithm != BBP_ALG_MPS && p->algorithm != BBP_ALG_FUSED) return BBP_EINVAL;
  if (p->algorithm == BBP_ALG_MPS && (p->k > bbp::kMaxK || p->D > bbp::kMaxD)) return BBP_EUNSUPPORTED;
  if (p->launch_warps != 0 && p->launch_warps != 2 && p->launch_warps != 3 && p->launch_warps != 4 &&
      p->launch_warps != 6 && p->launch_warps != 8 && p->launch_warps != 16)
    return BBP_EINVAL;
  if (p->launch_cosets != 0 && p->launch_cosets != 1 && p->launch_cosets != 2 && p->launch_cosets != 4)
    return BBP_EINVAL;
  if (p->launch_ctas_per_sm < 0 || p->launch_ctas_per_sm > 32) return BBP_EINVAL;
  if (p->launch_messages < 0 || p->launch_messages > 3) return BBP_EINVAL;
  if (p->algorithm == BBP_ALG_FUSED) {
    if (p->k > bbp::kFusedMaxK) return BBP_EUNSUPPORTED;
    const bbp::Geo g = bbp::make_geo(p->d, p->k);
    int M = 0, ae = 0, w = 0, c = 0;
    bool gm = false;
    bbp::count_messages(g, 1, &M, &ae);
    if (!shape_of(p, g, M, &w, &c, &gm)) return BBP_EUNSUPPORTED;
  }
  return BBP_OK;
}

struct Sizes {
  Geo g;
  int M, arena_elems, m;
  size_t elem, arena_bytes, io_bytes;
  int warps, cosets;      // fused: launch shape
  bool gm;                // fused: messages in the workspace
  int lean;               // fused: every block update in register form (CTAs per SM it is sized for), else 0
  long long slots;        // fused with gm: message slots in the arena
};

// Fused path with its messages in the workspace: one slot of G cosets x M
// messages x (16 or 64) scalars per resident CTA, at most one per item.
long long fused_slots(int64_t B, int G) {
  const long long items = (long long)B * (4 / G);
  return items < bbp::kFusedSlots ? items : bbp::kFusedSlots;
}
size_t fused_slot_bytes(int k, int G, int M, size_t elem) { return (size_t)G * M * (k > 4 ? 64 : 16) * elem; }

Sizes sizes_for(const bbp_params* p, int64_t B) {
  Sizes s;
  s.g = bbp::make_geo(p->d, p->k);
  bbp::count_messages(s.g, p->D, &s.M, &s.arena_elems);
  s.m = 2 * p->d * (p->d - 1);
  s.elem = p->precision == BBP_FP64 ? sizeof(double) : sizeof(float);
  s.slots = 0;
  s.warps = s.cosets = 0;
  s.gm = false;
  s.lean = 0;
  if (p->algorithm != BBP_ALG_FUSED) {
    s.arena_bytes = align256((size_t)B * 4 * (size_t)s.arena_elems * s.elem);
  } else {
    int M1 = 0, ae = 0;
    bbp::count_messages(s.g, 1, &M1, &ae);
    s.arena_bytes = 0;
    if (shape_of(p, s.g, M1, &s.warps, &s.cosets, &s.gm, &s.lean) && s.gm) {
      s.slots = fused_slots(B, s.cosets);
      s.arena_bytes = align256((size_t)s.slots * fused_slot_bytes(p->k, s.cosets, M1, s.elem));
    }
    // The default register-form-only shape needs no workspace, but a mixed
    // batch cannot take it (it may hold any distance): the size returned
    // also covers the default shape bbp_decode_mixed takes for d_max.
    int w2 = 0, c2 = 0;
    bool gm2 = false;
    if (s.lean && p->launch_messages == 0 && shape_of(p, s.g, M1, &w2, &c2, &gm2, nullptr, false) && gm2)
      s.arena_bytes = align256((size_t)fused_slots(B, c2) * fused_slot_bytes(p->k, c2, M1, s.elem));
  }
  s.io_bytes = align256((size_t)B * s.m) + align256((size_t)B * 4 * 8) * 2 +
               align256((size_t)B * 4 * 4) * 2 + align256((size_t)B);
  return s;
}

}  // namespace

extern "C" {

const char* bbp_version(void) {
#ifdef BLOCKBP_CHECKS
  return "blockbp-gb300 0.1 (sm_103a, device bounds checks)";
#else
  return "blockbp-gb300 0.1 (sm_103a)";
#endif
}

const char* bbp_strerror(int code) {
  switch (code) {
    case BBP_OK: return "ok";
    case BBP_EINVAL: return "invalid argument";
    case BBP_ECUDA: return "CUDA runtime error";
    case BBP_ENOSPACE: return "workspace too small";
    case BBP_EUNSUPPORTED: return "block size or bond dimension outside the compiled kernels";
    case BBP_ETOOLARGE: return "batch needs more than the 32 MiB static workspace";
    default: return "unknown error";
  }
}

int bbp_workspace_bytes(const bbp_params* prm, int64_t B, int include_io, size_t* bytes) {
  const int rc = check_params(prm);
  if (rc != BBP_OK) return rc;
  if (!bytes || B < 0 || B > (int64_t(1) << 29)) return BBP_EINVAL;
  const Sizes s = sizes_for(prm, B);
  *bytes = s.arena_bytes + (include_io ? s.io_bytes : 0);
  return BBP_OK;
}

int bbp_decode_batch(const uint8_t* syndromes, int64_t B, const bbp_params* prm, double* logp,
                     double* delta, int32_t* iters, int32_t* flags, int8_t* decision, void* workspace,
                     size_t workspace_bytes, void* stream) {
  return bbp_decode_batch_ex(syndromes, B, prm, nullptr, nullptr, logp, delta, iters, flags, decision,
                             workspace, workspace_bytes, stream);
}

int bbp_decode_batch_ex(const uint8_t* syndromes, int64_t B, const bbp_params* prm, const float* init_msgs,
                        float* final_msgs, double* logp, double* delta, int32_t* iters, int32_t* flags,
                        int8_t* decision, void* workspace, size_t workspace_bytes, void* stream) {
  const int rc = check_params(prm);
  if (rc != BBP_OK) return rc;
  if (B < 0 || B > (int64_t(1) << 29)) return BBP_EINVAL;
  if (B == 0) return BBP_OK;
  const Sizes s = sizes_for(prm, B);
  if (!syndromes || !logp || !delta || !iters || !flags || !decision) return BBP_EINVAL;
  if (s.arena_bytes > 0 && !workspace) return BBP_EINVAL;
  if (reinterpret_cast<uintptr_t>(workspace) % 256 != 0) return BBP_EINVAL;
  if (workspace_bytes < s.arena_bytes) return BBP_ENOSPACE;
  bbp::LaunchArgs a;
  a.geo = s.g; a.M = s.M; a.D = prm->D; a.max_iter = prm->max_iter; a.arena_elems = s.arena_elems;
  a.p = prm->p; a.eta = prm->eta; a.delta0 = prm->delta0; a.delta1 = prm->delta1; a.cutoff = prm->cutoff;
  a.synd = syndromes; a.arena = workspace; a.logp = logp; a.delta = delta; a.iters = iters;
  a.flags = flags; a.decision = decision; a.B = B;
  if ((init_msgs || final_msgs) && (prm->algorithm != BBP_ALG_FUSED || prm->k > 4)) return BBP_EINVAL;
  a.init_msgs = init_msgs; a.final_msgs = final_msgs;
  a.slots = s.slots;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  cudaError_t e;
  if (prm->algorithm == BBP_ALG_FUSED) {
    if (s.warps == 0) return BBP_EUNSUPPORTED;
    e = prm->precision == BBP_FP64 ? bbp::launch_fused_f64(a, s.warps, s.cosets, s.gm, s.lean, st)
                                   : bbp::launch_fused_f32(a, s.warps, s.cosets, s.gm, s.lean, st);
  } else
    e = prm->precision == BBP_FP64 ? bbp::launch_decode_f64(a, st) : bbp::launch_decode_f32(a, st);
  if (e != cudaSuccess) return BBP_ECUDA;
  e = bbp::launch_decide(a, st);
  return e == cudaSuccess ? BBP_OK : BBP_ECUDA;
}

int bbp_decode_batch_host(const uint8_t* syndromes, int64_t B, const bbp_params* prm, double* logp,
                          double* delta, int32_t* iters, int32_t* flags, int8_t* decision,
                          void* workspace, size_t workspace_bytes, void* stream) {
  const int rc = check_params(prm);
  if (rc != BBP_OK) return rc;
  if (B < 0 || B > (int64_t(1) << 29)) return BBP_EINVAL;
  if (B == 0) return BBP_OK;
  if (!syndromes || !decision || !workspace) return BBP_EINVAL;
  if (reinterpret_cast<uintptr_t>(workspace) % 256 != 0) return BBP_EINVAL;
  const Sizes s = sizes_for(prm, B);
  if (workspace_bytes < s.arena_bytes + s.io_bytes) return BBP_ENOSPACE;
  char* base = static_cast<char*>(workspace) + s.arena_bytes;
  uint8_t* d_synd = reinterpret_cast<uint8_t*>(base);  base += align256((size_t)B * s.m);
  double* d_logp = reinterpret_cast<double*>(base);    base += align256((size_t)B * 4 * 8);
  double* d_delta = reinterpret_cast<double*>(base);   base += align256((size_t)B * 4 * 8);
  int32_t* d_iters = reinterpret_cast<int32_t*>(base); base += align256((size_t)B * 4 * 4);
  int32_t* d_flags = reinterpret_cast<int32_t*>(base); base += align256((size_t)B * 4 * 4);
  int8_t* d_dec = reinterpret_cast<int8_t*>(base);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (cudaMemcpyAsync(d_synd, syndromes, (size_t)B * s.m, cudaMemcpyHostToDevice, st) != cudaSuccess)
    return BBP_ECUDA;
  const int r = bbp_decode_batch(d_synd, B, prm, d_logp, d_delta, d_iters, d_flags, d_dec, workspace,
                                 s.arena_bytes, stream);
  if (r != BBP_OK) return r;
  if (cudaMemcpyAsync(decision, d_dec, (size_t)B, cudaMemcpyDeviceToHost, st) != cudaSuccess) return BBP_ECUDA;
  if (logp && cudaMemcpyAsync(logp, d_logp, (size_t)B * 32, cudaMemcpyDeviceToHost, st) != cudaSuccess)
    return BBP_ECUDA;
  if (delta && cudaMemcpyAsync(delta, d_delta, (size_t)B * 32, cudaMemcpyDeviceToHost, st) != cudaSuccess)
    return BBP_ECUDA;
  if (iters && cudaMemcpyAsync(iters, d_iters, (size_t)B * 16, cudaMemcpyDeviceToHost, st) != cudaSuccess)
    return BBP_ECUDA;
  if (flags && cudaMemcpyAsync(flags, d_flags, (size_t)B * 16, cudaMemcpyDeviceToHost, st) != cudaSuccess)
    return BBP_ECUDA;
  return cudaStreamSynchronize(st) == cudaSuccess ? BBP_OK : BBP_ECUDA;
}

int bbp_decode_mixed(const uint8_t* syndromes, const int64_t* offsets, const int32_t* d_of, const int32_t* order,
                     int64_t B, int32_t d_max, const bbp_params* prm, double* logp, double* delta, int32_t* iters,
                     int32_t* flags, int8_t* decision, void* workspace, size_t workspace_bytes, void* stream) {
  if (!prm || prm->algorithm != BBP_ALG_FUSED) return BBP_EINVAL;
  // The register-form-only kernels only on request (launch_messages = 3):
  // the caller vouches that every distance of the batch is odd.
  const bool lean_req = prm->launch_messages == 3;
  if (lean_req && (prm->k != 4 || d_max % 2 == 0)) return BBP_EUNSUPPORTED;
  bbp_params q = *prm;
  q.d = d_max;                                   // validate the largest geometry
  const int rc = check_params(&q);
  if (rc != BBP_OK) return rc;
  if (B < 0 || B > (int64_t(1) << 29)) return BBP_EINVAL;
  if (B == 0) return BBP_OK;
  if (!syndromes || !offsets || !d_of || !logp || !delta || !iters || !flags || !decision || !workspace)
    return BBP_EINVAL;
  if (workspace_bytes < 256 || reinterpret_cast<uintptr_t>(workspace) % 256 != 0) return BBP_ENOSPACE;
  bbp::LaunchArgs a;
  a.geo = bbp::make_geo(d_max, prm->k);
  a.M = 0; a.D = prm->D; a.max_iter = prm->max_iter; a.arena_elems = 0;
  a.p = prm->p; a.eta = prm->eta; a.delta0 = prm->delta0; a.delta1 = prm->delta1; a.cutoff = prm->cutoff;
  a.synd = syndromes; a.arena = nullptr; a.logp = logp; a.delta = delta; a.iters = iters;
  a.flags = flags; a.decision = decision; a.B = B;
  bbp::MixedLaunch m;
  m.d_of = d_of; m.offsets = offsets; m.order = order;
  m.counter = static_cast<unsigned long long*>(workspace);
  m.d_max = d_max; m.ctas_per_sm = prm->launch_ctas_per_sm;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  int Mmax = 0, ae = 0, w = 0, c = 0, lean = 0;
  bool gm = false;
  bbp::count_messages(a.geo, 1, &Mmax, &ae);
  if (!shape_of(prm, a.geo, Mmax, &w, &c, &gm, &lean, lean_req)) return BBP_EUNSUPPORTED;
  if (gm) {   // message slots after the counter
    const size_t elem = prm->precision == BBP_FP64 ? sizeof(double) : sizeof(float);
    m.slots = fused_slots(B, c);
    if (workspace_bytes < 256 + (size_t)m.slots * fused_slot_bytes(prm->k, c, Mmax, elem)) return BBP_ENOSPACE;
    m.slot_base = static_cast<char*>(workspace) + 256;
  }
  cudaError_t e = prm->precision == BBP_FP64 ? bbp::launch_fused_mixed_f64(a, m, w, c, gm, lean, st)
                                             : bbp::launch_fused_mixed_f32(a, m, w, c, gm, lean, st);
  if (e != cudaSuccess) return BBP_ECUDA;
  e = bbp::launch_decide(a, st);
  return e == cudaSuccess ? BBP_OK : BBP_ECUDA;
}

int bbp_sample(uint64_t seed, int64_t first_shot, int64_t B, int32_t d, double p, uint8_t* ex,
               uint8_t* ez, uint8_t* syndromes, int8_t* true_class, void* stream) {
  if (d < 2 || d > 64 || B < 0 || B > (int64_t(1) << 31) - 1 || first_shot < 0) return BBP_EINVAL;
  if (!(p > 0.0 && p < 0.75) || !syndromes || !true_class) return BBP_EINVAL;
  if (B == 0) return BBP_OK;
  const unsigned long long thr = (unsigned long long)((1.0 - p) * 9007199254740992.0);
  cudaError_t e = bbp::launch_sample(seed, first_shot, B, d, thr, ex, ez, syndromes, true_class,
                                     static_cast<cudaStream_t>(stream));
  return e == cudaSuccess ? BBP_OK : BBP_ECUDA;
}

int bbp_pure_error(int32_t d, const uint8_t* syndromes, int64_t B, uint8_t* fx, uint8_t* fz, void* stream) {
  if (d < 2 || d > 64 || B < 0 || B > (int64_t(1) << 31) - 1) return BBP_EINVAL;
  if (B == 0) return BBP_OK;
  if (!syndromes || !fx || !fz) return BBP_EINVAL;
  const cudaError_t e = bbp::launch_pure_error(d, syndromes, B, fx, fz, static_cast<cudaStream_t>(stream));
  return e == cudaSuccess ? BBP_OK : BBP_ECUDA;
}

}  // extern "C"
