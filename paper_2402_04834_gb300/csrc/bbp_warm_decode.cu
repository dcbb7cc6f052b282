// The learned decoder as one call: features of the distinct message rows,
// the warm-start network on the tensor cores, the expansion of each proposal
// to every coset it stands for, and the fused decode started from the
// proposals (the paper starts from uniform messages, Remark 2; learned
// techniques are its suggestion for future work, Sec. V).  A host-buffer
// variant copies the syndromes in and the results out.
#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include <vector>

#include "../../include/blockbp.h"
#include "bbp_fused.cuh"
#include "bbp_warm_features.cuh"

namespace {

using bbp::Geo;

size_t a256(size_t x) { return (x + 255) / 256 * 256; }

// Distinct feature rows of the geometry on the device, the same tables as
// bbp_message_classes: which logical strings each message's window sees
// (1, 2 or 4 rows), a running row offset by one thread, then the tables.
__global__ void classes_kernel(Geo g, int M, int32_t* off, int32_t* uniq_of, int32_t* row_key) {
  // seen[idx] for every message, kept in off[] until the scan.
  for (int idx = threadIdx.x; idx < M; idx += blockDim.x) off[idx] = 0;
  __syncthreads();
  if (threadIdx.x == 0) {
    int idx = 0;
    for (int I = 0; I < g.nb; ++I)
      for (int J = 0; J < g.nb; ++J)
        for (int dir = 0; dir < 4; ++dir)
          if (g.has(I, J, dir)) off[idx++] = (I * g.nb + J) * 4 + dir;   // message key, for now
  }
  __syncthreads();
  for (int idx = threadIdx.x; idx < M; idx += blockDim.x) {
    const int key = off[idx];
    const int seen = bbp::warm::window_logicals(g, bbp::warm::msg_geo(g, key / 4 / g.nb, (key / 4) % g.nb, key & 3));
    off[idx] = seen;
  }
  __syncthreads();
  if (threadIdx.x == 0) {   // exclusive scan of the row counts, the seen bits kept in the low two bits
    int u = 0;
    for (int idx = 0; idx < M; ++idx) {
      const int seen = off[idx];
      const int cnt = (seen & 1 ? 2 : 1) * (seen & 2 ? 2 : 1);
      off[idx] = (u << 2) | seen;
      u += cnt;
    }
  }
  __syncthreads();
  for (int idx = threadIdx.x; idx < M; idx += blockDim.x) {
    const int seen = off[idx] & 3, base = off[idx] >> 2;
    // Coset c = (bx, bz) is represented by (bx if the window sees X-bar, bz
    // if it sees Z-bar); representatives take rows in coset order I, X, Y, Z.
    int row_of_rep[4] = {-1, -1, -1, -1};
    int u = base;
    for (int c = 0; c < 4; ++c) {
      const int bx = (c == 1 || c == 2) && (seen & 1), bz = (c == 2 || c == 3) && (seen & 2);
      const int rep = bx ? (bz ? 2 : 1) : (bz ? 3 : 0);
      if (row_of_rep[rep] < 0) {
        row_of_rep[rep] = u;
        row_key[u++] = rep * M + idx;
      }
      uniq_of[c * M + idx] = row_of_rep[rep];
    }
  }
}

struct WarmPlan {
  int M, U;
  size_t tables, infer_ws, feats, lens, rows, msgs, arena, io, total_dev, total_host;
};

int plan_for(const bbp_params* prm, int64_t B, WarmPlan* w) {
  if (!prm || prm->algorithm != BBP_ALG_FUSED || prm->k > 4 || prm->d < 2 || prm->d > 64 || prm->k < 1)
    return BBP_EINVAL;
  if (B < 0 || B > (int64_t(1) << 29)) return BBP_EINVAL;
  int rc = bbp_message_count(prm, &w->M);
  if (rc != BBP_OK) return rc;
  std::vector<int32_t> uq(4 * (size_t)w->M), rk(4 * (size_t)w->M);
  rc = bbp_message_classes(prm, uq.data(), rk.data(), &w->U);
  if (rc != BBP_OK) return rc;
  size_t infer_ws = 0;
  if ((rc = bbp_warm_workspace_bytes(0, &infer_ws)) != BBP_OK) return rc;
  const size_t N = (size_t)B * w->U;
  w->tables = a256(3 * 4 * (size_t)w->M * sizeof(int32_t));   // scan scratch, uniq_of, row_key
  w->infer_ws = a256(infer_ws);
  w->feats = a256(N * (BBP_WARM_FEATURES / 32) * sizeof(uint32_t));   // feature bits
  w->lens = a256(N * sizeof(int32_t));
  w->rows = a256(N * BBP_WARM_OUT * sizeof(float));
  w->msgs = a256((size_t)B * 4 * w->M * BBP_WARM_OUT * sizeof(float));
  if ((rc = bbp_workspace_bytes(prm, B, 0, &w->arena)) != BBP_OK) return rc;
  w->arena = a256(w->arena);
  const size_t m = 2 * (size_t)prm->d * (prm->d - 1);
  w->io = a256((size_t)B * m) + 2 * a256((size_t)B * 4 * 8) + 2 * a256((size_t)B * 4 * 4) + a256((size_t)B);
  w->total_dev = w->tables + w->infer_ws + w->feats + w->lens + w->rows + w->msgs + w->arena;
  w->total_host = w->total_dev + w->io;
  return BBP_OK;
}

}  // namespace

extern "C" {

int bbp_decode_warm_workspace_bytes(const bbp_params* prm, int64_t B, int include_io, size_t* bytes) {
  if (!bytes) return BBP_EINVAL;
  WarmPlan w;
  const int rc = plan_for(prm, B, &w);
  if (rc != BBP_OK) return rc;
  *bytes = include_io ? w.total_host : w.total_dev;
  return BBP_OK;
}

int bbp_decode_warm(const float* theta, const uint8_t* syndromes, int64_t B, const bbp_params* prm, float alpha,
                    double* logp, double* delta, int32_t* iters, int32_t* flags, int8_t* decision, void* workspace,
                    size_t workspace_bytes, void* stream) {
  WarmPlan w;
  int rc = plan_for(prm, B, &w);
  if (rc != BBP_OK) return rc;
  if (!(alpha >= 0.f && alpha <= 1.f)) return BBP_EINVAL;
  if (B == 0) return BBP_OK;
  if (!theta || !syndromes || !logp || !delta || !iters || !flags || !decision || !workspace) return BBP_EINVAL;
  if (reinterpret_cast<uintptr_t>(workspace) % 256 != 0) return BBP_EINVAL;
  if (workspace_bytes < w.total_dev) return BBP_ENOSPACE;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  // The network's scratch first, so that its status word sits at byte
  // BBP_WARM_STATUS_OFFSET of the workspace as for bbp_warm_infer.
  char* p = static_cast<char*>(workspace);
  void* infer_ws = p;                                p += w.infer_ws;
  int32_t* off = reinterpret_cast<int32_t*>(p);
  int32_t* uniq_of = off + 4 * w.M;
  int32_t* row_key = uniq_of + 4 * w.M;
  p += w.tables;
  uint32_t* bits = reinterpret_cast<uint32_t*>(p);   p += w.feats;
  int32_t* lens = reinterpret_cast<int32_t*>(p);     p += w.lens;
  float* rows = reinterpret_cast<float*>(p);         p += w.rows;
  float* msgs = reinterpret_cast<float*>(p);         p += w.msgs;
  void* arena = p;
  const Geo g = bbp::make_geo(prm->d, prm->k);
  classes_kernel<<<1, 256, 0, st>>>(g, w.M, off, uniq_of, row_key);
  if (cudaGetLastError() != cudaSuccess) return BBP_ECUDA;
  // Features as bits (32 bytes a row instead of 1 KB of FP32), expanded to
  // the same BF16 operands inside the network kernel.
  if ((rc = bbp_message_feature_bits_rows(syndromes, B, prm, row_key, w.U, bits, lens, stream)) != BBP_OK) return rc;
  const long long N = (long long)B * w.U;
  for (long long a = 0; a < N; a += BBP_WARM_MAX_ROWS) {
    const long long n = N - a < BBP_WARM_MAX_ROWS ? N - a : BBP_WARM_MAX_ROWS;
    rc = bbp_warm_infer_bits(theta, bits + a * (BBP_WARM_FEATURES / 32), lens + a, n, prm->p, alpha,
                             rows + a * BBP_WARM_OUT, infer_ws, w.infer_ws, stream);
    if (rc != BBP_OK) return rc;
  }
  if ((rc = bbp_expand_rows(rows, B, w.U, uniq_of, w.M, msgs, stream)) != BBP_OK) return rc;
  return bbp_decode_batch_ex(syndromes, B, prm, msgs, nullptr, logp, delta, iters, flags, decision, arena, w.arena,
                             stream);
}

int bbp_decode_warm_host(const float* theta, const uint8_t* syndromes, int64_t B, const bbp_params* prm, float alpha,
                         double* logp, double* delta, int32_t* iters, int32_t* flags, int8_t* decision,
                         void* workspace, size_t workspace_bytes, void* stream) {
  WarmPlan w;
  int rc = plan_for(prm, B, &w);
  if (rc != BBP_OK) return rc;
  if (!(alpha >= 0.f && alpha <= 1.f)) return BBP_EINVAL;
  if (B == 0) return BBP_OK;
  if (!theta || !syndromes || !decision || !workspace) return BBP_EINVAL;
  if (reinterpret_cast<uintptr_t>(workspace) % 256 != 0) return BBP_EINVAL;
  if (workspace_bytes < w.total_host) return BBP_ENOSPACE;
  const size_t m = 2 * (size_t)prm->d * (prm->d - 1);
  char* base = static_cast<char*>(workspace) + w.total_dev;
  uint8_t* d_synd = reinterpret_cast<uint8_t*>(base);  base += a256((size_t)B * m);
  double* d_logp = reinterpret_cast<double*>(base);    base += a256((size_t)B * 4 * 8);
  double* d_delta = reinterpret_cast<double*>(base);   base += a256((size_t)B * 4 * 8);
  int32_t* d_iters = reinterpret_cast<int32_t*>(base); base += a256((size_t)B * 4 * 4);
  int32_t* d_flags = reinterpret_cast<int32_t*>(base); base += a256((size_t)B * 4 * 4);
  int8_t* d_dec = reinterpret_cast<int8_t*>(base);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (cudaMemcpyAsync(d_synd, syndromes, (size_t)B * m, cudaMemcpyHostToDevice, st) != cudaSuccess) return BBP_ECUDA;
  rc = bbp_decode_warm(theta, d_synd, B, prm, alpha, d_logp, d_delta, d_iters, d_flags, d_dec, workspace,
                       w.total_dev, stream);
  if (rc != BBP_OK) return rc;
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

}  // extern "C"
