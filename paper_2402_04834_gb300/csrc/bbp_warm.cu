// Learned warm start for the fused-block decoder: message features, the
// network F -> H -> H -> O with GELU (forward, backward, Adam), and its
// inference into initial messages.  The paper initialises every message to
// the uniform distribution (Remark 2) and names learned techniques as a way
// to improve BP (Sec. V); cold start stays the default and the fallback.
//
// Features of a message: see bbp_warm_features.cuh.
//
// Training is FP32 CUDA-core code: a 64 x 64-tile GEMM with bias / GELU
// epilogues and transposed operands for the backward pass.  Inference runs
// on the tensor cores (bbp_warm_tc.cu).
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "../../include/blockbp.h"
#include "bbp_fused.cuh"
#include "bbp_launch.h"
#include "bbp_warm_features.cuh"
#include "bbp_warm_tc.h"

namespace bbp {
namespace warm {

constexpr int F = BBP_WARM_FEATURES;   // 256
constexpr int H = BBP_WARM_HIDDEN;     // 256
constexpr int O = BBP_WARM_OUT;        // 16
constexpr int kParams = F * H + H + H * H + H + H * O + O;

// ---------------------------------------------------------------------------
// Features (bbp_warm_features.cuh), one CTA per (syndrome, coset).
__global__ void features_kernel(Geo g, int M, double p, const uint8_t* synd, float* feats, int32_t* lens) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int W = g.W, d = g.d, nb = g.nb;
  const int m = 2 * d * (d - 1);
  uint8_t* s = smem;
  uint8_t* frame = smem + align_up(m, 16);
  int16_t* meta = reinterpret_cast<int16_t*>(frame + align_up(W * W, 16));
  const long long cta = blockIdx.x;
  const long long shot = cta >> 2;
  const int coset = (int)(cta & 3);
  for (int i = threadIdx.x; i < m; i += blockDim.x) s[i] = synd[shot * m + i];
  __syncthreads();
  for (int e = threadIdx.x; e < W * W; e += blockDim.x) frame[e] = frame_byte(s, d, e / W, e % W, coset);
  if (threadIdx.x == 0) {
    int idx = 0;
    for (int I = 0; I < nb; ++I)
      for (int J = 0; J < nb; ++J)
        for (int dir = 0; dir < 4; ++dir)
          if (g.has(I, J, dir)) meta[idx++] = (int16_t)((I * nb + J) * 4 + dir);
  }
  __syncthreads();
  const float p10 = (float)(10.0 * p);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int idx = warp; idx < M; idx += nw) {
    const int key = meta[idx];
    const MsgGeo f = msg_geo(g, key / 4 / nb, (key / 4) % nb, key & 3);
    float* out = feats + (cta * M + idx) * F;
    // One window node per lane, its five channels at once (each channel's
    // 49 values are contiguous, so the stores stay coalesced).
    for (int pos = lane; pos < 49; pos += 32) {
      float c[5];
      window_node(g, f, pos, frame, s, c);
#pragma unroll
      for (int ch = 0; ch < 5; ++ch) out[ch * 49 + pos] = c[ch];
    }
    if (lane < F - 245) out[245 + lane] = tail_feature(f, 245 + lane, p10);
    if (lane == 0 && lens) lens[cta * M + idx] = 1 << f.h;
  }
}

// Features of listed rows: row u of syndrome b is (coset, message) =
// row_key[u] = coset * M + message; one CTA per syndrome holding the four
// coset frames.  Row (b, u) is written at b * U + u: 256 floats, or with
// BITS 256 bits (8 words; bit q of word q / 32 set where feature q is not
// zero: every feature is 0 or 1 except 10 p, which inference puts back).
template <bool BITS>
__global__ void features_rows_kernel(Geo g, int M, double p, const uint8_t* synd, const int32_t* row_key, int U,
                                     float* feats, uint32_t* bits, int32_t* lens) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int W = g.W, WW = W * W, d = g.d, nb = g.nb;
  const int m = 2 * d * (d - 1);
  uint8_t* s = smem;
  uint8_t* frames = smem + align_up(m, 16);
  int16_t* meta = reinterpret_cast<int16_t*>(frames + align_up(4 * WW, 16));
  const long long shot = blockIdx.x;
  for (int i = threadIdx.x; i < m; i += blockDim.x) s[i] = synd[shot * m + i];
  __syncthreads();
  for (int e = threadIdx.x; e < 4 * WW; e += blockDim.x) {
    const int c = e / WW, ij = e - c * WW;
    frames[e] = frame_byte(s, d, ij / W, ij % W, c);
  }
  if (threadIdx.x == 0) {
    int idx = 0;
    for (int I = 0; I < nb; ++I)
      for (int J = 0; J < nb; ++J)
        for (int dir = 0; dir < 4; ++dir)
          if (g.has(I, J, dir)) meta[idx++] = (int16_t)((I * nb + J) * 4 + dir);
  }
  __syncthreads();
  const float p10 = (float)(10.0 * p);
  if constexpr (BITS) {
    // A thread per row: its 49 window nodes in turn, each channel's bit set
    // in place (feature ch * 49 + pos; the loops unrolled so that the eight
    // words stay in registers), then the tail features.
    for (int u = threadIdx.x; u < U; u += blockDim.x) {
      const int key = row_key[u];
      const int coset = key / M, idx = key - coset * M;
      const int mk = meta[idx];
      const MsgGeo f = msg_geo(g, mk / 4 / nb, (mk / 4) % nb, mk & 3);
      const uint8_t* frame = frames + coset * WW;
      uint32_t w[8] = {0u, 0u, 0u, 0u, 0u, 0u, 0u, 0u};
#pragma unroll
      for (int pos = 0; pos < 49; ++pos) {
        float c[5];
        window_node(g, f, pos, frame, s, c);
#pragma unroll
        for (int ch = 0; ch < 5; ++ch)
          if (c[ch] != 0.f) w[(ch * 49 + pos) >> 5] |= 1u << ((ch * 49 + pos) & 31);
      }
#pragma unroll
      for (int q = 245; q < F; ++q)
        if (tail_feature(f, q, p10) != 0.f) w[q >> 5] |= 1u << (q & 31);
      uint4* out = reinterpret_cast<uint4*>(bits + (shot * U + u) * 8);
      out[0] = make_uint4(w[0], w[1], w[2], w[3]);
      out[1] = make_uint4(w[4], w[5], w[6], w[7]);
      if (lens) lens[shot * U + u] = 1 << f.h;
    }
  } else {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int u = warp; u < U; u += nw) {
      const int key = row_key[u];
      const int coset = key / M, idx = key - coset * M;
      const int mk = meta[idx];
      const MsgGeo f = msg_geo(g, mk / 4 / nb, (mk / 4) % nb, mk & 3);
      const uint8_t* frame = frames + coset * WW;
      float* out = feats + (shot * U + u) * F;
      for (int pos = lane; pos < 49; pos += 32) {
        float c[5];
        window_node(g, f, pos, frame, s, c);
#pragma unroll
        for (int ch = 0; ch < 5; ++ch) out[ch * 49 + pos] = c[ch];
      }
      if (lane < F - 245) out[245 + lane] = tail_feature(f, 245 + lane, p10);
      if (lane == 0 && lens) lens[shot * U + u] = 1 << f.h;
    }
  }
}

// msgs[b][c][idx] = rows[b][uniq_of[c * M + idx]], 16 floats each (four
// float4 per message, one per thread).
__global__ void expand_rows_kernel(const float4* rows, long long B, int U, const int32_t* uniq_of, int M,
                                   float4* msgs) {
  const long long total = B * 4 * M * 4;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    const int q = (int)(t & 3);
    const long long r = t >> 2;                       // (b, c, idx)
    const long long b = r / (4 * M);
    const int cm = (int)(r - b * 4 * M);
    msgs[t] = rows[(b * U + uniq_of[cm]) * 4 + q];
  }
}

// ---------------------------------------------------------------------------
// GEMM: C[M x N] = op(A) op(B) (+ bias) with optional GELU, FP32.
// op(A) is A (M x K, row-major, lda) or A^T with A stored K x M; op(B) is B
// (K x N, ldb) or B^T with B stored N x K.  Optional outputs: the
// pre-activation Z and the activation C; accumulate adds into C.
__device__ __forceinline__ float gelu(float x) { return 0.5f * x * (1.f + erff(x * 0.70710678118654752f)); }
__device__ __forceinline__ float gelu_grad(float x) {
  return 0.5f * (1.f + erff(x * 0.70710678118654752f)) + x * expf(-0.5f * x * x) * 0.39894228040143268f;
}

template <bool TA, bool TB>
__global__ void __launch_bounds__(256) gemm_kernel(int Mr, int N, int K, const float* __restrict__ A, int lda,
                                                   const float* __restrict__ B, int ldb, float* C, int ldc,
                                                   const float* __restrict__ bias, float* Z, int act, int accumulate) {
  constexpr int BM = 64, BN = 64, BK = 16;
  __shared__ float As[BK][BM + 4];
  __shared__ float Bs[BK][BN + 4];
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
  float acc[4][4] = {};
  for (int k0 = 0; k0 < K; k0 += BK) {
    for (int e = threadIdx.x; e < BM * BK; e += 256) {
      // Walk the tile along the operand's contiguous dimension (coalesced).
      const int mm = TA ? e % BM : e / BK, kk = TA ? e / BM : e % BK;
      const int gm = m0 + mm, gk = k0 + kk;
      float v = 0.f;
      if (gm < Mr && gk < K) v = TA ? A[(long long)gk * lda + gm] : A[(long long)gm * lda + gk];
      As[kk][mm] = v;
    }
    for (int e = threadIdx.x; e < BN * BK; e += 256) {
      const int nn = TB ? e / BK : e % BN, kk = TB ? e % BK : e / BN;
      const int gn = n0 + nn, gk = k0 + kk;
      float v = 0.f;
      if (gn < N && gk < K) v = TB ? B[(long long)gn * ldb + gk] : B[(long long)gk * ldb + gn];
      Bs[kk][nn] = v;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      float a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[kk][ty * 4 + i];
#pragma unroll
      for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tx * 4 + j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] += a[i] * b[j];
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int gm = m0 + ty * 4 + i;
    if (gm >= Mr) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int gn = n0 + tx * 4 + j;
      if (gn >= N) continue;
      float v = acc[i][j] + (bias ? bias[gn] : 0.f);
      if (Z) Z[(long long)gm * ldc + gn] = v;
      if (act) v = gelu(v);
      float* cp = C + (long long)gm * ldc + gn;
      *cp = accumulate ? *cp + v : v;
    }
  }
}

template <bool TA, bool TB>
cudaError_t gemm(int Mr, int N, int K, const float* A, int lda, const float* B, int ldb, float* C, int ldc,
                 const float* bias, float* Z, int act, int accumulate, cudaStream_t st) {
  dim3 grid((N + 63) / 64, (Mr + 63) / 64);
  gemm_kernel<TA, TB><<<grid, 256, 0, st>>>(Mr, N, K, A, lda, B, ldb, C, ldc, bias, Z, act, accumulate);
  return cudaGetLastError();
}

// u = masked exp(o - max) / norm; per-row loss 1 - <u,t>^2 and dL/do (mean over N).
__global__ void head_kernel(const float* logits, const int32_t* lens, const float* targets, long long N,
                            float* gO, float* loss_sum) {
  const long long row = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (row >= N) return;
  const int n = lens[row];
  float o[O], mm[O];
  float mx = -INFINITY;
  for (int i = 0; i < O; ++i) { o[i] = logits[row * O + i]; if (i < n) mx = fmaxf(mx, o[i]); }
  float s2 = 0.f;
  for (int i = 0; i < O; ++i) { mm[i] = i < n ? expf(o[i] - mx) : 0.f; s2 += mm[i] * mm[i]; }
  const float nm = sqrtf(s2), inv = 1.f / nm;
  if (targets) {
    float cdot = 0.f;
    for (int i = 0; i < O; ++i) cdot += mm[i] * inv * targets[row * O + i];
    atomicAdd(loss_sum, 1.f - cdot * cdot);
    // dL/du = -2 c t / N; dL/dm = (gu - <gu,u> u) / |m|; dL/do = dL/dm * m.
    const float sc = -2.f * cdot / (float)N;
    float gu_u = 0.f;
    for (int i = 0; i < O; ++i) gu_u += sc * targets[row * O + i] * mm[i] * inv;
    for (int i = 0; i < O; ++i) {
      const float gu = sc * targets[row * O + i];
      gO[row * O + i] = (gu - gu_u * mm[i] * inv) * inv * mm[i];
    }
  }
}

__global__ void gelu_back_kernel(float* gA, const float* Z, long long n) {
  const long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (e < n) gA[e] *= gelu_grad(Z[e]);
}

// Column sums of G [N x C] into out[C] (overwrites).
__global__ void colsum_kernel(const float* G, long long N, int C, float* out) {
  const int c = blockIdx.x;
  float acc = 0.f;
  for (long long r = threadIdx.x; r < N; r += blockDim.x) acc += G[r * C + c];
  __shared__ float sh[256];
  sh[threadIdx.x] = acc;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[c] = sh[0];
}

__global__ void adam_kernel(float* th, const float* gr, float* m, float* v, long long n, float lr, float b1,
                            float b2, float eps, float c1, float c2) {
  const long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (e >= n) return;
  const float g = gr[e];
  const float mm = b1 * m[e] + (1.f - b1) * g;
  const float vv = b2 * v[e] + (1.f - b2) * g * g;
  m[e] = mm;
  v[e] = vv;
  th[e] -= lr * (mm / c1) / (sqrtf(vv / c2) + eps);
}

struct Params {
  const float *W1, *b1, *W2, *b2, *W3, *b3;
};
__host__ __device__ inline Params split(const float* th) {
  Params P;
  P.W1 = th; P.b1 = P.W1 + F * H; P.W2 = P.b1 + H; P.b2 = P.W2 + H * H; P.W3 = P.b2 + H; P.b3 = P.W3 + H * O;
  return P;
}

}  // namespace warm
}  // namespace bbp

using namespace bbp;
using namespace bbp::warm;

namespace {
size_t al256(size_t x) { return (x + 255) / 256 * 256; }
// Scratch of a forward (+ backward) pass over N rows: Z1, A1, Z2, A2 [N x H],
// logits and dL/dlogits [N x O], and two [N x H] gradient buffers.
size_t pass_bytes(long long N) {
  const size_t train = al256((size_t)N * H * 4) * 6 + al256((size_t)N * O * 4) * 2 + 256;
  const size_t infer = infer_tc_workspace_bytes();
  return train > infer ? train : infer;
}
}  // namespace

extern "C" {

int bbp_warm_param_count(void) { return kParams; }

int bbp_message_count(const bbp_params* prm, int32_t* M) {
  if (!prm || !M || prm->d < 2 || prm->k < 1) return BBP_EINVAL;
  const Geo g = make_geo(prm->d, prm->k);
  int m = 0, ae = 0;
  count_messages(g, 1, &m, &ae);
  *M = m;
  return BBP_OK;
}

int bbp_message_features(const uint8_t* syndromes, int64_t B, const bbp_params* prm, float* feats,
                         int32_t* lens, void* stream) {
  if (!prm || !syndromes || !feats || B < 0 || prm->d < 2 || prm->k < 1 || prm->k > kFusedK) return BBP_EINVAL;
  if (B == 0) return BBP_OK;
  const Geo g = make_geo(prm->d, prm->k);
  int M = 0, ae = 0;
  count_messages(g, 1, &M, &ae);
  const int m = 2 * g.d * (g.d - 1);
  const int smem = align_up(m, 16) + align_up(g.W * g.W, 16) + align_up(2 * M, 16);
  features_kernel<<<(unsigned)(B * 4), 256, smem, static_cast<cudaStream_t>(stream)>>>(g, M, prm->p, syndromes,
                                                                                      feats, lens);
  return cudaGetLastError() == cudaSuccess ? BBP_OK : BBP_ECUDA;
}

int bbp_message_classes(const bbp_params* prm, int32_t* uniq_of, int32_t* row_key, int32_t* n_rows) {
  if (!prm || !uniq_of || !row_key || !n_rows || prm->d < 2 || prm->d > 64 || prm->k < 1 || prm->k > kFusedK)
    return BBP_EINVAL;
  const Geo g = make_geo(prm->d, prm->k);
  int M = 0, ae = 0;
  count_messages(g, 1, &M, &ae);
  int idx = 0, u = 0;
  for (int I = 0; I < g.nb; ++I)
    for (int J = 0; J < g.nb; ++J)
      for (int dir = 0; dir < 4; ++dir) {
        if (!g.has(I, J, dir)) continue;
        // Coset c = (bx, bz) is represented by (bx if the window sees X-bar,
        // bz if it sees Z-bar); representatives in coset order I, X, Y, Z.
        const int seen = window_logicals(g, msg_geo(g, I, J, dir));
        int row_of_rep[4] = {-1, -1, -1, -1};
        for (int c = 0; c < 4; ++c) {
          const int bx = (c == 1 || c == 2) && (seen & 1), bz = (c == 2 || c == 3) && (seen & 2);
          const int rep = bx ? (bz ? 2 : 1) : (bz ? 3 : 0);
          if (row_of_rep[rep] < 0) {
            row_of_rep[rep] = u;
            row_key[u++] = rep * M + idx;
          }
          uniq_of[c * M + idx] = row_of_rep[rep];
        }
        ++idx;
      }
  *n_rows = u;
  return BBP_OK;
}

}  // extern "C"

namespace bbp {
namespace warm {

// Either output of features_rows_kernel (exactly one of feats, bits).
int features_rows(const uint8_t* syndromes, int64_t B, const bbp_params* prm, const int32_t* row_key, int32_t U,
                  float* feats, uint32_t* bits, int32_t* lens, cudaStream_t st) {
  if (!prm || !syndromes || !row_key || (!feats == !bits) || B < 0 || prm->d < 2 || prm->d > 64 || prm->k < 1 ||
      prm->k > kFusedK || U < 0)
    return BBP_EINVAL;
  if (B == 0 || U == 0) return BBP_OK;
  const Geo g = make_geo(prm->d, prm->k);
  int M = 0, ae = 0;
  count_messages(g, 1, &M, &ae);
  if (U > 4 * M) return BBP_EINVAL;
  const int m = 2 * g.d * (g.d - 1);
  const int smem = align_up(m, 16) + align_up(4 * g.W * g.W, 16) + align_up(2 * M, 16);
  auto kern = bits ? features_rows_kernel<true> : features_rows_kernel<false>;
  if (smem > 48 * 1024 && cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) != cudaSuccess)
    return BBP_ECUDA;
  kern<<<(unsigned)B, 256, smem, st>>>(g, M, prm->p, syndromes, row_key, U, feats, bits, lens);
  return cudaGetLastError() == cudaSuccess ? BBP_OK : BBP_ECUDA;
}

}  // namespace warm
}  // namespace bbp

extern "C" {

int bbp_message_features_rows(const uint8_t* syndromes, int64_t B, const bbp_params* prm, const int32_t* row_key,
                              int32_t U, float* feats, int32_t* lens, void* stream) {
  if (!feats) return BBP_EINVAL;
  return bbp::warm::features_rows(syndromes, B, prm, row_key, U, feats, nullptr, lens,
                                  static_cast<cudaStream_t>(stream));
}

int bbp_message_feature_bits_rows(const uint8_t* syndromes, int64_t B, const bbp_params* prm,
                                  const int32_t* row_key, int32_t U, uint32_t* bits, int32_t* lens, void* stream) {
  if (!bits) return BBP_EINVAL;
  return bbp::warm::features_rows(syndromes, B, prm, row_key, U, nullptr, bits, lens,
                                  static_cast<cudaStream_t>(stream));
}

int bbp_expand_rows(const float* rows, int64_t B, int32_t U, const int32_t* uniq_of, int32_t M, float* msgs,
                    void* stream) {
  if (!rows || !uniq_of || !msgs || B < 0 || U < 1 || M < 1) return BBP_EINVAL;
  if (B == 0) return BBP_OK;
  const long long total = B * 4 * (long long)M * 4;
  long long blocks = (total + 255) / 256;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return BBP_ECUDA;
  if (blocks > (long long)sms * 32) blocks = (long long)sms * 32;   // grid-stride beyond 32 blocks per SM
  expand_rows_kernel<<<(unsigned)blocks, 256, 0, static_cast<cudaStream_t>(stream)>>>(
      reinterpret_cast<const float4*>(rows), B, U, uniq_of, M, reinterpret_cast<float4*>(msgs));
  return cudaGetLastError() == cudaSuccess ? BBP_OK : BBP_ECUDA;
}

int bbp_warm_workspace_bytes(int64_t N, size_t* bytes) {
  if (!bytes || N < 0) return BBP_EINVAL;
  *bytes = pass_bytes(N);
  return BBP_OK;
}

int bbp_warm_infer(const float* theta, const float* feats, const int32_t* lens, int64_t N, float alpha,
                   float* msgs, void* workspace, size_t workspace_bytes, void* stream) {
  if (!theta || !feats || !lens || !msgs || N < 0 || N > BBP_WARM_MAX_ROWS) return BBP_EINVAL;
  if (!(alpha >= 0.f && alpha <= 1.f)) return BBP_EINVAL;
  if (N == 0) return BBP_OK;
  if (!workspace || workspace_bytes < infer_tc_workspace_bytes()) return BBP_ENOSPACE;
  if (reinterpret_cast<uintptr_t>(workspace) % 256 != 0) return BBP_EINVAL;
  return infer_tc(theta, feats, lens, N, alpha, msgs, workspace, static_cast<cudaStream_t>(stream)) == cudaSuccess
             ? BBP_OK
             : BBP_ECUDA;
}

int bbp_warm_infer_bits(const float* theta, const uint32_t* bits, const int32_t* lens, int64_t N, double p,
                        float alpha, float* msgs, void* workspace, size_t workspace_bytes, void* stream) {
  if (!theta || !bits || !lens || !msgs || N < 0 || N > BBP_WARM_MAX_ROWS) return BBP_EINVAL;
  if (!(alpha >= 0.f && alpha <= 1.f) || !(p > 0.0 && p < 0.75)) return BBP_EINVAL;
  if (N == 0) return BBP_OK;
  if (!workspace || workspace_bytes < infer_tc_workspace_bytes()) return BBP_ENOSPACE;
  if (reinterpret_cast<uintptr_t>(workspace) % 256 != 0) return BBP_EINVAL;
  return infer_tc_bits(theta, bits, lens, N, p, alpha, msgs, workspace, static_cast<cudaStream_t>(stream)) ==
                 cudaSuccess
             ? BBP_OK
             : BBP_ECUDA;
}

int bbp_warm_infer_syndromes(const float* theta, const uint8_t* syndromes, int64_t B, const bbp_params* prm,
                             float alpha, float* msgs, void* workspace, size_t workspace_bytes, void* stream) {
  if (!theta || !syndromes || !msgs || !prm || B < 0 || prm->d < 2 || prm->d > 64 || prm->k < 1 ||
      prm->k > kFusedK || !(prm->p > 0.0 && prm->p < 0.75))
    return BBP_EINVAL;
  if (!(alpha >= 0.f && alpha <= 1.f)) return BBP_EINVAL;
  if (B == 0) return BBP_OK;
  if (!workspace || workspace_bytes < infer_tc_workspace_bytes()) return BBP_ENOSPACE;
  if (reinterpret_cast<uintptr_t>(workspace) % 256 != 0) return BBP_EINVAL;
  const Geo g = make_geo(prm->d, prm->k);
  int M = 0, ae = 0;
  count_messages(g, 1, &M, &ae);
  if (M == 0) return BBP_OK;
  if (infer_tc_syndromes_smem(g, M) > kMaxSmemBytes) return BBP_EUNSUPPORTED;
  return infer_tc_syndromes(theta, syndromes, B, g, M, prm->p, alpha, msgs, workspace,
                            static_cast<cudaStream_t>(stream)) == cudaSuccess
             ? BBP_OK
             : BBP_ECUDA;
}

int bbp_warm_train_step(float* theta, float* adam_m, float* adam_v, int32_t step, float lr, const float* feats,
                        const float* targets, const int32_t* lens, int64_t N, float* grad, float* loss_sum,
                        void* workspace, size_t workspace_bytes, void* stream) {
  if (!theta || !feats || !targets || !lens || !grad || !loss_sum || N <= 0 || N > BBP_WARM_MAX_ROWS)
    return BBP_EINVAL;
  if (!workspace || workspace_bytes < pass_bytes(N)) return BBP_ENOSPACE;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const Params P = split(theta);
  float* gW1 = grad;
  float* gb1 = gW1 + F * H;
  float* gW2 = gb1 + H;
  float* gb2 = gW2 + H * H;
  float* gW3 = gb2 + H;
  float* gb3 = gW3 + H * O;
  char* w = static_cast<char*>(workspace);
  const size_t nh = al256((size_t)N * H * 4), no = al256((size_t)N * O * 4);
  float* Z1 = reinterpret_cast<float*>(w);
  float* A1 = reinterpret_cast<float*>(w + nh);
  float* Z2 = reinterpret_cast<float*>(w + 2 * nh);
  float* A2 = reinterpret_cast<float*>(w + 3 * nh);
  float* G1 = reinterpret_cast<float*>(w + 4 * nh);
  float* G2 = reinterpret_cast<float*>(w + 5 * nh);
  float* L = reinterpret_cast<float*>(w + 6 * nh);
  float* gO = reinterpret_cast<float*>(w + 6 * nh + no);
  const int n = (int)N;
  bool ok = true;
  ok = ok && gemm<false, false>(n, H, F, feats, F, P.W1, H, A1, H, P.b1, Z1, 1, 0, st) == cudaSuccess;
  ok = ok && gemm<false, false>(n, H, H, A1, H, P.W2, H, A2, H, P.b2, Z2, 1, 0, st) == cudaSuccess;
  ok = ok && gemm<false, false>(n, O, H, A2, H, P.W3, O, L, O, P.b3, nullptr, 0, 0, st) == cudaSuccess;
  if (!ok) return BBP_ECUDA;
  if (cudaMemsetAsync(loss_sum, 0, sizeof(float), st) != cudaSuccess) return BBP_ECUDA;
  head_kernel<<<(unsigned)((N + 127) / 128), 128, 0, st>>>(L, lens, targets, N, gO, loss_sum);
  // Layer 3: gW3 = A2^T gO, gb3 = colsum gO, gA2 = gO W3^T.
  ok = ok && gemm<true, false>(H, O, n, A2, H, gO, O, gW3, O, nullptr, nullptr, 0, 0, st) == cudaSuccess;
  colsum_kernel<<<O, 256, 0, st>>>(gO, N, O, gb3);
  ok = ok && gemm<false, true>(n, H, O, gO, O, P.W3, O, G2, H, nullptr, nullptr, 0, 0, st) == cudaSuccess;
  gelu_back_kernel<<<(unsigned)(((long long)N * H + 255) / 256), 256, 0, st>>>(G2, Z2, (long long)N * H);
  // Layer 2.
  ok = ok && gemm<true, false>(H, H, n, A1, H, G2, H, gW2, H, nullptr, nullptr, 0, 0, st) == cudaSuccess;
  colsum_kernel<<<H, 256, 0, st>>>(G2, N, H, gb2);
  ok = ok && gemm<false, true>(n, H, H, G2, H, P.W2, H, G1, H, nullptr, nullptr, 0, 0, st) == cudaSuccess;
  gelu_back_kernel<<<(unsigned)(((long long)N * H + 255) / 256), 256, 0, st>>>(G1, Z1, (long long)N * H);
  // Layer 1.
  ok = ok && gemm<true, false>(F, H, n, feats, F, G1, H, gW1, H, nullptr, nullptr, 0, 0, st) == cudaSuccess;
  colsum_kernel<<<H, 256, 0, st>>>(G1, N, H, gb1);
  if (!ok || cudaGetLastError() != cudaSuccess) return BBP_ECUDA;
  if (step > 0 && adam_m && adam_v) {
    const float b1 = 0.9f, b2 = 0.999f;
    const float c1 = 1.f - powf(b1, (float)step), c2 = 1.f - powf(b2, (float)step);
    adam_kernel<<<(unsigned)((kParams + 255) / 256), 256, 0, st>>>(theta, grad, adam_m, adam_v, kParams, lr, b1,
                                                                  b2, 1e-8f, c1, c2);
  }
  return cudaGetLastError() == cudaSuccess ? BBP_OK : BBP_ECUDA;
}

}  // extern "C"
