// Inference of the warm-start network on the 5th-generation tensor cores.
//
// The network maps each directed block edge's 256 features to a proposal
// for its initial message (the paper starts from uniform messages, Remark 2,
// and names learned techniques as a way to improve BP, Sec. V).  Its two
// 256 x 256 layers are the one dense contraction of the decoder, so they run
// as tcgen05 MMAs: BF16 operands in shared memory, FP32 accumulators in
// tensor memory (TMEM), one thread issuing the MMAs, completion signalled
// on an mbarrier.  One persistent CTA per SM takes tiles of 128 rows and
// runs all three layers back to back: X (features, rounded to BF16) and
// the layer's weights are staged in shared memory in the K-major,
// no-swizzle core-matrix layout; each layer's accumulators are read back
// with tcgen05.ld, biased and passed through GELU, rounded to BF16 and
// written over the operand tile as the next layer's input; the output
// layer's 16 logits per row go through the message head.
//
// Each layer's weights are moved by the bulk-copy engine (cp.async.bulk,
// completion on a second mbarrier), issued by one thread so that they
// stream in while the threads stage the features or run the previous
// layer's epilogue.
//
// Every mbarrier wait is bounded: a wait that gives up marks the tile's
// messages NaN (the decoder then starts those messages uniform), sets the
// status word and the CTA frees its TMEM and returns.
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "../../include/blockbp.h"
#include "bbp_warm_features.cuh"
#include "bbp_warm_tc.h"

namespace bbp {
namespace warm {
namespace {

constexpr int TM = 128;                       // rows per tile (MMA M)
constexpr int KD = 256;                       // K of every layer (features = hidden = 256)
constexpr int NH = BBP_WARM_HIDDEN;           // 256
constexpr int NO = BBP_WARM_OUT;              // 16
constexpr int kCore = 128;                    // one core matrix: 8 rows x 16 bytes
constexpr int kTileA = TM * KD * 2;           // 64 KB: BF16 operand tile
constexpr int kTileB = NH * KD * 2;           // 128 KB: one hidden layer's BF16 weights
constexpr int kTileB3 = NO * KD * 2;          // 8 KB: the output layer's weights
constexpr int kThreads = 512;                 // 16 warps: four per TMEM lane quarter
constexpr int kParts = kThreads / 128;        // column parts of a lane quarter in the epilogues
constexpr uint32_t kLBO = kCore;              // K-adjacent core matrices
constexpr uint32_t kSBO = (KD / 8) * kCore;   // 8-row groups
constexpr uint32_t kTmemCols = 512;
constexpr long long kWaitTries = 1ll << 22;

static_assert(BBP_WARM_FEATURES == KD && BBP_WARM_HIDDEN == KD, "layers of width 256");

// Byte offset of element (row, k) of a K-major BF16 operand in the
// no-swizzle layout: 8 x 8 core matrices of 128 contiguous bytes (row r of
// a core matrix at 16 r), K-adjacent core matrices kLBO apart, 8-row groups
// kSBO apart.
__host__ __device__ constexpr int core_off(int row, int k) {
  return ((row >> 3) * (KD / 8) + (k >> 3)) * kCore + (row & 7) * 16 + (k & 7) * 2;
}

__device__ __forceinline__ uint32_t su32(const void* p) { return static_cast<uint32_t>(__cvta_generic_to_shared(p)); }

// Shared-memory matrix descriptor of tcgen05: start address, leading and
// stride byte offsets (all >> 4), descriptor version 1, no swizzle.
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr) {
  return (uint64_t)((saddr >> 4) & 0x3FFFu) | ((uint64_t)((kLBO >> 4) & 0x3FFFu) << 16) |
         ((uint64_t)((kSBO >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}

// Instruction descriptor of kind::f16: FP32 accumulator, BF16 A and B, both
// K-major, N >> 3 at bit 17, M >> 4 at bit 24.
__host__ __device__ constexpr uint32_t instr_desc(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mbar_init(uint64_t* b, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(su32(b)), "r"(count) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* b, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(su32(b)), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ bool mbar_wait(uint64_t* b, uint32_t parity) {
  for (long long i = 0; i < kWaitTries; ++i)
    if (mbar_try_wait(b, parity)) return true;
  return false;
}
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void tc_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tmem_alloc(uint32_t* slot, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(slot)), "r"(ncols)
               : "memory");
}
__device__ __forceinline__ void tmem_relinquish() {
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}
__device__ __forceinline__ void mma_bf16(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\ttcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d),
      "l"(a), "l"(b), "r"(idesc), "r"(acc)
      : "memory");
}
__device__ __forceinline__ void mma_commit(uint64_t* b) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(su32(b)) : "memory");
}
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&v)[32]) {
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
               : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15]), "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]), "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
               : "r"(taddr));
}
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&v)[16]) {
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, [%16];"
               : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
               : "r"(taddr));
}
__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// GELU(x) = x Phi(x) = 0.5 x (1 + erf(x / sqrt 2)), with erf by the
// rational approximation of Abramowitz & Stegun, Handbook of Mathematical
// Functions, formula 7.1.26: 1 - erf(z) = poly(t) exp(-z^2), t = 1 / (1 +
// p z), |error| <= 1.5e-7 for z >= 0 (odd in z).  With z = |x| / sqrt 2
// and h = 0.5 |x| poly(t) exp(-x^2 / 2): GELU(x) = max(x, 0) - h for either
// sign of x.  The hardware reciprocal and exponential keep it below 1e-6 in
// FP32, far below the BF16 rounding of the activations the epilogue
// writes, in fewer instructions than the library erf; the two hidden
// epilogues are most of the kernel's instructions.
__device__ __forceinline__ float gelu_f(float x) {
  const float ax = fabsf(x);
  const float t = __fdividef(1.f, fmaf(0.3275911f * 0.70710678118654752f, ax, 1.f));
  const float poly =
      t * fmaf(t, fmaf(t, fmaf(t, fmaf(t, 1.061405429f, -1.453152027f), 1.421413741f), -0.284496736f), 0.254829592f);
  const float h = 0.5f * ax * poly * __expf(-0.5f * x * x);
  return fmaxf(x, 0.f) - h;
}

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
  const __nv_bfloat162 h = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<const uint32_t*>(&h);
}

// theta (FP32: W1 [F x H], b1, W2 [H x H], b2, W3 [H x O], b3, row-major
// [k][n]) -> the B operands of the three layers, B[n][k] = W[k][n] in BF16,
// in the core-matrix layout.
__global__ void prep_weights_kernel(const float* __restrict__ theta, unsigned char* __restrict__ wt) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  const int n12 = NH * KD;
  int layer, n, k;
  if (e < 2 * n12) {
    layer = e / n12;
    const int r = e - layer * n12;
    k = r / NH;
    n = r - k * NH;
  } else if (e < 2 * n12 + NO * KD) {
    layer = 2;
    const int r = e - 2 * n12;
    k = r / NO;
    n = r - k * NO;
  } else {
    return;
  }
  const int w_off = layer == 0 ? 0 : (layer == 1 ? KD * NH + NH : 2 * (KD * NH + NH));
  const int ncols = layer == 2 ? NO : NH;
  const float w = theta[w_off + k * ncols + n];
  __nv_bfloat16* dst = reinterpret_cast<__nv_bfloat16*>(wt + layer * kTileB + core_off(n, k));
  *dst = __float2bfloat16_rn(w);
}

// One thread: a layer's weights (bytes, a multiple of 16) from global into
// shared memory with the bulk-copy engine in chunks; the mbarrier's phase
// completes when all bytes have landed.
constexpr int kBulkChunk = 16384;
__device__ __forceinline__ void load_weights(unsigned char* dst, const unsigned char* src, int bytes, uint64_t* bar) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(su32(bar)), "r"(bytes) : "memory");
  for (int off = 0; off < bytes; off += kBulkChunk) {
    const int n = bytes - off < kBulkChunk ? bytes - off : kBulkChunk;
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     su32(dst + off)),
                 "l"(src + off), "r"(n), "r"(su32(bar))
                 : "memory");
  }
}

// Accumulators of a hidden layer (TMEM columns [0, 256)) -> + bias, GELU,
// BF16 -> the operand tile.  Warp w reads TMEM lanes 32 (w % 4) .. (its
// rows; a warp reaches only its own lane quarter) and columns
// (256 / kParts) (w / 4) .. + 256 / kParts - 1.
__device__ __forceinline__ void hidden_epilogue(uint32_t tmem, unsigned char* sA, const float* bias, int warp,
                                                int lane) {
  constexpr int kCols = NH / kParts;
  const int q = warp & 3, part = warp >> 2;
  const int row = 32 * q + lane;
#pragma unroll 1
  for (int ch = 0; ch < kCols / 32; ++ch) {
    const int col0 = kCols * part + 32 * ch;
    uint32_t v[32];
    tmem_ld32(tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)col0, v);
    tmem_wait_ld();
#pragma unroll
    for (int j = 0; j < 32; j += 8) {
      uint4 pk;
      pk.x = pack_bf16(gelu_f(__uint_as_float(v[j + 0]) + bias[col0 + j + 0]),
                       gelu_f(__uint_as_float(v[j + 1]) + bias[col0 + j + 1]));
      pk.y = pack_bf16(gelu_f(__uint_as_float(v[j + 2]) + bias[col0 + j + 2]),
                       gelu_f(__uint_as_float(v[j + 3]) + bias[col0 + j + 3]));
      pk.z = pack_bf16(gelu_f(__uint_as_float(v[j + 4]) + bias[col0 + j + 4]),
                       gelu_f(__uint_as_float(v[j + 5]) + bias[col0 + j + 5]));
      pk.w = pack_bf16(gelu_f(__uint_as_float(v[j + 6]) + bias[col0 + j + 6]),
                       gelu_f(__uint_as_float(v[j + 7]) + bias[col0 + j + 7]));
      *reinterpret_cast<uint4*>(sA + core_off(row, col0 + j)) = pk;
    }
  }
}

// The 16 MMAs (K = 256 in steps of 16) of one layer, issued by one thread,
// then a commit that arrives on the mbarrier when they have completed.
__device__ __forceinline__ void issue_layer(uint32_t d_tmem, const unsigned char* sA, const unsigned char* sB,
                                            uint32_t idesc, uint64_t* mbar) {
  const uint32_t a0 = su32(sA), b0 = su32(sB);
#pragma unroll 1
  for (int kb = 0; kb < KD / 16; ++kb)
    mma_bf16(d_tmem, smem_desc(a0 + kb * 2 * kCore), smem_desc(b0 + kb * 2 * kCore), idesc, kb > 0 ? 1u : 0u);
  mma_commit(mbar);
}

// Where a tile's features come from.
constexpr int kFromFeats = 0, kFromSyndromes = 1, kFromBits = 2;

struct MlpArgs {
  const float* feats;        // feature rows [N][256] (from a features tensor), or
  const uint32_t* bits;      //   as bits [N][8] (feature 253 stands for p10), with
  const int32_t* lens;       //   their message lengths;
  const uint8_t* synd;       // syndromes [N / (4 M)][m]: features computed here
  Geo g;
  int M, max_pairs;
  float p10;
  long long N;
  const unsigned char* wt;
  const float *b1, *b2, *b3;
  float alpha;
  float* msgs;
  int32_t* status;
};

// One row of a tile in the syndrome-fed kernel: its (syndrome, coset) pair
// within the tile and its message's geometry.
struct RowGeo {
  int16_t r0, r1, c0, c1;
  int8_t pair, dir, h, ncols;
};

// Shared memory of the syndrome-fed kernel beyond the operand tiles: the
// message table, the tile's row table, then per (syndrome, coset) pair of a
// tile its syndrome and its frame.
__host__ __device__ inline int synd_extra_bytes(const Geo& g, int M, int max_pairs) {
  const int m = 2 * g.d * (g.d - 1);
  return align_up(2 * M, 16) + align_up(TM * (int)sizeof(RowGeo), 16) +
         max_pairs * (align_up(m, 16) + align_up(g.W * g.W, 16));
}

template <int kSrc>
__global__ void __launch_bounds__(kThreads, 1) mlp_tc_kernel(MlpArgs a) {
  constexpr bool kSynd = kSrc == kFromSyndromes;
  extern __shared__ __align__(1024) unsigned char smem[];
  unsigned char* sA = smem;                 // operand tile / hidden activations
  unsigned char* sB = smem + kTileA;        // weights of the current layer
  __shared__ __align__(8) uint64_t mbar;    // MMA completion
  __shared__ __align__(8) uint64_t wbar;    // weights landed in sB
  __shared__ uint32_t tmem_slot;
  __shared__ float sb1[NH], sb2[NH], sb3[NO];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const long long N = a.N;
  const float alpha = a.alpha;
  const unsigned char* wt = a.wt;
  for (int i = tid; i < NH; i += kThreads) { sb1[i] = a.b1[i]; sb2[i] = a.b2[i]; }
  if (tid < NO) sb3[tid] = a.b3[tid];
  // Syndrome-fed: the message table (index -> (I, J, dir)) once per CTA.
  const Geo g = a.g;
  const int M = a.M, m = 2 * g.d * (g.d - 1), WW = g.W * g.W;
  int16_t* meta = reinterpret_cast<int16_t*>(smem + kTileA + kTileB);
  RowGeo* rows = reinterpret_cast<RowGeo*>(smem + kTileA + kTileB + align_up(2 * M, 16));
  uint8_t* pair_base = reinterpret_cast<uint8_t*>(rows) + align_up(TM * (int)sizeof(RowGeo), 16);
  const int pair_stride = align_up(m, 16) + align_up(WW, 16);
  if (kSynd && tid == 0) {
    int idx = 0;
    for (int I = 0; I < g.nb; ++I)
      for (int J = 0; J < g.nb; ++J)
        for (int dir = 0; dir < 4; ++dir)
          if (g.has(I, J, dir)) meta[idx++] = (int16_t)((I * g.nb + J) * 4 + dir);
  }
  if (tid == 0) {
    mbar_init(&mbar, 1);
    mbar_init(&wbar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    tmem_alloc(&tmem_slot, kTmemCols);
    tmem_relinquish();
  }
  tc_before();
  __syncthreads();
  tc_after();
  const uint32_t tmem = tmem_slot;
  uint32_t phase = 0, wphase = 0;
  int ok = 1;
  const long long ntiles = (N + TM - 1) / TM;
  for (long long tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const long long r0 = tile * TM;
    // The first layer's weights stream in while the threads build X.
    if (tid == 0) load_weights(sB, wt, kTileB, &wbar);
    if (kSynd) {
      // Syndromes and frames of the (syndrome, coset) pairs the tile touches.
      const long long p0 = r0 / M;
      const long long plast = ((r0 + TM < N ? r0 + TM : N) - 1) / M;
      const int np = (int)(plast - p0 + 1);
      for (int e = tid; e < np * m; e += kThreads) {
        const int pi = e / m, i = e - pi * m;
        pair_base[pi * pair_stride + i] = a.synd[((p0 + pi) >> 2) * m + i];
      }
      __syncthreads();
      for (int e = tid; e < np * WW; e += kThreads) {
        const int pi = e / WW, ij = e - pi * WW;
        uint8_t* pb = pair_base + pi * pair_stride;
        pb[align_up(m, 16) + ij] = frame_byte(pb, g.d, ij / g.W, ij % g.W, (int)((p0 + pi) & 3));
      }
      // Row table: pair and message geometry of each row, once per tile.
      if (tid < TM && r0 + tid < N) {
        const int local = (int)(r0 + tid - p0 * M);
        const int pi = local / M;
        const int key = meta[local - pi * M];
        const MsgGeo f = msg_geo(g, key / 4 / g.nb, (key / 4) % g.nb, key & 3);
        RowGeo rg;
        rg.r0 = (int16_t)f.r0; rg.r1 = (int16_t)f.r1; rg.c0 = (int16_t)f.c0; rg.c1 = (int16_t)f.c1;
        rg.pair = (int8_t)pi; rg.dir = (int8_t)f.dir; rg.h = (int8_t)f.h; rg.ncols = (int8_t)f.ncols;
        rows[tid] = rg;
      }
      __syncthreads();
      // X: the features of rows r0 .. r0 + 127 (bbp_warm_features.cuh), in
      // BF16: one window node of one row per task (its five channels), then
      // the eleven tail features of each row.
      __nv_bfloat16* xa = reinterpret_cast<__nv_bfloat16*>(sA);
      for (int task = tid; task < TM * 49; task += kThreads) {
        const int row = task & (TM - 1), pos = task >> 7;
        float c[5] = {0.f, 0.f, 0.f, 0.f, 0.f};
        if (r0 + row < N) {
          const RowGeo rg = rows[row];
          MsgGeo f;
          f.r0 = rg.r0; f.r1 = rg.r1; f.c0 = rg.c0; f.c1 = rg.c1;
          f.dir = rg.dir; f.h = rg.h; f.ncols = rg.ncols;
          const uint8_t* pb = pair_base + rg.pair * pair_stride;
          window_node(g, f, pos, pb + align_up(m, 16), pb, c);
        }
#pragma unroll
        for (int ch = 0; ch < 5; ++ch) xa[core_off(row, ch * 49 + pos) / 2] = __float2bfloat16_rn(c[ch]);
      }
      for (int task = tid; task < TM * (KD - 245); task += kThreads) {
        const int row = task & (TM - 1), q = 245 + (task >> 7);
        float v = 0.f;
        if (r0 + row < N) {
          const RowGeo rg = rows[row];
          MsgGeo f;
          f.dir = rg.dir; f.h = rg.h;
          v = tail_feature(f, q, a.p10);
        }
        xa[core_off(row, q) / 2] = __float2bfloat16_rn(v);
      }
    } else if (kSrc == kFromBits) {
      // X from feature bits: 1 where a bit is set (feature 253: 10 p, the one
      // feature that is not 0 or 1), rounded to BF16 exactly as the FP32
      // path rounds the same features (one 32-feature word of one row per
      // task; consecutive threads, consecutive rows).
      const uint16_t one = 0x3F80u;
      const __nv_bfloat16 pb = __float2bfloat16_rn(a.p10);
      const uint16_t p10b = *reinterpret_cast<const uint16_t*>(&pb);
#pragma unroll 2
      for (int task = tid; task < TM * 8; task += kThreads) {
        const int row = task & (TM - 1), wd = task >> 7;
        const long long gr = r0 + row;
        const uint32_t b = gr < N ? a.bits[gr * 8 + wd] : 0u;
#pragma unroll
        for (int c8 = 0; c8 < 4; ++c8) {
          uint32_t h[8];
#pragma unroll
          for (int j = 0; j < 8; ++j) {
            const int q = 32 * wd + 8 * c8 + j;
            h[j] = (b >> (8 * c8 + j)) & 1u ? (q == 253 ? p10b : one) : 0u;
          }
          *reinterpret_cast<uint4*>(sA + core_off(row, 32 * wd + 8 * c8)) =
              make_uint4(h[0] | (h[1] << 16), h[2] | (h[3] << 16), h[4] | (h[5] << 16), h[6] | (h[7] << 16));
        }
      }
    } else {
      // X: rows r0 .. r0 + 127 of the FP32 features, rounded to BF16 (one
      // 8-element chunk of one row per task; consecutive threads, consecutive rows).
#pragma unroll 8
      for (int task = tid; task < TM * (KD / 8); task += kThreads) {
        const int row = task & (TM - 1), ch = task >> 7;
        const long long gr = r0 + row;
        uint4 pk = make_uint4(0u, 0u, 0u, 0u);
        if (gr < N) {
          const float4* src = reinterpret_cast<const float4*>(a.feats + gr * KD + ch * 8);
          const float4 x0 = src[0], x1 = src[1];
          pk.x = pack_bf16(x0.x, x0.y); pk.y = pack_bf16(x0.z, x0.w);
          pk.z = pack_bf16(x1.x, x1.y); pk.w = pack_bf16(x1.z, x1.w);
        }
        *reinterpret_cast<uint4*>(sA + core_off(row, ch * 8)) = pk;
      }
    }
    // Three layers: operands written by the threads become visible to the
    // tensor cores (proxy fence, barrier), the weights have landed (the
    // issuing thread waits on their mbarrier), one thread issues, all wait.
#pragma unroll 1
    for (int layer = 0; layer < 3 && ok; ++layer) {
      int wdone = 1;
      if (tid == 0) wdone = mbar_wait(&wbar, wphase) ? 1 : 0;
      wphase ^= 1u;
      fence_proxy_async();
      tc_before();
      ok = __syncthreads_and(wdone);
      if (!ok) break;
      tc_after();
      if (tid == 0)
        issue_layer(layer < 2 ? tmem : tmem + NH, sA, sB, layer < 2 ? instr_desc(TM, NH) : instr_desc(TM, NO), &mbar);
      const int done = mbar_wait(&mbar, phase) ? 1 : 0;
      phase ^= 1u;
      ok = __syncthreads_and(done);
      if (!ok) break;
      tc_after();
      if (layer < 2) {
        // The MMAs have read sA and sB: the next layer's weights stream into
        // sB while the threads overwrite sA with the activations.
        if (tid == 0) load_weights(sB, wt + (layer + 1) * kTileB, layer == 0 ? kTileB : kTileB3, &wbar);
        hidden_epilogue(tmem, sA, layer == 0 ? sb1 : sb2, warp, lane);
      }
    }
    if (!ok) {
      // Give up on this tile: NaN proposals make the decoder start uniform.
      for (int e = tid; e < TM * NO; e += kThreads) {
        const long long gr = r0 + e / NO;
        if (gr < N) a.msgs[gr * NO + (e % NO)] = __int_as_float(0x7fc00000);
      }
      if (tid == 0) atomicExch(a.status, 1);
      break;
    }
    // Output layer: TMEM columns [256, 272) hold the logits of row 32 q + lane.
    if (warp < 4) {
      uint32_t v[16];
      tmem_ld16(tmem + ((uint32_t)(32 * warp) << 16) + (uint32_t)NH, v);
      tmem_wait_ld();
      const long long gr = r0 + 32 * warp + lane;
      if (gr < N) {
        int n;
        if (kSynd) {
          n = 1 << rows[32 * warp + lane].h;
        } else {
          n = a.lens[gr];
        }
        float o[NO], mm[NO];
        float mx = -INFINITY;
#pragma unroll
        for (int i = 0; i < NO; ++i) {
          o[i] = __uint_as_float(v[i]) + sb3[i];
          if (i < n) mx = fmaxf(mx, o[i]);
        }
        float s2 = 0.f;
#pragma unroll
        for (int i = 0; i < NO; ++i) {
          mm[i] = i < n ? expf(o[i] - mx) : 0.f;
          s2 += mm[i] * mm[i];
        }
        const float inv = 1.f / sqrtf(s2), un = rsqrtf((float)n);
        // Proposal blended with the uniform start: (1 - alpha) uniform + alpha u.
        float b[NO], s2b = 0.f;
#pragma unroll
        for (int i = 0; i < NO; ++i) {
          b[i] = i < n ? (1.f - alpha) * un + alpha * mm[i] * inv : 0.f;
          s2b += b[i] * b[i];
        }
        const float ib = rsqrtf(s2b);
        float4* dst = reinterpret_cast<float4*>(a.msgs + gr * NO);
#pragma unroll
        for (int i = 0; i < NO; i += 4) dst[i / 4] = make_float4(b[i] * ib, b[i + 1] * ib, b[i + 2] * ib, b[i + 3] * ib);
      }
    }
    // The next tile overwrites sA, sB and TMEM only after every read here.
    tc_before();
    __syncthreads();
    tc_after();
  }
  if (!ok) {
    // A wait gave up: let the MMAs and copies in flight finish (bounded)
    // before TMEM and shared memory go.
    mbar_wait(&mbar, phase ^ 1u);
    if (tid == 0) mbar_wait(&wbar, wphase ^ 1u);
  }
  tc_before();
  __syncthreads();
  tc_after();
  if (warp == 0) tmem_dealloc(tmem, kTmemCols);
}

}  // namespace

size_t infer_tc_workspace_bytes() { return (size_t)kStatusOffset + 256; }

namespace {

// Weights into the workspace, status cleared, then the persistent kernel.
template <int kSrc>
cudaError_t launch_mlp(const float* theta, MlpArgs a, int extra_smem, void* workspace, cudaStream_t st) {
  unsigned char* wt = static_cast<unsigned char*>(workspace);
  a.wt = wt;
  a.status = reinterpret_cast<int32_t*>(wt + kStatusOffset);
  a.b1 = theta + KD * NH;
  a.b2 = a.b1 + NH + NH * NH;
  a.b3 = a.b2 + NH + NH * NO;
  const int nw = 2 * NH * KD + NO * KD;
  prep_weights_kernel<<<(nw + 255) / 256, 256, 0, st>>>(theta, wt);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  if ((e = cudaMemsetAsync(a.status, 0, sizeof(int32_t), st)) != cudaSuccess) return e;
  const int smem = kTileA + kTileB + extra_smem;
  if ((e = cudaFuncSetAttribute(mlp_tc_kernel<kSrc>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem)) !=
      cudaSuccess)
    return e;
  int dev = 0, sms = 0;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
  if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
  const long long ntiles = (a.N + TM - 1) / TM;
  const unsigned grid = (unsigned)(ntiles < sms ? ntiles : sms);
  mlp_tc_kernel<kSrc><<<grid, kThreads, smem, st>>>(a);
  return cudaGetLastError();
}

}  // namespace

cudaError_t infer_tc(const float* theta, const float* feats, const int32_t* lens, long long N, float alpha,
                     float* msgs, void* workspace, cudaStream_t st) {
  MlpArgs a{};
  a.feats = feats; a.lens = lens; a.N = N; a.alpha = alpha; a.msgs = msgs;
  return launch_mlp<kFromFeats>(theta, a, 0, workspace, st);
}

cudaError_t infer_tc_bits(const float* theta, const uint32_t* bits, const int32_t* lens, long long N, double p,
                          float alpha, float* msgs, void* workspace, cudaStream_t st) {
  MlpArgs a{};
  a.bits = bits; a.lens = lens; a.N = N; a.alpha = alpha; a.msgs = msgs;
  a.p10 = (float)(10.0 * p);
  return launch_mlp<kFromBits>(theta, a, 0, workspace, st);
}

int infer_tc_syndromes_smem(const Geo& g, int M) {
  const int max_pairs = (TM - 1) / M + 2;
  return kTileA + kTileB + synd_extra_bytes(g, M, max_pairs) + 4096;   // + static shared memory
}

cudaError_t infer_tc_syndromes(const float* theta, const uint8_t* synd, long long B, const Geo& g, int M, double p,
                               float alpha, float* msgs, void* workspace, cudaStream_t st) {
  MlpArgs a{};
  a.synd = synd; a.g = g; a.M = M; a.max_pairs = (TM - 1) / M + 2;
  a.p10 = (float)(10.0 * p);
  a.N = B * 4 * (long long)M; a.alpha = alpha; a.msgs = msgs;
  return launch_mlp<kFromSyndromes>(theta, a, synd_extra_bytes(g, M, a.max_pairs), workspace, st);
}

}  // namespace warm
}  // namespace bbp
