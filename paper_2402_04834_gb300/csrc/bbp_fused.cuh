// Fused-block BP (Remark 9; the form the paper ran for k = 1, 2, 4): every
// k x k block acts as one vertex with four legs of dimension 2^k and the
// messages are dense vectors, so there is no MPS truncation at all.  Where
// the MPS form of Sec. III.D truncates nothing, both compute the same
// numbers.
//
// One CTA decodes one (syndrome, coset); all messages live in shared memory
// (M dense vectors of 2^k).  A warp contracts one block with its incoming
// messages node by node on a dense state indexed by
//     [a | rows of the chain | b | v]   (most to least significant bits)
// where v is the vertical leg inside the current column and a / b carry the
// top / bottom side message.  A side message m(t_0 .. t_{w-1}) is fed one
// leg per column through its exact copy / data / copy factorisation: the
// first floor(w/2) legs are recorded in a, the middle column contracts a
// with m and leaves in a the values expected for the remaining legs, which
// the last columns check off.  All dimensions are powers of two, so every
// index is a bit field.  Every loop is bounded and no CTA waits on another.
#pragma once

#include "bbp_kernels.cuh"

namespace bbp {

constexpr int kFusedK = 4;                 // largest block side of the fused path
constexpr int kFusedVec = 1 << kFusedK;    // dense message length
constexpr int kFusedState = 512;           // 2^(2 + 4 + 2 + 1)

template <typename T>
struct __align__(16) FusedWS {
  T s0[kFusedState];
  T s1[kFusedState];
  T wn[kFusedK * 16];      // node tensors of the current column
  T mt[kFusedVec];         // side message A in consumption order
  T mb[kFusedVec];         // side message B in consumption order
};

// Shared-memory layout of one fused CTA.
struct FusedLayout {
  int synd, frame, msg_of, meta, work, ovl, rlog, misc, msgs, ws, total;
};

template <typename T>
BBP_HD FusedLayout fused_layout(const Geo& g, int M, int nwarps) {
  FusedLayout L;
  const int m = 2 * g.d * (g.d - 1);
  int o = 0;
  L.synd = o;   o = align_up(o + m, 16);
  L.frame = o;  o = align_up(o + g.W * g.W, 16);
  L.msg_of = o; o = align_up(o + 2 * g.nb * g.nb * 4, 16);
  L.meta = o;   o = align_up(o + 2 * M, 16);
  L.work = o;   o = align_up(o + 2 * 2 * M, 16);
  L.ovl = o;    o = align_up(o + 8 * M, 16);
  L.rlog = o;   o = align_up(o + 8 * (g.nb * g.nb + M), 16);
  L.misc = o;   o = align_up(o + 64, 16);
  L.msgs = o;   o = align_up(o + (int)sizeof(T) * kFusedVec * M, 16);
  L.ws = o;     o = align_up(o + nwarps * (int)sizeof(FusedWS<T>), 16);
  L.total = o;
  return L;
}

template <typename T> struct Vec2;
template <> struct Vec2<float> { using type = float2; };
template <> struct Vec2<double> { using type = double2; };

__device__ __forceinline__ int bitrev(int x, int w) {
  return (int)(__brev((unsigned)x) >> (32 - w));
}

struct FState {
  int ab, h, bb, hv;   // bit widths of a, rows, b, v
  __device__ __forceinline__ int size() const { return 1 << (ab + h + bb + hv); }
  __device__ __forceinline__ int idx(int a, int H, int b, int v) const {
    return ((((a << h) | H) << bb | b) << hv) | v;
  }
};

// Contract block f (rotated so that f.dir points right) with its incoming
// dense messages; leaves the outgoing vector over the chain in ws.s0 and
// returns the log of the norms taken out (read-out only; FP64, in lane 0).
template <typename T, int K>
__device__ __forceinline__ double fused_sweep(FusedWS<T>& ws, const Ctx<T, K>& c, const T* msgs, const Frame& f,
                                           bool readout, int lane) {
  const int h = f.h, nc = f.ncols;
  T* cur = ws.s0;
  T* nxt = ws.s1;
  // Initial state: the message on the side opposite the outgoing one.
  for (int H = lane; H < (1 << h); H += 32)
    cur[H] = f.in_idx >= 0 ? msgs[f.in_idx * kFusedVec + H] : (H == 0 ? T(1) : T(0));
  // Side messages in consumption order.
  for (int i = lane; i < (1 << nc); i += 32) {
    const int j = f.rev ? bitrev(i, nc) : i;
    ws.mt[i] = f.a_idx >= 0 ? msgs[f.a_idx * kFusedVec + j] : T(0);
    ws.mb[i] = f.b_idx >= 0 ? msgs[f.b_idx * kFusedVec + j] : T(0);
  }
  __syncwarp();
  FState st{0, h, 0, 0};
  const int sd = nc >> 1;               // the column that holds the data site
  const int nf = nc - sd - 1;           // legs still expected after it
  double log_scale = 0.0;               // accumulated by lane 0 only
  // Which parity the in/out legs carry: a qubit's tensor is pi(f (+) (x, z))
  // with one of x, z the parity of its in/out legs (alpha) and the other the
  // parity of its chain legs (beta); alpha is z for horizontal-edge qubits
  // swept along rows and for vertical-edge qubits swept along columns.
  const bool rowwise = f.dir == kDirR || f.dir == kDirL;
  for (int t = 0; t < nc; ++t) {
    // Side message A: enters the column as its vertical leg v.  Output
    // entries come in pairs (v = 0, 1) sharing (a, rows, b).
    {
      FState ns = st;
      ns.hv = 1;
      if (f.a_idx < 0) ns.ab = 0;
      else if (t < sd) ns.ab = st.ab + 1;
      else if (t == sd) ns.ab = nf;
      else ns.ab = st.ab - 1;
      using V2 = typename Vec2<T>::type;
      const int np = ns.size() >> 1;
      const int hb = h + st.bb;                        // bits of (rows, b)
      const int low = (1 << hb) - 1;
      for (int e2 = lane; e2 < np; e2 += 32) {
        const int a2 = e2 >> hb, hbv = e2 & low;       // (rows, b) part is shared by in and out
        V2 o;
        if (f.a_idx < 0) {
          o.x = cur[e2]; o.y = T(0);
        } else if (t < sd) {
          const T x = cur[((a2 >> 1) << hb) | hbv];
          if (a2 & 1) { o.x = T(0); o.y = x; } else { o.x = x; o.y = T(0); }
        } else if (t == sd) {
          T s0 = T(0), s1 = T(0);
          for (int a = 0; a < (1 << st.ab); ++a) {
            const T x = cur[(a << hb) | hbv];
            s0 += ws.mt[((a << 1) << nf) | a2] * x;
            s1 += ws.mt[(((a << 1) | 1) << nf) | a2] * x;
          }
          o.x = s0; o.y = s1;
        } else {
          o.x = cur[(a2 << hb) | hbv];
          o.y = cur[(((1 << (st.ab - 1)) | a2) << hb) | hbv];
        }
        *reinterpret_cast<V2*>(nxt + 2 * e2) = o;
      }
      __syncwarp();
      T* tmp = cur; cur = nxt; nxt = tmp;
      st = ns;
    }
    // The column's nodes, top to bottom: chain position s is row bit h-1-s.
    // Each lane takes quads of entries that differ only in the node's row bit
    // (l -> r) and in v (u -> d): out[r][d] = sum_{l,u} in[l][u] w[l][r][u][d],
    // read and written as two pairs of adjacent entries.
    for (int s = 0; s < h; ++s) {
      const int P = (h - 1 - s) + st.bb + 1;          // bit of the node's row in the index
      const int bitP = 1 << P;
      const int nq = st.size() >> 2;
      const int lowmask = (1 << (P - 1)) - 1;
      using V2 = typename Vec2<T>::type;
      int ni, nj;
      f.node(t, s, &ni, &nj);
      const bool interior = ni > 0 && nj > 0 && ni < c.g.W - 1 && nj < c.g.W - 1;
      if (interior && s + 1 < h) {
        int mi, mj;
        f.node(t, s + 1, &mi, &mj);
        if (mi > 0 && mj > 0 && mi < c.g.W - 1 && mj < c.g.W - 1) {
          // Two interior chain neighbours, one check and one qubit, in one
          // pass: the check's copy tensor ties the vertical leg between them
          // to the check's own row bit c.
          const bool check_first = (ni + nj) & 1;
          const int qi = check_first ? mi : ni, qj = check_first ? mj : nj;
          const int fr = c.frame[qi * c.g.W + qj];
          const int fx = fr & 1, fz = (fr >> 1) & 1;
          const bool alpha_is_z = ((qi & 1) == 0) == rowwise;
          T gt[4];
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            const int al = q >> 1, be = q & 1;
            const int xb = alpha_is_z ? be : al, zb = alpha_is_z ? al : be;
            gt[q] = ((fx ^ xb) | (fz ^ zb)) ? c.pE : c.pI;
          }
          if (check_first) {
            // out[c, r, d] = sum_l in[c, l, v=c] g[l^r][c^d]; rows bits P (c) and P-1 (qubit).
            const int Q = P - 1, bitQ = 1 << Q, lowq = (1 << (Q - 1)) - 1;
            for (int g = lane; g < nq; g += 32) {
              const int base = ((g >> (Q - 1)) << (Q + 1)) | ((g & lowq) << 1);
              const int cb = (base >> P) & 1;
              const T x0 = cur[base | cb];
              const T x1 = cur[base | bitQ | cb];
              // g[a][c ^ d] by selects (a dynamic index would put gt in local memory)
              const T g00 = cb ? gt[1] : gt[0], g01 = cb ? gt[0] : gt[1];
              const T g10 = cb ? gt[3] : gt[2], g11 = cb ? gt[2] : gt[3];
              V2 o0, o1;
              o0.x = x0 * g00 + x1 * g10;   // r = 0, d = 0
              o0.y = x0 * g01 + x1 * g11;   // r = 0, d = 1
              o1.x = x0 * g10 + x1 * g00;   // r = 1, d = 0
              o1.y = x0 * g11 + x1 * g01;   // r = 1, d = 1
              *reinterpret_cast<V2*>(nxt + base) = o0;
              *reinterpret_cast<V2*>(nxt + (base | bitQ)) = o1;
            }
          } else {
            // out[r, c, v] = [v = c] sum_{l,u} in[l, c, u] g[l^r][u^c]; qubit bit P, check bit P-1.
            const int cpos = P - 1;
            for (int g = lane; g < nq; g += 32) {
              const int base = ((g >> (P - 1)) << (P + 1)) | ((g & lowmask) << 1);
              const int cb = (base >> cpos) & 1;
              const V2 i0 = *reinterpret_cast<const V2*>(cur + base);          // in[0][u=0,1]
              const V2 i1 = *reinterpret_cast<const V2*>(cur + (base | bitP)); // in[1][u=0,1]
              // g[l ^ r][u ^ c]
              const T g00 = cb ? gt[1] : gt[0], g01 = cb ? gt[0] : gt[1];
              const T g10 = cb ? gt[3] : gt[2], g11 = cb ? gt[2] : gt[3];
              const T r0 = i0.x * g00 + i0.y * g01 + i1.x * g10 + i1.y * g11;
              const T r1 = i0.x * g10 + i0.y * g11 + i1.x * g00 + i1.y * g01;
              V2 o0, o1;
              o0.x = cb ? T(0) : r0; o0.y = cb ? r0 : T(0);
              o1.x = cb ? T(0) : r1; o1.y = cb ? r1 : T(0);
              *reinterpret_cast<V2*>(nxt + base) = o0;
              *reinterpret_cast<V2*>(nxt + (base | bitP)) = o1;
            }
          }
          __syncwarp();
          T* tmp = cur; cur = nxt; nxt = tmp;
          ++s;
          continue;
        }
      }
      if (interior && !((ni + nj) & 1)) {
        // Interior qubit: out[r][d] = sum_{l,u} in[l][u] g[l^r][u^d], an XOR
        // convolution with the 2 x 2 table g[alpha][beta].
        const int fr = c.frame[ni * c.g.W + nj];
        const int fx = fr & 1, fz = (fr >> 1) & 1;
        const bool alpha_is_z = ((ni & 1) == 0) == rowwise;
        T gt[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const int al = q >> 1, be = q & 1;
          const int xb = alpha_is_z ? be : al, zb = alpha_is_z ? al : be;
          gt[q] = ((fx ^ xb) | (fz ^ zb)) ? c.pE : c.pI;
        }
        for (int g = lane; g < nq; g += 32) {
          const int base = ((g >> (P - 1)) << (P + 1)) | ((g & lowmask) << 1);
          const V2 i0 = *reinterpret_cast<const V2*>(cur + base);          // in[0][0], in[0][1]
          const V2 i1 = *reinterpret_cast<const V2*>(cur + (base | bitP)); // in[1][0], in[1][1]
          V2 o0, o1;
          o0.x = i0.x * gt[0] + i0.y * gt[1] + i1.x * gt[2] + i1.y * gt[3];
          o0.y = i0.x * gt[1] + i0.y * gt[0] + i1.x * gt[3] + i1.y * gt[2];
          o1.x = i0.x * gt[2] + i0.y * gt[3] + i1.x * gt[0] + i1.y * gt[1];
          o1.y = i0.x * gt[3] + i0.y * gt[2] + i1.x * gt[1] + i1.y * gt[0];
          *reinterpret_cast<V2*>(nxt + base) = o0;
          *reinterpret_cast<V2*>(nxt + (base | bitP)) = o1;
        }
        __syncwarp();
        T* tmp = cur; cur = nxt; nxt = tmp;
        continue;
      }
      if (interior) {
        // Interior check: a copy tensor over four legs, out[r][d] = [r = d] in[r][r].
        for (int g = lane; g < nq; g += 32) {
          const int base = ((g >> (P - 1)) << (P + 1)) | ((g & lowmask) << 1);
          const V2 i0 = *reinterpret_cast<const V2*>(cur + base);
          const V2 i1 = *reinterpret_cast<const V2*>(cur + (base | bitP));
          V2 o0, o1;
          o0.x = i0.x; o0.y = T(0);
          o1.x = T(0); o1.y = i1.y;
          *reinterpret_cast<V2*>(nxt + base) = o0;
          *reinterpret_cast<V2*>(nxt + (base | bitP)) = o1;
        }
        __syncwarp();
        T* tmp = cur; cur = nxt; nxt = tmp;
        continue;
      }
      // Border node: the general 16-entry tensor (missing legs carry 0).
      if (lane < 16)
        ws.wn[lane] = node_value<T>(c.frame, c.g.W, c.pI, c.pE, ni, nj, f.dir, (lane >> 3) & 1, (lane >> 2) & 1,
                                    (lane >> 1) & 1, lane & 1);
      __syncwarp();
      T w[16];
#pragma unroll
      for (int q = 0; q < 16; ++q) w[q] = ws.wn[q];
      __syncwarp();
      for (int g = lane; g < nq; g += 32) {
        const int base = ((g >> (P - 1)) << (P + 1)) | ((g & lowmask) << 1);
        const V2 i0 = *reinterpret_cast<const V2*>(cur + base);          // (l=0,u=0), (l=0,u=1)
        const V2 i1 = *reinterpret_cast<const V2*>(cur + (base | bitP)); // (l=1,u=0), (l=1,u=1)
        V2 o0, o1;
        // w index: ((l*2 + r)*2 + u)*2 + d
        o0.x = i0.x * w[0] + i0.y * w[2] + i1.x * w[8] + i1.y * w[10];     // r=0, d=0
        o0.y = i0.x * w[1] + i0.y * w[3] + i1.x * w[9] + i1.y * w[11];     // r=0, d=1
        o1.x = i0.x * w[4] + i0.y * w[6] + i1.x * w[12] + i1.y * w[14];    // r=1, d=0
        o1.y = i0.x * w[5] + i0.y * w[7] + i1.x * w[13] + i1.y * w[15];    // r=1, d=1
        *reinterpret_cast<V2*>(nxt + base) = o0;
        *reinterpret_cast<V2*>(nxt + (base | bitP)) = o1;
      }
      __syncwarp();
      T* tmp = cur; cur = nxt; nxt = tmp;
    }
    // Side message B: closes the column's vertical leg.
    {
      FState ns = st;
      ns.hv = 0;
      if (f.b_idx < 0) ns.bb = 0;
      else if (t < sd) ns.bb = st.bb + 1;
      else if (t == sd) ns.bb = nf;
      else ns.bb = st.bb - 1;
      const int n = ns.size();
      if (!(f.b_idx >= 0 && t < sd)) {   // recording v as b's new low bit changes no index
        for (int e = lane; e < n; e += 32) {
          T val;
          if (f.b_idx < 0) {
            val = cur[e << 1];                          // v = 0, b has no bits
          } else if (t == sd) {
            const int b2 = e & ((1 << ns.bb) - 1), ah = e >> ns.bb;   // (a, rows)
            val = T(0);
            for (int b = 0; b < (1 << st.bb); ++b) {
              const int bi = ((ah << st.bb) | b) << 1;
              val += ws.mb[((b << 1) << nf) | b2] * cur[bi] + ws.mb[(((b << 1) | 1) << nf) | b2] * cur[bi | 1];
            }
          } else {
            const int b2 = e & ((1 << ns.bb) - 1), ah = e >> ns.bb;
            const int hi0 = ((ah << st.bb) | b2) << 1;                        // b top bit 0, v = 0
            const int hi1 = ((ah << st.bb) | (1 << (st.bb - 1)) | b2) << 1 | 1; // b top bit 1, v = 1
            val = cur[hi0] + cur[hi1];
          }
          nxt[e] = val;
        }
        __syncwarp();
        T* tmp = cur; cur = nxt; nxt = tmp;
      }
      st = ns;
    }
    if (readout) {   // keep the block value in range; its log goes to the read-out
      const int n = st.size();
      T acc = 0;
      for (int e = lane; e < n; e += 32) acc += cur[e] * cur[e];
      acc = warp_sum(acc);
      const T nrm = xsqrt(acc);
      if (nrm > T(0)) {
        const T inv = T(1) / nrm;
        for (int e = lane; e < n; e += 32) cur[e] *= inv;
        if (lane == 0) log_scale += log((double)nrm);
      }
      __syncwarp();
    }
  }
  if (cur != ws.s0) {
    for (int H = lane; H < (1 << h); H += 32) ws.s0[H] = cur[H];
    __syncwarp();
  }
  return log_scale;
}

// Unit L2 norm (Remark 3) of the 2^w vector x; returns the norm.
template <typename T>
__device__ __forceinline__ T fused_normalize(T* x, int n, int lane) {
  T acc = 0;
  for (int e = lane; e < n; e += 32) acc += x[e] * x[e];
  acc = warp_sum(acc);
  const T nrm = xsqrt(acc);
  const T inv = nrm > T(0) ? T(1) / nrm : T(0);
  __syncwarp();
  for (int e = lane; e < n; e += 32) x[e] *= inv;
  __syncwarp();
  return nrm;
}

template <typename T>
__device__ __forceinline__ double fused_dot(const T* x, const T* y, int n, int lane) {
  double acc = 0.0;
  for (int e = lane; e < n; e += 32) acc += (double)x[e] * (double)y[e];
  return warp_sum(acc);
}

// The per-message term 2 - 2 <x, y>^2 of Delta (Remark 4) for unit vectors
// x (new) and y (old).  FP64 evaluates it as written.  FP32 evaluates the
// same quantity as s (2 - s / 2) with s = ||x - y||^2 (an identity for unit
// vectors): no cancellation when a message barely moved, and no FP64
// instruction per update (FP64 issues at 1/64 of the FP32 rate here).
template <typename T> struct DeltaTerm;
template <> struct DeltaTerm<double> {
  static __device__ __forceinline__ double eval(const double* x, const double* y, int n, int lane) {
    const double o = fused_dot(x, y, n, lane);
    return 2.0 - 2.0 * o * o;
  }
};
template <> struct DeltaTerm<float> {
  static __device__ __forceinline__ float eval(const float* x, const float* y, int n, int lane) {
    float s = 0.f;
    for (int e = lane; e < n; e += 32) {
      const float t = x[e] - y[e];
      s += t * t;
    }
    s = warp_sum(s);
    return s * (2.f - 0.5f * s);
  }
};

// Resident CTAs per SM the register budget is sized for: 32 warps per SM in
// FP32 (64 registers a thread), 16 in FP64; shared memory at d = 11 allows it.
template <typename T, int NW> struct FusedMinBlocks { static constexpr int value = 32 / NW > 1 ? 32 / NW : 1; };
template <int NW> struct FusedMinBlocks<double, NW> { static constexpr int value = 16 / NW > 1 ? 16 / NW : 1; };

// One (syndrome, coset) decoded by the whole CTA: syn_src holds the
// syndrome's m bytes and ``cta`` indexes the outputs (syndrome * 4 + coset).
template <typename T, int NW>
__device__ __forceinline__ void fused_item(const KArgs<T>& a, const Geo g, const int M, const uint8_t* syn_src,
                                           const long long cta, const int coset, unsigned char* smem) {
  using WS = FusedWS<T>;
  const int W = g.W, d = g.d, nb = g.nb;
  const int m = 2 * d * (d - 1);
  const FusedLayout Lo = fused_layout<T>(g, M, NW);
  uint8_t* synd = smem + Lo.synd;
  uint8_t* frame = smem + Lo.frame;
  int16_t* msg_of = reinterpret_cast<int16_t*>(smem + Lo.msg_of);
  int16_t* meta = reinterpret_cast<int16_t*>(smem + Lo.meta);
  int16_t* work = reinterpret_cast<int16_t*>(smem + Lo.work);
  double* ovl = reinterpret_cast<double*>(smem + Lo.ovl);
  double* rlog = reinterpret_cast<double*>(smem + Lo.rlog);
  int* misc = reinterpret_cast<int*>(smem + Lo.misc);
  double* dsh = reinterpret_cast<double*>(smem + Lo.misc + 48);
  T* msgs = reinterpret_cast<T*>(smem + Lo.msgs);
  WS* wsa = reinterpret_cast<WS*>(smem + Lo.ws);

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;

  for (int i = tid; i < m; i += NW * 32) synd[i] = syn_src[i];
  __syncthreads();
  const int bx = (coset == 1 || coset == 2), bz = (coset == 2 || coset == 3);
  for (int e = tid; e < W * W; e += NW * 32) {
    const int i = e / W, j = e % W;
    int fx = 0, fz = 0;
    if ((i & 1) == 0 && (j & 1) == 0) {
      const int r = i >> 1, cc = j >> 1;
      for (int c2 = 0; c2 < cc; ++c2) fx ^= synd[r * (d - 1) + c2];
      for (int r2 = 0; r2 < r; ++r2) fz ^= synd[d * (d - 1) + r2 * d + cc];
      if (bx && r == 0) fx ^= 1;
      if (bz && cc == 0) fz ^= 1;
    }
    frame[e] = (uint8_t)(fx | (fz << 1));
  }
  if (tid == 0) {
    int idx = 0, n0 = 0, n1 = 0;
    for (int I = 0; I < nb; ++I)
      for (int J = 0; J < nb; ++J)
        for (int dir = 0; dir < 4; ++dir) {
          const int key = (I * nb + J) * 4 + dir;
          if (g.has(I, J, dir)) {
            msg_of[key] = (int16_t)idx;
            meta[idx] = (int16_t)key;
            if (((I + J) & 1) == 0) work[n0++] = (int16_t)idx;
            else work[M + n1++] = (int16_t)idx;
            ++idx;
          } else {
            msg_of[key] = -1;
          }
        }
    misc[0] = 0; misc[1] = 0; misc[2] = n0; misc[3] = n1;
  }
  __syncthreads();

  Ctx<T, kFusedK> c;
  c.g = g; c.D = 0; c.cutoff2 = T(0);
  c.pI = (T)(1.0 - a.p); c.pE = (T)(a.p / 3.0);
  c.frame = frame; c.msg_of = msg_of; c.msg_off = nullptr; c.dims = nullptr;
  c.arena = nullptr; c.e0 = nullptr; c.cta_flags = &misc[1];

  // Remark 2: uniform messages of unit norm, unless initial messages are
  // given (learned warm start): those are renormalised on entry.
  for (int idx = warp; idx < M; idx += NW) {
    const int key = meta[idx];
    const int w = g.side_len(key / 4 / nb, (key / 4) % nb, key & 3);
    T* x = msgs + idx * kFusedVec;
    if (a.init_msgs) {
      const float* src = a.init_msgs + (cta * M + idx) * kFusedVec;
      for (int i = lane; i < kFusedVec; i += 32) x[i] = i < (1 << w) ? (T)src[i] : T(0);
      __syncwarp();
      const T nrm = fused_normalize(x, 1 << w, lane);
      if (!(nrm > T(0))) {                            // unusable proposal: fall back to uniform
        const T u = (T)rsqrt((double)(1 << w));
        for (int i = lane; i < (1 << w); i += 32) x[i] = u;
        __syncwarp();
      }
    } else {
      const T u = (T)rsqrt((double)(1 << w));
      for (int i = lane; i < kFusedVec; i += 32) x[i] = i < (1 << w) ? u : T(0);
    }
  }
  __syncthreads();

  WS& ws = wsa[warp];
  const T eta = (T)a.eta, one_m_eta = T(1) - eta;
  double delta = 0.0;
  int it_done = 0;
  for (int it = 1; it <= a.max_iter && M > 0; ++it) {
    for (int color = 0; color < 2; ++color) {       // Remark 8
      const int nwork = misc[2 + color];
      const int16_t* lst = work + color * M;
      for (;;) {
        int item = 0;
        if (lane == 0) item = atomicAdd(&misc[0], 1);
        item = __shfl_sync(kFull, item, 0);
        if (item >= nwork) break;
        const int idx = lst[item];
        const int key = meta[idx];
        const int I = key / 4 / nb, J = (key / 4) % nb, dir = key & 3;
        const Frame f = make_frame(c, I, J, dir);
        fused_sweep(ws, c, msgs, f, false, lane);
        const int n = 1 << f.h;
        T* x = ws.s0;
        T* old = msgs + idx * kFusedVec;
        fused_normalize(x, n, lane);                                  // Remark 3
        for (int e = lane; e < n; e += 32) x[e] = one_m_eta * x[e] + eta * old[e];   // Remark 7
        __syncwarp();
        fused_normalize(x, n, lane);
        const T term = DeltaTerm<T>::eval(x, old, n, lane);
        __syncwarp();
        for (int e = lane; e < n; e += 32) old[e] = x[e];
        if (lane == 0) ovl[idx] = (double)term;
        __syncwarp();
      }
      __syncthreads();
      if (tid == 0) misc[0] = 0;
      __syncthreads();
    }
    if (warp == 0) {                                   // Remark 4
      double acc = 0.0;
      for (int i = lane; i < M; i += 32) acc += ovl[i];
      acc = warp_sum(acc);
      if (lane == 0) dsh[0] = sqrt(fmax(acc, 0.0)) / M;
    }
    __syncthreads();
    delta = dsh[0];
    it_done = it;
    if (delta < a.delta0) break;
  }

  if (a.final_msgs)
    for (int e = tid; e < M * kFusedVec; e += NW * 32) a.final_msgs[cta * M * kFusedVec + e] = (float)msgs[e];

  // Lemma 1 read-out.
  if (tid == 0) {
    int ne = 0;
    for (int idx = 0; idx < M; ++idx) {
      const int dir = meta[idx] & 3;
      if (dir == kDirR || dir == kDirD) work[ne++] = (int16_t)idx;
    }
    misc[4] = ne;
    misc[0] = 0;
  }
  __syncthreads();
  const int nedge = misc[4];
  const int nblk = nb * nb;
  for (;;) {
    int item = 0;
    if (lane == 0) item = atomicAdd(&misc[0], 1);
    item = __shfl_sync(kFull, item, 0);
    if (item >= nblk + nedge) break;
    if (item < nblk) {
      const int I = item / nb, J = item % nb;
      const Frame f = make_frame(c, I, J, kDirR);
      const double ls = fused_sweep(ws, c, msgs, f, true, lane);   // valid in lane 0
      const int right = J + 1 < nb ? msg_index(c, I, J + 1, kDirL) : -1;
      double z;
      if (right >= 0) z = fused_dot(ws.s0, msgs + right * kFusedVec, 1 << f.h, lane);
      else z = (double)ws.s0[0];
      if (lane == 0) {
        rlog[item] = ls + log(fabs(z));
        if (!(z > 0.0)) atomicOr(&misc[1], kFlagBlock);
      }
      __syncwarp();
    } else {
      const int e = item - nblk;
      const int idx = work[e];
      const int key = meta[idx];
      const int I = key / 4 / nb, J = (key / 4) % nb, dir = key & 3;
      const int other = dir == kDirR ? msg_index(c, I, J + 1, kDirL) : msg_index(c, I + 1, J, kDirU);
      const int w = g.side_len(I, J, dir);
      const double o = fused_dot(msgs + idx * kFusedVec, msgs + other * kFusedVec, 1 << w, lane);
      if (lane == 0) {
        rlog[item] = -log(fabs(o));
        if (!(o > 0.0)) atomicOr(&misc[1], kFlagOverlap);
      }
    }
  }
  __syncthreads();
  if (warp == 0) {
    double acc = 0.0;
    for (int i = lane; i < nblk + nedge; i += 32) acc += rlog[i];
    acc = warp_sum(acc);
    if (lane == 0) {
      int fl = misc[1];
      if (!isfinite(acc)) fl |= kFlagNonfinite;
      if (!(delta < a.delta1)) fl |= kFlagUntrusted;
      a.logp[cta] = acc;
      a.delta[cta] = delta;
      a.iters[cta] = it_done;
      a.flags[cta] = fl;
    }
  }
}


template <typename T, int NW>
__global__ void __launch_bounds__(NW * 32, (FusedMinBlocks<T, NW>::value)) fused_kernel(KArgs<T> a) {
  extern __shared__ __align__(16) unsigned char smem[];
  const long long cta = blockIdx.x;
  const int m = 2 * a.geo.d * (a.geo.d - 1);
  fused_item<T, NW>(a, a.geo, a.M, a.synd + (cta >> 2) * m, cta, (int)(cta & 3), smem);
}

// A batch of syndromes of different distances in one persistent launch: CTAs
// take (syndrome, coset) items from a global counter in the order given
// (largest distance first balances the tail) until the batch is done.
struct MixedArgs {
  const int32_t* d_of;          // distance of each syndrome
  const int64_t* offsets;       // byte offset of each syndrome in the packed buffer
  const int32_t* order;         // syndrome order of the items, or null
  unsigned long long* counter;  // zero before the launch
  long long n_items;            // 4 * B
  int k;
};

template <typename T, int NW>
__global__ void __launch_bounds__(NW * 32, (FusedMinBlocks<T, NW>::value)) fused_mixed_kernel(KArgs<T> a, MixedArgs mx) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ long long item_sh;
  for (;;) {
    if (threadIdx.x == 0) item_sh = (long long)atomicAdd(mx.counter, 1ull);
    __syncthreads();
    const long long item = item_sh;
    __syncthreads();
    if (item >= mx.n_items) break;
    const long long shot = mx.order ? (long long)mx.order[item >> 2] : (item >> 2);
    const int coset = (int)(item & 3);
    const Geo g = make_geo(mx.d_of[shot], mx.k);
    int M = 0, ae = 0;
    count_messages(g, 1, &M, &ae);
    fused_item<T, NW>(a, g, M, a.synd + mx.offsets[shot], shot * 4 + coset, coset, smem);
    __syncthreads();
  }
}

}  // namespace bbp
