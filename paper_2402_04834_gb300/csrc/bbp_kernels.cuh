// Device code of the blockBP decoder (arXiv:2402.04834, Sec. III.D,
// Algorithm 1, Remarks 2-8, Lemma 1) for sm_103a.
//
// One CTA decodes one (syndrome, coset) pair from start to end: it builds
// the coset frame f_s * L (Algorithm 1, first steps), keeps the MPS messages
// of all M directed block edges in a global-memory arena, runs the
// chessboard schedule (Remark 8) with one warp per message update and a
// __syncthreads() between half-rounds, evaluates Delta (Remark 4) and the
// Bethe read-out of Lemma 1.  No CTA ever waits on another CTA.
//
// A warp owns a shared-memory workspace holding the running boundary MPS of
// one block contraction.  The linear algebra is warp-cooperative on that
// workspace: an LQ step by two passes of modified Gram-Schmidt in registers
// (right-to-left canonicalisation sweep) and one-sided Jacobi SVD with
// truncation (left-to-right sweep), the textbook MPS compression of
// Sec. III.A.  Every loop is bounded; nothing spins.
#pragma once

#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "bbp_geometry.h"

namespace bbp {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kMaxSweeps = 48;          // one-sided Jacobi sweep limit
constexpr int kFlagUntrusted = 1, kFlagOverlap = 2, kFlagBlock = 4, kFlagNonfinite = 8;
constexpr int kFlagCapacity = 1 << 16;  // a bond exceeded its slot (never expected)
constexpr int kFlagCheck = 1 << 17;     // a device-checked index or size was out of range

// Device bounds checks.  Built with -DBLOCKBP_CHECKS (a separate library,
// build(checks=True)), every table index the kernels derive (message
// indices, list entries, slot offsets, record indices) is tested against
// its buffer before use; a failed test sets kFlagCheck in *flags and the
// access is skipped.  The default build compiles the tests away.
#ifdef BLOCKBP_CHECKS
constexpr bool kChecks = true;
#else
constexpr bool kChecks = false;
#endif
__device__ __forceinline__ bool dev_check(bool ok, int* flags) {
  if constexpr (kChecks) {
    if (!ok) {
      atomicOr(flags, kFlagCheck);
      return false;
    }
  }
  return true;
}

template <typename T> struct Eps;
template <> struct Eps<double> { static __device__ __forceinline__ double v() { return 2.220446049250313e-16; } };
template <> struct Eps<float> { static __device__ __forceinline__ float v() { return 1.1920928955078125e-7f; } };

__device__ __forceinline__ double xsqrt(double x) { return sqrt(x); }
__device__ __forceinline__ float xsqrt(float x) { return sqrtf(x); }
__device__ __forceinline__ double xabs(double x) { return fabs(x); }
__device__ __forceinline__ float xabs(float x) { return fabsf(x); }

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
  return v;
}

// Sum over aligned groups of G lanes (G a power of two); every lane of a
// group gets the bitwise-identical result (xor butterfly, commutative adds).
template <typename T>
__device__ __forceinline__ T group_sum(T v, int G) {
  for (int o = G >> 1; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
  return v;
}

// Per-warp shared-memory workspace.  SITE holds one (2D) x 2 x (2D) site.
template <typename T, int K, int DM>
struct WarpWS {
  static constexpr int SITE = 8 * DM * DM;
  static constexpr int VM = 4 * DM * DM;
  T psi[K][SITE];      // running MPS, site s is row-major [left][phys][right]
  T tmp[SITE];         // scratch site
  T mat[SITE];         // Gram-Schmidt coefficients / S V^T
  T vm[VM];            // the L factor of a right-to-left step
  T wn[K * 16];        // node tensors of the current column, [s][in][out][cp][cn]
  int bond[K + 2];     // bond[s] = left bond of site s; bond[h] = right end bond
};

// Read-only view of one MPS site: element (a, p, b) = ptr[a*sa + p*sp + b*sb].
template <typename T>
struct SiteRef {
  const T* ptr;
  int na, nb, sa, sp, sb;
  __device__ __forceinline__ T at(int a, int p, int b) const { return ptr[a * sa + p * sp + b * sb]; }
};

template <typename T>
struct KArgs {
  Geo geo;
  int M, D, max_iter, arena_elems;
  double p, eta, delta0, delta1, cutoff;
  const uint8_t* synd;
  T* arena;
  double* logp;
  double* delta;
  int32_t* iters;
  int32_t* flags;
  const float* init_msgs;   // fused path: [cta][M][16] initial messages, or null (uniform)
  float* final_msgs;        // fused path: [cta][M][16] messages after the BP loop, or null
  long long n_items;        // fused path, messages in the workspace: (syndrome, coset group) items
  long long slot_elems;     // fused path, messages in the workspace: scalars of one CTA's slot in arena
  // The constants above in working precision, rounded once by the host
  // (set_working): kernels read them as arguments, so no FP64 instruction
  // recomputes them inside an FP32 kernel's loops.
  T pI_w, pE_w;             // pi(I) = 1 - p, pi(X) = p / 3
  T eta_w, one_m_eta_w;     // eta, 1 - eta (the latter in working precision)
  T cutoff2_w;              // cutoff^2
};

// Fill KArgs' working-precision constants from its double parameters (the
// host's IEEE double arithmetic and rounding to T).
template <typename T>
inline void set_working(KArgs<T>& k) {
  k.pI_w = (T)(1.0 - k.p);
  k.pE_w = (T)(k.p / 3.0);
  k.eta_w = (T)k.eta;
  k.one_m_eta_w = T(1) - k.eta_w;
  k.cutoff2_w = (T)(k.cutoff * k.cutoff);
}

// Everything a warp needs to reach the CTA's shared tables.
template <typename T, int K>
struct Ctx {
  Geo g;
  int D;
  T cutoff2;               // cutoff^2 on squared singular values
  T pI, pE;                // pi(I) and pi(X) = pi(Y) = pi(Z)
  const uint8_t* frame;    // [W][W] bit 0 = x, bit 1 = z of f_s * L
  const int16_t* msg_of;   // [(I*nb+J)*4+dir] -> message index or -1
  const int32_t* msg_off;  // element offset of each message slot in the arena
  int8_t* dims;            // [M][K+1] bond dims of every message
  T* arena;                // this CTA's message arena
  const T* e0;             // the trivial border site (1, 0)
  int* cta_flags;
};

// ---------------------------------------------------------------------------
// Node tensors of the coset network (Sec. III.A; the construction is rebuilt
// from Eq. noise-cosets): check nodes are copy tensors over their existing
// legs, qubit nodes are pi(f_e (+) P(legs)).  Legs are given in the rotated
// frame (in, out, chain-prev, chain-next) of direction ``dir``; legs that
// leave the grid must carry 0.
template <typename T>
__device__ __forceinline__ T node_value(const uint8_t* frame, int W, T pI, T pE, int i, int j,
                                        int dir, int in, int out, int cp, int cn) {
  int l, r, u, dn;
  switch (dir) {
    case kDirR: l = in; r = out; u = cp; dn = cn; break;
    case kDirL: r = in; l = out; u = cp; dn = cn; break;
    case kDirD: u = in; dn = out; l = cp; r = cn; break;
    default:    dn = in; u = out; l = cp; r = cn; break;
  }
  const bool hl = j > 0, hr = j < W - 1, hu = i > 0, hd = i < W - 1;
  if ((!hl && l) || (!hr && r) || (!hu && u) || (!hd && dn)) return T(0);
  if ((i + j) & 1) {  // check node: copy tensor
    int v = -1;
    bool ok = true;
    if (hl) v = l;
    if (hr) { if (v < 0) v = r; else ok = ok && (r == v); }
    if (hu) { if (v < 0) v = u; else ok = ok && (u == v); }
    if (hd) { if (v < 0) v = dn; else ok = ok && (dn == v); }
    return ok ? T(1) : T(0);
  }
  const int f = frame[i * W + j];
  int x, z;
  if ((i & 1) == 0) { x = u ^ dn; z = l ^ r; }   // horizontal-edge qubit
  else              { x = l ^ r;  z = u ^ dn; }  // vertical-edge qubit
  return (((f & 1) ^ x) | (((f >> 1) & 1) ^ z)) ? pE : pI;
}

// ---------------------------------------------------------------------------
// Message access.
template <typename T, int K>
__device__ __forceinline__ SiteRef<T> msg_site(const Ctx<T, K>& c, int idx, int w, int s, bool reversed) {
  SiteRef<T> r;
  if (idx < 0) {  // border: trivial dim-1 message, realised as e0 = (1, 0)
    r.ptr = c.e0; r.na = 1; r.nb = 1; r.sa = 0; r.sp = 1; r.sb = 0;
    return r;
  }
  const int site = reversed ? (w - 1 - s) : s;
  const int8_t* dm = c.dims + idx * (K + 1);
  const int bl = dm[site], br = dm[site + 1];
  r.ptr = c.arena + c.msg_off[idx] + msg_site_offset(site, w, c.D);
  if (!reversed) { r.na = bl; r.nb = br; r.sa = 2 * br; r.sp = br; r.sb = 1; }
  else           { r.na = br; r.nb = bl; r.sa = 1; r.sp = br; r.sb = 2 * br; }
  return r;
}

template <typename T, int K, int DM>
__device__ __forceinline__ SiteRef<T> psi_site(const WarpWS<T, K, DM>& ws, int s) {
  SiteRef<T> r;
  r.ptr = ws.psi[s]; r.na = ws.bond[s]; r.nb = ws.bond[s + 1];
  r.sa = 2 * r.nb; r.sp = r.nb; r.sb = 1;
  return r;
}

template <typename T>
__device__ __forceinline__ void warp_copy(T* dst, const T* src, int n, int lane) {
  for (int e = lane; e < n; e += 32) dst[e] = src[e];
}

// Quotient by a small runtime divisor without an integer division: exact for
// 0 <= e < 2^16 and 1 <= d <= 2^10, since (e + 1/2)/d stays at least 1/(2d)
// away from an integer and the float product errs by far less.
struct FastDiv {
  float rcp;
  int d;
  __device__ __forceinline__ explicit FastDiv(int dd) : rcp(1.0f / (float)dd), d(dd) {}
  __device__ __forceinline__ int quo(int e) const { return __float2int_rz(((float)e + 0.5f) * rcp); }
};

// ---------------------------------------------------------------------------
// Right-to-left step: site s = L Q with Q row-orthonormal, Q stays at site s,
// L is absorbed into site s-1.  Q comes from two passes of row-oriented
// modified Gram-Schmidt held in registers: row a of the (pl x 2pr) site
// matrix lives in lanes a and a+16, each holding 2D of its columns; step j
// broadcasts q_j by shuffles and every later row projects it out.  A row
// whose residual falls below tau times its own norm is linearly dependent
// on the earlier rows and is dropped (its coefficients stay in L), so the
// bond shrinks to the numerical rank.  The two passes give orthogonality to
// working precision whenever the rows are independent to tau.
template <typename T> struct GsTau;
template <> struct GsTau<double> { static __device__ __forceinline__ double v() { return 1e-13; } };
template <> struct GsTau<float> { static __device__ __forceinline__ float v() { return 5e-7f; } };

template <typename T, int K, int DM>
__device__ __noinline__ void lq_step(WarpWS<T, K, DM>& ws, int s, int lane) {
  constexpr int HC = 2 * DM;                 // columns per half-row
  const int pl = ws.bond[s], pr = ws.bond[s + 1];
  const int nc = 2 * pr;                     // row length (<= 4D)
  const int row = lane & 15, half = lane >> 4;
  const bool own = row < pl;
  T x[HC];
  const T* A = ws.psi[s];
#pragma unroll
  for (int t = 0; t < HC; ++t) {
    const int cc = half * HC + t;
    x[t] = (own && cc < nc) ? A[row * nc + cc] : T(0);
  }
  T nrm0 = 0;
#pragma unroll
  for (int t = 0; t < HC; ++t) nrm0 += x[t] * x[t];
  nrm0 += __shfl_xor_sync(kFull, nrm0, 16);
  T* L1 = ws.mat;                             // [pass][a][j] coefficients, pl x pl each
  T* L2 = ws.mat + 4 * DM * DM;
  for (int e = lane; e < 2 * 4 * DM * DM; e += 32) ws.mat[e] = T(0);
  __syncwarp();
  const T tau2 = GsTau<T>::v() * GsTau<T>::v();
  unsigned kept = 0;                          // bit j set: q_j is a row of Q
  for (int pass = 0; pass < 2; ++pass) {
    T* Lc = pass == 0 ? L1 : L2;
    T ref = pass == 0 ? nrm0 : T(1);
    for (int j = 0; j < pl; ++j) {
      // Normalise row j (its residual after q_0..q_{j-1} were projected out).
      T n2 = 0;
#pragma unroll
      for (int t = 0; t < HC; ++t) n2 += x[t] * x[t];
      n2 += __shfl_xor_sync(kFull, n2, 16);
      const T nj2 = __shfl_sync(kFull, n2, j);
      const T rj2 = __shfl_sync(kFull, ref, j);
      const bool indep = (pass == 0) ? (nj2 > tau2 * rj2 && nj2 > T(0)) : (((kept >> j) & 1u) && nj2 > T(0));
      if (pass == 0 && indep) kept |= 1u << j;
      const T inv = indep ? T(1) / xsqrt(nj2) : T(0);
      if (row == j) {
#pragma unroll
        for (int t = 0; t < HC; ++t) x[t] *= inv;
        if (half == 0) Lc[j * pl + j] = indep ? xsqrt(nj2) : T(0);
      }
      if (!indep) continue;
      // Broadcast q_j and project it out of the later rows.
      T q[HC];
#pragma unroll
      for (int t = 0; t < HC; ++t) q[t] = __shfl_sync(kFull, x[t], j + 16 * half);
      T cf = 0;
#pragma unroll
      for (int t = 0; t < HC; ++t) cf += x[t] * q[t];
      cf += __shfl_xor_sync(kFull, cf, 16);
      if (own && row > j) {
#pragma unroll
        for (int t = 0; t < HC; ++t) x[t] -= cf * q[t];
        if (half == 0) Lc[row * pl + j] = cf;
      }
    }
  }
  __syncwarp();
  // Compact the kept rows: Q (r x nc) into site s.
  if (kept == 0u) {          // zero site: keep one (zero) row so every bond stays >= 1
    kept = 1u;
    if (row == 0) {
#pragma unroll
      for (int t = 0; t < HC; ++t) x[t] = T(0);
    }
  }
  const int r = __popc(kept);
  const int myidx = __popc(kept & ((1u << row) - 1u));
  T* Q = ws.psi[s];
  if (own && ((kept >> row) & 1u)) {
#pragma unroll
    for (int t = 0; t < HC; ++t) {
      const int cc = half * HC + t;
      if (cc < nc) Q[myidx * nc + cc] = x[t];
    }
  }
  // L = L1 * L2 restricted to kept columns: L[a][k] (pl x r) into vm.
  T* Lm = ws.vm;
  const FastDiv dr(r);
  for (int e = lane; e < pl * r; e += 32) {
    const int aa = dr.quo(e), kk = e - aa * r;
    int j2 = 0, cnt = 0;
    for (j2 = 0; j2 < pl; ++j2) {
      if ((kept >> j2) & 1u) { if (cnt == kk) break; ++cnt; }
    }
    T acc = 0;
    for (int j = 0; j <= aa; ++j) acc += L1[aa * pl + j] * L2[j * pl + j2];
    Lm[e] = acc;
  }
  __syncwarp();
  // Site s-1 <- site s-1 * L.
  const int bl = ws.bond[s - 1];
  T* out = ws.tmp;
  const T* P = ws.psi[s - 1];
  for (int e = lane; e < bl * 2 * r; e += 32) {
    const int rr = dr.quo(e), kk = e - rr * r;
    T acc = 0;
    for (int aa = 0; aa < pl; ++aa) acc += P[rr * pl + aa] * Lm[aa * r + kk];
    out[e] = acc;
  }
  __syncwarp();
  warp_copy(ws.psi[s - 1], out, bl * 2 * r, lane);
  if (lane == 0) ws.bond[s] = r;
  __syncwarp();
}

// ---------------------------------------------------------------------------
// Round-robin (circle method) partner of column j in round r for np (even)
// players: every pair meets exactly once in np-1 rounds.
__device__ __forceinline__ int rr_partner(int j, int r, int np) {
  const int nm = np - 1;                 // r < nm, 0 <= j < np
  if (j == 0) return 1 + r;
  int a = j - 1 - r;
  if (a < 0) a += nm;
  if (a == 0) return 0;
  int b = nm - a + r;
  if (b >= nm) b -= nm;
  return 1 + b;
}

// Left-to-right step at site s: one-sided (Hestenes) Jacobi SVD of the
// (2 pl) x pr site matrix, keep at most D singular values above
// cutoff * sigma_1, site s <- U, site s+1 <- S V^T * site s+1.
//
// Column j of A and of V live in registers of lanes j (rows 0..D-1) and
// j+16 (rows D..2D-1); a round exchanges whole columns with the partner
// lane, so the three inner products need one shuffle each and no
// reduction tree.  Both partners evaluate the rotation from bitwise-equal
// operands.  Pairs where both columns are below (cutoff/4) sigma_F/sqrt(n)
// or either column is at rounding level (eps ||A||_F / 16) are skipped:
// they cannot change the kept subspace, and rotating rounding noise never
// converges.  The rounding level sits at eps/16 rather than eps: FP32
// columns between the two still carry directions that change log P by up to
// a few 1e-3 when dropped (measured at d = 11, p = 0.05).
template <typename T, int K, int DM>
__device__ __noinline__ void svd_step(WarpWS<T, K, DM>& ws, const Ctx<T, K>& c, int s, int lane) {
  static_assert(DM <= 8, "register Jacobi holds at most 16 columns");
  const int pl = ws.bond[s], pr = ws.bond[s + 1];
  const int m = 2 * pl, n = pr;
  const int col = lane & 15, half = lane >> 4;
  const int row0 = half * DM;
  const bool on = col < n;
  T a[DM], v[DM];
  const T* S = ws.psi[s];
#pragma unroll
  for (int t = 0; t < DM; ++t) {
    const int i = row0 + t;
    a[t] = (on && i < m) ? S[i * n + col] : T(0);
    v[t] = (on && i == col) ? T(1) : T(0);
  }
  T fro = 0;
#pragma unroll
  for (int t = 0; t < DM; ++t) fro += a[t] * a[t];
  fro = warp_sum(fro);
  const T eps = Eps<T>::v();
  const T tol = T(4) * eps * xsqrt(T(m));
  const T thr2 = c.cutoff2 * fro / (T(16) * T(n));
  const T noise2 = eps * eps * fro / T(256);
  const int np = (n + 1) & ~1;
  if (n >= 2) {
    for (int sweep = 0; sweep < kMaxSweeps; ++sweep) {
      bool rotated = false;
      for (int rnd = 0; rnd < np - 1; ++rnd) {
        const int pj = on ? rr_partner(col, rnd, np) : col;
        const int src = (pj & 15) | (half << 4);
        T pa[DM], pv[DM];
#pragma unroll
        for (int t = 0; t < DM; ++t) {
          pa[t] = __shfl_sync(kFull, a[t], src);
          pv[t] = __shfl_sync(kFull, v[t], src);
        }
        T own = 0, oth = 0, cr = 0;
#pragma unroll
        for (int t = 0; t < DM; ++t) { own += a[t] * a[t]; oth += pa[t] * pa[t]; cr += a[t] * pa[t]; }
        own += __shfl_xor_sync(kFull, own, 16);
        oth += __shfl_xor_sync(kFull, oth, 16);
        cr += __shfl_xor_sync(kFull, cr, 16);
        const bool lo = col < pj;
        const T al = lo ? own : oth, be = lo ? oth : own;
        const bool act = on && pj < n && pj != col;
        const bool skip = (al < thr2 && be < thr2) || al < noise2 || be < noise2;
        if (act && !skip && cr != T(0) && xabs(cr) > tol * xsqrt(al) * xsqrt(be)) {
          const T zeta = (be - al) / (T(2) * cr);
          const T tt = (zeta >= T(0) ? T(1) : T(-1)) / (xabs(zeta) + xsqrt(T(1) + zeta * zeta));
          const T cs = T(1) / xsqrt(T(1) + tt * tt);
          const T sn = cs * tt;
          if (lo) {
#pragma unroll
            for (int t = 0; t < DM; ++t) { a[t] = cs * a[t] - sn * pa[t]; v[t] = cs * v[t] - sn * pv[t]; }
          } else {
#pragma unroll
            for (int t = 0; t < DM; ++t) { a[t] = sn * pa[t] + cs * a[t]; v[t] = sn * pv[t] + cs * v[t]; }
          }
          rotated = true;
        }
      }
      if (!__any_sync(kFull, rotated)) break;
    }
  }
  // Squared singular values, their order and the kept count.
  T sq = 0;
#pragma unroll
  for (int t = 0; t < DM; ++t) sq += a[t] * a[t];
  sq += __shfl_xor_sync(kFull, sq, 16);
  if (!on) sq = T(-1);
  int rank = 0;
  T smax = 0;
  for (int i = 0; i < n; ++i) {
    const T si = __shfl_sync(kFull, sq, i);
    rank += (si > sq || (si == sq && i < col)) ? 1 : 0;
    smax = si > smax ? si : smax;
  }
  // A singular value is kept above cutoff * sigma_1 and above the rounding
  // floor of the Jacobi sweep (eps ||A||_F / 16), below which its direction
  // is not resolved; the floor only binds in FP32.
  const T floor2 = c.cutoff2 * smax > noise2 ? c.cutoff2 * smax : noise2;
  int keep = 0;
  for (int i = 0; i < n; ++i) keep += (__shfl_sync(kFull, sq, i) > floor2) ? 1 : 0;
  int r = imin(imin(keep, c.D), m);
  if (r < 1) r = 1;
  __syncwarp();
  // Site s <- U (m x r) row-major as (pl, 2, r); mat <- S V^T (r x n).
  T* dst = ws.psi[s];
  T* svt = ws.mat;
  if (on && rank < r) {
    const T sg = xsqrt(sq);
    const T inv = sg > T(0) ? T(1) / sg : T(0);
#pragma unroll
    for (int t = 0; t < DM; ++t) {
      const int i = row0 + t;
      if (i < m) dst[i * r + rank] = a[t] * inv;
      if (i < n) svt[rank * n + i] = sg * v[t];
    }
  }
  __syncwarp();
  // Site s+1 <- (S V^T) * site s+1.
  const int nx = 2 * ws.bond[s + 2];
  const T* B = ws.psi[s + 1];
  T* out = ws.tmp;
  const FastDiv dnx(nx);
  for (int e = lane; e < r * nx; e += 32) {
    const int kk = dnx.quo(e), qq = e - kk * nx;
    T acc = 0;
    for (int b = 0; b < n; ++b) acc += svt[kk * n + b] * B[b * nx + qq];
    out[e] = acc;
  }
  __syncwarp();
  warp_copy(ws.psi[s + 1], out, r * nx, lane);
  if (lane == 0) ws.bond[s + 1] = r;
  __syncwarp();
}

// Divide the last site by its Frobenius norm; return log(norm) when
// want_log (only the read-out keeps the scale; the log is an FP64 call,
// which GB300 issues at 1/64 of the FP32 rate), else 0.
template <typename T, int K, int DM>
__device__ double normalize_last(WarpWS<T, K, DM>& ws, int h, int lane, bool want_log) {
  const int n = ws.bond[h - 1] * 2 * ws.bond[h];
  T* A = ws.psi[h - 1];
  T acc = 0;
  for (int e = lane; e < n; e += 32) acc += A[e] * A[e];
  acc = warp_sum(acc);
  const T nrm = xsqrt(acc);
  if (nrm > T(0) && isfinite(nrm)) {
    const T inv = T(1) / nrm;
    for (int e = lane; e < n; e += 32) A[e] *= inv;
  }
  __syncwarp();
  return want_log ? log((double)nrm) : 0.0;
}

// MPS compression (Sec. III.A): QR sweep right to left, truncated SVD sweep
// left to right, normalisation (Remark 3).  Returns the log of the norm
// when want_log.
template <typename T, int K, int DM>
__device__ __noinline__ double compress(WarpWS<T, K, DM>& ws, const Ctx<T, K>& c, int h, int lane, bool want_log) {
  for (int s = h - 1; s >= 1; --s) lq_step(ws, s, lane);
  for (int s = 0; s + 1 < h; ++s) svd_step(ws, c, s, lane);
  return normalize_last(ws, h, lane, want_log);
}

// Accumulation of the overlaps' transfer matrices: double in FP64 kernels;
// in FP32 kernels a float pair (head + tail, about 48 bits), whose
// multiply-adds run on the FP32 pipe: native FP64 there would issue at
// 1/64 of the rate, and the overlap must hold 1 - <m|m'> of converged
// messages (1e-7 and below) for Delta (Remark 4).
struct F2 {
  float h, l;
};
template <typename T> struct OvAcc;
template <> struct OvAcc<double> {
  using V = double;
  static __device__ __forceinline__ V zero() { return 0.0; }
  static __device__ __forceinline__ V one() { return 1.0; }
  static __device__ __forceinline__ V mac(V acc, V x, double y) { return fma(x, y, acc); }
  static __device__ __forceinline__ double value(V v) { return v; }
};
template <> struct OvAcc<float> {
  using V = F2;
  static __device__ __forceinline__ V zero() { return F2{0.f, 0.f}; }
  static __device__ __forceinline__ V one() { return F2{1.f, 0.f}; }
  // acc + x y with x a pair and y a float: the head product exactly (its
  // rounding error by fma), the tail product, then a two-sum into acc.
  static __device__ __forceinline__ V mac(V acc, V x, float y) {
    const float ph = __fmul_rn(x.h, y);
    const float pl = __fmaf_rn(x.l, y, __fmaf_rn(x.h, y, -ph));
    const float s = __fadd_rn(acc.h, ph);
    const float bv = __fsub_rn(s, acc.h);
    const float e = __fadd_rn(__fadd_rn(__fsub_rn(acc.h, __fsub_rn(s, bv)), __fsub_rn(ph, bv)), __fadd_rn(acc.l, pl));
    const float hh = __fadd_rn(s, e);
    return F2{hh, __fsub_rn(e, __fsub_rn(hh, s))};
  }
  static __device__ __forceinline__ double value(V v) { return (double)v.h + (double)v.l; }
};

// <A|B> of two MPS views with end bonds 1, the transfer matrices
// accumulated as OvAcc<T> (8 bytes an entry) in the (tmp, mat) pair.
template <typename T, int K, int DM, typename FA, typename FB>
__device__ double mps_overlap(WarpWS<T, K, DM>& ws, int h, FA sa, FB sb, int lane) {
  using Acc = OvAcc<T>;
  using V = typename Acc::V;
  static_assert(sizeof(V) == sizeof(double), "transfer matrices of 8-byte entries");
  V* E = reinterpret_cast<V*>(ws.tmp);
  V* F = E + 2 * DM * DM;             // E <= (2D x D), F <= D x 2 x 2D
  if (lane == 0) E[0] = Acc::one();
  int ea = 1, eb = 1;
  __syncwarp();
  for (int s = 0; s < h; ++s) {
    const SiteRef<T> A = sa(s), B = sb(s);
    // F[b][p][c] = sum_a E[a][b] A(a, p, c)
    const int nF = eb * 2 * A.nb;
    const FastDiv dA(A.nb);
    for (int e = lane; e < nF; e += 32) {
      const int q = dA.quo(e), cc = e - q * A.nb, b = q >> 1, p = q & 1;
      V acc = Acc::zero();
      for (int a = 0; a < ea; ++a) acc = Acc::mac(acc, E[a * eb + b], A.at(a, p, cc));
      F[e] = acc;
    }
    __syncwarp();
    // E'[c][d] = sum_{b,p} F[b][p][c] B(b, p, d)
    const int nE = A.nb * B.nb;
    const FastDiv dB(B.nb);
    for (int e = lane; e < nE; e += 32) {
      const int cc = dB.quo(e), dd = e - cc * B.nb;
      V acc = Acc::zero();
      for (int b = 0; b < eb; ++b)
        for (int p = 0; p < 2; ++p) acc = Acc::mac(acc, F[(b * 2 + p) * A.nb + cc], B.at(b, p, dd));
      E[e] = acc;
    }
    ea = A.nb;
    eb = B.nb;
    __syncwarp();
  }
  return Acc::value(E[0]);
}

// ---------------------------------------------------------------------------
// Block geometry in the rotated frame of direction ``dir`` (outgoing side).
struct Frame {
  int I, J, dir, h, ncols, r0, r1, c0, c1;
  int in_idx, a_idx, b_idx;      // message indices (-1 = border)
  int in_w, a_w, b_w;
  bool rev;                      // side messages consumed in reverse site order
  __device__ __forceinline__ void node(int t, int s, int* i, int* j) const {
    switch (dir) {
      case kDirR: *i = r0 + s; *j = c0 + t; break;
      case kDirL: *i = r0 + s; *j = c1 - 1 - t; break;
      case kDirD: *i = r0 + t; *j = c0 + s; break;
      default:    *i = r1 - 1 - t; *j = c0 + s; break;
    }
  }
};

template <typename T, int K>
__device__ __forceinline__ int msg_index(const Ctx<T, K>& c, int I, int J, int dir) {
  if (I < 0 || J < 0 || I >= c.g.nb || J >= c.g.nb) return -1;
  return c.msg_of[(I * c.g.nb + J) * 4 + dir];
}

template <typename T, int K>
__device__ Frame make_frame(const Ctx<T, K>& c, int I, int J, int dir) {
  Frame f;
  f.I = I; f.J = J; f.dir = dir;
  f.r0 = c.g.lo(I); f.r1 = c.g.hi(I); f.c0 = c.g.lo(J); f.c1 = c.g.hi(J);
  const int hr = f.r1 - f.r0, hc = f.c1 - f.c0;
  // Incoming messages: left = (I, J-1) sending R, right = (I, J+1) sending L,
  // top = (I-1, J) sending D, bottom = (I+1, J) sending U.
  const int left = J > 0 ? msg_index(c, I, J - 1, kDirR) : -1;
  const int right = J + 1 < c.g.nb ? msg_index(c, I, J + 1, kDirL) : -1;
  const int top = I > 0 ? msg_index(c, I - 1, J, kDirD) : -1;
  const int bot = I + 1 < c.g.nb ? msg_index(c, I + 1, J, kDirU) : -1;
  if (dir == kDirR || dir == kDirL) {
    f.h = hr; f.ncols = hc;
    f.in_idx = dir == kDirR ? left : right;
    f.a_idx = top; f.b_idx = bot;
    f.in_w = hr; f.a_w = hc; f.b_w = hc;
    f.rev = dir == kDirL;
  } else {
    f.h = hc; f.ncols = hr;
    f.in_idx = dir == kDirD ? top : bot;
    f.a_idx = left; f.b_idx = right;
    f.in_w = hc; f.a_w = hr; f.b_w = hr;
    f.rev = dir == kDirU;
  }
  return f;
}

// Apply column t of the rotated block with its two side-message sites.
template <typename T, int K, int DM>
__device__ __noinline__ void absorb(WarpWS<T, K, DM>& ws, const Ctx<T, K>& c, const Frame& f, int t, int lane) {
  const int h = f.h;
  // Node tensors of the column: wn[s][in][out][cp][cn].
  for (int e = lane; e < h * 16; e += 32) {
    const int s = e >> 4, q = e & 15;
    int i, j;
    f.node(t, s, &i, &j);
    ws.wn[e] = node_value<T>(c.frame, c.g.W, c.pI, c.pE, i, j, f.dir, (q >> 3) & 1, (q >> 2) & 1,
                             (q >> 1) & 1, q & 1);
  }
  const SiteRef<T> SA = msg_site(c, f.a_idx, f.a_w, t, f.rev);
  const SiteRef<T> SB = msg_site(c, f.b_idx, f.b_w, t, f.rev);
  __syncwarp();
  if (SA.na != ws.bond[0] || SB.na != ws.bond[h]) {   // end bonds must chain up
    if (lane == 0) atomicOr(c.cta_flags, kFlagCapacity);
    return;
  }
  const T* Wn = ws.wn;
  if (h == 1) {
    const int pl = ws.bond[0], pr = ws.bond[1];
    const int X = SA.nb, Y = SB.nb;
    const T* P = ws.psi[0];
    const FastDiv dY(Y);
    for (int e = lane; e < X * 2 * Y; e += 32) {
      const int q = dY.quo(e), yy = e - q * Y, xo = q >> 1, o = q & 1;
      T acc = 0;
      for (int a = 0; a < pl; ++a)
        for (int b = 0; b < pr; ++b)
          for (int i = 0; i < 2; ++i) {
            const T pv = P[(a * 2 + i) * pr + b];
            for (int cp = 0; cp < 2; ++cp)
              for (int cn = 0; cn < 2; ++cn)
                acc += SA.at(a, cp, xo) * pv * Wn[(((i * 2 + o) * 2 + cp) * 2) + cn] * SB.at(b, cn, yy);
          }
      ws.tmp[e] = acc;
    }
    __syncwarp();
    warp_copy(ws.psi[0], ws.tmp, X * 2 * Y, lane);
    if (lane == 0) { ws.bond[0] = X; ws.bond[1] = Y; }
    __syncwarp();
    return;
  }
  int nb_new[K + 1];
  nb_new[0] = SA.nb;
  for (int s = 1; s < h; ++s) nb_new[s] = 2 * ws.bond[s];
  nb_new[h] = SB.nb;
  for (int s = 0; s < h; ++s) {
    const int pl = ws.bond[s], pr = ws.bond[s + 1];
    const T* P = ws.psi[s];
    const T* Ws = Wn + s * 16;
    int total;
    if (s == 0) {
      const int X = SA.nb, nr = 2 * pr;
      total = X * 2 * nr;
      const FastDiv dn(nr);
      for (int e = lane; e < total; e += 32) {
        const int q = dn.quo(e), bn = e - q * nr, xo = q >> 1, o = q & 1, b = bn >> 1, cn = bn & 1;
        T acc = 0;
        for (int a = 0; a < pl; ++a)
          for (int cp = 0; cp < 2; ++cp) {
            const T sa = SA.at(a, cp, xo);
            if (sa == T(0)) continue;
            for (int i = 0; i < 2; ++i)
              acc += sa * P[(a * 2 + i) * pr + b] * Ws[((i * 2 + o) * 2 + cp) * 2 + cn];
          }
        ws.tmp[e] = acc;
      }
    } else if (s == h - 1) {
      const int Y = SB.nb;
      total = 2 * pl * 2 * Y;
      const FastDiv dY(Y);
      for (int e = lane; e < total; e += 32) {
        const int q = dY.quo(e), yy = e - q * Y, o = q & 1, pc = q >> 1, pp = pc >> 1, cp = pc & 1;
        T acc = 0;
        for (int i = 0; i < 2; ++i)
          for (int b = 0; b < pr; ++b) {
            const T pv = P[(pp * 2 + i) * pr + b];
            if (pv == T(0)) continue;
            for (int cn = 0; cn < 2; ++cn)
              acc += pv * Ws[((i * 2 + o) * 2 + cp) * 2 + cn] * SB.at(b, cn, yy);
          }
        ws.tmp[e] = acc;
      }
    } else {
      const int nr = 2 * pr;
      total = 2 * pl * 2 * nr;
      const FastDiv dn(nr);
      for (int e = lane; e < total; e += 32) {
        const int q = dn.quo(e), bn = e - q * nr, o = q & 1, pc = q >> 1;
        const int pp = pc >> 1, cp = pc & 1, b = bn >> 1, cn = bn & 1;
        T acc = 0;
        for (int i = 0; i < 2; ++i) acc += P[(pp * 2 + i) * pr + b] * Ws[((i * 2 + o) * 2 + cp) * 2 + cn];
        ws.tmp[e] = acc;
      }
    }
    __syncwarp();
    warp_copy(ws.psi[s], ws.tmp, total, lane);
    __syncwarp();
  }
  if (lane == 0)
    for (int s = 0; s <= h; ++s) ws.bond[s] = nb_new[s];
  __syncwarp();
}

// Load the incoming message (or the trivial border state) into psi.
template <typename T, int K, int DM>
__device__ __noinline__ void load_in(WarpWS<T, K, DM>& ws, const Ctx<T, K>& c, const Frame& f, int lane) {
  const int h = f.h;
  if (f.in_idx < 0) {
    for (int s = lane; s < h; s += 32) { ws.psi[s][0] = T(1); ws.psi[s][1] = T(0); }
    for (int s = lane; s <= h; s += 32) ws.bond[s] = 1;
  } else {
    const int8_t* dm = c.dims + f.in_idx * (K + 1);
    const T* base = c.arena + c.msg_off[f.in_idx];
    for (int s = 0; s < h; ++s) {
      const int n = dm[s] * 2 * dm[s + 1];
      warp_copy(ws.psi[s], base + msg_site_offset(s, h, c.D), n, lane);
    }
    for (int s = lane; s <= h; s += 32) ws.bond[s] = dm[s];
  }
  __syncwarp();
}

// Boundary-MPS contraction of one block towards ``dir`` (Eq. BP-update on
// blocks).  With readout the last column is not compressed (Lemma 1 read-out
// closes it exactly).  Returns the accumulated log scale.
template <typename T, int K, int DM>
__device__ __noinline__ double block_sweep(WarpWS<T, K, DM>& ws, const Ctx<T, K>& c, const Frame& f, bool readout,
                              int lane) {
  load_in(ws, c, f, lane);
  double log_scale = 0.0;
  for (int t = 0; t < f.ncols; ++t) {
    absorb(ws, c, f, t, lane);
    if (!readout || t + 1 < f.ncols) log_scale += compress(ws, c, f.h, lane, readout);
  }
  return log_scale;
}

// Damping (Remark 7): psi <- normalise(compress((1-eta) psi + eta old)).
template <typename T, int K, int DM>
__device__ __noinline__ void damp(WarpWS<T, K, DM>& ws, const Ctx<T, K>& c, int idx, int w, T eta, int lane) {
  const int8_t* od = c.dims + idx * (K + 1);
  const T* base = c.arena + c.msg_off[idx];
  const T a1 = T(1) - eta;
  if (w == 1) {
    const T* o = base;
    for (int e = lane; e < 2; e += 32) ws.psi[0][e] = a1 * ws.psi[0][e] + eta * o[e];
    __syncwarp();
  } else {
    int nb_new[K + 1];
    nb_new[0] = 1;
    nb_new[w] = 1;
    for (int s = 1; s < w; ++s) nb_new[s] = ws.bond[s] + od[s];
    for (int s = 0; s < w; ++s) {
      const int l1 = ws.bond[s], r1 = ws.bond[s + 1], l2 = od[s], r2 = od[s + 1];
      const T* P = ws.psi[s];
      const T* O = base + msg_site_offset(s, w, c.D);
      const int L = (s == 0) ? 1 : l1 + l2;
      const int R = (s == w - 1) ? 1 : r1 + r2;
      const int total = L * 2 * R;
      const FastDiv dR(R);
      for (int e = lane; e < total; e += 32) {
        const int q = dR.quo(e), b = e - q * R, a = q >> 1, p = q & 1;
        T v = 0;
        if (s == 0) {
          v = (b < r1) ? a1 * P[p * r1 + b] : eta * O[p * r2 + (b - r1)];
        } else if (s == w - 1) {
          v = (a < l1) ? P[a * 2 + p] : O[(a - l1) * 2 + p];
        } else {
          if (a < l1 && b < r1) v = P[(a * 2 + p) * r1 + b];
          else if (a >= l1 && b >= r1) v = O[((a - l1) * 2 + p) * r2 + (b - r1)];
        }
        ws.tmp[e] = v;
      }
      __syncwarp();
      warp_copy(ws.psi[s], ws.tmp, total, lane);
      __syncwarp();
    }
    if (lane == 0)
      for (int s = 0; s <= w; ++s) ws.bond[s] = nb_new[s];
    __syncwarp();
  }
  compress(ws, c, w, lane, false);
}

// Store psi as message idx (bond dims checked against the slot bounds).
template <typename T, int K, int DM>
__device__ __noinline__ void store_msg(WarpWS<T, K, DM>& ws, const Ctx<T, K>& c, int idx, int w, int lane) {
  bool fits = true;
  for (int s = 0; s < w; ++s)
    fits = fits && ws.bond[s] <= msg_bl(s, w, c.D) && ws.bond[s + 1] <= msg_br(s, w, c.D);
  if (!fits) {
    if (lane == 0) atomicOr(c.cta_flags, kFlagCapacity);
    return;
  }
  T* base = c.arena + c.msg_off[idx];
  for (int s = 0; s < w; ++s)
    warp_copy(base + msg_site_offset(s, w, c.D), ws.psi[s], ws.bond[s] * 2 * ws.bond[s + 1], lane);
  int8_t* dm = c.dims + idx * (K + 1);
  for (int s = lane; s <= w; s += 32) dm[s] = (int8_t)ws.bond[s];
  __syncwarp();
}

// ---------------------------------------------------------------------------
// The decoder kernel: one CTA per (syndrome, coset).
template <typename T, int K, int DM, int NW>
__global__ void __launch_bounds__(NW * 32) decode_kernel(KArgs<T> a) {
  extern __shared__ __align__(16) unsigned char smem[];
  using WS = WarpWS<T, K, DM>;
  const Geo g = a.geo;
  const int W = g.W, d = g.d, nb = g.nb, M = a.M;
  const int m = 2 * d * (d - 1);
  const CtaLayout Lo = cta_layout(g, M, K, NW, (int)sizeof(WS));
  uint8_t* synd = smem + Lo.synd;
  uint8_t* frame = smem + Lo.frame;
  int16_t* msg_of = reinterpret_cast<int16_t*>(smem + Lo.msg_of);
  int32_t* msg_off = reinterpret_cast<int32_t*>(smem + Lo.msg_off);
  int16_t* meta = reinterpret_cast<int16_t*>(smem + Lo.meta);      // message -> (I*nb+J)*4+dir
  int8_t* dims = reinterpret_cast<int8_t*>(smem + Lo.dims);
  int16_t* work = reinterpret_cast<int16_t*>(smem + Lo.work);     // [2][M]
  double* ovl = reinterpret_cast<double*>(smem + Lo.ovl);
  double* rlog = reinterpret_cast<double*>(smem + Lo.rlog);
  int* misc = reinterpret_cast<int*>(smem + Lo.misc);              // counter, flags, nwork0, nwork1, nedge, stop
  T* e0 = reinterpret_cast<T*>(smem + Lo.misc + 32);
  double* dsh = reinterpret_cast<double*>(smem + Lo.misc + 48);
  WS* wsa = reinterpret_cast<WS*>(smem + Lo.ws);

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const long long cta = blockIdx.x;
  const long long shot = cta >> 2;
  const int coset = (int)(cta & 3);
  T* arena = a.arena + cta * (long long)a.arena_elems;

  // Syndrome and the coset frame f_s * L (Algorithm 1; pure-error strings to
  // the right / bottom boundary, logicals on row 0 / column 0).
  for (int i = tid; i < m; i += NW * 32) synd[i] = a.synd[shot * m + i];
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
  // Message tables: directed block edges in (I, J, dir) order.
  if (tid == 0) {
    int idx = 0, off = 0, n0 = 0, n1 = 0;
    for (int I = 0; I < nb; ++I)
      for (int J = 0; J < nb; ++J)
        for (int dir = 0; dir < 4; ++dir) {
          const int key = (I * nb + J) * 4 + dir;
          if (g.has(I, J, dir)) {
            msg_of[key] = (int16_t)idx;
            meta[idx] = (int16_t)key;
            msg_off[idx] = off;
            off += msg_slot_elems(g.side_len(I, J, dir), a.D);
            if (((I + J) & 1) == 0) work[n0++] = (int16_t)idx;
            else work[M + n1++] = (int16_t)idx;
            ++idx;
          } else {
            msg_of[key] = -1;
          }
        }
    misc[0] = 0; misc[1] = 0; misc[2] = n0; misc[3] = n1;
    e0[0] = T(1); e0[1] = T(0);
    if (!dev_check(idx == M && n0 + n1 == M && off <= a.arena_elems, &misc[1])) misc[2] = misc[3] = 0;
  }
  __syncthreads();

  Ctx<T, K> c;
  c.g = g; c.D = a.D;
  c.cutoff2 = a.cutoff2_w;
  c.pI = a.pI_w; c.pE = a.pE_w;
  c.frame = frame; c.msg_of = msg_of; c.msg_off = msg_off; c.dims = dims;
  c.arena = arena; c.e0 = e0; c.cta_flags = &misc[1];

  // Remark 2: uniform initial messages, bond 1, every site (1, 1)/sqrt(2).
  const T u = (T)0.70710678118654752440;
  for (int idx = warp; idx < M; idx += NW) {
    const int key = meta[idx];
    const int w = g.side_len(key / 4 / nb, (key / 4) % nb, key & 3);
    T* base = arena + msg_off[idx];
    for (int s = lane; s < w; s += 32) {
      T* site = base + msg_site_offset(s, w, a.D);
      site[0] = u; site[1] = u;
    }
    for (int s = lane; s <= w; s += 32) dims[idx * (K + 1) + s] = 1;
  }
  __syncthreads();

  WS& ws = wsa[warp];
  double delta = 0.0;
  int it_done = 0;
  for (int it = 1; it <= a.max_iter && M > 0; ++it) {   // one block: no messages, no BP loop
    for (int color = 0; color < 2; ++color) {       // Remark 8
      const int nwork = misc[2 + color];
      const int16_t* lst = work + color * M;
      for (;;) {
        int item = 0;
        if (lane == 0) item = atomicAdd(&misc[0], 1);
        item = __shfl_sync(kFull, item, 0);
        if (item >= nwork) break;
        const int idx = lst[item];
        if (!dev_check(idx >= 0 && idx < M, &misc[1])) continue;
        const int key = meta[idx];
        const int I = key / 4 / nb, J = (key / 4) % nb, dir = key & 3;
        const Frame f = make_frame(c, I, J, dir);
        block_sweep(ws, c, f, false, lane);
        damp(ws, c, idx, f.h, a.eta_w, lane);
        const double o = mps_overlap(ws, f.h, [&](int s) { return psi_site(ws, s); },
                                     [&](int s) { return msg_site(c, idx, f.h, s, false); }, lane);
        store_msg(ws, c, idx, f.h, lane);
        if (lane == 0) ovl[idx] = o;
      }
      __syncthreads();
      if (tid == 0) misc[0] = 0;
      __syncthreads();
    }
    // Remark 4: Delta = sqrt(sum_i 2 - 2 <m_i^t | m_i^(t-1)>^2) / M.
    if (warp == 0) {
      double acc = 0.0;
      for (int i = lane; i < M; i += 32) acc += 2.0 - 2.0 * ovl[i] * ovl[i];
      acc = warp_sum(acc);
      if (lane == 0) dsh[0] = M > 0 ? sqrt(fmax(acc, 0.0)) / M : 0.0;
    }
    __syncthreads();
    delta = dsh[0];
    it_done = it;
    if (delta < a.delta0) break;
  }

  // Lemma 1 read-out: log P = sum_v log Z_v - sum_e log <m_uv | m_vu>.
  int nedge = 0;
  if (tid == 0) {
    for (int idx = 0; idx < M; ++idx) {
      const int dir = meta[idx] & 3;
      if (dir == kDirR || dir == kDirD) work[nedge++] = (int16_t)idx;
    }
    misc[4] = nedge;
    misc[0] = 0;
  }
  __syncthreads();
  nedge = misc[4];
  const int nblk = nb * nb;
  for (;;) {
    int item = 0;
    if (lane == 0) item = atomicAdd(&misc[0], 1);
    item = __shfl_sync(kFull, item, 0);
    if (item >= nblk + nedge) break;
    if (item < nblk) {
      const int I = item / nb, J = item % nb;
      const Frame f = make_frame(c, I, J, kDirR);
      const double ls = block_sweep(ws, c, f, true, lane);
      const int right = J + 1 < nb ? msg_index(c, I, J + 1, kDirL) : -1;
      if (!dev_check(right >= -1 && right < M, &misc[1])) continue;
      const double z = mps_overlap(ws, f.h, [&](int s) { return psi_site(ws, s); },
                                   [&](int s) { return msg_site(c, right, f.h, s, false); }, lane);
      if (lane == 0) {
        rlog[item] = ls + log(fabs(z));
        if (!(z > 0.0)) atomicOr(&misc[1], kFlagBlock);
      }
    } else {
      const int e = item - nblk;
      const int idx = work[e];
      if (!dev_check(idx >= 0 && idx < M, &misc[1])) continue;
      const int key = meta[idx];
      const int I = key / 4 / nb, J = (key / 4) % nb, dir = key & 3;
      const int other = dir == kDirR ? msg_index(c, I, J + 1, kDirL) : msg_index(c, I + 1, J, kDirU);
      if (!dev_check(other >= 0 && other < M, &misc[1])) continue;
      const int w = g.side_len(I, J, dir);
      const double o = mps_overlap(ws, w, [&](int s) { return msg_site(c, idx, w, s, false); },
                                   [&](int s) { return msg_site(c, other, w, s, false); }, lane);
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

}  // namespace bbp
