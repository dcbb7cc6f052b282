// Fused-block BP (Remark 9; the form the paper ran for k = 1, 2, 4): every
// k x k block acts as one vertex with four legs of dimension 2^k and the
// messages are dense vectors, so there is no MPS truncation at all.  Where
// the MPS form of Sec. III.D truncates nothing, both compute the same
// numbers.
//
// One CTA decodes G of the four cosets of one syndrome (G = 1, 2 or 4); all
// their messages live in shared memory (G x M dense vectors of 2^k).  The
// cosets share the network's geometry, and every node off the first row
// and column has the same Pauli frame in all of them (the logical strings
// of Sec. II run along row 0 and column 0), so a warp updates one directed
// block edge for all cosets of the CTA that are still iterating at once:
// index arithmetic, node tables and synchronisation are paid once for G
// vectors.  A coset whose Delta drops below delta0 is frozen (its messages
// and iteration count stay as they were), exactly as if it ran alone.
//
// A warp contracts one block with its incoming messages node by node on a
// dense state indexed by
//     [slot | a | rows of the chain | b | v]   (most to least significant bits)
// where slot picks the coset, v is the vertical leg inside the current
// column and a / b carry the top / bottom side message.  A side message
// m(t_0 .. t_{w-1}) is fed one leg per column through its exact copy / data /
// copy factorisation: the first floor(w/2) legs are recorded in a, the
// middle column contracts a with m and leaves in a the values expected for
// the remaining legs, which the last columns check off.  All dimensions are
// powers of two, so every index is a bit field.  Every loop is bounded and
// no CTA waits on another.
#pragma once

#include "bbp_kernels.cuh"

namespace bbp {

constexpr int kFusedK = 4;                 // block side of the learned warm start's messages
constexpr int kFusedVec = 1 << kFusedK;    // their dense length
constexpr int kFusedMaxG = 4;              // cosets per CTA

// Sizes of the kernels compiled for block sides up to K (K = 4 or 6): dense
// messages of 2^K entries and a per-coset state of at most 2^(2K) entries
// (a block with h rows and nc columns never holds more than h + nc bits:
// a and b together carry at most nc).
template <int K> struct FusedDim {
  static constexpr int vec = 1 << K;
  static constexpr int slot = 1 << (2 * K);
};

// Per-warp scratch for G cosets, carved from shared memory.
template <typename T>
struct FusedWS {   // (sizes for block side K: slot = FusedDim<K>::slot, vec = FusedDim<K>::vec)
  T* s0;   // state, G * slot
  T* s1;   // state, G * slot
  T* wn;   // node tensors, 16 per coset
  T* mt;   // side message A in consumption order, vec per coset (at k = 4 at least two)
  T* mb;   // side message B in consumption order, vec per coset (at k = 4 at least two)
};

// lean: every block update of the kernel runs in register form (k = 4,
// every block 4 x 4 or one node wide), so the state buffers only hold the
// outgoing vectors (16 entries per coset).
template <typename T, int K>
BBP_HD int fused_ws_slot(bool lean) {
  return lean ? FusedDim<K>::vec : FusedDim<K>::slot;
}

// Side-message vectors each of ws.mt / ws.mb holds: one per coset, and at
// k = 4 at least two (the two half-warp jobs of a register-form pass).
template <int K>
BBP_HD int fused_side_vecs(int G) { return K == 4 && G < 2 ? 2 : G; }

template <typename T, int K>
BBP_HD int fused_ws_bytes(int G, bool lean = false) {
  return align_up((int)sizeof(T) * (G * (2 * fused_ws_slot<T, K>(lean) + 16) +
                                    2 * fused_side_vecs<K>(G) * FusedDim<K>::vec),
                  16);
}

template <typename T, int K>
__device__ __forceinline__ FusedWS<T> fused_ws_at(unsigned char* base, int G, bool lean = false) {
  FusedWS<T> w;
  T* p = reinterpret_cast<T*>(base);
  const int slot = fused_ws_slot<T, K>(lean);
  w.s0 = p;
  w.s1 = p + G * slot;
  w.wn = p + 2 * G * slot;
  w.mt = w.wn + 16 * G;
  w.mb = w.mt + FusedDim<K>::vec * fused_side_vecs<K>(G);
  return w;
}

// Geometries whose every block has a register form at k = 4: the last
// block row / column is one node wide (W = 4 n + 1, every odd d).
BBP_HD bool register_form_only(const Geo& g) { return g.k == 4 && g.W % 4 == 1; }

// What a register-form block update needs beyond the messages and the qubit
// ids, fixed for a syndrome: the incoming message opposite the outgoing
// side, the side messages attached at the upper (s' = 0) and lower end of
// the chain, each an index or -1 on the grid border; the block's shape;
// flags (bit 0: the chain is read bottom to top, or for a one-node chain
// column 0 holds a check; bit 1: the side messages are consumed in reverse
// site order); and the qubit masks of the border vectors of the incoming /
// upper / lower side (bits 0-3 / 4-7 / 8-11, bit n - 1 - k set where leg k
// meets a qubit).
constexpr int kShapeNone = 0, kShapeQuad = 1, kShapeCol = 2, kShapeRow = 3, kShapeDot = 4;
constexpr int kQuadRev = 1, kQuadSideRev = 2;
struct QuadTask {
  int16_t in_idx, up_idx, lo_idx;
  uint16_t masks;
  uint8_t shape, flags;
};

// Shared-memory layout of one fused CTA.
struct FusedLayout {
  int synd, frame, msg_of, meta, work, ovl, rlog, misc, qdesc, qid, msgs, ws, ws_stride, total;
};

// gm: the messages live in a workspace slot of the CTA (always for k = 5,
// 6; on request for k <= 4), not in shared memory.
template <typename T, int K>
BBP_HD FusedLayout fused_layout(const Geo& g, int M, int nwarps, int G, bool gm = (K > 4), bool lean = false) {
  FusedLayout L;
  const int m = 2 * g.d * (g.d - 1);
  int o = 0;
  L.synd = o;   o = align_up(o + m, 16);
  L.frame = o;  o = align_up(o + G * g.W * g.W, 16);
  L.msg_of = o; o = align_up(o + 2 * g.nb * g.nb * 4, 16);
  L.meta = o;   o = align_up(o + 2 * M, 16);
  L.work = o;   o = align_up(o + 2 * 2 * M, 16);
  L.ovl = o;    o = align_up(o + (int)sizeof(T) * G * M, 16);
  L.rlog = o;   o = align_up(o + 8 * G * (g.nb * g.nb + M), 16);
  L.misc = o;   o = align_up(o + 128, 16);
  // 4 x 4 block updates (k = 4): a descriptor per message and the qubit
  // ids of each (coset, message), built once per syndrome.
  L.qdesc = o;  if (K == 4 && g.k == 4) o = align_up(o + (int)sizeof(QuadTask) * M, 16);
  L.qid = o;    if (K == 4 && g.k == 4) o = align_up(o + 2 * G * M, 16);
  L.msgs = o;   // the messages, unless they live in the workspace
  if (!gm) o = align_up(o + (int)sizeof(T) * FusedDim<K>::vec * G * M, 16);
  L.ws = o;
  L.ws_stride = fused_ws_bytes<T, K>(G, lean);
  o = align_up(o + nwarps * L.ws_stride, 16);
  L.total = o;
  return L;
}

template <typename T> struct Vec2;
template <> struct Vec2<float> { using type = float2; };
template <> struct Vec2<double> { using type = double2; };

// (Index fields below occupy disjoint bits; they are added rather than or-ed
// so that the compiler can advance the addresses instead of rebuilding them.)
//
// The data column of side message A with SD recorded legs and NF legs still
// to come (k = 5, 6: NF = 2), one coset, the message in registers: each
// lane takes groups hbv of (rows, b), reads in[a, hbv] for the 2^SD values
// of a once and writes out[a2, hbv, v] = sum_a m[a, v, a2] in[a, hbv].
template <typename T, int SD, int NF>
__device__ __forceinline__ void data_column_a(const T* mt, const T* cur, T* nxt, int ib, int ob, int hb,
                                              int lane) {
  using V2 = typename Vec2<T>::type;
  constexpr int NA = 1 << SD, NO = 1 << NF, NM = 1 << (SD + 1 + NF);
  T mr[NM];
#pragma unroll
  for (int i = 0; i < NM; ++i) mr[i] = mt[i];
  const int low = (1 << hb) - 1;
  for (int hbv = lane; hbv <= low; hbv += 32) {
    T x[NA];
#pragma unroll
    for (int a = 0; a < NA; ++a) x[a] = cur[ib + (a << hb) + hbv];
#pragma unroll
    for (int a2 = 0; a2 < NO; ++a2) {
      T s0 = T(0), s1 = T(0);
#pragma unroll
      for (int a = 0; a < NA; ++a) {
        s0 += mr[((a << 1) << NF) | a2] * x[a];
        s1 += mr[(((a << 1) | 1) << NF) | a2] * x[a];
      }
      V2 o;
      o.x = s0; o.y = s1;
      *reinterpret_cast<V2*>(nxt + 2 * (ob + (a2 << hb) + hbv)) = o;
    }
  }
}

// The data column of side message B (SD recorded legs, NF to come), one
// coset: each lane takes groups al of (a, rows), reads the 2^SD pairs
// in[al, b, v] once and writes out[al, b2] = sum_{b,v} m[b, v, b2] in[al, b, v].
template <typename T, int SD, int NF>
__device__ __forceinline__ void data_column_b(const T* mb, const T* cur, T* nxt, int ab0, int hah, int lane) {
  using V2 = typename Vec2<T>::type;
  constexpr int NB = 1 << SD, NO = 1 << NF, NM = 1 << (SD + 1 + NF);
  T mr[NM];
#pragma unroll
  for (int i = 0; i < NM; ++i) mr[i] = mb[i];
  for (int al = lane; al < (1 << hah); al += 32) {
    const int ah = ab0 + al;
    V2 x[NB];
#pragma unroll
    for (int b = 0; b < NB; ++b) x[b] = *reinterpret_cast<const V2*>(cur + (((ah << SD) + b) << 1));
#pragma unroll
    for (int b2 = 0; b2 < NO; ++b2) {
      T val = T(0);
#pragma unroll
      for (int b = 0; b < NB; ++b)
        val += mr[((b << 1) << NF) | b2] * x[b].x + mr[(((b << 1) | 1) << NF) | b2] * x[b].y;
      nxt[(ah << NF) | b2] = val;
    }
  }
}

__device__ __forceinline__ int bitrev(int x, int w) {
  return (int)(__brev((unsigned)x) >> (32 - w));
}

struct FState {
  int ab, h, bb, hv;   // bit widths of a, rows, b, v (per coset)
  __device__ __forceinline__ int bits() const { return ab + h + bb + hv; }
  __device__ __forceinline__ int size() const { return 1 << bits(); }
};

// Coset (0 .. G-1 within the CTA) held by slot s; slots are packed 2 bits each.
__device__ __forceinline__ int slot_coset(unsigned cos_of, int s) { return (int)((cos_of >> (2 * s)) & 3u); }

// The qubit table g[alpha][beta] = pi(f (+) (x, z)) of an interior qubit:
// one of x, z is the parity of its in/out legs (alpha), the other the
// parity of its chain legs (beta); alpha is z for horizontal-edge qubits
// swept along rows and for vertical-edge qubits swept along columns.
// Exactly one entry is pi(I): the one whose (x, z) equals the frame's
// (fx, fz), at index q = (alpha, beta) = (fz, fx) = the frame byte itself
// when alpha is z, and (fx, fz) = the byte with its two bits swapped when
// alpha is x.
template <typename T, int K>
__device__ __forceinline__ void qubit_table(const Ctx<T, K>& c, int qi, int qj, bool rowwise, T gt[4]) {
  const int fr = c.frame[qi * c.g.W + qj];
  const bool alpha_is_z = ((qi & 1) == 0) == rowwise;
  const int qi_id = alpha_is_z ? fr : (((fr & 1) << 1) | (fr >> 1));
#pragma unroll
  for (int q = 0; q < 4; ++q) gt[q] = q == qi_id ? c.pI : c.pE;
}

// Log of a product of positive factors, for the read-out (Lemma 1).  FP64
// sums the factors' logs; FP32 keeps the product as a float mantissa and a
// binary exponent and takes one FP64 log at the end (FP64 issues at 1/64
// of the FP32 rate here).  Used by one lane.
template <typename T> struct LogAcc;
template <> struct LogAcc<double> {
  double s = 0.0;
  __device__ __forceinline__ void mul(double x) { s += log(x); }
  __device__ __forceinline__ double value() const { return s; }
};
template <> struct LogAcc<float> {
  float m = 1.f;
  int e = 0;
  __device__ __forceinline__ void mul(float x) {
    int ex;
    m *= frexpf(x, &ex);
    e += ex;
    m = frexpf(m, &ex);
    e += ex;
  }
  __device__ __forceinline__ void mul(const LogAcc<float>& o) {
    int ex;
    m = frexpf(m * o.m, &ex);
    e += o.e + ex;
  }
  __device__ __forceinline__ double value() const { return log((double)m) + (double)e * 0.6931471805599453; }
};

// Contract block f (rotated so that f.dir points right) with its incoming
// dense messages for the n cosets of cos_of (messages of coset q at
// msgs + q * stride; c.frame is the frame of slot 0's coset and frames holds
// all G frames).  Leaves the outgoing vectors over the chain in ws.s0, slot
// s at s << h.  For the read-out (ls not null) every column's state is
// renormalised per coset and the norms taken out go to ls[slot] (lane 0).
template <typename T, int K>
__device__ __forceinline__ void fused_sweep_body(const FusedWS<T>& ws, const Ctx<T, K>& c, const T* msgs, int stride,
                                                 unsigned cos_of, int n, const uint8_t* frames, const Frame& f,
                                                 LogAcc<T>* ls, int lane) {
  using V2 = typename Vec2<T>::type;
  const int h = f.h, nc = f.ncols;
  T* cur = ws.s0;
  T* nxt = ws.s1;
  // Initial state: the message on the side opposite the outgoing one.
  for (int e = lane; e < (n << h); e += 32) {
    const int H = e & ((1 << h) - 1);
    const T* ms = msgs + slot_coset(cos_of, e >> h) * stride;
    cur[e] = f.in_idx >= 0 ? ms[f.in_idx * FusedDim<K>::vec + H] : (H == 0 ? T(1) : T(0));
  }
  // Side messages in consumption order.
  for (int e = lane; e < (n << nc); e += 32) {
    const int i = e & ((1 << nc) - 1);
    const int j = f.rev ? bitrev(i, nc) : i;
    const T* ms = msgs + slot_coset(cos_of, e >> nc) * stride;
    ws.mt[e] = f.a_idx >= 0 ? ms[f.a_idx * FusedDim<K>::vec + j] : T(0);
    ws.mb[e] = f.b_idx >= 0 ? ms[f.b_idx * FusedDim<K>::vec + j] : T(0);
  }
  __syncwarp();
  FState st{0, h, 0, 0};
  const int sd = nc >> 1;               // the column that holds the data site
  const int nf = nc - sd - 1;           // legs still expected after it
  const bool rowwise = f.dir == kDirR || f.dir == kDirL;
  const int WW = c.g.W * c.g.W;
  for (int t = 0; t < nc; ++t) {
    // Side message A: enters the column as its vertical leg v.  Output
    // entries come in pairs (v = 0, 1) sharing (slot, a, rows, b).
    {
      FState ns = st;
      ns.hv = 1;
      if (f.a_idx < 0) ns.ab = 0;
      else if (t < sd) ns.ab = st.ab + 1;
      else if (t == sd) ns.ab = nf;
      else ns.ab = st.ab - 1;
      const int np = n << (ns.bits() - 1);
      const int hb = h + st.bb;                        // bits of (rows, b)
      const int low = (1 << hb) - 1;
      if (K > 4 && t == sd && f.a_idx >= 0 && hb >= 5 && nf == 2 && (sd == 2 || sd == 3)) {
        for (int s = 0; s < n; ++s) {
          const int ib = s << (st.ab + hb), ob = s << (nf + hb);
          if (sd == 3) data_column_a<T, 3, 2>(ws.mt + (s << nc), cur, nxt, ib, ob, hb, lane);
          else data_column_a<T, 2, 2>(ws.mt + (s << nc), cur, nxt, ib, ob, hb, lane);
        }
      } else if (t == sd && f.a_idx >= 0 && hb >= 5 && nf <= 1) {
        // The data column, one coset at a time with its side message in
        // registers: each lane reads the 2^ab values in[a, rows, b] of its
        // (rows, b) once and writes all outputs (a2, v) of that group.
        const int na = 1 << st.ab;                     // st.ab = sd <= 2
        for (int s = 0; s < n; ++s) {
          T mr[16];
#pragma unroll
          for (int i = 0; i < 16; ++i) mr[i] = i < (1 << nc) ? ws.mt[(s << nc) + i] : T(0);
          const int ib = s << (st.ab + hb), ob = s << (nf + hb);
          for (int hbv = lane; hbv <= low; hbv += 32) {
            T x[4];
#pragma unroll
            for (int a = 0; a < 4; ++a) x[a] = a < na ? cur[ib + (a << hb) + hbv] : T(0);
            if (nf == 1) {
#pragma unroll
              for (int a2 = 0; a2 < 2; ++a2) {
                T s0 = T(0), s1 = T(0);
#pragma unroll
                for (int a = 0; a < 4; ++a) {
                  s0 += mr[(a << 2) | a2] * x[a];
                  s1 += mr[(((a << 1) | 1) << 1) | a2] * x[a];
                }
                V2 o;
                o.x = s0; o.y = s1;
                *reinterpret_cast<V2*>(nxt + 2 * (ob + (a2 << hb) + hbv)) = o;
              }
            } else {
              T s0 = T(0), s1 = T(0);
#pragma unroll
              for (int a = 0; a < 4; ++a) {
                s0 += mr[a << 1] * x[a];
                s1 += mr[(a << 1) | 1] * x[a];
              }
              V2 o;
              o.x = s0; o.y = s1;
              *reinterpret_cast<V2*>(nxt + 2 * (ob + hbv)) = o;
            }
          }
        }
      } else if (f.a_idx >= 0 && t < sd) {
        // Record v as a's new low bit: out[(slot, a, a'), hbv, v] = [a' = v]
        // in[(slot, a), hbv]; each input entry is read once and written to
        // both of its output pairs.
        const int nin = n << st.bits();
        constexpr int U = K > 4 ? 2 : 1;               // entries per lane and step (loads first)
        for (int e00 = lane; e00 < nin; e00 += 32 * U) {
          T xs[U];
          int es[U];
#pragma unroll
          for (int u = 0; u < U; ++u) {
            es[u] = U == 1 ? e00 : min(e00 + 32 * u, nin - 1);
            xs[u] = cur[es[u]];
          }
#pragma unroll
          for (int u = 0; u < U; ++u) {
            const int e = es[u];
            const int e0 = (((e >> hb) << 1) << hb) | (e & low);   // a' = 0
            V2 o0, o1;
            o0.x = xs[u]; o0.y = T(0);
            o1.x = T(0); o1.y = xs[u];
            *reinterpret_cast<V2*>(nxt + 2 * e0) = o0;
            *reinterpret_cast<V2*>(nxt + 2 * (e0 | (1 << hb))) = o1;
          }
        }
      } else if (K > 4 && f.a_idx >= 0 && t > sd) {
        // Move a's top bit into v: out[(slot, a), hbv, v] = in[(slot, v, a), hbv]
        // (two entries per lane and step, loads first).
        const int top = 1 << (st.ab - 1);
        for (int e20 = lane; e20 < np; e20 += 64) {
          V2 os[2];
          int es[2];
#pragma unroll
          for (int u = 0; u < 2; ++u) {
            const int e2 = min(e20 + 32 * u, np - 1);
            const int a2f = e2 >> hb, hbv = e2 & low;
            const int ai = ((a2f >> ns.ab) << st.ab) | (a2f & ((1 << ns.ab) - 1));
            os[u].x = cur[(ai << hb) | hbv];
            os[u].y = cur[((ai | top) << hb) | hbv];
            es[u] = e2;
          }
#pragma unroll
          for (int u = 0; u < 2; ++u) *reinterpret_cast<V2*>(nxt + 2 * es[u]) = os[u];
        }
      } else
      for (int e2 = lane; e2 < np; e2 += 32) {
        const int a2f = e2 >> hb, hbv = e2 & low;      // a2f = (slot, a); (rows, b) is shared by in and out
        V2 o;
        if (f.a_idx < 0) {
          o.x = cur[e2]; o.y = T(0);
        } else if (t < sd) {
          const T x = cur[((a2f >> 1) << hb) | hbv];
          if (a2f & 1) { o.x = T(0); o.y = x; } else { o.x = x; o.y = T(0); }
        } else if (t == sd) {
          const int s = a2f >> nf, a2 = a2f & ((1 << nf) - 1);
          const T* mt = ws.mt + (s << nc);
          const int ib = s << (st.ab + hb);
          T s0 = T(0), s1 = T(0);
          for (int a = 0; a < (1 << st.ab); ++a) {
            const T x = cur[ib | (a << hb) | hbv];
            s0 += mt[((a << 1) << nf) | a2] * x;
            s1 += mt[(((a << 1) | 1) << nf) | a2] * x;
          }
          o.x = s0; o.y = s1;
        } else {
          const int ai = ((a2f >> ns.ab) << st.ab) | (a2f & ((1 << ns.ab) - 1));
          o.x = cur[(ai << hb) | hbv];
          o.y = cur[((ai | (1 << (st.ab - 1))) << hb) | hbv];
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
    const int lnq = st.bits() - 2;                    // quads per coset, log2
    const int nq = n << lnq;
    // The base of a quad has the row bit P and bit 0 (v) clear, so the other
    // entries of the quad are at base + bitP, base + 1, base + bitP + 1.
    // k = 5, 6 (few warps per SM): each lane loads U quads before it stores
    // any; a lane past the end repeats the last quad (same values, same
    // addresses).  Quad g sits at base 4g - 2 (g & low); for k <= 4 the row
    // bit P is at most h + b <= 4 + 2 (b holds at most nc / 2 legs), so
    // 2^(P-1) divides 32, g & low stays lane & low and a lane's base grows by
    // exactly 128 per step.
    constexpr int U = K > 4 ? 4 : 1;
    for (int s = 0; s < h; ++s) {
      const int P = (h - 1 - s) + st.bb + 1;          // bit of the node's row in the index
      const int bitP = 1 << P;
      const int lowmask = (1 << (P - 1)) - 1;
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
          T gt[4];
          qubit_table(c, check_first ? mi : ni, check_first ? mj : nj, rowwise, gt);
          if (check_first) {
            // out[c, r, d] = sum_l in[c, l, v=c] g[l^r][c^d]; rows bits P (c) and P-1 (qubit).
            const int Q = P - 1, bitQ = 1 << Q, lowq = (1 << (Q - 1)) - 1;
            int bq = 4 * lane - 2 * (lane & lowq);   // k <= 4: base of quad g0, +128 per step
            // k <= 4: bit P <= 6 of the base does not change in steps of 128,
            // so the check bit and its table entries are fixed per lane.
            const int cbl = (bq >> P) & 1;
            const T l00 = cbl ? gt[1] : gt[0], l01 = cbl ? gt[0] : gt[1];
            const T l10 = cbl ? gt[3] : gt[2], l11 = cbl ? gt[2] : gt[3];
            for (int g0 = lane; g0 < nq; g0 += 32 * U, bq += 128) {
              int bs[U], cbs[U];
              T x0s[U], x1s[U];
#pragma unroll
              for (int u = 0; u < U; ++u) {
                const int g = U == 1 ? g0 : min(g0 + 32 * u, nq - 1);
                bs[u] = K <= 4 ? bq : ((g >> (Q - 1)) << (Q + 1)) | ((g & lowq) << 1);
                cbs[u] = K <= 4 ? cbl : (bs[u] >> P) & 1;
                x0s[u] = cur[bs[u] + cbs[u]];
                x1s[u] = cur[bs[u] + bitQ + cbs[u]];
              }
#pragma unroll
              for (int u = 0; u < U; ++u) {
                const int base = bs[u], cb = cbs[u];
                const T x0 = x0s[u], x1 = x1s[u];
                // g[a][c ^ d] by selects (a dynamic index would put gt in local memory)
                const T g00 = K <= 4 ? l00 : (cb ? gt[1] : gt[0]), g01 = K <= 4 ? l01 : (cb ? gt[0] : gt[1]);
                const T g10 = K <= 4 ? l10 : (cb ? gt[3] : gt[2]), g11 = K <= 4 ? l11 : (cb ? gt[2] : gt[3]);
                V2 o0, o1;
                o0.x = x0 * g00 + x1 * g10;   // r = 0, d = 0
                o0.y = x0 * g01 + x1 * g11;   // r = 0, d = 1
                o1.x = x0 * g10 + x1 * g00;   // r = 1, d = 0
                o1.y = x0 * g11 + x1 * g01;   // r = 1, d = 1
                *reinterpret_cast<V2*>(nxt + base) = o0;
                *reinterpret_cast<V2*>(nxt + (base + bitQ)) = o1;
              }
            }
          } else {
            // out[r, c, v] = [v = c] sum_{l,u} in[l, c, u] g[l^r][u^c]; qubit bit P, check bit P-1.
            const int cpos = P - 1;
            // k <= 4: bit P - 1 <= 5 of the base is fixed per lane (see above).
            const int cbl = ((4 * lane - 2 * (lane & lowmask)) >> cpos) & 1;
            const T l00 = cbl ? gt[1] : gt[0], l01 = cbl ? gt[0] : gt[1];
            const T l10 = cbl ? gt[3] : gt[2], l11 = cbl ? gt[2] : gt[3];
            for (int g0 = lane, bq = 4 * lane - 2 * (lane & lowmask); g0 < nq; g0 += 32 * U, bq += 128) {
              int bs[U];
              V2 i0s[U], i1s[U];
#pragma unroll
              for (int u = 0; u < U; ++u) {
                const int g = U == 1 ? g0 : min(g0 + 32 * u, nq - 1);
                bs[u] = K <= 4 ? bq : ((g >> (P - 1)) << (P + 1)) | ((g & lowmask) << 1);
                i0s[u] = *reinterpret_cast<const V2*>(cur + bs[u]);          // in[0][u=0,1]
                i1s[u] = *reinterpret_cast<const V2*>(cur + (bs[u] + bitP)); // in[1][u=0,1]
              }
#pragma unroll
              for (int u = 0; u < U; ++u) {
                const int base = bs[u];
                const int cb = K <= 4 ? cbl : (base >> cpos) & 1;
                const V2 i0 = i0s[u], i1 = i1s[u];
                // g[l ^ r][u ^ c]
                const T g00 = K <= 4 ? l00 : (cb ? gt[1] : gt[0]), g01 = K <= 4 ? l01 : (cb ? gt[0] : gt[1]);
                const T g10 = K <= 4 ? l10 : (cb ? gt[3] : gt[2]), g11 = K <= 4 ? l11 : (cb ? gt[2] : gt[3]);
                const T r0 = i0.x * g00 + i0.y * g01 + i1.x * g10 + i1.y * g11;
                const T r1 = i0.x * g10 + i0.y * g11 + i1.x * g00 + i1.y * g01;
                V2 o0, o1;
                o0.x = cb ? T(0) : r0; o0.y = cb ? r0 : T(0);
                o1.x = cb ? T(0) : r1; o1.y = cb ? r1 : T(0);
                *reinterpret_cast<V2*>(nxt + base) = o0;
                *reinterpret_cast<V2*>(nxt + (base + bitP)) = o1;
              }
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
        T gt[4];
        qubit_table(c, ni, nj, rowwise, gt);
        for (int g0 = lane, bq = 4 * lane - 2 * (lane & lowmask); g0 < nq; g0 += 32 * U, bq += 128) {
          int bs[U];
          V2 i0s[U], i1s[U];
#pragma unroll
          for (int u = 0; u < U; ++u) {
            const int g = U == 1 ? g0 : min(g0 + 32 * u, nq - 1);
            bs[u] = K <= 4 ? bq : ((g >> (P - 1)) << (P + 1)) | ((g & lowmask) << 1);
            i0s[u] = *reinterpret_cast<const V2*>(cur + bs[u]);          // in[0][0], in[0][1]
            i1s[u] = *reinterpret_cast<const V2*>(cur + (bs[u] + bitP)); // in[1][0], in[1][1]
          }
#pragma unroll
          for (int u = 0; u < U; ++u) {
            const V2 i0 = i0s[u], i1 = i1s[u];
            V2 o0, o1;
            o0.x = i0.x * gt[0] + i0.y * gt[1] + i1.x * gt[2] + i1.y * gt[3];
            o0.y = i0.x * gt[1] + i0.y * gt[0] + i1.x * gt[3] + i1.y * gt[2];
            o1.x = i0.x * gt[2] + i0.y * gt[3] + i1.x * gt[0] + i1.y * gt[1];
            o1.y = i0.x * gt[3] + i0.y * gt[2] + i1.x * gt[1] + i1.y * gt[0];
            *reinterpret_cast<V2*>(nxt + bs[u]) = o0;
            *reinterpret_cast<V2*>(nxt + (bs[u] + bitP)) = o1;
          }
        }
        __syncwarp();
        T* tmp = cur; cur = nxt; nxt = tmp;
        continue;
      }
      if (interior) {
        // Interior check: a copy tensor over four legs, out[r][d] = [r = d] in[r][r].
        for (int g0 = lane, bq = 4 * lane - 2 * (lane & lowmask); g0 < nq; g0 += 32 * U, bq += 128) {
          int bs[U];
          T i0x[U], i1y[U];
#pragma unroll
          for (int u = 0; u < U; ++u) {
            const int g = U == 1 ? g0 : min(g0 + 32 * u, nq - 1);
            bs[u] = K <= 4 ? bq : ((g >> (P - 1)) << (P + 1)) | ((g & lowmask) << 1);
            i0x[u] = reinterpret_cast<const V2*>(cur + bs[u])->x;
            i1y[u] = reinterpret_cast<const V2*>(cur + (bs[u] + bitP))->y;
          }
#pragma unroll
          for (int u = 0; u < U; ++u) {
            V2 o0, o1;
            o0.x = i0x[u]; o0.y = T(0);
            o1.x = T(0); o1.y = i1y[u];
            *reinterpret_cast<V2*>(nxt + bs[u]) = o0;
            *reinterpret_cast<V2*>(nxt + (bs[u] + bitP)) = o1;
          }
        }
        __syncwarp();
        T* tmp = cur; cur = nxt; nxt = tmp;
        continue;
      }
      // Border node: the general 16-entry tensor (missing legs carry 0).  On
      // row 0 and column 0 the frame, hence the tensor, depends on the coset.
      const bool per_coset = n > 1 && (ni == 0 || nj == 0);
      if (!per_coset) {
        if (lane < 16)
          ws.wn[lane] = node_value<T>(c.frame, c.g.W, c.pI, c.pE, ni, nj, f.dir, (lane >> 3) & 1,
                                      (lane >> 2) & 1, (lane >> 1) & 1, lane & 1);
      } else {
        for (int q = lane; q < 16 * n; q += 32)
          ws.wn[q] = node_value<T>(frames + slot_coset(cos_of, q >> 4) * WW, c.g.W, c.pI, c.pE, ni, nj, f.dir,
                                   (q >> 3) & 1, (q >> 2) & 1, (q >> 1) & 1, q & 1);
      }
      __syncwarp();
      T w[16];
#pragma unroll
      for (int q = 0; q < 16; ++q) w[q] = ws.wn[q];
      for (int g = lane; g < nq; g += 32) {
        if (per_coset) {
          const T* wq = ws.wn + ((g >> lnq) << 4);
#pragma unroll
          for (int q = 0; q < 16; ++q) w[q] = wq[q];
        }
        const int base = ((g >> (P - 1)) << (P + 1)) | ((g & lowmask) << 1);
        const V2 i0 = *reinterpret_cast<const V2*>(cur + base);          // (l=0,u=0), (l=0,u=1)
        const V2 i1 = *reinterpret_cast<const V2*>(cur + (base + bitP)); // (l=1,u=0), (l=1,u=1)
        V2 o0, o1;
        // w index: ((l*2 + r)*2 + u)*2 + d
        o0.x = i0.x * w[0] + i0.y * w[2] + i1.x * w[8] + i1.y * w[10];     // r=0, d=0
        o0.y = i0.x * w[1] + i0.y * w[3] + i1.x * w[9] + i1.y * w[11];     // r=0, d=1
        o1.x = i0.x * w[4] + i0.y * w[6] + i1.x * w[12] + i1.y * w[14];    // r=1, d=0
        o1.y = i0.x * w[5] + i0.y * w[7] + i1.x * w[13] + i1.y * w[15];    // r=1, d=1
        *reinterpret_cast<V2*>(nxt + base) = o0;
        *reinterpret_cast<V2*>(nxt + (base + bitP)) = o1;
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
      const int nt = n << ns.bits();
      const int hah = st.ab + h;                       // bits of (a, rows)
      if (K > 4 && t == sd && f.b_idx >= 0 && hah >= 5 && nf == 2 && (sd == 2 || sd == 3)) {
        for (int s = 0; s < n; ++s) {
          if (sd == 3) data_column_b<T, 3, 2>(ws.mb + (s << nc), cur, nxt, s << hah, hah, lane);
          else data_column_b<T, 2, 2>(ws.mb + (s << nc), cur, nxt, s << hah, hah, lane);
        }
        __syncwarp();
        T* tmp = cur; cur = nxt; nxt = tmp;
      } else if (t == sd && f.b_idx >= 0 && hah >= 5 && nf <= 1) {
        // The data column, one coset at a time with its side message in
        // registers: each lane reads the 2^bb pairs in[a, rows, b, v] of its
        // (a, rows) once and writes all outputs b2 of that group.
        const int nbb = 1 << st.bb;                    // st.bb = sd <= 2
        for (int s = 0; s < n; ++s) {
          T mr[16];
#pragma unroll
          for (int i = 0; i < 16; ++i) mr[i] = i < (1 << nc) ? ws.mb[(s << nc) + i] : T(0);
          for (int al = lane; al < (1 << hah); al += 32) {
            const int ah = (s << hah) + al;
            V2 x[4];
#pragma unroll
            for (int b = 0; b < 4; ++b) {
              if (b < nbb) {
                x[b] = *reinterpret_cast<const V2*>(cur + (((ah << st.bb) + b) << 1));
              } else {
                x[b].x = T(0); x[b].y = T(0);
              }
            }
            if (nf == 1) {
              V2 o;
              T val = T(0);
#pragma unroll
              for (int b = 0; b < 4; ++b) val += mr[(b << 2)] * x[b].x + mr[(((b << 1) | 1) << 1)] * x[b].y;
              o.x = val;
              val = T(0);
#pragma unroll
              for (int b = 0; b < 4; ++b) val += mr[(b << 2) | 1] * x[b].x + mr[(((b << 1) | 1) << 1) | 1] * x[b].y;
              o.y = val;
              *reinterpret_cast<V2*>(nxt + (ah << 1)) = o;
            } else {
              T val = T(0);
#pragma unroll
              for (int b = 0; b < 4; ++b) val += mr[b << 1] * x[b].x + mr[(b << 1) | 1] * x[b].y;
              nxt[ah] = val;
            }
          }
        }
        __syncwarp();
        T* tmp = cur; cur = nxt; nxt = tmp;
      } else if (K > 4 && f.b_idx >= 0 && t > sd) {
        // Close v against b's top bit: out[(slot, a, rows), b] = in[.., (0, b), v = 0]
        // + in[.., (1, b), v = 1] (two outputs per lane and step, loads first).
        const int top = 1 << (st.bb - 1);
        for (int e0 = lane; e0 < nt; e0 += 64) {
          T vs[2];
          int es[2];
#pragma unroll
          for (int u = 0; u < 2; ++u) {
            const int e = min(e0 + 32 * u, nt - 1);
            const int b2 = e & ((1 << ns.bb) - 1), ah = e >> ns.bb;
            vs[u] = cur[((ah << st.bb) | b2) << 1] + cur[(((ah << st.bb) | top | b2) << 1) | 1];
            es[u] = e;
          }
#pragma unroll
          for (int u = 0; u < 2; ++u) nxt[es[u]] = vs[u];
        }
        __syncwarp();
        T* tmp = cur; cur = nxt; nxt = tmp;
      } else if (!(f.b_idx >= 0 && t < sd)) {   // recording v as b's new low bit changes no index
        for (int e = lane; e < nt; e += 32) {
          T val;
          if (f.b_idx < 0) {
            val = cur[e << 1];                          // v = 0, b has no bits
          } else if (t == sd) {
            const int b2 = e & ((1 << ns.bb) - 1), ah = e >> ns.bb;   // (slot, a, rows)
            const T* mb = ws.mb + ((ah >> (st.ab + h)) << nc);
            val = T(0);
            for (int b = 0; b < (1 << st.bb); ++b) {
              const int bi = ((ah << st.bb) | b) << 1;
              val += mb[((b << 1) << nf) | b2] * cur[bi] + mb[(((b << 1) | 1) << nf) | b2] * cur[bi | 1];
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
    if (ls) {   // keep each coset's block value in range; the logs go to the read-out
      const int S = st.size();
#pragma unroll
      for (int q = 0; q < kFusedMaxG; ++q) {
        if (q < n) {
          T* cq = cur + q * S;
          T acc = 0;
          for (int e = lane; e < S; e += 32) acc += cq[e] * cq[e];
          acc = warp_sum(acc);
          const T nrm = xsqrt(acc);
          if (nrm > T(0)) {
            const T inv = T(1) / nrm;
            for (int e = lane; e < S; e += 32) cq[e] *= inv;
            if (lane == 0) ls[q].mul(nrm);
          }
        }
      }
      __syncwarp();
    }
  }
  if (cur != ws.s0) {
    for (int e = lane; e < (n << h); e += 32) ws.s0[e] = cur[e];
    __syncwarp();
  }
}

// Block sides up to 4: one out-of-line copy (the kernels that also hold the
// register forms keep their hot loop small in the instruction cache);
// block sides 5 and 6 inline it (their loop is this sweep).
template <typename T, int K>
__device__ __noinline__ void fused_sweep_call(const FusedWS<T>& ws, const Ctx<T, K>& c, const T* msgs, int stride,
                                              unsigned cos_of, int n, const uint8_t* frames, const Frame& f,
                                              LogAcc<T>* ls, int lane) {
  fused_sweep_body<T, K>(ws, c, msgs, stride, cos_of, n, frames, f, ls, lane);
}

template <typename T, int K>
__device__ __forceinline__ void fused_sweep(const FusedWS<T>& ws, const Ctx<T, K>& c, const T* msgs, int stride,
                                            unsigned cos_of, int n, const uint8_t* frames, const Frame& f,
                                            LogAcc<T>* ls, int lane) {
  if constexpr (K <= 4) fused_sweep_call<T, K>(ws, c, msgs, stride, cos_of, n, frames, f, ls, lane);
  else fused_sweep_body<T, K>(ws, c, msgs, stride, cos_of, n, frames, f, ls, lane);
}

// <x, y> over n <= 64 entries for the read-out, in the working precision.
template <typename T>
__device__ __forceinline__ T read_dot(const T* x, const T* y, int n, int lane) {
  T acc = lane < n ? x[lane] * y[lane] : T(0);
  if (n > 32 && lane + 32 < n) acc += x[lane + 32] * y[lane + 32];
  return warp_sum(acc);
}

// The per-message term 2 - 2 <x, y>^2 of Delta (Remark 4) for unit vectors
// x (new) and y (old), each held one entry per lane in a group of lanes.
// FP64 evaluates it as written.  FP32 evaluates the same quantity as
// s (2 - s / 2) with s = ||x - y||^2 (an identity for unit vectors): no
// cancellation when a message barely moved, and no FP64 instruction per
// update (FP64 issues at 1/64 of the FP32 rate here).
template <typename T> struct DeltaTerm;
template <> struct DeltaTerm<double> {
  static __device__ __forceinline__ double eval(double x, double y, int width) {
    const double o = group_sum(x * y, width);
    return fma(-2.0 * o, o, 2.0);
  }
  // A 64-entry vector held as entries lane and lane + 32.
  static __device__ __forceinline__ double eval2(double x0, double y0, double x1, double y1) {
    const double o = warp_sum(x0 * y0 + x1 * y1);
    return fma(-2.0 * o, o, 2.0);
  }
};
template <> struct DeltaTerm<float> {
  static __device__ __forceinline__ float eval(float x, float y, int width) {
    const float t = x - y;
    const float s = group_sum(t * t, width);
    return s * fmaf(-0.5f, s, 2.f);
  }
  static __device__ __forceinline__ float eval2(float x0, float y0, float x1, float y1) {
    const float t0 = x0 - y0, t1 = x1 - y1;
    const float s = warp_sum(t0 * t0 + t1 * t1);
    return s * fmaf(-0.5f, s, 2.f);
  }
};

// 1 / sqrt(s), 0 for s = 0: the scale of a unit-norm vector (Remark 3).
// FP32 takes the hardware reciprocal square root (a scale factor, whose last
// bit does not matter); FP64 the rounded square root and quotient.
__device__ __forceinline__ float inv_norm(float s) { return s > 0.f ? rsqrtf(s) : 0.f; }
__device__ __forceinline__ double inv_norm(double s) { return s > 0.0 ? 1.0 / sqrt(s) : 0.0; }
__device__ __forceinline__ float2 inv_norm(float2 s) { return make_float2(inv_norm(s.x), inv_norm(s.y)); }
__device__ __forceinline__ double2 inv_norm(double2 s) { return make_double2(inv_norm(s.x), inv_norm(s.y)); }

// Unit L2 norm (Remark 3) of the vector held by a group of lanes.
template <typename T>
__device__ __forceinline__ T group_normalize(T v, int width) {
  return v * inv_norm(group_sum(v * v, width));
}

// After a sweep: normalise the new messages in ws.s0 (Remark 3), damp them
// with the stored ones (Remark 7), normalise again, record each coset's
// Delta term in ovl[coset * M + idx] and store the result.  Entry e of the
// n x 2^h outgoing vectors sits in lane e % 32 (e < 64: G <= 4, h <= 4 or
// G = 1, h <= 6); a vector of 64 entries spans both halves.
template <typename T, int K>
__device__ __forceinline__ void fused_update(const FusedWS<T>& ws, T* msgs, int stride, unsigned cos_of, int n,
                                             int idx, int h, T eta, T one_m_eta, T* ovl, int M, int lane) {
  const int width = 1 << h, tot = n << h;
  if (K > 5 && width > 32) {
    // One vector of 64 entries (k = 6, one coset): entries lane and lane + 32
    // are reduced together.
    const int q = slot_coset(cos_of, 0);
    T* old0 = msgs + q * stride + idx * FusedDim<K>::vec + lane;
    T* old1 = old0 + 32;
    T x0 = ws.s0[lane], x1 = ws.s0[lane + 32];
    const T y0 = *old0, y1 = *old1;
    T nrm = xsqrt(warp_sum(x0 * x0 + x1 * x1));
    T inv = nrm > T(0) ? T(1) / nrm : T(0);
    x0 = fma(one_m_eta, x0 * inv, eta * y0);
    x1 = fma(one_m_eta, x1 * inv, eta * y1);
    nrm = xsqrt(warp_sum(x0 * x0 + x1 * x1));
    inv = nrm > T(0) ? T(1) / nrm : T(0);
    x0 *= inv;
    x1 *= inv;
    const T term = DeltaTerm<T>::eval2(x0, y0, x1, y1);
    *old0 = x0;
    *old1 = x1;
    if (lane == 0) ovl[q * M + idx] = term;
    __syncwarp();
    return;
  }
#pragma unroll
  for (int r = 0; r < 2; ++r) {
    if (r == 1 && tot <= 32) break;
    const int e = lane + 32 * r;
    const bool on = e < tot;
    const int q = on ? slot_coset(cos_of, e >> h) : 0;
    T* old = msgs + q * stride + idx * FusedDim<K>::vec + (e & (width - 1));
    T x = on ? ws.s0[e] : T(0);
    const T y = on ? *old : T(0);
    x = group_normalize(x, width);
    x = fma(one_m_eta, x, eta * y);
    x = group_normalize(x, width);
    const T term = DeltaTerm<T>::eval(x, y, width);
    if (on) {
      *old = x;
      if ((e & (width - 1)) == 0) ovl[q * M + idx] = term;
    }
  }
  __syncwarp();
}

// ---------------------------------------------------------------------------
// Block update of a 4 x 4 block in registers.
//
// Along a column of a 4 x 4 block checks and qubits alternate.  A check is a
// copy tensor (Sec. III.A), so its row leg, its two chain legs and (in the
// top or bottom row) the side message's leg are one and the same bit; a
// qubit's tensor pi(f + (x, z)) depends only on the parity of its in/out
// legs (alpha) and of its chain legs (beta): g[alpha][beta].  A column
// therefore acts on the 16-entry row state as two 2-point XOR convolutions
// (one per qubit row) whose beta is a parity of bits that the checks fix,
// and the side messages' legs are either tied to a row bit (check in the
// top / bottom row) or enter a qubit's beta.  Written out column by column
// this is a short sequence of butterflies over single row bits: a lane holds
// one (coset, row) entry of the state, with the still-open side-message legs
// in registers, and the butterflies exchange partners with warp shuffles (row
// bit s of the chain is lane bit 3 - s).  Two cosets per pass (lanes 0-15
// and 16-31).  Sides on the grid border have no message; they act as the
// product vector of their nodes' missing legs: ones for a check (a copy
// tensor over its remaining legs) and e_0 for a qubit (a missing leg carries
// 0), which is what the general node-by-node path computes there.

// g[0][be] and g[1][be] of a qubit whose pi(I) entry sits at id = (alpha, beta).
template <typename T>
__device__ __forceinline__ void qpair(int id, int be, T pI, T pE, T& g0, T& g1) {
  const bool hit = (id & 1) == be;
  const bool hi = (id >> 1) & 1;
  g0 = (hit && !hi) ? pI : pE;
  g1 = (hit && hi) ? pI : pE;
}

// Coefficient v (0 .. 3) of the qubit in field f of t = ids ^ lane pattern:
// pI where the field equals v.  With the lane's bit be at the field's beta
// position, the field is (alpha, beta ^ be): g[0][be], g[1][be] are
// v = 0, 2 and g[0][be ^ 1], g[1][be ^ 1] are v = 1, 3.
template <typename T>
__device__ __forceinline__ T qco(unsigned t, int f, unsigned v, T pI, T pE) {
  return ((t ^ (v << (2 * f))) & (3u << (2 * f))) == 0u ? pI : pE;   // constant masks: one logic op
}

template <typename T>
__device__ __forceinline__ T qval(int id, int al, int be, T pI, T pE) {
  return ((al << 1) | be) == id ? pI : pE;
}

template <typename T>
__device__ __forceinline__ T shx(T v, int mask) {
  return __shfl_xor_sync(kFull, v, mask);
}

// Shapes with a register form (k = 4): 4 x 4 blocks, and the blocks of one
// row or one column of nodes that the last block row / column leaves at odd
// d (4 x 1, 1 x 4, 1 x 1).
template <int K>
__device__ __forceinline__ int block_shape(const Frame& f) {
  if (K != 4) return kShapeNone;
  if (f.h == 4 && f.ncols == 4) return kShapeQuad;
  if (f.h == 4 && f.ncols == 1) return kShapeCol;
  if (f.h == 1 && f.ncols == 4) return kShapeRow;
  if (f.h == 1 && f.ncols == 1) return kShapeDot;
  return kShapeNone;
}

template <typename T, int K>
__device__ __forceinline__ QuadTask quad_task(const Frame& f) {
  QuadTask q;
  const int shape = block_shape<K>(f);
  const int h = f.h, nc = f.ncols;
  int i00, j00;
  f.node(0, 0, &i00, &j00);
  const bool chk0 = (i00 + j00) & 1;                         // column 0 starts with a check
  const bool rev = chk0 && h > 1;                            // chain read bottom to top
  const int up_s = rev ? h - 1 : 0, lo_s = rev ? 0 : h - 1;
  int qm_up = 0, qm_lo = 0, qm_in = 0;
  for (int u = 0; u < nc; ++u) {
    int i, j;
    f.node(u, up_s, &i, &j);
    if (!((i + j) & 1)) qm_up |= 1 << (nc - 1 - u);
    f.node(u, lo_s, &i, &j);
    if (!((i + j) & 1)) qm_lo |= 1 << (nc - 1 - u);
  }
  for (int u = 0; u < h; ++u) {
    int i, j;
    f.node(0, u, &i, &j);
    if (!((i + j) & 1)) qm_in |= 1 << (h - 1 - u);
  }
  q.in_idx = (int16_t)f.in_idx;
  q.up_idx = (int16_t)(rev ? f.b_idx : f.a_idx);
  q.lo_idx = (int16_t)(rev ? f.a_idx : f.b_idx);
  q.masks = (uint16_t)(qm_in | (qm_up << 4) | (qm_lo << 8));
  q.shape = (uint8_t)shape;
  q.flags = (uint8_t)((chk0 ? kQuadRev : 0) | (f.rev ? kQuadSideRev : 0));
  return q;
}

// The ids (2 bits each, pi(I) at (alpha, beta)) of the qubits of a block in
// register form, for one coset frame.  4 x 4: id[t][0] the upper, id[t][1]
// the lower qubit of column t (chain positions 0, 2 for even t and 1, 3 for
// odd t, read from the top or, reversed, from the bottom) at bits
// 2 (2t + u); 4 x 1: the qubits at s' = 0 and 2; 1 x 4: the qubits of
// columns 0 and 2, or 1 and 3; 1 x 1: the node (a qubit, or a check).
__device__ __forceinline__ int node_id(const Frame& f, const uint8_t* fr, int W, int t, int s) {
  const bool rowwise = f.dir == kDirR || f.dir == kDirL;
  int i, j;
  f.node(t, s, &i, &j);
  const int fv = fr[i * W + j];
  const bool alpha_is_z = ((i & 1) == 0) == rowwise;
  return alpha_is_z ? fv : (((fv & 1) << 1) | (fv >> 1));
}

__device__ __forceinline__ uint16_t quad_ids(const Frame& f, const uint8_t* fr, int W, const QuadTask& q) {
  const bool rev = (q.flags & kQuadRev) != 0;
  unsigned v = 0;
  if (q.shape == kShapeQuad) {
    for (int t = 0; t < 4; ++t)
      for (int u = 0; u < 2; ++u) {
        const int sq = (t & 1) + 2 * u;
        v |= (unsigned)node_id(f, fr, W, t, rev ? 3 - sq : sq) << (2 * (2 * t + u));
      }
  } else if (q.shape == kShapeCol) {
    v = (unsigned)node_id(f, fr, W, 0, rev ? 3 : 0) | ((unsigned)node_id(f, fr, W, 0, rev ? 1 : 2) << 2);
  } else if (q.shape == kShapeRow) {
    const int t0 = rev ? 1 : 0;
    v = (unsigned)node_id(f, fr, W, t0, 0) | ((unsigned)node_id(f, fr, W, t0 + 2, 0) << 2);
  } else if (q.shape == kShapeDot) {
    v = (unsigned)node_id(f, fr, W, 0, 0);
  }
  return (uint16_t)v;
}

// Four consecutive scalars at a 16-byte aligned address.
__device__ __forceinline__ void vcopy4(const float* p, float (&v)[4]) {
  const float4 q = *reinterpret_cast<const float4*>(p);
  v[0] = q.x; v[1] = q.y; v[2] = q.z; v[3] = q.w;
}
__device__ __forceinline__ void vcopy4(const double* p, double (&v)[4]) {
  const double2 q0 = reinterpret_cast<const double2*>(p)[0], q1 = reinterpret_cast<const double2*>(p)[1];
  v[0] = q0.x; v[1] = q0.y; v[2] = q1.x; v[3] = q1.y;
}
__device__ __forceinline__ void vstore4(float* p, const float (&v)[4]) {
  *reinterpret_cast<float4*>(p) = make_float4(v[0], v[1], v[2], v[3]);
}
__device__ __forceinline__ void vstore4(double* p, const double (&v)[4]) {
  reinterpret_cast<double2*>(p)[0] = make_double2(v[0], v[1]);
  reinterpret_cast<double2*>(p)[1] = make_double2(v[2], v[3]);
}

// Sum over aligned groups of 16 lanes (xor butterfly: every lane of a group
// gets the same bits).
// (Adds that are never contracted with the product feeding them, so that
// every kernel compiled from this gives the same bits.)
__device__ __forceinline__ float radd(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ double radd(double a, double b) { return __dadd_rn(a, b); }
template <typename T>
__device__ __forceinline__ T gsum16(T v) {
#pragma unroll
  for (int o = 8; o > 0; o >>= 1) v = radd(v, shx(v, o));
  return v;
}

// What the register forms need to finish a message update themselves (the
// steps of fused_update): the messages, the damping and the Delta terms.
template <typename T>
struct QuadUpd {
  T* msgs;
  T eta, one_m_eta;
  T* ovl;
  int M;
};

// The message update (the steps of fused_update: normalisation, Remark 3;
// damping with the stored message y, Remark 7; normalisation; the Delta
// term, Remark 4, FP32 as s (2 - s / 2) with s = ||x - y||^2, FP64 as
// 2 - 2 <x, y>^2) of coset cq's new 16-entry vector of message idx, held
// one entry per lane of a 16-lane group (entry Rn in this lane), from
// registers.
template <typename T, int K>
__device__ __forceinline__ void reg_update16(T out, bool on, int cq, int idx, int R, int Rn, int stride,
                                             const QuadUpd<T>& up) {
  T* old = up.msgs + cq * stride + idx * FusedDim<K>::vec + Rn;
  const T y = *old;
  T x = out * inv_norm(gsum16(out * out));
  x = fma(up.one_m_eta, x, up.eta * y);
  x = x * inv_norm(gsum16(x * x));
  T term;
  if constexpr (sizeof(T) == 4) {
    const T t = x - y;
    const T sq = gsum16(t * t);
    term = sq * fma(T(-0.5), sq, T(2));
  } else {
    const T o = gsum16(x * y);
    term = fma(T(-2) * o, o, T(2));
  }
  if (on) {
    *old = x;
    if (R == 0) up.ovl[cq * up.M + idx] = term;
  }
}

// The same for a 2-entry vector (v0, v1) that every lane of the group
// holds whole; the writer lane stores it.
template <typename T, int K>
__device__ __forceinline__ void reg_update2(T v0, T v1, bool on, int cq, int idx, bool writer, int stride,
                                            const QuadUpd<T>& up) {
  T* old = up.msgs + cq * stride + idx * FusedDim<K>::vec;
  const T y0 = old[0], y1 = old[1];
  T inv = inv_norm(radd(v0 * v0, v1 * v1));
  T x0 = fma(up.one_m_eta, v0 * inv, up.eta * y0), x1 = fma(up.one_m_eta, v1 * inv, up.eta * y1);
  inv = inv_norm(radd(x0 * x0, x1 * x1));
  x0 = x0 * inv;
  x1 = x1 * inv;
  T term;
  if constexpr (sizeof(T) == 4) {
    const T t0 = x0 - y0, t1 = x1 - y1;
    const T sq = radd(t0 * t0, t1 * t1);
    term = sq * fma(T(-0.5), sq, T(2));
  } else {
    const T o = radd(x0 * y0, x1 * y1);
    term = fma(T(-2) * o, o, T(2));
  }
  __syncwarp();   // every lane has read the stored message
  if (on && writer) {
    old[0] = x0;
    old[1] = x1;
    up.ovl[cq * up.M + idx] = term;
  }
}

// One half-warp job of the register forms: coset cq of message idx, with
// the message's descriptor qt and the coset's qubit ids idv.  Lanes
// 16 h .. 16 h + 15 of a warp run the job of their half h; a half without a
// job of the warp's shape repeats the other half's job with on = false (it
// keeps the warp's shuffles company and stores nothing).  slot: where the
// read-out takes the outgoing vector (ws.s0, slot << h); sside: the slot of
// the job's staged side messages in ws.mt / ws.mb (sside << 4).
struct HalfJob {
  QuadTask qt;
  int cq, idx, slot, sside;
  unsigned idv;
  bool on;
};

// The side messages of the n cosets of cos_of for one message (descriptor
// qt), staged for the quad and row forms at slot s << 4 of ws.mt / ws.mb:
// the same contents stage_sides gives one job.
template <typename T, int K>
__device__ __forceinline__ void stage_all_sides(const FusedWS<T>& ws, const T* msgs, int stride, const QuadTask& qt,
                                                unsigned cos_of, int n, int lane) {
  constexpr int VEC = FusedDim<K>::vec;
  const bool srev = qt.flags & kQuadSideRev;
  const int qm_up = (qt.masks >> 4) & 15, qm_lo = (qt.masks >> 8) & 15;
  for (int t = lane; t < (n << 3); t += 32) {            // a lane per (slot, side, quarter)
    const int sl = t >> 3, side = (t >> 2) & 1, i0 = (t & 3) << 2;
    const int midx = side ? qt.lo_idx : qt.up_idx;
    const int qm = side ? qm_lo : qm_up;
    T v[4];
    if (midx >= 0) {
      const T* ms = msgs + slot_coset(cos_of, sl) * stride + midx * VEC;
      if (srev) {
#pragma unroll
        for (int u = 0; u < 4; ++u) v[u] = ms[bitrev(i0 + u, 4)];
      } else {
        vcopy4(ms + i0, v);
      }
    } else {
#pragma unroll
      for (int u = 0; u < 4; ++u) v[u] = ((i0 + u) & qm) ? T(0) : T(1);
    }
    vstore4((side ? ws.mb : ws.mt) + (sl << 4) + i0, v);
  }
  __syncwarp();
}

// The side messages of a job in consumption order, the upper one (attached
// at s' = 0) in ws.mt and the lower one in ws.mb, half h at h << 4, entries
// 4 u .. 4 u + 3 per lane (lanes 0 .. 7 of the half; messages and buffers
// are 16-byte aligned).  A side on the grid border has no message: the
// product vector of its nodes' missing legs (1 for a check, e_0 for a
// qubit), bit n - 1 - t for node t.
template <typename T, int K>
__device__ __forceinline__ void stage_sides(const FusedWS<T>& ws, const T* msgs, int stride, const HalfJob& jb,
                                            int lane) {
  constexpr int VEC = FusedDim<K>::vec;
  const int t = lane & 15, hi = lane >> 4;
  if (t < 8) {
    const bool srev = jb.qt.flags & kQuadSideRev;
    const int side = t >> 2, i0 = (t & 3) << 2;
    const int midx = side ? jb.qt.lo_idx : jb.qt.up_idx;
    const int qm = side ? (jb.qt.masks >> 8) & 15 : (jb.qt.masks >> 4) & 15;
    T v[4];
    if (midx >= 0) {
      const T* ms = msgs + jb.cq * stride + midx * VEC;
      if (srev) {
#pragma unroll
        for (int u = 0; u < 4; ++u) v[u] = ms[bitrev(i0 + u, 4)];
      } else {
        vcopy4(ms + i0, v);
      }
    } else {
#pragma unroll
      for (int u = 0; u < 4; ++u) v[u] = ((i0 + u) & qm) ? T(0) : T(1);
    }
    vstore4((side ? ws.mb : ws.mt) + (hi << 4) + i0, v);
  }
  __syncwarp();
}

// Register form of a block of one column of 4 nodes (4 x 1 rotated): the
// column acts as in quad_pass's column 0, both side messages have one leg.
template <typename T, int K, bool UPD>
__device__ __forceinline__ void col_pass(const FusedWS<T>& ws, T pI, T pE, const T* msgs, int stride,
                                         const HalfJob& jb, int lane, const QuadUpd<T>& upd) {
  constexpr int VEC = FusedDim<K>::vec;
  const QuadTask& qt = jb.qt;
  const bool rev = qt.flags & kQuadRev;
  const int qm_in = qt.masks & 15, qm_up = (qt.masks >> 4) & 15, qm_lo = (qt.masks >> 8) & 15;
  const int R = lane & 15;
  const int r1 = (R >> 2) & 1, r3 = R & 1;
  const int Rn = rev ? bitrev(R, 4) : R;
  const T* mq = msgs + jb.cq * stride;
  // Ids against the lane's row bits (qco): the top qubit (field 0) with be
  // = r1, the lower one (field 1) with be = r1 ^ r3.
  const unsigned tq = jb.idv ^ (((unsigned)r1 * 5u) ^ ((unsigned)r3 * 4u));
  const T x = qt.in_idx >= 0 ? mq[qt.in_idx * VEC + Rn] : ((Rn & qm_in) ? T(0) : T(1));
  const T a0 = qt.up_idx >= 0 ? mq[qt.up_idx * VEC] : T(1);
  const T a1 = qt.up_idx >= 0 ? mq[qt.up_idx * VEC + 1] : (qm_up ? T(0) : T(1));
  const T bb = qt.lo_idx >= 0 ? mq[qt.lo_idx * VEC + r3] : ((r3 && qm_lo) ? T(0) : T(1));
  const T k0 = qco(tq, 1, 0u, pI, pE), k1 = qco(tq, 1, 2u, pI, pE);
  const T u = fma(k1, shx(x, 2), k0 * x);
  const T uf = shx(u, 8);
  const T h0 = qco(tq, 0, 0u, pI, pE), h1 = qco(tq, 0, 2u, pI, pE);   // top leg 0
  const T m0 = qco(tq, 0, 1u, pI, pE), m1 = qco(tq, 0, 3u, pI, pE);   // top leg 1
  const T out = bb * fma(a1, fma(m1, uf, m0 * u), a0 * fma(h1, uf, h0 * u));
  if constexpr (UPD) {
    reg_update16<T, K>(out, jb.on, jb.cq, jb.idx, R, Rn, stride, upd);
  } else {
    if (jb.on) ws.s0[(jb.slot << 4) | Rn] = out;
  }
  __syncwarp();
}

// Register form of a block of one row of 4 nodes (1 x 4 rotated): a lane
// takes one assignment of the four side legs that the two qubits see (the
// legs at the checks are tied to the row leg), the 16 lanes of a coset sum.
template <typename T, int K, bool UPD, bool STAGE>
__device__ __forceinline__ void row_pass(const FusedWS<T>& ws, T pI, T pE, const T* msgs, int stride,
                                         const HalfJob& jb, int lane, const QuadUpd<T>& upd) {
  constexpr int VEC = FusedDim<K>::vec;
  const QuadTask& qt = jb.qt;
  const bool chk0 = qt.flags & kQuadRev, srev = qt.flags & kQuadSideRev;
  const int qm_in = qt.masks & 15, qm_up = (qt.masks >> 4) & 15, qm_lo = (qt.masks >> 8) & 15;
  const int j = lane & 15, hi = lane >> 4;
  const T* mq = msgs + jb.cq * stride;
  if constexpr (STAGE) {                     // this job's side messages at slot hi
    const int jj = srev ? bitrev(j, 4) : j;
    ws.mt[(hi << 4) | j] = qt.up_idx >= 0 ? mq[qt.up_idx * VEC + jj] : ((j & qm_up) ? T(0) : T(1));
    ws.mb[(hi << 4) | j] = qt.lo_idx >= 0 ? mq[qt.lo_idx * VEC + jj] : ((j & qm_lo) ? T(0) : T(1));
    __syncwarp();
  }
  const int x0 = (j >> 3) & 1, x2 = (j >> 2) & 1, y0 = (j >> 1) & 1, y2 = j & 1;
  const T* mA = ws.mt + (jb.sside << 4);
  const T* mB = ws.mb + (jb.sside << 4);
  const int ia = (int)(jb.idv & 3u), ib = (int)((jb.idv >> 2) & 3u);
  const T in0 = qt.in_idx >= 0 ? mq[qt.in_idx * VEC] : T(1);
  const T in1 = qt.in_idx >= 0 ? mq[qt.in_idx * VEC + 1] : (qm_in ? T(0) : T(1));
  T part[2];
  if (!chk0) {
    // qubit, check, qubit, check: the lane's legs are (a0, a2, b0, b2);
    // the checks tie a1 = b1 to the row leg l1 and a3 = b3 to r.
#pragma unroll
    for (int r = 0; r < 2; ++r) part[r] = T(0);
#pragma unroll
    for (int l1 = 0; l1 < 2; ++l1) {
      T g0, g1;
      qpair(ia, x0 ^ y0, pI, pE, g0, g1);
      const T hh = l1 ? in0 * g1 + in1 * g0 : in0 * g0 + in1 * g1;
#pragma unroll
      for (int r = 0; r < 2; ++r)
        part[r] += hh * mA[(x0 << 3) | (l1 << 2) | (x2 << 1) | r] * mB[(y0 << 3) | (l1 << 2) | (y2 << 1) | r] *
                   qval(ib, l1 ^ r, x2 ^ y2, pI, pE);
    }
  } else {
    // check, qubit, check, qubit: the lane's legs are (a1, a3, b1, b3); the
    // checks tie a0 = b0 = l0 and a2 = b2 = l2.
    part[0] = part[1] = T(0);
#pragma unroll
    for (int l0 = 0; l0 < 2; ++l0)
#pragma unroll
      for (int l2 = 0; l2 < 2; ++l2) {
        const T w = (l0 ? in1 : in0) * mA[(l0 << 3) | (x0 << 2) | (l2 << 1) | x2] *
                    mB[(l0 << 3) | (y0 << 2) | (l2 << 1) | y2] * qval(ia, l0 ^ l2, x0 ^ y0, pI, pE);
        part[0] += w * qval(ib, l2, x2 ^ y2, pI, pE);
        part[1] += w * qval(ib, l2 ^ 1, x2 ^ y2, pI, pE);
      }
  }
#pragma unroll
  for (int m = 8; m >= 1; m >>= 1) {
    part[0] += shx(part[0], m);
    part[1] += shx(part[1], m);
  }
  if constexpr (UPD) {
    reg_update2<T, K>(part[0], part[1], jb.on, jb.cq, jb.idx, j == 0, stride, upd);
  } else {
    if (jb.on && j < 2) ws.s0[(jb.slot << 1) | j] = j ? part[1] : part[0];
  }
  __syncwarp();
}

// Register form of a single node (1 x 1): lane (l, a, b, r) of the node's
// legs, summed over l, a, b.
template <typename T, int K, bool UPD>
__device__ __forceinline__ void dot_pass(const FusedWS<T>& ws, T pI, T pE, const T* msgs, int stride,
                                         const HalfJob& jb, int lane, const QuadUpd<T>& upd) {
  constexpr int VEC = FusedDim<K>::vec;
  const QuadTask& qt = jb.qt;
  const bool chk = qt.flags & kQuadRev;
  const int qm_in = qt.masks & 15, qm_up = (qt.masks >> 4) & 15, qm_lo = (qt.masks >> 8) & 15;
  const int j = lane & 15;
  const int l = (j >> 3) & 1, a = (j >> 2) & 1, b = (j >> 1) & 1, r = j & 1;
  const T* mq = msgs + jb.cq * stride;
  const int id = (int)(jb.idv & 3u);
  const T mi = qt.in_idx >= 0 ? mq[qt.in_idx * VEC + l] : ((l && qm_in) ? T(0) : T(1));
  const T ma = qt.up_idx >= 0 ? mq[qt.up_idx * VEC + a] : ((a && qm_up) ? T(0) : T(1));
  const T mb = qt.lo_idx >= 0 ? mq[qt.lo_idx * VEC + b] : ((b && qm_lo) ? T(0) : T(1));
  const T nv = chk ? ((l == r && a == r && b == r) ? T(1) : T(0)) : qval(id, l ^ r, a ^ b, pI, pE);
  T v = mi * ma * mb * nv;
  v += shx(v, 8);
  v += shx(v, 4);
  v += shx(v, 2);
  if constexpr (UPD) {
    const T w = shx(v, 1);                     // the other entry
    reg_update2<T, K>(r ? w : v, r ? v : w, jb.on, jb.cq, jb.idx, j == 0, stride, upd);
  } else {
    if (jb.on && j < 2) ws.s0[(jb.slot << 1) | j] = v;
  }
  __syncwarp();
}

// The outgoing vector of a 4 x 4 block (f.h == f.ncols == 4) for a job,
// into ws.s0 at the job's slot (slot << 4), as fused_sweep leaves it; with
// UPD the message update itself instead (normalisation, Remark 3; damping,
// Remark 7; the Delta term, Remark 4), from registers.  Columns t = 0..3
// hold qubits at chain positions {0, 2} or {1, 3}, alternating from column
// to column.  Both node tensors are symmetric in their two chain legs, so
// reading the chain bottom to top (position s' = 3 - s, the side messages
// exchanged) turns a block whose column 0 starts with a check into one
// whose column 0 starts with a qubit; only that case is written out.
template <typename T, int K, bool UPD, bool STAGE>
__device__ __forceinline__ void quad_pass(const FusedWS<T>& ws, T pI, T pE, const T* msgs, int stride,
                                          const HalfJob& jb, int lane, const QuadUpd<T>& upd) {
  constexpr int VEC = FusedDim<K>::vec;
  const QuadTask& qt = jb.qt;
  if constexpr (STAGE) stage_sides<T, K>(ws, msgs, stride, jb, lane);   // at slot hi
  const bool rev = qt.flags & kQuadRev;
  const int qm_in = qt.masks & 15;
  const int R = lane & 15, hi = lane >> 4;
  const int r0 = (R >> 3) & 1, r1 = (R >> 2) & 1, r2 = (R >> 1) & 1, r3 = R & 1;
  const int Rn = rev ? bitrev(R, 4) : R;                     // the lane's row in the block's own order
  const int cq = jb.cq;
  const T* mA = ws.mt + (jb.sside << 4);
  const T* mB = ws.mb + (jb.sside << 4);
  // The qubit ids (field 2 t + u: the upper, u = 0, or lower qubit of
  // column t) against the lane's row bits: be of each field's first use,
  // r1 (0, 0), r1 ^ r3 (0, 1), r0 ^ r2 (1, 0), r2 (1, 1), r1 (2, 0),
  // r1 ^ r3 (2, 1), r0 ^ r2 (3, 0), r2 (3, 1); and r3 at the alpha bit of
  // (1, 1), whose coefficients the lanes of odd rows take swapped.
  const unsigned lq = ((unsigned)r0 * 0x1010u) ^ ((unsigned)r1 * 0x0505u) ^ ((unsigned)r2 * 0x5050u) ^
                      ((unsigned)r3 * 0x0484u);
  const unsigned tq = jb.idv ^ lq;
  const T x = qt.in_idx >= 0 ? msgs[cq * stride + qt.in_idx * VEC + Rn] : ((Rn & qm_in) ? T(0) : T(1));
  // Column 0 (qubits at 0, 2): the upper leg a0 is recorded, the lower leg
  // b0 is tied to r3 by the check at 3.
  T S0[2];
  {
    const T k0 = qco(tq, 1, 0u, pI, pE), k1 = qco(tq, 1, 2u, pI, pE);
    const T u = fma(k1, shx(x, 2), k0 * x);
    const T uf = shx(u, 8);
#pragma unroll
    for (int a0 = 0; a0 < 2; ++a0) {
      const T h0 = qco(tq, 0, (unsigned)a0, pI, pE), h1 = qco(tq, 0, 2u + a0, pI, pE);
      S0[a0] = fma(h1, uf, h0 * u);
    }
  }
  // Column 2's coefficients: the lower qubit (c2k0, c2k1) and the upper
  // one, g[l0 ^ r0][v ^ r1] for v = 0, 1.
  const T c2k0 = qco(tq, 5, 0u, pI, pE), c2k1 = qco(tq, 5, 2u, pI, pE);
  const T g00 = qco(tq, 4, 0u, pI, pE), g10 = qco(tq, 4, 2u, pI, pE);   // v = 0
  const T g01 = qco(tq, 4, 1u, pI, pE), g11 = qco(tq, 4, 3u, pI, pE);   // v = 1
  // Column 1 (qubits at 1, 3): a1 is tied to r0 by the check at 0; the
  // lower leg b1 is recorded.  S1[b0][b1] for one a0 at a time, folded
  // into column 2 at once.  Column 2 (qubits at 0, 2) is the data column
  // of both side messages: the upper leg v is summed against A[a0 a1 v e],
  // the lower leg w = r3 against B[b0 b1 w f].
  const T h0 = qco(tq, 2, 0u, pI, pE), h1 = qco(tq, 2, 2u, pI, pE);
  T kk0[2], kk1[2];                                        // [b1]: g[r3][r2 ^ b1], g[!r3][r2 ^ b1]
#pragma unroll
  for (int b1 = 0; b1 < 2; ++b1) {
    kk0[b1] = qco(tq, 3, (unsigned)b1, pI, pE);
    kk1[b1] = qco(tq, 3, 2u + b1, pI, pE);
  }
  // Column 3's upper leg e is tied to r0 by its check: only e = r0 of
  // A[a0 a1 v e] and of everything after it reaches this lane's output.
  T Y[2][2];                                               // [b0][b1], e = r0
#pragma unroll
  for (int a0 = 0; a0 < 2; ++a0) {
    T S1[2][2];
    {
      const T o = S0[a0], p = shx(o, 1);
      const T X0 = r3 ? p : o, X1 = r3 ? o : p;
      // The upper qubit's butterfly over r1 first: the lower qubit's
      // coefficients (r2, r3) are the same in both lanes it pairs.
      const T T0 = fma(h1, shx(X0, 4), h0 * X0), T1 = fma(h1, shx(X1, 4), h0 * X1);
#pragma unroll
      for (int b1 = 0; b1 < 2; ++b1) {
        S1[0][b1] = kk0[b1] * T0;
        S1[1][b1] = kk1[b1] * T1;
      }
    }
    // A0: row bit 0 kept (l0 = r0 = a1), A1: flipped (l0 = a1 = !r0); v
    // summed against column 2's upper qubit, e = r0.
    const T* ma = mA + (a0 << 3) + r0;
    const T A0 = fma(ma[(r0 << 2) + 2], g01, ma[r0 << 2] * g00);
    const T A1 = fma(ma[((r0 ^ 1) << 2) + 2], g11, ma[(r0 ^ 1) << 2] * g10);
#pragma unroll
    for (int b0 = 0; b0 < 2; ++b0)
#pragma unroll
      for (int b1 = 0; b1 < 2; ++b1) {
        const T s1 = S1[b0][b1];
        const T u = fma(c2k1, shx(s1, 2), c2k0 * s1);
        const T uf = shx(u, 8);
        Y[b0][b1] = a0 == 0 ? fma(A0, u, A1 * uf) : fma(A0, u, fma(A1, uf, Y[b0][b1]));
      }
  }
  T S2[2];                                                 // [ff], e = r0
  {
    const T* mb = mB + (r3 << 1);                          // B[b0 b1 r3 ff] at mb[4 (2 b0 + b1) + ff]
#pragma unroll
    for (int ff = 0; ff < 2; ++ff)
      S2[ff] = fma(mb[12 + ff], Y[1][1], fma(mb[8 + ff], Y[1][0], fma(mb[4 + ff], Y[0][1], mb[ff] * Y[0][0])));
  }
  // Column 3 (qubits at 1, 3): the upper leg e is tied to r0, the lower
  // leg f closes against B's expected value.
  T out;
  {
    const T z0 = S2[0], z1 = S2[1];
    const T p0 = shx(z0, 1), p1 = shx(z1, 1);
    const T k0 = qco(tq, 7, 0u, pI, pE), k1 = qco(tq, 7, 2u, pI, pE);
    const T m0 = qco(tq, 7, 1u, pI, pE), m1 = qco(tq, 7, 3u, pI, pE);
    const T uu = fma(m1, p1, fma(m0, z1, fma(k1, p0, k0 * z0)));
    const T g0 = qco(tq, 6, 0u, pI, pE), g1 = qco(tq, 6, 2u, pI, pE);
    out = fma(g1, shx(uu, 4), g0 * uu);
  }
  if constexpr (UPD) {
    reg_update16<T, K>(out, jb.on, cq, jb.idx, R, Rn, stride, upd);
  } else {
    if (jb.on) ws.s0[(jb.slot << 4) | Rn] = out;
  }
  __syncwarp();
}

// Sum over aligned groups of 8 lanes, every lane of a group getting the
// same bits.
template <typename T>
__device__ __forceinline__ T gsum8(T v) {
#pragma unroll
  for (int o = 4; o > 0; o >>= 1) v = radd(v, shx(v, o));
  return v;
}

// reg_update16 for a lane holding two entries of the 16-entry vector,
// out[q] at Rn[q] (the rows differing in row bit 0), over groups of 8
// lanes: the same sums in the same order (the first level of gsum16 adds a
// lane's value to its row-bit-0 partner's, here the lane's own pair).
template <typename T, int K>
__device__ __forceinline__ void reg_update16x2(const T (&out)[2], bool on, int cq, int idx, bool writer,
                                               const int (&Rn)[2], int stride, const QuadUpd<T>& up) {
  T* old = up.msgs + cq * stride + idx * FusedDim<K>::vec;
  const T y0 = old[Rn[0]], y1 = old[Rn[1]];
  const T i1 = inv_norm(gsum8(radd(out[0] * out[0], out[1] * out[1])));
  T x0 = out[0] * i1, x1 = out[1] * i1;
  x0 = fma(up.one_m_eta, x0, up.eta * y0);
  x1 = fma(up.one_m_eta, x1, up.eta * y1);
  const T i2 = inv_norm(gsum8(radd(x0 * x0, x1 * x1)));
  x0 = x0 * i2;
  x1 = x1 * i2;
  T term;
  if constexpr (sizeof(T) == 4) {
    const T t0 = x0 - y0, t1 = x1 - y1;
    const T sq = gsum8(radd(t0 * t0, t1 * t1));
    term = sq * fma(T(-0.5), sq, T(2));
  } else {
    const T o = gsum8(radd(x0 * y0, x1 * y1));
    term = fma(T(-2) * o, o, T(2));
  }
  if (on) {
    old[Rn[0]] = x0;
    old[Rn[1]] = x1;
    if (writer) up.ovl[cq * up.M + idx] = term;
  }
}

// quad_pass for up to four cosets of one message at once: lane (slot
// c = lane >> 3, j = lane & 7) holds rows R = 8 q + j, q = 0, 1, of coset
// slot c, so row bit r0 = q lives in registers (quad_pass's exchanges
// with lane ^ 8 become register swaps; its other shuffles stay inside the
// 8-lane group).  Slots >= n repeat slot 0 and store nothing.  The side
// messages are staged for slots 0 .. n - 1 (stage_all_sides).  Every value
// is quad_pass's, bit for bit.
template <typename T, int K, bool UPD>
__device__ __forceinline__ void quad_pass4(const FusedWS<T>& ws, T pI, T pE, const T* msgs, int stride,
                                           const QuadTask& qt, int idx, unsigned cos_of, int n, const uint16_t* qid,
                                           int qid_stride, int lane, const QuadUpd<T>& upd) {
  constexpr int VEC = FusedDim<K>::vec;
  const int c = lane >> 3, j = lane & 7;
  const bool on = c < n;
  const int sl = on ? c : 0;
  const int cq = slot_coset(cos_of, sl);
  const bool rev = qt.flags & kQuadRev;
  const int qm_in = qt.masks & 15;
  const int r1 = (j >> 2) & 1, r2 = (j >> 1) & 1, r3 = j & 1;
  int Rn[2];
#pragma unroll
  for (int q = 0; q < 2; ++q) Rn[q] = rev ? bitrev((q << 3) | j, 4) : ((q << 3) | j);
  const T* mA = ws.mt + (sl << 4);
  const T* mB = ws.mb + (sl << 4);
  // quad_pass's lane pattern at r0 = 0; r0 = 1 flips the beta bits of
  // fields 2 and 6 (be = r0 ^ r2), the only ones depending on r0.
  const unsigned tq = (unsigned)qid[cq * qid_stride] ^ (((unsigned)r1 * 0x0505u) ^ ((unsigned)r2 * 0x5050u) ^
                                                        ((unsigned)r3 * 0x0484u));
  unsigned tr[2];
  tr[0] = tq;
  tr[1] = tq ^ 0x1010u;
  T x[2];
#pragma unroll
  for (int q = 0; q < 2; ++q)
    x[q] = qt.in_idx >= 0 ? msgs[cq * stride + qt.in_idx * VEC + Rn[q]] : ((Rn[q] & qm_in) ? T(0) : T(1));
  // Column 0.
  T S0[2][2];                                              // [a0][q]
  {
    const T k0 = qco(tq, 1, 0u, pI, pE), k1 = qco(tq, 1, 2u, pI, pE);
    T u[2];
#pragma unroll
    for (int q = 0; q < 2; ++q) u[q] = fma(k1, shx(x[q], 2), k0 * x[q]);
#pragma unroll
    for (int a0 = 0; a0 < 2; ++a0) {
      const T h0 = qco(tq, 0, (unsigned)a0, pI, pE), h1 = qco(tq, 0, 2u + a0, pI, pE);
#pragma unroll
      for (int q = 0; q < 2; ++q) S0[a0][q] = fma(h1, u[q ^ 1], h0 * u[q]);
    }
  }
  const T c2k0 = qco(tq, 5, 0u, pI, pE), c2k1 = qco(tq, 5, 2u, pI, pE);
  const T g00 = qco(tq, 4, 0u, pI, pE), g10 = qco(tq, 4, 2u, pI, pE);
  const T g01 = qco(tq, 4, 1u, pI, pE), g11 = qco(tq, 4, 3u, pI, pE);
  T h0[2], h1[2];
#pragma unroll
  for (int q = 0; q < 2; ++q) {
    h0[q] = qco(tr[q], 2, 0u, pI, pE);
    h1[q] = qco(tr[q], 2, 2u, pI, pE);
  }
  T kk0[2], kk1[2];
#pragma unroll
  for (int b1 = 0; b1 < 2; ++b1) {
    kk0[b1] = qco(tq, 3, (unsigned)b1, pI, pE);
    kk1[b1] = qco(tq, 3, 2u + b1, pI, pE);
  }
  T Y[2][2][2];                                            // [b0][b1][q], e = r0 = q
#pragma unroll
  for (int a0 = 0; a0 < 2; ++a0) {
    T S1[2][2][2];                                         // [b0][b1][q]
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      const T o = S0[a0][q], p = shx(o, 1);
      const T X0 = r3 ? p : o, X1 = r3 ? o : p;
      const T T0 = fma(h1[q], shx(X0, 4), h0[q] * X0), T1 = fma(h1[q], shx(X1, 4), h0[q] * X1);
#pragma unroll
      for (int b1 = 0; b1 < 2; ++b1) {
        S1[0][b1][q] = kk0[b1] * T0;
        S1[1][b1][q] = kk1[b1] * T1;
      }
    }
    // A[a0 a1 v e] at mA[8 a0 + 4 a1 + 2 v + e]: row q takes e = q, A0 with
    // a1 = q and A1 with a1 = !q.
    T lo[4], hi4[4];
    vcopy4(mA + (a0 << 3), lo);                            // a1 = 0: [2 v + e]
    vcopy4(mA + (a0 << 3) + 4, hi4);                       // a1 = 1
    T A0[2], A1[2];
    A0[0] = fma(lo[2], g01, lo[0] * g00);
    A1[0] = fma(hi4[2], g11, hi4[0] * g10);
    A0[1] = fma(hi4[3], g01, hi4[1] * g00);
    A1[1] = fma(lo[3], g11, lo[1] * g10);
#pragma unroll
    for (int b0 = 0; b0 < 2; ++b0)
#pragma unroll
      for (int b1 = 0; b1 < 2; ++b1) {
        T u[2];
#pragma unroll
        for (int q = 0; q < 2; ++q) {
          const T s1 = S1[b0][b1][q];
          u[q] = fma(c2k1, shx(s1, 2), c2k0 * s1);
        }
#pragma unroll
        for (int q = 0; q < 2; ++q)
          Y[b0][b1][q] = a0 == 0 ? fma(A0[q], u[q], A1[q] * u[q ^ 1])
                                 : fma(A0[q], u[q], fma(A1[q], u[q ^ 1], Y[b0][b1][q]));
      }
  }
  T out[2];
  {
    const T* mb = mB + (r3 << 1);                          // B[b0 b1 r3 ff] at mb[4 (2 b0 + b1) + ff]
    const T k0 = qco(tq, 7, 0u, pI, pE), k1 = qco(tq, 7, 2u, pI, pE);
    const T m0 = qco(tq, 7, 1u, pI, pE), m1 = qco(tq, 7, 3u, pI, pE);
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      T S2[2];
#pragma unroll
      for (int ff = 0; ff < 2; ++ff)
        S2[ff] = fma(mb[12 + ff], Y[1][1][q], fma(mb[8 + ff], Y[1][0][q], fma(mb[4 + ff], Y[0][1][q],
                                                                             mb[ff] * Y[0][0][q])));
      const T z0 = S2[0], z1 = S2[1];
      const T p0 = shx(z0, 1), p1 = shx(z1, 1);
      const T uu = fma(m1, p1, fma(m0, z1, fma(k1, p0, k0 * z0)));
      const T g0 = qco(tr[q], 6, 0u, pI, pE), g1 = qco(tr[q], 6, 2u, pI, pE);
      out[q] = fma(g1, shx(uu, 4), g0 * uu);
    }
  }
  if constexpr (UPD) {
    reg_update16x2<T, K>(out, on, cq, idx, j == 0, Rn, stride, upd);
  } else {
    if (on) {
      ws.s0[(sl << 4) | Rn[0]] = out[0];
      ws.s0[(sl << 4) | Rn[1]] = out[1];
    }
  }
  __syncwarp();
}

// col_pass for up to four cosets of one message at once, lane and rows as
// in quad_pass4; every value is col_pass's, bit for bit.
template <typename T, int K, bool UPD>
__device__ __forceinline__ void col_pass4(const FusedWS<T>& ws, T pI, T pE, const T* msgs, int stride,
                                          const QuadTask& qt, int idx, unsigned cos_of, int n, const uint16_t* qid,
                                          int qid_stride, int lane, const QuadUpd<T>& upd) {
  constexpr int VEC = FusedDim<K>::vec;
  const int c = lane >> 3, j = lane & 7;
  const bool on = c < n;
  const int sl = on ? c : 0;
  const int cq = slot_coset(cos_of, sl);
  const bool rev = qt.flags & kQuadRev;
  const int qm_in = qt.masks & 15, qm_up = (qt.masks >> 4) & 15, qm_lo = (qt.masks >> 8) & 15;
  const int r1 = (j >> 2) & 1, r3 = j & 1;
  int Rn[2];
#pragma unroll
  for (int q = 0; q < 2; ++q) Rn[q] = rev ? bitrev((q << 3) | j, 4) : ((q << 3) | j);
  const T* mq = msgs + cq * stride;
  const unsigned tq = (unsigned)qid[cq * qid_stride] ^ (((unsigned)r1 * 5u) ^ ((unsigned)r3 * 4u));
  T x[2];
#pragma unroll
  for (int q = 0; q < 2; ++q)
    x[q] = qt.in_idx >= 0 ? mq[qt.in_idx * VEC + Rn[q]] : ((Rn[q] & qm_in) ? T(0) : T(1));
  const T a0 = qt.up_idx >= 0 ? mq[qt.up_idx * VEC] : T(1);
  const T a1 = qt.up_idx >= 0 ? mq[qt.up_idx * VEC + 1] : (qm_up ? T(0) : T(1));
  const T bb = qt.lo_idx >= 0 ? mq[qt.lo_idx * VEC + r3] : ((r3 && qm_lo) ? T(0) : T(1));
  const T k0 = qco(tq, 1, 0u, pI, pE), k1 = qco(tq, 1, 2u, pI, pE);
  const T h0 = qco(tq, 0, 0u, pI, pE), h1 = qco(tq, 0, 2u, pI, pE);
  const T m0 = qco(tq, 0, 1u, pI, pE), m1 = qco(tq, 0, 3u, pI, pE);
  T u[2], out[2];
#pragma unroll
  for (int q = 0; q < 2; ++q) u[q] = fma(k1, shx(x[q], 2), k0 * x[q]);
#pragma unroll
  for (int q = 0; q < 2; ++q) {
    const T uf = u[q ^ 1];
    out[q] = bb * fma(a1, fma(m1, uf, m0 * u[q]), a0 * fma(h1, uf, h0 * u[q]));
  }
  if constexpr (UPD) {
    reg_update16x2<T, K>(out, on, cq, idx, j == 0, Rn, stride, upd);
  } else {
    if (on) {
      ws.s0[(sl << 4) | Rn[0]] = out[0];
      ws.s0[(sl << 4) | Rn[1]] = out[1];
    }
  }
  __syncwarp();
}

// row_pass for up to four cosets of one message at once: lane (slot c,
// j = lane & 7) takes the side-leg assignments (x0, x2, y0, y2) with
// (x2, y0, y2) = j and x0 = 0, 1 in registers; the two are added first, as
// row_pass's first butterfly level adds them (x0 is its lane bit 3).  The
// side messages are staged for slots 0 .. n - 1.
template <typename T, int K, bool UPD>
__device__ __forceinline__ void row_pass4(const FusedWS<T>& ws, T pI, T pE, const T* msgs, int stride,
                                          const QuadTask& qt, int idx, unsigned cos_of, int n, const uint16_t* qid,
                                          int qid_stride, int lane, const QuadUpd<T>& upd) {
  constexpr int VEC = FusedDim<K>::vec;
  const int c = lane >> 3, j = lane & 7;
  const bool on = c < n;
  const int sl = on ? c : 0;
  const int cq = slot_coset(cos_of, sl);
  const bool chk0 = qt.flags & kQuadRev;
  const int qm_in = qt.masks & 15;
  const T* mq = msgs + cq * stride;
  const int x2 = (j >> 2) & 1, y0 = (j >> 1) & 1, y2 = j & 1;
  const T* mA = ws.mt + (sl << 4);
  const T* mB = ws.mb + (sl << 4);
  const unsigned idv = qid[cq * qid_stride];
  const int ia = (int)(idv & 3u), ib = (int)((idv >> 2) & 3u);
  const T in0 = qt.in_idx >= 0 ? mq[qt.in_idx * VEC] : T(1);
  const T in1 = qt.in_idx >= 0 ? mq[qt.in_idx * VEC + 1] : (qm_in ? T(0) : T(1));
  T pq[2][2];                                              // [x0][r]
#pragma unroll
  for (int x0 = 0; x0 < 2; ++x0) {
    T* part = pq[x0];
    if (!chk0) {
#pragma unroll
      for (int r = 0; r < 2; ++r) part[r] = T(0);
#pragma unroll
      for (int l1 = 0; l1 < 2; ++l1) {
        T g0, g1;
        qpair(ia, x0 ^ y0, pI, pE, g0, g1);
        const T hh = l1 ? in0 * g1 + in1 * g0 : in0 * g0 + in1 * g1;
#pragma unroll
        for (int r = 0; r < 2; ++r)
          part[r] += hh * mA[(x0 << 3) | (l1 << 2) | (x2 << 1) | r] * mB[(y0 << 3) | (l1 << 2) | (y2 << 1) | r] *
                     qval(ib, l1 ^ r, x2 ^ y2, pI, pE);
      }
    } else {
      part[0] = part[1] = T(0);
#pragma unroll
      for (int l0 = 0; l0 < 2; ++l0)
#pragma unroll
        for (int l2 = 0; l2 < 2; ++l2) {
          const T w = (l0 ? in1 : in0) * mA[(l0 << 3) | (x0 << 2) | (l2 << 1) | x2] *
                      mB[(l0 << 3) | (y0 << 2) | (l2 << 1) | y2] * qval(ia, l0 ^ l2, x0 ^ y0, pI, pE);
          part[0] += w * qval(ib, l2, x2 ^ y2, pI, pE);
          part[1] += w * qval(ib, l2 ^ 1, x2 ^ y2, pI, pE);
        }
    }
  }
  T part[2];
#pragma unroll
  for (int r = 0; r < 2; ++r) part[r] = pq[0][r] + pq[1][r];
#pragma unroll
  for (int m = 4; m >= 1; m >>= 1) {
    part[0] += shx(part[0], m);
    part[1] += shx(part[1], m);
  }
  if constexpr (UPD) {
    reg_update2<T, K>(part[0], part[1], on, cq, idx, j == 0, stride, upd);
  } else {
    if (on && j < 2) ws.s0[(sl << 1) | j] = j ? part[1] : part[0];
  }
  __syncwarp();
}

// Every iterating coset of one message in passes of two (cosets sp + h in
// half h), the side messages staged by the caller (stage_all_sides); the
// shape is dispatched once, outside the passes.
template <typename T, int K, int SHAPE, bool UPD>
__device__ __forceinline__ void msg_passes(const FusedWS<T>& ws, T pI, T pE, const T* msgs, int stride,
                                           const QuadTask& qt, int idx, unsigned cos_of, int n, const uint16_t* qid,
                                           int qid_stride, int lane, const QuadUpd<T>& upd) {
  if (n > 2) {                                // three or four cosets: one pass, 8 lanes each
    if constexpr (SHAPE == kShapeQuad) {
      quad_pass4<T, K, UPD>(ws, pI, pE, msgs, stride, qt, idx, cos_of, n, qid, qid_stride, lane, upd);
      return;
    } else if constexpr (SHAPE == kShapeCol) {
      col_pass4<T, K, UPD>(ws, pI, pE, msgs, stride, qt, idx, cos_of, n, qid, qid_stride, lane, upd);
      return;
    } else if constexpr (SHAPE == kShapeRow) {
      row_pass4<T, K, UPD>(ws, pI, pE, msgs, stride, qt, idx, cos_of, n, qid, qid_stride, lane, upd);
      return;
    }
  }
  const int hi = lane >> 4;
  for (int sp = 0; sp < n; sp += 2) {
    HalfJob jb;
    jb.on = sp + hi < n;
    const int sl = jb.on ? sp + hi : sp;
    jb.cq = slot_coset(cos_of, sl);
    jb.idx = idx;
    jb.slot = jb.sside = sl;
    jb.qt = qt;
    jb.idv = qid[jb.cq * qid_stride];
    if constexpr (SHAPE == kShapeQuad) quad_pass<T, K, UPD, false>(ws, pI, pE, msgs, stride, jb, lane, upd);
    else if constexpr (SHAPE == kShapeCol) col_pass<T, K, UPD>(ws, pI, pE, msgs, stride, jb, lane, upd);
    else if constexpr (SHAPE == kShapeRow) row_pass<T, K, UPD, false>(ws, pI, pE, msgs, stride, jb, lane, upd);
    else dot_pass<T, K, UPD>(ws, pI, pE, msgs, stride, jb, lane, upd);
  }
}

template <typename T, int K, bool UPD>
__device__ __forceinline__ void msg_register_form(int shape, const FusedWS<T>& ws, T pI, T pE, const T* msgs,
                                                  int stride, const QuadTask& qt, int idx, unsigned cos_of, int n,
                                                  const uint16_t* qid, int qid_stride, int lane,
                                                  const QuadUpd<T>& upd) {
  if (shape == kShapeQuad || shape == kShapeRow) stage_all_sides<T, K>(ws, msgs, stride, qt, cos_of, n, lane);
  if (shape == kShapeQuad)
    msg_passes<T, K, kShapeQuad, UPD>(ws, pI, pE, msgs, stride, qt, idx, cos_of, n, qid, qid_stride, lane, upd);
  else if (shape == kShapeCol)
    msg_passes<T, K, kShapeCol, UPD>(ws, pI, pE, msgs, stride, qt, idx, cos_of, n, qid, qid_stride, lane, upd);
  else if (shape == kShapeRow)
    msg_passes<T, K, kShapeRow, UPD>(ws, pI, pE, msgs, stride, qt, idx, cos_of, n, qid, qid_stride, lane, upd);
  else
    msg_passes<T, K, kShapeDot, UPD>(ws, pI, pE, msgs, stride, qt, idx, cos_of, n, qid, qid_stride, lane, upd);
}

// 2^-e exactly (0 <= e < 126), from the exponent bits.
template <typename T> __device__ __forceinline__ T pow2_neg(int e);
template <> __device__ __forceinline__ float pow2_neg<float>(int e) { return __int_as_float((127 - e) << 23); }
template <> __device__ __forceinline__ double pow2_neg<double>(int e) {
  return __longlong_as_double((long long)(1023 - e) << 52);
}

// Stable compaction by the whole CTA: items 0 .. n - 1 in order, emit(i, r)
// for every item with flag(i), r its rank among them; returns their count.
// scratch: NW ints of shared memory.  Every thread of the CTA calls it.
template <int NW, typename Flag, typename Emit>
__device__ __forceinline__ int cta_compact(int n, int* scratch, Flag flag, Emit emit) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  int base = 0;
  for (int c0 = 0; c0 < n; c0 += NW * 32) {
    const int i = c0 + tid;
    const bool f = i < n && flag(i);
    const unsigned b = __ballot_sync(kFull, f);
    if (lane == 0) scratch[warp] = __popc(b);
    __syncthreads();
    int off = base, tot = 0;
#pragma unroll
    for (int w = 0; w < NW; ++w) {
      const int cw = scratch[w];
      off += w < warp ? cw : 0;
      tot += cw;
    }
    if (f) emit(i, off + __popc(b & ((1u << lane) - 1u)));
    __syncthreads();
    base += tot;
  }
  return base;
}

// Message item of coset job j when every message has n jobs.
__device__ __forceinline__ int job_item(int j, int n) { return n == 4 ? j >> 2 : n == 2 ? j >> 1 : n == 1 ? j : j / 3; }

// A job of any register form (shape: the warp's, the same in both halves).
// STAGE: the quad and row forms stage the job's side messages themselves
// (at slot hi, sside = hi); else the caller has (stage_all_sides).
template <typename T, int K, bool UPD, bool STAGE>
__device__ __forceinline__ void reg_pass(int shape, const FusedWS<T>& ws, T pI, T pE, const T* msgs, int stride,
                                         const HalfJob& jb, int lane, const QuadUpd<T>& upd) {
  if (shape == kShapeQuad) quad_pass<T, K, UPD, STAGE>(ws, pI, pE, msgs, stride, jb, lane, upd);
  else if (shape == kShapeCol) col_pass<T, K, UPD>(ws, pI, pE, msgs, stride, jb, lane, upd);
  else if (shape == kShapeRow) row_pass<T, K, UPD, STAGE>(ws, pI, pE, msgs, stride, jb, lane, upd);
  else dot_pass<T, K, UPD>(ws, pI, pE, msgs, stride, jb, lane, upd);
}

// Resident CTAs per SM the register budget is sized for: with one coset per
// CTA, 32 warps per SM in FP32 (64 registers a thread) and 16 in FP64; with
// more cosets per CTA shared memory allows half as many; with k = 6 states
// (16 KB a buffer in FP32) the shared memory decides.
// LB > 0: the register-form-only kernel (lean buffers), sized for LB
// resident CTAs per SM.
template <typename T, int NW, int G, int K, int LB = 0> struct FusedMinBlocks {
  static constexpr int warps = K > 4 ? NW : (sizeof(T) == 4 ? 32 : 16) / (G > 1 ? 2 : 1);
  static constexpr int value = LB > 0 ? LB : (warps / NW > 1 ? warps / NW : 1);
};

// Cosets c0 .. c0 + G - 1 of one syndrome decoded by the whole CTA: syn_src
// holds the syndrome's m bytes and outputs go to row syn * 4 + coset.
// GM: the messages live in gmsgs, this CTA's slot in global memory (the slot
// is L2-resident and touched only a few times per block sweep); always for
// k = 5, 6.  Otherwise they live in shared memory and gmsgs is null.
template <typename T, int NW, int G, int K, bool GM, int LB = 0>
__device__ __forceinline__ void fused_item(const KArgs<T>& a, const Geo g, const int M, const uint8_t* syn_src,
                                           const long long syn, const int c0, unsigned char* smem, T* gmsgs) {
  const int W = g.W, d = g.d, nb = g.nb, WW = W * W;
  const int m = 2 * d * (d - 1);
  static_assert(K <= 4 || G == 1, "k = 6 states hold one coset per CTA");
  constexpr int VEC = FusedDim<K>::vec;
  constexpr bool kLean = LB > 0;
  static_assert(!kLean || K == 4, "register-form-only kernels are for k = 4");
  const FusedLayout Lo = fused_layout<T, K>(g, M, NW, G, GM, kLean);
  uint8_t* synd = smem + Lo.synd;
  uint8_t* frames = smem + Lo.frame;
  int16_t* msg_of = reinterpret_cast<int16_t*>(smem + Lo.msg_of);
  int16_t* meta = reinterpret_cast<int16_t*>(smem + Lo.meta);
  int16_t* work = reinterpret_cast<int16_t*>(smem + Lo.work);
  T* ovl = reinterpret_cast<T*>(smem + Lo.ovl);                // Delta term of each (coset, message)
  QuadTask* qdesc = reinterpret_cast<QuadTask*>(smem + Lo.qdesc);
  uint16_t* qid = reinterpret_cast<uint16_t*>(smem + Lo.qid);
  double* rlog = reinterpret_cast<double*>(smem + Lo.rlog);
  // misc: [0] counter, [1] cosets converged (bit q), [2..4] list sizes,
  // [8 + q] flags, [12 + q] iterations done; dsh[q]: the sum of coset q's
  // Delta terms at its last iteration.
  int* misc = reinterpret_cast<int*>(smem + Lo.misc);
  double* dsh = reinterpret_cast<double*>(smem + Lo.misc + 64);
  T* msgs = GM ? gmsgs : reinterpret_cast<T*>(smem + Lo.msgs);
  const int stride = M * VEC;                                // messages of one coset

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, hi = lane >> 4;
  const FusedWS<T> ws = fused_ws_at<T, K>(smem + Lo.ws + warp * Lo.ws_stride, G, kLean);

  for (int i = tid; i < m; i += NW * 32) synd[i] = syn_src[i];
  if (tid == 0) {
    misc[0] = 0; misc[1] = 0; misc[4] = 0; misc[7] = 0;
    for (int q = 0; q < 4; ++q) {
      misc[8 + q] = 0;
      misc[12 + q] = 0;
      dsh[q] = 0.0;
    }
  }
  // Pauli frame f_s L of each coset (Algorithm 1): the pure error's bits as
  // running XORs, a thread per row of horizontal-edge qubits for x (the
  // flagged sites to its left) and one per column for z (the flagged
  // plaquettes above), built in the last frame slot; then every coset's
  // frame, that one with the logical strings (X on row 0, Z on column 0).
  // Frames are zero off the horizontal-edge qubits.
  uint8_t* fr_s = frames + (G - 1) * WW;
  for (int e = tid; e < WW; e += NW * 32) fr_s[e] = 0;
  __syncthreads();
  if (tid < d) {
    int x = 0;
    for (int cc = 0; cc < d; ++cc) {
      fr_s[(2 * tid) * W + 2 * cc] = (uint8_t)x;
      if (cc < d - 1) x ^= synd[tid * (d - 1) + cc];
    }
  }
  __syncthreads();
  if (tid < d) {
    int z = 0;
    for (int r = 0; r < d; ++r) {
      fr_s[(2 * r) * W + 2 * tid] |= (uint8_t)(z << 1);
      if (r < d - 1) z ^= synd[d * (d - 1) + r * d + tid];
    }
  }
  __syncthreads();
  for (int pass = 0; pass < 2; ++pass) {      // the other slots first, then the last one in place
    const int q0 = pass == 0 ? 0 : G - 1, q1 = pass == 0 ? G - 1 : G;
    for (int e = tid; e < (q1 - q0) * WW; e += NW * 32) {
      const int q = q0 + e / WW, ij = e % WW;
      const int i = ij / W, j = ij - (ij / W) * W;
      const int coset = c0 + q;
      const bool bx = coset == 1 || coset == 2, bz = coset == 2 || coset == 3;
      const bool hq = ((i | j) & 1) == 0;
      frames[q * WW + ij] =
          (uint8_t)(fr_s[ij] ^ ((bx && hq && i == 0) ? 1 : 0) ^ ((bz && hq && j == 0) ? 2 : 0));
    }
    __syncthreads();
  }
  // Message table by stable compaction in (I, J, dir) order: each directed
  // block edge's index and key.  The first per-warp buffers serve as the
  // compactions' scratch (NW ints) until the message updates start.
  int* scr = reinterpret_cast<int*>(smem + Lo.ws);
  const int NK = nb * nb * 4;
  for (int key = tid; key < NK; key += NW * 32) msg_of[key] = -1;
  __syncthreads();
  auto has_key = [&](int key) { return g.has(key / 4 / nb, (key / 4) % nb, key & 3); };
  auto color_of = [&](int key) { return (key / 4 / nb + (key / 4) % nb) & 1; };
  const int nmsg = cta_compact<NW>(NK, scr, has_key, [&](int key, int r) {
    msg_of[key] = (int16_t)r;
    meta[r] = (int16_t)key;
  });

  Ctx<T, K> c;
  c.g = g; c.D = 0; c.cutoff2 = T(0);
  c.pI = a.pI_w; c.pE = a.pE_w;
  c.frame = frames; c.msg_of = msg_of; c.msg_off = nullptr; c.dims = nullptr;
  c.arena = nullptr; c.e0 = nullptr; c.cta_flags = &misc[8];

  const bool quads = K == 4 && g.k == 4;   // 4 x 4 blocks take quad_pass
  if (quads) {                              // their descriptors (geometry) and qubit ids (per coset)
    for (int idx = tid; idx < M; idx += NW * 32) {
      const int key = meta[idx];
      const Frame f = make_frame(c, key / 4 / nb, (key / 4) % nb, key & 3);
      QuadTask qt = quad_task<T, K>(f);
      if (!dev_check(qt.in_idx >= -1 && qt.in_idx < M && qt.up_idx >= -1 && qt.up_idx < M && qt.lo_idx >= -1 &&
                         qt.lo_idx < M && qt.shape <= kShapeDot,
                     &misc[8]))
        qt.shape = kShapeNone;
      qdesc[idx] = qt;
      for (int q = 0; q < G; ++q) qid[q * M + idx] = quad_ids(f, frames + q * WW, W, qt);
    }
    __syncthreads();
  }
  // Each colour's list (Remark 8): the messages of the register forms
  // first, grouped by shape (a warp pass pairs two coset jobs of one
  // shape), their count in misc[5 + colour]; then those of the node-by-node
  // path; key order within a group.  The order within a colour does not
  // matter for the results: its messages read only the other colour's.
  int ncol[2];
  for (int color = 0; color < 2; ++color) {
    int placed = 0, nreg = 0;
    const int ngroups = quads ? 5 : 1;
    for (int gi = 0; gi < ngroups; ++gi) {
      const int sh = gi < 4 ? kShapeQuad + gi : kShapeNone;
      placed += cta_compact<NW>(
          NK, scr,
          [&](int key) {
            return has_key(key) && color_of(key) == color && (!quads || qdesc[msg_of[key]].shape == sh);
          },
          [&](int key, int r) { work[color * M + placed + r] = msg_of[key]; });
      if (gi == 3) nreg = placed;
    }
    ncol[color] = placed;
    if (tid == 0) misc[5 + color] = quads ? nreg : 0;
  }
  if (tid == 0) {
    misc[2] = ncol[0];
    misc[3] = ncol[1];
    if (!dev_check(nmsg == M && ncol[0] + ncol[1] == M, &misc[8])) misc[2] = misc[3] = 0;
  }
  __syncthreads();

  // Remark 2: uniform messages of unit norm, unless initial messages are
  // given (learned warm start): those are renormalised on entry.
  if constexpr (K <= 4) {
    // A message per half-warp, two per half in flight (the proposals come
    // from HBM); the norm's sum in gsum16's order, which is group_sum's
    // over 32 lanes for vectors of at most 16 entries.
    const int sub = lane & 15;
    for (int b0 = 2 * warp; b0 < G * M; b0 += 4 * NW) {   // the same trip count in both halves (shuffles)
      const int q0 = b0 + hi;
      T v[2];
      int w[2];
      T* x[2];
      bool ok[2];
#pragma unroll
      for (int u = 0; u < 2; ++u) {
        const int qi = q0 + u * 2 * NW;
        ok[u] = qi < G * M;
        const int qq = ok[u] ? qi : 0;
        const int q = qq / M, idx = qq - q * M;
        const int key = meta[idx];
        w[u] = g.side_len(key / 4 / nb, (key / 4) % nb, key & 3);
        x[u] = msgs + q * stride + idx * VEC;
        v[u] = (a.init_msgs && ok[u] && sub < (1 << w[u]))
                   ? (T)a.init_msgs[((syn * 4 + c0 + q) * M + idx) * VEC + sub] : T(0);
      }
#pragma unroll
      for (int u = 0; u < 2; ++u) {
        const T nrm = xsqrt(gsum16(v[u] * v[u]));
        const bool uniform = !a.init_msgs || !(nrm > T(0));
        // 1 / sqrt(2^w): a power of two, times the rounded 1 / sqrt 2 for odd w.
        const T un = ((w[u] & 1) ? T(0.70710678118654752440) : T(1)) * pow2_neg<T>(w[u] >> 1);
        if (ok[u] && sub < VEC) x[u][sub] = uniform ? (sub < (1 << w[u]) ? un : T(0)) : v[u] * (T(1) / nrm);
      }
    }
  } else
  for (int qi = warp; qi < G * M; qi += NW) {
    const int q = qi / M, idx = qi - q * M;
    const int key = meta[idx];
    const int w = g.side_len(key / 4 / nb, (key / 4) % nb, key & 3);
    T* x = msgs + q * stride + idx * VEC;
    bool uniform = true;
    if (K <= 4 && a.init_msgs) {                    // proposals exist for k <= 4
      const float* src = a.init_msgs + ((syn * 4 + c0 + q) * M + idx) * VEC;
      const T v = lane < (1 << w) ? (T)src[lane] : T(0);
      const T nrm = xsqrt(group_sum(v * v, 32));
      uniform = !(nrm > T(0));
      if (!uniform && lane < VEC) x[lane] = v * (T(1) / nrm);
    }
    if (uniform) {                                   // no (or an unusable) proposal
      // 1 / sqrt(2^w): a power of two, times the rounded 1 / sqrt 2 for odd w.
      const T u = ((w & 1) ? T(0.70710678118654752440) : T(1)) * pow2_neg<T>(w >> 1);
      for (int i = lane; i < VEC; i += 32) x[i] = i < (1 << w) ? u : T(0);
    }
  }
  __syncthreads();

  const T eta = a.eta_w, one_m_eta = a.one_m_eta_w;
  unsigned act = (1u << G) - 1;                      // cosets still iterating
  for (int it = 1; it <= a.max_iter && M > 0 && act; ++it) {
    int n = 0;
    unsigned cos_of = 0;
#pragma unroll
    for (int q = 0; q < G; ++q)
      if ((act >> q) & 1u) { cos_of |= (unsigned)q << (2 * n); ++n; }
    c.frame = frames + (cos_of & 3u) * WW;
    const QuadUpd<T> upd{msgs, eta, one_m_eta, ovl, M};
    for (int color = 0; color < 2; ++color) {       // Remark 8
      const int nwork = misc[2 + color], nreg = misc[5 + color];
      const int16_t* lst = work + color * M;
      // The register forms.  Four cosets per CTA: a warp takes a message,
      // stages its side messages for every iterating coset once and runs
      // passes of two cosets (measured faster than pairing single coset
      // jobs, whose passes each stage and fetch for themselves).
      if constexpr (K == 4 && G == 4) {
        for (;;) {
          int item = 0;
          if (lane == 0) item = atomicAdd(&misc[0], 1);
          item = __shfl_sync(kFull, item, 0);
          if (item >= nreg) break;
          const int idx = lst[item];
          if (!dev_check(idx >= 0 && idx < M, &misc[8])) continue;
          const QuadTask qt = qdesc[idx];
          msg_register_form<T, K, true>(qt.shape, ws, c.pI, c.pE, msgs, stride, qt, idx, cos_of, n, qid + idx, M,
                                        lane, upd);
        }
      }
      // One or two cosets per CTA: coset jobs (message, coset), the n jobs of
      // a message consecutive, two per warp pass (one per half-warp), so that
      // no half idles when one coset of a message is iterating.
      const int njobs = nreg * n;
      for (;;) {
        if constexpr (K != 4 || G == 4) break;      // block sides 5, 6: no register forms
        int j0 = 0;
        if (lane == 0) j0 = atomicAdd(&misc[0], 2);
        j0 = __shfl_sync(kFull, j0, 0);
        if (j0 >= njobs) break;
        HalfJob jb;
        jb.on = j0 + hi < njobs;
        const int jm = jb.on ? j0 + hi : j0;       // a half without a job repeats the other's
        const int item = job_item(jm, n), sl = jm - item * n;
        jb.idx = lst[item];
        if (!dev_check(jb.idx >= 0 && jb.idx < M, &misc[8])) {
          jb.idx = 0;
          jb.on = false;
        }
        jb.cq = slot_coset(cos_of, sl);
        jb.slot = sl;
        jb.sside = hi;
        jb.qt = qdesc[jb.idx];
        jb.idv = qid[jb.cq * M + jb.idx];
        const int shp = jb.qt.shape;
        if (shp == __shfl_xor_sync(kFull, shp, 16)) {
          reg_pass<T, K, true, true>(shp, ws, c.pI, c.pE, msgs, stride, jb, lane, upd);
        } else {
          // The halves' jobs have different shapes (the boundary of two
          // shape groups): one shape at a time, the other half keeping company.
          for (int r = 0; r < 2; ++r) {
            HalfJob jr;
            jr.idx = __shfl_sync(kFull, jb.idx, 16 * r);
            jr.cq = __shfl_sync(kFull, jb.cq, 16 * r);
            jr.slot = 0;
            jr.sside = hi;
            jr.qt = qdesc[jr.idx];
            jr.idv = qid[jr.cq * M + jr.idx];
            jr.on = jb.on && hi == r;
            reg_pass<T, K, true, true>(jr.qt.shape, ws, c.pI, c.pE, msgs, stride, jr, lane, upd);
          }
        }
      }
      // The node-by-node path: whole messages, every coset at once.
      if constexpr (!kLean) {
        for (;;) {
          int item = 0;
          if (lane == 0) item = atomicAdd(&misc[7], 1);
          item = __shfl_sync(kFull, item, 0) + nreg;
          if (item >= nwork) break;
          const int idx = lst[item];
          if (!dev_check(idx >= 0 && idx < M, &misc[8])) continue;
          const int key = meta[idx];
          const Frame f = make_frame(c, key / 4 / nb, (key / 4) % nb, key & 3);
          fused_sweep(ws, c, msgs, stride, cos_of, n, frames, f, (LogAcc<T>*)nullptr, lane);
          fused_update<T, K>(ws, msgs, stride, cos_of, n, idx, f.h, eta, one_m_eta, ovl, M, lane);
        }
      } else {   // the host launches this kernel only where every block has a register form
        if (tid == 0 && nwork > nreg) atomicOr(&misc[8], kFlagCapacity);
      }
      __syncthreads();
      if (tid == 0) {
        misc[0] = 0;
        misc[7] = 0;
      }
      __syncthreads();
    }
    // Delta = sqrt(sum) / M < delta0 (Remark 4), compared as sum <
    // (delta0 M)^2 by the coset's warp, which sets the coset's bit in
    // misc[1]; the square root is taken once, after the loop.  The sum and
    // the compare run in working precision (FP32 terms, each already rounded
    // to FP32; no FP64 instruction in the loop of an FP32 kernel).
    if (warp < G && ((act >> warp) & 1u)) {
      T acc = T(0);
      for (int i = lane; i < M; i += 32) acc += ovl[warp * M + i];
      acc = warp_sum(acc);
      if (lane == 0) {
        const T d0sq = (T)((a.delta0 * M) * (a.delta0 * M));   // the exit threshold in working precision
        const T sum = acc > T(0) ? acc : T(0);
        dsh[warp] = (double)sum;
        misc[12 + warp] = it;
        if (sum < d0sq) atomicOr(&misc[1], 1 << warp);
      }
    }
    __syncthreads();
    act &= ~(unsigned)misc[1];
  }

  if (a.final_msgs)
    for (int e = tid; e < G * stride; e += NW * 32) {
      const int q = e / stride;
      a.final_msgs[(syn * 4 + c0 + q) * stride + (e - q * stride)] = (float)msgs[e];
    }

  // Lemma 1 read-out, all G cosets of a block (or edge) at once.
  // The undirected edges, each as its rightward / downward message, in
  // index order (the read-out's product order does not depend on the launch).
  const int nedge = cta_compact<NW>(
      M, scr, [&](int idx) { const int dir = meta[idx] & 3; return dir == kDirR || dir == kDirD; },
      [&](int idx, int r) { work[r] = (int16_t)idx; });
  if (tid == 0) misc[0] = 0;
  __syncthreads();
  const int nblk = nb * nb;
  const int per = nblk + nedge;
  const unsigned all = G == 1 ? 0u : (G == 2 ? 0x4u : 0xE4u);    // slot q holds coset q
  c.frame = frames;
  for (;;) {
    int item = 0;
    if (lane == 0) item = atomicAdd(&misc[0], 1);
    item = __shfl_sync(kFull, item, 0);
    if (item >= per) break;
    if (item < nblk) {
      // Z_v: the block's outgoing vector to the right, with every other
      // incoming message, closed against the message from the right.  Blocks
      // with a register form need no per-column rescaling (entries are sums
      // of products of node values and message entries, all at most 1).
      const int I = item / nb, J = item % nb;
      const Frame f = make_frame(c, I, J, kDirR);
      LogAcc<T> ls[kFusedMaxG];
      const int shape = quads ? block_shape<K>(f) : kShapeNone;
      if (shape != kShapeNone) {
        const QuadTask qt = quad_task<T, K>(f);
        uint16_t* idw = reinterpret_cast<uint16_t*>(ws.wn);
        if (lane < G) idw[lane] = quad_ids(f, frames + lane * WW, W, qt);
        __syncwarp();
        // Every coset q (slot q: the read-out's identity mapping `all`).
        msg_register_form<T, K, false>(shape, ws, c.pI, c.pE, msgs, stride, qt, 0, all, G, idw, 1, lane,
                                       QuadUpd<T>{});
      } else if constexpr (!kLean) {
        fused_sweep(ws, c, msgs, stride, all, G, frames, f, ls, lane);
      } else {
        if (lane == 0) atomicOr(&misc[8], kFlagCapacity);
      }
      const int right = J + 1 < nb ? msg_index(c, I, J + 1, kDirL) : -1;
      if (!dev_check(right >= -1 && right < M, &misc[8])) continue;
      // On the grid border the right side has no message.  The node-by-node
      // path gives missing legs the value 0, so only entry 0 survives; the
      // register forms treat every node as complete, so their vector is
      // closed against the border vector instead (1 at a check, whose copy
      // tensor spans its remaining legs; e_0 at a qubit).
      int qm_out = 0;
      if (right < 0 && shape != kShapeNone)
        for (int u = 0; u < f.h; ++u) {
          int i, j;
          f.node(f.ncols - 1, u, &i, &j);
          if (!((i + j) & 1)) qm_out |= 1 << (f.h - 1 - u);
        }
#pragma unroll
      for (int q = 0; q < G; ++q) {
        const T* mq = msgs + q * stride;
        T z;
        if (right >= 0) {
          z = read_dot(ws.s0 + (q << f.h), mq + right * VEC, 1 << f.h, lane);
        } else if (shape != kShapeNone) {
          const T v = (lane < (1 << f.h) && !(lane & qm_out)) ? ws.s0[(q << f.h) + lane] : T(0);
          z = warp_sum(v);
        } else {
          z = ws.s0[q << f.h];
        }
        if (lane == 0) {
          ls[q].mul(z < T(0) ? -z : z);
          if constexpr (sizeof(T) == 4) {   // the factor as mantissa and exponent
            reinterpret_cast<float*>(rlog + q * per + item)[0] = ls[q].m;
            reinterpret_cast<int*>(rlog + q * per + item)[1] = ls[q].e;
          } else {
            rlog[q * per + item] = ls[q].value();
          }
          if (!(z > T(0))) atomicOr(&misc[8 + q], kFlagBlock);
        }
      }
      __syncwarp();
    } else {
      const int idx = work[item - nblk];
      if (!dev_check(idx >= 0 && idx < M, &misc[8])) continue;
      const int key = meta[idx];
      const int I = key / 4 / nb, J = (key / 4) % nb, dir = key & 3;
      const int other = dir == kDirR ? msg_index(c, I, J + 1, kDirL) : msg_index(c, I + 1, J, kDirU);
      if (!dev_check(other >= 0 && other < M, &misc[8])) continue;
      const int w = g.side_len(I, J, dir);
#pragma unroll
      for (int q = 0; q < G; ++q) {
        const T* mq = msgs + q * stride;
        const T o = read_dot(mq + idx * VEC, mq + other * VEC, 1 << w, lane);
        if (lane == 0) {
          if constexpr (sizeof(T) == 4) {
            LogAcc<float> lo;
            lo.mul(fabsf(o));
            reinterpret_cast<float*>(rlog + q * per + item)[0] = lo.m;
            reinterpret_cast<int*>(rlog + q * per + item)[1] = lo.e;
          } else {
            rlog[q * per + item] = -log(fabs((double)o));
          }
          if (!(o > T(0))) atomicOr(&misc[8 + q], kFlagOverlap);
        }
      }
    }
  }
  __syncthreads();
  if (warp < G) {
    double acc = 0.0;
    if constexpr (sizeof(T) == 4) {
      // Products of the block values and of the edge overlaps in a fixed
      // order (lane-strided, then a fixed tree), one log each.
      LogAcc<float> pz, po;
      for (int i = lane; i < per; i += 32) {
        LogAcc<float> r;
        r.m = reinterpret_cast<const float*>(rlog + warp * per + i)[0];
        r.e = reinterpret_cast<const int*>(rlog + warp * per + i)[1];
        if (i < nblk) pz.mul(r); else po.mul(r);
      }
#pragma unroll
      for (int msk = 16; msk >= 1; msk >>= 1) {
        LogAcc<float> oz, oo;
        oz.m = __shfl_xor_sync(kFull, pz.m, msk);
        oz.e = __shfl_xor_sync(kFull, pz.e, msk);
        oo.m = __shfl_xor_sync(kFull, po.m, msk);
        oo.e = __shfl_xor_sync(kFull, po.e, msk);
        pz.mul(oz);
        po.mul(oo);
      }
      if (lane == 0) acc = pz.value() - po.value();   // FP64 logs on one lane (2 FP64 lanes a cycle per SM)
    } else {
      for (int i = lane; i < per; i += 32) acc += rlog[warp * per + i];
      acc = warp_sum(acc);
    }
    if (lane == 0) {
      const double dq = M > 0 ? sqrt(dsh[warp]) / M : 0.0;
      const int iq = misc[12 + warp];
      // Capacity and check failures are recorded on the first coset's word
      // and hold for every coset of the item.
      int fl = misc[8 + warp] | (misc[8] & (kFlagCapacity | kFlagCheck));
      if (!isfinite(acc)) fl |= kFlagNonfinite;
      if (!(dq < a.delta1)) fl |= kFlagUntrusted;
      const long long row = syn * 4 + c0 + warp;
      a.logp[row] = acc;
      a.delta[row] = dq;
      a.iters[row] = iq;
      a.flags[row] = fl;
    }
  }
}

// Messages in shared memory: one CTA per (syndrome, group of G cosets).
// Messages in the workspace (GM; always for k = 5, 6): a persistent grid,
// CTA b taking items b, b + gridDim.x, ... with its messages in slot b.
template <typename T, int NW, int G, int K, bool GM = (K > 4), int LB = 0>
__global__ void __launch_bounds__(NW * 32, (FusedMinBlocks<T, NW, G, K, LB>::value)) fused_kernel(KArgs<T> a) {
  extern __shared__ __align__(16) unsigned char smem[];
  constexpr int NG = 4 / G;
  const int m = 2 * a.geo.d * (a.geo.d - 1);
  if constexpr (GM) {
    T* gm = a.arena + (long long)blockIdx.x * a.slot_elems;
    for (long long item = blockIdx.x; item < a.n_items; item += gridDim.x) {
      const long long syn = item / NG;
      fused_item<T, NW, G, K, true, LB>(a, a.geo, a.M, a.synd + syn * m, syn, (int)(item % NG) * G, smem, gm);
      __syncthreads();
    }
  } else {
    const long long syn = blockIdx.x / NG;
    const int c0 = (int)(blockIdx.x % NG) * G;
    fused_item<T, NW, G, K, false, LB>(a, a.geo, a.M, a.synd + syn * m, syn, c0, smem, nullptr);
  }
}

// A batch of syndromes of different distances in one persistent launch: CTAs
// take (syndrome, coset group) items from a global counter in the order
// given (largest distance first balances the tail) until the batch is done.
struct MixedArgs {
  const int32_t* d_of;          // distance of each syndrome
  const int64_t* offsets;       // byte offset of each syndrome in the packed buffer
  const int32_t* order;         // syndrome order of the items, or null
  unsigned long long* counter;  // zero before the launch
  long long n_items;            // B * (4 / G)
  long long B;                  // syndromes
  int k, d_max;                 // shared memory is sized for d_max
};

// LB > 0: the register-form-only kernel (every distance of the batch odd).
template <typename T, int NW, int G, int K, bool GM = (K > 4), int LB = 0>
__global__ void __launch_bounds__(NW * 32, (FusedMinBlocks<T, NW, G, K, LB>::value))
    fused_mixed_kernel(KArgs<T> a, MixedArgs mx) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ long long item_sh;
  constexpr int NG = 4 / G;
  for (;;) {
    if (threadIdx.x == 0) item_sh = (long long)atomicAdd(mx.counter, 1ull);
    __syncthreads();
    const long long item = item_sh;
    __syncthreads();
    if (item >= mx.n_items) break;
    const long long shot = mx.order ? (long long)mx.order[item / NG] : (item / NG);
    const int c0 = (int)(item % NG) * G;
    // The batch comes from device buffers the host cannot read: a syndrome
    // index outside the batch is skipped, a distance outside 2..d_max (more
    // than the shared memory holds) gives its rows kFlagCheck and NaN.
    if (shot < 0 || shot >= mx.B) continue;
    const int d = mx.d_of[shot];
    if (d < 2 || d > mx.d_max) {
      if (threadIdx.x < G) {
        const long long row = shot * 4 + c0 + threadIdx.x;
        a.logp[row] = __longlong_as_double(0x7ff8000000000000ll);
        a.delta[row] = __longlong_as_double(0x7ff8000000000000ll);
        a.iters[row] = 0;
        a.flags[row] = kFlagCheck | kFlagNonfinite;
      }
      continue;
    }
    const Geo g = make_geo(d, mx.k);
    int M = 0, ae = 0;
    count_messages(g, 1, &M, &ae);
    fused_item<T, NW, G, K, GM, LB>(a, g, M, a.synd + mx.offsets[shot], shot, c0, smem,
                                    GM ? a.arena + (long long)blockIdx.x * a.slot_elems : nullptr);
    __syncthreads();
  }
}

}  // namespace bbp
