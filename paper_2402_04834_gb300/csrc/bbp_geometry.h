// Geometry of the blockBP decoder shared by the host API and the kernels:
// block partition (Algorithm 1, Remark 1), directed block edges (Sec. III.D),
// message slot sizes and the shared-memory layout of one CTA.
#pragma once

#include <stdint.h>

#ifdef __CUDACC__
#define BBP_HD __host__ __device__ __forceinline__
#else
#define BBP_HD inline
#endif

namespace bbp {

enum { kDirR = 0, kDirL = 1, kDirD = 2, kDirU = 3 };

BBP_HD int imin(int a, int b) { return a < b ? a : b; }
BBP_HD int imax(int a, int b) { return a > b ? a : b; }
BBP_HD int align_up(int x, int a) { return (x + a - 1) / a * a; }

// min(D, 2^e): the largest Schmidt rank across a cut with e two-level legs
// on its smaller side, capped at the bond dimension D.
BBP_HD int pow2cap(int e, int D) { return e >= 20 ? D : imin(D, 1 << e); }

// Bond bounds of site s of a w-site message (end bonds 1, physical dim 2).
BBP_HD int msg_bl(int s, int w, int D) { return pow2cap(imin(s, w - s), D); }
BBP_HD int msg_br(int s, int w, int D) { return pow2cap(imin(s + 1, w - s - 1), D); }

// Elements of a w-site message slot: sum over sites of bl * 2 * br.
BBP_HD int msg_slot_elems(int w, int D) {
  int e = 0;
  for (int s = 0; s < w; ++s) e += msg_bl(s, w, D) * 2 * msg_br(s, w, D);
  return e;
}

BBP_HD int msg_site_offset(int s, int w, int D) {
  int e = 0;
  for (int t = 0; t < s; ++t) e += msg_bl(t, w, D) * 2 * msg_br(t, w, D);
  return e;
}

struct Geo {
  int d, W, k, nb;
  BBP_HD int lo(int I) const { return I * k; }
  BBP_HD int hi(int I) const { return imin(I * k + k, W); }
  BBP_HD int len(int I) const { return hi(I) - lo(I); }
  BBP_HD bool has(int I, int J, int dir) const {
    switch (dir) {
      case kDirR: return J + 1 < nb;
      case kDirL: return J > 0;
      case kDirD: return I + 1 < nb;
      default: return I > 0;
    }
  }
  // Sites of the message crossing side ``dir`` of block (I, J).
  BBP_HD int side_len(int I, int J, int dir) const {
    return (dir == kDirR || dir == kDirL) ? len(I) : len(J);
  }
};

BBP_HD Geo make_geo(int d, int k) {
  Geo g;
  g.d = d;
  g.W = 2 * d - 1;
  g.k = k;
  g.nb = (g.W + k - 1) / k;
  return g;
}

// Number of directed block edges M and the message arena size of one
// (syndrome, coset), in elements.
BBP_HD void count_messages(const Geo& g, int D, int* M, int* arena_elems) {
  int m = 0, e = 0;
  for (int I = 0; I < g.nb; ++I)
    for (int J = 0; J < g.nb; ++J)
      for (int dir = 0; dir < 4; ++dir)
        if (g.has(I, J, dir)) {
          ++m;
          e += msg_slot_elems(g.side_len(I, J, dir), D);
        }
  *M = m;
  *arena_elems = align_up(e, 32);
}

// Shared-memory layout of one CTA (one syndrome x coset).
struct CtaLayout {
  int synd, frame, msg_of, msg_off, meta, dims, work, ovl, rlog, misc, ws, total;
};

BBP_HD CtaLayout cta_layout(const Geo& g, int M, int K, int nwarps, int ws_bytes) {
  CtaLayout L;
  int m = 2 * g.d * (g.d - 1);
  int o = 0;
  L.synd = o;    o = align_up(o + m, 16);
  L.frame = o;   o = align_up(o + g.W * g.W, 16);
  L.msg_of = o;  o = align_up(o + 2 * g.nb * g.nb * 4, 16);       // int16
  L.msg_off = o; o = align_up(o + 4 * M, 16);                     // int32
  L.meta = o;    o = align_up(o + 2 * M, 16);                     // int16 key of each message
  L.dims = o;    o = align_up(o + M * (K + 1), 16);               // int8
  L.work = o;    o = align_up(o + 2 * 2 * M, 16);                 // int16 x 2 colours
  L.ovl = o;     o = align_up(o + 8 * M, 16);                     // double
  L.rlog = o;    o = align_up(o + 8 * (g.nb * g.nb + M), 16);     // double
  L.misc = o;    o = align_up(o + 64, 16);
  L.ws = o;      o = align_up(o + nwarps * ws_bytes, 16);
  L.total = o;
  return L;
}

}  // namespace bbp
