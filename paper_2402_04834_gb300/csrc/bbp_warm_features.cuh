// Features of one directed block edge for the warm-start network, shared by
// the features kernel (training data) and the tensor-core inference kernel
// (which computes them on the fly from the syndrome), so that the network
// always sees the same inputs.
//
// The message from block (I, J) towards direction dir is read in the frame
// rotated so that dir points right: a 7 x 7 window of grid nodes, columns
// t = ncols-7 .. ncols-1 (the block's last columns and what lies behind
// it), rows s = -1 .. 5 of the chain, with five channels per node -- inside
// the grid, qubit, the coset frame's x bit and z bit (qubits), the syndrome
// bit (checks) -- then one-hot direction, one-hot message length, 10 p and
// a constant 1.
#pragma once

#include <stdint.h>

#include "bbp_geometry.h"

namespace bbp {
namespace warm {

// Position of a message's block in the grid, rotated so that dir points right.
struct MsgGeo {
  int dir, h, ncols, r0, r1, c0, c1;
  BBP_HD void node(int t, int s, int* i, int* j) const {
    switch (dir) {
      case kDirR: *i = r0 + s; *j = c0 + t; break;
      case kDirL: *i = r0 + s; *j = c1 - 1 - t; break;
      case kDirD: *i = r0 + t; *j = c0 + s; break;
      default:    *i = r1 - 1 - t; *j = c0 + s; break;
    }
  }
};

BBP_HD MsgGeo msg_geo(const Geo& g, int I, int J, int dir) {
  MsgGeo f;
  f.dir = dir;
  f.r0 = g.lo(I); f.r1 = g.hi(I); f.c0 = g.lo(J); f.c1 = g.hi(J);
  const bool rowwise = dir == kDirR || dir == kDirL;
  f.h = rowwise ? f.r1 - f.r0 : f.c1 - f.c0;
  f.ncols = rowwise ? f.c1 - f.c0 : f.r1 - f.r0;
  return f;
}

// Which logical strings the message's window sees: bit 0 if it holds a
// horizontal-edge qubit of grid row 0 (X-bar, flipped in cosets X and Y),
// bit 1 if one of grid column 0 (Z-bar, flipped in cosets Y and Z).  The
// coset frames differ nowhere else, so cosets that agree on the strings a
// window sees have the same features there.
BBP_HD int window_logicals(const Geo& g, const MsgGeo& f) {
  int seen = 0;
  for (int pos = 0; pos < 49; ++pos) {
    const int t = f.ncols - 7 + pos / 7, sp = -1 + pos % 7;
    int i, j;
    f.node(t, sp, &i, &j);
    if (i >= 0 && j >= 0 && i < g.W && j < g.W && (i & 1) == 0 && (j & 1) == 0) {
      if (i == 0) seen |= 1;
      if (j == 0) seen |= 2;
    }
  }
  return seen;
}

// Frame byte (x bit | z bit << 1) of grid node (i, j) for a coset: the pure
// error of the syndrome (x: checks A to the node's left in its row; z:
// checks B above it in its column) times the coset's logical string (X-bar
// on row 0, Z-bar on column 0).  Zero on checks and on vertical-edge qubits.
__device__ __forceinline__ uint8_t frame_byte(const uint8_t* synd, int d, int i, int j, int coset) {
  int fx = 0, fz = 0;
  if ((i & 1) == 0 && (j & 1) == 0) {
    const int r = i >> 1, cc = j >> 1;
    for (int c2 = 0; c2 < cc; ++c2) fx ^= synd[r * (d - 1) + c2];
    for (int r2 = 0; r2 < r; ++r2) fz ^= synd[d * (d - 1) + r2 * d + cc];
    if ((coset == 1 || coset == 2) && r == 0) fx ^= 1;
    if ((coset == 2 || coset == 3) && cc == 0) fz ^= 1;
  }
  return (uint8_t)(fx | (fz << 1));
}

// The five channels of window node pos (0 .. 48) of the message: inside the
// grid, qubit, frame x bit, frame z bit (qubits), syndrome bit (checks).
__device__ __forceinline__ void window_node(const Geo& g, const MsgGeo& f, int pos, const uint8_t* frame,
                                            const uint8_t* synd, float c[5]) {
  const int W = g.W, d = g.d;
  const int t = f.ncols - 7 + pos / 7, sp = -1 + pos % 7;
  int i, j;
  f.node(t, sp, &i, &j);
  c[0] = c[1] = c[2] = c[3] = c[4] = 0.f;
  if (!(i >= 0 && j >= 0 && i < W && j < W)) return;
  c[0] = 1.f;
  if (((i + j) & 1) == 0) {
    const int fr = frame[i * W + j];
    c[1] = 1.f;
    c[2] = (float)(fr & 1);
    c[3] = (float)((fr >> 1) & 1);
  } else {
    const int bit = (i & 1) == 0 ? (i >> 1) * (d - 1) + (j >> 1)              // A_(r,c)
                                 : d * (d - 1) + (i >> 1) * d + (j >> 1);     // B_(r,j)
    c[4] = (float)synd[bit];
  }
}

// Features 245 .. 255: one-hot direction, one-hot message length, 10 p, 1, 0.
__device__ __forceinline__ float tail_feature(const MsgGeo& f, int q, float p10) {
  if (q < 245 + 4) return (q - 245 == f.dir) ? 1.f : 0.f;
  if (q < 249 + 4) return (q - 249 == f.h - 1) ? 1.f : 0.f;
  if (q == 253) return p10;
  if (q == 254) return 1.f;
  return 0.f;
}

// Feature q (0 .. 255) of the message; frame is the coset's W x W frame.
__device__ __forceinline__ float message_feature(const Geo& g, const MsgGeo& f, int q, const uint8_t* frame,
                                                 const uint8_t* synd, float p10) {
  if (q < 5 * 49) {
    float c[5];
    window_node(g, f, q % 49, frame, synd, c);
    const int ch = q / 49;
    return ch == 0 ? c[0] : ch == 1 ? c[1] : ch == 2 ? c[2] : ch == 3 ? c[3] : c[4];
  }
  return tail_feature(f, q, p10);
}

}  // namespace warm
}  // namespace bbp
