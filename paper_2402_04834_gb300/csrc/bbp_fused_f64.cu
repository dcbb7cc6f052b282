// FP64 instances of the fused-block kernel (Remark 9) and the table of the
// compiled launch shapes (warps per CTA, cosets per CTA) of both precisions.
#include "bbp_decode_inst.cuh"

namespace bbp {

cudaError_t launch_fused_f64(const LaunchArgs& a, int warps, int cosets, bool gm, int lean, cudaStream_t st) {
  if (lean > 0) {                          // every block update in register form, sized for `lean` CTAs per SM
    switch (warps * 100 + cosets * 10 + lean) {
      case 424: return launch_fused_nw<double, 4, 2, 4, false, 4>(a, st);
      case 822: return launch_fused_nw<double, 8, 2, 4, false, 2>(a, st);
      default: return cudaErrorInvalidValue;
    }
  }
  if (a.geo.k > 4) {
    switch (warps * 10 + cosets) {
      case 21: return launch_fused_nw<double, 2, 1, 6>(a, st);
      case 31: return launch_fused_nw<double, 3, 1, 6>(a, st);
      default: return cudaErrorInvalidValue;
    }
  }
  if (gm) return warps * 10 + cosets == 42 ? launch_fused_nw<double, 4, 2, 4, true>(a, st) : cudaErrorInvalidValue;
  switch (warps * 10 + cosets) {
    case 81: return launch_fused_nw<double, 8, 1, 4>(a, st);
    case 42: return launch_fused_nw<double, 4, 2, 4>(a, st);
    case 82: return launch_fused_nw<double, 8, 2, 4>(a, st);
    case 44: return launch_fused_nw<double, 4, 4, 4>(a, st);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_fused_mixed_f64(const LaunchArgs& a, const MixedLaunch& m, int warps, int cosets, bool gm,
                                   int lean, cudaStream_t st) {
  if (lean > 0) {                          // every distance odd: every block update in register form
    switch (warps * 100 + cosets * 10 + lean) {
      case 424: return launch_fused_mixed_nw<double, 4, 2, 4, false, 4>(a, m, st);
      case 822: return launch_fused_mixed_nw<double, 8, 2, 4, false, 2>(a, m, st);
      default: return cudaErrorInvalidValue;
    }
  }
  if (a.geo.k > 4) {
    switch (warps * 10 + cosets) {
      case 21: return launch_fused_mixed_nw<double, 2, 1, 6>(a, m, st);
      case 31: return launch_fused_mixed_nw<double, 3, 1, 6>(a, m, st);
      default: return cudaErrorInvalidValue;
    }
  }
  if (gm)
    return warps * 10 + cosets == 42 ? launch_fused_mixed_nw<double, 4, 2, 4, true>(a, m, st) : cudaErrorInvalidValue;
  switch (warps * 10 + cosets) {
    case 81: return launch_fused_mixed_nw<double, 8, 1, 4>(a, m, st);
    case 42: return launch_fused_mixed_nw<double, 4, 2, 4>(a, m, st);
    case 82: return launch_fused_mixed_nw<double, 8, 2, 4>(a, m, st);
    case 44: return launch_fused_mixed_nw<double, 4, 4, 4>(a, m, st);
    default: return cudaErrorInvalidValue;
  }
}

namespace {

struct Shape {
  int warps, cosets;
  bool gm;        // messages in a workspace slot of the CTA instead of shared memory
  int lean = 0;   // > 0: every block update in register form, sized for this many CTAs per SM
};

// Compiled shapes in the order the default launch tries them: the
// register-form-only kernels where the geometry allows them, then
// shared-memory messages where they leave room for the CTAs per SM the
// register budget is sized for (FusedMinBlocks), then the same shape with
// its messages in the workspace.  Measured on the d = 11, p = 0.10 workload
// (GB300, ms per 10^4 syndromes): FP32 register form only (8,4) 16.3 at 3
// CTAs per SM, (8,2) 18.2; full kernels (8,4) 20.6, (4,2) 30.1, (8,2) 32.7,
// (4,4) 42.7, (4,1) 44.8, (8,1) 46.7, (16,1) 52.2; FP64 about 150 per 4096
// syndromes for (4,2) and (8,2), 176 for (4,4).
constexpr Shape kShapesF32[] = {{8, 4, false, 4}, {8, 4, false, 3}, {8, 2, false, 4}, {8, 4, false}, {8, 4, true}, {8, 2, false},
                                {8, 2, true}, {4, 2, false}, {4, 4, false}, {16, 1, false}, {8, 1, false},
                                {4, 1, false}};
constexpr Shape kShapesF64[] = {{4, 2, false, 4}, {8, 2, false, 2}, {4, 2, false}, {4, 2, true}, {8, 2, false},
                                {8, 1, false}, {4, 4, false}};

// Block sides 5 and 6: states of 2^12 entries, one coset per CTA, messages
// in the workspace; the most warps whose state buffers fit one SM first.
constexpr Shape kShapesF32K6[] = {{6, 1, true}, {4, 1, true}, {2, 1, true}};
constexpr Shape kShapesF64K6[] = {{3, 1, true}, {2, 1, true}};

// Resident CTAs per SM that the register budget of a shape is sized for
// (the host-side value of FusedMinBlocks).
int target_blocks(int precision, int k, const Shape& s) {
  if (s.lean > 0) return s.lean;
  const int warps = k > 4 ? s.warps : (precision == 0 ? 16 : 32) / (s.cosets > 1 ? 2 : 1);
  return warps / s.warps > 1 ? warps / s.warps : 1;
}

}  // namespace

int fused_smem_bytes(int precision, const Geo& g, int M, int warps, int cosets, bool gm, bool lean) {
  if (g.k > 4)
    return precision == 0 ? fused_smem_for<double, 6>(g, M, warps, cosets) : fused_smem_for<float, 6>(g, M, warps, cosets);
  return precision == 0 ? fused_smem_for<double, 4>(g, M, warps, cosets, gm, lean)
                        : fused_smem_for<float, 4>(g, M, warps, cosets, gm, lean);
}

bool fused_shape(int precision, const Geo& g, int M, int* warps, int* cosets, int* messages, bool allow_lean,
                 int* lean_blocks) {
  const bool k6 = g.k > 4;
  const Shape* sh = k6 ? (precision == 0 ? kShapesF64K6 : kShapesF32K6) : (precision == 0 ? kShapesF64 : kShapesF32);
  const int n = k6 ? (precision == 0 ? (int)(sizeof(kShapesF64K6) / sizeof(Shape)) : (int)(sizeof(kShapesF32K6) / sizeof(Shape)))
                   : (precision == 0 ? (int)(sizeof(kShapesF64) / sizeof(Shape)) : (int)(sizeof(kShapesF32) / sizeof(Shape)));
  // Pass 0 keeps only shapes whose shared memory allows their target CTAs
  // per SM; pass 1 any shape that fits.
  for (int pass = 0; pass < 2; ++pass) {
    for (int i = 0; i < n; ++i) {
      if (*warps != 0 && sh[i].warps != *warps) continue;
      if (*cosets != 0 && sh[i].cosets != *cosets) continue;
      const int mem = sh[i].lean > 0 ? 3 : (sh[i].gm ? 2 : 1);
      if (*messages != 0 && *messages != mem) continue;
      if (sh[i].lean > 0 && (!allow_lean || !register_form_only(g))) continue;
      const int smem = fused_smem_bytes(precision, g, M, sh[i].warps, sh[i].cosets, sh[i].gm, sh[i].lean > 0);
      if (smem > kMaxSmemBytes) continue;
      if (pass == 0 && kSmemPerSm / (smem + kSmemReservedPerCta) < target_blocks(precision, g.k, sh[i])) continue;
      *warps = sh[i].warps;
      *cosets = sh[i].cosets;
      *messages = mem;
      if (lean_blocks) *lean_blocks = sh[i].lean;
      return true;
    }
  }
  return false;
}

}  // namespace bbp
