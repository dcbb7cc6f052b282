// FP64 instances of the fused-block kernel (Remark 9) and the table of the
// compiled launch shapes (warps per CTA, cosets per CTA) of both precisions.
#include "bbp_decode_inst.cuh"

namespace bbp {

cudaError_t launch_fused_f64(const LaunchArgs& a, int warps, int cosets, cudaStream_t st) {
  if (a.geo.k > 4) {
    switch (warps * 10 + cosets) {
      case 21: return launch_fused_nw<double, 2, 1, 6>(a, st);
      case 31: return launch_fused_nw<double, 3, 1, 6>(a, st);
      default: return cudaErrorInvalidValue;
    }
  }
  switch (warps * 10 + cosets) {
    case 81: return launch_fused_nw<double, 8, 1, 4>(a, st);
    case 42: return launch_fused_nw<double, 4, 2, 4>(a, st);
    case 82: return launch_fused_nw<double, 8, 2, 4>(a, st);
    case 44: return launch_fused_nw<double, 4, 4, 4>(a, st);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_fused_mixed_f64(const LaunchArgs& a, const MixedLaunch& m, int warps, int cosets,
                                   cudaStream_t st) {
  if (a.geo.k > 4) {
    switch (warps * 10 + cosets) {
      case 21: return launch_fused_mixed_nw<double, 2, 1, 6>(a, m, st);
      case 31: return launch_fused_mixed_nw<double, 3, 1, 6>(a, m, st);
      default: return cudaErrorInvalidValue;
    }
  }
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
};

// Compiled shapes, in the order the default launch tries them: fastest
// first on the d = 11, p = 0.10 workload (GB300, syndromes/s: FP32 (8,4)
// 85.4k, (8,2) 69.9k, (4,2) 66.3k, (4,4) 56.7k, (16,1) 54.5k, (8,1) 53.2k,
// (4,1) 51.3k; FP64 (4,2) 16.8k, (8,1) 12.9k, (4,4) 11.9k), then by the
// shared memory they need, so that larger distances still find a shape.
constexpr Shape kShapesF32[] = {{8, 4}, {8, 2}, {4, 2}, {4, 4}, {16, 1}, {8, 1}, {4, 1}};
constexpr Shape kShapesF64[] = {{4, 2}, {8, 2}, {8, 1}, {4, 4}};

// Block sides 5 and 6: states of 2^12 entries, one coset per CTA, messages
// in the workspace; the most warps whose state buffers fit one SM first.
constexpr Shape kShapesF32K6[] = {{6, 1}, {4, 1}, {2, 1}};
constexpr Shape kShapesF64K6[] = {{3, 1}, {2, 1}};

}  // namespace

int fused_smem_bytes(int precision, const Geo& g, int M, int warps, int cosets) {
  if (g.k > 4)
    return precision == 0 ? fused_smem_for<double, 6>(g, M, warps, cosets) : fused_smem_for<float, 6>(g, M, warps, cosets);
  return precision == 0 ? fused_smem_for<double, 4>(g, M, warps, cosets) : fused_smem_for<float, 4>(g, M, warps, cosets);
}

bool fused_shape(int precision, const Geo& g, int M, int* warps, int* cosets) {
  const bool k6 = g.k > 4;
  const Shape* sh = k6 ? (precision == 0 ? kShapesF64K6 : kShapesF32K6) : (precision == 0 ? kShapesF64 : kShapesF32);
  const int n = k6 ? (precision == 0 ? (int)(sizeof(kShapesF64K6) / sizeof(Shape)) : (int)(sizeof(kShapesF32K6) / sizeof(Shape)))
                   : (precision == 0 ? (int)(sizeof(kShapesF64) / sizeof(Shape)) : (int)(sizeof(kShapesF32) / sizeof(Shape)));
  for (int i = 0; i < n; ++i) {
    if (*warps != 0 && sh[i].warps != *warps) continue;
    if (*cosets != 0 && sh[i].cosets != *cosets) continue;
    if (fused_smem_bytes(precision, g, M, sh[i].warps, sh[i].cosets) > kMaxSmemBytes) continue;
    *warps = sh[i].warps;
    *cosets = sh[i].cosets;
    return true;
  }
  return false;
}

}  // namespace bbp
