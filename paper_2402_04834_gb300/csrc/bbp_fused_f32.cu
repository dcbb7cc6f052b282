// FP32 instances of the fused-block kernel (Remark 9): FP32 state, node
// tensors and messages; Delta sums, log norms and the read-out in double.
#include "bbp_decode_inst.cuh"

namespace bbp {

cudaError_t launch_fused_f32(const LaunchArgs& a, int warps, int cosets, bool gm, int lean, cudaStream_t st) {
  if (lean > 0) {                          // every block update in register form, sized for `lean` CTAs per SM
    switch (warps * 100 + cosets * 10 + lean) {
      case 844: return launch_fused_nw<float, 8, 4, 4, false, 4>(a, st);
      case 843: return launch_fused_nw<float, 8, 4, 4, false, 3>(a, st);
      case 824: return launch_fused_nw<float, 8, 2, 4, false, 4>(a, st);
      default: return cudaErrorInvalidValue;
    }
  }
  if (a.geo.k > 4) {                       // block sides 5 and 6
    switch (warps * 10 + cosets) {
      case 21: return launch_fused_nw<float, 2, 1, 6>(a, st);
      case 41: return launch_fused_nw<float, 4, 1, 6>(a, st);
      case 61: return launch_fused_nw<float, 6, 1, 6>(a, st);
      default: return cudaErrorInvalidValue;
    }
  }
  if (gm) {                                // k <= 4, messages in the workspace
    switch (warps * 10 + cosets) {
      case 84: return launch_fused_nw<float, 8, 4, 4, true>(a, st);
      case 82: return launch_fused_nw<float, 8, 2, 4, true>(a, st);
      default: return cudaErrorInvalidValue;
    }
  }
  switch (warps * 10 + cosets) {
    case 41: return launch_fused_nw<float, 4, 1, 4>(a, st);
    case 81: return launch_fused_nw<float, 8, 1, 4>(a, st);
    case 161: return launch_fused_nw<float, 16, 1, 4>(a, st);
    case 42: return launch_fused_nw<float, 4, 2, 4>(a, st);
    case 82: return launch_fused_nw<float, 8, 2, 4>(a, st);
    case 44: return launch_fused_nw<float, 4, 4, 4>(a, st);
    case 84: return launch_fused_nw<float, 8, 4, 4>(a, st);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_fused_mixed_f32(const LaunchArgs& a, const MixedLaunch& m, int warps, int cosets, bool gm,
                                   int lean, cudaStream_t st) {
  if (lean > 0) {                          // every distance odd: every block update in register form
    switch (warps * 100 + cosets * 10 + lean) {
      case 844: return launch_fused_mixed_nw<float, 8, 4, 4, false, 4>(a, m, st);
      case 843: return launch_fused_mixed_nw<float, 8, 4, 4, false, 3>(a, m, st);
      case 824: return launch_fused_mixed_nw<float, 8, 2, 4, false, 4>(a, m, st);
      default: return cudaErrorInvalidValue;
    }
  }
  if (a.geo.k > 4) {
    switch (warps * 10 + cosets) {
      case 21: return launch_fused_mixed_nw<float, 2, 1, 6>(a, m, st);
      case 41: return launch_fused_mixed_nw<float, 4, 1, 6>(a, m, st);
      case 61: return launch_fused_mixed_nw<float, 6, 1, 6>(a, m, st);
      default: return cudaErrorInvalidValue;
    }
  }
  if (gm) {
    switch (warps * 10 + cosets) {
      case 84: return launch_fused_mixed_nw<float, 8, 4, 4, true>(a, m, st);
      case 82: return launch_fused_mixed_nw<float, 8, 2, 4, true>(a, m, st);
      default: return cudaErrorInvalidValue;
    }
  }
  switch (warps * 10 + cosets) {
    case 41: return launch_fused_mixed_nw<float, 4, 1, 4>(a, m, st);
    case 81: return launch_fused_mixed_nw<float, 8, 1, 4>(a, m, st);
    case 161: return launch_fused_mixed_nw<float, 16, 1, 4>(a, m, st);
    case 42: return launch_fused_mixed_nw<float, 4, 2, 4>(a, m, st);
    case 82: return launch_fused_mixed_nw<float, 8, 2, 4>(a, m, st);
    case 44: return launch_fused_mixed_nw<float, 4, 4, 4>(a, m, st);
    case 84: return launch_fused_mixed_nw<float, 8, 4, 4>(a, m, st);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace bbp
