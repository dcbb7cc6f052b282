// FP32 instance of the blockBP decoder kernel: tensors, QR and SVD in float;
// log norms, overlaps, Delta and the read-out sums in double.
#include "bbp_decode_inst.cuh"

namespace bbp {

cudaError_t launch_decode_f32(const LaunchArgs& a, cudaStream_t st) { return launch_decode_t<float>(a, st); }
cudaError_t launch_fused_f32(const LaunchArgs& a, int warps, cudaStream_t st) {
  if (warps == 4) return launch_fused_nw<float, 4>(a, st);
  if (warps == 16) return launch_fused_nw<float, 16>(a, st);
  return launch_fused_nw<float, 8>(a, st);
}
cudaError_t launch_fused_mixed_f32(const LaunchArgs& a, const MixedLaunch& m, int warps, cudaStream_t st) {
  if (warps == 4) return launch_fused_mixed_nw<float, 4>(a, m, st);
  if (warps == 16) return launch_fused_mixed_nw<float, 16>(a, m, st);
  return launch_fused_mixed_nw<float, 8>(a, m, st);
}

int cta_smem_bytes(int precision, const Geo& g, int M) {
  return precision == 0 ? smem_bytes_for<double>(g, M) : smem_bytes_for<float>(g, M);
}

int fused_smem_bytes(int precision, const Geo& g, int M, int warps) {
  return precision == 0 ? fused_smem_for<double>(g, M, 8) : fused_smem_for<float>(g, M, warps);
}

}  // namespace bbp
