// FP32 instance of the blockBP decoder kernel: tensors, QR and SVD in float;
// log norms, overlaps, Delta and the read-out sums in double.
#include "bbp_decode_inst.cuh"

namespace bbp {


cudaError_t launch_decode_f32(const LaunchArgs& a, cudaStream_t st) { return launch_decode_t<float>(a, st); }
int cta_smem_bytes(int precision, const Geo& g, int M) {
  return precision == 0 ? smem_bytes_for<double>(g, M) : smem_bytes_for<float>(g, M);
}

}  // namespace bbp
