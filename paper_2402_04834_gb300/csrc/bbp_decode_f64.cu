// FP64 instance of the blockBP decoder kernel and the decision kernel.
#include "bbp_decode_inst.cuh"

namespace bbp {

// Decision of Algorithm 1 / Remark 6 for each syndrome.
__global__ void decide_kernel(const double* logp, const double* delta, const int32_t* flags,
                              int8_t* decision, long long B) {
  const long long b = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (b >= B) return;
  int best = -1;
  for (int L = 0; L < 4; ++L) {
    if (flags[b * 4 + L] != 0) continue;
    if (best < 0 || logp[b * 4 + L] > logp[b * 4 + best]) best = L;
  }
  if (best < 0) {
    best = 0;
    for (int L = 1; L < 4; ++L)
      if (delta[b * 4 + L] < delta[b * 4 + best]) best = L;
  }
  decision[b] = (int8_t)best;
}


cudaError_t launch_decode_f64(const LaunchArgs& a, cudaStream_t st) { return launch_decode_t<double>(a, st); }
cudaError_t launch_decide(const LaunchArgs& a, cudaStream_t st) {
  const int tpb = 128;
  const unsigned grid = (unsigned)((a.B + tpb - 1) / tpb);
  decide_kernel<<<grid, tpb, 0, st>>>(a.logp, a.delta, a.flags, a.decision, a.B);
  return cudaGetLastError();
}

}  // namespace bbp
