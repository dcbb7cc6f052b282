// Seeded depolarizing sampler on the device (Sec. IV workload): errors,
// syndromes and the coset index of each error relative to the pure error;
// and the pure error f_s of given syndromes (Algorithm 1, first step).
#include <cuda_runtime.h>
#include <stdint.h>

#include "bbp_launch.h"

namespace bbp {

// SplitMix64 output function applied to x (Steele, Lea & Flood 2014).
__device__ __forceinline__ uint64_t splitmix64(uint64_t x) {
  uint64_t z = x + 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

__global__ void sample_kernel(uint64_t seed, long long first_shot, int d, unsigned long long thr,
                              uint8_t* ex, uint8_t* ez, uint8_t* synd, int8_t* true_class) {
  extern __shared__ uint8_t sm[];
  const int W = 2 * d - 1, n = d * d + (d - 1) * (d - 1), m = 2 * d * (d - 1);
  uint8_t* gx = sm;
  uint8_t* gz = sm + W * W;
  const long long b = blockIdx.x;
  const uint64_t shot = (uint64_t)(first_shot + b);
  const uint64_t ks = splitmix64(splitmix64(seed) ^ shot);
  for (int e = threadIdx.x; e < W * W; e += blockDim.x) { gx[e] = 0; gz[e] = 0; }
  __syncthreads();
  for (int q = threadIdx.x; q < n; q += blockDim.x) {
    const int pair = q / (2 * d - 1), rem = q % (2 * d - 1);
    const int i = rem < d ? 2 * pair : 2 * pair + 1;
    const int j = rem < d ? 2 * rem : 2 * (rem - d) + 1;
    const uint64_t r = splitmix64(ks ^ (uint64_t)q);
    uint8_t x = 0, z = 0;
    if ((r >> 11) >= thr) {
      const uint64_t kind = ((splitmix64(r) >> 32) * 3ull) >> 32;   // 0 X, 1 Y, 2 Z
      x = (kind <= 1);
      z = (kind >= 1);
    }
    gx[i * W + j] = x;
    gz[i * W + j] = z;
    if (ex) ex[b * n + q] = x;
    if (ez) ez[b * n + q] = z;
  }
  __syncthreads();
  for (int ci = threadIdx.x; ci < m; ci += blockDim.x) {
    int i, j;
    const uint8_t* g;
    if (ci < d * (d - 1)) { i = 2 * (ci / (d - 1)); j = 2 * (ci % (d - 1)) + 1; g = gx; }   // A_u sees x
    else { const int c2 = ci - d * (d - 1); i = 2 * (c2 / d) + 1; j = 2 * (c2 % d); g = gz; } // B_p sees z
    uint8_t v = 0;
    if (i > 0) v ^= g[(i - 1) * W + j];
    if (i < W - 1) v ^= g[(i + 1) * W + j];
    if (j > 0) v ^= g[i * W + j - 1];
    if (j < W - 1) v ^= g[i * W + j + 1];
    synd[b * m + ci] = v;
  }
  if (threadIdx.x == 0 && true_class) {
    // The pure error vanishes on the supports of both logicals, so the class
    // is read off the error alone: X-bar part from Z-bar = Z on column 0,
    // Z-bar part from X-bar = X on row 0.
    int bx = 0, bz = 0;
    for (int r = 0; r < d; ++r) bx ^= gx[(2 * r) * W + 0];
    for (int c = 0; c < d; ++c) bz ^= gz[0 * W + 2 * c];
    true_class[b] = (int8_t)(bx ? (bz ? 2 : 1) : (bz ? 3 : 0));
  }
}

cudaError_t launch_sample(uint64_t seed, long long first_shot, long long B, int d,
                          unsigned long long id_threshold, uint8_t* ex, uint8_t* ez,
                          uint8_t* synd, int8_t* true_class, cudaStream_t st) {
  const int W = 2 * d - 1;
  const int smem = 2 * W * W;
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(sample_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
  }
  sample_kernel<<<(unsigned)B, 128, smem, st>>>(seed, first_shot, d, id_threshold, ex, ez, synd, true_class);
  return cudaGetLastError();
}

// Pure error f_s (Algorithm 1 asks for any Pauli with syndrome s; the
// choice here): for every flagged site check A_(r,c) an X string on the
// horizontal edges h(r, c+1 .. d-1) to the right boundary, for every flagged
// plaquette B_(r,j) a Z string on h(r+1 .. d-1, j) down to the bottom.
// Horizontal-edge qubit h(r, cc) therefore carries x = XOR of A_(r,c) over
// c < cc and z = XOR of B_(r2,cc) over r2 < r; vertical-edge qubits carry
// nothing.  One thread per (syndrome, qubit), qubits in sampler order.
__global__ void pure_error_kernel(int d, const uint8_t* synd, long long B, uint8_t* fx, uint8_t* fz) {
  const int n = d * d + (d - 1) * (d - 1), m = 2 * d * (d - 1);
  const long long total = B * n;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    const long long b = t / n;
    const int q = (int)(t - b * n);
    const int pair = q / (2 * d - 1), rem = q % (2 * d - 1);
    uint8_t x = 0, z = 0;
    if (rem < d) {                                   // horizontal edge h(pair, rem)
      const uint8_t* s = synd + b * m;
      for (int c = 0; c < rem; ++c) x ^= s[pair * (d - 1) + c];
      for (int r2 = 0; r2 < pair; ++r2) z ^= s[d * (d - 1) + r2 * d + rem];
    }
    fx[t] = x;
    fz[t] = z;
  }
}

cudaError_t launch_pure_error(int d, const uint8_t* synd, long long B, uint8_t* fx, uint8_t* fz, cudaStream_t st) {
  const long long total = B * (long long)(d * d + (d - 1) * (d - 1));
  long long blocks = (total + 255) / 256;
  int dev = 0, sms = 0;
  cudaError_t e;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
  if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
  if (blocks > (long long)sms * 64) blocks = (long long)sms * 64;   // grid-stride beyond 64 blocks per SM
  pure_error_kernel<<<(unsigned)blocks, 256, 0, st>>>(d, synd, B, fx, fz);
  return cudaGetLastError();
}

}  // namespace bbp
