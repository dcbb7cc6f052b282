// Launchers of the compiled decoder instances (one translation unit per
// precision), called by the C ABI in bbp_api.cu.
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include "bbp_geometry.h"

namespace bbp {

// Compile-time capacity of the instances: block side k <= kMaxK and bond
// dimension D <= kMaxD; kWarps warps (message updates in flight) per CTA.
constexpr int kMaxK = 4;
constexpr int kMaxD = 8;
constexpr int kWarps = 4;

struct LaunchArgs {
  Geo geo;
  int M, D, max_iter, arena_elems;
  double p, eta, delta0, delta1, cutoff;
  const uint8_t* synd;
  void* arena;
  double* logp;
  double* delta;
  int32_t* iters;
  int32_t* flags;
  int8_t* decision;
  long long B;
  const float* init_msgs = nullptr;
  float* final_msgs = nullptr;
  long long slots = 0;            // fused, messages in the workspace: slots of G * M * vec scalars in arena
};

// Shared memory of one CTA in bytes for the given precision (0 = fp64, 1 = fp32).
int cta_smem_bytes(int precision, const Geo& g, int M);

// Fused-block path (Remark 9): block side k <= kFusedMaxK; kernels compiled
// for k <= 4 (messages in shared memory, or for some shapes in a workspace
// slot per resident CTA) and for k = 5, 6 (always in a workspace slot); at
// most kFusedSlots slots.
constexpr int kFusedMaxK = 6;
constexpr long long kFusedSlots = 512;
constexpr int kMaxSmemBytes = 227 * 1024;       // opt-in shared memory of one CTA
constexpr int kSmemPerSm = 228 * 1024;          // shared memory of one SM
constexpr int kSmemReservedPerCta = 1024;       // reserved by the runtime per resident CTA
int fused_smem_bytes(int precision, const Geo& g, int M, int warps, int cosets, bool gm, bool lean = false);
// Launch shape of the fused kernel: *warps / *cosets / *messages (1 shared
// memory, 2 workspace slots, 3 shared memory with every block update in
// register form: k = 4 with a one-node-wide last block) are requests
// (0 = any); on success they hold the first compiled shape that matches
// them, preferring shapes whose shared memory allows the CTAs per SM their
// registers are sized for; *lean_blocks (if given) the CTAs per SM a
// register-form-only kernel is compiled for (0 for the others).
bool fused_shape(int precision, const Geo& g, int M, int* warps, int* cosets, int* messages, bool allow_lean = true,
                 int* lean_blocks = nullptr);

struct MixedLaunch {
  const int32_t* d_of;
  const int64_t* offsets;
  const int32_t* order;
  unsigned long long* counter;
  int d_max;
  int ctas_per_sm;
  void* slot_base = nullptr;      // messages in the workspace: slots of G * M(d_max) * vec scalars
  long long slots = 0;
};

// lean: 0, or the CTAs per SM of the register-form-only kernel to launch.
cudaError_t launch_fused_f64(const LaunchArgs& a, int warps, int cosets, bool gm, int lean, cudaStream_t st);
cudaError_t launch_fused_f32(const LaunchArgs& a, int warps, int cosets, bool gm, int lean, cudaStream_t st);
// lean as for launch_fused_f32 / _f64 (every distance of the batch odd).
cudaError_t launch_fused_mixed_f64(const LaunchArgs& a, const MixedLaunch& mx, int warps, int cosets, bool gm,
                                   int lean, cudaStream_t st);
cudaError_t launch_fused_mixed_f32(const LaunchArgs& a, const MixedLaunch& mx, int warps, int cosets, bool gm,
                                   int lean, cudaStream_t st);
cudaError_t launch_decode_f64(const LaunchArgs& a, cudaStream_t st);
cudaError_t launch_decode_f32(const LaunchArgs& a, cudaStream_t st);
cudaError_t launch_decide(const LaunchArgs& a, cudaStream_t st);
cudaError_t launch_pure_error(int d, const uint8_t* synd, long long B, uint8_t* fx, uint8_t* fz, cudaStream_t st);
cudaError_t launch_sample(uint64_t seed, long long first_shot, long long B, int d,
                          unsigned long long id_threshold, uint8_t* ex, uint8_t* ez,
                          uint8_t* synd, int8_t* true_class, cudaStream_t st);

}  // namespace bbp
