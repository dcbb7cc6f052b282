// Instantiation of the decoder kernel for one scalar type.
#pragma once

#include "bbp_fused.cuh"
#include "bbp_kernels.cuh"
#include "bbp_launch.h"

namespace bbp {

template <typename T>
int smem_bytes_for(const Geo& g, int M) {
  return cta_layout(g, M, kMaxK, kWarps, (int)sizeof(WarpWS<T, kMaxK, kMaxD>)).total;
}

template <typename T>
cudaError_t launch_decode_t(const LaunchArgs& a, cudaStream_t st) {
  KArgs<T> k;
  k.geo = a.geo; k.M = a.M; k.D = a.D; k.max_iter = a.max_iter; k.arena_elems = a.arena_elems;
  k.p = a.p; k.eta = a.eta; k.delta0 = a.delta0; k.delta1 = a.delta1; k.cutoff = a.cutoff;
  k.synd = a.synd; k.arena = static_cast<T*>(a.arena);
  k.logp = a.logp; k.delta = a.delta; k.iters = a.iters; k.flags = a.flags;
  k.init_msgs = nullptr; k.final_msgs = nullptr;
  const int smem = smem_bytes_for<T>(a.geo, a.M);
  auto kern = decode_kernel<T, kMaxK, kMaxD, kWarps>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  const unsigned grid = (unsigned)(a.B * 4);
  kern<<<grid, kWarps * 32, smem, st>>>(k);
  return cudaGetLastError();
}

template <typename T>
int fused_smem_for(const Geo& g, int M) {
  return fused_layout<T>(g, M, kFusedWarps).total;
}

template <typename T>
cudaError_t launch_fused_t(const LaunchArgs& a, cudaStream_t st) {
  KArgs<T> k;
  k.geo = a.geo; k.M = a.M; k.D = a.D; k.max_iter = a.max_iter; k.arena_elems = 0;
  k.p = a.p; k.eta = a.eta; k.delta0 = a.delta0; k.delta1 = a.delta1; k.cutoff = a.cutoff;
  k.synd = a.synd; k.arena = nullptr;
  k.logp = a.logp; k.delta = a.delta; k.iters = a.iters; k.flags = a.flags;
  k.init_msgs = a.init_msgs; k.final_msgs = a.final_msgs;
  const int smem = fused_smem_for<T>(a.geo, a.M);
  auto kern = fused_kernel<T, kFusedWarps>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  const unsigned grid = (unsigned)(a.B * 4);
  kern<<<grid, kFusedWarps * 32, smem, st>>>(k);
  return cudaGetLastError();
}

}  // namespace bbp
