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
  k.n_items = 0; k.slot_elems = 0;
  set_working(k);
  const int smem = smem_bytes_for<T>(a.geo, a.M);
  auto kern = decode_kernel<T, kMaxK, kMaxD, kWarps>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  const unsigned grid = (unsigned)(a.B * 4);
  kern<<<grid, kWarps * 32, smem, st>>>(k);
  return cudaGetLastError();
}

template <typename T, int K>
int fused_smem_for(const Geo& g, int M, int warps, int cosets, bool gm = (K > 4), bool lean = false) {
  return fused_layout<T, K>(g, M, warps, cosets, gm, lean).total;
}

template <typename T>
KArgs<T> fused_args(const LaunchArgs& a) {
  KArgs<T> k;
  k.geo = a.geo; k.M = a.M; k.D = a.D; k.max_iter = a.max_iter; k.arena_elems = 0;
  k.p = a.p; k.eta = a.eta; k.delta0 = a.delta0; k.delta1 = a.delta1; k.cutoff = a.cutoff;
  k.synd = a.synd; k.arena = nullptr;
  k.logp = a.logp; k.delta = a.delta; k.iters = a.iters; k.flags = a.flags;
  k.init_msgs = a.init_msgs; k.final_msgs = a.final_msgs;
  k.n_items = 0; k.slot_elems = 0;
  set_working(k);
  return k;
}

// Persistent grid of a launch with its messages in workspace slots:
// resident CTAs, at most one per item and per message slot.
template <typename Kern>
cudaError_t persistent_grid(Kern kern, int threads, int smem, int ctas_per_sm, long long items, long long slots,
                            long long* grid) {
  cudaError_t e;
  int per_sm = ctas_per_sm;
  if (per_sm <= 0) {
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, smem)) != cudaSuccess) return e;
    if (per_sm < 1) per_sm = 1;
  }
  int dev = 0, sms = 0;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
  if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
  long long g = (long long)sms * per_sm;
  if (g > items) g = items;
  if (g > slots) g = slots;
  *grid = g;
  return g > 0 ? cudaSuccess : cudaErrorInvalidValue;
}

// GM: messages in the workspace (a.arena, a.slots slots of G * M * vec
// scalars), a persistent grid; always for k = 5, 6.
template <typename T, int NW, int G, int K, bool GM = (K > 4), int LB = 0>
cudaError_t launch_fused_nw(const LaunchArgs& a, cudaStream_t st) {
  const KArgs<T> k = fused_args<T>(a);
  const int smem = fused_smem_for<T, K>(a.geo, a.M, NW, G, GM, LB > 0);
  auto kern = fused_kernel<T, NW, G, K, GM, LB>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  const long long items = a.B * (4 / G);
  if (GM) {
    KArgs<T> kp = k;
    kp.arena = static_cast<T*>(a.arena);
    kp.n_items = items;
    kp.slot_elems = (long long)G * a.M * FusedDim<K>::vec;
    long long grid = 0;
    if ((e = persistent_grid(kern, NW * 32, smem, 0, items, a.slots, &grid)) != cudaSuccess) return e;
    kern<<<(unsigned)grid, NW * 32, smem, st>>>(kp);
    return cudaGetLastError();
  }
  kern<<<(unsigned)items, NW * 32, smem, st>>>(k);
  return cudaGetLastError();
}

template <typename T, int NW, int G, int K, bool GM = (K > 4), int LB = 0>
cudaError_t launch_fused_mixed_nw(const LaunchArgs& a, const MixedLaunch& m, cudaStream_t st) {
  const KArgs<T> k = fused_args<T>(a);
  const Geo gmax = make_geo(m.d_max, a.geo.k);
  int Mmax = 0, ae = 0;
  count_messages(gmax, 1, &Mmax, &ae);
  const int smem = fused_smem_for<T, K>(gmax, Mmax, NW, G, GM, LB > 0);
  auto kern = fused_mixed_kernel<T, NW, G, K, GM, LB>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  int per_sm = m.ctas_per_sm;
  if (per_sm <= 0) {
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, NW * 32, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) per_sm = 1;
  }
  int dev = 0, sms = 0;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
  if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
  MixedArgs mx;
  mx.d_of = m.d_of; mx.offsets = m.offsets; mx.order = m.order; mx.counter = m.counter;
  mx.n_items = a.B * (4 / G); mx.k = a.geo.k;
  mx.B = a.B; mx.d_max = m.d_max;
  long long grid = (long long)sms * per_sm;
  if (grid > mx.n_items) grid = mx.n_items;
  KArgs<T> kp = k;
  if (GM) {      // messages in the workspace, one slot per CTA
    kp.arena = static_cast<T*>(m.slot_base);
    kp.slot_elems = (long long)G * Mmax * FusedDim<K>::vec;
    if (grid > m.slots) grid = m.slots;
    if (grid < 1) return cudaErrorInvalidValue;
  }
  if ((e = cudaMemsetAsync(m.counter, 0, sizeof(unsigned long long), st)) != cudaSuccess) return e;
  kern<<<(unsigned)grid, NW * 32, smem, st>>>(kp, mx);
  return cudaGetLastError();
}

}  // namespace bbp
