// Decoding without any allocation: bbp_decode_batch_static.
//
// Some callers cannot call cudaMalloc at all: real-time decoding loops
// that must not take the allocator's locks or risk an out-of-memory error
// mid-run, and hosts that hand the decoder only the input and output
// buffers (a fixed memory budget owned by someone else).  For them the message arena lives in a fixed file-scope device
// array that every GPU loading this library reserves once, for the life
// of the process.
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/blockbp.h"
#include "bbp_launch.h"

namespace {

// The static message arena (BBP_STATIC_WORKSPACE_BYTES, 32 MiB).  In host
// code this name is only a stand-in for the device array, never a device
// address: the address is obtained per device with cudaGetSymbolAddress.
static __device__ __align__(256) unsigned char g_static_ws[BBP_STATIC_WORKSPACE_BYTES];

constexpr int kMaxDevices = 64;
void* g_ws_ptr[kMaxDevices];    // device address of g_static_ws, per device ordinal

// Looks the array up once per device, with that device current.
int static_workspace(void** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return BBP_ECUDA;
  if (dev < 0 || dev >= kMaxDevices) return BBP_EUNSUPPORTED;
  void* p = __atomic_load_n(&g_ws_ptr[dev], __ATOMIC_ACQUIRE);
  if (p == nullptr) {
    if (cudaGetSymbolAddress(&p, g_static_ws) != cudaSuccess || p == nullptr) return BBP_ECUDA;
    __atomic_store_n(&g_ws_ptr[dev], p, __ATOMIC_RELEASE);
  }
  *out = p;
  return BBP_OK;
}

}  // namespace

extern "C" int bbp_decode_batch_static(const uint8_t* syndromes, int64_t B, const bbp_params* prm,
                                       double* logp, double* delta, int32_t* iters, int32_t* flags,
                                       int8_t* decision, void* stream) {
  size_t need = 0;
  int rc = bbp_workspace_bytes(prm, B, 0, &need);
  if (rc != BBP_OK) return rc;
  bbp_params shared = {};
  if (need > (size_t)BBP_STATIC_WORKSPACE_BYTES && prm->algorithm == BBP_ALG_FUSED && prm->launch_messages == 0) {
    // The default shape keeps its messages in the workspace; a shape that
    // keeps them in shared memory needs none.
    shared = *prm;
    shared.launch_messages = 1;
    size_t need_shared = 0;
    if (bbp_workspace_bytes(&shared, B, 0, &need_shared) == BBP_OK) {
      prm = &shared;
      need = need_shared;
    }
  }
  if (need > (size_t)BBP_STATIC_WORKSPACE_BYTES) return BBP_ETOOLARGE;
  if (B == 0) return BBP_OK;
  if (!syndromes || !logp || !delta || !iters || !flags || !decision) return BBP_EINVAL;
  void* ws = nullptr;
  rc = static_workspace(&ws);
  if (rc != BBP_OK) return rc;
  return bbp_decode_batch(syndromes, B, prm, logp, delta, iters, flags, decision, ws,
                          (size_t)BBP_STATIC_WORKSPACE_BYTES, stream);
}
