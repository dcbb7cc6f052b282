// Tensor-core (tcgen05) inference of the warm-start network, called by the
// C ABI in bbp_warm.cu.
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include "../../include/blockbp.h"

namespace bbp {
namespace warm {

// Workspace: the three layers' BF16 weights in the tensor cores' operand
// layout (128 KB + 128 KB + 8 KB), then the int32 status word.
constexpr int kStatusOffset = 2 * (256 * 256 * 2) + 16 * 256 * 2;
static_assert(kStatusOffset == BBP_WARM_STATUS_OFFSET, "status word offset");
static_assert(kStatusOffset + 256 == BBP_WARM_INFER_WORKSPACE_BYTES, "inference workspace");

size_t infer_tc_workspace_bytes();

// msgs[N x 16] = proposals for feats[N x 256] (FP32 row-major), lens = 2^w per row.
cudaError_t infer_tc(const float* theta, const float* feats, const int32_t* lens, long long N, float alpha,
                     float* msgs, void* workspace, cudaStream_t st);

}  // namespace warm
}  // namespace bbp
