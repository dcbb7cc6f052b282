// Tensor-core (tcgen05) inference of the warm-start network, called by the
// C ABI in bbp_warm.cu.
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include "../../include/blockbp.h"
#include "bbp_geometry.h"

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

// The same from feature bits [N x 8 words] (bbp_warm.cu's features_rows with
// bits): bit q set where feature q is not zero; feature 253 is 10 p.
cudaError_t infer_tc_bits(const float* theta, const uint32_t* bits, const int32_t* lens, long long N, double p,
                          float alpha, float* msgs, void* workspace, cudaStream_t st);

// Features of the listed rows (bbp_message_features_rows), as FP32 rows
// [B*U x 256] (feats) or as bits [B*U x 8 words] (bits); exactly one of them.
int features_rows(const uint8_t* syndromes, int64_t B, const bbp_params* prm, const int32_t* row_key, int32_t U,
                  float* feats, uint32_t* bits, int32_t* lens, cudaStream_t st);

// Shared memory the syndrome-fed kernel needs at geometry g (bytes).
int infer_tc_syndromes_smem(const Geo& g, int M);

// msgs[B * 4 * M x 16] = proposals for every message of B syndromes, rows
// ordered (syndrome, coset, message), the features computed in the kernel.
cudaError_t infer_tc_syndromes(const float* theta, const uint8_t* synd, long long B, const Geo& g, int M, double p,
                               float alpha, float* msgs, void* workspace, cudaStream_t st);

}  // namespace warm
}  // namespace bbp
