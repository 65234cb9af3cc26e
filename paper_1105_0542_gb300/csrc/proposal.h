// Internal interface of the learned-proposal kernels.
#pragma once

#include <cstdint>

#include <cuda_runtime.h>

#include "sampler.h"

namespace su {

struct ProposalParams {
    SamplerParams base;          // path, tables, stream, items (128 samples each), outputs
    const unsigned char *blob;   // device: network blob (mlp::kBlobBytes)
    double T;                    // propagation time (a network input)
    float *outs;                 // per-sample mode: (shift, ls) per sample and heap index, or null
    int withhold;                // fault injection: the first tile withholds its MMA commit
};

size_t proposal_smem_bytes(const ProposalParams &Q);
int proposal_occupancy(const ProposalParams &Q, size_t smem);
cudaError_t launch_proposal(const ProposalParams &Q, int grid, size_t smem, cudaStream_t st);
cudaError_t launch_mlp_forward(const unsigned char *blob, const float *X, int64_t n, float *Y, int sms,
                               cudaStream_t st);

}  // namespace su
