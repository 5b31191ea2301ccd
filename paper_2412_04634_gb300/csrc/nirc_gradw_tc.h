// nirc_gradw_tc.h -- weight gradients of the training step on the tensor
// cores: for every layer, dW = sum over samples of delta x^T and
// db = sum of delta, from the stored BF16 deltas and layer inputs.
#pragma once

#include "nirc_internal.h"

namespace nirc {

struct DwJob {
    const uint16_t* dl;  // BF16 deltas [out][ld_dl] (samples contiguous)
    const uint16_t* x;   // BF16 layer inputs [in][ld_x]
    float* gw;        // W [out][in] then b [out]; the sums are added
    uint64_t ld_dl, ld_x;
    uint32_t out, in;  // out <= 64, in <= 79
};

struct DwJobs {
    DwJob j[kMaxHidden + 1];
    uint32_t n_jobs;
};

// Adds every job's dW and db over samples [0, m) into its gw.  BF16
// operands, FP32 accumulation in tensor memory, float atomics into gw (the
// order of the sums varies).
cudaError_t launch_grad_w_tc(const nirc_handle* h, const DwJobs& jobs, uint64_t m, cudaStream_t st);

}  // namespace nirc
