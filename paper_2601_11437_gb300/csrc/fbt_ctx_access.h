// Internal accessors of the opaque context for the host-side drivers (not exported in fbt.h).
#pragma once
#include <cuda_runtime.h>

#include "fbt.h"

namespace fbt {
cudaStream_t ctx_swap_stream(fbt_ctx* c, cudaStream_t s);   // returns the previous stream
int ctx_device(const fbt_ctx* c);
bool ctx_is_mixed(const fbt_ctx* c);        // FBT_PREC_MIXED context
long long ctx_n(const fbt_ctx* c);
// Algorithm 2 that also generates Sigma_alpha, Sigma_nu at theta and keeps them for a following
// Algorithm 3 evaluation at the same theta (the line search of Algorithm 1)
fbt_status loglik_keep_partials(fbt_ctx* c, const double theta[3], double* loglik);
// Records a CUDA failure for fbt_last_cuda_error() ("where: message") and returns FBT_ERR_CUDA.
fbt_status record_cuda_error(cudaError_t e, const char* where);
}  // namespace fbt
