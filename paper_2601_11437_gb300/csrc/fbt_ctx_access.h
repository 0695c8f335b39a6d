// Internal accessors of the opaque context for the host-side drivers (not exported in fbt.h).
#pragma once
#include <cuda_runtime.h>

#include "fbt.h"

namespace fbt {
cudaStream_t ctx_swap_stream(fbt_ctx* c, cudaStream_t s);   // returns the previous stream
int ctx_device(const fbt_ctx* c);
long long ctx_n(const fbt_ctx* c);
}  // namespace fbt
