// Internal accessors of the context for entry points implemented outside abi.cu.
#pragma once
#include <cuda_runtime.h>

#include "../../include/dmb.h"
#include "mlp_host.cuh"

// The context's surrogate network and stream; false if no network is loaded.
bool dmb_internal_surrogate(dmb_ctx *ctx, MlpDev *dev, cudaStream_t *stream);
// The CUDA device the context was created on (its stream and buffers live there).
int dmb_internal_device(const dmb_ctx *ctx);
// Record an error on the context (or the creation error when ctx is NULL) and return s.
dmb_status dmb_internal_fail(dmb_ctx *ctx, dmb_status s, const char *msg);
