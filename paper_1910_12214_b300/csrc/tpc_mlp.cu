// BF16 MLP surrogate of the space-point correction (placeholder until the
// network kernels are in place).
#include <cuda_runtime.h>

#include "tpc.h"
#include "tpc_internal.cuh"

cudaError_t tpc_launch_mlp_correction(const Buffers& b, cudaStream_t s) {
  (void)b;
  (void)s;
  return cudaErrorNotSupported;
}
