// Persistent batched kernel for batches whose keyframes have at most 4 source views.
#include "batch_kernel.cuh"

namespace pmsp {
template int batch_kernel_blocks_per_sm_t<4>();
template cudaError_t launch_batch_kernel_t<4>(const BatchArgs&, int, cudaStream_t);
}  // namespace pmsp
