// Instantiation of the per-pixel kernels for exactly 3 source views.
#include "pixel_lanes.cuh"
#include "pixel_split.cuh"

namespace pmsp {
template cudaError_t launch_pixel_kernel_ns<3, true>(const PixelParams&, int, cudaStream_t);
}  // namespace pmsp
