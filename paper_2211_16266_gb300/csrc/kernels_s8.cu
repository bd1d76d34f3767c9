// Instantiation of the per-pixel kernels for up to 8 source views.
#include "pixel_kernel.cuh"

namespace pmsp {
template cudaError_t launch_pixel_kernel_ns<8>(const PixelParams&, int, cudaStream_t);
}  // namespace pmsp
