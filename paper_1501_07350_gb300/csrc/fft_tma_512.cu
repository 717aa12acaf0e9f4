// fft_tma_512.cu -- instantiations of the asynchronous-output stage kernel
// (fft_warp_tma.cuh) for 512-point lines.
#include "fft_warp_tma.cuh"

namespace ofg {

cudaError_t launch_warp_tma_512(const StageLaunch& L, cudaStream_t st, bool* handled)
{
    if (L.args.G == 8) return launch_warp_tma_n<512, 8>(L, st, handled);
    if (L.args.G == 4) return launch_warp_tma_n<512, 4>(L, st, handled);
    *handled = false;
    return cudaSuccess;
}

}  // namespace ofg
