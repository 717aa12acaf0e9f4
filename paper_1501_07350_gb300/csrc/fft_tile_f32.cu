// fft_tile_f32.cu -- instantiations of the specialised stage kernels for one arithmetic:
// warp-per-line kernels for power-of-two lengths, tile kernels for the others.
// 256- and 512-point transposed stages take the asynchronous-output version
// (fft_tma_f32.cu) whenever the stage's output has its view.
#include "fft_tile.cuh"
#include "fft_warp.cuh"

namespace ofg {

cudaError_t launch_tile_f32(const StageLaunch& L, cudaStream_t st, bool* handled)
{
    *handled = false;
    if ((L.family == KERNEL_AUTO || L.family == KERNEL_WARP) && (L.args.n == 256 || L.args.n == 512)) {
        cudaError_t e = launch_warp_tma_f32(L, st, handled);
        if (*handled || e) return e;
    }
    if ((L.family == KERNEL_AUTO || L.family == KERNEL_WARP) && (L.args.G == 8 || L.args.G == 16)) {
        cudaError_t e = L.args.G == 8 ? launch_warp_g<ArF32, 8>(L, st, handled) : launch_warp_g<ArF32, 16>(L, st, handled);
        if (*handled || e) return e;
    }
    if ((L.family == KERNEL_AUTO || L.family == KERNEL_WARP) && warp_mixed_length(L.args.n)) {
        cudaError_t e = launch_warp_mixed_f32(L, st, handled);
        if (*handled || e) return e;
    }
    if (L.family == KERNEL_WARP) return cudaSuccess;
    if (L.args.G == 8) return launch_tile_g<ArF32, 8>(L, st, handled);
    if (L.args.G == 16) return launch_tile_g<ArF32, 16>(L, st, handled);
    return cudaSuccess;
}

}  // namespace ofg
