// fft_tile_df.cu -- instantiations of the specialised stage kernels for one arithmetic:
// warp-per-line kernels for power-of-two lengths, tile kernels for the others.
// The double-float warp kernels run the packed-lane policy (arith_pair.cuh);
// 256- and 512-point lines take the asynchronous-output kernel
// (fft_warp_tma.cuh, fft_tma_*.cu) whenever the stage's output has its view.
#include "fft_tile.cuh"
#include "fft_warp.cuh"

namespace ofg {

cudaError_t launch_tile_df(const StageLaunch& L, cudaStream_t st, bool* handled)
{
    *handled = false;
    if ((L.family == KERNEL_AUTO || L.family == KERNEL_WARP) && (L.args.n == 256 || L.args.n == 512)) {
        cudaError_t e = L.args.n == 256 ? launch_warp_tma_256(L, st, handled) : launch_warp_tma_512(L, st, handled);
        if (*handled || e) return e;
    }
    if ((L.family == KERNEL_AUTO || L.family == KERNEL_WARP) && (L.args.G == 4 || L.args.G == 8)) {
        cudaError_t e = L.args.G == 4 ? launch_warp_g<ArDP, 4>(L, st, handled) : launch_warp_g<ArDP, 8>(L, st, handled);
        if (*handled || e) return e;
    }
    if ((L.family == KERNEL_AUTO || L.family == KERNEL_WARP) && warp_mixed_length(L.args.n)) {
        cudaError_t e = launch_warp_mixed_df(L, st, handled);
        if (*handled || e) return e;
    }
    if (L.family == KERNEL_WARP) return cudaSuccess;
    if (L.args.G == 4) return launch_tile_g<ArDF, 4>(L, st, handled);
    if (L.args.G == 8) return launch_tile_g<ArDF, 8>(L, st, handled);
    return cudaSuccess;
}

}  // namespace ofg
