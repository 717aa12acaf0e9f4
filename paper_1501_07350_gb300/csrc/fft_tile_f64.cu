// fft_tile_f64.cu -- instantiations of the specialised stage kernel for one arithmetic.
#include "fft_tile.cuh"

namespace ofg {

cudaError_t launch_tile_f64(const StageLaunch& L, cudaStream_t st, bool* handled)
{
    if (L.args.G == 4) return launch_tile_g<ArF64, 4>(L, st, handled);
    if (L.args.G == 8) return launch_tile_g<ArF64, 8>(L, st, handled);
    *handled = false;
    return cudaSuccess;
}

}  // namespace ofg
