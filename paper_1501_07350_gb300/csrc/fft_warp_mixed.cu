// fft_warp_mixed.cu -- the warp-per-line stage kernel (fft_warp.cuh) for the
// mixed-radix line lengths 48, 96, 100, 108, 120, 144 and 160, in the packed
// double-float and the FP32 arithmetic.  Lines shorter than 256 points share
// a warp in lane groups, so the radix passes synchronise warps, not the CTA
// (the tile kernel's passes synchronise the CTA).
#include "fft_warp.cuh"

namespace ofg {

namespace {

template <class A, int G>
cudaError_t launch_warp_mixed_g(const StageLaunch& L, cudaStream_t st, bool* handled)
{
    const StageArgs& a = L.args;
    if (a.contig_store && (a.group_i2 || a.S1 != a.n || a.Sk != 1)) return cudaSuccess;
    *handled = true;
    switch (a.n) {
    case 48: return launch_warp_n<A, 48, G>(L, st);
    case 96: return launch_warp_n<A, 96, G>(L, st);
    case 100: return launch_warp_n<A, 100, G>(L, st);
    case 108: return launch_warp_n<A, 108, G>(L, st);
    case 120: return launch_warp_n<A, 120, G>(L, st);
    case 144: return launch_warp_n<A, 144, G>(L, st);
    case 160: return launch_warp_n<A, 160, G>(L, st);
    default: *handled = false; return cudaSuccess;
    }
}

}  // namespace

cudaError_t launch_warp_mixed_df(const StageLaunch& L, cudaStream_t st, bool* handled)
{
    *handled = false;
    if (L.args.G == 4) return launch_warp_mixed_g<ArDP, 4>(L, st, handled);
    if (L.args.G == 8) return launch_warp_mixed_g<ArDP, 8>(L, st, handled);
    return cudaSuccess;
}

cudaError_t launch_warp_mixed_f32(const StageLaunch& L, cudaStream_t st, bool* handled)
{
    *handled = false;
    if (L.args.G == 8) return launch_warp_mixed_g<ArF32, 8>(L, st, handled);
    if (L.args.G == 16) return launch_warp_mixed_g<ArF32, 16>(L, st, handled);
    return cudaSuccess;
}

}  // namespace ofg
