// fft_stage.cu -- one FFT stage of the 3-D transform: batched 1-D DFTs along
// the fastest axis of an ordering, with the transpose to the next ordering
// folded into the store (variant V2) or a plain contiguous store (V0/V1).
//
// Paper mapping (Duy & Ozaki, Sec. 3.1.1): steps (1)-(3) of the execution
// flow -- copy a line into the FFT buffer, transform, copy back -- become one
// pass over HBM: a CTA loads G whole lines into shared memory, runs the
// radix passes there, and writes the lines out; with V2 the write goes
// straight to the positions of the next ordering (steps (4)-(6) fused).
//
// Shared-memory tile: element i of line g lives at tile[i * (G + 1) + g].
//   - load: consecutive threads read consecutive i of one line (coalesced),
//     smem stride G + 1 (odd) -> no bank conflicts;
//   - radix passes: thread (g, slot); the G lanes of a slot touch consecutive
//     words -> no bank conflicts at any pass;
//   - transposed store: consecutive threads take consecutive g at one
//     frequency k, which are consecutive addresses of the next ordering.
//
// Radix pass (Stockham autosort, decimation in time).  After the passes with
// radices r_1..r_p (product m) the line holds, for every residue t < s = n/m,
// the m-point DFT of the subsequence x[t + s u] at positions t m + k.  The
// next radix r (s' = s / r) combines r of them:
//   Y'[t'][k + m q] = sum_j W_r^{j q} (W_{m r}^{j k} Y[t' + s' j][k]),
// with W_{m r}^{j k} = W_n^{j k s'} read from the twiddle table of length n.
#include <type_traits>

#include "fft_stage.h"

#include <algorithm>
#include "arith.cuh"
#include "stage_io.cuh"
#include "generic_stage.cuh"
#include "warp_plan.h"

namespace ofg {

template <class A>
__global__ void __launch_bounds__(kStageThreads, 2)
fft_stage_kernel(const StageArgs p)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ int64_t s_in[kMaxLinesPerCta];
    __shared__ int64_t s_out[kMaxLinesPerCta];
    generic_stage_tile<A>(p, blockIdx.x, smem_raw, s_in, s_out);
}

// ---------------------------------------------------- twiddle tables ----

// W[e] = exp(-2 pi i e / n), from the FP64 sincospi of 2e/n.  A double-float
// table (FMT_DF) holds n float4 entries (hi and lo parts), followed by the
// per-pass table of the packed product (warp_twiddle_kernel): 32 n bytes.
__global__ void twiddle_kernel(int n, int fmt, void* out)
{
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n) return;
    double s, c;
    sincospi((double)(2 * (int64_t)e) / (double)n, &s, &c);
    const double re = c, im = -s;
    if (fmt == FMT_C128) {
        reinterpret_cast<double2*>(out)[e] = make_double2(re, im);
    } else if (fmt == FMT_C64) {
        reinterpret_cast<float2*>(out)[e] = make_float2((float)re, (float)im);
    } else {
        const float hr = (float)re, hi = (float)im;
        const float lr = (float)(re - (double)hr), li = (float)(im - (double)hi);
        reinterpret_cast<float4*>(out)[e] = make_float4(hr, hi, lr, li);
    }
}

// The per-pass twiddle tables of the warp kernel's radix plan for the packed
// double-float product (arith_pair.cuh, warp_plan.h): entry e of pass p is
// W_n^(j k s_p), stored as the float4 (hi re, hi im, lo re, lo im) in a
// second array of n slots after the n float4 entries of the FMT_DF table.
__global__ void warp_twiddle_kernel(int n, void* out)
{
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= wtw_count(n)) return;
    int p = 1;
    while (p + 1 < wplan_len(n) && e >= wtw_offset(n, p + 1)) ++p;
    const int m = wplan_m(n, p), R = wplan_radix(n, p);
    const int s = n / (m * R);
    const int j = (e - wtw_offset(n, p)) / m + 1, k = (e - wtw_offset(n, p)) % m;
    const int ex = (int)(((int64_t)j * k * s) % n);
    double sn, c;
    sincospi((double)(2 * (int64_t)ex) / (double)n, &sn, &c);
    const double re = c, im = -sn;
    const float hr = (float)re, hi = (float)im;
    const float lr = (float)(re - (double)hr), li = (float)(im - (double)hi);
    float4* a = reinterpret_cast<float4*>(reinterpret_cast<char*>(out) + 16 * (size_t)n);
    a[e] = make_float4(hr, hi, lr, li);
}

// --------------------------------------------------------- host side ----

cudaError_t persistent_ctas_per_sm(const void* func, int threads, size_t dyn_smem, int* per_sm)
{
    // cudaOccupancyMaxActiveBlocksPerMultiprocessor has been seen to count one
    // CTA per SM where two were resident, so the limits are applied here; the
    // carveout is then set to what those CTAs need, leaving the rest as L1
    // (which the twiddle loads use)
    cudaError_t e = cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn_smem);
    cudaFuncAttributes fa;
    if (!e) e = cudaFuncGetAttributes(&fa, func);
    if (e) return e;
    int dev = 0, smem_sm = 0, resv = 0, regs_sm = 0, thr_sm = 0, blk_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
    cudaDeviceGetAttribute(&resv, cudaDevAttrReservedSharedMemoryPerBlock, dev);
    cudaDeviceGetAttribute(&regs_sm, cudaDevAttrMaxRegistersPerMultiprocessor, dev);
    cudaDeviceGetAttribute(&thr_sm, cudaDevAttrMaxThreadsPerMultiProcessor, dev);
    cudaDeviceGetAttribute(&blk_sm, cudaDevAttrMaxBlocksPerMultiprocessor, dev);
    const long cta_smem = (long)dyn_smem + (long)fa.sharedSizeBytes + resv;
    const long warps = (threads + 31) / 32;
    const long cta_regs = (long)((fa.numRegs + 7) & ~7) * 32 * warps;
    long n = blk_sm > 0 ? blk_sm : 32;
    if (cta_smem > 0 && smem_sm > 0) n = std::min(n, (long)smem_sm / cta_smem);
    if (cta_regs > 0) n = std::min(n, (long)regs_sm / cta_regs);
    n = std::min(n, (long)thr_sm / (32 * warps));
    if (n < 1) n = 1;
    *per_sm = (int)n;
    if (smem_sm > 0) {
        const long pct = std::min(100L, (100 * n * cta_smem + smem_sm - 1) / smem_sm + 2);
        e = cudaFuncSetAttribute(func, cudaFuncAttributePreferredSharedMemoryCarveout, (int)pct);
    }
    return e;
}

cudaError_t stage_kernels_init(int max_dyn_smem)
{
    cudaError_t e;
    if ((e = cudaFuncSetAttribute(fft_stage_kernel<ArF64>, cudaFuncAttributeMaxDynamicSharedMemorySize, max_dyn_smem))) return e;
    if ((e = cudaFuncSetAttribute(fft_stage_kernel<ArF32>, cudaFuncAttributeMaxDynamicSharedMemorySize, max_dyn_smem))) return e;
    return cudaFuncSetAttribute(fft_stage_kernel<ArDF>, cudaFuncAttributeMaxDynamicSharedMemorySize, max_dyn_smem);
}

#ifdef OPENFFT_CHECKED
__device__ int g_bounds_status;       // status word of launches whose plan has none
#endif

int* fallback_status_word()
{
#ifdef OPENFFT_CHECKED
    void* ptr = nullptr;
    if (cudaGetSymbolAddress(&ptr, g_bounds_status) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return static_cast<int*>(ptr);
#else
    return nullptr;
#endif
}

cudaError_t launch_stage(const StageLaunch& L0, cudaStream_t st)
{
    StageLaunch L = L0;
    const int64_t elems = L.args.M1 * L.args.M2 * (int64_t)L.args.n;
    if (!L.args.in_elems) L.args.in_elems = elems;
    if (!L.args.out_elems) L.args.out_elems = elems;
    if (!L.args.chk) L.args.chk = L.status ? L.status : fallback_status_word();
    if (L.family == KERNEL_R2C || L.family == KERNEL_C2R) return launch_real_stage(L, st);
    if (L.arith == ARITH_TC_TF32 || L.arith == ARITH_TC_BF16) return launch_dftgemm(L, st, L.status);
    bool handled = false;
    cudaError_t e = cudaSuccess;
    if (L.args.do_fft && L.family != KERNEL_GENERIC) {
        switch (L.arith) {
        case ARITH_F64: e = launch_tile_f64(L, st, &handled); break;
        case ARITH_F32: e = launch_tile_f32(L, st, &handled); break;
        default: e = launch_tile_df(L, st, &handled); break;
        }
        if (handled || e) return e;
    }
    const unsigned grid = (unsigned)L.grid;
    switch (L.arith) {
    case ARITH_F64: fft_stage_kernel<ArF64><<<grid, kStageThreads, L.smem, st>>>(L.args); break;
    case ARITH_F32: fft_stage_kernel<ArF32><<<grid, kStageThreads, L.smem, st>>>(L.args); break;
    default: fft_stage_kernel<ArDF><<<grid, kStageThreads, L.smem, st>>>(L.args); break;
    }
    return cudaGetLastError();
}

cudaError_t launch_twiddles(int n, int fmt, void* out, cudaStream_t st)
{
    twiddle_kernel<<<(n + 255) / 256, 256, 0, st>>>(n, fmt, out);
    if (fmt == FMT_DF && warp_length(n)) warp_twiddle_kernel<<<(wtw_count(n) + 255) / 256, 256, 0, st>>>(n, out);
    return cudaGetLastError();
}

}  // namespace ofg
