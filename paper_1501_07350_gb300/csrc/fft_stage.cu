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
#include "arith.cuh"
#include "stage_io.cuh"

namespace ofg {

// ------------------------------------------------------------ one pass ----

// Out of place between the two shared-memory tiles: each butterfly is read,
// twiddled, transformed and written to `dst` on its own, so only one
// butterfly is live per thread and one barrier ends the pass.
template <class A, int R>
__device__ __forceinline__ void radix_pass(const typename A::C* src, typename A::C* dst, int ld, int n,
                                           int m, int s, int slot, int slots,
                                           const typename A::W* __restrict__ tw)
{
    using C = typename A::C;
    const int nbf = n / R;
    // butterfly b = slot + u * slots -> (t, k) = (b / m, b % m), stepped without division
    const int dt = slots / m, dk = slots - dt * m;
    int t = slot / m, k = slot - t * m;
#pragma unroll 2
    for (int b = slot; b < nbf; b += slots) {
        C v[R];
#pragma unroll
        for (int j = 0; j < R; ++j) v[j] = src[((t + s * j) * m + k) * ld];
        if (k != 0) {
#pragma unroll
            for (int j = 1; j < R; ++j) v[j] = A::mul(v[j], __ldg(tw + j * k * s));
        }
        Dft<A, R>::run(v);
#pragma unroll
        for (int q = 0; q < R; ++q) dst[(t * m * R + k + m * q) * ld] = v[q];
        t += dt; k += dk;
        if (k >= m) { k -= m; ++t; }
    }
    __syncthreads();
}

// ---------------------------------------------------------- the kernel ----

template <class A>
__global__ void __launch_bounds__(kStageThreads, 2)
fft_stage_kernel(const StageArgs p)
{
    using C = typename A::C;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int tid = threadIdx.x;
    const int G = p.G, ld = G + 1, n = p.n;
    C* buf0 = reinterpret_cast<C*>(smem_raw);
    C* buf1 = buf0 + (size_t)n * ld;
    __shared__ int64_t s_in[kMaxLinesPerCta];
    __shared__ int64_t s_out[kMaxLinesPerCta];

    if (tid < G) {
        const int64_t cta = blockIdx.x;
        const int64_t outer = cta / p.ngroups, grp = cta - outer * p.ngroups;
        int64_t i1, i2;
        bool ok;
        if (!p.group_i2) { i1 = grp * G + tid; i2 = outer; ok = i1 < p.M1; }
        else             { i2 = grp * G + tid; i1 = outer; ok = i2 < p.M2; }
        s_in[tid] = ok ? (i1 + i2 * p.M1) * (int64_t)n : -1;
        s_out[tid] = ok ? i1 * p.S1 + i2 * p.S2 : -1;
    }
    __syncthreads();

    // (1) lines -> shared memory: every element is one asynchronous copy, so
    // all of the CTA's loads are in flight at once; format conversion and
    // conjugation follow in place, by the thread that issued the copy.
    const int total = G * n;
    {
        constexpr int EB = sizeof(C) >= 16 ? 16 : 8;       // bytes copied per element
        const char* src = reinterpret_cast<const char*>(p.in);
        const int dg = kStageThreads / n, di = kStageThreads - dg * n;
        int g = tid / n, i = tid - g * n;
        for (int e = tid; e < total; e += kStageThreads) {
            const int64_t base = s_in[g];
            C* dst = buf0 + i * ld + g;
            if (base >= 0) cp_async<EB>(dst, src + (base + i) * EB);
            else *dst = A::zero();
            i += di; g += dg;
            if (i >= n) { i -= n; ++g; }
        }
        cp_async_wait_all();
        const bool convert = sizeof(C) == 16 && p.in_fmt == FMT_C128 && EB == 16 && !std::is_same<A, ArF64>::value;
        if (convert || p.conj_in) {
            g = tid / n; i = tid - g * n;
            for (int e = tid; e < total; e += kStageThreads) {
                C* dst = buf0 + i * ld + g;
                C v;
                if (convert) v = Io<A>::from_c128(*reinterpret_cast<const double2*>(dst));
                else v = *dst;
                if (p.conj_in) v = A::conj(v);
                *dst = v;
                i += di; g += dg;
                if (i >= n) { i -= n; ++g; }
            }
        }
    }
    __syncthreads();

    // (2) radix passes, ping-pong between buf0 and buf1
    const C* cur = buf0;
    if (p.do_fft) {
        const int g = tid & (G - 1), slot = tid >> p.log2G, slots = kStageThreads >> p.log2G;
        C* a = buf0 + g;
        C* b = buf1 + g;
        const typename A::W* tw = reinterpret_cast<const typename A::W*>(p.tw);
        int m = 1;
        for (int ps = 0; ps < p.npass; ++ps) {
            const int r = p.radix[ps];
            const int s = n / (m * r);
            switch (r) {
            case 8: radix_pass<A, 8>(a, b, ld, n, m, s, slot, slots, tw); break;
            case 4: radix_pass<A, 4>(a, b, ld, n, m, s, slot, slots, tw); break;
            case 2: radix_pass<A, 2>(a, b, ld, n, m, s, slot, slots, tw); break;
            case 3: radix_pass<A, 3>(a, b, ld, n, m, s, slot, slots, tw); break;
            case 5: radix_pass<A, 5>(a, b, ld, n, m, s, slot, slots, tw); break;
            default: radix_pass<A, 7>(a, b, ld, n, m, s, slot, slots, tw); break;
            }
            m *= r;
            C* t = a; a = b; b = t;
        }
        cur = a - g;
    }

    // (3) shared memory -> next ordering
    const bool scale = p.scale != 1.0;
    if (p.contig_store) {
        const int dg = kStageThreads / n, di = kStageThreads - dg * n;
        int g = tid / n, k = tid - g * n;
        for (int e = tid; e < total; e += kStageThreads) {
            const int64_t base = s_out[g];
            if (base >= 0) {
                C v = cur[k * ld + g];
                if (p.conj_out) v = A::conj(v);
                if (scale) v = A::scale(v, p.scale);
                Io<A>::store(p.out, p.out_fmt, base + k * p.Sk, v);
            }
            k += di; g += dg;
            if (k >= n) { k -= n; ++g; }
        }
    } else {
        for (int e = tid; e < total; e += kStageThreads) {
            const int k = e >> p.log2G, g = e & (G - 1);
            const int64_t base = s_out[g];
            if (base < 0) continue;
            C v = cur[k * ld + g];
            if (p.conj_out) v = A::conj(v);
            if (scale) v = A::scale(v, p.scale);
            Io<A>::store(p.out, p.out_fmt, base + k * p.Sk, v);
        }
    }
}

// ---------------------------------------------------- twiddle tables ----

// W[e] = exp(-2 pi i e / n), from the FP64 sincospi of 2e/n.
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
        reinterpret_cast<float4*>(out)[e] =
            make_float4(hr, hi, (float)(re - (double)hr), (float)(im - (double)hi));
    }
}

// --------------------------------------------------------- host side ----

cudaError_t stage_kernels_init(int max_dyn_smem)
{
    cudaError_t e;
    if ((e = cudaFuncSetAttribute(fft_stage_kernel<ArF64>, cudaFuncAttributeMaxDynamicSharedMemorySize, max_dyn_smem))) return e;
    if ((e = cudaFuncSetAttribute(fft_stage_kernel<ArF32>, cudaFuncAttributeMaxDynamicSharedMemorySize, max_dyn_smem))) return e;
    return cudaFuncSetAttribute(fft_stage_kernel<ArDF>, cudaFuncAttributeMaxDynamicSharedMemorySize, max_dyn_smem);
}

cudaError_t launch_stage(const StageLaunch& L, cudaStream_t st)
{
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
    return cudaGetLastError();
}

}  // namespace ofg
