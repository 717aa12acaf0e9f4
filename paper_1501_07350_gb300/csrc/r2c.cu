// r2c.cu -- the real stages of the real 3-D transform (OPENFFT_R2C_F64 /
// OPENFFT_R2C_F32): the first stage of the forward transform (real c-lines ->
// half spectra, frequencies 0..n/2) and the last stage of the inverse (half
// spectra -> real c-lines).  The complex stages in between are the ordinary
// stage kernels run on the half arrays.
//
// Two real lines travel as one complex line z = x1 + i x2.
//   Forward: Z = DFT(z); with Zr[k] = conj Z[(n - k) mod n] the two spectra
//   are X1 = (Z + Zr) / 2 and X2 = -i (Z - Zr) / 2, and their frequencies
//   0..n/2 are stored, transposed, into the half array of the next ordering.
//   Inverse: the inverse pipeline conjugates on entry, so the half spectrum V
//   that reaches this stage gives the real line as the forward DFT of V's
//   Hermitian extension (a real result: the exit conjugation is void).  The
//   complex line is Z[k] = V1[k] + i V2[k] and Z[n - k] = conj V1[k] +
//   i conj V2[k] for 0 < k < n - k; Z[0] and, for even n, Z[n/2] take the real
//   parts of V1 and V2 only.  Re and Im of DFT(Z), times the scale, are the
//   two real lines.
//
// Power-of-two n (32..512): one warp per complex line (a pair of real lines)
// in the padded per-warp layout of the warp-per-line stage kernel, with its
// radix passes; persistent CTAs of 8 warps.  Other n: one CTA per tile of 2G
// real lines (G complex lines) in two ping-pong [n][G + 1] shared-memory
// tiles, with the radix passes of the generic stage kernel (any supported n,
// runtime radix plan).
#include <cuda_runtime.h>

#include "fft_stage.h"
#include "fft_warp.cuh"
#include "generic_stage.cuh"
#include "stage_io.cuh"

namespace ofg {

namespace {

// Two real values <-> one complex element, per arithmetic.
template <class A> struct RealPair;

// Scale is the output factor in the form `part` applies it (prepared once per
// thread by scale_of).
template <> struct RealPair<ArF64> {
    using T = double;
    using Scale = double;
    static constexpr bool kDF = false;
    __device__ __forceinline__ static double2 make(double a, double b) { return make_double2(a, b); }
    __device__ __forceinline__ static double2 re_parts(double2 u, double2 v) { return make_double2(u.x, v.x); }
    __device__ __forceinline__ static Scale scale_of(double s) { return s; }
    __device__ __forceinline__ static double part(double2 z, int im, Scale s) { return (im ? z.y : z.x) * s; }
};

template <> struct RealPair<ArF32> {
    using T = float;
    using Scale = float;
    static constexpr bool kDF = false;
    __device__ __forceinline__ static float2 make(float a, float b) { return make_float2(a, b); }
    __device__ __forceinline__ static float2 re_parts(float2 u, float2 v) { return make_float2(u.x, v.x); }
    __device__ __forceinline__ static Scale scale_of(double s) { return (float)s; }
    __device__ __forceinline__ static float part(float2 z, int im, Scale s) { return (im ? z.y : z.x) * s; }
};

// double-float: (re.hi, im.hi, re.lo, im.lo).  The output factor is split
// into floats (kh + kl) once, and the product is formed in double-float on
// the FP32 units (exact kh * hi plus first-order terms) before the single
// FP64 addition of the join.
template <> struct RealPair<ArDF> {
    using T = double;
    using Scale = float2;
    static constexpr bool kDF = true;
    __device__ __forceinline__ static float4 make(double a, double b) {
        const float2 ha = split_f64(a), hb = split_f64(b);
        return make_float4(ha.x, hb.x, ha.y, hb.y);
    }
    __device__ __forceinline__ static float4 re_parts(float4 u, float4 v) { return make_float4(u.x, v.x, u.z, v.z); }
    __device__ __forceinline__ static Scale scale_of(double s) {
        const float kh = (float)s;
        return make_float2(kh, (float)(s - (double)kh));
    }
    __device__ __forceinline__ static double part(float4 z, int im, Scale k) {
        const float h = im ? z.y : z.x, l = im ? z.w : z.z;
        const float ph = __fmul_rn(h, k.x);
        const float pl = __fmaf_rn(l, k.x, __fmaf_rn(h, k.y, __fmaf_rn(h, k.x, -ph)));
        return join_f64(ph, pl);
    }
};

// i z, by exact sign changes: conj(-i conj z)
template <class A>
__device__ __forceinline__ typename A::C mul_i(typename A::C z) { return A::conj(A::mul_mi(A::conj(z))); }

// The radix passes of the generic stage on a [n][G + 1] tile; returns the
// tile that holds the result.
template <class A>
__device__ __forceinline__ const typename A::C* tile_passes(const StageArgs& p, typename A::C* buf0,
                                                            typename A::C* buf1, int ld)
{
    using C = typename A::C;
    const int tid = threadIdx.x, n = p.n;
    const int g = tid & (p.G - 1), slot = tid >> p.log2G, slots = kStageThreads >> p.log2G;
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
    return a - g;
}

// Forward real stage.  Real line l (l < p.M1) at in + l n; output element
// (line l, frequency k <= n/2) at out[k Sk + l S1] in p.out_fmt.
template <class A>
__global__ void __launch_bounds__(kStageThreads) r2c_stage_kernel(const StageArgs p)
{
    using C = typename A::C;
    using RP = RealPair<A>;
    using T = typename RP::T;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int tid = threadIdx.x, G = p.G, ld = G + 1, n = p.n;
    C* buf0 = reinterpret_cast<C*>(smem_raw);
    C* buf1 = buf0 + (size_t)n * ld;
    const int64_t L = p.M1, l0 = (int64_t)blockIdx.x * 2 * G;
    const T* x = reinterpret_cast<const T*>(p.in);
    {   // real lines l0 + 2j, l0 + 2j + 1 -> complex line j
        const int dj = kStageThreads / n, di = kStageThreads - dj * n;
        int j = tid / n, i = tid - j * n;
        for (int e = tid; e < G * n; e += kStageThreads) {
            const int64_t la = l0 + 2 * j;
            const T a = la < L ? x[la * n + i] : T(0);
            const T b = la + 1 < L ? x[(la + 1) * n + i] : T(0);
            buf0[i * ld + j] = RP::make(a, b);
            i += di; j += dj;
            if (i >= n) { i -= n; ++j; }
        }
    }
    __syncthreads();
    const C* cur = tile_passes<A>(p, buf0, buf1, ld);
    // separate the two spectra, frequencies 0..n/2 of 2G lines
    const int nh = n / 2 + 1, lg2 = p.log2G + 1;
    for (int e = tid; e < (nh << lg2); e += kStageThreads) {
        const int k = e >> lg2, o = e & ((1 << lg2) - 1);
        const int64_t l = l0 + o;
        if (l >= L) continue;
        const int j = o >> 1;
        const C z = cur[k * ld + j];
        const C zr = A::conj(cur[(k == 0 ? 0 : n - k) * ld + j]);
        const C X = A::scale((o & 1) ? A::mul_mi(A::sub(z, zr)) : A::add(z, zr), 0.5);
        Io<A>::store(p.out, p.out_fmt, (int64_t)k * p.Sk + l * p.S1, X);
    }
}

// Inverse real stage.  Half line l (l < p.M1) at in + l (n/2 + 1), in
// p.in_fmt; real line l at out + l n, times p.scale.
template <class A>
__global__ void __launch_bounds__(kStageThreads) c2r_stage_kernel(const StageArgs p)
{
    using C = typename A::C;
    using RP = RealPair<A>;
    using T = typename RP::T;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int tid = threadIdx.x, G = p.G, ld = G + 1, n = p.n, nh = n / 2 + 1;
    C* buf0 = reinterpret_cast<C*>(smem_raw);
    C* buf1 = buf0 + (size_t)n * ld;
    const int64_t L = p.M1, l0 = (int64_t)blockIdx.x * 2 * G;
    const typename RP::Scale ks = RP::scale_of(p.scale);
    {   // half lines l0 + 2j, l0 + 2j + 1 -> Hermitian-extended complex line j
        const int dj = kStageThreads / nh, dk = kStageThreads - dj * nh;
        int j = tid / nh, k = tid - j * nh;
        for (int e = tid; e < G * nh; e += kStageThreads) {
            const int64_t la = l0 + 2 * j;
            const C v1 = la < L ? Io<A>::load(p.in, p.in_fmt, la * nh + k) : A::zero();
            const C v2 = la + 1 < L ? Io<A>::load(p.in, p.in_fmt, (la + 1) * nh + k) : A::zero();
            if (k == 0 || 2 * k == n) {
                buf0[k * ld + j] = RP::re_parts(v1, v2);
            } else {
                buf0[k * ld + j] = A::add(v1, mul_i<A>(v2));
                buf0[(n - k) * ld + j] = A::add(A::conj(v1), mul_i<A>(A::conj(v2)));
            }
            k += dk; j += dj;
            if (k >= nh) { k -= nh; ++j; }
        }
    }
    __syncthreads();
    const C* cur = tile_passes<A>(p, buf0, buf1, ld);
    T* y = reinterpret_cast<T*>(p.out);
    {   // Re / Im of complex line j -> real lines l0 + 2j / l0 + 2j + 1
        const int dout = kStageThreads / n, di = kStageThreads - dout * n;
        int o = tid / n, i = tid - o * n;
        for (int e = tid; e < 2 * G * n; e += kStageThreads) {
            const int64_t l = l0 + o;
            if (l < L) y[l * n + i] = (T)RP::part(cur[i * ld + (o >> 1)], o & 1, ks);
            i += di; o += dout;
            if (i >= n) { i -= n; ++o; }
        }
    }
}

// ------------------------------------------- warp per pair of real lines --

constexpr int kRealWarpG = 8;       // complex lines (warps) per CTA

// Real lines of lengths up to 256 are staged: each warp copies its two real
// lines of the next tile into shared memory (cp.async) while the current tile
// is transformed.  512-point lines load directly (the staging area would halve
// the CTAs per SM).
template <int N>
constexpr bool r2c_staged() { return N <= 256; }

// cp.async of real lines la, la + 1 (zeros beyond L) into raw[0, 2N)
template <class T, int N>
__device__ __forceinline__ void r2c_issue_raw(const T* __restrict__ x, int64_t L, int64_t la, T* raw, int lane)
{
    constexpr int PER = 16 / (int)sizeof(T);     // reals per 16-byte copy
    constexpr int CH = N / PER;                  // copies per line
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        T* dst = raw + h * N;
        if (la + h < L) {
            const T* src = x + (la + h) * N;
#pragma unroll
            for (int c = lane; c < CH; c += 32) cp_async<16>(dst + c * PER, src + c * PER);
        } else {
#pragma unroll
            for (int pos = lane; pos < N; pos += 32) dst[pos] = T(0);
        }
    }
    cp_async_commit();
}

// Forward real stage, power-of-two N: warp w of tile t takes real lines
// l0 + 2w and l0 + 2w + 1 (l0 = 2 G t); the CTA then separates the spectra of
// its 2G lines and stores frequency k of all of them (2G consecutive
// elements of the half array) at a time.
template <class A, int N, int G>
__global__ void __launch_bounds__(32 * G, warp_min_blocks(32 * G, sizeof(typename A::C)))
r2c_warp_kernel(const StageArgs p, int64_t ntiles)
{
    using C = typename A::C;
    using RP = RealPair<A>;
    using T = typename RP::T;
    constexpr int EB = sizeof(C);
    constexpr int LS = warp_line_stride<EB>(N);
    constexpr int TWO = 2 * G, SLOTS = 32 * G / TWO;
    constexpr bool STAGED = r2c_staged<N>();
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* tile = reinterpret_cast<C*>(smem_raw);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const typename A::W* tw = reinterpret_cast<const typename A::W*>(p.tw);
    const T* x = reinterpret_cast<const T*>(p.in);
    const int64_t L = p.M1;
    C* line = tile + warp * LS;
    T* raw = reinterpret_cast<T*>(tile + G * LS) + warp * 2 * N;     // this warp's staged real lines
    const int o = tid % TWO, slot = tid / TWO;          // store phase: line o of the tile
    const C* oline = tile + (o >> 1) * LS;
    int64_t t = blockIdx.x;
    if (STAGED && t < ntiles) r2c_issue_raw<T, N>(x, L, t * TWO + 2 * warp, raw, lane);
    for (; t < ntiles; t += gridDim.x) {
        const int64_t l0 = t * TWO;
        const int64_t la = l0 + 2 * warp, lb = la + 1;
        if constexpr (STAGED) {
            cp_async_wait_all();
            __syncwarp();
#pragma unroll
            for (int u = 0; u < N / 32; ++u) {
                const int pos = lane + 32 * u;
                line[wpad<EB>(pos)] = RP::make(raw[pos], raw[N + pos]);
            }
            __syncwarp();                                // raw is consumed: refill it with the next tile
            const int64_t tn = t + gridDim.x;
            if (tn < ntiles) r2c_issue_raw<T, N>(x, L, tn * TWO + 2 * warp, raw, lane);
        } else {
#pragma unroll
            for (int u = 0; u < N / 32; ++u) {
                const int pos = lane + 32 * u;
                const T a = la < L ? x[la * N + pos] : T(0);
                const T b = lb < L ? x[lb * N + pos] : T(0);
                line[wpad<EB>(pos)] = RP::make(a, b);
            }
            __syncwarp();
        }
        WarpLine<A, N>::template passes<0>(line, tw, lane);
        __syncthreads();                                 // every line of the tile is transformed
        const int64_t l = l0 + o;
        if (l < L) {
            for (int k = slot; k <= N / 2; k += SLOTS) {
                const C z = oline[wpad<EB>(k)];
                const C zr = A::conj(oline[wpad<EB>(k == 0 ? 0 : N - k)]);
                const C X = A::scale((o & 1) ? A::mul_mi(A::sub(z, zr)) : A::add(z, zr), 0.5);
                Io<A>::store(p.out, p.out_fmt, (int64_t)k * p.Sk + l * p.S1, X);
            }
        }
        __syncthreads();                                 // the tile buffer is free again
    }
    cp_async_wait_all();
}

// Format of the inverse real stage's input that the staged copy keeps as it is
// (the arithmetic's own element): double-float pairs, complex64, complex128.
template <class A>
constexpr int c2r_raw_fmt() { return sizeof(typename A::C) == 8 ? FMT_C64 : (RealPair<A>::kDF ? FMT_DF : FMT_C128); }

// cp.async of half lines la, la + 1 (NH elements each; zeros beyond L) into raw[0, 2 NH)
template <class A, int NH>
__device__ __forceinline__ void c2r_issue_raw(const typename A::C* __restrict__ in, int64_t L, int64_t la,
                                              typename A::C* raw, int lane)
{
    constexpr int EB = sizeof(typename A::C);
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        typename A::C* dst = raw + h * NH;
        if (la + h < L) {
            const typename A::C* src = in + (la + h) * NH;
            for (int k = lane; k < NH; k += 32) cp_async<EB>(dst + k, src + k);
        } else {
            for (int k = lane; k < NH; k += 32) dst[k] = A::zero();
        }
    }
    cp_async_commit();
}

// Inverse real stage, power-of-two N: warp w of tile t extends half lines
// l0 + 2w and l0 + 2w + 1, transforms, and writes the two real lines.  For
// N <= 256 with input in the arithmetic's own format, each warp copies its
// two half lines of the next tile into shared memory (cp.async) while the
// current tile is transformed.
template <class A, int N, int G>
__global__ void __launch_bounds__(32 * G, warp_min_blocks(32 * G, sizeof(typename A::C)))
c2r_warp_kernel(const StageArgs p, int64_t ntiles)
{
    using C = typename A::C;
    using RP = RealPair<A>;
    using T = typename RP::T;
    constexpr int EB = sizeof(C);
    constexpr int LS = warp_line_stride<EB>(N);
    constexpr int NH = N / 2 + 1;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* tile = reinterpret_cast<C*>(smem_raw);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const typename A::W* tw = reinterpret_cast<const typename A::W*>(p.tw);
    T* y = reinterpret_cast<T*>(p.out);
    const int64_t L = p.M1;
    C* line = tile + warp * LS;
    C* raw = tile + G * LS + warp * 2 * NH;              // this warp's staged half lines
    const bool staged = r2c_staged<N>() && p.in_fmt == c2r_raw_fmt<A>();
    const C* in = reinterpret_cast<const C*>(p.in);
    const typename RP::Scale ks = RP::scale_of(p.scale);
    int64_t t = blockIdx.x;
    if (staged && t < ntiles) c2r_issue_raw<A, NH>(in, L, t * 2 * G + 2 * warp, raw, lane);
    for (; t < ntiles; t += gridDim.x) {
        const int64_t la = t * 2 * G + 2 * warp, lb = la + 1;
        if (staged) {
            cp_async_wait_all();
            __syncwarp();
        }
        for (int k = lane; k < NH; k += 32) {
            C v1, v2;
            if (staged) {
                v1 = raw[k];
                v2 = raw[NH + k];
            } else {
                v1 = la < L ? Io<A>::load(p.in, p.in_fmt, la * NH + k) : A::zero();
                v2 = lb < L ? Io<A>::load(p.in, p.in_fmt, lb * NH + k) : A::zero();
            }
            if (k == 0 || 2 * k == N) {
                line[wpad<EB>(k)] = RP::re_parts(v1, v2);
            } else {
                line[wpad<EB>(k)] = A::add(v1, mul_i<A>(v2));
                line[wpad<EB>(N - k)] = A::add(A::conj(v1), mul_i<A>(A::conj(v2)));
            }
        }
        __syncwarp();
        if (staged) {                                    // raw is consumed: refill it with the next tile
            const int64_t tn = t + gridDim.x;
            if (tn < ntiles) c2r_issue_raw<A, NH>(in, L, tn * 2 * G + 2 * warp, raw, lane);
        }
        WarpLine<A, N>::template passes<0>(line, tw, lane);
#pragma unroll
        for (int u = 0; u < N / 32; ++u) {
            const int pos = lane + 32 * u;
            const C z = line[wpad<EB>(pos)];
            if (la < L) y[la * N + pos] = (T)RP::part(z, 0, ks);
            if (lb < L) y[lb * N + pos] = (T)RP::part(z, 1, ks);
        }
        __syncwarp();                                    // the line is free again
    }
    cp_async_wait_all();
}

template <class A, int N>
cudaError_t launch_real_warp(const StageLaunch& L, cudaStream_t st)
{
    constexpr int G = kRealWarpG;
    const bool fwd = L.family == KERNEL_R2C;
    // tile of G complex lines, and for the staged forward kernel the 2G real lines of the next tile
    const size_t smem = (size_t)G * warp_line_stride<sizeof(typename A::C)>(N) * sizeof(typename A::C) +
                        (!r2c_staged<N>() ? 0
                         : fwd ? (size_t)G * 2 * N * sizeof(typename RealPair<A>::T)
                               : (size_t)G * 2 * (N / 2 + 1) * sizeof(typename A::C));
    static int cached_r2c[kMaxDevices] = {}, cached_c2r[kMaxDevices] = {};   // CTAs per SM, 0 = unknown
    int* slot = device_slot(fwd ? cached_r2c : cached_c2r);
    int per_sm = slot ? *slot : 0;
    if (per_sm == 0) {
        cudaError_t e = fwd ? persistent_ctas_per_sm((const void*)r2c_warp_kernel<A, N, G>, 32 * G, smem, &per_sm)
                            : persistent_ctas_per_sm((const void*)c2r_warp_kernel<A, N, G>, 32 * G, smem, &per_sm);
        if (e) return e;
        if (slot) *slot = per_sm;
    }
    const int64_t ntiles = (L.args.M1 + 2 * G - 1) / (2 * G);
    int64_t grid = (int64_t)L.sms * per_sm;
    if (grid > ntiles) grid = ntiles;
    if (grid < 1) grid = 1;
    if (fwd) r2c_warp_kernel<A, N, G><<<(unsigned)grid, 32 * G, smem, st>>>(L.args, ntiles);
    else c2r_warp_kernel<A, N, G><<<(unsigned)grid, 32 * G, smem, st>>>(L.args, ntiles);
    return cudaGetLastError();
}

template <class A>
cudaError_t launch_real_a(const StageLaunch& L, cudaStream_t st)
{
    switch (L.args.n) {
    case 32: return launch_real_warp<A, 32>(L, st);
    case 64: return launch_real_warp<A, 64>(L, st);
    case 128: return launch_real_warp<A, 128>(L, st);
    case 256: return launch_real_warp<A, 256>(L, st);
    case 512: return launch_real_warp<A, 512>(L, st);
    default: break;
    }
    static int attr_r2c[kMaxDevices] = {}, attr_c2r[kMaxDevices] = {};     // attribute set on that device
    const unsigned grid = (unsigned)L.grid;
    if (L.family == KERNEL_R2C) {
        int* slot = device_slot(attr_r2c);
        if (!slot || !*slot) {
            cudaError_t e = cudaFuncSetAttribute(r2c_stage_kernel<A>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                 200 * 1024);
            if (e) return e;
            if (slot) *slot = 1;
        }
        r2c_stage_kernel<A><<<grid, kStageThreads, L.smem, st>>>(L.args);
    } else {
        int* slot = device_slot(attr_c2r);
        if (!slot || !*slot) {
            cudaError_t e = cudaFuncSetAttribute(c2r_stage_kernel<A>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                 200 * 1024);
            if (e) return e;
            if (slot) *slot = 1;
        }
        c2r_stage_kernel<A><<<grid, kStageThreads, L.smem, st>>>(L.args);
    }
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_real_stage(const StageLaunch& L, cudaStream_t st)
{
    switch (L.arith) {
    case ARITH_F64: return launch_real_a<ArF64>(L, st);
    case ARITH_F32: return launch_real_a<ArF32>(L, st);
    default: return launch_real_a<ArDF>(L, st);
    }
}

}  // namespace ofg
