// fft_warp_tma.cuh -- the double-float warp-per-line stage kernel with an
// asynchronous output path, for 256- and 512-point lines in tiles of 4 or 8.
//
// The radix passes are those of fft_warp.cuh (packed double-float policy,
// per-pass twiddle tables).  What differs is the output: the last radix pass
// writes its results into a staging area laid out as the output needs them,
// and one thread hands the whole tile to the tensor memory accelerator (a TMA
// tensor store, or one bulk copy per line for contiguous output), which
// drains it while the CTA goes on with the next tile.
// Transposed output (the fused transposes of steps (4)-(6), Sec. 3.1.1): the
// tile's G lines are consecutive in the output at every frequency k, so the
// staging area is [k][G lines] of 16-byte elements in the swizzle of the
// tensor store (rows of 128 bytes, 16-byte chunk index XOR row mod 8, for
// G = 8; rows of 64 bytes, chunk XOR (row / 2) mod 4, for G = 4), which also
// keeps the last pass's shared-memory writes free of bank conflicts.  The
// tensor map views the output as (grouped line coordinate, frequency, other
// line coordinate) with element strides (1, Sk, So).
//
// Tile layout: the tile's lines, which the staging area overlays once every
// line's last-pass inputs are in registers (a CTA barrier); the next tile's
// copies (cp.async) start when the copy engine has read the staging area.
// The lines are the CTA's only shared memory (19 KB for 4 lines of 256
// points, 38 KB for 4 of 512), so many CTAs stay resident (8 and 4 per SM,
// 32 warps) and one CTA's loads overlap the others' passes.  Measured on
// 256^3 this beat two input buffers with a separate staging area (4 CTAs per
// SM) by 6 %; on 512^3 double buffering with 3 CTAs per SM was 9 % slower.
#pragma once
#include <cuda.h>

#include <cstring>

#include "fft_warp.cuh"

namespace ofg {

__device__ __forceinline__ uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void tma_store_3d(const CUtensorMap* map, uint32_t src, int x, int y, int z)
{
    asm volatile("cp.async.bulk.tensor.3d.global.shared::cta.bulk_group [%0, {%2, %3, %4}], [%1];"
                 :: "l"(map), "r"(src), "r"(x), "r"(y), "r"(z) : "memory");
}
__device__ __forceinline__ void bulk_store(void* dst, uint32_t src, uint32_t bytes)
{
    asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" :: "l"(dst), "r"(src), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
// the copy engine has read every committed group's shared memory
__device__ __forceinline__ void bulk_wait_read_all() { asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory"); }
// every committed group is complete
__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }
// make this thread's generic-proxy shared-memory writes visible to the copy engine
__device__ __forceinline__ void fence_proxy_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
// the passes of line g synchronise the WPL warps that share it: the warp
// itself, or named barrier 1 + g (barrier 0 is the CTA's)
template <int WPL>
__device__ __forceinline__ void line_sync(int g)
{
    if constexpr (WPL == 1) __syncwarp();
    else asm volatile("bar.sync %0, %1;" ::"r"(1 + g), "r"(32 * WPL) : "memory");
}

// warps per line.  512-point lines take two: each lane then holds one
// radix-8 butterfly (8 values) instead of two, which halves the registers a
// thread needs (64) and doubles the resident warps per SM (32) for the same
// shared memory; measured 5 % faster on 512^3 than one warp per line (4-line
// CTAs), 4 % with 8-line CTAs.  256-point lines keep one: their 4 x 8 x 8 plan
// has 32 radix-8 butterflies per pass, and a second warp would idle there.
template <int N, int G>
constexpr int tma_wpl() { return N == 512 ? 2 : 1; }
// CTAs per SM the register allocation is sized for: 64 registers a thread,
// 32 warps per SM
template <int N, int G>
constexpr int tma_min_ctas() { return G == 8 ? (N == 512 ? 2 : 4) : (N == 256 ? 8 : 4); }

// byte offset of output element (frequency k, tile line g) in the transposed
// staging area: the tensor store's swizzle for rows of G x 16 bytes
template <int G>
__device__ __forceinline__ uint32_t staged_offset(int k, int g)
{
    if constexpr (G == 8) return (uint32_t)k * 128u + ((uint32_t)(g ^ (k & 7)) << 4);
    else return (uint32_t)k * 64u + ((uint32_t)(g ^ ((k >> 1) & 3)) << 4);
}

template <int N, int WPL>
struct TmaLine {
    using A = ArDP;
    using C = ArDP::C;
    using W = ArDP::W;
    static constexpr int kPasses = wplan_len(N);
    static constexpr int LS = warp_line_stride<16>(N);
    static_assert(kPasses >= 2, "the entry fix-up rides on an in-place first pass");

    // butterflies of pass P taken by part w of the line's threads.  FIX (first
    // pass only) is the entry fix-up of the stage's input, applied to each
    // value as the butterfly reads it: bit 1, the shared-memory line holds
    // complex128 (converted to double-float here); bit 0, conjugate (backward
    // transform).  Reading and fixing in one step saves a pass over the line.
    template <int P, int FIX = 0>
    __device__ __forceinline__ static void butterflies(const C* line, const W* __restrict__ tw, int lane, int w,
                                                       C (*v)[8], bool* ok)
    {
        constexpr int R = wplan_radix(N, P);
        constexpr int m = wplan_m(N, P);
        constexpr int s = N / (m * R);
        constexpr int NBF = N / R;
        constexpr int NB = (NBF + 32 * WPL - 1) / (32 * WPL);
#pragma unroll
        for (int u = 0; u < NB; ++u) {
            const int b = lane + 32 * (w + WPL * u);
            ok[u] = NBF % (32 * WPL) == 0 || b < NBF;
            if (ok[u]) {
#pragma unroll
                for (int j = 0; j < R; ++j) {
                    C x = line[wpad<16>(b + j * NBF)];
                    if constexpr ((FIX & 2) != 0)
                        x = Io<ArDP>::from_c128(make_double2(__longlong_as_double((long long)x.x),
                                                             __longlong_as_double((long long)x.y)));
                    if constexpr ((FIX & 1) != 0) x = A::conj(x);
                    v[u][j] = x;
                }
                if (m > 1) {
                    const int k = b % m;
#pragma unroll
                    for (int j = 1; j < R; ++j)
                        v[u][j] = A::mul(v[u][j], A::template warp_twiddle<N>(tw, wtw_offset(N, P), m, j, k, k * s));
                }
                Dft<A, R>::run(v[u]);
            }
        }
    }

    // an in-place pass (all but the last)
    template <int P, int FIX = 0>
    __device__ __forceinline__ static void pass(C* line, const W* __restrict__ tw, int lane, int w, int g)
    {
        constexpr int R = wplan_radix(N, P);
        constexpr int m = wplan_m(N, P);
        constexpr int NBF = N / R;
        constexpr int NB = (NBF + 32 * WPL - 1) / (32 * WPL);
        C v[NB][8];
        bool ok[NB];
        butterflies<P, FIX>(line, tw, lane, w, v, ok);
        line_sync<WPL>(g);
#pragma unroll
        for (int u = 0; u < NB; ++u) {
            if (ok[u]) {
                const int b = lane + 32 * (w + WPL * u);
                const int base = (b / m) * m * R + b % m;
#pragma unroll
                for (int q = 0; q < R; ++q) line[wpad<16>(base + m * q)] = v[u][q];
            }
        }
        line_sync<WPL>(g);
    }

    template <int P, int FIX = 0>
    __device__ __forceinline__ static void passes(C* line, const W* __restrict__ tw, int lane, int w, int g)
    {
        if constexpr (P < kPasses - 1) {
            pass<P, FIX>(line, tw, lane, w, g);
            passes<P + 1, 0>(line, tw, lane, w, g);
        }
    }

    // 16 output bytes of a result: the stage's output format, conjugated and
    // scaled on the backward transform's last stage
    template <bool CONJ_SCALE, bool EXT>
    __device__ __forceinline__ static uint4 out16(C v, double scale)
    {
        if constexpr (CONJ_SCALE) v = A::scale(A::conj(v), scale);
        if constexpr (EXT) {
            const double2 d = df_to_double2(A::to_float4(v));
            uint4 r;
            r.x = (uint32_t)__double_as_longlong(d.x);
            r.y = (uint32_t)((unsigned long long)__double_as_longlong(d.x) >> 32);
            r.z = (uint32_t)__double_as_longlong(d.y);
            r.w = (uint32_t)((unsigned long long)__double_as_longlong(d.y) >> 32);
            return r;
        } else {
            return make_uint4((uint32_t)v.x, (uint32_t)(v.x >> 32), (uint32_t)v.y, (uint32_t)(v.y >> 32));
        }
    }

    // the last pass, into the staging area.  Transposed output: [k][G lines]
    // swizzled rows over the tile's lines, so every line's inputs are read
    // (CTA barrier) before any result is written.  Contiguous output: [k] at
    // the start of the line's own buffer, after the line's warps have read it
    // (line barrier); the line's leader then stores it with one bulk copy, so
    // these stages never synchronise the CTA.
    template <int G, bool CONTIG, bool CONJ_SCALE, bool EXT>
    __device__ __forceinline__ static void last_pass(const C* line, const W* __restrict__ tw, unsigned char* stage,
                                                     int lane, int w, int g, double scale)
    {
        constexpr int P = kPasses - 1;
        constexpr int R = wplan_radix(N, P);
        constexpr int m = wplan_m(N, P);
        constexpr int NBF = N / R;
        constexpr int NB = (NBF + 32 * WPL - 1) / (32 * WPL);
        C v[NB][8];
        bool ok[NB];
        butterflies<P>(line, tw, lane, w, v, ok);
        if constexpr (CONTIG) line_sync<WPL>(g);
        else __syncthreads();
#pragma unroll
        for (int u = 0; u < NB; ++u) {
            if (ok[u]) {
                const int b = lane + 32 * (w + WPL * u);
                const int base = (b / m) * m * R + b % m;
#pragma unroll
                for (int q = 0; q < R; ++q) {
                    const int k = base + m * q;
                    const uint32_t off = CONTIG ? (uint32_t)k * 16u : staged_offset<G>(k, g);
                    *reinterpret_cast<uint4*>(stage + off) = out16<CONJ_SCALE, EXT>(v[u][q], scale);
                }
            }
        }
    }
};

// copies of this thread's share of line g (parts w of WPL)
template <int N, int WPL>
__device__ __forceinline__ void tma_issue_load(const StageArgs& p, const TileGeom& tg, int g, ArDP::C* line,
                                               int lane, int w)
{
    if (g < tg.valid) {
        const char* src = reinterpret_cast<const char*>(p.in) + (tg.line0 + g * tg.lstride) * (int64_t)(N * 16);
#pragma unroll
        for (int u = 0; u < N / (32 * WPL); ++u) {
            const int pos = lane + 32 * (w + WPL * u);
            if (in_bounds(p.chk, (tg.line0 + g * tg.lstride) * N + pos, p.in_elems))
                cp_async<16>(line + wpad<16>(pos), src + pos * 16);
        }
    } else {
#pragma unroll
        for (int u = 0; u < N / (32 * WPL); ++u) line[wpad<16>(lane + 32 * (w + WPL * u))] = ArDP::zero();
    }
    cp_async_commit();
}

template <int N, int G>
constexpr size_t tma_stage_bytes() { return (size_t)N * G * 16; }
// 1024-byte alignment slack (the 128-byte swizzle), then the tile's lines,
// which the staging area overlays
template <int N, int G>
constexpr size_t tma_smem_bytes() { return 1024 + (size_t)G * warp_line_stride<16>(N) * 16; }

template <int N, int G, bool CONTIG, bool CONJ_SCALE, bool EXT>
__global__ void __launch_bounds__(32 * G * tma_wpl<N, G>(), tma_min_ctas<N, G>())
fft_warp_tma_kernel(const StageArgs p, int64_t ntiles, const __grid_constant__ CUtensorMap tmap)
{
    constexpr int WPL = tma_wpl<N, G>();
    using L = TmaLine<N, WPL>;
    using C = ArDP::C;
    constexpr int LS = L::LS;
    static_assert(tma_stage_bytes<N, G>() <= (size_t)G * LS * 16, "staging must fit the lines");
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const uint32_t base = smem_addr(smem_raw);
    unsigned char* stage = smem_raw + (((base + 1023u) & ~1023u) - base);
    C* const lines = reinterpret_cast<C*>(stage);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int g = warp / WPL, w = warp % WPL;
    C* const line = lines + g * LS;
    const ArDP::W* tw = ArDP::table(p.tw, N);
    const bool convert = p.in_fmt == FMT_C128;

    for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const TileGeom tg = tile_geom(p, tile, G);
        // the previous tile's store has read the staging area: copy this tile in
        const bool leader = CONTIG ? (w == 0 && lane == 0) : tid == 0;
        if (leader) bulk_wait_read_all();
        if constexpr (CONTIG) line_sync<WPL>(g);
        else __syncthreads();
        tma_issue_load<N, WPL>(p, tg, g, line, lane, w);
        cp_async_wait_all();
        line_sync<WPL>(g);
        if (convert) {
            if (p.conj_in) L::template passes<0, 3>(line, tw, lane, w, g);
            else L::template passes<0, 2>(line, tw, lane, w, g);
        } else if (p.conj_in) {
            L::template passes<0, 1>(line, tw, lane, w, g);
        } else {
            L::template passes<0, 0>(line, tw, lane, w, g);
        }
        L::template last_pass<G, CONTIG, CONJ_SCALE, EXT>(line, tw, CONTIG ? reinterpret_cast<unsigned char*>(line) : stage,
                                                         lane, w, g, p.scale);
        fence_proxy_async_smem();
        if constexpr (CONTIG) {
            line_sync<WPL>(g);
            if (leader && g < tg.valid) {
                const int64_t o = tg.obase + g * tg.ostride;
                if (in_bounds(p.chk, o, p.out_elems) && in_bounds(p.chk, o + N - 1, p.out_elems))
                    bulk_store(reinterpret_cast<char*>(p.out) + o * 16, smem_addr(line), N * 16u);
                bulk_commit();
            }
            continue;
        }
        __syncthreads();
        if (tid == 0) {
            if constexpr (!CONTIG) {
#pragma unroll
                for (int kb = 0; kb < (N + 255) / 256; ++kb)
                    tma_store_3d(&tmap, smem_addr(stage) + (uint32_t)kb * 256u * (uint32_t)(G * 16),
                                 (int)((tile % p.ngroups) * G * 4), kb * 256, (int)(tile / p.ngroups));
            } else {
                char* first = reinterpret_cast<char*>(p.out) + tg.obase * 16;
                for (int gg = 0; gg < tg.valid; ++gg)
                    if (in_bounds(p.chk, tg.obase + gg * tg.ostride, p.out_elems) &&
                        in_bounds(p.chk, tg.obase + gg * tg.ostride + N - 1, p.out_elems))
                        bulk_store(first + (int64_t)gg * tg.ostride * 16, smem_addr(stage) + (uint32_t)gg * N * 16u,
                                   N * 16u);
            }
            bulk_commit();
        }
    }
    cp_async_wait_all();
    if (CONTIG ? (tid % (32 * WPL)) == 0 : tid == 0) bulk_wait_all();
}

// host side ----------------------------------------------------------------

using TensorMapEncodeFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                       const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                       CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

inline TensorMapEncodeFn tensor_map_encoder()
{
    static TensorMapEncodeFn fn = nullptr;
    static bool tried = false;
    if (!tried) {
        tried = true;
        void* f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<TensorMapEncodeFn>(f);
        else
            cudaGetLastError();
    }
    return fn;
}

// The transposed output as a 3-D tensor of 4-byte words: (grouped line
// coordinate x 4, frequency, other line coordinate); box (8 lines, 256 or n
// frequencies, 1).  false if the stage's geometry has no such view.
inline bool transposed_store_map(const StageArgs& a, int G, CUtensorMap* map)
{
    const int64_t Mg = a.group_i2 ? a.M2 : a.M1, Mo = a.group_i2 ? a.M1 : a.M2;
    const int64_t Sg = a.group_i2 ? a.S2 : a.S1, So = a.group_i2 ? a.S1 : a.S2;
    if (Sg != 1 || a.Sk < 1 || Mg * 4 > (int64_t)0xFFFFFFFF || Mo > 0xFFFFFFFF) return false;
    if ((reinterpret_cast<uintptr_t>(a.out) & 15) != 0) return false;
    TensorMapEncodeFn enc = tensor_map_encoder();
    if (!enc) return false;
    const int64_t s1 = a.Sk * 16;
    const int64_t s2 = Mo > 1 ? So * 16 : s1 * a.n;
    if (s1 >= ((int64_t)1 << 40) || s2 >= ((int64_t)1 << 40) || s2 <= 0) return false;
    const cuuint64_t dims[3] = {(cuuint64_t)(Mg * 4), (cuuint64_t)a.n, (cuuint64_t)Mo};
    const cuuint64_t strides[2] = {(cuuint64_t)s1, (cuuint64_t)s2};
    const cuuint32_t box[3] = {(cuuint32_t)(4 * G), (cuuint32_t)(a.n < 256 ? a.n : 256), 1u};
    const cuuint32_t estr[3] = {1u, 1u, 1u};
    return enc(map, CU_TENSOR_MAP_DATA_TYPE_UINT32, 3, a.out, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
               G == 8 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_64B, CU_TENSOR_MAP_L2_PROMOTION_NONE,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) ==
           CUDA_SUCCESS;
}

template <int N, int G, bool CONTIG, bool CONJ_SCALE, bool EXT>
cudaError_t launch_warp_tma_v(const StageLaunch& L, const CUtensorMap& map, cudaStream_t st)
{
    auto kern = fft_warp_tma_kernel<N, G, CONTIG, CONJ_SCALE, EXT>;
    const size_t smem = tma_smem_bytes<N, G>();
    static int cached[kMaxDevices] = {};
    int* slot = device_slot(cached);
    int per_sm = slot ? *slot : 0;
    if (per_sm == 0) {
        cudaError_t e = persistent_ctas_per_sm((const void*)kern, 32 * G * tma_wpl<N, G>(), smem, &per_sm);
        if (e) return e;
        if (slot) *slot = per_sm;
    }
    const int64_t ntiles = L.grid;
    int64_t grid = (int64_t)L.sms * per_sm;
    if (grid > ntiles) grid = ntiles;
    if (grid < 1) grid = 1;
    kern<<<(unsigned)grid, 32 * G * tma_wpl<N, G>(), smem, st>>>(L.args, ntiles, map);
    return cudaGetLastError();
}

// The asynchronous-output kernel for n = 256 / 512 and 4 or 8 lines per CTA,
// when the stage's output has the view it needs; *handled = false otherwise.
template <int N, int G>
cudaError_t launch_warp_tma_n(const StageLaunch& L, cudaStream_t st, bool* handled)
{
    const StageArgs& a = L.args;
    CUtensorMap map;
    std::memset(&map, 0, sizeof(map));
    const bool contig = a.contig_store != 0;
    if (contig) {
        if (a.group_i2 || a.S1 != a.n || a.Sk != 1 || (reinterpret_cast<uintptr_t>(a.out) & 15) != 0) {
            *handled = false;
            return cudaSuccess;
        }
    } else if (!transposed_store_map(a, G, &map)) {
        *handled = false;
        return cudaSuccess;
    }
#ifdef OPENFFT_CHECKED
    // The copy engine clips a tensor store to the map's extent; the checked
    // build takes this kernel only when that extent lies inside the output
    // array, and leaves other stages to the per-element checks of the warp
    // kernel, which report an index outside it.
    if (!contig) {
        const int64_t Mg = a.group_i2 ? a.M2 : a.M1, Mo = a.group_i2 ? a.M1 : a.M2;
        const int64_t So = a.group_i2 ? a.S1 : a.S2;
        if ((Mg - 1) + (int64_t)(a.n - 1) * a.Sk + (Mo > 1 ? (Mo - 1) * So : 0) >= a.out_elems) {
            *handled = false;
            return cudaSuccess;
        }
    }
#endif
    *handled = true;
    const bool ext = a.out_fmt != FMT_DF, cs = a.conj_out != 0;
    if (contig) {
        if (cs) return ext ? launch_warp_tma_v<N, G, true, true, true>(L, map, st) : launch_warp_tma_v<N, G, true, true, false>(L, map, st);
        return ext ? launch_warp_tma_v<N, G, true, false, true>(L, map, st) : launch_warp_tma_v<N, G, true, false, false>(L, map, st);
    }
    if (cs) return ext ? launch_warp_tma_v<N, G, false, true, true>(L, map, st) : launch_warp_tma_v<N, G, false, true, false>(L, map, st);
    return ext ? launch_warp_tma_v<N, G, false, false, true>(L, map, st) : launch_warp_tma_v<N, G, false, false, false>(L, map, st);
}

}  // namespace ofg
