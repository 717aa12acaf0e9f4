// fft_tile.cuh -- FFT stage kernel specialised at compile time for one line
// length N (radix plan, thread mapping and every shared-memory offset are
// constants), persistent over tiles of G lines, with the next tile's lines
// copied into shared memory (cp.async) while the current tile is transformed.
//
// Same contract as fft_stage_kernel (fft_stage.h): lines l = i1 + i2 M1 of
// length N, output (l, k) at i1 S1 + i2 S2 + k Sk, a tile = G consecutive
// values of the coordinate whose output stride is 1.  Same radix pass
// (Stockham autosort, decimation in time), done in place: each thread reads
// its butterflies into registers, the CTA synchronises, and the results are
// written back.
#pragma once
#include <type_traits>

#include "arith.cuh"
#include "fft_stage.h"
#include "stage_io.cuh"

namespace ofg {

// ----------------------------------------------- compile-time radix plan --

constexpr int plan_len(int n)
{
    int c = 0;
    while (n % 8 == 0) { n /= 8; ++c; }
    while (n % 4 == 0) { n /= 4; ++c; }
    while (n % 2 == 0) { n /= 2; ++c; }
    while (n % 3 == 0) { n /= 3; ++c; }
    while (n % 5 == 0) { n /= 5; ++c; }
    while (n % 7 == 0) { n /= 7; ++c; }
    return c;
}

constexpr int plan_radix(int n, int idx)
{
    const int rs[6] = {8, 4, 2, 3, 5, 7};
    int c = 0;
    for (int r : rs)
        while (n % r == 0) {
            if (c == idx) return r;
            n /= r;
            ++c;
        }
    return 1;
}

// product of the radices before pass idx
constexpr int plan_m(int n, int idx)
{
    int m = 1;
    for (int i = 0; i < idx; ++i) m *= plan_radix(n, i);
    return m;
}

template <class A, int N, int G, int T>
struct Tile {
    using C = typename A::C;
    using W = typename A::W;
    static constexpr int kLd = G + 1;            // shared-memory row stride (elements)
    static constexpr int kElems = N * kLd;       // elements of one tile buffer
    static constexpr int kSlots = T / G;         // threads per line
    static constexpr int kPasses = plan_len(N);

    // one radix pass, in place on the column of line g
    template <int P>
    __device__ __forceinline__ static void pass(C* col, const W* __restrict__ tw, int slot)
    {
        constexpr int R = plan_radix(N, P);
        constexpr int m = plan_m(N, P);
        constexpr int s = N / (m * R);
        constexpr int NBF = N / R;
        constexpr int NB = (NBF + kSlots - 1) / kSlots;
        C v[NB][R];
#pragma unroll
        for (int u = 0; u < NB; ++u) {
            const int b = slot + u * kSlots;
            if (NBF % kSlots == 0 || b < NBF) {
                const int t = b / m, k = b - (b / m) * m;
                const C* src = col + (t * m + k) * kLd;
#pragma unroll
                for (int j = 0; j < R; ++j) v[u][j] = src[j * s * m * kLd];
                if (m > 1) {
                    const int ks = k * s;
#pragma unroll
                    for (int j = 1; j < R; ++j) v[u][j] = A::mul(v[u][j], __ldg(tw + j * ks));
                }
                Dft<A, R>::run(v[u]);
            }
        }
        __syncthreads();
#pragma unroll
        for (int u = 0; u < NB; ++u) {
            const int b = slot + u * kSlots;
            if (NBF % kSlots == 0 || b < NBF) {
                const int t = b / m, k = b - (b / m) * m;
                C* dst = col + (t * m * R + k) * kLd;
#pragma unroll
                for (int q = 0; q < R; ++q) dst[q * m * kLd] = v[u][q];
            }
        }
        __syncthreads();
    }

    template <int P>
    __device__ __forceinline__ static void passes(C* col, const W* __restrict__ tw, int slot)
    {
        if constexpr (P < kPasses) {
            pass<P>(col, tw, slot);
            passes<P + 1>(col, tw, slot);
        }
    }
};

// Tile -> its first line, line stride, number of valid lines, first output
// offset and output stride between lines.
struct TileGeom {
    int64_t line0, lstride, obase, ostride;
    int valid;
};

__device__ __forceinline__ TileGeom tile_geom(const StageArgs& p, int64_t tile, int G)
{
    TileGeom t;
    // 32-bit division whenever the operands fit (launch grids always do):
    // the 64-bit one is a long software sequence run twice per tile
    int64_t outer, grp;
    if (((uint64_t)tile | (uint64_t)p.ngroups) >> 32 == 0) {
        const uint32_t o = (uint32_t)tile / (uint32_t)p.ngroups;
        outer = o;
        grp = (int64_t)((uint32_t)tile - o * (uint32_t)p.ngroups);
    } else {
        outer = tile / p.ngroups;
        grp = tile - outer * p.ngroups;
    }
    const int64_t first = grp * G;
    if (!p.group_i2) {
        t.line0 = first + outer * p.M1; t.lstride = 1;
        t.obase = first * p.S1 + outer * p.S2; t.ostride = p.S1;
        t.valid = (int)(p.M1 - first < G ? p.M1 - first : G);
    } else {
        t.line0 = outer + first * p.M1; t.lstride = p.M1;
        t.obase = outer * p.S1 + first * p.S2; t.ostride = p.S2;
        t.valid = (int)(p.M2 - first < G ? p.M2 - first : G);
    }
    return t;
}

// Element e = g N + i of a tile (line g, position i) -> shared-memory slot.
template <int N, int G>
__device__ __forceinline__ int slot_of(int e) { return (e % N) * (G + 1) + e / N; }

// Issue the asynchronous copies of one tile.  Lines of a tile are either
// consecutive in memory (lstride = 1: element e sits at e * EB from the
// first line) or lstride lines apart.
template <class A, int N, int G, int T>
__device__ __forceinline__ void tile_issue_loads(const StageArgs& p, const TileGeom& tg,
                                                 typename A::C* buf, int tid)
{
    using C = typename A::C;
    constexpr int EB = sizeof(C) >= 16 ? 16 : 8;
    constexpr int TOTAL = G * N;
    constexpr int ITERS = (TOTAL + T - 1) / T;
    const char* first = reinterpret_cast<const char*>(p.in) + tg.line0 * (int64_t)(N * EB);
    const int64_t gstride = tg.lstride * (int64_t)(N * EB);
#pragma unroll
    for (int it = 0; it < ITERS; ++it) {
        const int e = tid + it * T;
        if (TOTAL % T == 0 || e < TOTAL) {
            const int g = e / N;
            C* dst = buf + slot_of<N, G>(e);
            const char* src = tg.lstride == 1 ? first + (int64_t)e * EB
                                              : first + g * gstride + (e - g * N) * EB;
            const int64_t idx = tg.line0 * N + (tg.lstride == 1 ? (int64_t)e : g * tg.lstride * N + (e - g * N));
            if (g < tg.valid) {
                if (in_bounds(p.chk, idx, p.in_elems)) cp_async<EB>(dst, src);
            } else {
                *dst = A::zero();
            }
        }
    }
    cp_async_commit();
}

// In-place entry fix-up of this thread's own copies: complex128 -> working
// format and/or conjugation (backward transforms).
template <class A, int N, int G, int T, bool CONVERT, bool CONJ>
__device__ __forceinline__ void tile_fix(typename A::C* buf, int tid)
{
    using C = typename A::C;
    constexpr int TOTAL = G * N;
    constexpr int ITERS = (TOTAL + T - 1) / T;
#pragma unroll
    for (int it = 0; it < ITERS; ++it) {
        const int e = tid + it * T;
        if (TOTAL % T == 0 || e < TOTAL) {
            C* x = buf + slot_of<N, G>(e);
            C v;
            if constexpr (CONVERT) v = Io<A>::from_c128(*reinterpret_cast<const double2*>(x));
            else v = *x;
            if constexpr (CONJ) v = A::conj(v);
            *x = v;
        }
    }
}

template <class A, bool CONJ_SCALE, bool EXT>
__device__ __forceinline__ void put(void* ptr, typename A::C v, double scale)
{
    if constexpr (CONJ_SCALE) v = A::scale(A::conj(v), scale);
    if constexpr (EXT) Io<A>::store_ext(ptr, v);
    else Io<A>::store_mid(ptr, v);
}

// Store one tile.  Transposed: thread (g, slot) writes line g at frequencies
// k = slot, slot + T/G, ... through a pointer that advances by (T/G) Sk
// elements; consecutive threads hit consecutive lines, i.e. consecutive
// addresses of the next ordering.  Contiguous (Sk = 1, line stride N): element
// e of the tile goes to e * EB from the tile's first output.
template <class A, int N, int G, int T, bool CONTIG, bool CONJ_SCALE, bool EXT>
__device__ __forceinline__ void tile_store(const StageArgs& p, const TileGeom& tg,
                                           const typename A::C* buf, int tid)
{
    using C = typename A::C;
    constexpr int EB = EXT ? Io<A>::kExtBytes : Io<A>::kMidBytes;
    constexpr int TOTAL = G * N;
    char* first = reinterpret_cast<char*>(p.out) + tg.obase * EB;
    if constexpr (!CONTIG) {
        const int g = tid % G, slot = tid / G;
        if (g >= tg.valid) return;
        char* ptr = first + (g * tg.ostride + slot * p.Sk) * EB;
        const int64_t step = (int64_t)(T / G) * p.Sk * EB;
#pragma unroll 4
        for (int k = slot; k < N; k += T / G) {
            if (in_bounds(p.chk, tg.obase + g * tg.ostride + (int64_t)k * p.Sk, p.out_elems))
                put<A, CONJ_SCALE, EXT>(ptr, buf[k * (G + 1) + g], p.scale);
            ptr += step;
        }
    } else {
        constexpr int ITERS = (TOTAL + T - 1) / T;
#pragma unroll
        for (int it = 0; it < ITERS; ++it) {
            const int e = tid + it * T;
            if ((TOTAL % T == 0 || e < TOTAL) && e / N < tg.valid && in_bounds(p.chk, tg.obase + e, p.out_elems))
                put<A, CONJ_SCALE, EXT>(first + (int64_t)e * EB, buf[slot_of<N, G>(e)], p.scale);
        }
    }
}

template <class A, int N, int G, int T>
__device__ __forceinline__ void tile_store_dispatch(const StageArgs& p, const TileGeom& tg,
                                                    const typename A::C* buf, int tid)
{
    const bool ext = p.out_fmt != FMT_DF;
    const bool cs = p.conj_out != 0;          // conjugation and scaling come together
    if (!p.contig_store) {
        if (cs) { if (ext) tile_store<A, N, G, T, false, true, true>(p, tg, buf, tid); else tile_store<A, N, G, T, false, true, false>(p, tg, buf, tid); }
        else    { if (ext) tile_store<A, N, G, T, false, false, true>(p, tg, buf, tid); else tile_store<A, N, G, T, false, false, false>(p, tg, buf, tid); }
    } else {
        if (cs) { if (ext) tile_store<A, N, G, T, true, true, true>(p, tg, buf, tid); else tile_store<A, N, G, T, true, true, false>(p, tg, buf, tid); }
        else    { if (ext) tile_store<A, N, G, T, true, false, true>(p, tg, buf, tid); else tile_store<A, N, G, T, true, false, false>(p, tg, buf, tid); }
    }
}

// resident CTAs per SM the register budget is sized for (>= 32 warps at T >= 256)
constexpr int tile_min_blocks(int T) { return T >= 512 ? 2 : (T >= 256 ? 3 : 4); }

template <class A, int N, int G, int T>
__global__ void __launch_bounds__(T, tile_min_blocks(T))
fft_tile_kernel(const StageArgs p, int64_t ntiles)
{
    using TL = Tile<A, N, G, T>;
    using C = typename A::C;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* cur = reinterpret_cast<C*>(smem_raw);
    C* nxt = cur + TL::kElems;
    const int tid = threadIdx.x;
    const int g_mine = tid % G, slot = tid / G;
    const typename A::W* tw = reinterpret_cast<const typename A::W*>(p.tw);
    const bool convert = Io<A>::kConverts && p.in_fmt == FMT_C128;

    int64_t tile = blockIdx.x;
    if (tile < ntiles) tile_issue_loads<A, N, G, T>(p, tile_geom(p, tile, G), cur, tid);
    for (; tile < ntiles; tile += gridDim.x) {
        const TileGeom tg = tile_geom(p, tile, G);
        cp_async_wait_all();
        if (convert) { if (p.conj_in) tile_fix<A, N, G, T, true, true>(cur, tid); else tile_fix<A, N, G, T, true, false>(cur, tid); }
        else if (p.conj_in) tile_fix<A, N, G, T, false, true>(cur, tid);
        __syncthreads();
        // the next tile's copies overlap this tile's passes and stores
        const int64_t next = tile + gridDim.x;
        if (next < ntiles) tile_issue_loads<A, N, G, T>(p, tile_geom(p, next, G), nxt, tid);
        TL::template passes<0>(cur + g_mine, tw, slot);
        tile_store_dispatch<A, N, G, T>(p, tg, cur, tid);
        __syncthreads();          // cur becomes the next prefetch target
        C* t = cur; cur = nxt; nxt = t;
    }
    cp_async_wait_all();
}

}  // namespace ofg

namespace ofg {

// threads per CTA: about eight elements per thread, between 128 and 512
constexpr int tile_threads(int N, int G)
{
    const int t = N * G / 8;
    return t < 128 ? 128 : (t > 512 ? 512 : t);
}

template <class A, int N, int G>
cudaError_t launch_tile_n(const StageLaunch& L, cudaStream_t st)
{
    constexpr int T = tile_threads(N, G);
    using TL = Tile<A, N, G, T>;
    const size_t smem = 2 * (size_t)TL::kElems * sizeof(typename A::C);
    static int cached[kMaxDevices] = {};          // CTAs per SM on each device, 0 = not yet known
    int* slot = device_slot(cached);
    int blocks_per_sm = slot ? *slot : 0;
    if (blocks_per_sm == 0) {
        cudaError_t e = persistent_ctas_per_sm((const void*)fft_tile_kernel<A, N, G, T>, T, smem, &blocks_per_sm);
        if (e) return e;
        if (slot) *slot = blocks_per_sm;
    }
    const int64_t ntiles = L.grid;
    int64_t grid = (int64_t)L.sms * blocks_per_sm;
    if (grid > ntiles) grid = ntiles;
    if (grid < 1) grid = 1;
    fft_tile_kernel<A, N, G, T><<<(unsigned)grid, T, smem, st>>>(L.args, ntiles);
    return cudaGetLastError();
}

// Launch the specialised kernel for (N, G) if there is one; *handled = false otherwise.
template <class A, int G>
cudaError_t launch_tile_g(const StageLaunch& L, cudaStream_t st, bool* handled)
{
    const StageArgs& a = L.args;
    // contiguous stores assume lines of the output in order (S1 = n, Sk = 1)
    if (a.contig_store && (a.group_i2 || a.S1 != a.n || a.Sk != 1)) { *handled = false; return cudaSuccess; }
    *handled = true;
    switch (L.args.n) {
    case 32: return launch_tile_n<A, 32, G>(L, st);
    case 48: return launch_tile_n<A, 48, G>(L, st);
    case 64: return launch_tile_n<A, 64, G>(L, st);
    case 96: return launch_tile_n<A, 96, G>(L, st);
    case 100: return launch_tile_n<A, 100, G>(L, st);
    case 108: return launch_tile_n<A, 108, G>(L, st);
    case 120: return launch_tile_n<A, 120, G>(L, st);
    case 128: return launch_tile_n<A, 128, G>(L, st);
    case 144: return launch_tile_n<A, 144, G>(L, st);
    case 160: return launch_tile_n<A, 160, G>(L, st);
    case 256: return launch_tile_n<A, 256, G>(L, st);
    case 512: return launch_tile_n<A, 512, G>(L, st);
    default: *handled = false; return cudaSuccess;
    }
}

}  // namespace ofg
