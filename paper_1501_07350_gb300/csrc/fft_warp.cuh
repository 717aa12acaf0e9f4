// fft_warp.cuh -- FFT stage kernel for power-of-two line lengths (32..512):
// one warp per line.  The radix passes of a line need only its own warp, so
// they synchronise with __syncwarp; the CTA synchronises twice per tile, around
// the store that gathers the G lines of the tile (the transposed store writes
// G consecutive elements of the next ordering at each frequency).
//
// Per-warp line layout in shared memory: one padding element per 128 bytes
// (element p at p + (p >> 3) for 16-byte elements, p + (p >> 4) for 8-byte
// ones).  With the radix order "remainder radix (2 or 4) first, then radix 8"
// every read (positions b + j N/R, b = lane + 32 u) and every write
// (t m R + k + m q) of a Stockham pass is free of bank conflicts for 16-byte
// elements and at most 2-way for 8-byte ones (checked for N = 32..512); lines
// sit an odd number of elements apart, so the transposed store (consecutive
// lanes = consecutive lines) is conflict-free too.
//
// The radix pass is the same Stockham decimation-in-time step as in
// fft_stage.cu; in-place in the warp's line with a __syncwarp between reads
// and writes.  Tiles are processed persistently; the next tile's lines are
// copied (cp.async) while the current tile is transformed.
#pragma once
#include "arith.cuh"
#include "arith_pair.cuh"
#include "fft_stage.h"
#include "fft_tile.cuh"
#include "stage_io.cuh"
#include "warp_plan.h"

namespace ofg {

// one padding element per 128 bytes of line: per 8 elements of 16 bytes,
// per 16 elements of 8 bytes
template <int EB>
__host__ __device__ constexpr int wpad(int p) { return p + (p >> (EB >= 16 ? 3 : 4)); }

// shared-memory stride between lines: odd, at least the padded length
template <int EB>
constexpr int warp_line_stride(int N) { return (wpad<EB>(N - 1) + 1) | 1; }

template <class A, int N>
struct WarpLine {
    using C = typename A::C;
    using W = typename A::W;
    static constexpr int kPasses = wplan_len(N);
    static constexpr int EB = sizeof(C);
    static constexpr int LS = warp_line_stride<EB>(N);

    // One radix pass over the warp's Q L lines at line0 + l LS.  The lanes
    // form Q groups of S = 32 / Q; lane bl of group q takes butterflies
    // bl, bl + S, ... of lines q L + i (i < L), so the L lines share the
    // twiddle loads and give each thread L independent butterflies, and lines
    // with fewer than 32 butterflies per pass still occupy every lane.
    // The pass's results go through put(l, k, value): value k of the warp's
    // line l (l < Q L), after every lane has read its inputs.
    template <int P, int L, int Q, class Put>
    __device__ __forceinline__ static void pass_to(const C* line0, const W* __restrict__ tw, int lane, Put put)
    {
        constexpr int R = wplan_radix(N, P);
        constexpr int m = wplan_m(N, P);
        constexpr int s = N / (m * R);
        constexpr int NBF = N / R;
        constexpr int S = 32 / Q;
        constexpr int NB = (NBF + S - 1) / S;
        const int bl = lane % S;
        const int l0 = (lane / S) * L;
        line0 += l0 * LS;
        C v[L][NB][R];
#pragma unroll
        for (int u = 0; u < NB; ++u) {
            const int b = bl + S * u;
            if (NBF % S == 0 || b < NBF) {
#pragma unroll
                for (int i = 0; i < L; ++i)
#pragma unroll
                    for (int j = 0; j < R; ++j) v[i][u][j] = line0[i * LS + wpad<EB>(b + j * NBF)];
                if (m > 1) {
                    const int k = b % m;
                    const int ks = k * s;
#pragma unroll
                    for (int j = 1; j < R; ++j) {
                        const W w = A::template warp_twiddle<N>(tw, wtw_offset(N, P), m, j, k, ks);
#pragma unroll
                        for (int i = 0; i < L; ++i) v[i][u][j] = A::mul(v[i][u][j], w);
                    }
                }
#pragma unroll
                for (int i = 0; i < L; ++i) Dft<A, R>::run(v[i][u]);
            }
        }
        __syncwarp();
#pragma unroll
        for (int u = 0; u < NB; ++u) {
            const int b = bl + S * u;
            if (NBF % S == 0 || b < NBF) {
                const int t = b / m, k = b % m;
                const int base = t * m * R + k;
#pragma unroll
                for (int i = 0; i < L; ++i)
#pragma unroll
                    for (int q = 0; q < R; ++q) put(l0 + i, base + m * q, v[i][u][q]);
            }
        }
    }

    template <int P, int L, int Q = 1>
    __device__ __forceinline__ static void pass(C* line0, const W* __restrict__ tw, int lane)
    {
        pass_to<P, L, Q>(line0, tw, lane, [=](int l, int k, const C& x) { line0[l * LS + wpad<EB>(k)] = x; });
        __syncwarp();
    }

    template <int P, int L = 1, int Q = 1>
    __device__ __forceinline__ static void passes(C* line0, const W* __restrict__ tw, int lane)
    {
        if constexpr (P < kPasses) {
            pass<P, L, Q>(line0, tw, lane);
            passes<P + 1, L, Q>(line0, tw, lane);
        }
    }

    // every pass but the last, in place
    template <int P, int L = 1, int Q = 1>
    __device__ __forceinline__ static void passes_but_last(C* line0, const W* __restrict__ tw, int lane)
    {
        if constexpr (P < kPasses - 1) {
            pass<P, L, Q>(line0, tw, lane);
            passes_but_last<P + 1, L, Q>(line0, tw, lane);
        }
    }
};

// copies of line g (= warp) of a tile
template <class A, int N>
__device__ __forceinline__ void warp_issue_load(const StageArgs& p, const TileGeom& tg, int g,
                                                typename A::C* line, int lane)
{
    constexpr int EB = sizeof(typename A::C) >= 16 ? 16 : 8;
    if (g < tg.valid) {
        const char* src = reinterpret_cast<const char*>(p.in) + (tg.line0 + g * tg.lstride) * (int64_t)(N * EB);
#pragma unroll
        for (int u = 0; u < (N + 31) / 32; ++u) {
            const int pos = lane + 32 * u;
            if ((N % 32 == 0 || pos < N) && in_bounds(p.chk, (tg.line0 + g * tg.lstride) * N + pos, p.in_elems))
                cp_async<EB>(line + wpad<sizeof(typename A::C)>(pos), src + pos * EB);
        }
    } else {
#pragma unroll
        for (int u = 0; u < (N + 31) / 32; ++u)
            if (N % 32 == 0 || lane + 32 * u < N) line[wpad<sizeof(typename A::C)>(lane + 32 * u)] = A::zero();
    }
    cp_async_commit();
}

template <class A, int N, bool CONVERT, bool CONJ>
__device__ __forceinline__ void warp_fix(typename A::C* line, int lane)
{
    using C = typename A::C;
#pragma unroll
    for (int u = 0; u < (N + 31) / 32; ++u) {
        if (N % 32 != 0 && lane + 32 * u >= N) break;
        C* x = line + wpad<sizeof(C)>(lane + 32 * u);
        C v;
        if constexpr (CONVERT) v = Io<A>::from_c128(*reinterpret_cast<const double2*>(x));
        else v = *x;
        if constexpr (CONJ) v = A::conj(v);
        *x = v;
    }
}

template <class A, int N, int G, int L, bool CONTIG, bool CONJ_SCALE, bool EXT>
__device__ __forceinline__ void warp_tile_store(const StageArgs& p, const TileGeom& tg,
                                                const typename A::C* buf, int tid)
{
    constexpr int CB = sizeof(typename A::C);
    constexpr int LS = warp_line_stride<CB>(N);
    constexpr int EB = EXT ? Io<A>::kExtBytes : Io<A>::kMidBytes;
    constexpr int SL = 32 / L;             // threads per line of the tile
    char* first = reinterpret_cast<char*>(p.out) + tg.obase * EB;
    if constexpr (!CONTIG) {
        // thread (g, slot): line g, frequencies slot, slot + SL, ...
        const int g = tid % G, slot = tid / G;
        if (g >= tg.valid) return;
        const typename A::C* line = buf + g * LS;
        char* ptr = first + (g * tg.ostride + slot * p.Sk) * EB;
        const int64_t step = (int64_t)SL * p.Sk * EB;
#pragma unroll 4
        for (int k = slot; k < N; k += SL) {
            if (in_bounds(p.chk, tg.obase + g * tg.ostride + (int64_t)k * p.Sk, p.out_elems))
                put<A, CONJ_SCALE, EXT>(ptr, line[wpad<CB>(k)], p.scale);
            ptr += step;
        }
    } else {
        // warp w stores its own lines w L + i, each contiguous in the output
        const int lane = tid & 31;
#pragma unroll
        for (int i = 0; i < L; ++i) {
            const int g = (tid >> 5) * L + i;
            if (g >= tg.valid) return;
            const typename A::C* line = buf + g * LS;
            char* ptr = first + (int64_t)g * tg.ostride * EB;
#pragma unroll
            for (int u = 0; u < (N + 31) / 32; ++u) {
                const int k = lane + 32 * u;
                if ((N % 32 == 0 || k < N) && in_bounds(p.chk, tg.obase + (int64_t)g * tg.ostride + k, p.out_elems))
                    put<A, CONJ_SCALE, EXT>(ptr + k * EB, line[wpad<CB>(k)], p.scale);
            }
        }
    }
}

template <class A, int N, int G, int L>
__device__ __forceinline__ void warp_store_dispatch(const StageArgs& p, const TileGeom& tg,
                                                    const typename A::C* buf, int tid)
{
    const bool ext = p.out_fmt != FMT_DF;
    const bool cs = p.conj_out != 0;
    if (!p.contig_store) {
        if (cs) { if (ext) warp_tile_store<A, N, G, L, false, true, true>(p, tg, buf, tid); else warp_tile_store<A, N, G, L, false, true, false>(p, tg, buf, tid); }
        else    { if (ext) warp_tile_store<A, N, G, L, false, false, true>(p, tg, buf, tid); else warp_tile_store<A, N, G, L, false, false, false>(p, tg, buf, tid); }
    } else {
        if (cs) { if (ext) warp_tile_store<A, N, G, L, true, true, true>(p, tg, buf, tid); else warp_tile_store<A, N, G, L, true, true, false>(p, tg, buf, tid); }
        else    { if (ext) warp_tile_store<A, N, G, L, true, false, true>(p, tg, buf, tid); else warp_tile_store<A, N, G, L, true, false, false>(p, tg, buf, tid); }
    }
}

// register budget: 128 per thread for 16-byte elements and for 8-byte ones
// in CTAs of 128 threads (two lines per warp, four CTAs per SM), 64-85 for
// larger CTAs of 8-byte elements
constexpr int warp_min_blocks(int T, int EB)
{
    return EB >= 16 ? (512 / T > 0 ? 512 / T : 1) : (T >= 512 ? 2 : (T <= 128 ? 4 : 3));
}

// Tiles are double-buffered (the next tile's copies overlap this tile's
// passes) except for 512-point lines of 16-byte elements: there one buffer
// halves the shared memory, so four CTAs fit on an SM instead of three, and the
// other CTAs cover the copy latency.
template <class A, int N>
constexpr bool warp_double_buffer() { return !(N >= 512 && sizeof(typename A::C) >= 16); }

// Lines per warp: FP32 passes are short and wait on shared memory, so each
// warp takes two lines (two independent butterflies per thread and pass, one
// set of twiddle loads); the double-float and FP64 passes carry enough
// arithmetic per line and need the registers.
template <class A, int N, int G>
constexpr int warp_lines_per_warp() { return (sizeof(typename A::C) == 8 && G % 2 == 0) ? 2 : 1; }

// Line groups per warp: a radix-8 pass over n < 256 points has n / 8 < 32
// butterflies, so up to 256 / n lines share a warp (a power of two, as many
// as the tile has room for), one group of lanes per line.
template <class A, int N, int G>
constexpr int warp_line_groups()
{
    int q = 1;                                 // a power of two: 32 / q lanes per line
    while (2 * q <= 256 / N && 2 * q <= G / warp_lines_per_warp<A, N, G>()) q *= 2;
    return q;
}
template <class A, int N, int G>
constexpr int warp_threads() { return 32 * G / (warp_lines_per_warp<A, N, G>() * warp_line_groups<A, N, G>()); }

template <class A, int N, int G>
__global__ void __launch_bounds__(warp_threads<A, N, G>(), warp_min_blocks(warp_threads<A, N, G>(), sizeof(typename A::C)))
fft_warp_kernel(const StageArgs p, int64_t ntiles)
{
    using C = typename A::C;
    constexpr int Q = warp_line_groups<A, N, G>();
    constexpr int L1 = warp_lines_per_warp<A, N, G>();      // lines per lane group
    constexpr int L = L1 * Q;                                // this warp's lines
    constexpr int LS = warp_line_stride<sizeof(C)>(N);
    constexpr bool DB = warp_double_buffer<A, N>();
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* cur = reinterpret_cast<C*>(smem_raw);
    C* nxt = DB ? cur + G * LS : cur;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int g0 = warp * L;                // this warp's first line of the tile
    const typename A::W* tw = A::table(p.tw, N);
    const bool convert = Io<A>::kConverts && p.in_fmt == FMT_C128;

    int64_t tile = blockIdx.x;
    if (DB && tile < ntiles) {
        const TileGeom tg = tile_geom(p, tile, G);
#pragma unroll
        for (int i = 0; i < L; ++i) warp_issue_load<A, N>(p, tg, g0 + i, cur + (g0 + i) * LS, lane);
    }
    for (; tile < ntiles; tile += gridDim.x) {
        const TileGeom tg = tile_geom(p, tile, G);
        C* line0 = cur + g0 * LS;
        if (!DB) {
#pragma unroll
            for (int i = 0; i < L; ++i) warp_issue_load<A, N>(p, tg, g0 + i, line0 + i * LS, lane);
        }
        cp_async_wait_all();
#pragma unroll
        for (int i = 0; i < L; ++i) {
            C* line = line0 + i * LS;
            if (convert) { if (p.conj_in) warp_fix<A, N, true, true>(line, lane); else warp_fix<A, N, true, false>(line, lane); }
            else if (p.conj_in) warp_fix<A, N, false, true>(line, lane);
        }
        __syncwarp();
        const int64_t next = tile + gridDim.x;
        if (DB && next < ntiles) {
            const TileGeom tn = tile_geom(p, next, G);
#pragma unroll
            for (int i = 0; i < L; ++i) warp_issue_load<A, N>(p, tn, g0 + i, nxt + (g0 + i) * LS, lane);
        }
        WarpLine<A, N>::template passes<0, L1, Q>(line0, tw, lane);
        __syncthreads();                   // every line of the tile is transformed
        warp_store_dispatch<A, N, G, L>(p, tg, cur, tid);
        __syncthreads();                   // cur becomes the next copy target
        C* t = cur; cur = nxt; nxt = t;
    }
    cp_async_wait_all();
}

template <class A, int N, int G>
cudaError_t launch_warp_n(const StageLaunch& L, cudaStream_t st)
{
    constexpr int T = warp_threads<A, N, G>();
    const size_t smem = (warp_double_buffer<A, N>() ? 2 : 1) * (size_t)G * warp_line_stride<sizeof(typename A::C)>(N) *
                        sizeof(typename A::C);
    static int cached[kMaxDevices] = {};          // CTAs per SM on each device, 0 = not yet known
    int* slot = device_slot(cached);
    int blocks_per_sm = slot ? *slot : 0;
    if (blocks_per_sm == 0) {
        cudaError_t e = persistent_ctas_per_sm((const void*)fft_warp_kernel<A, N, G>, T, smem, &blocks_per_sm);
        if (e) return e;
        if (slot) *slot = blocks_per_sm;
    }
    const int64_t ntiles = L.grid;
    int64_t grid = (int64_t)L.sms * blocks_per_sm;
    if (grid > ntiles) grid = ntiles;
    if (grid < 1) grid = 1;
    fft_warp_kernel<A, N, G><<<(unsigned)grid, T, smem, st>>>(L.args, ntiles);
    return cudaGetLastError();
}

// power-of-two lengths go to the warp-per-line kernel
template <class A, int G>
cudaError_t launch_warp_g(const StageLaunch& L, cudaStream_t st, bool* handled)
{
    const StageArgs& a = L.args;
    if (a.contig_store && (a.group_i2 || a.S1 != a.n || a.Sk != 1)) { *handled = false; return cudaSuccess; }
    *handled = true;
    switch (a.n) {
    case 32: return launch_warp_n<A, 32, G>(L, st);
    case 64: return launch_warp_n<A, 64, G>(L, st);
    case 128: return launch_warp_n<A, 128, G>(L, st);
    case 256: return launch_warp_n<A, 256, G>(L, st);
    case 512: return launch_warp_n<A, 512, G>(L, st);
    default: *handled = false; return cudaSuccess;
    }
}

}  // namespace ofg
