// dftgemm.cu -- FFT stage whose small DFT blocks are dense complex GEMMs on
// the tcgen05 tensor cores, in split precision (the precision forms
// OPENFFT_C2C_SPLIT_TF32 / OPENFFT_C2C_SPLIT_BF16, complex64 data).
//
// A line of length n = R S is transformed in two GEMM passes (four-step):
//   pass 1, rows (g, t), t < S:  Y[t][q] = sum_{j<R} x[t + S j] W_R^{j q}       (q < R)
//   pass 2, rows (g, k), k < R:  Z[k + R q] = sum_{j<S} (W_n^{j k} Y[j][k]) W_S^{j q}   (q < S)
// which is the DFT of x in natural order (the Stockham steps with radices R
// and S).  Each pass is D = A B^T with the complex data real-ified and
// interleaved: A row = (re x_0, im x_0, re x_1, ...), and B[2q][2j] = c,
// B[2q][2j+1] = s, B[2q+1][2j] = -s, B[2q+1][2j+1] = c for W^{jq} = c - i s.
// Both operands are split into a high part (tf32 or bf16) and the rounded
// remainder; D = A_hi B_hi + A_hi B_lo + A_lo B_hi accumulates in fp32 in
// tensor memory.  K and N are padded with zeros to the MMA granularity.
//
// One CTA of 256 threads (two warpgroups; warps w and w + 4 share the
// tensor-memory lanes 32 (w % 4) ..) per tile of G lines, persistent over
// tiles.  The B operands (hi / lo images of both passes) are built once per
// plan in global memory and copied, with the twiddle table, to shared memory
// when the CTA starts.  Per tile and pass: every 128-row block of A is
// staged (row blk * 128 + lane; warpgroup h takes half of the 16-byte K
// groups of the row: whole core-matrix rows, one integer division per row),
// thread 0 issues the MMAs of all blocks (block b accumulates in tensor-memory
// columns 64 b ..) and commits them to one mbarrier, and every thread reads
// its share of the 16-column chunks of its row back into the line buffer.
// The lines of the next tile are loaded into registers while this tile runs
// and written to shared memory after its store.
//
// Line buffer layout: line g at g * np; pass 1 writes Y[t][q] at t * Rp + q
// with Rp = R rounded up to odd (conflict-free row-per-thread stores), and np
// (>= S Rp) is an odd multiple of 16 / G so that the store phase, which reads
// one element of each of G lines per group of G threads, is conflict-free.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>

#include "../../include/openfft_gb.h"
#include "dftgemm.h"
#include "fft_stage.h"
#include "fft_tile.cuh"
#include "stage_io.cuh"
#include "tc.cuh"

namespace ofg {

namespace {

constexpr int kThreads = 256;
constexpr int kPrefetch = 16;                     // register prefetch: up to 16 elements per thread
constexpr int kMaxBlocks = 4;                     // 128-row blocks per pass (tensor-memory columns 64 each)
constexpr long long kWaitBudget = 2000000000LL;   // about one second of clock cycles

// Test controls (process-wide): the completion-wait budget in clock cycles,
// and a switch that leaves the MMAs of every block unissued and uncommitted so
// that the bounded completion waits run out (nothing is in flight then).
__device__ long long g_wait_budget = kWaitBudget;
__device__ int g_skip_mma = 0;

struct GemmShape {
    int n, R, S, G, Rp, np;
    int K1, N1, K2, N2;          // padded real K / N of the two passes
    int M1, M2;                  // rows (G S, G R) padded to multiples of 128
    int es;                      // operand bytes (4 tf32, 2 bf16)
    int tcols;                   // tensor-memory columns: 64 per 128-row block
    // shared-memory byte offsets; the B image is [b1 hi | b1 lo | b2 hi | b2 lo]
    int off_lines, off_ahi, off_alo, off_b, off_tw, b_bytes, smem;
    int b1lo, b2hi, b2lo;        // offsets within the B image
};

__host__ __device__ int pad_to(int v, int m) { return (v + m - 1) / m * m; }

template <bool TF32>
__device__ __forceinline__ void put_split(unsigned char* hi, unsigned char* lo, uint32_t off, float x)
{
    if (TF32) {
        const float h = tc::round_tf32(x);
        *reinterpret_cast<float*>(hi + off) = h;
        *reinterpret_cast<float*>(lo + off) = tc::round_tf32(x - h);
    } else {
        const __nv_bfloat16 h = __float2bfloat16_rn(x);
        *reinterpret_cast<__nv_bfloat16*>(hi + off) = h;
        *reinterpret_cast<__nv_bfloat16*>(lo + off) = __float2bfloat16_rn(x - __bfloat162float(h));
    }
}

// One 16-byte K group of a row of A: CPG complex values (2 for tf32, 4 for
// bf16), real-ified (re, im, re, im, ...), split into hi and lo.
template <bool TF32>
__device__ __forceinline__ void put_group(unsigned char* hi, unsigned char* lo, uint32_t off, const float2* x)
{
    if (TF32) {
        float4 h, l;
        h.x = tc::round_tf32(x[0].x); l.x = tc::round_tf32(x[0].x - h.x);
        h.y = tc::round_tf32(x[0].y); l.y = tc::round_tf32(x[0].y - h.y);
        h.z = tc::round_tf32(x[1].x); l.z = tc::round_tf32(x[1].x - h.z);
        h.w = tc::round_tf32(x[1].y); l.w = tc::round_tf32(x[1].y - h.w);
        *reinterpret_cast<float4*>(hi + off) = h;
        *reinterpret_cast<float4*>(lo + off) = l;
    } else {
        uint32_t hw[4], lw[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const __nv_bfloat162 h = __floats2bfloat162_rn(x[i].x, x[i].y);
            const float2 hf = __bfloat1622float2(h);
            const __nv_bfloat162 l = __floats2bfloat162_rn(x[i].x - hf.x, x[i].y - hf.y);
            hw[i] = *reinterpret_cast<const uint32_t*>(&h);
            lw[i] = *reinterpret_cast<const uint32_t*>(&l);
        }
        *reinterpret_cast<uint4*>(hi + off) = make_uint4(hw[0], hw[1], hw[2], hw[3]);
        *reinterpret_cast<uint4*>(lo + off) = make_uint4(lw[0], lw[1], lw[2], lw[3]);
    }
}

// B image of the real-ified DFT matrices of sizes R (pass 1) and S (pass 2),
// each N x K, K-major: W_r^{jq} = W_n^{(jq mod r) (n / r)}.
template <bool TF32>
__global__ void dftgemm_image_kernel(const float2* __restrict__ tw, GemmShape sh, unsigned char* __restrict__ out)
{
    const int es = sh.es;
    const int e1 = sh.N1 * sh.K1, total = e1 + sh.N2 * sh.K2;
    for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < total; idx += gridDim.x * blockDim.x) {
        const bool second = idx >= e1;
        const int e = second ? idx - e1 : idx;
        const int K = second ? sh.K2 : sh.K1, r = second ? sh.S : sh.R;
        const int row = e / K, col = e - row * K;
        float v = 0.f;
        const int q = row >> 1, j = col >> 1;
        if (q < r && j < r) {
            const float2 w = tw[((j * q) % r) * (sh.n / r)];      // (c, -s)
            const float c = w.x, s = -w.y;
            const int rr = row & 1, cc = col & 1;
            v = rr == 0 ? (cc == 0 ? c : s) : (cc == 0 ? -s : c);
        }
        unsigned char* hi = out + (second ? sh.b2hi : 0);
        unsigned char* lo = out + (second ? sh.b2lo : sh.b1lo);
        put_split<TF32>(hi, lo, tc::op_offset(row, col, K * es / 16, es), v);
    }
}

// Issue D = A_hi B_hi + A_hi B_lo + A_lo B_hi for one 128-row block (thread 0).
template <bool TF32>
__device__ __forceinline__ void issue_block(uint32_t d_tmem, uint32_t a_hi, uint32_t a_lo, uint32_t b_hi, uint32_t b_lo,
                                            int K, int N, int es)
{
    const int KT = K * es / 16;
    const uint32_t id = tc::idesc(TF32 ? tc::kTypeTF32 : tc::kTypeBF16, 128, N);
    const uint32_t pa[3] = {a_hi, a_hi, a_lo};
    const uint32_t pb[3] = {b_hi, b_lo, b_hi};
    uint32_t acc = 0;
    for (int pr = 0; pr < 3; ++pr)
        for (int kc = 0; kc < KT / 2; ++kc) {
            const uint64_t ad = tc::smem_desc(pa[pr] + kc * 256, 128, KT * 128);
            const uint64_t bd = tc::smem_desc(pb[pr] + kc * 256, 128, KT * 128);
            tc::mma<TF32>(d_tmem, ad, bd, id, acc);
            acc = 1;
        }
}

// Elements of a tile, walked e = tid + kThreads m: (line g, position i).
// Global source of line g: in + (line0 + g lstride) n.
struct TileWalk {
    const float2* line;          // start of line g in global memory
    int g, i;
};

__device__ __forceinline__ void walk_advance(TileWalk& w, const TileGeom& tg, const float2* in, int n)
{
    w.i += kThreads;
    if (w.i >= n) {
        do { w.i -= n; ++w.g; } while (w.i >= n);
        w.line = in + (tg.line0 + (int64_t)w.g * tg.lstride) * n;
    }
}

// Load this thread's elements of `tile` into registers (lines past the end
// of the grouped range read as zero).  cnt = ceil(G n / kThreads) <= kPrefetch.
__device__ __forceinline__ void fetch_regs(const StageArgs& p, const GemmShape& sh, int64_t tile, float2* r, int cnt)
{
    const TileGeom tg = tile_geom(p, tile, sh.G);
    const float2* in = reinterpret_cast<const float2*>(p.in);
    TileWalk w;
    w.g = 0; w.i = threadIdx.x;
    while (w.i >= sh.n) { w.i -= sh.n; ++w.g; }
    w.line = in + (tg.line0 + (int64_t)w.g * tg.lstride) * sh.n;
#pragma unroll
    for (int m = 0; m < kPrefetch; ++m) {
        if (m < cnt) {
            r[m] = (w.g < tg.valid) ? __ldg(w.line + w.i) : make_float2(0.f, 0.f);
            walk_advance(w, tg, in, sh.n);
        }
    }
}

__device__ __forceinline__ void put_regs(const GemmShape& sh, const float2* r, int cnt, float2* lines)
{
    int g = 0, i = threadIdx.x;
    while (i >= sh.n) { i -= sh.n; ++g; }
#pragma unroll
    for (int m = 0; m < kPrefetch; ++m) {
        if (m < cnt) {
            if (g < sh.G) lines[g * sh.np + i] = r[m];
            i += kThreads;
            while (i >= sh.n) { i -= sh.n; ++g; }
        }
    }
}

// Direct load of a tile (tiles too large for the register prefetch).
__device__ __forceinline__ void load_tile(const StageArgs& p, const GemmShape& sh, int64_t tile, float2* lines)
{
    const TileGeom tg = tile_geom(p, tile, sh.G);
    const float2* in = reinterpret_cast<const float2*>(p.in);
    TileWalk w;
    w.g = 0; w.i = threadIdx.x;
    while (w.i >= sh.n) { w.i -= sh.n; ++w.g; }
    w.line = in + (tg.line0 + (int64_t)w.g * tg.lstride) * sh.n;
    while (w.g < sh.G) {
        float2* dst = lines + w.g * sh.np + w.i;
        if (w.g < tg.valid) cp_async<8>(dst, w.line + w.i);
        else *dst = make_float2(0.f, 0.f);
        walk_advance(w, tg, in, sh.n);
    }
    cp_async_wait_all();
}

// Stage block blk of A for pass PASS: row blk * 128 + lane, K groups
// [kk0, kk1) (this warpgroup's half).  Pass 0 rows (g, t) hold x[t + S j]
// (j < R); pass 1 rows (g, k) hold W_n^{jk} Y[j][k] (j < S).
template <bool TF32, int PASS>
__device__ __forceinline__ void stage_block(const GemmShape& sh, const float2* lines, unsigned char* a_hi,
                                            unsigned char* a_lo, const float2* tws, int conj_in, int blk)
{
    constexpr int CPG = TF32 ? 2 : 4;               // complex values per 16-byte K group
    const int K = PASS ? sh.K2 : sh.K1;
    const int KT = K * sh.es / 16;
    const int rows = PASS ? sh.G * sh.R : sh.G * sh.S;
    const int jmax = PASS ? sh.S : sh.R;
    const int div = PASS ? sh.R : sh.S;
    const int step = PASS ? sh.Rp : sh.S;
    const int lane = threadIdx.x & 127, half = threadIdx.x >> 7;
    const int kh = (KT + 1) >> 1;
    const int kk0 = half ? kh : 0, kk1 = half ? KT : kh;
    const int row = blk * 128 + lane;
    const uint32_t base = (uint32_t)(blk * 128 * K * sh.es) + (uint32_t)((lane >> 3) * KT) * 128 + (lane & 7) * 16;
    float2 x[CPG];
    if (row < rows) {
        const int g = row / div, r = row - g * div;
        // groups [kk0, kfull) hold only real entries (j < jmax); [kfull, kk1) the padded tail
        const int kfull = max(kk0, min(kk1, jmax / CPG));
        const float2* sp = lines + g * sh.np + r + kk0 * CPG * step;
        const float2* tp = tws + kk0 * CPG * r;
        uint32_t off = base + kk0 * 128;
        for (int kk = kk0; kk < kfull; ++kk, off += 128) {
#pragma unroll
            for (int c = 0; c < CPG; ++c) {
                float2 v = *sp;
                sp += step;
                if (PASS == 0) {
                    if (conj_in) v.y = -v.y;
                } else {
                    const float2 w = *tp;
                    tp += r;
                    v = make_float2(fmaf(v.x, w.x, -v.y * w.y), fmaf(v.x, w.y, v.y * w.x));
                }
                x[c] = v;
            }
            put_group<TF32>(a_hi, a_lo, off, x);
        }
        for (int kk = kfull; kk < kk1; ++kk, off += 128) {
#pragma unroll
            for (int c = 0; c < CPG; ++c) {
                const int j = kk * CPG + c;
                float2 v = make_float2(0.f, 0.f);
                if (j < jmax) {
                    v = *sp;
                    if (PASS == 0) {
                        if (conj_in) v.y = -v.y;
                    } else {
                        const float2 w = *tp;
                        v = make_float2(fmaf(v.x, w.x, -v.y * w.y), fmaf(v.x, w.y, v.y * w.x));
                    }
                }
                sp += step;
                tp += r;
                x[c] = v;
            }
            put_group<TF32>(a_hi, a_lo, off, x);
        }
    } else {
#pragma unroll
        for (int c = 0; c < CPG; ++c) x[c] = make_float2(0.f, 0.f);
        for (int kk = kk0; kk < kk1; ++kk) put_group<TF32>(a_hi, a_lo, base + kk * 128, x);
    }
}

// One GEMM pass: each 128-row block is staged and its MMAs issued (block b
// accumulates in tensor-memory columns 64 b .. and completes on mbar[b]) while
// the next block is staged; then every block's rows are written back: pass 0
// writes Y[t][q] to line position t * Rp + q, pass 1 writes Z[k + R q].
// Returns false (every thread) when a completion wait ran out.
template <bool TF32, int PASS>
__device__ __forceinline__ bool gemm_pass(const GemmShape& sh, float2* lines, unsigned char* smem, const float2* tws,
                                          int conj_in, uint32_t d_tmem, uint64_t* mbar, uint32_t& phases,
                                          int* status, int* s_abort, long long budget, int skip_mma)
{
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 127, half = tid >> 7;
    const int K = PASS ? sh.K2 : sh.K1, N = PASS ? sh.N2 : sh.N1;
    const int rows = PASS ? sh.G * sh.R : sh.G * sh.S;
    const int nblk = (PASS ? sh.M2 : sh.M1) / 128;
    const int qmax = PASS ? sh.S : sh.R;
    const int div = PASS ? sh.R : sh.S;
    unsigned char* a_hi = smem + sh.off_ahi;
    unsigned char* a_lo = smem + sh.off_alo;
    for (int blk = 0; blk < nblk; ++blk) {
        stage_block<TF32, PASS>(sh, lines, a_hi, a_lo, tws, conj_in, blk);
        tc::fence_smem_to_async();
        tc::fence_before_sync();
        __syncthreads();
        if (tid == 0 && !skip_mma) {
            tc::fence_after_sync();
            const uint32_t bb = tc::smem_u32(smem + sh.off_b);
            const uint32_t bh = PASS ? bb + sh.b2hi : bb, bl = bb + (PASS ? sh.b2lo : sh.b1lo);
            const uint32_t ao = (uint32_t)(blk * 128 * K * sh.es);
            issue_block<TF32>(d_tmem + (uint32_t)(64 * blk), tc::smem_u32(a_hi) + ao, tc::smem_u32(a_lo) + ao,
                              bh, bl, K, N, sh.es);
            tc::commit(&mbar[blk]);
        }
    }
    // Completion: the commit after the last block tracks every MMA of the
    // pass.  Warp 0 polls it; the other warps wait at the barrier, where they
    // take no issue slots from the other CTAs on the SM.
    const int last = nblk - 1;
    if (warp == 0) {
        bool ok = tc::mbar_wait(&mbar[last], (phases >> last) & 1u, budget);
        ok = __all_sync(0xffffffffu, ok);
        if (!ok && tid == 0) { atomicCAS(status, OPENFFT_OK, OPENFFT_ERR_TIMEOUT); *s_abort = 1; }
    }
    phases ^= (1u << nblk) - 1u;                      // every block's barrier completed one phase
    __syncthreads();
    if (*s_abort) return false;
    tc::fence_after_sync();
    const int qs = PASS ? sh.R : 1;
    for (int blk = 0; blk < nblk; ++blk) {
        const int row = blk * 128 + lane;
        const bool live = row < rows;
        const int g = live ? row / div : 0, r = live ? row - g * div : 0;
        float2* dst = PASS ? lines + g * sh.np + r : lines + g * sh.np + r * sh.Rp;
        const uint32_t taddr = d_tmem + ((uint32_t)((warp & 3) * 32) << 16) + (uint32_t)(64 * blk);
        // this warpgroup's 16-column chunks: 16 half + 32 i (at most two, N <= 64)
        const int c0 = 16 * half;
        if (c0 >= N) continue;
        float v[32];
        const bool two = c0 + 32 < N;
        if (two) tc::ld16x2(taddr + (uint32_t)c0, taddr + (uint32_t)(c0 + 32), v);
        else tc::ld16(taddr + (uint32_t)c0, v);
        if (live) {
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                const int q = (c0 >> 1) + i;
                if (q < qmax) dst[q * qs] = make_float2(v[2 * i], v[2 * i + 1]);
            }
            if (two) {
#pragma unroll
                for (int i = 0; i < 8; ++i) {
                    const int q = ((c0 + 32) >> 1) + i;
                    if (q < qmax) dst[q * qs] = make_float2(v[16 + 2 * i], v[16 + 2 * i + 1]);
                }
            }
        }
    }
    tc::fence_before_sync();
    __syncthreads();
    return *s_abort == 0;
}

// Write the tile to the next ordering (conjugation and scale of backward
// transforms at the store).
__device__ __forceinline__ void store_tile(const StageArgs& p, const GemmShape& sh, int64_t tile, const float2* lines)
{
    const TileGeom tg = tile_geom(p, tile, sh.G);
    float2* first = reinterpret_cast<float2*>(p.out) + tg.obase;
    const float sc = (float)p.scale;
    const int n = sh.n, G = sh.G, tid = threadIdx.x;
    if (!p.contig_store) {
        const int g = tid & (G - 1), slot = tid / G, kstep = kThreads / G;
        if (g < tg.valid) {
            float2* o = first + g * tg.ostride + (int64_t)slot * p.Sk;
            const int64_t ostep = (int64_t)kstep * p.Sk;
            for (int k = slot; k < n; k += kstep, o += ostep) {
                float2 v = lines[g * sh.np + k];
                if (p.conj_out) v = make_float2(v.x * sc, -v.y * sc);
                *o = v;
            }
        }
    } else {
        int g = 0, k = tid;
        while (k >= n) { k -= n; ++g; }
        while (g < tg.valid) {
            float2 v = lines[g * sh.np + k];
            if (p.conj_out) v = make_float2(v.x * sc, -v.y * sc);
            first[g * tg.ostride + (int64_t)k * p.Sk] = v;
            k += kThreads;
            while (k >= n) { k -= n; ++g; }
        }
    }
}

template <bool TF32>
__global__ void __launch_bounds__(kThreads) dftgemm_kernel(const StageArgs p, const GemmShape sh, int64_t ntiles,
                                                           int* status)
{
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ __align__(8) uint64_t mbar[kMaxBlocks];
    __shared__ uint32_t tmem_base;
    __shared__ int s_abort;
    const int tid = threadIdx.x, warp = tid >> 5;
    float2* const lines = reinterpret_cast<float2*>(smem + sh.off_lines);
    float2* const tws = reinterpret_cast<float2*>(smem + sh.off_tw);
    const int cnt = (sh.G * sh.n + kThreads - 1) / kThreads;
    const bool prefetch = cnt <= kPrefetch;
    const long long budget = g_wait_budget;
    const int skip_mma = g_skip_mma;

    // B image and twiddle table -> shared memory
    const char* bsrc = reinterpret_cast<const char*>(p.aux);
    for (int o = tid * 16; o < sh.b_bytes; o += kThreads * 16) cp_async<16>(smem + sh.off_b + o, bsrc + o);
    const float2* twg = reinterpret_cast<const float2*>(p.tw);
    for (int i = tid; i < sh.n; i += kThreads) tws[i] = twg[i];
    if (warp == 0) tc::tmem_alloc(&tmem_base, (uint32_t)sh.tcols);
    if (tid == 0) {
        for (int b = 0; b < kMaxBlocks; ++b) tc::mbar_init(&mbar[b], 1);
        s_abort = 0;
    }
    cp_async_wait_all();
    int64_t tile = blockIdx.x;
    float2 r[kPrefetch];
    if (tile < ntiles && prefetch) {
        fetch_regs(p, sh, tile, r, cnt);
        put_regs(sh, r, cnt, lines);
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t d_tmem = tmem_base;
    uint32_t phases = 0;                              // bit b: phase of mbar[b]

    for (; tile < ntiles; tile += gridDim.x) {
        const int64_t next = tile + gridDim.x;
        if (!prefetch) {
            load_tile(p, sh, tile, lines);
            __syncthreads();
        } else if (next < ntiles) {
            fetch_regs(p, sh, next, r, cnt);          // in flight while this tile runs
        }
        if (!gemm_pass<TF32, 0>(sh, lines, smem, tws, p.conj_in, d_tmem, mbar, phases, status, &s_abort, budget,
                                skip_mma)) break;
        if (!gemm_pass<TF32, 1>(sh, lines, smem, tws, 0, d_tmem, mbar, phases, status, &s_abort, budget,
                                skip_mma)) break;
        store_tile(p, sh, tile, lines);
        __syncthreads();                              // every read of this tile's lines is done
        if (prefetch && next < ntiles) {
            put_regs(sh, r, cnt, lines);
            __syncthreads();
        }
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(d_tmem, (uint32_t)sh.tcols);
}

// Least np >= S * Rp that is an odd multiple of 16 / G (G <= 16), odd for G >= 16.
int line_stride(int base, int G)
{
    const int m = G >= 16 ? 1 : 16 / G;
    int np = pad_to(base, m);
    if ((np / m) % 2 == 0) np += m;
    return np;
}

GemmShape make_shape(int n, int R, int S, int G, bool tf32)
{
    GemmShape g;
    const int kstep = tf32 ? 8 : 16;
    g.n = n; g.R = R; g.S = S; g.G = G; g.es = tf32 ? 4 : 2;
    g.Rp = R | 1;
    g.np = line_stride(S * g.Rp, G);
    g.K1 = pad_to(2 * R, kstep); g.N1 = pad_to(2 * R, 16);
    g.K2 = pad_to(2 * S, kstep); g.N2 = pad_to(2 * S, 16);
    g.M1 = pad_to(G * S, 128); g.M2 = pad_to(G * R, 128);
    const int nblk = std::max(g.M1, g.M2) / 128;
    g.tcols = nblk <= 1 ? 64 : (nblk <= 2 ? 128 : (nblk <= 4 ? 256 : 512));
    const int s1 = g.N1 * g.K1 * g.es, s2 = g.N2 * g.K2 * g.es;
    g.b1lo = s1; g.b2hi = 2 * s1; g.b2lo = 2 * s1 + s2;
    g.b_bytes = 2 * s1 + 2 * s2;
    int off = 0;
    auto take = [&](int bytes) { const int o = off; off += pad_to(bytes, 128); return o; };
    g.off_lines = take(G * g.np * 8);
    const int abytes = std::max(g.M1 * g.K1, g.M2 * g.K2) * g.es;
    g.off_ahi = take(abytes); g.off_alo = take(abytes);
    g.off_b = take(g.b_bytes);
    g.off_tw = take(n * 8);
    g.smem = off;
    return g;
}

}  // namespace

cudaError_t dftgemm_test_controls(int what, long long value)
{
    if (what == 1) {
        const long long b = value > 0 ? value : kWaitBudget;
        return cudaMemcpyToSymbol(g_wait_budget, &b, sizeof(b));
    }
    const int v = value != 0;
    return cudaMemcpyToSymbol(g_skip_mma, &v, sizeof(v));
}

// Factor n = R S (2 <= R, S <= 32) with the least padded GEMM work.
bool dftgemm_factor(int n, int tf32, int* R, int* S)
{
    const int kstep = tf32 ? 8 : 16;
    long best = -1;
    for (int r = 2; r <= 32; ++r) {
        if (n % r) continue;
        const int s = n / r;
        if (s < 2 || s > 32) continue;
        const long cost = (long)s * pad_to(2 * r, kstep) * pad_to(2 * r, 16) + (long)r * pad_to(2 * s, kstep) * pad_to(2 * s, 16);
        if (best < 0 || cost < best) { best = cost; *R = r; *S = s; }
    }
    return best >= 0;
}

size_t dftgemm_image_bytes(int n, int R, int S, bool tf32)
{
    return (size_t)make_shape(n, R, S, 1, tf32).b_bytes;
}

cudaError_t launch_dftgemm_image(int n, int R, int S, bool tf32, const void* tw, void* out, cudaStream_t st)
{
    const GemmShape sh = make_shape(n, R, S, 1, tf32);
    const int total = sh.N1 * sh.K1 + sh.N2 * sh.K2;
    const int blocks = (total + 255) / 256;
    if (tf32) dftgemm_image_kernel<true><<<blocks, 256, 0, st>>>((const float2*)tw, sh, (unsigned char*)out);
    else dftgemm_image_kernel<false><<<blocks, 256, 0, st>>>((const float2*)tw, sh, (unsigned char*)out);
    return cudaGetLastError();
}

cudaError_t launch_dftgemm(const StageLaunch& L, cudaStream_t st, int* status)
{
    const StageArgs& a = L.args;
    const bool tf32 = L.arith == ARITH_TC_TF32;
    const int R = a.radix[0], S = a.radix[1];
    const GemmShape sh = make_shape(a.n, R, S, a.G, tf32);
    // resident CTAs: the kernel's own limits, and 512 tensor-memory columns per
    // SM (a CTA that cannot allocate would wait for another to finish)
    int per_sm = 1;
    cudaError_t e = tf32 ? persistent_ctas_per_sm((const void*)dftgemm_kernel<true>, kThreads, sh.smem, &per_sm)
                         : persistent_ctas_per_sm((const void*)dftgemm_kernel<false>, kThreads, sh.smem, &per_sm);
    if (e) return e;
    per_sm = std::max(1, std::min(per_sm, 512 / sh.tcols));
    const int64_t ntiles = L.grid;
    int64_t grid = (int64_t)L.sms * per_sm;
    if (grid > ntiles) grid = ntiles;
    if (grid < 1) grid = 1;
    if (tf32) dftgemm_kernel<true><<<(unsigned)grid, kThreads, sh.smem, st>>>(a, sh, ntiles, status);
    else dftgemm_kernel<false><<<(unsigned)grid, kThreads, sh.smem, st>>>(a, sh, ntiles, status);
    return cudaGetLastError();
}

// Lines per tile: Gt (a power of two, <= 16) halved until the shared memory
// fits, and while it is above 4 until two CTAs fit on an SM (a single CTA per
// SM leaves the MMA and barrier latencies of a tile exposed).
int dftgemm_lines(int n, int R, int S, bool tf32, int Gt)
{
    auto fits = [&](int G) {
        const GemmShape sh = make_shape(n, R, S, G, tf32);
        return sh.smem <= 200 * 1024 && sh.tcols <= 256;
    };
    int G = Gt < 1 ? 1 : (Gt > 16 ? 16 : Gt);
    while (G > 1 && !fits(G)) G /= 2;
    while (G > 4 && make_shape(n, R, S, G, tf32).smem > 112 * 1024) G /= 2;
    return fits(G) ? G : 0;
}

}  // namespace ofg
