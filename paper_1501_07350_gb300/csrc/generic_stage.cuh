// generic_stage.cuh -- the stage computation for any supported line length
// (factors 2, 3, 5, 7; runtime radix plan), as a device function used by the
// generic stage kernel and by the batched kernel.
//
// Radix pass (Stockham autosort, decimation in time).  After the passes with
// radices r_1..r_p (product m) the line holds, for every residue t < s = n/m,
// the m-point DFT of the subsequence x[t + s u] at positions t m + k.  The
// next radix r (s' = s / r) combines r of them:
//   Y'[t'][k + m q] = sum_j W_r^{j q} (W_{m r}^{j k} Y[t' + s' j][k]),
// with W_{m r}^{j k} = W_n^{j k s'} read from the twiddle table of length n.
#pragma once
#include <type_traits>

#include "arith.cuh"
#include "fft_stage.h"
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

// One tile (G lines) of a stage with any supported length: runtime radix plan,
// two ping-pong shared-memory tiles of n x (G + 1) elements at smem_raw.
// s_in / s_out: shared scratch of kMaxLinesPerCta entries each.
template <class A>
__device__ __forceinline__ void generic_stage_tile(const StageArgs& p, int64_t cta, unsigned char* smem_raw,
                                                   int64_t* s_in, int64_t* s_out)
{
    using C = typename A::C;
    const int tid = threadIdx.x;
    const int G = p.G, ld = G + 1, n = p.n;
    C* buf0 = reinterpret_cast<C*>(smem_raw);
    C* buf1 = buf0 + (size_t)n * ld;

    if (tid < G) {
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
            if (base >= 0) {
                if (in_bounds(p.chk, base + i, p.in_elems)) cp_async<EB>(dst, src + (base + i) * EB);
            } else {
                *dst = A::zero();
            }
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
            if (base >= 0 && in_bounds(p.chk, base + k * p.Sk, p.out_elems)) {
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
            if (base < 0 || !in_bounds(p.chk, base + k * p.Sk, p.out_elems)) continue;
            C v = cur[k * ld + g];
            if (p.conj_out) v = A::conj(v);
            if (scale) v = A::scale(v, p.scale);
            Io<A>::store(p.out, p.out_fmt, base + k * p.Sk, v);
        }
    }
}

}  // namespace ofg
