// warp_plan.h -- radix plan of the warp-per-line stage kernel for power-of-two
// line lengths n = 32..512: the remainder radix (n / 8^k, which is 1, 2 or 4)
// first, then radix 8.  Pass p combines R_p sub-transforms of length m_p (the
// product of the earlier radices) with the twiddles W_n^(j k s_p), j < R_p,
// k < m_p, s_p = n / (m_p R_p).
//
// The packed double-float policy reads those twiddles from per-pass tables:
// pass p >= 1 keeps entry (j, k) at wtw_offset(n, p) + (j - 1) m_p + k, so a
// warp's lanes (consecutive k) read consecutive entries.  The tables of all
// passes together hold wtw_count(n) < n entries.
#pragma once

namespace ofg {

constexpr bool warp_length(int n) { return n >= 32 && n <= 512 && (n & (n - 1)) == 0; }

__host__ __device__ constexpr int wplan_len(int n)
{
    int c = 0;
    while (n % 8 == 0) { n /= 8; ++c; }
    return c + (n > 1 ? 1 : 0);
}

__host__ __device__ constexpr int wplan_radix(int n, int idx)
{
    int r = n;
    while (r % 8 == 0) r /= 8;
    if (r > 1) return idx == 0 ? r : 8;
    return 8;
}

__host__ __device__ constexpr int wplan_m(int n, int idx)
{
    int m = 1;
    for (int i = 0; i < idx; ++i) m *= wplan_radix(n, i);
    return m;
}

// first entry of pass p's twiddle table (passes 1 .. wplan_len - 1)
__host__ __device__ constexpr int wtw_offset(int n, int p)
{
    int off = 0;
    for (int i = 1; i < p; ++i) off += (wplan_radix(n, i) - 1) * wplan_m(n, i);
    return off;
}

__host__ __device__ constexpr int wtw_count(int n) { return wtw_offset(n, wplan_len(n)); }

}  // namespace ofg
