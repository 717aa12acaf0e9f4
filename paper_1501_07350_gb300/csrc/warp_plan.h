// warp_plan.h -- radix plan of the warp-per-line stage kernel.  Power-of-two
// line lengths n = 32..512: the remainder radix (n / 8^k, which is 1, 2 or 4)
// first, then radix 8.  The mixed-radix lengths 48..160: the radices 8, 4, 2,
// 3, 5, 7 in that order, as many times as each divides.  Pass p combines R_p
// sub-transforms of length m_p (the product of the earlier radices) with the
// twiddles W_n^(j k s_p), j < R_p, k < m_p, s_p = n / (m_p R_p).
//
// The packed double-float policy reads those twiddles from per-pass tables:
// pass p >= 1 keeps entry (j, k) at wtw_offset(n, p) + (j - 1) m_p + k, so a
// warp's lanes (consecutive k) read consecutive entries.  The tables of all
// passes together hold wtw_count(n) < n entries.
#pragma once

namespace ofg {

__host__ __device__ constexpr bool warp_pow2(int n) { return n > 0 && (n & (n - 1)) == 0; }
// the mixed-radix lengths the warp kernel is instantiated for
__host__ __device__ constexpr bool warp_mixed_length(int n)
{
    return n == 48 || n == 96 || n == 100 || n == 108 || n == 120 || n == 144 || n == 160;
}
__host__ __device__ constexpr bool warp_length(int n)
{
    return (n >= 32 && n <= 512 && warp_pow2(n)) || warp_mixed_length(n);
}

__host__ __device__ constexpr int wplan_len(int n)
{
    int c = 0;
    if (warp_pow2(n)) {
        while (n % 8 == 0) { n /= 8; ++c; }
        return c + (n > 1 ? 1 : 0);
    }
    const int rs[6] = {8, 4, 2, 3, 5, 7};
    for (int r : rs)
        while (n % r == 0) { n /= r; ++c; }
    return c;
}

__host__ __device__ constexpr int wplan_radix(int n, int idx)
{
    if (warp_pow2(n)) {
        int r = n;
        while (r % 8 == 0) r /= 8;
        if (r > 1) return idx == 0 ? r : 8;
        return 8;
    }
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
