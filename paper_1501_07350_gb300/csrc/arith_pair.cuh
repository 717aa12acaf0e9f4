// arith_pair.cuh -- the double-float arithmetic of arith.cuh (ArDF) with the
// real and imaginary lanes of every step in one packed FP32x2 instruction.
//
// sm_100 and later execute add / sub / mul / fma on .f32x2 operands: two IEEE
// binary32 operations, each rounded to nearest, in one instruction.  A packed
// instruction takes one issue slot for two lanes and holds the FMA pipe for two
// cycles, so the FP32 work per lane is that of scalar instructions at half the
// issue slots.  With scalar instructions the double-float stage kernels were
// bound by instruction issue; with packed ones the FMA pipe is their limit.
//
// Representation (ArDP): a complex value is C = {h, l}, h = (re.hi, im.hi) and
// l = (re.lo, im.lo), each a 64-bit register pair -- the same 16 bytes, in the
// same order, as ArDF's float4 (re.hi, im.hi, re.lo, im.lo), so the two
// policies share every global and shared-memory format.  Additions, the
// butterflies' multiplications by -i and the real scalings perform per lane
// exactly the operations of ArDF, in the same order, so results are bit for
// bit those of ArDF.  The twiddle product computes the same terms; only the
// order of the four first-order terms of the imaginary lo part differs.
//
// There is no packed negation: a twiddle product's rounding error
// e = fma(a, b, -p) is formed as -e = fma(a, -b, p) with the negated factor
// among the twiddle's lane pairs (sign-bit flips of the table entry) and the
// sign folded into the next addition; a scaling by a constant negates p by its
// sign bits.  Multiplication by -i swaps the lanes of a pair, which costs
// register moves, so the radix-4 and radix-8 butterflies fuse it into the
// addition that consumes it (add_mi / sub_mi, lane signs through fma by
// (+1, -1)).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "arith.cuh"

namespace ofg {

using u64 = unsigned long long;

__device__ __forceinline__ u64 p2_add(u64 a, u64 b)
{
    u64 d;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ u64 p2_sub(u64 a, u64 b)
{
    u64 d;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ u64 p2_mul(u64 a, u64 b)
{
    u64 d;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ u64 p2_fma(u64 a, u64 b, u64 c)
{
    u64 d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}
// (lo lane, hi lane) -> 64-bit pair
__device__ __forceinline__ u64 p2_pack(float lo, float hi)
{
    u64 d;
    asm("mov.b64 %0, {%1, %2};" : "=l"(d) : "f"(lo), "f"(hi));
    return d;
}
__device__ __forceinline__ void p2_unpack(u64 v, float& lo, float& hi)
{
    asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v));
}
__device__ __forceinline__ u64 p2_swap(u64 v)
{
    float lo, hi;
    p2_unpack(v, lo, hi);
    return p2_pack(hi, lo);
}
__device__ __forceinline__ u64 p2_splat(float x) { return p2_pack(x, x); }

// lane signs of -i d = (d.im, -d.re) once d's lanes are swapped
constexpr u64 kSgnPM = 0xBF8000003F800000ull;   // (+1, -1)
constexpr u64 kSgnMP = 0x3F800000BF800000ull;   // (-1, +1)
constexpr u64 kSignHi = 0x8000000000000000ull;  // sign bit of the high lane
constexpr u64 kSignLo = 0x0000000080000000ull;  // sign bit of the low lane
constexpr u64 kSignBoth = 0x8000000080000000ull;  // sign bits of both lanes

struct ArDP {
    using C = ulonglong2;                 // x = (re.hi, im.hi), y = (re.lo, im.lo)
    // Twiddle w = (x + z) + i (y + w) (the float4 of ArDF's table) as the
    // lane pairs of the packed product:
    //   a = (t0, t0n), t0 = (x, x), t0n = (-x, -x);  b = (t1, t1n), t1 = (-y, y), t1n = (y, -y);
    //   c = (t2, t3), t2 = (z, z), t3 = (-w, w).
    struct W { ulonglong2 a, b, c; };
    static constexpr int kElemBytes = 16;

    // The FMT_DF twiddle table of a power-of-two length n <= 512 holds n
    // float4 entries (ArDF) followed by the per-pass table of the warp
    // kernel's radix plan (warp_plan.h): entry e = off_p + (j - 1) m + k is
    // the float4 (x, y, z, w) of W_n^(j k s_p), so a warp's lanes read
    // consecutive entries.  table() points at the per-pass table.  The lane
    // pairs of W are built from the entry with sign-bit operations (integer
    // pipe): one 16-byte load per twiddle instead of three.
    __device__ __forceinline__ static const W* table(const void* tw, int n)
    {
        return reinterpret_cast<const W*>(reinterpret_cast<const char*>(tw) + 16 * (size_t)n);
    }
    template <int N>
    __device__ __forceinline__ static W warp_twiddle(const W* tw, int off, int m, int j, int k, int)
    {
        const int e = off + (j - 1) * m + k;
        const float4 q = __ldg(reinterpret_cast<const float4*>(tw) + e);
        const u64 xx = p2_splat(q.x), yy = p2_splat(q.y), zz = p2_splat(q.z), ww = p2_splat(q.w);
        W w;
        w.a.x = xx;
        w.a.y = xx ^ kSignBoth;            // (-x, -x)
        w.b.x = yy ^ kSignLo;              // (-y, y)
        w.b.y = yy ^ kSignHi;              // (y, -y)
        w.c.x = zz;
        w.c.y = ww ^ kSignLo;              // (-w, w)
        return w;
    }

    __device__ __forceinline__ static C make(u64 h, u64 l) { C r; r.x = h; r.y = l; return r; }
    __device__ __forceinline__ static C zero() { return make(0ull, 0ull); }

    // Knuth TwoSum on both lanes: s + e == a + b exactly (per lane).
    __device__ __forceinline__ static void two_sum(u64 a, u64 b, u64& s, u64& e)
    {
        s = p2_add(a, b);
        const u64 bb = p2_sub(s, a);
        e = p2_add(p2_sub(a, p2_sub(s, bb)), p2_sub(b, bb));
    }
    __device__ __forceinline__ static C add(C a, C b)
    {
        u64 s, e;
        two_sum(a.x, b.x, s, e);
        return make(s, p2_add(e, p2_add(a.y, b.y)));
    }
    // TwoSum(a, -b): the error term (-b) - bb is formed as -(b + bb)
    __device__ __forceinline__ static C sub(C a, C b)
    {
        const u64 s = p2_sub(a.x, b.x);
        const u64 bb = p2_sub(s, a.x);
        const u64 u = p2_sub(a.x, p2_sub(s, bb));
        const u64 e = p2_sub(u, p2_add(b.x, bb));
        return make(s, p2_add(e, p2_sub(a.y, b.y)));
    }
    // b + sg * ds, lane-wise, where ds = d with swapped lanes and sg a pair of
    // signs; ng = -sg.  With (sg, ng) = ((+1,-1), (-1,+1)) this is b + (-i) d,
    // with the two exchanged b - (-i) d.
    __device__ __forceinline__ static C add_signed(C b, u64 dsh, u64 dsl, u64 sg, u64 ng)
    {
        const u64 s = p2_fma(dsh, sg, b.x);
        const u64 bb = p2_sub(s, b.x);
        const u64 u = p2_sub(b.x, p2_sub(s, bb));
        const u64 e = p2_sub(u, p2_fma(dsh, ng, bb));
        return make(s, p2_add(e, p2_fma(dsl, sg, b.y)));
    }
    __device__ __forceinline__ static C add_mi(C b, C d)      // b + (-i) d
    {
        return add_signed(b, p2_swap(d.x), p2_swap(d.y), kSgnPM, kSgnMP);
    }
    __device__ __forceinline__ static C sub_mi(C b, C d)      // b - (-i) d
    {
        return add_signed(b, p2_swap(d.x), p2_swap(d.y), kSgnMP, kSgnPM);
    }
    // both from one swap of d
    __device__ __forceinline__ static void addsub_mi(C b, C d, C& plus, C& minus)
    {
        const u64 dsh = p2_swap(d.x), dsl = p2_swap(d.y);
        plus = add_signed(b, dsh, dsl, kSgnPM, kSgnMP);
        minus = add_signed(b, dsh, dsl, kSgnMP, kSgnPM);
    }

    // a * w: hi products exact (FMA TwoProduct), first-order lo terms.
    __device__ __forceinline__ static C mul(C a, const W& w)
    {
        const u64 ahs = p2_swap(a.x), als = p2_swap(a.y);
        const u64 p = p2_mul(a.x, w.a.x);                 // (x.re w.re, x.im w.re)
        const u64 en = p2_fma(a.x, w.a.y, p);             // minus its rounding error
        const u64 q = p2_mul(ahs, w.b.x);                 // (-x.im w.im, x.re w.im)
        const u64 fn = p2_fma(ahs, w.b.y, q);
        u64 s, es;
        two_sum(p, q, s, es);
        u64 l = p2_sub(es, p2_add(en, fn));
        l = p2_fma(a.x, w.c.x, l);
        l = p2_fma(a.y, w.a.x, l);
        l = p2_fma(ahs, w.c.y, l);
        l = p2_fma(als, w.b.x, l);
        return make(s, l);
    }
    // multiply by the real constant k = kh + kl.  The product's rounding
    // error is fma(a, kh, -p) with -p formed by flipping both sign bits: with
    // -p formed as a product by the negated constant, ptxas (-O1 and above)
    // was seen to lose the error term.
    __device__ __forceinline__ static C scale(C a, double k)
    {
        const float kh = (float)k;
        const float kl = (float)(k - (double)kh);
        const u64 KH = p2_splat(kh), KL = p2_splat(kl);
        const u64 p = p2_mul(a.x, KH);
        u64 e = p2_fma(a.x, KH, p ^ kSignBoth);
        e = p2_fma(a.x, KL, e);
        e = p2_fma(a.y, KH, e);
        return make(p, e);
    }
    __device__ __forceinline__ static C mul_mi(C a)
    {
        return make(p2_swap(a.x) ^ kSignHi, p2_swap(a.y) ^ kSignHi);   // (im, -re)
    }
    __device__ __forceinline__ static C conj(C a) { return make(a.x ^ kSignHi, a.y ^ kSignHi); }

    __device__ __forceinline__ static C from_float4(float4 v)
    {
        return make(p2_pack(v.x, v.y), p2_pack(v.z, v.w));
    }
    __device__ __forceinline__ static float4 to_float4(C v)
    {
        float4 r;
        p2_unpack(v.x, r.x, r.y);
        p2_unpack(v.y, r.z, r.w);
        return r;
    }
};

// Butterflies of the paired policy: the -i factors fused into the additions.
template <> struct Dft<ArDP, 2> {
    __device__ __forceinline__ static void run(ArDP::C* x)
    {
        const auto t = ArDP::sub(x[0], x[1]);
        x[0] = ArDP::add(x[0], x[1]);
        x[1] = t;
    }
};

template <> struct Dft<ArDP, 4> {
    __device__ __forceinline__ static void run(ArDP::C* x)
    {
        const auto a = ArDP::add(x[0], x[2]), b = ArDP::sub(x[0], x[2]);
        const auto c = ArDP::add(x[1], x[3]), d = ArDP::sub(x[1], x[3]);
        x[0] = ArDP::add(a, c);
        x[2] = ArDP::sub(a, c);
        ArDP::addsub_mi(b, d, x[1], x[3]);            // b + (-i) d, b - (-i) d
    }
};

template <> struct Dft<ArDP, 8> {
    __device__ __forceinline__ static void run(ArDP::C* x)
    {
        ArDP::C e[4] = {x[0], x[2], x[4], x[6]};
        ArDP::C o[4] = {x[1], x[3], x[5], x[7]};
        Dft<ArDP, 4>::run(e);
        Dft<ArDP, 4>::run(o);
        // W8 o1 = (o1 + (-i) o1) / sqrt2;  W8^3 o3 = ((-i) o3 - o3) / sqrt2 = -t3
        const auto o1 = ArDP::scale(ArDP::add_mi(o[1], o[1]), kSqrtHalf);
        const auto t3 = ArDP::scale(ArDP::sub_mi(o[3], o[3]), kSqrtHalf);
        x[0] = ArDP::add(e[0], o[0]); x[4] = ArDP::sub(e[0], o[0]);
        x[1] = ArDP::add(e[1], o1);   x[5] = ArDP::sub(e[1], o1);
        ArDP::addsub_mi(e[2], o[2], x[2], x[6]);      // e2 +- W8^2 o2, W8^2 = -i
        x[3] = ArDP::sub(e[3], t3);   x[7] = ArDP::add(e[3], t3);
    }
};

}  // namespace ofg
