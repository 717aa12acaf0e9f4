// arith.cuh -- complex arithmetic policies of the FFT stage kernels and the
// small DFT butterflies built on them.
//
// A policy A provides the register/shared-memory complex type A::C, the
// twiddle-table entry type A::W, and add/sub/multiply/real-scale operations.
//   ArF64 : IEEE double on the FP64 units.
//   ArF32 : IEEE float.
//   ArDF  : "double-float": a value is hi + lo with hi, lo floats, combined by
//           error-free transformations (Knuth's TwoSum, Dekker/FMA TwoProduct)
//           on the FP32 units.  Renormalisation is lazy: lo collects the
//           rounding errors of hi and its own error is O(u^2) of the operand
//           magnitudes, which keeps the norm-wise FFT error near 1e-14.
//
// The butterflies compute the forward DFT y_q = sum_j x_j exp(-2 pi i j q / r);
// the backward transform is obtained by conjugating on load and on store.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace ofg {

// --------------------------------------------------------------- FP64 ----
struct ArF64 {
    using C = double2;
    using W = double2;
    static constexpr int kElemBytes = 16;
    // twiddle table of a line length n (one W per exponent) and its load
    __device__ __forceinline__ static const W* table(const void* tw, int) { return reinterpret_cast<const W*>(tw); }
    __device__ __forceinline__ static W ldw(const W* p) { return __ldg(p); }
    // twiddle W_N^(j ks) of a warp-kernel pass (the per-pass arguments are
    // for policies with per-pass tables)
    template <int N>
    __device__ __forceinline__ static W warp_twiddle(const W* tw, int, int, int j, int, int ks) { return __ldg(tw + j * ks); }
    __device__ __forceinline__ static C zero() { return make_double2(0.0, 0.0); }
    __device__ __forceinline__ static C add(C a, C b) { return make_double2(a.x + b.x, a.y + b.y); }
    __device__ __forceinline__ static C sub(C a, C b) { return make_double2(a.x - b.x, a.y - b.y); }
    __device__ __forceinline__ static C mul(C a, W w) {
        return make_double2(fma(a.x, w.x, -a.y * w.y), fma(a.x, w.y, a.y * w.x));
    }
    // multiply by the real constant k
    __device__ __forceinline__ static C scale(C a, double k) { return make_double2(a.x * k, a.y * k); }
    // multiply by -i
    __device__ __forceinline__ static C mul_mi(C a) { return make_double2(a.y, -a.x); }
    __device__ __forceinline__ static C conj(C a) { return make_double2(a.x, -a.y); }
};

// --------------------------------------------------------------- FP32 ----
struct ArF32 {
    using C = float2;
    using W = float2;
    static constexpr int kElemBytes = 8;
    // twiddle table of a line length n (one W per exponent) and its load
    __device__ __forceinline__ static const W* table(const void* tw, int) { return reinterpret_cast<const W*>(tw); }
    __device__ __forceinline__ static W ldw(const W* p) { return __ldg(p); }
    // twiddle W_N^(j ks) of a warp-kernel pass (the per-pass arguments are
    // for policies with per-pass tables)
    template <int N>
    __device__ __forceinline__ static W warp_twiddle(const W* tw, int, int, int j, int, int ks) { return __ldg(tw + j * ks); }
    __device__ __forceinline__ static C zero() { return make_float2(0.f, 0.f); }
    __device__ __forceinline__ static C add(C a, C b) { return make_float2(a.x + b.x, a.y + b.y); }
    __device__ __forceinline__ static C sub(C a, C b) { return make_float2(a.x - b.x, a.y - b.y); }
    __device__ __forceinline__ static C mul(C a, W w) {
        return make_float2(fmaf(a.x, w.x, -a.y * w.y), fmaf(a.x, w.y, a.y * w.x));
    }
    __device__ __forceinline__ static C scale(C a, double k) {
        const float kf = (float)k;
        return make_float2(a.x * kf, a.y * kf);
    }
    __device__ __forceinline__ static C mul_mi(C a) { return make_float2(a.y, -a.x); }
    __device__ __forceinline__ static C conj(C a) { return make_float2(a.x, -a.y); }
};

// -------------------------------------------------------- double-float ----
// C = (re.hi, im.hi, re.lo, im.lo); value = (x + z) + i (y + w).
struct ArDF {
    using C = float4;
    using W = float4;
    static constexpr int kElemBytes = 16;
    // twiddle table of a line length n (one W per exponent) and its load
    __device__ __forceinline__ static const W* table(const void* tw, int) { return reinterpret_cast<const W*>(tw); }
    __device__ __forceinline__ static W ldw(const W* p) { return __ldg(p); }
    // twiddle W_N^(j ks) of a warp-kernel pass (the per-pass arguments are
    // for policies with per-pass tables)
    template <int N>
    __device__ __forceinline__ static W warp_twiddle(const W* tw, int, int, int j, int, int ks) { return __ldg(tw + j * ks); }

    // Knuth TwoSum: s + e == a + b exactly.
    __device__ __forceinline__ static void two_sum(float a, float b, float& s, float& e) {
        s = __fadd_rn(a, b);
        float bb = __fsub_rn(s, a);
        e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    }
    __device__ __forceinline__ static C zero() { return make_float4(0.f, 0.f, 0.f, 0.f); }
    __device__ __forceinline__ static C add(C a, C b) {
        float sr, er, si, ei;
        two_sum(a.x, b.x, sr, er);
        two_sum(a.y, b.y, si, ei);
        return make_float4(sr, si, __fadd_rn(er, __fadd_rn(a.z, b.z)), __fadd_rn(ei, __fadd_rn(a.w, b.w)));
    }
    __device__ __forceinline__ static C sub(C a, C b) {
        float sr, er, si, ei;
        two_sum(a.x, -b.x, sr, er);
        two_sum(a.y, -b.y, si, ei);
        return make_float4(sr, si, __fadd_rn(er, __fsub_rn(a.z, b.z)), __fadd_rn(ei, __fsub_rn(a.w, b.w)));
    }
    // (a.x + a.z)(w.x + w.z) - (a.y + a.w)(w.y + w.w), and the imaginary part,
    // with exact hi*hi products (FMA TwoProduct) and first-order lo terms.
    __device__ __forceinline__ static C mul(C a, W w) {
        float p1 = __fmul_rn(a.x, w.x), e1 = __fmaf_rn(a.x, w.x, -p1);
        float p2 = __fmul_rn(a.y, w.y), e2 = __fmaf_rn(a.y, w.y, -p2);
        float sr, er;
        two_sum(p1, -p2, sr, er);
        float lr = __fadd_rn(__fsub_rn(e1, e2), er);
        lr = __fmaf_rn(a.x, w.z, lr);
        lr = __fmaf_rn(a.z, w.x, lr);
        lr = __fmaf_rn(-a.y, w.w, lr);
        lr = __fmaf_rn(-a.w, w.y, lr);
        float p3 = __fmul_rn(a.x, w.y), e3 = __fmaf_rn(a.x, w.y, -p3);
        float p4 = __fmul_rn(a.y, w.x), e4 = __fmaf_rn(a.y, w.x, -p4);
        float si, ei;
        two_sum(p3, p4, si, ei);
        float li = __fadd_rn(__fadd_rn(e3, e4), ei);
        li = __fmaf_rn(a.x, w.w, li);
        li = __fmaf_rn(a.z, w.y, li);
        li = __fmaf_rn(a.y, w.z, li);
        li = __fmaf_rn(a.w, w.x, li);
        return make_float4(sr, si, lr, li);
    }
    // multiply by the real constant k = kh + kl (split at compile time)
    __device__ __forceinline__ static C scale(C a, double k) {
        const float kh = (float)k;
        const float kl = (float)(k - (double)kh);
        float pr = __fmul_rn(a.x, kh), er = __fmaf_rn(a.x, kh, -pr);
        float pi = __fmul_rn(a.y, kh), ei = __fmaf_rn(a.y, kh, -pi);
        er = __fmaf_rn(a.z, kh, __fmaf_rn(a.x, kl, er));
        ei = __fmaf_rn(a.w, kh, __fmaf_rn(a.y, kl, ei));
        return make_float4(pr, pi, er, ei);
    }
    __device__ __forceinline__ static C mul_mi(C a) { return make_float4(a.y, -a.x, a.w, -a.z); }
    __device__ __forceinline__ static C conj(C a) { return make_float4(a.x, -a.y, a.z, -a.w); }
};

// ---------------------------------------------------------- butterflies ----
// Constants of the small DFTs (values of cos / sin at rational multiples of pi).
constexpr double kSqrtHalf = 0.70710678118654752440084436210484903928;
constexpr double kSin60 = 0.86602540378443864676372317075293618347;   // sin(2 pi / 3)
constexpr double kC51 = 0.30901699437494742410229341718281905886;     // cos(2 pi / 5)
constexpr double kC52 = -0.80901699437494742410229341718281905886;    // cos(4 pi / 5)
constexpr double kS51 = 0.95105651629515357211643933337938214340;     // sin(2 pi / 5)
constexpr double kS52 = 0.58778525229247312916870595463907276860;     // sin(4 pi / 5)
constexpr double kC71 = 0.62348980185873353052500488400423981064;     // cos(2 pi / 7)
constexpr double kC72 = -0.22252093395631440428890256449679475947;    // cos(4 pi / 7)
constexpr double kC73 = -0.90096886790241912623610231950744505117;    // cos(6 pi / 7)
constexpr double kS71 = 0.78183148246802980870844452667405775023;     // sin(2 pi / 7)
constexpr double kS72 = 0.97492791218182360701813168299393121153;     // sin(4 pi / 7)
constexpr double kS73 = 0.43388373911755812047576833284835875461;     // sin(6 pi / 7)

template <class A, int R> struct Dft;

template <class A> struct Dft<A, 2> {
    __device__ __forceinline__ static void run(typename A::C* x) {
        auto t = A::sub(x[0], x[1]);
        x[0] = A::add(x[0], x[1]);
        x[1] = t;
    }
};

template <class A> struct Dft<A, 3> {
    __device__ __forceinline__ static void run(typename A::C* x) {
        auto t = A::add(x[1], x[2]);
        auto d = A::mul_mi(A::scale(A::sub(x[1], x[2]), kSin60));   // -i sin60 (x1 - x2)
        auto m = A::sub(x[0], A::scale(t, 0.5));
        x[0] = A::add(x[0], t);
        x[1] = A::add(m, d);
        x[2] = A::sub(m, d);
    }
};

template <class A> struct Dft<A, 4> {
    __device__ __forceinline__ static void run(typename A::C* x) {
        auto a = A::add(x[0], x[2]), b = A::sub(x[0], x[2]);
        auto c = A::add(x[1], x[3]), d = A::mul_mi(A::sub(x[1], x[3]));
        x[0] = A::add(a, c);
        x[2] = A::sub(a, c);
        x[1] = A::add(b, d);
        x[3] = A::sub(b, d);
    }
};

template <class A> struct Dft<A, 5> {
    __device__ __forceinline__ static void run(typename A::C* x) {
        auto t1 = A::add(x[1], x[4]), t2 = A::add(x[2], x[3]);
        auto d1 = A::sub(x[1], x[4]), d2 = A::sub(x[2], x[3]);
        auto a1 = A::add(x[0], A::add(A::scale(t1, kC51), A::scale(t2, kC52)));
        auto a2 = A::add(x[0], A::add(A::scale(t1, kC52), A::scale(t2, kC51)));
        auto b1 = A::mul_mi(A::add(A::scale(d1, kS51), A::scale(d2, kS52)));   // -i (s1 d1 + s2 d2)
        auto b2 = A::mul_mi(A::sub(A::scale(d1, kS52), A::scale(d2, kS51)));   // -i (s2 d1 - s1 d2)
        x[0] = A::add(x[0], A::add(t1, t2));
        x[1] = A::add(a1, b1);
        x[4] = A::sub(a1, b1);
        x[2] = A::add(a2, b2);
        x[3] = A::sub(a2, b2);
    }
};

template <class A> struct Dft<A, 7> {
    __device__ __forceinline__ static void run(typename A::C* x) {
        auto t1 = A::add(x[1], x[6]), t2 = A::add(x[2], x[5]), t3 = A::add(x[3], x[4]);
        auto d1 = A::sub(x[1], x[6]), d2 = A::sub(x[2], x[5]), d3 = A::sub(x[3], x[4]);
        auto a1 = A::add(x[0], A::add(A::scale(t1, kC71), A::add(A::scale(t2, kC72), A::scale(t3, kC73))));
        auto a2 = A::add(x[0], A::add(A::scale(t1, kC72), A::add(A::scale(t2, kC73), A::scale(t3, kC71))));
        auto a3 = A::add(x[0], A::add(A::scale(t1, kC73), A::add(A::scale(t2, kC71), A::scale(t3, kC72))));
        // y_q = a_q - i sum_j sin(2 pi j q / 7) d_j
        auto b1 = A::mul_mi(A::add(A::scale(d1, kS71), A::add(A::scale(d2, kS72), A::scale(d3, kS73))));
        auto b2 = A::mul_mi(A::sub(A::scale(d1, kS72), A::add(A::scale(d2, kS73), A::scale(d3, kS71))));
        auto b3 = A::mul_mi(A::sub(A::scale(d1, kS73), A::sub(A::scale(d2, kS71), A::scale(d3, kS72))));
        x[0] = A::add(x[0], A::add(t1, A::add(t2, t3)));
        x[1] = A::add(a1, b1); x[6] = A::sub(a1, b1);
        x[2] = A::add(a2, b2); x[5] = A::sub(a2, b2);
        x[3] = A::add(a3, b3); x[4] = A::sub(a3, b3);
    }
};

template <class A> struct Dft<A, 8> {
    __device__ __forceinline__ static void run(typename A::C* x) {
        // even / odd radix-4 halves, then y_k = E_k + W8^k O_k, y_{k+4} = E_k - W8^k O_k
        typename A::C e[4] = {x[0], x[2], x[4], x[6]};
        typename A::C o[4] = {x[1], x[3], x[5], x[7]};
        Dft<A, 4>::run(e);
        Dft<A, 4>::run(o);
        // W8 = (1 - i)/sqrt2: (re, im) -> ((re + im), (im - re)) / sqrt2
        auto o1 = A::scale(A::add(o[1], A::mul_mi(o[1])), kSqrtHalf);
        auto o2 = A::mul_mi(o[2]);
        // W8^3 = (-1 - i)/sqrt2 = -i W8
        auto o3 = A::scale(A::sub(A::mul_mi(o[3]), o[3]), kSqrtHalf);
        x[0] = A::add(e[0], o[0]); x[4] = A::sub(e[0], o[0]);
        x[1] = A::add(e[1], o1);   x[5] = A::sub(e[1], o1);
        x[2] = A::add(e[2], o2);   x[6] = A::sub(e[2], o2);
        x[3] = A::add(e[3], o3);   x[7] = A::sub(e[3], o3);
    }
};

}  // namespace ofg
