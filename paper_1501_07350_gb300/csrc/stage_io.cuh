// stage_io.cuh -- element loads/stores of the stage kernels: global formats
// (complex128, complex64, double-float pairs), the conversions between
// double and double-float, and asynchronous global->shared copies.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "arith.cuh"
#include "arith_pair.cuh"
#include "fft_stage.h"

namespace ofg {

// ------------------------------------------------ element load / store ----

template <class A> struct Io;

template <> struct Io<ArF64> {
    static constexpr bool kConverts = false;
    static constexpr int kExtBytes = 16, kMidBytes = 16;
    __device__ __forceinline__ static void store_ext(void* p, double2 v) { *reinterpret_cast<double2*>(p) = v; }
    __device__ __forceinline__ static void store_mid(void* p, double2 v) { *reinterpret_cast<double2*>(p) = v; }
    __device__ __forceinline__ static double2 from_c128(double2 v) { return v; }
    __device__ __forceinline__ static double2 load(const void* p, int, int64_t i) {
        return __ldg(reinterpret_cast<const double2*>(p) + i);
    }
    __device__ __forceinline__ static void store(void* p, int, int64_t i, double2 v) {
        reinterpret_cast<double2*>(p)[i] = v;
    }
};

template <> struct Io<ArF32> {
    static constexpr bool kConverts = false;
    static constexpr int kExtBytes = 8, kMidBytes = 8;
    __device__ __forceinline__ static void store_ext(void* p, float2 v) { *reinterpret_cast<float2*>(p) = v; }
    __device__ __forceinline__ static void store_mid(void* p, float2 v) { *reinterpret_cast<float2*>(p) = v; }
    __device__ __forceinline__ static float2 from_c128(double2 v) { return make_float2((float)v.x, (float)v.y); }
    __device__ __forceinline__ static float2 load(const void* p, int, int64_t i) {
        return __ldg(reinterpret_cast<const float2*>(p) + i);
    }
    __device__ __forceinline__ static void store(void* p, int, int64_t i, float2 v) {
        reinterpret_cast<float2*>(p)[i] = v;
    }
};

// Double-float: external arrays hold complex128; intermediate arrays hold the
// (hi, lo) pairs themselves (FMT_DF), so conversions happen once on entry and
// once on exit of the 3-D transform.  Both conversions use integer and FP32
// instructions only (the FP64 and conversion units are slow on this part).

// d -> (h, r): h keeps the sign, exponent and leading 24 significant bits of
// d (truncated), r the next 23 bits, so |d - h - r| <= 2^-47 |d|.
// |d| < 2^-126 is flushed to zero; r is dropped below 2^-103.
__device__ __forceinline__ float2 split_f64(double d)
{
    const unsigned long long bits = (unsigned long long)__double_as_longlong(d);
    const uint32_t hw = (uint32_t)(bits >> 32), lw = (uint32_t)bits;
    if ((hw & 0x7FFFFFFFu) - (920u << 20) < (231u << 20)) {
        // 2^-103 <= |d| < 2^128, exponent e in [920, 1150]: the same h and r as
        // below in fewer instructions.  (hw:lw) << 3 puts the low 9 exponent
        // bits and the top 23 fraction bits in one word; subtracting 896 << 23
        // (mod 2^32) rebiases the exponent (e - 896 < 256 leaves bit 31 clear).
        const uint32_t hb = (__funnelshift_l(lw, hw, 3) - 0xC0000000u) | (hw & 0x80000000u);
        const uint32_t pw = (hb & 0xFF800000u) - (23u << 23);          // sign, exponent e - 919
        const float F = __uint_as_float(pw | ((lw >> 6) & 0x7FFFFFu));
        return make_float2(__uint_as_float(hb), __fsub_rn(F, __uint_as_float(pw)));
    }
    const uint32_t sign = hw & 0x80000000u;
    const int e = (int)((hw >> 20) & 0x7FFu);              // biased double exponent
    const int fe = e - 1023 + 127;                          // biased float exponent of h
    if (fe <= 0) return make_float2(__uint_as_float(sign), 0.f);
    if (fe >= 255) {                                        // too large for a float, inf, nan
        const bool nan = e == 0x7FF && (((hw & 0xFFFFFu) | lw) != 0);
        return make_float2(__uint_as_float(sign | 0x7F800000u | (nan ? 0x400000u : 0u)), 0.f);
    }
    const float h = __uint_as_float(sign | ((uint32_t)fe << 23) | ((hw & 0xFFFFFu) << 3) | (lw >> 29));
    // the low 29 fraction bits are worth (lw & 0x1FFFFFFF) * 2^(e-1075); their
    // top 23 bits form the fraction of F = (1 + m 2^-23) 2^(xe-127), and
    // F - 2^(xe-127) (exact) is their value.
    const int xe = e - 919;
    float r = 0.f;
    if (xe >= 1) {
        const float F = __uint_as_float(sign | ((uint32_t)xe << 23) | ((lw & 0x1FFFFFFFu) >> 6));
        const float Pw = __uint_as_float(sign | ((uint32_t)xe << 23));
        r = __fsub_rn(F, Pw);
    }
    return make_float2(h, r);
}

// Exact float -> double by bit manipulation (no conversion unit): the sign
// stays, the exponent is rebiased (+896) and the 23 fraction bits become the
// top of the 52.  Zero and subnormal floats give a signed zero (a subnormal
// lo part is below 2^-126, far under the hi part's last place); infinities and
// NaNs keep their class.
__device__ __forceinline__ double f2d_bits(float f)
{
    const uint32_t b = __float_as_uint(f);
    const uint32_t e = (b >> 23) & 0xFFu;
    if (e - 1u < 254u)                                      // normal float
        return __hiloint2double((int)((b & 0x80000000u) | (((b & 0x7FFFFFFFu) >> 3) + (896u << 20))), (int)(b << 29));
    const uint32_t sign = b & 0x80000000u;
    if (e == 0) return __hiloint2double((int)sign, 0);
    return __hiloint2double((int)(sign | 0x7FF00000u | ((b & 0x7FFFFFu) ? 0x80000u : 0u)), 0);
}

// (h, l) -> the double nearest h + l: both parts are exact as doubles, and one
// FP64 addition (on the otherwise idle FP64 pipe) rounds their sum once.
__device__ __forceinline__ double join_f64(float h, float l)
{
    return __dadd_rn(f2d_bits(h), f2d_bits(l));
}

__device__ __forceinline__ float4 df_from_double2(double2 v) {
    const float2 r = split_f64(v.x), i = split_f64(v.y);
    return make_float4(r.x, i.x, r.y, i.y);
}
__device__ __forceinline__ double2 df_to_double2(float4 v) {
    return make_double2(join_f64(v.x, v.z), join_f64(v.y, v.w));
}

template <> struct Io<ArDF> {
    static constexpr bool kConverts = true;
    static constexpr int kExtBytes = 16, kMidBytes = 16;
    __device__ __forceinline__ static void store_ext(void* p, float4 v) { *reinterpret_cast<double2*>(p) = df_to_double2(v); }
    __device__ __forceinline__ static void store_mid(void* p, float4 v) { *reinterpret_cast<float4*>(p) = v; }
    __device__ __forceinline__ static float4 from_c128(double2 v) { return df_from_double2(v); }
    __device__ __forceinline__ static float4 load(const void* p, int fmt, int64_t i) {
        if (fmt == FMT_DF) return __ldg(reinterpret_cast<const float4*>(p) + i);
        return df_from_double2(__ldg(reinterpret_cast<const double2*>(p) + i));
    }
    __device__ __forceinline__ static void store(void* p, int fmt, int64_t i, float4 v) {
        if (fmt == FMT_DF) reinterpret_cast<float4*>(p)[i] = v;
        else reinterpret_cast<double2*>(p)[i] = df_to_double2(v);
    }
};

// The paired double-float policy has ArDF's bytes in ArDF's order.
template <> struct Io<ArDP> {
    static constexpr bool kConverts = true;
    static constexpr int kExtBytes = 16, kMidBytes = 16;
    __device__ __forceinline__ static void store_ext(void* p, ulonglong2 v) { *reinterpret_cast<double2*>(p) = df_to_double2(ArDP::to_float4(v)); }
    __device__ __forceinline__ static void store_mid(void* p, ulonglong2 v) { *reinterpret_cast<ulonglong2*>(p) = v; }
    __device__ __forceinline__ static ulonglong2 from_c128(double2 v) { return ArDP::from_float4(df_from_double2(v)); }
    __device__ __forceinline__ static ulonglong2 load(const void* p, int fmt, int64_t i) {
        return ArDP::from_float4(Io<ArDF>::load(p, fmt, i));
    }
    __device__ __forceinline__ static void store(void* p, int fmt, int64_t i, ulonglong2 v) {
        Io<ArDF>::store(p, fmt, i, ArDP::to_float4(v));
    }
};

// -------------------------------------------------- asynchronous copies ----

// global -> shared copy of one element that bypasses registers (cp.async).
template <int BYTES>
__device__ __forceinline__ void cp_async(void* smem_dst, const void* gmem_src)
{
    const uint32_t d = (uint32_t)__cvta_generic_to_shared(smem_dst);
    if (BYTES == 16)
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(gmem_src) : "memory");
    else
        asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(d), "l"(gmem_src) : "memory");
}
__device__ __forceinline__ void cp_async_commit()
{
    asm volatile("cp.async.commit_group;\n" ::: "memory");
}
// wait for all of this thread's outstanding copies
__device__ __forceinline__ void cp_async_wait_all()
{
    asm volatile("cp.async.commit_group;\ncp.async.wait_all;\n" ::: "memory");
}

}  // namespace ofg
