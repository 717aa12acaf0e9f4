// noalloc.cu -- openfft_exec_c2c_noalloc: the 3-D transform without a plan and
// without any device allocation, for callers that may not allocate device
// memory themselves (for example a host framework whose own allocator owns
// the whole device budget, or a code path that must not pay for the implicit
// device synchronisation of cudaMalloc / cudaFree).
//
// The intermediate array and the twiddle tables live in one file-scope
// __device__ array of fixed size, which every GPU that loads this library
// keeps until the process exits.  Host code only ever passes the array's
// device address, obtained once per device with cudaGetSymbolAddress (the
// host-side symbol itself is not a device address).  Every call shares the
// array and overwrites all of it that it reads, so nothing needs clearing;
// two calls whose kernels overlap on the GPU (different streams, no ordering)
// race on it.
//
// The path is the fused variant with the default arithmetic of the dtype
// (double-float for complex128, FP32 for complex64), the same kernels as
// openfft_exec_c2c, launched on the caller's stream.
#include <cuda_runtime.h>

#include <cstring>
#include <mutex>

#include "../../include/openfft_gb.h"
#include "fft_stage.h"

namespace ofg {
int set_last_error(int status, const char* msg);   // capi.cu
}

using namespace ofg;

namespace {

constexpr size_t kScratchBytes = 16u << 20;                // intermediate array (16 MiB)
constexpr int kNoallocMaxLen = 2048;                       // longest axis
constexpr size_t kTwiddleSlot = (size_t)kNoallocMaxLen * 64;        // largest table (FMT_DF)
constexpr size_t kTwiddleBytes = 3 * kTwiddleSlot;                    // three axis tables

__device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes + kTwiddleBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_scratch_ptr[kMaxDevices] = {};

// Device address of the scratch array on the current device, looked up on the
// first call on that device and cached.  A device reset (cudaDeviceReset, or a
// context torn down and created again) can move the array: the cache entry is
// dropped whenever a call on that device meets a CUDA error, and
// forget_scratch_address() drops it explicitly.
int scratch_address(void** out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return set_last_error(OPENFFT_ERR_CUDA, cudaGetErrorString(e));
    if (dev < 0 || dev >= kMaxDevices) return set_last_error(OPENFFT_ERR_UNSUPPORTED, "device index too large");
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_scratch_ptr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p)
            return set_last_error(OPENFFT_ERR_CUDA, "cudaGetSymbolAddress of the static scratch array failed");
        g_scratch_ptr[dev] = p;
    }
    *out = g_scratch_ptr[dev];
    return OPENFFT_OK;
}

void forget_scratch_address()
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return;
    std::lock_guard<std::mutex> lk(g_mu);
    g_scratch_ptr[dev] = nullptr;
}

int cuda_fail(cudaError_t e)
{
    forget_scratch_address();
    return set_last_error(OPENFFT_ERR_CUDA, cudaGetErrorString(e));
}

bool radix_plan(int n, StageArgs& a)
{
    int m = n, c = 0;
    const int rs[6] = {8, 4, 2, 3, 5, 7};
    for (int r : rs)
        while (m % r == 0) {
            if (c >= kMaxPasses) return false;
            a.radix[c++] = r;
            m /= r;
        }
    a.npass = c;
    return m == 1;
}

// One stage: lines of length n, l = i1 + i2*M1, out(l, k) = i1*S1 + i2*S2 + k*Sk.
int stage(int n, int arith, const void* tw, int sms, int64_t M1, int64_t M2, int64_t S1, int64_t S2,
          int64_t Sk, int group_i2, int contig, int in_fmt, int out_fmt, int conj_in, int conj_out,
          double scale, StageLaunch& L)
{
    std::memset(&L, 0, sizeof(L));
    StageArgs& a = L.args;
    if (!radix_plan(n, a)) return set_last_error(OPENFFT_ERR_UNSUPPORTED_RADIX, "axis length must factor into 2, 3, 5, 7");
    const int E = arith == ARITH_F32 ? 8 : 16;
    int G = arith == ARITH_F32 ? 16 : 8;
    const int64_t Mg = group_i2 ? M2 : M1;
    while (G > 1 && (int64_t)(G / 2) >= Mg) G /= 2;
    while (G > 1 && 2 * (size_t)n * (G + 1) * E > 200 * 1024) G /= 2;
    // the same final checks as the plan path: two tiles of G lines must fit in
    // shared memory, and the grid in a launch
    if (2 * (size_t)n * (G + 1) * E > 200 * 1024) return set_last_error(OPENFFT_ERR_UNSUPPORTED_RADIX, "axis too long for one CTA");
    int lg = 0;
    while ((1 << lg) < G) ++lg;
    a.tw = tw;
    a.M1 = M1; a.M2 = M2; a.S1 = S1; a.S2 = S2; a.Sk = Sk;
    a.ngroups = (Mg + G - 1) / G;
    a.scale = scale;
    a.n = n; a.G = G; a.log2G = lg;
    a.group_i2 = group_i2; a.contig_store = contig;
    a.conj_in = conj_in; a.conj_out = conj_out; a.do_fft = 1;
    a.in_fmt = in_fmt; a.out_fmt = out_fmt;
    L.arith = arith;
    L.grid = a.ngroups * (group_i2 ? M1 : M2);
    L.smem = 2 * (size_t)n * (G + 1) * E;
    L.sms = sms;
    L.family = KERNEL_AUTO;
    if (L.grid > 0x7fffffffLL) return set_last_error(OPENFFT_ERR_UNSUPPORTED, "grid too large");
    return OPENFFT_OK;
}

}  // namespace

extern "C" int openfft_exec_c2c_noalloc(int Na, int Nb, int Nc, int P, int dtype,
                                        const void* in, void* out, int dir, void* stream)
{
    if (Na < 1 || Nb < 1 || Nc < 1 || P < 1) return set_last_error(OPENFFT_ERR_INVALID_ARG, "sizes and P must be >= 1");
    if (!in || !out) return set_last_error(OPENFFT_ERR_INVALID_ARG, "null buffer");
    if (in == out) return set_last_error(OPENFFT_ERR_ALIAS, "in and out must differ (out-of-place only)");
    if (dir != OPENFFT_FORWARD && dir != OPENFFT_BACKWARD) return set_last_error(OPENFFT_ERR_INVALID_ARG, "dir must be -1 or +1");
    if (dtype != OPENFFT_C2C_F64 && dtype != OPENFFT_C2C_F32)
        return set_last_error(OPENFFT_ERR_UNSUPPORTED, "openfft_exec_c2c_noalloc supports OPENFFT_C2C_F64 and OPENFFT_C2C_F32");
    const int64_t a = Na, b = Nb, c = Nc, N = a * b * c;
    if ((int64_t)P > a * b || (int64_t)P > c * a || (int64_t)P > c * b)
        return set_last_error(OPENFFT_ERR_P_TOO_LARGE, "P exceeds N1*N2 of an ordering (Eq. 2 undefined)");
    const int arith = dtype == OPENFFT_C2C_F32 ? ARITH_F32 : ARITH_DF;
    const size_t E = arith == ARITH_F32 ? 8 : 16;
    if (Na > kNoallocMaxLen || Nb > kNoallocMaxLen || Nc > kNoallocMaxLen || (size_t)N * E > kScratchBytes)
        return set_last_error(OPENFFT_ERR_UNSUPPORTED,
                              "openfft_exec_c2c_noalloc: N * element size exceeds its 16 MiB static scratch "
                              "array (or an axis exceeds 2048); use openfft_plan for larger transforms");
    void* base = nullptr;
    int st = scratch_address(&base);
    if (st) return st;
    cudaStream_t s = (cudaStream_t)stream;
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaError_t e = stage_kernels_init(200 * 1024);
    if (e) return cuda_fail(e);

    unsigned char* scratch = static_cast<unsigned char*>(base);
    unsigned char* twb = scratch + kScratchBytes;
    void* tw[3] = {twb, twb + kTwiddleSlot, twb + 2 * kTwiddleSlot};
    const int lens[3] = {Na, Nb, Nc};
    const int twf = arith == ARITH_F32 ? FMT_C64 : FMT_DF;
    for (int ax = 0; ax < 3; ++ax)
        if ((e = launch_twiddles(lens[ax], twf, tw[ax], s))) return cuda_fail(e);

    const int ext = arith == ARITH_F32 ? FMT_C64 : FMT_C128;
    const int mid = arith == ARITH_F32 ? FMT_C64 : FMT_DF;
    StageLaunch L[3];
    if (dir == OPENFFT_FORWARD) {
        if ((st = stage(Nc, arith, tw[2], sms, a * b, 1, 1, 0, a * b, 0, 0, ext, mid, 0, 0, 1.0, L[0]))) return st;
        if ((st = stage(Nb, arith, tw[1], sms, a, c, 1, b * a, a, 0, 0, mid, mid, 0, 0, 1.0, L[1]))) return st;
        if ((st = stage(Na, arith, tw[0], sms, c * b, 1, a, 0, 1, 0, 1, mid, ext, 0, 0, 1.0, L[2]))) return st;
    } else {
        if ((st = stage(Na, arith, tw[0], sms, b, c, 1, a * b, b, 0, 0, ext, mid, 1, 0, 1.0, L[0]))) return st;
        if ((st = stage(Nb, arith, tw[1], sms, a, c, b * c, 1, c, 1, 0, mid, mid, 0, 0, 1.0, L[1]))) return st;
        if ((st = stage(Nc, arith, tw[2], sms, a * b, 1, c, 0, 1, 0, 1, mid, ext, 0, 1, 1.0 / (double)N, L[2]))) return st;
    }
    L[0].args.in = in;      L[0].args.out = scratch;
    L[1].args.in = scratch; L[1].args.out = out;
    L[2].args.in = out;     L[2].args.out = out;
    for (int i = 0; i < 3; ++i)
        if ((e = launch_stage(L[i], s))) return cuda_fail(e);
    return OPENFFT_OK;
}
