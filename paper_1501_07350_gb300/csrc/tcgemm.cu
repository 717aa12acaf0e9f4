// tcgemm.cu -- split-precision GEMM on the tcgen05 tensor cores:
// D = A B^T with A (M x K) and B (N x K) in fp32, each operand split into a
// high part (tf32 or bf16) and the rounded remainder, and
//   D = A_hi B_hi^T + A_hi B_lo^T + A_lo B_hi^T
// accumulated in fp32 in tensor memory (the A_lo B_lo term is below the
// accumulation error).  This is the contraction the DFT-GEMM form of the FFT
// stages is built on (small DFT blocks recast as dense complex GEMMs).
//
// One CTA of 128 threads per 128-row block of A: the threads stage the
// operand tiles into shared memory in the canonical K-major layout (tc.cuh),
// thread 0 issues the MMAs and commits them to an mbarrier, every thread
// waits on it (bounded), and each thread reads its row of D from tensor
// memory.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "../../include/openfft_gb.h"
#include "tc.cuh"

namespace ofg {
int set_last_error(int status, const char* msg);   // capi.cu
}

using namespace ofg;

namespace {

constexpr long long kWaitBudget = 2000000000LL;   // about one second of clock cycles

template <bool TF32>
__device__ __forceinline__ void put_operand(unsigned char* hi, unsigned char* lo, uint32_t off, float x, bool split)
{
    if (TF32) {
        const float h = tc::round_tf32(x);
        *reinterpret_cast<float*>(hi + off) = h;
        *reinterpret_cast<float*>(lo + off) = split ? tc::round_tf32(x - h) : 0.f;
    } else {
        const __nv_bfloat16 h = __float2bfloat16_rn(x);
        *reinterpret_cast<__nv_bfloat16*>(hi + off) = h;
        *reinterpret_cast<__nv_bfloat16*>(lo + off) = __float2bfloat16_rn(split ? x - __bfloat162float(h) : 0.f);
    }
}

template <bool TF32>
__global__ void __launch_bounds__(128) tc_gemm_kernel(const float* __restrict__ A, const float* __restrict__ B,
                                                      float* __restrict__ D, int M, int N, int K, int split,
                                                      int ncols, int* status)
{
    constexpr int ES = TF32 ? 4 : 2;
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ __align__(8) uint64_t mbar;
    __shared__ uint32_t tmem_base;
    const int tid = threadIdx.x, warp = tid >> 5;
    const int KT = K * ES / 16;                         // 16-byte K groups
    // each region is allocated twice its size and zero-filled
    const size_t a_bytes = (size_t)128 * K * ES, b_bytes = (size_t)N * K * ES;
    unsigned char* a_hi = smem;
    unsigned char* a_lo = a_hi + 2 * a_bytes;
    unsigned char* b_hi = a_lo + 2 * a_bytes;
    unsigned char* b_lo = b_hi + 2 * b_bytes;
    const size_t total = 4 * a_bytes + 4 * b_bytes;
    for (size_t i = tid * 16; i < total; i += 128 * 16) *reinterpret_cast<uint4*>(smem + i) = make_uint4(0, 0, 0, 0);
    if (warp == 0) tc::tmem_alloc(&tmem_base, (uint32_t)ncols);
    if (tid == 0) tc::mbar_init(&mbar, 1);
    __syncthreads();
    const int row0 = blockIdx.x * 128;
    for (int idx = tid; idx < 128 * K; idx += 128) {
        const int r = idx / K, k = idx - r * K;
        const float x = row0 + r < M ? A[(size_t)(row0 + r) * K + k] : 0.f;
        put_operand<TF32>(a_hi, a_lo, tc::op_offset(r, k, KT, ES), x, split != 0);
    }
    for (int idx = tid; idx < N * K; idx += 128) {
        const int r = idx / K, k = idx - r * K;
        put_operand<TF32>(b_hi, b_lo, tc::op_offset(r, k, KT, ES), B[(size_t)r * K + k], split != 0);
    }
    tc::fence_smem_to_async();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t d_tmem = tmem_base;
    if (tid == 0) {
        const uint32_t id = tc::idesc(TF32 ? tc::kTypeTF32 : tc::kTypeBF16, 128, N);
        const unsigned char* pa[3] = {a_hi, a_hi, a_lo};
        const unsigned char* pb[3] = {b_hi, b_lo, b_hi};
        const int nprod = split ? 3 : 1;
        uint32_t acc = 0;
        for (int pr = 0; pr < nprod; ++pr)
            for (int kc = 0; kc < KT / 2; ++kc) {       // 32 bytes of K per MMA
                const uint64_t ad = tc::smem_desc(tc::smem_u32(pa[pr]) + kc * 256, 128, KT * 128);
                const uint64_t bd = tc::smem_desc(tc::smem_u32(pb[pr]) + kc * 256, 128, KT * 128);
                tc::mma<TF32>(d_tmem, ad, bd, id, acc);
                acc = 1;
            }
        tc::commit(&mbar);
    }
    const bool ok = tc::mbar_wait(&mbar, 0, kWaitBudget);
    if (!ok && tid == 0) atomicExch(status, OPENFFT_ERR_TIMEOUT);
    tc::fence_after_sync();
    if (ok) {
        const int row = row0 + tid;
        for (int c0 = 0; c0 < N; c0 += 16) {
            float v[16];
            tc::ld16(d_tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, v);
            if (row < M)
                for (int i = 0; i < 16; ++i) D[(size_t)row * N + c0 + i] = v[i];
        }
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(d_tmem, (uint32_t)ncols);
}

}  // namespace

extern "C" int openfft_tc_gemm(int tf32, int split, int M, int N, int K, const float* A, const float* B, float* D)
{
    const int ES = tf32 ? 4 : 2, kstep = 32 / ES;
    if (!A || !B || !D || M < 1 || N < 16 || N > 64 || N % 16 || K < kstep || K > 64 || K % kstep)
        return set_last_error(OPENFFT_ERR_INVALID_ARG, "openfft_tc_gemm: N in {16,32,48,64}, K a multiple of 8 (tf32) / 16 (bf16) up to 64");
    float *dA = nullptr, *dB = nullptr, *dD = nullptr;
    int* dst = nullptr;
    const int mblocks = (M + 127) / 128;
    cudaError_t e = cudaMalloc(&dA, sizeof(float) * (size_t)M * K);
    if (!e) e = cudaMalloc(&dB, sizeof(float) * (size_t)N * K);
    if (!e) e = cudaMalloc(&dD, sizeof(float) * (size_t)M * N);
    if (!e) e = cudaMalloc(&dst, sizeof(int));
    if (!e) e = cudaMemcpy(dA, A, sizeof(float) * (size_t)M * K, cudaMemcpyHostToDevice);
    if (!e) e = cudaMemcpy(dB, B, sizeof(float) * (size_t)N * K, cudaMemcpyHostToDevice);
    if (!e) e = cudaMemset(dst, 0, sizeof(int));
    const size_t smem = 4 * (size_t)128 * K * ES + 4 * (size_t)N * K * ES;
    const int ncols = N <= 32 ? 32 : 64;
    if (!e) {
        if (tf32) {
            e = cudaFuncSetAttribute(tc_gemm_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            if (!e) tc_gemm_kernel<true><<<mblocks, 128, smem>>>(dA, dB, dD, M, N, K, split, ncols, dst);
        } else {
            e = cudaFuncSetAttribute(tc_gemm_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            if (!e) tc_gemm_kernel<false><<<mblocks, 128, smem>>>(dA, dB, dD, M, N, K, split, ncols, dst);
        }
        if (!e) e = cudaGetLastError();
        if (!e) e = cudaDeviceSynchronize();
    }
    int status = 0;
    if (!e) e = cudaMemcpy(&status, dst, sizeof(int), cudaMemcpyDeviceToHost);
    if (!e) e = cudaMemcpy(D, dD, sizeof(float) * (size_t)M * N, cudaMemcpyDeviceToHost);
    cudaFree(dA); cudaFree(dB); cudaFree(dD); cudaFree(dst);
    if (e) return set_last_error(OPENFFT_ERR_CUDA, cudaGetErrorString(e));
    if (status) return set_last_error(status, "tensor-core MMA completion wait ran out");
    return OPENFFT_OK;
}
