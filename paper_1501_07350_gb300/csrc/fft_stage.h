// fft_stage.h -- host-visible description of one FFT stage launch.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>
#include "checked.h"

namespace ofg {

constexpr int kStageThreads = 256;     // threads per CTA of the stage kernel
constexpr int kMaxLinesPerCta = 32;    // G <= 32
constexpr int kMaxPasses = 16;
constexpr int kMaxLen = 2048;          // longest supported axis (two tiles of one line fit in smem)

// element formats in global memory (real arrays of the real transform: R64 / R32)
enum { FMT_C128 = 0, FMT_C64 = 1, FMT_DF = 2, FMT_R64 = 3, FMT_R32 = 4 };
// arithmetic: FP64, FP32, double-float, and the split-precision tensor-core
// DFT-GEMM forms (complex64 data)
enum { ARITH_F64 = 0, ARITH_F32 = 1, ARITH_DF = 2, ARITH_TC_TF32 = 3, ARITH_TC_BF16 = 4 };

// Lines of a stage are l = i1 + i2 * M1 (i1 < M1, i2 < M2), each contiguous
// of length n at in + l * n.  Output element (l, k) goes to
// out[i1 * S1 + i2 * S2 + k * Sk].  A CTA takes G consecutive values of i1
// (group_i2 = 0) or of i2 (group_i2 = 1), the coordinate whose output stride
// is 1, so a store at fixed k writes G consecutive elements.
struct StageArgs {
    const void* in;
    void* out;
    const void* tw;            // twiddle table of length n (W[e] = exp(-2 pi i e / n))
    const void* aux;           // DFT-GEMM stages: operand image of the DFT matrices
    int64_t M1, M2, S1, S2, Sk;
    int64_t ngroups;           // ceil(M_grouped / G)
    double scale;              // applied at store (1.0 = none)
    int n, G, log2G;
    int group_i2, contig_store;
    int npass;
    int radix[kMaxPasses];
    int conj_in, conj_out, do_fft;
    int in_fmt, out_fmt;
    // elements of the arrays that in and out point into, counted from those
    // pointers (launch_stage fills in M1 M2 n when left 0), and the status
    // word of the bounds checks; read only by the checked build (checked.h)
    int64_t in_elems, out_elems;
    int* chk;
};


struct StageLaunch {
    StageArgs args;
    int arith;
    int64_t grid;              // CTAs of the generic kernel = tiles of G lines
    size_t smem;               // dynamic shared memory of the generic kernel
    int sms;                   // multiprocessors of the device (persistent grids)
    int family;                // KERNEL_*: which stage kernel runs this launch
    int* status;               // device status word (DFT-GEMM stages)
};

// stage kernel families: warp-per-line (power-of-two n), tile (specialised n),
// generic (any n); AUTO takes the first that has an instantiation for (n, G)
enum { KERNEL_AUTO = 0, KERNEL_WARP = 1, KERNEL_TILE = 2, KERNEL_GENERIC = 3 };
// the real stages of the real transform (r2c.cu): the forward stage 1 and the
// inverse's last stage; M1 = number of real lines, G = complex lines per CTA
enum { KERNEL_R2C = 4, KERNEL_C2R = 5 };
cudaError_t launch_real_stage(const StageLaunch& L, cudaStream_t st);

cudaError_t stage_kernels_init(int max_dyn_smem);
// Device allocation of the library's workspaces (capi.cu): cudaMalloc, except
// that a test control (openfft_debug_alloc_fail) can make the n-th call fail
// as if the device were out of memory.
cudaError_t dev_malloc(void** ptr, size_t bytes);
// Resident CTAs per SM of a persistent kernel with `threads` threads and
// `dyn_smem` bytes of dynamic shared memory, from the kernel's own limits
// (shared memory with the whole carveout as shared memory, registers,
// threads); sets the kernel's dynamic shared memory limit and carveout.
cudaError_t persistent_ctas_per_sm(const void* func, int threads, size_t dyn_smem, int* per_sm);
// Launch properties are cached per device (kernel attributes are per device):
// the current device's slot of `slots`, or nullptr beyond kMaxDevices (then
// the caller recomputes on every launch).
constexpr int kMaxDevices = 64;
inline int* device_slot(int (&slots)[kMaxDevices])
{
    int d = 0;
    if (cudaGetDevice(&d) != cudaSuccess || d < 0 || d >= kMaxDevices) return nullptr;
    return &slots[d];
}
// specialised kernels (fft_tile_*.cu); *handled = false when (n, G) has none
cudaError_t launch_tile_f64(const StageLaunch& L, cudaStream_t st, bool* handled);
cudaError_t launch_tile_f32(const StageLaunch& L, cudaStream_t st, bool* handled);
cudaError_t launch_tile_df(const StageLaunch& L, cudaStream_t st, bool* handled);
// the asynchronous-output double-float kernels (fft_tma_256.cu, fft_tma_512.cu)
cudaError_t launch_warp_tma_256(const StageLaunch& L, cudaStream_t st, bool* handled);
cudaError_t launch_warp_tma_512(const StageLaunch& L, cudaStream_t st, bool* handled);
cudaError_t launch_warp_tma_f32(const StageLaunch& L, cudaStream_t st, bool* handled);
cudaError_t launch_warp_mixed_df(const StageLaunch& L, cudaStream_t st, bool* handled);
cudaError_t launch_warp_mixed_f32(const StageLaunch& L, cudaStream_t st, bool* handled);
cudaError_t launch_stage(const StageLaunch& L, cudaStream_t st);
// Twiddle table of length n in format fmt (FMT_C128, FMT_C64 or FMT_DF);
// twiddle_bytes(n, fmt) bytes at out.
cudaError_t launch_twiddles(int n, int fmt, void* out, cudaStream_t st);
inline size_t twiddle_bytes(int n, int fmt) { return (size_t)n * (fmt == FMT_C64 ? 8 : (fmt == FMT_DF ? 32 : 16)); }

// DFT-GEMM stages (dftgemm.cu): n = R S with 2 <= R, S <= 32 (radix[0] = R,
// radix[1] = S); status receives OPENFFT_ERR_TIMEOUT if an MMA wait runs out.
// The stage reads the split operand image of its two DFT matrices from
// args.aux (dftgemm_image_bytes bytes, built once by launch_dftgemm_image from
// the complex64 twiddle table of length n).
bool dftgemm_factor(int n, int tf32, int* R, int* S);
int dftgemm_lines(int n, int R, int S, bool tf32, int Gt);
size_t dftgemm_image_bytes(int n, int R, int S, bool tf32);
cudaError_t launch_dftgemm_image(int n, int R, int S, bool tf32, const void* tw, void* out, cudaStream_t st);
cudaError_t launch_dftgemm(const StageLaunch& L, cudaStream_t st, int* status);

}  // namespace ofg
