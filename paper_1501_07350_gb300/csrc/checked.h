// checked.h -- bounds checks of the checked build (-DOPENFFT_CHECKED).
//
// In the checked build every global element index of the C2C stage kernels,
// the explicit transpose kernels and the multi-device pack / unpack kernels
// is tested against the length of the array it addresses before the access.
// An index outside [0, lim) is not accessed: the thread skips that element,
// and the first such index found stores OPENFFT_ERR_BOUNDS (9) in a device
// status word, which the host reads after the stream has drained (the plan's
// status word at openfft_sync, or the word of openfft_debug_bounds_status
// for calls whose plan has none).  Nothing traps: the context stays usable.
// In the normal build in_bounds() is the constant true and the checks vanish.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace ofg {

constexpr int kErrBounds = 9;        // OPENFFT_ERR_BOUNDS of the C ABI

struct Bounds {
    int* chk = nullptr;              // status word (nullptr: the fallback word)
    int64_t lim = INT64_MAX;         // elements of the array addressed
};

#ifdef OPENFFT_CHECKED
__device__ __forceinline__ bool in_bounds(int* chk, int64_t idx, int64_t lim)
{
    if (idx >= 0 && idx < lim) return true;
    if (chk) atomicCAS(chk, 0, kErrBounds);
    return false;
}
#else
__device__ __forceinline__ bool in_bounds(int*, int64_t, int64_t) { return true; }
#endif

__device__ __forceinline__ bool in_bounds(const Bounds& b, int64_t idx) { return in_bounds(b.chk, idx, b.lim); }

// Device status word for launches whose plan has none (fft_stage.cu); its
// address on the current device, or nullptr outside the checked build.
int* fallback_status_word();

}  // namespace ofg
