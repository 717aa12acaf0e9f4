// dftgemm.h -- host controls of the DFT-GEMM stages (dftgemm.cu) beyond the
// stage launch itself.
#pragma once
#include <cuda_runtime.h>

namespace ofg {

// Test controls, process-wide: what = 1 sets the MMA completion-wait budget
// to `value` clock cycles (value <= 0: the default, about one second);
// what = 2 with value != 0 leaves every block's MMAs unissued and
// uncommitted, so that the bounded waits run out (value = 0 undoes it).
cudaError_t dftgemm_test_controls(int what, long long value);

}  // namespace ofg
