// redistribute.h -- host entry points of the explicit transpose kernels (V0/V1).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>
#include <vector>
#include "decomp.h"

namespace ofg {

// Count matrix C[r*P+s], pack bases sbase[r*P+s], unpack bases rbase[s*P+r]
// and the exchange chunk list (src offset, dst offset, length) of transpose t.
void build_transpose_tables(const Transpose& t, std::vector<int64_t>& C, std::vector<int64_t>& sbase,
                            std::vector<int64_t>& rbase, std::vector<int64_t>& chunks, int64_t chunk_len);

cudaError_t launch_pack(const Transpose& t, int elem_bytes, const void* src, void* send,
                        const int64_t* sbase, int64_t N, int sms, cudaStream_t st);
cudaError_t launch_exchange(int elem_bytes, const int64_t* chunks, int64_t nchunks,
                            const void* send, void* recv, int sms, cudaStream_t st);
cudaError_t launch_unpack(const Transpose& t, int elem_bytes, const void* buf, void* dst,
                          const int64_t* base, int from_send, int64_t N, int sms, cudaStream_t st);

}  // namespace ofg
