// redistribute.h -- host entry points of the explicit transpose kernels (V0/V1).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>
#include <vector>
#include "decomp.h"
#include "checked.h"

namespace ofg {

// Count matrix C[r*P+s], pack bases sbase[r*P+s], unpack bases rbase[s*P+r]
// and the exchange chunk list (src offset, dst offset, length) of transpose t.
// sdispl_out[r*P+s] / rdispl_out[s*P+r]: send / receive displacement of segment (r, s).
void build_transpose_tables(const Transpose& t, std::vector<int64_t>& C, std::vector<int64_t>& sbase,
                            std::vector<int64_t>& rbase, std::vector<int64_t>& chunks, int64_t chunk_len,
                            std::vector<int64_t>* sdispl_out = nullptr, std::vector<int64_t>* rdispl_out = nullptr);

// schedules of the stepped exchanges
enum { SCHED_PER_SENDER = 0, SCHED_BLOCKED = 1, SCHED_SHIFTED = 2 };
constexpr int64_t kBlockSize = 32;   // B_SIZE of the paper's blocked methods (Sec. 3.2.1)
int64_t num_steps(int sched, int64_t P, int64_t B);
int64_t pairs_per_step(int sched, int64_t P, int64_t B);
cudaError_t launch_segment_exchange(int sched, int64_t P, int64_t B, int64_t step, int elem_bytes,
                                    const int64_t* C, const int64_t* sdispl, const int64_t* rdispl,
                                    const void* send, void* recv, cudaStream_t st, const Bounds& b = Bounds());
cudaError_t launch_segment_unpack(const Transpose& t, int sched, int64_t B, int64_t step, int elem_bytes,
                                  const void* send, void* dst, const int64_t* sbase, cudaStream_t st, const Bounds& b = Bounds());

cudaError_t launch_pack(const Transpose& t, int elem_bytes, const void* src, void* send,
                        const int64_t* sbase, int64_t N, int sms, cudaStream_t st, const Bounds& b = Bounds());
cudaError_t launch_exchange(int elem_bytes, const int64_t* chunks, int64_t nchunks,
                            const void* send, void* recv, int sms, cudaStream_t st, const Bounds& b = Bounds());
cudaError_t launch_unpack(const Transpose& t, int elem_bytes, const void* buf, void* dst,
                          const int64_t* base, int from_send, int64_t N, int sms, cudaStream_t st, const Bounds& b = Bounds());

}  // namespace ofg
