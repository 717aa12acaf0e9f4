// batch.h -- host entry points of the batched persistent kernel (batch.cu).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace ofg {

struct BatchPlan;

// `fail` records an OPENFFT_* status and message and returns the status.
int batch_create(int count, const int* dims, const int* P, int dtype, int sms, BatchPlan** out,
                 int (*fail)(int, const char*));
int batch_exec(BatchPlan* b, const void* const* in, void* const* out, int dir, cudaStream_t user,
               int (*fail)(int, const char*));
int batch_status(BatchPlan* b, int (*fail)(int, const char*));
void batch_destroy(BatchPlan* b);
int batch_set_wait_budget(BatchPlan* b, long long cycles);
int batch_inject_stall(BatchPlan* b, int enable);
int64_t batch_items(BatchPlan* b);
int batch_count(BatchPlan* b);
int64_t batch_points(BatchPlan* b, int i);

}  // namespace ofg
