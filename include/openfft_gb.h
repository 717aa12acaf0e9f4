/*
 * openfft_gb.h -- C ABI of a GB300 (sm_103a) 3-D complex-to-complex FFT under
 * the communication-optimal decomposition of OpenFFT (Duy & Ozaki,
 * "Performance Tuning of a Parallel 3-D FFT Package OpenFFT").
 *
 * Model.  The user's array A has shape [Na][Nb][Nc], c fastest ("abc" order,
 * Eq. 1 with N1 = Na, N2 = Nb, N3 = Nc).  P logical ranks share it: rank r
 * owns the 1-D index range [x^s_r, x^e_r] of Eqs. 2-4 (slabs if P <= leading
 * dimension, pencils up to the product of the first two, Eqs. 8-9).  The
 * transform runs the paper's order (Sec. 2): 1-D FFTs along c in abc, a
 * transpose to cab ([Nc][Na][Nb]), 1-D FFTs along b, a transpose to cba
 * ([Nc][Nb][Na]), 1-D FFTs along a.  The forward result is left in cba order
 * and rank r's output box is [x^s_r, x^e_r] of Eqs. 2-4 applied to
 * (N1,N2,N3) = (Nc,Nb,Na).  All ranks live in one GPU's memory: the
 * concatenation of the ranks' boxes is the global array of that order, so a
 * transpose is a device-local permutation.
 *
 * Conventions.  FORWARD computes X[ka,kb,kc] = sum A[a,b,c] exp(-2 pi i
 * (a ka/Na + b kb/Nb + c kc/Nc)), unnormalised, and writes it at cba index
 * (kc*Nb + kb)*Na + ka.  BACKWARD takes a cba-ordered spectrum, uses
 * exp(+2 pi i ...), divides by N = Na*Nb*Nc, and writes abc order, so
 * BACKWARD(FORWARD(A)) = A.
 *
 * Memory.  `in` / `out` of openfft_exec_c2c are DEVICE pointers owned by the
 * caller, N elements each of the plan's element type (complex128 = two
 * doubles for OPENFFT_C2C_F64, complex64 = two floats otherwise), 16-byte
 * aligned.  Out of place only; `in` is not modified.  The plan owns all
 * workspace, allocated once by openfft_plan (the paper moves buffer
 * allocation out of the execution phase, Sec. 3.2.4); openfft_exec_c2c
 * allocates nothing.  The host-buffer calls allocate their two staging arrays
 * (and streams) on a plan's first host-buffer call.
 *
 * Errors.  Functions returning int return an OPENFFT_* status (0 = OK).
 * openfft_plan returns NULL on error.  openfft_last_error() gives a message
 * for the calling thread's last failure.  Exec is asynchronous on the plan's
 * stream; device-side failures are reported by openfft_sync().  A plan is not
 * safe for concurrent use from several threads.
 */
#ifndef OPENFFT_GB_H
#define OPENFFT_GB_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct openfft_plan_s* openfft_plan_t;

/* Element type and arithmetic of a plan. */
enum {
    OPENFFT_C2C_F64 = 0,        /* complex128 in/out, FP64-accurate (<= 1e-12 rel. L2)   */
    OPENFFT_C2C_F32 = 1,        /* complex64 in/out, FP32 arithmetic                     */
    OPENFFT_C2C_SPLIT_BF16 = 2, /* complex64 in/out, tensor-core DFT-GEMM, bf16 hi/lo (<= 1e-4) */
    OPENFFT_C2C_SPLIT_TF32 = 3, /* complex64 in/out, tensor-core DFT-GEMM, tf32 hi/lo (<= 1e-5) */
    OPENFFT_R2C_F64 = 4,        /* real transform: double in, complex128 half spectrum out (FP64-accurate) */
    OPENFFT_R2C_F32 = 5         /* real transform: float in, complex64 half spectrum out (FP32) */
};

/* Sign of the exponent. */
enum { OPENFFT_FORWARD = -1, OPENFFT_BACKWARD = 1 };

/* Status codes. */
enum {
    OPENFFT_OK = 0,
    OPENFFT_ERR_INVALID_ARG = 1,       /* a size < 1, P < 1, bad dir/dtype/null pointer     */
    OPENFFT_ERR_P_TOO_LARGE = 2,       /* P > N1*N2 for some ordering: Eq. 2 is undefined  */
    OPENFFT_ERR_UNSUPPORTED_RADIX = 3, /* an axis length with a prime factor other than 2,3,5,7 or above 2048 */
    OPENFFT_ERR_CUDA = 4,              /* a CUDA runtime call failed                        */
    OPENFFT_ERR_NOMEM = 5,             /* device allocation failed (plan time, or the first host-buffer call) */
    OPENFFT_ERR_TIMEOUT = 6,           /* a bounded device wait ran out (batched kernel)    */
    OPENFFT_ERR_ALIAS = 7,             /* in == out                                         */
    OPENFFT_ERR_UNSUPPORTED = 8,       /* the request is valid but this build does not do it */
    OPENFFT_ERR_BOUNDS = 9             /* checked build only: a kernel met a global index outside its array */
};

/* Transpose variants: the paper's six communication methods (Sec. 3.2.1),
 * recast for ranks that share one memory, and the fused form.
 *   FUSED (V2):  the transpose is folded into the store of each FFT stage: one
 *                HBM read and one write per stage (the default).
 * The explicit methods store each stage's box unchanged, pack per-destination
 * send segments (ascending source index, step (4) of Sec. 3.1.1), move them
 * (step (5)) and unpack them into the next ordering (step (6)):
 *   PACK_EXCHANGE_UNPACK (Alltoallv): one exchange over the count matrix, then
 *                unpack;
 *   ISEND_WAITALL:       every sender's segments moved in its own launch (P
 *                launches), then unpack;
 *   ISEND_WAITALL_BLOCK: ranks in groups of B_SIZE = 32; ceil(P/32) steps, step
 *                k moving the pairs (r, s) with floor(s/32) = (floor(r/32) + k)
 *                mod ceil(P/32); then unpack;
 *   PACK_UNPACK (Isend_Waitsome): every receiver unpacks straight from the
 *                senders' segments (unpack on arrival);
 *   ISEND_WAITSOME_BLOCK: the blocked steps, each unpacking its segments on
 *                arrival;
 *   SENDRECV:    P shifted steps, step i moving the pairs (r, (r + i) mod P),
 *                then unpack. */
enum {
    OPENFFT_VARIANT_PACK_EXCHANGE_UNPACK = 0,
    OPENFFT_VARIANT_PACK_UNPACK = 1,
    OPENFFT_VARIANT_FUSED = 2,
    OPENFFT_VARIANT_ISEND_WAITALL = 3,
    OPENFFT_VARIANT_ISEND_WAITALL_BLOCK = 4,
    OPENFFT_VARIANT_ISEND_WAITSOME_BLOCK = 5,
    OPENFFT_VARIANT_SENDRECV = 6
};

/* Arithmetic used for OPENFFT_C2C_F64.
 *   NATIVE: IEEE double on the FP64 units.
 *   DOUBLE_FLOAT: each double is carried as an unevaluated sum of two floats
 *   and the butterflies use error-free transformations on the FP32 units
 *   (about 48 significant bits; finite inputs with |x| < 2^90 and outputs
 *   below 2^126).  Both meet the FP64 bound of 1e-12 relative L2.  The float
 *   exponent range also bounds small values: on entry a component below
 *   2^-103 in magnitude keeps only its leading 24 bits and one below 2^-126
 *   becomes zero, so data whose magnitudes all lie that low should be scaled
 *   first or transformed with NATIVE. */
enum { OPENFFT_ARITH_NATIVE = 0, OPENFFT_ARITH_DOUBLE_FLOAT = 1 };
/* Arithmetic of the split-precision plans (OPENFFT_C2C_SPLIT_TF32 / _BF16):
 * every axis n = R S (2 <= R, S <= 32) is transformed by two tensor-core
 * GEMM passes with the R- and S-point DFT matrices, operands split into a
 * high part and the rounded remainder, fp32 accumulation (stated bounds:
 * 1e-5 relative L2 for tf32, 1e-4 for bf16). */
enum { OPENFFT_ARITH_TC_TF32 = 2, OPENFFT_ARITH_TC_BF16 = 3 };

/* Tuning modes of openfft_set_tuning (Sec. 3.2.3: auto-tuning on, off = the
 * default method, or a user-selected method). */
enum {
    OPENFFT_TUNE_DEFAULT = 0,    /* fixed default variant                         */
    OPENFFT_TUNE_EXHAUSTIVE = 1, /* time every candidate twice, keep the fastest   */
    OPENFFT_TUNE_LEARNED = 2,    /* the installed cost model's fastest candidate (no model: DEFAULT) */
    OPENFFT_TUNE_USER = 3,       /* candidate index given by the caller            */
    OPENFFT_TUNE_SAVED = 4       /* the recorded choice for this problem (openfft_tuning_*), else EXHAUSTIVE */
};

/* ------------------------------------------------------------ plans ---- */

/* Plan a 3-D C2C transform of [Na][Nb][Nc] over P logical ranks (Sec. 3.1.1,
 * initialisation phase): validates the sizes, computes the boxes of the three
 * orderings (Eqs. 2-9) and the radix plans, allocates the workspace (two
 * scratch arrays of N elements, twiddle tables, transpose tables) and builds
 * the twiddle tables on the device.  Uses the current CUDA device.
 * Returns NULL on error (see openfft_last_error / openfft_last_status). */
openfft_plan_t openfft_plan(int Na, int Nb, int Nc, int P, int dtype);

/* Execute one transform (execution phase, repeatable).  in/out: device
 * pointers as described above; dir: OPENFFT_FORWARD or OPENFFT_BACKWARD.
 * Asynchronous on the plan's stream.  Returns OPENFFT_OK, INVALID_ARG,
 * ALIAS or CUDA. */
int openfft_exec_c2c(openfft_plan_t plan, const void* in, void* out, int dir);

/* Real transforms (plans of dtype OPENFFT_R2C_F64 / OPENFFT_R2C_F32).  The
 * paper names real transforms as future work; they are built here on the same
 * decomposition:
 *   - input of openfft_exec_r2c: the real abc array [Na][Nb][Nc] (double or
 *     float), rank r's box at openfft_box(plan, 0, r, ...) in real elements;
 *   - output: the half spectrum X[ka][kb][kc], kc <= Nc/2, in cba order
 *     [Nch][Nb][Na] with Nch = Nc/2 + 1 (complex128 or complex64); the
 *     complex arrays are decomposed by Eqs. 2-9 with Nc replaced by Nch, so
 *     rank r's output box is openfft_box(plan, 1, r, ...) in that array;
 *   - openfft_exec_c2r takes such a half spectrum and writes the real abc
 *     array: the real part of the inverse DFT of the spectrum extended by
 *     Hermitian symmetry along c, divided by N = Na*Nb*Nc (only the real
 *     parts of kc = 0 and, for even Nc, kc = Nc/2 count).
 * P must satisfy P <= Na*Nb, P <= Nch*Na and P <= Nch*Nb (P_TOO_LARGE
 * otherwise).  Device pointers, 16-byte aligned, in != out (ALIAS); the
 * fused variant only.  openfft_exec_c2c on a real plan, or these on a
 * complex plan, returns INVALID_ARG.  Asynchronous on the plan's stream. */
int openfft_exec_r2c(openfft_plan_t plan, const void* in, void* out);
int openfft_exec_c2r(openfft_plan_t plan, const void* in, void* out);

/* Same transform with HOST buffers: copies `host_in` to plan-owned device
 * memory, executes, copies the result to `host_out` and waits (complex
 * plans only; N elements of the plan's external type each way).  The copies
 * run on the plan's upload and download streams (openfft_set_copy_streams)
 * in ranges of lines, so that the first stage starts on each range of the
 * input as soon as it has arrived and each range of the last stage's output
 * is copied back as soon as it is written (the host link, not the transform,
 * bounds this call).  The result is bit for bit that of openfft_exec_c2c.
 * Page-locked host memory gives the fastest copies; `host_in` may equal
 * `host_out`.  The plan allocates its two device staging arrays, its copy
 * streams and their events on the first call.
 * While the phase timer is on (openfft_set_timing) the copies bracket the
 * whole transform instead. */
int openfft_exec_c2c_host(openfft_plan_t plan, const void* host_in, void* host_out, int dir);

/* openfft_exec_c2c_host without the final wait: returns once the copies and
 * launches are enqueued.  `host_in` must stay unchanged and `host_out`
 * unread until openfft_sync(plan) returns (it waits for the plan's copy
 * stream and its stream).  Successive calls on one plan run in order.  Calls
 * on different plans may overlap their copies: the host-to-device copy of one
 * plan can run beside the device-to-host copy of another.  Same results, bit
 * for bit, as the synchronous call.  Call openfft_sync before switching the
 * plan to another stream (openfft_set_stream), since openfft_sync waits on the
 * current one. */
int openfft_exec_c2c_host_async(openfft_plan_t plan, const void* host_in, void* host_out, int dir);

/* Streams of the host-buffer calls' copies: uploads on `h2d`, downloads on
 * `d2h` (each a cudaStream_t).  Both NULL (the default) = two streams the
 * plan creates and owns.  Plans given the same two streams queue their
 * transfers in call order across plans, so one plan's upload runs beside
 * another's download instead of sharing the link with the other uploads.
 * The caller keeps the streams alive until the plan is destroyed or given
 * other streams: openfft_destroy and this call wait for the copies queued on
 * them.  INVALID_ARG if exactly one of the two is NULL. */
int openfft_set_copy_streams(openfft_plan_t plan, void* h2d, void* d2h);

/* Number of line ranges of openfft_exec_c2c_host: 1 (no overlap) to 32;
 * 0 (the default) takes one per 8 MiB of the array, 1 to 16.  INVALID_ARG
 * outside 0..32. */
int openfft_set_host_chunks(openfft_plan_t plan, int chunks);

/* Finalisation phase: frees everything the plan owns.  NULL-safe. */
void openfft_destroy(openfft_plan_t plan);

/* Waits for the plan's stream and its copy streams, and reports device-side
 * errors. */
int openfft_sync(openfft_plan_t plan);

/* Use `stream` (a cudaStream_t; NULL = legacy default stream) for exec. */
int openfft_set_stream(openfft_plan_t plan, void* stream);

/* ------------------------------------------------ queries / controls --- */

/* Message for the calling thread's last failure ("" if none). */
const char* openfft_last_error(void);
/* Status of the calling thread's last failure (OPENFFT_OK if none). */
int openfft_last_status(void);

/* Box of `rank` in the input (which = 0: abc ordering) or output
 * (which = 1: cba ordering) decomposition of the FORWARD transform:
 * start/end 3-D coordinates (Eqs. 5-7, in the ordering's own dimension
 * order), 1-D offset x^s and element count x^e - x^s + 1 (Eqs. 3-4).
 * Any pointer may be NULL. */
int openfft_box(openfft_plan_t plan, int which, int rank,
                int64_t start[3], int64_t end[3], int64_t* offset, int64_t* count);

/* P x P count matrix of one transpose, row = sending rank, column =
 * receiving rank (the volumes of Sec. 4.1): exchange 1 = abc->cab,
 * 2 = cab->cba, -2 = cba->cab, -1 = cab->abc.  PxP: host array of P*P. */
int openfft_counts(openfft_plan_t plan, int exchange, int64_t* PxP);

/* Host-only forms of the two queries above, needing no plan and no GPU.
 * layout: 0 = abc, 1 = cab, 2 = cba. */
int openfft_decomp_box(int Na, int Nb, int Nc, int P, int layout, int rank,
                       int64_t start[3], int64_t end[3], int64_t* offset, int64_t* count);
int openfft_decomp_counts(int Na, int Nb, int Nc, int P, int exchange, int64_t* PxP);

/* Degree (1 = slabs, 2 = pencils) of `layout` for P ranks; -1 if undefined. */
int openfft_decomp_degree(int Na, int Nb, int Nc, int P, int layout);

/* Choose how the plan is executed.  mode: OPENFFT_TUNE_*.  With USER,
 * `candidate` indexes the list of openfft_num_candidates (otherwise ignored).
 * EXHAUSTIVE runs every candidate twice on plan-owned buffers (the paper's
 * 2 runs per method) and keeps the fastest.  SAVED takes the choice recorded
 * for this problem (see openfft_tuning_save below). */
int openfft_set_tuning(openfft_plan_t plan, int mode, int candidate);

/* Stage-kernel families: one warp per line (power-of-two lengths 32..512 and
 * the mixed-radix lengths 48..160), tiles of lines specialised per length, or
 * the generic kernel (any length); AUTO takes the first of these that exists
 * for the length. */
enum { OPENFFT_KERNEL_AUTO = 0, OPENFFT_KERNEL_WARP = 1, OPENFFT_KERNEL_TILE = 2, OPENFFT_KERNEL_GENERIC = 3 };

/* Number of execution candidates of this plan and a description of one
 * (redistribution variant, arithmetic, lines per CTA, kernel family).
 * Candidate 0 is the default (OPENFFT_TUNE_DEFAULT). */
int openfft_num_candidates(openfft_plan_t plan);
int openfft_candidate(openfft_plan_t plan, int index, int* variant, int* arith,
                      int* lines_per_cta, int* kernel);

/* Persisted tuning choices: the paper's "User-select" reuse of a method chosen
 * by an earlier tuning run, so that the initialisation skips the timing runs
 * (Sec. 3.2.3).  A process-wide table maps a problem (Na, Nb, Nc, P, dtype) to
 * the candidate its tuning chose, described as openfft_candidate describes it
 * (variant, arithmetic, lines per CTA, kernel family).  Every EXHAUSTIVE or
 * LEARNED tuning records its choice; OPENFFT_TUNE_SAVED selects the recorded
 * candidate, and runs (and records) EXHAUSTIVE when the problem has no entry or
 * its entry describes no candidate of this plan.  Thread-safe.
 *
 * openfft_tuning_save writes the table to a text file, one problem per line:
 * "Na Nb Nc P dtype variant arith lines_per_cta kernel" (lines starting with
 * '#' are comments).  openfft_tuning_load merges such a file into the table
 * (entries of the file replace those of the same problem); a malformed line
 * (not nine integers, a size or P below 1, an unknown dtype) makes the call
 * return OPENFFT_ERR_INVALID_ARG naming the line, with the table unchanged.
 * openfft_tuning_lookup sets *found to 1 and choice[0..3] to the entry of a
 * problem, or *found to 0.  openfft_tuning_clear empties the table.  None of
 * these calls touches the GPU. */
int openfft_tuning_save(const char* path);
int openfft_tuning_load(const char* path);
int openfft_tuning_lookup(int Na, int Nb, int Nc, int P, int dtype, int* found, int choice[4]);
int openfft_tuning_clear(void);
/* Index of the candidate exec currently uses. */
int openfft_current_candidate(openfft_plan_t plan);

/* Breakdown of execution time (Sec. 3.1.2: FFT, Buffer (Comm) = pack and
 * unpack, Communication = exchange).  While enabled, exec records CUDA
 * events around every kernel it launches on the plan's stream.
 * openfft_get_timing waits for the stream, adds the recorded intervals up by
 * phase since the previous call, and resets them:
 *   ms[0] / launches[0]: FFT stage kernels (with V2 they include the fused
 *                        transposes),
 *   ms[1] / launches[1]: pack and unpack kernels,
 *   ms[2] / launches[2]: exchange kernels,
 *   ms[3] / launches[3]: whole execs (first kernel start to last kernel end)
 *                        and the number of execs.
 * Events come from a plan-owned pool created by openfft_set_timing; when it
 * is full, exec first folds the recorded intervals into the totals (which
 * waits for the stream). */
int openfft_set_timing(openfft_plan_t plan, int enable);
int openfft_get_timing(openfft_plan_t plan, double ms[4], int64_t launches[4]);

/* ------------------------------------------------ learned cost model -- */

/* The run-time choice of Sec. 3.2.3 made by a learned cost model instead of
 * timing every candidate: a multilayer perceptron (d inputs -> H tanh -> H
 * tanh -> 1) predicts the natural logarithm of a candidate's execution time
 * in milliseconds from features of the problem (sizes, P, dtype) and of the
 * candidate (learned.py trains on the log ratio to the problem's fastest
 * candidate, capped at 1: only the order of one problem's candidates matters
 * to the pick).
 * It is trained on the timings the exhaustive tuner measures
 * (openfft_tune_times), on the GPU, by this library's kernels.
 *
 * Parameters are a flat float array of openfft_mlp_num_params(d, H) values:
 * W1[d][H], b1[H], W2[H][H], b2[H], W3[H], b3 (row-major; layer k computes
 * act(x W_k + b_k)).  X: n rows of d features (row-major), y: n targets.  All
 * arrays are HOST arrays; the functions copy to and from the device and
 * return when done. */
int openfft_mlp_num_params(int d, int hidden);
/* yhat[s] = f(X[s]). */
int openfft_mlp_predict(int d, int hidden, const float* params, const float* X, int n, float* yhat);
/* Mean squared error over the n samples and its gradient w.r.t. params. */
int openfft_mlp_loss_grad(int d, int hidden, const float* params, const float* X, const float* y, int n,
                          float* loss, float* grad);
/* `steps` full-batch Adam steps (beta1 0.9, beta2 0.999, eps 1e-8, learning
 * rate lr) from the given params, updated in place; losses (may be NULL)
 * receives the loss before each step.  One step is captured in a CUDA graph
 * and replayed. */
int openfft_mlp_train(int d, int hidden, const float* X, const float* y, int n, int steps, float lr,
                      float* params, float* losses);

/* Number of features per (problem, candidate) (the model's d). */
int openfft_num_features(void);
/* Features of candidate `index` of `plan` (openfft_num_features() floats). */
int openfft_candidate_features(openfft_plan_t plan, int index, float* features);
/* Time every candidate of `plan` twice (the faster run is kept) on
 * plan-owned buffers; ms[i] = -1 for a candidate that cannot run.  This is the
 * dataset writer of the learned model and the reference of its regret.  The
 * current selection is kept. */
int openfft_tune_times(openfft_plan_t plan, float* ms);
/* Install (params != NULL, count >= 1) or remove (params == NULL) the
 * process-wide cost model used by OPENFFT_TUNE_LEARNED: an ensemble of
 * `count` networks whose predictions are averaged; params holds count
 * consecutive parameter sets.  d must equal openfft_num_features().  The
 * parameters are copied. */
int openfft_set_cost_model(int count, int d, int hidden, const float* params);

/* ------------------------------------------------ tensor-core GEMM ----- */

/* Split-precision GEMM on the tcgen05 tensor cores, the contraction of the
 * DFT-GEMM form: D[M][N] = A[M][K] B[N][K]^T with fp32 host arrays.  Each
 * operand is split into a high part (tf32 if tf32 != 0, else bf16) and the
 * rounded remainder; with split != 0 D accumulates A_hi B_hi + A_hi B_lo +
 * A_lo B_hi in fp32 (without split, A_hi B_hi only).  N in {16, 32, 48, 64},
 * K a multiple of 8 (tf32) or 16 (bf16) up to 64, any M.  Copies to and from
 * the device and waits. */
int openfft_tc_gemm(int tf32, int split, int M, int N, int K, const float* A, const float* B, float* D);

/* One transpose alone (for testing the permutation): `in` holds the source
 * ordering, `out` receives the destination ordering, bit for bit.
 * exchange as in openfft_counts; variant: OPENFFT_VARIANT_*. */
int openfft_redistribute(openfft_plan_t plan, int exchange, int variant,
                         const void* in, void* out);

/* ------------------------------------------------------------ batched -- */

/* Plan `count` independent 3-D transforms of uneven sizes, run together in one
 * persistent kernel launch replayed from a captured CUDA graph.  NaNbNc: host
 * array of 3*count sizes (transform i is [NaNbNc[3i]][NaNbNc[3i+1]][NaNbNc[3i+2]]);
 * P: host array of count rank counts (each transform uses the decomposition of
 * Eqs. 2-9 with its own P).  dtype: OPENFFT_C2C_F32 (complex64, FP32) or
 * OPENFFT_C2C_F64 (complex128, double-float).  The plan allocates each
 * transform's scratch array, the twiddle tables and the work-queue tables.
 * Returns NULL on error. */
openfft_plan_t openfft_plan_many(int count, const int* NaNbNc, const int* P, int dtype);

/* Execute all transforms of a batched plan.  in / out: host arrays of `count`
 * DEVICE pointers (transform i reads in[i], writes out[i], layouts as for
 * openfft_exec_c2c; in[i] != out[i]).  One graph replay runs every stage of
 * every transform: work items (tiles of lines of one stage of one transform)
 * are taken from a device queue in stage-major order; an item of stage s
 * waits (bounded, about one second) for the stage s-1 tiles of its transform.
 * Ordered after prior work on the plan's stream; the plan's stream waits for
 * it.  A wait that runs out is reported as OPENFFT_ERR_TIMEOUT by
 * openfft_sync.  Changing the pointer set waits for earlier replays. */
int openfft_exec_many(openfft_plan_t plan, const void* const* in, void* const* out, int dir);

/* Test controls of a batched plan: what = 1 sets the wait budget to `value`
 * clock cycles; what = 2 with value != 0 makes the second-stage items of
 * transform 0 (forward) wait for one first-stage tile more than exists, so
 * that their wait runs out (value = 0 undoes it). */
int openfft_batch_debug(openfft_plan_t plan, int what, long long value);

/* Test controls of the tensor-core DFT-GEMM stages (OPENFFT_C2C_SPLIT_* plans),
 * process-wide: what = 1 sets the budget of their bounded MMA completion
 * waits to `value` clock cycles (value <= 0: the default, about one second);
 * what = 2 with value != 0 makes the stages issue and commit no MMAs, so that
 * every completion wait runs out: the kernel stores OPENFFT_ERR_TIMEOUT, frees
 * its tensor memory and returns, and openfft_sync reports the status
 * (value = 0 undoes it).  Nothing is in flight when a wait runs out. */
int openfft_tc_debug(int what, long long value);

/* Test control: the nth device allocation the library makes from now on
 * (plans, batched and distributed plans, host-buffer staging, tuning
 * buffers) fails as if the device were out of memory; the call making it
 * returns OPENFFT_ERR_NOMEM after freeing what it had allocated.  nth = 0
 * switches it off; it switches itself off after the failure.  INVALID_ARG
 * for nth < 0.  Not thread-safe with concurrent plan creation. */
int openfft_debug_alloc_fail(long long nth);

/* The checked build (compiled with -DOPENFFT_CHECKED; the library of the same
 * ABI under another file name) tests every global element index of the C2C
 * stage kernels (all forms), of the explicit transposes (pack, exchange,
 * unpack, the stepped exchanges) and of the multi-device pack / unpack
 * against the length of the array it addresses.  An index outside it is not
 * accessed, and OPENFFT_ERR_BOUNDS is stored in a device status word: the
 * plan's, reported by openfft_sync, or, for calls without one (D-dimensional,
 * multi-device and allocation-free calls), a word per device that
 * openfft_debug_bounds_status reads.  Nothing traps.  The real-to-complex,
 * batched and tensor-core stage kernels are not checked.
 * openfft_checked_build returns 1 in that build, 0 otherwise. */
int openfft_checked_build(void);

/* Checked build: synchronises the device, stores in *status the per-device
 * bounds status word (OPENFFT_OK or OPENFFT_ERR_BOUNDS) and clears it.  Other
 * builds: *status = OPENFFT_OK and the call returns OPENFFT_ERR_UNSUPPORTED. */
int openfft_debug_bounds_status(int* status);

/* ------------------------------------------- over several devices ----- */

/* The transform over G devices (one process each), device g holding the
 * contiguous block of logical ranks [floor(g P / G), floor((g+1) P / G)):
 * the paper's distributed execution flow (Sec. 3.1.1, steps (1)-(6)) with
 * the ranks of one device sharing its memory.  Because every rank's box is a
 * contiguous slice of its ordering (Eqs. 3-4), device g holds one contiguous
 * slice of each ordering (openfft_dist_rows).  Each transpose is one
 * all-to-all with variable counts among the devices (the Alltoallv method of
 * Sec. 3.2.1): the library packs (step 4) and unpacks (step 6); the caller's
 * communication library moves the segments (step 5; NCCL send / recv on
 * GPUs, gloo on CPUs).  Segment g -> h holds D[g][h] elements, the sum of the
 * P x P count matrix over the two devices' ranks, in ascending source index;
 * in g's send buffer the segments are ordered by destination device, in h's
 * receive buffer by source device, each contiguous.  1 <= G <= P; every other
 * argument and error is as for openfft_plan and openfft_counts
 * (exchange 1 = abc->cab, 2 = cab->cba, -2 = cba->cab, -1 = cab->abc). */
typedef struct openfft_dist_plan_s* openfft_dist_plan_t;

/* Host only: device g's slice of `layout` (0 = abc, 1 = cab, 2 = cba): 1-D
 * offset and element count.  Either pointer may be NULL. */
int openfft_dist_rows(int Na, int Nb, int Nc, int P, int G, int layout, int g, int64_t* offset, int64_t* count);
/* Host only: the G x G device count matrix of one transpose (row = sender),
 * into the host array GxG of G*G entries. */
int openfft_dist_counts(int Na, int Nb, int Nc, int P, int G, int exchange, int64_t* GxG);
/* Host only: pack (step 4) / unpack (step 6) of device g on HOST buffers of
 * elem_bytes-byte elements (any element type; values are moved, not read).
 * pack: `src` = g's source slice (openfft_dist_rows of the source ordering),
 * `send` = sum of g's row of the count matrix.  unpack: `recv` = sum of g's
 * column, `dst` = g's destination slice. */
int openfft_dist_pack_host(int Na, int Nb, int Nc, int P, int G, int exchange, int g, int elem_bytes,
                           const void* src, void* send);
int openfft_dist_unpack_host(int Na, int Nb, int Nc, int P, int G, int exchange, int g, int elem_bytes,
                             const void* recv, void* dst);

/* Plan of device g (the calling process's current CUDA device) for
 * OPENFFT_C2C_F64 (double-float arithmetic, complex128 at the ends and in
 * the exchanges between stages: 16-byte elements) or OPENFFT_C2C_F32
 * (complex64, 8-byte elements).  Allocates the twiddle tables and the
 * exchange tables; the caller owns every data buffer.  NULL on error. */
openfft_dist_plan_t openfft_dist_plan(int Na, int Nb, int Nc, int P, int G, int g, int dtype);
void openfft_dist_destroy(openfft_dist_plan_t plan);                       /* NULL-safe */
int openfft_dist_set_stream(openfft_dist_plan_t plan, void* stream);       /* cudaStream_t */
/* Bytes per element of the plan's buffers (16 or 8). */
int openfft_dist_elem_bytes(openfft_dist_plan_t plan);
/* Per-peer element counts of this device in one transpose: send_counts[h]
 * to device h, recv_counts[g'] from device g' (host arrays of G; either may
 * be NULL). */
int openfft_dist_exchange_counts(openfft_dist_plan_t plan, int exchange, int64_t* send_counts,
                                 int64_t* recv_counts);
/* Line-local FFT stage (steps (1)-(3)) of this device's slice, DEVICE
 * pointers, contiguous in and out (in == out allowed):
 *   FORWARD  stage 1: c-lines of the abc slice (in: complex128 / complex64),
 *            stage 2: b-lines of the cab slice, stage 3: a-lines of the cba
 *            slice (out: complex128 / complex64);
 *   BACKWARD stage 1: a-lines of cba (conjugated on entry), stage 2: b-lines
 *            of cab, stage 3: c-lines of abc (conjugated and divided by N).
 * Between stages the buffers hold the plan's internal format (double-float
 * pairs for OPENFFT_C2C_F64), which pack and unpack move unchanged. */
int openfft_dist_stage(openfft_dist_plan_t plan, int stage, int dir, const void* in, void* out);
/* Pack (step 4) and unpack (step 6) of one transpose on DEVICE buffers of
 * openfft_dist_elem_bytes elements, asynchronous on the plan's stream. */
int openfft_dist_pack(openfft_dist_plan_t plan, int exchange, const void* src, void* send);
int openfft_dist_unpack(openfft_dist_plan_t plan, int exchange, const void* recv, void* dst);

/* -------------------------------------------- 4-D and 5-D transforms ---- */

/* D-dimensional transforms (D = 3, 4, 5) under the same decomposition.  The
 * paper cites 4-D and 5-D transforms (Sec. 1) without their transpose
 * orders; this library's reading generalises Sec. 2's abc -> cab -> cba:
 * ordering s = 1..D of A[N_1]...[N_D] (d_D fastest) is
 * (d_D, ..., d_{D-s+2}, d_1, ..., d_{D-s+1}); stage s transforms the
 * fastest axis of ordering s with the transpose to ordering s + 1 fused into
 * its store.  FORWARD takes the array as given (ordering 1) and leaves the
 * spectrum in ordering D, the reversed axes: X[k_1..k_D] at index
 * ((k_D N_{D-1} + k_{D-1}) N_{D-2} + ...) N_1 + k_1.  BACKWARD takes
 * ordering D, returns ordering 1 and divides by N.  Each ordering is
 * decomposed by Eqs. 2-9 with (N1, N2, N3) = (its first dimension, its
 * second, the product of the rest), so P <= min over orderings of N1 N2
 * (OPENFFT_ERR_P_TOO_LARGE otherwise).  dims: host array of ndim axis
 * lengths, each with factors 2, 3, 5, 7 only and <= 2048.  Arithmetic as for
 * openfft_plan's default candidate (double-float for OPENFFT_C2C_F64, FP32
 * for OPENFFT_C2C_F32); the plan owns an N-element workspace and the twiddle
 * tables; `in` / `out` are caller-owned device arrays of N elements, in !=
 * out.  Asynchronous on the plan's stream. */
typedef struct openfft_nd_plan_s* openfft_nd_plan_t;
openfft_nd_plan_t openfft_nd_plan(int ndim, const int* dims, int P, int dtype);   /* NULL on error */
int openfft_nd_exec(openfft_nd_plan_t plan, const void* in, void* out, int dir);
void openfft_nd_destroy(openfft_nd_plan_t plan);                                  /* NULL-safe */
int openfft_nd_set_stream(openfft_nd_plan_t plan, void* stream);                  /* cudaStream_t */
/* Box of `rank` in the input (which = 0: ordering 1) or output (which = 1:
 * ordering D) decomposition: 1-D offset x^s and element count (Eqs. 3-4). */
int openfft_nd_box(openfft_nd_plan_t plan, int which, int rank, int64_t* offset, int64_t* count);
/* Host only: the same box for any ordering s = 1..ndim, and the P x P count
 * matrix (row = sender) of transpose `exchange`: s -> s + 1 for exchange = s
 * > 0, s + 1 -> s for exchange = -s (an O(N) enumeration). */
int openfft_nd_decomp_box(int ndim, const int* dims, int P, int ordering, int rank, int64_t* offset, int64_t* count);
int openfft_nd_decomp_counts(int ndim, const int* dims, int P, int exchange, int64_t* PxP);

/* ------------------------------------------------- allocation-free ----- */

/* The same transform as openfft_exec_c2c (fused variant, default arithmetic
 * of the dtype), for callers that may not allocate device memory: it needs no
 * plan and calls no cudaMalloc, cudaFree or allocating library routine, so it
 * fits a host framework whose own allocator owns the device budget, or a code
 * path that must not pay for the device synchronisation a cudaMalloc or
 * cudaFree can imply.  The paper has no counterpart of this entry point.
 *
 * The caller passes device pointers `in` / `out` (N elements of complex128
 * for OPENFFT_C2C_F64, complex64 for OPENFFT_C2C_F32, 16-byte aligned, in !=
 * out) and a cudaStream_t `stream` (NULL = legacy default stream); P, the
 * layouts and dir are as for openfft_plan / openfft_exec_c2c.  The
 * intermediate array and twiddle tables live in a 16 MiB (+384 KiB) static
 * device array that every GPU loading this library keeps until the process
 * exits: N times the element size (16 or 8 bytes) must not exceed 16 MiB and
 * no axis may exceed 2048, otherwise the call returns OPENFFT_ERR_UNSUPPORTED
 * without touching the GPU.  The array's device address is looked up on the
 * first call on each device (with that device current) and kept, so make that
 * first call before any stream capture.  A device reset (cudaDeviceReset) can
 * move the array: the address is looked up again after any call on that
 * device has returned OPENFFT_ERR_CUDA, so after a reset the first call that
 * fails with OPENFFT_ERR_CUDA is followed by calls that work again.  Every
 * call writes all of the array it later reads, so nothing needs clearing
 * between calls.  All calls share the array: calls whose
 * kernels may overlap on the GPU (unordered streams) race and must be
 * serialised by the caller.  Asynchronous on `stream`. */
int openfft_exec_c2c_noalloc(int Na, int Nb, int Nc, int P, int dtype,
                             const void* in, void* out, int dir, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* OPENFFT_GB_H */
