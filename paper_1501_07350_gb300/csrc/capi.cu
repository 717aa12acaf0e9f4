// capi.cu -- the C ABI of include/openfft_gb.h: plans (initialisation phase),
// execution, finalisation, decomposition queries and run-time tuning.
//
// Paper mapping (Duy & Ozaki): Sec. 3.1.1 calculation flow (init / exec /
// finalize), Sec. 2 decomposition (Eqs. 2-9) and transpose order, Sec. 3.2.1
// communication methods (the transpose variants), Sec. 3.2.3 auto-tuning
// (every candidate run twice, fastest kept; default method; user select),
// Sec. 3.2.4 (all buffers allocated once, at plan time).
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <cstring>
#include <algorithm>
#include <array>
#include <atomic>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/openfft_gb.h"
#include "decomp.h"
#include "dftgemm.h"
#include "fft_stage.h"
#include "redistribute.h"
#include "batch.h"

using namespace ofg;

namespace ofg {

// 0: allocations behave; k > 0: the k-th allocation from now fails (once)
static std::atomic<long long> g_alloc_fail_at{0};

cudaError_t dev_malloc(void** ptr, size_t bytes)
{
    long long k = g_alloc_fail_at.load();
    while (k > 0 && !g_alloc_fail_at.compare_exchange_weak(k, k - 1)) {
    }
    if (k == 1) {
        *ptr = nullptr;
        return cudaErrorMemoryAllocation;
    }
    return cudaMalloc(ptr, bytes);
}

}  // namespace ofg

namespace {

thread_local std::string g_err;
thread_local int g_status = OPENFFT_OK;

int fail(int status, const std::string& msg)
{
    g_status = status;
    g_err = msg;
    return status;
}

int cuda_fail(cudaError_t e, const char* what)
{
    return fail(OPENFFT_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

// ----------------------------------------------------------------- radix --

bool radix_plan(int n, std::vector<int>& rad)
{
    rad.clear();
    int m = n;
    while (m % 8 == 0) { rad.push_back(8); m /= 8; }
    while (m % 4 == 0) { rad.push_back(4); m /= 4; }
    while (m % 2 == 0) { rad.push_back(2); m /= 2; }
    while (m % 3 == 0) { rad.push_back(3); m /= 3; }
    while (m % 5 == 0) { rad.push_back(5); m /= 5; }
    while (m % 7 == 0) { rad.push_back(7); m /= 7; }
    return m == 1 && (int)rad.size() <= kMaxPasses;
}

int ilog2(int g) { int l = 0; while ((1 << l) < g) ++l; return l; }

// ------------------------------------------------------------ candidates --

struct Candidate {
    int variant;   // OPENFFT_VARIANT_*
    int arith;     // ARITH_*
    int G;         // lines per CTA target (power of two)
    int family;    // KERNEL_*
};

// one step of an execution
enum OpKind { OP_STAGE, OP_PACK, OP_EXCHANGE, OP_UNPACK, OP_SEG_EXCHANGE, OP_SEG_UNPACK };
enum Buf { B_IN, B_OUT, B_A, B_B };

struct Op {
    OpKind kind;
    int src, dst;            // Buf ids
    StageLaunch stage;       // OP_STAGE
    int tix;                 // transpose table index (0..3) for pack/exchange/unpack
    int from_send;           // OP_UNPACK
    int sched;               // OP_SEG_*: SCHED_*
    int64_t step;            // OP_SEG_*: step of the schedule
};

struct TransposeTables {
    Transpose t;
    std::vector<int64_t> C;
    int64_t* d_sbase = nullptr;
    int64_t* d_rbase = nullptr;
    int64_t* d_chunks = nullptr;
    int64_t nchunks = 0;
    int64_t* d_C = nullptr;       // count matrix [r*P+s]
    int64_t* d_sdispl = nullptr;  // send displacement of segment (r, s) [r*P+s]
    int64_t* d_rdispl = nullptr;  // receive displacement of segment (r, s) [s*P+r]
};

}  // namespace

// Host-buffer execution overlaps the host<->device copies with the line-local
// first and last stages in at most this many line ranges.
constexpr int kMaxHostChunks = 32;

struct openfft_plan_s {
    int Na, Nb, Nc, P, dtype;
    int64_t N;
    int device = 0, sms = 148;
    cudaStream_t stream = nullptr;
    size_t elem_bytes = 16;       // bytes of one element in the workspace
    void* bufA = nullptr;
    void* bufB = nullptr;
    void* tw[3][3] = {};          // [axis a,b,c][FMT_C128, FMT_C64, FMT_DF]
    std::vector<int> rad[3];      // radix plans of Na, Nb, Nc
    TransposeTables tt[4];        // index: 0 = R1, 1 = R2, 2 = R2', 3 = R1'
    std::vector<Candidate> cands;
    int current = 0;
    std::vector<Op> ops_fwd, ops_bwd;
    void* stage_in = nullptr;     // host-exec staging (lazy)
    void* stage_out = nullptr;
    // host-exec copies: plan-owned upload / download streams (lazy), or the
    // caller's (openfft_set_copy_streams)
    cudaStream_t own_h2d = nullptr, own_d2h = nullptr;
    cudaStream_t user_h2d = nullptr, user_d2h = nullptr;
    bool user_copy_streams = false;
    cudaEvent_t host_ev[2 * kMaxHostChunks + 2] = {};   // ranges in, ranges out, stage 1 read, download done
    int host_chunks = 0;                           // 0 = chosen by size
    // execution-time breakdown
    bool timing = false;
    std::vector<cudaEvent_t> ev;  // pool
    std::vector<int> ev_cat;      // category of the interval ending at event i (-1: exec start)
    size_t ev_used = 0;
    double t_ms[4] = {0, 0, 0, 0};
    int64_t t_launch[4] = {0, 0, 0, 0};
    BatchPlan* batch = nullptr;   // set for plans made by openfft_plan_many
    int* d_status = nullptr;      // device status word of the tensor-core stages
    void* bimg[3] = {};           // DFT-GEMM operand images per axis (split dtypes)
    bool real = false;            // real transform (OPENFFT_R2C_*): half arrays after stage 1
    int Ncx = 0;                  // c extent of the complex arrays: Nc, or Nc / 2 + 1 for real plans
};

namespace {

int tix_of(int which) { return which == 1 ? 0 : (which == 2 ? 1 : (which == -2 ? 2 : 3)); }

int elem_bytes_of(int arith) { return (arith == ARITH_F64 || arith == ARITH_DF) ? 16 : 8; }
bool is_tc(int arith) { return arith == ARITH_TC_TF32 || arith == ARITH_TC_BF16; }

// Build the launch of one stage: lines of length n; l = i1 + i2*M1;
// out(l,k) = i1*S1 + i2*S2 + k*Sk.
int make_stage(openfft_plan_s* p, int axis, int arith, int Gt, int family, int64_t M1, int64_t M2,
               int64_t S1, int64_t S2, int64_t Sk, int group_i2, int contig, int in_fmt,
               int out_fmt, int conj_in, int conj_out, double scale, int do_fft, StageLaunch& L)
{
    const int n = axis == 0 ? p->Na : (axis == 1 ? p->Nb : p->Nc);
    const std::vector<int>& rad = p->rad[axis];
    const int E = elem_bytes_of(arith);
    if (is_tc(arith) && do_fft) {
        // DFT-GEMM stage: n = R S, tiles of Gt lines (as many as fit)
        int R = 0, S = 0;
        if (!dftgemm_factor(n, arith == ARITH_TC_TF32, &R, &S))
            return fail(OPENFFT_ERR_UNSUPPORTED_RADIX, "DFT-GEMM form: every axis must be R*S with 2 <= R, S <= 32");
        int G = dftgemm_lines(n, R, S, arith == ARITH_TC_TF32, Gt);
        if (!G) return fail(OPENFFT_ERR_UNSUPPORTED_RADIX, "DFT-GEMM form: axis too long for one CTA");
        if (!p->bimg[axis]) return fail(OPENFFT_ERR_INVALID_ARG, "DFT-GEMM form: plan has no operand image");
        const int64_t Mg = group_i2 ? M2 : M1;
        StageArgs& a = L.args;
        std::memset(&a, 0, sizeof(a));
        a.tw = p->tw[axis][FMT_C64];
        a.aux = p->bimg[axis];
        a.M1 = M1; a.M2 = M2; a.S1 = S1; a.S2 = S2; a.Sk = Sk;
        a.ngroups = (Mg + G - 1) / G;
        a.scale = scale;
        a.n = n; a.G = G; a.log2G = ilog2(G);
        a.group_i2 = group_i2; a.contig_store = contig;
        a.npass = 2; a.radix[0] = R; a.radix[1] = S;
        a.conj_in = conj_in; a.conj_out = conj_out; a.do_fft = 1;
        a.in_fmt = in_fmt; a.out_fmt = out_fmt;
        L.arith = arith; L.sms = p->sms; L.family = family; L.status = p->d_status;
        L.grid = a.ngroups * (group_i2 ? M1 : M2);
        L.smem = 0;
        return OPENFFT_OK;
    }
    const size_t cap = 200 * 1024;
    int G = Gt;
    const int64_t Mg = group_i2 ? M2 : M1;
    while (G > 1 && (int64_t)(G / 2) >= Mg) G /= 2;           // no more lanes than lines
    while (G > 1 && 2 * (size_t)n * (G + 1) * E > cap) G /= 2;
    if (2 * (size_t)n * (G + 1) * E > cap) return fail(OPENFFT_ERR_UNSUPPORTED_RADIX, "axis too long for one CTA");
    StageArgs& a = L.args;
    std::memset(&a, 0, sizeof(a));
    a.in = nullptr; a.out = nullptr;
    const int twf = arith == ARITH_F64 ? FMT_C128 : ((arith == ARITH_F32 || is_tc(arith)) ? FMT_C64 : FMT_DF);
    a.tw = p->tw[axis][twf];
    a.M1 = M1; a.M2 = M2; a.S1 = S1; a.S2 = S2; a.Sk = Sk;
    a.ngroups = (Mg + G - 1) / G;
    a.scale = scale;
    a.n = n; a.G = G; a.log2G = ilog2(G);
    a.group_i2 = group_i2; a.contig_store = contig;
    a.npass = (int)rad.size();
    for (size_t i = 0; i < rad.size(); ++i) a.radix[i] = rad[i];
    a.conj_in = conj_in; a.conj_out = conj_out; a.do_fft = do_fft;
    a.in_fmt = in_fmt; a.out_fmt = out_fmt;
    L.arith = arith;
    L.sms = p->sms;
    L.family = family;
    L.status = p->d_status;
    L.grid = a.ngroups * (group_i2 ? M1 : M2);
    L.smem = 2 * (size_t)n * (G + 1) * E;     // two ping-pong tiles
    if (L.grid > 0x7fffffffLL) return fail(OPENFFT_ERR_UNSUPPORTED, "grid too large");
    return OPENFFT_OK;
}

// The real stage of a real plan: forward = stage 1 (real c-lines -> half
// spectra, stored transposed into the cab half array [Ncx][Na][Nb]), backward
// = the last stage (abc half array [Na][Nb][Ncx] -> real c-lines, times 1/N).
int make_real_stage(openfft_plan_s* p, int arith, int Gt, bool forward, int mid_fmt, StageLaunch& L)
{
    const int n = p->Nc;
    const int E = elem_bytes_of(arith);
    const int64_t lines = (int64_t)p->Na * p->Nb;
    int G = Gt;
    while (G > 1 && (int64_t)G >= lines) G /= 2;          // no more complex lines than line pairs
    while (G > 1 && 2 * (size_t)n * (G + 1) * E > 200 * 1024) G /= 2;
    if (2 * (size_t)n * (G + 1) * E > 200 * 1024) return fail(OPENFFT_ERR_UNSUPPORTED_RADIX, "axis too long for one CTA");
    StageArgs& a = L.args;
    std::memset(&a, 0, sizeof(a));
    const int twf = arith == ARITH_F64 ? FMT_C128 : (arith == ARITH_F32 ? FMT_C64 : FMT_DF);
    a.tw = p->tw[2][twf];
    a.M1 = lines; a.M2 = 1;
    a.S1 = 1; a.S2 = 0; a.Sk = lines;
    a.ngroups = (lines + 2 * G - 1) / (2 * G);
    a.scale = forward ? 1.0 : 1.0 / (double)p->N;
    a.n = n; a.G = G; a.log2G = ilog2(G);
    a.npass = (int)p->rad[2].size();
    for (size_t i = 0; i < p->rad[2].size(); ++i) a.radix[i] = p->rad[2][i];
    a.do_fft = 1;
    const int real_fmt = arith == ARITH_F32 ? FMT_R32 : FMT_R64;
    a.in_fmt = forward ? real_fmt : mid_fmt;
    a.out_fmt = forward ? mid_fmt : real_fmt;
    L.arith = arith; L.sms = p->sms; L.family = forward ? KERNEL_R2C : KERNEL_C2R; L.status = p->d_status;
    L.grid = a.ngroups;
    L.smem = 2 * (size_t)n * (G + 1) * E;
    if (L.grid > 0x7fffffffLL) return fail(OPENFFT_ERR_UNSUPPORTED, "grid too large");
    return OPENFFT_OK;
}

Op stage_op(int src, int dst, const StageLaunch& L)
{
    Op o; std::memset(&o, 0, sizeof(o));
    o.kind = OP_STAGE; o.src = src; o.dst = dst; o.stage = L;
    return o;
}

Op redist_op(OpKind k, int src, int dst, int tix, int from_send, int sched = 0, int64_t step = 0)
{
    Op o; std::memset(&o, 0, sizeof(o));
    o.kind = k; o.src = src; o.dst = dst; o.tix = tix; o.from_send = from_send;
    o.sched = sched; o.step = step;
    return o;
}

// The paper's communication methods (Sec. 3.2.1) as the ops of one transpose
// from buffer `from` (send segments go to `other`): returns where the
// destination ordering lands (`final_to` if given).
int transpose_ops(std::vector<Op>& ops, int variant, int tix, int from, int final_to, int64_t P)
{
    const int other = from == B_A ? B_B : B_A;
    ops.push_back(redist_op(OP_PACK, from, other, tix, 0));             // step (4)
    int landing;
    auto stepped_exchange = [&](int sched) {                            // step (5), in steps
        const int64_t n = num_steps(sched, P, kBlockSize);
        for (int64_t k = 0; k < n; ++k) ops.push_back(redist_op(OP_SEG_EXCHANGE, other, from, tix, 0, sched, k));
    };
    switch (variant) {
    case OPENFFT_VARIANT_PACK_EXCHANGE_UNPACK:                          // Alltoallv
        ops.push_back(redist_op(OP_EXCHANGE, other, from, tix, 0));
        landing = final_to >= 0 ? final_to : other;
        ops.push_back(redist_op(OP_UNPACK, from, landing, tix, 0));
        break;
    case OPENFFT_VARIANT_ISEND_WAITALL:
        stepped_exchange(SCHED_PER_SENDER);
        landing = final_to >= 0 ? final_to : other;
        ops.push_back(redist_op(OP_UNPACK, from, landing, tix, 0));
        break;
    case OPENFFT_VARIANT_ISEND_WAITALL_BLOCK:
        stepped_exchange(SCHED_BLOCKED);
        landing = final_to >= 0 ? final_to : other;
        ops.push_back(redist_op(OP_UNPACK, from, landing, tix, 0));
        break;
    case OPENFFT_VARIANT_SENDRECV:
        stepped_exchange(SCHED_SHIFTED);
        landing = final_to >= 0 ? final_to : other;
        ops.push_back(redist_op(OP_UNPACK, from, landing, tix, 0));
        break;
    case OPENFFT_VARIANT_ISEND_WAITSOME_BLOCK: {                         // unpack each group's segments
        landing = final_to >= 0 ? final_to : from;
        const int64_t n = num_steps(SCHED_BLOCKED, P, kBlockSize);
        for (int64_t k = 0; k < n; ++k)
            ops.push_back(redist_op(OP_SEG_UNPACK, other, landing, tix, 1, SCHED_BLOCKED, k));
        break;
    }
    default:                                                             // Isend_Waitsome
        landing = final_to >= 0 ? final_to : from;
        ops.push_back(redist_op(OP_UNPACK, other, landing, tix, 1));
        break;
    }
    return landing;
}

// Build the forward and backward op lists of candidate c.
int build_ops(openfft_plan_s* p, const Candidate& c)
{
    const int64_t Na = p->Na, Nb = p->Nb, Nc = p->Nc, N = p->N;
    const int ar = c.arith;
    const int ext = (ar == ARITH_F32 || is_tc(ar)) ? FMT_C64 : FMT_C128;   // user arrays
    const int mid = ar == ARITH_DF ? FMT_DF : ext;                          // workspace arrays
    const double invN = 1.0 / (double)N;
    std::vector<Op>& F = p->ops_fwd;
    std::vector<Op>& B = p->ops_bwd;
    F.clear(); B.clear();
    StageLaunch L;
    int st;
    if (p->real) {
        // real transform, fused stores only; the complex stages run on the
        // half arrays (c extent Ncx = Nc / 2 + 1)
        if (c.variant != OPENFFT_VARIANT_FUSED) return fail(OPENFFT_ERR_UNSUPPORTED, "real plans run the fused variant");
        const int64_t Nh = p->Ncx;
        // forward: real c-lines -> cab half; b-lines of cab -> cba; a-lines of cba in place
        if ((st = make_real_stage(p, ar, c.G, true, mid, L))) return st;
        F.push_back(stage_op(B_IN, B_A, L));
        if ((st = make_stage(p, 1, ar, c.G, c.family, Na, Nh, 1, Nb * Na, Na, 0, 0, mid, mid, 0, 0, 1.0, 1, L))) return st;
        F.push_back(stage_op(B_A, B_OUT, L));
        if ((st = make_stage(p, 0, ar, c.G, c.family, Nh * Nb, 1, Na, 0, 1, 0, 1, mid, ext, 0, 0, 1.0, 1, L))) return st;
        F.push_back(stage_op(B_OUT, B_OUT, L));
        // backward: a-lines of cba -> cab (conjugated on entry); b-lines of cab
        // -> abc half [Na][Nb][Nh]; real c-lines out (times 1/N)
        if ((st = make_stage(p, 0, ar, c.G, c.family, Nb, Nh, 1, Na * Nb, Nb, 0, 0, ext, mid, 1, 0, 1.0, 1, L))) return st;
        B.push_back(stage_op(B_IN, B_A, L));
        if ((st = make_stage(p, 1, ar, c.G, c.family, Na, Nh, Nb * Nh, 1, Nh, 1, 0, mid, mid, 0, 0, 1.0, 1, L))) return st;
        B.push_back(stage_op(B_A, B_B, L));
        if ((st = make_real_stage(p, ar, c.G, false, mid, L))) return st;
        B.push_back(stage_op(B_B, B_OUT, L));
        return OPENFFT_OK;
    }
    if (c.variant == OPENFFT_VARIANT_FUSED) {
        // forward: c-lines of abc -> cab; b-lines of cab -> cba; a-lines of cba in place
        if ((st = make_stage(p, 2, ar, c.G, c.family, Na * Nb, 1, 1, 0, Na * Nb, 0, 0, ext, mid, 0, 0, 1.0, 1, L))) return st;
        F.push_back(stage_op(B_IN, B_A, L));
        if ((st = make_stage(p, 1, ar, c.G, c.family, Na, Nc, 1, Nb * Na, Na, 0, 0, mid, mid, 0, 0, 1.0, 1, L))) return st;
        F.push_back(stage_op(B_A, B_OUT, L));
        if ((st = make_stage(p, 0, ar, c.G, c.family, Nc * Nb, 1, Na, 0, 1, 0, 1, mid, ext, 0, 0, 1.0, 1, L))) return st;
        F.push_back(stage_op(B_OUT, B_OUT, L));
        // backward (conjugate on entry and exit): a-lines of cba -> cab; b-lines
        // of cab -> abc (grouped along c, whose output stride is 1); c-lines in place
        if ((st = make_stage(p, 0, ar, c.G, c.family, Nb, Nc, 1, Na * Nb, Nb, 0, 0, ext, mid, 1, 0, 1.0, 1, L))) return st;
        B.push_back(stage_op(B_IN, B_A, L));
        if ((st = make_stage(p, 1, ar, c.G, c.family, Na, Nc, Nb * Nc, 1, Nc, 1, 0, mid, mid, 0, 0, 1.0, 1, L))) return st;
        B.push_back(stage_op(B_A, B_OUT, L));
        if ((st = make_stage(p, 2, ar, c.G, c.family, Na * Nb, 1, Nc, 0, 1, 0, 1, mid, ext, 0, 1, invN, 1, L))) return st;
        B.push_back(stage_op(B_OUT, B_OUT, L));
        return OPENFFT_OK;
    }
    // explicit variants: contiguous stage stores, transposes through A and B
    auto transpose = [&](std::vector<Op>& ops, int tix, int from, int final_to) {
        return transpose_ops(ops, c.variant, tix, from, final_to, p->P);
    };
    auto other_of = [](int b) { return b == B_A ? B_B : B_A; };
    // forward
    if ((st = make_stage(p, 2, ar, c.G, c.family, Na * Nb, 1, Nc, 0, 1, 0, 1, ext, mid, 0, 0, 1.0, 1, L))) return st;
    F.push_back(stage_op(B_IN, B_A, L));
    int x = transpose(F, 0, B_A, -1);                // abc -> cab
    if ((st = make_stage(p, 1, ar, c.G, c.family, Nc * Na, 1, Nb, 0, 1, 0, 1, mid, mid, 0, 0, 1.0, 1, L))) return st;
    F.push_back(stage_op(x, other_of(x), L));
    transpose(F, 1, other_of(x), B_OUT);             // cab -> cba lands in out
    if ((st = make_stage(p, 0, ar, c.G, c.family, Nc * Nb, 1, Na, 0, 1, 0, 1, mid, ext, 0, 0, 1.0, 1, L))) return st;
    F.push_back(stage_op(B_OUT, B_OUT, L));
    // backward
    if ((st = make_stage(p, 0, ar, c.G, c.family, Nc * Nb, 1, Na, 0, 1, 0, 1, ext, mid, 1, 0, 1.0, 1, L))) return st;
    B.push_back(stage_op(B_IN, B_A, L));
    x = transpose(B, 2, B_A, -1);                    // cba -> cab
    if ((st = make_stage(p, 1, ar, c.G, c.family, Nc * Na, 1, Nb, 0, 1, 0, 1, mid, mid, 0, 0, 1.0, 1, L))) return st;
    B.push_back(stage_op(x, other_of(x), L));
    transpose(B, 3, other_of(x), B_OUT);             // cab -> abc lands in out
    if ((st = make_stage(p, 2, ar, c.G, c.family, Na * Nb, 1, Nc, 0, 1, 0, 1, mid, ext, 0, 1, invN, 1, L))) return st;
    B.push_back(stage_op(B_OUT, B_OUT, L));
    return OPENFFT_OK;
}

void* resolve(openfft_plan_s* p, int b, const void* in, void* out)
{
    switch (b) {
    case B_IN: return const_cast<void*>(in);
    case B_OUT: return out;
    case B_A: return p->bufA;
    default: return p->bufB;
    }
}

// Add the recorded intervals to the per-phase totals (waits for the stream).
int fold_timing(openfft_plan_s* p)
{
    if (p->ev_used == 0) return OPENFFT_OK;
    cudaError_t e = cudaEventSynchronize(p->ev[p->ev_used - 1]);
    if (e) return cuda_fail(e, "timing event");
    size_t start = 0;
    for (size_t i = 1; i < p->ev_used; ++i) {
        const int cat = p->ev_cat[i];
        if (cat < 0) {                              // a new exec starts at event i
            float ms = 0.f;
            cudaEventElapsedTime(&ms, p->ev[start], p->ev[i - 1]);
            p->t_ms[3] += ms; p->t_launch[3] += 1;
            start = i;
            continue;
        }
        float ms = 0.f;
        cudaEventElapsedTime(&ms, p->ev[i - 1], p->ev[i]);
        p->t_ms[cat] += ms;
        p->t_launch[cat] += 1;
    }
    float ms = 0.f;
    cudaEventElapsedTime(&ms, p->ev[start], p->ev[p->ev_used - 1]);
    p->t_ms[3] += ms; p->t_launch[3] += 1;
    p->ev_used = 0;
    return OPENFFT_OK;
}

int record(openfft_plan_s* p, int cat)
{
    cudaError_t e = cudaEventRecord(p->ev[p->ev_used], p->stream);
    if (e) return cuda_fail(e, "timing event");
    p->ev_cat[p->ev_used++] = cat;
    return OPENFFT_OK;
}

// Runs ops[i0, i1) on the plan's stream (the whole list by default).
int run_ops(openfft_plan_s* p, const std::vector<Op>& ops, const void* in, void* out, int arith,
            size_t i0 = 0, size_t i1 = SIZE_MAX)
{
    const int E = elem_bytes_of(arith);
    if (i1 > ops.size()) i1 = ops.size();
    if (p->timing) {
        if (p->ev_used + ops.size() + 1 > p->ev.size()) { int st = fold_timing(p); if (st) return st; }
        int st = record(p, -1);
        if (st) return st;
    }
    Bounds bnd;                   // every buffer of a transpose holds N elements
    bnd.chk = p->d_status; bnd.lim = p->N;
    for (size_t i = i0; i < i1; ++i) {
        const Op& o = ops[i];
        void* s = resolve(p, o.src, in, out);
        void* d = resolve(p, o.dst, in, out);
        cudaError_t e = cudaSuccess;
        if (o.kind == OP_STAGE) {
            StageLaunch L = o.stage;
            L.args.in = s; L.args.out = d;
            e = launch_stage(L, p->stream);
        } else if (o.kind == OP_SEG_EXCHANGE) {
            const TransposeTables& T = p->tt[o.tix];
            e = launch_segment_exchange(o.sched, p->P, kBlockSize, o.step, E, T.d_C, T.d_sdispl, T.d_rdispl, s, d, p->stream, bnd);
        } else if (o.kind == OP_SEG_UNPACK) {
            const TransposeTables& T = p->tt[o.tix];
            e = launch_segment_unpack(T.t, o.sched, kBlockSize, o.step, E, s, d, T.d_sbase, p->stream, bnd);
        } else {
            const TransposeTables& T = p->tt[o.tix];
            if (o.kind == OP_PACK) e = launch_pack(T.t, E, s, d, T.d_sbase, p->N, p->sms, p->stream, bnd);
            else if (o.kind == OP_EXCHANGE) e = launch_exchange(E, T.d_chunks, T.nchunks, s, d, p->sms, p->stream, bnd);
            else e = launch_unpack(T.t, E, s, d, o.from_send ? T.d_sbase : T.d_rbase, o.from_send, p->N, p->sms, p->stream, bnd);
        }
        if (e != cudaSuccess) return cuda_fail(e, "kernel launch");
        if (p->timing) {
            const int cat = o.kind == OP_STAGE ? 0 : ((o.kind == OP_EXCHANGE || o.kind == OP_SEG_EXCHANGE) ? 2 : 1);
            int st = record(p, cat);
            if (st) return st;
        }
    }
    return OPENFFT_OK;
}

int select_candidate(openfft_plan_s* p, int idx)
{
    if (idx < 0 || idx >= (int)p->cands.size()) return fail(OPENFFT_ERR_INVALID_ARG, "candidate index out of range");
    int st = build_ops(p, p->cands[(size_t)idx]);
    if (st) return st;
    p->current = idx;
    return OPENFFT_OK;
}

int validate_dims(int Na, int Nb, int Nc, int P)
{
    if (Na < 1 || Nb < 1 || Nc < 1 || P < 1) return fail(OPENFFT_ERR_INVALID_ARG, "sizes and P must be >= 1");
    const int64_t a = Na, b = Nb, c = Nc;
    if ((int64_t)P > a * b || (int64_t)P > c * a || (int64_t)P > c * b)
        return fail(OPENFFT_ERR_P_TOO_LARGE, "P exceeds N1*N2 of an ordering (Eq. 2 undefined)");
    return OPENFFT_OK;
}

void free_plan(openfft_plan_s* p)
{
    if (!p) return;
    cudaFree(p->bufA); cudaFree(p->bufB);
    for (auto& row : p->tw) for (void* t : row) cudaFree(t);
    for (void* b : p->bimg) cudaFree(b);
    for (auto& T : p->tt) {
        cudaFree(T.d_sbase); cudaFree(T.d_rbase); cudaFree(T.d_chunks);
        cudaFree(T.d_C); cudaFree(T.d_sdispl); cudaFree(T.d_rdispl);
    }
    cudaFree(p->stage_in); cudaFree(p->stage_out);
    if (p->user_copy_streams) { cudaStreamSynchronize(p->user_h2d); cudaStreamSynchronize(p->user_d2h); }
    if (p->own_h2d) { cudaStreamSynchronize(p->own_h2d); cudaStreamDestroy(p->own_h2d); }
    if (p->own_d2h) { cudaStreamSynchronize(p->own_d2h); cudaStreamDestroy(p->own_d2h); }
    for (cudaEvent_t e : p->host_ev) if (e) cudaEventDestroy(e);
    cudaFree(p->d_status);
    for (cudaEvent_t e : p->ev) cudaEventDestroy(e);
    if (p->batch) batch_destroy(p->batch);
    delete p;
}

int box_of(const Ordering& o, int rank, int64_t start[3], int64_t end[3], int64_t* offset, int64_t* count)
{
    if (rank < 0 || rank >= o.P) return fail(OPENFFT_ERR_INVALID_ARG, "rank out of range");
    const int64_t xs = box_begin(o, rank), xe = box_begin(o, rank + 1) - 1;
    auto to3 = [&](int64_t x, int64_t v[3]) {           // Eqs. 5-7
        int64_t d0 = x / (o.D1 * o.D2);
        int64_t d1 = (x - d0 * o.D1 * o.D2) / o.D2;
        v[0] = d0; v[1] = d1; v[2] = x - d0 * o.D1 * o.D2 - d1 * o.D2;
    };
    if (start) to3(xs, start);
    if (end) { if (xe >= xs) to3(xe, end); else end[0] = end[1] = end[2] = -1; }
    if (offset) *offset = xs;
    if (count) *count = xe - xs + 1;
    return OPENFFT_OK;
}

}  // namespace

namespace ofg {
// error reporting for entry points defined in other translation units
int set_last_error(int status, const char* msg) { return fail(status, msg); }
}  // namespace ofg

namespace {
int fail_cstr(int status, const char* msg) { return fail(status, msg); }

// ---------------------------------------------------------- cost model --

constexpr int kFeatures = 21;

// Features of (problem, candidate) for the learned cost model.
void candidate_features(const openfft_plan_s* p, const Candidate& c, float* f)
{
    auto l2 = [](double x) { return (float)std::log2(x); };
    auto pow2 = [](int n) { return (n & (n - 1)) == 0 ? 1.f : 0.f; };
    f[0] = l2(p->Na) / 10.f; f[1] = l2(p->Nb) / 10.f; f[2] = l2(p->Nc) / 10.f;
    f[3] = l2((double)p->N) / 30.f;
    f[4] = l2(p->P) / 10.f;
    f[5] = (p->dtype == OPENFFT_C2C_F64 || p->dtype == OPENFFT_R2C_F64) ? 1.f : 0.f;
    f[6] = 0.f;                                            // log2(batch) / 7, batch = 1
    f[7] = c.variant == OPENFFT_VARIANT_FUSED ? 1.f : 0.f;
    f[8] = c.variant == OPENFFT_VARIANT_PACK_UNPACK ? 1.f : 0.f;
    f[9] = c.variant == OPENFFT_VARIANT_PACK_EXCHANGE_UNPACK ? 1.f : 0.f;
    f[10] = c.arith == ARITH_DF ? 1.f : 0.f;
    f[11] = c.arith == ARITH_F64 ? 1.f : 0.f;
    f[12] = l2(c.G) / 4.f;
    f[13] = (c.family == KERNEL_AUTO || c.family == KERNEL_WARP) ? 1.f : 0.f;
    f[14] = c.family == KERNEL_TILE ? 1.f : 0.f;
    f[15] = c.family == KERNEL_GENERIC ? 1.f : 0.f;
    f[16] = (pow2(p->Na) + pow2(p->Nb) + pow2(p->Nc)) / 3.f;
    f[17] = c.variant == OPENFFT_VARIANT_ISEND_WAITALL ? 1.f : 0.f;
    f[18] = c.variant == OPENFFT_VARIANT_ISEND_WAITALL_BLOCK ? 1.f : 0.f;
    f[19] = c.variant == OPENFFT_VARIANT_ISEND_WAITSOME_BLOCK ? 1.f : 0.f;
    f[20] = c.variant == OPENFFT_VARIANT_SENDRECV ? 1.f : 0.f;
}

std::mutex g_model_mu;
std::vector<float> g_model;          // parameters of the installed cost models (an ensemble)
int g_model_d = 0, g_model_h = 0, g_model_k = 0;

// Time every candidate twice (the paper's two runs per method) on plan-owned
// buffers and keep the faster run; the current selection is restored.
int time_candidates(openfft_plan_s* p, std::vector<float>& ms)
{
    const size_t bytes = (size_t)p->N * p->elem_bytes;
    void *tin = nullptr, *tout = nullptr;
    if (dev_malloc((void**)&tin, bytes) || dev_malloc((void**)&tout, bytes)) {
        cudaGetLastError(); cudaFree(tin);
        return fail(OPENFFT_ERR_NOMEM, "tuning buffers");
    }
    cudaMemsetAsync(tin, 0, bytes, p->stream);
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0); cudaEventCreate(&e1);
    const int keep = p->current;
    int st = OPENFFT_OK;
    ms.assign(p->cands.size(), -1.f);
    for (int i = 0; i < (int)p->cands.size() && !st; ++i) {
        if (select_candidate(p, i)) { g_status = OPENFFT_OK; continue; }   // not buildable here
        float best = 1e30f;
        for (int rep = 0; rep < 2 && !st; ++rep) {
            cudaEventRecord(e0, p->stream);
            st = p->real ? openfft_exec_r2c(p, tin, tout) : openfft_exec_c2c(p, tin, tout, OPENFFT_FORWARD);
            cudaEventRecord(e1, p->stream);
            cudaEventSynchronize(e1);
            float t = 0.f;
            cudaEventElapsedTime(&t, e0, e1);
            best = t < best ? t : best;
        }
        ms[(size_t)i] = best;
    }
    cudaEventDestroy(e0); cudaEventDestroy(e1);
    cudaFree(tin); cudaFree(tout);
    select_candidate(p, keep);
    return st;
}

}  // namespace

// =================================================================== ABI ==

extern "C" {

const char* openfft_last_error(void) { return g_err.c_str(); }
int openfft_last_status(void) { return g_status; }

int openfft_debug_alloc_fail(long long nth)
{
    if (nth < 0) return fail(OPENFFT_ERR_INVALID_ARG, "nth must be >= 0");
    g_alloc_fail_at.store(nth);
    return OPENFFT_OK;
}

int openfft_debug_bounds_status(int* status)
{
    if (!status) return fail(OPENFFT_ERR_INVALID_ARG, "null status");
    *status = OPENFFT_OK;
#ifdef OPENFFT_CHECKED
    int* w = fallback_status_word();
    if (!w) return fail(OPENFFT_ERR_CUDA, "status word of the checked build");
    cudaError_t e;
    if ((e = cudaDeviceSynchronize()) || (e = cudaMemcpy(status, w, sizeof(int), cudaMemcpyDeviceToHost)) ||
        (e = cudaMemset(w, 0, sizeof(int))))
        return cuda_fail(e, "status word of the checked build");
    return OPENFFT_OK;
#else
    return fail(OPENFFT_ERR_UNSUPPORTED, "not the checked build (OPENFFT_CHECKED)");
#endif
}

int openfft_checked_build(void)
{
#ifdef OPENFFT_CHECKED
    return 1;
#else
    return 0;
#endif
}

int openfft_decomp_degree(int Na, int Nb, int Nc, int P, int layout)
{
    if (Na < 1 || Nb < 1 || Nc < 1 || P < 1 || layout < 0 || layout > 2) return -1;
    return ordering_of(layout, Na, Nb, Nc, P).degree;
}

int openfft_decomp_box(int Na, int Nb, int Nc, int P, int layout, int rank,
                       int64_t start[3], int64_t end[3], int64_t* offset, int64_t* count)
{
    int st = validate_dims(Na, Nb, Nc, P);
    if (st) return st;
    if (layout < 0 || layout > 2) return fail(OPENFFT_ERR_INVALID_ARG, "layout must be 0, 1 or 2");
    return box_of(ordering_of(layout, Na, Nb, Nc, P), rank, start, end, offset, count);
}

int openfft_decomp_counts(int Na, int Nb, int Nc, int P, int exchange, int64_t* PxP)
{
    int st = validate_dims(Na, Nb, Nc, P);
    if (st) return st;
    if (!PxP) return fail(OPENFFT_ERR_INVALID_ARG, "null output");
    if (exchange != 1 && exchange != 2 && exchange != -1 && exchange != -2)
        return fail(OPENFFT_ERR_INVALID_ARG, "exchange must be 1, 2, -2 or -1");
    Transpose t = make_transpose(exchange, Na, Nb, Nc, P);
    for (int64_t r = 0; r < P; ++r)
        for (int64_t s = 0; s < P; ++s) PxP[r * P + s] = pair_count(t, r, s);
    return OPENFFT_OK;
}

openfft_plan_t openfft_plan(int Na, int Nb, int Nc, int P, int dtype)
{
    if (dtype < OPENFFT_C2C_F64 || dtype > OPENFFT_R2C_F32) {
        fail(OPENFFT_ERR_INVALID_ARG, "unknown dtype");
        return nullptr;
    }
    const bool real = dtype == OPENFFT_R2C_F64 || dtype == OPENFFT_R2C_F32;
    // the complex arrays of a real plan are the half arrays (c extent Nc / 2 + 1)
    const int Ncx = real ? Nc / 2 + 1 : Nc;
    if (Nc < 1 || validate_dims(Na, Nb, Ncx, P)) {
        if (Nc < 1) fail(OPENFFT_ERR_INVALID_ARG, "sizes and P must be >= 1");
        return nullptr;
    }
    const bool c64 = dtype != OPENFFT_C2C_F64 && dtype != OPENFFT_R2C_F64;   // complex64 data
    openfft_plan_s* p = new openfft_plan_s();
    p->Na = Na; p->Nb = Nb; p->Nc = Nc; p->P = P; p->dtype = dtype;
    p->real = real; p->Ncx = Ncx;
    p->N = (int64_t)Na * Nb * Nc;
    const int lens[3] = {Na, Nb, Nc};
    for (int ax = 0; ax < 3; ++ax)
        if (!radix_plan(lens[ax], p->rad[ax]) || lens[ax] > kMaxLen) {
            fail(OPENFFT_ERR_UNSUPPORTED_RADIX, "axis length must factor into 2, 3, 5, 7 and be <= 2048");
            delete p;
            return nullptr;
        }
    cudaError_t e;
    if ((e = cudaGetDevice(&p->device))) { cuda_fail(e, "cudaGetDevice"); delete p; return nullptr; }
    cudaDeviceGetAttribute(&p->sms, cudaDevAttrMultiProcessorCount, p->device);
    if ((e = stage_kernels_init(200 * 1024))) { cuda_fail(e, "kernel attributes"); delete p; return nullptr; }
    p->elem_bytes = c64 ? 8 : 16;
    const size_t bytes = (size_t)p->N * p->elem_bytes;
    if (dev_malloc((void**)&p->bufA, bytes) || dev_malloc((void**)&p->bufB, bytes)) {
        cudaGetLastError();
        fail(OPENFFT_ERR_NOMEM, "workspace allocation failed");
        free_plan(p);
        return nullptr;
    }
    // twiddle tables (FP64 sincospi on the device)
    for (int ax = 0; ax < 3; ++ax) {
        const int fmts[2] = {c64 ? FMT_C64 : FMT_C128, c64 ? -1 : FMT_DF};
        for (int f : fmts) {
            if (f < 0) continue;
            if (dev_malloc((void**)&p->tw[ax][f], twiddle_bytes(lens[ax], f))) {
                cudaGetLastError();
                fail(OPENFFT_ERR_NOMEM, "twiddle allocation failed");
                free_plan(p);
                return nullptr;
            }
            if ((e = launch_twiddles(lens[ax], f, p->tw[ax][f], nullptr))) { cuda_fail(e, "twiddles"); free_plan(p); return nullptr; }
        }
    }
    // operand images of the DFT-GEMM stages (split dtypes; an axis that does
    // not factor keeps none and the plan is refused when its stages are built)
    if (dtype == OPENFFT_C2C_SPLIT_TF32 || dtype == OPENFFT_C2C_SPLIT_BF16) {
        const bool tf32 = dtype == OPENFFT_C2C_SPLIT_TF32;
        for (int ax = 0; ax < 3; ++ax) {
            int R = 0, S = 0;
            if (!dftgemm_factor(lens[ax], tf32, &R, &S)) continue;
            if (dev_malloc((void**)&p->bimg[ax], dftgemm_image_bytes(lens[ax], R, S, tf32))) {
                cudaGetLastError();
                fail(OPENFFT_ERR_NOMEM, "operand image allocation failed");
                free_plan(p);
                return nullptr;
            }
            if ((e = launch_dftgemm_image(lens[ax], R, S, tf32, p->tw[ax][FMT_C64], p->bimg[ax], nullptr))) {
                cuda_fail(e, "operand image"); free_plan(p); return nullptr;
            }
        }
    }
    // transpose tables for the explicit variants
    const int whichs[4] = {1, 2, -2, -1};
    for (int i = 0; i < 4; ++i) {
        TransposeTables& T = p->tt[i];
        T.t = make_transpose(whichs[i], Na, Nb, Ncx, P);
        std::vector<int64_t> sb, rb, ch, sd, rd;
        build_transpose_tables(T.t, T.C, sb, rb, ch, 8192, &sd, &rd);
        T.nchunks = (int64_t)ch.size() / 3;
        const size_t pp = sb.size() * sizeof(int64_t);
        if (dev_malloc((void**)&T.d_sbase, pp) || dev_malloc((void**)&T.d_rbase, pp) ||
            dev_malloc((void**)&T.d_chunks, ch.size() * sizeof(int64_t) + 8) ||
            dev_malloc((void**)&T.d_C, pp) || dev_malloc((void**)&T.d_sdispl, pp) || dev_malloc((void**)&T.d_rdispl, pp)) {
            cudaGetLastError();
            fail(OPENFFT_ERR_NOMEM, "transpose table allocation failed");
            free_plan(p);
            return nullptr;
        }
        cudaMemcpy(T.d_sbase, sb.data(), pp, cudaMemcpyHostToDevice);
        cudaMemcpy(T.d_rbase, rb.data(), pp, cudaMemcpyHostToDevice);
        if (!ch.empty()) cudaMemcpy(T.d_chunks, ch.data(), ch.size() * sizeof(int64_t), cudaMemcpyHostToDevice);
        cudaMemcpy(T.d_C, T.C.data(), pp, cudaMemcpyHostToDevice);
        cudaMemcpy(T.d_sdispl, sd.data(), pp, cudaMemcpyHostToDevice);
        cudaMemcpy(T.d_rdispl, rd.data(), pp, cudaMemcpyHostToDevice);
    }
    if (dev_malloc((void**)&p->d_status, sizeof(int)) || cudaMemset(p->d_status, 0, sizeof(int))) {
        cudaGetLastError();
        fail(OPENFFT_ERR_NOMEM, "status word");
        free_plan(p);
        return nullptr;
    }
    if ((e = cudaDeviceSynchronize())) { cuda_fail(e, "plan setup"); free_plan(p); return nullptr; }
    // candidates (Sec. 3.2.3: the set the tuner chooses from).  The fused
    // variant is tried with every stage-kernel family and tile width; the six
    // explicit pack / communicate / unpack methods of Sec. 3.2.1 with the
    // default kernel.  The first candidate is the default.
    {
        std::vector<int> ariths;
        if (dtype == OPENFFT_C2C_F32 || dtype == OPENFFT_R2C_F32) ariths = {ARITH_F32};
        else if (dtype == OPENFFT_C2C_SPLIT_TF32) ariths = {ARITH_TC_TF32};
        else if (dtype == OPENFFT_C2C_SPLIT_BF16) ariths = {ARITH_TC_BF16};
        else ariths = {ARITH_DF, ARITH_F64};
        const bool f32 = c64;
        const int gw = f32 ? 16 : 8, gn = f32 ? 8 : 4;
        for (int ar : ariths) {
            if (real) {                    // real plans: the fused variant with every kernel family
                p->cands.push_back(Candidate{OPENFFT_VARIANT_FUSED, ar, gw, KERNEL_AUTO});
                p->cands.push_back(Candidate{OPENFFT_VARIANT_FUSED, ar, gn, KERNEL_AUTO});
                p->cands.push_back(Candidate{OPENFFT_VARIANT_FUSED, ar, gw, KERNEL_TILE});
                p->cands.push_back(Candidate{OPENFFT_VARIANT_FUSED, ar, gn, KERNEL_TILE});
                p->cands.push_back(Candidate{OPENFFT_VARIANT_FUSED, ar, gw, KERNEL_GENERIC});
                continue;
            }
            if (is_tc(ar)) {               // the DFT-GEMM form: fused stores only, tiles of 8 / 16 / 4 lines
                for (int g : {8, 16, 4}) p->cands.push_back(Candidate{OPENFFT_VARIANT_FUSED, ar, g, KERNEL_AUTO});
                continue;
            }
            p->cands.push_back(Candidate{OPENFFT_VARIANT_FUSED, ar, gw, KERNEL_AUTO});
            p->cands.push_back(Candidate{OPENFFT_VARIANT_FUSED, ar, gn, KERNEL_AUTO});
            p->cands.push_back(Candidate{OPENFFT_VARIANT_FUSED, ar, gw, KERNEL_TILE});
            p->cands.push_back(Candidate{OPENFFT_VARIANT_FUSED, ar, gn, KERNEL_TILE});
            p->cands.push_back(Candidate{OPENFFT_VARIANT_FUSED, ar, gw, KERNEL_GENERIC});
            p->cands.push_back(Candidate{OPENFFT_VARIANT_PACK_UNPACK, ar, gw, KERNEL_AUTO});
            p->cands.push_back(Candidate{OPENFFT_VARIANT_PACK_EXCHANGE_UNPACK, ar, gw, KERNEL_AUTO});
            p->cands.push_back(Candidate{OPENFFT_VARIANT_ISEND_WAITALL, ar, gw, KERNEL_AUTO});
            p->cands.push_back(Candidate{OPENFFT_VARIANT_ISEND_WAITALL_BLOCK, ar, gw, KERNEL_AUTO});
            p->cands.push_back(Candidate{OPENFFT_VARIANT_ISEND_WAITSOME_BLOCK, ar, gw, KERNEL_AUTO});
            p->cands.push_back(Candidate{OPENFFT_VARIANT_SENDRECV, ar, gw, KERNEL_AUTO});
        }
    }
    if (select_candidate(p, 0)) { free_plan(p); return nullptr; }
    return p;
}

void openfft_destroy(openfft_plan_t plan)
{
    if (!plan) return;
    cudaStreamSynchronize(plan->stream);
    free_plan(plan);
}

int openfft_set_stream(openfft_plan_t plan, void* stream)
{
    if (!plan) return fail(OPENFFT_ERR_INVALID_ARG, "null plan");
    plan->stream = (cudaStream_t)stream;
    return OPENFFT_OK;
}

int openfft_exec_c2c(openfft_plan_t plan, const void* in, void* out, int dir)
{
    if (!plan || !in || !out) return fail(OPENFFT_ERR_INVALID_ARG, "null plan or buffer");
    if (plan->batch) return fail(OPENFFT_ERR_INVALID_ARG, "batched plan: use openfft_exec_many");
    if (plan->real) return fail(OPENFFT_ERR_INVALID_ARG, "real plan: use openfft_exec_r2c / openfft_exec_c2r");
    if (in == out) return fail(OPENFFT_ERR_ALIAS, "in and out must differ (out-of-place only)");
    if (dir != OPENFFT_FORWARD && dir != OPENFFT_BACKWARD) return fail(OPENFFT_ERR_INVALID_ARG, "dir must be -1 or +1");
    const Candidate& c = plan->cands[(size_t)plan->current];
    return run_ops(plan, dir == OPENFFT_FORWARD ? plan->ops_fwd : plan->ops_bwd, in, out, c.arith);
}

int openfft_exec_r2c(openfft_plan_t plan, const void* in, void* out)
{
    if (!plan || !in || !out) return fail(OPENFFT_ERR_INVALID_ARG, "null plan or buffer");
    if (!plan->real) return fail(OPENFFT_ERR_INVALID_ARG, "not a real plan (OPENFFT_R2C_*)");
    if (in == out) return fail(OPENFFT_ERR_ALIAS, "in and out must differ (out-of-place only)");
    const Candidate& c = plan->cands[(size_t)plan->current];
    return run_ops(plan, plan->ops_fwd, in, out, c.arith);
}

int openfft_exec_c2r(openfft_plan_t plan, const void* in, void* out)
{
    if (!plan || !in || !out) return fail(OPENFFT_ERR_INVALID_ARG, "null plan or buffer");
    if (!plan->real) return fail(OPENFFT_ERR_INVALID_ARG, "not a real plan (OPENFFT_R2C_*)");
    if (in == out) return fail(OPENFFT_ERR_ALIAS, "in and out must differ (out-of-place only)");
    const Candidate& c = plan->cands[(size_t)plan->current];
    return run_ops(plan, plan->ops_bwd, in, out, c.arith);
}

namespace {

// The streams of host-exec copies: the caller's, or plan-owned ones created
// on first use (with the plan's copy events).
cudaStream_t h2d_stream(const openfft_plan_s* p) { return p->user_copy_streams ? p->user_h2d : p->own_h2d; }
cudaStream_t d2h_stream(const openfft_plan_s* p) { return p->user_copy_streams ? p->user_d2h : p->own_d2h; }

cudaError_t ensure_copy_streams(openfft_plan_s* p)
{
    cudaError_t e;
    if (!p->host_ev[0])
        for (cudaEvent_t& ev : p->host_ev)
            if ((e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming))) return e;
    if (p->user_copy_streams) return cudaSuccess;
    if (!p->own_h2d && (e = cudaStreamCreateWithFlags(&p->own_h2d, cudaStreamNonBlocking))) return e;
    if (!p->own_d2h && (e = cudaStreamCreateWithFlags(&p->own_d2h, cudaStreamNonBlocking))) return e;
    return cudaSuccess;
}

int fmt_bytes(int fmt)
{
    return fmt == FMT_C64 || fmt == FMT_R64 ? 8 : (fmt == FMT_R32 ? 4 : 16);
}

// A stage launch restricted to the lines whose coordinate u lies in [u0, u1):
// u = i2 when M2 > 1, else u = i1 (then i2 = 0 and M1 plays no part in the
// addresses).  The restricted launch reads from in + *in_off and writes to
// out + *out_off (elements); *lines is its number of lines, which are
// contiguous in the input.
StageLaunch stage_lines(const StageLaunch& L, int64_t u0, int64_t u1, int64_t* in_off, int64_t* out_off,
                        int64_t* lines)
{
    StageLaunch c = L;
    StageArgs& a = c.args;
    const int64_t whole = a.M1 * a.M2 * (int64_t)a.n;
    if (a.M2 > 1) {
        *in_off = u0 * a.M1 * a.n; *out_off = u0 * a.S2; *lines = (u1 - u0) * a.M1;
        a.M2 = u1 - u0;
    } else {
        *in_off = u0 * a.n; *out_off = u0 * a.S1; *lines = u1 - u0;
        a.M1 = u1 - u0;
    }
    const int64_t Mg = a.group_i2 ? a.M2 : a.M1;
    a.ngroups = (Mg + a.G - 1) / a.G;
    a.in_elems = (a.in_elems ? a.in_elems : whole) - *in_off;
    a.out_elems = (a.out_elems ? a.out_elems : whole) - *out_off;
    c.grid = a.ngroups * (a.group_i2 ? a.M1 : a.M2);
    return c;
}

// Boundaries of k line ranges of a stage: multiples of G when the split
// coordinate is the one that tiles group, so tiles stay whole.
std::vector<int64_t> line_ranges(const StageArgs& a, int k)
{
    const int64_t U = a.M2 > 1 ? a.M2 : a.M1;
    const int64_t q = ((a.M2 > 1) == (a.group_i2 != 0)) ? a.G : 1;
    std::vector<int64_t> b{0};
    for (int i = 1; i < k; ++i) {
        const int64_t u = U * i / k / q * q;
        if (u > b.back() && u < U) b.push_back(u);
    }
    b.push_back(U);
    return b;
}

// The first op can start on each range as soon as its input has arrived: a
// stage reading the user input whose lines cover the whole array.
bool splits_input(const openfft_plan_s* p, const Op& o)
{
    return o.kind == OP_STAGE && o.src == B_IN && o.stage.family != KERNEL_R2C &&
           o.stage.args.M1 * o.stage.args.M2 * o.stage.args.n == p->N;
}

// The last op's ranges can leave as soon as they are written: a stage writing
// the user output line by line (contiguous lines of n elements).
bool splits_output(const openfft_plan_s* p, const Op& o)
{
    const StageArgs& a = o.stage.args;
    return o.kind == OP_STAGE && o.dst == B_OUT && o.stage.family != KERNEL_C2R && a.contig_store &&
           a.Sk == 1 && a.S1 == a.n && (a.M2 == 1 || a.S2 == a.M1 * a.n) && a.M1 * a.M2 * a.n == p->N;
}

int host_ranges(const openfft_plan_s* p, size_t bytes)
{
    if (p->host_chunks > 0) return std::min(p->host_chunks, kMaxHostChunks);
    const size_t per = (size_t)8 << 20;        // ranges of at least 8 MiB
    return (int)std::max<size_t>(1, std::min<size_t>(16, bytes / per));
}

}  // namespace

int openfft_set_host_chunks(openfft_plan_t plan, int chunks)
{
    if (!plan) return fail(OPENFFT_ERR_INVALID_ARG, "null plan");
    if (chunks < 0 || chunks > kMaxHostChunks) return fail(OPENFFT_ERR_INVALID_ARG, "chunks must be 0..32");
    plan->host_chunks = chunks;
    return OPENFFT_OK;
}

namespace {
int exec_host(openfft_plan_t plan, const void* host_in, void* host_out, int dir, bool wait);
}

int openfft_set_copy_streams(openfft_plan_t plan, void* h2d, void* d2h)
{
    if (!plan) return fail(OPENFFT_ERR_INVALID_ARG, "null plan");
    if ((h2d == nullptr) != (d2h == nullptr))
        return fail(OPENFFT_ERR_INVALID_ARG, "give both copy streams, or neither for the plan's own");
    // copies already queued on the streams being replaced finish first
    cudaError_t e;
    if (plan->user_copy_streams &&
        ((e = cudaStreamSynchronize(plan->user_h2d)) || (e = cudaStreamSynchronize(plan->user_d2h))))
        return cuda_fail(e, "copy stream synchronize");
    if ((plan->own_h2d && (e = cudaStreamSynchronize(plan->own_h2d))) ||
        (plan->own_d2h && (e = cudaStreamSynchronize(plan->own_d2h))))
        return cuda_fail(e, "copy stream synchronize");
    plan->user_copy_streams = h2d != nullptr;
    plan->user_h2d = (cudaStream_t)h2d;
    plan->user_d2h = (cudaStream_t)d2h;
    return OPENFFT_OK;
}

int openfft_exec_c2c_host(openfft_plan_t plan, const void* host_in, void* host_out, int dir)
{
    return exec_host(plan, host_in, host_out, dir, true);
}

int openfft_exec_c2c_host_async(openfft_plan_t plan, const void* host_in, void* host_out, int dir)
{
    return exec_host(plan, host_in, host_out, dir, false);
}

namespace {

// Host-buffer execution; with `wait` false it returns once everything is
// enqueued (openfft_sync waits for the copies as well).
int exec_host(openfft_plan_t plan, const void* host_in, void* host_out, int dir, bool wait)
{
    if (!plan || !host_in || !host_out) return fail(OPENFFT_ERR_INVALID_ARG, "null plan or buffer");
    if (plan->batch) return fail(OPENFFT_ERR_INVALID_ARG, "batched plan: use openfft_exec_many");
    if (plan->real) return fail(OPENFFT_ERR_INVALID_ARG, "real plan: use openfft_exec_r2c / openfft_exec_c2r");
    if (dir != OPENFFT_FORWARD && dir != OPENFFT_BACKWARD) return fail(OPENFFT_ERR_INVALID_ARG, "dir must be -1 or +1");
    const size_t bytes = (size_t)plan->N * plan->elem_bytes;
    if (!plan->stage_in) {
        if (dev_malloc((void**)&plan->stage_in, bytes) || dev_malloc((void**)&plan->stage_out, bytes)) {
            cudaGetLastError();
            cudaFree(plan->stage_in); plan->stage_in = nullptr;
            return fail(OPENFFT_ERR_NOMEM, "staging allocation failed");
        }
    }
    const std::vector<Op>& ops = dir == OPENFFT_FORWARD ? plan->ops_fwd : plan->ops_bwd;
    const int arith = plan->cands[(size_t)plan->current].arith;
    cudaError_t e;
    if ((e = ensure_copy_streams(plan))) return cuda_fail(e, "copy streams");
    cudaEvent_t ev_read = plan->host_ev[2 * kMaxHostChunks];          // stage 1 has read the staging input
    cudaEvent_t ev_sent = plan->host_ev[2 * kMaxHostChunks + 1];      // the download of the staging output is done
    if (plan->timing || ops.size() < 3) {
        // one copy each way around the whole transform, on the plan's stream
        // (the phase timer brackets whole ops)
        cudaStream_t st = plan->stream;
        if ((e = cudaStreamWaitEvent(st, ev_sent, 0)) ||
            (e = cudaMemcpyAsync(plan->stage_in, host_in, bytes, cudaMemcpyHostToDevice, st))) return cuda_fail(e, "H2D");
        int status = run_ops(plan, ops, plan->stage_in, plan->stage_out, arith);
        if (status) return status;
        if ((e = cudaMemcpyAsync(host_out, plan->stage_out, bytes, cudaMemcpyDeviceToHost, st)) ||
            (e = cudaEventRecord(ev_read, st)) || (e = cudaEventRecord(ev_sent, st)))
            return cuda_fail(e, "D2H");
        if (wait && (e = cudaStreamSynchronize(st))) return cuda_fail(e, "sync");
        return OPENFFT_OK;
    }
    // Uploads and downloads run on their own streams, range by range: the
    // first stage starts on each range of lines as soon as it has arrived, and
    // each range of the last stage's output leaves as soon as it is written.
    cudaStream_t st = plan->stream, hs = h2d_stream(plan), ds = d2h_stream(plan);
    cudaEvent_t* ev_in = plan->host_ev;
    cudaEvent_t* ev_out = plan->host_ev + kMaxHostChunks;
    const int k = host_ranges(plan, bytes);
    const char* hin = static_cast<const char*>(host_in);
    char* hout = static_cast<char*>(host_out);
    char* din = static_cast<char*>(plan->stage_in);
    char* dout = static_cast<char*>(plan->stage_out);
    // Across calls on this plan, which run in order: the upload waits until
    // the previous call's download is done (that also covers its first stage
    // reading the staging input, and a host buffer this call reads that the
    // previous call writes).  This call's work on the plan's stream, which
    // writes the staging output, waits for that download as well.  Events
    // never recorded make these waits no-ops.  Calls on other plans are not
    // ordered against this one: with shared copy streams, one plan's upload
    // can run beside another's download.
    if ((e = cudaStreamWaitEvent(hs, ev_read, 0)) || (e = cudaStreamWaitEvent(hs, ev_sent, 0)) ||
        (e = cudaStreamWaitEvent(st, ev_sent, 0)))
        return cuda_fail(e, "copy order");
    const Op& first = ops.front();
    const Op& last = ops.back();
    size_t i0 = 0, i1 = ops.size();
    if (splits_input(plan, first)) {
        const StageArgs& a = first.stage.args;
        const std::vector<int64_t> b = line_ranges(a, k);
        const int Ein = fmt_bytes(a.in_fmt), Eout = fmt_bytes(a.out_fmt);
        for (size_t j = 0; j + 1 < b.size(); ++j) {
            int64_t io, oo, lines;
            stage_lines(first.stage, b[j], b[j + 1], &io, &oo, &lines);
            if ((e = cudaMemcpyAsync(din + io * Ein, hin + io * Ein, (size_t)(lines * a.n * Ein), cudaMemcpyHostToDevice, hs)) ||
                (e = cudaEventRecord(ev_in[j], hs)))
                return cuda_fail(e, "H2D");
        }
        char* d = static_cast<char*>(resolve(plan, first.dst, din, dout));
        for (size_t j = 0; j + 1 < b.size(); ++j) {
            int64_t io, oo, lines;
            StageLaunch L = stage_lines(first.stage, b[j], b[j + 1], &io, &oo, &lines);
            L.args.in = din + io * Ein;
            L.args.out = d + oo * Eout;
            if ((e = cudaStreamWaitEvent(st, ev_in[j], 0)) || (e = launch_stage(L, st))) return cuda_fail(e, "first stage");
        }
        if ((e = cudaEventRecord(ev_read, st))) return cuda_fail(e, "copy order");
        i0 = 1;
    } else {
        if ((e = cudaMemcpyAsync(din, hin, bytes, cudaMemcpyHostToDevice, hs)) || (e = cudaEventRecord(ev_in[0], hs)) ||
            (e = cudaStreamWaitEvent(st, ev_in[0], 0)))
            return cuda_fail(e, "H2D");
    }
    const bool split_out = splits_output(plan, last);
    if (split_out) i1 = ops.size() - 1;
    int status = run_ops(plan, ops, din, dout, arith, i0, i1);
    if (status) return status;
    if (i0 == 0 && (e = cudaEventRecord(ev_read, st))) return cuda_fail(e, "copy order");
    if (split_out) {
        const StageArgs& a = last.stage.args;
        const std::vector<int64_t> b = line_ranges(a, k);
        const int Ein = fmt_bytes(a.in_fmt), Eout = fmt_bytes(a.out_fmt);
        const char* s = static_cast<const char*>(resolve(plan, last.src, din, dout));
        for (size_t j = 0; j + 1 < b.size(); ++j) {
            int64_t io, oo, lines;
            StageLaunch L = stage_lines(last.stage, b[j], b[j + 1], &io, &oo, &lines);
            L.args.in = s + io * Ein;
            L.args.out = dout + oo * Eout;
            if ((e = launch_stage(L, st)) || (e = cudaEventRecord(ev_out[j], st)) || (e = cudaStreamWaitEvent(ds, ev_out[j], 0)) ||
                (e = cudaMemcpyAsync(hout + oo * Eout, dout + oo * Eout, (size_t)(lines * a.n * Eout), cudaMemcpyDeviceToHost, ds)))
                return cuda_fail(e, "last stage");
        }
    } else {
        if ((e = cudaEventRecord(ev_out[0], st)) || (e = cudaStreamWaitEvent(ds, ev_out[0], 0)) ||
            (e = cudaMemcpyAsync(hout, dout, bytes, cudaMemcpyDeviceToHost, ds)))
            return cuda_fail(e, "D2H");
    }
    if ((e = cudaEventRecord(ev_sent, ds))) return cuda_fail(e, "copy order");
    if (!wait) return OPENFFT_OK;
    if ((e = cudaStreamSynchronize(ds))) return cuda_fail(e, "sync");
    if ((e = cudaStreamSynchronize(st))) return cuda_fail(e, "sync");
    return OPENFFT_OK;
}

}  // namespace

int openfft_sync(openfft_plan_t plan)
{
    if (!plan) return fail(OPENFFT_ERR_INVALID_ARG, "null plan");
    if (plan->batch) {
        cudaError_t e = cudaStreamSynchronize(plan->stream);
        if (e) return cuda_fail(e, "stream synchronize");
        return batch_status(plan->batch, &fail_cstr);
    }
    cudaError_t e;
    cudaStream_t hs = h2d_stream(plan), ds = d2h_stream(plan);
    if ((hs && (e = cudaStreamSynchronize(hs))) || (ds && (e = cudaStreamSynchronize(ds))))
        return cuda_fail(e, "copy stream synchronize");
    if ((e = cudaStreamSynchronize(plan->stream))) return cuda_fail(e, "stream synchronize");
    int st = 0;
    if (plan->d_status) {
        if ((e = cudaMemcpy(&st, plan->d_status, sizeof(int), cudaMemcpyDeviceToHost))) return cuda_fail(e, "status word");
        if (st) {
            cudaMemset(plan->d_status, 0, sizeof(int));
            return fail(st, st == OPENFFT_ERR_BOUNDS ? "a global index outside its array (checked build)"
                                                     : "a bounded tensor-core completion wait ran out");
        }
    }
    return OPENFFT_OK;
}

int openfft_box(openfft_plan_t plan, int which, int rank, int64_t start[3], int64_t end[3],
                int64_t* offset, int64_t* count)
{
    if (!plan) return fail(OPENFFT_ERR_INVALID_ARG, "null plan");
    if (which != 0 && which != 1) return fail(OPENFFT_ERR_INVALID_ARG, "which must be 0 (abc) or 1 (cba)");
    // real plans: the input box is in the real abc array, the output box in
    // the cba half array (c extent Nc / 2 + 1)
    return box_of(ordering_of(which == 0 ? ABC : CBA, plan->Na, plan->Nb, which == 0 ? plan->Nc : plan->Ncx, plan->P),
                  rank, start, end, offset, count);
}

int openfft_counts(openfft_plan_t plan, int exchange, int64_t* PxP)
{
    if (!plan || !PxP) return fail(OPENFFT_ERR_INVALID_ARG, "null plan or output");
    if (exchange != 1 && exchange != 2 && exchange != -1 && exchange != -2)
        return fail(OPENFFT_ERR_INVALID_ARG, "exchange must be 1, 2, -2 or -1");
    const std::vector<int64_t>& C = plan->tt[tix_of(exchange)].C;
    std::memcpy(PxP, C.data(), C.size() * sizeof(int64_t));
    return OPENFFT_OK;
}

int openfft_num_candidates(openfft_plan_t plan) { return plan ? (int)plan->cands.size() : 0; }

int openfft_candidate(openfft_plan_t plan, int index, int* variant, int* arith, int* lines_per_cta, int* kernel)
{
    if (!plan || index < 0 || index >= (int)plan->cands.size()) return fail(OPENFFT_ERR_INVALID_ARG, "bad candidate");
    const Candidate& c = plan->cands[(size_t)index];
    if (variant) *variant = c.variant;
    if (arith) *arith = c.arith == ARITH_DF ? (int)OPENFFT_ARITH_DOUBLE_FLOAT
                      : (c.arith == ARITH_TC_TF32 ? (int)OPENFFT_ARITH_TC_TF32
                      : (c.arith == ARITH_TC_BF16 ? (int)OPENFFT_ARITH_TC_BF16 : (int)OPENFFT_ARITH_NATIVE));
    if (lines_per_cta) *lines_per_cta = c.G;
    if (kernel) *kernel = c.family;
    return OPENFFT_OK;
}

int openfft_current_candidate(openfft_plan_t plan) { return plan ? plan->current : -1; }

}  // extern "C"

// ------------------------------------------------ persisted tuning choices --
// The candidate each tuned problem chose, described as openfft_candidate
// describes it, per (Na, Nb, Nc, P, dtype): the paper's "User-select" reuse of
// an earlier tuning (Sec. 3.2.3).  Process-wide; saved to and merged from
// text files.
namespace {

using TunedKey = std::array<int, 5>;
using TunedChoice = std::array<int, 4>;
std::mutex g_tuned_mu;
std::map<TunedKey, TunedChoice> g_tuned;

TunedKey tuned_key(const openfft_plan_s* p) { return TunedKey{p->Na, p->Nb, p->Nc, p->P, p->dtype}; }

TunedChoice describe_candidate(openfft_plan_s* p, int index)
{
    TunedChoice c{};
    openfft_candidate(p, index, &c[0], &c[1], &c[2], &c[3]);
    return c;
}

void record_choice(openfft_plan_s* p)
{
    const TunedChoice c = describe_candidate(p, p->current);
    std::lock_guard<std::mutex> lk(g_tuned_mu);
    g_tuned[tuned_key(p)] = c;
}

// index of the recorded candidate of p's problem, -1 if none
int saved_candidate(openfft_plan_s* p)
{
    TunedChoice want;
    {
        std::lock_guard<std::mutex> lk(g_tuned_mu);
        auto it = g_tuned.find(tuned_key(p));
        if (it == g_tuned.end()) return -1;
        want = it->second;
    }
    for (int i = 0; i < (int)p->cands.size(); ++i)
        if (describe_candidate(p, i) == want) return i;
    return -1;
}

bool valid_dtype(int dtype)
{
    return dtype == OPENFFT_C2C_F64 || dtype == OPENFFT_C2C_F32 || dtype == OPENFFT_C2C_SPLIT_BF16 ||
           dtype == OPENFFT_C2C_SPLIT_TF32 || dtype == OPENFFT_R2C_F64 || dtype == OPENFFT_R2C_F32;
}

}  // namespace

extern "C" {

int openfft_tuning_save(const char* path)
{
    if (!path) return fail(OPENFFT_ERR_INVALID_ARG, "null path");
    std::map<TunedKey, TunedChoice> copy;
    {
        std::lock_guard<std::mutex> lk(g_tuned_mu);
        copy = g_tuned;
    }
    FILE* f = std::fopen(path, "w");
    if (!f) return fail(OPENFFT_ERR_INVALID_ARG, (std::string("cannot write ") + path).c_str());
    bool ok = std::fprintf(f, "# openfft tuning choices: Na Nb Nc P dtype variant arith lines_per_cta kernel\n") > 0;
    for (const auto& e : copy)
        ok = ok && std::fprintf(f, "%d %d %d %d %d %d %d %d %d\n", e.first[0], e.first[1], e.first[2], e.first[3],
                                e.first[4], e.second[0], e.second[1], e.second[2], e.second[3]) > 0;
    ok = (std::fclose(f) == 0) && ok;
    return ok ? OPENFFT_OK : fail(OPENFFT_ERR_INVALID_ARG, (std::string("cannot write ") + path).c_str());
}

int openfft_tuning_load(const char* path)
{
    if (!path) return fail(OPENFFT_ERR_INVALID_ARG, "null path");
    FILE* f = std::fopen(path, "r");
    if (!f) return fail(OPENFFT_ERR_INVALID_ARG, (std::string("cannot read ") + path).c_str());
    std::map<TunedKey, TunedChoice> add;
    char line[512];
    int lineno = 0;
    while (std::fgets(line, sizeof line, f)) {
        ++lineno;
        const char* s = line;
        while (*s == ' ' || *s == '\t') ++s;
        if (*s == '#' || *s == '\n' || *s == '\r' || *s == '\0') continue;
        int v[9], used = 0;
        const int n = std::sscanf(s, "%d %d %d %d %d %d %d %d %d %n", &v[0], &v[1], &v[2], &v[3], &v[4], &v[5], &v[6],
                                  &v[7], &v[8], &used);
        const bool rest_empty = n == 9 && s[used] == '\0';
        if (n != 9 || !rest_empty || v[0] < 1 || v[1] < 1 || v[2] < 1 || v[3] < 1 || !valid_dtype(v[4])) {
            std::fclose(f);
            return fail(OPENFFT_ERR_INVALID_ARG, (std::string(path) + ": malformed line " + std::to_string(lineno)).c_str());
        }
        add[TunedKey{v[0], v[1], v[2], v[3], v[4]}] = TunedChoice{v[5], v[6], v[7], v[8]};
    }
    std::fclose(f);
    std::lock_guard<std::mutex> lk(g_tuned_mu);
    for (const auto& e : add) g_tuned[e.first] = e.second;
    return OPENFFT_OK;
}

int openfft_tuning_lookup(int Na, int Nb, int Nc, int P, int dtype, int* found, int choice[4])
{
    if (!found) return fail(OPENFFT_ERR_INVALID_ARG, "null output");
    std::lock_guard<std::mutex> lk(g_tuned_mu);
    auto it = g_tuned.find(TunedKey{Na, Nb, Nc, P, dtype});
    *found = it != g_tuned.end();
    if (*found && choice)
        for (int i = 0; i < 4; ++i) choice[i] = it->second[(size_t)i];
    return OPENFFT_OK;
}

int openfft_tuning_clear(void)
{
    std::lock_guard<std::mutex> lk(g_tuned_mu);
    g_tuned.clear();
    return OPENFFT_OK;
}

int openfft_set_tuning(openfft_plan_t plan, int mode, int candidate)
{
    if (!plan) return fail(OPENFFT_ERR_INVALID_ARG, "null plan");
    if (plan->batch) return fail(OPENFFT_ERR_INVALID_ARG, "batched plans have a single execution path");
    switch (mode) {
    case OPENFFT_TUNE_SAVED: {
        const int idx = saved_candidate(plan);
        if (idx >= 0 && select_candidate(plan, idx) == OPENFFT_OK) return OPENFFT_OK;
        return openfft_set_tuning(plan, OPENFFT_TUNE_EXHAUSTIVE, 0);
    }
    case OPENFFT_TUNE_DEFAULT:
        return select_candidate(plan, 0);
    case OPENFFT_TUNE_USER:
        return select_candidate(plan, candidate);
    case OPENFFT_TUNE_EXHAUSTIVE: {
        std::vector<float> ms;
        int st = time_candidates(plan, ms);
        if (st) return st;
        int best = -1;
        for (int i = 0; i < (int)ms.size(); ++i)
            if (ms[(size_t)i] >= 0.f && (best < 0 || ms[(size_t)i] < ms[(size_t)best])) best = i;
        if (best < 0) return fail(OPENFFT_ERR_UNSUPPORTED, "no candidate ran");
        const int sel = select_candidate(plan, best);
        if (!sel) record_choice(plan);
        return sel;
    }
    case OPENFFT_TUNE_LEARNED: {
        std::vector<float> model;
        int d, h, k;
        {
            std::lock_guard<std::mutex> lk(g_model_mu);
            model = g_model; d = g_model_d; h = g_model_h; k = g_model_k;
        }
        if (model.empty()) return select_candidate(plan, 0);          // no model: the default
        const int nc = (int)plan->cands.size();
        std::vector<float> X((size_t)nc * kFeatures), y((size_t)nc, 0.f), yk((size_t)nc);
        for (int i = 0; i < nc; ++i) candidate_features(plan, plan->cands[(size_t)i], &X[(size_t)i * kFeatures]);
        const size_t np = (size_t)openfft_mlp_num_params(d, h);
        for (int m = 0; m < k; ++m) {                                   // mean prediction of the ensemble
            int st = openfft_mlp_predict(d, h, model.data() + (size_t)m * np, X.data(), nc, yk.data());
            if (st) return st;
            for (int i = 0; i < nc; ++i) y[(size_t)i] += yk[(size_t)i] / (float)k;
        }
        // lowest predicted time; a candidate that cannot be built falls back to the next
        std::vector<int> order((size_t)nc);
        for (int i = 0; i < nc; ++i) order[(size_t)i] = i;
        std::sort(order.begin(), order.end(), [&](int a2, int b2) { return y[(size_t)a2] < y[(size_t)b2]; });
        for (int i : order)
            if (!select_candidate(plan, i)) {
                record_choice(plan);
                return OPENFFT_OK;
            }
        return fail(OPENFFT_ERR_UNSUPPORTED, "no candidate can be built");
    }
    default:
        return fail(OPENFFT_ERR_INVALID_ARG, "unknown tuning mode");
    }
}

int openfft_num_features(void) { return kFeatures; }

int openfft_candidate_features(openfft_plan_t plan, int index, float* features)
{
    if (!plan || plan->batch || !features || index < 0 || index >= (int)plan->cands.size())
        return fail(OPENFFT_ERR_INVALID_ARG, "bad plan, candidate or output");
    candidate_features(plan, plan->cands[(size_t)index], features);
    return OPENFFT_OK;
}

int openfft_tune_times(openfft_plan_t plan, float* ms)
{
    if (!plan || plan->batch || !ms) return fail(OPENFFT_ERR_INVALID_ARG, "bad plan or output");
    std::vector<float> t;
    int st = time_candidates(plan, t);
    if (st) return st;
    std::memcpy(ms, t.data(), t.size() * sizeof(float));
    return OPENFFT_OK;
}

int openfft_set_cost_model(int count, int d, int hidden, const float* params)
{
    std::lock_guard<std::mutex> lk(g_model_mu);
    if (!params || count == 0) { g_model.clear(); g_model_d = g_model_h = g_model_k = 0; return OPENFFT_OK; }
    if (count < 1 || d != kFeatures || hidden < 1 || hidden > 256)
        return fail(OPENFFT_ERR_INVALID_ARG, "count >= 1 and d == openfft_num_features() required");
    g_model.assign(params, params + (size_t)count * openfft_mlp_num_params(d, hidden));
    g_model_d = d; g_model_h = hidden; g_model_k = count;
    return OPENFFT_OK;
}

openfft_plan_t openfft_plan_many(int count, const int* NaNbNc, const int* P, int dtype)
{
    int dev = 0, sms = 148;
    cudaError_t e = cudaGetDevice(&dev);
    if (e) { cuda_fail(e, "cudaGetDevice"); return nullptr; }
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if ((e = stage_kernels_init(200 * 1024))) { cuda_fail(e, "kernel attributes"); return nullptr; }
    BatchPlan* b = nullptr;
    if (batch_create(count, NaNbNc, P, dtype, sms, &b, &fail_cstr)) return nullptr;
    openfft_plan_s* p = new openfft_plan_s();
    p->Na = NaNbNc[0]; p->Nb = NaNbNc[1]; p->Nc = NaNbNc[2]; p->P = P[0]; p->dtype = dtype;
    p->N = 0;
    p->device = dev; p->sms = sms;
    p->batch = b;
    return p;
}

int openfft_exec_many(openfft_plan_t plan, const void* const* in, void* const* out, int dir)
{
    if (!plan || !plan->batch) return fail(OPENFFT_ERR_INVALID_ARG, "not a batched plan (openfft_plan_many)");
    return batch_exec(plan->batch, in, out, dir, plan->stream, &fail_cstr);
}

int openfft_batch_debug(openfft_plan_t plan, int what, long long value)
{
    if (!plan || !plan->batch) return fail(OPENFFT_ERR_INVALID_ARG, "not a batched plan");
    if (what == 1) return batch_set_wait_budget(plan->batch, value);
    if (what == 2) {
        if (batch_inject_stall(plan->batch, value != 0)) return fail(OPENFFT_ERR_CUDA, "stall injection");
        return OPENFFT_OK;
    }
    return fail(OPENFFT_ERR_INVALID_ARG, "what must be 1 (wait budget) or 2 (stall injection)");
}

int openfft_tc_debug(int what, long long value)
{
    if (what != 1 && what != 2) return fail(OPENFFT_ERR_INVALID_ARG, "what must be 1 (wait budget) or 2 (skip the MMAs)");
    cudaError_t e = dftgemm_test_controls(what, value);
    if (e) return cuda_fail(e, "DFT-GEMM test controls");
    return OPENFFT_OK;
}

int openfft_set_timing(openfft_plan_t plan, int enable)
{
    if (!plan) return fail(OPENFFT_ERR_INVALID_ARG, "null plan");
    if (enable && plan->ev.empty()) {
        plan->ev.resize(4096);
        plan->ev_cat.resize(4096);
        for (cudaEvent_t& e : plan->ev) {
            cudaError_t err = cudaEventCreate(&e);
            if (err) return cuda_fail(err, "cudaEventCreate");
        }
    }
    if (!enable && plan->timing) { int st = fold_timing(plan); if (st) return st; }
    plan->timing = enable != 0;
    return OPENFFT_OK;
}

int openfft_get_timing(openfft_plan_t plan, double ms[4], int64_t launches[4])
{
    if (!plan || !ms || !launches) return fail(OPENFFT_ERR_INVALID_ARG, "null plan or output");
    int st = fold_timing(plan);
    if (st) return st;
    for (int i = 0; i < 4; ++i) {
        ms[i] = plan->t_ms[i]; launches[i] = plan->t_launch[i];
        plan->t_ms[i] = 0; plan->t_launch[i] = 0;
    }
    return OPENFFT_OK;
}

int openfft_redistribute(openfft_plan_t plan, int exchange, int variant, const void* in, void* out)
{
    if (!plan || !in || !out) return fail(OPENFFT_ERR_INVALID_ARG, "null plan or buffer");
    if (in == out) return fail(OPENFFT_ERR_ALIAS, "in and out must differ");
    if (exchange != 1 && exchange != 2 && exchange != -1 && exchange != -2)
        return fail(OPENFFT_ERR_INVALID_ARG, "exchange must be 1, 2, -2 or -1");
    const int64_t Na = plan->Na, Nb = plan->Nb, Nc = plan->Nc;
    const int E = (int)plan->elem_bytes;
    const int ar = plan->elem_bytes == 8 ? ARITH_F32 : ARITH_F64;
    const int fmt = ar == ARITH_F32 ? FMT_C64 : FMT_C128;
    const TransposeTables& T = plan->tt[tix_of(exchange)];
    cudaError_t e = cudaSuccess;
    if (variant == OPENFFT_VARIANT_FUSED) {
        // the stage kernel with its radix passes switched off: the fused store alone
        StageLaunch L;
        int st;
        switch (exchange) {
        case 1: st = make_stage(plan, 2, ar, 8, KERNEL_GENERIC, Na * Nb, 1, 1, 0, Na * Nb, 0, 0, fmt, fmt, 0, 0, 1.0, 0, L); break;
        case 2: st = make_stage(plan, 1, ar, 8, KERNEL_GENERIC, Na, Nc, 1, Nb * Na, Na, 0, 0, fmt, fmt, 0, 0, 1.0, 0, L); break;
        case -2: st = make_stage(plan, 0, ar, 8, KERNEL_GENERIC, Nb, Nc, 1, Na * Nb, Nb, 0, 0, fmt, fmt, 0, 0, 1.0, 0, L); break;
        default: st = make_stage(plan, 1, ar, 8, KERNEL_GENERIC, Na, Nc, Nb * Nc, 1, Nc, 1, 0, fmt, fmt, 0, 0, 1.0, 0, L); break;
        }
        if (st) return st;
        L.args.in = in; L.args.out = out;
        e = launch_stage(L, plan->stream);
    } else if (variant >= OPENFFT_VARIANT_PACK_EXCHANGE_UNPACK && variant <= OPENFFT_VARIANT_SENDRECV) {
        // the ops of one transpose: send segments in A, receive buffers in B
        std::vector<Op> ops;
        transpose_ops(ops, variant, tix_of(exchange), B_B, B_OUT, plan->P);
        Bounds bnd;
        bnd.chk = plan->d_status; bnd.lim = plan->N;
        for (const Op& o : ops) {
            const void* src = o.src == B_IN ? in : (o.src == B_OUT ? out : (o.src == B_A ? plan->bufA : plan->bufB));
            void* dst = o.dst == B_OUT ? out : (o.dst == B_A ? plan->bufA : plan->bufB);
            if (o.kind == OP_PACK) src = in;                 // the source ordering is the caller's input
            if (o.kind == OP_PACK) e = launch_pack(T.t, E, src, dst, T.d_sbase, plan->N, plan->sms, plan->stream, bnd);
            else if (o.kind == OP_EXCHANGE) e = launch_exchange(E, T.d_chunks, T.nchunks, src, dst, plan->sms, plan->stream, bnd);
            else if (o.kind == OP_UNPACK) e = launch_unpack(T.t, E, src, dst, o.from_send ? T.d_sbase : T.d_rbase, o.from_send, plan->N, plan->sms, plan->stream, bnd);
            else if (o.kind == OP_SEG_EXCHANGE) e = launch_segment_exchange(o.sched, plan->P, kBlockSize, o.step, E, T.d_C, T.d_sdispl, T.d_rdispl, src, dst, plan->stream, bnd);
            else e = launch_segment_unpack(T.t, o.sched, kBlockSize, o.step, E, src, dst, T.d_sbase, plan->stream, bnd);
            if (e) break;
        }
    } else {
        return fail(OPENFFT_ERR_INVALID_ARG, "unknown variant");
    }
    if (e) return cuda_fail(e, "redistribution launch");
    return OPENFFT_OK;
}

}  // extern "C"
