// nd.cu -- D-dimensional transforms (D = 3..5) under the decomposition.
//
// The paper cites 4-D and 5-D transforms under the same decomposition
// (Sec. 1) without their transpose orders.  Reading taken, generalising the
// 3-D order abc -> cab -> cba of Sec. 2: ordering s = 1..D of A[N_1]...[N_D]
// (d_D fastest) is (d_D, ..., d_{D-s+2}, d_1, ..., d_{D-s+1}); stage s
// transforms the fastest axis of ordering s and its store writes ordering
// s + 1 (the transpose fused into the store, as in the 3-D fused variant).
// The forward result is left in ordering D (the reversed axes); the backward
// transform runs the orderings in reverse and divides by N.  Each ordering is
// decomposed by Eqs. 2-9 with (N1, N2, N3) = (its first dimension, its
// second, the product of the rest).
//
// Stage geometry (lines l = i1 + i2 M1, output (l, k) at i1 S1 + i2 S2 + k Sk):
//   forward stage s < D, n = N_{D-s+1}, M = N_1...N_{D-s}, Q = N_{D-s+2}...N_D:
//     i1 = position in d_1..d_{D-s} (M1 = M, S1 = 1), i2 = prefix (M2 = Q,
//     S2 = n M), Sk = M;
//   backward stage t < D, n = N_t, M' = N_1...N_{t-1}, x = d_{t+1}, and the
//     prefix p over d_{t+2}..d_D: output (p, r', k, x) at
//     p M' n N_x + (r' n + k) N_x + x.  With M' = 1 one launch takes
//     (i1, i2) = (x, p); with no p one launch takes (r', x); otherwise one
//     launch per p (the stage descriptor has two line coordinates);
//   the last stage of either direction is contiguous, in place.
#include <cuda_runtime.h>

#include <cstring>
#include <vector>

#include "../../include/openfft_gb.h"
#include "decomp.h"
#include "fft_stage.h"

namespace ofg {
int set_last_error(int status, const char* msg);   // capi.cu
}

using namespace ofg;

namespace {

constexpr int kMaxNd = 5;

void nd_axes(int D, int s, int* axes)
{
    int k = 0;
    for (int i = 0; i < s - 1; ++i) axes[k++] = D - 1 - i;
    for (int i = 0; i < D - s + 1; ++i) axes[k++] = i;
}

// Eq. 2-4 of ordering s as a 3-D ordering (N1, N2, product of the rest)
Ordering nd_ordering(int D, const int* dims, int s, int P)
{
    int axes[kMaxNd];
    nd_axes(D, s, axes);
    int64_t rest = 1;
    for (int j = 2; j < D; ++j) rest *= dims[axes[j]];
    return make_ordering(dims[axes[0]], dims[axes[1]], rest, P);
}

int check_nd(int ndim, const int* dims, int P)
{
    if (ndim < 3 || ndim > kMaxNd || !dims) return set_last_error(OPENFFT_ERR_INVALID_ARG, "ndim must be 3, 4 or 5");
    for (int i = 0; i < ndim; ++i)
        if (dims[i] < 1) return set_last_error(OPENFFT_ERR_INVALID_ARG, "dims must be >= 1");
    if (P < 1) return set_last_error(OPENFFT_ERR_INVALID_ARG, "P must be >= 1");
    for (int s = 1; s <= ndim; ++s)
        if (nd_ordering(ndim, dims, s, P).degree < 0)
            return set_last_error(OPENFFT_ERR_P_TOO_LARGE, "P exceeds N1*N2 of an ordering (Eq. 2 undefined)");
    return OPENFFT_OK;
}

bool radix_of(int n, StageArgs& a)
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

// one launch: the stage descriptor and the element offsets of its arrays
struct NdLaunch {
    StageLaunch L;
    int src, dst;            // 0 = user input, 1 = user output, 2 = workspace
    int64_t in_off, out_off; // elements
};

}  // namespace

struct openfft_nd_plan_s {
    int D, P, dtype, arith;
    int dims[kMaxNd];
    int64_t N;
    int sms = 148;
    cudaStream_t stream = nullptr;
    void* work = nullptr;
    void* tw[kMaxNd] = {};
    std::vector<NdLaunch> fwd, bwd;
};

namespace {

void free_nd(openfft_nd_plan_s* p)
{
    if (!p) return;
    cudaFree(p->work);
    for (void* t : p->tw) cudaFree(t);
    delete p;
}

int add_stage(openfft_nd_plan_s* p, std::vector<NdLaunch>& ops, int axis, int64_t M1, int64_t M2, int64_t S1,
              int64_t S2, int64_t Sk, int group_i2, int contig, bool first, bool last, int dir, int src, int dst,
              int64_t in_off, int64_t out_off)
{
    NdLaunch op;
    std::memset(&op, 0, sizeof(op));
    StageLaunch& L = op.L;
    StageArgs& a = L.args;
    const int n = p->dims[axis];
    radix_of(n, a);
    const bool f32 = p->arith == ARITH_F32;
    const int E = f32 ? 8 : 16;
    int G = f32 ? 16 : 8;
    const int64_t Mg = group_i2 ? M2 : M1;
    while (G > 1 && (int64_t)(G / 2) >= Mg) G /= 2;
    while (G > 1 && 2 * (size_t)n * (G + 1) * E > 200 * 1024) G /= 2;
    if (2 * (size_t)n * (G + 1) * E > 200 * 1024) return set_last_error(OPENFFT_ERR_UNSUPPORTED_RADIX, "axis too long for one CTA");
    int lg = 0;
    while ((1 << lg) < G) ++lg;
    const int ext = f32 ? FMT_C64 : FMT_C128, mid = f32 ? FMT_C64 : FMT_DF;
    a.tw = p->tw[axis];
    a.M1 = M1; a.M2 = M2; a.S1 = S1; a.S2 = S2; a.Sk = Sk;
    a.ngroups = (Mg + G - 1) / G;
    a.n = n; a.G = G; a.log2G = lg;
    a.group_i2 = group_i2; a.contig_store = contig; a.do_fft = 1;
    a.in_fmt = first ? ext : mid;
    a.out_fmt = last ? ext : mid;
    a.conj_in = (dir == OPENFFT_BACKWARD && first) ? 1 : 0;
    a.conj_out = (dir == OPENFFT_BACKWARD && last) ? 1 : 0;
    a.scale = a.conj_out ? 1.0 / (double)p->N : 1.0;
    L.arith = p->arith;
    L.grid = a.ngroups * (group_i2 ? M1 : M2);
    L.smem = 2 * (size_t)n * (G + 1) * E;
    L.sms = p->sms;
    L.family = KERNEL_AUTO;
    if (L.grid > 0x7fffffffLL) return set_last_error(OPENFFT_ERR_UNSUPPORTED, "grid too large");
    op.src = src; op.dst = dst; op.in_off = in_off; op.out_off = out_off;
    ops.push_back(op);
    return OPENFFT_OK;
}

// Forward: stage s (s < D) writes the user output when D - 1 - s is even,
// the workspace otherwise, so that stage D - 1 lands in the output and the
// last stage runs in place there.
int build_forward(openfft_nd_plan_s* p)
{
    const int D = p->D;
    int src = 0;
    for (int s = 1; s <= D; ++s) {
        const int axis = D - s;
        const int64_t n = p->dims[axis];
        int64_t M = 1, Q = 1;
        for (int i = 0; i < axis; ++i) M *= p->dims[i];
        for (int i = axis + 1; i < D; ++i) Q *= p->dims[i];
        int st;
        if (s < D) {
            const int dst = (D - 1 - s) % 2 == 0 ? 1 : 2;
            st = add_stage(p, p->fwd, axis, M, Q, 1, n * M, M, 0, 0, s == 1, false, OPENFFT_FORWARD, src, dst, 0, 0);
            src = dst;
        } else {
            st = add_stage(p, p->fwd, axis, Q, 1, n, 0, 1, 0, 1, false, true, OPENFFT_FORWARD, 1, 1, 0, 0);
        }
        if (st) return st;
    }
    return OPENFFT_OK;
}

int build_backward(openfft_nd_plan_s* p)
{
    const int D = p->D;
    int src = 0;
    for (int t = 1; t <= D; ++t) {
        const int axis = t - 1;
        const int64_t n = p->dims[axis];
        int st;
        if (t == D) {
            st = add_stage(p, p->bwd, axis, p->N / n, 1, n, 0, 1, 0, 1, false, true, OPENFFT_BACKWARD, 1, 1, 0, 0);
            if (st) return st;
            break;
        }
        int64_t Mp = 1, Pc = 1;
        for (int i = 0; i < axis; ++i) Mp *= p->dims[i];
        for (int i = t + 1; i < D; ++i) Pc *= p->dims[i];
        const int64_t Nx = p->dims[t];
        const int dst = (D - 1 - t) % 2 == 0 ? 1 : 2;
        const bool first = t == 1;
        if (Mp == 1) {
            st = add_stage(p, p->bwd, axis, Nx, Pc, 1, n * Nx, Nx, 0, 0, first, false, OPENFFT_BACKWARD, src, dst, 0, 0);
            if (st) return st;
        } else {
            const int64_t block = Mp * n * Nx;
            for (int64_t q = 0; q < Pc; ++q) {
                st = add_stage(p, p->bwd, axis, Mp, Nx, n * Nx, 1, Nx, 1, 0, first, false, OPENFFT_BACKWARD, src, dst,
                               q * block, q * block);
                if (st) return st;
            }
        }
        src = dst;
    }
    return OPENFFT_OK;
}

int box_nd(int ndim, const int* dims, int P, int s, int rank, int64_t* offset, int64_t* count)
{
    const Ordering o = nd_ordering(ndim, dims, s, P);
    if (rank < 0 || rank >= P) return set_last_error(OPENFFT_ERR_INVALID_ARG, "rank out of range");
    const int64_t xs = box_begin(o, rank), xe = box_begin(o, rank + 1);
    if (offset) *offset = xs;
    if (count) *count = xe - xs;
    return OPENFFT_OK;
}

}  // namespace

extern "C" {

int openfft_nd_decomp_box(int ndim, const int* dims, int P, int ordering, int rank, int64_t* offset, int64_t* count)
{
    int st = check_nd(ndim, dims, P);
    if (st) return st;
    if (ordering < 1 || ordering > ndim) return set_last_error(OPENFFT_ERR_INVALID_ARG, "ordering must be 1..ndim");
    return box_nd(ndim, dims, P, ordering, rank, offset, count);
}

int openfft_nd_decomp_counts(int ndim, const int* dims, int P, int exchange, int64_t* PxP)
{
    int st = check_nd(ndim, dims, P);
    if (st) return st;
    const int s = exchange > 0 ? exchange : -exchange;
    if (!PxP || s < 1 || s >= ndim) return set_last_error(OPENFFT_ERR_INVALID_ARG, "exchange must be +-1..ndim-1");
    const int sa = exchange > 0 ? s : s + 1, sb = exchange > 0 ? s + 1 : s;
    const Ordering oa = nd_ordering(ndim, dims, sa, P), ob = nd_ordering(ndim, dims, sb, P);
    int ax_a[kMaxNd], ax_b[kMaxNd];
    nd_axes(ndim, sa, ax_a);
    nd_axes(ndim, sb, ax_b);
    int64_t N = 1;
    for (int i = 0; i < ndim; ++i) N *= dims[i];
    std::memset(PxP, 0, sizeof(int64_t) * (size_t)P * P);
    int64_t v[kMaxNd];
    for (int64_t x = 0; x < N; ++x) {
        int64_t r = x;
        for (int j = ndim - 1; j >= 0; --j) { v[ax_a[j]] = r % dims[ax_a[j]]; r /= dims[ax_a[j]]; }
        int64_t y = 0;
        for (int j = 0; j < ndim; ++j) y = y * dims[ax_b[j]] + v[ax_b[j]];
        const int64_t src = row_owner(oa, x / oa.D2), dst = row_owner(ob, y / ob.D2);
        PxP[src * P + dst] += 1;
    }
    return OPENFFT_OK;
}

openfft_nd_plan_t openfft_nd_plan(int ndim, const int* dims, int P, int dtype)
{
    if (check_nd(ndim, dims, P)) return nullptr;
    if (dtype != OPENFFT_C2C_F64 && dtype != OPENFFT_C2C_F32) {
        set_last_error(OPENFFT_ERR_UNSUPPORTED, "D-dimensional plans support OPENFFT_C2C_F64 and OPENFFT_C2C_F32");
        return nullptr;
    }
    auto* p = new openfft_nd_plan_s();
    p->D = ndim; p->P = P; p->dtype = dtype;
    p->arith = dtype == OPENFFT_C2C_F32 ? ARITH_F32 : ARITH_DF;
    p->N = 1;
    for (int i = 0; i < ndim; ++i) {
        p->dims[i] = dims[i];
        p->N *= dims[i];
        StageArgs a;
        if (!radix_of(dims[i], a) || dims[i] > kMaxLen) {
            set_last_error(OPENFFT_ERR_UNSUPPORTED_RADIX, "axis length must factor into 2, 3, 5, 7 and be <= 2048");
            delete p;
            return nullptr;
        }
    }
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&p->sms, cudaDevAttrMultiProcessorCount, dev);
    cudaError_t e = stage_kernels_init(200 * 1024);
    if (e) { set_last_error(OPENFFT_ERR_CUDA, cudaGetErrorString(e)); delete p; return nullptr; }
    const size_t E = p->arith == ARITH_F32 ? 8 : 16;
    if (dev_malloc(&p->work, (size_t)p->N * E)) {
        cudaGetLastError();
        set_last_error(OPENFFT_ERR_NOMEM, "workspace allocation failed");
        free_nd(p);
        return nullptr;
    }
    const int twf = p->arith == ARITH_F32 ? FMT_C64 : FMT_DF;
    for (int i = 0; i < ndim; ++i) {
        if (dev_malloc(&p->tw[i], twiddle_bytes(dims[i], twf))) {
            cudaGetLastError();
            set_last_error(OPENFFT_ERR_NOMEM, "twiddle allocation failed");
            free_nd(p);
            return nullptr;
        }
        if ((e = launch_twiddles(dims[i], twf, p->tw[i], nullptr))) {
            set_last_error(OPENFFT_ERR_CUDA, cudaGetErrorString(e));
            free_nd(p);
            return nullptr;
        }
    }
    int st = build_forward(p);
    if (!st) st = build_backward(p);
    if (st) { free_nd(p); return nullptr; }
    if ((e = cudaDeviceSynchronize())) { set_last_error(OPENFFT_ERR_CUDA, cudaGetErrorString(e)); free_nd(p); return nullptr; }
    return p;
}

void openfft_nd_destroy(openfft_nd_plan_t p) { free_nd(p); }

int openfft_nd_set_stream(openfft_nd_plan_t p, void* stream)
{
    if (!p) return set_last_error(OPENFFT_ERR_INVALID_ARG, "null plan");
    p->stream = static_cast<cudaStream_t>(stream);
    return OPENFFT_OK;
}

int openfft_nd_box(openfft_nd_plan_t p, int which, int rank, int64_t* offset, int64_t* count)
{
    if (!p || (which != 0 && which != 1)) return set_last_error(OPENFFT_ERR_INVALID_ARG, "plan or which");
    return box_nd(p->D, p->dims, p->P, which == 0 ? 1 : p->D, rank, offset, count);
}

int openfft_nd_exec(openfft_nd_plan_t p, const void* in, void* out, int dir)
{
    if (!p || !in || !out) return set_last_error(OPENFFT_ERR_INVALID_ARG, "null plan or buffer");
    if (in == out) return set_last_error(OPENFFT_ERR_ALIAS, "in and out must differ (out-of-place only)");
    if (dir != OPENFFT_FORWARD && dir != OPENFFT_BACKWARD) return set_last_error(OPENFFT_ERR_INVALID_ARG, "dir must be -1 or +1");
    const size_t E = p->arith == ARITH_F32 ? 8 : 16;
    const void* bufs_in[3] = {in, out, p->work};
    void* bufs_out[3] = {nullptr, out, p->work};
    for (const NdLaunch& op : dir == OPENFFT_FORWARD ? p->fwd : p->bwd) {
        StageLaunch L = op.L;
        L.args.in = static_cast<const char*>(bufs_in[op.src]) + op.in_off * (int64_t)E;
        L.args.out = static_cast<char*>(bufs_out[op.dst]) + op.out_off * (int64_t)E;
        L.args.in_elems = p->N - op.in_off;        // every buffer holds N elements
        L.args.out_elems = p->N - op.out_off;
        cudaError_t e = launch_stage(L, p->stream);
        if (e) return set_last_error(OPENFFT_ERR_CUDA, cudaGetErrorString(e));
    }
    return OPENFFT_OK;
}

}  // extern "C"
