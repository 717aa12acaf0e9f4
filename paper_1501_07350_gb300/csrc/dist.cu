// dist.cu -- the transform over G devices (processes), each holding a
// contiguous block of the P logical ranks: the paper's distributed execution
// (Duy & Ozaki, Sec. 3.1.1 steps (1)-(6)) with the ranks of one device
// sharing its memory.
//
// Device g of G holds logical ranks [floor(g P / G), floor((g + 1) P / G)).
// Every rank's box is a contiguous slice of its ordering's 1-D index space
// (Eqs. 3-4), so device g holds one contiguous slice of each ordering too:
// the rows [row_begin(rank0(g)), row_begin(rank0(g + 1))) of that ordering.
// A transpose (R1 abc -> cab, R2 cab -> cba, and their inverses) becomes one
// all-to-all with variable counts among the devices:
//   pack   (step 4): device g writes each element it holds into the send
//          segment of the device owning its destination, at its rank in
//          ascending source index inside that segment (the order the
//          single-memory pack uses for each pair of ranks);
//   the all-to-all-v itself (step 5) is done by the caller's communication
//          library (NCCL send / recv groups on GPUs, gloo on CPUs): segment
//          g -> h, of D[g][h] elements, goes from send displacement
//          sum_{h' < h} D[g][h'] of g to receive displacement
//          sum_{g' < g} D[g'][h] of h;
//   unpack (step 6): device h reads each element of its destination slice
//          from the received segments.
// D[g][h] is the sum of the P x P count matrix over the two devices' ranks.
// Positions come from the closed forms of decomp.h with the devices' row
// ranges in place of the ranks' ones.  The 1-D FFT stages are line-local:
// each device transforms the whole lines of its slice with the stage kernels
// of fft_stage.h, contiguous in and out.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/openfft_gb.h"
#include "decomp.h"
#include "fft_stage.h"

namespace ofg {
int set_last_error(int status, const char* msg);   // capi.cu
}

using namespace ofg;

namespace {

constexpr int kMaxDistDevices = 1024;

// first logical rank of device g (Eq. 2 with the ranks as the divided axis)
int64_t rank0(int64_t P, int64_t G, int64_t g) { return (P * g) / G; }
DHD int64_t device_of(int64_t P, int64_t G, int64_t r) { return ((r + 1) * G - 1) / P; }

int transpose_layouts(int which, int* src, int* dst)
{
    switch (which) {
    case 1: *src = ABC; *dst = CAB; return 0;
    case 2: *src = CAB; *dst = CBA; return 0;
    case -2: *src = CBA; *dst = CAB; return 0;
    case -1: *src = CAB; *dst = ABC; return 0;
    default: return -1;
    }
}

int check_dims(int Na, int Nb, int Nc, int P, int G)
{
    if (Na < 1 || Nb < 1 || Nc < 1 || P < 1 || G < 1)
        return set_last_error(OPENFFT_ERR_INVALID_ARG, "sizes, P and G must be >= 1");
    if (G > P) return set_last_error(OPENFFT_ERR_INVALID_ARG, "G must not exceed P (every device holds a rank)");
    if (G > kMaxDistDevices) return set_last_error(OPENFFT_ERR_INVALID_ARG, "G exceeds 1024");
    const int64_t a = Na, b = Nb, c = Nc;
    if ((int64_t)P > a * b || (int64_t)P > c * a || (int64_t)P > c * b)
        return set_last_error(OPENFFT_ERR_P_TOO_LARGE, "P exceeds N1*N2 of an ordering (Eq. 2 undefined)");
    return OPENFFT_OK;
}

// Rows [*R0, *R1) of ordering o held by device g.
void device_rows(const Ordering& o, int64_t G, int64_t g, int64_t* R0, int64_t* R1)
{
    *R0 = row_begin(o, rank0(o.P, G, g));
    *R1 = row_begin(o, rank0(o.P, G, g + 1));
}

// Per-device view of one transpose: the device's source rows, every device's
// destination rows, and the pack / unpack bases.
struct DistSide {
    Transpose t;
    int64_t G, me;
    int64_t R0, R1;               // my source rows
    int64_t Q0, Q1;               // my destination rows
    std::vector<int64_t> q0, q1;  // destination rows of every device
    std::vector<int64_t> r0;      // first source row of every device
    std::vector<int64_t> send, recv;    // counts per peer (elements)
    std::vector<int64_t> sdispl, rdispl;
    std::vector<int64_t> spre;    // prefix_to(R0_me, q0[h], q1[h]) per destination h
    std::vector<int64_t> rpre;    // prefix_to(r0[g], Q0, Q1) per source g
};

void make_side(int which, int Na, int Nb, int Nc, int P, int G, int me, DistSide& d)
{
    d.t = make_transpose(which, Na, Nb, Nc, P);
    d.G = G; d.me = me;
    device_rows(d.t.src, G, me, &d.R0, &d.R1);
    device_rows(d.t.dst, G, me, &d.Q0, &d.Q1);
    d.q0.resize(G); d.q1.resize(G); d.r0.resize(G + 1);
    for (int h = 0; h < G; ++h) device_rows(d.t.dst, G, h, &d.q0[h], &d.q1[h]);
    for (int g = 0; g <= G; ++g) d.r0[g] = row_begin(d.t.src, rank0(P, G, g));
    d.send.resize(G); d.recv.resize(G); d.sdispl.resize(G); d.rdispl.resize(G);
    d.spre.resize(G); d.rpre.resize(G);
    int64_t so = 0, ro = 0;
    for (int h = 0; h < G; ++h) {
        d.spre[h] = prefix_to(d.t, d.R0, d.q0[h], d.q1[h]);
        d.send[h] = prefix_to(d.t, d.R1, d.q0[h], d.q1[h]) - d.spre[h];
        d.sdispl[h] = so; so += d.send[h];
    }
    for (int g = 0; g < G; ++g) {
        d.rpre[g] = prefix_to(d.t, d.r0[g], d.Q0, d.Q1);
        d.recv[g] = prefix_to(d.t, d.r0[g + 1], d.Q0, d.Q1) - d.rpre[g];
        d.rdispl[g] = ro; ro += d.recv[g];
    }
}

// Send position of source element (row q, element e) of device `me` whose
// destination row lies with device h.
DHD int64_t pack_pos(const Transpose& t, int64_t q, int64_t e, int64_t Qh0, int64_t Qh1, int64_t sdispl_h,
                     int64_t spre_h)
{
    int64_t e_lo, cnt;
    row_range(t, q, Qh0, Qh1, &e_lo, &cnt);
    return sdispl_h + prefix_to(t, q, Qh0, Qh1) - spre_h + (e - e_lo);
}

// ------------------------------------------------------------- host side --

void pack_host(const DistSide& d, int P, int eb, const unsigned char* src, unsigned char* send)
{
    const Transpose& t = d.t;
    const int64_t Ls = row_len(t), Ld = dst_row_len(t);
    const int64_t n = (d.R1 - d.R0) * Ls;
    for (int64_t x = 0; x < n; ++x) {
        const int64_t q = d.R0 + x / Ls, e = x % Ls;
        const int64_t y = dest_index(t, q, e);
        const int64_t h = device_of(P, d.G, row_owner(t.dst, y / Ld));
        const int64_t pos = pack_pos(t, q, e, d.q0[h], d.q1[h], d.sdispl[h], d.spre[h]);
        std::memcpy(send + pos * eb, src + x * eb, (size_t)eb);
    }
}

void unpack_host(const DistSide& d, int P, int eb, const unsigned char* recv, unsigned char* dst)
{
    const Transpose& t = d.t;
    const int64_t Ld = dst_row_len(t);
    const int64_t n = (d.Q1 - d.Q0) * Ld;
    for (int64_t yl = 0; yl < n; ++yl) {
        const int64_t y = d.Q0 * Ld + yl;
        int64_t q, e;
        source_of(t, y, &q, &e);
        const int64_t g = device_of(P, d.G, row_owner(t.src, q));
        const int64_t pos = pack_pos(t, q, e, d.Q0, d.Q1, d.rdispl[g], d.rpre[g]);
        std::memcpy(dst + yl * eb, recv + pos * eb, (size_t)eb);
    }
}

// ----------------------------------------------------------- device side --

struct DevTables {
    int64_t* q0 = nullptr;     // [G] destination row begin per device
    int64_t* q1 = nullptr;     // [G]
    int64_t* sdispl = nullptr; // [G]
    int64_t* spre = nullptr;   // [G]
    int64_t* rdispl = nullptr; // [G]
    int64_t* rpre = nullptr;   // [G]
};

template <class E>
__global__ void dist_pack_kernel(const Transpose t, int64_t P, int64_t G, int64_t R0, int64_t n,
                                 const int64_t* __restrict__ q0, const int64_t* __restrict__ q1,
                                 const int64_t* __restrict__ sdispl, const int64_t* __restrict__ spre,
                                 const E* __restrict__ src, E* __restrict__ send, const Bounds b)
{
    const int64_t Ls = row_len(t), Ld = dst_row_len(t);
    for (int64_t x = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; x < n; x += (int64_t)gridDim.x * blockDim.x) {
        const int64_t q = R0 + x / Ls, e = x % Ls;
        const int64_t y = dest_index(t, q, e);
        const int64_t h = device_of(P, G, row_owner(t.dst, y / Ld));
        const int64_t pos = pack_pos(t, q, e, q0[h], q1[h], sdispl[h], spre[h]);
        if (in_bounds(b, pos)) send[pos] = src[x];
    }
}

template <class E>
__global__ void dist_unpack_kernel(const Transpose t, int64_t P, int64_t G, int64_t Q0, int64_t Q1, int64_t n,
                                   const int64_t* __restrict__ rdispl, const int64_t* __restrict__ rpre,
                                   const E* __restrict__ recv, E* __restrict__ dst, const Bounds b)
{
    const int64_t Ld = dst_row_len(t);
    for (int64_t yl = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; yl < n; yl += (int64_t)gridDim.x * blockDim.x) {
        int64_t q, e;
        source_of(t, Q0 * Ld + yl, &q, &e);
        const int64_t g = device_of(P, G, row_owner(t.src, q));
        const int64_t pos = pack_pos(t, q, e, Q0, Q1, rdispl[g], rpre[g]);
        if (in_bounds(b, pos)) dst[yl] = recv[pos];
    }
}

bool radix_plan_of(int n, StageArgs& a)
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

}  // namespace

struct openfft_dist_plan_s {
    int Na, Nb, Nc, P, G, g, dtype, arith;
    int sms = 148;
    cudaStream_t stream = nullptr;
    void* tw[3] = {};              // twiddle tables of axes a, b, c
    DistSide side[4];              // R1, R2, R2', R1'
    DevTables dt[4];
};

namespace {

int side_index(int which) { return which == 1 ? 0 : (which == 2 ? 1 : (which == -2 ? 2 : 3)); }

void free_dist(openfft_dist_plan_s* p)
{
    if (!p) return;
    for (auto& t : p->tw) cudaFree(t);
    for (auto& d : p->dt) {
        cudaFree(d.q0); cudaFree(d.q1); cudaFree(d.sdispl); cudaFree(d.spre); cudaFree(d.rdispl); cudaFree(d.rpre);
    }
    delete p;
}

int upload(int64_t** dst, const std::vector<int64_t>& v)
{
    if (dev_malloc((void**)dst, sizeof(int64_t) * std::max<size_t>(1, v.size()))) { cudaGetLastError(); return 1; }
    return cudaMemcpy(*dst, v.data(), sizeof(int64_t) * v.size(), cudaMemcpyHostToDevice) != cudaSuccess;
}

}  // namespace

extern "C" {

int openfft_dist_rows(int Na, int Nb, int Nc, int P, int G, int layout, int g, int64_t* offset, int64_t* count)
{
    int st = check_dims(Na, Nb, Nc, P, G);
    if (st) return st;
    if (layout < 0 || layout > 2 || g < 0 || g >= G) return set_last_error(OPENFFT_ERR_INVALID_ARG, "layout or device index");
    const Ordering o = ordering_of(layout, Na, Nb, Nc, P);
    int64_t R0, R1;
    device_rows(o, G, g, &R0, &R1);
    if (offset) *offset = R0 * o.D2;
    if (count) *count = (R1 - R0) * o.D2;
    return OPENFFT_OK;
}

int openfft_dist_counts(int Na, int Nb, int Nc, int P, int G, int exchange, int64_t* GxG)
{
    int st = check_dims(Na, Nb, Nc, P, G);
    if (st) return st;
    int sl, dl;
    if (!GxG || transpose_layouts(exchange, &sl, &dl)) return set_last_error(OPENFFT_ERR_INVALID_ARG, "exchange or output");
    for (int g = 0; g < G; ++g) {
        DistSide d;
        make_side(exchange, Na, Nb, Nc, P, G, g, d);
        for (int h = 0; h < G; ++h) GxG[(int64_t)g * G + h] = d.send[h];
    }
    return OPENFFT_OK;
}

int openfft_dist_pack_host(int Na, int Nb, int Nc, int P, int G, int exchange, int g, int elem_bytes,
                           const void* src, void* send)
{
    int st = check_dims(Na, Nb, Nc, P, G);
    if (st) return st;
    int sl, dl;
    if (transpose_layouts(exchange, &sl, &dl) || g < 0 || g >= G || elem_bytes < 1 || !src || !send)
        return set_last_error(OPENFFT_ERR_INVALID_ARG, "exchange, device index, element size or buffers");
    DistSide d;
    make_side(exchange, Na, Nb, Nc, P, G, g, d);
    pack_host(d, P, elem_bytes, static_cast<const unsigned char*>(src), static_cast<unsigned char*>(send));
    return OPENFFT_OK;
}

int openfft_dist_unpack_host(int Na, int Nb, int Nc, int P, int G, int exchange, int g, int elem_bytes,
                             const void* recv, void* dst)
{
    int st = check_dims(Na, Nb, Nc, P, G);
    if (st) return st;
    int sl, dl;
    if (transpose_layouts(exchange, &sl, &dl) || g < 0 || g >= G || elem_bytes < 1 || !recv || !dst)
        return set_last_error(OPENFFT_ERR_INVALID_ARG, "exchange, device index, element size or buffers");
    DistSide d;
    make_side(exchange, Na, Nb, Nc, P, G, g, d);
    unpack_host(d, P, elem_bytes, static_cast<const unsigned char*>(recv), static_cast<unsigned char*>(dst));
    return OPENFFT_OK;
}

openfft_dist_plan_t openfft_dist_plan(int Na, int Nb, int Nc, int P, int G, int g, int dtype)
{
    if (check_dims(Na, Nb, Nc, P, G)) return nullptr;
    if (g < 0 || g >= G) { set_last_error(OPENFFT_ERR_INVALID_ARG, "device index out of range"); return nullptr; }
    if (dtype != OPENFFT_C2C_F64 && dtype != OPENFFT_C2C_F32) {
        set_last_error(OPENFFT_ERR_UNSUPPORTED, "distributed plans support OPENFFT_C2C_F64 and OPENFFT_C2C_F32");
        return nullptr;
    }
    for (int n : {Na, Nb, Nc}) {
        StageArgs a;
        if (!radix_plan_of(n, a) || n > kMaxLen) {
            set_last_error(OPENFFT_ERR_UNSUPPORTED_RADIX, "axis length must factor into 2, 3, 5, 7 and be <= 2048");
            return nullptr;
        }
    }
    auto* p = new openfft_dist_plan_s();
    p->Na = Na; p->Nb = Nb; p->Nc = Nc; p->P = P; p->G = G; p->g = g; p->dtype = dtype;
    p->arith = dtype == OPENFFT_C2C_F32 ? ARITH_F32 : ARITH_DF;
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&p->sms, cudaDevAttrMultiProcessorCount, dev);
    cudaError_t e = stage_kernels_init(200 * 1024);
    if (e) { set_last_error(OPENFFT_ERR_CUDA, cudaGetErrorString(e)); free_dist(p); return nullptr; }
    const int lens[3] = {Na, Nb, Nc};
    const int twf = p->arith == ARITH_F32 ? FMT_C64 : FMT_DF;
    for (int ax = 0; ax < 3; ++ax) {
        if (dev_malloc((void**)&p->tw[ax], twiddle_bytes(lens[ax], twf))) {
            cudaGetLastError();
            set_last_error(OPENFFT_ERR_NOMEM, "twiddle allocation failed");
            free_dist(p);
            return nullptr;
        }
        if ((e = launch_twiddles(lens[ax], twf, p->tw[ax], nullptr))) {
            set_last_error(OPENFFT_ERR_CUDA, cudaGetErrorString(e));
            free_dist(p);
            return nullptr;
        }
    }
    const int whiches[4] = {1, 2, -2, -1};
    for (int i = 0; i < 4; ++i) {
        make_side(whiches[i], Na, Nb, Nc, P, G, g, p->side[i]);
        const DistSide& d = p->side[i];
        DevTables& t = p->dt[i];
        if (upload(&t.q0, d.q0) || upload(&t.q1, d.q1) || upload(&t.sdispl, d.sdispl) || upload(&t.spre, d.spre) ||
            upload(&t.rdispl, d.rdispl) || upload(&t.rpre, d.rpre)) {
            set_last_error(OPENFFT_ERR_NOMEM, "exchange table allocation failed");
            free_dist(p);
            return nullptr;
        }
    }
    if ((e = cudaDeviceSynchronize())) { set_last_error(OPENFFT_ERR_CUDA, cudaGetErrorString(e)); free_dist(p); return nullptr; }
    return p;
}

void openfft_dist_destroy(openfft_dist_plan_t p) { free_dist(p); }

int openfft_dist_set_stream(openfft_dist_plan_t p, void* stream)
{
    if (!p) return set_last_error(OPENFFT_ERR_INVALID_ARG, "null plan");
    p->stream = static_cast<cudaStream_t>(stream);
    return OPENFFT_OK;
}

int openfft_dist_exchange_counts(openfft_dist_plan_t p, int exchange, int64_t* send_counts, int64_t* recv_counts)
{
    int sl, dl;
    if (!p || transpose_layouts(exchange, &sl, &dl)) return set_last_error(OPENFFT_ERR_INVALID_ARG, "plan or exchange");
    const DistSide& d = p->side[side_index(exchange)];
    for (int h = 0; h < p->G; ++h) {
        if (send_counts) send_counts[h] = d.send[h];
        if (recv_counts) recv_counts[h] = d.recv[h];
    }
    return OPENFFT_OK;
}

int openfft_dist_elem_bytes(openfft_dist_plan_t p)
{
    if (!p) return set_last_error(OPENFFT_ERR_INVALID_ARG, "null plan");
    return p->arith == ARITH_F32 ? 8 : 16;
}

int openfft_dist_stage(openfft_dist_plan_t p, int stage, int dir, const void* in, void* out)
{
    if (!p || !in || !out) return set_last_error(OPENFFT_ERR_INVALID_ARG, "null plan or buffer");
    if (stage < 1 || stage > 3) return set_last_error(OPENFFT_ERR_INVALID_ARG, "stage must be 1, 2 or 3");
    if (dir != OPENFFT_FORWARD && dir != OPENFFT_BACKWARD) return set_last_error(OPENFFT_ERR_INVALID_ARG, "dir must be -1 or +1");
    // forward: c-lines of abc, b-lines of cab, a-lines of cba; backward the reverse
    static const int fwd_layout[3] = {ABC, CAB, CBA};
    const int layout = dir == OPENFFT_FORWARD ? fwd_layout[stage - 1] : fwd_layout[3 - stage];
    const int axis = layout == ABC ? 2 : (layout == CAB ? 1 : 0);        // transformed axis
    const int lens[3] = {p->Na, p->Nb, p->Nc};
    const int n = lens[axis];
    const Ordering o = ordering_of(layout, p->Na, p->Nb, p->Nc, p->P);
    int64_t R0, R1;
    device_rows(o, p->G, p->g, &R0, &R1);
    const int64_t lines = R1 - R0;
    if (lines == 0) return OPENFFT_OK;
    const bool f32 = p->arith == ARITH_F32;
    const int ext = f32 ? FMT_C64 : FMT_C128, mid = f32 ? FMT_C64 : FMT_DF;
    StageLaunch L;
    std::memset(&L, 0, sizeof(L));
    StageArgs& a = L.args;
    radix_plan_of(n, a);
    const int E = f32 ? 8 : 16;
    int G = f32 ? 16 : 8;
    while (G > 1 && (int64_t)(G / 2) >= lines) G /= 2;
    while (G > 1 && 2 * (size_t)n * (G + 1) * E > 200 * 1024) G /= 2;
    if (2 * (size_t)n * (G + 1) * E > 200 * 1024) return set_last_error(OPENFFT_ERR_UNSUPPORTED_RADIX, "axis too long for one CTA");
    int lg = 0;
    while ((1 << lg) < G) ++lg;
    a.in = in; a.out = out;
    a.tw = p->tw[axis];
    a.M1 = lines; a.M2 = 1; a.S1 = n; a.S2 = 0; a.Sk = 1;
    a.ngroups = (lines + G - 1) / G;
    a.n = n; a.G = G; a.log2G = lg;
    a.group_i2 = 0; a.contig_store = 1; a.do_fft = 1;
    a.in_fmt = stage == 1 ? ext : mid;
    a.out_fmt = stage == 3 ? ext : mid;
    a.conj_in = (dir == OPENFFT_BACKWARD && stage == 1) ? 1 : 0;
    a.conj_out = (dir == OPENFFT_BACKWARD && stage == 3) ? 1 : 0;
    a.scale = a.conj_out ? 1.0 / ((double)p->Na * p->Nb * p->Nc) : 1.0;
    L.arith = p->arith;
    L.grid = a.ngroups;
    L.smem = 2 * (size_t)n * (G + 1) * E;
    L.sms = p->sms;
    L.family = KERNEL_AUTO;
    if (L.grid > 0x7fffffffLL) return set_last_error(OPENFFT_ERR_UNSUPPORTED, "grid too large");
    cudaError_t e = launch_stage(L, p->stream);
    return e ? set_last_error(OPENFFT_ERR_CUDA, cudaGetErrorString(e)) : OPENFFT_OK;
}

int openfft_dist_pack(openfft_dist_plan_t p, int exchange, const void* src, void* send)
{
    int sl, dl;
    if (!p || transpose_layouts(exchange, &sl, &dl) || !src || !send)
        return set_last_error(OPENFFT_ERR_INVALID_ARG, "plan, exchange or buffers");
    const int i = side_index(exchange);
    const DistSide& d = p->side[i];
    const DevTables& t = p->dt[i];
    const int64_t n = (d.R1 - d.R0) * row_len(d.t);
    if (n == 0) return OPENFFT_OK;
    const unsigned grid = (unsigned)std::min<int64_t>((n + 255) / 256, (int64_t)p->sms * 8);
    Bounds bnd;                                  // the send buffer holds this device's n elements
    bnd.chk = fallback_status_word(); bnd.lim = n;
    if (p->arith == ARITH_F32)
        dist_pack_kernel<float2><<<grid, 256, 0, p->stream>>>(d.t, p->P, p->G, d.R0, n, t.q0, t.q1, t.sdispl, t.spre,
                                                             static_cast<const float2*>(src), static_cast<float2*>(send), bnd);
    else
        dist_pack_kernel<double2><<<grid, 256, 0, p->stream>>>(d.t, p->P, p->G, d.R0, n, t.q0, t.q1, t.sdispl, t.spre,
                                                              static_cast<const double2*>(src), static_cast<double2*>(send), bnd);
    cudaError_t e = cudaGetLastError();
    return e ? set_last_error(OPENFFT_ERR_CUDA, cudaGetErrorString(e)) : OPENFFT_OK;
}

int openfft_dist_unpack(openfft_dist_plan_t p, int exchange, const void* recv, void* dst)
{
    int sl, dl;
    if (!p || transpose_layouts(exchange, &sl, &dl) || !recv || !dst)
        return set_last_error(OPENFFT_ERR_INVALID_ARG, "plan, exchange or buffers");
    const int i = side_index(exchange);
    const DistSide& d = p->side[i];
    const DevTables& t = p->dt[i];
    const int64_t n = (d.Q1 - d.Q0) * dst_row_len(d.t);
    if (n == 0) return OPENFFT_OK;
    const unsigned grid = (unsigned)std::min<int64_t>((n + 255) / 256, (int64_t)p->sms * 8);
    Bounds bnd;                                  // the receive buffer holds this device's n elements
    bnd.chk = fallback_status_word(); bnd.lim = n;
    if (p->arith == ARITH_F32)
        dist_unpack_kernel<float2><<<grid, 256, 0, p->stream>>>(d.t, p->P, p->G, d.Q0, d.Q1, n, t.rdispl, t.rpre,
                                                               static_cast<const float2*>(recv), static_cast<float2*>(dst), bnd);
    else
        dist_unpack_kernel<double2><<<grid, 256, 0, p->stream>>>(d.t, p->P, p->G, d.Q0, d.Q1, n, t.rdispl, t.rpre,
                                                                static_cast<const double2*>(recv), static_cast<double2*>(dst), bnd);
    cudaError_t e = cudaGetLastError();
    return e ? set_last_error(OPENFFT_ERR_CUDA, cudaGetErrorString(e)) : OPENFFT_OK;
}

}  // extern "C"
