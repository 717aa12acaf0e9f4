// batch.cu -- many 3-D transforms of uneven sizes in one persistent launch,
// replayed from a captured CUDA graph.
//
// Work items are runs of up to kTilesPerItem (16) tiles (of G lines each) of one
// stage of one transform, handed out
// in stage-major order (every stage-1 tile of every transform, then every
// stage-2 tile, then every stage-3 tile) through one atomic queue head.  A
// stage-s item of transform i first waits until all stage-(s-1) tiles of
// transform i are done (a per-(stage, transform) counter).  Those items have
// lower queue indices, so they were handed to CTAs that were already running
// and that never wait on anything later: the waits always end.  Each wait is
// still bounded (clock64 budget); on expiry the kernel records
// OPENFFT_ERR_TIMEOUT in a status word, every CTA stops taking items, and the
// host reads the status at openfft_sync.
//
// Per item the CTA runs the same stage computation as the single-transform
// path: compile-time-specialised tile bodies for the common lengths, the
// generic body otherwise.  Data written by one CTA and read by another in a
// later stage is loaded with cp.async.cg (through L2, not L1) after an
// acquire on the counter; writers fence before releasing.
#include <cuda_runtime.h>

#include <cstring>
#include <vector>

#include "../../include/openfft_gb.h"
#include "batch.h"
#include "fft_stage.h"
#include "fft_tile.cuh"
#include "generic_stage.cuh"

namespace ofg {

constexpr int kBatchThreads = 256;
constexpr int kTilesPerItem = 16;          // tiles of one (stage, transform) per work item (the
                                           // queue and dependency work of an item is serial)

struct BatchCounters {
    unsigned long long next;   // queue head
    int status;                // OPENFFT_OK or OPENFFT_ERR_TIMEOUT
    int pad;
    // followed by done[3 * count]
};

struct BatchDev {
    const StageArgs* stages;       // [2 directions][3 stages][count]
    const int64_t* item_base;      // [3 * count + 1]: queue index of the first tile of (stage, transform)
    const unsigned* need;          // [3 * count]: tiles of (stage, transform)
    void* const* ptrs;             // [2 * count]: in_i, out_i (device pointers)
    void* const* scratch;          // [count]
    BatchCounters* ctr;
    unsigned* done;                // [3 * count]
    int count;
    int dir_index;                 // 0 forward, 1 backward
    long long wait_budget;         // clock64 cycles
};

// Tiles [t0, t1) of one stage of one transform; the next tile's lines are
// copied into the second buffer while the current tile is transformed.
template <class A, int N, int G>
__device__ __noinline__ void tile_item(const StageArgs& p, int64_t t0, int64_t t1, typename A::C* buf,
                                       int tid)
{
    using C = typename A::C;
    constexpr int T = kBatchThreads;
    C* cur = buf;
    C* nxt = buf + Tile<A, N, G, T>::kElems;
    const bool convert = Io<A>::kConverts && p.in_fmt == FMT_C128;
    tile_issue_loads<A, N, G, T>(p, tile_geom(p, t0, G), cur, tid);
    for (int64_t t = t0; t < t1; ++t) {
        const TileGeom tg = tile_geom(p, t, G);
        cp_async_wait_all();
        if (convert) { if (p.conj_in) tile_fix<A, N, G, T, true, true>(cur, tid); else tile_fix<A, N, G, T, true, false>(cur, tid); }
        else if (p.conj_in) tile_fix<A, N, G, T, false, true>(cur, tid);
        __syncthreads();
        if (t + 1 < t1) tile_issue_loads<A, N, G, T>(p, tile_geom(p, t + 1, G), nxt, tid);
        Tile<A, N, G, T>::template passes<0>(cur + tid % G, reinterpret_cast<const typename A::W*>(p.tw), tid / G);
        tile_store_dispatch<A, N, G, T>(p, tg, cur, tid);
        __syncthreads();
        C* x = cur; cur = nxt; nxt = x;
    }
    cp_async_wait_all();
}

// the tile bodies are compiled for G lines per tile; contiguous tile stores
// assume the lines of the output in order
template <int G>
__device__ __forceinline__ bool tile_ok(const StageArgs& p)
{
    return p.G == G && (!p.contig_store || (!p.group_i2 && p.S1 == p.n && p.Sk == 1));
}

// Shared-memory layout of the batched kernel: [tile buffer | queue prefix
// item_base (3 count + 1 int64) | tile counts need (3 count uint32)].
template <class A, int G>
__global__ void __launch_bounds__(kBatchThreads, sizeof(typename A::C) == 8 ? 3 : 2)
batch_kernel(const BatchDev d, size_t buf_bytes)
{
    using C = typename A::C;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ int64_t s_in[kMaxLinesPerCta];
    __shared__ int64_t s_out[kMaxLinesPerCta];
    __shared__ StageArgs s_p;
    __shared__ int64_t s_tile;        // first tile of the item
    __shared__ int s_q, s_abort;
    const int tid = threadIdx.x;
    const int nq = 3 * d.count;
    int64_t* sh_base = reinterpret_cast<int64_t*>(smem_raw + buf_bytes);
    unsigned* sh_need = reinterpret_cast<unsigned*>(sh_base + nq + 1);
    for (int k = tid; k <= nq; k += kBatchThreads) sh_base[k] = d.item_base[k];
    for (int k = tid; k < nq; k += kBatchThreads) sh_need[k] = d.need[k];
    __syncthreads();
    const int64_t total = sh_base[nq];
    volatile int* status = &d.ctr->status;

    for (;;) {
        if (tid == 0) {
            const int64_t j = (int64_t)atomicAdd(&d.ctr->next, 1ull);
            int abort = *status != OPENFFT_OK || j >= total;
            int q = 0;
            if (!abort) {
                // (stage, transform) of item j: last q with item_base[q] <= j
                int lo = 0, hi = nq - 1;
                while (lo < hi) {
                    const int mid = (lo + hi + 1) >> 1;
                    if (sh_base[mid] <= j) lo = mid; else hi = mid - 1;
                }
                q = lo;
                const int s = q / d.count;
                if (s > 0) {
                    volatile unsigned* cnt = &d.done[q - d.count];
                    const unsigned want = sh_need[q - d.count];
                    const long long t0 = clock64();
                    while (*cnt < want) {
                        if (*status != OPENFFT_OK) { abort = 1; break; }
                        if (clock64() - t0 > d.wait_budget) {
                            atomicCAS(&d.ctr->status, OPENFFT_OK, OPENFFT_ERR_TIMEOUT);
                            abort = 1;
                            break;
                        }
                        __nanosleep(128);
                    }
                    __threadfence();               // acquire: order the loads after the counter
                }
            }
            s_abort = abort;
            s_q = q;
            s_tile = abort ? 0 : (j - sh_base[q]) * kTilesPerItem;
        }
        __syncthreads();
        if (s_abort) break;
        const int q = s_q, s = q / d.count, i = q - s * d.count;
        // stage descriptor of (stage, transform) into shared memory, pointers patched
        if (tid < (int)(sizeof(StageArgs) / 4)) {
            reinterpret_cast<int*>(&s_p)[tid] = __ldg(reinterpret_cast<const int*>(&d.stages[d.dir_index * nq + q]) + tid);
        }
        __syncthreads();
        if (tid == 0) {
            void* in_i = d.ptrs[2 * i];
            void* out_i = d.ptrs[2 * i + 1];
            void* sc = d.scratch[i];
            s_p.in = s == 0 ? in_i : (s == 1 ? sc : out_i);
            s_p.out = s == 0 ? sc : out_i;
        }
        __syncthreads();
        const StageArgs& p = s_p;
        const int64_t t0 = s_tile;
        const int64_t ntile = p.ngroups * (p.group_i2 ? p.M1 : p.M2);
        const int64_t t1 = t0 + kTilesPerItem < ntile ? t0 + kTilesPerItem : ntile;
        C* buf = reinterpret_cast<C*>(smem_raw);
        bool done_item = false;
        if (tile_ok<G>(p)) {
            done_item = true;
            switch (p.n) {
            case 48: tile_item<A, 48, G>(p, t0, t1, buf, tid); break;
            case 64: tile_item<A, 64, G>(p, t0, t1, buf, tid); break;
            case 96: tile_item<A, 96, G>(p, t0, t1, buf, tid); break;
            case 100: tile_item<A, 100, G>(p, t0, t1, buf, tid); break;
            case 108: tile_item<A, 108, G>(p, t0, t1, buf, tid); break;
            case 120: tile_item<A, 120, G>(p, t0, t1, buf, tid); break;
            default: done_item = false; break;
            }
        }
        if (!done_item)
            for (int64_t t = t0; t < t1; ++t) {
                generic_stage_tile<A>(p, t, smem_raw, s_in, s_out);
                __syncthreads();
            }
        __threadfence();                           // release this thread's stores
        __syncthreads();
        if (tid == 0) atomicAdd(&d.done[q], 1u);
    }
}

// --------------------------------------------------------------- host ----

namespace {

bool radix_plan(int n, StageArgs& a)
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

int lg2(int g) { int l = 0; while ((1 << l) < g) ++l; return l; }

}  // namespace

struct BatchPlan {
    int count = 0, dtype = 0, arith = 0, G = 8;
    std::vector<int> dims;                     // 3 * count
    std::vector<int64_t> N;                    // per transform
    size_t smem = 0;
    int grid = 0;
    // device memory
    StageArgs* d_stages = nullptr;
    int64_t* d_item_base = nullptr;
    unsigned* d_need = nullptr;
    void** d_ptrs = nullptr;
    void** d_scratch = nullptr;
    unsigned char* d_ctr = nullptr;            // BatchCounters + done[3*count]
    size_t ctr_bytes = 0;
    std::vector<void*> scratch;
    std::vector<void*> twiddles;
    // host staging of the pointer table (page-locked, read by the graph's copy node)
    void** h_ptrs = nullptr;
    std::vector<void*> cur_ptrs;
    // graph
    cudaStream_t own = nullptr;
    cudaEvent_t ev_in = nullptr, ev_out = nullptr;
    cudaGraphExec_t exec[2] = {nullptr, nullptr};
    long long wait_budget = 2000000000LL;      // about one second of clock64 cycles
    unsigned need_extra = 0;                   // test hook: extra tiles the first wait expects
    int64_t items_per_stage[3] = {0, 0, 0};
};

static void free_batch(BatchPlan* b)
{
    if (!b) return;
    for (auto& e : b->exec) if (e) cudaGraphExecDestroy(e);
    if (b->own) cudaStreamDestroy(b->own);
    if (b->ev_in) cudaEventDestroy(b->ev_in);
    if (b->ev_out) cudaEventDestroy(b->ev_out);
    cudaFree(b->d_stages); cudaFree(b->d_item_base); cudaFree(b->d_need);
    cudaFree(b->d_ptrs); cudaFree(b->d_scratch); cudaFree(b->d_ctr);
    for (void* p : b->scratch) cudaFree(p);
    for (void* p : b->twiddles) cudaFree(p);
    if (b->h_ptrs) cudaFreeHost(b->h_ptrs);
    delete b;
}

void batch_destroy(BatchPlan* b) { free_batch(b); }

int batch_create(int count, const int* dims, const int* P, int dtype, int sms, BatchPlan** out,
                 int (*fail)(int, const char*))
{
    if (count < 1 || !dims || !P) return fail(OPENFFT_ERR_INVALID_ARG, "count >= 1 and non-null arrays required");
    if (dtype != OPENFFT_C2C_F64 && dtype != OPENFFT_C2C_F32) return fail(OPENFFT_ERR_UNSUPPORTED, "batched plans take F64 or F32");
    BatchPlan* b = new BatchPlan();
    b->count = count;
    b->dtype = dtype;
    b->arith = dtype == OPENFFT_C2C_F32 ? ARITH_F32 : ARITH_DF;
    b->G = dtype == OPENFFT_C2C_F32 ? 16 : 8;
    b->dims.assign(dims, dims + 3 * count);
    const int E = dtype == OPENFFT_C2C_F32 ? 8 : 16;
    const int ext = dtype == OPENFFT_C2C_F32 ? FMT_C64 : FMT_C128;
    const int mid = dtype == OPENFFT_C2C_F32 ? FMT_C64 : FMT_DF;
    const int twf = dtype == OPENFFT_C2C_F32 ? FMT_C64 : FMT_DF;
    std::vector<StageArgs> st((size_t)2 * 3 * count);
    cudaError_t e;
    // twiddle tables per distinct length
    std::vector<int> tw_len;
    auto twiddle_for = [&](int n) -> const void* {
        for (size_t k = 0; k < tw_len.size(); ++k) if (tw_len[k] == n) return b->twiddles[k];
        void* t = nullptr;
        if (dev_malloc((void**)&t, twiddle_bytes(n, twf))) return nullptr;
        if (launch_twiddles(n, twf, t, nullptr)) { cudaFree(t); return nullptr; }
        tw_len.push_back(n);
        b->twiddles.push_back(t);
        return t;
    };
    for (int i = 0; i < count; ++i) {
        const int64_t Na = dims[3 * i], Nb = dims[3 * i + 1], Nc = dims[3 * i + 2];
        if (Na < 1 || Nb < 1 || Nc < 1 || P[i] < 1) { free_batch(b); return fail(OPENFFT_ERR_INVALID_ARG, "sizes and P must be >= 1"); }
        if (P[i] > Na * Nb || P[i] > Nc * Na || P[i] > Nc * Nb) { free_batch(b); return fail(OPENFFT_ERR_P_TOO_LARGE, "P exceeds N1*N2 of an ordering (Eq. 2 undefined)"); }
        const int64_t N = Na * Nb * Nc;
        b->N.push_back(N);
        void* sc = nullptr;
        if (dev_malloc((void**)&sc, (size_t)N * E)) { cudaGetLastError(); free_batch(b); return fail(OPENFFT_ERR_NOMEM, "batched workspace"); }
        b->scratch.push_back(sc);
        // forward / backward stage geometry, as in the fused single-transform path
        struct Geo { int64_t n, M1, M2, S1, S2, Sk; int g2, contig, in_fmt, out_fmt, cin, cout; double scale; };
        const double invN = 1.0 / (double)N;
        const Geo geo[2][3] = {
            {{Nc, Na * Nb, 1, 1, 0, Na * Nb, 0, 0, ext, mid, 0, 0, 1.0},
             {Nb, Na, Nc, 1, Nb * Na, Na, 0, 0, mid, mid, 0, 0, 1.0},
             {Na, Nc * Nb, 1, Na, 0, 1, 0, 1, mid, ext, 0, 0, 1.0}},
            {{Na, Nb, Nc, 1, Na * Nb, Nb, 0, 0, ext, mid, 1, 0, 1.0},
             {Nb, Na, Nc, Nb * Nc, 1, Nc, 1, 0, mid, mid, 0, 0, 1.0},
             {Nc, Na * Nb, 1, Nc, 0, 1, 0, 1, mid, ext, 0, 1, invN}}};
        for (int dir = 0; dir < 2; ++dir)
            for (int s = 0; s < 3; ++s) {
                const Geo& g = geo[dir][s];
                StageArgs& a = st[(size_t)dir * 3 * count + (size_t)s * count + i];
                std::memset(&a, 0, sizeof(a));
                const int n = (int)g.n;
                if (n > kMaxLen || !radix_plan(n, a)) { free_batch(b); return fail(OPENFFT_ERR_UNSUPPORTED_RADIX, "axis length must factor into 2, 3, 5, 7 and be <= 2048"); }
                int G = b->G;
                const int64_t Mg = g.g2 ? g.M2 : g.M1;
                while (G > 1 && (int64_t)(G / 2) >= Mg) G /= 2;
                while (G > 1 && 2 * (size_t)n * (G + 1) * E > 200 * 1024) G /= 2;
                // the tile bodies are compiled for the plan's G: other widths take the generic body
                a.tw = twiddle_for(n);
                if (!a.tw) { cudaGetLastError(); free_batch(b); return fail(OPENFFT_ERR_NOMEM, "twiddle tables"); }
                a.M1 = g.M1; a.M2 = g.M2; a.S1 = g.S1; a.S2 = g.S2; a.Sk = g.Sk;
                a.ngroups = (Mg + G - 1) / G;
                a.scale = g.scale;
                a.n = n; a.G = G; a.log2G = lg2(G);
                a.group_i2 = g.g2; a.contig_store = g.contig;
                a.conj_in = g.cin; a.conj_out = g.cout; a.do_fft = 1;
                a.in_fmt = g.in_fmt; a.out_fmt = g.out_fmt;
                const size_t sm = 2 * (size_t)n * (G + 1) * E;
                if (sm > b->smem) b->smem = sm;
            }
    }
    b->ctr_bytes = sizeof(BatchCounters) + sizeof(unsigned) * (size_t)3 * count;
    if (dev_malloc((void**)&b->d_stages, st.size() * sizeof(StageArgs)) ||
        dev_malloc((void**)&b->d_item_base, sizeof(int64_t) * (size_t)(2 * (3 * count + 1))) ||
        dev_malloc((void**)&b->d_need, sizeof(unsigned) * (size_t)(2 * 3 * count)) ||
        dev_malloc((void**)&b->d_ptrs, sizeof(void*) * (size_t)(2 * count)) ||
        dev_malloc((void**)&b->d_scratch, sizeof(void*) * (size_t)count) ||
        dev_malloc((void**)&b->d_ctr, b->ctr_bytes) ||
        cudaMallocHost(&b->h_ptrs, sizeof(void*) * (size_t)(2 * count))) {
        cudaGetLastError();
        free_batch(b);
        return fail(OPENFFT_ERR_NOMEM, "batched plan tables");
    }
    // per direction (the two traverse the axes in opposite orders): tiles per
    // (stage, transform) and the stage-major queue prefix
    std::vector<int64_t> bases((size_t)2 * (3 * count + 1));
    std::vector<unsigned> needs((size_t)2 * 3 * count);
    for (int dir = 0; dir < 2; ++dir) {
        int64_t acc = 0;
        for (int q = 0; q < 3 * count; ++q) {
            const StageArgs& a = st[(size_t)dir * 3 * count + q];
            const int64_t tiles = a.ngroups * (a.group_i2 ? a.M1 : a.M2);
            const int64_t items = (tiles + kTilesPerItem - 1) / kTilesPerItem;
            bases[(size_t)dir * (3 * count + 1) + q] = acc;
            needs[(size_t)dir * 3 * count + q] = (unsigned)items;
            acc += items;
            if (dir == 0) b->items_per_stage[q / count] += items;
        }
        bases[(size_t)dir * (3 * count + 1) + 3 * count] = acc;
    }
    e = cudaMemcpy(b->d_stages, st.data(), st.size() * sizeof(StageArgs), cudaMemcpyHostToDevice);
    if (!e) e = cudaMemcpy(b->d_item_base, bases.data(), bases.size() * sizeof(int64_t), cudaMemcpyHostToDevice);
    if (!e) e = cudaMemcpy(b->d_need, needs.data(), needs.size() * sizeof(unsigned), cudaMemcpyHostToDevice);
    if (!e) e = cudaMemcpy(b->d_scratch, b->scratch.data(), sizeof(void*) * (size_t)count, cudaMemcpyHostToDevice);
    if (!e) e = cudaStreamCreateWithFlags(&b->own, cudaStreamNonBlocking);
    if (!e) e = cudaEventCreateWithFlags(&b->ev_in, cudaEventDisableTiming);
    if (!e) e = cudaEventCreateWithFlags(&b->ev_out, cudaEventDisableTiming);
    if (e) { free_batch(b); return fail(OPENFFT_ERR_CUDA, cudaGetErrorString(e)); }
    // launch shape: persistent, as many CTAs as fit (tile buffer + queue tables)
    b->smem = (b->smem + 15) & ~(size_t)15;
    const size_t tables = sizeof(int64_t) * (size_t)(3 * count + 1) + sizeof(unsigned) * (size_t)(3 * count);
    if (b->smem + tables > 200 * 1024) { free_batch(b); return fail(OPENFFT_ERR_UNSUPPORTED, "batch too large for the queue tables in shared memory"); }
    int per_sm = 1;
    if (b->arith == ARITH_F32)
        e = persistent_ctas_per_sm((const void*)batch_kernel<ArF32, 16>, kBatchThreads, b->smem + tables, &per_sm);
    else
        e = persistent_ctas_per_sm((const void*)batch_kernel<ArDF, 8>, kBatchThreads, b->smem + tables, &per_sm);
    if (e) { free_batch(b); return fail(OPENFFT_ERR_CUDA, cudaGetErrorString(e)); }
    b->grid = sms * (per_sm > 0 ? per_sm : 1);
    e = cudaDeviceSynchronize();
    if (e) { free_batch(b); return fail(OPENFFT_ERR_CUDA, cudaGetErrorString(e)); }
    *out = b;
    return OPENFFT_OK;
}

static cudaError_t launch_batch(BatchPlan* b, int dir_index, cudaStream_t s)
{
    BatchDev d;
    d.stages = b->d_stages;
    d.item_base = b->d_item_base + (size_t)dir_index * (3 * b->count + 1);
    d.need = b->d_need + (size_t)dir_index * 3 * b->count;
    d.ptrs = b->d_ptrs;
    d.scratch = b->d_scratch;
    d.ctr = reinterpret_cast<BatchCounters*>(b->d_ctr);
    d.done = reinterpret_cast<unsigned*>(b->d_ctr + sizeof(BatchCounters));
    d.count = b->count;
    d.dir_index = dir_index;
    d.wait_budget = b->wait_budget;
    cudaError_t e = cudaMemsetAsync(b->d_ctr, 0, b->ctr_bytes, s);
    if (e) return e;
    e = cudaMemcpyAsync(b->d_ptrs, b->h_ptrs, sizeof(void*) * (size_t)(2 * b->count), cudaMemcpyHostToDevice, s);
    if (e) return e;
    const size_t tables = sizeof(int64_t) * (size_t)(3 * b->count + 1) + sizeof(unsigned) * (size_t)(3 * b->count);
    const size_t sm = b->smem + tables;
    if (b->arith == ARITH_F32) batch_kernel<ArF32, 16><<<b->grid, kBatchThreads, sm, s>>>(d, b->smem);
    else batch_kernel<ArDF, 8><<<b->grid, kBatchThreads, sm, s>>>(d, b->smem);
    return cudaGetLastError();
}

int batch_exec(BatchPlan* b, const void* const* in, void* const* out, int dir, cudaStream_t user,
               int (*fail)(int, const char*))
{
    if (!b || !in || !out) return fail(OPENFFT_ERR_INVALID_ARG, "null plan or pointer arrays");
    if (dir != OPENFFT_FORWARD && dir != OPENFFT_BACKWARD) return fail(OPENFFT_ERR_INVALID_ARG, "dir must be -1 or +1");
    std::vector<void*> ptrs((size_t)2 * b->count);
    for (int i = 0; i < b->count; ++i) {
        if (!in[i] || !out[i]) return fail(OPENFFT_ERR_INVALID_ARG, "null transform buffer");
        if (in[i] == out[i]) return fail(OPENFFT_ERR_ALIAS, "in and out must differ (out-of-place only)");
        ptrs[(size_t)2 * i] = const_cast<void*>(in[i]);
        ptrs[(size_t)2 * i + 1] = out[i];
    }
    cudaError_t e;
    if (ptrs != b->cur_ptrs) {
        // the graph's copy node reads h_ptrs when it runs: wait for earlier replays first
        if ((e = cudaStreamSynchronize(b->own))) return fail(OPENFFT_ERR_CUDA, cudaGetErrorString(e));
        std::memcpy(b->h_ptrs, ptrs.data(), sizeof(void*) * ptrs.size());
        b->cur_ptrs = ptrs;
    }
    const int di = dir == OPENFFT_FORWARD ? 0 : 1;
    if (!b->exec[di]) {
        cudaGraph_t g = nullptr;
        if ((e = cudaStreamBeginCapture(b->own, cudaStreamCaptureModeThreadLocal))) return fail(OPENFFT_ERR_CUDA, cudaGetErrorString(e));
        cudaError_t le = launch_batch(b, di, b->own);
        e = cudaStreamEndCapture(b->own, &g);
        if (le || e) { if (g) cudaGraphDestroy(g); return fail(OPENFFT_ERR_CUDA, cudaGetErrorString(le ? le : e)); }
        e = cudaGraphInstantiate(&b->exec[di], g, 0);
        cudaGraphDestroy(g);
        if (e) { b->exec[di] = nullptr; return fail(OPENFFT_ERR_CUDA, cudaGetErrorString(e)); }
    }
    // order the replay after the caller's stream and the caller's stream after the replay
    if ((e = cudaEventRecord(b->ev_in, user))) return fail(OPENFFT_ERR_CUDA, cudaGetErrorString(e));
    if ((e = cudaStreamWaitEvent(b->own, b->ev_in, 0))) return fail(OPENFFT_ERR_CUDA, cudaGetErrorString(e));
    if ((e = cudaGraphLaunch(b->exec[di], b->own))) return fail(OPENFFT_ERR_CUDA, cudaGetErrorString(e));
    if ((e = cudaEventRecord(b->ev_out, b->own))) return fail(OPENFFT_ERR_CUDA, cudaGetErrorString(e));
    if ((e = cudaStreamWaitEvent(user, b->ev_out, 0))) return fail(OPENFFT_ERR_CUDA, cudaGetErrorString(e));
    return OPENFFT_OK;
}

int batch_status(BatchPlan* b, int (*fail)(int, const char*))
{
    cudaError_t e = cudaStreamSynchronize(b->own);
    if (e) return fail(OPENFFT_ERR_CUDA, cudaGetErrorString(e));
    BatchCounters c;
    e = cudaMemcpy(&c, b->d_ctr, sizeof(c), cudaMemcpyDeviceToHost);
    if (e) return fail(OPENFFT_ERR_CUDA, cudaGetErrorString(e));
    if (c.status != OPENFFT_OK) return fail(c.status, "a bounded dependency wait of the batched kernel ran out");
    return OPENFFT_OK;
}

int batch_set_wait_budget(BatchPlan* b, long long cycles)
{
    b->wait_budget = cycles;
    return OPENFFT_OK;
}

int batch_inject_stall(BatchPlan* b, int enable)
{
    // test hook (forward direction, stage 1 of transform 0): its stage-2 items
    // wait for one more stage-1 tile than exists, so the bounded wait runs out
    const size_t off = 0;
    unsigned v = 0;
    cudaError_t e = cudaMemcpy(&v, b->d_need + off, sizeof(unsigned), cudaMemcpyDeviceToHost);
    if (e) return OPENFFT_ERR_CUDA;
    const unsigned base = v - b->need_extra;
    b->need_extra = enable ? 1u : 0u;
    v = base + b->need_extra;
    e = cudaMemcpy(b->d_need + off, &v, sizeof(unsigned), cudaMemcpyHostToDevice);
    return e ? OPENFFT_ERR_CUDA : OPENFFT_OK;
}

int64_t batch_items(BatchPlan* b) { return b->items_per_stage[0] + b->items_per_stage[1] + b->items_per_stage[2]; }
int batch_count(BatchPlan* b) { return b->count; }
int64_t batch_points(BatchPlan* b, int i) { return b->N[(size_t)i]; }

}  // namespace ofg
