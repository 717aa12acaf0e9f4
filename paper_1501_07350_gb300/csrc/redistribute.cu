// redistribute.cu -- the explicit transpose variants V0 and V1: steps (4)-(6)
// of OpenFFT's execution flow (Duy & Ozaki, Sec. 3.1.1) among P logical ranks
// that share one GPU's memory.
//
//   pack      (step 4): every element of the source ordering is written into
//             the send segment (r -> s) of its owner r, at its rank in
//             ascending source index inside that segment;
//   exchange  (step 5): every segment is copied to the receive buffer of s,
//             segments from lower source ranks first (one all-to-all with
//             variable counts, the Alltoallv / Isend-Irecv-Waitall methods);
//   unpack    (step 6): every element of the destination ordering is read from
//             the receive buffer (V0) or straight from the sender's segment
//             (V1, the unpack-on-arrival of Isend_Waitsome) and stored in place.
//
// Positions come from the closed forms of decomp.h; per rank pair the plan
// precomputes base offsets so each element needs only its own row's prefix.
#include "redistribute.h"

namespace ofg {

template <class E>
__global__ void pack_kernel(const Transpose t, const E* __restrict__ src, E* __restrict__ send,
                            const int64_t* __restrict__ sbase, int64_t N, const Bounds b)
{
    const int64_t P = t.src.P;
    const int64_t Ls = row_len(t), Ld = dst_row_len(t);
    for (int64_t x = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; x < N;
         x += (int64_t)gridDim.x * blockDim.x) {
        const int64_t q = x / Ls, e = x - q * Ls;
        const int64_t r = row_owner(t.src, q);
        const int64_t y = dest_index(t, q, e);
        const int64_t s = row_owner(t.dst, y / Ld);
        const int64_t Q0 = row_begin(t.dst, s), Q1 = row_begin(t.dst, s + 1);
        int64_t e_lo, cnt;
        row_range(t, q, Q0, Q1, &e_lo, &cnt);
        const int64_t pos = sbase[r * P + s] + prefix_to(t, q, Q0, Q1) + (e - e_lo);
        if (in_bounds(b, pos)) send[pos] = src[x];
    }
}

// chunks: (src offset, dst offset, length) triples, one CTA per chunk
template <class E>
__global__ void exchange_kernel(const int64_t* __restrict__ chunks, int64_t nchunks,
                                const E* __restrict__ send, E* __restrict__ recv, const Bounds b)
{
    for (int64_t c = blockIdx.x; c < nchunks; c += gridDim.x) {
        const int64_t so = chunks[3 * c], ro = chunks[3 * c + 1], len = chunks[3 * c + 2];
        for (int64_t j = threadIdx.x; j < len; j += blockDim.x)
            if (in_bounds(b, so + j) && in_bounds(b, ro + j)) recv[ro + j] = send[so + j];
    }
}

// from_send = 0: buf is the receive buffer, base indexed [s * P + r];
// from_send = 1: buf is the send buffer,    base indexed [r * P + s].
template <class E>
__global__ void unpack_kernel(const Transpose t, const E* __restrict__ buf, E* __restrict__ dst,
                              const int64_t* __restrict__ base, int from_send, int64_t N, const Bounds bd)
{
    const int64_t P = t.src.P;
    const int64_t Ld = dst_row_len(t);
    for (int64_t y = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; y < N;
         y += (int64_t)gridDim.x * blockDim.x) {
        int64_t q, e;
        source_of(t, y, &q, &e);
        const int64_t r = row_owner(t.src, q);
        const int64_t s = row_owner(t.dst, y / Ld);
        const int64_t Q0 = row_begin(t.dst, s), Q1 = row_begin(t.dst, s + 1);
        int64_t e_lo, cnt;
        row_range(t, q, Q0, Q1, &e_lo, &cnt);
        const int64_t rank = prefix_to(t, q, Q0, Q1) + (e - e_lo);
        const int64_t b = from_send ? base[r * P + s] : base[s * P + r];
        if (in_bounds(bd, b + rank)) dst[y] = buf[b + rank];
    }
}

// ------------------------------------------------- stepped schedules ----
//
// The paper's methods differ in how the P x P segments are scheduled:
//   per sender  (Isend_Waitall):           step r moves the segments (r, s), all s;
//   blocked     (Isend_Wait*_Block):       groups of B ranks; step k moves the pairs
//                                          (r, s) with floor(s/B) = (floor(r/B) + k) mod G,
//                                          G = ceil(P/B) steps in total;
//   shifted     (Sendrecv):                step i moves the pairs (r, (r + i) mod P).
// pair_of maps (step, index within the step) to (r, s); -1 if the index is empty.

__device__ __forceinline__ void pair_of(int sched, int64_t P, int64_t B, int64_t step, int64_t idx,
                                        int64_t* r, int64_t* s)
{
    if (sched == SCHED_PER_SENDER) { *r = step; *s = idx; return; }
    if (sched == SCHED_SHIFTED) { *r = idx; *s = (idx + step) % P; return; }
    // blocked: idx = r * B + j
    const int64_t G = (P + B - 1) / B;
    const int64_t rr = idx / B, j = idx - rr * B;
    const int64_t ss = ((rr / B + step) % G) * B + j;
    *r = rr;
    *s = ss < P ? ss : -1;
}

int64_t pairs_per_step(int sched, int64_t P, int64_t B)
{
    if (sched == SCHED_BLOCKED) return P * B;
    return P;
}

int64_t num_steps(int sched, int64_t P, int64_t B)
{
    if (sched == SCHED_BLOCKED) return (P + B - 1) / B;
    return P;
}

// blockIdx.x: pair of the step; blockIdx.y (of gridDim.y): share of the pair,
// so that a step with few pairs still spreads over the GPU.  Copy segment
// (r, s) from its send displacement to its receive displacement.
template <class E>
__global__ void segment_exchange_kernel(int sched, int64_t P, int64_t B, int64_t step,
                                        const int64_t* __restrict__ C, const int64_t* __restrict__ sdispl,
                                        const int64_t* __restrict__ rdispl, const E* __restrict__ send,
                                        E* __restrict__ recv, const Bounds b)
{
    int64_t r, s;
    pair_of(sched, P, B, step, blockIdx.x, &r, &s);
    if (s < 0) return;
    const int64_t len = C[r * P + s];
    const int64_t so = sdispl[r * P + s], ro = rdispl[s * P + r];
    const E* src = send + so;
    E* dst = recv + ro;
    const int64_t stride = (int64_t)gridDim.y * blockDim.x;
    for (int64_t j = (int64_t)blockIdx.y * blockDim.x + threadIdx.x; j < len; j += stride)
        if (in_bounds(b, so + j) && in_bounds(b, ro + j)) dst[j] = src[j];
}

// blockIdx.x: pair of the step, blockIdx.y: share of it.  The receiver takes
// the elements of segment (r, s) straight from the sender's send buffer and
// writes them to their places in the destination ordering (unpack on
// arrival).  Threads walk the source rows of rank r; each row holds a
// contiguous run of elements for s.
template <class E>
__global__ void segment_unpack_kernel(const Transpose t, int sched, int64_t B, int64_t step,
                                      const E* __restrict__ send, E* __restrict__ dst,
                                      const int64_t* __restrict__ sbase, const Bounds b)
{
    const int64_t P = t.src.P;
    int64_t r, s;
    pair_of(sched, P, B, step, blockIdx.x, &r, &s);
    if (s < 0) return;
    const int64_t R0 = row_begin(t.src, r), R1 = row_begin(t.src, r + 1);
    const int64_t Q0 = row_begin(t.dst, s), Q1 = row_begin(t.dst, s + 1);
    const int64_t base = sbase[r * P + s];
    const int64_t stride = (int64_t)gridDim.y * blockDim.x;
    for (int64_t q = R0 + (int64_t)blockIdx.y * blockDim.x + threadIdx.x; q < R1; q += stride) {
        int64_t e_lo, cnt;
        row_range(t, q, Q0, Q1, &e_lo, &cnt);
        if (cnt <= 0) continue;
        const int64_t pos = base + prefix_to(t, q, Q0, Q1);
        for (int64_t e = 0; e < cnt; ++e) {
            const int64_t y = dest_index(t, q, e_lo + e);
            if (in_bounds(b, y) && in_bounds(b, pos + e)) dst[y] = send[pos + e];
        }
    }
}

// Shares per pair: enough CTAs for four per SM over the pairs of a step.
static dim3 step_grid(int64_t pairs)
{
    static int sms = 0;
    if (!sms) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (sms < 1) sms = 1;
    }
    int64_t y = (4 * (int64_t)sms + pairs - 1) / pairs;
    if (y < 1) y = 1;
    if (y > 1024) y = 1024;
    return dim3((unsigned)pairs, (unsigned)y);
}

cudaError_t launch_segment_exchange(int sched, int64_t P, int64_t B, int64_t step, int elem_bytes,
                                    const int64_t* C, const int64_t* sdispl, const int64_t* rdispl,
                                    const void* send, void* recv, cudaStream_t st, const Bounds& b)
{
    const dim3 grid = step_grid(pairs_per_step(sched, P, B));
    if (elem_bytes == 16)
        segment_exchange_kernel<uint4><<<grid, 128, 0, st>>>(sched, P, B, step, C, sdispl, rdispl,
                                                             (const uint4*)send, (uint4*)recv, b);
    else
        segment_exchange_kernel<uint2><<<grid, 128, 0, st>>>(sched, P, B, step, C, sdispl, rdispl,
                                                             (const uint2*)send, (uint2*)recv, b);
    return cudaGetLastError();
}

cudaError_t launch_segment_unpack(const Transpose& t, int sched, int64_t B, int64_t step, int elem_bytes,
                                  const void* send, void* dst, const int64_t* sbase, cudaStream_t st,
                                  const Bounds& b)
{
    const dim3 grid = step_grid(pairs_per_step(sched, t.src.P, B));
    if (elem_bytes == 16)
        segment_unpack_kernel<uint4><<<grid, 128, 0, st>>>(t, sched, B, step, (const uint4*)send, (uint4*)dst, sbase, b);
    else
        segment_unpack_kernel<uint2><<<grid, 128, 0, st>>>(t, sched, B, step, (const uint2*)send, (uint2*)dst, sbase, b);
    return cudaGetLastError();
}

static unsigned grid_for(int64_t N, int sms)
{
    int64_t want = (N + 255) / 256;
    int64_t cap = (int64_t)sms * 16;
    return (unsigned)(want < cap ? (want > 0 ? want : 1) : cap);
}

cudaError_t launch_pack(const Transpose& t, int elem_bytes, const void* src, void* send,
                        const int64_t* sbase, int64_t N, int sms, cudaStream_t st, const Bounds& b)
{
    if (N == 0) return cudaSuccess;
    if (elem_bytes == 16)
        pack_kernel<uint4><<<grid_for(N, sms), 256, 0, st>>>(t, (const uint4*)src, (uint4*)send, sbase, N, b);
    else
        pack_kernel<uint2><<<grid_for(N, sms), 256, 0, st>>>(t, (const uint2*)src, (uint2*)send, sbase, N, b);
    return cudaGetLastError();
}

cudaError_t launch_exchange(int elem_bytes, const int64_t* chunks, int64_t nchunks,
                            const void* send, void* recv, int sms, cudaStream_t st, const Bounds& b)
{
    if (nchunks == 0) return cudaSuccess;
    int64_t cap = (int64_t)sms * 16;
    unsigned grid = (unsigned)(nchunks < cap ? nchunks : cap);
    if (elem_bytes == 16)
        exchange_kernel<uint4><<<grid, 256, 0, st>>>(chunks, nchunks, (const uint4*)send, (uint4*)recv, b);
    else
        exchange_kernel<uint2><<<grid, 256, 0, st>>>(chunks, nchunks, (const uint2*)send, (uint2*)recv, b);
    return cudaGetLastError();
}

cudaError_t launch_unpack(const Transpose& t, int elem_bytes, const void* buf, void* dst,
                          const int64_t* base, int from_send, int64_t N, int sms, cudaStream_t st,
                          const Bounds& b)
{
    if (N == 0) return cudaSuccess;
    if (elem_bytes == 16)
        unpack_kernel<uint4><<<grid_for(N, sms), 256, 0, st>>>(t, (const uint4*)buf, (uint4*)dst, base, from_send, N, b);
    else
        unpack_kernel<uint2><<<grid_for(N, sms), 256, 0, st>>>(t, (const uint2*)buf, (uint2*)dst, base, from_send, N, b);
    return cudaGetLastError();
}

// ------------------------------------------------------------ host tables --

void build_transpose_tables(const Transpose& t, std::vector<int64_t>& C, std::vector<int64_t>& sbase,
                            std::vector<int64_t>& rbase, std::vector<int64_t>& chunks, int64_t chunk_len,
                            std::vector<int64_t>* sdispl_out, std::vector<int64_t>* rdispl_out)
{
    const int64_t P = t.src.P;
    C.assign((size_t)(P * P), 0);
    std::vector<int64_t> pre((size_t)(P * P));   // prefix_to(R0_r) for destination s
    for (int64_t r = 0; r < P; ++r)
        for (int64_t s = 0; s < P; ++s) {
            const int64_t Q0 = row_begin(t.dst, s), Q1 = row_begin(t.dst, s + 1);
            const int64_t R0 = row_begin(t.src, r), R1 = row_begin(t.src, r + 1);
            const int64_t a = prefix_to(t, R0, Q0, Q1);
            C[(size_t)(r * P + s)] = prefix_to(t, R1, Q0, Q1) - a;
            pre[(size_t)(r * P + s)] = a;
        }
    sbase.assign((size_t)(P * P), 0);
    rbase.assign((size_t)(P * P), 0);
    std::vector<int64_t> sdispl((size_t)(P * P)), rdispl((size_t)(P * P));
    for (int64_t r = 0; r < P; ++r) {
        int64_t off = box_begin(t.src, r);
        for (int64_t s = 0; s < P; ++s) {
            sdispl[(size_t)(r * P + s)] = off;
            sbase[(size_t)(r * P + s)] = off - pre[(size_t)(r * P + s)];
            off += C[(size_t)(r * P + s)];
        }
    }
    for (int64_t s = 0; s < P; ++s) {
        int64_t off = box_begin(t.dst, s);
        for (int64_t r = 0; r < P; ++r) {
            rdispl[(size_t)(s * P + r)] = off;
            rbase[(size_t)(s * P + r)] = off - pre[(size_t)(r * P + s)];
            off += C[(size_t)(r * P + s)];
        }
    }
    if (sdispl_out) *sdispl_out = sdispl;
    if (rdispl_out) *rdispl_out = rdispl;
    chunks.clear();
    for (int64_t s = 0; s < P; ++s)
        for (int64_t r = 0; r < P; ++r) {
            int64_t len = C[(size_t)(r * P + s)];
            int64_t so = sdispl[(size_t)(r * P + s)], ro = rdispl[(size_t)(s * P + r)];
            for (int64_t j = 0; j < len; j += chunk_len) {
                chunks.push_back(so + j);
                chunks.push_back(ro + j);
                chunks.push_back(len - j < chunk_len ? len - j : chunk_len);
            }
        }
}

}  // namespace ofg
