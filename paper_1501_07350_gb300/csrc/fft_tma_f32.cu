// fft_tma_f32.cu -- the FP32 warp kernel (two lines per warp, fft_warp.cuh)
// with the asynchronous transposed output of fft_warp_tma.cuh, for 256- and
// 512-point lines in tiles of 8 or 16.
//
// The radix passes are the warp kernel's.  The last one writes the tile into
// a staging area laid out as the output needs it,
// [k][G lines] of 8-byte elements in the tensor store's swizzle (16-byte
// chunk index = line / 2, XOR (k / 2) mod 4 for 64-byte rows, G = 8, or k mod 8
// for 128-byte rows, G = 16), and one thread hands it to a TMA tensor store;
// the threads go on with the next tile while the copy engine drains it.  The
// tiles stay double-buffered (the next tile's lines are copied in during the
// passes), and the staging area is separate, reused one tile later after the
// copy engine has read it.  Transposed stages without conjugation or scaling
// only (the fused variant's first two stages); the others keep the warp
// kernel's stores.
#include "fft_warp_tma.cuh"

namespace ofg {

namespace {

constexpr int kF32LinesPerWarp = 2;

template <int G>
__device__ __forceinline__ uint32_t staged_offset_f32(int k, int g)
{
    const uint32_t f = G == 16 ? (uint32_t)(k & 7) : (uint32_t)((k >> 1) & 3);
    return (uint32_t)k * (uint32_t)(8 * G) + (((uint32_t)(g >> 1) ^ f) << 4) + ((uint32_t)(g & 1) << 3);
}

template <int N, int G>
constexpr int f32_tma_threads() { return 32 * G / kF32LinesPerWarp; }

template <int N, int G>
constexpr size_t f32_tma_smem()
{
    // 1024-byte alignment slack, the staging area, two tile buffers
    return 1024 + (size_t)N * G * 8 + 2 * (size_t)G * warp_line_stride<8>(N) * 8;
}

template <int N, int G>
__global__ void __launch_bounds__(f32_tma_threads<N, G>(), G == 8 ? 4 : 2)
fft_warp_tma_f32_kernel(const StageArgs p, int64_t ntiles, const __grid_constant__ CUtensorMap tmap)
{
    using A = ArF32;
    using C = A::C;
    constexpr int L = kF32LinesPerWarp;
    constexpr int LS = warp_line_stride<8>(N);
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const uint32_t base = smem_addr(smem_raw);
    unsigned char* stage = smem_raw + (((base + 1023u) & ~1023u) - base);
    C* cur = reinterpret_cast<C*>(stage + (size_t)N * G * 8);
    C* nxt = cur + G * LS;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int g0 = warp * L;
    const A::W* tw = A::table(p.tw, N);

    int64_t tile = blockIdx.x;
    if (tile < ntiles) {
        const TileGeom tg = tile_geom(p, tile, G);
#pragma unroll
        for (int i = 0; i < L; ++i) warp_issue_load<A, N>(p, tg, g0 + i, cur + (g0 + i) * LS, lane);
    }
    for (; tile < ntiles; tile += gridDim.x) {
        C* line0 = cur + g0 * LS;
        cp_async_wait_all();
        if (p.conj_in) {
#pragma unroll
            for (int i = 0; i < L; ++i) warp_fix<A, N, false, true>(line0 + i * LS, lane);
        }
        __syncwarp();
        const int64_t next = tile + gridDim.x;
        if (next < ntiles) {
            const TileGeom tn = tile_geom(p, next, G);
#pragma unroll
            for (int i = 0; i < L; ++i) warp_issue_load<A, N>(p, tn, g0 + i, nxt + (g0 + i) * LS, lane);
        }
        WarpLine<A, N>::template passes_but_last<0, L>(line0, tw, lane);
        // the previous tile's store has read the staging area; the last pass
        // writes its results there
        if (tid == 0) bulk_wait_read_all();
        __syncthreads();
        WarpLine<A, N>::template pass_to<WarpLine<A, N>::kPasses - 1, L, 1>(
            line0, tw, lane,
            [=](int l, int k, const C& x) { *reinterpret_cast<C*>(stage + staged_offset_f32<G>(k, g0 + l)) = x; });
        fence_proxy_async_smem();
        __syncthreads();
        if (tid == 0) {
#pragma unroll
            for (int kb = 0; kb < (N + 255) / 256; ++kb)
                tma_store_3d(&tmap, smem_addr(stage) + (uint32_t)kb * 256u * (uint32_t)(G * 8),
                             (int)((tile % p.ngroups) * G * 2), kb * 256, (int)(tile / p.ngroups));
            bulk_commit();
        }
        C* t = cur; cur = nxt; nxt = t;
    }
    cp_async_wait_all();
    if (tid == 0) bulk_wait_all();
}

// The transposed output of 8-byte elements as a 3-D tensor of 4-byte words:
// (grouped line coordinate x 2, frequency, other line coordinate), box
// (G lines, 256 or n frequencies, 1).
bool transposed_store_map_f32(const StageArgs& a, int G, CUtensorMap* map)
{
    const int64_t Mg = a.group_i2 ? a.M2 : a.M1, Mo = a.group_i2 ? a.M1 : a.M2;
    const int64_t Sg = a.group_i2 ? a.S2 : a.S1, So = a.group_i2 ? a.S1 : a.S2;
    if (Sg != 1 || a.Sk < 1 || Mg * 2 > (int64_t)0xFFFFFFFF || Mo > 0xFFFFFFFF) return false;
    if ((reinterpret_cast<uintptr_t>(a.out) & 15) != 0) return false;
    TensorMapEncodeFn enc = tensor_map_encoder();
    if (!enc) return false;
    const int64_t s1 = a.Sk * 8;
    const int64_t s2 = Mo > 1 ? So * 8 : s1 * a.n;
    if ((s1 & 15) != 0 || (s2 & 15) != 0) return false;            // strides are 16-byte multiples
    if (s1 >= ((int64_t)1 << 40) || s2 >= ((int64_t)1 << 40) || s2 <= 0) return false;
    const cuuint64_t dims[3] = {(cuuint64_t)(Mg * 2), (cuuint64_t)a.n, (cuuint64_t)Mo};
    const cuuint64_t strides[2] = {(cuuint64_t)s1, (cuuint64_t)s2};
    const cuuint32_t box[3] = {(cuuint32_t)(2 * G), (cuuint32_t)(a.n < 256 ? a.n : 256), 1u};
    const cuuint32_t estr[3] = {1u, 1u, 1u};
    return enc(map, CU_TENSOR_MAP_DATA_TYPE_UINT32, 3, a.out, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
               G == 16 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_64B, CU_TENSOR_MAP_L2_PROMOTION_NONE,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

template <int N, int G>
cudaError_t launch_f32_tma_n(const StageLaunch& L, cudaStream_t st, bool* handled)
{
    const StageArgs& a = L.args;
    CUtensorMap map;
    std::memset(&map, 0, sizeof(map));
    if (!transposed_store_map_f32(a, G, &map)) return cudaSuccess;
#ifdef OPENFFT_CHECKED
    {   // the copy engine clips to the map's extent: take this kernel only inside the array
        const int64_t Mg = a.group_i2 ? a.M2 : a.M1, Mo = a.group_i2 ? a.M1 : a.M2;
        const int64_t So = a.group_i2 ? a.S1 : a.S2;
        if ((Mg - 1) + (int64_t)(a.n - 1) * a.Sk + (Mo > 1 ? (Mo - 1) * So : 0) >= a.out_elems) return cudaSuccess;
    }
#endif
    *handled = true;
    auto kern = fft_warp_tma_f32_kernel<N, G>;
    constexpr size_t smem = f32_tma_smem<N, G>();
    static int cached[kMaxDevices] = {};
    int* slot = device_slot(cached);
    int per_sm = slot ? *slot : 0;
    if (per_sm == 0) {
        cudaError_t e = persistent_ctas_per_sm((const void*)kern, f32_tma_threads<N, G>(), smem, &per_sm);
        if (e) return e;
        if (slot) *slot = per_sm;
    }
    const int64_t ntiles = L.grid;
    int64_t grid = (int64_t)L.sms * per_sm;
    if (grid > ntiles) grid = ntiles;
    if (grid < 1) grid = 1;
    kern<<<(unsigned)grid, f32_tma_threads<N, G>(), smem, st>>>(L.args, ntiles, map);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_warp_tma_f32(const StageLaunch& L, cudaStream_t st, bool* handled)
{
    *handled = false;
    const StageArgs& a = L.args;
    if (a.contig_store || a.conj_out || a.scale != 1.0 || a.in_fmt == FMT_R32 || a.out_fmt == FMT_R32) return cudaSuccess;
    if (a.n == 256) return a.G == 8 ? launch_f32_tma_n<256, 8>(L, st, handled) : (a.G == 16 ? launch_f32_tma_n<256, 16>(L, st, handled) : cudaSuccess);
    if (a.n == 512) return a.G == 8 ? launch_f32_tma_n<512, 8>(L, st, handled) : (a.G == 16 ? launch_f32_tma_n<512, 16>(L, st, handled) : cudaSuccess);
    return cudaSuccess;
}

}  // namespace ofg
