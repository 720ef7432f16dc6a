// pc_compress.cu -- launch of the single-stream compression kernel.
#include <cuda_runtime.h>

#include "pc_compress.cuh"

namespace pcx {


// Long streams of short basic blocks (short_tiles_ok): look-back tiles of up
// to 128 whole blocks (compress_tile_short).
template <typename T, uint32_t WB>
static cudaError_t launch_compress_short(const LaunchArgs &a, bool &taken)
{
    taken = false;
    if (!short_tiles_ok(PC_VARIANT_BASIC, sizeof(T) * 8, WB, a.L)) return cudaSuccess;
    const uint32_t tb = short_tile_blocks(sizeof(T) * 8, a.L);
    const uint64_t n_tiles = ceil_div(a.n_blocks, (uint64_t)tb);
    if (n_tiles < kSmallTiles) return cudaSuccess;
    taken = true;
    auto kern = k_compress_short<T, WB>;
    const uint32_t smem = short_smem(sizeof(T) * 8, a.L);
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, cudaSharedmemCarveoutMaxShared);
    if (e != cudaSuccess) return e;
    int per_sm = 0, dev = 0, sms = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kShortThreads, smem)) != cudaSuccess)
        return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    uint64_t grid = (uint64_t)per_sm * sms;
    if (n_tiles < grid) grid = n_tiles;
    StreamArgs sa;
    sa.in = a.in;
    sa.n = a.n;
    sa.L = a.L;
    sa.out = static_cast<uint8_t *>(a.out);
    sa.out_bytes = a.out_count;
    sa.status = a.status;
    sa.n_blocks = a.n_blocks;
    sa.n_tiles = n_tiles;
    sa.tb = tb;
    sa.ot = OrbitTable{a.orb_flags, a.orb_hdr, static_cast<ulonglong2 *>(a.orb_slots), &a.ws->orbit_cursor};
    kern<<<(unsigned)grid, kShortThreads, smem, a.stream>>>(sa, a.ws, a.limit_ns);
    return cudaGetLastError();
}

template <typename T, uint32_t WB, uint32_t VAR, bool ORB, uint32_t NT>
static cudaError_t launch_compress_t(const LaunchArgs &a)
{
    if constexpr (VAR == PC_VARIANT_BASIC) {
        bool taken = false;
        const cudaError_t e = launch_compress_short<T, WB>(a, taken);
        if (taken || e != cudaSuccess) return e;
    }
    const TileCfg cfg1 = tile_cfg(kKernelCompress, VAR, sizeof(T) * 8, WB, a.L, ORB, NT);
    // basic streams long enough for look-back tiles of several full stage
    // tiles on every SM: one look-back per multi_k stage tiles
    // (compress_tile_multi); where a stage budget for four CTAs per SM still
    // gives stage tiles of >= 24 blocks, that smaller stage (measured +2 % at
    // L = 1024; smaller stage tiles lose more than the extra CTA gains)
    // advanced 16-bit streams (series table) take the same look-back tiles,
    // with stage tiles of the four-CTA budget so that their larger per-tile
    // arrays still leave three CTAs per SM
    constexpr bool kAdvMulti = VAR == PC_VARIANT_ADVANCED && ORB && sizeof(T) == 2 && NT == kThreads;
    constexpr bool kMultiOk = (VAR == PC_VARIANT_BASIC && NT == kThreads) || kAdvMulti;
    const TileCfg cfg4 = tile_cfg(kKernelCompress, VAR, sizeof(T) * 8, WB, a.L, ORB, NT, kTileBudgetMulti4);
    const bool four = kMultiOk && cfg4.tb >= 24;
    const TileCfg cfgm = four ? cfg4 : cfg1;
    const uint32_t k = multi_k(cfgm.tb);
    const bool multi = kMultiOk && (!kAdvMulti || four) && k >= 2 && a.tb == cfg1.tb && cfgm.tb >= 8 &&
                       (a.L * sizeof(T)) % 16 == 0 && ceil_div(a.n_blocks, (uint64_t)k * cfgm.tb) >= kSmallTiles;
    auto kern = !multi ? k_compress<T, WB, VAR, ORB, NT, false, false>
                : four ? k_compress<T, WB, VAR, ORB, NT, kMultiOk, kMultiOk>
                       : k_compress<T, WB, VAR, ORB, NT, kMultiOk, false>;
    TileCfg cfg = multi ? cfgm : cfg1;
    if (multi && kAdvMulti) cfg.smem = multi_smem<VAR>(cfg);
    const uint64_t n_tiles = multi ? ceil_div(a.n_blocks, (uint64_t)k * cfg.tb) : a.n_tiles;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)cfg.smem);
    if (e != cudaSuccess) return e;
    // all of the unified L1 / shared storage as shared memory, so that the
    // register-allowed tiles per SM also fit in shared memory
    e = cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, cudaSharedmemCarveoutMaxShared);
    if (e != cudaSuccess) return e;
    int per_sm = 0, dev = 0, sms = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, NT, cfg.smem)) != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    uint64_t grid = (uint64_t)per_sm * sms;
    if (n_tiles < grid) grid = n_tiles;
    if (grid < 1) grid = 1;
    StreamArgs sa;
    sa.in = a.in;
    sa.n = a.n;
    sa.L = a.L;
    sa.out = static_cast<uint8_t *>(a.out);
    sa.out_bytes = a.out_count;
    sa.status = a.status;
    sa.n_blocks = a.n_blocks;
    sa.n_tiles = n_tiles;
    sa.tb = multi ? k * cfg.tb : a.tb;
    sa.ot = OrbitTable{a.orb_flags, a.orb_hdr, static_cast<ulonglong2 *>(a.orb_slots), &a.ws->orbit_cursor};
    kern<<<(unsigned)grid, NT, cfg.smem, a.stream>>>(sa, a.ws, a.limit_ns);
    return cudaGetLastError();
}

template <typename T, uint32_t WB, uint32_t VAR, bool ORB>
static cudaError_t launch_compress_nt(const LaunchArgs &a)
{
    return a.nt == 128 ? launch_compress_t<T, WB, VAR, ORB, 128>(a) : launch_compress_t<T, WB, VAR, ORB, 256>(a);
}

// One CTA: clear the series tables' flags and cursors unless the header's tag
// says they were built for this layout and word size, then set the tag.
__global__ void k_orbit_prepare(WsHeader *ws, uint32_t *flags, uint64_t flag_bytes, uint32_t *cursor0,
                                uint32_t *cursor1, uint64_t tag)
{
    __shared__ uint32_t stale;
    if (threadIdx.x == 0) stale = ws->orbit_tag != tag;
    __syncthreads();
    if (!stale) return;
    uint4 *f = reinterpret_cast<uint4 *>(flags);
    for (uint64_t i = threadIdx.x; i < flag_bytes / 16; i += blockDim.x) f[i] = make_uint4(0u, 0u, 0u, 0u);
    __syncthreads();
    if (threadIdx.x == 0) {
        *cursor0 = 0;
        if (cursor1) *cursor1 = 0;
        ws->orbit_tag = tag;
    }
}

cudaError_t launch_orbit_prepare(WsHeader *ws, uint32_t *flags, uint64_t flag_bytes, uint32_t *cursor0,
                                 uint32_t *cursor1, uint64_t tag, cudaStream_t stream)
{
    k_orbit_prepare<<<1, 1024, 0, stream>>>(ws, flags, flag_bytes, cursor0, cursor1, tag);
    return cudaGetLastError();
}

cudaError_t launch_compress(const LaunchArgs &a)
{
    const uint32_t key = (a.d == 32 ? 4u : 0u) | (a.w == 64 ? 2u : 0u) | (a.variant ? 1u : 0u);
    switch (key) {
    case 0: return launch_compress_nt<uint16_t, 32, 0, false>(a);
    case 1: return a.orbit ? launch_compress_nt<uint16_t, 32, 1, true>(a) : launch_compress_nt<uint16_t, 32, 1, false>(a);
    case 2: return launch_compress_nt<uint16_t, 64, 0, false>(a);
    case 3: return a.orbit ? launch_compress_nt<uint16_t, 64, 1, true>(a) : launch_compress_nt<uint16_t, 64, 1, false>(a);
    case 4: return launch_compress_nt<uint32_t, 32, 0, false>(a);
    case 5: return a.orbit ? launch_compress_nt<uint32_t, 32, 1, true>(a) : launch_compress_nt<uint32_t, 32, 1, false>(a);
    case 6: return launch_compress_nt<uint32_t, 64, 0, false>(a);
    default: return a.orbit ? launch_compress_nt<uint32_t, 64, 1, true>(a) : launch_compress_nt<uint32_t, 64, 1, false>(a);
    }
}

}  // namespace pcx
