// pc_batch.cu -- many independent streams compressed in one persistent launch.
//
// The plan (device memory, written by pc_batch_plan) holds one descriptor per
// item and the prefix of the items' tile counts.  The kernel hands out global
// tickets; a ticket is mapped to (item, tile) by a binary search over the
// prefix and compressed by the same tile routine as pc_compress, with the
// item's own parameters, look-back words and series table (one table per
// word size).  Since tickets are taken in order, the tiles of an item are too,
// and a tile only waits on tiles owned by running CTAs.
#include <cuda_runtime.h>

#include <cstring>
#include <vector>

#include "pc.h"
#include "pc_compress.cuh"

namespace pcx {

struct BatchItemDev {
    const void *in;
    uint64_t n;
    void *out;
    uint64_t *out_bytes;
    uint64_t n_blocks;
    uint64_t n_tiles;  // real tiles (0 for an empty item, which still owns one ticket)
    uint32_t L;
    uint32_t key;      // short tiles << 3 | dtype 32 << 2 | word 64 << 1 | advanced
    uint32_t tb;       // blocks per tile
    uint32_t pad_;
};
static_assert(sizeof(BatchItemDev) % 16 == 0, "descriptors stay 16-byte aligned");

// Batch workspace: header, the two series tables (w = 32, 64: flags, flags,
// headers, slots, headers, slots; kept across calls, see ws_layout), then the
// look-back words (one per tile of every item).
struct BatchLayout {
    uint64_t off_flags32, off_flags64, off_hdr32, off_slots32, off_hdr64, off_slots64, off_status, n_status,
        bytes;
};

PCX_HD BatchLayout batch_layout(uint64_t total_tiles)
{
    BatchLayout b;
    b.off_flags32 = sizeof(WsHeader);
    b.off_flags64 = b.off_flags32 + kOrbitFlagsBytes;
    b.off_hdr32 = b.off_flags64 + kOrbitFlagsBytes;
    b.off_slots32 = b.off_hdr32 + kOrbitHdrBytes;
    b.off_hdr64 = b.off_slots32 + kOrbitSlotBytes;
    b.off_slots64 = b.off_hdr64 + kOrbitHdrBytes;
    b.off_status = b.off_slots64 + kOrbitSlotBytes;
    b.n_status = total_tiles + 1;
    b.bytes = b.off_status + 8 * b.n_status;
    return b;
}

template <uint32_t D, uint32_t WB, uint32_t VAR>
__device__ __forceinline__ void empty_item(const StreamArgs &sa)
{
    if (threadIdx.x == 0) write_empty_stream<D, WB, VAR>(sa);
}

template <uint32_t NT>
__global__ void __launch_bounds__(NT)
k_compress_batch(const BatchItemDev *__restrict__ items, const uint64_t *__restrict__ prefix, uint32_t n_items,
                 uint64_t total_tiles, WsHeader *ws, uint64_t *status, OrbitTable ot32, OrbitTable ot64,
                 uint64_t limit_ns)
{
    extern __shared__ __align__(16) uint8_t smem[];
    __shared__ uint64_t s_tile;
    __shared__ uint32_t s_item;
    stage_bars_init();
    uint32_t phase = 0;
    for (;;) {
        if (threadIdx.x == 0) {
            // a CTA whose staging died takes no further tile
            const uint64_t t = g_stage_dead ? ~0ull : (uint64_t)atomicAdd(&ws->ticket, 1u);
            uint32_t lo = 0, hi = n_items - 1;  // largest i with prefix[i] <= t
            if (t < total_tiles) {
                while (lo < hi) {
                    const uint32_t mid = (lo + hi + 1) >> 1;
                    if (prefix[mid] <= t) lo = mid;
                    else hi = mid - 1;
                }
            }
            s_tile = t;
            s_item = lo;
        }
        __syncthreads();
        const uint64_t t = s_tile;
        const uint32_t i = s_item;
        __syncthreads();
        if (t >= total_tiles) break;
        const BatchItemDev it = items[i];
        StreamArgs sa;
        sa.in = it.in;
        sa.n = it.n;
        sa.L = it.L;
        sa.out = static_cast<uint8_t *>(it.out);
        sa.out_bytes = it.out_bytes;
        sa.status = status + prefix[i];
        sa.n_blocks = it.n_blocks;
        sa.n_tiles = it.n_tiles;
        sa.tb = it.tb;
        sa.ot = (it.key & 2u) ? ot64 : ot32;
        const uint64_t tile = t - prefix[i];
        if (it.n_tiles == 0) {
            switch (it.key & 7u) {
            case 0: empty_item<16, 32, 0>(sa); break;
            case 1: empty_item<16, 32, 1>(sa); break;
            case 2: empty_item<16, 64, 0>(sa); break;
            case 3: empty_item<16, 64, 1>(sa); break;
            case 4: empty_item<32, 32, 0>(sa); break;
            case 5: empty_item<32, 32, 1>(sa); break;
            case 6: empty_item<32, 64, 0>(sa); break;
            default: empty_item<32, 64, 1>(sa); break;
            }
            continue;
        }
        if constexpr (NT == kShortThreads) {
            if (it.key & 8u) {  // short basic blocks: look-back tiles of whole short blocks
                switch (it.key & 6u) {
                case 0: compress_tile_short<uint16_t, 32>(sa, tile, smem, ws, limit_ns, phase); break;
                case 2: compress_tile_short<uint16_t, 64>(sa, tile, smem, ws, limit_ns, phase); break;
                case 4: compress_tile_short<uint32_t, 32>(sa, tile, smem, ws, limit_ns, phase); break;
                default: compress_tile_short<uint32_t, 64>(sa, tile, smem, ws, limit_ns, phase); break;
                }
                continue;
            }
        }
        switch (it.key) {
        case 0: compress_tile<uint16_t, 32, 0, false, NT>(sa, tile, smem, ws, limit_ns, phase); break;
        case 1: compress_tile<uint16_t, 32, 1, true, NT>(sa, tile, smem, ws, limit_ns, phase); break;
        case 2: compress_tile<uint16_t, 64, 0, false, NT>(sa, tile, smem, ws, limit_ns, phase); break;
        case 3: compress_tile<uint16_t, 64, 1, true, NT>(sa, tile, smem, ws, limit_ns, phase); break;
        case 4: compress_tile<uint32_t, 32, 0, false, NT>(sa, tile, smem, ws, limit_ns, phase); break;
        case 5: compress_tile<uint32_t, 32, 1, true, NT>(sa, tile, smem, ws, limit_ns, phase); break;
        case 6: compress_tile<uint32_t, 64, 0, false, NT>(sa, tile, smem, ws, limit_ns, phase); break;
        default: compress_tile<uint32_t, 64, 1, true, NT>(sa, tile, smem, ws, limit_ns, phase); break;
        }
    }
}

// One batch descriptor per segment from its option (segments path).  Every
// segment is a single tile (checked by pc_segments_describe), so the tile
// prefix is the identity.
__global__ void k_segment_items(const SourceDev *__restrict__ src, uint32_t n_src, uint64_t n_seg,
                                const uint8_t *__restrict__ options, uint32_t d, uint32_t variant,
                                uint64_t seg_stride, BatchItemDev *__restrict__ items, uint64_t *__restrict__ prefix,
                                WsHeader *ws)
{
    const uint64_t k = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k == 0) prefix[n_seg] = n_seg;
    if (k >= n_seg) return;
    const SourceDev s = src[source_of(src, n_src, k)];
    const uint64_t j = k - s.seg_first;
    uint32_t o = options[k];
    if (o >= PC_CHOOSER_OPTIONS) {
        record_error(ws, PC_ERR_INVALID_ARG);
        o = 0;
    }
    const uint32_t L = option_block_len(o), w = option_word_bits(o);
    BatchItemDev it;
    it.in = static_cast<const uint8_t *>(s.in) + j * PC_SEGMENT_SAMPLES * (d / 8);
    it.n = umin64(PC_SEGMENT_SAMPLES, s.n - j * PC_SEGMENT_SAMPLES);
    it.out = static_cast<uint8_t *>(s.out) + j * seg_stride;
    it.out_bytes = s.out_bytes + j;
    it.n_blocks = ceil_div(it.n, L);
    it.n_tiles = 1;
    it.tb = (uint32_t)it.n_blocks;  // the whole segment is one tile
    it.L = L;
    it.key = (d == 32 ? 4u : 0u) | (w == 64 ? 2u : 0u) | (variant ? 1u : 0u);
    it.pad_ = 0;
    items[k] = it;
    prefix[k] = k;
}

// ------------------------------------------------- warp-per-segment path
//
// A segment is a whole stream of at most 32 blocks, so it needs neither a
// look-back nor a CTA: one warp stages it, finds every block's min / max,
// counts, scans and packs it, and writes its header.  A CTA of 8 warps runs
// 8 segments at once with no barrier.  Used for 16-bit data (every base is
// in the series table) and for the basic variant.

// Shared memory of one warp: per-block vmin / B, then the stage (the widest
// layout over the options: ceil(4096 / L) slots of L + kPad samples).
constexpr uint32_t kSegVarsBytes = 32 * 4 + 32 * 8;

PCX_HD uint32_t seg_slot_bytes(uint32_t L, uint32_t d) { return (uint32_t)round_up((uint64_t)(L + kPad) * (d / 8), 16); }

PCX_HD uint32_t seg_warp_bytes(uint32_t d)
{
    uint32_t m = 0;
    for (uint32_t i = 0; i < 6; ++i) {
        const uint32_t L = 128u << i;
        const uint32_t b = (uint32_t)ceil_div(PC_SEGMENT_SAMPLES, L) * seg_slot_bytes(L, d);
        if (b > m) m = b;
    }
    return kSegVarsBytes + m;
}

template <typename T, uint32_t WB, uint32_t VAR>
__device__ void seg_warp(const T *__restrict__ in, uint32_t n, uint32_t L, uint8_t *out, uint64_t *out_bytes,
                         uint8_t *wsm, const OrbitTable &ot, WsHeader *ws, uint64_t limit_ns)
{
    using Word = typename WordOf<T, WB>::type;
    constexpr uint32_t D = sizeof(T) * 8;
    constexpr uint32_t VE = 16 / sizeof(T);
    const uint32_t lane = threadIdx.x & 31u;
    uint32_t *s_vmin = reinterpret_cast<uint32_t *>(wsm);
    uint64_t *s_B = reinterpret_cast<uint64_t *>(wsm + 128);
    uint8_t *stage = wsm + kSegVarsBytes;
    const uint32_t nblk = (n + L - 1) / L;
    const uint32_t S = seg_slot_bytes(L, D);

    // 1. stage: 16-byte granules (a block is a whole number of them), the
    // ragged end element by element
    const uint32_t vpb = L / VE, nvec = n / VE;
    for (uint32_t v = lane; v < nvec; v += 32) {
        const uint32_t b = v / vpb, o = v - b * vpb;
        cp_async16(stage + b * S + o * 16u, reinterpret_cast<const uint4 *>(in) + v);
    }
    cp_async_commit();
    for (uint32_t i = nvec * VE + lane; i < n; i += 32) {
        const uint32_t b = i / L;
        reinterpret_cast<T *>(stage + b * S)[i - b * L] = in[i];
    }
    cp_async_wait<0>();
    __syncwarp();

    // 2. min / max per block (padding set to the minimum)
    for (uint32_t b = 0; b < nblk; ++b) {
        const uint32_t n_b = min(L, n - b * L);
        block_minmax<T>(reinterpret_cast<T *>(stage + b * S), n_b, &s_vmin[b], &s_B[b]);
    }
    __syncwarp();

    // 3. lane b: block b's count (Eq. 1-2, or the series table of Sec. 3.2)
    uint32_t W = 0, p = 0, p1 = 0, vmin = 0;
    uint64_t B = 1, K = 0, K2 = 0;
    PackK pk{0u, 0u, 0u, 0u};
    OrbitView v{};
    if (lane < nblk) {
        B = s_B[lane];
        vmin = s_vmin[lane];
        const uint32_t n_b = min(L, n - lane * L);
        if (B > 1) {
            if constexpr (VAR == PC_VARIANT_BASIC) {
                p = basic_p(B, WB);
                W = (n_b + p - 1) / p;
                pk = basic_pack_k(B, p, vmin, WB);
            } else {
                const uint64_t h = orbit_get<WB>(ot, (uint32_t)B, L, ws, limit_ns);  // B <= 65536 for 16-bit data
                if (h != ~0ull) {
                    v = orbit_view(ot, h);
                    W = orbit_words_cached(ot, v, n_b, L);
                    p1 = eq1_p(B, WB);
                    uint64_t geo = 0, pw = 1, geo0 = 0;
                    for (uint32_t k = 0; k < p1; ++k) {
                        geo0 = geo;
                        geo += pw;
                        pw *= B;
                    }
                    K = geo * vmin;
                    K2 = geo0 * vmin;
                }
            }
        }
    }
    const uint32_t incl = warp_incl_scan_u32(W);
    const uint32_t woff = incl - W;
    const uint32_t total = __shfl_sync(0xFFFFFFFFu, incl, 31);

    // 4. table entries, table padding, header, size
    if (lane < nblk) {
        if constexpr (D == 16) reinterpret_cast<uint32_t *>(out + PC_HEADER_BYTES)[lane] = vmin | ((uint32_t)(B - 1) << 16);
        else reinterpret_cast<uint64_t *>(out + PC_HEADER_BYTES)[lane] = (uint64_t)vmin | ((B - 1) << 32);
    }
    const uint64_t payload_off = PC_HEADER_BYTES + table_bytes(nblk, D);
    for (uint64_t o = PC_HEADER_BYTES + (uint64_t)nblk * 2u * (D / 8) + lane; o < payload_off; o += 32) out[o] = 0;
    if (lane == 0) {
        write_header<D, WB, VAR>(out, L, n, nblk, total);
        *out_bytes = payload_off + (uint64_t)total * (WB / 8);
    }

    // 5. pack block by block
    Word *payload = reinterpret_cast<Word *>(out + payload_off);
    for (uint32_t b = 0; b < nblk; ++b) {
        const uint32_t Wb = __shfl_sync(0xFFFFFFFFu, W, b);
        const uint32_t ob = __shfl_sync(0xFFFFFFFFu, woff, b);
        const uint32_t B32 = (uint32_t)__shfl_sync(0xFFFFFFFFu, B, b);  // B < 2^32 here unless p = 1
        const uint64_t Kb = __shfl_sync(0xFFFFFFFFu, K, b);
        const T *u = reinterpret_cast<const T *>(stage + b * S);
        if (Wb == 0) continue;
        if constexpr (VAR == PC_VARIANT_BASIC) {
            const PackK pkb{__shfl_sync(0xFFFFFFFFu, pk.D, b), __shfl_sync(0xFFFFFFFFu, pk.Kf, b),
                            __shfl_sync(0xFFFFFFFFu, pk.Kt, b), __shfl_sync(0xFFFFFFFFu, pk.shape, b)};
            pack_basic_block<T, WB>(u, Wb, __shfl_sync(0xFFFFFFFFu, p, b), B32, pkb, payload + ob);
        } else {
            OrbitView vb;
            vb.off = __shfl_sync(0xFFFFFFFFu, v.off, b);
            vb.Q = __shfl_sync(0xFFFFFFFFu, v.Q, b);
            vb.P = __shfl_sync(0xFFFFFFFFu, v.P, b);
            vb.SQ = __shfl_sync(0xFFFFFFFFu, v.SQ, b);
            vb.G = __shfl_sync(0xFFFFFFFFu, v.G, b);
            vb.mgP.m = __shfl_sync(0xFFFFFFFFu, v.mgP.m, b);
            vb.mgP.a = __shfl_sync(0xFFFFFFFFu, v.mgP.a, b);
            vb.mgP.s = __shfl_sync(0xFFFFFFFFu, v.mgP.s, b);
            adv_words_orbit<T, WB>(ot, vb, u, Wb, B32, __shfl_sync(0xFFFFFFFFu, vmin, b),
                                   __shfl_sync(0xFFFFFFFFu, p1, b), Kb, __shfl_sync(0xFFFFFFFFu, K2, b),
                                   payload + ob);
        }
    }
    __syncwarp();  // the stage is free for the next segment
}

template <typename T, uint32_t VAR>
__global__ void __launch_bounds__(kThreads)
k_compress_segments_w(const SourceDev *__restrict__ src, uint32_t n_src, uint64_t n_seg,
                      const uint8_t *__restrict__ options, uint64_t seg_stride, uint32_t warp_bytes, WsHeader *ws,
                      OrbitTable ot32, OrbitTable ot64, uint64_t limit_ns)
{
    extern __shared__ __align__(16) uint8_t smem[];
    const uint32_t warp = threadIdx.x >> 5, lane = threadIdx.x & 31u;
    uint8_t *wsm = smem + warp * warp_bytes;
    const uint64_t nw = (uint64_t)gridDim.x * kWarps;
    for (uint64_t k = (uint64_t)blockIdx.x * kWarps + warp; k < n_seg; k += nw) {
        const SourceDev s = src[source_of(src, n_src, k)];
        const uint64_t j = k - s.seg_first;
        uint32_t o = options[k];
        if (o >= PC_CHOOSER_OPTIONS) {
            if (lane == 0) record_error(ws, PC_ERR_INVALID_ARG);
            o = 0;
        }
        const uint32_t L = option_block_len(o);
        const T *in = static_cast<const T *>(s.in) + j * PC_SEGMENT_SAMPLES;
        const uint32_t n = (uint32_t)umin64(PC_SEGMENT_SAMPLES, s.n - j * PC_SEGMENT_SAMPLES);
        uint8_t *out = static_cast<uint8_t *>(s.out) + j * seg_stride;
        if (option_word_bits(o) == 64) seg_warp<T, 64, VAR>(in, n, L, out, s.out_bytes + j, wsm, ot64, ws, limit_ns);
        else seg_warp<T, 32, VAR>(in, n, L, out, s.out_bytes + j, wsm, ot32, ws, limit_ns);
    }
}

// Running totals of the sources (segments path): the source's first segment
// counts the call, every segment adds its stream size.
__global__ void k_segment_totals(const SourceDev *__restrict__ src, uint32_t n_src, uint64_t n_seg)
{
    const uint64_t k = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n_seg) return;
    const SourceDev s = src[source_of(src, n_src, k)];
    if (!s.totals) return;
    const uint64_t j = k - s.seg_first;
    if (j == 0) atomicAdd(reinterpret_cast<unsigned long long *>(s.totals), 1ull);
    atomicAdd(reinterpret_cast<unsigned long long *>(s.totals + 1), (unsigned long long)s.out_bytes[j]);
}

}  // namespace pcx

using namespace pcx;

namespace {

bool a16(const void *p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

// Items of short basic blocks take the short-block tiles in 256-thread
// launches.
bool item_short(const pc_params &p, uint32_t nt)
{
    return nt == kShortThreads && short_tiles_ok(p.variant, p.dtype_bits, p.word_bits, p.block_len);
}

uint32_t item_tb(const pc_params &p, uint32_t nt)
{
    if (item_short(p, nt)) return short_tile_blocks(p.dtype_bits, p.block_len);
    return tile_cfg(kKernelCompress, p.variant, p.dtype_bits, p.word_bits, p.block_len, true, nt).tb;
}

uint64_t item_tiles(const pc_batch_item &it, uint32_t nt)
{
    const pc_params &p = it.params;
    return ceil_div(ceil_div(it.n_samples, p.block_len), item_tb(p, nt));
}

// Per call: header words and look-back words cleared, the tables kept or
// cleared (tag check on the device).
cudaError_t clear_batch_workspace(uint8_t *base, const BatchLayout &lay, cudaStream_t s)
{
    WsHeader *ws = reinterpret_cast<WsHeader *>(base);
    cudaError_t e = cudaMemsetAsync(base, 0, 12, s);
    if (e != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(base + lay.off_status, 0, 8 * lay.n_status, s)) != cudaSuccess) return e;
    return launch_orbit_prepare(ws, reinterpret_cast<uint32_t *>(base + lay.off_flags32), 2 * kOrbitFlagsBytes,
                                &ws->orbit_cursor, &ws->reserved_cursor64, kOrbitTagBatch, s);
}

OrbitTable batch_table(uint8_t *base, uint64_t off_flags, uint64_t off_hdr, uint64_t off_slots, uint32_t *cursor)
{
    return OrbitTable{reinterpret_cast<uint32_t *>(base + off_flags), reinterpret_cast<uint64_t *>(base + off_hdr),
                      reinterpret_cast<ulonglong2 *>(base + off_slots), cursor};
}

// The persistent batch kernel over a plan (items, prefix) with workspace
// `base` laid out by batch_layout(total_tiles); the workspace is cleared by
// the caller.
template <uint32_t NT>
pc_status launch_batch_t(const BatchItemDev *items, const uint64_t *prefix, uint32_t n_items, uint64_t total_tiles,
                         uint32_t smem, uint8_t *base, cudaStream_t s)
{
    const BatchLayout lay = batch_layout(total_tiles);
    WsHeader *ws = reinterpret_cast<WsHeader *>(base);
    const OrbitTable ot32 = batch_table(base, lay.off_flags32, lay.off_hdr32, lay.off_slots32, &ws->orbit_cursor);
    const OrbitTable ot64 = batch_table(base, lay.off_flags64, lay.off_hdr64, lay.off_slots64, &ws->reserved_cursor64);
    auto kern = k_compress_batch<NT>;
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
        return PC_ERR_CUDA;
    int dev = 0, sms = 0, per_sm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, NT, smem) != cudaSuccess)
        return PC_ERR_CUDA;
    if (per_sm < 1) return PC_ERR_UNSUPPORTED;
    uint64_t grid = (uint64_t)per_sm * sms;
    if (total_tiles < grid) grid = total_tiles;
    kern<<<(unsigned)grid, NT, smem, s>>>(items, prefix, n_items, total_tiles, ws,
                                                reinterpret_cast<uint64_t *>(base + lay.off_status), ot32, ot64,
                                                kWaitLimitNs);
    return cudaGetLastError() == cudaSuccess ? PC_OK : PC_ERR_CUDA;
}

pc_status launch_batch(const BatchItemDev *items, const uint64_t *prefix, uint32_t n_items, uint64_t total_tiles,
                       uint32_t smem, uint32_t nt, uint8_t *base, cudaStream_t s)
{
    return nt == 128 ? launch_batch_t<128>(items, prefix, n_items, total_tiles, smem, base, s)
                     : launch_batch_t<256>(items, prefix, n_items, total_tiles, smem, base, s);
}

template <typename T, uint32_t VAR>
pc_status launch_segments_w_t(const pc_segments_info *info, const SourceDev *src, const uint8_t *options,
                              uint8_t *base, const BatchLayout &lay, cudaStream_t s)
{
    WsHeader *ws = reinterpret_cast<WsHeader *>(base);
    const OrbitTable ot32 = batch_table(base, lay.off_flags32, lay.off_hdr32, lay.off_slots32, &ws->orbit_cursor);
    const OrbitTable ot64 = batch_table(base, lay.off_flags64, lay.off_hdr64, lay.off_slots64, &ws->reserved_cursor64);
    auto kern = k_compress_segments_w<T, VAR>;
    const uint32_t wb = seg_warp_bytes(sizeof(T) * 8);
    const uint32_t smem = kWarps * wb;
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
        return PC_ERR_CUDA;
    int dev = 0, sms = 0, per_sm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kThreads, smem) != cudaSuccess)
        return PC_ERR_CUDA;
    if (per_sm < 1) return PC_ERR_UNSUPPORTED;
    uint64_t grid = (uint64_t)per_sm * sms;
    const uint64_t need = ceil_div(info->n_segments, kWarps);
    if (need < grid) grid = need;
    kern<<<(unsigned)grid, kThreads, smem, s>>>(src, info->n_sources, info->n_segments, options, info->seg_stride,
                                                wb, ws, ot32, ot64, kWaitLimitNs);
    return cudaGetLastError() == cudaSuccess ? PC_OK : PC_ERR_CUDA;
}

pc_status launch_segments_w(const pc_segments_info *info, const SourceDev *src, const uint8_t *options,
                            uint8_t *base, const BatchLayout &lay, cudaStream_t s)
{
    if (info->dtype_bits == 16)
        return info->variant ? launch_segments_w_t<uint16_t, 1>(info, src, options, base, lay, s)
                             : launch_segments_w_t<uint16_t, 0>(info, src, options, base, lay, s);
    return launch_segments_w_t<uint32_t, 0>(info, src, options, base, lay, s);
}

pc_params option_params(uint32_t o, uint32_t d, uint32_t variant)
{
    pc_params p;
    std::memset(&p, 0, sizeof(p));
    p.variant = variant;
    p.dtype_bits = d;
    p.word_bits = option_word_bits(o);
    p.block_len = option_block_len(o);
    return p;
}

// Slot size, shared memory and the single-tile check over all options.
pc_status segment_facts(uint32_t d, uint32_t variant, uint64_t &stride, uint32_t &smem)
{
    stride = 0;
    smem = 0;
    for (uint32_t o = 0; o < PC_CHOOSER_OPTIONS; ++o) {
        const pc_params p = option_params(o, d, variant);
        uint64_t need = 0;
        if (pc_bound(&p, PC_SEGMENT_SAMPLES, &need) != PC_OK) return PC_ERR_INVALID_ARG;
        need = round_up(need, 16);
        if (need > stride) stride = need;
        const TileCfg cfg = tile_cfg(kKernelCompress, variant, d, p.word_bits, p.block_len, true);
        if (ceil_div(PC_SEGMENT_SAMPLES, p.block_len) > cfg.tb) return PC_ERR_UNSUPPORTED;
        if (cfg.smem > smem) smem = cfg.smem;
    }
    return PC_OK;
}

}  // namespace

extern "C" {

pc_status pc_batch_describe(const pc_batch_item *items, uint32_t n_items, pc_batch_info *info)
{
    if (!items || !info || n_items == 0) return PC_ERR_INVALID_ARG;
    const uint32_t nt = info->cta_threads == 128 ? 128u : 256u;
    uint64_t total = 0;
    uint32_t smem = 0;
    for (uint32_t i = 0; i < n_items; ++i) {
        const pc_batch_item &it = items[i];
        const pc_params &p = it.params;
        if (p.variant > 1 || (p.dtype_bits != 16 && p.dtype_bits != 32) || (p.word_bits != 32 && p.word_bits != 64) ||
            p.block_len == 0)
            return PC_ERR_INVALID_ARG;
        if (p.block_len > PC_MAX_BLOCK_LEN) return PC_ERR_UNSUPPORTED;
        if ((!it.d_in && it.n_samples) || !it.d_out || !it.d_out_bytes) return PC_ERR_INVALID_ARG;
        if (!a16(it.d_in) || !a16(it.d_out) || (reinterpret_cast<uintptr_t>(it.d_out_bytes) & 7u))
            return PC_ERR_INVALID_ARG;
        uint64_t need = 0;
        pc_bound(&p, it.n_samples, &need);
        if (it.out_capacity < need) return PC_ERR_CAPACITY;
        const uint64_t t = item_tiles(it, nt);
        total += t ? t : 1;
        const TileCfg cfg = tile_cfg(kKernelCompress, p.variant, p.dtype_bits, p.word_bits, p.block_len, true, nt);
        const uint32_t need_smem = item_short(p, nt) ? short_smem(p.dtype_bits, p.block_len) : cfg.smem;
        if (need_smem > smem) smem = need_smem;
    }
    if (total >> 31) return PC_ERR_UNSUPPORTED;  // tickets are 32-bit
    info->n_items = n_items;
    info->cta_threads = nt;
    info->reserved = 0;
    info->smem_bytes = smem;
    info->total_tiles = total;
    info->plan_bytes = sizeof(BatchItemDev) * (uint64_t)n_items + 8 * ((uint64_t)n_items + 1);
    info->workspace_bytes = batch_layout(total).bytes;
    return PC_OK;
}

pc_status pc_batch_plan(const pc_batch_item *items, uint32_t n_items, const pc_batch_info *info, void *d_plan,
                        pc_stream_t stream)
{
    if (!items || !info || !d_plan || !a16(d_plan) || n_items != info->n_items) return PC_ERR_INVALID_ARG;
    std::vector<uint8_t> host(info->plan_bytes);
    BatchItemDev *dv = reinterpret_cast<BatchItemDev *>(host.data());
    uint64_t *prefix = reinterpret_cast<uint64_t *>(host.data() + sizeof(BatchItemDev) * (uint64_t)n_items);
    uint64_t run = 0;
    for (uint32_t i = 0; i < n_items; ++i) {
        const pc_batch_item &it = items[i];
        const pc_params &p = it.params;
        BatchItemDev d;
        std::memset(&d, 0, sizeof(d));
        d.in = it.d_in;
        d.n = it.n_samples;
        d.out = it.d_out;
        d.out_bytes = it.d_out_bytes;
        d.n_blocks = ceil_div(it.n_samples, p.block_len);
        d.n_tiles = item_tiles(it, info->cta_threads);
        d.tb = item_tb(p, info->cta_threads);
        d.L = p.block_len;
        d.key = (item_short(p, info->cta_threads) ? 8u : 0u) | (p.dtype_bits == 32 ? 4u : 0u) |
                (p.word_bits == 64 ? 2u : 0u) | (p.variant ? 1u : 0u);
        dv[i] = d;
        prefix[i] = run;
        run += d.n_tiles ? d.n_tiles : 1;
    }
    prefix[n_items] = run;
    if (run != info->total_tiles) return PC_ERR_INVALID_ARG;
    if (cudaMemcpyAsync(d_plan, host.data(), info->plan_bytes, cudaMemcpyHostToDevice,
                        static_cast<cudaStream_t>(stream)) != cudaSuccess)
        return PC_ERR_CUDA;
    return PC_OK;
}

pc_status pc_compress_batch(const pc_batch_info *info, const void *d_plan, void *d_workspace,
                            uint64_t workspace_bytes, pc_stream_t stream)
{
    if (!info || !d_plan || !d_workspace || !a16(d_plan) || !a16(d_workspace)) return PC_ERR_INVALID_ARG;
    if (workspace_bytes < info->workspace_bytes || info->n_items == 0) return PC_ERR_INVALID_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const BatchLayout lay = batch_layout(info->total_tiles);
    if (clear_batch_workspace(static_cast<uint8_t *>(d_workspace), lay, s) != cudaSuccess) return PC_ERR_CUDA;
    const BatchItemDev *items = static_cast<const BatchItemDev *>(d_plan);
    const uint64_t *prefix = reinterpret_cast<const uint64_t *>(static_cast<const uint8_t *>(d_plan) +
                                                                sizeof(BatchItemDev) * (uint64_t)info->n_items);
    return launch_batch(items, prefix, info->n_items, info->total_tiles, info->smem_bytes, info->cta_threads,
                        static_cast<uint8_t *>(d_workspace), s);
}

// ---------------------------------------------------------------- segments

static uint64_t seg_count(uint64_t n) { return ceil_div(n, PC_SEGMENT_SAMPLES); }

pc_status pc_segments_describe(const pc_source *src, uint32_t n_sources, uint32_t dtype_bits, uint32_t variant,
                               pc_segments_info *info)
{
    if (!src || !info || n_sources == 0 || (dtype_bits != 16 && dtype_bits != 32) || variant > 1)
        return PC_ERR_INVALID_ARG;
    uint64_t stride = 0;
    uint32_t smem = 0;
    const pc_status st = segment_facts(dtype_bits, variant, stride, smem);
    if (st != PC_OK) return st;
    uint64_t total = 0;
    uint32_t has_totals = 0;
    for (uint32_t i = 0; i < n_sources; ++i) {
        const pc_source &so = src[i];
        if (so.d_totals) has_totals = 1;
        const uint64_t k = seg_count(so.n_samples);
        if (k == 0) continue;
        if (!so.d_in || !so.d_out || !so.d_out_bytes || !a16(so.d_in) || !a16(so.d_out) ||
            (reinterpret_cast<uintptr_t>(so.d_out_bytes) & 7u))
            return PC_ERR_INVALID_ARG;
        if (so.out_capacity / stride < k) return PC_ERR_CAPACITY;
        total += k;
        if (so.d_totals && (reinterpret_cast<uintptr_t>(so.d_totals) & 7u)) return PC_ERR_INVALID_ARG;
        if (total >> 31) return PC_ERR_UNSUPPORTED;
    }
    info->n_sources = n_sources;
    info->dtype_bits = dtype_bits;
    info->variant = variant;
    info->smem_bytes = smem;
    info->has_totals = has_totals;
    info->n_segments = total;
    info->seg_stride = stride;
    info->plan_bytes = sizeof(SourceDev) * (uint64_t)n_sources;
    info->workspace_bytes = round_up(batch_layout(total).bytes, 16) + sizeof(BatchItemDev) * total + 8 * (total + 1);
    return PC_OK;
}

pc_status pc_segments_plan(const pc_source *src, uint32_t n_sources, const pc_segments_info *info, void *d_plan,
                           pc_stream_t stream)
{
    if (!src || !info || !d_plan || !a16(d_plan) || n_sources != info->n_sources) return PC_ERR_INVALID_ARG;
    std::vector<SourceDev> host(n_sources);
    uint64_t first = 0;
    bool any_totals = false;
    for (uint32_t i = 0; i < n_sources; ++i) {
        SourceDev &d = host[i];
        std::memset(&d, 0, sizeof(d));
        d.in = src[i].d_in;
        d.n = src[i].n_samples;
        d.out = src[i].d_out;
        d.out_bytes = src[i].d_out_bytes;
        d.seg_first = first;
        d.totals = src[i].d_totals;
        first += seg_count(src[i].n_samples);
        if (d.totals) any_totals = true;
    }
    if (first != info->n_segments || any_totals != (info->has_totals != 0)) return PC_ERR_INVALID_ARG;
    if (cudaMemcpyAsync(d_plan, host.data(), info->plan_bytes, cudaMemcpyHostToDevice,
                        static_cast<cudaStream_t>(stream)) != cudaSuccess)
        return PC_ERR_CUDA;
    return PC_OK;
}

pc_status pc_compress_segments(const pc_segments_info *info, const void *d_plan, const uint8_t *d_options,
                               void *d_workspace, uint64_t workspace_bytes, pc_stream_t stream)
{
    if (!info) return PC_ERR_INVALID_ARG;
    if (info->n_segments == 0) return PC_OK;
    if (!d_plan || !d_options || !d_workspace || !a16(d_plan) || !a16(d_workspace) || info->n_sources == 0 ||
        (info->dtype_bits != 16 && info->dtype_bits != 32) || info->variant > 1)
        return PC_ERR_INVALID_ARG;
    if (workspace_bytes < info->workspace_bytes) return PC_ERR_INVALID_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const uint64_t n_seg = info->n_segments;
    const BatchLayout lay = batch_layout(n_seg);
    uint8_t *base = static_cast<uint8_t *>(d_workspace);
    const SourceDev *src = static_cast<const SourceDev *>(d_plan);
    if (clear_batch_workspace(static_cast<uint8_t *>(d_workspace), lay, s) != cudaSuccess) return PC_ERR_CUDA;
    pc_status st = PC_OK;
    if (info->dtype_bits == 16 || info->variant == PC_VARIANT_BASIC) {
        st = launch_segments_w(info, src, d_options, base, lay, s);
    } else {
        // 32-bit advanced: bases above 65536 walk the series in shared
        // memory, so these segments go through the CTA tile routine
        BatchItemDev *items = reinterpret_cast<BatchItemDev *>(base + round_up(lay.bytes, 16));
        uint64_t *prefix = reinterpret_cast<uint64_t *>(items + n_seg);
        k_segment_items<<<(unsigned)ceil_div(n_seg, 256), 256, 0, s>>>(
            src, info->n_sources, n_seg, d_options, info->dtype_bits, info->variant, info->seg_stride, items, prefix,
            reinterpret_cast<WsHeader *>(base));
        if (cudaGetLastError() != cudaSuccess) return PC_ERR_CUDA;
        st = launch_batch(items, prefix, (uint32_t)n_seg, n_seg, info->smem_bytes, kThreads, base, s);
    }
    if (st != PC_OK || !info->has_totals) return st;
    k_segment_totals<<<(unsigned)ceil_div(n_seg, 256), 256, 0, s>>>(static_cast<const SourceDev *>(d_plan),
                                                                  info->n_sources, n_seg);
    return cudaGetLastError() == cudaSuccess ? PC_OK : PC_ERR_CUDA;
}

}  // extern "C"
