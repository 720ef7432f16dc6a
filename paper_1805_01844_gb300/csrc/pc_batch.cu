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
    uint32_t key;      // dtype 32 << 2 | word 64 << 1 | advanced
    uint64_t pad_;
};
static_assert(sizeof(BatchItemDev) % 16 == 0, "descriptors stay 16-byte aligned");

// Batch workspace: header, two series-table flag arrays (w = 32, 64), the
// look-back words (one per tile of every item), then the two tables.
struct BatchLayout {
    uint64_t off_flags32, off_flags64, off_status, clear_bytes, off_hdr32, off_slots32, off_hdr64, off_slots64,
        bytes;
};

PCX_HD BatchLayout batch_layout(uint64_t total_tiles)
{
    BatchLayout b;
    b.off_flags32 = sizeof(WsHeader);
    b.off_flags64 = b.off_flags32 + kOrbitFlagsBytes;
    b.off_status = b.off_flags64 + kOrbitFlagsBytes;
    b.clear_bytes = b.off_status + 8 * (total_tiles + 1);
    b.off_hdr32 = round_up(b.clear_bytes, 16);
    b.off_slots32 = b.off_hdr32 + kOrbitHdrBytes;
    b.off_hdr64 = b.off_slots32 + kOrbitSlotBytes;
    b.off_slots64 = b.off_hdr64 + kOrbitHdrBytes;
    b.bytes = b.off_slots64 + kOrbitSlotBytes;
    return b;
}

template <uint32_t D, uint32_t WB, uint32_t VAR>
__device__ __forceinline__ void empty_item(const StreamArgs &sa)
{
    if (threadIdx.x == 0) write_empty_stream<D, WB, VAR>(sa);
}

__global__ void __launch_bounds__(kThreads)
k_compress_batch(const BatchItemDev *__restrict__ items, const uint64_t *__restrict__ prefix, uint32_t n_items,
                 uint64_t total_tiles, WsHeader *ws, uint64_t *status, OrbitTable ot32, OrbitTable ot64,
                 uint64_t limit_ns)
{
    extern __shared__ __align__(16) uint8_t smem[];
    __shared__ uint64_t s_tile;
    __shared__ uint32_t s_item;
    for (;;) {
        if (threadIdx.x == 0) {
            const uint64_t t = atomicAdd(&ws->ticket, 1u);
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
        sa.ot = (it.key & 2u) ? ot64 : ot32;
        const uint64_t tile = t - prefix[i];
        if (it.n_tiles == 0) {
            switch (it.key) {
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
        switch (it.key) {
        case 0: compress_tile<uint16_t, 32, 0, false>(sa, tile, smem, ws, limit_ns); break;
        case 1: compress_tile<uint16_t, 32, 1, true>(sa, tile, smem, ws, limit_ns); break;
        case 2: compress_tile<uint16_t, 64, 0, false>(sa, tile, smem, ws, limit_ns); break;
        case 3: compress_tile<uint16_t, 64, 1, true>(sa, tile, smem, ws, limit_ns); break;
        case 4: compress_tile<uint32_t, 32, 0, false>(sa, tile, smem, ws, limit_ns); break;
        case 5: compress_tile<uint32_t, 32, 1, true>(sa, tile, smem, ws, limit_ns); break;
        case 6: compress_tile<uint32_t, 64, 0, false>(sa, tile, smem, ws, limit_ns); break;
        default: compress_tile<uint32_t, 64, 1, true>(sa, tile, smem, ws, limit_ns); break;
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
    it.L = L;
    it.key = (d == 32 ? 4u : 0u) | (w == 64 ? 2u : 0u) | (variant ? 1u : 0u);
    it.pad_ = 0;
    items[k] = it;
    prefix[k] = k;
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

uint64_t item_tiles(const pc_batch_item &it)
{
    const pc_params &p = it.params;
    const TileCfg cfg = tile_cfg(kKernelCompress, p.variant, p.dtype_bits, p.word_bits, p.block_len, true);
    return ceil_div(ceil_div(it.n_samples, p.block_len), cfg.tb);
}

OrbitTable batch_table(uint8_t *base, uint64_t off_flags, uint64_t off_hdr, uint64_t off_slots, uint32_t *cursor)
{
    return OrbitTable{reinterpret_cast<uint32_t *>(base + off_flags), reinterpret_cast<uint64_t *>(base + off_hdr),
                      reinterpret_cast<ulonglong2 *>(base + off_slots), cursor};
}

// The persistent batch kernel over a plan (items, prefix) with workspace
// `base` laid out by batch_layout(total_tiles); the workspace is cleared by
// the caller.
pc_status launch_batch(const BatchItemDev *items, const uint64_t *prefix, uint32_t n_items, uint64_t total_tiles,
                       uint32_t smem, uint8_t *base, cudaStream_t s)
{
    const BatchLayout lay = batch_layout(total_tiles);
    WsHeader *ws = reinterpret_cast<WsHeader *>(base);
    const OrbitTable ot32 = batch_table(base, lay.off_flags32, lay.off_hdr32, lay.off_slots32, &ws->orbit_cursor);
    const OrbitTable ot64 = batch_table(base, lay.off_flags64, lay.off_hdr64, lay.off_slots64, &ws->reserved_cursor64);
    auto kern = k_compress_batch;
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
        return PC_ERR_CUDA;
    int dev = 0, sms = 0, per_sm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kThreads, smem) != cudaSuccess)
        return PC_ERR_CUDA;
    if (per_sm < 1) return PC_ERR_UNSUPPORTED;
    uint64_t grid = (uint64_t)per_sm * sms;
    if (total_tiles < grid) grid = total_tiles;
    kern<<<(unsigned)grid, kThreads, smem, s>>>(items, prefix, n_items, total_tiles, ws,
                                                reinterpret_cast<uint64_t *>(base + lay.off_status), ot32, ot64,
                                                kWaitLimitNs);
    return cudaGetLastError() == cudaSuccess ? PC_OK : PC_ERR_CUDA;
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
        const uint64_t t = item_tiles(it);
        total += t ? t : 1;
        const TileCfg cfg = tile_cfg(kKernelCompress, p.variant, p.dtype_bits, p.word_bits, p.block_len, true);
        if (cfg.smem > smem) smem = cfg.smem;
    }
    if (total >> 31) return PC_ERR_UNSUPPORTED;  // tickets are 32-bit
    info->n_items = n_items;
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
        d.n_tiles = item_tiles(it);
        d.L = p.block_len;
        d.key = (p.dtype_bits == 32 ? 4u : 0u) | (p.word_bits == 64 ? 2u : 0u) | (p.variant ? 1u : 0u);
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
    if (cudaMemsetAsync(d_workspace, 0, lay.clear_bytes, s) != cudaSuccess) return PC_ERR_CUDA;
    const BatchItemDev *items = static_cast<const BatchItemDev *>(d_plan);
    const uint64_t *prefix = reinterpret_cast<const uint64_t *>(static_cast<const uint8_t *>(d_plan) +
                                                                sizeof(BatchItemDev) * (uint64_t)info->n_items);
    return launch_batch(items, prefix, info->n_items, info->total_tiles, info->smem_bytes,
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
    BatchItemDev *items = reinterpret_cast<BatchItemDev *>(base + round_up(lay.bytes, 16));
    uint64_t *prefix = reinterpret_cast<uint64_t *>(items + n_seg);
    if (cudaMemsetAsync(d_workspace, 0, lay.clear_bytes, s) != cudaSuccess) return PC_ERR_CUDA;
    k_segment_items<<<(unsigned)ceil_div(n_seg, 256), 256, 0, s>>>(
        static_cast<const SourceDev *>(d_plan), info->n_sources, n_seg, d_options, info->dtype_bits, info->variant,
        info->seg_stride, items, prefix, reinterpret_cast<WsHeader *>(base));
    if (cudaGetLastError() != cudaSuccess) return PC_ERR_CUDA;
    const pc_status st = launch_batch(items, prefix, (uint32_t)n_seg, n_seg, info->smem_bytes, base, s);
    if (st != PC_OK || !info->has_totals) return st;
    k_segment_totals<<<(unsigned)ceil_div(n_seg, 256), 256, 0, s>>>(static_cast<const SourceDev *>(d_plan),
                                                                  info->n_sources, n_seg);
    return cudaGetLastError() == cudaSuccess ? PC_OK : PC_ERR_CUDA;
}

}  // extern "C"
