// pc_segmented.cu -- format version 2 (segmented streams): the block length
// and word size chosen per segment of the data, recorded in one code byte per
// segment of a single stream instead of one 64-byte stream header per
// segment.  Assembly of a version-2 stream from the per-segment version-1
// streams that pc_compress_segments writes (one kernel), and the host side of
// its C ABI (bound, workspace sizes, assembly, decoding; the decoding kernels
// are in pc_decompress.cu).
#include <cuda_runtime.h>

#include <cstdint>

#include "pc.h"
#include "pc_device.cuh"
#include "pc_kernels.h"

namespace pcx {

// One thread per segment reads its version-1 stream's header, checks it
// against the segment and gives the body size (table and words, each padded
// to 8 bytes); a block-wide scan and the bounded look-back over tiles of
// kV2TileSegs segments give every body's offset; then each warp copies its
// segments' table entries and words (4-byte units) into place.  The last tile
// writes the paddings of the code and size arrays, the header and the size.
template <uint32_t NT>
__global__ void __launch_bounds__(NT)
k_v2_assemble(const uint8_t *__restrict__ slots, uint64_t seg_stride, uint64_t n_seg, uint64_t n, uint32_t seg_len,
              uint32_t d, uint32_t variant, uint8_t *__restrict__ out, uint64_t cap, uint64_t *out_bytes, WsHeader *ws,
              uint64_t *status, uint64_t limit_ns)
{
    static_assert(NT == kV2TileSegs, "one thread per segment of a tile");
    constexpr uint32_t NW = NT / 32;
    __shared__ uint64_t warp_tot[NW];
    __shared__ uint64_t s_off[NT];
    __shared__ uint32_t s_tb[NT], s_wb[NT];
    __shared__ uint64_t s_excl;
    __shared__ uint32_t s_tile, s_ok;
    const uint32_t warp = threadIdx.x >> 5, lane = threadIdx.x & 31u;
    const uint32_t db = d / 8;
    const V2Geom g = v2_geom(n_seg);
    uint32_t *sizes = reinterpret_cast<uint32_t *>(out + g.sizes_at);
    const uint64_t n_tiles = ceil_div(n_seg, kV2TileSegs);
    auto finish = [&](uint64_t total) {  // one thread
        for (uint64_t o = PC_HEADER_BYTES + n_seg; o < g.sizes_at; ++o) out[o] = 0;
        for (uint64_t o = g.sizes_at + 4 * n_seg; o < g.bodies_at; ++o) out[o] = 0;
        uint32_t *h = reinterpret_cast<uint32_t *>(out);
        uint64_t *h64 = reinterpret_cast<uint64_t *>(out);
        h[0] = 0x504D4350u;  // "PCMP"
        h[1] = 2u | (variant << 16) | (d << 24);
        h[2] = 0;
        h[3] = seg_len;
        h64[2] = n;
        h64[3] = n_seg;
        h64[4] = total;
        h64[5] = h64[6] = h64[7] = 0;
        *out_bytes = g.bodies_at + total;
    };
    if (n_tiles == 0) {
        if (blockIdx.x == 0 && threadIdx.x == 0) finish(0);
        return;
    }
    for (;;) {
        if (threadIdx.x == 0) s_tile = atomicAdd(&ws->ticket, 1u);
        __syncthreads();
        const uint64_t tile = s_tile;
        if (tile >= n_tiles) break;
        const uint64_t sg = tile * kV2TileSegs + threadIdx.x;
        uint64_t body = 0;
        uint32_t tb = 0, wbytes = 0;
        if (sg < n_seg) {
            const uint8_t *slot = slots + sg * seg_stride;
            const uint32_t *h = reinterpret_cast<const uint32_t *>(slot);
            const uint64_t *h64 = reinterpret_cast<const uint64_t *>(slot);
            const uint64_t n_s = umin64(seg_len, n - sg * seg_len);
            const uint32_t L = h[3], w = h[2];
            bool ok = h[0] == 0x504D4350u && h[1] == (1u | (variant << 16) | (d << 24)) && (w == 32 || w == 64) &&
                      L >= 1 && L <= (1u << kV2MaxLog2L) && (L & (L - 1)) == 0 && h64[2] == n_s &&
                      h64[3] == ceil_div(n_s, L);
            uint32_t code = 0;
            if (ok) {
                const uint64_t nb = h64[3], pw = h64[4];
                const uint64_t tbytes = table_bytes(nb, d);
                ok = PC_HEADER_BYTES + tbytes <= seg_stride && pw <= (seg_stride - PC_HEADER_BYTES - tbytes) / (w / 8) &&
                     tbytes + pw * (w / 8) <= 0xFFFFFFF0ull;  // sizes in 32-bit fields
                if (ok) {
                    tb = (uint32_t)(nb * 2 * db);
                    wbytes = (uint32_t)(pw * (w / 8));
                    code = (31u - __clz(L)) | (w == 64 ? 0x80u : 0u);
                }
            }
            if (!ok) record_error(ws, PC_ERR_INVALID_ARG);
            body = round8(tb) + round8(wbytes);
            out[PC_HEADER_BYTES + sg] = (uint8_t)code;
            sizes[sg] = (uint32_t)(body / 8);
        }
        s_tb[threadIdx.x] = tb;
        s_wb[threadIdx.x] = wbytes;
        // block-wide exclusive scan of the body sizes
        uint64_t incl = body;
#pragma unroll
        for (uint32_t o = 1; o < 32; o <<= 1) {
            const uint64_t t = __shfl_up_sync(0xFFFFFFFFu, incl, o);
            if (lane >= o) incl += t;
        }
        if (lane == 31) warp_tot[warp] = incl;
        __syncthreads();
        if (warp == 0) {
            const uint64_t t = lane < NW ? warp_tot[lane] : 0ull;
            uint64_t ti = t;
#pragma unroll
            for (uint32_t o = 1; o < 32; o <<= 1) {
                const uint64_t u = __shfl_up_sync(0xFFFFFFFFu, ti, o);
                if (lane >= o) ti += u;
            }
            if (lane < NW) warp_tot[lane] = ti - t;
            const uint64_t agg = __shfl_sync(0xFFFFFFFFu, ti, 31);
            uint64_t excl = 0;
            const bool ok = lookback_warp(status, tile, agg, ws, limit_ns, &excl);
            if (lane == 0) {
                s_excl = excl;
                s_ok = ok ? 1u : 0u;
                if (ok && tile == n_tiles - 1) finish(excl + agg);
            }
        }
        __syncthreads();
        s_off[threadIdx.x] = s_excl + warp_tot[warp] + (incl - body);
        __syncthreads();
        if (s_ok) {
            const uint32_t m = (uint32_t)umin64(kV2TileSegs, n_seg - tile * kV2TileSegs);
            for (uint32_t k = warp; k < m; k += NW) {
                const uint64_t s2 = tile * kV2TileSegs + k;
                const uint32_t tbk = s_tb[k], wbk = s_wb[k];
                const uint64_t at = g.bodies_at + s_off[k], bk = round8(tbk) + round8(wbk);
                if (at > cap || bk > cap - at) {
                    if (lane == 0) record_error(ws, PC_ERR_CAPACITY);
                    continue;
                }
                const uint32_t *src = reinterpret_cast<const uint32_t *>(slots + s2 * seg_stride);
                const uint32_t nb = tbk / (2 * db);
                uint32_t *dst = reinterpret_cast<uint32_t *>(out + at);
                for (uint32_t i = lane; i < tbk / 4; i += 32) dst[i] = src[PC_HEADER_BYTES / 4 + i];
                if (lane == 0 && round8(tbk) != tbk) dst[tbk / 4] = 0;
                const uint32_t *wsrc = src + (PC_HEADER_BYTES + table_bytes(nb, d)) / 4;
                uint32_t *wdst = dst + round8(tbk) / 4;
                for (uint32_t i = lane; i < wbk / 4; i += 32) wdst[i] = wsrc[i];
                if (lane == 0 && round8(wbk) != wbk) wdst[wbk / 4] = 0;
            }
        }
        __syncthreads();
    }
}

cudaError_t launch_v2_assemble(const V2AssembleArgs &a)
{
    cudaError_t e;
    uint8_t *base = static_cast<uint8_t *>(a.workspace);
    WsHeader *ws = reinterpret_cast<WsHeader *>(base);
    const V2Layout lay = v2_layout(false, false, a.n_segments);
    uint64_t *status = reinterpret_cast<uint64_t *>(base + lay.off_status);
    if ((e = cudaMemsetAsync(base, 0, sizeof(WsHeader), a.stream)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(status, 0, 8 * lay.n_status, a.stream)) != cudaSuccess) return e;
    int dev = 0, sms = 0, per_sm = 0;
    auto kern = k_v2_assemble<kV2TileSegs>;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kV2TileSegs, 0)) != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    uint64_t grid = (uint64_t)per_sm * sms;
    const uint64_t tiles = ceil_div(a.n_segments, kV2TileSegs);
    if (tiles < grid) grid = tiles;
    if (grid < 1) grid = 1;
    kern<<<(unsigned)grid, kV2TileSegs, 0, a.stream>>>(static_cast<const uint8_t *>(a.slots), a.seg_stride,
                                                       a.n_segments, a.n, a.seg_len, a.d, a.variant,
                                                       static_cast<uint8_t *>(a.out), a.out_capacity, a.out_bytes,
                                                       ws, status, a.limit_ns);
    return cudaGetLastError();
}

}  // namespace pcx

using namespace pcx;

namespace {

bool v2_args_ok(uint32_t variant, uint32_t dtype_bits, uint32_t seg_len)
{
    return variant <= 1 && (dtype_bits == 16 || dtype_bits == 32) && seg_len >= 1;
}

bool al16(const void *p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

}  // namespace

extern "C" {

pc_status pc_bound_v2(uint32_t variant, uint32_t dtype_bits, uint32_t seg_len, uint64_t n_samples, uint64_t *max_bytes)
{
    if (!v2_args_ok(variant, dtype_bits, seg_len) || !max_bytes) return PC_ERR_INVALID_ARG;
    const uint64_t n_seg = ceil_div(n_samples, seg_len);
    uint64_t total = v2_geom(n_seg).bodies_at;
    for (int last = 0; last < 2 && n_seg > 0; ++last) {
        const uint64_t ns = last ? n_samples - (n_seg - 1) * seg_len : seg_len;
        const uint64_t count = last ? 1 : n_seg - 1;
        if (count == 0) continue;
        uint64_t worst = 0;
        for (uint32_t k = 0; k <= kV2MaxLog2L; ++k)
            for (uint32_t w = 32; w <= 64; w += 32) {
                const pc_params p{variant, dtype_bits, w, 1u << k};
                uint64_t b = 0;
                const pc_status st = pc_bound(&p, ns, &b);
                if (st != PC_OK) return st;
                const uint64_t nb = ceil_div(ns, p.block_len);
                const uint64_t body = round8(nb * 2 * (dtype_bits / 8)) +
                                      round8(b - PC_HEADER_BYTES - table_bytes(nb, dtype_bits));
                if (body > worst) worst = body;
            }
        total += count * worst;
    }
    *max_bytes = total;
    return PC_OK;
}

pc_status pc_assemble_v2_workspace_size(uint64_t n_segments, uint64_t *bytes)
{
    if (!bytes) return PC_ERR_INVALID_ARG;
    *bytes = v2_layout(false, false, n_segments).bytes;
    return PC_OK;
}

pc_status pc_assemble_v2(const void *d_slots, uint64_t seg_stride, uint64_t n_segments, uint64_t n_samples,
                         uint32_t seg_len, uint32_t dtype_bits, uint32_t variant, void *d_out, uint64_t out_capacity,
                         uint64_t *d_out_bytes, void *d_workspace, uint64_t workspace_bytes, pc_stream_t stream)
{
    if (!v2_args_ok(variant, dtype_bits, seg_len) || n_segments != ceil_div(n_samples, seg_len))
        return PC_ERR_INVALID_ARG;
    if ((!d_slots && n_segments) || !d_out || !d_out_bytes || !d_workspace) return PC_ERR_INVALID_ARG;
    if (!al16(d_slots) || seg_stride % 16 != 0 || seg_stride < PC_HEADER_BYTES || !al16(d_out) ||
        (reinterpret_cast<uintptr_t>(d_out_bytes) & 7u) != 0 || !al16(d_workspace))
        return PC_ERR_INVALID_ARG;
    if (workspace_bytes < v2_layout(false, false, n_segments).bytes) return PC_ERR_INVALID_ARG;
    if (out_capacity < v2_geom(n_segments).bodies_at) return PC_ERR_CAPACITY;
    V2AssembleArgs a{};
    a.slots = d_slots;
    a.seg_stride = seg_stride;
    a.n_segments = n_segments;
    a.n = n_samples;
    a.seg_len = seg_len;
    a.d = dtype_bits;
    a.variant = variant;
    a.out = d_out;
    a.out_capacity = out_capacity;
    a.out_bytes = d_out_bytes;
    a.workspace = d_workspace;
    a.limit_ns = kWaitLimitNs;
    a.stream = static_cast<cudaStream_t>(stream);
    return launch_v2_assemble(a) == cudaSuccess ? PC_OK : PC_ERR_CUDA;
}

pc_status pc_decompress_v2_workspace_size(uint32_t variant, uint32_t dtype_bits, uint32_t seg_len,
                                          uint64_t capacity_samples, uint64_t *bytes)
{
    if (!v2_args_ok(variant, dtype_bits, seg_len) || !bytes) return PC_ERR_INVALID_ARG;
    *bytes = v2_layout(variant == PC_VARIANT_ADVANCED, true, ceil_div(capacity_samples, seg_len)).bytes;
    return PC_OK;
}

pc_status pc_decompress_v2(const void *d_in, uint64_t in_bytes, uint32_t variant, uint32_t dtype_bits,
                           uint32_t seg_len, void *d_out, uint64_t out_capacity_samples, uint64_t *d_n_samples,
                           void *d_workspace, uint64_t workspace_bytes, pc_stream_t stream)
{
    if (!v2_args_ok(variant, dtype_bits, seg_len)) return PC_ERR_INVALID_ARG;
    if (variant == PC_VARIANT_ADVANCED && dtype_bits == 32) return PC_ERR_UNSUPPORTED;
    if (!d_in || (!d_out && out_capacity_samples) || !d_n_samples || !d_workspace) return PC_ERR_INVALID_ARG;
    if (!al16(d_in) || !al16(d_out) || (reinterpret_cast<uintptr_t>(d_n_samples) & 7u) != 0 || !al16(d_workspace))
        return PC_ERR_INVALID_ARG;
    if (in_bytes < PC_HEADER_BYTES) return PC_ERR_CORRUPT;
    const uint64_t max_segments = ceil_div(out_capacity_samples, seg_len);
    if (workspace_bytes < v2_layout(variant == PC_VARIANT_ADVANCED, true, max_segments).bytes)
        return PC_ERR_INVALID_ARG;
    V2DecodeArgs a{};
    a.in = d_in;
    a.in_bytes = in_bytes;
    a.variant = variant;
    a.d = dtype_bits;
    a.seg_len = seg_len;
    a.cap = out_capacity_samples;
    a.max_segments = max_segments;
    a.out = d_out;
    a.n_out = d_n_samples;
    a.workspace = d_workspace;
    a.limit_ns = kWaitLimitNs;
    a.stream = static_cast<cudaStream_t>(stream);
    return launch_v2_decode(a) == cudaSuccess ? PC_OK : PC_ERR_CUDA;
}

}  // extern "C"
