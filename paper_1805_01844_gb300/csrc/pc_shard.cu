// pc_shard.cu -- one stream as block-aligned shards: placement of a shard's
// stream in the whole stream (pc_stitch) and the stream of a block range cut
// back out of a whole stream (pc_slice).
//
// Blocks are independent (Sec. 3.3), and a block's word count follows from
// its table entry alone (Eqs. 1-2 for the basic variant, the split-base
// series of Sec. 3.2 for the advanced one), so the whole stream's table is the
// shards' tables one after the other and its payload the shards' payloads one
// after the other: the only exchange is the exclusive prefix of the shards'
// payload sizes.
#include <cuda_runtime.h>

#include <cstdint>

#include "pc.h"
#include "pc_device.cuh"
#include "pc_kernels.h"

namespace pcx {
namespace {

constexpr uint32_t kCopyThreads = 256;
constexpr uint32_t kMaxShards = 1u << 16;

// Whole 4-byte words: table entries (4 or 8 bytes) and 32-bit payload words.
__device__ __forceinline__ void copy_u32(uint32_t *dst, const uint32_t *src, uint64_t n)
{
    const uint64_t i0 = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x, step = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t i = i0; i < n; i += step) dst[i] = __ldg(src + i);
}

__device__ __forceinline__ void copy_u64(uint64_t *dst, const uint64_t *src, uint64_t n)
{
    const uint64_t i0 = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x, step = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t i = i0; i < n; i += step) dst[i] = __ldg(src + i);
}

// A 64-byte header as pc_compress writes it (format version 1).
__device__ __forceinline__ void put_header(uint8_t *out, uint32_t variant, uint32_t d, uint32_t w, uint32_t L,
                                           uint64_t n, uint64_t n_blocks, uint64_t payload_words)
{
    uint32_t *h = reinterpret_cast<uint32_t *>(out);
    h[0] = 0x504D4350u;  // "PCMP"
    h[1] = 1u | (variant << 16) | (d << 24);
    h[2] = w;
    h[3] = L;
    uint64_t *h64 = reinterpret_cast<uint64_t *>(out);
    h64[2] = n;
    h64[3] = n_blocks;
    h64[4] = payload_words;
    h64[5] = 0;
    h64[6] = 0;
    h64[7] = 0;
}

// The header at `in` is a version-1 header of these parameters with n samples,
// n_blocks blocks and payload_words words.
__device__ __forceinline__ bool header_is(const uint8_t *in, uint32_t variant, uint32_t d, uint32_t w, uint32_t L,
                                          uint64_t n, uint64_t n_blocks, uint64_t payload_words)
{
    const uint32_t *h = reinterpret_cast<const uint32_t *>(in);
    const uint64_t *h64 = reinterpret_cast<const uint64_t *>(in);
    return h[0] == 0x504D4350u && h[1] == (1u | (variant << 16) | (d << 24)) && h[2] == w && h[3] == L &&
           h64[2] == n && h64[3] == n_blocks && h64[4] == payload_words && h64[5] == 0 && h64[6] == 0 &&
           h64[7] == 0;
}

// pc_stitch: every CTA places its share of the shard's table entries and
// payload words; CTA 0 of shard 0 writes the header, CTA 0 of the last shard
// the table padding and the total size.
__global__ void __launch_bounds__(kCopyThreads)
k_stitch(const uint8_t *__restrict__ shard, const uint64_t *__restrict__ shard_bytes, uint32_t K, uint32_t k,
         uint64_t n, uint32_t variant, uint32_t d, uint32_t w, uint32_t L, uint8_t *__restrict__ out,
         uint64_t out_cap, uint64_t *out_bytes, WsHeader *ws)
{
    __shared__ pc_stitch_region r;
    __shared__ uint32_t code;
    if (threadIdx.x == 0) {
        code = stitch_region(d, w, L, n, K, k, shard_bytes, r);
        if (code == PC_OK) {
            const uint64_t ns = r.n_blocks == 0 ? 0 : umin64(n, (r.first_block + r.n_blocks) * L) - r.first_block * L;
            if (!header_is(shard, variant, d, w, L, ns, r.n_blocks, r.payload_bytes / (w / 8u)))
                code = PC_ERR_CORRUPT;
            else if (r.total_bytes > out_cap)
                code = PC_ERR_CAPACITY;
        }
        if (code != PC_OK && blockIdx.x == 0) record_error(ws, code);
    }
    __syncthreads();
    if (code != PC_OK) return;
    copy_u32(reinterpret_cast<uint32_t *>(out + r.table_dst), reinterpret_cast<const uint32_t *>(shard + r.table_src),
             r.table_bytes / 4);
    if (w == 64)
        copy_u64(reinterpret_cast<uint64_t *>(out + r.payload_dst),
                 reinterpret_cast<const uint64_t *>(shard + r.payload_src), r.payload_bytes / 8);
    else
        copy_u32(reinterpret_cast<uint32_t *>(out + r.payload_dst),
                 reinterpret_cast<const uint32_t *>(shard + r.payload_src), r.payload_bytes / 4);
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        if (k == 0)
            put_header(out, variant, d, w, L, n, ceil_div(n, L), (r.total_bytes - r.payload_start) / (w / 8u));
        if (k == K - 1) {
            for (uint64_t o = r.pad_dst; o < r.payload_start; ++o) out[o] = 0;
            if (out_bytes) *out_bytes = r.total_bytes;
        }
    }
}

// pc_slice, first kernel: the word counts of the blocks before the range
// (ws->reserved[0]) and inside it (ws->reserved[1]), summed over a grid-stride
// pass of the table.  Advanced blocks walk their series (no table needed).
template <typename T, uint32_t WB, uint32_t VAR>
__global__ void __launch_bounds__(kCopyThreads)
k_slice_count(const uint8_t *__restrict__ in, uint64_t in_bytes, uint32_t L, uint64_t fb, uint64_t nb, WsHeader *ws)
{
    constexpr uint32_t D = sizeof(T) * 8;
    constexpr uint64_t kDmax = D == 16 ? 0xFFFFull : 0xFFFFFFFFull;
    __shared__ uint64_t s_before[kCopyThreads / 32], s_inside[kCopyThreads / 32];
    __shared__ uint32_t s_ok;
    const uint64_t *h64 = reinterpret_cast<const uint64_t *>(in);
    const uint32_t *h = reinterpret_cast<const uint32_t *>(in);
    if (threadIdx.x == 0) {
        uint32_t code = PC_OK;
        const uint64_t n = h64[2], NB = h64[3];
        if (h[0] != 0x504D4350u || h[1] != (1u | (VAR << 16) | (D << 24)) || h[2] != WB || h[3] != L ||
            h64[5] != 0 || h64[6] != 0 || h64[7] != 0 || NB != n / L + (n % L != 0) ||
            NB > (in_bytes - PC_HEADER_BYTES) / (2 * (D / 8)))
            code = PC_ERR_CORRUPT;
        else if (fb > NB || nb > NB - fb)
            code = PC_ERR_INVALID_ARG;
        if (code != PC_OK && blockIdx.x == 0) record_error(ws, code);
        s_ok = code == PC_OK;
    }
    __syncthreads();
    if (!s_ok) return;
    const uint64_t n = h64[2], end = fb + nb;
    uint64_t before = 0, inside = 0;
    const uint64_t i0 = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x, step = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t b = i0; b < end; b += step) {
        uint64_t vmin, Bm1;
        if constexpr (D == 16) {
            const uint32_t e = reinterpret_cast<const uint32_t *>(in + PC_HEADER_BYTES)[b];
            vmin = e & 0xFFFFu;
            Bm1 = e >> 16;
        } else {
            const uint64_t e = reinterpret_cast<const uint64_t *>(in + PC_HEADER_BYTES)[b];
            vmin = e & 0xFFFFFFFFull;
            Bm1 = e >> 32;
        }
        if (vmin + Bm1 > kDmax) {
            record_error(ws, PC_ERR_CORRUPT);
            continue;
        }
        const uint64_t B = Bm1 + 1;
        const uint32_t n_b = (uint32_t)umin64(L, n - b * L);
        uint32_t W = 0;
        if (B > 1) {
            if constexpr (VAR == PC_VARIANT_BASIC) {
                const uint32_t p = basic_p(B, WB);
                W = (n_b + p - 1) / p;
            } else {
                W = walk_series<WB>(B, n_b, nullptr, 0);
            }
        }
        if (b < fb) before += W;
        else inside += W;
    }
    before = warp_sum_u64(before);
    inside = warp_sum_u64(inside);
    const uint32_t warp = threadIdx.x >> 5, lane = threadIdx.x & 31u;
    if (lane == 0) {
        s_before[warp] = before;
        s_inside[warp] = inside;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        uint64_t a = 0, c = 0;
        for (uint32_t i = 0; i < kCopyThreads / 32; ++i) {
            a += s_before[i];
            c += s_inside[i];
        }
        if (a) atomicAdd(reinterpret_cast<unsigned long long *>(&ws->reserved[0]), (unsigned long long)a);
        if (c) atomicAdd(reinterpret_cast<unsigned long long *>(&ws->reserved[1]), (unsigned long long)c);
    }
}

// pc_slice, second kernel: header, table entries, padding and payload of the
// range, from the counts of the first kernel.
template <uint32_t D, uint32_t WB>
__global__ void __launch_bounds__(kCopyThreads)
k_slice_copy(const uint8_t *__restrict__ in, uint64_t in_bytes, uint32_t variant, uint32_t L, uint64_t fb,
             uint64_t nb, uint8_t *__restrict__ out, uint64_t out_cap, uint64_t *out_bytes, WsHeader *ws)
{
    constexpr uint64_t E = 2u * (D / 8u), WBY = WB / 8u;
    __shared__ uint64_t s_src, s_words, s_ns;
    __shared__ uint32_t s_ok;
    if (threadIdx.x == 0) {
        s_ok = 0;
        if (*reinterpret_cast<volatile uint32_t *>(&ws->status) == PC_OK) {
            const uint64_t *h64 = reinterpret_cast<const uint64_t *>(in);
            const uint64_t n = h64[2], NB = h64[3];
            const uint64_t before = ws->reserved[0], inside = ws->reserved[1];
            const uint64_t poff = PC_HEADER_BYTES + table_bytes(NB, D);
            const uint64_t ns = nb == 0 ? 0 : umin64(n, (fb + nb) * L) - fb * L;
            const uint64_t size = PC_HEADER_BYTES + table_bytes(nb, D) + inside * WBY;
            if (poff > in_bytes || before + inside > (in_bytes - poff) / WBY || before + inside > h64[4]) {
                if (blockIdx.x == 0) record_error(ws, PC_ERR_CORRUPT);
            } else if (size > out_cap) {
                if (blockIdx.x == 0) record_error(ws, PC_ERR_CAPACITY);
            } else {
                s_src = poff + before * WBY;
                s_words = inside;
                s_ns = ns;
                s_ok = 1;
            }
        }
    }
    __syncthreads();
    if (!s_ok) return;
    copy_u32(reinterpret_cast<uint32_t *>(out + PC_HEADER_BYTES),
             reinterpret_cast<const uint32_t *>(in + PC_HEADER_BYTES + fb * E), nb * E / 4);
    const uint64_t dst = PC_HEADER_BYTES + table_bytes(nb, D);
    if (WB == 64)
        copy_u64(reinterpret_cast<uint64_t *>(out + dst), reinterpret_cast<const uint64_t *>(in + s_src), s_words);
    else
        copy_u32(reinterpret_cast<uint32_t *>(out + dst), reinterpret_cast<const uint32_t *>(in + s_src), s_words);
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        put_header(out, variant, D, WB, L, s_ns, nb, s_words);
        for (uint64_t o = PC_HEADER_BYTES + nb * E; o < dst; ++o) out[o] = 0;
        *out_bytes = dst + s_words * WBY;
    }
}

uint32_t copy_grid(uint64_t units)
{
    int dev = 0, sms = 152;
    if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const uint64_t want = ceil_div(units, kCopyThreads * 4ull);
    const uint64_t cap = (uint64_t)sms * 8u;
    return (uint32_t)(want < 1 ? 1 : want > cap ? cap : want);
}

template <typename T, uint32_t WB, uint32_t VAR>
cudaError_t launch_slice_t(const void *in, uint64_t in_bytes, uint32_t L, uint64_t fb, uint64_t nb, void *out,
                           uint64_t out_cap, uint64_t *out_bytes, WsHeader *ws, cudaStream_t s)
{
    k_slice_count<T, WB, VAR><<<copy_grid(fb + nb), kCopyThreads, 0, s>>>(static_cast<const uint8_t *>(in), in_bytes,
                                                                         L, fb, nb, ws);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_slice_copy<sizeof(T) * 8, WB><<<copy_grid(nb * 64), kCopyThreads, 0, s>>>(
        static_cast<const uint8_t *>(in), in_bytes, VAR, L, fb, nb, static_cast<uint8_t *>(out), out_cap, out_bytes,
        ws);
    return cudaGetLastError();
}

}  // namespace
}  // namespace pcx

using namespace pcx;

namespace {

pc_status check_shard_params(const pc_params *p)
{
    if (!p) return PC_ERR_INVALID_ARG;
    if (p->variant > 1 || (p->dtype_bits != 16 && p->dtype_bits != 32) ||
        (p->word_bits != 32 && p->word_bits != 64) || p->block_len == 0)
        return PC_ERR_INVALID_ARG;
    if (p->block_len > PC_MAX_BLOCK_LEN) return PC_ERR_UNSUPPORTED;
    return PC_OK;
}

bool aligned(const void *p, uintptr_t a) { return (reinterpret_cast<uintptr_t>(p) & (a - 1)) == 0; }

}  // namespace

extern "C" {

pc_status pc_shard_range(const pc_params *params, uint64_t n_samples, uint32_t n_shards, uint32_t shard,
                         uint64_t *first_sample, uint64_t *n_shard_samples)
{
    pc_status st = check_shard_params(params);
    if (st != PC_OK) return st;
    if (n_shards == 0 || shard >= n_shards || !first_sample || !n_shard_samples) return PC_ERR_INVALID_ARG;
    const uint64_t L = params->block_len;
    uint64_t f, c;
    shard_blocks(ceil_div(n_samples, L), n_shards, shard, f, c);
    *first_sample = f * L;
    *n_shard_samples = c == 0 ? 0 : umin64(n_samples, (f + c) * L) - f * L;
    return PC_OK;
}

pc_status pc_stitch_layout(const pc_params *params, uint64_t n_samples, uint32_t n_shards, uint32_t shard,
                           const uint64_t *shard_bytes, pc_stitch_region *region)
{
    pc_status st = check_shard_params(params);
    if (st != PC_OK) return st;
    if (n_shards == 0 || shard >= n_shards || !shard_bytes || !region) return PC_ERR_INVALID_ARG;
    pc_stitch_region r{};
    const uint32_t code = stitch_region(params->dtype_bits, params->word_bits, params->block_len, n_samples,
                                        n_shards, shard, shard_bytes, r);
    if (code != PC_OK) return static_cast<pc_status>(code);
    *region = r;
    return PC_OK;
}

pc_status pc_stitch(const void *d_shard, const uint64_t *d_shard_bytes, uint32_t n_shards, uint32_t shard,
                    uint64_t n_samples, const pc_params *params, void *d_out, uint64_t out_capacity,
                    uint64_t *d_out_bytes, void *d_workspace, uint64_t workspace_bytes, pc_stream_t stream)
{
    pc_status st = check_shard_params(params);
    if (st != PC_OK) return st;
    if (n_shards == 0 || n_shards > kMaxShards || shard >= n_shards) return PC_ERR_INVALID_ARG;
    if (!d_shard || !d_shard_bytes || !d_out || !d_workspace || (shard == n_shards - 1 && !d_out_bytes))
        return PC_ERR_INVALID_ARG;
    if (!aligned(d_shard, 16) || !aligned(d_out, 16) || !aligned(d_shard_bytes, 8) || !aligned(d_workspace, 16) ||
        (d_out_bytes && !aligned(d_out_bytes, 8)) || workspace_bytes < sizeof(WsHeader))
        return PC_ERR_INVALID_ARG;
    uint64_t need = 0;
    pc_bound(params, n_samples, &need);
    if (out_capacity < need) return PC_ERR_CAPACITY;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (cudaMemsetAsync(d_workspace, 0, sizeof(WsHeader), s) != cudaSuccess) return PC_ERR_CUDA;
    uint64_t first = 0, count = 0;
    shard_blocks(ceil_div(n_samples, params->block_len), n_shards, shard, first, count);
    const uint64_t units = count * (2u * params->dtype_bits / 8u) / 4u +
                           count * (uint64_t)params->block_len * params->dtype_bits / params->word_bits;
    k_stitch<<<copy_grid(units), kCopyThreads, 0, s>>>(
        static_cast<const uint8_t *>(d_shard), d_shard_bytes, n_shards, shard, n_samples, params->variant,
        params->dtype_bits, params->word_bits, params->block_len, static_cast<uint8_t *>(d_out), out_capacity,
        d_out_bytes, static_cast<WsHeader *>(d_workspace));
    return cudaGetLastError() == cudaSuccess ? PC_OK : PC_ERR_CUDA;
}

pc_status pc_slice(const void *d_in, uint64_t in_bytes, const pc_params *params, uint64_t first_block,
                   uint64_t n_blocks, void *d_out, uint64_t out_capacity, uint64_t *d_out_bytes,
                   void *d_workspace, uint64_t workspace_bytes, pc_stream_t stream)
{
    pc_status st = check_shard_params(params);
    if (st != PC_OK) return st;
    if (!d_in || !d_out || !d_out_bytes || !d_workspace) return PC_ERR_INVALID_ARG;
    if (!aligned(d_in, 16) || !aligned(d_out, 16) || !aligned(d_out_bytes, 8) || !aligned(d_workspace, 16) ||
        workspace_bytes < sizeof(WsHeader))
        return PC_ERR_INVALID_ARG;
    if (in_bytes < PC_HEADER_BYTES) return PC_ERR_CORRUPT;
    if (n_blocks > (~0ull - first_block) / params->block_len) return PC_ERR_INVALID_ARG;
    uint64_t need = 0;
    pc_bound(params, n_blocks * params->block_len, &need);
    if (out_capacity < need) return PC_ERR_CAPACITY;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (cudaMemsetAsync(d_workspace, 0, sizeof(WsHeader), s) != cudaSuccess) return PC_ERR_CUDA;
    WsHeader *ws = static_cast<WsHeader *>(d_workspace);
    const uint32_t L = params->block_len;
    const uint32_t key = (params->dtype_bits == 32 ? 4u : 0u) | (params->word_bits == 64 ? 2u : 0u) |
                         (params->variant ? 1u : 0u);
    cudaError_t e;
    switch (key) {
    case 0: e = launch_slice_t<uint16_t, 32, 0>(d_in, in_bytes, L, first_block, n_blocks, d_out, out_capacity, d_out_bytes, ws, s); break;
    case 1: e = launch_slice_t<uint16_t, 32, 1>(d_in, in_bytes, L, first_block, n_blocks, d_out, out_capacity, d_out_bytes, ws, s); break;
    case 2: e = launch_slice_t<uint16_t, 64, 0>(d_in, in_bytes, L, first_block, n_blocks, d_out, out_capacity, d_out_bytes, ws, s); break;
    case 3: e = launch_slice_t<uint16_t, 64, 1>(d_in, in_bytes, L, first_block, n_blocks, d_out, out_capacity, d_out_bytes, ws, s); break;
    case 4: e = launch_slice_t<uint32_t, 32, 0>(d_in, in_bytes, L, first_block, n_blocks, d_out, out_capacity, d_out_bytes, ws, s); break;
    case 5: e = launch_slice_t<uint32_t, 32, 1>(d_in, in_bytes, L, first_block, n_blocks, d_out, out_capacity, d_out_bytes, ws, s); break;
    case 6: e = launch_slice_t<uint32_t, 64, 0>(d_in, in_bytes, L, first_block, n_blocks, d_out, out_capacity, d_out_bytes, ws, s); break;
    default: e = launch_slice_t<uint32_t, 64, 1>(d_in, in_bytes, L, first_block, n_blocks, d_out, out_capacity, d_out_bytes, ws, s); break;
    }
    return e == cudaSuccess ? PC_OK : PC_ERR_CUDA;
}

}  // extern "C"
