// pc_api.cu -- host side of the C ABI declared in include/pc.h: argument
// checks, sizes, workspace clearing and kernel launches.  No allocation, no
// global state, no synchronisation except in pc_last_device_status.
#include <cuda_runtime.h>

#include <cstdint>
#include <cstring>

#include "pc.h"
#include "pc_kernels.h"

using namespace pcx;

namespace {

bool aligned16(const void *p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }
bool aligned8(const void *p) { return (reinterpret_cast<uintptr_t>(p) & 7u) == 0; }

pc_status check_params(const pc_params *p)
{
    if (!p) return PC_ERR_INVALID_ARG;
    if (p->variant > 1 || (p->dtype_bits != 16 && p->dtype_bits != 32) ||
        (p->word_bits != 32 && p->word_bits != 64) || p->block_len == 0)
        return PC_ERR_INVALID_ARG;
    if (p->block_len > PC_MAX_BLOCK_LEN) return PC_ERR_UNSUPPORTED;
    return PC_OK;
}

WsLayout layout_for(const pc_params *p, uint64_t n, bool orbit)
{
    return ws_layout(p->variant, p->dtype_bits, p->word_bits, p->block_len, n, orbit);
}

// The workspace decides the advanced variant's mode: with room for the series
// table (pc_workspace_size) the table is used; with only the look-back words
// and offsets, each block walks its series.  false if it is too small.
bool pick_layout(const pc_params *p, uint64_t n, uint64_t workspace_bytes, WsLayout &lay)
{
    lay = layout_for(p, n, true);
    if (workspace_bytes >= lay.bytes) return true;
    lay = layout_for(p, n, false);
    return workspace_bytes >= lay.bytes;
}

// Per call: the header's ticket, status and timeout count, and the look-back
// words, cleared; the series table kept if its tag names this word size
// (without a table the cursors and the tag are cleared too).
cudaError_t clear_workspace(void *d_workspace, const WsLayout &lay, uint32_t w, cudaStream_t s)
{
    uint8_t *base = static_cast<uint8_t *>(d_workspace);
    WsHeader *ws = reinterpret_cast<WsHeader *>(base);
    cudaError_t e = cudaMemsetAsync(base, 0, lay.orbit ? 12 : 32, s);
    if (e != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(base + lay.off_status, 0, 8 * lay.n_status, s)) != cudaSuccess) return e;
    if (!lay.orbit) return cudaSuccess;
    return launch_orbit_prepare(ws, reinterpret_cast<uint32_t *>(base + lay.off_flags), kOrbitFlagsBytes,
                                &ws->orbit_cursor, nullptr, kOrbitTagOne | w, s);
}

void fill_workspace(LaunchArgs &a, void *d_workspace, const WsLayout &lay)
{
    uint8_t *base = static_cast<uint8_t *>(d_workspace);
    a.ws = reinterpret_cast<WsHeader *>(base);
    a.status = reinterpret_cast<uint64_t *>(base + lay.off_status);
    a.n_status = lay.n_status;
    a.offsets = reinterpret_cast<uint64_t *>(base + lay.off_offsets);
    a.n_offsets = lay.n_offsets;
    a.orbit = lay.orbit;
    a.orb_flags = lay.orbit ? reinterpret_cast<uint32_t *>(base + lay.off_flags) : nullptr;
    a.orb_hdr = lay.orbit ? reinterpret_cast<uint64_t *>(base + lay.off_hdr) : nullptr;
    a.orb_slots = lay.orbit ? static_cast<void *>(base + lay.off_slots) : nullptr;
}

}  // namespace

extern "C" {

pc_status pc_bound(const pc_params *params, uint64_t n_samples, uint64_t *max_bytes)
{
    pc_status st = check_params(params);
    if (st != PC_OK) return st;
    if (!max_bytes) return PC_ERR_INVALID_ARG;
    const uint64_t L = params->block_len;
    const uint64_t n_blocks = ceil_div(n_samples, L);
    uint64_t total = PC_HEADER_BYTES + table_bytes(n_blocks, params->dtype_bits);
    if (n_blocks > 0) {
        const uint64_t last = n_samples - (n_blocks - 1) * L;
        const uint64_t wbytes = params->word_bits / 8;
        total += (n_blocks - 1) * words_bound(params->variant, params->dtype_bits, params->word_bits, L) * wbytes;
        total += words_bound(params->variant, params->dtype_bits, params->word_bits, last) * wbytes;
    }
    *max_bytes = total;
    return PC_OK;
}

pc_status pc_workspace_size(const pc_params *params, uint64_t n_samples, uint64_t *bytes)
{
    pc_status st = check_params(params);
    if (st != PC_OK) return st;
    if (!bytes) return PC_ERR_INVALID_ARG;
    *bytes = layout_for(params, n_samples, true).bytes;
    return PC_OK;
}

pc_status pc_compress(const void *d_in, uint64_t n_samples, const pc_params *params, void *d_out,
                      uint64_t out_capacity, uint64_t *d_out_bytes, void *d_workspace,
                      uint64_t workspace_bytes, pc_stream_t stream)
{
    pc_status st = check_params(params);
    if (st != PC_OK) return st;
    if ((!d_in && n_samples) || !d_out || !d_out_bytes || !d_workspace) return PC_ERR_INVALID_ARG;
    if (!aligned16(d_in) || !aligned16(d_out) || !aligned8(d_out_bytes) || !aligned16(d_workspace))
        return PC_ERR_INVALID_ARG;
    WsLayout lay;
    const bool fits = pick_layout(params, n_samples, workspace_bytes, lay);
    const uint64_t n_blocks = ceil_div(n_samples, params->block_len);
    const uint32_t nt = compress_threads(params->variant, params->dtype_bits, params->word_bits, params->block_len);
    const TileCfg cfg = tile_cfg(kKernelCompress, params->variant, params->dtype_bits, params->word_bits,
                                 params->block_len, lay.orbit, nt);
    const uint32_t tb = small_stream_tb(n_blocks, cfg.tb);
    const uint64_t n_tiles = ceil_div(n_blocks, tb);
    if (n_tiles >> 31) return PC_ERR_UNSUPPORTED;  // tile tickets are 32-bit
    uint64_t need = 0;
    pc_bound(params, n_samples, &need);
    if (out_capacity < need) return PC_ERR_CAPACITY;
    if (!fits) return PC_ERR_INVALID_ARG;

    LaunchArgs a{};
    a.in = d_in;
    a.n = n_samples;
    a.L = params->block_len;
    a.d = params->dtype_bits;
    a.w = params->word_bits;
    a.variant = params->variant;
    a.out = d_out;
    a.out_count = d_out_bytes;
    fill_workspace(a, d_workspace, lay);
    a.n_blocks = n_blocks;
    a.n_tiles = n_tiles;
    a.nt = nt;
    a.tb = tb;
    a.limit_ns = kWaitLimitNs;
    a.stream = static_cast<cudaStream_t>(stream);
    if (clear_workspace(d_workspace, lay, a.w, a.stream) != cudaSuccess) return PC_ERR_CUDA;
    if (launch_compress(a) != cudaSuccess) return PC_ERR_CUDA;
    return PC_OK;
}

pc_status pc_decompress(const void *d_in, uint64_t in_bytes, const pc_params *params, void *d_out,
                        uint64_t out_capacity_samples, uint64_t *d_n_samples, void *d_workspace,
                        uint64_t workspace_bytes, pc_stream_t stream)
{
    pc_status st = check_params(params);
    if (st != PC_OK) return st;
    if (!d_in || (!d_out && out_capacity_samples) || !d_n_samples || !d_workspace) return PC_ERR_INVALID_ARG;
    if (!aligned16(d_in) || !aligned16(d_out) || !aligned8(d_n_samples) || !aligned16(d_workspace))
        return PC_ERR_INVALID_ARG;
    if (in_bytes < PC_HEADER_BYTES) return PC_ERR_CORRUPT;
    // the workspace holds the look-back words and the decoding-tile offsets of
    // a stream of up to out_capacity_samples samples (and the series table)
    WsLayout lay;
    if (!pick_layout(params, out_capacity_samples, workspace_bytes, lay)) return PC_ERR_INVALID_ARG;

    LaunchArgs a{};
    a.in = d_in;
    a.in_bytes = in_bytes;
    a.L = params->block_len;
    a.d = params->dtype_bits;
    a.w = params->word_bits;
    a.variant = params->variant;
    a.out = d_out;
    a.cap = out_capacity_samples;
    a.out_count = d_n_samples;
    // warp tiles of the decoder, from the largest stream the call accepts
    a.tb = small_stream_tb(ceil_div(out_capacity_samples, params->block_len),
                           dec_tile_cap(params->variant, params->dtype_bits, params->word_bits, params->block_len));
    fill_workspace(a, d_workspace, lay);
    a.limit_ns = kWaitLimitNs;
    a.stream = static_cast<cudaStream_t>(stream);
    // header words and look-back words cleared, the series table kept or
    // cleared; offsets are written before they are read
    if (clear_workspace(d_workspace, lay, a.w, a.stream) != cudaSuccess) return PC_ERR_CUDA;
    if (launch_decompress(a) != cudaSuccess) return PC_ERR_CUDA;
    return PC_OK;
}

pc_status pc_parse_header(const void *host_header, uint64_t nbytes, pc_params *params, uint64_t *n_samples)
{
    if (!host_header || !params || !n_samples) return PC_ERR_INVALID_ARG;
    if (nbytes < PC_HEADER_BYTES) return PC_ERR_CORRUPT;
    const uint8_t *h = static_cast<const uint8_t *>(host_header);
    auto le = [&](unsigned off, unsigned k) {
        uint64_t v = 0;
        for (unsigned i = 0; i < k; ++i) v |= (uint64_t)h[off + i] << (8 * i);
        return v;
    };
    if (std::memcmp(h, "PCMP", 4) != 0 || le(4, 2) != 1) return PC_ERR_CORRUPT;
    for (unsigned i = 9; i < 12; ++i)
        if (h[i]) return PC_ERR_CORRUPT;
    for (unsigned i = 40; i < 64; ++i)
        if (h[i]) return PC_ERR_CORRUPT;
    pc_params p;
    p.variant = h[6];
    p.dtype_bits = h[7];
    p.word_bits = h[8];
    p.block_len = (uint32_t)le(12, 4);
    const uint64_t n = le(16, 8), nb = le(24, 8);
    if (check_params(&p) == PC_ERR_INVALID_ARG) return PC_ERR_CORRUPT;
    if (nb != n / p.block_len + (n % p.block_len != 0)) return PC_ERR_CORRUPT;
    *params = p;
    *n_samples = n;
    return PC_OK;
}

pc_status pc_last_device_status(const void *d_workspace, pc_stream_t stream)
{
    if (!d_workspace) return PC_ERR_INVALID_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (cudaStreamSynchronize(s) != cudaSuccess) return PC_ERR_CUDA;
    uint32_t code = 0;
    const WsHeader *ws = static_cast<const WsHeader *>(d_workspace);
    if (cudaMemcpy(&code, &ws->status, sizeof(code), cudaMemcpyDeviceToHost) != cudaSuccess)
        return PC_ERR_CUDA;
    return static_cast<pc_status>(code);
}

pc_status pc_selftest_bounded_wait(void *d_workspace, uint64_t workspace_bytes, uint32_t limit_us,
                                   pc_stream_t stream)
{
    if (!d_workspace || !aligned16(d_workspace) || workspace_bytes < sizeof(WsHeader) + 16)
        return PC_ERR_INVALID_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (cudaMemsetAsync(d_workspace, 0, sizeof(WsHeader) + 16, s) != cudaSuccess) return PC_ERR_CUDA;
    WsHeader *ws = static_cast<WsHeader *>(d_workspace);
    uint64_t *status = reinterpret_cast<uint64_t *>(static_cast<uint8_t *>(d_workspace) + sizeof(WsHeader));
    if (launch_selftest_wait(ws, status, (uint64_t)limit_us * 1000ull, s) != cudaSuccess) return PC_ERR_CUDA;
    return PC_OK;
}

const char *pc_strerror(pc_status status)
{
    switch (status) {
    case PC_OK: return "ok";
    case PC_ERR_INVALID_ARG: return "invalid argument";
    case PC_ERR_CAPACITY: return "output capacity too small";
    case PC_ERR_CORRUPT: return "corrupt or truncated stream";
    case PC_ERR_CUDA: return "CUDA error";
    case PC_ERR_TIMEOUT: return "bounded device wait ran out";
    case PC_ERR_UNSUPPORTED: return "unsupported parameters";
    }
    return "unknown status";
}

}  // extern "C"
