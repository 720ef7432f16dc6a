// pc_kernels.h -- internal interface between the host API (pc_api.cu) and
// the kernel translation units.  Not installed; no torch or user types.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

#include "pc_common.cuh"

namespace pcx {

struct LaunchArgs {
    const void *in;        // compress: samples; decompress: stream bytes
    uint64_t n;            // compress: samples
    uint64_t in_bytes;     // decompress: stream bytes available
    uint32_t L, d, w, variant;
    void *out;             // compress: stream; decompress: samples
    uint64_t cap;          // decompress: sample capacity
    uint64_t *out_count;   // compress: stream bytes; decompress: samples
    WsHeader *ws;
    uint64_t *status;      // look-back words
    uint64_t n_status;     // look-back words available
    uint64_t *offsets;     // decompression: payload offset per decoding tile (+ total)
    uint64_t n_offsets;    // entries available in offsets
    uint64_t n_blocks, n_tiles;
    uint32_t nt;             // compression: threads per CTA (128 or 256)
    uint32_t tb;             // compression: blocks per tile; decompression: blocks per warp tile
    bool orbit;              // advanced: the series table is in the workspace
    uint32_t *orb_flags;
    uint64_t *orb_hdr;
    void *orb_slots;
    uint64_t limit_ns;
    cudaStream_t stream;
};

cudaError_t launch_compress(const LaunchArgs &a);
// Keep or clear the series tables of a workspace (see ws_layout).
cudaError_t launch_orbit_prepare(WsHeader *ws, uint32_t *flags, uint64_t flag_bytes, uint32_t *cursor0,
                                 uint32_t *cursor1, uint64_t tag, cudaStream_t stream);
cudaError_t launch_decompress(const LaunchArgs &a);
cudaError_t launch_selftest_wait(WsHeader *ws, uint64_t *status, uint64_t limit_ns, cudaStream_t stream);

// Decoding of a version-2 (segmented) stream: workspace laid out by
// v2_layout(advanced, true, max_segments).
struct V2DecodeArgs {
    const void *in;
    uint64_t in_bytes;
    uint32_t variant, d, seg_len;
    uint64_t cap;           // sample capacity of out
    uint64_t max_segments;  // ceil(cap / seg_len): offsets in the workspace
    void *out;
    uint64_t *n_out;
    void *workspace;
    uint64_t limit_ns;
    cudaStream_t stream;
};
cudaError_t launch_v2_decode(const V2DecodeArgs &a);

// Assembly of a version-2 stream from per-segment version-1 streams.
struct V2AssembleArgs {
    const void *slots;
    uint64_t seg_stride, n_segments, n;
    uint32_t seg_len, d, variant;
    void *out;
    uint64_t out_capacity;
    uint64_t *out_bytes;
    void *workspace;
    uint64_t limit_ns;
    cudaStream_t stream;
};
cudaError_t launch_v2_assemble(const V2AssembleArgs &a);

}  // namespace pcx
