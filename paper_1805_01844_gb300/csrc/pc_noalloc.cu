// pc_noalloc.cu -- pc_compress_noalloc: compression for callers that cannot
// allocate device memory.
//
// pc_compress needs a small device workspace (a 64-byte header with the tile
// ticket and the error word, plus one 8-byte look-back word per tile), which
// its caller allocates.  Some callers cannot: a data-acquisition loop that
// must not call cudaMalloc once it is running (the call can fail under
// memory pressure or synchronise the device in the middle of a readout), or
// code embedded in a host framework that owns the device allocator and
// forbids raw allocations.  For them this entry point takes its workspace
// from a fixed static device array instead, and allocates nothing.
//
// The array below is part of libpc.so's device image: every GPU that loads
// the library holds these PC_NOALLOC_SCRATCH_BYTES bytes until the process
// exits.  In host code its name is only a host-side stand-in, so its device
// address is looked up with cudaGetSymbolAddress, once per device, with that
// device current, on the first call made on that device.
#include <cuda_runtime.h>

#include <mutex>

#include "pc.h"
#include "pc_kernels.h"

namespace {

// Shared by every pc_compress_noalloc call on a device; it keeps the last
// call's contents (pc_compress clears the part a call uses before its kernel).
static __device__ __align__(256) unsigned char g_noalloc_scratch[PC_NOALLOC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
std::mutex g_scratch_mu;
void *g_scratch_addr[kMaxDevices];  // device address of g_noalloc_scratch, per device

pc_status scratch_of_current_device(void **addr)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return PC_ERR_CUDA;
    if (dev < 0 || dev >= kMaxDevices) return PC_ERR_UNSUPPORTED;
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    if (g_scratch_addr[dev] == nullptr) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || p == nullptr) return PC_ERR_CUDA;
        g_scratch_addr[dev] = p;
    }
    *addr = g_scratch_addr[dev];
    return PC_OK;
}

}  // namespace

extern "C" pc_status pc_compress_noalloc(const void *d_in, uint64_t n_samples, const pc_params *params,
                                         void *d_out, uint64_t out_capacity, uint64_t *d_out_bytes,
                                         pc_stream_t stream)
{
    if (!params) return PC_ERR_INVALID_ARG;
    uint64_t need = 0;
    pc_status st = pc_workspace_size(params, n_samples, &need);
    if (st != PC_OK) return st;
    // the smallest workspace pc_compress accepts: the look-back words, without
    // the advanced variant's series table (its blocks then walk the series)
    need = pcx::ws_layout(params->variant, params->dtype_bits, params->word_bits, params->block_len,
                          n_samples, false).bytes;
    if (need > PC_NOALLOC_SCRATCH_BYTES) return PC_ERR_UNSUPPORTED;  // stream too long for the static scratch
    void *scratch = nullptr;
    if ((st = scratch_of_current_device(&scratch)) != PC_OK) return st;
    return pc_compress(d_in, n_samples, params, d_out, out_capacity, d_out_bytes, scratch,
                       PC_NOALLOC_SCRATCH_BYTES, stream);
}
