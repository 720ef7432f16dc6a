// pc_stats.cu -- byte-value occurrences of a buffer (Sec. 5, Fig. 11: the
// byte profile of a file before and after polynomial compression).
//
// One kernel: a grid-stride pass of 16-byte loads, a 256-bin histogram per
// warp in shared memory (so lanes of different warps do not contend), the
// warps' bins summed per CTA and added once to the 64-bit global bins.
#include <cuda_runtime.h>

#include <cstdint>

#include "pc.h"

namespace {

constexpr uint32_t kHistThreads = 256;
constexpr uint32_t kHistWarps = kHistThreads / 32;

__device__ __forceinline__ void count_word(uint32_t *h, uint32_t v)
{
    atomicAdd(&h[v & 0xFFu], 1u);
    atomicAdd(&h[(v >> 8) & 0xFFu], 1u);
    atomicAdd(&h[(v >> 16) & 0xFFu], 1u);
    atomicAdd(&h[v >> 24], 1u);
}

__global__ void __launch_bounds__(kHistThreads)
k_byte_histogram(const uint8_t *__restrict__ in, uint64_t n, unsigned long long *__restrict__ hist)
{
    __shared__ uint32_t h[kHistWarps][256];
    const uint32_t warp = threadIdx.x >> 5;
    for (uint32_t i = threadIdx.x; i < kHistWarps * 256; i += kHistThreads) (&h[0][0])[i] = 0;
    __syncthreads();
    uint32_t *mine = h[warp];
    // the head up to a 16-byte boundary, the 16-byte body, the tail
    const uint64_t head = (16 - (reinterpret_cast<uintptr_t>(in) & 15u)) & 15u;
    const uint64_t nh = head < n ? head : n;
    const uint64_t gid = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x, step = (uint64_t)gridDim.x * blockDim.x;
    if (gid < nh) atomicAdd(&mine[in[gid]], 1u);
    const uint64_t nv = (n - nh) / 16;
    const uint4 *v4 = reinterpret_cast<const uint4 *>(in + nh);
    for (uint64_t i = gid; i < nv; i += step) {
        const uint4 v = __ldcs(v4 + i);
        count_word(mine, v.x);
        count_word(mine, v.y);
        count_word(mine, v.z);
        count_word(mine, v.w);
    }
    for (uint64_t i = nh + nv * 16 + gid; i < n; i += step) atomicAdd(&mine[in[i]], 1u);
    __syncthreads();
    for (uint32_t b = threadIdx.x; b < 256; b += kHistThreads) {
        uint64_t s = 0;
        for (uint32_t w = 0; w < kHistWarps; ++w) s += h[w][b];
        if (s) atomicAdd(&hist[b], (unsigned long long)s);
    }
}

}  // namespace

extern "C" pc_status pc_byte_histogram(const void *d_bytes, uint64_t n_bytes, uint64_t *d_hist, pc_stream_t stream)
{
    if ((!d_bytes && n_bytes) || !d_hist || (reinterpret_cast<uintptr_t>(d_hist) & 7u)) return PC_ERR_INVALID_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (cudaMemsetAsync(d_hist, 0, 256 * sizeof(uint64_t), s) != cudaSuccess) return PC_ERR_CUDA;
    if (n_bytes == 0) return PC_OK;
    int dev = 0, sms = 152;
    if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    uint64_t want = (n_bytes / 16 + kHistThreads - 1) / kHistThreads;
    const uint64_t cap = (uint64_t)sms * 8u;  // eight CTAs per SM: a few waves of the 16-byte loads
    if (want > cap) want = cap;
    if (want < 1) want = 1;
    k_byte_histogram<<<(unsigned)want, kHistThreads, 0, s>>>(static_cast<const uint8_t *>(d_bytes), n_bytes,
                                                             reinterpret_cast<unsigned long long *>(d_hist));
    return cudaGetLastError() == cudaSuccess ? PC_OK : PC_ERR_CUDA;
}
