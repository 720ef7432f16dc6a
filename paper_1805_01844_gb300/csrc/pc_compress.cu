// pc_compress.cu -- the fused compression kernel (sm_103a).
//
// One CTA per tile of `tb` blocks, tiles handed out in order from an atomic
// ticket.  Per tile:
//   1. 16-byte streaming loads of the tile's samples into shared memory;
//   2. per block (one warp each): min / max (Sec. 3.1), B = max - min + 1;
//   3. word counts: basic W = ceil(n_b / p) with p from Eq. 1; advanced W from
//      the split-base series of Sec. 3.2, one lane per block;
//   4. warp scan of the counts, decoupled look-back across tiles for the
//      payload offset of the tile;
//   5. block table entries (min, B - 1) and the packed words, each word one
//      Horner evaluation over its digits, stored coalesced.
// The last tile writes the header, the table padding and the stream size.
#include <cuda_runtime.h>

#include "pc_device.cuh"
#include "pc_kernels.h"

namespace pcx {

template <typename T, uint32_t WB>
struct WordOf;
template <typename T>
struct WordOf<T, 32> { using type = uint32_t; };
template <typename T>
struct WordOf<T, 64> { using type = uint64_t; };

// (lo, hi) <- (lo, hi) * m + a  in 64-bit arithmetic from 32-bit multiplies;
// exact whenever the true result is below 2^64.
__device__ __forceinline__ void mad64(uint32_t &lo, uint32_t &hi, uint32_t m, uint32_t a)
{
    uint64_t t = (uint64_t)lo * m + a;
    hi = hi * m + (uint32_t)(t >> 32);
    lo = (uint32_t)t;
}

// Eq. 2, word j of a block: s_j = sum_{i<p} u[j p + i] B^i, evaluated by
// Horner from the highest digit; u = v - vmin; padding samples hold vmin.
template <typename T, uint32_t WB>
__device__ __forceinline__ typename WordOf<T, WB>::type
basic_word(const T *dg, uint32_t p, uint32_t B32, uint32_t vmin)
{
    if constexpr (WB == 32) {
        uint32_t acc = 0;
        for (int k = (int)p - 1; k >= 0; --k) acc = acc * B32 + ((uint32_t)dg[k] - vmin);
        return acc;
    } else {
        uint32_t lo = 0, hi = 0;
        for (int k = (int)p - 1; k >= 0; --k) mad64(lo, hi, B32, (uint32_t)dg[k] - vmin);
        return ((uint64_t)hi << 32) | lo;
    }
}

// Sec. 3.2, word i of a block:
//   s_i = r_i + R_i (sum_{k=1}^{p_i} u_{q_i+k} B^{p_i-k} + r'_{i-1} B^{p_i})
// with the split sample e = u[q_i + p_i], r_i = e mod R_i, and
// r'_{i-1} = u[q_i - 1] div R_{i-1} (the high part of the previous split).
template <typename T, uint32_t WB>
__device__ __forceinline__ typename WordOf<T, WB>::type
adv_word(const T *u, const uint64_t *sched, uint32_t i, uint32_t B32, uint32_t vmin)
{
    const uint64_t e = sched[i];
    const uint32_t R = (uint32_t)e;
    const uint32_t p = (uint32_t)(e >> 32) & 0xFFu;
    const uint32_t q = (uint32_t)(e >> 40);
    uint32_t top = 0;
    if (i > 0) {
        const uint32_t Rprev = (uint32_t)sched[i - 1];
        top = ((uint32_t)u[q - 1] - vmin) / Rprev;
    }
    const uint32_t es = (uint32_t)u[q + p] - vmin;
    const uint32_t r = es - (es / R) * R;
    if constexpr (WB == 64 && sizeof(T) == 4) {
        if (B32 == 0) {  // B = 2^32 (held as 0 in 32 bits): p_i <= 1
            uint32_t lo = top, hi = 0;
            if (p == 1) { hi = lo; lo = (uint32_t)u[q] - vmin; }
            mad64(lo, hi, R, r);
            return ((uint64_t)hi << 32) | lo;
        }
    }
    if constexpr (WB == 32) {
        uint32_t acc = top;
        for (uint32_t k = 0; k < p; ++k) acc = acc * B32 + ((uint32_t)u[q + k] - vmin);
        return acc * R + r;
    } else {
        uint32_t lo = top, hi = 0;
        for (uint32_t k = 0; k < p; ++k) mad64(lo, hi, B32, (uint32_t)u[q + k] - vmin);
        mad64(lo, hi, R, r);
        return ((uint64_t)hi << 32) | lo;
    }
}

template <typename T, uint32_t WB, uint32_t VAR>
__global__ void __launch_bounds__(kThreads)
k_compress(const T *__restrict__ in, uint64_t n, uint32_t L, uint8_t *__restrict__ out,
           uint64_t *__restrict__ out_bytes, WsHeader *ws, uint64_t *status,
           uint64_t n_blocks, uint64_t n_tiles, uint64_t limit_ns)
{
    using Word = typename WordOf<T, WB>::type;
    constexpr uint32_t D = sizeof(T) * 8;
    extern __shared__ __align__(16) uint8_t smem[];
    const TileCfg cfg = tile_cfg(VAR, D, WB, L);
    BlockVars &bv = *reinterpret_cast<BlockVars *>(smem + cfg.off_blk);
    uint64_t *sched_all = reinterpret_cast<uint64_t *>(smem + cfg.off_sched);
    const uint32_t warp = threadIdx.x >> 5, lane = threadIdx.x & 31u;
    const uint64_t payload_off = PC_HEADER_BYTES + table_bytes(n_blocks, D);

    auto write_header = [&](uint64_t payload_words) {
        uint32_t *h = reinterpret_cast<uint32_t *>(out);
        h[0] = 0x504D4350u;  // "PCMP"
        h[1] = 1u | (VAR << 16) | (D << 24);
        h[2] = WB;
        h[3] = L;
        uint64_t *h64 = reinterpret_cast<uint64_t *>(out);
        h64[2] = n;
        h64[3] = n_blocks;
        h64[4] = payload_words;
        h64[5] = 0;
        h64[6] = 0;
        h64[7] = 0;
        *out_bytes = payload_off + payload_words * (WB / 8);
    };

    if (n_tiles == 0) {
        if (blockIdx.x == 0 && threadIdx.x == 0) write_header(0);
        return;
    }

    for (;;) {
        if (threadIdx.x == 0) bv.tile = atomicAdd(&ws->ticket, 1u);
        __syncthreads();
        const uint64_t tile = bv.tile;
        if (tile >= n_tiles) break;
        const uint64_t blk0 = tile * cfg.tb;
        const uint32_t nblk = (uint32_t)umin64(cfg.tb, n_blocks - blk0);
        const uint64_t g0 = blk0 * L;
        const uint64_t cnt = umin64(n - g0, (uint64_t)nblk * L);

        // 1. stage the tile
        load_tile<T>(in, g0, cnt, L, smem, cfg.stage_bytes);
        __syncthreads();

        // 2. min / max per block
        for (uint32_t b = warp; b < nblk; b += kWarps) {
            const uint32_t n_b = (uint32_t)umin64(L, cnt - (uint64_t)b * L);
            block_minmax<T>(reinterpret_cast<T *>(smem + (uint64_t)b * cfg.stage_bytes), n_b,
                            &bv.vmin[b], &bv.B[b]);
        }
        __syncthreads();

        // 3-4. word counts, scan, look-back
        if (warp == 0) {
            uint32_t W = 0;
            if (lane < nblk) {
                const uint64_t B = bv.B[lane];
                const uint32_t n_b = (uint32_t)umin64(L, cnt - (uint64_t)lane * L);
                if (B > 1) {
                    if constexpr (VAR == PC_VARIANT_BASIC) {
                        const uint32_t p = basic_p(B, WB);
                        bv.p[lane] = p;
                        W = (n_b + p - 1) / p;
                    } else {
                        W = walk_series<WB>(B, n_b, sched_all + (uint64_t)lane * cfg.wcap, cfg.wcap);
                        if (W == ~0u) {
                            record_error(ws, PC_ERR_INVALID_ARG);
                            W = 0;
                        }
                    }
                }
                bv.W[lane] = W;
            }
            const uint32_t incl = warp_incl_scan_u32(W);
            if (lane < nblk) bv.woff[lane] = incl - W;
            const uint32_t agg = __shfl_sync(0xFFFFFFFFu, incl, 31);
            uint64_t excl = 0;
            const bool ok = lookback_warp(status, tile, agg, ws, limit_ns, &excl);
            if (lane == 0) {
                bv.excl = excl;
                bv.ok = ok ? 1u : 0u;
            }
        }
        __syncthreads();

        if (bv.ok) {
            // 5a. block table: (vmin, B - 1) per block
            for (uint32_t b = threadIdx.x; b < nblk; b += kThreads) {
                const uint64_t gb = blk0 + b;
                const uint64_t Bm1 = bv.B[b] - 1;
                if constexpr (D == 16) {
                    reinterpret_cast<uint32_t *>(out + PC_HEADER_BYTES)[gb] =
                        bv.vmin[b] | ((uint32_t)Bm1 << 16);
                } else {
                    reinterpret_cast<uint64_t *>(out + PC_HEADER_BYTES)[gb] =
                        (uint64_t)bv.vmin[b] | (Bm1 << 32);
                }
            }
            // 5b. packed words, one warp per block, lanes over words
            Word *payload = reinterpret_cast<Word *>(out + payload_off);
            for (uint32_t b = warp; b < nblk; b += kWarps) {
                const uint32_t W = bv.W[b];
                if (W == 0) continue;
                const T *u = reinterpret_cast<const T *>(smem + (uint64_t)b * cfg.stage_bytes);
                const uint32_t vmin = bv.vmin[b];
                const uint32_t B32 = (uint32_t)bv.B[b];  // B = 2^32 only with p = 1: never multiplies
                Word *dst = payload + bv.excl + bv.woff[b];
                if constexpr (VAR == PC_VARIANT_BASIC) {
                    const uint32_t p = bv.p[b];
                    for (uint32_t j = lane; j < W; j += 32)
                        dst[j] = basic_word<T, WB>(u + (uint64_t)j * p, p, B32, vmin);
                } else {
                    const uint64_t *sched = sched_all + (uint64_t)b * cfg.wcap;
                    for (uint32_t j = lane; j < W; j += 32)
                        dst[j] = adv_word<T, WB>(u, sched, j, B32, vmin);
                }
            }
            // 5c. the last tile closes the stream
            if (tile == n_tiles - 1) {
                const uint64_t payload_words = bv.excl + bv.woff[nblk - 1] + bv.W[nblk - 1];
                const uint64_t tend = PC_HEADER_BYTES + n_blocks * 2u * (D / 8);
                for (uint64_t o = tend + threadIdx.x; o < payload_off; o += kThreads) out[o] = 0;
                if (threadIdx.x == 0) write_header(payload_words);
            }
        }
        __syncthreads();
    }
}

template <typename T, uint32_t WB, uint32_t VAR>
static cudaError_t launch_compress_t(const LaunchArgs &a)
{
    auto kern = k_compress<T, WB, VAR>;
    const TileCfg cfg = tile_cfg(VAR, sizeof(T) * 8, WB, a.L);
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)cfg.smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0, dev = 0, sms = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kThreads, cfg.smem)) != cudaSuccess)
        return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    uint64_t grid = (uint64_t)per_sm * sms;
    if (a.n_tiles < grid) grid = a.n_tiles;
    if (grid < 1) grid = 1;
    kern<<<(unsigned)grid, kThreads, cfg.smem, a.stream>>>(
        static_cast<const T *>(a.in), a.n, a.L, static_cast<uint8_t *>(a.out), a.out_count,
        a.ws, a.status, a.n_blocks, a.n_tiles, a.limit_ns);
    return cudaGetLastError();
}

cudaError_t launch_compress(const LaunchArgs &a)
{
    const uint32_t key = (a.d == 32 ? 4u : 0u) | (a.w == 64 ? 2u : 0u) | (a.variant ? 1u : 0u);
    switch (key) {
    case 0: return launch_compress_t<uint16_t, 32, 0>(a);
    case 1: return launch_compress_t<uint16_t, 32, 1>(a);
    case 2: return launch_compress_t<uint16_t, 64, 0>(a);
    case 3: return launch_compress_t<uint16_t, 64, 1>(a);
    case 4: return launch_compress_t<uint32_t, 32, 0>(a);
    case 5: return launch_compress_t<uint32_t, 32, 1>(a);
    case 6: return launch_compress_t<uint32_t, 64, 0>(a);
    default: return launch_compress_t<uint32_t, 64, 1>(a);
    }
}

}  // namespace pcx
