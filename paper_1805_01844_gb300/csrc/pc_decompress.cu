// pc_decompress.cu -- the decompression kernel (sm_103a).
//
// A persistent grid; each CTA validates the stream header, then takes tiles
// of blocks in order from an atomic ticket.  Per tile:
//   1. block table entries -> (min, B) -> word counts (basic: Eq. 1, 2;
//      advanced: the split-base series of Sec. 3.2, one lane per block);
//   2. warp scan + decoupled look-back -> payload offset of the tile, checked
//      against the stream bounds before anything is read;
//   3. one warp per block, lanes over words: polynomial division of each word
//      into its digits (Sec. 3.1), with per-block magic reciprocals of B and
//      of B^h (the largest power <= 2^32) so that the per-digit path has no
//      division instruction, and validity checks of every word;
//   4. coalesced 16-byte stores of the tile's samples.
#include <cuda_runtime.h>

#include "pc_device.cuh"
#include "pc_kernels.h"

namespace pcx {

template <typename T, uint32_t WB>
struct WordT;
template <typename T>
struct WordT<T, 32> { using type = uint32_t; };
template <typename T>
struct WordT<T, 64> { using type = uint64_t; };

// s = q D + r for an invariant D in [2, 2^32]: q is estimated from
// M = floor((2^64 - 1) / D) by a high multiply, and is q or q - 1 (s < 2^64),
// fixed by one compare.
__device__ __forceinline__ uint64_t divmod_inv64(uint64_t s, uint64_t D, uint64_t M, uint64_t &r)
{
    uint64_t q = __umul64hi(s, M);
    uint64_t rr = s - q * D;
    if (rr >= D) {
        ++q;
        rr -= D;
    }
    r = rr;
    return q;
}

// Digits of x (< B^k), least significant first, into dst[0..k), plus vmin.
template <typename T>
__device__ __forceinline__ void put_digits(T *dst, uint32_t x, uint32_t k, uint32_t B32, Magic32 mg,
                                           uint32_t vmin)
{
    for (uint32_t i = 0; i + 1 < k; ++i) {
        const uint32_t q = magic_div(x, mg);
        dst[i] = (T)(x - q * B32 + vmin);
        x = q;
    }
    dst[k - 1] = (T)(x + vmin);
}

template <typename T, uint32_t WB, uint32_t VAR>
__global__ void __launch_bounds__(kThreads)
k_decompress(const uint8_t *__restrict__ in, uint64_t in_bytes, uint32_t L, T *__restrict__ out,
             uint64_t cap, uint64_t *__restrict__ n_out, WsHeader *ws, uint64_t *status,
             uint64_t ws_tiles, uint64_t limit_ns)
{
    using Word = typename WordT<T, WB>::type;
    constexpr uint32_t D = sizeof(T) * 8;
    constexpr uint32_t DB = D / 8, WBY = WB / 8;
    constexpr uint64_t kDmax = D == 16 ? 0xFFFFull : 0xFFFFFFFFull;
    extern __shared__ __align__(16) uint8_t smem[];
    const TileCfg cfg = tile_cfg(VAR, D, WB, L);
    BlockVars &bv = *reinterpret_cast<BlockVars *>(smem + cfg.off_blk);
    uint64_t *sched_all = reinterpret_cast<uint64_t *>(smem + cfg.off_sched);
    uint32_t *tops_all = reinterpret_cast<uint32_t *>(smem + cfg.off_tops);
    __shared__ uint64_t hdr[4];  // n, n_blocks, payload_words, error code
    const uint32_t warp = threadIdx.x >> 5, lane = threadIdx.x & 31u;

    // ---- header: every CTA validates it (64 bytes, L2-resident)
    if (threadIdx.x == 0) {
        const uint32_t *h = reinterpret_cast<const uint32_t *>(in);
        const uint64_t *h64 = reinterpret_cast<const uint64_t *>(in);
        uint64_t code = 0;
        const uint64_t n = h64[2], nb = h64[3], pw = h64[4];
        if (h[0] != 0x504D4350u || h[1] != (1u | (VAR << 16) | (D << 24)) || h[2] != WB || h[3] != L ||
            h64[5] != 0 || h64[6] != 0 || h64[7] != 0)
            code = PC_ERR_CORRUPT;
        else if (nb != n / L + (n % L != 0))
            code = PC_ERR_CORRUPT;
        else if (n > cap)
            code = PC_ERR_CAPACITY;
        else if (nb > (in_bytes - PC_HEADER_BYTES) / (2 * DB))
            code = PC_ERR_CORRUPT;
        else {
            const uint64_t poff = PC_HEADER_BYTES + table_bytes(nb, D);
            if (poff > in_bytes || pw > (in_bytes - poff) / WBY)
                code = PC_ERR_CORRUPT;
            else if (ceil_div(nb, cfg.tb) > ws_tiles)
                code = PC_ERR_INVALID_ARG;
        }
        hdr[0] = n;
        hdr[1] = nb;
        hdr[2] = pw;
        hdr[3] = code;
    }
    __syncthreads();
    if (hdr[3] != 0) {
        if (blockIdx.x == 0 && threadIdx.x == 0) record_error(ws, (uint32_t)hdr[3]);
        return;
    }
    const uint64_t n = hdr[0], n_blocks = hdr[1], payload_words = hdr[2];
    const uint64_t n_tiles = ceil_div(n_blocks, cfg.tb);
    const uint64_t payload_off = PC_HEADER_BYTES + table_bytes(n_blocks, D);
    const Word *payload = reinterpret_cast<const Word *>(in + payload_off);
    if (n_tiles == 0) {
        if (blockIdx.x == 0 && threadIdx.x == 0) {
            if (payload_words != 0) record_error(ws, PC_ERR_CORRUPT);
            *n_out = 0;
        }
        return;
    }

    for (;;) {
        if (threadIdx.x == 0) {
            bv.tile = atomicAdd(&ws->ticket, 1u);
            bv.bad = 0;
        }
        __syncthreads();
        const uint64_t tile = bv.tile;
        if (tile >= n_tiles) break;
        const uint64_t blk0 = tile * cfg.tb;
        const uint32_t nblk = (uint32_t)umin64(cfg.tb, n_blocks - blk0);
        const uint64_t g0 = blk0 * L;
        const uint64_t cnt = umin64(n - g0, (uint64_t)nblk * L);

        // 1-2. table -> counts -> scan -> look-back -> bounds
        if (warp == 0) {
            uint32_t W = 0;
            if (lane < nblk) {
                const uint64_t gb = blk0 + lane;
                uint64_t vmin, Bm1;
                if constexpr (D == 16) {
                    const uint32_t e = reinterpret_cast<const uint32_t *>(in + PC_HEADER_BYTES)[gb];
                    vmin = e & 0xFFFFu;
                    Bm1 = e >> 16;
                } else {
                    const uint64_t e = reinterpret_cast<const uint64_t *>(in + PC_HEADER_BYTES)[gb];
                    vmin = e & 0xFFFFFFFFull;
                    Bm1 = e >> 32;
                }
                if (vmin + Bm1 > kDmax) {
                    record_error(ws, PC_ERR_CORRUPT);
                    Bm1 = 0;
                }
                const uint64_t B = Bm1 + 1;
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
                bv.vmin[lane] = (uint32_t)vmin;
                bv.B[lane] = B;
                bv.W[lane] = W;
            }
            const uint32_t incl = warp_incl_scan_u32(W);
            if (lane < nblk) bv.woff[lane] = incl - W;
            const uint32_t agg = __shfl_sync(0xFFFFFFFFu, incl, 31);
            uint64_t excl = 0;
            bool ok = lookback_warp(status, tile, agg, ws, limit_ns, &excl);
            if (lane == 0) {
                const uint64_t end = excl + agg;
                if (ok && end > payload_words) {  // payload_words fits in in_bytes (header check)
                    record_error(ws, PC_ERR_CORRUPT);
                    ok = false;
                }
                if (ok && tile == n_tiles - 1) {
                    if (end != payload_words) record_error(ws, PC_ERR_CORRUPT);
                    for (uint64_t o = PC_HEADER_BYTES + n_blocks * 2 * DB; o < payload_off; ++o)
                        if (in[o] != 0) record_error(ws, PC_ERR_CORRUPT);
                }
                bv.excl = excl;
                bv.ok = ok ? 1u : 0u;
            }
        }
        __syncthreads();

        if (bv.ok) {
            // 3. decode, one warp per block
            for (uint32_t b = warp; b < nblk; b += kWarps) {
                T *u = reinterpret_cast<T *>(smem + (uint64_t)b * cfg.stage_bytes);
                const uint32_t W = bv.W[b];
                const uint32_t vmin = bv.vmin[b];
                const uint64_t B = bv.B[b];
                const uint32_t n_b = (uint32_t)umin64(L, cnt - (uint64_t)b * L);
                if (W == 0) {  // B = 1: every sample is the minimum
                    for (uint32_t i = lane; i < n_b; i += 32) u[i] = (T)vmin;
                    continue;
                }
                const Word *src = payload + bv.excl + bv.woff[b];
                const uint32_t B32 = (uint32_t)B;
                bool bad = false;
                if constexpr (VAR == PC_VARIANT_BASIC) {
                    const uint32_t p = bv.p[b];
                    const Magic32 mg = magic32(B);
                    // B^p bounds every full word; B^k the last (k real digits)
                    const uint32_t k_last = n_b - (W - 1) * p;
                    uint64_t lim_full = 1, lim_last = 1;
                    for (uint32_t i = 0; i < p; ++i) {
                        if (i < k_last) lim_last *= B;
                        lim_full *= B;
                    }
                    uint32_t hstar = 1;  // largest h with B^h <= 2^32
                    uint64_t Dh = B;
                    while (Dh <= (1ull << 32) / B) {
                        Dh *= B;
                        ++hstar;
                    }
                    const uint64_t MD = ~0ull / Dh;
                    for (uint32_t j = lane; j < W; j += 32) {
                        const uint64_t s = src[j];
                        bad |= s >= (j == W - 1 ? lim_last : lim_full);
                        T *dst = u + (uint64_t)j * p;
                        if (WB == 32 || p <= hstar) {
                            put_digits<T>(dst, (uint32_t)s, p, B32, mg, vmin);
                        } else {
                            uint64_t qv = s;
                            uint32_t rem = p;
                            while (rem > hstar) {
                                uint64_t piece;
                                qv = divmod_inv64(qv, Dh, MD, piece);
                                put_digits<T>(dst, (uint32_t)piece, hstar, B32, mg, vmin);
                                dst += hstar;
                                rem -= hstar;
                            }
                            put_digits<T>(dst, (uint32_t)qv, rem, B32, mg, vmin);
                        }
                    }
                } else {
                    const uint64_t *sched = sched_all + (uint64_t)b * cfg.wcap;
                    uint32_t *tops = tops_all + (uint64_t)b * cfg.wcap;
                    const uint64_t MB = ~0ull / B;
                    // phase A: digits, low parts r_i into the split slots, high parts aside
                    for (uint32_t i = lane; i < W; i += 32) {
                        const uint64_t e = sched[i];
                        const uint32_t R = (uint32_t)e;
                        const uint32_t p = (uint32_t)(e >> 32) & 0xFFu;
                        const uint32_t q = (uint32_t)(e >> 40);
                        const uint64_t s = src[i];
                        uint64_t body = s / R;
                        const uint32_t r = (uint32_t)(s - body * R);
                        for (uint32_t k = p; k > 0; --k) {
                            uint64_t dgt;
                            body = divmod_inv64(body, B, MB, dgt);
                            const uint32_t idx = q + k - 1;
                            if (idx < n_b) u[idx] = (T)(dgt + vmin);
                            else bad |= dgt != 0;
                        }
                        if (i == 0) bad |= body != 0;
                        else {
                            bad |= body > 0xFFFFFFFFull;
                            tops[i] = (uint32_t)body;
                        }
                        const uint32_t split = q + p;
                        if (split >= n_b) bad |= r != 0;
                        else u[split] = (T)r;
                    }
                    __syncwarp();
                    // phase B: re-join each split sample, e = r'_{i-1} R_{i-1} + r_{i-1}
                    for (uint32_t i = lane; i < W; i += 32) {
                        if (i == 0) continue;
                        const uint32_t Rp = (uint32_t)sched[i - 1];
                        const uint32_t q = (uint32_t)(sched[i] >> 40);
                        const uint64_t val = (uint64_t)tops[i] * Rp + (uint32_t)u[q - 1];
                        bad |= val >= B;
                        u[q - 1] = (T)(val + vmin);
                    }
                }
                if (bad) atomicOr(&bv.bad, 1u);
                __syncwarp();
            }
            __syncthreads();
            if (threadIdx.x == 0 && bv.bad) record_error(ws, PC_ERR_CORRUPT);
            // 4. samples out
            store_tile<T>(out, g0, cnt, L, smem, cfg.stage_bytes);
            if (tile == n_tiles - 1 && threadIdx.x == 0) *n_out = n;
        }
        __syncthreads();
    }
}

template <typename T, uint32_t WB, uint32_t VAR>
static cudaError_t launch_decompress_t(const LaunchArgs &a)
{
    auto kern = k_decompress<T, WB, VAR>;
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
    if (a.ws_tiles < grid) grid = a.ws_tiles;
    if (grid < 1) grid = 1;
    kern<<<(unsigned)grid, kThreads, cfg.smem, a.stream>>>(
        static_cast<const uint8_t *>(a.in), a.in_bytes, a.L, static_cast<T *>(a.out), a.cap,
        a.out_count, a.ws, a.status, a.ws_tiles, a.limit_ns);
    return cudaGetLastError();
}

cudaError_t launch_decompress(const LaunchArgs &a)
{
    const uint32_t key = (a.d == 32 ? 4u : 0u) | (a.w == 64 ? 2u : 0u) | (a.variant ? 1u : 0u);
    switch (key) {
    case 0: return launch_decompress_t<uint16_t, 32, 0>(a);
    case 1: return launch_decompress_t<uint16_t, 32, 1>(a);
    case 2: return launch_decompress_t<uint16_t, 64, 0>(a);
    case 3: return launch_decompress_t<uint16_t, 64, 1>(a);
    case 4: return launch_decompress_t<uint32_t, 32, 0>(a);
    case 5: return launch_decompress_t<uint32_t, 32, 1>(a);
    case 6: return launch_decompress_t<uint32_t, 64, 0>(a);
    default: return launch_decompress_t<uint32_t, 64, 1>(a);
    }
}

// Self-test of the bounded wait: tile 1 looks back at tile 0, which nothing
// ever publishes; the wait must give up after limit_ns and record a timeout.
__global__ void k_selftest_wait(WsHeader *ws, uint64_t *status, uint64_t limit_ns)
{
    uint64_t excl = 0;
    lookback_warp(status, 1, 0, ws, limit_ns, &excl);
}

cudaError_t launch_selftest_wait(WsHeader *ws, uint64_t *status, uint64_t limit_ns, cudaStream_t stream)
{
    k_selftest_wait<<<1, 32, 0, stream>>>(ws, status, limit_ns);
    return cudaGetLastError();
}

}  // namespace pcx
