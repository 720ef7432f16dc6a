// pc_compress.cuh -- device code of the fused compression kernels (sm_103a),
// shared by the single-stream kernel (pc_compress.cu) and the batch kernel
// (pc_batch.cu).
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
#pragma once

#include <cuda_runtime.h>

#include <type_traits>

#include "pc_device.cuh"
#include "pc_kernels.h"
#include "pc_orbit.cuh"

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

// Horner over p raw samples starting from acc = top (the advanced word puts
// its first sample in the highest power); modulo 2^w.
template <typename T, uint32_t WB, uint32_t P>
__device__ __forceinline__ uint64_t horner_top_k(uint32_t top, const T *dg, uint32_t B32)
{
    if constexpr (WB == 32) {
        uint32_t acc = top;
#pragma unroll
        for (uint32_t k = 0; k < P; ++k) acc = acc * B32 + (uint32_t)dg[k];
        return acc;
    } else {
        uint32_t lo = top, hi = 0;
#pragma unroll
        for (uint32_t k = 0; k < P; ++k) mad64(lo, hi, B32, (uint32_t)dg[k]);
        return ((uint64_t)hi << 32) | lo;
    }
}

template <typename T, uint32_t WB>
__device__ __forceinline__ uint64_t horner_top(uint32_t top, const T *dg, uint32_t p, uint32_t B32)
{
    switch (p) {
    case 0: return top;
    case 1: return horner_top_k<T, WB, 1>(top, dg, B32);
    case 2: return horner_top_k<T, WB, 2>(top, dg, B32);
    case 3: return horner_top_k<T, WB, 3>(top, dg, B32);
    case 4: return horner_top_k<T, WB, 4>(top, dg, B32);
    case 5: return horner_top_k<T, WB, 5>(top, dg, B32);
    case 6: return horner_top_k<T, WB, 6>(top, dg, B32);
    case 7: return horner_top_k<T, WB, 7>(top, dg, B32);
    case 8: return horner_top_k<T, WB, 8>(top, dg, B32);
    case 9: return horner_top_k<T, WB, 9>(top, dg, B32);
    case 10: return horner_top_k<T, WB, 10>(top, dg, B32);
    case 11: return horner_top_k<T, WB, 11>(top, dg, B32);
    case 12: return horner_top_k<T, WB, 12>(top, dg, B32);
    default:
        if constexpr (WB == 32) {
            uint32_t acc = top;
            for (uint32_t k = 0; k < p; ++k) acc = acc * B32 + (uint32_t)dg[k];
            return acc;
        } else {
            uint32_t lo = top, hi = 0;
            for (uint32_t k = 0; k < p; ++k) mad64(lo, hi, B32, (uint32_t)dg[k]);
            return ((uint64_t)hi << 32) | lo;
        }
    }
}

// Sec. 3.2 words of one block from the series table, one warp, lanes over
// consecutive words; R_{i-1} and its reciprocal come from the lane before
// (the previous 32 words' last lane for lane 0).  Word i:
//   r'_{i-1} = u[q_i - 1] div R_{i-1},  r_i = u[q_i + p_i] mod R_i,
//   s_i = (Horner(r'_{i-1}; u[q_i .. q_i + p_i)) - K_{p_i}) R_i + r_i.
template <typename T, uint32_t WB>
__device__ __forceinline__ void adv_words_orbit(const OrbitTable &ot, const OrbitView &v, const T *u,
                                                uint32_t W, uint32_t B32, uint32_t vmin, uint32_t p1,
                                                uint64_t Kp1, uint64_t Kp0,
                                                typename WordOf<T, WB>::type *dst)
{
    using Word = typename WordOf<T, WB>::type;
    const uint32_t lane = threadIdx.x & 31u;
    uint32_t cR = 1, cm = 0, ca = 0, cs = 0;  // carry: entry of the word before this chunk
    for (uint32_t j0 = 0; j0 < W; j0 += 32) {
        const uint32_t i = j0 + lane;
        const bool valid = i < W;
        SeriesEntry e;
        if (valid) e = orbit_entry(ot, v, i);
        else e = SeriesEntry{1u, 0u, 0u, Magic32{0xFFFFFFFFu, 0xFFFFFFFFu, 0u}};
        uint32_t Rp = __shfl_up_sync(0xFFFFFFFFu, e.R, 1);
        Magic32 mp;
        mp.m = __shfl_up_sync(0xFFFFFFFFu, e.mgR.m, 1);
        mp.a = __shfl_up_sync(0xFFFFFFFFu, e.mgR.a, 1);
        mp.s = __shfl_up_sync(0xFFFFFFFFu, e.mgR.s, 1);
        if (lane == 0) {
            Rp = cR;
            mp = Magic32{cm, ca, cs};
        }
        cR = __shfl_sync(0xFFFFFFFFu, e.R, 31);
        cm = __shfl_sync(0xFFFFFFFFu, e.mgR.m, 31);
        ca = __shfl_sync(0xFFFFFFFFu, e.mgR.a, 31);
        cs = __shfl_sync(0xFFFFFFFFu, e.mgR.s, 31);
        if (!valid) continue;
        const uint32_t top = i > 0 ? magic_div((uint32_t)u[e.q - 1] - vmin, mp) : 0u;
        const uint32_t es = (uint32_t)u[e.q + e.p] - vmin;
        const uint32_t r = es - magic_div(es, e.mgR) * e.R;
        const uint64_t acc = horner_top<T, WB>(top, u + e.q, e.p, B32) - (e.p == p1 ? Kp1 : Kp0);
        if constexpr (WB == 32) {
            dst[i] = (Word)((uint32_t)acc * e.R + r);
        } else {
            uint32_t lo = (uint32_t)acc, hi = (uint32_t)(acc >> 32);
            mad64(lo, hi, e.R, r);
            dst[i] = ((uint64_t)hi << 32) | lo;
        }
    }
}

// Basic words j0 + lane + 32 k (k < NK) of one block by one warp, NK words
// per lane in lockstep so that their Horner chains are independent for the
// scheduler.  Each word is summed as 32-bit pieces (PackK): one 32-bit
// multiply-add per digit, one 64-bit multiply-add per piece boundary.  Lanes
// past the last word recompute the last word and do not store it.
// 16x2 min/max in the multi-stage basic tiles (measured: +2 % on camera
// events at L = 1024; in the single-stage tiles, whose short blocks run in
// 128-thread CTAs, -15 % at L = 256)
#ifndef PCX_MINMAX_U16X2
#define PCX_MINMAX_U16X2 1
#endif
#ifndef PCX_PACK_FLAT
#define PCX_PACK_FLAT 1
#endif
#ifndef PCX_PACK_UNROLL
#define PCX_PACK_UNROLL 1
#endif

template <typename T, uint32_t WB, uint32_t NK, bool FULL = false>
__device__ __forceinline__ void pack_basic_group(const T *u, uint32_t j0, uint32_t W, uint32_t p, uint32_t B32,
                                                 PackK pk, typename WordOf<T, WB>::type *dst)
{
    using Word = typename WordOf<T, WB>::type;
    const uint32_t lane = threadIdx.x & 31u;
    const T *g[NK];
#pragma unroll
    for (uint32_t k = 0; k < NK; ++k) {
        const uint32_t j = FULL ? j0 + lane + 32 * k : min(j0 + lane + 32 * k, W - 1);
        g[k] = u + j * p;
    }
    Word acc[NK];
    if constexpr (WB == 32) {  // one piece
        uint32_t a[NK];
#pragma unroll
        for (uint32_t k = 0; k < NK; ++k) a[k] = g[k][p - 1];
#pragma unroll 2  // 32-bit words: measured +8 % at L = 256 (none at 64 bits)
        for (int d = (int)p - 2; d >= 0; --d) {
#pragma unroll
            for (uint32_t k = 0; k < NK; ++k) a[k] = a[k] * B32 + (uint32_t)g[k][d];
        }
#pragma unroll
        for (uint32_t k = 0; k < NK; ++k) acc[k] = a[k] - pk.Kt;
    } else {
        const int p32 = (int)(pk.shape & 0xFFu), t = (int)(pk.shape >> 16);
        uint32_t a[NK], lo[NK], hi[NK];
        // the top piece: digits p - 1 down to p - t
        int d = (int)p - 1;
#pragma unroll
        for (uint32_t k = 0; k < NK; ++k) a[k] = g[k][d];
#if PCX_PACK_UNROLL
#pragma unroll 2
#endif
        for (--d; d >= (int)p - t; --d) {
#pragma unroll
            for (uint32_t k = 0; k < NK; ++k) a[k] = a[k] * B32 + (uint32_t)g[k][d];
        }
#pragma unroll
        for (uint32_t k = 0; k < NK; ++k) {
            lo[k] = a[k] - pk.Kt;
            hi[k] = 0;
        }
        // the lower pieces, p32 digits each: d is the top digit of the next one
        for (; d >= 0; d -= p32) {
#pragma unroll
            for (uint32_t k = 0; k < NK; ++k) a[k] = g[k][d];
#if PCX_PACK_UNROLL
#pragma unroll 2
#endif
            for (int e = d - 1; e > d - p32; --e) {
#pragma unroll
                for (uint32_t k = 0; k < NK; ++k) a[k] = a[k] * B32 + (uint32_t)g[k][e];
            }
#pragma unroll
            for (uint32_t k = 0; k < NK; ++k) mad64(lo[k], hi[k], pk.D, a[k] - pk.Kf);
        }
#pragma unroll
        for (uint32_t k = 0; k < NK; ++k) acc[k] = ((uint64_t)hi[k] << 32) | lo[k];
    }
#pragma unroll
    for (uint32_t k = 0; k < NK; ++k) {
        const uint32_t j = j0 + lane + 32 * k;
        if (FULL || j < W) dst[j] = acc[k];
    }
}

// One basic word (as in pack_basic_group, for one lane): digits dg[0..p) of
// raw samples, summed as 32-bit pieces (PackK).
template <typename T, uint32_t WB>
__device__ __forceinline__ typename WordOf<T, WB>::type basic_word_pk(const T *dg, uint32_t p, uint32_t B32,
                                                                     PackK pk)
{
    uint32_t a = dg[p - 1];
    if constexpr (WB == 32) {
        for (int d = (int)p - 2; d >= 0; --d) a = a * B32 + (uint32_t)dg[d];
        return a - pk.Kt;
    } else {
        const int p32 = (int)(pk.shape & 0xFFu), t = (int)(pk.shape >> 16);
        int d = (int)p - 2;
        for (; d >= (int)p - t; --d) a = a * B32 + (uint32_t)dg[d];
        uint32_t lo = a - pk.Kt, hi = 0;
        for (; d >= 0; d -= p32) {
            a = dg[d];
            for (int e = d - 1; e > d - p32; --e) a = a * B32 + (uint32_t)dg[e];
            mad64(lo, hi, pk.D, a - pk.Kf);
        }
        return ((uint64_t)hi << 32) | lo;
    }
}

// Basic words of a whole tile with few words per block (short blocks): the
// tile's words taken as one sequence, a lane per word, so lanes do not idle
// on blocks of fewer than 32 words.  Word g belongs to the last block b with
// woff[b] <= g (a block without words shares its offset with the next).
template <typename T, uint32_t WB, uint32_t NT>
__device__ __forceinline__ void pack_basic_flat(const uint8_t *stage, uint32_t stage_bytes, const uint32_t *woff,
                                                const uint32_t *p_of, const uint64_t *B_of, const PackK *pk_of,
                                                uint32_t nblk, uint32_t agg, typename WordOf<T, WB>::type *dst)
{
    for (uint32_t g = threadIdx.x; g < agg; g += NT) {
        uint32_t lo = 0, hi = nblk - 1;
        while (lo < hi) {
            const uint32_t mid = (lo + hi + 1) >> 1;
            if (woff[mid] <= g) lo = mid;
            else hi = mid - 1;
        }
        const uint32_t p = p_of[lo];
        const T *dg = reinterpret_cast<const T *>(stage + (uint64_t)lo * stage_bytes) + (g - woff[lo]) * p;
        dst[g] = basic_word_pk<T, WB>(dg, p, (uint32_t)B_of[lo], pk_of[lo]);
    }
}

// Basic words of one block by one warp: groups of 128 words (four per lane),
// then the last 1..127 words in the fewest lockstep slots per lane.
template <typename T, uint32_t WB>
__device__ __forceinline__ void pack_basic_block(const T *u, uint32_t W, uint32_t p, uint32_t B32, PackK pk,
                                                 typename WordOf<T, WB>::type *dst)
{
    uint32_t j0 = 0;
    for (; j0 + 128 <= W; j0 += 128) pack_basic_group<T, WB, 4, true>(u, j0, W, p, B32, pk, dst);
    const uint32_t rest = W - j0;
    if (rest > 96) pack_basic_group<T, WB, 4>(u, j0, W, p, B32, pk, dst);
    else if (rest > 64) pack_basic_group<T, WB, 3>(u, j0, W, p, B32, pk, dst);
    else if (rest > 32) pack_basic_group<T, WB, 2>(u, j0, W, p, B32, pk, dst);
    else if (rest > 0) pack_basic_group<T, WB, 1>(u, j0, W, p, B32, pk, dst);
}

// The 64-byte stream header (format version 1, include/pc.h).
template <uint32_t D, uint32_t WB, uint32_t VAR>
__device__ __forceinline__ void write_header(uint8_t *out, uint32_t L, uint64_t n, uint64_t n_blocks,
                                             uint64_t payload_words)
{
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
}

// One mbarrier per warp for the bulk copies of its blocks (compression tiles).
__shared__ uint64_t g_stage_bar[kMaxTileBlocks / 4];
// Set when a staging wait gave up: the CTA issues no more bulk copies and
// packs nothing more, its tile publishes an error for the look-back of its
// successors, and it takes no further tile.  A bulk copy that never completes
// may still write into the stage when the CTA exits.
__shared__ uint32_t g_stage_dead;

__device__ __forceinline__ void stage_bars_init()
{
    if (threadIdx.x < kMaxTileBlocks / 4) mbar_init(&g_stage_bar[threadIdx.x], 1);
    if (threadIdx.x == 0) g_stage_dead = 0;
    mbar_init_fence();
    __syncthreads();
}

// The staging state of the CTA, as lane 0 of the calling warp sees it.
__device__ __forceinline__ bool stage_dead()
{
    uint32_t d = 0;
    if ((threadIdx.x & 31u) == 0) d = *reinterpret_cast<volatile uint32_t *>(&g_stage_dead);
    return __shfl_sync(0xFFFFFFFFu, d, 0) != 0;
}

// Bounded wait for a warp's staged blocks; on giving up, records the timeout
// and marks the CTA's staging dead.
__device__ __forceinline__ void stage_wait(uint32_t warp, uint32_t phase, WsHeader *ws, uint64_t limit_ns)
{
    if (!mbar_wait(&g_stage_bar[warp], phase & 1u, limit_ns) && (threadIdx.x & 31u) == 0) {
        record_error(ws, PC_ERR_TIMEOUT);
        *reinterpret_cast<volatile uint32_t *>(&g_stage_dead) = 1u;
    }
}

// One stream as the compression kernels see it.
struct StreamArgs {
    const void *in;
    uint64_t n;
    uint32_t L;
    uint8_t *out;
    uint64_t *out_bytes;
    uint64_t *status;  // look-back words of this stream's tiles
    uint64_t n_blocks, n_tiles;
    uint32_t tb;       // blocks per tile (the tile layout's, or fewer for a short stream)
    OrbitTable ot;
};

// Compress tile `tile` of stream `sa` with the whole CTA: stage its samples,
// min / max per block (Sec. 3.1), word counts (Eq. 1-2, or the split-base
// series of Sec. 3.2), scan and publish the tile's aggregate, look back to
// its payload offset, then write its table entries and packed words; the last
// tile writes the header, the table padding and the stream size.
template <typename T, uint32_t WB, uint32_t VAR, bool ORB, uint32_t NT = kThreads>
__device__ void compress_tile(const StreamArgs &sa, uint64_t tile, uint8_t *smem, WsHeader *ws, uint64_t limit_ns,
                              uint32_t &phase)
{
    using Word = typename WordOf<T, WB>::type;
    constexpr uint32_t D = sizeof(T) * 8;
    const uint32_t L = sa.L;
    const TileCfg cfg = tile_cfg(kKernelCompress, VAR, D, WB, L, ORB, NT);
    BlockVars &bv = *reinterpret_cast<BlockVars *>(smem + cfg.off_blk);
    uint64_t *sched_all = reinterpret_cast<uint64_t *>(smem + cfg.off_sched);
    const uint32_t warp = threadIdx.x >> 5, lane = threadIdx.x & 31u;
    const T *in = static_cast<const T *>(sa.in);
    const uint64_t n = sa.n, n_blocks = sa.n_blocks, n_tiles = sa.n_tiles;
    const uint64_t payload_off = PC_HEADER_BYTES + table_bytes(n_blocks, D);
    const uint64_t blk0 = tile * sa.tb;
    const uint32_t nblk = (uint32_t)umin64(sa.tb, n_blocks - blk0);
    const uint64_t cnt = umin64(n - blk0 * L, (uint64_t)nblk * L);

    if ((L * sizeof(T)) % 16 == 0) {
        // 1-2. each warp stages its own blocks and finds their min / max as
        // soon as they land: lane 0 issues one bulk copy (TMA engine) per
        // block, completing on the warp's mbarrier; the ragged end of the
        // last block comes element by element
        constexpr uint32_t VE = 16 / sizeof(T);
        {  // (a CTA whose staging died takes no further tile, so it never comes here again)
            // lane i issues the copy of the warp's i-th block (blocks warp,
            // warp + NT / 32, ...), once lane 0 has set the expected bytes
            constexpr uint32_t NW = NT / 32;
            uint32_t bytes = 0;
            for (uint32_t b = warp + lane * NW; b < nblk; b += 32 * NW)
                bytes += ((uint32_t)umin64(L, cnt - (uint64_t)b * L) / VE) * 16u;
            bytes = __reduce_add_sync(0xFFFFFFFFu, bytes);
            fence_proxy_async_smem();  // the stage's earlier generic accesses before the async writes
            if (lane == 0) mbar_arrive_expect_tx(&g_stage_bar[warp], bytes);
            __syncwarp();
            for (uint32_t b = warp + lane * NW; b < nblk; b += 32 * NW) {
                const uint32_t nb16 = ((uint32_t)umin64(L, cnt - (uint64_t)b * L) / VE) * 16u;
                if (nb16)
                    bulk_copy_g2s(smem + (uint64_t)b * cfg.stage_bytes, in + (blk0 + b) * L, nb16,
                                  &g_stage_bar[warp]);
            }
        }
        if (cnt % VE != 0 && (nblk - 1) % (NT / 32) == warp) {  // only the stream's last block can be ragged
            const uint32_t b = nblk - 1;
            const uint32_t n_b = (uint32_t)(cnt - (uint64_t)b * L);
            T *dst = reinterpret_cast<T *>(smem + (uint64_t)b * cfg.stage_bytes);
            for (uint32_t e = n_b / VE * VE + lane; e < n_b; e += 32) dst[e] = in[(blk0 + b) * L + e];
        }
        stage_wait(warp, phase, ws, limit_ns);
        ++phase;  // every warp's barrier completed one phase
        __syncwarp();
        for (uint32_t b = warp; b < nblk; b += (NT / 32)) {
            const uint32_t n_b = (uint32_t)umin64(L, cnt - (uint64_t)b * L);
            block_minmax<T>(reinterpret_cast<T *>(smem + (uint64_t)b * cfg.stage_bytes), n_b, &bv.vmin[b],
                                                    &bv.B[b]);
        }
        __syncthreads();
    } else {
        // 1. stage
        load_tile<T, NT>(in, blk0 * L, cnt, L, smem, cfg.stage_bytes);
        __syncthreads();
        // 2. min / max per block
        for (uint32_t b = warp; b < nblk; b += (NT / 32)) {
            const uint32_t n_b = (uint32_t)umin64(L, cnt - (uint64_t)b * L);
            block_minmax<T>(reinterpret_cast<T *>(smem + (uint64_t)b * cfg.stage_bytes), n_b, &bv.vmin[b],
                                                    &bv.B[b]);
        }
        __syncthreads();
    }

    // 3-4. word counts, scan, aggregate, look-back
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
                    bv.pk[lane] = basic_pack_k(B, p, bv.vmin[lane], WB);
                } else if (ORB && B <= kOrbitMaxB) {
                    // the series from the table: O(1) per word
                    const uint64_t h = orbit_get<WB>(sa.ot, (uint32_t)B, L, ws, limit_ns);
                    if (h != ~0ull) {
                        const OrbitView v = orbit_view(sa.ot, h);
                        W = orbit_words_cached(sa.ot, v, n_b, L);
                        bv.orb_off[lane] = v.off;
                        bv.orb_Q[lane] = v.Q;
                        bv.orb_P[lane] = v.P;
                        bv.orb_SQ[lane] = v.SQ;
                        bv.orb_G[lane] = v.G;
                        bv.orb_mgm[lane] = v.mgP.m;
                        bv.orb_mga[lane] = v.mgP.a;
                        bv.orb_mgs[lane] = v.mgP.s;
                        const uint32_t p1 = eq1_p(B, WB);
                        uint64_t geo = 0, pw = 1, geo0 = 0;  // 1 + B + ... + B^(p-1)
                        for (uint32_t k = 0; k < p1; ++k) {
                            geo0 = geo;
                            geo += pw;
                            pw *= B;
                        }
                        bv.p1[lane] = p1;
                        bv.K[lane] = geo * bv.vmin[lane];
                        bv.K2[lane] = geo0 * bv.vmin[lane];
                    }
                    bv.mode[lane] = 1;
                } else {
                    W = walk_series<WB>(B, n_b, sched_all + (uint64_t)lane * cfg.wcap, cfg.wcap);
                    if (W == ~0u) {
                        record_error(ws, PC_ERR_INVALID_ARG);
                        W = 0;
                    }
                    bv.mode[lane] = 0;
                }
            }
            bv.W[lane] = W;
        }
        const uint32_t incl = warp_incl_scan_u32(W);
        if (lane < nblk) bv.woff[lane] = incl - W;
        const uint32_t agg = __shfl_sync(0xFFFFFFFFu, incl, 31);
        uint64_t excl = 0;
        bool ok = false;
        if (stage_dead()) {  // the staged samples are not whole: successors stop on this tile's error
            if (lane == 0) st_release(&sa.status[tile], kFlagError);
        } else {
            lookback_publish(sa.status, tile, agg);
            ok = lookback_complete(sa.status, tile, agg, ws, limit_ns, &excl);
        }
        if (lane == 0) {
            bv.agg = agg;
            bv.excl = excl;
            bv.ok = ok ? 1u : 0u;
        }
    }
    __syncthreads();

    // 5. table entries, packed words, and the stream's closing bytes
    if (bv.ok) {
        for (uint32_t b = threadIdx.x; b < nblk; b += NT) {
            const uint64_t gb = blk0 + b;
            const uint64_t Bm1 = bv.B[b] - 1;
            if constexpr (D == 16) {
                reinterpret_cast<uint32_t *>(sa.out + PC_HEADER_BYTES)[gb] = bv.vmin[b] | ((uint32_t)Bm1 << 16);
            } else {
                reinterpret_cast<uint64_t *>(sa.out + PC_HEADER_BYTES)[gb] = (uint64_t)bv.vmin[b] | (Bm1 << 32);
            }
        }
        Word *payload = reinterpret_cast<Word *>(sa.out + payload_off);
        // short basic blocks (fewer than 16 words on average): a lane per word
        // over the whole tile instead of a warp per block (measured at 2^30
        // white-noise samples, w = 64: L = 64 +14 %, L = 128 +8 %)
        const bool flat = VAR == PC_VARIANT_BASIC && PCX_PACK_FLAT && bv.agg < 16u * nblk;
        if (flat)
            pack_basic_flat<T, WB, NT>(smem, cfg.stage_bytes, bv.woff, bv.p, bv.B, bv.pk, nblk, bv.agg,
                                       payload + bv.excl);
        for (uint32_t b = warp; b < nblk && !flat; b += (NT / 32)) {
            const uint32_t W = bv.W[b];
            if (W == 0) continue;
            const T *u = reinterpret_cast<const T *>(smem + (uint64_t)b * cfg.stage_bytes);
            const uint32_t vmin = bv.vmin[b];
            const uint32_t B32 = (uint32_t)bv.B[b];  // B = 2^32 only with p = 1: never multiplies
            Word *dst = payload + bv.excl + bv.woff[b];
            if constexpr (VAR == PC_VARIANT_BASIC) {
                pack_basic_block<T, WB>(u, W, bv.p[b], B32, bv.pk[b], dst);
            } else {
                if (ORB && bv.mode[b]) {
                    const OrbitView v{bv.orb_off[b], bv.orb_Q[b], bv.orb_P[b], bv.orb_SQ[b], bv.orb_G[b],
                                      Magic32{bv.orb_mgm[b], bv.orb_mga[b], bv.orb_mgs[b]}};
                    adv_words_orbit<T, WB>(sa.ot, v, u, W, B32, vmin, bv.p1[b], bv.K[b], bv.K2[b], dst);
                } else {
                    const uint64_t *sched = sched_all + (uint64_t)b * cfg.wcap;
                    for (uint32_t j = lane; j < W; j += 32) dst[j] = adv_word<T, WB>(u, sched, j, B32, vmin);
                }
            }
        }
        if (tile == n_tiles - 1) {
            const uint64_t payload_words = bv.excl + bv.agg;
            const uint64_t tend = PC_HEADER_BYTES + n_blocks * 2u * (D / 8);
            for (uint64_t o = tend + threadIdx.x; o < payload_off; o += NT) sa.out[o] = 0;
            if (threadIdx.x == 0) {
                write_header<D, WB, VAR>(sa.out, L, n, n_blocks, payload_words);
                *sa.out_bytes = payload_off + payload_words * (WB / 8);
            }
        }
    }
    __syncthreads();  // the stage and the per-tile arrays are free again
}

// Basic variant, long streams: one look-back tile spans K stage tiles
// (K tb blocks, sa.tb = K tb) staged one after the other in the same shared
// memory.  Each stage tile's min / max are taken before the next overwrites
// its slots; after the single look-back the last stage tile is packed where
// it sits and each warp restages its own blocks of the earlier ones (just
// read, so from L2) and packs them, last to first.  A look-back per K tb
// blocks instead of per tb: measured, each tile's look-back waits several
// microseconds on its predecessors' aggregates, and smaller tiles compress
// markedly slower.
constexpr uint32_t kMultiMaxBlocks = 96;  // blocks of one look-back tile

struct MultiVars {  // per-tile arrays, in the BlockVars space of the stage
    PackK pk[kMultiMaxBlocks];     // the 32-bit pieces of the block's words; p in shape bits 24-31
    uint32_t Bm1[kMultiMaxBlocks];  // B - 1
    uint32_t vmin[kMultiMaxBlocks];
    uint32_t W[kMultiMaxBlocks];
    uint32_t woff[kMultiMaxBlocks];
    uint64_t excl;
    uint32_t agg;
    uint32_t ok;
};
static_assert(sizeof(MultiVars) <= sizeof(BlockVars), "look-back tile arrays fit the stage tile arrays");

// The advanced variant's per-tile arrays (16-bit data, series table): each
// block's view of its base's series and the Horner constants of its words;
// larger than BlockVars, so the launch reserves its size after the stage.
struct AdvMultiVars {
    uint64_t K[kMultiMaxBlocks];   // vmin (1 + ... + B^(p_1 - 1)) mod 2^w
    uint64_t K2[kMultiMaxBlocks];  // the same for p_1 - 1 digits
    uint32_t Bm1[kMultiMaxBlocks];
    uint32_t vmin[kMultiMaxBlocks];
    uint32_t W[kMultiMaxBlocks];
    uint32_t woff[kMultiMaxBlocks];
    uint32_t p1[kMultiMaxBlocks];
    uint32_t off[kMultiMaxBlocks], Q[kMultiMaxBlocks], P[kMultiMaxBlocks], SQ[kMultiMaxBlocks], G[kMultiMaxBlocks];
    uint32_t mgm[kMultiMaxBlocks], mga[kMultiMaxBlocks], mgs[kMultiMaxBlocks];
    uint64_t excl;
    uint32_t agg;
    uint32_t ok;
};

template <uint32_t VAR>
using MultiVarsOf = typename std::conditional<VAR == PC_VARIANT_BASIC, MultiVars, AdvMultiVars>::type;

// Shared memory of a multi-stage tile: the stage, then the per-tile arrays.
template <uint32_t VAR>
PCX_HD uint32_t multi_smem(const TileCfg &cfg)
{
    return (uint32_t)round_up((uint64_t)cfg.off_blk + sizeof(MultiVarsOf<VAR>), 16);
}

// Stage tiles per look-back tile for stage tiles of tb blocks.
#ifndef PCX_MULTI_K_MAX
#define PCX_MULTI_K_MAX 8
#endif
PCX_HD uint32_t multi_k(uint32_t tb)
{
    uint32_t k = kMultiMaxBlocks / tb;
    return k > PCX_MULTI_K_MAX ? PCX_MULTI_K_MAX : k;
}

template <typename T, uint32_t WB, uint32_t NT, bool FOUR, uint32_t VAR = PC_VARIANT_BASIC>
__device__ void compress_tile_multi(const StreamArgs &sa, uint64_t tile, uint8_t *smem, WsHeader *ws,
                                    uint64_t limit_ns, uint32_t &phase)
{
    using Word = typename WordOf<T, WB>::type;
    constexpr uint32_t D = sizeof(T) * 8;
    constexpr uint32_t VE = 16 / sizeof(T);
    constexpr uint32_t NW = NT / 32;
    constexpr bool ADV = VAR == PC_VARIANT_ADVANCED;
    const uint32_t L = sa.L;
    const TileCfg cfg = tile_cfg(kKernelCompress, VAR, D, WB, L, ADV, NT, FOUR ? kTileBudgetMulti4 : 0u);
    const uint32_t H = cfg.tb;  // blocks per stage tile; sa.tb = K H
    MultiVarsOf<VAR> &mv = *reinterpret_cast<MultiVarsOf<VAR> *>(smem + cfg.off_blk);
    const uint32_t warp = threadIdx.x >> 5, lane = threadIdx.x & 31u;
    const T *in = static_cast<const T *>(sa.in);
    const uint64_t n = sa.n, n_blocks = sa.n_blocks, n_tiles = sa.n_tiles;
    const uint64_t payload_off = PC_HEADER_BYTES + table_bytes(n_blocks, D);
    const uint64_t blk0 = tile * sa.tb;
    const uint32_t nblk = (uint32_t)umin64(sa.tb, n_blocks - blk0);
    const uint32_t nst = (nblk + H - 1) / H;  // stage tiles in this tile
    auto nh = [&](uint32_t h) -> uint32_t { return nblk - h * H < H ? nblk - h * H : H; };
    auto n_of = [&](uint32_t b) -> uint32_t { return (uint32_t)umin64(L, n - (blk0 + b) * L); };
    auto slot = [&](uint32_t b) -> T * { return reinterpret_cast<T *>(smem + (uint64_t)(b % H) * cfg.stage_bytes); };

    // this warp's blocks of stage tile h into their slots: one bulk copy per
    // block (lane 0) on the warp's mbarrier, the ragged end by plain loads.
    // A stage tile that will be restaged is read with evict_last priority
    // in L2, the last reads of every tile with evict_first.
    auto stage = [&](uint32_t h, bool again) {
        const uint32_t m = nh(h);
        __syncwarp();  // the warp's earlier accesses to its slots come first
        const bool dead = __any_sync(0xFFFFFFFFu, stage_dead());
        if (!dead) {  // lane i copies the warp's i-th block, once lane 0 has set the expected bytes
            uint32_t bytes = 0;
            for (uint32_t b = warp + lane * NW; b < m; b += 32 * NW) bytes += (n_of(h * H + b) / VE) * 16u;
            bytes = __reduce_add_sync(0xFFFFFFFFu, bytes);
            const uint64_t policy = again ? l2_policy_evict_last() : l2_policy_evict_first();
            fence_proxy_async_smem();
            if (lane == 0) mbar_arrive_expect_tx(&g_stage_bar[warp], bytes);
            __syncwarp();
            for (uint32_t b = warp + lane * NW; b < m; b += 32 * NW) {
                const uint32_t nb16 = (n_of(h * H + b) / VE) * 16u;
                if (nb16)
                    bulk_copy_g2s_hint(slot(b), in + (blk0 + h * H + b) * L, nb16, &g_stage_bar[warp], policy);
            }
        }
        if (n % VE != 0 && blk0 + h * H + m == n_blocks && (m - 1) % NW == warp) {  // the stream's ragged last block
            const uint32_t b = m - 1;
            const uint32_t n_b = n_of(h * H + b);
            T *dst = slot(b);
            for (uint32_t e = n_b / VE * VE + lane; e < n_b; e += 32) dst[e] = in[(blk0 + h * H + b) * L + e];
        }
        if (!dead) stage_wait(warp, phase, ws, limit_ns);
        ++phase;  // every warp's barrier completed one phase
        __syncwarp();
    };

    // 1-2. min / max, stage tile by stage tile over the same slots
    for (uint32_t h = 0; h < nst; ++h) {
        stage(h, h + 1 < nst);
        for (uint32_t b = warp; b < nh(h); b += NW) {
            uint64_t Bb;
            block_minmax<T, PCX_MINMAX_U16X2 && !ADV>(slot(b), n_of(h * H + b), &mv.vmin[h * H + b], &Bb);
            if (lane == 0) mv.Bm1[h * H + b] = (uint32_t)(Bb - 1);
        }
    }
    __syncthreads();

    // 3-4. word counts (lane per block, 32 at a time), scan, aggregate, look-back
    if (warp == 0) {
        uint32_t run = 0;
        for (uint32_t b0 = 0; b0 < nblk; b0 += 32) {
            const uint32_t b = b0 + lane;
            uint32_t W = 0;
            if (b < nblk) {
                const uint64_t B = (uint64_t)mv.Bm1[b] + 1;
                if (B > 1) {
                    if constexpr (!ADV) {
                        const uint32_t p = basic_p(B, WB);
                        W = (n_of(b) + p - 1) / p;
                        PackK pk = basic_pack_k(B, p, mv.vmin[b], WB);
                        pk.shape |= p << 24;
                        mv.pk[b] = pk;
                    } else {  // the series from the table (16-bit data: every base is in it)
                        const uint64_t hd = orbit_get<WB>(sa.ot, (uint32_t)B, L, ws, limit_ns);
                        if (hd != ~0ull) {
                            const OrbitView v = orbit_view(sa.ot, hd);
                            W = orbit_words_cached(sa.ot, v, n_of(b), L);
                            mv.off[b] = v.off;
                            mv.Q[b] = v.Q;
                            mv.P[b] = v.P;
                            mv.SQ[b] = v.SQ;
                            mv.G[b] = v.G;
                            mv.mgm[b] = v.mgP.m;
                            mv.mga[b] = v.mgP.a;
                            mv.mgs[b] = v.mgP.s;
                            const uint32_t p1 = eq1_p(B, WB);
                            uint64_t geo = 0, pw = 1, geo0 = 0;  // 1 + B + ... + B^(p-1)
                            for (uint32_t kk = 0; kk < p1; ++kk) {
                                geo0 = geo;
                                geo += pw;
                                pw *= B;
                            }
                            mv.p1[b] = p1;
                            mv.K[b] = geo * mv.vmin[b];
                            mv.K2[b] = geo0 * mv.vmin[b];
                        }
                    }
                }
                mv.W[b] = W;
            }
            const uint32_t incl = warp_incl_scan_u32(W);
            if (b < nblk) mv.woff[b] = run + incl - W;
            run += __shfl_sync(0xFFFFFFFFu, incl, 31);
        }
        const uint32_t agg = run;
        uint64_t excl = 0;
        bool ok = false;
        if (stage_dead()) {  // the staged samples are not whole: successors stop on this tile's error
            if (lane == 0) st_release(&sa.status[tile], kFlagError);
        } else {
            lookback_publish(sa.status, tile, agg);
            ok = lookback_complete(sa.status, tile, agg, ws, limit_ns, &excl);
        }
        if (lane == 0) {
            mv.agg = agg;
            mv.excl = excl;
            mv.ok = ok ? 1u : 0u;
        }
    }
    __syncthreads();

    // 5. table entries; the last stage tile packed from the stage, then each
    // warp restages and packs its blocks of the earlier ones; the stream's
    // closing bytes
    if (mv.ok) {
        for (uint32_t b = threadIdx.x; b < nblk; b += NT) {
            const uint64_t gb = blk0 + b;
            const uint64_t Bm1 = mv.Bm1[b];
            if constexpr (D == 16) {
                reinterpret_cast<uint32_t *>(sa.out + PC_HEADER_BYTES)[gb] = mv.vmin[b] | ((uint32_t)Bm1 << 16);
            } else {
                reinterpret_cast<uint64_t *>(sa.out + PC_HEADER_BYTES)[gb] = (uint64_t)mv.vmin[b] | (Bm1 << 32);
            }
        }
        Word *payload = reinterpret_cast<Word *>(sa.out + payload_off) + mv.excl;
        for (uint32_t h = nst; h-- > 0;) {
            if (h + 1 < nst) {
                stage(h, false);
                if (stage_dead()) continue;  // this warp's restaged blocks may be incomplete: pack none
                for (uint32_t b = warp; b < nh(h); b += NW) {  // padding: this stage tile's minimum again
                    T *u = slot(b);
                    const uint32_t n_b = n_of(h * H + b);
                    for (uint32_t i = lane; i < kPad; i += 32) u[n_b + i] = (T)mv.vmin[h * H + b];
                }
                __syncwarp();
            }
            for (uint32_t b = warp; b < nh(h); b += NW) {
                const uint32_t bb = h * H + b;
                const uint32_t W = mv.W[bb];
                if (W == 0) continue;
                if constexpr (!ADV) {
                    PackK pk = mv.pk[bb];
                    const uint32_t p = pk.shape >> 24;
                    pk.shape &= 0xFFFFFFu;
                    pack_basic_block<T, WB>(slot(b), W, p, mv.Bm1[bb] + 1u, pk, payload + mv.woff[bb]);
                } else {
                    const OrbitView v{mv.off[bb], mv.Q[bb], mv.P[bb], mv.SQ[bb], mv.G[bb],
                                      Magic32{mv.mgm[bb], mv.mga[bb], mv.mgs[bb]}};
                    adv_words_orbit<T, WB>(sa.ot, v, slot(b), W, mv.Bm1[bb] + 1u, mv.vmin[bb], mv.p1[bb], mv.K[bb],
                                           mv.K2[bb], payload + mv.woff[bb]);
                }
            }
        }
        if (tile == n_tiles - 1) {
            const uint64_t payload_words = mv.excl + mv.agg;
            const uint64_t tend = PC_HEADER_BYTES + n_blocks * 2u * (D / 8);
            for (uint64_t o = tend + threadIdx.x; o < payload_off; o += NT) sa.out[o] = 0;
            if (threadIdx.x == 0) {
                write_header<D, WB, VAR>(sa.out, L, n, n_blocks, payload_words);
                *sa.out_bytes = payload_off + payload_words * (WB / 8);
            }
        }
    }
    __syncthreads();  // the stage and the tile arrays are free again
}

// Header of an empty stream (no blocks).
template <uint32_t D, uint32_t WB, uint32_t VAR>
__device__ void write_empty_stream(const StreamArgs &sa)
{
    write_header<D, WB, VAR>(sa.out, sa.L, 0, 0, 0);
    *sa.out_bytes = PC_HEADER_BYTES;
}

// Single-stream compression: a persistent grid, tiles taken in order from an
// atomic ticket (so a tile only waits on tiles owned by running CTAs).
// CTAs per SM the register allocation must allow: basic tiles (74 KB of
// shared memory) fit three to an SM once registers are capped at 85; so do
// advanced tiles of 16-bit data (about 74 KB at L = 1024; measured: at 84
// registers, which round up past a third of the register file, only two fit
// and compression ran 24 % slower), while 32-bit advanced tiles that walk
// their series use up to 100 KB and fit two.
// ---- short basic blocks (L <= 256) ---------------------------------------
// A look-back tile of up to kShortTileBlocks short blocks, staged whole (no
// restaging): each warp stages its blocks as in compress_tile; after one CTA
// barrier, groups of L / VE lanes take a block's min/max together (one
// 16-byte shared load per lane, a reduction over the group) and set its
// padding; a thread per block counts its words; a CTA scan and one look-back
// per tile; table entries by a thread per block and words packed a lane per
// word across the tile (pack_basic_flat).  The stream's ragged last block
// takes block_minmax.
constexpr uint32_t kShortTileBlocks = 128;
constexpr uint32_t kShortThreads = 256;

struct ShortVars {
    uint64_t B[kShortTileBlocks];
    PackK pk[kShortTileBlocks];
    uint32_t vmin[kShortTileBlocks];
    uint32_t W[kShortTileBlocks];
    uint32_t woff[kShortTileBlocks];
    uint32_t p[kShortTileBlocks];
    uint32_t wtot[kShortThreads / 32];
    uint64_t excl;
    uint32_t agg;
    uint32_t ok;
};

PCX_HD uint32_t short_stage_bytes(uint32_t d, uint32_t L)
{
    return (uint32_t)round_up((uint64_t)(L + kPad) * (d / 8), 16);
}

#ifndef PCX_SHORT_TILES
#define PCX_SHORT_TILES 1
#endif
#ifndef PCX_SHORT_MAXL
#define PCX_SHORT_MAXL 256
#endif
// Streams (or batch items) of short basic blocks that take these tiles: a
// block is a power of two of 16-byte vectors, at most 32 (one per lane of a
// group), and L <= 128, or L = 256 with 64-bit words for 16-bit data (with
// 32-bit words, ~43 words per block, L = 256 measured 18 % slower than the
// multi-stage tiles; with 64-bit words 1-14 % faster).
PCX_HD bool short_tiles_ok(uint32_t variant, uint32_t d, uint32_t w, uint32_t L)
{
    const uint32_t ve = 16 / (d / 8), g = L / ve;
    return PCX_SHORT_TILES && variant == PC_VARIANT_BASIC && L <= PCX_SHORT_MAXL && L % ve == 0 && g <= 32 &&
           (g & (g - 1)) == 0 && (L <= 128 || w == 64);
}

// Blocks per look-back tile: 128, or fewer so that a tile's samples stay
// within 32 KB (four CTAs of 256 threads share an SM's shared memory).
PCX_HD uint32_t short_tile_blocks(uint32_t d, uint32_t L)
{
    const uint32_t tb = 32768u / (L * (d / 8));
    return tb < kShortTileBlocks ? tb : kShortTileBlocks;
}

PCX_HD uint32_t short_smem(uint32_t d, uint32_t L)
{
    return (uint32_t)round_up((uint64_t)short_tile_blocks(d, L) * short_stage_bytes(d, L) + sizeof(ShortVars), 16);
}

template <typename T, uint32_t WB>
__device__ void compress_tile_short(const StreamArgs &sa, uint64_t tile, uint8_t *smem, WsHeader *ws,
                                    uint64_t limit_ns, uint32_t &phase)
{
    using Word = typename WordOf<T, WB>::type;
    constexpr uint32_t D = sizeof(T) * 8, NT = kShortThreads, NW = NT / 32;
    constexpr uint32_t VE = 16 / sizeof(T);
    const uint32_t L = sa.L;
    const uint32_t SB = short_stage_bytes(D, L);
    ShortVars &sv = *reinterpret_cast<ShortVars *>(smem + (uint64_t)sa.tb * SB);
    const uint32_t warp = threadIdx.x >> 5, lane = threadIdx.x & 31u;
    const T *in = static_cast<const T *>(sa.in);
    const uint64_t n = sa.n, n_blocks = sa.n_blocks, n_tiles = sa.n_tiles;
    const uint64_t payload_off = PC_HEADER_BYTES + table_bytes(n_blocks, D);
    const uint64_t blk0 = tile * sa.tb;
    const uint32_t nblk = (uint32_t)umin64(sa.tb, n_blocks - blk0);
    const uint64_t cnt = umin64(n - blk0 * L, (uint64_t)nblk * L);
    auto slot = [&](uint32_t b) -> T * { return reinterpret_cast<T *>(smem + (uint64_t)b * SB); };

    // 1. each warp stages its blocks (warp, warp + NW, ...): lane i issues the
    // bulk copy of the warp's i-th block once lane 0 has set the expected bytes
    {
        uint32_t bytes = 0;
        for (uint32_t b = warp + lane * NW; b < nblk; b += 32 * NW)
            bytes += ((uint32_t)umin64(L, cnt - (uint64_t)b * L) / VE) * 16u;
        bytes = __reduce_add_sync(0xFFFFFFFFu, bytes);
        fence_proxy_async_smem();
        if (lane == 0) mbar_arrive_expect_tx(&g_stage_bar[warp], bytes);
        __syncwarp();
        for (uint32_t b = warp + lane * NW; b < nblk; b += 32 * NW) {
            const uint32_t nb16 = ((uint32_t)umin64(L, cnt - (uint64_t)b * L) / VE) * 16u;
            if (nb16) bulk_copy_g2s(slot(b), in + (blk0 + b) * L, nb16, &g_stage_bar[warp]);
        }
    }
    const bool ragged = cnt % L != 0;  // the stream's last block is short (only that one can be)
    if (cnt % VE != 0 && (nblk - 1) % NW == warp) {
        const uint32_t b = nblk - 1;
        const uint32_t n_b = (uint32_t)(cnt - (uint64_t)b * L);
        for (uint32_t e = n_b / VE * VE + lane; e < n_b; e += 32) slot(b)[e] = in[(blk0 + b) * L + e];
    }
    stage_wait(warp, phase, ws, limit_ns);
    ++phase;
    __syncthreads();  // every block staged: any group may take any block

    // 2. min / max: G lanes per whole block, a 16-byte vector each
    {
        const uint32_t G = L / VE, gi = threadIdx.x & (G - 1);
        const uint32_t gmask = G == 32 ? 0xFFFFFFFFu : (((1u << G) - 1u) << (lane & ~(G - 1)));
        const uint32_t nfull = ragged ? nblk - 1 : nblk;
        for (uint32_t b = threadIdx.x / G; b < nfull; b += NT / G) {
            const uint4 x = reinterpret_cast<const uint4 *>(slot(b))[gi];
            uint32_t mn, mx;
            if constexpr (sizeof(T) == 2) {
                const uint32_t pmn = min_u16x2(min_u16x2(x.x, x.y), min_u16x2(x.z, x.w));
                const uint32_t pmx = max_u16x2(max_u16x2(x.x, x.y), max_u16x2(x.z, x.w));
                mn = min(pmn & 0xFFFFu, pmn >> 16);
                mx = max(pmx & 0xFFFFu, pmx >> 16);
            } else {
                mn = min(min(x.x, x.y), min(x.z, x.w));
                mx = max(max(x.x, x.y), max(x.z, x.w));
            }
            mn = __reduce_min_sync(gmask, mn);
            mx = __reduce_max_sync(gmask, mx);
            for (uint32_t i = gi; i < kPad; i += G) slot(b)[L + i] = (T)mn;
            if (gi == 0) {
                sv.vmin[b] = mn;
                sv.B[b] = (uint64_t)mx - mn + 1;
            }
        }
        if (ragged && warp == NW - 1) {
            const uint32_t b = nblk - 1;
            block_minmax<T>(slot(b), (uint32_t)(cnt - (uint64_t)b * L), &sv.vmin[b], &sv.B[b]);
        }
    }
    __syncthreads();

    // 3-4. word counts (a thread per block), CTA scan, look-back
    uint32_t W = 0;
    if (threadIdx.x < nblk) {
        const uint32_t b = threadIdx.x;
        const uint64_t B = sv.B[b];
        if (B > 1) {
            const uint32_t n_b = (uint32_t)umin64(L, cnt - (uint64_t)b * L);
            const uint32_t p = basic_p(B, WB);
            sv.p[b] = p;
            W = (n_b + p - 1) / p;
            sv.pk[b] = basic_pack_k(B, p, sv.vmin[b], WB);
        }
        sv.W[b] = W;
    }
    const uint32_t incl = warp_incl_scan_u32(W);
    if (lane == 31) sv.wtot[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        const uint32_t t = lane < NW ? sv.wtot[lane] : 0u;
        const uint32_t ti = warp_incl_scan_u32(t);
        const uint32_t agg = __shfl_sync(0xFFFFFFFFu, ti, 31);
        uint64_t excl = 0;
        bool ok = false;
        if (stage_dead()) {  // the staged samples are not whole: successors stop on this tile's error
            if (lane == 0) st_release(&sa.status[tile], kFlagError);
        } else {
            lookback_publish(sa.status, tile, agg);
            ok = lookback_complete(sa.status, tile, agg, ws, limit_ns, &excl);
        }
        __syncwarp();
        if (lane < NW) sv.wtot[lane] = ti - t;
        if (lane == 0) {
            sv.agg = agg;
            sv.excl = excl;
            sv.ok = ok ? 1u : 0u;
        }
    }
    __syncthreads();
    if (threadIdx.x < nblk) sv.woff[threadIdx.x] = sv.wtot[warp] + incl - W;
    __syncthreads();

    // 5. table entries, packed words, and the stream's closing bytes
    if (sv.ok) {
        for (uint32_t b = threadIdx.x; b < nblk; b += NT) {
            const uint64_t gb = blk0 + b;
            const uint64_t Bm1 = sv.B[b] - 1;
            if constexpr (D == 16) {
                reinterpret_cast<uint32_t *>(sa.out + PC_HEADER_BYTES)[gb] = sv.vmin[b] | ((uint32_t)Bm1 << 16);
            } else {
                reinterpret_cast<uint64_t *>(sa.out + PC_HEADER_BYTES)[gb] = (uint64_t)sv.vmin[b] | (Bm1 << 32);
            }
        }
        Word *payload = reinterpret_cast<Word *>(sa.out + payload_off);
        pack_basic_flat<T, WB, NT>(smem, SB, sv.woff, sv.p, sv.B, sv.pk, nblk, sv.agg, payload + sv.excl);
        if (tile == n_tiles - 1) {
            const uint64_t payload_words = sv.excl + sv.agg;
            const uint64_t tend = PC_HEADER_BYTES + n_blocks * 2u * (D / 8);
            for (uint64_t o = tend + threadIdx.x; o < payload_off; o += NT) sa.out[o] = 0;
            if (threadIdx.x == 0) {
                write_header<D, WB, PC_VARIANT_BASIC>(sa.out, L, n, n_blocks, payload_words);
                *sa.out_bytes = payload_off + payload_words * (WB / 8);
            }
        }
    }
    __syncthreads();  // the stage and the tile arrays are free again
}

template <typename T, uint32_t WB>
__global__ void __launch_bounds__(kShortThreads, 4) k_compress_short(StreamArgs sa, WsHeader *ws, uint64_t limit_ns)
{
    extern __shared__ __align__(16) uint8_t smem[];
    __shared__ uint32_t s_tile;
    stage_bars_init();
    uint32_t phase = 0;
    for (;;) {
        if (threadIdx.x == 0) s_tile = g_stage_dead ? 0xFFFFFFFFu : atomicAdd(&ws->ticket, 1u);
        __syncthreads();
        const uint64_t tile = s_tile;
        __syncthreads();
        if (tile >= sa.n_tiles) break;
        compress_tile_short<T, WB>(sa, tile, smem, ws, limit_ns, phase);
    }
}

#ifndef PCX_COMPRESS_MIN_CTAS_BASIC
#define PCX_COMPRESS_MIN_CTAS_BASIC 3
#endif
#ifndef PCX_COMPRESS_MIN_CTAS_ADVANCED
#define PCX_COMPRESS_MIN_CTAS_ADVANCED 3
#endif
// 128-thread CTAs (half-size tiles): twice as many per SM.
template <uint32_t VAR, uint32_t NT>
constexpr int kCompressMinCtas =
    (VAR == PC_VARIANT_BASIC ? PCX_COMPRESS_MIN_CTAS_BASIC : PCX_COMPRESS_MIN_CTAS_ADVANCED) * (NT <= 128 ? 2 : 1);

// MULTI: look-back tiles of several stage tiles (compress_tile_multi); FOUR:
// its stage tiles sized for four CTAs per SM (registers capped at 64).
template <typename T, uint32_t WB, uint32_t VAR, bool ORB, uint32_t NT, bool MULTI = false, bool FOUR = false>
__global__ void __launch_bounds__(NT, FOUR && VAR == PC_VARIANT_BASIC ? 4 : kCompressMinCtas<VAR, NT>)
k_compress(StreamArgs sa, WsHeader *ws, uint64_t limit_ns)
{
    extern __shared__ __align__(16) uint8_t smem[];
    __shared__ uint32_t s_tile;
    if (sa.n_tiles == 0) {
        if (blockIdx.x == 0 && threadIdx.x == 0) write_empty_stream<sizeof(T) * 8, WB, VAR>(sa);
        return;
    }
    stage_bars_init();
    uint32_t phase = 0;
    for (;;) {
        // a CTA whose staging died takes no further tile
        if (threadIdx.x == 0) s_tile = g_stage_dead ? 0xFFFFFFFFu : atomicAdd(&ws->ticket, 1u);
        __syncthreads();
        const uint64_t tile = s_tile;
        __syncthreads();
        if (tile >= sa.n_tiles) break;
        if constexpr (MULTI) compress_tile_multi<T, WB, NT, FOUR, VAR>(sa, tile, smem, ws, limit_ns, phase);
        else compress_tile<T, WB, VAR, ORB, NT>(sa, tile, smem, ws, limit_ns, phase);
    }
}

}  // namespace pcx
