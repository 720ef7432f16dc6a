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

// Eq. 2, word j of a block: s_j = sum_{i<p} u[j p + i] B^i with u = v - vmin.
// Evaluated by Horner from the highest digit on the raw samples v, modulo
// 2^w, minus K = vmin (1 + B + ... + B^(p-1)) mod 2^w: the difference is the
// true s_j, which is < 2^w.  Padding samples hold vmin, i.e. digit 0.
template <typename T, uint32_t WB, uint32_t P>
__device__ __forceinline__ typename WordOf<T, WB>::type horner_k(const T *dg, uint32_t B32)
{
    if constexpr (WB == 32) {
        uint32_t acc = dg[P - 1];
#pragma unroll
        for (int k = (int)P - 2; k >= 0; --k) acc = acc * B32 + (uint32_t)dg[k];
        return acc;
    } else {
        uint32_t lo = dg[P - 1], hi = 0;
#pragma unroll
        for (int k = (int)P - 2; k >= 0; --k) mad64(lo, hi, B32, (uint32_t)dg[k]);
        return ((uint64_t)hi << 32) | lo;
    }
}

template <typename T, uint32_t WB>
__device__ __forceinline__ typename WordOf<T, WB>::type
basic_word(const T *dg, uint32_t p, uint32_t B32, uint64_t K)
{
    using Word = typename WordOf<T, WB>::type;
    Word acc;
    switch (p) {
    case 1: acc = horner_k<T, WB, 1>(dg, B32); break;
    case 2: acc = horner_k<T, WB, 2>(dg, B32); break;
    case 3: acc = horner_k<T, WB, 3>(dg, B32); break;
    case 4: acc = horner_k<T, WB, 4>(dg, B32); break;
    case 5: acc = horner_k<T, WB, 5>(dg, B32); break;
    case 6: acc = horner_k<T, WB, 6>(dg, B32); break;
    case 7: acc = horner_k<T, WB, 7>(dg, B32); break;
    case 8: acc = horner_k<T, WB, 8>(dg, B32); break;
    case 9: acc = horner_k<T, WB, 9>(dg, B32); break;
    case 10: acc = horner_k<T, WB, 10>(dg, B32); break;
    case 11: acc = horner_k<T, WB, 11>(dg, B32); break;
    case 12: acc = horner_k<T, WB, 12>(dg, B32); break;
    default:
        if constexpr (WB == 32) {
            uint32_t a = dg[p - 1];
            for (int k = (int)p - 2; k >= 0; --k) a = a * B32 + (uint32_t)dg[k];
            acc = a;
        } else {
            uint32_t lo = dg[p - 1], hi = 0;
            for (int k = (int)p - 2; k >= 0; --k) mad64(lo, hi, B32, (uint32_t)dg[k]);
            acc = ((uint64_t)hi << 32) | lo;
        }
    }
    return acc - (Word)K;
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

// Basic words of one block by one warp, four words per lane in lockstep so
// that their Horner chains are independent for the scheduler.  Lanes past the
// last word recompute the last word and do not store it.
template <typename T, uint32_t WB>
__device__ __forceinline__ void pack_basic_block(const T *u, uint32_t W, uint32_t p, uint32_t B32, uint64_t K,
                                                 typename WordOf<T, WB>::type *dst)
{
    using Word = typename WordOf<T, WB>::type;
    const uint32_t lane = threadIdx.x & 31u;
    for (uint32_t j0 = 0; j0 < W; j0 += 128) {
        const T *g[4];
#pragma unroll
        for (uint32_t k = 0; k < 4; ++k) {
            const uint32_t j = min(j0 + lane + 32 * k, W - 1);
            g[k] = u + j * p;
        }
        Word acc[4];
        if constexpr (WB == 32) {
            uint32_t a[4];
#pragma unroll
            for (uint32_t k = 0; k < 4; ++k) a[k] = g[k][p - 1];
            for (int d = (int)p - 2; d >= 0; --d) {
#pragma unroll
                for (uint32_t k = 0; k < 4; ++k) a[k] = a[k] * B32 + (uint32_t)g[k][d];
            }
#pragma unroll
            for (uint32_t k = 0; k < 4; ++k) acc[k] = a[k] - (uint32_t)K;
        } else {
            uint32_t lo[4], hi[4];
#pragma unroll
            for (uint32_t k = 0; k < 4; ++k) {
                lo[k] = g[k][p - 1];
                hi[k] = 0;
            }
            for (int d = (int)p - 2; d >= 0; --d) {
#pragma unroll
                for (uint32_t k = 0; k < 4; ++k) mad64(lo[k], hi[k], B32, (uint32_t)g[k][d]);
            }
#pragma unroll
            for (uint32_t k = 0; k < 4; ++k) acc[k] = (((uint64_t)hi[k] << 32) | lo[k]) - K;
        }
#pragma unroll
        for (uint32_t k = 0; k < 4; ++k) {
            const uint32_t j = j0 + lane + 32 * k;
            if (j < W) dst[j] = acc[k];
        }
    }
}

template <typename T, uint32_t WB, uint32_t VAR, bool ORB>
__global__ void __launch_bounds__(kThreads)
k_compress(const T *__restrict__ in, uint64_t n, uint32_t L, uint8_t *__restrict__ out,
           uint64_t *__restrict__ out_bytes, WsHeader *ws, uint64_t *status,
           uint64_t n_blocks, uint64_t n_tiles, uint64_t limit_ns, OrbitTable ot)
{
    using Word = typename WordOf<T, WB>::type;
    constexpr uint32_t D = sizeof(T) * 8;
    extern __shared__ __align__(16) uint8_t smem[];
    const TileCfg cfg = tile_cfg(kKernelCompress, VAR, D, WB, L, ORB);
    const bool piped = cfg.slots == 2;
    const uint32_t warp = threadIdx.x >> 5, lane = threadIdx.x & 31u;
    const uint64_t payload_off = PC_HEADER_BYTES + table_bytes(n_blocks, D);

    auto slot = [&](uint32_t s) { return smem + (uint64_t)s * cfg.slot_bytes; };
    auto vars = [&](uint32_t s) -> BlockVars & {
        return *reinterpret_cast<BlockVars *>(slot(s) + cfg.off_blk);
    };
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

    // 1. take the next ticket into slot s and start loading its samples
    //    (asynchronously when two slots are in flight)
    auto acquire = [&](uint32_t s) {
        if (threadIdx.x == 0) vars(s).tile = atomicAdd(&ws->ticket, 1u);
        __syncthreads();
        const uint64_t t = vars(s).tile;
        if (t < n_tiles) {
            const uint64_t b0 = t * cfg.tb;
            const uint32_t nb = (uint32_t)umin64(cfg.tb, n_blocks - b0);
            const uint64_t c = umin64(n - b0 * L, (uint64_t)nb * L);
            if (piped) load_tile_async<T>(in, b0 * L, c, L, slot(s), cfg.stage_bytes);
            else load_tile<T>(in, b0 * L, c, L, slot(s), cfg.stage_bytes);
        }
        if (piped) cp_async_commit();
    };

    // 2-3. min / max per block, word counts, scan; the tile's aggregate is
    //      published as soon as it is known
    auto analyze = [&](uint32_t s) {
        BlockVars &bv = vars(s);
        uint8_t *stage = slot(s);
        uint64_t *sched_all = reinterpret_cast<uint64_t *>(stage + cfg.off_sched);
        const uint64_t tile = bv.tile;
        const uint64_t blk0 = tile * cfg.tb;
        const uint32_t nblk = (uint32_t)umin64(cfg.tb, n_blocks - blk0);
        const uint64_t cnt = umin64(n - blk0 * L, (uint64_t)nblk * L);
        for (uint32_t b = warp; b < nblk; b += kWarps) {
            const uint32_t n_b = (uint32_t)umin64(L, cnt - (uint64_t)b * L);
            block_minmax<T>(reinterpret_cast<T *>(stage + (uint64_t)b * cfg.stage_bytes), n_b, &bv.vmin[b],
                            &bv.B[b]);
        }
        __syncthreads();
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
                        uint64_t geo = 0, pw = 1;  // 1 + B + ... + B^(p-1), mod 2^64
                        for (uint32_t i = 0; i < p; ++i) {
                            geo += pw;
                            pw *= B;
                        }
                        bv.K[lane] = geo * bv.vmin[lane];
                    } else if (ORB && B <= kOrbitMaxB) {
                        // the series from the table: O(1) per word
                        const uint64_t h = orbit_get<WB>(ot, (uint32_t)B, ws, limit_ns);
                        if (h == ~0ull) {
                            W = 0;
                        } else {
                            const OrbitView v = orbit_view(ot, h);
                            W = orbit_words(ot, v, n_b);
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
            if (lane == 0) bv.agg = agg;
            lookback_publish(status, tile, agg);
        }
    };

    // 4-5. look-back to the tile's payload offset, table entries, packed words
    auto finish = [&](uint32_t s) {
        BlockVars &bv = vars(s);
        uint8_t *stage = slot(s);
        const uint64_t *sched_all = reinterpret_cast<const uint64_t *>(stage + cfg.off_sched);
        const uint64_t tile = bv.tile;
        const uint64_t blk0 = tile * cfg.tb;
        const uint32_t nblk = (uint32_t)umin64(cfg.tb, n_blocks - blk0);
        if (warp == 0) {
            uint64_t excl = 0;
            const bool ok = lookback_complete(status, tile, bv.agg, ws, limit_ns, &excl);
            if (lane == 0) {
                bv.excl = excl;
                bv.ok = ok ? 1u : 0u;
            }
        }
        __syncthreads();
        if (!bv.ok) return;
        for (uint32_t b = threadIdx.x; b < nblk; b += kThreads) {
            const uint64_t gb = blk0 + b;
            const uint64_t Bm1 = bv.B[b] - 1;
            if constexpr (D == 16) {
                reinterpret_cast<uint32_t *>(out + PC_HEADER_BYTES)[gb] = bv.vmin[b] | ((uint32_t)Bm1 << 16);
            } else {
                reinterpret_cast<uint64_t *>(out + PC_HEADER_BYTES)[gb] = (uint64_t)bv.vmin[b] | (Bm1 << 32);
            }
        }
        Word *payload = reinterpret_cast<Word *>(out + payload_off);
        for (uint32_t b = warp; b < nblk; b += kWarps) {
            const uint32_t W = bv.W[b];
            if (W == 0) continue;
            const T *u = reinterpret_cast<const T *>(stage + (uint64_t)b * cfg.stage_bytes);
            const uint32_t vmin = bv.vmin[b];
            const uint32_t B32 = (uint32_t)bv.B[b];  // B = 2^32 only with p = 1: never multiplies
            Word *dst = payload + bv.excl + bv.woff[b];
            if constexpr (VAR == PC_VARIANT_BASIC) {
                pack_basic_block<T, WB>(u, W, bv.p[b], B32, bv.K[b], dst);
            } else {
                if (ORB && bv.mode[b]) {
                    const OrbitView v{bv.orb_off[b], bv.orb_Q[b], bv.orb_P[b], bv.orb_SQ[b], bv.orb_G[b],
                                      Magic32{bv.orb_mgm[b], bv.orb_mga[b], bv.orb_mgs[b]}};
                    adv_words_orbit<T, WB>(ot, v, u, W, B32, vmin, bv.p1[b], bv.K[b], bv.K2[b], dst);
                } else {
                    const uint64_t *sched = sched_all + (uint64_t)b * cfg.wcap;
                    for (uint32_t j = lane; j < W; j += 32) dst[j] = adv_word<T, WB>(u, sched, j, B32, vmin);
                }
            }
        }
        if (tile == n_tiles - 1) {  // the last tile closes the stream
            const uint64_t payload_words = bv.excl + bv.agg;
            const uint64_t tend = PC_HEADER_BYTES + n_blocks * 2u * (D / 8);
            for (uint64_t o = tend + threadIdx.x; o < payload_off; o += kThreads) out[o] = 0;
            if (threadIdx.x == 0) write_header(payload_words);
        }
    };

    // Two slots: while one tile is finished, the next one's samples stream in;
    // each tile is analysed (and its aggregate published) as soon as its
    // samples have landed.  Tiles are finished in ticket order.
    acquire(0);
    if (piped) cp_async_wait<0>();
    __syncthreads();
    if (vars(0).tile < n_tiles) analyze(0);
    __syncthreads();
    if (piped) acquire(1);
    uint32_t c = 0;
    while (vars(c).tile < n_tiles) {
        finish(c);
        __syncthreads();
        if (piped) {
            cp_async_wait<0>();
            __syncthreads();
            if (vars(c ^ 1u).tile < n_tiles) analyze(c ^ 1u);
            __syncthreads();
            acquire(c);
            c ^= 1u;
        } else {
            acquire(0);
            __syncthreads();
            if (vars(0).tile < n_tiles) analyze(0);
            __syncthreads();
        }
    }
    if (piped) cp_async_wait<0>();
}

template <typename T, uint32_t WB, uint32_t VAR, bool ORB>
static cudaError_t launch_compress_t(const LaunchArgs &a)
{
    auto kern = k_compress<T, WB, VAR, ORB>;
    const TileCfg cfg = tile_cfg(kKernelCompress, VAR, sizeof(T) * 8, WB, a.L, ORB);
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
    OrbitTable ot{a.orb_flags, a.orb_hdr, static_cast<ulonglong2 *>(a.orb_slots), &a.ws->orbit_cursor};
    kern<<<(unsigned)grid, kThreads, cfg.smem, a.stream>>>(
        static_cast<const T *>(a.in), a.n, a.L, static_cast<uint8_t *>(a.out), a.out_count,
        a.ws, a.status, a.n_blocks, a.n_tiles, a.limit_ns, ot);
    return cudaGetLastError();
}

cudaError_t launch_compress(const LaunchArgs &a)
{
    const uint32_t key = (a.d == 32 ? 4u : 0u) | (a.w == 64 ? 2u : 0u) | (a.variant ? 1u : 0u);
    switch (key) {
    case 0: return launch_compress_t<uint16_t, 32, 0, false>(a);
    case 1: return a.orbit ? launch_compress_t<uint16_t, 32, 1, true>(a) : launch_compress_t<uint16_t, 32, 1, false>(a);
    case 2: return launch_compress_t<uint16_t, 64, 0, false>(a);
    case 3: return a.orbit ? launch_compress_t<uint16_t, 64, 1, true>(a) : launch_compress_t<uint16_t, 64, 1, false>(a);
    case 4: return launch_compress_t<uint32_t, 32, 0, false>(a);
    case 5: return a.orbit ? launch_compress_t<uint32_t, 32, 1, true>(a) : launch_compress_t<uint32_t, 32, 1, false>(a);
    case 6: return launch_compress_t<uint32_t, 64, 0, false>(a);
    default: return a.orbit ? launch_compress_t<uint32_t, 64, 1, true>(a) : launch_compress_t<uint32_t, 64, 1, false>(a);
    }
}

}  // namespace pcx
