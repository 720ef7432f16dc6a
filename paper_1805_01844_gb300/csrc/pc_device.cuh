// pc_device.cuh -- device building blocks of the sm_103a kernels:
// memory-ordering primitives, the bounded decoupled look-back over tiles
// (Merrill & Garland 2016, "Single-pass Parallel Prefix Scan with Decoupled
// Look-back"), tile staging, the per-block min/max reduction, and the
// split-base series of Sec. 3.2.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

#include "pc_common.cuh"

#ifndef PCX_MINMAX_PACKED
#define PCX_MINMAX_PACKED 0
#endif

namespace pcx {

__device__ __forceinline__ uint64_t ld_acquire(const uint64_t *p)
{
    uint64_t v;
    asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_release(uint64_t *p, uint64_t v)
{
    asm volatile("st.release.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

__device__ __forceinline__ uint64_t globaltimer()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Ampere-style asynchronous global -> shared copies (16-byte granules, L2
// only), grouped and awaited per thread; they let the next tile stream in
// while the current one is packed.
__device__ __forceinline__ void cp_async16(void *smem, const void *gmem)
{
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(s), "l"(gmem) : "memory");
}

// 4- or 8-byte asynchronous copy (a packed word), cached in L1 and L2.
template <uint32_t BYTES>
__device__ __forceinline__ void cp_async_small(void *smem, const void *gmem)
{
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], %2;" ::"r"(s), "l"(gmem), "n"(BYTES) : "memory");
}

// Store of one T (16 or 32 bits, the low bits of v) at a 32-bit shared address.
template <typename T>
__device__ __forceinline__ void st_shared(uint32_t a, uint32_t v);
template <>
__device__ __forceinline__ void st_shared<uint16_t>(uint32_t a, uint32_t v)
{
    asm volatile("st.shared.u16 [%0], %1;" ::"r"(a), "h"((unsigned short)v) : "memory");
}
template <>
__device__ __forceinline__ void st_shared<uint32_t>(uint32_t a, uint32_t v)
{
    asm volatile("st.shared.u32 [%0], %1;" ::"r"(a), "r"(v) : "memory");
}

// Bulk (TMA engine) copies global -> shared completing on an mbarrier.
__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count)
{
    const unsigned a = (unsigned)__cvta_generic_to_shared(bar);
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(a), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_init_fence()
{
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void fence_proxy_async_smem()
{
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes)
{
    const unsigned a = (unsigned)__cvta_generic_to_shared(bar);
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(a), "r"(bytes) : "memory");
}

// bytes: a multiple of 16; both addresses 16-byte aligned
__device__ __forceinline__ void bulk_copy_g2s(void *smem, const void *gmem, uint32_t bytes, uint64_t *bar)
{
    const unsigned d = (unsigned)__cvta_generic_to_shared(smem);
    const unsigned a = (unsigned)__cvta_generic_to_shared(bar);
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                 ::"r"(d), "l"(gmem), "r"(bytes), "r"(a) : "memory");
}

// The same with an L2 eviction-priority policy (createpolicy) for the lines
// it reads: evict_last for data read again soon, evict_first for data read
// for the last time.
__device__ __forceinline__ void bulk_copy_g2s_hint(void *smem, const void *gmem, uint32_t bytes, uint64_t *bar,
                                                   uint64_t policy)
{
    const unsigned d = (unsigned)__cvta_generic_to_shared(smem);
    const unsigned a = (unsigned)__cvta_generic_to_shared(bar);
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint [%0], [%1], %2, [%3], %4;"
        ::"r"(d), "l"(gmem), "r"(bytes), "r"(a), "l"(policy) : "memory");
}

__device__ __forceinline__ uint64_t l2_policy_evict_last()
{
    uint64_t p;
    asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
    return p;
}

__device__ __forceinline__ uint64_t l2_policy_evict_first()
{
    uint64_t p;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
    return p;
}

// Bounded wait for the mbarrier phase of the given parity; false if it gave up.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, uint64_t limit_ns)
{
    const unsigned a = (unsigned)__cvta_generic_to_shared(bar);
    const uint64_t t0 = globaltimer();
    for (uint32_t spins = 0;; ++spins) {
        uint32_t done;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
            : "=r"(done)
            : "r"(a), "r"(parity)
            : "memory");
        if (done) return true;
        if (spins > (1u << 22) || globaltimer() - t0 > limit_ns) return false;
    }
}

__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }

template <int N>
__device__ __forceinline__ void cp_async_wait()
{
    asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

__device__ __forceinline__ void record_error(WsHeader *ws, uint32_t code)
{
    atomicCAS(&ws->status, 0u, code);
}

__device__ __forceinline__ uint64_t warp_sum_u64(uint64_t v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xFFFFFFFFu, v, o);
    return v;
}

__device__ __forceinline__ uint32_t warp_incl_scan_u32(uint32_t v)
{
    const uint32_t lane = threadIdx.x & 31u;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t t = __shfl_up_sync(0xFFFFFFFFu, v, o);
        if (lane >= (uint32_t)o) v += t;
    }
    return v;
}

// Decoupled look-back, in two halves run by one full warp.  The first
// publishes this tile's aggregate (tile 0 publishes its inclusive prefix
// directly).  The second sums predecessors' aggregates 32 at a time until it
// meets an inclusive prefix, then publishes this tile's inclusive prefix.
// Every wait is bounded by `limit_ns` of %globaltimer and an iteration cap;
// when either runs out, or a predecessor published an error, the tile
// publishes an error (so successors stop waiting on it), records the reason
// and returns false.
__device__ __forceinline__ void lookback_publish(uint64_t *status, uint64_t tile, uint64_t agg)
{
    if ((threadIdx.x & 31u) == 0) st_release(&status[tile], (tile == 0 ? kFlagPrefix : kFlagAgg) | agg);
}

__device__ __noinline__ static bool lookback_complete(uint64_t *status, uint64_t tile, uint64_t agg,
                                                      WsHeader *ws, uint64_t limit_ns, uint64_t *excl_out)
{
    const uint32_t lane = threadIdx.x & 31u;
    if (tile == 0) {
        *excl_out = 0;
        return true;
    }
    uint64_t excl = 0;
    int64_t base = (int64_t)tile - 1;
    const uint64_t t0 = globaltimer();
    uint32_t spins = 0;
    for (;;) {
        const int64_t idx = base - (int64_t)lane;
        const uint64_t s = idx >= 0 ? ld_acquire(&status[idx]) : kFlagPrefix;
        const uint32_t flag = (uint32_t)(s >> 62);
        const uint32_t stopm = __ballot_sync(0xFFFFFFFFu, flag >= 2u);
        const uint32_t zerom = __ballot_sync(0xFFFFFFFFu, flag == 0u);
        const uint32_t first = stopm ? (uint32_t)(__ffs(stopm) - 1) : 31u;
        const uint32_t upto = first == 31u ? 0xFFFFFFFFu : ((2u << first) - 1u);
        if (zerom & upto) {
            int out = 0;
            if (lane == 0) out = (++spins > (1u << 24)) || (globaltimer() - t0 > limit_ns);
            out = __shfl_sync(0xFFFFFFFFu, out, 0);
            if (out) {
                if (lane == 0) {
                    st_release(&status[tile], kFlagError);
                    record_error(ws, PC_ERR_TIMEOUT);
                    atomicAdd(&ws->timeouts, 1u);
                }
                return false;
            }
            __nanosleep(64);
            continue;
        }
        const uint32_t errm = __ballot_sync(0xFFFFFFFFu, flag == 3u);
        if (errm & upto) {
            if (lane == 0) st_release(&status[tile], kFlagError);
            return false;
        }
        uint64_t v = lane <= first ? (s & kValueMask) : 0;
        excl += warp_sum_u64(v);
        if (stopm) break;
        base -= 32;
    }
    if (lane == 0) st_release(&status[tile], kFlagPrefix | (excl + agg));
    *excl_out = excl;
    return true;
}

// Both halves back to back.
__device__ __forceinline__ bool lookback_warp(uint64_t *status, uint64_t tile, uint64_t agg, WsHeader *ws,
                                              uint64_t limit_ns, uint64_t *excl_out)
{
    lookback_publish(status, tile, agg);
    return lookback_complete(status, tile, agg, ws, limit_ns, excl_out);
}

// Copy `cnt` samples starting at global element g0 into the tile stage:
// element e goes to slot (e / L) at offset (e % L).  16-byte vector copies
// when a block's bytes are a multiple of 16 (then every block starts 16-byte
// aligned in both spaces), element copies otherwise.
template <typename T, uint32_t NT = kThreads>
__device__ __forceinline__ void load_tile(const T *__restrict__ in, uint64_t g0, uint64_t cnt,
                                          uint32_t L, uint8_t *stage, uint32_t stage_bytes)
{
    if ((L * sizeof(T)) % 16 == 0) {
        constexpr uint32_t VE = 16 / sizeof(T);
        const uint32_t vpb = L / VE;  // vectors per block
        const uint64_t nvec = cnt / VE;
        const uint4 *src = reinterpret_cast<const uint4 *>(in + g0);
        uint32_t b = threadIdx.x / vpb, o = threadIdx.x - b * vpb;
        const uint32_t sb = NT / vpb, so = NT - sb * vpb;
        uint64_t v = threadIdx.x;
        // four loads in flight per thread before their shared-memory stores
        for (; v + 3 * NT < nvec; v += 4 * NT) {
            uint4 x[4];
            uint32_t bb[4], oo[4];
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                x[k] = __ldcs(src + v + k * NT);
                bb[k] = b;
                oo[k] = o;
                o += so;
                b += sb;
                if (o >= vpb) { o -= vpb; ++b; }
            }
#pragma unroll
            for (int k = 0; k < 4; ++k)
                *reinterpret_cast<uint4 *>(stage + (uint64_t)bb[k] * stage_bytes + oo[k] * 16u) = x[k];
        }
        for (; v < nvec; v += NT) {
            uint4 x = __ldcs(src + v);
            *reinterpret_cast<uint4 *>(stage + (uint64_t)b * stage_bytes + o * 16u) = x;
            o += so;
            b += sb;
            if (o >= vpb) { o -= vpb; ++b; }
        }
        for (uint64_t e = nvec * VE + threadIdx.x; e < cnt; e += NT) {
            uint32_t bi = (uint32_t)(e / L), oi = (uint32_t)(e - (uint64_t)bi * L);
            reinterpret_cast<T *>(stage + (uint64_t)bi * stage_bytes)[oi] = in[g0 + e];
        }
    } else {
        for (uint64_t e = threadIdx.x; e < cnt; e += NT) {
            uint32_t bi = (uint32_t)(e / L), oi = (uint32_t)(e - (uint64_t)bi * L);
            reinterpret_cast<T *>(stage + (uint64_t)bi * stage_bytes)[oi] = in[g0 + e];
        }
    }
}

// Inverse of load_tile: write the staged samples of the tile to global memory.
template <typename T>
__device__ __forceinline__ void store_tile(T *__restrict__ out, uint64_t g0, uint64_t cnt,
                                           uint32_t L, const uint8_t *stage, uint32_t stage_bytes)
{
    if ((L * sizeof(T)) % 16 == 0) {
        constexpr uint32_t VE = 16 / sizeof(T);
        const uint32_t vpb = L / VE;
        const uint64_t nvec = cnt / VE;
        uint4 *dst = reinterpret_cast<uint4 *>(out + g0);
        uint32_t b = threadIdx.x / vpb, o = threadIdx.x - b * vpb;
        const uint32_t sb = kThreads / vpb, so = kThreads - sb * vpb;
        for (uint64_t v = threadIdx.x; v < nvec; v += kThreads) {
            __stcs(dst + v, *reinterpret_cast<const uint4 *>(stage + (uint64_t)b * stage_bytes + o * 16u));
            o += so;
            b += sb;
            if (o >= vpb) { o -= vpb; ++b; }
        }
        for (uint64_t e = nvec * VE + threadIdx.x; e < cnt; e += kThreads) {
            uint32_t bi = (uint32_t)(e / L), oi = (uint32_t)(e - (uint64_t)bi * L);
            out[g0 + e] = reinterpret_cast<const T *>(stage + (uint64_t)bi * stage_bytes)[oi];
        }
    } else {
        for (uint64_t e = threadIdx.x; e < cnt; e += kThreads) {
            uint32_t bi = (uint32_t)(e / L), oi = (uint32_t)(e - (uint64_t)bi * L);
            out[g0 + e] = reinterpret_cast<const T *>(stage + (uint64_t)bi * stage_bytes)[oi];
        }
    }
}

// Two 16-bit lanes of a 32-bit register at once (sm_90 and later).
__device__ __forceinline__ uint32_t min_u16x2(uint32_t a, uint32_t b)
{
    uint32_t d;
    asm("min.u16x2 %0, %1, %2;" : "=r"(d) : "r"(a), "r"(b));
    return d;
}

__device__ __forceinline__ uint32_t max_u16x2(uint32_t a, uint32_t b)
{
    uint32_t d;
    asm("max.u16x2 %0, %1, %2;" : "=r"(d) : "r"(a), "r"(b));
    return d;
}

// Sec. 3.1: minimum and maximum of one staged block, by one warp, with
// 16-byte shared-memory reads, packed 16x2 min/max for uint16 samples and a
// redux.sync reduction across the warp.  Then the kPad padding samples after
// the block are set to the minimum (offset 0).  PACKED: uint16 pairs by the
// 16x2 min/max instructions (basic-variant kernels); otherwise the two halves
// of each 32-bit word are kept apart with plain 32-bit min/max.
template <typename T, bool PACKED = false>
__device__ __forceinline__ void block_minmax(T *blk, uint32_t n_b, uint32_t *vmin_out,
                                             uint64_t *B_out)
{
    const uint32_t lane = threadIdx.x & 31u;
    uint32_t mn = 0xFFFFFFFFu, mx = 0;
    constexpr uint32_t VE = 16 / sizeof(T);
    const uint32_t nvec = n_b / VE;
    const uint4 *v4 = reinterpret_cast<const uint4 *>(blk);
    if (sizeof(T) == 2 && PACKED) {
        uint32_t pmn = 0xFFFFFFFFu, pmx = 0;
        for (uint32_t i = lane; i < nvec; i += 32) {
            const uint4 x = v4[i];
            pmn = min_u16x2(pmn, min_u16x2(min_u16x2(x.x, x.y), min_u16x2(x.z, x.w)));
            pmx = max_u16x2(pmx, max_u16x2(max_u16x2(x.x, x.y), max_u16x2(x.z, x.w)));
        }
        mn = min(pmn & 0xFFFFu, pmn >> 16);
        mx = max(pmx & 0xFFFFu, pmx >> 16);
    } else if (sizeof(T) == 2) {
#if PCX_MINMAX_PACKED
        uint32_t pmn = 0xFFFFFFFFu, pmx = 0;
        for (uint32_t i = lane; i < nvec; i += 32) {
            uint4 x = v4[i];
            pmn = __vminu2(pmn, __vminu2(__vminu2(x.x, x.y), __vminu2(x.z, x.w)));
            pmx = __vmaxu2(pmx, __vmaxu2(__vmaxu2(x.x, x.y), __vmaxu2(x.z, x.w)));
        }
        mn = min(pmn & 0xFFFFu, pmn >> 16);
        mx = max(pmx & 0xFFFFu, pmx >> 16);
#else
        // the two halves of each 32-bit word kept apart: plain 32-bit min/max
        uint32_t lmn = 0xFFFFFFFFu, lmx = 0, hmn = 0xFFFFFFFFu, hmx = 0;
        for (uint32_t i = lane; i < nvec; i += 32) {
            const uint4 x = v4[i];
            lmn = min(min(lmn, min(x.x & 0xFFFFu, x.y & 0xFFFFu)), min(x.z & 0xFFFFu, x.w & 0xFFFFu));
            lmx = max(max(lmx, max(x.x & 0xFFFFu, x.y & 0xFFFFu)), max(x.z & 0xFFFFu, x.w & 0xFFFFu));
            hmn = min(min(hmn, min(x.x, x.y)), min(x.z, x.w));  // high halves order the words
            hmx = max(max(hmx, max(x.x, x.y)), max(x.z, x.w));
        }
        mn = min(lmn, hmn >> 16);
        mx = max(lmx, hmx >> 16);
#endif
    } else {
        for (uint32_t i = lane; i < nvec; i += 32) {
            uint4 x = v4[i];
            mn = min(mn, min(min(x.x, x.y), min(x.z, x.w)));
            mx = max(mx, max(max(x.x, x.y), max(x.z, x.w)));
        }
    }
    for (uint32_t i = nvec * VE + lane; i < n_b; i += 32) {
        uint32_t v = blk[i];
        mn = min(mn, v);
        mx = max(mx, v);
    }
    mn = __reduce_min_sync(0xFFFFFFFFu, mn);
    mx = __reduce_max_sync(0xFFFFFFFFu, mx);
    for (uint32_t i = lane; i < kPad; i += 32) blk[n_b + i] = (T)mn;
    if (lane == 0) {
        *vmin_out = mn;
        *B_out = (uint64_t)mx - mn + 1;
    }
}

// The split-base series of Sec. 3.2 for one block, walked by one thread:
//   p_i = max{p : R'_{i-1} B^p <= C},  R_i = floor(C / (R'_{i-1} B^p_i)),
//   R'_i = ceil(B / R_i),  R'_0 = 1,
// with q_i = elements before word i's whole digits (q_1 = 0,
// q_{i+1} = q_i + p_i + 1); the block ends with the first word whose split
// slot q_i + p_i lies past its end.  Since R'_{i-1} <= B, p_i is p_1 or
// p_1 - 1, decided by R'_{i-1} <= E1 = floor(C / B^p_1); then
// R_i = floor(E / R'_{i-1}) with E = E1 or E0 = floor(C / B^(p_1 - 1)).
// Entries are packed as R | p << 32 | q << 40 (R < 2^32, p < 64, q < 2^24).
// Returns the word count, or ~0u if it would exceed `cap` (not reachable for
// valid B; guards the shared-memory array).  With sched == nullptr the series
// is only counted.
template <uint32_t WB>
__device__ static uint32_t walk_series(uint64_t B, uint32_t n_b, uint64_t *sched, uint32_t cap)
{
    const uint64_t C = WB == 64 ? ~0ull : 0xFFFFFFFFull;
    const uint32_t p1 = eq1_p(B, WB);
    uint64_t E1, E0;
    if (p1 == 0) {  // B > C (B = 2^32, 32-bit words): p_i = 0 throughout
        E1 = 0;
        E0 = C;
    } else {
        uint64_t Bp = 1;
        for (uint32_t k = 0; k + 1 < p1; ++k) Bp *= B;  // B^(p1-1)
        E0 = C / Bp;
        E1 = E0 / B;  // floor(floor(C / B^(p1-1)) / B) = floor(C / B^p1)
    }
    uint64_t x = 1;  // R'_{i-1}
    uint32_t q = 0, i = 0;
    for (;;) {
        uint32_t p;
        uint64_t R;
        if (x <= E1) {
            p = p1;
            R = E1 / x;
        } else {
            p = p1 == 0 ? 0 : p1 - 1;
            R = E0 / x;
        }
        if (sched) {
            if (i >= cap) return ~0u;
            sched[i] = R | ((uint64_t)p << 32) | ((uint64_t)q << 40);
        }
        ++i;
        const uint32_t split = q + p;
        if (split >= n_b) break;
        q = split + 1;
        x = (B - 1) / R + 1;  // ceil(B / R)
    }
    return i;
}

}  // namespace pcx
