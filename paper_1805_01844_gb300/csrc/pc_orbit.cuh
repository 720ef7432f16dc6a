// pc_orbit.cuh -- the split-base series of Sec. 3.2 as a lookup table.
//
// The series R'_0 = 1, p_i = max{p : R'_{i-1} B^p <= C},
// R_i = floor(C / (R'_{i-1} B^p_i)), R'_i = ceil(B / R_i) depends on (B, w)
// only, and its state R'_{i-1} lives in [1, B], so the sequence of states is
// eventually periodic: a pre-period of Q steps, then a cycle of P steps.  For
// every base B <= 65536 that a call meets, one lane walks the series once,
// finds (Q, P) with Brent's cycle detection (Brent 1980, "An improved Monte
// Carlo factorization algorithm"), and publishes the Q + P steps, each with
// R_i, p_i, S_i = sum_{k<i} (p_k + 1) (the samples consumed before word i)
// and the magic reciprocal of R_i.  Word i of any block with that base is then
// found in O(1): step k = i (i < Q + P) or Q + (i - Q) mod P, with
// q_i = S_k + ((i - Q) div P) G where G = S_{Q+P} - S_Q.  Over all 16-bit
// bases the orbits hold about 0.7 million steps (about 11 per base on
// average, 511 at most), so the table is small and filled lazily, once per
// base per call, under a claim / publish protocol with bounded waits.
#pragma once

#include <cstdint>

#include "pc_device.cuh"

namespace pcx {

constexpr uint32_t kOrbitMaxB = 65536;       // bases served by the table
constexpr uint64_t kOrbitCap = 1ull << 20;   // step slots in the workspace (16 bytes each)
constexpr uint32_t kOrbitStepLimit = 16384;  // Brent steps before a base is given up

struct OrbitTable {
    uint32_t *flags;   // [kOrbitMaxB + 1]: 0 empty, 1 being built, 2 ready, 3 failed
    uint64_t *hdr;     // [kOrbitMaxB + 1]: first slot | Q << 32 | P << 48
    ulonglong2 *ent;   // [kOrbitCap]: x = R | p << 16 | S << 24 | magic.s << 48 | round-down << 53, y = magic.m
    uint32_t *cursor;  // next free slot
};

// Constants of the series for one base B in [2, 65536]: p_1 >= 1,
// E1 = floor(C / B^p_1) and E0 = floor(C / B^(p_1 - 1)); both < 2^32.
struct SeriesConst {
    uint32_t B, p1, E1, E0;
};

template <uint32_t WB>
__device__ __forceinline__ SeriesConst series_const(uint32_t B)
{
    const uint64_t C = WB == 64 ? ~0ull : 0xFFFFFFFFull;
    const uint32_t p1 = eq1_p(B, WB);
    uint64_t Bp = 1;
    for (uint32_t k = 0; k + 1 < p1; ++k) Bp *= B;
    const uint64_t E0 = C / Bp;  // < B^2 <= 2^32
    return SeriesConst{B, p1, (uint32_t)(E0 / B), (uint32_t)E0};
}

// One step of the series from state x = R'_{i-1} (x <= B): p_i is p_1 when
// x B^p_1 <= C, i.e. x <= E1, else p_1 - 1; R_i = floor(E / x).
__device__ __forceinline__ uint32_t series_step(const SeriesConst &c, uint32_t x, uint32_t &p, uint32_t &R)
{
    if (x <= c.E1) {
        p = c.p1;
        R = c.E1 / x;
    } else {
        p = c.p1 - 1;
        R = c.E0 / x;
    }
    return (c.B - 1) / R + 1;  // R'_i = ceil(B / R_i)
}

__device__ __forceinline__ uint32_t ld_acquire32(const uint32_t *p)
{
    uint32_t v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_release32(uint32_t *p, uint32_t v)
{
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Per-block view of an orbit.
struct OrbitView {
    uint32_t off, Q, P, SQ, G;
    Magic32 mgP;
};

__device__ __forceinline__ uint32_t orbit_S(const OrbitTable &ot, uint32_t slot)
{
    return (uint32_t)(__ldcg(&ot.ent[slot].x) >> 24) & 0xFFFFFFu;
}

// Words of a block of n_b samples: the smallest m >= 1 with q_m >= n_b + 1
// (q_m = samples consumed by m words), from the orbit's prefix sums.
__device__ __forceinline__ uint32_t orbit_words(const OrbitTable &ot, const OrbitView &v, uint32_t n_b)
{
    const uint32_t T = n_b + 1;
    uint32_t lo, hi, add = 0, base = 0;  // search m in [lo, hi] over S(base + m) + add
    if (T <= v.SQ + v.G) {
        lo = 1;
        hi = v.Q + v.P;
    } else {
        const uint32_t c = (T - v.SQ - 1) / v.G;
        add = c * v.G;
        base = c * v.P;  // m = Q + c P + r, r in [1, P]
        lo = v.Q + 1;
        hi = v.Q + v.P;
    }
    while (lo < hi) {
        const uint32_t mid = (lo + hi) >> 1;
        if (orbit_S(ot, v.off + mid) + add >= T) hi = mid;
        else lo = mid + 1;
    }
    return base + lo;
}

// Walk the series of B, find its pre-period Q and period P, reserve Q + P + 3
// slots and fill them: the Q + P steps, the total S_{Q+P}, the block view
// (S_Q, G and the magic reciprocal of P) and the word count of a full block
// of the requesting call's length L; publish the header.  ~0 on failure
// (recorded).
__device__ __noinline__ static uint64_t orbit_build(const OrbitTable &ot, const SeriesConst &c, uint32_t L,
                                                   WsHeader *ws)
{
    uint32_t p, R, steps = 1;
    // Brent: the cycle length P
    uint32_t power = 1, lam = 1, tort = 1, hare = series_step(c, 1, p, R);
    while (tort != hare) {
        if (power == lam) {
            tort = hare;
            power <<= 1;
            lam = 0;
        }
        hare = series_step(c, hare, p, R);
        ++lam;
        if (++steps > kOrbitStepLimit) goto fail;
    }
    {
        // the pre-period Q: two walkers P steps apart meet at the cycle's start
        tort = 1;
        hare = 1;
        for (uint32_t i = 0; i < lam; ++i) hare = series_step(c, hare, p, R);
        uint32_t mu = 0;
        while (tort != hare) {
            tort = series_step(c, tort, p, R);
            hare = series_step(c, hare, p, R);
            ++mu;
            if (++steps > kOrbitStepLimit) goto fail;
        }
        const uint32_t Q = mu, P = lam, n = Q + P + 3;
        const uint32_t off = atomicAdd(ot.cursor, n);
        if ((uint64_t)off + n > kOrbitCap) goto fail;
        uint32_t x = 1, S = 0, SQ = 0;
        for (uint32_t k = 0; k < Q + P; ++k) {
            if (k == Q) SQ = S;
            const uint32_t xn = series_step(c, x, p, R);
            const Magic32 mg = magic32(R);
            ulonglong2 e;
            e.x = (uint64_t)R | ((uint64_t)p << 16) | ((uint64_t)S << 24) | ((uint64_t)mg.s << 48) |
                  ((uint64_t)(mg.a != 0) << 53);
            e.y = mg.m;
            ot.ent[off + k] = e;
            S += p + 1;
            x = xn;
        }
        ulonglong2 last;
        last.x = (uint64_t)S << 24;
        last.y = 0;
        ot.ent[off + Q + P] = last;
        const Magic32 mgP = magic32(P);
        ulonglong2 view;
        view.x = (uint64_t)SQ | ((uint64_t)(S - SQ) << 24) | ((uint64_t)mgP.s << 48) | ((uint64_t)(mgP.a != 0) << 53);
        view.y = mgP.m;
        ot.ent[off + Q + P + 1] = view;
        // the cache: words of a full block of the requesting call's length
        OrbitView v;
        v.off = off;
        v.Q = Q;
        v.P = P;
        v.SQ = SQ;
        v.G = S - SQ;
        v.mgP = mgP;
        ot.ent[off + Q + P + 2] = ulonglong2{((unsigned long long)L << 32) | orbit_words(ot, v, L), 0ull};
        const uint64_t h = (uint64_t)off | ((uint64_t)Q << 32) | ((uint64_t)P << 48);
        ot.hdr[c.B] = h;
        st_release32(&ot.flags[c.B], 2u);  // orders the slots and the header before it
        return h;
    }
fail:
    st_release32(&ot.flags[c.B], 3u);
    record_error(ws, PC_ERR_UNSUPPORTED);
    return ~0ull;
}

// Header of the orbit of B (2 <= B <= 65536): built by the first lane that
// asks, waited for (bounded) by the others.  ~0 on failure (recorded).
template <uint32_t WB>
__device__ uint64_t orbit_get(const OrbitTable &ot, uint32_t B, uint32_t L, WsHeader *ws, uint64_t limit_ns)
{
    uint32_t f = ld_acquire32(&ot.flags[B]);
    if (f == 2u) return __ldcg(&ot.hdr[B]);
    if (f == 0u && atomicCAS(&ot.flags[B], 0u, 1u) == 0u) return orbit_build(ot, series_const<WB>(B), L, ws);
    const uint64_t t0 = globaltimer();
    uint32_t spins = 0;
    while ((f = ld_acquire32(&ot.flags[B])) == 1u || f == 0u) {
        if (++spins > (1u << 24) || globaltimer() - t0 > limit_ns) {
            record_error(ws, PC_ERR_TIMEOUT);
            atomicAdd(&ws->timeouts, 1u);
            return ~0ull;
        }
        __nanosleep(64);
    }
    if (f != 2u) return ~0ull;
    return __ldcg(&ot.hdr[B]);
}

// The view of a block: one 16-byte load of the slot after the orbit's steps.
__device__ __forceinline__ OrbitView orbit_view(const OrbitTable &ot, uint64_t h)
{
    OrbitView v;
    v.off = (uint32_t)h;
    v.Q = (uint32_t)(h >> 32) & 0xFFFFu;
    v.P = (uint32_t)(h >> 48);
    const ulonglong2 e = __ldcg(&ot.ent[v.off + v.Q + v.P + 1]);
    v.SQ = (uint32_t)e.x & 0xFFFFFFu;
    v.G = (uint32_t)(e.x >> 24) & 0xFFFFFFu;
    v.mgP.m = (uint32_t)e.y;
    v.mgP.s = (uint32_t)(e.x >> 48) & 31u;
    v.mgP.a = ((e.x >> 53) & 1u) ? v.mgP.m : 0u;
    return v;
}

// Words of a block of n_b samples in a stream of block length L: a full
// block (n_b = L) reads the orbit's cache, which the builder filled with
// L' << 32 | words of a full block of the block length L' of the call that
// built it; otherwise, or for another length, the prefix search.
__device__ __forceinline__ uint32_t orbit_words_cached(const OrbitTable &ot, const OrbitView &v, uint32_t n_b,
                                                       uint32_t L)
{
    if (n_b == L) {
        const unsigned long long c = __ldcg(&ot.ent[v.off + v.Q + v.P + 2].x);
        if ((uint32_t)(c >> 32) == L) return (uint32_t)c;
    }
    return orbit_words(ot, v, n_b);
}

// Series entry of word i: R_i, p_i, q_i and the magic reciprocal of R_i.
struct SeriesEntry {
    uint32_t R, p, q;
    Magic32 mgR;
};

__device__ __forceinline__ SeriesEntry orbit_entry(const OrbitTable &ot, const OrbitView &v, uint32_t i)
{
    uint32_t k = i, cyc = 0;
    if (i >= v.Q + v.P) {
        const uint32_t t = i - v.Q;
        cyc = magic_div(t, v.mgP);
        k = v.Q + t - cyc * v.P;
    }
    const ulonglong2 e = __ldcg(&ot.ent[v.off + k]);
    SeriesEntry s;
    s.R = (uint32_t)e.x & 0xFFFFu;
    s.p = (uint32_t)(e.x >> 16) & 0xFFu;
    s.q = ((uint32_t)(e.x >> 24) & 0xFFFFFFu) + cyc * v.G;
    s.mgR.m = (uint32_t)e.y;
    s.mgR.s = (uint32_t)(e.x >> 48) & 31u;
    s.mgR.a = ((e.x >> 53) & 1u) ? s.mgR.m : 0u;
    return s;
}

}  // namespace pcx
