// pc_decompress.cu -- the decompression kernels (sm_103a).
//
// Two launches on the caller's stream:
//   k_offsets  every CTA validates the stream header; one thread per block
//              turns its table entry (min, B) into a word count (basic: Eq. 1,
//              2; advanced: the split-base series of Sec. 3.2), and a block
//              scan plus the bounded decoupled look-back over tiles gives the
//              payload offset of each decoding tile;
//   k_decode   round-robin over decoding tiles with no look-back left: one
//              warp per block, lanes over words; polynomial division of each
//              word into its digits (Sec. 3.1) with per-block magic
//              reciprocals of B and of B^h (the largest power <= 2^32), so the
//              per-digit path has no division instruction, plus validity
//              checks of every word; coalesced 16-byte stores of the samples.
#include <cuda_runtime.h>

#include "pc_device.cuh"
#include "pc_kernels.h"
#include "pc_orbit.cuh"

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

// The same for D <= 2^31: the estimate's remainder s - q D lies in [0, 2 D),
// below 2^32, so it is formed and corrected in 32-bit arithmetic.
__device__ __forceinline__ uint64_t divmod_inv64_r32(uint64_t s, uint32_t D, uint64_t M, uint32_t &r)
{
    uint64_t q = __umul64hi(s, M);
    uint32_t rr = (uint32_t)s - (uint32_t)q * D;
    if (rr >= D) {
        ++q;
        rr -= D;
    }
    r = rr;
    return q;
}

// NK words split by D = B^h* (<= 2^32): hv = s div D, x = s mod D; one
// branch per call (D is the block's), then NK independent divisions.
template <uint32_t NK, typename W>
__device__ __forceinline__ void split_words(uint64_t (&hv)[NK], uint32_t (&x)[NK], const W (&s)[NK], uint64_t D,
                                            uint64_t M)
{
    if (D <= 0x80000000ull) {
#pragma unroll
        for (uint32_t k = 0; k < NK; ++k) {
            uint32_t lo;
            hv[k] = divmod_inv64_r32(s[k], (uint32_t)D, M, lo);
            x[k] = lo;
        }
    } else {
#pragma unroll
        for (uint32_t k = 0; k < NK; ++k) {
            uint64_t lo;
            hv[k] = divmod_inv64(s[k], D, M, lo);
            x[k] = (uint32_t)lo;
        }
    }
}

// Digits of x (< B^k), least significant first, into dst[0..k), plus vmin;
// returns the top digit (x div B^(k-1)), which is < B for a valid word.
// K digits fully unrolled; one indexed branch per call picks K.
template <typename T, uint32_t K>
__device__ __forceinline__ uint32_t put_digits_k(T *dst, uint32_t x, uint32_t B32, Magic32 mg, uint32_t vmin)
{
#pragma unroll
    for (uint32_t i = 0; i + 1 < K; ++i) {
        const uint32_t q = magic_div(x, mg);
        dst[i] = (T)(x - q * B32 + vmin);
        x = q;
    }
    dst[K - 1] = (T)(x + vmin);
    return x;
}

template <typename T>
__device__ __forceinline__ uint32_t put_digits(T *dst, uint32_t x, uint32_t k, uint32_t B32, Magic32 mg,
                                               uint32_t vmin)
{
    switch (k) {
    case 1: dst[0] = (T)(x + vmin); return x;
    case 2: return put_digits_k<T, 2>(dst, x, B32, mg, vmin);
    case 3: return put_digits_k<T, 3>(dst, x, B32, mg, vmin);
    case 4: return put_digits_k<T, 4>(dst, x, B32, mg, vmin);
    case 5: return put_digits_k<T, 5>(dst, x, B32, mg, vmin);
    case 6: return put_digits_k<T, 6>(dst, x, B32, mg, vmin);
    case 7: return put_digits_k<T, 7>(dst, x, B32, mg, vmin);
    case 8: return put_digits_k<T, 8>(dst, x, B32, mg, vmin);
    default:
        for (uint32_t i = 0; i + 1 < k; ++i) {
            const uint32_t q = magic_div(x, mg);
            dst[i] = (T)(x - q * B32 + vmin);
            x = q;
        }
        dst[k - 1] = (T)(x + vmin);
        return x;
    }
}

// Advanced words hold their first sample in the highest power, so digits
// come out last sample first.  rev_exact: x holds exactly k digits; written to
// last[0], last[-1], ..., last[-(k-1)] (k - 1 divisions, the top one is x).
// rev_quot: k divisions; the k digits are written the same way and the
// remaining quotient is returned.
#ifndef PCX_REV_EXACT_SPEC
#define PCX_REV_EXACT_SPEC 1
#endif

template <typename T, uint32_t K>
__device__ __forceinline__ void rev_exact_k(T *last, uint32_t x, uint32_t B32, Magic32 mg, uint32_t vmin)
{
#pragma unroll
    for (uint32_t i = 0; i + 1 < K; ++i) {
        const uint32_t q = magic_div(x, mg);
        *(last - i) = (T)(x - q * B32 + vmin);
        x = q;
    }
    *(last - (K - 1)) = (T)(x + vmin);
}

// (k is the same for every lane of the warp: one block's h*)
template <typename T>
__device__ __forceinline__ void rev_exact(T *last, uint32_t x, uint32_t k, uint32_t B32, Magic32 mg,
                                          uint32_t vmin)
{
#if PCX_REV_EXACT_SPEC
    switch (k) {
    case 2: rev_exact_k<T, 2>(last, x, B32, mg, vmin); return;
    case 3: rev_exact_k<T, 3>(last, x, B32, mg, vmin); return;
    case 4: rev_exact_k<T, 4>(last, x, B32, mg, vmin); return;
    case 5: rev_exact_k<T, 5>(last, x, B32, mg, vmin); return;
    case 6: rev_exact_k<T, 6>(last, x, B32, mg, vmin); return;
    default: break;
    }
#endif
    for (uint32_t i = 0; i + 1 < k; ++i) {
        const uint32_t q = magic_div(x, mg);
        *(last - i) = (T)(x - q * B32 + vmin);
        x = q;
    }
    *(last - (k - 1)) = (T)(x + vmin);
}

template <typename T, uint32_t K>
__device__ __forceinline__ uint32_t rev_quot_k(T *last, uint32_t x, uint32_t B32, Magic32 mg, uint32_t vmin)
{
#pragma unroll
    for (uint32_t i = 0; i < K; ++i) {
        const uint32_t q = magic_div(x, mg);
        *(last - i) = (T)(x - q * B32 + vmin);
        x = q;
    }
    return x;
}

template <typename T>
__device__ __forceinline__ uint32_t rev_quot(T *last, uint32_t x, uint32_t k, uint32_t B32, Magic32 mg,
                                             uint32_t vmin)
{
    switch (k) {
    case 0: return x;
    case 1: return rev_quot_k<T, 1>(last, x, B32, mg, vmin);
    case 2: return rev_quot_k<T, 2>(last, x, B32, mg, vmin);
    case 3: return rev_quot_k<T, 3>(last, x, B32, mg, vmin);
    case 4: return rev_quot_k<T, 4>(last, x, B32, mg, vmin);
    case 5: return rev_quot_k<T, 5>(last, x, B32, mg, vmin);
    case 6: return rev_quot_k<T, 6>(last, x, B32, mg, vmin);
    case 7: return rev_quot_k<T, 7>(last, x, B32, mg, vmin);
    case 8: return rev_quot_k<T, 8>(last, x, B32, mg, vmin);
    default:
        for (uint32_t i = 0; i < k; ++i) {
            const uint32_t q = magic_div(x, mg);
            *(last - i) = (T)(x - q * B32 + vmin);
            x = q;
        }
        return x;
    }
}

// Two advanced words of one lane in lockstep (independent division
// chains for the scheduler): rev_exact and rev_quot on (last0, x0) and
// (last1, x1) at once; k is the same for both (and for the whole warp).
template <typename T, uint32_t K>
__device__ __forceinline__ void rev_exact2_k(T *l0, uint32_t x0, T *l1, uint32_t x1, uint32_t B32, Magic32 mg,
                                             uint32_t vmin)
{
#pragma unroll
    for (uint32_t i = 0; i + 1 < K; ++i) {
        const uint32_t q0 = magic_div(x0, mg), q1 = magic_div(x1, mg);
        *(l0 - i) = (T)(x0 - q0 * B32 + vmin);
        *(l1 - i) = (T)(x1 - q1 * B32 + vmin);
        x0 = q0;
        x1 = q1;
    }
    *(l0 - (K - 1)) = (T)(x0 + vmin);
    *(l1 - (K - 1)) = (T)(x1 + vmin);
}

template <typename T>
__device__ __forceinline__ void rev_exact2(T *l0, uint32_t x0, T *l1, uint32_t x1, uint32_t k, uint32_t B32,
                                           Magic32 mg, uint32_t vmin)
{
    switch (k) {
    case 2: rev_exact2_k<T, 2>(l0, x0, l1, x1, B32, mg, vmin); return;
    case 3: rev_exact2_k<T, 3>(l0, x0, l1, x1, B32, mg, vmin); return;
    case 4: rev_exact2_k<T, 4>(l0, x0, l1, x1, B32, mg, vmin); return;
    case 5: rev_exact2_k<T, 5>(l0, x0, l1, x1, B32, mg, vmin); return;
    case 6: rev_exact2_k<T, 6>(l0, x0, l1, x1, B32, mg, vmin); return;
    default: break;
    }
    for (uint32_t i = 0; i + 1 < k; ++i) {
        const uint32_t q0 = magic_div(x0, mg), q1 = magic_div(x1, mg);
        *(l0 - i) = (T)(x0 - q0 * B32 + vmin);
        *(l1 - i) = (T)(x1 - q1 * B32 + vmin);
        x0 = q0;
        x1 = q1;
    }
    *(l0 - (k - 1)) = (T)(x0 + vmin);
    *(l1 - (k - 1)) = (T)(x1 + vmin);
}

template <typename T, uint32_t K>
__device__ __forceinline__ void rev_quot2_k(T *l0, uint32_t &x0, T *l1, uint32_t &x1, uint32_t B32, Magic32 mg,
                                            uint32_t vmin)
{
#pragma unroll
    for (uint32_t i = 0; i < K; ++i) {
        const uint32_t q0 = magic_div(x0, mg), q1 = magic_div(x1, mg);
        *(l0 - i) = (T)(x0 - q0 * B32 + vmin);
        *(l1 - i) = (T)(x1 - q1 * B32 + vmin);
        x0 = q0;
        x1 = q1;
    }
}

// k digits of each, the quotients left in x0 and x1.
template <typename T>
__device__ __forceinline__ void rev_quot2(T *l0, uint32_t &x0, T *l1, uint32_t &x1, uint32_t k, uint32_t B32,
                                          Magic32 mg, uint32_t vmin)
{
    switch (k) {
    case 0: return;
    case 1: rev_quot2_k<T, 1>(l0, x0, l1, x1, B32, mg, vmin); return;
    case 2: rev_quot2_k<T, 2>(l0, x0, l1, x1, B32, mg, vmin); return;
    case 3: rev_quot2_k<T, 3>(l0, x0, l1, x1, B32, mg, vmin); return;
    case 4: rev_quot2_k<T, 4>(l0, x0, l1, x1, B32, mg, vmin); return;
    case 5: rev_quot2_k<T, 5>(l0, x0, l1, x1, B32, mg, vmin); return;
    default: break;
    }
    for (uint32_t i = 0; i < k; ++i) {
        const uint32_t q0 = magic_div(x0, mg), q1 = magic_div(x1, mg);
        *(l0 - i) = (T)(x0 - q0 * B32 + vmin);
        *(l1 - i) = (T)(x1 - q1 * B32 + vmin);
        x0 = q0;
        x1 = q1;
    }
}

// s = body R + r for R < 2^16 by long division with R's magic reciprocal:
// the high 32-bit word first (any 32-bit dividend), then two 16-bit steps
// whose partial dividends r 2^16 + 16 bits stay below R 2^16 <= 2^32.
__device__ __forceinline__ uint64_t divmod_small64(uint64_t s, uint32_t R, Magic32 mg, uint32_t &r)
{
    const uint32_t s1 = (uint32_t)(s >> 32), s0 = (uint32_t)s;
    const uint32_t q1 = magic_div(s1, mg);
    uint32_t rr = s1 - q1 * R;
    uint32_t x = (rr << 16) | (s0 >> 16);
    const uint32_t q2 = magic_div(x, mg);
    rr = x - q2 * R;
    x = (rr << 16) | (s0 & 0xFFFFu);
    const uint32_t q3 = magic_div(x, mg);
    r = x - q3 * R;
    return ((uint64_t)q1 << 32) + ((uint64_t)q2 << 16) + q3;
}

// Header of a stream, validated by every CTA of the offsets kernel against
// the expected parameters, the buffer size, the output capacity and the
// workspace.  Returns a pc_status.
template <typename T, uint32_t WB, uint32_t VAR>
__device__ uint32_t check_header(const uint8_t *in, uint64_t in_bytes, uint32_t L, uint64_t cap,
                                 uint64_t status_cap, uint64_t offsets_cap, uint32_t dtb,
                                 uint64_t &n, uint64_t &nb, uint64_t &pw)
{
    constexpr uint32_t D = sizeof(T) * 8, DB = D / 8, WBY = WB / 8;
    const uint32_t *h = reinterpret_cast<const uint32_t *>(in);
    const uint64_t *h64 = reinterpret_cast<const uint64_t *>(in);
    n = h64[2];
    nb = h64[3];
    pw = h64[4];
    if (h[0] != 0x504D4350u || h[1] != (1u | (VAR << 16) | (D << 24)) || h[2] != WB || h[3] != L ||
        h64[5] != 0 || h64[6] != 0 || h64[7] != 0)
        return PC_ERR_CORRUPT;
    if (nb != n / L + (n % L != 0)) return PC_ERR_CORRUPT;
    if (n > cap) return PC_ERR_CAPACITY;
    if (nb > (in_bytes - PC_HEADER_BYTES) / (2 * DB)) return PC_ERR_CORRUPT;
    const uint64_t poff = PC_HEADER_BYTES + table_bytes(nb, D);
    if (poff > in_bytes || pw > (in_bytes - poff) / WBY) return PC_ERR_CORRUPT;
    if (ceil_div(nb, kOffsetTileBlocks) > status_cap || ceil_div(nb, dtb) + 1 > offsets_cap)
        return PC_ERR_INVALID_ARG;
    return PC_OK;
}

// Word count of a block from its table entry (basic: Eq. 1-2; advanced: the
// length of the split-base series of Sec. 3.2).
template <uint32_t WB, uint32_t VAR, bool ORB>
__device__ __forceinline__ uint32_t block_words(uint64_t B, uint32_t n_b, uint32_t L, const OrbitTable &ot,
                                                WsHeader *ws, uint64_t limit_ns)
{
    if (B <= 1) return 0;
    if constexpr (VAR == PC_VARIANT_BASIC) {
        const uint32_t p = basic_p(B, WB);
        return (n_b + p - 1) / p;
    } else {
        if (ORB && B <= kOrbitMaxB) {
            const uint64_t h = orbit_get<WB>(ot, (uint32_t)B, L, ws, limit_ns);
            if (h == ~0ull) return 0;
            return orbit_words_cached(ot, orbit_view(ot, h), n_b, L);
        }
        return walk_series<WB>(B, n_b, nullptr, 0);
    }
}

// Offsets kernel: one thread per block reads its table entry and word count;
// a block-wide scan and the bounded decoupled look-back over tiles of
// kOffsetTileBlocks blocks give every block's payload offset, of which the
// first block of each decoding tile is stored (plus the total).
template <typename T, uint32_t WB, uint32_t VAR, bool ORB>
__global__ void __launch_bounds__(kThreads)
k_offsets(const uint8_t *__restrict__ in, uint64_t in_bytes, uint32_t L, uint64_t cap,
          uint64_t *__restrict__ n_out, WsHeader *ws, uint64_t *status, uint64_t status_cap,
          uint64_t *offsets, uint64_t offsets_cap, uint32_t dtb, uint64_t limit_ns, OrbitTable ot)
{
    constexpr uint32_t D = sizeof(T) * 8, DB = D / 8;
    constexpr uint64_t kDmax = D == 16 ? 0xFFFFull : 0xFFFFFFFFull;
    __shared__ uint64_t hdr[4];
    __shared__ uint32_t warp_tot[kWarps];
    __shared__ uint64_t s_excl;
    __shared__ uint32_t s_tile, s_ok;
    const uint32_t warp = threadIdx.x >> 5, lane = threadIdx.x & 31u;

    if (threadIdx.x == 0) {
        uint64_t n, nb, pw;
        const uint32_t code = check_header<T, WB, VAR>(in, in_bytes, L, cap, status_cap, offsets_cap, dtb,
                                                       n, nb, pw);
        hdr[0] = n;
        hdr[1] = nb;
        hdr[2] = pw;
        hdr[3] = code;
    }
    __syncthreads();
    if (hdr[3] != PC_OK) {
        if (blockIdx.x == 0 && threadIdx.x == 0) record_error(ws, (uint32_t)hdr[3]);
        return;
    }
    const uint64_t n = hdr[0], n_blocks = hdr[1], payload_words = hdr[2];
    const uint64_t n_tiles = ceil_div(n_blocks, kOffsetTileBlocks);
    const uint64_t n_dtiles = ceil_div(n_blocks, dtb);
    const uint64_t payload_off = PC_HEADER_BYTES + table_bytes(n_blocks, D);
    if (n_tiles == 0) {
        if (blockIdx.x == 0 && threadIdx.x == 0) {
            if (payload_words != 0) record_error(ws, PC_ERR_CORRUPT);
            offsets[0] = 0;
            *n_out = 0;
        }
        return;
    }

    for (;;) {
        if (threadIdx.x == 0) s_tile = atomicAdd(&ws->ticket, 1u);
        __syncthreads();
        const uint64_t tile = s_tile;
        if (tile >= n_tiles) break;
        const uint64_t b = tile * kOffsetTileBlocks + threadIdx.x;
        uint32_t W = 0;
        if (b < n_blocks) {
            uint64_t vmin, Bm1;
            if constexpr (D == 16) {
                const uint32_t e = reinterpret_cast<const uint32_t *>(in + PC_HEADER_BYTES)[b];
                vmin = e & 0xFFFFu;
                Bm1 = e >> 16;
            } else {
                const uint64_t e = reinterpret_cast<const uint64_t *>(in + PC_HEADER_BYTES)[b];
                vmin = e & 0xFFFFFFFFull;
                Bm1 = e >> 32;
            }
            if (vmin + Bm1 > kDmax) {
                record_error(ws, PC_ERR_CORRUPT);
                Bm1 = 0;
            }
            const uint32_t n_b = (uint32_t)umin64(L, n - b * L);
            W = block_words<WB, VAR, ORB>(Bm1 + 1, n_b, L, ot, ws, limit_ns);
        }
        // block-wide exclusive scan of W
        const uint32_t incl = warp_incl_scan_u32(W);
        if (lane == 31) warp_tot[warp] = incl;
        __syncthreads();
        if (warp == 0) {
            const uint32_t t = lane < kWarps ? warp_tot[lane] : 0u;
            const uint32_t ti = warp_incl_scan_u32(t);
            if (lane < kWarps) warp_tot[lane] = ti - t;
            const uint32_t agg = __shfl_sync(0xFFFFFFFFu, ti, 31);
            uint64_t excl = 0;
            const bool ok = lookback_warp(status, tile, agg, ws, limit_ns, &excl);
            if (lane == 0) {
                s_excl = excl;
                s_ok = ok ? 1u : 0u;
            }
        }
        __syncthreads();
        if (s_ok && b < n_blocks) {
            const uint64_t off = s_excl + warp_tot[warp] + (incl - W);
            if (b % dtb == 0) offsets[b / dtb] = off;
            if (b == n_blocks - 1) {
                const uint64_t total = off + W;
                offsets[n_dtiles] = total;
                if (total != payload_words) record_error(ws, PC_ERR_CORRUPT);
                for (uint64_t o = PC_HEADER_BYTES + n_blocks * 2 * DB; o < payload_off; ++o)
                    if (in[o] != 0) record_error(ws, PC_ERR_CORRUPT);
            }
        }
        __syncthreads();
    }
}

// Decoding kernel: no look-back left.  Tiles are taken round-robin; per tile
// the table gives (min, B, W) per block, the offsets kernel the payload
// offset; one warp per block loads its words four per lane at a time and
// splits them into digits in shared memory; the tile's samples then leave in
// coalesced 16-byte streaming stores.
template <typename T, uint32_t WB, uint32_t VAR, bool ORB>
__global__ void __launch_bounds__(kThreads, 3)
k_decode(const uint8_t *__restrict__ in, uint32_t L, T *__restrict__ out, uint64_t *__restrict__ n_out,
         WsHeader *ws, const uint64_t *__restrict__ offsets, OrbitTable ot, uint64_t limit_ns)
{
    using Word = typename WordT<T, WB>::type;
    constexpr uint32_t D = sizeof(T) * 8;
    constexpr uint32_t KB = 4;  // words per lane in flight
    extern __shared__ __align__(16) uint8_t smem[];
    const TileCfg cfg = tile_cfg(kKernelDecode, VAR, D, WB, L, ORB);
    BlockVars &bv = *reinterpret_cast<BlockVars *>(smem + cfg.off_blk);
    uint64_t *sched_all = reinterpret_cast<uint64_t *>(smem + cfg.off_sched);
    uint32_t *tops_all = reinterpret_cast<uint32_t *>(smem + cfg.off_tops);
    const uint32_t warp = threadIdx.x >> 5, lane = threadIdx.x & 31u;

    if (*reinterpret_cast<volatile uint32_t *>(&ws->status) != PC_OK) return;  // the offsets kernel rejected the stream
    const uint64_t *h64 = reinterpret_cast<const uint64_t *>(in);
    const uint64_t n = h64[2], n_blocks = h64[3];
    const uint64_t n_tiles = ceil_div(n_blocks, cfg.tb);
    const uint64_t payload_off = PC_HEADER_BYTES + table_bytes(n_blocks, D);
    const Word *payload = reinterpret_cast<const Word *>(in + payload_off);

    for (uint64_t tile = blockIdx.x; tile < n_tiles; tile += gridDim.x) {
        const uint64_t blk0 = tile * cfg.tb;
        const uint32_t nblk = (uint32_t)umin64(cfg.tb, n_blocks - blk0);
        const uint64_t g0 = blk0 * L;
        const uint64_t cnt = umin64(n - g0, (uint64_t)nblk * L);
        if (threadIdx.x == 0) bv.bad = 0;
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
                const uint64_t B = Bm1 + 1;  // entries were range-checked by the offsets kernel
                const uint32_t n_b = (uint32_t)umin64(L, cnt - (uint64_t)lane * L);
                if (B > 1) {
                    // division constants of this block, computed once by its lane
                    const Magic32 mg = magic32(B);
                    bv.mg_m[lane] = mg.m;
                    bv.mg_a[lane] = mg.a;
                    bv.mg_s[lane] = mg.s;
                    uint32_t hs = 1;
                    uint64_t Dh = B;
                    while (Dh <= (1ull << 32) / B) {
                        Dh *= B;
                        ++hs;
                    }
                    bv.hstar[lane] = hs;
                    bv.dec.Dh[lane] = Dh;
                    bv.dec.MD[lane] = ~0ull / Dh;
                    if constexpr (VAR == PC_VARIANT_BASIC) {
                        const uint32_t p = basic_p(B, WB);
                        bv.p[lane] = p;
                        W = (n_b + p - 1) / p;
                    } else if (ORB && B <= kOrbitMaxB) {
                        const uint64_t h = orbit_get<WB>(ot, (uint32_t)B, L, ws, limit_ns);
                        if (h != ~0ull) {
                            const OrbitView v = orbit_view(ot, h);
                            W = orbit_words_cached(ot, v, n_b, L);
                            bv.orb_off[lane] = v.off;
                            bv.orb_Q[lane] = v.Q;
                            bv.orb_P[lane] = v.P;
                            bv.orb_SQ[lane] = v.SQ;
                            bv.orb_G[lane] = v.G;
                            bv.orb_mgm[lane] = v.mgP.m;
                            bv.orb_mga[lane] = v.mgP.a;
                            bv.orb_mgs[lane] = v.mgP.s;
                        }
                        bv.mode[lane] = 1;
                    } else {
                        W = walk_series<WB>(B, n_b, sched_all + (uint64_t)lane * cfg.wcap, cfg.wcap);
                        if (W == ~0u) W = 0;  // not reachable: B was range-checked
                        bv.mode[lane] = 0;
                    }
                }
                bv.vmin[lane] = (uint32_t)vmin;
                bv.B[lane] = B;
                bv.W[lane] = W;
            }
            const uint32_t incl = warp_incl_scan_u32(W);
            if (lane < nblk) bv.woff[lane] = incl - W;
            if (lane == 0) bv.excl = offsets[tile];
        }
        __syncthreads();

        // decode, one warp per block
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
                const Magic32 mg{bv.mg_m[b], bv.mg_a[b], bv.mg_s[b]};
                const uint32_t hstar = bv.hstar[b];
                const uint64_t Dh = bv.dec.Dh[b], MD = bv.dec.MD[b];
                // a full word is valid iff its top digit is < B; the last word's
                // digits past the block (written to the padding) must be 0
                for (uint32_t j0 = 0; j0 < W; j0 += 32 * KB) {
                    Word sv[KB];
#pragma unroll
                    for (uint32_t k = 0; k < KB; ++k) {
                        const uint32_t j = j0 + lane + 32 * k;
                        sv[k] = j < W ? __ldcs(src + j) : Word(0);
                    }
#pragma unroll
                    for (uint32_t k = 0; k < KB; ++k) {
                        const uint32_t j = j0 + lane + 32 * k;
                        if (j >= W) break;
                        const uint64_t s = sv[k];
                        T *dst = u + j * p;
                        uint32_t top;
                        if (WB == 32 || p <= hstar) {
                            top = put_digits<T>(dst, (uint32_t)s, p, B32, mg, vmin);
                            if (WB == 64) bad |= (s >> 32) != 0;
                        } else {
                            uint64_t lo;
                            uint64_t qv = divmod_inv64(s, Dh, MD, lo);
                            put_digits<T>(dst, (uint32_t)lo, hstar, B32, mg, vmin);
                            uint32_t rem = p - hstar;
                            if (rem > hstar) {  // p = 2 h* + 1: one more piece of h* digits
                                qv = divmod_inv64(qv, Dh, MD, lo);
                                put_digits<T>(dst + hstar, (uint32_t)lo, hstar, B32, mg, vmin);
                                dst += hstar;
                                rem -= hstar;
                            }
                            bad |= (qv >> 32) != 0;
                            top = put_digits<T>(dst + hstar, (uint32_t)qv, rem, B32, mg, vmin);
                        }
                        bad |= top >= B;
                    }
                }
                // padding digits of the last word must be zero
                if (lane == 0) {
                    const uint32_t end = W * p;
                    for (uint32_t i = n_b; i < end; ++i) bad |= (uint32_t)u[i] != vmin;
                }
            } else if (ORB && bv.mode[b]) {
                // one pass, lanes over consecutive words: word i yields its p_i
                // whole samples, its low part r_i and the high part r'_{i-1}
                // that, with r_{i-1} from the lane before, re-joins sample q_i - 1
                const OrbitView v{bv.orb_off[b], bv.orb_Q[b], bv.orb_P[b], bv.orb_SQ[b], bv.orb_G[b],
                                  Magic32{bv.orb_mgm[b], bv.orb_mga[b], bv.orb_mgs[b]}};
                const Magic32 mg{bv.mg_m[b], bv.mg_a[b], bv.mg_s[b]};
                const uint32_t hstar = bv.hstar[b];
                const uint64_t Dh = bv.dec.Dh[b], MD = bv.dec.MD[b];
                uint32_t cR = 1, cr = 0;  // carry: R and r of the word before this chunk
                uint32_t qlast = 0, plast = 0;
                for (uint32_t j0 = 0; j0 < W; j0 += 32) {
                    const uint32_t i = j0 + lane;
                    const bool valid = i < W;
                    SeriesEntry e;
                    uint64_t s = 0;
                    if (valid) {
                        e = orbit_entry(ot, v, i);
                        s = __ldcs(src + i);
                    } else {
                        e = SeriesEntry{1u, 0u, 0u, Magic32{0xFFFFFFFFu, 0xFFFFFFFFu, 0u}};
                    }
                    uint32_t r = 0;
                    uint64_t body = 0;
                    if (valid) {
                        if constexpr (WB == 32) {
                            const uint32_t q32 = magic_div((uint32_t)s, e.mgR);
                            r = (uint32_t)s - q32 * e.R;
                            body = q32;
                        } else {
                            body = divmod_small64(s, e.R, e.mgR, r);
                        }
                    }
                    uint32_t Rp = __shfl_up_sync(0xFFFFFFFFu, e.R, 1);
                    uint32_t rp = __shfl_up_sync(0xFFFFFFFFu, r, 1);
                    if (lane == 0) {
                        Rp = cR;
                        rp = cr;
                    }
                    cR = __shfl_sync(0xFFFFFFFFu, e.R, 31);
                    cr = __shfl_sync(0xFFFFFFFFu, r, 31);
                    if (!valid) continue;
                    // p_i whole digits, last sample first, then the high part
                    T *last = u + e.q + e.p - 1;
                    uint32_t rem = e.p;
                    while (rem >= hstar && (body >> 32) != 0) {
                        uint64_t lo;
                        body = divmod_inv64(body, Dh, MD, lo);
                        rev_exact<T>(last, (uint32_t)lo, hstar, B32, mg, vmin);
                        last -= hstar;
                        rem -= hstar;
                    }
                    bad |= (body >> 32) != 0;
                    const uint32_t top = rev_quot<T>(last, (uint32_t)body, rem, B32, mg, vmin);
                    if (i == 0) {
                        bad |= top != 0;
                    } else {
                        const uint64_t val = (uint64_t)top * Rp + rp;
                        bad |= val >= B;
                        u[e.q - 1] = (T)(val + vmin);
                    }
                    if (e.q + e.p >= n_b) bad |= r != 0;  // the split slot is padding
                    if (i == W - 1) {
                        qlast = e.q;
                        plast = e.p;
                    }
                }
                // whole digits past the block (padding) must be zero
                const uint32_t src_lane = (W - 1) & 31u;
                qlast = __shfl_sync(0xFFFFFFFFu, qlast, src_lane);
                plast = __shfl_sync(0xFFFFFFFFu, plast, src_lane);
                if (lane == 0)
                    for (uint32_t i = n_b; i < qlast + plast; ++i) bad |= (uint32_t)u[i] != vmin;
            } else {
                const uint64_t *sched = sched_all + (uint64_t)b * cfg.wcap;
                uint32_t *tops = tops_all + (uint64_t)b * cfg.wcap;
                const uint64_t MB = ~0ull / B;
                // phase A: digits, low parts r_i into the split slots, high parts aside
                for (uint32_t j0 = 0; j0 < W; j0 += 32 * KB) {
                    Word sv[KB];
#pragma unroll
                    for (uint32_t k = 0; k < KB; ++k) {
                        const uint32_t j = j0 + lane + 32 * k;
                        sv[k] = j < W ? __ldcs(src + j) : Word(0);
                    }
#pragma unroll
                    for (uint32_t k = 0; k < KB; ++k) {
                        const uint32_t i = j0 + lane + 32 * k;
                        if (i >= W) break;
                        const uint64_t e = sched[i];
                        const uint32_t R = (uint32_t)e;
                        const uint32_t p = (uint32_t)(e >> 32) & 0xFFu;
                        const uint32_t q = (uint32_t)(e >> 40);
                        const uint64_t s = sv[k];
                        uint64_t body = s / R;
                        const uint32_t r = (uint32_t)(s - body * R);
                        for (uint32_t kk = p; kk > 0; --kk) {
                            uint64_t dgt;
                            body = divmod_inv64(body, B, MB, dgt);
                            const uint32_t idx = q + kk - 1;
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
        store_tile<T>(out, g0, cnt, L, smem, cfg.stage_bytes);
        if (tile == n_tiles - 1 && threadIdx.x == 0) *n_out = n;
        __syncthreads();
    }
}

// Basic words j0 + lane + 32 k (k < NK) of one block, NK words per lane in
// lockstep (NK independent division chains).  Digits land at u[j p + i]
// (u at shared address ua; each lane walks its digits with a 32-bit shared
// address); lanes past the last word write theirs to the junk slots at
// junka.  Returns true if a word is not the image of valid digits.
template <typename T, uint32_t WB, uint32_t NK, bool FULL = false>
__device__ __forceinline__ bool decode_basic_group(const typename WordT<T, WB>::type *src /* shared */,
                                                   uint32_t src0, uint32_t ua, uint32_t junka, uint32_t j0, uint32_t W,
                                                   uint32_t p, uint32_t hstar, uint64_t B, uint32_t vmin, Magic32 mg,
                                                   uint64_t Dh, uint64_t MD)
{
    using Word = typename WordT<T, WB>::type;
    constexpr uint32_t E = sizeof(T);
    const uint32_t lane = threadIdx.x & 31u;
    const uint32_t B32 = (uint32_t)B;
    bool bad = false;
    Word sv[NK];
    uint32_t d[NK];  // shared address of the lane's next digit
    bool ok[NK];
#pragma unroll
    for (uint32_t k = 0; k < NK; ++k) {
        const uint32_t j = j0 + lane + 32 * k;
        ok[k] = FULL || j < W;  // a full group: every lane's words exist
        sv[k] = ok[k] ? src[j - src0] : Word(0);  // src: the staged words from word src0 on
        d[k] = ok[k] ? ua + j * p * E : junka;
    }
    // h digits of each x[k], least significant first
    auto piece = [&](uint32_t (&x)[NK], uint32_t h) {
#pragma unroll 2  // h* = 3 for bases 257..1625: two divisions per piece, unrolled
        for (uint32_t i = 0; i + 1 < h; ++i) {
#pragma unroll
            for (uint32_t k = 0; k < NK; ++k) {
                const uint32_t q = magic_div(x[k], mg);
                st_shared<T>(d[k], x[k] - q * B32 + vmin);
                d[k] += E;
                x[k] = q;
            }
        }
#pragma unroll
        for (uint32_t k = 0; k < NK; ++k) {
            st_shared<T>(d[k], x[k] + vmin);
            d[k] += E;
        }
    };
    uint32_t x[NK];
    uint32_t rem = p;
    if (WB == 64 && p > hstar) {
        // split each word into pieces of h* digits (B^h* <= 2^32)
        uint64_t hv[NK];
        split_words<NK, Word>(hv, x, sv, Dh, MD);
        piece(x, hstar);
        rem = p - hstar;
        if (rem > hstar) {  // p = 2 h* + 1: a middle piece of h* digits
            split_words<NK, uint64_t>(hv, x, hv, Dh, MD);
            piece(x, hstar);
            rem -= hstar;
        }
#pragma unroll
        for (uint32_t k = 0; k < NK; ++k) {
            bad |= ok[k] && (hv[k] >> 32) != 0;
            x[k] = (uint32_t)hv[k];
        }
    } else {
#pragma unroll
        for (uint32_t k = 0; k < NK; ++k) {
            if (WB == 64) bad |= ok[k] && ((uint64_t)sv[k] >> 32) != 0;
            x[k] = (uint32_t)sv[k];
        }
    }
    piece(x, rem);
#pragma unroll
    for (uint32_t k = 0; k < NK; ++k)  // the top digit (piece leaves it in x); B <= 2^16 for 16-bit data
        bad |= ok[k] && (sizeof(T) == 2 ? x[k] >= B32 : x[k] >= B);
    return bad;
}

#ifndef PCX_DEC_TAIL3
#define PCX_DEC_TAIL3 1
#endif

// Basic words [jb, je) of one block by one warp (src holds them from word jb
// on): groups of 128 words (four per lane in lockstep), then the rest 32 at
// a time, so W words cost ceil(W / 32) lane slots rather than a multiple of 4.
// (Two instantiations only: separate 2- and 3-word tails, and versions
// specialised on h*, measured slower.)
template <typename T, uint32_t WB>
__device__ __forceinline__ bool decode_basic_block(const typename WordT<T, WB>::type *src /* shared */, T *u,
                                                   T *junk, uint32_t jb, uint32_t je, uint32_t p, uint32_t hstar,
                                                   uint64_t B, uint32_t vmin, Magic32 mg, uint64_t Dh, uint64_t MD)
{
    bool bad = false;
    const uint32_t ua = (uint32_t)__cvta_generic_to_shared(u), junka = (uint32_t)__cvta_generic_to_shared(junk);
    uint32_t j0 = jb;
    for (; j0 + 128 <= je; j0 += 128)
        bad |= decode_basic_group<T, WB, 4, true>(src, jb, ua, junka, j0, je, p, hstar, B, vmin, mg, Dh, MD);
#if PCX_DEC_TAIL3
    // 65-96 words left (a block of white noise, L = 1024, w = 64, has ~86):
    // three words per lane in lockstep instead of three one-word rounds
    if (je - j0 > 64 && je - j0 <= 96) {
        bad |= decode_basic_group<T, WB, 3>(src, jb, ua, junka, j0, je, p, hstar, B, vmin, mg, Dh, MD);
        return bad;
    }
#endif
    for (; j0 < je; j0 += 32)
        bad |= decode_basic_group<T, WB, 1>(src, jb, ua, junka, j0, je, p, hstar, B, vmin, mg, Dh, MD);
    return bad;
}

// A decoded block's samples from a warp's shared slot to global memory:
// 16-byte streaming stores when blocks are whole 16-byte vectors.
template <typename T>
__device__ __forceinline__ void copy_block_out(T *dstg, const T *u, uint32_t n_b, uint32_t L)
{
    const uint32_t lane = threadIdx.x & 31u;
    if ((L * sizeof(T)) % 16 == 0) {
        constexpr uint32_t VE = 16 / sizeof(T);
        const uint32_t nv = n_b / VE;
        const uint4 *sv4 = reinterpret_cast<const uint4 *>(u);
        uint4 *dv4 = reinterpret_cast<uint4 *>(dstg);
        for (uint32_t v = lane; v < nv; v += 32) __stcs(dv4 + v, sv4[v]);
        for (uint32_t i = nv * VE + lane; i < n_b; i += 32) dstg[i] = u[i];
    } else {
        for (uint32_t i = lane; i < n_b; i += 32) dstg[i] = u[i];
    }
}

// Per-block decoding parameters.  In k_decode_w lane b sets up block b of its
// warp's tile and stores the record in the warp's shared record array: the
// first kDecRecBasic bytes for the basic variant, all of it (with the series
// view) for the advanced one.
struct alignas(16) DecBlock {
    uint64_t B, Dh, MD;
    uint64_t lim;  // basic: B^r when the last word's top p - r digits are padding, else 0
    uint32_t vmin, W, woff, p, n_b, hstar;
    Magic32 mg;
    uint32_t pad_[3];
    OrbitView ov;
};
static_assert(offsetof(DecBlock, ov) == kDecRecBasic && sizeof(DecBlock) == kDecRecAdvanced,
              "decoder record sizes");

// Lane `lane`'s record into the array (16-byte stores), for lane < nblk.
template <uint32_t VAR>
__device__ __forceinline__ void store_rec(uint8_t *recs, const DecBlock &d, uint32_t lane)
{
    constexpr uint32_t NV = (VAR == PC_VARIANT_BASIC ? kDecRecBasic : kDecRecAdvanced) / 16;
    const uint4 *v = reinterpret_cast<const uint4 *>(&d);
    uint4 *dst = reinterpret_cast<uint4 *>(recs + lane * (NV * 16));
#pragma unroll
    for (uint32_t i = 0; i < NV; ++i) dst[i] = v[i];
}

#ifndef PCX_ADV_SPLIT_R32
#define PCX_ADV_SPLIT_R32 1
#endif

// Advanced words [jb, je) of one block by one warp (src holds them from word
// jb on), two words per lane in lockstep (words j0 + lane and j0 + 32 +
// lane) while more than 32 are left, then one: each word divided by its R_i, R_{i-1} and r_{i-1} taken from the
// word before (the carry cR, cr for the first), then p_1 digits of every
// word whatever its digit count (see below), the split sample re-joined.
// Lanes past the range write into the junk slots.  qlast / plast: q and p of
// word W - 1 when it is in the range.  Returns true for an invalid word.
template <typename T, uint32_t WB>
__device__ __forceinline__ bool adv_decode_words(const OrbitTable &ot, const DecBlock &k,
                                                 const typename WordT<T, WB>::type *src, uint32_t jb, uint32_t je,
                                                 uint32_t W, T *u, T *junk, uint32_t vmin, uint32_t n_b,
                                                 uint32_t &cR, uint32_t &cr, uint32_t &qlast, uint32_t &plast)
{
    constexpr uint32_t FULLM = 0xFFFFFFFFu;
    const uint32_t lane = threadIdx.x & 31u;
    const uint32_t hstar = k.hstar, B32 = (uint32_t)k.B, p1 = k.p;
    const uint32_t ns = WB == 64 ? p1 / hstar : 0u, rem0 = p1 - ns * hstar;
    bool bad = false;
    uint32_t j0 = jb;
    for (; j0 + 32 < je; j0 += 64) {
        const uint32_t i0 = j0 + lane, i1 = i0 + 32;
        const bool v0 = i0 < je, v1 = i1 < je;
        const SeriesEntry dummy{1u, p1, 0u, Magic32{0xFFFFFFFFu, 0xFFFFFFFFu, 0u}};  // R = 1: divides by one
        SeriesEntry e0 = dummy, e1 = dummy;
        uint64_t s0 = 0, s1 = 0;
        if (v0) {
            e0 = orbit_entry(ot, k.ov, i0);
            s0 = src[i0 - jb];
        }
        if (v1) {
            e1 = orbit_entry(ot, k.ov, i1);
            s1 = src[i1 - jb];
        }
        uint32_t r0, r1;
        uint64_t b0, b1;
        if constexpr (WB == 32) {
            const uint32_t q0 = magic_div((uint32_t)s0, e0.mgR), q1 = magic_div((uint32_t)s1, e1.mgR);
            r0 = (uint32_t)s0 - q0 * e0.R;
            r1 = (uint32_t)s1 - q1 * e1.R;
            b0 = q0;
            b1 = q1;
        } else {
            b0 = divmod_small64(s0, e0.R, e0.mgR, r0);
            b1 = divmod_small64(s1, e1.R, e1.mgR, r1);
        }
        // R_{i-1} and r_{i-1}: the lane before, the last lane of the group
        // before for word j0 + 32, the carry for word j0
        uint32_t Rp0 = __shfl_up_sync(FULLM, e0.R, 1), rp0 = __shfl_up_sync(FULLM, r0, 1);
        uint32_t Rp1 = __shfl_up_sync(FULLM, e1.R, 1), rp1 = __shfl_up_sync(FULLM, r1, 1);
        const uint32_t R31 = __shfl_sync(FULLM, e0.R, 31), r31 = __shfl_sync(FULLM, r0, 31);
        if (lane == 0) {
            Rp0 = cR;
            rp0 = cr;
            Rp1 = R31;
            rp1 = r31;
        }
        cR = __shfl_sync(FULLM, e1.R, 31);
        cr = __shfl_sync(FULLM, r1, 31);
        // every lane takes p_1 digits, whether its word holds p_1 or p_1 - 1
        // samples, so the warp's control flow is the same for all words: a
        // word of p_1 - 1 samples puts its top remainder r'_(i-1) in the p_1-th
        // digit, stored at u[q_i - 1], the slot its split sample takes below
        T *l0 = v0 ? u + e0.q + e0.p - 1 : junk + p1 - 1;
        T *l1 = v1 ? u + e1.q + e1.p - 1 : junk + p1 - 1;
        if constexpr (WB == 64) {
            for (uint32_t t = 0; t < ns; ++t) {
                uint32_t lo0, lo1;
#if PCX_ADV_SPLIT_R32
                if (k.Dh <= 0x80000000ull) {  // remainders formed in 32 bits (as the basic decoder's splits)
                    b0 = divmod_inv64_r32(b0, (uint32_t)k.Dh, k.MD, lo0);
                    b1 = divmod_inv64_r32(b1, (uint32_t)k.Dh, k.MD, lo1);
                } else
#endif
                {
                    uint64_t w0, w1;
                    b0 = divmod_inv64(b0, k.Dh, k.MD, w0);
                    b1 = divmod_inv64(b1, k.Dh, k.MD, w1);
                    lo0 = (uint32_t)w0;
                    lo1 = (uint32_t)w1;
                }
                rev_exact2<T>(l0, lo0, l1, lo1, hstar, B32, k.mg, vmin);
                l0 -= hstar;
                l1 -= hstar;
            }
            bad |= (v0 && (b0 >> 32) != 0) || (v1 && (b1 >> 32) != 0);
        }
        uint32_t x0 = (uint32_t)b0, x1 = (uint32_t)b1;
        rev_quot2<T>(l0, x0, l1, x1, rem0, B32, k.mg, vmin);
        if (v0) {
            uint32_t top = x0;
            if (e0.p != p1) {
                top = (uint32_t)u[e0.q - 1] - vmin;
                bad |= x0 != 0;
            }
            if (i0 == 0) {
                bad |= top != 0;
            } else {
                const uint64_t val = (uint64_t)top * Rp0 + rp0;
                bad |= val >= k.B;
                u[e0.q - 1] = (T)(val + vmin);
            }
            if (e0.q + e0.p >= n_b) bad |= r0 != 0;
            if (i0 == W - 1) {
                qlast = e0.q;
                plast = e0.p;
            }
        }
        if (v1) {
            uint32_t top = x1;
            if (e1.p != p1) {
                top = (uint32_t)u[e1.q - 1] - vmin;
                bad |= x1 != 0;
            }
            const uint64_t val = (uint64_t)top * Rp1 + rp1;  // word j0 + 32 + lane is never word 0
            bad |= val >= k.B;
            u[e1.q - 1] = (T)(val + vmin);
            if (e1.q + e1.p >= n_b) bad |= r1 != 0;
            if (i1 == W - 1) {
                qlast = e1.q;
                plast = e1.p;
            }
        }
    }
    if (j0 < je) {  // 1-32 words left: one word per lane
        const uint32_t i = j0 + lane;
        const bool v = i < je;
        SeriesEntry e{1u, p1, 0u, Magic32{0xFFFFFFFFu, 0xFFFFFFFFu, 0u}};
        uint64_t sw = 0;
        if (v) {
            e = orbit_entry(ot, k.ov, i);
            sw = src[i - jb];
        }
        uint32_t r;
        uint64_t body;
        if constexpr (WB == 32) {
            const uint32_t q = magic_div((uint32_t)sw, e.mgR);
            r = (uint32_t)sw - q * e.R;
            body = q;
        } else {
            body = divmod_small64(sw, e.R, e.mgR, r);
        }
        uint32_t Rp = __shfl_up_sync(FULLM, e.R, 1), rp = __shfl_up_sync(FULLM, r, 1);
        if (lane == 0) {
            Rp = cR;
            rp = cr;
        }
        cR = __shfl_sync(FULLM, e.R, 31);
        cr = __shfl_sync(FULLM, r, 31);
        if (v) {
            T *last = u + e.q + e.p - 1;
            if constexpr (WB == 64) {
                for (uint32_t t = 0; t < ns; ++t) {
                    uint32_t lo;
#if PCX_ADV_SPLIT_R32
                    if (k.Dh <= 0x80000000ull) {
                        body = divmod_inv64_r32(body, (uint32_t)k.Dh, k.MD, lo);
                    } else
#endif
                    {
                        uint64_t w;
                        body = divmod_inv64(body, k.Dh, k.MD, w);
                        lo = (uint32_t)w;
                    }
                    rev_exact<T>(last, lo, hstar, B32, k.mg, vmin);
                    last -= hstar;
                }
                bad |= (body >> 32) != 0;
            }
            const uint32_t qtop = rev_quot<T>(last, (uint32_t)body, rem0, B32, k.mg, vmin);
            uint32_t top = qtop;
            if (e.p != p1) {
                top = (uint32_t)u[e.q - 1] - vmin;
                bad |= qtop != 0;
            }
            if (i == 0) {
                bad |= top != 0;
            } else {
                const uint64_t val = (uint64_t)top * Rp + rp;
                bad |= val >= k.B;
                u[e.q - 1] = (T)(val + vmin);
            }
            if (e.q + e.p >= n_b) bad |= r != 0;
            if (i == W - 1) {
                qlast = e.q;
                plast = e.p;
            }
        }
    }
    return bad;
}

// A block's record from its table entry (vmin, B - 1), range-checked by the
// caller.
template <uint32_t WB, uint32_t VAR, bool ORB>
__device__ __forceinline__ DecBlock dec_setup_entry(uint64_t vmin, uint64_t Bm1, uint32_t n_b, uint32_t L,
                                                    const OrbitTable &ot, WsHeader *ws, uint64_t limit_ns)
{
    DecBlock d{};
    d.B = Bm1 + 1;
    d.vmin = (uint32_t)vmin;
    d.n_b = n_b;
    if (d.B <= 1) return d;
    d.mg = magic32(d.B);
    d.hstar = 1;
    d.Dh = d.B;
    while (d.Dh <= (1ull << 32) / d.B) {
        d.Dh *= d.B;
        ++d.hstar;
    }
    d.MD = ~0ull / d.Dh;
    if constexpr (VAR == PC_VARIANT_BASIC) {
        d.p = basic_p(d.B, WB);
        d.W = (n_b + d.p - 1) / d.p;
        // the last word's digits past the block's end are padding (offset 0):
        // with valid digits that is word < B^r, r = its digits inside the
        // block (B^r < B^p < 2^w)
        const uint32_t r = n_b - (d.W - 1) * d.p;
        if (r < d.p) {
            d.lim = 1;
            for (uint32_t i = 0; i < r; ++i) d.lim *= d.B;
        }
    } else {
        d.p = eq1_p(d.B, WB);  // p_1: every word holds p_1 or p_1 - 1 whole samples
        const uint64_t h = orbit_get<WB>(ot, (uint32_t)d.B, L, ws, limit_ns);  // B <= 65536 here
        if (h != ~0ull) {
            d.ov = orbit_view(ot, h);
            d.W = orbit_words_cached(ot, d.ov, n_b, L);
        }
    }
    return d;
}

template <uint32_t WB, uint32_t VAR, bool ORB>
__device__ __forceinline__ DecBlock dec_setup(const uint8_t *in, uint64_t gb, uint32_t n_b, uint32_t L,
                                              const OrbitTable &ot,
                                              WsHeader *ws, uint64_t limit_ns, uint32_t D)
{
    uint64_t vmin, Bm1;
    if (D == 16) {
        const uint32_t e = reinterpret_cast<const uint32_t *>(in + PC_HEADER_BYTES)[gb];
        vmin = e & 0xFFFFu;
        Bm1 = e >> 16;
    } else {
        const uint64_t e = reinterpret_cast<const uint64_t *>(in + PC_HEADER_BYTES)[gb];
        vmin = e & 0xFFFFFFFFull;
        Bm1 = e >> 32;
    }
    // entries were range-checked by the offsets kernel
    return dec_setup_entry<WB, VAR, ORB>(vmin, Bm1, n_b, L, ot, ws, limit_ns);
}

// One basic word by one lane, its block's constants per lane: digits
// (least significant first) d_i of s, i < p, the first nd of them stored at
// shared address a (+ vmin), the rest checked to be 0 (padding).  Returns
// true if the word is not the image of valid digits.
template <typename T, uint32_t WB>
__device__ __forceinline__ bool decode_word_lane(uint64_t s, uint32_t p, uint32_t nd, uint32_t hstar, uint64_t B,
                                                 uint32_t vmin, Magic32 mg, uint64_t Dh, uint64_t MD, uint32_t a)
{
    constexpr uint32_t E = sizeof(T);
    const uint32_t B32 = (uint32_t)B;
    bool bad = false;
    uint32_t i = 0;
    // h digits of x; returns the last quotient (the piece's top digit)
    auto piece = [&](uint32_t x, uint32_t h) -> uint32_t {
        for (uint32_t t = 0; t + 1 < h; ++t, ++i) {
            const uint32_t q = magic_div(x, mg);
            const uint32_t dg = x - q * B32;
            if (i < nd) st_shared<T>(a + i * E, dg + vmin);
            else bad |= dg != 0;
            x = q;
        }
        if (i < nd) st_shared<T>(a + i * E, x + vmin);
        else bad |= x != 0;
        ++i;
        return x;
    };
    uint32_t rem = p;
    uint64_t hv = s;
    if (WB == 64 && p > hstar) {
        uint32_t lo;
        if (Dh <= 0x80000000ull) hv = divmod_inv64_r32(hv, (uint32_t)Dh, MD, lo);
        else {
            uint64_t l64;
            hv = divmod_inv64(hv, Dh, MD, l64);
            lo = (uint32_t)l64;
        }
        piece(lo, hstar);
        rem = p - hstar;
        if (rem > hstar) {  // p = 2 h* + 1: a middle piece of h* digits
            if (Dh <= 0x80000000ull) hv = divmod_inv64_r32(hv, (uint32_t)Dh, MD, lo);
            else {
                uint64_t l64;
                hv = divmod_inv64(hv, Dh, MD, l64);
                lo = (uint32_t)l64;
            }
            piece(lo, hstar);
            rem -= hstar;
        }
    }
    if (WB == 64) bad |= (hv >> 32) != 0;
    const uint32_t top = piece((uint32_t)hv, rem);
    bad |= sizeof(T) == 2 ? top >= B32 : top >= B;
    return bad;
}

// The words [0, Wt) of a warp tile (global, from g), a lane per word in
// rounds of 32: each lane finds its block (the last record whose word offset
// is <= its word; offsets only grow), decodes its word with that block's
// constants and stores the digits at the block's samples in the tile's
// shared buffer ut (block b at b L); blocks without words are filled with
// their minimum.  The next round's word is loaded before the current one is
// decoded.  Returns true for an invalid word (this lane's).
template <typename T, uint32_t WB>
__device__ bool decode_flat_tile(const typename WordT<T, WB>::type *g, uint32_t Wt, const uint8_t *recs,
                                 uint32_t kRec, uint32_t nblk, uint32_t L, T *ut)
{
    using Word = typename WordT<T, WB>::type;
    const uint32_t lane = threadIdx.x & 31u;
    auto rec = [&](uint32_t b) -> const DecBlock & { return *reinterpret_cast<const DecBlock *>(recs + b * kRec); };
    const uint32_t ua = (uint32_t)__cvta_generic_to_shared(ut);
    bool bad = false;
    uint32_t b = 0;
    Word s = lane < Wt ? g[lane] : Word(0);
    for (uint32_t g0 = 0; g0 < Wt; g0 += 32) {
        const uint32_t j = g0 + lane;
        const Word next = j + 32 < Wt ? g[j + 32] : Word(0);
        if (j < Wt) {
            while (b + 1 < nblk && rec(b + 1).woff <= j) ++b;
            const DecBlock &k = rec(b);
            const uint32_t jw = j - k.woff, first = jw * k.p;
            const uint32_t nd = min(k.p, k.n_b - first);
            bad |= decode_word_lane<T, WB>((uint64_t)s, k.p, nd, k.hstar, k.B, k.vmin, k.mg, k.Dh, k.MD,
                                           ua + (b * L + first) * (uint32_t)sizeof(T));
        }
        s = next;
    }
    for (uint32_t c = 0; c < nblk; ++c) {
        const DecBlock &k = rec(c);
        if (k.W == 0)
            for (uint32_t i = lane; i < k.n_b; i += 32) ut[c * L + i] = (T)k.vmin;
    }
    return bad;
}

// Warp-granular decoding (basic, and advanced with the series table on 16-bit
// data): no shared barrier at all.  A warp owns a tile of consecutive blocks
// (up to dec_tile_cap, fewer for a short stream); lane b sets up block b
// (table entry, word count, division constants, series view) and stores its
// record in the warp's shared record array, then the warp decodes the blocks
// one by one into its own shared-memory slot and stores each block's samples
// with 16-byte streaming stores.  5 CTAs of 4 warps per SM: registers capped
// at 102 (PCX_DECODE_MIN_CTAS).
template <typename T, uint32_t WB, uint32_t VAR, bool ORB, bool CHUNKED>
__global__ void __launch_bounds__(kDecWarpsMax * 32, PCX_DECODE_MIN_CTAS)
k_decode_w(const uint8_t *__restrict__ in, uint32_t L, T *__restrict__ out, uint64_t *__restrict__ n_out,
           WsHeader *ws, const uint64_t *__restrict__ offsets, OrbitTable ot, uint64_t limit_ns, uint32_t wtb)
{
    using Word = typename WordT<T, WB>::type;
    constexpr uint32_t D = sizeof(T) * 8;
    extern __shared__ __align__(16) uint8_t smem[];
    const uint32_t warp = threadIdx.x >> 5, lane = threadIdx.x & 31u;
    // per warp: one block's samples (+ padding, + junk for idle lanes), then
    // two buffers of packed words: a whole block's (the next block streams in
    // while the current one is decoded), or, for long blocks, kDecChunk words
    // (the next chunk, of this block or the next, streams in)
    const uint32_t cw = dec_chunk_words(VAR, D, WB, L);
    const uint32_t slot_bytes = (uint32_t)round_up((uint64_t)(L + 2 * kPad) * sizeof(T), 16);
    const uint32_t warp_bytes = decw_warp_bytes(VAR, D, WB, L);
    const uint32_t nwarps = blockDim.x >> 5;
    T *u = reinterpret_cast<T *>(smem + warp * warp_bytes);
    Word *wbuf = reinterpret_cast<Word *>(smem + warp * warp_bytes + slot_bytes);
    // then the tile's block records
    constexpr uint32_t kRec = VAR == PC_VARIANT_BASIC ? kDecRecBasic : kDecRecAdvanced;
    uint8_t *recs = smem + warp * warp_bytes + decw_front_bytes(VAR, D, WB, L, dec_tile_cap(VAR, D, WB, L));
    auto rec = [&](uint32_t b) -> const DecBlock & { return *reinterpret_cast<const DecBlock *>(recs + b * kRec); };
    const bool flat = dec_flat(VAR, D, WB, L);  // the flat path reuses the slot and buffers for the tile's samples

    if (*reinterpret_cast<volatile uint32_t *>(&ws->status) != PC_OK) return;
    const uint64_t *h64 = reinterpret_cast<const uint64_t *>(in);
    const uint64_t n = h64[2], n_blocks = h64[3];
    const uint64_t n_wt = ceil_div(n_blocks, wtb);
    const uint64_t payload_off = PC_HEADER_BYTES + table_bytes(n_blocks, D);
    const Word *payload = reinterpret_cast<const Word *>(in + payload_off);
    const uint64_t gw0 = (uint64_t)blockIdx.x * nwarps + warp, nw = (uint64_t)gridDim.x * nwarps;
    bool bad = false;

    for (uint64_t wt = gw0; wt < n_wt; wt += nw) {
        const uint64_t blk0 = wt * wtb;
        const uint32_t nblk = (uint32_t)umin64(wtb, n_blocks - blk0);
        uint32_t nz;  // lanes (blocks) with words
        {
            DecBlock mine{};
            if (lane < nblk) {
                const uint64_t gb = blk0 + lane;
                const uint32_t n_b = (uint32_t)umin64(L, n - gb * L);
                mine = dec_setup<WB, VAR, ORB>(in, gb, n_b, L, ot, ws, limit_ns, D);
            }
            const uint32_t incl = warp_incl_scan_u32(mine.W);
            mine.woff = incl - mine.W;
            nz = __ballot_sync(0xFFFFFFFFu, lane < nblk && mine.W > 0);
            if (lane < nblk) store_rec<VAR>(recs, mine, lane);
            __syncwarp();
        }
        if constexpr (!CHUNKED && VAR == PC_VARIANT_BASIC) {
            if (flat) {  // short blocks: a lane per word across the tile
                const uint32_t Wt = __shfl_sync(0xFFFFFFFFu, nz ? rec(nblk - 1).woff + rec(nblk - 1).W : 0u, 0);
                bad |= decode_flat_tile<T, WB>(payload + offsets[wt], Wt, recs, kRec, nblk, L, u);
                __syncwarp();
                uint32_t nt = 0;  // the tile's samples
                for (uint32_t b = 0; b < nblk; ++b) nt += rec(b).n_b;
                copy_block_out<T>(out + blk0 * L, u, nt, L);
                __syncwarp();
                if (wt == n_wt - 1 && lane == 0) *n_out = n;
                continue;
            }
        }
        if constexpr (!CHUNKED) {
            const uint64_t base = offsets[wt];
            auto prefetch = [&](uint32_t b) {  // block b's words into buffer b & 1
                const uint32_t Wb = rec(b).W, ob = rec(b).woff;
                const Word *g = payload + base + ob;
                Word *dstw = wbuf + (b & 1u) * cw;
                uint32_t j = lane;
                for (; j + 96 < Wb; j += 128) {  // four words per lane per step
                    cp_async_small<sizeof(Word)>(dstw + j, g + j);
                    cp_async_small<sizeof(Word)>(dstw + j + 32, g + j + 32);
                    cp_async_small<sizeof(Word)>(dstw + j + 64, g + j + 64);
                    cp_async_small<sizeof(Word)>(dstw + j + 96, g + j + 96);
                }
                for (; j < Wb; j += 32) cp_async_small<sizeof(Word)>(dstw + j, g + j);
                cp_async_commit();
            };
            prefetch(0);

            for (uint32_t b = 0; b < nblk; ++b) {
                if (b + 1 < nblk) prefetch(b + 1);
                else cp_async_commit();
                cp_async_wait<1>();
                __syncwarp();
                const DecBlock &k = rec(b);
                const uint64_t gb = blk0 + b;
                const uint32_t vmin = k.vmin, W = k.W, n_b = k.n_b;
                const Word *wsrc = wbuf + (b & 1u) * cw;
                if (W == 0) {
                    for (uint32_t i = lane; i < n_b; i += 32) u[i] = (T)vmin;
                } else if constexpr (VAR == PC_VARIANT_BASIC) {
                    const uint32_t p = k.p;
                    bad |= decode_basic_block<T, WB>(wsrc, u, u + L + kPad, 0, W, p, k.hstar, k.B, vmin, k.mg, k.Dh, k.MD);
                    if (k.lim != 0) bad |= (uint64_t)wsrc[W - 1] >= k.lim;
                } else {
                    uint32_t cR = 1, cr = 0, qlast = 0, plast = 0;
                    bad |= adv_decode_words<T, WB>(ot, k, wsrc, 0, W, W, u, u + L + kPad, vmin, n_b, cR, cr, qlast,
                                                   plast);
                    __syncwarp();
                    const uint32_t src_lane = (W - 1) & 31u;
                    qlast = __shfl_sync(0xFFFFFFFFu, qlast, src_lane);
                    plast = __shfl_sync(0xFFFFFFFFu, plast, src_lane);
                    if (lane == 0)
                        for (uint32_t i = n_b; i < qlast + plast; ++i) bad |= (uint32_t)u[i] != vmin;
                }
                __syncwarp();
                // this block's samples out
                T *dstg = out + gb * L;
                copy_block_out<T>(dstg, u, n_b, L);
                __syncwarp();
            }
        } else {
            const uint64_t base = offsets[wt];
            auto prefetch = [&](uint32_t b, uint32_t c, uint32_t slot) {  // chunk c of block b into a buffer
                const uint32_t Wb = rec(b).W, ob = rec(b).woff;
                const uint32_t j0 = c * cw, cnt = min(cw, Wb - j0);
                const Word *g = payload + base + ob + j0;
                Word *dstw = wbuf + slot * cw;
                for (uint32_t j = lane; j < cnt; j += 32) cp_async_small<sizeof(Word)>(dstw + j, g + j);
                cp_async_commit();
            };
            uint32_t slot = 0;
            if (nz) prefetch((uint32_t)__ffs(nz) - 1u, 0, 0);

            for (uint32_t b = 0; b < nblk; ++b) {
                const DecBlock &k = rec(b);
                const uint64_t gb = blk0 + b;
                const uint32_t vmin = k.vmin, W = k.W, n_b = k.n_b;
                if (W == 0) {
                    for (uint32_t i = lane; i < n_b; i += 32) u[i] = (T)vmin;
                } else {
                    const uint32_t nch = (W + cw - 1) / cw;
                    uint32_t cR = 1, cr = 0, qlast = 0, plast = 0;  // advanced: carries across words
                    for (uint32_t c = 0; c < nch; ++c) {
                        // the next chunk: this block's next, else the next block with words
                        if (c + 1 < nch) {
                            prefetch(b, c + 1, slot ^ 1u);
                        } else {
                            const uint32_t later = nz & ~((2u << b) - 1u);
                            if (later) prefetch((uint32_t)__ffs(later) - 1u, 0, slot ^ 1u);
                            else cp_async_commit();
                        }
                        cp_async_wait<1>();
                        __syncwarp();
                        const Word *wsrc = wbuf + slot * cw;
                        const uint32_t jb = c * cw, je = min(W, jb + cw);
                        if constexpr (VAR == PC_VARIANT_BASIC) {
                            bad |= decode_basic_block<T, WB>(wsrc, u, u + L + kPad, jb, je, k.p, k.hstar, k.B, vmin, k.mg,
                                                             k.Dh, k.MD);
                        } else {
                            bad |= adv_decode_words<T, WB>(ot, k, wsrc, jb, je, W, u, u + L + kPad, vmin, n_b, cR, cr,
                                                           qlast, plast);
                        }
                        __syncwarp();  // the buffer is free for the chunk after next
                        slot ^= 1u;
                    }
                    // digits past the block's end must be padding (offset 0)
                    uint32_t end;
                    if constexpr (VAR == PC_VARIANT_BASIC) {
                        end = W * k.p;
                    } else {
                        const uint32_t src_lane = (W - 1) & 31u;
                        qlast = __shfl_sync(0xFFFFFFFFu, qlast, src_lane);
                        plast = __shfl_sync(0xFFFFFFFFu, plast, src_lane);
                        end = qlast + plast;
                    }
                    for (uint32_t i = n_b + lane; i < end; i += 32) bad |= (uint32_t)u[i] != vmin;
                }
                __syncwarp();
                // this block's samples out
                T *dstg = out + gb * L;
                copy_block_out<T>(dstg, u, n_b, L);
                __syncwarp();
            }
        }
        if (wt == n_wt - 1 && lane == 0) *n_out = n;
    }
    cp_async_wait<0>();
    if (__any_sync(0xFFFFFFFFu, bad) && lane == 0) record_error(ws, PC_ERR_CORRUPT);
}

template <typename T, uint32_t WB, uint32_t VAR, bool ORB>
static cudaError_t launch_decompress_t(const LaunchArgs &a)
{
    cudaError_t e;
    int dev = 0, sms = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    const TileCfg cfg = tile_cfg(kKernelDecode, VAR, sizeof(T) * 8, WB, a.L, ORB);
    const OrbitTable ot{a.orb_flags, a.orb_hdr, static_cast<ulonglong2 *>(a.orb_slots), &a.ws->orbit_cursor};
    // 1. offsets (look-back over tiles of kOffsetTileBlocks blocks)
    {
        auto kern = k_offsets<T, WB, VAR, ORB>;
        int per_sm = 0;
        if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kThreads, 0)) != cudaSuccess)
            return e;
        if (per_sm < 1) return cudaErrorInvalidConfiguration;
        uint64_t grid = (uint64_t)per_sm * sms;
        const uint64_t need = a.n_status;  // never more tiles than status words
        if (need < grid) grid = need;
        if (grid < 1) grid = 1;
        constexpr bool kWarpTiles = VAR == PC_VARIANT_BASIC || (ORB && sizeof(T) == 2);
        const uint32_t dtb = kWarpTiles ? a.tb : cfg.tb;
        kern<<<(unsigned)grid, kThreads, 0, a.stream>>>(
            static_cast<const uint8_t *>(a.in), a.in_bytes, a.L, a.cap, a.out_count, a.ws, a.status,
            a.n_status, a.offsets, a.n_offsets, dtb, a.limit_ns, ot);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    // 2. decode: warp tiles where no serial walk is needed, CTA tiles otherwise
    constexpr bool kWarpPath = VAR == PC_VARIANT_BASIC || (ORB && sizeof(T) == 2);
    if constexpr (kWarpPath) {
        auto kern = dec_chunked(VAR, sizeof(T) * 8, WB, a.L) ? k_decode_w<T, WB, VAR, ORB, true>
                                                             : k_decode_w<T, WB, VAR, ORB, false>;
        const uint32_t nwarps = decw_warps(VAR, sizeof(T) * 8, WB, a.L);
        if (nwarps < 1) return cudaErrorInvalidConfiguration;
        const uint32_t smem = nwarps * decw_warp_bytes(VAR, sizeof(T) * 8, WB, a.L);
        if ((e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) !=
            cudaSuccess)
            return e;

        int per_sm = 0;
        if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, nwarps * 32, smem)) != cudaSuccess)
            return e;
        if (per_sm < 1) return cudaErrorInvalidConfiguration;
        uint64_t grid = (uint64_t)per_sm * sms;
        const uint64_t need = ceil_div(a.n_offsets, nwarps);  // warp tiles <= offsets - 1
        if (need < grid) grid = need;
        if (grid < 1) grid = 1;
        kern<<<(unsigned)grid, nwarps * 32, smem, a.stream>>>(
            static_cast<const uint8_t *>(a.in), a.L, static_cast<T *>(a.out), a.out_count, a.ws, a.offsets, ot,
            a.limit_ns, a.tb);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    } else {
        auto kern = k_decode<T, WB, VAR, ORB>;
        if ((e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)cfg.smem)) !=
            cudaSuccess)
            return e;
        int per_sm = 0;
        if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kThreads, cfg.smem)) != cudaSuccess)
            return e;
        if (per_sm < 1) return cudaErrorInvalidConfiguration;
        uint64_t grid = (uint64_t)per_sm * sms;
        const uint64_t need = a.n_offsets;  // decoding tiles + 1
        if (need < grid) grid = need;
        if (grid < 1) grid = 1;
        kern<<<(unsigned)grid, kThreads, cfg.smem, a.stream>>>(
            static_cast<const uint8_t *>(a.in), a.L, static_cast<T *>(a.out), a.out_count, a.ws, a.offsets, ot,
            a.limit_ns);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    return cudaSuccess;
}

cudaError_t launch_decompress(const LaunchArgs &a)
{
    const uint32_t key = (a.d == 32 ? 4u : 0u) | (a.w == 64 ? 2u : 0u) | (a.variant ? 1u : 0u);
    switch (key) {
    case 0: return launch_decompress_t<uint16_t, 32, 0, false>(a);
    case 1: return a.orbit ? launch_decompress_t<uint16_t, 32, 1, true>(a) : launch_decompress_t<uint16_t, 32, 1, false>(a);
    case 2: return launch_decompress_t<uint16_t, 64, 0, false>(a);
    case 3: return a.orbit ? launch_decompress_t<uint16_t, 64, 1, true>(a) : launch_decompress_t<uint16_t, 64, 1, false>(a);
    case 4: return launch_decompress_t<uint32_t, 32, 0, false>(a);
    case 5: return a.orbit ? launch_decompress_t<uint32_t, 32, 1, true>(a) : launch_decompress_t<uint32_t, 32, 1, false>(a);
    case 6: return launch_decompress_t<uint32_t, 64, 0, false>(a);
    default: return a.orbit ? launch_decompress_t<uint32_t, 64, 1, true>(a) : launch_decompress_t<uint32_t, 64, 1, false>(a);
    }
}

// ---- format version 2 (segmented streams) --------------------------------

// Body offsets of a version-2 stream: every CTA checks the header; one thread
// per segment reads its code and stored body size; a block-wide scan and the
// bounded look-back over tiles of kV2TileSegs segments give every body's
// offset.  The last tile checks that the sizes add up to the header's
// body_bytes and that the two arrays' paddings are zero.
template <uint32_t NT>
__global__ void __launch_bounds__(NT)
k_v2_offsets(const uint8_t *__restrict__ in, uint64_t in_bytes, uint32_t variant, uint32_t d, uint32_t seg_len,
             uint64_t cap, uint64_t max_segments, uint64_t *__restrict__ n_out, WsHeader *ws, uint64_t *status,
             uint64_t *offsets, uint64_t limit_ns)
{
    constexpr uint32_t NW = NT / 32;
    __shared__ uint64_t hdr[3];
    __shared__ uint64_t warp_tot[NW];
    __shared__ uint64_t s_excl;
    __shared__ uint32_t s_code, s_tile, s_ok;
    const uint32_t warp = threadIdx.x >> 5, lane = threadIdx.x & 31u;
    if (threadIdx.x == 0) {  // the host checked in_bytes >= PC_HEADER_BYTES
        const uint32_t *h = reinterpret_cast<const uint32_t *>(in);
        const uint64_t *h64 = reinterpret_cast<const uint64_t *>(in);
        const uint64_t n = h64[2], n_seg = h64[3], body = h64[4];
        uint32_t code = PC_OK;
        if (h[0] != 0x504D4350u || h[1] != (2u | (variant << 16) | (d << 24)) || h[2] != 0 || h[3] != seg_len ||
            h64[5] != 0 || h64[6] != 0 || h64[7] != 0 || n_seg != ceil_div(n, seg_len))
            code = PC_ERR_CORRUPT;
        else if (n > cap || n_seg > max_segments)
            code = PC_ERR_CAPACITY;
        else {
            const V2Geom g = v2_geom(n_seg);
            if (g.bodies_at > in_bytes || body > in_bytes - g.bodies_at) code = PC_ERR_CORRUPT;
        }
        hdr[0] = n;
        hdr[1] = n_seg;
        hdr[2] = body;
        s_code = code;
    }
    __syncthreads();
    if (s_code != PC_OK) {
        if (blockIdx.x == 0 && threadIdx.x == 0) record_error(ws, s_code);
        return;
    }
    const uint64_t n = hdr[0], n_seg = hdr[1], body_bytes = hdr[2];
    const V2Geom g = v2_geom(n_seg);
    const uint32_t *sizes = reinterpret_cast<const uint32_t *>(in + g.sizes_at);
    const uint64_t n_tiles = ceil_div(n_seg, kV2TileSegs);
    if (n_tiles == 0) {
        if (blockIdx.x == 0 && threadIdx.x == 0) {
            if (body_bytes != 0) record_error(ws, PC_ERR_CORRUPT);
            offsets[0] = 0;
            *n_out = 0;
        }
        return;
    }
    for (;;) {
        if (threadIdx.x == 0) s_tile = atomicAdd(&ws->ticket, 1u);
        __syncthreads();
        const uint64_t tile = s_tile;
        if (tile >= n_tiles) break;
        uint64_t v = 0;  // this thread's segments' sizes (kV2TileSegs / NT of them), bytes
        uint64_t mine[kV2TileSegs / NT];
#pragma unroll
        for (uint32_t i = 0; i < kV2TileSegs / NT; ++i) {
            const uint64_t sg = tile * kV2TileSegs + threadIdx.x * (kV2TileSegs / NT) + i;
            mine[i] = 0;
            if (sg < n_seg) {
                if (!v2_code_ok(in[PC_HEADER_BYTES + sg])) record_error(ws, PC_ERR_CORRUPT);
                mine[i] = 8ull * sizes[sg];
            }
            v += mine[i];
        }
        // block-wide exclusive scan of v (64-bit: up to 2^35 bytes per thread)
        uint64_t incl = v;
#pragma unroll
        for (uint32_t o = 1; o < 32; o <<= 1) {
            const uint64_t t = __shfl_up_sync(0xFFFFFFFFu, incl, o);
            if (lane >= o) incl += t;
        }
        if (lane == 31) warp_tot[warp] = incl;
        __syncthreads();
        if (warp == 0) {
            const uint64_t t = lane < NW ? warp_tot[lane] : 0ull;
            uint64_t ti = t;
#pragma unroll
            for (uint32_t o = 1; o < 32; o <<= 1) {
                const uint64_t u = __shfl_up_sync(0xFFFFFFFFu, ti, o);
                if (lane >= o) ti += u;
            }
            if (lane < NW) warp_tot[lane] = ti - t;
            const uint64_t agg = __shfl_sync(0xFFFFFFFFu, ti, 31);
            uint64_t excl = 0;
            const bool ok = lookback_warp(status, tile, agg, ws, limit_ns, &excl);
            if (lane == 0) {
                s_excl = excl;
                s_ok = ok ? 1u : 0u;
            }
        }
        __syncthreads();
        if (s_ok) {
            uint64_t off = s_excl + warp_tot[warp] + (incl - v);
#pragma unroll
            for (uint32_t i = 0; i < kV2TileSegs / NT; ++i) {
                const uint64_t sg = tile * kV2TileSegs + threadIdx.x * (kV2TileSegs / NT) + i;
                if (sg < n_seg) {
                    offsets[sg] = off;
                    if (sg == n_seg - 1) {
                        offsets[n_seg] = off + mine[i];
                        if (off + mine[i] != body_bytes) record_error(ws, PC_ERR_CORRUPT);
                        for (uint64_t o = PC_HEADER_BYTES + n_seg; o < g.sizes_at; ++o)
                            if (in[o] != 0) record_error(ws, PC_ERR_CORRUPT);
                        for (uint64_t o = g.sizes_at + 4 * n_seg; o < g.bodies_at; ++o)
                            if (in[o] != 0) record_error(ws, PC_ERR_CORRUPT);
                        *n_out = n;
                    }
                }
                off += mine[i];
            }
        }
        __syncthreads();
    }
}

// One segment of a version-2 stream by one warp: its blocks' word counts
// (lane per block, 32 at a time) must give the stored body size; then the
// blocks are set up 32 at a time (records in the warp's shared memory) and
// decoded one by one as k_decode_w decodes a chunked block: words staged
// kDecChunk at a time, digits into the warp's sample slot, samples out.
// Returns true if the segment is corrupt.
template <typename T, uint32_t WB, uint32_t VAR>
__device__ bool v2_segment(const uint8_t *body, uint64_t size, uint32_t n_s, uint32_t L, uint32_t slot_elems,
                           T *__restrict__ out, uint8_t *wsm, const OrbitTable &ot, WsHeader *ws, uint64_t limit_ns)
{
    using Word = typename WordT<T, WB>::type;
    constexpr uint32_t D = sizeof(T) * 8, DB = D / 8;
    constexpr uint64_t kDmax = D == 16 ? 0xFFFFull : 0xFFFFFFFFull;
    constexpr uint32_t kRec = VAR == PC_VARIANT_BASIC ? kDecRecBasic : kDecRecAdvanced;
    const uint32_t lane = threadIdx.x & 31u;
    T *u = reinterpret_cast<T *>(wsm);
    T *junk = u + slot_elems - kPad;
    const uint32_t slot_bytes = (uint32_t)round_up((uint64_t)slot_elems * sizeof(T), 16);
    Word *wbuf = reinterpret_cast<Word *>(wsm + slot_bytes);
    uint8_t *recs = wsm + slot_bytes + kDecChunk * sizeof(Word);
    auto rec = [&](uint32_t b) -> const DecBlock & { return *reinterpret_cast<const DecBlock *>(recs + b * kRec); };

    const uint32_t nb = (n_s + L - 1) / L;
    const uint64_t tb = (uint64_t)nb * 2 * DB, words_at = round8(tb);
    if (words_at > size) return true;
    auto entry = [&](uint32_t b, uint64_t &vmin, uint64_t &Bm1) {
        if constexpr (D == 16) {
            const uint32_t e = reinterpret_cast<const uint32_t *>(body)[b];
            vmin = e & 0xFFFFu;
            Bm1 = e >> 16;
        } else {
            const uint64_t e = reinterpret_cast<const uint64_t *>(body)[b];
            vmin = e & 0xFFFFFFFFull;
            Bm1 = e >> 32;
        }
    };
    // 1. word counts: the stored size must be the table's
    bool bad = false;
    uint64_t total = 0;
    for (uint32_t b0 = 0; b0 < nb; b0 += 32) {
        const uint32_t b = b0 + lane;
        uint32_t W = 0;
        if (b < nb) {
            uint64_t vmin, Bm1;
            entry(b, vmin, Bm1);
            if (vmin + Bm1 > kDmax) {
                bad = true;
                Bm1 = 0;
            }
            W = block_words<WB, VAR, true>(Bm1 + 1, min(L, n_s - b * L), L, ot, ws, limit_ns);
        }
        total += warp_sum_u64(W);
    }
    if (__any_sync(0xFFFFFFFFu, bad) || words_at + round8(total * (WB / 8)) != size) return true;
    for (uint64_t o = tb + lane; o < words_at; o += 32) bad |= body[o] != 0;
    for (uint64_t o = words_at + total * (WB / 8) + lane; o < size; o += 32) bad |= body[o] != 0;
    const Word *words = reinterpret_cast<const Word *>(body + words_at);

    // 2. blocks, 32 records at a time
    uint64_t run = 0;  // words of the earlier rounds
    for (uint32_t b0 = 0; b0 < nb; b0 += 32) {
        const uint32_t m = min(32u, nb - b0);
        DecBlock mine{};
        if (lane < m) {
            uint64_t vmin, Bm1;
            entry(b0 + lane, vmin, Bm1);
            mine = dec_setup_entry<WB, VAR, true>(vmin, Bm1, min(L, n_s - (b0 + lane) * L), L, ot, ws, limit_ns);
        }
        const uint32_t incl = warp_incl_scan_u32(mine.W);
        mine.woff = incl - mine.W;
        __syncwarp();  // the previous round's records are read
        if (lane < m) store_rec<VAR>(recs, mine, lane);
        __syncwarp();
        for (uint32_t b = 0; b < m; ++b) {
            const DecBlock &k = rec(b);
            const uint32_t vmin = k.vmin, W = k.W, n_b = k.n_b;
            if (W == 0) {
                for (uint32_t i = lane; i < n_b; i += 32) u[i] = (T)vmin;
            } else {
                const uint32_t nch = (W + kDecChunk - 1) / kDecChunk;
                uint32_t cR = 1, cr = 0, qlast = 0, plast = 0;  // advanced: carries across words
                for (uint32_t c = 0; c < nch; ++c) {
                    const uint32_t jb = c * kDecChunk, je = min(W, jb + kDecChunk);
                    const Word *g = words + run + k.woff + jb;
                    for (uint32_t j = lane; j < je - jb; j += 32) wbuf[j] = g[j];
                    __syncwarp();
                    if constexpr (VAR == PC_VARIANT_BASIC) {
                        bad |= decode_basic_block<T, WB>(wbuf, u, junk, jb, je, k.p, k.hstar, k.B, vmin, k.mg, k.Dh,
                                                         k.MD);
                    } else {
                        bad |= adv_decode_words<T, WB>(ot, k, wbuf, jb, je, W, u, junk, vmin, n_b, cR, cr, qlast,
                                                       plast);
                    }
                    __syncwarp();  // the buffer is free for the next chunk
                }
                // digits past the block's end must be padding (offset 0)
                uint32_t end;
                if constexpr (VAR == PC_VARIANT_BASIC) {
                    end = W * k.p;
                } else {
                    const uint32_t src_lane = (W - 1) & 31u;
                    qlast = __shfl_sync(0xFFFFFFFFu, qlast, src_lane);
                    plast = __shfl_sync(0xFFFFFFFFu, plast, src_lane);
                    end = qlast + plast;
                }
                for (uint32_t i = n_b + lane; i < end; i += 32) bad |= (uint32_t)u[i] != vmin;
            }
            __syncwarp();
            T *dst = out + (uint64_t)(b0 + b) * L;
            for (uint32_t i = lane; i < n_b; i += 32) dst[i] = u[i];
            __syncwarp();
        }
        run += __shfl_sync(0xFFFFFFFFu, incl, 31);
    }
    return __any_sync(0xFFFFFFFFu, bad);
}

// Shared memory of one warp of k_v2_decode: the sample slot of the longest
// block (at most the segment), one chunk of words, 32 block records.
PCX_HD uint32_t v2_slot_elems(uint32_t seg_len)
{
    return (seg_len < (1u << kV2MaxLog2L) ? seg_len : (1u << kV2MaxLog2L)) + 2 * kPad;
}
PCX_HD uint32_t v2_warp_bytes(uint32_t variant, uint32_t d, uint32_t seg_len)
{
    return (uint32_t)(round_up((uint64_t)v2_slot_elems(seg_len) * (d / 8), 16) + kDecChunk * 8ull +
                      32ull * (variant == PC_VARIANT_BASIC ? kDecRecBasic : kDecRecAdvanced));
}

// Decoding of a version-2 stream: a warp per segment, round-robin; the
// segment's code picks the word size.
template <typename T, uint32_t VAR>
__global__ void __launch_bounds__(kDecWarpsMax * 32)
k_v2_decode(const uint8_t *__restrict__ in, uint32_t seg_len, T *__restrict__ out, WsHeader *ws,
            const uint64_t *__restrict__ offsets, OrbitTable ot32, OrbitTable ot64, uint64_t limit_ns,
            uint32_t warp_bytes)
{
    extern __shared__ __align__(16) uint8_t smem[];
    const uint32_t warp = threadIdx.x >> 5, lane = threadIdx.x & 31u;
    if (*reinterpret_cast<volatile uint32_t *>(&ws->status) != PC_OK) return;
    const uint64_t *h64 = reinterpret_cast<const uint64_t *>(in);
    const uint64_t n = h64[2], n_seg = h64[3];
    const V2Geom g = v2_geom(n_seg);
    const uint32_t *sizes = reinterpret_cast<const uint32_t *>(in + g.sizes_at);
    uint8_t *wsm = smem + warp * warp_bytes;
    const uint32_t nwarps = blockDim.x >> 5;
    const uint32_t slot_elems = v2_slot_elems(seg_len);
    bool bad = false;
    for (uint64_t sg = (uint64_t)blockIdx.x * nwarps + warp; sg < n_seg; sg += (uint64_t)gridDim.x * nwarps) {
        const uint32_t code = in[PC_HEADER_BYTES + sg];
        if (!v2_code_ok(code)) {  // recorded by the offsets kernel
            bad = true;
            continue;
        }
        const uint32_t L = v2_L(code);
        const uint32_t n_s = (uint32_t)umin64(seg_len, n - sg * seg_len);
        const uint8_t *body = in + g.bodies_at + offsets[sg];
        const uint64_t size = 8ull * sizes[sg];
        T *dst = out + sg * seg_len;
        if (v2_w(code) == 64) bad |= v2_segment<T, 64, VAR>(body, size, n_s, L, slot_elems, dst, wsm, ot64, ws, limit_ns);
        else bad |= v2_segment<T, 32, VAR>(body, size, n_s, L, slot_elems, dst, wsm, ot32, ws, limit_ns);
    }
    if (__any_sync(0xFFFFFFFFu, bad) && lane == 0) record_error(ws, PC_ERR_CORRUPT);
}

template <typename T, uint32_t VAR>
static cudaError_t launch_v2_decode_t(const V2DecodeArgs &a)
{
    cudaError_t e;
    int dev = 0, sms = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    uint8_t *base = static_cast<uint8_t *>(a.workspace);
    WsHeader *ws = reinterpret_cast<WsHeader *>(base);
    const V2Layout lay = v2_layout(VAR == PC_VARIANT_ADVANCED, true, a.max_segments);
    uint64_t *status = reinterpret_cast<uint64_t *>(base + lay.off_status);
    uint64_t *offsets = reinterpret_cast<uint64_t *>(base + lay.off_offsets);
    const OrbitTable ot32{reinterpret_cast<uint32_t *>(base + lay.off_flags32),
                          reinterpret_cast<uint64_t *>(base + lay.off_hdr32),
                          reinterpret_cast<ulonglong2 *>(base + lay.off_slots32), &ws->orbit_cursor};
    const OrbitTable ot64{reinterpret_cast<uint32_t *>(base + lay.off_flags64),
                          reinterpret_cast<uint64_t *>(base + lay.off_hdr64),
                          reinterpret_cast<ulonglong2 *>(base + lay.off_slots64), &ws->reserved_cursor64};
    if ((e = cudaMemsetAsync(base, 0, VAR == PC_VARIANT_ADVANCED ? 12 : 32, a.stream)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(status, 0, 8 * lay.n_status, a.stream)) != cudaSuccess) return e;
    if constexpr (VAR == PC_VARIANT_ADVANCED) {
        if ((e = launch_orbit_prepare(ws, ot32.flags, 2 * kOrbitFlagsBytes, &ws->orbit_cursor,
                                      &ws->reserved_cursor64, kOrbitTagV2, a.stream)) != cudaSuccess)
            return e;
    }
    {
        auto kern = k_v2_offsets<kThreads>;
        int per_sm = 0;
        if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kThreads, 0)) != cudaSuccess) return e;
        if (per_sm < 1) return cudaErrorInvalidConfiguration;
        uint64_t grid = (uint64_t)per_sm * sms;
        if (lay.n_status < grid) grid = lay.n_status;
        kern<<<(unsigned)grid, kThreads, 0, a.stream>>>(static_cast<const uint8_t *>(a.in), a.in_bytes, VAR,
                                                        sizeof(T) * 8, a.seg_len, a.cap, a.max_segments, a.n_out, ws,
                                                        status, offsets, a.limit_ns);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    {
        auto kern = k_v2_decode<T, VAR>;
        const uint32_t wb = v2_warp_bytes(VAR, sizeof(T) * 8, a.seg_len);
        const uint32_t smem = kDecWarpsMax * wb;
        if ((e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) != cudaSuccess)
            return e;
        int per_sm = 0;
        if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kDecWarpsMax * 32, smem)) !=
            cudaSuccess)
            return e;
        if (per_sm < 1) return cudaErrorInvalidConfiguration;
        uint64_t grid = (uint64_t)per_sm * sms;
        const uint64_t need = ceil_div(a.max_segments, kDecWarpsMax);
        if (need < grid) grid = need;
        if (grid < 1) grid = 1;
        kern<<<(unsigned)grid, kDecWarpsMax * 32, smem, a.stream>>>(static_cast<const uint8_t *>(a.in), a.seg_len,
                                                                    static_cast<T *>(a.out), ws, offsets, ot32, ot64,
                                                                    a.limit_ns, wb);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    return cudaSuccess;
}

cudaError_t launch_v2_decode(const V2DecodeArgs &a)
{
    if (a.d == 16) return a.variant ? launch_v2_decode_t<uint16_t, 1>(a) : launch_v2_decode_t<uint16_t, 0>(a);
    if (a.variant == 0) return launch_v2_decode_t<uint32_t, 0>(a);
    return cudaErrorNotSupported;  // 32-bit advanced: bases above the series table need the serial walk
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
