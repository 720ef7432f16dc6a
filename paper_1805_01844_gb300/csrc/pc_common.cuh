// pc_common.cuh -- definitions shared by the host API and the sm_103a kernels
// of the polynomial compression library (arXiv:1805.01844).
//
// Tiles: a CTA of kThreads threads processes a tile of `tb` consecutive
// blocks.  The tile's samples are staged in shared memory, one slot of
// S = block_len + kPad samples per block; the kPad samples after each block
// are filled with the block minimum so that digits past the end of a block
// read as offset 0 (the zero padding of the last word, Eq. 2 and Sec. 3.2)
// without a bounds test in the packing loops.
#pragma once

#include <cstdint>

#include "pc.h"

#if defined(__CUDACC__)
#define PCX_HD __host__ __device__ __forceinline__
#else
#define PCX_HD inline
#endif

namespace pcx {

constexpr uint32_t kThreads = 256;
constexpr uint32_t kWarps = kThreads / 32;
constexpr uint32_t kPad = 64;           // > largest digit count per word (63, B = 2, w = 64)
constexpr uint32_t kMaxTileBlocks = 32;  // one look-back / chain-walk lane per block
constexpr uint64_t kWaitLimitNs = 1000000000ull;  // bounded device waits: 1 s

// Workspace: this 64-byte header, then one 64-bit look-back status word per
// tile.  A status word is (flag << 62) | value with flag 0 = not ready,
// 1 = tile aggregate, 2 = inclusive prefix, 3 = error.
struct WsHeader {
    uint32_t ticket;    // next tile to hand out (tiles are taken in order)
    uint32_t status;    // first device-side error, a pc_status; 0 = none
    uint32_t timeouts;  // bounded waits that ran out
    uint32_t reserved0;
    uint64_t reserved[6];
};
static_assert(sizeof(WsHeader) == 64, "workspace header is 64 bytes");

constexpr uint64_t kFlagAgg = 1ull << 62;
constexpr uint64_t kFlagPrefix = 2ull << 62;
constexpr uint64_t kFlagError = 3ull << 62;
constexpr uint64_t kValueMask = (1ull << 62) - 1;

PCX_HD uint64_t ceil_div(uint64_t a, uint64_t b) { return (a + b - 1) / b; }
PCX_HD uint64_t umin64(uint64_t a, uint64_t b) { return a < b ? a : b; }
PCX_HD uint64_t round_up(uint64_t a, uint64_t m) { return (a + m - 1) / m * m; }

PCX_HD uint64_t mulhi64(uint64_t a, uint64_t b)
{
#if defined(__CUDA_ARCH__)
    return __umul64hi(a, b);
#else
    return (uint64_t)(((unsigned __int128)a * b) >> 64);
#endif
}

// Eq. 1 (Sec. 3.1) in integer form: the largest p with B^p <= 2^w - 1.
// B >= 2, B <= 2^32, w in {32, 64}.
PCX_HD uint32_t eq1_p(uint64_t B, uint32_t w)
{
    uint64_t x = 1;
    uint32_t p = 0;
    for (;;) {
        if (w == 64) {
            if (mulhi64(x, B) != 0) break;
            x *= B;
        } else {
            uint64_t y = x * B;  // x < 2^32, B <= 2^32: no overflow
            if (y > 0xFFFFFFFFull) break;
            x = y;
        }
        ++p;
    }
    return p;
}

// Digits per word of the basic variant: Eq. 1 clamped to >= 1 (B = 2^32 with
// 32-bit words stores one offset per word).
PCX_HD uint32_t basic_p(uint64_t B, uint32_t w)
{
    uint32_t p = eq1_p(B, w);
    return p == 0 ? 1u : p;
}

// Largest word count of a block of n_b samples over every base B in
// [1, 2^d].  Basic: ceil(n_b / p(2^d)).  Advanced: each word consumes
// p_i + 1 >= p_1(B) >= p_1(2^d) samples (p_i is p_1 or p_1 - 1), and the last
// word is the first whose split slot lies past the end, hence at most
// ceil((n_b + 1) / max(1, p_1(2^d))) words.
PCX_HD uint64_t words_bound(uint32_t variant, uint32_t d, uint32_t w, uint64_t n_b)
{
    if (n_b == 0) return 0;
    uint64_t Bmax = 1ull << d;
    uint32_t p = eq1_p(Bmax, w);
    if (p == 0) p = 1;
    return variant == PC_VARIANT_BASIC ? ceil_div(n_b, p) : ceil_div(n_b + 1, p);
}

// Shared-memory layout of one tile (identical on host and device).
struct TileCfg {
    uint32_t tb;          // blocks per tile
    uint32_t S;           // staged samples per block (block_len + kPad)
    uint32_t stage_bytes; // bytes per staged block (multiple of 16)
    uint32_t wcap;        // schedule entries per block (advanced), else 0
    uint32_t off_sched;   // u64 [tb][wcap]: R | p << 32 | q << 40
    uint32_t off_tops;    // u32 [tb][wcap]: decoded high parts r'_{i-1}
    uint32_t off_blk;     // per-block scalars, see BlockVars
    uint32_t smem;        // total dynamic shared memory
};

struct BlockVars {        // per-tile arrays in shared memory
    uint64_t B[kMaxTileBlocks];
    uint32_t vmin[kMaxTileBlocks];
    uint32_t W[kMaxTileBlocks];
    uint32_t woff[kMaxTileBlocks];
    uint32_t p[kMaxTileBlocks];
    uint64_t excl;        // payload words before this tile
    uint32_t tile;
    uint32_t ok;
    uint32_t bad;
    uint32_t pad_[3];
};

PCX_HD TileCfg tile_cfg(uint32_t variant, uint32_t d, uint32_t w, uint32_t L)
{
    TileCfg c;
    c.S = L + kPad;
    c.stage_bytes = (uint32_t)round_up((uint64_t)c.S * (d / 8), 16);
    c.wcap = variant == PC_VARIANT_ADVANCED ? (uint32_t)words_bound(variant, d, w, L) : 0u;
    uint32_t per_block = c.stage_bytes + c.wcap * 12u;
    uint32_t budget = variant == PC_VARIANT_ADVANCED ? 96u * 1024u : 64u * 1024u;
    uint32_t tb = budget / per_block;
    if (tb < 1) tb = 1;
    if (tb > kMaxTileBlocks) tb = kMaxTileBlocks;
    if (tb >= 8) tb &= ~7u;  // keeps every tile 16-byte aligned in global memory
    c.tb = tb;
    uint32_t off = tb * c.stage_bytes;
    c.off_sched = off;
    off += tb * c.wcap * 8u;
    c.off_tops = off;
    off += tb * c.wcap * 4u;
    off = (uint32_t)round_up(off, 16);
    c.off_blk = off;
    off += (uint32_t)sizeof(BlockVars);
    c.smem = (uint32_t)round_up(off, 16);
    return c;
}

PCX_HD uint64_t table_bytes(uint64_t n_blocks, uint32_t d)
{
    return round_up(n_blocks * 2u * (d / 8u), 16);
}

// Division of a 32-bit x by an invariant d >= 2 without a divide instruction:
// q = (x * m + a) >> (32 + s).  Power of two d = 2^k: m = 2^(32-k), a = 0,
// s = 0.  Otherwise s = floor(log2 d) and m = ceil(2^(32+s) / d) when
// m d - 2^(32+s) <= 2^s (round-up method, Granlund & Montgomery 1994,
// Thm. 4.2), else m = floor(2^(32+s) / d) with a = m (round-down method with
// increment, Robison 2005).  Both are exact for every x < 2^32.
struct Magic32 {
    uint32_t m;
    uint32_t a;
    uint32_t s;
};

PCX_HD Magic32 magic32(uint64_t d)
{
    Magic32 r;
    if ((d & (d - 1)) == 0) {  // d = 2^k, 1 <= k <= 32
        uint32_t k = 0;
        while ((1ull << k) < d) ++k;
        r.m = (uint32_t)(1ull << (32 - k));
        r.a = 0;
        r.s = 0;
        if (k == 0) { r.m = 0xFFFFFFFFu; r.a = 0xFFFFFFFFu; }  // d = 1: (x+1)(2^32-1) >> 32 = x
        return r;
    }
    uint32_t l = 0;
    while ((2ull << l) <= d) ++l;  // 2^l < d < 2^(l+1)
    uint64_t two = 1ull << (32 + l);
    uint64_t up = two / d + 1;  // ceil, d does not divide 2^(32+l)
    uint64_t e = up * d - two;
    if (e <= (1ull << l)) {
        r.m = (uint32_t)up;
        r.a = 0;
    } else {
        r.m = (uint32_t)(up - 1);
        r.a = r.m;
    }
    r.s = l;
    return r;
}

PCX_HD uint32_t magic_div(uint32_t x, Magic32 mg)
{
    return (uint32_t)(((uint64_t)x * mg.m + mg.a) >> (32 + mg.s));
}

}  // namespace pcx
