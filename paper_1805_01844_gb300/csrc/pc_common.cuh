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

#ifndef PCX_THREADS
#define PCX_THREADS 256
#endif
constexpr uint32_t kThreads = PCX_THREADS;
constexpr uint32_t kWarps = kThreads / 32;
constexpr uint32_t kPad = 64;           // > largest digit count per word (63, B = 2, w = 64)
constexpr uint32_t kMaxTileBlocks = 32;  // one look-back / chain-walk lane per block
constexpr uint64_t kWaitLimitNs = 1000000000ull;  // bounded device waits: 1 s
#ifndef PCX_TILE_BUDGET_BASIC
#define PCX_TILE_BUDGET_BASIC (72u * 1024u)
#endif
#ifndef PCX_TILE_BUDGET_ADVANCED
#define PCX_TILE_BUDGET_ADVANCED (100u * 1024u)
#endif
// shared memory a tile may use; sets the blocks per tile
constexpr uint32_t kTileBudgetBasic = PCX_TILE_BUDGET_BASIC;
constexpr uint32_t kTileBudgetAdvanced = PCX_TILE_BUDGET_ADVANCED;

// Workspace: this 64-byte header, then one 64-bit look-back status word per
// tile.  A status word is (flag << 62) | value with flag 0 = not ready,
// 1 = tile aggregate, 2 = inclusive prefix, 3 = error.
struct WsHeader {
    uint32_t ticket;    // next tile to hand out (tiles are taken in order)
    uint32_t status;    // first device-side error, a pc_status; 0 = none
    uint32_t timeouts;  // bounded waits that ran out
    uint32_t orbit_cursor;  // next free slot of the series table (advanced)
    uint32_t reserved_cursor64;  // same, second table of a batch (64-bit words)
    uint32_t reserved1;
    uint64_t orbit_tag;  // series tables valid for this layout and word size (see ws_layout)
    uint64_t reserved[4];
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

// Eq. 1 (Sec. 3.1) in integer form: the largest p with B^p <= 2^w - 1,
// together with 1 + B + ... + B^(p-1) (mod 2^64), in one pass of p
// multiplications.  B >= 2, B <= 2^32, w in {32, 64}.  Below 2^32 each step
// is a 64 x 32-bit product held as 96 bits (two 32-bit multiplies), whose
// top 32 bits say whether B^(p+1) still fits 64 bits.
PCX_HD uint32_t eq1_p_geo(uint64_t B, uint32_t w, uint64_t &geo)
{
    uint64_t x = 1, g = 0;  // x = B^p, g = 1 + ... + B^(p-1)
    uint32_t p = 0;
    if (B <= 0xFFFFFFFFull) {
        const uint32_t b = (uint32_t)B;
        for (;;) {
            const uint64_t lo = (uint64_t)(uint32_t)x * b;
            const uint64_t mid = (x >> 32) * b + (lo >> 32);  // < 2^64
            const uint64_t y = (mid << 32) | (uint32_t)lo;  // x b mod 2^64
            if (w == 64 ? (mid >> 32) != 0 : y > 0xFFFFFFFFull) break;
            g += x;
            x = y;
            ++p;
        }
    } else if (w == 64) {  // B = 2^32: B^1 fits, B^2 = 2^64 does not
        g = 1;
        p = 1;
    }
    geo = g;
    return p;
}

PCX_HD uint32_t eq1_p(uint64_t B, uint32_t w)
{
    uint64_t g;
    return eq1_p_geo(B, w, g);
}

// Digits per word of the basic variant: Eq. 1 clamped to >= 1 (B = 2^32 with
// 32-bit words stores one offset per word), and its geometric sum.
PCX_HD uint32_t basic_p_geo(uint64_t B, uint32_t w, uint64_t &geo)
{
    const uint32_t p = eq1_p_geo(B, w, geo);
    if (p == 0) {
        geo = 1;
        return 1u;
    }
    return p;
}

PCX_HD uint32_t basic_p(uint64_t B, uint32_t w)
{
    uint64_t g;
    return basic_p_geo(B, w, g);
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
    uint32_t slot_bytes;  // bytes of the tile's shared memory
    uint32_t off_sched;   // within a slot: u64 [tb][wcap]: R | p << 32 | q << 40
    uint32_t off_tops;    // within a slot: u32 [tb][wcap]: decoded high parts r'_{i-1}
    uint32_t off_blk;     // within a slot: per-block scalars, see BlockVars
    uint32_t smem;        // total dynamic shared memory
};

// Basic words as 32-bit pieces (compression): a word of p digits is
// np = ceil(p / p32) pieces of p32 digits, p32 = max{k : B^k <= 2^32 - 1},
// the top one of t = p - (np - 1) p32 digits, so that each piece is a 32-bit
// Horner sum and s = ((top D + piece_{np-2}) D + ...) D + piece_0 with
// D = B^p32.  Pieces are summed over raw samples, so each subtracts
// vmin (1 + B + ... + B^(len-1)) mod 2^32: Kf for a full piece, Kt for the
// top one (the true piece is below 2^32, so the difference mod 2^32 is exact).
// 32-bit words (and B = 2^32) have one piece: p32 = t = p, np = 1.
struct PackK {
    uint32_t D, Kf, Kt;
    uint32_t shape;  // p32 | np << 8 | t << 16
};

PCX_HD PackK basic_pack_k(uint64_t B, uint32_t p, uint32_t vmin, uint32_t w)
{
    PackK r{0u, 0u, 0u, 0u};
    uint32_t p32 = p, np = 1, t = p;
    if (w == 64 && B <= 0xFFFFFFFFull) {
        uint64_t pw = 1;
        uint32_t g = 0;
        p32 = 0;
        while (pw * B <= 0xFFFFFFFFull) {  // pw <= 2^32 - 1 and B < 2^32: no overflow
            g += (uint32_t)pw;
            pw *= B;
            ++p32;
        }
        r.D = (uint32_t)pw;
        r.Kf = vmin * g;
        np = (p + p32 - 1) / p32;
        t = p - (np - 1) * p32;
    }
    uint32_t g = 0, pw = 1;  // 1 + B + ... + B^(t-1) mod 2^32
    for (uint32_t i = 0; i < t; ++i) {
        g += pw;
        pw *= (uint32_t)B;
    }
    r.Kt = vmin * g;
    r.shape = p32 | (np << 8) | (t << 16);
    return r;
}

struct BlockVars {        // per-tile arrays in shared memory
    uint64_t B[kMaxTileBlocks];
    uint32_t vmin[kMaxTileBlocks];
    uint32_t W[kMaxTileBlocks];
    uint32_t woff[kMaxTileBlocks];
    uint32_t p[kMaxTileBlocks];
    union {
        // decoding only: per-block division constants (see k_decode)
        struct {
            uint64_t Dh[kMaxTileBlocks];  // B^h*, the largest power of B <= 2^32
            uint64_t MD[kMaxTileBlocks];  // floor((2^64 - 1) / Dh)
        } dec;
        PackK pk[kMaxTileBlocks];  // compression, basic variant: the 32-bit pieces of its words
    };
    uint32_t mg_m[kMaxTileBlocks]; // magic reciprocal of B (Magic32)
    uint32_t mg_a[kMaxTileBlocks];
    uint32_t mg_s[kMaxTileBlocks];
    uint32_t hstar[kMaxTileBlocks];
    // compression only: vmin * (1 + B + ... + B^(p-1)) mod 2^w (see basic_word);
    // advanced: K for p = p_1, K2 for p = p_1 - 1
    uint64_t K[kMaxTileBlocks];
    uint64_t K2[kMaxTileBlocks];
    // advanced: per-block view of the series table (mode 1) or serial walk (mode 0)
    uint32_t mode[kMaxTileBlocks];
    uint32_t p1[kMaxTileBlocks];
    uint32_t orb_off[kMaxTileBlocks];
    uint32_t orb_Q[kMaxTileBlocks];
    uint32_t orb_P[kMaxTileBlocks];
    uint32_t orb_SQ[kMaxTileBlocks];
    uint32_t orb_G[kMaxTileBlocks];
    uint32_t orb_mgm[kMaxTileBlocks];
    uint32_t orb_mga[kMaxTileBlocks];
    uint32_t orb_mgs[kMaxTileBlocks];
    uint64_t excl;        // payload words before this tile
    uint64_t tile;        // tile index, >= n_tiles when the slot is empty
    uint32_t agg;         // payload words of this tile
    uint32_t ok;
    uint32_t bad;
    uint32_t pad_;
};

enum : uint32_t { kKernelCompress = 0, kKernelDecode = 1 };

// Tile of the compression kernel (kind 0) or of the decoding kernel (kind 1).
// Basic compression with look-back tiles of several stage tiles, four CTAs
// per SM: the stage budget that fits four (used where it still gives stage
// tiles of >= 24 blocks, see compress_tile_multi).
#ifndef PCX_TILE_BUDGET_MULTI4
#define PCX_TILE_BUDGET_MULTI4 (54u * 1024u)
#endif
constexpr uint32_t kTileBudgetMulti4 = PCX_TILE_BUDGET_MULTI4;

PCX_HD TileCfg tile_cfg(uint32_t kind, uint32_t variant, uint32_t d, uint32_t w, uint32_t L, bool orbit,
                        uint32_t nt = kThreads, uint32_t budget_override = 0)
{
    TileCfg c;
    c.S = L + kPad;
    c.stage_bytes = (uint32_t)round_up((uint64_t)c.S * (d / 8), 16);
    // the serial walk keeps a block's schedule in shared memory; with the series
    // table, 16-bit data never walks (every base is <= 65536)
    const bool walk = variant == PC_VARIANT_ADVANCED && !(orbit && d == 16);
    c.wcap = walk ? (uint32_t)words_bound(variant, d, w, L) : 0u;
    // a 128-thread CTA gets about half the shared memory of a 256-thread one
    const uint32_t budget = budget_override ? budget_override
                                            : (variant == PC_VARIANT_ADVANCED ? kTileBudgetAdvanced : kTileBudgetBasic) /
                                                  (nt <= 128 ? 2u : 1u);
    const uint32_t per_block = c.stage_bytes + c.wcap * 12u;
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
    c.slot_bytes = (uint32_t)round_up(off, 16);
    c.smem = c.slot_bytes;
    return c;
}

// Threads per CTA of the single-stream compression kernel: 128-thread CTAs
// (half-size tiles, more CTAs per SM) for basic blocks of <= 128 samples,
// where the per-tile work is small; 256 otherwise, which also gives long
// streams the look-back tiles of several stage tiles (measured on camera
// events, w = 64: L = 512 +25 %, L = 256 +3 % over 128 threads; L = 128 -9 %
// on white noise).
PCX_HD uint32_t compress_threads(uint32_t variant, uint32_t d, uint32_t w, uint32_t L)
{
    (void)d;
    (void)w;
    return variant == PC_VARIANT_BASIC && L <= 128 ? 128u : 256u;
}

// Blocks per tile of the decompression offsets kernel (one thread per block).
constexpr uint32_t kOffsetTileBlocks = kThreads;

// Short streams: with few blocks, full tiles would leave most SMs idle, so
// tiles shrink (halving while the stream has fewer than kSmallTiles tiles)
// down to one block.  Compression tiles and the decoder's warp tiles (at most
// 32 blocks each) follow the same rule; the workspace always has room for
// 2 kSmallTiles + 1 look-back words and offsets.
constexpr uint64_t kSmallTiles = 2432;  // 152 SMs x 16

PCX_HD uint32_t small_stream_tb(uint64_t n_blocks, uint32_t tb)
{
    while (tb > 1 && ceil_div(n_blocks, tb) < kSmallTiles) tb = (tb + 1) / 2;
    return tb;
}

// Warp-granular decoding: shared memory of one warp (one block's samples
// with padding and a junk area, two buffers of packed words) and the warps
// per CTA that fit a 200 KB budget (1 to 4).
constexpr uint32_t kDecChunk = 256;  // packed words staged at a time per warp (a multiple of 128)

// Long blocks (two word buffers of a whole block above 8 KB) are decoded in
// chunks of kDecChunk words, so that a warp's shared memory stays small and
// enough warps share an SM; shorter ones stage a whole block's words.
PCX_HD bool dec_chunked(uint32_t variant, uint32_t d, uint32_t w, uint32_t L)
{
    return 2 * words_bound(variant, d, w, L) * (w / 8) > 8192;
}

PCX_HD uint32_t dec_chunk_words(uint32_t variant, uint32_t d, uint32_t w, uint32_t L)
{
    return dec_chunked(variant, d, w, L) ? kDecChunk : (uint32_t)words_bound(variant, d, w, L);
}

// The warp decoder's per-block records (the decoder's DecBlock): basic
// variant, advanced variant.
constexpr uint32_t kDecRecBasic = 80;
constexpr uint32_t kDecRecAdvanced = 112;
constexpr uint32_t kDecWarpsMax = 4;  // warps per CTA of the warp decoder
// CTAs of the warp decoder per SM that its register allocation allows
#ifndef PCX_DECODE_MIN_CTAS
#define PCX_DECODE_MIN_CTAS 5
#endif
constexpr uint32_t kSmemPerSm = 228u * 1024u;  // shared memory per SM, and the part each CTA reserves
constexpr uint32_t kSmemReservedPerCta = 1024u;

PCX_HD uint32_t dec_words_bytes(uint32_t variant, uint32_t d, uint32_t w, uint32_t L)
{
    return (uint32_t)round_up(2 * (uint64_t)dec_chunk_words(variant, d, w, L) * (w / 8), 16);
}

// Short basic blocks are decoded a lane per word across the warp's whole tile
// (k_decode_w's flat path): the tile's samples are assembled in shared
// memory and leave in one run of 16-byte stores.
#ifndef PCX_DEC_FLAT_MAXL
#define PCX_DEC_FLAT_MAXL 128
#endif
PCX_HD bool dec_flat(uint32_t variant, uint32_t d, uint32_t w, uint32_t L)
{
    return variant == PC_VARIANT_BASIC && !dec_chunked(variant, d, w, L) && L <= PCX_DEC_FLAT_MAXL &&
           (L * (d / 8)) % 16 == 0;
}

// Shared memory of one warp of the warp decoder before its block records: a
// block's sample slot and two word buffers, or (flat path) the samples of a
// tile of `recs` blocks.
PCX_HD uint32_t decw_front_bytes(uint32_t variant, uint32_t d, uint32_t w, uint32_t L, uint32_t recs)
{
    const uint64_t slot = round_up((uint64_t)(L + 2 * kPad) * (d / 8), 16) + dec_words_bytes(variant, d, w, L);
    const uint64_t flat = dec_flat(variant, d, w, L) ? round_up((uint64_t)recs * L * (d / 8), 16) : 0;
    return (uint32_t)(slot > flat ? slot : flat);
}

// Shared memory of one warp of the warp decoder: the front part above, the
// records of a tile of up to `recs` blocks.
PCX_HD uint32_t decw_warp_bytes_for(uint32_t variant, uint32_t d, uint32_t w, uint32_t L, uint32_t recs)
{
    const uint64_t rec = (uint64_t)recs * (variant == PC_VARIANT_BASIC ? kDecRecBasic : kDecRecAdvanced);
    return (uint32_t)(decw_front_bytes(variant, d, w, L, recs) + rec);
}

// Warps per CTA that fit a 200 KB budget (1 to 4; 0: does not fit, which no
// parameters reach) and the warps per SM that result.
PCX_HD uint32_t decw_warps_for(uint32_t variant, uint32_t d, uint32_t w, uint32_t L, uint32_t recs)
{
    uint32_t k = (200u * 1024u) / decw_warp_bytes_for(variant, d, w, L, recs);
    return k > kDecWarpsMax ? kDecWarpsMax : k;
}

PCX_HD uint32_t decw_warps_per_sm(uint32_t variant, uint32_t d, uint32_t w, uint32_t L, uint32_t recs)
{
    const uint32_t k = decw_warps_for(variant, d, w, L, recs);
    if (k == 0) return 0;
    uint32_t ctas = kSmemPerSm / (k * decw_warp_bytes_for(variant, d, w, L, recs) + kSmemReservedPerCta);
    if (ctas > PCX_DECODE_MIN_CTAS) ctas = PCX_DECODE_MIN_CTAS;
    return ctas * k;
}

// Blocks per warp tile of the warp decoder: 32 (one lane each), or 16 where
// the records of 32 blocks would cost resident warps.
PCX_HD uint32_t dec_tile_cap(uint32_t variant, uint32_t d, uint32_t w, uint32_t L)
{
    return decw_warps_per_sm(variant, d, w, L, 32) >= decw_warps_per_sm(variant, d, w, L, 16) ? 32u : 16u;
}

PCX_HD uint32_t decw_warp_bytes(uint32_t variant, uint32_t d, uint32_t w, uint32_t L)
{
    return decw_warp_bytes_for(variant, d, w, L, dec_tile_cap(variant, d, w, L));
}

PCX_HD uint32_t decw_warps(uint32_t variant, uint32_t d, uint32_t w, uint32_t L)
{
    return decw_warps_for(variant, d, w, L, dec_tile_cap(variant, d, w, L));
}

// Workspace layout: the header; the series table (advanced with the table:
// flags, headers, slots) at fixed offsets; the look-back words; the
// decoding-tile offsets plus the total (decompression).  The table depends on
// (B, w) only, so it is kept across calls that reuse the workspace: a call
// clears the header's first words and its look-back words, and a one-CTA
// kernel clears the table's flags only when the header's tag does not name
// this layout and word size (a fresh workspace, another word size, or a call
// of another layout in between, which rewrites or clears the tag).
constexpr uint64_t kOrbitFlagsBytes = 262160;     // (65536 + 1) u32, padded to 16
constexpr uint64_t kOrbitHdrBytes = 524304;       // (65536 + 1) u64, padded to 16
constexpr uint64_t kOrbitSlotBytes = 16ull << 20; // 2^20 slots of 16 bytes
constexpr uint64_t kOrbitTagOne = 0x4F52424954310000ull;    // | w: one table, single stream
constexpr uint64_t kOrbitTagBatch = 0x4F52424954320000ull;  // two tables (w = 32, 64): batches

struct WsLayout {
    uint64_t n_status;     // look-back words
    uint64_t n_offsets;    // decoding-tile offsets
    bool orbit;            // series table present
    uint64_t off_flags, off_hdr, off_slots, off_status, off_offsets;
    uint64_t bytes;
};

PCX_HD WsLayout ws_layout(uint32_t variant, uint32_t d, uint32_t w, uint32_t L, uint64_t n, bool orbit)
{
    const uint64_t n_blocks = ceil_div(n, L);
    WsLayout lay;
    lay.orbit = orbit && variant == PC_VARIANT_ADVANCED;
    const uint32_t ctb = tile_cfg(kKernelCompress, variant, d, w, L, lay.orbit, compress_threads(variant, d, w, L)).tb;
    const uint64_t ctiles = ceil_div(n_blocks, small_stream_tb(n_blocks, ctb));
    const uint64_t otiles = ceil_div(n_blocks, kOffsetTileBlocks);
    const uint64_t dtiles_cta = ceil_div(n_blocks, tile_cfg(kKernelDecode, variant, d, w, L, lay.orbit).tb);
    const uint64_t dtiles_warp = ceil_div(n_blocks, small_stream_tb(n_blocks, dec_tile_cap(variant, d, w, L)));
    const uint64_t dtiles = dtiles_cta > dtiles_warp ? dtiles_cta : dtiles_warp;
    lay.n_status = (ctiles > otiles ? ctiles : otiles) + 1;  // + 1: the self-test uses two words
    lay.n_offsets = dtiles + 1;
    lay.off_flags = sizeof(WsHeader);
    lay.off_hdr = lay.off_flags + (lay.orbit ? kOrbitFlagsBytes : 0);
    lay.off_slots = lay.off_hdr + (lay.orbit ? kOrbitHdrBytes : 0);
    lay.off_status = lay.off_slots + (lay.orbit ? kOrbitSlotBytes : 0);
    lay.off_offsets = lay.off_status + 8 * lay.n_status;
    lay.bytes = round_up(lay.off_offsets + 8 * lay.n_offsets, 16);
    return lay;
}

PCX_HD uint64_t table_bytes(uint64_t n_blocks, uint32_t d)
{
    return round_up(n_blocks * 2u * (d / 8u), 16);
}

// ---- format version 2: segmented streams --------------------------------
// The block length and word size change along the data: segments of seg_len
// samples, each compressed blockwise with its own (L, w).  After the 64-byte
// header (version 2; u32 seg_len at byte 12, then u64 n_samples, n_segments,
// body_bytes) come one code byte per segment (log2 L | (w == 64) << 7), then
// one u32 body size per segment in units of 8 bytes, each array zero-padded
// to a multiple of 8 bytes, then the bodies: the segment's block table
// (vmin, B - 1) zero-padded to 8 bytes, then its packed words zero-padded to
// 8 bytes.  The stored sizes let every segment be found by a prefix sum.
constexpr uint32_t kV2MaxLog2L = 13;     // L <= 8192
constexpr uint32_t kV2TileSegs = 256;    // segments per look-back tile of the v2 kernels
constexpr uint64_t kOrbitTagV2 = 0x4F52424954330000ull;  // two tables (w = 32, 64): v2 decoding

PCX_HD uint64_t round8(uint64_t x) { return (x + 7) / 8 * 8; }
PCX_HD bool v2_code_ok(uint32_t c) { return (c & 0x60u) == 0 && (c & 0x1Fu) <= kV2MaxLog2L; }
PCX_HD uint32_t v2_L(uint32_t c) { return 1u << (c & 0x1Fu); }
PCX_HD uint32_t v2_w(uint32_t c) { return (c & 0x80u) ? 64u : 32u; }

struct V2Geom {
    uint64_t sizes_at, bodies_at;
};
PCX_HD V2Geom v2_geom(uint64_t n_seg)
{
    V2Geom g;
    g.sizes_at = PC_HEADER_BYTES + round8(n_seg);
    g.bodies_at = g.sizes_at + round8(4 * n_seg);
    return g;
}

// Workspace of the v2 kernels: the header, (advanced decoding) two series
// tables laid out as a batch's, look-back words per tile of kV2TileSegs
// segments, and (decoding) one body offset per segment.
struct V2Layout {
    uint64_t off_flags32, off_flags64, off_hdr32, off_slots32, off_hdr64, off_slots64;
    uint64_t off_status, n_status, off_offsets, n_offsets, bytes;
};
PCX_HD V2Layout v2_layout(bool tables, bool offsets, uint64_t max_segments)
{
    V2Layout l;
    l.off_flags32 = sizeof(WsHeader);
    l.off_flags64 = l.off_flags32 + (tables ? kOrbitFlagsBytes : 0);
    l.off_hdr32 = l.off_flags64 + (tables ? kOrbitFlagsBytes : 0);
    l.off_slots32 = l.off_hdr32 + (tables ? kOrbitHdrBytes : 0);
    l.off_hdr64 = l.off_slots32 + (tables ? kOrbitSlotBytes : 0);
    l.off_slots64 = l.off_hdr64 + (tables ? kOrbitHdrBytes : 0);
    l.off_status = l.off_slots64 + (tables ? kOrbitSlotBytes : 0);
    l.n_status = (max_segments + kV2TileSegs - 1) / kV2TileSegs + 1;
    l.off_offsets = l.off_status + 8 * l.n_status;
    l.n_offsets = offsets ? max_segments + 1 : 0;
    l.bytes = round_up(l.off_offsets + 8 * l.n_offsets, 16);
    return l;
}

// Segments path (learned chooser): the device copy of a pc_source plus the
// index of its first segment among all sources' segments.  An empty source
// owns no segment.
struct SourceDev {
    const void *in;
    uint64_t n;
    void *out;
    uint64_t *out_bytes;
    uint64_t seg_first;
    uint64_t *totals;
};
static_assert(sizeof(SourceDev) == 48, "source descriptors are 48 bytes");

// Option o = 2 i + j of the chooser: block length 128 << i, word size 32 / 64.
PCX_HD uint32_t option_block_len(uint32_t o) { return 128u << (o >> 1); }
PCX_HD uint32_t option_word_bits(uint32_t o) { return (o & 1u) ? 64u : 32u; }

// The source owning global segment k: the largest i with seg_first <= k
// (empty sources share their successor's seg_first and precede it, so they
// are never picked).
PCX_HD uint32_t source_of(const SourceDev *src, uint32_t n_src, uint64_t k)
{
    uint32_t lo = 0, hi = n_src - 1;
    while (lo < hi) {
        const uint32_t mid = (lo + hi + 1) >> 1;
        if (src[mid].seg_first <= k) lo = mid;
        else hi = mid - 1;
    }
    return lo;
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
    // (x m + a) >> (32 + s), taken as the high word shifted by s (s <= 31):
    // a 32-bit shift instead of a variable 64-bit one
    const uint64_t t = (uint64_t)x * mg.m + mg.a;
    return (uint32_t)(t >> 32) >> mg.s;
}

}  // namespace pcx

namespace pcx {

// ---- sharding (Sec. 3.3: blocks are independent) -------------------------
// Shard k of K of n_blocks blocks: the first n_blocks % K shards get one
// block more than the others.
PCX_HD void shard_blocks(uint64_t n_blocks, uint32_t K, uint32_t k, uint64_t &first, uint64_t &count)
{
    const uint64_t q = n_blocks / K, r = n_blocks % K;
    first = (uint64_t)k * q + (k < r ? (uint64_t)k : r);
    count = q + (k < r ? 1u : 0u);
}

// Placement of shard k's pieces in the whole stream from every shard's stream
// size (host or device memory): the exclusive prefix of the shards' payload
// words.  Returns PC_OK, or PC_ERR_CORRUPT if a size is not a header, a table
// of that shard's blocks and whole words.
PCX_HD uint32_t stitch_region(uint32_t d, uint32_t w, uint32_t L, uint64_t n, uint32_t K, uint32_t k,
                              const uint64_t *shard_bytes, pc_stitch_region &r)
{
    const uint64_t NB = ceil_div(n, L), E = 2u * (d / 8u), WBY = w / 8u;
    uint64_t before = 0, total = 0, mine = 0;
    for (uint32_t j = 0; j < K; ++j) {
        uint64_t f, c;
        shard_blocks(NB, K, j, f, c);
        const uint64_t head = PC_HEADER_BYTES + table_bytes(c, d), sz = shard_bytes[j];
        if (sz < head || (sz - head) % WBY != 0) return PC_ERR_CORRUPT;
        const uint64_t pw = (sz - head) / WBY;
        if (j < k) before += pw;
        if (j == k) mine = pw;
        total += pw;
    }
    uint64_t first, count;
    shard_blocks(NB, K, k, first, count);
    r.first_block = first;
    r.n_blocks = count;
    r.payload_start = PC_HEADER_BYTES + table_bytes(NB, d);
    r.total_bytes = r.payload_start + total * WBY;
    r.table_src = PC_HEADER_BYTES;
    r.table_dst = PC_HEADER_BYTES + first * E;
    r.table_bytes = count * E;
    r.payload_src = PC_HEADER_BYTES + table_bytes(count, d);
    r.payload_dst = r.payload_start + before * WBY;
    r.payload_bytes = mine * WBY;
    r.pad_dst = PC_HEADER_BYTES + NB * E;
    return PC_OK;
}

}  // namespace pcx
