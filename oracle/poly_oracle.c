/*
 * poly_oracle.c -- plain, slow, obviously-correct CPU oracle for polynomial
 * lossless compression (Aubert et al., "Polynomial data compression for
 * large-scale physics experiments", arXiv:1805.01844).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may link or call
 * this file: only the test suite, the smoke check and the benchmark's CPU
 * baseline / reference legs use it.  It shares no code, header, table or
 * constant with the CUDA implementation.
 *
 * Every arithmetic step is written in the order the paper gives it, with
 * unsigned __int128 intermediates so that no product can overflow.  There is
 * no blocking, fusion or reordering beyond what the method itself states.
 *
 * What it computes, with the passage each function follows:
 *   po_eq1_p        -- Sec. 3.1, Eq. 1: number of base-B digits per word,
 *                      integer form p = max{p : B^p <= 2^w - 1}.
 *   po_basic_*      -- Sec. 3.1, Eq. 2: s_j = sum_i v_{i+p(j-1)} B^{i-1}
 *                      (first value in the lowest power), decoded by
 *                      polynomial division.
 *   po_adv_*        -- Sec. 3.2, Eqs. 3-11 and the series for the whole
 *                      vector: split base R_i * R'_i >= B, word
 *                      s_i = r_i + R_i (sum_k v_{q_i+k} B^{p_i-k} + r'_{i-1} B^{p_i}).
 *   po_compress /
 *   po_decompress   -- Sec. 3.3 (blocked compression) and Fig. 2 (minimum
 *                      then base stored once per block, then the packed data).
 *   po_*_v2         -- the same blocked compression with the block length
 *                      and word size chosen per segment of the data (the
 *                      block-size choice of Sec. 3.3 and Sec. 4.2, Fig. 7),
 *                      one code byte per segment (format version 2).
 *
 * Readings where the paper is silent or garbled (each is listed in the design
 * notes of the repository):
 *   - capacity constant: 2^w - 1 with w in {32, 64} replaces 2^32 - 1;
 *     p is computed with integers, never with a floating-point logarithm.
 *   - basic variant: p is clamped to >= 1 (only B = 2^32 with w = 32 hits it;
 *     an offset < 2^32 then occupies one word by itself).
 *   - B == 1: a block is stored with zero payload words.
 *   - the range 1 <= j < n/p of Eq. 2 is read as j = 1..ceil(n_b/p); missing
 *     digits of the last word are 0 (both variants).
 *   - advanced series, index reading: word i holds, from the most significant
 *     end, the high part r'_{i-1} of the element split off word i-1, then p_i
 *     whole elements (first element at the highest power), then the low part
 *     r_i of the next element.  q_i counts the elements before word i's whole
 *     digits: q_1 = 0, q_{i+1} = q_i + p_i + 1.  The vector ends with the
 *     first word whose split slot lies past the end (that slot is 0).
 *   - base stored as B - 1 (B = 2^d does not fit in d bits).
 */
#include <stdint.h>
#include <stddef.h>
#include <string.h>
#include <stdlib.h>

typedef unsigned __int128 u128;

enum {
    PO_OK = 0,
    PO_ERR_INVALID_ARG = 1,
    PO_ERR_CAPACITY = 2,
    PO_ERR_CORRUPT = 3,
    PO_ERR_UNSUPPORTED = 6
};

#define PO_HEADER_BYTES 64u

/* ---------------------------------------------------------------- Eq. 1 -- */

/* C = 2^w - 1, the largest value one packed word can hold. */
static u128 po_capacity(unsigned w) { return (((u128)1) << w) - 1; }

/* Eq. 1 in integer form: the largest p >= 0 with B^p <= 2^w - 1.
 * B >= 2, 1 <= w <= 64, B <= 2^33 (so that B^p * B never leaves 128 bits). */
unsigned po_eq1_p(uint64_t B, unsigned w)
{
    u128 C = po_capacity(w);
    u128 power = 1; /* B^p */
    unsigned p = 0;
    while (power * (u128)B <= C) {
        power *= (u128)B;
        p += 1;
    }
    return p;
}

/* ------------------------------------------------------ basic, Eq. 2 ----- */

/* digits per word of the basic variant (Eq. 1, clamped to >= 1) */
static unsigned po_basic_p(uint64_t B, unsigned w)
{
    unsigned p = po_eq1_p(B, w);
    return p == 0 ? 1u : p;
}

/* number of packed words for a block of n_b offsets in base B */
uint64_t po_basic_count(uint64_t B, unsigned w, uint64_t n_b)
{
    if (B <= 1 || n_b == 0) return 0;
    uint64_t p = po_basic_p(B, w);
    return (n_b + p - 1) / p;
}

/* Eq. 2: word j (0-based) = sum_{i=0}^{p-1} u[j p + i] * B^i. */
uint64_t po_basic_pack(uint64_t B, unsigned w, const uint64_t *u, uint64_t n_b,
                       uint64_t *words)
{
    uint64_t W = po_basic_count(B, w, n_b);
    if (W == 0) return 0;
    uint64_t p = po_basic_p(B, w);
    for (uint64_t j = 0; j < W; ++j) {
        u128 s = 0;
        u128 power = 1; /* B^i */
        for (uint64_t i = 0; i < p; ++i) {
            uint64_t idx = j * p + i;
            uint64_t digit = idx < n_b ? u[idx] : 0;
            s += (u128)digit * power;
            power *= (u128)B;
        }
        words[j] = (uint64_t)s;
    }
    return W;
}

/* Polynomial division: digit i of word j is (s div B^i) mod B.  A word is
 * rejected if it is not the image of valid digits: s >= B^k where k is the
 * number of real (non-padding) digits it holds. */
int po_basic_unpack(uint64_t B, unsigned w, const uint64_t *words, uint64_t n_words,
                    uint64_t n_b, uint64_t *u)
{
    if (B <= 1) {
        if (n_words != 0) return PO_ERR_CORRUPT;
        for (uint64_t i = 0; i < n_b; ++i) u[i] = 0;
        return PO_OK;
    }
    uint64_t W = po_basic_count(B, w, n_b);
    if (n_words != W) return PO_ERR_CORRUPT;
    uint64_t p = po_basic_p(B, w);
    for (uint64_t j = 0; j < W; ++j) {
        u128 s = words[j];
        uint64_t k = n_b - j * p < p ? n_b - j * p : p; /* real digits */
        u128 limit = 1;
        for (uint64_t i = 0; i < k; ++i) limit *= (u128)B;
        if (s >= limit) return PO_ERR_CORRUPT;
        for (uint64_t i = 0; i < k; ++i) {
            u[j * p + i] = (uint64_t)(s % B);
            s /= B;
        }
    }
    return PO_OK;
}

/* -------------------------------------------- advanced, Sec. 3.2 --------- */

/* One step of the split-base series (the unnumbered system after Eq. 11):
 *   p_i  = max{p : R'_{i-1} B^p <= C}          (floor((ln C - ln R'_{i-1}) / ln B))
 *   R_i  = floor(C / (R'_{i-1} B^{p_i}))
 *   R'_i = ceil(B / R_i)
 * Rprev is R'_{i-1} (R'_0 = 1). */
static void po_adv_step(uint64_t B, unsigned w, uint64_t Rprev,
                        unsigned *p_i, uint64_t *R_i, uint64_t *Rp_i)
{
    u128 C = po_capacity(w);
    u128 denom = Rprev; /* R'_{i-1} B^p */
    unsigned p = 0;
    while (denom * (u128)B <= C) {
        denom *= (u128)B;
        p += 1;
    }
    u128 R = C / denom;
    *p_i = p;
    *R_i = (uint64_t)R;
    *Rp_i = (uint64_t)(((u128)B + R - 1) / R);
}

/* Schedule of a block: per word i (0-based here) its p_i, R_i, R'_i and q_i.
 * Returns the number of words; fills at most `cap` entries (pointers may be
 * NULL to only count). */
uint64_t po_adv_schedule(uint64_t B, unsigned w, uint64_t n_b,
                         uint32_t *p_out, uint64_t *R_out, uint64_t *Rp_out,
                         uint64_t *q_out, uint64_t cap)
{
    if (B <= 1 || n_b == 0) return 0;
    uint64_t Rprev = 1; /* R'_0 */
    uint64_t q = 0;     /* elements before this word's whole digits */
    uint64_t i = 0;
    for (;;) {
        unsigned p;
        uint64_t R, Rp;
        po_adv_step(B, w, Rprev, &p, &R, &Rp);
        if (i < cap) {
            if (p_out) p_out[i] = p;
            if (R_out) R_out[i] = R;
            if (Rp_out) Rp_out[i] = Rp;
            if (q_out) q_out[i] = q;
        }
        i += 1;
        uint64_t split = q + p; /* index of the element split by this word */
        if (split >= n_b) break; /* the split slot is padding: last word */
        q = split + 1;
        Rprev = Rp;
    }
    return i;
}

uint64_t po_adv_count(uint64_t B, unsigned w, uint64_t n_b)
{
    return po_adv_schedule(B, w, n_b, NULL, NULL, NULL, NULL, 0);
}

/* s_i = r_i + R_i * ( sum_{k=1}^{p_i} v_{q_i+k} B^{p_i-k} + r'_{i-1} B^{p_i} )
 * with the split element e = v_{q_i+p_i+1} (1-based), r'_i = e div R_i,
 * r_i = e - r'_i R_i.  Elements past n_b are 0. */
uint64_t po_adv_pack(uint64_t B, unsigned w, const uint64_t *u, uint64_t n_b,
                     uint64_t *words)
{
    if (B <= 1 || n_b == 0) return 0;
    uint64_t Rprev = 1;  /* R'_{i-1} */
    uint64_t rpprev = 0; /* r'_{i-1} */
    uint64_t q = 0;
    uint64_t i = 0;
    for (;;) {
        unsigned p;
        uint64_t R, Rp;
        po_adv_step(B, w, Rprev, &p, &R, &Rp);
        /* sum_{k=1}^{p} v_{q+k} B^{p-k}, 0-based element q+k-1 */
        u128 body = 0;
        for (unsigned k = 1; k <= p; ++k) {
            uint64_t idx = q + k - 1;
            uint64_t digit = idx < n_b ? u[idx] : 0;
            u128 power = 1;
            for (unsigned e = 0; e < p - k; ++e) power *= (u128)B;
            body += (u128)digit * power;
        }
        u128 top = 1;
        for (unsigned e = 0; e < p; ++e) top *= (u128)B;
        body += (u128)rpprev * top;
        uint64_t split = q + p;
        uint64_t e_split = split < n_b ? u[split] : 0;
        uint64_t rp = e_split / R;
        uint64_t r = e_split - rp * R;
        u128 s = (u128)r + (u128)R * body;
        words[i] = (uint64_t)s;
        i += 1;
        if (split >= n_b) break;
        q = split + 1;
        Rprev = Rp;
        rpprev = rp;
    }
    return i;
}

/* Inverse of po_adv_pack.  Rejects any word that is not the image of valid
 * digits: a top part r'_{i-1} >= R'_{i-1}, a re-joined split element >= B, a
 * non-zero padding digit, or a non-zero low part in a padding split slot. */
int po_adv_unpack(uint64_t B, unsigned w, const uint64_t *words, uint64_t n_words,
                  uint64_t n_b, uint64_t *u)
{
    if (B <= 1) {
        if (n_words != 0) return PO_ERR_CORRUPT;
        for (uint64_t i = 0; i < n_b; ++i) u[i] = 0;
        return PO_OK;
    }
    if (n_words != po_adv_count(B, w, n_b)) return PO_ERR_CORRUPT;
    uint64_t Rprev = 1;
    uint64_t Rlast = 1;  /* R_{i-1} */
    uint64_t rlast = 0;  /* r_{i-1} */
    uint64_t q = 0;
    for (uint64_t i = 0; i < n_words; ++i) {
        unsigned p;
        uint64_t R, Rp;
        po_adv_step(B, w, Rprev, &p, &R, &Rp);
        u128 s = words[i];
        uint64_t r = (uint64_t)(s % R);
        u128 body = s / R;
        /* whole digits, least significant first = last element first */
        for (unsigned k = p; k >= 1; --k) {
            uint64_t digit = (uint64_t)(body % B);
            body /= B;
            uint64_t idx = q + k - 1;
            if (idx < n_b) u[idx] = digit;
            else if (digit != 0) return PO_ERR_CORRUPT;
        }
        /* what is left is r'_{i-1}, the high part of the element split off
         * the previous word */
        if (body >= (u128)Rprev) return PO_ERR_CORRUPT;
        if (i > 0) {
            u128 e = body * (u128)Rlast + rlast;
            if (e >= (u128)B) return PO_ERR_CORRUPT;
            u[q - 1] = (uint64_t)e;
        }
        uint64_t split = q + p;
        if (split >= n_b) {
            if (r != 0) return PO_ERR_CORRUPT;
            if (i + 1 != n_words) return PO_ERR_CORRUPT;
            break;
        }
        q = split + 1;
        Rprev = Rp;
        Rlast = R;
        rlast = r;
    }
    return PO_OK;
}

/* ------------------------------------------ blocked stream, Sec. 3.3 ----- */

/* Stream layout (all little-endian):
 *   header, 64 bytes:  "PCMP", u16 version = 1, u8 variant, u8 dtype_bits,
 *                      u8 word_bits, 3 zero bytes, u32 block_len,
 *                      u64 n_samples, u64 n_blocks, u64 payload_words,
 *                      24 zero bytes
 *   block table:       per block (vmin, B - 1), each a dtype_bits field,
 *                      zero-padded to a multiple of 16 bytes
 *   payload:           per block, its packed words (word_bits each)       */

static void put_le(uint8_t *dst, uint64_t v, unsigned nbytes)
{
    for (unsigned i = 0; i < nbytes; ++i) dst[i] = (uint8_t)(v >> (8 * i));
}

static uint64_t get_le(const uint8_t *src, unsigned nbytes)
{
    uint64_t v = 0;
    for (unsigned i = 0; i < nbytes; ++i) v |= (uint64_t)src[i] << (8 * i);
    return v;
}

static uint64_t po_count(unsigned variant, uint64_t B, unsigned w, uint64_t n_b)
{
    return variant == 0 ? po_basic_count(B, w, n_b) : po_adv_count(B, w, n_b);
}

static int po_params_ok(unsigned variant, unsigned d, unsigned w, uint64_t L)
{
    return (variant == 0 || variant == 1) && (d == 16 || d == 32) &&
           (w == 32 || w == 64) && L >= 1 && L <= 0xFFFFFFFFull;
}

static uint64_t po_table_bytes(uint64_t n_blocks, unsigned d)
{
    uint64_t t = n_blocks * 2 * (d / 8);
    return (t + 15) / 16 * 16;
}

/* Worst-case stream size for n samples: every block at its largest word count
 * over all B in [1, 2^d]. */
int po_bound(unsigned variant, unsigned d, unsigned w, uint64_t L, uint64_t n,
             uint64_t *max_bytes)
{
    if (!po_params_ok(variant, d, w, L)) return PO_ERR_INVALID_ARG;
    uint64_t n_blocks = (n + L - 1) / L;
    uint64_t total = PO_HEADER_BYTES + po_table_bytes(n_blocks, d);
    /* per block length class: full blocks and the last one */
    uint64_t Bmax = (uint64_t)1 << d;
    uint64_t pmin = variant == 0 ? po_basic_p(Bmax, w) : po_eq1_p(Bmax, w);
    for (int last = 0; last < 2; ++last) {
        uint64_t nb, count;
        if (n_blocks == 0) break;
        if (!last) { nb = L; count = n_blocks - 1; }
        else { nb = n - (n_blocks - 1) * L; count = 1; }
        if (count == 0) continue;
        /* basic: ceil(n_b/p) is largest at the largest B.  advanced: every word
         * consumes at least p_1(B) >= p_1(2^d) elements (p_i >= p_1 - 1 plus
         * the split slot), hence at most ceil((n_b + 1) / p_1) words, or
         * n_b + 1 words when p_1 = 0. */
        uint64_t Wb;
        if (variant == 0) Wb = (nb + pmin - 1) / pmin;
        else Wb = pmin == 0 ? nb + 1 : (nb + 1 + pmin - 1) / pmin;
        total += count * Wb * (w / 8);
    }
    *max_bytes = total;
    return PO_OK;
}

uint64_t po_stream_bytes(unsigned d, unsigned w, uint64_t n_blocks, uint64_t payload_words)
{
    return PO_HEADER_BYTES + po_table_bytes(n_blocks, d) + payload_words * (w / 8);
}

int po_compress(const void *in, uint64_t n, unsigned variant, unsigned d, unsigned w,
                uint64_t L, uint8_t *out, uint64_t cap, uint64_t *out_bytes)
{
    if (!po_params_ok(variant, d, w, L)) return PO_ERR_INVALID_ARG;
    uint64_t bound;
    po_bound(variant, d, w, L, n, &bound);
    if (cap < bound) return PO_ERR_CAPACITY;
    uint64_t n_blocks = (n + L - 1) / L;
    unsigned db = d / 8, wb = w / 8;
    uint64_t table_off = PO_HEADER_BYTES;
    uint64_t payload_off = table_off + po_table_bytes(n_blocks, d);
    memset(out, 0, payload_off);

    uint64_t payload_words = 0;
    /* scratch for one block: offsets and packed words (at most n_b + 1) */
    uint64_t *u = (uint64_t *)malloc((L + 2) * sizeof(uint64_t));
    uint64_t *words = (uint64_t *)malloc((L + 2) * sizeof(uint64_t));
    if (!u || !words) { free(u); free(words); return PO_ERR_INVALID_ARG; }

    for (uint64_t b = 0; b < n_blocks; ++b) {
        uint64_t start = b * L;
        uint64_t n_b = n - start < L ? n - start : L;
        /* Sec. 3.1: minimum and maximum of the block */
        uint64_t vmin = UINT64_MAX, vmax = 0;
        for (uint64_t i = 0; i < n_b; ++i) {
            uint64_t v = d == 16 ? ((const uint16_t *)in)[start + i]
                                 : ((const uint32_t *)in)[start + i];
            if (v < vmin) vmin = v;
            if (v > vmax) vmax = v;
        }
        uint64_t B = vmax - vmin + 1; /* base B = vmax - vmin + 1 */
        for (uint64_t i = 0; i < n_b; ++i) {
            uint64_t v = d == 16 ? ((const uint16_t *)in)[start + i]
                                 : ((const uint32_t *)in)[start + i];
            u[i] = v - vmin; /* offsets in [0, B) */
        }
        /* Fig. 2: the minimum, then the base, stored once per block */
        put_le(out + table_off + b * 2 * db, vmin, db);
        put_le(out + table_off + b * 2 * db + db, B - 1, db);
        uint64_t W = variant == 0 ? po_basic_pack(B, w, u, n_b, words)
                                  : po_adv_pack(B, w, u, n_b, words);
        for (uint64_t j = 0; j < W; ++j)
            put_le(out + payload_off + (payload_words + j) * wb, words[j], wb);
        payload_words += W;
    }
    /* header */
    memcpy(out, "PCMP", 4);
    put_le(out + 4, 1, 2);
    out[6] = (uint8_t)variant;
    out[7] = (uint8_t)d;
    out[8] = (uint8_t)w;
    put_le(out + 12, L, 4);
    put_le(out + 16, n, 8);
    put_le(out + 24, n_blocks, 8);
    put_le(out + 32, payload_words, 8);
    *out_bytes = payload_off + payload_words * wb;
    free(u);
    free(words);
    return PO_OK;
}

/* Header fields, for tests. */
int po_read_header(const uint8_t *in, uint64_t in_bytes, unsigned *variant, unsigned *d,
                   unsigned *w, uint64_t *L, uint64_t *n, uint64_t *n_blocks,
                   uint64_t *payload_words)
{
    if (in_bytes < PO_HEADER_BYTES) return PO_ERR_CORRUPT;
    if (memcmp(in, "PCMP", 4) != 0) return PO_ERR_CORRUPT;
    if (get_le(in + 4, 2) != 1) return PO_ERR_CORRUPT;
    for (unsigned i = 9; i < 12; ++i) if (in[i] != 0) return PO_ERR_CORRUPT;
    for (unsigned i = 40; i < 64; ++i) if (in[i] != 0) return PO_ERR_CORRUPT;
    *variant = in[6];
    *d = in[7];
    *w = in[8];
    *L = get_le(in + 12, 4);
    *n = get_le(in + 16, 8);
    *n_blocks = get_le(in + 24, 8);
    *payload_words = get_le(in + 32, 8);
    if (!po_params_ok(*variant, *d, *w, *L)) return PO_ERR_CORRUPT;
    if (*n_blocks != (*n + *L - 1) / *L) return PO_ERR_CORRUPT;
    return PO_OK;
}

int po_decompress(const uint8_t *in, uint64_t in_bytes, void *out, uint64_t cap,
                  uint64_t *n_out)
{
    unsigned variant, d, w;
    uint64_t L, n, n_blocks, payload_words;
    *n_out = 0;
    int st = po_read_header(in, in_bytes, &variant, &d, &w, &L, &n, &n_blocks,
                            &payload_words);
    if (st != PO_OK) return st;
    if (n > cap) return PO_ERR_CAPACITY;
    unsigned db = d / 8, wb = w / 8;
    uint64_t table_off = PO_HEADER_BYTES;
    /* the table must fit before any of it is read */
    if (n_blocks > (in_bytes - table_off) / (2 * db)) return PO_ERR_CORRUPT;
    uint64_t payload_off = table_off + po_table_bytes(n_blocks, d);
    if (payload_off > in_bytes) return PO_ERR_CORRUPT;
    for (uint64_t i = table_off + n_blocks * 2 * db; i < payload_off; ++i)
        if (in[i] != 0) return PO_ERR_CORRUPT;
    /* block word counts from the table alone, then the payload size */
    uint64_t sum = 0;
    uint64_t dmax = d == 16 ? 0xFFFFull : 0xFFFFFFFFull;
    for (uint64_t b = 0; b < n_blocks; ++b) {
        uint64_t n_b = n - b * L < L ? n - b * L : L;
        uint64_t vmin = get_le(in + table_off + b * 2 * db, db);
        uint64_t Bm1 = get_le(in + table_off + b * 2 * db + db, db);
        if (vmin + Bm1 > dmax) return PO_ERR_CORRUPT;
        sum += po_count(variant, Bm1 + 1, w, n_b);
    }
    if (sum != payload_words) return PO_ERR_CORRUPT;
    if (payload_words > (in_bytes - payload_off) / wb) return PO_ERR_CORRUPT;

    uint64_t *u_buf = (uint64_t *)malloc((L + 2) * sizeof(uint64_t));
    uint64_t *w_buf = (uint64_t *)malloc((L + 2) * sizeof(uint64_t));
    if (!u_buf || !w_buf) { free(u_buf); free(w_buf); return PO_ERR_INVALID_ARG; }
    uint64_t off = 0;
    for (uint64_t b = 0; b < n_blocks; ++b) {
        uint64_t start = b * L;
        uint64_t n_b = n - start < L ? n - start : L;
        uint64_t vmin = get_le(in + table_off + b * 2 * db, db);
        uint64_t B = get_le(in + table_off + b * 2 * db + db, db) + 1;
        uint64_t W = po_count(variant, B, w, n_b);
        for (uint64_t j = 0; j < W; ++j)
            w_buf[j] = get_le(in + payload_off + (off + j) * wb, wb);
        st = variant == 0 ? po_basic_unpack(B, w, w_buf, W, n_b, u_buf)
                          : po_adv_unpack(B, w, w_buf, W, n_b, u_buf);
        if (st != PO_OK) { free(u_buf); free(w_buf); return st; }
        for (uint64_t i = 0; i < n_b; ++i) {
            uint64_t v = u_buf[i] + vmin;
            if (d == 16) ((uint16_t *)out)[start + i] = (uint16_t)v;
            else ((uint32_t *)out)[start + i] = (uint32_t)v;
        }
        off += W;
    }
    free(u_buf);
    free(w_buf);
    *n_out = n;
    return PO_OK;
}

/* --------------------------- segmented stream (format version 2) ----- */

/* The block length is the parameter the paper tunes by hand from ratio
 * curves (Sec. 3.3, Sec. 4.2 Fig. 7).  A version-2 stream lets that choice
 * change along the data: the samples are cut into segments of seg_len
 * samples, and each segment is compressed blockwise (as above) with its own
 * block length L and word size w, recorded in one code byte.  Layout (all
 * little-endian):
 *   header, 64 bytes:  "PCMP", u16 version = 2, u8 variant, u8 dtype_bits,
 *                      4 zero bytes, u32 seg_len, u64 n_samples,
 *                      u64 n_segments, u64 body_bytes, 24 zero bytes
 *   codes:             one byte per segment, log2(L) | (w == 64) << 7, L a
 *                      power of two in [1, 8192]; zero-padded to a multiple
 *                      of 8 bytes
 *   sizes:             per segment, u32 body size in units of 8 bytes;
 *                      zero-padded to a multiple of 8 bytes
 *   bodies:            per segment in order: its block table (vmin, B - 1),
 *                      zero-padded to a multiple of 8 bytes, then its packed
 *                      words, zero-padded to a multiple of 8 bytes
 * A segment's body size also follows from its table alone (its word
 * counts); it is stored so that a reader finds every segment from a prefix
 * sum of the sizes, without walking the bodies one after another, and a
 * stored size that disagrees with the table is a corrupt stream. */

#define PO_V2_MAX_LOG2_L 13u

static uint64_t po_round8(uint64_t x) { return (x + 7) / 8 * 8; }

static int po_v2_code_ok(unsigned code)
{
    return (code & 0x60u) == 0 && (code & 0x1Fu) <= PO_V2_MAX_LOG2_L;
}

static uint64_t po_v2_L(unsigned code) { return (uint64_t)1 << (code & 0x1Fu); }
static unsigned po_v2_w(unsigned code) { return (code & 0x80u) ? 64u : 32u; }

/* Largest body of a segment of n_s samples under code `code`: its table
 * plus the largest word count of the blocked bound above. */
static uint64_t po_v2_body_bound(unsigned variant, unsigned d, unsigned code, uint64_t n_s)
{
    uint64_t L = po_v2_L(code), v1;
    unsigned w = po_v2_w(code);
    uint64_t nb = (n_s + L - 1) / L;
    po_bound(variant, d, w, L, n_s, &v1);
    uint64_t word_bytes = v1 - PO_HEADER_BYTES - po_table_bytes(nb, d);
    return po_round8(nb * 2 * (d / 8)) + po_round8(word_bytes);
}

/* Worst-case size of a version-2 stream of n samples, over every code. */
int po_bound_v2(unsigned variant, unsigned d, uint64_t seg_len, uint64_t n, uint64_t *max_bytes)
{
    if (!po_params_ok(variant, d, 32, seg_len)) return PO_ERR_INVALID_ARG;
    uint64_t n_seg = (n + seg_len - 1) / seg_len;
    uint64_t total = PO_HEADER_BYTES + po_round8(n_seg) + po_round8(4 * n_seg);
    for (int last = 0; last < 2; ++last) {
        uint64_t ns, count;
        if (n_seg == 0) break;
        if (!last) { ns = seg_len; count = n_seg - 1; }
        else { ns = n - (n_seg - 1) * seg_len; count = 1; }
        if (count == 0) continue;
        uint64_t worst = 0;
        for (unsigned k = 0; k <= PO_V2_MAX_LOG2_L; ++k)
            for (unsigned wide = 0; wide < 2; ++wide) {
                uint64_t b = po_v2_body_bound(variant, d, k | (wide << 7), ns);
                if (b > worst) worst = b;
            }
        total += count * worst;
    }
    *max_bytes = total;
    return PO_OK;
}

/* Each segment compressed alone by po_compress with its (L, w); its table
 * entries and words then move into the segment's body. */
int po_compress_v2(const void *in, uint64_t n, unsigned variant, unsigned d, uint64_t seg_len,
                   const uint8_t *codes, uint8_t *out, uint64_t cap, uint64_t *out_bytes)
{
    if (!po_params_ok(variant, d, 32, seg_len)) return PO_ERR_INVALID_ARG;
    uint64_t n_seg = (n + seg_len - 1) / seg_len;
    for (uint64_t s = 0; s < n_seg; ++s)
        if (!po_v2_code_ok(codes[s])) return PO_ERR_INVALID_ARG;
    unsigned db = d / 8;
    uint64_t sizes_at = PO_HEADER_BYTES + po_round8(n_seg);
    uint64_t bodies_at = sizes_at + po_round8(4 * n_seg), pos = bodies_at;
    if (cap < pos) return PO_ERR_CAPACITY;
    memset(out, 0, pos);
    for (uint64_t s = 0; s < n_seg; ++s) out[PO_HEADER_BYTES + s] = codes[s];
    for (uint64_t s = 0; s < n_seg; ++s) {
        uint64_t start = s * seg_len;
        uint64_t n_s = n - start < seg_len ? n - start : seg_len;
        uint64_t L = po_v2_L(codes[s]);
        unsigned w = po_v2_w(codes[s]), wb = w / 8;
        uint64_t v1cap, v1bytes;
        po_bound(variant, d, w, L, n_s, &v1cap);
        uint8_t *v1 = (uint8_t *)malloc(v1cap);
        if (!v1) return PO_ERR_INVALID_ARG;
        const uint8_t *src = (const uint8_t *)in + start * db;
        int st = po_compress(src, n_s, variant, d, w, L, v1, v1cap, &v1bytes);
        if (st != PO_OK) { free(v1); return st; }
        uint64_t nb = get_le(v1 + 24, 8), pw = get_le(v1 + 32, 8);
        uint64_t tb = nb * 2 * db, body = po_round8(tb) + po_round8(pw * wb);
        if (cap - pos < body) { free(v1); return PO_ERR_CAPACITY; }
        memset(out + pos, 0, body);
        memcpy(out + pos, v1 + PO_HEADER_BYTES, tb);
        memcpy(out + pos + po_round8(tb), v1 + PO_HEADER_BYTES + po_table_bytes(nb, d), pw * wb);
        if (body / 8 > 0xFFFFFFFFull) { free(v1); return PO_ERR_UNSUPPORTED; }
        put_le(out + sizes_at + 4 * s, body / 8, 4);
        pos += body;
        free(v1);
    }
    memcpy(out, "PCMP", 4);
    put_le(out + 4, 2, 2);
    out[6] = (uint8_t)variant;
    out[7] = (uint8_t)d;
    put_le(out + 12, seg_len, 4);
    put_le(out + 16, n, 8);
    put_le(out + 24, n_seg, 8);
    put_le(out + 32, pos - bodies_at, 8);
    *out_bytes = pos;
    return PO_OK;
}

static int po_zero(const uint8_t *p, uint64_t n)
{
    for (uint64_t i = 0; i < n; ++i) if (p[i] != 0) return 0;
    return 1;
}

int po_decompress_v2(const uint8_t *in, uint64_t in_bytes, void *out, uint64_t cap, uint64_t *n_out)
{
    *n_out = 0;
    if (in_bytes < PO_HEADER_BYTES) return PO_ERR_CORRUPT;
    if (memcmp(in, "PCMP", 4) != 0 || get_le(in + 4, 2) != 2) return PO_ERR_CORRUPT;
    unsigned variant = in[6], d = in[7];
    uint64_t seg_len = get_le(in + 12, 4), n = get_le(in + 16, 8);
    uint64_t n_seg = get_le(in + 24, 8), body_bytes = get_le(in + 32, 8);
    if (!po_zero(in + 8, 4) || !po_zero(in + 40, 24)) return PO_ERR_CORRUPT;
    if (!po_params_ok(variant, d, 32, seg_len)) return PO_ERR_CORRUPT;
    if (n_seg != (n + seg_len - 1) / seg_len) return PO_ERR_CORRUPT;
    /* codes and bodies must lie inside the buffer */
    if (n_seg > (in_bytes - PO_HEADER_BYTES) / 5) return PO_ERR_CORRUPT;
    uint64_t sizes_at = PO_HEADER_BYTES + po_round8(n_seg);
    uint64_t pos = sizes_at + po_round8(4 * n_seg);
    if (pos > in_bytes || body_bytes > in_bytes - pos) return PO_ERR_CORRUPT;
    uint64_t end = pos + body_bytes;
    if (!po_zero(in + PO_HEADER_BYTES + n_seg, sizes_at - PO_HEADER_BYTES - n_seg)) return PO_ERR_CORRUPT;
    if (!po_zero(in + sizes_at + 4 * n_seg, pos - sizes_at - 4 * n_seg)) return PO_ERR_CORRUPT;
    if (n > cap) return PO_ERR_CAPACITY;
    unsigned db = d / 8;
    uint64_t dmax = d == 16 ? 0xFFFFull : 0xFFFFFFFFull;
    for (uint64_t s = 0; s < n_seg; ++s) {
        unsigned code = in[PO_HEADER_BYTES + s];
        if (!po_v2_code_ok(code)) return PO_ERR_CORRUPT;
        uint64_t start = s * seg_len;
        uint64_t n_s = n - start < seg_len ? n - start : seg_len;
        uint64_t L = po_v2_L(code);
        unsigned w = po_v2_w(code), wb = w / 8;
        uint64_t nb = (n_s + L - 1) / L, tb = nb * 2 * db;
        if (po_round8(tb) > end - pos) return PO_ERR_CORRUPT;
        const uint8_t *table = in + pos;
        if (!po_zero(table + tb, po_round8(tb) - tb)) return PO_ERR_CORRUPT;
        uint64_t W = 0;
        for (uint64_t b = 0; b < nb; ++b) {
            uint64_t n_b = n_s - b * L < L ? n_s - b * L : L;
            uint64_t vmin = get_le(table + b * 2 * db, db), Bm1 = get_le(table + b * 2 * db + db, db);
            if (vmin + Bm1 > dmax) return PO_ERR_CORRUPT;
            W += po_count(variant, Bm1 + 1, w, n_b);
        }
        uint64_t words_at = pos + po_round8(tb);
        if (W > (end - words_at) / wb || po_round8(W * wb) > end - words_at) return PO_ERR_CORRUPT;
        if (!po_zero(in + words_at + W * wb, po_round8(W * wb) - W * wb)) return PO_ERR_CORRUPT;
        /* the blocks of the segment, as in po_decompress */
        uint64_t *u_buf = (uint64_t *)malloc((L + 2) * sizeof(uint64_t));
        uint64_t *w_buf = (uint64_t *)malloc((L + 2) * sizeof(uint64_t));
        if (!u_buf || !w_buf) { free(u_buf); free(w_buf); return PO_ERR_INVALID_ARG; }
        uint64_t off = 0;
        for (uint64_t b = 0; b < nb; ++b) {
            uint64_t n_b = n_s - b * L < L ? n_s - b * L : L;
            uint64_t vmin = get_le(table + b * 2 * db, db);
            uint64_t B = get_le(table + b * 2 * db + db, db) + 1;
            uint64_t Wb = po_count(variant, B, w, n_b);
            for (uint64_t j = 0; j < Wb; ++j) w_buf[j] = get_le(in + words_at + (off + j) * wb, wb);
            int st = variant == 0 ? po_basic_unpack(B, w, w_buf, Wb, n_b, u_buf)
                                  : po_adv_unpack(B, w, w_buf, Wb, n_b, u_buf);
            if (st != PO_OK) { free(u_buf); free(w_buf); return st; }
            for (uint64_t i = 0; i < n_b; ++i) {
                uint64_t v = u_buf[i] + vmin, k = start + b * L + i;
                if (d == 16) ((uint16_t *)out)[k] = (uint16_t)v;
                else ((uint32_t *)out)[k] = (uint32_t)v;
            }
            off += Wb;
        }
        free(u_buf);
        free(w_buf);
        uint64_t next = words_at + po_round8(W * wb);
        if (get_le(in + sizes_at + 4 * s, 4) * 8 != next - pos) return PO_ERR_CORRUPT;
        pos = next;
    }
    if (pos != end) return PO_ERR_CORRUPT;
    *n_out = n;
    return PO_OK;
}
