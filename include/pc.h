/*
 * pc.h -- C ABI of the GB300 polynomial compression library (libpc.so).
 *
 * Lossless compression of small-range integer samples dominated by white
 * noise, after Aubert et al., "Polynomial data compression for large-scale
 * physics experiments" (arXiv:1805.01844):
 *   - the samples are cut into blocks of block_len consecutive samples
 *     (Sec. 3.3, blocked compression);
 *   - each block stores its minimum and its base B = max - min + 1 once
 *     (Sec. 3.1 and Fig. 2) and packs the offsets v - min as base-B digits
 *     into 32- or 64-bit words, either
 *       basic    (Sec. 3.1, Eqs. 1-2): p = max{p : B^p <= 2^w - 1} digits per
 *                word, first sample in the lowest power, or
 *       advanced (Sec. 3.2, Eqs. 3-11 and the series after them): the last
 *                base of a word is split into R_i * R'_i >= B so that one
 *                sample straddles two consecutive words, first sample in the
 *                highest power;
 *   - decompression inverts the packing by repeated division by B.
 *
 * Everything runs on the GPU in hand-written sm_103a kernels; there is no CPU
 * path.  All buffers are owned by the caller, the library allocates nothing
 * and keeps no state between calls, and all work is ordered on the caller's
 * CUDA stream.  Entry points return after enqueuing work; the host return
 * code covers argument checks and launch errors, while conditions found on
 * the device (a corrupt stream, a wait that ran out) are recorded in the
 * workspace and read back with pc_last_device_status().  No kernel traps, and
 * every device-side wait is bounded (about one second).
 *
 * STREAM FORMAT, version 1 (all fields little-endian):
 *   offset 0   header, 64 bytes
 *              "PCMP" | u16 version = 1 | u8 variant | u8 dtype_bits |
 *              u8 word_bits | 3 zero bytes | u32 block_len | u64 n_samples |
 *              u64 n_blocks = ceil(n_samples / block_len) | u64 payload_words |
 *              24 zero bytes
 *   offset 64  block table: per block (min, B - 1), each field dtype_bits
 *              wide, zero-padded to a multiple of 16 bytes.  B - 1 is stored
 *              because B = 2^dtype_bits does not fit in dtype_bits.
 *   then       payload: for each block in order, its packed words
 *              (word_bits each).  A block with B = 1 has no words.
 *   The word count of a block is a function of (variant, B, word_bits,
 *   samples in the block) only, so any block can be located from the table
 *   alone ("readable by part", Sec. 4.3).
 */
#ifndef PC_H
#define PC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    PC_OK = 0,
    PC_ERR_INVALID_ARG = 1,  /* bad parameter, NULL or misaligned pointer, workspace too small */
    PC_ERR_CAPACITY = 2,     /* output buffer smaller than required */
    PC_ERR_CORRUPT = 3,      /* the input is not a valid stream */
    PC_ERR_CUDA = 4,         /* a CUDA launch or copy failed */
    PC_ERR_TIMEOUT = 5,      /* a bounded device-side wait ran out */
    PC_ERR_UNSUPPORTED = 6   /* valid parameters outside what the kernels support */
} pc_status;

/* Compression parameters (also the stream's own header fields). */
typedef struct {
    uint32_t variant;    /* 0 = basic (Sec. 3.1, Eq. 2), 1 = advanced (Sec. 3.2) */
    uint32_t dtype_bits; /* sample width: 16 (uint16) or 32 (uint32) */
    uint32_t word_bits;  /* packed word width: 32 or 64 (the paper uses 32) */
    uint32_t block_len;  /* samples per block, 1 .. PC_MAX_BLOCK_LEN (Sec. 3.3) */
} pc_params;

#define PC_HEADER_BYTES 64u
#define PC_MAX_BLOCK_LEN 8192u
#define PC_VARIANT_BASIC 0u
#define PC_VARIANT_ADVANCED 1u

/* A cudaStream_t passed as an opaque pointer; NULL is the legacy default
 * stream. */
typedef void *pc_stream_t;

/* Upper bound on the stream size, in bytes, of n_samples samples compressed
 * with *params: header + table + every block at its largest word count over
 * all bases B in [1, 2^dtype_bits] (basic: ceil(n_b / p(2^d)); advanced: at
 * most ceil((n_b + 1) / p_1(2^d)) words, n_b + 1 when p_1 = 0).  Host only.
 * Errors: PC_ERR_INVALID_ARG for bad params or NULL max_bytes;
 * PC_ERR_UNSUPPORTED for block_len > PC_MAX_BLOCK_LEN. */
pc_status pc_bound(const pc_params *params, uint64_t n_samples, uint64_t *max_bytes);

/* Bytes of device workspace pc_compress / pc_decompress need for streams of
 * at most n_samples samples with *params: a 64-byte header, 8 bytes per tile
 * of blocks (look-back words, decoding offsets) and, for the advanced variant,
 * a table of the split-base series of every base B <= 65536 the stream meets
 * (about 17 MB, filled lazily by the kernels).  The table depends on the base
 * and the word size only, so it is kept across calls that reuse the
 * workspace (a tag in the workspace header records the word size it was
 * built for; any other content, including a fresh allocation, is cleared by
 * the first call).  Calls that share a workspace must not overlap on the
 * GPU.  The advanced variant also runs with a smaller workspace that only
 * has room for the look-back words and offsets; each block then walks its
 * series serially (same bytes, slower).  Host only.  Errors as for pc_bound. */
pc_status pc_workspace_size(const pc_params *params, uint64_t n_samples, uint64_t *bytes);

/* Compress n_samples samples (uint16 or uint32 per params->dtype_bits) from
 * device memory d_in into a version-1 stream at device memory d_out: blocked
 * compression (Sec. 3.3) with, per block, the minimum and base of Sec. 3.1
 * (Fig. 2's block header) and the packing of Eq. 2 (basic, Sec. 3.1) or of
 * the split-base series (advanced, Sec. 3.2).
 *   d_in           device pointer, 16-byte aligned (may be NULL if n_samples = 0)
 *   d_out          device pointer, 16-byte aligned, out_capacity bytes; must be
 *                  at least pc_bound(params, n_samples) (else PC_ERR_CAPACITY)
 *   d_out_bytes    device pointer to one uint64_t: the stream size, written
 *                  by the device when the work completes
 *   d_workspace    device pointer, 16-byte aligned, workspace_bytes >=
 *                  pc_workspace_size(params, n_samples) (else PC_ERR_INVALID_ARG);
 *                  cleared by this call, must not be shared with work that
 *                  overlaps on the GPU
 *   stream         CUDA stream the work is ordered on
 * The stream bytes are identical for any launch configuration: each block's
 * words land at the exclusive prefix sum of the word counts before it, found
 * in one pass by a decoupled look-back over tiles of blocks.
 * Device-side status (PC_ERR_TIMEOUT if a look-back wait ran out) is read
 * with pc_last_device_status(d_workspace, stream). */
pc_status pc_compress(const void *d_in, uint64_t n_samples, const pc_params *params,
                      void *d_out, uint64_t out_capacity, uint64_t *d_out_bytes,
                      void *d_workspace, uint64_t workspace_bytes, pc_stream_t stream);

/* Decompress the stream of in_bytes bytes at device memory d_in into device
 * memory d_out (uint16 or uint32 samples): the inverse of the packing by
 * repeated division by B, Sec. 3.1 ("polynomial division"), and, for the
 * advanced variant, by the split bases R_i of Sec. 3.2.  The params argument
 * is this library's addition to the boundary: it selects the kernel
 * instantiation on the host without reading the stream's header back from
 * the device (which would synchronise the stream); the device checks it
 * against the header.
 *   params         the parameters the stream was written with; the device
 *                  checks that the header matches them (else PC_ERR_CORRUPT)
 *   d_in           device pointer, 16-byte aligned
 *   d_out          device pointer, 16-byte aligned, room for
 *                  out_capacity_samples samples; a stream with more samples
 *                  is rejected on the device with PC_ERR_CAPACITY and nothing
 *                  is written
 *   d_n_samples    device pointer to one uint64_t: n_samples of the stream,
 *                  written by the device
 *   d_workspace    as for pc_compress, sized for out_capacity_samples
 * Every read stays inside [d_in, d_in + in_bytes).  The device rejects
 * (PC_ERR_CORRUPT) a bad header, a table entry with min + B - 1 above the
 * dtype range, a payload shorter than the table implies or a word count that
 * differs from the header, and any word that is not the image of valid
 * digits (a value >= B^k, a non-zero padding digit, a re-joined split sample
 * >= B).  The decoder therefore accepts exactly the streams pc_compress can
 * produce.  After an error the content of d_out is unspecified.
 * in_bytes < 64 returns PC_ERR_CORRUPT from the host. */
pc_status pc_decompress(const void *d_in, uint64_t in_bytes, const pc_params *params,
                        void *d_out, uint64_t out_capacity_samples, uint64_t *d_n_samples,
                        void *d_workspace, uint64_t workspace_bytes, pc_stream_t stream);

/* Parse a stream header that the caller has copied to host memory (at least
 * 64 bytes).  Fills *params and *n_samples.  Host only; PC_ERR_CORRUPT if the
 * header is not a valid version-1 header. */
pc_status pc_parse_header(const void *host_header, uint64_t nbytes, pc_params *params,
                          uint64_t *n_samples);

/* Synchronise `stream` and return the device-side status recorded in the
 * workspace by the last pc_compress / pc_decompress that used it: PC_OK,
 * PC_ERR_CORRUPT, PC_ERR_CAPACITY, PC_ERR_INVALID_ARG (workspace too small
 * for the stream's tiles) or PC_ERR_TIMEOUT.  PC_ERR_CUDA if the
 * synchronisation or the copy fails. */
pc_status pc_last_device_status(const void *d_workspace, pc_stream_t stream);

/* Self-test of the bounded device wait used by the look-back: launches one
 * block that waits on a status word nothing ever sets, with a limit of
 * limit_us microseconds, and records PC_ERR_TIMEOUT in the workspace when the
 * wait gives up (read it with pc_last_device_status).  The same wait routine
 * guards every look-back in pc_compress / pc_decompress.  d_workspace needs
 * pc_workspace_size(params, 0) bytes for any params. */
pc_status pc_selftest_bounded_wait(void *d_workspace, uint64_t workspace_bytes,
                                   uint32_t limit_us, pc_stream_t stream);

/* ---- batches: many independent streams in one launch -------------------
 * Every item is an independent stream with its own parameters (dtype, word
 * size, variant, block length); the output of each item is exactly the
 * stream pc_compress would produce for it.  The work is ordered as:
 *   pc_batch_describe   host only: launch facts and device sizes
 *   pc_batch_plan       one host-to-device copy of the item descriptors and
 *                       a tile prefix into caller memory d_plan
 *   pc_compress_batch   a memset and one persistent kernel on `stream`, which
 *                       can be captured in a CUDA graph and replayed as long
 *                       as the plan and the buffers stay in place.
 * Tiles of all items share one ticket counter; within an item they keep the
 * in-order look-back of pc_compress.  Bounded waits as for pc_compress. */
typedef struct {
    const void *d_in;       /* device samples, 16-byte aligned (NULL if n_samples = 0) */
    uint64_t n_samples;
    pc_params params;
    void *d_out;            /* device stream buffer, 16-byte aligned */
    uint64_t out_capacity;  /* >= pc_bound(&params, n_samples), else PC_ERR_CAPACITY */
    uint64_t *d_out_bytes;  /* device: this item's stream size, written by the device */
} pc_batch_item;

typedef struct {
    uint32_t n_items;
    uint32_t smem_bytes;      /* dynamic shared memory of the launch */
    uint64_t total_tiles;     /* tiles over all items (an empty item counts 1) */
    uint64_t plan_bytes;      /* device bytes pc_batch_plan writes */
    uint64_t workspace_bytes; /* device workspace pc_compress_batch needs */
    uint32_t cta_threads;     /* in: 128 or 256 threads per CTA (anything else: 256); out: the value used */
    uint32_t reserved;
} pc_batch_info;

/* Validate items (same rules as pc_compress) and fill *info.  Host only.
 * info->cta_threads is read first: 128-thread CTAs take half-size tiles and
 * run twice as many per SM (faster for short blocks); the plan and the
 * launch follow the value describe settles on. */
pc_status pc_batch_describe(const pc_batch_item *items, uint32_t n_items, pc_batch_info *info);

/* Copy the descriptors and the tile prefix of items to device memory d_plan
 * (info->plan_bytes bytes, 16-byte aligned) on `stream`.  items is read before
 * the call returns. */
pc_status pc_batch_plan(const pc_batch_item *items, uint32_t n_items, const pc_batch_info *info, void *d_plan,
                        pc_stream_t stream);

/* Compress every item of a plan: clears the workspace (info->workspace_bytes
 * bytes, 16-byte aligned) and launches one persistent kernel.  Device-side
 * status as for pc_compress (pc_last_device_status(d_workspace, stream)). */
pc_status pc_compress_batch(const pc_batch_info *info, const void *d_plan, void *d_workspace,
                            uint64_t workspace_bytes, pc_stream_t stream);

/* ---- learned block-parameter chooser ------------------------------------
 * The paper picks the block size by hand from ratio-versus-size curves
 * (Sec. 4.2, Fig. 7; Sec. 4.3.2, Fig. 10).  Here a small MLP picks, for every
 * segment of PC_SEGMENT_SAMPLES samples, one of PC_CHOOSER_OPTIONS parameter
 * choices: option o = 2 i + j means block length 128 << i (i = 0..5) and
 * word size 32 (j = 0) or 64 (j = 1).  The choice changes the parameters of
 * each segment's stream, never the format, so losslessness is untouched.
 * Features (PC_CHOOSER_FEATURES per segment, FP32, each roughly in [0, 1]):
 *   0 min / dmax, 1 max / dmax, 2 log2(max - min + 1) / d,
 *   3..18 fraction of the 32 sub-blocks of 128 samples whose range r has
 *         floor(log2(r + 1)) = 0..15 (15 also counts larger),
 *   19 mean / dmax, 20 log2(variance + 1) / 2d, 21 fraction of sub-blocks
 *   whose range exceeds 4 (smallest sub-block range + 1), 22 d / 32,
 *   23 (segment index mod 64) / 64;   d = dtype bits, dmax = 2^d - 1.
 * MLP 24 -> 64 -> 64 -> 12, ReLU, softmax.  Weight buffer (PC_MLP_WEIGHT_BYTES,
 * 16-byte aligned): BF16 W1[64][24], W2[64][64], W3[12][64], then FP32 b1[64],
 * b2[64], b3[12].  Training buffers are FP32 in the same order
 * (PC_MLP_PARAMS values).  All products accumulate in FP32. */
#define PC_SEGMENT_SAMPLES 4096u
#define PC_CHOOSER_FEATURES 24u
#define PC_CHOOSER_HIDDEN 64u
#define PC_CHOOSER_OPTIONS 12u
#define PC_MLP_PARAMS 6540u
#define PC_MLP_WEIGHT_BYTES 13360u

/* Features of every segment of d_in (n_samples of dtype_bits) into
 * d_features[ceil(n / 4096)][24]. */
pc_status pc_segment_features(const void *d_in, uint64_t n_samples, uint32_t dtype_bits, float *d_features,
                              pc_stream_t stream);

/* Logits (optional, [n][12]) and the arg-max option (optional, [n]) of n
 * feature rows. */
pc_status pc_mlp_forward(const void *d_weights, const float *d_x, uint64_t n, float *d_logits, uint8_t *d_choice,
                         pc_stream_t stream);

/* Adds to d_grad[PC_MLP_PARAMS] the gradient of the mean softmax
 * cross-entropy of n rows with labels d_labels[n] (options), and the summed
 * loss to *d_loss, at the BF16 weights d_weights. */
pc_status pc_mlp_grad(const void *d_weights, const float *d_x, const uint8_t *d_labels, uint64_t n, float *d_grad,
                      float *d_loss, pc_stream_t stream);

/* One Adam step (beta 0.9 / 0.999, eps 1e-8, step >= 1) on the FP32 master
 * copy; rewrites the BF16 weights from it and clears d_grad. */
pc_status pc_mlp_adam(float *d_master, void *d_weights, float *d_grad, float *d_m, float *d_v, uint32_t step,
                      float lr, pc_stream_t stream);

/* ---- segments: the chooser's whole path on the device --------------------
 * A list of sources (device sample arrays) is cut into segments of
 * PC_SEGMENT_SAMPLES samples (the last segment of a source may be shorter; a
 * source of 0 samples has no segment).  Segments are numbered over all
 * sources in order.  Segment j of a source is an ordinary version-1 stream
 * written to its fixed output slot d_out + j * seg_stride, its size to
 * d_out_bytes[j]; seg_stride holds the stream of a full segment under every
 * one of the PC_CHOOSER_OPTIONS options.  Features, choices and parameters
 * stay in device memory, so features -> pc_mlp_forward -> compression runs
 * without a host round trip:
 *   pc_segments_describe   host only: sizes and launch facts
 *   pc_segments_plan       one host-to-device copy of the source table
 *   pc_segments_features   feature rows of every segment (one kernel)
 *   pc_compress_segments   every segment with its own option: a memset, one
 *                          kernel (a warp per segment; for 32-bit advanced
 *                          data a descriptor kernel and the batch kernel), and
 *                          (if any source has d_totals) a kernel adding to the
 *                          totals.
 * Feature 23 uses the segment's index within its source, so a segment's
 * features, choice and stream do not depend on the other sources.  A source
 * of 0 samples is skipped entirely (it adds nothing to its totals). */
typedef struct {
    const void *d_in;       /* device samples, 16-byte aligned (NULL if n_samples = 0) */
    uint64_t n_samples;
    void *d_out;            /* device, 16-byte aligned: slot j at d_out + j * seg_stride */
    uint64_t out_capacity;  /* >= ceil(n_samples / 4096) * seg_stride, else PC_ERR_CAPACITY */
    uint64_t *d_out_bytes;  /* device, [ceil(n_samples / 4096)] stream sizes */
    uint64_t *d_totals;     /* device running totals of the source's stream, or NULL:
                               [0] += 1 and [1] += the sum of its stream sizes per call */
} pc_source;

typedef struct {
    uint32_t n_sources;
    uint32_t dtype_bits;
    uint32_t variant;
    uint32_t smem_bytes;      /* dynamic shared memory of the batch launch */
    uint32_t has_totals;      /* 1 if some source has d_totals */
    uint32_t reserved;
    uint64_t n_segments;      /* over all sources */
    uint64_t seg_stride;      /* bytes per output slot, a multiple of 16 */
    uint64_t plan_bytes;      /* device bytes pc_segments_plan writes */
    uint64_t workspace_bytes; /* device workspace pc_compress_segments needs */
} pc_segments_info;

/* Validate the sources and fill *info.  Host only.  PC_ERR_UNSUPPORTED if
 * the segment count reaches 2^31. */
pc_status pc_segments_describe(const pc_source *src, uint32_t n_sources, uint32_t dtype_bits, uint32_t variant,
                               pc_segments_info *info);

/* Copy the source table to device memory d_plan (info->plan_bytes bytes,
 * 16-byte aligned) on `stream`; src is read before the call returns. */
pc_status pc_segments_plan(const pc_source *src, uint32_t n_sources, const pc_segments_info *info, void *d_plan,
                           pc_stream_t stream);

/* Feature rows of every segment into d_features[n_segments][24] (the
 * features of pc_segment_features, segment index counted within its source). */
pc_status pc_segments_features(const pc_segments_info *info, const void *d_plan, float *d_features,
                               pc_stream_t stream);

/* Compress every segment with option d_options[k] (device, [n_segments]).
 * An option >= PC_CHOOSER_OPTIONS is recorded as PC_ERR_INVALID_ARG in the
 * workspace status (pc_last_device_status) and that segment is compressed
 * with option 0, so every slot still holds a valid stream of its samples.
 * d_workspace: info->workspace_bytes, 16-byte aligned.  No-op if there are no
 * segments.  Bounded waits as for pc_compress. */
pc_status pc_compress_segments(const pc_segments_info *info, const void *d_plan, const uint8_t *d_options,
                               void *d_workspace, uint64_t workspace_bytes, pc_stream_t stream);

/* ---- sharding: one stream split into block-aligned shards and stitched --
 * Blocks are independent (Sec. 3.3, blocked compression), and a block's word
 * count is a function of its table entry alone, so a stream is "readable by
 * part" (Sec. 4.3).  One stream of n_samples can therefore be compressed as
 * K shards of whole blocks (one per GPU, or several on one GPU), each an
 * ordinary stream from pc_compress, and stitched into exactly the bytes a
 * single pc_compress call would write:
 *   pc_shard_range    host: the block-aligned sample range of shard k
 *   (exchange)        every shard's stream size, 8 bytes per shard, gathered
 *                     to wherever stitching runs (an all-gather across ranks)
 *   pc_stitch         device: shard k's table entries and payload copied to
 *                     their place in the whole stream (the exclusive prefix of
 *                     the shards' payload sizes), plus the header (shard 0)
 *                     and the table padding and total size (shard K - 1)
 *   pc_stitch_layout  host: the same placement as byte ranges, for callers
 *                     that move the pieces themselves (a collective, a file)
 * The inverse, pc_slice, cuts the stream of a block range back out of a whole
 * stream (a scan of the table gives the range's payload offset), so each rank
 * decompresses its own blocks with pc_decompress. */
typedef struct {
    uint64_t total_bytes;    /* size of the whole stream */
    uint64_t first_block;    /* shard's blocks: [first_block, first_block + n_blocks) */
    uint64_t n_blocks;
    uint64_t table_src;      /* shard's table entries: shard stream bytes [table_src, + table_bytes) */
    uint64_t table_dst;      /*   go to whole-stream bytes [table_dst, + table_bytes) */
    uint64_t table_bytes;
    uint64_t payload_src;    /* shard's payload: [payload_src, + payload_bytes) */
    uint64_t payload_dst;    /*   goes to [payload_dst, + payload_bytes) */
    uint64_t payload_bytes;
    uint64_t pad_dst;        /* the whole stream's table padding, zeros: [pad_dst, payload start) */
    uint64_t payload_start;  /* offset of the whole stream's payload */
} pc_stitch_region;

/* Shard `shard` of n_shards of a stream of n_samples with *params: whole
 * blocks, the first n_blocks % n_shards shards one block more than the rest.
 * *first_sample = its first sample, *n_shard_samples its length (0 for a
 * shard without blocks).  Host only.  PC_ERR_INVALID_ARG for n_shards = 0,
 * shard >= n_shards, NULL outputs or bad params. */
pc_status pc_shard_range(const pc_params *params, uint64_t n_samples, uint32_t n_shards, uint32_t shard,
                         uint64_t *first_sample, uint64_t *n_shard_samples);

/* Where shard `shard`'s pieces go in the whole stream, given every shard's
 * stream size shard_bytes[n_shards] (host memory).  Host only.
 * PC_ERR_CORRUPT if a size cannot be a stream of its shard's blocks. */
pc_status pc_stitch_layout(const pc_params *params, uint64_t n_samples, uint32_t n_shards, uint32_t shard,
                           const uint64_t *shard_bytes, pc_stitch_region *region);

/* Copy shard `shard`'s stream d_shard (as pc_compress wrote it for the
 * samples of pc_shard_range) into its place in the whole stream at d_out.
 *   d_shard_bytes  device, [n_shards]: every shard's stream size (what each
 *                  pc_compress wrote to its d_out_bytes, gathered)
 *   d_out          device, 16-byte aligned, out_capacity >= pc_bound(params,
 *                  n_samples) (else PC_ERR_CAPACITY); the calls of all shards
 *                  with one d_out write disjoint bytes and together the whole
 *                  stream, in any order, on any streams
 *   d_out_bytes    device, one uint64_t: the whole stream's size, written by
 *                  the call of shard n_shards - 1 (may be NULL for the others)
 *   d_workspace    device, >= 64 bytes, 16-byte aligned: status word, read
 *                  with pc_last_device_status (PC_ERR_CORRUPT if the shard
 *                  stream's header or a size does not match its shard)
 * One kernel, no look-back, no allocation. */
pc_status pc_stitch(const void *d_shard, const uint64_t *d_shard_bytes, uint32_t n_shards, uint32_t shard,
                    uint64_t n_samples, const pc_params *params, void *d_out, uint64_t out_capacity,
                    uint64_t *d_out_bytes, void *d_workspace, uint64_t workspace_bytes, pc_stream_t stream);

/* The stream of blocks [first_block, first_block + n_blocks) of the whole
 * stream d_in (in_bytes bytes, written with *params): a header for those
 * samples, their table entries and their payload words, i.e. exactly what
 * pc_compress writes for those samples.  Two kernels: the word counts of the
 * blocks before and inside the range from the table (a reduction), then the
 * copy.  d_out: 16-byte aligned, out_capacity >= pc_bound(params, n_blocks *
 * block_len) (else PC_ERR_CAPACITY); d_out_bytes: device, its size;
 * d_workspace: >= 64 bytes, 16-byte aligned (pc_last_device_status:
 * PC_ERR_CORRUPT for a bad header, table entry or payload shorter than the
 * table implies; PC_ERR_INVALID_ARG for a range past the last block). */
pc_status pc_slice(const void *d_in, uint64_t in_bytes, const pc_params *params, uint64_t first_block,
                   uint64_t n_blocks, void *d_out, uint64_t out_capacity, uint64_t *d_out_bytes,
                   void *d_workspace, uint64_t workspace_bytes, pc_stream_t stream);

/* ---- byte profile (Sec. 5, Fig. 11) --------------------------------------
 * Occurrences of each byte value 0..255 in n_bytes bytes of device memory
 * d_bytes (any alignment): d_hist is device memory of 256 uint64_t
 * (8-byte aligned), cleared and then filled on `stream`.  The paper compares
 * the byte profile of a file before and after polynomial compression (a
 * flatter profile after).  PC_ERR_INVALID_ARG for NULL pointers. */
pc_status pc_byte_histogram(const void *d_bytes, uint64_t n_bytes, uint64_t *d_hist, pc_stream_t stream);

/* ---- format version 2: block length and word size per segment ---------
 * The paper picks the block length by hand from ratio curves (Sec. 3.3;
 * Sec. 4.2, Fig. 7; Sec. 4.3.2, Fig. 10).  A version-2 stream records that
 * choice per segment of the data in one stream: samples are cut into
 * segments of seg_len samples (the last may be shorter), and each segment is
 * compressed blockwise with its own (L, w), L a power of two <= 8192.
 * Layout, little-endian:
 *   header, 64 bytes: "PCMP", u16 version = 2, u8 variant, u8 dtype_bits,
 *     4 zero bytes, u32 seg_len, u64 n_samples, u64 n_segments,
 *     u64 body_bytes, 24 zero bytes;
 *   codes: one byte per segment, log2(L) | (w == 64) << 7, zero-padded to a
 *     multiple of 8 bytes;
 *   sizes: per segment, u32 body size in units of 8 bytes, zero-padded to a
 *     multiple of 8 bytes (every segment is found by a prefix sum);
 *   bodies: per segment, its block table (vmin, B - 1), zero-padded to 8
 *     bytes, then its packed words, zero-padded to 8 bytes.
 * A segment's body holds the same table entries and words as the version-1
 * stream of that segment alone; 64 bytes of header per segment become 5.
 *
 * pc_bound_v2: worst-case stream size over every code (host only).
 * pc_assemble_v2: one version-2 stream from the version-1 streams of
 *   n_segments consecutive segments, segment j at d_slots + j * seg_stride
 *   (16-byte aligned, seg_stride a multiple of 16: the slots that
 *   pc_compress_segments writes for one source, seg_len =
 *   PC_SEGMENT_SAMPLES).  Each slot's header must name this variant and
 *   dtype, a power-of-two block length <= 8192 and the segment's sample
 *   count, and fit its slot; otherwise PC_ERR_INVALID_ARG is recorded in the
 *   workspace status and the segment gets an empty body.  A body that would
 *   pass out_capacity records PC_ERR_CAPACITY (out_capacity >=
 *   pc_bound_v2 always suffices).  *d_out_bytes gets the stream size.
 *   Workspace: pc_assemble_v2_workspace_size bytes, 16-byte aligned.
 * pc_decompress_v2: the samples of a version-2 stream of this variant, dtype
 *   and seg_len (all checked against its header) into d_out (capacity in
 *   samples); *d_n_samples gets the count.  Corrupt streams (header, codes,
 *   paddings, stored sizes that disagree with the tables, invalid words) are
 *   recorded as PC_ERR_CORRUPT in the workspace status, read by
 *   pc_last_device_status.  PC_ERR_UNSUPPORTED for advanced 32-bit data
 *   (bases above 65536 need the serial series walk; the CPU reference decodes
 *   them).  Workspace: pc_decompress_v2_workspace_size bytes for the
 *   capacity, 16-byte aligned.
 * Bounded waits and host-side error returns as for pc_compress. */
pc_status pc_bound_v2(uint32_t variant, uint32_t dtype_bits, uint32_t seg_len, uint64_t n_samples,
                      uint64_t *max_bytes);
pc_status pc_assemble_v2_workspace_size(uint64_t n_segments, uint64_t *bytes);
pc_status pc_assemble_v2(const void *d_slots, uint64_t seg_stride, uint64_t n_segments, uint64_t n_samples,
                         uint32_t seg_len, uint32_t dtype_bits, uint32_t variant, void *d_out, uint64_t out_capacity,
                         uint64_t *d_out_bytes, void *d_workspace, uint64_t workspace_bytes, pc_stream_t stream);
pc_status pc_decompress_v2_workspace_size(uint32_t variant, uint32_t dtype_bits, uint32_t seg_len,
                                          uint64_t capacity_samples, uint64_t *bytes);
pc_status pc_decompress_v2(const void *d_in, uint64_t in_bytes, uint32_t variant, uint32_t dtype_bits,
                           uint32_t seg_len, void *d_out, uint64_t out_capacity_samples, uint64_t *d_n_samples,
                           void *d_workspace, uint64_t workspace_bytes, pc_stream_t stream);

/* Compression without any device allocation, for callers that cannot
 * allocate device memory once they run: a data-acquisition loop that must not
 * call cudaMalloc mid-readout (it can fail under memory pressure or
 * synchronise the device), or code inside a framework that owns the device
 * allocator.  The paper has no counterpart; it is an interface of this
 * library.  Same arguments, checks and output as pc_compress, but the
 * workspace is a static device array of PC_NOALLOC_SCRATCH_BYTES bytes inside
 * libpc.so, held by every GPU that loads the library until the process exits.
 *   - the call needs the look-back part of the workspace only (the header,
 *     one 8-byte word per tile and the decoding offsets pc_workspace_size
 *     also counts, without the advanced variant's series table); where that
 *     exceeds PC_NOALLOC_SCRATCH_BYTES the call returns PC_ERR_UNSUPPORTED
 *     before touching the device.  With 1 MiB that allows about 2.1e9 uint16
 *     samples at block_len 1024 (basic or advanced), 5.4e8 at block_len 256;
 *   - advanced streams compress with the serial series walk of each block
 *     (the series table does not fit the scratch): the same bytes, slower;
 *   - the first call on a device looks up the array's device address with
 *     cudaGetSymbolAddress (with that device current); make that first call
 *     before any stream capture;
 *   - every call on a device shares the array: calls that overlap on the GPU
 *     race and must be serialised by the caller (same stream, or events);
 *   - the device-side status lives in the shared array and is not readable;
 *     a bounded look-back wait that ran out leaves *d_out_bytes unwritten, so
 *     set it to 0 before the call to detect that.
 * Calls no cudaMalloc, cudaFree or other allocating routine. */
#define PC_NOALLOC_SCRATCH_BYTES (1u << 20)
pc_status pc_compress_noalloc(const void *d_in, uint64_t n_samples, const pc_params *params,
                              void *d_out, uint64_t out_capacity, uint64_t *d_out_bytes,
                              pc_stream_t stream);

/* Static description of an error code. */
const char *pc_strerror(pc_status status);

#ifdef __cplusplus
}
#endif

#endif /* PC_H */
