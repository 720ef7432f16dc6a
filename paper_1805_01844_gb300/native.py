"""ctypes binding of libpc.so (include/pc.h): argument marshalling only.

Every step of compression and decompression runs in the library's CUDA
kernels; this module passes device pointers, sizes and the CUDA stream of
torch tensors through the C ABI and turns status codes into exceptions.  It
fails loudly when the library is missing: there is no other code path.
"""
import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libpc.so")

PC_OK, PC_ERR_INVALID_ARG, PC_ERR_CAPACITY, PC_ERR_CORRUPT = 0, 1, 2, 3
PC_ERR_CUDA, PC_ERR_TIMEOUT, PC_ERR_UNSUPPORTED = 4, 5, 6
HEADER_BYTES = 64
MAX_BLOCK_LEN = 8192
BASIC, ADVANCED = 0, 1

EXPORTS = ("pc_bound", "pc_workspace_size", "pc_compress", "pc_decompress",
           "pc_parse_header", "pc_last_device_status", "pc_selftest_bounded_wait",
           "pc_strerror", "pc_compress_noalloc", "pc_batch_describe", "pc_batch_plan",
           "pc_compress_batch", "pc_segment_features", "pc_mlp_forward", "pc_mlp_grad", "pc_mlp_adam",
           "pc_segments_describe", "pc_segments_plan", "pc_segments_features", "pc_compress_segments",
           "pc_shard_range", "pc_stitch_layout", "pc_stitch", "pc_slice", "pc_byte_histogram",
           "pc_bound_v2", "pc_assemble_v2_workspace_size", "pc_assemble_v2", "pc_decompress_v2_workspace_size",
           "pc_decompress_v2")
SEGMENT_SAMPLES, CHOOSER_FEATURES, CHOOSER_OPTIONS = 4096, 24, 12
MLP_PARAMS, MLP_WEIGHT_BYTES = 6540, 13360
NOALLOC_SCRATCH_BYTES = 1 << 20


class PcParams(ctypes.Structure):
    _fields_ = [("variant", ctypes.c_uint32), ("dtype_bits", ctypes.c_uint32),
                ("word_bits", ctypes.c_uint32), ("block_len", ctypes.c_uint32)]

    def __repr__(self):
        return "PcParams(variant=%d, dtype_bits=%d, word_bits=%d, block_len=%d)" % (
            self.variant, self.dtype_bits, self.word_bits, self.block_len)


class PcBatchItem(ctypes.Structure):
    _fields_ = [("d_in", ctypes.c_void_p), ("n_samples", ctypes.c_uint64), ("params", PcParams),
                ("d_out", ctypes.c_void_p), ("out_capacity", ctypes.c_uint64),
                ("d_out_bytes", ctypes.c_void_p)]


class PcBatchInfo(ctypes.Structure):
    _fields_ = [("n_items", ctypes.c_uint32), ("smem_bytes", ctypes.c_uint32),
                ("total_tiles", ctypes.c_uint64), ("plan_bytes", ctypes.c_uint64),
                ("workspace_bytes", ctypes.c_uint64), ("cta_threads", ctypes.c_uint32),
                ("reserved", ctypes.c_uint32)]


class PcSource(ctypes.Structure):
    _fields_ = [("d_in", ctypes.c_void_p), ("n_samples", ctypes.c_uint64), ("d_out", ctypes.c_void_p),
                ("out_capacity", ctypes.c_uint64), ("d_out_bytes", ctypes.c_void_p),
                ("d_totals", ctypes.c_void_p)]


class PcSegmentsInfo(ctypes.Structure):
    _fields_ = [("n_sources", ctypes.c_uint32), ("dtype_bits", ctypes.c_uint32), ("variant", ctypes.c_uint32),
                ("smem_bytes", ctypes.c_uint32), ("has_totals", ctypes.c_uint32), ("reserved", ctypes.c_uint32),
                ("n_segments", ctypes.c_uint64), ("seg_stride", ctypes.c_uint64),
                ("plan_bytes", ctypes.c_uint64), ("workspace_bytes", ctypes.c_uint64)]


class PcStitchRegion(ctypes.Structure):
    _fields_ = [(name, ctypes.c_uint64) for name in (
        "total_bytes", "first_block", "n_blocks", "table_src", "table_dst", "table_bytes",
        "payload_src", "payload_dst", "payload_bytes", "pad_dst", "payload_start")]

    def as_dict(self):
        return {name: int(getattr(self, name)) for name, _ in self._fields_}


class PcError(RuntimeError):
    def __init__(self, code, what):
        msg = "%s: %s (status %d)" % (what, strerror(code) if _lib else "", code)
        super().__init__(msg)
        self.code = code


_lib = None


def load(path=LIB_PATH):
    """Load libpc.so (build it with paper_1805_01844_gb300.build.build())."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError("libpc.so not found at %s: build it first "
                           "(python -c 'import __graft_entry__ as g; g.build()')" % path)
    L = ctypes.CDLL(path)
    u64, u32, vp = ctypes.c_uint64, ctypes.c_uint32, ctypes.c_void_p
    pp = ctypes.POINTER(PcParams)
    u64p = ctypes.POINTER(ctypes.c_uint64)
    st = ctypes.c_int
    L.pc_bound.argtypes = [pp, u64, u64p]
    L.pc_bound.restype = st
    L.pc_workspace_size.argtypes = [pp, u64, u64p]
    L.pc_workspace_size.restype = st
    L.pc_compress.argtypes = [vp, u64, pp, vp, u64, vp, vp, u64, vp]
    L.pc_compress.restype = st
    L.pc_decompress.argtypes = [vp, u64, pp, vp, u64, vp, vp, u64, vp]
    L.pc_decompress.restype = st
    L.pc_parse_header.argtypes = [vp, u64, pp, u64p]
    L.pc_parse_header.restype = st
    L.pc_last_device_status.argtypes = [vp, vp]
    L.pc_last_device_status.restype = st
    L.pc_selftest_bounded_wait.argtypes = [vp, u64, u32, vp]
    L.pc_selftest_bounded_wait.restype = st
    L.pc_compress_noalloc.argtypes = [vp, u64, pp, vp, u64, vp, vp]
    L.pc_compress_noalloc.restype = st
    ip = ctypes.POINTER(PcBatchItem)
    fp = ctypes.POINTER(PcBatchInfo)
    L.pc_batch_describe.argtypes = [ip, u32, fp]
    L.pc_batch_describe.restype = st
    L.pc_batch_plan.argtypes = [ip, u32, fp, vp, vp]
    L.pc_batch_plan.restype = st
    L.pc_compress_batch.argtypes = [fp, vp, vp, u64, vp]
    L.pc_compress_batch.restype = st
    f32p = ctypes.c_void_p
    L.pc_segment_features.argtypes = [vp, u64, u32, f32p, vp]
    L.pc_segment_features.restype = st
    L.pc_mlp_forward.argtypes = [vp, f32p, u64, f32p, vp, vp]
    L.pc_mlp_forward.restype = st
    L.pc_mlp_grad.argtypes = [vp, f32p, vp, u64, f32p, f32p, vp]
    L.pc_mlp_grad.restype = st
    L.pc_mlp_adam.argtypes = [f32p, vp, f32p, f32p, f32p, u32, ctypes.c_float, vp]
    L.pc_mlp_adam.restype = st
    sp = ctypes.POINTER(PcSource)
    gp = ctypes.POINTER(PcSegmentsInfo)
    L.pc_segments_describe.argtypes = [sp, u32, u32, u32, gp]
    L.pc_segments_describe.restype = st
    L.pc_segments_plan.argtypes = [sp, u32, gp, vp, vp]
    L.pc_segments_plan.restype = st
    L.pc_segments_features.argtypes = [gp, vp, f32p, vp]
    L.pc_segments_features.restype = st
    L.pc_compress_segments.argtypes = [gp, vp, vp, vp, u64, vp]
    L.pc_compress_segments.restype = st
    rp = ctypes.POINTER(PcStitchRegion)
    L.pc_shard_range.argtypes = [pp, u64, u32, u32, u64p, u64p]
    L.pc_shard_range.restype = st
    L.pc_stitch_layout.argtypes = [pp, u64, u32, u32, u64p, rp]
    L.pc_stitch_layout.restype = st
    L.pc_stitch.argtypes = [vp, vp, u32, u32, u64, pp, vp, u64, vp, vp, u64, vp]
    L.pc_stitch.restype = st
    L.pc_slice.argtypes = [vp, u64, pp, u64, u64, vp, u64, vp, vp, u64, vp]
    L.pc_slice.restype = st
    L.pc_byte_histogram.argtypes = [vp, u64, vp, vp]
    L.pc_byte_histogram.restype = st
    L.pc_bound_v2.argtypes = [u32, u32, u32, u64, u64p]
    L.pc_bound_v2.restype = st
    L.pc_assemble_v2_workspace_size.argtypes = [u64, u64p]
    L.pc_assemble_v2_workspace_size.restype = st
    L.pc_assemble_v2.argtypes = [vp, u64, u64, u64, u32, u32, u32, vp, u64, vp, vp, u64, vp]
    L.pc_assemble_v2.restype = st
    L.pc_decompress_v2_workspace_size.argtypes = [u32, u32, u32, u64, u64p]
    L.pc_decompress_v2_workspace_size.restype = st
    L.pc_decompress_v2.argtypes = [vp, u64, u32, u32, u32, vp, u64, vp, vp, u64, vp]
    L.pc_decompress_v2.restype = st
    L.pc_strerror.argtypes = [st]
    L.pc_strerror.restype = ctypes.c_char_p
    _lib = L
    return L


def strerror(code):
    return load().pc_strerror(int(code)).decode()


def _check(code, what):
    if code != PC_OK:
        raise PcError(code, what)


def params(variant=BASIC, dtype_bits=16, word_bits=64, block_len=1024):
    return PcParams(int(variant), int(dtype_bits), int(word_bits), int(block_len))


def bound(p, n_samples):
    out = ctypes.c_uint64(0)
    _check(load().pc_bound(ctypes.byref(p), int(n_samples), ctypes.byref(out)), "pc_bound")
    return int(out.value)


def workspace_size(p, n_samples):
    out = ctypes.c_uint64(0)
    _check(load().pc_workspace_size(ctypes.byref(p), int(n_samples), ctypes.byref(out)),
           "pc_workspace_size")
    return int(out.value)


def parse_header(host_bytes):
    """(PcParams, n_samples) from the first 64 bytes of a stream (host bytes)."""
    buf = ctypes.create_string_buffer(bytes(host_bytes[:HEADER_BYTES]), HEADER_BYTES)
    p = PcParams()
    n = ctypes.c_uint64(0)
    _check(load().pc_parse_header(buf, len(host_bytes[:HEADER_BYTES]), ctypes.byref(p),
                                  ctypes.byref(n)), "pc_parse_header")
    return p, int(n.value)


def compress_raw(d_in, n_samples, p, d_out, out_capacity, d_out_bytes, d_ws, ws_bytes, stream):
    """pc_compress on raw device addresses (ints); returns the host status."""
    return load().pc_compress(d_in or None, int(n_samples), ctypes.byref(p), d_out,
                              int(out_capacity), d_out_bytes, d_ws, int(ws_bytes), stream or None)


def decompress_raw(d_in, in_bytes, p, d_out, cap_samples, d_n, d_ws, ws_bytes, stream):
    """pc_decompress on raw device addresses (ints); returns the host status."""
    return load().pc_decompress(d_in, int(in_bytes), ctypes.byref(p), d_out or None,
                                int(cap_samples), d_n, d_ws, int(ws_bytes), stream or None)


def last_device_status(d_ws, stream):
    return int(load().pc_last_device_status(d_ws, stream or None))


def selftest_bounded_wait(d_ws, ws_bytes, limit_us, stream):
    return int(load().pc_selftest_bounded_wait(d_ws, int(ws_bytes), int(limit_us), stream or None))


def compress_noalloc_raw(d_in, n_samples, p, d_out, out_capacity, d_out_bytes, stream):
    """pc_compress_noalloc on raw device addresses: no workspace argument, the
    library's static scratch is used.  Returns the host status."""
    return load().pc_compress_noalloc(d_in or None, int(n_samples), ctypes.byref(p), d_out,
                                      int(out_capacity), d_out_bytes, stream or None)


def batch_describe(items, cta_threads=256):
    """items: list of PcBatchItem.  Returns (ctypes array, PcBatchInfo)."""
    arr = (PcBatchItem * len(items))(*items)
    info = PcBatchInfo()
    info.cta_threads = cta_threads
    _check(load().pc_batch_describe(arr, len(items), ctypes.byref(info)), "pc_batch_describe")
    return arr, info


def batch_plan(arr, info, d_plan, stream):
    _check(load().pc_batch_plan(arr, info.n_items, ctypes.byref(info), d_plan, stream or None), "pc_batch_plan")


def compress_batch(info, d_plan, d_ws, ws_bytes, stream):
    """pc_compress_batch; returns the host status."""
    return load().pc_compress_batch(ctypes.byref(info), d_plan, d_ws, int(ws_bytes), stream or None)


def segments_describe(sources, dtype_bits, variant):
    """sources: list of PcSource.  Returns (ctypes array, PcSegmentsInfo)."""
    arr = (PcSource * len(sources))(*sources)
    info = PcSegmentsInfo()
    _check(load().pc_segments_describe(arr, len(sources), dtype_bits, variant, ctypes.byref(info)),
           "pc_segments_describe")
    return arr, info


def segments_plan(arr, info, d_plan, stream):
    _check(load().pc_segments_plan(arr, info.n_sources, ctypes.byref(info), d_plan, stream or None),
           "pc_segments_plan")


def segments_features(info, d_plan, d_features, stream):
    _check(load().pc_segments_features(ctypes.byref(info), d_plan, d_features, stream or None),
           "pc_segments_features")


def compress_segments(info, d_plan, d_options, d_ws, ws_bytes, stream):
    """pc_compress_segments; returns the host status."""
    return load().pc_compress_segments(ctypes.byref(info), d_plan, d_options, d_ws, int(ws_bytes), stream or None)


def segment_stride(dtype_bits, variant):
    """Output slot bytes per segment (pc_segments_describe of a one-segment
    probe; needs no device memory: the pointers are never dereferenced)."""
    src = PcSource(16, 1, 16, 1 << 40, 8, None)
    _, info = segments_describe([src], dtype_bits, variant)
    return info.seg_stride



def shard_range(p, n_samples, n_shards, shard):
    """(first sample, sample count) of block-aligned shard `shard` of `n_shards`."""
    f, c = ctypes.c_uint64(0), ctypes.c_uint64(0)
    _check(load().pc_shard_range(ctypes.byref(p), int(n_samples), int(n_shards), int(shard), ctypes.byref(f),
                                 ctypes.byref(c)), "pc_shard_range")
    return int(f.value), int(c.value)


def stitch_layout(p, n_samples, n_shards, shard, shard_bytes):
    """Placement of shard `shard` in the whole stream (dict of byte offsets),
    from every shard's stream size (host integers)."""
    arr = (ctypes.c_uint64 * int(n_shards))(*[int(b) for b in shard_bytes])
    r = PcStitchRegion()
    _check(load().pc_stitch_layout(ctypes.byref(p), int(n_samples), int(n_shards), int(shard), arr,
                                   ctypes.byref(r)), "pc_stitch_layout")
    return r.as_dict()


def stitch_raw(d_shard, d_shard_bytes, n_shards, shard, n_samples, p, d_out, out_capacity, d_out_bytes, d_ws,
               ws_bytes, stream):
    """pc_stitch on raw device addresses; returns the host status."""
    return load().pc_stitch(d_shard, d_shard_bytes, int(n_shards), int(shard), int(n_samples), ctypes.byref(p),
                            d_out, int(out_capacity), d_out_bytes or None, d_ws, int(ws_bytes), stream or None)


def slice_raw(d_in, in_bytes, p, first_block, n_blocks, d_out, out_capacity, d_out_bytes, d_ws, ws_bytes, stream):
    """pc_slice on raw device addresses; returns the host status."""
    return load().pc_slice(d_in, int(in_bytes), ctypes.byref(p), int(first_block), int(n_blocks), d_out,
                           int(out_capacity), d_out_bytes, d_ws, int(ws_bytes), stream or None)


def byte_histogram_raw(d_bytes, n_bytes, d_hist, stream):
    """pc_byte_histogram on raw device addresses; returns the host status."""
    return load().pc_byte_histogram(d_bytes or None, int(n_bytes), d_hist, stream or None)


def bound_v2(variant, dtype_bits, seg_len, n):
    out = ctypes.c_uint64(0)
    _check(load().pc_bound_v2(variant, dtype_bits, seg_len, int(n), ctypes.byref(out)), "pc_bound_v2")
    return int(out.value)


def assemble_v2_workspace_size(n_segments):
    out = ctypes.c_uint64(0)
    _check(load().pc_assemble_v2_workspace_size(int(n_segments), ctypes.byref(out)),
           "pc_assemble_v2_workspace_size")
    return int(out.value)


def decompress_v2_workspace_size(variant, dtype_bits, seg_len, capacity):
    out = ctypes.c_uint64(0)
    _check(load().pc_decompress_v2_workspace_size(variant, dtype_bits, seg_len, int(capacity), ctypes.byref(out)),
           "pc_decompress_v2_workspace_size")
    return int(out.value)


def assemble_v2_raw(d_slots, seg_stride, n_segments, n, seg_len, dtype_bits, variant, d_out, out_capacity,
                    d_out_bytes, d_ws, ws_bytes, stream):
    """pc_assemble_v2 on raw device addresses; returns the host status."""
    return load().pc_assemble_v2(d_slots or None, int(seg_stride), int(n_segments), int(n), seg_len, dtype_bits,
                                 variant, d_out, int(out_capacity), d_out_bytes, d_ws, int(ws_bytes),
                                 stream or None)


def decompress_v2_raw(d_in, in_bytes, variant, dtype_bits, seg_len, d_out, cap, d_n, d_ws, ws_bytes, stream):
    """pc_decompress_v2 on raw device addresses; returns the host status."""
    return load().pc_decompress_v2(d_in, int(in_bytes), variant, dtype_bits, seg_len, d_out or None, int(cap), d_n,
                                   d_ws, int(ws_bytes), stream or None)
