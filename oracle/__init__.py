"""CPU oracle for polynomial lossless compression (arXiv:1805.01844).

TEST INFRASTRUCTURE ONLY: imported by the test suite, the smoke check and the
benchmark's CPU-baseline / reference legs, never by the product path.  The
arithmetic lives in ``poly_oracle.c`` (plain C, 128-bit intermediates); this
module only marshals arguments through ctypes.

Functions and the passage each follows:
  eq1_p            Sec. 3.1, Eq. 1 (integer form)
  basic_pack/...   Sec. 3.1, Eq. 2 and the polynomial division that inverts it
  adv_schedule     Sec. 3.2, the split-base series (p_i, R_i, R'_i, q_i)
  adv_pack/...     Sec. 3.2, word s_i of the series and its inverse
  compress/...     Sec. 3.3 blocked compression, Fig. 2 block header
  compress_v2/...  the same with (L, w) chosen per segment of the data, one
                   code byte each (format version 2; the block-size choice of
                   Sec. 3.3 and Sec. 4.2, Fig. 7)
"""
import ctypes

import numpy as np

from . import build as _build

_lib = None

OK, ERR_INVALID_ARG, ERR_CAPACITY, ERR_CORRUPT, ERR_UNSUPPORTED = 0, 1, 2, 3, 6
HEADER_BYTES = 64

_u64p = ctypes.POINTER(ctypes.c_uint64)
_u32p = ctypes.POINTER(ctypes.c_uint32)


class OracleError(RuntimeError):
    def __init__(self, code, what):
        super().__init__("%s failed with status %d" % (what, code))
        self.code = code


def lib():
    global _lib
    if _lib is None:
        L = ctypes.CDLL(_build.build())
        u64, u32, uint = ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint
        vp = ctypes.c_void_p
        L.po_eq1_p.argtypes = [u64, uint]
        L.po_eq1_p.restype = uint
        L.po_basic_count.argtypes = [u64, uint, u64]
        L.po_basic_count.restype = u64
        L.po_basic_pack.argtypes = [u64, uint, _u64p, u64, _u64p]
        L.po_basic_pack.restype = u64
        L.po_basic_unpack.argtypes = [u64, uint, _u64p, u64, u64, _u64p]
        L.po_basic_unpack.restype = ctypes.c_int
        L.po_adv_schedule.argtypes = [u64, uint, u64, _u32p, _u64p, _u64p, _u64p, u64]
        L.po_adv_schedule.restype = u64
        L.po_adv_count.argtypes = [u64, uint, u64]
        L.po_adv_count.restype = u64
        L.po_adv_pack.argtypes = [u64, uint, _u64p, u64, _u64p]
        L.po_adv_pack.restype = u64
        L.po_adv_unpack.argtypes = [u64, uint, _u64p, u64, u64, _u64p]
        L.po_adv_unpack.restype = ctypes.c_int
        L.po_bound.argtypes = [uint, uint, uint, u64, u64, _u64p]
        L.po_bound.restype = ctypes.c_int
        L.po_stream_bytes.argtypes = [uint, uint, u64, u64]
        L.po_stream_bytes.restype = u64
        L.po_compress.argtypes = [vp, u64, uint, uint, uint, u64, vp, u64, _u64p]
        L.po_compress.restype = ctypes.c_int
        L.po_decompress.argtypes = [vp, u64, vp, u64, _u64p]
        L.po_decompress.restype = ctypes.c_int
        L.po_bound_v2.argtypes = [uint, uint, u64, u64, _u64p]
        L.po_bound_v2.restype = ctypes.c_int
        L.po_compress_v2.argtypes = [vp, u64, uint, uint, u64, vp, vp, u64, _u64p]
        L.po_compress_v2.restype = ctypes.c_int
        L.po_decompress_v2.argtypes = [vp, u64, vp, u64, _u64p]
        L.po_decompress_v2.restype = ctypes.c_int
        _lib = L
    return _lib


def _u64arr(values):
    a = np.ascontiguousarray(np.asarray(values, dtype=np.uint64))
    return a, a.ctypes.data_as(_u64p)


def eq1_p(B, w):
    """Eq. 1: the largest p with B**p <= 2**w - 1 (B >= 2)."""
    return int(lib().po_eq1_p(int(B), int(w)))


def pack_count(variant, B, w, n_b):
    if variant == 0:
        return int(lib().po_basic_count(int(B), int(w), int(n_b)))
    return int(lib().po_adv_count(int(B), int(w), int(n_b)))


def pack_block(variant, B, w, u):
    """Pack offsets u (each in [0, B)) into words of w bits (1 <= w <= 64)."""
    u, up = _u64arr(u)
    n = pack_count(variant, B, w, len(u))
    out = np.zeros(max(n, 1), dtype=np.uint64)
    fn = lib().po_basic_pack if variant == 0 else lib().po_adv_pack
    got = fn(int(B), int(w), up, len(u), out.ctypes.data_as(_u64p))
    assert got == n
    return out[:n].copy()


def unpack_block(variant, B, w, words, n_b):
    """Inverse of pack_block; raises OracleError(ERR_CORRUPT) on a bad word."""
    words, wp = _u64arr(words)
    out = np.zeros(max(n_b, 1), dtype=np.uint64)
    fn = lib().po_basic_unpack if variant == 0 else lib().po_adv_unpack
    st = fn(int(B), int(w), wp, len(words), int(n_b), out.ctypes.data_as(_u64p))
    if st != OK:
        raise OracleError(st, "unpack_block")
    return out[:n_b].copy()


def adv_schedule(B, w, n_b):
    """Split-base series of Sec. 3.2: list of (p_i, R_i, R'_i, q_i) per word."""
    n = pack_count(1, B, w, n_b)
    p = np.zeros(max(n, 1), dtype=np.uint32)
    R = np.zeros(max(n, 1), dtype=np.uint64)
    Rp = np.zeros(max(n, 1), dtype=np.uint64)
    q = np.zeros(max(n, 1), dtype=np.uint64)
    lib().po_adv_schedule(int(B), int(w), int(n_b), p.ctypes.data_as(_u32p),
                          R.ctypes.data_as(_u64p), Rp.ctypes.data_as(_u64p),
                          q.ctypes.data_as(_u64p), n)
    return [(int(p[i]), int(R[i]), int(Rp[i]), int(q[i])) for i in range(n)]


def bound(variant, dtype_bits, word_bits, block_len, n):
    out = ctypes.c_uint64(0)
    st = lib().po_bound(variant, dtype_bits, word_bits, block_len, n, ctypes.byref(out))
    if st != OK:
        raise OracleError(st, "bound")
    return int(out.value)


def stream_bytes(dtype_bits, word_bits, n_blocks, payload_words):
    return int(lib().po_stream_bytes(dtype_bits, word_bits, n_blocks, payload_words))


def compress(x, variant, word_bits, block_len):
    """Blocked compression of a 1-D uint16/uint32 array into a byte stream."""
    x = np.ascontiguousarray(x)
    if x.dtype == np.uint16:
        d = 16
    elif x.dtype == np.uint32:
        d = 32
    else:
        raise TypeError("oracle.compress takes uint16 or uint32 samples")
    cap = bound(variant, d, word_bits, block_len, x.size)
    out = np.zeros(cap, dtype=np.uint8)
    nbytes = ctypes.c_uint64(0)
    st = lib().po_compress(x.ctypes.data, x.size, variant, d, word_bits, block_len,
                           out.ctypes.data, cap, ctypes.byref(nbytes))
    if st != OK:
        raise OracleError(st, "compress")
    return out[:nbytes.value].tobytes()


def header(stream):
    """Decoded header fields of a stream (no validation beyond parsing)."""
    b = bytes(stream[:HEADER_BYTES])
    return dict(magic=b[0:4], version=int.from_bytes(b[4:6], "little"),
                variant=b[6], dtype_bits=b[7], word_bits=b[8],
                block_len=int.from_bytes(b[12:16], "little"),
                n_samples=int.from_bytes(b[16:24], "little"),
                n_blocks=int.from_bytes(b[24:32], "little"),
                payload_words=int.from_bytes(b[32:40], "little"))


def decompress(stream, capacity=None):
    """Inverse of compress; raises OracleError on a corrupt stream."""
    buf = np.frombuffer(bytes(stream), dtype=np.uint8)
    h = header(stream) if len(buf) >= HEADER_BYTES else dict(dtype_bits=16, n_samples=0)
    dt = np.uint32 if h["dtype_bits"] == 32 else np.uint16
    if capacity is None:
        capacity = h["n_samples"] if h["n_samples"] < (1 << 34) else 0
    out = np.zeros(max(capacity, 1), dtype=dt)
    n_out = ctypes.c_uint64(0)
    st = lib().po_decompress(buf.ctypes.data if len(buf) else None, len(buf),
                             out.ctypes.data, capacity, ctypes.byref(n_out))
    if st != OK:
        raise OracleError(st, "decompress")
    return out[:n_out.value].copy()


def v2_code(block_len, word_bits):
    """Format-2 code byte of a segment: log2(L) | (w == 64) << 7."""
    k = int(block_len).bit_length() - 1
    if block_len != 1 << k or k > 13 or word_bits not in (32, 64):
        raise ValueError("block length must be a power of two <= 8192, words 32 or 64 bits")
    return k | (0x80 if word_bits == 64 else 0)


def bound_v2(variant, dtype_bits, seg_len, n):
    out = ctypes.c_uint64(0)
    st = lib().po_bound_v2(variant, dtype_bits, seg_len, n, ctypes.byref(out))
    if st != OK:
        raise OracleError(st, "bound_v2")
    return int(out.value)


def compress_v2(x, variant, seg_len, codes):
    """Format-2 stream of x: segment s of seg_len samples compressed with the
    (L, w) of codes[s] (see v2_code)."""
    x = np.ascontiguousarray(x)
    d = {np.dtype(np.uint16): 16, np.dtype(np.uint32): 32}[x.dtype]
    codes = np.ascontiguousarray(np.asarray(codes, dtype=np.uint8))
    n_seg = -(-x.size // seg_len)
    if codes.size < n_seg:
        raise ValueError("one code per segment")
    cap = bound_v2(variant, d, seg_len, x.size)
    out = np.zeros(cap, dtype=np.uint8)
    nbytes = ctypes.c_uint64(0)
    st = lib().po_compress_v2(x.ctypes.data, x.size, variant, d, seg_len, codes.ctypes.data if codes.size else None,
                              out.ctypes.data, cap, ctypes.byref(nbytes))
    if st != OK:
        raise OracleError(st, "compress_v2")
    return out[:nbytes.value].tobytes()


def header_v2(stream):
    b = bytes(stream[:HEADER_BYTES])
    return dict(magic=b[0:4], version=int.from_bytes(b[4:6], "little"), variant=b[6], dtype_bits=b[7],
                seg_len=int.from_bytes(b[12:16], "little"), n_samples=int.from_bytes(b[16:24], "little"),
                n_segments=int.from_bytes(b[24:32], "little"), body_bytes=int.from_bytes(b[32:40], "little"))


def decompress_v2(stream, capacity=None):
    """Inverse of compress_v2; raises OracleError on a corrupt stream."""
    buf = np.frombuffer(bytes(stream), dtype=np.uint8)
    h = header_v2(stream) if len(buf) >= HEADER_BYTES else dict(dtype_bits=16, n_samples=0)
    dt = np.uint32 if h["dtype_bits"] == 32 else np.uint16
    if capacity is None:
        capacity = h["n_samples"] if h["n_samples"] < (1 << 34) else 0
    out = np.zeros(max(capacity, 1), dtype=dt)
    n_out = ctypes.c_uint64(0)
    st = lib().po_decompress_v2(buf.ctypes.data if len(buf) else None, len(buf), out.ctypes.data, capacity,
                                ctypes.byref(n_out))
    if st != OK:
        raise OracleError(st, "decompress_v2")
    return out[:n_out.value].copy()
