"""GB300-native polynomial lossless compression (arXiv:1805.01844).

Blocked polynomial packing of small-range integer samples: per block the
minimum and the base B = max - min + 1 (Sec. 3.1), then the offsets as base-B
digits in 32- or 64-bit words, basic (Eq. 2) or split-base advanced
(Sec. 3.2); decompression by repeated division.  The work runs in the CUDA
kernels of libpc.so (C ABI in include/pc.h); this package only marshals
torch device tensors into that ABI.

    import torch, paper_1805_01844_gb300 as pc
    codec = pc.Codec(variant=pc.BASIC, dtype_bits=16, word_bits=64, block_len=1024)
    stream, nbytes = codec.compress(x_cuda_int16)        # async, nbytes on device
    y, n = codec.decompress(stream, int(nbytes.item()), x.numel())
"""
from . import native
from .native import ADVANCED, BASIC, PcError

__all__ = ["Codec", "BASIC", "ADVANCED", "PcError", "compress", "decompress", "native"]


def _torch():
    import torch

    return torch


def _dtype_bits(t):
    torch = _torch()
    if t.dtype in (torch.int16, getattr(torch, "uint16", None)):
        return 16
    if t.dtype in (torch.int32, getattr(torch, "uint32", None)):
        return 32
    raise TypeError("samples must be 16- or 32-bit integers (int16/uint16/int32/uint32), got %s" % t.dtype)


def _stream_handle(stream, device):
    torch = _torch()
    s = stream if stream is not None else torch.cuda.current_stream(device)
    return s.cuda_stream


class Codec:
    """Compression parameters plus the device buffers one call needs.

    The workspace is sized once for `max_samples` and reused; calls that
    share a Codec must not overlap on the GPU (they share the workspace)."""

    def __init__(self, variant=BASIC, dtype_bits=16, word_bits=64, block_len=1024,
                 max_samples=0, device="cuda"):
        torch = _torch()
        self.params = native.params(variant, dtype_bits, word_bits, block_len)
        self.device = torch.device(device)
        self._ws = None
        self._ws_bytes = 0
        self._count = torch.zeros(2, dtype=torch.int64, device=self.device)
        if max_samples:
            self._ensure_ws(max_samples)

    # -- buffers
    def _ensure_ws(self, n):
        need = native.workspace_size(self.params, n)
        if self._ws is None or self._ws_bytes < need:
            torch = _torch()
            self._ws = torch.empty((need + 15) // 16 * 16, dtype=torch.uint8, device=self.device)
            self._ws_bytes = self._ws.numel()
        return self._ws

    def bound(self, n_samples):
        return native.bound(self.params, n_samples)

    # -- the two calls of the C ABI
    def compress(self, x, out=None, stream=None):
        """Compress a contiguous CUDA tensor of samples.  Returns (stream
        buffer of pc_bound bytes, int64 device scalar with the stream size).
        Asynchronous on `stream` (default: the current stream)."""
        torch = _torch()
        if not x.is_cuda or not x.is_contiguous():
            raise ValueError("compress takes a contiguous CUDA tensor")
        if _dtype_bits(x) != self.params.dtype_bits:
            raise TypeError("sample width %d does not match the codec's dtype_bits %d"
                            % (_dtype_bits(x), self.params.dtype_bits))
        n = x.numel()
        cap = self.bound(n)
        if out is None:
            out = torch.empty(cap, dtype=torch.uint8, device=x.device)
        ws = self._ensure_ws(n)
        nbytes = self._count[0:1]
        st = native.compress_raw(x.data_ptr() if n else None, n, self.params, out.data_ptr(),
                                 out.numel(), nbytes.data_ptr(), ws.data_ptr(), self._ws_bytes,
                                 _stream_handle(stream, x.device))
        if st != native.PC_OK:
            raise PcError(st, "pc_compress")
        return out, nbytes

    def decompress(self, stream_buf, in_bytes, capacity, out=None, stream=None):
        """Decompress `in_bytes` bytes of a CUDA uint8 stream buffer into a
        tensor of `capacity` samples.  Returns (samples, int64 device scalar
        with the decoded sample count).  Asynchronous."""
        torch = _torch()
        dt = torch.int16 if self.params.dtype_bits == 16 else torch.int32
        if out is None:
            out = torch.empty(max(int(capacity), 1), dtype=dt, device=stream_buf.device)
        ws = self._ensure_ws(capacity)
        n_out = self._count[1:2]
        st = native.decompress_raw(stream_buf.data_ptr(), in_bytes, self.params, out.data_ptr(),
                                   capacity, n_out.data_ptr(), ws.data_ptr(), self._ws_bytes,
                                   _stream_handle(stream, stream_buf.device))
        if st != native.PC_OK:
            raise PcError(st, "pc_decompress")
        return out, n_out

    def device_status(self, stream=None):
        """Synchronise and return the device-side status of the last call."""
        if self._ws is None:
            return native.PC_OK
        return native.last_device_status(self._ws.data_ptr(), _stream_handle(stream, self.device))


def compress(x, variant=BASIC, word_bits=64, block_len=1024):
    """Synchronous convenience: compress `x` and return the stream as a CUDA
    uint8 tensor of exactly the stream's size."""
    codec = Codec(variant, _dtype_bits(x), word_bits, block_len, device=x.device)
    buf, nbytes = codec.compress(x)
    st = codec.device_status()
    if st != native.PC_OK:
        raise PcError(st, "pc_compress (device)")
    return buf[: int(nbytes.item())]


def decompress(stream_buf):
    """Synchronous convenience: decompress a CUDA uint8 stream tensor."""
    head = stream_buf[: native.HEADER_BYTES].cpu().numpy().tobytes()
    p, n = native.parse_header(head)
    codec = Codec(p.variant, p.dtype_bits, p.word_bits, p.block_len, device=stream_buf.device)
    out, n_out = codec.decompress(stream_buf, stream_buf.numel(), n)
    st = codec.device_status()
    if st != native.PC_OK:
        raise PcError(st, "pc_decompress (device)")
    return out[:n]
