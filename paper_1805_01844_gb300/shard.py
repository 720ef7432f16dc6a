"""One stream as block-aligned shards (Sec. 3.3: blocks are independent;
Sec. 4.3: a stream is readable by part).

Each shard is a range of whole blocks, compressed by pc_compress into an
ordinary stream; the only exchange between shards is every shard's stream
size (8 bytes each), from which pc_stitch places each shard's table entries
and payload in the whole stream -- byte for byte the stream one pc_compress
call over all samples would write.  pc_slice cuts the stream of a block range
back out, so each shard decompresses its own blocks.

    ShardedCodec      K shards on one device (in-process), for tests and for
                      splitting work that does not fit one call
    exchange_sizes    all-gather of the shards' stream sizes across ranks
    compress_shard_and_place
                      one rank's part under torch.distributed: compress the
                      rank's shard, exchange sizes, stitch its pieces into a
                      whole-stream buffer on this rank (the other ranks'
                      byte ranges are left as they are)

All compression, stitching and slicing runs in libpc.so's kernels; this module
only sequences the calls and moves sizes between ranks.
"""
from . import native

__all__ = ["ShardedCodec", "exchange_sizes", "compress_shard_and_place"]


def _torch():
    import torch

    return torch


def _stream(device, stream=None):
    torch = _torch()
    return (stream if stream is not None else torch.cuda.current_stream(device)).cuda_stream


class ShardedCodec:
    """n_samples samples of one stream as n_shards block-aligned shards on one
    device: compress every shard, stitch the whole stream; slice a block range
    back out and decompress it."""

    def __init__(self, variant, dtype_bits, word_bits, block_len, n_samples, n_shards, device="cuda"):
        torch = _torch()
        from . import Codec

        self.p = native.params(variant, dtype_bits, word_bits, block_len)
        self.n = int(n_samples)
        self.k = int(n_shards)
        self.device = torch.device(device)
        self.ranges = [native.shard_range(self.p, self.n, self.k, j) for j in range(self.k)]
        self.codecs = [Codec(variant, dtype_bits, word_bits, block_len, max_samples=max(c, 1), device=self.device)
                       for _, c in self.ranges]
        L = self.p.block_len
        self.shard_bufs = [torch.empty(native.bound(self.p, -(-c // L) * L), dtype=torch.uint8, device=self.device)
                           for _, c in self.ranges]
        # every shard's stream size lands in its slot of one device array: the
        # array pc_stitch reads (on several ranks, the all-gathered sizes)
        self.sizes = torch.zeros(self.k, dtype=torch.int64, device=self.device)
        self.total = torch.zeros(1, dtype=torch.int64, device=self.device)
        self.ws = torch.zeros(64, dtype=torch.uint8, device=self.device)

    def bound(self):
        return native.bound(self.p, self.n)

    def compress(self, x, out=None, stream=None):
        """Compress a contiguous CUDA tensor of n_samples samples shard by
        shard and stitch the whole stream into `out`.  Returns (out, device
        int64 scalar with the stream size).  Asynchronous."""
        torch = _torch()
        if x.numel() != self.n:
            raise ValueError("expected %d samples, got %d" % (self.n, x.numel()))
        if out is None:
            out = torch.empty(self.bound(), dtype=torch.uint8, device=self.device)
        s = _stream(self.device, stream)
        for j, (f, c) in enumerate(self.ranges):
            codec = self.codecs[j]
            ws = codec._ensure_ws(max(c, 1))
            xs = x[f:f + c]
            if c and xs.data_ptr() % 16:  # a shard start that is not 16-byte aligned is compressed from a copy
                xs = xs.clone()
            st = native.compress_raw(xs.data_ptr() if c else None, c, self.p, self.shard_bufs[j].data_ptr(),
                                     self.shard_bufs[j].numel(), self.sizes.data_ptr() + 8 * j, ws.data_ptr(),
                                     codec._ws_bytes, s)
            if st != native.PC_OK:
                raise native.PcError(st, "pc_compress (shard %d)" % j)
        for j in range(self.k):
            st = native.stitch_raw(self.shard_bufs[j].data_ptr(), self.sizes.data_ptr(), self.k, j, self.n, self.p,
                                   out.data_ptr(), out.numel(), self.total.data_ptr() if j == self.k - 1 else None,
                                   self.ws.data_ptr(), self.ws.numel(), s)
            if st != native.PC_OK:
                raise native.PcError(st, "pc_stitch (shard %d)" % j)
        return out, self.total

    def device_status(self, stream=None):
        """Synchronise; the first device-side error of the shards'
        compressions and of the stitching (PC_OK if none)."""
        s = _stream(self.device, stream)
        for codec in self.codecs:
            st = codec.device_status(stream)
            if st != native.PC_OK:
                return st
        return native.last_device_status(self.ws.data_ptr(), s)

    def slice(self, stream_buf, in_bytes, first_block, n_blocks, out=None, stream=None):
        """The stream of blocks [first_block, first_block + n_blocks) of a
        whole stream.  Returns (buffer, device int64 scalar with its size)."""
        torch = _torch()
        cap = native.bound(self.p, n_blocks * self.p.block_len)
        if out is None:
            out = torch.empty(max(cap, 64), dtype=torch.uint8, device=self.device)
        nbytes = torch.zeros(1, dtype=torch.int64, device=self.device)
        st = native.slice_raw(stream_buf.data_ptr(), in_bytes, self.p, first_block, n_blocks, out.data_ptr(),
                              out.numel(), nbytes.data_ptr(), self.ws.data_ptr(), self.ws.numel(),
                              _stream(self.device, stream))
        if st != native.PC_OK:
            raise native.PcError(st, "pc_slice")
        return out, nbytes

    def decompress(self, stream_buf, in_bytes, out=None, stream=None):
        """Decompress a whole stream shard by shard: each shard's block range
        is sliced out and decoded into its place in `out`."""
        torch = _torch()
        dt = torch.int16 if self.p.dtype_bits == 16 else torch.int32
        if out is None:
            out = torch.empty(max(self.n, 1), dtype=dt, device=self.device)
        L = self.p.block_len
        for j, (f, c) in enumerate(self.ranges):
            if c == 0:
                continue
            piece, nbytes = self.slice(stream_buf, in_bytes, f // L, -(-c // L), out=self.shard_bufs[j], stream=stream)
            st = native.last_device_status(self.ws.data_ptr(), _stream(self.device, stream))
            if st != native.PC_OK:
                raise native.PcError(st, "pc_slice (device)")
            codec = self.codecs[j]
            dst = out[f:f + c]
            if dst.data_ptr() % 16 == 0:
                codec.decompress(piece, int(nbytes.item()), c, out=dst, stream=stream)
            else:  # a shard start that is not 16-byte aligned decodes into an aligned buffer first
                tmp, _ = codec.decompress(piece, int(nbytes.item()), c, stream=stream)
                dst.copy_(tmp[:c])
        return out


def exchange_sizes(local_size, group=None):
    """All-gather of every rank's stream size (an int64 tensor of one element
    on this rank's device, as pc_compress wrote it): the sharded stream's one
    exchange, 8 bytes per rank.  Returns an int64 tensor [world size]."""
    torch = _torch()
    import torch.distributed as dist

    world = dist.get_world_size(group)
    sizes = torch.empty(world, dtype=torch.int64, device=local_size.device)
    dist.all_gather_into_tensor(sizes, local_size.reshape(1), group=group)
    return sizes


def compress_shard_and_place(x_shard, p, n_total, out, group=None, stream=None):
    """One rank's part of a sharded stream under torch.distributed: rank r
    compresses shard r of the world size (x_shard holds exactly the samples of
    native.shard_range), exchanges stream sizes with the other ranks, and
    stitches its own pieces into `out` (a whole-stream buffer on this rank;
    rank 0 also writes the header, the last rank the table padding).  Returns
    (sizes tensor, layout dict of this rank's byte ranges, device int64 scalar
    with the whole stream's size on the last rank)."""
    torch = _torch()
    import torch.distributed as dist
    from . import Codec

    rank, world = dist.get_rank(group), dist.get_world_size(group)
    f, c = native.shard_range(p, n_total, world, rank)
    if x_shard.numel() != c:
        raise ValueError("rank %d's shard has %d samples, expected %d" % (rank, x_shard.numel(), c))
    dev = x_shard.device
    codec = Codec(p.variant, p.dtype_bits, p.word_bits, p.block_len, max_samples=max(c, 1), device=dev)
    buf = torch.empty(native.bound(p, c), dtype=torch.uint8, device=dev)
    _, nbytes = codec.compress(x_shard, out=buf, stream=stream)
    sizes = exchange_sizes(nbytes, group)
    ws = torch.zeros(64, dtype=torch.uint8, device=dev)
    total = torch.zeros(1, dtype=torch.int64, device=dev)
    st = native.stitch_raw(buf.data_ptr(), sizes.data_ptr(), world, rank, n_total, p, out.data_ptr(), out.numel(),
                           total.data_ptr(), ws.data_ptr(), ws.numel(), _stream(dev, stream))
    if st != native.PC_OK:
        raise native.PcError(st, "pc_stitch")
    layout = native.stitch_layout(p, n_total, world, rank, sizes.cpu().tolist())
    return sizes, layout, total
