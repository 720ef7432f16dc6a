"""Round trips of host buffers through the GPU codec, pipelined over
consecutive calls: the upload of one call's samples overlaps the downloads of
the previous call's stream and decoded samples (a host link moves data both
ways at once), and the codec kernels run on their own CUDA stream between
them.  Each call is an ordinary pc_compress / pc_decompress pair on pinned
host memory; only the ordering of the copies changes.

    rt = RoundTrip(variant, dtype_bits, word_bits, block_len, n_samples)
    for host_in in chunks:            # pinned int16 / int32 tensors of n samples
        rt.submit(host_in)            # returns at once
        done = rt.completed()         # (host stream bytes, host samples) of earlier calls
    rt.drain()

Two slots of device and host buffers alternate, so at most two calls are in
flight.  The stream of a call is read back at its exact size, which the host
learns once that call's compression has finished (while the next call's
upload is already queued).
"""
from . import native

__all__ = ["RoundTrip"]


def _torch():
    import torch

    return torch


class RoundTrip:
    def __init__(self, variant, dtype_bits, word_bits, block_len, n_samples, device="cuda"):
        torch = _torch()
        from . import Codec

        self.device = torch.device(device)
        self.n = int(n_samples)
        dt = torch.int16 if dtype_bits == 16 else torch.int32
        self.codecs = [Codec(variant, dtype_bits, word_bits, block_len, max_samples=self.n, device=self.device)
                       for _ in range(2)]
        cap = self.codecs[0].bound(self.n)
        self.xin = [torch.empty(self.n, dtype=dt, device=self.device) for _ in range(2)]
        self.sbuf = [torch.empty(cap, dtype=torch.uint8, device=self.device) for _ in range(2)]
        self.ybuf = [torch.empty(self.n, dtype=dt, device=self.device) for _ in range(2)]
        self.host_stream = [torch.empty(cap, dtype=torch.uint8, pin_memory=True) for _ in range(2)]
        self.host_out = [torch.empty(self.n, dtype=dt, pin_memory=True) for _ in range(2)]
        self.s_up = torch.cuda.Stream(self.device)
        self.s_codec = torch.cuda.Stream(self.device)
        self.s_down = torch.cuda.Stream(self.device)
        ev = lambda: [torch.cuda.Event() for _ in range(2)]  # noqa: E731
        self.ev_up, self.ev_codec, self.ev_down = ev(), ev(), ev()
        self.k = 0
        self.pending = None  # slot of the call whose downloads are not queued yet
        self.done = []

    def submit(self, host_in):
        """Queue one round trip of host_in (pinned, n samples)."""
        b = self.k % 2
        self.k += 1
        codec = self.codecs[b]
        # the slot's previous downloads must be done before its buffers are reused
        self.s_up.wait_event(self.ev_down[b])
        with _torch().cuda.stream(self.s_up):
            self.xin[b].copy_(host_in, non_blocking=True)
        self.ev_up[b].record(self.s_up)
        self.s_codec.wait_event(self.ev_up[b])
        codec.compress(self.xin[b], out=self.sbuf[b], stream=self.s_codec)
        codec.decompress(self.sbuf[b], self.sbuf[b].numel(), self.n, out=self.ybuf[b], stream=self.s_codec)
        self.ev_codec[b].record(self.s_codec)
        if self.pending is not None:
            self._download(self.pending)
        self.pending = b

    def _download(self, b):
        torch = _torch()
        self.ev_codec[b].synchronize()
        nbytes = int(self.codecs[b]._count[0].item())
        self.s_down.wait_event(self.ev_codec[b])
        with torch.cuda.stream(self.s_down):
            self.host_stream[b][:nbytes].copy_(self.sbuf[b][:nbytes], non_blocking=True)
            self.host_out[b].copy_(self.ybuf[b], non_blocking=True)
        self.ev_down[b].record(self.s_down)
        self.done.append((b, nbytes))

    def drain(self):
        """Queue the last call's downloads and wait for everything."""
        if self.pending is not None:
            self._download(self.pending)
            self.pending = None
        self.s_down.synchronize()
        for codec in self.codecs:  # device-side status of both slots' last calls
            st = codec.device_status(stream=self.s_codec)
            if st != native.PC_OK:
                raise native.PcError(st, "round trip (device)")

    def completed(self):
        """(slot, stream bytes) of the calls whose downloads were queued since
        the last call; their host buffers are valid once drain() returned or
        ev_down of the slot completed."""
        out, self.done = self.done, []
        return out
