"""Batches of independent streams in one launch (pc_batch_* in include/pc.h),
and an autotuner for the block length and word size of each stream.

Marshalling only: the compression itself is the library's persistent batch
kernel.  A Batch can be captured in a CUDA graph (a memset and one kernel)
and replayed while its tensors stay in place."""
import torch

from . import native
from . import _dtype_bits, _stream_handle


class Batch:
    """Compress `tensors` (CUDA, contiguous, 16/32-bit) with per-stream
    `params` (native.PcParams) in one launch; outputs are v1 streams."""

    def __init__(self, tensors, params, device=None, outs=None, workspace=None, stream=None, cta_threads=256):
        """outs: optional caller-owned uint8 output tensors (one per item, each
        at least pc_bound bytes, 16-byte aligned); workspace: optional
        caller-owned uint8 tensor reused across launches; cta_threads: 128 or
        256 threads per CTA of the launch (see autotune_threads)."""
        assert len(tensors) == len(params) and tensors
        self.device = device or tensors[0].device
        self.tensors = tensors
        self.params = params
        items = []
        self.nbytes = torch.zeros(len(tensors), dtype=torch.int64, device=self.device)
        caps, offs, total = [], [], 0
        for i, (x, p) in enumerate(zip(tensors, params)):
            if _dtype_bits(x) != p.dtype_bits:
                raise TypeError("stream %d: sample width does not match dtype_bits" % i)
            cap = native.bound(p, x.numel())
            caps.append(cap)
            offs.append(total)
            total += (cap + 15) // 16 * 16
        if outs is None:
            # every item's output is a 16-byte aligned slice of one buffer
            self.buffer = torch.empty(max(total, 16), dtype=torch.uint8, device=self.device)
            self.outs = [self.buffer[o:o + c] for o, c in zip(offs, caps)]
        else:
            self.outs = list(outs)
        nb = self.nbytes.data_ptr()
        for i, (x, p) in enumerate(zip(tensors, params)):
            items.append(native.PcBatchItem(x.data_ptr() if x.numel() else None, x.numel(), p,
                                            self.outs[i].data_ptr(), self.outs[i].numel(), nb + 8 * i))
        self._arr, self.info = native.batch_describe(items, cta_threads)
        self.plan = torch.empty((self.info.plan_bytes + 15) // 16 * 16, dtype=torch.uint8, device=self.device)
        if workspace is not None and workspace.numel() >= self.info.workspace_bytes:
            self.ws = workspace
        else:
            self.ws = torch.empty((self.info.workspace_bytes + 15) // 16 * 16, dtype=torch.uint8,
                                  device=self.device)
        native.batch_plan(self._arr, self.info, self.plan.data_ptr(), _stream_handle(stream, self.device))

    def compress(self, stream=None):
        st = native.compress_batch(self.info, self.plan.data_ptr(), self.ws.data_ptr(), self.ws.numel(),
                                   _stream_handle(stream, self.device))
        if st != native.PC_OK:
            raise native.PcError(st, "pc_compress_batch")

    def device_status(self, stream=None):
        return native.last_device_status(self.ws.data_ptr(), _stream_handle(stream, self.device))

    def capture(self):
        """A CUDA graph of one batch compression (warm up first)."""
        self.compress()
        torch.cuda.synchronize(self.device)
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            self.compress()
        return g

    def streams(self):
        """Host bytes of every output stream (synchronises)."""
        sizes = self.nbytes.cpu().tolist()
        return [o[:k].cpu().numpy().tobytes() for o, k in zip(self.outs, sizes)]


LENGTHS = (128, 256, 512, 1024, 2048, 4096)
WORDS = (32, 64)


def autotune(x, variant=native.BASIC, sample=1 << 18, lengths=LENGTHS, words=WORDS, time_slack=None,
             time_sample=1 << 22, reps=3):
    """Block length and word size for stream `x`: every candidate compresses
    the first `sample` samples with the library; the smallest stream wins, a
    tie going to the longer block (fewer blocks, less per-block work).  With
    `time_slack`, every candidate is also timed (CUDA events, `reps`
    compressions of the first `time_sample` samples after a warm-up) and only
    the candidates within (1 + time_slack) of the fastest one's time compete
    on size: short blocks compress markedly slower, and a slightly smaller
    stream rarely pays for that."""
    from . import Codec

    d = _dtype_bits(x)
    head = x[:sample].contiguous()
    cands = []
    for w in words:
        for L in lengths:
            codec = Codec(variant, d, w, L, max_samples=max(head.numel(), min(x.numel(), time_sample)),
                          device=x.device)
            _, nb = codec.compress(head)
            t = 0.0
            if time_slack is not None:
                th = x[:time_sample].contiguous()
                out = torch.empty(codec.bound(th.numel()), dtype=torch.uint8, device=x.device)
                codec.compress(th, out=out)
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record()
                for _ in range(reps):
                    codec.compress(th, out=out)
                e1.record()
                torch.cuda.synchronize(x.device)
                t = e0.elapsed_time(e1) / reps
            cands.append((int(nb.item()), -L, -w, t, native.params(variant, d, w, L)))
    if time_slack is not None:
        t_min = min(c[3] for c in cands)
        cands = [c for c in cands if c[3] <= (1.0 + time_slack) * t_min]
    return min(cands, key=lambda c: c[:3])[4]


def autotune_threads(tensors, params, candidates=(128, 256), reps=5):
    """Threads per CTA for a batch: each candidate compresses the whole batch
    `reps` times after a warm-up, timed with CUDA events; the fastest wins.
    Returns (threads, {threads: ms per launch})."""
    times = {}
    for nt in candidates:
        b = Batch(tensors, params, cta_threads=nt)
        b.compress()
        torch.cuda.synchronize(b.device)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            b.compress()
        e1.record()
        torch.cuda.synchronize(b.device)
        times[nt] = e0.elapsed_time(e1) / reps
        del b
    best = min(times, key=lambda k: (times[k], k))
    return best, times

