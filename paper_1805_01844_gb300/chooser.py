"""Learned block-parameter chooser (pc_segment_features / pc_mlp_* in
include/pc.h): marshalling of the library's feature, MLP and batch kernels.

Per segment of 4096 samples an MLP picks one of 12 options (block length
128..4096 x word size 32/64).  The options only change the parameters of each
segment's stream; every segment is an ordinary version-1 stream, compressed
in one batch launch, so losslessness is untouched; assemble_v2 then joins a
source's segments into one version-2 stream, which records each segment's
(L, w) in a code byte instead of a 64-byte header.  The plain heuristic (one
fixed option for every segment) is the fallback.
"""
import numpy as np
import torch

from . import native

SEG = native.SEGMENT_SAMPLES
OPTIONS = native.CHOOSER_OPTIONS
LENGTHS = (128, 256, 512, 1024, 2048, 4096)
PLAIN_OPTION = 7  # block length 1024, 64-bit words: the fixed default


def option_params(o, dtype_bits, variant):
    return native.params(variant, dtype_bits, (32, 64)[o % 2], LENGTHS[o // 2])


def _bits(x):
    return 16 if x.element_size() == 2 else 32


def _stream(device):
    return torch.cuda.current_stream(device).cuda_stream


def segment_features(x):
    """Feature rows [ceil(n / 4096), 24] (FP32) of a CUDA sample tensor."""
    n = x.numel()
    nseg = -(-n // SEG)
    out = torch.empty((max(nseg, 1), native.CHOOSER_FEATURES), dtype=torch.float32, device=x.device)
    st = native.load().pc_segment_features(x.data_ptr() if n else None, n, _bits(x), out.data_ptr(),
                                           _stream(x.device))
    if st != native.PC_OK:
        raise native.PcError(st, "pc_segment_features")
    return out[:nseg]


def segments(x):
    """Views of x, one per segment (all 16-byte aligned)."""
    n = x.numel()
    return [x[s:s + SEG] for s in range(0, n, SEG)]


class Segments:
    """Sources cut into segments of 4096 samples, each compressed on the
    device with its own option (pc_segments_* in include/pc.h).  Segment j of
    source i is a version-1 stream in slot j of outs[i] (slot = seg_stride
    bytes), its size in nbytes[i][j].  Build once per set of sources; then
    features() and compress(options) run without a host round trip."""

    def __init__(self, sources, variant=native.ADVANCED, outs=None, nbytes=None, totals=None, workspace=None,
                 stream=None):
        """sources: CUDA sample tensors (one dtype); outs / nbytes: optional
        caller-owned uint8 / int64 tensors per source; totals: optional int64
        device tensors [2] per source (events, bytes), or None entries."""
        assert sources
        self.device = sources[0].device
        self.sources = [x.reshape(-1) for x in sources]
        self.dtype_bits = _bits(self.sources[0])
        self.variant = variant
        self.stride = native.segment_stride(self.dtype_bits, variant)
        self.counts = [-(-x.numel() // SEG) for x in self.sources]
        if outs is None:
            total = sum(self.counts)
            self.buffer = torch.empty(max(total, 1) * self.stride, dtype=torch.uint8, device=self.device)
            self.sizes = torch.zeros(max(total, 1), dtype=torch.int64, device=self.device)
            outs, nbytes, k = [], [], 0
            for c in self.counts:
                outs.append(self.buffer[k * self.stride:(k + c) * self.stride])
                nbytes.append(self.sizes[k:k + c])
                k += c
        self.outs, self.nbytes = list(outs), list(nbytes)
        totals = totals or [None] * len(self.sources)
        src = []
        for x, o, nb, t in zip(self.sources, self.outs, self.nbytes, totals):
            if _bits(x) != self.dtype_bits:
                raise TypeError("all sources must have the same sample width")
            n = x.numel()
            src.append(native.PcSource(x.data_ptr() if n else None, n, o.data_ptr() if n else None, o.numel(),
                                       nb.data_ptr() if n else None, t.data_ptr() if t is not None else None))
        self._arr, self.info = native.segments_describe(src, self.dtype_bits, variant)
        self.n_segments = int(self.info.n_segments)
        self.plan = torch.empty(max((self.info.plan_bytes + 15) // 16 * 16, 16), dtype=torch.uint8,
                                device=self.device)
        ws = self.info.workspace_bytes
        if workspace is not None and workspace.numel() >= ws:
            self.ws = workspace
        else:
            self.ws = torch.empty(max((ws + 15) // 16 * 16, 16), dtype=torch.uint8, device=self.device)
        self._stream = stream
        native.segments_plan(self._arr, self.info, self.plan.data_ptr(), self._handle())

    def _handle(self):
        s = self._stream if self._stream is not None else torch.cuda.current_stream(self.device)
        return s.cuda_stream

    def features(self):
        """Feature rows [n_segments, 24] (FP32, device)."""
        out = torch.empty((max(self.n_segments, 1), native.CHOOSER_FEATURES), dtype=torch.float32,
                          device=self.device)
        native.segments_features(self.info, self.plan.data_ptr(), out.data_ptr(), self._handle())
        return out[:self.n_segments]

    def compress(self, options):
        """Compress every segment with its option (uint8 device tensor)."""
        options = options.contiguous()
        assert options.dtype == torch.uint8 and options.numel() >= self.n_segments
        st = native.compress_segments(self.info, self.plan.data_ptr(), options.data_ptr(), self.ws.data_ptr(),
                                      self.ws.numel(), self._handle())
        if st != native.PC_OK:
            raise native.PcError(st, "pc_compress_segments")

    def device_status(self):
        return native.last_device_status(self.ws.data_ptr(), self._handle())

    def streams(self, i):
        """Host bytes of every segment stream of source i (synchronises)."""
        sizes = self.nbytes[i].cpu().tolist()
        o = self.outs[i]
        return [o[j * self.stride:j * self.stride + k].cpu().numpy().tobytes() for j, k in enumerate(sizes)]

    def total_bytes(self):
        return int(sum(int(nb.sum().item()) for nb in self.nbytes))

    def assemble_v2(self, i, out=None, out_bytes=None, workspace=None):
        """Source i's segment streams as one version-2 stream (per-segment
        (L, w) codes instead of a 64-byte header per segment; pc_assemble_v2).
        Returns (uint8 device buffer, int64 device tensor [1] of its size);
        no host synchronisation."""
        n = self.sources[i].numel()
        cap = native.bound_v2(self.variant, self.dtype_bits, SEG, n)
        if out is None:
            out = torch.empty((cap + 15) // 16 * 16, dtype=torch.uint8, device=self.device)
        if out_bytes is None:
            out_bytes = torch.zeros(1, dtype=torch.int64, device=self.device)
        wsb = native.assemble_v2_workspace_size(self.counts[i])
        if workspace is None or workspace.numel() < wsb:
            workspace = torch.empty((wsb + 15) // 16 * 16, dtype=torch.uint8, device=self.device)
        st = native.assemble_v2_raw(self.outs[i].data_ptr() if n else None, self.stride, self.counts[i], n, SEG,
                                    self.dtype_bits, self.variant, out.data_ptr(), out.numel(), out_bytes.data_ptr(),
                                    workspace.data_ptr(), workspace.numel(), self._handle())
        if st != native.PC_OK:
            raise native.PcError(st, "pc_assemble_v2")
        self._v2_ws = workspace
        return out, out_bytes

    def v2_status(self):
        """Device status of the last assemble_v2 (synchronises)."""
        return native.last_device_status(self._v2_ws.data_ptr(), self._handle())


def v2_code(o):
    """Format-2 code byte of chooser option o: log2(L) | (w == 64) << 7."""
    return (7 + o // 2) | (0x80 if o % 2 else 0)


def decompress_v2(buf, in_bytes, variant, dtype_bits, capacity, seg_len=SEG, out=None, workspace=None,
                  stream=None):
    """Samples of a version-2 stream (pc_decompress_v2).  Returns (samples,
    int64 device count, workspace); check native.last_device_status on the
    workspace for corrupt streams."""
    dev = buf.device
    dt = torch.int16 if dtype_bits == 16 else torch.int32
    if out is None:
        out = torch.empty(max(capacity, 8), dtype=dt, device=dev)
    n_out = torch.zeros(1, dtype=torch.int64, device=dev)
    wsb = native.decompress_v2_workspace_size(variant, dtype_bits, seg_len, capacity)
    if workspace is None or workspace.numel() < wsb:
        workspace = torch.empty((wsb + 15) // 16 * 16, dtype=torch.uint8, device=dev)
    s = (stream or torch.cuda.current_stream(dev)).cuda_stream
    st = native.decompress_v2_raw(buf.data_ptr(), in_bytes, variant, dtype_bits, seg_len, out.data_ptr(), capacity,
                                  n_out.data_ptr(), workspace.data_ptr(), workspace.numel(), s)
    if st != native.PC_OK:
        raise native.PcError(st, "pc_decompress_v2")
    return out, n_out, workspace


def compress_segments(x, options, variant=native.ADVANCED):
    """Compress every segment of x with its option (device uint8 tensor or
    list) in one pass; returns the Segments (streams in .outs[0], sizes in
    .nbytes[0])."""
    seg = Segments([x], variant)
    if not torch.is_tensor(options):
        options = torch.tensor(list(options), dtype=torch.uint8)
    seg.compress(options.to(device=x.device, dtype=torch.uint8))
    return seg


def exhaustive_sizes(x, variant=native.ADVANCED, times=None):
    """Stream size of every segment under every option: [nseg, 12] int64
    (every segment compressed 12 times on the device).  If `times` is a
    list, the GPU time (ms, CUDA events) of each option's pass over all
    segments is appended to it."""
    seg = Segments([x], variant)
    nseg = seg.n_segments
    sizes = torch.empty((nseg, OPTIONS), dtype=torch.int64, device=x.device)
    for o in range(OPTIONS):
        opts = torch.full((nseg,), o, dtype=torch.uint8, device=x.device)
        if times is not None:
            seg.compress(opts)  # warm-up (the series table of the workspace)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
        seg.compress(opts)
        if times is not None:
            e1.record()
        st = seg.device_status()
        if st != native.PC_OK:
            raise native.PcError(st, "pc_compress_segments (device)")
        if times is not None:
            times.append(e0.elapsed_time(e1))
        sizes[:, o] = seg.nbytes[0]
    return sizes


def labels_within_time(sizes, times, limit):
    """Minimum-size labels among the options whose pass over the segments
    took at most `limit` ms (a throughput floor); the fastest option if none
    qualifies.  sizes: [nseg, 12] device tensor; times: 12 floats."""
    allowed = torch.tensor([t <= limit for t in times], device=sizes.device)
    if not bool(allowed.any()):
        allowed[int(np.argmin(times))] = True
    big = torch.iinfo(torch.int64).max
    masked = torch.where(allowed.view(1, -1), sizes, torch.full_like(sizes, big))
    return torch.argmin(masked, dim=1).to(torch.uint8)


class Chooser:
    """The MLP: BF16 weights for inference, FP32 master, Adam state."""

    def __init__(self, device="cuda", seed=0):
        self.device = torch.device(device)
        rng = np.random.default_rng(seed)
        P = []
        for fan_out, fan_in in ((64, 24), (64, 64), (12, 64)):
            P.append(rng.normal(0.0, np.sqrt(2.0 / fan_in), fan_out * fan_in))
        P += [np.zeros(64), np.zeros(64), np.zeros(12)]
        master = np.concatenate(P).astype(np.float32)
        self.master = torch.from_numpy(master).to(self.device)
        self.weights = torch.empty(native.MLP_WEIGHT_BYTES, dtype=torch.uint8, device=self.device)
        self._sync_weights()
        z = lambda: torch.zeros(native.MLP_PARAMS, dtype=torch.float32, device=self.device)  # noqa: E731
        self.m, self.v, self.grad = z(), z(), z()
        self.loss = torch.zeros(1, dtype=torch.float32, device=self.device)
        self.step = 0

    def _sync_weights(self):
        """BF16 weights (round to nearest even) and FP32 biases from the master."""
        nw = 64 * 24 + 64 * 64 + 12 * 64
        wq = self.master[:nw].to(torch.bfloat16).view(torch.uint8)
        bias = self.master[nw:].contiguous().view(torch.uint8)
        self.weights[: 2 * nw].copy_(wq)
        self.weights[2 * nw:].copy_(bias)

    def set_master(self, flat):
        self.master.copy_(torch.as_tensor(flat, dtype=torch.float32))
        self._sync_weights()

    def weights_f64(self):
        """The BF16-rounded weights and FP32 biases as float64 (for checks)."""
        nw = 64 * 24 + 64 * 64 + 12 * 64
        w = self.weights[: 2 * nw].view(torch.bfloat16).double().cpu().numpy()
        b = self.weights[2 * nw:].view(torch.float32).double().cpu().numpy()
        return np.concatenate([w, b])

    def logits(self, X):
        n = X.shape[0]
        out = torch.empty((max(n, 1), OPTIONS), dtype=torch.float32, device=self.device)
        st = native.load().pc_mlp_forward(self.weights.data_ptr(), X.data_ptr(), n, out.data_ptr(), None,
                                          _stream(self.device))
        if st != native.PC_OK:
            raise native.PcError(st, "pc_mlp_forward")
        return out[:n]

    def predict(self, X):
        n = X.shape[0]
        out = torch.empty(max(n, 1), dtype=torch.uint8, device=self.device)
        st = native.load().pc_mlp_forward(self.weights.data_ptr(), X.data_ptr(), n, None, out.data_ptr(),
                                          _stream(self.device))
        if st != native.PC_OK:
            raise native.PcError(st, "pc_mlp_forward")
        return out[:n]

    def loss_grad(self, X, y):
        """(mean loss, gradient[6540]) at the current BF16 weights."""
        self.grad.zero_()
        self.loss.zero_()
        st = native.load().pc_mlp_grad(self.weights.data_ptr(), X.data_ptr(), y.data_ptr(), X.shape[0],
                                       self.grad.data_ptr(), self.loss.data_ptr(), _stream(self.device))
        if st != native.PC_OK:
            raise native.PcError(st, "pc_mlp_grad")
        return float(self.loss.item()) / X.shape[0], self.grad.clone()

    def train(self, X, y, epochs=30, batch=512, lr=3e-3, seed=0):
        """Adam on mini-batches; returns the mean loss of each epoch."""
        g = torch.Generator(device=self.device)
        g.manual_seed(seed)
        n = X.shape[0]
        lib = native.load()
        history = []
        for _ in range(epochs):
            perm = torch.randperm(n, generator=g, device=self.device)
            self.loss.zero_()
            for i in range(0, n, batch):
                idx = perm[i:i + batch]
                xb = X[idx].contiguous()
                yb = y[idx].contiguous()
                s = _stream(self.device)
                st = lib.pc_mlp_grad(self.weights.data_ptr(), xb.data_ptr(), yb.data_ptr(), xb.shape[0],
                                     self.grad.data_ptr(), self.loss.data_ptr(), s)
                if st != native.PC_OK:
                    raise native.PcError(st, "pc_mlp_grad")
                self.step += 1
                st = lib.pc_mlp_adam(self.master.data_ptr(), self.weights.data_ptr(), self.grad.data_ptr(),
                                     self.m.data_ptr(), self.v.data_ptr(), self.step, lr, s)
                if st != native.PC_OK:
                    raise native.PcError(st, "pc_mlp_adam")
            history.append(float(self.loss.item()) / n)
        return history

    def save(self, path):
        np.save(path, self.master.cpu().numpy())

    def load(self, path):
        self.set_master(np.load(path))
