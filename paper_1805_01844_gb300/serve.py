"""Serving loop: camera events compressed as they arrive, with continuous
batching on the device.

Four camera geometries (pixels x time samples of uint16) each form a stream.
Every stream owns a pool of input and output slots allocated once in HBM,
inside a device-memory budget (8 GB by default), and its running totals
(events, compressed bytes) stay on the device.  Events arrive as a Poisson
process.  The scheduler admits an arriving event as soon as its stream has a
free slot (else it waits on the host), copies it into the slot, and on every
tick launches one batch kernel (pc_compress_batch) over everything admitted
since the last launch, on the next of several CUDA streams, so batches
overlap on the GPU while new events keep arriving.  When a batch's completion
event fires, its slots are freed.  Latency = completion time - arrival time.

With the learned chooser on, each event is cut into segments of 4096 samples
whose parameters the MLP picks (one batch item per segment, written one after
the other into the event's output slot); otherwise each event is one item
with the plain parameters.
"""
import time
from collections import deque

import numpy as np
import torch

from . import native
from .batch import Batch

GEOMETRIES = ((1855, 40), (2048, 128), (11328, 25), (1296, 64))  # pixels x samples


def event_host(geom, seed):
    """One event of a camera geometry: per-pixel pedestal U(250, 350) plus
    white noise of sigma 5, rows = time samples (Sec. 4.3.1 layout), uint16."""
    pixels, samples = geom
    rng = np.random.default_rng(seed)
    ped = rng.uniform(250.0, 350.0, pixels)
    x = np.rint(rng.normal(0.0, 5.0, (samples, pixels)) + ped)
    return np.clip(x, 0, 65535).astype(np.uint16).reshape(-1)


def _event_items(x, out, variant, base_params, chooser):
    """Batch items of one event (an input slot x, an output slot out)."""
    if chooser is None:
        return [x], [base_params], [out]
    from .chooser import SEG, option_params, segment_features

    opts = chooser.predict(segment_features(x)).cpu().tolist()
    tensors, params, outs, off = [], [], [], 0
    for k, o in enumerate(opts):
        seg = x[k * SEG:(k + 1) * SEG]
        p = option_params(int(o), 16, variant)
        cap = (native.bound(p, seg.numel()) + 15) // 16 * 16
        tensors.append(seg)
        params.append(p)
        outs.append(out[off:off + cap])
        off += cap
    return tensors, params, outs


def event_out_bytes(n, base_params, chooser_on):
    """Output slot size of an event of n samples (all segment streams fit)."""
    if not chooser_on:
        return (native.bound(base_params, n) + 15) // 16 * 16
    from .chooser import SEG

    worst = 0
    for k in range(0, n, SEG):
        m = min(SEG, n - k)
        worst += max((native.bound(native.params(base_params.variant, 16, w, L), m) + 15) // 16 * 16
                     for L in (128, 256, 512, 1024, 2048, 4096) for w in (32, 64))
    return worst


class StreamPool:
    """Per-camera slots in HBM: inputs, output streams, device totals."""

    def __init__(self, geom, slots, out_bytes, device):
        self.geom = geom
        self.n = geom[0] * geom[1]
        self.inp = torch.empty((slots, self.n), dtype=torch.int16, device=device)
        self.out = torch.empty((slots, out_bytes), dtype=torch.uint8, device=device)
        self.free = deque(range(slots))
        self.events = torch.zeros(1, dtype=torch.int64, device=device)
        self.bytes = torch.zeros(1, dtype=torch.int64, device=device)

    def nbytes(self):
        return self.inp.numel() * 2 + self.out.numel()


class Server:
    def __init__(self, device="cuda", budget=8 << 30, n_streams=3, variant=native.ADVANCED,
                 block_len=1024, word_bits=64, chooser=None, slot_cap=256):
        self.device = torch.device(device)
        self.variant = variant
        self.chooser = chooser
        self.params = native.params(variant, 16, word_bits, block_len)
        outb = [event_out_bytes(g[0] * g[1], self.params, chooser is not None) for g in GEOMETRIES]
        per_event = sum(g[0] * g[1] * 2 + o for g, o in zip(GEOMETRIES, outb))
        ws_reserve = n_streams * (40 << 20)  # batch workspaces (series tables + look-back words)
        slots = int(max(1, min(slot_cap, (budget - ws_reserve) // per_event)))
        self.pools = [StreamPool(g, slots, o, self.device) for g, o in zip(GEOMETRIES, outb)]
        self.cuda_streams = [torch.cuda.Stream(self.device) for _ in range(n_streams)]
        self.workspaces = [None] * n_streams
        self.budget = budget
        assert sum(p.nbytes() for p in self.pools) + ws_reserve <= budget

    def run(self, events, rate=20000.0, seed=0, keep=()):
        """Serve events = [(geometry index, host uint16 array)] arriving as a
        Poisson process of `rate` per second.  Returns metrics, and the
        compressed output of every event index in `keep` (list of streams)."""
        rng = np.random.default_rng(seed)
        arrivals = np.cumsum(rng.exponential(1.0 / rate, len(events)))
        pinned = [(gi, torch.from_numpy(x.view(np.int16)).pin_memory()) for gi, x in events]
        keep = set(keep)
        waiting, admitted, inflight = deque(), [], deque()
        done_time = np.zeros(len(events))
        kept, raw, nxt, finished, rr = {}, 0, 0, 0, 0
        t0 = time.perf_counter()
        while finished < len(events):
            now = time.perf_counter() - t0
            while nxt < len(events) and arrivals[nxt] <= now:
                waiting.append(nxt)
                nxt += 1
            # retire finished batches: record completion, collect kept outputs, free slots
            while inflight and inflight[0][0].query():
                _, members, b = inflight.popleft()
                tdone = time.perf_counter() - t0
                if keep & {m[0] for m in members}:
                    sizes = b.nbytes.cpu().tolist()
                for e, gi, slot, lo, hi in members:
                    done_time[e] = tdone
                    if e in keep:
                        kept[e] = [b.outs[k][:sizes[k]].cpu().numpy().tobytes() for k in range(lo, hi)]
                    self.pools[gi].free.append(slot)
                    finished += 1
            # admit arrived events into free slots of their stream
            si = rr % len(self.cuda_streams)
            stream = self.cuda_streams[si]
            still = deque()
            for e in waiting:
                gi, t = pinned[e]
                pool = self.pools[gi]
                if pool.free:
                    slot = pool.free.popleft()
                    with torch.cuda.stream(stream):
                        pool.inp[slot].copy_(t, non_blocking=True)
                    admitted.append((e, gi, slot))
                    raw += t.numel() * 2
                else:
                    still.append(e)
            waiting = still
            # one batch launch over everything admitted since the last one
            if admitted:
                with torch.cuda.stream(stream):
                    tensors, params, outs, members = [], [], [], []
                    for e, gi, slot in admitted:
                        pool = self.pools[gi]
                        tt, pp, oo = _event_items(pool.inp[slot], pool.out[slot], self.variant, self.params,
                                                  self.chooser)
                        members.append((e, gi, slot, len(tensors), len(tensors) + len(tt)))
                        tensors += tt
                        params += pp
                        outs += oo
                    b = Batch(tensors, params, device=self.device, outs=outs, workspace=self.workspaces[si],
                              stream=stream)
                    self.workspaces[si] = b.ws
                    b.compress(stream=stream)
                    # per-stream totals stay on the device
                    item_stream = torch.tensor([gi for (_, gi, _, lo, hi) in members for _ in range(lo, hi)],
                                               device=self.device)
                    per = torch.zeros(len(self.pools), dtype=torch.int64, device=self.device)
                    per.index_add_(0, item_stream, b.nbytes)
                    cnt = torch.bincount(torch.tensor([gi for (_, gi, _) in admitted], device=self.device),
                                         minlength=len(self.pools))
                    for pi, pool in enumerate(self.pools):
                        pool.bytes += per[pi]
                        pool.events += cnt[pi]
                    ev = torch.cuda.Event()
                    ev.record(stream)
                inflight.append((ev, members, b))
                admitted = []
                rr += 1
            elif nxt < len(events) and not waiting:
                gap = arrivals[nxt] - (time.perf_counter() - t0)
                if gap > 0:
                    time.sleep(min(gap, 2e-4))
        wall = time.perf_counter() - t0
        torch.cuda.synchronize(self.device)
        lat = (done_time - arrivals) * 1e3
        comp = int(sum(int(p.bytes.item()) for p in self.pools))
        return {"events": len(events), "rate_per_s": rate, "wall_s": wall,
                "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
                "gbs": raw / wall / 1e9, "raw_bytes": raw, "stream_bytes": comp,
                "ratio": raw / max(comp, 1), "chooser": self.chooser is not None,
                "budget_bytes": self.budget, "slots_per_stream": int(self.pools[0].inp.shape[0]),
                "kept": kept}


def compress_alone(x, variant=native.ADVANCED, block_len=1024, word_bits=64, chooser=None):
    """The same event compressed on its own (one batch of its items)."""
    x = x.contiguous()
    p = native.params(variant, 16, word_bits, block_len)
    out = torch.empty(event_out_bytes(x.numel(), p, chooser is not None), dtype=torch.uint8, device=x.device)
    tt, pp, oo = _event_items(x, out, variant, p, chooser)
    b = Batch(tt, pp, outs=oo)
    b.compress()
    sizes = b.nbytes.cpu().tolist()
    return [b.outs[k][:sizes[k]].cpu().numpy().tobytes() for k in range(len(tt))]
