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
whose parameters the MLP picks; features, choices and the per-segment
compression of all admitted events run on the device without a host round
trip (pc_segments_*), each segment's stream in its own slot of the event's
output area; with v2, each event's segments are then joined into one
version-2 stream (a code byte and a size per segment instead of a 64-byte
header; pc_assemble_v2, one call per event).  Otherwise each event is one
batch item with the plain parameters.
"""
import time
from collections import deque

import numpy as np
import torch

from . import native
from .batch import Batch
from .chooser import Segments

GEOMETRIES = ((1855, 40), (2048, 128), (11328, 25), (1296, 64))  # pixels x samples


def event_host(geom, seed):
    """One event of a camera geometry (pixels x time samples, rows = time
    samples as in Sec. 4.3.1), uint16, with the white-noise model of the
    65,536-sample workload: Gaussian, mean 300, sigma 5, rounded and clipped."""
    pixels, samples = geom
    rng = np.random.default_rng(seed)
    x = np.rint(rng.normal(300.0, 5.0, (samples, pixels)))
    return np.clip(x, 0, 65535).astype(np.uint16).reshape(-1)


def event_out_bytes(n, base_params, chooser_on):
    """Output slot size of an event of n samples: its whole stream, or with
    the chooser one segment slot per 4096 samples."""
    if not chooser_on:
        return (native.bound(base_params, n) + 15) // 16 * 16
    return -(-n // native.SEGMENT_SAMPLES) * native.segment_stride(16, base_params.variant)


class StreamPool:
    """Per-camera slots in HBM: inputs, output streams, segment sizes."""

    def __init__(self, geom, slots, out_bytes, device, totals):
        self.geom = geom
        self.n = geom[0] * geom[1]
        self.inp = torch.empty((slots, self.n), dtype=torch.int16, device=device)
        self.out = torch.empty((slots, out_bytes), dtype=torch.uint8, device=device)
        self.nbytes = torch.zeros((slots, -(-self.n // native.SEGMENT_SAMPLES)), dtype=torch.int64, device=device)
        self.free = deque(range(slots))
        self.totals = totals  # device int64 [2]: events, compressed bytes

    def nbytes_held(self):
        v2 = getattr(self, "v2out", None)
        return (self.inp.numel() * 2 + self.out.numel() + self.nbytes.numel() * 8 +
                (v2.numel() + self.v2n.numel() * 8 if v2 is not None else 0))


class Server:
    def __init__(self, device="cuda", budget=8 << 30, n_streams=3, variant=native.ADVANCED,
                 block_len=1024, word_bits=64, chooser=None, slot_cap=256, v2=False):
        self.device = torch.device(device)
        self.variant = variant
        self.chooser = chooser
        self.v2 = bool(v2 and chooser is not None)
        self.params = native.params(variant, 16, word_bits, block_len)
        outb = [event_out_bytes(g[0] * g[1], self.params, chooser is not None) for g in GEOMETRIES]
        v2b = [(native.bound_v2(variant, 16, native.SEGMENT_SAMPLES, g[0] * g[1]) + 15) // 16 * 16 if self.v2 else 0
               for g in GEOMETRIES]
        per_event = sum(g[0] * g[1] * 2 + o + v + 8 * -(-g[0] * g[1] // native.SEGMENT_SAMPLES) + 8
                        for g, o, v in zip(GEOMETRIES, outb, v2b))
        ws_reserve = n_streams * (48 << 20)  # launch workspaces (series tables, look-back words, plans)
        slots = int(max(1, min(slot_cap, (budget - ws_reserve) // per_event)))
        # per-stream running totals (events, compressed bytes) stay on the device
        self.totals = torch.zeros((len(GEOMETRIES), 2), dtype=torch.int64, device=self.device)
        self.pools = [StreamPool(g, slots, o, self.device, self.totals[i])
                      for i, (g, o) in enumerate(zip(GEOMETRIES, outb))]
        for pool, v in zip(self.pools, v2b):  # the events' version-2 streams and their sizes
            pool.v2out = torch.empty((slots, v), dtype=torch.uint8, device=self.device) if v else None
            pool.v2n = torch.zeros(slots, dtype=torch.int64, device=self.device) if v else None
        self.cuda_streams = [torch.cuda.Stream(self.device) for _ in range(n_streams)]
        self.workspaces = [None] * n_streams
        self.v2_workspaces = [None] * n_streams
        self.budget = budget
        assert sum(p.nbytes_held() for p in self.pools) + ws_reserve <= budget

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
        self.totals.zero_()
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
                for k, (e, gi, slot) in enumerate(members):
                    done_time[e] = tdone
                    if e in keep:
                        kept[e] = _streams_of(b, k)
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
            # one launch sequence over everything admitted since the last one
            if admitted:
                with torch.cuda.stream(stream):
                    b = self._launch(admitted, si, stream)
                    ev = torch.cuda.Event()
                    ev.record(stream)
                inflight.append((ev, admitted, b))
                admitted = []
                rr += 1
            elif nxt < len(events) and not waiting:
                gap = arrivals[nxt] - (time.perf_counter() - t0)
                if gap > 0:
                    time.sleep(min(gap, 2e-4))
        wall = time.perf_counter() - t0
        torch.cuda.synchronize(self.device)
        lat = (done_time - arrivals) * 1e3
        tot = self.totals.cpu().numpy()
        comp = int(tot[:, 1].sum())
        assert int(tot[:, 0].sum()) == len(events)
        return {"events": len(events), "rate_per_s": rate, "wall_s": wall,
                "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
                "gbs": raw / wall / 1e9, "raw_bytes": raw, "stream_bytes": comp,
                "ratio": raw / max(comp, 1), "chooser": self.chooser is not None,
                "budget_bytes": self.budget, "slots_per_stream": int(self.pools[0].inp.shape[0]),
                "kept": kept}

    def _launch(self, admitted, si, stream):
        """Compress the admitted events (e, pool, slot) on `stream`: the plain
        path is one batch launch with one item per event; with the chooser,
        features, the MLP and the per-segment compression of all of them."""
        if self.chooser is not None:
            pools = [self.pools[gi] for _, gi, _ in admitted]
            seg = Segments([p.inp[slot] for p, (_, _, slot) in zip(pools, admitted)], self.variant,
                           outs=[p.out[slot] for p, (_, _, slot) in zip(pools, admitted)],
                           nbytes=[p.nbytes[slot] for p, (_, _, slot) in zip(pools, admitted)],
                           totals=None if self.v2 else [p.totals for p in pools], workspace=self.workspaces[si],
                           stream=stream)
            self.workspaces[si] = seg.ws
            seg.compress(self.chooser.predict(seg.features()))
            if self.v2:
                seg.v2_slots = []
                for k, (p, (_, _, slot)) in enumerate(zip(pools, admitted)):
                    seg.assemble_v2(k, out=p.v2out[slot], out_bytes=p.v2n[slot:slot + 1],
                                    workspace=self.v2_workspaces[si])
                    self.v2_workspaces[si] = seg._v2_ws
                    seg.v2_slots.append((p, slot))
                idx = torch.tensor([gi for _, gi, _ in admitted], dtype=torch.int64).pin_memory()
                idx = idx.to(self.device, non_blocking=True)
                sizes = torch.cat([p.v2n[slot:slot + 1] for p, slot in seg.v2_slots])
                self.totals[:, 1].index_add_(0, idx, sizes)
                self.totals[:, 0].index_add_(0, idx, torch.ones_like(sizes))
                seg.idx = idx  # kept alive until the launch completes
            return seg
        tensors = [self.pools[gi].inp[slot] for _, gi, slot in admitted]
        outs = [self.pools[gi].out[slot] for _, gi, slot in admitted]
        b = Batch(tensors, [self.params] * len(tensors), device=self.device, outs=outs,
                  workspace=self.workspaces[si], stream=stream)
        self.workspaces[si] = b.ws
        b.compress(stream=stream)
        idx = torch.tensor([gi for _, gi, _ in admitted], dtype=torch.int64).pin_memory()
        idx = idx.to(self.device, non_blocking=True)
        self.totals[:, 1].index_add_(0, idx, b.nbytes)
        self.totals[:, 0].index_add_(0, idx, torch.ones_like(b.nbytes))
        b.idx = idx  # kept alive until the launch completes
        return b


def _streams_of(b, k):
    """Host bytes of the streams of member k of a finished launch."""
    if isinstance(b, Segments):
        if getattr(b, "v2_slots", None):
            p, slot = b.v2_slots[k]
            return [p.v2out[slot][:int(p.v2n[slot].item())].cpu().numpy().tobytes()]
        return b.streams(k)
    n = int(b.nbytes[k].item())
    return [b.outs[k][:n].cpu().numpy().tobytes()]


def compress_alone(x, variant=native.ADVANCED, block_len=1024, word_bits=64, chooser=None, v2=False):
    """The same event compressed on its own: its stream, or with the chooser
    the streams of its segments (v2: their version-2 stream)."""
    x = x.contiguous()
    if chooser is not None:
        seg = Segments([x], variant)
        seg.compress(chooser.predict(seg.features()))
        if v2:
            buf, nb = seg.assemble_v2(0)
            return [buf[:int(nb.item())].cpu().numpy().tobytes()]
        return seg.streams(0)
    p = native.params(variant, 16, word_bits, block_len)
    b = Batch([x], [p])
    b.compress()
    return _streams_of(b, 0)
