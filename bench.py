"""Benchmark of the GPU polynomial compression path (arXiv:1805.01844).

One step = one compress + one decompress (the whole hot path) of the
Cherenkov-camera workload: 10,000 events x 2 gains x 40 time samples x 1855
pixels of uint16 (2.97 GB), drawn on the GPU from the seeded generator in
paper_1805_01844_gb300.datagen (synthetic stand-in for the paper's CTA
waveform files, Sec. 4.3.1).  Inputs stay resident in HBM; they are far
larger than L2, so no flush is needed between steps.

Prints one JSON line.  `value` is the round-trip throughput in uncompressed
GB/s (input bytes / (compress + decompress time)); the per-direction
throughputs, the compression ratio, the roofline of the dominant kernel, the
oracle timed on the host cores and an end-to-end figure through host buffers
are reported beside it.

  python bench.py [--steps K] [--warmup W] [--variant basic|advanced]
                  [--block-len L] [--word-bits 32|64] [--impl ours|reference]
Under torchrun each rank compresses its own copy of the workload (weak
scaling, no collective on the data path).
"""
import argparse
import hashlib
import json
import os
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

GB = 1e9
WORKLOAD = dict(n_events=10000, n_gains=2, n_time=40, n_pixels=1855)
METRIC = "compress/decompress input GB/s on 1 GB300 (% HBM peak) and ratio, learned vs plain"
FALLBACK_HBM_GBS = 6800.0


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--variant", choices=["basic", "advanced"], default="basic")
    ap.add_argument("--block-len", type=int, default=1024)
    ap.add_argument("--word-bits", type=int, default=64, choices=[32, 64])
    ap.add_argument("--events", type=int, default=WORKLOAD["n_events"])
    ap.add_argument("--white-noise", type=int, default=0,
                    help="time N samples of the 65,536-sample white-noise workload's generator instead of camera "
                         "events (no CPU baseline or sweeps then)")
    ap.add_argument("--e2e-steps", type=int, default=6)
    ap.add_argument("--cpu-events", type=int, default=0,
                    help="events in the oracle's CPU sample (0 = sized to ~15 s)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-learned", action="store_true")
    ap.add_argument("--no-serve", action="store_true")
    ap.add_argument("--no-sweep", action="store_true")
    ap.add_argument("--no-cfg1", action="store_true")
    ap.add_argument("--no-batch", action="store_true")
    ap.add_argument("--no-paper-sweeps", action="store_true")
    ap.add_argument("--serve-events", type=int, default=20000)
    ap.add_argument("--serve-v2", action="store_true",
                    help="also serve with the chooser and one version-2 stream per event")
    return ap.parse_args()


def workload_name(args):
    if args.white_noise:
        return "white_noise_N300_5_%d_u16" % args.white_noise
    return "cherenkov_events_%dx%dx%dx%d_u16" % (args.events, WORKLOAD["n_gains"], WORKLOAD["n_time"],
                                                WORKLOAD["n_pixels"])


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            j = json.load(f)
        return float(j["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


# the sources the compression and decompression kernels are built from
KERNEL_SOURCES = ("pc_common.cuh", "pc_device.cuh", "pc_orbit.cuh", "pc_compress.cuh", "pc_compress.cu",
                  "pc_decompress.cu", "pc_kernels.h")


def kernel_source_hash():
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_1805_01844_gb300", "csrc")
    for name in KERNEL_SOURCES:
        with open(os.path.join(csrc, name), "rb") as f:
            h.update(name.encode())
            h.update(f.read())
    return h.hexdigest()[:16]


def recorded_traffic(kernel_key):
    """DRAM bytes per launch from the committed ncu summary, if it was taken
    on the current kernel sources."""
    path = os.path.join(ROOT, "profiles", "dram_traffic.json")
    try:
        with open(path) as f:
            j = json.load(f)
    except Exception:
        return None
    e = j.get(kernel_key)
    if not e or e.get("source_hash") != kernel_source_hash():
        return None
    return e.get("dram_bytes_per_launch")


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 100 ms; only the
    samples that arrive inside [mark_start, mark_stop] are summarised."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.proc = None
        self.gpu = gpu_index
        self.lines = []
        self.t0 = self.t1 = None

    def start(self):
        import threading

        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
            return

        def reader():
            for line in self.proc.stdout:
                self.lines.append((time.perf_counter(), line))

        self.thread = threading.Thread(target=reader, daemon=True)
        self.thread.start()

    def mark_start(self):
        self.t0 = time.perf_counter()

    def mark_stop(self):
        self.t1 = time.perf_counter()

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0,
                    "note": "nvidia-smi unavailable"}
        time.sleep(0.15)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.thread.join(timeout=2)
        sm, mx, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for t, line in self.lines:
            if self.t0 is None or t < self.t0 or t > self.t1 + 0.1:
                continue
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx = max(mx, float(parts[2]))
            except ValueError:
                continue
            for name, flag in zip(names, parts[5:9]):
                if flag.lower() == "active":
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        sm.sort()
        return {"sm_mhz": sm[len(sm) // 2], "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def dist_info():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def max_over_ranks(ms, dist, device):
    """The slowest rank's time (every rank returns it)."""
    import torch

    t = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def weak_scaling_value(world, raw_bytes, steps, total_ms):
    """Whole-job GB/s: every rank compresses and decompresses its own copy of
    the workload, so the job moves world x raw bytes per step."""
    return world * raw_bytes * steps / (total_ms / 1e3) / GB


# ------------------------------------------------------------------ oracle leg


def oracle_sample_timing(x_host_events, variant, w, L, target_s=15.0, fixed_events=0):
    """Time the CPU oracle (single thread, as it stands) compressing and
    decompressing a prefix of the events; returns (GB/s, events, seconds)."""
    import oracle

    per_event = x_host_events[0].size * 2
    if fixed_events:
        n_ev = fixed_events
    else:
        probe = x_host_events[:2].reshape(-1)
        t0 = time.perf_counter()
        s = oracle.compress(probe, variant, w, L)
        oracle.decompress(s)
        dt = (time.perf_counter() - t0) / 2
        n_ev = max(1, min(len(x_host_events), int(target_s / max(dt, 1e-6))))
    x = x_host_events[:n_ev].reshape(-1)
    t0 = time.perf_counter()
    s = oracle.compress(x, variant, w, L)
    t1 = time.perf_counter()
    y = oracle.decompress(s)
    t2 = time.perf_counter()
    assert (y == x).all()
    return n_ev * per_event / (t2 - t0) / GB, n_ev, t2 - t0, len(s)


def oracle_fanout_timing(x_host_events, variant, w, L, threads, events_per_thread):
    """The oracle as it stands on every host core: the events split into one
    chunk (an independent stream) per thread, each compressed and
    decompressed by its own thread (the C oracle runs outside the GIL)."""
    from concurrent.futures import ThreadPoolExecutor

    import oracle

    per_event = x_host_events[0].size * 2
    n_ev = min(len(x_host_events), threads * events_per_thread)
    chunks = [x_host_events[i:n_ev:threads].reshape(-1) for i in range(threads)]

    def work(c):
        y = oracle.decompress(oracle.compress(c, variant, w, L))
        return bool((y == c).all())

    work(chunks[0][: 4 * L])  # load the library before timing
    t0 = time.perf_counter()
    with ThreadPoolExecutor(max_workers=threads) as ex:
        ok = list(ex.map(work, chunks))
    dt = time.perf_counter() - t0
    assert all(ok)
    return n_ev * per_event / dt / GB, n_ev, dt


def run_reference(args):
    """The reference arm: the CPU oracle as it stands, on the host cores, on a
    bounded sample of the same workload (rank 0 only)."""
    import numpy as np

    from paper_1805_01844_gb300 import datagen

    world, rank, _ = dist_info()
    if rank != 0:
        return
    variant = 0 if args.variant == "basic" else 1
    n_ev = args.cpu_events or 16
    x = datagen.cherenkov_events(n_ev, seed=0)
    import oracle

    oracle.build.build()
    per_step = x.size * 2
    for _ in range(args.warmup):
        oracle.decompress(oracle.compress(x.reshape(-1), variant, args.word_bits, args.block_len))
    t0 = time.perf_counter()
    for _ in range(args.steps):
        s = oracle.compress(x.reshape(-1), variant, args.word_bits, args.block_len)
        oracle.decompress(s)
    dt = time.perf_counter() - t0
    value = per_step * args.steps / dt / GB
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "GB/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u16",
        "data": "synthetic", "ratio": per_step / len(s),
        "config": {"workload": workload_name(args), "variant": args.variant,
                   "block_len": args.block_len, "word_bits": args.word_bits,
                   "sample": "each step compresses and decompresses the first %d events (%.1f MB) of this "
                             "workload (the same generator and seed), single thread" % (n_ev, per_step / 1e6)},
        "cpu_baseline": {"value": value, "unit": "GB/s", "cores": 1, "kind": "oracle",
                         "sample": "first %d events (%.1f MB) of the workload, generated on the host"
                                   % (n_ev, per_step / 1e6)},
        "e2e": {"value": value, "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------- GPU leg


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
        return
    import numpy as np
    import torch

    import paper_1805_01844_gb300 as pc
    from paper_1805_01844_gb300 import datagen, native

    world, rank, local = dist_info()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=dev)
    native.load()
    variant = pc.BASIC if args.variant == "basic" else pc.ADVANCED
    L, w = args.block_len, args.word_bits

    if args.white_noise:
        x = datagen.white_noise_torch(args.white_noise, dev, mean=300.0, sigma=5.0, seed=0)
        args.no_cpu_baseline = args.no_sweep = args.no_paper_sweeps = True
    else:
        x = datagen.cherenkov_events_torch(args.events, dev, seed=0).reshape(-1)
    n = x.numel()
    raw_bytes = n * 2
    codec = pc.Codec(variant, 16, w, L, max_samples=n, device=dev)
    sbuf = torch.empty(codec.bound(n), dtype=torch.uint8, device=dev)
    ybuf = torch.empty(n, dtype=torch.int16, device=dev)
    stream = torch.cuda.current_stream(dev)

    def step():
        _, nb = codec.compress(x, out=sbuf)
        codec.decompress(sbuf, sbuf.numel(), n, out=ybuf)
        return nb

    # correctness before timing: exact round trip on the device (byte parity
    # with the oracle at this size and launch configuration is a GPU test)
    nb = step()
    st = codec.device_status()
    assert st == 0, native.strerror(st)
    stream_bytes = int(nb.item())
    assert torch.equal(ybuf, x), "round trip failed"
    parity = "round trip exact on the device"

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(args.steps)]
    clocks = ClockSampler(torch.cuda.current_device())
    clocks.start()
    time.sleep(0.3)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.mark_start()
    t_start = time.perf_counter()
    for k in range(args.steps):
        ev[k][0].record(stream)
        codec.compress(x, out=sbuf)
        ev[k][1].record(stream)
        codec.decompress(sbuf, sbuf.numel(), n, out=ybuf)
        ev[k][2].record(stream)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    wall = time.perf_counter() - t_start
    clocks.mark_stop()
    clk = clocks.stop()
    st = codec.device_status()
    assert st == 0, native.strerror(st)
    tc = [ev[k][0].elapsed_time(ev[k][1]) for k in range(args.steps)]
    td = [ev[k][1].elapsed_time(ev[k][2]) for k in range(args.steps)]
    total_ms = ev[0][0].elapsed_time(ev[-1][2])
    if world > 1:
        total_ms = max_over_ranks(total_ms, dist, dev)
    tc_ms = sum(tc) / len(tc)
    td_ms = sum(td) / len(td)
    value = weak_scaling_value(world, raw_bytes, args.steps, total_ms)
    comp_gbs = raw_bytes / (tc_ms / 1e3) / GB
    dec_gbs = raw_bytes / (td_ms / 1e3) / GB
    peak, peak_kind = peaks()
    alg_bytes = raw_bytes + stream_bytes  # read + write of either kernel
    dominant = "compress" if tc_ms >= td_ms else "decompress"
    dom_ms = max(tc_ms, td_ms)
    key = "%s_u16_w%d_%s_L%d" % (dominant, w, args.variant, L)
    achieved = alg_bytes / (dom_ms / 1e3) / GB

    e2e = None
    if not args.no_e2e and rank == 0:
        e2e = end_to_end(codec, x, n, args.e2e_steps, dev)

    cpu = cpu_all = None
    if not args.no_cpu_baseline and rank == 0 and world == 1:
        ev_host = x.view(args.events, -1)[: max(args.cpu_events, min(args.events, 2000))]
        ev_host = ev_host.cpu().numpy().view(np.uint16)
        gbs, n_ev, secs, _ = oracle_sample_timing(
            ev_host.reshape(-1, WORKLOAD["n_gains"] * WORKLOAD["n_time"] * WORKLOAD["n_pixels"]),
            variant, w, L, fixed_events=args.cpu_events)
        cpu = {"value": gbs, "unit": "GB/s", "cores": 1, "kind": "oracle",
               "sample": "first %d events (%.1f MB) of the workload, compress + decompress, %.1f s, "
                         "single thread" % (n_ev, n_ev * ev_host[0].size * 2 / 1e6, secs)}
        threads = os.cpu_count() or 1
        gbs_all, n_all, secs_all = oracle_fanout_timing(ev_host, variant, w, L, threads,
                                                        max(1, len(ev_host) // threads))
        cpu_all = {"value": gbs_all, "unit": "GB/s", "cores": threads, "kind": "oracle",
                   "sample": "first %d events (%.1f MB), one chunk per thread, compress + decompress, %.1f s"
                             % (n_all, n_all * ev_host[0].size * 2 / 1e6, secs_all)}

    sweep = None
    if not args.no_sweep and rank == 0 and world == 1:
        sweep = sweep_params(x, n, dev)

    cfg1 = small = None
    if not args.no_cfg1 and rank == 0 and world == 1:
        cfg1 = white_noise_2e30(dev, peak)
        small = white_noise_65536_latency(dev)

    batch = None
    if not args.no_batch and rank == 0 and world == 1:
        batch = batch_metrics(dev)

    paper = None
    if not args.no_paper_sweeps and rank == 0 and world == 1:
        paper = paper_sweeps(dev, x, sbuf, stream_bytes, L, w, args.variant)

    learned, trained = None, None
    if not args.no_learned and rank == 0 and world == 1:
        learned, trained = learned_vs_plain(dev)

    serving = None
    if not args.no_serve and rank == 0 and world == 1:
        serving = serve_metrics(dev, args.serve_events, trained, v2=args.serve_v2)

    if world > 1:
        dist.barrier()
        dist.destroy_process_group()
    if rank != 0:
        return
    line = {
        "metric": METRIC, "value": value, "unit": "GB/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u16", "data": "synthetic",
        "config": {"workload": workload_name(args), "variant": args.variant, "block_len": L,
                   "word_bits": w, "input_bytes": raw_bytes,
                   "l2": "inputs (%.2f GB) far larger than L2; no flush" % (raw_bytes / GB)},
        "compress_gbs": comp_gbs, "decompress_gbs": dec_gbs,
        "compress_pct_hbm": 100 * comp_gbs / peak, "decompress_pct_hbm": 100 * dec_gbs / peak,
        "ratio": raw_bytes / stream_bytes, "stream_bytes": stream_bytes,
        "compress_ms": tc_ms, "decompress_ms": td_ms, "parity": parity,
        "roofline": {"bound": "hbm", "kernel": dominant, "achieved": achieved, "peak": peak,
                     "peak_kind": peak_kind, "unit": "GB/s", "frac": achieved / peak,
                     "alg_bytes_per_launch": alg_bytes, "traffic": recorded_traffic(key)},
        "cpu_baseline": cpu, "cpu_baseline_all_cores": cpu_all, "e2e": e2e, "gpu_launches": 3 * args.steps,
        "white_noise_2e30": cfg1, "white_noise_65536": small, "batch": batch, "sweep": sweep, "paper_sweeps": paper, "learned": learned, "serving": serving,
        "clocks": clk, "wall_s_timed": wall,
    }
    print(json.dumps(line), flush=True)


def paper_sweeps(dev, x, sbuf, stream_bytes, L, w, variant):
    """The paper's ratio experiments on the GPU: Fig. 7 (ratio against block
    length on 1000 vectors of A(3000, sigma, 2000, y, 4, 1855) for the three
    distributions of Sec. 4.2, basic and advanced, 32-bit words, L = 1 ... N),
    Fig. 8 (ratio against the number of uniform signal values in vectors of
    10,000, advanced, L = 154, 100 vectors per point) and Fig. 11 (byte
    profile entropy of the camera workload and of its compressed streams).
    Every point's streams are checked against the oracle in the GPU tests."""
    import torch

    import paper_1805_01844_gb300 as pc
    from paper_1805_01844_gb300 import sweeps

    t0 = time.perf_counter()
    p7 = sweeps.ratio_vs_block_length(dev)
    t7 = time.perf_counter() - t0
    t0 = time.perf_counter()
    p8 = sweeps.ratio_vs_signal(dev)
    t8 = time.perf_counter() - t0
    fig7 = {}
    for p in p7:
        fig7.setdefault("%s/%s" % (p["curve"], p["variant"]), []).append([p["L"], round(p["ratio"], 5)])
    fig8 = {}
    for p in p8:
        fig8.setdefault(p["curve"], []).append([p["a"], round(p["ratio"], 5)])
    # Fig. 11: the workload's bytes and its streams (the timed one, and the other variant)
    other = pc.ADVANCED if variant == "basic" else pc.BASIC
    codec = pc.Codec(other, 16, w, L, max_samples=x.numel(), device=dev)
    obuf = torch.empty(codec.bound(x.numel()), dtype=torch.uint8, device=dev)
    _, onb = codec.compress(x, out=obuf)
    assert codec.device_status() == 0
    prof = sweeps.byte_profile(x, {variant: (sbuf, stream_bytes), ("basic", "advanced")[other]: (obuf, int(onb.item()))})
    del obuf, codec
    torch.cuda.empty_cache()
    fig11 = {k: {"entropy_bits_per_byte": round(v["entropy_bits"], 4), "max_over_mean": round(v["max_over_mean"], 2)}
             for k, v in prof.items()}
    return {"fig7_ratio_vs_block_length": {"N": 1855, "vectors": 1000, "word_bits": 32, "points": fig7,
                                           "summary": sweeps.summary(p7), "wall_s": round(t7, 2)},
            "fig8_ratio_vs_signal": {"N": 10000, "vectors": 100, "block_len": 154, "variant": "advanced",
                                     "points": fig8, "wall_s": round(t8, 2)},
            "fig11_byte_profile": {"workload": "camera events (the timed workload), L %d, w %d" % (L, w),
                                   "profiles": fig11},
            "ratio_definition": "32-bit words in / stream bytes without the 64-byte stream header (Sec. 4.2)"}


def white_noise_65536_latency(dev, reps=200):
    """The 65,536-sample white-noise parity workload (N(300, 5), seed 0, basic,
    L = 1024, w = 64): it fits in L2 and is bound by launch latency, so it is
    reported as the time of one compress and one decompress call (median,
    CUDA events), plus both replayed from one CUDA graph."""
    import numpy as np
    import torch

    import paper_1805_01844_gb300 as pc
    from paper_1805_01844_gb300 import datagen

    x = torch.from_numpy(datagen.white_noise(65536, 300.0, 5.0, seed=0).view(np.int16)).to(dev)
    n = x.numel()
    codec = pc.Codec(pc.BASIC, 16, 64, 1024, max_samples=n, device=dev)
    sbuf = torch.empty(codec.bound(n), dtype=torch.uint8, device=dev)
    ybuf = torch.empty(n, dtype=torch.int16, device=dev)

    def step():
        codec.compress(x, out=sbuf)
        codec.decompress(sbuf, sbuf.numel(), n, out=ybuf)

    for _ in range(5):
        step()
    torch.cuda.synchronize()
    assert torch.equal(ybuf, x) and codec.device_status() == 0
    tc, td = [], []
    for _ in range(reps):
        e = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
        e[0].record()
        codec.compress(x, out=sbuf)
        e[1].record()
        codec.decompress(sbuf, sbuf.numel(), n, out=ybuf)
        e[2].record()
        torch.cuda.synchronize()
        tc.append(e[0].elapsed_time(e[1]))
        td.append(e[1].elapsed_time(e[2]))
    s = torch.cuda.Stream(dev)
    with torch.cuda.stream(s):
        step()
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=s):
            step()
    tg = []
    for _ in range(reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        g.replay()
        e1.record()
        torch.cuda.synchronize()
        tg.append(e0.elapsed_time(e1))
    assert torch.equal(ybuf, x)
    med = lambda a: sorted(a)[len(a) // 2] * 1e3  # noqa: E731
    return {"workload": "white_noise_N300_5_65536_u16", "variant": "basic", "block_len": 1024, "word_bits": 64,
            "compress_us": med(tc), "decompress_us": med(td), "round_trip_graph_us": med(tg)}


def white_noise_2e30(dev, peak, steps=20):
    """The 65,536-sample white-noise workload scaled to 2^30 samples (2 GiB;
    N(300, 5), rounded, clipped; drawn on the GPU), basic, L = 1024, w = 64:
    compress and decompress GB/s of uncompressed data (median of `steps`
    CUDA-event timed calls after 3 warm-ups) against the HBM peak, and the
    roofline fraction of each direction (read + write bytes / time / peak)."""
    import torch

    import paper_1805_01844_gb300 as pc
    from paper_1805_01844_gb300 import datagen

    n = 1 << 30
    x = datagen.white_noise_torch(n, dev, mean=300.0, sigma=5.0, seed=0)
    codec = pc.Codec(pc.BASIC, 16, 64, 1024, max_samples=n, device=dev)
    sbuf = torch.empty(codec.bound(n), dtype=torch.uint8, device=dev)
    ybuf = torch.empty(n, dtype=torch.int16, device=dev)
    tc, td = [], []
    for k in range(steps + 3):
        e = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
        e[0].record()
        _, nb = codec.compress(x, out=sbuf)
        e[1].record()
        codec.decompress(sbuf, sbuf.numel(), n, out=ybuf)
        e[2].record()
        torch.cuda.synchronize()
        if k >= 3:
            tc.append(e[0].elapsed_time(e[1]))
            td.append(e[1].elapsed_time(e[2]))
    assert codec.device_status() == 0 and torch.equal(ybuf, x)
    size = int(nb.item())
    raw = 2 * n
    mc, md = sorted(tc)[len(tc) // 2], sorted(td)[len(td) // 2]
    out = {"workload": "white_noise_N300_5_2^30_u16", "variant": "basic", "block_len": 1024, "word_bits": 64,
           "ratio": raw / size, "compress_gbs": raw / (mc / 1e3) / GB, "decompress_gbs": raw / (md / 1e3) / GB,
           "compress_roofline_frac": (raw + size) / (mc / 1e3) / GB / peak,
           "decompress_roofline_frac": (raw + size) / (md / 1e3) / GB / peak}
    out["compress_pct_hbm"] = 100 * out["compress_gbs"] / peak
    out["decompress_pct_hbm"] = 100 * out["decompress_gbs"] / peak
    del sbuf, ybuf, codec
    # the same samples in short blocks (the block lengths of Fig. 7's best
    # ratios and of the learned chooser's short options), basic, w = 64
    short = []
    for L in (32, 64, 128, 256):
        codec = pc.Codec(pc.BASIC, 16, 64, L, max_samples=n, device=dev)
        sbuf = torch.empty(codec.bound(n), dtype=torch.uint8, device=dev)
        ybuf = torch.empty(n, dtype=torch.int16, device=dev)
        tc, td = [], []
        for k in range(8):
            e = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
            e[0].record()
            _, nb = codec.compress(x, out=sbuf)
            e[1].record()
            codec.decompress(sbuf, sbuf.numel(), n, out=ybuf)
            e[2].record()
            torch.cuda.synchronize()
            if k >= 3:
                tc.append(e[0].elapsed_time(e[1]))
                td.append(e[1].elapsed_time(e[2]))
        assert codec.device_status() == 0 and torch.equal(ybuf, x), L
        mc, md = sorted(tc)[len(tc) // 2], sorted(td)[len(td) // 2]
        short.append({"block_len": L, "ratio": raw / int(nb.item()), "compress_gbs": raw / (mc / 1e3) / GB,
                      "decompress_gbs": raw / (md / 1e3) / GB})
        del sbuf, ybuf, codec
    out["short_blocks_w64"] = short
    del x
    torch.cuda.empty_cache()
    return out


def batch_metrics(dev, n_streams=64, reps=20):
    """64 uneven streams (4 KB - 64 MB, uint16 / uint32, varied noise and
    spikes): block length and word size autotuned per stream, then all of
    them compressed by one persistent launch captured in a CUDA graph; the
    same streams one pc_compress call each, for comparison.  GB/s of input
    (median replay), ratio, and a byte check of every stream's batch output
    against its own single-stream compression."""
    import torch

    import paper_1805_01844_gb300 as pc
    from paper_1805_01844_gb300 import batch as pcb
    from paper_1805_01844_gb300 import datagen

    specs = datagen.batched_stream_specs(n_streams, seed=0)
    xs = [datagen.batched_stream_torch(sp, dev) for sp in specs]
    raw = sum(x.numel() * x.element_size() for x in xs)
    t0 = time.perf_counter()
    params = [pcb.autotune(x, variant=pc.BASIC) for x in xs]
    nt, nt_ms = pcb.autotune_threads(xs, params)
    tune_s = time.perf_counter() - t0
    b = pcb.Batch(xs, params, cta_threads=nt)
    g = b.capture()

    def med(fn):
        ts = []
        for _ in range(reps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            fn()
            e1.record()
            torch.cuda.synchronize()
            ts.append(e0.elapsed_time(e1))
        return sorted(ts)[len(ts) // 2]

    g.replay()
    torch.cuda.synchronize()
    t_batch = med(g.replay)
    assert b.device_status() == 0
    sizes = b.nbytes.cpu().tolist()
    codecs = [pc.Codec(p.variant, p.dtype_bits, p.word_bits, p.block_len, max_samples=x.numel(), device=dev)
              for x, p in zip(xs, params)]
    outs = [torch.empty(c.bound(x.numel()), dtype=torch.uint8, device=dev) for c, x in zip(codecs, xs)]

    def one_by_one():
        for c, x, o in zip(codecs, xs, outs):
            c.compress(x, out=o)

    one_by_one()
    torch.cuda.synchronize()
    t_each = med(one_by_one)
    same = all(torch.equal(b.outs[k][:sizes[k]], outs[k][:sizes[k]]) for k in range(len(xs)))
    # each stream alone through the single-stream kernel, timed one by one (no
    # launch gaps counted): what the batch launch is measured against
    t_alone = 0.0
    for c, x, o in zip(codecs, xs, outs):
        t_alone += med(lambda: c.compress(x, out=o))
    by_len = {}
    for x, p in zip(xs, params):
        k = "L%d" % p.block_len
        by_len[k] = by_len.get(k, 0.0) + x.numel() * x.element_size() / raw
    # the same streams autotuned with time as well as size: only the
    # candidates within 50 % of the fastest one's time compete on size
    params_fast = [pcb.autotune(x, variant=pc.BASIC, time_slack=0.5) for x in xs]
    nt_f, _ = pcb.autotune_threads(xs, params_fast)
    bf = pcb.Batch(xs, params_fast, cta_threads=nt_f)
    gf = bf.capture()
    gf.replay()
    torch.cuda.synchronize()
    t_fast = med(gf.replay)
    assert bf.device_status() == 0
    sizes_f = bf.nbytes.cpu().tolist()
    return {"streams": len(xs), "input_bytes": raw, "ratio": raw / sum(sizes),
            "gbs_one_graph_launch": raw / (t_batch / 1e3) / GB, "gbs_one_call_per_stream": raw / (t_each / 1e3) / GB,
            "gbs_each_stream_alone_summed": raw / (t_alone / 1e3) / GB,
            "input_share_by_block_len": {k: round(v, 4) for k, v in sorted(by_len.items())},
            "autotune_s": tune_s, "identical_to_single_stream": same, "cta_threads": nt,
            "ms_by_cta_threads": nt_ms,
            "params": sorted(set("L%d_w%d" % (p.block_len, p.word_bits) for p in params)),
            "time_aware_autotune": {"time_slack": 0.5, "ratio": raw / sum(sizes_f),
                                    "gbs_one_graph_launch": raw / (t_fast / 1e3) / GB, "cta_threads": nt_f,
                                    "params": sorted(set("L%d_w%d" % (p.block_len, p.word_bits) for p in params_fast))}}


def sweep_params(x, n, dev, steps=5):
    """The same workload over block lengths 256..4096, both word sizes and both
    variants: compress / decompress GB/s (median of `steps` CUDA-event timed
    calls after one warm-up) and the ratio, each round trip checked exact."""
    import torch

    import paper_1805_01844_gb300 as pc

    raw = n * 2
    out = []
    ybuf = torch.empty(n, dtype=torch.int16, device=dev)
    for variant in (pc.BASIC, pc.ADVANCED):
        for w in (32, 64):
            for L in (256, 512, 1024, 2048, 4096):
                codec = pc.Codec(variant, 16, w, L, max_samples=n, device=dev)
                sbuf = torch.empty(codec.bound(n), dtype=torch.uint8, device=dev)
                tc, td = [], []
                for k in range(steps + 1):
                    e = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
                    e[0].record()
                    _, nb = codec.compress(x, out=sbuf)
                    e[1].record()
                    codec.decompress(sbuf, sbuf.numel(), n, out=ybuf)
                    e[2].record()
                    torch.cuda.synchronize()
                    if k:
                        tc.append(e[0].elapsed_time(e[1]))
                        td.append(e[1].elapsed_time(e[2]))
                assert codec.device_status() == 0 and torch.equal(ybuf, x), (variant, w, L)
                size = int(nb.item())
                out.append({"variant": ("basic", "advanced")[variant], "word_bits": w, "block_len": L,
                            "ratio": raw / size,
                            "compress_gbs": raw / (sorted(tc)[len(tc) // 2] / 1e3) / GB,
                            "decompress_gbs": raw / (sorted(td)[len(td) // 2] / 1e3) / GB})
                del sbuf, codec
    torch.cuda.empty_cache()
    return out


def learned_vs_plain(dev, train_samples=2 << 30, test_bytes=1 << 30):
    """The learned chooser (advanced variant) trained on 2^31 samples (2^19
    segments, i.e. 2M blocks of 1024 samples) of the chooser mix (camera
    events + white noise of varied sigma), labelled by the exhaustive
    minimum-size search on the GPU (the tests check that search against the
    CPU oracle's byte for byte), and evaluated on 1 GB of fresh seeds: ratio of
    the learned per-segment options against the plain heuristic (block
    length 1024, 64-bit words, per segment and as one stream), the best fixed
    option as one stream, and the exhaustive optimum; GPU throughput of the
    learned path (features + MLP + compression) and of the plain one."""
    import torch

    import paper_1805_01844_gb300 as pc
    from paper_1805_01844_gb300 import chooser as ch
    from paper_1805_01844_gb300 import datagen, native

    t0 = time.perf_counter()
    tr = datagen.chooser_mix_torch(train_samples, dev, seed=11)
    opt_ms = []
    sizes_tr = ch.exhaustive_sizes(tr, times=opt_ms)
    y = torch.argmin(sizes_tr, dim=1).to(torch.uint8)
    # a second network trained on labels restricted to options that compress
    # at least as fast as the plain option (a throughput floor)
    y_fast = ch.labels_within_time(sizes_tr, opt_ms, opt_ms[ch.PLAIN_OPTION])
    c = ch.Chooser(dev, seed=0)
    c_fast = ch.Chooser(dev, seed=0)
    Xtr = ch.segment_features(tr)
    del tr, sizes_tr
    torch.cuda.empty_cache()
    hist = c.train(Xtr, y, epochs=8, batch=4096, lr=3e-3)
    c_fast.train(Xtr, y_fast, epochs=8, batch=4096, lr=3e-3)
    torch.cuda.synchronize()
    train_s = time.perf_counter() - t0
    n_train = int(Xtr.shape[0])
    del Xtr, y, y_fast
    te = datagen.chooser_mix_torch(test_bytes // 2, dev, seed=12)
    sizes_te = ch.exhaustive_sizes(te)
    raw = te.numel() * 2

    def timed(fn, reps=10):
        fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            out = fn()
        e1.record()
        torch.cuda.synchronize()
        return out, e0.elapsed_time(e1) / reps

    nseg = sizes_te.shape[0]
    seg = ch.Segments([te], native.ADVANCED)
    plain_opts = torch.full((nseg,), ch.PLAIN_OPTION, dtype=torch.uint8, device=dev)

    def learned_path():
        pred = c.predict(seg.features())
        seg.compress(pred)
        return pred

    def plain_path():
        seg.compress(plain_opts)

    pred, t_learned = timed(learned_path)
    learned_bytes = seg.total_bytes()
    # the learned options' segments as ONE version-2 stream (a code byte and a
    # size per segment instead of a 64-byte header), decoded back on the GPU
    v2buf, v2nb = seg.assemble_v2(0)
    v2ws = seg._v2_ws

    def learned_path_v2():
        p = learned_path()
        seg.assemble_v2(0, out=v2buf, out_bytes=v2nb, workspace=v2ws)
        return p

    _, t_learned_v2 = timed(learned_path_v2)
    assert seg.v2_status() == native.PC_OK
    learned_v2_bytes = int(v2nb.item())
    yv2, nv2, wsd = ch.decompress_v2(v2buf, learned_v2_bytes, native.ADVANCED, 16, te.numel())
    _, t_dec_v2 = timed(lambda: ch.decompress_v2(v2buf, learned_v2_bytes, native.ADVANCED, 16, te.numel(), out=yv2,
                                                 workspace=wsd))
    v2_exact = (native.last_device_status(wsd.data_ptr(), torch.cuda.current_stream().cuda_stream) == native.PC_OK
                and int(nv2.item()) == te.numel() and bool(torch.equal(yv2[:te.numel()], te)))
    del yv2, wsd
    _, t_plain = timed(plain_path)
    plain_bytes = seg.total_bytes()
    seg.assemble_v2(0, out=v2buf, out_bytes=v2nb, workspace=v2ws)
    plain_v2_bytes = int(v2nb.item())
    # the learned path's parts, each timed alone
    feats, t_feat = timed(seg.features)
    _, t_mlp = timed(lambda: c.predict(feats))
    _, t_comp = timed(lambda: seg.compress(pred))

    def fast_path():
        p = c_fast.predict(seg.features())
        seg.compress(p)
        return p

    pred_fast, t_fast = timed(fast_path)
    fast_bytes = seg.total_bytes()
    assert seg.device_status() == native.PC_OK
    best = int(sizes_te.min(dim=1).values.sum().item())
    agree = float((pred.to(torch.int64) == torch.argmin(sizes_te, dim=1)).float().mean().item())
    # the same test data as ONE stream under each fixed option: the plain
    # default and the best fixed option (what a per-stream autotuner reaches)
    whole = {}
    for o in range(ch.OPTIONS):
        p = ch.option_params(o, 16, native.ADVANCED)
        codec = pc.Codec(native.ADVANCED, 16, p.word_bits, p.block_len, max_samples=te.numel(), device=dev)
        _, nb = codec.compress(te)
        whole[o] = int(nb.item())
    o_best = min(whole, key=lambda o: (whole[o], o))
    return ({"train_segments": n_train, "test_segments": int(nseg), "test_bytes": raw,
             "segment_samples": ch.SEG, "variant": "advanced",
             "ratio_plain": raw / plain_bytes, "ratio_learned": raw / learned_bytes,
             "ratio_learned_v2": raw / learned_v2_bytes, "ratio_plain_v2": raw / plain_v2_bytes,
             "gbs_learned_v2": raw / (t_learned_v2 / 1e3) / GB,
             "v2_decompress_gbs": raw / (t_dec_v2 / 1e3) / GB, "v2_round_trip_exact": v2_exact,
             "ratio_exhaustive": raw / best, "learned_vs_exhaustive_loss": learned_bytes / best - 1.0,
             "ratio_plain_whole_stream": raw / whole[ch.PLAIN_OPTION],
             "ratio_best_fixed_whole_stream": raw / whole[o_best], "best_fixed_option": o_best,
             "label_agreement": agree, "gbs_plain": raw / (t_plain / 1e3) / GB,
             "gbs_learned": raw / (t_learned / 1e3) / GB, "train_s": train_s,
             "learned_path_ms": {"features": t_feat, "mlp": t_mlp, "compress_learned_options": t_comp,
                                 "total": t_learned, "compress_plain_option": t_plain},
             "option_gbs_train": [round(n_train * ch.SEG * 2 / (t / 1e3) / GB, 1) for t in opt_ms],
             "throughput_floor": {"labels": "smallest option among those at least as fast as the plain one "
                                            "on the training segments",
                                  "allowed_options": [o for o, t in enumerate(opt_ms)
                                                      if t <= opt_ms[ch.PLAIN_OPTION]],
                                  "ratio": raw / fast_bytes, "gbs": raw / (t_fast / 1e3) / GB},
             "train_loss_first_last": [hist[0], hist[-1]],
             "note": "per-segment v1 streams (ratio_learned, ratio_plain) and the same segments as one "
                     "version-2 stream (_v2), all on the device (features, MLP, per-segment compression, "
                     "assembly); "
                     "data: camera events + white noise of varied sigma, train seed 11, test seed 12"},
            c)


def serve_metrics(dev, n_events, trained=None, v2=False):
    """The serving loop at 20k events/s (Poisson) from four camera
    geometries, continuous batching under an 8 GB budget, chooser off and on."""
    import numpy as np

    from paper_1805_01844_gb300 import serve
    from paper_1805_01844_gb300.chooser import Chooser

    rng = np.random.default_rng(0)
    pool = [(gi, serve.event_host(serve.GEOMETRIES[gi], 1000 + k))
            for k, gi in enumerate([k % 4 for k in range(64)])]
    ev = [pool[int(rng.integers(0, len(pool)))] for _ in range(n_events)]
    out = {}
    ch_l = trained or Chooser(dev, seed=0)
    runs = [("plain", None, False), ("learned", ch_l, False)] + ([("learned_v2", ch_l, True)] if v2 else [])
    for name, ch, use_v2 in runs:
        srv = serve.Server(dev, budget=8 << 30, n_streams=3, chooser=ch, v2=use_v2)
        srv.run(ev[: min(500, n_events)], rate=20000.0, seed=1)  # warm-up
        m = srv.run(ev, rate=20000.0, seed=2)
        m.pop("kept", None)
        out[name] = {k: m[k] for k in ("events", "rate_per_s", "p50_ms", "p99_ms", "gbs", "ratio", "wall_s",
                                       "slots_per_stream")}
    out["note"] = ("plain = one stream per event (advanced, L 1024, w 64); learned = the chooser trained in the "
                   "'learned' section, one stream per 4096-sample segment, each with a 64-byte header (~1.7 % at "
                   "this ratio); learned_v2 (--serve-v2) = the same segments joined into one version-2 stream per "
                   "event (a code byte and a 4-byte size per segment; one pc_assemble_v2 call per event); pedestal "
                   "+ noise events; events cycle a pool of 64")
    return out


def end_to_end(codec, x, n, steps, dev):
    """Same round trip through the public API with host buffers: pinned host
    samples -> H2D -> compress -> D2H of the stream (its exact size) ->
    decompress -> D2H of the samples, all inside the timed region."""
    import torch

    host_in = torch.empty(n, dtype=torch.int16, pin_memory=True)
    host_in.copy_(x.cpu())
    host_stream = torch.empty(codec.bound(n), dtype=torch.uint8, pin_memory=True)
    host_out = torch.empty(n, dtype=torch.int16, pin_memory=True)
    xin = torch.empty_like(x)
    sbuf = torch.empty(codec.bound(n), dtype=torch.uint8, device=dev)
    ybuf = torch.empty(n, dtype=torch.int16, device=dev)

    def one():  # one step at a time: upload, compress, download the stream, decompress, download
        xin.copy_(host_in, non_blocking=True)
        _, nb = codec.compress(xin, out=sbuf)
        nbytes = int(nb.item())
        host_stream[:nbytes].copy_(sbuf[:nbytes], non_blocking=True)
        codec.decompress(sbuf, nbytes, n, out=ybuf)
        host_out.copy_(ybuf, non_blocking=True)
        torch.cuda.synchronize()
        return nbytes

    one()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    tot_stream = 0
    for _ in range(steps):
        tot_stream += one()
    dt = time.perf_counter() - t0
    assert torch.equal(host_out, host_in)
    raw = n * 2
    seq = raw * steps / dt / GB
    # the same round trips pipelined over consecutive steps (the package's
    # RoundTrip): a step's upload overlaps the previous step's downloads
    from paper_1805_01844_gb300.pipeline import RoundTrip

    p = codec.params
    rt = RoundTrip(p.variant, p.dtype_bits, p.word_bits, p.block_len, n, device=dev)
    rt.submit(host_in)
    rt.drain()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(steps):
        rt.submit(host_in)
    rt.drain()
    dt = time.perf_counter() - t0
    done = rt.completed()
    for b in range(2):
        assert torch.equal(rt.host_out[b], host_in)
    nb = done[-1][1]
    assert torch.equal(rt.host_stream[done[-1][0]][:nb], host_stream[:nb])
    return {"value": raw * steps / dt / GB, "unit": "GB/s", "h2d_bytes_per_step": raw,
            "d2h_bytes_per_step": tot_stream // steps + raw,
            "pipelined": "consecutive steps overlap (an upload with the previous step's downloads), "
                         "through paper_1805_01844_gb300.pipeline.RoundTrip",
            "sequential_gbs": seq}


if __name__ == "__main__":
    main()
