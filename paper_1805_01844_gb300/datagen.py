"""Seeded synthetic inputs for the compression path and its tests.

This module holds no compression arithmetic: it only draws integer samples
with the structure of the workloads the paper compresses -- white noise
dominating a sparse signal (Sec. 2, Fig. 1), the simulated pixel distribution
A(mu, sigma, x, y, a, N) of Sec. 4.1 (Eq. A), and Cherenkov-camera waveform
matrices with M[i][j] = time i of pixel j (Sec. 4.3.1).  Both the CUDA path
and the CPU oracle take their inputs from here; neither is imported.

Host generators use numpy's PCG64 (``numpy.random.default_rng``); the large
device generators use torch's CUDA Philox generator with the same recipe.
Rounding is half-to-even, then values are clipped to the dtype (or detector)
range.
"""
import numpy as np

# ---------------------------------------------------------------- host side


def white_noise(n=65536, mean=300.0, sigma=5.0, seed=0, dtype=np.uint16):
    """Gaussian white noise rounded and clipped to the dtype range."""
    rng = np.random.default_rng(seed)
    hi = np.iinfo(dtype).max
    return np.clip(np.rint(rng.normal(mean, sigma, n)), 0, hi).astype(dtype)


def paper_distribution(mu, sigma, x, y, a, N, seed=0, dtype=np.uint32):
    """A(mu, sigma, x, y, a, N) = N(mu, sigma)^(N-a) U U(x, y)^a (Sec. 4.1).

    The a uniform 'signal' values sit at uniformly random positions among the
    N - a Gaussian 'noise' values."""
    rng = np.random.default_rng(seed)
    hi = np.iinfo(dtype).max
    v = np.rint(rng.normal(mu, sigma, N))
    pos = rng.choice(N, size=a, replace=False)
    v[pos] = np.rint(rng.uniform(x, y, a))
    return np.clip(v, 0, hi).astype(dtype)


def cherenkov_events(n_events, n_pixels=1855, n_gains=2, n_time=40, seed=0,
                     pulse_frac=0.02, pulse_mean=200.0, pulse_width=3.0,
                     saturation=4095):
    """Camera waveforms, layout [event][gain][time][pixel] (uint16).

    Per (gain, pixel): pedestal mean U(250, 350) and noise sigma U(3, 8), fixed
    across events.  Per event, round(pulse_frac * n_pixels) pixels carry a
    Gaussian pulse of width (sigma) pulse_width samples, amplitude
    Exp(pulse_mean) ADC and centre U[0, n_time), added to both gains.  Values
    saturate at `saturation`."""
    rng = np.random.default_rng(seed)
    ped = rng.uniform(250.0, 350.0, (n_gains, 1, n_pixels))
    sig = rng.uniform(3.0, 8.0, (n_gains, 1, n_pixels))
    out = np.empty((n_events, n_gains, n_time, n_pixels), dtype=np.uint16)
    n_pulse = int(round(pulse_frac * n_pixels))
    t = np.arange(n_time, dtype=np.float64)[:, None]
    for e in range(n_events):
        wave = rng.normal(0.0, 1.0, (n_gains, n_time, n_pixels)) * sig + ped
        pix = rng.choice(n_pixels, size=n_pulse, replace=False)
        amp = rng.exponential(pulse_mean, n_pulse)
        t0 = rng.uniform(0.0, n_time, n_pulse)
        shape = amp[None, :] * np.exp(-0.5 * ((t - t0[None, :]) / pulse_width) ** 2)
        wave[:, :, pix] += shape[None, :, :]
        out[e] = np.clip(np.rint(wave), 0, saturation)
    return out


def edge_block(B, n, seed=0, vmin=0, dtype=np.uint16):
    """n samples in [vmin, vmin + B - 1], uniform, except that (for n >= 2) one
    random position holds vmin and another holds vmin + B - 1, so that the
    block's range is exactly B."""
    rng = np.random.default_rng(seed)
    v = rng.integers(0, B, n, dtype=np.uint64)
    if n >= 2:
        i0, i1 = rng.choice(n, size=2, replace=False)
        v[i0] = 0
        v[i1] = B - 1
    return (v + vmin).astype(dtype)


# -------------------------------------------------------------- device side


def cherenkov_events_torch(n_events, device, n_pixels=1855, n_gains=2, n_time=40,
                           seed=0, pulse_frac=0.02, pulse_mean=200.0,
                           pulse_width=3.0, saturation=4095, chunk=500):
    """Same recipe as `cherenkov_events`, drawn on the GPU with torch's
    generator; returns a contiguous int16 tensor holding the uint16 bit
    pattern (all values are <= 4095), layout [event][gain][time][pixel]."""
    import torch

    g = torch.Generator(device=device)
    g.manual_seed(seed)
    f32 = torch.float32
    ped = torch.rand((n_gains, 1, n_pixels), generator=g, device=device, dtype=f32) * 100.0 + 250.0
    sig = torch.rand((n_gains, 1, n_pixels), generator=g, device=device, dtype=f32) * 5.0 + 3.0
    out = torch.empty((n_events, n_gains, n_time, n_pixels), dtype=torch.int16, device=device)
    n_pulse = int(round(pulse_frac * n_pixels))
    t = torch.arange(n_time, device=device, dtype=f32).view(1, n_time, 1)
    for e0 in range(0, n_events, chunk):
        e1 = min(n_events, e0 + chunk)
        m = e1 - e0
        wave = torch.randn((m, n_gains, n_time, n_pixels), generator=g, device=device, dtype=f32)
        wave.mul_(sig).add_(ped)
        pix = torch.rand((m, n_pixels), generator=g, device=device).argsort(dim=1)[:, :n_pulse]
        u = torch.rand((m, n_pulse), generator=g, device=device).clamp_min_(1e-12)
        amp = -pulse_mean * torch.log(u)
        t0 = torch.rand((m, n_pulse), generator=g, device=device) * n_time
        shape = amp.view(m, 1, n_pulse) * torch.exp(
            -0.5 * ((t - t0.view(m, 1, n_pulse)) / pulse_width) ** 2)  # [m, T, P']
        idx = pix.view(m, 1, 1, n_pulse).expand(m, n_gains, n_time, n_pulse)
        wave.scatter_add_(3, idx, shape.view(m, 1, n_time, n_pulse).expand(m, n_gains, n_time, n_pulse).contiguous())
        out[e0:e1] = torch.round(wave).clamp_(0, saturation).to(torch.int16)
    return out


def white_noise_torch(n, device, mean=300.0, sigma=5.0, seed=0):
    """Gaussian white noise on the GPU, uint16 bit pattern in an int16 tensor."""
    import torch

    g = torch.Generator(device=device)
    g.manual_seed(seed)
    x = torch.randn(n, generator=g, device=device) * sigma + mean
    return torch.round(x).clamp_(0, 65535).to(torch.int32).to(torch.int16)


def chooser_mix_torch(n_samples, device, seed=0, noise_frac=0.2, chunk_segments=64):
    """Data for the block-parameter chooser from the two workload generators:
    camera events (`cherenkov_events_torch`, whole events) for about
    1 - noise_frac of the samples, then Gaussian white noise around 300 (the
    65,536-sample workload's generator) in chunks of `chunk_segments` segments
    of 4096 samples, each chunk with its own sigma, log-uniform in [1, 100].
    int16 tensor (uint16 bit pattern) of exactly n_samples samples."""
    import torch

    per_event = 2 * 40 * 1855
    n_events = int((1.0 - noise_frac) * n_samples) // per_event
    parts = []
    if n_events:
        parts.append(cherenkov_events_torch(n_events, device, seed=seed).reshape(-1))
    rest = n_samples - n_events * per_event
    g = np.random.default_rng(seed + 1)
    step = chunk_segments * 4096
    for k, c0 in enumerate(range(0, rest, step)):
        m = min(step, rest - c0)
        sigma = float(np.exp(g.uniform(0.0, np.log(100.0))))
        parts.append(white_noise_torch(m, device, mean=300.0, sigma=sigma, seed=seed * 100003 + k))
    return torch.cat(parts) if len(parts) > 1 else parts[0]


# ------------------------------------------------------ batches of streams


def batched_stream_specs(n_streams=64, min_bytes=4096, max_bytes=64 << 20, seed=0):
    """Specs of independent streams: byte length log-uniform in
    [min_bytes, max_bytes], dtype uint16 or uint32 at random, white noise with
    sigma log-uniform in [1, 2000] around a mean U(100, 10000), and 0.5 %
    spikes of uniform amplitude up to the dtype maximum."""
    rng = np.random.default_rng(seed)
    specs = []
    for s in range(n_streams):
        nbytes = float(np.exp(rng.uniform(np.log(min_bytes), np.log(max_bytes))))
        dtype = np.uint16 if rng.integers(0, 2) == 0 else np.uint32
        n = max(1, int(nbytes) // np.dtype(dtype).itemsize)
        sigma = float(np.exp(rng.uniform(0.0, np.log(2000.0))))
        mean = float(rng.uniform(100.0, 10000.0))
        specs.append(dict(n=n, dtype=dtype, mean=mean, sigma=sigma, spike_frac=0.005,
                          seed=int(rng.integers(0, 2 ** 31))))
    return specs


def batched_stream(spec):
    """Host samples of one stream spec (numpy)."""
    rng = np.random.default_rng(spec["seed"])
    hi = np.iinfo(spec["dtype"]).max
    v = np.rint(rng.normal(spec["mean"], spec["sigma"], spec["n"]))
    k = int(round(spec["spike_frac"] * spec["n"]))
    if k:
        pos = rng.choice(spec["n"], size=k, replace=False)
        v[pos] = rng.uniform(0, hi, k)
    return np.clip(np.rint(v), 0, hi).astype(spec["dtype"])


def batched_stream_torch(spec, device):
    """Device samples of one stream spec (torch's generator; int16/int32 bit
    patterns of the uint16/uint32 values)."""
    import torch

    g = torch.Generator(device=device)
    g.manual_seed(spec["seed"])
    n = spec["n"]
    hi = float(np.iinfo(spec["dtype"]).max)
    v = torch.randn(n, generator=g, device=device, dtype=torch.float64) * spec["sigma"] + spec["mean"]
    k = int(round(spec["spike_frac"] * n))
    if k:
        pos = torch.randint(0, n, (k,), generator=g, device=device)
        v[pos] = torch.rand(k, generator=g, device=device, dtype=torch.float64) * hi
    v = torch.round(v).clamp_(0, hi)
    if spec["dtype"] == np.uint16:
        return v.to(torch.int32).to(torch.int16)
    return v.to(torch.int64).to(torch.int32)
