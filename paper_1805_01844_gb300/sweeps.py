"""The paper's compression-ratio experiments, run on the GPU.

  ratio_vs_block_length   Sec. 4.2, Fig. 7: the ratio of vectors drawn from
                          A(mu, sigma, x, y, a, N) (Sec. 4.1) against the block
                          length, from one sample per block to the whole vector
                          (the unblocked method), basic and advanced
  ratio_vs_signal         Sec. 4.2, Fig. 8: the ratio against the number a of
                          uniform "signal" values among the N
  byte_profile            Sec. 5, Fig. 11: byte-value occurrences of the input
                          and of its compressed stream, and their entropy

Every vector is its own stream and every point is one batched launch over all
vectors (pc_compress_batch), so the stream of each vector is the one
pc_compress would write for it alone.  The ratio is taken, as in the paper's
simulated experiments, against 32-bit words: 4 N bytes per vector over its
stream without the 64-byte stream header (the per-block minimum and base are
counted, as the paper's block header).  Only marshalling and sums happen here;
the compression and the histogram are the library's kernels.
"""
import math

import numpy as np

from . import datagen, native

# Sec. 4.2's three distributions (mu = 3000, x = 2000, a = 4): Fig. 7 and 8's
# red (sigma 500, y 45000), blue (sigma 500, y 100000), green (sigma 1000, y 45000)
CURVES = (
    dict(name="sigma500_y45000", mu=3000.0, sigma=500.0, x=2000.0, y=45000.0),
    dict(name="sigma500_y100000", mu=3000.0, sigma=500.0, x=2000.0, y=100000.0),
    dict(name="sigma1000_y45000", mu=3000.0, sigma=1000.0, x=2000.0, y=45000.0),
)
BLOCK_LENGTHS = (1, 2, 4, 8, 16, 32, 48, 64, 96, 128, 154, 200, 256, 384, 512, 768, 1024, 1500)
SIGNAL_COUNTS = (1, 2, 4, 10, 20, 50, 100, 200, 500, 1000, 2000, 3000, 5000)


def _torch():
    import torch

    return torch


def vectors(curve, n_vec, N, a, seed=0):
    """n_vec vectors of A(mu, sigma, x, y, a, N) (uint32), one seed each."""
    return np.stack([datagen.paper_distribution(curve["mu"], curve["sigma"], curve["x"], curve["y"], a, N,
                                                seed=seed + i) for i in range(n_vec)])


def to_device(x, device):
    """Host vectors [n_vec, N] (uint32) as a CUDA int32 tensor whose rows start
    16 bytes apart at least (the row stride rounded up to 4 samples), the
    alignment the library requires of every stream's samples.  Returns the
    rows as a list of contiguous views."""
    torch = _torch()
    n_vec, N = x.shape
    pad = np.zeros((n_vec, (N + 3) // 4 * 4), dtype=np.uint32)
    pad[:, :N] = x
    xd = torch.from_numpy(pad.view(np.int32)).to(device)
    return [xd[i, :N] for i in range(n_vec)]


def batch_stream_sizes(rows, variant, word_bits, block_len):
    """Stream size of every row (CUDA int32 views of uint32 samples, 16-byte
    aligned, from to_device) compressed as its own stream, all rows in one
    batched launch.  Returns a host int64 array."""
    from .batch import Batch

    p = native.params(variant, 32, word_bits, block_len)
    b = Batch(rows, [p] * len(rows))
    b.compress()
    st = b.device_status()
    if st != native.PC_OK:
        raise native.PcError(st, "pc_compress_batch (device)")
    return b.nbytes.cpu().numpy().astype(np.int64)


def ratio_of(sizes, N):
    """Sec. 4.2's ratio: 32-bit words in over stream bytes out (no stream header)."""
    return 4.0 * N * len(sizes) / float(np.sum(np.asarray(sizes) - native.HEADER_BYTES))


def ratio_vs_block_length(device, n_vec=1000, N=1855, lengths=BLOCK_LENGTHS, curves=CURVES, word_bits=32,
                          seed=0, a=4):
    """Fig. 7: for each distribution, variant and block length (plus the whole
    vector, L = N), the ratio over n_vec vectors.  Returns a list of points
    {curve, variant, L, ratio, stream_bytes}."""
    out = []
    for curve in curves:
        xd = to_device(vectors(curve, n_vec, N, a, seed), device)
        for variant in (native.BASIC, native.ADVANCED):
            for L in list(lengths) + [N]:
                if L > N or L > native.MAX_BLOCK_LEN:
                    continue
                sizes = batch_stream_sizes(xd, variant, word_bits, L)
                out.append(dict(curve=curve["name"], variant=("basic", "advanced")[variant], L=int(L),
                                ratio=ratio_of(sizes, N), stream_bytes=int(sizes.sum())))
    return out


def ratio_vs_signal(device, n_vec=100, N=10000, counts=SIGNAL_COUNTS, curves=CURVES, block_len=154, word_bits=32,
                    variant=native.ADVANCED, seed=0):
    """Fig. 8: the ratio against the number of uniform signal values a (the
    signal fraction a / N) for vectors of N = 10,000 values, with the block
    length of Sec. 4.2's best case (154).  Returns points {curve, a,
    signal_fraction, ratio, stream_bytes}."""
    out = []
    for curve in curves:
        for a in counts:
            if a > N:
                continue
            xd = to_device(vectors(curve, n_vec, N, a, seed + 7919 * a), device)
            sizes = batch_stream_sizes(xd, variant, word_bits, block_len)
            out.append(dict(curve=curve["name"], a=int(a), signal_fraction=a / N, ratio=ratio_of(sizes, N),
                            stream_bytes=int(sizes.sum())))
    return out


def byte_histogram(buf, nbytes=None, stream=None):
    """Occurrences of each byte value in the first nbytes bytes of a CUDA
    tensor (pc_byte_histogram).  Returns a CUDA int64 tensor [256]."""
    torch = _torch()
    n = buf.numel() * buf.element_size() if nbytes is None else int(nbytes)
    hist = torch.empty(256, dtype=torch.int64, device=buf.device)
    s = (stream if stream is not None else torch.cuda.current_stream(buf.device)).cuda_stream
    st = native.byte_histogram_raw(buf.data_ptr(), n, hist.data_ptr(), s)
    if st != native.PC_OK:
        raise native.PcError(st, "pc_byte_histogram")
    return hist


def entropy_bits(hist):
    """Shannon entropy of a byte histogram, bits per byte (8 = flat)."""
    h = np.asarray(hist, dtype=np.float64)
    p = h[h > 0] / h.sum()
    return float(-(p * np.log2(p)).sum())


def byte_profile(x, streams):
    """Fig. 11: the byte profile of the samples x (a CUDA tensor) and of each
    compressed stream (name -> (CUDA uint8 buffer, size)).  Returns
    {name: {"hist": [256], "entropy_bits": e}} with "input" for x."""
    out = {"input": byte_histogram(x)}
    for name, (buf, size) in streams.items():
        out[name] = byte_histogram(buf, size)
    res = {}
    for name, h in out.items():
        hh = h.cpu().tolist()
        res[name] = {"hist": hh, "entropy_bits": entropy_bits(hh), "max_over_mean": max(hh) / (sum(hh) / 256.0)}
    return res


def summary(points, key="L"):
    """Best point and the unblocked point of each (curve, variant) in a Fig. 7
    sweep, with the loss of the longest blocks against the best."""
    res = {}
    for p in points:
        k = (p["curve"], p["variant"])
        res.setdefault(k, []).append(p)
    out = {}
    for (c, v), ps in res.items():
        best = max(ps, key=lambda q: q["ratio"])
        last = max(ps, key=lambda q: q[key])
        out["%s/%s" % (c, v)] = dict(best_L=best[key], best_ratio=best["ratio"], unblocked_L=last[key],
                                     unblocked_ratio=last["ratio"],
                                     unblocked_loss=1.0 - last["ratio"] / best["ratio"] if best["ratio"] else math.nan)
    return out
