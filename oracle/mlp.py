"""CPU oracle of the learned block-parameter chooser.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).  Plain numpy in float64:

  features(x, d, seg0)    segment statistics, one row per 4096 samples, in
                          the order include/pc.h documents
  forward(P, X)           MLP 24 -> 64 -> 64 -> 12 with ReLU, logits
  loss_grad(P, X, y)      mean softmax cross-entropy and its gradient,
                          written out layer by layer (chain rule)
  labels(x, variant)      exhaustive minimum-size search: every one of the 12
                          (block length, word size) options compressed by the
                          C oracle, the smallest stream wins (ties: lowest option)

P is a dict of float64 arrays W1[64,24], W2[64,64], W3[12,64], b1, b2, b3.
"""
import numpy as np

from . import compress

SEG = 4096
LENGTHS = (128, 256, 512, 1024, 2048, 4096)
NAMES = ("W1", "W2", "W3", "b1", "b2", "b3")
SHAPES = {"W1": (64, 24), "W2": (64, 64), "W3": (12, 64), "b1": (64,), "b2": (64,), "b3": (12,)}


def option_params(o):
    """(block length, word bits) of option o = 2 i + j."""
    return LENGTHS[o // 2], (32, 64)[o % 2]


def features(x, d, seg0=0):
    """Feature rows of the segments of x (uint16/uint32 array)."""
    x = np.asarray(x)
    nseg = -(-x.size // SEG)
    out = np.zeros((nseg, 24))
    dmax = 2.0 ** d - 1.0
    for s in range(nseg):
        seg = x[s * SEG:(s + 1) * SEG].astype(np.float64)
        ranges, valid = [], []
        for b in range(32):
            sub = seg[b * 128:(b + 1) * 128]
            if sub.size:
                ranges.append(sub.max() - sub.min())
                valid.append(True)
        ranges = np.array(ranges)
        cls = np.minimum(np.floor(np.log2(ranges + 1.0)), 15).astype(int)
        hist = np.bincount(cls, minlength=16)[:16] / 32.0
        rmin = ranges.min()
        spikes = np.sum(ranges > 4.0 * (rmin + 1.0)) / 32.0
        mean = seg.mean()
        var = max((seg * seg).mean() - mean * mean, 0.0)
        out[s, 0] = seg.min() / dmax
        out[s, 1] = seg.max() / dmax
        out[s, 2] = np.log2(seg.max() - seg.min() + 1.0) / d
        out[s, 3:19] = hist
        out[s, 19] = mean / dmax
        out[s, 20] = np.log2(var + 1.0) / (2.0 * d)
        out[s, 21] = spikes
        out[s, 22] = d / 32.0
        out[s, 23] = ((seg0 + s) % 64) / 64.0
    return out


def forward(P, X):
    H1 = np.maximum(X @ P["W1"].T + P["b1"], 0.0)
    H2 = np.maximum(H1 @ P["W2"].T + P["b2"], 0.0)
    return H2 @ P["W3"].T + P["b3"]


def loss_grad(P, X, y):
    """Mean cross-entropy of softmax(forward) against labels y, and its
    gradient with respect to every parameter."""
    n = X.shape[0]
    A1 = X @ P["W1"].T + P["b1"]
    H1 = np.maximum(A1, 0.0)
    A2 = H1 @ P["W2"].T + P["b2"]
    H2 = np.maximum(A2, 0.0)
    Z = H2 @ P["W3"].T + P["b3"]
    Zs = Z - Z.max(axis=1, keepdims=True)
    E = np.exp(Zs)
    Pr = E / E.sum(axis=1, keepdims=True)
    loss = -np.mean(np.log(Pr[np.arange(n), y]))
    dZ = Pr.copy()
    dZ[np.arange(n), y] -= 1.0
    dZ /= n
    G = {"W3": dZ.T @ H2, "b3": dZ.sum(axis=0)}
    dH2 = (dZ @ P["W3"]) * (A2 > 0)
    G["W2"] = dH2.T @ H1
    G["b2"] = dH2.sum(axis=0)
    dH1 = (dH2 @ P["W2"]) * (A1 > 0)
    G["W1"] = dH1.T @ X
    G["b1"] = dH1.sum(axis=0)
    return loss, G


def flatten(P):
    return np.concatenate([np.asarray(P[k], dtype=np.float64).ravel() for k in NAMES])


def unflatten(v):
    P, o = {}, 0
    for k in NAMES:
        size = int(np.prod(SHAPES[k]))
        P[k] = np.asarray(v[o:o + size], dtype=np.float64).reshape(SHAPES[k])
        o += size
    return P


def labels(x, variant=1):
    """Exhaustive minimum-size option of every segment of x, by compressing it
    with all 12 options (C oracle).  Returns (labels, sizes[nseg, 12])."""
    x = np.asarray(x)
    nseg = -(-x.size // SEG)
    sizes = np.zeros((nseg, 12), dtype=np.int64)
    for s in range(nseg):
        seg = np.ascontiguousarray(x[s * SEG:(s + 1) * SEG])
        for o in range(12):
            L, w = option_params(o)
            sizes[s, o] = len(compress(seg, variant, w, L))
    return np.argmin(sizes, axis=1).astype(np.uint8), sizes
