"""Parity at the benchmark's full size and launch configuration: the 2.97 GB
camera workload (10,000 events x 2 x 40 x 1855 uint16) compressed and
decompressed exactly as bench.py times it.  The whole round trip is compared
on the device; sampled blocks spread over the stream are compared with the
oracle byte for byte (table entry and payload words at offsets recomputed
from the oracle's word counts), and the stream size with the oracle's count."""
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import numpy as np  # noqa: E402

import oracle  # noqa: E402
import paper_1805_01844_gb300 as pc  # noqa: E402
from paper_1805_01844_gb300 import datagen, native  # noqa: E402


def sampled_parity(x, sbuf, stream_bytes, variant, w, L, n_samples=64, seed=0):
    """Check sampled blocks of the GPU stream against the oracle: table
    entries and payload words of blocks spread over the whole stream, with
    payload offsets recomputed from the table by the oracle's word counts."""
    n = x.numel()
    n_blocks = -(-n // L)
    table = sbuf[64: 64 + 4 * n_blocks].cpu().numpy().view(np.uint32)
    vmin = (table & 0xFFFF).astype(np.int64)
    B = (table >> 16).astype(np.int64) + 1
    nb = np.full(n_blocks, L, dtype=np.int64)
    nb[-1] = n - (n_blocks - 1) * L
    counts = np.zeros(n_blocks, dtype=np.int64)
    for b_val in np.unique(B):
        for nb_val in np.unique(nb[B == b_val]):
            m = (B == b_val) & (nb == nb_val)
            counts[m] = oracle.pack_count(variant, int(b_val), w, int(nb_val))
    offs = np.concatenate([[0], np.cumsum(counts)])
    payload_off = 64 + (4 * n_blocks + 15) // 16 * 16
    assert payload_off + offs[-1] * (w // 8) == stream_bytes, "stream size differs from the oracle's count"
    rng = np.random.default_rng(seed)
    picks = sorted(set([0, n_blocks - 1] + [int(b) for b in rng.integers(0, n_blocks, n_samples)]))
    wdt = np.uint64 if w == 64 else np.uint32
    for b in picks:
        xs = x[b * L: b * L + nb[b]].cpu().numpy().view(np.uint16)
        lo, hi = int(xs.min()), int(xs.max())
        assert (vmin[b], B[b]) == (lo, hi - lo + 1), "table entry of block %d" % b
        want = oracle.pack_block(variant, hi - lo + 1, w, xs.astype(np.uint64) - lo)
        a = payload_off + offs[b] * (w // 8)
        got = sbuf[a: a + counts[b] * (w // 8)].cpu().numpy().view(wdt)
        assert np.array_equal(got.astype(np.uint64), want), "payload of block %d" % b
    return "ok: %d sampled blocks byte-identical to the oracle, stream size equal" % len(picks)



@pytest.fixture(scope="module")
def workload():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    dev = torch.device("cuda:0")
    x = datagen.cherenkov_events_torch(10000, dev, seed=0).reshape(-1)
    yield x
    del x
    torch.cuda.empty_cache()


@pytest.mark.parametrize("variant,w,L", [(0, 64, 1024), (1, 64, 1024), (0, 32, 256), (1, 32, 4096)])
def test_full_size_round_trip_and_sampled_parity(workload, variant, w, L):
    x = workload
    n = x.numel()
    dev = x.device
    codec = pc.Codec(variant, 16, w, L, max_samples=n, device=dev)
    sbuf = torch.empty(codec.bound(n), dtype=torch.uint8, device=dev)
    _, nb = codec.compress(x, out=sbuf)
    y, n_out = codec.decompress(sbuf, sbuf.numel(), n)
    assert codec.device_status() == native.PC_OK
    assert int(n_out.item()) == n
    assert torch.equal(y[:n], x)
    msg = sampled_parity(x, sbuf, int(nb.item()), variant, w, L, n_samples=48, seed=variant + L)
    assert msg.startswith("ok")
