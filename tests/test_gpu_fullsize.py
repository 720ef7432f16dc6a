"""Parity at the benchmark's full size and launch configuration: the 2.97 GB
camera workload (10,000 events x 2 x 40 x 1855 uint16) compressed and
decompressed exactly as bench.py times it.  The whole round trip is compared
on the device; sampled blocks spread over the stream are compared with the
oracle byte for byte (table entry and payload words at offsets recomputed
from the oracle's word counts), and the stream size with the oracle's count."""
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import bench  # noqa: E402
import paper_1805_01844_gb300 as pc  # noqa: E402
from paper_1805_01844_gb300 import datagen, native  # noqa: E402


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
    msg = bench.sampled_parity(x, sbuf, int(nb.item()), variant, w, L, n_samples=48, seed=variant + L)
    assert msg.startswith("ok")
