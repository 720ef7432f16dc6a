"""The paper's ratio experiments on the GPU (Sec. 4.2, Figs. 7-8; Sec. 5,
Fig. 11): every point of a sweep is a batched launch over independent
vectors of A(mu, sigma, x, y, a, N), and every vector's stream must be the
oracle's stream of that vector, byte for byte; the byte histogram kernel must
count exactly what numpy counts."""
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import numpy as np  # noqa: E402

import oracle  # noqa: E402
from paper_1805_01844_gb300 import native, sweeps  # noqa: E402


def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch.device("cuda:0")


@pytest.mark.parametrize("n,offset", [(0, 0), (1, 0), (15, 3), (4096, 0), (1_000_003, 7), (50_000_000, 9)])
def test_byte_histogram_counts_every_byte(n, offset):
    d = dev()
    rng = np.random.default_rng(n + offset)
    host = rng.integers(0, 256, n + offset + 5, dtype=np.uint8)
    host[offset: offset + n // 3] = 17  # a skewed profile
    buf = torch.from_numpy(host).to(d)
    got = sweeps.byte_histogram(buf[offset:offset + n], n).cpu().numpy()
    want = np.bincount(host[offset:offset + n], minlength=256)
    assert np.array_equal(got, want)


@pytest.mark.parametrize("curve", sweeps.CURVES, ids=[c["name"] for c in sweeps.CURVES])
def test_block_length_sweep_streams_equal_the_oracle(curve):
    """Fig. 7's sweep on a few vectors: every block length from 1 to the whole
    vector, both variants; every vector's stream equals the oracle's."""
    d = dev()
    n_vec, N = 6, 1855
    x = sweeps.vectors(curve, n_vec, N, 4, seed=3)
    xd = sweeps.to_device(x, d)
    for variant in (native.BASIC, native.ADVANCED):
        for L in (1, 7, 64, 154, 1000, N):
            sizes = sweeps.batch_stream_sizes(xd, variant, 32, L)
            want = [len(oracle.compress(x[i], variant, 32, L)) for i in range(n_vec)]
            assert sizes.tolist() == want, (curve["name"], variant, L)


def test_batched_vector_streams_are_the_oracle_bytes():
    d = dev()
    from paper_1805_01844_gb300.batch import Batch

    x = sweeps.vectors(sweeps.CURVES[1], 5, 1855, 4, seed=11)
    xd = sweeps.to_device(x, d)
    for variant in (native.BASIC, native.ADVANCED):
        p = native.params(variant, 32, 32, 154)
        b = Batch(xd, [p] * 5)
        b.compress()
        assert b.device_status() == native.PC_OK
        assert b.streams() == [oracle.compress(x[i], variant, 32, 154) for i in range(5)]


def test_signal_sweep_streams_equal_the_oracle():
    """Fig. 8's sweep on a few vectors of 10,000 values."""
    d = dev()
    for a in (1, 1000, 5000):
        x = sweeps.vectors(sweeps.CURVES[2], 3, 10000, a, seed=a)
        xd = sweeps.to_device(x, d)
        sizes = sweeps.batch_stream_sizes(xd, native.ADVANCED, 32, 154)
        assert sizes.tolist() == [len(oracle.compress(x[i], 1, 32, 154)) for i in range(3)]


def test_gpu_sweep_reproduces_section_4_2():
    """On 200 vectors of A(3000, 500, 2000, 45000, 4, 1855) the GPU sweep's
    advanced ratio at L = 154 is the paper's 2.47054 within 3 % and the
    unblocked one its 2.10361 within 1 % (the random numbers differ from the
    paper's, so this is statistical), and the longest blocks lose 15-35 %
    against the best (the paper: 25 % for sigma = 500)."""
    d = dev()
    pts = sweeps.ratio_vs_block_length(d, n_vec=200, curves=sweeps.CURVES[:1], lengths=(64, 100, 128, 154, 200, 256))
    by = {(p["variant"], p["L"]): p["ratio"] for p in pts}
    assert abs(by[("advanced", 154)] - 2.47054) / 2.47054 < 0.03
    assert abs(by[("advanced", 1855)] - 2.10361) / 2.10361 < 0.01
    s = sweeps.summary(pts)["sigma500_y45000/advanced"]
    assert 0.15 < s["unblocked_loss"] < 0.35
