"""GPU parity: the CUDA path through the C ABI against the CPU oracle.

Compression is integer work, so the bar is byte equality of the whole stream
with the oracle's, plus an exact round trip through the GPU decoder and exact
GPU decoding of the oracle's own streams.  Inputs span several tiles with a
ragged tail, every base B of 16-bit data, sampled bases of 32-bit data, odd
block lengths, the paper's simulated distribution (Sec. 4.1) and camera
waveforms (Sec. 4.3.1)."""
import numpy as np
import pytest

import oracle
from paper_1805_01844_gb300 import datagen, native

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1805_01844_gb300 as pc  # noqa: E402


def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch.device("cuda:0")


def to_dev(x):
    x = np.ascontiguousarray(x)
    view = x.view(np.int16) if x.dtype == np.uint16 else x.view(np.int32)
    return torch.from_numpy(view.copy()).to(dev())


def gpu_compress(x, variant, w, L):
    d = x.dtype.itemsize * 8
    codec = pc.Codec(variant, d, w, L, max_samples=x.size, device=dev())
    xd = to_dev(x)
    buf, nbytes = codec.compress(xd)
    st = codec.device_status()
    assert st == 0, native.strerror(st)
    return buf[: int(nbytes.item())].cpu().numpy().tobytes(), codec, xd


def gpu_decompress(stream, variant, d, w, L, capacity, expect_status=0):
    codec = pc.Codec(variant, d, w, L, max_samples=capacity, device=dev())
    sd = torch.from_numpy(np.frombuffer(stream, dtype=np.uint8).copy()).to(dev())
    out, n = codec.decompress(sd, len(stream), capacity)
    st = codec.device_status()
    assert st == expect_status, (native.strerror(st), expect_status)
    if st != 0:
        return None
    n = int(n.item())
    arr = out[:n].cpu().numpy()
    return arr.view(np.uint16) if d == 16 else arr.view(np.uint32)


def check(x, variant, w, L):
    want = oracle.compress(x, variant, w, L)
    got, _, _ = gpu_compress(x, variant, w, L)
    assert len(got) == len(want)
    if got != want:
        a = np.frombuffer(got, np.uint8)
        b = np.frombuffer(want, np.uint8)
        i = int(np.nonzero(a != b)[0][0])
        raise AssertionError("stream differs from the oracle at byte %d of %d" % (i, len(want)))
    d = x.dtype.itemsize * 8
    y = gpu_decompress(want, variant, d, w, L, x.size)
    assert np.array_equal(y, x)


CONFIGS = [(v, w) for v in (0, 1) for w in (32, 64)]


@pytest.mark.parametrize("variant,w", CONFIGS)
def test_white_noise_65536(variant, w):
    """65,536 uint16 samples of N(300, 5), seed 0, blocks of 1024."""
    x = datagen.white_noise(65536, 300.0, 5.0, seed=0)
    check(x, variant, w, 1024)


@pytest.mark.parametrize("variant,w", CONFIGS)
@pytest.mark.parametrize("dtype", [np.uint16, np.uint32])
def test_sizes_and_ragged_tails(variant, w, dtype):
    rng = np.random.default_rng(7)
    hi = np.iinfo(dtype).max
    for L in (1, 8, 16, 154, 1000, 1024, 4096, 8192):
        for n in (0, 1, L - 1, L, L + 1, 37 * L + 5):
            if n < 0:
                continue
            x = np.clip(rng.normal(5000, 40, n).round(), 0, hi).astype(dtype)
            check(x, variant, w, L)


@pytest.mark.parametrize("variant,w", CONFIGS)
def test_every_base_of_uint16(variant, w):
    """One block of 16 samples for every B in [1, 65536] (min and max both
    present), so every digit count, magic reciprocal and split series of
    16-bit data is exercised."""
    L = 16
    blocks = []
    for B in range(1, 65537):
        vmin = (B * 7919) % (65537 - B)
        blocks.append(datagen.edge_block(B, L, seed=B, vmin=vmin))
    x = np.concatenate(blocks)
    check(x, variant, w, L)


@pytest.mark.parametrize("variant,w", CONFIGS)
def test_sampled_bases_of_uint32(variant, w):
    rng = np.random.default_rng(11)
    Bs = [1, 2, 3, 255, 256, 65535, 65536, 65537, 2 ** 31 - 1, 2 ** 31, 2 ** 31 + 1,
          2 ** 32 - 2, 2 ** 32 - 1, 2 ** 32]
    Bs += [int(b) for b in rng.integers(2, 2 ** 32, 300)]
    Bs += [int(2 ** rng.uniform(1, 32)) for _ in range(300)]
    L = 64
    blocks = []
    for i, B in enumerate(Bs):
        vmin = int(rng.integers(0, 2 ** 32 - B + 1))
        blocks.append(datagen.edge_block(B, L, seed=i, vmin=vmin, dtype=np.uint32))
    check(np.concatenate(blocks), variant, w, L)


@pytest.mark.parametrize("variant,w", CONFIGS)
def test_paper_distribution_blocks_of_154(variant, w):
    """A(3000, 500, 2000, 45000, 4, 1855) of Sec. 4.1 as 32-bit samples, in
    blocks of 154 (the best block size of Sec. 4.2; 616 bytes, not a multiple
    of 16, so the element-wise staging path runs)."""
    x = np.concatenate([datagen.paper_distribution(3000, 500, 2000, 45000, 4, 1855, seed=s)
                        for s in range(40)])
    check(x, variant, w, 154)


@pytest.mark.parametrize("variant,w", CONFIGS)
@pytest.mark.parametrize("L", [256, 1024, 4096])
def test_camera_events(variant, w, L):
    x = datagen.cherenkov_events(6, seed=3).reshape(-1)
    check(x, variant, w, L)


@pytest.mark.parametrize("variant", [0, 1])
def test_constant_and_extreme_blocks(variant):
    L = 512
    parts = [np.full(L, 7, np.uint16), np.full(L, 65535, np.uint16),
             np.tile(np.array([0, 65535], np.uint16), L // 2),
             np.zeros(L, np.uint16), np.arange(L, dtype=np.uint16)]
    x = np.concatenate(parts * 9 + [np.full(100, 3, np.uint16)])
    for w in (32, 64):
        check(x, variant, w, L)
    x32 = np.concatenate([np.full(L, 2 ** 32 - 1, np.uint32),
                          np.tile(np.array([0, 2 ** 32 - 1], np.uint32), L // 2),
                          np.zeros(L, np.uint32)] * 5)
    for w in (32, 64):
        check(x32, variant, w, L)


def test_launch_configuration_independence():
    """Same bytes whatever the interleaving of tiles across CTAs: repeated
    runs on a stream of many tiles are identical."""
    x = datagen.white_noise(3_000_000, 300.0, 5.0, seed=5)
    want = oracle.compress(x, 0, 64, 1024)
    for _ in range(3):
        got, _, _ = gpu_compress(x, 0, 64, 1024)
        assert got == want


@pytest.mark.parametrize("variant,w", CONFIGS)
@pytest.mark.parametrize("dtype", [np.uint16, np.uint32])
@pytest.mark.parametrize("L", [32, 64, 128, 256])
def test_short_blocks_with_constant_blocks_among_them(variant, w, dtype, L):
    """Short blocks (a few words each, packed a lane per word across the
    tile's blocks), one in three constant (no words) and some wide, over many
    tiles with a ragged last block."""
    rng = np.random.default_rng(L + w + 3 * variant)
    n_blocks = 32 * 40 + 7
    hi = np.iinfo(dtype).max
    x = np.clip(rng.normal(900, 30, n_blocks * L), 0, hi).astype(dtype)
    for b in range(n_blocks):
        r = int(rng.integers(0, 6))
        if r < 2:
            x[b * L:(b + 1) * L] = int(rng.integers(0, hi))
        elif r == 2:
            x[b * L + int(rng.integers(0, L))] = hi
    check(x[: n_blocks * L - L // 2 + 1], variant, w, L)
