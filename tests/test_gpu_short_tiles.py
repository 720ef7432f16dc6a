"""Long streams of short 16-bit basic blocks (L = 8 ... 256) are compressed
with look-back tiles of 128 (L = 256: 64) whole blocks (group min/max, a thread per block
for the word counts, words packed a lane per word across the tile).  Every
byte of such streams equals the oracle's — constant blocks (no words), wide
blocks, a ragged last block — and the stream decodes back."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import oracle  # noqa: E402
import paper_1805_01844_gb300 as pc  # noqa: E402
from paper_1805_01844_gb300 import native  # noqa: E402

SMALL_TILES = 2432  # tiles a stream needs before it takes these tiles (152 SMs x 16)


@pytest.mark.parametrize("L,w", [(8, 64), (32, 32), (64, 64), (128, 32), (128, 64), (256, 64)])
def test_short_block_tiles_match_oracle(L, w):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    dev = torch.device("cuda:0")
    tile_blocks = 128 if L <= 128 else 64  # blocks per look-back tile
    n_blocks = tile_blocks * SMALL_TILES + 77
    n = (n_blocks - 1) * L + max(1, L // 2 - 3)  # ragged last block
    rng = np.random.default_rng(L + w)
    x = np.clip(rng.normal(1200, 9, n), 0, 65535).astype(np.uint16)
    nb = -(-n // L)
    for b in rng.integers(0, nb - 1, nb // 50):  # constant blocks
        x[b * L:(b + 1) * L] = 4321
    x[rng.integers(0, n, n // 3000)] = 65535  # wide blocks
    x[-3:] = [0, 65535, 17]  # the ragged last block spans the whole range
    want = oracle.compress(x, 0, w, L)
    xd = torch.from_numpy(x.view(np.int16)).to(dev)
    codec = pc.Codec(0, 16, w, L, max_samples=n, device=dev)
    sbuf = torch.empty(codec.bound(n), dtype=torch.uint8, device=dev)
    _, nbytes = codec.compress(xd, out=sbuf)
    assert codec.device_status() == native.PC_OK
    k = int(nbytes.item())
    assert k == len(want)
    assert sbuf[:k].cpu().numpy().tobytes() == want
    y, n_out = codec.decompress(sbuf, k, n)
    assert codec.device_status() == native.PC_OK
    assert int(n_out.item()) == n and torch.equal(y[:n], xd)
