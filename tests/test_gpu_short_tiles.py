"""Long streams of short basic blocks (16-bit L = 8 ... 256, 32-bit L = 16,
128) are compressed with look-back tiles of up to 128 whole blocks (group min/max, a thread per block
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


@pytest.mark.parametrize("d,L,w", [(16, 8, 64), (16, 32, 32), (16, 64, 64), (16, 128, 32), (16, 128, 64),
                                   (16, 256, 64), (32, 16, 32), (32, 128, 64)])
def test_short_block_tiles_match_oracle(d, L, w):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    dev = torch.device("cuda:0")
    tile_blocks = min(128, 32768 // (L * d // 8))  # blocks per look-back tile
    n_blocks = tile_blocks * SMALL_TILES + 77
    n = (n_blocks - 1) * L + max(1, L // 2 - 3)  # ragged last block
    rng = np.random.default_rng(L + w + d)
    dt = np.uint16 if d == 16 else np.uint32
    hi = np.iinfo(dt).max
    x = np.clip(rng.normal(1200 if d == 16 else 3e6, 9 if d == 16 else 4000, n), 0, hi).astype(dt)
    nb = -(-n // L)
    for b in rng.integers(0, nb - 1, nb // 50):  # constant blocks
        x[b * L:(b + 1) * L] = 4321
    x[rng.integers(0, n, n // 3000)] = hi  # wide blocks
    x[-3:] = [0, hi, 17]  # the ragged last block spans the whole range
    want = oracle.compress(x, 0, w, L)
    xd = torch.from_numpy(x.view(np.int16 if d == 16 else np.int32)).to(dev)
    codec = pc.Codec(0, d, w, L, max_samples=n, device=dev)
    sbuf = torch.empty(codec.bound(n), dtype=torch.uint8, device=dev)
    _, nbytes = codec.compress(xd, out=sbuf)
    assert codec.device_status() == native.PC_OK
    k = int(nbytes.item())
    assert k == len(want)
    assert sbuf[:k].cpu().numpy().tobytes() == want
    y, n_out = codec.decompress(sbuf, k, n)
    assert codec.device_status() == native.PC_OK
    assert int(n_out.item()) == n and torch.equal(y[:n], xd)
