"""Long basic streams are compressed with look-back tiles of several stage
tiles (one look-back per K stage tiles, the earlier ones restaged after the
last is packed).  Every byte of such streams equals the oracle's, for ragged
ends where the last look-back tile has one, two or three stage tiles, the last
partial, and for both word sizes."""
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import numpy as np  # noqa: E402

import oracle  # noqa: E402
import paper_1805_01844_gb300 as pc  # noqa: E402
from paper_1805_01844_gb300 import datagen, native  # noqa: E402

SMALL_TILES = 2432  # tiles a stream needs before its compression takes multi-stage tiles (152 SMs x 16)


def stage_blocks(L, d=16):
    # blocks per stage tile of the basic compressor: 72 KB over (L + 64)-sample slots, a multiple of 8
    tb = min(32, (72 * 1024) // (((L + 64) * (d // 8) + 15) // 16 * 16))
    return tb & ~7 if tb >= 8 else tb


def stage_tiles_per_lookback(tb):
    # stage tiles per look-back tile: up to 96 blocks, at most 8 stage tiles
    return min(8, 96 // tb)


@pytest.mark.parametrize("d,L,w,extra_blocks", [(16, 1024, 64, 70), (16, 1024, 64, 5), (16, 1024, 32, 40),
                                                 (16, 4096, 64, 9), (32, 1024, 64, 50), (16, 512, 64, 7),
                                                 (16, 256, 32, 50), (16, 256, 64, 33)])
def test_multi_stage_tiles_match_oracle(d, L, w, extra_blocks):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    dev = torch.device("cuda:0")
    tb = stage_blocks(L, d)
    n_blocks = stage_tiles_per_lookback(tb) * tb * SMALL_TILES + extra_blocks
    n = (n_blocks - 1) * L + min(777, L - 5)  # ragged last block
    dt = np.uint16 if d == 16 else np.uint32
    x = datagen.white_noise(n, 300.0 if d == 16 else 70000.0, 5.0, seed=L + w + extra_blocks, dtype=dt)
    # a few wide blocks so that several bases occur
    for b in range(0, n_blocks - 1, 997):
        x[b * L] = 4000 if d == 16 else 3000000
    want = oracle.compress(x, 0, w, L)
    xd = torch.from_numpy(x.view(np.int16 if d == 16 else np.int32)).to(dev)
    codec = pc.Codec(0, d, w, L, max_samples=n, device=dev)
    sbuf = torch.empty(codec.bound(n), dtype=torch.uint8, device=dev)
    _, nb = codec.compress(xd, out=sbuf)
    assert codec.device_status() == native.PC_OK
    got = sbuf[: int(nb.item())].cpu().numpy().tobytes()
    assert len(got) == len(want)
    assert got == want
