"""Whole-stream byte parity of the advanced variant (Sec. 3.2) at sizes where
compression runs full tiles: streams with more than 2,432 tiles of the
largest tile (32 blocks), so no tile is halved for a short stream, whatever
the tile size of the configuration.  Each configuration is compressed twice
through one workspace, the second time on fresh data with other wide blocks,
so that the series table kept in the workspace across calls is both reused
and extended; every byte of both streams is compared with the oracle, and
both decode back exactly.  The last tile is partial and the last block
ragged."""
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import numpy as np  # noqa: E402

import oracle  # noqa: E402
import paper_1805_01844_gb300 as pc  # noqa: E402
from paper_1805_01844_gb300 import datagen, native  # noqa: E402

FULL_TILES = 2432 * 32  # blocks above which no configuration halves its tiles
MULTI_TILES = 2432 * 96  # blocks above which 16-bit streams take look-back tiles of several stage tiles


def input_with_wide_blocks(n, L, d, seed, spike_every, spike):
    dt = np.uint16 if d == 16 else np.uint32
    x = datagen.white_noise(n, 300.0 if d == 16 else 70000.0, 5.0, seed=seed, dtype=dt)
    n_blocks = -(-n // L)
    rng = np.random.default_rng(seed + 1)
    # wide blocks with many different bases, so that many series are built
    for b in range(0, n_blocks - 1, spike_every):
        x[b * L + int(rng.integers(0, L))] = int(rng.integers(spike // 4, spike))
    return x


@pytest.mark.parametrize("d,L,w,extra", [(16, 1024, 64, 13), (16, 4096, 32, 5), (32, 1024, 64, 29),
                                         (16, 1024, 64, MULTI_TILES - FULL_TILES + 37),
                                         (16, 512, 32, MULTI_TILES - FULL_TILES + 70)])
def test_advanced_full_tiles_match_oracle_twice_on_one_workspace(d, L, w, extra):
    """The last two cases are long enough for look-back tiles of four stage
    tiles of 24 blocks (the last look-back tile partial)."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    dev = torch.device("cuda:0")
    n_blocks = FULL_TILES + extra
    n = (n_blocks - 1) * L + 611  # ragged last block
    codec = pc.Codec(pc.ADVANCED, d, w, L, max_samples=n, device=dev)
    sbuf = torch.empty(codec.bound(n), dtype=torch.uint8, device=dev)
    spike = 60000 if d == 16 else 3_000_000_000
    for call, (seed, every) in enumerate([(L + w, 977), (L + w + 100, 331)]):
        x = input_with_wide_blocks(n, L, d, seed, every, spike)
        want = oracle.compress(x, pc.ADVANCED, w, L)
        xd = torch.from_numpy(x.view(np.int16 if d == 16 else np.int32)).to(dev)
        sbuf.fill_(0xA5)
        _, nb = codec.compress(xd, out=sbuf)
        assert codec.device_status() == native.PC_OK
        k = int(nb.item())
        assert k == len(want), "call %d: stream size" % call
        got = sbuf[:k].cpu().numpy().tobytes()
        assert got == want, "call %d: stream bytes differ from the oracle" % call
        y, n_out = codec.decompress(sbuf, k, n)
        assert codec.device_status() == native.PC_OK
        assert int(n_out.item()) == n
        assert torch.equal(y[:n], xd), "call %d: round trip" % call
        del xd, y
