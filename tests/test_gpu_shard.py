"""One stream as K block-aligned shards on one GPU (Sec. 3.3: blocks are
independent): each shard compressed by pc_compress, the K stream sizes
exchanged through one device array, pc_stitch placing every shard's pieces.
The stitched stream must equal the oracle's stream of all samples byte for
byte; pc_slice of each shard's block range must equal the oracle's stream of
that shard's samples; decompressing the slices must give the samples back."""
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import numpy as np  # noqa: E402

import oracle  # noqa: E402
from paper_1805_01844_gb300 import datagen, native  # noqa: E402
from paper_1805_01844_gb300.shard import ShardedCodec  # noqa: E402

CASES = [
    # variant, d, w, L, n, K
    (0, 16, 64, 1024, 300 * 1024 + 77, 2),
    (0, 16, 64, 1024, 300 * 1024 + 77, 3),
    (1, 16, 64, 1024, 257 * 1024 + 5, 7),
    (1, 16, 32, 256, 1000 * 256, 3),
    (0, 32, 64, 1001, 90 * 1001 + 999, 7),  # shard starts not 16-byte aligned in the samples
    (1, 32, 32, 128, 50 * 128 + 1, 3),
    (0, 16, 32, 64, 3 * 64 + 5, 7),  # fewer blocks than shards: three shards are empty
    (0, 16, 64, 1024, 0, 3),  # no samples at all
]


@pytest.mark.parametrize("variant,d,w,L,n,K", CASES)
def test_sharded_stream_equals_the_oracle_stream(variant, d, w, L, n, K):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    dev = torch.device("cuda:0")
    dt = np.uint16 if d == 16 else np.uint32
    x = datagen.white_noise(max(n, 1), 300.0 if d == 16 else 90000.0, 6.0, seed=n + K, dtype=dt)[:n]
    if n:
        x[:: 4099] = 4000 if d == 16 else 3_000_000_000
    want = oracle.compress(x, variant, w, L)
    xd = torch.from_numpy(x.view(np.int16 if d == 16 else np.int32).copy()).to(dev)
    sc = ShardedCodec(variant, d, w, L, n, K, device=dev)
    out = torch.full((sc.bound(),), 0xA5, dtype=torch.uint8, device=dev)
    _, nbytes = sc.compress(xd, out=out)
    assert sc.device_status() == native.PC_OK
    k = int(nbytes.item())
    assert k == len(want)
    assert out[:k].cpu().numpy().tobytes() == want
    # each shard's block range cut back out: the oracle's stream of its samples
    for j, (f, c) in enumerate(sc.ranges):
        if c == 0:
            continue
        piece, pn = sc.slice(out, k, f // L, -(-c // L))
        assert sc.device_status() == native.PC_OK
        assert piece[: int(pn.item())].cpu().numpy().tobytes() == oracle.compress(x[f:f + c], variant, w, L)
    y = sc.decompress(out, k)
    torch.cuda.synchronize()
    assert torch.equal(y[:n], xd)


def test_slice_rejects_a_range_past_the_last_block():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    dev = torch.device("cuda:0")
    n, L = 10 * 256, 256
    x = datagen.white_noise(n, 300.0, 5.0, seed=2)
    xd = torch.from_numpy(x.view(np.int16)).to(dev)
    sc = ShardedCodec(0, 16, 64, L, n, 2, device=dev)
    out, nbytes = sc.compress(xd)
    k = int(nbytes.item())
    sc.slice(out, k, 8, 3)  # blocks 8, 9, 10: block 10 does not exist
    assert native.last_device_status(sc.ws.data_ptr(), torch.cuda.current_stream(dev).cuda_stream) == \
        native.PC_ERR_INVALID_ARG
