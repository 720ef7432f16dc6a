"""The series table of the advanced variant lives in the caller's workspace
and is kept across calls that reuse it.  Whatever the workspace held before
(garbage, a table for the other word size, another layout's data, a call of
the basic variant), every stream must still equal the oracle's and decode
exactly."""
import numpy as np
import pytest

import oracle
from paper_1805_01844_gb300 import datagen, native

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1805_01844_gb300 import chooser as ch  # noqa: E402
from paper_1805_01844_gb300.batch import Batch  # noqa: E402


def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch.device("cuda:0")


def to_dev(x):
    view = x.view(np.int16) if x.dtype == np.uint16 else x.view(np.int32)
    return torch.from_numpy(view.copy()).to(dev())


def data(n, seed):
    x = datagen.paper_distribution(3000, 500, 2000, 45000, 4, n, seed=seed)
    return np.clip(x, 0, 65535).astype(np.uint16)


def run(x, variant, w, L, ws, decode=True):
    """Compress (and decode) x through the raw ABI with the shared workspace."""
    p = native.params(variant, 16, w, L)
    xd = to_dev(x)
    cap = native.bound(p, x.size)
    out = torch.empty(cap, dtype=torch.uint8, device=dev())
    cnt = torch.zeros(2, dtype=torch.int64, device=dev())
    h = torch.cuda.current_stream().cuda_stream
    assert native.compress_raw(xd.data_ptr(), x.size, p, out.data_ptr(), cap, cnt.data_ptr(), ws.data_ptr(),
                               ws.numel(), h) == native.PC_OK
    assert native.last_device_status(ws.data_ptr(), h) == native.PC_OK
    nb = int(cnt[0].item())
    got = out[:nb].cpu().numpy().tobytes()
    assert got == oracle.compress(x, variant, w, L), (variant, w, L)
    if decode:
        y = torch.empty(x.size, dtype=torch.int16, device=dev())
        assert native.decompress_raw(out.data_ptr(), nb, p, y.data_ptr(), x.size, cnt[1:].data_ptr(),
                                     ws.data_ptr(), ws.numel(), h) == native.PC_OK
        assert native.last_device_status(ws.data_ptr(), h) == native.PC_OK
        assert np.array_equal(y.cpu().numpy().view(np.uint16), x)


def test_one_workspace_through_changing_calls():
    sizes = (300000, 123457, 4096 * 7 + 5)
    need = max(native.workspace_size(native.params(1, 16, w, L), n)
               for n in sizes for w in (32, 64) for L in (154, 1024))
    ws = torch.full(((need + 15) // 16 * 16,), 0xA5, dtype=torch.uint8, device=dev())  # garbage first
    x = [data(n, 10 + k) for k, n in enumerate(sizes)]
    run(x[0], 1, 64, 1024, ws)
    run(x[1], 1, 64, 154, ws)      # same word size: table kept, another block length and size
    run(x[2], 1, 32, 1024, ws)     # other word size: table rebuilt
    run(x[0], 1, 64, 1024, ws)     # back again
    run(x[1], 0, 64, 1024, ws)     # basic: no table, tag cleared
    run(x[2], 1, 64, 154, ws)
    ws.fill_(0x5C)                 # the caller scribbles over the workspace
    run(x[0], 1, 32, 154, ws)
    run(x[1], 1, 32, 1024, ws)


def test_batches_and_segments_reuse_their_workspace():
    rng = np.random.default_rng(7)
    xs = [data(int(n), 30 + k) for k, n in enumerate(rng.integers(1000, 200000, 6))]
    params = [native.params(1, 16, (32, 64)[k % 2], (154, 1024)[k % 3 == 0]) for k in range(len(xs))]
    ws = torch.full((((40 << 20) + 15) // 16 * 16,), 0x33, dtype=torch.uint8, device=dev())  # garbage first
    for rep in range(3):
        b = Batch([to_dev(x) for x in xs], params, workspace=ws)
        assert b.ws is ws
        b.compress()
        assert b.device_status() == 0
        for x, p, s in zip(xs, params, b.streams()):
            assert s == oracle.compress(x, p.variant, p.word_bits, p.block_len), rep
    # the same workspace through the segments path (same layout, same tag)
    seg = ch.Segments([to_dev(x) for x in xs[:3]], native.ADVANCED, workspace=ws)
    assert seg.ws is ws
    opts = torch.from_numpy(rng.integers(0, 12, seg.n_segments).astype(np.uint8)).to(dev())
    for _ in range(2):
        seg.compress(opts)
        assert seg.device_status() == 0
    k = 0
    for i, x in enumerate(xs[:3]):
        for j, s in enumerate(seg.streams(i)):
            L, w = (128 << (int(opts[k]) // 2)), (32, 64)[int(opts[k]) % 2]
            assert s == oracle.compress(x[j * 4096:(j + 1) * 4096], 1, w, L)
            k += 1
