"""pc_compress_noalloc, the entry point for callers that cannot allocate
device memory (for example a readout loop that must not call cudaMalloc once
running): it must produce exactly the stream pc_compress produces, on
consecutive calls that reuse its static scratch, and refuse streams too long
for that scratch.  This file is collected last on purpose."""
import numpy as np
import pytest

from paper_1805_01844_gb300 import datagen, native

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_noalloc_matches_pc_compress_on_consecutive_calls():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1805_01844_gb300 as pc

    dev = torch.device("cuda:0")
    stream = torch.cuda.current_stream(dev).cuda_stream
    cases = [(pc.BASIC, 64, 1024, 0, 3_000_000), (pc.ADVANCED, 32, 256, 1, 700_001)]
    for variant, w, L, seed, n in cases:  # two calls in a row on the same scratch
        x = datagen.white_noise(n, 300.0, 5.0, seed=seed)
        xd = torch.from_numpy(x.view(np.int16).copy()).to(dev)
        codec = pc.Codec(variant, 16, w, L, max_samples=n, device=dev)
        ref, ref_n = codec.compress(xd)
        assert codec.device_status() == native.PC_OK
        p = native.params(variant, 16, w, L)
        out = torch.full((native.bound(p, n),), 0xAB, dtype=torch.uint8, device=dev)
        nbytes = torch.zeros(1, dtype=torch.int64, device=dev)
        st = native.compress_noalloc_raw(xd.data_ptr(), n, p, out.data_ptr(), out.numel(),
                                         nbytes.data_ptr(), stream)
        assert st == native.PC_OK, native.strerror(st)
        torch.cuda.synchronize()
        k = int(ref_n.item())
        assert int(nbytes.item()) == k
        assert torch.equal(out[:k], ref[:k])


def test_noalloc_near_its_scratch_limit_matches_pc_compress():
    """A basic uint16 stream at block_len 256 sized a few tiles under the
    scratch limit, so that the look-back words fill almost all of the static
    array: the same bytes as pc_compress, and it decodes back exactly."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1805_01844_gb300 as pc

    dev = torch.device("cuda:0")
    stream = torch.cuda.current_stream(dev).cuda_stream
    p = native.params(pc.BASIC, 16, 32, 256)
    lo, hi = 0, 1 << 32
    while hi - lo > 1:
        m = (lo + hi) // 2
        if native.workspace_size(p, m) <= native.NOALLOC_SCRATCH_BYTES:
            lo = m
        else:
            hi = m
    n = lo - 256 * 40 - 77  # ragged last block, a few tiles under the limit
    assert native.workspace_size(p, n) > native.NOALLOC_SCRATCH_BYTES * 0.99
    x = datagen.white_noise_torch(n, dev, 300.0, 5.0, seed=3)
    codec = pc.Codec(pc.BASIC, 16, 32, 256, max_samples=n, device=dev)
    ref, ref_n = codec.compress(x)
    assert codec.device_status() == native.PC_OK
    out = torch.full((native.bound(p, n),), 0x5A, dtype=torch.uint8, device=dev)
    nbytes = torch.zeros(1, dtype=torch.int64, device=dev)
    st = native.compress_noalloc_raw(x.data_ptr(), n, p, out.data_ptr(), out.numel(), nbytes.data_ptr(), stream)
    assert st == native.PC_OK, native.strerror(st)
    torch.cuda.synchronize()
    k = int(ref_n.item())
    assert int(nbytes.item()) == k
    assert torch.equal(out[:k], ref[:k])
    y, n_out = codec.decompress(out, k, n)
    assert codec.device_status() == native.PC_OK
    assert int(n_out.item()) == n and torch.equal(y[:n], x)
