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


def test_noalloc_rejects_streams_beyond_its_scratch():
    p = native.params(native.BASIC, 16, 64, 1)  # one block per sample: many tiles
    too_many = 40_000_000
    assert native.workspace_size(p, too_many) > native.NOALLOC_SCRATCH_BYTES
    fake = 1 << 40  # never dereferenced: the size check comes first
    st = native.compress_noalloc_raw(fake, too_many, p, fake, native.bound(p, too_many), fake, None)
    assert st == native.PC_ERR_UNSUPPORTED
