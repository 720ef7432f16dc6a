"""Format version 2 (segmented streams) on the GPU against the oracle.

The block length is the parameter the paper tunes by hand (Sec. 3.3;
Sec. 4.2, Fig. 7); a version-2 stream records it, with the word size, per
segment.  Streams assembled on the GPU from the per-segment compressions of
the learned chooser's path must equal the oracle's version-2 stream byte for
byte; the GPU decoder must give back the samples of the oracle's streams for
every one of the 28 codes (block lengths 1 to 8192, blocks longer than the
segment included) and flag corrupt streams."""
import numpy as np
import pytest

import oracle
from paper_1805_01844_gb300 import datagen, native

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1805_01844_gb300 import chooser  # noqa: E402

SEG = native.SEGMENT_SAMPLES


def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch.device("cuda:0")


def to_dev(x):
    return torch.from_numpy(x.view(np.int16 if x.dtype == np.uint16 else np.int32).copy()).to(dev())


def samples(dtype, n, seed):
    rng = np.random.default_rng(seed)
    hi = np.iinfo(dtype).max
    x = np.clip(rng.normal(2000, 25, n), 0, hi).astype(dtype)
    x[rng.integers(0, n, max(n // 900, 1))] = hi // 5  # spikes: wide blocks here and there
    x[: min(n, 3 * SEG)] = 777  # constant segments (blocks without words)
    return x


def gpu_decode(stream, variant, d, seg_len, n, expect=native.PC_OK):
    buf = torch.from_numpy(np.frombuffer(stream, dtype=np.uint8).copy()).to(dev())
    out, n_out, ws = chooser.decompress_v2(buf, len(stream), variant, d, n, seg_len=seg_len)
    st = native.last_device_status(ws.data_ptr(), torch.cuda.current_stream().cuda_stream)
    assert st == expect, (native.strerror(st), native.strerror(expect))
    if st != native.PC_OK:
        return None
    assert int(n_out.item()) == n
    y = out[:n].cpu().numpy()
    return y.view(np.uint16) if d == 16 else y.view(np.uint32)


@pytest.mark.parametrize("variant,dtype", [(0, np.uint16), (1, np.uint16), (0, np.uint32), (1, np.uint32)])
def test_assembled_stream_matches_oracle(variant, dtype):
    """Every segment with a random chooser option (ragged last segment): the
    GPU's version-2 stream equals the oracle's, twice on one workspace, and
    decodes back (32-bit advanced: the GPU decoder reports unsupported)."""
    n = 37 * SEG + 1234
    x = samples(dtype, n, seed=variant + 7 * (dtype == np.uint32))
    rng = np.random.default_rng(3)
    for call in range(2):
        opts = rng.integers(0, native.CHOOSER_OPTIONS, -(-n // SEG)).astype(np.uint8)
        seg = chooser.Segments([to_dev(x)], variant)
        seg.compress(torch.from_numpy(opts).to(dev()))
        buf, nb = seg.assemble_v2(0)
        assert seg.v2_status() == native.PC_OK
        got = buf[: int(nb.item())].cpu().numpy().tobytes()
        want = oracle.compress_v2(x, variant, SEG, [chooser.v2_code(int(o)) for o in opts])
        assert len(got) == len(want), "call %d" % call
        assert got == want, "call %d: stream differs from the oracle" % call
        # each segment's 64-byte header became a code byte and a 4-byte size
        # (paddings to 8 bytes instead of 16 for the table: at most 4 more)
        assert len(got) <= seg.total_bytes() - 55 * len(opts) + 75
        d = x.dtype.itemsize * 8
        if variant == 1 and d == 32:
            buf2 = torch.from_numpy(np.frombuffer(want, dtype=np.uint8).copy()).to(dev())
            with pytest.raises(native.PcError) as e:
                chooser.decompress_v2(buf2, len(want), variant, d, n)
            assert e.value.code == native.PC_ERR_UNSUPPORTED
        else:
            assert np.array_equal(gpu_decode(want, variant, d, SEG, n), x)
        x = samples(dtype, n, seed=100 + call)


@pytest.mark.parametrize("variant,dtype", [(0, np.uint16), (1, np.uint16), (0, np.uint32)])
@pytest.mark.parametrize("seg_len", [700, 10000])
def test_every_code_decodes(variant, dtype, seg_len):
    """All 28 codes, cycled over the segments: block lengths 1 to 8192 (more
    than 32 blocks per segment, and blocks longer than the segment), both
    word sizes; the oracle's stream decodes exactly on the GPU."""
    codes = [k | (0x80 if wide else 0) for k in range(14) for wide in (0, 1)]
    n_seg = 2 * len(codes) + 1
    n = (n_seg - 1) * seg_len + seg_len // 3
    x = samples(dtype, n, seed=seg_len + variant)
    cs = [codes[s % len(codes)] for s in range(n_seg)]
    s = oracle.compress_v2(x, variant, seg_len, cs)
    assert np.array_equal(gpu_decode(s, variant, x.dtype.itemsize * 8, seg_len, n), x)


def test_empty_stream():
    x = np.zeros(0, dtype=np.uint16)
    s = oracle.compress_v2(x, 1, SEG, [])
    seg = chooser.Segments([to_dev(np.zeros(0, np.uint16))], 1)
    buf, nb = seg.assemble_v2(0)
    assert seg.v2_status() == native.PC_OK
    assert buf[: int(nb.item())].cpu().numpy().tobytes() == s
    assert gpu_decode(s, 1, 16, SEG, 0).size == 0


def test_corrupt_streams_are_flagged():
    n = 9 * SEG + 77
    x = samples(np.uint16, n, seed=11)
    cs = [chooser.v2_code(o) for o in (0, 3, 5, 7, 11, 1, 2, 9, 4, 6)]
    s = bytearray(oracle.compress_v2(x, 1, SEG, cs))
    assert np.array_equal(gpu_decode(bytes(s), 1, 16, SEG, n), x)
    sizes_at = 64 + 16
    # a code out of range, reserved code bits, a stored size, n_samples + 256
    # (more words than stored), seg_len
    for pos, val in [(64 + 2, 0x0E), (64 + 3, 0x47), (sizes_at + 4, None), (17, None), (12, None)]:
        bad = bytearray(s)
        bad[pos] = val if val is not None else (bad[pos] + 1) & 0xFF
        with pytest.raises(oracle.OracleError):
            oracle.decompress_v2(bytes(bad), n + 300)
        gpu_decode(bytes(bad), 1, 16, SEG, n + 300, expect=native.PC_ERR_CORRUPT)
    # the stream read as basic, or with another segment length: the header disagrees
    gpu_decode(bytes(s), 0, 16, SEG, n, expect=native.PC_ERR_CORRUPT)
    gpu_decode(bytes(s), 1, 16, 2048, n, expect=native.PC_ERR_CORRUPT)
    # too small an output
    gpu_decode(bytes(s), 1, 16, SEG, n - 1, expect=native.PC_ERR_CAPACITY)
