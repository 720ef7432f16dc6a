"""Device-side failure detection, made to happen without faulting the GPU:
corrupt and truncated streams, a short output, a workspace too small for the
stream, parameters that do not match the header, and a bounded wait that
runs out on a status word nothing sets.  The decoder's verdict is compared
with the oracle's on the same bytes."""
import time

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


def run_decode(stream, p, capacity, in_bytes=None, ws_samples=None):
    codec = pc.Codec(p.variant, p.dtype_bits, p.word_bits, p.block_len,
                     max_samples=capacity if ws_samples is None else ws_samples, device=dev())
    # keep the buffer exactly in_bytes long so that an over-read would leave it
    nb = len(stream) if in_bytes is None else in_bytes
    sd = torch.from_numpy(np.frombuffer(stream[:nb], dtype=np.uint8).copy()).to(dev())
    codec.decompress(sd, nb, capacity)
    return codec.device_status()


def oracle_verdict(stream, capacity):
    try:
        oracle.decompress(stream, capacity=capacity)
        return 0
    except oracle.OracleError as e:
        return e.code


@pytest.mark.parametrize("variant", [0, 1])
@pytest.mark.parametrize("w", [32, 64])
def test_corruptions_match_oracle(variant, w):
    x = datagen.white_noise(20000, 300.0, 5.0, seed=2)
    s = oracle.compress(x, variant, w, 1024)
    p = native.params(variant, 16, w, 1024)
    n_blocks = 20
    payload_off = 64 + ((n_blocks * 4 + 15) // 16) * 16
    cases = {
        "ok": s,
        "magic": b"X" + s[1:],
        "version": s[:4] + b"\x02" + s[5:],
        "reserved": s[:9] + b"\x01" + s[10:],
        "n_blocks": s[:24] + (21).to_bytes(8, "little") + s[32:],
        "payload_words+1": s[:32] + (int.from_bytes(s[32:40], "little") + 1).to_bytes(8, "little") + s[40:],
        "table_pad": s[:payload_off - 1] + b"\x01" + s[payload_off:],
        "table_overflow": s[:64] + (65535).to_bytes(2, "little") + (5).to_bytes(2, "little") + s[68:],
        "word_all_ones": s[:-(w // 8)] + b"\xff" * (w // 8),
        "first_word_all_ones": s[:payload_off] + b"\xff" * (w // 8) + s[payload_off + w // 8:],
    }
    if variant == 0:
        # a nonzero digit in the padding of the last block's last word, the
        # word still below B^p (every digit valid): only the padding check
        # rejects it
        e = int.from_bytes(s[64 + 4 * (n_blocks - 1):64 + 4 * n_blocks], "little")
        B = (e >> 16) + 1
        pw = 0
        while B ** (pw + 1) <= 2 ** w - 1:
            pw += 1
        last = int.from_bytes(s[-(w // 8):], "little")
        n_last = x.size - (n_blocks - 1) * 1024
        assert n_last % pw != 0 and last < B ** (pw - 1)
        cases["padding_digit"] = s[:-(w // 8)] + (last + B ** (pw - 1)).to_bytes(w // 8, "little")
    for name, stream in cases.items():
        want = oracle_verdict(stream, x.size)
        got = run_decode(stream, p, x.size)
        assert got == want, (name, got, want)
        if name != "ok":
            assert want == native.PC_ERR_CORRUPT, name
    # truncation at several points: never read past in_bytes, always CORRUPT
    for cut in (64, payload_off, payload_off + 8, len(s) - 1):
        assert oracle_verdict(s[:cut], x.size) == native.PC_ERR_CORRUPT
        assert run_decode(s, p, x.size, in_bytes=cut) == native.PC_ERR_CORRUPT
    # capacity and parameter mismatch
    assert run_decode(s, p, x.size - 1, ws_samples=x.size) == native.PC_ERR_CAPACITY
    other = native.params(1 - variant, 16, w, 1024)
    assert run_decode(s, other, x.size) == native.PC_ERR_CORRUPT
    other = native.params(variant, 16, w, 512)
    assert run_decode(s, other, x.size) == native.PC_ERR_CORRUPT


def test_random_bit_flips_never_misdecode_silently():
    """A flipped payload bit either makes the stream invalid (CORRUPT) or
    decodes to other samples; the GPU and the oracle agree on which, and on
    the samples."""
    rng = np.random.default_rng(9)
    x = datagen.white_noise(8192, 300.0, 5.0, seed=4)
    for variant in (0, 1):
        s = bytearray(oracle.compress(x, variant, 64, 1024))
        p = native.params(variant, 16, 64, 1024)
        for _ in range(12):
            t = bytearray(s)
            pos = int(rng.integers(128, len(t)))
            t[pos] ^= 1 << int(rng.integers(0, 8))
            want = oracle_verdict(bytes(t), x.size)
            assert run_decode(bytes(t), p, x.size) == want


def test_workspace_too_small_for_stream():
    """A workspace sized for fewer samples than the output capacity is refused
    by the host (PC_ERR_INVALID_ARG) before anything is launched; one sized
    for the capacity but smaller than a stream that exceeds it never gets
    used past its end either (the capacity check comes first)."""
    d = dev()
    x = datagen.white_noise(200000, 300.0, 5.0, seed=1)
    s = oracle.compress(x, 0, 64, 256)
    p = native.params(0, 16, 64, 256)
    ws_bytes = native.workspace_size(p, 1000)
    ws = torch.empty(ws_bytes, dtype=torch.uint8, device=d)
    sd = torch.from_numpy(np.frombuffer(s, dtype=np.uint8).copy()).to(d)
    out = torch.empty(x.size, dtype=torch.int16, device=d)
    n_out = torch.zeros(1, dtype=torch.int64, device=d)
    stream = torch.cuda.current_stream(d).cuda_stream
    assert native.decompress_raw(sd.data_ptr(), len(s), p, out.data_ptr(), x.size, n_out.data_ptr(),
                                 ws.data_ptr(), ws_bytes, stream) == native.PC_ERR_INVALID_ARG
    assert native.decompress_raw(sd.data_ptr(), len(s), p, out.data_ptr(), 1000, n_out.data_ptr(),
                                 ws.data_ptr(), ws_bytes, stream) == native.PC_OK
    assert native.last_device_status(ws.data_ptr(), stream) == native.PC_ERR_CAPACITY


def test_bounded_wait_gives_up():
    """The look-back wait used by both kernels, aimed at a status word that
    nothing publishes, returns after its limit with PC_ERR_TIMEOUT and leaves
    the context usable."""
    d = dev()
    p = native.params(0, 16, 64, 1024)
    nbytes = native.workspace_size(p, 0)
    ws = torch.empty(nbytes, dtype=torch.uint8, device=d)
    stream = torch.cuda.current_stream(d).cuda_stream
    t0 = time.time()
    assert native.selftest_bounded_wait(ws.data_ptr(), nbytes, 20000, stream) == 0
    assert native.last_device_status(ws.data_ptr(), stream) == native.PC_ERR_TIMEOUT
    assert time.time() - t0 < 5.0
    # the context still works
    x = datagen.white_noise(5000, seed=0)
    xd = torch.from_numpy(x.view(np.int16).copy()).to(d)
    buf = pc.compress(xd, 0, 64, 1024)
    assert buf.cpu().numpy().tobytes() == oracle.compress(x, 0, 64, 1024)
