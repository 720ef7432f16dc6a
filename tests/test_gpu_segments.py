"""The chooser's device path (pc_segments_*): sources of ragged lengths cut
into 4096-sample segments, each compressed with its own option.  Every
segment stream must be byte-identical to the oracle's stream of that segment
under that option, the features to the oracle's per source, the device
totals to the stream sizes, and a source's results must not depend on the
other sources of the call."""
import numpy as np
import pytest

import oracle
from oracle import mlp
from paper_1805_01844_gb300 import native

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1805_01844_gb300 import chooser as ch  # noqa: E402

SEG = 4096
LENGTHS = (0, 1, 4095, 4096, 4097, 3 * 4096 + 17, 8 * 4096, 2 * 4096 + 4095)


def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch.device("cuda:0")


def source(n, d, seed):
    """Pedestal plus noise with spikes and a few constant stretches."""
    rng = np.random.default_rng(seed)
    top = 65535 if d == 16 else 4294967295
    x = np.rint(rng.normal(0, float(rng.uniform(1, 40)), n) + float(rng.uniform(100, 3000)))
    if n > 100:
        spikes = rng.choice(n, max(1, n // 300), replace=False)
        x[spikes] = rng.integers(0, top, spikes.size)
        a = int(rng.integers(0, n - 64))
        x[a:a + 64] = x[a]
    x = np.clip(x, 0, top)
    return x.astype(np.uint16 if d == 16 else np.uint32)


def to_dev(x):
    view = x.view(np.int16) if x.dtype == np.uint16 else x.view(np.int32)
    return torch.from_numpy(view.copy()).to(dev())


def seg_options(n_seg, seed):
    return np.random.default_rng(seed).integers(0, 12, n_seg).astype(np.uint8)


@pytest.mark.parametrize("d,variant", [(16, 0), (16, 1), (32, 0), (32, 1)])
def test_every_segment_matches_the_oracle(d, variant):
    xs = [source(n, d, 100 + k) for k, n in enumerate(LENGTHS)]
    sg = ch.Segments([to_dev(x) for x in xs], variant)
    counts = [-(-x.size // SEG) for x in xs]
    assert sg.n_segments == sum(counts)
    opts = seg_options(sg.n_segments, d + variant)
    opts[: min(12, sg.n_segments)] = np.arange(min(12, sg.n_segments))  # every option at least once
    sg.compress(torch.from_numpy(opts).to(dev()))
    assert sg.device_status() == native.PC_OK
    k = 0
    for i, x in enumerate(xs):
        got = sg.streams(i)
        assert len(got) == counts[i]
        for j, s in enumerate(got):
            L, w = mlp.option_params(int(opts[k]))
            assert s == oracle.compress(x[j * SEG:(j + 1) * SEG], variant, w, L), (i, j, int(opts[k]))
            k += 1


@pytest.mark.parametrize("d", [16, 32])
def test_features_per_source_match_the_oracle(d):
    xs = [source(n, d, 300 + k) for k, n in enumerate(LENGTHS)]
    sg = ch.Segments([to_dev(x) for x in xs], native.ADVANCED)
    got = sg.features().cpu().numpy()
    want = np.concatenate([mlp.features(x, d) for x in xs if x.size])
    np.testing.assert_allclose(got, want, rtol=2e-6, atol=1e-7)


def test_a_source_alone_and_in_a_mix_agree():
    xs = [source(n, 16, 500 + k) for k, n in enumerate((70000, 5000, 130000, 4096))]
    c = ch.Chooser(dev(), seed=5)
    mix = ch.Segments([to_dev(x) for x in xs], native.ADVANCED)
    fm = mix.features()
    mix.compress(c.predict(fm))
    for i, x in enumerate(xs):
        one = ch.Segments([to_dev(x)], native.ADVANCED)
        f1 = one.features()
        one.compress(c.predict(f1))
        k0 = sum(-(-y.size // SEG) for y in xs[:i])
        assert torch.equal(f1, fm[k0:k0 + f1.shape[0]])
        assert one.streams(0) == mix.streams(i)


def test_device_totals():
    xs = [source(n, 16, 700 + k) for k, n in enumerate((9000, 0, 4096, 20000))]
    tot = torch.zeros((2, 2), dtype=torch.int64, device=dev())
    sg = ch.Segments([to_dev(x) for x in xs], native.BASIC, totals=[tot[0], None, tot[1], tot[0]])
    opts = torch.from_numpy(seg_options(sg.n_segments, 1)).to(dev())
    for _ in range(2):
        sg.compress(opts)
    sizes = [sum(len(s) for s in sg.streams(i)) for i in range(4)]
    assert tot.cpu().tolist() == [[4, 2 * (sizes[0] + sizes[3])], [2, 2 * sizes[2]]]


def test_an_invalid_option_is_reported_and_the_slot_stays_valid():
    x = source(3 * SEG, 16, 900)
    sg = ch.Segments([to_dev(x)], native.ADVANCED)
    sg.compress(torch.tensor([5, 12, 200], dtype=torch.uint8, device=dev()))
    assert sg.device_status() == native.PC_ERR_INVALID_ARG
    got = sg.streams(0)
    assert got[0] == oracle.compress(x[:SEG], 1, 64, 512)
    assert got[1] == oracle.compress(x[SEG:2 * SEG], 1, 32, 128)  # option 0
    assert got[2] == oracle.compress(x[2 * SEG:], 1, 32, 128)


def test_graph_replay():
    """features -> MLP -> compression captured once and replayed."""
    xs = [source(n, 16, 950 + k) for k, n in enumerate((50000, 12288))]
    c = ch.Chooser(dev(), seed=9)
    sg = ch.Segments([to_dev(x) for x in xs], native.ADVANCED)
    s = torch.cuda.Stream(dev())
    with torch.cuda.stream(s):
        sg._stream = s
        sg.compress(c.predict(sg.features()))  # warm-up on the capture stream
        torch.cuda.synchronize(dev())
        want = [sg.streams(i) for i in range(2)]
        sg.nbytes[0].zero_()
        sg.nbytes[1].zero_()
        sg.buffer.zero_()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=s):
            sg.compress(c.predict(sg.features()))
    g.replay()
    torch.cuda.synchronize(dev())
    assert [sg.streams(i) for i in range(2)] == want
