"""The learned block-parameter chooser on the GPU: features, forward pass and
gradient of the hand-written BF16/FP32 kernels against the fp64 CPU oracle,
the GPU's exhaustive size search against the oracle's, and what a network
trained on the oracle's labels gains over the plain heuristic."""
import numpy as np
import pytest

import oracle
from oracle import mlp
from paper_1805_01844_gb300 import datagen, native

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1805_01844_gb300 import chooser as ch  # noqa: E402


def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch.device("cuda:0")


def to_dev(x):
    view = x.view(np.int16) if x.dtype == np.uint16 else x.view(np.int32)
    return torch.from_numpy(view.copy()).to(dev())


def mixed_data(seed, n_events=2, noise=1):
    """Camera events (config 2) and white noise of several sigmas (config 1's
    generator), 16-bit."""
    parts = [datagen.cherenkov_events(n_events, seed=seed).reshape(-1)]
    rng = np.random.default_rng(seed)
    for k in range(noise):
        x = datagen.white_noise(4096 * 40, float(rng.uniform(100, 3000)), float(rng.uniform(1, 60)),
                                seed=seed * 7 + k)
        spikes = rng.choice(x.size, x.size // 400, replace=False)
        x[spikes] = rng.integers(0, 65535, spikes.size)
        parts.append(x)
    x = np.concatenate(parts)
    return x[: x.size // 4096 * 4096]


def test_features_match_oracle():
    for x in (mixed_data(1), datagen.batched_stream(datagen.batched_stream_specs(1, 100000, 100001, seed=3)[0])):
        d = x.dtype.itemsize * 8
        got = ch.segment_features(to_dev(x)).cpu().numpy()
        want = mlp.features(x, d)
        np.testing.assert_allclose(got, want, rtol=2e-6, atol=1e-7)
        # an array that does not start 16-byte aligned takes the scalar loads
        shifted = to_dev(np.concatenate([x[:1], x]))[1:]
        assert shifted.data_ptr() % 16
        np.testing.assert_array_equal(ch.segment_features(shifted).cpu().numpy(), got)


def test_forward_and_gradient_match_oracle():
    """BF16 weights, FP32 accumulation against fp64 on the same BF16-rounded
    weights: logits within 1e-4, gradient within 1e-4 relative (plus 1e-7)."""
    c = ch.Chooser(dev(), seed=3)
    rng = np.random.default_rng(0)
    X = rng.uniform(0, 1, (300, 24)).astype(np.float32)
    y = rng.integers(0, 12, 300).astype(np.uint8)
    Xd = torch.from_numpy(X).to(dev())
    yd = torch.from_numpy(y).to(dev())
    P = mlp.unflatten(c.weights_f64())
    np.testing.assert_allclose(c.logits(Xd).cpu().numpy(), mlp.forward(P, X.astype(np.float64)),
                               rtol=1e-4, atol=1e-4)
    loss, g = c.loss_grad(Xd, yd)
    want_loss, G = mlp.loss_grad(P, X.astype(np.float64), y.astype(np.int64))
    assert abs(loss - want_loss) < 1e-4 * abs(want_loss) + 1e-6
    np.testing.assert_allclose(g.cpu().numpy(), mlp.flatten(G), rtol=1e-4, atol=1e-7)


def test_gpu_exhaustive_sizes_match_oracle():
    x = mixed_data(2, n_events=1, noise=1)[: 4096 * 24]
    sizes = ch.exhaustive_sizes(to_dev(x)).cpu().numpy()
    lab, want = mlp.labels(x, 1)
    assert np.array_equal(sizes, want)
    assert np.array_equal(np.argmin(sizes, axis=1), lab)


@pytest.mark.parametrize("variant", [native.BASIC, native.ADVANCED])
def test_gpu_labels_equal_the_oracle_labels_on_a_thousand_segments(variant):
    """The training labels the benchmark takes from the GPU's exhaustive
    search are the CPU oracle's labels: every size of every option, over
    about 1,300 segments of camera events and white noise of several sigmas
    with spikes (the chooser's training mix), for both variants."""
    x = mixed_data(5, n_events=16, noise=12)
    assert x.size // 4096 >= 1000
    sizes = ch.exhaustive_sizes(to_dev(x), variant).cpu().numpy()
    lab, want = mlp.labels(x, variant)
    assert np.array_equal(sizes, want)
    assert np.array_equal(np.argmin(sizes, axis=1).astype(np.uint8), lab)


def test_trained_chooser_beats_plain_heuristic():
    """Train on oracle labels of configs 1-2 data, evaluate on fresh seeds:
    the learned per-segment options give a smaller total than the plain
    heuristic (one fixed option) and stay close to the exhaustive optimum."""
    xtr = np.concatenate([mixed_data(s, n_events=2, noise=2) for s in (10, 11, 12)])
    ytr, _ = mlp.labels(xtr, 1)
    xte = np.concatenate([mixed_data(s, n_events=2, noise=2) for s in (20, 21)])
    _, ste = mlp.labels(xte, 1)
    c = ch.Chooser(dev(), seed=0)
    Xtr = ch.segment_features(to_dev(xtr))
    hist = c.train(Xtr, torch.from_numpy(ytr).to(dev()), epochs=60, batch=256, lr=3e-3)
    assert hist[-1] < hist[0]
    pred = c.predict(ch.segment_features(to_dev(xte))).cpu().numpy()
    learned = ste[np.arange(len(pred)), pred].sum()
    plain = ste[:, ch.PLAIN_OPTION].sum()
    best = ste.min(axis=1).sum()
    assert learned < plain, (learned, plain, best)
    assert learned <= best * 1.02, (learned, best)
    # the learned options through the GPU batch path give exactly those sizes
    b = ch.compress_segments(to_dev(xte), pred)
    assert b.device_status() == 0
    assert b.total_bytes() == learned
