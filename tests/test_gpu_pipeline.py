"""Pipelined round trips of pinned host buffers (pipeline.RoundTrip): with
consecutive calls in flight, every call's host stream equals the oracle's
stream of its samples byte for byte and its host samples equal the input."""
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import numpy as np  # noqa: E402

import oracle  # noqa: E402
from paper_1805_01844_gb300 import datagen  # noqa: E402
from paper_1805_01844_gb300.pipeline import RoundTrip  # noqa: E402


@pytest.mark.parametrize("variant,w,L", [(0, 64, 1024), (1, 32, 256)])
def test_pipelined_round_trips_equal_the_oracle(variant, w, L):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    dev = torch.device("cuda:0")
    n = 300 * L + 17
    rt = RoundTrip(variant, 16, w, L, n, device=dev)
    inputs = []
    for k in range(5):
        x = datagen.white_noise(n, 300.0 + 50 * k, 4.0 + k, seed=k)
        x[:: 997] = 9000
        h = torch.from_numpy(x.view(np.int16).copy()).pin_memory()
        inputs.append((x, h))
        rt.submit(h)
    rt.drain()
    done = rt.completed()
    assert len(done) == 5
    # the host buffers of the last two calls (one per slot) hold their results
    for k in (3, 4):
        b, nbytes = done[k]
        x, h = inputs[k]
        assert torch.equal(rt.host_out[b], h)
        assert rt.host_stream[b][:nbytes].numpy().tobytes() == oracle.compress(x, variant, w, L)
