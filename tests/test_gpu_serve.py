"""The serving loop: Poisson arrivals of events from four camera geometries,
continuous batching on several CUDA streams under a device-memory budget.
Every event's compressed result must be byte-identical whether it was
compressed alone or in the mix, with the learned chooser off and on, and it
must decompress to the event."""
import numpy as np
import pytest

import oracle
from paper_1805_01844_gb300 import native

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1805_01844_gb300 import serve  # noqa: E402
from paper_1805_01844_gb300.chooser import Chooser  # noqa: E402


def events(n, seed):
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n):
        gi = int(rng.integers(0, len(serve.GEOMETRIES)))
        out.append((gi, serve.event_host(serve.GEOMETRIES[gi], seed * 100000 + i)))
    return out


@pytest.mark.parametrize("use_chooser,v2", [(False, False), (True, False), (True, True)])
def test_results_identical_alone_and_in_the_mix(use_chooser, v2):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    dev = torch.device("cuda:0")
    ch = Chooser(dev, seed=1) if use_chooser else None
    srv = serve.Server(dev, budget=1 << 30, n_streams=3, chooser=ch, slot_cap=16, v2=v2)
    ev = events(600, seed=3 + use_chooser)
    keep = list(range(0, 600, 37))
    m = srv.run(ev, rate=20000.0, seed=1, keep=keep)
    assert m["events"] == 600 and m["ratio"] > 1.5
    assert m["p99_ms"] >= m["p50_ms"] > 0
    assert set(m["kept"]) == set(keep)
    for e in keep:
        gi, x = ev[e]
        xd = torch.from_numpy(x.view(np.int16).copy()).to(dev)
        alone = serve.compress_alone(xd, chooser=ch, v2=v2)
        assert m["kept"][e] == alone, e
        # every piece is a stream of its segment (or of the whole event; v2:
        # the event's version-2 stream)
        dec = oracle.decompress_v2 if v2 else oracle.decompress
        y = np.concatenate([dec(s) for s in alone])
        assert np.array_equal(y, x)


@pytest.mark.parametrize("use_chooser,v2", [(False, False), (True, False), (True, True)])
def test_device_totals_match_streams(use_chooser, v2):
    """The per-camera totals kept in device memory add up every event's
    streams exactly once."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    dev = torch.device("cuda:0")
    ch = Chooser(dev, seed=2) if use_chooser else None
    srv = serve.Server(dev, budget=1 << 30, n_streams=2, chooser=ch, slot_cap=8, v2=v2)
    ev = events(120, seed=7)
    m = srv.run(ev, rate=50000.0, seed=3, keep=range(120))
    assert m["stream_bytes"] == sum(len(s) for e in range(120) for s in m["kept"][e])
    per = srv.totals.cpu().numpy()
    for gi in range(len(serve.GEOMETRIES)):
        mine = [e for e in range(120) if ev[e][0] == gi]
        assert per[gi, 0] == len(mine)
        assert per[gi, 1] == sum(len(s) for e in mine for s in m["kept"][e])
