"""Batches: many independent streams of mixed dtype, word size, variant and
block length in one persistent launch (and replayed from a CUDA graph).
Every item's output must be byte-identical to the oracle's stream of that
item alone; the autotuner's choice must be the smallest candidate."""
import numpy as np
import pytest

import oracle
from paper_1805_01844_gb300 import datagen, native

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1805_01844_gb300 as pc  # noqa: E402
from paper_1805_01844_gb300.batch import Batch, autotune, autotune_threads  # noqa: E402


def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch.device("cuda:0")


def to_dev(x):
    view = x.view(np.int16) if x.dtype == np.uint16 else x.view(np.int32)
    return torch.from_numpy(view.copy()).to(dev())


def small_specs(n_streams, seed):
    return datagen.batched_stream_specs(n_streams, min_bytes=64, max_bytes=2 << 20, seed=seed)


@pytest.mark.parametrize("cta_threads", [256, 128])
def test_batch_matches_oracle_per_item(cta_threads):
    rng = np.random.default_rng(3)
    specs = small_specs(40, seed=1)
    hosts, tensors, params = [], [], []
    for i, sp in enumerate(specs):
        x = datagen.batched_stream(sp)
        d = x.dtype.itemsize * 8
        p = native.params(int(rng.integers(0, 2)), d, int(rng.choice([32, 64])),
                          int(rng.choice([1, 77, 128, 256, 1000, 1024, 4096])))
        hosts.append(x)
        tensors.append(to_dev(x))
        params.append(p)
    # an empty item and a one-sample item
    for n in (0, 1):
        x = np.full(n, 7, np.uint16)
        hosts.append(x)
        tensors.append(to_dev(x))
        params.append(native.params(1, 16, 64, 1024))
    b = Batch(tensors, params, cta_threads=cta_threads)
    assert b.info.cta_threads == cta_threads
    b.compress()
    assert b.device_status() == 0
    got = b.streams()
    for x, p, s in zip(hosts, params, got):
        want = oracle.compress(x, p.variant, p.word_bits, p.block_len)
        assert s == want, p


def test_batch_graph_replay_is_identical():
    specs = small_specs(16, seed=2)
    hosts = [datagen.batched_stream(sp) for sp in specs]
    tensors = [to_dev(x) for x in hosts]
    params = [native.params(i % 2, x.dtype.itemsize * 8, 64, 1024) for i, x in enumerate(hosts)]
    b = Batch(tensors, params)
    g = b.capture()
    for o in b.outs:
        o.zero_()
    b.nbytes.zero_()
    g.replay()
    g.replay()
    torch.cuda.synchronize()
    assert b.device_status() == 0
    for x, p, s in zip(hosts, params, b.streams()):
        assert s == oracle.compress(x, p.variant, p.word_bits, p.block_len)


def test_autotune_picks_the_smallest_candidate():
    sp = datagen.batched_stream_specs(1, min_bytes=200000, max_bytes=200001, seed=5)[0]
    x = datagen.batched_stream(sp)
    p = autotune(to_dev(x), sample=1 << 16)
    head = x[: 1 << 16]
    sizes = {(L, w): len(oracle.compress(head, 0, w, L)) for L in (128, 256, 512, 1024, 2048, 4096)
             for w in (32, 64)}
    assert len(oracle.compress(head, 0, p.word_bits, p.block_len)) == min(sizes.values())


def test_autotune_threads_returns_a_candidate():
    specs = small_specs(8, seed=4)
    tensors = [to_dev(datagen.batched_stream(sp)) for sp in specs]
    params = [native.params(0, t.element_size() * 8, 64, 256) for t in tensors]
    nt, times = autotune_threads(tensors, params, reps=2)
    assert nt in (128, 256) and set(times) == {128, 256} and times[nt] == min(times.values())



def test_time_aware_autotune_stays_within_the_size_rule():
    """With a time slack the choice is still a candidate of the oracle's
    size table, and with an unbounded slack it is the smallest one."""
    sp = datagen.batched_stream_specs(1, min_bytes=400000, max_bytes=400001, seed=6)[0]
    x = datagen.batched_stream(sp)
    head = x[: 1 << 16]
    sizes = {(L, w): len(oracle.compress(head, 0, w, L)) for L in (128, 256, 512, 1024, 2048, 4096)
             for w in (32, 64)}
    p = autotune(to_dev(x), sample=1 << 16, time_slack=0.5, time_sample=1 << 17)
    assert (p.block_len, p.word_bits) in sizes
    q = autotune(to_dev(x), sample=1 << 16, time_slack=1e9, time_sample=1 << 17)
    assert sizes[(q.block_len, q.word_bits)] == min(sizes.values())


def test_short_block_items_match_oracle():
    """Basic items of short blocks (16- and 32-bit) take look-back tiles of
    whole short blocks in 256-thread launches: every item equals the oracle's
    stream, from one sample to several tiles, ragged last blocks included."""
    rng = np.random.default_rng(9)
    hosts, tensors, params = [], [], []
    for i, (L, w) in enumerate([(8, 64), (32, 32), (64, 64), (128, 32), (128, 64), (256, 64), (256, 32), (16, 64)]):
        for n in (1, L * 128 - 3, L * 300 + 5):
            x = np.clip(rng.normal(500, 20, n), 0, 65535).astype(np.uint16)
            if n > 10:
                x[rng.integers(0, n, max(1, n // 500))] = 65535
                x[: min(n, 3 * L)] = 9
            hosts.append(x)
            tensors.append(to_dev(x))
            params.append(native.params(0, 16, w, L))
    for L, w in [(4, 64), (32, 32), (128, 64)]:  # 32-bit samples
        x = np.clip(rng.normal(2e6, 300, L * 200 + 3), 0, 2 ** 32 - 1).astype(np.uint32)
        x[5] = 2 ** 32 - 1
        hosts.append(x)
        tensors.append(to_dev(x))
        params.append(native.params(0, 32, w, L))
    b = Batch(tensors, params, cta_threads=256)
    b.compress()
    assert b.device_status() == 0
    for x, p, s in zip(hosts, params, b.streams()):
        assert s == oracle.compress(x, 0, p.word_bits, p.block_len), p
