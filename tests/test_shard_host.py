"""Sharded streams on the host (no GPU): the block-aligned partition of
pc_shard_range, and the placement of pc_stitch_layout, which must put the
oracle's streams of the shards together into exactly the oracle's stream of
all samples (blocks are independent, Sec. 3.3); plus the one exchange, every
rank's stream size, all-gathered over two gloo CPU ranks."""
import os
import socket

import numpy as np
import pytest

import oracle
from paper_1805_01844_gb300 import datagen, native


def stitch_on_host(p, n, pieces):
    """Whole stream from the shards' streams (bytes) by the product's layout."""
    sizes = [len(b) for b in pieces]
    out = None
    for k, b in enumerate(pieces):
        r = native.stitch_layout(p, n, len(pieces), k, sizes)
        if out is None:
            out = bytearray(r["total_bytes"])
        out[r["table_dst"]:r["table_dst"] + r["table_bytes"]] = b[r["table_src"]:r["table_src"] + r["table_bytes"]]
        out[r["payload_dst"]:r["payload_dst"] + r["payload_bytes"]] = \
            b[r["payload_src"]:r["payload_src"] + r["payload_bytes"]]
    out[0:64] = pieces[0][0:64]  # header fields below are re-derived and checked
    return out, r


@pytest.mark.parametrize("n,L,K", [(10 * 1024 + 77, 1024, 3), (4 * 256, 256, 7), (37, 8, 2), (0, 64, 3),
                                   (5 * 100 + 1, 100, 5)])
def test_shard_range_partitions_whole_blocks(n, L, K):
    p = native.params(0, 16, 64, L)
    got = [native.shard_range(p, n, K, k) for k in range(K)]
    nb = -(-n // L)
    pos = 0
    for k, (f, c) in enumerate(got):
        assert f == pos and f % L == 0
        assert c == 0 or (f + c == n or (f + c) % L == 0)
        blocks = -(-c // L)
        assert blocks in (nb // K, nb // K + 1)
        assert (blocks == nb // K + 1) == (k < nb % K)
        pos += c
    assert pos == n


@pytest.mark.parametrize("variant,d,w,L,n,K", [(0, 16, 64, 1024, 23 * 1024 + 5, 3), (1, 16, 32, 256, 40 * 256, 7),
                                               (0, 32, 32, 100, 9 * 100 + 37, 4), (1, 32, 64, 64, 3 * 64 + 1, 6)])
def test_stitch_layout_joins_oracle_shards_into_the_oracle_stream(variant, d, w, L, n, K):
    dt = np.uint16 if d == 16 else np.uint32
    x = datagen.white_noise(n, 300.0 if d == 16 else 90000.0, 7.0, seed=n, dtype=dt)
    x[::97] = 5000 if d == 16 else 4_000_000
    p = native.params(variant, d, w, L)
    pieces = []
    for k in range(K):
        f, c = native.shard_range(p, n, K, k)
        pieces.append(oracle.compress(x[f:f + c], variant, w, L))
    whole, last = stitch_on_host(p, n, pieces)
    want = oracle.compress(x, variant, w, L)
    assert last["total_bytes"] == len(want)
    h = oracle.header(want)
    whole[16:24] = int(n).to_bytes(8, "little")
    whole[24:32] = int(h["n_blocks"]).to_bytes(8, "little")
    whole[32:40] = int((len(want) - last["payload_start"]) // (w // 8)).to_bytes(8, "little")
    assert bytes(whole) == want


def test_stitch_layout_rejects_a_size_that_is_not_a_stream_of_its_shard():
    p = native.params(0, 16, 64, 1024)
    n, K = 10 * 1024, 2
    sizes = [64 + 32 + 8 * 100, 64 + 32 + 8 * 90 + 3]  # second: not whole words
    with pytest.raises(native.PcError):
        native.stitch_layout(p, n, K, 0, sizes)


def free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world, port, out_dir):
    import sys

    import torch
    import torch.distributed as dist

    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import oracle as orc
    from paper_1805_01844_gb300 import datagen as dg
    from paper_1805_01844_gb300 import native as nat
    from paper_1805_01844_gb300 import shard

    dist.init_process_group("gloo", init_method="tcp://127.0.0.1:%d" % port, rank=rank, world_size=world)
    n, L = 13 * 1024 + 300, 1024
    x = dg.white_noise(n, 300.0, 5.0, seed=21)
    p = nat.params(0, 16, 64, L)
    f, c = nat.shard_range(p, n, world, rank)
    mine = orc.compress(x[f:f + c], 0, 64, L)  # this rank's shard stream (the GPU's job on a GPU machine)
    sizes = shard.exchange_sizes(torch.tensor([len(mine)], dtype=torch.int64)).tolist()
    r = nat.stitch_layout(p, n, world, rank, sizes)
    buf = torch.zeros(r["total_bytes"], dtype=torch.int64)  # one byte per element: disjoint pieces sum exactly
    b = np.frombuffer(mine, dtype=np.uint8).astype(np.int64)
    buf[r["table_dst"]:r["table_dst"] + r["table_bytes"]] = torch.from_numpy(
        b[r["table_src"]:r["table_src"] + r["table_bytes"]])
    buf[r["payload_dst"]:r["payload_dst"] + r["payload_bytes"]] = torch.from_numpy(
        b[r["payload_src"]:r["payload_src"] + r["payload_bytes"]])
    dist.all_reduce(buf)
    if rank == 0:
        whole = bytearray(buf.to(torch.uint8).numpy().tobytes())
        want = orc.compress(x, 0, 64, L)
        # the header is pc_stitch's job on the device (shard 0); table, padding and payload come from the ranks
        ok = len(whole) == len(want) and whole[64:] == want[64:]
        with open(os.path.join(out_dir, "ok"), "w") as fh:
            fh.write("%d %d %d %s" % (ok, len(whole), len(want), sizes))
    dist.destroy_process_group()


def test_size_exchange_on_two_gloo_ranks(tmp_path):
    import torch.multiprocessing as mp

    port = free_port()
    mp.start_processes(_rank, args=(2, port, str(tmp_path)), nprocs=2, join=True, start_method="spawn")
    ok, got, want, sizes = open(os.path.join(str(tmp_path), "ok")).read().split(" ", 3)
    assert ok == "1", (got, want, sizes)
