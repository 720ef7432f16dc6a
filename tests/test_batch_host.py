"""Host side of the batch plan (no GPU): in 256-thread launches, basic items
of short blocks are cut into look-back tiles of whole short blocks (up to
128 blocks, at most 32 KB of samples), other items into the tiles of the
single-stream compressor; 128-thread launches never use the short tiles."""
import pytest

from paper_1805_01844_gb300 import native


def item(n, d, w, L, variant=0):
    fake = 1 << 20  # 16-byte aligned; describe reads no device memory
    p = native.params(variant, d, w, L)
    return native.PcBatchItem(fake, n, p, fake, native.bound(p, n), fake)


def short_tile_blocks(d, L):
    return min(128, 32768 // (L * d // 8))


@pytest.mark.parametrize("d,w,L", [(16, 64, 8), (16, 32, 128), (16, 64, 256), (32, 64, 128), (32, 32, 4)])
def test_short_items_take_whole_short_block_tiles(d, w, L):
    n = 1000 * L + 3
    _, info = native.batch_describe([item(n, d, w, L)], cta_threads=256)
    assert info.total_tiles == -(-(-(-n // L)) // short_tile_blocks(d, L))
    _, info128 = native.batch_describe([item(n, d, w, L)], cta_threads=128)
    assert info128.total_tiles > info.total_tiles  # 32-block tiles or fewer


@pytest.mark.parametrize("d,w,L,variant", [(16, 32, 256, 0), (32, 64, 256, 0), (16, 64, 128, 1), (16, 64, 154, 0),
                                           (16, 64, 1024, 0)])
def test_other_items_keep_the_regular_tiles(d, w, L, variant):
    """16-bit L = 256 with 32-bit words, 32-bit L = 256 (64 vectors per
    block), the advanced variant, block lengths that are not a power of two
    of 16-byte vectors, and long blocks keep tiles of at most 32 blocks."""
    n = 2000 * L
    _, info = native.batch_describe([item(n, d, w, L, variant)], cta_threads=256)
    assert info.total_tiles >= -(-2000 // 32)
