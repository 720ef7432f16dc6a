"""Host-side limits of pc_compress_noalloc (no GPU needed): a stream whose
look-back workspace does not fit the library's static scratch is refused
with PC_ERR_UNSUPPORTED before anything touches the device, including a
stream just one block over the limit.  The pointers passed are never
dereferenced, because the size check comes first."""
from paper_1805_01844_gb300 import native

FAKE = 1 << 40  # aligned, never dereferenced


def largest_accepted(p):
    """Largest sample count whose workspace (without the advanced variant's
    series table, which the static scratch never holds) fits the scratch."""
    basic = native.params(native.BASIC, p.dtype_bits, p.word_bits, p.block_len)
    lo, hi = 0, 1 << 40
    while hi - lo > 1:
        m = (lo + hi) // 2
        if native.workspace_size(basic, m) <= native.NOALLOC_SCRATCH_BYTES:
            lo = m
        else:
            hi = m
    return lo


def test_noalloc_rejects_streams_beyond_its_scratch():
    p = native.params(native.BASIC, 16, 64, 1)  # one block per sample: many tiles
    too_many = 40_000_000
    assert native.workspace_size(p, too_many) > native.NOALLOC_SCRATCH_BYTES
    st = native.compress_noalloc_raw(FAKE, too_many, p, FAKE, native.bound(p, too_many), FAKE, None)
    assert st == native.PC_ERR_UNSUPPORTED


def test_noalloc_limit_is_about_2e9_uint16_samples_at_block_len_1024():
    p = native.params(native.BASIC, 16, 64, 1024)
    n = largest_accepted(p)
    assert 2.0e9 < n < 2.2e9
    over = n + 1024 * 64  # a few tiles more
    st = native.compress_noalloc_raw(FAKE, over, p, FAKE, native.bound(p, over), FAKE, None)
    assert st == native.PC_ERR_UNSUPPORTED


def test_noalloc_advanced_limit_ignores_the_series_table():
    """The advanced variant's pc_workspace_size counts its ~17 MB series
    table, larger than the whole scratch; the no-alloc call checks the
    look-back part only, so it refuses advanced streams past that limit and
    not before."""
    pa = native.params(native.ADVANCED, 16, 64, 1024)
    assert native.workspace_size(pa, 1024) > native.NOALLOC_SCRATCH_BYTES
    n = largest_accepted(pa)
    over = n + 1024 * 64
    st = native.compress_noalloc_raw(FAKE, over, pa, FAKE, native.bound(pa, over), FAKE, None)
    assert st == native.PC_ERR_UNSUPPORTED
