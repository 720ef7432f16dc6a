"""Format version 2, host side (no GPU): the library's worst-case size equals
the oracle's for every segment-length class, and the entry points reject bad
arguments before touching the device."""
import ctypes

import pytest

import oracle
from paper_1805_01844_gb300 import native


@pytest.mark.parametrize("variant", [0, 1])
@pytest.mark.parametrize("d", [16, 32])
def test_bound_v2_equals_oracle(variant, d):
    for seg_len, n in [(4096, 0), (4096, 1), (4096, 4096), (4096, 10 ** 6 + 3), (700, 12345), (1, 5), (10000, 99999)]:
        assert native.bound_v2(variant, d, seg_len, n) == oracle.bound_v2(variant, d, seg_len, n), (seg_len, n)


def test_v2_argument_checks():
    L = native.load()
    out = ctypes.c_uint64(0)
    assert L.pc_bound_v2(2, 16, 4096, 10, ctypes.byref(out)) == native.PC_ERR_INVALID_ARG
    assert L.pc_bound_v2(0, 8, 4096, 10, ctypes.byref(out)) == native.PC_ERR_INVALID_ARG
    assert L.pc_bound_v2(0, 16, 0, 10, ctypes.byref(out)) == native.PC_ERR_INVALID_ARG
    # segment count must match the samples; NULL output
    assert L.pc_assemble_v2(None, 4096, 2, 4096, 4096, 16, 0, None, 0, None, None, 0, None) == \
        native.PC_ERR_INVALID_ARG
    # advanced 32-bit decoding is not supported on the GPU
    assert L.pc_decompress_v2(None, 64, 1, 32, 4096, None, 0, None, None, 0, None) == native.PC_ERR_UNSUPPORTED
    assert L.pc_decompress_v2(None, 64, 1, 16, 4096, None, 0, None, None, 0, None) == native.PC_ERR_INVALID_ARG
    assert native.decompress_v2_workspace_size(1, 16, 4096, 10 ** 6) > native.decompress_v2_workspace_size(
        0, 16, 4096, 10 ** 6)
