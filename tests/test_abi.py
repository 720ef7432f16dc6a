"""Host-side checks of the C ABI (no GPU needed): the library loads, exports
every entry point include/pc.h declares, and its host-only calls agree with
the oracle and reject bad arguments before touching the device."""
import ctypes
import os
import re

import numpy as np
import pytest

import oracle
from paper_1805_01844_gb300 import build as pcbuild
from paper_1805_01844_gb300 import datagen, native

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    pcbuild.build()
    return native.load()


def declared_entry_points():
    src = open(os.path.join(ROOT, "include", "pc.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(pc_[a-z0-9_]+)\s*\(", src)))


def test_exports_every_declared_symbol(lib):
    names = declared_entry_points()
    assert len(names) >= 8
    for name in names:
        assert hasattr(lib, name), name
    assert set(names) == set(native.EXPORTS)


@pytest.mark.parametrize("variant", [0, 1])
@pytest.mark.parametrize("d", [16, 32])
@pytest.mark.parametrize("w", [32, 64])
def test_bound_matches_oracle(lib, variant, d, w):
    for L in (1, 7, 154, 1024, 4096, 8192):
        for n in (0, 1, L - 1, L, L + 1, 10 * L + 3, 123457):
            if n < 0:
                continue
            p = native.params(variant, d, w, L)
            assert native.bound(p, n) == oracle.bound(variant, d, w, L, n), (L, n)


def test_parse_header_of_oracle_streams(lib):
    x = datagen.white_noise(5000, seed=1)
    for variant in (0, 1):
        for w in (32, 64):
            s = oracle.compress(x, variant, w, 333)
            p, n = native.parse_header(s)
            assert (p.variant, p.dtype_bits, p.word_bits, p.block_len, n) == (variant, 16, w, 333, 5000)
    bad = bytearray(oracle.compress(x, 0, 64, 100))
    bad[3] = ord("X")
    with pytest.raises(native.PcError) as e:
        native.parse_header(bytes(bad))
    assert e.value.code == native.PC_ERR_CORRUPT


def test_argument_checks_happen_on_the_host(lib):
    """Bad parameters, NULL or misaligned pointers and a short output buffer
    are rejected before any CUDA call (so this runs without a GPU)."""
    good = native.params(0, 16, 64, 1024)
    fake = 1 << 40  # a 16-byte aligned address that is never dereferenced
    ws = native.workspace_size(good, 4096)
    cap = native.bound(good, 4096)
    cases = [
        (native.params(2, 16, 64, 1024), fake, fake, cap, fake, native.PC_ERR_INVALID_ARG),
        (native.params(0, 8, 64, 1024), fake, fake, cap, fake, native.PC_ERR_INVALID_ARG),
        (native.params(0, 16, 48, 1024), fake, fake, cap, fake, native.PC_ERR_INVALID_ARG),
        (native.params(0, 16, 64, 0), fake, fake, cap, fake, native.PC_ERR_INVALID_ARG),
        (native.params(0, 16, 64, 8193), fake, fake, cap, fake, native.PC_ERR_UNSUPPORTED),
        (good, fake + 2, fake, cap, fake, native.PC_ERR_INVALID_ARG),
        (good, fake, fake + 8, cap, fake, native.PC_ERR_INVALID_ARG),
        (good, fake, fake, cap, fake + 4, native.PC_ERR_INVALID_ARG),
        (good, fake, fake, cap - 1, fake, native.PC_ERR_CAPACITY),
        (good, None, fake, cap, fake, native.PC_ERR_INVALID_ARG),
    ]
    for p, d_in, d_out, c, d_ws, want in cases:
        st = native.compress_raw(d_in, 4096, p, d_out, c, fake, d_ws, ws, None)
        assert st == want, (p, want, st)
    assert native.compress_raw(fake, 4096, good, fake, cap, fake, fake, ws - 1, None) == native.PC_ERR_INVALID_ARG
    # decompress: a stream shorter than its header is corrupt without looking
    assert native.decompress_raw(fake, 63, good, fake, 10, fake, fake, ws, None) == native.PC_ERR_CORRUPT
    assert native.decompress_raw(fake, 640, good, fake + 1, 10, fake, fake, ws, None) == native.PC_ERR_INVALID_ARG


def test_strerror(lib):
    for code in range(7):
        assert native.strerror(code)


def test_every_tile_configuration_fits_shared_memory(tmp_path):
    """Host-compiled check of the kernels' tile layout (pc_common.cuh) for
    every variant, sample width, word width and block length 1..8192: the
    dynamic shared memory stays within the 227 KB a CTA can have and tiles
    hold 1..32 blocks, for both CTA sizes of the compression kernel; the warp
    decoder's tiles (32 blocks, or 16) keep the most resident warps."""
    import shutil
    import subprocess

    if shutil.which("g++") is None:
        pytest.skip("no host C++ compiler")
    src = tmp_path / "tc.cpp"
    src.write_text(r'''
#include <cstdio>
#include "pc_common.cuh"
using namespace pcx;
int main() {
  for (unsigned k = 0; k < 2; ++k) for (unsigned v = 0; v < 2; ++v)
  for (unsigned d = 16; d <= 32; d += 16) for (unsigned w = 32; w <= 64; w += 32)
  for (unsigned L = 1; L <= 8192; ++L) for (int orb = 0; orb < 2; ++orb) for (unsigned nt = 128; nt <= 256; nt *= 2) {
    TileCfg c = tile_cfg(k, v, d, w, L, orb != 0, nt);
    if (c.smem > 227u * 1024u || c.tb < 1 || c.tb > 32) { printf("bad %u %u %u %u %u\n", k, v, d, w, L); return 1; }
    if (k == 1) {
      unsigned nw = decw_warps(v, d, w, L), cap = dec_tile_cap(v, d, w, L);
      if (nw < 1 || nw > 4 || nw * decw_warp_bytes(v, d, w, L) > 227u * 1024u) { printf("decw %u %u %u %u\n", v, d, w, L); return 1; }
      // warp tiles of 32 blocks, or 16 where the records of 32 would cost resident warps
      if ((cap != 16 && cap != 32) || decw_warps_per_sm(v, d, w, L, cap) < decw_warps_per_sm(v, d, w, L, 48 - cap)) {
        printf("cap %u %u %u %u\n", v, d, w, L); return 1;
      }
    }
  }
  printf("ok\n");
  return 0;
}
''')
    exe = tmp_path / "tc"
    subprocess.check_call(["g++", "-std=c++17", "-O1", "-I" + os.path.join(ROOT, "include"),
                           "-I" + os.path.join(ROOT, "paper_1805_01844_gb300", "csrc"), str(src), "-o", str(exe)])
    assert subprocess.run([str(exe)], capture_output=True, text=True).stdout.strip() == "ok"


@pytest.mark.parametrize("d", [16, 32])
@pytest.mark.parametrize("variant", [0, 1])
def test_segment_slots_hold_every_option(lib, d, variant):
    """The segment slot is the largest stream of a full segment over the 12
    options (the oracle's bound), rounded up to 16 bytes."""
    want = max(oracle.bound(variant, d, (32, 64)[o % 2], 128 << (o // 2), 4096) for o in range(12))
    assert native.segment_stride(d, variant) == (want + 15) // 16 * 16


def test_segments_describe_checks_on_the_host(lib):
    fake = 1 << 40
    stride = native.segment_stride(16, 1)

    def src(n, d_in=fake, d_out=fake, cap=None, nb=fake, tot=None):
        k = -(-n // 4096)
        return native.PcSource(d_in, n, d_out, k * stride if cap is None else cap, nb, tot)

    def code(sources, d=16, variant=1):
        arr = (native.PcSource * len(sources))(*sources)
        info = native.PcSegmentsInfo()
        return lib.pc_segments_describe(arr, len(sources), d, variant, ctypes.byref(info)), info

    st, info = code([src(10000), src(0, None, None, 0, None), src(4096, tot=fake + 16)])
    assert st == native.PC_OK
    assert (info.n_segments, info.seg_stride, info.has_totals, info.n_sources) == (4, stride, 1, 3)
    assert info.plan_bytes == 3 * 48 and info.workspace_bytes > 4 * 64
    assert code([src(10000)], d=8)[0] == native.PC_ERR_INVALID_ARG
    assert code([src(10000)], variant=2)[0] == native.PC_ERR_INVALID_ARG
    assert code([src(10000, d_in=fake + 2)])[0] == native.PC_ERR_INVALID_ARG
    assert code([src(10000, d_out=fake + 8)])[0] == native.PC_ERR_INVALID_ARG
    assert code([src(10000, nb=fake + 4)])[0] == native.PC_ERR_INVALID_ARG
    assert code([src(10000, tot=fake + 4)])[0] == native.PC_ERR_INVALID_ARG
    assert code([src(10000, d_in=None)])[0] == native.PC_ERR_INVALID_ARG
    assert code([src(10000, cap=3 * stride - 1)])[0] == native.PC_ERR_CAPACITY
    assert code([src(1 << 43)])[0] == native.PC_ERR_UNSUPPORTED  # 2^31 segments
    arr = (native.PcSource * 1)(src(10))
    assert lib.pc_segments_describe(arr, 0, 16, 1, ctypes.byref(native.PcSegmentsInfo())) == \
        native.PC_ERR_INVALID_ARG
    # no segments at all: nothing to do, and compressing is a no-op
    st, info = code([src(0, None, None, 0, None)])
    assert st == native.PC_OK and info.n_segments == 0
    assert native.compress_segments(info, None, None, None, 0, None) == native.PC_OK


def test_magic_division_is_exact(tmp_path):
    """Host-compiled check of the 32-bit magic reciprocals the kernels divide
    by (pc_common.cuh): for every divisor 2..2^17 and a spread of larger ones
    up to 2^32, the quotient of dividends at the edges (0, 1, d - 1, d, d + 1,
    the multiples of d next to 2^32, 2^32 - 1) and pseudo-random ones equals
    plain integer division."""
    import shutil
    import subprocess

    if shutil.which("g++") is None:
        pytest.skip("no host C++ compiler")
    src = tmp_path / "md.cpp"
    src.write_text(r'''
#include <cstdio>
#include <cstdint>
#include "pc_common.cuh"
using namespace pcx;
static uint64_t rs = 88172645463325252ull;
static uint32_t rnd() { rs ^= rs << 13; rs ^= rs >> 7; rs ^= rs << 17; return (uint32_t)rs; }
static int check(uint64_t d) {
  const Magic32 mg = magic32(d);
  uint64_t xs[16];
  int k = 0;
  const uint64_t top = 0xFFFFFFFFull, last = top / d * d;
  xs[k++] = 0; xs[k++] = 1; xs[k++] = d - 1; xs[k++] = d <= top ? d : 0; xs[k++] = d + 1 <= top ? d + 1 : 0;
  xs[k++] = top; xs[k++] = top - 1; xs[k++] = last; xs[k++] = last ? last - 1 : 0;
  for (int i = 0; i < 7; ++i) xs[k++] = rnd();
  for (int i = 0; i < k; ++i) {
    const uint32_t x = (uint32_t)xs[i];
    if (magic_div(x, mg) != (uint32_t)(x / d)) { printf("bad d=%llu x=%u\n", (unsigned long long)d, x); return 1; }
  }
  return 0;
}
int main() {
  for (uint64_t d = 2; d <= (1u << 17); ++d) if (check(d)) return 1;
  for (int i = 0; i < 200000; ++i) { uint64_t d = ((uint64_t)rnd() | 2u); if (check(d)) return 1; }
  for (int e = 17; e <= 32; ++e) {
    const uint64_t p = 1ull << e;
    if (check(p) || check(p - 1) || (e < 32 && check(p + 1))) return 1;
  }
  printf("ok\n");
  return 0;
}
''')
    exe = tmp_path / "md"
    subprocess.check_call(["g++", "-std=c++17", "-O2", "-I" + os.path.join(ROOT, "include"),
                           "-I" + os.path.join(ROOT, "paper_1805_01844_gb300", "csrc"), str(src), "-o", str(exe)])
    assert subprocess.run([str(exe)], capture_output=True, text=True).stdout.strip() == "ok"


def test_digits_per_word_and_geometric_sum(tmp_path):
    """Host-compiled check of Eq. 1 in integer form as the kernels compute it
    (pc_common.cuh eq1_p_geo: p = max{p : B^p <= 2^w - 1} and
    1 + B + ... + B^(p-1) mod 2^64 in one pass of 64 x 32-bit steps), against
    128-bit brute force for every B in 2..2^20, the bases next to every
    integer k-th root of 2^32 - 1 and 2^64 - 1, the powers of two, and the top
    of the range; plus Eq. 1's values worked by hand for a few bases."""
    import shutil
    import subprocess

    if shutil.which("g++") is None:
        pytest.skip("no host C++ compiler")
    src = tmp_path / "eq1.cpp"
    src.write_text(r'''
#include <cstdio>
#include <cstdint>
#include "pc_common.cuh"
using namespace pcx;
typedef unsigned __int128 u128;
static uint32_t brute_p(uint64_t B, uint32_t w) {
  const u128 C = w == 64 ? (u128)~0ull : (u128)0xFFFFFFFFull;
  u128 x = 1; uint32_t p = 0;
  while (x * B <= C) { x *= B; ++p; }
  return p;
}
static uint64_t brute_geo(uint64_t B, uint32_t p) {
  uint64_t g = 0, x = 1;
  for (uint32_t i = 0; i < p; ++i) { g += x; x *= B; }
  return g;
}
static int check(uint64_t B) {
  for (uint32_t w = 32; w <= 64; w += 32) {
    uint64_t g;
    const uint32_t p = eq1_p_geo(B, w, g), rp = brute_p(B, w);
    if (p != rp || g != brute_geo(B, rp)) { printf("bad B=%llu w=%u\n", (unsigned long long)B, w); return 1; }
    const uint32_t pb = basic_p_geo(B, w, g), rb = rp ? rp : 1;
    if (pb != rb || g != brute_geo(B, rb) || basic_p(B, w) != rb || eq1_p(B, w) != rp) {
      printf("bad basic B=%llu w=%u\n", (unsigned long long)B, w); return 1;
    }
  }
  return 0;
}
static uint64_t iroot(u128 c, uint32_t k) {  // largest r with r^k <= c
  uint64_t lo = 1, hi = 1ull << 33;
  while (lo < hi) {
    const uint64_t mid = lo + (hi - lo + 1) / 2;
    u128 x = 1; bool over = false;
    for (uint32_t i = 0; i < k && !over; ++i) { if (x > c / mid) over = true; else x *= mid; }
    if (!over && x <= c) lo = mid; else hi = mid - 1;
  }
  return lo;
}
int main() {
  for (uint64_t B = 2; B <= (1ull << 20); ++B) if (check(B)) return 1;
  for (uint32_t k = 1; k <= 64; ++k)
    for (int c = 0; c < 2; ++c) {
      const uint64_t r = iroot(c ? (u128)~0ull : (u128)0xFFFFFFFFull, k);
      for (int64_t d = -2; d <= 2; ++d) {
        const int64_t B = (int64_t)r + d;
        if (B >= 2 && (uint64_t)B <= (1ull << 32) && check((uint64_t)B)) return 1;
      }
    }
  for (uint32_t e = 1; e <= 32; ++e)
    for (int d = -1; d <= 1; ++d) {
      const uint64_t B = (1ull << e) + d;
      if (B >= 2 && B <= (1ull << 32) && check(B)) return 1;
    }
  for (uint64_t B = 0xFFFFFFFFull - 4096; B <= (1ull << 32); ++B) if (check(B)) return 1;
  const uint64_t Bs[] = {2, 3, 7, 9, 16, 34, 42, 256, 3850, 65535, 65536, 4294967295ull, 4294967296ull};
  for (uint64_t B : Bs) printf("%llu %u %u\n", (unsigned long long)B, eq1_p(B, 32), eq1_p(B, 64));
  printf("ok\n");
  return 0;
}
''')
    exe = tmp_path / "eq1"
    subprocess.check_call(["g++", "-std=c++17", "-O2", "-I" + os.path.join(ROOT, "include"),
                           "-I" + os.path.join(ROOT, "paper_1805_01844_gb300", "csrc"), str(src), "-o", str(exe)])
    out = subprocess.run([str(exe)], capture_output=True, text=True).stdout.split("\n")
    assert out[-2] == "ok", out[-5:]
    got = {int(r.split()[0]): (int(r.split()[1]), int(r.split()[2])) for r in out[:-2]}
    # Eq. 1 by hand: B^p <= 2^w - 1 < B^(p+1)
    want = {2: (31, 63), 3: (20, 40), 7: (11, 22), 9: (10, 20), 16: (7, 15), 34: (6, 12), 42: (5, 11),
            256: (3, 7), 3850: (2, 5), 65535: (2, 4), 65536: (1, 3), 4294967295: (1, 2), 4294967296: (0, 1)}
    assert got == want
