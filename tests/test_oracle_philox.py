"""Pins for the oracle's Philox4x32-10 (CPU only).

The oracle's generator is written from the SC'11 definition (Salmon et al.).
It is pinned against a second, independent implementation -- PyTorch's
header-only `at::philox_engine`, compiled here into a small test program --
and against properties any correct Philox4x32 has (a bijection of the
counter for a fixed key; uniform bytes).
"""
import os
import subprocess
import tempfile

import numpy as np
import pytest
from scipy import stats

import oracle

_TORCH_PROG = r"""
#include <ATen/core/PhiloxRNGEngine.h>
#include <cstdio>
#include <cstdint>
int main() {
  unsigned long long seed, sub, off;
  while (std::scanf("%llu %llu %llu", &seed, &sub, &off) == 3) {
    at::philox_engine eng(seed, sub, off);
    unsigned a = eng(), b = eng(), c = eng(), d = eng();
    std::printf("%u %u %u %u\n", a, b, c, d);
  }
  return 0;
}
"""


def _torch_philox_program():
    torch = pytest.importorskip("torch")
    inc = os.path.join(os.path.dirname(torch.__file__), "include")
    hdr = os.path.join(inc, "ATen", "core", "PhiloxRNGEngine.h")
    if not os.path.exists(hdr):
        pytest.skip("PyTorch's Philox header is not installed")
    d = tempfile.mkdtemp(prefix="philox_pin_")
    src = os.path.join(d, "p.cpp")
    exe = os.path.join(d, "p")
    with open(src, "w") as f:
        f.write(_TORCH_PROG)
    r = subprocess.run(["g++", "-std=c++17", "-O1", "-I", inc, src, "-o", exe],
                       capture_output=True, text=True)
    if r.returncode != 0:
        pytest.skip("cannot compile against PyTorch's Philox header: " + r.stderr[:200])
    return exe


def test_philox_matches_pytorch_engine():
    """Counter (off_lo, off_hi, sub_lo, sub_hi), key (seed_lo, seed_hi)."""
    exe = _torch_philox_program()
    rng = np.random.default_rng(7)
    n = 3000
    seeds = rng.integers(0, 2**64, size=n, dtype=np.uint64)
    subs = rng.integers(0, 2**64, size=n, dtype=np.uint64)
    offs = rng.integers(0, 2**64, size=n, dtype=np.uint64)
    # corner cases: all-zero and all-one words
    seeds[:4] = [0, 2**64 - 1, 0, 42]
    subs[:4] = [0, 2**64 - 1, 2**64 - 1, 0]
    offs[:4] = [0, 2**64 - 1, 0, 0]
    inp = "\n".join("%d %d %d" % (int(s), int(b), int(o))
                    for s, b, o in zip(seeds, subs, offs)) + "\n"
    out = subprocess.run([exe], input=inp, capture_output=True, text=True, check=True).stdout
    ref = np.array([[int(v) for v in line.split()] for line in out.strip().split("\n")],
                   dtype=np.uint64).astype(np.uint32)
    mask = np.uint64(0xFFFFFFFF)
    ctr = np.stack([offs & mask, offs >> np.uint64(32), subs & mask, subs >> np.uint64(32)],
                   axis=1).astype(np.uint32)
    key = np.stack([seeds & mask, seeds >> np.uint64(32)], axis=1).astype(np.uint32)
    got = oracle.philox4x32_10(ctr, key)
    assert np.array_equal(got, ref)


def test_philox_counter_bijection_no_repeats():
    """For a fixed key the 128-bit map is a bijection: 2^18 distinct counters
    give 2^18 distinct outputs (and the first words alone almost surely
    differ too)."""
    n = 1 << 18
    c = np.arange(n, dtype=np.uint32)
    ctr = np.stack([c, np.zeros_like(c), np.full_like(c, 5), np.full_like(c, 9)], axis=1)
    out = oracle.philox4x32_10(ctr, [[42, 0]])
    packed = out.view(np.dtype((np.void, 16))).reshape(-1)
    assert np.unique(packed).size == n


def test_philox_bytes_uniform_and_pairs_independent():
    n = 1 << 16
    c = np.arange(n, dtype=np.uint32)
    ctr = np.stack([np.zeros_like(c), c, np.full_like(c, 3), np.full_like(c, 1)], axis=1)
    out = oracle.philox4x32_10(ctr, [[123, 456]])
    b = out.view(np.uint8).reshape(-1)
    hist = np.bincount(b, minlength=256)
    chi2, p = stats.chisquare(hist)
    assert p > 1e-4
    # serial pairs of nibbles
    nib = (b & 0xF).astype(np.int64)
    pairs = nib[:-1:2] * 16 + nib[1::2]
    chi2, p = stats.chisquare(np.bincount(pairs, minlength=256))
    assert p > 1e-4


def test_key_and_counter_words_all_matter():
    base_c = np.array([[1, 2, 3, 4]], dtype=np.uint32)
    base_k = np.array([[5, 6]], dtype=np.uint32)
    ref = oracle.philox4x32_10(base_c, base_k)
    for j in range(4):
        c = base_c.copy()
        c[0, j] ^= 1
        assert not np.array_equal(oracle.philox4x32_10(c, base_k), ref)
    for j in range(2):
        k = base_k.copy()
        k[0, j] ^= 1
        assert not np.array_equal(oracle.philox4x32_10(base_c, k), ref)
