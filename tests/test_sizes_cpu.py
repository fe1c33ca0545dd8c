"""Stored-entry counts behind the int32 size limit (csrc/vag_sizes.h, the code
the symbolic phase runs before its 32-bit scan, compiled here with g++):
the CSR entries and the padded sliced-ELL entries of a matrix from its row
lengths, against numpy, and the limit itself on counts just below and above
2^31 - 1.  CPU only."""
import os
import subprocess
import tempfile

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1602_03641_gb300", "csrc")

HARNESS = r"""
#include <cstdio>
#include <vector>
#include "vag_sizes.h"
// input: n, then n row lengths; output: entries padded fits
int main() {
  long long n;
  if (std::scanf("%lld", &n) != 1) return 1;
  std::vector<int> len((size_t)n);
  for (auto &v : len) std::scanf("%d", &v);
  int64_t e = 0, p = 0;
  vag::sell_entry_counts(len.data(), len.size(), &e, &p);
  std::printf("%lld %lld %d\n", (long long)e, (long long)p, vag::fits_int32_indices(len.data(), len.size()) ? 1 : 0);
  return 0;
}
"""


@pytest.fixture(scope="module")
def exe():
    d = tempfile.mkdtemp()
    src, out = os.path.join(d, "h.cpp"), os.path.join(d, "h")
    with open(src, "w") as f:
        f.write(HARNESS)
    subprocess.run(["g++", "-O2", "-std=c++17", "-I", CSRC, src, "-o", out], check=True)
    return out


def run(exe, lengths):
    text = f"{len(lengths)} " + " ".join(str(int(v)) for v in lengths) + "\n"
    e, p, ok = subprocess.run([exe], input=text, capture_output=True, text=True, check=True).stdout.split()
    return int(e), int(p), ok == "1"


def reference(lengths):
    lengths = np.asarray(lengths, np.int64)
    pad = np.zeros((len(lengths) + 31) // 32 * 32, np.int64)
    pad[:len(lengths)] = lengths
    return int(lengths.sum()), int(32 * pad.reshape(-1, 32).max(axis=1).sum())


@pytest.mark.parametrize("n", [0, 1, 31, 32, 33, 1000, 4097])
def test_counts_match_numpy(exe, n):
    rng = np.random.default_rng(n)
    lengths = rng.integers(0, 161, size=n)
    e, p, ok = run(exe, lengths)
    assert (e, p) == reference(lengths)
    assert ok


def test_the_limit(exe):
    # one slice of rows long enough to pass 2^31 - 1 entries in total
    w = (2**31 - 1) // 32
    e, p, ok = run(exe, [w] * 32)
    assert (e, p) == (32 * w, 32 * w) and ok               # 2^31 - 32: fits
    e, p, ok = run(exe, [w] * 32 + [32])
    assert e == 32 * w + 32 and e > 2**31 - 1 and not ok   # one more row: too many entries
    # the entries fit but their padding does not
    e, p, ok = run(exe, [w + 1] + [0] * 31)
    assert e == w + 1 and p == 32 * (w + 1) and p > 2**31 - 1 and not ok
