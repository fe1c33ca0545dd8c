// Stored-entry counts of a sparse matrix given its row lengths, in 64-bit:
// the CSR entries and the entries of its sliced-ELL copy (32-row slices, each
// padded to its longest row).  Row pointers, slice offsets and column indices
// of this library are int32, so a matrix whose counts pass INT32_MAX cannot
// be stored; the symbolic phase checks this before its 32-bit scan.  Plain
// C++ (no CUDA), checked on the CPU.
#pragma once

#include <stddef.h>
#include <stdint.h>

namespace vag {

inline void sell_entry_counts(const int *row_len, size_t n, int64_t *entries, int64_t *padded) {
  int64_t e = 0, p = 0;
  for (size_t r0 = 0; r0 < n; r0 += 32) {
    const size_t r1 = r0 + 32 < n ? r0 + 32 : n;
    int w = 0;
    for (size_t r = r0; r < r1; ++r) {
      e += row_len[r];
      if (row_len[r] > w) w = row_len[r];
    }
    p += 32 * (int64_t)w;
  }
  *entries = e;
  *padded = p;
}

inline bool fits_int32_indices(const int *row_len, size_t n) {
  int64_t e = 0, p = 0;
  sell_entry_counts(row_len, n, &e, &p);
  return e <= INT32_MAX && p <= INT32_MAX;
}

}  // namespace vag
