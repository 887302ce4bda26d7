// Integer-only device primitives used by the pattern builder: an exclusive
// prefix sum and a bitonic sort of (uint64 key, uint32 value) pairs.  Both
// are deterministic: their results do not depend on scheduling.
#pragma once

#include <cuda_runtime.h>
#include <cstdint>

namespace pf {

// out[i] = sum_{j<i} in[j] for i in [0, n]; out has n+1 entries.
// `tmp` needs scan_tmp_elems(n) int64 entries.
size_t scan_tmp_elems(int64_t n);
template <class T>
int exclusive_scan(const T *in, int64_t *out, int64_t n, int64_t *tmp, cudaStream_t s);

// Sorts n pairs ascending by (key, value).  n may be any size; buffers must
// hold sort_padded(n) entries (the tail is used for padding).
int64_t sort_padded(int64_t n);
int bitonic_sort_pairs(uint64_t *keys, uint32_t *vals, int64_t n, cudaStream_t s);

}  // namespace pf
