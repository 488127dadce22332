// Device-wide primitives used by the index build and the result compaction:
// exclusive prefix sums and a stable LSD radix sort of (key, value) pairs.
#pragma once

#include "pj_common.cuh"

namespace pj {

// out[k] = in[0] + ... + in[k-1] for k < n (out must not alias in).
template <class T>
void exclusive_scan(const Ctx& c, const T* in, T* out, size_t n);

// Stable sort of n (key, value) pairs by the low nbits of the key (LSD, 8-bit
// digits).  Sorted pairs end up in keys/vals.
template <class K>
void radix_sort_pairs(const Ctx& c, K* keys, uint32_t* vals, size_t n, int nbits);

// Device-sized forms, for work recorded into a CUDA graph: the launch covers
// `cap` items and the kernels process the first min(cap, *n_dev) of them
// (n_dev NULL: all cap).  exclusive_scan_dn also writes the sum of those
// items to *total when total is not NULL.  radix_sort_pairs_dn ping-pongs
// between (keys, vals) and (keys2, vals2) and returns true when the sorted
// pairs end up in the second pair of arrays; with vals NULL it sorts the
// keys alone (vals2 unused).
template <class T>
void exclusive_scan_dn(const Ctx& c, const T* in, T* out, size_t cap, const unsigned long long* n_dev,
                       unsigned long long* total);
template <class K>
bool radix_sort_pairs_dn(const Ctx& c, K* keys, uint32_t* vals, K* keys2, uint32_t* vals2, size_t cap,
                         const unsigned long long* n_dev, int nbits);

// Copy a u32 array into a u64 array (used before 64-bit offset scans).
void widen_u32(const Ctx& c, const uint32_t* in, uint64_t* out, size_t n);

}  // namespace pj
