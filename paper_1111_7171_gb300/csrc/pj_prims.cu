// Exclusive scan and stable LSD radix sort, written for this library.
//
// Scan: tiles of 4096 values per 1024-thread block (4 per thread), block
// totals scanned recursively, then added back.
//
// Every kernel also takes an optional device-resident item count (n_dev):
// the launch is sized for a capacity, and the kernels read the actual count
// (clamped to the capacity) when they start.  Tiles past the count exit at
// once.  This lets a captured CUDA graph run the primitives on sizes that are
// only known on the device.
//
// Radix sort: 8-bit digits, one pass per digit.  Each pass runs a histogram
// kernel (per-tile digit counts, stored digit-major so that one exclusive
// scan over them yields every (digit, tile) output offset) and a scatter
// kernel.  Inside a 2048-item tile each warp owns 256 consecutive items,
// handled 32 at a time; lanes holding the same digit find each other with
// match.any, so the rank of an item among equal digits follows input order
// and the sort is stable.  The scatter reorders the tile by digit in shared
// memory before writing, so each digit's items leave as one contiguous run.
#include "pj_prims.cuh"

#include <algorithm>

namespace pj {

namespace {

constexpr int SCAN_THREADS = 1024;
constexpr int SCAN_ITEMS = 4;
constexpr int SCAN_TILE = SCAN_THREADS * SCAN_ITEMS;

__device__ __forceinline__ size_t dev_count(size_t cap, const unsigned long long* n_dev) {
  return n_dev ? (size_t)min((unsigned long long)cap, *n_dev) : cap;
}

template <class T>
__global__ void __launch_bounds__(SCAN_THREADS) k_scan_tiles(const T* __restrict__ in, T* __restrict__ out,
                                                             T* __restrict__ tile_sums, size_t n,
                                                             const unsigned long long* __restrict__ n_dev) {
  __shared__ T warp_tot[32];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  n = dev_count(n, n_dev);
  if ((size_t)blockIdx.x * SCAN_TILE >= n) {  // whole block past the count
    if (tid == 0 && tile_sums) tile_sums[blockIdx.x] = T(0);
    return;
  }
  const size_t base = (size_t)blockIdx.x * SCAN_TILE + (size_t)tid * SCAN_ITEMS;
  T v[SCAN_ITEMS];
  T sum = 0;
#pragma unroll
  for (int k = 0; k < SCAN_ITEMS; ++k) {
    v[k] = (base + k < n) ? in[base + k] : T(0);
    sum += v[k];
  }
  T incl = warp_incl_scan(sum);
  if (lane == 31) warp_tot[warp] = incl;
  __syncwarp();
  __syncthreads();
  if (warp == 0) {
    T w = warp_tot[lane];
    T wi = warp_incl_scan(w);
    warp_tot[lane] = wi - w;  // exclusive offset of each warp
    if (lane == 31 && tile_sums) tile_sums[blockIdx.x] = wi;
  }
  __syncwarp();
  __syncthreads();
  T run = incl - sum + warp_tot[warp];
#pragma unroll
  for (int k = 0; k < SCAN_ITEMS; ++k) {
    if (base + k < n) out[base + k] = run;
    run += v[k];
  }
}

template <class T>
__global__ void k_scan_add(T* __restrict__ out, const T* __restrict__ tile_off, size_t n,
                           const unsigned long long* __restrict__ n_dev) {
  n = dev_count(n, n_dev);
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    out[i] += tile_off[i / SCAN_TILE];
}

// *total = in[0] + ... + in[n-1], from the exclusive scan's last entry.
template <class T>
__global__ void k_scan_total(const T* __restrict__ in, const T* __restrict__ out, size_t n,
                             const unsigned long long* __restrict__ n_dev, unsigned long long* total) {
  n = dev_count(n, n_dev);
  *total = n ? (unsigned long long)out[n - 1] + (unsigned long long)in[n - 1] : 0ull;
}

__global__ void k_widen(const uint32_t* __restrict__ in, uint64_t* __restrict__ out, size_t n) {
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = in[i];
}

constexpr int RS_THREADS = 256;
constexpr int RS_WARPS = RS_THREADS / 32;
constexpr int RS_ROUNDS = 8;   // items per lane
constexpr int RS_WARP_ITEMS = 32 * RS_ROUNDS;
constexpr int RS_TILE = RS_WARPS * RS_WARP_ITEMS;  // 2048

template <class K>
__global__ void __launch_bounds__(RS_THREADS) k_rs_hist(const K* __restrict__ keys, size_t n, int shift,
                                                        uint32_t* __restrict__ hist, unsigned ntiles,
                                                        const unsigned long long* __restrict__ n_dev) {
  __shared__ uint32_t h[256];
  const int tid = threadIdx.x;
  n = dev_count(n, n_dev);
  if ((size_t)blockIdx.x * RS_TILE >= n) {  // empty tile: a zero column
    hist[(size_t)tid * ntiles + blockIdx.x] = 0;
    return;
  }
  h[tid] = 0;
  __syncthreads();
  const size_t base = (size_t)blockIdx.x * RS_TILE;
#pragma unroll 4
  for (int k = 0; k < RS_TILE / RS_THREADS; ++k) {
    const size_t i = base + (size_t)k * RS_THREADS + tid;
    if (i < n) atomicAdd(&h[(unsigned)(keys[i] >> shift) & 0xFFu], 1u);
  }
  __syncwarp();
  __syncthreads();
  hist[(size_t)tid * ntiles + blockIdx.x] = h[tid];
}

// VALS false: keys only (vin, vout unused).
template <class K, bool VALS>
__global__ void __launch_bounds__(RS_THREADS) k_rs_scatter(const K* __restrict__ kin, const uint32_t* __restrict__ vin,
                                                           K* __restrict__ kout, uint32_t* __restrict__ vout,
                                                           size_t n, int shift, const uint32_t* __restrict__ offs,
                                                           unsigned ntiles,
                                                           const unsigned long long* __restrict__ n_dev) {
  // The tile is first reordered by digit in shared memory (stably), then
  // written out digit segment by digit segment, so that neighbouring threads
  // write neighbouring addresses.
  __shared__ uint32_t wcnt[RS_WARPS][256];
  __shared__ uint32_t local_start[256], global_start[256];
  __shared__ K skey[RS_TILE];
  __shared__ uint32_t sval[VALS ? RS_TILE : 1];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  n = dev_count(n, n_dev);
  if ((size_t)blockIdx.x * RS_TILE >= n) return;
  for (int d = tid; d < RS_WARPS * 256; d += RS_THREADS) (&wcnt[0][0])[d] = 0;
  __syncthreads();
  const size_t tbase = (size_t)blockIdx.x * RS_TILE;
  const size_t wbase = tbase + (size_t)warp * RS_WARP_ITEMS;
  K key[RS_ROUNDS];
  uint32_t val[RS_ROUNDS];
  uint32_t rank[RS_ROUNDS];
  const unsigned lt = lanemask_lt();
#pragma unroll
  for (int r = 0; r < RS_ROUNDS; ++r) {
    const size_t i = wbase + (size_t)r * 32 + lane;
    const bool valid = i < n;
    key[r] = valid ? kin[i] : K(0);
    val[r] = (VALS && valid) ? vin[i] : 0u;
    const unsigned d = valid ? ((unsigned)(key[r] >> shift) & 0xFFu) : 256u + lane;
    const unsigned peers = __match_any_sync(FULL, d);
    const int leader = __ffs(peers) - 1;
    uint32_t cnt = 0;
    if (valid && lane == leader) cnt = wcnt[warp][d];
    cnt = __shfl_sync(FULL, cnt, leader);
    rank[r] = cnt + __popc(peers & lt);
    __syncwarp();
    if (valid && lane == leader) wcnt[warp][d] = cnt + __popc(peers);
    __syncwarp();
  }
  __syncthreads();
  {
    // one thread per digit: the warps' starts inside the digit, the digit's
    // count in the tile, its start in the tile (block scan) and in the output
    const int d = tid;
    uint32_t run = 0;
#pragma unroll
    for (int w = 0; w < RS_WARPS; ++w) {
      const uint32_t t = wcnt[w][d];
      wcnt[w][d] = run;
      run += t;
    }
    __shared__ uint32_t wsum[RS_WARPS];
    const uint32_t incl = warp_incl_scan(run);
    if (lane == 31) wsum[warp] = incl;
    __syncwarp();
    __syncthreads();
    uint32_t before = 0;
    for (int w = 0; w < warp; ++w) before += wsum[w];
    local_start[d] = before + incl - run;
    global_start[d] = offs[(size_t)d * ntiles + blockIdx.x];
  }
  __syncthreads();
#pragma unroll
  for (int r = 0; r < RS_ROUNDS; ++r) {
    const size_t i = wbase + (size_t)r * 32 + lane;
    if (i < n) {
      const unsigned d = (unsigned)(key[r] >> shift) & 0xFFu;
      const uint32_t lp = local_start[d] + wcnt[warp][d] + rank[r];
      skey[lp] = key[r];
      if (VALS) sval[lp] = val[r];
    }
  }
  __syncthreads();
  const int valid_items = (int)min((size_t)RS_TILE, n - tbase);
  for (int j = tid; j < valid_items; j += RS_THREADS) {
    const K k = skey[j];
    const unsigned d = (unsigned)(k >> shift) & 0xFFu;
    const uint32_t pos = global_start[d] + (uint32_t)(j - (int)local_start[d]);
    kout[pos] = k;
    if (VALS) vout[pos] = sval[j];
  }
}

}  // namespace

template <class T>
void exclusive_scan_dn(const Ctx& c, const T* in, T* out, size_t cap, const unsigned long long* n_dev,
                       unsigned long long* total) {
  if (cap == 0) {
    if (total) PJ_CUDA(cudaMemsetAsync(total, 0, sizeof(*total), c.stream));
    return;
  }
  const unsigned tiles = ceil_div(cap, SCAN_TILE);
  if (tiles == 1) {
    k_scan_tiles<T><<<1, SCAN_THREADS, 0, c.stream>>>(in, out, nullptr, cap, n_dev);
    PJ_LAUNCHED("k_scan_tiles");
  } else {
    DBuf<T> sums(c, tiles), sums_off(c, tiles);
    k_scan_tiles<T><<<tiles, SCAN_THREADS, 0, c.stream>>>(in, out, sums.p, cap, n_dev);
    PJ_LAUNCHED("k_scan_tiles");
    exclusive_scan_dn<T>(c, sums.p, sums_off.p, tiles, nullptr, nullptr);
    // a device count launches a capacity-sized grid: keep it to one wave of
    // grid-stride blocks
    const unsigned grid = n_dev ? std::min<unsigned>(ceil_div(cap, 256), sm_grid_cap(8)) : ceil_div(cap, 256);
    k_scan_add<T><<<grid, 256, 0, c.stream>>>(out, sums_off.p, cap, n_dev);
    PJ_LAUNCHED("k_scan_add");
  }
  if (total) {
    k_scan_total<T><<<1, 1, 0, c.stream>>>(in, out, cap, n_dev, total);
    PJ_LAUNCHED("k_scan_total");
  }
}

template <class T>
void exclusive_scan(const Ctx& c, const T* in, T* out, size_t n) {
  if (n == 0) return;
  exclusive_scan_dn<T>(c, in, out, n, nullptr, nullptr);
}

template <class K>
bool radix_sort_pairs_dn(const Ctx& c, K* keys, uint32_t* vals, K* keys2, uint32_t* vals2, size_t cap,
                         const unsigned long long* n_dev, int nbits) {
  if (cap == 0 || nbits <= 0) return false;
  if (cap > 0xFFFFFFFFull) fail(PJ_EINVAL, "radix sort: more than 2^32 items");
  const unsigned ntiles = ceil_div(cap, RS_TILE);
  DBuf<uint32_t> hist(c, (size_t)256 * ntiles), offs(c, (size_t)256 * ntiles);
  K* ka = keys;
  uint32_t* va = vals;
  K* kb = keys2;
  uint32_t* vb = vals2;
  const int passes = (nbits + 7) / 8;
  for (int p = 0; p < passes; ++p) {
    const int shift = 8 * p;
    k_rs_hist<K><<<ntiles, RS_THREADS, 0, c.stream>>>(ka, cap, shift, hist.p, ntiles, n_dev);
    PJ_LAUNCHED("k_rs_hist");
    exclusive_scan<uint32_t>(c, hist.p, offs.p, (size_t)256 * ntiles);
    if (vals)
      k_rs_scatter<K, true><<<ntiles, RS_THREADS, 0, c.stream>>>(ka, va, kb, vb, cap, shift, offs.p, ntiles, n_dev);
    else
      k_rs_scatter<K, false><<<ntiles, RS_THREADS, 0, c.stream>>>(ka, nullptr, kb, nullptr, cap, shift, offs.p, ntiles,
                                                                 n_dev);
    PJ_LAUNCHED("k_rs_scatter");
    K* tk = ka; ka = kb; kb = tk;
    uint32_t* tv = va; va = vb; vb = tv;
  }
  return ka != keys;
}

template <class K>
void radix_sort_pairs(const Ctx& c, K* keys, uint32_t* vals, size_t n, int nbits) {
  if (n <= 1 || nbits <= 0) return;
  if (n > 0xFFFFFFFFull) fail(PJ_EINVAL, "radix sort: more than 2^32 items");
  DBuf<K> k2(c, n);
  DBuf<uint32_t> v2(c, n);
  if (radix_sort_pairs_dn<K>(c, keys, vals, k2.p, v2.p, n, nullptr, nbits)) {
    PJ_CUDA(cudaMemcpyAsync(keys, k2.p, n * sizeof(K), cudaMemcpyDeviceToDevice, c.stream));
    PJ_CUDA(cudaMemcpyAsync(vals, v2.p, n * sizeof(uint32_t), cudaMemcpyDeviceToDevice, c.stream));
  }
}

void widen_u32(const Ctx& c, const uint32_t* in, uint64_t* out, size_t n) {
  if (n == 0) return;
  k_widen<<<ceil_div(n, 256), 256, 0, c.stream>>>(in, out, n);
  PJ_LAUNCHED("k_widen");
}

template void exclusive_scan_dn<uint32_t>(const Ctx&, const uint32_t*, uint32_t*, size_t,
                                          const unsigned long long*, unsigned long long*);
template void exclusive_scan_dn<unsigned long long>(const Ctx&, const unsigned long long*, unsigned long long*, size_t,
                                                    const unsigned long long*, unsigned long long*);
template bool radix_sort_pairs_dn<unsigned long long>(const Ctx&, unsigned long long*, uint32_t*, unsigned long long*,
                                                      uint32_t*, size_t, const unsigned long long*, int);
template void exclusive_scan<uint32_t>(const Ctx&, const uint32_t*, uint32_t*, size_t);
template void exclusive_scan<uint64_t>(const Ctx&, const uint64_t*, uint64_t*, size_t);
template void exclusive_scan<unsigned long long>(const Ctx&, const unsigned long long*, unsigned long long*, size_t);
template void radix_sort_pairs<uint32_t>(const Ctx&, uint32_t*, uint32_t*, size_t, int);
template void radix_sort_pairs<uint64_t>(const Ctx&, uint64_t*, uint32_t*, size_t, int);
template void radix_sort_pairs<unsigned long long>(const Ctx&, unsigned long long*, uint32_t*, size_t, int);

}  // namespace pj
