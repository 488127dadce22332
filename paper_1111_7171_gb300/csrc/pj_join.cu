// Probe and verification half of the hot path, and the join entry points.
//
//   A4  multi-match-aware substring selection + index lookup (Sec. 4.2,
//       Alg. 2, Lemma 2): one thread per (probing string, indexed length l,
//       segment i) group looks up the selected substrings s[p, l_i] of its
//       window.  k_group_counts counts the non-empty posting runs, a prefix
//       sum places them, k_group_hits writes them as Hits.
//   A6  extension-based verification (Sec. 5.2, Alg. 3): k_verify_hits
//       expands the hits' runs into candidates (q, r, i, p); each thread takes
//       runs of consecutive candidates: segment bytes compared, then
//       d_l = VERIFYSTRINGPAIR(s_l, r_l, i-1) and, if it passes,
//       d_r = VERIFYSTRINGPAIR(s_r, r_r, tau+1-i), each the length-aware band
//       of Sec. 5.1 held in registers with the Lemma 4 early exit.
//   A8  pairs whose indexed (shorter-in-order) string has length <= tau have
//       no even partition (footnote to Sec. 3.1): k_fallback verifies them
//       directly, one thread per short string.
//   A5/A7  accepted matches (pair key, d_l + d_r) are radix-sorted by key,
//       each run of equal keys keeps its least ed (the exact ED of the pair),
//       and runs are compacted by prefix sum into sorted (a, b, ed) records.
//   A9  k_fused_self runs selection, lookups, distinct-pair formation and
//       whole-pair verification of the self join in one persistent kernel
//       (warps pull probes from a device counter); the chunked form above
//       stays for what it does not keep in shared memory.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <chrono>
#include <fstream>
#include <map>
#include <mutex>
#include <sstream>
#include <cstring>
#include <string>

#include <cooperative_groups.h>

#include "pj_internal.cuh"
#include "pj_plan.cuh"
#include "pj_prims.cuh"
#include "pj_probe.cuh"

namespace pj {

namespace cg = cooperative_groups;

struct Counters {
  unsigned long long accepted;
  unsigned long long lookups;
  unsigned long long candidates;
  unsigned long long cells;
  unsigned long long fallback;
  unsigned long long hits;
  unsigned long long err;  // bit 0: run or posting outside the index; bit 1: probe limit
  unsigned long long filtered;  // candidates rejected by the character-count bound
};

struct AccOut {
  unsigned long long* key;
  uint32_t* ed;
  unsigned long long cap;
};

constexpr int BLOCK = 256;

// The kernels of this file use no warp-level collectives and no block
// barriers: every thread works alone and publishes through global atomics or
// prefix sums.  (Earlier forms that placed shuffles, ballots or
// __syncthreads right after the divergent verification loops lost the
// contributions of lanes still inside those loops.)

__device__ __forceinline__ void add_counter(unsigned long long* c, unsigned long long v) {
  if (v) atomicAdd(c, v);
}

// ---------------------------------------------------------------- A4 ------

// Group t of a chunk: its probe q, its index g within q's groups, and the
// view (threshold) the group belongs to; false for the padding groups of the
// last probe block.
//
// MULTI: thresholds differ per probe and q is found by binary search over
// the per-probe group offsets.  Otherwise, with v.interleave, probes are
// interleaved: groups come in blocks of PROBE_BLOCK probes, and inside a
// block the group index g runs outer and the probe inner, so the 32 lanes of
// a warp look up the same (length, segment) group of 32 different probes.  A
// group's window size depends on its segment i and on |s| - l, so these
// lanes run loops of about the same length; 32 consecutive groups of one
// probe span windows of 1 to tau + 1 positions.  For long strings the lanes
// then read 32 different strings instead of one, which costs more than the
// divergence saves, so interleaving is chosen per join by string length;
// without it, a probe's groups are visited in v.gorder's order (widest
// windows first), so that consecutive lanes still get windows of about the
// same size.
// Hits come out ordered by probe block, so a probe cut-over aligned to a
// block boundary still splits them in two.
constexpr uint32_t PROBE_BLOCK = 32;

__host__ __device__ __forceinline__ unsigned long long interleaved_groups(uint32_t pcount, int G) {
  return (unsigned long long)((pcount + PROBE_BLOCK - 1) / PROBE_BLOCK) * PROBE_BLOCK * (unsigned long long)G;
}

template <bool SELF, bool MULTI>
__device__ __forceinline__ bool group_of(const ProbeView& v, unsigned long long t, uint32_t& q, int& g,
                                         ProbeView& vt) {
  if (MULTI) {
    const unsigned long long tg = v.qgoff[v.pbegin] + t;
    uint32_t lo = v.pbegin, hi = v.pbegin + v.pcount;  // last q with qgoff[q] <= tg
    while (hi - lo > 1) {
      const uint32_t mid = lo + ((hi - lo) >> 1);
      if (v.qgoff[mid] <= tg) lo = mid; else hi = mid;
    }
    q = lo;
    g = (int)(tg - v.qgoff[q]);
    vt = view_for_tau(v, v.ptau[q]);
    return true;
  } else if (!v.interleave) {  // chunks hold fewer than 2^32 groups
    const uint32_t G = (uint32_t)groups_per_probe(v.tau, SELF);
    const uint32_t local = (uint32_t)t / G;
    g = (int)((uint32_t)t - local * G);
    if (v.gorder) g = (int)v.gorder[g];
    q = v.pbegin + local;
    vt = v;
    return local < v.pcount;
  } else {
    const uint32_t span = PROBE_BLOCK * (uint32_t)groups_per_probe(v.tau, SELF);
    const uint32_t blk = (uint32_t)t / span;
    const uint32_t r = (uint32_t)t - blk * span;
    g = (int)(r / PROBE_BLOCK);
    const uint32_t local = blk * PROBE_BLOCK + r % PROBE_BLOCK;
    q = v.pbegin + local;
    vt = v;
    return local < v.pcount;
  }
}

// Sizes that a kernel reads from device memory when it starts: the launch
// covers a capacity `cap`, n_dev (if not NULL) holds the actual count.
__device__ __forceinline__ unsigned long long dev_count(unsigned long long cap, const unsigned long long* n_dev) {
  return n_dev ? min(cap, *n_dev) : cap;
}

// The hit of candidate c: the last hit whose first candidate is <= c
// (cand_off ascending from cand_off[0] = 0).  The whole warp searches for one
// c: each round every lane tests one of 32 evenly spaced offsets and a
// ballot keeps the last that is <= c, so about log32(n_hits) dependent
// loads replace log2(n_hits).  All 32 lanes call it with the same c.
__device__ __forceinline__ unsigned long long warp_hit_of(const unsigned long long* __restrict__ cand_off,
                                                          unsigned long long n_hits, unsigned long long c) {
  const unsigned lane = threadIdx.x & 31u;
  unsigned long long lo = 0, n = n_hits;  // the hit is in [lo, lo + n)
  while (n > 1) {
    const unsigned long long step = (n + 31) >> 5;
    const bool le = lane * step < n && cand_off[lo + lane * step] <= c;
    const unsigned b = __ballot_sync(FULL, le);
    const unsigned long long j = b ? 31 - __clz(b) : 0;  // lane 0 tests lo, which is <= c
    lo += j * step;
    n = min(step, n - j * step);
  }
  return lo;
}

// The hit of candidate c >= base, given hb = the hit of base.  Every hit has
// at least one candidate, so it is one of hb .. hb + (c - base).  The warp
// loads the first candidates of the 32 hits after hb at once; a lane whose c
// falls before the last of them finds its hit among those registers in five
// shuffle steps, any other lane by binary search over the rest of its bounded
// range.  All 32 lanes call it (each with its own c >= base).
__device__ __forceinline__ unsigned long long lane_hit_of(const unsigned long long* __restrict__ cand_off,
                                                          unsigned long long n_hits, unsigned long long hb,
                                                          unsigned long long base, unsigned long long c) {
  const unsigned lane = threadIdx.x & 31u;
  const unsigned long long hj = hb + 1 + lane;
  const unsigned long long first = hj < n_hits ? cand_off[hj] : ~0ull;
  unsigned p = 0;  // hits among hb+1 .. hb+31 whose first candidate is <= c
#pragma unroll
  for (unsigned s = 16; s >= 1; s >>= 1) {
    const unsigned long long o = __shfl_sync(FULL, first, p + s - 1);
    if (o <= c) p += s;
  }
  const unsigned long long last = __shfl_sync(FULL, first, 31);
  if (last > c) return hb + p;
  unsigned long long lo = hb + 32, hi = min(n_hits, hb + (c - base) + 1);
  while (hi - lo > 1) {
    const unsigned long long mid = (lo + hi) >> 1;
    if (cand_off[mid] <= c) lo = mid; else hi = mid;
  }
  return lo;
}

// Pass 1 for one group: the number of non-empty lookups and the mask of the
// window positions that found one.  The window's substrings overlap, so
// their keys are rolled from one position to the next.
template <bool SELF>
__device__ __forceinline__ void count_group(const ProbeView& vt, uint32_t q, int g, uint32_t& nh,
                                            unsigned long long& mask, unsigned long long& lookups, int& err) {
  nh = 0;
  mask = 0;
  int l, i, P, li, lo, hi;
  if (group_window(vt, SELF, q, (int)vt.plen[q], g, l, i, P, li, lo, hi)) {
    window_lookups(vt, SELF, q, (int)vt.plen[q], l, i, li, lo, hi, vt.pbytes + vt.poff[q], err,
                   [&](int p, uint32_t, uint32_t) {
                     ++nh;
                     mask |= 1ull << (p - lo);
                   });
    lookups += (unsigned long long)(hi - lo + 1);
  }
}

// Pass 1: counts and masks of every group (probe, length, segment).
template <bool SELF, bool MULTI>
__global__ void __launch_bounds__(BLOCK) k_group_counts(const ProbeView v, unsigned long long n_groups,
                                                        uint32_t* __restrict__ counts,
                                                        unsigned long long* __restrict__ masks, Counters* ctr,
                                                        const unsigned long long* __restrict__ n_dev) {
  n_groups = dev_count(n_groups, n_dev);
  unsigned long long lookups = 0;
  int err = 0;
  for (unsigned long long t = (unsigned long long)blockIdx.x * BLOCK + threadIdx.x; t < n_groups;
       t += (unsigned long long)gridDim.x * BLOCK) {
    uint32_t q;
    int g;
    ProbeView vt;
    uint32_t nh = 0;
    unsigned long long mask = 0;
    if (group_of<SELF, MULTI>(v, t, q, g, vt)) count_group<SELF>(vt, q, g, nh, mask, lookups, err);
    counts[t] = nh;
    masks[t] = mask;
  }
  add_counter(&ctr->lookups, lookups);
  if (err) atomicOr(&ctr->err, (unsigned long long)err);
}

// Pass 2: the positions pass 1 marked are looked up again and written as
// Hits at the group's prefix-sum offset (offsets at or past hits_cap are not
// written).
template <bool SELF, bool MULTI>
__global__ void __launch_bounds__(BLOCK) k_group_hits(const ProbeView v, unsigned long long n_groups,
                                                      const uint32_t* __restrict__ counts,
                                                      const unsigned long long* __restrict__ masks,
                                                      const uint32_t* __restrict__ hit_off, Hit* __restrict__ hits,
                                                      const unsigned long long* __restrict__ n_dev,
                                                      unsigned long long hits_cap) {
  n_groups = dev_count(n_groups, n_dev);
  for (unsigned long long t = (unsigned long long)blockIdx.x * BLOCK + threadIdx.x; t < n_groups;
       t += (unsigned long long)gridDim.x * BLOCK) {
    if (counts[t] == 0) continue;
    uint32_t q;
    int g;
    ProbeView vt;
    if (!group_of<SELF, MULTI>(v, t, q, g, vt)) continue;
    const int ls = (int)vt.plen[q];
    const uint8_t* s = vt.pbytes + vt.poff[q];
    int l, i, P, li, lo, hi;
    int err = 0;
    uint32_t pos = hit_off[t];
    const uint32_t end = (uint32_t)min(hits_cap, (unsigned long long)pos + counts[t]);
    const uint32_t tau_tag = MULTI ? ((uint32_t)vt.tau << 24) : 0u;
    if (group_window(vt, SELF, q, ls, g, l, i, P, li, lo, hi)) {
      unsigned long long m = masks[t];
      while (m && pos < end) {
        const int p = lo + (__ffsll((long long)m) - 1);
        m &= m - 1;
        uint32_t b;
        const uint32_t c = lookup_key(vt, SELF, q, ls, l, seg_key(s + p, li, l, i), b, err);
        if (c) {
          Hit hh{q, b, c, (uint32_t)p | ((uint32_t)i << 16) | tau_tag, 0ull, 0ull};
          if (vt.hit_sides) {
            hh.sl = side_signature(s, p);
            hh.sr = side_signature(s + p + li, ls - p - li);
          }
          hits[pos++] = hh;
        }
      }
    }
  }
}

__global__ void k_hit_counts(const Hit* __restrict__ hits, unsigned long long n, unsigned long long* __restrict__ cnt,
                             const unsigned long long* __restrict__ n_dev) {
  n = dev_count(n, n_dev);
  for (unsigned long long k = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; k < n;
       k += (unsigned long long)gridDim.x * blockDim.x)
    cnt[k] = hits[k].count;
}

// ------------------------------------------------- selection ablation -----
//
// For every group (probing string, indexed length, segment) of the self
// join whose lists are non-empty, the number of substrings each selection
// method of Sec. 4 would look up: length-based, shift-based, position-aware
// (Sec. 4.1) and multi-match-aware (Sec. 4.2, what the join looks up).
struct SelCounts {
  unsigned long long w[4];
  unsigned long long groups;
};

__global__ void __launch_bounds__(BLOCK) k_selection_counts(const ProbeView v, unsigned long long n_groups,
                                                            SelCounts* out) {
  const unsigned long long G = (unsigned long long)groups_per_probe(v.tau, true);
  unsigned long long c[4] = {0, 0, 0, 0}, groups = 0;
  for (unsigned long long t = (unsigned long long)blockIdx.x * BLOCK + threadIdx.x; t < n_groups;
       t += (unsigned long long)gridDim.x * BLOCK) {
    const uint32_t q = v.pbegin + (uint32_t)(t / G);
    int w[4];
    if (group_selection_sizes(v, true, q, (int)v.plen[q], (int)(t % G), w)) {
      ++groups;
#pragma unroll
      for (int m = 0; m < 4; ++m) c[m] += (unsigned long long)w[m];
    }
  }
#pragma unroll
  for (int m = 0; m < 4; ++m) add_counter(&out->w[m], c[m]);
  add_counter(&out->groups, groups);
}

// ---------------------------------------------------------------- A6 ------

constexpr int V_RUN = 8;  // candidates per lane per step

// Lane l of a warp verifies candidates base + l + 32 k (k < V_RUN): the 32
// lanes take consecutive candidates, which mostly belong to one posting run
// and so share the probing string, the segment, the position and the
// indexed length -- the verification loops then have equal trip counts up to
// early termination.  Each lane finds its first hit from the warp's
// (warp_hit_of, lane_hit_of) and walks forward from there, reloading the hit
// only when it crosses into the next one.
template <int MAXW, bool SELF, bool MULTI>
__global__ void __launch_bounds__(512) k_verify_hits(const ProbeView v, const Hit* __restrict__ hits,
                                                       const unsigned long long* __restrict__ cand_off,
                                                       unsigned long long n_hits, unsigned long long c_begin,
                                                       unsigned long long n_cand, AccOut out, Counters* ctr,
                                                       const unsigned long long* __restrict__ dn) {
  if (dn) {  // device sizes: dn[0] hits (clamped to n_hits), dn[1] candidates
    n_hits = min(n_hits, dn[0]);
    n_cand = dn[1];
  }
  unsigned long long cells = 0, filtered = 0;
  int err = 0;
  const unsigned lane = threadIdx.x & 31u;
  const unsigned long long warp = ((unsigned long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const unsigned long long n_warps = ((unsigned long long)gridDim.x * blockDim.x) >> 5;
  const unsigned long long span = 32ull * V_RUN;
  for (unsigned long long base = c_begin + warp * span; base < n_cand; base += n_warps * span) {
    unsigned long long c = base + lane;
    unsigned long long h = lane_hit_of(cand_off, n_hits, warp_hit_of(cand_off, n_hits, base), base, c);
    if (c >= n_cand) continue;
    unsigned long long c_lo = cand_off[h];
    unsigned long long c_hi = h + 1 < n_hits ? cand_off[h + 1] : n_cand;
    Hit hit = hits[h];
    ProbeView vt = MULTI ? view_for_tau(v, (int)(hit.pi >> 24)) : v;
    HitCtx hc = hit_ctx(vt, hit);
    for (int k = 0; k < V_RUN && c < n_cand; ++k, c += 32) {
      if (c >= c_hi) {  // into a later hit
        do {
          ++h;
          c_lo = c_hi;
          c_hi = h + 1 < n_hits ? cand_off[h + 1] : n_cand;
        } while (c >= c_hi);
        hit = hits[h];
        if (MULTI) vt = view_for_tau(v, (int)(hit.pi >> 24));
        hc = hit_ctx(vt, hit);
      }
      unsigned long long key = 0;
      int ed = 0;
      if (verify_in_hit<MAXW>(vt, SELF, hc, (uint32_t)(c - c_lo), key, ed, cells, filtered, err)) {
        const unsigned long long pos = atomicAdd(&ctr->accepted, 1ull);
        if (pos < out.cap) {
          out.key[pos] = key;
          out.ed[pos] = (uint32_t)ed;
        }
      }
    }
  }
  add_counter(&ctr->cells, cells);
  add_counter(&ctr->filtered, filtered);
  if (err) atomicOr(&ctr->err, (unsigned long long)err);
}

// The same verification with a screen and a per-warp queue.  The candidates
// are dealt to the warps round robin in chunks of `chunk` (Q_CHUNK, or up to
// 4 Q_CHUNK for launches long enough that every warp gets thousands of
// chunks: fewer searches of the candidate offsets); a warp walks a
// chunk in steps of 32 * S_RUN: in a step, lane l screens candidates base +
// l + 32 k (k < S_RUN) -- valid sid, not the probe itself, the side bounds
// of the extension screen -- so that every load of a posting record is one
// coalesced 512-byte request for the warp.  The warp searches the candidate
// offsets once per chunk; after that, every lane walks from hit to hit on its
// own as its candidates advance (hits are in candidate order).  Chunks of a
// few thousand candidates keep the warps' loads even: survivors and their
// DP work cluster in places.  Survivors enter a queue in shared memory (one ballot per
// 32 candidates), each with its probe, sid and (position, segment,
// threshold); while 32 or more are queued, each lane takes one and runs
// extension verification.  Screened-out candidates cost no DP slot, so the
// warps' DP lanes stay full.  The ballots and the queue loop run the same
// number of times in all 32 lanes, and queue entries are read before the
// next writes only after a __syncwarp.
constexpr int Q_BLOCK = 256;
constexpr int Q_WARPS = Q_BLOCK / 32;
constexpr int S_RUN = 8;                 // candidates one lane screens per step
constexpr int Q_CAP = 32 * S_RUN + 32;   // < 32 left + up to 32 * S_RUN new
constexpr unsigned long long Q_CHUNK = 8ull * 32 * S_RUN;  // candidates a warp takes at a time (at least)

// Chunk of a queued verification launch over n candidates on `grid` blocks:
// Q_CHUNK, times up to 4 when every warp gets at least 512 chunks of that
// size (measured on 2.2e10 candidates: 3% less time with 4; on 3e8, where a
// warp gets 30 chunks, larger chunks unbalance the warps).
static unsigned long long queued_chunk(unsigned long long n, unsigned grid) {
  const unsigned long long per_warp = n / ((unsigned long long)grid * Q_WARPS * Q_CHUNK);
  return Q_CHUNK * std::min<unsigned long long>(4, std::max<unsigned long long>(1, per_warp / 512));
}

// One lane's hit: index h, its posting for candidate c is rec_base + c
// (mod 2^32: posting indices are 32-bit), and what the screen needs of it.
struct LaneHit {
  uint32_t h;
  uint32_t rec_base;
  uint32_t q, pi;
  unsigned long long sl, sr;  // the probe's side signatures around the match
};

__device__ __forceinline__ void lane_hit_set(const Hit* __restrict__ hits, uint32_t h, unsigned long long c_lo,
                                             LaneHit& lh) {
  const Hit hit = hits[h];
  lh.h = h;
  lh.rec_base = hit.begin - (uint32_t)c_lo;
  lh.q = hit.q;
  lh.pi = hit.pi;
  lh.sl = hit.sl;
  lh.sr = hit.sr;
}

// Extension verification of one queue entry: probe q, indexed sid r, and
// the match's position, segment and threshold packed in pi.
template <int MAXW, bool SELF, bool MULTI>
__device__ __forceinline__ void verify_queued_entry(const ProbeView& v, uint32_t q, uint32_t r, uint32_t pi,
                                                    AccOut out, Counters* ctr, unsigned long long& cells) {
  const ProbeView vt = MULTI ? view_for_tau(v, (int)(pi >> 24)) : v;
  HitCtx hc;
  hc.q = q;
  hc.begin = 0;
  hc.p = (int)(pi & 0xFFFFu);
  hc.i = (int)((pi >> 16) & 0xFFu);
  if (vt.pref) {
    const unsigned long long ref = vt.pref[q];
    hc.ls = (int)(ref & 0xFFFFu);
    hc.s = vt.pbytes + (ref >> 16);
  } else {
    hc.ls = (int)vt.plen[q];
    hc.s = vt.pbytes + vt.poff[q];
  }
  unsigned long long key = 0;
  int ed = 0;
  if (verify_screened<MAXW>(vt, SELF, hc, r, key, ed, cells)) {
    const unsigned long long pos = atomicAdd(&ctr->accepted, 1ull);
    if (pos < out.cap) {
      out.key[pos] = key;
      out.ed[pos] = (uint32_t)ed;
    }
  }
}

template <int MAXW, bool SELF, bool MULTI>
__global__ void __launch_bounds__(Q_BLOCK) k_verify_queued(const ProbeView v, const Hit* __restrict__ hits,
                                                            const unsigned long long* __restrict__ cand_off,
                                                            unsigned long long n_hits, unsigned long long c_begin,
                                                            unsigned long long n_cand, AccOut out, Counters* ctr,
                                                            const unsigned long long* __restrict__ dn,
                                                            unsigned long long chunk) {
  __shared__ uint32_t q_q[Q_WARPS][Q_CAP];
  __shared__ uint32_t q_sid[Q_WARPS][Q_CAP];
  __shared__ uint32_t q_pi[Q_WARPS][Q_CAP];
  if (dn) {
    n_hits = min(n_hits, dn[0]);
    n_cand = dn[1];
  }
  unsigned long long cells = 0, filtered = 0;
  int err = 0;
  const unsigned lane = threadIdx.x & 31u, wib = threadIdx.x >> 5;
  const unsigned long long warp = ((unsigned long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const unsigned long long n_warps = ((unsigned long long)gridDim.x * blockDim.x) >> 5;
  const unsigned long long span = 32ull * S_RUN;
  int qn = 0;  // the same in every lane
  LaneHit lh;
  lh.h = UINT32_MAX;
  // chunks of `chunk` candidates, dealt to the warps round robin
  for (unsigned long long r0 = c_begin + warp * chunk; r0 < n_cand; r0 += n_warps * chunk) {
    const unsigned long long r1 = min(n_cand, r0 + chunk);
    // each lane's hit: its first candidate's, found by a warp search; then
    // every lane walks forward on its own as its candidates advance
    unsigned long long l_hi;  // first candidate after the lane's hit
    {
      const unsigned long long cf = min(r0 + lane, r1 - 1);
      const unsigned long long h = lane_hit_of(cand_off, n_hits, warp_hit_of(cand_off, n_hits, r0), r0, cf);
      lane_hit_set(hits, (uint32_t)h, cand_off[h], lh);
      l_hi = h + 1 < n_hits ? cand_off[h + 1] : n_cand;
    }
    for (unsigned long long base = r0; base < r1; base += span) {
      // screen; each survivor goes straight into the queue (one ballot per 32)
#pragma unroll
      for (int k = 0; k < S_RUN; ++k) {
        const unsigned long long c0 = base + 32ull * k;
        if (c0 >= r1) break;  // the same in every lane
        const unsigned long long c = c0 + lane;
        bool pass = false;
        uint32_t r = 0;
        if (c < r1) {
          if (c >= l_hi) {  // into a later hit: walk to it
            unsigned long long h = lh.h, lo;
            do {
              ++h;
              lo = l_hi;
              l_hi = h + 1 < n_hits ? cand_off[h + 1] : n_cand;
            } while (c >= l_hi);
            lane_hit_set(hits, (uint32_t)h, lo, lh);
          }
          const ProbeView vt = MULTI ? view_for_tau(v, (int)(lh.pi >> 24)) : v;
          const PostRec rec = vt.precs[lh.rec_base + (uint32_t)c];
          r = rec_sid(rec);
          if (r >= vt.n_index) {
            err |= 1;
          } else if (!(SELF && r == lh.q)) {
            // the side bounds against the two sides' thresholds i - 1 and tau + 1 - i
            const int i = (int)((lh.pi >> 16) & 0xFFu);
            if (v.pbm && v.hit_sides && (side_bound(lh.sl, rec_left(rec)) > i - 1 ||
                          side_bound(lh.sr, rec_right(rec)) > vt.tau + 1 - i))
              ++filtered;
            else
              pass = true;
          }
        }
        const unsigned b = __ballot_sync(FULL, pass);
        if (pass) {
          const int slot = qn + __popc(b & lanemask_lt());
          q_q[wib][slot] = lh.q;
          q_sid[wib][slot] = r;
          q_pi[wib][slot] = lh.pi;
        }
        qn += __popc(b);
      }
      __syncwarp();
      while (qn >= 32) {  // the same in every lane
        qn -= 32;
        const uint32_t q2 = q_q[wib][qn + lane], r2 = q_sid[wib][qn + lane], p2 = q_pi[wib][qn + lane];
        __syncwarp();  // taken before any later write
        verify_queued_entry<MAXW, SELF, MULTI>(v, q2, r2, p2, out, ctr, cells);
      }
    }
  }
  __syncwarp();
  if ((int)lane < qn) verify_queued_entry<MAXW, SELF, MULTI>(v, q_q[wib][lane], q_sid[wib][lane], q_pi[wib][lane],
                                                             out, ctr, cells);
  add_counter(&ctr->cells, cells);
  add_counter(&ctr->filtered, filtered);
  if (err) atomicOr(&ctr->err, (unsigned long long)err);
}

// One warp per candidate (long strings): the warp walks candidates
// c_begin + w, c_begin + w + n_warps, ...; every lane runs the same code on
// the same candidate, so the shuffles and ballots of vsp_warp see a
// converged warp.  Lane 0 publishes results.
template <bool SELF, bool MULTI>
__global__ void __launch_bounds__(512) k_verify_warp(const ProbeView v, const Hit* __restrict__ hits,
                                                       const unsigned long long* __restrict__ cand_off,
                                                       unsigned long long n_hits, unsigned long long c_begin,
                                                       unsigned long long c_end, AccOut out, Counters* ctr) {
  const unsigned lane = threadIdx.x & 31u;
  const unsigned long long warp = ((unsigned long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const unsigned long long n_warps = ((unsigned long long)gridDim.x * blockDim.x) >> 5;
  unsigned long long cells = 0;
  int err = 0;
  for (unsigned long long c = c_begin + warp; c < c_end; c += n_warps) {
    __syncwarp();
    const unsigned long long lo = warp_hit_of(cand_off, n_hits, c);
    const Hit hit = hits[lo];
    const ProbeView vt = MULTI ? view_for_tau(v, (int)(hit.pi >> 24)) : v;
    unsigned long long key = 0;
    int ed = 0;
    const bool ok = verify_candidate_warp(vt, SELF, hit, (uint32_t)(c - cand_off[lo]), key, ed, cells, err);
    if (ok && lane == 0) {
      const unsigned long long pos = atomicAdd(&ctr->accepted, 1ull);
      if (pos < out.cap) {
        out.key[pos] = key;
        out.ed[pos] = (uint32_t)ed;
      }
    }
  }
  __syncwarp();
  if (lane == 0) {
    add_counter(&ctr->cells, cells);
    if (err) atomicOr(&ctr->err, (unsigned long long)err);
  }
}

// First hit whose probe id is >= q (hits are in probe order).
__global__ void k_hit_lower_bound(const Hit* __restrict__ hits, unsigned long long n, uint32_t q,
                                  unsigned long long* out) {
  unsigned long long lo = 0, hi = n;
  while (lo < hi) {
    const unsigned long long mid = (lo + hi) >> 1;
    if (hits[mid].q < q) lo = mid + 1; else hi = mid;
  }
  *out = lo;
}

// ------------------------------------------------------ A5 + A6, mode L --
//
// Materialised mode: the candidates of a chunk become pair keys, are sorted
// and made unique, and every distinct pair is verified ONCE over the whole
// strings with the length-aware VERIFYSTRINGPAIR (Sec. 5.1), which returns
// min(tau + 1, ED) exactly.  Near-duplicate long strings share a segment
// match for almost every one of their tau + 1 segments, so extension
// verification (one DP pass per match) would verify each such pair up to
// tau + 1 times; here it is verified once.  Keys are made of sids: probe sid
// (self join) or probe index (R != S) << pshift | indexed sid.

constexpr unsigned long long NO_PAIR = ~0ull;

// Lane l of a warp writes the keys of candidates base + l + 32 k (the walk
// of k_verify_hits).
template <bool SELF>
__global__ void __launch_bounds__(BLOCK) k_pair_keys(const ProbeView v, const Hit* __restrict__ hits,
                                                     const unsigned long long* __restrict__ cand_off,
                                                     unsigned long long n_hits, unsigned long long c_begin,
                                                     unsigned long long c_end, int pshift,
                                                     unsigned long long* __restrict__ keys, Counters* ctr,
                                                     const unsigned long long* __restrict__ dn) {
  if (dn) {  // device sizes: dn[0] hits (clamped to n_hits), dn[1] candidates (clamped to c_end)
    n_hits = min(n_hits, dn[0]);
    c_end = min(c_end, dn[1]);
  }
  const unsigned lane = threadIdx.x & 31u;
  const unsigned long long warp = ((unsigned long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const unsigned long long n_warps = ((unsigned long long)gridDim.x * blockDim.x) >> 5;
  const unsigned long long span = 32ull * V_RUN;
  int err = 0;
  for (unsigned long long base = c_begin + warp * span; base < c_end; base += n_warps * span) {
    unsigned long long c = base + lane;
    unsigned long long h = lane_hit_of(cand_off, n_hits, warp_hit_of(cand_off, n_hits, base), base, c);
    if (c >= c_end) continue;
    unsigned long long c_lo = cand_off[h];
    unsigned long long c_hi = h + 1 < n_hits ? cand_off[h + 1] : c_end;
    Hit hit = hits[h];
    for (int k = 0; k < V_RUN && c < c_end; ++k, c += 32) {
      if (c >= c_hi) {
        do {
          ++h;
          c_lo = c_hi;
          c_hi = h + 1 < n_hits ? cand_off[h + 1] : c_end;
        } while (c >= c_hi);
        hit = hits[h];
      }
      const uint32_t r = v.postings[hit.begin + (uint32_t)(c - c_lo)];
      unsigned long long key = NO_PAIR;
      if (r >= v.n_index) {
        err |= 1;
      } else if (!(SELF && r == hit.q)) {
        const uint32_t x = SELF ? min(hit.q, r) : hit.q, y = SELF ? max(hit.q, r) : r;
        key = ((unsigned long long)x << pshift) | y;
      }
      keys[c - c_begin] = key;
    }
  }
  if (err) atomicOr(&ctr->err, (unsigned long long)err);
}

__global__ void k_unique_keys(const unsigned long long* __restrict__ keys, const uint32_t* __restrict__ flags,
                              const uint32_t* __restrict__ pos, unsigned long long n,
                              unsigned long long* __restrict__ ukeys, const unsigned long long* __restrict__ n_dev) {
  n = dev_count(n, n_dev);
  for (unsigned long long k = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; k < n;
       k += (unsigned long long)gridDim.x * blockDim.x)
    if (flags[k]) ukeys[pos[k]] = keys[k];
}

// The strings of a pair key (x from the probe side, y from the index side).
__device__ __forceinline__ void pair_strings(const ProbeView& v, bool self, unsigned long long key, int pshift,
                                             uint32_t& x, uint32_t& y, const uint8_t*& sx, int& lx,
                                             const uint8_t*& sy, int& ly) {
  x = (uint32_t)(key >> pshift);
  y = (uint32_t)(key & ((1ull << pshift) - 1));
  sx = v.pbytes + v.poff[x];
  lx = (int)v.plen[x];
  sy = v.ibytes + v.ioff[y];
  ly = (int)v.ilen[y];
  (void)self;
}

__device__ __forceinline__ unsigned long long pair_out_key(const ProbeView& v, bool self, uint32_t x, uint32_t y) {
  const uint32_t qid = v.pid ? v.pid[x] : x;
  const uint32_t rid = v.iperm[y];
  const uint32_t ka = self ? min(qid, rid) : qid;
  const uint32_t kb = self ? max(qid, rid) : rid;
  return ((unsigned long long)ka << v.key_shift) | kb;
}

__device__ __forceinline__ void append_match(Counters* ctr, const AccOut& out, unsigned long long key, int ed) {
  const unsigned long long pos = atomicAdd(&ctr->accepted, 1ull);
  if (pos < out.cap) {
    out.key[pos] = key;
    out.ed[pos] = (uint32_t)ed;
  }
}

// Shared prefixes (Sec. 5.3).  Distinct pairs are sorted by (probe, indexed
// sid), and sids order each length's strings by their first eight bytes, so
// consecutive pairs of one probe whose indexed strings have the same length
// often share a prefix.  A verifier (thread or warp) then takes a run of
// consecutive pairs and keeps one band state across them: with the rows over
// the indexed string r, rows 1..c of two r's sharing their first c
// characters are identical.  Before each pair it computes c against the
// string whose band it holds; if that string was stopped by Lemma 4 at a row
// e <= c, this pair stops there too (same rows, same lengths); if the band
// was kept at a row <= c, the scan resumes after it.  The row kept is the
// common prefix with the next pair of the group.  Verifiers take the groups
// round robin, and most groups are single pairs, so the load stays spread.
// Enabled by PJ_SHARE_PREFIX=1 (off by default: on the synthetic workloads
// consecutive pairs of a probe rarely share a prefix of the same length).
constexpr int PAIR_RUN = 64;  // longest group of consecutive pairs one verifier takes

// The band state a verifier keeps between consecutive pairs.
struct KeptBand {
  uint32_t x = UINT32_MAX;    // probe of the pair that owns it
  int len = -1;               // length of its indexed string
  const uint8_t* r = nullptr; // its indexed string
  int row = 0;                // row after which the band was kept (0: none)
  int dead = 0;               // row at which Lemma 4 stopped it (0: ran to the end)
};

// A distinct pair with its strings (x: probe side, y: index side).
struct PairView {
  uint32_t x, y;
  const uint8_t *sx, *sy;
  int lx, ly;
};

__device__ __forceinline__ bool pair_view(const ProbeView& v, bool self, const unsigned long long* ukeys,
                                          unsigned long long n, unsigned long long u, int pshift, PairView& p) {
  if (u >= n) return false;
  const unsigned long long key = ukeys[u];
  if (key == NO_PAIR) return false;
  pair_strings(v, self, key, pshift, p.x, p.y, p.sx, p.lx, p.sy, p.ly);
  return true;
}

// Consecutive pairs whose rows can be shared: the same probe, indexed
// strings of the same length, no longer than the probe (the rows run over
// the shorter string).
__device__ __forceinline__ bool same_group(const PairView& a, const PairView& b) {
  return a.x == b.x && a.ly == b.ly && a.ly <= a.lx;
}

// One thread per distinct pair, or (v.share_prefix) one thread per group of
// consecutive pairs that can share rows (same probe, indexed strings of one
// length; at most PAIR_RUN, groups split at multiples of PAIR_RUN), the
// band kept across them.
template <int MAXW, bool SELF>
__global__ void __launch_bounds__(BLOCK) k_verify_pairs(const ProbeView v, const unsigned long long* __restrict__ ukeys,
                                                        unsigned long long n, int pshift, AccOut out, Counters* ctr,
                                                        const unsigned long long* __restrict__ n_dev) {
  n = dev_count(n, n_dev);
  unsigned long long cells = 0, filtered = 0;
  if (!v.share_prefix) {
    for (unsigned long long u = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; u < n;
         u += (unsigned long long)gridDim.x * blockDim.x) {
      const unsigned long long key = ukeys[u];
      if (key == NO_PAIR) continue;
      uint32_t x, y;
      const uint8_t *sx, *sy;
      int lx, ly;
      pair_strings(v, SELF, key, pshift, x, y, sx, lx, sy, ly);
      if (v.pbm && signature_bound(v.pbm[x], v.ibm[y]) > v.tau) {
        ++filtered;
        continue;
      }
      const int d = vsp<MAXW>(sx, lx, sy, ly, v.tau, cells);
      if (d <= v.tau) append_match(ctr, out, pair_out_key(v, SELF, x, y), d);
    }
  } else {
    for (unsigned long long u = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; u < n;
         u += (unsigned long long)gridDim.x * blockDim.x) {
      PairView cur;
      if (!pair_view(v, SELF, ukeys, n, u, pshift, cur)) continue;
      if (u % PAIR_RUN != 0) {  // inside a group that an earlier position starts
        PairView prev;
        if (pair_view(v, SELF, ukeys, n, u - 1, pshift, prev) && same_group(prev, cur)) continue;
      }
      KeptBand kb;
      int V[MAXW], snap[MAXW];
      for (unsigned long long w = u;;) {
        PairView nxt;
        const bool more = w + 1 < n && (w + 1) % PAIR_RUN != 0 && pair_view(v, SELF, ukeys, n, w + 1, pshift, nxt) &&
                          same_group(cur, nxt);
        if (v.pbm && signature_bound(v.pbm[cur.x], v.ibm[cur.y]) > v.tau) {
          ++filtered;
        } else if (cur.ly > cur.lx) {  // rows over the shorter string: nothing to share
          const int d = vsp<MAXW>(cur.sx, cur.lx, cur.sy, cur.ly, v.tau, cells);
          if (d <= v.tau) append_match(ctr, out, pair_out_key(v, SELF, cur.x, cur.y), d);
        } else if (cur.lx - cur.ly <= v.tau) {
          const int keep = more ? common_prefix(cur.sy, nxt.sy, cur.ly) : 0;
          int start = 0, d = v.tau + 1, dead = 0;
          bool skip = false;
          if (kb.x == cur.x && kb.len == cur.ly) {
            const int c = common_prefix(cur.sy, kb.r, cur.ly);
            if (kb.dead && c >= kb.dead) {
              skip = true;  // the same rows stop the scan at the same row
            } else if (kb.row && c >= kb.row) {
              start = kb.row;
#pragma unroll
              for (int k = 0; k < MAXW; ++k) V[k] = snap[k];
            }
          }
          if (!skip) {
            d = vsp_rows<MAXW>(cur.sy, cur.ly, cur.sx, cur.lx, v.tau, start, V, keep, snap, dead, cells);
            kb.x = cur.x;
            kb.len = cur.ly;
            kb.r = cur.sy;
            kb.row = keep > start ? (!dead || dead >= keep ? keep : 0) : (keep == start ? start : 0);
            kb.dead = dead;
          }
          if (d <= v.tau) append_match(ctr, out, pair_out_key(v, SELF, cur.x, cur.y), d);
        }
        if (!more) break;
        ++w;
        cur = nxt;
      }
    }
  }
  add_counter(&ctr->cells, cells);
  add_counter(&ctr->filtered, filtered);
}

// Length of the common prefix of a and b (n bytes at most), by the whole
// warp; every lane must call it with the same arguments.
__device__ __forceinline__ int warp_common_prefix(const uint8_t* a, const uint8_t* b, int n) {
  const int lane = threadIdx.x & 31;
  int res = n;
  for (int k = 0; k < n; k += 32) {
    const int j = k + lane;
    const unsigned m = __ballot_sync(FULL, j < n && a[j] != b[j]);
    if (m) {
      res = k + __ffs((int)m) - 1;
      break;
    }
  }
  return res;
}

// One warp per distinct pair (long strings): the shuffle-scan band of
// vsp_warp; every lane runs the same code on the same pair.  With
// v.share_prefix, one warp per group of pairs that can share rows (as
// k_verify_pairs), the band kept across them (vsp_warp_rows).
template <bool SELF>
__global__ void __launch_bounds__(BLOCK) k_verify_pairs_warp(const ProbeView v,
                                                             const unsigned long long* __restrict__ ukeys,
                                                             unsigned long long n, int pshift, AccOut out,
                                                             Counters* ctr,
                                                             const unsigned long long* __restrict__ n_dev) {
  n = dev_count(n, n_dev);
  const unsigned lane = threadIdx.x & 31u;
  const unsigned long long warp = ((unsigned long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const unsigned long long n_warps = ((unsigned long long)gridDim.x * blockDim.x) >> 5;
  unsigned long long cells = 0;
  if (!v.share_prefix) {
    for (unsigned long long u = warp; u < n; u += n_warps) {
      __syncwarp();
      const unsigned long long key = ukeys[u];
      if (key == NO_PAIR) continue;  // uniform across the warp
      uint32_t x, y;
      const uint8_t *sx, *sy;
      int lx, ly;
      pair_strings(v, SELF, key, pshift, x, y, sx, lx, sy, ly);
      if (v.pbm && signature_bound(v.pbm[x], v.ibm[y]) > v.tau) continue;  // uniform across the warp
      const int d = vsp_warp(sx, lx, sy, ly, v.tau, cells);
      if (d <= v.tau && lane == 0) append_match(ctr, out, pair_out_key(v, SELF, x, y), d);
    }
  } else {
    for (unsigned long long u = warp; u < n; u += n_warps) {
      __syncwarp();
      PairView cur;
      if (!pair_view(v, SELF, ukeys, n, u, pshift, cur)) continue;  // uniform across the warp
      if (u % PAIR_RUN != 0) {
        PairView prev;
        if (pair_view(v, SELF, ukeys, n, u - 1, pshift, prev) && same_group(prev, cur)) continue;  // uniform
      }
      KeptBand kb;
      int V0 = 0, V1 = 0, S0 = 0, S1 = 0;
      for (unsigned long long w = u;;) {
        PairView nxt;
        const bool more = w + 1 < n && (w + 1) % PAIR_RUN != 0 && pair_view(v, SELF, ukeys, n, w + 1, pshift, nxt) &&
                          same_group(cur, nxt);
        if (v.pbm && signature_bound(v.pbm[cur.x], v.ibm[cur.y]) > v.tau) {
          // screened out (uniform across the warp)
        } else if (cur.ly > cur.lx) {
          const int d = vsp_warp(cur.sx, cur.lx, cur.sy, cur.ly, v.tau, cells);
          if (d <= v.tau && lane == 0) append_match(ctr, out, pair_out_key(v, SELF, cur.x, cur.y), d);
        } else if (cur.lx - cur.ly <= v.tau) {
          const int keep = more ? warp_common_prefix(cur.sy, nxt.sy, cur.ly) : 0;
          int start = 0, d = v.tau + 1, dead = 0;
          bool skip = false;
          if (kb.x == cur.x && kb.len == cur.ly) {
            const int c = warp_common_prefix(cur.sy, kb.r, cur.ly);
            if (kb.dead && c >= kb.dead) {
              skip = true;
            } else if (kb.row && c >= kb.row) {
              start = kb.row;
              V0 = S0;
              V1 = S1;
            }
          }
          if (!skip) {
            d = vsp_warp_rows(cur.sy, cur.ly, cur.sx, cur.lx, v.tau, start, V0, V1, keep, S0, S1, dead, cells);
            kb.x = cur.x;
            kb.len = cur.ly;
            kb.r = cur.sy;
            kb.row = keep > start ? (!dead || dead >= keep ? keep : 0) : (keep == start ? start : 0);
            kb.dead = dead;
          }
          if (d <= v.tau && lane == 0) append_match(ctr, out, pair_out_key(v, SELF, cur.x, cur.y), d);
        }
        if (!more) break;
        ++w;
        cur = nxt;
      }
    }
  }
  __syncwarp();
  if (lane == 0) add_counter(&ctr->cells, cells);
}

// ------------------------------------------------ fused self join (A9) ---
//
// One persistent kernel for the whole-pair (mode L) self join.  Each warp
// takes work items -- `ppi` consecutive probing strings -- from a device
// counter (work[0]), from the two ends of the length order in turn, and runs
// the whole path for its item without leaving the SM:
//   * multi-match-aware selection and the lookups of every (probe, length,
//     segment) group, the window's keys rolled (Sec. 4.2, Alg. 2): for short
//     and medium strings an item is 32 probes, a lane per probe, and the
//     lanes take the same group number together (windows of about one size,
//     as the interleaved probe pass does); for long strings the lanes share
//     one probe's groups, widest windows first;
//   * every posting of a non-empty run is a candidate pair (q, r) -- runs
//     longer than FRUN_MIN are queued and expanded by the whole warp, a
//     posting per lane, after the lookups; runs longer than FRUN_BIG (the
//     short probes of a high threshold, whose segments are a few characters)
//     leave the kernel as Hits (work[2] counts them) for the materialised
//     mode-L pipeline, which spreads them over the whole GPU -- and a hash set
//     in the warp's shared memory keeps the first occurrence of each pair, so
//     the item's distinct pairs come out without a sort (a pair (q, r), r < q,
//     is only found by probe q, hence only in q's item);
//   * the whole-string character-count screen and one whole-pair banded
//     verification per distinct pair (Sec. 5.1): 32 pairs at a time, a lane
//     per pair, the last partial batch carried into the warp's next item so
//     that lanes stay busy; or, for probes at least `warp_from` long, one pair
//     at a time by the whole warp.
// Warps never wait for one another, so one warp's lookups overlap another's
// verification.  A pair that finds its item's list full goes to the global
// overflow list as a pair key, verified afterwards by the materialised
// mode-L pipeline (ovf: FOVF_LISTS counters, then as many lists of ovf_cap
// keys); a pair verified twice is merged by the final dedupe (least ed per
// pair).  work[1] counts the distinct pairs verified here.
constexpr int FB = 256;          // 8 independent warps per block
constexpr int FSET_BITS = 9;
constexpr int FSET = 1 << FSET_BITS;  // pair slots of a warp's hash set
constexpr int FLIST = 224;       // distinct pairs one item keeps (the set stays under half full)
constexpr int FTASKS = 64;       // (probe, group) tasks per item at least
constexpr int FRUNS = 32;        // posting runs a warp expands together, per item
constexpr uint32_t FRUN_MIN = 8; // runs longer than this are expanded by the whole warp
constexpr uint32_t FRUN_BIG = 16;   // runs longer than this leave the kernel as Hits
constexpr unsigned long long FTAG_MAX = (1ull << 24) - 1;
constexpr int FOVF_LISTS = 64;   // overflow sub-lists (the item at j from the long end appends to list j mod 64)

// One warp's shared state.  A set slot holds tag << 40 | (q - first probe of
// the item) << 32 | r; slots whose tag is not the current item's are free.
struct FusedWarp {
  unsigned long long set[FSET];
  unsigned long long carry[32];  // (q << 32 | r) pairs waiting for a full batch
  unsigned long long runs[FRUNS];  // long posting runs: (q - first probe) << 56 | count << 32 | begin
  uint16_t list[FLIST];          // set slots of the item's distinct pairs, in insertion order
  int nlist, nruns;
};

__device__ __forceinline__ unsigned long long fused_overflow_key(uint32_t q, uint32_t r, int pshift) {
  return ((unsigned long long)min(q, r) << pshift) | max(q, r);
}

// Inserts candidate pair (q, r) of the current item; a new pair is listed,
// or sent to the overflow list when the item's list is full.
// ovf_n: the item's overflow sub-list counter; ovf_keys: its region of
// ovf_cap entries.
__device__ __forceinline__ void fused_insert(FusedWarp& w, unsigned long long tag, uint32_t qrel, uint32_t q,
                                             uint32_t r, int pshift, unsigned long long* __restrict__ ovf_n,
                                             unsigned long long* __restrict__ ovf_keys, unsigned long long ovf_cap) {
  volatile unsigned long long* set = w.set;
  if (*(volatile int*)&w.nlist < FLIST) {
    const unsigned long long val = (tag << 40) | ((unsigned long long)qrel << 32) | r;
    unsigned h = (r * 0x9E3779B1u + qrel * 0x85EBCA77u) >> (32 - FSET_BITS);
    for (int n = 0; n < 2 * FSET; ++n) {
      const unsigned long long cur = set[h];
      if (cur == val) return;  // seen before in this item
      if ((cur >> 40) != tag) {  // a free slot
        const unsigned long long prev = atomicCAS(&w.set[h], cur, val);
        if (prev == cur) {
          const int pos = atomicAdd(&w.nlist, 1);
          if (pos < FLIST) {
            w.list[pos] = (uint16_t)h;
            return;
          }
          break;  // listed nowhere: overflow (later copies are found in the set)
        }
        if (prev == val) return;
        continue;  // taken meanwhile: look at the slot again
      }
      h = (h + 1) & (FSET - 1);
    }
  }
  // one atomic per group of lanes that overflow together
  const cg::coalesced_group lanes = cg::coalesced_threads();
  unsigned long long o = 0;
  if (lanes.thread_rank() == 0) o = atomicAdd(ovf_n, (unsigned long long)lanes.size());
  o = lanes.shfl(o, 0) + lanes.thread_rank();
  if (o < ovf_cap) ovf_keys[o] = fused_overflow_key(q, r, pshift);
}

template <int MAXW>
__device__ __forceinline__ void fused_verify_thread(const ProbeView& v, uint32_t q, uint32_t r, const AccOut& out,
                                                    Counters* ctr, unsigned long long& cells,
                                                    unsigned long long& filtered) {
  if (v.pbm && signature_bound(v.pbm[q], v.ibm[r]) > v.tau) {
    ++filtered;
    return;
  }
  const int d = vsp<MAXW>(v.pbytes + v.poff[q], (int)v.plen[q], v.ibytes + v.ioff[r], (int)v.ilen[r], v.tau, cells);
  if (d <= v.tau) append_match(ctr, out, pair_out_key(v, true, q, r), d);
}

// FORM: FUSED_THREAD (every pair a lane), FUSED_WARP (every pair a warp) or
// FUSED_CUT (a warp per pair for probes at least warp_from long); the single
// forms leave the other verification out of the kernel and its registers.
enum { FUSED_THREAD = 0, FUSED_WARP = 1, FUSED_CUT = 2 };

template <int MAXW, int FORM>
__global__ void __launch_bounds__(FB) k_fused_self(const ProbeView v, int ppi, int warp_from,
                                                   unsigned long long* __restrict__ work,
                                                   unsigned long long* __restrict__ ovf, unsigned long long ovf_cap,
                                                   Hit* __restrict__ heavy, unsigned long long heavy_cap,
                                                   int pshift, AccOut out, Counters* ctr) {
  __shared__ FusedWarp fw[FB / 32];
  const unsigned lane = threadIdx.x & 31u;
  FusedWarp& w = fw[threadIdx.x >> 5];
  for (int k = (int)lane; k < FSET; k += 32) w.set[k] = 0;  // tag 0 is no item's
  const int G = groups_per_probe(v.tau, true);
  const unsigned long long n_items = ((unsigned long long)v.pcount + ppi - 1) / ppi;
  unsigned long long lookups = 0, cells = 0, wcells = 0, n_cand = 0, filtered = 0, pairs = 0;
  int err = 0;
  int ncarry = 0;                // the same in every lane
  unsigned long long tag = 0;    // the current item's tag, 1..FTAG_MAX
  for (;;) {
    unsigned long long it = 0;
    if (lane == 0) {
      it = atomicAdd(&work[0], 1ull);
      w.nlist = 0;
      w.nruns = 0;
    }
    it = __shfl_sync(FULL, it, 0);
    if (it >= n_items) break;
    if (++tag > FTAG_MAX) {  // tags wrapped: free every slot
      for (int k = (int)lane; k < FSET; k += 32) w.set[k] = 0;
      tag = 1;
    }
    __syncwarp();
    // items from both ends in turn: the longest probes (the costliest
    // verifications) and the shortest (the longest posting runs) start first
    uint32_t q_beg, q_end;
    const unsigned long long j = fused_item(it, n_items, v.pbegin, v.pcount, ppi, q_beg, q_end);
    const unsigned sub = (unsigned)(j % FOVF_LISTS);  // neighbouring items (alike in cost) on different lists
    unsigned long long* const ovf_n = ovf + sub;
    unsigned long long* const ovf_keys = ovf + FOVF_LISTS + sub * ovf_cap;
    const int nq = (int)(q_end - q_beg);
    auto group = [&](uint32_t qrel, int g) {
      const uint32_t q = q_beg + qrel;
      const int ls = (int)v.plen[q];
      int l, i, P, li, lo, hi;
      if (!group_window(v, true, q, ls, g, l, i, P, li, lo, hi)) return;
      window_lookups(v, true, q, ls, l, i, li, lo, hi, v.pbytes + v.poff[q], err, [&](int, uint32_t b, uint32_t cnt) {
        if (cnt > FRUN_BIG) {  // a very long run: to the materialised pipeline
          const cg::coalesced_group lanes = cg::coalesced_threads();
          unsigned long long hv = 0;
          if (lanes.thread_rank() == 0) hv = atomicAdd(&work[2], (unsigned long long)lanes.size());
          hv = lanes.shfl(hv, 0) + lanes.thread_rank();
          if (hv < heavy_cap) {
            heavy[hv] = Hit{q, b, cnt, 0u, 0ull, 0ull};
            n_cand += cnt;
            return;
          }
        }
        if (cnt > FRUN_MIN && cnt < (1u << 24)) {  // a long run: queued for the whole warp
          const int slot = atomicAdd(&w.nruns, 1);
          if (slot < FRUNS) {
            w.runs[slot] = ((unsigned long long)qrel << 56) | ((unsigned long long)cnt << 32) | b;
            n_cand += cnt;
            return;
          }
        }
        for (uint32_t k = 0; k < cnt; ++k) {
          const uint32_t r = v.postings[b + k];
          if (r >= v.n_index) {
            err |= 1;
            continue;
          }
          ++n_cand;
          fused_insert(w, tag, qrel, q, r, pshift, ovf_n, ovf_keys, ovf_cap);
        }
      });
      lookups += (unsigned long long)(hi - lo + 1);
    };
    if (v.interleave) {  // a lane per probe, the lanes on the same group g (windows of about one size)
      if ((int)lane < nq)
        for (int g = 0; g < G; ++g) group(lane, g);
    } else {  // the lanes on consecutive groups of a probe, widest windows first
      for (int t = (int)lane; t < nq * G; t += 32) {
        const int g = t % G;
        group((uint32_t)(t / G), v.gorder ? (int)v.gorder[g] : g);
      }
    }
    __syncwarp();
    const int nr = ::min(*(volatile int*)&w.nruns, FRUNS);
    for (int k = 0; k < nr; ++k) {  // the long runs, a posting per lane
      const unsigned long long run = w.runs[k];
      const uint32_t qrel = (uint32_t)(run >> 56), cnt = (uint32_t)(run >> 32) & 0xFFFFFFu, b = (uint32_t)run;
      for (uint32_t j = lane; j < cnt; j += 32) {
        const uint32_t r = v.postings[b + j];
        if (r >= v.n_index) {
          err |= 1;
          continue;
        }
        fused_insert(w, tag, qrel, q_beg + qrel, r, pshift, ovf_n, ovf_keys, ovf_cap);
      }
    }
    __syncwarp();
    const int nd = ::min(*(volatile int*)&w.nlist, FLIST);
    // pair k of the item's list
    auto listed = [&](int k, uint32_t& q, uint32_t& r) {
      const unsigned long long val = w.set[w.list[k]];
      q = q_beg + (uint32_t)((val >> 32) & 0xFFu);
      r = (uint32_t)val;
    };
    const bool by_warp = FORM == FUSED_WARP || (FORM == FUSED_CUT && (int)v.plen[q_end - 1] >= warp_from);
    if (by_warp) {  // a warp per pair
      if constexpr (FORM != FUSED_WARP) {
        if (ncarry) {  // pairs a lane per pair left from a shorter item
          if ((int)lane < ncarry) {
            ++pairs;
            fused_verify_thread<MAXW>(v, (uint32_t)(w.carry[lane] >> 32), (uint32_t)w.carry[lane], out, ctr, cells,
                                      filtered);
          }
          ncarry = 0;
          __syncwarp();
        }
      }
      for (int k = 0; k < nd; ++k) {
        uint32_t q, r;
        listed(k, q, r);
        if (lane == 0) ++pairs;
        if (v.pbm && signature_bound(v.pbm[q], v.ibm[r]) > v.tau) {  // the same in every lane
          if (lane == 0) ++filtered;
          continue;
        }
        const int d = vsp_warp(v.pbytes + v.poff[q], (int)v.plen[q], v.ibytes + v.ioff[r], (int)v.ilen[r], v.tau,
                               wcells);
        if (d <= v.tau && lane == 0) append_match(ctr, out, pair_out_key(v, true, q, r), d);
      }
    } else if constexpr (FORM != FUSED_WARP) {  // a lane per pair: carried pairs first, then the item's
      const int total = ncarry + nd;
      const int full = total & ~31;
      for (int base = 0; base < full; base += 32) {
        const int k = base + (int)lane;
        uint32_t q, r;
        if (k < ncarry) {
          q = (uint32_t)(w.carry[k] >> 32);
          r = (uint32_t)w.carry[k];
        } else {
          listed(k - ncarry, q, r);
        }
        ++pairs;
        fused_verify_thread<MAXW>(v, q, r, out, ctr, cells, filtered);
      }
      const int rem = total - full;
      unsigned long long cv = 0;
      if ((int)lane < rem) {
        const int k = full + (int)lane;
        if (k < ncarry) {
          cv = w.carry[k];
        } else {
          uint32_t q, r;
          listed(k - ncarry, q, r);
          cv = ((unsigned long long)q << 32) | r;
        }
      }
      __syncwarp();
      if ((int)lane < rem) w.carry[lane] = cv;
      ncarry = rem;
    }
    __syncwarp();  // the list, the set and the carry are rewritten by the next item
  }
  if constexpr (FORM != FUSED_WARP) {
    if ((int)lane < ncarry) {
      ++pairs;
      fused_verify_thread<MAXW>(v, (uint32_t)(w.carry[lane] >> 32), (uint32_t)w.carry[lane], out, ctr, cells,
                                filtered);
    }
  }
  add_counter(&ctr->lookups, lookups);
  add_counter(&ctr->candidates, n_cand);
  add_counter(&ctr->filtered, filtered);
  add_counter(&work[1], pairs);
  if (err) atomicOr(&ctr->err, (unsigned long long)err);
  // the warp form counts each pair's cells in all 32 lanes: lane 0 reports them
  add_counter(&ctr->cells, cells + (lane == 0 ? wcells : 0ull));
}

// ---------------------------------------------------------------- A8 ------

// Pairs whose indexed string is too short to partition (length <= tau).
// SELF: every short sid x against the sids y > x with |y| <= |x| + tau.
// Otherwise: every probe x against the indexed strings of length <= tau
// within the length filter.  One thread per x.
template <int MAXW, bool SELF, bool MULTI>
__global__ void __launch_bounds__(BLOCK) k_fallback(const ProbeView v, uint32_t xcount, AccOut out, Counters* ctr,
                                                    const unsigned long long* __restrict__ n_dev) {
  xcount = (uint32_t)dev_count(xcount, n_dev);
  unsigned long long cells = 0, pairs = 0;
  for (uint32_t x = blockIdx.x * BLOCK + threadIdx.x; x < xcount; x += gridDim.x * BLOCK) {
    const int tau = MULTI ? (int)v.ptau[x] : v.tau;
    const uint8_t* xs = v.pbytes + v.poff[x];
    const int lx = (int)v.plen[x];
    uint32_t y0, y1;
    if (SELF) {
      y0 = x + 1;
      y1 = v.ibbeg[min(lx + tau, v.ilmax) + 1];
    } else {
      const int llo = max(0, lx - tau);
      const int lhi = min(min(tau, lx + tau), v.ilmax);
      y0 = llo <= lhi ? v.ibbeg[llo] : 0u;
      y1 = llo <= lhi ? v.ibbeg[lhi + 1] : 0u;
    }
    const uint32_t qid = v.pid ? v.pid[x] : x;
    for (uint32_t y = y0; y < y1; ++y) {
      ++pairs;
      const int d = vsp<MAXW>(xs, lx, v.ibytes + v.ioff[y], (int)v.ilen[y], tau, cells);
      if (d <= tau) {
        const uint32_t rid = v.iperm[y];
        const uint32_t ka = SELF ? min(qid, rid) : qid;
        const uint32_t kb = SELF ? max(qid, rid) : rid;
        const unsigned long long pos = atomicAdd(&ctr->accepted, 1ull);
        if (pos < out.cap) {
          out.key[pos] = ((unsigned long long)ka << v.key_shift) | kb;
          out.ed[pos] = (uint32_t)d;
        }
      }
    }
  }
  if (cells) atomicAdd(&ctr->cells, cells);
  if (pairs) atomicAdd(&ctr->fallback, pairs);
}

// ------------------------------------------------------------ A5 + A7 -----

__global__ void k_run_heads(const unsigned long long* __restrict__ keys, unsigned long long n,
                            uint32_t* __restrict__ flags, const unsigned long long* __restrict__ n_dev) {
  n = dev_count(n, n_dev);
  for (unsigned long long k = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; k < n;
       k += (unsigned long long)gridDim.x * blockDim.x)
    flags[k] = (k == 0 || keys[k] != keys[k - 1]) ? 1u : 0u;
}

// Each run of equal keys becomes one pair with the run's least ed, written
// at the run's prefix-sum position (positions at or past out_cap are not
// written).
__global__ void k_emit_pairs(const unsigned long long* __restrict__ keys, const uint32_t* __restrict__ eds,
                             const uint32_t* __restrict__ flags, const uint32_t* __restrict__ pos,
                             unsigned long long n, int key_shift, pj_pair* __restrict__ out,
                             const unsigned long long* __restrict__ n_dev, unsigned long long out_cap) {
  n = dev_count(n, n_dev);
  for (unsigned long long k = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; k < n;
       k += (unsigned long long)gridDim.x * blockDim.x) {
    if (!flags[k] || pos[k] >= out_cap) continue;
    const unsigned long long key = keys[k];
    uint32_t ed = eds[k];
    for (unsigned long long j = k + 1; j < n && keys[j] == key; ++j) ed = min(ed, eds[j]);
    pj_pair pr;
    pr.a = (uint32_t)(key >> key_shift);
    pr.b = (uint32_t)(key & ((1ull << key_shift) - 1));
    pr.ed = ed;
    out[pos[k]] = pr;
  }
}

// The packed form of the accepted matches for the final sort: the pair key
// with ed in its top 6 bits (pair keys of at most PACKED_KEY_BITS bits,
// ed <= tau <= 32).  Runs are then told apart by the low bits, and each
// run's least ed is the least top field.
constexpr int PACKED_KEY_BITS = 58;

__global__ void k_pack_ed(unsigned long long* __restrict__ keys, const uint32_t* __restrict__ eds,
                          unsigned long long n) {
  for (unsigned long long k = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; k < n;
       k += (unsigned long long)gridDim.x * blockDim.x)
    keys[k] |= (unsigned long long)eds[k] << PACKED_KEY_BITS;
}

__global__ void k_run_heads_masked(const unsigned long long* __restrict__ keys, unsigned long long n,
                                   unsigned long long mask, uint32_t* __restrict__ flags) {
  for (unsigned long long k = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; k < n;
       k += (unsigned long long)gridDim.x * blockDim.x)
    flags[k] = (k == 0 || ((keys[k] ^ keys[k - 1]) & mask) != 0) ? 1u : 0u;
}

__global__ void k_emit_packed(const unsigned long long* __restrict__ keys, const uint32_t* __restrict__ flags,
                              const uint32_t* __restrict__ pos, unsigned long long n, int key_shift,
                              pj_pair* __restrict__ out, unsigned long long out_cap) {
  constexpr unsigned long long M = (1ull << PACKED_KEY_BITS) - 1;
  for (unsigned long long k = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; k < n;
       k += (unsigned long long)gridDim.x * blockDim.x) {
    if (!flags[k] || pos[k] >= out_cap) continue;
    const unsigned long long key = keys[k] & M;
    uint32_t ed = (uint32_t)(keys[k] >> PACKED_KEY_BITS);
    for (unsigned long long j = k + 1; j < n && (keys[j] & M) == key; ++j)
      ed = min(ed, (uint32_t)(keys[j] >> PACKED_KEY_BITS));
    pj_pair pr;
    pr.a = (uint32_t)(key >> key_shift);
    pr.b = (uint32_t)(key & ((1ull << key_shift) - 1));
    pr.ed = ed;
    out[pos[k]] = pr;
  }
}

// ------------------------------------------------------------- launch -----

// Grid for grid-stride loops over `cap` items, 256 threads a block: one wave
// of at most 8 blocks per SM.
static unsigned stride_grid(unsigned long long cap) {
  return (unsigned)std::max<unsigned long long>(1, std::min<unsigned long long>((cap + 255) / 256, sm_grid_cap(8)));
}

template <class K>
static unsigned persistent_grid(K kernel, unsigned long long work_blocks, int block = BLOCK) {
  int bps = 0;
  PJ_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, kernel, block, 0));
  const unsigned long long full = (unsigned long long)std::max(1, bps) * sm_count();
  return (unsigned)std::max<unsigned long long>(1, std::min(full, work_blocks));
}

template <int MAXW, bool SELF, bool MULTI>
static void launch_verify(const Ctx& c, const ProbeView& v, const Hit* hits, const unsigned long long* off,
                          unsigned long long n_hits, unsigned long long c_begin, unsigned long long c_end,
                          AccOut out, Counters* ctr, int block) {
  if (v.queued) {
    const unsigned gq = persistent_grid(k_verify_queued<MAXW, SELF, MULTI>,
                                        (c_end - c_begin + (unsigned long long)Q_BLOCK * S_RUN - 1) /
                                            ((unsigned long long)Q_BLOCK * S_RUN), Q_BLOCK);
    k_verify_queued<MAXW, SELF, MULTI><<<gq, Q_BLOCK, 0, c.stream>>>(v, hits, off, n_hits, c_begin, c_end, out, ctr,
                                                                    nullptr, queued_chunk(c_end - c_begin, gq));
    PJ_LAUNCHED("k_verify_queued");
    return;
  }
  const unsigned grid = persistent_grid(k_verify_hits<MAXW, SELF, MULTI>,
                                        (c_end - c_begin + (unsigned long long)block * V_RUN - 1) /
                                            ((unsigned long long)block * V_RUN), block);
  // lanes past c_end in the last warp span are skipped inside the kernel
  k_verify_hits<MAXW, SELF, MULTI><<<grid, block, 0, c.stream>>>(v, hits, off, n_hits, c_begin, c_end, out, ctr,
                                                                  nullptr);
  PJ_LAUNCHED("k_verify_hits");
}

template <bool SELF, bool MULTI>
static void launch_verify_warp(const Ctx& c, const ProbeView& v, const Hit* hits, const unsigned long long* off,
                               unsigned long long n_hits, unsigned long long c_begin, unsigned long long c_end,
                               AccOut out, Counters* ctr, int block) {
  const unsigned grid = persistent_grid(k_verify_warp<SELF, MULTI>,
                                        (c_end - c_begin + (block / 32) - 1) / (block / 32), block);
  k_verify_warp<SELF, MULTI><<<grid, block, 0, c.stream>>>(v, hits, off, n_hits, c_begin, c_end, out, ctr);
  PJ_LAUNCHED("k_verify_warp");
}

template <int MAXW, bool SELF, bool MULTI>
static void launch_fallback(const Ctx& c, const ProbeView& v, uint32_t xcount, AccOut out, Counters* ctr) {
  const unsigned grid = persistent_grid(k_fallback<MAXW, SELF, MULTI>, (xcount + BLOCK - 1) / BLOCK);
  k_fallback<MAXW, SELF, MULTI><<<grid, BLOCK, 0, c.stream>>>(v, xcount, out, ctr, nullptr);
  PJ_LAUNCHED("k_fallback");
}

#define PJ_BY_TAU(tau, CALL)          \
  do {                                \
    const int t_ = (tau);             \
    if (t_ <= 1) { CALL(2); }         \
    else if (t_ <= 2) { CALL(3); }    \
    else if (t_ <= 4) { CALL(5); }    \
    else if (t_ <= 8) { CALL(9); }    \
    else if (t_ <= 16) { CALL(17); }  \
    else { CALL(33); }                \
  } while (0)

struct ResultPriv {
  Ctx ctx;
  size_t pinned_bytes = 0;  // host pairs in a block of the pinned pool (0: malloc)
};

// Host blocks for host results, reused across calls: page-locked and mapped
// into the device's address space (cudaHostAlloc), so that the last kernel
// of a join writes the pairs straight into host memory instead of a device
// buffer followed by a copy.  Page-locking a large block is slow, hence the
// reuse.  PJ_HOST_POOL=pageable keeps plain malloc blocks instead (written
// by a copy from the device).  pj_result_free hands blocks back; at most
// PINNED_POOL_KEEP bytes stay cached, larger blocks are released.
constexpr size_t PINNED_POOL_KEEP = 8ull << 30;
constexpr size_t PINNED_MIN = 1ull << 20;  // smaller results use malloc

static std::mutex g_pinned_mu;
static std::multimap<size_t, void*> g_pinned_free;  // size -> block
static size_t g_pinned_cached = 0;

static bool pool_pinned() {
  static const bool on = [] {
    const char* e = getenv("PJ_HOST_POOL");
    return !(e && strcmp(e, "pageable") == 0);
  }();
  return on;
}

static void pool_release(void* p) {
  if (pool_pinned()) cudaFreeHost(p);
  else free(p);
}

static void* pinned_get(size_t bytes, size_t* got) {
  {
    std::lock_guard<std::mutex> g(g_pinned_mu);
    auto it = g_pinned_free.lower_bound(bytes);
    if (it != g_pinned_free.end() && it->first <= 2 * bytes) {  // reuse a block at most twice as large
      *got = it->first;
      void* p = it->second;
      g_pinned_cached -= it->first;
      g_pinned_free.erase(it);
      return p;
    }
  }
  void* p = nullptr;
  if (pool_pinned()) {
    if (cudaHostAlloc(&p, bytes, cudaHostAllocMapped) != cudaSuccess) {
      cudaGetLastError();
      return nullptr;
    }
  } else {
    p = malloc(bytes);
    if (!p) return nullptr;
  }
  *got = bytes;
  return p;
}

static void pinned_put(void* p, size_t bytes) {
  std::lock_guard<std::mutex> g(g_pinned_mu);
  while (g_pinned_cached + bytes > PINNED_POOL_KEEP && !g_pinned_free.empty()) {  // evict the smallest
    auto it = g_pinned_free.begin();
    pool_release(it->second);
    g_pinned_cached -= it->first;
    g_pinned_free.erase(it);
  }
  if (g_pinned_cached + bytes > PINNED_POOL_KEEP) {
    pool_release(p);
    return;
  }
  g_pinned_free.emplace(bytes, p);
  g_pinned_cached += bytes;
}

// Sizing knobs, overridable through the environment (used by tests to drive
// the chunked and growing paths at small sizes):
//   PJ_GROUP_BUDGET      groups probed per chunk          (default 64 Mi)
//   PJ_LAUNCH_CANDS      candidates per verification launch (default 1 Gi)
//   PJ_ACCEPT_INITIAL    initial accepted-match capacity  (default 4 Mi)
//   PJ_GRAPH_MAX_GROUPS  groups of a recorded self join   (default 256 Mi)
//   PJ_GRAPH_TIGHT       1: record self joins with half their counts as
//                        capacities, so that every replay overflows
static unsigned long long env_knob(const char* name, unsigned long long dflt) {
  const char* e = getenv(name);
  if (!e || !e[0]) return dflt;
  const unsigned long long v = strtoull(e, nullptr, 10);
  return v ? v : dflt;
}

struct Timings {
  float probe = 0.f, verify = 0.f, fallback = 0.f, dedupe = 0.f;
  unsigned long long distinct = 0;  // mode L: distinct pairs verified
};

// Accepted-match buffer that grows between launches: after a launch that
// overflowed it, the buffer is enlarged (keeping the entries accepted before
// that launch), the counter is wound back and the launch runs again.
struct AcceptBuf {
  const Ctx& c;
  Counters* ctr;
  DBuf<unsigned long long> key;
  DBuf<uint32_t> ed;
  unsigned long long cap = 0;
  unsigned long long last = 0;  // accepted count after the last run()
  AcceptBuf(const Ctx& ctx, Counters* counters, unsigned long long initial) : c(ctx), ctr(counters) {
    key.reset(c, initial);
    ed.reset(c, initial);
    cap = initial;
  }
  AccOut out() const { return AccOut{key.p, ed.p, cap}; }
  unsigned long long read_count() const {
    unsigned long long n = 0;
    PJ_CUDA(cudaMemcpyAsync(&n, &ctr->accepted, sizeof(n), cudaMemcpyDeviceToHost, c.stream));
    c.sync();
    return n;
  }
  // Runs `launch` (which appends to out()); retries once after growing to
  // `want(after)` entries if the buffer overflowed.
  template <class Launch, class Want>
  void run(Launch launch, Want want) {
    Counters saved{};  // all counters, so that a re-run launch is counted once
    PJ_CUDA(cudaMemcpyAsync(&saved, ctr, sizeof(saved), cudaMemcpyDeviceToHost, c.stream));
    c.sync();
    const unsigned long long before = saved.accepted;
    launch(out());
    const unsigned long long after = read_count();
    last = after;
    if (after <= cap) return;
    grow(std::max<unsigned long long>(after, want(after)), before);
    PJ_CUDA(cudaMemcpyAsync(ctr, &saved, sizeof(saved), cudaMemcpyHostToDevice, c.stream));
    c.sync();  // `saved` lives on this stack frame
    launch(out());
    last = read_count();
    if (last > cap) fail(PJ_ECUDA, "accepted-match buffer overflowed after growing");
  }
  // Grows (keeping the entries so far) to hold `need` entries, before a
  // launch that would otherwise overflow and run twice.
  void reserve(unsigned long long need) {
    if (need > cap) grow(need, std::min(last, cap));
  }
  void grow(unsigned long long new_cap, unsigned long long keep) {
    DBuf<unsigned long long> k2(c, new_cap);
    DBuf<uint32_t> e2(c, new_cap);
    if (keep) {
      PJ_CUDA(cudaMemcpyAsync(k2.p, key.p, keep * sizeof(unsigned long long), cudaMemcpyDeviceToDevice, c.stream));
      PJ_CUDA(cudaMemcpyAsync(e2.p, ed.p, keep * sizeof(uint32_t), cudaMemcpyDeviceToDevice, c.stream));
    }
    key = std::move(k2);
    ed = std::move(e2);
    cap = new_cap;
  }
};

// Probe + verify for all probing strings, in chunks of probing strings whose
// groups fit the hit buffer; then the short-string fallback.  Returns the
// number of accepted matches (the buffer holds min(that, out.cap)).
// Probe one chunk of probing strings: per-group hit counts, their prefix
// sum, the hits, and the candidate offsets of the hits (n_hits + 1 entries).
template <bool SELF, bool MULTI>
static void probe_chunk(const Ctx& c, const ProbeView& v, unsigned long long n_groups, Counters* ctr,
                        DBuf<uint32_t>& gcount, DBuf<uint32_t>& goff, DBuf<Hit>& hits, DBuf<unsigned long long>& cnt,
                        DBuf<unsigned long long>& off, unsigned long long& n_hits, unsigned long long& n_cand) {
  gcount.reset(c, n_groups);
  goff.reset(c, n_groups);
  DBuf<unsigned long long> gmask(c, n_groups);
  const unsigned g1 = persistent_grid(k_group_counts<SELF, MULTI>, (n_groups + BLOCK - 1) / BLOCK);
  k_group_counts<SELF, MULTI><<<g1, BLOCK, 0, c.stream>>>(v, n_groups, gcount.p, gmask.p, ctr, nullptr);
  PJ_LAUNCHED("k_group_counts");
  exclusive_scan<uint32_t>(c, gcount.p, goff.p, n_groups);
  uint32_t last[2] = {0, 0};
  PJ_CUDA(cudaMemcpyAsync(&last[0], goff.p + n_groups - 1, sizeof(uint32_t), cudaMemcpyDeviceToHost, c.stream));
  PJ_CUDA(cudaMemcpyAsync(&last[1], gcount.p + n_groups - 1, sizeof(uint32_t), cudaMemcpyDeviceToHost, c.stream));
  c.sync();
  n_hits = (unsigned long long)last[0] + last[1];
  n_cand = 0;
  if (n_hits == 0) return;
  hits.reset(c, n_hits);
  const unsigned g2 = persistent_grid(k_group_hits<SELF, MULTI>, (n_groups + BLOCK - 1) / BLOCK);
  k_group_hits<SELF, MULTI><<<g2, BLOCK, 0, c.stream>>>(v, n_groups, gcount.p, gmask.p, goff.p, hits.p, nullptr,
                                                        n_hits);
  PJ_LAUNCHED("k_group_hits");
  trace_mark(c, "join: probe (hits)");
  cnt.reset(c, n_hits + 1);
  off.reset(c, n_hits + 1);
  PJ_CUDA(cudaMemsetAsync(cnt.p + n_hits, 0, sizeof(unsigned long long), c.stream));
  k_hit_counts<<<ceil_div(n_hits, 256), 256, 0, c.stream>>>(hits.p, n_hits, cnt.p, nullptr);
  PJ_LAUNCHED("k_hit_counts");
  exclusive_scan<unsigned long long>(c, cnt.p, off.p, n_hits + 1);
  PJ_CUDA(cudaMemcpyAsync(&n_cand, off.p + n_hits, sizeof(n_cand), cudaMemcpyDeviceToHost, c.stream));
  c.sync();
}

// The warp cut-over probe rounded up to the chunk's next probe-block boundary
// (hits are ordered by probe block; both verification forms give the same
// results, so moving the cut by a few probes changes nothing but speed).
static uint32_t aligned_cut(const ProbeView& v, uint32_t q_cut) {
  if (q_cut <= v.pbegin) return v.pbegin;
  const unsigned long long k = ((unsigned long long)(q_cut - v.pbegin) + PROBE_BLOCK - 1) / PROBE_BLOCK;
  return (uint32_t)std::min<unsigned long long>(UINT32_MAX, v.pbegin + k * PROBE_BLOCK);
}

// Index of the first candidate whose probe id is >= q (hits ordered by probe
// block, q at a block boundary).
static unsigned long long first_candidate_of(const Ctx& c, const DBuf<Hit>& hits, const DBuf<unsigned long long>& off,
                                             unsigned long long n_hits, unsigned long long n_cand, uint32_t q) {
  DBuf<unsigned long long> hcut(c, 1);
  k_hit_lower_bound<<<1, 1, 0, c.stream>>>(hits.p, n_hits, q, hcut.p);
  PJ_LAUNCHED("k_hit_lower_bound");
  unsigned long long h_cut = 0, c_cut = n_cand;
  PJ_CUDA(cudaMemcpyAsync(&h_cut, hcut.p, sizeof(h_cut), cudaMemcpyDeviceToHost, c.stream));
  c.sync();
  if (h_cut < n_hits) {
    PJ_CUDA(cudaMemcpyAsync(&c_cut, off.p + h_cut, sizeof(c_cut), cudaMemcpyDeviceToHost, c.stream));
    c.sync();
  }
  return c_cut;
}

// Candidates above which extension verification starts with a short launch
// that measures the acceptance rate (measured on the short workload: without
// it, 3.8e9 / 2.9e8 / 5.8e6 candidates took 2–18% less time; 2.2e10 took 1.2%
// more, its costliest candidates -- the shortest probes' -- then sharing the
// long launch's larger chunks).
constexpr unsigned long long SIZING_MIN_CANDS = 1ull << 33;

// Largest number of candidates of one chunk verified in mode L (32 B of
// scratch per candidate); bigger chunks use extension verification.
constexpr unsigned long long PAIR_MODE_MAX_CANDS = 1ull << 27;

// Mode L from a list of n_keys candidate pair keys (in k0, unsorted, k0 of
// n_keys entries): radix sort, distinct pairs, one whole-string
// verification each.  Returns the number of distinct pairs.
template <bool SELF>
static unsigned long long verify_pair_keys(const Ctx& c, const ProbeView& v, DBuf<unsigned long long>& k0,
                                           unsigned long long n_cand, Counters* ctr, AccOut* scratch,
                                           AcceptBuf* acc) {
  const int pshift = bits_for(v.n_index);
  const int nbits = pshift + (SELF ? pshift : bits_for((unsigned long long)v.pbegin + v.pcount));
  DBuf<unsigned long long> k1(c, n_cand);
  DBuf<uint32_t> v0(c, n_cand), v1(c, n_cand);
  const bool second = radix_sort_pairs_dn<unsigned long long>(c, k0.p, v0.p, k1.p, v1.p, n_cand, nullptr, nbits);
  unsigned long long* sorted = second ? k1.p : k0.p;
  unsigned long long* ukeys = second ? k0.p : k1.p;
  DBuf<uint32_t> flags(c, n_cand), pos(c, n_cand);
  DBuf<unsigned long long> n_unique(c, 1);
  k_run_heads<<<stride_grid(n_cand), 256, 0, c.stream>>>(sorted, n_cand, flags.p, nullptr);
  PJ_LAUNCHED("k_run_heads");
  exclusive_scan_dn<uint32_t>(c, flags.p, pos.p, n_cand, nullptr, n_unique.p);
  k_unique_keys<<<stride_grid(n_cand), 256, 0, c.stream>>>(sorted, flags.p, pos.p, n_cand, ukeys, nullptr);
  PJ_LAUNCHED("k_unique_keys");
  unsigned long long U = 0;
  PJ_CUDA(cudaMemcpyAsync(&U, n_unique.p, sizeof(U), cudaMemcpyDeviceToHost, c.stream));
  c.sync();
  auto launch = [&](AccOut o) {
    if (v.pair_warp) {
      const unsigned gw = persistent_grid(k_verify_pairs_warp<SELF>, (U + BLOCK / 32 - 1) / (BLOCK / 32));
      k_verify_pairs_warp<SELF><<<gw, BLOCK, 0, c.stream>>>(v, ukeys, U, pshift, o, ctr, nullptr);
      PJ_LAUNCHED("k_verify_pairs_warp");
    } else {
#define PJ_CALL(W)                                                                                    \
  do {                                                                                               \
    const unsigned gt = persistent_grid(k_verify_pairs<W, SELF>, (U + BLOCK - 1) / BLOCK);           \
    k_verify_pairs<W, SELF><<<gt, BLOCK, 0, c.stream>>>(v, ukeys, U, pshift, o, ctr, nullptr);        \
    PJ_LAUNCHED("k_verify_pairs");                                                                   \
  } while (0)
      PJ_BY_TAU(v.tau, PJ_CALL);
#undef PJ_CALL
    }
  };
  if (acc) acc->run(launch, [&](unsigned long long after) { return 2 * after; });
  else launch(*scratch);
  return U;
}

// Mode L for one chunk's candidates [0, n_cand): pair keys, then
// verify_pair_keys.  Returns the number of distinct pairs.
template <bool SELF>
static unsigned long long verify_pairs_chunk(const Ctx& c, const ProbeView& v, const Hit* hits,
                                             const unsigned long long* off, unsigned long long n_hits,
                                             unsigned long long n_cand, Counters* ctr, AccOut* scratch,
                                             AcceptBuf* acc) {
  const int pshift = bits_for(v.n_index);
  DBuf<unsigned long long> k0(c, n_cand);
  const unsigned g = persistent_grid(k_pair_keys<SELF>, (n_cand + (unsigned long long)BLOCK * V_RUN - 1) /
                                                            ((unsigned long long)BLOCK * V_RUN));
  k_pair_keys<SELF><<<g, BLOCK, 0, c.stream>>>(v, hits, off, n_hits, 0, n_cand, pshift, k0.p, ctr, nullptr);
  PJ_LAUNCHED("k_pair_keys");
  return verify_pair_keys<SELF>(c, v, k0, n_cand, ctr, scratch, acc);
}

// Candidate pairs the fused kernel can send to one overflow sub-list; a join
// with more falls back to the chunked pipeline.
constexpr unsigned long long FUSED_OVF_CAP = 1ull << 20;

// The overflow sub-lists, one after another: list k (n[k] keys at
// src + k * cap) to dst + start[k], a block per list.
__global__ void k_gather_lists(const unsigned long long* __restrict__ src, const unsigned long long* __restrict__ n,
                               const unsigned long long* __restrict__ start, unsigned long long cap,
                               unsigned long long* __restrict__ dst) {
  const unsigned k = blockIdx.x;
  const unsigned long long m = min(n[k], cap);
  for (unsigned long long i = threadIdx.x; i < m; i += blockDim.x) dst[start[k] + i] = src[k * cap + i];
}

// Probes per work item of the fused kernel: a lane per probe when groups are
// interleaved, else at least FTASKS groups for a warp.
static int fused_ppi(const ProbeView& v) {
  return v.interleave ? 32 : std::max(1, FTASKS / groups_per_probe(v.tau, true));
}

// The fused kernel's verification form for v's probes (the lengths of its
// shortest and longest probe against fused_warp_from).
static int fused_form_of(const Ctx& c, const ProbeView& v) {
  uint32_t lens[2] = {0, 0};
  PJ_CUDA(cudaMemcpyAsync(&lens[0], v.plen + v.pbegin, sizeof(uint32_t), cudaMemcpyDeviceToHost, c.stream));
  PJ_CUDA(cudaMemcpyAsync(&lens[1], v.plen + v.pbegin + v.pcount - 1, sizeof(uint32_t), cudaMemcpyDeviceToHost,
                          c.stream));
  c.sync();
  return v.fused_warp_from <= (int)lens[0] ? FUSED_WARP : v.fused_warp_from > (int)lens[1] ? FUSED_THREAD : FUSED_CUT;
}

// Capacities of the fused kernel's lists for v's probes: keys per overflow
// sub-list, long runs.
static unsigned long long fused_ovf_cap(const ProbeView& v) {
  return std::min<unsigned long long>(FUSED_OVF_CAP,
                                      std::max<unsigned long long>(1 << 12, 16ull * v.pcount / FOVF_LISTS));
}
static unsigned long long fused_heavy_cap(const ProbeView& v) {
  return std::max<unsigned long long>(1 << 16, v.pcount);
}

// The fused self join (k_fused_self) over all of v's probes, then mode L over
// the overflow list, appending to acc.  False (nothing appended) when the
// overflow list would not hold the overflow: the caller runs the chunked
// pipeline instead.
static bool fused_self_join(const Ctx& c, const ProbeView& v, AcceptBuf& acc, Counters* ctr, Timings& tm) {
  EventTimer tv(c.stream);
  tv.start();
  const int pshift = bits_for(v.n_index);
  const int ppi = fused_ppi(v);
  const int form = fused_form_of(c, v);
  const unsigned long long n_items = ((unsigned long long)v.pcount + ppi - 1) / ppi;
  const unsigned long long ovf_cap = fused_ovf_cap(v);
  const unsigned long long heavy_cap = fused_heavy_cap(v);
  DBuf<unsigned long long> work, ovf;
  DBuf<Hit> heavy;
  try {  // lists the device (or its budget) cannot hold: the chunked pipeline instead
    work.reset(c, 3);
    ovf.reset(c, FOVF_LISTS + FOVF_LISTS * ovf_cap);
    heavy.reset(c, heavy_cap);
  } catch (const Error& e) {
    if (e.code != PJ_ENOMEM) throw;
    return false;
  }
  Counters saved{};
  PJ_CUDA(cudaMemcpyAsync(&saved, ctr, sizeof(saved), cudaMemcpyDeviceToHost, c.stream));
  c.sync();
  EventTimer tk(c.stream);  // the kernel alone (PJ_TRACE)
  acc.run(
      [&](AccOut o) {
        tk.start();
        PJ_CUDA(cudaMemsetAsync(work.p, 0, 3 * sizeof(unsigned long long), c.stream));
        PJ_CUDA(cudaMemsetAsync(ovf.p, 0, FOVF_LISTS * sizeof(unsigned long long), c.stream));
#define PJ_FORM(W, F)                                                                                          \
  do {                                                                                                        \
    const unsigned g = persistent_grid(k_fused_self<W, F>, n_items, FB);                                      \
    k_fused_self<W, F><<<g, FB, 0, c.stream>>>(v, ppi, v.fused_warp_from, work.p, ovf.p, ovf_cap, heavy.p,      \
                                               heavy_cap, pshift, o, ctr);                                    \
    PJ_LAUNCHED("k_fused_self");                                                                              \
  } while (0)
#define PJ_CALL(W)                               \
  do {                                           \
    if (form == FUSED_THREAD) PJ_FORM(W, FUSED_THREAD); \
    else if (form == FUSED_WARP) PJ_FORM(W, FUSED_WARP); \
    else PJ_FORM(W, FUSED_CUT);                  \
  } while (0)
        PJ_BY_TAU(v.tau, PJ_CALL);
#undef PJ_CALL
#undef PJ_FORM
        tk.stop();
      },
      [&](unsigned long long after) { return 2 * after; });
  unsigned long long n_work[3] = {0, 0, 0}, n_sub[FOVF_LISTS], start[FOVF_LISTS];
  PJ_CUDA(cudaMemcpyAsync(n_sub, ovf.p, sizeof(n_sub), cudaMemcpyDeviceToHost, c.stream));
  PJ_CUDA(cudaMemcpyAsync(n_work, work.p, sizeof(n_work), cudaMemcpyDeviceToHost, c.stream));
  c.sync();
  unsigned long long n_ovf = 0, sub_max = 0;
  for (int k = 0; k < FOVF_LISTS; ++k) {
    start[k] = n_ovf;
    n_ovf += n_sub[k];
    sub_max = std::max(sub_max, n_sub[k]);
  }
  const unsigned long long n_heavy = n_work[2];
  // the long runs' candidates: offsets of the Hits' runs
  DBuf<unsigned long long> cnt, off;
  unsigned long long n_hcand = 0;
  if (n_heavy && n_heavy <= heavy_cap) {
    cnt.reset(c, n_heavy + 1);
    off.reset(c, n_heavy + 1);
    PJ_CUDA(cudaMemsetAsync(cnt.p + n_heavy, 0, sizeof(unsigned long long), c.stream));
    k_hit_counts<<<ceil_div(n_heavy, 256), 256, 0, c.stream>>>(heavy.p, n_heavy, cnt.p, nullptr);
    PJ_LAUNCHED("k_hit_counts");
    exclusive_scan<unsigned long long>(c, cnt.p, off.p, n_heavy + 1);
    PJ_CUDA(cudaMemcpyAsync(&n_hcand, off.p + n_heavy, sizeof(n_hcand), cudaMemcpyDeviceToHost, c.stream));
    c.sync();
  }
  if (getenv("PJ_TRACE"))
    fprintf(stderr,
            "[pj] fused: probes from %u, %llu items of %d probes, kernel %.3f ms, %llu distinct pairs in-kernel, "
            "%llu to the overflow list, %llu long runs (%llu candidates)\n",
            v.pbegin, n_items, ppi, tk.ms(), n_work[1], n_ovf, n_heavy, n_hcand);
  if (sub_max > ovf_cap || n_heavy > heavy_cap || n_ovf + n_hcand > PAIR_MODE_MAX_CANDS) {
    // wind the counters back: the chunked pipeline redoes the join
    PJ_CUDA(cudaMemcpyAsync(ctr, &saved, sizeof(saved), cudaMemcpyHostToDevice, c.stream));
    c.sync();
    return false;
  }
  tm.distinct += n_work[1];
  if (n_ovf + n_hcand) {  // mode L over the long runs' candidates and the overflow list
    DBuf<unsigned long long> keys(c, n_hcand + n_ovf);
    if (n_hcand) {
      const unsigned g = persistent_grid(k_pair_keys<true>, (n_hcand + (unsigned long long)BLOCK * V_RUN - 1) /
                                                                ((unsigned long long)BLOCK * V_RUN));
      k_pair_keys<true><<<g, BLOCK, 0, c.stream>>>(v, heavy.p, off.p, n_heavy, 0, n_hcand, pshift, keys.p, ctr,
                                                   nullptr);
      PJ_LAUNCHED("k_pair_keys");
    }
    if (n_ovf) {
      DBuf<unsigned long long> dstart(c, FOVF_LISTS);
      PJ_CUDA(cudaMemcpyAsync(dstart.p, start, sizeof(start), cudaMemcpyHostToDevice, c.stream));
      k_gather_lists<<<FOVF_LISTS, 256, 0, c.stream>>>(ovf.p + FOVF_LISTS, ovf.p, dstart.p, ovf_cap,
                                                       keys.p + n_hcand);
      PJ_LAUNCHED("k_gather_lists");
      c.sync();  // `start` lives on this stack frame
    }
    ProbeView vp = v;
    vp.pair_warp = v.fused_warp_from == 0;
    tm.distinct += verify_pair_keys<true>(c, vp, keys, n_hcand + n_ovf, ctr, nullptr, &acc);
  }
  tv.stop();
  tm.verify += tv.ms();
  trace_mark(c, "join: fused select + probe + verify");
  return true;
}

template <bool SELF, bool MULTI>
static void probe_and_verify(const Ctx& c, const ProbeView& v0, uint32_t fb_count, AcceptBuf& acc, Counters* ctr,
                             Counters& h, Timings& tm, const unsigned long long* h_qgoff) {
  EventTimer tp(c.stream), tv(c.stream), tf(c.stream);
  const int G = MULTI ? 1 : groups_per_probe(v0.tau, SELF);
  const unsigned long long group_budget = std::min(env_knob("PJ_GROUP_BUDGET", 64ull << 20), 1ull << 31);
  // candidates per verification launch after the first: one launch unless
  // PJ_LAUNCH_CANDS asks for more (the accepted-match buffer is sized before
  // each launch from the rate so far, so launches rarely run twice)
  const unsigned long long launch_cands = env_knob("PJ_LAUNCH_CANDS", 1ull << 40);
  const uint32_t chunk_items = (uint32_t)std::max<unsigned long long>(1, group_budget / G);
  DBuf<Hit> hits;
  DBuf<uint32_t> gcount, goff;
  DBuf<unsigned long long> cnt, off;
  unsigned long long total_cand = 0, verified = 0;
  bool fused_done = false;
  ProbeView vc = v0;  // the probes of the chunked pipeline
  if (SELF && !MULTI && v0.fused && v0.pcount) {  // the fused persistent kernel over the probes from fused_q_cut
    const uint32_t end = v0.pbegin + v0.pcount;
    const uint32_t qf = std::min(end, std::max(v0.pbegin, v0.fused_q_cut));
    ProbeView vf = v0;
    vf.pbegin = qf;
    vf.pcount = end - qf;
    fused_done = vf.pcount > 0 && fused_self_join(c, vf, acc, ctr, tm);
    if (fused_done) vc.pcount = qf - v0.pbegin;
  }
  for (uint32_t done = 0; done < vc.pcount;) {
    ProbeView v = vc;
    v.pbegin = vc.pbegin + done;
    v.pcount = std::min(chunk_items, vc.pcount - done);
    unsigned long long n_groups =
        (MULTI || !v.interleave) ? (unsigned long long)v.pcount * G : interleaved_groups(v.pcount, G);
    if (MULTI) {  // probes whose groups fit the budget (at least one)
      uint32_t q1 = v.pbegin + 1;
      while (q1 < vc.pbegin + vc.pcount && h_qgoff[q1 + 1] - h_qgoff[v.pbegin] <= group_budget) ++q1;
      v.pcount = q1 - v.pbegin;
      n_groups = h_qgoff[q1] - h_qgoff[v.pbegin];
      if (n_groups == 0) {
        done += v.pcount;
        continue;
      }
    }
    tp.start();
    unsigned long long n_hits = 0, n_cand = 0;
    probe_chunk<SELF, MULTI>(c, v, n_groups, ctr, gcount, goff, hits, cnt, off, n_hits, n_cand);
    if (n_hits == 0) {
      tp.stop();
      tm.probe += tp.ms();
      done += v.pcount;
      continue;
    }
    tp.stop();
    tm.probe += tp.ms();
    debug_dump(c, "hits", hits.p, n_hits * sizeof(Hit));
    debug_dump(c, "cand_off", off.p, (n_hits + 1) * sizeof(unsigned long long));
    h.candidates += n_cand;
    h.hits += n_hits;
    total_cand += n_cand;
    const double remaining_groups = (double)(vc.pcount - done - v.pcount) / std::max(1u, v.pcount) + 1.0;  // chunks left
    if (!MULTI && v.pair_mode && n_cand <= PAIR_MODE_MAX_CANDS) {  // mode L
      tv.start();
      tm.distinct += verify_pairs_chunk<SELF>(c, v, hits.p, off.p, n_hits, n_cand, ctr, nullptr, &acc);
      tv.stop();
      tm.verify += tv.ms();
      verified += n_cand;
      trace_mark(c, "join: verify (distinct pairs)");
      done += v.pcount;
      continue;
    }
    // Joins of up to SIZING_MIN_CANDS candidates verify in one launch with
    // room for 1/16 of them accepted; bigger ones first verify 1/64 of their
    // candidates in a short launch, whose acceptance rate sizes the buffer
    // for the rest (an overflowed launch would run again).
    const bool sizing = n_cand > SIZING_MIN_CANDS;
    if (verified == 0 && env_knob("PJ_ACCEPT_RESERVE", 1)) {  // PJ_ACCEPT_RESERVE=0: grow on overflow only (tests)
      // the room is allocated before the first launch: growing the buffer
      // between launches measured slower than the same allocation made here
      // (a few milliseconds at a billion candidates)
      unsigned long long room = sizing ? std::min(n_cand / 64, 1ull << 30) : std::min(n_cand / 16, 1ull << 31);
      if (c.budget) {
        std::lock_guard<std::mutex> g(c.budget->mu);
        const size_t left = c.budget->limit > c.budget->cur ? c.budget->limit - c.budget->cur : 0;
        room = std::min<unsigned long long>(room, left / 8 / 12);
      }
      acc.reserve(room);
    }
    // candidates [c_cut, n_cand) belong to long probes: one warp per candidate
    unsigned long long c_cut = n_cand;
    const uint32_t q_cut = aligned_cut(v, v.warp_q_cut);
    if (SELF && !MULTI && q_cut < v.pbegin + v.pcount) c_cut = first_candidate_of(c, hits, off, n_hits, n_cand, q_cut);
    for (unsigned long long cb = 0; cb < n_cand;) {
      const bool warp_range = cb >= c_cut;
      // a big join's first launch is short, so that the accepted-match buffer
      // is sized from its acceptance rate before the long launch runs
      const unsigned long long step =
          verified == 0 && sizing ? std::min(launch_cands, std::max(1ull << 22, n_cand / 64)) : launch_cands;
      const unsigned long long ce = std::min(warp_range ? n_cand : c_cut, cb + step);
      if (verified > 0) {  // room for this launch at the rate so far (+25%), for the join's rest if bigger
        const double rate = (double)acc.last / (double)verified;
        const double left = (double)(n_cand - cb) + (remaining_groups - 1.0) * (double)n_cand;
        acc.reserve((unsigned long long)(acc.last + 1.25 * rate * std::max((double)(ce - cb), left)) + (1ull << 20));
      }
      tv.start();
      acc.run(
          [&](AccOut o) {
            if (warp_range) {
              launch_verify_warp<SELF, MULTI>(c, v, hits.p, off.p, n_hits, cb, ce, o, ctr, v.block_warp);
            } else {
#define PJ_CALL(W) launch_verify<W, SELF, MULTI>(c, v, hits.p, off.p, n_hits, cb, ce, o, ctr, v.block_thread)
              PJ_BY_TAU(v.tau, PJ_CALL);
#undef PJ_CALL
            }
          },
          [&](unsigned long long after) {  // project the whole join from the rate so far
            const double rate = (double)after / (double)(verified + (ce - cb));
            const double left = (double)(n_cand - ce) + (remaining_groups - 1.0) * (double)n_cand;
            return (unsigned long long)(1.25 * (after + rate * left)) + (1ull << 20);
          });
      tv.stop();
      tm.verify += tv.ms();
      verified += ce - cb;
      cb = ce;
    }
    trace_mark(c, "join: verify");
    done += v.pcount;
  }
  if (fb_count) {
    ProbeView v = v0;
    tf.start();
    acc.run(
        [&](AccOut o) {
#define PJ_CALL(W) launch_fallback<W, SELF, MULTI>(c, v, fb_count, o, ctr)
          PJ_BY_TAU(v.tau, PJ_CALL);
#undef PJ_CALL
        },
        [&](unsigned long long after) { return 2 * after; });
    tf.stop();
    tm.fallback += tf.ms();
  }
  const unsigned long long cand = h.candidates, nh = h.hits;
  PJ_CUDA(cudaMemcpyAsync(&h, ctr, sizeof(Counters), cudaMemcpyDeviceToHost, c.stream));
  c.sync();
  // the chunked pipeline counts candidates and hits on the host, the fused
  // kernel its candidates on the device
  h.candidates = cand + (fused_done ? h.candidates : 0ull);
  h.hits = nh;
  if (h.err)
    fail(PJ_ECUDA, std::string("segment index consistency check failed (") +
                       ((h.err & 1) ? "posting outside the index" : "probe limit reached") + ")");
}

// Runs the join, retries once with an exact-size buffer if the accepted
// matches overflowed, then dedupes and compacts into *out.
static void run_join(const Ctx& c, const ProbeView& v, bool self, uint32_t fb_count, int a_bits,
                     bool results_on_device, pj_result* out, const unsigned long long* h_qgoff = nullptr) {
  Counters h{};
  Timings tm;
  DBuf<Counters> ctr(c, 1);
  PJ_CUDA(cudaMemsetAsync(ctr.p, 0, sizeof(Counters), c.stream));
  unsigned long long acc_initial = env_knob("PJ_ACCEPT_INITIAL", 4ull << 20);
  if (c.budget) {  // under a device budget, start at 1/64 of what is left of it (the buffer grows)
    std::lock_guard<std::mutex> g(c.budget->mu);
    const size_t left = c.budget->limit > c.budget->cur ? c.budget->limit - c.budget->cur : 0;
    acc_initial = std::max<unsigned long long>(1024, std::min<unsigned long long>(acc_initial, left / 64 / 12));
  }
  AcceptBuf acc(c, ctr.p, acc_initial);
  if (self) probe_and_verify<true, false>(c, v, fb_count, acc, ctr.p, h, tm, nullptr);
  else if (v.ptau) probe_and_verify<false, true>(c, v, fb_count, acc, ctr.p, h, tm, h_qgoff);
  else probe_and_verify<false, false>(c, v, fb_count, acc, ctr.p, h, tm, nullptr);
  DBuf<unsigned long long>& acc_key = acc.key;
  DBuf<uint32_t>& acc_ed = acc.ed;
  const uint64_t cap = acc.cap;
  const uint64_t nacc = h.accepted;
  EventTimer td(c.stream);
  td.start();
  debug_dump(c, "acc_key", acc_key.p, std::min<uint64_t>(nacc, cap) * sizeof(unsigned long long));
  debug_dump(c, "acc_ed", acc_ed.p, std::min<uint64_t>(nacc, cap) * sizeof(uint32_t));
  uint64_t count = 0;
  DBuf<pj_pair> pairs;
  void* host_block = nullptr;  // host results written by the emit kernel (mapped pool block)
  size_t host_got = 0;
  if (nacc > 0) {
    const int kbits = v.key_shift + a_bits;
    // ed rides in the key's top bits when the pair key leaves room: the sort
    // then moves 8 bytes per match instead of 12
    const bool packed = kbits <= PACKED_KEY_BITS;
    DBuf<unsigned long long> key2(c, nacc);
    DBuf<uint32_t> ed2;
    if (packed) {
      k_pack_ed<<<ceil_div(nacc, 256), 256, 0, c.stream>>>(acc_key.p, acc_ed.p, nacc);
      PJ_LAUNCHED("k_pack_ed");
    } else {
      ed2.reset(c, nacc);
    }
    // sorted into whichever buffer (pair) the last pass wrote (no copy back)
    const bool second = radix_sort_pairs_dn<unsigned long long>(c, acc_key.p, packed ? nullptr : acc_ed.p, key2.p,
                                                                packed ? nullptr : ed2.p, nacc, nullptr, kbits);
    const unsigned long long* skeys = second ? key2.p : acc_key.p;
    const uint32_t* seds = packed ? nullptr : second ? ed2.p : acc_ed.p;
    const unsigned long long kmask = packed ? (1ull << PACKED_KEY_BITS) - 1 : ~0ull;
    trace_mark(c, "join: sort accepted");
    DBuf<uint32_t> flags(c, nacc), pos(c, nacc);
    k_run_heads_masked<<<ceil_div(nacc, 256), 256, 0, c.stream>>>(skeys, nacc, kmask, flags.p);
    PJ_LAUNCHED("k_run_heads_masked");
    exclusive_scan<uint32_t>(c, flags.p, pos.p, nacc);
    uint32_t last[2] = {0, 0};
    PJ_CUDA(cudaMemcpyAsync(&last[0], pos.p + nacc - 1, sizeof(uint32_t), cudaMemcpyDeviceToHost, c.stream));
    PJ_CUDA(cudaMemcpyAsync(&last[1], flags.p + nacc - 1, sizeof(uint32_t), cudaMemcpyDeviceToHost, c.stream));
    c.sync();
    count = (uint64_t)last[0] + last[1];
    pj_pair* dst = nullptr;
    if (!results_on_device && pool_pinned() && count * sizeof(pj_pair) >= PINNED_MIN) {  // emit into host memory
      host_block = pinned_get(count * sizeof(pj_pair), &host_got);
      void* dp = nullptr;
      if (host_block && cudaHostGetDevicePointer(&dp, host_block, 0) == cudaSuccess) {
        dst = static_cast<pj_pair*>(dp);
      } else if (host_block) {
        cudaGetLastError();
        pinned_put(host_block, host_got);
        host_block = nullptr;
      }
    }
    if (!dst) {
      pairs.reset(c, count);
      dst = pairs.p;
    }
    if (packed) {
      k_emit_packed<<<ceil_div(nacc, 256), 256, 0, c.stream>>>(skeys, flags.p, pos.p, nacc, v.key_shift, dst, count);
      PJ_LAUNCHED("k_emit_packed");
    } else {
      k_emit_pairs<<<ceil_div(nacc, 256), 256, 0, c.stream>>>(skeys, seds, flags.p, pos.p, nacc, v.key_shift, dst,
                                                               nullptr, count);
      PJ_LAUNCHED("k_emit_pairs");
    }
  }
  td.stop();
  tm.dedupe = td.ms();
  trace_mark(c, "join: dedupe + compact");
  out->count = count;
  out->stats.lookups = h.lookups;
  out->stats.candidates = h.candidates;
  out->stats.accepted = h.accepted;
  out->stats.dp_cells = h.cells;
  out->stats.filtered = h.filtered;
  out->stats.distinct_pairs = tm.distinct;
  out->stats.fallback_pairs = h.fallback;
  out->stats.hits = h.hits;
  out->stats.probe_ms = tm.probe;
  out->stats.verify_ms = tm.verify;
  out->stats.fallback_ms = tm.fallback;
  out->stats.dedupe_ms = tm.dedupe;
  out->priv = new ResultPriv{c};
  if (results_on_device) {
    out->on_device = 1;
    if (count == 0) pairs.reset(c, 1);
    out->pairs = pairs.p;
    pairs.p = nullptr;  // ownership moves to the result
    c.sync();
  } else if (host_block) {
    out->on_device = 0;
    out->pairs = static_cast<pj_pair*>(host_block);
    static_cast<ResultPriv*>(out->priv)->pinned_bytes = host_got;
    c.sync();
    trace_mark(c, "join: results to host");
  } else {
    out->on_device = 0;
    const size_t bytes = std::max<uint64_t>(count, 1) * sizeof(pj_pair);
    size_t got = 0;
    void* pinned = bytes >= PINNED_MIN ? pinned_get(bytes, &got) : nullptr;
    if (pinned) {
      out->pairs = static_cast<pj_pair*>(pinned);
      static_cast<ResultPriv*>(out->priv)->pinned_bytes = got;
    } else {
      out->pairs = static_cast<pj_pair*>(malloc(bytes));
      if (!out->pairs) fail(PJ_ENOMEM, "host result allocation failed");
    }
    trace_mark(c, pinned ? "join: host block (pinned)" : "join: host block (malloc)");
    if (count)
      PJ_CUDA(cudaMemcpyAsync(out->pairs, pairs.p, count * sizeof(pj_pair), cudaMemcpyDeviceToHost, c.stream));
    c.sync();
    trace_mark(c, "join: results to host");
  }
}

// ------------------------------------------------------------ autotune ----
//
// Decides, for one threshold's self join, (1) the probe length from which
// candidates are verified one warp per candidate instead of one thread per
// candidate, and (2) the block size of the thread-per-candidate kernel.
// Probes are in length order, so a cut-over length splits the candidates
// into a thread range and a warp range.  Every configuration -- cut-over in
// {never, 0, 64, 128, ..., 2048} restricted to the lengths present, block
// size in {128, 256, 512} -- verifies the same prefix of the candidates (at
// most 2^26) into a scratch buffer whose results are dropped; the fastest
// (best of two runs, CUDA events) wins.  Decisions are cached per workload
// signature for the process and, when the index names a cache file
// (pj_options.autotune_cache, else the environment variable
// PJ_AUTOTUNE_CACHE), in that file (one "signature|cut|block|mode|from" line
// each).

struct TuneResult {
  int warp_min_len = 65536;  // with `fused`: the fused kernel's warp-per-pair cut
  int block_thread = 256;
  int pair_mode = 0;  // mode L
  int pair_warp = 0;
  int fused = 0;  // mode L by the fused kernel (k_fused_self)
  int fused_from_len = 0;  // with `fused`: shorter probes run in the chunked mode-L pipeline
};

static std::mutex g_tune_mu;
static std::map<std::string, TuneResult> g_tune_cache;

static std::string tune_signature(const pj_index& idx, int tau) {
  const int lmin = idx.n ? [&] {
    for (int l = 0; l <= idx.lmax; ++l)
      if (idx.h_bbeg[l + 1] > idx.h_bbeg[l]) return l;
    return 0;
  }() : 0;
  char buf[160];
  snprintf(buf, sizeof(buf), "self tau=%d n=%u len=%d..%d avg=%.1f", tau, idx.n, lmin, idx.lmax,
           idx.n ? (double)idx.total_bytes / idx.n : 0.0);
  return buf;
}

// The autotune cache file: the index's option, else PJ_AUTOTUNE_CACHE.
static const char* tune_cache_path(const pj_index& idx) {
  if (!idx.autotune_cache.empty()) return idx.autotune_cache.c_str();
  return getenv("PJ_AUTOTUNE_CACHE");
}

static bool tune_from_file(const char* path, const std::string& key, TuneResult& r) {
  if (!path || !path[0]) return false;
  std::ifstream f(path);
  std::string line;
  bool found = false;
  while (std::getline(f, line)) {
    const size_t a = line.find('|'), b = line.rfind('|');
    if (a == std::string::npos || a == b || line.substr(0, a) != key) continue;
    // signature|cut|block|pairs|from (pairs: 0 extension, 1 thread per pair,
    // 2 warp per pair, 3 the fused kernel with a warp per pair from length
    // `cut` for the probes from length `from`)
    const size_t m = line.find('|', a + 1);
    if (m == std::string::npos || m == b) continue;
    const size_t pm_at = line.find('|', m + 1);
    if (pm_at == std::string::npos || pm_at == b) continue;
    r.warp_min_len = atoi(line.c_str() + a + 1);
    r.block_thread = atoi(line.c_str() + m + 1);
    const int pm = atoi(line.c_str() + pm_at + 1);
    r.pair_mode = pm > 0;
    r.pair_warp = pm == 2;
    r.fused = pm == 3;
    r.fused_from_len = atoi(line.c_str() + b + 1);
    found = true;  // the last line for a key wins
  }
  return found;
}

static void tune_to_file(const char* path, const std::string& key, const TuneResult& r) {
  if (!path || !path[0]) return;
  FILE* f = fopen(path, "a");
  if (!f) return;
  fprintf(f, "%s|%d|%d|%d|%d\n", key.c_str(), r.warp_min_len, r.block_thread,
          r.fused ? 3 : r.pair_mode ? 1 + r.pair_warp : 0, r.fused_from_len);
  fclose(f);
}

// Average string length from which the autotuner tries the fused kernel.
constexpr double FUSED_MIN_AVG_LEN = 32.0;

static TuneResult autotune_self(pj_index& idx, const ProbeView& v0) {
  const Ctx& c = idx.ctx;
  TuneResult best;
  const int tau = v0.tau;
  const int G = groups_per_probe(tau, true);
  const unsigned long long group_budget = std::min(env_knob("PJ_GROUP_BUDGET", 64ull << 20), 1ull << 31);
  ProbeView v = v0;
  v.pcount = (uint32_t)std::min<unsigned long long>(v0.pcount, std::max<unsigned long long>(1, group_budget / G));
  if (v.pcount == 0) return best;
  DBuf<Counters> ctr(c, 1);
  PJ_CUDA(cudaMemsetAsync(ctr.p, 0, sizeof(Counters), c.stream));
  DBuf<uint32_t> gcount, goff;
  DBuf<Hit> hits;
  DBuf<unsigned long long> cnt, off;
  unsigned long long n_hits = 0, n_cand = 0;
  probe_chunk<true, false>(c, v, v.interleave ? interleaved_groups(v.pcount, G) : (unsigned long long)v.pcount * G,
                           ctr.p, gcount, goff, hits, cnt, off, n_hits, n_cand);
  if (n_cand == 0) return best;
  // the timed range: a prefix of the candidates (probes are in length order,
  // so it covers the shortest probes; capped to bound the tuning time)
  const unsigned long long S = std::min<unsigned long long>(n_cand, 1ull << 26);
  DBuf<unsigned long long> scr_key(c, S);
  DBuf<uint32_t> scr_ed(c, S);
  const AccOut scratch{scr_key.p, scr_ed.p, S};
  // cut-over candidates: never, and every bucket edge inside the lengths present
  std::vector<int> cuts{65536};
  const int edges[] = {0, 64, 128, 256, 512, 1024, 2048};
  for (int e : edges)
    if (e <= idx.lmax && idx.h_bbeg[std::min(e, idx.lmax + 1)] < v.pbegin + v.pcount) cuts.push_back(e);
  const int blocks[] = {128, 256, 512};
  EventTimer tm(c.stream);
  double best_ms = 1e30;
  for (int cut : cuts) {
    unsigned long long c_cut = S;
    if (cut < 65536) {
      const uint32_t q_cut = aligned_cut(v, std::max<uint32_t>(idx.h_bbeg[std::max(0, cut)], v.pbegin));
      c_cut = std::min(S, first_candidate_of(c, hits, off, n_hits, n_cand, q_cut));
    }
    for (int blk : blocks) {
      if (c_cut == 0 && blk != 256) continue;  // all warp path: the thread block size is moot
      double ms = 1e30;
      for (int rep = 0; rep < 2; ++rep) {
        PJ_CUDA(cudaMemsetAsync(ctr.p, 0, sizeof(Counters), c.stream));
        tm.start();
        if (c_cut > 0) {
#define PJ_CALL(W) launch_verify<W, true, false>(c, v, hits.p, off.p, n_hits, 0, c_cut, scratch, ctr.p, blk)
          PJ_BY_TAU(tau, PJ_CALL);
#undef PJ_CALL
        }
        if (c_cut < S) launch_verify_warp<true, false>(c, v, hits.p, off.p, n_hits, c_cut, S, scratch, ctr.p, 256);
        tm.stop();
        ms = std::min(ms, (double)tm.ms());
      }
      if (getenv("PJ_TRACE"))
        fprintf(stderr, "[pj] autotune tau=%d cut=%d block=%d: %.3f ms over %llu candidates\n", tau, cut, blk, ms,
                (unsigned long long)S);
      if (ms < best_ms) {
        best_ms = ms;
        best.warp_min_len = cut;
        best.block_thread = blk;
      }
    }
  }
  // mode L on the same candidates: pair keys, sort, distinct pairs, one
  // whole-string verification each (thread or warp per pair)
  if (S <= PAIR_MODE_MAX_CANDS) {
    for (int pw = 0; pw < 2; ++pw) {
      ProbeView vp = v;
      vp.pair_mode = 1;
      vp.pair_warp = pw;
      double ms = 1e30;
      for (int rep = 0; rep < 2; ++rep) {
        PJ_CUDA(cudaMemsetAsync(ctr.p, 0, sizeof(Counters), c.stream));
        AccOut sc = scratch;
        tm.start();
        verify_pairs_chunk<true>(c, vp, hits.p, off.p, n_hits, S, ctr.p, &sc, nullptr);
        tm.stop();
        ms = std::min(ms, (double)tm.ms());
      }
      if (getenv("PJ_TRACE"))
        fprintf(stderr, "[pj] autotune tau=%d distinct pairs (%s): %.3f ms over %llu candidates\n", tau,
                pw ? "warp" : "thread", ms, (unsigned long long)S);
      if (ms < best_ms) {
        best_ms = ms;
        best.pair_mode = 1;
        best.pair_warp = pw;
      }
    }
  }
  // the fused kernel does selection, probing and verification in one launch:
  // whole joins of the sample with it (the probes shorter than `from` in the
  // chunked mode-L pipeline), against a whole join with the best choice above,
  // when that choice was timed over every candidate of the sample and the
  // strings are not short (short strings have few-character segments and
  // long posting runs, which the chunked pipeline spreads over the GPU)
  const double avg_len = idx.n ? (double)idx.total_bytes / idx.n : 0.0;
  if (S == n_cand && avg_len >= FUSED_MIN_AVG_LEN) {
    gcount.release();
    goff.release();
    hits.release();
    cnt.release();
    off.release();
    AcceptBuf facc(c, ctr.p, std::min<unsigned long long>(S, 1ull << 20));
    auto whole_join_ms = [&](const ProbeView& vj) {
      double ms = 1e30;
      for (int rep = 0; rep < 2; ++rep) {
        PJ_CUDA(cudaMemsetAsync(ctr.p, 0, sizeof(Counters), c.stream));
        Counters hh{};
        Timings ft;
        tm.start();
        probe_and_verify<true, false>(c, vj, 0, facc, ctr.p, hh, ft, nullptr);
        tm.stop();
        ms = std::min(ms, (double)tm.ms());
      }
      return ms;
    };
    {  // the chunked pipeline with the choice so far, as a whole join of the sample
      ProbeView vb = v;
      vb.pair_mode = best.pair_mode;
      vb.pair_warp = best.pair_warp;
      if (vb.pair_mode) vb.hit_sides = 0;
      vb.block_thread = best.block_thread;
      if (!best.pair_mode && best.warp_min_len <= idx.lmax) vb.warp_q_cut = idx.h_bbeg[std::max(0, best.warp_min_len)];
      best_ms = whole_join_ms(vb);
    }
    const uint32_t q_last = v.pbegin + v.pcount - 1;
    std::vector<int> froms{0};
    for (int e : {16, 32, 64, 128, 256})
      if (e <= idx.lmax && idx.h_bbeg[e] > v.pbegin && idx.h_bbeg[e] <= q_last) froms.push_back(e);
    for (int from : froms) {
      for (int cut : {65536, 0}) {
        ProbeView vf = v;
        vf.pair_mode = 1;
        vf.pair_warp = cut == 0;
        vf.hit_sides = 0;
        vf.fused = 1;
        vf.fused_warp_from = cut;
        vf.fused_q_cut = from > 0 ? idx.h_bbeg[from] : 0;
        const double ms = whole_join_ms(vf);
        if (getenv("PJ_TRACE"))
          fprintf(stderr, "[pj] autotune tau=%d fused from length %d, warp per pair %s: %.3f ms (best so far %.3f ms)\n",
                  tau, from, cut == 0 ? "yes" : "no", ms, best_ms);
        if (ms < best_ms) {
          best_ms = ms;
          best.pair_mode = 1;
          best.pair_warp = cut == 0;
          best.fused = 1;
          best.warp_min_len = cut;
          best.fused_from_len = from;
        }
      }
    }
  }
  if (getenv("PJ_TRACE"))
    fprintf(stderr,
            "[pj] autotune tau=%d: warp from length %d, block %d, distinct pairs %d (warp %d), fused %d from length "
            "%d\n",
            tau, best.warp_min_len, best.block_thread, best.pair_mode, best.pair_warp, best.fused,
            best.fused_from_len);
  return best;
}

// Strings longer than this on average are verified in mode L by default:
// near-duplicate long strings match on most of their segments.
constexpr double PAIR_MODE_MIN_AVG_LEN = 256.0;

static void default_mode(const pj_index& idx, TuneResult& r) {
  const double avg = idx.n ? (double)idx.total_bytes / idx.n : 0.0;
  r.pair_mode = avg > PAIR_MODE_MIN_AVG_LEN ? 1 : 0;
  r.pair_warp = r.pair_mode;
}

// The index's verify_mode option, then PJ_VERIFY_PAIRS=0|1|2 (extension,
// thread per pair, warp per pair), override the choice.
static void force_mode(const pj_index& idx, TuneResult& r) {
  if (idx.verify_mode == PJ_VERIFY_EXTENSION) {
    r.pair_mode = 0;
  } else if (idx.verify_mode == PJ_VERIFY_PAIRS && !r.pair_mode) {
    TuneResult d;
    default_mode(idx, d);
    r.pair_mode = 1;
    r.pair_warp = d.pair_warp;
  }
  const char* pm = getenv("PJ_VERIFY_PAIRS");
  if (pm && pm[0]) {
    const int m = atoi(pm);
    r.pair_mode = m > 0;
    r.pair_warp = m == 2;
  }
  if (!r.pair_mode) r.fused = 0;
}

// PJ_FUSED=0|1|2 (chunked pipeline, the fused kernel with a thread per
// pair, the fused kernel with a warp per pair) overrides a self join's
// choice, PJ_FUSED_FROM=<length> the shortest probe length of the fused
// kernel.
static void force_fused(TuneResult& r) {
  const char* fz = getenv("PJ_FUSED");
  if (fz && fz[0]) {
    const int m = atoi(fz);
    r.fused = m > 0;
    r.fused_from_len = 0;
    if (r.fused) {
      r.pair_mode = 1;
      r.pair_warp = m == 2;
      r.warp_min_len = m == 2 ? 0 : 65536;
    }
  }
  const char* ff = getenv("PJ_FUSED_FROM");
  if (r.fused && ff && ff[0]) r.fused_from_len = std::max(0, atoi(ff));
}

// The tuning of a self join: environment overrides, then the caches, then a
// fresh measurement (when the index asks for autotuning).
static TuneResult self_join_tuning(pj_index& idx, const ProbeView& v, float* tune_ms) {
  TuneResult r;
  *tune_ms = 0.f;
  if (idx.autotune) {
    const std::string key = tune_signature(idx, v.tau);
    std::lock_guard<std::mutex> g(g_tune_mu);
    auto it = g_tune_cache.find(key);
    if (it != g_tune_cache.end()) {
      r = it->second;
    } else if (tune_from_file(tune_cache_path(idx), key, r)) {
      g_tune_cache[key] = r;
    } else {
      const auto t0 = std::chrono::steady_clock::now();
      r = autotune_self(idx, v);
      *tune_ms = std::chrono::duration<float, std::milli>(std::chrono::steady_clock::now() - t0).count();
      g_tune_cache[key] = r;
      tune_to_file(tune_cache_path(idx), key, r);
    }
  }
  if (!idx.autotune) default_mode(idx, r);
  force_mode(idx, r);
  force_fused(r);
  const char* e = getenv("PJ_WARP_MIN_LEN");
  if (e && e[0]) r.warp_min_len = atoi(e);
  const char* bk = getenv("PJ_VERIFY_BLOCK");
  if (bk && bk[0]) r.block_thread = atoi(bk);
  if (r.block_thread != 128 && r.block_thread != 256 && r.block_thread != 512) r.block_thread = 256;
  return r;
}

// Probe interleaving (see group_of) for strings of this average length or
// shorter; PJ_PROBE_INTERLEAVE=0/1 overrides.
constexpr double INTERLEAVE_MAX_AVG_LEN = 256.0;

static ProbeView index_side(const pj_index& idx, const Partition& part) {
  ProbeView v{};
  v.seg_magic = seg_magic(part.tau + 1);
  v.scheme = part.scheme;
  const double avg = idx.n ? (double)idx.total_bytes / idx.n : 0.0;
  v.interleave = avg <= INTERLEAVE_MAX_AVG_LEN ? 1 : 0;
  const char* il = getenv("PJ_PROBE_INTERLEAVE");
  if (il && il[0]) v.interleave = atoi(il) ? 1 : 0;
  v.warp_q_cut = UINT32_MAX;
  v.block_thread = 256;
  v.block_warp = 256;
  const char* vq = getenv("PJ_VERIFY_QUEUE");
  v.queued = vq && vq[0] ? atoi(vq) : 1;
  v.hit_sides = v.queued && part.sides;  // off for mode L, which verifies whole strings
  // shared prefixes in mode L: off unless PJ_SHARE_PREFIX=1 (on the
  // synthetic workloads it saves under 2% of the DP cells and costs time)
  const char* sp = getenv("PJ_SHARE_PREFIX");
  v.share_prefix = sp && sp[0] ? atoi(sp) : 0;
  v.ibytes = idx.sbytes.p;
  v.ioff = idx.soff.p;
  v.ilen = idx.slen.p;
  v.iref = idx.sref.p;
  v.ibbeg = idx.bbeg.p;
  v.ilmax = idx.lmax;
  v.iperm = idx.perm.p;
  v.n_index = idx.n;
  v.table = part.table.p;
  v.table_fp = part.fp.p;
  v.table_pb = part.presence_bytes;
  v.precs = part.precs.p;
  v.ibm = idx.sbm.p;
  v.mask = part.table.n - 1;
  v.postings = part.postings.p;
  v.n_postings = part.n_records;
  v.tau = part.tau;
  return v;
}

// ------------------------------------------------------------ join plans --
//
// A self join of an unchanged index repeats exactly.  With graph_joins, its
// first eager run at a threshold is followed by recording the whole
// pipeline into a CUDA graph: sizes kept on the device as in query plans,
// every capacity set from that run's own counts (groups, hits, candidates,
// distinct pairs, accepted matches, pairs).  Later self joins of the
// threshold replay the graph -- one launch and one synchronisation -- and
// copy the pairs out.  A replay whose counts exceed the recorded capacities
// (which an unchanged index cannot produce) is discarded and the join runs
// eagerly.  Not recorded: joins with a warp-per-candidate range, or with more
// than PJ_GRAPH_MAX_GROUPS probe groups (2^28 by default; the graph probes
// all groups in one pass, where the eager join takes chunks).

// fz (the fused form, else NULL): fz[2] nonzero when one of its lists
// outgrew its capacity; its candidates are then counted in ctr->candidates.
__global__ void k_self_finish(const Counters* __restrict__ ctr, const PlanSizes* __restrict__ sizes,
                              const unsigned long long* __restrict__ unique, PlanHeader* header,
                              const unsigned long long* __restrict__ fz) {
  PlanHeader h;
  h.groups = 0;
  h.hits = sizes->hits;
  h.cands = fz ? ctr->candidates : sizes->cands;
  h.overflow = fz ? fz[2] : 0ull;
  const unsigned long long in_kernel = fz ? fz[3] : 0ull;
  h.accepted = ctr->accepted;
  h.pairs = sizes->pairs;
  h.lookups = ctr->lookups;
  h.cells = ctr->cells;
  h.fallback = ctr->fallback;
  h.err = ctr->err;
  h.filtered = ctr->filtered;
  h.unique = *unique + in_kernel;
  *header = h;
}

struct SelfPlan {
  Ctx ctx;  // the index's allocator on the plan's own stream
  cudaStream_t stream = nullptr;
  int warp_min_len = 0, block_thread = 0, pair_mode = 0, pair_warp = 0, fused = 0,
      fused_from_len = 0;  // the tuning it was recorded with
  uint32_t fb_count = 0;
  int a_bits = 0;
  unsigned long long n_groups = 0, cap_hits = 0, cap_cands = 0, cap_acc = 0, cap_pairs = 0;
  unsigned long long n_cand = 0;  // the eager run's candidates (sets the verification chunk)
  DBuf<unsigned char> counters, arena;
  DBuf<PlanSizes> sizes;
  DBuf<unsigned long long> nuniq, gmask, hcnt, hoff, pk0, pk1, ukeys, ak0, ak1;
  DBuf<uint32_t> gcounts, goff, pv0, pv1, pflags, ppos, ae0, ae1, flags, pos;
  DBuf<Hit> hits;
  DBuf<pj_pair> out;
  // the fused form: k_fused_self over probes [q_cut, end), the chunked
  // mode-L pipeline over the shorter ones
  uint32_t q_cut = 0;
  int fused_form = 0, ppi = 1;
  unsigned long long ovf_cap = 0, heavy_cap = 0;
  DBuf<unsigned long long> fwork, fovf, fhcnt, fhoff, fhk, fz, fstart;
  DBuf<Hit> fheavy;
  HostBuf header;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  uint32_t kernels = 0;

  ~SelfPlan() {
    if (stream) cudaStreamSynchronize(stream);
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
    DBuf<unsigned long long>* b64[] = {&nuniq, &gmask, &hcnt, &hoff, &pk0, &pk1, &ukeys, &ak0, &ak1,
                                       &fwork, &fovf, &fhcnt, &fhoff, &fhk, &fz, &fstart};
    for (auto* b : b64) b->release();
    fheavy.release();
    DBuf<uint32_t>* b32[] = {&gcounts, &goff, &pv0, &pv1, &pflags, &ppos, &ae0, &ae1, &flags, &pos};
    for (auto* b : b32) b->release();
    counters.release();
    arena.release();
    sizes.release();
    hits.release();
    out.release();
    if (stream) {
      cudaStreamSynchronize(stream);
      cudaStreamDestroy(stream);
    }
  }
};

// The recorded fused join's bookkeeping: fz[0] = long runs kept (at most
// heavy_cap), fz[3] = distinct pairs verified in the kernel, and, in
// k_fused_tail_starts, the place of every list of pair
// keys after the chunked pipeline's sz->cands: the 64 overflow sub-lists,
// then the long runs' keys (fz[1] of them); sz->cands becomes the total, the
// chunked pipeline's candidates join ctr->candidates, and fz[2] flags a list
// that outgrew its capacity (the replay is then discarded).
__global__ void k_fused_heavy_n(const unsigned long long* __restrict__ work, unsigned long long heavy_cap,
                                unsigned long long* __restrict__ fz) {
  fz[0] = min(work[2], heavy_cap);
  fz[2] = work[2] > heavy_cap ? 1ull : 0ull;
  fz[3] = work[1];  // distinct pairs verified in the kernel
}

__global__ void k_fused_tail_starts(const unsigned long long* __restrict__ ovf_n, unsigned long long ovf_cap,
                                    unsigned long long* __restrict__ fz, unsigned long long* __restrict__ start,
                                    PlanSizes* sz, Counters* ctr, unsigned long long cap_keys) {
  unsigned long long at = sz->cands, flag = fz[2];
  ctr->candidates += sz->cands;
  for (int k = 0; k < FOVF_LISTS; ++k) {
    start[k] = at;
    at += min(ovf_n[k], ovf_cap);
    if (ovf_n[k] > ovf_cap) flag = 1;
  }
  start[FOVF_LISTS] = at;
  at += fz[1];
  if (at > cap_keys) flag = 1;
  sz->cands = min(at, cap_keys);
  fz[2] = flag;
}

// Lists k < 64: overflow sub-list k; list 64: the long runs' keys.  Block k
// copies list k to dst + start[k] (clamped to cap).
__global__ void k_fused_gather(const unsigned long long* __restrict__ ovf, unsigned long long ovf_cap,
                               const unsigned long long* __restrict__ hk, const unsigned long long* __restrict__ fz,
                               const unsigned long long* __restrict__ start, unsigned long long* __restrict__ dst,
                               unsigned long long cap) {
  const unsigned k = blockIdx.x;
  const unsigned long long* src = k < FOVF_LISTS ? ovf + FOVF_LISTS + k * ovf_cap : hk;
  const unsigned long long m = k < FOVF_LISTS ? min(ovf[k], ovf_cap) : fz[1];
  const unsigned long long s = start[k];
  for (unsigned long long i = threadIdx.x; i < m && s + i < cap; i += blockDim.x) dst[s + i] = src[i];
}

static void record_fused_tail(const Ctx& c, const ProbeView& v, SelfPlan& P, Counters* ctr, PlanSizes* sz,
                              const AccOut& acc) {
  ProbeView vf = v;
  vf.pbegin = P.q_cut;
  vf.pcount = v.pbegin + v.pcount - P.q_cut;
  const int pshift = bits_for(v.n_index);
  const unsigned long long n_items = ((unsigned long long)vf.pcount + P.ppi - 1) / P.ppi;
  PJ_CUDA(cudaMemsetAsync(P.fwork.p, 0, 3 * sizeof(unsigned long long), c.stream));
  PJ_CUDA(cudaMemsetAsync(P.fovf.p, 0, FOVF_LISTS * sizeof(unsigned long long), c.stream));
  PJ_CUDA(cudaMemsetAsync(P.fz.p, 0, 4 * sizeof(unsigned long long), c.stream));
#define PJ_FORM(W, F)                                                                                          \
  do {                                                                                                        \
    const unsigned g = persistent_grid(k_fused_self<W, F>, n_items, FB);                                      \
    k_fused_self<W, F><<<g, FB, 0, c.stream>>>(vf, P.ppi, vf.fused_warp_from, P.fwork.p, P.fovf.p, P.ovf_cap,   \
                                               P.fheavy.p, P.heavy_cap, pshift, acc, ctr);                    \
    PJ_LAUNCHED("k_fused_self");                                                                              \
  } while (0)
#define PJ_CALL(W)                                             \
  do {                                                         \
    if (P.fused_form == FUSED_THREAD) PJ_FORM(W, FUSED_THREAD); \
    else if (P.fused_form == FUSED_WARP) PJ_FORM(W, FUSED_WARP); \
    else PJ_FORM(W, FUSED_CUT);                                \
  } while (0)
  PJ_BY_TAU(v.tau, PJ_CALL);
#undef PJ_CALL
#undef PJ_FORM
  // the long runs' pair keys
  k_fused_heavy_n<<<1, 1, 0, c.stream>>>(P.fwork.p, P.heavy_cap, P.fz.p);
  PJ_LAUNCHED("k_fused_heavy_n");
  k_hit_counts<<<stride_grid(P.heavy_cap), 256, 0, c.stream>>>(P.fheavy.p, P.heavy_cap, P.fhcnt.p, P.fz.p);
  PJ_LAUNCHED("k_hit_counts");
  exclusive_scan_dn<unsigned long long>(c, P.fhcnt.p, P.fhoff.p, P.heavy_cap, P.fz.p, P.fz.p + 1);
  const unsigned gk = persistent_grid(k_pair_keys<true>, ~0ull >> 8);
  k_pair_keys<true><<<gk, BLOCK, 0, c.stream>>>(vf, P.fheavy.p, P.fhoff.p, P.heavy_cap, 0, P.cap_cands, pshift,
                                                P.fhk.p, ctr, P.fz.p);
  PJ_LAUNCHED("k_pair_keys");
  // every list after the chunked pipeline's keys
  k_fused_tail_starts<<<1, 1, 0, c.stream>>>(P.fovf.p, P.ovf_cap, P.fz.p, P.fstart.p, sz, ctr, P.cap_cands);
  PJ_LAUNCHED("k_fused_tail_starts");
  k_fused_gather<<<FOVF_LISTS + 1, 256, 0, c.stream>>>(P.fovf.p, P.ovf_cap, P.fhk.p, P.fz.p, P.fstart.p, P.pk0.p,
                                                        P.cap_cands);
  PJ_LAUNCHED("k_fused_gather");
}

static void record_self_plan(const Ctx& c, const ProbeView& v, SelfPlan& P) {
  Counters* ctr = reinterpret_cast<Counters*>(P.counters.p);
  PlanSizes* sz = P.sizes.p;
  PJ_CUDA(cudaMemsetAsync(ctr, 0, sizeof(Counters), c.stream));
  ProbeView vc = v;  // the probes of the chunked pipeline
  if (P.fused) vc.pcount = P.q_cut - v.pbegin;
  // A4
  if (P.n_groups) {
    const unsigned g1 = persistent_grid(k_group_counts<true, false>, (P.n_groups + BLOCK - 1) / BLOCK);
    k_group_counts<true, false><<<g1, BLOCK, 0, c.stream>>>(vc, P.n_groups, P.gcounts.p, P.gmask.p, ctr, nullptr);
    PJ_LAUNCHED("k_group_counts");
    exclusive_scan_dn<uint32_t>(c, P.gcounts.p, P.goff.p, P.n_groups, nullptr, &sz->hits);
    const unsigned g2 = persistent_grid(k_group_hits<true, false>, (P.n_groups + BLOCK - 1) / BLOCK);
    k_group_hits<true, false><<<g2, BLOCK, 0, c.stream>>>(vc, P.n_groups, P.gcounts.p, P.gmask.p, P.goff.p,
                                                          P.hits.p, nullptr, P.cap_hits);
    PJ_LAUNCHED("k_group_hits");
    k_hit_counts<<<stride_grid(P.cap_hits), 256, 0, c.stream>>>(P.hits.p, P.cap_hits, P.hcnt.p, &sz->hits);
    PJ_LAUNCHED("k_hit_counts");
    exclusive_scan_dn<unsigned long long>(c, P.hcnt.p, P.hoff.p, P.cap_hits, &sz->hits, &sz->cands);
  } else {  // every probe in the fused kernel
    PJ_CUDA(cudaMemsetAsync(sz, 0, sizeof(PlanSizes), c.stream));
  }
  // A5 (mode L) + A6 + A8
  const AccOut acc{P.ak0.p, P.ae0.p, P.cap_acc};
  if (!P.pair_mode) {
    PJ_CUDA(cudaMemsetAsync(P.nuniq.p, 0, sizeof(unsigned long long), c.stream));
#define PJ_CALL(W)                                                                                              \
  do {                                                                                                         \
    const unsigned gv = persistent_grid(k_verify_queued<W, true, false>, ~0ull >> 8, Q_BLOCK);                  \
    k_verify_queued<W, true, false><<<gv, Q_BLOCK, 0, c.stream>>>(v, P.hits.p, P.hoff.p, P.cap_hits, 0, 0, acc,  \
                                                                  ctr, &sz->hits, queued_chunk(P.n_cand, gv));  \
    PJ_LAUNCHED("k_verify_queued");                                                                            \
  } while (0)
    PJ_BY_TAU(v.tau, PJ_CALL);
#undef PJ_CALL
  } else {
    const int pshift = bits_for(v.n_index);
    if (P.n_groups) {
      const unsigned gk = persistent_grid(k_pair_keys<true>, ~0ull >> 8);
      k_pair_keys<true><<<gk, BLOCK, 0, c.stream>>>(vc, P.hits.p, P.hoff.p, P.cap_hits, 0, P.cap_cands, pshift,
                                                    P.pk0.p, ctr, &sz->hits);
      PJ_LAUNCHED("k_pair_keys");
    }
    if (P.fused) record_fused_tail(c, v, P, ctr, sz, acc);  // its pair keys after the chunked ones
    const bool second = radix_sort_pairs_dn<unsigned long long>(c, P.pk0.p, P.pv0.p, P.pk1.p, P.pv1.p, P.cap_cands,
                                                                &sz->cands, 2 * pshift);
    const unsigned long long* sorted = second ? P.pk1.p : P.pk0.p;
    k_run_heads<<<stride_grid(P.cap_cands), 256, 0, c.stream>>>(sorted, P.cap_cands, P.pflags.p, &sz->cands);
    PJ_LAUNCHED("k_run_heads");
    exclusive_scan_dn<uint32_t>(c, P.pflags.p, P.ppos.p, P.cap_cands, &sz->cands, P.nuniq.p);
    k_unique_keys<<<stride_grid(P.cap_cands), 256, 0, c.stream>>>(sorted, P.pflags.p, P.ppos.p, P.cap_cands,
                                                                  P.ukeys.p, &sz->cands);
    PJ_LAUNCHED("k_unique_keys");
    if (P.pair_warp) {
      const unsigned gw = persistent_grid(k_verify_pairs_warp<true>, ~0ull >> 8);
      k_verify_pairs_warp<true><<<gw, BLOCK, 0, c.stream>>>(v, P.ukeys.p, P.cap_cands, pshift, acc, ctr, P.nuniq.p);
      PJ_LAUNCHED("k_verify_pairs_warp");
    } else {
#define PJ_CALL(W)                                                                                              \
  do {                                                                                                         \
    const unsigned gt = persistent_grid(k_verify_pairs<W, true>, ~0ull >> 8);                                   \
    k_verify_pairs<W, true><<<gt, BLOCK, 0, c.stream>>>(v, P.ukeys.p, P.cap_cands, pshift, acc, ctr, P.nuniq.p);  \
    PJ_LAUNCHED("k_verify_pairs");                                                                             \
  } while (0)
      PJ_BY_TAU(v.tau, PJ_CALL);
#undef PJ_CALL
    }
  }
  if (P.fb_count) {
#define PJ_CALL(W)                                                                                              \
  do {                                                                                                         \
    const unsigned gf = persistent_grid(k_fallback<W, true, false>, (P.fb_count + BLOCK - 1) / BLOCK);          \
    k_fallback<W, true, false><<<gf, BLOCK, 0, c.stream>>>(v, P.fb_count, acc, ctr, nullptr);                   \
    PJ_LAUNCHED("k_fallback");                                                                                 \
  } while (0)
    PJ_BY_TAU(v.tau, PJ_CALL);
#undef PJ_CALL
  }
  // A5 + A7
  const bool second = radix_sort_pairs_dn<unsigned long long>(c, P.ak0.p, P.ae0.p, P.ak1.p, P.ae1.p, P.cap_acc,
                                                              &ctr->accepted, v.key_shift + P.a_bits);
  const unsigned long long* keys = second ? P.ak1.p : P.ak0.p;
  const uint32_t* eds = second ? P.ae1.p : P.ae0.p;
  k_run_heads<<<stride_grid(P.cap_acc), 256, 0, c.stream>>>(keys, P.cap_acc, P.flags.p, &ctr->accepted);
  PJ_LAUNCHED("k_run_heads");
  exclusive_scan_dn<uint32_t>(c, P.flags.p, P.pos.p, P.cap_acc, &ctr->accepted, &sz->pairs);
  k_emit_pairs<<<stride_grid(P.cap_acc), 256, 0, c.stream>>>(keys, eds, P.flags.p, P.pos.p, P.cap_acc, v.key_shift,
                                                             P.out.p, &ctr->accepted, P.cap_pairs);
  PJ_LAUNCHED("k_emit_pairs");
  k_self_finish<<<1, 1, 0, c.stream>>>(ctr, sz, P.nuniq.p, static_cast<PlanHeader*>(P.header.dev),
                                       P.fused ? P.fz.p : nullptr);
  PJ_LAUNCHED("k_self_finish");
}

// Recorded capacity for a count of the eager run: the count plus slack; with
// PJ_GRAPH_TIGHT=1 (tests) half the count, so that replays overflow and take
// the eager path.
static unsigned long long with_slack(unsigned long long n) {
  return env_knob("PJ_GRAPH_TIGHT", 0) ? std::max(1ull, n / 2) : n + n / 64 + 1024;
}

// Records the self join described by v and st (the counts of its eager
// run); returns nullptr when the join is not eligible.
static std::shared_ptr<SelfPlan> make_self_plan(pj_index& idx, const ProbeView& v, const TuneResult& tr,
                                                uint32_t fb_count, const pj_stats& st, uint64_t pairs) {
  const int G = groups_per_probe(v.tau, true);
  const uint32_t end = v.pbegin + v.pcount;
  // the fused form: the chunked pipeline over probes [pbegin, q_cut)
  const uint32_t q_cut = tr.fused ? std::min(end, std::max(v.pbegin, v.fused_q_cut)) : end;
  const uint32_t n_chunked = q_cut - v.pbegin;
  const unsigned long long n_groups =
      v.interleave ? interleaved_groups(n_chunked, G) : (unsigned long long)n_chunked * G;
  if (n_groups == 0 && !tr.fused) return nullptr;  // nothing to probe
  // one probe pass over all groups (16 B each), however the eager join chunked them
  if (n_groups > std::min(env_knob("PJ_GRAPH_MAX_GROUPS", 1ull << 28), 1ull << 31)) return nullptr;
  if (!tr.pair_mode && aligned_cut(v, v.warp_q_cut) < v.pbegin + v.pcount) return nullptr;  // a warp range
  if (tr.pair_mode && st.candidates > PAIR_MODE_MAX_CANDS) return nullptr;        // mode L skipped eagerly
  auto P = std::make_shared<SelfPlan>();
  PJ_CUDA(cudaStreamCreateWithFlags(&P->stream, cudaStreamNonBlocking));
  P->ctx = idx.ctx;
  P->ctx.stream = P->stream;
  P->warp_min_len = tr.warp_min_len;
  P->block_thread = tr.block_thread;
  P->pair_mode = tr.pair_mode;
  P->pair_warp = tr.pair_warp;
  P->fused = tr.fused;
  P->fused_from_len = tr.fused_from_len;
  P->fb_count = fb_count;
  P->a_bits = bits_for(idx.n);
  P->n_groups = n_groups;
  P->cap_hits = with_slack(st.hits);
  P->cap_cands = tr.pair_mode ? with_slack(st.candidates) : 1;
  P->n_cand = st.candidates;
  P->cap_acc = std::min<unsigned long long>(0xFFFFFFFFull, with_slack(st.accepted));
  P->cap_pairs = with_slack(pairs);
  const Ctx& c = P->ctx;
  P->counters.reset(c, 64);
  P->sizes.reset(c, 1);
  P->nuniq.reset(c, 1);
  P->gcounts.reset(c, n_groups);
  P->goff.reset(c, n_groups);
  P->gmask.reset(c, n_groups);
  P->hits.reset(c, P->cap_hits);
  P->hcnt.reset(c, P->cap_hits);
  P->hoff.reset(c, P->cap_hits);
  P->pk0.reset(c, P->cap_cands);
  P->pk1.reset(c, P->cap_cands);
  P->pv0.reset(c, P->cap_cands);
  P->pv1.reset(c, P->cap_cands);
  P->pflags.reset(c, P->cap_cands);
  P->ppos.reset(c, P->cap_cands);
  P->ukeys.reset(c, P->cap_cands);
  P->ak0.reset(c, P->cap_acc);
  P->ak1.reset(c, P->cap_acc);
  P->ae0.reset(c, P->cap_acc);
  P->ae1.reset(c, P->cap_acc);
  P->flags.reset(c, P->cap_acc);
  P->pos.reset(c, P->cap_acc);
  P->out.reset(c, P->cap_pairs);
  P->header.reset(sizeof(PlanHeader), true);
  if (tr.fused) {
    ProbeView vf = v;
    vf.pbegin = q_cut;
    vf.pcount = end - q_cut;
    P->q_cut = q_cut;
    P->ppi = fused_ppi(vf);
    P->fused_form = fused_form_of(c, vf);
    P->ovf_cap = fused_ovf_cap(vf);
    P->heavy_cap = fused_heavy_cap(vf);
    P->fwork.reset(c, 3);
    P->fovf.reset(c, FOVF_LISTS + FOVF_LISTS * P->ovf_cap);
    P->fheavy.reset(c, P->heavy_cap);
    P->fhcnt.reset(c, P->heavy_cap + 1);
    P->fhoff.reset(c, P->heavy_cap + 1);
    P->fhk.reset(c, P->cap_cands);
    P->fz.reset(c, 4);
    P->fstart.reset(c, FOVF_LISTS + 1);
  }
  size_t arena_bytes = scan_temp_bytes(n_groups, 4) + scan_temp_bytes(P->cap_hits, 8) +
                       2 * scan_temp_bytes(P->cap_cands, 4) + sort_temp_bytes(P->cap_cands) +
                       scan_temp_bytes(P->cap_acc, 4) + sort_temp_bytes(P->cap_acc) +
                       scan_temp_bytes(P->heavy_cap, 8) + (1u << 16);
  for (int attempt = 0;; ++attempt) {
    P->arena.reset(c, arena_bytes);
    c.sync();
    Arena ar;
    ar.base = P->arena.p;
    ar.cap = arena_bytes;
    Ctx rc;
    rc.stream = P->stream;
    rc.alloc = arena_alloc;
    rc.free_fn = arena_free;
    rc.alloc_ctx = &ar;
    cudaGraph_t g = nullptr;
    PJ_CUDA(cudaStreamBeginCapture(P->stream, cudaStreamCaptureModeRelaxed));
    set_recording(true);
    bool ok = true;
    Error err{PJ_OK, ""};
    try {
      record_self_plan(rc, v, *P);
    } catch (const Error& e) {
      ok = false;
      err = e;
    }
    set_recording(false);
    const cudaError_t ce = cudaStreamEndCapture(P->stream, &g);
    if (!ok || ce != cudaSuccess || !g) {
      if (g) cudaGraphDestroy(g);
      cudaGetLastError();
      if (!ok && ar.exhausted && attempt < 4) {
        arena_bytes *= 2;
        continue;
      }
      if (!ok) throw err;
      fail(PJ_ECUDA, std::string("self-join graph capture failed: ") + cudaGetErrorString(ce));
    }
    P->graph = g;
    if (cudaGraphInstantiate(&P->exec, g, 0) != cudaSuccess) {
      cudaGetLastError();
      P->exec = nullptr;
      fail(PJ_ECUDA, "self-join graph: cudaGraphInstantiate failed");
    }
    size_t n = 0;
    PJ_CUDA(cudaGraphGetNodes(g, nullptr, &n));
    std::vector<cudaGraphNode_t> nodes(n);
    PJ_CUDA(cudaGraphGetNodes(g, nodes.data(), &n));
    for (size_t k = 0; k < n; ++k) {
      cudaGraphNodeType t;
      PJ_CUDA(cudaGraphNodeGetType(nodes[k], &t));
      if (t == cudaGraphNodeTypeKernel) ++P->kernels;
    }
    return P;
  }
}

// Replays P into *out; false when the counts did not fit (the caller then
// runs the join eagerly).
static bool replay_self_plan(SelfPlan& P, const Ctx& rc, bool on_device, pj_result* out) {
  EventTimer t(P.stream);
  t.start();
  PJ_CUDA(cudaGraphLaunch(P.exec, P.stream));
  count_launches(P.kernels);
  t.stop();
  P.ctx.sync();
  PlanHeader h;
  memcpy(&h, P.header.p, sizeof(h));
  if (h.err)
    fail(PJ_ECUDA, std::string("segment index consistency check failed (") +
                       ((h.err & 1) ? "posting outside the index" : "probe limit reached") + ")");
  if (h.hits > P.cap_hits || (P.pair_mode && !P.fused && h.cands > P.cap_cands) || h.accepted > P.cap_acc ||
      h.pairs > P.cap_pairs || h.overflow)
    return false;
  const uint64_t count = h.pairs;
  out->count = count;
  out->stats.lookups = h.lookups;
  out->stats.candidates = h.cands;
  out->stats.accepted = h.accepted;
  out->stats.dp_cells = h.cells;
  out->stats.filtered = h.filtered;
  out->stats.fallback_pairs = h.fallback;
  out->stats.hits = h.hits;
  out->stats.distinct_pairs = h.unique;
  out->stats.graph_replay = 1;
  out->stats.graph_ms = t.ms();
  auto* priv = new ResultPriv{rc};
  out->priv = priv;
  const size_t bytes = std::max<uint64_t>(count, 1) * sizeof(pj_pair);
  if (on_device) {
    out->on_device = 1;
    out->pairs = static_cast<pj_pair*>(rc.get(bytes));
    if (count)
      PJ_CUDA(cudaMemcpyAsync(out->pairs, P.out.p, count * sizeof(pj_pair), cudaMemcpyDeviceToDevice, rc.stream));
  } else {
    out->on_device = 0;
    size_t got = 0;
    void* blk = bytes >= PINNED_MIN ? pinned_get(bytes, &got) : nullptr;
    if (blk) {
      out->pairs = static_cast<pj_pair*>(blk);
      priv->pinned_bytes = got;
    } else {
      out->pairs = static_cast<pj_pair*>(malloc(bytes));
      if (!out->pairs) fail(PJ_ENOMEM, "host result allocation failed");
    }
    if (count)
      PJ_CUDA(cudaMemcpyAsync(out->pairs, P.out.p, count * sizeof(pj_pair), cudaMemcpyDeviceToHost, rc.stream));
  }
  rc.sync();
  return true;
}

// The self join over probes with sids in [q_lo, q_hi) (all of them by
// default).  Every similar pair is found by exactly one probe -- the later of
// its two strings in sid order -- so joins over disjoint probe ranges return
// disjoint pair sets whose union is the whole join.  Pairs with a string too
// short to partition are verified directly by the join whose `fallback` is
// set (by default: the one whose range starts at sid 0).
static void self_join_impl(pj_index& idx, int tau, pj_result* out, bool on_device, uint32_t q_lo = 0,
                           uint32_t q_hi = UINT32_MAX, int fallback = -1) {
  trace_mark(idx.ctx, "join: start");
  const bool whole = q_lo == 0 && q_hi >= idx.n && fallback != 0;
  float part_ms = 0.f;
  ensure_partition(idx, tau, &part_ms);
  struct DumpAfter {
    pj_index& idx;
    int tau;
    ~DumpAfter() {
      if (!getenv("PJ_DEBUG_DUMP")) return;
      try {
        debug_dump(idx.ctx, "after_postings", idx.parts[tau].postings.p, idx.parts[tau].postings.bytes());
        debug_dump(idx.ctx, "after_sbytes", idx.sbytes.p, idx.sbytes.bytes());
        debug_dump(idx.ctx, "after_soff", idx.soff.p, idx.soff.bytes());
        debug_dump(idx.ctx, "after_slen", idx.slen.p, idx.slen.bytes());
      } catch (...) {
      }
    }
  } dump_after{idx, tau};
  const Partition& part = idx.parts[tau];
  ProbeView v = index_side(idx, part);
  v.pbytes = idx.sbytes.p;
  v.poff = idx.soff.p;
  v.plen = idx.slen.p;
  const uint32_t q_end = std::min<uint32_t>(q_hi, idx.n);
  v.pbegin = std::min(std::max(part.first, q_lo), q_end);
  v.pcount = q_end - v.pbegin;
  const uint32_t fb_count = (fallback < 0 ? q_lo == 0 : fallback != 0) ? part.first : 0u;
  v.pid = idx.perm.p;
  v.pref = idx.sref.p;
  v.pbm = idx.sbm.p;
  v.phash = idx.sph.p;
  v.key_shift = bits_for(idx.n);
  v.gorder = part.gorder[1].p;
  v.warp_q_cut = UINT32_MAX;
  float tune_ms = 0.f;
  TuneResult tr;
  if (v.pcount) {
    tr = self_join_tuning(idx, v, &tune_ms);
  } else {  // nothing to probe: only the fallback (if any) runs
    default_mode(idx, tr);
  }
  if (tr.warp_min_len <= idx.lmax && !tr.fused) v.warp_q_cut = idx.h_bbeg[std::max(0, tr.warp_min_len)];
  v.block_thread = tr.block_thread;
  v.pair_mode = tr.pair_mode;
  v.pair_warp = tr.pair_warp;
  v.fused = tr.fused;
  v.fused_warp_from = tr.warp_min_len;
  v.fused_q_cut = tr.fused_from_len <= 0 ? 0u
                  : tr.fused_from_len > idx.lmax ? UINT32_MAX
                                                 : idx.h_bbeg[tr.fused_from_len];
  if (v.pair_mode) v.hit_sides = 0;
  if (idx.graph_joins && whole) {
    if (idx.self_plans.size() < idx.parts.size()) idx.self_plans.resize(idx.parts.size());
    SelfPlan* sp = static_cast<SelfPlan*>(idx.self_plans[tau].get());
    if (sp && (sp->warp_min_len != tr.warp_min_len || sp->block_thread != tr.block_thread ||
               sp->pair_mode != tr.pair_mode || sp->pair_warp != tr.pair_warp || sp->fused != tr.fused ||
               sp->fused_from_len != tr.fused_from_len)) {
      idx.self_plans[tau].reset();  // recorded with another tuning
      sp = nullptr;
    }
    if (sp) {
      if (replay_self_plan(*sp, idx.ctx, on_device, out)) {
        out->stats.partition_ms = part_ms;
        out->stats.verify_block = tr.block_thread;
        out->stats.warp_min_len = tr.warp_min_len;
        out->stats.verify_mode = tr.pair_mode ? PJ_VERIFY_PAIRS : PJ_VERIFY_EXTENSION;
        out->stats.pair_warp = tr.pair_mode ? tr.pair_warp : 0;
        out->stats.fused = tr.fused;
        return;
      }
      pj_result_free(out);  // counts above the recorded capacities: run eagerly, record again
      idx.self_plans[tau].reset();
    }
  }
  run_join(idx.ctx, v, true, fb_count, bits_for(idx.n), on_device, out);
  if (idx.graph_joins && whole && !idx.self_plans[tau]) {
    try {  // a join that cannot be recorded (device or host memory) still has its result
      std::shared_ptr<SelfPlan> p = make_self_plan(idx, v, tr, part.first, out->stats, out->count);
      if (p) idx.self_plans[tau] = std::static_pointer_cast<void>(p);
    } catch (...) {
      cudaGetLastError();
    }
  }
  out->stats.partition_ms = part_ms;
  out->stats.verify_block = tr.block_thread;
  out->stats.warp_min_len = tr.warp_min_len;
  out->stats.tune_ms = tune_ms;
  out->stats.verify_mode = tr.pair_mode ? PJ_VERIFY_PAIRS : PJ_VERIFY_EXTENSION;
  out->stats.pair_warp = tr.pair_mode ? tr.pair_warp : 0;
  out->stats.fused = tr.fused;
}

void self_join_range(pj_index& idx, int tau, uint32_t q_lo, uint32_t q_hi, bool fallback, pj_result* out,
                     bool on_device) {
  ensure_partition(idx, tau, nullptr);
  self_join_impl(idx, tau, out, on_device, q_lo, q_hi, fallback ? 1 : 0);
}

void host_result(pj_result* out, pj_pair* pairs, uint64_t count) {
  out->pairs = pairs;
  out->count = count;
  out->on_device = 0;
  out->priv = new ResultPriv{};
}

static void probe_join_impl(const Ctx& c, const pj_index& idx, const Partition& part, const ProbeSet& R,
                            pj_result* out, bool on_device) {
  ProbeView v = index_side(idx, part);
  v.pbytes = R.bytes;
  v.poff = R.off;
  v.plen = R.len.p;
  v.pbegin = 0;
  v.pcount = R.n;
  v.pid = nullptr;
  v.pbm = R.bm.p;
  v.key_shift = bits_for(idx.n);
  v.gorder = part.gorder[0].p;
  TuneResult mode;
  default_mode(idx, mode);
  force_mode(idx, mode);
  v.pair_mode = mode.pair_mode;
  v.pair_warp = mode.pair_warp;
  if (v.pair_mode) v.hit_sides = 0;
  const bool has_short = part.first > 0;  // indexed strings too short to partition
  run_join(c, v, false, has_short ? R.n : 0, bits_for(R.n), on_device, out);
  out->stats.verify_mode = mode.pair_mode ? PJ_VERIFY_PAIRS : PJ_VERIFY_EXTENSION;
  out->stats.pair_warp = mode.pair_mode ? mode.pair_warp : 0;
}

void query_multi_impl(const Ctx& c, pj_index& idx, const ProbeSet& R, const uint8_t* h_tau, pj_result* out,
                      bool on_device) {
  const int tau_max = (int)idx.parts.size() - 1;
  int tmax = 0;
  bool present[PJ_TAU_LIMIT + 1] = {};
  std::vector<unsigned long long> qgoff((size_t)R.n + 1, 0);
  for (uint32_t q = 0; q < R.n; ++q) {
    const int t = h_tau[q];
    if (t > tau_max) fail(PJ_EINVAL, "query threshold " + std::to_string(t) + " above the index's tau_max");
    if (idx.parts[t].tau != t) fail(PJ_EINVAL, "index for tau " + std::to_string(t) + " not built");
    present[t] = true;
    tmax = std::max(tmax, t);
    qgoff[q + 1] = qgoff[q] + (unsigned long long)groups_per_probe(t, false);
  }
  std::vector<PartView> hp((size_t)tau_max + 1);
  bool has_short = false;
  for (int t = 0; t <= tau_max; ++t) {
    PartView pv{};
    if (present[t]) {
      const Partition& part = idx.parts[t];
      pv = PartView{part.table.p, part.fp.p, part.presence_bytes, part.precs.p, part.table.n - 1,
                    part.postings.p, part.n_records, part.first, t, seg_magic(t + 1), part.scheme};
      has_short |= part.first > 0;
    }
    hp[t] = pv;
  }
  DBuf<uint8_t> d_tau(c, std::max<uint32_t>(R.n, 1));
  DBuf<unsigned long long> d_qgoff(c, (size_t)R.n + 1);
  DBuf<PartView> d_parts(c, hp.size());
  if (R.n) PJ_CUDA(cudaMemcpyAsync(d_tau.p, h_tau, R.n, cudaMemcpyHostToDevice, c.stream));
  PJ_CUDA(cudaMemcpyAsync(d_qgoff.p, qgoff.data(), qgoff.size() * sizeof(unsigned long long), cudaMemcpyHostToDevice,
                          c.stream));
  PJ_CUDA(cudaMemcpyAsync(d_parts.p, hp.data(), hp.size() * sizeof(PartView), cudaMemcpyHostToDevice, c.stream));
  ProbeView v = index_side(idx, idx.parts[tmax]);
  v.pbytes = R.bytes;
  v.poff = R.off;
  v.plen = R.len.p;
  v.pbegin = 0;
  v.pcount = R.n;
  v.pid = nullptr;
  v.pbm = R.bm.p;
  v.key_shift = bits_for(idx.n);
  v.ptau = d_tau.p;
  v.qgoff = d_qgoff.p;
  v.parts = d_parts.p;
  run_join(c, v, false, has_short ? R.n : 0, bits_for(R.n), on_device, out, qgoff.data());
}

// ------------------------------------------------------------ query plan --
//
// query_multi_impl with every size kept on the device, for recording into a
// CUDA graph: each launch is sized for a capacity and reads the actual count
// from PlanSizes / Counters when it starts; nothing is read back by the host.
// Overflowing a capacity only drops writes; the totals are still counted and
// the host reruns with larger buffers.

static_assert(sizeof(Counters) == 64, "plan counters are 64 bytes");

// Lengths and group counts of the batch; queries past n get 0 groups, so the
// group offsets of every q >= n equal the total (group_of searches all cap_q).
__global__ void k_plan_groups(const uint8_t* __restrict__ bytes, const uint64_t* __restrict__ off,
                              const uint8_t* __restrict__ tau, uint32_t cap_q, const PlanSizes* __restrict__ sizes,
                              uint32_t* __restrict__ len, Sig* __restrict__ bm,
                              unsigned long long* __restrict__ gcnt) {
  const unsigned long long n = sizes->n;
  for (uint32_t q = blockIdx.x * blockDim.x + threadIdx.x; q < cap_q; q += gridDim.x * blockDim.x) {
    if (q < n) {
      len[q] = (uint32_t)(off[q + 1] - off[q]);
      bm[q] = char_signature(bytes + off[q], (int)len[q]);
      gcnt[q] = (unsigned long long)groups_per_probe((int)tau[q], false);
    } else {
      gcnt[q] = 0;
    }
  }
}

__global__ void k_plan_finish(const Counters* __restrict__ ctr, const PlanSizes* __restrict__ sizes,
                              PlanHeader* header) {
  PlanHeader h;
  h.groups = sizes->groups;
  h.hits = sizes->hits;
  h.cands = sizes->cands;
  h.accepted = ctr->accepted;
  h.pairs = sizes->pairs;
  h.lookups = ctr->lookups;
  h.cells = ctr->cells;
  h.fallback = ctr->fallback;
  h.err = ctr->err;
  h.filtered = ctr->filtered;
  h.unique = 0;
  *header = h;
}

void record_query_plan(const Ctx& c, const pj_index& idx, const PlanDev& d) {
  const int tau_max = (int)idx.parts.size() - 1;
  ProbeView v = index_side(idx, idx.parts[tau_max]);
  v.pbytes = d.bytes;
  v.poff = d.off;
  v.plen = d.len;
  v.pbegin = 0;
  v.pcount = d.cap_q;
  v.pid = nullptr;
  v.key_shift = bits_for(idx.n);
  v.ptau = d.tau;
  v.qgoff = d.qgoff;
  v.parts = d.parts;
  v.pbm = d.bm;
  bool has_short = false;
  for (int t = 0; t <= tau_max; ++t) has_short |= idx.parts[t].first > 0;
  Counters* ctr = static_cast<Counters*>(d.counters);
  PlanSizes* sz = d.sizes;
  PJ_CUDA(cudaMemsetAsync(ctr, 0, sizeof(Counters), c.stream));

  // A4: groups of every query, lookups, hits, candidate offsets
  k_plan_groups<<<stride_grid(d.cap_q), 256, 0, c.stream>>>(d.bytes, d.off, d.tau, d.cap_q, sz, d.len, d.bm, d.gcnt);
  PJ_LAUNCHED("k_plan_groups");
  exclusive_scan_dn<unsigned long long>(c, d.gcnt, d.qgoff, d.cap_q, nullptr, &sz->groups);
  const unsigned g1 = persistent_grid(k_group_counts<false, true>, (d.cap_groups + BLOCK - 1) / BLOCK);
  k_group_counts<false, true><<<g1, BLOCK, 0, c.stream>>>(v, d.cap_groups, d.gcounts, d.gmask, ctr, &sz->groups);
  PJ_LAUNCHED("k_group_counts");
  exclusive_scan_dn<uint32_t>(c, d.gcounts, d.goff, d.cap_groups, &sz->groups, &sz->hits);
  const unsigned g2 = persistent_grid(k_group_hits<false, true>, (d.cap_groups + BLOCK - 1) / BLOCK);
  k_group_hits<false, true><<<g2, BLOCK, 0, c.stream>>>(v, d.cap_groups, d.gcounts, d.gmask, d.goff, d.hits,
                                                        &sz->groups, d.cap_hits);
  PJ_LAUNCHED("k_group_hits");
  k_hit_counts<<<stride_grid(d.cap_hits), 256, 0, c.stream>>>(d.hits, d.cap_hits, d.hcnt, &sz->hits);
  PJ_LAUNCHED("k_hit_counts");
  exclusive_scan_dn<unsigned long long>(c, d.hcnt, d.hoff, d.cap_hits, &sz->hits, &sz->cands);

  // A6 + A8: verification of every candidate, then the short indexed strings
  const AccOut acc{d.acc_key[0], d.acc_ed[0], d.cap_acc};
#define PJ_CALL(W)                                                                                              \
  do {                                                                                                         \
    const unsigned gv = persistent_grid(k_verify_queued<W, false, true>, ~0ull >> 8, Q_BLOCK);                  \
    k_verify_queued<W, false, true><<<gv, Q_BLOCK, 0, c.stream>>>(v, d.hits, d.hoff, d.cap_hits, 0, 0, acc, ctr, \
                                                                  &sz->hits, Q_CHUNK);                         \
    PJ_LAUNCHED("k_verify_queued");                                                                            \
    if (has_short) {                                                                                           \
      const unsigned gf = persistent_grid(k_fallback<W, false, true>, (d.cap_q + BLOCK - 1) / BLOCK);           \
      k_fallback<W, false, true><<<gf, BLOCK, 0, c.stream>>>(v, d.cap_q, acc, ctr, &sz->n);                     \
      PJ_LAUNCHED("k_fallback");                                                                               \
    }                                                                                                          \
  } while (0)
  PJ_BY_TAU(tau_max, PJ_CALL);
#undef PJ_CALL

  // A5 + A7: sort the accepted matches, keep each key's least ed, compact
  const int nbits = v.key_shift + bits_for(d.cap_q);
  const bool second = radix_sort_pairs_dn<unsigned long long>(c, d.acc_key[0], d.acc_ed[0], d.acc_key[1],
                                                              d.acc_ed[1], d.cap_acc, &ctr->accepted, nbits);
  const unsigned long long* keys = d.acc_key[second ? 1 : 0];
  const uint32_t* eds = d.acc_ed[second ? 1 : 0];
  k_run_heads<<<stride_grid(d.cap_acc), 256, 0, c.stream>>>(keys, d.cap_acc, d.flags, &ctr->accepted);
  PJ_LAUNCHED("k_run_heads");
  exclusive_scan_dn<uint32_t>(c, d.flags, d.pos, d.cap_acc, &ctr->accepted, &sz->pairs);
  k_emit_pairs<<<stride_grid(d.cap_acc), 256, 0, c.stream>>>(keys, eds, d.flags, d.pos, d.cap_acc, v.key_shift,
                                                             d.out_pairs, &ctr->accepted, d.cap_pairs);
  PJ_LAUNCHED("k_emit_pairs");
  k_plan_finish<<<1, 1, 0, c.stream>>>(ctr, sz, d.header);
  PJ_LAUNCHED("k_plan_finish");
}

}  // namespace pj

// ------------------------------------------------------------------ C ABI --

static void clear_result(pj_result* out) {
  if (out) memset(out, 0, sizeof(*out));
}

extern "C" {

int pj_self_join(pj_index* idx, int tau, pj_result* out) {
  clear_result(out);
  try {
    if (!idx || !out) pj::fail(PJ_EINVAL, "pj_self_join: NULL argument");
    if (tau < 0 || tau >= (int)idx->parts.size()) pj::fail(PJ_EINVAL, "pj_self_join: tau outside 0..tau_max");
    std::lock_guard<std::mutex> g(idx->mu);
    pj::self_join_impl(*idx, tau, out, idx->results_on_device);
    if (idx->ctx.budget) out->stats.device_peak = idx->ctx.budget->peak;
    return PJ_OK;
  } catch (const pj::Error& e) {
    pj::set_last_error(e.msg);
    pj_result_free(out);
    return e.code;
  } catch (const std::bad_alloc&) {
    pj::set_last_error("host allocation failed");
    pj_result_free(out);
    return PJ_ENOMEM;
  }
}

int pj_count_selection(pj_index* idx, int tau, pj_selection* out) {
  if (out) memset(out, 0, sizeof(*out));
  try {
    if (!idx || !out) pj::fail(PJ_EINVAL, "pj_count_selection: NULL argument");
    if (tau < 0 || tau >= (int)idx->parts.size()) pj::fail(PJ_EINVAL, "pj_count_selection: tau outside 0..tau_max");
    std::lock_guard<std::mutex> g(idx->mu);
    const pj::Ctx& c = idx->ctx;
    pj::ProbeView v{};
    v.plen = idx->slen.p;
    v.ibbeg = idx->bbeg.p;
    v.ilmax = idx->lmax;
    v.tau = tau;
    v.seg_magic = pj::seg_magic(tau + 1);
    v.scheme = idx->scheme;
    v.pbegin = tau + 1 <= idx->lmax ? idx->h_bbeg[tau + 1] : idx->n;  // shorter probes select nothing
    v.pcount = idx->n - v.pbegin;
    const unsigned long long n_groups = (unsigned long long)v.pcount * pj::groups_per_probe(tau, true);
    pj::DBuf<pj::SelCounts> d(c, 1);
    PJ_CUDA(cudaMemsetAsync(d.p, 0, sizeof(pj::SelCounts), c.stream));
    if (n_groups) {
      pj::k_selection_counts<<<pj::stride_grid(n_groups), pj::BLOCK, 0, c.stream>>>(v, n_groups, d.p);
      PJ_LAUNCHED("k_selection_counts");
    }
    pj::SelCounts h{};
    PJ_CUDA(cudaMemcpyAsync(&h, d.p, sizeof(h), cudaMemcpyDeviceToHost, c.stream));
    c.sync();
    out->length_based = h.w[0];
    out->shift_based = h.w[1];
    out->position_aware = h.w[2];
    out->multi_match = h.w[3];
    out->groups = h.groups;
    return PJ_OK;
  } catch (const pj::Error& e) {
    pj::set_last_error(e.msg);
    return e.code;
  }
}

int pj_join(const pj_strings* R, const pj_strings* S, int tau, const pj_options* opt, pj_result* out) {
  clear_result(out);
  pj_index* tmp = nullptr;
  try {
    if (!R || !S || !out) pj::fail(PJ_EINVAL, "pj_join: NULL argument");
    if (tau < 0 || tau > PJ_TAU_LIMIT) pj::fail(PJ_EINVAL, "pj_join: tau out of range");
    tmp = new pj_index();
    tmp->ctx = pj::make_ctx(opt);
    tmp->results_on_device = opt ? opt->results_on_device != 0 : false;
    tmp->verify_mode = opt ? opt->verify_mode : PJ_VERIFY_AUTO;
    tmp->scheme = opt ? opt->partition : PJ_PARTITION_EVEN;
    if (tmp->scheme != PJ_PARTITION_EVEN && tmp->scheme != PJ_PARTITION_CENTER)
      pj::fail(PJ_EINVAL, "pj_join: unknown partition scheme");
    PJ_CUDA(cudaGetDevice(&tmp->device));
    pj::build_store(*tmp, *S);
    tmp->parts.resize(tau + 1);
    pj::build_partition(*tmp, tau, tmp->parts[tau]);
    {  // the probe set's buffers refer to tmp->ctx: released before tmp
      pj::ProbeSet P;
      pj::upload_probe_set(tmp->ctx, *R, P);
      pj::probe_join_impl(tmp->ctx, *tmp, tmp->parts[tau], P, out, tmp->results_on_device);
      tmp->ctx.sync();
    }
    if (tmp->ctx.budget) out->stats.device_peak = tmp->ctx.budget->peak;
    delete tmp;
    return PJ_OK;
  } catch (const pj::Error& e) {
    pj::set_last_error(e.msg);
    pj_result_free(out);
    delete tmp;
    return e.code;
  } catch (const std::bad_alloc&) {
    pj::set_last_error("host allocation failed");
    pj_result_free(out);
    delete tmp;
    return PJ_ENOMEM;
  }
}

int pj_query(pj_index* idx, const pj_strings* batch, int tau, pj_result* out) {
  clear_result(out);
  try {
    if (!idx || !batch || !out) pj::fail(PJ_EINVAL, "pj_query: NULL argument");
    if (tau < 0 || tau >= (int)idx->parts.size()) pj::fail(PJ_EINVAL, "pj_query: tau outside 0..tau_max");
    std::lock_guard<std::mutex> g(idx->mu);
    float part_ms = 0.f;
    pj::Partition& part = pj::ensure_partition(*idx, tau, &part_ms);
    pj::ProbeSet P;
    pj::upload_probe_set(idx->ctx, *batch, P);
    pj::probe_join_impl(idx->ctx, *idx, part, P, out, idx->results_on_device);
    out->stats.partition_ms = part_ms;
    return PJ_OK;
  } catch (const pj::Error& e) {
    pj::set_last_error(e.msg);
    pj_result_free(out);
    return e.code;
  } catch (const std::bad_alloc&) {
    pj::set_last_error("host allocation failed");
    pj_result_free(out);
    return PJ_ENOMEM;
  }
}

int pj_query_multi(pj_index* idx, const pj_strings* batch, const uint8_t* taus, pj_result* out) {
  clear_result(out);
  try {
    if (!idx || !batch || !out || (!taus && batch->n)) pj::fail(PJ_EINVAL, "pj_query_multi: NULL argument");
    std::lock_guard<std::mutex> g(idx->mu);
    bool seen[PJ_TAU_LIMIT + 1] = {};
    for (uint32_t q = 0; q < batch->n; ++q) {
      if ((int)taus[q] >= (int)idx->parts.size()) pj::fail(PJ_EINVAL, "pj_query_multi: tau outside 0..tau_max");
      seen[taus[q]] = true;
    }
    for (int t = 0; t < (int)idx->parts.size(); ++t)
      if (seen[t]) pj::ensure_partition(*idx, t, nullptr);
    pj::ProbeSet P;
    pj::upload_probe_set(idx->ctx, *batch, P);
    pj::query_multi_impl(idx->ctx, *idx, P, taus, out, idx->results_on_device);
    return PJ_OK;
  } catch (const pj::Error& e) {
    pj::set_last_error(e.msg);
    pj_result_free(out);
    return e.code;
  } catch (const std::bad_alloc&) {
    pj::set_last_error("host allocation failed");
    pj_result_free(out);
    return PJ_ENOMEM;
  }
}

void pj_result_free(pj_result* res) {
  if (!res) return;
  auto* priv = static_cast<pj::ResultPriv*>(res->priv);
  if (res->pairs) {
    if (res->on_device) {
      if (priv) {
        priv->ctx.put(res->pairs);
        cudaStreamSynchronize(priv->ctx.stream);
      }
    } else if (priv && priv->pinned_bytes) {
      pj::pinned_put(res->pairs, priv->pinned_bytes);
    } else {
      free(res->pairs);
    }
  }
  delete priv;
  memset(res, 0, sizeof(*res));
}

}  // extern "C"
