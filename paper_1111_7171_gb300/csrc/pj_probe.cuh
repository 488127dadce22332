// Per-thread steps of selection, probing and verification (Sec. 4.2, Alg. 2,
// Sec. 5.2, Alg. 3), shared by the kernels and by host-side checks.
//
// Work is split into two collective-free phases:
//   * a "group" is one (probing string q, indexed length l, segment i); its
//     multi-match window gives at most tau + 1 positions p, each one lookup;
//     a lookup whose (filtered) posting run is non-empty becomes a Hit;
//   * a "candidate" is one posting of a Hit's run, i.e. one match
//     (q, r, i, p), verified by extension-based verification.
#pragma once

#include "pj_internal.cuh"
#include "pj_verify.cuh"

namespace pj {

// A lookup with a non-empty posting run.  pi = p | (i << 16) | (tau << 24);
// the tau byte is used by multi-threshold batches only.  sl and sr are the
// side signatures (side_signature) of the probe left of the selected
// substring, s[0, p), and right of it, s[p + l_i, |s|), for the screen in
// front of extension verification.
struct __align__(16) Hit {
  uint32_t q;
  uint32_t begin;
  uint32_t count;
  uint32_t pi;
  unsigned long long sl, sr;
};

// One threshold's segment index, as seen by the kernels.
struct PartView {
  const Slot* table;
  const uint8_t* fp;  // slot fingerprints, then the presence bitmap
  unsigned pb;        // presence bitmap bytes per slot
  const PostRec* precs;
  unsigned long long mask;
  const uint32_t* postings;
  unsigned long long n_postings;
  uint32_t first;  // first sid of length >= tau + 1
  int tau;
  unsigned long long seg_magic;  // seg_magic(tau + 1)
  int scheme;                    // partition scheme (PJ_PARTITION_*)
};

struct ProbeView {
  // probing strings: id q has bytes pbytes[poff[q] .. poff[q] + plen[q])
  const uint8_t* pbytes;
  const uint64_t* poff;
  const uint32_t* plen;
  uint32_t pbegin, pcount;  // probe ids pbegin .. pbegin + pcount - 1
  const uint32_t* pid;      // probe id -> reported id (NULL: identity)
  const unsigned long long* pref;  // poff << 16 | plen in one word (NULL: read poff and plen)
  // indexed strings, sid order
  const uint8_t* ibytes;
  const uint64_t* ioff;
  const uint32_t* ilen;
  const unsigned long long* iref;  // ioff << 16 | ilen in one word (NULL: read ioff and ilen)
  const uint32_t* ibbeg;  // first sid of each length, ilmax + 2 entries
  int ilmax;
  const uint32_t* iperm;  // sid -> reported id
  uint32_t n_index;
  const Slot* table;
  const uint8_t* table_fp;  // slot fingerprints, then the presence bitmap (NULL: probe the slots directly)
  unsigned table_pb;        // presence bitmap bytes per slot
  const uint32_t* phash;    // probe-side prefix values from poff[q] + q (NULL: computed per window)
  unsigned long long mask;
  const uint32_t* postings;
  const PostRec* precs;  // postings' records (same order)
  unsigned long long n_postings;
  int tau;
  unsigned long long seg_magic;  // seg_magic(tau + 1): partitions without a division
  int scheme;                    // partition scheme of the indexed strings (PJ_PARTITION_*)
  int key_shift;  // pair key = a << key_shift | b
  // multi-threshold batches (R != S only): probe q has threshold ptau[q],
  // its groups are qgoff[q] .. qgoff[q+1]-1, parts[tau] is tau's index
  const uint8_t* ptau;
  const unsigned long long* qgoff;
  const PartView* parts;
  // self join: probes q >= warp_q_cut (the long ones; probes are in length
  // order) are verified one warp per candidate; UINT32_MAX = never
  uint32_t warp_q_cut;
  int block_thread;  // block size of the thread-per-candidate verification
  int interleave;    // probe groups interleaved across probes (see group_of)
  const uint16_t* gorder;  // groups of one probe in visiting order (NULL: natural order)
  // character signatures of the probing and the indexed strings (NULL: no
  // character-count bound)
  const Sig* pbm;
  const Sig* ibm;
  int queued;     // thread-per-candidate verification with a screen and per-warp queues
  int hit_sides;  // hits carry the probe's side signatures (Hit::sl, sr) and the queued screen tests them
  int pair_mode;  // 1: mode L (distinct candidate pairs verified once over the whole strings)
  int pair_warp;  // mode L: one warp per pair instead of one thread
  int share_prefix;  // mode L: consecutive pairs of a probe share the DP rows of common prefixes (Sec. 5.3)
  int fused;         // self join, mode L: one persistent select/probe/verify kernel (k_fused_self)
  int fused_warp_from;  // fused form: probes at least this long verify their pairs one warp per pair
  uint32_t fused_q_cut;  // fused form: probes q >= fused_q_cut run in the fused kernel, the shorter ones
                         // (the longest posting runs) in the chunked mode-L pipeline
  int block_warp;    // block size of the warp-per-candidate verification
};

// The view of threshold tau inside a multi-threshold batch.
__host__ __device__ __forceinline__ ProbeView view_for_tau(const ProbeView& v, int tau) {
  ProbeView t = v;
  const PartView& pv = v.parts[tau];
  t.table = pv.table;
  t.table_fp = pv.fp;
  t.table_pb = pv.pb;
  t.precs = pv.precs;
  t.mask = pv.mask;
  t.postings = pv.postings;
  t.n_postings = pv.n_postings;
  t.tau = tau;
  t.seg_magic = pv.seg_magic;
  t.scheme = pv.scheme;
  return t;
}

// Groups per probing string: lengths |s|-tau..|s| (self join, Alg. 1)
// or |s|-tau..|s|+tau (R != S, Sec. 3.2), times tau + 1 segments.
__host__ __device__ __forceinline__ int groups_per_probe(int tau, bool self) {
  return (tau + 1) * (self ? tau + 1 : 2 * tau + 1);
}

// The lists of group g of probing string q (length ls): indexed length l,
// segment i, its even-partition start P and length li.  False when L_l^i is
// empty when q probes it (no such length indexed, or no string of it visited
// before q).
__host__ __device__ __forceinline__ bool group_lists(const ProbeView& v, bool self, uint32_t q, int ls, int g,
                                                     int& l, int& i, int& P, int& li) {
  const int tau = v.tau, parts = tau + 1;
  l = ls - tau + g / parts;
  i = 1 + g % parts;
  if (l < parts || l > v.ilmax) return false;
  const uint32_t b0 = v.ibbeg[l];
  uint32_t b1 = v.ibbeg[l + 1];
  if (self && l == ls && b1 > q) b1 = q;  // only strings visited before q
  if (b1 <= b0) return false;
  segment_m(l, parts, v.seg_magic, v.scheme, i, P, li);
  return true;
}

// Group g's multi-match window [lo, hi] of start positions in q (Sec. 4.2):
//   lo = max(P - (i-1), P + D - (tau+1-i)),  hi = min(P + (i-1), P + D + (tau+1-i)),
// clipped to [0, ls - li], with D = ls - l.  False when the group selects
// nothing (empty lists or an empty window).
__host__ __device__ __forceinline__ bool group_window(const ProbeView& v, bool self, uint32_t q, int ls, int g,
                                                      int& l, int& i, int& P, int& li, int& lo, int& hi) {
  if (!group_lists(v, self, q, ls, g, l, i, P, li)) return false;
  const int parts = v.tau + 1;
  const int D = ls - l;
  lo = max(0, max(P - (i - 1), P + D - (parts - i)));
  hi = min(ls - li, min(P + (i - 1), P + D + (parts - i)));
  return hi >= lo;
}

// floor(a / 2) for any sign of a
__host__ __device__ __forceinline__ int floor_half(int a) { return a >= 0 ? a / 2 : -((1 - a) / 2); }

// Sizes of the start-position windows that each selection method of Sec. 4
// picks for group g (substrings s[p, l_i] that exist in s, 0 <= p <= |s| -
// l_i): w[0] length-based (every position), w[1] shift-based ([P_i - tau,
// P_i + tau]), w[2] position-aware (Sec. 4.1, [P_i - floor((tau - D)/2),
// P_i + floor((tau + D)/2)]), w[3] multi-match-aware (Sec. 4.2, the window
// the join looks up); D = |s| - l.  False when the group's lists are empty.
__host__ __device__ __forceinline__ bool group_selection_sizes(const ProbeView& v, bool self, uint32_t q, int ls,
                                                               int g, int (&w)[4]) {
  int l, i, P, li;
  w[0] = w[1] = w[2] = w[3] = 0;
  if (!group_lists(v, self, q, ls, g, l, i, P, li)) return false;
  const int tau = v.tau, parts = tau + 1, D = ls - l, last = ls - li;
  if (last < 0) return true;
  const int lo[4] = {0, P - tau, P - floor_half(tau - D), max(P - (i - 1), P + D - (parts - i))};
  const int hi[4] = {last, P + tau, P + floor_half(tau + D), min(P + (i - 1), P + D + (parts - i))};
#pragma unroll
  for (int m = 0; m < 4; ++m) w[m] = max(0, min(hi[m], last) - max(lo[m], 0) + 1);
  return true;
}

__host__ __device__ __forceinline__ int table_find_any(const Slot* t, const uint8_t* fp, unsigned pb,
                                                       unsigned long long mask, unsigned long long key,
                                                       uint32_t& begin, uint32_t& count) {
  return table_find(t, fp, pb, mask, key, begin, count);
}

// Lookup of the key of s[p, li] in L_l^i.  Returns the number of postings to
// verify (for the self join with l == |s|, only sids below q: runs ascend)
// and sets begin.  err |= 1 for a run outside the postings, 2 for the probe
// limit.
__host__ __device__ __forceinline__ uint32_t lookup_key(const ProbeView& v, bool self, uint32_t q, int ls, int l,
                                                        unsigned long long key, uint32_t& begin, int& err) {
  uint32_t cnt = 0;
  begin = 0;
  const int found = table_find_any(v.table, v.table_fp, v.table_pb, v.mask, key, begin, cnt);
  if (found < 0) {
    err |= 2;
    return 0;
  }
  if (found == 0) return 0;
  if ((unsigned long long)begin + cnt > v.n_postings) {
    err |= 1;
    return 0;
  }
  if (self && l == ls) {
    uint32_t x0 = 0, x1 = cnt;
    while (x0 < x1) {
      const uint32_t mid = (x0 + x1) >> 1;
      if (v.postings[begin + mid] < q) x0 = mid + 1; else x1 = mid;
    }
    cnt = x0;
  }
  return cnt;
}

// Work item `it` (0 <= it < n_items, n_items = ceil(pcount / ppi)) of the
// fused self join: the items are handed out from the two ends of the probes'
// length order in turn (longest, shortest, second longest, ...), so item
// `it` is position j from the long end (returned) and covers probes
// [q_beg, q_end), ppi of them except the shortest item.
__host__ __device__ __forceinline__ unsigned long long fused_item(unsigned long long it, unsigned long long n_items,
                                                                  uint32_t pbegin, uint32_t pcount, int ppi,
                                                                  uint32_t& q_beg, uint32_t& q_end) {
  const unsigned long long j = (it & 1) ? n_items - 1 - (it >> 1) : (it >> 1);
  q_end = (uint32_t)((unsigned long long)pbegin + pcount - j * (unsigned long long)ppi);
  q_beg = q_end > pbegin + (uint32_t)ppi ? q_end - (uint32_t)ppi : pbegin;
  return j;
}

// The lookups of a group's window: substrings s[p, li], p = lo .. hi, in
// L_l^i, their keys rolled from one position to the next.  f(p, begin,
// count) is called, in order of p, for every lookup that found postings to
// verify.  (Loading the presence words of 8 positions back to back, so that
// their latencies overlap, measured slower: the loop is bound by its integer
// instructions, and the batch's extra registers cost occupancy.  Testing the
// whole window's presence bits first and looking up the passing positions
// after measured 5% faster on long strings at tau 32 and slower elsewhere.)
template <class F>
__device__ __forceinline__ void window_lookups(const ProbeView& v, bool self, uint32_t q, int ls, int l, int i, int li,
                                               int lo, int hi, const uint8_t* s, int& err, F f) {
  const uint32_t pw = seg_pow(li);
  uint32_t V = v.phash && li > SEG_EXACT_MAX ? seg_value_from_prefix(v.phash + v.poff[q] + q, lo, li, pw)
                                             : seg_value(s + lo, li);
  for (int p = lo;; ++p) {
    uint32_t b;
    const uint32_t cnt = lookup_key(v, self, q, ls, l, seg_key_of(V, l, i), b, err);
    if (cnt) f(p, b, cnt);
    if (p == hi) break;
    V = seg_roll(V, s[p], s[p + li], li, pw);  // p + li <= hi - 1 + li < ls
  }
}

// Lookup of s[p, li] in L_l^i (lookup_key with the key computed here).
__host__ __device__ __forceinline__ uint32_t lookup(const ProbeView& v, bool self, const uint8_t* s, int ls,
                                                    uint32_t q, int l, int i, int p, int li, uint32_t& begin,
                                                    int& err) {
  return lookup_key(v, self, q, ls, l, seg_key(s + p, li, l, i), begin, err);
}

// What the verification of a candidate needs from its hit: the probing
// string, the matched position p and the segment number i.
struct HitCtx {
  uint32_t q, begin;
  int p, i, ls;
  const uint8_t* s;
};

__host__ __device__ __forceinline__ HitCtx hit_ctx(const ProbeView& v, const Hit& h) {
  HitCtx c;
  c.q = h.q;
  c.begin = h.begin;
  c.p = (int)(h.pi & 0xFFFFu);
  c.i = (int)((h.pi >> 16) & 0xFFu);
  c.ls = (int)v.plen[h.q];
  c.s = v.pbytes + v.poff[h.q];
  return c;
}

// Extension verification (Sec. 5.2, Alg. 3) of indexed string r against the
// hit described by hc, r already screened (a valid sid, not the probe
// itself).  Returns true with the pair key and ed = d_l + d_r when accepted.
template <int MAXW>
__host__ __device__ __forceinline__ bool verify_screened(const ProbeView& v, bool self, const HitCtx& hc, uint32_t r,
                                                         unsigned long long& key, int& ed,
                                                         unsigned long long& cells) {
  // Single exit: see vsp().
  bool ok = false;
  const int i = hc.i;
  // r's length and bytes: one load of its packed reference, so that the
  // byte loads do not wait for a second dependent load
  int lr;
  const uint8_t* rb;
  if (v.iref) {
    const unsigned long long ref = v.iref[r];
    lr = (int)(ref & 0xFFFFu);
    rb = v.ibytes + (ref >> 16);
  } else {
    lr = (int)v.ilen[r];
    rb = v.ibytes + v.ioff[r];
  }
  if (i >= 1 && i <= v.tau + 1 && lr >= v.tau + 1) {  // r is a partitioned string
    int P, li;
    segment_m(lr, v.tau + 1, v.seg_magic, v.scheme, i, P, li);
    // exact keys (segments of at most SEG_EXACT_MAX bytes) guarantee the
    // segment match; hashed ones are compared
    if (hc.p + li <= hc.ls && verify_ext<MAXW>(hc.s, hc.ls, rb, lr, i, hc.p, li, P, v.tau,
                                               li > SEG_EXACT_MAX, ed, cells)) {
      const uint32_t qid = v.pid ? v.pid[hc.q] : hc.q;
      const uint32_t rid = v.iperm[r];
      const uint32_t ka = self ? min(qid, rid) : qid;
      const uint32_t kb = self ? max(qid, rid) : rid;
      key = ((unsigned long long)ka << v.key_shift) | kb;
      ok = true;
    }
  }
  return ok;
}

// The screen in front of every verification: r must be a valid sid (else
// err |= 1), not the probe itself (a colliding run may hold it), and pass
// the character-count bound (else ++filtered).
__host__ __device__ __forceinline__ bool screen_candidate(const ProbeView& v, bool self, uint32_t q, uint32_t r,
                                                          unsigned long long& filtered, int& err) {
  bool pass = false;
  if (r >= v.n_index) {
    err |= 1;
  } else if (!(self && r == q)) {
    if (v.pbm && signature_bound(v.pbm[q], v.ibm[r]) > v.tau) ++filtered;
    else pass = true;
  }
  return pass;
}

// Verify candidate `off` of the hit described by hc (screen, then
// verify_screened).
template <int MAXW>
__host__ __device__ __forceinline__ bool verify_in_hit(const ProbeView& v, bool self, const HitCtx& hc, uint32_t off,
                                                       unsigned long long& key, int& ed, unsigned long long& cells,
                                                       unsigned long long& filtered, int& err) {
  const uint32_t r = v.postings[hc.begin + off];
  return screen_candidate(v, self, hc.q, r, filtered, err) && verify_screened<MAXW>(v, self, hc, r, key, ed, cells);
}

// Verify candidate `off` of hit h (see verify_in_hit).
template <int MAXW>
__host__ __device__ __forceinline__ bool verify_candidate(const ProbeView& v, bool self, const Hit& h, uint32_t off,
                                                          unsigned long long& key, int& ed,
                                                          unsigned long long& cells, int& err) {
  unsigned long long filtered = 0;
  return verify_in_hit<MAXW>(v, self, hit_ctx(v, h), off, key, ed, cells, filtered, err);
}

#ifdef __CUDACC__
// verify_candidate for a whole warp on one candidate (long strings); every
// lane must call it with the same arguments.
__device__ __forceinline__ bool verify_candidate_warp(const ProbeView& v, bool self, const Hit& h, uint32_t off,
                                                      unsigned long long& key, int& ed, unsigned long long& cells,
                                                      int& err) {
  bool ok = false;
  const uint32_t r = v.postings[h.begin + off];
  const uint32_t q = h.q;
  const int p = (int)(h.pi & 0xFFFFu);
  const int i = (int)((h.pi >> 16) & 0xFFu);
  if (r >= v.n_index) {
    err |= 1;
  } else if (!(self && r == q) && !(v.pbm && signature_bound(v.pbm[q], v.ibm[r]) > v.tau)) {
    const int ls = (int)v.plen[q];
    const int lr = (int)v.ilen[r];
    if (i >= 1 && i <= v.tau + 1 && lr >= v.tau + 1) {
      int P, li;
      segment_m(lr, v.tau + 1, v.seg_magic, v.scheme, i, P, li);
      if (p + li <= ls &&
          verify_ext_warp(v.pbytes + v.poff[q], ls, v.ibytes + v.ioff[r], lr, i, p, li, P, v.tau, li > SEG_EXACT_MAX,
                          ed, cells)) {
        const uint32_t qid = v.pid ? v.pid[q] : q;
        const uint32_t rid = v.iperm[r];
        const uint32_t ka = self ? min(qid, rid) : qid;
        const uint32_t kb = self ? max(qid, rid) : rid;
        key = ((unsigned long long)ka << v.key_shift) | kb;
        ok = true;
      }
    }
  }
  return ok;
}
#endif

}  // namespace pj
