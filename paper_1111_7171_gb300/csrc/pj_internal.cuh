// Internal data layout of the GB300 Pass-Join index.
//
// Strings live in HBM in "sorted-id" (sid) order: ascending length, then
// ascending first eight bytes (first byte highest, zero-padded), then input
// id -- close to the alphabetical order Alg. 1 visits in, so that strings
// with long common prefixes are neighbours.  Strings of one length l occupy the contiguous sid
// range [bbeg[l], bbeg[l+1]), which is the paper's group S_l (Sec. 3.2), and
// "visited before" in the self join (Alg. 1: by length, then a fixed order)
// becomes plain sid order.
//
// For each threshold tau the index holds the tau+1 even segments (Sec. 3.1)
// of every string of length >= tau+1 as records (key, sid), where the key is
// a 64-bit hash of (l, i, segment bytes).  Records sorted by key give the
// inverted lists L_l^i(w) as contiguous runs of the postings array (sids in
// ascending order inside a run); an open-addressing table maps a key to its
// run.  Hash collisions only merge runs: every candidate's segment is
// byte-compared before verification, so results stay exact.
#pragma once

#include <algorithm>
#include <cstring>
#include <memory>
#include <mutex>
#include <vector>

#include "pj_common.cuh"

namespace pj {

#ifndef __CUDA_ARCH__
using std::max;
using std::min;
#endif

struct __align__(16) Slot {
  unsigned long long key;  // 0 = empty
  uint32_t begin;          // first posting of the run
  uint32_t count;          // run length
};

// Reciprocal of the segment count for even_segment_m: m = ceil(2^32 / parts).
__host__ __device__ __forceinline__ unsigned long long seg_magic(int parts) {
  return parts < 1 ? 0ull : ((1ull << 32) + (unsigned long long)parts - 1ull) / (unsigned long long)parts;
}

// Even partition (Sec. 3.1) of a length-l string into tau+1 segments: the
// first tau+1-k have floor(l/(tau+1)) characters, the last k one more, with
// k = l - floor(l/(tau+1))*(tau+1).  Segment i is 1-based; P = 0-based start.
//
// floor(l / parts) is one multiply by m = seg_magic(parts) (0: computed
// here): m exceeds 2^32 / parts by less than 1, so l * m / 2^32 exceeds
// l / parts by less than l / 2^32 < 2^-16 for l < 2^16, while the
// fractional part of l / parts is at most 1 - 1/parts <= 1 - 2^-6; the
// floor is exact for every string length (< 2^16) and tau <= 32.
__host__ __device__ __forceinline__ void even_segment_m(int l, int parts, unsigned long long m, int i, int& P,
                                                        int& li) {
  if (m == 0) m = seg_magic(parts);
  const int base = (int)(((unsigned long long)(unsigned)l * m) >> 32);
  const int k = l - base * parts;
  const int first_long = parts - k + 1;  // segments i >= first_long are longer
  li = base + (i >= first_long ? 1 : 0);
  P = (i - 1) * base + (i > first_long ? i - first_long : 0);
}

__host__ __device__ __forceinline__ void even_segment(int l, int tau, int i, int& P, int& li) {
  const int parts = tau + 1;
  const int base = l / parts;
  const int k = l - base * parts;
  const int first_long = parts - k + 1;  // segments i >= first_long are longer
  li = base + (i >= first_long ? 1 : 0);
  P = (i - 1) * base + (i > first_long ? i - first_long : 0);
}

// Partition schemes (pj_options.partition).  Both cut a length-l string into
// parts = tau + 1 segments of floor(l / parts) characters, k = l - floor(l /
// parts) * parts of them one longer; they differ in which segments are the
// longer ones:
//   PJ_PARTITION_EVEN   the last k (Sec. 3.1, the paper's even partition);
//   PJ_PARTITION_CENTER the k segments nearest the middle (ordered by
//                       |2i - (parts + 1)|, ties to the left), where the
//                       multi-match windows (Sec. 4.2) are widest, so that
//                       the more selective segments are looked up at the most
//                       positions.
// The longer segments form one run [lo, hi] in both: the last k for EVEN;
// for CENTER, with c the middle segment (the left one of the two middles
// when parts is even), lo = c - floor(k / 2), hi = c + floor((k - 1) / 2)
// for odd parts and lo = c - floor((k - 1) / 2), hi = c + floor(k / 2) for
// even parts.  Then l_i = base + [lo <= i <= hi] and P_i = (i - 1) * base +
// min(max(i - lo, 0), k).  Multi-match selection, extension verification
// and the completeness of Lemma 1 only need the segments to depend on the
// length alone, which both schemes satisfy.
__host__ __device__ __forceinline__ void scheme_segment(int l, int parts, int base, int scheme, int i, int& P,
                                                        int& li) {
  const int k = l - base * parts;
  int lo;
  if (scheme == PJ_PARTITION_CENTER) {
    const int c = (parts + 1) >> 1;
    lo = (parts & 1) ? c - (k >> 1) : c - ((k - 1) >> 1);  // k = 0: an empty run (lo > hi)
  } else {
    lo = parts - k + 1;
  }
  const int hi = lo + k - 1;
  li = base + (i >= lo && i <= hi ? 1 : 0);
  P = (i - 1) * base + min(max(i - lo, 0), k);
}

// The partition of the given scheme, floor(l / parts) by the multiply of
// even_segment_m (m = seg_magic(parts), or 0 to compute it).
__host__ __device__ __forceinline__ void segment_m(int l, int parts, unsigned long long m, int scheme, int i, int& P,
                                                   int& li) {
  if (scheme == PJ_PARTITION_EVEN) {
    even_segment_m(l, parts, m, i, P, li);
    return;
  }
  if (m == 0) m = seg_magic(parts);
  const int base = (int)(((unsigned long long)(unsigned)l * m) >> 32);
  scheme_segment(l, parts, base, scheme, i, P, li);
}

// Segment keys: key = V << 32 | l << 8 | i for segment i of a length-l
// string, where V is
//   * the segment's bytes themselves (first byte lowest) when it has at most
//     SEG_EXACT_MAX bytes -- then equal keys mean equal segments, and
//     candidates found through such a key need no byte compare;
//   * otherwise the polynomial hash V = sum_k x[k] * SEG_B^(n-1-k) mod 2^32,
//     which the probe rolls from one window position to the next in O(1):
//     V(x[p+1 .. p+1+n)) = (V(x[p .. p+n)) - x[p] * SEG_B^(n-1)) * SEG_B + x[p+n].
// l and i are stored exactly, so only hashed segments of the same (l, i)
// can share a key; that merges their posting runs, and every candidate of a
// hashed key has its segment bytes compared before verification.  Keys are
// never 0 (i >= 1), which marks an empty table slot.
constexpr int SEG_EXACT_MAX = 4;
constexpr uint32_t SEG_B = 0x9E3779B1u;  // odd

__host__ __device__ __forceinline__ uint32_t seg_value(const uint8_t* p, int len) {
  uint32_t v = 0;
  if (len <= SEG_EXACT_MAX) {
    for (int k = 0; k < len; ++k) v |= (uint32_t)p[k] << (8 * k);
  } else {
    for (int k = 0; k < len; ++k) v = v * SEG_B + p[k];
  }
  return v;
}

// SEG_B^(len-1) mod 2^32 (len >= 1), by repeated squaring.
__host__ __device__ __forceinline__ uint32_t seg_pow(int len) {
  uint32_t r = 1, b = SEG_B;
  for (unsigned e = (unsigned)(len - 1); e; e >>= 1) {
    if (e & 1u) r *= b;
    b *= b;
  }
  return r;
}

// The value of the window one position right: drop `out`, append `in`.
__host__ __device__ __forceinline__ uint32_t seg_roll(uint32_t v, uint8_t out, uint8_t in, int len, uint32_t pw) {
  if (len <= SEG_EXACT_MAX) return (len < 4 ? v & ((1u << (8 * len)) - 1u) : v) >> 8 | (uint32_t)in << (8 * (len - 1));
  return (v - (uint32_t)out * pw) * SEG_B + in;
}

// Prefix values of a string x: H[0] = 0, H[k + 1] = H[k] * SEG_B + x[k]
// (mod 2^32), so that H[k] = sum_{j<k} x[j] * SEG_B^(k-1-j).  The hashed
// value of x[p .. p+n) is then H[p + n] - H[p] * SEG_B^n, with SEG_B^n =
// seg_pow(n) * SEG_B: any window's value in O(1) (n > SEG_EXACT_MAX).
__host__ __device__ __forceinline__ uint32_t seg_value_from_prefix(const uint32_t* H, int p, int n, uint32_t pw) {
  return H[p + n] - H[p] * (pw * SEG_B);
}

__host__ __device__ __forceinline__ unsigned long long seg_key_of(uint32_t v, int l, int i) {
  return ((unsigned long long)v << 32) | ((uint32_t)l << 8) | (uint32_t)i;
}

// 64-bit key of segment number i of a length-l string with the given bytes.
__host__ __device__ __forceinline__ unsigned long long seg_key(const uint8_t* p, int len, int l, int i) {
  return seg_key_of(seg_value(p, len), l, i);
}

// Table slot hash of a key: its two halves combined and passed through the
// 32-bit finaliser of MurmurHash3.  Tables have at most 2^32 slots.
__host__ __device__ __forceinline__ uint32_t key_mix(unsigned long long key) {
  uint32_t h = (uint32_t)(key >> 32) ^ ((uint32_t)key * 0x9E3779B1u);
  h ^= h >> 16;
  h *= 0x85ebca6bu;
  h ^= h >> 13;
  h *= 0xc2b2ae35u;
  h ^= h >> 16;
  return h;
}

// One-byte fingerprint of a key, kept beside each table slot (0 = empty):
// the top byte of the mix, folded with a multiplicative hash of V so that
// it stays informative when the slot index also uses the top bits.
__host__ __device__ __forceinline__ uint8_t key_fp(unsigned long long key, uint32_t mix) {
  const uint8_t f = (uint8_t)((mix ^ ((uint32_t)(key >> 32) * 0x2545F491u)) >> 24);
  return f ? f : (uint8_t)1;
}

// Character-count bound.  A string's signature is a thermometer code of its
// character counts: characters fall into SIG_BUCKETS = 24 buckets (c mod
// 24), and bucket b owns bits 4b .. 4b+3 (word b / 8 of w), of which the
// lowest min(count_b, 4) are set.  For two strings, the popcount of
// sx & ~sy over the words is the sum over buckets of the surplus of x's
// (saturated) count over y's, and likewise the other way.  An insertion or
// a deletion changes one bucket's count by one, a substitution moves one
// count from a bucket to another, so an edit lowers each surplus sum by at
// most one and
//   ED(x, y) >= max(popcount(sx & ~sy), popcount(sy & ~sx)).
// (Bucketing and saturation only shrink the surpluses.)  Candidates whose
// bound exceeds tau are rejected before any DP.  This test is not part of
// Pass-Join; it only drops pairs that cannot be similar.
constexpr int SIG_BUCKETS = 24;

struct __align__(16) Sig {
  uint32_t w[4];  // 96 signature bits in w[0..2]; w[3] is 0
};

__host__ __device__ __forceinline__ Sig char_signature(const uint8_t* p, int n) {
  Sig t = {{0u, 0u, 0u, 0u}};
  for (int k = 0; k < n; ++k) {
    const int b = (int)(p[k] % SIG_BUCKETS);
    const int word = b >> 3, sh = 4 * (b & 7);
    const uint32_t field = (t.w[word] >> sh) & 15u;  // 0, 1, 3, 7 or 15
    if (field != 15u) t.w[word] |= (field + 1u) << sh;  // set the next bit
  }
  return t;
}

__host__ __device__ __forceinline__ int popcount32(uint32_t x) {
#ifdef __CUDA_ARCH__
  return __popc(x);
#else
  return __builtin_popcount(x);
#endif
}

__host__ __device__ __forceinline__ int signature_bound(const Sig& x, const Sig& y) {
  int a = 0, b = 0;
  for (int k = 0; k < 3; ++k) {
    a += popcount32(x.w[k] & ~y.w[k]);
    b += popcount32(y.w[k] & ~x.w[k]);
  }
  return a > b ? a : b;
}

// Longest linear-probe sequence a lookup follows.  At load factor <= 1/2 a
// run of this many occupied slots does not occur in a correct table, so a
// lookup that reaches it reports an inconsistent index instead of scanning.
constexpr int TABLE_MAX_PROBES = 4096;

// 0x80 in every byte of w that is zero, 0 elsewhere (exact: the per-byte sum
// below cannot carry into the next byte).
__host__ __device__ __forceinline__ unsigned long long zero_bytes(unsigned long long w) {
  const unsigned long long lo7 = 0x7F7F7F7F7F7F7F7Full;
  return ~(((w & lo7) + lo7) | w | lo7);
}

__host__ __device__ __forceinline__ unsigned long long load_fp8(const uint8_t* p) {  // p 8-byte aligned
#ifdef __CUDA_ARCH__
  return __ldg(reinterpret_cast<const unsigned long long*>(p));
#else
  unsigned long long w;
  memcpy(&w, p, 8);
  return w;
#endif
}

__host__ __device__ __forceinline__ int first_set64(unsigned long long x) {  // x != 0
#ifdef __CUDA_ARCH__
  return __ffsll((long long)x) - 1;
#else
  return __builtin_ctzll(x);
#endif
}

__host__ __device__ __forceinline__ bool slot_matches(const Slot* t, unsigned long long h, unsigned long long key,
                                                      uint32_t& begin, uint32_t& count, unsigned long long& k) {
#ifdef __CUDA_ARCH__
  const uint4 raw = __ldg(reinterpret_cast<const uint4*>(t + h));
  k = ((unsigned long long)raw.y << 32) | raw.x;
  if (k != key) return false;
  begin = raw.z;
  count = raw.w;
#else
  k = t[h].key;
  if (k != key) return false;
  begin = t[h].begin;
  count = t[h].count;
#endif
  return true;
}

// Layout of a table's fingerprint array for S = mask + 1 slots: bytes
// [0, S) hold key_fp of each used slot (0 for empty ones), the next pb * S
// bytes (pb = 1 or 2, chosen per table) a presence bitmap of W = pb * S / 4
// 32-bit words (8 pb bits per slot: 16 to 32 bits per key per byte at load
// factor 1/4 to 1/2) in which every stored key sets two bits of one word:
// word mix & (W - 1), bits mix >> 27 and (mix >> 22) & 31, mix =
// key_mix(key).  An absent key finds one of its two bits clear in about
// 98% or more of lookups, so in most steps of a warp's probe loop no lane
// goes on to the fingerprint walk.
// Bytes of a table's fingerprint array (fingerprints, then the bitmap of pb
// bytes per slot).
__host__ __device__ __forceinline__ unsigned long long fp_array_bytes(unsigned long long slots, unsigned pb) {
  return (1 + pb) * slots;
}

__host__ __device__ __forceinline__ void presence_of(uint32_t mix, unsigned long long mask, unsigned pb,
                                                     unsigned long long& word, uint32_t& bits) {
  word = mix & (((mask + 1) * pb / 4) - 1);
  bits = (1u << (mix >> 27)) | (1u << ((mix >> 22) & 31u));
}

__host__ __device__ __forceinline__ uint32_t load_u32(const uint8_t* p) {  // p 4-byte aligned
#ifdef __CUDA_ARCH__
  return __ldg(reinterpret_cast<const uint32_t*>(p));
#else
  uint32_t w;
  memcpy(&w, p, 4);
  return w;
#endif
}

// 1: found (begin, count); 0: not present; -1: probe limit reached.  The
// probe sequence is linear from slot key_mix(key) & mask.  With fingerprints
// (fp not NULL; layout above) a lookup first tests the key's presence bits
// -- one 4-byte load, and most absent keys stop there -- then walks the
// fingerprint bytes (a small array that stays in L2) eight slots at a
// time: one aligned 8-byte load gives the slots of a bucket, byte-parallel
// compares give those that are empty and those whose fingerprint matches,
// and a 16-byte slot is read only for a match before the first empty slot.
__host__ __device__ __forceinline__ int table_find(const Slot* __restrict__ t, const uint8_t* __restrict__ fp,
                                                   unsigned pb, unsigned long long mask, unsigned long long key,
                                                   uint32_t& begin, uint32_t& count) {
  const uint32_t mix = key_mix(key);
  unsigned long long h = mix & mask;
  unsigned long long k = 0;
  if (!fp) {
    for (int probe = 0; probe < TABLE_MAX_PROBES; ++probe) {
      if (slot_matches(t, h, key, begin, count, k)) return 1;
      if (k == 0) return 0;
      h = (h + 1) & mask;
    }
    return -1;
  }
  unsigned long long word;
  uint32_t bits;
  presence_of(mix, mask, pb, word, bits);
  if ((load_u32(fp + (mask + 1) + (word << 2)) & bits) != bits) return 0;
  // mask + 1 (the slot count) is a power of two >= 8, so buckets of 8 never wrap
  const unsigned long long f8 = 0x0101010101010101ull * key_fp(key, mix);
  unsigned long long b = h & ~7ull;
  unsigned long long live = ~0ull << (8 * (h & 7));  // the first bucket from slot h on
  for (int step = 0; step < TABLE_MAX_PROBES / 8; ++step) {
    const unsigned long long w = load_fp8(fp + b);
    const unsigned long long empty = zero_bytes(w) & live;
    unsigned long long match = zero_bytes(w ^ f8) & live;
    if (empty) match &= (empty & (~empty + 1ull)) - 1ull;  // slots before the first empty one
    while (match) {
      if (slot_matches(t, b + (first_set64(match) >> 3), key, begin, count, k)) return 1;
      match &= match - 1ull;
    }
    if (empty) return 0;
    b = (b + 8) & mask;
    live = ~0ull;
  }
  return -1;
}

// Side signatures, for the screen in front of extension verification.
// Extension verification (Sec. 5.2, Alg. 3) accepts a match of segment i
// only if ED(s_l, r_l) <= i - 1 and ED(s_r, r_r) <= tau + 1 - i, where s_l,
// r_l are the parts left of the matched substring and segment, and s_r, r_r
// the parts right of them.  The character-count bound above holds for each
// side on its own, with thresholds that add up to tau, so testing the two
// sides rejects far more matches than testing the whole strings.  A side
// signature is a 48-bit thermometer code: characters fall into SIDE_BUCKETS
// = 12 buckets (c mod 12), bucket b owns bits 4b .. 4b+3, of which the lowest
// min(count_b, 4) are set; the bound of two sides is the larger of the two
// popcounts of x & ~y and y & ~x.
constexpr int SIDE_BUCKETS = 12;

__host__ __device__ __forceinline__ unsigned long long side_signature(const uint8_t* p, int n) {
  unsigned long long t = 0;
  for (int k = 0; k < n; ++k) {
    const int sh = 4 * (int)(p[k] % SIDE_BUCKETS);
    const unsigned long long field = (t >> sh) & 15ull;  // 0, 1, 3, 7 or 15
    if (field != 15ull) t |= (field + 1ull) << sh;       // set the next bit
  }
  return t;
}

__host__ __device__ __forceinline__ int popcount64(unsigned long long x) {
#ifdef __CUDA_ARCH__
  return __popcll(x);
#else
  return __builtin_popcountll(x);
#endif
}

__host__ __device__ __forceinline__ int side_bound(unsigned long long x, unsigned long long y) {
  const int a = popcount64(x & ~y), b = popcount64(y & ~x);
  return a > b ? a : b;
}

// What the screen in front of extension verification needs about one
// posting, stored beside the postings in the same order so that the
// candidates of a run are read as one coalesced 16-byte stream: the sid and
// the side signatures of the indexed string around the posting's segment
// (48 bits left of it in w[0] and the low half of w[1], 48 bits right of it
// in the high half of w[1] and w[2]).
struct __align__(16) PostRec {
  uint32_t sid;
  uint32_t w[3];
};

__host__ __device__ __forceinline__ uint32_t rec_sid(const PostRec& r) { return r.sid; }
__host__ __device__ __forceinline__ unsigned long long rec_left(const PostRec& r) {
  return (unsigned long long)r.w[0] | ((unsigned long long)(r.w[1] & 0xFFFFu) << 32);
}
__host__ __device__ __forceinline__ unsigned long long rec_right(const PostRec& r) {
  return (unsigned long long)(r.w[1] >> 16) | ((unsigned long long)r.w[2] << 16);
}
__host__ __device__ __forceinline__ PostRec make_rec(uint32_t sid, unsigned long long left, unsigned long long right) {
  PostRec r;
  r.sid = sid;
  r.w[0] = (uint32_t)left;
  r.w[1] = (uint32_t)((left >> 32) & 0xFFFFu) | (uint32_t)((right & 0xFFFFu) << 16);
  r.w[2] = (uint32_t)(right >> 16);
  return r;
}

// One threshold's segment index.
struct Partition {
  int tau = -1;
  uint32_t first = 0;        // first sid with length >= tau + 1
  uint64_t n_records = 0;    // (n - first) * (tau + 1)
  uint64_t n_unique = 0;     // distinct keys
  DBuf<Slot> table;          // power-of-two capacity
  DBuf<uint8_t> fp;          // key_fp of each used slot (0 for empty ones), then the presence bitmap
  unsigned presence_bytes = 1;  // bitmap bytes per slot (2 for indexes of long strings)
  int scheme = PJ_PARTITION_EVEN;  // partition scheme (pj_options.partition)
  DBuf<uint32_t> postings;   // sids, runs in key order, ascending inside a run
  DBuf<PostRec> precs;       // one record per posting, same order
  bool sides = false;        // the records carry side signatures (else 0): indexes of strings that
                             // are verified by extension verification by default
  // group visiting order for one probe: the (length, segment) groups sorted
  // by window size, widest first; [0] for R != S probes, [1] for the self join
  DBuf<uint16_t> gorder[2];
};

}  // namespace pj

// Opaque index handle of the C ABI.
struct pj_index {
  pj::Ctx ctx;
  int device = 0;
  std::mutex mu;             // serialises calls that use the index
  bool results_on_device = false;
  bool lazy = false;         // thresholds are built on first use
  bool autotune = false;     // tune the verification of each threshold's self join
  int scheme = PJ_PARTITION_EVEN;  // partition scheme of every threshold's segment index
  std::string autotune_cache;  // file of tuning decisions (empty: PJ_AUTOTUNE_CACHE)
  int verify_mode = PJ_VERIFY_AUTO;
  bool graph_joins = false;  // self joins replay a recorded graph (see pj_options.graph_joins)
  // recorded self joins by threshold (type-erased: the plan type lives with
  // the join code); released before the partitions they read
  std::vector<std::shared_ptr<void>> self_plans;
  float build_ms = 0.f;
  uint32_t n = 0;
  int lmax = 0;              // longest string
  uint64_t total_bytes = 0;
  pj::DBuf<uint8_t> sbytes;  // strings in sid order
  pj::DBuf<uint64_t> soff;   // n + 1 offsets
  pj::DBuf<uint32_t> slen;   // lengths by sid
  pj::DBuf<uint32_t> perm;   // sid -> input id
  pj::DBuf<uint32_t> bbeg;   // lmax + 2 bucket starts by length
  pj::DBuf<pj::Sig> sbm;     // character signatures by sid (char_signature)
  pj::DBuf<uint32_t> sph;    // prefix values (seg_value_from_prefix) by sid, |s| + 1 from soff[sid] + sid
  pj::DBuf<unsigned long long> sref;  // soff[sid] << 16 | slen[sid] by sid
  std::vector<uint32_t> h_bbeg;
  std::vector<pj::Partition> parts;  // index = tau
  uint64_t device_bytes() const;
};

namespace pj {

// Builds the sorted store of S into idx (host or device input).
void build_store(pj_index& idx, const pj_strings& S);
// Builds the segment index of idx for one threshold.
void build_partition(pj_index& idx, int tau, Partition& part);
// Returns idx.parts[tau], building it first if the index is lazy and it is
// not built yet (*ms receives the device time spent, else 0).
Partition& ensure_partition(pj_index& idx, int tau, float* ms);

// Device copy of a probe set (R or a query batch) in input order.
struct ProbeSet {
  DBuf<uint8_t> own_bytes;   // device copy when the input was on the host
  DBuf<uint64_t> own_off;
  const uint8_t* bytes = nullptr;  // string k = bytes[off[k] .. off[k+1])
  const uint64_t* off = nullptr;
  DBuf<uint32_t> len;
  DBuf<Sig> bm;  // character signatures
  uint32_t n = 0;
  int lmax = 0;
};
void upload_probe_set(const Ctx& c, const pj_strings& R, ProbeSet& out);

// R != S probe of a resident index where probe q has threshold h_tau[q]
// (host array).  Every threshold present must be built.  Work is ordered on
// c's stream and uses c's allocator; the index is only read.
void query_multi_impl(const Ctx& c, pj_index& idx, const ProbeSet& R, const uint8_t* h_tau, pj_result* out,
                      bool on_device);

void set_last_error(const std::string& msg);

// Self join of idx over the probes with sids in [q_lo, q_hi): the pairs whose
// later string (sid order) lies in that range; `fallback` adds the pairs
// with a string too short to partition (all of them, whatever the range).
void self_join_range(pj_index& idx, int tau, uint32_t q_lo, uint32_t q_hi, bool fallback, pj_result* out,
                     bool on_device);
// Makes *out a host result over `pairs` (malloc'd; pj_result_free frees it).
void host_result(pj_result* out, pj_pair* pairs, uint64_t count);

}  // namespace pj
