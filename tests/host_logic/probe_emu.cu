// Host-side run of the probe/verify kernels' per-thread logic (pj_probe.cuh,
// pj_verify.cuh) on one string set, for CPU tests.  The device index layout
// is rebuilt here with plain loops: strings in (length, id) order, segment
// records sorted stably by key, runs in an open-addressing table.  The two
// phases are then run exactly as the kernels split them: every group's
// window lookups produce hits, and every posting of every hit is verified.
//
// usage: probe_emu <bytes file> <offsets file> <tau> [<query bytes> <query offsets>]
// prints: "stats lookups candidates accepted hits" then one "a b ed" line per
// pair, sorted.
#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <fstream>
#include <iterator>
#include <map>
#include <numeric>
#include <vector>

#include "pj_probe.cuh"

using namespace pj;
typedef unsigned long long ull;

static std::vector<char> slurp(const char* path) {
  std::ifstream f(path, std::ios::binary);
  return std::vector<char>((std::istreambuf_iterator<char>(f)), std::istreambuf_iterator<char>());
}

int main(int argc, char** argv) {
  if (argc != 4 && argc != 6) return 2;
  const int tau = atoi(argv[3]);
  std::vector<char> bb = slurp(argv[1]), ob = slurp(argv[2]);
  std::vector<uint64_t> off(ob.size() / 8);
  memcpy(off.data(), ob.data(), ob.size());
  const uint32_t n = (uint32_t)off.size() - 1;
  // store in sid order
  std::vector<uint32_t> perm(n);
  std::iota(perm.begin(), perm.end(), 0u);
  std::stable_sort(perm.begin(), perm.end(),
                   [&](uint32_t x, uint32_t y) { return off[x + 1] - off[x] < off[y + 1] - off[y]; });
  std::vector<uint32_t> slen(n);
  std::vector<uint64_t> soff(n + 1, 0);
  for (uint32_t s = 0; s < n; ++s) {
    slen[s] = (uint32_t)(off[perm[s] + 1] - off[perm[s]]);
    soff[s + 1] = soff[s] + slen[s];
  }
  std::vector<uint8_t> sb(std::max<uint64_t>(soff[n], 1));
  for (uint32_t s = 0; s < n; ++s) memcpy(&sb[soff[s]], &bb[off[perm[s]]], slen[s]);
  const int lmax = n ? (int)*std::max_element(slen.begin(), slen.end()) : 0;
  std::vector<uint32_t> bbeg(lmax + 2);
  for (int l = 0; l <= lmax + 1; ++l)
    bbeg[l] = (uint32_t)(std::lower_bound(slen.begin(), slen.end(), (uint32_t)l) - slen.begin());
  const uint32_t first = bbeg[std::min(tau + 1, lmax + 1)];
  // segment records -> runs -> table
  std::vector<std::pair<ull, uint32_t>> rec;
  for (uint32_t s = first; s < n; ++s)
    for (int i = 1; i <= tau + 1; ++i) {
      int P, li;
      even_segment((int)slen[s], tau, i, P, li);
      rec.push_back({seg_key(&sb[soff[s] + P], li, (int)slen[s], i), s});
    }
  std::stable_sort(rec.begin(), rec.end(), [](const auto& x, const auto& y) { return x.first < y.first; });
  std::vector<uint32_t> post(std::max<size_t>(rec.size(), 1));
  for (size_t k = 0; k < rec.size(); ++k) post[k] = rec[k].second;
  size_t U = 0;
  for (size_t k = 0; k < rec.size(); ++k) U += (k == 0 || rec[k].first != rec[k - 1].first);
  ull cap = 1024;
  while (cap < 2 * U) cap <<= 1;
  std::vector<Slot> table(cap);
  memset(table.data(), 0, cap * sizeof(Slot));
  for (size_t k = 0; k < rec.size();) {
    size_t e = k;
    while (e < rec.size() && rec[e].first == rec[k].first) ++e;
    ull h = key_mix(rec[k].first) & (cap - 1);
    while (table[h].key) h = (h + 1) & (cap - 1);
    table[h].key = rec[k].first;
    table[h].begin = (uint32_t)k;
    table[h].count = (uint32_t)(e - k);
    k = e;
  }
  // fingerprint bytes and presence bitmap as the index build sets them
  // (none with PJ_EMU_NO_FP)
  const unsigned pb = soff[n] > 256 * (ull)n ? 2 : 1;  // as the index build chooses
  std::vector<uint8_t> fp(fp_array_bytes(cap, pb), 0);
  for (ull h = 0; h < cap; ++h)
    if (table[h].key) {
      const uint32_t mix = key_mix(table[h].key);
      fp[h] = key_fp(table[h].key, mix);
      ull word;
      uint32_t bits;
      presence_of(mix, cap - 1, pb, word, bits);
      for (int k = 0; k < 4; ++k) fp[cap + 4 * word + k] |= (uint8_t)(bits >> (8 * k));
    }
  const bool use_fp = !getenv("PJ_EMU_NO_FP");
  std::vector<ull> ref(n);  // packed offset << 16 | length, as the store keeps it
  for (uint32_t k = 0; k < n; ++k) ref[k] = ((ull)soff[k] << 16) | slen[k];
  ProbeView v{};
  v.table_fp = use_fp ? fp.data() : nullptr;
  v.table_pb = pb;
  v.iref = use_fp ? ref.data() : nullptr;  // the no-fingerprint run also covers the unpacked reads
  v.ibytes = sb.data();
  v.ioff = soff.data();
  v.ilen = slen.data();
  v.ibbeg = bbeg.data();
  v.ilmax = lmax;
  v.iperm = perm.data();
  v.n_index = n;
  v.table = table.data();
  v.mask = cap - 1;
  v.postings = post.data();
  v.n_postings = rec.size();
  v.tau = tau;
  v.key_shift = 32;
  const bool self = argc == 4;
  std::vector<char> qb, qo;
  std::vector<uint64_t> qoff;
  std::vector<uint32_t> qlen;
  if (self) {
    v.pbytes = sb.data();
    v.poff = soff.data();
    v.plen = slen.data();
    v.pbegin = first;
    v.pcount = n - first;
    v.pid = perm.data();
  } else {
    qb = slurp(argv[4]);
    qo = slurp(argv[5]);
    qoff.resize(qo.size() / 8);
    memcpy(qoff.data(), qo.data(), qo.size());
    qlen.resize(qoff.size() - 1);
    for (size_t k = 0; k + 1 < qoff.size(); ++k) qlen[k] = (uint32_t)(qoff[k + 1] - qoff[k]);
    if (qb.empty()) qb.push_back(0);
    v.pbytes = reinterpret_cast<const uint8_t*>(qb.data());
    v.poff = qoff.data();
    v.plen = qlen.data();
    v.pbegin = 0;
    v.pcount = (uint32_t)qlen.size();
    v.pid = nullptr;
  }
  // phase 1: groups -> hits, as the kernels split it: pass 1 rolls the
  // window's substring hashes and records the positions that found a
  // posting run; pass 2 looks those positions up again and emits the hits.
  const int G = groups_per_probe(tau, self);
  std::vector<Hit> hits;
  ull lookups = 0;
  int err = 0;
  for (ull t = 0; t < (ull)v.pcount * G; ++t) {
    const uint32_t q = v.pbegin + (uint32_t)(t / G);
    const int ls = (int)v.plen[q];
    const uint8_t* s = v.pbytes + v.poff[q];
    int l, i, P, li, lo, hi;
    if (!group_window(v, self, q, ls, (int)(t % G), l, i, P, li, lo, hi)) continue;
    ull mask = 0;
    uint32_t V = seg_value(s + lo, li);
    const uint32_t pw = seg_pow(li);
    for (int p = lo;; ++p) {
      ++lookups;
      uint32_t b;
      if (lookup_key(v, self, q, ls, l, seg_key_of(V, l, i), b, err)) mask |= 1ull << (p - lo);
      if (p == hi) break;
      V = seg_roll(V, s[p], s[p + li], li, pw);
    }
    for (int p = lo; p <= hi; ++p) {
      if (!(mask >> (p - lo) & 1)) continue;
      uint32_t b;
      const uint32_t c = lookup(v, self, s, ls, q, l, i, p, li, b, err);
      if (c) hits.push_back(Hit{q, b, c, (uint32_t)p | ((uint32_t)i << 16)});
    }
  }
  // phase 2: candidates
  std::map<ull, int> best;
  ull cand = 0, acc = 0, cells = 0;
  for (const Hit& h : hits)
    for (uint32_t k = 0; k < h.count; ++k) {
      ++cand;
      ull key;
      int ed;
      if (verify_candidate<33>(v, self, h, k, key, ed, cells, err)) {
        ++acc;
        auto it = best.find(key);
        if (it == best.end() || it->second > ed) best[key] = ed;
      }
    }
  // short strings: direct verification (as the fallback kernel)
  if (self) {
    for (uint32_t x = 0; x < first; ++x)
      for (uint32_t y = x + 1; y < bbeg[std::min((int)slen[x] + tau, lmax) + 1]; ++y) {
        const int d = vsp<33>(&sb[soff[x]], (int)slen[x], &sb[soff[y]], (int)slen[y], tau, cells);
        if (d <= tau) best[((ull)std::min(perm[x], perm[y]) << 32) | std::max(perm[x], perm[y])] = d;
      }
  } else if (first > 0) {
    for (uint32_t x = 0; x < v.pcount; ++x) {
      const int lx = (int)v.plen[x];
      const int llo = std::max(0, lx - tau), lhi = std::min(std::min(tau, lx + tau), lmax);
      if (llo > lhi) continue;
      for (uint32_t y = bbeg[llo]; y < bbeg[lhi + 1]; ++y) {
        const int d = vsp<33>(v.pbytes + v.poff[x], lx, &sb[soff[y]], (int)slen[y], tau, cells);
        if (d <= tau) best[((ull)x << 32) | perm[y]] = d;
      }
    }
  }
  printf("stats %llu %llu %llu %zu %d\n", lookups, cand, acc, hits.size(), err);
  for (const auto& kv : best) printf("%llu %llu %d\n", kv.first >> 32, kv.first & 0xffffffffull, kv.second);
  return 0;
}
