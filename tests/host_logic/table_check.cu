// The segment table's lookup (table_find) with fingerprints -- presence
// bitmap, eight fingerprint bytes per load, byte-parallel compares -- against plain
// linear probing over the slots, on tables filled to load factor 1/2 with
// clustered home slots, runs that wrap past the last slot, and absent keys
// whose fingerprints collide with present ones.  Host build of the same
// __host__ __device__ code the kernels run.
//
// prints "cases N bad M"
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <random>
#include <vector>

#include "pj_internal.cuh"

using namespace pj;
typedef unsigned long long ull;

static int plain_find(const std::vector<Slot>& t, ull mask, ull key, uint32_t& begin, uint32_t& count) {
  ull h = key_mix(key) & mask;
  for (size_t probe = 0; probe <= mask; ++probe) {
    if (t[h].key == key) {
      begin = t[h].begin;
      count = t[h].count;
      return 1;
    }
    if (t[h].key == 0) return 0;
    h = (h + 1) & mask;
  }
  return 0;
}

int main() {
  std::mt19937_64 rng(7);
  ull cases = 0, bad = 0;
  for (int trial = 0; trial < 60; ++trial) {
    const ull cap = 1024ull << (trial % 4);
    const ull mask = cap - 1;
    const ull n = cap / 2 - (trial % 3) * 7;  // up to load factor 1/2
    std::vector<Slot> t(cap);
    memset(t.data(), 0, cap * sizeof(Slot));
    std::vector<ull> keys;
    // clustered: keys drawn until their home slot falls in a few narrow
    // ranges (one of them the table's end, so runs wrap to slot 0)
    const bool clustered = trial % 2 == 1;
    while (keys.size() < n) {
      const ull key = rng() | 1ull;
      const ull home = key_mix(key) & mask;
      if (clustered && !(home >= cap - 40 || home < 24 || (home >= cap / 2 && home < cap / 2 + 64) ||
                         rng() % 8 == 0))
        continue;
      ull h = home;
      bool dup = false;
      while (t[h].key) {
        if (t[h].key == key) dup = true;
        h = (h + 1) & mask;
      }
      if (dup) continue;
      t[h].key = key;
      t[h].begin = (uint32_t)keys.size();
      t[h].count = (uint32_t)(key >> 40) + 1;
      keys.push_back(key);
    }
    const unsigned pb = 1 + (trial / 4) % 2;  // 1 or 2 bitmap bytes per slot, every size and fill
    std::vector<uint8_t> fp(fp_array_bytes(cap, pb), 0);  // fingerprints, then the presence bitmap
    for (ull h = 0; h < cap; ++h)
      if (t[h].key) {
        const uint32_t mix = key_mix(t[h].key);
        fp[h] = key_fp(t[h].key, mix);
        ull word;
        uint32_t bits;
        presence_of(mix, mask, pb, word, bits);
        for (int k = 0; k < 4; ++k) fp[cap + 4 * word + k] |= (uint8_t)(bits >> (8 * k));
      }
    auto check = [&](ull key) {
      uint32_t b0 = 0, c0 = 0, b1 = 0, c1 = 0, b2 = 0, c2 = 0;
      const int want = plain_find(t, mask, key, b0, c0);
      const int got = table_find(t.data(), fp.data(), pb, mask, key, b1, c1);
      const int got_nofp = table_find(t.data(), nullptr, pb, mask, key, b2, c2);
      ++cases;
      if (got != want || got_nofp != want || (want == 1 && (b1 != b0 || c1 != c0 || b2 != b0 || c2 != c0))) ++bad;
    };
    for (ull key : keys) check(key);  // present
    for (int k = 0; k < 4000; ++k) check(rng() | 1ull);  // absent (almost surely)
    // absent keys with the fingerprint of a present key at their home slot,
    // or whose presence bit is set
    for (int k = 0; k < 200000; ++k) {
      const ull key = rng() | 1ull;
      const uint32_t mix = key_mix(key);
      const ull h = mix & mask;
      ull word;
      uint32_t bits, have;
      presence_of(mix, mask, pb, word, bits);
      memcpy(&have, &fp[cap + 4 * word], 4);
      if ((t[h].key && fp[h] == key_fp(key, mix) && t[h].key != key) || (have & bits) == bits) check(key);
    }
  }
  printf("cases %llu bad %llu\n", cases, bad);
  return bad != 0;
}
