// Host-side check of the even partition used by the kernels
// (even_segment_m, pj_internal.cuh: floor(l / parts) by one multiply with a
// precomputed reciprocal) against the plain integer division of the
// partition rule of Sec. 3.1, for every string length 0..65535 and every
// segment count 1..33, every segment i.  Also checks that the segments tile
// the string.  Then checks the probe's rolling segment value (seg_roll)
// against the direct one (seg_value) over every window of random strings,
// for exact (short) and hashed segments, and the value taken from prefix
// values (seg_value_from_prefix) for hashed ones; that keys and fingerprints are
// never 0; and that exact keys of different short segments differ.  Prints
// "bad=<mismatches>".
#include <cstdio>

#include "pj_internal.cuh"

int main() {
  long bad = 0;
  for (int parts = 1; parts <= 33; ++parts) {
    const unsigned long long m = pj::seg_magic(parts);
    for (int l = 0; l < 65536; ++l) {
      int end = 0;
      for (int i = 1; i <= parts; ++i) {
        int P0, l0, P1, l1, P2, l2;
        pj::even_segment(l, parts - 1, i, P0, l0);
        pj::even_segment_m(l, parts, m, i, P1, l1);
        pj::even_segment_m(l, parts, 0, i, P2, l2);
        // the rule itself: the first parts - k segments have floor(l/parts)
        // characters, the last k one more, k = l mod parts
        const int base = l / parts, k = l % parts;
        const int want_len = base + (i > parts - k ? 1 : 0);
        if (P0 != P1 || l0 != l1 || P1 != P2 || l1 != l2 || l1 != want_len || P1 != end) {
          if (bad < 5) printf("parts=%d l=%d i=%d: %d/%d %d/%d want start %d len %d\n", parts, l, i, P0, l0, P1, l1,
                              end, want_len);
          ++bad;
        }
        end = P1 + l1;
      }
      if (end != l) ++bad;
    }
  }
  unsigned long long x = 88172645463325252ull;  // xorshift64
  for (int it = 0; it < 20000; ++it) {
    x ^= x << 13; x ^= x >> 7; x ^= x << 17;
    const int n = 1 + (int)(x % 300);
    const int len = it % 3 == 0 ? 1 + (int)((x >> 20) % 6) : 1 + (int)((x >> 20) % n);  // exact and hashed
    if (len > n) continue;
    uint8_t buf[300];
    for (int k = 0; k < n; ++k) {
      x ^= x << 13; x ^= x >> 7; x ^= x << 17;
      buf[k] = (uint8_t)(x >> 24);
    }
    uint32_t v = pj::seg_value(buf, len);
    const uint32_t pw = pj::seg_pow(len);
    uint32_t H[301];  // prefix values, as the store keeps them for the probe
    H[0] = 0;
    for (int k = 0; k < n; ++k) H[k + 1] = H[k] * pj::SEG_B + buf[k];
    for (int p = 0; p + len <= n; ++p) {
      if (v != pj::seg_value(buf + p, len)) ++bad;
      if (len > pj::SEG_EXACT_MAX && pj::seg_value_from_prefix(H, p, len, pw) != v) ++bad;
      const unsigned long long key = pj::seg_key_of(v, n, 1 + p % 33);
      if (key == 0 || pj::key_fp(key, pj::key_mix(key)) == 0) ++bad;
      if (p + len < n) v = pj::seg_roll(v, buf[p], buf[p + len], len, pw);
    }
  }
  // exact keys: different short segments never share a key
  for (int len = 1; len <= pj::SEG_EXACT_MAX; ++len)
    for (int it = 0; it < 20000; ++it) {
      uint8_t a[4], b[4];
      x ^= x << 13; x ^= x >> 7; x ^= x << 17;
      for (int k = 0; k < 4; ++k) {
        a[k] = (uint8_t)(x >> (8 * k));
        b[k] = (uint8_t)(x >> (8 * k + 32));
      }
      if (it & 1) b[it % len] = a[it % len];  // near misses too
      bool same = true;
      for (int k = 0; k < len; ++k) same &= a[k] == b[k];
      if ((pj::seg_key(a, len, 7, 2) == pj::seg_key(b, len, 7, 2)) != same) ++bad;
    }
  printf("bad=%ld\n", bad);
  return 0;
}
