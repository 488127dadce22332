// Host-side check of the even partition used by the kernels
// (even_segment_m, pj_internal.cuh: floor(l / parts) by one multiply with a
// precomputed reciprocal) against the plain integer division of the
// partition rule of Sec. 3.1, for every string length 0..65535 and every
// segment count 1..33, every segment i.  Also checks that the segments tile
// the string.  Prints "bad=<mismatches>".
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
  printf("bad=%ld\n", bad);
  return 0;
}
