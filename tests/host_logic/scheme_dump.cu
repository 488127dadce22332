// Prints the segments the kernels use for every length 1..160 and 1..33
// segments under each partition scheme (scheme_segment / segment_m in
// pj_internal.cuh), one line "scheme parts l P_1 l_1 P_2 l_2 ...", for the
// CPU test that compares them with the oracle's definitions.
#include <cstdio>

#include "pj_internal.cuh"

int main() {
  for (int scheme = 0; scheme <= 1; ++scheme)
    for (int parts = 1; parts <= 33; ++parts)
      for (int l = parts; l <= 160; ++l) {
        printf("%d %d %d", scheme, parts, l);
        for (int i = 1; i <= parts; ++i) {
          int P, li;
          pj::segment_m(l, parts, 0, scheme, i, P, li);
          printf(" %d %d", P, li);
        }
        printf("\n");
      }
  return 0;
}
