// Host-side check of the character-count bounds used before verification
// (signature_bound of char_signature, and side_bound of side_signature for
// the parts around a match, pj_internal.cuh): they never exceed the
// edit distance of Def. 1 (plain Wagner-Fischer DP), on random strings over
// small alphabets, over all 256 byte values (buckets shared by c and
// c + 24k) and with runs of repeated characters (saturated counts), and it
// is exact on pairs that differ only by characters absent from the other
// string.  Prints "bad=<violations> tight=<exact cases>".
#include <cstdio>
#include <random>
#include <string>
#include <vector>

#include "pj_internal.cuh"

static int ed(const std::string& a, const std::string& b) {
  std::vector<int> p(b.size() + 1), c(b.size() + 1);
  for (size_t j = 0; j <= b.size(); ++j) p[j] = (int)j;
  for (size_t i = 1; i <= a.size(); ++i) {
    c[0] = (int)i;
    for (size_t j = 1; j <= b.size(); ++j)
      c[j] = std::min(std::min(p[j] + 1, c[j - 1] + 1), p[j - 1] + (a[i - 1] != b[j - 1] ? 1 : 0));
    std::swap(p, c);
  }
  return p[b.size()];
}

int main() {
  std::mt19937 g(7);
  long bad = 0, tight = 0, side_tight = 0;
  const int alpha[] = {2, 5, 27, 64, 200, 256};
  for (int A : alpha)
    for (int it = 0; it < 40000; ++it) {
      const int la = g() % 16, lb = g() % 16;
      std::string a, b;
      for (int k = 0; k < la; ++k) a += (char)(g() % A);
      for (int k = 0; k < lb; ++k) b += (char)(g() % A);
      if (it % 5 == 0) b = a.substr(0, la / 2) + std::string(g() % 9, (char)(g() % A)) + a.substr(la / 2);  // runs
      const int bound = pj::signature_bound(pj::char_signature((const uint8_t*)a.data(), la),
                                            pj::char_signature((const uint8_t*)b.data(), (int)b.size()));
      const int d = ed(a, b);  // b may have been rebuilt above
      if (bound > d) {
        if (bad < 5) printf("A=%d bound %d > ed %d\n", A, bound, d);
        ++bad;
      }
      // the side signatures of the extension screen (12 buckets, counts capped at 4)
      const int sbound = pj::side_bound(pj::side_signature((const uint8_t*)a.data(), la),
                                        pj::side_signature((const uint8_t*)b.data(), (int)b.size()));
      if (sbound > d) {
        if (bad < 5) printf("A=%d side bound %d > ed %d\n", A, sbound, d);
        ++bad;
      }
      side_tight += sbound == d && d > 0;
      tight += bound == d && d > 0;
    }
  // substituting k characters by characters the string lacks: bound = ED = k
  for (int k = 1; k <= 6; ++k) {
    std::string a = "abcdefghij", b = a;
    for (int m = 0; m < k; ++m) b[m] = (char)('k' + m);  // buckets (c mod 24) absent from a
    const int bound = pj::signature_bound(pj::char_signature((const uint8_t*)a.data(), 10),
                                          pj::char_signature((const uint8_t*)b.data(), 10));
    if (bound != k || ed(a, b) != k) ++bad;
  }
  printf("side_tight=%ld\n", side_tight);
  printf("bad=%ld tight=%ld\n", bad, tight);
  return 0;
}
