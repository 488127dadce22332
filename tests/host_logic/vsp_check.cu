// Host-side check of the verification kernel's VERIFYSTRINGPAIR (vsp<W>,
// pj_verify.cuh): min(t + 1, ED) against a plain Wagner-Fischer DP, for every
// register width the kernels use (2, 3, 5, 9, 17, 33).  Two kinds of inputs:
// short random strings over {a, b, c} (every band shape, clipped bands), and
// long pairs (40..160 characters) where the second string is the first
// after up to t + 3 random edits, so that the band of the wide instances is
// filled and the edit distance sits around the threshold.
// Prints "W=<w> bad=<mismatches> near=<pairs with |ED - t| <= 1>" per width.
#include <cstdio>
#include <cstring>
#include <random>
#include <string>
#include <vector>
#include "pj_verify.cuh"
static int ed(const std::string& a, const std::string& b) {
  std::vector<int> p(b.size() + 1), c(b.size() + 1);
  for (size_t j = 0; j <= b.size(); ++j) p[j] = (int)j;
  for (size_t i = 1; i <= a.size(); ++i) {
    c[0] = (int)i;
    for (size_t j = 1; j <= b.size(); ++j) c[j] = std::min({p[j] + 1, c[j - 1] + 1, p[j - 1] + (a[i - 1] != b[j - 1])});
    std::swap(p, c);
  }
  return p[b.size()];
}
static std::string edited(std::mt19937& g, std::string s, int k) {
  for (int e = 0; e < k; ++e) {
    const int op = (int)(g() % 3);
    if (op == 0 || s.empty()) s.insert(s.begin() + (long)(g() % (s.size() + 1)), char('a' + g() % 3));
    else if (op == 1) s.erase(s.begin() + (long)(g() % s.size()));
    else s[g() % s.size()] = char('a' + g() % 3);
  }
  return s;
}
template <int W> int run(int tmax) {
  std::mt19937 g(1);
  int bad = 0, near = 0;
  for (int it = 0; it < 200000; ++it) {
    std::string a, b;
    int t = (int)(g() % (tmax + 1));
    if (it % 4 == 3) {  // long pair around the threshold
      const int la = 40 + (int)(g() % 121);
      for (int k = 0; k < la; ++k) a += char('a' + g() % 3);
      b = edited(g, a, (int)(g() % (t + 4)));
    } else {
      const int la = (int)(g() % 12), lb = (int)(g() % 12);
      for (int k = 0; k < la; ++k) a += char('a' + g() % 3);
      for (int k = 0; k < lb; ++k) b += char('a' + g() % 3);
    }
    unsigned long long cells = 0;
    const int v = pj::vsp<W>((const uint8_t*)a.data(), (int)a.size(), (const uint8_t*)b.data(), (int)b.size(), t, cells);
    const int full = ed(a, b);
    const int want = std::min(t + 1, full);
    if (full >= t - 1 && full <= t + 1) ++near;
    if (v != want) {
      if (bad < 5) printf("W=%d t=%d a=%s b=%s got %d want %d\n", W, t, a.c_str(), b.c_str(), v, want);
      bad++;
    }
  }
  printf("W=%d bad=%d near=%d\n", W, bad, near);
  return bad;
}
int main() {
  run<2>(1);
  run<3>(2);
  run<5>(4);
  run<9>(8);
  run<17>(16);
  run<33>(32);
  return 0;
}
