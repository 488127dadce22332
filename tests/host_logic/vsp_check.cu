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
// Shared-prefix form (vsp_rows): a run of strings r that share prefixes,
// each verified against s with the band kept across them exactly as the
// mode-L kernel does (resume after the kept row when the common prefix
// reaches it, stop at the kept dead row when the prefix reaches that);
// every result must equal min(t + 1, ED) and the rows saved are counted.
template <int W> int run_shared(int tmax) {
  std::mt19937 g(11);
  int bad = 0;
  long saved = 0, resumed = 0, skipped = 0;
  for (int it = 0; it < 20000; ++it) {
    const int t = 1 + (int)(g() % tmax);
    std::string s;
    const int ls = 20 + (int)(g() % 30);
    for (int k = 0; k < ls; ++k) s += char('a' + g() % 3);
    // a run of 6 strings of one length, each derived from the previous by an
    // edit at a random position (so consecutive ones share a prefix)
    std::vector<std::string> rs;
    std::string r = edited(g, s, (int)(g() % (t + 2)));
    const int L = (int)r.size();
    for (int k = 0; k < 6; ++k) {
      rs.push_back(r);
      r[g() % L] = char('a' + g() % 3);
    }
    int V[W], snap[W];
    int krow = 0, kdead = 0, klen = -1;
    std::string kr;
    for (size_t k = 0; k < rs.size(); ++k) {
      const std::string& y = rs[k];
      if (std::abs((int)y.size() - (int)s.size()) > t || y.empty()) continue;
      int keep = 0;
      if (k + 1 < rs.size() && rs[k + 1].size() == y.size())
        keep = pj::common_prefix((const uint8_t*)y.data(), (const uint8_t*)rs[k + 1].data(), (int)y.size());
      int start = 0, d = t + 1, dead = 0;
      bool skip = false;
      if ((int)y.size() == klen) {
        const int c = pj::common_prefix((const uint8_t*)y.data(), (const uint8_t*)kr.data(), (int)y.size());
        if (kdead && c >= kdead) {
          skip = true;
          ++skipped;
        } else if (krow && c >= krow) {
          start = krow;
          for (int j = 0; j < W; ++j) V[j] = snap[j];
          saved += start;
          ++resumed;
        }
      }
      unsigned long long cells = 0;
      if (!skip) {
        d = pj::vsp_rows<W>((const uint8_t*)y.data(), (int)y.size(), (const uint8_t*)s.data(), (int)s.size(), t,
                            start, V, keep, snap, dead, cells);
        klen = (int)y.size();
        kr = y;
        krow = keep > start ? (!dead || dead >= keep ? keep : 0) : (keep == start ? start : 0);
        kdead = dead;
      }
      const int want = std::min(t + 1, ed(y, s));
      if (d != want) {
        if (bad < 5) printf("shared W=%d t=%d k=%zu got %d want %d\n", W, t, k, d, want);
        ++bad;
      }
    }
  }
  printf("shared W=%d bad=%d resumed=%ld skipped=%ld rows_saved=%ld\n", W, bad, resumed, skipped, saved);
  return bad;
}

int main() {
  run_shared<5>(4);
  run_shared<9>(8);
  run_shared<17>(16);
  run<2>(1);
  run<3>(2);
  run<5>(4);
  run<9>(8);
  run<17>(16);
  run<33>(32);
  return 0;
}
