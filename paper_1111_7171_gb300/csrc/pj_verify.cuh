// Verification routines of the hot path (Sec. 5.1, Sec. 5.2, Alg. 3),
// usable from device code and, for checks on the CPU, from host code.
#pragma once

#include <stdint.h>
#include <stdlib.h>

#include <cuda_runtime.h>

#include <algorithm>
#include <cstdlib>

namespace pj {

#ifndef __CUDA_ARCH__
using std::abs;
using std::max;
using std::min;
#endif

// VERIFYSTRINGPAIR (Alg. 3): min(t + 1, ED(x, y)).  Rows run over the shorter
// string a, columns over the longer b, D = |b| - |a|.  Row i keeps only the
// cells j in [i - floor((t - D)/2), i + floor((t + D)/2)] (Sec. 5.1): at
// most t + 1 <= MAXW registers, indexed by diagonal d = j - i.  Values are
// saturated at t + 1 (exact for the capped result).  After each row the
// expected edit distance E(i, j) = M(i, j) + |D - (j - i)| is minimised over
// the band; if it exceeds t the pair is dissimilar (Lemma 4).
template <int MAXW>
__host__ __device__ __forceinline__ int vsp(const uint8_t* x, int nx, const uint8_t* y, int ny, int t,
                                            unsigned long long& cells) {
  // Single exit and structured loops only: callers reach warp and block
  // barriers right after this function, so every lane must leave it through
  // the same path.
  const uint8_t* a = nx <= ny ? x : y;
  const uint8_t* b = nx <= ny ? y : x;
  const int na = nx <= ny ? nx : ny;
  const int nb = nx <= ny ? ny : nx;
  const int D = nb - na;
  const int cap = t + 1;
  int res = cap;
  if (D <= t && na == 0) res = D;
  if (D <= t && na > 0) {
    const int dlo = -((t - D) >> 1);
    const int w = ((t + D) >> 1) - dlo + 1;  // <= t + 1 <= MAXW
    int V[MAXW];
    int eoff[MAXW];
#pragma unroll
    for (int k = 0; k < MAXW; ++k) {
      const int j = dlo + k;  // row 0: M(0, j) = j
      V[k] = (k < w && j >= 0 && j <= nb) ? min(j, cap) : cap;
      eoff[k] = abs(D - dlo - k);
    }
    bool alive = true;
    for (int i = 1; i <= na; ++i) {
      const uint8_t ca = a[i - 1];
      int left = cap;
      int emin = cap;
      const int j0 = i + dlo;
#pragma unroll
      for (int k = 0; k < MAXW; ++k) {
        const int j = j0 + k;
        const int up = (k + 1 < MAXW) ? V[k + 1] : cap;
        int val = cap;
        if (k < w && j >= 0 && j <= nb) {
          if (j == 0) {
            val = min(i, cap);
          } else {
            const int diag = V[k] + (ca != b[j - 1] ? 1 : 0);
            val = min(min(diag, up + 1), min(left + 1, cap));
          }
        }
        V[k] = val;
        left = val;
        emin = min(emin, val + eoff[k]);
      }
      cells += (unsigned long long)w;
      if (emin > t) {  // Lemma 4: every expected edit distance exceeds t
        alive = false;
        break;
      }
    }
    if (alive) {
      const int kres = D - dlo;
#pragma unroll
      for (int k = 0; k < MAXW; ++k)
        if (k == kres) res = V[k];
    }
  }
  return res;
}

// Extension-based verification of one match (Sec. 5.2, Alg. 3).  s has the
// selected substring at p; r is the indexed string whose segment i (start P,
// length li) it matched.  Returns true with ed = d_l + d_r when accepted.
template <int MAXW>
__host__ __device__ __forceinline__ bool verify_ext(const uint8_t* s, int ls, const uint8_t* r, int lr, int i, int p, int li,
                                                    int P, int tau, int& ed, unsigned long long& cells) {
  bool same = true;
  for (int k = 0; k < li; ++k) {
    if (s[p + k] != r[P + k]) {  // hash collision, not a match
      same = false;
      break;
    }
  }
  bool ok = false;
  if (same) {
    const int tl = i - 1, tr = tau + 1 - i;
    const int dl = vsp<MAXW>(s, p, r, P, tl, cells);
    if (dl <= tl) {
      const int dr = vsp<MAXW>(s + p + li, ls - p - li, r + P + li, lr - P - li, tr, cells);
      if (dr <= tr) {
        ed = dl + dr;
        ok = true;
      }
    }
  }
  return ok;
}

}  // namespace pj
