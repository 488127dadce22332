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

// VERIFYSTRINGPAIR (Alg. 3): min(t + 1, ED(x, y)).
//
// Rows run over the shorter string a, columns over the longer b, D = |b| -
// |a| <= t.  Row i holds the diagonals d = j - i from dlo = -floor((t-D)/2)
// upward: the length-aware band of Sec. 5.1 is d <= floor((t+D)/2), and the
// W registers (W >= t + 1) may cover a few more diagonals above it.  Any
// value computed over a superset of the band is the cost of a real
// alignment, and the band holds every alignment of cost <= t, so every value
// <= t comes out exact.  Cells left of column 0 start at t + 1 and stay at
// least t + 1 (every input to them is), which makes M(i, 0) = i fall out of
// the recurrence while i <= t, and a value >= t + 1 never lowers a cell
// below t + 1; so values are not clamped cell by cell, only the result is.
// Cells right of column |b| never feed a cell inside the matrix, so the
// characters of b are read at clamped indices and the inner loop has no
// bounds checks.
//
// After each row the expected edit distance E(i, j) = M(i, j) + |D - (j - i)|
// is minimised over the row; if every E exceeds t the pair is dissimilar
// (Lemma 4).  cells counts the length-aware band cells of the rows evaluated.
//
// Single exit and structured loops only: callers may reach synchronisation
// points right after this function.
template <int W>
__host__ __device__ __forceinline__ int vsp_band(const uint8_t* a, int na, const uint8_t* b, int nb, int t,
                                                 unsigned long long& cells) {
  const int D = nb - na;
  const int cap = t + 1;
  const int dlo = -((t - D) >> 1);
  const int w = ((t + D) >> 1) - dlo + 1;  // length-aware band width, <= t + 1 <= W
  const int blast = nb - 1;                // nb >= na >= 1
  int V[W];
  int eoff[W];
  uint8_t B[W];  // B[k] = b[i + dlo + k - 1] for the current row i (index clamped to [0, nb))
#pragma unroll
  for (int k = 0; k < W; ++k) {
    const int j = dlo + k;  // row 0: M(0, j) = j
    V[k] = j < 0 ? cap : j;
    eoff[k] = abs(D - dlo - k);
    B[k] = b[min(max(j, 0), blast)];  // b index for row 1
  }
  bool alive = true;
  int rows = 0;
  for (int i = 1; i <= na; ++i) {
    const uint8_t ca = a[i - 1];
    int left = cap;
    int emin = cap;
#pragma unroll
    for (int k = 0; k < W; ++k) {
      const int up = (k + 1 < W) ? V[k + 1] : cap;
      const int diag = V[k] + (ca != B[k] ? 1 : 0);
      const int val = min(diag, min(up, left) + 1);
      V[k] = val;
      left = val;
      emin = min(emin, val + eoff[k]);
    }
    ++rows;
    if (emin > t) {  // Lemma 4: every expected edit distance of the row exceeds t
      alive = false;
      break;
    }
    const int jn = i + dlo + W - 1;  // next row's last column character
#pragma unroll
    for (int k = 0; k + 1 < W; ++k) B[k] = B[k + 1];
    B[W - 1] = b[min(max(jn, 0), blast)];
  }
  cells += (unsigned long long)(rows * w);
  int res = cap;
  if (alive) {
    const int kres = D - dlo;
#pragma unroll
    for (int k = 0; k < W; ++k)
      if (k == kres) res = min(V[k], cap);
  }
  return res;
}

// VERIFYSTRINGPAIR for narrow bands, with the band width W and the diagonal
// of the result KRES = D - dlo fixed at compile time.  Row 0 holds
// M(0, j) = |j| (the real values for j >= 0, and for j < 0 a virtual
// extension of b that only ever yields values >= min(i + |j|, t + 2) in row
// i, so cells <= t stay exact).  Then neighbouring cells of a row differ by
// at most 1 -- left to right by the recurrence, right to left by induction
// over the rows -- so E(i, k) = V[k] + |KRES - k| is smallest at k = KRES
// and the Lemma 4 test over the row is the single test V[KRES] > t.
template <int W, int KRES>
__host__ __device__ __forceinline__ int vsp_band_k(const uint8_t* a, int na, const uint8_t* b, int nb, int t,
                                                   int dlo, int w, unsigned long long& cells) {
  constexpr int KR = KRES < W ? KRES : W - 1;  // instances with KRES >= W are never called
  const int cap = t + 1;
  const int blast = nb - 1;
  int V[W];
  uint8_t B[W];
#pragma unroll
  for (int k = 0; k < W; ++k) {
    const int j = dlo + k;
    V[k] = abs(j);
    B[k] = b[min(max(j, 0), blast)];
  }
  bool alive = true;
  int rows = 0;
  for (int i = 1; i <= na; ++i) {
    const uint8_t ca = a[i - 1];
    int left = cap;
#pragma unroll
    for (int k = 0; k < W; ++k) {
      const int up = (k + 1 < W) ? V[k + 1] : cap;
      const int diag = V[k] + (ca != B[k] ? 1 : 0);
      const int val = min(diag, min(up, left) + 1);
      V[k] = val;
      left = val;
    }
    ++rows;
    if (V[KR] > t) {  // Lemma 4 (see above)
      alive = false;
      break;
    }
    const int jn = i + dlo + W - 1;
#pragma unroll
    for (int k = 0; k + 1 < W; ++k) B[k] = B[k + 1];
    B[W - 1] = b[min(max(jn, 0), blast)];
  }
  cells += (unsigned long long)(rows * w);
  return alive ? min(V[KR], cap) : cap;
}

// vsp_band_k with the result diagonal kres chosen at run time: one code path
// for every band shape of width W, so that the lanes of a warp verifying
// different matches run it together instead of one compile-time instance
// after another.  Lemma 4 is the same single test, on V[kres] (selected by
// an unrolled compare; the registers are not indexed dynamically).
template <int W>
__host__ __device__ __forceinline__ int vsp_band_r(const uint8_t* a, int na, const uint8_t* b, int nb, int t,
                                                   int dlo, int w, int kres, unsigned long long& cells) {
  const int cap = t + 1;
  const int blast = nb - 1;
  int V[W];
  uint8_t B[W];
#pragma unroll
  for (int k = 0; k < W; ++k) {
    const int j = dlo + k;
    V[k] = abs(j);
    B[k] = b[min(max(j, 0), blast)];
  }
  bool alive = true;
  int rows = 0;
  int vres = cap;
  for (int i = 1; i <= na; ++i) {
    const uint8_t ca = a[i - 1];
    int left = cap;
#pragma unroll
    for (int k = 0; k < W; ++k) {
      const int up = (k + 1 < W) ? V[k + 1] : cap;
      const int diag = V[k] + (ca != B[k] ? 1 : 0);
      const int val = min(diag, min(up, left) + 1);
      V[k] = val;
      left = val;
    }
    ++rows;
    vres = cap;
#pragma unroll
    for (int k = 0; k < W; ++k)
      if (k == kres) vres = V[k];
    if (vres > t) {  // Lemma 4 (see vsp_band_k)
      alive = false;
      break;
    }
    const int jn = i + dlo + W - 1;
#pragma unroll
    for (int k = 0; k + 1 < W; ++k) B[k] = B[k + 1];
    B[W - 1] = b[min(max(jn, 0), blast)];
  }
  cells += (unsigned long long)(rows * w);
  return alive ? min(vres, cap) : cap;
}

// Everything of one VERIFYSTRINGPAIR call that depends only on the lengths
// and the threshold: in extension verification it is the same for every
// candidate of a posting run (same probe, position, segment and indexed
// length), so it is prepared once per run.
struct VspPlan {
  int t, na, nb;     // a = the shorter part
  int dlo, w, kres;  // band start, length-aware width, diagonal of the result
  int kind;          // 0: D > t, 1: a empty (result D), 2: t = 0 (exact compare), 3: band
  int W;             // band registers (3: 2, 3, 5, 9, 17 or 33)
  bool swap;         // a is the y part
};

__host__ __device__ __forceinline__ VspPlan vsp_plan(int nx, int ny, int t, int maxw) {
  VspPlan p;
  p.t = t;
  p.swap = nx > ny;
  p.na = p.swap ? ny : nx;
  p.nb = p.swap ? nx : ny;
  const int D = p.nb - p.na;
  p.dlo = -((t - D) >> 1);
  p.w = ((t + D) >> 1) - p.dlo + 1;
  p.kres = D - p.dlo;
  p.kind = D > t ? 0 : p.na == 0 ? 1 : t == 0 ? 2 : 3;
  const int need = t + 1;
  p.W = need <= 2 ? 2 : need <= 3 ? 3 : need <= 5 ? 5 : need <= 9 ? 9 : need <= 17 ? 17 : 33;
  if (p.W > maxw) p.W = maxw;
  return p;
}

#define PJ_KRES_CASES_2(W) case 0: r = vsp_band_k<W, 0>(a, p.na, b, p.nb, p.t, p.dlo, p.w, cells); break; \
                           case 1: r = vsp_band_k<W, 1>(a, p.na, b, p.nb, p.t, p.dlo, p.w, cells); break;
#define PJ_KRES_CASES_3(W) PJ_KRES_CASES_2(W) \
                           case 2: r = vsp_band_k<W, 2>(a, p.na, b, p.nb, p.t, p.dlo, p.w, cells); break;
#define PJ_KRES_CASES_5(W) PJ_KRES_CASES_3(W) \
                           case 3: r = vsp_band_k<W, 3>(a, p.na, b, p.nb, p.t, p.dlo, p.w, cells); break; \
                           case 4: r = vsp_band_k<W, 4>(a, p.na, b, p.nb, p.t, p.dlo, p.w, cells); break;
#define PJ_KRES_CASES_9(W) PJ_KRES_CASES_5(W) \
                           case 5: r = vsp_band_k<W, 5>(a, p.na, b, p.nb, p.t, p.dlo, p.w, cells); break; \
                           case 6: r = vsp_band_k<W, 6>(a, p.na, b, p.nb, p.t, p.dlo, p.w, cells); break; \
                           case 7: r = vsp_band_k<W, 7>(a, p.na, b, p.nb, p.t, p.dlo, p.w, cells); break; \
                           case 8: r = vsp_band_k<W, 8>(a, p.na, b, p.nb, p.t, p.dlo, p.w, cells); break;

// VERIFYSTRINGPAIR (Alg. 3) of x and y with a prepared plan: min(t + 1, ED).
template <int MAXW>
__host__ __device__ __forceinline__ int vsp_run(const VspPlan& p, const uint8_t* x, const uint8_t* y,
                                                unsigned long long& cells) {
  const uint8_t* a = p.swap ? y : x;
  const uint8_t* b = p.swap ? x : y;
  int r = p.t + 1;
  if (p.kind == 1) {
    r = p.nb - p.na;
  } else if (p.kind == 2) {  // exact match of equal lengths
    bool eq = true;
    for (int k = 0; k < p.na; ++k) {
      if (a[k] != b[k]) {
        eq = false;
        break;
      }
    }
    cells += (unsigned long long)p.na;
    r = eq ? 0 : 1;
  } else if (p.kind == 3 && MAXW <= 5) {
    // narrow bands: one code path for every band width and result diagonal,
    // so that the lanes of a warp verifying different matches do not run the
    // compile-time instances below one after another
    r = vsp_band_r<MAXW>(a, p.na, b, p.nb, p.t, p.dlo, p.w, p.kres, cells);
  } else if (p.kind == 3) {
    if (p.W <= 2 || MAXW <= 2) {
      switch (p.kres) { PJ_KRES_CASES_2((MAXW < 2 ? MAXW : 2)) }
    } else if (p.W <= 3 || MAXW <= 3) {
      switch (p.kres) { PJ_KRES_CASES_3((MAXW < 3 ? MAXW : 3)) }
    } else if (p.W <= 5 || MAXW <= 5) {
      switch (p.kres) { PJ_KRES_CASES_5((MAXW < 5 ? MAXW : 5)) }
    } else if (p.W <= 9 || MAXW <= 9) {
      switch (p.kres) { PJ_KRES_CASES_9((MAXW < 9 ? MAXW : 9)) }
    } else if (p.W <= 17 || MAXW <= 17) {
      r = vsp_band<(MAXW < 17 ? MAXW : 17)>(a, p.na, b, p.nb, p.t, cells);
    } else {
      r = vsp_band<MAXW>(a, p.na, b, p.nb, p.t, cells);
    }
  }
  return r;
}

#undef PJ_KRES_CASES_2
#undef PJ_KRES_CASES_3
#undef PJ_KRES_CASES_5
#undef PJ_KRES_CASES_9

// VERIFYSTRINGPAIR (Alg. 3): min(t + 1, ED(x, y)), t <= MAXW - 1.
template <int MAXW>
__host__ __device__ __forceinline__ int vsp(const uint8_t* x, int nx, const uint8_t* y, int ny, int t,
                                            unsigned long long& cells) {
  return vsp_run<MAXW>(vsp_plan(nx, ny, t, MAXW), x, y, cells);
}

// Shared-prefix form of VERIFYSTRINGPAIR (Sec. 5.3), for verifying one
// probing string s against a sequence of indexed strings r in (nearly)
// alphabetical order: the rows run over r and the columns over s, so rows
// 1..c of two r's that share their first c characters (and their length,
// hence the band) are identical, and the second can start from the band
// values after row c of the first.
//
// Band: diagonals d = j - i from dlo = -floor((t - D)/2), D = |s| - |r| (any
// sign, |D| <= t), W registers; cells left of column 0 start at t + 1, and
// Lemma 4 tests E(i, j) = M(i, j) + |D - (j - i)| over the row (as vsp_band).
// V holds the band after row `start` (start = 0: it is set here to row 0);
// rows start + 1 .. |r| are computed, a copy of the band after row snap_row
// is left in snap when that row is computed, and dead receives the row at
// which Lemma 4 stopped the scan (0 when it ran to the end).  Returns
// min(t + 1, ED(r, s)).  Requires |r| >= 1 and |D| <= t.
template <int W>
__host__ __device__ __forceinline__ int vsp_rows(const uint8_t* r, int nr, const uint8_t* s, int ns, int t, int start,
                                                 int (&V)[W], int snap_row, int (&snap)[W], int& dead,
                                                 unsigned long long& cells) {
  const int D = ns - nr;
  const int cap = t + 1;
  const int dlo = -((t - D) >> 1);
  const int w = ((t + D) >> 1) - dlo + 1;
  const int slast = ns - 1;
  int eoff[W];
  uint8_t B[W];  // B[k] = s[i + dlo + k - 1] for the row i being computed (index clamped)
#pragma unroll
  for (int k = 0; k < W; ++k) {
    const int j = dlo + k;
    if (start == 0) V[k] = j < 0 ? cap : j;  // row 0: M(0, j) = j
    eoff[k] = abs(D - dlo - k);
    B[k] = ns > 0 ? s[min(max(start + j, 0), slast)] : (uint8_t)0;
  }
  dead = 0;
  int rows = 0;
  for (int i = start + 1; i <= nr; ++i) {
    const uint8_t ca = r[i - 1];
    int left = cap;
    int emin = cap;
#pragma unroll
    for (int k = 0; k < W; ++k) {
      const int up = (k + 1 < W) ? V[k + 1] : cap;
      const int diag = V[k] + (ca != B[k] ? 1 : 0);
      const int val = min(diag, min(up, left) + 1);
      V[k] = val;
      left = val;
      emin = min(emin, val + eoff[k]);
    }
    ++rows;
    if (i == snap_row) {
#pragma unroll
      for (int k = 0; k < W; ++k) snap[k] = V[k];
    }
    if (emin > t) {  // Lemma 4
      dead = i;
      break;
    }
    const int jn = i + dlo + W - 1;
#pragma unroll
    for (int k = 0; k + 1 < W; ++k) B[k] = B[k + 1];
    B[W - 1] = ns > 0 ? s[min(max(jn, 0), slast)] : (uint8_t)0;
  }
  cells += (unsigned long long)(rows * w);
  int res = cap;
  if (!dead) {
    const int kres = D - dlo;
#pragma unroll
    for (int k = 0; k < W; ++k)
      if (k == kres) res = min(V[k], cap);
  }
  return res;
}

// Length of the common prefix of a and b (n bytes at most).
__host__ __device__ __forceinline__ int common_prefix(const uint8_t* a, const uint8_t* b, int n) {
  int k = 0;
  while (k < n && a[k] == b[k]) ++k;
  return k;
}

#ifdef __CUDACC__
// Warp-cooperative VERIFYSTRINGPAIR for long strings: all 32 lanes of a warp
// work on ONE pair, lane l holding band diagonals k = 2l and 2l+1 (up to 64
// diagonals, so t <= 63).  A row needs the previous row's value one diagonal
// up (a shuffle from the next lane) and, for the left neighbour in the same
// row, a min-plus prefix over the lanes: lane l's two cells map the value L
// left of them to min(B_l, L + 2) with B_l = min(x_1, x_0 + 1), and these
// maps compose by a 5-step shuffle scan.  The Lemma 4 test is one ballot per
// row (any lane with an expected edit distance <= t).  Every lane runs the
// same control flow: callers must enter it with the whole warp converged and
// with the same arguments in every lane.
__device__ __forceinline__ int vsp_warp(const uint8_t* x, int nx, const uint8_t* y, int ny, int t,
                                        unsigned long long& cells) {
  const unsigned FULLM = 0xffffffffu;
  const int lane = threadIdx.x & 31;
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
    const int w = ((t + D) >> 1) - dlo + 1;
    const int k0 = 2 * lane, k1 = 2 * lane + 1;
    int V0 = dlo + k0 < 0 ? cap : min(dlo + k0, cap);
    int V1 = dlo + k1 < 0 ? cap : min(dlo + k1, cap);
    const int e0 = abs(D - dlo - k0), e1 = abs(D - dlo - k1);
    bool alive = true;
    for (int i = 1; i <= na; ++i) {
      const uint8_t ca = a[i - 1];
      const int jb0 = i + dlo + k0 - 1, jb1 = jb0 + 1;
      const int c0 = (jb0 >= 0 && jb0 < nb) ? (int)b[jb0] : -1;
      const int c1 = (jb1 >= 0 && jb1 < nb) ? (int)b[jb1] : -1;
      const int upn = __shfl_down_sync(FULLM, V0, 1);
      const int up1 = lane == 31 ? cap : upn;
      const int x0 = min(V0 + ((int)ca != c0 ? 1 : 0), V1 + 1);
      const int x1 = min(V1 + ((int)ca != c1 ? 1 : 0), up1 + 1);
      int S = min(x1, x0 + 1);
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int T = __shfl_up_sync(FULLM, S, o);
        if (lane >= o) S = min(S, T + 2 * o);
      }
      const int Sl = __shfl_up_sync(FULLM, S, 1);
      const int L = lane == 0 ? cap : Sl;
      V0 = min(min(x0, L + 1), cap);
      V1 = min(min(x1, V0 + 1), cap);
      cells += (unsigned long long)w;
      if (!__any_sync(FULLM, (V0 + e0 <= t) || (V1 + e1 <= t))) {  // Lemma 4
        alive = false;
        break;
      }
    }
    const int kres = D - dlo;
    const int mine = (kres & 1) ? V1 : V0;
    const int v = __shfl_sync(FULLM, mine, (kres >> 1) & 31);
    if (alive) res = v;
  }
  return res;
}

// vsp_warp with the rows over r and the columns over s whatever their
// lengths (D = |s| - |r| of either sign, |D| <= t), resumable like vsp_rows:
// V0, V1 hold each lane's two band values after row `start` (set here when
// start = 0), rows start + 1 .. |r| are computed, the values after row
// snap_row are copied to S0, S1 when that row is computed, and dead receives
// the row at which Lemma 4 stopped the scan (0: ran to the end).  Every lane
// must call it with the same arguments, the warp converged.
__device__ __forceinline__ int vsp_warp_rows(const uint8_t* r, int nr, const uint8_t* s, int ns, int t, int start,
                                             int& V0, int& V1, int snap_row, int& S0, int& S1, int& dead,
                                             unsigned long long& cells) {
  const unsigned FULLM = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  const int D = ns - nr;
  const int cap = t + 1;
  const int dlo = -((t - D) >> 1);
  const int w = ((t + D) >> 1) - dlo + 1;
  const int k0 = 2 * lane, k1 = 2 * lane + 1;
  if (start == 0) {
    V0 = dlo + k0 < 0 ? cap : min(dlo + k0, cap);
    V1 = dlo + k1 < 0 ? cap : min(dlo + k1, cap);
  }
  const int e0 = abs(D - dlo - k0), e1 = abs(D - dlo - k1);
  dead = 0;
  for (int i = start + 1; i <= nr; ++i) {
    const uint8_t ca = r[i - 1];
    const int jb0 = i + dlo + k0 - 1, jb1 = jb0 + 1;
    const int c0 = (jb0 >= 0 && jb0 < ns) ? (int)s[jb0] : -1;
    const int c1 = (jb1 >= 0 && jb1 < ns) ? (int)s[jb1] : -1;
    const int upn = __shfl_down_sync(FULLM, V0, 1);
    const int up1 = lane == 31 ? cap : upn;
    const int x0 = min(V0 + ((int)ca != c0 ? 1 : 0), V1 + 1);
    const int x1 = min(V1 + ((int)ca != c1 ? 1 : 0), up1 + 1);
    int S = min(x1, x0 + 1);
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int T = __shfl_up_sync(FULLM, S, o);
      if (lane >= o) S = min(S, T + 2 * o);
    }
    const int Sl = __shfl_up_sync(FULLM, S, 1);
    const int L = lane == 0 ? cap : Sl;
    V0 = min(min(x0, L + 1), cap);
    V1 = min(min(x1, V0 + 1), cap);
    cells += (unsigned long long)w;
    if (i == snap_row) {
      S0 = V0;
      S1 = V1;
    }
    if (!__any_sync(FULLM, (V0 + e0 <= t) || (V1 + e1 <= t))) {  // Lemma 4
      dead = i;
      break;
    }
  }
  const int kres = D - dlo;
  const int mine = (kres & 1) ? V1 : V0;
  const int v = __shfl_sync(FULLM, mine, (kres >> 1) & 31);
  return dead ? cap : v;
}

// extension-based verification with the warp-cooperative VERIFYSTRINGPAIR
// (the side with the smaller threshold first, as in verify_ext)
__device__ __forceinline__ bool verify_ext_warp(const uint8_t* s, int ls, const uint8_t* r, int lr, int i, int p,
                                                int li, int P, int tau, bool check_segment, int& ed,
                                                unsigned long long& cells) {
  bool same = true;
  for (int k = 0; check_segment && k < li; ++k) {
    if (s[p + k] != r[P + k]) {
      same = false;
      break;
    }
  }
  bool ok = false;
  if (same) {
    const int tl = i - 1, tr = tau + 1 - i;
    const bool rf = tr < tl;
    const int t1 = rf ? tr : tl, t2 = rf ? tl : tr;
    const int d1 = rf ? vsp_warp(s + p + li, ls - p - li, r + P + li, lr - P - li, t1, cells)
                      : vsp_warp(s, p, r, P, t1, cells);
    if (d1 <= t1) {
      const int d2 = rf ? vsp_warp(s, p, r, P, t2, cells)
                        : vsp_warp(s + p + li, ls - p - li, r + P + li, lr - P - li, t2, cells);
      if (d2 <= t2) {
        ed = d1 + d2;
        ok = true;
      }
    }
  }
  return ok;
}
#endif

// Extension-based verification of one match (Sec. 5.2, Alg. 3).  s has the
// selected substring at p; r is the indexed string whose segment i (start P,
// length li) it matched; check_segment false when the lookup already proved
// the two segments equal.  Returns true with ed = d_l + d_r when accepted.
// Both sides must pass (d_l <= i-1 and d_r <= tau+1-i), so they may be
// checked in either order: the side with the smaller threshold goes first
// (its band is narrower and it rejects more often).
template <int MAXW>
__host__ __device__ __forceinline__ bool verify_ext(const uint8_t* s, int ls, const uint8_t* r, int lr, int i, int p, int li,
                                                    int P, int tau, bool check_segment, int& ed,
                                                    unsigned long long& cells) {
  bool same = true;
  for (int k = 0; check_segment && k < li; ++k) {
    if (s[p + k] != r[P + k]) {  // hash collision, not a match
      same = false;
      break;
    }
  }
  bool ok = false;
  if (same) {
    const int tl = i - 1, tr = tau + 1 - i;
    const bool rf = tr < tl;
    const uint8_t* x1 = rf ? s + p + li : s;
    const uint8_t* y1 = rf ? r + P + li : r;
    const int n1 = rf ? ls - p - li : p, m1 = rf ? lr - P - li : P;
    const uint8_t* x2 = rf ? s : s + p + li;
    const uint8_t* y2 = rf ? r : r + P + li;
    const int n2 = rf ? p : ls - p - li, m2 = rf ? P : lr - P - li;
    const int t1 = rf ? tr : tl, t2 = rf ? tl : tr;
    const int d1 = vsp<MAXW>(x1, n1, y1, m1, t1, cells);
    if (d1 <= t1) {
      const int d2 = vsp<MAXW>(x2, n2, y2, m2, t2, cells);
      if (d2 <= t2) {
        ed = d1 + d2;
        ok = true;
      }
    }
  }
  return ok;
}

}  // namespace pj
