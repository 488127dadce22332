/*
 * Pass-Join CPU oracle: plain brute-force edit-distance similarity join.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * benchmark's CPU-baseline leg may load this library.  It shares no code,
 * header, table or helper with the CUDA path.
 *
 * What it computes is the plain definition of the problem, not the method:
 *
 *   Def. 1 (Sec. 2): given string sets R, S and a threshold tau, report every
 *   pair <r, s> with ED(r, s) <= tau, where ED is the minimum number of
 *   single-character insertions, deletions and substitutions.
 *
 *   ED is evaluated with the Wagner-Fischer recurrence of Sec. 5.1:
 *     M(0, j) = j,  M(i, 0) = i,
 *     M(i, j) = min(M(i-1, j) + 1, M(i, j-1) + 1, M(i-1, j-1) + delta),
 *   delta = 0 iff the i-th character of r equals the j-th character of s.
 *   (The paper writes the recurrence for 0 <= j, which would reference
 *   M(i, -1); the oracle reads the first column as M(i, 0) = i.)
 *
 *   Pairs whose lengths differ by more than tau are skipped without a DP:
 *   ED(r, s) >= ||r| - |s|| (the length filter named in Sec. 3.2).
 *
 * A second, faster variant ("banded") restricts each row to |i - j| <= tau
 * (the 2*tau+1 band named in Sec. 5.1 as prior work) and stops once a whole
 * row exceeds tau.  Every cell outside the band has M(i, j) >= |i - j| > tau,
 * and a row whose minimum exceeds tau bounds every later row from below, so
 * min(tau + 1, ED) is unchanged.  It exists only so that sampled checks at
 * full workload sizes finish; the tests pin it to the plain DP.
 *
 * Output convention (self join): one record per unordered pair of distinct
 * ids, a < b, sorted by (a, b).  Join: a indexes R, b indexes S, sorted.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef struct {
  uint32_t a, b, ed;
} oracle_pair;

/* ---------------------------------------------------------------- ED ---- */

/* Full Wagner-Fischer DP over the (|r|+1) x (|s|+1) matrix, two rows kept. */
static int32_t ed_full(const uint8_t* r, int64_t nr, const uint8_t* s, int64_t ns,
                       int32_t* row_prev, int32_t* row_cur) {
  for (int64_t j = 0; j <= ns; ++j) row_prev[j] = (int32_t)j; /* M(0, j) = j */
  for (int64_t i = 1; i <= nr; ++i) {
    row_cur[0] = (int32_t)i; /* M(i, 0) = i */
    for (int64_t j = 1; j <= ns; ++j) {
      int32_t del = row_prev[j] + 1;
      int32_t ins = row_cur[j - 1] + 1;
      int32_t sub = row_prev[j - 1] + (r[i - 1] == s[j - 1] ? 0 : 1);
      int32_t m = del < ins ? del : ins;
      row_cur[j] = m < sub ? m : sub;
    }
    int32_t* t = row_prev;
    row_prev = row_cur;
    row_cur = t;
  }
  return row_prev[ns];
}

/* Banded DP: cells with |i - j| > tau are taken as tau + 1, values saturate
 * at tau + 1, and the scan stops once a row's minimum exceeds tau.  Returns
 * min(tau + 1, ED).  Both row buffers hold ns + 1 entries. */
static int32_t ed_banded(const uint8_t* r, int64_t nr, const uint8_t* s, int64_t ns,
                         int32_t tau, int32_t* row_prev, int32_t* row_cur) {
  const int32_t cap = tau + 1;
  int64_t d = nr > ns ? nr - ns : ns - nr;
  if (d > tau) return cap;
  for (int64_t j = 0; j <= ns; ++j) row_prev[j] = j <= tau ? (int32_t)j : cap; /* row 0 */
  for (int64_t i = 1; i <= nr; ++i) {
    int64_t jlo = i - tau, jhi = i + tau;
    if (jlo < 0) jlo = 0;
    if (jhi > ns) jhi = ns;
    if (jlo >= 1) row_cur[jlo - 1] = cap; /* left neighbour of the band */
    int32_t row_min = cap;
    for (int64_t j = jlo; j <= jhi; ++j) {
      int32_t v;
      if (j == 0) {
        v = (int32_t)i; /* M(i, 0) = i; jlo == 0 implies i <= tau */
      } else {
        int32_t del = row_prev[j] + 1;
        int32_t ins = row_cur[j - 1] + 1;
        int32_t sub = row_prev[j - 1] + (r[i - 1] == s[j - 1] ? 0 : 1);
        v = del < ins ? del : ins;
        v = v < sub ? v : sub;
      }
      if (v > cap) v = cap;
      row_cur[j] = v;
      if (v < row_min) row_min = v;
    }
    if (jhi + 1 <= ns) row_cur[jhi + 1] = cap; /* read as "up" by the next row */
    if (row_min > tau) return cap;
    int32_t* t = row_prev;
    row_prev = row_cur;
    row_cur = t;
  }
  int32_t v = row_prev[ns];
  return v > cap ? cap : v;
}

/* Public: plain ED of two byte strings. */
int32_t oracle_ed(const uint8_t* r, int64_t nr, const uint8_t* s, int64_t ns) {
  int32_t* buf = (int32_t*)malloc(sizeof(int32_t) * 2 * (size_t)(ns + 1));
  if (!buf) return -1;
  int32_t v = ed_full(r, nr, s, ns, buf, buf + ns + 1);
  free(buf);
  return v;
}

/* Public: min(tau + 1, ED) by the banded variant. */
int32_t oracle_ed_banded(const uint8_t* r, int64_t nr, const uint8_t* s, int64_t ns,
                         int32_t tau) {
  if (tau < 0) return -1;
  int32_t* buf = (int32_t*)malloc(sizeof(int32_t) * 2 * (size_t)(ns + 1));
  if (!buf) return -1;
  int32_t v = ed_banded(r, nr, s, ns, tau, buf, buf + ns + 1);
  free(buf);
  return v;
}

/* ------------------------------------------------------------ joins ---- */

typedef struct {
  oracle_pair* v;
  int64_t n, cap;
} pair_vec;

static int vec_push(pair_vec* pv, uint32_t a, uint32_t b, uint32_t ed) {
  if (pv->n == pv->cap) {
    int64_t nc = pv->cap ? pv->cap * 2 : 1024;
    oracle_pair* nv = (oracle_pair*)realloc(pv->v, sizeof(oracle_pair) * (size_t)nc);
    if (!nv) return -1;
    pv->v = nv;
    pv->cap = nc;
  }
  pv->v[pv->n].a = a;
  pv->v[pv->n].b = b;
  pv->v[pv->n].ed = ed;
  pv->n++;
  return 0;
}

static int cmp_pair(const void* x, const void* y) {
  const oracle_pair* p = (const oracle_pair*)x;
  const oracle_pair* q = (const oracle_pair*)y;
  if (p->a != q->a) return p->a < q->a ? -1 : 1;
  if (p->b != q->b) return p->b < q->b ? -1 : 1;
  return 0;
}

static int64_t max_len(const uint64_t* off, int64_t n) {
  int64_t m = 0;
  for (int64_t k = 0; k < n; ++k) {
    int64_t l = (int64_t)(off[k + 1] - off[k]);
    if (l > m) m = l;
  }
  return m;
}

/*
 * Generic all-pairs driver.  Rows: strings of set A; for each x in A the
 * candidate partners are y in B (y > x when self, all of B otherwise).
 * Every partner within the length filter gets a full DP (or the banded
 * variant).  Results go to out (capacity cap); the return value is the total
 * number of similar pairs, which the caller compares with cap.
 */
static int64_t join_driver(const uint8_t* abytes, const uint64_t* aoff, int64_t na,
                           const uint8_t* bbytes, const uint64_t* boff, int64_t nb,
                           int self, int32_t tau, int banded, oracle_pair* out, int64_t cap,
                           int nthreads) {
  if (tau < 0) return -1;
  int64_t lmax = max_len(boff, nb);
  int64_t lmax_a = max_len(aoff, na);
  if (lmax_a > lmax) lmax = lmax_a;
  int nt = 1;
#ifdef _OPENMP
  nt = nthreads > 0 ? nthreads : omp_get_max_threads();
#endif
  pair_vec* vecs = (pair_vec*)calloc((size_t)nt, sizeof(pair_vec));
  if (!vecs) return -1;
  int failed = 0;
#ifdef _OPENMP
#pragma omp parallel num_threads(nt)
#endif
  {
    int tid = 0;
#ifdef _OPENMP
    tid = omp_get_thread_num();
#endif
    int32_t* buf = (int32_t*)malloc(sizeof(int32_t) * 2 * (size_t)(lmax + 2));
    if (!buf) failed = 1;
#ifdef _OPENMP
#pragma omp for schedule(dynamic, 16)
#endif
    for (int64_t x = 0; x < na; ++x) {
      if (!buf) continue;
      const uint8_t* sx = abytes + aoff[x];
      int64_t lx = (int64_t)(aoff[x + 1] - aoff[x]);
      for (int64_t y = self ? x + 1 : 0; y < nb; ++y) {
        const uint8_t* sy = bbytes + boff[y];
        int64_t ly = (int64_t)(boff[y + 1] - boff[y]);
        int64_t dl = lx > ly ? lx - ly : ly - lx;
        if (dl > tau) continue; /* length filter */
        int32_t d;
        if (banded) {
          d = ed_banded(sx, lx, sy, ly, tau, buf, buf + ly + 1);
        } else {
          d = ed_full(sx, lx, sy, ly, buf, buf + ly + 1);
        }
        if (d <= tau) {
          if (vec_push(&vecs[tid], (uint32_t)x, (uint32_t)y, (uint32_t)d)) failed = 1;
        }
      }
    }
    free(buf);
  }
  int64_t total = 0;
  for (int t = 0; t < nt; ++t) total += vecs[t].n;
  if (!failed && total <= cap && out) {
    int64_t k = 0;
    for (int t = 0; t < nt; ++t) {
      memcpy(out + k, vecs[t].v, sizeof(oracle_pair) * (size_t)vecs[t].n);
      k += vecs[t].n;
    }
    qsort(out, (size_t)total, sizeof(oracle_pair), cmp_pair);
  }
  for (int t = 0; t < nt; ++t) free(vecs[t].v);
  free(vecs);
  return failed ? -1 : total;
}

/* Self join of one string set (Def. 1 with R = S, Sec. 2).  Returns the
 * number of similar pairs (a < b), or -1 on error.  If it exceeds cap the
 * output buffer is left untouched; call again with a larger buffer. */
int64_t oracle_self_join(const uint8_t* bytes, const uint64_t* off, int64_t n, int32_t tau,
                         int banded, oracle_pair* out, int64_t cap, int nthreads) {
  return join_driver(bytes, off, n, bytes, off, n, 1, tau, banded, out, cap, nthreads);
}

/* Join of two distinct sets (Def. 1, R != S): a indexes R, b indexes S. */
int64_t oracle_join(const uint8_t* rbytes, const uint64_t* roff, int64_t nr,
                    const uint8_t* sbytes, const uint64_t* soff, int64_t ns, int32_t tau,
                    int banded, oracle_pair* out, int64_t cap, int nthreads) {
  return join_driver(rbytes, roff, nr, sbytes, soff, ns, 0, tau, banded, out, cap, nthreads);
}

int oracle_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

/*
 * Sampled check at full workload sizes: for each of nq query strings, every
 * string y of the set S with ED(q, y) <= tau (Def. 1 restricted to one row of
 * R x S).  Parallel over S rather than over the queries, since nq is small.
 * Output a = query index, b = index in S, sorted by (a, b).  When exclude is
 * non-NULL, pairs (q, exclude[q]) are dropped (a string is not its own match
 * in a self join).
 */
int64_t oracle_similar_to(const uint8_t* qbytes, const uint64_t* qoff, int64_t nq,
                          const uint8_t* sbytes, const uint64_t* soff, int64_t ns,
                          int32_t tau, int banded, const int64_t* exclude,
                          oracle_pair* out, int64_t cap, int nthreads) {
  if (tau < 0) return -1;
  int64_t lmax = max_len(soff, ns);
  int64_t lq = max_len(qoff, nq);
  if (lq > lmax) lmax = lq;
  int nt = 1;
#ifdef _OPENMP
  nt = nthreads > 0 ? nthreads : omp_get_max_threads();
#endif
  pair_vec* vecs = (pair_vec*)calloc((size_t)nt, sizeof(pair_vec));
  if (!vecs) return -1;
  int failed = 0;
#ifdef _OPENMP
#pragma omp parallel num_threads(nt)
#endif
  {
    int tid = 0;
#ifdef _OPENMP
    tid = omp_get_thread_num();
#endif
    int32_t* buf = (int32_t*)malloc(sizeof(int32_t) * 2 * (size_t)(lmax + 2));
    if (!buf) failed = 1;
    for (int64_t q = 0; q < nq; ++q) {
      const uint8_t* sq = qbytes + qoff[q];
      int64_t lx = (int64_t)(qoff[q + 1] - qoff[q]);
#ifdef _OPENMP
#pragma omp for schedule(dynamic, 4096)
#endif
      for (int64_t y = 0; y < ns; ++y) {
        if (!buf) continue;
        if (exclude && exclude[q] == y) continue;
        const uint8_t* sy = sbytes + soff[y];
        int64_t ly = (int64_t)(soff[y + 1] - soff[y]);
        int64_t dl = lx > ly ? lx - ly : ly - lx;
        if (dl > tau) continue;
        int32_t d = banded ? ed_banded(sq, lx, sy, ly, tau, buf, buf + ly + 1)
                           : ed_full(sq, lx, sy, ly, buf, buf + ly + 1);
        if (d <= tau) {
          if (vec_push(&vecs[tid], (uint32_t)q, (uint32_t)y, (uint32_t)d)) failed = 1;
        }
      }
    }
    free(buf);
  }
  int64_t total = 0;
  for (int t = 0; t < nt; ++t) total += vecs[t].n;
  if (!failed && total <= cap && out) {
    int64_t k = 0;
    for (int t = 0; t < nt; ++t) {
      memcpy(out + k, vecs[t].v, sizeof(oracle_pair) * (size_t)vecs[t].n);
      k += vecs[t].n;
    }
    qsort(out, (size_t)total, sizeof(oracle_pair), cmp_pair);
  }
  for (int t = 0; t < nt; ++t) free(vecs[t].v);
  free(vecs);
  return failed ? -1 : total;
}
