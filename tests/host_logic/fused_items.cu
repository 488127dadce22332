// Checks the fused self join's work items (fused_item in pj_probe.cuh) on the
// host: for every probe range and items size tried, the items cover every
// probe exactly once, each item holds ppi consecutive probes except the one
// that ends at the range's first probe, and the items alternate between the
// two ends of the length order.  Prints "ok <cases>" or the first failure.
#include <cstdio>
#include <vector>

#include "pj_probe.cuh"

int main() {
  long cases = 0;
  const unsigned begins[] = {0u, 1u, 37u, 1000u};
  for (unsigned pbegin : begins)
    for (unsigned pcount = 1; pcount <= 300; ++pcount)
      for (int ppi = 1; ppi <= 40; ++ppi) {
        const unsigned long long n_items = (pcount + ppi - 1) / ppi;
        std::vector<int> seen(pcount, 0);
        for (unsigned long long it = 0; it < n_items; ++it) {
          uint32_t q_beg = 0, q_end = 0;
          const unsigned long long j = pj::fused_item(it, n_items, pbegin, pcount, ppi, q_beg, q_end);
          if (j >= n_items || q_beg < pbegin || q_end > pbegin + pcount || q_beg >= q_end) {
            printf("bad item: begin %u count %u ppi %d it %llu -> j %llu [%u, %u)\n", pbegin, pcount, ppi, it, j,
                   q_beg, q_end);
            return 1;
          }
          if (q_end - q_beg != (unsigned)ppi && q_beg != pbegin) {
            printf("short item inside the range: begin %u count %u ppi %d it %llu\n", pbegin, pcount, ppi, it);
            return 1;
          }
          const bool long_end = (it & 1) == 0;
          if (long_end && j != it / 2) {
            printf("even item not from the long end: count %u ppi %d it %llu j %llu\n", pcount, ppi, it, j);
            return 1;
          }
          for (uint32_t q = q_beg; q < q_end; ++q) ++seen[q - pbegin];
        }
        for (unsigned k = 0; k < pcount; ++k)
          if (seen[k] != 1) {
            printf("probe %u covered %d times: begin %u count %u ppi %d\n", pbegin + k, seen[k], pbegin, pcount, ppi);
            return 1;
          }
        ++cases;
      }
  printf("ok %ld\n", cases);
  return 0;
}
