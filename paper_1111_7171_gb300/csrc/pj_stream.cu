// Self joins split by probing string: a resident index joined shard by
// shard, and a set too large for the device joined window by window.
//
// Every similar pair of the self join is found by exactly one probe: the
// later of its two strings in the store's sid order (Alg. 1 probes each string
// against the strings visited before it).  Joins over disjoint ranges of
// probing strings therefore return disjoint pair sets whose union is the
// whole join.
//
//   pj_self_join_shard   splits the probes of a resident index into
//                        n_shards equal sid ranges (one per GPU or per call).
//   pj_self_join_stream  never holds the whole set on the device.  When the
//                        strings are visited by length, the only inverted
//                        lists a string of length |s| probes are those of
//                        lengths |s| - tau .. |s| (Sec. 3.2), so a window of
//                        consecutive probing strings needs on the device only
//                        itself plus the strings before it whose length is
//                        at least its first probe's length - tau.  Each
//                        window builds a temporary store and segment index
//                        of that set and self-joins it with only its own
//                        strings probing; the host maps the window's pairs
//                        back to input ids and merges the windows' sorted
//                        results.
#include <algorithm>
#include <deque>
#include <future>
#include <queue>
#include <vector>

#include "pj_internal.cuh"

namespace pj {
namespace {

struct Window {
  uint32_t p0, p1;  // probing strings: positions p0 .. p1 - 1 of the store order
};

// Device bytes a window's store, segment index and join scratch are expected
// to take (the budget check during the build and join is exact; this only
// sizes the first attempt).
uint64_t window_estimate(const std::vector<uint64_t>& cum_bytes, const std::vector<uint32_t>& len_of,
                         const std::vector<uint32_t>& lbeg, uint32_t p0, uint32_t p1, int tau) {
  const int l0 = (int)len_of[p0];
  const uint32_t d0 = lbeg[std::max(0, l0 - tau)];
  const uint64_t nd = p1 - d0, np = p1 - p0;
  const uint64_t bytes = cum_bytes[p1] - cum_bytes[d0];
  const uint64_t parts = (uint64_t)tau + 1;
  return bytes * 6 + nd * 96 + nd * parts * 128 + np * parts * parts * 32 + (8ull << 20);
}

void self_join_stream(const pj_strings& S, int tau, const pj_options* opt, pj_result* out) {
  if (S.on_device) fail(PJ_EINVAL, "pj_self_join_stream: the strings must be in host memory");
  if (opt && opt->partition != PJ_PARTITION_EVEN && opt->partition != PJ_PARTITION_CENTER)
    fail(PJ_EINVAL, "pj_self_join_stream: unknown partition scheme");
  const uint32_t n = S.n;
  if (!S.offsets || (!S.bytes && n > 0)) fail(PJ_EINVAL, "pj_strings: NULL bytes or offsets");
  // (length, first eight bytes, id) order on the host, as the store orders
  // strings: a stable counting sort by length, then a sort within each length
  std::vector<uint32_t> len(n);
  int lmax = 0;
  for (uint32_t k = 0; k < n; ++k) {
    if (S.offsets[k + 1] < S.offsets[k] || S.offsets[k + 1] - S.offsets[k] > PJ_MAX_STRING_LEN)
      fail(PJ_EINVAL, "pj_strings: offsets decrease or a string is longer than 65535 bytes");
    len[k] = (uint32_t)(S.offsets[k + 1] - S.offsets[k]);
    lmax = std::max(lmax, (int)len[k]);
  }
  std::vector<uint32_t> lbeg((size_t)lmax + 2, 0);  // first position of each length
  for (uint32_t k = 0; k < n; ++k) ++lbeg[len[k] + 1];
  for (int l = 0; l <= lmax; ++l) lbeg[l + 1] += lbeg[l];
  std::vector<uint32_t> order(n), len_of(n);
  {
    std::vector<uint32_t> next(lbeg.begin(), lbeg.end() - 1);
    for (uint32_t k = 0; k < n; ++k) order[next[len[k]]++] = k;
  }
  // within each length, the store's order: by the first eight bytes (first
  // byte highest, zero-padded), then by id -- so that every window's own
  // store keeps the window's strings in this order and its probe range
  // stays a range of its sids
  {
    auto prefix_key = [&](uint32_t id) {
      unsigned long long key = 0;
      const uint8_t* p = S.bytes + S.offsets[id];
      for (uint32_t j = 0; j < 8; ++j) key = (key << 8) | (j < len[id] ? p[j] : 0u);
      return key;
    };
    std::vector<std::pair<unsigned long long, uint32_t>> tmp;
    for (int l = 0; l <= lmax; ++l) {
      const uint32_t b = lbeg[l], e = lbeg[l + 1];
      if (e - b < 2) continue;
      tmp.clear();
      for (uint32_t j = b; j < e; ++j) tmp.emplace_back(prefix_key(order[j]), order[j]);
      std::sort(tmp.begin(), tmp.end());  // ties: ascending id
      for (uint32_t j = b; j < e; ++j) order[j] = tmp[j - b].second;
    }
  }
  std::vector<uint64_t> cum_bytes((size_t)n + 1, 0);
  for (uint32_t p = 0; p < n; ++p) {
    len_of[p] = len[order[p]];
    cum_bytes[p + 1] = cum_bytes[p] + len_of[p];
  }

  Ctx base = make_ctx(opt);
  if (!base.budget) {  // no budget given: three quarters of the free device memory
    size_t free_b = 0, total_b = 0;
    PJ_CUDA(cudaMemGetInfo(&free_b, &total_b));
    base.budget = std::make_shared<Budget>();
    base.budget->limit = free_b / 4 * 3;
  }
  const uint64_t target = base.budget->limit / 2;
  // the first window holds every string of length <= 2 tau: pairs with a
  // string too short to partition (length <= tau) are verified directly, and
  // both their strings are then in that window
  const uint32_t first_min = lbeg[std::min(2 * tau + 1, lmax + 1)];

  std::deque<Window> todo;
  for (uint32_t p0 = 0; p0 < n;) {
    uint32_t lo = std::max(p0 + 1, p0 == 0 ? first_min : 0u), hi = n;  // largest p1 in [lo, n] that fits
    if (lo >= n || window_estimate(cum_bytes, len_of, lbeg, p0, n, tau) <= target) {
      lo = n;
    } else {
      while (lo < hi) {
        const uint32_t mid = lo + (hi - lo + 1) / 2;
        if (window_estimate(cum_bytes, len_of, lbeg, p0, mid, tau) <= target) lo = mid; else hi = mid - 1;
      }
    }
    todo.push_back(Window{p0, lo});
    p0 = lo;
  }

  std::vector<std::vector<pj_pair>> parts;
  pj_stats total{};
  uint32_t windows = 0;
  std::vector<uint8_t> hbytes;
  std::vector<uint64_t> hoff;
  while (!todo.empty()) {
    const Window w = todo.front();
    todo.pop_front();
    const int l0 = (int)len_of[w.p0];
    const uint32_t d0 = lbeg[std::max(0, l0 - tau)];
    // the window's strings in the store order, as one host string set
    const uint32_t nd = w.p1 - d0;
    hbytes.resize(std::max<uint64_t>(1, cum_bytes[w.p1] - cum_bytes[d0]));
    hoff.assign((size_t)nd + 1, 0);
    for (uint32_t k = 0; k < nd; ++k) {
      const uint32_t id = order[d0 + k];
      const uint64_t L = len[id];
      if (L) memcpy(hbytes.data() + hoff[k], S.bytes + S.offsets[id], L);
      hoff[k + 1] = hoff[k] + L;
    }
    pj_strings ws{hbytes.data(), hoff.data(), nd, 0};
    pj_result r{};
    pj_index* tmp = new pj_index();
    try {
      tmp->ctx = base;  // shares the call's budget
      tmp->verify_mode = opt ? opt->verify_mode : PJ_VERIFY_AUTO;
      tmp->scheme = opt ? opt->partition : PJ_PARTITION_EVEN;
      tmp->autotune = opt ? opt->autotune != 0 : false;
      if (opt && opt->autotune_cache) tmp->autotune_cache = opt->autotune_cache;
      PJ_CUDA(cudaGetDevice(&tmp->device));
      build_store(*tmp, ws);
      tmp->parts.resize(tau + 1);
      build_partition(*tmp, tau, tmp->parts[tau]);
      self_join_range(*tmp, tau, w.p0 - d0, w.p1 - d0, w.p0 == 0, &r, false);
      tmp->ctx.sync();
    } catch (const Error& e) {
      pj_result_free(&r);
      pj_index_free(tmp);
      const bool splittable = w.p1 - w.p0 >= 2 && (w.p0 != 0 || w.p0 + (w.p1 - w.p0) / 2 >= first_min);
      if (e.code != PJ_ENOMEM || !splittable) throw;
      const uint32_t mid = w.p0 + (w.p1 - w.p0) / 2;  // too large for the budget: split and retry
      todo.push_front(Window{mid, w.p1});
      todo.push_front(Window{w.p0, mid});
      continue;
    }
    pj_index_free(tmp);
    ++windows;
    // window positions -> input ids (each pair as a < b), sorted
    std::vector<pj_pair> v(r.count);
    for (uint64_t k = 0; k < r.count; ++k) {
      const uint32_t x = order[d0 + r.pairs[k].a], y = order[d0 + r.pairs[k].b];
      v[k] = pj_pair{std::min(x, y), std::max(x, y), r.pairs[k].ed};
    }
    const pj_stats& st = r.stats;
    total.lookups += st.lookups;
    total.candidates += st.candidates;
    total.accepted += st.accepted;
    total.dp_cells += st.dp_cells;
    total.fallback_pairs += st.fallback_pairs;
    total.hits += st.hits;
    total.filtered += st.filtered;
    total.distinct_pairs += st.distinct_pairs;
    total.probe_ms += st.probe_ms;
    total.verify_ms += st.verify_ms;
    total.fallback_ms += st.fallback_ms;
    total.dedupe_ms += st.dedupe_ms;
    total.partition_ms += st.partition_ms;
    total.tune_ms += st.tune_ms;
    total.verify_block = st.verify_block;
    total.warp_min_len = st.warp_min_len;
    total.verify_mode = st.verify_mode;
    total.pair_warp = st.pair_warp;
    pj_result_free(&r);
    parts.push_back(std::move(v));
  }

  // sort every window's pairs (in parallel), then merge them by (a, b)
  auto less = [](const pj_pair& x, const pj_pair& y) { return x.a != y.a ? x.a < y.a : x.b < y.b; };
  {
    std::vector<std::future<void>> jobs;
    for (auto& v : parts) jobs.push_back(std::async(std::launch::async, [&v, &less] { std::sort(v.begin(), v.end(), less); }));
    for (auto& j : jobs) j.get();
  }
  uint64_t count = 0;
  for (const auto& v : parts) count += v.size();
  pj_pair* res = static_cast<pj_pair*>(malloc(std::max<uint64_t>(count, 1) * sizeof(pj_pair)));
  if (!res) fail(PJ_ENOMEM, "host result allocation failed");
  using Head = std::pair<size_t, size_t>;  // (window, position)
  auto later = [&](const Head& x, const Head& y) { return less(parts[y.first][y.second], parts[x.first][x.second]); };
  std::priority_queue<Head, std::vector<Head>, decltype(later)> heap(later);
  for (size_t k = 0; k < parts.size(); ++k)
    if (!parts[k].empty()) heap.push(Head{k, 0});
  uint64_t o = 0;
  while (!heap.empty()) {
    const Head h = heap.top();
    heap.pop();
    res[o++] = parts[h.first][h.second];
    if (h.second + 1 < parts[h.first].size()) heap.push(Head{h.first, h.second + 1});
  }
  host_result(out, res, count);
  out->stats = total;
  out->stats.windows = windows;
  out->stats.device_peak = base.budget->peak;
}

}  // namespace
}  // namespace pj

extern "C" {

int pj_self_join_shard(pj_index* idx, int tau, uint32_t shard, uint32_t n_shards, pj_result* out) {
  if (out) memset(out, 0, sizeof(*out));
  try {
    if (!idx || !out) pj::fail(PJ_EINVAL, "pj_self_join_shard: NULL argument");
    if (tau < 0 || tau >= (int)idx->parts.size()) pj::fail(PJ_EINVAL, "pj_self_join_shard: tau outside 0..tau_max");
    if (n_shards == 0 || shard >= n_shards) pj::fail(PJ_EINVAL, "pj_self_join_shard: shard outside 0..n_shards-1");
    std::lock_guard<std::mutex> g(idx->mu);
    const uint32_t first = pj::ensure_partition(*idx, tau, nullptr).first;
    const uint64_t m = idx->n - first;
    const uint32_t q_lo = first + (uint32_t)(m * shard / n_shards);
    const uint32_t q_hi = first + (uint32_t)(m * (shard + 1) / n_shards);
    pj::self_join_range(*idx, tau, q_lo, q_hi, shard == 0, out, idx->results_on_device);
    if (idx->ctx.budget) out->stats.device_peak = idx->ctx.budget->peak;
    return PJ_OK;
  } catch (const pj::Error& e) {
    pj::set_last_error(e.msg);
    pj_result_free(out);
    return e.code;
  } catch (const std::bad_alloc&) {
    pj::set_last_error("host allocation failed");
    pj_result_free(out);
    return PJ_ENOMEM;
  }
}

int pj_self_join_stream(const pj_strings* S, int tau, const pj_options* opt, pj_result* out) {
  if (out) memset(out, 0, sizeof(*out));
  try {
    if (!S || !out) pj::fail(PJ_EINVAL, "pj_self_join_stream: NULL argument");
    if (tau < 0 || tau > PJ_TAU_LIMIT) pj::fail(PJ_EINVAL, "pj_self_join_stream: tau out of range");
    pj::self_join_stream(*S, tau, opt, out);
    return PJ_OK;
  } catch (const pj::Error& e) {
    pj::set_last_error(e.msg);
    pj_result_free(out);
    return e.code;
  } catch (const std::bad_alloc&) {
    pj::set_last_error("host allocation failed");
    pj_result_free(out);
    return PJ_ENOMEM;
  }
}

}  // extern "C"
