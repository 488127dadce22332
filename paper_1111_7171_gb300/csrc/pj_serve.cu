// Continuous-batching query server over a resident index.
//
// Requests (a batch of query strings and one threshold each) are queued by
// pj_server_submit.  Each of `slots` worker threads owns a CUDA stream; when
// a slot is free it takes every pending request it can admit -- bounded by a
// query count, a byte count and the device memory currently free -- and runs
// them as ONE multi-threshold batch (query_multi_impl: one probe pass and
// one verification pass for all of them; with use_plans, one replay of the
// slot's query plan, a CUDA graph of the same pipeline).  Requests that arrive while other
// batches run are admitted by the next free slot, so several batches overlap
// on the device.  Results are split back per request; each request's pairs
// are exactly what pj_query returns for it alone.
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <memory>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "pj_internal.cuh"

namespace pj {
namespace {

using Clock = std::chrono::steady_clock;

struct Request {
  uint64_t ticket = 0;
  int tau = 0;
  std::vector<uint8_t> bytes;
  std::vector<uint64_t> off;  // n + 1, starting at 0
  uint32_t n = 0;
  enum State { PENDING, RUNNING, DONE, FAILED, CANCELLED } state = PENDING;
  std::vector<pj_pair> pairs;
  pj_stats stats{};
  int code = PJ_OK;
  std::string msg;
  Clock::time_point t_submit, t_start, t_done;
  uint32_t batch_requests = 0;
};

}  // namespace
}  // namespace pj

struct pj_server {
  pj_index* idx = nullptr;
  pj_server_options opt{};
  std::vector<std::thread> slots;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<std::shared_ptr<pj::Request>> pending;
  std::unordered_map<uint64_t, std::shared_ptr<pj::Request>> all;
  bool stopping = false;
  uint64_t next_ticket = 1;
  uint64_t n_batches = 0, n_requests = 0, n_queries = 0, max_batch_requests = 0;
  uint32_t in_flight = 0, max_in_flight = 0;
  std::vector<pj_plan*> plans;  // one per slot (use_plans)
};

namespace pj {
namespace {

// Runs one batch of requests on the slot's stream; on PJ_ENOMEM splits it.
void run_batch(pj_server& S, const Ctx& c, pj_plan* plan, std::vector<std::shared_ptr<Request>>& batch, size_t lo,
               size_t hi) {
  // concatenate the requests' strings and thresholds
  std::vector<uint64_t> off(1, 0);
  std::vector<uint8_t> bytes, taus;
  std::vector<uint32_t> first(hi - lo + 1, 0);
  for (size_t k = lo; k < hi; ++k) {
    const Request& r = *batch[k];
    first[k - lo] = (uint32_t)taus.size();
    const uint64_t base = bytes.size();
    bytes.insert(bytes.end(), r.bytes.begin(), r.bytes.end());
    for (uint32_t q = 0; q < r.n; ++q) off.push_back(base + r.off[q + 1]);
    taus.insert(taus.end(), r.n, (uint8_t)r.tau);
  }
  first[hi - lo] = (uint32_t)taus.size();
  pj_strings in{};
  in.bytes = bytes.empty() ? nullptr : bytes.data();
  uint8_t dummy = 0;
  if (!in.bytes) in.bytes = &dummy;
  in.offsets = off.data();
  in.n = (uint32_t)taus.size();
  in.on_device = 0;
  pj_result res{};
  int code = PJ_OK;
  std::string msg;
  try {
    if (plan && in.n <= S.opt.max_batch_queries && bytes.size() <= S.opt.max_batch_bytes) {
      code = pj_plan_query(plan, &in, taus.data(), &res);
      if (code != PJ_OK) msg = pj_last_error();
    } else {  // no plan, or one request larger than the plan's limits
      ProbeSet P;
      upload_probe_set(c, in, P);
      query_multi_impl(c, *S.idx, P, taus.data(), &res, false);
    }
  } catch (const Error& e) {
    code = e.code;
    msg = e.msg;
  } catch (const std::bad_alloc&) {
    code = PJ_ENOMEM;
    msg = "host allocation failed";
  }
  if (code == PJ_ENOMEM && hi - lo > 1) {  // admission by memory: halve and retry
    pj_result_free(&res);
    const size_t mid = lo + (hi - lo) / 2;
    run_batch(S, c, plan, batch, lo, mid);
    run_batch(S, c, plan, batch, mid, hi);
    return;
  }
  // split the pairs (sorted by query position) back per request
  std::vector<std::vector<pj_pair>> parts(hi - lo);
  if (code == PJ_OK) {
    size_t k = 0;
    for (uint64_t e = 0; e < res.count; ++e) {
      pj_pair p = res.pairs[e];
      while (p.a >= first[k + 1]) ++k;
      p.a -= first[k];
      parts[k].push_back(p);
    }
  }
  const pj_stats st = res.stats;
  pj_result_free(&res);
  std::lock_guard<std::mutex> g(S.mu);
  const auto now = Clock::now();
  for (size_t k = lo; k < hi; ++k) {
    Request& r = *batch[k];
    r.t_done = now;
    r.batch_requests = (uint32_t)(hi - lo);
    if (r.state == Request::CANCELLED) continue;
    if (code == PJ_OK) {
      r.pairs.swap(parts[k - lo]);
      r.stats = st;
      r.state = Request::DONE;
    } else {
      r.code = code;
      r.msg = msg;
      r.state = Request::FAILED;
    }
  }
  S.cv_done.notify_all();
}

void slot_main(pj_server* Sp, int slot) {
  pj_server& S = *Sp;
  pj_plan* plan = S.plans.empty() ? nullptr : S.plans[slot];
  cudaSetDevice(S.idx->device);
  cudaStream_t stream = nullptr;
  if (cudaStreamCreateWithFlags(&stream, cudaStreamNonBlocking) != cudaSuccess) stream = nullptr;
  Ctx c;
  c.stream = stream;
  for (;;) {
    std::vector<std::shared_ptr<Request>> batch;
    {
      std::unique_lock<std::mutex> lk(S.mu);
      S.cv_work.wait(lk, [&] { return S.stopping || !S.pending.empty(); });
      if (S.stopping && S.pending.empty()) break;
      // admission: query and byte caps, scaled down when device memory is short
      uint64_t max_q = S.opt.max_batch_queries, max_b = S.opt.max_batch_bytes;
      size_t free_b = 0, total_b = 0;
      if (cudaMemGetInfo(&free_b, &total_b) == cudaSuccess && S.opt.bytes_per_query > 0) {
        const uint64_t usable = free_b > S.opt.device_reserve ? free_b - S.opt.device_reserve : 0;
        max_q = std::min<uint64_t>(max_q, std::max<uint64_t>(1, usable / S.opt.bytes_per_query));
      }
      uint64_t nq = 0, nb = 0;
      while (!S.pending.empty()) {
        const auto& r = S.pending.front();
        if (!batch.empty() && (nq + r->n > max_q || nb + r->bytes.size() > max_b)) break;
        nq += r->n;
        nb += r->bytes.size();
        r->state = Request::RUNNING;
        r->t_start = Clock::now();
        batch.push_back(r);
        S.pending.pop_front();
      }
      S.n_batches++;
      S.n_queries += nq;
      S.max_batch_requests = std::max<uint64_t>(S.max_batch_requests, batch.size());
      S.in_flight++;
      S.max_in_flight = std::max(S.max_in_flight, S.in_flight);
    }
    run_batch(S, c, plan, batch, 0, batch.size());
    std::lock_guard<std::mutex> g(S.mu);
    S.in_flight--;
  }
  if (stream) {
    cudaStreamSynchronize(stream);
    cudaStreamDestroy(stream);
  }
}

}  // namespace
}  // namespace pj

extern "C" {

void pj_server_options_init(pj_server_options* o) {
  if (!o) return;
  memset(o, 0, sizeof(*o));
  o->slots = 3;
  o->max_batch_queries = 1u << 16;
  o->max_batch_bytes = 16ull << 20;
  o->bytes_per_query = 64ull << 10;
  o->device_reserve = 2ull << 30;
}

int pj_server_start(pj_index* idx, const pj_server_options* opt, pj_server** out) {
  if (out) *out = nullptr;
  pj_server* S = nullptr;
  try {
    if (!idx || !out) pj::fail(PJ_EINVAL, "pj_server_start: NULL argument");
    S = new pj_server();
    S->idx = idx;
    pj_server_options_init(&S->opt);
    if (opt) S->opt = *opt;
    if (S->opt.slots < 1 || S->opt.slots > 16) pj::fail(PJ_EINVAL, "pj_server_start: slots outside 1..16");
    {
      std::lock_guard<std::mutex> g(idx->mu);  // every threshold built before the slots read the index
      for (int t = 0; t < (int)idx->parts.size(); ++t) pj::ensure_partition(*idx, t, nullptr);
      idx->ctx.sync();
    }
    if (S->opt.use_plans) {
      pj_plan_options po;
      pj_plan_options_init(&po);
      po.max_queries = S->opt.max_batch_queries;
      po.max_bytes = S->opt.max_batch_bytes;
      for (int k = 0; k < S->opt.slots; ++k) {
        pj_plan* p = nullptr;
        const int code = pj_plan_create(idx, &po, &p);
        if (code != PJ_OK) pj::fail(code, std::string("pj_server_start: ") + pj_last_error());
        S->plans.push_back(p);
      }
    }
    for (int k = 0; k < S->opt.slots; ++k) S->slots.emplace_back(pj::slot_main, S, k);
    *out = S;
    return PJ_OK;
  } catch (const pj::Error& e) {
    pj::set_last_error(e.msg);
    if (S)
      for (pj_plan* p : S->plans) pj_plan_free(p);
    delete S;
    return e.code;
  }
}

int pj_server_submit(pj_server* S, const pj_strings* batch, int tau, uint64_t* ticket) {
  try {
    if (!S || !batch || !ticket) pj::fail(PJ_EINVAL, "pj_server_submit: NULL argument");
    if (batch->on_device) pj::fail(PJ_EINVAL, "pj_server_submit: the batch must be in host memory");
    if (tau < 0 || tau >= (int)S->idx->parts.size()) pj::fail(PJ_EINVAL, "pj_server_submit: tau outside 0..tau_max");
    if (!batch->offsets || (!batch->bytes && batch->n)) pj::fail(PJ_EINVAL, "pj_server_submit: NULL strings");
    auto r = std::make_shared<pj::Request>();
    r->tau = tau;
    r->n = batch->n;
    const uint64_t o0 = batch->offsets[0];
    r->off.resize((size_t)batch->n + 1);
    for (uint32_t q = 0; q <= batch->n; ++q) {
      if (q && batch->offsets[q] < batch->offsets[q - 1]) pj::fail(PJ_EINVAL, "pj_server_submit: offsets decrease");
      r->off[q] = batch->offsets[q] - o0;
    }
    r->bytes.assign(batch->bytes ? batch->bytes + o0 : nullptr, batch->bytes ? batch->bytes + batch->offsets[batch->n] : nullptr);
    r->t_submit = pj::Clock::now();
    std::lock_guard<std::mutex> g(S->mu);
    if (S->stopping) pj::fail(PJ_ECANCELED, "pj_server_submit: server stopping");
    r->ticket = S->next_ticket++;
    S->all[r->ticket] = r;
    S->pending.push_back(r);
    S->n_requests++;
    *ticket = r->ticket;
    S->cv_work.notify_one();
    return PJ_OK;
  } catch (const pj::Error& e) {
    pj::set_last_error(e.msg);
    return e.code;
  } catch (const std::bad_alloc&) {
    pj::set_last_error("host allocation failed");
    return PJ_ENOMEM;
  }
}

int pj_server_wait(pj_server* S, uint64_t ticket, int timeout_ms, pj_result* out, pj_request_times* times) {
  if (out) memset(out, 0, sizeof(*out));
  try {
    if (!S || !out) pj::fail(PJ_EINVAL, "pj_server_wait: NULL argument");
    std::unique_lock<std::mutex> lk(S->mu);
    auto it = S->all.find(ticket);
    if (it == S->all.end()) pj::fail(PJ_EINVAL, "pj_server_wait: unknown ticket");
    std::shared_ptr<pj::Request> r = it->second;
    auto done = [&] { return r->state == pj::Request::DONE || r->state == pj::Request::FAILED ||
                             r->state == pj::Request::CANCELLED; };
    if (timeout_ms < 0) S->cv_done.wait(lk, done);
    else if (!S->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), done)) {
      pj::set_last_error("pj_server_wait: request not finished within the timeout");
      return PJ_ETIMEDOUT;
    }
    S->all.erase(ticket);
    if (times) {
      times->queue_ms = std::chrono::duration<float, std::milli>(r->t_start - r->t_submit).count();
      times->service_ms = std::chrono::duration<float, std::milli>(r->t_done - r->t_start).count();
      times->batch_requests = r->batch_requests;
    }
    if (r->state == pj::Request::CANCELLED) {
      pj::set_last_error("pj_server_wait: request was cancelled");
      return PJ_ECANCELED;
    }
    if (r->state == pj::Request::FAILED) {
      pj::set_last_error(r->msg);
      return r->code;
    }
    out->count = r->pairs.size();
    out->pairs = static_cast<pj_pair*>(malloc(std::max<size_t>(1, r->pairs.size()) * sizeof(pj_pair)));
    if (!out->pairs) pj::fail(PJ_ENOMEM, "pj_server_wait: host allocation failed");
    if (!r->pairs.empty()) memcpy(out->pairs, r->pairs.data(), r->pairs.size() * sizeof(pj_pair));
    out->stats = r->stats;
    out->on_device = 0;
    return PJ_OK;
  } catch (const pj::Error& e) {
    pj::set_last_error(e.msg);
    return e.code;
  }
}

int pj_server_cancel(pj_server* S, uint64_t ticket) {
  if (!S) return PJ_EINVAL;
  std::lock_guard<std::mutex> g(S->mu);
  auto it = S->all.find(ticket);
  if (it == S->all.end()) return PJ_EINVAL;
  pj::Request& r = *it->second;
  if (r.state == pj::Request::PENDING) {
    for (auto q = S->pending.begin(); q != S->pending.end(); ++q)
      if ((*q)->ticket == ticket) {
        S->pending.erase(q);
        break;
      }
    r.t_start = r.t_done = pj::Clock::now();
  }
  if (r.state == pj::Request::PENDING || r.state == pj::Request::RUNNING) r.state = pj::Request::CANCELLED;
  S->cv_done.notify_all();
  return PJ_OK;
}

int pj_server_stats(pj_server* S, pj_server_counters* out) {
  if (!S || !out) return PJ_EINVAL;
  std::lock_guard<std::mutex> g(S->mu);
  out->requests = S->n_requests;
  out->batches = S->n_batches;
  out->queries = S->n_queries;
  out->max_batch_requests = S->max_batch_requests;
  out->max_in_flight = S->max_in_flight;
  out->pending = S->pending.size();
  return PJ_OK;
}

void pj_server_stop(pj_server* S) {
  if (!S) return;
  {
    std::lock_guard<std::mutex> g(S->mu);
    S->stopping = true;
  }
  S->cv_work.notify_all();
  for (auto& t : S->slots) t.join();
  for (pj_plan* p : S->plans) pj_plan_free(p);
  {
    std::lock_guard<std::mutex> g(S->mu);
    for (auto& kv : S->all)
      if (kv.second->state == pj::Request::PENDING) kv.second->state = pj::Request::CANCELLED;
  }
  S->cv_done.notify_all();
  delete S;
}

}  // extern "C"
