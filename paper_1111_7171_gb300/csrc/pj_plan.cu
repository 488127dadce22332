// Query plans: the multi-threshold query pipeline (the R != S join of
// Sec. 3.2 with per-query thresholds) recorded once into a CUDA graph and
// replayed for every batch.
//
// A plan preallocates every buffer for its capacities, records
// record_query_plan into a graph on its own stream (temporaries of the scan
// and sort primitives come from an arena that lives as long as the graph)
// and, per batch, issues the batch's host-to-device copies, one graph launch
// and one stream synchronisation.  The graph writes the pairs and a header of
// counts into mapped pinned host memory.  When the header shows that a
// capacity was too small, the buffer grows, the graph is recorded again and
// the batch runs again, so results never depend on the capacities.
#include <algorithm>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "pj_plan.cuh"

namespace pj {

}  // namespace pj

struct pj_plan {
  pj_index* idx = nullptr;
  int device = 0;
  std::mutex mu;
  cudaStream_t stream = nullptr;
  pj::Ctx ctx;  // the index's allocator, on the plan's stream
  pj::PlanDev d{};
  uint64_t cap_bytes = 0;
  // device buffers
  pj::DBuf<uint8_t> bytes, tau;
  pj::DBuf<uint64_t> off;
  pj::DBuf<pj::PlanSizes> sizes;
  pj::DBuf<uint32_t> len, gcounts, goff, flags, pos, acc_ed0, acc_ed1;
  pj::DBuf<unsigned long long> gcnt, qgoff, gmask, hcnt, hoff, acc_key0, acc_key1;
  pj::DBuf<pj::Sig> bm;
  pj::DBuf<pj::PartView> parts;
  pj::DBuf<unsigned char> counters, arena;
  pj::DBuf<pj::Hit> hits;
  // pinned host buffers
  pj::HostBuf h_bytes, h_off, h_tau, h_n, h_pairs, h_header;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  uint32_t nodes = 0, kernels = 0;
  uint64_t runs = 0, captures = 0;

  uint64_t device_bytes() const {
    return bytes.bytes() + tau.bytes() + off.bytes() + sizes.bytes() + len.bytes() + gcounts.bytes() + goff.bytes() +
           flags.bytes() + pos.bytes() + acc_ed0.bytes() + acc_ed1.bytes() + gcnt.bytes() + qgoff.bytes() +
           gmask.bytes() + bm.bytes() + hcnt.bytes() + hoff.bytes() + acc_key0.bytes() + acc_key1.bytes() + parts.bytes() + counters.bytes() +
           arena.bytes() + hits.bytes();
  }
  uint64_t host_bytes() const {
    return h_bytes.bytes + h_off.bytes + h_tau.bytes + h_n.bytes + h_pairs.bytes + h_header.bytes;
  }
  void drop_graph() {
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
    exec = nullptr;
    graph = nullptr;
  }
  void release_all() {
    if (stream) cudaStreamSynchronize(stream);  // nothing of the plan in flight
    drop_graph();
    pj::DBuf<uint8_t>* b8[] = {&bytes, &tau};
    for (auto* b : b8) b->release();
    off.release();
    sizes.release();
    pj::DBuf<uint32_t>* b32[] = {&len, &gcounts, &goff, &flags, &pos, &acc_ed0, &acc_ed1};
    for (auto* b : b32) b->release();
    pj::DBuf<unsigned long long>* b64[] = {&gcnt, &qgoff, &gmask, &hcnt, &hoff, &acc_key0, &acc_key1};
    for (auto* b : b64) b->release();
    bm.release();
    parts.release();
    counters.release();
    arena.release();
    hits.release();
    if (stream) cudaStreamSynchronize(stream);
    h_bytes.release();
    h_off.release();
    h_tau.release();
    h_n.release();
    h_pairs.release();
    h_header.release();
  }
};

namespace pj {
namespace {

constexpr unsigned long long MAX_CAP_ACC = 0xFFFFFFFFull;  // radix sort and u32 positions

// (Re)allocates the capacity-dependent buffers for d's capacities.
void alloc_hits(pj_plan& P) {
  P.hits.reset(P.ctx, P.d.cap_hits);
  P.hcnt.reset(P.ctx, P.d.cap_hits);
  P.hoff.reset(P.ctx, P.d.cap_hits);
  P.d.hits = P.hits.p;
  P.d.hcnt = P.hcnt.p;
  P.d.hoff = P.hoff.p;
}

void alloc_acc(pj_plan& P) {
  P.acc_key0.reset(P.ctx, P.d.cap_acc);
  P.acc_key1.reset(P.ctx, P.d.cap_acc);
  P.acc_ed0.reset(P.ctx, P.d.cap_acc);
  P.acc_ed1.reset(P.ctx, P.d.cap_acc);
  P.flags.reset(P.ctx, P.d.cap_acc);
  P.pos.reset(P.ctx, P.d.cap_acc);
  P.d.acc_key[0] = P.acc_key0.p;
  P.d.acc_key[1] = P.acc_key1.p;
  P.d.acc_ed[0] = P.acc_ed0.p;
  P.d.acc_ed[1] = P.acc_ed1.p;
  P.d.flags = P.flags.p;
  P.d.pos = P.pos.p;
}

void alloc_pairs(pj_plan& P) {
  P.h_pairs.reset(P.d.cap_pairs * sizeof(pj_pair), true);
  P.d.out_pairs = static_cast<pj_pair*>(P.h_pairs.dev);
}

// Records the pipeline into a fresh graph and instantiates it.
void capture(pj_plan& P) {
  P.drop_graph();
  size_t arena_bytes = scan_temp_bytes(P.d.cap_q, 8) + scan_temp_bytes(P.d.cap_groups, 4) +
                       scan_temp_bytes(P.d.cap_hits, 8) + scan_temp_bytes(P.d.cap_acc, 4) +
                       sort_temp_bytes(P.d.cap_acc) + (1u << 16);
  for (int attempt = 0;; ++attempt) {
    P.arena.reset(P.ctx, arena_bytes);
    P.ctx.sync();
    Arena ar;
    ar.base = P.arena.p;
    ar.cap = arena_bytes;
    Ctx rc;
    rc.stream = P.stream;
    rc.alloc = arena_alloc;
    rc.free_fn = arena_free;
    rc.alloc_ctx = &ar;
    cudaGraph_t g = nullptr;
    PJ_CUDA(cudaStreamBeginCapture(P.stream, cudaStreamCaptureModeRelaxed));
    set_recording(true);
    bool ok = true;
    Error err{PJ_OK, ""};
    try {
      record_query_plan(rc, *P.idx, P.d);
    } catch (const Error& e) {
      ok = false;
      err = e;
    }
    set_recording(false);
    const cudaError_t ce = cudaStreamEndCapture(P.stream, &g);
    if (!ok || ce != cudaSuccess || !g) {
      if (g) cudaGraphDestroy(g);
      cudaGetLastError();
      if (!ok && ar.exhausted && attempt < 4) {  // the estimate was short: retry with more
        arena_bytes *= 2;
        continue;
      }
      if (!ok) throw err;
      fail(PJ_ECUDA, std::string("query plan: graph capture failed: ") + cudaGetErrorString(ce));
    }
    P.graph = g;
    const cudaError_t ie = cudaGraphInstantiate(&P.exec, g, 0);
    if (ie != cudaSuccess) {
      cudaGetLastError();
      P.exec = nullptr;
      P.drop_graph();
      fail(PJ_ECUDA, std::string("query plan: cudaGraphInstantiate failed: ") + cudaGetErrorString(ie));
    }
    size_t n = 0;
    PJ_CUDA(cudaGraphGetNodes(g, nullptr, &n));
    std::vector<cudaGraphNode_t> nodes(n);
    PJ_CUDA(cudaGraphGetNodes(g, nodes.data(), &n));
    uint32_t kernels = 0;
    for (size_t k = 0; k < n; ++k) {
      cudaGraphNodeType t;
      PJ_CUDA(cudaGraphNodeGetType(nodes[k], &t));
      if (t == cudaGraphNodeTypeKernel) ++kernels;
    }
    P.nodes = (uint32_t)n;
    P.kernels = kernels;
    ++P.captures;
    return;
  }
}

uint64_t grown(uint64_t cap, uint64_t need, uint64_t limit, const char* what) {
  if (need > limit)
    fail(PJ_ENOMEM, std::string("query plan: the batch needs ") + std::to_string(need) + " " + what +
                        ", more than a plan can hold (" + std::to_string(limit) + "); split the batch");
  return std::min<uint64_t>(limit, 2 * std::max<uint64_t>(cap, need));
}

void create(pj_plan& P, pj_index& idx, const pj_plan_options& o) {
  const int tau_max = (int)idx.parts.size() - 1;
  if (o.max_queries == 0 || o.max_queries > (1u << 24)) fail(PJ_EINVAL, "query plan: max_queries outside 1..2^24");
  if (o.max_bytes == 0 || o.max_bytes > (1ull << 40)) fail(PJ_EINVAL, "query plan: max_bytes outside 1..2^40");
  const uint64_t cap_groups = (uint64_t)o.max_queries * groups_per_probe(tau_max, false);
  // group hit offsets are 32-bit: every group looks up at most tau_max + 1 substrings
  if (cap_groups * (uint64_t)(tau_max + 1) > 0xFFFFFFFFull)
    fail(PJ_EINVAL, "query plan: max_queries too large for tau_max " + std::to_string(tau_max));
  P.idx = &idx;
  P.device = idx.device;
  int dev = 0;
  PJ_CUDA(cudaGetDevice(&dev));
  if (dev != idx.device) fail(PJ_EINVAL, "query plan: the index lives on another device");
  for (int t = 0; t <= tau_max; ++t) ensure_partition(idx, t, nullptr);
  idx.ctx.sync();
  PJ_CUDA(cudaStreamCreateWithFlags(&P.stream, cudaStreamNonBlocking));
  P.ctx = idx.ctx;
  P.ctx.stream = P.stream;
  P.cap_bytes = o.max_bytes;
  PlanDev& d = P.d;
  d.cap_q = o.max_queries;
  d.cap_groups = cap_groups;
  // defaults: about two hits per group and 128 accepted matches per query
  // (the short-string workload at tau = 4 averages 1.7 and 217 at full
  // self-join scale); capacities grow when a batch needs more
  d.cap_hits = o.hits_capacity ? o.hits_capacity : std::max<uint64_t>(1u << 16, 2 * cap_groups);
  d.cap_hits = std::min<uint64_t>(d.cap_hits, cap_groups * (uint64_t)(tau_max + 1));
  d.cap_acc = o.accepted_capacity ? o.accepted_capacity
                                  : std::min<uint64_t>(1ull << 27, std::max<uint64_t>(1u << 16, 128ull * o.max_queries));
  d.cap_acc = std::min(d.cap_acc, MAX_CAP_ACC);
  d.cap_pairs = o.pairs_capacity ? o.pairs_capacity : std::max<uint64_t>(1u << 16, d.cap_acc / 2);
  d.cap_pairs = std::min(d.cap_pairs, MAX_CAP_ACC);

  P.bytes.reset(P.ctx, o.max_bytes + 16);
  P.off.reset(P.ctx, (size_t)d.cap_q + 1);
  P.tau.reset(P.ctx, d.cap_q);
  P.sizes.reset(P.ctx, 1);
  P.len.reset(P.ctx, d.cap_q);
  P.bm.reset(P.ctx, d.cap_q);
  P.gcnt.reset(P.ctx, d.cap_q);
  P.qgoff.reset(P.ctx, d.cap_q);
  P.gcounts.reset(P.ctx, d.cap_groups);
  P.goff.reset(P.ctx, d.cap_groups);
  P.gmask.reset(P.ctx, d.cap_groups);
  P.counters.reset(P.ctx, 64);
  d.bytes = P.bytes.p;
  d.off = P.off.p;
  d.tau = P.tau.p;
  d.sizes = P.sizes.p;
  d.len = P.len.p;
  d.bm = P.bm.p;
  d.gcnt = P.gcnt.p;
  d.qgoff = P.qgoff.p;
  d.gcounts = P.gcounts.p;
  d.goff = P.goff.p;
  d.gmask = P.gmask.p;
  d.counters = P.counters.p;
  std::vector<PartView> hp((size_t)tau_max + 1);
  for (int t = 0; t <= tau_max; ++t) {
    const Partition& part = idx.parts[t];
    hp[t] = PartView{part.table.p, part.fp.p, part.presence_bytes, part.precs.p, part.table.n - 1,
                     part.postings.p, part.n_records, part.first, t, seg_magic(t + 1), part.scheme};
  }
  P.parts.reset(P.ctx, hp.size());
  PJ_CUDA(cudaMemcpyAsync(P.parts.p, hp.data(), hp.size() * sizeof(PartView), cudaMemcpyHostToDevice, P.stream));
  PJ_CUDA(cudaMemsetAsync(P.sizes.p, 0, sizeof(PlanSizes), P.stream));
  d.parts = P.parts.p;
  alloc_hits(P);
  alloc_acc(P);
  P.h_bytes.reset(o.max_bytes + 16, false);
  P.h_off.reset(((size_t)d.cap_q + 1) * sizeof(uint64_t), false);
  P.h_tau.reset(d.cap_q, false);
  P.h_n.reset(sizeof(unsigned long long), false);
  P.h_header.reset(sizeof(PlanHeader), true);
  d.header = static_cast<PlanHeader*>(P.h_header.dev);
  alloc_pairs(P);
  P.ctx.sync();  // hp lives on this stack frame
  capture(P);
}

void plan_query(pj_plan& P, const pj_strings& b, const uint8_t* taus, pj_result* out) {
  if (b.on_device) fail(PJ_EINVAL, "pj_plan_query: the batch must be in host memory");
  if (b.n > P.d.cap_q)
    fail(PJ_EINVAL, "pj_plan_query: " + std::to_string(b.n) + " strings exceed the plan's max_queries " +
                        std::to_string(P.d.cap_q));
  if (b.n && (!b.bytes || !b.offsets || !taus)) fail(PJ_EINVAL, "pj_plan_query: NULL strings or thresholds");
  const int tau_max = (int)P.idx->parts.size() - 1;
  const uint32_t n = b.n;
  out->on_device = 0;
  out->priv = nullptr;
  if (n == 0) {
    out->pairs = static_cast<pj_pair*>(malloc(sizeof(pj_pair)));
    if (!out->pairs) fail(PJ_ENOMEM, "host result allocation failed");
    out->count = 0;
    return;
  }
  // validate and stage the batch (offsets rebased to 0)
  const uint64_t base = b.offsets[0];
  uint64_t* hoff = static_cast<uint64_t*>(P.h_off.p);
  for (uint32_t q = 0; q < n; ++q) {
    if (b.offsets[q + 1] < b.offsets[q] || b.offsets[q + 1] - b.offsets[q] > 65535)
      fail(PJ_EINVAL, "pj_strings: offsets decrease or a string is longer than 65535 bytes");
    if ((int)taus[q] > tau_max) fail(PJ_EINVAL, "pj_plan_query: tau outside 0..tau_max");
    hoff[q] = b.offsets[q] - base;
  }
  const uint64_t total = b.offsets[n] - base;
  hoff[n] = total;
  if (total > P.cap_bytes)
    fail(PJ_EINVAL, "pj_plan_query: " + std::to_string(total) + " bytes exceed the plan's max_bytes " +
                        std::to_string(P.cap_bytes));
  memcpy(P.h_tau.p, taus, n);
  if (total) memcpy(P.h_bytes.p, b.bytes + base, total);
  *static_cast<unsigned long long*>(P.h_n.p) = n;
  PJ_CUDA(cudaMemcpyAsync(P.off.p, P.h_off.p, ((size_t)n + 1) * sizeof(uint64_t), cudaMemcpyHostToDevice, P.stream));
  PJ_CUDA(cudaMemcpyAsync(P.tau.p, P.h_tau.p, n, cudaMemcpyHostToDevice, P.stream));
  if (total) PJ_CUDA(cudaMemcpyAsync(P.bytes.p, P.h_bytes.p, total, cudaMemcpyHostToDevice, P.stream));
  PJ_CUDA(cudaMemcpyAsync(&P.sizes.p->n, P.h_n.p, sizeof(unsigned long long), cudaMemcpyHostToDevice, P.stream));

  PlanHeader h{};
  for (int attempt = 0;; ++attempt) {
    PJ_CUDA(cudaGraphLaunch(P.exec, P.stream));
    count_launches(P.kernels);
    P.ctx.sync();
    ++P.runs;
    memcpy(&h, P.h_header.p, sizeof(h));
    if (h.err)
      fail(PJ_ECUDA, std::string("segment index consistency check failed (") +
                         ((h.err & 1) ? "posting outside the index" : "probe limit reached") + ")");
    const bool short_of_room = h.hits > P.d.cap_hits || h.accepted > P.d.cap_acc || h.pairs > P.d.cap_pairs;
    if (short_of_room && attempt >= 8) fail(PJ_ECUDA, "query plan: capacities still too small after growing");
    if (h.hits > P.d.cap_hits) {
      P.d.cap_hits = grown(P.d.cap_hits, h.hits, P.d.cap_groups * (uint64_t)(tau_max + 1), "hits");
      alloc_hits(P);
    } else if (h.accepted > P.d.cap_acc) {
      P.d.cap_acc = grown(P.d.cap_acc, h.accepted, MAX_CAP_ACC, "accepted matches");
      alloc_acc(P);
    } else if (h.pairs > P.d.cap_pairs) {
      P.d.cap_pairs = grown(P.d.cap_pairs, h.pairs, MAX_CAP_ACC, "pairs");
      alloc_pairs(P);
    } else {
      break;
    }
    capture(P);
  }
  out->count = h.pairs;
  out->pairs = static_cast<pj_pair*>(malloc(std::max<uint64_t>(h.pairs, 1) * sizeof(pj_pair)));
  if (!out->pairs) fail(PJ_ENOMEM, "host result allocation failed");
  if (h.pairs) memcpy(out->pairs, P.h_pairs.p, h.pairs * sizeof(pj_pair));
  out->stats.lookups = h.lookups;
  out->stats.candidates = h.cands;
  out->stats.accepted = h.accepted;
  out->stats.dp_cells = h.cells;
  out->stats.fallback_pairs = h.fallback;
  out->stats.hits = h.hits;
}

}  // namespace
}  // namespace pj

extern "C" {

void pj_plan_options_init(pj_plan_options* o) {
  if (!o) return;
  memset(o, 0, sizeof(*o));
  o->max_queries = 4096;
  o->max_bytes = 1ull << 20;
}

int pj_plan_create(pj_index* idx, const pj_plan_options* opt, pj_plan** out) {
  if (out) *out = nullptr;
  pj_plan* P = nullptr;
  try {
    if (!idx || !out) pj::fail(PJ_EINVAL, "pj_plan_create: NULL argument");
    pj_plan_options o;
    pj_plan_options_init(&o);
    if (opt) o = *opt;
    P = new pj_plan();
    {
      std::lock_guard<std::mutex> g(idx->mu);
      pj::create(*P, *idx, o);
    }
    *out = P;
    return PJ_OK;
  } catch (const pj::Error& e) {
    pj::set_last_error(e.msg);
    if (P) {
      P->release_all();
      if (P->stream) cudaStreamDestroy(P->stream);
      delete P;
    }
    return e.code;
  } catch (const std::bad_alloc&) {
    pj::set_last_error("host allocation failed");
    if (P) {
      P->release_all();
      if (P->stream) cudaStreamDestroy(P->stream);
      delete P;
    }
    return PJ_ENOMEM;
  }
}

int pj_plan_query(pj_plan* plan, const pj_strings* batch, const uint8_t* taus, pj_result* out) {
  if (out) memset(out, 0, sizeof(*out));
  try {
    if (!plan || !batch || !out) pj::fail(PJ_EINVAL, "pj_plan_query: NULL argument");
    std::lock_guard<std::mutex> g(plan->mu);
    PJ_CUDA(cudaSetDevice(plan->device));
    pj::plan_query(*plan, *batch, taus, out);
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

int pj_plan_get_info(const pj_plan* plan, pj_plan_info* out) {
  if (!plan || !out) {
    pj::set_last_error("pj_plan_get_info: NULL argument");
    return PJ_EINVAL;
  }
  pj_plan* P = const_cast<pj_plan*>(plan);
  std::lock_guard<std::mutex> g(P->mu);
  memset(out, 0, sizeof(*out));
  out->runs = P->runs;
  out->recaptures = P->captures ? P->captures - 1 : 0;
  out->graph_nodes = P->nodes;
  out->graph_kernels = P->kernels;
  out->hits_capacity = P->d.cap_hits;
  out->accepted_capacity = P->d.cap_acc;
  out->pairs_capacity = P->d.cap_pairs;
  out->device_bytes = P->device_bytes();
  out->host_bytes = P->host_bytes();
  return PJ_OK;
}

void pj_plan_free(pj_plan* plan) {
  if (!plan) return;
  {
    std::lock_guard<std::mutex> g(plan->mu);
    cudaSetDevice(plan->device);
    plan->release_all();
    if (plan->stream) cudaStreamDestroy(plan->stream);
    plan->stream = nullptr;
  }
  delete plan;
}

}  // extern "C"
