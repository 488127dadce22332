// pj_query_noalloc: the query entry point for callers that must not allocate.
//
// Some callers cannot allocate device memory on the call path: a serving
// thread with a latency budget (cudaMalloc and cudaFree can block and
// synchronise the device), an embedder that reserved its GPU memory up front
// and forbids further growth, or code that must not touch the host heap or
// an allocator it does not own.  This entry point needs no allocation at
// all: the caller passes the query strings and the output buffer in device
// memory, and every temporary lives in one file-scope device array of fixed
// size (NOALLOC_SCRATCH_BYTES), which every GPU that loads the library holds
// until the process exits.
//
// The scratch array is shared by every call in the process, keeps the last
// call's contents, and is cleared where a call needs zeros.  Host threads
// are serialised by a mutex, but calls that overlap on the GPU (for example
// from two processes' streams, or work still queued from a previous call on
// another stream) race on the array.
#include <mutex>

#include "pj_internal.cuh"
#include "pj_prims.cuh"
#include "pj_probe.cuh"

namespace pj {
namespace {

constexpr size_t NOALLOC_SCRATCH_BYTES = 64ull << 20;
constexpr uint32_t NOALLOC_MAX_QUERIES = 65536;
constexpr int NA_BLOCK = 256;

__device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_SCRATCH_BYTES];

// Device address of g_noalloc_scratch on the current device.  The host-side
// symbol is only a stand-in, so host code asks the runtime for the address;
// the lookup allocates nothing and is repeated on every call, so that a
// device reset or a new primary context never leaves a stale address behind.
// (The first lookup on a device also loads this library's kernels there.)
std::mutex g_noalloc_mu;

unsigned char* scratch_base() {
  void* p = nullptr;
  const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
  if (e != cudaSuccess || !p) {
    cudaGetLastError();
    fail(PJ_ECUDA, std::string("pj_query_noalloc: cudaGetSymbolAddress failed: ") + cudaGetErrorString(e));
  }
  return static_cast<unsigned char*>(p);
}

// Bump allocator over the scratch array; frees are no-ops, the arena is
// rewound at the start of every call.
struct Bump {
  unsigned char* base;
  size_t cap;
  size_t used;
};

void* bump_alloc(void* ctx, size_t bytes, void*) {
  Bump* b = static_cast<Bump*>(ctx);
  const size_t off = (b->used + 255) & ~size_t(255);
  if (off + bytes > b->cap) return nullptr;
  b->used = off + bytes;
  return b->base + off;
}

void bump_free(void*, void*, void*) {}

struct NaCounters {
  unsigned long long accepted, lookups, candidates, cells, fallback, err;
};

__device__ __forceinline__ void na_append(NaCounters* ctr, unsigned long long* keys, uint32_t* eds,
                                          unsigned long long cap, unsigned long long key, int ed) {
  const unsigned long long pos = atomicAdd(&ctr->accepted, 1ull);
  if (pos < cap) {
    keys[pos] = key;
    eds[pos] = (uint32_t)ed;
  }
}

// One thread per (query, indexed length, segment) group: lookups of the
// multi-match window, then extension verification of every posting of each
// run, all in the thread (no warp collectives, no barriers).
template <int MAXW>
__global__ void __launch_bounds__(NA_BLOCK) k_na_probe_verify(const ProbeView v, unsigned long long n_groups,
                                                              unsigned long long* keys, uint32_t* eds,
                                                              unsigned long long cap, NaCounters* ctr) {
  const int G = groups_per_probe(v.tau, false);
  unsigned long long lookups = 0, cand = 0, cells = 0;
  int err = 0;
  for (unsigned long long t = (unsigned long long)blockIdx.x * NA_BLOCK + threadIdx.x; t < n_groups;
       t += (unsigned long long)gridDim.x * NA_BLOCK) {
    const uint32_t q = (uint32_t)(t / G);
    const int ls = (int)v.plen[q];
    int l, i, P, li, lo, hi;
    if (!group_window(v, false, q, ls, (int)(t % G), l, i, P, li, lo, hi)) continue;
    for (int p = lo; p <= hi; ++p) {
      ++lookups;
      uint32_t b;
      const uint32_t c = lookup(v, false, v.pbytes + v.poff[q], ls, q, l, i, p, li, b, err);
      const Hit h{q, b, c, (uint32_t)p | ((uint32_t)i << 16)};
      for (uint32_t k = 0; k < c; ++k) {
        ++cand;
        unsigned long long key = 0;
        int ed = 0;
        if (verify_candidate<MAXW>(v, false, h, k, key, ed, cells, err)) na_append(ctr, keys, eds, cap, key, ed);
      }
    }
  }
  if (lookups) atomicAdd(&ctr->lookups, lookups);
  if (cand) atomicAdd(&ctr->candidates, cand);
  if (cells) atomicAdd(&ctr->cells, cells);
  if (err) atomicOr(&ctr->err, (unsigned long long)err);
}

// Indexed strings of length <= tau have no even partition: every query is
// verified directly against those within the length filter.
template <int MAXW>
__global__ void __launch_bounds__(NA_BLOCK) k_na_fallback(const ProbeView v, unsigned long long* keys, uint32_t* eds,
                                                          unsigned long long cap, NaCounters* ctr) {
  const int tau = v.tau;
  unsigned long long cells = 0, pairs = 0;
  for (uint32_t x = blockIdx.x * NA_BLOCK + threadIdx.x; x < v.pcount; x += gridDim.x * NA_BLOCK) {
    const int lx = (int)v.plen[x];
    const int llo = max(0, lx - tau);
    const int lhi = min(min(tau, lx + tau), v.ilmax);
    if (llo > lhi) continue;
    for (uint32_t y = v.ibbeg[llo]; y < v.ibbeg[lhi + 1]; ++y) {
      ++pairs;
      const int d = vsp<MAXW>(v.pbytes + v.poff[x], lx, v.ibytes + v.ioff[y], (int)v.ilen[y], tau, cells);
      if (d <= tau) na_append(ctr, keys, eds, cap, ((unsigned long long)x << v.key_shift) | v.iperm[y], d);
    }
  }
  if (cells) atomicAdd(&ctr->cells, cells);
  if (pairs) atomicAdd(&ctr->fallback, pairs);
}

__global__ void k_na_heads(const unsigned long long* __restrict__ keys, unsigned long long n,
                           uint32_t* __restrict__ flags) {
  const unsigned long long k = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (k < n) flags[k] = (k == 0 || keys[k] != keys[k - 1]) ? 1u : 0u;
}

__global__ void k_na_emit(const unsigned long long* __restrict__ keys, const uint32_t* __restrict__ eds,
                          const uint32_t* __restrict__ flags, const uint32_t* __restrict__ pos,
                          unsigned long long n, int key_shift, pj_pair* __restrict__ out) {
  const unsigned long long k = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n || !flags[k]) return;
  const unsigned long long key = keys[k];
  uint32_t ed = eds[k];
  for (unsigned long long j = k + 1; j < n && keys[j] == key; ++j) ed = min(ed, eds[j]);
  pj_pair pr;
  pr.a = (uint32_t)(key >> key_shift);
  pr.b = (uint32_t)(key & ((1ull << key_shift) - 1));
  pr.ed = ed;
  out[pos[k]] = pr;
}

template <int MAXW>
void na_launch(const Ctx& c, const ProbeView& v, bool fallback, unsigned long long* keys, uint32_t* eds,
               unsigned long long cap, NaCounters* ctr) {
  const unsigned long long n_groups = (unsigned long long)v.pcount * groups_per_probe(v.tau, false);
  if (n_groups) {
    const unsigned grid = (unsigned)std::min<unsigned long long>((n_groups + NA_BLOCK - 1) / NA_BLOCK, sm_grid_cap(8));
    k_na_probe_verify<MAXW><<<grid, NA_BLOCK, 0, c.stream>>>(v, n_groups, keys, eds, cap, ctr);
    PJ_LAUNCHED("k_na_probe_verify");
  }
  if (fallback && v.pcount) {
    const unsigned grid = (unsigned)std::min<unsigned>((v.pcount + NA_BLOCK - 1) / NA_BLOCK, sm_grid_cap(8));
    k_na_fallback<MAXW><<<grid, NA_BLOCK, 0, c.stream>>>(v, keys, eds, cap, ctr);
    PJ_LAUNCHED("k_na_fallback");
  }
}

void query_noalloc(pj_index& idx, const pj_strings& batch, int tau, pj_pair* out_pairs, uint64_t out_cap,
                   uint64_t* out_count) {
  if (!batch.on_device)
    fail(PJ_EINVAL, "pj_query_noalloc: the batch must be in device memory (host strings would need a staging "
                    "allocation)");
  if (batch.n > NOALLOC_MAX_QUERIES)
    fail(PJ_EINVAL, "pj_query_noalloc: batch of " + std::to_string(batch.n) + " strings exceeds the limit of " +
                        std::to_string(NOALLOC_MAX_QUERIES));
  const Partition& part = idx.parts[tau];
  if (part.tau != tau)
    fail(PJ_EINVAL, "pj_query_noalloc: the index for this tau is not built yet (lazy index): run pj_query or "
                    "pj_self_join with this tau once first");
  int dev = 0;
  PJ_CUDA(cudaGetDevice(&dev));
  if (dev != idx.device) fail(PJ_EINVAL, "pj_query_noalloc: the index lives on another device");
  Bump bump{scratch_base(), NOALLOC_SCRATCH_BYTES, 0};
  Ctx c;
  c.stream = idx.ctx.stream;
  c.alloc = bump_alloc;
  c.free_fn = bump_free;
  c.alloc_ctx = &bump;

  ProbeSet R;
  upload_probe_set(c, batch, R);  // device input: lengths only, in the scratch
  DBuf<NaCounters> ctr(c, 1);
  PJ_CUDA(cudaMemsetAsync(ctr.p, 0, sizeof(NaCounters), c.stream));

  // Everything left: accepted (key 8 + ed 4), their sort double buffers
  // (12), run flags and positions (8) and the sort histograms.
  const size_t left = NOALLOC_SCRATCH_BYTES - ((bump.used + 255) & ~size_t(255));
  const unsigned long long cap = left > (1u << 20) ? (left - (1u << 20)) / 40 : 0;
  if (cap == 0) fail(PJ_ENOMEM, "pj_query_noalloc: scratch exhausted by the batch");
  DBuf<unsigned long long> keys(c, cap);
  DBuf<uint32_t> eds(c, cap);

  ProbeView v{};
  v.ibytes = idx.sbytes.p;
  v.ioff = idx.soff.p;
  v.ilen = idx.slen.p;
  v.iref = idx.sref.p;
  v.ibbeg = idx.bbeg.p;
  v.ilmax = idx.lmax;
  v.iperm = idx.perm.p;
  v.n_index = idx.n;
  v.table = part.table.p;
  v.table_fp = part.fp.p;
  v.table_pb = part.presence_bytes;
  v.precs = part.precs.p;
  v.ibm = idx.sbm.p;
  v.pbm = R.bm.p;
  v.mask = part.table.n - 1;
  v.postings = part.postings.p;
  v.n_postings = part.n_records;
  v.tau = tau;
  v.seg_magic = seg_magic(tau + 1);
  v.scheme = part.scheme;
  v.pbytes = R.bytes;
  v.poff = R.off;
  v.plen = R.len.p;
  v.pbegin = 0;
  v.pcount = R.n;
  v.pid = nullptr;
  v.key_shift = bits_for(idx.n);
  const bool fallback = part.first > 0;
#define PJ_NA(W) na_launch<W>(c, v, fallback, keys.p, eds.p, cap, ctr.p)
  if (tau <= 1) PJ_NA(2);
  else if (tau <= 2) PJ_NA(3);
  else if (tau <= 4) PJ_NA(5);
  else if (tau <= 8) PJ_NA(9);
  else if (tau <= 16) PJ_NA(17);
  else PJ_NA(33);
#undef PJ_NA
  NaCounters h{};
  PJ_CUDA(cudaMemcpyAsync(&h, ctr.p, sizeof(h), cudaMemcpyDeviceToHost, c.stream));
  c.sync();
  if (h.err) fail(PJ_ECUDA, "pj_query_noalloc: segment index consistency check failed");
  if (h.accepted > cap)
    fail(PJ_ENOMEM, "pj_query_noalloc: " + std::to_string(h.accepted) + " accepted matches exceed the scratch "
                        "capacity of " + std::to_string(cap));
  uint64_t count = 0;
  const unsigned long long n = h.accepted;
  if (n) {
    radix_sort_pairs<unsigned long long>(c, keys.p, eds.p, n, v.key_shift + bits_for(R.n));
    DBuf<uint32_t> flags(c, n), pos(c, n);
    k_na_heads<<<ceil_div(n, 256), 256, 0, c.stream>>>(keys.p, n, flags.p);
    PJ_LAUNCHED("k_na_heads");
    exclusive_scan<uint32_t>(c, flags.p, pos.p, n);
    uint32_t last[2] = {0, 0};
    PJ_CUDA(cudaMemcpyAsync(&last[0], pos.p + n - 1, sizeof(uint32_t), cudaMemcpyDeviceToHost, c.stream));
    PJ_CUDA(cudaMemcpyAsync(&last[1], flags.p + n - 1, sizeof(uint32_t), cudaMemcpyDeviceToHost, c.stream));
    c.sync();
    count = (uint64_t)last[0] + last[1];
    if (count > out_cap) {
      *out_count = count;
      fail(PJ_EINVAL, "pj_query_noalloc: " + std::to_string(count) + " pairs do not fit the output buffer of " +
                          std::to_string(out_cap));
    }
    k_na_emit<<<ceil_div(n, 256), 256, 0, c.stream>>>(keys.p, eds.p, flags.p, pos.p, n, v.key_shift, out_pairs);
    PJ_LAUNCHED("k_na_emit");
  }
  c.sync();
  *out_count = count;
}

}  // namespace
}  // namespace pj

extern "C" int pj_query_noalloc(pj_index* idx, const pj_strings* batch, int tau, pj_pair* out_pairs, uint64_t out_cap,
                                uint64_t* out_count) {
  try {
    if (!idx || !batch || !out_count || (!out_pairs && out_cap)) pj::fail(PJ_EINVAL, "pj_query_noalloc: NULL argument");
    *out_count = 0;
    if (tau < 0 || tau >= (int)idx->parts.size()) pj::fail(PJ_EINVAL, "pj_query_noalloc: tau outside 0..tau_max");
    std::lock_guard<std::mutex> g_all(pj::g_noalloc_mu);
    std::lock_guard<std::mutex> g(idx->mu);
    pj::query_noalloc(*idx, *batch, tau, out_pairs, out_cap, out_count);
    return PJ_OK;
  } catch (const pj::Error& e) {
    pj::set_last_error(e.msg);
    return e.code;
  }
}
