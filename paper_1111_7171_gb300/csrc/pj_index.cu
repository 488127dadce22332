// Packed string store and segment index (the build half of the hot path).
//
//   A1  lengths + validation, the sid order (stable radix sorts by the
//       first eight bytes, then by length: by length, then first eight
//       bytes, then id), offsets by prefix sum, warp-per-string gather of
//       the bytes into sid order, length buckets (Sec. 3.2 groups S_l; the
//       sort by length, then alphabetically, that Alg. 1 starts with).
//   A2  even partition of every string of length >= tau+1 into tau+1
//       segments and one (key, sid) record per segment (Sec. 3.1).
//   A3  records sorted by key -> runs = inverted lists L_l^i(w) (Sec. 3.2),
//       run heads by flag + prefix sum, open-addressing table key -> run.
#include <cstdio>
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

#include "pj_internal.cuh"
#include "pj_prims.cuh"

namespace pj {

// ------------------------------------------------------------ plumbing ----

static thread_local std::string g_last_error;

void set_last_error(const std::string& msg) { g_last_error = msg; }
const std::string& last_error() { return g_last_error; }

void fail(int code, const std::string& msg) { throw Error{code, msg}; }

static std::atomic<unsigned long long> g_launches{0};
static thread_local bool g_recording = false;
void count_launch() {
  if (!g_recording) g_launches.fetch_add(1, std::memory_order_relaxed);
}
int sm_count() {
  constexpr int MAX_DEVICES = 64;
  static std::atomic<int> cached[MAX_DEVICES];  // 0 = not looked up yet
  int dev = 0;
  PJ_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= MAX_DEVICES) {
    int sms = 0;
    PJ_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    return sms;
  }
  int sms = cached[dev].load(std::memory_order_relaxed);
  if (!sms) {
    PJ_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    cached[dev].store(sms, std::memory_order_relaxed);
  }
  return sms;
}

void count_launches(unsigned long long k) { g_launches.fetch_add(k, std::memory_order_relaxed); }
void set_recording(bool on) { g_recording = on; }

void check_cuda(cudaError_t e, const char* what, const char* file, int line) {
  if (e == cudaSuccess) return;
  char buf[512];
  snprintf(buf, sizeof(buf), "%s failed at %s:%d: %s (%s)", what, file, line, cudaGetErrorName(e),
           cudaGetErrorString(e));
  fail(e == cudaErrorMemoryAllocation ? PJ_ENOMEM : PJ_ECUDA, buf);
}

void* Ctx::get(size_t bytes) const {
  void* p = nullptr;
  if (budget) {  // reserve first, so that concurrent callers cannot pass the limit together
    std::lock_guard<std::mutex> g(budget->mu);
    if (budget->cur + bytes > budget->limit)
      fail(PJ_ENOMEM, "device budget of " + std::to_string(budget->limit) + " bytes exceeded: " +
                          std::to_string(budget->cur) + " held, " + std::to_string(bytes) + " more asked");
    budget->cur += bytes;
    budget->peak = std::max(budget->peak, budget->cur);
  }
  struct Unreserve {  // gives the reservation back if the allocation fails
    const Ctx* c;
    size_t n;
    bool keep = false;
    ~Unreserve() {
      if (keep || !c->budget) return;
      std::lock_guard<std::mutex> g(c->budget->mu);
      c->budget->cur -= n;
    }
  } unreserve{this, bytes};
  if (alloc) {
    p = alloc(alloc_ctx, bytes, (void*)stream);
    if (!p) fail(PJ_ENOMEM, "device allocator returned NULL for " + std::to_string(bytes) + " bytes");
  } else {
    cudaError_t e = cudaMallocAsync(&p, bytes, stream);
    if (e != cudaSuccess) {
      cudaGetLastError();
      fail(PJ_ENOMEM, "cudaMallocAsync of " + std::to_string(bytes) + " bytes failed: " + cudaGetErrorString(e));
    }
  }
  if (budget) {
    std::lock_guard<std::mutex> g(budget->mu);
    budget->live[p] = bytes;
  }
  unreserve.keep = true;
  return p;
}

void Ctx::put(void* p) const {
  if (!p) return;
  if (budget) {
    std::lock_guard<std::mutex> g(budget->mu);
    auto it = budget->live.find(p);
    if (it != budget->live.end()) {
      budget->cur -= it->second;
      budget->live.erase(it);
    }
  }
  if (alloc) {
    free_fn(alloc_ctx, p, (void*)stream);
  } else {
    cudaFreeAsync(p, stream);
  }
}

Ctx make_ctx(const pj_options* opt) {
  Ctx c;
  if (opt) {
    c.stream = (cudaStream_t)opt->stream;
    c.alloc = opt->alloc;
    c.free_fn = opt->free;
    c.alloc_ctx = opt->alloc_ctx;
    if ((c.alloc == nullptr) != (c.free_fn == nullptr)) fail(PJ_EINVAL, "pj_options: alloc and free must be set together");
    if (opt->device_budget) {
      c.budget = std::make_shared<Budget>();
      c.budget->limit = (size_t)opt->device_budget;
    }
  }
  return c;
}

static bool trace_enabled() {
  static const bool on = [] {
    const char* v = getenv("PJ_TRACE");
    return v && v[0] && v[0] != '0';
  }();
  return on;
}

void trace_mark(const Ctx& c, const char* phase) {
  if (!trace_enabled()) return;
  static thread_local std::chrono::steady_clock::time_point last = std::chrono::steady_clock::now();
  cudaError_t e = cudaStreamSynchronize(c.stream);
  const auto now = std::chrono::steady_clock::now();
  const double ms = std::chrono::duration<double, std::milli>(now - last).count();
  fprintf(stderr, "[pj] %-28s %9.3f ms  %s\n", phase, ms, e == cudaSuccess ? "" : cudaGetErrorString(e));
  fflush(stderr);
  last = now;
}

void trace_note(const char* what) {
  if (!trace_enabled()) return;
  fprintf(stderr, "[pj]   . %s\n", what);
  fflush(stderr);
}

void debug_dump(const Ctx& c, const char* name, const void* dev, size_t bytes) {
  const char* prefix = getenv("PJ_DEBUG_DUMP");
  if (!prefix || !prefix[0]) return;
  std::vector<char> h(bytes);
  if (bytes) PJ_CUDA(cudaMemcpyAsync(h.data(), dev, bytes, cudaMemcpyDeviceToHost, c.stream));
  c.sync();
  const std::string path = std::string(prefix) + "." + name;
  FILE* f = fopen(path.c_str(), "wb");
  if (!f) return;
  if (bytes) fwrite(h.data(), 1, bytes, f);
  fclose(f);
}

// ---------------------------------------------------------------- A1 ------

namespace {

// Sort key of input string k: its first eight bytes, first byte highest,
// zero-padded (so that a stable sort by it, then by length, orders each
// length's strings alphabetically by their first eight bytes, ties by id).
__global__ void k_prefix_keys(const uint8_t* __restrict__ bytes, const uint64_t* __restrict__ off, uint32_t n,
                              unsigned long long* __restrict__ keys) {
  const uint32_t k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  const uint64_t a = off[k];
  const uint64_t len = off[k + 1] - a;
  unsigned long long key = 0;
  for (int j = 0; j < 8; ++j) key = (key << 8) | (j < (int)len ? bytes[a + j] : 0u);
  keys[k] = key;
}

// Lengths in the current order of ids: len[j] = |string ids[j]|.
__global__ void k_lengths_of(const uint64_t* __restrict__ off, const uint32_t* __restrict__ ids, uint32_t n,
                             uint32_t* __restrict__ len) {
  const uint32_t j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j < n) len[j] = (uint32_t)(off[ids[j] + 1] - off[ids[j]]);
}

__global__ void k_lengths(const uint64_t* __restrict__ off, uint32_t n, uint32_t* __restrict__ len,
                          uint32_t* __restrict__ ids, int* __restrict__ err, unsigned* __restrict__ lmax) {
  const uint32_t k = blockIdx.x * blockDim.x + threadIdx.x;
  unsigned l = 0;
  if (k < n) {
    const uint64_t a = off[k], b = off[k + 1];
    if (b < a || b - a > PJ_MAX_STRING_LEN) {
      atomicOr(err, 1);
    } else {
      l = (unsigned)(b - a);
    }
    len[k] = l;
    ids[k] = k;
  }
  // one atomic per warp
  unsigned m = l;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(FULL, m, o));
  if ((threadIdx.x & 31) == 0 && m) atomicMax(lmax, m);
}

// One warp per string: copy its bytes from input order to sid order.
__global__ void k_gather(const uint8_t* __restrict__ in_bytes, const uint64_t* __restrict__ in_off,
                         const uint32_t* __restrict__ perm, const uint64_t* __restrict__ soff,
                         uint8_t* __restrict__ sbytes, uint32_t n) {
  const uint32_t warps = (gridDim.x * blockDim.x) >> 5;
  const int lane = threadIdx.x & 31;
  for (uint32_t sid = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; sid < n; sid += warps) {
    const uint64_t src = in_off[perm[sid]];
    const uint64_t dst = soff[sid];
    const uint32_t L = (uint32_t)(soff[sid + 1] - dst);
    for (uint32_t k = lane; k < L; k += 32) sbytes[dst + k] = in_bytes[src + k];
  }
}

// Character signatures of n strings (bytes[off[k] .. off[k+1])), one thread each.
__global__ void k_signatures(const uint8_t* __restrict__ bytes, const uint64_t* __restrict__ off, uint32_t n,
                          Sig* __restrict__ bm) {
  for (uint32_t k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x)
    bm[k] = char_signature(bytes + off[k], (int)(off[k + 1] - off[k]));
}

// Prefix values (seg_value_from_prefix) of n strings: string k's |k| + 1
// values start at H[off[k] + k].  One warp per string, 32 bytes per step:
// each byte is the affine map h -> h * SEG_B + byte, and a shuffle scan
// composes the maps of the step's bytes, which are then applied to the
// value carried in from the previous step.
__global__ void k_prefix_values(const uint8_t* __restrict__ bytes, const uint64_t* __restrict__ off, uint32_t n,
                                uint32_t* __restrict__ H) {
  const unsigned lane = threadIdx.x & 31u;
  const uint64_t warp = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const uint64_t n_warps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
  for (uint64_t k = warp; k < n; k += n_warps) {
    const uint64_t o = off[k], len = off[k + 1] - o;
    uint32_t* h = H + o + k;
    if (lane == 0) h[0] = 0;
    uint32_t carry = 0;
    for (uint64_t c = 0; c < len; c += 32) {
      const uint64_t j = c + lane;
      uint32_t a = j < len ? SEG_B : 1u, v = j < len ? (uint32_t)bytes[o + j] : 0u;
#pragma unroll
      for (int d = 1; d < 32; d <<= 1) {
        const uint32_t ap = __shfl_up_sync(FULL, a, d), vp = __shfl_up_sync(FULL, v, d);
        if ((int)lane >= d) {
          v = vp * a + v;
          a = ap * a;
        }
      }
      const uint32_t val = carry * a + v;
      if (j < len) h[j + 1] = val;
      carry = __shfl_sync(FULL, val, 31);
    }
  }
}

// ref[k] = off[k] << 16 | len[k] (lengths < 2^16, offsets < 2^48).
__global__ void k_refs(const uint64_t* __restrict__ off, const uint32_t* __restrict__ len, uint32_t n,
                       unsigned long long* __restrict__ ref) {
  for (uint32_t k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x)
    ref[k] = ((unsigned long long)off[k] << 16) | len[k];
}

// bbeg[l] = first sid whose length is >= l, for l = 0 .. lmax + 1.
__global__ void k_buckets(const uint32_t* __restrict__ slen, uint32_t n, uint32_t* __restrict__ bbeg, int lmax) {
  const uint32_t sid = blockIdx.x * blockDim.x + threadIdx.x;
  if (sid > n) return;
  const int cur = sid < n ? (int)slen[sid] : lmax + 1;
  const int prev = sid > 0 ? (int)slen[sid - 1] : -1;
  for (int l = prev + 1; l <= cur; ++l) bbeg[l] = sid;
}

// ---------------------------------------------------------------- A2 ------

__global__ void k_seg_records(const uint8_t* __restrict__ sbytes, const uint64_t* __restrict__ soff,
                              const uint32_t* __restrict__ slen, uint32_t first, uint64_t n_records, int tau,
                              int scheme, unsigned long long* __restrict__ keys, uint32_t* __restrict__ vals) {
  const uint64_t r = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= n_records) return;
  const uint32_t sid = first + (uint32_t)(r / (tau + 1));
  const int i = (int)(r % (tau + 1)) + 1;
  const int l = (int)slen[sid];
  int P, li;
  segment_m(l, tau + 1, 0, scheme, i, P, li);
  keys[r] = seg_key(sbytes + soff[sid] + P, li, l, i);
  vals[r] = sid;
}

// ---------------------------------------------------------------- A3 ------

// The side signatures of every partitioned string around each of its
// segments: for sid first + x and segment i, sides[x * (tau + 1) + i - 1] =
// (signature of the bytes before the segment, signature of the bytes after
// it).  One thread per string: the prefix codes come from one pass forward,
// the suffix codes from one pass backward.
__global__ void k_side_sigs(const uint8_t* __restrict__ sbytes, const uint64_t* __restrict__ soff,
                            const uint32_t* __restrict__ slen, uint32_t first, uint32_t n, int tau, int scheme,
                            ulonglong2* __restrict__ sides) {
  for (uint32_t x = blockIdx.x * blockDim.x + threadIdx.x; first + x < n; x += gridDim.x * blockDim.x) {
    const uint32_t sid = first + x;
    const uint8_t* s = sbytes + soff[sid];
    const int l = (int)slen[sid];
    ulonglong2* out = sides + (uint64_t)x * (tau + 1);
    unsigned long long t = 0;
    int k = 0;
    for (int i = 1; i <= tau + 1; ++i) {  // prefixes: bytes [0, P_i)
      int P, li;
      segment_m(l, tau + 1, 0, scheme, i, P, li);
      for (; k < P; ++k) {
        const int sh = 4 * (int)(s[k] % SIDE_BUCKETS);
        const unsigned long long field = (t >> sh) & 15ull;
        if (field != 15ull) t |= (field + 1ull) << sh;
      }
      out[i - 1].x = t;
    }
    t = 0;
    k = l;
    for (int i = tau + 1; i >= 1; --i) {  // suffixes: bytes [P_i + l_i, l)
      int P, li;
      segment_m(l, tau + 1, 0, scheme, i, P, li);
      for (; k > P + li; --k) {
        const int sh = 4 * (int)(s[k - 1] % SIDE_BUCKETS);
        const unsigned long long field = (t >> sh) & 15ull;
        if (field != 15ull) t |= (field + 1ull) << sh;
      }
      out[i - 1].y = t;
    }
  }
}

// Posting records in posting order: the sid and its side signatures around
// the segment of the record's key (segment number in the key's low byte), or
// none (0) when sides is NULL.
__global__ void k_post_records(const uint32_t* __restrict__ postings, const unsigned long long* __restrict__ keys,
                               uint64_t n, uint32_t first, int tau, const ulonglong2* __restrict__ sides,
                               PostRec* __restrict__ recs) {
  for (uint64_t k = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (uint64_t)gridDim.x * blockDim.x) {
    const uint32_t sid = postings[k];
    if (!sides) {
      recs[k] = make_rec(sid, 0ull, 0ull);
      continue;
    }
    const int i = (int)(keys[k] & 0xFFu);
    const ulonglong2 sd = sides[(uint64_t)(sid - first) * (tau + 1) + i - 1];
    recs[k] = make_rec(sid, sd.x, sd.y);
  }
}

__global__ void k_head_flags(const unsigned long long* __restrict__ keys, uint64_t n, uint32_t* __restrict__ flags) {
  const uint64_t k = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k < n) flags[k] = (k == 0 || keys[k] != keys[k - 1]) ? 1u : 0u;
}

__global__ void k_heads(const uint32_t* __restrict__ flags, const uint32_t* __restrict__ uidx, uint64_t n,
                        uint32_t* __restrict__ heads) {
  const uint64_t k = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k < n && flags[k]) heads[uidx[k]] = (uint32_t)k;
  if (k == 0) heads[uidx[n - 1] + flags[n - 1]] = (uint32_t)n;
}

__global__ void k_table_insert(const unsigned long long* __restrict__ keys, const uint32_t* __restrict__ heads,
                               uint64_t n_unique, Slot* __restrict__ table, uint8_t* __restrict__ fp,
                               unsigned pb, unsigned long long mask, int* __restrict__ err) {
  const uint64_t u = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (u >= n_unique) return;
  const uint32_t b = heads[u], e = heads[u + 1];
  const unsigned long long key = keys[b];
  const uint32_t mix = key_mix(key);
  unsigned long long h = mix & mask;
  for (unsigned long long probe = 0; probe <= mask; ++probe) {
    const unsigned long long prev = atomicCAS(&table[h].key, 0ull, key);
    if (prev == 0ull) {
      table[h].begin = b;
      table[h].count = e - b;
      fp[h] = key_fp(key, mix);
      unsigned long long word;
      uint32_t bits;
      presence_of(mix, mask, pb, word, bits);
      atomicOr(reinterpret_cast<uint32_t*>(fp + mask + 1) + word, bits);
      return;
    }
    h = (h + 1) & mask;
  }
  atomicOr(err, 2);  // table full (cannot happen at load factor <= 1/2)
}

}  // namespace

// Stage a string set on the device (bytes rebased to offset 0).
static void stage_strings(const Ctx& c, const pj_strings& S, DBuf<uint8_t>& bytes, DBuf<uint64_t>& off,
                          const uint8_t** dbytes, const uint64_t** doff, uint64_t* total) {
  const uint32_t n = S.n;
  if (!S.offsets || (!S.bytes && n > 0)) fail(PJ_EINVAL, "pj_strings: NULL bytes or offsets");
  if (S.on_device) {
    uint64_t o[2];
    PJ_CUDA(cudaMemcpyAsync(&o[0], S.offsets, sizeof(uint64_t), cudaMemcpyDeviceToHost, c.stream));
    PJ_CUDA(cudaMemcpyAsync(&o[1], S.offsets + n, sizeof(uint64_t), cudaMemcpyDeviceToHost, c.stream));
    c.sync();
    if (o[1] < o[0]) fail(PJ_EINVAL, "pj_strings: offsets decrease");
    *dbytes = S.bytes;
    *doff = S.offsets;
    *total = o[1] - o[0];
    return;
  }
  const uint64_t o0 = S.offsets[0];
  for (uint32_t k = 0; k < n; ++k)
    if (S.offsets[k + 1] < S.offsets[k]) fail(PJ_EINVAL, "pj_strings: offsets decrease at " + std::to_string(k));
  const uint64_t tot = S.offsets[n] - o0;
  off.reset(c, (size_t)n + 1);
  std::vector<uint64_t> h(n + 1);
  for (uint32_t k = 0; k <= n; ++k) h[k] = S.offsets[k] - o0;
  PJ_CUDA(cudaMemcpyAsync(off.p, h.data(), (n + 1) * sizeof(uint64_t), cudaMemcpyHostToDevice, c.stream));
  bytes.reset(c, tot ? tot : 1);
  if (tot) PJ_CUDA(cudaMemcpyAsync(bytes.p, S.bytes + o0, tot, cudaMemcpyHostToDevice, c.stream));
  c.sync();  // h goes out of scope
  *dbytes = bytes.p;
  *doff = off.p;
  *total = tot;
}

void build_store(pj_index& idx, const pj_strings& S) {
  const Ctx& c = idx.ctx;
  const uint32_t n = S.n;
  idx.n = n;
  DBuf<uint8_t> in_bytes_buf;
  DBuf<uint64_t> in_off_buf;
  const uint8_t* in_bytes = nullptr;
  const uint64_t* in_off = nullptr;
  uint64_t total = 0;
  trace_mark(c, "build: start");
  stage_strings(c, S, in_bytes_buf, in_off_buf, &in_bytes, &in_off, &total);
  idx.total_bytes = total;
  trace_mark(c, "build: stage input");

  DBuf<int> err(c, 1);
  DBuf<unsigned> lmax(c, 1);
  PJ_CUDA(cudaMemsetAsync(err.p, 0, sizeof(int), c.stream));
  PJ_CUDA(cudaMemsetAsync(lmax.p, 0, sizeof(unsigned), c.stream));
  idx.slen.reset(c, n);
  idx.perm.reset(c, n);
  if (n) {
    k_lengths<<<ceil_div(n, 256), 256, 0, c.stream>>>(in_off, n, idx.slen.p, idx.perm.p, err.p, lmax.p);
    PJ_LAUNCHED("k_lengths");
  }
  int h_err = 0;
  unsigned h_lmax = 0;
  PJ_CUDA(cudaMemcpyAsync(&h_err, err.p, sizeof(int), cudaMemcpyDeviceToHost, c.stream));
  PJ_CUDA(cudaMemcpyAsync(&h_lmax, lmax.p, sizeof(unsigned), cudaMemcpyDeviceToHost, c.stream));
  c.sync();
  if (h_err) fail(PJ_EINVAL, "pj_strings: offsets decrease or a string is longer than 65535 bytes");
  idx.lmax = (int)h_lmax;

  // sid order: by length, then by the first eight bytes, then by id -- a
  // fixed order within each length, as Alg. 1's "visited before" needs; the
  // paper visits alphabetically (Sec. 3.2), and near-alphabetical order puts
  // strings with long common prefixes next to each other, which the
  // whole-pair verification exploits (shared prefixes, Sec. 5.3).  Two
  // stable radix sorts: by the prefix key, then by length.
  if (n) {
    DBuf<unsigned long long> pkey(c, n);
    k_prefix_keys<<<ceil_div(n, 256), 256, 0, c.stream>>>(in_bytes, in_off, n, pkey.p);
    PJ_LAUNCHED("k_prefix_keys");
    radix_sort_pairs<unsigned long long>(c, pkey.p, idx.perm.p, n, 64);
    k_lengths_of<<<ceil_div(n, 256), 256, 0, c.stream>>>(in_off, idx.perm.p, n, idx.slen.p);
    PJ_LAUNCHED("k_lengths_of");
  }
  radix_sort_pairs<uint32_t>(c, idx.slen.p, idx.perm.p, n, bits_for((uint64_t)idx.lmax + 1));
  trace_mark(c, "build: lengths + sort");

  DBuf<uint64_t> len64(c, (size_t)n + 1);
  PJ_CUDA(cudaMemsetAsync(len64.p + n, 0, sizeof(uint64_t), c.stream));
  widen_u32(c, idx.slen.p, len64.p, n);
  idx.soff.reset(c, (size_t)n + 1);
  exclusive_scan<uint64_t>(c, len64.p, idx.soff.p, (size_t)n + 1);

  idx.sbytes.reset(c, total ? total : 1);
  if (n) {
    const unsigned blocks = std::min<unsigned>(ceil_div((size_t)n * 32, 256), sm_grid_cap(16));
    k_gather<<<blocks, 256, 0, c.stream>>>(in_bytes, in_off, idx.perm.p, idx.soff.p, idx.sbytes.p, n);
    PJ_LAUNCHED("k_gather");
  }
  idx.sbm.reset(c, n ? n : 1);
  if (n) {
    k_signatures<<<std::min<unsigned>(ceil_div(n, 256), sm_grid_cap(8)), 256, 0, c.stream>>>(idx.sbytes.p, idx.soff.p, n,
                                                                                    idx.sbm.p);
    PJ_LAUNCHED("k_signatures");
  }
  if (total >> 48) fail(PJ_EINVAL, "pj_strings: more than 2^48 bytes");
  idx.sref.reset(c, n ? n : 1);
  if (n) {
    k_refs<<<std::min<unsigned>(ceil_div(n, 256), sm_grid_cap(8)), 256, 0, c.stream>>>(idx.soff.p, idx.slen.p, n,
                                                                                idx.sref.p);
    PJ_LAUNCHED("k_refs");
  }
  idx.sph.reset(c, (size_t)total + n + 1);
  if (n) {
    const unsigned blocks = std::min<unsigned>(ceil_div((size_t)n * 32, 256), sm_grid_cap(16));
    k_prefix_values<<<blocks, 256, 0, c.stream>>>(idx.sbytes.p, idx.soff.p, n, idx.sph.p);
    PJ_LAUNCHED("k_prefix_values");
  }
  idx.bbeg.reset(c, (size_t)idx.lmax + 2);
  k_buckets<<<ceil_div((size_t)n + 1, 256), 256, 0, c.stream>>>(idx.slen.p, n, idx.bbeg.p, idx.lmax);
  PJ_LAUNCHED("k_buckets");
  trace_mark(c, "build: gather + buckets");
  idx.h_bbeg.resize((size_t)idx.lmax + 2);
  PJ_CUDA(cudaMemcpyAsync(idx.h_bbeg.data(), idx.bbeg.p, idx.h_bbeg.size() * sizeof(uint32_t),
                          cudaMemcpyDeviceToHost, c.stream));
  c.sync();
}

// Average indexed length above which a table gets 2 presence-bitmap bytes
// per slot instead of 1 (long strings: 6% faster probes at tau = 32; medium
// ones: 3% slower with the larger table).
constexpr uint64_t PRESENCE2_MIN_AVG_LEN = 256;
// Indexes of strings longer than this on average are verified whole-pair by
// default (PJ_VERIFY_AUTO) and build no side signatures.
constexpr uint64_t SIDES_MAX_AVG_LEN = 256;

void check_partition(const Ctx& c, const Partition& part);

// Window size of group (length offset, segment i) when nothing clips it
// (Sec. 4.2): with a = i - 1, b = tau + 1 - i and D = |s| - l the window
// [max(P - a, P + D - b), min(P + a, P + D + b)] holds
// min(a, D + b) + min(a, b - D) + 1 positions.
static std::vector<uint16_t> group_order(int tau, bool self) {
  const int parts = tau + 1, G = parts * (self ? parts : 2 * tau + 1);
  std::vector<std::pair<int, int>> w(G);
  for (int g = 0; g < G; ++g) {
    const int D = tau - g / parts, i = 1 + g % parts, a = i - 1, b = parts - i;
    w[g] = {-std::max(0, std::min(a, D + b) + std::min(a, b - D) + 1), g};
  }
  std::stable_sort(w.begin(), w.end());
  std::vector<uint16_t> order(G);
  for (int k = 0; k < G; ++k) order[k] = (uint16_t)w[k].second;
  return order;
}

void build_partition(pj_index& idx, int tau, Partition& part) {
  const Ctx& c = idx.ctx;
  part.tau = tau;
  part.scheme = idx.scheme;
  for (int self = 0; self < 2; ++self) {
    const std::vector<uint16_t> order = group_order(tau, self != 0);
    part.gorder[self].reset(c, order.size());
    PJ_CUDA(cudaMemcpyAsync(part.gorder[self].p, order.data(), order.size() * sizeof(uint16_t),
                            cudaMemcpyHostToDevice, c.stream));
    c.sync();  // order is a local
  }
  const int lcut = tau + 1 <= idx.lmax + 1 ? tau + 1 : idx.lmax + 1;
  part.first = idx.h_bbeg[lcut];
  const uint64_t nrec = (uint64_t)(idx.n - part.first) * (uint64_t)(tau + 1);
  part.n_records = nrec;
  if (nrec > 0xFFFFFFF0ull) fail(PJ_EINVAL, "segment index: more than 2^32 records");
  part.postings.reset(c, nrec);
  // Presence bitmap of 2 bytes per slot for indexes of long strings, whose
  // probes make many lookups per stored key (fewer false positives), else 1
  // (a smaller table for L2).
  part.presence_bytes = idx.n && idx.total_bytes > PRESENCE2_MIN_AVG_LEN * idx.n ? 2 : 1;
  if (nrec == 0) {  // an empty table of the smallest size: every lookup finds nothing
    part.n_unique = 0;
    part.table.reset(c, 1024);
    part.fp.reset(c, fp_array_bytes(1024, part.presence_bytes));
    part.precs.reset(c, 1);
    PJ_CUDA(cudaMemsetAsync(part.table.p, 0, 1024 * sizeof(Slot), c.stream));
    PJ_CUDA(cudaMemsetAsync(part.fp.p, 0, fp_array_bytes(1024, part.presence_bytes), c.stream));
    return;
  }
  DBuf<unsigned long long> keys(c, nrec);
  k_seg_records<<<ceil_div(nrec, 256), 256, 0, c.stream>>>(idx.sbytes.p, idx.soff.p, idx.slen.p, part.first, nrec,
                                                           tau, part.scheme, keys.p, part.postings.p);
  PJ_LAUNCHED("k_seg_records");
  trace_mark(c, "partition: records");
  radix_sort_pairs<unsigned long long>(c, keys.p, part.postings.p, nrec, 64);
  trace_mark(c, "partition: sort");

  DBuf<uint32_t> flags(c, nrec), uidx(c, nrec);
  k_head_flags<<<ceil_div(nrec, 256), 256, 0, c.stream>>>(keys.p, nrec, flags.p);
  PJ_LAUNCHED("k_head_flags");
  exclusive_scan<uint32_t>(c, flags.p, uidx.p, nrec);
  uint32_t last[2] = {0, 0};
  PJ_CUDA(cudaMemcpyAsync(&last[0], uidx.p + nrec - 1, sizeof(uint32_t), cudaMemcpyDeviceToHost, c.stream));
  PJ_CUDA(cudaMemcpyAsync(&last[1], flags.p + nrec - 1, sizeof(uint32_t), cudaMemcpyDeviceToHost, c.stream));
  c.sync();
  const uint64_t n_unique = (uint64_t)last[0] + last[1];
  part.n_unique = n_unique;
  DBuf<uint32_t> heads(c, n_unique + 1);
  k_heads<<<ceil_div(nrec, 256), 256, 0, c.stream>>>(flags.p, uidx.p, nrec, heads.p);
  PJ_LAUNCHED("k_heads");
  if (n_unique > (1ull << 31)) fail(PJ_EINVAL, "segment index: more than 2^31 distinct segments");
  uint64_t cap = 1024;
  while (cap < 2 * n_unique) cap <<= 1;
  part.table.reset(c, cap);
  part.fp.reset(c, fp_array_bytes(cap, part.presence_bytes));  // fingerprints, then the presence bitmap
  PJ_CUDA(cudaMemsetAsync(part.table.p, 0, cap * sizeof(Slot), c.stream));
  PJ_CUDA(cudaMemsetAsync(part.fp.p, 0, fp_array_bytes(cap, part.presence_bytes), c.stream));
  DBuf<int> err(c, 1);
  PJ_CUDA(cudaMemsetAsync(err.p, 0, sizeof(int), c.stream));
  k_table_insert<<<ceil_div(n_unique, 256), 256, 0, c.stream>>>(keys.p, heads.p, n_unique, part.table.p, part.fp.p,
                                                                part.presence_bytes, cap - 1, err.p);
  PJ_LAUNCHED("k_table_insert");
  int h_err = 0;
  PJ_CUDA(cudaMemcpyAsync(&h_err, err.p, sizeof(int), cudaMemcpyDeviceToHost, c.stream));
  c.sync();
  if (h_err) fail(PJ_ECUDA, "segment table insertion failed");
  part.precs.reset(c, nrec);
  // Side signatures serve the extension screen; indexes of long strings are
  // verified whole-pair by default, and their records skip them.
  part.sides = !(idx.n && idx.total_bytes > SIDES_MAX_AVG_LEN * idx.n);
  if (!part.sides) {
    k_post_records<<<std::min<unsigned>(ceil_div(nrec, 256), sm_grid_cap(16)), 256, 0, c.stream>>>(
        part.postings.p, keys.p, nrec, part.first, tau, nullptr, part.precs.p);
    PJ_LAUNCHED("k_post_records");
  } else {
    DBuf<ulonglong2> sides(c, nrec);
    const uint32_t np = idx.n - part.first;
    k_side_sigs<<<std::min<unsigned>(ceil_div(np, 128), sm_grid_cap(16)), 128, 0, c.stream>>>(
        idx.sbytes.p, idx.soff.p, idx.slen.p, part.first, idx.n, tau, part.scheme, sides.p);
    PJ_LAUNCHED("k_side_sigs");
    k_post_records<<<std::min<unsigned>(ceil_div(nrec, 256), sm_grid_cap(16)), 256, 0, c.stream>>>(
        part.postings.p, keys.p, nrec, part.first, tau, sides.p, part.precs.p);
    PJ_LAUNCHED("k_post_records");
  }
  trace_mark(c, "partition: table");
  if (getenv("PJ_CHECK_INDEX")) check_partition(c, part);
  if (getenv("PJ_DEBUG_DUMP")) {
    const std::string t = std::to_string(tau);
    debug_dump(c, ("build_postings" + t).c_str(), part.postings.p, part.postings.bytes());
    debug_dump(c, ("build_table" + t).c_str(), part.table.p, part.table.bytes());
    debug_dump(c, "build_sbytes", idx.sbytes.p, idx.sbytes.bytes());
    debug_dump(c, "build_soff", idx.soff.p, idx.soff.bytes());
    debug_dump(c, "build_slen", idx.slen.p, idx.slen.bytes());
    debug_dump(c, "build_perm", idx.perm.p, idx.perm.bytes());
  }
}

// Host-side audit of one partition (environment PJ_CHECK_INDEX=1): the runs
// tile the postings exactly, every posting is a valid sid, every slot's
// fingerprint matches its key (0 for empty slots), the presence bitmap holds
// exactly the bits of the stored keys, and the table keeps at least half of
// its slots empty.
void check_partition(const Ctx& c, const Partition& part) {
  std::vector<Slot> t(part.table.n);
  std::vector<uint8_t> fp(part.fp.n);
  std::vector<uint32_t> post(part.n_records);
  PJ_CUDA(cudaMemcpyAsync(t.data(), part.table.p, t.size() * sizeof(Slot), cudaMemcpyDeviceToHost, c.stream));
  PJ_CUDA(cudaMemcpyAsync(fp.data(), part.fp.p, fp.size(), cudaMemcpyDeviceToHost, c.stream));
  if (!post.empty())
    PJ_CUDA(cudaMemcpyAsync(post.data(), part.postings.p, post.size() * 4, cudaMemcpyDeviceToHost, c.stream));
  c.sync();
  uint64_t empty = 0, used = 0, covered = 0;
  std::vector<uint8_t> seen(part.n_records, 0);
  const unsigned pb = part.presence_bytes;
  if (fp.size() != fp_array_bytes(t.size(), pb)) fail(PJ_ECUDA, "index audit: fingerprint array size");
  std::vector<uint8_t> bits(pb * t.size(), 0);  // the presence bitmap the stored keys give
  for (size_t h = 0; h < t.size(); ++h) {
    const Slot& s = t[h];
    if (fp[h] != (s.key ? key_fp(s.key, key_mix(s.key)) : 0)) fail(PJ_ECUDA, "index audit: fingerprint mismatch");
    if (s.key) {
      unsigned long long word;
      uint32_t wbits;
      presence_of(key_mix(s.key), t.size() - 1, pb, word, wbits);
      for (int k = 0; k < 4; ++k) bits[4 * word + k] |= (uint8_t)(wbits >> (8 * k));
    }
    if (s.key == 0) {
      ++empty;
      continue;
    }
    ++used;
    if ((uint64_t)s.begin + s.count > part.n_records || s.count == 0) fail(PJ_ECUDA, "index audit: bad run");
    for (uint32_t k = s.begin; k < s.begin + s.count; ++k) {
      if (seen[k]) fail(PJ_ECUDA, "index audit: overlapping runs");
      seen[k] = 1;
      ++covered;
    }
  }
  if (memcmp(bits.data(), fp.data() + t.size(), bits.size()) != 0) fail(PJ_ECUDA, "index audit: presence bitmap");
  fprintf(stderr, "[pj] audit tau=%d: slots=%zu used=%llu empty=%llu runs=%llu covered=%llu of %llu\n", part.tau,
          t.size(), (unsigned long long)used, (unsigned long long)empty, (unsigned long long)part.n_unique,
          (unsigned long long)covered, (unsigned long long)part.n_records);
  if (used != part.n_unique || covered != part.n_records || empty < t.size() / 2)
    fail(PJ_ECUDA, "index audit failed");
}

Partition& ensure_partition(pj_index& idx, int tau, float* ms) {
  Partition& part = idx.parts[tau];
  if (ms) *ms = 0.f;
  if (part.tau == tau) return part;
  EventTimer t(idx.ctx.stream);
  t.start();
  build_partition(idx, tau, part);
  t.stop();
  const float dt = t.ms();
  if (ms) *ms = dt;
  return part;
}

void upload_probe_set(const Ctx& c, const pj_strings& R, ProbeSet& out) {
  const uint8_t* dbytes = nullptr;
  const uint64_t* doff = nullptr;
  uint64_t total = 0;
  DBuf<uint8_t> bb;
  DBuf<uint64_t> ob;
  stage_strings(c, R, bb, ob, &dbytes, &doff, &total);
  out.n = R.n;
  // keep the device copy (host input) or reference the caller's (device input)
  out.len.reset(c, R.n);
  DBuf<uint32_t> ids(c, R.n);
  DBuf<int> err(c, 1);
  DBuf<unsigned> lmax(c, 1);
  PJ_CUDA(cudaMemsetAsync(err.p, 0, sizeof(int), c.stream));
  PJ_CUDA(cudaMemsetAsync(lmax.p, 0, sizeof(unsigned), c.stream));
  if (R.n) {
    k_lengths<<<ceil_div(R.n, 256), 256, 0, c.stream>>>(doff, R.n, out.len.p, ids.p, err.p, lmax.p);
    PJ_LAUNCHED("k_lengths");
  }
  int h_err = 0;
  unsigned h_lmax = 0;
  PJ_CUDA(cudaMemcpyAsync(&h_err, err.p, sizeof(int), cudaMemcpyDeviceToHost, c.stream));
  PJ_CUDA(cudaMemcpyAsync(&h_lmax, lmax.p, sizeof(unsigned), cudaMemcpyDeviceToHost, c.stream));
  c.sync();
  if (h_err) fail(PJ_EINVAL, "pj_strings: offsets decrease or a string is longer than 65535 bytes");
  out.lmax = (int)h_lmax;
  out.bm.reset(c, R.n ? R.n : 1);
  if (R.n) {
    k_signatures<<<std::min<unsigned>(ceil_div(R.n, 256), sm_grid_cap(8)), 256, 0, c.stream>>>(dbytes, doff, R.n, out.bm.p);
    PJ_LAUNCHED("k_signatures");
  }
  out.bytes = dbytes;
  out.off = doff;
  out.own_bytes = std::move(bb);
  out.own_off = std::move(ob);
}

}  // namespace pj

// ------------------------------------------------------------------ C ABI --

uint64_t pj_index::device_bytes() const {
  uint64_t b = sbytes.bytes() + soff.bytes() + slen.bytes() + perm.bytes() + bbeg.bytes() + sbm.bytes() + sph.bytes() +
               sref.bytes();
  for (const auto& p : parts)
    b += p.table.bytes() + p.fp.bytes() + p.postings.bytes() + p.precs.bytes() + p.gorder[0].bytes() +
         p.gorder[1].bytes();
  return b;
}

extern "C" {

void pj_options_init(pj_options* opt) {
  if (!opt) return;
  memset(opt, 0, sizeof(*opt));
  opt->verify_mode = PJ_VERIFY_AUTO;
}

int pj_build_index(const pj_strings* S, int tau_max, const pj_options* opt, pj_index** out) {
  if (out) *out = nullptr;
  pj_index* idx = nullptr;
  try {
    if (!S || !out) pj::fail(PJ_EINVAL, "pj_build_index: NULL argument");
    if (tau_max < 0 || tau_max > PJ_TAU_LIMIT) pj::fail(PJ_EINVAL, "pj_build_index: tau_max out of range");
    idx = new pj_index();
    idx->ctx = pj::make_ctx(opt);
    idx->results_on_device = opt ? opt->results_on_device != 0 : false;
    idx->lazy = opt ? opt->lazy_partitions != 0 : false;
    idx->autotune = opt ? opt->autotune != 0 : false;
    idx->scheme = opt ? opt->partition : PJ_PARTITION_EVEN;
    if (idx->scheme != PJ_PARTITION_EVEN && idx->scheme != PJ_PARTITION_CENTER)
      pj::fail(PJ_EINVAL, "pj_build_index: unknown partition scheme");
    if (opt && opt->autotune_cache) idx->autotune_cache = opt->autotune_cache;
    idx->verify_mode = opt ? opt->verify_mode : PJ_VERIFY_AUTO;
    idx->graph_joins = opt ? opt->graph_joins != 0 : false;
    PJ_CUDA(cudaGetDevice(&idx->device));
    pj::EventTimer timer(idx->ctx.stream);
    timer.start();
    pj::build_store(*idx, *S);
    idx->parts.resize(tau_max + 1);
    if (!idx->lazy)
      for (int t = 0; t <= tau_max; ++t) pj::build_partition(*idx, t, idx->parts[t]);
    timer.stop();
    idx->build_ms = timer.ms();
    idx->ctx.sync();
    *out = idx;
    return PJ_OK;
  } catch (const pj::Error& e) {
    pj::set_last_error(e.msg);
    delete idx;
    return e.code;
  } catch (const std::bad_alloc&) {
    pj::set_last_error("host allocation failed");
    delete idx;
    return PJ_ENOMEM;
  }
}

uint32_t pj_index_size(const pj_index* idx) { return idx ? idx->n : 0; }
float pj_index_build_ms(const pj_index* idx) { return idx ? idx->build_ms : 0.f; }
uint64_t pj_kernel_launches(void) { return pj::g_launches.load(); }
int pj_index_tau_max(const pj_index* idx) { return idx ? (int)idx->parts.size() - 1 : 0; }
uint64_t pj_index_device_bytes(const pj_index* idx) { return idx ? idx->device_bytes() : 0; }

void pj_index_free(pj_index* idx) {
  if (!idx) return;
  cudaStream_t s = idx->ctx.stream;
  idx->self_plans.clear();  // recorded self joins first: they read the partitions
  delete idx;  // buffers are released stream-ordered
  cudaStreamSynchronize(s);
}

const char* pj_strerror(int code) {
  switch (code) {
    case PJ_OK: return "PJ_OK";
    case PJ_EINVAL: return "PJ_EINVAL: invalid argument";
    case PJ_ENOMEM: return "PJ_ENOMEM: out of memory";
    case PJ_ECUDA: return "PJ_ECUDA: CUDA error";
    case PJ_ETIMEDOUT: return "PJ_ETIMEDOUT: wait timed out";
    case PJ_ECANCELED: return "PJ_ECANCELED: request cancelled";
    default: return "unknown pj error";
  }
}

const char* pj_last_error(void) { return pj::last_error().c_str(); }

}  // extern "C"
