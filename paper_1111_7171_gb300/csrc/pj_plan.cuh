// Buffers of a query plan (the multi-threshold query pipeline recorded into
// a CUDA graph) as the recording code sees them.  The plan object owns them;
// the recording code only launches work on them.
#pragma once

#include <algorithm>
#include <string>

#include "pj_internal.cuh"
#include "pj_probe.cuh"

namespace pj {

// Sizes of one run, produced and consumed on the device.  hits and cands are
// adjacent: the verification kernel reads both through one pointer.
struct PlanSizes {
  unsigned long long n;       // queries in the batch (copied in by the host)
  unsigned long long groups;  // sum of the queries' group counts
  unsigned long long hits;    // non-empty lookups (may exceed the capacity)
  unsigned long long cands;   // candidates of the hits that fit
  unsigned long long pairs;   // distinct pairs (may exceed the capacity)
};

// What the last kernel of a run writes to mapped host memory.
struct PlanHeader {
  unsigned long long groups, hits, cands, accepted, pairs;
  unsigned long long lookups, cells, fallback, err;
  unsigned long long filtered, unique;  // screened-out candidates; distinct pairs (mode L)
  unsigned long long overflow;          // nonzero: a list of the fused self join outgrew its capacity
};

struct PlanDev {
  uint32_t cap_q;                 // queries per batch
  unsigned long long cap_groups;  // cap_q * groups of the largest threshold
  unsigned long long cap_hits, cap_acc, cap_pairs;
  // batch, written by host-to-device copies before each launch
  const uint8_t* bytes;
  const uint64_t* off;  // cap_q + 1, rebased to 0
  const uint8_t* tau;   // cap_q
  PlanSizes* sizes;
  // pipeline state
  uint32_t* len;                  // cap_q
  Sig* bm;                        // cap_q character signatures
  unsigned long long* gcnt;       // cap_q groups per query
  unsigned long long* qgoff;      // cap_q group offsets
  const PartView* parts;          // tau_max + 1 thresholds
  void* counters;                 // 64 bytes, zeroed by the graph
  uint32_t* gcounts;              // cap_groups
  uint32_t* goff;                 // cap_groups
  unsigned long long* gmask;      // cap_groups window-position masks
  Hit* hits;                      // cap_hits
  unsigned long long* hcnt;       // cap_hits
  unsigned long long* hoff;       // cap_hits
  unsigned long long* acc_key[2]; // cap_acc each (sort double buffer)
  uint32_t* acc_ed[2];
  uint32_t* flags;                // cap_acc
  uint32_t* pos;                  // cap_acc
  // outputs in mapped pinned host memory (device-visible addresses)
  pj_pair* out_pairs;             // cap_pairs
  PlanHeader* header;
};

// Pinned host memory, optionally mapped into the device address space.
struct HostBuf {
  void* p = nullptr;
  void* dev = nullptr;
  size_t bytes = 0;
  HostBuf() = default;
  HostBuf(const HostBuf&) = delete;
  HostBuf& operator=(const HostBuf&) = delete;
  ~HostBuf() { release(); }
  void reset(size_t n, bool mapped) {
    release();
    const size_t b = std::max<size_t>(n, 64);
    const cudaError_t e = cudaHostAlloc(&p, b, mapped ? cudaHostAllocMapped : cudaHostAllocDefault);
    if (e != cudaSuccess) {
      cudaGetLastError();
      p = nullptr;
      fail(PJ_ENOMEM, "cudaHostAlloc of " + std::to_string(b) + " bytes failed: " + cudaGetErrorString(e));
    }
    bytes = b;
    if (mapped) PJ_CUDA(cudaHostGetDevicePointer(&dev, p, 0));
  }
  void release() {
    if (p) cudaFreeHost(p);
    p = dev = nullptr;
    bytes = 0;
  }
};

// Bump allocator over the arena that holds the recorded primitives'
// temporaries; frees are no-ops (the arena is released with the graph).
struct Arena {
  unsigned char* base = nullptr;
  size_t cap = 0, used = 0;
  bool exhausted = false;
};

inline void* arena_alloc(void* ctx, size_t bytes, void*) {
  Arena* a = static_cast<Arena*>(ctx);
  const size_t off = (a->used + 255) & ~size_t(255);
  if (off + bytes > a->cap) {
    a->exhausted = true;
    return nullptr;
  }
  a->used = off + bytes;
  return a->base + off;
}

inline void arena_free(void*, void*, void*) {}

inline size_t align256(size_t b) { return (b + 255) & ~size_t(255); }

// Temporaries of exclusive_scan_dn over n items of es bytes: two arrays of
// tile sums per level of the recursion.
inline size_t scan_temp_bytes(size_t n, size_t es) {
  size_t b = 0;
  while (n > 4096) {
    n = (n + 4095) / 4096;
    b += 2 * align256(n * es);
  }
  return b;
}

// Temporaries of radix_sort_pairs_dn over n items: digit histograms and
// their offsets (256 per 2048-item tile), and their scan.
inline size_t sort_temp_bytes(size_t n) {
  const size_t h = 256 * ((n + 2047) / 2048);
  return 2 * align256(h * 4) + scan_temp_bytes(h, 4);
}

// Enqueues the whole query pipeline for the buffers in d on c's stream
// without any host synchronisation (meant to run under stream capture).
// Temporaries come from c's allocator and must outlive the recorded work.
void record_query_plan(const Ctx& c, const pj_index& idx, const PlanDev& d);

}  // namespace pj
