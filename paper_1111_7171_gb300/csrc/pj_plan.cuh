// Buffers of a query plan (the multi-threshold query pipeline recorded into
// a CUDA graph) as the recording code sees them.  The plan object owns them;
// the recording code only launches work on them.
#pragma once

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

// Enqueues the whole query pipeline for the buffers in d on c's stream
// without any host synchronisation (meant to run under stream capture).
// Temporaries come from c's allocator and must outlive the recorded work.
void record_query_plan(const Ctx& c, const pj_index& idx, const PlanDev& d);

}  // namespace pj
