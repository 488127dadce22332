// Shared host/device plumbing of the Pass-Join CUDA library: error
// propagation, the caller-supplied (or stream-ordered) device allocator, RAII
// device buffers and a few warp helpers.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <memory>
#include <mutex>
#include <string>
#include <unordered_map>
#include <utility>

#include "passjoin.h"

namespace pj {

// ----------------------------------------------------------------- errors --

struct Error {
  int code;
  std::string msg;
};

[[noreturn]] void fail(int code, const std::string& msg);
void check_cuda(cudaError_t e, const char* what, const char* file, int line);
void count_launch();
// Launches enqueued while a graph is recorded are not launches: the counter
// skips them on the recording thread, and each replay of the graph adds its
// kernel nodes.
void set_recording(bool on);
void count_launches(unsigned long long k);
#define PJ_CUDA(call) ::pj::check_cuda((call), #call, __FILE__, __LINE__)
// After every kernel launch: count it and surface launch errors.
#define PJ_LAUNCHED(name)                                                  \
  do {                                                                     \
    ::pj::count_launch();                                                  \
    ::pj::check_cuda(cudaGetLastError(), name, __FILE__, __LINE__);        \
  } while (0)

// -------------------------------------------------------------- allocator --

// A device-memory budget (pj_options.device_budget): the bytes held at once
// through every context that shares it, the most ever held, and the limit
// past which an allocation fails with PJ_ENOMEM instead of being made.
struct Budget {
  std::mutex mu;
  size_t limit = 0;
  size_t cur = 0;
  size_t peak = 0;
  std::unordered_map<void*, size_t> live;
};

// Device memory and the stream every piece of work of one call is ordered on.
struct Ctx {
  cudaStream_t stream = nullptr;
  pj_alloc_fn alloc = nullptr;
  pj_free_fn free_fn = nullptr;
  void* alloc_ctx = nullptr;
  std::shared_ptr<Budget> budget;  // NULL: no limit, nothing counted

  void* get(size_t bytes) const;
  void put(void* p) const;
  void sync() const { PJ_CUDA(cudaStreamSynchronize(stream)); }
};

Ctx make_ctx(const pj_options* opt);

// Device time between start() and stop(), measured with CUDA events on one
// stream.  ms() synchronises on the stop event.
struct EventTimer {
  cudaEvent_t a = nullptr, b = nullptr;
  cudaStream_t s = nullptr;
  explicit EventTimer(cudaStream_t stream) : s(stream) {
    PJ_CUDA(cudaEventCreate(&a));
    PJ_CUDA(cudaEventCreate(&b));
  }
  ~EventTimer() {
    if (a) cudaEventDestroy(a);
    if (b) cudaEventDestroy(b);
  }
  EventTimer(const EventTimer&) = delete;
  EventTimer& operator=(const EventTimer&) = delete;
  void start() { PJ_CUDA(cudaEventRecord(a, s)); }
  void stop() { PJ_CUDA(cudaEventRecord(b, s)); }
  float ms() {
    PJ_CUDA(cudaEventSynchronize(b));
    float t = 0.f;
    PJ_CUDA(cudaEventElapsedTime(&t, a, b));
    return t;
  }
};

// Phase trace on stderr, enabled by the environment variable PJ_TRACE=1: each
// call synchronises the stream and prints the time since the previous mark.
void trace_mark(const Ctx& c, const char* phase);
// Same trace, without synchronising (marks host-side progress only).
void trace_note(const char* what);
// With the environment variable PJ_DEBUG_DUMP=<prefix>, writes `bytes` bytes
// of device memory to the file <prefix>.<name> (after synchronising).
void debug_dump(const Ctx& c, const char* name, const void* dev, size_t bytes);

// Device array of T obtained from a Ctx; freed (stream-ordered) on scope exit.
// It keeps a copy of the context that allocated it (allocator and stream),
// so it may outlive that Ctx object.
template <class T>
struct DBuf {
  Ctx ctx;
  T* p = nullptr;
  size_t n = 0;

  DBuf() = default;
  DBuf(const Ctx& c, size_t count) { reset(c, count); }
  DBuf(const DBuf&) = delete;
  DBuf& operator=(const DBuf&) = delete;
  DBuf(DBuf&& o) noexcept { *this = std::move(o); }
  DBuf& operator=(DBuf&& o) noexcept {
    if (this != &o) {
      release();
      ctx = o.ctx;
      p = o.p;
      n = o.n;
      o.p = nullptr;
      o.n = 0;
    }
    return *this;
  }
  ~DBuf() { release(); }

  void reset(const Ctx& c, size_t count) {
    release();
    ctx = c;
    n = count;
    p = static_cast<T*>(c.get((count ? count : 1) * sizeof(T)));
  }
  void release() {
    if (p) ctx.put(p);
    p = nullptr;
    n = 0;
  }
  T* get() const { return p; }
  size_t bytes() const { return n * sizeof(T); }
};

// ------------------------------------------------------------ small utils --

inline unsigned ceil_div(size_t a, size_t b) { return (unsigned)((a + b - 1) / b); }

// Streaming multiprocessors of the current device (looked up once per
// device), and the grid cap of a grid-stride kernel that keeps `per_sm`
// blocks on every SM.
int sm_count();
inline unsigned sm_grid_cap(unsigned per_sm) { return (unsigned)sm_count() * per_sm; }

inline int bits_for(uint64_t v) {  // bits needed to hold values < v (at least 1)
  int b = 1;
  while (b < 64 && (uint64_t(1) << b) < v) ++b;
  return b;
}

constexpr unsigned FULL = 0xffffffffu;

__device__ __forceinline__ unsigned lanemask_lt() {
  unsigned m;
  asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
  return m;
}

// Inclusive warp scan (all 32 lanes participate).
template <class T>
__device__ __forceinline__ T warp_incl_scan(T v) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    T t = __shfl_up_sync(FULL, v, o);
    if (lane >= o) v += t;
  }
  return v;
}

template <class T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(FULL, v, o);
  return v;
}

// Number of lanes whose (non-decreasing) inclusive prefix value is <= f,
// i.e. the lane that owns flat item f.  Every lane must call it.
__device__ __forceinline__ int warp_owner(int incl, int f) {
  int pos = 0;
#pragma unroll
  for (int step = 16; step > 0; step >>= 1) {
    int v = __shfl_sync(FULL, incl, pos + step - 1);
    if (v <= f) pos += step;
  }
  return pos;
}

}  // namespace pj
