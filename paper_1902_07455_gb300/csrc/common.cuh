// Shared internals of liblrfg: status handling, the device memory pool, the context, TT containers.
#pragma once

#include <cuda_runtime.h>
#include <cstddef>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/lrfg.h"

namespace lrfg {

// ------------------------------------------------------------------------------------------------
// errors: every entry point returns an lrfg_status; internal code throws Error and the C-ABI layer
// converts it (no exception crosses the ABI).
// ------------------------------------------------------------------------------------------------
struct Error {
  lrfg_status status;
  std::string msg;
};

[[noreturn]] void fail(lrfg_status st, const char* fmt, ...);

#define LRFG_CUDA(call)                                                                          \
  do {                                                                                          \
    cudaError_t e_ = (call);                                                                    \
    if (e_ != cudaSuccess)                                                                      \
      ::lrfg::fail(e_ == cudaErrorMemoryAllocation ? LRFG_ENOMEM : LRFG_ECUDA, "%s: %s (%s:%d)", \
                   #call, cudaGetErrorString(e_), __FILE__, __LINE__);                          \
  } while (0)

#define LRFG_CHECK_LAUNCH() LRFG_CUDA(cudaGetLastError())

#define LRFG_REQUIRE(cond, ...)                        \
  do {                                                 \
    if (!(cond)) ::lrfg::fail(LRFG_EINVAL, __VA_ARGS__); \
  } while (0)

// ------------------------------------------------------------------------------------------------
// device memory pool: caching allocator keyed by rounded size (powers of two from 256 B to 64 MiB,
// 2 MiB multiples above).  Blocks go back to their free list on release and are returned to the
// driver only by trim() / destruction.
// All users of one pool work on the pool's single stream, so reuse needs no events.
// ------------------------------------------------------------------------------------------------
class DevicePool {
 public:
  explicit DevicePool(size_t budget) : budget_(budget) {}
  ~DevicePool() { trim(); }
  void* alloc(size_t bytes);
  void release(void* p);
  void trim();
  size_t in_use() const { return in_use_; }
  size_t reserved() const { return reserved_; }

 private:
  std::map<size_t, std::vector<void*>> sized_;  // free blocks by rounded size
  std::map<void*, size_t> live_size_;            // blocks handed out
  size_t budget_, in_use_ = 0, reserved_ = 0;
};

// RAII buffer from the pool
template <typename T>
class DBuf {
 public:
  DBuf() = default;
  DBuf(DevicePool* pool, size_t n) : pool_(pool), n_(n) {
    p_ = n ? static_cast<T*>(pool->alloc(n * sizeof(T))) : nullptr;
  }
  DBuf(const DBuf&) = delete;
  DBuf& operator=(const DBuf&) = delete;
  DBuf(DBuf&& o) noexcept : pool_(o.pool_), p_(o.p_), n_(o.n_) { o.p_ = nullptr; o.n_ = 0; }
  DBuf& operator=(DBuf&& o) noexcept {
    if (this != &o) { reset(); pool_ = o.pool_; p_ = o.p_; n_ = o.n_; o.p_ = nullptr; o.n_ = 0; }
    return *this;
  }
  ~DBuf() { reset(); }
  void reset() { if (p_ && pool_) pool_->release(p_); p_ = nullptr; n_ = 0; }
  T* get() const { return p_; }
  size_t size() const { return n_; }

 private:
  DevicePool* pool_ = nullptr;
  T* p_ = nullptr;
  size_t n_ = 0;
};

// ------------------------------------------------------------------------------------------------
// tensor train on the device: carriage j has shape (r[j], N[j], r[j+1]), row-major, r[0]=r[d]=1.
// ------------------------------------------------------------------------------------------------
struct TT {
  int d = 0;
  int N[3] = {0, 0, 0};
  int r[4] = {1, 1, 1, 1};
  DBuf<double> core[3];
  size_t core_elems(int j) const { return (size_t)r[j] * N[j] * r[j + 1]; }
  int max_rank() const { int m = 1; for (int j = 1; j < d; ++j) m = r[j] > m ? r[j] : m; return m; }
};

// twiddle tables W[j] = exp(-2 pi i j / N), cached per N on the device
struct Twiddles {
  double2* W = nullptr;
  int N = 0;
};

}  // namespace lrfg

// the context owns the device, the stream, the pool and cached tables
struct lrfg_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;  // caller's stream (NULL: the legacy default stream)
  lrfg::DevicePool* pool = nullptr;
  std::map<int, lrfg::Twiddles> twiddles;
  std::string last_error;
  int num_sms = 0;
  int max_smem_optin = 0;
  long long kernel_launches = 0;  // launches issued through this context (instrumentation)
  long long live_objects = 0;     // problems and fields not yet freed
};

namespace lrfg {
const Twiddles& twiddles_for(lrfg_ctx* ctx, int N);
inline void count_launch(lrfg_ctx* ctx, int n = 1) { ctx->kernel_launches += n; }
}  // namespace lrfg
