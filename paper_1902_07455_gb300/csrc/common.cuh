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
  // LRFG_POOL_POISON=1 in the environment fills every block handed out with NaN bytes (a debugging
  // aid: a kernel that reads memory it did not write then yields NaN instead of stale values)
  explicit DevicePool(size_t budget);
  ~DevicePool() { trim(); }
  void* alloc(size_t bytes);
  void release(void* p);
  void trim();
  size_t in_use() const { return in_use_; }
  size_t reserved() const { return reserved_; }
  // high-water mark of in_use() since the last reset_peak()
  size_t peak() const { return peak_; }
  void reset_peak() { peak_ = in_use_; }

 private:
  std::map<size_t, std::vector<void*>> sized_;  // free blocks by rounded size
  std::map<void*, size_t> live_size_;            // blocks handed out
  size_t budget_, in_use_ = 0, reserved_ = 0, peak_ = 0;
  bool poison_ = false;
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
  float2* Wf = nullptr;  // the same table rounded to FP32 (made on first use)
  int N = 0;
};

}  // namespace lrfg

namespace lrfg {
// kernel classes for live timing and accounting (names exported through lrfg_profile_read)
enum KClass {
  KC_FFT_FIBRES = 0,  // complex fibre FFTs (mode-wise FFT, full-format complex axes)
  KC_FIBRE_OP,        // real fibres under one Fourier multiplier (gradient / divergence)
  KC_GAUSS_MULTI,     // real fibres under the exponential-sum multipliers (preconditioner)
  KC_R2C,             // full format: real rows -> half spectra
  KC_C2R,             // full format: half spectra -> real rows
  KC_POINTWISE,       // full format: Fourier multipliers and PCG updates
  KC_REDUCE,          // dot products and energy sums
  KC_GEMM,            // FP64 GEMM (Gram matrices, contractions)
  KC_EIGEN,           // small symmetric eigen-decompositions
  KC_KHATRI_RAO,      // TT Hadamard (Khatri–Rao carriages)
  KC_TT_MISC,         // block embedding, balancing, scaling, transposes, fills
  KC_CHOL,            // pivoted Cholesky factors of the Gram matrices (TT rounding)
  KC_SKETCH,          // fused Khatri-Rao contractions of the randomised rounding
  KC_GEMM32,          // FP32 products (the sketch side of the mixed-precision randomised rounding)
  KC_ROWS_FUSED,      // full format: half spectra -> real rows -> times the coefficient -> half spectra
  KC_COUNT
};
struct KStats {
  long long launches = 0;
  double flops = 0.0;  // algorithmic floating-point operations issued
  double bytes = 0.0;  // algorithmic DRAM bytes (ideal: each operand read once, result written once)
  double ms = 0.0;     // device time from events (only while profiling is on)
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
  bool profiling = false;         // record events around every launch
  lrfg::KStats stats[lrfg::KC_COUNT];
  std::vector<std::pair<int, std::pair<cudaEvent_t, cudaEvent_t>>> pending;  // (class, (start, stop))
  std::vector<cudaEvent_t> event_pool;
  // device-side work counters (flops, bytes per class) for kernels whose work depends on data (active
  // sizes read on the device, e.g. numerical ranks); folded into stats when the profile is read
  double* work_dev = nullptr;
  // split-K arrival counters, one per output tile of a split product (all zero between launches)
  unsigned int* splitk_cnt = nullptr;
};

namespace lrfg {
const Twiddles& twiddles_for(lrfg_ctx* ctx, int N);

cudaEvent_t take_event(lrfg_ctx* ctx);
void resolve_profile(lrfg_ctx* ctx);  // synchronises, folds pending event pairs into stats

// Accounts one kernel launch of class kc (flops / bytes algorithmic) and, while profiling is on,
// brackets it with events on the context's stream.
class KTimer {
 public:
  KTimer(lrfg_ctx* ctx, KClass kc, double flops, double bytes) : ctx_(ctx), kc_(kc) {
    ctx->kernel_launches += 1;
    KStats& s = ctx->stats[kc];
    s.launches += 1;
    s.flops += flops;
    s.bytes += bytes;
    if (ctx->profiling) {
      start_ = take_event(ctx);
      cudaEventRecord(start_, ctx->stream);
    }
  }
  ~KTimer() {
    if (start_) {
      cudaEvent_t stop = take_event(ctx_);
      cudaEventRecord(stop, ctx_->stream);
      ctx_->pending.push_back({(int)kc_, {start_, stop}});
    }
  }

 private:
  lrfg_ctx* ctx_;
  KClass kc_;
  cudaEvent_t start_ = nullptr;
};

// capacity of the split-K arrival counters (a split product has fewer than 4 x 2 x 152 output tiles), and
// of the group counters of the two-level reduction (at most kSplitKGroups groups per tile), stored after them
constexpr int kSplitKCounters = 4096;
constexpr int kSplitKGroups = 64;

// the device counter pair (flops, bytes) of class kc
inline double* work_counter(lrfg_ctx* ctx, KClass kc) { return ctx->work_dev ? ctx->work_dev + 2 * (int)kc : nullptr; }
// adds its work to stats: kernels with data-dependent sizes, counted once per batch item on the device
__device__ __forceinline__ void add_work(double* counter, double flops, double bytes) {
  if (counter) {
    atomicAdd(counter, flops);
    atomicAdd(counter + 1, bytes);
  }
}
void fold_device_work(lrfg_ctx* ctx);
// Raises the dynamic shared-memory limit of kernel `func` on the current device to at least `bytes`.
// The limit only grows: contexts on other host threads may be launching the same kernel with a larger
// tile, and lowering it under them would make their launches fail.
cudaError_t raise_smem_limit(const void* func, size_t bytes);
}  // namespace lrfg

// the same with the class given as an expression
#define LRFG_LAUNCH_KC(ctx, kcexpr, flops, bytes, ...)                        \
  do {                                                                        \
    ::lrfg::KTimer kt_((ctx), (kcexpr), (double)(flops), (double)(bytes));    \
    __VA_ARGS__;                                                              \
    LRFG_CHECK_LAUNCH();                                                      \
  } while (0)

// launch a kernel with accounting: LRFG_LAUNCH(ctx, KC_GEMM, flops, bytes, kernel<<<...>>>(args));
#define LRFG_LAUNCH(ctx, kc, flops, bytes, ...)                 \
  do {                                                          \
    ::lrfg::KTimer kt_((ctx), ::lrfg::kc, (double)(flops), (double)(bytes)); \
    __VA_ARGS__;                                                \
    LRFG_CHECK_LAUNCH();                                        \
  } while (0)
