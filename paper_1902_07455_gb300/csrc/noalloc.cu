// Tensor-train inner product that allocates no device memory.
//
// Some callers cannot allocate device memory at the point where they need an inner product: host
// applications that hand all device memory to their own allocator and forbid libraries from taking more,
// and real-time loops that must not block on the driver's allocator.  For them, lrfg_tt_dot_noalloc
// computes the same contraction as lrfg_tt_dot with its intermediates in one file-scope device array of
// fixed size instead of the context's pool.  Its products run in one pass over the contracted index (no
// split-K partial sums, which would need a workspace from the pool), and it records no profiling events.
#include <algorithm>
#include <map>
#include <mutex>

#include "ops.cuh"

namespace lrfg {

// 4 MiB of scratch; every GPU that loads the library holds it until the process exits.
constexpr size_t kTTDotScratchDoubles = size_t(1) << 19;
static __device__ __align__(256) double g_tt_dot_scratch[kTTDotScratchDoubles];

// Device address of the scratch array on the current device, looked up once per device.  In host
// code the array's name is only a host-side stand-in, so the address must come from
// cudaGetSymbolAddress with that device current.
static double* tt_dot_scratch_address(int device) {
  static std::mutex mu;
  static std::map<int, double*> addr;
  std::lock_guard<std::mutex> lock(mu);
  auto it = addr.find(device);
  if (it != addr.end()) return it->second;
  double* p = nullptr;
  LRFG_CUDA(cudaGetSymbolAddress((void**)&p, g_tt_dot_scratch));
  addr[device] = p;
  return p;
}

}  // namespace lrfg

using namespace lrfg;

extern "C" lrfg_status lrfg_tt_dot_noalloc(lrfg_ctx* ctx, const lrfg_tt* x, const lrfg_tt* y, double* result) {
  if (!ctx) return LRFG_EINVAL;
  try {
    LRFG_CUDA(cudaSetDevice(ctx->device));
    LRFG_REQUIRE(x && y && result, "null argument");
    LRFG_REQUIRE(x->d == y->d && x->d >= 1 && x->d <= 3, "TT orders must match and be 1..3");
    const int d = x->d;
    for (int j = 0; j < d; ++j) {
      LRFG_REQUIRE(x->N[j] == y->N[j] && x->N[j] >= 1, "TT grids differ");
      LRFG_REQUIRE(x->cores[j] && y->cores[j], "null carriage");
    }
    LRFG_REQUIRE(x->r[0] == 1 && y->r[0] == 1 && x->r[d] == 1 && y->r[d] == 1, "TT boundary ranks must be 1");
    // scratch layout: two W regions used alternately (W_j is a x c, W_{j+1} is b x e), then V (c x n b)
    size_t maxW = 1, maxV = 0;
    for (int j = 0; j < d; ++j) {
      const size_t a = x->r[j], b = x->r[j + 1], c = y->r[j], e = y->r[j + 1], n = x->N[j];
      maxW = std::max(maxW, std::max(a * c, b * e));
      maxV = std::max(maxV, c * n * b);
    }
    const size_t need = 2 * maxW + maxV;
    LRFG_REQUIRE(need <= kTTDotScratchDoubles,
                 "lrfg_tt_dot_noalloc: the contraction needs %zu doubles of scratch, more than the %zu available "
                 "(use lrfg_tt_dot)", need, kTTDotScratchDoubles);
    double* scratch = tt_dot_scratch_address(ctx->device);
    double* Wbuf[2] = {scratch, scratch + maxW};
    double* V = scratch + 2 * maxW;
    // no events while it runs: a profiled context would otherwise record a pair per launch
    const bool profiling = ctx->profiling;
    ctx->profiling = false;
    struct Restore {
      lrfg_ctx* c;
      bool p;
      ~Restore() { c->profiling = p; }
    } restore{ctx, profiling};
    // W_0 = [1]; each carriage: V = W^T x_j (c x n b), W' = V^T y_j (b x e) contracting over (c n)
    fill(ctx, Wbuf[0], 1.0, 1);
    for (int j = 0; j < d; ++j) {
      const int a = x->r[j], b = x->r[j + 1], c = y->r[j], e = y->r[j + 1], n = x->N[j];
      double* W = Wbuf[j & 1];
      double* Wn = (j == d - 1) ? result : Wbuf[(j + 1) & 1];
      gemm_nosplit(ctx, 1, 0, c, n * b, a, 1.0, W, c, 0, x->cores[j], n * b, 0, 0.0, V, n * b, 0);
      gemm_nosplit(ctx, 1, 0, b, e, c * n, 1.0, V, b, 0, y->cores[j], e, 0, 0.0, Wn, e, 0);
    }
    ctx->last_error.clear();
    return LRFG_OK;
  } catch (const Error& e) {
    ctx->last_error = e.msg;
    return e.status;
  } catch (...) {
    ctx->last_error = "unexpected internal error";
    return LRFG_ECUDA;
  }
}
