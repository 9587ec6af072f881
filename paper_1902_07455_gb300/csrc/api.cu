// C ABI of liblrfg: contexts, problems (resident coefficient + operator + solvers), fields.
//
// Operator and solver composition (Sec. 2.2.2, 2.3, 3.2, 3.3 of arXiv:1902.07455):
//  * FULL: the Fourier-space GaNi operator grad^* F A~ F^{-1} grad^ on half spectra, PCG with the
//    Laplacian preconditioner P^-1 = 1/(k.k), A_eff by the rectangle rule.
//  * TT: the truncated operator T P~^-1 T grad^* F T A~ F^{-1} grad^ of Eq. (Pls_lowrank) in its
//    real-space form.  Mode-wise F is a scaled unitary map, so truncation commutes with it, and
//    F^{-1} grad^_a F is the real circulant D_a acting on the fibres of carriage a.  The real-space
//    operator therefore is  v -> T P~^-1 T( sum_a -D_a T(a (.) D_a v) ),  the same field as the paper's
//    Fourier-space form, with real carriages.  The minimal-residual iteration of Sec. 3.3 runs on it.
#include <chrono>
#include <cmath>
#include <type_traits>
#include <cstdarg>
#include <cstdlib>
#include <algorithm>
#include <map>
#include <mutex>
#include <new>
#include <vector>

#include "full.cuh"

namespace lrfg {

void fail(lrfg_status st, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  throw Error{st, std::string(buf)};
}

// ------------------------------------------------------------------------------------------------
// DevicePool
// ------------------------------------------------------------------------------------------------
static size_t rounded(size_t bytes) {
  if (bytes < 256) return 256;
  if (bytes <= (64ull << 20)) {
    size_t p = 256;
    while (p < bytes) p <<= 1;
    return p;
  }
  const size_t g = 2ull << 20;
  return (bytes + g - 1) / g * g;
}

DevicePool::DevicePool(size_t budget) : budget_(budget) {
  const char* v = std::getenv("LRFG_POOL_POISON");
  poison_ = v && v[0] == '1';
}

void* DevicePool::alloc(size_t bytes) {
  size_t sz = rounded(bytes);
  auto& lst = sized_[sz];
  void* p = nullptr;
  if (!lst.empty()) {
    p = lst.back();
    lst.pop_back();
  } else {
    if (budget_ && reserved_ + sz > budget_) {
      trim();
      if (reserved_ + sz > budget_)
        fail(LRFG_ENOMEM, "device pool budget exceeded: %zu + %zu > %zu bytes", reserved_, sz, budget_);
    }
    cudaError_t e = cudaMalloc(&p, sz);
    if (e != cudaSuccess) {
      cudaGetLastError();
      trim();
      e = cudaMalloc(&p, sz);
      if (e != cudaSuccess) {
        cudaGetLastError();
        fail(LRFG_ENOMEM, "cudaMalloc(%zu) failed: %s", sz, cudaGetErrorString(e));
      }
    }
    reserved_ += sz;
  }
  live_size_[p] = sz;
  in_use_ += sz;
  if (in_use_ > peak_) peak_ = in_use_;
  if (poison_) {
    cudaDeviceSynchronize();
    cudaMemset(p, 0xff, sz);
    cudaDeviceSynchronize();  // the fill is complete before any stream uses the block
  }
  return p;
}

void DevicePool::release(void* p) {
  auto it = live_size_.find(p);
  if (it == live_size_.end()) return;
  size_t sz = it->second;
  live_size_.erase(it);
  in_use_ -= sz;
  sized_[sz].push_back(p);
}

void DevicePool::trim() {
  // the pool's stream must be idle before cached blocks are returned to the driver
  cudaDeviceSynchronize();
  for (auto& kv : sized_) {
    for (void* p : kv.second) {
      cudaFree(p);
      reserved_ -= kv.first;
    }
    kv.second.clear();
  }
}

cudaEvent_t take_event(lrfg_ctx* ctx) {
  if (!ctx->event_pool.empty()) {
    cudaEvent_t e = ctx->event_pool.back();
    ctx->event_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  LRFG_CUDA(cudaEventCreate(&e));
  return e;
}

void fold_device_work(lrfg_ctx* ctx) {
  if (!ctx->work_dev) return;
  double h[2 * KC_COUNT];
  LRFG_CUDA(cudaStreamSynchronize(ctx->stream));
  LRFG_CUDA(cudaMemcpyAsync(h, ctx->work_dev, sizeof(h), cudaMemcpyDeviceToHost, ctx->stream));
  LRFG_CUDA(cudaMemsetAsync(ctx->work_dev, 0, sizeof(h), ctx->stream));
  LRFG_CUDA(cudaStreamSynchronize(ctx->stream));
  for (int k = 0; k < KC_COUNT; ++k) {
    ctx->stats[k].flops += h[2 * k];
    ctx->stats[k].bytes += h[2 * k + 1];
  }
}

cudaError_t raise_smem_limit(const void* func, size_t bytes) {
  static std::mutex mu;
  static std::map<std::pair<int, const void*>, size_t> limit;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lock(mu);
  size_t& cur = limit[{dev, func}];
  if (bytes <= cur) return cudaSuccess;
  e = cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  if (e == cudaSuccess) cur = bytes;
  return e;
}

void resolve_profile(lrfg_ctx* ctx) {
  if (ctx->pending.empty()) return;
  LRFG_CUDA(cudaStreamSynchronize(ctx->stream));
  for (auto& p : ctx->pending) {
    float ms = 0.f;
    LRFG_CUDA(cudaEventElapsedTime(&ms, p.second.first, p.second.second));
    ctx->stats[p.first].ms += ms;
    ctx->event_pool.push_back(p.second.first);
    ctx->event_pool.push_back(p.second.second);
  }
  ctx->pending.clear();
}

static const char* kClassNames[KC_COUNT] = {
    "fft_fibres", "fibre_operator", "gauss_multi", "r2c_rows", "c2r_rows", "pointwise",
    "reduce", "gemm", "eigen", "khatri_rao", "tt_misc", "gram_factor", "sketch", "gemm_f32", "rows_fused"};

}  // namespace lrfg

using namespace lrfg;

// ------------------------------------------------------------------------------------------------
// objects
// ------------------------------------------------------------------------------------------------
struct lrfg_field {
  lrfg_ctx* ctx = nullptr;
  lrfg_format fmt = LRFG_FULL;
  int d = 0;
  int N[3] = {0, 0, 0};
  TT tt;              // TT: real-space carriages
  TK tk;              // TUCKER: real-space core and factors
  DBuf<double2> half; // FULL: Phi u (unnormalised half spectrum)
};

struct lrfg_problem {
  lrfg_ctx* ctx = nullptr;
  lrfg_opts opts{};
  int d = 0;
  int N[3] = {0, 0, 0};
  TT a_tt;                   // TT coefficient (LRFG_TT)
  TK a_tk;                   // Tucker coefficient (LRFG_TUCKER)
  DBuf<double> a_full;       // grid coefficient (LRFG_FULL)
  std::vector<double> pt, pw;  // exponential sum of P~^-1
  FullGrid g{};
  DBuf<double2> wc;          // FULL workspace: one half spectrum
  DBuf<double> wr;           // FULL workspace: one real grid
  DBuf<double> inv64;        // FULL: reciprocal tables of k.k (the grid g points at them)
  DBuf<float> inv32;
  // LRFG_MIXED (FULL only): FP32 copies of the coefficient and FP32 workspaces
  DBuf<float> a_full_f;
  DBuf<float2> wcf;
  DBuf<float> wrf;
  // constant anisotropic part B (d x d row-major, 3 x 3 storage) of A~ = a I + B; aniso = B != 0
  double B[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
  bool aniso = false;
  // Ga (exact integration, FULL / FP64): the double grid M = 2N - 1, (|N| / |M|) A~ on it, workspaces
  bool ga = false;
  FullGrid gM{};
  DBuf<double> a_ga, wrM;
  DBuf<double2> wcM;
  // Ga in TT: the modified coefficient on the double grid, and its projection on the grid (right-hand side);
  // with an anisotropic part also the modified coefficient of the constant 1
  TT a_ga_tt, a_down_tt, ones_ga_tt;
  // Ga in Tucker / CP: the same in Tucker form (tkga views them)
  TK a_ga_tk, a_down_tk, ones_ga_tk;
  TKGa tkga{};
  // randomised rounding (opts.sketch_over > 0): the sketch TT of ranks rank + sketch_over, by rank
  std::map<int, TT> sketches;
};

namespace {

__global__ void first_nonpositive_kernel(const double* __restrict__ v, long long n, unsigned long long* first) {
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x) {
    const double x = v[t];
    if (!(isfinite(x) && x > 0.0)) atomicMin(first, (unsigned long long)t);
  }
}

// index of the first entry that is not positive and finite, or -1
long long first_nonpositive(lrfg_ctx* ctx, const double* v, long long n) {
  DBuf<unsigned long long> first(ctx->pool, 1);
  LRFG_CUDA(cudaMemsetAsync(first.get(), 0xff, sizeof(unsigned long long), ctx->stream));
  const long long blocks = std::max(1LL, std::min((n + 255) / 256, 16LL * (ctx->num_sms > 0 ? ctx->num_sms : 152)));
  LRFG_LAUNCH(ctx, KC_REDUCE, (double)n, sizeof(double) * (double)n,
              first_nonpositive_kernel<<<(unsigned)blocks, 256, 0, ctx->stream>>>(v, n, first.get()));
  unsigned long long h = 0;
  LRFG_CUDA(cudaMemcpyAsync(&h, first.get(), sizeof(h), cudaMemcpyDeviceToHost, ctx->stream));
  LRFG_CUDA(cudaStreamSynchronize(ctx->stream));
  return h == ~0ULL ? -1 : (long long)h;
}

template <class F>
lrfg_status guard(lrfg_ctx* ctx, F&& f) {
  try {
    if (ctx) LRFG_CUDA(cudaSetDevice(ctx->device));
    f();
    if (ctx) ctx->last_error.clear();
    return LRFG_OK;
  } catch (const Error& e) {
    if (ctx) ctx->last_error = e.msg;
    return e.status;
  } catch (const std::bad_alloc&) {
    if (ctx) ctx->last_error = "host allocation failed";
    return LRFG_ENOMEM;
  } catch (...) {
    if (ctx) ctx->last_error = "unexpected internal error";
    return LRFG_ECUDA;
  }
}

long long grid_size(int d, const int* N) {
  long long s = 1;
  for (int j = 0; j < d; ++j) s *= N[j];
  return s;
}

void check_grid(int d, const int* N) {
  LRFG_REQUIRE(d == 2 || d == 3, "d must be 2 or 3 (got %d)", d);
  LRFG_REQUIRE(N != nullptr, "null grid sizes");
  for (int j = 0; j < d; ++j) {
    LRFG_REQUIRE(N[j] >= 3 && (N[j] % 2 == 1), "grid size N[%d] = %d must be odd and >= 3", j, N[j]);
  }
}

void check_tt(const lrfg_tt* x) {
  LRFG_REQUIRE(x != nullptr, "null TT");
  check_grid(x->d, x->N);
  LRFG_REQUIRE(x->r[0] == 1 && x->r[x->d] == 1, "TT boundary ranks must be 1");
  for (int j = 1; j < x->d; ++j) LRFG_REQUIRE(x->r[j] >= 1, "TT rank r[%d] = %d < 1", j, x->r[j]);
  for (int j = 0; j < x->d; ++j) LRFG_REQUIRE(x->cores[j] != nullptr, "null TT carriage %d", j);
}

// CP (canonical) solutions exist for d = 2 only, where they are Tucker tensors whose truncation (QR of
// both factors, SVD of R1 diag(c) R2^T, App. A.1.3) is the d = 2 Tucker truncation: they share its path
bool tucker_like(int fmt) { return fmt == LRFG_TUCKER || fmt == LRFG_CP; }

// B symmetric (to 1e-12 of its largest entry) and positive semidefinite: the eigenvalues of the d x d
// matrix by cyclic Jacobi rotations (d <= 3) must be >= -1e-12 max|B|.  Returns true when B != 0.
bool check_aniso(int d, const double* Bin, double* B) {
  double bmax = 0.0;
  for (int i = 0; i < d; ++i)
    for (int j = 0; j < d; ++j) {
      const double v = Bin[i * 3 + j];
      LRFG_REQUIRE(std::isfinite(v), "anisotropic part B must be finite");
      bmax = std::max(bmax, std::fabs(v));
    }
  for (int t = 0; t < 9; ++t) B[t] = 0.0;
  if (bmax == 0.0) return false;
  for (int i = 0; i < d; ++i)
    for (int j = 0; j < d; ++j) {
      LRFG_REQUIRE(std::fabs(Bin[i * 3 + j] - Bin[j * 3 + i]) <= 1e-12 * bmax, "anisotropic part B must be symmetric");
      B[i * 3 + j] = 0.5 * (Bin[i * 3 + j] + Bin[j * 3 + i]);
    }
  double M[3][3];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) M[i][j] = (i < d && j < d) ? B[i * 3 + j] : 0.0;
  for (int sweep = 0; sweep < 50; ++sweep) {
    double off = 0.0;
    for (int p = 0; p < d; ++p)
      for (int q = p + 1; q < d; ++q) off += M[p][q] * M[p][q];
    if (off <= 1e-32 * bmax * bmax) break;
    for (int p = 0; p < d; ++p)
      for (int q = p + 1; q < d; ++q) {
        if (M[p][q] == 0.0) continue;
        const double th = 0.5 * (M[q][q] - M[p][p]) / M[p][q];
        const double t = (th >= 0.0 ? 1.0 : -1.0) / (std::fabs(th) + std::sqrt(th * th + 1.0));
        const double c = 1.0 / std::sqrt(t * t + 1.0), sn = t * c;
        for (int k = 0; k < d; ++k) {  // columns p, q
          const double mp = M[k][p], mq = M[k][q];
          M[k][p] = c * mp - sn * mq;
          M[k][q] = sn * mp + c * mq;
        }
        for (int k = 0; k < d; ++k) {  // rows p, q
          const double mp = M[p][k], mq = M[q][k];
          M[p][k] = c * mp - sn * mq;
          M[q][k] = sn * mp + c * mq;
        }
      }
  }
  for (int i = 0; i < d; ++i)
    LRFG_REQUIRE(M[i][i] >= -1e-12 * bmax, "anisotropic part B must be positive semidefinite (eigenvalue %g)", M[i][i]);
  return true;
}

void check_tucker(const lrfg_tucker* x) {
  LRFG_REQUIRE(x != nullptr, "null Tucker tensor");
  check_grid(x->d, x->N);
  LRFG_REQUIRE(x->core != nullptr, "null Tucker core");
  for (int j = 0; j < x->d; ++j) {
    LRFG_REQUIRE(x->r[j] >= 1 && x->r[j] <= x->N[j] * 64, "Tucker rank r[%d] = %d out of range", j, x->r[j]);
    LRFG_REQUIRE(x->factors[j] != nullptr, "null Tucker factor %d", j);
  }
}

void upload_tucker(lrfg_ctx* ctx, const lrfg_tucker* src, int on_device, TK& dst) {
  tk_alloc(ctx, dst, src->d, src->N, src->r);
  size_t nc = 1;
  for (int j = 0; j < src->d; ++j) nc *= (size_t)src->r[j];
  const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  LRFG_CUDA(cudaMemcpyAsync(dst.core.get(), src->core, sizeof(double) * nc, kind, ctx->stream));
  for (int j = 0; j < src->d; ++j)
    LRFG_CUDA(cudaMemcpyAsync(dst.fac[j].get(), src->factors[j], sizeof(double) * src->N[j] * src->r[j], kind,
                              ctx->stream));
}

size_t core_elems(const lrfg_tt* x, int j) { return (size_t)x->r[j] * x->N[j] * x->r[j + 1]; }

void upload_tt(lrfg_ctx* ctx, const lrfg_tt* src, int on_device, TT& dst) {
  tt_alloc(ctx, dst, src->d, src->N, src->r);
  for (int j = 0; j < src->d; ++j) {
    size_t n = core_elems(src, j);
    if (!on_device) {
      for (size_t i = 0; i < n; ++i)
        LRFG_REQUIRE(std::isfinite(src->cores[j][i]), "non-finite value in TT carriage %d", j);
    }
    LRFG_CUDA(cudaMemcpyAsync(dst.core[j].get(), src->cores[j], sizeof(double) * n,
                              on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, ctx->stream));
  }
}

void publish_tt(const TT& src, lrfg_tt* dst) {
  dst->d = src.d;
  for (int j = 0; j < 3; ++j) dst->N[j] = src.N[j];
  for (int j = 0; j < 4; ++j) dst->r[j] = src.r[j];
}

// copies carriages of an internal TT into caller buffers
void download_tt(lrfg_ctx* ctx, const TT& src, double* const* cores, int on_device) {
  for (int j = 0; j < src.d; ++j) {
    LRFG_REQUIRE(cores[j] != nullptr, "null output carriage %d", j);
    LRFG_CUDA(cudaMemcpyAsync(cores[j], src.core[j].get(), sizeof(double) * src.core_elems(j),
                              on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, ctx->stream));
  }
  if (!on_device) LRFG_CUDA(cudaStreamSynchronize(ctx->stream));
}

void ones_tt(lrfg_ctx* ctx, int d, const int* N, TT& x) {
  int r[4] = {1, 1, 1, 1};
  tt_alloc(ctx, x, d, N, r);
  for (int j = 0; j < d; ++j) fill(ctx, x.core[j].get(), 1.0, N[j]);
}

// the anisotropic part for the Tucker path, or null when isotropic
const double* aniso_b(const lrfg_problem* P) { return P->aniso ? P->B : nullptr; }

// E.B E for the 3 x 3 row-major storage of B
double quad_form(const double* B, const double* E, int d) {
  double v = 0.0;
  for (int i = 0; i < d; ++i)
    for (int j = 0; j < d; ++j) v += E[i] * B[i * 3 + j] * E[j];
  return v;
}

// Ga descriptor of a Tucker / CP problem (null: GaNi)
const TKGa* tk_ga(const lrfg_problem* P) { return P->ga && tucker_like(P->opts.fmt) ? &P->tkga : nullptr; }

// ---- TT operator pieces -----------------------------------------------------------------------

// the sketch of the randomised rounding at truncation rank r (null: deterministic rounding)
const TTView* sketch_for(lrfg_problem* P, int r, TTView& view) {
  if (P->opts.sketch_over <= 0 || P->ga) return nullptr;
  const int ell = r + P->opts.sketch_over;
  auto it = P->sketches.find(ell);
  if (it == P->sketches.end()) {
    TT om;
    sketch_tt(P->ctx, P->d, P->N, ell, (unsigned long long)P->opts.sketch_seed, om);
    it = P->sketches.emplace(ell, std::move(om)).first;
  }
  view = view_of(it->second);
  return &view;
}


// e = D_alpha v (scaled): carriage alpha replaced, the others shared with v
struct ModeReplaced {
  DBuf<double> core;
  TTView view;
};

void mode_replace(lrfg_ctx* ctx, const TTView& v, int alpha, double scale, ModeReplaced& out) {
  size_t n = (size_t)v.r[alpha] * v.N[alpha] * v.r[alpha + 1];
  out.core = DBuf<double>(ctx->pool, n);
  fibre_operator(ctx, v.core[alpha], out.core.get(), v.r[alpha], v.N[alpha], v.r[alpha + 1], LRFG_MUL_DERIV, 0.0,
                 scale);
  out.view = v;
  out.view.core[alpha] = out.core.get();
}

// copy of a TT (or each item of a batch stacked along the first rank index) with every carriage mapped by
// a Ga mode map (sizes N <-> M)
void tt_ga_map(lrfg_ctx* ctx, const TTView& x, int nb, const int* n_out, int mode, TTBatch& out) {
  out.d = x.d;
  out.nb = nb;
  for (int j = 0; j < 3; ++j) out.N[j] = j < x.d ? n_out[j] : 0;
  for (int j = 0; j < 4; ++j) out.r[j] = x.r[j];
  for (int j = 0; j < x.d; ++j) {
    out.core[j] = DBuf<double>(ctx->pool, out.elems(j) * nb);
    ga_resample(ctx, x.core[j], out.core[j].get(), (long long)nb * x.r[j], x.N[j], x.r[j + 1], n_out[j], mode);
  }
}

// Ga operator in TT (Eq. (ls_Ga_fourier) with the truncations of Eq. (Pls_lowrank)): the gradient components
// interpolated to the double grid, the Khatri-Rao product with the modified coefficient and T there, the
// projection back to the grid, then the divergence, the sum and the preconditioner as for GaNi
void lr_apply_ga(lrfg_problem* P, const TTView& v, TT& out, int r) {
  lrfg_ctx* ctx = P->ctx;
  const double tol = P->opts.rank_tol;
  const int d = P->d;
  const TTView a = view_of(P->a_ga_tt);
  int M[3] = {0, 0, 0};
  for (int j = 0; j < d; ++j) M[j] = a.N[j];
  TTBatch vu;  // v on the double grid
  tt_ga_map(ctx, v, 1, M, GA_UP, vu);
  DBuf<double> gu[3];  // gradient carriages D_a v_a on the double grid
  for (int alpha = 0; alpha < d; ++alpha) {
    DBuf<double> g(ctx->pool, (size_t)v.r[alpha] * v.N[alpha] * v.r[alpha + 1]);
    fibre_operator(ctx, v.core[alpha], g.get(), v.r[alpha], v.N[alpha], v.r[alpha + 1], LRFG_MUL_DERIV, 0.0, 1.0);
    gu[alpha] = DBuf<double>(ctx->pool, (size_t)v.r[alpha] * M[alpha] * v.r[alpha + 1]);
    ga_resample(ctx, g.get(), gu[alpha].get(), v.r[alpha], v.N[alpha], v.r[alpha + 1], M[alpha], GA_UP);
  }
  int rk[4];
  for (int j = 0; j <= d; ++j) rk[j] = a.r[j] * v.r[j];
  TTBatch kr;
  ttb_alloc(ctx, kr, d, M, rk, d);
  for (int alpha = 0; alpha < d; ++alpha)
    for (int j = 0; j < d; ++j)
      khatri_rao(ctx, a.core[j], a.r[j], a.N[j], a.r[j + 1], (j == alpha) ? gu[j].get() : vu.core[j].get(), v.r[j],
                 v.r[j + 1], kr.core[j].get() + (size_t)alpha * kr.elems(j));
  TTView terms[3];
  TTBatch wd;        // I* F_M back to the grid, every item (isotropic)
  TTBatch wda[3];    // the same, component by component (anisotropic)
  if (!P->aniso) {
    for (auto& g : gu) g.reset();
    vu = TTBatch();
    TTBatch w;
    tt_round_batch(ctx, batch_view(kr), r, w, tol);  // T on the double grid
    kr = TTBatch();
    tt_ga_map(ctx, item_view(w, 0), d, P->N, GA_DOWN, wd);
    for (int alpha = 0; alpha < d; ++alpha) terms[alpha] = item_view(wd, alpha);
  } else {
    // A~ = a~ I + B 1~ (1~ the modified coefficient of the constant 1): component a on the double grid is
    // a~ (.) e_a + sum_b B[a][b] 1~ (.) e_b (a TT sum, zero entries of B skipped), then T there
    const TTView one = view_of(P->ones_ga_tt);
    TT oe[3];
    for (int beta = 0; beta < d; ++beta) {
      TTView e = item_view(vu, 0);
      e.core[beta] = gu[beta].get();
      tt_hadamard(ctx, one, e, oe[beta]);  // 1~ (.) e_b, rank of e_b
    }
    for (auto& g : gu) g.reset();
    vu = TTBatch();
    for (int alpha = 0; alpha < d; ++alpha) {
      TTView xs[4];
      double sc[4];
      int m = 0;
      xs[m] = item_view(kr, alpha);
      sc[m++] = 1.0;
      for (int beta = 0; beta < d; ++beta) {
        const double bab = P->B[alpha * 3 + beta];
        if (bab == 0.0) continue;
        xs[m] = view_of(oe[beta]);
        sc[m++] = bab;
      }
      TT sum, wa;
      tt_add_many(ctx, xs, sc, m, sum);
      tt_round(ctx, view_of(sum), r, wa, tol);  // T on the double grid
      tt_ga_map(ctx, view_of(wa), 1, P->N, GA_DOWN, wda[alpha]);
      terms[alpha] = item_view(wda[alpha], 0);
    }
    kr = TTBatch();
  }
  for (int alpha = 0; alpha < d; ++alpha) {
    double* c = const_cast<double*>(terms[alpha].core[alpha]);
    fibre_operator(ctx, c, c, terms[alpha].r[alpha], terms[alpha].N[alpha], terms[alpha].r[alpha + 1],
                   LRFG_MUL_DERIV, 0.0, -1.0);
  }
  TT acc;
  tt_add_many(ctx, terms, nullptr, d, acc);
  TT sdiv;
  tt_round(ctx, view_of(acc), r, sdiv, tol);
  tt_precond(ctx, view_of(sdiv), P->pt, P->pw, r, out, tol);
}

// rank r of every truncation (the problem's rank, or the current rank of a rank-adapting solve).  mixed: the
// operator of the mixed-precision path (FP32 fibre transforms and FP32 sketch side of the randomised rounding;
// carriages, projections, eigen-decompositions and inner products in FP64)
void lr_apply(lrfg_problem* P, const TTView& v, TT& out, int r, bool mixed = false) {
  if (P->ga) {
    lr_apply_ga(P, v, out, r);
    return;
  }
  lrfg_ctx* ctx = P->ctx;
  const double tol = P->opts.rank_tol;
  const int d = P->d;
  const TTView a = view_of(P->a_tt);
  // gradient carriages D_a v_a (rank kept; the other carriages are shared with v)
  DBuf<double> grad[3];
  for (int alpha = 0; alpha < d; ++alpha) {
    grad[alpha] = DBuf<double>(ctx->pool, (size_t)v.r[alpha] * v.N[alpha] * v.r[alpha + 1]);
    fibre_operator(ctx, v.core[alpha], grad[alpha].get(), v.r[alpha], v.N[alpha], v.r[alpha + 1], LRFG_MUL_DERIV,
                   0.0, 1.0, mixed);
  }
  // material products A~ e_a for all components at once (Khatri–Rao carriages), one batch of d TTs
  int rk[4];
  for (int j = 0; j <= d; ++j) rk[j] = a.r[j] * v.r[j];
  TTView omv;
  const TTView* om = sketch_for(P, r, omv);
  TTBatch kr;
  TTBatch w;
  TT wa[3];
  TTView terms[3];
  if (om && !P->aniso) {
    // randomised rounding of the d products, which are never formed
    SketchSource z;
    z.kind = SketchSource::KHATRI_RAO;
    z.d = d;
    z.nb = d;
    z.x = a;
    for (int j = 0; j < 3; ++j) z.N[j] = v.N[j];
    for (int j = 0; j <= d; ++j) {
      z.s[j] = rk[j];
      z.ry[j] = v.r[j];
    }
    for (int alpha = 0; alpha < d; ++alpha)
      for (int j = 0; j < d; ++j) z.y[j][alpha] = (j == alpha) ? grad[j].get() : v.core[j];
    tt_round_sketch(ctx, z, *om, r, w, tol, mixed, !P->opts.sketch_keep);  // T, all components in one sweep
    for (auto& g : grad) g.reset();
    for (int alpha = 0; alpha < d; ++alpha) terms[alpha] = item_view(w, alpha);
  } else {
    ttb_alloc(ctx, kr, d, v.N, rk, d);
    for (int alpha = 0; alpha < d; ++alpha)
      for (int j = 0; j < d; ++j)
        khatri_rao(ctx, a.core[j], a.r[j], a.N[j], a.r[j + 1], (j == alpha) ? grad[j].get() : v.core[j], v.r[j],
                   v.r[j + 1], kr.core[j].get() + (size_t)alpha * kr.elems(j));
  }
  if (om && !P->aniso) {
    // done above
  } else if (!P->aniso) {
    for (auto& g : grad) g.reset();
    tt_round_batch(ctx, batch_view(kr), r, w, tol);              // T, all components in one sweep
    kr = TTBatch();
    for (int alpha = 0; alpha < d; ++alpha) terms[alpha] = item_view(w, alpha);
  } else {
    // component a of A~ e with the constant anisotropic part: a (.) e_a + sum_b B[a][b] e_b (a TT sum in
    // block form, zero entries of B skipped), then T
    for (int alpha = 0; alpha < d; ++alpha) {
      TTView xs[4];
      double sc[4];
      int m = 0;
      xs[m] = item_view(kr, alpha);
      sc[m++] = 1.0;
      for (int beta = 0; beta < d; ++beta) {
        const double bab = P->B[alpha * 3 + beta];
        if (bab == 0.0) continue;
        xs[m] = v;
        xs[m].core[beta] = grad[beta].get();
        sc[m++] = bab;
      }
      TT sum;
      tt_add_many(ctx, xs, sc, m, sum);
      tt_round(ctx, view_of(sum), r, wa[alpha], tol);             // T
      terms[alpha] = view_of(wa[alpha]);
    }
    for (auto& g : grad) g.reset();
    kr = TTBatch();
  }
  // divergence terms: -D_a on carriage a of component a, then the block sum over a
  for (int alpha = 0; alpha < d; ++alpha) {
    double* c = const_cast<double*>(terms[alpha].core[alpha]);
    fibre_operator(ctx, c, c, terms[alpha].r[alpha], terms[alpha].N[alpha], terms[alpha].r[alpha + 1], LRFG_MUL_DERIV,
                   0.0, -1.0, mixed);
  }
  TT acc;
  tt_add_many(ctx, terms, nullptr, d, acc);
  TT sdiv;
  tt_round(ctx, view_of(acc), r, sdiv, tol);                   // T after the sum
  tt_precond(ctx, view_of(sdiv), P->pt, P->pw, r, out, tol, om, mixed, !(om && P->opts.sketch_keep));  // T P~^-1
}

void lr_rhs(lrfg_problem* P, const double* E, TT& out, int rank) {
  lrfg_ctx* ctx = P->ctx;
  TT acc;
  bool have = false;
  for (int alpha = 0; alpha < P->d; ++alpha) {
    if (E[alpha] == 0.0) continue;
    ModeReplaced t;
    // E_a D_a a (Ga: the projection of the modified coefficient on the grid, I* F_M A~)
    mode_replace(ctx, view_of(P->ga ? P->a_down_tt : P->a_tt), alpha, E[alpha], t);
    if (!have) {
      tt_copy(ctx, t.view, acc);
      have = true;
    } else {
      TT s;
      tt_add(ctx, 1.0, nullptr, view_of(acc), 1.0, nullptr, t.view, s);
      acc = std::move(s);
    }
  }
  if (!have) {
    int r[4] = {1, 1, 1, 1};
    tt_alloc(ctx, out, P->d, P->N, r);
    for (int j = 0; j < P->d; ++j) fill(ctx, out.core[j].get(), 0.0, P->N[j]);
    return;
  }
  TTView omv;
  tt_precond(ctx, view_of(acc), P->pt, P->pw, rank, out, P->opts.rank_tol,
             sketch_for(P, rank, omv));                                           // T P~^-1 (one truncation)
}

// Ga: sum over the double grid of A~ |E + e|^2 (exact integration), e the gradient interpolated there
double lr_aeff_ga(lrfg_problem* P, const double* E, const TTView& u) {
  lrfg_ctx* ctx = P->ctx;
  const int d = P->d;
  const TTView a = view_of(P->a_ga_tt);
  int M[3] = {0, 0, 0};
  for (int j = 0; j < d; ++j) M[j] = a.N[j];
  TT ones;
  ones_tt(ctx, d, M, ones);
  double EE = 0.0;
  for (int j = 0; j < d; ++j) EE += E[j] * E[j];
  double val = EE * tt_dot(ctx, a, view_of(ones));
  TTBatch uu;
  tt_ga_map(ctx, u, 1, M, GA_UP, uu);
  DBuf<double> gu[3];
  TTView es[3];
  for (int alpha = 0; alpha < d; ++alpha) {
    DBuf<double> g(ctx->pool, (size_t)u.r[alpha] * u.N[alpha] * u.r[alpha + 1]);
    fibre_operator(ctx, u.core[alpha], g.get(), u.r[alpha], u.N[alpha], u.r[alpha + 1], LRFG_MUL_DERIV, 0.0, 1.0);
    gu[alpha] = DBuf<double>(ctx->pool, (size_t)u.r[alpha] * M[alpha] * u.r[alpha + 1]);
    ga_resample(ctx, g.get(), gu[alpha].get(), u.r[alpha], u.N[alpha], u.r[alpha + 1], M[alpha], GA_UP);
    TTView e = item_view(uu, 0);
    e.core[alpha] = gu[alpha].get();
    es[alpha] = e;
    TT ae;
    tt_hadamard(ctx, a, e, ae);
    if (E[alpha] != 0.0) val += 2.0 * E[alpha] * tt_dot(ctx, view_of(ae), view_of(ones));
    val += tt_dot(ctx, view_of(ae), e);
  }
  if (P->aniso) {
    // the part of B 1~: E.B E <1~, 1> + 2 sum_ab E_b B[b][a] <1~ (.) e_a, 1> + sum_ab B[a][b] <1~ (.) e_a, e_b>
    const TTView one = view_of(P->ones_ga_tt);
    val += quad_form(P->B, E, d) * tt_dot(ctx, one, view_of(ones));
    for (int al = 0; al < d; ++al) {
      TT oe;
      bool made = false;
      for (int be = 0; be < d; ++be) {
        const double bab = P->B[al * 3 + be];
        if (bab == 0.0) continue;
        if (!made) {
          tt_hadamard(ctx, one, es[al], oe);
          made = true;
        }
        val += 2.0 * E[be] * P->B[be * 3 + al] * tt_dot(ctx, view_of(oe), view_of(ones));
        val += bab * tt_dot(ctx, view_of(oe), es[be]);
      }
    }
  }
  return val;
}

double lr_aeff(lrfg_problem* P, const double* E, const TTView& u) {
  if (P->ga) return lr_aeff_ga(P, E, u);
  lrfg_ctx* ctx = P->ctx;
  const double size = (double)grid_size(P->d, P->N);
  TT ones;
  ones_tt(ctx, P->d, P->N, ones);
  double EE = 0.0;
  for (int j = 0; j < P->d; ++j) EE += E[j] * E[j];
  double val = EE * tt_dot(ctx, view_of(P->a_tt), view_of(ones)) / size;
  ModeReplaced e[3];
  for (int alpha = 0; alpha < P->d; ++alpha) {
    mode_replace(ctx, u, alpha, 1.0, e[alpha]);
    TT ae;
    tt_hadamard(ctx, view_of(P->a_tt), e[alpha].view, ae);
    if (E[alpha] != 0.0) val += 2.0 * E[alpha] * tt_dot(ctx, view_of(ae), view_of(ones)) / size;
    val += tt_dot(ctx, view_of(ae), e[alpha].view) / size;
  }
  if (P->aniso) {
    // (E + e).B(E + e) averaged: E.B E + sum_ab B_ab <e_a, e_b> / |N| (e has zero mean)
    val += quad_form(P->B, E, P->d);
    for (int alpha = 0; alpha < P->d; ++alpha)
      for (int beta = 0; beta < P->d; ++beta) {
        const double bab = P->B[alpha * 3 + beta];
        if (bab != 0.0) val += bab * tt_dot(ctx, e[alpha].view, e[beta].view) / size;
      }
  }
  return val;
}

// ---- FULL operator pieces ---------------------------------------------------------------------

// storage of the FULL operator in precision R: coefficient and workspaces
template <typename R> struct FullWork;
template <> struct FullWork<double> {
  const double* a; double2* wc; double* wr;
  explicit FullWork(lrfg_problem* P) : a(P->a_full.get()), wc(P->wc.get()), wr(P->wr.get()) {}
};
template <> struct FullWork<float> {
  const float* a; float2* wc; float* wr;
  explicit FullWork(lrfg_problem* P) : a(P->a_full_f.get()), wc(P->wcf.get()), wr(P->wrf.get()) {
    LRFG_REQUIRE(a && wc && wr, "FP32 workspaces exist only for LRFG_MIXED problems");
  }
};

// Ga operator (FP64): per component, the gradient zero-padded to the double grid, multiplied there by the
// modified coefficient, transformed back and projected on the frequencies of the grid, then grad^*
void full_apply_ga(lrfg_problem* P, const double2* v, double2* out, int precond) {
  lrfg_ctx* ctx = P->ctx;
  const FullGrid& g = P->g;
  const FullGrid& gM = P->gM;
  const double inv = 1.0 / (double)g.n_real;
  for (int alpha = 0; alpha < g.d; ++alpha) {
    half_mul_grad(ctx, g, v, P->wc.get(), alpha, inv);                           // grad^ (1/|N| of Phi^-1)
    half_inject(ctx, g, gM, P->wc.get(), P->wcM.get());                          // I
    full_inverse<double>(ctx, gM, P->wcM.get(), P->a_ga.get(), 1.0, P->wrM.get());  // A~ F_M^-1
    full_forward<double>(ctx, gM, P->wrM.get(), nullptr, 1.0, P->wcM.get());     // F_M
    half_project(ctx, g, gM, P->wcM.get(), P->wc.get());                         // I*
    half_acc_div(ctx, g, (const double2*)P->wc.get(), out, alpha, 1.0, alpha == 0,
                 precond && alpha == g.d - 1 && !P->aniso);                       // grad^*
  }
  // constant anisotropic part: its exact integral is the grid's, grad^* F B F^-1 grad^ = 4 pi^2 k.B k, on the
  // scale of the double-grid product above: A~ carries the double grid's quadrature weight 1 / |M| (a constant
  // material c gives c / |M| times the GaNi operator), so B enters as B / |M|
  if (P->aniso) {
    double Bs[9];
    for (int i = 0; i < 9; ++i) Bs[i] = P->B[i] / (double)gM.n_real;
    half_acc_aniso(ctx, g, v, out, Bs, precond);
  }
}

template <typename R>
void full_apply(lrfg_problem* P, const typename CplxOf<R>::T* v, typename CplxOf<R>::T* out, int precond) {
  if constexpr (std::is_same<R, double>::value) {
    if (P->ga) {
      full_apply_ga(P, v, out, precond);
      return;
    }
  }
  lrfg_ctx* ctx = P->ctx;
  const FullGrid& g = P->g;
  FullWork<R> w(P);
  const double inv = 1.0 / (double)g.n_real;
  for (int alpha = 0; alpha < g.d; ++alpha) {
    // grad^ (with 1/|N| of Phi^-1) and F^-1 on the complex axes, then on the rows fused with A~ and F there,
    // then F on the complex axes and grad^* (P~^-1 after the last component)
    half_grad_fibres_inverse(ctx, g, v, w.wc, alpha, inv);
    full_rows_mul<R>(ctx, g, w.wc, w.a, R(1));
    half_fibres_forward_div(ctx, g, w.wc, out, alpha, 1.0, alpha == 0, precond && alpha == g.d - 1 && !P->aniso);
  }
  // constant anisotropic part: grad^* F B F^-1 grad^ is the multiplier 4 pi^2 k.B k
  if (P->aniso) half_acc_aniso(ctx, g, v, out, P->B, precond);
}

template <typename R>
void full_rhs(lrfg_problem* P, const double* E, typename CplxOf<R>::T* b, int precond) {
  lrfg_ctx* ctx = P->ctx;
  const FullGrid& g = P->g;
  if constexpr (std::is_same<R, double>::value) {
    if (P->ga) {  // - grad^* I* F_M A~ E
      full_forward<double>(ctx, P->gM, P->a_ga.get(), nullptr, 1.0, P->wcM.get());
      half_project(ctx, g, P->gM, P->wcM.get(), P->wc.get());
      for (int alpha = 0; alpha < g.d; ++alpha)
        half_acc_div(ctx, g, (const double2*)P->wc.get(), b, alpha, -E[alpha], alpha == 0,
                     precond && alpha == g.d - 1);
      return;
    }
  }
  FullWork<R> w(P);
  full_forward<R>(ctx, g, w.a, nullptr, R(1), w.wc);
  for (int alpha = 0; alpha < g.d; ++alpha)
    half_acc_div(ctx, g, (const typename CplxOf<R>::T*)w.wc, b, alpha, -E[alpha], alpha == 0,
                 precond && alpha == g.d - 1);
}

double full_aeff(lrfg_problem* P, const double* E, const double2* v) {
  lrfg_ctx* ctx = P->ctx;
  const FullGrid& g = P->g;
  DBuf<double> acc(ctx->pool, 1);
  if (P->ga) {
    // exact integration: sum over the double grid of A~ |E + e|^2, e the gradient there
    for (int alpha = 0; alpha < g.d; ++alpha) {
      half_mul_grad(ctx, g, v, P->wc.get(), alpha, 1.0 / (double)g.n_real);
      half_inject(ctx, g, P->gM, P->wc.get(), P->wcM.get());
      full_inverse<double>(ctx, P->gM, P->wcM.get(), nullptr, 1.0, P->wrM.get());
      energy_sum(ctx, P->gM, (const double*)P->wrM.get(), P->a_ga.get(), E[alpha], acc.get(), alpha > 0);
    }
    DBuf<double> accB(ctx->pool, 1);
    if (P->aniso) aniso_energy_sum(ctx, g, v, P->B, accB.get(), 0);  // sum over the grid of e.B e
    double h = 0.0, hb = 0.0;
    LRFG_CUDA(cudaMemcpyAsync(&h, acc.get(), sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
    if (P->aniso) LRFG_CUDA(cudaMemcpyAsync(&hb, accB.get(), sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
    LRFG_CUDA(cudaStreamSynchronize(ctx->stream));
    // the stored coefficient is (|N| / |M|) A~
    double val = h * (double)P->gM.n_real / (double)g.n_real;
    if (P->aniso) val += hb / (double)g.n_real + quad_form(P->B, E, g.d);
    return val;
  }
  for (int alpha = 0; alpha < g.d; ++alpha) {
    half_mul_grad(ctx, g, v, P->wc.get(), alpha, 1.0 / (double)g.n_real);
    full_inverse<double>(ctx, g, P->wc.get(), nullptr, 1.0, P->wr.get());
    energy_sum(ctx, g, (const double*)P->wr.get(), P->a_full.get(), E[alpha], acc.get(), alpha > 0);
  }
  // (E + e).B(E + e) summed over the grid: |N| E.B E + sum_x e.B e (e has zero mean)
  if (P->aniso) aniso_energy_sum(ctx, g, v, P->B, acc.get(), 1);
  double h = 0.0;
  LRFG_CUDA(cudaMemcpyAsync(&h, acc.get(), sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
  LRFG_CUDA(cudaStreamSynchronize(ctx->stream));
  if (P->aniso) h += (double)g.n_real * quad_form(P->B, E, g.d);
  return h / (double)g.n_real;
}

void new_field(lrfg_ctx* ctx, lrfg_format fmt, int d, const int* N, lrfg_field** out) {
  lrfg_field* f = new lrfg_field();
  ctx->live_objects++;
  f->ctx = ctx;
  f->fmt = fmt;
  f->d = d;
  for (int j = 0; j < 3; ++j) f->N[j] = j < d ? N[j] : 0;
  *out = f;
}

// undo new_field() for a field that never reached the caller
void discard_field(lrfg_field* f) {
  f->ctx->live_objects--;
  delete f;
}

void check_field(const lrfg_problem* P, const lrfg_field* f) {
  LRFG_REQUIRE(f != nullptr, "null field");
  LRFG_REQUIRE(f->fmt == P->opts.fmt || (tucker_like(f->fmt) && tucker_like(P->opts.fmt)),
               "field format does not match the problem");
  LRFG_REQUIRE(f->d == P->d, "field order does not match the problem");
  for (int j = 0; j < P->d; ++j) LRFG_REQUIRE(f->N[j] == P->N[j], "field grid does not match the problem");
}

void apply_into(lrfg_problem* P, const lrfg_field* in, lrfg_field* out) {
  check_field(P, in);
  if (P->opts.fmt == LRFG_FULL) {
    if (!out->half.get()) out->half = DBuf<double2>(P->ctx->pool, P->g.n_half);
    if (P->opts.prec == LRFG_MIXED) {
      // FP32 operator between FP64 fields
      DBuf<float2> xi(P->ctx->pool, P->g.n_half), xo(P->ctx->pool, P->g.n_half);
      convert(P->ctx, (const double2*)in->half.get(), xi.get(), P->g.n_half);
      full_apply<float>(P, xi.get(), xo.get(), 1);
      convert(P->ctx, (const float2*)xo.get(), out->half.get(), P->g.n_half);
    } else {
      full_apply<double>(P, in->half.get(), out->half.get(), 1);
    }
  } else if (tucker_like(P->opts.fmt)) {
    TK res;
    tk_apply(P->ctx, tk_view(P->a_tk), tk_view(in->tk), P->pt, P->pw, P->opts.rank, res, P->opts.rank_tol, aniso_b(P),
             tk_ga(P));
    out->tk = std::move(res);
  } else {
    TT res;
    lr_apply(P, view_of(in->tt), res, P->opts.rank, P->opts.prec == LRFG_MIXED);
    out->tt = std::move(res);
  }
}

// Preconditioned CG on the full grid (Sec. 3.3, Sec. 4) with vectors stored in precision R; the
// scalars (inner products, step lengths) are FP64 device values, the residual test runs on the host.
template <typename R>
void solve_full(lrfg_problem* P, const double* E, lrfg_result* res, lrfg_field** u_out) {
  using V = typename CplxOf<R>::T;
  lrfg_ctx* ctx = P->ctx;
  const FullGrid& g = P->g;
  const long long n = g.n_half;
  DBuf<V> u(ctx->pool, n), r(ctx->pool, n), z(ctx->pool, n), p(ctx->pool, n), q(ctx->pool, n);
  DBuf<double> s(ctx->pool, 6);  // rz, pq, zz, rz_new, alpha, beta
  double* d_rz = s.get();
  double* d_pq = s.get() + 1;
  double* d_zz = s.get() + 2;
  double* d_rzn = s.get() + 3;
  double* d_alpha = s.get() + 4;
  double* d_beta = s.get() + 5;
  LRFG_CUDA(cudaMemsetAsync(u.get(), 0, sizeof(V) * n, ctx->stream));
  full_rhs<R>(P, E, r.get(), 0);
  half_precond(ctx, g, (const V*)r.get(), z.get());
  LRFG_CUDA(cudaMemcpyAsync(p.get(), z.get(), sizeof(V) * n, cudaMemcpyDeviceToDevice, ctx->stream));
  half_dot(ctx, g, (const V*)r.get(), (const V*)z.get(), d_rz);
  half_dot(ctx, g, (const V*)z.get(), (const V*)z.get(), d_zz);
  double zz0 = 0.0;
  LRFG_CUDA(cudaMemcpyAsync(&zz0, d_zz, sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
  LRFG_CUDA(cudaStreamSynchronize(ctx->stream));
  const double nb = std::sqrt(zz0);
  int it = 0;
  double rel = nb > 0.0 ? 1.0 : 0.0;
  int applies = 0;
  while (nb > 0.0 && it < P->opts.maxit) {
    full_apply<R>(P, p.get(), q.get(), 0);
    ++applies;
    half_dot(ctx, g, (const V*)p.get(), (const V*)q.get(), d_pq, d_rz, d_alpha, 1);  // alpha = rz / pq
    pcg_update(ctx, g, u.get(), r.get(), (const V*)p.get(), (const V*)q.get(), z.get(), (const double*)d_alpha);
    half_dot(ctx, g, (const V*)z.get(), (const V*)z.get(), d_zz);
    ++it;
    double zz = 0.0;
    LRFG_CUDA(cudaMemcpyAsync(&zz, d_zz, sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
    LRFG_CUDA(cudaStreamSynchronize(ctx->stream));
    rel = std::sqrt(std::max(zz, 0.0)) / nb;
    if (rel <= P->opts.tol) break;
    half_dot(ctx, g, (const V*)r.get(), (const V*)z.get(), d_rzn, d_rz, d_beta, 2);  // beta = rz_new / rz
    pcg_direction(ctx, g, p.get(), (const V*)z.get(), (const double*)d_beta);
    LRFG_CUDA(cudaMemcpyAsync(d_rz, d_rzn, sizeof(double), cudaMemcpyDeviceToDevice, ctx->stream));
  }
  res->iters = it;
  res->rel_resid = rel;
  res->converged = rel <= P->opts.tol ? 1 : 0;
  res->applies = applies;
  for (int j = 0; j < 4; ++j) res->ranks[j] = 1;
  // the solution is handed out, and A_eff evaluated, in FP64
  DBuf<double2> u64;
  if constexpr (std::is_same<R, double>::value) {
    u64 = std::move(u);
  } else {
    u64 = DBuf<double2>(ctx->pool, n);
    convert(ctx, (const V*)u.get(), u64.get(), n);
  }
  res->Aeff = full_aeff(P, E, u64.get());
  if (u_out) {
    lrfg_field* f;
    new_field(ctx, LRFG_FULL, P->d, P->N, &f);
    f->half = std::move(u64);
    *u_out = f;
  }
}

// rank cap of a grid coefficient's TT compression: opts.coeff_rank, or the solution rank when 0
int coeff_rank(const lrfg_opts& o) { return o.coeff_rank > 0 ? o.coeff_rank : o.rank; }

void solve_tucker(lrfg_problem* P, const double* E, lrfg_result* res, lrfg_field** u_out) {
  TK best;
  const TKSolveResult r = tk_solve(P->ctx, tk_view(P->a_tk), E, P->pt, P->pw, P->opts.rank, P->opts.tol,
                                   P->opts.maxit, P->opts.stop_on_increase, best, P->opts.rank_tol, aniso_b(P),
                                   P->opts.rank_start, P->opts.rank_step, tk_ga(P));
  res->iters = r.iters;
  res->rel_resid = r.rel_resid;
  res->converged = r.rel_resid <= P->opts.tol ? 1 : 0;
  res->applies = r.applies;
  res->Aeff = r.Aeff;
  for (int j = 0; j < 4; ++j) res->ranks[j] = j < P->d ? best.r[j] : 1;
  if (u_out) {
    lrfg_field* f;
    new_field(P->ctx, P->opts.fmt, P->d, P->N, &f);
    f->tk = std::move(best);
    *u_out = f;
  }
}

// Minimal-residual iteration with truncation (Sec. 3.3), stopped when the residual fails to decrease
// (Sec. 4.3), at tol or maxit; the iterate of smallest residual is returned.  Rank adaptation (the solver
// Sec. 4.3 proposes; opts.rank_start > 0): every T truncates to the current rank r_c, starting at
// rank_start; when the residual fails to decrease below the cap opts.rank, r_c rises by rank_step, the
// right-hand side is rebuilt at r_c and the iteration restarts from the best iterate, whose residual is
// recomputed at r_c and becomes the new reference.  LRFG_MIXED: the step q = C r uses the mixed-precision operator,
// the residual r = T(b - C u) the FP64 one, so the iteration is a defect correction whose fixed point is the FP64
// solution (the step length only has to reduce the FP64 residual).
void solve_tt(lrfg_problem* P, const double* E, lrfg_result* res, lrfg_field** u_out) {
  lrfg_ctx* ctx = P->ctx;
  const int cap = P->opts.rank;
  const bool adapt = P->opts.rank_start > 0;
  int rc = adapt ? std::min(P->opts.rank_start, cap) : cap;
  const double rtol = P->opts.rank_tol;
  TT b;
  lr_rhs(P, E, b, rc);
  double nb = std::sqrt(std::max(tt_dot(ctx, view_of(b), view_of(b)), 0.0));
  TT u, r, best_u;
  bool u_zero = true, best_zero = true;
  double best = INFINITY;
  int best_it = 0, it = 0, applies = 0;
  tt_copy(ctx, view_of(b), r);
  // r <- T(b - C u) at the current rank
  auto residual = [&]() {
    TT cu, diff, rn;
    lr_apply(P, view_of(u), cu, rc);
    ++applies;
    tt_add(ctx, 1.0, nullptr, view_of(b), -1.0, nullptr, view_of(cu), diff);
    tt_round(ctx, view_of(diff), rc, rn, rtol);
    r = std::move(rn);
  };
  int since_best = 0;  // iterations since the last new smallest residual (stop_on_increase > 1: the patience)
  int cap_steps = 0;   // steps taken at the cap (the tolerance ends a rank-adapting solve only after one)
  while (nb > 0.0) {
    double nr = std::sqrt(std::max(tt_dot(ctx, view_of(r), view_of(r)), 0.0)) / nb;
    if (it == 0 && u_zero) nr = 1.0;  // r = b
    const bool improved = nr < best;
    if (improved) {
      best = nr;
      best_it = it;
      best_zero = u_zero;
      since_best = 0;
      if (!u_zero) tt_copy(ctx, view_of(u), best_u);
    }
    if (adapt && rc < cap && (!improved || nr <= P->opts.tol)) {
      // stagnation, or the tolerance met, below the cap (the residual there is truncated at the lower rank):
      // raise the rank and restart from the best iterate, again while the restarted residual is within it
      do {
        rc = std::min(cap, rc + std::max(1, P->opts.rank_step));
        TT nbv;
        lr_rhs(P, E, nbv, rc);
        b = std::move(nbv);
        nb = std::sqrt(std::max(tt_dot(ctx, view_of(b), view_of(b)), 0.0));
        u_zero = best_zero;
        if (u_zero) {
          tt_copy(ctx, view_of(b), r);
        } else {
          tt_copy(ctx, view_of(best_u), u);
          residual();
        }
        nr = u_zero ? 1.0 : std::sqrt(std::max(tt_dot(ctx, view_of(r), view_of(r)), 0.0)) / nb;
        best = nr;
        since_best = 0;
      } while (rc < cap && nr <= P->opts.tol);
    } else if (!improved && P->opts.stop_on_increase && ++since_best >= P->opts.stop_on_increase) {
      break;  // (at the cap the rank-adapting iteration stops as the fixed-rank one)
    }
    if ((nr <= P->opts.tol && (!adapt || (rc >= cap && cap_steps > 0))) || it >= P->opts.maxit) break;
    TT q;
    lr_apply(P, view_of(r), q, rc, P->opts.prec == LRFG_MIXED);  // (mixed: the search direction's operator)
    ++applies;
    const double qq = tt_dot(ctx, view_of(q), view_of(q));
    if (qq == 0.0) break;
    const double omega = tt_dot(ctx, view_of(q), view_of(r)) / qq;
    TT un;
    if (u_zero) {
      TT scaled;
      tt_copy(ctx, view_of(r), scaled);
      axpby(ctx, (long long)scaled.core_elems(0), omega, r.core[0].get(), 0.0, scaled.core[0].get());
      tt_round(ctx, view_of(scaled), rc, un, rtol);
    } else {
      TT s;
      tt_add(ctx, 1.0, nullptr, view_of(u), omega, nullptr, view_of(r), s);
      tt_round(ctx, view_of(s), rc, un, rtol);
    }
    u = std::move(un);
    u_zero = false;
    ++it;
    if (rc >= cap) ++cap_steps;
    residual();
  }
  if (best_zero || !best_u.d) {
    // the best iterate is u_0 = 0
    int rr[4] = {1, 1, 1, 1};
    best_u = TT();
    tt_alloc(ctx, best_u, P->d, P->N, rr);
    for (int j = 0; j < P->d; ++j) fill(ctx, best_u.core[j].get(), 0.0, P->N[j]);
  }
  res->iters = best_it;
  res->rel_resid = nb > 0.0 ? best : 0.0;
  res->converged = res->rel_resid <= P->opts.tol ? 1 : 0;
  res->applies = applies;
  for (int j = 0; j < 4; ++j) res->ranks[j] = best_u.r[j];
  res->Aeff = lr_aeff(P, E, view_of(best_u));
  if (u_out) {
    lrfg_field* f;
    new_field(ctx, LRFG_TT, P->d, P->N, &f);
    f->tt = std::move(best_u);
    *u_out = f;
  }
}

// ---- several right-hand sides of one TT problem in lockstep --------------------------------------

// whether solve_tt_many can run the problem's options (isotropic GaNi TT at a fixed rank)
bool lockstep_ok(const lrfg_problem* P) {
  return P->opts.fmt == LRFG_TT && !P->ga && !P->aniso && P->opts.rank_tol == 0.0 && P->d >= 2;
}

// The operator of lr_apply on nb items at once (items of identical ranks, stored item after item): the gradient,
// material, divergence, sum and preconditioner stages each take one launch sequence for all items.  Item b's
// material product takes the coefficient of problem Ps[b] (Ps null: P's for every item); the problems share P's
// grid, options, coefficient ranks, exponential sum and sketch.
void apply_batch(lrfg_problem* P, const TTBatchView& v, TTBatch& out, int r, bool mixed = false,
                 lrfg_problem* const* Ps = nullptr) {
  lrfg_ctx* ctx = P->ctx;
  const int d = P->d, nb = v.nb;
  const TTView a = view_of(P->a_tt);
  auto coeff_core = [&](int b, int j) -> const double* { return Ps ? Ps[b]->a_tt.core[j].get() : a.core[j]; };
  TTView omv;
  const TTView* om = sketch_for(P, r, omv);
  // gradient carriages D_a v_a of every item (items contiguous: one launch per mode)
  DBuf<double> grad[3];
  for (int al = 0; al < d; ++al) {
    grad[al] = DBuf<double>(ctx->pool, v.elems(al) * nb);
    fibre_operator(ctx, v.core[al], grad[al].get(), (long long)v.r[al] * nb, v.N[al], v.r[al + 1], LRFG_MUL_DERIV,
                   0.0, 1.0, mixed);
  }
  // material products, item (al, b) = a (.) e_al of item b at al * nb + b, truncated together
  int rk[4];
  for (int j = 0; j <= d; ++j) rk[j] = a.r[j] * v.r[j];
  const int m = d * nb;
  TTBatch w;
  if (om) {
    LRFG_REQUIRE(m <= kMaxSketchItems, "too many right-hand sides for one lockstep batch (%d)", nb);
    SketchSource z;
    z.kind = SketchSource::KHATRI_RAO;
    z.d = d;
    z.nb = m;
    z.x = a;
    for (int j = 0; j < 3; ++j) z.N[j] = v.N[j];
    for (int j = 0; j <= d; ++j) {
      z.s[j] = rk[j];
      z.ry[j] = v.r[j];
    }
    for (int al = 0; al < d; ++al)
      for (int b = 0; b < nb; ++b)
        for (int j = 0; j < d; ++j) {
          z.y[j][al * nb + b] = (j == al ? grad[j].get() : v.core[j]) + (size_t)b * v.elems(j);
          if (Ps) z.xi[j][al * nb + b] = coeff_core(b, j);
        }
    tt_round_sketch(ctx, z, *om, r, w, 0.0, mixed, !P->opts.sketch_keep);
  } else {
    TTBatch kr;
    ttb_alloc(ctx, kr, d, v.N, rk, m);
    for (int al = 0; al < d; ++al)
      for (int b = 0; b < nb; ++b)
        for (int j = 0; j < d; ++j)
          khatri_rao(ctx, coeff_core(b, j), a.r[j], a.N[j], a.r[j + 1],
                     (j == al ? grad[j].get() : v.core[j]) + (size_t)b * v.elems(j), v.r[j], v.r[j + 1],
                     kr.core[j].get() + (size_t)(al * nb + b) * kr.elems(j));
    tt_round_batch(ctx, batch_view(kr), r, w, 0.0);
  }
  for (auto& g : grad) g.reset();
  // divergence: -D_al on carriage al of the items of component al (contiguous), then the block sum over al
  TTBatchView terms[3];
  for (int al = 0; al < d; ++al) {
    double* c = w.core[al].get() + (size_t)al * nb * w.elems(al);
    fibre_operator(ctx, c, c, (long long)w.r[al] * nb, w.N[al], w.r[al + 1], LRFG_MUL_DERIV, 0.0, -1.0, mixed);
    TTBatchView t = batch_view(w);
    t.nb = nb;
    for (int j = 0; j < d; ++j) t.core[j] = w.core[j].get() + (size_t)al * nb * w.elems(j);
    terms[al] = t;
  }
  TTBatch acc;
  ttb_add_many(ctx, terms, d, nullptr, nullptr, acc);
  w = TTBatch();
  TTBatch sdiv;
  tt_round_batch(ctx, batch_view(acc), r, sdiv, 0.0);          // T after the sum
  acc = TTBatch();
  ttb_precond(ctx, batch_view(sdiv), P->pt, P->pw, r, out, 0.0, om, mixed, !(om && P->opts.sketch_keep));
}

// copy of item b of `src` into item b of `dst` (same shapes)
void ttb_copy_item(lrfg_ctx* ctx, const TTBatch& src, TTBatch& dst, int b) {
  for (int j = 0; j < src.d; ++j)
    LRFG_CUDA(cudaMemcpyAsync(dst.core[j].get() + (size_t)b * dst.elems(j), src.core[j].get() + (size_t)b * src.elems(j),
                              sizeof(double) * src.elems(j), cudaMemcpyDeviceToDevice, ctx->stream));
}

// The minimal-residual iteration of solve_tt for nb right-hand sides E_i (row i of E, d entries each) in
// lockstep: the same steps, the operator applied to all residuals (and iterates) in one launch sequence.  Each
// item keeps its own step length, best iterate and stopping test; items that have stopped ride along until
// the last one stops, their results frozen.  The results equal solve_tt's up to the rounding order of the
// batched products.
// Rank adaptation in lockstep (opts.rank_start > 0): the items share one current rank.  An item whose residual
// fails to decrease, or meets the tolerance, below the cap is frozen (its best iterate kept, its later iterates
// ignored, its iteration count not advanced); once every unfinished item is frozen the common rank rises by
// rank_step (to the cap), the
// right-hand sides are rebuilt at it and every unfinished item restarts from its best iterate with its residual
// recomputed.  Each item thus follows the rank-adapting iteration of solve_tt, only waiting for the others before
// a rise.  At the cap a failure to decrease ends the item, as there.
// Ps (null: P for every item): item i solves problem Ps[i] (its own coefficient; grid, coefficient ranks and options
// those of P), so several microstructures of one shape share every launch.
void solve_tt_many(lrfg_problem* P, const double* E, int nb, lrfg_result* res, lrfg_problem* const* Ps = nullptr) {
  lrfg_ctx* ctx = P->ctx;
  auto prob = [&](int i) { return Ps ? Ps[i] : P; };
  const int d = P->d, cap = P->opts.rank;
  const bool adapt = P->opts.rank_start > 0;
  int rk = adapt ? std::min(P->opts.rank_start, cap) : cap;
  // trains of possibly different ranks packed into one batch at the largest ranks (zero blocks elsewhere);
  // null entries are zero trains
  auto pack = [&](const std::vector<const TT*>& xs, TTBatch& out) {
    int rr[4] = {1, 1, 1, 1};
    for (const TT* x : xs)
      if (x)
        for (int j = 0; j <= d; ++j) rr[j] = std::max(rr[j], x->r[j]);
    ttb_alloc(ctx, out, d, P->N, rr, nb);
    for (int i = 0; i < nb; ++i) {
      const TT* x = xs[i];
      const bool same = x && std::equal(x->r, x->r + d + 1, rr);
      for (int j = 0; j < d; ++j) {
        double* dst = out.core[j].get() + (size_t)i * out.elems(j);
        if (same) {
          LRFG_CUDA(cudaMemcpyAsync(dst, x->core[j].get(), sizeof(double) * out.elems(j), cudaMemcpyDeviceToDevice,
                                    ctx->stream));
          continue;
        }
        fill(ctx, dst, 0.0, (long long)out.elems(j));
        if (x) tt_embed(ctx, x->core[j].get(), x->r[j], P->N[j], x->r[j + 1], dst, rr[j], rr[j + 1], 0, 0);
      }
    }
  };
  DBuf<double> dots(ctx->pool, (size_t)2 * nb);
  std::vector<double> h(2 * nb);
  auto host_dots = [&](const TTBatch& x, const TTBatch& y, const TTBatch* x2, const TTBatch* y2) {
    ttb_dot_device(ctx, batch_view(x), batch_view(y), dots.get());
    if (x2) ttb_dot_device(ctx, batch_view(*x2), batch_view(*y2), dots.get() + nb);
    LRFG_CUDA(cudaMemcpyAsync(h.data(), dots.get(), sizeof(double) * (x2 ? 2 : 1) * nb, cudaMemcpyDeviceToHost,
                              ctx->stream));
    LRFG_CUDA(cudaStreamSynchronize(ctx->stream));
  };
  // right-hand sides at the current rank (item by item), packed, and their norms
  TTBatch b;
  std::vector<double> nb2(nb);
  auto build_rhs = [&]() {
    std::vector<TT> bs(nb);
    std::vector<const TT*> ptr(nb);
    for (int i = 0; i < nb; ++i) {
      lr_rhs(prob(i), E + (size_t)i * d, bs[i], rk);
      ptr[i] = &bs[i];
    }
    pack(ptr, b);
    host_dots(b, b, nullptr, nullptr);
    for (int i = 0; i < nb; ++i) nb2[i] = std::sqrt(std::max(h[i], 0.0));
  };
  build_rhs();
  std::vector<double> best(nb, INFINITY);
  std::vector<int> best_it(nb, 0), active(nb, 1), best_zero(nb, 1), since_best(nb, 0), frozen(nb, 0), its(nb, 0);
  std::vector<int> cap_steps(nb, 0);  // steps each item took at the cap
  std::vector<double> omega(nb);
  DBuf<double> om_dev(ctx->pool, (size_t)nb);
  TTBatch u, r;
  std::vector<TT> best_u(nb);  // each item's best iterate (its ranks may differ from the current ones)
  bool u_zero = true;
  int applies = 0;
  // r = b
  ttb_alloc(ctx, r, d, P->N, b.r, nb);
  for (int i = 0; i < nb; ++i) ttb_copy_item(ctx, b, r, i);
  auto any_active = [&]() { return std::any_of(active.begin(), active.end(), [](int a) { return a != 0; }); };
  // r <- T(b - C u) and the relative residuals
  std::vector<double> nr(nb, 1.0);
  auto residual = [&]() {
    TTBatch cu;
    apply_batch(P, batch_view(u), cu, rk, false, Ps);
    ++applies;
    TTBatchView t[2] = {batch_view(b), batch_view(cu)};
    const double hs[2] = {1.0, -1.0};
    TTBatch diff;
    ttb_add_many(ctx, t, 2, hs, nullptr, diff);
    TTBatch rn;
    tt_round_batch(ctx, batch_view(diff), rk, rn, 0.0);
    r = std::move(rn);
    host_dots(r, r, nullptr, nullptr);
    for (int i = 0; i < nb; ++i) nr[i] = nb2[i] > 0.0 ? std::sqrt(std::max(h[i], 0.0)) / nb2[i] : 0.0;
  };
  for (int i = 0; i < nb; ++i)
    if (nb2[i] == 0.0) { active[i] = 0; best[i] = 0.0; }
  bool restarted = false;
  while (true) {
    for (int i = 0; i < nb; ++i) {
      if (!active[i] || frozen[i]) continue;
      bool improved = false;
      if (restarted) {
        // the recomputed residual at the new rank is the new reference
        best[i] = nr[i];
      } else if (nr[i] < best[i]) {
        improved = true;
        best[i] = nr[i];
        best_it[i] = its[i];
        best_zero[i] = u_zero ? 1 : 0;
        since_best[i] = 0;
        if (!u_zero) tt_copy(ctx, item_view(u, i), best_u[i]);
      }
      const bool failed = !restarted && !improved;
      if (adapt && rk < cap && (failed || nr[i] <= P->opts.tol)) {
        // stagnation, or the tolerance met, below the cap: wait for the next rise
        frozen[i] = 1;
        continue;
      }
      // at the cap (or at a fixed rank) the stop rule on a rise of the residual
      if (failed && P->opts.stop_on_increase && ++since_best[i] >= P->opts.stop_on_increase) {
        active[i] = 0;
        continue;
      }
      if ((nr[i] <= P->opts.tol && (!adapt || cap_steps[i] > 0)) || its[i] >= P->opts.maxit) active[i] = 0;
    }
    restarted = false;
    if (!any_active()) break;
    bool all_frozen = true;
    for (int i = 0; i < nb; ++i)
      if (active[i] && !frozen[i]) all_frozen = false;
    if (all_frozen) {
      // raise the common rank; every unfinished item restarts from its best iterate
      rk = std::min(cap, rk + std::max(1, P->opts.rank_step));
      build_rhs();
      std::vector<const TT*> ptr(nb, nullptr);
      bool all_zero = true;
      for (int i = 0; i < nb; ++i) {
        frozen[i] = 0;
        since_best[i] = 0;
        if (!best_zero[i] && best_u[i].d) {
          ptr[i] = &best_u[i];
          all_zero = false;
        }
      }
      if (all_zero) {
        u_zero = true;
        u = TTBatch();
        ttb_alloc(ctx, r, d, P->N, b.r, nb);
        for (int i = 0; i < nb; ++i) ttb_copy_item(ctx, b, r, i);
        std::fill(nr.begin(), nr.end(), 1.0);
      } else {
        u_zero = false;
        pack(ptr, u);
        residual();
        for (int i = 0; i < nb; ++i)
          if (!ptr[i]) nr[i] = 1.0;  // u = 0: r = b (up to the rounding of b at its own rank)
      }
      restarted = true;
      continue;
    }
    // q = C r; omega = (q, r) / (q, q)
    TTBatch q;
    apply_batch(P, batch_view(r), q, rk, P->opts.prec == LRFG_MIXED, Ps);
    ++applies;
    host_dots(q, q, &q, &r);
    for (int i = 0; i < nb; ++i) omega[i] = (h[i] > 0.0) ? h[nb + i] / h[i] : 0.0;
    LRFG_CUDA(cudaMemcpyAsync(om_dev.get(), omega.data(), sizeof(double) * nb, cudaMemcpyHostToDevice, ctx->stream));
    // u <- T(u + omega r)
    TTBatch sum;
    if (u_zero) {
      TTBatchView t = batch_view(r);
      const double* ds[1] = {om_dev.get()};
      ttb_add_many(ctx, &t, 1, nullptr, ds, sum);
    } else {
      TTBatchView t[2] = {batch_view(u), batch_view(r)};
      const double* ds[2] = {nullptr, om_dev.get()};
      ttb_add_many(ctx, t, 2, nullptr, ds, sum);
    }
    TTBatch un;
    tt_round_batch(ctx, batch_view(sum), rk, un, 0.0);
    u = std::move(un);
    u_zero = false;
    for (int i = 0; i < nb; ++i)
      if (active[i] && !frozen[i]) {
        ++its[i];
        if (rk >= cap) ++cap_steps[i];
      }
    residual();
  }
  for (int i = 0; i < nb; ++i) {
    lrfg_result& o = res[i];
    o = lrfg_result{};
    o.iters = best_it[i];
    o.rel_resid = nb2[i] > 0.0 ? best[i] : 0.0;
    o.converged = o.rel_resid <= P->opts.tol ? 1 : 0;
    o.applies = applies;
    if (best_zero[i] || !best_u[i].d) {
      TT z;
      int r1[4] = {1, 1, 1, 1};
      tt_alloc(ctx, z, d, P->N, r1);
      for (int j = 0; j < d; ++j) fill(ctx, z.core[j].get(), 0.0, P->N[j]);
      o.Aeff = lr_aeff(prob(i), E + (size_t)i * d, view_of(z));
      for (int j = 0; j < 4; ++j) o.ranks[j] = 1;
    } else {
      o.Aeff = lr_aeff(prob(i), E + (size_t)i * d, view_of(best_u[i]));
      for (int j = 0; j < 4; ++j) o.ranks[j] = j <= d ? best_u[i].r[j] : 1;
    }
  }
}

}  // namespace

// ------------------------------------------------------------------------------------------------
// C ABI
// ------------------------------------------------------------------------------------------------
extern "C" {

const char* lrfg_strerror(lrfg_status st) {
  switch (st) {
    case LRFG_OK: return "ok";
    case LRFG_EINVAL: return "invalid argument";
    case LRFG_ENOMEM: return "out of device memory (or over the context's budget)";
    case LRFG_ENOCONV: return "iteration cap reached before the tolerance";
    case LRFG_ECUDA: return "CUDA runtime error";
    case LRFG_ETIMEOUT: return "device-side wait timed out";
    case LRFG_ENOTSUP: return "not supported";
  }
  return "unknown status";
}

const char* lrfg_last_error(const lrfg_ctx* ctx) { return ctx ? ctx->last_error.c_str() : "null context"; }

lrfg_status lrfg_create(lrfg_ctx** out, int device, void* stream, size_t budget) {
  if (!out) return LRFG_EINVAL;
  *out = nullptr;
  lrfg_ctx* ctx = new (std::nothrow) lrfg_ctx();
  if (!ctx) return LRFG_ENOMEM;
  ctx->device = device;
  lrfg_status st = guard(ctx, [&] {
    int n = 0;
    LRFG_CUDA(cudaGetDeviceCount(&n));
    LRFG_REQUIRE(device >= 0 && device < n, "device %d out of range (%d devices)", device, n);
    LRFG_CUDA(cudaSetDevice(device));
    LRFG_CUDA(cudaDeviceGetAttribute(&ctx->num_sms, cudaDevAttrMultiProcessorCount, device));
    LRFG_CUDA(cudaDeviceGetAttribute(&ctx->max_smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, device));
    ctx->stream = (cudaStream_t)stream;  // NULL: the legacy default stream
    ctx->pool = new DevicePool(budget);
    LRFG_CUDA(cudaMalloc(&ctx->work_dev, sizeof(double) * 2 * KC_COUNT));
    LRFG_CUDA(cudaMemsetAsync(ctx->work_dev, 0, sizeof(double) * 2 * KC_COUNT, ctx->stream));
    const size_t ncnt = (size_t)kSplitKCounters * (1 + kSplitKGroups);
    LRFG_CUDA(cudaMalloc(&ctx->splitk_cnt, sizeof(unsigned int) * ncnt));
    LRFG_CUDA(cudaMemsetAsync(ctx->splitk_cnt, 0, sizeof(unsigned int) * ncnt, ctx->stream));
    LRFG_CUDA(cudaStreamSynchronize(ctx->stream));
  });
  if (st != LRFG_OK) {
    delete ctx;
    return st;
  }
  *out = ctx;
  return LRFG_OK;
}

lrfg_status lrfg_destroy(lrfg_ctx* ctx) {
  if (!ctx) return LRFG_EINVAL;
  if (ctx->live_objects > 0) {
    ctx->last_error = "free every problem and field of this context before destroying it";
    return LRFG_EINVAL;
  }
  cudaSetDevice(ctx->device);
  if (ctx->stream) cudaStreamSynchronize(ctx->stream);
  delete ctx->pool;
  if (ctx->work_dev) cudaFree(ctx->work_dev);
  if (ctx->splitk_cnt) cudaFree(ctx->splitk_cnt);
  for (auto& kv : ctx->twiddles) {
    cudaFree(kv.second.W);
    if (kv.second.Wf) cudaFree(kv.second.Wf);
  }
  for (auto& p : ctx->pending) {
    cudaEventDestroy(p.second.first);
    cudaEventDestroy(p.second.second);
  }
  for (cudaEvent_t e : ctx->event_pool) cudaEventDestroy(e);
  delete ctx;
  return LRFG_OK;
}

lrfg_status lrfg_sync(lrfg_ctx* ctx) {
  if (!ctx) return LRFG_EINVAL;
  return guard(ctx, [&] { LRFG_CUDA(cudaStreamSynchronize(ctx->stream)); });
}

long long lrfg_launch_count(const lrfg_ctx* ctx) { return ctx ? ctx->kernel_launches : -1; }

int lrfg_profile_classes(void) { return KC_COUNT; }

const char* lrfg_profile_class_name(int k) { return (k >= 0 && k < KC_COUNT) ? kClassNames[k] : ""; }

lrfg_status lrfg_profile_enable(lrfg_ctx* ctx, int on) {
  if (!ctx) return LRFG_EINVAL;
  return guard(ctx, [&] {
    if (!on) resolve_profile(ctx);
    ctx->profiling = on != 0;
  });
}

lrfg_status lrfg_profile_reset(lrfg_ctx* ctx) {
  if (!ctx) return LRFG_EINVAL;
  return guard(ctx, [&] {
    resolve_profile(ctx);
    fold_device_work(ctx);
    for (auto& st : ctx->stats) st = KStats{};
  });
}

lrfg_status lrfg_profile_read(lrfg_ctx* ctx, int n, long long* launches, double* flops, double* bytes, double* ms) {
  if (!ctx) return LRFG_EINVAL;
  return guard(ctx, [&] {
    LRFG_REQUIRE(n >= 0 && n <= KC_COUNT, "n must be in [0, %d]", (int)KC_COUNT);
    resolve_profile(ctx);
    fold_device_work(ctx);
    for (int k = 0; k < n; ++k) {
      if (launches) launches[k] = ctx->stats[k].launches;
      if (flops) flops[k] = ctx->stats[k].flops;
      if (bytes) bytes[k] = ctx->stats[k].bytes;
      if (ms) ms[k] = ctx->stats[k].ms;
    }
  });
}

lrfg_status lrfg_pool_bytes(const lrfg_ctx* ctx, size_t* in_use, size_t* reserved) {
  if (!ctx || !in_use || !reserved) return LRFG_EINVAL;
  *in_use = ctx->pool->in_use();
  *reserved = ctx->pool->reserved();
  return LRFG_OK;
}

lrfg_status lrfg_fft_fibres(lrfg_ctx* ctx, const double* in, double* out, int outer, int N, int inner, int sign) {
  if (!ctx) return LRFG_EINVAL;
  return guard(ctx, [&] {
    LRFG_REQUIRE(outer >= 0 && inner >= 0, "negative batch");
    LRFG_REQUIRE((in && out) || (long long)outer * inner == 0, "null buffer");
    LRFG_REQUIRE(sign == 1 || sign == -1, "sign must be +1 or -1");
    LRFG_REQUIRE(N >= 1 && N % 2 == 1, "N must be odd");
    fft_fibres<double2>(ctx, (const double2*)in, (double2*)out, outer, N, inner, sign);
  });
}

lrfg_status lrfg_fft_fibres_f32(lrfg_ctx* ctx, const float* in, float* out, int outer, int N, int inner, int sign) {
  if (!ctx) return LRFG_EINVAL;
  return guard(ctx, [&] {
    LRFG_REQUIRE(outer >= 0 && inner >= 0, "negative batch");
    LRFG_REQUIRE((in && out) || (long long)outer * inner == 0, "null buffer");
    LRFG_REQUIRE(sign == 1 || sign == -1, "sign must be +1 or -1");
    LRFG_REQUIRE(N >= 1 && N % 2 == 1, "N must be odd");
    fft_fibres<float2>(ctx, (const float2*)in, (float2*)out, outer, N, inner, sign);
  });
}

lrfg_status lrfg_fibre_operator(lrfg_ctx* ctx, const double* in, double* out, int outer, int N, int inner,
                                lrfg_multiplier kind, double param, double scale) {
  if (!ctx) return LRFG_EINVAL;
  return guard(ctx, [&] {
    LRFG_REQUIRE(outer >= 0 && inner >= 0, "negative batch");
    LRFG_REQUIRE((in && out) || (long long)outer * inner == 0, "null buffer");
    LRFG_REQUIRE(N >= 1 && N % 2 == 1, "N must be odd");
    fibre_operator(ctx, in, out, outer, N, inner, (int)kind, param, scale);
  });
}

lrfg_status lrfg_tt_hadamard(lrfg_ctx* ctx, const lrfg_tt* x, const lrfg_tt* y, lrfg_tt* out) {
  if (!ctx) return LRFG_EINVAL;
  return guard(ctx, [&] {
    check_tt(x);
    check_tt(y);
    LRFG_REQUIRE(out != nullptr, "null output");
    TT res;
    tt_hadamard(ctx, view_of(*x), view_of(*y), res);
    publish_tt(res, out);
    download_tt(ctx, res, out->cores, 1);
  });
}

lrfg_status lrfg_tt_add(lrfg_ctx* ctx, double alpha, const lrfg_tt* x, double beta, const lrfg_tt* y, lrfg_tt* out) {
  if (!ctx) return LRFG_EINVAL;
  return guard(ctx, [&] {
    check_tt(x);
    check_tt(y);
    LRFG_REQUIRE(out != nullptr, "null output");
    TT res;
    tt_add(ctx, alpha, nullptr, view_of(*x), beta, nullptr, view_of(*y), res);
    publish_tt(res, out);
    download_tt(ctx, res, out->cores, 1);
  });
}

lrfg_status lrfg_tt_round_tol(lrfg_ctx* ctx, const lrfg_tt* x, int rmax, double tol, lrfg_tt* out) {
  if (!ctx) return LRFG_EINVAL;
  return guard(ctx, [&] {
    check_tt(x);
    LRFG_REQUIRE(out != nullptr, "null output");
    LRFG_REQUIRE(rmax >= 1, "rmax must be >= 1");
    LRFG_REQUIRE(tol >= 0.0 && tol < 1.0, "tol must be in [0, 1) (got %g)", tol);
    TT res;
    tt_round(ctx, view_of(*x), rmax, res, tol);
    publish_tt(res, out);
    download_tt(ctx, res, out->cores, 1);
  });
}

static void round_sketch_common(lrfg_ctx* ctx, SketchSource& z, int d, const int* N, int ell, unsigned long long seed,
                                int rmax, double tol, lrfg_tt* out) {
  LRFG_REQUIRE(out != nullptr, "null output");
  LRFG_REQUIRE(d >= 2, "randomised rounding needs d = 2 or 3");
  LRFG_REQUIRE(rmax >= 1 && ell >= 1, "rmax and ell must be >= 1");
  LRFG_REQUIRE(tol >= 0.0 && tol < 1.0, "tol must be in [0, 1) (got %g)", tol);
  TT om;
  sketch_tt(ctx, d, N, ell, seed, om);
  TTBatch ob;
  tt_round_sketch(ctx, z, view_of(om), rmax, ob, tol);
  TT res;
  res.d = ob.d;
  for (int j = 0; j < 3; ++j) res.N[j] = ob.N[j];
  for (int j = 0; j < 4; ++j) res.r[j] = ob.r[j];
  for (int j = 0; j < ob.d; ++j) res.core[j] = std::move(ob.core[j]);
  publish_tt(res, out);
  download_tt(ctx, res, out->cores, 1);
}

lrfg_status lrfg_tt_round_sketch(lrfg_ctx* ctx, const lrfg_tt* x, int ell, unsigned long long seed, int rmax,
                                 double tol, lrfg_tt* out) {
  if (!ctx) return LRFG_EINVAL;
  return guard(ctx, [&] {
    check_tt(x);
    SketchSource z;
    z.kind = SketchSource::DENSE;
    z.d = x->d;
    for (int j = 0; j < 3; ++j) z.N[j] = j < x->d ? x->N[j] : 0;
    for (int j = 0; j <= x->d; ++j) z.s[j] = x->r[j];
    for (int j = 0; j < x->d; ++j) z.dense[j] = x->cores[j];
    round_sketch_common(ctx, z, x->d, x->N, ell, seed, rmax, tol, out);
  });
}

lrfg_status lrfg_tt_hadamard_round_sketch(lrfg_ctx* ctx, const lrfg_tt* x, const lrfg_tt* y, int ell,
                                          unsigned long long seed, int rmax, double tol, lrfg_tt* out) {
  if (!ctx) return LRFG_EINVAL;
  return guard(ctx, [&] {
    check_tt(x);
    check_tt(y);
    LRFG_REQUIRE(x->d == y->d, "Hadamard of TTs of different order");
    for (int j = 0; j < x->d; ++j) LRFG_REQUIRE(x->N[j] == y->N[j], "Hadamard of TTs on different grids");
    SketchSource z;
    z.kind = SketchSource::KHATRI_RAO;
    z.d = x->d;
    z.x = view_of(*x);
    for (int j = 0; j < 3; ++j) z.N[j] = j < x->d ? x->N[j] : 0;
    for (int j = 0; j <= x->d; ++j) {
      z.s[j] = x->r[j] * y->r[j];
      z.ry[j] = y->r[j];
    }
    for (int j = 0; j < x->d; ++j) z.y[j][0] = y->cores[j];
    round_sketch_common(ctx, z, x->d, x->N, ell, seed, rmax, tol, out);
  });
}

lrfg_status lrfg_tt_round(lrfg_ctx* ctx, const lrfg_tt* x, int rmax, lrfg_tt* out) {
  return lrfg_tt_round_tol(ctx, x, rmax, 0.0, out);
}

lrfg_status lrfg_tucker_round(lrfg_ctx* ctx, const lrfg_tucker* x, int rmax, lrfg_tucker* out) {
  return lrfg_tucker_round_tol(ctx, x, rmax, 0.0, out);
}

lrfg_status lrfg_tucker_round_tol(lrfg_ctx* ctx, const lrfg_tucker* x, int rmax, double tol, lrfg_tucker* out) {
  if (!ctx) return LRFG_EINVAL;
  return guard(ctx, [&] {
    check_tucker(x);
    LRFG_REQUIRE(out != nullptr && out->core != nullptr, "null output");
    LRFG_REQUIRE(rmax >= 1, "rmax must be >= 1");
    LRFG_REQUIRE(tol >= 0.0 && tol < 1.0, "tol must be in [0, 1) (got %g)", tol);
    TKView v{};
    v.d = x->d;
    for (int j = 0; j < 3; ++j) {
      v.N[j] = j < x->d ? x->N[j] : 1;
      v.r[j] = j < x->d ? x->r[j] : 1;
      v.fac[j] = j < x->d ? x->factors[j] : nullptr;
    }
    v.core = x->core;
    TK res;
    tk_round(ctx, v, rmax, res, tol);
    out->d = res.d;
    size_t nc = 1;
    for (int j = 0; j < 3; ++j) {
      out->N[j] = x->N[j];
      out->r[j] = res.r[j];
      if (j < res.d) nc *= (size_t)res.r[j];
    }
    LRFG_CUDA(cudaMemcpyAsync(out->core, res.core.get(), sizeof(double) * nc, cudaMemcpyDeviceToDevice, ctx->stream));
    for (int j = 0; j < res.d; ++j) {
      LRFG_REQUIRE(out->factors[j] != nullptr, "null output factor %d", j);
      LRFG_CUDA(cudaMemcpyAsync(out->factors[j], res.fac[j].get(), sizeof(double) * res.N[j] * res.r[j],
                                cudaMemcpyDeviceToDevice, ctx->stream));
    }
    LRFG_CUDA(cudaStreamSynchronize(ctx->stream));
  });
}

lrfg_status lrfg_tt_dot(lrfg_ctx* ctx, const lrfg_tt* x, const lrfg_tt* y, double* result) {
  if (!ctx) return LRFG_EINVAL;
  return guard(ctx, [&] {
    check_tt(x);
    check_tt(y);
    LRFG_REQUIRE(result != nullptr, "null result");
    *result = tt_dot(ctx, view_of(*x), view_of(*y));
  });
}

lrfg_status lrfg_tt_precond(lrfg_ctx* ctx, const lrfg_tt* x, double pinv_eps, int rmax, lrfg_tt* out) {
  if (!ctx) return LRFG_EINVAL;
  return guard(ctx, [&] {
    check_tt(x);
    LRFG_REQUIRE(out != nullptr, "null output");
    LRFG_REQUIRE(rmax >= 1, "rmax must be >= 1");
    LRFG_REQUIRE(pinv_eps > 0.0 && pinv_eps < 1.0, "pinv_eps must be in (0,1)");
    double xmax = 0.0;
    for (int j = 0; j < x->d; ++j) xmax += (double)((x->N[j] - 1) / 2) * ((x->N[j] - 1) / 2);
    std::vector<double> t, w;
    expsum_inverse(xmax, pinv_eps, t, w);
    TT res;
    tt_precond(ctx, view_of(*x), t, w, rmax, res);
    publish_tt(res, out);
    download_tt(ctx, res, out->cores, 1);
  });
}

lrfg_status lrfg_tt_compress(lrfg_ctx* ctx, int d, const int N[3], const double* values, int rmax, double tol,
                             lrfg_tt* out) {
  if (!ctx) return LRFG_EINVAL;
  return guard(ctx, [&] {
    check_grid(d, N);
    LRFG_REQUIRE(values && out, "null buffer");
    LRFG_REQUIRE(rmax >= 1, "rmax must be >= 1");
    TT res;
    tt_compress(ctx, d, N, values, rmax, tol, res);
    publish_tt(res, out);
    download_tt(ctx, res, out->cores, 1);
  });
}

lrfg_status lrfg_tt_expand(lrfg_ctx* ctx, const lrfg_tt* x, double* values) {
  if (!ctx) return LRFG_EINVAL;
  return guard(ctx, [&] {
    check_tt(x);
    LRFG_REQUIRE(values != nullptr, "null output");
    tt_expand(ctx, view_of(*x), values);
  });
}

lrfg_status lrfg_problem_create(lrfg_ctx* ctx, const lrfg_coeff* coeff, const lrfg_opts* opts, lrfg_problem** out) {
  if (!ctx) return LRFG_EINVAL;
  if (out) *out = nullptr;
  lrfg_problem* P = nullptr;
  lrfg_status st = guard(ctx, [&] {
    LRFG_REQUIRE(coeff && opts && out, "null argument");
    check_grid(coeff->d, coeff->N);
    LRFG_REQUIRE(opts->fmt == LRFG_FULL || opts->fmt == LRFG_TT || tucker_like(opts->fmt),
                 "solution format must be LRFG_FULL, LRFG_CP, LRFG_TUCKER or LRFG_TT");
    if (opts->fmt == LRFG_CP && coeff->d != 2)
      fail(LRFG_ENOTSUP, "LRFG_CP is provided for d = 2 (its truncation is ill-posed for d >= 3, App. A.1)");
    LRFG_REQUIRE(opts->prec == LRFG_FP64 || opts->prec == LRFG_MIXED, "unknown precision %d", (int)opts->prec);
    if (opts->prec == LRFG_MIXED && opts->fmt != LRFG_FULL && !(opts->fmt == LRFG_TT && opts->disc == LRFG_GANI))
      fail(LRFG_ENOTSUP, "LRFG_MIXED is implemented for LRFG_FULL and LRFG_TT (GaNi) solutions");
    LRFG_REQUIRE(opts->maxit >= 0, "maxit must be >= 0");
    LRFG_REQUIRE(opts->tol >= 0.0, "tol must be >= 0");
    if (opts->fmt != LRFG_FULL) LRFG_REQUIRE(opts->rank >= 1, "low-rank solve needs rank >= 1 (got %d)", opts->rank);
    LRFG_REQUIRE(opts->rank_tol >= 0.0 && opts->rank_tol < 1.0, "rank_tol must be in [0, 1) (got %g)", opts->rank_tol);
    LRFG_REQUIRE(opts->coeff_rank >= 0, "coeff_rank must be >= 0 (got %d)", opts->coeff_rank);
    LRFG_REQUIRE(opts->rank_start >= 0 && opts->rank_step >= 0, "rank_start and rank_step must be >= 0");
    LRFG_REQUIRE(opts->disc == LRFG_GANI || opts->disc == LRFG_GA, "unknown discretisation %d", (int)opts->disc);
    LRFG_REQUIRE(opts->sketch_over >= 0, "sketch_over must be >= 0 (got %d)", opts->sketch_over);
    LRFG_REQUIRE(opts->sketch_keep == 0 || opts->sketch_over > 0, "sketch_keep needs sketch_over > 0");
    if (opts->sketch_over > 0 && (opts->fmt != LRFG_TT || opts->disc != LRFG_GANI))
      fail(LRFG_ENOTSUP, "the randomised rounding (sketch_over > 0) is implemented for LRFG_TT GaNi solutions");
    if (opts->disc == LRFG_GA && opts->prec != LRFG_FP64) fail(LRFG_ENOTSUP, "LRFG_GA is implemented in LRFG_FP64");
    LRFG_REQUIRE(coeff->fmt == LRFG_FULL || coeff->fmt == LRFG_TT || coeff->fmt == LRFG_TUCKER,
                 "coefficient format must be FULL, TT or TUCKER");
    P = new lrfg_problem();
    ctx->live_objects++;
    P->ctx = ctx;
    P->opts = *opts;
    if (P->opts.pinv_eps <= 0.0) P->opts.pinv_eps = 0.1;
    LRFG_REQUIRE(P->opts.pinv_eps < 1.0, "pinv_eps must be < 1");
    P->d = coeff->d;
    for (int j = 0; j < 3; ++j) P->N[j] = j < coeff->d ? coeff->N[j] : 0;
    P->aniso = check_aniso(P->d, coeff->B, P->B);
    P->ga = opts->disc == LRFG_GA;
    const long long n = grid_size(P->d, P->N);
    // coefficient -> device
    if (coeff->fmt == LRFG_FULL) {
      LRFG_REQUIRE(coeff->values != nullptr, "null coefficient values");
      DBuf<double> a(ctx->pool, n);
      LRFG_CUDA(cudaMemcpyAsync(a.get(), coeff->values, sizeof(double) * n,
                                coeff->on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, ctx->stream));
      // validated on the device (grids of 10^9 points and more)
      const long long bad = first_nonpositive(ctx, a.get(), n);
      LRFG_REQUIRE(bad < 0, "coefficient must be positive and finite (index %lld)", bad);
      if (opts->fmt == LRFG_FULL) {
        P->a_full = std::move(a);
      } else if (tucker_like(opts->fmt)) {
        tk_compress(ctx, P->d, P->N, a.get(), 64, 1e-7, P->a_tk);
      } else {
        tt_compress(ctx, P->d, P->N, a.get(), coeff_rank(*opts), opts->rank_tol, P->a_tt);
      }
    } else if (coeff->fmt == LRFG_TUCKER) {
      LRFG_REQUIRE(coeff->tk.d == coeff->d, "coefficient Tucker order differs from d");
      for (int j = 0; j < coeff->d; ++j) LRFG_REQUIRE(coeff->tk.N[j] == coeff->N[j], "coefficient Tucker grid differs");
      check_tucker(&coeff->tk);
      TK a;
      upload_tucker(ctx, &coeff->tk, coeff->on_device, a);
      if (tucker_like(opts->fmt)) {
        P->a_tk = std::move(a);
      } else {
        P->a_full = DBuf<double>(ctx->pool, n);
        tk_expand(ctx, tk_view(a), P->a_full.get());
        if (opts->fmt == LRFG_TT)
          tt_compress(ctx, P->d, P->N, P->a_full.get(), coeff_rank(*opts), opts->rank_tol, P->a_tt);
      }
    } else {
      LRFG_REQUIRE(coeff->tt.d == coeff->d, "coefficient TT order differs from d");
      for (int j = 0; j < coeff->d; ++j) LRFG_REQUIRE(coeff->tt.N[j] == coeff->N[j], "coefficient TT grid differs");
      check_tt(&coeff->tt);
      TT a;
      upload_tt(ctx, &coeff->tt, coeff->on_device, a);
      if (opts->fmt == LRFG_TT) {
        P->a_tt = std::move(a);
      } else {
        P->a_full = DBuf<double>(ctx->pool, n);
        tt_expand(ctx, view_of(a), P->a_full.get());
        if (tucker_like(opts->fmt)) tk_compress(ctx, P->d, P->N, P->a_full.get(), 64, 1e-7, P->a_tk);
      }
    }
    if (opts->fmt == LRFG_FULL) {
      P->g = make_grid(P->d, P->N);
      make_inv_tables(ctx, P->g, P->inv64, P->inv32);
      P->wc = DBuf<double2>(ctx->pool, P->g.n_half);
      P->wr = DBuf<double>(ctx->pool, P->g.n_real);
      if (P->ga) {
        int M[3] = {0, 0, 0};
        for (int j = 0; j < P->d; ++j) {
          M[j] = 2 * P->N[j] - 1;
          make_plan(M[j], 27);  // LRFG_ENOTSUP when the double grid has a prime factor above 31
        }
        P->gM = make_grid(P->d, M);
        P->a_ga = DBuf<double>(ctx->pool, P->gM.n_real);
        P->wrM = DBuf<double>(ctx->pool, P->gM.n_real);
        P->wcM = DBuf<double2>(ctx->pool, P->gM.n_half);
        ga_coefficient(ctx, P->g, P->gM, P->a_full.get(), P->wc.get(), P->wcM.get(), P->a_ga.get());
      }
      if (P->opts.prec == LRFG_MIXED) {
        P->a_full_f = DBuf<float>(ctx->pool, n);
        convert(ctx, (const double*)P->a_full.get(), P->a_full_f.get(), n);
        P->wcf = DBuf<float2>(ctx->pool, P->g.n_half);
        P->wrf = DBuf<float>(ctx->pool, P->g.n_real);
      }
    } else {
      double xmax = 0.0;
      for (int j = 0; j < P->d; ++j) xmax += (double)((P->N[j] - 1) / 2) * ((P->N[j] - 1) / 2);
      expsum_inverse(xmax, P->opts.pinv_eps, P->pt, P->pw);
      if (P->ga) {
        // the modified coefficient mode by mode from the TT of pixel values, and its projection
        int M[3] = {0, 0, 0};
        for (int j = 0; j < P->d; ++j) {
          M[j] = 2 * P->N[j] - 1;
          make_plan(M[j], 27);  // LRFG_ENOTSUP when the double grid has a prime factor above 31
        }
        if (tucker_like(opts->fmt)) {
          // the factors of a's pixel values mapped to the modified coefficient, and its projection
          tk_ga_map(ctx, tk_view(P->a_tk), M, GA_EXTEND, P->a_ga_tk);
          tk_ga_map(ctx, tk_view(P->a_ga_tk), P->N, GA_DOWN, P->a_down_tk);
          P->tkga.a_ga = tk_view(P->a_ga_tk);
          P->tkga.a_down = tk_view(P->a_down_tk);
          if (P->aniso) {
            TK one;
            int r1[3] = {1, 1, 1};
            tk_alloc(ctx, one, P->d, P->N, r1);
            fill(ctx, one.core.get(), 1.0, 1);
            for (int j = 0; j < P->d; ++j) fill(ctx, one.fac[j].get(), 1.0, P->N[j]);
            tk_ga_map(ctx, tk_view(one), M, GA_EXTEND, P->ones_ga_tk);
            P->tkga.ones_ga = tk_view(P->ones_ga_tk);
          }
        } else {
          TTBatch ag, ad;
          tt_ga_map(ctx, view_of(P->a_tt), 1, M, GA_EXTEND, ag);
          tt_ga_map(ctx, item_view(ag, 0), 1, P->N, GA_DOWN, ad);
          P->a_ga_tt.d = P->a_down_tt.d = P->d;
          for (int j = 0; j < 3; ++j) {
            P->a_ga_tt.N[j] = ag.N[j];
            P->a_down_tt.N[j] = ad.N[j];
          }
          for (int j = 0; j < 4; ++j) P->a_ga_tt.r[j] = P->a_down_tt.r[j] = ag.r[j];
          for (int j = 0; j < P->d; ++j) {
            P->a_ga_tt.core[j] = std::move(ag.core[j]);
            P->a_down_tt.core[j] = std::move(ad.core[j]);
          }
          if (P->aniso) {
            TT one;
            ones_tt(ctx, P->d, P->N, one);
            TTBatch og;
            tt_ga_map(ctx, view_of(one), 1, M, GA_EXTEND, og);
            P->ones_ga_tt.d = P->d;
            for (int j = 0; j < 3; ++j) P->ones_ga_tt.N[j] = og.N[j];
            for (int j = 0; j < 4; ++j) P->ones_ga_tt.r[j] = og.r[j];
            for (int j = 0; j < P->d; ++j) P->ones_ga_tt.core[j] = std::move(og.core[j]);
          }
        }
      }
    }
    LRFG_CUDA(cudaStreamSynchronize(ctx->stream));
    *out = P;
  });
  if (st != LRFG_OK && P) {
    delete P;
    ctx->live_objects--;
  }
  return st;
}

lrfg_status lrfg_problem_free(lrfg_problem* P) {
  if (!P) return LRFG_EINVAL;
  lrfg_ctx* ctx = P->ctx;
  cudaSetDevice(ctx->device);
  cudaStreamSynchronize(ctx->stream);
  delete P;
  ctx->live_objects--;
  return LRFG_OK;
}

lrfg_status lrfg_problem_coeff_ranks(const lrfg_problem* P, int ranks[4]) {
  if (!P || !ranks) return LRFG_EINVAL;
  for (int j = 0; j < 4; ++j)
    ranks[j] = P->opts.fmt == LRFG_TT ? P->a_tt.r[j] : (tucker_like(P->opts.fmt) && j < P->d ? P->a_tk.r[j] : 1);
  return LRFG_OK;
}

lrfg_status lrfg_problem_apply(lrfg_problem* P, const lrfg_field* in, lrfg_field** out) {
  if (!P) return LRFG_EINVAL;
  lrfg_field* f = nullptr;
  lrfg_status st = guard(P->ctx, [&] {
    LRFG_REQUIRE(out != nullptr, "null output");
    new_field(P->ctx, P->opts.fmt, P->d, P->N, &f);
    apply_into(P, in, f);
    *out = f;
  });
  if (st != LRFG_OK && f) discard_field(f);
  return st;
}

lrfg_status lrfg_problem_apply_into(lrfg_problem* P, const lrfg_field* in, lrfg_field* out) {
  if (!P) return LRFG_EINVAL;
  return guard(P->ctx, [&] {
    LRFG_REQUIRE(out != nullptr && out != in, "output must be a different, existing field");
    check_field(P, out);
    apply_into(P, in, out);
  });
}

lrfg_status lrfg_problem_rhs(lrfg_problem* P, const double* E, lrfg_field** out) {
  if (!P) return LRFG_EINVAL;
  lrfg_field* f = nullptr;
  lrfg_status st = guard(P->ctx, [&] {
    LRFG_REQUIRE(E && out, "null argument");
    for (int j = 0; j < P->d; ++j) LRFG_REQUIRE(std::isfinite(E[j]), "E must be finite");
    new_field(P->ctx, P->opts.fmt, P->d, P->N, &f);
    if (P->opts.fmt == LRFG_FULL) {
      f->half = DBuf<double2>(P->ctx->pool, P->g.n_half);
      if (P->opts.prec == LRFG_MIXED) {
        DBuf<float2> bf(P->ctx->pool, P->g.n_half);
        full_rhs<float>(P, E, bf.get(), 1);
        convert(P->ctx, (const float2*)bf.get(), f->half.get(), P->g.n_half);
      } else {
        full_rhs<double>(P, E, f->half.get(), 1);
      }
    } else if (tucker_like(P->opts.fmt)) {
      tk_rhs(P->ctx, tk_view(P->a_tk), E, P->pt, P->pw, P->opts.rank, f->tk, P->opts.rank_tol, tk_ga(P));
    } else {
      lr_rhs(P, E, f->tt, P->opts.rank);
    }
    *out = f;
  });
  if (st != LRFG_OK && f) discard_field(f);
  return st;
}

lrfg_status lrfg_problem_solve(lrfg_problem* P, const double* E, lrfg_result* res, lrfg_field** u_out) {
  if (!P) return LRFG_EINVAL;
  if (u_out) *u_out = nullptr;
  bool noconv = false;
  lrfg_status st = guard(P->ctx, [&] {
    LRFG_REQUIRE(E && res, "null argument");
    for (int j = 0; j < P->d; ++j) LRFG_REQUIRE(std::isfinite(E[j]), "E must be finite");
    *res = lrfg_result{};
    auto t0 = std::chrono::steady_clock::now();
    if (P->opts.fmt == LRFG_FULL) {
      if (P->opts.prec == LRFG_MIXED) solve_full<float>(P, E, res, u_out);
      else solve_full<double>(P, E, res, u_out);
    }
    else if (tucker_like(P->opts.fmt)) solve_tucker(P, E, res, u_out);
    else solve_tt(P, E, res, u_out);
    LRFG_CUDA(cudaStreamSynchronize(P->ctx->stream));
    res->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    noconv = !res->converged && !(P->opts.fmt != LRFG_FULL && P->opts.stop_on_increase && res->applies > 0 &&
                                  res->iters < P->opts.maxit);
  });
  if (st == LRFG_OK && noconv) return LRFG_ENOCONV;
  return st;
}

lrfg_status lrfg_problem_aeff(lrfg_problem* P, const double* E, const lrfg_field* u, double* Aeff) {
  if (!P) return LRFG_EINVAL;
  return guard(P->ctx, [&] {
    LRFG_REQUIRE(E && Aeff, "null argument");
    check_field(P, u);
    *Aeff = (P->opts.fmt == LRFG_FULL)     ? full_aeff(P, E, u->half.get())
            : tucker_like(P->opts.fmt)     ? tk_aeff(P->ctx, tk_view(P->a_tk), E, tk_view(u->tk), aniso_b(P), tk_ga(P))
                                           : lr_aeff(P, E, view_of(u->tt));
  });
}

lrfg_status lrfg_problem_solve_many(lrfg_problem* P, int nb, const double* E, lrfg_result* res) {
  if (!P) return LRFG_EINVAL;
  bool noconv = false;
  lrfg_status st = guard(P->ctx, [&] {
    LRFG_REQUIRE(E && res && nb >= 1, "null argument or nb < 1");
    for (int i = 0; i < nb * P->d; ++i) LRFG_REQUIRE(std::isfinite(E[i]), "E must be finite");
    auto t0 = std::chrono::steady_clock::now();
    if (lockstep_ok(P) && nb * P->d <= kMaxSketchItems) {
      solve_tt_many(P, E, nb, res);
      LRFG_CUDA(cudaStreamSynchronize(P->ctx->stream));
    } else {
      for (int i = 0; i < nb; ++i) {
        const lrfg_status s1 = lrfg_problem_solve(P, E + (size_t)i * P->d, res + i, nullptr);
        if (s1 != LRFG_OK && s1 != LRFG_ENOCONV) fail(s1, "%s", P->ctx->last_error.c_str());
      }
    }
    const double sec = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    for (int i = 0; i < nb; ++i) {
      res[i].seconds = sec;
      if (!res[i].converged && !(P->opts.fmt != LRFG_FULL && P->opts.stop_on_increase && res[i].applies > 0 &&
                                 res[i].iters < P->opts.maxit))
        noconv = true;
    }
  });
  if (st == LRFG_OK && noconv) return LRFG_ENOCONV;
  return st;
}

// whether problems P and Q can share one lockstep solve: the same grid, options and coefficient TT ranks
static bool same_shape(const lrfg_problem* P, const lrfg_problem* Q) {
  if (P->ctx != Q->ctx || P->d != Q->d) return false;
  for (int j = 0; j < P->d; ++j)
    if (P->N[j] != Q->N[j]) return false;
  for (int j = 0; j <= P->d; ++j)
    if (P->a_tt.r[j] != Q->a_tt.r[j]) return false;
  const lrfg_opts &a = P->opts, &b = Q->opts;
  return a.fmt == b.fmt && a.prec == b.prec && a.rank == b.rank && a.pinv_eps == b.pinv_eps && a.tol == b.tol &&
         a.maxit == b.maxit && a.stop_on_increase == b.stop_on_increase && a.rank_tol == b.rank_tol &&
         a.rank_start == b.rank_start && a.rank_step == b.rank_step && a.disc == b.disc &&
         a.sketch_over == b.sketch_over && a.sketch_seed == b.sketch_seed && a.sketch_keep == b.sketch_keep;
}

lrfg_status lrfg_problems_solve(int np, lrfg_problem* const* Ps, const double* E, lrfg_result* res) {
  if (np < 1 || !Ps || !Ps[0]) return LRFG_EINVAL;
  lrfg_problem* P = Ps[0];
  bool noconv = false;
  lrfg_status st = guard(P->ctx, [&] {
    LRFG_REQUIRE(E && res, "null argument");
    for (int i = 0; i < np; ++i) {
      LRFG_REQUIRE(Ps[i] && Ps[i]->ctx == P->ctx, "problems must share one context");
      LRFG_REQUIRE(Ps[i]->d == P->d, "problems must have the same dimension d");
    }
    for (int i = 0; i < np * P->d; ++i) LRFG_REQUIRE(std::isfinite(E[i]), "E must be finite");
    bool together = np * P->d <= kMaxSketchItems;
    for (int i = 0; i < np && together; ++i) together = lockstep_ok(Ps[i]) && same_shape(P, Ps[i]);
    auto t0 = std::chrono::steady_clock::now();
    if (together) {
      solve_tt_many(P, E, np, res, Ps);
      LRFG_CUDA(cudaStreamSynchronize(P->ctx->stream));
    } else {
      for (int i = 0; i < np; ++i) {
        const lrfg_status s1 = lrfg_problem_solve(Ps[i], E + (size_t)i * P->d, res + i, nullptr);
        if (s1 != LRFG_OK && s1 != LRFG_ENOCONV) fail(s1, "problem %d: %s", i, P->ctx->last_error.c_str());
      }
    }
    const double sec = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    for (int i = 0; i < np; ++i) {
      res[i].seconds = sec;
      const lrfg_opts& o = Ps[i]->opts;
      if (!res[i].converged &&
          !(o.fmt != LRFG_FULL && o.stop_on_increase && res[i].applies > 0 && res[i].iters < o.maxit))
        noconv = true;
    }
  });
  if (st == LRFG_OK && noconv) return LRFG_ENOCONV;
  return st;
}

// The homogenised tensor of Eq. (homog): A_eff E.E is a quadratic form in E (Sec. 2.1), so its diagonal comes
// from the solves with E = e_a and every off-diagonal entry from one more solve by polarisation,
// A_ab = (q(e_a + e_b) - q(e_a) - q(e_b)) / 2, q(E) = A_eff E.E: d (d + 1) / 2 solves in all.
lrfg_status lrfg_problem_aeff_tensor(lrfg_problem* P, double* A, lrfg_result* results) {
  if (!P) return LRFG_EINVAL;
  if (!A) {
    P->ctx->last_error = "null argument";
    return LRFG_EINVAL;
  }
  const int d = P->d;
  double q[3][3] = {};
  // the d (d + 1) / 2 right-hand sides, solved together (in lockstep where the problem allows it)
  std::vector<double> Es;
  for (int a = 0; a < d; ++a)
    for (int b = a; b < d; ++b)
      for (int j = 0; j < d; ++j) Es.push_back((j == a || j == b) ? 1.0 : 0.0);
  const int ns = (int)Es.size() / d;
  std::vector<lrfg_result> rs(ns);
  const lrfg_status st = lrfg_problem_solve_many(P, ns, Es.data(), rs.data());
  if (st != LRFG_OK && st != LRFG_ENOCONV) return st;
  const bool noconv = st == LRFG_ENOCONV;
  int k = 0;
  for (int a = 0; a < d; ++a)
    for (int b = a; b < d; ++b, ++k) {
      if (results) results[k] = rs[k];
      q[a][b] = rs[k].Aeff;
    }
  for (int a = 0; a < d; ++a) {
    A[a * d + a] = q[a][a];
    for (int b = a + 1; b < d; ++b) A[a * d + b] = A[b * d + a] = 0.5 * (q[a][b] - q[a][a] - q[b][b]);
  }
  P->ctx->last_error.clear();
  return noconv ? LRFG_ENOCONV : LRFG_OK;
}

lrfg_status lrfg_solve(lrfg_ctx* ctx, const lrfg_coeff* coeff, const double* E, const lrfg_opts* opts,
                       lrfg_result* res, lrfg_field** u_out) {
  lrfg_problem* P = nullptr;
  lrfg_status st = lrfg_problem_create(ctx, coeff, opts, &P);
  if (st != LRFG_OK) return st;
  st = lrfg_problem_solve(P, E, res, u_out);
  lrfg_problem_free(P);
  return st;
}

lrfg_status lrfg_field_from_full(lrfg_ctx* ctx, int d, const int N[3], const double* values, int on_device,
                                 lrfg_field** out) {
  if (!ctx) return LRFG_EINVAL;
  lrfg_field* f = nullptr;
  lrfg_status st = guard(ctx, [&] {
    check_grid(d, N);
    LRFG_REQUIRE(values && out, "null argument");
    new_field(ctx, LRFG_FULL, d, N, &f);
    FullGrid g = make_grid(d, N);
    DBuf<double> tmp(ctx->pool, g.n_real);
    LRFG_CUDA(cudaMemcpyAsync(tmp.get(), values, sizeof(double) * g.n_real,
                              on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, ctx->stream));
    f->half = DBuf<double2>(ctx->pool, g.n_half);
    full_forward<double>(ctx, g, tmp.get(), nullptr, 1.0, f->half.get());
    LRFG_CUDA(cudaStreamSynchronize(ctx->stream));
    *out = f;
  });
  if (st != LRFG_OK && f) discard_field(f);
  return st;
}

lrfg_status lrfg_field_from_tt(lrfg_ctx* ctx, const lrfg_tt* x, int on_device, lrfg_field** out) {
  if (!ctx) return LRFG_EINVAL;
  lrfg_field* f = nullptr;
  lrfg_status st = guard(ctx, [&] {
    check_tt(x);
    LRFG_REQUIRE(out != nullptr, "null output");
    new_field(ctx, LRFG_TT, x->d, x->N, &f);
    upload_tt(ctx, x, on_device, f->tt);
    LRFG_CUDA(cudaStreamSynchronize(ctx->stream));
    *out = f;
  });
  if (st != LRFG_OK && f) discard_field(f);
  return st;
}

lrfg_status lrfg_field_from_tucker(lrfg_ctx* ctx, const lrfg_tucker* x, int on_device, lrfg_field** out) {
  if (!ctx) return LRFG_EINVAL;
  lrfg_field* f = nullptr;
  lrfg_status st = guard(ctx, [&] {
    check_tucker(x);
    LRFG_REQUIRE(out != nullptr, "null output");
    new_field(ctx, LRFG_TUCKER, x->d, x->N, &f);
    upload_tucker(ctx, x, on_device, f->tk);
    LRFG_CUDA(cudaStreamSynchronize(ctx->stream));
    *out = f;
  });
  if (st != LRFG_OK && f) discard_field(f);
  return st;
}

lrfg_status lrfg_field_info(const lrfg_field* f, lrfg_format* fmt, int* d, int N[3], int r[4]) {
  if (!f) return LRFG_EINVAL;
  if (fmt) *fmt = f->fmt;
  if (d) *d = f->d;
  if (N) for (int j = 0; j < 3; ++j) N[j] = f->N[j];
  if (r)
    for (int j = 0; j < 4; ++j)
      r[j] = f->fmt == LRFG_TT ? f->tt.r[j] : (tucker_like(f->fmt) && j < f->d ? f->tk.r[j] : 1);
  return LRFG_OK;
}

lrfg_status lrfg_field_export_full(lrfg_ctx* ctx, const lrfg_field* f, double* values, int on_device) {
  if (!ctx) return LRFG_EINVAL;
  return guard(ctx, [&] {
    LRFG_REQUIRE(f && values, "null argument");
    const long long n = grid_size(f->d, f->N);
    DBuf<double> dst;
    double* target = values;
    if (!on_device) { dst = DBuf<double>(ctx->pool, n); target = dst.get(); }
    if (f->fmt == LRFG_FULL) {
      FullGrid g = make_grid(f->d, f->N);
      DBuf<double2> tmp(ctx->pool, g.n_half);
      LRFG_CUDA(cudaMemcpyAsync(tmp.get(), f->half.get(), sizeof(double2) * g.n_half, cudaMemcpyDeviceToDevice,
                                ctx->stream));
      full_inverse<double>(ctx, g, tmp.get(), nullptr, 1.0 / (double)g.n_real, target);
    } else if (tucker_like(f->fmt)) {
      tk_expand(ctx, tk_view(f->tk), target);
    } else {
      tt_expand(ctx, view_of(f->tt), target);
    }
    if (!on_device)
      LRFG_CUDA(cudaMemcpyAsync(values, target, sizeof(double) * n, cudaMemcpyDeviceToHost, ctx->stream));
    LRFG_CUDA(cudaStreamSynchronize(ctx->stream));
  });
}

lrfg_status lrfg_field_export_tt(lrfg_ctx* ctx, const lrfg_field* f, double* const cores[3], int on_device) {
  if (!ctx) return LRFG_EINVAL;
  return guard(ctx, [&] {
    LRFG_REQUIRE(f && cores, "null argument");
    LRFG_REQUIRE(f->fmt == LRFG_TT, "field is not a TT");
    download_tt(ctx, f->tt, cores, on_device);
    LRFG_CUDA(cudaStreamSynchronize(ctx->stream));
  });
}

lrfg_status lrfg_field_free(lrfg_field* f) {
  if (!f) return LRFG_EINVAL;
  lrfg_ctx* ctx = f->ctx;
  cudaSetDevice(ctx->device);
  cudaStreamSynchronize(ctx->stream);
  delete f;
  ctx->live_objects--;
  return LRFG_OK;
}

}  // extern "C"
