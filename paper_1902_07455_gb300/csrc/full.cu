// Full-format comparison path (hot-path row a9): real <-> half-spectrum d-dimensional FFTs, the
// pointwise Fourier multipliers of the GaNi operator, and the reductions of PCG and A_eff.
//
// A grid (N_0, .., N_{d-1}) of reals has the half spectrum (N_0, .., N_{d-2}, H), H = (N_{d-1}+1)/2:
// the last axis keeps k >= 0 only (Hermitian symmetry of real fields, Sec. 2.2.1).  Forward transform:
// real-to-complex rows along the last axis (two real rows packed per complex FFT), then complex fibres
// along the other axes.  Transforms are unnormalised (Phi = |N| F_N); scalings are folded into the
// pointwise kernels.
#include <algorithm>
#include <cmath>

#include "full.cuh"

namespace lrfg {

static unsigned grid1d(lrfg_ctx* ctx, long long n) {
  long long g = (n + 255) / 256;
  long long cap = 16LL * (ctx->num_sms > 0 ? ctx->num_sms : 152);
  return (unsigned)std::max(1LL, std::min(g, cap));
}

FullGrid make_grid(int d, const int* N) {
  FullGrid g{};
  g.d = d;
  g.n_real = 1;
  for (int j = 0; j < d; ++j) { g.N[j] = N[j]; g.n_real *= N[j]; }
  g.H = (N[d - 1] + 1) / 2;
  g.rows = g.n_real / N[d - 1];
  g.n_half = g.rows * g.H;
  return g;
}

// ------------------------------------------------------------------------------------------------
// real rows -> half spectra (forward), optional pre-multiplication by a coefficient
// ------------------------------------------------------------------------------------------------
template <typename R>
__global__ void __launch_bounds__(256, 3) r2c_rows_kernel(const R* __restrict__ in, const R* __restrict__ coef, R scale,
                                                       typename CplxOf<R>::T* __restrict__ out, long long rows, int N,
                                                       int H, int TF, FftPlan pl,
                                                       const typename CplxOf<R>::T* __restrict__ Wg) {
  using V = typename CplxOf<R>::T;
  const float invN = 1.0f / (float)N, invH = 1.0f / (float)H;
  extern __shared__ __align__(16) unsigned char smraw_r2c[];
  V* sm = (V*)smraw_r2c;
  V* W = sm;
  V* a = sm + 2 * N;
  V* b = a + (size_t)TF * N;
  for (int j = threadIdx.x; j < N; j += blockDim.x) W[j] = Wg[j];
  const long long r0 = (long long)blockIdx.x * 2 * TF;
  const int nr = (int)min(2LL * TF, rows - r0);
  const int nrow = min(nr, TF);
  for (int t = threadIdx.x; t < nrow * N; t += blockDim.x) a[t] = mkc<V>(R(0), R(0));
  __syncthreads();
  // the tile's rows are contiguous: issue kU loads per thread before using any of them
  {
    constexpr int kU = 8;
    const R* src = in + (size_t)r0 * N;
    const R* cs = coef ? coef + (size_t)r0 * N : nullptr;
    const int total = nr * N;
    for (int base = threadIdx.x; base < total; base += kU * blockDim.x) {
      R v[kU], c[kU];
#pragma unroll
      for (int u = 0; u < kU; ++u) {
        const int t = base + u * blockDim.x;
        v[u] = t < total ? src[t] : R(0);
        c[u] = (cs && t < total) ? cs[t] : R(1);
      }
#pragma unroll
      for (int u = 0; u < kU; ++u) {
        const int t = base + u * blockDim.x;
        if (t < total) {
          const int f = small_div(t, N, invN), n = t - f * N;
          const R x = v[u] * c[u] * scale;
          if (f < TF) a[(size_t)f * N + n].x = x; else a[(size_t)(f - TF) * N + n].y = x;
        }
      }
    }
  }
  __syncthreads();
  V* Z = stockham_rows<-1>(a, b, nrow, N, pl, (const V*)W);
  // split: X[k] = (Z[k] + conj Z[N-k]) / 2,  Y[k] = (Z[k] - conj Z[N-k]) / (2i)
  for (int t = threadIdx.x; t < nr * H; t += blockDim.x) {
    const int f = small_div(t, H, invH), k = t - f * H;
    int row = f < TF ? f : f - TF;
    V z = Z[(size_t)row * N + k];
    V zc = Z[(size_t)row * N + ((N - k) % N)];
    V v;
    if (f < TF) v = mkc<V>(R(0.5) * (z.x + zc.x), R(0.5) * (z.y - zc.y));
    else v = mkc<V>(R(0.5) * (z.y + zc.y), R(-0.5) * (z.x - zc.x));
    out[(size_t)(r0 + f) * H + k] = v;
  }
}

// half spectra -> real rows (inverse, unnormalised), optional post-multiplication by a coefficient
template <typename R>
__global__ void __launch_bounds__(256, 3) c2r_rows_kernel(const typename CplxOf<R>::T* __restrict__ in,
                                                       const R* __restrict__ coef, R scale, R* __restrict__ out,
                                                       long long rows, int N, int H, int TF, FftPlan pl,
                                                       const typename CplxOf<R>::T* __restrict__ Wg) {
  using V = typename CplxOf<R>::T;
  const float invN = 1.0f / (float)N;
  extern __shared__ __align__(16) unsigned char smraw_c2r[];
  V* sm = (V*)smraw_c2r;
  V* W = sm;
  V* a = sm + 2 * N;
  V* b = a + (size_t)TF * N;
  for (int j = threadIdx.x; j < N; j += blockDim.x) W[j] = Wg[j];
  const long long r0 = (long long)blockIdx.x * 2 * TF;
  const int nr = (int)min(2LL * TF, rows - r0);
  const int nrow = min(nr, TF);
  for (int t = threadIdx.x; t < nrow * N; t += blockDim.x) a[t] = mkc<V>(R(0), R(0));
  __syncthreads();
  // Z[k] = X[k] + i Y[k] over the full range, X[N-k] = conj X[k]; one thread per (row, k), kU (row, k)
  // pairs per thread loaded before any is used
  {
    constexpr int kU = 4;
    const int total = nrow * N;
    for (int base = threadIdx.x; base < total; base += kU * blockDim.x) {
      V x0[kU], x1[kU];
#pragma unroll
      for (int u = 0; u < kU; ++u) {
        const int t = base + u * blockDim.x;
        x0[u] = mkc<V>(R(0), R(0));
        x1[u] = mkc<V>(R(0), R(0));
        if (t < total) {
          const int row = small_div(t, N, invN), k = t - row * N;
          const int kk = k < H ? k : N - k;
          x0[u] = in[(size_t)(r0 + row) * H + kk];
          if (row + TF < nr) x1[u] = in[(size_t)(r0 + row + TF) * H + kk];
        }
      }
#pragma unroll
      for (int u = 0; u < kU; ++u) {
        const int t = base + u * blockDim.x;
        if (t < total) {
          const int row = small_div(t, N, invN), k = t - row * N;
          V p = x0[u], q = x1[u];
          if (k >= H) { p.y = -p.y; q.y = -q.y; }
          a[(size_t)row * N + k] = mkc<V>(p.x - q.y, p.y + q.x);
        }
      }
    }
  }
  __syncthreads();
  V* Z = stockham_rows<1>(a, b, nrow, N, pl, (const V*)W);
  for (int t = threadIdx.x; t < nr * N; t += blockDim.x) {
    const int f = small_div(t, N, invN), n = t - f * N;
    int row = f < TF ? f : f - TF;
    V z = Z[(size_t)row * N + n];
    R v = (f < TF ? z.x : z.y) * scale;
    size_t gi = (size_t)(r0 + f) * N + n;
    if (coef) v *= coef[gi];
    out[gi] = v;
  }
}

template <typename R>
static int row_tile(lrfg_ctx* ctx, int N, size_t* smem) {
  using V = typename CplxOf<R>::T;
  // at most 72 KB for N <= 300, so that three blocks share an SM
  size_t limit = 72 * 1024;
  if (N > 300) limit = (size_t)std::min(ctx->max_smem_optin, 200 * 1024);
  long long per = 2LL * N * (long long)sizeof(V);
  long long tf = ((long long)limit - 2LL * N * (long long)sizeof(V)) / per;
  tf = std::max(1LL, std::min(tf, 32LL));
  *smem = (size_t)(2LL * N * sizeof(V) + tf * per);
  return (int)tf;
}

template <typename R>
void full_forward(lrfg_ctx* ctx, const FullGrid& g, const R* real_in, const R* coef, R scale,
                  typename CplxOf<R>::T* half_out) {
  using V = typename CplxOf<R>::T;
  const int N = g.N[g.d - 1];
  FftPlan pl = make_plan(N, plan_radix<V>());
  LRFG_CUDA(ensure_roots(ctx->device));
  const V* W = twiddle_table<R>(ctx, N);
  size_t smem;
  int TF = row_tile<R>(ctx, N, &smem);
  long long blocks = (g.rows + 2LL * TF - 1) / (2LL * TF);
  LRFG_CUDA(cudaFuncSetAttribute(r2c_rows_kernel<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  LRFG_LAUNCH(ctx, KC_R2C, 2.5 * N * std::log2((double)N) * (double)g.rows,
              (double)g.rows * (N * sizeof(R) * (coef ? 2 : 1) + g.H * sizeof(V)),
              r2c_rows_kernel<R><<<(unsigned)blocks, 256, smem, ctx->stream>>>(real_in, coef, scale, half_out, g.rows, N,
                                                                                g.H, TF, pl, W));
  // complex axes, innermost first
  long long inner = g.H;
  for (int ax = g.d - 2; ax >= 0; --ax) {
    long long outer = 1;
    for (int j = 0; j < ax; ++j) outer *= g.N[j];
    fft_fibres(ctx, half_out, half_out, outer, g.N[ax], inner, -1);
    inner *= g.N[ax];
  }
}

template <typename R>
void full_inverse(lrfg_ctx* ctx, const FullGrid& g, typename CplxOf<R>::T* half_inout, const R* coef, R scale,
                  R* real_out) {
  using V = typename CplxOf<R>::T;
  long long inner = g.n_half;
  for (int ax = 0; ax <= g.d - 2; ++ax) {
    inner /= g.N[ax];
    long long outer = g.n_half / (inner * g.N[ax]);
    fft_fibres(ctx, half_inout, half_inout, outer, g.N[ax], inner, 1);
  }
  const int N = g.N[g.d - 1];
  FftPlan pl = make_plan(N, plan_radix<V>());
  LRFG_CUDA(ensure_roots(ctx->device));
  const V* W = twiddle_table<R>(ctx, N);
  size_t smem;
  int TF = row_tile<R>(ctx, N, &smem);
  long long blocks = (g.rows + 2LL * TF - 1) / (2LL * TF);
  LRFG_CUDA(cudaFuncSetAttribute(c2r_rows_kernel<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  LRFG_LAUNCH(ctx, KC_C2R, 2.5 * N * std::log2((double)N) * (double)g.rows,
              (double)g.rows * (N * sizeof(R) * (coef ? 2 : 1) + g.H * sizeof(V)),
              c2r_rows_kernel<R><<<(unsigned)blocks, 256, smem, ctx->stream>>>(half_inout, coef, scale, real_out, g.rows,
                                                                                N, g.H, TF, pl, W));
}

template void full_forward<double>(lrfg_ctx*, const FullGrid&, const double*, const double*, double, double2*);
template void full_forward<float>(lrfg_ctx*, const FullGrid&, const float*, const float*, float, float2*);
template void full_inverse<double>(lrfg_ctx*, const FullGrid&, double2*, const double*, double, double*);
template void full_inverse<float>(lrfg_ctx*, const FullGrid&, float2*, const float*, float, float*);

// ------------------------------------------------------------------------------------------------
// pointwise Fourier multipliers on the half spectrum (multipliers formed in FP64, applied in R)
// ------------------------------------------------------------------------------------------------
struct KIndex {
  int d, N0, N1, N2, H;
};

__device__ __forceinline__ void kvec(long long t, const KIndex& ki, int* k) {
  int kl = (int)(t % ki.H);
  long long rest = t / ki.H;
  if (ki.d == 3) {
    int i1 = (int)(rest % ki.N1), i0 = (int)(rest / ki.N1);
    k[0] = freq_of(i0, ki.N0);
    k[1] = freq_of(i1, ki.N1);
    k[2] = kl;
  } else {
    k[0] = freq_of((int)rest, ki.N0);
    k[1] = kl;
    k[2] = 0;
  }
}

// out = in * (2 pi i k_alpha) * scale
template <typename V>
__global__ void mul_grad_kernel(const V* __restrict__ in, V* out, long long n, KIndex ki, int alpha, double scale) {
  using R = typename RealOf<V>::T;
  const double two_pi = 6.283185307179586476925286766559;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x) {
    int k[3];
    kvec(t, ki, k);
    const R f = (R)(two_pi * (double)k[alpha] * scale);
    V v = in[t];
    out[t] = mkc<V>(-v.y * f, v.x * f);
  }
}

// acc = (init ? 0 : acc) + in * (-2 pi i k_alpha) * scale; if precond, then acc /= k.k (0 at k=0)
template <typename V>
__global__ void acc_div_kernel(const V* __restrict__ in, V* acc, long long n, KIndex ki, int alpha, double scale,
                               int init, int precond) {
  using R = typename RealOf<V>::T;
  const double two_pi = 6.283185307179586476925286766559;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x) {
    int k[3];
    kvec(t, ki, k);
    const R f = (R)(-two_pi * (double)k[alpha] * scale);
    V v = in[t];
    V r = mkc<V>(-v.y * f, v.x * f);
    if (!init) { V o = acc[t]; r.x += o.x; r.y += o.y; }
    if (precond) {
      const int kk = k[0] * k[0] + k[1] * k[1] + k[2] * k[2];
      const R s = kk > 0 ? (R)(1.0 / (double)kk) : R(0);
      r.x *= s;
      r.y *= s;
    }
    acc[t] = r;
  }
}

template <typename V>
__global__ void precond_kernel(const V* __restrict__ in, V* out, long long n, KIndex ki) {
  using R = typename RealOf<V>::T;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x) {
    int k[3];
    kvec(t, ki, k);
    const int kk = k[0] * k[0] + k[1] * k[1] + k[2] * k[2];
    const R s = kk > 0 ? (R)(1.0 / (double)kk) : R(0);
    V v = in[t];
    out[t] = mkc<V>(v.x * s, v.y * s);
  }
}

static KIndex kindex(const FullGrid& g) {
  KIndex ki;
  ki.d = g.d;
  ki.N0 = g.N[0];
  ki.N1 = g.d == 3 ? g.N[1] : 1;
  ki.N2 = g.d == 3 ? g.N[2] : g.N[1];
  ki.H = g.H;
  return ki;
}

template <typename V>
void half_mul_grad(lrfg_ctx* ctx, const FullGrid& g, const V* in, V* out, int alpha, double scale) {
  LRFG_LAUNCH(ctx, KC_POINTWISE, 2.0 * g.n_half, 2.0 * sizeof(V) * g.n_half,
              mul_grad_kernel<V><<<grid1d(ctx, g.n_half), 256, 0, ctx->stream>>>(in, out, g.n_half, kindex(g), alpha,
                                                                                  scale));
}

template <typename V>
void half_acc_div(lrfg_ctx* ctx, const FullGrid& g, const V* in, V* acc, int alpha, double scale, int init,
                  int precond) {
  LRFG_LAUNCH(ctx, KC_POINTWISE, 4.0 * g.n_half, (init ? 2.0 : 3.0) * sizeof(V) * g.n_half,
              acc_div_kernel<V><<<grid1d(ctx, g.n_half), 256, 0, ctx->stream>>>(in, acc, g.n_half, kindex(g), alpha,
                                                                                 scale, init, precond));
}

template <typename V>
void half_precond(lrfg_ctx* ctx, const FullGrid& g, const V* in, V* out) {
  LRFG_LAUNCH(ctx, KC_POINTWISE, 2.0 * g.n_half, 2.0 * sizeof(V) * g.n_half,
              precond_kernel<V><<<grid1d(ctx, g.n_half), 256, 0, ctx->stream>>>(in, out, g.n_half, kindex(g)));
}

// ------------------------------------------------------------------------------------------------
// reductions (accumulated in FP64 whatever the storage type): Hermitian-weighted inner product of
// half spectra, and the A_eff energy density
// ------------------------------------------------------------------------------------------------
constexpr int kRedBlocks = 304;

template <typename V>
__global__ void __launch_bounds__(256) half_dot_kernel(const V* __restrict__ x, const V* __restrict__ y, long long n,
                                                       int H, double* partial) {
  __shared__ double red[8];
  double s = 0.0;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x) {
    V a = x[t], b = y[t];
    double w = (t % H) == 0 ? 1.0 : 2.0;
    s += w * ((double)a.x * (double)b.x + (double)a.y * (double)b.y);
  }
  for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffff, s, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double v = 0.0;
    for (int i = 0; i < 8; ++i) v += red[i];
    partial[blockIdx.x] = v;
  }
}

template <typename R>
__global__ void __launch_bounds__(256) energy_kernel(const R* __restrict__ e, const R* __restrict__ a, double E,
                                                     long long n, double* partial) {
  __shared__ double red[8];
  double s = 0.0;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x) {
    double f = E + (double)e[t];
    s += (double)a[t] * f * f;
  }
  for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffff, s, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double v = 0.0;
    for (int i = 0; i < 8; ++i) v += red[i];
    partial[blockIdx.x] = v;
  }
}

__global__ void finish_sum_kernel(const double* __restrict__ partial, int n, double* out, int accumulate) {
  __shared__ double red[8];
  double s = 0.0;
  for (int t = threadIdx.x; t < n; t += blockDim.x) s += partial[t];
  for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffff, s, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double v = 0.0;
    for (int i = 0; i < 8; ++i) v += red[i];
    *out = accumulate ? *out + v : v;
  }
}

template <typename V>
void half_dot(lrfg_ctx* ctx, const FullGrid& g, const V* x, const V* y, double* out_dev) {
  DBuf<double> partial(ctx->pool, kRedBlocks);
  LRFG_LAUNCH(ctx, KC_REDUCE, 4.0 * g.n_half, 2.0 * sizeof(V) * g.n_half,
              half_dot_kernel<V><<<kRedBlocks, 256, 0, ctx->stream>>>(x, y, g.n_half, g.H, partial.get()));
  LRFG_LAUNCH(ctx, KC_REDUCE, kRedBlocks, kRedBlocks * sizeof(double),
              finish_sum_kernel<<<1, 256, 0, ctx->stream>>>(partial.get(), kRedBlocks, out_dev, 0));
}

template <typename R>
void energy_sum(lrfg_ctx* ctx, const FullGrid& g, const R* e, const R* a, double E, double* out_dev, int accumulate) {
  DBuf<double> partial(ctx->pool, kRedBlocks);
  LRFG_LAUNCH(ctx, KC_REDUCE, 4.0 * g.n_real, 2.0 * sizeof(R) * g.n_real,
              energy_kernel<R><<<kRedBlocks, 256, 0, ctx->stream>>>(e, a, E, g.n_real, partial.get()));
  LRFG_LAUNCH(ctx, KC_REDUCE, kRedBlocks, kRedBlocks * sizeof(double),
              finish_sum_kernel<<<1, 256, 0, ctx->stream>>>(partial.get(), kRedBlocks, out_dev, accumulate));
}

// ------------------------------------------------------------------------------------------------
// PCG vector updates with device FP64 scalars: alpha = num / den
// ------------------------------------------------------------------------------------------------
template <typename V>
__global__ void pcg_update_kernel(V* u, V* r, const V* __restrict__ p, const V* __restrict__ q, V* z, long long n,
                                  KIndex ki, const double* __restrict__ num, const double* __restrict__ den) {
  using R = typename RealOf<V>::T;
  const double ad = (*den != 0.0) ? (*num) / (*den) : 0.0;
  const R alpha = (R)ad;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x) {
    V pv = p[t], qv = q[t], uv = u[t], rv = r[t];
    uv.x += alpha * pv.x;
    uv.y += alpha * pv.y;
    rv.x -= alpha * qv.x;
    rv.y -= alpha * qv.y;
    u[t] = uv;
    r[t] = rv;
    int k[3];
    kvec(t, ki, k);
    const int kk = k[0] * k[0] + k[1] * k[1] + k[2] * k[2];
    const R s = kk > 0 ? (R)(1.0 / (double)kk) : R(0);
    z[t] = mkc<V>(rv.x * s, rv.y * s);
  }
}

// p = z + (num/den) p
template <typename V>
__global__ void pcg_direction_kernel(V* p, const V* __restrict__ z, long long n, const double* __restrict__ num,
                                     const double* __restrict__ den) {
  using R = typename RealOf<V>::T;
  const double bd = (*den != 0.0) ? (*num) / (*den) : 0.0;
  const R beta = (R)bd;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x) {
    V pv = p[t], zv = z[t];
    p[t] = mkc<V>(zv.x + beta * pv.x, zv.y + beta * pv.y);
  }
}

template <typename V>
void pcg_update(lrfg_ctx* ctx, const FullGrid& g, V* u, V* r, const V* p, const V* q, V* z, const double* num,
                const double* den) {
  LRFG_LAUNCH(ctx, KC_POINTWISE, 10.0 * g.n_half, 7.0 * sizeof(V) * g.n_half,
              pcg_update_kernel<V><<<grid1d(ctx, g.n_half), 256, 0, ctx->stream>>>(u, r, p, q, z, g.n_half, kindex(g),
                                                                                    num, den));
}

template <typename V>
void pcg_direction(lrfg_ctx* ctx, const FullGrid& g, V* p, const V* z, const double* num, const double* den) {
  LRFG_LAUNCH(ctx, KC_POINTWISE, 4.0 * g.n_half, 3.0 * sizeof(V) * g.n_half,
              pcg_direction_kernel<V><<<grid1d(ctx, g.n_half), 256, 0, ctx->stream>>>(p, z, g.n_half, num, den));
}

// element-wise conversions between storage precisions (round to nearest)
__device__ __forceinline__ float cvt(double x, float*) { return (float)x; }
__device__ __forceinline__ double cvt(float x, double*) { return (double)x; }
__device__ __forceinline__ float2 cvt(double2 x, float2*) { return make_float2((float)x.x, (float)x.y); }
__device__ __forceinline__ double2 cvt(float2 x, double2*) { return make_double2((double)x.x, (double)x.y); }

template <typename A, typename B>
__global__ void convert_kernel(const A* __restrict__ in, B* out, long long n) {
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x)
    out[t] = cvt(in[t], (B*)nullptr);
}

template <typename A, typename B>
void convert(lrfg_ctx* ctx, const A* in, B* out, long long n) {
  if (n <= 0) return;
  LRFG_LAUNCH(ctx, KC_POINTWISE, 0, (sizeof(A) + sizeof(B)) * (double)n,
              convert_kernel<A, B><<<grid1d(ctx, n), 256, 0, ctx->stream>>>(in, out, n));
}

#define LRFG_FULL_INSTANTIATE(V, R)                                                                         \
  template void half_mul_grad<V>(lrfg_ctx*, const FullGrid&, const V*, V*, int, double);                  \
  template void half_acc_div<V>(lrfg_ctx*, const FullGrid&, const V*, V*, int, double, int, int);         \
  template void half_precond<V>(lrfg_ctx*, const FullGrid&, const V*, V*);                                \
  template void half_dot<V>(lrfg_ctx*, const FullGrid&, const V*, const V*, double*);                    \
  template void energy_sum<R>(lrfg_ctx*, const FullGrid&, const R*, const R*, double, double*, int);      \
  template void pcg_update<V>(lrfg_ctx*, const FullGrid&, V*, V*, const V*, const V*, V*, const double*,   \
                              const double*);                                                             \
  template void pcg_direction<V>(lrfg_ctx*, const FullGrid&, V*, const V*, const double*, const double*);
LRFG_FULL_INSTANTIATE(double2, double)
LRFG_FULL_INSTANTIATE(float2, float)
template void convert<double, float>(lrfg_ctx*, const double*, float*, long long);
template void convert<float, double>(lrfg_ctx*, const float*, double*, long long);
template void convert<double2, float2>(lrfg_ctx*, const double2*, float2*, long long);
template void convert<float2, double2>(lrfg_ctx*, const float2*, double2*, long long);

}  // namespace lrfg
