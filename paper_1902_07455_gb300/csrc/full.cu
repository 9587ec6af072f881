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
__global__ void __launch_bounds__(256) r2c_rows_kernel(const double* __restrict__ in, const double* __restrict__ coef,
                                                       double scale, double2* __restrict__ out, long long rows, int N,
                                                       int H, int TF, FftPlan pl, const double2* __restrict__ Wg) {
  extern __shared__ double2 sm[];
  double2* W = sm;
  double2* a = sm + 2 * N;
  double2* b = a + (size_t)TF * N;
  for (int j = threadIdx.x; j < N; j += blockDim.x) W[j] = Wg[j];
  const long long r0 = (long long)blockIdx.x * 2 * TF;
  const int nr = (int)min(2LL * TF, rows - r0);
  const int nrow = min(nr, TF);
  for (int t = threadIdx.x; t < nrow * N; t += blockDim.x) a[t] = make_double2(0.0, 0.0);
  __syncthreads();
  for (int t = threadIdx.x; t < nr * N; t += blockDim.x) {
    int f = t / N, n = t - (t / N) * N;
    size_t gi = (size_t)(r0 + f) * N + n;
    double v = in[gi];
    if (coef) v *= coef[gi];
    v *= scale;
    if (f < TF) a[(size_t)f * N + n].x = v; else a[(size_t)(f - TF) * N + n].y = v;
  }
  __syncthreads();
  double2* Z = stockham_rows<-1>(a, b, nrow, N, pl, W);
  // split: X[k] = (Z[k] + conj Z[N-k]) / 2,  Y[k] = (Z[k] - conj Z[N-k]) / (2i)
  for (int t = threadIdx.x; t < nr * H; t += blockDim.x) {
    int f = t / H, k = t - (t / H) * H;
    int row = f < TF ? f : f - TF;
    double2 z = Z[(size_t)row * N + k];
    double2 zc = Z[(size_t)row * N + ((N - k) % N)];
    double2 v;
    if (f < TF) v = make_double2(0.5 * (z.x + zc.x), 0.5 * (z.y - zc.y));
    else v = make_double2(0.5 * (z.y + zc.y), -0.5 * (z.x - zc.x));
    out[(size_t)(r0 + f) * H + k] = v;
  }
}

// half spectra -> real rows (inverse, unnormalised), optional post-multiplication by a coefficient
__global__ void __launch_bounds__(256) c2r_rows_kernel(const double2* __restrict__ in, const double* __restrict__ coef,
                                                       double scale, double* __restrict__ out, long long rows, int N,
                                                       int H, int TF, FftPlan pl, const double2* __restrict__ Wg) {
  extern __shared__ double2 sm[];
  double2* W = sm;
  double2* a = sm + 2 * N;
  double2* b = a + (size_t)TF * N;
  for (int j = threadIdx.x; j < N; j += blockDim.x) W[j] = Wg[j];
  const long long r0 = (long long)blockIdx.x * 2 * TF;
  const int nr = (int)min(2LL * TF, rows - r0);
  const int nrow = min(nr, TF);
  for (int t = threadIdx.x; t < nrow * N; t += blockDim.x) a[t] = make_double2(0.0, 0.0);
  __syncthreads();
  // Z[k] = X[k] + i Y[k] over the full range, X[N-k] = conj X[k]; one thread per (row, k)
  for (int t = threadIdx.x; t < nrow * N; t += blockDim.x) {
    int row = t / N, k = t - (t / N) * N;
    double2 z = make_double2(0.0, 0.0);
    for (int half = 0; half < 2; ++half) {
      int f = row + half * TF;
      if (f >= nr) break;
      double2 x;
      if (k < H) x = in[(size_t)(r0 + f) * H + k];
      else { x = in[(size_t)(r0 + f) * H + (N - k)]; x.y = -x.y; }
      if (half == 0) { z.x += x.x; z.y += x.y; } else { z.x -= x.y; z.y += x.x; }
    }
    a[(size_t)row * N + k] = z;
  }
  __syncthreads();
  double2* Z = stockham_rows<1>(a, b, nrow, N, pl, W);
  for (int t = threadIdx.x; t < nr * N; t += blockDim.x) {
    int f = t / N, n = t - (t / N) * N;
    int row = f < TF ? f : f - TF;
    double2 z = Z[(size_t)row * N + n];
    double v = (f < TF ? z.x : z.y) * scale;
    size_t gi = (size_t)(r0 + f) * N + n;
    if (coef) v *= coef[gi];
    out[gi] = v;
  }
}

static int row_tile(lrfg_ctx* ctx, int N, size_t* smem) {
  size_t limit = 100 * 1024;
  if (N > 300) limit = (size_t)std::min(ctx->max_smem_optin, 200 * 1024);
  long long per = 2LL * N * (long long)sizeof(double2);
  long long tf = ((long long)limit - 2LL * N * (long long)sizeof(double2)) / per;
  tf = std::max(1LL, std::min(tf, 32LL));
  *smem = (size_t)(2LL * N * sizeof(double2) + tf * per);
  return (int)tf;
}

void full_forward(lrfg_ctx* ctx, const FullGrid& g, const double* real_in, const double* coef, double scale,
                  double2* half_out) {
  const int N = g.N[g.d - 1];
  FftPlan pl = make_plan(N);
  const Twiddles& tw = twiddles_for(ctx, N);
  size_t smem;
  int TF = row_tile(ctx, N, &smem);
  long long blocks = (g.rows + 2LL * TF - 1) / (2LL * TF);
  LRFG_CUDA(cudaFuncSetAttribute(r2c_rows_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  LRFG_LAUNCH(ctx, KC_R2C, 2.5 * N * std::log2((double)N) * (double)g.rows,
              (double)g.rows * (N * sizeof(double) * (coef ? 2 : 1) + g.H * sizeof(double2)),
              r2c_rows_kernel<<<(unsigned)blocks, 256, smem, ctx->stream>>>(real_in, coef, scale, half_out, g.rows, N,
                                                                             g.H, TF, pl, tw.W));
  // complex axes, innermost first
  long long inner = g.H;
  for (int ax = g.d - 2; ax >= 0; --ax) {
    long long outer = 1;
    for (int j = 0; j < ax; ++j) outer *= g.N[j];
    fft_fibres(ctx, half_out, half_out, outer, g.N[ax], inner, -1);
    inner *= g.N[ax];
  }
}

void full_inverse(lrfg_ctx* ctx, const FullGrid& g, double2* half_inout, const double* coef, double scale,
                  double* real_out) {
  long long inner = g.n_half;
  for (int ax = 0; ax <= g.d - 2; ++ax) {
    inner /= g.N[ax];
    long long outer = g.n_half / (inner * g.N[ax]);
    fft_fibres(ctx, half_inout, half_inout, outer, g.N[ax], inner, 1);
  }
  const int N = g.N[g.d - 1];
  FftPlan pl = make_plan(N);
  const Twiddles& tw = twiddles_for(ctx, N);
  size_t smem;
  int TF = row_tile(ctx, N, &smem);
  long long blocks = (g.rows + 2LL * TF - 1) / (2LL * TF);
  LRFG_CUDA(cudaFuncSetAttribute(c2r_rows_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  LRFG_LAUNCH(ctx, KC_C2R, 2.5 * N * std::log2((double)N) * (double)g.rows,
              (double)g.rows * (N * sizeof(double) * (coef ? 2 : 1) + g.H * sizeof(double2)),
              c2r_rows_kernel<<<(unsigned)blocks, 256, smem, ctx->stream>>>(half_inout, coef, scale, real_out, g.rows,
                                                                             N, g.H, TF, pl, tw.W));
}

// ------------------------------------------------------------------------------------------------
// pointwise Fourier multipliers on the half spectrum
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
__global__ void mul_grad_kernel(const double2* __restrict__ in, double2* out, long long n, KIndex ki, int alpha,
                                double scale) {
  const double two_pi = 6.283185307179586476925286766559;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x) {
    int k[3];
    kvec(t, ki, k);
    double f = two_pi * (double)k[alpha] * scale;
    double2 v = in[t];
    out[t] = make_double2(-v.y * f, v.x * f);
  }
}

// acc = (init ? 0 : acc) + in * (-2 pi i k_alpha) * scale; if precond, then acc /= k.k (0 at k=0)
__global__ void acc_div_kernel(const double2* __restrict__ in, double2* acc, long long n, KIndex ki, int alpha,
                               double scale, int init, int precond) {
  const double two_pi = 6.283185307179586476925286766559;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x) {
    int k[3];
    kvec(t, ki, k);
    double f = -two_pi * (double)k[alpha] * scale;
    double2 v = in[t];
    double2 r = make_double2(-v.y * f, v.x * f);
    if (!init) { double2 o = acc[t]; r.x += o.x; r.y += o.y; }
    if (precond) {
      double kk = (double)k[0] * k[0] + (double)k[1] * k[1] + (double)k[2] * k[2];
      double s = kk > 0.0 ? 1.0 / kk : 0.0;
      r.x *= s;
      r.y *= s;
    }
    acc[t] = r;
  }
}

__global__ void precond_kernel(const double2* __restrict__ in, double2* out, long long n, KIndex ki) {
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x) {
    int k[3];
    kvec(t, ki, k);
    double kk = (double)k[0] * k[0] + (double)k[1] * k[1] + (double)k[2] * k[2];
    double s = kk > 0.0 ? 1.0 / kk : 0.0;
    double2 v = in[t];
    out[t] = make_double2(v.x * s, v.y * s);
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

void half_mul_grad(lrfg_ctx* ctx, const FullGrid& g, const double2* in, double2* out, int alpha, double scale) {
  LRFG_LAUNCH(ctx, KC_POINTWISE, 2.0 * g.n_half, 2.0 * sizeof(double2) * g.n_half,
              mul_grad_kernel<<<grid1d(ctx, g.n_half), 256, 0, ctx->stream>>>(in, out, g.n_half, kindex(g), alpha,
                                                                               scale));
}

void half_acc_div(lrfg_ctx* ctx, const FullGrid& g, const double2* in, double2* acc, int alpha, double scale, int init,
                  int precond) {
  LRFG_LAUNCH(ctx, KC_POINTWISE, 4.0 * g.n_half, (init ? 2.0 : 3.0) * sizeof(double2) * g.n_half,
              acc_div_kernel<<<grid1d(ctx, g.n_half), 256, 0, ctx->stream>>>(in, acc, g.n_half, kindex(g), alpha, scale,
                                                                              init, precond));
}

void half_precond(lrfg_ctx* ctx, const FullGrid& g, const double2* in, double2* out) {
  LRFG_LAUNCH(ctx, KC_POINTWISE, 2.0 * g.n_half, 2.0 * sizeof(double2) * g.n_half,
              precond_kernel<<<grid1d(ctx, g.n_half), 256, 0, ctx->stream>>>(in, out, g.n_half, kindex(g)));
}

// ------------------------------------------------------------------------------------------------
// reductions: Hermitian-weighted inner product of half spectra, and the A_eff energy density
// ------------------------------------------------------------------------------------------------
constexpr int kRedBlocks = 304;

__global__ void __launch_bounds__(256) half_dot_kernel(const double2* __restrict__ x, const double2* __restrict__ y,
                                                       long long n, int H, double* partial) {
  __shared__ double red[8];
  double s = 0.0;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x) {
    double2 a = x[t], b = y[t];
    double w = (t % H) == 0 ? 1.0 : 2.0;
    s += w * (a.x * b.x + a.y * b.y);
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

__global__ void __launch_bounds__(256) energy_kernel(const double* __restrict__ e, const double* __restrict__ a,
                                                     double E, long long n, double* partial) {
  __shared__ double red[8];
  double s = 0.0;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x) {
    double f = E + e[t];
    s += a[t] * f * f;
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

void half_dot(lrfg_ctx* ctx, const FullGrid& g, const double2* x, const double2* y, double* out_dev) {
  DBuf<double> partial(ctx->pool, kRedBlocks);
  LRFG_LAUNCH(ctx, KC_REDUCE, 4.0 * g.n_half, 2.0 * sizeof(double2) * g.n_half,
              half_dot_kernel<<<kRedBlocks, 256, 0, ctx->stream>>>(x, y, g.n_half, g.H, partial.get()));
  LRFG_LAUNCH(ctx, KC_REDUCE, kRedBlocks, kRedBlocks * sizeof(double),
              finish_sum_kernel<<<1, 256, 0, ctx->stream>>>(partial.get(), kRedBlocks, out_dev, 0));
}

void energy_sum(lrfg_ctx* ctx, const FullGrid& g, const double* e, const double* a, double E, double* out_dev,
                int accumulate) {
  DBuf<double> partial(ctx->pool, kRedBlocks);
  LRFG_LAUNCH(ctx, KC_REDUCE, 4.0 * g.n_real, 2.0 * sizeof(double) * g.n_real,
              energy_kernel<<<kRedBlocks, 256, 0, ctx->stream>>>(e, a, E, g.n_real, partial.get()));
  LRFG_LAUNCH(ctx, KC_REDUCE, kRedBlocks, kRedBlocks * sizeof(double),
              finish_sum_kernel<<<1, 256, 0, ctx->stream>>>(partial.get(), kRedBlocks, out_dev, accumulate));
}

// ------------------------------------------------------------------------------------------------
// PCG vector updates with device scalars: alpha = s[0] / s[1]
// ------------------------------------------------------------------------------------------------
__global__ void pcg_update_kernel(double2* u, double2* r, const double2* __restrict__ p, const double2* __restrict__ q,
                                  double2* z, long long n, KIndex ki, const double* __restrict__ num,
                                  const double* __restrict__ den) {
  const double alpha = (*den != 0.0) ? (*num) / (*den) : 0.0;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x) {
    double2 pv = p[t], qv = q[t], uv = u[t], rv = r[t];
    uv.x += alpha * pv.x;
    uv.y += alpha * pv.y;
    rv.x -= alpha * qv.x;
    rv.y -= alpha * qv.y;
    u[t] = uv;
    r[t] = rv;
    int k[3];
    kvec(t, ki, k);
    double kk = (double)k[0] * k[0] + (double)k[1] * k[1] + (double)k[2] * k[2];
    double s = kk > 0.0 ? 1.0 / kk : 0.0;
    z[t] = make_double2(rv.x * s, rv.y * s);
  }
}

// p = z + (num/den) p
__global__ void pcg_direction_kernel(double2* p, const double2* __restrict__ z, long long n,
                                     const double* __restrict__ num, const double* __restrict__ den) {
  const double beta = (*den != 0.0) ? (*num) / (*den) : 0.0;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x) {
    double2 pv = p[t], zv = z[t];
    p[t] = make_double2(zv.x + beta * pv.x, zv.y + beta * pv.y);
  }
}

void pcg_update(lrfg_ctx* ctx, const FullGrid& g, double2* u, double2* r, const double2* p, const double2* q,
                double2* z, const double* num, const double* den) {
  LRFG_LAUNCH(ctx, KC_POINTWISE, 10.0 * g.n_half, 7.0 * sizeof(double2) * g.n_half,
              pcg_update_kernel<<<grid1d(ctx, g.n_half), 256, 0, ctx->stream>>>(u, r, p, q, z, g.n_half, kindex(g), num,
                                                                                 den));
}

void pcg_direction(lrfg_ctx* ctx, const FullGrid& g, double2* p, const double2* z, const double* num,
                   const double* den) {
  LRFG_LAUNCH(ctx, KC_POINTWISE, 4.0 * g.n_half, 3.0 * sizeof(double2) * g.n_half,
              pcg_direction_kernel<<<grid1d(ctx, g.n_half), 256, 0, ctx->stream>>>(p, z, g.n_half, num, den));
}

}  // namespace lrfg
