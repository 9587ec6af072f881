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

// half spectra -> real rows -> times the coefficient -> half spectra, in one pass over the rows: the C2R pass,
// the material product and the R2C pass of the operator fused, so the real grid never goes to memory.  Both
// directions pair rows f and f + TF in one complex FFT (real and imaginary parts), so after the inverse
// transform the product acts on the two parts in place and the forward transform runs on the result as is.
// `in` and `out` may alias (a block reads all of its rows before it writes them).
template <typename R>
__global__ void __launch_bounds__(256, 3) c2r_mul_r2c_rows_kernel(const typename CplxOf<R>::T* in,
                                                               const R* __restrict__ coef, R scale,
                                                               typename CplxOf<R>::T* out, long long rows, int N,
                                                               int H, int TF, FftPlan pl,
                                                               const typename CplxOf<R>::T* __restrict__ Wg) {
  using V = typename CplxOf<R>::T;
  const float invN = 1.0f / (float)N, invH = 1.0f / (float)H;
  extern __shared__ __align__(16) unsigned char smraw_fused[];
  V* sm = (V*)smraw_fused;
  V* W = sm;
  V* a = sm + 2 * N;
  V* b = a + (size_t)TF * N;
  for (int j = threadIdx.x; j < N; j += blockDim.x) W[j] = Wg[j];
  const long long r0 = (long long)blockIdx.x * 2 * TF;
  const int nr = (int)min(2LL * TF, rows - r0);
  const int nrow = min(nr, TF);
  // Z[k] = X[k] + i Y[k] over the full range from the two half spectra (X[N-k] = conj X[k])
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
  // the product with the coefficient on both real rows of each complex row, in place
  {
    constexpr int kU = 4;
    const int total = nrow * N;
    const R* c0 = coef + (size_t)r0 * N;
    for (int base = threadIdx.x; base < total; base += kU * blockDim.x) {
      R ca[kU], cb[kU];
#pragma unroll
      for (int u = 0; u < kU; ++u) {
        const int t = base + u * blockDim.x;
        ca[u] = R(0);
        cb[u] = R(0);
        if (t < total) {
          const int row = small_div(t, N, invN);
          ca[u] = c0[t];
          if (row + TF < nr) cb[u] = c0[t + (size_t)TF * N];
        }
      }
#pragma unroll
      for (int u = 0; u < kU; ++u) {
        const int t = base + u * blockDim.x;
        if (t < total) {
          const V z = Z[t];
          Z[t] = mkc<V>(z.x * scale * ca[u], z.y * scale * cb[u]);
        }
      }
    }
  }
  __syncthreads();
  V* Z2 = stockham_rows<-1>(Z, Z == a ? b : a, nrow, N, pl, (const V*)W);
  // split: X[k] = (Z[k] + conj Z[N-k]) / 2,  Y[k] = (Z[k] - conj Z[N-k]) / (2i)
  for (int t = threadIdx.x; t < nr * H; t += blockDim.x) {
    const int f = small_div(t, H, invH), k = t - f * H;
    const int row = f < TF ? f : f - TF;
    const V z = Z2[(size_t)row * N + k];
    const V zc = Z2[(size_t)row * N + ((N - k) % N)];
    V v;
    if (f < TF) v = mkc<V>(R(0.5) * (z.x + zc.x), R(0.5) * (z.y - zc.y));
    else v = mkc<V>(R(0.5) * (z.y + zc.y), R(-0.5) * (z.x - zc.x));
    out[(size_t)(r0 + f) * H + k] = v;
  }
}

// ------------------------------------------------------------------------------------------------
// FP32 rows of length N = P1 P2: the fused C2R -> product -> R2C pass of the operator with the two
// register passes of fft2_fibres_kernel per direction, over a tile of 32 complex rows (real rows r0 + j
// and r0 + 32 + j in the real and imaginary parts of complex row j).  The tile lives once in shared
// memory as Z[n][j] with row stride 33 (conflict-free both along n and along j); every pass reads its
// inputs to registers, waits at a barrier and writes its outputs in place, so no second buffer is needed
// and three blocks fit an SM.  Global traffic is coalesced along each row: the half spectra in, the
// coefficient rows, the half spectra out.  `in` and `out` may alias (a block reads all its rows first).
// ------------------------------------------------------------------------------------------------
constexpr int kRowsLd = 33;

// one Stockham pass pair of the transform of the tile, in place (see the header of fft_device.cuh):
// pass 1 radix P1 (warp w = c < P2 takes x[c + P2 r]), pass 2 radix P2 with w_N^{f r} (f = w + P2 jb)
template <int SIGN, int P1, int P2>
__device__ __forceinline__ void rows2_transform(float2* Z, const float2* W, int w, int lane) {
  constexpr int N = P1 * P2;
  {
    float2 x[P1];
#pragma unroll
    for (int r = 0; r < P1; ++r) x[r] = Z[(w + P2 * r) * kRowsLd + lane];
    __syncthreads();
    RegDFT<P1, SIGN, float2>::run(x);
#pragma unroll
    for (int q = 0; q < P1; ++q) Z[(w * P1 + q) * kRowsLd + lane] = x[q];
  }
  __syncthreads();
  {
    float2 y[P1 / P2][P2];
#pragma unroll
    for (int jb = 0; jb < P1 / P2; ++jb)
#pragma unroll
      for (int r = 0; r < P2; ++r) y[jb][r] = Z[(r * P1 + w + P2 * jb) * kRowsLd + lane];
    __syncthreads();
#pragma unroll
    for (int jb = 0; jb < P1 / P2; ++jb) {
      const int f = w + P2 * jb;
#pragma unroll
      for (int r = 1; r < P2; ++r) y[jb][r] = cmul(y[jb][r], tw<SIGN>(W, f * r));
      RegDFT<P2, SIGN, float2>::run(y[jb]);
#pragma unroll
      for (int q = 0; q < P2; ++q) Z[(f + P1 * q) * kRowsLd + lane] = y[jb][q];
    }
  }
  __syncthreads();
  (void)N;
}

template <int P1, int P2>
__global__ void __launch_bounds__(32 * P2, 3) rows2_mul_kernel(const float2* in, const float* __restrict__ coef,
                                                              float scale, float2* out, long long rows,
                                                              const float2* __restrict__ Wg) {
  constexpr int N = P1 * P2, H = (N + 1) / 2, NT = 32 * P2;
  extern __shared__ __align__(16) unsigned char smraw_rows2[];
  float2* Z = (float2*)smraw_rows2;  // [N][kRowsLd]
  float2* W = Z + N * kRowsLd;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const long long r0 = (long long)blockIdx.x * 64;
  const int nr = (int)min(64LL, rows - r0);  // real rows of this tile: j < nr (real parts), 32 + j < nr (imaginary)
  for (int j = threadIdx.x; j < N; j += NT) W[j] = Wg[j];
  // Z[k] = X[k] + i Y[k] and Z[N - k] = conj X[k] + i conj Y[k] from the two half spectra
  {
    // the tile's loads in two rounds of requests (two latencies per block)
    constexpr int total = 32 * H;
    constexpr int kU = (total + 2 * NT - 1) / (2 * NT);
    for (int e0 = threadIdx.x; e0 < total; e0 += kU * NT) {
      float2 a[kU], b[kU];
#pragma unroll
      for (int u = 0; u < kU; ++u) {
        const int e = e0 + u * NT;
        const int j = e / H;
        a[u] = make_float2(0.f, 0.f);
        b[u] = make_float2(0.f, 0.f);
        if (e < total && j < nr) a[u] = in[(size_t)r0 * H + e];
        if (e < total && j + 32 < nr) b[u] = in[(size_t)(r0 + 32) * H + e];
      }
#pragma unroll
      for (int u = 0; u < kU; ++u) {
        const int e = e0 + u * NT;
        if (e < total) {
          const int j = e / H, k = e - j * H;
          Z[k * kRowsLd + j] = make_float2(a[u].x - b[u].y, a[u].y + b[u].x);
          if (k) Z[(N - k) * kRowsLd + j] = make_float2(a[u].x + b[u].y, b[u].x - a[u].y);
        }
      }
    }
  }
  __syncthreads();
  rows2_transform<1, P1, P2>(Z, W, w, lane);
  // the real rows times the coefficient: Z[n][j] = (x_j[n], x_{32+j}[n]); each thread's coefficients are
  // requested before any is used
  {
    constexpr int per = (32 * N + NT - 1) / NT;
    const float* c0 = coef + (size_t)r0 * N;
    float ca[per], cb[per];
#pragma unroll
    for (int u = 0; u < per; ++u) {
      const int e = threadIdx.x + u * NT;
      const int j = e / N;
      ca[u] = (e < 32 * N && j < nr) ? c0[e] : 0.f;
      cb[u] = (e < 32 * N && j + 32 < nr) ? c0[(size_t)32 * N + e] : 0.f;
    }
#pragma unroll
    for (int u = 0; u < per; ++u) {
      const int e = threadIdx.x + u * NT;
      if (e < 32 * N) {
        const int j = e / N, n = e - j * N;
        float2* p = Z + n * kRowsLd + j;
        const float2 z = *p;
        *p = make_float2(z.x * scale * ca[u], z.y * scale * cb[u]);
      }
    }
  }
  __syncthreads();
  rows2_transform<-1, P1, P2>(Z, W, w, lane);
  // split: X[k] = (Z[k] + conj Z[N-k]) / 2, Y[k] = (Z[k] - conj Z[N-k]) / (2i)
  {
    constexpr int total = 32 * H;
    for (int e = threadIdx.x; e < total; e += NT) {
      const int j = e / H, k = e - j * H;
      const float2 z = Z[k * kRowsLd + j];
      const float2 zc = Z[(k ? N - k : 0) * kRowsLd + j];
      if (j < nr) out[(size_t)r0 * H + e] = make_float2(0.5f * (z.x + zc.x), 0.5f * (z.y - zc.y));
      if (j + 32 < nr) out[(size_t)(r0 + 32) * H + e] = make_float2(0.5f * (z.y + zc.y), -0.5f * (z.x - zc.x));
    }
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
  LRFG_CUDA(raise_smem_limit((const void*)r2c_rows_kernel<R>, smem));
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
  LRFG_CUDA(raise_smem_limit((const void*)c2r_rows_kernel<R>, smem));
  LRFG_LAUNCH(ctx, KC_C2R, 2.5 * N * std::log2((double)N) * (double)g.rows,
              (double)g.rows * (N * sizeof(R) * (coef ? 2 : 1) + g.H * sizeof(V)),
              c2r_rows_kernel<R><<<(unsigned)blocks, 256, smem, ctx->stream>>>(half_inout, coef, scale, real_out, g.rows,
                                                                                N, g.H, TF, pl, W));
}

template <int P1, int P2>
static void rows2_launch(lrfg_ctx* ctx, const FullGrid& g, float2* half_inout, const float* coef, float scale) {
  constexpr int N = P1 * P2;
  const size_t smem = sizeof(float2) * (size_t)N * (kRowsLd + 1);
  const long long blocks = (g.rows + 63) / 64;
  LRFG_REQUIRE(blocks < (1LL << 31), "too many rows");
  const float2* W = twiddle_table<float>(ctx, N);
  LRFG_CUDA(raise_smem_limit((const void*)rows2_mul_kernel<P1, P2>, smem));
  LRFG_LAUNCH(ctx, KC_ROWS_FUSED, 5.0 * N * std::log2((double)N) * (double)g.rows,
              (double)g.rows * (2.0 * g.H * sizeof(float2) + N * sizeof(float)),
              rows2_mul_kernel<P1, P2><<<(unsigned)blocks, 32 * P2, smem, ctx->stream>>>(half_inout, coef, scale,
                                                                                        half_inout, g.rows, W));
}

template <typename R>
void full_rows_mul(lrfg_ctx* ctx, const FullGrid& g, typename CplxOf<R>::T* half_inout, const R* coef, R scale) {
  using V = typename CplxOf<R>::T;
  const int N = g.N[g.d - 1];
  if constexpr (sizeof(R) == sizeof(float)) {
    LRFG_CUDA(ensure_roots(ctx->device));
    if (N == 243) return rows2_launch<27, 9>(ctx, g, half_inout, coef, scale);
    if (N == 81) return rows2_launch<9, 9>(ctx, g, half_inout, coef, scale);
  }
  FftPlan pl = make_plan(N, plan_radix<V>());
  LRFG_CUDA(ensure_roots(ctx->device));
  const V* W = twiddle_table<R>(ctx, N);
  size_t smem;
  int TF = row_tile<R>(ctx, N, &smem);
  long long blocks = (g.rows + 2LL * TF - 1) / (2LL * TF);
  LRFG_CUDA(raise_smem_limit((const void*)c2r_mul_r2c_rows_kernel<R>, smem));
  LRFG_LAUNCH(ctx, KC_ROWS_FUSED, 5.0 * N * std::log2((double)N) * (double)g.rows,
              (double)g.rows * (2.0 * g.H * sizeof(V) + N * sizeof(R)),
              c2r_mul_r2c_rows_kernel<R><<<(unsigned)blocks, 256, smem, ctx->stream>>>(
                  half_inout, coef, scale, half_inout, g.rows, N, g.H, TF, pl, W));
}

template void full_rows_mul<double>(lrfg_ctx*, const FullGrid&, double2*, const double*, double);
template void full_rows_mul<float>(lrfg_ctx*, const FullGrid&, float2*, const float*, float);

template void full_forward<double>(lrfg_ctx*, const FullGrid&, const double*, const double*, double, double2*);
template void full_forward<float>(lrfg_ctx*, const FullGrid&, const float*, const float*, float, float2*);
template void full_inverse<double>(lrfg_ctx*, const FullGrid&, double2*, const double*, double, double*);
template void full_inverse<float>(lrfg_ctx*, const FullGrid&, float2*, const float*, float, float*);

// ------------------------------------------------------------------------------------------------
// pointwise Fourier multipliers on the half spectrum.  Launch map: blockIdx.x = row (all indices but
// the last), blockIdx.y * blockDim.x + threadIdx.x = k_last, so a thread finds its frequencies without
// per-element division.  Multipliers are formed in the storage precision R from R-rounded constants;
// 1/(k.k) comes from a table of exactly rounded reciprocals (no per-element division).
// ------------------------------------------------------------------------------------------------
struct RowMap {
  int d, N0, N1, H;
};

static RowMap rowmap(const FullGrid& g) {
  RowMap m;
  m.d = g.d;
  m.N0 = g.N[0];
  m.N1 = g.d == 3 ? g.N[1] : 1;
  m.H = g.H;
  return m;
}

static dim3 row_block(const FullGrid& g) { return dim3((unsigned)std::min(256, ((g.H + 31) / 32) * 32)); }
static dim3 row_grid(const FullGrid& g) {
  const unsigned bx = row_block(g).x;
  return dim3((unsigned)g.rows, (unsigned)((g.H + bx - 1) / bx));
}

// frequencies of (row, kl); returns false past the end of the row
__device__ __forceinline__ bool row_k(const RowMap& m, int& k0, int& k1, int& k2, size_t& t) {
  const int row = blockIdx.x;
  const int kl = blockIdx.y * blockDim.x + threadIdx.x;
  if (kl >= m.H) return false;
  if (m.d == 3) {
    const int i0 = row / m.N1, i1 = row - i0 * m.N1;
    k0 = freq_of(i0, m.N0);
    k1 = freq_of(i1, m.N1);
    k2 = kl;
  } else {
    k0 = freq_of(row, m.N0);
    k1 = kl;
    k2 = 0;
  }
  t = (size_t)row * m.H + kl;
  return true;
}

// out = in * (2 pi i k_alpha) * scale   (c2 = 2 pi scale, rounded to R)
template <typename V>
__global__ void mul_grad_kernel(const V* __restrict__ in, V* out, RowMap m, int alpha,
                                typename RealOf<V>::T c2) {
  using R = typename RealOf<V>::T;
  int k[3];
  size_t t;
  if (!row_k(m, k[0], k[1], k[2], t)) return;
  const R f = c2 * (R)k[alpha];
  const V v = in[t];
  out[t] = mkc<V>(-v.y * f, v.x * f);
}

// acc = (init ? 0 : acc) + in * (-2 pi i k_alpha) * scale; if precond, then acc /= k.k (0 at k=0)
template <typename V>
__global__ void acc_div_kernel(const V* __restrict__ in, V* acc, RowMap m, int alpha, typename RealOf<V>::T c2,
                               int init, int precond, const typename RealOf<V>::T* __restrict__ inv_kk) {
  using R = typename RealOf<V>::T;
  int k[3];
  size_t t;
  if (!row_k(m, k[0], k[1], k[2], t)) return;
  const R f = -c2 * (R)k[alpha];
  const V v = in[t];
  V r = mkc<V>(-v.y * f, v.x * f);
  if (!init) {
    const V o = acc[t];
    r.x += o.x;
    r.y += o.y;
  }
  if (precond) {
    const R s = inv_kk[k[0] * k[0] + k[1] * k[1] + k[2] * k[2]];
    r.x *= s;
    r.y *= s;
  }
  acc[t] = r;
}

template <typename V>
__global__ void precond_kernel(const V* __restrict__ in, V* out, RowMap m,
                               const typename RealOf<V>::T* __restrict__ inv_kk) {
  using R = typename RealOf<V>::T;
  int k[3];
  size_t t;
  if (!row_k(m, k[0], k[1], k[2], t)) return;
  const R s = inv_kk[k[0] * k[0] + k[1] * k[1] + k[2] * k[2]];
  const V v = in[t];
  out[t] = mkc<V>(v.x * s, v.y * s);
}

// the six distinct entries of a symmetric 3 x 3 B times a constant: (b00, b11, b22, b01, b02, b12)
template <typename R>
struct SymB {
  R b[6];
};

template <typename R>
static SymB<R> sym_b(const double* B, double c) {
  SymB<R> s;
  s.b[0] = (R)(c * B[0]);
  s.b[1] = (R)(c * B[4]);
  s.b[2] = (R)(c * B[8]);
  s.b[3] = (R)(c * B[1]);
  s.b[4] = (R)(c * B[2]);
  s.b[5] = (R)(c * B[5]);
  return s;
}

template <typename R>
__device__ __forceinline__ R quad_b(const SymB<R>& s, int k0, int k1, int k2) {
  const R x = (R)k0, y = (R)k1, z = (R)k2;
  return s.b[0] * x * x + s.b[1] * y * y + s.b[2] * z * z + (R)2 * (s.b[3] * x * y + s.b[4] * x * z + s.b[5] * y * z);
}

// acc += (c k.B k) in; then, if precond, acc /= k.k (0 at k = 0)
template <typename V>
__global__ void acc_aniso_kernel(const V* __restrict__ in, V* acc, RowMap m, SymB<typename RealOf<V>::T> sb,
                                 int precond, const typename RealOf<V>::T* __restrict__ inv_kk) {
  using R = typename RealOf<V>::T;
  int k[3];
  size_t t;
  if (!row_k(m, k[0], k[1], k[2], t)) return;
  const R q = quad_b(sb, k[0], k[1], k[2]);
  const V v = in[t];
  V r = acc[t];
  r.x += q * v.x;
  r.y += q * v.y;
  if (precond) {
    const R s = inv_kk[k[0] * k[0] + k[1] * k[1] + k[2] * k[2]];
    r.x *= s;
    r.y *= s;
  }
  acc[t] = r;
}

template <typename R> static const R* inv_table(const FullGrid& g);
template <> const double* inv_table<double>(const FullGrid& g) { return g.inv_kk64; }
template <> const float* inv_table<float>(const FullGrid& g) { return g.inv_kk32; }

__global__ void inv_table_kernel(double* t64, float* t32, int n) {
  for (int m = blockIdx.x * blockDim.x + threadIdx.x; m < n; m += gridDim.x * blockDim.x) {
    const double v = m > 0 ? 1.0 / (double)m : 0.0;
    t64[m] = v;
    t32[m] = m > 0 ? 1.0f / (float)m : 0.0f;
  }
}

void make_inv_tables(lrfg_ctx* ctx, FullGrid& g, DBuf<double>& t64, DBuf<float>& t32) {
  long long kmax = 0;
  for (int j = 0; j < g.d; ++j) kmax += (long long)((g.N[j] - 1) / 2) * ((g.N[j] - 1) / 2);
  const int n = (int)kmax + 1;
  t64 = DBuf<double>(ctx->pool, n);
  t32 = DBuf<float>(ctx->pool, n);
  LRFG_LAUNCH(ctx, KC_POINTWISE, n, 12.0 * n,
              inv_table_kernel<<<std::max(1, std::min(1024, (n + 255) / 256)), 256, 0, ctx->stream>>>(t64.get(),
                                                                                                      t32.get(), n));
  g.inv_kk64 = t64.get();
  g.inv_kk32 = t32.get();
}

static double two_pi_times(double scale) { return 6.283185307179586476925286766559 * scale; }

template <typename V>
void half_mul_grad(lrfg_ctx* ctx, const FullGrid& g, const V* in, V* out, int alpha, double scale) {
  using R = typename RealOf<V>::T;
  LRFG_LAUNCH(ctx, KC_POINTWISE, 2.0 * g.n_half, 2.0 * sizeof(V) * g.n_half,
              mul_grad_kernel<V><<<row_grid(g), row_block(g), 0, ctx->stream>>>(in, out, rowmap(g), alpha,
                                                                                 (R)two_pi_times(scale)));
}

template <typename V>
void half_acc_div(lrfg_ctx* ctx, const FullGrid& g, const V* in, V* acc, int alpha, double scale, int init,
                  int precond) {
  using R = typename RealOf<V>::T;
  LRFG_REQUIRE(!precond || inv_table<R>(g), "reciprocal table missing");
  LRFG_LAUNCH(ctx, KC_POINTWISE, 4.0 * g.n_half, (init ? 2.0 : 3.0) * sizeof(V) * g.n_half,
              acc_div_kernel<V><<<row_grid(g), row_block(g), 0, ctx->stream>>>(
                  in, acc, rowmap(g), alpha, (R)two_pi_times(scale), init, precond, inv_table<R>(g)));
}

// The complex-axis passes of the operator around its fused rows, with grad^ folded into the first
// inverse pass (axis 0) and grad^* (with P~^-1 on the last component) into the last forward one.
template <typename R>
static FibreMul<R> fibre_mul(const FullGrid& g, int mode, int alpha, double scale, int init, int precond) {
  FibreMul<R> fm{};
  fm.mode = mode;
  fm.alpha = alpha;
  fm.d = g.d;
  fm.N1 = g.d == 3 ? g.N[1] : 1;
  fm.H = g.H;
  fm.init = init;
  fm.precond = precond;
  fm.c2 = (R)two_pi_times(scale);
  fm.inv_kk = inv_table<R>(g);
  return fm;
}

template <typename V>
void half_grad_fibres_inverse(lrfg_ctx* ctx, const FullGrid& g, const V* in, V* half, int alpha, double scale) {
  using R = typename RealOf<V>::T;
  long long inner = g.n_half / g.N[0];
  fft_fibres_mul(ctx, in, half, g.N[0], inner, fibre_mul<R>(g, 1, alpha, scale, 0, 0));
  for (int ax = 1; ax <= g.d - 2; ++ax) {
    inner /= g.N[ax];
    fft_fibres(ctx, half, half, g.n_half / (inner * g.N[ax]), g.N[ax], inner, 1);
  }
}

template <typename V>
void half_fibres_forward_div(lrfg_ctx* ctx, const FullGrid& g, V* half, V* acc, int alpha, double scale, int init,
                             int precond) {
  using R = typename RealOf<V>::T;
  long long inner = g.H;
  for (int ax = g.d - 2; ax >= 1; --ax) {
    long long outer = 1;
    for (int j = 0; j < ax; ++j) outer *= g.N[j];
    fft_fibres(ctx, half, half, outer, g.N[ax], inner, -1);
    inner *= g.N[ax];
  }
  fft_fibres_mul(ctx, (const V*)half, acc, g.N[0], inner, fibre_mul<R>(g, 2, alpha, scale, init, precond));
}

template void half_grad_fibres_inverse<double2>(lrfg_ctx*, const FullGrid&, const double2*, double2*, int, double);
template void half_grad_fibres_inverse<float2>(lrfg_ctx*, const FullGrid&, const float2*, float2*, int, double);
template void half_fibres_forward_div<double2>(lrfg_ctx*, const FullGrid&, double2*, double2*, int, double, int, int);
template void half_fibres_forward_div<float2>(lrfg_ctx*, const FullGrid&, float2*, float2*, int, double, int, int);

// ------------------------------------------------------------------------------------------------
// Ga: injection / projection between the half spectra of the grid (N) and the double grid (M = 2N - 1)
// ------------------------------------------------------------------------------------------------
__device__ __forceinline__ int wrap(int k, int n) { return k >= 0 ? k : k + n; }

// over the half spectrum of gM: the coefficient of the same frequency on g, or 0 outside Z_N
__global__ void inject_kernel(const double2* __restrict__ in, double2* __restrict__ out, RowMap mN, RowMap mM) {
  int k[3];
  size_t t;
  if (!row_k(mM, k[0], k[1], k[2], t)) return;
  const int h0 = (mN.N0 - 1) / 2, h1 = (mN.N1 - 1) / 2;
  double2 v = make_double2(0.0, 0.0);
  if (mN.d == 3) {
    if (abs(k[0]) <= h0 && abs(k[1]) <= h1 && k[2] < mN.H)
      v = in[((size_t)wrap(k[0], mN.N0) * mN.N1 + wrap(k[1], mN.N1)) * mN.H + k[2]];
  } else {
    if (abs(k[0]) <= h0 && k[1] < mN.H) v = in[(size_t)wrap(k[0], mN.N0) * mN.H + k[1]];
  }
  out[t] = v;
}

// over the half spectrum of g: the coefficient of the same frequency on gM
__global__ void project_kernel(const double2* __restrict__ in, double2* __restrict__ out, RowMap mN, RowMap mM) {
  int k[3];
  size_t t;
  if (!row_k(mN, k[0], k[1], k[2], t)) return;
  size_t tm;
  if (mN.d == 3)
    tm = ((size_t)wrap(k[0], mM.N0) * mM.N1 + wrap(k[1], mM.N1)) * mM.H + k[2];
  else
    tm = (size_t)wrap(k[0], mM.N0) * mM.H + k[1];
  out[t] = in[tm];
}

// s(m) = int over a cell of width 1/n of e^{2 pi i m t} dt = sin(pi m / n) / (pi m), 1/n at m = 0
__device__ __forceinline__ double cell_sinc(int m, int n) {
  if (m == 0) return 1.0 / n;
  const double x = 3.141592653589793238462643383279502884 * (double)m;
  return sin(x / (double)n) / x;
}

// X[m] = scale * (Phi a)(m mod N) * prod_a s(m_a) over the half spectrum of gM (Phi a from its half
// spectrum on g, by Hermitian symmetry where the last frequency wraps to a negative one)
__global__ void ga_spectrum_kernel(const double2* __restrict__ pa, double2* __restrict__ X, RowMap mN, RowMap mM,
                                   int NL, double scale) {
  int m[3];
  size_t t;
  if (!row_k(mM, m[0], m[1], m[2], t)) return;
  const int d = mN.d;
  // representatives in Z_N of m mod N, per axis
  const int n0 = mN.N0, n1 = d == 3 ? mN.N1 : NL, n2 = NL;
  int k0 = ((m[0] % n0) + n0) % n0;
  k0 = k0 <= (n0 - 1) / 2 ? k0 : k0 - n0;
  int k1 = ((m[1] % n1) + n1) % n1;
  k1 = k1 <= (n1 - 1) / 2 ? k1 : k1 - n1;
  int k2 = 0;
  if (d == 3) {
    k2 = ((m[2] % n2) + n2) % n2;
    k2 = k2 <= (n2 - 1) / 2 ? k2 : k2 - n2;
  }
  const int kl = d == 3 ? k2 : k1;  // last-axis frequency
  bool cj = false;
  if (kl < 0) {  // (Phi a)(k) = conj((Phi a)(-k)) for real a
    k0 = -k0;
    k1 = -k1;
    k2 = -k2;
    cj = true;
  }
  double2 v;
  if (d == 3)
    v = pa[((size_t)wrap(k0, n0) * mN.N1 + wrap(k1, mN.N1)) * mN.H + k2];
  else
    v = pa[(size_t)wrap(k0, n0) * mN.H + k1];
  if (cj) v.y = -v.y;
  double S = scale * cell_sinc(m[0], n0) * cell_sinc(m[1], n1);
  if (d == 3) S *= cell_sinc(m[2], n2);
  X[t] = make_double2(S * v.x, S * v.y);
}

void half_inject(lrfg_ctx* ctx, const FullGrid& g, const FullGrid& gM, const double2* in, double2* out) {
  LRFG_LAUNCH(ctx, KC_POINTWISE, 0.0, sizeof(double2) * (double)(g.n_half + gM.n_half),
              inject_kernel<<<row_grid(gM), row_block(gM), 0, ctx->stream>>>(in, out, rowmap(g), rowmap(gM)));
}

void half_project(lrfg_ctx* ctx, const FullGrid& g, const FullGrid& gM, const double2* in, double2* out) {
  LRFG_LAUNCH(ctx, KC_POINTWISE, 0.0, 2.0 * sizeof(double2) * (double)g.n_half,
              project_kernel<<<row_grid(g), row_block(g), 0, ctx->stream>>>(in, out, rowmap(g), rowmap(gM)));
}

void ga_coefficient(lrfg_ctx* ctx, const FullGrid& g, const FullGrid& gM, const double* a, double2* half_g,
                    double2* half_m, double* out) {
  full_forward<double>(ctx, g, a, nullptr, 1.0, half_g);  // Phi a on g
  const double scale = (double)g.n_real / ((double)gM.n_real * (double)gM.n_real);
  LRFG_LAUNCH(ctx, KC_POINTWISE, 20.0 * gM.n_half, sizeof(double2) * (double)(g.n_half + gM.n_half),
              ga_spectrum_kernel<<<row_grid(gM), row_block(gM), 0, ctx->stream>>>(half_g, half_m, rowmap(g), rowmap(gM),
                                                                                 g.N[g.d - 1], scale));
  full_inverse<double>(ctx, gM, half_m, nullptr, 1.0, out);  // (|N| / |M|^2) Phi*_M X
}

template <typename V>
void half_acc_aniso(lrfg_ctx* ctx, const FullGrid& g, const V* in, V* acc, const double* B, int precond) {
  using R = typename RealOf<V>::T;
  LRFG_REQUIRE(!precond || inv_table<R>(g), "reciprocal table missing");
  const double c = 4.0 * 9.869604401089358618834490999876;  // 4 pi^2
  LRFG_LAUNCH(ctx, KC_POINTWISE, 14.0 * g.n_half, 3.0 * sizeof(V) * g.n_half,
              acc_aniso_kernel<V><<<row_grid(g), row_block(g), 0, ctx->stream>>>(
                  in, acc, rowmap(g), sym_b<R>(B, c), precond, inv_table<R>(g)));
}

template <typename V>
void half_precond(lrfg_ctx* ctx, const FullGrid& g, const V* in, V* out) {
  using R = typename RealOf<V>::T;
  LRFG_REQUIRE(inv_table<R>(g), "reciprocal table missing");
  LRFG_LAUNCH(ctx, KC_POINTWISE, 2.0 * g.n_half, 2.0 * sizeof(V) * g.n_half,
              precond_kernel<V><<<row_grid(g), row_block(g), 0, ctx->stream>>>(in, out, rowmap(g), inv_table<R>(g)));
}

// ------------------------------------------------------------------------------------------------
// reductions: Hermitian-weighted inner product of half spectra, and the A_eff energy density.
// FP64 data accumulate in FP64.  FP32 data: each product is split exactly (p + e, e = fma(a, b, -p))
// and both parts are summed per thread with error-free two-sums (Knuth) in FP32, so the per-thread
// partial is accurate to ~n eps32^2 of the sum of magnitudes (FP64 class) while the work runs on the
// FP32 pipe; partials are combined in FP64.
// ------------------------------------------------------------------------------------------------
constexpr int kRedBlocks = 1216;  // 8 blocks per SM

__device__ __forceinline__ void two_sum_acc(float& s, float& c, float x) {
  const float t = s + x;
  const float bp = t - s;
  c += (s - (t - bp)) + (x - bp);
  s = t;
}

template <typename V>
__global__ void __launch_bounds__(256) half_dot_kernel(const V* __restrict__ x, const V* __restrict__ y, long long n,
                                                       int H, double* partial) {
  __shared__ double red[8];
  double s = 0.0;
  const long long stride = (long long)gridDim.x * blockDim.x;
  long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  int kl = (int)(t % H);
  const int kstep = (int)(stride % H);
  if constexpr (sizeof(V) == sizeof(float2)) {
    // four elements' loads in flight before any is used
    constexpr int kU = 4;
    float fs = 0.0f, fc = 0.0f;
    for (; t < n; t += kU * stride) {
      V a[kU], b[kU];
#pragma unroll
      for (int u = 0; u < kU; ++u) {
        const long long tu = t + u * stride;
        a[u] = tu < n ? x[tu] : mkc<V>(0.0f, 0.0f);
        b[u] = tu < n ? y[tu] : mkc<V>(0.0f, 0.0f);
      }
#pragma unroll
      for (int u = 0; u < kU; ++u) {
        const float w = kl == 0 ? 1.0f : 2.0f;
        const float p1 = a[u].x * b[u].x, e1 = fmaf(a[u].x, b[u].x, -p1);
        const float p2 = a[u].y * b[u].y, e2 = fmaf(a[u].y, b[u].y, -p2);
        two_sum_acc(fs, fc, w * p1);
        two_sum_acc(fs, fc, w * p2);
        fc += w * (e1 + e2);
        kl += kstep;
        if (kl >= H) kl -= H;
      }
    }
    s = (double)fs + (double)fc;
  } else {
    for (; t < n; t += stride) {
      const V a = x[t], b = y[t];
      const double w = kl == 0 ? 1.0 : 2.0;
      s += w * ((double)a.x * (double)b.x + (double)a.y * (double)b.y);
      kl += kstep;
      if (kl >= H) kl -= H;
    }
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

// sum over the full spectrum of (k.B k) |v_k|^2 (B pre-scaled), from the half spectrum with weights 1 / 2
__global__ void __launch_bounds__(256) aniso_energy_kernel(const double2* __restrict__ v, long long n, int H, int d,
                                                           int N0, int N1, SymB<double> sb, double* partial) {
  __shared__ double red[8];
  double s = 0.0;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x) {
    const long long row = t / H;
    const int kl = (int)(t - row * H);
    int k0, k1, k2;
    if (d == 3) {
      const int i0 = (int)(row / N1), i1 = (int)(row - (long long)i0 * N1);
      k0 = freq_of(i0, N0);
      k1 = freq_of(i1, N1);
      k2 = kl;
    } else {
      k0 = freq_of((int)row, N0);
      k1 = kl;
      k2 = 0;
    }
    const double2 x = v[t];
    const double w = kl == 0 ? 1.0 : 2.0;
    s += w * quad_b(sb, k0, k1, k2) * (x.x * x.x + x.y * x.y);
  }
  for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffff, s, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double r = 0.0;
    for (int i = 0; i < 8; ++i) r += red[i];
    partial[blockIdx.x] = r;
  }
}

// *out (+)= sum of partials; then, if ratio: mode 1 -> *ratio = *aux / *out, mode 2 -> *out / *aux
// (0 when the divisor is 0): the PCG step lengths, formed once on the device
__global__ void finish_sum_kernel(const double* __restrict__ partial, int n, double* out, int accumulate,
                                  const double* aux, double* ratio, int mode) {
  __shared__ double red[8];
  double s = 0.0;
  for (int t = threadIdx.x; t < n; t += blockDim.x) s += partial[t];
  for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffff, s, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double v = 0.0;
    for (int i = 0; i < 8; ++i) v += red[i];
    v = accumulate ? *out + v : v;
    *out = v;
    if (ratio) {
      const double num = mode == 1 ? *aux : v, den = mode == 1 ? v : *aux;
      *ratio = den != 0.0 ? num / den : 0.0;
    }
  }
}

template <typename V>
void half_dot(lrfg_ctx* ctx, const FullGrid& g, const V* x, const V* y, double* out_dev, const double* aux,
              double* ratio, int mode) {
  DBuf<double> partial(ctx->pool, kRedBlocks);
  LRFG_LAUNCH(ctx, KC_REDUCE, 4.0 * g.n_half, 2.0 * sizeof(V) * g.n_half,
              half_dot_kernel<V><<<kRedBlocks, 256, 0, ctx->stream>>>(x, y, g.n_half, g.H, partial.get()));
  LRFG_LAUNCH(ctx, KC_REDUCE, kRedBlocks, kRedBlocks * sizeof(double),
              finish_sum_kernel<<<1, 256, 0, ctx->stream>>>(partial.get(), kRedBlocks, out_dev, 0, aux, ratio, mode));
}

void aniso_energy_sum(lrfg_ctx* ctx, const FullGrid& g, const double2* v, const double* B, double* out_dev,
                      int accumulate) {
  DBuf<double> partial(ctx->pool, kRedBlocks);
  const double c = 4.0 * 9.869604401089358618834490999876 / (double)g.n_real;  // 4 pi^2 / |N|
  LRFG_LAUNCH(ctx, KC_REDUCE, 16.0 * g.n_half, sizeof(double2) * (double)g.n_half,
              aniso_energy_kernel<<<kRedBlocks, 256, 0, ctx->stream>>>(v, g.n_half, g.H, g.d, g.N[0],
                                                                         g.d == 3 ? g.N[1] : 1, sym_b<double>(B, c),
                                                                         partial.get()));
  LRFG_LAUNCH(ctx, KC_REDUCE, kRedBlocks, kRedBlocks * sizeof(double),
              finish_sum_kernel<<<1, 256, 0, ctx->stream>>>(partial.get(), kRedBlocks, out_dev, accumulate, nullptr,
                                                            nullptr, 0));
}

template <typename R>
void energy_sum(lrfg_ctx* ctx, const FullGrid& g, const R* e, const R* a, double E, double* out_dev, int accumulate) {
  DBuf<double> partial(ctx->pool, kRedBlocks);
  LRFG_LAUNCH(ctx, KC_REDUCE, 4.0 * g.n_real, 2.0 * sizeof(R) * g.n_real,
              energy_kernel<R><<<kRedBlocks, 256, 0, ctx->stream>>>(e, a, E, g.n_real, partial.get()));
  LRFG_LAUNCH(ctx, KC_REDUCE, kRedBlocks, kRedBlocks * sizeof(double),
              finish_sum_kernel<<<1, 256, 0, ctx->stream>>>(partial.get(), kRedBlocks, out_dev, accumulate, nullptr,
                                                            nullptr, 0));
}

// ------------------------------------------------------------------------------------------------
// PCG vector updates with a device FP64 step length (rounded once to R)
// ------------------------------------------------------------------------------------------------
template <typename V>
__global__ void pcg_update_kernel(V* u, V* r, const V* __restrict__ p, const V* __restrict__ q, V* z, RowMap m,
                                  const double* __restrict__ alpha_dev,
                                  const typename RealOf<V>::T* __restrict__ inv_kk) {
  using R = typename RealOf<V>::T;
  int k[3];
  size_t t;
  if (!row_k(m, k[0], k[1], k[2], t)) return;
  const R alpha = (R)(*alpha_dev);
  V pv = p[t], qv = q[t], uv = u[t], rv = r[t];
  uv.x += alpha * pv.x;
  uv.y += alpha * pv.y;
  rv.x -= alpha * qv.x;
  rv.y -= alpha * qv.y;
  u[t] = uv;
  r[t] = rv;
  const R s = inv_kk[k[0] * k[0] + k[1] * k[1] + k[2] * k[2]];
  z[t] = mkc<V>(rv.x * s, rv.y * s);
}

// p = z + beta p
template <typename V>
__global__ void pcg_direction_kernel(V* p, const V* __restrict__ z, long long n, const double* __restrict__ beta_dev) {
  using R = typename RealOf<V>::T;
  const R beta = (R)(*beta_dev);
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x) {
    V pv = p[t], zv = z[t];
    p[t] = mkc<V>(zv.x + beta * pv.x, zv.y + beta * pv.y);
  }
}

template <typename V>
void pcg_update(lrfg_ctx* ctx, const FullGrid& g, V* u, V* r, const V* p, const V* q, V* z, const double* alpha) {
  using R = typename RealOf<V>::T;
  LRFG_REQUIRE(inv_table<R>(g), "reciprocal table missing");
  LRFG_LAUNCH(ctx, KC_POINTWISE, 10.0 * g.n_half, 7.0 * sizeof(V) * g.n_half,
              pcg_update_kernel<V><<<row_grid(g), row_block(g), 0, ctx->stream>>>(u, r, p, q, z, rowmap(g), alpha,
                                                                                  inv_table<R>(g)));
}

template <typename V>
void pcg_direction(lrfg_ctx* ctx, const FullGrid& g, V* p, const V* z, const double* beta) {
  LRFG_LAUNCH(ctx, KC_POINTWISE, 4.0 * g.n_half, 3.0 * sizeof(V) * g.n_half,
              pcg_direction_kernel<V><<<grid1d(ctx, g.n_half), 256, 0, ctx->stream>>>(p, z, g.n_half, beta));
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
  template void half_acc_aniso<V>(lrfg_ctx*, const FullGrid&, const V*, V*, const double*, int);          \
  template void half_dot<V>(lrfg_ctx*, const FullGrid&, const V*, const V*, double*, const double*, double*, int); \
  template void energy_sum<R>(lrfg_ctx*, const FullGrid&, const R*, const R*, double, double*, int);      \
  template void pcg_update<V>(lrfg_ctx*, const FullGrid&, V*, V*, const V*, const V*, V*, const double*);  \
  template void pcg_direction<V>(lrfg_ctx*, const FullGrid&, V*, const V*, const double*);
LRFG_FULL_INSTANTIATE(double2, double)
LRFG_FULL_INSTANTIATE(float2, float)
template void convert<double, float>(lrfg_ctx*, const double*, float*, long long);
template void convert<float, double>(lrfg_ctx*, const float*, double*, long long);
template void convert<double2, float2>(lrfg_ctx*, const double2*, float2*, long long);
template void convert<float2, double2>(lrfg_ctx*, const float2*, double2*, long long);

}  // namespace lrfg
