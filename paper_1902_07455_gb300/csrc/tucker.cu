// Tucker format on the GPU (App. A.2): core c of shape (r_0, .., r_{d-1}) and factor matrices B_j of
// shape (N_j, r_j), u = sum_i c[i] b^(0)[i_0] x .. x b^(d-1)[i_{d-1}] (Eq. (tucker)), held in real space
// like the TT carriages (the mode-wise F commutes with the format).  Rows a1-a8 in this format:
//   gradient / divergence / Gaussian multipliers act on one factor (fibre FFTs along N_j);
//   Hadamard product = row-wise Khatri-Rao of the factor pairs + Kronecker product of the cores
//     (App. A.2.1, pair index i*s + k);
//   sum = concatenated factors + block-diagonal core;
//   truncation T (App. A.2.3) = orthonormalise every factor, move its triangular factor into the core,
//     HOSVD of the core, factors Q_j V_j.  The orthonormalisation is the Gram/Cholesky form used by the
//     TT rounding: factor columns scaled to unit norm, pivoted Cholesky of the Gram matrix (stopping at
//     the numerical rank), Q = B Pc; the HOSVD takes the top eigenvectors of each mode's Gram matrix of
//     the core (its active size is the numerical rank of that factor).
#include <algorithm>
#include <cmath>
#include <vector>

#include "ops.cuh"

namespace lrfg {

static unsigned grid_of(lrfg_ctx* ctx, long long n) {
  long long g = (n + 255) / 256;
  long long cap = 16LL * (ctx->num_sms > 0 ? ctx->num_sms : 152);
  return (unsigned)std::max(1LL, std::min(g, cap));
}

TKView tk_view(const TK& x) {
  TKView v{};
  v.d = x.d;
  for (int j = 0; j < 3; ++j) {
    v.N[j] = x.N[j];
    v.r[j] = x.r[j];
    v.fac[j] = x.fac[j].get();
  }
  v.core = x.core.get();
  return v;
}

static size_t core_size(int d, const int* r) {
  size_t s = 1;
  for (int j = 0; j < d; ++j) s *= (size_t)r[j];
  return s;
}

void tk_alloc(lrfg_ctx* ctx, TK& x, int d, const int* N, const int* r) {
  x.d = d;
  for (int j = 0; j < 3; ++j) {
    x.N[j] = j < d ? N[j] : 1;
    x.r[j] = j < d ? r[j] : 1;
  }
  x.core = DBuf<double>(ctx->pool, core_size(d, x.r));
  for (int j = 0; j < d; ++j) x.fac[j] = DBuf<double>(ctx->pool, (size_t)x.N[j] * x.r[j]);
  for (int j = d; j < 3; ++j) x.fac[j] = DBuf<double>();
}

void tk_copy(lrfg_ctx* ctx, const TKView& x, TK& out) {
  tk_alloc(ctx, out, x.d, x.N, x.r);
  LRFG_CUDA(cudaMemcpyAsync(out.core.get(), x.core, sizeof(double) * core_size(x.d, x.r), cudaMemcpyDeviceToDevice,
                            ctx->stream));
  for (int j = 0; j < x.d; ++j)
    LRFG_CUDA(cudaMemcpyAsync(out.fac[j].get(), x.fac[j], sizeof(double) * x.N[j] * x.r[j], cudaMemcpyDeviceToDevice,
                              ctx->stream));
}

// ------------------------------------------------------------------------------------------------
// mode products and mode Gram matrices of a dense core (row-major, d = 2 or 3)
// ------------------------------------------------------------------------------------------------
// out = in x_j op(M): mode j of size dims[j] becomes m; op(M) = M (m x dims[j], leading dim ldm) or,
// with transM, the transpose of M stored as (dims[j] x m, leading dim ldm)
static void mode_mult(lrfg_ctx* ctx, const double* in, int d, const int* dims, int j, const double* M, int m, int ldm,
                      int transM, double* out) {
  const int n0 = dims[0], n1 = dims[1], n2 = d == 3 ? dims[2] : 1;
  if (d == 2) {
    if (j == 0) gemm(ctx, transM, 0, m, n1, n0, 1.0, M, ldm, 0, in, n1, 0, 0.0, out, n1, 0);
    else gemm(ctx, 0, transM ? 0 : 1, n0, m, n1, 1.0, in, n1, 0, M, ldm, 0, 0.0, out, m, 0);
    return;
  }
  if (j == 0) {
    gemm(ctx, transM, 0, m, n1 * n2, n0, 1.0, M, ldm, 0, in, n1 * n2, 0, 0.0, out, n1 * n2, 0);
  } else if (j == 1) {
    gemm(ctx, transM, 0, m, n2, n1, 1.0, M, ldm, 0, in, n2, (long long)n1 * n2, 0.0, out, n2, (long long)m * n2, n0);
  } else {
    gemm(ctx, 0, transM ? 0 : 1, n0 * n1, m, n2, 1.0, in, n2, 0, M, ldm, 0, 0.0, out, m, 0);
  }
}

// (i0, i1, i2) -> (i1, i0, i2)
__global__ void swap01_kernel(const double* __restrict__ in, double* out, int n0, int n1, int n2) {
  const long long total = (long long)n0 * n1 * n2;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total; t += (long long)gridDim.x * blockDim.x) {
    const int i2 = (int)(t % n2);
    const long long rest = t / n2;
    const int i1 = (int)(rest % n1), i0 = (int)(rest / n1);
    out[((size_t)i1 * n0 + i0) * n2 + i2] = in[t];
  }
}

// S = (mode-j unfolding)(mode-j unfolding)^T, dims[j] x dims[j]
static void mode_gram(lrfg_ctx* ctx, const double* in, int d, const int* dims, int j, double* S) {
  const long long tot = (long long)core_size(d, dims);
  const int nj = dims[j];
  const int rest = (int)(tot / nj);
  if (j == 0) {
    gemm(ctx, 0, 1, nj, nj, rest, 1.0, in, rest, 0, in, rest, 0, 0.0, S, nj, 0);
  } else if (j == d - 1) {
    gemm(ctx, 1, 0, nj, nj, rest, 1.0, in, nj, 0, in, nj, 0, 0.0, S, nj, 0);
  } else {
    DBuf<double> tmp(ctx->pool, (size_t)tot);
    LRFG_LAUNCH(ctx, KC_TT_MISC, 0.0, 16.0 * tot,
                swap01_kernel<<<grid_of(ctx, tot), 256, 0, ctx->stream>>>(in, tmp.get(), dims[0], dims[1], dims[2]));
    gemm(ctx, 0, 1, nj, nj, rest, 1.0, tmp.get(), rest, 0, tmp.get(), rest, 0, 0.0, S, nj, 0);
  }
}

// ------------------------------------------------------------------------------------------------
// element-wise kernels: unit-column balancing of a Gram matrix, Kronecker product of cores, block
// embedding of cores
// ------------------------------------------------------------------------------------------------
// c_i = 1 / sqrt(G_ii) (1 for a zero column), G <- C G C
__global__ void unit_balance_kernel(double* G, double* c, int m) {
  extern __shared__ double cs[];
  for (int i = threadIdx.x; i < m; i += blockDim.x) {
    const double g = G[(size_t)i * m + i];
    cs[i] = g > 0.0 ? 1.0 / sqrt(g) : 1.0;
    c[i] = cs[i];
  }
  __syncthreads();
  for (int t = threadIdx.x; t < m * m; t += blockDim.x) {
    const int i = t / m, j = t - (t / m) * m;
    G[t] *= cs[i] * cs[j];
  }
}

struct Dims3 {
  int a[3];
};

// out[(i0 ry0 + k0), (i1 ry1 + k1), (i2 ry2 + k2)] = x[i0, i1, i2] y[k0, k1, k2]
__global__ void kron_core_kernel(const double* __restrict__ x, Dims3 rx, const double* __restrict__ y, Dims3 ry,
                                 double* out, int d) {
  const long long nx = (long long)rx.a[0] * rx.a[1] * rx.a[2], ny = (long long)ry.a[0] * ry.a[1] * ry.a[2];
  const long long total = nx * ny;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total; t += (long long)gridDim.x * blockDim.x) {
    // output multi-index (o0, o1, o2), o_j = i_j ry_j + k_j
    long long rest = t;
    int o[3];
    for (int j = d - 1; j >= 0; --j) {
      const int nj = rx.a[j] * ry.a[j];
      o[j] = (int)(rest % nj);
      rest /= nj;
    }
    long long ix = 0, iy = 0;
    for (int j = 0; j < d; ++j) {
      ix = ix * rx.a[j] + o[j] / ry.a[j];
      iy = iy * ry.a[j] + o[j] % ry.a[j];
    }
    out[t] = x[ix] * y[iy];
  }
}

// out[off + i] += s * x[i] for a block of shape rb inside a core of shape ro (out zeroed before)
__global__ void embed_core_kernel(const double* __restrict__ x, Dims3 rb, double* out, Dims3 ro, Dims3 off, double s,
                                  int d) {
  const long long total = (long long)rb.a[0] * rb.a[1] * rb.a[2];
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total; t += (long long)gridDim.x * blockDim.x) {
    long long rest = t;
    int i[3] = {0, 0, 0};
    for (int j = d - 1; j >= 0; --j) {
      i[j] = (int)(rest % rb.a[j]);
      rest /= rb.a[j];
    }
    long long o = 0;
    for (int j = 0; j < d; ++j) o = o * ro.a[j] + (off.a[j] + i[j]);
    out[o] = s * x[t];
  }
}

static Dims3 dims3(int d, const int* r) {
  Dims3 x;
  for (int j = 0; j < 3; ++j) x.a[j] = j < d ? r[j] : 1;
  return x;
}

// ------------------------------------------------------------------------------------------------
// format operations
// ------------------------------------------------------------------------------------------------
void tk_mode_operator(lrfg_ctx* ctx, const TKView& x, int j, int kind, double param, double scale, TK& out) {
  tk_copy(ctx, x, out);
  fibre_operator(ctx, x.fac[j], out.fac[j].get(), 1, x.N[j], x.r[j], kind, param, scale);
}

void tk_hadamard(lrfg_ctx* ctx, const TKView& x, const TKView& y, TK& out) {
  LRFG_REQUIRE(x.d == y.d, "Hadamard of Tucker tensors of different order");
  int r[3];
  for (int j = 0; j < x.d; ++j) {
    LRFG_REQUIRE(x.N[j] == y.N[j], "Hadamard of Tucker tensors on different grids");
    r[j] = x.r[j] * y.r[j];
  }
  tk_alloc(ctx, out, x.d, x.N, r);
  for (int j = 0; j < x.d; ++j) khatri_rao(ctx, x.fac[j], 1, x.N[j], x.r[j], y.fac[j], 1, y.r[j], out.fac[j].get());
  const long long total = (long long)core_size(x.d, r);
  LRFG_LAUNCH(ctx, KC_KHATRI_RAO, (double)total, 8.0 * total,
              kron_core_kernel<<<grid_of(ctx, total), 256, 0, ctx->stream>>>(x.core, dims3(x.d, x.r), y.core,
                                                                             dims3(y.d, y.r), out.core.get(), x.d));
}

void tk_add_many(lrfg_ctx* ctx, const TKView* xs, const double* scales, int nb, TK& out) {
  const int d = xs[0].d;
  int r[3] = {0, 0, 0};
  for (int b = 0; b < nb; ++b)
    for (int j = 0; j < d; ++j) {
      LRFG_REQUIRE(xs[b].d == d && xs[b].N[j] == xs[0].N[j], "sum of Tucker tensors of different shapes");
      r[j] += xs[b].r[j];
    }
  tk_alloc(ctx, out, d, xs[0].N, r);
  const size_t tot = core_size(d, r);
  LRFG_CUDA(cudaMemsetAsync(out.core.get(), 0, sizeof(double) * tot, ctx->stream));
  int off[3] = {0, 0, 0};
  for (int b = 0; b < nb; ++b) {
    for (int j = 0; j < d; ++j)
      LRFG_CUDA(cudaMemcpy2DAsync(out.fac[j].get() + off[j], sizeof(double) * r[j], xs[b].fac[j],
                                  sizeof(double) * xs[b].r[j], sizeof(double) * xs[b].r[j], xs[b].N[j],
                                  cudaMemcpyDeviceToDevice, ctx->stream));
    const long long nbk = (long long)core_size(d, xs[b].r);
    LRFG_LAUNCH(ctx, KC_TT_MISC, 0.0, 16.0 * nbk,
                embed_core_kernel<<<grid_of(ctx, nbk), 256, 0, ctx->stream>>>(
                    xs[b].core, dims3(d, xs[b].r), out.core.get(), dims3(d, r), dims3(d, off),
                    scales ? scales[b] : 1.0, d));
    for (int j = 0; j < d; ++j) off[j] += xs[b].r[j];
  }
}

void tk_round(lrfg_ctx* ctx, const TKView& x, int rmax, TK& out, double tol) {
  LRFG_REQUIRE(rmax >= 1, "truncation rank must be >= 1 (got %d)", rmax);
  const int d = x.d;
  int r[3], k[3];
  for (int j = 0; j < 3; ++j) r[j] = j < d ? x.r[j] : 1;
  for (int j = 0; j < d; ++j) k[j] = std::min(rmax, r[j]);
  // 1. orthonormal basis of every factor: Gram, unit-column balancing, pivoted Cholesky
  DBuf<double> RAc[3], Pc[3];
  DBuf<int> rho(ctx->pool, 3);
  for (int j = 0; j < d; ++j) {
    const int m = r[j];
    DBuf<double> G(ctx->pool, (size_t)m * m), c(ctx->pool, m), RA(ctx->pool, (size_t)m * m);
    gemm(ctx, 1, 0, m, m, x.N[j], 1.0, x.fac[j], m, 0, x.fac[j], m, 0, 0.0, G.get(), m, 0);
    LRFG_LAUNCH(ctx, KC_TT_MISC, 2.0 * m * m, 16.0 * m * m,
                unit_balance_kernel<<<1, 256, sizeof(double) * m, ctx->stream>>>(G.get(), c.get(), m));
    RAc[j] = DBuf<double>(ctx->pool, (size_t)m * m);
    Pc[j] = DBuf<double>(ctx->pool, (size_t)m * m);
    gram_factor(ctx, G.get(), c.get(), m, 1, RA.get(), RAc[j].get(), Pc[j].get(), rho.get() + j);
  }
  // 2. core' = core x_j RAc_j (B_j = Q_j RAc_j)
  DBuf<double> c1(ctx->pool, core_size(d, r)), c2(ctx->pool, core_size(d, r));
  LRFG_CUDA(cudaMemcpyAsync(c1.get(), x.core, sizeof(double) * core_size(d, r), cudaMemcpyDeviceToDevice, ctx->stream));
  for (int j = 0; j < d; ++j) {
    mode_mult(ctx, c1.get(), d, r, j, RAc[j].get(), r[j], r[j], 0, c2.get());
    std::swap(c1, c2);
  }
  // 3. HOSVD of core': top k_j eigenvectors of each mode Gram (active size rho_j), new factors Q_j V_j;
  // with a tolerance, k_j is decided from the eigenvalues of every mode (one synchronisation)
  DBuf<double> V[3];
  DBuf<int> kd(ctx->pool, 3);
  for (int j = 0; j < d; ++j) {
    const int m = r[j];
    DBuf<double> S(ctx->pool, (size_t)m * m), w(ctx->pool, m);
    V[j] = DBuf<double>(ctx->pool, (size_t)m * m);
    mode_gram(ctx, c1.get(), d, r, j, S.get());
    syevx_sized(ctx, S.get(), rho.get() + j, w.get(), V[j].get(), m, k[j], 1);
    if (tol > 0.0) tol_ranks(ctx, S.get(), rho.get() + j, w.get(), V[j].get(), m, k[j], tol * tol / d, 1, kd.get() + j);
  }
  if (tol > 0.0) {
    int kh[3] = {1, 1, 1};
    LRFG_CUDA(cudaMemcpyAsync(kh, kd.get(), sizeof(int) * d, cudaMemcpyDeviceToHost, ctx->stream));
    LRFG_CUDA(cudaStreamSynchronize(ctx->stream));
    for (int j = 0; j < d; ++j) k[j] = std::max(1, std::min(kh[j], k[j]));
  }
  tk_alloc(ctx, out, d, x.N, k);
  for (int j = 0; j < d; ++j) {
    const int m = r[j];
    DBuf<double> P(ctx->pool, (size_t)m * k[j]);
    gemm(ctx, 0, 0, m, k[j], m, 1.0, Pc[j].get(), m, 0, V[j].get(), m, 0, 0.0, P.get(), k[j], 0);
    gemm(ctx, 0, 0, x.N[j], k[j], m, 1.0, x.fac[j], m, 0, P.get(), k[j], 0, 0.0, out.fac[j].get(), k[j], 0);
  }
  // 4. core'' = core' x_j V_j^T
  int dims[3] = {r[0], r[1], r[2]};
  for (int j = 0; j < d; ++j) {
    double* dst = (j == d - 1) ? out.core.get() : c2.get();
    mode_mult(ctx, c1.get(), d, dims, j, V[j].get(), k[j], r[j], 1, dst);
    dims[j] = k[j];
    if (j != d - 1) std::swap(c1, c2);
  }
}

void tk_dot_device(lrfg_ctx* ctx, const TKView& x, const TKView& y, double* out_dev) {
  LRFG_REQUIRE(x.d == y.d, "dot of Tucker tensors of different order");
  const int d = x.d;
  int dims[3] = {y.r[0], y.r[1], d == 3 ? y.r[2] : 1};
  size_t cap = core_size(d, y.r);
  size_t capx = 1;
  for (int j = 0; j < d; ++j) capx *= (size_t)std::max(x.r[j], y.r[j]);
  cap = std::max(cap, capx);
  DBuf<double> t1(ctx->pool, cap), t2(ctx->pool, cap);
  LRFG_CUDA(cudaMemcpyAsync(t1.get(), y.core, sizeof(double) * core_size(d, y.r), cudaMemcpyDeviceToDevice, ctx->stream));
  for (int j = 0; j < d; ++j) {
    LRFG_REQUIRE(x.N[j] == y.N[j], "dot of Tucker tensors on different grids");
    DBuf<double> G(ctx->pool, (size_t)x.r[j] * y.r[j]);
    gemm(ctx, 1, 0, x.r[j], y.r[j], x.N[j], 1.0, x.fac[j], x.r[j], 0, y.fac[j], y.r[j], 0, 0.0, G.get(), y.r[j], 0);
    mode_mult(ctx, t1.get(), d, dims, j, G.get(), x.r[j], y.r[j], 0, t2.get());
    dims[j] = x.r[j];
    std::swap(t1, t2);
  }
  dot_device(ctx, x.core, t1.get(), (long long)core_size(d, x.r), out_dev);
}

double tk_dot(lrfg_ctx* ctx, const TKView& x, const TKView& y) {
  DBuf<double> s(ctx->pool, 1);
  tk_dot_device(ctx, x, y, s.get());
  double h = 0.0;
  LRFG_CUDA(cudaMemcpyAsync(&h, s.get(), sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
  LRFG_CUDA(cudaStreamSynchronize(ctx->stream));
  return h;
}

void tk_expand(lrfg_ctx* ctx, const TKView& x, double* values) {
  const int d = x.d;
  int dims[3] = {x.r[0], x.r[1], d == 3 ? x.r[2] : 1};
  size_t cap = 1;
  for (int j = 0; j < d; ++j) cap *= (size_t)std::max(x.N[j], x.r[j]);
  DBuf<double> t1(ctx->pool, cap), t2(ctx->pool, cap);
  LRFG_CUDA(cudaMemcpyAsync(t1.get(), x.core, sizeof(double) * core_size(d, x.r), cudaMemcpyDeviceToDevice, ctx->stream));
  for (int j = 0; j < d; ++j) {
    double* dst = (j == d - 1) ? values : t2.get();
    mode_mult(ctx, t1.get(), d, dims, j, x.fac[j], x.N[j], x.r[j], 0, dst);
    dims[j] = x.N[j];
    if (j != d - 1) std::swap(t1, t2);
  }
}

// HOSVD of a grid (App. A.2.3): factors = top eigenvectors of each mode's Gram matrix, ranks
// min(rmax, N_j) reduced to the singular values above tol * sigma_max (tol > 0); core = A x_j U_j^T
void tk_compress(lrfg_ctx* ctx, int d, const int* N, const double* values, int rmax, double tol, TK& out) {
  int k[3] = {1, 1, 1};
  std::vector<DBuf<double>> V(d);
  for (int j = 0; j < d; ++j) {
    const int m = N[j];
    const int kk = std::min(rmax, m);
    DBuf<double> S(ctx->pool, (size_t)m * m), w(ctx->pool, m);
    V[j] = DBuf<double>(ctx->pool, (size_t)m * m);
    int nd[3] = {N[0], N[1], d == 3 ? N[2] : 1};
    mode_gram(ctx, values, d, nd, j, S.get());
    syevx(ctx, S.get(), w.get(), V[j].get(), m, kk, 1);
    k[j] = kk;
    if (tol > 0.0) {
      std::vector<double> hw(kk);
      LRFG_CUDA(cudaMemcpyAsync(hw.data(), w.get(), sizeof(double) * kk, cudaMemcpyDeviceToHost, ctx->stream));
      LRFG_CUDA(cudaStreamSynchronize(ctx->stream));
      int keep = 1;
      for (int i = 1; i < kk; ++i)
        if (hw[i] > tol * tol * hw[0]) keep = i + 1;
      k[j] = keep;
    }
  }
  tk_alloc(ctx, out, d, N, k);
  for (int j = 0; j < d; ++j)
    LRFG_CUDA(cudaMemcpy2DAsync(out.fac[j].get(), sizeof(double) * k[j], V[j].get(), sizeof(double) * N[j],
                                sizeof(double) * k[j], N[j], cudaMemcpyDeviceToDevice, ctx->stream));
  size_t cap = 1;
  for (int j = 0; j < d; ++j) cap *= (size_t)N[j];
  DBuf<double> t1(ctx->pool, cap), t2(ctx->pool, cap);
  int dims[3] = {N[0], N[1], d == 3 ? N[2] : 1};
  const double* src = values;
  for (int j = 0; j < d; ++j) {
    double* dst = (j == d - 1) ? out.core.get() : (j % 2 == 0 ? t1.get() : t2.get());
    mode_mult(ctx, src, d, dims, j, V[j].get(), k[j], N[j], 1, dst);
    dims[j] = k[j];
    src = dst;
  }
}

// P~^-1 x = sum_m w_m (G_m x .. x G_m) x: factors [G_1 B_j, .., G_R B_j], core block-diagonal with the
// blocks w_m c; then T
void tk_precond(lrfg_ctx* ctx, const TKView& x, const std::vector<double>& t, const std::vector<double>& w, int rmax,
                TK& out, double tol) {
  const int d = x.d, R = (int)t.size();
  int r[3];
  for (int j = 0; j < d; ++j) r[j] = R * x.r[j];
  TK big;
  tk_alloc(ctx, big, d, x.N, r);
  std::vector<double> ones(R, 1.0);
  for (int j = 0; j < d; ++j) {
    const size_t e = (size_t)x.N[j] * x.r[j];
    DBuf<double> terms(ctx->pool, e * R);
    fibre_gauss_multi(ctx, x.fac[j], terms.get(), (long long)e, 1, x.N[j], x.r[j], t.data(), ones.data(), R);
    for (int m = 0; m < R; ++m)
      LRFG_CUDA(cudaMemcpy2DAsync(big.fac[j].get() + (size_t)m * x.r[j], sizeof(double) * r[j],
                                  terms.get() + (size_t)m * e, sizeof(double) * x.r[j], sizeof(double) * x.r[j],
                                  x.N[j], cudaMemcpyDeviceToDevice, ctx->stream));
  }
  LRFG_CUDA(cudaMemsetAsync(big.core.get(), 0, sizeof(double) * core_size(d, r), ctx->stream));
  const long long nbk = (long long)core_size(d, x.r);
  for (int m = 0; m < R; ++m) {
    int off[3];
    for (int j = 0; j < d; ++j) off[j] = m * x.r[j];
    LRFG_LAUNCH(ctx, KC_TT_MISC, 0.0, 16.0 * nbk,
                embed_core_kernel<<<grid_of(ctx, nbk), 256, 0, ctx->stream>>>(
                    x.core, dims3(d, x.r), big.core.get(), dims3(d, r), dims3(d, off), w[m], d));
  }
  tk_round(ctx, tk_view(big), rmax, out, tol);
}

// ------------------------------------------------------------------------------------------------
// the truncated operator, right-hand side, A_eff and minimal-residual solve in Tucker format
// (Eq. (Pls_lowrank), Sec. 3.3) -- the same steps as the TT path
// ------------------------------------------------------------------------------------------------
void tk_ga_map(lrfg_ctx* ctx, const TKView& x, const int* n_out, int mode, TK& out) {
  tk_alloc(ctx, out, x.d, n_out, x.r);
  LRFG_CUDA(cudaMemcpyAsync(out.core.get(), x.core, sizeof(double) * core_size(x.d, x.r), cudaMemcpyDeviceToDevice,
                            ctx->stream));
  for (int j = 0; j < x.d; ++j) ga_resample(ctx, x.fac[j], out.fac[j].get(), 1, x.N[j], x.r[j], n_out[j], mode);
}

// Ga (Eq. (ls_Ga_fourier) with the truncations of Eq. (Pls_lowrank)): each gradient component's factors
// interpolated to the double grid, the product with the modified coefficient and T there, the factors
// projected back, then the divergence, the sum and the preconditioner as for GaNi
static void tk_material_ga(lrfg_ctx* ctx, const TKGa& ga, const TKView& e, int rank, TK& out, double rtol) {
  TK eu, ae, wr;
  tk_ga_map(ctx, e, ga.a_ga.N, GA_UP, eu);
  tk_hadamard(ctx, ga.a_ga, tk_view(eu), ae);  // A~ (.) e_alpha on the double grid
  tk_round(ctx, tk_view(ae), rank, wr, rtol);  // T there
  tk_ga_map(ctx, tk_view(wr), e.N, GA_DOWN, out);
}

void tk_apply(lrfg_ctx* ctx, const TKView& a, const TKView& v, const std::vector<double>& pt,
              const std::vector<double>& pw, int rank, TK& out, double rtol, const double* B, const TKGa* ga) {
  const int d = v.d;
  TK w[3], es[3];
  for (int alpha = 0; alpha < d; ++alpha)
    tk_mode_operator(ctx, v, alpha, LRFG_MUL_DERIV, 0.0, 1.0, es[alpha]);         // gradient, mode alpha
  // Ga with an anisotropic part: A~ = a~ I + B 1~ on the double grid, component a is a~ (.) e_a +
  // sum_b B[a][b] 1~ (.) e_b before its T (the gradients interpolated there once, 1~ (.) e_b once)
  TK eu[3], oe[3];
  if (ga && B)
    for (int beta = 0; beta < d; ++beta) {
      tk_ga_map(ctx, tk_view(es[beta]), ga->a_ga.N, GA_UP, eu[beta]);
      tk_hadamard(ctx, ga->ones_ga, tk_view(eu[beta]), oe[beta]);
    }
  for (int alpha = 0; alpha < d; ++alpha) {
    TK ae, wr;
    if (ga && B) {
      TK prod, sum, wm;
      tk_hadamard(ctx, ga->a_ga, tk_view(eu[alpha]), prod);
      TKView xs[4];
      double sc[4];
      int m = 0;
      xs[m] = tk_view(prod);
      sc[m++] = 1.0;
      for (int beta = 0; beta < d; ++beta)
        if (B[alpha * 3 + beta] != 0.0) {
          xs[m] = tk_view(oe[beta]);
          sc[m++] = B[alpha * 3 + beta];
        }
      tk_add_many(ctx, xs, sc, m, sum);
      tk_round(ctx, tk_view(sum), rank, wm, rtol);  // T on the double grid
      tk_ga_map(ctx, tk_view(wm), v.N, GA_DOWN, wr);
      tk_mode_operator(ctx, tk_view(wr), alpha, LRFG_MUL_DERIV, 0.0, -1.0, w[alpha]);  // divergence
      continue;
    }
    if (ga) {
      tk_material_ga(ctx, *ga, tk_view(es[alpha]), rank, wr, rtol);
      tk_mode_operator(ctx, tk_view(wr), alpha, LRFG_MUL_DERIV, 0.0, -1.0, w[alpha]);  // divergence
      continue;
    }
    tk_hadamard(ctx, a, tk_view(es[alpha]), ae);                                  // a (.) e_alpha
    if (B) {
      // constant anisotropic part: + sum_beta B[alpha][beta] e_beta (zero entries skipped)
      TKView xs[4];
      double sc[4];
      int m = 0;
      xs[m] = tk_view(ae);
      sc[m++] = 1.0;
      for (int beta = 0; beta < d; ++beta)
        if (B[alpha * 3 + beta] != 0.0) {
          xs[m] = tk_view(es[beta]);
          sc[m++] = B[alpha * 3 + beta];
        }
      TK sum;
      tk_add_many(ctx, xs, sc, m, sum);
      ae = std::move(sum);
    }
    tk_round(ctx, tk_view(ae), rank, wr, rtol);                                   // T
    tk_mode_operator(ctx, tk_view(wr), alpha, LRFG_MUL_DERIV, 0.0, -1.0, w[alpha]);  // divergence
  }
  TKView terms[3];
  for (int alpha = 0; alpha < d; ++alpha) terms[alpha] = tk_view(w[alpha]);
  TK acc, s;
  tk_add_many(ctx, terms, nullptr, d, acc);
  tk_round(ctx, tk_view(acc), rank, s, rtol);  // T after the sum
  tk_precond(ctx, tk_view(s), pt, pw, rank, out, rtol);
}

void tk_rhs(lrfg_ctx* ctx, const TKView& a_in, const double* E, const std::vector<double>& pt,
            const std::vector<double>& pw, int rank, TK& out, double rtol, const TKGa* ga) {
  // Ga: -T P~^-1 grad^* I* F_M A~ E, i.e. the GaNi form with the projection of A~ on the grid
  const TKView a = ga ? ga->a_down : a_in;
  const int d = a.d;
  TK t[3];
  TKView terms[3];
  int n = 0;
  for (int alpha = 0; alpha < d; ++alpha) {
    if (E[alpha] == 0.0) continue;
    tk_mode_operator(ctx, a, alpha, LRFG_MUL_DERIV, 0.0, E[alpha], t[n]);  // E_a D_a a
    terms[n] = tk_view(t[n]);
    ++n;
  }
  if (n == 0) {
    int r[3] = {1, 1, 1};
    tk_alloc(ctx, out, d, a.N, r);
    fill(ctx, out.core.get(), 0.0, 1);
    for (int j = 0; j < d; ++j) fill(ctx, out.fac[j].get(), 0.0, a.N[j]);
    return;
  }
  TK acc;
  tk_add_many(ctx, terms, nullptr, n, acc);
  tk_precond(ctx, tk_view(acc), pt, pw, rank, out, rtol);  // T P~^-1
}

static void tk_ones(lrfg_ctx* ctx, int d, const int* N, TK& x) {
  int r[3] = {1, 1, 1};
  tk_alloc(ctx, x, d, N, r);
  fill(ctx, x.core.get(), 1.0, 1);
  for (int j = 0; j < d; ++j) fill(ctx, x.fac[j].get(), 1.0, N[j]);
}

double tk_aeff(lrfg_ctx* ctx, const TKView& a_in, const double* E, const TKView& u_in, const double* B,
               const TKGa* ga) {
  // Ga: the exact integral, the sum over the double grid of A~ |E + e|^2 (A~ carries the quadrature weights),
  // with u interpolated there (its gradient on the double grid is the interpolated gradient: zero padding
  // keeps the frequencies)
  TK uu;
  if (ga) tk_ga_map(ctx, u_in, ga->a_ga.N, GA_UP, uu);
  const TKView a = ga ? ga->a_ga : a_in;
  const TKView u = ga ? tk_view(uu) : u_in;
  const int d = a.d;
  double size = 1.0;
  if (!ga)
    for (int j = 0; j < d; ++j) size *= a.N[j];
  TK ones;
  tk_ones(ctx, d, a.N, ones);
  double EE = 0.0;
  for (int j = 0; j < d; ++j) EE += E[j] * E[j];
  double val = EE * tk_dot(ctx, a, tk_view(ones)) / size;
  TK e[3];
  for (int alpha = 0; alpha < d; ++alpha) {
    TK ae;
    tk_mode_operator(ctx, u, alpha, LRFG_MUL_DERIV, 0.0, 1.0, e[alpha]);
    tk_hadamard(ctx, a, tk_view(e[alpha]), ae);
    if (E[alpha] != 0.0) val += 2.0 * E[alpha] * tk_dot(ctx, tk_view(ae), tk_view(ones)) / size;
    val += tk_dot(ctx, tk_view(ae), tk_view(e[alpha])) / size;
  }
  if (B && ga) {
    // the part of B 1~ (exact integration): E.B E <1~, 1> + 2 sum_ab E_b B[b][a] <1~ (.) e_a, 1> +
    // sum_ab B[a][b] <1~ (.) e_a, e_b>
    const TKView one = ga->ones_ga;
    double ebe = 0.0;
    for (int i = 0; i < d; ++i)
      for (int j = 0; j < d; ++j) ebe += E[i] * B[i * 3 + j] * E[j];
    val += ebe * tk_dot(ctx, one, tk_view(ones));
    for (int al = 0; al < d; ++al) {
      TK oe;
      bool made = false;
      for (int be = 0; be < d; ++be) {
        const double bab = B[al * 3 + be];
        if (bab == 0.0) continue;
        if (!made) {
          tk_hadamard(ctx, one, tk_view(e[al]), oe);
          made = true;
        }
        val += 2.0 * E[be] * B[be * 3 + al] * tk_dot(ctx, tk_view(oe), tk_view(ones));
        val += bab * tk_dot(ctx, tk_view(oe), tk_view(e[be]));
      }
    }
  } else if (B) {
    // (E + e).B(E + e) averaged: E.B E + sum_ab B_ab <e_a, e_b> / |N| (e has zero mean)
    for (int i = 0; i < d; ++i)
      for (int j = 0; j < d; ++j) {
        const double bij = B[i * 3 + j];
        if (bij == 0.0) continue;
        val += E[i] * bij * E[j] + bij * tk_dot(ctx, tk_view(e[i]), tk_view(e[j])) / size;
      }
  }
  return val;
}

// u_{i+1} = T(u_i + omega_i r_i), r_i = T(b - C u_i) (r_0 = b), omega_i = (C r_i, r_i) / ||C r_i||^2; stop
// when ||r|| fails to decrease (stop_on_increase), at tol or maxit; the iterate of smallest residual is kept.
// Rank adaptation (rank_start > 0, the solver Sec. 4.3 proposes): truncations start at rank_start; when the
// residual fails to decrease, or meets tol, below the cap `rank` (tol is a statement about the cap's solution;
// the residual below it is truncated at the lower rank), the rank rises by rank_step, the right-hand side is
// rebuilt and the iteration restarts from the best iterate with its residual recomputed at the new rank.
TKSolveResult tk_solve(lrfg_ctx* ctx, const TKView& a, const double* E, const std::vector<double>& pt,
                       const std::vector<double>& pw, int rank, double tol, int maxit, int stop_on_increase,
                       TK& best_u, double rtol, const double* B, int rank_start, int rank_step, const TKGa* ga) {
  TKSolveResult res{};
  const bool adapt = rank_start > 0;
  int rc = adapt ? std::min(rank_start, rank) : rank;
  TK b;
  tk_rhs(ctx, a, E, pt, pw, rc, b, rtol, ga);
  double nb = std::sqrt(std::max(tk_dot(ctx, tk_view(b), tk_view(b)), 0.0));
  TK u, r;
  bool u_zero = true, best_zero = true;
  double best = INFINITY;
  int best_it = 0, it = 0, applies = 0;
  tk_copy(ctx, tk_view(b), r);
  auto residual = [&]() {  // r <- T(b - C u) at the current rank
    TK cu, diff, rn;
    tk_apply(ctx, a, tk_view(u), pt, pw, rc, cu, rtol, B, ga);
    ++applies;
    TKView xs[2] = {tk_view(b), tk_view(cu)};
    const double sc[2] = {1.0, -1.0};
    tk_add_many(ctx, xs, sc, 2, diff);
    tk_round(ctx, tk_view(diff), rc, rn, rtol);
    r = std::move(rn);
  };
  int since_best = 0;  // iterations since the last new smallest residual (stop_on_increase > 1: the patience)
  int cap_steps = 0;   // steps taken at the cap (the tolerance ends a rank-adapting solve only after one)
  while (nb > 0.0) {
    double nr = std::sqrt(std::max(tk_dot(ctx, tk_view(r), tk_view(r)), 0.0)) / nb;
    if (it == 0 && u_zero) nr = 1.0;  // r = b
    const bool improved = nr < best;
    if (improved) {
      best = nr;
      best_it = it;
      best_zero = u_zero;
      since_best = 0;
      if (!u_zero) tk_copy(ctx, tk_view(u), best_u);
    }
    if (adapt && rc < rank && (!improved || nr <= tol)) {
      // stagnation, or the tolerance met, below the cap: raise the rank, restart from the best iterate
      do {
        rc = std::min(rank, rc + std::max(1, rank_step));
        TK nbv;
        tk_rhs(ctx, a, E, pt, pw, rc, nbv, rtol, ga);
        b = std::move(nbv);
        nb = std::sqrt(std::max(tk_dot(ctx, tk_view(b), tk_view(b)), 0.0));
        u_zero = best_zero;
        if (u_zero) {
          tk_copy(ctx, tk_view(b), r);
        } else {
          tk_copy(ctx, tk_view(best_u), u);
          residual();
        }
        nr = u_zero ? 1.0 : std::sqrt(std::max(tk_dot(ctx, tk_view(r), tk_view(r)), 0.0)) / nb;
        best = nr;
        since_best = 0;
      } while (rc < rank && nr <= tol);
    } else if (!improved && stop_on_increase && ++since_best >= stop_on_increase) {
      break;  // (at the cap the rank-adapting iteration stops as the fixed-rank one)
    }
    if ((nr <= tol && (!adapt || (rc >= rank && cap_steps > 0))) || it >= maxit) break;
    TK q;
    tk_apply(ctx, a, tk_view(r), pt, pw, rc, q, rtol, B, ga);
    ++applies;
    const double qq = tk_dot(ctx, tk_view(q), tk_view(q));
    if (qq == 0.0) break;
    const double omega = tk_dot(ctx, tk_view(q), tk_view(r)) / qq;
    TK un;
    if (u_zero) {
      TK scaled;
      tk_copy(ctx, tk_view(r), scaled);
      axpby(ctx, (long long)core_size(r.d, r.r), omega, r.core.get(), 0.0, scaled.core.get());
      tk_round(ctx, tk_view(scaled), rc, un, rtol);
    } else {
      TKView xs[2] = {tk_view(u), tk_view(r)};
      const double sc[2] = {1.0, omega};
      TK s;
      tk_add_many(ctx, xs, sc, 2, s);
      tk_round(ctx, tk_view(s), rc, un, rtol);
    }
    u = std::move(un);
    u_zero = false;
    ++it;
    if (rc >= rank) ++cap_steps;
    residual();
  }
  if (best_zero || !best_u.d) {
    // the best iterate is u_0 = 0
    int rr[3] = {1, 1, 1};
    best_u = TK();
    tk_alloc(ctx, best_u, a.d, a.N, rr);
    fill(ctx, best_u.core.get(), 0.0, 1);
    for (int j = 0; j < a.d; ++j) fill(ctx, best_u.fac[j].get(), 0.0, a.N[j]);
  }
  res.iters = best_it;
  res.rel_resid = nb > 0.0 ? best : 0.0;
  res.applies = applies;
  res.Aeff = tk_aeff(ctx, a, E, tk_view(best_u), B, ga);
  return res;
}

}  // namespace lrfg
