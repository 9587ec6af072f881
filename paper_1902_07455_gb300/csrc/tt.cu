// Tensor-train operations on the device (hot-path rows a3 material Hadamard, a4 truncation, a5 sum,
// a6 preconditioner, a7 inner products) and TT-SVD compression of a full coefficient.
//
// Carriage j is row-major (r_j, N_j, r_{j+1}); its left unfolding is the (r_j N_j) x r_{j+1} matrix
// with the same memory, its right unfolding the r_j x (N_j r_{j+1}) matrix with the same memory.
#include <algorithm>
#include <cmath>

#include "ops.cuh"

namespace lrfg {

TTView view_of(const TT& x) {
  TTView v{};
  v.d = x.d;
  for (int j = 0; j < 3; ++j) v.N[j] = x.N[j];
  for (int j = 0; j < 4; ++j) v.r[j] = x.r[j];
  for (int j = 0; j < x.d; ++j) v.core[j] = x.core[j].get();
  return v;
}

TTView view_of(const lrfg_tt& x) {
  TTView v{};
  v.d = x.d;
  for (int j = 0; j < 3; ++j) v.N[j] = x.N[j];
  for (int j = 0; j < 4; ++j) v.r[j] = x.r[j];
  for (int j = 0; j < x.d; ++j) v.core[j] = x.cores[j];
  return v;
}

static size_t celems(const TTView& x, int j) { return (size_t)x.r[j] * x.N[j] * x.r[j + 1]; }

void tt_alloc(lrfg_ctx* ctx, TT& x, int d, const int* N, const int* r) {
  x.d = d;
  for (int j = 0; j < 3; ++j) x.N[j] = j < d ? N[j] : 0;
  for (int j = 0; j < 4; ++j) x.r[j] = j <= d ? r[j] : 1;
  x.r[0] = 1;
  x.r[d] = 1;
  for (int j = 0; j < d; ++j) x.core[j] = DBuf<double>(ctx->pool, (size_t)x.r[j] * x.N[j] * x.r[j + 1]);
}

void tt_copy(lrfg_ctx* ctx, const TTView& src, TT& dst) {
  tt_alloc(ctx, dst, src.d, src.N, src.r);
  for (int j = 0; j < src.d; ++j)
    LRFG_CUDA(cudaMemcpyAsync(dst.core[j].get(), src.core[j], sizeof(double) * celems(src, j),
                              cudaMemcpyDeviceToDevice, ctx->stream));
}

static unsigned grid1d(lrfg_ctx* ctx, long long n) {
  long long g = (n + 255) / 256;
  long long cap = 16LL * (ctx->num_sms > 0 ? ctx->num_sms : 152);
  return (unsigned)std::max(1LL, std::min(g, cap));
}

// ------------------------------------------------------------------------------------------------
// a3: Khatri–Rao product of carriages (App. A.3.1): out[(i*c+k), n, (j*e+l)] = x[i,n,j] y[k,n,l]
// ------------------------------------------------------------------------------------------------
__global__ void khatri_rao_kernel(const double* __restrict__ x, const double* __restrict__ y, double* out, int a,
                                  int c, int n, int b, int e) {
  const long long total = (long long)a * c * n * b * e;
  const int be = b * e;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total; t += (long long)gridDim.x * blockDim.x) {
    int col = (int)(t % be);
    long long rest = t / be;
    int nn = (int)(rest % n);
    int row = (int)(rest / n);
    int i = row / c, k = row - (row / c) * c;
    int j = col / e, l = col - (col / e) * e;
    out[t] = x[((size_t)i * n + nn) * b + j] * y[((size_t)k * n + nn) * e + l];
  }
}

void khatri_rao(lrfg_ctx* ctx, const double* x, int a, int n, int b, const double* y, int c, int e, double* dst) {
  long long total = (long long)a * c * n * b * e;
  if (total == 0) return;
  const double in_bytes = sizeof(double) * ((double)a * n * b + (double)c * n * e);
  LRFG_LAUNCH(ctx, KC_KHATRI_RAO, (double)total, sizeof(double) * (double)total + in_bytes,
              khatri_rao_kernel<<<grid1d(ctx, total), 256, 0, ctx->stream>>>(x, y, dst, a, c, n, b, e));
}

void tt_hadamard(lrfg_ctx* ctx, const TTView& x, const TTView& y, TT& out) {
  LRFG_REQUIRE(x.d == y.d, "Hadamard of TTs of different order");
  int r[4];
  for (int j = 0; j <= x.d; ++j) r[j] = x.r[j] * y.r[j];
  for (int j = 0; j < x.d; ++j) LRFG_REQUIRE(x.N[j] == y.N[j], "Hadamard of TTs on different grids");
  tt_alloc(ctx, out, x.d, x.N, r);
  for (int j = 0; j < x.d; ++j) {
    long long total = (long long)r[j] * x.N[j] * r[j + 1];
    const double in_bytes = sizeof(double) * ((double)x.r[j] * x.N[j] * x.r[j + 1] + (double)y.r[j] * y.N[j] * y.r[j + 1]);
    LRFG_LAUNCH(ctx, KC_KHATRI_RAO, (double)total, sizeof(double) * (double)total + in_bytes,
                khatri_rao_kernel<<<grid1d(ctx, total), 256, 0, ctx->stream>>>(
                    x.core[j], y.core[j], out.core[j].get(), x.r[j], y.r[j], x.N[j], x.r[j + 1], y.r[j + 1]));
  }
}

// ------------------------------------------------------------------------------------------------
// a5: block sum alpha x + beta y; the scalars multiply the first carriage only
// ------------------------------------------------------------------------------------------------
__global__ void block_embed_kernel(const double* __restrict__ src, int a, int n, int b, double* dst, int A, int B,
                                   int oa, int ob, double s, const double* __restrict__ s_dev) {
  const long long total = (long long)a * n * b;
  const double sc = s_dev ? s * (*s_dev) : s;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total; t += (long long)gridDim.x * blockDim.x) {
    int jb = (int)(t % b);
    long long rest = t / b;
    int nn = (int)(rest % n);
    int ia = (int)(rest / n);
    dst[((size_t)(ia + oa) * n + nn) * B + (jb + ob)] = sc * src[t];
  }
}

static void embed(lrfg_ctx* ctx, const double* src, int a, int n, int b, double* dst, int A, int B, int oa, int ob,
                  double s, const double* s_dev) {
  long long total = (long long)a * n * b;
  if (total == 0) return;
  LRFG_LAUNCH(ctx, KC_TT_MISC, (double)total, 2.0 * sizeof(double) * total,
              block_embed_kernel<<<grid1d(ctx, total), 256, 0, ctx->stream>>>(src, a, n, b, dst, A, B, oa, ob, s, s_dev));
}

void tt_embed(lrfg_ctx* ctx, const double* src, int a, int n, int b, double* dst, int A, int B, int oa, int ob) {
  embed(ctx, src, a, n, b, dst, A, B, oa, ob, 1.0, nullptr);
}

void tt_add_many(lrfg_ctx* ctx, const TTView* xs, const double* scales, int nb, TT& out) {
  LRFG_REQUIRE(nb >= 1, "empty sum");
  const int d = xs[0].d;
  int r[4];
  r[0] = 1;
  r[d] = 1;
  for (int j = 1; j < d; ++j) {
    r[j] = 0;
    for (int i = 0; i < nb; ++i) r[j] += xs[i].r[j];
  }
  for (int i = 0; i < nb; ++i) {
    LRFG_REQUIRE(xs[i].d == d, "sum of TTs of different order");
    for (int j = 0; j < d; ++j) LRFG_REQUIRE(xs[i].N[j] == xs[0].N[j], "sum of TTs on different grids");
  }
  tt_alloc(ctx, out, d, xs[0].N, r);
  for (int j = 0; j < d; ++j) {
    double* dst = out.core[j].get();
    const int A = r[j], B = r[j + 1], n = xs[0].N[j];
    if (d > 1 && j != 0 && j != d - 1) fill(ctx, dst, 0.0, (long long)A * n * B);
    int oa = 0, ob = 0;
    for (int i = 0; i < nb; ++i) {
      const TTView& x = xs[i];
      if (d == 1) LRFG_REQUIRE(false, "use tt_add for order-1 tensors");
      if (j == 0) embed(ctx, x.core[j], 1, n, x.r[1], dst, 1, B, 0, ob, scales ? scales[i] : 1.0, nullptr);
      else if (j == d - 1) embed(ctx, x.core[j], x.r[j], n, 1, dst, A, 1, oa, 0, 1.0, nullptr);
      else embed(ctx, x.core[j], x.r[j], n, x.r[j + 1], dst, A, B, oa, ob, 1.0, nullptr);
      oa += x.r[j];
      ob += x.r[j + 1];
    }
  }
}

void tt_add(lrfg_ctx* ctx, double alpha, const double* alpha_dev, const TTView& x, double beta, const double* beta_dev,
            const TTView& y, TT& out) {
  LRFG_REQUIRE(x.d == y.d, "sum of TTs of different order");
  const int d = x.d;
  for (int j = 0; j < d; ++j) LRFG_REQUIRE(x.N[j] == y.N[j], "sum of TTs on different grids");
  int r[4];
  r[0] = 1;
  r[d] = 1;
  for (int j = 1; j < d; ++j) r[j] = x.r[j] + y.r[j];
  tt_alloc(ctx, out, d, x.N, r);
  for (int j = 0; j < d; ++j) {
    double* dst = out.core[j].get();
    const int A = r[j], B = r[j + 1], n = x.N[j];
    if (d == 1) {
      fill(ctx, dst, 0.0, (long long)n);
      // out = alpha x + beta y elementwise (both 1 x n x 1)
      embed(ctx, x.core[0], 1, n, 1, dst, 1, 1, 0, 0, alpha, alpha_dev);
      // accumulate beta y: reuse axpby on a scaled copy
      DBuf<double> tmp(ctx->pool, n);
      embed(ctx, y.core[0], 1, n, 1, tmp.get(), 1, 1, 0, 0, beta, beta_dev);
      axpby(ctx, n, 1.0, tmp.get(), 1.0, dst);
      continue;
    }
    if (j != 0 && j != d - 1) fill(ctx, dst, 0.0, (long long)A * n * B);
    const bool first = (j == 0);
    if (j == 0) {
      embed(ctx, x.core[j], 1, n, x.r[1], dst, 1, B, 0, 0, alpha, alpha_dev);
      embed(ctx, y.core[j], 1, n, y.r[1], dst, 1, B, 0, x.r[1], beta, beta_dev);
    } else if (j == d - 1) {
      embed(ctx, x.core[j], x.r[j], n, 1, dst, A, 1, 0, 0, 1.0, nullptr);
      embed(ctx, y.core[j], y.r[j], n, 1, dst, A, 1, x.r[j], 0, 1.0, nullptr);
    } else {
      embed(ctx, x.core[j], x.r[j], n, x.r[j + 1], dst, A, B, 0, 0, 1.0, nullptr);
      embed(ctx, y.core[j], y.r[j], n, y.r[j + 1], dst, A, B, x.r[j], x.r[j + 1], 1.0, nullptr);
    }
    (void)first;
  }
}

// ------------------------------------------------------------------------------------------------
// a4: rank truncation by Gram-SVD.  TT rounding (App. A.3.3) computes, from left to right, the
// truncated SVD of the unfolding  X_{<=j} = M_j * Rest_j, where M_j is the current left part and
// Rest_j the original carriages right of bond j.  With R_j = Rest_j Rest_j^T (a right-to-left sweep
// of Gram contractions), the left singular vectors of M_j Rest_j follow from two small symmetric
// eigen-problems (the Gram-SVD of Al Daas, Ballard & Benner, "Parallel algorithms for tensor train
// arithmetic", SIAM J. Sci. Comput. 44 (2022)):
//     M^T M = V diag(lam) V^T,   R_A = diag(lam)^{1/2} V^T,   R_A R_j R_A^T = U diag(sig^2) U^T,
//     left factor  Y = M V diag(lam)^{-1/2} U_k  (orthonormal columns),
//     transfer     T = U_k^T R_A                 (= Y^T M),   next left part  T x carriage j+1.
// Directions with lam <= tau lam_max (numerically zero) are dropped from R_A.
// ------------------------------------------------------------------------------------------------
// Bond balancing: with c_i = (R_ii / GA_ii)^{1/4} the diagonal scaling M -> M C, Rest -> C^{-1} Rest
// leaves the tensor unchanged and equalises the two Gram diagonals (GA -> C GA C, R -> C^{-1} R C^{-1}).
// It keeps the eigen-decompositions accurate when the columns of the left part and the rows of the
// right part have very different scales (e.g. after Khatri–Rao products and exponential sums).
__global__ void balance_kernel(double* GAg, double* Rg, double* cg, int m) {
  extern __shared__ double cs[];
  double* GA = GAg + (size_t)blockIdx.x * m * m;
  double* R = Rg + (size_t)blockIdx.x * m * m;
  double* c = cg + (size_t)blockIdx.x * m;
  for (int i = threadIdx.x; i < m; i += blockDim.x) {
    double ga = GA[(size_t)i * m + i], rb = R[(size_t)i * m + i];
    cs[i] = (ga > 0.0 && rb > 0.0) ? sqrt(sqrt(rb / ga)) : 1.0;
    c[i] = cs[i];
  }
  __syncthreads();
  for (int t = threadIdx.x; t < m * m; t += blockDim.x) {
    int i = t / m, j = t - (t / m) * m;
    double f = cs[i] * cs[j];
    GA[t] *= f;
    R[t] /= f;
  }
}

// Estimate of diag(R1) for R1 = C1 (R2 (x) I) C1^T without forming it: the terms with R2's diagonal,
// sum_{i, b'} C1[a][i][b']^2 R2[b'][b'] (exact when R2 is diagonal).  It only sets the balancing
// scales, which change rounding errors, not the truncation.  One block per (a, item).
__global__ void diag_estimate_kernel(const double* __restrict__ C1g, const double* __restrict__ R2g, int a_dim, int n,
                                     int b2, double* dg) {
  const size_t item = blockIdx.y;
  const double* C1 = C1g + item * (size_t)a_dim * n * b2 + (size_t)blockIdx.x * n * b2;
  const double* R2 = R2g + item * (size_t)b2 * b2;
  __shared__ double red[32];
  double s = 0.0;
  for (int t = threadIdx.x; t < n * b2; t += blockDim.x) {
    const int bp = t % b2;
    const double v = C1[t];
    s += v * v * R2[(size_t)bp * b2 + bp];
  }
  for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffff, s, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double v = 0.0;
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) v += red[i];
    dg[item * a_dim + blockIdx.x] = v;
  }
}

// balancing from GA's diagonal and a given right diagonal: c = (r_ii / GA_ii)^{1/4}, GA <- C GA C
__global__ void balance_diag_kernel(double* GAg, const double* __restrict__ rdg, double* cg, int m) {
  extern __shared__ double cs[];
  double* GA = GAg + (size_t)blockIdx.x * m * m;
  const double* rd = rdg + (size_t)blockIdx.x * m;
  double* c = cg + (size_t)blockIdx.x * m;
  for (int i = threadIdx.x; i < m; i += blockDim.x) {
    const double ga = GA[(size_t)i * m + i], rb = rd[i];
    cs[i] = (ga > 0.0 && rb > 0.0) ? sqrt(sqrt(rb / ga)) : 1.0;
    c[i] = cs[i];
  }
  __syncthreads();
  for (int t = threadIdx.x; t < m * m; t += blockDim.x) {
    const int i = t / m, j = t - (t / m) * m;
    GA[t] *= cs[i] * cs[j];
  }
}

// P[b][t] *= c[b] / sigma_t, sigma_t = sqrt(w_t) (0 where w_t <= 0); one batch item per blockIdx.y
__global__ void scale_rows_cols_kernel(double* Pg, const double* __restrict__ cg, const double* __restrict__ wg,
                                       int b, int k) {
  const size_t item = blockIdx.y;
  double* P = Pg + item * (size_t)b * k;
  const double* c = cg + item * (size_t)b;
  const double* w = wg + item * (size_t)b;
  const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (size_t)b * k) return;
  const int row = (int)(t / k), col = (int)(t - (t / k) * k);
  const double sg = w[col] > 0.0 ? sqrt(w[col]) : 0.0;
  P[t] = sg > 0.0 ? P[t] * c[row] / sg : 0.0;
}

// Tolerance truncation (App. A.3.3): at a bond with singular values sigma_i (eigenvalues w_i = sigma_i^2
// of S, whose trace is the squared norm of the unfolding) keep the smallest k with
// sum_{i >= k} w_i <= tol_j^2 trace(S), at least 1 and at most the cap kcap.  Each item gets its own k;
// the columns of its eigenvector block beyond it are zeroed, so an item's truncation is exactly its own
// rank-k one while the batch shares the storage rank max_b k_b.  One block per item.
__global__ void tol_rank_kernel(const double* __restrict__ Sg, const int* __restrict__ rk, const double* __restrict__ wg,
                                double* Vg, int b, int kcap, double tol2, int* kout) {
  const size_t item = blockIdx.x;
  const double* S = Sg + item * (size_t)b * b;
  const double* w = wg + item * (size_t)b;
  double* V = Vg + item * (size_t)b * b;
  __shared__ int ks;
  if (threadIdx.x == 0) {
    const int act = rk ? min(rk[item], b) : b;
    double tr = 0.0;
    for (int i = 0; i < act; ++i) tr += S[(size_t)i * b + i];
    int k = kcap;
    double kept = 0.0;
    for (int i = 0; i < min(kcap, act); ++i) {  // w holds min(kcap, act) eigenvalues
      kept += fmax(w[i], 0.0);
      if (tr - kept <= tol2 * tr) { k = i + 1; break; }
    }
    ks = max(k, 1);
    kout[item] = ks;
  }
  __syncthreads();
  const int k = ks;
  for (int t = threadIdx.x; t < b * (kcap - k); t += blockDim.x) {
    const int row = t / (kcap - k), col = k + t - (t / (kcap - k)) * (kcap - k);
    V[(size_t)row * b + col] = 0.0;
  }
}

void tol_ranks(lrfg_ctx* ctx, const double* S, const int* rk, const double* w, double* V, int b, int kcap, double tol2,
               int nb, int* k_dev) {
  LRFG_LAUNCH(ctx, KC_TT_MISC, (double)b * nb, sizeof(double) * ((double)b * kcap + 2.0 * b) * nb,
              tol_rank_kernel<<<nb, 128, 0, ctx->stream>>>(S, rk, w, V, b, kcap, tol2, k_dev));
}

void tt_round_batch(lrfg_ctx* ctx, const TTBatchView& x, int rmax, TTBatch& out, double tol) {
  LRFG_REQUIRE(rmax >= 1, "truncation rank must be >= 1 (got %d)", rmax);
  LRFG_REQUIRE(tol >= 0.0 && tol < 1.0, "truncation tolerance must be in [0, 1) (got %g)", tol);
  const int d = x.d, nb = x.nb;
  LRFG_REQUIRE(d >= 1 && d <= 3 && nb >= 1, "TT order must be 1..3");
  // ranks after the (implicit) right-to-left orthogonalisation and after truncation, as in TT rounding;
  // with a tolerance, rr[j+1] is the cap and the rank is decided at the bond
  int sp[4], rr[4];
  sp[d] = 1;
  for (int j = d - 1; j >= 1; --j) sp[j] = std::min(x.r[j], x.N[j] * sp[j + 1]);
  rr[0] = 1;
  for (int j = 0; j < d - 1; ++j) rr[j + 1] = std::min(rmax, std::min(rr[j] * x.N[j], sp[j + 1]));
  rr[d] = 1;
  const double tol_j = d > 1 ? tol / std::sqrt((double)(d - 1)) : 0.0;
  if (tol > 0.0) {
    out.d = d;
    out.nb = nb;
    for (int j = 0; j < 3; ++j) out.N[j] = j < d ? x.N[j] : 0;
    for (int j = 0; j < 4; ++j) out.r[j] = 1;
  } else {
    ttb_alloc(ctx, out, d, x.N, rr, nb);
  }
  if (d == 1) {
    if (tol > 0.0) out.core[0] = DBuf<double>(ctx->pool, out.elems(0) * nb);
    LRFG_CUDA(cudaMemcpyAsync(out.core[0].get(), x.core[0], sizeof(double) * x.elems(0) * nb,
                              cudaMemcpyDeviceToDevice, ctx->stream));
    return;
  }
  // right Gram matrices R[j] (s_j x s_j per batch item) of the carriages j..d-1, j = 1..d-1
  DBuf<double> R[4];
  {
    const int j = d - 1;
    const int s = x.r[j], n = x.N[j];
    const long long sx = (long long)x.elems(j), ss = (long long)s * s;
    R[j] = DBuf<double>(ctx->pool, (size_t)ss * nb);
    gemm(ctx, 0, 1, s, s, n, 1.0, x.core[j], n, sx, x.core[j], n, sx, 0.0, R[j].get(), s, ss, nb);
    // d = 3: bond 0 contracts carriage 1 with R[2] after projecting on its left basis (below), so the
    // Gram of carriages 1..2 (the 2 N s^3 term that dominates the rounding of rank-s products) is not
    // formed
    for (int jj = d - 2; jj >= (d == 3 ? 2 : 1); --jj) {
      const int a = x.r[jj], nn = x.N[jj], b = x.r[jj + 1];
      const long long sxj = (long long)x.elems(jj), sb = (long long)b * b, sa = (long long)a * a;
      DBuf<double> T(ctx->pool, (size_t)sxj * nb);
      gemm(ctx, 0, 0, a * nn, b, b, 1.0, x.core[jj], b, sxj, R[jj + 1].get(), b, sb, 0.0, T.get(), b, sxj, nb);
      R[jj] = DBuf<double>(ctx->pool, (size_t)sa * nb);
      gemm(ctx, 0, 1, a, a, nn * b, 1.0, T.get(), nn * b, sxj, x.core[jj], nn * b, sxj, 0.0, R[jj].get(), a, sa, nb);
    }
  }
  // left sweep
  DBuf<double> Z(ctx->pool, x.elems(0) * nb);
  LRFG_CUDA(cudaMemcpyAsync(Z.get(), x.core[0], sizeof(double) * x.elems(0) * nb, cudaMemcpyDeviceToDevice,
                            ctx->stream));
  for (int j = 0; j < d - 1; ++j) {
    if (tol > 0.0) rr[j + 1] = std::min(rmax, std::min(rr[j] * x.N[j], sp[j + 1]));  // cap after bond j-1
    const int a = rr[j], n = x.N[j], b = x.r[j + 1], kcap = rr[j + 1];
    const int rows = a * n;
    const long long sz = (long long)rows * b, sbb = (long long)b * b;
    long long sbk = (long long)b * kcap, skk = (long long)kcap * kcap, sout = 0;
    int k = kcap;
    DBuf<double> GA(ctx->pool, (size_t)sbb * nb), cb(ctx->pool, (size_t)b * nb);
    gemm(ctx, 1, 0, b, b, rows, 1.0, Z.get(), b, sz, Z.get(), b, sz, 0.0, GA.get(), b, sbb, nb);
    const bool projected = (d == 3 && j == 0);
    if (projected) {
      const int n1 = x.N[1], b2 = x.r[2];
      DBuf<double> rd(ctx->pool, (size_t)b * nb);
      LRFG_LAUNCH(ctx, KC_TT_MISC, 3.0 * b * n1 * (double)b2 * nb, sizeof(double) * (double)x.elems(1) * nb,
                  diag_estimate_kernel<<<dim3(b, nb), 256, 0, ctx->stream>>>(x.core[1], R[2].get(), b, n1, b2,
                                                                           rd.get()));
      LRFG_LAUNCH(ctx, KC_TT_MISC, 2.0 * sbb * nb, 2.0 * sizeof(double) * sbb * nb,
                  balance_diag_kernel<<<nb, 256, sizeof(double) * b, ctx->stream>>>(GA.get(), rd.get(), cb.get(), b));
    } else {
      LRFG_LAUNCH(ctx, KC_TT_MISC, 2.0 * sbb * nb, 4.0 * sizeof(double) * sbb * nb,
                  balance_kernel<<<nb, 256, sizeof(double) * b, ctx->stream>>>(GA.get(), R[j + 1].get(), cb.get(), b));
    }
    // The unfolding X = M N (M: rows x b left part, N: b x cols right part) has the Gram matrices
    // GA = M^T M and R = N N^T.  Only the side whose numerical rank is smaller is factored (pivoted
    // Cholesky stops at that rank), and the eigenproblem has that rank as its size.  The left part's
    // rank is at most `rows`, the right part's at most `cols`: the smaller of the two picks the side.
    long long cols = 1;
    for (int i = j + 1; i < d; ++i) cols *= x.N[i];
    const bool left_side = projected || (long long)rows <= cols;
    DBuf<int> rk(ctx->pool, (size_t)nb);
    DBuf<double> F(ctx->pool, (size_t)sbb * nb), F1(ctx->pool, (size_t)sbb * nb), S(ctx->pool, (size_t)sbb * nb);
    DBuf<double> sig(ctx->pool, (size_t)b * nb), US(ctx->pool, (size_t)sbb * nb);
    DBuf<double> P(ctx->pool, (size_t)sbk * nb), T(ctx->pool, (size_t)sbk * nb);
    // the bond's rank: the cap, or with a tolerance the largest of the items' own ranks (their
    // eigenvector columns beyond their own rank zeroed); then the output carriage j
    auto settle_rank = [&]() {
      if (tol > 0.0) {
        DBuf<int> kd(ctx->pool, (size_t)nb);
        tol_ranks(ctx, S.get(), rk.get(), sig.get(), US.get(), b, kcap, tol_j * tol_j, nb, kd.get());
        std::vector<int> kh(nb);
        LRFG_CUDA(cudaMemcpyAsync(kh.data(), kd.get(), sizeof(int) * nb, cudaMemcpyDeviceToHost, ctx->stream));
        LRFG_CUDA(cudaStreamSynchronize(ctx->stream));
        k = 1;
        for (int v : kh) k = std::max(k, std::min(v, kcap));
        rr[j + 1] = k;
        out.r[j + 1] = k;
        out.core[j] = DBuf<double>(ctx->pool, out.elems(j) * nb);
        sbk = (long long)b * k;
        skk = (long long)k * k;
      }
      sout = (long long)out.elems(j);
    };
    if (left_side) {
      // GA ~ RA^T RA, Q = M Pc orthonormal; S = RA R RA^T (nonzero block rho_A x rho_A); Y = Q U_k,
      // transfer T = U_k^T RAc
      DBuf<double> RAc(ctx->pool, (size_t)sbb * nb), Pc(ctx->pool, (size_t)sbb * nb);
      gram_factor(ctx, GA.get(), cb.get(), b, nb, F.get(), RAc.get(), Pc.get(), rk.get());
      if (projected) {
        // S = RAc C1 (R2 (x) I) C1^T RAc^T on the rho_A active rows: Wc = RAc C1 (rho x N1 x b2),
        // Q = Wc R2, S = Q Wc^T over (N1, b2)
        const int n1 = x.N[1], b2 = x.r[2];
        const long long sw = (long long)b * n1 * b2, sr2 = (long long)b2 * b2;
        DBuf<double> Wc(ctx->pool, (size_t)sw * nb), Qw(ctx->pool, (size_t)sw * nb);
        gemm_dyn(ctx, 0, 0, b, n1 * b2, b, 1.0, RAc.get(), b, sbb, x.core[1], n1 * b2, (long long)x.elems(1), 0.0,
                 Wc.get(), n1 * b2, sw, nb, rk.get(), 1, nullptr, 1);
        gemm_dyn(ctx, 0, 0, b * n1, b2, b2, 1.0, Wc.get(), b2, sw, R[2].get(), b2, sr2, 0.0, Qw.get(), b2, sw, nb,
                 rk.get(), n1, nullptr, 1);
        gemm_dyn(ctx, 0, 1, b, b, n1 * b2, 1.0, Qw.get(), n1 * b2, sw, Wc.get(), n1 * b2, sw, 0.0, S.get(), b, sbb,
                 nb, rk.get(), 1, rk.get(), 1);
      } else {
        gemm(ctx, 0, 0, b, b, b, 1.0, F.get(), b, sbb, R[j + 1].get(), b, sbb, 0.0, F1.get(), b, sbb, nb);
        gemm(ctx, 0, 1, b, b, b, 1.0, F1.get(), b, sbb, F.get(), b, sbb, 0.0, S.get(), b, sbb, nb);
      }
      syevx_sized(ctx, S.get(), rk.get(), sig.get(), US.get(), b, kcap, nb);
      settle_rank();
      gemm(ctx, 0, 0, b, k, b, 1.0, Pc.get(), b, sbb, US.get(), b, sbb, 0.0, P.get(), k, sbk, nb);
      gemm(ctx, 0, 0, rows, k, b, 1.0, Z.get(), b, sz, P.get(), k, sbk, 0.0, out.core[j].get(), k, sout, nb);
      gemm(ctx, 1, 0, k, b, b, 1.0, US.get(), b, sbb, RAc.get(), b, sbb, 0.0, T.get(), b, sbk, nb);
    } else {
      // R ~ RB^T RB; the left singular vectors of X are those of M C RB^T (C the balancing): from the
      // eigenvectors W of S' = RB GA RB^T (nonzero block rho_R x rho_R), Y = M C RB^T W Sigma^-1, made
      // orthonormal again by a pivoted-Cholesky pass on Y^T Y (any orthonormal basis of the span gives
      // the same truncation); transfer T = Y^T M, computed explicitly
      gram_factor(ctx, R[j + 1].get(), nullptr, b, nb, F.get(), nullptr, nullptr, rk.get());
      gemm(ctx, 0, 0, b, b, b, 1.0, F.get(), b, sbb, GA.get(), b, sbb, 0.0, F1.get(), b, sbb, nb);
      gemm(ctx, 0, 1, b, b, b, 1.0, F1.get(), b, sbb, F.get(), b, sbb, 0.0, S.get(), b, sbb, nb);
      syevx_sized(ctx, S.get(), rk.get(), sig.get(), US.get(), b, kcap, nb);
      settle_rank();
      DBuf<double> P0(ctx->pool, (size_t)sbk * nb);
      gemm(ctx, 1, 0, b, k, b, 1.0, F.get(), b, sbb, US.get(), b, sbb, 0.0, P0.get(), k, sbk, nb);
      LRFG_LAUNCH(ctx, KC_TT_MISC, 2.0 * sbk * nb, 2.0 * sizeof(double) * sbk * nb,
                  scale_rows_cols_kernel<<<dim3((unsigned)((sbk + 255) / 256), nb), 256, 0, ctx->stream>>>(
                      P0.get(), cb.get(), sig.get(), b, k));
      DBuf<double> Y0(ctx->pool, (size_t)rows * k * nb), G(ctx->pool, (size_t)skk * nb);
      DBuf<double> GR(ctx->pool, (size_t)skk * nb), GP(ctx->pool, (size_t)skk * nb);
      gemm(ctx, 0, 0, rows, k, b, 1.0, Z.get(), b, sz, P0.get(), k, sbk, 0.0, Y0.get(), k, (long long)rows * k, nb);
      gemm(ctx, 1, 0, k, k, rows, 1.0, Y0.get(), k, (long long)rows * k, Y0.get(), k, (long long)rows * k, 0.0,
           G.get(), k, skk, nb);
      DBuf<double> ones(ctx->pool, (size_t)k * nb);
      fill(ctx, ones.get(), 1.0, (long long)k * nb);
      gram_factor(ctx, G.get(), ones.get(), k, nb, GR.get(), nullptr, GP.get(), nullptr);
      gemm(ctx, 0, 0, rows, k, k, 1.0, Y0.get(), k, (long long)rows * k, GP.get(), k, skk, 0.0, out.core[j].get(),
           k, sout, nb);
      gemm(ctx, 1, 0, k, b, rows, 1.0, out.core[j].get(), k, sout, Z.get(), b, sz, 0.0, T.get(), b, sbk, nb);
    }
    // next left part: T (k x b) times carriage j+1 as b x (N s)
    const int n1 = x.N[j + 1], c1 = x.r[j + 2];
    const long long szn = (long long)k * n1 * c1;
    DBuf<double> Zn(ctx->pool, (size_t)szn * nb);
    gemm(ctx, 0, 0, k, n1 * c1, b, 1.0, T.get(), b, sbk, x.core[j + 1], n1 * c1, (long long)x.elems(j + 1), 0.0,
         Zn.get(), n1 * c1, szn, nb);
    Z = std::move(Zn);
  }
  if (tol > 0.0) out.core[d - 1] = DBuf<double>(ctx->pool, out.elems(d - 1) * nb);
  LRFG_CUDA(cudaMemcpyAsync(out.core[d - 1].get(), Z.get(), sizeof(double) * out.elems(d - 1) * nb,
                            cudaMemcpyDeviceToDevice, ctx->stream));
}

void ttb_alloc(lrfg_ctx* ctx, TTBatch& x, int d, const int* N, const int* r, int nb) {
  x.d = d;
  x.nb = nb;
  for (int j = 0; j < 3; ++j) x.N[j] = j < d ? N[j] : 0;
  for (int j = 0; j < 4; ++j) x.r[j] = j <= d ? r[j] : 1;
  x.r[0] = 1;
  x.r[d] = 1;
  for (int j = 0; j < d; ++j) x.core[j] = DBuf<double>(ctx->pool, x.elems(j) * nb);
}

TTBatchView batch_view(const TTBatch& x) {
  TTBatchView v{};
  v.d = x.d;
  v.nb = x.nb;
  for (int j = 0; j < 3; ++j) v.N[j] = x.N[j];
  for (int j = 0; j < 4; ++j) v.r[j] = x.r[j];
  for (int j = 0; j < x.d; ++j) v.core[j] = x.core[j].get();
  return v;
}

TTView item_view(const TTBatch& x, int b) {
  TTView v{};
  v.d = x.d;
  for (int j = 0; j < 3; ++j) v.N[j] = x.N[j];
  for (int j = 0; j < 4; ++j) v.r[j] = x.r[j];
  for (int j = 0; j < x.d; ++j) v.core[j] = x.core[j].get() + (size_t)b * x.elems(j);
  return v;
}

void tt_round(lrfg_ctx* ctx, const TTView& x, int rmax, TT& out, double tol) {
  if (x.d == 1) { tt_copy(ctx, x, out); return; }
  TTBatchView bv{};
  bv.d = x.d;
  bv.nb = 1;
  for (int j = 0; j < 3; ++j) bv.N[j] = x.N[j];
  for (int j = 0; j < 4; ++j) bv.r[j] = x.r[j];
  for (int j = 0; j < x.d; ++j) bv.core[j] = x.core[j];
  TTBatch ob;
  tt_round_batch(ctx, bv, rmax, ob, tol);
  out.d = ob.d;
  for (int j = 0; j < 3; ++j) out.N[j] = ob.N[j];
  for (int j = 0; j < 4; ++j) out.r[j] = ob.r[j];
  for (int j = 0; j < ob.d; ++j) out.core[j] = std::move(ob.core[j]);
}

// ------------------------------------------------------------------------------------------------
// a7: inner product by left-to-right contraction: W_{j+1}[b,e] = sum W_j[a,c] x_j[a,n,b] y_j[c,n,e]
// ------------------------------------------------------------------------------------------------
void tt_dot_device(lrfg_ctx* ctx, const TTView& x, const TTView& y, double* out_dev) {
  LRFG_REQUIRE(x.d == y.d, "dot of TTs of different order");
  DBuf<double> W(ctx->pool, 1);
  fill(ctx, W.get(), 1.0, 1);
  for (int j = 0; j < x.d; ++j) {
    const int a = x.r[j], b = x.r[j + 1], c = y.r[j], e = y.r[j + 1], n = x.N[j];
    LRFG_REQUIRE(n == y.N[j], "dot of TTs on different grids");
    // V (c x (n b)) = W^T (c x a) * x_j (a x (n b))
    DBuf<double> V(ctx->pool, (size_t)c * n * b);
    gemm(ctx, 1, 0, c, n * b, a, 1.0, W.get(), c, 0, x.core[j], n * b, 0, 0.0, V.get(), n * b, 0);
    // W' (b x e) = V^T ((c n) x b)^T * y_j ((c n) x e)
    double* dst = (j == x.d - 1) ? out_dev : nullptr;
    DBuf<double> Wn;
    if (!dst) { Wn = DBuf<double>(ctx->pool, (size_t)b * e); dst = Wn.get(); }
    gemm(ctx, 1, 0, b, e, c * n, 1.0, V.get(), b, 0, y.core[j], e, 0, 0.0, dst, e, 0);
    if (j != x.d - 1) W = std::move(Wn);
  }
}

double tt_dot(lrfg_ctx* ctx, const TTView& x, const TTView& y) {
  DBuf<double> d(ctx->pool, 1);
  tt_dot_device(ctx, x, y, d.get());
  double h = 0.0;
  LRFG_CUDA(cudaMemcpyAsync(&h, d.get(), sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
  LRFG_CUDA(cudaStreamSynchronize(ctx->stream));
  return h;
}

// expand: F_1 = G_0 (N0 x r1); F_{j+1} = F_j (P x r_j) G_j (r_j x N_j r_{j+1})
void tt_expand(lrfg_ctx* ctx, const TTView& x, double* values) {
  const int d = x.d;
  if (d == 1) {
    LRFG_CUDA(cudaMemcpyAsync(values, x.core[0], sizeof(double) * x.N[0], cudaMemcpyDeviceToDevice, ctx->stream));
    return;
  }
  long long P = x.N[0];
  DBuf<double> F(ctx->pool, celems(x, 0));
  LRFG_CUDA(cudaMemcpyAsync(F.get(), x.core[0], sizeof(double) * celems(x, 0), cudaMemcpyDeviceToDevice, ctx->stream));
  for (int j = 1; j < d; ++j) {
    const int a = x.r[j], n = x.N[j], b = x.r[j + 1];
    double* dst;
    DBuf<double> Fn;
    if (j == d - 1) dst = values; else { Fn = DBuf<double>(ctx->pool, (size_t)P * n * b); dst = Fn.get(); }
    LRFG_REQUIRE(P < (1LL << 31), "expanded grid too large");
    gemm(ctx, 0, 0, (int)P, n * b, a, 1.0, F.get(), a, 0, x.core[j], n * b, 0, 0.0, dst, n * b, 0);
    P *= n;
    if (j != d - 1) F = std::move(Fn);
  }
}

// ------------------------------------------------------------------------------------------------
// TT-SVD of a full array (App. A.3.3, first case) via Gram eigen-decompositions of the unfoldings:
// for j < d-1 the left singular vectors of the (r_j N_j) x rest unfolding from its row Gram matrix
// when r_j N_j is the smaller side, else the right ones from the column Gram matrix.
// ------------------------------------------------------------------------------------------------
__global__ void transpose_kernel(const double* __restrict__ in, int rows, int cols, double* out) {
  const long long total = (long long)rows * cols;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total; t += (long long)gridDim.x * blockDim.x) {
    int i = (int)(t / cols), j = (int)(t % cols);
    out[(size_t)j * rows + i] = in[t];
  }
}

// out (cols x rows) = in (rows x cols)^T
static void transpose(lrfg_ctx* ctx, const double* in, int rows, int cols, double* out) {
  long long total = (long long)rows * cols;
  if (total == 0) return;
  LRFG_LAUNCH(ctx, KC_TT_MISC, 0, 2.0 * sizeof(double) * total,
              transpose_kernel<<<grid1d(ctx, total), 256, 0, ctx->stream>>>(in, rows, cols, out));
}

static int keep_rank(const std::vector<double>& lam, int rmax, double tol_j) {
  const int m = (int)lam.size();
  int k = std::min(rmax, m);
  if (tol_j > 0.0) {
    double total = 0.0;
    for (double l : lam) total += std::max(l, 0.0);
    double tail = 0.0;
    int kk = m;
    for (int i = m - 1; i >= 1; --i) {
      double t2 = tail + std::max(lam[i], 0.0);
      if (t2 <= tol_j * tol_j * total) { tail = t2; kk = i; } else break;
    }
    k = std::min(k, kk);
  }
  return std::max(k, 1);
}

void tt_compress(lrfg_ctx* ctx, int d, const int* N, const double* values, int rmax, double tol, TT& out) {
  LRFG_REQUIRE(d >= 2 && d <= 3, "compression needs d in {2,3}");
  LRFG_REQUIRE(rmax >= 1, "rank must be >= 1");
  const double tol_j = tol > 0.0 ? tol / std::sqrt((double)(d - 1)) : 0.0;
  long long total = 1;
  for (int j = 0; j < d; ++j) total *= N[j];
  // current remainder C: rows = r_j N_j, cols = N_{j+1}...N_{d-1}
  DBuf<double> C(ctx->pool, (size_t)total);
  LRFG_CUDA(cudaMemcpyAsync(C.get(), values, sizeof(double) * total, cudaMemcpyDeviceToDevice, ctx->stream));
  int r[4] = {1, 1, 1, 1};
  std::vector<DBuf<double>> cores(d);
  int rj = 1;
  long long cols = total / N[0];
  for (int j = 0; j < d - 1; ++j) {
    const int rows = rj * N[j];
    LRFG_REQUIRE(cols < (1LL << 31), "unfolding too wide");
    const bool use_rows = rows <= cols;
    const int m = use_rows ? rows : (int)cols;
    DBuf<double> G(ctx->pool, (size_t)m * m), lam(ctx->pool, m), V(ctx->pool, (size_t)m * m);
    if (use_rows)
      gemm(ctx, 0, 1, m, m, (int)cols, 1.0, C.get(), (int)cols, 0, C.get(), (int)cols, 0, 0.0, G.get(), m, 0);
    else
      gemm(ctx, 1, 0, m, m, rows, 1.0, C.get(), (int)cols, 0, C.get(), (int)cols, 0, 0.0, G.get(), m, 0);
    syevj(ctx, G.get(), lam.get(), V.get(), m);
    std::vector<double> hl(m);
    LRFG_CUDA(cudaMemcpyAsync(hl.data(), lam.get(), sizeof(double) * m, cudaMemcpyDeviceToHost, ctx->stream));
    LRFG_CUDA(cudaStreamSynchronize(ctx->stream));
    const int k = std::min(keep_rank(hl, rmax, tol_j), std::min(rows, (int)cols));
    // V's first k columns, packed (m x k)
    DBuf<double> Vk(ctx->pool, (size_t)m * k);
    LRFG_CUDA(cudaMemcpy2DAsync(Vk.get(), sizeof(double) * k, V.get(), sizeof(double) * m, sizeof(double) * k, m,
                                cudaMemcpyDeviceToDevice, ctx->stream));
    if (use_rows) {
      // core = U_k (rows x k); remainder = U_k^T C (k x cols)
      cores[j] = DBuf<double>(ctx->pool, (size_t)rows * k);
      LRFG_CUDA(cudaMemcpyAsync(cores[j].get(), Vk.get(), sizeof(double) * rows * k, cudaMemcpyDeviceToDevice, ctx->stream));
      DBuf<double> Cn(ctx->pool, (size_t)k * cols);
      gemm(ctx, 1, 0, k, (int)cols, rows, 1.0, Vk.get(), k, 0, C.get(), (int)cols, 0, 0.0, Cn.get(), (int)cols, 0);
      C = std::move(Cn);
    } else {
      // right singular vectors V_k (cols x k): core = C V_k (rows x k), remainder = V_k^T (k x cols)
      cores[j] = DBuf<double>(ctx->pool, (size_t)rows * k);
      gemm(ctx, 0, 0, rows, k, (int)cols, 1.0, C.get(), (int)cols, 0, Vk.get(), k, 0, 0.0, cores[j].get(), k, 0);
      DBuf<double> Cn(ctx->pool, (size_t)k * cols);
      transpose(ctx, Vk.get(), (int)cols, k, Cn.get());
      C = std::move(Cn);
    }
    r[j + 1] = k;
    rj = k;
    cols /= N[j + 1];
  }
  cores[d - 1] = std::move(C);
  out.d = d;
  for (int j = 0; j < 3; ++j) out.N[j] = j < d ? N[j] : 0;
  for (int j = 0; j <= d; ++j) out.r[j] = r[j];
  for (int j = 0; j < d; ++j) out.core[j] = std::move(cores[j]);
}

// ------------------------------------------------------------------------------------------------
// mode operators and the exponential-sum preconditioner (a1, a6)
// ------------------------------------------------------------------------------------------------
void tt_mode_operator(lrfg_ctx* ctx, const TTView& x, int j, int kind, double param, double scale, TT& out) {
  tt_copy(ctx, x, out);
  fibre_operator(ctx, x.core[j], out.core[j].get(), x.r[j], x.N[j], x.r[j + 1], kind, param, scale);
}

void expsum_inverse(double xmax, double eps, std::vector<double>& t, std::vector<double>& w) {
  // sinc (trapezoidal) quadrature of 1/x = int exp(tau - x e^tau) d tau:  t_m = e^{tau_m}, w_m = h e^{tau_m}
  LRFG_REQUIRE(eps > 0.0 && eps < 1.0 && xmax >= 1.0, "exponential sum needs 0 < eps < 1, xmax >= 1");
  const double pi = 3.14159265358979323846;
  const double h = pi * pi / std::log(32.0 / eps);
  const double tau_min = std::log(eps / (2.0 * xmax));
  const double tau_max = std::log(std::log(2.0 / eps));
  const int R = (int)std::ceil((tau_max - tau_min) / h) + 1;
  t.resize(R);
  w.resize(R);
  for (int m = 0; m < R; ++m) {
    double tau = tau_min + h * m;
    t[m] = std::exp(tau);
    w[m] = h * std::exp(tau);
  }
}

void tt_precond(lrfg_ctx* ctx, const TTView& x, const std::vector<double>& t, const std::vector<double>& w, int rmax,
                TT& out, double tol, const TTView* omega, bool fp32, bool final) {
  // P~^-1 x = sum_m w_m (G_m x ... x G_m) x with G_m = F^-1 diag(exp(-t_m k^2)) F per mode: a TT whose
  // carriages are block rows (first), block diagonal (middle) and block columns (last) over m.
  const int d = x.d;
  const int R = (int)t.size();
  int r[4];
  r[0] = 1;
  r[d] = 1;
  for (int j = 1; j < d; ++j) r[j] = R * x.r[j];
  std::vector<double> ones(R, 1.0);
  if (omega && d >= 2) {
    // randomised rounding: the blocks G_m x_j enter the sketch contractions as they are (never embedded in the
    // block-diagonal carriage)
    SketchSource z;
    z.kind = SketchSource::BLOCKS;
    z.d = d;
    z.nb = 1;
    z.nblocks = R;
    DBuf<double> terms[3];
    for (int j = 0; j < d; ++j) {
      z.N[j] = x.N[j];
      const size_t e = (size_t)x.r[j] * x.N[j] * x.r[j + 1];
      terms[j] = DBuf<double>(ctx->pool, e * R);
      fibre_gauss_multi(ctx, x.core[j], terms[j].get(), (long long)e, x.r[j], x.N[j], x.r[j + 1], t.data(),
                        (j == 0) ? w.data() : ones.data(), R, fp32);
      z.blocks[j] = terms[j].get();
    }
    for (int j = 0; j <= d; ++j) {
      z.s[j] = r[j];
      z.ry[j] = x.r[j];
    }
    TTBatch ob;
    tt_round_sketch(ctx, z, *omega, rmax, ob, tol, fp32, final);
    out.d = ob.d;
    for (int j = 0; j < 3; ++j) out.N[j] = ob.N[j];
    for (int j = 0; j < 4; ++j) out.r[j] = ob.r[j];
    for (int j = 0; j < ob.d; ++j) out.core[j] = std::move(ob.core[j]);
    return;
  }
  TT big;
  tt_alloc(ctx, big, d, x.N, r);
  for (int j = 0; j < d; ++j) {
    const int a = x.r[j], n = x.N[j], b = x.r[j + 1];
    const size_t e = (size_t)a * n * b;
    DBuf<double> terms(ctx->pool, e * R);
    fibre_gauss_multi(ctx, x.core[j], terms.get(), (long long)e, a, n, b, t.data(), (j == 0) ? w.data() : ones.data(), R,
                      fp32);
    double* dst = big.core[j].get();
    if (d > 1 && j != 0 && j != d - 1) fill(ctx, dst, 0.0, (long long)r[j] * n * r[j + 1]);
    for (int m = 0; m < R; ++m) {
      const double* src = terms.get() + m * e;
      if (d == 1) {
        // single mode: plain sum of the terms
        if (m == 0) LRFG_CUDA(cudaMemcpyAsync(dst, src, sizeof(double) * e, cudaMemcpyDeviceToDevice, ctx->stream));
        else axpby(ctx, (long long)e, 1.0, src, 1.0, dst);
      } else if (j == 0) {
        embed(ctx, src, 1, n, b, dst, 1, r[1], 0, m * b, 1.0, nullptr);
      } else if (j == d - 1) {
        embed(ctx, src, a, n, 1, dst, r[j], 1, m * a, 0, 1.0, nullptr);
      } else {
        embed(ctx, src, a, n, b, dst, r[j], r[j + 1], m * a, m * b, 1.0, nullptr);
      }
    }
  }
  tt_round(ctx, view_of(big), rmax, out, tol);
}

}  // namespace lrfg
