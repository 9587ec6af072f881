// Randomised TT rounding of the operator's products (hot-path rows a3/a4 for the material product and a6 for the
// exponential-sum preconditioner).
//
// The deterministic rounding of App. A.3.3 costs O(N s^3) in the input rank s, and after the material product
// (s = r_A r) and the P~^-1 product (s = R r) it dominated one application of Eq. (Pls_lowrank).  This file
// implements "randomize-then-orthogonalize" (Al Daas, Ballard, Cazeaux, Hallman, Miedlar, Pasha, Reid, Saibaba,
// "Randomized algorithms for rounding in the tensor-train format", SIAM J. Sci. Comput. 45 (2023) A74-A95):
//   1. right-to-left contraction with a sketch TT Omega of ranks l:  W_{d-1} = Z_{d-1} Omega_{d-1}^T,
//      W_{j-1} = sum_n Z_j[:, n, :] W_j Omega_j[:, n, :]^T;
//   2. left to right: A = X_j W_j, Q = orth(A), X_j <- Q, X_{j+1} <- (Q^T X_j) x Z_{j+1};
//   3. the rank-l result, left-orthonormal after step 2, is truncated to the target rank or tolerance by the
//      truncated SVDs of App. A.3.3 taken from the right (truncate_left_orth, below).
// The products are never formed: the middle carriage of a Khatri-Rao product Z_1 = x_1 (.) y_1 enters steps 1
// and 2 through two fused kernels that contract x's and y's carriages one after the other (r_A^2 r l + r_A r^2 l
// multiply-adds per fibre index instead of r_A^2 r^2 l), and the block-diagonal middle carriage of the
// preconditioner's product through batched products over its blocks.  orth(A) is CholeskyQR2: a pivoted
// Cholesky factor of A^T A gives a first basis A P L^{-T}, and a second pass on that basis makes it orthonormal
// to rounding.  The first pass stops at pivots below 1e-16 of
// the largest (singular values below ~1e-8 of the largest at the bond: rounding noise of an FP64 Gram matrix);
// its basis is then orthonormal only to ~eps sigma_1^2 / sigma_k^2 in the smallest kept directions, but it lies
// in the span of A to rounding, and the second pass makes it orthonormal without changing that span.
// The sketch has Rademacher entries from SplitMix64 (Steele, Lea, Flood, OOPSLA 2014): entry t of carriage j is
// the sign (top bit) of output (j + 1) 2^40 + t of stream `seed`, the same stream the oracle draws.
#include <algorithm>
#include <cmath>

#include "ops.cuh"

namespace lrfg {

// ------------------------------------------------------------------------------------------------
// sketch carriages
// ------------------------------------------------------------------------------------------------
__device__ __forceinline__ unsigned long long splitmix64_at(unsigned long long seed, unsigned long long i) {
  unsigned long long z = seed + (i + 1ull) * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

__global__ void rademacher_kernel(double* out, long long n, unsigned long long seed, unsigned long long base) {
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x)
    out[t] = (splitmix64_at(seed, base + (unsigned long long)t) >> 63) ? -1.0 : 1.0;
}

static unsigned grid_of(lrfg_ctx* ctx, long long n) {
  long long g = (n + 255) / 256;
  long long cap = 16LL * (ctx->num_sms > 0 ? ctx->num_sms : 152);
  return (unsigned)std::max(1LL, std::min(g, cap));
}

void sketch_tt(lrfg_ctx* ctx, int d, const int* N, int ell, unsigned long long seed, TT& out) {
  LRFG_REQUIRE(ell >= 1, "sketch rank must be >= 1");
  int r[4] = {1, 1, 1, 1};
  for (int j = 1; j < d; ++j) r[j] = ell;
  tt_alloc(ctx, out, d, N, r);
  for (int j = 0; j < d; ++j) {
    const long long n = (long long)out.r[j] * out.N[j] * out.r[j + 1];
    LRFG_LAUNCH(ctx, KC_TT_MISC, 0.0, 8.0 * n,
                rademacher_kernel<<<grid_of(ctx, n), 256, 0, ctx->stream>>>(out.core[j].get(), n, seed,
                                                                           (unsigned long long)(j + 1) << 40));
  }
}

// ------------------------------------------------------------------------------------------------
// fused Khatri-Rao contractions of the middle carriage z[(i,k), n, (i',k')] = x[i,n,i'] y[k,n,k']
// ------------------------------------------------------------------------------------------------
struct ItemPtrs {
  const double* p[kMaxSketchItems];
};

// T[b][(i,k), n, l] = sum_{i',k'} x[i,n,i'] y_b[k,n,k'] W_b[(i',k'), l]: one block per (n, l-chunk, item);
// U[i',k,c] = sum_k' y[k,k'] W[(i',k'), c], then T[(i,k),c] = sum_i' x[i,i'] U[i',k,c]
// S = double, or float on the sketch side of the mixed-precision path (x, y read in FP64 and rounded)
template <typename S>
__global__ void __launch_bounds__(256) kr_right_kernel(const __grid_constant__ ItemPtrs x, int a0, int a1,
                                                       const __grid_constant__ ItemPtrs y,
                                                       int r0, int r1, int N, const S* __restrict__ W,
                                                       long long sW, int ell, int LC, S* T, long long sT) {
  extern __shared__ __align__(16) unsigned char smraw_kr[];
  S* sm = (S*)smraw_kr;
  const int n = blockIdx.x, l0 = blockIdx.y * LC, b = blockIdx.z;
  const int lc = min(LC, ell - l0);
  S* Ws = sm;                               // (a1 r1) x LC
  S* Us = Ws + (size_t)a1 * r1 * LC;        // (a1 r0) x LC
  S* Xs = Us + (size_t)a1 * r0 * LC;        // a0 x a1
  S* Ys = Xs + (size_t)a0 * a1;             // r0 x r1
  const double* yb = y.p[b];
  const double* xb = x.p[b];
  const S* Wb = W + (size_t)b * sW;
  for (int t = threadIdx.x; t < a0 * a1; t += blockDim.x) {
    const int i = t / a1, ip = t - i * a1;
    Xs[t] = (S)xb[((size_t)i * N + n) * a1 + ip];
  }
  for (int t = threadIdx.x; t < r0 * r1; t += blockDim.x) {
    const int k = t / r1, kp = t - k * r1;
    Ys[t] = (S)yb[((size_t)k * N + n) * r1 + kp];
  }
  for (int t = threadIdx.x; t < a1 * r1 * LC; t += blockDim.x) {
    const int row = t / LC, c = t - row * LC;
    Ws[t] = c < lc ? Wb[(size_t)row * ell + l0 + c] : (S)0;
  }
  __syncthreads();
  for (int t = threadIdx.x; t < a1 * r0 * LC; t += blockDim.x) {
    const int row = t / LC, c = t - row * LC;  // row = i' r0 + k
    const int ip = row / r0, k = row - ip * r0;
    const S* yk = Ys + (size_t)k * r1;
    const S* wc = Ws + (size_t)ip * r1 * LC + c;
    S s0 = 0, s1 = 0;
    int kp = 0;
    for (; kp + 1 < r1; kp += 2) {
      s0 = fma(yk[kp], wc[(size_t)kp * LC], s0);
      s1 = fma(yk[kp + 1], wc[(size_t)(kp + 1) * LC], s1);
    }
    if (kp < r1) s0 = fma(yk[kp], wc[(size_t)kp * LC], s0);
    Us[t] = s0 + s1;
  }
  __syncthreads();
  S* Tb = T + (size_t)b * sT;
  for (int t = threadIdx.x; t < a0 * r0 * LC; t += blockDim.x) {
    const int row = t / LC, c = t - row * LC;  // row = i r0 + k
    if (c >= lc) continue;
    const int i = row / r0, k = row - i * r0;
    const S* xi = Xs + (size_t)i * a1;
    S s = 0;
    for (int ip = 0; ip < a1; ++ip) s = fma(xi[ip], Us[((size_t)ip * r0 + k) * LC + c], s);
    Tb[((size_t)row * N + n) * ell + l0 + c] = s;
  }
}

// Out[b][l, n, (i',k')] = sum_{i,k} M_b[l, (i,k)] x[i,n,i'] y_b[k,n,k']: one block per (n, l-chunk, item);
// V[c,i,k'] = sum_k M[c,(i,k)] y[k,k'], then Out[c,(i',k')] = sum_i V[c,i,k'] x[i,i']
__global__ void __launch_bounds__(256) kr_left_kernel(const __grid_constant__ ItemPtrs x, int a0, int a1,
                                                      const __grid_constant__ ItemPtrs y,
                                                      int r0, int r1, int N, const double* __restrict__ M,
                                                      long long sM, int ell, int LC, double* Out, long long sO) {
  extern __shared__ __align__(16) double sm[];
  const int n = blockIdx.x, l0 = blockIdx.y * LC, b = blockIdx.z;
  const int lc = min(LC, ell - l0);
  const int s0w = a0 * r0, s1w = a1 * r1;
  double* Ms = sm;                               // LC x (a0 r0)
  double* Vs = Ms + (size_t)LC * s0w;            // LC x (a0 r1)
  double* Xs = Vs + (size_t)LC * a0 * r1;        // a0 x a1
  double* Ys = Xs + (size_t)a0 * a1;             // r0 x r1
  const double* yb = y.p[b];
  const double* xb = x.p[b];
  const double* Mb = M + (size_t)b * sM;
  for (int t = threadIdx.x; t < a0 * a1; t += blockDim.x) {
    const int i = t / a1, ip = t - i * a1;
    Xs[t] = xb[((size_t)i * N + n) * a1 + ip];
  }
  for (int t = threadIdx.x; t < r0 * r1; t += blockDim.x) {
    const int k = t / r1, kp = t - k * r1;
    Ys[t] = yb[((size_t)k * N + n) * r1 + kp];
  }
  for (int t = threadIdx.x; t < LC * s0w; t += blockDim.x) {
    const int c = t / s0w, col = t - c * s0w;
    Ms[t] = c < lc ? Mb[(size_t)(l0 + c) * s0w + col] : 0.0;
  }
  __syncthreads();
  for (int t = threadIdx.x; t < LC * a0 * r1; t += blockDim.x) {
    const int ci = t / r1, kp = t - ci * r1;  // ci = c a0 + i
    const int c = ci / a0, i = ci - c * a0;
    const double* m = Ms + (size_t)c * s0w + (size_t)i * r0;
    double s0 = 0.0, s1 = 0.0;
    int k = 0;
    for (; k + 1 < r0; k += 2) {
      s0 = fma(m[k], Ys[(size_t)k * r1 + kp], s0);
      s1 = fma(m[k + 1], Ys[(size_t)(k + 1) * r1 + kp], s1);
    }
    if (k < r0) s0 = fma(m[k], Ys[(size_t)k * r1 + kp], s0);
    Vs[t] = s0 + s1;
  }
  __syncthreads();
  double* Ob = Out + (size_t)b * sO;
  for (int t = threadIdx.x; t < LC * s1w; t += blockDim.x) {
    const int c = t / s1w, col = t - c * s1w;  // col = i' r1 + k'
    if (c >= lc) continue;
    const int ip = col / r1, kp = col - ip * r1;
    const double* v = Vs + (size_t)c * a0 * r1 + kp;
    double s = 0.0;
    for (int i = 0; i < a0; ++i) s = fma(v[(size_t)i * r1], Xs[(size_t)i * a1 + ip], s);
    Ob[((size_t)(l0 + c) * N + n) * s1w + col] = s;
  }
}

// Khatri-Rao carriage of every item: out[b][(i,k), n, (i',k')] = x[i,n,i'] y_b[k,n,k'] (first and last carriages of
// the product, which the rounding needs explicitly; they are small)
__global__ void kr_items_kernel(const __grid_constant__ ItemPtrs x, int a0, int a1, const __grid_constant__ ItemPtrs y, int r0,
                                int r1, int N, int nb, double* out) {
  const long long per = (long long)a0 * r0 * N * a1 * r1, total = per * nb;
  const int s1w = a1 * r1;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total; t += (long long)gridDim.x * blockDim.x) {
    const int b = (int)(t / per);
    const long long q = t - b * per;
    const int col = (int)(q % s1w);
    const long long rest = q / s1w;
    const int n = (int)(rest % N), row = (int)(rest / N);
    const int i = row / r0, k = row - i * r0, ip = col / r1, kp = col - ip * r1;
    out[t] = x.p[b][((size_t)i * N + n) * a1 + ip] * y.p[b][((size_t)k * N + n) * r1 + kp];
  }
}

// chunk of the sketch index per block so that the shared memory of one block stays within `budget` bytes
static int chunk_for(size_t per_col, size_t fixed, int ell, size_t budget) {
  for (int lc : {32, 16, 8, 4, 2, 1})
    if (lc <= std::max(ell, 1) && fixed + per_col * lc <= budget) return lc;
  return 1;
}

template <typename S>
static void kr_right(lrfg_ctx* ctx, const ItemPtrs& x, int xn, int a0, int a1, const ItemPtrs& y, int r0, int r1, int N, int nb,
                     const S* W, int ell, S* T) {
  const size_t budget = 100 * 1024;
  const size_t fixed = sizeof(S) * ((size_t)a0 * a1 + (size_t)r0 * r1);
  const size_t per = sizeof(S) * ((size_t)a1 * r1 + (size_t)a1 * r0);
  const int LC = chunk_for(per, fixed, ell, budget);
  const size_t smem = fixed + per * LC;
  LRFG_REQUIRE(smem <= 200 * 1024, "sketch contraction too large for shared memory (ranks %d x %d)", a1, r1);
  LRFG_CUDA(raise_smem_limit((const void*)kr_right_kernel<S>, smem));
  dim3 grid(N, (ell + LC - 1) / LC, nb);
  const double flops = 2.0 * nb * N * (double)ell * ((double)a1 * r0 * r1 + (double)a0 * r0 * a1);
  const double bytes = sizeof(S) * nb * ((double)a0 * r0 * N * ell + (double)a1 * r1 * ell) +
                       sizeof(double) * ((double)xn * a0 * N * a1 + (double)nb * r0 * N * r1);
  LRFG_LAUNCH(ctx, KC_SKETCH, flops, bytes,
              kr_right_kernel<S><<<grid, 256, smem, ctx->stream>>>(x, a0, a1, y, r0, r1, N, W, (long long)a1 * r1 * ell,
                                                                  ell, LC, T, (long long)a0 * r0 * N * ell));
}

static void kr_left(lrfg_ctx* ctx, const ItemPtrs& x, int xn, int a0, int a1, const ItemPtrs& y, int r0, int r1, int N, int nb,
                    const double* M, int ell, double* Out) {
  const size_t budget = 100 * 1024;
  const size_t fixed = sizeof(double) * ((size_t)a0 * a1 + (size_t)r0 * r1);
  const size_t per = sizeof(double) * ((size_t)a0 * r0 + (size_t)a0 * r1);
  const int LC = chunk_for(per, fixed, ell, budget);
  const size_t smem = fixed + per * LC;
  LRFG_REQUIRE(smem <= 200 * 1024, "sketch projection too large for shared memory (ranks %d x %d)", a0, r0);
  LRFG_CUDA(raise_smem_limit((const void*)kr_left_kernel, smem));
  dim3 grid(N, (ell + LC - 1) / LC, nb);
  const double flops = 2.0 * nb * N * (double)ell * ((double)a0 * r1 * r0 + (double)a1 * r1 * a0);
  const double bytes = sizeof(double) * nb * ((double)ell * N * a1 * r1 + (double)r0 * N * r1 + (double)ell * a0 * r0) +
                       sizeof(double) * (double)xn * a0 * N * a1;
  LRFG_LAUNCH(ctx, KC_SKETCH, flops, bytes,
              kr_left_kernel<<<grid, 256, smem, ctx->stream>>>(x, a0, a1, y, r0, r1, N, M, (long long)ell * a0 * r0,
                                                              ell, LC, Out, (long long)ell * N * a1 * r1));
}

// ------------------------------------------------------------------------------------------------
// block-diagonal middle carriage (the exponential-sum product): blocks F_m (r0 x N x r1), m < R
// ------------------------------------------------------------------------------------------------
// out[l, n, m r1 + k'] = tmp[m][l, n, k']
__global__ void block_interleave_kernel(const double* __restrict__ tmp, int R, int ell, int N, int r1, double* out) {
  const long long total = (long long)R * ell * N * r1;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total; t += (long long)gridDim.x * blockDim.x) {
    const int kp = (int)(t % r1);
    long long rest = t / r1;
    const int n = (int)(rest % N);
    rest /= N;
    const int l = (int)(rest % ell);
    const int m = (int)(rest / ell);
    out[((size_t)l * N + n) * ((size_t)R * r1) + (size_t)m * r1 + kp] = tmp[t];
  }
}

// ------------------------------------------------------------------------------------------------
// CholeskyQR2 of nb matrices A (m x l, row-major, item stride m l) into Q (same layout): columns beyond the
// numerical rank are zero.
// ------------------------------------------------------------------------------------------------
static void cholqr2(lrfg_ctx* ctx, const double* A, int m, int l, int nb, double* Q) {
  const long long sa = (long long)m * l, sl = (long long)l * l;
  DBuf<double> G(ctx->pool, (size_t)sl * nb), RA(ctx->pool, (size_t)sl * nb), Pc(ctx->pool, (size_t)sl * nb);
  DBuf<double> ones(ctx->pool, (size_t)l * nb), Q1(ctx->pool, (size_t)sa * nb);
  fill(ctx, ones.get(), 1.0, (long long)l * nb);
  gemm(ctx, 1, 0, l, l, m, 1.0, A, l, sa, A, l, sa, 0.0, G.get(), l, sl, nb);
  gram_factor(ctx, G.get(), ones.get(), l, nb, RA.get(), nullptr, Pc.get(), nullptr, 1e-16);
  gemm(ctx, 0, 0, m, l, l, 1.0, A, l, sa, Pc.get(), l, sl, 0.0, Q1.get(), l, sa, nb);
  gemm(ctx, 1, 0, l, l, m, 1.0, Q1.get(), l, sa, Q1.get(), l, sa, 0.0, G.get(), l, sl, nb);
  gram_factor(ctx, G.get(), ones.get(), l, nb, RA.get(), nullptr, Pc.get(), nullptr, 1e-16);
  gemm(ctx, 0, 0, m, l, l, 1.0, Q1.get(), l, sa, Pc.get(), l, sl, 0.0, Q, l, sa, nb);
}

// ------------------------------------------------------------------------------------------------
// Truncation of the left-orthonormal rank-l result, from the right (App. A.3.3's truncated SVDs with the
// modes read backwards).  Carriages 0..d-2 of y are left-orthonormal, so at bond j (from d-1 down to 1) the
// SVD of the whole unfolding is that of the current carriage j unfolded as a x (n b).  By Gram-SVD:
//     S = C_w C_w^T = V diag(w) V^T   (C_w: carriage j with its last index scaled by the previous bond's
//                                      singular values sqrt(w'); C_w = C at bond d-1),
//     carriage j  <- V_k^T C          (k x n b; the weights stay in the carriages to the right),
//     carriage j-1 <- carriage j-1 V_k (still left-orthonormal: V_k has orthonormal columns).
// The trace of S is the squared norm of the tensor truncated so far, so the tolerance rule of tol_ranks applies
// bond by bond with tol / sqrt(d-1), as in the rounding from the left.  No pivoted-Cholesky factor and no right
// Gram sweep: the orthogonalisation half of the deterministic rounding was done by the sketch's left sweep.
// ------------------------------------------------------------------------------------------------
// out[item][row][t] = X[item][row][t] * sqrt(max(w[item][t], 0)) for t < k (w has stride ws per item)
__global__ void scale_cols_sqrt_kernel(const double* __restrict__ X, const double* __restrict__ wg, int rows, int k,
                                       int ws, double* __restrict__ out) {
  const size_t item = blockIdx.y;
  const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (size_t)rows * k) return;
  const double w = wg[item * ws + (int)(t % k)];
  out[item * (size_t)rows * k + t] = X[item * (size_t)rows * k + t] * (w > 0.0 ? sqrt(w) : 0.0);
}

static void truncate_left_orth(lrfg_ctx* ctx, const TTBatch& y, int rmax, TTBatch& out, double tol) {
  const int d = y.d, nb = y.nb;
  int kr[4] = {1, 1, 1, 1};
  for (int j = d - 1; j >= 1; --j) kr[j] = std::min(rmax, std::min(y.r[j], y.N[j] * kr[j + 1]));
  const double tol_j = d > 1 ? tol / std::sqrt((double)(d - 1)) : 0.0;
  if (tol > 0.0) {
    out.d = d;
    out.nb = nb;
    for (int j = 0; j < 3; ++j) out.N[j] = j < d ? y.N[j] : 0;
    for (int j = 0; j < 4; ++j) out.r[j] = 1;
  } else {
    ttb_alloc(ctx, out, d, y.N, kr, nb);
  }
  // C: carriage j before its truncation (a x cols per item); Cw: the same with the last index weighted
  const double* C = y.core[d - 1].get();
  DBuf<double> Xp, Cw, wprev;
  const double* Cg = C;
  int b = 1;  // rank right of bond j after its truncation
  for (int j = d - 1; j >= 1; --j) {
    const int a = y.r[j], n = y.N[j], cols = n * b, kcap = kr[j];
    const long long sc = (long long)a * cols, saa = (long long)a * a;
    DBuf<double> S(ctx->pool, (size_t)saa * nb), w(ctx->pool, (size_t)a * nb), V(ctx->pool, (size_t)saa * nb);
    gemm(ctx, 0, 1, a, a, cols, 1.0, Cg, cols, sc, Cg, cols, sc, 0.0, S.get(), a, saa, nb);
    syevx(ctx, S.get(), w.get(), V.get(), a, kcap, nb);
    int k = kcap;
    if (tol > 0.0) {
      DBuf<int> kd(ctx->pool, (size_t)nb);
      tol_ranks(ctx, S.get(), nullptr, w.get(), V.get(), a, kcap, tol_j * tol_j, nb, kd.get());
      std::vector<int> kh(nb);
      LRFG_CUDA(cudaMemcpyAsync(kh.data(), kd.get(), sizeof(int) * nb, cudaMemcpyDeviceToHost, ctx->stream));
      LRFG_CUDA(cudaStreamSynchronize(ctx->stream));
      k = 1;
      for (int v : kh) k = std::max(k, std::min(v, kcap));
      out.r[j] = k;
      out.core[j] = DBuf<double>(ctx->pool, out.elems(j) * nb);
    }
    // carriage j of the output: V_k^T C (k x cols)
    gemm(ctx, 1, 0, k, cols, a, 1.0, V.get(), a, saa, C, cols, sc, 0.0, out.core[j].get(), cols,
         (long long)k * cols, nb);
    // carriage j-1 times V_k: rows = r_{j-1} N_{j-1}
    const int rows = y.r[j - 1] * y.N[j - 1];
    const long long sx = (long long)rows * a, sk = (long long)rows * k;
    double* dst;
    DBuf<double> next;
    if (j - 1 == 0) {
      if (tol > 0.0) out.core[0] = DBuf<double>(ctx->pool, out.elems(0) * nb);
      dst = out.core[0].get();
    } else {
      next = DBuf<double>(ctx->pool, (size_t)sk * nb);
      dst = next.get();
    }
    gemm(ctx, 0, 0, rows, k, a, 1.0, y.core[j - 1].get(), a, sx, V.get(), a, saa, 0.0, dst, k, sk, nb);
    if (j - 1 >= 1) {
      // the next bond's Gram sees carriage j-1 with its last index weighted by this bond's singular values
      DBuf<double> cw(ctx->pool, (size_t)sk * nb);
      LRFG_LAUNCH(ctx, KC_TT_MISC, (double)sk * nb, 2.0 * sizeof(double) * sk * nb,
                  scale_cols_sqrt_kernel<<<dim3((unsigned)((sk + 255) / 256), nb), 256, 0, ctx->stream>>>(
                      dst, w.get(), rows, k, a, cw.get()));
      Xp = std::move(next);
      Cw = std::move(cw);
      C = Xp.get();
      Cg = Cw.get();
      b = k;
    }
  }
}

// ------------------------------------------------------------------------------------------------
// the rounding driver
// ------------------------------------------------------------------------------------------------
// A = X W for the left sweep: in FP64, or (fp32) X rounded to FP32 times the FP32 W, the result widened again
static void sketch_product(lrfg_ctx* ctx, bool fp32, int m, int l, int k, const double* X, long long sx,
                           const double* W64, const float* W32, long long sw, double* A, int nb) {
  const long long sa = (long long)m * l;
  if (!fp32) {
    gemm(ctx, 0, 0, m, l, k, 1.0, X, k, sx, W64, l, sw, 0.0, A, l, sa, nb);
    return;
  }
  DBuf<float> X32(ctx->pool, (size_t)sx * nb), A32(ctx->pool, (size_t)sa * nb);
  to_f32(ctx, X, X32.get(), sx * nb);
  gemm_f32(ctx, 0, 0, m, l, k, 1.0, X32.get(), k, sx, W32, l, sw, 0.0, A32.get(), l, sa, nb);
  to_f64(ctx, A32.get(), A, sa * nb);
}

void tt_round_sketch(lrfg_ctx* ctx, const SketchSource& z, const TTView& omega, int rmax, TTBatch& out, double tol,
                     bool fp32, bool final) {
  const int d = z.d, nb = z.nb;
  LRFG_REQUIRE(d >= 2 && d <= 3, "randomised rounding needs d = 2 or 3");
  LRFG_REQUIRE(nb >= 1 && nb <= kMaxSketchItems, "randomised rounding batch of %d items", nb);
  LRFG_REQUIRE(omega.d == d, "sketch order");
  const int* N = z.N;
  const int* s = z.s;
  int l[4] = {1, 1, 1, 1};
  for (int j = 1; j < d; ++j) l[j] = omega.r[j];
  // first and last carriages, materialised per item: Z0 (N x s1), Zl (s_{d-1} x N)
  const long long e0 = (long long)N[0] * s[1], el = (long long)s[d - 1] * N[d - 1];
  DBuf<double> Z0(ctx->pool, (size_t)e0 * nb), Zl(ctx->pool, (size_t)el * nb);
  z.materialise(ctx, 0, Z0.get());
  z.materialise(ctx, d - 1, Zl.get());
  // right sweep: W[d-1] = Zl Omega_{d-1}^T  (s_{d-1} x l_{d-1}), then W[1] = (Z1 x_3 W2) Omega_1^T.  With fp32 the
  // sweep runs in FP32: it only decides the subspaces the left sweep projects on (in FP64)
  DBuf<double> W[3];
  DBuf<float> W32[3], om32[3];
  if (fp32)
    for (int j = 0; j < d; ++j) {
      const long long e = (long long)omega.r[j] * N[j] * omega.r[j + 1];
      om32[j] = DBuf<float>(ctx->pool, (size_t)e);
      to_f32(ctx, omega.core[j], om32[j].get(), e);
    }
  {
    const int j = d - 1;
    if (fp32) {
      W32[j] = DBuf<float>(ctx->pool, (size_t)s[j] * l[j] * nb);
      DBuf<float> Zl32(ctx->pool, (size_t)el * nb);
      to_f32(ctx, Zl.get(), Zl32.get(), el * nb);
      gemm_f32(ctx, 0, 1, s[j], l[j], N[j], 1.0, Zl32.get(), N[j], el, om32[j].get(), N[j], 0, 0.0, W32[j].get(), l[j],
               (long long)s[j] * l[j], nb);
    } else {
      W[j] = DBuf<double>(ctx->pool, (size_t)s[j] * l[j] * nb);
      gemm(ctx, 0, 1, s[j], l[j], N[j], 1.0, Zl.get(), N[j], el, omega.core[j], N[j], 0, 0.0, W[j].get(), l[j],
           (long long)s[j] * l[j], nb);
    }
  }
  if (d == 3) {
    // T1 = Z1 x_3 W2 (s1 x N1 x l2), W1 = T1 Omega_1^T over (n, l2)
    const long long st = (long long)s[1] * N[1] * l[2];
    if (fp32) {
      DBuf<float> T1(ctx->pool, (size_t)st * nb);
      z.right_middle_f32(ctx, W32[2].get(), l[2], T1.get());
      W32[1] = DBuf<float>(ctx->pool, (size_t)s[1] * l[1] * nb);
      gemm_f32(ctx, 0, 1, s[1], l[1], N[1] * l[2], 1.0, T1.get(), N[1] * l[2], st, om32[1].get(), N[1] * l[2], 0, 0.0,
               W32[1].get(), l[1], (long long)s[1] * l[1], nb);
    } else {
      DBuf<double> T1(ctx->pool, (size_t)st * nb);
      z.right_middle(ctx, W[2].get(), l[2], T1.get());
      W[1] = DBuf<double>(ctx->pool, (size_t)s[1] * l[1] * nb);
      gemm(ctx, 0, 1, s[1], l[1], N[1] * l[2], 1.0, T1.get(), N[1] * l[2], st, omega.core[1], N[1] * l[2], 0, 0.0,
           W[1].get(), l[1], (long long)s[1] * l[1], nb);
    }
  }
  // left sweep
  TTBatch y;
  y.d = d;
  y.nb = nb;
  for (int j = 0; j < 3; ++j) y.N[j] = j < d ? N[j] : 0;
  y.r[0] = 1;
  for (int j = 1; j < d; ++j) y.r[j] = l[j];
  y.r[d] = 1;
  // bond 1: A = Z0 W1 (N0 x l1), Q0 = orth(A), M1 = Q0^T Z0 (l1 x s1)
  const long long sq0 = (long long)N[0] * l[1];
  y.core[0] = DBuf<double>(ctx->pool, (size_t)sq0 * nb);
  DBuf<double> M(ctx->pool, (size_t)l[1] * s[1] * nb);
  {
    DBuf<double> A(ctx->pool, (size_t)sq0 * nb);
    sketch_product(ctx, fp32, N[0], l[1], s[1], Z0.get(), e0, W[1].get(), W32[1].get(), (long long)s[1] * l[1],
                   A.get(), nb);
    cholqr2(ctx, A.get(), N[0], l[1], nb, y.core[0].get());
    gemm(ctx, 1, 0, l[1], s[1], N[0], 1.0, y.core[0].get(), l[1], sq0, Z0.get(), s[1], e0, 0.0, M.get(), s[1],
         (long long)l[1] * s[1], nb);
  }
  Z0.reset();
  if (d == 3) {
    // X1 = M1 x_1 Z1 (l1 x N1 x s2); bond 2: A = X1 W2 ((l1 N1) x l2), Q1 = orth(A), M2 = Q1^T X1 (l2 x s2)
    const long long sx = (long long)l[1] * N[1] * s[2], sq1 = (long long)l[1] * N[1] * l[2];
    DBuf<double> X1(ctx->pool, (size_t)sx * nb);
    z.left_middle(ctx, M.get(), l[1], X1.get());
    y.core[1] = DBuf<double>(ctx->pool, (size_t)sq1 * nb);
    {
      DBuf<double> A(ctx->pool, (size_t)sq1 * nb);
      sketch_product(ctx, fp32, l[1] * N[1], l[2], s[2], X1.get(), sx, W[2].get(), W32[2].get(),
                     (long long)s[2] * l[2], A.get(), nb);
      cholqr2(ctx, A.get(), l[1] * N[1], l[2], nb, y.core[1].get());
    }
    M = DBuf<double>(ctx->pool, (size_t)l[2] * s[2] * nb);
    gemm(ctx, 1, 0, l[2], s[2], l[1] * N[1], 1.0, y.core[1].get(), l[2], sq1, X1.get(), s[2], sx, 0.0, M.get(), s[2],
         (long long)l[2] * s[2], nb);
  }
  // last carriage: M_{d-1} Zl  (l_{d-1} x N_{d-1})
  const int jl = d - 1;
  const long long sy = (long long)l[jl] * N[jl];
  y.core[jl] = DBuf<double>(ctx->pool, (size_t)sy * nb);
  gemm(ctx, 0, 0, l[jl], N[jl], s[jl], 1.0, M.get(), s[jl], (long long)l[jl] * s[jl], Zl.get(), N[jl], el, 0.0,
       y.core[jl].get(), N[jl], sy, nb);
  // truncation of the left-orthonormal rank-l result from the right (or, without `final`, that result itself)
  if (!final) {
    out = std::move(y);
    return;
  }
  truncate_left_orth(ctx, y, rmax, out, tol);
}

// ------------------------------------------------------------------------------------------------
// sources
// ------------------------------------------------------------------------------------------------
// carriage j of every item's coefficient factor: its own (xi) or the shared one (x)
static ItemPtrs coeff_items(const SketchSource& z, int j) {
  ItemPtrs p{};
  for (int b = 0; b < z.nb; ++b) p.p[b] = z.xi[j][b] ? z.xi[j][b] : z.x.core[j];
  return p;
}

void SketchSource::materialise(lrfg_ctx* ctx, int j, double* dst) const {
  const long long e = (long long)s[j] * N[j] * s[j + 1];
  if (kind == KHATRI_RAO) {
    ItemPtrs p{};
    for (int b = 0; b < nb; ++b) p.p[b] = y[j][b];
    const long long total = e * nb;
    const double xn = xi[j][0] ? nb : 1;
    LRFG_LAUNCH(ctx, KC_KHATRI_RAO, (double)total,
                sizeof(double) * ((double)total + xn * x.r[j] * N[j] * x.r[j + 1] + (double)nb * ry[j] * N[j] * ry[j + 1]),
                kr_items_kernel<<<grid_of(ctx, total), 256, 0, ctx->stream>>>(coeff_items(*this, j), x.r[j], x.r[j + 1],
                                                                            p, ry[j], ry[j + 1], N[j], nb, dst));
    return;
  }
  for (int b = 0; b < nb; ++b) {
    double* o = dst + (size_t)b * e;
    if (kind == DENSE) {
      LRFG_CUDA(cudaMemcpyAsync(o, dense[j] + (size_t)b * e, sizeof(double) * e, cudaMemcpyDeviceToDevice,
                                ctx->stream));
    } else if (kind == KHATRI_RAO) {
      khatri_rao(ctx, xi[j][b] ? xi[j][b] : x.core[j], x.r[j], N[j], x.r[j + 1], y[j][b], ry[j], ry[j + 1], o);
    } else {
      // exponential-sum blocks F_m of carriage j (r_j x N x r_{j+1} each, weights already in carriage 0)
      const int R = nblocks, a = ry[j], c = ry[j + 1];
      const long long be = (long long)a * N[j] * c, bs = bstride[j] ? bstride[j] : be;
      const double* src = blocks[j] + (size_t)b * be;
      if (j == 0) {
        for (int m = 0; m < R; ++m) tt_embed(ctx, src + m * bs, 1, N[j], c, o, 1, R * c, 0, m * c);
      } else {
        for (int m = 0; m < R; ++m) tt_embed(ctx, src + m * bs, a, N[j], 1, o, R * a, 1, m * a, 0);
      }
    }
  }
}

void SketchSource::right_middle(lrfg_ctx* ctx, const double* W, int ell, double* T) const {
  const int n = N[1];
  if (kind == DENSE) {
    const long long e = (long long)s[1] * n * s[2];
    gemm(ctx, 0, 0, s[1] * n, ell, s[2], 1.0, dense[1], s[2], e, W, ell, (long long)s[2] * ell, 0.0, T, ell,
         (long long)s[1] * n * ell, nb);
  } else if (kind == KHATRI_RAO) {
    ItemPtrs p{};
    for (int b = 0; b < nb; ++b) p.p[b] = y[1][b];
    kr_right<double>(ctx, coeff_items(*this, 1), xi[1][0] ? nb : 1, x.r[1], x.r[2], p, ry[1], ry[2], n, nb, W, ell, T);
  } else {
    // T[(m,k), n, l] = sum_k' F_m[k, n, k'] W[(m,k'), l]: for each item, one product per block
    const int R = nblocks, a = ry[1], c = ry[2];
    const long long be = (long long)a * n * c, bs = bstride[1] ? bstride[1] : be;
    for (int b = 0; b < nb; ++b)
      gemm(ctx, 0, 0, a * n, ell, c, 1.0, blocks[1] + (size_t)b * be, c, bs, W + (size_t)b * s[2] * ell, ell,
           (long long)c * ell, 0.0, T + (size_t)b * s[1] * n * ell, ell, (long long)a * n * ell, R);
  }
}

void SketchSource::right_middle_f32(lrfg_ctx* ctx, const float* W, int ell, float* T) const {
  const int n = N[1];
  if (kind == KHATRI_RAO) {
    ItemPtrs p{};
    for (int b = 0; b < nb; ++b) p.p[b] = y[1][b];
    kr_right<float>(ctx, coeff_items(*this, 1), xi[1][0] ? nb : 1, x.r[1], x.r[2], p, ry[1], ry[2], n, nb, W, ell, T);
  } else if (kind == DENSE) {
    const long long e = (long long)s[1] * n * s[2];
    DBuf<float> Z32(ctx->pool, (size_t)e * nb);
    to_f32(ctx, dense[1], Z32.get(), e * nb);
    gemm_f32(ctx, 0, 0, s[1] * n, ell, s[2], 1.0, Z32.get(), s[2], e, W, ell, (long long)s[2] * ell, 0.0, T, ell,
             (long long)s[1] * n * ell, nb);
  } else {
    const int R = nblocks, a = ry[1], c = ry[2];
    const long long be = (long long)a * n * c, bs = bstride[1] ? bstride[1] : be;
    const long long extent = (R - 1) * bs + nb * be;
    DBuf<float> B32(ctx->pool, (size_t)extent);
    to_f32(ctx, blocks[1], B32.get(), extent);
    for (int b = 0; b < nb; ++b)
      gemm_f32(ctx, 0, 0, a * n, ell, c, 1.0, B32.get() + (size_t)b * be, c, bs, W + (size_t)b * s[2] * ell, ell,
               (long long)c * ell, 0.0, T + (size_t)b * s[1] * n * ell, ell, (long long)a * n * ell, R);
  }
}

void SketchSource::left_middle(lrfg_ctx* ctx, const double* M, int ell, double* X) const {
  const int n = N[1];
  if (kind == DENSE) {
    const long long e = (long long)s[1] * n * s[2];
    gemm(ctx, 0, 0, ell, n * s[2], s[1], 1.0, M, s[1], (long long)ell * s[1], dense[1], n * s[2], e, 0.0, X, n * s[2],
         (long long)ell * n * s[2], nb);
  } else if (kind == KHATRI_RAO) {
    ItemPtrs p{};
    for (int b = 0; b < nb; ++b) p.p[b] = y[1][b];
    kr_left(ctx, coeff_items(*this, 1), xi[1][0] ? nb : 1, x.r[1], x.r[2], p, ry[1], ry[2], n, nb, M, ell, X);
  } else {
    // tmp[m][l, n, k'] = sum_k M[l, (m,k)] F_m[k, n, k'], then interleaved into X[l, n, (m,k')], item by item
    const int R = nblocks, a = ry[1], c = ry[2];
    const long long be = (long long)a * n * c, bs = bstride[1] ? bstride[1] : be;
    DBuf<double> tmp(ctx->pool, (size_t)R * ell * n * c);
    const long long total = (long long)R * ell * n * c;
    for (int b = 0; b < nb; ++b) {
      gemm(ctx, 0, 0, ell, n * c, a, 1.0, M + (size_t)b * ell * s[1], R * a, (long long)a, blocks[1] + (size_t)b * be,
           n * c, bs, 0.0, tmp.get(), n * c, (long long)ell * n * c, R);
      LRFG_LAUNCH(ctx, KC_TT_MISC, 0.0, 16.0 * total,
                  block_interleave_kernel<<<grid_of(ctx, total), 256, 0, ctx->stream>>>(
                      tmp.get(), R, ell, n, c, X + (size_t)b * ell * n * s[2]));
    }
  }
}

}  // namespace lrfg
