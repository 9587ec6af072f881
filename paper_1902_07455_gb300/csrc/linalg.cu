// Dense FP64 building blocks for the rank truncation and the solvers: batched GEMM (Gram matrices and
// core contractions), a cyclic two-sided Jacobi eigensolver for the small symmetric Gram matrices,
// and reductions.
#include <algorithm>
#include <cmath>

#include "ops.cuh"

namespace lrfg {

// ------------------------------------------------------------------------------------------------
// GEMM: 64x64 output tile per block, k-step 16, 256 threads with 4x4 outputs each (rows ty+16i,
// columns tx+16j).  Long-K products split K across blocks (split-K) and accumulate with atomics.
// ------------------------------------------------------------------------------------------------
constexpr int GT = 64, GK = 16;

template <bool TA, bool TB>
__global__ void __launch_bounds__(256) dgemm_kernel(int M, int N, int K, double alpha, const double* __restrict__ A,
                                                    int lda, long long sA, const double* __restrict__ B, int ldb,
                                                    long long sB, double beta, double* C, int ldc, long long sC,
                                                    int splits, int kchunk) {
  __shared__ double As[GK][GT + 1];
  __shared__ double Bs[GK][GT + 1];
  const int batch = blockIdx.z / splits, split = blockIdx.z - (blockIdx.z / splits) * splits;
  A += (size_t)batch * sA;
  B += (size_t)batch * sB;
  C += (size_t)batch * sC;
  const int m0 = blockIdx.y * GT, n0 = blockIdx.x * GT;
  const int kbeg = split * kchunk, kend = min(K, kbeg + kchunk);
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  double acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = 0.0;
  for (int k0 = kbeg; k0 < kend; k0 += GK) {
    for (int e = threadIdx.x; e < GT * GK; e += 256) {
      int mm, kk;
      if (TA) { mm = e % GT; kk = e / GT; } else { kk = e % GK; mm = e / GK; }
      int gm = m0 + mm, gk = k0 + kk;
      double v = 0.0;
      if (gm < M && gk < kend) v = TA ? A[(size_t)gk * lda + gm] : A[(size_t)gm * lda + gk];
      As[kk][mm] = v;
    }
    for (int e = threadIdx.x; e < GT * GK; e += 256) {
      int nn, kk;
      if (TB) { kk = e % GK; nn = e / GK; } else { nn = e % GT; kk = e / GT; }
      int gn = n0 + nn, gk = k0 + kk;
      double v = 0.0;
      if (gn < N && gk < kend) v = TB ? B[(size_t)gn * ldb + gk] : B[(size_t)gk * ldb + gn];
      Bs[kk][nn] = v;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < GK; ++kk) {
      double a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[kk][ty + 16 * i];
#pragma unroll
      for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tx + 16 * j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    int gm = m0 + ty + 16 * i;
    if (gm >= M) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      int gn = n0 + tx + 16 * j;
      if (gn >= N) continue;
      double* c = C + (size_t)gm * ldc + gn;
      if (splits > 1) {
        atomicAdd(c, alpha * acc[i][j]);
      } else {
        *c = (beta == 0.0) ? alpha * acc[i][j] : alpha * acc[i][j] + beta * (*c);
      }
    }
  }
}

__global__ void scale_matrix_kernel(double* C, int M, int N, int ldc, long long sC, int batch, double beta) {
  long long total = (long long)M * N * batch;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total; t += (long long)gridDim.x * blockDim.x) {
    long long b = t / ((long long)M * N);
    long long rem = t - b * M * N;
    int i = (int)(rem / N), j = (int)(rem % N);
    double* c = C + (size_t)b * sC + (size_t)i * ldc + j;
    *c = (beta == 0.0) ? 0.0 : beta * (*c);
  }
}

void gemm(lrfg_ctx* ctx, int transA, int transB, int M, int N, int K, double alpha, const double* A, int lda,
          long long sA, const double* B, int ldb, long long sB, double beta, double* C, int ldc, long long sC,
          int batch) {
  if (M <= 0 || N <= 0 || batch <= 0) return;
  if (K <= 0) {
    LRFG_LAUNCH(ctx, KC_GEMM, (double)M * N * batch, 2.0 * sizeof(double) * M * N * batch,
                scale_matrix_kernel<<<std::min(1024LL, ((long long)M * N * batch + 255) / 256), 256, 0, ctx->stream>>>(
                    C, M, N, ldc, sC, batch, beta));
    return;
  }
  const int tm = (M + GT - 1) / GT, tn = (N + GT - 1) / GT;
  long long tiles = (long long)tm * tn * batch;
  int target = 2 * (ctx->num_sms > 0 ? ctx->num_sms : 152);
  int splits = 1;
  if (tiles < target) {
    splits = (int)std::min<long long>((target + tiles - 1) / tiles, (K + 255) / 256);
    if (splits < 1) splits = 1;
  }
  int kchunk = (K + splits - 1) / splits;
  kchunk = ((kchunk + GK - 1) / GK) * GK;
  splits = (K + kchunk - 1) / kchunk;
  LRFG_REQUIRE((long long)batch * splits < 65535, "gemm batch too large");
  if (splits > 1) {
    LRFG_LAUNCH(ctx, KC_GEMM, (double)M * N * batch, 2.0 * sizeof(double) * M * N * batch,
                scale_matrix_kernel<<<std::min(1024LL, ((long long)M * N * batch + 255) / 256), 256, 0, ctx->stream>>>(
                    C, M, N, ldc, sC, batch, beta));
  }
  dim3 grid(tn, tm, batch * splits);
  const double flops = 2.0 * M * N * (double)K * batch;
  const double bytes = sizeof(double) * ((double)M * K + (double)K * N + (double)M * N) * batch;
  if (!transA && !transB)
    LRFG_LAUNCH(ctx, KC_GEMM, flops, bytes, dgemm_kernel<false, false><<<grid, 256, 0, ctx->stream>>>(
        M, N, K, alpha, A, lda, sA, B, ldb, sB, beta, C, ldc, sC, splits, kchunk));
  else if (transA && !transB)
    LRFG_LAUNCH(ctx, KC_GEMM, flops, bytes, dgemm_kernel<true, false><<<grid, 256, 0, ctx->stream>>>(
        M, N, K, alpha, A, lda, sA, B, ldb, sB, beta, C, ldc, sC, splits, kchunk));
  else if (!transA && transB)
    LRFG_LAUNCH(ctx, KC_GEMM, flops, bytes, dgemm_kernel<false, true><<<grid, 256, 0, ctx->stream>>>(
        M, N, K, alpha, A, lda, sA, B, ldb, sB, beta, C, ldc, sC, splits, kchunk));
  else
    LRFG_LAUNCH(ctx, KC_GEMM, flops, bytes, dgemm_kernel<true, true><<<grid, 256, 0, ctx->stream>>>(
        M, N, K, alpha, A, lda, sA, B, ldb, sB, beta, C, ldc, sC, splits, kchunk));
}

// ------------------------------------------------------------------------------------------------
// Symmetric eigensolver: cyclic two-sided Jacobi with the round-robin (circle) ordering, so that each
// round applies m'/2 disjoint rotations in parallel (Golub & Van Loan, "Matrix Computations", 4th ed.,
// Sec. 8.5 — the 2x2 symmetric Schur step and parallel orderings).  One block per matrix; the working
// matrices live in shared memory when they fit, otherwise in a global scratch slice.
// ------------------------------------------------------------------------------------------------
constexpr int kJacobiMaxSweeps = 30;

__device__ __forceinline__ void rr_pair(int round, int i, int mp, int* p, int* q) {
  // circle method: player mp-1 fixed, the others rotate
  const int n1 = mp - 1;
  if (i == 0) { *p = round % n1; *q = n1; return; }
  *p = (round + i) % n1;
  *q = (round - i + n1) % n1;
}

__global__ void __launch_bounds__(256) jacobi_kernel(double* Ag, double* w, double* Vout, int m, double* scratch,
                                                     int use_smem) {
  extern __shared__ double sm[];
  const int mp = m + (m & 1);
  const int npair = mp / 2;
  double* A;
  double* V;
  double* Ain = Ag + (size_t)blockIdx.x * m * m;
  double* cs = sm;            // 2 * npair (c, s)
  int* pq = (int*)(cs + 2 * npair);  // 2 * npair
  double* red = (double*)(pq + 2 * npair + ((2 * npair) & 1));  // 64 doubles for reductions
  int* rank = (int*)(red + 64);      // m ints
  if (use_smem) {
    A = (double*)(rank + m + (m & 1));
    V = A + (size_t)m * m;
  } else {
    A = scratch + (size_t)blockIdx.x * 2 * m * m;
    V = A + (size_t)m * m;
  }
  for (int t = threadIdx.x; t < m * m; t += blockDim.x) {
    A[t] = Ain[t];
    V[t] = ((t / m) == (t % m)) ? 1.0 : 0.0;
  }
  __syncthreads();
  // reference scale: Frobenius norm of A
  double loc = 0.0;
  for (int t = threadIdx.x; t < m * m; t += blockDim.x) loc += A[t] * A[t];
  for (int o = 16; o; o >>= 1) loc += __shfl_xor_sync(0xffffffff, loc, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = loc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) s += red[i];
    red[32] = s;
  }
  __syncthreads();
  const double fro2 = red[32];
  const double tiny = 1e-300;
  if (m > 1 && fro2 > 0.0) {
    for (int sweep = 0; sweep < kJacobiMaxSweeps; ++sweep) {
      for (int round = 0; round < mp - 1; ++round) {
        for (int i = threadIdx.x; i < npair; i += blockDim.x) {
          int p, q;
          rr_pair(round, i, mp, &p, &q);
          if (p > q) { int t = p; p = q; q = t; }
          double c = 1.0, s = 0.0;
          if (q < m) {
            double apq = A[(size_t)p * m + q];
            double app = A[(size_t)p * m + p], aqq = A[(size_t)q * m + q];
            if (fabs(apq) > tiny && fabs(apq) > 1e-18 * sqrt(fabs(app * aqq))) {
              double tau = (aqq - app) / (2.0 * apq);
              double t = (tau >= 0.0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
              c = 1.0 / sqrt(1.0 + t * t);
              s = t * c;
            }
          } else {
            q = -1;
          }
          cs[2 * i] = c;
          cs[2 * i + 1] = s;
          pq[2 * i] = p;
          pq[2 * i + 1] = q;
        }
        __syncthreads();
        // rows: A <- J^T A
        for (int t = threadIdx.x; t < npair * m; t += blockDim.x) {
          int i = t / m, j = t - (t / m) * m;
          int p = pq[2 * i], q = pq[2 * i + 1];
          if (q < 0) continue;
          double c = cs[2 * i], s = cs[2 * i + 1];
          if (s == 0.0) continue;
          double ap = A[(size_t)p * m + j], aq = A[(size_t)q * m + j];
          A[(size_t)p * m + j] = c * ap - s * aq;
          A[(size_t)q * m + j] = s * ap + c * aq;
        }
        __syncthreads();
        // columns: A <- A J, V <- V J
        for (int t = threadIdx.x; t < npair * m; t += blockDim.x) {
          int i = t / m, j = t - (t / m) * m;
          int p = pq[2 * i], q = pq[2 * i + 1];
          if (q < 0) continue;
          double c = cs[2 * i], s = cs[2 * i + 1];
          if (s == 0.0) continue;
          double ap = A[(size_t)j * m + p], aq = A[(size_t)j * m + q];
          A[(size_t)j * m + p] = c * ap - s * aq;
          A[(size_t)j * m + q] = s * ap + c * aq;
          double vp = V[(size_t)j * m + p], vq = V[(size_t)j * m + q];
          V[(size_t)j * m + p] = c * vp - s * vq;
          V[(size_t)j * m + q] = s * vp + c * vq;
        }
        __syncthreads();
      }
      // convergence: off-diagonal mass relative to ||A||_F
      double off = 0.0;
      for (int t = threadIdx.x; t < m * m; t += blockDim.x) {
        int i = t / m, j = t - (t / m) * m;
        if (i != j) off += A[t] * A[t];
      }
      for (int o = 16; o; o >>= 1) off += __shfl_xor_sync(0xffffffff, off, o);
      if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = off;
      __syncthreads();
      if (threadIdx.x == 0) {
        double s = 0.0;
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) s += red[i];
        red[33] = s;
      }
      __syncthreads();
      const double offs = red[33];
      __syncthreads();
      if (offs <= (double)m * (double)m * 1e-30 * fro2) break;
    }
  }
  // sort descending: rank[j] = position of eigenvalue j (ties by index)
  for (int j = threadIdx.x; j < m; j += blockDim.x) {
    double lj = A[(size_t)j * m + j];
    int pos = 0;
    for (int i = 0; i < m; ++i) {
      double li = A[(size_t)i * m + i];
      if (li > lj || (li == lj && i < j)) ++pos;
    }
    rank[j] = pos;
  }
  __syncthreads();
  double* wb = w + (size_t)blockIdx.x * m;
  double* Vb = Vout + (size_t)blockIdx.x * m * m;
  for (int j = threadIdx.x; j < m; j += blockDim.x) wb[rank[j]] = A[(size_t)j * m + j];
  for (int t = threadIdx.x; t < m * m; t += blockDim.x) {
    int i = t / m, j = t - (t / m) * m;
    Vb[(size_t)i * m + rank[j]] = V[t];
  }
}

void syevj(lrfg_ctx* ctx, double* A, double* w, double* V, int m, int batch) {
  if (m <= 0 || batch <= 0) return;
  const int mp = m + (m & 1);
  const int npair = mp / 2;
  size_t head = sizeof(double) * 2 * npair + sizeof(int) * (2 * npair + ((2 * npair) & 1)) + sizeof(double) * 64 +
                sizeof(int) * (m + (m & 1));
  head = (head + 15) / 16 * 16;
  size_t full = head + sizeof(double) * 2 * (size_t)m * m;
  int use_smem = full <= (size_t)std::min(ctx->max_smem_optin, 200 * 1024) ? 1 : 0;
  size_t smem = use_smem ? full : head;
  DBuf<double> scratch;
  if (!use_smem) scratch = DBuf<double>(ctx->pool, (size_t)2 * m * m * batch);
  LRFG_CUDA(cudaFuncSetAttribute(jacobi_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  // one sweep of the two-sided cyclic Jacobi costs about 9 m^3 flops (rows, columns and V)
  LRFG_LAUNCH(ctx, KC_EIGEN, 9.0 * (double)m * m * m * batch, 3.0 * sizeof(double) * (double)m * m * batch,
              jacobi_kernel<<<batch, 256, smem, ctx->stream>>>(A, w, V, m, scratch.get(), use_smem));
}

// ------------------------------------------------------------------------------------------------
// elementwise and reductions
// ------------------------------------------------------------------------------------------------
__global__ void fill_kernel(double* x, double v, long long n) {
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x)
    x[t] = v;
}

__global__ void axpby_kernel(long long n, double a, const double* __restrict__ x, double b, double* y) {
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x)
    y[t] = (b == 0.0) ? a * x[t] : a * x[t] + b * y[t];
}

static unsigned grid_for(lrfg_ctx* ctx, long long n) {
  long long g = (n + 255) / 256;
  long long cap = 8LL * (ctx->num_sms > 0 ? ctx->num_sms : 152);
  return (unsigned)std::max(1LL, std::min(g, cap));
}

void fill(lrfg_ctx* ctx, double* x, double v, long long n) {
  if (n <= 0) return;
  LRFG_LAUNCH(ctx, KC_TT_MISC, 0, sizeof(double) * (double)n,
              fill_kernel<<<grid_for(ctx, n), 256, 0, ctx->stream>>>(x, v, n));
}

void axpby(lrfg_ctx* ctx, long long n, double alpha, const double* x, double beta, double* y) {
  if (n <= 0) return;
  LRFG_LAUNCH(ctx, KC_TT_MISC, 3.0 * n, 3.0 * sizeof(double) * n,
              axpby_kernel<<<grid_for(ctx, n), 256, 0, ctx->stream>>>(n, alpha, x, beta, y));
}

// two-stage deterministic dot: fixed grid of partial sums, then one block sums them in order
constexpr int kDotBlocks = 304;

__global__ void __launch_bounds__(256) dot_partial_kernel(const double* __restrict__ x, const double* __restrict__ y,
                                                          long long n, double* partial) {
  __shared__ double red[8];
  double s = 0.0;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x)
    s = fma(x[t], y[t], s);
  for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffff, s, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double v = 0.0;
    for (int i = 0; i < 8; ++i) v += red[i];
    partial[blockIdx.x] = v;
  }
}

__global__ void sum_partials_kernel(const double* __restrict__ partial, int n, double* out) {
  __shared__ double red[8];
  double s = 0.0;
  for (int t = threadIdx.x; t < n; t += blockDim.x) s += partial[t];
  for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffff, s, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double v = 0.0;
    for (int i = 0; i < 8; ++i) v += red[i];
    *out = v;
  }
}

void dot_device(lrfg_ctx* ctx, const double* x, const double* y, long long n, double* out) {
  DBuf<double> partial(ctx->pool, kDotBlocks);
  LRFG_LAUNCH(ctx, KC_REDUCE, 2.0 * n, 2.0 * sizeof(double) * n,
              dot_partial_kernel<<<kDotBlocks, 256, 0, ctx->stream>>>(x, y, n, partial.get()));
  LRFG_LAUNCH(ctx, KC_REDUCE, kDotBlocks, kDotBlocks * sizeof(double),
              sum_partials_kernel<<<1, 256, 0, ctx->stream>>>(partial.get(), kDotBlocks, out));
}

double dot_host(lrfg_ctx* ctx, const double* x, const double* y, long long n) {
  DBuf<double> d(ctx->pool, 1);
  dot_device(ctx, x, y, n, d.get());
  double h = 0.0;
  LRFG_CUDA(cudaMemcpyAsync(&h, d.get(), sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
  LRFG_CUDA(cudaStreamSynchronize(ctx->stream));
  return h;
}

}  // namespace lrfg
