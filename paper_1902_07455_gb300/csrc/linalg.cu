// Dense FP64 building blocks for the rank truncation and the solvers: batched GEMM (Gram matrices and
// core contractions), a cyclic two-sided Jacobi eigensolver for the small symmetric Gram matrices,
// and reductions.
#include <algorithm>
#include <cmath>
#include <type_traits>

#include "ops.cuh"

namespace lrfg {

// ------------------------------------------------------------------------------------------------
// GEMM, FP64.  On this part the FP64 pipe (2 FMA/clk/SM) is the bottleneck of every product here, so
// the kernel is built to waste none of it: a block owns a 64 x 64 (small products: 32 x 32) output block
// (clipped to the active sizes, which may be read from the device), each of its 256 threads owns up to 16
// (4) outputs of that block exactly (no padded tile rows or columns are computed), operands are staged
// through shared memory in k-steps of 32, and long K is split across blocks until about two blocks per SM are busy (split-K: each
// split writes its partial block to a workspace; the last split of a tile to arrive, found by an arrival
// counter, sums the partials in split order, so every product, and with it every solve, is bitwise
// reproducible whatever else runs on the GPU, and no second launch is needed).  With many splits the sum is
// two-level: the splits form groups of about sqrt(splits); the last split of each group to arrive sums its
// group's partials in order into a group partial, and the last group sums the group partials in order — the
// reduction then runs on as many blocks as there are groups instead of on one.  An output costs two
// shared-memory reads per FMA, far below the shared-memory bandwidth at the FP64 rate.
// ------------------------------------------------------------------------------------------------
constexpr int GK = 32;  // k-step

// pk[j] = (row << 16) | column of output j within the block
template <int NR, int TILE, typename T>
__device__ __forceinline__ void gemm_fma_rows(T* acc, const T (*As)[TILE + 1], const T (*Bs)[TILE + 1],
                                              const int* pk, int kk_end) {
  for (int kk = 0; kk < kk_end; ++kk) {
#pragma unroll
    for (int j = 0; j < NR; ++j) acc[j] = fma(As[kk][pk[j] >> 16], Bs[kk][pk[j] & 0xffff], acc[j]);
  }
}

// dynM / dynN (optional, per batch item): the product is computed only for rows < dynM[b] * mulM and
// columns < dynN[b] * mulN (data-dependent active sizes, e.g. numerical ranks); the rest of C is not
// written.  With splits > 1 the partial sums go to part[((split * batches + item) * M + row) * N + column]
// (M, N the static sizes).  TILE = 64 (16 outputs per thread), 32 (4 per thread, for small products:
// four times the blocks, so that a product of a few tiles still spreads over the SMs) or 16 (one per thread,
// for products of one or a few 32-tiles with a short K, see gemm_impl).
// T = double (the FP64 products) or float (the FP32 sketch products of the mixed-precision path).
template <bool TA, bool TB, int TILE, typename T>
__global__ void __launch_bounds__(256) dgemm_kernel(int M, int N, int K, double alpha_d, const T* __restrict__ A,
                                                    int lda, long long sA, const T* __restrict__ B, int ldb,
                                                    long long sB, double beta_d, T* C, int ldc, long long sC,
                                                    int splits, int kchunk, const int* __restrict__ dynM, int mulM,
                                                    const int* __restrict__ dynN, int mulN, double* work,
                                                    T* __restrict__ part, unsigned int* __restrict__ cnt,
                                                    int gsize) {
  constexpr int NMAX = TILE * TILE / 256;
  const T alpha = (T)alpha_d, beta = (T)beta_d;
  __shared__ T As[GK][TILE + 1];
  __shared__ T Bs[GK][TILE + 1];
  const int batch = blockIdx.z;
  const int bm = blockIdx.y / splits, split = blockIdx.y - (blockIdx.y / splits) * splits;
  const int bn = blockIdx.x;
  A += (size_t)batch * sA;
  B += (size_t)batch * sB;
  C += (size_t)batch * sC;
  const int Ms = M, Ns = N;
  if (dynM) M = min(M, dynM[batch] * mulM);
  if (dynN) N = min(N, dynN[batch] * mulN);
  if (work && bm == 0 && bn == 0 && split == 0 && threadIdx.x == 0)
    add_work(work, 2.0 * M * N * (double)K, (double)sizeof(T) * ((double)M * K + (double)K * N + (double)M * N));
  const int m0 = bm * TILE, n0 = bn * TILE;
  const int Mb = min(TILE, M - m0), Nb = min(TILE, N - n0);
  if (Mb <= 0 || Nb <= 0) return;
  const int kbeg = split * kchunk, kend = min(K, kbeg + kchunk);
  // this thread's outputs o = t + 256 j < Mb Nb, as (row, column) within the block
  const int tot = Mb * Nb;
  const int nact = tot > (int)threadIdx.x ? min(NMAX, (tot - (int)threadIdx.x + 255) / 256) : 0;
  int pk[NMAX];
  T acc[NMAX];
#pragma unroll
  for (int j = 0; j < NMAX; ++j) {
    const int o = threadIdx.x + 256 * j;
    const int m = o / Nb;
    pk[j] = j < nact ? (m << 16) | (o - m * Nb) : 0;
    acc[j] = (T)0;
  }
  for (int k0 = kbeg; k0 < kend; k0 += GK) {
    const int kc = min(GK, kend - k0);
    for (int e = threadIdx.x; e < TILE * GK; e += 256) {
      int mm, kk;
      if (TA) { mm = e % TILE; kk = e / TILE; } else { kk = e % GK; mm = e / GK; }
      T v = (T)0;
      if (mm < Mb && kk < kc) v = TA ? A[(size_t)(k0 + kk) * lda + m0 + mm] : A[(size_t)(m0 + mm) * lda + k0 + kk];
      As[kk][mm] = v;
    }
    for (int e = threadIdx.x; e < TILE * GK; e += 256) {
      int nn, kk;
      if (TB) { kk = e % GK; nn = e / GK; } else { nn = e % TILE; kk = e / TILE; }
      T v = (T)0;
      if (nn < Nb && kk < kc) v = TB ? B[(size_t)(n0 + nn) * ldb + k0 + kk] : B[(size_t)(k0 + kk) * ldb + n0 + nn];
      Bs[kk][nn] = v;
    }
    __syncthreads();
    if constexpr (NMAX == 16) {
      switch (nact) {
        case 16: gemm_fma_rows<16, TILE>(acc, As, Bs, pk, kc); break;
        case 15: gemm_fma_rows<15, TILE>(acc, As, Bs, pk, kc); break;
        case 14: gemm_fma_rows<14, TILE>(acc, As, Bs, pk, kc); break;
        case 13: gemm_fma_rows<13, TILE>(acc, As, Bs, pk, kc); break;
        case 12: gemm_fma_rows<12, TILE>(acc, As, Bs, pk, kc); break;
        case 11: gemm_fma_rows<11, TILE>(acc, As, Bs, pk, kc); break;
        case 10: gemm_fma_rows<10, TILE>(acc, As, Bs, pk, kc); break;
        case 9: gemm_fma_rows<9, TILE>(acc, As, Bs, pk, kc); break;
        case 8: gemm_fma_rows<8, TILE>(acc, As, Bs, pk, kc); break;
        case 7: gemm_fma_rows<7, TILE>(acc, As, Bs, pk, kc); break;
        case 6: gemm_fma_rows<6, TILE>(acc, As, Bs, pk, kc); break;
        case 5: gemm_fma_rows<5, TILE>(acc, As, Bs, pk, kc); break;
        case 4: gemm_fma_rows<4, TILE>(acc, As, Bs, pk, kc); break;
        case 3: gemm_fma_rows<3, TILE>(acc, As, Bs, pk, kc); break;
        case 2: gemm_fma_rows<2, TILE>(acc, As, Bs, pk, kc); break;
        case 1: gemm_fma_rows<1, TILE>(acc, As, Bs, pk, kc); break;
        default: break;
      }
    } else if constexpr (NMAX == 4) {
      switch (nact) {
        case 4: gemm_fma_rows<4, TILE>(acc, As, Bs, pk, kc); break;
        case 3: gemm_fma_rows<3, TILE>(acc, As, Bs, pk, kc); break;
        case 2: gemm_fma_rows<2, TILE>(acc, As, Bs, pk, kc); break;
        case 1: gemm_fma_rows<1, TILE>(acc, As, Bs, pk, kc); break;
        default: break;
      }
    } else {
      if (nact == 1) gemm_fma_rows<1, TILE>(acc, As, Bs, pk, kc);
    }
    __syncthreads();
  }
  if (splits > 1) {
    const size_t pstride = (size_t)gridDim.z * Ms * Ns;  // between the splits of one output
    T* P = part + (size_t)batch * Ms * Ns;
#pragma unroll
    for (int j = 0; j < NMAX; ++j) {
      if (j >= nact) break;
      P[split * pstride + (size_t)(m0 + (pk[j] >> 16)) * Ns + n0 + (pk[j] & 0xffff)] = acc[j];
    }
    __shared__ unsigned int s_last;
    const size_t tile_id = ((size_t)batch * gridDim.y / splits + bm) * gridDim.x + bn;
    unsigned int* c = cnt + tile_id;
    // the partials the tile's last block sums: every split's (one level), or every group's (two levels: the
    // group partials sit after the splits' in the workspace)
    int nsum = splits;
    const T* S = P;
    if (gsize < splits) {
      const int ngroups = (splits + gsize - 1) / gsize;
      const int g = split / gsize, g0 = g * gsize, gn = min(gsize, splits - g0);
      unsigned int* cg = cnt + kSplitKCounters + tile_id * kSplitKGroups + g;
      __threadfence();
      __syncthreads();
      if (threadIdx.x == 0) {
        const unsigned int prev = atomicAdd(cg, 1u);
        s_last = (prev == (unsigned int)gn - 1u) ? 1u : 0u;
      }
      __syncthreads();
      if (!s_last) return;
      __threadfence();
      // the group's last split: its partials in split order into group partial g
#pragma unroll
      for (int j = 0; j < NMAX; ++j) {
        if (j >= nact) break;
        const size_t off = (size_t)(m0 + (pk[j] >> 16)) * Ns + n0 + (pk[j] & 0xffff);
        T v = (T)0;
        for (int s = g0; s < g0 + gn; ++s) v += __ldcg(P + s * pstride + off);
        P[(size_t)(splits + g) * pstride + off] = v;
      }
      if (threadIdx.x == 0) *cg = 0u;
      nsum = ngroups;
      S = P + (size_t)splits * pstride;
    }
    // the last (split or group) of this tile to arrive sums the partials in order
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) {
      const unsigned int prev = atomicAdd(c, 1u);
      s_last = (prev == (unsigned int)nsum - 1u) ? 1u : 0u;
    }
    __syncthreads();
    if (!s_last) return;
    __threadfence();
#pragma unroll
    for (int j = 0; j < NMAX; ++j) {
      if (j >= nact) break;
      const size_t off = (size_t)(m0 + (pk[j] >> 16)) * Ns + n0 + (pk[j] & 0xffff);
      T v = (T)0;
      for (int s = 0; s < nsum; ++s) v += __ldcg(S + s * pstride + off);
      T* cp = C + (size_t)(m0 + (pk[j] >> 16)) * ldc + n0 + (pk[j] & 0xffff);
      *cp = (beta_d == 0.0) ? alpha * v : alpha * v + beta * (*cp);
    }
    if (threadIdx.x == 0) *c = 0u;  // ready for the next product
    return;
  }
#pragma unroll
  for (int j = 0; j < NMAX; ++j) {
    if (j >= nact) break;
    T* c = C + (size_t)(m0 + (pk[j] >> 16)) * ldc + n0 + (pk[j] & 0xffff);
    *c = (beta_d == 0.0) ? alpha * acc[j] : alpha * acc[j] + beta * (*c);
  }
}

template <int TILE, typename T>
static void launch_dgemm(lrfg_ctx* ctx, int transA, int transB, dim3 grid, double flops, double bytes, int M, int N,
                         int K, double alpha, const T* A, int lda, long long sA, const T* B, int ldb,
                         long long sB, double beta, T* C, int ldc, long long sC, int splits, int kchunk,
                         const int* dynM, int mulM, const int* dynN, int mulN, double* work, T* part,
                         int gsize = 1 << 30) {
  if (!transA && !transB)
    LRFG_LAUNCH_KC(ctx, (std::is_same<T, float>::value ? KC_GEMM32 : KC_GEMM), flops, bytes, dgemm_kernel<false, false, TILE, T><<<grid, 256, 0, ctx->stream>>>(
        M, N, K, alpha, A, lda, sA, B, ldb, sB, beta, C, ldc, sC, splits, kchunk, dynM, mulM, dynN, mulN, work, part,
        ctx->splitk_cnt, gsize));
  else if (transA && !transB)
    LRFG_LAUNCH_KC(ctx, (std::is_same<T, float>::value ? KC_GEMM32 : KC_GEMM), flops, bytes, dgemm_kernel<true, false, TILE, T><<<grid, 256, 0, ctx->stream>>>(
        M, N, K, alpha, A, lda, sA, B, ldb, sB, beta, C, ldc, sC, splits, kchunk, dynM, mulM, dynN, mulN, work, part,
        ctx->splitk_cnt, gsize));
  else if (!transA && transB)
    LRFG_LAUNCH_KC(ctx, (std::is_same<T, float>::value ? KC_GEMM32 : KC_GEMM), flops, bytes, dgemm_kernel<false, true, TILE, T><<<grid, 256, 0, ctx->stream>>>(
        M, N, K, alpha, A, lda, sA, B, ldb, sB, beta, C, ldc, sC, splits, kchunk, dynM, mulM, dynN, mulN, work, part,
        ctx->splitk_cnt, gsize));
  else
    LRFG_LAUNCH_KC(ctx, (std::is_same<T, float>::value ? KC_GEMM32 : KC_GEMM), flops, bytes, dgemm_kernel<true, true, TILE, T><<<grid, 256, 0, ctx->stream>>>(
        M, N, K, alpha, A, lda, sA, B, ldb, sB, beta, C, ldc, sC, splits, kchunk, dynM, mulM, dynN, mulN, work, part,
        ctx->splitk_cnt, gsize));
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
  gemm_dyn(ctx, transA, transB, M, N, K, alpha, A, lda, sA, B, ldb, sB, beta, C, ldc, sC, batch, nullptr, 1,
           nullptr, 1);
}

template <typename T>
static void gemm_impl(lrfg_ctx* ctx, int transA, int transB, int M, int N, int K, double alpha, const T* A, int lda,
                      long long sA, const T* B, int ldb, long long sB, double beta, T* C, int ldc, long long sC,
                      int batch, const int* dynM, int mulM, const int* dynN, int mulN) {
  if (M <= 0 || N <= 0 || batch <= 0) return;
  if (K <= 0) {
    LRFG_REQUIRE((std::is_same<T, double>::value), "FP32 product with an empty inner dimension");
    LRFG_LAUNCH(ctx, KC_GEMM, (double)M * N * batch, 2.0 * sizeof(double) * M * N * batch,
                scale_matrix_kernel<<<std::min(1024LL, ((long long)M * N * batch + 255) / 256), 256, 0, ctx->stream>>>(
                    (double*)C, M, N, ldc, sC, batch, beta));
    return;
  }
  LRFG_REQUIRE(batch < 65536, "gemm batch too large");
  const int nsm = ctx->num_sms > 0 ? ctx->num_sms : 152;
  // blocks expected to be active: the static count, or for data-dependent sizes a quarter of it (the
  // numerical ranks are typically well below their bounds), at least one per item
  auto active_tiles = [&](int tile) {
    long long a = (long long)((M + tile - 1) / tile) * ((N + tile - 1) / tile) * batch;
    if (dynM || dynN) a = std::max<long long>(batch, a / 4);
    return a;
  };
  // 32 x 32 tiles for thin products (one side <= 32: the 64-row staging would be mostly padding), when
  // 64 x 64 ones would leave most SMs idle, or when they fill the SMs more evenly: the FP64 pipe is shared by
  // the blocks of an SM, so a product takes as long as its busiest SM, ceil(blocks / SMs) blocks (static
  // sizes only: with data-dependent sizes the active tiles are not known here, and the split count is what
  // spreads those products)
  auto fill = [&](long long blocks) { return (double)blocks / (double)(((blocks + nsm - 1) / nsm) * nsm); };
  const bool dyn = dynM || dynN;
  int tile = (!dyn && (std::min(M, N) <= 32 || active_tiles(64) < nsm ||
                       fill(active_tiles(32)) > fill(active_tiles(64)) + 0.05))
                 ? 32
                 : 64;
  // 16 x 16 tiles when even the largest split of the 32-tiles leaves most SMs idle: one k-step of a 32-tile
  // block is 32 K FMAs, 8 us of one SM's FP64 pipe, so a product of a few 32-tiles whose K is too short to
  // split further runs on a few SMs for that long; 16-tiles give four times the blocks at a quarter of the work
  if (tile == 32 && active_tiles(32) * std::max(1, K / GK) < nsm) tile = 16;
  const long long active = active_tiles(tile);
  // split long K until about two blocks per SM are busy, without passing that (a second, partial round of
  // blocks would cost as much as the first)
  const int target = 2 * nsm;
  int splits = 1;
  if (active < target) {
    splits = (int)std::min<long long>((target + active - 1) / active, std::max(1, K / GK));
    if (active * splits > target) splits = (int)std::max<long long>(1, target / active);
  }
  int kchunk = (K + splits - 1) / splits;
  kchunk = ((kchunk + GK - 1) / GK) * GK;
  splits = (K + kchunk - 1) / kchunk;
  const int bmn = (M + tile - 1) / tile, bnn = (N + tile - 1) / tile;
  LRFG_REQUIRE((long long)bmn * splits < 65536, "gemm too many row blocks x splits");
  if (splits > 1)
    LRFG_REQUIRE((long long)bmn * bnn * batch <= kSplitKCounters, "split-K product with too many output tiles");
  // two-level reduction of the partials from 9 splits on: groups of ceil(sqrt(splits))
  int gsize = 1 << 30, ngroups = 0;
  if (splits > 8) {
    gsize = (int)std::ceil(std::sqrt((double)splits));
    ngroups = (splits + gsize - 1) / gsize;
    LRFG_REQUIRE(ngroups <= kSplitKGroups, "split-K product with too many groups (%d)", ngroups);
  }
  DBuf<T> part;
  if (splits > 1) part = DBuf<T>(ctx->pool, (size_t)(splits + ngroups) * M * N * batch);
  // products with data-dependent sizes count their work on the device
  double* work = (dynM || dynN) ? work_counter(ctx, KC_GEMM) : nullptr;
  const double flops = work ? 0.0 : 2.0 * M * N * (double)K * batch;
  const double bytes = work ? 0.0 : sizeof(T) * ((double)M * K + (double)K * N + (double)M * N) * batch;
  dim3 grid(bnn, bmn * splits, batch);
  if (tile == 16)
    launch_dgemm<16, T>(ctx, transA, transB, grid, flops, bytes, M, N, K, alpha, A, lda, sA, B, ldb, sB, beta, C, ldc,
                     sC, splits, kchunk, dynM, mulM, dynN, mulN, work, part.get(), gsize);
  else if (tile == 32)
    launch_dgemm<32, T>(ctx, transA, transB, grid, flops, bytes, M, N, K, alpha, A, lda, sA, B, ldb, sB, beta, C, ldc,
                     sC, splits, kchunk, dynM, mulM, dynN, mulN, work, part.get(), gsize);
  else
    launch_dgemm<64, T>(ctx, transA, transB, grid, flops, bytes, M, N, K, alpha, A, lda, sA, B, ldb, sB, beta, C, ldc,
                     sC, splits, kchunk, dynM, mulM, dynN, mulN, work, part.get(), gsize);
}

void gemm_dyn(lrfg_ctx* ctx, int transA, int transB, int M, int N, int K, double alpha, const double* A, int lda,
              long long sA, const double* B, int ldb, long long sB, double beta, double* C, int ldc, long long sC,
              int batch, const int* dynM, int mulM, const int* dynN, int mulN) {
  gemm_impl<double>(ctx, transA, transB, M, N, K, alpha, A, lda, sA, B, ldb, sB, beta, C, ldc, sC, batch, dynM, mulM,
                    dynN, mulN);
}

void gemm_f32(lrfg_ctx* ctx, int transA, int transB, int M, int N, int K, double alpha, const float* A, int lda,
              long long sA, const float* B, int ldb, long long sB, double beta, float* C, int ldc, long long sC,
              int batch) {
  gemm_impl<float>(ctx, transA, transB, M, N, K, alpha, A, lda, sA, B, ldb, sB, beta, C, ldc, sC, batch, nullptr, 1,
                   nullptr, 1);
}

// The same product in one pass over K (no split-K): it needs no partial-sum workspace, so it takes nothing
// from the context's pool.  For callers that must not allocate.
void gemm_nosplit(lrfg_ctx* ctx, int transA, int transB, int M, int N, int K, double alpha, const double* A, int lda,
                  long long sA, const double* B, int ldb, long long sB, double beta, double* C, int ldc, long long sC,
                  int batch) {
  if (M <= 0 || N <= 0 || batch <= 0) return;
  if (K <= 0) {
    LRFG_LAUNCH(ctx, KC_GEMM, (double)M * N * batch, 2.0 * sizeof(double) * M * N * batch,
                scale_matrix_kernel<<<std::min(1024LL, ((long long)M * N * batch + 255) / 256), 256, 0, ctx->stream>>>(
                    C, M, N, ldc, sC, batch, beta));
    return;
  }
  LRFG_REQUIRE(batch < 65536, "gemm batch too large");
  const int nsm = ctx->num_sms > 0 ? ctx->num_sms : 152;
  const long long tiles64 = (long long)((M + 63) / 64) * ((N + 63) / 64) * batch;
  const int tile = tiles64 < nsm ? 32 : 64;
  const int bmn = (M + tile - 1) / tile, bnn = (N + tile - 1) / tile;
  LRFG_REQUIRE(bmn < 65536, "gemm too many row blocks");
  const int kchunk = ((K + GK - 1) / GK) * GK;
  const double flops = 2.0 * M * N * (double)K * batch;
  const double bytes = sizeof(double) * ((double)M * K + (double)K * N + (double)M * N) * batch;
  dim3 grid(bnn, bmn, batch);
  if (tile == 32)
    launch_dgemm<32, double>(ctx, transA, transB, grid, flops, bytes, M, N, K, alpha, A, lda, sA, B, ldb, sB, beta, C,
                             ldc, sC, 1, kchunk, nullptr, 1, nullptr, 1, nullptr, nullptr);
  else
    launch_dgemm<64, double>(ctx, transA, transB, grid, flops, bytes, M, N, K, alpha, A, lda, sA, B, ldb, sB, beta, C,
                             ldc, sC, 1, kchunk, nullptr, 1, nullptr, 1, nullptr, nullptr);
}

// ------------------------------------------------------------------------------------------------
// Symmetric eigensolver, two stages:
//  1. cyclic two-sided Jacobi with the round-robin (circle) ordering, so that each round applies m'/2
//     disjoint rotations in parallel (Golub & Van Loan, "Matrix Computations", 4th ed., Sec. 8.5: the
//     2x2 symmetric Schur step and parallel orderings).  One block per matrix, working matrices in
//     shared memory when they fit, else in a global scratch slice.  The working precision T is FP32
//     for speed (GB300 issues FP32 at ~58x its FP64 rate) or FP64.
//  2. (FP32 start) refinement to FP64 accuracy by the iteration of Ogita & Aishima, "Iterative
//     refinement for symmetric eigenvalue decomposition", Japan J. Indust. Appl. Math. 35 (2018):
//        R = I - X^T X,  S = X^T A X,  lam_i = S_ii / (1 - R_ii),
//        E_ij = (S_ij + lam_j R_ij) / (lam_j - lam_i)  if |lam_i - lam_j| > delta,  R_ij / 2 otherwise,
//        X <- X + X E,   delta = 2 (||S - diag(lam)|| + ||A|| ||R||),
//     which converges quadratically; eigenvalues closer than delta are treated as a cluster whose
//     invariant subspace (not its individual vectors) is refined.  All of it is GEMM work in FP64.
// ------------------------------------------------------------------------------------------------
constexpr int kJacobiMaxSweeps = 30;
constexpr int kJacobiThreads = 512;

__device__ __forceinline__ void rr_pair(int round, int i, int mp, int* p, int* q) {
  // circle method: player mp-1 fixed, the others rotate
  const int n1 = mp - 1;
  if (i == 0) { *p = round % n1; *q = n1; return; }
  *p = (round + i) % n1;
  *q = (round - i + n1) % n1;
}

template <typename T>
__device__ __forceinline__ T block_sum(T v, T* red) {
  for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffff, v, o);
  __syncthreads();
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  T s = 0;
  for (int i = 0; i < (int)(blockDim.x >> 5); ++i) s += red[i];
  return s;
}

template <typename T>
__global__ void __launch_bounds__(kJacobiThreads) jacobi_kernel(const double* __restrict__ Ag, double* w,
                                                               double* Vout, int m, T* scratch, int use_smem,
                                                               T eps) {
  extern __shared__ __align__(16) unsigned char smraw[];
  const int mp = m + (m & 1);
  const int npair = mp / 2;
  T* cs = (T*)smraw;                                   // 2 npair (c, s)
  int* pq = (int*)(cs + 2 * npair);                    // 2 npair
  T* red = (T*)(pq + 2 * npair);                       // 32 partial sums
  int* rank = (int*)(red + 32);                        // m (+1) ints
  T* A;
  T* V;
  if (use_smem == 2) {         // A and V in shared memory
    A = (T*)(rank + m + (m & 1));
    V = A + (size_t)m * m;
  } else if (use_smem == 1) {  // A in shared memory, V in a global scratch slice
    A = (T*)(rank + m + (m & 1));
    V = scratch + (size_t)blockIdx.x * m * m;
  } else {
    A = scratch + (size_t)blockIdx.x * 2 * m * m;
    V = A + (size_t)m * m;
  }
  const double* Ain = Ag + (size_t)blockIdx.x * m * m;
  for (int t = threadIdx.x; t < m * m; t += blockDim.x) {
    A[t] = (T)Ain[t];
    V[t] = ((t / m) == (t % m)) ? T(1) : T(0);
  }
  __syncthreads();
  T loc = 0;
  for (int t = threadIdx.x; t < m * m; t += blockDim.x) loc += A[t] * A[t];
  const T fro2 = block_sum(loc, red);
  const T tol2 = T(16) * eps * eps * fro2;
  T prev_off = fro2;
  if (m > 1 && fro2 > T(0)) {
    for (int sweep = 0; sweep < kJacobiMaxSweeps; ++sweep) {
      for (int round = 0; round < mp - 1; ++round) {
        for (int i = threadIdx.x; i < npair; i += blockDim.x) {
          int p, q;
          rr_pair(round, i, mp, &p, &q);
          if (p > q) { int t = p; p = q; q = t; }
          T c = 1, s = 0;
          if (q < m) {
            T apq = A[(size_t)p * m + q];
            T app = A[(size_t)p * m + p], aqq = A[(size_t)q * m + q];
            if (apq != T(0) && fabs(apq) > T(0.01) * eps * sqrt(fabs(app * aqq))) {
              T tau = (aqq - app) / (T(2) * apq);
              T t = (tau >= T(0) ? T(1) : T(-1)) / (fabs(tau) + sqrt(T(1) + tau * tau));
              c = T(1) / sqrt(T(1) + t * t);
              s = t * c;
            }
          } else {
            q = -1;
          }
          cs[2 * i] = c;
          cs[2 * i + 1] = s;
          pq[2 * i] = p;
          pq[2 * i + 1] = (s == T(0)) ? -1 : q;
        }
        __syncthreads();
        // rows: A <- J^T A
        for (int t = threadIdx.x; t < npair * m; t += blockDim.x) {
          int i = t / m, j = t - (t / m) * m;
          int q = pq[2 * i + 1];
          if (q < 0) continue;
          int p = pq[2 * i];
          T c = cs[2 * i], s = cs[2 * i + 1];
          T ap = A[(size_t)p * m + j], aq = A[(size_t)q * m + j];
          A[(size_t)p * m + j] = c * ap - s * aq;
          A[(size_t)q * m + j] = s * ap + c * aq;
        }
        __syncthreads();
        // columns: A <- A J, V <- V J
        for (int t = threadIdx.x; t < npair * m; t += blockDim.x) {
          int i = t / m, j = t - (t / m) * m;
          int q = pq[2 * i + 1];
          if (q < 0) continue;
          int p = pq[2 * i];
          T c = cs[2 * i], s = cs[2 * i + 1];
          T ap = A[(size_t)j * m + p], aq = A[(size_t)j * m + q];
          A[(size_t)j * m + p] = c * ap - s * aq;
          A[(size_t)j * m + q] = s * ap + c * aq;
          T vp = V[(size_t)j * m + p], vq = V[(size_t)j * m + q];
          V[(size_t)j * m + p] = c * vp - s * vq;
          V[(size_t)j * m + q] = s * vp + c * vq;
        }
        __syncthreads();
      }
      T off = 0;
      for (int t = threadIdx.x; t < m * m; t += blockDim.x) {
        int i = t / m, j = t - (t / m) * m;
        if (i != j) off += A[t] * A[t];
      }
      off = block_sum(off, red);
      // converged, or rounding has stopped the decrease (off-diagonal mass at the precision floor)
      if (off <= tol2 || (off > T(0.25) * prev_off && off <= T(4096) * eps * eps * fro2)) break;
      prev_off = off;
    }
  }
  // sort descending: rank[j] = position of eigenvalue j (ties by index)
  for (int j = threadIdx.x; j < m; j += blockDim.x) {
    T lj = A[(size_t)j * m + j];
    int pos = 0;
    for (int i = 0; i < m; ++i) {
      T li = A[(size_t)i * m + i];
      if (li > lj || (li == lj && i < j)) ++pos;
    }
    rank[j] = pos;
  }
  __syncthreads();
  double* wb = w + (size_t)blockIdx.x * m;
  double* Vb = Vout + (size_t)blockIdx.x * m * m;
  for (int j = threadIdx.x; j < m; j += blockDim.x) wb[rank[j]] = (double)A[(size_t)j * m + j];
  for (int t = threadIdx.x; t < m * m; t += blockDim.x) {
    int i = t / m, j = t - (t / m) * m;
    Vb[(size_t)i * m + rank[j]] = (double)V[t];
  }
}

template <typename T>
static void jacobi_launch(lrfg_ctx* ctx, const double* A, double* w, double* V, int m, int batch) {
  const int mp = m + (m & 1);
  const int npair = mp / 2;
  size_t head = sizeof(T) * 2 * npair + sizeof(int) * 2 * npair + sizeof(T) * 32 + sizeof(int) * (m + (m & 1));
  head = (head + 15) / 16 * 16;
  const size_t limit = (size_t)std::min(ctx->max_smem_optin, 220 * 1024);
  const size_t one = head + sizeof(T) * (size_t)m * m, two = one + sizeof(T) * (size_t)m * m;
  int use_smem = two <= limit ? 2 : (one <= limit ? 1 : 0);
  size_t smem = use_smem == 2 ? two : (use_smem == 1 ? one : head);
  DBuf<T> scratch;
  if (use_smem == 1) scratch = DBuf<T>(ctx->pool, (size_t)m * m * batch);
  if (use_smem == 0) scratch = DBuf<T>(ctx->pool, (size_t)2 * m * m * batch);
  LRFG_CUDA(raise_smem_limit((const void*)jacobi_kernel<T>, smem));
  const T eps = sizeof(T) == 4 ? (T)1.1920929e-07 : (T)2.220446049250313e-16;
  // one sweep of the two-sided cyclic Jacobi costs about 9 m^3 flops (rows, columns and V)
  LRFG_LAUNCH(ctx, KC_EIGEN, 9.0 * (double)m * m * m * batch, 3.0 * sizeof(double) * (double)m * m * batch,
              jacobi_kernel<T><<<batch, kJacobiThreads, smem, ctx->stream>>>(A, w, V, m, scratch.get(), use_smem,
                                                                              eps));
}

// Ogita–Aishima correction from G = X^T X and S = X^T A X (one block per matrix): writes lam and E.
__global__ void __launch_bounds__(512) oa_correction_kernel(const double* __restrict__ Ag, const double* __restrict__ Gg,
                                                            const double* __restrict__ Sg, double* lamg, double* Eg,
                                                            int m) {
  __shared__ double red[32];
  const size_t off = (size_t)blockIdx.x * m * m;
  const double* A = Ag + off;
  const double* G = Gg + off;
  const double* S = Sg + off;
  double* E = Eg + off;
  double* lam = lamg + (size_t)blockIdx.x * m;
  for (int i = threadIdx.x; i < m; i += blockDim.x) lam[i] = S[(size_t)i * m + i] / G[(size_t)i * m + i];
  __syncthreads();
  double a2 = 0.0, r2 = 0.0, s2 = 0.0;
  for (int t = threadIdx.x; t < m * m; t += blockDim.x) {
    int i = t / m, j = t - (t / m) * m;
    double r = (i == j ? 1.0 : 0.0) - G[t];
    double sd = (i == j) ? S[t] - lam[i] : S[t];
    a2 += A[t] * A[t];
    r2 += r * r;
    s2 += sd * sd;
  }
  a2 = block_sum(a2, red);
  r2 = block_sum(r2, red);
  s2 = block_sum(s2, red);
  const double delta = 2.0 * (sqrt(s2) + sqrt(a2) * sqrt(r2));
  for (int t = threadIdx.x; t < m * m; t += blockDim.x) {
    int i = t / m, j = t - (t / m) * m;
    double r = (i == j ? 1.0 : 0.0) - G[t];
    double e;
    if (i == j) {
      e = 0.5 * r;
    } else {
      double gap = lam[j] - lam[i];
      e = (fabs(gap) > delta) ? (S[t] + lam[j] * r) / gap : 0.5 * r;
    }
    E[t] = e;
  }
}

void syevj_mixed(lrfg_ctx* ctx, double* A, double* w, double* V, int m, int batch) {
  if (m <= 0 || batch <= 0) return;
  jacobi_launch<float>(ctx, A, w, V, m, batch);
  if (m == 1) return;
  const long long mm = (long long)m * m;
  DBuf<double> G(ctx->pool, mm * batch), AV(ctx->pool, mm * batch), S(ctx->pool, mm * batch),
      E(ctx->pool, mm * batch), Vn(ctx->pool, mm * batch);
  for (int it = 0; it < 3; ++it) {
    gemm(ctx, 1, 0, m, m, m, 1.0, V, m, mm, V, m, mm, 0.0, G.get(), m, mm, batch);
    gemm(ctx, 0, 0, m, m, m, 1.0, A, m, mm, V, m, mm, 0.0, AV.get(), m, mm, batch);
    gemm(ctx, 1, 0, m, m, m, 1.0, V, m, mm, AV.get(), m, mm, 0.0, S.get(), m, mm, batch);
    LRFG_LAUNCH(ctx, KC_EIGEN, 8.0 * (double)mm * batch, 4.0 * sizeof(double) * mm * batch,
                oa_correction_kernel<<<batch, 512, 0, ctx->stream>>>(A, G.get(), S.get(), w, E.get(), m));
    LRFG_CUDA(cudaMemcpyAsync(Vn.get(), V, sizeof(double) * mm * batch, cudaMemcpyDeviceToDevice, ctx->stream));
    gemm(ctx, 0, 0, m, m, m, 1.0, V, m, mm, E.get(), m, mm, 1.0, Vn.get(), m, mm, batch);
    LRFG_CUDA(cudaMemcpyAsync(V, Vn.get(), sizeof(double) * mm * batch, cudaMemcpyDeviceToDevice, ctx->stream));
  }
}

void syevj(lrfg_ctx* ctx, double* A, double* w, double* V, int m, int batch) {
  if (m <= 0 || batch <= 0) return;
  jacobi_launch<double>(ctx, A, w, V, m, batch);
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

__global__ void to_f32_kernel(const double* __restrict__ in, float* __restrict__ out, long long n) {
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x)
    out[t] = (float)in[t];
}

__global__ void to_f64_kernel(const float* __restrict__ in, double* __restrict__ out, long long n) {
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x)
    out[t] = (double)in[t];
}

void to_f32(lrfg_ctx* ctx, const double* in, float* out, long long n) {
  if (n <= 0) return;
  LRFG_LAUNCH(ctx, KC_TT_MISC, 0.0, 12.0 * n, to_f32_kernel<<<grid_for(ctx, n), 256, 0, ctx->stream>>>(in, out, n));
}

void to_f64(lrfg_ctx* ctx, const float* in, double* out, long long n) {
  if (n <= 0) return;
  LRFG_LAUNCH(ctx, KC_TT_MISC, 0.0, 12.0 * n, to_f64_kernel<<<grid_for(ctx, n), 256, 0, ctx->stream>>>(in, out, n));
}

}  // namespace lrfg
