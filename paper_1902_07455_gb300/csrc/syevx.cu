// FP64 symmetric eigensolver for the k largest eigenpairs (k = n: all of them) of a batch of matrices:
//  1. Householder tridiagonalisation  Q^T A Q = T  (Golub & Van Loan, "Matrix Computations", 4th ed.,
//     Alg. 8.3.1), reflectors kept in the columns below the diagonal;
//  2. eigenvalues of T by bisection on Sturm counts of the LDL^T recurrence (G&VL Sec. 8.4.1), one warp per
//     eigenvalue in a launch of its own;
//  3. eigenvectors of T by inverse iteration (G&VL Sec. 8.2.2) with the tridiagonal LU factorisation
//     of T - lambda I with partial pivoting (G&VL Sec. 4.3), three passes, vectors of eigenvalues closer
//     than 1e-3 ||T|| re-orthogonalised against each other by modified Gram-Schmidt after each pass;
//  4. back-transformation by the stored reflectors.
// About 4/3 n^3 + 2 k n^2 flops against ~9 n^3 per sweep (and several sweeps) for cyclic Jacobi, with the
// same absolute accuracy (eps ||A||), which is what the Gram-SVD truncation needs.
#include <algorithm>
#include <cfloat>
#include <cmath>

#include "ops.cuh"

namespace lrfg {

constexpr int kSyevxThreads = 512;

__device__ __forceinline__ double warp_sum(double v) {
  for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffff, v, o);
  return v;
}

// Block sum: warp partials, then warp 0 alone combines them (FP64 issue slots are scarce: 2 lanes/clk/SM)
// Sum over the block of v, where only threads < nact can hold nonzero values: only their warps shuffle
// (every FP64 add of an idle warp would still cost the SM's FP64 pipe 16 cycles).  Result in red[32].
__device__ double block_reduce_sum(double v, double* red, int nact) {
  const int nwa = min((int)(blockDim.x >> 5), (nact + 31) >> 5);
  const int warp = threadIdx.x >> 5;
  if (warp < nwa) v = warp_sum(v);
  __syncthreads();
  if ((threadIdx.x & 31) == 0 && warp < nwa) red[warp] = v;
  __syncthreads();
  if (threadIdx.x < 32) {
    double s = ((int)threadIdx.x < nwa) ? red[threadIdx.x] : 0.0;
    if (nwa > 1) s = warp_sum(s);
    if (threadIdx.x == 0) red[32] = s;
  }
  __syncthreads();
  return red[32];
}

// Number of eigenvalues of the symmetric tridiagonal (d, e) below x: sign changes of the Sturm sequence
// p_0 = 1, p_1 = d_0 - x, p_{i+1} = (d_i - x) p_i - e_{i-1}^2 p_{i-1} (Barth, Martin & Wilkinson, Numer. Math.
// 9 (1967) 386-393), a zero term taking the sign opposite to its predecessor.  Division-free (FP64
// division is a long dependent chain on this part); the pair (p_{i-1}, p_i) is rescaled by exact powers of
// two every four steps to stay in range.  The caller scales T by a power of two to |T| < 1, so that four
// steps change |p| by at most a factor 3^4 (growth) or 2^-212 (cancellation) within the 2^(+-600) window.
__device__ __forceinline__ int sign_of(double p, int sprev) {
  // sign from the bit pattern (integer pipe): +1, -1, or opposite of the predecessor for a zero
  const long long bits = __double_as_longlong(p);
  if ((bits & 0x7fffffffffffffffLL) == 0) return -sprev;
  return bits < 0 ? -1 : 1;
}

__device__ int sturm_count(const double* d, const double* e2, int n, double x) {
  const double up = 0x1p+600, down = 0x1p-600;
  double pm = 1.0, p = d[0] - x;
  int sprev = 1, c = 0;
  int s = sign_of(p, sprev);
  c += s != sprev;
  sprev = s;
  int i = 1;
  while (i < n) {
    const int iend = min(n, i + 4);
    for (; i < iend; ++i) {
      double pn = fma(d[i] - x, p, -e2[i - 1] * pm);
      pm = p;
      p = pn;
      s = sign_of(p, sprev);
      c += s != sprev;
      sprev = s;
    }
    const int ep = (int)((__double_as_longlong(p) >> 52) & 0x7ff), epm = (int)((__double_as_longlong(pm) >> 52) & 0x7ff);
    if (ep > 1023 + 600 || epm > 1023 + 600) { p *= down; pm *= down; }
    else if (ep < 1023 - 600 && epm < 1023 - 600) { p *= up; pm *= up; }
  }
  return c;
}

// The same count in FP32 (rescaling by 2^(+-60)), used only to localise eigenvalues before the FP64
// multisection; its brackets are verified with FP64 counts.
__device__ int sturm_count_f32(const float* d, const float* e2, int n, float x) {
  const float up = 0x1p+60f, down = 0x1p-60f;
  float pm = 1.0f, p = d[0] - x;
  int sprev = 1, c = 0;
  int s = (__float_as_int(p) & 0x7fffffff) == 0 ? -sprev : (__float_as_int(p) < 0 ? -1 : 1);
  c += s != sprev;
  sprev = s;
  for (int i = 1; i < n; ++i) {
    float pn = fmaf(d[i] - x, p, -e2[i - 1] * pm);
    pm = p;
    p = pn;
    const int ep = (__float_as_int(p) >> 23) & 0xff, epm = (__float_as_int(pm) >> 23) & 0xff;
    if (ep > 127 + 60) { p *= down; pm *= down; }
    else if (ep < 127 - 60 && epm < 127 - 60) { p *= up; pm *= up; }
    s = (__float_as_int(p) & 0x7fffffff) == 0 ? -sprev : (__float_as_int(p) < 0 ? -1 : 1);
    c += s != sprev;
    sprev = s;
  }
  return c;
}

// LU with partial pivoting of the tridiagonal T - lam I (sub = super = e, diag d - lam).  Factors in
// dl (multipliers), dd (reciprocals of the diagonal of U), du (1st super), du2 (2nd super), piv (1 = rows
// i, i+1 swapped).
__device__ void trid_factor(const double* d, const double* e, int n, double lam, double tiny, double* dl, double* dd,
                            double* du, double* du2, int* piv) {
  for (int i = 0; i < n; ++i) dd[i] = d[i] - lam;
  for (int i = 0; i < n - 1; ++i) {
    dl[i] = e[i];
    du[i] = e[i];
    du2[i] = 0.0;
    piv[i] = 0;
  }
  for (int i = 0; i < n - 1; ++i) {
    if (fabs(dd[i]) >= fabs(dl[i])) {
      if (dd[i] == 0.0) dd[i] = tiny;
      double f = dl[i] / dd[i];
      dl[i] = f;
      dd[i + 1] -= f * du[i];
    } else {
      double f = dd[i] / dl[i];
      dd[i] = dl[i];
      dl[i] = f;
      double t = du[i];
      du[i] = dd[i + 1];
      dd[i + 1] = t - f * dd[i + 1];
      if (i < n - 2) {
        du2[i] = du[i + 1];
        du[i + 1] = -f * du[i + 1];
      }
      piv[i] = 1;
    }
  }
  if (dd[n - 1] == 0.0) dd[n - 1] = tiny;
  for (int i = 0; i < n; ++i) dd[i] = 1.0 / dd[i];  // the solves multiply by the reciprocal pivots
}

__device__ void trid_solve(int n, const double* dl, const double* dd, const double* du, const double* du2,
                           const int* piv, double* b) {
  for (int i = 0; i < n - 1; ++i) {
    if (!piv[i]) {
      b[i + 1] -= dl[i] * b[i];
    } else {
      double t = b[i];
      b[i] = b[i + 1];
      b[i + 1] = t - dl[i] * b[i];
    }
  }
  // back substitution, rescaling the computed tail when a term would overflow (the direction is what
  // inverse iteration needs)
  const double big = 1e150;
  for (int i = n - 1; i >= 0; --i) {
    double v = b[i];
    if (i + 1 < n) v -= du[i] * b[i + 1];
    if (i + 2 < n) v -= du2[i] * b[i + 2];
    double y = v * dd[i];
    if (fabs(y) > big) {
      for (int l = i + 1; l < n; ++l) b[l] *= 1e-150;
      y *= 1e-150;
    }
    b[i] = y;
  }
}

// Gershgorin interval of the tridiagonal (d, e) and the largest e_i^2, by warp 0 (lanes over the rows), left in
// red[35] (lower end), red[36] (upper end), red[37]; e2 <- e^2 (e2[n-1] = 0).  All threads of the block call it.
__device__ void trid_gershgorin(const double* d, const double* e, double* e2, int n, double* red) {
  const int tid = threadIdx.x, nthr = blockDim.x;
  if (tid < 32) {
    double l0 = INFINITY, h0 = -INFINITY, em = 0.0;
    for (int i = tid; i < n; i += 32) {
      const double r = (i > 0 ? fabs(e[i - 1]) : 0.0) + (i < n - 1 ? fabs(e[i]) : 0.0);
      l0 = fmin(l0, d[i] - r);
      h0 = fmax(h0, d[i] + r);
      if (i < n - 1) em = fmax(em, e[i] * e[i]);
    }
    for (int o = 16; o; o >>= 1) {
      l0 = fmin(l0, __shfl_xor_sync(0xffffffff, l0, o));
      h0 = fmax(h0, __shfl_xor_sync(0xffffffff, h0, o));
      em = fmax(em, __shfl_xor_sync(0xffffffff, em, o));
    }
    if (tid == 0) {
      red[35] = l0;
      red[36] = h0;
      red[37] = em;
    }
  }
  __syncthreads();
  for (int i = tid; i < n; i += nthr) e2[i] = (i < n - 1) ? e[i] * e[i] : 0.0;
  __syncthreads();
}

// ---- the decomposition in three launches -----------------------------------------------------------------
// K1 (one block per matrix) tridiagonalises and bounds the spectrum; K2 (one warp per wanted eigenvalue, all
// matrices) bisects; K3 (one block per matrix) runs inverse iteration, re-orthogonalises within clusters,
// back-transforms and writes the outputs.  The bisection is a chain of dependent FP64 Sturm recurrences per
// point; inside one block the k eigenvalues shared one SM's FP64 pipe (2 FMA/clk), one warp each they get one
// SM each, so every lane can take its own point (33-way multisection, about 5 bits per count instead of 2).
// Per-item global scratch (doubles): a header (active size, Gershgorin interval, largest e_i^2, reduced-problem
// flag and nA), d, e, beta (nl each), lam (kl), the reflectors W (n x n, leading dimension n), the vectors Y
// (kl x nl, vector-major) and the inverse-iteration LU factors (kl x 5 nl).
constexpr int kHdr = 8;

static size_t syevx_scratch_per(int nl, int kl) {
  return kHdr + 3 * (size_t)nl + kl + (size_t)nl * nl + (size_t)kl * nl + (size_t)kl * 5 * nl;
}

struct SyevxScratch {
  double *hdr, *d, *e, *beta, *lam, *W, *Y, *lu;
};

__device__ __forceinline__ SyevxScratch syevx_scratch(double* scratch, int nl, int kl, int item) {
  SyevxScratch g;
  g.hdr = scratch + (size_t)item * (kHdr + 3 * (size_t)nl + kl + (size_t)nl * nl + (size_t)kl * nl +
                                    (size_t)kl * 5 * nl);
  g.d = g.hdr + kHdr;
  g.e = g.d + nl;
  g.beta = g.e + nl;
  g.lam = g.beta + nl;
  g.W = g.lam + kl;
  g.Y = g.W + (size_t)nl * nl;
  g.lu = g.Y + (size_t)kl * nl;
  return g;
}

// K1.  nl, kl: the launch sizes (strides of the inputs and outputs).  Optional reduced problem (nAg != null):
// the symmetric input A = B B^T has its nonzero block in the leading nA x nA corner, and A2 = B^T B (B: nl x nl,
// nonzero block nA x nB) has it in the leading nB x nB corner.  The smaller of the two is decomposed; when that
// is A2, K3 maps the left vectors back as u = B w / sigma, re-orthonormalises them (modified Gram-Schmidt) and
// completes them by unit vectors when B has fewer than k nonzero singular values.
__global__ void __launch_bounds__(kSyevxThreads) syevx_tri_kernel(const double* __restrict__ Ag, int nl, int kl,
                                                                  double* wg, double* Vg, int ldv, double* scratch,
                                                                  int use_smem, const int* __restrict__ nAg,
                                                                  const int* __restrict__ nBg,
                                                                  const double* __restrict__ A2g,
                                                                  const double* __restrict__ Bg, double* work) {
  extern __shared__ __align__(16) double sm[];
  double* red = sm;            // 33 (32 partials + the result) + padding
  double* d = red + 40;        // nl
  double* e = d + nl;          // nl
  double* beta = e + nl;       // nl
  double* pv = beta + nl;      // nl: p / w of the current reflector
  double* vv = pv + nl;        // nl: current reflector v
  double* e2 = vv + nl;        // nl
  const size_t nnl = (size_t)nl * nl;
  const SyevxScratch g = syevx_scratch(scratch, nl, kl, blockIdx.x);
  double* W = use_smem ? (e2 + nl) : g.W;
  const int tid = threadIdx.x, nthr = blockDim.x;
  double* wout = wg + (size_t)blockIdx.x * nl;
  double* Vout = Vg + (size_t)blockIdx.x * (size_t)nl * ldv;
  // the problem actually decomposed: n x n, k vectors
  const int nA = nAg ? max(0, min(nl, nAg[blockIdx.x])) : nl;
  const int nB = nBg ? max(0, min(nl, nBg[blockIdx.x])) : nl;
  const bool viaB = (nAg != nullptr) && (A2g != nullptr) && (Bg != nullptr) && nB < nA;
  const int n = viaB ? nB : nA;
  const int k = min(kl, n);
  const double* A = (viaB ? A2g : Ag) + (size_t)blockIdx.x * nnl;
  if (tid == 0) {
    add_work(work, 4.0 / 3.0 * n * (double)n * n + 4.0 * (double)k * n * n + 60.0 * k * n,
             sizeof(double) * (2.0 * n * n + (double)k * n));
    g.hdr[0] = (double)n;
    g.hdr[4] = viaB ? 1.0 : 0.0;
    g.hdr[5] = (double)nA;
  }
  for (int t = tid; t < kl; t += nthr) wout[t] = 0.0;
  for (size_t q = tid; q < (size_t)nl * kl; q += nthr) {
    const int i = (int)(q / kl), t = (int)(q - (q / kl) * kl);
    Vout[(size_t)i * ldv + t] = 0.0;
  }
  if (n == 0) return;
  for (size_t t = tid; t < (size_t)n * n; t += nthr) {
    const int i = (int)(t / n), j = (int)(t - (t / n) * n);
    W[t] = A[(size_t)i * nl + j];
  }
  __syncthreads();

  // 1. tridiagonalisation
  for (int j = 0; j + 2 < n; ++j) {
    const int m = n - j - 1;
    double x0 = W[(size_t)(j + 1) * n + j];
    double loc = 0.0;
    for (int i = tid; i < m; i += nthr) {
      double xi = W[(size_t)(j + 1 + i) * n + j];
      vv[i] = xi;
      if (i > 0) loc += xi * xi;
    }
    const double tail2 = block_reduce_sum(loc, red, m);
    if (tail2 == 0.0) {
      if (tid == 0) {
        d[j] = W[(size_t)j * n + j];
        e[j] = x0;
        beta[j] = 0.0;
      }
      __syncthreads();
      continue;
    }
    // the reflector's scalars once (a square root and a division are long FP64 sequences: computed by
    // every thread they would occupy the FP64 pipe for thousands of cycles)
    if (tid == 0) {
      const double alpha = -copysign(sqrt(x0 * x0 + tail2), x0);
      const double v0 = x0 - alpha;
      const double bb = 2.0 / (tail2 + v0 * v0);
      vv[0] = v0;
      d[j] = W[(size_t)j * n + j];
      e[j] = alpha;
      beta[j] = bb;
      red[34] = bb;
    }
    __syncthreads();
    const double b = red[34];
    // keep v in column j below the diagonal for the back-transformation
    for (int i = tid; i < m; i += nthr) W[(size_t)(j + 1 + i) * n + j] = vv[i];
    // p = b A22 v: thread i takes row i, reading column i of the symmetric trailing block so that
    // neighbouring threads read neighbouring words (no warp reductions, which cost FP64 issue slots)
    for (int i = tid; i < m; i += nthr) {
      const double* col = W + (size_t)(j + 1) * n + (j + 1 + i);
      // four independent accumulators: an FP64 FMA has a 64-cycle latency on this part
      double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
      int l = 0;
      for (; l + 3 < m; l += 4) {
        s0 = fma(col[(size_t)l * n], vv[l], s0);
        s1 = fma(col[(size_t)(l + 1) * n], vv[l + 1], s1);
        s2 = fma(col[(size_t)(l + 2) * n], vv[l + 2], s2);
        s3 = fma(col[(size_t)(l + 3) * n], vv[l + 3], s3);
      }
      for (; l < m; ++l) s0 = fma(col[(size_t)l * n], vv[l], s0);
      pv[i] = b * ((s0 + s1) + (s2 + s3));
    }
    const int warp = tid >> 5, lane = tid & 31, nw = nthr >> 5;
    __syncthreads();
    double kl = 0.0;
    for (int i = tid; i < m; i += nthr) kl += vv[i] * pv[i];
    const double K = 0.5 * b * block_reduce_sum(kl, red, m);
    for (int i = tid; i < m; i += nthr) pv[i] -= K * vv[i];
    __syncthreads();
    // A22 -= v w^T + w v^T (one warp per row)
    for (int i = warp; i < m; i += nw) {
      double* row = W + (size_t)(j + 1 + i) * n + (j + 1);
      const double vi = vv[i], wi = pv[i];
      for (int l = lane; l < m; l += 32) row[l] -= vi * pv[l] + wi * vv[l];
    }
    __syncthreads();
  }
  if (tid == 0) {
    if (n >= 2) {
      d[n - 2] = W[(size_t)(n - 2) * n + (n - 2)];
      e[n - 2] = W[(size_t)(n - 1) * n + (n - 2)];
      if (n >= 3) beta[n - 2] = 0.0;
    }
    d[n - 1] = W[(size_t)(n - 1) * n + (n - 1)];
    e[n - 1] = 0.0;
    beta[n - 1] = 0.0;
  }
  __syncthreads();

  trid_gershgorin(d, e, e2, n, red);
  if (tid == 0) {
    g.hdr[1] = red[35];
    g.hdr[2] = red[36];
    g.hdr[3] = red[37];
  }
  for (int i = tid; i < n; i += nthr) {
    g.d[i] = d[i];
    g.e[i] = e[i];
    g.beta[i] = beta[i];
  }
  if (use_smem)
    for (size_t t = tid; t < (size_t)n * n; t += nthr) g.W[t] = W[t];
}

// K2.  Eigenvalue t (the t-th largest) of the tridiagonal of item blockIdx.y, one warp: (a) FP32 localisation
// in the Gershgorin interval by five rounds of 33-way multisection (about 25 bits); (b) that bracket, widened
// and verified with FP64 counts (else the Gershgorin interval), then 33-way FP64 multisection on a copy of T
// scaled by a power of two to |T| in [0.5, 1) (the counts' range window) down to the absolute resolution
// eps ||T||: the eigenvalues of an FP64 Gram core carry errors of that size, and inverse iteration only needs
// the shift to that accuracy.
__global__ void __launch_bounds__(32) syevx_bisect_kernel(int nl, int kl, double* scratch) {
  extern __shared__ __align__(16) double sm[];
  const SyevxScratch g = syevx_scratch(scratch, nl, kl, blockIdx.y);
  const int n = (int)g.hdr[0];
  const int t = blockIdx.x, lane = threadIdx.x;
  if (t >= min(kl, n)) return;
  const double lo = g.hdr[1], hi = g.hdr[2], emax2 = g.hdr[3];
  const double tnorm = fmax(fabs(lo), fabs(hi));
  if (tnorm == 0.0) {
    if (lane == 0) g.lam[t] = 0.0;
    return;
  }
  float* df = (float*)sm;   // n floats
  float* e2f = df + n;      // n floats
  double* ds = sm + n;      // n: the scaled diagonal
  double* e2s = ds + n;     // n: the scaled e^2
  int texp = 0;
  frexp(tnorm, &texp);
  const double sg = ldexp(1.0, -texp), sg2 = sg * sg;
  for (int i = lane; i < n; i += 32) {
    const double ei = (i < n - 1) ? g.e[i] : 0.0;
    const double di = g.d[i];
    df[i] = (float)di;
    e2f[i] = (float)(ei * ei);
    ds[i] = di * sg;
    e2s[i] = (ei * ei) * sg2;
  }
  __syncwarp();
  const int idx = n - 1 - t;
  const double pivmin = DBL_MIN * fmax(1.0, emax2);
  const double glo = lo - 2.0 * DBL_EPSILON * tnorm - pivmin, ghi = hi + 2.0 * DBL_EPSILON * tnorm + pivmin;
  float af = (float)glo, cf = (float)ghi;
  for (int it = 0; it < 5; ++it) {
    const float h = (cf - af) * (1.0f / 33.0f);
    const float x = af + h * (float)(lane + 1);
    const unsigned above = __ballot_sync(0xffffffff, sturm_count_f32(df, e2f, n, x) > idx);
    const int f = above ? (__ffs(above) - 1) : 32;
    const float na = (f == 0) ? af : af + h * (float)f;
    const float nc = (f == 32) ? cf : af + h * (float)(f + 1);
    if (!(na < nc)) break;  // FP32 resolution reached
    af = na;
    cf = nc;
  }
  const double wf = (double)cf - (double)af;
  double a = fmax(glo, (double)af - 4.0 * wf - 1e-6 * tnorm) * sg;
  double c = fmin(ghi, (double)cf + 4.0 * wf + 1e-6 * tnorm) * sg;
  int ca = (lane == 0) ? sturm_count(ds, e2s, n, a) : 0;
  int cc = (lane == 1) ? sturm_count(ds, e2s, n, c) : 0;
  ca = __shfl_sync(0xffffffff, ca, 0);
  cc = __shfl_sync(0xffffffff, cc, 1);
  if (!(ca <= idx && cc > idx)) {
    a = glo * sg;
    c = ghi * sg;
  }
  const double floor_s = (DBL_EPSILON * tnorm + 4.0 * pivmin) * sg;
  for (int it = 0; it < 40; ++it) {
    if (c - a <= 2.0 * DBL_EPSILON * fmax(fabs(a), fabs(c)) + floor_s) break;
    const double h = (c - a) * (1.0 / 33.0);
    const double x = a + h * (double)(lane + 1);
    const unsigned above = __ballot_sync(0xffffffff, sturm_count(ds, e2s, n, x) > idx);
    // the first point whose count exceeds idx bounds the eigenvalue from above
    const int f = above ? (__ffs(above) - 1) : 32;
    const double na = (f == 0) ? a : a + h * (double)f;
    const double nc = (f == 32) ? c : a + h * (double)(f + 1);
    if (!(na < nc)) break;
    a = na;
    c = nc;
  }
  if (lane == 0) g.lam[t] = 0.5 * (a + c) / sg;
}

// K3.  Eigenvectors of T by inverse iteration (three passes; vectors of eigenvalues closer than 1e-3 ||T||
// re-orthogonalised after each pass), the back-transformation and the outputs.
__global__ void __launch_bounds__(kSyevxThreads) syevx_vec_kernel(int nl, int kl, double* wg, double* Vg, int ldv,
                                                                  double* scratch, int smem_flags,
                                                                  const double* __restrict__ Bg) {
  extern __shared__ __align__(16) double sm[];
  const SyevxScratch g = syevx_scratch(scratch, nl, kl, blockIdx.x);
  const int n = (int)g.hdr[0];
  if (n == 0) return;
  double* red = sm;            // 40
  double* d = red + 40;        // nl
  double* e = d + nl;          // nl
  double* beta = e + nl;       // nl
  double* lam = beta + nl;     // kl
  // the vectors, their LU factors and the reflectors in shared memory where they fit (flags 1, 2, 4): the
  // solves, the re-orthogonalisation and the back-transformation are dependent chains of their loads
  // strides in shared memory are odd numbers of doubles, so that the lanes of a warp walking different vectors
  // (inverse iteration: one lane per vector) or different rows (the warp sums) hit different banks
  const int npad = nl | 1;
  double* next = lam + kl;
  double* Y = g.Y;
  double* lu = g.lu;
  double* W = g.W;
  if (smem_flags & 1) { Y = next; next += (size_t)kl * npad; }
  if (smem_flags & 2) { lu = next; next += (size_t)kl * 5 * npad; }
  if (smem_flags & 4) W = next;
  const size_t nnl = (size_t)nl * nl;
  const bool viaB = g.hdr[4] != 0.0;
  const int nA = (int)g.hdr[5];
  const int k = min(kl, n);
  const int tid = threadIdx.x, nthr = blockDim.x;
  const int warp = tid >> 5, lane = tid & 31, nw = nthr >> 5;
  const int yst = (smem_flags & 1) ? npad : n;       // between vectors of Y
  const int fst = (smem_flags & 2) ? npad : n;       // between the fields of one vector's LU factors
  const int wld = (smem_flags & 4) ? npad : n;       // leading dimension of the reflectors
  double* wout = wg + (size_t)blockIdx.x * nl;
  double* Vout = Vg + (size_t)blockIdx.x * (size_t)nl * ldv;
  for (int i = tid; i < n; i += nthr) {
    d[i] = g.d[i];
    e[i] = g.e[i];
    beta[i] = g.beta[i];
  }
  for (int t = tid; t < k; t += nthr) lam[t] = g.lam[t];
  if (smem_flags & 4)
    for (size_t t = tid; t < (size_t)n * n; t += nthr) W[(t / n) * wld + t % n] = g.W[t];
  __syncthreads();
  const double tnorm = fmax(fabs(g.hdr[1]), fabs(g.hdr[2]));
  if (tnorm == 0.0) {
    // the zero matrix: eigenvalues 0, eigenvectors the unit vectors
    for (size_t q = tid; q < (size_t)k * n; q += nthr) {
      const int t = (int)(q / n), i = (int)(q - (q / n) * n);
      Y[(size_t)t * yst + i] = (i == t) ? 1.0 : 0.0;
    }
  } else {
  // separate exactly equal eigenvalues slightly so that their factorisations differ
  if (tid == 0) {
    const double sep = 10.0 * DBL_EPSILON * tnorm;
    for (int t = 1; t < k; ++t)
      if (lam[t - 1] - lam[t] < sep) lam[t] = lam[t - 1] - sep;
  }
  __syncthreads();

  // 3. inverse iteration, three passes with cluster re-orthogonalisation
  const double tiny = DBL_EPSILON * fmax(tnorm, DBL_MIN);
  for (int t = tid; t < k; t += nthr) {
    double* y = Y + (size_t)t * yst;
    // deterministic start vector with entries in [0.5, 1.5)
    unsigned h = 2166136261u ^ (unsigned)(t * 2654435761u);
    for (int i = 0; i < n; ++i) {
      h = h * 1664525u + 1013904223u;
      y[i] = 0.5 + (double)(h >> 8) * (1.0 / 16777216.0);
    }
    double* f = lu + (size_t)t * 5 * fst;
    trid_factor(d, e, n, lam[t], tiny, f, f + fst, f + 2 * fst, f + 3 * fst, (int*)(f + 4 * fst));
  }
  __syncthreads();
  const double ortol = 1e-3 * tnorm;
  for (int pass = 0; pass < 3; ++pass) {
    for (int t = tid; t < k; t += nthr) {
      double* y = Y + (size_t)t * yst;
      const double* f = lu + (size_t)t * 5 * fst;
      trid_solve(n, f, f + fst, f + 2 * fst, f + 3 * fst, (const int*)(f + 4 * fst), y);
      double s = 0.0;
      for (int i = 0; i < n; ++i) s += y[i] * y[i];
      if (s > 0.0 && isfinite(s)) {
        s = 1.0 / sqrt(s);
        for (int i = 0; i < n; ++i) y[i] *= s;
      } else {
        // a breakdown (all-zero or overflowed solve): restart from a unit vector, the
        // re-orthogonalisation and the next pass recover the direction
        for (int i = 0; i < n; ++i) y[i] = (i == (t * 7 + pass) % n) ? 1.0 : 0.0;
      }
    }
    __syncthreads();
    // modified Gram-Schmidt within clusters, by warp 0, in descending order of the eigenvalues (one warp and no
    // block barrier: the pairs are a dependent chain, and barriers between them cost more than the warp's sums)
    if (tid < 32) {
      for (int t = 1; t < k; ++t) {
        double* yt = Y + (size_t)t * yst;
        bool touched = false;
        for (int s2 = t - 1; s2 >= 0 && lam[s2] - lam[t] <= ortol; --s2) {
          const double* ys = Y + (size_t)s2 * yst;
          double dp = 0.0;
          for (int i = tid; i < n; i += 32) dp += ys[i] * yt[i];
          dp = warp_sum(dp);
          for (int i = tid; i < n; i += 32) yt[i] -= dp * ys[i];
          touched = true;
        }
        if (touched) {
          double q2 = 0.0;
          for (int i = tid; i < n; i += 32) q2 += yt[i] * yt[i];
          q2 = warp_sum(q2);
          const double sc = q2 > 0.0 ? 1.0 / sqrt(q2) : 0.0;
          for (int i = tid; i < n; i += 32) yt[i] *= sc;
        }
        __syncwarp();
      }
    }
    __syncthreads();
  }

  // 4. back-transformation x = H_0 H_1 ... H_{n-3} y (one warp per vector; the reflectors are read-only)
  for (int t = warp; t < k; t += nw) {
    double* yv = Y + (size_t)t * yst;
    for (int j = n - 3; j >= 0; --j) {
      const double b = beta[j];
      if (b == 0.0) continue;
      const int m = n - j - 1;
      double* y = yv + (j + 1);
      double s = 0.0;
      for (int i = lane; i < m; i += 32) s += W[(size_t)(j + 1 + i) * wld + j] * y[i];
      s = b * warp_sum(s);
      for (int i = lane; i < m; i += 32) y[i] -= s * W[(size_t)(j + 1 + i) * wld + j];
      __syncwarp();
    }
  }
  __syncthreads();

  }  // tnorm != 0
  __syncthreads();

  // outputs: eigenvalues descending, eigenvectors as the first k columns of V (leading dimension ldv)
  for (int t = tid; t < k; t += nthr) wout[t] = lam[t];
  if (!viaB) {
    for (size_t q = tid; q < (size_t)k * n; q += nthr) {
      int t = (int)(q / n), i = (int)(q - (q / n) * n);
      Vout[(size_t)i * ldv + t] = Y[(size_t)t * yst + i];
    }
    return;
  }
  // left vectors u_t = B w_t / sigma_t (length nA, vector-major in lu, which inverse iteration no longer
  // needs), then modified Gram-Schmidt (twice) in descending order, completed by unit vectors where
  // sigma_t vanishes or B has fewer than kl singular values; at most min(kl, nA) columns
  double* U = lu;
  const double* B = Bg + (size_t)blockIdx.x * nnl;
  for (size_t q = tid; q < (size_t)k * nA; q += nthr) {
    const int t = (int)(q / nA), i = (int)(q - (q / nA) * nA);
    const double sg = lam[t] > 0.0 ? sqrt(lam[t]) : 0.0;
    double acc = 0.0;
    for (int l = 0; l < n; ++l) acc = fma(B[(size_t)i * nl + l], Y[(size_t)t * yst + l], acc);
    U[q] = sg > 0.0 ? acc / sg : 0.0;
  }
  __syncthreads();
  const int kout = min(kl, nA);
  if (tid < 32) {
    int next_unit = 0;
    for (int t = 0; t < kout; ++t) {
      double* ut = U + (size_t)t * nA;
      if (t >= k) {
        for (int i = tid; i < nA; i += 32) ut[i] = 0.0;
      }
      for (int attempt = 0; attempt <= nA; ++attempt) {
        double n0 = 0.0;
        for (int i = tid; i < nA; i += 32) n0 += ut[i] * ut[i];
        n0 = warp_sum(n0);
        for (int pass = 0; pass < 2; ++pass)
          for (int s2 = 0; s2 < t; ++s2) {
            const double* us = U + (size_t)s2 * nA;
            double dp = 0.0;
            for (int i = tid; i < nA; i += 32) dp += us[i] * ut[i];
            dp = warp_sum(dp);
            for (int i = tid; i < nA; i += 32) ut[i] -= dp * us[i];
          }
        double n1 = 0.0;
        for (int i = tid; i < nA; i += 32) n1 += ut[i] * ut[i];
        n1 = warp_sum(n1);
        if (n0 > 0.0 && n1 > 0.25 * n0) {
          const double sc = 1.0 / sqrt(n1);
          for (int i = tid; i < nA; i += 32) ut[i] *= sc;
          break;
        }
        // no usable direction: restart from the next unit vector
        const int uidx = next_unit++ % nA;
        for (int i = tid; i < nA; i += 32) ut[i] = (i == uidx) ? 1.0 : 0.0;
        __syncwarp();
      }
      __syncwarp();
    }
  }
  __syncthreads();
  for (size_t q = tid; q < (size_t)kout * nA; q += nthr) {
    const int t = (int)(q / nA), i = (int)(q - (q / nA) * nA);
    Vout[(size_t)i * ldv + t] = U[q];
  }
}


static void syevx_launch(lrfg_ctx* ctx, const double* A, double* w, double* V, int n, int k, int batch,
                         const int* nA, const int* nB, const double* A2, const double* B) {
  if (n <= 0 || batch <= 0 || k <= 0) return;
  k = std::min(k, n);
  LRFG_REQUIRE(k < 65536 && batch < 65536, "eigensolver grid too large (k = %d, batch = %d)", k, batch);
  DBuf<double> scratch(ctx->pool, syevx_scratch_per(n, k) * batch);
  const size_t lim = (size_t)std::min(ctx->max_smem_optin, 200 * 1024);
  const size_t wbytes = sizeof(double) * (size_t)n * n;
  // K1: the reflectors in shared memory when they fit
  const size_t head1 = sizeof(double) * (40 + 6 * (size_t)n);
  const int smem_w1 = head1 + wbytes <= lim ? 1 : 0;
  const size_t smem1 = head1 + (smem_w1 ? wbytes : 0);
  LRFG_CUDA(raise_smem_limit((const void*)syevx_tri_kernel, smem1));
  // algorithmic work at the active size, counted by each block on the device
  LRFG_LAUNCH(ctx, KC_EIGEN, 0.0, 0.0,
              syevx_tri_kernel<<<batch, kSyevxThreads, smem1, ctx->stream>>>(A, n, k, w, V, n, scratch.get(),
                                                                             smem_w1, nA, nB, A2, B,
                                                                             work_counter(ctx, KC_EIGEN)));
  // K2: one warp per wanted eigenvalue of every item
  const size_t smem2 = sizeof(double) * 3 * (size_t)n;
  LRFG_CUDA(raise_smem_limit((const void*)syevx_bisect_kernel, smem2));
  LRFG_LAUNCH(ctx, KC_EIGEN, 0.0, 0.0,
              syevx_bisect_kernel<<<dim3((unsigned)k, (unsigned)batch), 32, smem2, ctx->stream>>>(n, k,
                                                                                                scratch.get()));
  // K3: the vectors, then their LU factors, then the reflectors in shared memory while they fit
  size_t smem3 = sizeof(double) * (40 + 3 * (size_t)n + (size_t)k);
  int flags3 = 0;
  const size_t npad = (size_t)(n | 1);  // K3's odd shared-memory strides
  const size_t parts[3] = {sizeof(double) * (size_t)k * npad, sizeof(double) * (size_t)k * 5 * npad,
                           sizeof(double) * (size_t)n * npad};
  for (int q = 0; q < 3; ++q)
    if (smem3 + parts[q] <= lim) {
      smem3 += parts[q];
      flags3 |= 1 << q;
    }
  LRFG_CUDA(raise_smem_limit((const void*)syevx_vec_kernel, smem3));
  LRFG_LAUNCH(ctx, KC_EIGEN, 0.0, 0.0,
              syevx_vec_kernel<<<batch, kSyevxThreads, smem3, ctx->stream>>>(n, k, w, V, n, scratch.get(), flags3,
                                                                             B));
}

void syevx(lrfg_ctx* ctx, const double* A, double* w, double* V, int n, int k, int batch) {
  syevx_launch(ctx, A, w, V, n, k, batch, nullptr, nullptr, nullptr, nullptr);
}

void syevx_sized(lrfg_ctx* ctx, const double* A, const int* n_eff, double* w, double* V, int n, int k, int batch) {
  syevx_launch(ctx, A, w, V, n, k, batch, n_eff, nullptr, nullptr, nullptr);
}

void syevx_product(lrfg_ctx* ctx, const double* BBt, const double* BtB, const double* B, const int* nA,
                   const int* nB, double* w, double* V, int n, int k, int batch) {
  syevx_launch(ctx, BBt, w, V, n, k, batch, nA, nB, BtB, B);
}

}  // namespace lrfg

namespace lrfg {

// ------------------------------------------------------------------------------------------------
// Factor of a (balanced) Gram matrix for the Gram-SVD: pivoted Cholesky P^T G P = L L^T (Golub & Van
// Loan Sec. 4.2, diagonal pivoting for semidefinite matrices), stopped when the largest remaining
// pivot falls below tau = 1e-16 times the largest initial diagonal (numerical rank rho).  The entries
// of an FP64 Gram matrix carry absolute errors of about eps64 times its largest diagonal, so smaller
// pivots are rounding noise: keeping them makes the basis M L^{-T} lose orthogonality in those
// directions (error ~ eps / sqrt(pivot)), dropping more loses their content (~ sqrt(pivot)).  The two
// balance near tau = eps64; an emulation of the truncations of the rank-10 solve at 243^3 (Hadamard
// products with the coefficient, exponential-sum outputs) gives relative errors against the SVD
// truncation of 4e-10..3e-9 at 1e-16, against 1.4e-8..1e-7 at 1e-20 and 7e-9..1.4e-8 at 1e-14.
// Outputs, for the orthonormal basis Q = M C P L11^{-T} of the left part M (C the balancing scaling):
//   RA  (b x b): rows i < rho hold L^T P^T (so G = RA^T RA up to the dropped Schur complement),
//   RAc (b x b): RA with column j divided by c_j (undoes the balancing in the transfer matrix),
//   Pc  (b x b): Pc[perm[l]][q] = c[perm[l]] (L11^{-1})[q][l] for l, q < rho (so Q = M Pc).
// One block per matrix; the working matrices are in shared memory when they fit.
// ------------------------------------------------------------------------------------------------
constexpr int kCholThreads = 512;

// shared-memory layout of gram_factor_kernel: bytes of the header before the two b x b work matrices
__host__ __device__ inline size_t chol_head_bytes(int b) {
  size_t bytes = sizeof(double) * (32 + 2 * (size_t)b) + sizeof(int) * (32 + 3 * (size_t)b + 2);
  return (bytes + 255) / 256 * 256;
}

// Left-looking form (Golub & Van Loan Sec. 4.2.8 ordering with diagonal pivoting): pivot k takes the
// largest remaining diagonal of the Schur complement, kept as a vector, and only column k of L is formed,
// L[i][k] = (G[i][p] - sum_{l<k} L[i][l] L[p][l]) / L[p][k], for the rows not yet pivots; b rho^2 / 2
// multiply-adds up to the numerical rank instead of the b^2 rho of updating the whole trailing block.
// Column k of L is stored over column p = perm[k] of the working copy of G (that column is read only at
// this step), so L[j][l] sits at W[j][perm[l]].  The search for the next pivot runs in the same phase as
// the column (each warp over the rows it has just updated), so a pivot costs two barriers.
__global__ void __launch_bounds__(kCholThreads) gram_factor_kernel(const double* __restrict__ Gg,
                                                                   const double* __restrict__ cg, int b, double tau,
                                                                   double* RAg, double* RAcg, double* Pcg,
                                                                   int* rhog, double* scratch, int use_smem,
                                                                   double* work) {
  extern __shared__ __align__(16) double sm[];
  double* redv = sm;                   // 32 values
  double* dv = redv + 32;              // b: remaining diagonal of the Schur complement
  double* rd = dv + b;                 // b: reciprocals of the diagonal of L11
  int* redi = (int*)(rd + b);          // 32 indices
  int* perm = redi + 32;               // b: perm[k] = row of pivot k
  int* done = perm + b;                // b: 1 once a row is a pivot
  int* pos = done + b;                 // b: pivot position of a row
  int* flag = pos + b;                 // 2: rho, pivot
  const size_t bb = (size_t)b * b;
  double* W = use_smem ? (double*)((unsigned char*)sm + chol_head_bytes(b)) : scratch + (size_t)blockIdx.x * 2 * bb;
  double* Li = W + bb;                 // L11^{-1}
  const double* G = Gg + (size_t)blockIdx.x * bb;
  const double* c = cg ? cg + (size_t)blockIdx.x * b : nullptr;
  double* RA = RAg + (size_t)blockIdx.x * bb;
  double* RAc = RAcg ? RAcg + (size_t)blockIdx.x * bb : nullptr;
  double* Pc = Pcg ? Pcg + (size_t)blockIdx.x * bb : nullptr;
  const int tid = threadIdx.x, nthr = blockDim.x, lane = tid & 31, warp = tid >> 5, nw = nthr >> 5;
  for (size_t t = tid; t < bb; t += nthr) W[t] = G[t];
  double md = 0.0;
  for (int i = tid; i < b; i += nthr) {
    const double gi = G[(size_t)i * b + i];
    dv[i] = gi;
    done[i] = 0;
    pos[i] = b;
    perm[i] = i;
    md = fmax(md, gi);
  }
  for (int o = 16; o; o >>= 1) md = fmax(md, __shfl_xor_sync(0xffffffff, md, o));
  if (lane == 0) redv[warp] = md;
  __syncthreads();
  if (tid == 0) {
    double m = 0.0;
    for (int i = 0; i < nw; ++i) m = fmax(m, redv[i]);
    redv[31] = m;
    flag[0] = b;
  }
  __syncthreads();
  const double maxd0 = redv[31];
  const int nwa = min(nw, (b + 31) >> 5);  // warps that hold rows
  // per-warp candidates for the next pivot (largest remaining diagonal; ties: smallest row) from the rows
  // this thread holds, after its own updates (two barriers per pivot)
  auto warp_candidates = [&]() {
    double best = -1.0;
    int bi = b;
    for (int i = tid; i < b; i += nthr) {
      if (done[i]) continue;
      const double v = dv[i];
      if (v > best || (v == best && i < bi)) { best = v; bi = i; }
    }
    if (warp < nwa) {
      for (int o = 16; o; o >>= 1) {
        const double ov = __shfl_xor_sync(0xffffffff, best, o);
        const int oi = __shfl_xor_sync(0xffffffff, bi, o);
        if (ov > best || (ov == best && oi < bi)) { best = ov; bi = oi; }
      }
      if (lane == 0) { redv[warp] = best; redi[warp] = bi; }
    }
  };
  warp_candidates();
  __syncthreads();
  for (int k = 0; k < b; ++k) {
    if (tid == 0) {
      double bv = -1.0;
      int bx = b;
      for (int i = 0; i < nwa; ++i)
        if (redv[i] > bv || (redv[i] == bv && redi[i] < bx)) { bv = redv[i]; bx = redi[i]; }
      if (!(bv > tau * maxd0) || !(bv > 0.0) || bx >= b) {
        flag[0] = k;
      } else {
        // the pivot's square root and reciprocal once, broadcast (see the eigensolver's reflector scalars)
        const double lkk = sqrt(bv);
        flag[1] = bx;
        done[bx] = 1;
        pos[bx] = k;
        perm[k] = bx;
        redv[29] = lkk;
        redv[30] = 1.0 / lkk;
      }
    }
    __syncthreads();
    if (flag[0] == k) break;
    const int p = flag[1];
    const double inv = redv[30];
    const double* rowp = W + (size_t)p * b;
    // column k of L for the rows that are not pivots (four independent accumulators: FP64 FMA latency)
    for (int i = tid; i < b; i += nthr) {
      if (done[i]) continue;
      const double* rowi = W + (size_t)i * b;
      double s0 = rowi[p], s1 = 0.0, s2 = 0.0, s3 = 0.0;
      int l = 0;
      for (; l + 3 < k; l += 4) {
        const int c0 = perm[l], c1 = perm[l + 1], c2 = perm[l + 2], c3 = perm[l + 3];
        s0 = fma(-rowi[c0], rowp[c0], s0);
        s1 = fma(-rowi[c1], rowp[c1], s1);
        s2 = fma(-rowi[c2], rowp[c2], s2);
        s3 = fma(-rowi[c3], rowp[c3], s3);
      }
      for (; l < k; ++l) s0 = fma(-rowi[perm[l]], rowp[perm[l]], s0);
      const double lik = ((s0 + s1) + (s2 + s3)) * inv;
      W[(size_t)i * b + p] = lik;
      dv[i] = fma(-lik, lik, dv[i]);
    }
    if (tid == 0) W[(size_t)p * b + p] = redv[29];
    warp_candidates();
    __syncthreads();
  }
  const int rho = flag[0];
  if (rhog && tid == 0) rhog[blockIdx.x] = rho;
  if (tid == 0) {
    // column q of L: (b - q - 1) rows of q multiply-adds; the triangular inverse (rho^3/6)
    double f = 0.0;
    for (int q = 0; q < rho; ++q) f += (double)(b - q - 1) * q;
    add_work(work, 2.0 * f + (Pc ? rho * (double)rho * rho / 3.0 : 0.0), sizeof(double) * 4.0 * bb);
  }
  // outputs: RA row k < rho, column j = L[j][k] for rows j that are not earlier pivots (upper triangular in
  // pivot order), RAc = RA with column j divided by c_j
  for (size_t t = tid; t < bb; t += nthr) {
    const int k = (int)(t / b), j = (int)(t - (t / b) * b);
    double v = 0.0;
    if (k < rho && pos[j] >= k) v = W[(size_t)j * b + perm[k]];
    RA[t] = v;
    if (RAc) RAc[t] = v / c[j];
  }
  if (!Pc) return;
  // L11^{-1} in pivot order: L11[i][l] = W[perm[i]][perm[l]]; reciprocal diagonal first, then one thread per
  // column q, forward substitution with four accumulators
  for (int i = tid; i < rho; i += nthr) rd[i] = 1.0 / W[(size_t)perm[i] * b + perm[i]];
  __syncthreads();
  for (int q = tid; q < rho; q += nthr) {
    for (int i = 0; i < q; ++i) Li[(size_t)i * b + q] = 0.0;
    for (int i = q; i < rho; ++i) {
      const double* rowi = W + (size_t)perm[i] * b;
      double s0 = (i == q) ? 1.0 : 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
      int l = q;
      for (; l + 3 < i; l += 4) {
        s0 = fma(-rowi[perm[l]], Li[(size_t)l * b + q], s0);
        s1 = fma(-rowi[perm[l + 1]], Li[(size_t)(l + 1) * b + q], s1);
        s2 = fma(-rowi[perm[l + 2]], Li[(size_t)(l + 2) * b + q], s2);
        s3 = fma(-rowi[perm[l + 3]], Li[(size_t)(l + 3) * b + q], s3);
      }
      for (; l < i; ++l) s0 = fma(-rowi[perm[l]], Li[(size_t)l * b + q], s0);
      Li[(size_t)i * b + q] = ((s0 + s1) + (s2 + s3)) * rd[i];
    }
  }
  __syncthreads();
  // Pc[perm[l]][q] = c[perm[l]] (L11^{-1})[q][l]
  for (size_t t = tid; t < bb; t += nthr) {
    const int r = (int)(t / b), q = (int)(t - (t / b) * b);  // Pc row r (original index), column q
    const int l = pos[r];
    const double v = (l < rho && q < rho && q >= l) ? c[r] * Li[(size_t)q * b + l] : 0.0;
    Pc[t] = v;
  }
}

void gram_factor(lrfg_ctx* ctx, const double* G, const double* c, int b, int batch, double* RA, double* RAc,
                 double* Pc, int* rho, double tau) {
  if (b <= 0 || batch <= 0) return;
  const size_t head = chol_head_bytes(b);
  const size_t full = head + sizeof(double) * 2 * (size_t)b * b;
  const int use_smem = full <= (size_t)std::min(ctx->max_smem_optin, 220 * 1024) ? 1 : 0;
  const size_t smem = use_smem ? full : head;
  DBuf<double> scratch;
  if (!use_smem) scratch = DBuf<double>(ctx->pool, (size_t)2 * b * b * batch);
  LRFG_CUDA(raise_smem_limit((const void*)gram_factor_kernel, smem));
  // algorithmic work up to the numerical rank, counted by each block on the device
  LRFG_LAUNCH(ctx, KC_CHOL, 0.0, 0.0,
              gram_factor_kernel<<<batch, kCholThreads, smem, ctx->stream>>>(G, c, b, tau, RA, RAc, Pc, rho,
                                                                               scratch.get(), use_smem,
                                                                               work_counter(ctx, KC_CHOL)));
}

}  // namespace lrfg

using namespace lrfg;

extern "C" lrfg_status lrfg_sym_eig(lrfg_ctx* ctx, const double* A, int n, int k, int batch, double* w, double* V) {
  if (!ctx) return LRFG_EINVAL;
  try {
    LRFG_CUDA(cudaSetDevice(ctx->device));
    LRFG_REQUIRE(A && w && V, "null argument");
    LRFG_REQUIRE(n >= 1 && k >= 1 && batch >= 1, "need n >= 1, k >= 1, batch >= 1 (got %d, %d, %d)", n, k, batch);
    syevx(ctx, A, w, V, n, std::min(k, n), batch);
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
