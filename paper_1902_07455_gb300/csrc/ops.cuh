// Internal host-side entry points of the kernels (one translation unit each implements a group).
#pragma once

#include "common.cuh"
#include "fft_device.cuh"

namespace lrfg {

// ---- fft.cu -------------------------------------------------------------------------------------
// passes for length N with register radices up to max_radix (27 for FP32 data, 9 for FP64, whose
// larger register footprint would limit occupancy)
FftPlan make_plan(int N, int max_radix);
template <typename V>
constexpr int plan_radix() { return sizeof(V) == sizeof(float2) ? 27 : 9; }
// device twiddle table W[j] = exp(-2 pi i j / N) in FP64 (double) or rounded to FP32 (float)
template <typename R>
const typename CplxOf<R>::T* twiddle_table(lrfg_ctx* ctx, int N);
// batched complex DFT along the middle axis of (outer, N, inner); sign -1 forward, +1 inverse
// (V = double2 or float2)
template <typename V>
void fft_fibres(lrfg_ctx* ctx, const V* in, V* out, long long outer, int N, long long inner, int sign);
// The gradient and divergence multipliers of the full-format operator (Eq. 2.10) folded into its axis-0
// fibre pass over the half spectrum (N0, inner) of a d = 2 or 3 grid, inner = N1 * H or H, so that fibre i
// holds the frequencies (k0 = n, i / H, i % H) or (n, i):
//  mode 1, inverse DFT: out = F^-1 (in * 2 pi i k_alpha * scale), the product taken on the staged tile;
//  mode 2, forward DFT: acc = ((init ? 0 : acc) - 2 pi i k_alpha * scale * F in) * (precond ? 1/(k.k) : 1),
//  the result of the transform never stored.
// The products are the ones of the separate pointwise kernels, in the same order and precision.
template <typename R>
struct FibreMul {
  int mode, alpha, d, N1, H, init, precond;
  R c2;             // 2 pi scale, rounded to R
  const R* inv_kk;  // 1/(k.k) indexed by k.k, 0 at k = 0 (mode 2 with precond)
};
template <typename V>
void fft_fibres_mul(lrfg_ctx* ctx, const V* in, V* out, int N0, long long inner,
                    const FibreMul<typename RealOf<V>::T>& fm);
// Ga mode maps on real fibres (outer, n_in, inner) -> (outer, n_out, inner), M = 2N - 1 (Sec. 2.2.3):
//  GA_UP      N -> M  band-limited interpolation to the double grid, F_M^-1 I F_N;
//  GA_DOWN    M -> N  projection, F_N^-1 I* F_M;
//  GA_EXTEND  N -> M  pixel values to the one-axis modified coefficient, M^-1 Phi*_M (s(m) (Phi_N g)(m mod N)),
//             s(m) = sin(pi m / N) / (pi m)
enum { GA_UP = 0, GA_DOWN = 1, GA_EXTEND = 2 };
void ga_resample(lrfg_ctx* ctx, const double* in, double* out, long long outer, int n_in, long long inner, int n_out,
                 int mode);
// real fibres: out = scale * F^-1 diag(m) F in, m given by kind/param (lrfg_multiplier); fp32: the transforms
// in FP32 (data read and written in FP64)
void fibre_operator(lrfg_ctx* ctx, const double* in, double* out, long long outer, int N, long long inner,
                    int kind, double param, double scale, bool fp32 = false);
// real fibres, many Gaussian multipliers at once: out_m = scale_m F^-1 diag(exp(-t_m k^2)) F in,
// written to out + m * out_stride for m = 0..nm-1 (the exponential-sum preconditioner terms)
void fibre_gauss_multi(lrfg_ctx* ctx, const double* in, double* out, long long out_stride, long long outer,
                       int N, long long inner, const double* t, const double* scale, int nm, bool fp32 = false);

// ---- linalg.cu ----------------------------------------------------------------------------------
// C[b] = alpha * op(A[b]) * op(B[b]) + beta * C[b], row-major, op = transpose when trans* != 0.
// A[b] is (transA ? K x M : M x K) with leading dimension lda, batch stride sA (elements); same for B.
void gemm(lrfg_ctx* ctx, int transA, int transB, int M, int N, int K, double alpha, const double* A, int lda,
          long long sA, const double* B, int ldb, long long sB, double beta, double* C, int ldc, long long sC,
          int batch = 1);
// The same with data-dependent active sizes: rows < dynM[b] * mulM, columns < dynN[b] * mulN of item b
// (either pointer may be null); the rest of C is left as it was (zeroed for split-K products).  The
// algorithmic count uses the static sizes.
void gemm_dyn(lrfg_ctx* ctx, int transA, int transB, int M, int N, int K, double alpha, const double* A, int lda,
              long long sA, const double* B, int ldb, long long sB, double beta, double* C, int ldc, long long sC,
              int batch, const int* dynM, int mulM, const int* dynN, int mulN);
// FP32 product (same layout rules, FP32 operands and accumulation)
void gemm_f32(lrfg_ctx* ctx, int transA, int transB, int M, int N, int K, double alpha, const float* A, int lda,
              long long sA, const float* B, int ldb, long long sB, double beta, float* C, int ldc, long long sC,
              int batch = 1);
void to_f32(lrfg_ctx* ctx, const double* in, float* out, long long n);
void to_f64(lrfg_ctx* ctx, const float* in, double* out, long long n);
// The same product in one pass over K (never split): no partial-sum workspace, nothing taken from the pool.
void gemm_nosplit(lrfg_ctx* ctx, int transA, int transB, int M, int N, int K, double alpha, const double* A, int lda,
                  long long sA, const double* B, int ldb, long long sB, double beta, double* C, int ldc, long long sC,
                  int batch = 1);
// symmetric eigen-decomposition of `batch` m x m matrices (row-major, stride m*m): eigenvalues in
// descending order into w (stride m), eigenvectors as the COLUMNS of V (row-major m x m, stride m*m).
// A is left unchanged.  syevj: FP64 Jacobi (absolute accuracy eps64 ||A||).  syevj_mixed: FP32 Jacobi +
// three FP64 Ogita–Aishima refinement steps; its eigenvectors are accurate only for eigenvalues that
// FP32 separates (gaps above ~1e-6 ||A||), so it serves the mixed-precision path, not the FP64 one.
void syevj(lrfg_ctx* ctx, double* A, double* w, double* V, int m, int batch = 1);
void syevj_mixed(lrfg_ctx* ctx, double* A, double* w, double* V, int m, int batch = 1);
// FP64 k largest eigenpairs by tridiagonalisation, bisection and inverse iteration: w[0..k) descending,
// eigenvectors in the first k columns of V (n x n row-major per batch item).  A is left unchanged.
void syevx(lrfg_ctx* ctx, const double* A, double* w, double* V, int n, int k, int batch = 1);
// Top-k left singular pairs of B (n x n per item, nonzero block nA[b] x nB[b]) from BBt = B B^T and
// BtB = B^T B: the smaller of the two nonzero blocks is decomposed (w = sigma^2); left vectors in the
// first k columns of V, completed to min(k, nA) orthonormal columns.
// The same on the leading n_eff[b] x n_eff[b] block of A (the rest of A is zero); the eigenvector
// rows beyond n_eff and the columns beyond min(k, n_eff) are zero.
void syevx_sized(lrfg_ctx* ctx, const double* A, const int* n_eff, double* w, double* V, int n, int k, int batch);
void syevx_product(lrfg_ctx* ctx, const double* BBt, const double* BtB, const double* B, const int* nA,
                   const int* nB, double* w, double* V, int n, int k, int batch);
// Gram-SVD factors from a balanced Gram matrix G (b x b per item) and the balancing c: pivoted
// Cholesky; writes RA (G ~ RA^T RA, nonzero rows first), RAc and Pc (b x b each per item; skipped when
// null, and then c may be null), and the numerical rank into rho (may be null).
// tau: the pivoted Cholesky stops when the largest remaining pivot is below tau times the largest diagonal.
void gram_factor(lrfg_ctx* ctx, const double* G, const double* c, int b, int batch, double* RA, double* RAc,
                 double* Pc, int* rho = nullptr, double tau = 1e-16);
// elementwise helpers
void fill(lrfg_ctx* ctx, double* x, double v, long long n);
void axpby(lrfg_ctx* ctx, long long n, double alpha, const double* x, double beta, double* y);  // y = a x + b y
double dot_host(lrfg_ctx* ctx, const double* x, const double* y, long long n);  // synchronises
// device-scalar dot: *out = sum x*y (no host sync)
void dot_device(lrfg_ctx* ctx, const double* x, const double* y, long long n, double* out);

// ---- tt.cu --------------------------------------------------------------------------------------
struct TTView {  // non-owning view of a TT with device carriages
  int d;
  int N[3];
  int r[4];
  const double* core[3];
};
// nb tensor trains of identical shape stored item after item in one buffer per carriage
struct TTBatch {
  int d = 0, nb = 0;
  int N[3] = {0, 0, 0};
  int r[4] = {1, 1, 1, 1};
  DBuf<double> core[3];
  size_t elems(int j) const { return (size_t)r[j] * N[j] * r[j + 1]; }
};
struct TTBatchView {
  int d, nb;
  int N[3];
  int r[4];
  const double* core[3];  // item b of carriage j at core[j] + b * elems(j)
  size_t elems(int j) const { return (size_t)r[j] * N[j] * r[j + 1]; }
};
void ttb_alloc(lrfg_ctx* ctx, TTBatch& x, int d, const int* N, const int* r, int nb);
TTBatchView batch_view(const TTBatch& x);
TTView item_view(const TTBatch& x, int b);
// rank truncation of every item of a batch (one batched Gram-SVD sweep): rank rmax, or with tol > 0 the
// smallest ranks <= rmax whose truncation error is <= tol ||x|| per item (tol / sqrt(d-1) per bond)
void tt_round_batch(lrfg_ctx* ctx, const TTBatchView& x, int rmax, TTBatch& out, double tol = 0.0);
TTView view_of(const TT& x);
TTView view_of(const lrfg_tt& x);
void tt_alloc(lrfg_ctx* ctx, TT& x, int d, const int* N, const int* r);
void tt_copy(lrfg_ctx* ctx, const TTView& src, TT& dst);
void tt_hadamard(lrfg_ctx* ctx, const TTView& x, const TTView& y, TT& out);
// Khatri–Rao product of one carriage pair into dst: (a c) x n x (b e)
void khatri_rao(lrfg_ctx* ctx, const double* x, int a, int n, int b, const double* y, int c, int e, double* dst);
// sum of nb TTs (views) in block form, each item scaled by scales[i] (on the first carriage)
void tt_add_many(lrfg_ctx* ctx, const TTView* xs, const double* scales, int nb, TT& out);
// out = alpha x + beta y; alpha_dev / beta_dev (may be null) are device scalars multiplying alpha/beta
void tt_add(lrfg_ctx* ctx, double alpha, const double* alpha_dev, const TTView& x, double beta,
            const double* beta_dev, const TTView& y, TT& out);
void tt_round(lrfg_ctx* ctx, const TTView& x, int rmax, TT& out, double tol = 0.0);
// Tolerance ranks of `nb` truncations: for item i, S (b x b, active block rk[i], may be null = b) with
// its top eigenvalues w (stride b, min(kcap, active) of them) and eigenvectors V (b x b, columns):
// k_dev[i] = the smallest k in [1, kcap] with trace(S) - sum_{t<k} w_t <= tol2 trace(S) (kcap if none);
// V's columns k_dev[i] .. kcap-1 are zeroed.
void tol_ranks(lrfg_ctx* ctx, const double* S, const int* rk, const double* w, double* V, int b, int kcap, double tol2,
               int nb, int* k_dev);
void tt_dot_device(lrfg_ctx* ctx, const TTView& x, const TTView& y, double* out_dev);
double tt_dot(lrfg_ctx* ctx, const TTView& x, const TTView& y);
void tt_expand(lrfg_ctx* ctx, const TTView& x, double* values);
void tt_compress(lrfg_ctx* ctx, int d, const int* N, const double* values, int rmax, double tol, TT& out);
// mode operator on carriage j (spectral multiplier along the mode index)
void tt_mode_operator(lrfg_ctx* ctx, const TTView& x, int j, int kind, double param, double scale, TT& out);
// exponential sum of 1/x on [1, xmax]: nodes t and weights w (host)
void expsum_inverse(double xmax, double eps, std::vector<double>& t, std::vector<double>& w);
// out = T(P~^-1 x) with the exponential sum (t, w); omega non-null: T is the randomised rounding with that sketch
void tt_precond(lrfg_ctx* ctx, const TTView& x, const std::vector<double>& t, const std::vector<double>& w,
                int rmax, TT& out, double tol = 0.0, const TTView* omega = nullptr, bool fp32 = false,
                bool final = true);

// block copy of a carriage (a x n x b) into a larger one (A x n x B) at rank offsets (oa, ob)
void tt_embed(lrfg_ctx* ctx, const double* src, int a, int n, int b, double* dst, int A, int B, int oa, int ob);

// ---- sketch.cu ----------------------------------------------------------------------------------
// Randomised rounding (randomize-then-orthogonalize) of products that are never formed.  A source describes
// nb tensor trains z_b of order d with ranks s: DENSE carriages (item after item), KHATRI_RAO products
// z_b = x (.) y_b (x shared, y_b's carriages given per item, ranks ry), or BLOCKS (nb = 1): the exponential-sum
// product whose carriage j holds nblocks blocks of shape (ry[j], N, ry[j+1]) at blocks[j] + m * block size,
// first carriage block-concatenated along its last index, last along its first, middle block-diagonal (nb items:
// bstride apart between blocks, one block size apart between items).
constexpr int kMaxSketchItems = 32;
struct SketchSource {
  enum Kind { DENSE = 0, KHATRI_RAO = 1, BLOCKS = 2 };
  Kind kind = DENSE;
  int d = 0, nb = 1;
  int N[3] = {0, 0, 0};
  int s[4] = {1, 1, 1, 1};
  const double* dense[3] = {nullptr, nullptr, nullptr};
  TTView x{};                                      // KHATRI_RAO: the coefficient factor (ranks, shared carriages)
  const double* xi[3][kMaxSketchItems] = {};       // KHATRI_RAO: item b's own coefficient carriages (null: x's)
  const double* y[3][kMaxSketchItems] = {};
  int ry[4] = {1, 1, 1, 1};
  int nblocks = 0;
  const double* blocks[3] = {nullptr, nullptr, nullptr};
  long long bstride[3] = {0, 0, 0};  // BLOCKS: elements between blocks m and m+1 (0: one block's size); item b's
                                     // blocks start b block sizes further on
  void materialise(lrfg_ctx* ctx, int j, double* dst) const;                      // first or last carriage
  void right_middle(lrfg_ctx* ctx, const double* W, int ell, double* T) const;     // T = Z_1 x_3 W
  void right_middle_f32(lrfg_ctx* ctx, const float* W, int ell, float* T) const;   // the same in FP32
  void left_middle(lrfg_ctx* ctx, const double* M, int ell, double* X) const;      // X = M x_1 Z_1
};
// Rademacher sketch TT of inner ranks ell (SplitMix64 stream `seed`)
void sketch_tt(lrfg_ctx* ctx, int d, const int* N, int ell, unsigned long long seed, TT& out);
// randomised rounding of every item to rank rmax (tolerance tol > 0: the smallest ranks <= rmax within it)
// fp32: the right sweep and the sketched products in FP32 (they only choose the subspaces; every projection of
// the tensor's values stays FP64).  final = false: return the rank-l left-orthonormal result of the sketch
// without the deterministic rounding to rmax / tol.
void tt_round_sketch(lrfg_ctx* ctx, const SketchSource& z, const TTView& omega, int rmax, TTBatch& out,
                     double tol = 0.0, bool fp32 = false, bool final = true);

// ---- ttbatch.cu ---------------------------------------------------------------------------------
TTView item_view_of(const TTBatchView& x, int b);
// out_i = sum_t s_t,i x_t,i in block form for every item i (s_t,i = hs[t] * ds[t][i], either may be null; the
// scale multiplies the first carriage)
void ttb_add_many(lrfg_ctx* ctx, const TTBatchView* xs, int m, const double* hs, const double* const* ds,
                  TTBatch& out);
// out_dev[i] = <x_i, y_i>
void ttb_dot_device(lrfg_ctx* ctx, const TTBatchView& x, const TTBatchView& y, double* out_dev);
// out_i = T(P~^-1 x_i) (omega non-null: randomised rounding, one launch sequence for all items)
void ttb_precond(lrfg_ctx* ctx, const TTBatchView& x, const std::vector<double>& t, const std::vector<double>& w,
                 int rmax, TTBatch& out, double tol, const TTView* omega, bool fp32 = false, bool final = true);

// ---- tucker.cu ----------------------------------------------------------------------------------
// Tucker tensor on the device: core (r_0, .., r_{d-1}) row-major, factor j (N_j, r_j) row-major
struct TK {
  int d = 0;
  int N[3] = {1, 1, 1};
  int r[3] = {1, 1, 1};
  DBuf<double> core;
  DBuf<double> fac[3];
};
struct TKView {
  int d;
  int N[3];
  int r[3];
  const double* core;
  const double* fac[3];
};
struct TKSolveResult {
  double Aeff;
  int iters;
  double rel_resid;
  int applies;
};
// Ga in Tucker / CP format (Sec. 2.2.3): the modified coefficient on the double grid M = 2N - 1 and its
// projection back to the grid (the right-hand side's coefficient), both with the factors of a's pixel values
// mapped mode by mode
struct TKGa {
  TKView a_ga;     // on M
  TKView a_down;   // on N
  TKView ones_ga;  // on M: the modified coefficient of the constant 1 (with an anisotropic part B)
};
TKView tk_view(const TK& x);
void tk_alloc(lrfg_ctx* ctx, TK& x, int d, const int* N, const int* r);
void tk_copy(lrfg_ctx* ctx, const TKView& x, TK& out);
void tk_mode_operator(lrfg_ctx* ctx, const TKView& x, int j, int kind, double param, double scale, TK& out);
void tk_hadamard(lrfg_ctx* ctx, const TKView& x, const TKView& y, TK& out);
void tk_add_many(lrfg_ctx* ctx, const TKView* xs, const double* scales, int nb, TK& out);
// truncation to multilinear ranks <= rmax; with tol > 0 each mode keeps the smallest rank whose dropped
// singular values of the core unfolding have norm <= tol / sqrt(d) ||x|| (App. A.2.3 HOSVD bound)
void tk_round(lrfg_ctx* ctx, const TKView& x, int rmax, TK& out, double tol = 0.0);
void tk_dot_device(lrfg_ctx* ctx, const TKView& x, const TKView& y, double* out_dev);
double tk_dot(lrfg_ctx* ctx, const TKView& x, const TKView& y);
void tk_expand(lrfg_ctx* ctx, const TKView& x, double* values);
void tk_compress(lrfg_ctx* ctx, int d, const int* N, const double* values, int rmax, double tol, TK& out);
void tk_precond(lrfg_ctx* ctx, const TKView& x, const std::vector<double>& t, const std::vector<double>& w, int rmax,
                TK& out, double tol = 0.0);
// every factor of x resampled to the grid n_out by the Ga mode map `mode` (GA_UP / GA_DOWN / GA_EXTEND)
void tk_ga_map(lrfg_ctx* ctx, const TKView& x, const int* n_out, int mode, TK& out);
// ga: Ga (null: GaNi); B is then null (isotropic)
void tk_apply(lrfg_ctx* ctx, const TKView& a, const TKView& v, const std::vector<double>& pt,
              const std::vector<double>& pw, int rank, TK& out, double rtol = 0.0, const double* B = nullptr,
              const TKGa* ga = nullptr);
void tk_rhs(lrfg_ctx* ctx, const TKView& a, const double* E, const std::vector<double>& pt,
            const std::vector<double>& pw, int rank, TK& out, double rtol = 0.0, const TKGa* ga = nullptr);
// B: the constant anisotropic part (3 x 3 row-major storage) or null
double tk_aeff(lrfg_ctx* ctx, const TKView& a, const double* E, const TKView& u, const double* B = nullptr,
               const TKGa* ga = nullptr);
TKSolveResult tk_solve(lrfg_ctx* ctx, const TKView& a, const double* E, const std::vector<double>& pt,
                       const std::vector<double>& pw, int rank, double tol, int maxit, int stop_on_increase,
                       TK& best_u, double rtol = 0.0, const double* B = nullptr, int rank_start = 0,
                       int rank_step = 1, const TKGa* ga = nullptr);

}  // namespace lrfg
