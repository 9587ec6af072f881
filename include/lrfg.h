/*
 * lrfg.h — C ABI of liblrfg: low-rank Fourier–Galerkin homogenisation on one GB300 GPU (sm_103a).
 *
 * The library computes the effective (homogenised) conductivity of a periodic cell Y = (-1/2,1/2)^d,
 * d in {2,3}, as defined in arXiv:1902.07455 Sec. 2.1, Eq. (homog):
 *     A_eff E.E = min over zero-mean periodic v of  int_Y A(x)(E + grad v).(E + grad v) dx,
 * discretised by the Fourier–Galerkin method with numerical integration (GaNi, Sec. 2.2.2) on an odd
 * grid N^d, or with exact integration on the double grid 2N - 1 (Ga, Sec. 2.2.3; lrfg_opts.disc),
 * preconditioned by the Fourier Laplacian (Sec. 2.3, Eq. (Pls_fourier)).  Solution formats:
 *   LRFG_FULL    the N^d grid; preconditioned CG (Sec. 3.3, Sec. 4);
 *   LRFG_TT      tensor train of rank r (fixed, or chosen by a tolerance, or raised during the iteration:
 *                lrfg_opts.rank_tol, rank_start); the truncated operator of Eq. (Pls_lowrank) and the
 *                minimal-residual iteration with truncation of Sec. 3.3;
 *   LRFG_TUCKER  Tucker tensor of fixed multilinear rank r (App. A.2), same operator and iteration,
 *                truncation by factor orthonormalisation + HOSVD of the core (App. A.2.3);
 *   LRFG_CP      canonical format, d = 2 only (App. A.1; Sec. 3.1 leaves d >= 3 out as ill-posed):
 *                there u = sum_i c_i x_i (x) y_i is a Tucker tensor and the CP truncation (QR of both
 *                factors, SVD of R1 diag(c) R2^T, App. A.1.3) is the d = 2 Tucker truncation, so CP
 *                problems run the Tucker path; their fields are Tucker fields (LRFG_ENOTSUP for d = 3).
 * The coefficient is A(x) = a(x) I + B: a scalar field a given as grid values, a tensor train or a Tucker
 * tensor, plus an optional constant symmetric positive semidefinite anisotropic part B (Sec. 4.4).
 * A Tucker problem built from grid values or a TT compresses the coefficient by HOSVD of its grid,
 * keeping singular values above 1e-7 of the largest in each mode (at most 64 per mode): the HOSVD
 * takes them from FP64 Gram matrices, which resolve singular values down to about sqrt(eps) of the
 * largest, so smaller ones are rounding noise.
 *
 * Conventions for every call:
 *   - every function returns an lrfg_status; no exception or signal crosses the ABI;
 *     lrfg_last_error(ctx) gives a one-line description of the last failure on that context;
 *   - N must be odd and >= 3 (Sec. 2.2.1: even N brings Nyquist frequencies); d in {2,3};
 *     violations, null pointers, non-finite or non-positive coefficients give LRFG_EINVAL;
 *   - grid arrays are row-major with storage index i along an axis holding x = k/N,
 *     k = i for i <= (N-1)/2 and k = i - N otherwise (the DFT order);
 *   - TT carriage j has shape (r[j], N[j], r[j+1]) row-major, r[0] = r[d] = 1 (App. A.3, Eq. (TT));
 *   - a Tucker core has shape (r[0], .., r[d-1]) row-major and factor j shape (N[j], r[j]) row-major;
 *   - "device" pointers are CUDA device addresses on the context's device; "host" pointers are
 *     ordinary host memory; inputs are caller-owned and not retained after the call returns;
 *     objects created by the library (lrfg_problem, lrfg_field) are freed by their *_free call;
 *   - all device work is issued on the context's stream; calls that return host values
 *     (A_eff, dots, solve results) synchronise that stream, the others are asynchronous;
 *   - one context per host thread; a context is not thread-safe (the lrfg_batch executor runs many
 *     solves concurrently, each worker thread with its own context and stream);
 *   - LRFG_ENOMEM means the context's HBM budget (or the device) cannot hold the request.
 * Arithmetic: FP64 throughout (LRFG_FP64); results are bitwise reproducible (no floating-point atomics).
 * LRFG_MIXED (LRFG_FULL GaNi solutions only; LRFG_ENOTSUP otherwise) stores the PCG vectors, the coefficient and the FFT work in FP32 and keeps every inner
 * product, step length, residual test and the A_eff evaluation in FP64; the solution field it hands
 * out is FP64.  It is an extension of the paper's FP64 method (the paper fixes no precision), for
 * tolerances down to about 1e-5.
 */
#ifndef LRFG_H
#define LRFG_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  LRFG_OK = 0,
  LRFG_EINVAL = 1,   /* invalid argument */
  LRFG_ENOMEM = 2,   /* HBM budget or device memory exhausted */
  LRFG_ENOCONV = 3,  /* iteration cap reached before the tolerance; results are still filled */
  LRFG_ECUDA = 4,    /* a CUDA runtime error; the message names the call */
  LRFG_ETIMEOUT = 5, /* reserved for bounded device-side waits */
  LRFG_ENOTSUP = 6   /* valid but not supported by the library */
} lrfg_status;

typedef enum { LRFG_FULL = 0, LRFG_CP = 1, LRFG_TUCKER = 2, LRFG_TT = 3 } lrfg_format;
typedef enum { LRFG_FP64 = 0, LRFG_MIXED = 1 } lrfg_prec;
/* discretisation: numerical integration on the grid (GaNi, Sec. 2.2.2) or exact integration on the
 * double grid 2N - 1 (Ga, Sec. 2.2.3) */
typedef enum { LRFG_GANI = 0, LRFG_GA = 1 } lrfg_disc;

/* spectral multipliers m(k) applied along one mode by F^{-1} diag(m) F (Sec. 2.2.1, Sec. 3.2) */
typedef enum {
  LRFG_MUL_IDENTITY = 0, /* m(k) = 1 */
  LRFG_MUL_DERIV = 1,    /* m(k) = 2 pi i k: the gradient factor of Sec. 2.2.1 along one mode */
  LRFG_MUL_GAUSS = 2     /* m(k) = exp(-t k^2), t = param: one factor of the exponential-sum P~^-1 */
} lrfg_multiplier;

typedef struct lrfg_ctx lrfg_ctx;
typedef struct lrfg_problem lrfg_problem;
typedef struct lrfg_field lrfg_field;

/* A tensor train whose carriages are caller-owned buffers (device or host as the call states). */
typedef struct {
  int d;
  int N[3];
  int r[4];          /* r[0] = r[d] = 1 */
  double* cores[3];  /* carriage j: r[j] * N[j] * r[j+1] doubles, row-major (r[j], N[j], r[j+1]) */
} lrfg_tt;

/* A Tucker tensor (App. A.2, Eq. (tucker)) whose core and factors are caller-owned buffers. */
typedef struct {
  int d;
  int N[3];
  int r[3];             /* multilinear ranks r[0..d-1] */
  double* core;         /* r[0] * .. * r[d-1] doubles, row-major */
  double* factors[3];   /* factor j: N[j] * r[j] doubles, row-major (N[j], r[j]) */
} lrfg_tucker;

/* Coefficient a(x) of A(x) = a(x) I (Sec. 2.1, Eq. (A); GaNi samples a(x_k), Sec. 2.2.2). */
typedef struct {
  int d;
  int N[3];
  lrfg_format fmt;      /* LRFG_FULL: `values` (N^d grid values); LRFG_TT: `tt`; LRFG_TUCKER: `tk` */
  const double* values; /* grid values, row-major, positive and finite */
  lrfg_tt tt;           /* carriages of a; the coefficient's TT ranks are its own (r_A) */
  int on_device;        /* 1: values / tt.cores / tk buffers are device pointers; 0: host pointers */
  lrfg_tucker tk;       /* core and factors of a (LRFG_TUCKER) */
  double B[9];          /* constant anisotropic part, d x d row-major (leading d x d of the 3 x 3 array):
                           A~(x) = a(x) I + B (the modified materials of Sec. 4.4).  All zero = isotropic.
                           B must be symmetric and positive semidefinite (LRFG_EINVAL otherwise); every
                           solution format */
} lrfg_coeff;

typedef struct {
  lrfg_format fmt;      /* solution format: LRFG_FULL (PCG), LRFG_TT or LRFG_TUCKER (minimal residual) */
  lrfg_prec prec;       /* LRFG_FP64, or LRFG_MIXED with fmt == LRFG_FULL */
  int rank;             /* LRFG_TT: the fixed rank of every truncation T (Sec. 4.2), or the rank cap */
  double pinv_eps;      /* LRFG_TT: relative accuracy of the exponential-sum P~^-1 on [1, max k.k]
                           (0 selects 0.1) */
  double tol;           /* relative residual tolerance (preconditioned residual) */
  int maxit;            /* iteration cap */
  int stop_on_increase; /* low-rank formats: 1 = stop when the residual norm fails to decrease (Sec. 4.3);
                           k > 1 = stop after k consecutive iterations without a new smallest residual (the
                           patience: the randomised rounding's residual wanders near its floor); 0 = off */
  double rank_tol;      /* LRFG_TT / LRFG_TUCKER: 0 = fixed rank `rank`.  > 0: every truncation T keeps the
                           smallest ranks (at most `rank`) whose relative Frobenius error is <= rank_tol:
                           tol / sqrt(d-1) per TT bond (App. A.3.3), tol / sqrt(d) per Tucker mode (App.
                           A.2.3); a grid coefficient is TT-compressed with the same tolerance */
  int coeff_rank;       /* LRFG_TT with grid values: rank cap r_A of the coefficient's TT-SVD (0: `rank`) */
  int rank_start;       /* low-rank formats: 0 = fixed rank.  > 0: rank-adapting MinRes (the solver Sec. 4.3
                           proposes): truncations start at rank_start; when the residual fails to decrease,
                           or meets tol, below the cap `rank`, the rank rises by rank_step, the right-hand
                           side is rebuilt and the iteration restarts from the best iterate (tol is read as a
                           statement about the cap's solution: below it the residual is truncated at the
                           lower rank); at the cap it stops as the fixed-rank iteration, by stop_on_increase */
  int rank_step;        /* rank increment of the rank-adapting MinRes (0 selects 1) */
  lrfg_disc disc;       /* LRFG_GANI (default), or LRFG_GA with LRFG_FP64 (every solution format, with or without
                           an anisotropic part B, which enters as part of the material, A~ = a~ I + B 1~): the
                           grid values of a
                           are read as a pixel-wise constant material (a_p on the cell of side 1/N centred at
                           x_p), its integrals against the double-grid basis are computed exactly (DoGIP), and
                           A_eff is the exact integral of a |E + grad u|^2.  N_j and the double grid 2N_j - 1
                           must have prime factors <= 31 (LRFG_ENOTSUP otherwise; e.g. N = 13, 25, 63, 81,
                           189, 363) */
  int sketch_over;      /* LRFG_TT with LRFG_GANI: 0 = every T is the deterministic TT rounding (App. A.3.3).
                           p > 0: the material products and the P~^-1 product (the truncations whose input rank
                           is r_A r and R_P r) use the randomised rounding of lrfg_tt_round_sketch with a sketch
                           of ranks rank + p (products never formed); the other truncations stay deterministic.
                           An extension of the paper's method (Al Daas et al. 2023); LRFG_ENOTSUP elsewhere */
  unsigned int sketch_seed; /* SplitMix64 stream of that sketch */
  int sketch_keep;      /* with sketch_over > 0: 0 = the randomised truncations of the products end with the
                           truncation from the right to `rank`; 1 = they return the sketch's rank rank + sketch_over
                           (the intermediate rank of the product truncations, the other truncations unchanged:
                           the operator's output then has rank rank + sketch_over) */
} lrfg_opts;

typedef struct {
  double Aeff;      /* A_eff E.E (Eq. (homog)) */
  int iters;        /* iterations of the returned iterate */
  double rel_resid; /* relative residual norm of the returned iterate */
  int converged;    /* 1 if rel_resid <= tol */
  int applies;      /* operator applications performed */
  int ranks[4];     /* TT ranks of the solution (LRFG_TT) */
  double seconds;   /* wall time of the solve on the host clock, including synchronisation */
} lrfg_result;

/* ---------------------------------------------------------------------------------------------
 * context
 * ------------------------------------------------------------------------------------------- */

/* Create a context on CUDA device `device`.  `stream` is the cudaStream_t all work is issued on (NULL:
 * the legacy default stream).  `hbm_budget_bytes` caps the library's device pool (0: no cap).
 * lrfg_destroy fails with LRFG_EINVAL while problems or fields of the context are still alive. */
lrfg_status lrfg_create(lrfg_ctx** ctx, int device, void* stream, size_t hbm_budget_bytes);
lrfg_status lrfg_destroy(lrfg_ctx* ctx);
/* A static string naming a status (never NULL). */
const char* lrfg_strerror(lrfg_status st);
/* The message of the context's last failed call ("" after a success); owned by the context, valid until its
 * next call. */
const char* lrfg_last_error(const lrfg_ctx* ctx);
/* Wait for the context's stream. */
lrfg_status lrfg_sync(lrfg_ctx* ctx);
/* Number of kernels this context has launched so far (instrumentation). */
long long lrfg_launch_count(const lrfg_ctx* ctx);
/* Measured FP64 rates of the context's device in TFLOP/s (instrumentation: the roofline denominator of the
 * FP64-bound kernels): fused multiply-add on the FP64 pipe (8 independent chains per thread, 8 blocks of 256
 * threads per SM) and the FP64 tensor-core instruction mma.sync m8n8k4 (4 accumulators per warp); each timed
 * over one launch with CUDA events after a warm-up launch.  Synchronises the stream. */
lrfg_status lrfg_probe_fp64(lrfg_ctx* ctx, double* fma_tflops, double* dmma_tflops);
/* Bytes currently held by the context's device pool (in use, and reserved including cached). */
lrfg_status lrfg_pool_bytes(const lrfg_ctx* ctx, size_t* in_use, size_t* reserved);

/* Kernel accounting.  Every launch is counted per kernel class (lrfg_profile_classes() classes named
 * by lrfg_profile_class_name) with its algorithmic floating-point operations and DRAM bytes (each operand
 * read once, each result written once).  While profiling is enabled, every launch is also bracketed by
 * CUDA events on the context's stream and its device time is added to its class.  lrfg_profile_read
 * synchronises the stream and copies the first n classes' totals (any output pointer may be NULL). */
int lrfg_profile_classes(void);
const char* lrfg_profile_class_name(int k);
lrfg_status lrfg_profile_enable(lrfg_ctx* ctx, int on);
lrfg_status lrfg_profile_reset(lrfg_ctx* ctx);
lrfg_status lrfg_profile_read(lrfg_ctx* ctx, int n, long long* launches, double* flops, double* bytes, double* ms);

/* ---------------------------------------------------------------------------------------------
 * mode-wise operators on fibres (rows a1, a2 of the hot path)
 * ------------------------------------------------------------------------------------------- */

/* Batched 1D DFT along the middle axis of a complex (re,im interleaved) FP64 device array of shape
 * (outer, N, inner): y[o,f,i] = sum_n x[o,n,i] exp(sign 2 pi i f n / N), unnormalised; sign = -1
 * is N * F_N and sign = +1 is F_N^{-1} of Sec. 2.2.1 (the mode-wise FFT of App. A.3.2).  `in` and
 * `out` may alias.  N odd (radices 3, 5, 7 and any other prime). */
lrfg_status lrfg_fft_fibres(lrfg_ctx* ctx, const double* in, double* out, int outer, int N, int inner,
                            int sign);

/* The same transform of a complex FP32 device array (re,im interleaved floats), in FP32 arithmetic with
 * FP32-rounded twiddles: the fibre passes of the LRFG_MIXED full format.  Relative error a few
 * u_32 log2(N) of the fibre's norm. */
lrfg_status lrfg_fft_fibres_f32(lrfg_ctx* ctx, const float* in, float* out, int outer, int N, int inner,
                                int sign);

/* out = scale * F_N^{-1} diag(m) F_N in along the middle axis of a REAL FP64 device array of shape
 * (outer, N, inner): the real-space form of a Fourier multiplier acting on one mode.  With
 * LRFG_MUL_DERIV this is one component of F^{-1} grad^ F (Sec. 2.2.1, Eq. (grad_trig)) applied to TT
 * carriage fibres, i.e. the rank-preserving gradient of Sec. 3.2.  `in` and `out` may alias. */
lrfg_status lrfg_fibre_operator(lrfg_ctx* ctx, const double* in, double* out, int outer, int N, int inner,
                                lrfg_multiplier kind, double param, double scale);

/* ---------------------------------------------------------------------------------------------
 * tensor-train operations on caller-owned device carriages (rows a3, a4, a5, a6, a7)
 * ------------------------------------------------------------------------------------------- */

/* Element-wise product: carriages combine by the Khatri–Rao product of App. A.3.1,
 * out_j[(i,k), n, (j,l)] = x_j[i,n,j] y_j[k,n,l] with pair index i*s + k.  out->r is set to the
 * products of the ranks; out->cores must each hold r_x[j] r_y[j] N[j] r_x[j+1] r_y[j+1] doubles. */
lrfg_status lrfg_tt_hadamard(lrfg_ctx* ctx, const lrfg_tt* x, const lrfg_tt* y, lrfg_tt* out);

/* out = alpha x + beta y in block-carriage form (ranks add; the TT sum referred to in Sec. 3.1.3).
 * out->cores must each hold (rx[j]+ry[j]) N[j] (rx[j+1]+ry[j+1]) doubles (first/last: one side 1). */
lrfg_status lrfg_tt_add(lrfg_ctx* ctx, double alpha, const lrfg_tt* x, double beta, const lrfg_tt* y,
                        lrfg_tt* out);

/* The eigenproblem inside every truncation T (App. A.3.3): the Gram-SVD rounding truncates each bond through
 * the k largest eigenpairs of a small symmetric positive semidefinite Gram core.  For `batch` symmetric FP64
 * matrices A (device, n x n row-major each, only symmetric input is meaningful, left unchanged): w (device,
 * n doubles per item) receives the k largest eigenvalues in descending order in w[0..k); V (device, n x n
 * row-major per item) the matching orthonormal eigenvectors in its first k columns.  Entries of w past k and
 * columns of V past k are not written.  Absolute accuracy about eps ||A|| (Householder tridiagonalisation, bisection, inverse
 * iteration with re-orthogonalisation of eigenvalues closer than 1e-3 ||A||; one thread block per matrix).
 * k >= 1 (k > n is clamped to n); n >= 1, batch >= 1.  Asynchronous on the context's stream. */
lrfg_status lrfg_sym_eig(lrfg_ctx* ctx, const double* A, int n, int k, int batch, double* w, double* V);

/* Rank truncation T (App. A.3.3) to ranks <= rmax: the result equals TT rounding (right-to-left
 * orthogonalisation, then left-to-right truncated SVDs) up to rounding; computed from Gram matrices
 * of the unfoldings (Gram-SVD).  out->r is set; out->cores must each hold
 * min(rmax, x->r[j]) N[j] min(rmax, x->r[j+1]) doubles.  Carriages 1..d-1 of out are
 * left-orthonormal. */
lrfg_status lrfg_tt_round(lrfg_ctx* ctx, const lrfg_tt* x, int rmax, lrfg_tt* out);
/* The same with a tolerance (tol in [0, 1), 0 = lrfg_tt_round): the smallest ranks <= rmax whose
 * relative Frobenius error is <= tol, tol / sqrt(d-1) per bond (App. A.3.3); the output ranks in out->r
 * may be below the cap, the carriages are written contiguously with those ranks. */
lrfg_status lrfg_tt_round_tol(lrfg_ctx* ctx, const lrfg_tt* x, int rmax, double tol, lrfg_tt* out);
/* Tucker truncation T (App. A.2.3) of a Tucker tensor with device buffers into out (device buffers of
 * at least prod_j min(rmax, r_j) core and N_j min(rmax, r_j) factor doubles; out->r is set): every
 * factor orthonormalised (unit-column balanced Gram matrix, pivoted Cholesky), its triangular factor
 * moved into the core, then the HOSVD of the core keeps min(rmax, r_j) vectors per mode. */
lrfg_status lrfg_tucker_round(lrfg_ctx* ctx, const lrfg_tucker* x, int rmax, lrfg_tucker* out);
/* The same with a tolerance: per mode the smallest rank <= rmax whose dropped singular values of the
 * core unfolding have norm <= tol / sqrt(d) of the tensor's (App. A.2.3); out->r holds the ranks, the
 * core and factors are written contiguously with them. */
lrfg_status lrfg_tucker_round_tol(lrfg_ctx* ctx, const lrfg_tucker* x, int rmax, double tol, lrfg_tucker* out);

/* Randomised truncation of a TT with device carriages ("randomize-then-orthogonalize", Al Daas, Ballard, Cazeaux,
 * Hallman, Miedlar, Pasha, Reid, Saibaba, SIAM J. Sci. Comput. 45 (2023) A74-A95; an extension of the paper's
 * deterministic rounding of App. A.3.3, whose cost grows like N s^3 in the input rank s):
 *   1. the sketch Omega: a TT of inner ranks `ell` with entries +-1, entry t of carriage j the sign (top bit) of
 *      output (j + 1) 2^40 + t of the SplitMix64 stream `seed` (Steele, Lea, Flood, OOPSLA 2014);
 *   2. W_{d-1} = x_{d-1} Omega_{d-1}^T, W_{j-1} = sum_n x_j[:, n, :] W_j Omega_j[:, n, :]^T (right to left);
 *   3. left to right: A = X_j W_j, Q = orth(A) (CholeskyQR2, directions below ~1e-6 of the largest singular
 *      value at the bond dropped), X_j <- Q, X_{j+1} <- (Q^T X_j) x_{j+1};
 *   4. the rank-ell result, left-orthonormal after step 3, truncated to ranks <= rmax by the truncated SVDs of
 *      App. A.3.3 taken from the right (tol > 0: the smallest such ranks within the relative tolerance tol,
 *      tol / sqrt(d-1) per bond, as lrfg_tt_round_tol).
 * When x's ranks do not exceed ell the result equals the deterministic rounding taken in that direction (up to
 * rounding); that is lrfg_tt_round's result for d = 2, or when only one bond loses rank.  d = 2 or 3.  out->r is
 * set; out->cores must each hold min(rmax, ..) N[j] min(rmax, ..) doubles. */
lrfg_status lrfg_tt_round_sketch(lrfg_ctx* ctx, const lrfg_tt* x, int ell, unsigned long long seed, int rmax,
                                 double tol, lrfg_tt* out);
/* The same truncation of the element-wise product x (.) y (App. A.3.1) without forming it: the Khatri–Rao middle
 * carriage enters steps 2 and 3 through contractions with x's and y's carriages in turn. */
lrfg_status lrfg_tt_hadamard_round_sketch(lrfg_ctx* ctx, const lrfg_tt* x, const lrfg_tt* y, int ell,
                                          unsigned long long seed, int rmax, double tol, lrfg_tt* out);

/* Euclidean inner product <x, y> = sum_k x[k] y[k] of two TTs (FP64 contraction). */
lrfg_status lrfg_tt_dot(lrfg_ctx* ctx, const lrfg_tt* x, const lrfg_tt* y, double* result);

/* The same inner product as lrfg_tt_dot, for callers that cannot allocate device memory when they need
 * it: applications whose own allocator owns all device memory, and loops that must not wait on the
 * driver's allocator.  (The paper has no counterpart: this is a calling convention of the library, not
 * part of the method.)
 *   - allocates nothing: the contraction intermediates live in one file-scope 4 MiB device array
 *     (524288 doubles) that every GPU loading the library holds until the process exits; its products
 *     run in one pass over the contracted index (no split-K partial sums), and nothing is taken from the
 *     context's pool; no profiling events are recorded (launches are still counted);
 *   - x, y: device carriages as for lrfg_tt_dot; `result` is a DEVICE pointer to one double, written
 *     asynchronously on the context's stream (nothing is synchronised or copied to the host);
 *   - the intermediates must fit: 2 max_j(r_x[j] r_y[j]) + max_j(r_y[j] N[j] r_x[j+1]) <= 524288
 *     doubles, else LRFG_EINVAL with a message (nothing is launched); e.g. ranks 40 x 40 fit up to
 *     N = 325;
 *   - the first call on a device looks up the array's device address (cudaGetSymbolAddress with that
 *     device current); make that first call before any stream capture begins;
 *   - all calls share the one array and overwrite it: calls whose work overlaps on the GPU (on
 *     different streams or contexts of the same device, or from several host threads) race. */
lrfg_status lrfg_tt_dot_noalloc(lrfg_ctx* ctx, const lrfg_tt* x, const lrfg_tt* y, double* result);

/* out = T(P~^-1 x) in real space: the exponential-sum preconditioner of accuracy pinv_eps applied as a
 * sum of separable Gaussian multipliers (rank R_P x r_x), then truncated to rmax (Sec. 2.3, 3.2).
 * out->cores must each hold min(rmax, R_P x->r[j]) N[j] min(rmax, R_P x->r[j+1]) doubles. */
lrfg_status lrfg_tt_precond(lrfg_ctx* ctx, const lrfg_tt* x, double pinv_eps, int rmax, lrfg_tt* out);

/* TT-SVD of a full device grid array (App. A.3.3, first case) to ranks <= rmax (and relative
 * accuracy tol when tol > 0).  out->cores must each hold min(rmax, ...) N[j] min(rmax, ...) doubles. */
lrfg_status lrfg_tt_compress(lrfg_ctx* ctx, int d, const int N[3], const double* values, int rmax,
                             double tol, lrfg_tt* out);

/* Expand a TT into a full device grid array of N^d doubles. */
lrfg_status lrfg_tt_expand(lrfg_ctx* ctx, const lrfg_tt* x, double* values);

/* ---------------------------------------------------------------------------------------------
 * problems: a resident coefficient plus workspace, the operator, the solvers (rows a1-a9)
 * ------------------------------------------------------------------------------------------- */

/* Make the coefficient device-resident for the given options (copies it; caller buffers may be
 * freed afterwards).  For LRFG_TT a FULL coefficient is compressed by TT-SVD to rank opts->coeff_rank
 * (opts->rank when 0), with the tolerance opts->rank_tol when it is > 0. */
lrfg_status lrfg_problem_create(lrfg_ctx* ctx, const lrfg_coeff* coeff, const lrfg_opts* opts,
                                lrfg_problem** problem);
/* Waits for the context's stream, then releases the problem (LRFG_EINVAL for NULL). */
lrfg_status lrfg_problem_free(lrfg_problem* problem);
/* TT ranks of the resident coefficient (r_A), or all 1 for LRFG_FULL. */
lrfg_status lrfg_problem_coeff_ranks(const lrfg_problem* problem, int ranks[4]);

/* One application of the preconditioned GaNi operator (the benchmark unit):
 *   LRFG_FULL: out = P^-1 grad^* F A~ F^-1 grad^ in on the Fourier half spectrum (Eq. (Pls_GaNi_fourier));
 *   LRFG_TT:   out = T P~^-1 T grad^* F T A~ F^-1 grad^ in (Eq. (Pls_lowrank)), computed in real space.
 * `in` must come from the same problem format and grid; *out is a new field. */
lrfg_status lrfg_problem_apply(lrfg_problem* problem, const lrfg_field* in, lrfg_field** out);
/* Same, into an existing field of the right format (no allocation of a new field object). */
lrfg_status lrfg_problem_apply_into(lrfg_problem* problem, const lrfg_field* in, lrfg_field* out);

/* Right-hand side b~ = -P^-1 grad^* F A~ E (FULL) or -T P~^-1 grad^* F A~ E (TT), Eq. (Pls_lowrank). */
lrfg_status lrfg_problem_rhs(lrfg_problem* problem, const double* E, lrfg_field** out);

/* Solve for E (host array of d doubles): FULL by PCG, TT by the minimal-residual iteration.
 * Fills *res; *u_out (may be NULL) receives the solution field.  Returns LRFG_ENOCONV (with *res
 * filled) when maxit is reached above tol and stop_on_increase did not end the iteration. */
lrfg_status lrfg_problem_solve(lrfg_problem* problem, const double* E, lrfg_result* res,
                               lrfg_field** u_out);

/* A_eff E.E = (1/|N|) sum_k a(x_k) |E + e(x_k)|^2, e = F^{-1} grad^ u (Eq. (homog), Sec. 2.2.2). */
lrfg_status lrfg_problem_aeff(lrfg_problem* problem, const double* E, const lrfg_field* u, double* Aeff);

/* Solve for nb macroscopic fields at once: E is a host array of nb x d doubles (row i = E_i), res receives nb
 * results (res[i].seconds is the wall time of the whole call).  For LRFG_TT problems with an isotropic GaNi
 * coefficient without tolerance truncation (rank_tol = 0) and nb d <= 32, the minimal-residual iterations of the
 * nb right-hand sides run in lockstep: every operator application, truncation and inner product takes one
 * launch sequence for all of them (each keeps its own step length, best iterate and stopping test; the results
 * equal separate solves up to the rounding order of the batched products).  With rank adaptation the items share
 * the current rank: an item that would raise it waits (frozen) until all unfinished items would, then all
 * restart from their best iterates at the next rank, which leaves each item's sequence that of its own solve.
 * Otherwise the nb solves run one after the other.  Status as lrfg_problem_solve (LRFG_ENOCONV if any right-hand side reached maxit). */
lrfg_status lrfg_problem_solve_many(lrfg_problem* problem, int nb, const double* E, lrfg_result* res);
/* Solve np problems of one shape together (a batch of microstructures): problem i for E_i (row i of E, a host
 * array of np x d doubles); res[i] receives its result (res[i].seconds is the wall time of the whole call).  The
 * problems must belong to one context.  When every problem is one lrfg_problem_solve_many runs in lockstep
 * (isotropic GaNi LRFG_TT, rank_tol = 0), all have the same grid, equal options (after their defaults are applied)
 * and equal coefficient TT ranks, and np d <= 32, their minimal-residual iterations (Sec. 4.3) run in lockstep: one
 * launch sequence per operator application (Eq. (Pls_lowrank)), truncation and inner product for all np, item i
 * with problem i's coefficient and right-hand side and its own step length, best iterate and stopping test (with
 * rank adaptation, the shared rank as in lrfg_problem_solve_many); each result equals problem i's own solve up to
 * the rounding order of the batched products.  Otherwise the problems are solved one after the other.  LRFG_EINVAL
 * for np < 1, a null problem, problems of different contexts or of different d; otherwise status as lrfg_problem_solve_many. */
lrfg_status lrfg_problems_solve(int np, lrfg_problem* const* problems, const double* E, lrfg_result* res);
/* The homogenised tensor A_eff (d x d, symmetric) of Eq. (homog): the diagonal A_aa from the solves with
 * E = e_a, each off-diagonal entry by polarisation of the quadratic form q(E) = A_eff E.E (Sec. 2.1),
 * A_ab = (q(e_a + e_b) - q(e_a) - q(e_b)) / 2 — d (d + 1) / 2 solves with the problem's options, run
 * through lrfg_problem_solve_many (in lockstep where it allows).
 *   A        host array of d * d doubles, row-major, written on return (caller-owned);
 *   results  NULL, or a host array of d (d + 1) / 2 lrfg_result, one per solve in the order
 *            (a, b) = (0,0), (0,1), .., (0,d-1), (1,1), .., (d-1,d-1) with E = e_a (+ e_b when b != a).
 * Returns the first failing solve's status (A is then not written), LRFG_ENOCONV when some solve
 * reached its iteration cap above the tolerance (A is still written), else LRFG_OK. */
lrfg_status lrfg_problem_aeff_tensor(lrfg_problem* problem, double* A, lrfg_result* results);

/* One-shot convenience: create a problem, solve, free it. */
lrfg_status lrfg_solve(lrfg_ctx* ctx, const lrfg_coeff* coeff, const double* E, const lrfg_opts* opts,
                       lrfg_result* res, lrfg_field** u_out);

/* ---------------------------------------------------------------------------------------------
 * batch / serving executor (an extension beyond the paper: many independent solves of Sec. 4's
 * problems, of different d, N, format and rank, overlapped on one GPU)
 *
 * W worker threads, each with its own non-blocking stream and context, take submitted requests in
 * FIFO order.  A request starts when a worker is free and its device footprint fits, beside the
 * footprints of the requests running, in hbm_budget_bytes (0: no cap; a request larger than the
 * budget runs alone).  The footprint is the pool high-water mark measured on the last solve of the
 * same shape (d, N, coefficient format and rank, solution format, precision, rank), or an estimate
 * from the sizes before one ran.  Each request is one lrfg_solve on its worker's context, so its
 * result is that of the same solve run alone.
 *
 * Batching across requests (lrfg_batch_set_group, off by default): a worker that takes the head request also
 * takes the queued requests that one lockstep solve can share with it (isotropic GaNi LRFG_TT solves with
 * rank_tol = 0 of TT coefficients with equal grid and ranks, equal options), in queue order while their
 * footprints fit, up to the group size, and solves them together by lrfg_problems_solve: one launch sequence per
 * operator application, truncation and inner product for all of them.  Each result then equals its own solve up
 * to the rounding order of the batched products.  Requests that arrive while a group runs form the next group.
 * ------------------------------------------------------------------------------------------- */

typedef struct lrfg_batch lrfg_batch;

typedef struct {
  double queue_s;    /* submission to start (waiting for a worker and for HBM) */
  double run_s;      /* start to completion */
  double total_s;    /* submission to completion: the request's latency */
  double peak_bytes; /* device pool high-water mark of the solve (of the whole group's lockstep solve) */
  int worker;        /* worker that ran it */
  int group;         /* requests solved together with it in lockstep, itself included (1: alone) */
  char message[200]; /* lrfg_last_error of the failed solve ("" on success) */
} lrfg_batch_report;

/* Start `workers` (1..64) worker threads on `device`.  LRFG_ECUDA if a stream or context cannot be
 * created (nothing is left behind). */
lrfg_status lrfg_batch_create(lrfg_batch** out, int device, int workers, size_t hbm_budget_bytes);
/* Queue one solve.  The coefficient must be in host memory (on_device = 0): its buffers are copied
 * before the call returns, as are E (d doubles) and *opts.  *ticket identifies the request.  Invalid
 * sizes give LRFG_EINVAL here; everything else lrfg_solve checks is reported by lrfg_batch_poll. */
lrfg_status lrfg_batch_submit(lrfg_batch* batch, const lrfg_coeff* coeff, const double* E, const lrfg_opts* opts,
                              unsigned long long* ticket);
/* Requests of one lockstep key taken together, at most max_requests (1..32; 1, the default, takes them one
 * at a time).  It applies to groups formed after the call.  LRFG_EINVAL outside 1..32. */
lrfg_status lrfg_batch_set_group(lrfg_batch* batch, int max_requests);
/* *ready = 1 when the request has completed; then *solve_status (lrfg_solve's status), *res and
 * *report (each may be NULL) are filled and the ticket is retired (a second poll gives LRFG_EINVAL).
 * wait = 1 blocks until it completes.  LRFG_EINVAL for an unknown or retired ticket. */
lrfg_status lrfg_batch_poll(lrfg_batch* batch, unsigned long long ticket, int wait, int* ready,
                            lrfg_status* solve_status, lrfg_result* res, lrfg_batch_report* report);
/* Requests waiting, running, and the footprint bytes admitted for the running ones (each may be NULL). */
lrfg_status lrfg_batch_info(lrfg_batch* batch, int* queued, int* running, size_t* in_flight_bytes);
/* Drop the requests not yet started (a poll waiting on one returns it with solve status LRFG_EINVAL),
 * wait for the running ones and for threads inside lrfg_batch_poll, stop the workers, free everything.
 * No call may use the executor after this one has started. */
lrfg_status lrfg_batch_destroy(lrfg_batch* batch);

/* ---------------------------------------------------------------------------------------------
 * fields
 * ------------------------------------------------------------------------------------------- */

/* Field from grid values u (N^d doubles): FULL keeps its Fourier half spectrum, TT is not allowed
 * here (use lrfg_field_from_tt). */
lrfg_status lrfg_field_from_full(lrfg_ctx* ctx, int d, const int N[3], const double* values, int on_device,
                                 lrfg_field** out);
/* Field from TT carriages of real grid values (copied). */
lrfg_status lrfg_field_from_tt(lrfg_ctx* ctx, const lrfg_tt* x, int on_device, lrfg_field** out);
/* A Tucker field (for LRFG_TUCKER problems) from a Tucker tensor in host or device buffers. */
lrfg_status lrfg_field_from_tucker(lrfg_ctx* ctx, const lrfg_tucker* x, int on_device, lrfg_field** out);
/* r: TT ranks r[0..d] for TT fields, multilinear ranks r[0..d-1] for Tucker fields, 1 otherwise. */
lrfg_status lrfg_field_info(const lrfg_field* f, lrfg_format* fmt, int* d, int N[3], int r[4]);
/* Grid values of the field into `values` (N^d doubles, host or device as on_device says). */
lrfg_status lrfg_field_export_full(lrfg_ctx* ctx, const lrfg_field* f, double* values, int on_device);
/* TT carriages of a TT field into caller buffers of the sizes lrfg_field_info implies. */
lrfg_status lrfg_field_export_tt(lrfg_ctx* ctx, const lrfg_field* f, double* const cores[3], int on_device);
/* Waits for the context's stream, then releases the field (LRFG_EINVAL for NULL). */
lrfg_status lrfg_field_free(lrfg_field* f);

#ifdef __cplusplus
}
#endif

#endif /* LRFG_H */
