// Full-format (N^d grid) building blocks: half-spectrum FFTs, Fourier multipliers, reductions.
#pragma once

#include "ops.cuh"

namespace lrfg {

struct FullGrid {
  int d;
  int N[3];
  int H;             // (N_{d-1} + 1) / 2
  long long rows;    // product of all but the last size
  long long n_real;  // N_0 ... N_{d-1}
  long long n_half;  // rows * H
  // exactly rounded 1/m for m = 0..sum_a ((N_a-1)/2)^2 (0 at m = 0): the preconditioner 1/(k.k); set
  // by make_inv_tables for grids that run the PCG kernels
  const double* inv_kk64 = nullptr;
  const float* inv_kk32 = nullptr;
};

FullGrid make_grid(int d, const int* N);
void make_inv_tables(lrfg_ctx* ctx, FullGrid& g, DBuf<double>& t64, DBuf<float>& t32);
// half_out = Phi(scale * coef .* real_in)   (coef may be null); Phi = unnormalised forward DFT
template <typename R>
void full_forward(lrfg_ctx* ctx, const FullGrid& g, const R* real_in, const R* coef, R scale,
                  typename CplxOf<R>::T* half_out);
// real_out = coef .* (scale * Phi^{*}(half))  (unnormalised inverse; half is overwritten)
template <typename R>
void full_inverse(lrfg_ctx* ctx, const FullGrid& g, typename CplxOf<R>::T* half_inout, const R* coef, R scale,
                  R* real_out);
// the complex-axis passes of full_inverse (before its rows) with grad^ folded into the first of them:
// half = Phi^{-1} on axes 0..d-2 of (in * 2 pi i k_alpha * scale)
template <typename V>
void half_grad_fibres_inverse(lrfg_ctx* ctx, const FullGrid& g, const V* in, V* half, int alpha, double scale);
// the complex-axis passes of full_forward (after its rows) with grad^* folded into the last of them, as
// half_acc_div does with the transformed half (which is left in an intermediate state)
template <typename V>
void half_fibres_forward_div(lrfg_ctx* ctx, const FullGrid& g, V* half, V* acc, int alpha, double scale, int init,
                             int precond);
// the last-axis passes of full_inverse and full_forward fused around a product with the real coefficient:
// half <- R2C(scale * coef (.) C2R(half)) along the rows (unnormalised transforms, in place)
template <typename R>
void full_rows_mul(lrfg_ctx* ctx, const FullGrid& g, typename CplxOf<R>::T* half_inout, const R* coef, R scale);
template <typename V>
void half_mul_grad(lrfg_ctx* ctx, const FullGrid& g, const V* in, V* out, int alpha, double scale);
template <typename V>
void half_acc_div(lrfg_ctx* ctx, const FullGrid& g, const V* in, V* acc, int alpha, double scale, int init,
                  int precond);
template <typename V>
void half_precond(lrfg_ctx* ctx, const FullGrid& g, const V* in, V* out);
// the constant anisotropic part of A~ = a I + B: acc += 4 pi^2 (k.B k) in, then, if precond, acc /= k.k
// (-div(B grad u) is the Fourier multiplier 4 pi^2 k.B k; B symmetric, 3 x 3 row-major storage)
template <typename V>
void half_acc_aniso(lrfg_ctx* ctx, const FullGrid& g, const V* in, V* acc, const double* B, int precond);
// out_dev (+)= (4 pi^2 / |N|) sum over the full spectrum of (k.B k) |v_k|^2 = sum_x e(x).B e(x) for the
// gradient field e of u with half spectrum v = Phi u (FP64)
void aniso_energy_sum(lrfg_ctx* ctx, const FullGrid& g, const double2* v, const double* B, double* out_dev,
                      int accumulate);
// Hermitian-weighted real inner product over the full spectrum (FP64 accumulation) into a device scalar
// optional: *ratio = *aux / result (mode 1) or result / *aux (mode 2), 0 for a zero divisor
template <typename V>
void half_dot(lrfg_ctx* ctx, const FullGrid& g, const V* x, const V* y, double* out_dev, const double* aux = nullptr,
              double* ratio = nullptr, int mode = 0);
// out_dev (+)= sum_k a_k (E + e_k)^2 (FP64 accumulation)
template <typename R>
void energy_sum(lrfg_ctx* ctx, const FullGrid& g, const R* e, const R* a, double E, double* out_dev, int accumulate);
// u += alpha p, r -= alpha q, z = P^-1 r (alpha a device scalar)
template <typename V>
void pcg_update(lrfg_ctx* ctx, const FullGrid& g, V* u, V* r, const V* p, const V* q, V* z, const double* alpha);
// p = z + beta p (beta a device scalar)
template <typename V>
void pcg_direction(lrfg_ctx* ctx, const FullGrid& g, V* p, const V* z, const double* beta);
template <typename A, typename B>
void convert(lrfg_ctx* ctx, const A* in, B* out, long long n);
// Ga (exact integration on the double grid gM, M = 2N - 1 per axis): zero padding I of a half spectrum of
// the grid g into one of gM, and its adjoint I* (the frequencies of g taken out of gM)
void half_inject(lrfg_ctx* ctx, const FullGrid& g, const FullGrid& gM, const double2* in, double2* out);
void half_project(lrfg_ctx* ctx, const FullGrid& g, const FullGrid& gM, const double2* in, double2* out);
// Ga modified coefficient of a pixel-wise constant a (values on the cells of g): out = (|N| / |M|) A~ on gM,
// A~[j] = int a phi^j_M dx; work: two half spectra (one of g, one of gM) and nothing else
void ga_coefficient(lrfg_ctx* ctx, const FullGrid& g, const FullGrid& gM, const double* a, double2* half_g,
                    double2* half_m, double* out);

}  // namespace lrfg
