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
};

FullGrid make_grid(int d, const int* N);
// half_out = Phi(scale * coef .* real_in)   (coef may be null); Phi = unnormalised forward DFT
void full_forward(lrfg_ctx* ctx, const FullGrid& g, const double* real_in, const double* coef, double scale,
                  double2* half_out);
// real_out = coef .* (scale * Phi^{*}(half))  (unnormalised inverse; half is overwritten)
void full_inverse(lrfg_ctx* ctx, const FullGrid& g, double2* half_inout, const double* coef, double scale,
                  double* real_out);
void half_mul_grad(lrfg_ctx* ctx, const FullGrid& g, const double2* in, double2* out, int alpha, double scale);
void half_acc_div(lrfg_ctx* ctx, const FullGrid& g, const double2* in, double2* acc, int alpha, double scale, int init,
                  int precond);
void half_precond(lrfg_ctx* ctx, const FullGrid& g, const double2* in, double2* out);
// Hermitian-weighted real inner product over the full spectrum, written to a device scalar
void half_dot(lrfg_ctx* ctx, const FullGrid& g, const double2* x, const double2* y, double* out_dev);
// out_dev (+)= sum_k a_k (E + e_k)^2
void energy_sum(lrfg_ctx* ctx, const FullGrid& g, const double* e, const double* a, double E, double* out_dev,
                int accumulate);
void pcg_update(lrfg_ctx* ctx, const FullGrid& g, double2* u, double2* r, const double2* p, const double2* q,
                double2* z, const double* num, const double* den);
void pcg_direction(lrfg_ctx* ctx, const FullGrid& g, double2* p, const double2* z, const double* num,
                   const double* den);

}  // namespace lrfg
