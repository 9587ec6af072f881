// Batched tensor-train operations for solving several right-hand sides of one problem in lockstep: nb tensor
// trains of identical shape and ranks stored item after item (TTBatch), every launch covering all items.
// These are the block sum of Sec. 3.1 (the TT sum in block form), the inner products of Sec. 3.3 and the
// exponential-sum preconditioner of Sec. 2.3 in its low-rank form, each the batched counterpart of tt.cu's.
#include <algorithm>
#include <cmath>

#include "ops.cuh"

namespace lrfg {

static unsigned grid_n(lrfg_ctx* ctx, long long n) {
  long long g = (n + 255) / 256;
  long long cap = 16LL * (ctx->num_sms > 0 ? ctx->num_sms : 152);
  return (unsigned)std::max(1LL, std::min(g, cap));
}

// dst item i, block at rank offsets (oa, ob) of an (A, n, B) carriage <- scale_i * src item i (a, n, b)
__global__ void embed_batch_kernel(const double* __restrict__ src, long long ss, int a, int n, int b, double* dst,
                                   long long ds, int A, int B, int oa, int ob, double s,
                                   const double* __restrict__ s_dev, int nb) {
  const long long per = (long long)a * n * b, total = per * nb;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total; t += (long long)gridDim.x * blockDim.x) {
    const int item = (int)(t / per);
    const long long q = t - item * per;
    const int jb = (int)(q % b);
    const long long rest = q / b;
    const int nn = (int)(rest % n);
    const int ia = (int)(rest / n);
    const double sc = s_dev ? s * s_dev[item] : s;
    dst[(size_t)item * ds + ((size_t)(ia + oa) * n + nn) * B + (jb + ob)] = sc * src[(size_t)item * ss + q];
  }
}

void ttb_add_many(lrfg_ctx* ctx, const TTBatchView* xs, int m, const double* hs, const double* const* ds,
                  TTBatch& out) {
  LRFG_REQUIRE(m >= 1, "empty sum");
  const int d = xs[0].d, nb = xs[0].nb;
  int r[4] = {1, 1, 1, 1};
  for (int j = 1; j < d; ++j) {
    r[j] = 0;
    for (int t = 0; t < m; ++t) r[j] += xs[t].r[j];
  }
  for (int t = 0; t < m; ++t) LRFG_REQUIRE(xs[t].d == d && xs[t].nb == nb, "batched sum of unlike batches");
  ttb_alloc(ctx, out, d, xs[0].N, r, nb);
  for (int j = 0; j < d; ++j) {
    const int n = xs[0].N[j], A = out.r[j], B = out.r[j + 1];
    double* dst = out.core[j].get();
    if (d == 1 || (j != 0 && j != d - 1)) fill(ctx, dst, 0.0, (long long)out.elems(j) * nb);
    int oa = 0, ob = 0;
    for (int t = 0; t < m; ++t) {
      const TTBatchView& x = xs[t];
      const int a = x.r[j], b = x.r[j + 1];
      const double s = (j == 0 && hs) ? hs[t] : 1.0;
      const double* sd = (j == 0 && ds) ? ds[t] : nullptr;
      const long long total = (long long)a * n * b * nb;
      if (d == 1) {
        LRFG_REQUIRE(m == 1, "batched sum of order-1 trains");
      }
      const int boa = (j == 0) ? 0 : oa, bob = (j == d - 1) ? 0 : ob;
      LRFG_LAUNCH(ctx, KC_TT_MISC, (double)total, 2.0 * sizeof(double) * total,
                  embed_batch_kernel<<<grid_n(ctx, total), 256, 0, ctx->stream>>>(
                      x.core[j], (long long)x.elems(j), a, n, b, dst, (long long)out.elems(j), A, B, boa, bob, s, sd,
                      nb));
      oa += a;
      ob += b;
    }
  }
}

void ttb_dot_device(lrfg_ctx* ctx, const TTBatchView& x, const TTBatchView& y, double* out_dev) {
  LRFG_REQUIRE(x.d == y.d && x.nb == y.nb, "batched dot of unlike batches");
  const int nb = x.nb;
  DBuf<double> W(ctx->pool, (size_t)nb);
  fill(ctx, W.get(), 1.0, nb);
  for (int j = 0; j < x.d; ++j) {
    const int a = x.r[j], b = x.r[j + 1], c = y.r[j], e = y.r[j + 1], n = x.N[j];
    LRFG_REQUIRE(n == y.N[j], "dot of TTs on different grids");
    // V_i (c x (n b)) = W_i^T (c x a) x_i,j (a x (n b));  W'_i (b x e) = V_i^T y_i,j over (c n)
    DBuf<double> V(ctx->pool, (size_t)c * n * b * nb);
    gemm(ctx, 1, 0, c, n * b, a, 1.0, W.get(), c, (long long)a * c, x.core[j], n * b, (long long)x.elems(j), 0.0,
         V.get(), n * b, (long long)c * n * b, nb);
    double* dst = (j == x.d - 1) ? out_dev : nullptr;
    DBuf<double> Wn;
    if (!dst) { Wn = DBuf<double>(ctx->pool, (size_t)b * e * nb); dst = Wn.get(); }
    gemm(ctx, 1, 0, b, e, c * n, 1.0, V.get(), b, (long long)c * n * b, y.core[j], e, (long long)y.elems(j), 0.0,
         dst, e, (long long)b * e, nb);
    if (j != x.d - 1) W = std::move(Wn);
  }
}

void ttb_precond(lrfg_ctx* ctx, const TTBatchView& x, const std::vector<double>& t, const std::vector<double>& w,
                 int rmax, TTBatch& out, double tol, const TTView* omega, bool fp32, bool final) {
  const int d = x.d, nb = x.nb;
  const int R = (int)t.size();
  if (!omega || d < 2) {
    // deterministic rounding: item by item, packed into one batch
    std::vector<TT> parts(nb);
    for (int b = 0; b < nb; ++b) tt_precond(ctx, item_view_of(x, b), t, w, rmax, parts[b], tol, nullptr, fp32);
    int r[4] = {1, 1, 1, 1};
    for (int j = 0; j <= d; ++j) r[j] = parts[0].r[j];
    for (int b = 1; b < nb; ++b)
      for (int j = 0; j <= d; ++j) LRFG_REQUIRE(parts[b].r[j] == r[j], "batched preconditioner with unlike ranks");
    ttb_alloc(ctx, out, d, x.N, r, nb);
    for (int b = 0; b < nb; ++b)
      for (int j = 0; j < d; ++j)
        LRFG_CUDA(cudaMemcpyAsync(out.core[j].get() + (size_t)b * out.elems(j), parts[b].core[j].get(),
                                  sizeof(double) * out.elems(j), cudaMemcpyDeviceToDevice, ctx->stream));
    return;
  }
  // the blocks G_m x_j of every item in one launch per carriage: terms[j][m][item] (a x N x b each)
  std::vector<double> ones(R, 1.0);
  SketchSource z;
  z.kind = SketchSource::BLOCKS;
  z.d = d;
  z.nb = nb;
  z.nblocks = R;
  DBuf<double> terms[3];
  for (int j = 0; j < d; ++j) {
    z.N[j] = x.N[j];
    const size_t e = x.elems(j);
    terms[j] = DBuf<double>(ctx->pool, e * nb * R);
    fibre_gauss_multi(ctx, x.core[j], terms[j].get(), (long long)(e * nb), (long long)x.r[j] * nb, x.N[j], x.r[j + 1],
                      t.data(), (j == 0) ? w.data() : ones.data(), R, fp32);
    z.blocks[j] = terms[j].get();
    z.bstride[j] = (long long)(e * nb);
  }
  for (int j = 0; j <= d; ++j) {
    z.s[j] = (j == 0 || j == d) ? 1 : R * x.r[j];
    z.ry[j] = x.r[j];
  }
  tt_round_sketch(ctx, z, *omega, rmax, out, tol, fp32, final);
}

TTView item_view_of(const TTBatchView& x, int b) {
  TTView v{};
  v.d = x.d;
  for (int j = 0; j < 3; ++j) v.N[j] = x.N[j];
  for (int j = 0; j < 4; ++j) v.r[j] = x.r[j];
  for (int j = 0; j < x.d; ++j) v.core[j] = x.core[j] + (size_t)b * x.elems(j);
  return v;
}

}  // namespace lrfg
