// Measured FP64 rates of the device (instrumentation): the roofline denominators of the FP64 kernels.
//
// The library's dense kernels (products, eigensolver, pivoted Cholesky, FP64 FFT passes) are bound by the FP64
// pipe, whose rate is not in the vendor's copy/GEMM peaks.  Two loops measure it on the context's device:
//   - FFMA64: every thread runs 8 independent fused multiply-add chains (enough to cover the FP64 latency),
//     grid = 8 blocks of 256 threads per SM;
//   - DMMA:   every warp issues mma.sync m8n8k4 FP64 (the FP64 tensor-core instruction, 512 flops) on 4
//     independent accumulators.
// Each kernel is launched once to warm up, then timed with CUDA events over one launch of ~10^9..10^10 flops.
#include <cstdio>

#include "ops.cuh"

namespace lrfg {

__global__ void __launch_bounds__(256) fma64_loop_kernel(double* out, int iters, double a, double b) {
  double x0 = threadIdx.x * 1e-9, x1 = x0 + 1e-9, x2 = x0 + 2e-9, x3 = x0 + 3e-9;
  double x4 = x0 + 4e-9, x5 = x0 + 5e-9, x6 = x0 + 6e-9, x7 = x0 + 7e-9;
  for (int i = 0; i < iters; ++i) {
    x0 = fma(x0, a, b); x1 = fma(x1, a, b); x2 = fma(x2, a, b); x3 = fma(x3, a, b);
    x4 = fma(x4, a, b); x5 = fma(x5, a, b); x6 = fma(x6, a, b); x7 = fma(x7, a, b);
  }
  const double s = ((x0 + x1) + (x2 + x3)) + ((x4 + x5) + (x6 + x7));
  if (s == 12345.678) out[blockIdx.x] = s;  // keeps the loop alive; never true for these inputs
}

__global__ void __launch_bounds__(256) dmma_loop_kernel(double* out, int iters) {
  const int lane = threadIdx.x & 31;
  const double av = 1.0 + lane * 1e-12, bv = 1.0 - lane * 1e-12;
  double c[4][2];
#pragma unroll
  for (int k = 0; k < 4; ++k) c[k][0] = c[k][1] = 0.0;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < 4; ++k)
      asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0, %1}, {%2}, {%3}, {%0, %1};\n"
                   : "+d"(c[k][0]), "+d"(c[k][1])
                   : "d"(av), "d"(bv));
  }
  double s = 0.0;
#pragma unroll
  for (int k = 0; k < 4; ++k) s += c[k][0] + c[k][1];
  if (s == 12345.678) out[blockIdx.x] = s;
}

}  // namespace lrfg

using namespace lrfg;

extern "C" lrfg_status lrfg_probe_fp64(lrfg_ctx* ctx, double* fma_tflops, double* dmma_tflops) {
  if (!ctx) return LRFG_EINVAL;
  try {
    LRFG_CUDA(cudaSetDevice(ctx->device));
    LRFG_REQUIRE(fma_tflops && dmma_tflops, "null argument");
    const int nsm = ctx->num_sms > 0 ? ctx->num_sms : 152;
    const int blocks = 8 * nsm, threads = 256;
    DBuf<double> sink(ctx->pool, (size_t)blocks);
    cudaEvent_t e0 = take_event(ctx), e1 = take_event(ctx);
    float ms = 0.0f;
    // FFMA64: 8 chains x 2 flops per iteration per thread
    const int it_fma = 4096;
    fma64_loop_kernel<<<blocks, threads, 0, ctx->stream>>>(sink.get(), 64, 0.999999, 1e-7);
    LRFG_CHECK_LAUNCH();
    LRFG_CUDA(cudaEventRecord(e0, ctx->stream));
    fma64_loop_kernel<<<blocks, threads, 0, ctx->stream>>>(sink.get(), it_fma, 0.999999, 1e-7);
    LRFG_CHECK_LAUNCH();
    LRFG_CUDA(cudaEventRecord(e1, ctx->stream));
    LRFG_CUDA(cudaEventSynchronize(e1));
    LRFG_CUDA(cudaEventElapsedTime(&ms, e0, e1));
    *fma_tflops = 16.0 * it_fma * (double)blocks * threads / (ms * 1e-3) / 1e12;
    // DMMA: 4 accumulators x 512 flops per iteration per warp
    const int it_mma = 1024;
    dmma_loop_kernel<<<blocks, threads, 0, ctx->stream>>>(sink.get(), 16);
    LRFG_CHECK_LAUNCH();
    LRFG_CUDA(cudaEventRecord(e0, ctx->stream));
    dmma_loop_kernel<<<blocks, threads, 0, ctx->stream>>>(sink.get(), it_mma);
    LRFG_CHECK_LAUNCH();
    LRFG_CUDA(cudaEventRecord(e1, ctx->stream));
    LRFG_CUDA(cudaEventSynchronize(e1));
    LRFG_CUDA(cudaEventElapsedTime(&ms, e0, e1));
    *dmma_tflops = 4.0 * 512.0 * it_mma * (double)blocks * (threads / 32) / (ms * 1e-3) / 1e12;
    ctx->event_pool.push_back(e0);
    ctx->event_pool.push_back(e1);
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
