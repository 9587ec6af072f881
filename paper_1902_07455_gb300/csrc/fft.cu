// Mode-wise batched FFTs of fibres (hot-path rows a1 and a2): complex fibres, and real fibres under a
// Fourier multiplier F^{-1} diag(m) F (gradient 2 pi i k, Gaussian exp(-t k^2)).
//
// A fibre is (o, :, i) of an (outer, N, inner) array; a block stages TF whole fibres in shared memory
// with coalesced loads (consecutive threads take consecutive inner indices when inner >= TF, else
// consecutive elements of one fibre), runs the Stockham passes there, and writes back the same way.
// Real fibres are packed two per complex row (x + i y): a real-symmetric multiplier maps it to
// Mx + i My, so one complex transform pair serves two real fibres.
#include <cmath>

#include "ops.cuh"

namespace lrfg {

FftPlan make_plan(int N, int max_radix) {
  FftPlan pl{};
  pl.N = N;
  pl.nst = 0;
  int n = N;
  // register radices first (27, 9 as allowed), then 5, 7, 3, then the remaining primes (generic passes);
  // the order of the passes does not change the transform
  const int pref[] = {27, 9, 5, 7, 3};
  for (int p : pref) {
    if (p > max_radix) continue;
    while (n % p == 0) {
      if (pl.nst >= kMaxStages) fail(LRFG_ENOTSUP, "grid size %d has too many factors", N);
      pl.radix[pl.nst++] = p;
      n /= p;
    }
  }
  for (int p = 11; n > 1; p += 2) {
    while (n % p == 0) {
      if (p > kMaxGenericRadix) fail(LRFG_ENOTSUP, "grid size %d has a prime factor %d > %d", N, p, kMaxGenericRadix);
      if (pl.nst >= kMaxStages) fail(LRFG_ENOTSUP, "grid size %d has too many factors", N);
      pl.radix[pl.nst++] = p;
      n /= p;
    }
  }
  return pl;
}

const Twiddles& twiddles_for(lrfg_ctx* ctx, int N) {
  LRFG_CUDA(ensure_roots(ctx->device));
  auto it = ctx->twiddles.find(N);
  if (it != ctx->twiddles.end()) return it->second;
  std::vector<double2> h(N);
  const double two_pi = 6.283185307179586476925286766559;
  for (int j = 0; j < N; ++j) {
    // reduce the angle to [0, pi/4]-friendly symmetric form for accuracy: exp(-2 pi i j/N)
    double ang = two_pi * (double)j / (double)N;
    h[j] = make_double2(std::cos(ang), -std::sin(ang));
  }
  Twiddles t;
  t.N = N;
  LRFG_CUDA(cudaMalloc(&t.W, sizeof(double2) * N));
  // on the context's stream (ordered before its kernels, also when that stream is non-blocking)
  LRFG_CUDA(cudaMemcpyAsync(t.W, h.data(), sizeof(double2) * N, cudaMemcpyHostToDevice, ctx->stream));
  LRFG_CUDA(cudaStreamSynchronize(ctx->stream));
  return ctx->twiddles.emplace(N, t).first->second;
}

template <>
const double2* twiddle_table<double>(lrfg_ctx* ctx, int N) {
  return twiddles_for(ctx, N).W;
}

template <>
const float2* twiddle_table<float>(lrfg_ctx* ctx, int N) {
  Twiddles& t = const_cast<Twiddles&>(twiddles_for(ctx, N));
  if (!t.Wf) {
    std::vector<float2> h(N);
    const double two_pi = 6.283185307179586476925286766559;
    for (int j = 0; j < N; ++j) {
      double ang = two_pi * (double)j / (double)N;
      h[j] = make_float2((float)std::cos(ang), (float)-std::sin(ang));
    }
    LRFG_CUDA(cudaMalloc(&t.Wf, sizeof(float2) * N));
    LRFG_CUDA(cudaMemcpyAsync(t.Wf, h.data(), sizeof(float2) * N, cudaMemcpyHostToDevice, ctx->stream));
    LRFG_CUDA(cudaStreamSynchronize(ctx->stream));
  }
  return t.Wf;
}

static int tile_fibres(lrfg_ctx* ctx, int N, int rows_per_fibre_pair, size_t* smem_out, size_t elem = sizeof(double2)) {
  // shared memory: twiddles N + 2 buffers of TF rows (+ N multipliers for the operator kernels)
  size_t limit = 100 * 1024;
  if (N > 300) limit = (size_t)std::min(ctx->max_smem_optin, 200 * 1024);
  long long per = 2LL * N * (long long)elem;
  long long fixed = 2LL * N * (long long)elem;
  long long tf = ((long long)limit - fixed) / per;
  if (tf > 64) tf = 64;
  if (tf < 1) tf = 1;
  (void)rows_per_fibre_pair;
  *smem_out = (size_t)(fixed + tf * per);
  return (int)tf;
}

// Fewer rows per tile when the fibres are few (the carriages of a low-rank tensor: r^2 fibres of one length),
// so that the launch still spreads over about `target` blocks instead of leaving most SMs idle.
static int spread_tf(int tf_max, long long nfib, long long target) {
  long long tf = (nfib + 2 * target - 1) / (2 * target);
  return (int)std::max(1LL, std::min((long long)tf_max, tf));
}

// ----------------------------------------------------------------------------------------------------
// complex fibres
// ----------------------------------------------------------------------------------------------------
// frequencies (k1, k2) of fibre i of the axis-0 pass over a d = 2 or 3 half spectrum
template <typename R>
__device__ __forceinline__ void fibre_freqs(const FibreMul<R>& fm, long long i, int& k1, int& k2) {
  if (fm.d == 3) {
    const int i1 = (int)(i / fm.H);
    k1 = freq_of(i1, fm.N1);
    k2 = (int)(i - (long long)i1 * fm.H);
  } else {
    k1 = (int)i;
    k2 = 0;
  }
}

// v * (2 pi i k) * scale, f = c2 k
template <typename V>
__device__ __forceinline__ V times_2pi_ik(V v, typename RealOf<V>::T f) {
  return mkc<V>(-v.y * f, v.x * f);
}

// mode 2 of FibreMul: the divergence term of element (k0, k1, k2) accumulated into *dst
template <typename V>
__device__ __forceinline__ void acc_div_store(const FibreMul<typename RealOf<V>::T>& fm, V* dst, V x, int k0, int k1,
                                              int k2) {
  using R = typename RealOf<V>::T;
  const int ka = fm.alpha == 0 ? k0 : (fm.alpha == 1 ? k1 : k2);
  V r = times_2pi_ik<V>(x, -fm.c2 * (R)ka);
  if (!fm.init) {
    const V o = *dst;
    r.x += o.x;
    r.y += o.y;
  }
  if (fm.precond) {
    const R s = fm.inv_kk[k0 * k0 + k1 * k1 + k2 * k2];
    r.x *= s;
    r.y *= s;
  }
  *dst = r;
}

// OP 0: plain transform; OP 1 and 2: the modes of FibreMul (outer = 1)
template <int SIGN, typename V, int OP>
__global__ void __launch_bounds__(256, 3) fft_fibres_kernel(const V* in, V* out, long long outer, int N, long long inner,
                                                         int TF, FftPlan pl, const V* __restrict__ Wg,
                                                         FibreMul<typename RealOf<V>::T> fm) {
  using R = typename RealOf<V>::T;
  extern __shared__ __align__(16) unsigned char smraw_fib[];
  V* sm = (V*)smraw_fib;
  V* W = sm;
  V* a = sm + 2 * N;
  V* b = a + (size_t)TF * N;
  const long long nfib = outer * inner;
  const long long g0 = (long long)blockIdx.x * TF;
  const int nf = (int)min((long long)TF, nfib - g0);
  const int total = nf * N;
  const bool across = inner >= TF;
  if (across) {
    // thread -> one fibre f of the tile and every step-th element of it: neighbouring threads take
    // neighbouring fibres (contiguous addresses); all index division happens once per thread
    const int step = blockDim.x / nf;
    const int f = threadIdx.x % nf, n0 = threadIdx.x / nf;
    const long long g = g0 + f;
    const long long o = g / inner, i = g - o * inner;
    const V* src = in + (size_t)o * N * (size_t)inner + (size_t)i;
    if (n0 < step)
      for (int n = n0; n < N; n += step) cp_async<sizeof(V)>(a + (size_t)f * N + n, src + (size_t)n * inner);
  } else {
    for (int t = threadIdx.x; t < total; t += blockDim.x) {
      const int f = small_div(t, N, 1.0f / (float)N), n = t - f * N;
      const long long g = g0 + f;
      const long long o = g / inner, i = g - o * inner;
      cp_async<sizeof(V)>(a + (size_t)f * N + n, in + ((size_t)o * N + n) * (size_t)inner + (size_t)i);
    }
  }
  for (int j = threadIdx.x; j < N; j += blockDim.x) W[j] = Wg[j];
  cp_async_wait_all();
  if constexpr (OP == 1) {
    // each thread scales the elements it copied itself (its own copies are complete after the wait)
    if (across) {
      const int step = blockDim.x / nf;
      const int f = threadIdx.x % nf, n0 = threadIdx.x / nf;
      int k1, k2;
      fibre_freqs(fm, g0 + f, k1, k2);
      const R fc = fm.c2 * (R)(fm.alpha == 1 ? k1 : k2);
      if (n0 < step)
        for (int n = n0; n < N; n += step) {
          V* p = a + (size_t)f * N + n;
          *p = times_2pi_ik<V>(*p, fm.alpha == 0 ? fm.c2 * (R)freq_of(n, N) : fc);
        }
    } else {
      for (int t = threadIdx.x; t < total; t += blockDim.x) {
        const int f = small_div(t, N, 1.0f / (float)N), n = t - f * N;
        int k1, k2;
        fibre_freqs(fm, g0 + f, k1, k2);
        const int ka = fm.alpha == 0 ? freq_of(n, N) : (fm.alpha == 1 ? k1 : k2);
        a[t] = times_2pi_ik<V>(a[t], fm.c2 * (R)ka);
      }
    }
  }
  __syncthreads();
  V* res = stockham_rows<SIGN>(a, b, nf, N, pl, (const V*)W);
  if (across) {
    const int step = blockDim.x / nf;
    const int f = threadIdx.x % nf, n0 = threadIdx.x / nf;
    const long long g = g0 + f;
    const long long o = g / inner, i = g - o * inner;
    V* dst = out + (size_t)o * N * (size_t)inner + (size_t)i;
    if constexpr (OP == 2) {
      int k1, k2;
      fibre_freqs(fm, i, k1, k2);
      if (n0 < step)
        for (int n = n0; n < N; n += step)
          acc_div_store<V>(fm, dst + (size_t)n * inner, res[(size_t)f * N + n], freq_of(n, N), k1, k2);
    } else {
      if (n0 < step)
        for (int n = n0; n < N; n += step) dst[(size_t)n * inner] = res[(size_t)f * N + n];
    }
  } else {
    for (int t = threadIdx.x; t < total; t += blockDim.x) {
      const int f = small_div(t, N, 1.0f / (float)N), n = t - f * N;
      const long long g = g0 + f;
      const long long o = g / inner, i = g - o * inner;
      V* dst = out + ((size_t)o * N + n) * (size_t)inner + (size_t)i;
      if constexpr (OP == 2) {
        int k1, k2;
        fibre_freqs(fm, i, k1, k2);
        acc_div_store<V>(fm, dst, res[(size_t)f * N + n], freq_of(n, N), k1, k2);
      } else {
        *dst = res[(size_t)f * N + n];
      }
    }
  }
}

// ----------------------------------------------------------------------------------------------------
// FP32 complex fibres of length N = P1 P2 in two register passes with one trip through shared memory.
// A block takes 32 consecutive fibres, lane = fibre, so every global access of a warp touches 32
// neighbouring inner indices.  The two Stockham stages of the header of fft_device.cuh, written out:
//  pass 1 (radix P1, L = 1; warp w = c < P2): x[c + P2 r], r < P1, loaded straight from global memory,
//         a P1-point DFT in registers, Z[c P1 + q] (q < P1) to shared memory;
//  pass 2 (radix P2, L = P1; f = w, w + P2, ... < P1): Z[r P1 + f] (r < P2) times w_N^{f r}, a P2-point
//         DFT, X[f + P1 q] (q < P2) stored straight to global memory.
// Against the staged kernel this saves the staging round trips through shared memory, one of its
// two buffers and the per-butterfly index arithmetic.  A block reads all of its fibres before it
// writes any, and fibres belong to one block, so in == out is allowed.  OP as in fft_fibres_kernel.
// ----------------------------------------------------------------------------------------------------
// three blocks per SM where their shared memory fits
template <int P1, int P2, int OP>
constexpr int fft2_min_blocks() {
  return P1 * P2 * 32 * 8 * 3 <= 200 * 1024 ? 3 : 2;
}

template <int SIGN, int P1, int P2, int OP>
__global__ void __launch_bounds__(32 * P2, fft2_min_blocks<P1, P2, OP>()) fft2_fibres_kernel(
    const float2* in, float2* out, long long outer, long long inner, const float2* __restrict__ Wg, FibreMul<float> fm) {
  static_assert(P1 % P2 == 0, "pass 2 takes P1 / P2 butterflies per warp");
  constexpr int N = P1 * P2;
  extern __shared__ __align__(16) unsigned char smraw_fib2[];
  float2* Z = (float2*)smraw_fib2;  // [N][32]
  float2* W = Z + N * 32;           // w_N^j, j < N
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const long long g = (long long)blockIdx.x * 32 + lane;
  const bool valid = g < outer * inner;
  long long o = 0, i = 0;
  if (valid) {
    o = g / inner;
    i = g - o * inner;
  }
  int k1 = 0, k2 = 0;
  if constexpr (OP != 0) fibre_freqs(fm, i, k1, k2);
  const size_t base = (size_t)o * N * (size_t)inner + (size_t)i;
  for (int j = threadIdx.x; j < N; j += blockDim.x) W[j] = Wg[j];

  float2 x[P1];
#pragma unroll
  for (int r = 0; r < P1; ++r) x[r] = valid ? in[base + (size_t)(w + P2 * r) * (size_t)inner] : make_float2(0.f, 0.f);
  if constexpr (OP == 1) {
    // k_0 varies along the fibre: multiply before the transform; k_1 and k_2 are constant on it and
    // the product commutes with the transform, so it is taken after pass 2 (fewer live registers)
    if (fm.alpha == 0) {
#pragma unroll
      for (int r = 0; r < P1; ++r) x[r] = times_2pi_ik<float2>(x[r], fm.c2 * (float)freq_of(w + P2 * r, N));
    }
  }
  RegDFT<P1, SIGN, float2>::run(x);
#pragma unroll
  for (int q = 0; q < P1; ++q) Z[(w * P1 + q) * 32 + lane] = x[q];
  __syncthreads();

#pragma unroll
  for (int jb = 0; jb < P1 / P2; ++jb) {
    const int f = w + P2 * jb;
    float2 y[P2], prev[P2];
    if constexpr (OP == 2) {
      // the accumulator's old values, all requested before the transform so that their latencies overlap
#pragma unroll
      for (int q = 0; q < P2; ++q)
        prev[q] = valid && !fm.init ? out[base + (size_t)(f + P1 * q) * (size_t)inner] : make_float2(0.f, 0.f);
    }
#pragma unroll
    for (int r = 0; r < P2; ++r) {
      y[r] = Z[(r * P1 + f) * 32 + lane];
      if (r) y[r] = cmul(y[r], tw<SIGN>((const float2*)W, f * r));
    }
    RegDFT<P2, SIGN, float2>::run(y);
    if (valid) {
#pragma unroll
      for (int q = 0; q < P2; ++q) {
        const int n = f + P1 * q;
        float2* dst = out + base + (size_t)n * (size_t)inner;
        if constexpr (OP == 2) {
          const int k0 = freq_of(n, N);
          const int ka = fm.alpha == 0 ? k0 : (fm.alpha == 1 ? k1 : k2);
          float2 r = times_2pi_ik<float2>(y[q], -fm.c2 * (float)ka);
          if (!fm.init) {
            r.x += prev[q].x;
            r.y += prev[q].y;
          }
          if (fm.precond) {
            // the correctly rounded reciprocal, the value the table holds, without its scattered gather
            const int kk = k0 * k0 + k1 * k1 + k2 * k2;
            const float sc = kk ? __frcp_rn((float)kk) : 0.f;
            r.x *= sc;
            r.y *= sc;
          }
          *dst = r;
        } else if constexpr (OP == 1) {
          *dst = fm.alpha == 0 ? y[q] : times_2pi_ik<float2>(y[q], fm.c2 * (float)(fm.alpha == 1 ? k1 : k2));
        } else {
          *dst = y[q];
        }
      }
    }
  }
}

// N = P1 P2 served by fft2_fibres_kernel (FP32), else 0
static int fft2_split(int N) {
  if (N == 243) return 27;
  if (N == 81) return 9;
  return 0;
}

template <int SIGN, int P1, int P2, int OP>
static void fft2_launch(lrfg_ctx* ctx, const float2* in, float2* out, long long outer, long long inner,
                        const FibreMul<float>& fm, double flops, double bytes) {
  constexpr int N = P1 * P2;
  const size_t smem = sizeof(float2) * (size_t)N * 33;
  const long long blocks = (outer * inner + 31) / 32;
  LRFG_REQUIRE(blocks < (1LL << 31), "too many fibres");
  const float2* W = twiddle_table<float>(ctx, N);
  LRFG_CUDA(raise_smem_limit((const void*)fft2_fibres_kernel<SIGN, P1, P2, OP>, smem));
  LRFG_LAUNCH(ctx, KC_FFT_FIBRES, flops, bytes,
              fft2_fibres_kernel<SIGN, P1, P2, OP><<<(unsigned)blocks, 32 * P2, smem, ctx->stream>>>(in, out, outer,
                                                                                                 inner, W, fm));
}

template <int SIGN, int OP>
static bool fft2_dispatch(lrfg_ctx* ctx, const float2* in, float2* out, long long outer, int N, long long inner,
                          const FibreMul<float>& fm, double flops, double bytes) {
  switch (fft2_split(N)) {
    case 27: fft2_launch<SIGN, 27, 9, OP>(ctx, in, out, outer, inner, fm, flops, bytes); return true;
    case 9: fft2_launch<SIGN, 9, 9, OP>(ctx, in, out, outer, inner, fm, flops, bytes); return true;
    default: return false;
  }
}

template <typename V, int SIGN, int OP>
static bool fft2_try(lrfg_ctx* ctx, const V* in, V* out, long long outer, int N, long long inner,
                     const FibreMul<typename RealOf<V>::T>& fm, double flops, double bytes) {
  if constexpr (sizeof(V) == sizeof(float2)) {
    return fft2_dispatch<SIGN, OP>(ctx, (const float2*)in, (float2*)out, outer, N, inner, fm, flops, bytes);
  } else {
    return false;
  }
}

// Tile for the complex fibre FFT: whole 128-byte segments along the contiguous index (TF * sizeof(V) >=
// 128) and at most 72 KB of shared memory, so that three blocks share an SM and one block's transform
// overlaps the others' loads and stores.
static int tile_complex(lrfg_ctx* ctx, int N, size_t elem, size_t* smem_out) {
  const long long row = (long long)N * (long long)elem;
  long long limit = 72 * 1024;
  const long long tf_min = std::max<long long>(1, 128 / (long long)elem);
  if (2 * row + 2 * tf_min * row > limit) limit = std::min<long long>(ctx->max_smem_optin, 200 * 1024);
  long long tf = (limit - 2 * row) / (2 * row);
  tf = std::max<long long>(1, std::min<long long>(tf, 32));
  if (tf > tf_min) tf = (tf / tf_min) * tf_min;
  *smem_out = (size_t)(2 * row + 2 * tf * row);
  return (int)tf;
}

template <typename V>
void fft_fibres(lrfg_ctx* ctx, const V* in, V* out, long long outer, int N, long long inner, int sign) {
  using R = typename RealOf<V>::T;
  LRFG_REQUIRE(N >= 1 && (N % 2 == 1), "fft length must be odd (got %d)", N);
  LRFG_REQUIRE(outer >= 0 && inner >= 0, "negative batch");
  if (outer == 0 || inner == 0) return;
  FftPlan pl = make_plan(N, plan_radix<V>());
  const V* W = twiddle_table<R>(ctx, N);
  size_t smem;
  int TF = tile_complex(ctx, N, sizeof(V), &smem);
  long long nfib = outer * inner;
  long long blocks = (nfib + TF - 1) / TF;
  LRFG_REQUIRE(blocks < (1LL << 31), "too many fibres");
  const double flops = 5.0 * N * std::log2((double)N) * (double)nfib;   // radix-2-equivalent count
  const double bytes = 2.0 * sizeof(V) * (double)N * (double)nfib;
  const FibreMul<R> none{};
  if (sign < 0 ? fft2_try<V, -1, 0>(ctx, in, out, outer, N, inner, none, flops, bytes)
               : fft2_try<V, 1, 0>(ctx, in, out, outer, N, inner, none, flops, bytes))
    return;
  if (sign < 0) {
    LRFG_CUDA(raise_smem_limit((const void*)fft_fibres_kernel<-1, V, 0>, smem));
    LRFG_LAUNCH(ctx, KC_FFT_FIBRES, flops, bytes,
                fft_fibres_kernel<-1, V, 0><<<(unsigned)blocks, 256, smem, ctx->stream>>>(in, out, outer, N, inner, TF,
                                                                                         pl, W, none));
  } else {
    LRFG_CUDA(raise_smem_limit((const void*)fft_fibres_kernel<1, V, 0>, smem));
    LRFG_LAUNCH(ctx, KC_FFT_FIBRES, flops, bytes,
                fft_fibres_kernel<1, V, 0><<<(unsigned)blocks, 256, smem, ctx->stream>>>(in, out, outer, N, inner, TF,
                                                                                        pl, W, none));
  }
}
template void fft_fibres<double2>(lrfg_ctx*, const double2*, double2*, long long, int, long long, int);
template void fft_fibres<float2>(lrfg_ctx*, const float2*, float2*, long long, int, long long, int);

template <typename V>
void fft_fibres_mul(lrfg_ctx* ctx, const V* in, V* out, int N0, long long inner, const FibreMul<typename RealOf<V>::T>& fm) {
  using R = typename RealOf<V>::T;
  LRFG_REQUIRE(N0 >= 1 && (N0 % 2 == 1), "fft length must be odd (got %d)", N0);
  LRFG_REQUIRE(fm.mode == 1 || fm.mode == 2, "multiplier mode %d", fm.mode);
  LRFG_REQUIRE(fm.d == 2 || fm.d == 3, "d = %d", fm.d);
  LRFG_REQUIRE(inner == (long long)(fm.d == 3 ? fm.N1 : 1) * fm.H, "axis-0 fibres of a half spectrum expected");
  LRFG_REQUIRE(fm.mode == 1 || in != out, "the accumulator cannot hold the input");
  LRFG_REQUIRE(!(fm.mode == 2 && fm.precond) || fm.inv_kk, "reciprocal table missing");
  if (inner == 0) return;
  FftPlan pl = make_plan(N0, plan_radix<V>());
  const V* W = twiddle_table<R>(ctx, N0);
  size_t smem;
  int TF = tile_complex(ctx, N0, sizeof(V), &smem);
  long long blocks = (inner + TF - 1) / TF;
  LRFG_REQUIRE(blocks < (1LL << 31), "too many fibres");
  const double n_el = (double)N0 * (double)inner;
  const double flops = 5.0 * N0 * std::log2((double)N0) * (double)inner + (fm.mode == 1 ? 2.0 : 4.0) * n_el;
  const double bytes = (fm.mode == 1 || fm.init ? 2.0 : 3.0) * sizeof(V) * n_el;
  if (fm.mode == 1 ? fft2_try<V, 1, 1>(ctx, in, out, 1, N0, inner, fm, flops, bytes)
                   : fft2_try<V, -1, 2>(ctx, in, out, 1, N0, inner, fm, flops, bytes))
    return;
  if (fm.mode == 1) {
    LRFG_CUDA(raise_smem_limit((const void*)fft_fibres_kernel<1, V, 1>, smem));
    LRFG_LAUNCH(ctx, KC_FFT_FIBRES, flops, bytes,
                fft_fibres_kernel<1, V, 1><<<(unsigned)blocks, 256, smem, ctx->stream>>>(in, out, 1, N0, inner, TF, pl,
                                                                                        W, fm));
  } else {
    LRFG_CUDA(raise_smem_limit((const void*)fft_fibres_kernel<-1, V, 2>, smem));
    LRFG_LAUNCH(ctx, KC_FFT_FIBRES, flops, bytes,
                fft_fibres_kernel<-1, V, 2><<<(unsigned)blocks, 256, smem, ctx->stream>>>(in, out, 1, N0, inner, TF, pl,
                                                                                         W, fm));
  }
}
template void fft_fibres_mul<double2>(lrfg_ctx*, const double2*, double2*, int, long long, const FibreMul<double>&);
template void fft_fibres_mul<float2>(lrfg_ctx*, const float2*, float2*, int, long long, const FibreMul<float>&);

// ----------------------------------------------------------------------------------------------------
// real fibres under a multiplier: rows hold fibre f (real part) and fibre f + TF (imaginary part)
// ----------------------------------------------------------------------------------------------------
__device__ __forceinline__ double2 multiplier(int kind, int k, double param) {
  if (kind == LRFG_MUL_DERIV) return make_double2(0.0, 6.283185307179586476925286766559 * (double)k);
  if (kind == LRFG_MUL_GAUSS) return make_double2(exp(-param * (double)k * (double)k), 0.0);
  return make_double2(1.0, 0.0);
}

// V = double2 (FP64 transforms) or float2 (FP32 transforms of FP64 data: the mixed-precision path); the fibres
// are read and written in FP64 either way.
template <typename V>
__global__ void __launch_bounds__(256) fibre_op_kernel(const double* in, double* out, long long outer,
                                                       int N, long long inner, int TF, FftPlan pl,
                                                       const V* __restrict__ Wg, int kind, double param,
                                                       double scale) {
  using R = typename RealOf<V>::T;
  extern __shared__ __align__(16) unsigned char smraw_op[];
  V* sm = (V*)smraw_op;
  V* W = sm;
  V* M = sm + N;
  V* a = sm + 2 * N;
  V* b = a + (size_t)TF * N;
  for (int j = threadIdx.x; j < N; j += blockDim.x) {
    W[j] = Wg[j];
    const double2 m = multiplier(kind, freq_of(j, N), param);
    M[j] = mkc<V>((R)m.x, (R)m.y);
  }
  const long long nfib = outer * inner;
  const long long g0 = (long long)blockIdx.x * (2LL * TF);
  const int nf = (int)min(2LL * TF, nfib - g0);   // real fibres in this tile
  const int rows = min(nf, TF);
  for (int t = threadIdx.x; t < rows * N; t += blockDim.x) a[t] = mkc<V>((R)0, (R)0);
  __syncthreads();
  const int total = nf * N;
  const bool across = inner >= 2 * TF;
  for (int t = threadIdx.x; t < total; t += blockDim.x) {
    int f, n;
    if (across) { f = t % nf; n = t / nf; } else { f = t / N; n = t % N; }
    long long g = g0 + f;
    long long o = g / inner, i = g - o * inner;
    const R v = (R)in[((size_t)o * N + n) * (size_t)inner + (size_t)i];
    if (f < TF) a[(size_t)f * N + n].x = v; else a[(size_t)(f - TF) * N + n].y = v;
  }
  __syncthreads();
  V* res = stockham_rows<-1>(a, b, rows, N, pl, W);
  V* other = (res == a) ? b : a;
  for (int t = threadIdx.x; t < rows * N; t += blockDim.x) {
    int n = t % N;
    res[t] = cmul(res[t], M[n]);
  }
  __syncthreads();
  res = stockham_rows<1>(res, other, rows, N, pl, W);
  const double s = scale / (double)N;
  for (int t = threadIdx.x; t < total; t += blockDim.x) {
    int f, n;
    if (across) { f = t % nf; n = t / nf; } else { f = t / N; n = t % N; }
    long long g = g0 + f;
    long long o = g / inner, i = g - o * inner;
    V v = (f < TF) ? res[(size_t)f * N + n] : res[(size_t)(f - TF) * N + n];
    out[((size_t)o * N + n) * (size_t)inner + (size_t)i] = s * (double)((f < TF) ? v.x : v.y);
  }
}

template <typename V>
static void fibre_operator_t(lrfg_ctx* ctx, const double* in, double* out, long long outer, int N, long long inner,
                             int kind, double param, double scale) {
  FftPlan pl = make_plan(N, plan_radix<V>());
  const V* W = twiddle_table<typename RealOf<V>::T>(ctx, N);
  size_t smem;
  int TF = tile_fibres(ctx, N, 2, &smem, sizeof(V));
  long long nfib = outer * inner;
  const int nsm = ctx->num_sms > 0 ? ctx->num_sms : 152;
  TF = spread_tf(TF, nfib, 2LL * nsm);
  smem = (size_t)(2LL * N * sizeof(V) + (long long)TF * 2LL * N * sizeof(V));
  long long blocks = (nfib + 2LL * TF - 1) / (2LL * TF);
  LRFG_REQUIRE(blocks < (1LL << 31), "too many fibres");
  LRFG_CUDA(raise_smem_limit((const void*)fibre_op_kernel<V>, smem));
  // two complex transforms per pair of real fibres
  const double flops = 5.0 * N * std::log2((double)N) * (double)nfib;
  const double bytes = 2.0 * sizeof(double) * (double)N * (double)nfib;
  LRFG_LAUNCH(ctx, KC_FIBRE_OP, flops, bytes,
              fibre_op_kernel<V><<<(unsigned)blocks, 256, smem, ctx->stream>>>(in, out, outer, N, inner, TF, pl, W,
                                                                                kind, param, scale));
}

void fibre_operator(lrfg_ctx* ctx, const double* in, double* out, long long outer, int N, long long inner,
                    int kind, double param, double scale, bool fp32) {
  LRFG_REQUIRE(N >= 1 && (N % 2 == 1), "fibre length must be odd (got %d)", N);
  LRFG_REQUIRE(kind == LRFG_MUL_IDENTITY || kind == LRFG_MUL_DERIV || kind == LRFG_MUL_GAUSS,
               "unknown multiplier %d", kind);
  if (outer == 0 || inner == 0) return;
  if (fp32) fibre_operator_t<float2>(ctx, in, out, outer, N, inner, kind, param, scale);
  else fibre_operator_t<double2>(ctx, in, out, outer, N, inner, kind, param, scale);
}

// Many Gaussian multipliers of one input: the forward transform is shared, each term m gets its own
// multiply + inverse transform and is written to out + m * out_stride.
template <typename V>
__global__ void __launch_bounds__(256) fibre_gauss_multi_kernel(const double* __restrict__ in, double* out,
                                                                long long out_stride, long long outer, int N,
                                                                long long inner, int TF, FftPlan pl,
                                                                const V* __restrict__ Wg,
                                                                const double* __restrict__ tm,
                                                                const double* __restrict__ sc, int nm, int mper) {
  using R = typename RealOf<V>::T;
  extern __shared__ __align__(16) unsigned char smraw_gm[];
  V* sm = (V*)smraw_gm;
  V* W = sm;
  V* spec = sm + N;              // TF rows: the shared forward spectrum
  V* a = spec + (size_t)TF * N;  // TF rows
  V* b = a + (size_t)TF * N;     // TF rows
  for (int j = threadIdx.x; j < N; j += blockDim.x) W[j] = Wg[j];
  const long long nfib = outer * inner;
  const long long g0 = (long long)blockIdx.x * (2LL * TF);
  const int nf = (int)min(2LL * TF, nfib - g0);
  const int rows = min(nf, TF);
  for (int t = threadIdx.x; t < rows * N; t += blockDim.x) a[t] = mkc<V>((R)0, (R)0);
  __syncthreads();
  const int total = nf * N;
  const bool across = inner >= 2 * TF;
  for (int t = threadIdx.x; t < total; t += blockDim.x) {
    int f, n;
    if (across) { f = t % nf; n = t / nf; } else { f = t / N; n = t % N; }
    long long g = g0 + f;
    long long o = g / inner, i = g - o * inner;
    const R v = (R)in[((size_t)o * N + n) * (size_t)inner + (size_t)i];
    if (f < TF) a[(size_t)f * N + n].x = v; else a[(size_t)(f - TF) * N + n].y = v;
  }
  __syncthreads();
  V* res = stockham_rows<-1>(a, b, rows, N, pl, W);
  for (int t = threadIdx.x; t < rows * N; t += blockDim.x) spec[t] = res[t];
  __syncthreads();
  const int m_end = min(nm, (int)(blockIdx.y + 1) * mper);
  for (int m = blockIdx.y * mper; m < m_end; ++m) {
    const double t_m = tm[m];
    for (int t = threadIdx.x; t < rows * N; t += blockDim.x) {
      int k = freq_of(t % N, N);
      a[t] = cscale(spec[t], (R)exp(-t_m * (double)k * (double)k));
    }
    __syncthreads();
    V* r2 = stockham_rows<1>(a, b, rows, N, pl, W);
    const double s = sc[m] / (double)N;
    double* o_m = out + (size_t)m * (size_t)out_stride;
    for (int t = threadIdx.x; t < total; t += blockDim.x) {
      int f, n;
      if (across) { f = t % nf; n = t / nf; } else { f = t / N; n = t % N; }
      long long g = g0 + f;
      long long o = g / inner, i = g - o * inner;
      V v = (f < TF) ? r2[(size_t)f * N + n] : r2[(size_t)(f - TF) * N + n];
      o_m[((size_t)o * N + n) * (size_t)inner + (size_t)i] = s * (double)((f < TF) ? v.x : v.y);
    }
    __syncthreads();
  }
}

template <typename V>
static void fibre_gauss_multi_t(lrfg_ctx* ctx, const double* in, double* out, long long out_stride, long long outer,
                                int N, long long inner, const double* t, const double* scale, int nm) {
  FftPlan pl = make_plan(N, plan_radix<V>());
  const V* Wt = twiddle_table<typename RealOf<V>::T>(ctx, N);
  size_t limit = 100 * 1024;
  if (N > 300) limit = (size_t)std::min(ctx->max_smem_optin, 200 * 1024);
  long long per = 3LL * N * (long long)sizeof(V);
  long long tf = ((long long)limit - (long long)N * (long long)sizeof(V)) / per;
  if (tf > 64) tf = 64;
  if (tf < 1) tf = 1;
  // few fibres (low-rank carriages): smaller tiles, and the terms split over grid.y (each block redoes the
  // shared forward transform of its tile), so that the launch covers the SMs
  const int nsm = ctx->num_sms > 0 ? ctx->num_sms : 152;
  const long long nfib0 = outer * inner;
  tf = spread_tf((int)tf, nfib0, 2LL * nsm);
  const long long bx = (nfib0 + 2 * tf - 1) / (2 * tf);
  const int mchunks = (int)std::max(1LL, std::min((long long)nm, (4LL * nsm + bx - 1) / bx));
  const int mper = (nm + mchunks - 1) / mchunks;
  size_t smem = (size_t)(N * sizeof(V) + tf * per);
  // device copies of the node and scale tables
  DBuf<double> dt(ctx->pool, nm), ds(ctx->pool, nm);
  LRFG_CUDA(cudaMemcpyAsync(dt.get(), t, sizeof(double) * nm, cudaMemcpyHostToDevice, ctx->stream));
  LRFG_CUDA(cudaMemcpyAsync(ds.get(), scale, sizeof(double) * nm, cudaMemcpyHostToDevice, ctx->stream));
  long long nfib = outer * inner;
  long long blocks = (nfib + 2 * tf - 1) / (2 * tf);
  LRFG_REQUIRE(blocks < (1LL << 31), "too many fibres");
  LRFG_CUDA(raise_smem_limit((const void*)fibre_gauss_multi_kernel<V>, smem));
  // one forward and nm inverse complex transforms per pair of real fibres (algorithmic count)
  const double flops = 2.5 * N * std::log2((double)N) * (double)nfib * (1.0 + nm);
  const double bytes = sizeof(double) * (double)N * (double)nfib * (1.0 + nm);
  const int mgrid = (nm + mper - 1) / mper;
  LRFG_LAUNCH(ctx, KC_GAUSS_MULTI, flops, bytes,
              fibre_gauss_multi_kernel<V><<<dim3((unsigned)blocks, (unsigned)mgrid), 256, smem, ctx->stream>>>(
                  in, out, out_stride, outer, N, inner, (int)tf, pl, Wt, dt.get(), ds.get(), nm, mper));
  // the pool hands these blocks out again only to later work on the same stream
}

void fibre_gauss_multi(lrfg_ctx* ctx, const double* in, double* out, long long out_stride, long long outer,
                       int N, long long inner, const double* t, const double* scale, int nm, bool fp32) {
  LRFG_REQUIRE(N >= 1 && (N % 2 == 1), "fibre length must be odd (got %d)", N);
  if (outer == 0 || inner == 0 || nm == 0) return;
  if (fp32) fibre_gauss_multi_t<float2>(ctx, in, out, out_stride, outer, N, inner, t, scale, nm);
  else fibre_gauss_multi_t<double2>(ctx, in, out, out_stride, outer, N, inner, t, scale, nm);
}


// ------------------------------------------------------------------------------------------------
// Ga mode maps (Sec. 2.2.3) on real fibres: forward transform on n_in points, a spectral map to n_out
// points, inverse transform; the maps are exact in exact arithmetic (zero padding, truncation, periodic
// extension with the cell sinc), the transforms the library's fibre FFTs.
// ------------------------------------------------------------------------------------------------
__global__ void real_to_complex_kernel(const double* __restrict__ in, double2* __restrict__ out, long long n) {
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x)
    out[t] = make_double2(in[t], 0.0);
}

__global__ void complex_to_real_kernel(const double2* __restrict__ in, double* __restrict__ out, long long n) {
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x)
    out[t] = in[t].x;
}

__device__ __forceinline__ int freq_rep(int i, int n) { return i <= (n - 1) / 2 ? i : i - n; }

// out[o][m][i] = weight(m) * in[o][src(m)][i] over (outer, n_out, inner)
__global__ void ga_spectral_map_kernel(const double2* __restrict__ in, double2* __restrict__ out, long long outer,
                                       int n_in, long long inner, int n_out, int mode, int n_grid) {
  const long long total = outer * n_out * inner;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total; t += (long long)gridDim.x * blockDim.x) {
    const long long i = t % inner;
    const long long q = t / inner;
    const int m = (int)(q % n_out);
    const long long o = q / n_out;
    const int f = freq_rep(m, n_out);
    int src = -1;
    double wgt = 0.0;
    if (mode == GA_UP) {  // zero padding, F_N = Phi_N / N
      if (abs(f) <= (n_in - 1) / 2) { src = f < 0 ? f + n_in : f; wgt = 1.0 / n_in; }
    } else if (mode == GA_DOWN) {  // the frequencies of the small grid, F_M = Phi_M / M
      src = f < 0 ? f + n_in : f;
      wgt = 1.0 / n_in;
    } else {  // periodic extension times the cell sinc of the pixel grid n_grid, and M^-1
      src = ((f % n_in) + n_in) % n_in;
      const double x = 3.141592653589793238462643383279502884 * (double)f;
      const double s = f == 0 ? 1.0 / n_grid : sin(x / (double)n_grid) / x;
      wgt = s / n_out;
    }
    double2 v = make_double2(0.0, 0.0);
    if (src >= 0) {
      const double2 u = in[(o * n_in + src) * inner + i];
      v = make_double2(wgt * u.x, wgt * u.y);
    }
    out[t] = v;
  }
}

void ga_resample(lrfg_ctx* ctx, const double* in, double* out, long long outer, int n_in, long long inner, int n_out,
                 int mode) {
  const long long nin = outer * n_in * inner, nout = outer * n_out * inner;
  if (nin == 0 || nout == 0) return;
  const unsigned gin = (unsigned)std::min<long long>((nin + 255) / 256, 8LL * ctx->num_sms);
  const unsigned gout = (unsigned)std::min<long long>((nout + 255) / 256, 8LL * ctx->num_sms);
  DBuf<double2> a(ctx->pool, (size_t)nin), b(ctx->pool, (size_t)nout);
  LRFG_LAUNCH(ctx, KC_TT_MISC, 0.0, 24.0 * nin, real_to_complex_kernel<<<gin, 256, 0, ctx->stream>>>(in, a.get(), nin));
  fft_fibres<double2>(ctx, a.get(), a.get(), outer, n_in, inner, -1);
  LRFG_LAUNCH(ctx, KC_TT_MISC, 2.0 * nout, 32.0 * nout,
              ga_spectral_map_kernel<<<gout, 256, 0, ctx->stream>>>(a.get(), b.get(), outer, n_in, inner, n_out, mode,
                                                                    mode == GA_EXTEND ? n_in : 0));
  fft_fibres<double2>(ctx, b.get(), b.get(), outer, n_out, inner, 1);
  LRFG_LAUNCH(ctx, KC_TT_MISC, 0.0, 24.0 * nout,
              complex_to_real_kernel<<<gout, 256, 0, ctx->stream>>>(b.get(), out, nout));
}

}  // namespace lrfg
