// Batched odd-length complex FFTs of fibres staged in shared memory (FP64 double2 or FP32 float2).
//
// Mixed-radix Stockham autosort, decimation in time.  After the stages with radices p_0..p_{s-1}
// (L = p_0...p_{s-1}), row entry c*L + f holds the length-L DFT (frequency f) of the subsequence
// x[c + (N/L) t], t = 0..L-1.  A radix-p stage with m' = N/(L p) combines p such subsequences:
//   Z'[c'][f + L q] = sum_r w_p^{q r} ( w_{Lp}^{f r} Z[c' + m' r][f] ),   q, r = 0..p-1,
// with w_M = exp(sign 2 pi i / M).  It starts from the natural order (L = 1) and ends in natural
// order (L = N), so no digit reversal is needed.  Inter-pass twiddles come from one table
// W[j] = exp(-2 pi i j / N) (w_{Lp}^{f r} = W[f r m']).  A pass of composite radix p (9, 27) does its
// p-point DFT in registers by Cooley-Tukey splitting p = P Q (index n = n1 + P n2, k = Q k1 + k2):
//   X[Q k1 + k2] = sum_{n1} w_P^{n1 k1} w_p^{n1 k2} sum_{n2} x[n1 + P n2] w_Q^{n2 k2},
// with the roots of unity of each radix in constant memory (compile-time indices, so they are
// operands of the arithmetic instructions); fewer passes through shared memory and far fewer
// instructions per point than radix-3 passes.
#pragma once

#include <cuda_runtime.h>

#include <cmath>
#include <mutex>

namespace lrfg {

constexpr int kMaxStages = 24;
constexpr int kMaxGenericRadix = 31;

// roots of unity exp(-2 pi i j / p) of the register radices, concatenated (filled once per device)
constexpr int kRootOff3 = 0, kRootOff5 = 3, kRootOff7 = 8, kRootOff9 = 15, kRootOff27 = 24, kRootCount = 51;
__constant__ double2 c_roots_d[kRootCount];
__constant__ float2 c_roots_f[kRootCount];

// Fills this translation unit's root tables on the current device (once per device); returns the CUDA
// status of the copies.
static inline cudaError_t ensure_roots(int device) {
  static std::mutex mu;
  static unsigned long long done = 0;  // one bit per device
  std::lock_guard<std::mutex> lock(mu);
  if (device >= 0 && device < 64 && (done >> device & 1ULL)) return cudaSuccess;
  double2 hd[kRootCount];
  float2 hf[kRootCount];
  const int radix[5] = {3, 5, 7, 9, 27}, off[5] = {kRootOff3, kRootOff5, kRootOff7, kRootOff9, kRootOff27};
  const double two_pi = 6.283185307179586476925286766559;
  for (int q = 0; q < 5; ++q)
    for (int j = 0; j < radix[q]; ++j) {
      const double ang = two_pi * (double)j / (double)radix[q];
      hd[off[q] + j] = make_double2(std::cos(ang), -std::sin(ang));
      hf[off[q] + j] = make_float2((float)std::cos(ang), (float)-std::sin(ang));
    }
  cudaError_t e = cudaMemcpyToSymbol(c_roots_d, hd, sizeof(hd));
  if (e == cudaSuccess) e = cudaMemcpyToSymbol(c_roots_f, hf, sizeof(hf));
  // complete before kernels on any stream (non-blocking ones included) read the tables
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  if (e == cudaSuccess && device >= 0 && device < 64) done |= 1ULL << device;
  return e;
}

struct FftPlan {
  int N;
  int nst;
  int radix[kMaxStages];
};

// complex vector type of a real type
template <typename R> struct CplxOf;
template <> struct CplxOf<double> { using T = double2; };
template <> struct CplxOf<float> { using T = float2; };
template <typename V> struct RealOf;
template <> struct RealOf<double2> { using T = double; };
template <> struct RealOf<float2> { using T = float; };

template <typename V>
__device__ __forceinline__ V mkc(typename RealOf<V>::T x, typename RealOf<V>::T y) {
  V v;
  v.x = x;
  v.y = y;
  return v;
}
template <typename V>
__device__ __forceinline__ V cmul(V a, V b) {
  return mkc<V>(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
template <typename V>
__device__ __forceinline__ V cadd(V a, V b) { return mkc<V>(a.x + b.x, a.y + b.y); }
template <typename V>
__device__ __forceinline__ V csub(V a, V b) { return mkc<V>(a.x - b.x, a.y - b.y); }
template <typename V>
__device__ __forceinline__ V cscale(V a, typename RealOf<V>::T s) { return mkc<V>(a.x * s, a.y * s); }
// i * s * a
template <typename V>
__device__ __forceinline__ V cimul(V a, typename RealOf<V>::T s) { return mkc<V>(-a.y * s, a.x * s); }

// twiddle W[j]^(-sign): forward (sign -1) uses W, inverse (sign +1) its conjugate
template <int SIGN, typename V>
__device__ __forceinline__ V tw(const V* W, int j) {
  V w = W[j];
  if (SIGN > 0) w.y = -w.y;
  return w;
}

// One radix-p butterfly: inputs Z[c + m' r][f] (row offset (c + m' r) L + f), outputs Z'[c][f + L q].
template <int SIGN, typename V>
__device__ __forceinline__ void butterfly(int p, const V* __restrict__ in, V* __restrict__ out, int c, int f, int L,
                                          int mp, int N, const V* W) {
  using R = typename RealOf<V>::T;
  if (p == 3) {
    V x0 = in[c * L + f];
    V x1 = in[(c + mp) * L + f];
    V x2 = in[(c + 2 * mp) * L + f];
    if (f) {
      x1 = cmul(x1, tw<SIGN>(W, f * mp));
      x2 = cmul(x2, tw<SIGN>(W, 2 * f * mp));
    }
    const R s = (R)0.86602540378443864676;  // sin(2 pi / 3) = sqrt(3)/2
    V t1 = cadd(x1, x2), t2 = csub(x1, x2);
    V m = csub(x0, cscale(t1, (R)0.5));
    V u = cimul(t2, (R)SIGN * s);
    V* o = out + c * L * 3 + f;
    o[0] = cadd(x0, t1);
    o[L] = cadd(m, u);
    o[2 * L] = csub(m, u);
  } else if (p == 5) {
    V x0 = in[c * L + f];
    V x1 = in[(c + mp) * L + f];
    V x2 = in[(c + 2 * mp) * L + f];
    V x3 = in[(c + 3 * mp) * L + f];
    V x4 = in[(c + 4 * mp) * L + f];
    if (f) {
      int j = f * mp;
      x1 = cmul(x1, tw<SIGN>(W, j));
      x2 = cmul(x2, tw<SIGN>(W, 2 * j));
      x3 = cmul(x3, tw<SIGN>(W, 3 * j));
      x4 = cmul(x4, tw<SIGN>(W, 4 * j));
    }
    // cos/sin of 2 pi/5 and 4 pi/5: (sqrt5-1)/4, -(sqrt5+1)/4, sqrt((5+sqrt5)/8), sqrt((5-sqrt5)/8)
    const R c1 = (R)0.30901699437494742410, c2 = (R)-0.80901699437494742410;
    const R s1 = (R)0.95105651629515357212, s2 = (R)0.58778525229247312917;
    V a1 = cadd(x1, x4), b1 = csub(x1, x4), a2 = cadd(x2, x3), b2 = csub(x2, x3);
    V m1 = cadd(x0, cadd(cscale(a1, c1), cscale(a2, c2)));
    V m2 = cadd(x0, cadd(cscale(a1, c2), cscale(a2, c1)));
    V n1 = cimul(cadd(cscale(b1, s1), cscale(b2, s2)), (R)SIGN);
    V n2 = cimul(csub(cscale(b1, s2), cscale(b2, s1)), (R)SIGN);
    V* o = out + c * L * 5 + f;
    o[0] = cadd(x0, cadd(a1, a2));
    o[L] = cadd(m1, n1);
    o[2 * L] = cadd(m2, n2);
    o[3 * L] = csub(m2, n2);
    o[4 * L] = csub(m1, n1);
  } else {
    // generic prime radix (7, 11, ...): direct length-p DFT with table twiddles
    V x[kMaxGenericRadix];
    for (int r = 0; r < p; ++r) {
      V v = in[(c + r * mp) * L + f];
      if (r && f) v = cmul(v, tw<SIGN>(W, f * r * mp));
      x[r] = v;
    }
    const int step = N / p;
    V* o = out + c * L * p + f;
    for (int q = 0; q < p; ++q) {
      V acc = x[0];
      for (int r = 1; r < p; ++r) acc = cadd(acc, cmul(x[r], tw<SIGN>(W, ((q * r) % p) * step)));
      o[q * L] = acc;
    }
  }
}

// Transform `nf` rows of length pl.N (row stride ld) held in `a`, using `b` as scratch.  All threads
// of the block take part; returns the buffer that holds the result (a or b).  Ends with a barrier.
template <int P>
struct RootOff;
template <> struct RootOff<3> { static constexpr int v = kRootOff3; };
template <> struct RootOff<5> { static constexpr int v = kRootOff5; };
template <> struct RootOff<7> { static constexpr int v = kRootOff7; };
template <> struct RootOff<9> { static constexpr int v = kRootOff9; };
template <> struct RootOff<27> { static constexpr int v = kRootOff27; };

// w_P^j (forward: exp(-2 pi i j / P), inverse: its conjugate); j a compile-time constant after unrolling
template <int P, int SIGN, typename V>
__device__ __forceinline__ V root(int j) {
  V w;
  if constexpr (sizeof(V) == sizeof(double2)) {
    const double2 t = c_roots_d[RootOff<P>::v + j % P];
    w.x = t.x;
    w.y = t.y;
  } else {
    const float2 t = c_roots_f[RootOff<P>::v + j % P];
    w.x = t.x;
    w.y = t.y;
  }
  if (SIGN > 0) w.y = -w.y;
  return w;
}

template <int P, int SIGN, typename V>
struct RegDFT;

template <int SIGN, typename V>
struct RegDFT<3, SIGN, V> {
  static __device__ __forceinline__ void run(V* x) {
    using R = typename RealOf<V>::T;
    const R s = (R)0.86602540378443864676;  // sin(2 pi / 3)
    V t1 = cadd(x[1], x[2]), t2 = csub(x[1], x[2]);
    V m = csub(x[0], cscale(t1, (R)0.5));
    V u = cimul(t2, (R)SIGN * s);
    x[0] = cadd(x[0], t1);
    x[1] = cadd(m, u);
    x[2] = csub(m, u);
  }
};

template <int SIGN, typename V>
struct RegDFT<5, SIGN, V> {
  static __device__ __forceinline__ void run(V* x) {
    using R = typename RealOf<V>::T;
    const R c1 = (R)0.30901699437494742410, c2 = (R)-0.80901699437494742410;
    const R s1 = (R)0.95105651629515357212, s2 = (R)0.58778525229247312917;
    V a1 = cadd(x[1], x[4]), b1 = csub(x[1], x[4]), a2 = cadd(x[2], x[3]), b2 = csub(x[2], x[3]);
    V m1 = cadd(x[0], cadd(cscale(a1, c1), cscale(a2, c2)));
    V m2 = cadd(x[0], cadd(cscale(a1, c2), cscale(a2, c1)));
    V n1 = cimul(cadd(cscale(b1, s1), cscale(b2, s2)), (R)SIGN);
    V n2 = cimul(csub(cscale(b1, s2), cscale(b2, s1)), (R)SIGN);
    x[0] = cadd(x[0], cadd(a1, a2));
    x[1] = cadd(m1, n1);
    x[2] = cadd(m2, n2);
    x[3] = csub(m2, n2);
    x[4] = csub(m1, n1);
  }
};

template <int SIGN, typename V>
struct RegDFT<7, SIGN, V> {  // direct sum
  static __device__ __forceinline__ void run(V* x) {
    V y[7];
#pragma unroll
    for (int q = 0; q < 7; ++q) {
      V acc = x[0];
#pragma unroll
      for (int r = 1; r < 7; ++r) acc = cadd(acc, cmul(x[r], root<7, SIGN, V>(q * r)));
      y[q] = acc;
    }
#pragma unroll
    for (int q = 0; q < 7; ++q) x[q] = y[q];
  }
};

// p = P Q in registers (see the header comment)
template <int P, int Q, int SIGN, typename V>
__device__ __forceinline__ void reg_dft_split(V* x) {
  constexpr int p = P * Q;
  V y[P][Q];
#pragma unroll
  for (int n1 = 0; n1 < P; ++n1) {
    V t[Q];
#pragma unroll
    for (int n2 = 0; n2 < Q; ++n2) t[n2] = x[n1 + P * n2];
    RegDFT<Q, SIGN, V>::run(t);
#pragma unroll
    for (int k2 = 0; k2 < Q; ++k2) y[n1][k2] = (n1 && k2) ? cmul(t[k2], root<p, SIGN, V>(n1 * k2)) : t[k2];
  }
#pragma unroll
  for (int k2 = 0; k2 < Q; ++k2) {
    V t[P];
#pragma unroll
    for (int n1 = 0; n1 < P; ++n1) t[n1] = y[n1][k2];
    RegDFT<P, SIGN, V>::run(t);
#pragma unroll
    for (int k1 = 0; k1 < P; ++k1) x[Q * k1 + k2] = t[k1];
  }
}

template <int SIGN, typename V>
struct RegDFT<9, SIGN, V> {
  static __device__ __forceinline__ void run(V* x) { reg_dft_split<3, 3, SIGN, V>(x); }
};
template <int SIGN, typename V>
struct RegDFT<27, SIGN, V> {
  static __device__ __forceinline__ void run(V* x) { reg_dft_split<3, 9, SIGN, V>(x); }
};

// x / d for 0 <= x < 2^22 and 1 <= d < 2^22 from a float reciprocal, corrected to the exact quotient
// (cheaper than the integer division sequence in the per-butterfly index arithmetic)
__device__ __forceinline__ int small_div(int x, int d, float inv) {
  int q = __float2int_rz((float)x * inv);
  const int r = x - q * d;
  if (r < 0) --q;
  else if (r >= d) ++q;
  return q;
}

// One Stockham pass of register radix P over nf rows (row stride ld) from a into b.
template <int P, int SIGN, typename V>
__device__ __forceinline__ void stockham_pass(const V* __restrict__ a, V* __restrict__ b, int nf, int ld, int N,
                                              int L, const V* W) {
  const int mp = N / (L * P);
  const int nb = N / P;
  const int total = nb * nf;
  const float inv_nb = 1.0f / (float)nb, inv_L = 1.0f / (float)L;
  for (int t = threadIdx.x; t < total; t += blockDim.x) {
    const int row = small_div(t, nb, inv_nb);
    const int bt = t - row * nb;
    const int c = small_div(bt, L, inv_L);
    const int f = bt - c * L;
    const V* in = a + row * ld + c * L + f;
    V* out = b + row * ld + c * L * P + f;
    V x[P];
#pragma unroll
    for (int r = 0; r < P; ++r) x[r] = in[r * mp * L];
    if (f) {
#pragma unroll
      for (int r = 1; r < P; ++r) x[r] = cmul(x[r], tw<SIGN>(W, f * r * mp));
    }
    RegDFT<P, SIGN, V>::run(x);
#pragma unroll
    for (int q = 0; q < P; ++q) out[q * L] = x[q];
  }
}

// Transform `nf` rows of length pl.N (row stride ld) held in `a`, using `b` as scratch.  All threads
// of the block take part; returns the buffer that holds the result (a or b).  Ends with a barrier.
template <int SIGN, typename V>
__device__ V* stockham_rows(V* a, V* b, int nf, int ld, const FftPlan& pl, const V* W) {
  const int N = pl.N;
  int L = 1;
  for (int s = 0; s < pl.nst; ++s) {
    const int p = pl.radix[s];
    switch (p) {
      case 3: stockham_pass<3, SIGN>(a, b, nf, ld, N, L, W); break;
      case 5: stockham_pass<5, SIGN>(a, b, nf, ld, N, L, W); break;
      case 7: stockham_pass<7, SIGN>(a, b, nf, ld, N, L, W); break;
      case 9: stockham_pass<9, SIGN>(a, b, nf, ld, N, L, W); break;
      case 27:
        // FP32 only (plan_radix): 27 FP64 complex values would cost too many registers
        if constexpr (sizeof(V) == sizeof(float2)) {
          stockham_pass<27, SIGN>(a, b, nf, ld, N, L, W);
          break;
        }
        [[fallthrough]];
      default: {
        const int mp = N / (L * p);
        const int nb = N / p;
        const int total = nb * nf;
        const float inv_nb = 1.0f / (float)nb, inv_L = 1.0f / (float)L;
        for (int t = threadIdx.x; t < total; t += blockDim.x) {
          const int row = small_div(t, nb, inv_nb);
          const int bt = t - row * nb;
          const int c = small_div(bt, L, inv_L);
          const int f = bt - c * L;
          butterfly<SIGN>(p, a + row * ld, b + row * ld, c, f, L, mp, N, W);
        }
      }
    }
    __syncthreads();
    V* tmp = a;
    a = b;
    b = tmp;
    L *= p;
  }
  return a;
}

// Asynchronous global -> shared copies (cp.async, no register staging), so that a block keeps all of its
// tile's loads in flight at once; sizes 4, 8 or 16 bytes, both addresses aligned to the size.
template <int BYTES>
__device__ __forceinline__ void cp_async(void* smem, const void* gmem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  if (BYTES == 16) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
  } else {
    asm volatile("cp.async.ca.shared.global [%0], [%1], %2;\n" ::"r"(s), "l"(gmem), "n"(BYTES) : "memory");
  }
}
__device__ __forceinline__ void cp_async_wait_all() {
  asm volatile("cp.async.commit_group;\n" ::: "memory");
  asm volatile("cp.async.wait_group 0;\n" ::: "memory");
}

// frequency k in Z_N of storage index n
__device__ __forceinline__ int freq_of(int n, int N) { return n <= (N - 1) / 2 ? n : n - N; }

}  // namespace lrfg
