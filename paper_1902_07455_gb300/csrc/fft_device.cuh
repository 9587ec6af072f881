// Batched odd-length complex FFTs of fibres staged in shared memory (FP64 double2 or FP32 float2).
//
// Mixed-radix Stockham autosort, decimation in time.  After the stages with radices p_0..p_{s-1}
// (L = p_0...p_{s-1}), row entry c*L + f holds the length-L DFT (frequency f) of the subsequence
// x[c + (N/L) t], t = 0..L-1.  A radix-p stage with m' = N/(L p) combines p such subsequences:
//   Z'[c'][f + L q] = sum_r w_p^{q r} ( w_{Lp}^{f r} Z[c' + m' r][f] ),   q, r = 0..p-1,
// with w_M = exp(sign 2 pi i / M).  It starts from the natural order (L = 1) and ends in natural
// order (L = N), so no digit reversal is needed.  Twiddles come from one table
// W[j] = exp(-2 pi i j / N) (w_{Lp}^{f r} = W[f r m'], w_p^{q r} = W[(q r mod p) N / p]).
#pragma once

#include <cuda_runtime.h>

namespace lrfg {

constexpr int kMaxStages = 24;
constexpr int kMaxGenericRadix = 31;

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
template <int SIGN, typename V>
__device__ V* stockham_rows(V* a, V* b, int nf, int ld, const FftPlan& pl, const V* W) {
  const int N = pl.N;
  int L = 1;
  for (int s = 0; s < pl.nst; ++s) {
    const int p = pl.radix[s];
    const int mp = N / (L * p);
    const int nb = N / p;
    const int total = nb * nf;
    for (int t = threadIdx.x; t < total; t += blockDim.x) {
      int row = t / nb;
      int bt = t - row * nb;
      int f = bt % L;
      int c = bt / L;
      butterfly<SIGN>(p, a + row * ld, b + row * ld, c, f, L, mp, N, W);
    }
    __syncthreads();
    V* tmp = a;
    a = b;
    b = tmp;
    L *= p;
  }
  return a;
}

// frequency k in Z_N of storage index n
__device__ __forceinline__ int freq_of(int n, int N) { return n <= (N - 1) / 2 ? n : n - N; }

}  // namespace lrfg
