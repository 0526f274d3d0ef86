// Small-radix DFT codelets and a batched line transform in shared memory.
//
// The plane-wave kinetic term of Eq. LocalKS is diagonal in G, so H x needs a
// forward and an inverse 3D DFT of every vector.  Each 1D transform of length
// n = n1 * n2 (n1, n2 in {1,2,3,4,5,6,8}) is done in two register passes
// (Cooley-Tukey "four-step"): with j = n2*j1 + j2 and k = k1 + n1*k2,
//   X[k1 + n1 k2] = sum_j2 w_n2^(j2 k2) [ w_n^(j2 k1) sum_j1 x[n2 j1 + j2] w_n1^(j1 k1) ],
// w_n = exp(DIR 2 pi i / n), DIR = -1 forward, +1 inverse (unnormalised).
// Twiddles come from a table of exp(-2 pi i m / n) filled on the host in FP64.
#pragma once
#include "kernels.h"

namespace dgdft {

// twiddle tables (private to the translation unit that includes this header;
// filled by upload_twiddles): entry n(n-1)/2 + m holds exp(-2 pi i m / n)
static __device__ double2 g_tw64[kTwiddleCount];
static __device__ float2 g_tw32[kTwiddleCount];

template <typename T> __device__ __forceinline__ cplx<T> cadd(cplx<T> a, cplx<T> b) { return {a.re + b.re, a.im + b.im}; }
template <typename T> __device__ __forceinline__ cplx<T> csub(cplx<T> a, cplx<T> b) { return {a.re - b.re, a.im - b.im}; }
template <typename T> __device__ __forceinline__ cplx<T> cmul(cplx<T> a, cplx<T> b) {
  return {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re};
}
template <typename T> __device__ __forceinline__ cplx<T> cscale(cplx<T> a, T s) { return {a.re * s, a.im * s}; }
// DIR * i * z
template <int DIR, typename T> __device__ __forceinline__ cplx<T> mul_di(cplx<T> z) {
  return DIR > 0 ? cplx<T>{-z.im, z.re} : cplx<T>{z.im, -z.re};
}

template <typename T> __device__ __forceinline__ cplx<T> twiddle(int n, int m);
template <> __device__ __forceinline__ cplx<double> twiddle<double>(int n, int m) {
  double2 w = g_tw64[twiddle_offset(n) + m];
  return {w.x, w.y};
}
template <> __device__ __forceinline__ cplx<float> twiddle<float>(int n, int m) {
  float2 w = g_tw32[twiddle_offset(n) + m];
  return {w.x, w.y};
}

// ---- codelets: in-place DFT of a[0..R) with w = exp(DIR 2 pi i / R) ----
template <int DIR, typename T> __device__ __forceinline__ void dft3(cplx<T>& a0, cplx<T>& a1, cplx<T>& a2) {
  const T h3 = T(0.86602540378443864676);  // sqrt(3)/2
  cplx<T> s = cadd(a1, a2), d = csub(a1, a2);
  cplx<T> m = {a0.re - T(0.5) * s.re, a0.im - T(0.5) * s.im};
  cplx<T> r = cscale(mul_di<DIR>(d), h3);
  a0 = cadd(a0, s);
  a1 = cadd(m, r);
  a2 = csub(m, r);
}
template <int DIR, typename T> __device__ __forceinline__ void dft4(cplx<T>& a0, cplx<T>& a1, cplx<T>& a2, cplx<T>& a3) {
  cplx<T> t0 = cadd(a0, a2), t1 = csub(a0, a2), t2 = cadd(a1, a3), t3 = mul_di<DIR>(csub(a1, a3));
  a0 = cadd(t0, t2);
  a2 = csub(t0, t2);
  a1 = cadd(t1, t3);
  a3 = csub(t1, t3);
}

template <int R, int DIR, typename T> __device__ __forceinline__ void dft(cplx<T>* a) {
  if constexpr (R == 1) {
  } else if constexpr (R == 2) {
    cplx<T> t = a[0];
    a[0] = cadd(t, a[1]);
    a[1] = csub(t, a[1]);
  } else if constexpr (R == 3) {
    dft3<DIR>(a[0], a[1], a[2]);
  } else if constexpr (R == 4) {
    dft4<DIR>(a[0], a[1], a[2], a[3]);
  } else if constexpr (R == 5) {
    const T c1 = T(0.30901699437494742410), c2 = T(-0.80901699437494742410);  // cos(2pi/5), cos(4pi/5)
    const T s1 = T(0.95105651629515357212), s2 = T(0.58778525229247312917);   // sin(2pi/5), sin(4pi/5)
    cplx<T> p1 = cadd(a[1], a[4]), d1 = csub(a[1], a[4]);
    cplx<T> p2 = cadd(a[2], a[3]), d2 = csub(a[2], a[3]);
    cplx<T> m1 = {a[0].re + c1 * p1.re + c2 * p2.re, a[0].im + c1 * p1.im + c2 * p2.im};
    cplx<T> m2 = {a[0].re + c2 * p1.re + c1 * p2.re, a[0].im + c2 * p1.im + c1 * p2.im};
    cplx<T> r1 = mul_di<DIR>(cplx<T>{s1 * d1.re + s2 * d2.re, s1 * d1.im + s2 * d2.im});
    cplx<T> r2 = mul_di<DIR>(cplx<T>{s2 * d1.re - s1 * d2.re, s2 * d1.im - s1 * d2.im});
    a[0] = cadd(a[0], cadd(p1, p2));
    a[1] = cadd(m1, r1);
    a[4] = csub(m1, r1);
    a[2] = cadd(m2, r2);
    a[3] = csub(m2, r2);
  } else if constexpr (R == 6) {
    // even/odd split into two DFT3: X_k = E_{k%3} + w6^k O_{k%3}
    cplx<T> e0 = a[0], e1 = a[2], e2 = a[4], o0 = a[1], o1 = a[3], o2 = a[5];
    dft3<DIR>(e0, e1, e2);
    dft3<DIR>(o0, o1, o2);
    const T h3 = T(0.86602540378443864676);
    cplx<T> w1 = {T(0.5), T(DIR) * h3}, w2 = {T(-0.5), T(DIR) * h3};
    cplx<T> q1 = cmul(o1, w1), q2 = cmul(o2, w2);
    a[0] = cadd(e0, o0);
    a[3] = csub(e0, o0);
    a[1] = cadd(e1, q1);
    a[4] = csub(e1, q1);
    a[2] = cadd(e2, q2);
    a[5] = csub(e2, q2);
  } else if constexpr (R == 8) {
    cplx<T> e0 = a[0], e1 = a[2], e2 = a[4], e3 = a[6], o0 = a[1], o1 = a[3], o2 = a[5], o3 = a[7];
    dft4<DIR>(e0, e1, e2, e3);
    dft4<DIR>(o0, o1, o2, o3);
    const T r2 = T(0.70710678118654752440);
    cplx<T> q1 = cmul(o1, cplx<T>{r2, T(DIR) * r2});
    cplx<T> q2 = mul_di<DIR>(o2);
    cplx<T> q3 = cmul(o3, cplx<T>{-r2, T(DIR) * r2});
    a[0] = cadd(e0, o0);
    a[4] = csub(e0, o0);
    a[1] = cadd(e1, q1);
    a[5] = csub(e1, q1);
    a[2] = cadd(e2, q2);
    a[6] = csub(e2, q2);
    a[3] = cadd(e3, q3);
    a[7] = csub(e3, q3);
  }
}

// pass 1 of line l: thread t < n2 takes x[n2 j1 + t], j1 < R (=n1); writes tmp[k1 n2 + t]
template <int R, int DIR, typename T>
__device__ __forceinline__ void line_pass1(const cplx<T>* __restrict__ src, int es, cplx<T>* __restrict__ tl, int n,
                                           int n2, int t) {
  cplx<T> a[R];
#pragma unroll
  for (int j1 = 0; j1 < R; j1++) a[j1] = src[(n2 * j1 + t) * es];
  dft<R, DIR>(a);
#pragma unroll
  for (int k1 = 0; k1 < R; k1++) {
    cplx<T> w = twiddle<T>(n, t * k1);  // t*k1 <= (n2-1)(n1-1) < n
    if (DIR > 0) w.im = -w.im;
    tl[k1 * n2 + t] = cmul(a[k1], w);
  }
}

// pass 2 of line l: thread t < n1 takes tmp[t n2 + j2], j2 < R (=n2); writes X[t + n1 k2]
template <int R, int DIR, typename T>
__device__ __forceinline__ void line_pass2(const cplx<T>* __restrict__ tl, cplx<T>* __restrict__ dst, int ed, int n1,
                                           int t) {
  cplx<T> a[R];
#pragma unroll
  for (int j2 = 0; j2 < R; j2++) a[j2] = tl[t * R + j2];
  dft<R, DIR>(a);
#pragma unroll
  for (int k2 = 0; k2 < R; k2++) dst[(t + n1 * k2) * ed] = a[k2];
}

#define DGDFT_RADIX_SWITCH(r, CALL) \
  switch (r) {                      \
    case 1: CALL(1); break;         \
    case 2: CALL(2); break;         \
    case 3: CALL(3); break;         \
    case 4: CALL(4); break;         \
    case 5: CALL(5); break;         \
    case 6: CALL(6); break;         \
    case 8: CALL(8); break;         \
    default: break;                 \
  }

// Batched out-of-place line DFT by the whole CTA (every thread must call it).
// Line l, element j is read from src[l*ls + j*es] and written to dst[l*ld + j*ed];
// tmp holds nlines*n scratch.  src may equal dst.  Ends with __syncthreads().
template <int DIR, typename T>
__device__ void fft_lines(const cplx<T>* src, int ls, int es, cplx<T>* dst, int ld, int ed, cplx<T>* tmp, int nlines,
                          int n1, int n2) {
  const int n = n1 * n2;
  for (int w = threadIdx.x; w < nlines * n2; w += blockDim.x) {
    const int l = w / n2, t = w - l * n2;
#define P1(R) line_pass1<R, DIR, T>(src + (long long)l * ls, es, tmp + l * n, n, n2, t)
    DGDFT_RADIX_SWITCH(n1, P1)
#undef P1
  }
  __syncthreads();
  for (int w = threadIdx.x; w < nlines * n1; w += blockDim.x) {
    const int l = w / n1, t = w - l * n1;
#define P2(R) line_pass2<R, DIR, T>(tmp + l * n, dst + (long long)l * ld, ed, n1, t)
    DGDFT_RADIX_SWITCH(n2, P2)
#undef P2
  }
  __syncthreads();
}

}  // namespace dgdft
