// The Kalman gain and covariance update in double-float arithmetic: every
// quantity of the update that FP32 would round is carried as an unevaluated
// sum hi + lo of two floats, built from error-free transformations (Knuth's
// TwoSum, TAOCP vol. 2 Sec. 4.2.2; the FMA form of Dekker's TwoProduct), and
// the final sums are compensated in the manner of Ogita, Rump and Oishi's
// Sum2 (SIAM J. Sci. Comput. 26 (2005) 1955).  The results are rounded to
// FP32 once, like those of the FP64 update.
//
// Why: the final fit runs the update of low-pT loopers in FP64 to keep the
// covariance's cancellation C - K H C from eating the FP32 mantissa.  On
// GB300 the FP64 unit is about 1/60 of the FP32 rate, so fast mode does the
// same update on the FP32 pipe with about 2^-46 relative precision per term
// instead of 2^-53: the rounded results differ from the FP64 update's only
// where a result lies within that margin of a rounding boundary.  (Strict
// mode keeps the FP64 update, which the oracle defines.)
//
// Host-compilable, so that a CPU test can compare it with the FP64 update and
// an extended-precision evaluation.  Every operation is an explicitly rounded
// one: the transformations are exact only if no multiply and add are fused
// behind their back.
#pragma once

#include <cmath>

#ifdef __CUDACC__
#define TPC_DF __host__ __device__ __forceinline__
#define TPC_DF_UNROLL _Pragma("unroll")
#else
#define TPC_DF inline
#define TPC_DF_UNROLL
#endif

namespace tpc {

TPC_DF float df_add(float a, float b) {
#ifdef __CUDA_ARCH__
  return __fadd_rn(a, b);
#else
  return a + b;
#endif
}

TPC_DF float df_sub(float a, float b) {
#ifdef __CUDA_ARCH__
  return __fsub_rn(a, b);
#else
  return a - b;
#endif
}

TPC_DF float df_mul(float a, float b) {
#ifdef __CUDA_ARCH__
  return __fmul_rn(a, b);
#else
  return a * b;
#endif
}

TPC_DF float df_fma(float a, float b, float c) {
#ifdef __CUDA_ARCH__
  return __fmaf_rn(a, b, c);
#else
  return std::fmaf(a, b, c);
#endif
}

// s + e == a + b exactly, s = fl(a + b) (no ordering of |a|, |b| needed)
TPC_DF void two_sum(float a, float b, float& s, float& e) {
  s = df_add(a, b);
  const float bb = df_sub(s, a);
  e = df_add(df_sub(a, df_sub(s, bb)), df_sub(b, bb));
}

// p + e == a * b exactly (barring underflow), p = fl(a * b)
TPC_DF void two_prod(float a, float b, float& p, float& e) {
  p = df_mul(a, b);
  e = df_fma(a, b, -p);
}

// hi + lo ~= a * x + b * y with error about 2^-48 (|a x| + |b y|)
TPC_DF void df_dot2(float a, float x, float b, float y, float& hi, float& lo) {
  float p, pe, q, qe, e;
  two_prod(a, x, p, pe);
  two_prod(b, y, q, qe);
  two_sum(p, q, hi, e);
  lo = df_add(e, df_add(pe, qe));
}

// fl(v +- ((kh + kl) * x + (gh + gl) * y)) (kSub: minus): the two products of
// a double-float by a float (the hi part's product exact, the lo part's
// rounded), their sum with v compensated, one final rounding.
template <bool kSub>
TPC_DF float df_axpy2(float v, float kh, float kl, float x, float gh, float gl, float y) {
  float u, ue, w, we, s1, e1, s2, e2;
  two_prod(kh, x, u, ue);
  ue = df_fma(kl, x, ue);
  two_prod(gh, y, w, we);
  we = df_fma(gl, y, we);
  two_sum(v, kSub ? -u : u, s1, e1);
  two_sum(s1, kSub ? -w : w, s2, e2);
  const float t = df_add(ue, we);
  return df_add(s2, df_add(df_add(e1, e2), kSub ? -t : t));
}

// Kalman update of state p[5] and packed lower-triangular covariance c[15]
// (c[i(i+1)/2 + j], j <= i) by a 2-D measurement of (y, z) = (p[0], p[1]):
// residual (r0, r1), weight W = (H C H^T + V)^-1 = [[w00, w01], [w01, w11]].
// Gain K = C H^T W: k0 = C[:,0] w00 + C[:,1] w01, k1 = C[:,0] w01 + C[:,1] w11;
// p += k0 r0 + k1 r1; C -= k0 C[0,:] + k1 C[1,:].
TPC_DF void df_update(float* p, float* c, float r0, float r1, float w00, float w01, float w11) {
  const float h0[5] = {c[0], c[1], c[3], c[6], c[10]};
  const float h1[5] = {c[1], c[2], c[4], c[7], c[11]};
  float k0h[5], k0l[5], k1h[5], k1l[5];
  TPC_DF_UNROLL
  for (int i = 0; i < 5; ++i) {
    df_dot2(h0[i], w00, h1[i], w01, k0h[i], k0l[i]);
    df_dot2(h0[i], w01, h1[i], w11, k1h[i], k1l[i]);
  }
  TPC_DF_UNROLL
  for (int i = 0; i < 5; ++i) p[i] = df_axpy2<false>(p[i], k0h[i], k0l[i], r0, k1h[i], k1l[i], r1);
  int idx = 0;
  TPC_DF_UNROLL
  for (int i = 0; i < 5; ++i) {
    TPC_DF_UNROLL
    for (int j = 0; j <= i; ++j) {
      c[idx] = df_axpy2<true>(c[idx], k0h[i], k0l[i], h0[j], k1h[i], k1l[i], h1[j]);
      ++idx;
    }
  }
}

}  // namespace tpc
