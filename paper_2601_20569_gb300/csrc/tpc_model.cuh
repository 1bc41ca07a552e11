// Track model of the CUDA tracker: helix step, covariance transport,
// scattering, Kalman update, sector rotation and three-point seed.
//
// Every expression is a fixed sequence of IEEE binary operations with
// correctly rounded sqrt and divide.  Compiled with --fmad=false (strict
// mode) the results are bit-identical to an independent CPU evaluation of the
// same sequences (the paper's deterministic mode, Sec. 5); compiled with FMA
// contraction (fast mode) they agree to rounding.
//
// State at local x: p = (y, z, sin(phi), tan(lambda), q/pT); covariance c[15]
// lower triangle.  kappa = (q/pT) * kb is the signed curvature; sin(phi)
// changes by kappa*dx over a step dx; y by dx*tan((phi0+phi1)/2) (exact
// circle relation); z by tan(lambda) times the arc chord*asin(u)/u,
// u = kappa*chord/2.
#pragma once

#include "tpc_internal.h"
#include "tpc_df.cuh"
#include "tpc_fp64.cuh"

namespace tpc {

template <typename R> struct Trk {
  R p[5];
  R c[15];
  R x;
};

// 1/x: correctly rounded in strict mode; the hardware approximation (about
// one ulp) in fast mode.
__device__ __forceinline__ float frcp(float x) {
#ifdef TPC_FAST_ARITH
  return __fdividef(1.0f, x);
#else
  return 1.0f / x;
#endif
}

// asin(u)/u as an 8-term series in u^2 (coefficients (2n)!/(4^n (n!)^2 (2n+1))).
__device__ __forceinline__ float asinc_f(float u) {
  const float w = u * u;
  const float c1 = (float)(1.0 / 6.0), c2 = (float)(3.0 / 40.0), c3 = (float)(5.0 / 112.0),
              c4 = (float)(35.0 / 1152.0), c5 = (float)(63.0 / 2816.0),
              c6 = (float)(231.0 / 13312.0), c7 = (float)(143.0 / 10240.0);
  return 1.0f + w * (c1 + w * (c2 + w * (c3 + w * (c4 + w * (c5 + w * (c6 + w * c7))))));
}

// d/du of the series above (6 terms).
__device__ __forceinline__ float asinc_deriv_f(float u) {
  const float w = u * u;
  const float d1 = (float)(1.0 / 3.0), d2 = (float)(3.0 / 10.0), d3 = (float)(15.0 / 56.0),
              d4 = (float)(35.0 / 144.0), d5 = (float)(315.0 / 1408.0),
              d6 = (float)(693.0 / 3328.0);
  return u * (d1 + w * (d2 + w * (d3 + w * (d4 + w * (d5 + w * d6)))));
}

__device__ __forceinline__ void reset_cov(float* c, const KParams& P) {
#pragma unroll
  for (int i = 0; i < 15; ++i) c[i] = 0.0f;
  c[0] = P.seed_c[0];
  c[2] = P.seed_c[1];
  c[5] = P.seed_c[2];
  c[9] = P.seed_c[3];
  c[14] = P.seed_c[4];
}

struct StepJ {
  float p0, p1, p2;  // new y, z, sin(phi)
  float f02, f04, f12, f13, f14, f24;
};

// Helix step of p by dx.  Returns false when |sin(phi)| leaves the model domain.
__device__ __forceinline__ bool helix_step(const float* p, float dx, const KParams& P, StepJ& st,
                                           float lim) {
  const float kappa = p[4] * P.kb;
  const float s0 = p[2];
  const float s1 = s0 + kappa * dx;
  if (!(fabsf(s1) < lim)) return false;
#ifdef TPC_FAST_ARITH
  // fast mode: hardware reciprocal and reciprocal square root (a few ulp)
  // instead of the correctly rounded divide and square root
  const float a0 = 1.0f - s0 * s0, a1 = 1.0f - s1 * s1;
  const float rc0 = rsqrtf(a0), rc1 = rsqrtf(a1);
  const float c0 = a0 * rc0;
  const float c1 = a1 * rc1;
  const float N = s0 + s1;
  const float D = c0 + c1;
  const float iD = frcp(D);
  const float t = N * iD;
  const float tt = 1.0f + t * t;
  const float rL = rsqrtf(tt);
  const float L1 = tt * rL;
  const float chord = dx * L1;
  const float u = kappa * chord * 0.5f;
  const float ds = chord * asinc_f(u);
  const float B = rsqrtf(1.0f - u * u);
  const float Ap = asinc_deriv_f(u);
  st.p0 = p[0] + dx * t;
  st.p1 = p[1] + p[3] * ds;
  st.p2 = s1;
  const float iD2 = iD * iD;
  const float q0 = s0 * rc0, q1 = s1 * rc1;
  const float dt_ds0 = (2.0f * D + N * (q0 + q1)) * iD2;
  const float dt_dk = dx * (D + N * q1) * iD2;
  const float g = dx * t * rL;
#else
  const float c0 = sqrtf(1.0f - s0 * s0);
  const float c1 = sqrtf(1.0f - s1 * s1);
  const float N = s0 + s1;
  const float D = c0 + c1;
  const float t = N / D;
  const float L1 = sqrtf(1.0f + t * t);
  const float chord = dx * L1;
  const float u = kappa * chord * 0.5f;
  const float ds = chord * asinc_f(u);
  const float B = 1.0f / sqrtf(1.0f - u * u);
  const float Ap = asinc_deriv_f(u);
  st.p0 = p[0] + dx * t;
  st.p1 = p[1] + p[3] * ds;
  st.p2 = s1;
  const float iD2 = 1.0f / (D * D);
  const float q0 = s0 / c0, q1 = s1 / c1;
  const float dt_ds0 = (2.0f * D + N * (q0 + q1)) * iD2;
  const float dt_dk = dx * (D + N * q1) * iD2;
  const float g = dx * t / L1;
#endif
  st.f02 = dx * dt_ds0;
  st.f04 = dx * dt_dk * P.kb;
  st.f12 = p[3] * g * dt_ds0 * B;
  st.f13 = ds;
  st.f14 = p[3] * (g * dt_dk * B + 0.5f * chord * chord * Ap) * P.kb;
  st.f24 = dx * P.kb;
  return true;
}

// c <- F c F^T with F = identity + (f02, f04, f12, f13, f14, f24).  The sums
// run in ascending index order (the order of the dense product).
__device__ __forceinline__ void cov_transport(float* c, const StepJ& s) {
  // full symmetric matrix entries needed: M[i][j]
  const float m00 = c[0], m10 = c[1], m11 = c[2], m20 = c[3], m21 = c[4], m22 = c[5];
  const float m30 = c[6], m31 = c[7], m32 = c[8], m33 = c[9];
  const float m40 = c[10], m41 = c[11], m42 = c[12], m43 = c[13], m44 = c[14];
  // A = F M (rows 0,1,2 change), columns j = 0..4
  const float a00 = m00 + s.f02 * m20 + s.f04 * m40;
  const float a01 = m10 + s.f02 * m21 + s.f04 * m41;
  const float a02 = m20 + s.f02 * m22 + s.f04 * m42;
  const float a03 = m30 + s.f02 * m32 + s.f04 * m43;
  const float a04 = m40 + s.f02 * m42 + s.f04 * m44;
  const float a10 = m10 + s.f12 * m20 + s.f13 * m30 + s.f14 * m40;
  const float a11 = m11 + s.f12 * m21 + s.f13 * m31 + s.f14 * m41;
  const float a12 = m21 + s.f12 * m22 + s.f13 * m32 + s.f14 * m42;
  const float a13 = m31 + s.f12 * m32 + s.f13 * m33 + s.f14 * m43;
  const float a14 = m41 + s.f12 * m42 + s.f13 * m43 + s.f14 * m44;
  const float a20 = m20 + s.f24 * m40;
  const float a21 = m21 + s.f24 * m41;
  const float a22 = m22 + s.f24 * m42;
  const float a23 = m32 + s.f24 * m43;
  const float a24 = m42 + s.f24 * m44;
  // rows 3, 4 of A are rows 3, 4 of M
  const float a30 = m30, a31 = m31, a32 = m32, a33 = m33, a34 = m43;
  const float a40 = m40, a41 = m41, a42 = m42, a43 = m43, a44 = m44;
  // C' = A F^T, lower triangle
  c[0] = a00 + a02 * s.f02 + a04 * s.f04;
  c[1] = a10 + a12 * s.f02 + a14 * s.f04;
  c[2] = a11 + a12 * s.f12 + a13 * s.f13 + a14 * s.f14;
  c[3] = a20 + a22 * s.f02 + a24 * s.f04;
  c[4] = a21 + a22 * s.f12 + a23 * s.f13 + a24 * s.f14;
  c[5] = a22 + a24 * s.f24;
  c[6] = a30 + a32 * s.f02 + a34 * s.f04;
  c[7] = a31 + a32 * s.f12 + a33 * s.f13 + a34 * s.f14;
  c[8] = a32 + a34 * s.f24;
  c[9] = a33;
  c[10] = a40 + a42 * s.f02 + a44 * s.f04;
  c[11] = a41 + a42 * s.f12 + a43 * s.f13 + a44 * s.f14;
  c[12] = a42 + a44 * s.f24;
  c[13] = a43;
  c[14] = a44;
}

// Scattering noise per pad row crossed.
__device__ __forceinline__ void add_ms(float* c, const float* p, float dx, const KParams& P) {
  const float th2 = P.ms2 * (fabsf(dx) * P.pitch_inv);
  const float a = 1.0f + p[3] * p[3];
  c[5] = c[5] + th2 * (1.0f - p[2] * p[2]) * a;
  c[9] = c[9] + th2 * a * a;
}

// Extended-Kalman propagation to xnew (Jacobian at the current state).
__device__ __forceinline__ bool propagate(Trk<float>& t, float xnew, const KParams& P, float lim) {
  const float dx = xnew - t.x;
  StepJ st;
  if (!helix_step(t.p, dx, P, st, lim)) return false;
  t.p[0] = st.p0;
  t.p[1] = st.p1;
  t.p[2] = st.p2;
  cov_transport(t.c, st);
  add_ms(t.c, t.p, dx, P);
  t.x = xnew;
  return true;
}

struct Resid {
  float r0, r1, w00, w01, w11, chi2;
};

__device__ __forceinline__ Resid residual(const Trk<float>& t, float my, float mz,
                                          const KParams& P) {
  Resid R;
  R.r0 = my - t.p[0];
  R.r1 = mz - t.p[1];
  const float s00 = t.c[0] + P.sy2;
  const float s01 = t.c[1];
  const float s11 = t.c[2] + P.sz2;
  const float idet = frcp(s00 * s11 - s01 * s01);
  R.w00 = s11 * idet;
  R.w01 = -s01 * idet;
  R.w11 = s00 * idet;
  const float a0 = R.w00 * R.r0 + R.w01 * R.r1;
  const float a1 = R.w01 * R.r0 + R.w11 * R.r1;
  R.chi2 = R.r0 * a0 + R.r1 * a1;
  return R;
}

// chi2 only (no weight matrix kept): candidate scans.
__device__ __forceinline__ float chi2_of(const Trk<float>& t, float my, float mz,
                                         const KParams& P) {
  const float r0 = my - t.p[0];
  const float r1 = mz - t.p[1];
  const float s00 = t.c[0] + P.sy2;
  const float s01 = t.c[1];
  const float s11 = t.c[2] + P.sz2;
  const float idet = frcp(s00 * s11 - s01 * s01);
  const float w00 = s11 * idet;
  const float w01 = -s01 * idet;
  const float w11 = s00 * idet;
  const float a0 = w00 * r0 + w01 * r1;
  const float a1 = w01 * r0 + w11 * r1;
  return r0 * a0 + r1 * a1;
}

__device__ __forceinline__ void update(Trk<float>& t, const Resid& R) {
  // column 0 and 1 of C (index ci(i,0), ci(i,1))
  const float h0[5] = {t.c[0], t.c[1], t.c[3], t.c[6], t.c[10]};
  const float h1[5] = {t.c[1], t.c[2], t.c[4], t.c[7], t.c[11]};
  float k0[5], k1[5];
#pragma unroll
  for (int i = 0; i < 5; ++i) {
    k0[i] = h0[i] * R.w00 + h1[i] * R.w01;
    k1[i] = h0[i] * R.w01 + h1[i] * R.w11;
  }
#pragma unroll
  for (int i = 0; i < 5; ++i) t.p[i] = t.p[i] + (k0[i] * R.r0 + k1[i] * R.r1);
  int idx = 0;
#pragma unroll
  for (int i = 0; i < 5; ++i) {
#pragma unroll
    for (int j = 0; j <= i; ++j) {
      t.c[idx] = t.c[idx] - (k0[i] * h0[j] + k1[i] * h1[j]);
      ++idx;
    }
  }
}

// The same update with the gain and covariance arithmetic in FP64, rounded
// back to FP32 (the final fit's update of low-pT loopers).  Fast mode runs it
// in double-float arithmetic on the FP32 pipe instead (tpc_df.cuh: on GB300
// the FP64 unit is about 1/60 of the FP32 rate; the rounded results are those
// of the FP64 update unless one lies within about 2^-46 of a rounding
// boundary).
__device__ __forceinline__ void update_fp64(Trk<float>& t, const Resid& R) {
#ifdef TPC_FAST_ARITH
  df_update(t.p, t.c, R.r0, R.r1, R.w00, R.w01, R.w11);
#else
  const double w00 = widen(R.w00), w01 = widen(R.w01), w11 = widen(R.w11), r0 = widen(R.r0),
               r1 = widen(R.r1);
  const double h0[5] = {widen(t.c[0]), widen(t.c[1]), widen(t.c[3]), widen(t.c[6]),
                        widen(t.c[10])};
  const double h1[5] = {h0[1], widen(t.c[2]), widen(t.c[4]), widen(t.c[7]), widen(t.c[11])};
  double k0[5], k1[5];
#pragma unroll
  for (int i = 0; i < 5; ++i) {
    k0[i] = h0[i] * w00 + h1[i] * w01;
    k1[i] = h0[i] * w01 + h1[i] * w11;
  }
#pragma unroll
  for (int i = 0; i < 5; ++i) t.p[i] = narrow(widen(t.p[i]) + (k0[i] * r0 + k1[i] * r1));
  int idx = 0;
#pragma unroll
  for (int i = 0; i < 5; ++i) {
#pragma unroll
    for (int j = 0; j <= i; ++j) {
      t.c[idx] = narrow(widen(t.c[idx]) - (k0[i] * h0[j] + k1[i] * h1[j]));
      ++idx;
    }
  }
#endif
}

// Update with the gain and covariance arithmetic in FP64 when `fp64`.
__device__ __forceinline__ void update_as(Trk<float>& t, const Resid& R, bool fp64) {
  if (fp64)
    update_fp64(t, R);
  else
    update(t, R);
}

// Update of the refit: FP64 for loopers, judged at the update by the current
// |q/pT| > looper_qpt.  (The final fit classifies a track once, from its
// first segment's inner end, and calls update_as.)
__device__ __forceinline__ void fit_update(Trk<float>& t, const Resid& R, const KParams& P) {
  update_as(t, R, P.looper_qpt > 0.0f && fabsf(t.p[4]) > P.looper_qpt);
}

// Frame rotation to the adjacent sector (dir = +1: +20 deg).
__device__ __forceinline__ bool rotate(Trk<float>& t, int dir, const KParams& P, float lim) {
  const float ca = P.rot_c;
  const float sa = dir > 0 ? P.rot_s : -P.rot_s;
  const float snp = t.p[2];
  const float csp = sqrtf(1.0f - snp * snp);
  const float xn = t.x * ca + t.p[0] * sa;
  const float yn = t.p[0] * ca - t.x * sa;
  const float sn = snp * ca - csp * sa;
  const float cn = csp * ca + snp * sa;
  if (!(cn > 0.0f) || !(fabsf(sn) < lim)) return false;
  const float j00 = csp / cn;
  const float j10 = -sa * t.p[3] / cn;
  const float j20 = -sa * (t.p[4] * P.kb);
  const float j22 = cn / csp;
  const float m00 = t.c[0], m10 = t.c[1], m11 = t.c[2], m20 = t.c[3], m21 = t.c[4], m22 = t.c[5];
  const float m30 = t.c[6], m31 = t.c[7], m32 = t.c[8], m33 = t.c[9];
  const float m40 = t.c[10], m41 = t.c[11], m42 = t.c[12], m43 = t.c[13], m44 = t.c[14];
  // A = J M
  const float a00 = j00 * m00, a01 = j00 * m10, a02 = j00 * m20, a03 = j00 * m30, a04 = j00 * m40;
  const float a10 = j10 * m00 + m10, a11 = j10 * m10 + m11, a12 = j10 * m20 + m21,
              a13 = j10 * m30 + m31, a14 = j10 * m40 + m41;
  const float a20 = j20 * m00 + j22 * m20, a21 = j20 * m10 + j22 * m21,
              a22 = j20 * m20 + j22 * m22, a23 = j20 * m30 + j22 * m32,
              a24 = j20 * m40 + j22 * m42;
  (void)a01; (void)a03; (void)a13; (void)a14; (void)a23; (void)a24;
  // C' = A J^T
  t.c[0] = a00 * j00;
  t.c[1] = a10 * j00;
  t.c[2] = a10 * j10 + a11;
  t.c[3] = a20 * j00;
  t.c[4] = a20 * j10 + a21;
  t.c[5] = a20 * j20 + a22 * j22;
  t.c[6] = m30 * j00;
  t.c[7] = m30 * j10 + m31;
  t.c[8] = m30 * j20 + m32 * j22;
  t.c[9] = m33;
  t.c[10] = m40 * j00;
  t.c[11] = m40 * j10 + m41;
  t.c[12] = m40 * j20 + m42 * j22;
  t.c[13] = m43;
  t.c[14] = m44;
  (void)a02; (void)a04; (void)a12;
  t.x = xn;
  t.p[0] = yn;
  t.p[2] = sn;
  return true;
}

// Seed through three points of increasing x.
__device__ __forceinline__ bool seed3(const float* x, const float* y, const float* z,
                                      const KParams& P, Trk<float>& t) {
  const float ax = x[1] - x[0], ay = y[1] - y[0];
  const float bx = x[2] - x[1], by = y[2] - y[1];
  const float cx = x[2] - x[0], cy = y[2] - y[0];
  const float cross = ax * by - ay * bx;
  const float la = sqrtf(ax * ax + ay * ay);
  const float lb = sqrtf(bx * bx + by * by);
  const float lc = sqrtf(cx * cx + cy * cy);
  const float kappa = 2.0f * cross / (la * lb * lc);
  const float sh = kappa * lc * 0.5f;
  if (!(fabsf(sh) < 1.0f)) return false;
  const float ch = sqrtf(1.0f - sh * sh);
  const float snc = cy / lc, csc = cx / lc;
  const float snp = snc * ch - csc * sh;
  if (!(fabsf(snp) < P.max_snp)) return false;
  const float arc = lc * asinc_f(sh);
  t.x = x[0];
  t.p[0] = y[0];
  t.p[1] = z[0];
  t.p[2] = snp;
  t.p[3] = (z[2] - z[0]) / arc;
  t.p[4] = kappa / P.kb;
  reset_cov(t.c, P);
  return true;
}

// Stored track state (kStateF floats): p[5], the covariance's 15 elements,
// x, and the sector's bits.
__device__ __forceinline__ void put_state(float* dst, const Trk<float>& t, int sector) {
#pragma unroll
  for (int i = 0; i < 5; ++i) dst[i] = t.p[i];
#pragma unroll
  for (int i = 0; i < 15; ++i) dst[5 + i] = t.c[i];
  dst[20] = t.x;
  dst[21] = __int_as_float(sector);
}

__device__ __forceinline__ void get_state(const float* src, Trk<float>& t) {
#pragma unroll
  for (int i = 0; i < 5; ++i) t.p[i] = src[i];
#pragma unroll
  for (int i = 0; i < 15; ++i) t.c[i] = src[5 + i];
  t.x = src[20];
}

}  // namespace tpc
