// Checks the double-float Kalman update (fast mode's looper update) against
// the FP64 update (strict mode's, inputs widened exactly, results rounded to
// float once) and against an extended-precision (long double) evaluation of
// the same formulas, on states drawn from a Kalman filter run: a helix-like
// 5-parameter model (y, z, sin phi, tan lambda, q/pT) stepped over 1 cm pad
// rows with scattering noise and 2-D (y, z) measurements, restarted from the
// seed covariance diag(1, 1, 0.25, 0.25, 100) every 160 rows, with |q/pT| up
// to 20 (c).  The FP32 update is evaluated beside them for scale.
//
// Prints, per arm, the fraction of results equal to the FP64 update's and the
// largest distance from the long double result in float ulps, then
// "df_vs_fp64_mismatch <n> df_max_ulps <u> fp32_max_ulps <v>".
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <random>

#include "tpc_df.cuh"
#include "tpc_fp64.cuh"

namespace {

struct St {
  float p[5];
  float c[15];
};

// strict mode's FP64 update: the same formulas, operands widened exactly,
// every result rounded once to float
void update_fp64(St& t, float r0, float r1, float w00, float w01, float w11) {
  const double W00 = tpc::widen(w00), W01 = tpc::widen(w01), W11 = tpc::widen(w11);
  const double R0 = tpc::widen(r0), R1 = tpc::widen(r1);
  const int col0[5] = {0, 1, 3, 6, 10}, col1[5] = {1, 2, 4, 7, 11};
  double h0[5], h1[5], k0[5], k1[5];
  for (int i = 0; i < 5; ++i) {
    h0[i] = tpc::widen(t.c[col0[i]]);
    h1[i] = tpc::widen(t.c[col1[i]]);
  }
  for (int i = 0; i < 5; ++i) {
    k0[i] = h0[i] * W00 + h1[i] * W01;
    k1[i] = h0[i] * W01 + h1[i] * W11;
  }
  for (int i = 0; i < 5; ++i) t.p[i] = tpc::narrow(tpc::widen(t.p[i]) + (k0[i] * R0 + k1[i] * R1));
  int idx = 0;
  for (int i = 0; i < 5; ++i)
    for (int j = 0; j <= i; ++j, ++idx)
      t.c[idx] = tpc::narrow(tpc::widen(t.c[idx]) - (k0[i] * h0[j] + k1[i] * h1[j]));
}

// the same in long double, unrounded
void update_ld(const St& t, float r0, float r1, float w00, float w01, float w11, long double* out) {
  const int col0[5] = {0, 1, 3, 6, 10}, col1[5] = {1, 2, 4, 7, 11};
  long double h0[5], h1[5], k0[5], k1[5];
  for (int i = 0; i < 5; ++i) {
    h0[i] = t.c[col0[i]];
    h1[i] = t.c[col1[i]];
  }
  for (int i = 0; i < 5; ++i) {
    k0[i] = h0[i] * (long double)w00 + h1[i] * (long double)w01;
    k1[i] = h0[i] * (long double)w01 + h1[i] * (long double)w11;
  }
  for (int i = 0; i < 5; ++i) out[i] = (long double)t.p[i] + (k0[i] * r0 + k1[i] * r1);
  int idx = 0;
  for (int i = 0; i < 5; ++i)
    for (int j = 0; j <= i; ++j, ++idx)
      out[5 + idx] = (long double)t.c[idx] - (k0[i] * h0[j] + k1[i] * h1[j]);
}

void update_fp32(St& t, float r0, float r1, float w00, float w01, float w11) {
  const float h0[5] = {t.c[0], t.c[1], t.c[3], t.c[6], t.c[10]};
  const float h1[5] = {t.c[1], t.c[2], t.c[4], t.c[7], t.c[11]};
  float k0[5], k1[5];
  for (int i = 0; i < 5; ++i) {
    k0[i] = h0[i] * w00 + h1[i] * w01;
    k1[i] = h0[i] * w01 + h1[i] * w11;
  }
  for (int i = 0; i < 5; ++i) t.p[i] = t.p[i] + (k0[i] * r0 + k1[i] * r1);
  int idx = 0;
  for (int i = 0; i < 5; ++i)
    for (int j = 0; j <= i; ++j, ++idx) t.c[idx] = t.c[idx] - (k0[i] * h0[j] + k1[i] * h1[j]);
}

// distance of float f from x in ulps of float at x
double ulps(float f, long double x) {
  const float xf = (float)x;
  const double u = std::fabs((double)std::nextafter(xf, INFINITY) - (double)xf);
  if (u == 0.0 || !std::isfinite(u)) return 0.0;
  return (double)std::fabs((long double)f - x) / u;
}

uint32_t bits(float f) {
  uint32_t u;
  std::memcpy(&u, &f, 4);
  return u;
}

}  // namespace

int main() {
  std::mt19937_64 rng(20260120569ull);
  std::normal_distribution<double> gauss(0.0, 1.0);
  std::uniform_real_distribution<double> unif(0.0, 1.0);
  const double sy2 = 0.01, sz2 = 0.01, ms2 = 1e-6, kb = 1.5e-3;
  const long n_tracks = 4000, n_rows = 160;
  long n_out = 0, mismatch = 0;
  double df_max = 0.0, fp64_max = 0.0, fp32_max = 0.0;
  for (long trk = 0; trk < n_tracks; ++trk) {
    // filter state in long double; every update's input is its float copy
    long double p[5] = {0.0L, 0.0L, (long double)(0.6 * (2 * unif(rng) - 1)),
                        (long double)(2 * (2 * unif(rng) - 1)),
                        (long double)(20 * (2 * unif(rng) - 1))};
    long double C[5][5] = {};
    const double seed[5] = {1.0, 1.0, 0.25, 0.25, 100.0};
    for (int i = 0; i < 5; ++i) C[i][i] = seed[i];
    for (long row = 0; row < n_rows; ++row) {
      // transport over dx = 1: y += snp + kb q/2, z += tgl, snp += kb q
      const long double dx = 1.0L, k = kb * p[4];
      long double F[5][5] = {};
      for (int i = 0; i < 5; ++i) F[i][i] = 1.0L;
      F[0][2] = dx;
      F[0][4] = 0.5L * kb * dx * dx;
      F[1][3] = dx;
      F[2][4] = kb * dx;
      p[0] += dx * p[2] + 0.5L * k * dx * dx;
      p[1] += dx * p[3];
      p[2] += k * dx;
      if (std::fabs((double)p[2]) > 0.9) p[2] *= -0.5L;
      long double T[5][5] = {}, Cn[5][5] = {};
      for (int i = 0; i < 5; ++i)
        for (int j = 0; j < 5; ++j)
          for (int l = 0; l < 5; ++l) T[i][j] += F[i][l] * C[l][j];
      for (int i = 0; i < 5; ++i)
        for (int j = 0; j < 5; ++j)
          for (int l = 0; l < 5; ++l) Cn[i][j] += T[i][l] * F[j][l];
      Cn[2][2] += ms2;
      Cn[3][3] += ms2;
      St s;
      for (int i = 0; i < 5; ++i) s.p[i] = (float)p[i];
      for (int i = 0, idx = 0; i < 5; ++i)
        for (int j = 0; j <= i; ++j, ++idx) s.c[idx] = (float)Cn[i][j];
      // the float weight of the residual, as the tracker computes it
      const float s00 = s.c[0] + (float)sy2, s01 = s.c[1], s11 = s.c[2] + (float)sz2;
      const float idet = 1.0f / (s00 * s11 - s01 * s01);
      const float w00 = s11 * idet, w01 = -s01 * idet, w11 = s00 * idet;
      const float r0 = (float)(gauss(rng) * std::sqrt((double)s00));
      const float r1 = (float)(gauss(rng) * std::sqrt((double)s11));
      long double ref[20];
      update_ld(s, r0, r1, w00, w01, w11, ref);
      St a = s, b = s, c32 = s;
      tpc::df_update(a.p, a.c, r0, r1, w00, w01, w11);
      update_fp64(b, r0, r1, w00, w01, w11);
      update_fp32(c32, r0, r1, w00, w01, w11);
      for (int o = 0; o < 20; ++o) {
        const float fa = o < 5 ? a.p[o] : a.c[o - 5];
        const float fb = o < 5 ? b.p[o] : b.c[o - 5];
        const float fc = o < 5 ? c32.p[o] : c32.c[o - 5];
        ++n_out;
        if (bits(fa) != bits(fb)) ++mismatch;
        df_max = std::fmax(df_max, ulps(fa, ref[o]));
        fp64_max = std::fmax(fp64_max, ulps(fb, ref[o]));
        fp32_max = std::fmax(fp32_max, ulps(fc, ref[o]));
      }
      // continue the filter from the exact update (long double)
      long double pk[5], Ck[5][5];
      const long double W[2][2] = {{w00, w01}, {w01, w11}};
      long double K[5][2];
      for (int i = 0; i < 5; ++i)
        for (int m = 0; m < 2; ++m) K[i][m] = Cn[i][0] * W[0][m] + Cn[i][1] * W[1][m];
      for (int i = 0; i < 5; ++i) pk[i] = p[i] + K[i][0] * r0 + K[i][1] * r1;
      for (int i = 0; i < 5; ++i)
        for (int j = 0; j < 5; ++j) Ck[i][j] = Cn[i][j] - (K[i][0] * Cn[0][j] + K[i][1] * Cn[1][j]);
      for (int i = 0; i < 5; ++i) {
        p[i] = pk[i];
        for (int j = 0; j < 5; ++j) C[i][j] = 0.5L * (Ck[i][j] + Ck[j][i]);
      }
    }
  }
  std::printf("%ld results: df equal to the FP64 update %.6f; max |error| vs long double in "
              "float ulps: df %.3f, FP64 %.3f, FP32 %.3g\n",
              n_out, 1.0 - (double)mismatch / n_out, df_max, fp64_max, fp32_max);
  std::printf("df_vs_fp64_mismatch %ld df_max_ulps %.6f fp32_max_ulps %.6g\n", mismatch, df_max,
              fp32_max);
  return 0;
}
