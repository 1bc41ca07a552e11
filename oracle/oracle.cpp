// CPU ORACLE -- test infrastructure only.
//
// A plain, slow, sequential restatement of the TPC track reconstruction the
// paper describes (Sec. 2 "ALICE Run 3 TPC Tracking Performance" and Sec. 3
// "Tracking Improvements", Phases I and II).  Only the tests, the smoke check
// and the CPU baseline of the benchmark may load it; the product path never
// does.  It shares no code, header, table or constant with the CUDA library:
// every constant it uses arrives through the option struct from the caller.
//
// Templated on Real:
//   float  -- "strict" mode: compiled with -ffp-contract=off -fno-fast-math,
//             every formula a fixed sequence of IEEE binary operations and
//             correctly rounded sqrt/divide; the CUDA strict build evaluates
//             the same sequences, so both agree bit for bit (the paper's
//             deterministic mode, Sec. 5, compares CPU and GPU at bit level).
//   double -- precision reference (closed-form helix pins, gradients).
//
// The paper gives no formulas; the track model and every cut below are
// readings of its qualitative description (the library documentation lists
// them).  Stage order:
//   a1 per-row cluster index (the oracle's own search structure)
//   a2 CA neighbour finding        (Sec. 2: cellular-automaton seeding)
//   a3 neighbour cleaning          (mutual links)
//   a4 start hits                  (chains of >= 3 linked clusters)
//   a5 tracklet constructor        (Sec. 2: Kalman track following)
//   a6 tracklet selector           (Sec. 2 ambiguity solving, Sec. 3 Phase I
//                                   criterion: smaller chi2 first, shared
//                                   clusters counted from the outermost row)
//   a7 sector refit + merging      (Sec. 2 merging; Sec. 3 sector refit)
//   a8 distortion correction       (Sec. 2: space-charge correction maps)
//   a9 three-iteration refit       (Sec. 3 Phase I interpolation scheme)
//   a10 inner-region attachment    (Sec. 3 Phase II second ambiguity)
//   a12 refit gradient             (FP64 reverse-mode tape)
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <map>
#include <memory>
#include <string>
#include <vector>

extern "C" {
// Options: the physical inputs and every cut (mirrored by the Python binding).
// Derived constants (curvature factor, tangents, rotation sines) are computed
// here from these inputs, in double, and rounded once.
struct orc_options {
  float bz;              // tesla
  float sigma_y, sigma_z;  // cluster position resolution [cm]
  float ms_theta;        // multiple-scattering angle per pad row [rad]
  float link_wy, link_wz, link_chi2;
  float seed_c[5];       // diagonal of the seed covariance
  float follow_chi2;
  float max_snp;
  float score_w;
  float shared_frac;
  float merge_chi2, merge_dy, merge_dz;
  float int_chi2, final_chi2;
  int32_t max_miss;
  int32_t min_hits;
  int32_t merge_max_gap;
  int32_t inner_rows;
  int32_t cand_k;
  int32_t brute_force;  // 1: candidate search scans whole rows (self-check)
  int32_t n_rows;
  int32_t n_sectors;
};
}

namespace orc {

struct Named {
  std::string dtype;
  std::vector<uint8_t> bytes;
};

struct Result {
  std::map<std::string, Named> arrays;
  template <typename T>
  void put(const std::string& name, const std::vector<T>& v, const char* dtype) {
    Named& a = arrays[name];
    a.dtype = dtype;
    a.bytes.resize(v.size() * sizeof(T));
    if (!v.empty()) std::memcpy(a.bytes.data(), v.data(), a.bytes.size());
  }
};

template <typename Real> const char* real_name();
template <> const char* real_name<float>() { return "f4"; }
template <> const char* real_name<double>() { return "f8"; }

// asin(u)/u: std::asin in double mode; in float mode a fixed 8-term
// Maclaurin series in u^2 (coefficients (2n)!/(4^n (n!)^2 (2n+1))).
template <typename Real> Real asinc(Real u);
template <> double asinc<double>(double u) { return u == 0.0 ? 1.0 : std::asin(u) / u; }
template <> float asinc<float>(float u) {
  const float w = u * u;
  const float c1 = (float)(1.0 / 6.0), c2 = (float)(3.0 / 40.0), c3 = (float)(5.0 / 112.0),
              c4 = (float)(35.0 / 1152.0), c5 = (float)(63.0 / 2816.0),
              c6 = (float)(231.0 / 13312.0), c7 = (float)(143.0 / 10240.0);
  return 1.0f + w * (c1 + w * (c2 + w * (c3 + w * (c4 + w * (c5 + w * (c6 + w * c7))))));
}

// d/du [asin(u)/u]: (1/sqrt(1-u^2) - asin(u)/u)/u in double away from 0; in
// float (and near 0) the derivative of the series above, 6 terms.
template <typename Real> Real asinc_deriv(Real u);
template <> double asinc_deriv<double>(double u) {
  if (std::fabs(u) > 0.01) return (1.0 / std::sqrt(1.0 - u * u) - std::asin(u) / u) / u;
  const double w = u * u;
  return u * (1.0 / 3.0 + w * (3.0 / 10.0 + w * (15.0 / 56.0 + w * (35.0 / 144.0 +
             w * (315.0 / 1408.0 + w * (693.0 / 3328.0))))));
}
template <> float asinc_deriv<float>(float u) {
  const float w = u * u;
  const float d1 = (float)(1.0 / 3.0), d2 = (float)(3.0 / 10.0), d3 = (float)(15.0 / 56.0),
              d4 = (float)(35.0 / 144.0), d5 = (float)(315.0 / 1408.0),
              d6 = (float)(693.0 / 3328.0);
  return u * (d1 + w * (d2 + w * (d3 + w * (d4 + w * (d5 + w * d6)))));
}

inline int ci(int i, int j) { return i >= j ? i * (i + 1) / 2 + j : j * (j + 1) / 2 + i; }

template <typename Real>
struct Track {
  Real p[5];   // y, z, sin(phi), tan(lambda), q/pT
  Real c[15];  // lower triangle, index ci(i,j)
  Real x;
};

template <typename Real>
struct Params {
  Real kb, tan_half, rot_c, rot_s, link_wy, link_wz, link_chi2;
  Real seed_c[5], meas_sy2, meas_sz2, ms_theta2, row_pitch_inv, follow_chi2, max_snp, score_w,
      shared_frac, merge_chi2, merge_dy, merge_dz, int_chi2, final_chi2;
  int max_miss, min_hits, merge_max_gap, inner_rows, cand_k, brute_force, n_rows, n_sectors;
  std::vector<Real> row_x;
};

template <typename Real>
Params<Real> make_params(const orc_options& o, const double* row_x) {
  Params<Real> P;
  const double pi = 3.14159265358979323846;
  P.kb = (Real)(-(double)o.bz * 0.00299792458);
  P.tan_half = (Real)std::tan(10.0 * pi / 180.0);
  P.rot_c = (Real)std::cos(20.0 * pi / 180.0);
  P.rot_s = (Real)std::sin(20.0 * pi / 180.0);
  P.meas_sy2 = (Real)((double)o.sigma_y * (double)o.sigma_y);
  P.meas_sz2 = (Real)((double)o.sigma_z * (double)o.sigma_z);
  P.ms_theta2 = (Real)((double)o.ms_theta * (double)o.ms_theta);
  P.row_pitch_inv =
      (Real)((double)(o.n_rows - 1) / ((double)row_x[o.n_rows - 1] - (double)row_x[0]));
  P.link_wy = o.link_wy; P.link_wz = o.link_wz; P.link_chi2 = o.link_chi2;
  for (int i = 0; i < 5; ++i) P.seed_c[i] = o.seed_c[i];
  P.follow_chi2 = o.follow_chi2; P.max_snp = o.max_snp; P.score_w = o.score_w;
  P.shared_frac = o.shared_frac;
  P.merge_chi2 = o.merge_chi2; P.merge_dy = o.merge_dy; P.merge_dz = o.merge_dz;
  P.int_chi2 = o.int_chi2; P.final_chi2 = o.final_chi2;
  P.max_miss = o.max_miss; P.min_hits = o.min_hits; P.merge_max_gap = o.merge_max_gap;
  P.inner_rows = o.inner_rows; P.cand_k = o.cand_k; P.brute_force = o.brute_force;
  P.n_rows = o.n_rows; P.n_sectors = o.n_sectors;
  P.row_x.resize(o.n_rows);
  for (int r = 0; r < o.n_rows; ++r) P.row_x[r] = (Real)row_x[r];
  return P;
}

// --------------------------------------------------------------- Kalman model
// Covariance reset to the seed diagonal.
template <typename Real>
void reset_cov(Track<Real>& t, const Params<Real>& P) {
  for (int i = 0; i < 15; ++i) t.c[i] = 0;
  t.c[0] = P.seed_c[0]; t.c[2] = P.seed_c[1]; t.c[5] = P.seed_c[2];
  t.c[9] = P.seed_c[3]; t.c[14] = P.seed_c[4];
}

// Helix step x -> x + dx in a sector frame: sin(phi) grows linearly with x at
// rate kappa = (q/pT)*kb; y advances by dx*tan((phi0+phi1)/2) (the exact
// circle relation); z by tan(lambda) times the arc length, the arc being
// chord*asin(u)/u with u = kappa*chord/2.  Jacobian entries f02..f24 are the
// derivatives of (y,z,sin(phi)) by (sin(phi), tan(lambda), q/pT); the arc
// derivative uses d(arc)/d(chord) = 1/sqrt(1-u^2) and
// d(arc)/d(kappa) at fixed chord = chord^2/2 * d(asin(u)/u)/du.
template <typename Real>
struct Step {
  Real p[5];
  Real f02, f04, f12, f13, f14, f24;
};

template <typename Real>
bool helix_step(const Real* p, Real dx, const Params<Real>& P, Step<Real>& st) {
  const Real kappa = p[4] * P.kb;
  const Real s0 = p[2];
  const Real s1 = s0 + kappa * dx;
  if (!(std::fabs(s1) < P.max_snp)) return false;
  const Real c0 = std::sqrt(Real(1) - s0 * s0);
  const Real c1 = std::sqrt(Real(1) - s1 * s1);
  const Real N = s0 + s1;
  const Real D = c0 + c1;
  const Real t = N / D;
  const Real L1 = std::sqrt(Real(1) + t * t);
  const Real chord = dx * L1;
  const Real u = kappa * chord * Real(0.5);
  const Real ds = chord * asinc<Real>(u);
  const Real B = Real(1) / std::sqrt(Real(1) - u * u);
  const Real Ap = asinc_deriv<Real>(u);
  st.p[0] = p[0] + dx * t;
  st.p[1] = p[1] + p[3] * ds;
  st.p[2] = s1;
  st.p[3] = p[3];
  st.p[4] = p[4];
  const Real iD2 = Real(1) / (D * D);
  const Real q0 = s0 / c0, q1 = s1 / c1;
  const Real dt_ds0 = (Real(2) * D + N * (q0 + q1)) * iD2;
  const Real dt_dk = dx * (D + N * q1) * iD2;
  const Real g = dx * t / L1;
  st.f02 = dx * dt_ds0;
  st.f04 = dx * dt_dk * P.kb;
  st.f12 = p[3] * g * dt_ds0 * B;
  st.f13 = ds;
  st.f14 = p[3] * (g * dt_dk * B + Real(0.5) * chord * chord * Ap) * P.kb;
  st.f24 = dx * P.kb;
  return true;
}

// C <- F C F^T for F = identity plus f02, f04, f12, f13, f14, f24.
template <typename Real>
void cov_transport(Real* c, const Step<Real>& st) {
  Real M[5][5];
  for (int i = 0; i < 5; ++i)
    for (int j = 0; j < 5; ++j) M[i][j] = c[ci(i, j)];
  Real A[5][5];
  for (int j = 0; j < 5; ++j) {
    A[0][j] = M[0][j] + st.f02 * M[2][j] + st.f04 * M[4][j];
    A[1][j] = M[1][j] + st.f12 * M[2][j] + st.f13 * M[3][j] + st.f14 * M[4][j];
    A[2][j] = M[2][j] + st.f24 * M[4][j];
    A[3][j] = M[3][j];
    A[4][j] = M[4][j];
  }
  for (int i = 0; i < 5; ++i) {
    c[ci(i, 0)] = A[i][0] + A[i][2] * st.f02 + A[i][4] * st.f04;
    if (i >= 1) c[ci(i, 1)] = A[i][1] + A[i][2] * st.f12 + A[i][3] * st.f13 + A[i][4] * st.f14;
    if (i >= 2) c[ci(i, 2)] = A[i][2] + A[i][4] * st.f24;
    if (i >= 3) c[ci(i, 3)] = A[i][3];
    if (i >= 4) c[ci(i, 4)] = A[i][4];
  }
}

// Multiple scattering per pad row crossed, isotropic angle variance theta^2:
// Var(sin phi) += theta^2 (1 - sin^2 phi)(1 + tan^2 lambda),
// Var(tan lambda) += theta^2 (1 + tan^2 lambda)^2.
template <typename Real>
void add_ms(Real* c, const Real* p, Real dx, const Params<Real>& P) {
  const Real th2 = P.ms_theta2 * (std::fabs(dx) * P.row_pitch_inv);
  const Real a = Real(1) + p[3] * p[3];
  c[5] = c[5] + th2 * (Real(1) - p[2] * p[2]) * a;
  c[9] = c[9] + th2 * a * a;
}

// Extended-Kalman propagation (Jacobian at the current state) with scattering.
template <typename Real>
bool propagate(Track<Real>& t, Real xnew, const Params<Real>& P) {
  const Real dx = xnew - t.x;
  Step<Real> st;
  if (!helix_step(t.p, dx, P, st)) return false;
  for (int i = 0; i < 5; ++i) t.p[i] = st.p[i];
  cov_transport(t.c, st);
  add_ms(t.c, t.p, dx, P);
  t.x = xnew;
  return true;
}

// Predicted chi2 of a (y,z) measurement against the track, 2x2 inverse W.
template <typename Real>
struct Resid {
  Real r0, r1, w00, w01, w11, chi2;
};

template <typename Real>
Resid<Real> residual(const Track<Real>& t, Real my, Real mz, const Params<Real>& P) {
  Resid<Real> R;
  R.r0 = my - t.p[0];
  R.r1 = mz - t.p[1];
  const Real s00 = t.c[0] + P.meas_sy2;
  const Real s01 = t.c[1];
  const Real s11 = t.c[2] + P.meas_sz2;
  const Real idet = Real(1) / (s00 * s11 - s01 * s01);
  R.w00 = s11 * idet;
  R.w01 = -s01 * idet;
  R.w11 = s00 * idet;
  const Real a0 = R.w00 * R.r0 + R.w01 * R.r1;
  const Real a1 = R.w01 * R.r0 + R.w11 * R.r1;
  R.chi2 = R.r0 * a0 + R.r1 * a1;
  return R;
}

// Kalman update with gain K = C H^T W, C <- C - K H C.
template <typename Real>
void update(Track<Real>& t, const Resid<Real>& R) {
  Real k0[5], k1[5], h0[5], h1[5];
  for (int i = 0; i < 5; ++i) {
    h0[i] = t.c[ci(i, 0)];
    h1[i] = t.c[ci(i, 1)];
  }
  for (int i = 0; i < 5; ++i) {
    k0[i] = h0[i] * R.w00 + h1[i] * R.w01;
    k1[i] = h0[i] * R.w01 + h1[i] * R.w11;
  }
  for (int i = 0; i < 5; ++i) t.p[i] = t.p[i] + (k0[i] * R.r0 + k1[i] * R.r1);
  for (int i = 0; i < 5; ++i)
    for (int j = 0; j <= i; ++j) t.c[ci(i, j)] = t.c[ci(i, j)] - (k0[i] * h0[j] + k1[i] * h1[j]);
}

// Rotation of the local frame by +/-20 deg (to an adjacent sector): the
// position is re-expressed in the new frame (the state then sits at the new
// x), sin(phi) turns by the angle, and the covariance is transported with the
// Jacobian d(y',z',snp')/d(y,snp): csp/csp', -sin(a) tgl/csp', -sin(a) kappa
// (a shift along the track turns its direction), csp'/csp.
template <typename Real>
bool rotate(Track<Real>& t, int dir, const Params<Real>& P) {
  const Real ca = P.rot_c;
  const Real sa = dir > 0 ? P.rot_s : -P.rot_s;
  const Real snp = t.p[2];
  const Real csp = std::sqrt(Real(1) - snp * snp);
  const Real xn = t.x * ca + t.p[0] * sa;
  const Real yn = t.p[0] * ca - t.x * sa;
  const Real sn = snp * ca - csp * sa;
  const Real cn = csp * ca + snp * sa;
  if (!(cn > Real(0)) || !(std::fabs(sn) < P.max_snp)) return false;
  const Real j00 = csp / cn;
  const Real j10 = -sa * t.p[3] / cn;
  const Real j20 = -sa * (t.p[4] * P.kb);
  const Real j22 = cn / csp;
  Real M[5][5];
  for (int i = 0; i < 5; ++i)
    for (int j = 0; j < 5; ++j) M[i][j] = t.c[ci(i, j)];
  Real A[5][5];
  for (int j = 0; j < 5; ++j) {
    A[0][j] = j00 * M[0][j];
    A[1][j] = j10 * M[0][j] + M[1][j];
    A[2][j] = j20 * M[0][j] + j22 * M[2][j];
    A[3][j] = M[3][j];
    A[4][j] = M[4][j];
  }
  for (int i = 0; i < 5; ++i) {
    t.c[ci(i, 0)] = A[i][0] * j00;
    if (i >= 1) t.c[ci(i, 1)] = A[i][0] * j10 + A[i][1];
    if (i >= 2) t.c[ci(i, 2)] = A[i][0] * j20 + A[i][2] * j22;
    if (i >= 3) t.c[ci(i, 3)] = A[i][3];
    if (i >= 4) t.c[ci(i, 4)] = A[i][4];
  }
  t.x = xn;
  t.p[0] = yn;
  t.p[2] = sn;
  return true;
}

// Seed from three clusters (increasing x): curvature of the circle
// through them (2 * cross / product of the side lengths), direction at the
// first point = chord direction turned back by the half-angle whose sine is
// kappa*chord/2, tan(lambda) = dz over the arc.
template <typename Real>
bool seed3(const Real x[3], const Real y[3], const Real z[3], const Params<Real>& P,
           Track<Real>& t) {
  const Real ax = x[1] - x[0], ay = y[1] - y[0];
  const Real bx = x[2] - x[1], by = y[2] - y[1];
  const Real cx = x[2] - x[0], cy = y[2] - y[0];
  const Real cross = ax * by - ay * bx;
  const Real la = std::sqrt(ax * ax + ay * ay);
  const Real lb = std::sqrt(bx * bx + by * by);
  const Real lc = std::sqrt(cx * cx + cy * cy);
  const Real kappa = Real(2) * cross / (la * lb * lc);
  const Real sh = kappa * lc * Real(0.5);
  if (!(std::fabs(sh) < Real(1))) return false;
  const Real ch = std::sqrt(Real(1) - sh * sh);
  const Real snc = cy / lc, csc = cx / lc;
  const Real snp = snc * ch - csc * sh;
  if (!(std::fabs(snp) < P.max_snp)) return false;
  const Real arc = lc * asinc<Real>(sh);
  t.x = x[0];
  t.p[0] = y[0];
  t.p[1] = z[0];
  t.p[2] = snp;
  t.p[3] = (z[2] - z[0]) / arc;
  t.p[4] = kappa / P.kb;
  reset_cov(t, P);
  return true;
}

// ------------------------------------------------------------- input / index
template <typename Real>
struct Frame {
  long n = 0;
  std::vector<Real> y, z;
  std::vector<int> row, sector;
  // a1: ids of each (sector,row), sorted by (z, id)
  std::vector<std::vector<int>> rows;
  int rid(int s, int r, const Params<Real>& P) const { return s * P.n_rows + r; }
};

template <typename Real>
void build_rows(Frame<Real>& F, const Params<Real>& P) {
  F.rows.assign((size_t)P.n_sectors * P.n_rows, {});
  for (long i = 0; i < F.n; ++i) F.rows[F.rid(F.sector[i], F.row[i], P)].push_back((int)i);
  for (auto& v : F.rows)
    std::sort(v.begin(), v.end(), [&](int a, int b) {
      if (F.z[a] != F.z[b]) return F.z[a] < F.z[b];
      return a < b;
    });
}

// Visit ids of row (s,r) whose z lies within [lo, hi] (a superset filter; the
// callers apply their exact tests).  brute_force visits the whole row.
template <typename Real, typename Fn>
void for_row_range(const Frame<Real>& F, const Params<Real>& P, int s, int r, Real lo, Real hi,
                   Fn fn) {
  const auto& v = F.rows[F.rid(s, r, P)];
  if (P.brute_force) {
    for (int id : v) fn(id);
    return;
  }
  auto it = std::lower_bound(v.begin(), v.end(), lo, [&](int id, Real val) { return F.z[id] < val; });
  for (; it != v.end() && F.z[*it] <= hi; ++it) fn(*it);
}

// ------------------------------------------------------------- a2 neighbours
// For a cluster c on row r (1 <= r <= n_rows-2): among clusters d on r-1 and
// u on r+1 inside the windows |dy| <= Wy, |dz| <= Wz around c, choose the pair
// whose straight line d->u passes closest to c (squared distance of c to the
// line interpolated at x_c, in y and z); ties by (u id, d id); accept if the
// distance squared is below link_chi2.
template <typename Real>
void find_links(const Frame<Real>& F, const Params<Real>& P, std::vector<int>& up,
                std::vector<int>& dn) {
  up.assign(F.n, -1);
  dn.assign(F.n, -1);
  const Real margin = Real(0.01);
  for (long c = 0; c < F.n; ++c) {
    const int r = F.row[c], s = F.sector[c];
    if (r < 1 || r > P.n_rows - 2) continue;
    const Real yc = F.y[c], zc = F.z[c];
    std::vector<int> U, D;
    auto inwin = [&](int id) {
      return std::fabs(F.y[id] - yc) <= P.link_wy && std::fabs(F.z[id] - zc) <= P.link_wz;
    };
    for_row_range(F, P, s, r + 1, zc - P.link_wz - margin, zc + P.link_wz + margin, [&](int id) {
      if (inwin(id)) U.push_back(id);
    });
    for_row_range(F, P, s, r - 1, zc - P.link_wz - margin, zc + P.link_wz + margin, [&](int id) {
      if (inwin(id)) D.push_back(id);
    });
    const Real xd = P.row_x[r - 1], xc = P.row_x[r], xu = P.row_x[r + 1];
    const Real f = (xc - xd) / (xu - xd);
    Real best = 0;
    int bu = -1, bd = -1;
    for (int u : U)
      for (int d : D) {
        const Real yp = F.y[d] + (F.y[u] - F.y[d]) * f;
        const Real zp = F.z[d] + (F.z[u] - F.z[d]) * f;
        const Real ey = yp - yc, ez = zp - zc;
        const Real d2 = ey * ey + ez * ez;
        if (!(d2 < P.link_chi2)) continue;
        if (bu < 0 || d2 < best || (d2 == best && (u < bu || (u == bu && d < bd)))) {
          best = d2; bu = u; bd = d;
        }
      }
    up[c] = bu;
    dn[c] = bd;
  }
}

// a3: keep a link only if it is mutual.
inline void clean_links(const std::vector<int>& up, const std::vector<int>& dn,
                        std::vector<int>& cu, std::vector<int>& cd) {
  const long n = (long)up.size();
  cu.assign(n, -1);
  cd.assign(n, -1);
  for (long c = 0; c < n; ++c) {
    if (up[c] >= 0 && dn[up[c]] == c) cu[c] = up[c];
    if (dn[c] >= 0 && up[dn[c]] == c) cd[c] = dn[c];
  }
}

// a4: a start hit has no lower link and a chain of at least three clusters.
inline std::vector<int> start_hits(const std::vector<int>& cu, const std::vector<int>& cd) {
  std::vector<int> s;
  for (long c = 0; c < (long)cu.size(); ++c)
    if (cd[c] < 0 && cu[c] >= 0 && cu[cu[c]] >= 0) s.push_back((int)c);
  return s;
}

// ------------------------------------------------------------- a5 tracklets
template <typename Real>
struct Tracklet {
  int start = -1;
  int n = 0;            // clusters after the downward pass (0: invalid)
  Track<Real> t{};      // parameters at the innermost cluster
  Real chi2 = 0;
  int ndf = 0;
  std::vector<int> hits;  // outermost -> innermost
};

// Best cluster on (s,r) with chi2 < follow_chi2 against the prediction (ties:
// smaller id).  The y/z box bounds are the 2x2 Mahalanobis bounds, widened.
template <typename Real>
int pick(const Frame<Real>& F, const Params<Real>& P, const Track<Real>& t, int s, int r,
         Resid<Real>* out) {
  const Real hy = std::sqrt(P.follow_chi2 * (t.c[0] + P.meas_sy2)) * Real(1.001) + Real(0.01);
  const Real hz = std::sqrt(P.follow_chi2 * (t.c[2] + P.meas_sz2)) * Real(1.001) + Real(0.01);
  int best = -1;
  Resid<Real> bres{};
  const Real ylo = t.p[0] - hy, yhi = t.p[0] + hy;
  const Real margin = Real(0.01);
  for_row_range(F, P, s, r, t.p[1] - hz - margin, t.p[1] + hz + margin, [&](int id) {
    if (!(F.y[id] >= ylo && F.y[id] <= yhi)) return;
    if (std::fabs(F.z[id] - t.p[1]) > hz) return;
    const Resid<Real> R = residual(t, F.y[id], F.z[id], P);
    if (!(R.chi2 < P.follow_chi2)) return;
    if (best < 0 || R.chi2 < bres.chi2 || (R.chi2 == bres.chi2 && id < best)) {
      best = id;
      bres = R;
    }
  });
  if (best >= 0 && out) *out = bres;
  return best;
}

template <typename Real>
Tracklet<Real> construct(const Frame<Real>& F, const Params<Real>& P, const std::vector<int>& cu,
                         int start) {
  Tracklet<Real> T;
  T.start = start;
  std::vector<int> chain;
  for (int c = start; c >= 0; c = cu[c]) chain.push_back(c);
  const int s = F.sector[start];
  // seed points: first, middle and last cluster of the chain (longest lever arm)
  const int L = (int)chain.size();
  const int sel[3] = {chain[0], chain[(L - 1) / 2], chain[L - 1]};
  Real xs[3], ys[3], zs[3];
  for (int i = 0; i < 3; ++i) {
    xs[i] = P.row_x[F.row[sel[i]]];
    ys[i] = F.y[sel[i]];
    zs[i] = F.z[sel[i]];
  }
  Track<Real> t;
  if (!seed3(xs, ys, zs, P, t)) return T;
  std::vector<int> have(P.n_rows, -1);
  // upward: along the chain, then row-by-row following
  {
    Resid<Real> R = residual(t, F.y[chain[0]], F.z[chain[0]], P);
    update(t, R);
    have[F.row[chain[0]]] = chain[0];
  }
  Track<Real> last = t;
  int top = F.row[chain[0]];
  bool alive = true;
  for (size_t i = 1; i < chain.size(); ++i) {
    const int c = chain[i];
    if (!propagate(t, P.row_x[F.row[c]], P)) { alive = false; break; }
    Resid<Real> R = residual(t, F.y[c], F.z[c], P);
    update(t, R);
    have[F.row[c]] = c;
    last = t;
    top = F.row[c];
  }
  if (alive) {
    int miss = 0;
    for (int r = top + 1; r < P.n_rows; ++r) {
      if (!propagate(t, P.row_x[r], P)) break;
      if (std::fabs(t.p[0]) > t.x * P.tan_half) break;
      Resid<Real> R;
      const int c = pick(F, P, t, s, r, &R);
      if (c >= 0) {
        update(t, R);
        have[r] = c;
        last = t;
        top = r;
        miss = 0;
      } else if (++miss >= P.max_miss) {
        break;
      }
    }
  }
  // downward: refit from the top with a reset covariance, extend below the start
  const int r0 = F.row[start];
  t = last;
  reset_cov(t, P);
  Real chi2 = 0;
  int n = 0;
  std::vector<int> hits;
  {
    const int c = have[top];
    Resid<Real> R = residual(t, F.y[c], F.z[c], P);
    chi2 = chi2 + R.chi2;
    update(t, R);
    hits.push_back(c);
    ++n;
  }
  Track<Real> inner = t;
  int miss = 0;
  for (int r = top - 1; r >= 0; --r) {
    if (!propagate(t, P.row_x[r], P)) break;
    if (std::fabs(t.p[0]) > t.x * P.tan_half) break;
    if (r >= r0) {
      const int c = have[r];
      if (c < 0) continue;
      Resid<Real> R = residual(t, F.y[c], F.z[c], P);
      chi2 = chi2 + R.chi2;
      update(t, R);
      hits.push_back(c);
      ++n;
      inner = t;
    } else {
      Resid<Real> R;
      const int c = pick(F, P, t, s, r, &R);
      if (c >= 0) {
        chi2 = chi2 + R.chi2;
        update(t, R);
        hits.push_back(c);
        ++n;
        inner = t;
        miss = 0;
      } else if (++miss >= P.max_miss) {
        break;
      }
    }
  }
  if (n < P.min_hits) return T;
  T.n = n;
  T.t = inner;
  T.chi2 = chi2;
  T.ndf = 2 * n - 5;
  T.hits = hits;
  return T;
}

// ------------------------------------------------------------- a6 selector
// Order-preserving map of a float to uint32 (larger float -> larger uint).
inline uint32_t ordered_bits(float f) {
  uint32_t u;
  std::memcpy(&u, &f, 4);
  return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}

template <typename Real>
float score_of(const Tracklet<Real>& T, const Params<Real>& P) {
  // Phase I priority: global chi2 per degree of freedom outweighs the length.
  const Real sc = Real(T.n) - P.score_w * (T.chi2 / Real(T.ndf));
  return (float)sc;
}

inline uint64_t make_key(float score, int start_id) {
  return ((uint64_t)ordered_bits(score) << 32) | (uint64_t)(0xFFFFFFFFu - (uint32_t)start_id);
}

template <typename Real>
struct Selection {
  std::vector<uint64_t> owner_key;       // per cluster
  std::vector<int> accepted;             // per tracklet (0/1)
  std::vector<std::vector<int>> kept;    // per tracklet, outer -> inner
};

template <typename Real>
Selection<Real> select(const Frame<Real>& F, const Params<Real>& P,
                       const std::vector<Tracklet<Real>>& TL) {
  Selection<Real> S;
  S.owner_key.assign(F.n, 0);
  std::vector<uint64_t> key(TL.size(), 0);
  for (size_t i = 0; i < TL.size(); ++i) {
    if (TL[i].n == 0) continue;
    key[i] = make_key(score_of(TL[i], P), TL[i].start);
    for (int c : TL[i].hits) S.owner_key[c] = std::max(S.owner_key[c], key[i]);
  }
  S.accepted.assign(TL.size(), 0);
  S.kept.assign(TL.size(), {});
  for (size_t i = 0; i < TL.size(); ++i) {
    if (TL[i].n == 0) continue;
    int kept = 0, shared = 0;
    std::vector<int> k;
    for (int c : TL[i].hits) {
      if (S.owner_key[c] == key[i]) {
        k.push_back(c);
        ++kept;
      } else if (Real(shared + 1) <= P.shared_frac * Real(kept + 1)) {
        k.push_back(c);
        ++kept;
        ++shared;
      }
    }
    if (kept >= P.min_hits) {
      S.accepted[i] = 1;
      S.kept[i] = k;
    }
  }
  return S;
}

// ------------------------------------------------------------- driver
template <typename Real>
void run_sector_tracking(const Frame<Real>& F, const Params<Real>& P, Result& res) {
  std::vector<int> up, dn, cu, cd;
  find_links(F, P, up, dn);
  clean_links(up, dn, cu, cd);
  std::vector<int> starts = start_hits(cu, cd);
  res.put("link_up", up, "i4");
  res.put("link_dn", dn, "i4");
  res.put("clean_up", cu, "i4");
  res.put("clean_dn", cd, "i4");
  res.put("start", starts, "i4");
  std::vector<Tracklet<Real>> TL(starts.size());
  for (size_t i = 0; i < starts.size(); ++i) TL[i] = construct(F, P, cu, starts[i]);
  const int R = P.n_rows;
  std::vector<int> tl_n(TL.size()), tl_ndf(TL.size()), tl_hits(TL.size() * R, -1);
  std::vector<Real> tl_par(TL.size() * 5), tl_cov(TL.size() * 15), tl_chi2(TL.size()),
      tl_x(TL.size());
  for (size_t i = 0; i < TL.size(); ++i) {
    tl_n[i] = TL[i].n;
    tl_ndf[i] = TL[i].ndf;
    tl_chi2[i] = TL[i].chi2;
    tl_x[i] = TL[i].t.x;
    for (int k = 0; k < 5; ++k) tl_par[i * 5 + k] = TL[i].t.p[k];
    for (int k = 0; k < 15; ++k) tl_cov[i * 15 + k] = TL[i].t.c[k];
    for (size_t k = 0; k < TL[i].hits.size(); ++k) tl_hits[i * R + k] = TL[i].hits[k];
  }
  res.put("tl_start", starts, "i4");
  res.put("tl_n", tl_n, "i4");
  res.put("tl_ndf", tl_ndf, "i4");
  res.put("tl_hits", tl_hits, "i4");
  res.put("tl_param", tl_par, real_name<Real>());
  res.put("tl_cov", tl_cov, real_name<Real>());
  res.put("tl_chi2", tl_chi2, real_name<Real>());
  res.put("tl_x", tl_x, real_name<Real>());
  Selection<Real> S = select(F, P, TL);
  std::vector<int> acc(TL.size()), nk(TL.size()), kept(TL.size() * R, -1);
  std::vector<uint64_t> keys(TL.size(), 0);
  for (size_t i = 0; i < TL.size(); ++i) {
    acc[i] = S.accepted[i];
    nk[i] = (int)S.kept[i].size();
    for (size_t k = 0; k < S.kept[i].size(); ++k) kept[i * R + k] = S.kept[i][k];
    if (TL[i].n) keys[i] = make_key(score_of(TL[i], P), TL[i].start);
  }
  // sector-level attachment: owner tracklet's start id if that tracklet is accepted
  std::vector<int> owner(F.n, -1);
  std::map<int, size_t> by_start;
  for (size_t i = 0; i < TL.size(); ++i) by_start[TL[i].start] = i;
  for (long c = 0; c < F.n; ++c) {
    const uint64_t k = S.owner_key[c];
    if (!k) continue;
    const int sid = (int)(0xFFFFFFFFu - (uint32_t)(k & 0xFFFFFFFFu));
    const size_t i = by_start[sid];
    if (S.accepted[i]) owner[c] = sid;
  }
  res.put("tl_key", keys, "u8");
  res.put("tl_accept", acc, "i4");
  res.put("tl_nkept", nk, "i4");
  res.put("tl_kept", kept, "i4");
  res.put("sector_owner", owner, "i4");
}

template <typename Real>
Frame<Real> make_frame(long n, const float* y, const float* z, const uint8_t* row,
                       const uint8_t* sector, const Params<Real>& P) {
  Frame<Real> F;
  F.n = n;
  F.y.resize(n); F.z.resize(n); F.row.resize(n); F.sector.resize(n);
  for (long i = 0; i < n; ++i) {
    F.y[i] = y[i]; F.z[i] = z[i]; F.row[i] = row[i]; F.sector[i] = sector[i];
  }
  build_rows(F, P);
  return F;
}

}  // namespace orc

struct orc_result {
  orc::Result r;
};

extern "C" {

int orc_track(long n, const float* y, const float* z, const uint8_t* row, const uint8_t* sector,
              const double* row_x, const orc_options* opt, int use_double, orc_result** out) {
  if (!opt || !row_x || !out || n < 0) return 1;
  for (long i = 0; i < n; ++i)
    if (row[i] >= opt->n_rows || sector[i] >= opt->n_sectors || !std::isfinite(y[i]) ||
        !std::isfinite(z[i]))
      return 2;
  auto* R = new orc_result();
  if (use_double) {
    const auto P = orc::make_params<double>(*opt, row_x);
    const auto F = orc::make_frame<double>(n, y, z, row, sector, P);
    orc::run_sector_tracking(F, P, R->r);
  } else {
    const auto P = orc::make_params<float>(*opt, row_x);
    const auto F = orc::make_frame<float>(n, y, z, row, sector, P);
    orc::run_sector_tracking(F, P, R->r);
  }
  *out = R;
  return 0;
}

// Array lookup: dtype string ("i4","f4","f8","u8") and byte size.
long orc_info(const orc_result* h, const char* name, char* dtype_out) {
  if (!h || !name) return -1;
  auto it = h->r.arrays.find(name);
  if (it == h->r.arrays.end()) return -1;
  if (dtype_out) std::strncpy(dtype_out, it->second.dtype.c_str(), 7);
  return (long)it->second.bytes.size();
}

int orc_copy(const orc_result* h, const char* name, void* dst, long cap) {
  if (!h || !name || !dst) return 1;
  auto it = h->r.arrays.find(name);
  if (it == h->r.arrays.end()) return 2;
  if ((long)it->second.bytes.size() > cap) return 3;
  if (!it->second.bytes.empty()) std::memcpy(dst, it->second.bytes.data(), it->second.bytes.size());
  return 0;
}

long orc_names(const orc_result* h, char* buf, long cap) {
  std::string s;
  for (const auto& kv : h->r.arrays) s += kv.first + "\n";
  if ((long)s.size() + 1 <= cap && buf) std::memcpy(buf, s.c_str(), s.size() + 1);
  return (long)s.size() + 1;
}

void orc_free(orc_result* h) { delete h; }

// Single model operations in FP64 (or FP32 when use_double == 0), for pins.
// op 0: propagate state io[0..4] with covariance io[5..19] from x=io[20] to x=io[21]
//       (EKF with scattering); returns 0 on success, io updated, io[20] = new x.
// op 1: Kalman update of io[0..19] with measurement (io[20], io[21]); io[22] = chi2.
// op 2: rotate io[0..19] at x=io[20] by +20 deg (io[21] > 0) or -20 deg.
// op 3: seed from points io[0..8] = x0,y0,z0,x1,y1,z1,x2,y2,z2 -> io[9..23] state,
//       io[24] = x.
int orc_op(int op, int use_double, const orc_options* opt, const double* row_x, double* io) {
  auto run = [&](auto tag) -> int {
    using Real = decltype(tag);
    const auto P = orc::make_params<Real>(*opt, row_x);
    orc::Track<Real> t{};
    if (op <= 2) {
      for (int i = 0; i < 5; ++i) t.p[i] = (Real)io[i];
      for (int i = 0; i < 15; ++i) t.c[i] = (Real)io[5 + i];
    }
    if (op == 0) {
      t.x = (Real)io[20];
      if (!orc::propagate(t, (Real)io[21], P)) return 1;
      io[20] = t.x;
    } else if (op == 1) {
      const auto R = orc::residual(t, (Real)io[20], (Real)io[21], P);
      orc::update(t, R);
      io[22] = R.chi2;
    } else if (op == 2) {
      t.x = (Real)io[20];
      if (!orc::rotate(t, io[21] > 0 ? 1 : -1, P)) return 1;
      io[20] = t.x;
    } else if (op == 3) {
      Real x[3], y[3], z[3];
      for (int i = 0; i < 3; ++i) {
        x[i] = (Real)io[3 * i]; y[i] = (Real)io[3 * i + 1]; z[i] = (Real)io[3 * i + 2];
      }
      if (!orc::seed3(x, y, z, P, t)) return 1;
      for (int i = 0; i < 5; ++i) io[9 + i] = t.p[i];
      for (int i = 0; i < 15; ++i) io[14 + i] = t.c[i];
      io[29] = t.x;
      return 0;
    } else {
      return 2;
    }
    for (int i = 0; i < 5; ++i) io[i] = t.p[i];
    for (int i = 0; i < 15; ++i) io[5 + i] = t.c[i];
    return 0;
  };
  if (!opt || !io) return 3;
  return use_double ? run(double{}) : run(float{});
}

}  // extern "C"
