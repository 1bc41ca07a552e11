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
// and the optional parts, each behind an option that is off by default:
//   seeding iterations on leftover clusters       (Sec. 3, seed_iters)
//   merging across the central electrode          (Sec. 2 merging, Sec. 1 t0; ac_merge)
//   extrapolation inward, outward, over sectors   (Sec. 3 Phase III; ext_rows)
//   online cluster removal flags                  (Sec. 4; cr_mode)
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <map>
#include <memory>
#include <string>
#include <type_traits>
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
  float max_snp;         // |sin(phi)| limit of seeding and following
  float fit_max_snp;     // |sin(phi)| limit of refits, merging and the final fit
  float score_w;
  float shared_frac;
  float merge_chi2, merge_dy, merge_dz;
  float int_chi2, final_chi2;
  float attach_margin;   // widening of the Phase II search window [cm]
  float looper_qpt;      // |q/pT| above which the fit's update runs in FP64 (0: never)
  float edge_margin;     // following stops |y| > x*tan(10 deg) + edge_margin [cm]
  float ext_chi2;        // Phase III: candidate cut of the extrapolation (2 dof)
  // online cluster removal (Sec. 4)
  float cr_qpt;          // |q/pT| above which a track is very low pT (removal class)
  float cr_protect;      // half-width of the protective tube around physics tracks [cm]
  float cr_remove;       // half-width of the removal tube around removal-class tracks [cm]
  float cr_edge;         // protection 2: distance to the sector edge counted as "at the edge" [cm]
  float cr_occ_w;        // protection 2: half-width of the occupancy window [cm]
  float cr_p2_grow;      // protection 2: factor on the protective tube
  float cr_p2_shrink;    // protection 2: factor on the removal tube
  float cr_leg_dq;       // looper legs: relative |q/pT| difference
  float cr_leg_dtgl;     // looper legs: |tan(lambda_a) + tan(lambda_b)|
  float cr_leg_dc;       // looper legs: distance of the circle centres [cm]
  int32_t max_miss;
  int32_t min_hits;
  int32_t merge_max_gap;
  int32_t inner_rows;
  int32_t cand_k;
  int32_t brute_force;  // 1: candidate search scans whole rows (self-check)
  int32_t n_rows;
  int32_t n_sectors;
  int32_t ext_rows;     // Phase III: rows searched below / above a track's end clusters (0: off)
  int32_t seed_iters;   // sector-tracking iterations, the later ones on leftover clusters (>= 1)
  int32_t cr_mode;      // cluster removal: 0 off, 1 tubes + history, 2 also protection 2
  int32_t cr_occ_max;   // protection 2: clusters in the occupancy window above which it applies
  int32_t ac_merge;     // 1: merging across the central electrode (A <-> C sides)
  int32_t edge_rows;    // following into the adjacent sector from track ends at a sector
                        // edge: rows followed beyond the end (0: off)
  int32_t edge_min;     // clusters a segment found there needs to be kept
};
// Correction map of the oracle (host memory): layout [3][n_z][n_r][n_phi].
struct orc_map {
  int32_t n_phi, n_r, n_z;
  float r_min, r_max, z_min, z_max;
  const float* coeff;
};

}

namespace orc {

// Math entry points of the templated code (overloaded for the FP64 tape type).
template <class R> inline R o_sqrt(R x) { return std::sqrt(x); }
template <class R> inline R o_fabs(R x) { return std::fabs(x); }
template <class R> inline double o_floor(R x) { return std::floor((double)x); }
template <class R> inline R detach(R x) { return x; }

// ------------------------------------------------ FP64 reverse-mode tape
// An operator-overloading tape for the refit gradient (independent of the
// hand-written adjoint of the CUDA library): every arithmetic operation on a
// Var records its operands and local partial derivatives; a reverse sweep
// accumulates adjoints.  Values are FP64.
struct Tape {
  std::vector<int> a, b;
  std::vector<double> da, db;
  int push(int ia, double ga, int ib, double gb) {
    a.push_back(ia);
    da.push_back(ga);
    b.push_back(ib);
    db.push_back(gb);
    return (int)a.size() - 1;
  }
  void clear() { a.clear(); b.clear(); da.clear(); db.clear(); }
  // adjoints of every node given the seed on node `out`
  std::vector<double> reverse(int out) const {
    std::vector<double> adj(a.size(), 0.0);
    if (out < 0) return adj;
    adj[out] = 1.0;
    for (int i = out; i >= 0; --i) {
      const double g = adj[i];
      if (g == 0.0) continue;
      if (a[i] >= 0) adj[a[i]] += g * da[i];
      if (b[i] >= 0) adj[b[i]] += g * db[i];
    }
    return adj;
  }
};

inline Tape& tape() {
  static Tape t;
  return t;
}

struct Var {
  double v = 0.0;
  int id = -1;  // -1: constant
  Var() = default;
  Var(double x) : v(x), id(-1) {}
  Var(float x) : v(x), id(-1) {}
  Var(int x) : v(x), id(-1) {}
  Var(long x) : v((double)x), id(-1) {}
  static Var node(double v, int ia, double ga, int ib, double gb) {
    Var r;
    r.v = v;
    r.id = (ia < 0 && ib < 0) ? -1 : tape().push(ia, ga, ib, gb);
    return r;
  }
  static Var leaf(double v) {
    Var r;
    r.v = v;
    r.id = tape().push(-1, 0.0, -1, 0.0);
    return r;
  }
  explicit operator double() const { return v; }
  explicit operator float() const { return (float)v; }
  explicit operator int() const { return (int)v; }
};
inline Var operator+(Var x, Var y) { return Var::node(x.v + y.v, x.id, 1.0, y.id, 1.0); }
inline Var operator-(Var x, Var y) { return Var::node(x.v - y.v, x.id, 1.0, y.id, -1.0); }
inline Var operator*(Var x, Var y) { return Var::node(x.v * y.v, x.id, y.v, y.id, x.v); }
inline Var operator/(Var x, Var y) {
  const double q = x.v / y.v;
  return Var::node(q, x.id, 1.0 / y.v, y.id, -q / y.v);
}
inline Var operator-(Var x) { return Var::node(-x.v, x.id, -1.0, -1, 0.0); }
inline bool operator<(Var x, Var y) { return x.v < y.v; }
inline bool operator>(Var x, Var y) { return x.v > y.v; }
inline bool operator<=(Var x, Var y) { return x.v <= y.v; }
inline bool operator>=(Var x, Var y) { return x.v >= y.v; }
inline bool operator==(Var x, Var y) { return x.v == y.v; }
inline bool operator!=(Var x, Var y) { return x.v != y.v; }
inline Var o_sqrt(Var x) {
  const double s = std::sqrt(x.v);
  return Var::node(s, x.id, 0.5 / s, -1, 0.0);
}
inline Var o_fabs(Var x) { return Var::node(std::fabs(x.v), x.id, x.v < 0 ? -1.0 : 1.0, -1, 0.0); }
inline double o_floor(Var x) { return std::floor(x.v); }
inline Var detach(Var x) { return Var(x.v); }

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
  if (o_fabs(u) > 0.01) return (1.0 / o_sqrt(1.0 - u * u) - std::asin(u) / u) / u;
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

// Tape versions: value and derivative of the FP64 forms.  The derivative of
// asinc_deriv is not recorded: it only enters Jacobians, which the refit
// evaluates at its frozen reference (constants on the tape).
template <> Var asinc<Var>(Var u) {
  return Var::node(asinc<double>(u.v), u.id, asinc_deriv<double>(u.v), -1, 0.0);
}
template <> Var asinc_deriv<Var>(Var u) { return Var(asinc_deriv<double>(u.v)); }
template <> const char* real_name<Var>() { return "f8"; }

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
  Real seed_c[5], meas_sy2, meas_sz2, ms_theta2, row_pitch_inv, follow_chi2, max_snp, fit_max_snp, score_w,
      shared_frac, merge_chi2, merge_dy, merge_dz, int_chi2, final_chi2, attach_margin,
      edge_margin, looper_qpt, merge_zspan, ext_chi2;
  Real cr_qpt, cr_protect, cr_remove, cr_edge, cr_occ_w, cr_p2_grow, cr_p2_shrink, cr_leg_dq,
      cr_leg_dtgl, cr_leg_dc;
  int max_miss, min_hits, merge_max_gap, inner_rows, cand_k, brute_force, n_rows, n_sectors,
      ext_rows, seed_iters, cr_mode, cr_occ_max, ac_merge, edge_rows, edge_min;
  std::vector<Real> row_x;
  std::vector<Real> sec_cos, sec_sin;  // axis of sector s mod 18: ((s mod 18) + 0.5) * 20 deg
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
  P.follow_chi2 = o.follow_chi2; P.max_snp = o.max_snp; P.fit_max_snp = o.fit_max_snp;
  P.score_w = o.score_w;
  P.shared_frac = o.shared_frac;
  P.merge_chi2 = o.merge_chi2; P.merge_dy = o.merge_dy; P.merge_dz = o.merge_dz;
  P.int_chi2 = o.int_chi2; P.final_chi2 = o.final_chi2;
  P.attach_margin = o.attach_margin;
  P.edge_margin = o.edge_margin;
  P.looper_qpt = o.looper_qpt;
  // z reach of a merge pair: (max gap + 2) rows at the steepest allowed angle
  P.merge_zspan = (Real)((double)(o.merge_max_gap + 2) *
                         (((double)row_x[o.n_rows - 1] - (double)row_x[0]) / (double)(o.n_rows - 1)) /
                         o_sqrt(1.0 - (double)o.max_snp * (double)o.max_snp));
  P.max_miss = o.max_miss; P.min_hits = o.min_hits; P.merge_max_gap = o.merge_max_gap;
  P.inner_rows = o.inner_rows; P.cand_k = o.cand_k; P.brute_force = o.brute_force;
  P.n_rows = o.n_rows; P.n_sectors = o.n_sectors;
  P.ext_chi2 = o.ext_chi2; P.ext_rows = o.ext_rows;
  P.seed_iters = o.seed_iters < 1 ? 1 : o.seed_iters;
  P.cr_qpt = o.cr_qpt; P.cr_protect = o.cr_protect; P.cr_remove = o.cr_remove;
  P.cr_edge = o.cr_edge; P.cr_occ_w = o.cr_occ_w; P.cr_p2_grow = o.cr_p2_grow;
  P.cr_p2_shrink = o.cr_p2_shrink; P.cr_leg_dq = o.cr_leg_dq; P.cr_leg_dtgl = o.cr_leg_dtgl;
  P.cr_leg_dc = o.cr_leg_dc; P.cr_mode = o.cr_mode; P.cr_occ_max = o.cr_occ_max;
  P.ac_merge = o.ac_merge;
  P.edge_rows = o.edge_rows;
  P.edge_min = o.edge_min;
  P.sec_cos.resize(18);
  P.sec_sin.resize(18);
  for (int k = 0; k < 18; ++k) {
    const double a = ((double)k + 0.5) * 20.0 * pi / 180.0;
    P.sec_cos[k] = (Real)std::cos(a);
    P.sec_sin[k] = (Real)std::sin(a);
  }
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
bool helix_step(const Real* p, Real dx, const Params<Real>& P, Step<Real>& st, Real lim) {
  const Real kappa = p[4] * P.kb;
  const Real s0 = p[2];
  const Real s1 = s0 + kappa * dx;
  if (!(o_fabs(s1) < lim)) return false;
  const Real c0 = o_sqrt(Real(1) - s0 * s0);
  const Real c1 = o_sqrt(Real(1) - s1 * s1);
  const Real N = s0 + s1;
  const Real D = c0 + c1;
  const Real t = N / D;
  const Real L1 = o_sqrt(Real(1) + t * t);
  const Real chord = dx * L1;
  const Real u = kappa * chord * Real(0.5);
  const Real ds = chord * asinc<Real>(u);
  const Real B = Real(1) / o_sqrt(Real(1) - u * u);
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
  const Real th2 = P.ms_theta2 * (o_fabs(dx) * P.row_pitch_inv);
  const Real a = Real(1) + p[3] * p[3];
  c[5] = c[5] + th2 * (Real(1) - p[2] * p[2]) * a;
  c[9] = c[9] + th2 * a * a;
}

// Extended-Kalman propagation (Jacobian at the current state) with scattering.
template <typename Real>
bool propagate(Track<Real>& t, Real xnew, const Params<Real>& P, Real lim) {
  const Real dx = xnew - t.x;
  Step<Real> st;
  if (!helix_step(t.p, dx, P, st, lim)) return false;
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

// Kalman update with the gain and covariance arithmetic in FP64 when
// `fp64`, rounded back (the float build; the double build is FP64 throughout).
template <typename Real>
void update_as(Track<Real>& t, const Resid<Real>& R, bool fp64) {
  if constexpr (std::is_same<Real, float>::value) {
    if (fp64) {
      Track<double> d;
      for (int i = 0; i < 5; ++i) d.p[i] = t.p[i];
      for (int i = 0; i < 15; ++i) d.c[i] = t.c[i];
      d.x = t.x;
      const Resid<double> Rd{R.r0, R.r1, R.w00, R.w01, R.w11, R.chi2};
      update(d, Rd);
      for (int i = 0; i < 5; ++i) t.p[i] = (float)d.p[i];
      for (int i = 0; i < 15; ++i) t.c[i] = (float)d.c[i];
      return;
    }
  }
  update(t, R);
}

// Kalman update of the refit: FP64 for low-pT loopers, judged at the update
// by the current |q/pT| > looper_qpt.
template <typename Real>
void fit_update(Track<Real>& t, const Resid<Real>& R, const Params<Real>& P) {
  if constexpr (std::is_same<Real, float>::value)
    update_as(t, R, P.looper_qpt > 0.0f && std::fabs(t.p[4]) > P.looper_qpt);
  else
    update(t, R);
}

// Rotation of the local frame by +/-20 deg (to an adjacent sector): the
// position is re-expressed in the new frame (the state then sits at the new
// x), sin(phi) turns by the angle, and the covariance is transported with the
// Jacobian d(y',z',snp')/d(y,snp): csp/csp', -sin(a) tgl/csp', -sin(a) kappa
// (a shift along the track turns its direction), csp'/csp.
template <typename Real>
bool rotate(Track<Real>& t, int dir, const Params<Real>& P, Real lim) {
  const Real ca = P.rot_c;
  const Real sa = dir > 0 ? P.rot_s : -P.rot_s;
  const Real snp = t.p[2];
  const Real csp = o_sqrt(Real(1) - snp * snp);
  const Real xn = t.x * ca + t.p[0] * sa;
  const Real yn = t.p[0] * ca - t.x * sa;
  const Real sn = snp * ca - csp * sa;
  const Real cn = csp * ca + snp * sa;
  if (!(cn > Real(0)) || !(o_fabs(sn) < lim)) return false;
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
  const Real la = o_sqrt(ax * ax + ay * ay);
  const Real lb = o_sqrt(bx * bx + by * by);
  const Real lc = o_sqrt(cx * cx + cy * cy);
  const Real kappa = Real(2) * cross / (la * lb * lc);
  const Real sh = kappa * lc * Real(0.5);
  if (!(o_fabs(sh) < Real(1))) return false;
  const Real ch = o_sqrt(Real(1) - sh * sh);
  const Real snc = cy / lc, csc = cx / lc;
  const Real snp = snc * ch - csc * sh;
  if (!(o_fabs(snp) < P.max_snp)) return false;
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
  // clusters taken by the tracks of earlier seeding iterations (empty in the
  // first): the sector tracking of a later iteration does not see them
  std::vector<uint8_t> used;
  int rid(int s, int r, const Params<Real>& P) const { return s * P.n_rows + r; }
  bool taken(long id) const { return !used.empty() && used[id]; }
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
    if (r < 1 || r > P.n_rows - 2 || F.taken(c)) continue;
    const Real yc = F.y[c], zc = F.z[c];
    std::vector<int> U, D;
    auto inwin = [&](int id) {
      return !F.taken(id) && o_fabs(F.y[id] - yc) <= P.link_wy && o_fabs(F.z[id] - zc) <= P.link_wz;
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
// Clusters marked in `excl` (if given) are not candidates.
template <typename Real>
int pick(const Frame<Real>& F, const Params<Real>& P, const Track<Real>& t, int s, int r,
         Resid<Real>* out, const std::vector<char>* excl = nullptr) {
  const Real hy = o_sqrt(P.follow_chi2 * (t.c[0] + P.meas_sy2)) * Real(1.001) + Real(0.01);
  const Real hz = o_sqrt(P.follow_chi2 * (t.c[2] + P.meas_sz2)) * Real(1.001) + Real(0.01);
  int best = -1;
  Resid<Real> bres{};
  const Real ylo = t.p[0] - hy, yhi = t.p[0] + hy;
  const Real margin = Real(0.01);
  for_row_range(F, P, s, r, t.p[1] - hz - margin, t.p[1] + hz + margin, [&](int id) {
    if (F.taken(id) || (excl && (*excl)[id])) return;
    if (!(F.y[id] >= ylo && F.y[id] <= yhi)) return;
    if (o_fabs(F.z[id] - t.p[1]) > hz) return;
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
  if (!seed3(xs, ys, zs, P, t)) { T.ndf = -1; return T; }
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
    if (!propagate(t, P.row_x[F.row[c]], P, P.max_snp)) { alive = false; break; }
    Resid<Real> R = residual(t, F.y[c], F.z[c], P);
    update(t, R);
    have[F.row[c]] = c;
    last = t;
    top = F.row[c];
  }
  if (alive) {
    int miss = 0;
    for (int r = top + 1; r < P.n_rows; ++r) {
      if (!propagate(t, P.row_x[r], P, P.max_snp)) break;
      if (o_fabs(t.p[0]) > t.x * P.tan_half + P.edge_margin) break;
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
    if (!propagate(t, P.row_x[r], P, P.max_snp)) break;
    if (o_fabs(t.p[0]) > t.x * P.tan_half + P.edge_margin) break;
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
  if (n < P.min_hits) { T.ndf = -100 - n; return T; }
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

// ---------------------------------------------------- a8 distortion map
// Uniform cubic B-spline in (u, r, z): u = sector + 0.5 + 0.5*(y/x)/tan(10 deg)
// periodic over 18 sectors, control point j at u = (j+0.5)*18/n_phi; r and z
// clamped to the map range, control point j at j-1 knot spacings.  Weights
// (1-f)^3/6, (3f^3-6f^2+4)/6, (-3f^3+3f^2+3f+1)/6, f^3/6.
template <typename Real>
struct MapR {
  bool on = false;
  int nphi = 0, nr = 0, nz = 0;
  Real rmin = 0, zmin = 0, zmax = 0, phi_scale = 0, r_scale = 0, z_scale = 0;
  const float* c = nullptr;
  const Real* cv = nullptr;  // tape leaves of the coefficients (gradient runs)
};

template <typename Real>
void spline_w(Real f, Real* w) {
  const Real g = Real(1) - f;
  const Real f2 = f * f, f3 = f2 * f;
  w[0] = g * g * g / Real(6);
  w[1] = (Real(3) * f3 - Real(6) * f2 + Real(4)) / Real(6);
  w[2] = (Real(-3) * f3 + Real(3) * f2 + Real(3) * f + Real(1)) / Real(6);
  w[3] = f3 / Real(6);
}

// Clamped span: t in [0, n-3], i <= n-4.
template <typename Real>
void spline_span(Real t, int n, int& i, Real& f) {
  const Real tmax = Real(n - 3);
  if (t < Real(0)) t = Real(0);
  if (t > tmax) t = tmax;
  i = (int)o_floor(t);
  if (i > n - 4) i = n - 4;
  f = t - Real(i);
}

// Spline weights and base indices of one point (shared by evaluation and the
// gradient scatter).
template <typename Real>
struct SplinePoint {
  int ip, ir, iz;
  Real wp[4], wr[4], wz[4];
};

template <typename Real>
SplinePoint<Real> spline_point(const MapR<Real>& M, const Params<Real>& P, int sector, Real x,
                               Real y, Real zdrift) {
  SplinePoint<Real> sp;
  const int sphi = sector % (P.n_sectors / 2);
  const Real u = (Real(sphi) + Real(0.5)) + Real(0.5) * (y / x) / P.tan_half;
  const Real tp = u * M.phi_scale - Real(0.5);
  sp.ip = (int)o_floor(tp);
  const Real fp = tp - Real(sp.ip);
  const Real r = o_sqrt(x * x + y * y);
  Real fr, fz;
  spline_span((r - M.rmin) * M.r_scale, M.nr, sp.ir, fr);
  Real zc = zdrift;
  if (zc < M.zmin) zc = M.zmin;
  if (zc > M.zmax) zc = M.zmax;
  spline_span((zc - M.zmin) * M.z_scale, M.nz, sp.iz, fz);
  spline_w(fp, sp.wp);
  spline_w(fr, sp.wr);
  spline_w(fz, sp.wz);
  return sp;
}

inline int phi_index(int ip, int e, int nphi) { return ((ip - 1 + e) % nphi + nphi) % nphi; }

template <typename Real>
void map_eval(const MapR<Real>& M, const Params<Real>& P, int sector, Real x, Real y, Real zdrift,
              Real* D) {
  D[0] = D[1] = D[2] = Real(0);
  if (!M.on) return;
  const SplinePoint<Real> sp = spline_point(M, P, sector, x, y, zdrift);
  for (int comp = 0; comp < 3; ++comp) {
    Real acc = Real(0);
    for (int a = 0; a < 4; ++a)
      for (int b = 0; b < 4; ++b) {
        const Real wzr = sp.wz[a] * sp.wr[b];
        for (int e = 0; e < 4; ++e) {
          const long idx = (((long)comp * M.nz + (sp.iz + a)) * M.nr + (sp.ir + b)) * M.nphi +
                           phi_index(sp.ip, e, M.nphi);
          const Real cval = M.cv ? M.cv[idx] : (Real)M.c[idx];
          acc = acc + wzr * sp.wp[e] * cval;
        }
      }
    D[comp] = acc;
  }
}

// ---------------------------------------------- a7 sector refit and merging
template <typename Real>
struct SectorTrack {
  int key = -1;          // input id of the tracklet's start cluster
  int tl = -1;           // index of the tracklet
  int sector = 0;
  int rmin = 0, rmax = 0;
  std::vector<int> cl;   // kept clusters, innermost first
  Track<Real> ie{}, oe{};  // states at the innermost / outermost cluster
  int link = -1;         // segment found by the edge following: key of the track it continues
  int dir = 0;           // ... beyond that track's outermost (+1) or innermost (-1) cluster
};

// Refit of a sector track at the start of merging (Sec. 3, Phase I): outward
// from the tracklet parameters, then inward, covariance reset before each.
template <typename Real>
bool sector_refit(const Frame<Real>& F, const Params<Real>& P, const Track<Real>& start,
                  SectorTrack<Real>& S) {
  Track<Real> t = start;
  reset_cov(t, P);
  for (size_t i = 0; i < S.cl.size(); ++i) {
    const int c = S.cl[i];
    if (!propagate(t, P.row_x[F.row[c]], P, P.fit_max_snp)) return false;
    update(t, residual(t, F.y[c], F.z[c], P));
  }
  S.oe = t;
  reset_cov(t, P);
  for (size_t i = S.cl.size(); i-- > 0;) {
    const int c = S.cl[i];
    if (!propagate(t, P.row_x[F.row[c]], P, P.fit_max_snp)) return false;
    update(t, residual(t, F.y[c], F.z[c], P));
  }
  S.ie = t;
  return true;
}

// d^T C^-1 d for a 5-vector through a Cholesky factorisation; -1 if C is not
// positive definite.
template <typename Real>
Real chi2_5(const Real* d, const Real* c) {
  Real L[5][5] = {};
  for (int j = 0; j < 5; ++j) {
    Real s = c[ci(j, j)];
    for (int k = 0; k < j; ++k) s = s - L[j][k] * L[j][k];
    if (!(s > Real(0))) return Real(-1);
    L[j][j] = o_sqrt(s);
    for (int i = j + 1; i < 5; ++i) {
      Real v = c[ci(i, j)];
      for (int k = 0; k < j; ++k) v = v - L[i][k] * L[j][k];
      L[i][j] = v / L[j][j];
    }
  }
  Real yv[5];
  Real chi2 = Real(0);
  for (int i = 0; i < 5; ++i) {
    Real v = d[i];
    for (int k = 0; k < i; ++k) v = v - L[i][k] * yv[k];
    yv[i] = v / L[i][i];
    chi2 = chi2 + yv[i] * yv[i];
  }
  return chi2;
}

// chi2 of the 4-vector (y, sin phi, tan lambda, q/pT) of a 5-vector difference
// with the marginal covariance (z left out), by the same Cholesky steps.
template <typename Real>
Real chi2_4z(const Real* d, const Real* c) {
  const int ix[4] = {0, 2, 3, 4};
  Real L[4][4] = {};
  for (int j = 0; j < 4; ++j) {
    Real s = c[ci(ix[j], ix[j])];
    for (int k = 0; k < j; ++k) s = s - L[j][k] * L[j][k];
    if (!(s > Real(0))) return Real(-1);
    L[j][j] = o_sqrt(s);
    for (int i = j + 1; i < 4; ++i) {
      Real v = c[ci(ix[i], ix[j])];
      for (int k = 0; k < j; ++k) v = v - L[i][k] * L[j][k];
      L[i][j] = v / L[j][j];
    }
  }
  Real yv[4];
  Real chi2 = Real(0);
  for (int i = 0; i < 4; ++i) {
    Real v = d[ix[i]];
    for (int k = 0; k < i; ++k) v = v - L[i][k] * yv[k];
    yv[i] = v / L[i][i];
    chi2 = chi2 + yv[i] * yv[i];
  }
  return chi2;
}

// Candidate pair across the central electrode (Sec. 2: the merging joins
// tracks inside sectors, then between adjacent sectors of one half, then
// across the central electrode): the outer end of A and the inner end of B in
// the same azimuthal sector on the two sides, B's innermost row 1 to
// merge_max_gap rows above A's outermost.  In continuous readout the measured
// z of the two sides differ by 2 vd t0 with t0 unknown (Sec. 1), so z stays
// out of the chi2 (4 dof, summed covariances, below merge_chi2); instead the
// sum of A's outer-end and B's inner-end z, in which t0 cancels, must lie
// within twice merge_dz + |tan lambda| * merge_zspan (the electrode lies
// between the two ends).  dz = z_A - z_B at B's x (A propagated there) is the
// shift that brings B's side into A's measured z.
template <typename Real>
bool cross_test(const Params<Real>& P, const SectorTrack<Real>& A, const SectorTrack<Real>& B,
                Real& chi2, Real& dz) {
  const int half = P.n_sectors / 2;
  if (A.sector / half == B.sector / half || A.sector % half != B.sector % half) return false;
  const int gap = B.rmin - A.rmax;
  if (gap < 1 || gap > P.merge_max_gap) return false;
  const Real zwin = P.merge_dz + o_fabs(A.oe.p[3]) * P.merge_zspan;
  if (!(o_fabs(A.oe.p[1] + B.ie.p[1]) <= zwin + zwin)) return false;
  Track<Real> t = A.oe;
  if (!propagate(t, B.ie.x, P, P.fit_max_snp)) return false;
  Real d[5], c[15];
  for (int i = 0; i < 5; ++i) d[i] = B.ie.p[i] - t.p[i];
  if (!(o_fabs(d[0]) <= P.merge_dy)) return false;
  for (int i = 0; i < 15; ++i) c[i] = t.c[i] + B.ie.c[i];
  chi2 = chi2_4z(d, c);
  dz = t.p[1] - B.ie.p[1];
  return chi2 >= Real(0) && chi2 < P.merge_chi2;
}

// Candidate pair for merging the outer end of A with the inner end of B (Sec. 2:
// merging inside a sector and between adjacent sectors of one TPC half).
template <typename Real>
bool merge_test(const Params<Real>& P, const SectorTrack<Real>& A, const SectorTrack<Real>& B,
                Real& chi2) {
  const int half = P.n_sectors / 2;
  if (A.sector / half != B.sector / half) return false;
  const int ds = ((B.sector % half) - (A.sector % half) + half) % half;
  if (ds != 0 && ds != 1 && ds != half - 1) return false;
  const int gap = B.rmin - A.rmax;
  if (gap < 1 || gap > P.merge_max_gap) return false;
  const Real zwin = P.merge_dz + o_fabs(A.oe.p[3]) * P.merge_zspan;
  if (!(o_fabs(B.ie.p[1] - A.oe.p[1]) <= zwin)) return false;
  Track<Real> t = A.oe;
  if (ds == 1 && !rotate(t, 1, P, P.fit_max_snp)) return false;
  if (ds == half - 1 && !rotate(t, -1, P, P.fit_max_snp)) return false;
  if (!propagate(t, B.ie.x, P, P.fit_max_snp)) return false;
  Real d[5], c[15];
  for (int i = 0; i < 5; ++i) d[i] = B.ie.p[i] - t.p[i];
  if (!(o_fabs(d[0]) <= P.merge_dy) || !(o_fabs(d[1]) <= P.merge_dz)) return false;
  for (int i = 0; i < 15; ++i) c[i] = t.c[i] + B.ie.c[i];
  chi2 = chi2_5(d, c);
  return chi2 >= Real(0) && chi2 < P.merge_chi2;
}

// Edge following (Sec. 2): the sector tracking cannot find very short track
// segments, so tracks that end at a sector edge close to the upper or lower
// end of the TPC are propagated into the adjacent sector before the merging,
// and a track following there picks up the segment.  Reading: from each end of
// a sector track the end state is propagated row by row away from the track
// (outward from the outermost cluster, inward from the innermost) over at most
// edge_rows rows.  Where it crosses its sector's edge (|y| > x tan 10 deg) it
// continues in the neighbouring sector of the same side on that edge (rotation,
// then the row's x in the new frame); from the crossing on, every row's best
// free cluster (chi2 < follow_chi2, ties to the smaller id; free = kept by no
// sector track) is filtered in, until max_miss rows in a row have none, the
// track leaves that sector too, or the rows run out.  An end that crosses no
// edge within edge_rows rows is left alone.  A segment of at least edge_min
// clusters becomes a sector track of the neighbouring sector (its states: the
// filter after its first and after its last cluster), linked to the track it
// continues before the merging, which leaves the two linked ends alone.

// One row step: to row r, over the sector edge once.
template <typename Real>
bool edge_step(Track<Real>& t, int& sec, bool& crossed, int r, const Params<Real>& P) {
  if (!propagate(t, P.row_x[r], P, P.max_snp)) return false;
  if (!crossed && o_fabs(t.p[0]) > t.x * P.tan_half) {
    const int half = P.n_sectors / 2;
    const int dir = t.p[0] > Real(0) ? 1 : -1;
    if (!rotate(t, dir, P, P.max_snp)) return false;
    sec = sec - sec % half + (sec % half + (dir > 0 ? 1 : half - 1)) % half;
    if (!propagate(t, P.row_x[r], P, P.max_snp)) return false;
    crossed = true;
  }
  return !(o_fabs(t.p[0]) > t.x * P.tan_half + P.edge_margin);
}

// The segment beyond one end of A (dir = +1 outer, -1 inner); false if none.
template <typename Real>
bool edge_segment(const Frame<Real>& F, const Params<Real>& P, const std::vector<char>& kept,
                  const SectorTrack<Real>& A, int dir, SectorTrack<Real>& S) {
  Track<Real> t = dir > 0 ? A.oe : A.ie;
  int sec = A.sector;
  bool crossed = false;
  int miss = 0;
  std::vector<int> hits;
  Track<Real> first{}, last{};
  const int r0 = dir > 0 ? A.rmax : A.rmin;
  for (int e = 1; e <= P.edge_rows; ++e) {
    const int r = r0 + dir * e;
    if (r < 0 || r >= P.n_rows) break;
    if (!edge_step(t, sec, crossed, r, P)) break;
    if (!crossed) continue;
    Resid<Real> R;
    const int c = pick(F, P, t, sec, r, &R, &kept);
    if (c >= 0) {
      update(t, R);
      if (hits.empty()) first = t;
      last = t;
      hits.push_back(c);
      miss = 0;
    } else if (++miss >= P.max_miss) {
      break;
    }
  }
  if ((int)hits.size() < P.edge_min) return false;
  // segment keys: the track's key plus 2^29 (inner) or 2^30 (outer), above
  // every cluster id (at most 2^29 clusters), independent of the frame size
  S.key = A.key + (dir > 0 ? (1 << 30) : (1 << 29));
  S.sector = sec;
  S.dir = dir;
  if (dir > 0) {
    S.cl = hits;
    S.ie = first;
    S.oe = last;
  } else {
    S.cl.assign(hits.rbegin(), hits.rend());
    S.ie = last;
    S.oe = first;
  }
  S.rmin = F.row[S.cl.front()];
  S.rmax = F.row[S.cl.back()];
  return true;
}

// ------------------------------------------------- a9/a10 three-iteration fit
// Linearised Kalman filter: the state is carried as reference + deviation; the
// reference (the helix of the iteration's start state) is propagated exactly,
// the deviation with the Jacobian at the reference ("the initial parameters
// are used for the linearization", Sec. 2).
template <typename Real>
struct Lin {
  Track<Real> t;  // state, covariance, x
  Real r[5];      // reference at t.x
  int sector;
};

template <typename Real>
void lin_start(Lin<Real>& L, const Track<Real>& s, int sector, const Params<Real>& P) {
  L.t = s;
  reset_cov(L.t, P);
  for (int i = 0; i < 5; ++i) L.r[i] = detach(s.p[i]);
  L.sector = sector;
}

template <typename Real>
bool lin_rotate(Lin<Real>& L, int dir, const Params<Real>& P) {
  const Real ca = P.rot_c;
  const Real sa = dir > 0 ? P.rot_s : -P.rot_s;
  const Real snp = L.r[2];
  const Real csp = o_sqrt(Real(1) - snp * snp);
  const Real xn = L.t.x * ca + L.r[0] * sa;
  const Real yn = L.r[0] * ca - L.t.x * sa;
  const Real sn = snp * ca - csp * sa;
  const Real cn = csp * ca + snp * sa;
  if (!(cn > Real(0)) || !(o_fabs(sn) < P.fit_max_snp)) return false;
  const Real j00 = csp / cn;
  const Real j10 = -sa * L.r[3] / cn;
  const Real j20 = -sa * (L.r[4] * P.kb);
  const Real j22 = cn / csp;
  const Real d0 = L.t.p[0] - L.r[0], d1 = L.t.p[1] - L.r[1], d2 = L.t.p[2] - L.r[2];
  // covariance: same transport as the extended filter's rotation
  Real M[5][5];
  for (int i = 0; i < 5; ++i)
    for (int j = 0; j < 5; ++j) M[i][j] = L.t.c[ci(i, j)];
  Real A[5][5];
  for (int j = 0; j < 5; ++j) {
    A[0][j] = j00 * M[0][j];
    A[1][j] = j10 * M[0][j] + M[1][j];
    A[2][j] = j20 * M[0][j] + j22 * M[2][j];
    A[3][j] = M[3][j];
    A[4][j] = M[4][j];
  }
  for (int i = 0; i < 5; ++i) {
    L.t.c[ci(i, 0)] = A[i][0] * j00;
    if (i >= 1) L.t.c[ci(i, 1)] = A[i][0] * j10 + A[i][1];
    if (i >= 2) L.t.c[ci(i, 2)] = A[i][0] * j20 + A[i][2] * j22;
    if (i >= 3) L.t.c[ci(i, 3)] = A[i][3];
    if (i >= 4) L.t.c[ci(i, 4)] = A[i][4];
  }
  L.r[0] = yn;
  L.r[2] = sn;
  L.t.x = xn;
  L.t.p[0] = L.r[0] + j00 * d0;
  L.t.p[1] = L.r[1] + (j10 * d0 + d1);
  L.t.p[2] = L.r[2] + (j20 * d0 + j22 * d2);
  return true;
}

template <typename Real>
bool lin_propagate(Lin<Real>& L, Real xnew, const Params<Real>& P) {
  const Real dx = xnew - L.t.x;
  Step<Real> st;
  if (!helix_step(L.r, dx, P, st, P.fit_max_snp)) return false;
  const Real d0 = L.t.p[0] - L.r[0], d1 = L.t.p[1] - L.r[1], d2 = L.t.p[2] - L.r[2];
  const Real d3 = L.t.p[3] - L.r[3], d4 = L.t.p[4] - L.r[4];
  for (int i = 0; i < 3; ++i) L.r[i] = st.p[i];
  L.t.p[0] = L.r[0] + (d0 + st.f02 * d2 + st.f04 * d4);
  L.t.p[1] = L.r[1] + (d1 + st.f12 * d2 + st.f13 * d3 + st.f14 * d4);
  L.t.p[2] = L.r[2] + (d2 + st.f24 * d4);
  cov_transport(L.t.c, st);
  add_ms(L.t.c, L.r, dx, P);
  L.t.x = xnew;
  return true;
}

template <typename Real>
bool lin_goto(Lin<Real>& L, int sector, Real x, const Params<Real>& P) {
  if (sector != L.sector) {
    const int half = P.n_sectors / 2;
    const int ds = ((sector % half) - (L.sector % half) + half) % half;
    if (ds == 1) {
      if (!lin_rotate(L, 1, P)) return false;
    } else if (ds == half - 1) {
      if (!lin_rotate(L, -1, P)) return false;
    } else if (ds != 0) {
      return false;
    }
    // ds == 0: the same azimuthal sector on the other side of the central
    // electrode, whose local frame is the same
    L.sector = sector;
  }
  return lin_propagate(L, x, P);
}

// Distortion-corrected measurement of cluster (y, z) on the pad row at x,
// projected back onto the row along the reference helix:
// m = (y + Dy, z + Dz) - [ref(x + Dx) - ref(x)].
template <typename Real>
bool corrected(const MapR<Real>& M, const Params<Real>& P, int sector, Real x, Real y, Real z,
               Real z0, const Real* ref, Real& my, Real& mz) {
  Real D[3];
  map_eval(M, P, sector, x, y, z - z0, D);
  my = y + D[1];
  mz = z + D[2];
  if (D[0] != Real(0)) {
    Step<Real> st;
    if (!helix_step(ref, D[0], P, st, P.fit_max_snp)) return false;
    my = my - (st.p[0] - ref[0]);
    mz = mz - (st.p[1] - ref[1]);
  }
  return true;
}

// 2x2 symmetric inverse.
template <typename Real>
void inv2(Real a00, Real a01, Real a11, Real& i00, Real& i01, Real& i11) {
  const Real idet = Real(1) / (a00 * a11 - a01 * a01);
  i00 = a11 * idet;
  i01 = -a01 * idet;
  i11 = a00 * idet;
}

// Weighted mean of two (y,z) estimates (two-filter interpolation).
template <typename Real>
struct Interp {
  Real y, z, c00, c01, c11;
};

template <typename Real>
Interp<Real> interpolate(const Real* a, const Real* b) {
  // a, b: y, z, cyy, czy, czz
  Real wa00, wa01, wa11, wb00, wb01, wb11;
  inv2(a[2], a[3], a[4], wa00, wa01, wa11);
  inv2(b[2], b[3], b[4], wb00, wb01, wb11);
  Interp<Real> I;
  inv2(wa00 + wb00, wa01 + wb01, wa11 + wb11, I.c00, I.c01, I.c11);
  const Real v0 = (wa00 * a[0] + wa01 * a[1]) + (wb00 * b[0] + wb01 * b[1]);
  const Real v1 = (wa01 * a[0] + wa11 * a[1]) + (wb01 * b[0] + wb11 * b[1]);
  I.y = I.c00 * v0 + I.c01 * v1;
  I.z = I.c01 * v0 + I.c11 * v1;
  return I;
}

template <typename Real>
Real chi2_interp(const Interp<Real>& I, Real my, Real mz, const Params<Real>& P) {
  Real w00, w01, w11;
  inv2(I.c00 + P.meas_sy2, I.c01, I.c11 + P.meas_sz2, w00, w01, w11);
  const Real r0 = my - I.y, r1 = mz - I.z;
  return r0 * (w00 * r0 + w01 * r1) + r1 * (w01 * r0 + w11 * r1);
}

template <typename Real>
struct Station {
  int sector, row, cl;  // cl: cluster id or -1 (empty inner row)
};

template <typename Real>
struct FitTrack {
  int key;
  std::vector<Station<Real>> st;
  Track<Real> outer;       // start of iteration 1 (state at the last station)
  Real z0;                 // drift-coordinate offset for the map lookup
  // results
  std::vector<int> flag;   // per station: interpolation-rejected (iteration 2)
  std::vector<int> ncand;
  std::vector<int> cand;   // [station][cand_k]
  std::vector<Real> cchi;  // [station][cand_k]
  std::vector<int> assigned;
  bool looper = false;     // the final fit's updates run in FP64 (low-pT looper)
  int n_ext = 0;           // Phase III: rows extrapolated below the innermost station;
                           // their candidate slots follow the stations' in ncand/cand/cchi
  int n_out = 0;           // Phase III: rows extrapolated above the outermost station; their
                           // slots follow the ext_rows inward ones
  std::vector<int> ext_sec;  // sector of each extrapolated row (inward e, then ext_rows + e)
  bool ok = true;
  int fail_at = -1;        // diagnostics: 100*iteration + station of a failed step
  Track<Real> out{};
  int out_sector = 0;
  Real chi2 = 0;
  int n = 0;
  std::vector<int> used;   // clusters of iteration 3, innermost first
  std::vector<int> seg;    // sector tracks of the chain, first to last
  int side0 = 0;           // TPC side of the first segment
  Real zshift = 0;         // z shift of the clusters on the other side (merged across the
                           // central electrode): their measured z + zshift is in the first
                           // side's measured z
};

// Measured z of cluster id on sector `sector` in the frame of track T's first side.
template <typename Real>
Real track_z(const Frame<Real>& F, const Params<Real>& P, const FitTrack<Real>& T, int sector,
             int id) {
  const int half = P.n_sectors / 2;
  return T.zshift != Real(0) && (sector / half) % 2 != T.side0 ? F.z[id] + T.zshift : F.z[id];
}

// Shift of the window centre cz (first side's frame) into the measured z of `sector`.
template <typename Real>
Real window_z(const Params<Real>& P, const FitTrack<Real>& T, int sector, Real cz) {
  const int half = P.n_sectors / 2;
  return T.zshift != Real(0) && (sector / half) % 2 != T.side0 ? cz - T.zshift : cz;
}

// One three-iteration fit (Sec. 3, Phase I, with the Phase II candidate search
// when `phase2`): iteration 1 inward stores the predicted (y,z) and covariance
// at every station; iteration 2 outward interpolates with them, flags clusters
// with chi2 > int_chi2 and (phase2) collects up to cand_k candidates on inner
// rows; iteration 3 inward uses the surviving / assigned clusters with a
// simple chi2 cut.  Iteration 3 runs in fit_iteration3 after the second
// ambiguity solving.
// Phase III (Sec. 3): from the state at the innermost station after
// iteration 1 the track is extrapolated inward, from the state at the
// outermost station after iteration 2 outward, row by row over at most
// ext_rows rows of the same sector (stopping where the propagation fails or
// the track leaves the sector); every cluster of a row whose chi2 to the
// prediction is below ext_chi2 -- the stricter cut of the extrapolation --
// becomes a candidate, except clusters already held by a station outside the
// inner region of some track (`fixed`).  The candidates join the second
// ambiguity solving; iteration 3 continues over the inward rows and takes the
// outward ones through a forward extrapolation of the iteration-2 end state.
//
// Phase III candidates of one extrapolated row r of sector sec into slot
// `slot`: every cluster of the row not held by a station outside the inner
// region of some track (`fixed`) whose chi2 to the prediction E is below
// ext_chi2 -- the stricter cut of the extrapolation --, the best cand_k by
// (chi2, id).
template <typename Real>
void ext_row_candidates(const Frame<Real>& F, const Params<Real>& P, const MapR<Real>& M,
                        const std::vector<char>& fixed, FitTrack<Real>& T, const Lin<Real>& E,
                        int sec, int r, size_t slot) {
  // window centre: the prediction moved back by the map's shift there
  Real cy, cz;
  {
    Real D[3];
    map_eval(M, P, sec, E.t.x, E.t.p[0], E.t.p[1] - T.z0, D);
    Real sy = D[1], sz = D[2];
    if (D[0] != Real(0)) {
      Step<Real> stp;
      if (helix_step(E.r, D[0], P, stp, P.fit_max_snp)) {
        sy = sy - (stp.p[0] - E.r[0]);
        sz = sz - (stp.p[1] - E.r[1]);
      }
    }
    cy = E.t.p[0] - sy;
    cz = E.t.p[1] - sz;
  }
  const Real wy = o_sqrt(P.ext_chi2 * (E.t.c[0] + P.meas_sy2)) * Real(1.001) + P.attach_margin;
  const Real wz = o_sqrt(P.ext_chi2 * (E.t.c[2] + P.meas_sz2)) * Real(1.001) + P.attach_margin;
  std::vector<std::pair<Real, int>> cands;
  const Real czm = window_z(P, T, sec, cz);  // the row's measured z
  for_row_range(F, P, sec, r, czm - wz - Real(0.01), czm + wz + Real(0.01), [&](int id) {
    if (fixed[id]) return;
    if (!(o_fabs(F.y[id] - cy) <= wy && o_fabs(F.z[id] - czm) <= wz)) return;
    Real my, mz;
    if (!corrected(M, P, sec, E.t.x, F.y[id], track_z(F, P, T, sec, id), T.z0, E.r, my, mz))
      return;
    const Real c2 = residual(E.t, my, mz, P).chi2;
    if (c2 < P.ext_chi2) cands.push_back({c2, id});
  });
  std::sort(cands.begin(), cands.end(), [](const auto& u, const auto& v) {
    return u.first < v.first || (u.first == v.first && u.second < v.second);
  });
  const int nc = std::min((int)cands.size(), P.cand_k);
  T.ncand[slot] = nc;
  for (int j = 0; j < nc; ++j) {
    T.cand[slot * P.cand_k + j] = cands[j].second;
    T.cchi[slot * P.cand_k + j] = cands[j].first;
  }
}

// One row step of the Phase III extrapolation, also over sector boundaries
// (Sec. 3): to row r in the current sector; beyond the sector's edge there
// (|y| > x tan 10 deg) the track continues in the neighbouring sector of the
// same side on that edge (rotation, then the row's x in the new frame), and
// stops if it still lies beyond that sector's edge plus edge_margin.
template <typename Real>
bool ext_step(Lin<Real>& E, int& sec, int r, const Params<Real>& P) {
  if (!lin_goto(E, sec, P.row_x[r], P)) return false;
  if (o_fabs(E.t.p[0]) > E.t.x * P.tan_half) {
    const int half = P.n_sectors / 2;
    const int base = sec - sec % half;
    const int nsec = base + (sec % half + (E.t.p[0] > Real(0) ? 1 : half - 1)) % half;
    if (!lin_goto(E, nsec, P.row_x[r], P)) return false;
    sec = nsec;
  }
  return !(o_fabs(E.t.p[0]) > E.t.x * P.tan_half + P.edge_margin);
}

// Phase III (Sec. 3) inward: from the state after iteration 1 at the
// innermost station, row by row over at most ext_rows rows below it.
template <typename Real>
void extrapolate_inward(const Frame<Real>& F, const Params<Real>& P, const MapR<Real>& M,
                        const std::vector<char>& fixed, FitTrack<Real>& T, Lin<Real> E) {
  const int ns = (int)T.st.size();
  int sec = T.st[0].sector;
  const int r_first = T.st[0].row;
  T.n_ext = 0;
  for (int e = 0; e < P.ext_rows && r_first - 1 - e >= 0; ++e) {
    const int r = r_first - 1 - e;
    if (!ext_step(E, sec, r, P)) break;
    ext_row_candidates(F, P, M, fixed, T, E, sec, r, (size_t)ns + e);
    T.ext_sec[e] = sec;
    T.n_ext = e + 1;
  }
}

// Phase III outward: from the state after iteration 2 at the outermost
// station, the same over at most ext_rows rows above it.
template <typename Real>
void extrapolate_outward(const Frame<Real>& F, const Params<Real>& P, const MapR<Real>& M,
                         const std::vector<char>& fixed, FitTrack<Real>& T, Lin<Real> E) {
  const int ns = (int)T.st.size();
  int sec = T.st[ns - 1].sector;
  const int r_last = T.st[ns - 1].row;
  T.n_out = 0;
  for (int e = 0; e < P.ext_rows && r_last + 1 + e < P.n_rows; ++e) {
    const int r = r_last + 1 + e;
    if (!ext_step(E, sec, r, P)) break;
    ext_row_candidates(F, P, M, fixed, T, E, sec, r, (size_t)ns + P.ext_rows + e);
    T.ext_sec[P.ext_rows + e] = sec;
    T.n_out = e + 1;
  }
}

template <typename Real>
void fit_iterations12(const Frame<Real>& F, const Params<Real>& P, const MapR<Real>& M,
                      const std::vector<char>& fixed, FitTrack<Real>& T, bool phase2,
                      std::vector<Real>& store, Track<Real>& it2_end) {
  const int ns = (int)T.st.size();
  const int nslot = ns + (phase2 ? 2 * P.ext_rows : 0);
  store.assign((size_t)ns * 5, Real(0));
  T.flag.assign(ns, 0);
  T.ncand.assign(nslot, 0);
  T.ext_sec.assign(phase2 ? 2 * P.ext_rows : 0, -1);
  T.cand.assign((size_t)nslot * P.cand_k, -1);
  T.cchi.assign((size_t)nslot * P.cand_k, Real(0));
  Lin<Real> L;
  // iteration 1: inward
  lin_start(L, T.outer, T.st[ns - 1].sector, P);
  for (int k = ns - 1; k >= 0; --k) {
    const Station<Real>& s = T.st[k];
    if (k != ns - 1 && !lin_goto(L, s.sector, P.row_x[s.row], P)) {
      T.ok = false;
      T.fail_at = 1000 + k;
      return;
    }
    Real* sv = &store[(size_t)k * 5];
    sv[0] = L.t.p[0]; sv[1] = L.t.p[1]; sv[2] = L.t.c[0]; sv[3] = L.t.c[1]; sv[4] = L.t.c[2];
    if (s.cl >= 0) {
      Real my, mz;
      if (!corrected(M, P, s.sector, L.t.x, F.y[s.cl], track_z(F, P, T, s.sector, s.cl), T.z0,
                     L.r, my, mz)) {
        T.ok = false;
        return;
      }
      update_as(L.t, residual(L.t, my, mz, P), T.looper);
    }
  }
  if (phase2 && P.ext_rows > 0) extrapolate_inward(F, P, M, fixed, T, L);
  // iteration 2: outward
  const Track<Real> s1 = L.t;
  lin_start(L, s1, T.st[0].sector, P);
  for (int k = 0; k < ns; ++k) {
    const Station<Real>& s = T.st[k];
    if (k != 0 && !lin_goto(L, s.sector, P.row_x[s.row], P)) {
      T.ok = false;
      T.fail_at = 2000 + k;
      return;
    }
    const Real a[5] = {L.t.p[0], L.t.p[1], L.t.c[0], L.t.c[1], L.t.c[2]};
    const Interp<Real> I = interpolate(a, &store[(size_t)k * 5]);
    const bool inner = phase2 && s.row < P.inner_rows;
    if (s.cl >= 0 && !inner) {
      Real my, mz;
      if (!corrected(M, P, s.sector, L.t.x, F.y[s.cl], track_z(F, P, T, s.sector, s.cl), T.z0,
                     L.r, my, mz)) {
        T.ok = false;
        return;
      }
      T.flag[k] = chi2_interp(I, my, mz, P) > P.int_chi2 ? 1 : 0;
    }
    if (inner) {
      // Phase II: every cluster of the row compatible with the interpolation
      Real cy = I.y, cz = I.z;
      {
        Real D[3];
        map_eval(M, P, s.sector, L.t.x, I.y, I.z - T.z0, D);
        Real sy = D[1], sz = D[2];
        if (D[0] != Real(0)) {
          Step<Real> stp;
          if (helix_step(L.r, D[0], P, stp, P.fit_max_snp)) {
            sy = sy - (stp.p[0] - L.r[0]);
            sz = sz - (stp.p[1] - L.r[1]);
          }
        }
        cy = I.y - sy;
        cz = I.z - sz;
      }
      const Real wy = o_sqrt(P.int_chi2 * (I.c00 + P.meas_sy2)) * Real(1.001) + P.attach_margin;
      const Real wz = o_sqrt(P.int_chi2 * (I.c11 + P.meas_sz2)) * Real(1.001) + P.attach_margin;
      std::vector<std::pair<Real, int>> cands;
      const Real czm = window_z(P, T, s.sector, cz);  // the row's measured z
      for_row_range(F, P, s.sector, s.row, czm - wz - Real(0.01), czm + wz + Real(0.01), [&](int id) {
        if (!(o_fabs(F.y[id] - cy) <= wy && o_fabs(F.z[id] - czm) <= wz)) return;
        Real my, mz;
        if (!corrected(M, P, s.sector, L.t.x, F.y[id], track_z(F, P, T, s.sector, id), T.z0, L.r,
                       my, mz))
          return;
        const Real c2 = chi2_interp(I, my, mz, P);
        if (c2 < P.int_chi2) cands.push_back({c2, id});
      });
      std::sort(cands.begin(), cands.end(), [](const auto& u, const auto& v) {
        return u.first < v.first || (u.first == v.first && u.second < v.second);
      });
      const int nc = std::min((int)cands.size(), P.cand_k);
      T.ncand[k] = nc;
      for (int j = 0; j < nc; ++j) {
        T.cand[(size_t)k * P.cand_k + j] = cands[j].second;
        T.cchi[(size_t)k * P.cand_k + j] = cands[j].first;
      }
    }
    if (s.cl >= 0) {
      Real my, mz;
      if (!corrected(M, P, s.sector, L.t.x, F.y[s.cl], track_z(F, P, T, s.sector, s.cl), T.z0,
                     L.r, my, mz)) {
        T.ok = false;
        return;
      }
      update_as(L.t, residual(L.t, my, mz, P), T.looper);
    }
  }
  it2_end = L.t;
  if (phase2 && P.ext_rows > 0) extrapolate_outward(F, P, M, fixed, T, L);
}

template <typename Real>
void fit_iteration3(const Frame<Real>& F, const Params<Real>& P, const MapR<Real>& M,
                    FitTrack<Real>& T, bool phase2, const Track<Real>& start) {
  const int ns = (int)T.st.size();
  Lin<Real> L;
  lin_start(L, start, T.st[ns - 1].sector, P);
  T.chi2 = Real(0);
  T.n = 0;
  T.used.clear();
  bool have = false, reached = true;
  auto take = [&](int sector, int c) {
    Real my, mz;
    if (!corrected(M, P, sector, L.t.x, F.y[c], track_z(F, P, T, sector, c), T.z0, L.r, my, mz))
      return;
    const Resid<Real> R = residual(L.t, my, mz, P);
    if (R.chi2 > P.final_chi2) return;
    T.chi2 = T.chi2 + R.chi2;
    update_as(L.t, R, T.looper);
    ++T.n;
    T.used.push_back(c);
    T.out = L.t;
    T.out_sector = L.sector;
    have = true;
  };
  // Phase III outward rows: each assigned cluster is tested (simple cut) and
  // filtered against a forward extrapolation of the iteration-2 end state
  // (its own covariance, not reset), so that it joins the track without
  // moving the fit of the stations; they precede the stations in the list
  std::vector<int> outc;
  if (T.n_out > 0) {
    const size_t o0 = (size_t)ns + P.ext_rows;
    Lin<Real> E;
    E.t = start;
    for (int i = 0; i < 5; ++i) E.r[i] = detach(start.p[i]);
    E.sector = T.st[ns - 1].sector;
    for (int e = 0; e < T.n_out; ++e) {
      const int sec_out = T.ext_sec[P.ext_rows + e];
      if (!lin_goto(E, sec_out, P.row_x[T.st[ns - 1].row + 1 + e], P)) break;
      const int c = T.assigned[o0 + e];
      if (c < 0) continue;
      Real my, mz;
      if (!corrected(M, P, sec_out, E.t.x, F.y[c], track_z(F, P, T, sec_out, c), T.z0, E.r, my,
                     mz))
        continue;
      const Resid<Real> R = residual(E.t, my, mz, P);
      if (R.chi2 > P.final_chi2) continue;
      T.chi2 = T.chi2 + R.chi2;
      update_as(E.t, R, T.looper);
      ++T.n;
      outc.push_back(c);
    }
  }
  for (size_t i = outc.size(); i-- > 0;) T.used.push_back(outc[i]);
  // the stations inward, then the rows extrapolated below the innermost one
  for (int k = ns - 1; k >= -T.n_ext; --k) {
    int sector, row, c;
    if (k >= 0) {
      const Station<Real>& s = T.st[k];
      sector = s.sector;
      row = s.row;
      const bool inner = phase2 && s.row < P.inner_rows;
      c = inner ? T.assigned[k] : (T.flag[k] ? -1 : s.cl);
    } else {
      sector = T.ext_sec[-1 - k];
      row = T.st[0].row + k;
      c = T.assigned[ns - 1 - k];
    }
    if (k != ns - 1 && !lin_goto(L, sector, P.row_x[row], P)) {
      reached = false;
      break;
    }
    if (c >= 0) take(sector, c);
  }
  (void)reached;
  std::reverse(T.used.begin(), T.used.end());
  if (!have) T.n = 0;
}

// Station list of a merged track: every cluster (segments in order, rows
// increasing) plus the empty rows below inner_rows between two clusters of
// the same sector.
template <typename Real>
std::vector<Station<Real>> make_stations(const Frame<Real>& F, const Params<Real>& P,
                                         const std::vector<int>& cl, bool phase2) {
  std::vector<Station<Real>> st;
  for (size_t i = 0; i < cl.size(); ++i) {
    const int c = cl[i];
    if (phase2 && i > 0) {
      const int pc = cl[i - 1];
      if (F.sector[pc] == F.sector[c])
        for (int r = F.row[pc] + 1; r < F.row[c] && r < P.inner_rows; ++r)
          st.push_back({F.sector[c], r, -1});
    }
    st.push_back({F.sector[c], F.row[c], c});
  }
  return st;
}

// Second ambiguity solving (Sec. 3, Phase II): in round k every cluster still
// free goes to the best (chi2, track key) among the (track, row) pairs still
// without an assigned cluster that offer it as their k-th candidate.
template <typename Real>
void second_ambiguity(std::vector<FitTrack<Real>>& FT, const Params<Real>& P) {
  std::map<int, uint64_t> bid;
  std::map<int, bool> taken;
  for (auto& T : FT) T.assigned.assign(T.ncand.size(), -1);
  for (int k = 0; k < P.cand_k; ++k) {
    bid.clear();
    for (auto& T : FT) {
      if (!T.ok) continue;
      for (size_t s = 0; s < T.ncand.size(); ++s) {
        if (T.assigned[s] >= 0 || T.ncand[s] <= k) continue;
        const int c = T.cand[s * P.cand_k + k];
        if (taken.count(c)) continue;
        const uint64_t key = ((uint64_t)ordered_bits((float)T.cchi[s * P.cand_k + k]) << 32) |
                             (uint64_t)(uint32_t)T.key;
        auto it = bid.find(c);
        if (it == bid.end() || key < it->second) bid[c] = key;
      }
    }
    for (auto& T : FT) {
      if (!T.ok) continue;
      for (size_t s = 0; s < T.ncand.size(); ++s) {
        if (T.assigned[s] >= 0 || T.ncand[s] <= k) continue;
        const int c = T.cand[s * P.cand_k + k];
        if (taken.count(c)) continue;
        const uint64_t key = ((uint64_t)ordered_bits((float)T.cchi[s * P.cand_k + k]) << 32) |
                             (uint64_t)(uint32_t)T.key;
        if (bid[c] == key) T.assigned[s] = c;
      }
    }
    for (auto& kv : bid) taken[kv.first] = true;
  }
}

// ------------------------------------------- a12 refit with fixed clusters
// Refit of given tracks whose cluster lists are fixed.  An extended-Kalman
// pass outward over the uncorrected clusters, from the input parameters,
// gives the start of iteration 1 (independent of the map); iterations 1-3
// follow the final fit without the Phase II search.  With `frozen`, the
// references of iterations 2 and 3 and the discrete decisions (interpolation
// flags, the iteration-3 cut) are taken from a previous call, so the summed
// chi2 is a smooth function of the map: the function whose gradient the
// adjoint computes.
template <typename Real>
struct RefitIO {
  std::vector<Station<Real>> st;  // cluster stations, innermost first
  Real in_p[5];
  Real in_x;
  int in_sector = 0;
  double ref2[5] = {0, 0, 0, 0, 0}, ref3[5] = {0, 0, 0, 0, 0};
  std::vector<int> flag, acc;
  bool ok = false;
  Real chi2 = Real(0);
  int n = 0;
  Track<Real> out{};
  int out_sector = 0;
  Real zshift = Real(0);  // z shift of the clusters on the side other than side0's
  int side0 = 0;          // side of the innermost cluster
};

template <typename Real>
void lin_start2(Lin<Real>& L, const Track<Real>& s, const double* ref, int sector,
                const Params<Real>& P) {
  L.t = s;
  reset_cov(L.t, P);
  for (int i = 0; i < 5; ++i) L.r[i] = Real(ref[i]);
  L.sector = sector;
}

template <typename Real>
void refit_track(const Frame<Real>& F, const Params<Real>& P, const MapR<Real>& M,
                 RefitIO<Real>& R, bool frozen) {
  const int ns = (int)R.st.size();
  R.ok = false;
  R.chi2 = Real(0);
  R.n = 0;
  if (ns < 1) return;
  const int half = P.n_sectors / 2;
  const Real z0 = R.in_p[1] - R.in_p[3] * o_sqrt(R.in_x * R.in_x + R.in_p[0] * R.in_p[0]);
  // measured z of a station's cluster in the frame of the innermost cluster's side
  auto zof = [&](const Station<Real>& s) {
    return R.zshift != Real(0) && (s.sector / half) % 2 != R.side0 ? F.z[s.cl] + R.zshift
                                                                    : F.z[s.cl];
  };
  // start of iteration 1: extended-Kalman pass outward, uncorrected clusters
  Track<Real> t;
  for (int i = 0; i < 5; ++i) t.p[i] = R.in_p[i];
  t.x = R.in_x;
  reset_cov(t, P);
  int sec = R.in_sector;
  for (int k = 0; k < ns; ++k) {
    const Station<Real>& s = R.st[k];
    if (s.sector != sec) {
      // ds == 0: the same azimuthal sector across the central electrode
      const int ds = ((s.sector % half) - (sec % half) + half) % half;
      if (ds != 0 && ds != 1 && ds != half - 1) return;
      if (ds != 0 && !rotate(t, ds == 1 ? 1 : -1, P, P.fit_max_snp)) return;
      sec = s.sector;
    }
    if (!propagate(t, P.row_x[s.row], P, P.fit_max_snp)) return;
    update(t, residual(t, F.y[s.cl], zof(s), P));
  }
  // iteration 1: inward, predictions stored
  std::vector<Real> store((size_t)ns * 5);
  Lin<Real> L;
  lin_start(L, t, R.st[ns - 1].sector, P);
  for (int k = ns - 1; k >= 0; --k) {
    const Station<Real>& s = R.st[k];
    if (k != ns - 1 && !lin_goto(L, s.sector, P.row_x[s.row], P)) return;
    Real* sv = &store[(size_t)k * 5];
    sv[0] = L.t.p[0]; sv[1] = L.t.p[1]; sv[2] = L.t.c[0]; sv[3] = L.t.c[1]; sv[4] = L.t.c[2];
    Real my, mz;
    if (!corrected(M, P, s.sector, L.t.x, F.y[s.cl], zof(s), z0, L.r, my, mz)) return;
    fit_update(L.t, residual(L.t, my, mz, P), P);
  }
  // iteration 2: outward, interpolation flags
  {
    const Track<Real> s1 = L.t;
    if (!frozen) {
      for (int i = 0; i < 5; ++i) R.ref2[i] = (double)s1.p[i];
      R.flag.assign(ns, 0);
    }
    lin_start2(L, s1, R.ref2, R.st[0].sector, P);
  }
  for (int k = 0; k < ns; ++k) {
    const Station<Real>& s = R.st[k];
    if (k != 0 && !lin_goto(L, s.sector, P.row_x[s.row], P)) return;
    const Real a[5] = {L.t.p[0], L.t.p[1], L.t.c[0], L.t.c[1], L.t.c[2]};
    const Interp<Real> I = interpolate(a, &store[(size_t)k * 5]);
    Real my, mz;
    if (!corrected(M, P, s.sector, L.t.x, F.y[s.cl], zof(s), z0, L.r, my, mz)) return;
    if (!frozen) R.flag[k] = chi2_interp(I, my, mz, P) > P.int_chi2 ? 1 : 0;
    fit_update(L.t, residual(L.t, my, mz, P), P);
  }
  // iteration 3: inward, simple cut
  {
    const Track<Real> s2 = L.t;
    if (!frozen) {
      for (int i = 0; i < 5; ++i) R.ref3[i] = (double)s2.p[i];
      R.acc.assign(ns, 0);
    }
    lin_start2(L, s2, R.ref3, R.st[ns - 1].sector, P);
  }
  for (int k = ns - 1; k >= 0; --k) {
    const Station<Real>& s = R.st[k];
    if (k != ns - 1 && !lin_goto(L, s.sector, P.row_x[s.row], P)) break;
    if (R.flag[k]) continue;
    Real my, mz;
    if (!corrected(M, P, s.sector, L.t.x, F.y[s.cl], zof(s), z0, L.r, my, mz)) continue;
    const Resid<Real> Rs = residual(L.t, my, mz, P);
    const bool accept = frozen ? R.acc[k] != 0 : !(Rs.chi2 > P.final_chi2);
    if (!frozen) R.acc[k] = accept ? 1 : 0;
    if (!accept) continue;
    R.chi2 = R.chi2 + Rs.chi2;
    fit_update(L.t, Rs, P);
    ++R.n;
    R.out = L.t;
    R.out_sector = L.sector;
  }
  R.ok = R.n > 0;
}

// ------------------------------------------------------------- driver
template <typename Real>
struct SectorResult {
  std::vector<Tracklet<Real>> TL;
  Selection<Real> S;
};

// ------------------------------------------------ online cluster removal
// Sec. 4: clusters inside a protective tube around physics tracks are kept;
// of the others, those inside a removal tube around the secondary legs of
// loopers and around very-low-pT tracks are removed; the clusters of the
// tracklets a physics track was built from (its seeding history) are
// protected as well.  Readings (the section states the rules in words only):
// * a track is very low pT if |q/pT| at its innermost cluster > cr_qpt;
// * two looper tracks (|q/pT| > looper_qpt) of the same side are legs of one
//   looper if their |q/pT| differ by at most cr_leg_dq relative, their
//   tan(lambda) are opposite within cr_leg_dtgl and their circle centres in
//   global coordinates lie within cr_leg_dc; every leg is parametrised
//   outwards, so legs flown inwards carry the opposite signs.  Along a
//   looper |z| grows from the vertex and side * z_measured differs from |z|
//   by one constant of the collision, so the leg with the smallest side * z
//   at its innermost cluster comes first; a leg linked to one before it is a
//   secondary leg, and its parent is the first such leg (smallest
//   (side * z, key), the key breaking exact ties);
// * the tube follows the track's clusters: on a row with a cluster of the
//   track its centre is that cluster, on the rows between two consecutive
//   clusters of the same sector the linear interpolation from the lower-row
//   one; it holds the clusters of that row within the half-width in y and z;
// * protection 1 is the choice of a wide protective and a narrow removal tube
//   (cr_protect > cr_remove); protection 2 (cr_mode 2) multiplies them by
//   cr_p2_grow and cr_p2_shrink on the inner_rows innermost rows, within
//   cr_edge of the sector edge, and where more than cr_occ_max clusters lie
//   within cr_occ_w of the centre.
// Flags per cluster: 1 in a protective tube, 2 seeding history, 4 in a
// removal tube, 8 removed (4 and neither 1 nor 2).
template <typename Real>
void cluster_removal(const Frame<Real>& F, const Params<Real>& P, const SectorResult<Real>& SR,
                     const std::vector<SectorTrack<Real>>& ST,
                     const std::vector<const FitTrack<Real>*>& T, Result& res) {
  const int nt = (int)T.size();
  const int half = P.n_sectors / 2;
  std::vector<int> cls(nt, 0), parent(nt, -1), looper(nt, 0), blk(nt);
  std::vector<Real> cx(nt), cy(nt), zk(nt);
  for (int t = 0; t < nt; ++t) {
    const Track<Real>& o = T[t]->out;
    const int s = T[t]->out_sector;
    const Real q = o.p[4];
    blk[t] = s / half;
    const Real side = (s % P.n_sectors) < half ? Real(1) : Real(-1);
    zk[t] = side * o.p[1];
    if (o_fabs(q) > P.cr_qpt) cls[t] = 1;
    looper[t] = P.looper_qpt > Real(0) && o_fabs(q) > P.looper_qpt;
    // circle centre: the curvature centre lies 1/kappa along the left normal
    const Real rk = Real(1) / (P.kb * q);
    const Real sn = o.p[2];
    const Real cs = o_sqrt(Real(1) - sn * sn);
    const Real xc = o.x - sn * rk, yc = o.p[0] + cs * rk;
    const int a = s % 18;
    cx[t] = xc * P.sec_cos[a] - yc * P.sec_sin[a];
    cy[t] = xc * P.sec_sin[a] + yc * P.sec_cos[a];
  }
  // looper legs
  for (int a = 0; a < nt; ++a) {
    if (!looper[a]) continue;
    int best = -1;
    for (int b = 0; b < nt; ++b) {
      if (b == a || !looper[b] || blk[b] != blk[a]) continue;
      const Real qa = T[a]->out.p[4], qb = T[b]->out.p[4];
      if ((qa > Real(0)) == (qb > Real(0))) continue;
      const Real aa = o_fabs(qa), ab = o_fabs(qb);
      const Real mx = aa > ab ? aa : ab;
      if (!(o_fabs(aa - ab) <= P.cr_leg_dq * mx)) continue;
      if (!(o_fabs(T[a]->out.p[3] + T[b]->out.p[3]) <= P.cr_leg_dtgl)) continue;
      const Real dx = cx[a] - cx[b], dy = cy[a] - cy[b];
      if (!(dx * dx + dy * dy <= P.cr_leg_dc * P.cr_leg_dc)) continue;
      const bool before = zk[b] < zk[a] || (zk[b] == zk[a] && T[b]->key < T[a]->key);
      if (!before) continue;
      if (best < 0 || zk[b] < zk[best] || (zk[b] == zk[best] && T[b]->key < T[best]->key))
        best = b;
    }
    parent[a] = best;
    if (best >= 0) cls[a] = 2;
  }
  // tubes
  std::vector<int> flags(F.n, 0);
  auto tube = [&](int s, int r, Real yc, Real zc, bool protect) {
    Real h = protect ? P.cr_protect : P.cr_remove;
    if (P.cr_mode >= 2) {
      bool dyn = r < P.inner_rows || o_fabs(yc) > P.row_x[r] * P.tan_half - P.cr_edge;
      if (!dyn) {
        int occ = 0;
        for_row_range(F, P, s, r, zc - P.cr_occ_w, zc + P.cr_occ_w, [&](int id) {
          if (o_fabs(F.y[id] - yc) <= P.cr_occ_w && o_fabs(F.z[id] - zc) <= P.cr_occ_w) ++occ;
        });
        dyn = occ > P.cr_occ_max;
      }
      if (dyn) h = h * (protect ? P.cr_p2_grow : P.cr_p2_shrink);
    }
    for_row_range(F, P, s, r, zc - h, zc + h, [&](int id) {
      if (o_fabs(F.y[id] - yc) <= h && o_fabs(F.z[id] - zc) <= h) flags[id] |= protect ? 1 : 4;
    });
  };
  for (int t = 0; t < nt; ++t) {
    const bool protect = cls[t] == 0;
    const std::vector<int>& u = T[t]->used;
    for (size_t i = 0; i < u.size(); ++i) {
      const int c = u[i];
      tube(F.sector[c], F.row[c], F.y[c], F.z[c], protect);
      if (i + 1 == u.size()) break;
      const int d = u[i + 1];
      if (F.sector[d] != F.sector[c]) continue;
      const int lo = F.row[c] < F.row[d] ? c : d, hi = lo == c ? d : c;
      const int rl = F.row[lo], rh = F.row[hi];
      for (int r = rl + 1; r < rh; ++r) {
        const Real f = Real(r - rl) / Real(rh - rl);
        tube(F.sector[c], r, F.y[lo] + (F.y[hi] - F.y[lo]) * f,
             F.z[lo] + (F.z[hi] - F.z[lo]) * f, protect);
      }
    }
    if (protect)  // seeding history: every hit of the track's tracklets
      for (int sgi : T[t]->seg)
        if (ST[sgi].tl >= 0)  // (segments of the edge following come from no tracklet)
          for (int c : SR.TL[ST[sgi].tl].hits) flags[c] |= 2;
  }
  long nrem = 0;
  for (long c = 0; c < F.n; ++c)
    if ((flags[c] & 4) && !(flags[c] & 3)) {
      flags[c] |= 8;
      ++nrem;
    }
  res.put("cr_flags", flags, "i4");
  res.put("cr_class", cls, "i4");
  res.put("cr_parent", parent, "i4");
  std::vector<Real> cxy;
  for (int t = 0; t < nt; ++t) {
    cxy.push_back(cx[t]);
    cxy.push_back(cy[t]);
  }
  res.put("cr_centre", cxy, real_name<Real>());
}

template <typename Real>
void run_merge_fit(const Frame<Real>& F, const Params<Real>& P, const MapR<Real>& M,
                   const SectorResult<Real>& SR, Result& res) {
  // a7: sector refit of every accepted tracklet
  std::vector<SectorTrack<Real>> ST;
  for (size_t i = 0; i < SR.TL.size(); ++i) {
    if (!SR.S.accepted[i]) continue;
    SectorTrack<Real> S;
    S.key = SR.TL[i].start;
    S.tl = (int)i;
    S.cl.assign(SR.S.kept[i].rbegin(), SR.S.kept[i].rend());
    S.sector = F.sector[S.cl[0]];
    S.rmin = F.row[S.cl.front()];
    S.rmax = F.row[S.cl.back()];
    if (!sector_refit(F, P, SR.TL[i].t, S)) continue;
    ST.push_back(S);
  }
  std::sort(ST.begin(), ST.end(), [](const auto& a, const auto& b) { return a.key < b.key; });
  if (P.edge_rows > 0) {
    std::vector<char> kept(F.n, 0);
    for (const auto& S : ST)
      for (int c : S.cl) kept[c] = 1;
    const int n0 = (int)ST.size();
    for (int a = 0; a < n0; ++a)
      for (int dir : {1, -1}) {
        SectorTrack<Real> S;
        if (!edge_segment(F, P, kept, ST[a], dir, S)) continue;
        S.link = ST[a].key;
        ST.push_back(S);
      }
    // segment keys exceed every tracklet key: ordered by key, the segments
    // follow the tracks
    std::sort(ST.begin(), ST.end(), [](const auto& a, const auto& b) { return a.key < b.key; });
  }
  const int nst = (int)ST.size();
  std::vector<int> next(nst, -1), prev(nst, -1);
  std::map<int, int> index_of_key;
  for (int i = 0; i < nst; ++i)
    if (ST[i].link >= 0) index_of_key[ST[i].link] = -1;
  for (int i = 0; i < nst; ++i)
    if (index_of_key.count(ST[i].key)) index_of_key[ST[i].key] = i;
  for (int i = 0; i < nst; ++i) {
    if (ST[i].link < 0) continue;
    const int a = index_of_key[ST[i].link];
    if (ST[i].dir > 0) { next[a] = i; prev[i] = a; }
    else { next[i] = a; prev[a] = i; }
  }
  // a7: candidate pairs by sector, mutual best
  const int half = P.n_sectors / 2;
  // candidate lists by (sector, innermost row); the pair test requires
  // 1 <= rmin(B) - rmax(A) <= merge_max_gap, so only those rows are visited
  std::vector<std::vector<int>> by_sector((size_t)P.n_sectors * P.n_rows);
  for (int i = 0; i < nst; ++i) by_sector[(size_t)ST[i].sector * P.n_rows + ST[i].rmin].push_back(i);
  std::vector<int> bestB(nst, -1), bestA(nst, -1);
  std::vector<Real> chiB(nst, 0), chiA(nst, 0);
  for (int a = 0; a < nst; ++a) {
    if (next[a] >= 0) continue;  // outer end linked by the edge following
    const int sa = ST[a].sector;
    const int side = sa / half, ph = sa % half;
    for (int d : {0, 1, half - 1}) {
      const int sb = side * half + (ph + d) % half;
      for (int rb = ST[a].rmax + 1; rb <= ST[a].rmax + P.merge_max_gap && rb < P.n_rows; ++rb)
      for (int b : by_sector[(size_t)sb * P.n_rows + rb]) {
        if (b == a || prev[b] >= 0) continue;
        Real chi2;
        if (!merge_test(P, ST[a], ST[b], chi2)) continue;
        if (bestB[a] < 0 || chi2 < chiB[a] || (chi2 == chiB[a] && ST[b].key < ST[bestB[a]].key)) {
          bestB[a] = b;
          chiB[a] = chi2;
        }
        if (bestA[b] < 0 || chi2 < chiA[b] || (chi2 == chiA[b] && ST[a].key < ST[bestA[b]].key)) {
          bestA[b] = a;
          chiA[b] = chi2;
        }
      }
    }
  }
  for (int a = 0; a < nst; ++a)
    if (bestB[a] >= 0 && bestA[bestB[a]] == a) {
      next[a] = bestB[a];
      prev[bestB[a]] = a;
    }
  // then across the central electrode: chain ends (no successor) against
  // chain starts (no predecessor) on the other side, mutual best by (chi2, key)
  std::vector<Real> xdz(nst, Real(0));  // z shift of the side that starts at b
  if (P.ac_merge) {
    std::vector<int> xB(nst, -1), xA(nst, -1);
    std::vector<Real> xchiB(nst, 0), xchiA(nst, 0), xdzB(nst, 0);
    for (int a = 0; a < nst; ++a) {
      if (next[a] >= 0) continue;
      const int sb = (ST[a].sector + half) % (2 * half);
      for (int rb = ST[a].rmax + 1; rb <= ST[a].rmax + P.merge_max_gap && rb < P.n_rows; ++rb)
        for (int b : by_sector[(size_t)sb * P.n_rows + rb]) {
          if (prev[b] >= 0) continue;
          Real chi2, dz;
          if (!cross_test(P, ST[a], ST[b], chi2, dz)) continue;
          if (xB[a] < 0 || chi2 < xchiB[a] || (chi2 == xchiB[a] && ST[b].key < ST[xB[a]].key)) {
            xB[a] = b;
            xchiB[a] = chi2;
            xdzB[a] = dz;
          }
          if (xA[b] < 0 || chi2 < xchiA[b] || (chi2 == xchiA[b] && ST[a].key < ST[xA[b]].key)) {
            xA[b] = a;
            xchiA[b] = chi2;
          }
        }
    }
    for (int a = 0; a < nst; ++a)
      if (xB[a] >= 0 && xA[xB[a]] == a) {
        next[a] = xB[a];
        prev[xB[a]] = a;
        xdz[xB[a]] = xdzB[a];
      }
  }
  std::vector<int> st_key(nst), st_next(nst);
  std::vector<Real> st_ie(nst * 5), st_oe(nst * 5);
  for (int i = 0; i < nst; ++i) {
    st_key[i] = ST[i].key;
    st_next[i] = next[i] >= 0 ? ST[next[i]].key : -1;
    for (int k = 0; k < 5; ++k) {
      st_ie[i * 5 + k] = ST[i].ie.p[k];
      st_oe[i * 5 + k] = ST[i].oe.p[k];
    }
  }
  res.put("st_key", st_key, "i4");
  res.put("st_next", st_next, "i4");
  res.put("st_ie", st_ie, real_name<Real>());
  res.put("st_oe", st_oe, real_name<Real>());
  // merged tracks (chains), ordered by the key of their first segment
  std::vector<FitTrack<Real>> FT;
  for (int h = 0; h < nst; ++h) {
    if (prev[h] >= 0) continue;
    FitTrack<Real> T;
    T.key = ST[h].key;
    std::vector<int> cl;
    int last = h;
    T.side0 = (ST[h].sector / half) % 2;
    bool crossed = false;
    for (int s = h; s >= 0; s = next[s]) {
      cl.insert(cl.end(), ST[s].cl.begin(), ST[s].cl.end());
      T.seg.push_back(s);
      last = s;
      if (!crossed && (ST[s].sector / half) % 2 != T.side0) {
        crossed = true;
        T.zshift = xdz[s];
      }
    }
    T.st = make_stations(F, P, cl, true);
    T.outer = ST[last].oe;
    const Track<Real>& ie = ST[h].ie;
    // a low-pT looper (|q/pT| at the inner end of its first segment above
    // looper_qpt) runs every update of its final fit in FP64
    T.looper = P.looper_qpt > Real(0) && o_fabs(ie.p[4]) > P.looper_qpt;
    T.z0 = ie.p[1] - ie.p[3] * o_sqrt(ie.x * ie.x + ie.p[0] * ie.p[0]);
    FT.push_back(std::move(T));
  }
  // a9/a10 (+ Phase III): clusters held by a station outside the inner
  // region of any track are not extrapolation candidates
  std::vector<char> fixed(F.n, 0);
  if (P.ext_rows > 0)
    for (const auto& T : FT)
      for (const auto& s : T.st)
        if (s.cl >= 0 && s.row >= P.inner_rows) fixed[s.cl] = 1;
  std::vector<Track<Real>> it2_end(FT.size());
  std::vector<Real> store;
  for (size_t i = 0; i < FT.size(); ++i)
    fit_iterations12(F, P, M, fixed, FT[i], true, store, it2_end[i]);
  second_ambiguity(FT, P);
  for (size_t i = 0; i < FT.size(); ++i)
    if (FT[i].ok) fit_iteration3(F, P, M, FT[i], true, it2_end[i]);
  // a11: output tracks with at least min_hits clusters, attachments
  std::vector<int> key, ncl, offs(1, 0), ids, sect, ndf, flags;
  std::vector<Real> par, cov, chi2, xs, zsh;
  std::vector<int> attach(F.n, -1);
  for (auto& T : FT) {
    if (!T.ok || T.n < P.min_hits) continue;
    const int t = (int)key.size();
    key.push_back(T.key);
    ncl.push_back(T.n);
    for (int c : T.used) {
      ids.push_back(c);
      if (attach[c] < 0) attach[c] = t;
    }
    offs.push_back((int)ids.size());
    sect.push_back(T.out_sector);
    ndf.push_back(2 * T.n - 5);
    chi2.push_back(T.chi2);
    xs.push_back(T.out.x);
    zsh.push_back(T.zshift);
    for (int k = 0; k < 5; ++k) par.push_back(T.out.p[k]);
    for (int k = 0; k < 15; ++k) cov.push_back(T.out.c[k]);
  }
  res.put("trk_key", key, "i4");
  res.put("trk_ncl", ncl, "i4");
  res.put("trk_offset", offs, "i4");
  res.put("trk_ids", ids, "i4");
  res.put("trk_sector", sect, "i4");
  res.put("trk_ndf", ndf, "i4");
  res.put("trk_chi2", chi2, real_name<Real>());
  res.put("trk_x", xs, real_name<Real>());
  res.put("trk_zshift", zsh, real_name<Real>());
  res.put("trk_param", par, real_name<Real>());
  res.put("trk_cov", cov, real_name<Real>());
  res.put("attach", attach, "i4");
  if (P.cr_mode > 0) {
    std::vector<const FitTrack<Real>*> out;
    for (const auto& T : FT)
      if (T.ok && T.n >= P.min_hits) out.push_back(&T);
    cluster_removal(F, P, SR, ST, out, res);
  }
  // per merged track diagnostics (all chains, including rejected ones)
  std::vector<int> fk, fflag_n, fcand_n, fassigned_n, ffail, fn;
  for (auto& T : FT) {
    fk.push_back(T.key);
    ffail.push_back(T.ok ? -1 : T.fail_at);
    fn.push_back(T.n);
    int nf = 0, nc = 0, na = 0;
    for (size_t s = 0; s < T.st.size(); ++s) {
      nf += T.flag.empty() ? 0 : T.flag[s];
      nc += T.ncand.empty() ? 0 : T.ncand[s];
      na += T.assigned.empty() ? 0 : (T.assigned[s] >= 0);
    }
    fflag_n.push_back(nf);
    fcand_n.push_back(nc);
    fassigned_n.push_back(na);
  }
  res.put("fit_key", fk, "i4");
  res.put("fit_nflag", fflag_n, "i4");
  res.put("fit_ncand", fcand_n, "i4");
  res.put("fit_nassigned", fassigned_n, "i4");
  res.put("fit_fail", ffail, "i4");
  res.put("fit_n", fn, "i4");
  // Phase II candidates and assignments of every inner station
  std::vector<int> cs_key, cs_row, cs_sector, cs_n, cs_cand, cs_assigned;
  std::vector<Real> cs_chi;
  for (auto& T : FT) {
    if (!T.ok) continue;
    for (size_t s = 0; s < T.st.size(); ++s) {
      if (T.st[s].row >= P.inner_rows) continue;
      cs_key.push_back(T.key);
      cs_row.push_back(T.st[s].row);
      cs_sector.push_back(T.st[s].sector);
      cs_n.push_back(T.ncand[s]);
      for (int k = 0; k < P.cand_k; ++k) {
        cs_cand.push_back(T.cand[s * P.cand_k + k]);
        cs_chi.push_back(T.cchi[s * P.cand_k + k]);
      }
      cs_assigned.push_back(T.assigned[s]);
    }
  }
  res.put("cand_key", cs_key, "i4");
  res.put("cand_row", cs_row, "i4");
  res.put("cand_sector", cs_sector, "i4");
  res.put("cand_n", cs_n, "i4");
  res.put("cand_ids", cs_cand, "i4");
  res.put("cand_chi2", cs_chi, real_name<Real>());
  res.put("cand_assigned", cs_assigned, "i4");
  // Phase III candidates and assignments of every extrapolated row (inward
  // rows, then outward rows)
  std::vector<int> ex_key, ex_row, ex_sec, ex_n, ex_cand, ex_assigned, fit_next, fit_nout;
  std::vector<Real> ex_chi;
  for (auto& T : FT) {
    fit_next.push_back(T.ok ? T.n_ext : 0);
    fit_nout.push_back(T.ok ? T.n_out : 0);
    if (!T.ok) continue;
    const size_t ns = T.st.size();
    auto put = [&](size_t slot, int row, int sector) {
      ex_key.push_back(T.key);
      ex_row.push_back(row);
      ex_sec.push_back(sector);
      ex_n.push_back(T.ncand[slot]);
      for (int k = 0; k < P.cand_k; ++k) {
        ex_cand.push_back(T.cand[slot * P.cand_k + k]);
        ex_chi.push_back(T.cchi[slot * P.cand_k + k]);
      }
      ex_assigned.push_back(T.assigned[slot]);
    };
    for (int e = 0; e < T.n_ext; ++e) put(ns + e, T.st[0].row - 1 - e, T.ext_sec[e]);
    for (int e = 0; e < T.n_out; ++e)
      put(ns + P.ext_rows + e, T.st[ns - 1].row + 1 + e, T.ext_sec[P.ext_rows + e]);
  }
  res.put("fit_next", fit_next, "i4");
  res.put("fit_nout", fit_nout, "i4");
  res.put("ext_key", ex_key, "i4");
  res.put("ext_row", ex_row, "i4");
  res.put("ext_sector", ex_sec, "i4");
  res.put("ext_n", ex_n, "i4");
  res.put("ext_ids", ex_cand, "i4");
  res.put("ext_chi2", ex_chi, real_name<Real>());
  res.put("ext_assigned", ex_assigned, "i4");
}

// Sector tracking a2-a6, seed_iters times.  Sec. 3 (Phase III) runs the
// seeding again on the clusters left over after the ambiguity solving: every
// later iteration repeats a2-a6 on the clusters that no accepted tracklet of
// an earlier iteration kept, as if the others were not there.  A cluster is
// taken if an accepted tracklet kept it or starts at it (so that no two
// accepted tracklets share a start cluster, the sector tracks' key); the
// selection of an iteration is among its own tracklets.  The per-tracklet
// outputs are those of all iterations in order (tl_iter), the link arrays
// those of the last iteration.
template <typename Real>
SectorResult<Real> run_sector_tracking(Frame<Real>& F, const Params<Real>& P, Result& res) {
  const int R = P.n_rows;
  SectorResult<Real> SR;
  std::vector<int> up, dn, cu, cd, all_starts, tl_iter;
  std::vector<uint64_t> keys;
  std::vector<int> owner(F.n, -1);
  for (int it = 0; it < P.seed_iters; ++it) {
    find_links(F, P, up, dn);
    clean_links(up, dn, cu, cd);
    const std::vector<int> starts = start_hits(cu, cd);
    std::vector<Tracklet<Real>> TL(starts.size());
    for (size_t i = 0; i < starts.size(); ++i) TL[i] = construct(F, P, cu, starts[i]);
    Selection<Real> S = select(F, P, TL);
    // sector-level attachment: the owner tracklet's start id if it is accepted
    std::map<int, size_t> by_start;
    for (size_t i = 0; i < TL.size(); ++i) by_start[TL[i].start] = i;
    for (long c = 0; c < F.n; ++c) {
      const uint64_t k = S.owner_key[c];
      if (!k) continue;
      const int sid = (int)(0xFFFFFFFFu - (uint32_t)(k & 0xFFFFFFFFu));
      if (S.accepted[by_start[sid]]) owner[c] = sid;
    }
    if (F.used.empty()) F.used.assign(F.n, 0);
    for (size_t i = 0; i < TL.size(); ++i) {
      all_starts.push_back(TL[i].start);
      tl_iter.push_back(it);
      keys.push_back(TL[i].n ? make_key(score_of(TL[i], P), TL[i].start) : 0);
      if (S.accepted[i]) {
        for (int c : S.kept[i]) F.used[c] = 1;
        F.used[TL[i].start] = 1;
      }
      SR.TL.push_back(std::move(TL[i]));
      SR.S.accepted.push_back(S.accepted[i]);
      SR.S.kept.push_back(std::move(S.kept[i]));
    }
  }
  F.used.clear();  // the stages after the sector tracking see every cluster
  res.put("link_up", up, "i4");
  res.put("link_dn", dn, "i4");
  res.put("clean_up", cu, "i4");
  res.put("clean_dn", cd, "i4");
  res.put("start", all_starts, "i4");
  const std::vector<Tracklet<Real>>& TL = SR.TL;
  const size_t nt = TL.size();
  std::vector<int> tl_n(nt), tl_ndf(nt), tl_hits(nt * R, -1);
  std::vector<Real> tl_par(nt * 5), tl_cov(nt * 15), tl_chi2(nt), tl_x(nt);
  std::vector<int> acc(nt), nk(nt), kept(nt * R, -1);
  for (size_t i = 0; i < nt; ++i) {
    tl_n[i] = TL[i].n;
    tl_ndf[i] = TL[i].ndf;
    tl_chi2[i] = TL[i].chi2;
    tl_x[i] = TL[i].t.x;
    for (int k = 0; k < 5; ++k) tl_par[i * 5 + k] = TL[i].t.p[k];
    for (int k = 0; k < 15; ++k) tl_cov[i * 15 + k] = TL[i].t.c[k];
    for (size_t k = 0; k < TL[i].hits.size(); ++k) tl_hits[i * R + k] = TL[i].hits[k];
    acc[i] = SR.S.accepted[i];
    nk[i] = (int)SR.S.kept[i].size();
    for (size_t k = 0; k < SR.S.kept[i].size(); ++k) kept[i * R + k] = SR.S.kept[i][k];
  }
  res.put("tl_start", all_starts, "i4");
  res.put("tl_iter", tl_iter, "i4");
  res.put("tl_n", tl_n, "i4");
  res.put("tl_ndf", tl_ndf, "i4");
  res.put("tl_hits", tl_hits, "i4");
  res.put("tl_param", tl_par, real_name<Real>());
  res.put("tl_cov", tl_cov, real_name<Real>());
  res.put("tl_chi2", tl_chi2, real_name<Real>());
  res.put("tl_x", tl_x, real_name<Real>());
  res.put("tl_key", keys, "u8");
  res.put("tl_accept", acc, "i4");
  res.put("tl_nkept", nk, "i4");
  res.put("tl_kept", kept, "i4");
  res.put("sector_owner", owner, "i4");
  return SR;
}

template <typename Real, typename In>
Frame<Real> make_frame(long n, const In* y, const In* z, const uint8_t* row,
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

template <typename Real>
MapR<Real> make_map(const orc_map* m) {
  MapR<Real> M;
  if (!m || !m->coeff) return M;
  M.on = true;
  M.nphi = m->n_phi; M.nr = m->n_r; M.nz = m->n_z;
  M.rmin = m->r_min; M.zmin = m->z_min; M.zmax = m->z_max;
  M.phi_scale = (Real)((double)m->n_phi / 18.0);
  M.r_scale = (Real)((double)(m->n_r - 3) / ((double)m->r_max - (double)m->r_min));
  M.z_scale = (Real)((double)(m->n_z - 3) / ((double)m->z_max - (double)m->z_min));
  M.c = m->coeff;
  return M;
}

}  // namespace orc

struct orc_result {
  orc::Result r;
};

extern "C" {
// Tracks handed to the refit: cluster ids innermost first and the start
// parameters at the innermost cluster (sector frame `sector`, local x).
struct orc_tracks_in {
  long n_tracks;
  const int32_t* offset;  // [n_tracks + 1]
  const int32_t* ids;
  const double* par;      // [n_tracks][5]
  const double* x;
  const int32_t* sector;
  const double* zshift;   // [n_tracks] z shift of the far side (merged across the central
                          // electrode), or NULL for none
};
// Frozen references and decisions of a previous refit (optional).
struct orc_frozen {
  const double* ref;   // [n_tracks][10]: iteration-2 and iteration-3 references
  const int32_t* flag; // per cluster reference
  const int32_t* acc;  // per cluster reference
};
}

// mode: 0 = float, 1 = double, 2 = double with the tape gradient of
// sum_t w_t chi2_t with respect to the map coefficients.
template <typename Real>
static void refit_impl(long n, const float* y, const float* z, const uint8_t* row,
                       const uint8_t* sector, const double* row_x, const orc_options* opt,
                       const orc_map* map, const orc_tracks_in* T, const orc_frozen* frz,
                       const double* w, bool grad, orc::Result& res) {
  using namespace orc;
  const auto P = make_params<Real>(*opt, row_x);
  const auto F = make_frame<Real>(n, y, z, row, sector, P);
  MapR<Real> M = make_map<Real>(map);
  const long ncoef = (map && map->coeff) ? 3L * map->n_z * map->n_r * map->n_phi : 0;
  std::vector<double> gsum(grad ? ncoef : 0, 0.0);
  const long nt = T->n_tracks;
  std::vector<double> chi2(nt), par(nt * 5), xs(nt);
  std::vector<int> nn(nt), ok(nt), sec(nt);
  std::vector<double> fref(nt * 10, 0.0);
  std::vector<int> fflag(T->offset[nt], 0), facc(T->offset[nt], 0);
  for (long t = 0; t < nt; ++t) {
    RefitIO<Real> R;
    for (int i = T->offset[t]; i < T->offset[t + 1]; ++i) {
      const int c = T->ids[i];
      R.st.push_back({F.sector[c], F.row[c], c});
    }
    for (int i = 0; i < 5; ++i) R.in_p[i] = Real(T->par[t * 5 + i]);
    R.in_x = Real(T->x[t]);
    R.in_sector = T->sector[t];
    R.zshift = T->zshift ? Real(T->zshift[t]) : Real(0);
    if (!R.st.empty()) R.side0 = (R.st[0].sector / (P.n_sectors / 2)) % 2;
    const bool frozen = frz != nullptr;
    if (frozen) {
      for (int i = 0; i < 5; ++i) {
        R.ref2[i] = frz->ref[t * 10 + i];
        R.ref3[i] = frz->ref[t * 10 + 5 + i];
      }
      R.flag.assign(frz->flag + T->offset[t], frz->flag + T->offset[t + 1]);
      R.acc.assign(frz->acc + T->offset[t], frz->acc + T->offset[t + 1]);
    }
    std::vector<Real> leaves;
    if (grad && ncoef) {
      tape().clear();
      leaves.resize(ncoef);
      for (long i = 0; i < ncoef; ++i) leaves[i] = Real(Var::leaf((double)map->coeff[i]));
      M.cv = leaves.data();
    }
    refit_track(F, P, M, R, frozen);
    chi2[t] = (double)R.chi2;
    nn[t] = R.n;
    ok[t] = R.ok ? 1 : 0;
    sec[t] = R.out_sector;
    xs[t] = (double)R.out.x;
    for (int i = 0; i < 5; ++i) par[t * 5 + i] = (double)R.out.p[i];
    for (int i = 0; i < 5; ++i) {
      fref[t * 10 + i] = R.ref2[i];
      fref[t * 10 + 5 + i] = R.ref3[i];
    }
    for (size_t k = 0; k < R.flag.size(); ++k) fflag[T->offset[t] + k] = R.flag[k];
    for (size_t k = 0; k < R.acc.size(); ++k) facc[T->offset[t] + k] = R.acc[k];
    if (grad && ncoef) {
      if constexpr (std::is_same<Real, Var>::value) {
        if (R.ok && R.chi2.id >= 0) {
          const std::vector<double> adj = tape().reverse(R.chi2.id);
          for (long i = 0; i < ncoef; ++i) gsum[i] += w[t] * adj[leaves[i].id];
        }
      }
      M.cv = nullptr;
    }
  }
  // values of the float mode are exact in double
  res.put("rf_chi2", chi2, "f8");
  res.put("rf_n", nn, "i4");
  res.put("rf_ok", ok, "i4");
  res.put("rf_par", par, "f8");
  res.put("rf_x", xs, "f8");
  res.put("rf_sector", sec, "i4");
  res.put("frz_ref", fref, "f8");
  res.put("frz_flag", fflag, "i4");
  res.put("frz_acc", facc, "i4");
  if (grad) res.put("grad", gsum, "f8");
}

extern "C" int orc_refit(long n, const float* y, const float* z, const uint8_t* row,
                         const uint8_t* sector, const double* row_x, const orc_options* opt,
                         const orc_map* map, const orc_tracks_in* T, const orc_frozen* frz,
                         const double* w, int mode, orc_result** out) {
  if (!opt || !row_x || !out || !T || n < 0) return 1;
  auto* R = new orc_result();
  if (mode == 0)
    refit_impl<float>(n, y, z, row, sector, row_x, opt, map, T, frz, w, false, R->r);
  else if (mode == 1)
    refit_impl<double>(n, y, z, row, sector, row_x, opt, map, T, frz, w, false, R->r);
  else
    refit_impl<orc::Var>(n, y, z, row, sector, row_x, opt, map, T, frz, w, true, R->r);
  *out = R;
  return 0;
}

template <typename In>
static int track_impl(long n, const In* y, const In* z, const uint8_t* row, const uint8_t* sector,
                      const double* row_x, const orc_options* opt, const orc_map* map, int stages,
                      int use_double, orc_result** out) {
  if (!opt || !row_x || !out || n < 0) return 1;
  if (opt->edge_rows > 0 && n >= (1L << 29)) return 1;  // segment keys need ids below 2^29
  for (long i = 0; i < n; ++i)
    if (row[i] >= opt->n_rows || sector[i] >= opt->n_sectors || !std::isfinite(y[i]) ||
        !std::isfinite(z[i]))
      return 2;
  auto* R = new orc_result();
  auto run = [&](auto tag) {
    using Real = decltype(tag);
    const auto P = orc::make_params<Real>(*opt, row_x);
    auto F = orc::make_frame<Real>(n, y, z, row, sector, P);
    auto SR = orc::run_sector_tracking(F, P, R->r);
    if (stages >= 1) orc::run_merge_fit(F, P, orc::make_map<Real>(map), SR, R->r);
  };
  if (use_double)
    run(double{});
  else
    run(float{});
  *out = R;
  return 0;
}

// stages: 0 = sector tracking only, 1 = full chain (merging, fit, attachment)

extern "C" {

int orc_track(long n, const float* y, const float* z, const uint8_t* row, const uint8_t* sector,
              const double* row_x, const orc_options* opt, const orc_map* map, int stages,
              int use_double, orc_result** out) {
  return track_impl(n, y, z, row, sector, row_x, opt, map, stages, use_double, out);
}

// The same with FP64 cluster coordinates (precision pins with exact inputs).
int orc_track_f64(long n, const double* y, const double* z, const uint8_t* row,
                  const uint8_t* sector, const double* row_x, const orc_options* opt,
                  const orc_map* map, int stages, orc_result** out) {
  return track_impl(n, y, z, row, sector, row_x, opt, map, stages, 1, out);
}

// Correction of one cluster in FP64 (pins): io = {sector, x, y, z, z0, ref[5]} ->
// io[10..12] = D (map displacement), io[13..14] = projected measurement.
int orc_correct(const orc_options* opt, const double* row_x, const orc_map* map, double* io) {
  if (!opt || !io) return 1;
  const auto P = orc::make_params<double>(*opt, row_x);
  const auto M = orc::make_map<double>(map);
  double D[3];
  orc::map_eval(M, P, (int)io[0], io[1], io[2], io[3] - io[4], D);
  io[10] = D[0]; io[11] = D[1]; io[12] = D[2];
  double my, mz;
  if (!orc::corrected(M, P, (int)io[0], io[1], io[2], io[3], io[4], &io[5], my, mz)) return 2;
  io[13] = my;
  io[14] = mz;
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
      if (!orc::propagate(t, (Real)io[21], P, P.max_snp)) return 1;
      io[20] = t.x;
    } else if (op == 1) {
      const auto R = orc::residual(t, (Real)io[20], (Real)io[21], P);
      orc::update(t, R);
      io[22] = R.chi2;
    } else if (op == 2) {
      t.x = (Real)io[20];
      if (!orc::rotate(t, io[21] > 0 ? 1 : -1, P, P.max_snp)) return 1;
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

// Second ambiguity solving (Sec. 3, Phase II) on candidate lists given by
// the caller, for pins on hand-made cases.  Track t has n_slots (track, row)
// slots; slot s offers ncand[t*n_slots+s] <= cand_k candidates, best first:
// cluster ids cand[(t*n_slots+s)*cand_k + k] with chi2 chi2[...]; key[t] is
// the track key of the tie-break.  assigned[t*n_slots+s] receives the
// cluster given to the slot or -1.
int orc_second_ambiguity(int n_tracks, int n_slots, int cand_k, const int* key,
                         const int* ncand, const int* cand, const float* chi2, int* assigned) {
  if (n_tracks < 0 || n_slots < 0 || cand_k < 1 || (n_tracks > 0 && n_slots > 0 &&
      (!key || !ncand || !cand || !chi2 || !assigned)))
    return 3;
  orc::Params<float> P{};
  P.cand_k = cand_k;
  std::vector<orc::FitTrack<float>> FT((size_t)n_tracks);
  for (int t = 0; t < n_tracks; ++t) {
    auto& T = FT[t];
    T.key = key[t];
    T.ncand.assign(ncand + (long)t * n_slots, ncand + (long)(t + 1) * n_slots);
    const long b = (long)t * n_slots * cand_k, e = (long)(t + 1) * n_slots * cand_k;
    T.cand.assign(cand + b, cand + e);
    T.cchi.assign(chi2 + b, chi2 + e);
  }
  orc::second_ambiguity(FT, P);
  for (int t = 0; t < n_tracks; ++t)
    for (int sl = 0; sl < n_slots; ++sl) assigned[(long)t * n_slots + sl] = FT[t].assigned[sl];
  return 0;
}

}  // extern "C"
