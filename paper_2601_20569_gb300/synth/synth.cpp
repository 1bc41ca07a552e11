// Synthetic continuous-readout TPC time frames (physics simulation only).
//
// This module produces the seeded inputs that both the CUDA tracker and the
// CPU oracle consume: helix trajectories in a solenoidal field crossing the
// pad-row planes of 36 trapezoidal sectors, with multiple-scattering kinks,
// Gaussian cluster smearing, uniform noise clusters, Landau-distributed
// charges, collision times inside a 2.8 ms frame (Sec. 1 of the paper:
// collisions overlap and hits cannot be assigned to collisions before
// tracking) and an optional smooth space-charge distortion field.
//
// It contains none of the tracking arithmetic: trajectories are computed as
// exact circle/line intersections in FP64, never with a Kalman-style
// propagator.  Random numbers come from Philox4x32-10 (Salmon et al., SC'11),
// keyed by (seed) with counters (particle, stream, frame, draw), so a frame is
// reproducible independent of the thread count.
//
// Geometry (fixed): 18 azimuthal sectors per side, side A (z>0) = sectors
// 0..17, side C = 18..35; sector axis at azimuth (s%18 + 0.5)*20 deg; 152 pad
// rows at x_r = 85 + r*160/151 cm; acceptance |y| <= x*tan(10 deg).
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <string>
#include <vector>
#ifdef _OPENMP
#include <omp.h>
#endif

namespace {

constexpr int kPhiSectors = 18;
constexpr int kRows = 152;
constexpr double kPi = 3.14159265358979323846;
constexpr double kSectorWidth = 20.0 * kPi / 180.0;
constexpr double kBToCurv = 0.00299792458;  // GeV / (T cm)
constexpr double kZMax = 250.0;

double row_x(int r) { return 85.0 + r * (160.0 / 151.0); }
double tan_half() { return std::tan(10.0 * kPi / 180.0); }
double sector_alpha(int sphi) { return (sphi + 0.5) * kSectorWidth; }

// ---------------------------------------------------------------- Philox4x32-10
struct Philox {
  static void block(const uint32_t ctr[4], uint32_t k0, uint32_t k1, uint32_t out[4]) {
    uint32_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];
    for (int r = 0; r < 10; ++r) {
      if (r) {
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
      }
      const uint64_t p0 = (uint64_t)0xD2511F53u * x0;
      const uint64_t p1 = (uint64_t)0xCD9E8D57u * x2;
      const uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
      const uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
      const uint32_t y0 = hi1 ^ x1 ^ k0, y1 = lo1, y2 = hi0 ^ x3 ^ k1, y3 = lo0;
      x0 = y0; x1 = y1; x2 = y2; x3 = y3;
    }
    out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
  }
};

struct Rng {
  uint32_t k0, k1, c0, c1, c2, n = 0;
  uint32_t buf[4];
  int pos = 4;
  Rng(uint64_t seed, uint32_t a, uint32_t b, uint32_t c)
      : k0((uint32_t)seed), k1((uint32_t)(seed >> 32)), c0(a), c1(b), c2(c) {}
  uint32_t u32() {
    if (pos == 4) {
      const uint32_t ctr[4] = {c0, c1, c2, n++};
      Philox::block(ctr, k0, k1, buf);
      pos = 0;
    }
    return buf[pos++];
  }
  // uniform in the open interval (0,1)
  double uni() {
    const uint64_t hi = u32(), lo = u32();
    const uint64_t m = ((hi << 32) | lo) >> 11;
    return ((double)m + 0.5) * (1.0 / 9007199254740992.0);
  }
  double gauss() {
    const double u1 = uni(), u2 = uni();
    return std::sqrt(-2.0 * std::log(u1)) * std::cos(2.0 * kPi * u2);
  }
  double expo(double mean) { return -mean * std::log(uni()); }
  long poisson(double mean) {
    if (mean < 60.0) {
      const double L = std::exp(-mean);
      long k = 0;
      double p = uni();
      while (p > L) { ++k; p *= uni(); }
      return k;
    }
    const double v = std::floor(mean + std::sqrt(mean) * gauss() + 0.5);
    return v < 0 ? 0 : (long)v;
  }
};

enum Stream : uint32_t { kStreamParticle = 1, kStreamCluster = 2, kStreamEvent = 3, kStreamNoise = 4 };

}  // namespace

extern "C" {

// Layout mirrored by the Python binding (ctypes); all lengths in cm, momenta
// in GeV, times in microseconds, field in tesla.
struct synth_config {
  uint64_t seed;
  int32_t frame;
  int32_t mode;  // 0: one event of n_primaries at t0 = 0; 1: time frame
  int32_t n_primaries;
  int32_t mult_cap;
  double mean_collisions;
  double mean_mult;
  double frame_us;
  double vdrift;
  double bz;
  double pt_min, pt_max, pt_power;
  double eta_min, eta_max;
  double phi_min, phi_max;
  double sec_frac, sec_rmax;
  double ms_theta;
  double sigma;
  double noise_frac;
  double looper_frac, looper_pt_min, looper_pt_max;
  int32_t only_sector;   // -1: all sectors; else keep only this sector
  int32_t thin_sectors;  // 1: per-frame sector occupancy factors in [0.1, 1]
  int32_t max_legs;
  int32_t n_threads;
  int32_t store_truth;
  int32_t shuffle;
  double aim_radius;  // >0: phi_min/phi_max bound the azimuth at this radius, not the direction
  const float* map;  // distortion control points [3][nz][nr][nphi] or NULL
  int32_t map_nphi, map_nr, map_nz, map_pad;
  double map_rmin, map_rmax, map_zmin, map_zmax;
  double vz_sigma;  // >0: Gaussian spread of the collision vertex along z [cm] (else z = 0)
};

struct synth_result;
int synth_generate(const synth_config* cfg, synth_result** out);
long synth_count(const synth_result* r, const char* what);
int synth_copy(const synth_result* r, const char* what, void* dst, long cap_bytes);
void synth_free(synth_result* r);
void synth_philox(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);
int synth_distortion_profile(int nphi, int nr, int nz, double rmin, double rmax, double zmin,
                             double zmax, double amp, float* coeff);
int synth_eval_distortion(const float* coeff, int nphi, int nr, int nz, double rmin, double rmax,
                          double zmin, double zmax, int sector, double x, double y, double z,
                          double* d);
}

namespace {


struct Particle {
  double pt, q, tgl, phi0, vx, vy, vz, t0;
  int secondary;
};

struct Helix {
  double X, Y, Z, phi, tgl, kappa;  // global position, direction, dz/ds, signed curvature
};

struct Crossing {
  int sector, row, leg;
  double y, z;           // local y, true z (no drift-time shift)
  double snp, tgl, qpt;  // model convention (motion along +x of the sector)
  Helix h;               // trajectory state at the crossing (before the kink)
};

// Field model for distortions: uniform cubic B-spline in (u, r, z) where
// u = sector + 0.5 + 0.5*(y/x)/tan(10 deg) is periodic over 18 sectors.
struct DistField {
  const float* c = nullptr;
  int nphi = 0, nr = 0, nz = 0;
  double rmin = 0, rmax = 1, zmin = -1, zmax = 1;
  static void weights(double f, double w[4]) {
    const double g = 1.0 - f;
    w[0] = g * g * g / 6.0;
    w[1] = (3.0 * f * f * f - 6.0 * f * f + 4.0) / 6.0;
    w[2] = (-3.0 * f * f * f + 3.0 * f * f + 3.0 * f + 1.0) / 6.0;
    w[3] = f * f * f / 6.0;
  }
  static void span(double t, int n, int& i, double& f) {
    // clamped open uniform parametrisation: t in [0, n-3]
    const double tmax = (double)(n - 3);
    if (t < 0) t = 0;
    if (t > tmax) t = tmax;
    i = (int)std::floor(t);
    if (i > n - 4) i = n - 4;
    f = t - i;
  }
  void eval(int sector, double x, double y, double z, double d[3]) const {
    d[0] = d[1] = d[2] = 0;
    if (!c) return;
    const int sphi = sector % kPhiSectors;
    const double u = sphi + 0.5 + 0.5 * (y / x) / tan_half();
    const double tp = u * nphi / (double)kPhiSectors - 0.5;
    const int ip = (int)std::floor(tp);
    const double fp = tp - ip;
    const double r = std::sqrt(x * x + y * y);
    int ir, iz;
    double fr, fz;
    span((r - rmin) / (rmax - rmin) * (nr - 3), nr, ir, fr);
    double zc = std::min(std::max(z, zmin), zmax);
    span((zc - zmin) / (zmax - zmin) * (nz - 3), nz, iz, fz);
    double wp[4], wr[4], wz[4];
    weights(fp, wp);
    weights(fr, wr);
    weights(fz, wz);
    for (int comp = 0; comp < 3; ++comp) {
      double acc = 0;
      for (int a = 0; a < 4; ++a)
        for (int b = 0; b < 4; ++b)
          for (int e = 0; e < 4; ++e) {
            const int pp = ((ip - 1 + e) % nphi + nphi) % nphi;
            const long idx = (((long)comp * nz + (iz + a)) * nr + (ir + b)) * nphi + pp;
            acc += wz[a] * wr[b] * wp[e] * (double)c[idx];
          }
      d[comp] = acc;
    }
  }
};

// Arc length (>0) along the helix to the intersection with the line x_local = xr
// of the sector at azimuth alpha.  Returns the two solutions (or fewer).
int intersections(const Helix& h, double alpha, double xr, double s_out[2], double y_out[2],
                  double psi_out[2]) {
  const double ca = std::cos(alpha), sa = std::sin(alpha);
  const double ik = 1.0 / h.kappa;
  const double Xc = h.X - std::sin(h.phi) * ik, Yc = h.Y + std::cos(h.phi) * ik;
  const double cx = Xc * ca + Yc * sa, cy = -Xc * sa + Yc * ca;
  const double v = h.kappa * (xr - cx);
  if (v >= 1.0 || v <= -1.0) return 0;
  const double psi0 = h.phi - alpha;
  const double as = std::asin(v);
  const double cand[2] = {as, kPi - as};
  const double period = 2.0 * kPi;
  int n = 0;
  for (double psi : cand) {
    double d = h.kappa > 0 ? std::fmod(psi - psi0, period) : std::fmod(psi0 - psi, period);
    if (d < 0) d += period;
    const double s = d / std::fabs(h.kappa);
    s_out[n] = s;
    y_out[n] = cy - std::cos(psi) * ik;
    psi_out[n] = psi;
    ++n;
  }
  return n;
}

void advance(Helix& h, double s) {
  const double ik = 1.0 / h.kappa;
  const double Xc = h.X - std::sin(h.phi) * ik, Yc = h.Y + std::cos(h.phi) * ik;
  h.phi += h.kappa * s;
  h.X = Xc + std::sin(h.phi) * ik;
  h.Y = Yc - std::cos(h.phi) * ik;
  h.Z += h.tgl * s;
}

void trace(const synth_config& cfg, const Particle& p, Rng& rng, std::vector<Crossing>& out) {
  Helix h{p.vx, p.vy, p.vz, p.phi0, p.tgl, -p.q * cfg.bz * kBToCurv / p.pt};
  const double th = tan_half();
  const double s_eps = 1e-7;
  const double s_max = 2.0 * kPi / std::fabs(h.kappa) - 1e-6;
  int last_row = -1, last_sphi = -1, leg = 0, prev_dir = 0;
  for (int step = 0; step < 1200; ++step) {
    double best_s = 1e300, best_y = 0, best_psi = 0;
    int best_row = -1, best_sphi = -1;
    const int r_lo = last_row < 0 ? 0 : std::max(0, last_row - 1);
    const int r_hi = last_row < 0 ? 0 : std::min(kRows - 1, last_row + 1);
    // Nearby sectors first; if nothing is found within a short arc (the track
    // may loop inside the inner radius or outside the outer one and re-enter
    // far away), search all sectors so that no crossing is skipped.
    for (int pass = 0; pass < 2; ++pass) {
      const bool all = last_sphi < 0 || pass == 1;
      for (int r = r_lo; r <= r_hi; ++r) {
        const double xr = row_x(r);
        const int ds_lo = all ? 0 : -2, ds_hi = all ? kPhiSectors - 1 : 2;
        for (int ds = ds_lo; ds <= ds_hi; ++ds) {
          const int sphi = all ? ds : ((last_sphi + ds) % kPhiSectors + kPhiSectors) % kPhiSectors;
          double s2[2], y2[2], p2[2];
          const int n = intersections(h, sector_alpha(sphi), xr, s2, y2, p2);
          for (int i = 0; i < n; ++i) {
            if (s2[i] < s_eps || s2[i] > s_max) continue;
            if (std::fabs(y2[i]) > xr * th) continue;
            if (s2[i] < best_s) {
              best_s = s2[i]; best_y = y2[i]; best_psi = p2[i]; best_row = r; best_sphi = sphi;
            }
          }
        }
      }
      if (all || (best_row >= 0 && best_s < 40.0)) break;
    }
    if (best_row < 0) break;
    advance(h, best_s);
    if (std::fabs(h.Z) > kZMax) break;
    const double cpsi = std::cos(best_psi), spsi = std::sin(best_psi);
    const int dir = cpsi > 0 ? 1 : -1;
    if (prev_dir != 0 && dir != prev_dir) {
      ++leg;
      if (leg >= cfg.max_legs) break;
    }
    prev_dir = dir;
    Crossing c;
    c.sector = best_sphi + (h.Z > 0 ? 0 : kPhiSectors);
    c.row = best_row;
    c.leg = leg;
    c.y = best_y;
    c.z = h.Z;
    c.h = h;
    const double qpt = p.q / p.pt;
    if (dir > 0) {
      c.snp = spsi; c.tgl = h.tgl; c.qpt = qpt;
    } else {
      c.snp = -spsi; c.tgl = -h.tgl; c.qpt = -qpt;
    }
    out.push_back(c);
    last_row = best_row;
    last_sphi = best_sphi;
    if (cfg.ms_theta > 0) {
      const double g1 = rng.gauss(), g2 = rng.gauss();
      h.phi += cfg.ms_theta * g1 * std::sqrt(1.0 + h.tgl * h.tgl);
      h.tgl = std::tan(std::atan(h.tgl) + cfg.ms_theta * g2);
    }
  }
}

// Helix point at local x = xq near arc length s_ref of the crossing (for the
// distortion inversion).  h0 is the helix at the crossing.
bool helix_at_x(const Helix& h0, double alpha, double xq, double* y, double* z) {
  const double ca = std::cos(alpha), sa = std::sin(alpha);
  const double ik = 1.0 / h0.kappa;
  const double Xc = h0.X - std::sin(h0.phi) * ik, Yc = h0.Y + std::cos(h0.phi) * ik;
  const double cx = Xc * ca + Yc * sa, cy = -Xc * sa + Yc * ca;
  const double v = h0.kappa * (xq - cx);
  if (v >= 1.0 || v <= -1.0) return false;
  const double psi0 = h0.phi - alpha;
  const double as = std::asin(v);
  double best = 1e300;
  for (double psi : {as, kPi - as}) {
    double d = std::remainder(psi - psi0, 2.0 * kPi);  // signed, closest branch
    const double s = d / h0.kappa;
    if (std::fabs(s) < std::fabs(best)) {
      best = s;
      *y = cy - std::cos(psi) * ik;
    }
  }
  *z = h0.Z + h0.tgl * best;
  return std::fabs(best) < 50.0;
}

}  // namespace

struct synth_result {
  std::vector<float> y, z;
  std::vector<uint16_t> q;
  std::vector<uint8_t> row, sector;
  std::vector<int32_t> label;
  std::vector<double> ty, tz, tsnp, ttgl, tqpt;  // truth per cluster (optional)
  std::vector<double> tyu, tzu;  // undistorted crossing (with the drift shift), truth
  std::vector<double> p_pt, p_q, p_tgl, p_phi, p_t0, p_vx, p_vy;
  std::vector<int32_t> p_secondary, p_ncl_leg0, p_ncl_leg1;
  std::vector<double> sector_thin;
  double z_lo[2] = {0, 0}, z_hi[2] = {0, 0};
};

namespace {

uint16_t landau_charge(Rng& rng) {
  // Chambers-Mallows-Stuck sampler of the stable law alpha=1, beta=1 (Landau);
  // mode ~ -0.2228 in this parametrisation, shifted to 50 and scaled by 10.
  const double U = kPi * (rng.uni() - 0.5);
  const double W = rng.expo(1.0);
  const double hp = 0.5 * kPi;
  const double X = (2.0 / kPi) * ((hp + U) * std::tan(U) - std::log(hp * W * std::cos(U) / (hp + U)));
  double q = 50.0 + 10.0 * (X + 0.22278);
  if (q < 1) q = 1;
  if (q > 65535) q = 65535;
  return (uint16_t)std::lround(q);
}

}  // namespace

extern "C" {

void synth_philox(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
  Philox::block(ctr, key[0], key[1], out);
}

int synth_generate(const synth_config* cfgp, synth_result** out) {
  if (!cfgp || !out) return 1;
  const synth_config& cfg = *cfgp;
  auto* res = new synth_result();
  Rng ev(cfg.seed, 0, kStreamEvent, (uint32_t)cfg.frame);

  // Event structure: list of (particle, collision t0).
  std::vector<Particle> parts;
  // Occupancy modulation: acceptance factor 0.04^(0.5*(1+cos(phi - psi_side)))
  // of the azimuth at mid radius, with a random phase per side, so that the
  // load of the 36 sectors spans about a factor 10 within one frame.
  const double psi_side[2] = {2.0 * kPi * ev.uni(), 2.0 * kPi * ev.uni()};
  auto thin_factor = [&](double phi, int side) {
    if (!cfg.thin_sectors) return 1.0;
    return std::pow(0.04, 0.5 * (1.0 + std::cos(phi - psi_side[side])));
  };
  std::vector<double> thin(2 * kPhiSectors, 1.0);
  double mean_thin = 0;
  for (int s = 0; s < 2 * kPhiSectors; ++s) {
    thin[s] = thin_factor(sector_alpha(s % kPhiSectors), s / kPhiSectors);
    mean_thin += thin[s];
  }
  mean_thin /= thin.size();
  res->sector_thin = thin;

  std::vector<double> coll_t0;
  std::vector<long> coll_mult;
  if (cfg.mode == 0) {
    coll_t0.push_back(0.0);
    coll_mult.push_back(cfg.n_primaries);
  } else {
    const long nc = ev.poisson(cfg.mean_collisions);
    for (long i = 0; i < nc; ++i) {
      coll_t0.push_back(cfg.frame_us * ev.uni());
      double m = ev.expo(cfg.mean_mult);
      if (m > cfg.mult_cap) m = cfg.mult_cap;
      // Thinning removes particles by sector; rescale so the mean load is kept.
      coll_mult.push_back((long)std::floor(m / mean_thin + 0.5));
    }
  }
  long pid = 0;
  for (size_t ic = 0; ic < coll_t0.size(); ++ic) {
    // vertex z of the collision, from a stream of its own (drawn only when
    // the spread is on, so that the other draws do not change)
    double vz = 0.0;
    if (cfg.vz_sigma > 0) {
      Rng vr(cfg.seed, (uint32_t)ic, kStreamEvent + 16, (uint32_t)cfg.frame);
      vz = cfg.vz_sigma * vr.gauss();
    }
    for (long j = 0; j < coll_mult[ic]; ++j, ++pid) {
      Rng pr(cfg.seed, (uint32_t)pid, kStreamParticle, (uint32_t)cfg.frame);
      Particle p{};
      const double a = std::pow(cfg.pt_min, 1.0 - cfg.pt_power);
      const double b = std::pow(cfg.pt_max, 1.0 - cfg.pt_power);
      p.pt = std::pow(a + pr.uni() * (b - a), 1.0 / (1.0 - cfg.pt_power));
      if (cfg.looper_frac > 0 && pr.uni() < cfg.looper_frac)
        p.pt = cfg.looper_pt_min + pr.uni() * (cfg.looper_pt_max - cfg.looper_pt_min);
      p.q = pr.uni() < 0.5 ? -1.0 : 1.0;
      const double eta = cfg.eta_min + pr.uni() * (cfg.eta_max - cfg.eta_min);
      p.tgl = std::sinh(eta);
      p.phi0 = cfg.phi_min + pr.uni() * (cfg.phi_max - cfg.phi_min);
      // azimuth of the trajectory at mid radius (165 cm) for a track from the origin
      const double kap = -p.q * cfg.bz * kBToCurv / p.pt;
      const double bend = (kap > 0 ? 1.0 : -1.0) * std::asin(std::min(1.0, std::fabs(kap) * 165.0 / 2.0));
      if (cfg.aim_radius > 0) {
        const double b = (kap > 0 ? 1.0 : -1.0) *
                         std::asin(std::min(1.0, std::fabs(kap) * cfg.aim_radius / 2.0));
        p.phi0 -= b;
      }
      const double phi_mid = p.phi0 + bend;
      p.t0 = coll_t0[ic];
      p.vz = vz;
      p.secondary = 0;
      p.vx = p.vy = 0;
      if (cfg.sec_frac > 0 && pr.uni() < cfg.sec_frac) {
        const double rv = cfg.sec_rmax * pr.uni(), av = 2.0 * kPi * pr.uni();
        p.vx = rv * std::cos(av);
        p.vy = rv * std::sin(av);
        p.secondary = 1;
      }
      if (cfg.thin_sectors) {
        const int side = p.tgl >= 0 ? 0 : 1;
        if (pr.uni() > thin_factor(phi_mid, side)) continue;
      }
      parts.push_back(p);
      (void)j;
    }
  }
  const long np = (long)parts.size();
  std::vector<std::vector<Crossing>> cross(np);
  DistField field;
  if (cfg.map) {
    field.c = cfg.map;
    field.nphi = cfg.map_nphi; field.nr = cfg.map_nr; field.nz = cfg.map_nz;
    field.rmin = cfg.map_rmin; field.rmax = cfg.map_rmax;
    field.zmin = cfg.map_zmin; field.zmax = cfg.map_zmax;
  }
#ifdef _OPENMP
  if (cfg.n_threads > 0) omp_set_num_threads(cfg.n_threads);
#pragma omp parallel for schedule(dynamic, 64)
#endif
  for (long i = 0; i < np; ++i) {
    Rng pr(cfg.seed, (uint32_t)i, kStreamCluster, (uint32_t)cfg.frame);
    trace(cfg, parts[i], pr, cross[i]);
  }
  // Clusterize: noise, drift-time shift, distortion.
  std::vector<long> offs(np + 1, 0);
  for (long i = 0; i < np; ++i) {
    long n = 0;
    for (const auto& c : cross[i])
      if (cfg.only_sector < 0 || c.sector == cfg.only_sector) ++n;
    offs[i + 1] = offs[i] + n;
  }
  const long ntrk = offs[np];
  const long nnoise =
      cfg.noise_frac > 0 ? (long)std::floor(cfg.noise_frac / (1.0 - cfg.noise_frac) * ntrk + 0.5) : 0;
  const long ntot = ntrk + nnoise;
  res->y.resize(ntot); res->z.resize(ntot); res->q.resize(ntot);
  res->row.resize(ntot); res->sector.resize(ntot); res->label.resize(ntot);
  if (cfg.store_truth) {
    res->ty.assign(ntot, 0); res->tz.assign(ntot, 0); res->tsnp.assign(ntot, 0);
    res->ttgl.assign(ntot, 0); res->tqpt.assign(ntot, 0);
    res->tyu.assign(ntot, 0); res->tzu.assign(ntot, 0);
  }
  res->p_pt.resize(np); res->p_q.resize(np); res->p_tgl.resize(np); res->p_phi.resize(np);
  res->p_t0.resize(np); res->p_vx.resize(np); res->p_vy.resize(np);
  res->p_secondary.resize(np); res->p_ncl_leg0.assign(np, 0); res->p_ncl_leg1.assign(np, 0);
  const double vd = cfg.vdrift;
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 64)
#endif
  for (long i = 0; i < np; ++i) {
    const Particle& p = parts[i];
    res->p_pt[i] = p.pt; res->p_q[i] = p.q; res->p_tgl[i] = p.tgl; res->p_phi[i] = p.phi0;
    res->p_t0[i] = p.t0; res->p_vx[i] = p.vx; res->p_vy[i] = p.vy; res->p_secondary[i] = p.secondary;
    Rng cr(cfg.seed, (uint32_t)i, kStreamCluster + 16, (uint32_t)cfg.frame);
    long k = offs[i];
    for (const auto& c : cross[i]) {
      if (cfg.only_sector >= 0 && c.sector != cfg.only_sector) continue;
      const int side = c.sector < kPhiSectors ? 1 : -1;
      const double xr = row_x(c.row);
      double ym = c.y, zm = c.z;
      if (field.c) {
        // Find the measured point m on the pad row whose corrected position
        // m + D(m) lies on the true trajectory: fixed-point iteration.
        const double alpha = sector_alpha(c.sector % kPhiSectors);
        const Helix& h0 = c.h;
        for (int it = 0; it < 60; ++it) {
          double d[3];
          field.eval(c.sector, xr, ym, zm, d);
          double yh = 0, zh = 0;
          if (!helix_at_x(h0, alpha, xr + d[0], &yh, &zh)) break;
          const double yn = yh - d[1], zn = zh - d[2];
          const double delta = std::fabs(yn - ym) + std::fabs(zn - zm);
          ym = yn;
          zm = zn;
          if (delta < 1e-13) break;
        }
      }
      const double zshift = -side * vd * p.t0;
      res->y[k] = (float)(ym + cfg.sigma * cr.gauss());
      res->z[k] = (float)(zm + cfg.sigma * cr.gauss() + zshift);
      res->q[k] = landau_charge(cr);
      res->row[k] = (uint8_t)c.row;
      res->sector[k] = (uint8_t)c.sector;
      res->label[k] = (int32_t)(2 * i + c.leg);
      if (cfg.store_truth) {
        res->ty[k] = ym; res->tz[k] = zm + zshift;
        res->tyu[k] = c.y; res->tzu[k] = c.z + zshift;
        res->tsnp[k] = c.snp; res->ttgl[k] = c.tgl; res->tqpt[k] = c.qpt;
      }
      if (c.leg == 0) res->p_ncl_leg0[i]++; else res->p_ncl_leg1[i]++;
      ++k;
    }
  }
  // Noise clusters: uniform in (sector, row, y within acceptance, z in frame range).
  const double span_t = cfg.mode == 0 ? 0.0 : vd * cfg.frame_us;
  res->z_lo[0] = -span_t; res->z_hi[0] = kZMax;           // side A (measured)
  res->z_lo[1] = -kZMax; res->z_hi[1] = span_t;           // side C (measured)
  if (cfg.mode == 0) { res->z_lo[0] = 0; res->z_hi[1] = 0; }
  {
    Rng nr(cfg.seed, 0, kStreamNoise, (uint32_t)cfg.frame);
    for (long j = 0; j < nnoise; ++j) {
      const long k = ntrk + j;
      int s = cfg.only_sector >= 0 ? cfg.only_sector : (int)(nr.uni() * 2 * kPhiSectors);
      if (s > 2 * kPhiSectors - 1) s = 2 * kPhiSectors - 1;
      int r = (int)(nr.uni() * kRows);
      if (r > kRows - 1) r = kRows - 1;
      const double xr = row_x(r);
      const double yy = (2.0 * nr.uni() - 1.0) * xr * tan_half();
      const int side = s < kPhiSectors ? 0 : 1;
      const double zz = res->z_lo[side] + nr.uni() * (res->z_hi[side] - res->z_lo[side]);
      res->y[k] = (float)yy;
      res->z[k] = (float)zz;
      res->q[k] = landau_charge(nr);
      res->row[k] = (uint8_t)r;
      res->sector[k] = (uint8_t)s;
      res->label[k] = -1;
      if (cfg.store_truth) {
        res->ty[k] = yy; res->tz[k] = zz;
        res->tyu[k] = yy; res->tzu[k] = zz;
      }
    }
  }
  if (cfg.shuffle && ntot > 1) {
    Rng sr(cfg.seed, 1, kStreamNoise + 1, (uint32_t)cfg.frame);
    std::vector<long> perm(ntot);
    for (long i = 0; i < ntot; ++i) perm[i] = i;
    for (long i = ntot - 1; i > 0; --i) {
      const long j = (long)(sr.uni() * (i + 1));
      std::swap(perm[i], perm[j < i ? j : i]);
    }
    auto apply = [&](auto& v) {
      if (v.empty()) return;
      auto w = v;
      for (long i = 0; i < ntot; ++i) v[i] = w[perm[i]];
    };
    apply(res->y); apply(res->z); apply(res->q); apply(res->row); apply(res->sector);
    apply(res->label); apply(res->ty); apply(res->tz); apply(res->tsnp); apply(res->ttgl);
    apply(res->tqpt); apply(res->tyu); apply(res->tzu);
  }
  *out = res;
  return 0;
}

long synth_count(const synth_result* r, const char* what) {
  if (!r || !what) return -1;
  const std::string w(what);
  if (w == "clusters") return (long)r->y.size();
  if (w == "particles") return (long)r->p_pt.size();
  if (w == "truth") return (long)r->ty.size();
  return -1;
}

int synth_copy(const synth_result* r, const char* what, void* dst, long cap) {
  if (!r || !what || !dst) return 1;
  const std::string w(what);
  auto cp = [&](const auto& v) -> int {
    const long bytes = (long)(v.size() * sizeof(v[0]));
    if (bytes > cap) return 2;
    if (bytes) std::memcpy(dst, v.data(), bytes);
    return 0;
  };
  if (w == "y") return cp(r->y);
  if (w == "z") return cp(r->z);
  if (w == "q") return cp(r->q);
  if (w == "row") return cp(r->row);
  if (w == "sector") return cp(r->sector);
  if (w == "label") return cp(r->label);
  if (w == "ty") return cp(r->ty);
  if (w == "tz") return cp(r->tz);
  if (w == "tsnp") return cp(r->tsnp);
  if (w == "ttgl") return cp(r->ttgl);
  if (w == "tqpt") return cp(r->tqpt);
  if (w == "tyu") return cp(r->tyu);
  if (w == "tzu") return cp(r->tzu);
  if (w == "p_pt") return cp(r->p_pt);
  if (w == "p_q") return cp(r->p_q);
  if (w == "p_tgl") return cp(r->p_tgl);
  if (w == "p_phi") return cp(r->p_phi);
  if (w == "p_t0") return cp(r->p_t0);
  if (w == "p_vx") return cp(r->p_vx);
  if (w == "p_vy") return cp(r->p_vy);
  if (w == "p_secondary") return cp(r->p_secondary);
  if (w == "p_ncl_leg0") return cp(r->p_ncl_leg0);
  if (w == "p_ncl_leg1") return cp(r->p_ncl_leg1);
  if (w == "sector_thin") return cp(r->sector_thin);
  if (w == "z_range") {
    if (cap < (long)(4 * sizeof(double))) return 2;
    double v[4] = {r->z_lo[0], r->z_hi[0], r->z_lo[1], r->z_hi[1]};
    std::memcpy(dst, v, sizeof v);
    return 0;
  }
  return 3;
}

void synth_free(synth_result* r) { delete r; }

// Control points of the synthetic space-charge field: radial displacement
// amp*(85/r)^2*(1-|z|/250) plus half of that azimuthally, expressed in the
// sector-local frame at the sector centre (x = radial, y = azimuthal).
int synth_distortion_profile(int nphi, int nr, int nz, double rmin, double rmax, double zmin,
                             double zmax, double amp, float* coeff) {
  if (!coeff || nphi < 1 || nr < 4 || nz < 4) return 1;
  for (int iz = 0; iz < nz; ++iz)
    for (int ir = 0; ir < nr; ++ir)
      for (int ip = 0; ip < nphi; ++ip) {
        const double r = rmin + (rmax - rmin) * (ir - 1.0) / (nr - 3.0);
        const double z = zmin + (zmax - zmin) * (iz - 1.0) / (nz - 3.0);
        const double rr = std::max(r, 60.0);
        double fz = 1.0 - std::fabs(z) / 250.0;
        if (fz < 0) fz = 0;
        const double rad = amp * (85.0 / rr) * (85.0 / rr) * fz;
        const long base = ((long)iz * nr + ir) * nphi + ip;
        const long stride = (long)nz * nr * nphi;
        coeff[0 * stride + base] = (float)rad;
        coeff[1 * stride + base] = (float)(0.5 * rad);
        coeff[2 * stride + base] = 0.0f;
      }
  return 0;
}

int synth_eval_distortion(const float* coeff, int nphi, int nr, int nz, double rmin, double rmax,
                          double zmin, double zmax, int sector, double x, double y, double z,
                          double* d) {
  DistField f;
  f.c = coeff; f.nphi = nphi; f.nr = nr; f.nz = nz;
  f.rmin = rmin; f.rmax = rmax; f.zmin = zmin; f.zmax = zmax;
  f.eval(sector, x, y, z, d);
  return 0;
}

}  // extern "C"
