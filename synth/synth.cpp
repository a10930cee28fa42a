// synth.cpp -- seeded synthetic inputs for the track fitter and its tests.
//
// This module builds detector geometries, the solenoid field map and simulated tracks
// (measurements, seeds, truth). It serves both the CUDA fitter and the CPU oracle and
// holds none of the fitter's arithmetic: no Runge-Kutta-Nystrom stepping, no Jacobian,
// no Kalman update or smoother. Truth trajectories are exact helix segments (field taken
// at the segment midpoint); the simulated world scatters by a Gaussian kick of the
// Highland width and loses the Bethe mean energy at each crossed module, which is the
// physics the fitter is asked to model (paper Sec. 3: material effects for a muon
// hypothesis, uniform 2 T solenoid field along z).
//
// Random numbers: SplitMix64 (Steele, Lea, Flood 2014) seeds one xoshiro256** stream
// (Blackman, Vigna 2018) per (seed, event, track, attempt); normals by Box-Muller.

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <thread>
#include <vector>

namespace {

const double kPi = 3.14159265358979323846;
const double kC = 2.99792458e-4;  // GeV / (T mm)
const double kMe = 0.51099895e-3;  // GeV

// ------------------------------------------------------------------ RNG
uint64_t splitmix_next(uint64_t& x) {
  uint64_t z = (x += 0x9e3779b97f4a7c15ULL);
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
  return z ^ (z >> 31);
}

inline uint64_t rotl(uint64_t x, int k) { return (x << k) | (x >> (64 - k)); }

struct Rng {
  uint64_t s[4];
  explicit Rng(uint64_t seed, uint64_t a, uint64_t b, uint64_t c) {
    uint64_t x = seed;
    uint64_t k = splitmix_next(x);
    x = k ^ (a * 0xd1b54a32d192ed03ULL);
    k = splitmix_next(x);
    x = k ^ (b * 0xaef17502108ef2d9ULL);
    k = splitmix_next(x);
    x = k ^ (c * 0xf58f8c8e2a1b6b35ULL);
    for (int i = 0; i < 4; ++i) s[i] = splitmix_next(x);
  }
  uint64_t next() {
    uint64_t result = rotl(s[1] * 5, 7) * 9;
    uint64_t t = s[1] << 17;
    s[2] ^= s[0];
    s[3] ^= s[1];
    s[1] ^= s[2];
    s[0] ^= s[3];
    s[2] ^= t;
    s[3] = rotl(s[3], 45);
    return result;
  }
  double uniform() { return double(next() >> 11) * (1.0 / 9007199254740992.0); }  // [0, 1)
  double normal() {
    double u1 = 1.0 - uniform();  // (0, 1]
    double u2 = uniform();
    return std::sqrt(-2.0 * std::log(u1)) * std::cos(2.0 * kPi * u2);
  }
};

// ------------------------------------------------------------------ geometry
struct Surf {
  double u[3], v[3], n[3], c[3], t, X0;
  double hu, hv;  // half extents along u and v (inf: unbounded)
};

struct BarrelLayer {
  double r;
  int nphi;
  uint32_t first;  // id of (iz=0, iphi=0)
};
struct DiskRing {
  double rc;
  int nphi;
  uint32_t first;
};
struct Disk {
  double z;  // signed nominal z
  std::vector<DiskRing> rings;
};

struct Geometry {
  int kind;  // 0 telescope, 1 barrel + endcaps
  std::vector<Surf> s;
  std::vector<BarrelLayer> layers;
  std::vector<Disk> disks;
  int nrows;
  double row_pitch;
  double ring_pitch;
};

const double kBarrelRowPitch = 68.0;
const int kBarrelRows = 18;
const double kRingPitch = 68.0;

void make_frame(Surf& s, const double u[3], const double v[3]) {
  for (int i = 0; i < 3; ++i) {
    s.u[i] = u[i];
    s.v[i] = v[i];
  }
  s.n[0] = u[1] * v[2] - u[2] * v[1];
  s.n[1] = u[2] * v[0] - u[0] * v[2];
  s.n[2] = u[0] * v[1] - u[1] * v[0];
}

Geometry* telescope(int n_planes, double spacing, double t, double X0) {
  Geometry* g = new Geometry();
  g->kind = 0;
  for (int i = 0; i < n_planes; ++i) {
    Surf s;
    double u[3] = {0, 1, 0}, v[3] = {0, 0, 1};
    make_frame(s, u, v);  // n = +x
    s.c[0] = spacing * i;
    s.c[1] = s.c[2] = 0.0;
    s.t = t;
    s.X0 = X0;
    s.hu = s.hv = INFINITY;
    g->s.push_back(s);
  }
  return g;
}

// Barrel: 10 layers at r_i = 32 (1000/32)^(i/9) mm of flat 30 (r-phi) x 70 (z) mm modules,
// n_phi = ceil(2 pi r / 28), 18 rows of pitch 68 mm; modules alternate +1 mm in radius on a
// checkerboard so that overlapping neighbours are never coplanar. Endcaps: 7 disks per side
// at |z| = 600 + 400 j mm, rings of 70 mm (radial) x 30 mm modules with radial pitch 68 mm
// from r = 32 mm, n_phi = ceil(2 pi r_c / 28); modules alternate +1 mm in |z|.
Geometry* barrel_endcap(double t, double X0) {
  Geometry* g = new Geometry();
  g->kind = 1;
  g->nrows = kBarrelRows;
  g->row_pitch = kBarrelRowPitch;
  g->ring_pitch = kRingPitch;
  for (int li = 0; li < 10; ++li) {
    BarrelLayer L;
    L.r = 32.0 * std::pow(1000.0 / 32.0, li / 9.0);
    L.nphi = int(std::ceil(2.0 * kPi * L.r / 28.0));
    L.first = uint32_t(g->s.size());
    for (int iz = 0; iz < kBarrelRows; ++iz)
      for (int ip = 0; ip < L.nphi; ++ip) {
        double phi = 2.0 * kPi * ip / L.nphi;
        double cp = std::cos(phi), sp = std::sin(phi);
        double rr = L.r + (((ip + iz) % 2) ? 1.0 : 0.0);
        Surf s;
        double u[3] = {-sp, cp, 0.0}, v[3] = {0.0, 0.0, 1.0};
        make_frame(s, u, v);  // n = radial
        s.c[0] = rr * cp;
        s.c[1] = rr * sp;
        s.c[2] = (iz - 0.5 * (kBarrelRows - 1)) * kBarrelRowPitch;
        s.t = t;
        s.X0 = X0;
        s.hu = 15.0;
        s.hv = 35.0;
        g->s.push_back(s);
      }
    g->layers.push_back(L);
  }
  for (int side = 0; side < 2; ++side)
    for (int j = 0; j < 7; ++j) {
      Disk D;
      double zabs = 600.0 + 400.0 * j;
      D.z = side == 0 ? -zabs : zabs;
      for (int k = 0;; ++k) {
        double rin = 32.0 + kRingPitch * k;
        if (rin >= 1000.0) break;
        DiskRing R;
        R.rc = rin + 35.0;
        R.nphi = int(std::ceil(2.0 * kPi * R.rc / 28.0));
        R.first = uint32_t(g->s.size());
        for (int ip = 0; ip < R.nphi; ++ip) {
          double phi = 2.0 * kPi * ip / R.nphi;
          double cp = std::cos(phi), sp = std::sin(phi);
          Surf s;
          double u[3] = {cp, sp, 0.0}, v[3] = {-sp, cp, 0.0};
          make_frame(s, u, v);  // n = +z
          double off = ((ip + k) % 2) ? 1.0 : 0.0;
          s.c[0] = R.rc * cp;
          s.c[1] = R.rc * sp;
          s.c[2] = D.z + (D.z > 0 ? off : -off);
          s.t = t;
          s.X0 = X0;
          s.hu = 35.0;
          s.hv = 15.0;
          g->s.push_back(s);
        }
        D.rings.push_back(R);
      }
      g->disks.push_back(D);
    }
  return g;
}

// ------------------------------------------------------------------ field
struct FieldDesc {
  int kind;
  double B[3];
  int nr, nz;
  double r0, dr, z0, dz;
  const float* Br;
  const float* Bz;
};

void field_value(const FieldDesc& f, const double x[3], double B[3]) {
  if (f.kind == 0) {
    for (int i = 0; i < 3; ++i) B[i] = f.B[i];
    return;
  }
  double r = std::hypot(x[0], x[1]);
  double gr = (r - f.r0) / f.dr, gz = (x[2] - f.z0) / f.dz;
  if (gr < 0 || gz < 0 || gr > f.nr - 1 || gz > f.nz - 1) {
    B[0] = B[1] = B[2] = 0.0;
    return;
  }
  int i = std::min(int(gr), f.nr - 2), j = std::min(int(gz), f.nz - 2);
  double a = gr - i, b = gz - j;
  auto at = [&](const float* M, int jj, int ii) { return double(M[jj * f.nr + ii]); };
  double br = (1 - b) * ((1 - a) * at(f.Br, j, i) + a * at(f.Br, j, i + 1)) +
              b * ((1 - a) * at(f.Br, j + 1, i) + a * at(f.Br, j + 1, i + 1));
  double bz = (1 - b) * ((1 - a) * at(f.Bz, j, i) + a * at(f.Bz, j, i + 1)) +
              b * ((1 - a) * at(f.Bz, j + 1, i) + a * at(f.Bz, j + 1, i + 1));
  B[0] = r > 0 ? br * x[0] / r : 0.0;
  B[1] = r > 0 ? br * x[1] / r : 0.0;
  B[2] = bz;
}

// Bulirsch's generalised complete elliptic integral
//   cel(kc, p, c, s) = int_0^{pi/2} (c cos^2 t + s sin^2 t) / ((cos^2 t + p sin^2 t) sqrt(cos^2 t + kc^2 sin^2 t)) dt
// by his arithmetic-geometric-mean iteration (R. Bulirsch, Numer. Math. 13 (1969) 305).
double cel(double kc, double p, double c, double s) {
  if (kc == 0.0) return NAN;
  const double tol = 1e-15;
  double k = std::fabs(kc), pp = p, cc = c, ss = s, em = 1.0;
  if (p > 0.0) {
    pp = std::sqrt(p);
    ss = s / pp;
  } else {
    double f = kc * kc, q = 1.0 - f, g = 1.0 - pp;
    f -= pp;
    q *= (ss - c * pp);
    pp = std::sqrt(f / g);
    cc = (c - ss) / g;
    ss = -q / (g * g * pp) + cc * pp;
  }
  double f = cc;
  cc += ss / pp;
  double g = k / pp;
  ss = 2.0 * (ss + f * g);
  pp += g;
  g = em;
  em += k;
  double kk = k;
  for (int it = 0; it < 60 && std::fabs(g - k) > g * tol; ++it) {
    k = 2.0 * std::sqrt(kk);
    kk = k * em;
    f = cc;
    cc += ss / pp;
    g = kk / pp;
    ss = 2.0 * (ss + f * g);
    pp += g;
    g = em;
    em += k;
  }
  return 0.5 * kPi * (ss + cc * em) / (em * (em + pp));
}

// Field of an ideal finite solenoid (current sheet of radius a, half-length b) in units of
// B0 = mu0 n I / pi, by the closed form of Derby & Olbert (Am. J. Phys. 78 (2010) 229).
void solenoid(double a, double b, double rho, double z, double* Brho, double* Bz) {
  double zp = z + b, zm = z - b;
  double dp = std::sqrt(zp * zp + (rho + a) * (rho + a));
  double dm = std::sqrt(zm * zm + (rho + a) * (rho + a));
  double ap = a / dp, am = a / dm, bp = zp / dp, bm = zm / dm;
  double gam = (a - rho) / (a + rho);
  double kp = std::sqrt((zp * zp + (a - rho) * (a - rho)) / (zp * zp + (a + rho) * (a + rho)));
  double km = std::sqrt((zm * zm + (a - rho) * (a - rho)) / (zm * zm + (a + rho) * (a + rho)));
  *Brho = ap * cel(kp, 1.0, 1.0, -1.0) - am * cel(km, 1.0, 1.0, -1.0);
  *Bz = a / (a + rho) * (bp * cel(kp, gam * gam, 1.0, gam) - bm * cel(km, gam * gam, 1.0, gam));
}

// ------------------------------------------------------------------ physics of the simulated world
double highland_sim(double p, double beta, double x_over_x0) {
  return 0.0136 / (beta * p) * std::sqrt(x_over_x0) * (1.0 + 0.038 * std::log(x_over_x0 / (beta * beta)));
}

// Mean loss in silicon (Bethe, PDG constants), MeV cm^2/g; density effect by its
// high-energy asymptote.
double bethe_sim(double p, double m) {
  const double ZA = 0.49848, I = 173e-9, hwp = 31.05e-9, K = 0.307075;
  double bg = p / m, g = std::sqrt(1.0 + bg * bg), b2 = bg * bg / (g * g);
  double r = kMe / m;
  double wmax = 2.0 * kMe * bg * bg / (1.0 + 2.0 * g * r + r * r);
  double hd = std::log(hwp / I) + std::log(bg) - 0.5;
  if (hd < 0) hd = 0;
  return K * ZA / b2 * (0.5 * std::log(2.0 * kMe * bg * bg * wmax / (I * I)) - b2 - hd);
}

// ------------------------------------------------------------------ helix
// Exact motion for path length s in a constant field B: dT/ds = kC * qop * T x B.
void helix(const double r[3], const double T[3], double qop, const double B[3], double s, double ro[3],
           double To[3]) {
  double Bm = std::sqrt(B[0] * B[0] + B[1] * B[1] + B[2] * B[2]);
  double a = kC * qop * Bm;
  if (Bm == 0.0 || std::fabs(a * s) < 1e-12) {
    for (int i = 0; i < 3; ++i) {
      ro[i] = r[i] + s * T[i];
      To[i] = T[i];
    }
    return;
  }
  double b[3] = {B[0] / Bm, B[1] / Bm, B[2] / Bm};
  double tb = T[0] * b[0] + T[1] * b[1] + T[2] * b[2];
  double tpar[3], tperp[3], w[3];
  for (int i = 0; i < 3; ++i) {
    tpar[i] = tb * b[i];
    tperp[i] = T[i] - tpar[i];
  }
  w[0] = tperp[1] * b[2] - tperp[2] * b[1];
  w[1] = tperp[2] * b[0] - tperp[0] * b[2];
  w[2] = tperp[0] * b[1] - tperp[1] * b[0];
  double as = a * s, c = std::cos(as), sn = std::sin(as);
  for (int i = 0; i < 3; ++i) {
    ro[i] = r[i] + tpar[i] * s + tperp[i] * sn / a + w[i] * (1.0 - c) / a;
    To[i] = tpar[i] + tperp[i] * c + w[i] * sn;
  }
}

// ------------------------------------------------------------------ simulation
struct Params {
  int start;     // 0: origin on surface 0, 1: vertex (0, 0, z0)
  int mom_mode;  // 0: p uniform, 1: pT log-uniform, 2: p log-uniform
  double pmin, pmax;
  int dir_mode;  // 0: phi, dip uniform in +-ang about +x; 1: phi uniform, eta uniform +-eta_max
  double ang, eta_max, z0_sigma;
  double mass;
  double sigma_hit;  // smearing sigma (0: exact hits)
  double sigma_v;    // sigma whose square is written as V00 = V11
  int ms, eloss;
  double seed_sigma[5];  // l0, l1 (mm), phi (rad), theta (rad, or cot(theta) if seed_cot), relative q/p
  int seed_smear;
  int seed_cot;          // 1: seed_sigma[3] is the sigma of cot(theta): sigma_theta = s sin^2(theta)
  double cov_inflate;
  int min_hits, max_hits;
  double step;
  double r_max, z_max;
  double p_hole;  // probability that a crossing after the first gives no measurement (a hole)
};

struct Hit {
  uint32_t sid;
  double l0, l1, t0, t1;  // smeared and true local position
  bool hole;              // crossed without a measurement
};

struct TrackSim {
  std::vector<Hit> hits;
  double truth[5];
  double seed[5];
  double seedcov[15];
  double truth_last[5];
};

void local_of(const Surf& s, const double x[3], double& l0, double& l1) {
  double d[3] = {x[0] - s.c[0], x[1] - s.c[1], x[2] - s.c[2]};
  l0 = s.u[0] * d[0] + s.u[1] * d[1] + s.u[2] * d[2];
  l1 = s.v[0] * d[0] + s.v[1] * d[1] + s.v[2] * d[2];
}

double sdist(const Surf& s, const double x[3]) {
  return s.n[0] * (x[0] - s.c[0]) + s.n[1] * (x[1] - s.c[1]) + s.n[2] * (x[2] - s.c[2]);
}

void candidates(const Geometry& g, const double a[3], const double b[3], double margin, std::vector<uint32_t>& out) {
  out.clear();
  if (g.kind == 0) {
    for (uint32_t i = 0; i < g.s.size(); ++i) out.push_back(i);
    return;
  }
  double ra = std::hypot(a[0], a[1]), rb = std::hypot(b[0], b[1]);
  double rlo = std::min(ra, rb) - margin, rhi = std::max(ra, rb) + margin;
  double zlo = std::min(a[2], b[2]) - margin, zhi = std::max(a[2], b[2]) + margin;
  double xm[3] = {0.5 * (a[0] + b[0]), 0.5 * (a[1] + b[1]), 0.5 * (a[2] + b[2])};
  double phim = std::atan2(xm[1], xm[0]);
  if (phim < 0) phim += 2.0 * kPi;
  double rm = std::hypot(xm[0], xm[1]);
  for (const BarrelLayer& L : g.layers) {
    double band_hi = std::sqrt((L.r + 1.0) * (L.r + 1.0) + 15.0 * 15.0);
    if (rhi < L.r || rlo > band_hi) continue;
    int ip0 = int(std::floor(phim / (2.0 * kPi / L.nphi) + 0.5));
    int iz0 = int(std::floor(xm[2] / g.row_pitch + 0.5 * g.nrows));
    for (int diz = -1; diz <= 1; ++diz) {
      int iz = iz0 + diz;
      if (iz < 0 || iz >= g.nrows) continue;
      for (int dip = -2; dip <= 2; ++dip) {
        int ip = ((ip0 + dip) % L.nphi + L.nphi) % L.nphi;
        out.push_back(L.first + uint32_t(iz * L.nphi + ip));
      }
    }
  }
  for (const Disk& D : g.disks) {
    double zl = D.z > 0 ? D.z : D.z - 1.0, zh = D.z > 0 ? D.z + 1.0 : D.z;
    if (zhi < zl || zlo > zh) continue;
    for (size_t k = 0; k < D.rings.size(); ++k) {
      const DiskRing& R = D.rings[k];
      double half_len = 0.5 * std::sqrt((b[0] - a[0]) * (b[0] - a[0]) + (b[1] - a[1]) * (b[1] - a[1]));
      if (rm < R.rc - 36.0 - half_len - margin ||
          rm > std::sqrt((R.rc + 35.0) * (R.rc + 35.0) + 225.0) + half_len + margin)
        continue;
      int ip0 = int(std::floor(phim / (2.0 * kPi / R.nphi) + 0.5));
      for (int dip = -2; dip <= 2; ++dip) {
        int ip = ((ip0 + dip) % R.nphi + R.nphi) % R.nphi;
        out.push_back(R.first + uint32_t(ip));
      }
    }
  }
}

void bound_truth(const Surf& s, const double x[3], const double T[3], double qop, double out[5]) {
  local_of(s, x, out[0], out[1]);
  out[2] = std::atan2(T[1], T[0]);
  out[3] = std::acos(std::max(-1.0, std::min(1.0, T[2])));
  out[4] = qop;
}

// Simulates one track; returns false when it has fewer than min_hits hits.
bool simulate(const Geometry& g, const FieldDesc& f, const Params& P, Rng& rng, TrackSim& tr) {
  tr.hits.clear();
  double p, phi, theta;
  double u1 = rng.uniform(), u2 = rng.uniform(), u3 = rng.uniform(), u4 = rng.uniform();
  double q = (rng.uniform() < 0.5) ? -1.0 : 1.0;
  double x[3] = {0, 0, 0}, T[3];
  if (P.dir_mode == 0) {
    double az = -P.ang + 2.0 * P.ang * u1, dip = -P.ang + 2.0 * P.ang * u2;
    T[0] = std::cos(dip) * std::cos(az);
    T[1] = std::cos(dip) * std::sin(az);
    T[2] = std::sin(dip);
    theta = std::acos(T[2]);
  } else {
    phi = 2.0 * kPi * u1;
    double eta = -P.eta_max + 2.0 * P.eta_max * u2;
    theta = 2.0 * std::atan(std::exp(-eta));
    T[0] = std::sin(theta) * std::cos(phi);
    T[1] = std::sin(theta) * std::sin(phi);
    T[2] = std::cos(theta);
  }
  if (P.mom_mode == 0) {
    p = P.pmin + (P.pmax - P.pmin) * u3;
  } else {
    double v = std::exp(std::log(P.pmin) + (std::log(P.pmax) - std::log(P.pmin)) * u3);
    p = (P.mom_mode == 1) ? v / std::sin(theta) : v;
  }
  (void)u4;
  if (P.start == 1) x[2] = P.z0_sigma * rng.normal();
  double qop = q / p;
  double path = 0.0;
  uint32_t last = 0xffffffffu;
  bool on_first = (P.start == 0);
  std::vector<uint32_t> cand;
  for (int it = 0; it < 200000; ++it) {
    int hit_sid = -1;
    double s_hit = 0.0;
    double xb[3], Tb[3], B[3];
    if (on_first) {
      hit_sid = 0;
      on_first = false;
      std::memcpy(xb, x, sizeof(xb));
      std::memcpy(Tb, T, sizeof(Tb));
    } else {
      double h = P.step;
      double xm[3] = {x[0] + 0.5 * h * T[0], x[1] + 0.5 * h * T[1], x[2] + 0.5 * h * T[2]};
      field_value(f, xm, B);
      helix(x, T, qop, B, h, xb, Tb);
      double bmag = std::sqrt(B[0] * B[0] + B[1] * B[1] + B[2] * B[2]);
      double margin = 0.2 + 0.125 * h * h * kC * std::fabs(qop) * bmag;  // + sagitta of the step
      candidates(g, x, xb, margin, cand);
      double best = h + 1.0;
      for (uint32_t id : cand) {
        const Surf& s = g.s[id];
        double da = sdist(s, x), db = sdist(s, xb);
        if (id == last && std::fabs(da) < 1e-7) continue;
        if ((da > 0) == (db > 0) && da != 0.0) continue;
        if (da == 0.0) continue;
        // root of n.(x(s) - c) in the bracket [0, h]: Newton from the secant, bisection
        // whenever an iterate leaves the bracket
        double lo = 0.0, hi = h, xm2[3], Tm2[3];
        double sc = h * da / (da - db);
        for (int it = 0; it < 60; ++it) {
          helix(x, T, qop, B, sc, xm2, Tm2);
          double fs = sdist(s, xm2);
          if (std::fabs(fs) < 1e-12) break;
          if ((fs > 0) == (da > 0))
            lo = sc;
          else
            hi = sc;
          double dfs = s.n[0] * Tm2[0] + s.n[1] * Tm2[1] + s.n[2] * Tm2[2];
          double nx = sc - fs / dfs;
          sc = (nx > lo && nx < hi && std::isfinite(nx)) ? nx : 0.5 * (lo + hi);
          if (hi - lo < 1e-13) break;
        }
        if (sc >= best) continue;
        helix(x, T, qop, B, sc, xm2, Tm2);
        double l0, l1;
        local_of(s, xm2, l0, l1);
        if (std::fabs(l0) > s.hu || std::fabs(l1) > s.hv) continue;
        best = sc;
        hit_sid = int(id);
        s_hit = sc;
      }
      if (hit_sid >= 0) {
        helix(x, T, qop, B, s_hit, xb, Tb);
        // land exactly on the plane: one straight correction of the (bisection) remainder
        const Surf& s = g.s[hit_sid];
        double d = sdist(s, xb);
        double cn = s.n[0] * Tb[0] + s.n[1] * Tb[1] + s.n[2] * Tb[2];
        for (int i = 0; i < 3; ++i) xb[i] -= d / cn * Tb[i];
        path += s_hit;
      } else {
        path += h;
      }
    }
    std::memcpy(x, xb, sizeof(x));
    double nt = std::sqrt(Tb[0] * Tb[0] + Tb[1] * Tb[1] + Tb[2] * Tb[2]);
    for (int i = 0; i < 3; ++i) T[i] = Tb[i] / nt;
    if (hit_sid >= 0) {
      const Surf& s = g.s[hit_sid];
      Hit H;
      H.sid = uint32_t(hit_sid);
      local_of(s, x, H.t0, H.t1);
      H.l0 = H.t0 + P.sigma_hit * rng.normal();
      H.l1 = H.t1 + P.sigma_hit * rng.normal();
      // a hole: the module is crossed (its material acts) but gives no measurement; drawn only
      // when holes are asked for, so that other workloads keep their random streams
      H.hole = P.p_hole > 0.0 && !tr.hits.empty() && rng.uniform() < P.p_hole;
      if (tr.hits.empty()) bound_truth(s, x, T, qop, tr.truth);
      bound_truth(s, x, T, qop, tr.truth_last);
      tr.hits.push_back(H);
      last = uint32_t(hit_sid);
      if (int(tr.hits.size()) >= P.max_hits) break;
      // material of the crossed module
      if (s.t > 0 && (P.ms || P.eloss)) {
        double cn = std::fabs(s.n[0] * T[0] + s.n[1] * T[1] + s.n[2] * T[2]);
        double xx = s.t / cn;
        double pm = 1.0 / std::fabs(qop);
        double E = std::sqrt(pm * pm + P.mass * P.mass), beta = pm / E;
        if (P.ms) {
          double th0 = highland_sim(pm, beta, xx / s.X0);
          double th = std::acos(std::max(-1.0, std::min(1.0, T[2])));
          double ph = std::atan2(T[1], T[0]);
          double e1[3] = {std::cos(th) * std::cos(ph), std::cos(th) * std::sin(ph), -std::sin(th)};
          double e2[3] = {-std::sin(ph), std::cos(ph), 0.0};
          double a1 = th0 * rng.normal(), a2 = th0 * rng.normal();
          double Tn[3];
          for (int i = 0; i < 3; ++i) Tn[i] = T[i] + a1 * e1[i] + a2 * e2[i];
          double nn = std::sqrt(Tn[0] * Tn[0] + Tn[1] * Tn[1] + Tn[2] * Tn[2]);
          for (int i = 0; i < 3; ++i) T[i] = Tn[i] / nn;
        }
        if (P.eloss) {
          double dE = bethe_sim(pm, P.mass) * 2.329 * (xx * 0.1) * 1e-3;
          double E2 = E - dE;
          if (!(E2 > P.mass)) break;
          qop = q / std::sqrt(E2 * E2 - P.mass * P.mass);
        }
      }
    }
    double rr = std::hypot(x[0], x[1]);
    if (rr > P.r_max || std::fabs(x[2]) > P.z_max || path > 20000.0) break;
  }
  int n_measured = 0;
  for (const Hit& h : tr.hits) n_measured += h.hole ? 0 : 1;
  if (n_measured < P.min_hits) return false;
  // seed: truth at the first measurement smeared by the nominal sigmas; covariance
  // diag(sigma^2) * cov_inflate (a diffuse prior).
  double sth = std::sin(tr.truth[3]);
  double sg[5] = {P.seed_sigma[0], P.seed_sigma[1], P.seed_sigma[2],
                  P.seed_cot ? P.seed_sigma[3] * sth * sth : P.seed_sigma[3],
                  P.seed_sigma[4] * std::fabs(tr.truth[4])};
  for (int i = 0; i < 5; ++i) tr.seed[i] = tr.truth[i] + (P.seed_smear ? sg[i] * rng.normal() : 0.0);
  if (tr.seed[2] > kPi) tr.seed[2] -= 2.0 * kPi;
  if (tr.seed[2] <= -kPi) tr.seed[2] += 2.0 * kPi;
  int idx = 0;
  for (int i = 0; i < 5; ++i)
    for (int j = i; j < 5; ++j) tr.seedcov[idx++] = (i == j) ? sg[i] * sg[i] * P.cov_inflate : 0.0;
  return true;
}

struct Result {
  std::vector<uint32_t> offsets;
  std::vector<uint32_t> sid;
  std::vector<double> meas;   // [m][5]
  std::vector<double> hit_truth;  // [m][2]
  std::vector<double> truth;  // [n][5]
  std::vector<double> seed;   // [n][5]
  std::vector<double> seedcov;  // [n][15]
  std::vector<double> truth_last;  // [n][5]
  std::vector<uint32_t> event;
};

}  // namespace

extern "C" {

struct syn_field {
  int kind;
  double B[3];
  int nr, nz;
  double r0, dr, z0, dz;
  const float* Br;
  const float* Bz;
};

struct syn_params {
  int start, mom_mode;
  double pmin, pmax;
  int dir_mode;
  double ang, eta_max, z0_sigma, mass, sigma_hit, sigma_v;
  int ms, eloss;
  double seed_sigma[5];
  int seed_smear, seed_cot;
  double cov_inflate;
  int min_hits, max_hits;
  double step, r_max, z_max;
  double p_hole;
};

void* syn_geometry_telescope(int n_planes, double spacing, double t, double X0) {
  return telescope(n_planes, spacing, t, X0);
}
void* syn_geometry_barrel_endcap(double t, double X0) { return barrel_endcap(t, X0); }
uint32_t syn_geometry_size(void* g) { return uint32_t(static_cast<Geometry*>(g)->s.size()); }
// out: [n][16] = u[3] v[3] n[3] c[3] t X0 hu hv
void syn_geometry_export(void* g, double* out) {
  const Geometry* G = static_cast<Geometry*>(g);
  for (size_t i = 0; i < G->s.size(); ++i) {
    const Surf& s = G->s[i];
    double* o = out + 16 * i;
    for (int j = 0; j < 3; ++j) {
      o[j] = s.u[j];
      o[3 + j] = s.v[j];
      o[6 + j] = s.n[j];
      o[9 + j] = s.c[j];
    }
    o[12] = s.t;
    o[13] = s.X0;
    o[14] = s.hu;
    o[15] = s.hv;
  }
}
void syn_geometry_free(void* g) { delete static_cast<Geometry*>(g); }

// Layer structure of a barrel + endcap geometry, for navigation: n_layers (10 barrel + 14 disks)
// rows of 8 doubles and n_rings rows of 4 doubles.
//   barrel: [0, r (nominal), nphi, n_rows, row_pitch, first id, half_u, half_v]
//           module (iz, ip) = first + iz nphi + ip, centre z = (iz - (n_rows - 1) / 2) row_pitch
//   disk:   [1, z (signed nominal), n_rings, first ring row, ring_pitch, r_inner, half_u, half_v]
//   ring:   [r_centre, nphi, first id, 0]; module ip = first + ip
// A telescope has no layer structure (0 layers).
void syn_geometry_layer_sizes(void* g, uint32_t* n_layers, uint32_t* n_rings) {
  const Geometry* G = static_cast<Geometry*>(g);
  *n_layers = uint32_t(G->layers.size() + G->disks.size());
  uint32_t r = 0;
  for (const Disk& D : G->disks) r += uint32_t(D.rings.size());
  *n_rings = r;
}
void syn_geometry_layers(void* g, double* layers, double* rings) {
  const Geometry* G = static_cast<Geometry*>(g);
  size_t li = 0, ri = 0;
  for (const BarrelLayer& L : G->layers) {
    double* o = layers + 8 * li++;
    o[0] = 0; o[1] = L.r; o[2] = L.nphi; o[3] = G->nrows; o[4] = G->row_pitch; o[5] = L.first; o[6] = 15.0; o[7] = 35.0;
  }
  for (const Disk& D : G->disks) {
    double* o = layers + 8 * li++;
    o[0] = 1; o[1] = D.z; o[2] = double(D.rings.size()); o[3] = double(ri); o[4] = G->ring_pitch; o[5] = 32.0;
    o[6] = 35.0; o[7] = 15.0;
    for (const DiskRing& R : D.rings) {
      double* q = rings + 4 * ri++;
      q[0] = R.rc; q[1] = R.nphi; q[2] = R.first; q[3] = 0;
    }
  }
}

double syn_cel(double kc, double p, double c, double s) { return cel(kc, p, c, s); }

void syn_solenoid(double a, double b, double rho, double z, double* Brho, double* Bz) {
  solenoid(a, b, rho, z, Brho, Bz);
}

// Tabulates the solenoid field on nodes r = r0 + i dr, z = z0 + j dz into Br/Bz [nz][nr]
// (float), scaled so that B_z(0, 0) = bz_center. Nodes on the sheet edges (r = a, |z| = b)
// are log-singular and are evaluated at r = a (1 - 1e-6).
void syn_solenoid_map(int nr, int nz, double r0, double dr, double z0, double dz, double a, double b,
                      double bz_center, float* Br, float* Bz) {
  double br0, bz0;
  solenoid(a, b, 0.0, 0.0, &br0, &bz0);
  double scale = bz_center / bz0;
  for (int j = 0; j < nz; ++j)
    for (int i = 0; i < nr; ++i) {
      double r = r0 + i * dr, z = z0 + j * dz;
      if (std::fabs(r - a) < 1e-9 * a && std::fabs(std::fabs(z) - b) < 1e-9 * b) r = a * (1.0 - 1e-6);
      double vr, vz;
      solenoid(a, b, r, z, &vr, &vz);
      Br[j * nr + i] = float(vr * scale);
      Bz[j * nr + i] = float(vz * scale);
    }
}

void syn_event_counts(uint64_t seed, uint32_t n_events, uint32_t lo, uint32_t hi, uint32_t* out) {
  for (uint32_t e = 0; e < n_events; ++e) {
    Rng r(seed, e, 0xffffffffULL, 0);
    out[e] = lo + uint32_t(r.next() % uint64_t(hi - lo + 1));
  }
}

void* syn_simulate(void* geom, const syn_field* field, const syn_params* params, uint64_t seed,
                   uint32_t n_events, const uint32_t* tracks_per_event, int n_threads) {
  const Geometry& g = *static_cast<Geometry*>(geom);
  FieldDesc f;
  f.kind = field->kind;
  for (int i = 0; i < 3; ++i) f.B[i] = field->B[i];
  f.nr = field->nr; f.nz = field->nz; f.r0 = field->r0; f.dr = field->dr; f.z0 = field->z0; f.dz = field->dz;
  f.Br = field->Br; f.Bz = field->Bz;
  Params P;
  std::memcpy(&P, params, sizeof(P));
  std::vector<std::pair<uint32_t, uint32_t>> work;
  for (uint32_t e = 0; e < n_events; ++e)
    for (uint32_t t = 0; t < tracks_per_event[e]; ++t) work.push_back({e, t});
  std::vector<TrackSim> sims(work.size());
  std::atomic<size_t> next(0);
  auto run = [&]() {
    for (;;) {
      size_t i = next.fetch_add(64);
      if (i >= work.size()) break;
      size_t end = std::min(work.size(), i + 64);
      for (; i < end; ++i) {
        for (uint64_t attempt = 0;; ++attempt) {
          Rng rng(seed, work[i].first, work[i].second, attempt);
          if (simulate(g, f, P, rng, sims[i])) break;
          if (attempt > 10000) {
            sims[i].hits.clear();
            break;
          }
        }
      }
    }
  };
  int nt = std::max(1, n_threads);
  std::vector<std::thread> th;
  for (int t = 0; t < nt; ++t) th.emplace_back(run);
  for (auto& t : th) t.join();
  Result* R = new Result();
  R->offsets.push_back(0);
  for (size_t i = 0; i < sims.size(); ++i) {
    const TrackSim& s = sims[i];
    for (const Hit& h : s.hits) {
      // a hole: surface id with the no-measurement bit, its measurement fields NaN (unused)
      R->sid.push_back(h.hole ? (h.sid | 0x80000000u) : h.sid);
      double v = P.sigma_v * P.sigma_v;
      const double nan = std::nan("");
      double m[5] = {h.l0, h.l1, v, 0.0, v};
      if (h.hole)
        for (double& x : m) x = nan;
      R->meas.insert(R->meas.end(), m, m + 5);
      R->hit_truth.push_back(h.t0);
      R->hit_truth.push_back(h.t1);
    }
    R->offsets.push_back(uint32_t(R->sid.size()));
    R->truth.insert(R->truth.end(), s.truth, s.truth + 5);
    R->seed.insert(R->seed.end(), s.seed, s.seed + 5);
    R->seedcov.insert(R->seedcov.end(), s.seedcov, s.seedcov + 15);
    R->truth_last.insert(R->truth_last.end(), s.truth_last, s.truth_last + 5);
    R->event.push_back(work[i].first);
  }
  return R;
}

void syn_result_sizes(void* r, uint64_t* n_tracks, uint64_t* n_hits) {
  Result* R = static_cast<Result*>(r);
  *n_tracks = R->offsets.size() - 1;
  *n_hits = R->sid.size();
}

void syn_result_export(void* r, uint32_t* offsets, uint32_t* sid, double* meas, double* hit_truth, double* truth,
                       double* seed, double* seedcov, double* truth_last, uint32_t* event) {
  Result* R = static_cast<Result*>(r);
  std::memcpy(offsets, R->offsets.data(), R->offsets.size() * sizeof(uint32_t));
  std::memcpy(sid, R->sid.data(), R->sid.size() * sizeof(uint32_t));
  std::memcpy(meas, R->meas.data(), R->meas.size() * sizeof(double));
  std::memcpy(hit_truth, R->hit_truth.data(), R->hit_truth.size() * sizeof(double));
  std::memcpy(truth, R->truth.data(), R->truth.size() * sizeof(double));
  std::memcpy(seed, R->seed.data(), R->seed.size() * sizeof(double));
  std::memcpy(seedcov, R->seedcov.data(), R->seedcov.size() * sizeof(double));
  std::memcpy(truth_last, R->truth_last.data(), R->truth_last.size() * sizeof(double));
  std::memcpy(event, R->event.data(), R->event.size() * sizeof(uint32_t));
}

void syn_result_free(void* r) { delete static_cast<Result*>(r); }

}  // extern "C"
