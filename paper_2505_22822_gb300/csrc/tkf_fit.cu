// tkf_fit.cu -- Kalman-filter fit kernels for GB300 (sm_103a).
//
// One thread fits one track end to end with every per-track quantity in registers:
//   seed -> [update at k = 0] -> for k = 1..N-1: material at k-1 (Highland + Bethe mean
//   loss), RKN4 propagation to surface k with Jacobian transport, covariance transport,
//   gain-matrix update (Joseph form) + chi2, and one step of the smoother recursion.
// (Paper Sec. 2, second paragraph: RKN propagation with Jacobian transport, Kalman filter
// with chi2, RTS smoother for the first-measurement parameters.)
//
// Smoother. The RTS backward pass for the first surface,
//   p_0|N = p_0|0 + sum_{k>=1} G_k (p_k|k - p_k|k-1),  C_0|N = C_0|0 + sum_{k>=1} G_k (C_k|k - C_k|k-1) G_k^T,
// with G_k = A_0 ... A_{k-1} and A_j = C_j|j J_{j+1}^T C_{j+1|j}^-1, is evaluated forward in
// the same pass as the filter. With P_k = G_k C_k|k and R_k = P_{k-1} J_k^T one has
//   G_k C_k|k-1 H^T = R_k H^T,   P_k = R_k (I - K_k H)^T,
// so both sums need only R_k H^T (the first two columns of R_k), the gain K_k and S_k^-1:
//   p_0|N += R_k H^T S_k^-1 r_k,   C_0|N -= R_k H^T S_k^-1 H R_k^T.
// No C_{k+1|k}^-1 and no per-measurement state is stored: the smoother needs no scratch
// memory and no second pass (algebraically identical to the textbook RTS recursion).

#include <math.h>

#include "tkf_internal.cuh"

namespace tkf {
namespace {

constexpr double kKappa = 2.99792458e-4;  // GeV / (T mm)
constexpr double kPi = 3.14159265358979323846;
constexpr double kMe = 0.51099895e-3;  // GeV
constexpr double kBetheK = 0.307075;   // MeV cm^2 / mol

constexpr uint32_t kFatal = ~(TKF_TRACK_TOO_FEW_HITS | TKF_TRACK_OUT_OF_FIELD);

// index of (i, j) in the packed row-major upper triangle of a symmetric 5x5 matrix
__host__ __device__ constexpr int S(int i, int j) { return i <= j ? i * (9 - i) / 2 + j : j * (9 - j) / 2 + i; }

struct Surf {
  double u[3], v[3], n[3], c[3], t, x0, t_x0;
};

__device__ __forceinline__ void load_surf(const double* __restrict__ g, uint32_t id, Surf& s) {
  const double2* p = reinterpret_cast<const double2*>(g + size_t(id) * kSurfStride);
  double2 a0 = __ldg(p + 0), a1 = __ldg(p + 1), a2 = __ldg(p + 2), a3 = __ldg(p + 3);
  double2 a4 = __ldg(p + 4), a5 = __ldg(p + 5), a6 = __ldg(p + 6), a7 = __ldg(p + 7);
  s.u[0] = a0.x; s.u[1] = a0.y; s.u[2] = a1.x;
  s.v[0] = a1.y; s.v[1] = a2.x; s.v[2] = a2.y;
  s.n[0] = a3.x; s.n[1] = a3.y; s.n[2] = a4.x;
  s.c[0] = a4.y; s.c[1] = a5.x; s.c[2] = a5.y;
  s.t = a6.x; s.x0 = a6.y; s.t_x0 = a7.x;
}

__device__ __forceinline__ double dot3(const double a[3], const double b[3]) {
  return a[0] * b[0] + a[1] * b[1] + a[2] * b[2];
}

// ------------------------------------------------------------------ field policies
// Uniform field along z (the solenoid axis): T x B has no z component.
struct FieldUniformZ {
  double bz;
  static constexpr bool kUniform = true;
  __device__ __forceinline__ void at(const double*, double B[3], bool&) const {
    B[0] = 0.0; B[1] = 0.0; B[2] = bz;
  }
};

struct FieldUniform {
  double b[3];
  static constexpr bool kUniform = true;
  __device__ __forceinline__ void at(const double*, double B[3], bool&) const {
    B[0] = b[0]; B[1] = b[1]; B[2] = b[2];
  }
};

// Bilinear (r, z) interpolation of the (B_r, B_z) grid, FP64 arithmetic on FP32 nodes.
struct FieldGrid {
  const float2* __restrict__ grid;
  int nr, nz;
  double r0, z0, inv_dr, inv_dz;
  static constexpr bool kUniform = false;
  __device__ __forceinline__ void at(const double* x, double B[3], bool& oof) const {
    double r = sqrt(x[0] * x[0] + x[1] * x[1]);
    double fr = (r - r0) * inv_dr;
    double fz = (x[2] - z0) * inv_dz;
    if (!(fr >= 0.0 && fr <= double(nr - 1) && fz >= 0.0 && fz <= double(nz - 1))) {
      B[0] = B[1] = B[2] = 0.0;
      oof = true;
      return;
    }
    int ir = min(int(fr), nr - 2);
    int iz = min(int(fz), nz - 2);
    double a = fr - ir, b = fz - iz;
    const float2* g = grid + size_t(iz) * nr + ir;
    float2 g00 = __ldg(g), g01 = __ldg(g + 1), g10 = __ldg(g + nr), g11 = __ldg(g + nr + 1);
    double w00 = (1.0 - a) * (1.0 - b), w01 = a * (1.0 - b), w10 = (1.0 - a) * b, w11 = a * b;
    double br = w00 * g00.x + w01 * g01.x + w10 * g10.x + w11 * g11.x;
    double bz = w00 * g00.y + w01 * g01.y + w10 * g10.y + w11 * g11.y;
    if (r > 0.0) {
      double s = br / r;
      B[0] = s * x[0];
      B[1] = s * x[1];
    } else {
      B[0] = 0.0;
      B[1] = 0.0;
    }
    B[2] = bz;
  }
};

__device__ __forceinline__ void cross(const double a[3], const double b[3], double o[3]) {
  o[0] = a[1] * b[2] - a[2] * b[1];
  o[1] = a[2] * b[0] - a[0] * b[2];
  o[2] = a[0] * b[1] - a[1] * b[0];
}

// clamp((q)^(1/4), lo, hi) with the quarter root as two square roots
__device__ __forceinline__ double qroot(double q, double lo, double hi) {
  double f = sqrt(sqrt(q));
  return fmin(fmax(f, lo), hi);
}

// ------------------------------------------------------------------ propagation
// Adaptive RKN4 stepping of (r, T, lam) to the plane of `s`, transporting the derivative
// columns of (phi, theta, q/p): dr[c], dT[c] (c = 0, 1, 2). Step control (Lund 2009a):
// eps = h^2 |k1 - k2 - k3 + k4|_1; eps > tol rejects and sets h_ctrl = |h| max(1/4, (tol/eps)^1/4);
// an accepted step limited by h_ctrl sets h_ctrl = min(h_max, h_ctrl min(4, (tol/eps)^1/4)).
// Each step aims at the straight-line intersection; within surf_tol a straight step lands on the plane.
template <class F>
__device__ uint32_t propagate(const F& fld, const OptionsDev& o, const Surf& s, double r[3], double T[3],
                              double lam, double dr[3][3], double dT[3][3], double& h_ctrl,
                              uint32_t& attempts, uint32_t& rejected, double kend[3]) {
  uint32_t st = 0;
  bool first = true;
  uint32_t n_here = 0;
  const double lk = lam * kKappa;
  for (;;) {
    double dist = s.n[0] * (s.c[0] - r[0]) + s.n[1] * (s.c[1] - r[1]) + s.n[2] * (s.c[2] - r[2]);
    if (fabs(dist) <= o.surf_tol) {
      // close the last (<= surf_tol) distance with a straight step onto the plane
      const double sl = dist / dot3(s.n, T);
      for (int i = 0; i < 3; ++i) r[i] += sl * T[i];
      break;
    }
    double sl = dist / dot3(s.n, T);
    if (first && !(sl > -1.0 && isfinite(sl))) return st | TKF_TRACK_SURFACE_MISSED;
    first = false;
    if (n_here >= o.max_steps) return st | TKF_TRACK_MAX_STEPS;
    ++n_here;
    ++attempts;
    const bool limited = !(fabs(sl) < h_ctrl);
    const double h = limited ? copysign(h_ctrl, sl) : sl;
    const double h2 = 0.5 * h, h6 = h * (1.0 / 6.0);
    bool oof = false;
    double B1[3], B2[3], B4[3], Bt1[3], Bt2[3], Bt4[3];
    fld.at(r, B1, oof);
    for (int i = 0; i < 3; ++i) Bt1[i] = lk * B1[i];
    double k1[3], k2[3], k3[3], k4[3], T2[3], T3[3], T4[3];
    cross(T, Bt1, k1);
    if (F::kUniform) {
      for (int i = 0; i < 3; ++i) { B2[i] = B1[i]; Bt2[i] = Bt1[i]; }
    } else {
      double r2[3];
      for (int i = 0; i < 3; ++i) r2[i] = r[i] + h2 * T[i] + 0.125 * h * h * k1[i];
      fld.at(r2, B2, oof);
      for (int i = 0; i < 3; ++i) Bt2[i] = lk * B2[i];
    }
    for (int i = 0; i < 3; ++i) T2[i] = T[i] + h2 * k1[i];
    cross(T2, Bt2, k2);
    for (int i = 0; i < 3; ++i) T3[i] = T[i] + h2 * k2[i];
    cross(T3, Bt2, k3);
    if (F::kUniform) {
      for (int i = 0; i < 3; ++i) { B4[i] = B1[i]; Bt4[i] = Bt1[i]; }
    } else {
      double r4[3];
      for (int i = 0; i < 3; ++i) r4[i] = r[i] + h * T[i] + 0.5 * h * h * k3[i];
      fld.at(r4, B4, oof);
      for (int i = 0; i < 3; ++i) Bt4[i] = lk * B4[i];
    }
    for (int i = 0; i < 3; ++i) T4[i] = T[i] + h * k3[i];
    cross(T4, Bt4, k4);
    double eps = 0.0;
    for (int i = 0; i < 3; ++i) eps += fabs(k1[i] - k2[i] - k3[i] + k4[i]);
    eps *= h * h;
    if (eps > o.tol) {
      ++rejected;
      h_ctrl = fabs(h) * qroot(o.tol / eps, 0.25, 4.0);
      if (h_ctrl < o.h_min) return st | TKF_TRACK_STEP_UNDERFLOW;
      continue;
    }
    if (oof) st |= TKF_TRACK_OUT_OF_FIELD;
    // derivative columns through the accepted step (dB/dr neglected)
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      double q1[3], q2[3], q3[3], q4[3], u2[3], u3[3], u4[3];
      cross(dT[c], Bt1, q1);
      if (c == 2) {
        double e[3];
        double Bk1[3] = {kKappa * B1[0], kKappa * B1[1], kKappa * B1[2]};
        cross(T, Bk1, e);
        for (int i = 0; i < 3; ++i) q1[i] += e[i];
      }
      for (int i = 0; i < 3; ++i) u2[i] = dT[c][i] + h2 * q1[i];
      cross(u2, Bt2, q2);
      if (c == 2) {
        double e[3];
        double Bk2[3] = {kKappa * B2[0], kKappa * B2[1], kKappa * B2[2]};
        cross(T2, Bk2, e);
        for (int i = 0; i < 3; ++i) q2[i] += e[i];
      }
      for (int i = 0; i < 3; ++i) u3[i] = dT[c][i] + h2 * q2[i];
      cross(u3, Bt2, q3);
      if (c == 2) {
        double e[3];
        double Bk2[3] = {kKappa * B2[0], kKappa * B2[1], kKappa * B2[2]};
        cross(T3, Bk2, e);
        for (int i = 0; i < 3; ++i) q3[i] += e[i];
      }
      for (int i = 0; i < 3; ++i) u4[i] = dT[c][i] + h * q3[i];
      cross(u4, Bt4, q4);
      if (c == 2) {
        double e[3];
        double Bk4[3] = {kKappa * B4[0], kKappa * B4[1], kKappa * B4[2]};
        cross(T4, Bk4, e);
        for (int i = 0; i < 3; ++i) q4[i] += e[i];
      }
      for (int i = 0; i < 3; ++i) {
        dr[c][i] += h * dT[c][i] + h * h6 * (q1[i] + q2[i] + q3[i]);
        dT[c][i] += h6 * (q1[i] + 2.0 * q2[i] + 2.0 * q3[i] + q4[i]);
      }
    }
    for (int i = 0; i < 3; ++i) {
      r[i] += h * T[i] + h * h6 * (k1[i] + k2[i] + k3[i]);
      T[i] += h6 * (k1[i] + 2.0 * k2[i] + 2.0 * k3[i] + k4[i]);
    }
    if (limited) {
      double fac = (eps > 0.0) ? qroot(o.tol / eps, 0.25, 4.0) : 4.0;
      h_ctrl = fmin(o.h_max, h_ctrl * fac);
    }
  }
  double B[3], Bt[3];
  bool oof = false;
  fld.at(r, B, oof);
  if (oof) st |= TKF_TRACK_OUT_OF_FIELD;
  for (int i = 0; i < 3; ++i) Bt[i] = lk * B[i];
  cross(T, Bt, kend);
  return st;
}

// ------------------------------------------------------------------ material
// Thin layer at surface s crossed with unit direction T: returns theta0^2 (Highland) and
// lowers |q/p| by the Bethe mean loss (density effect: high-energy asymptote).
__device__ __forceinline__ uint32_t material(const Surf& s, const MaterialDev& m, double mass, const double T[3],
                                             double& lam, double& th0sq) {
  th0sq = 0.0;
  if (!(s.t > 0.0)) return 0;
  double x = s.t / fabs(dot3(s.n, T));
  double mom = 1.0 / fabs(lam);
  double E = sqrt(mom * mom + mass * mass);
  double beta = mom / E;
  double xx0 = x / s.x0;
  double th0 = 0.0136 / (beta * mom) * sqrt(xx0) * (1.0 + 0.038 * log(xx0 / (beta * beta)));
  th0sq = th0 * th0;
  double beta2 = beta * beta;
  double bg = mom / mass, bg2 = bg * bg;
  double gamma = E / mass;
  double me_m = kMe / mass;
  double wmax = 2.0 * kMe * bg2 / (1.0 + 2.0 * gamma * me_m + me_m * me_m);
  double I = m.i_ev * 1e-9;
  double half_delta = fmax(0.0, m.log_hwp_over_i + log(bg) - 0.5);
  double dedx = kBetheK * m.z_over_a / beta2 * (0.5 * log(2.0 * kMe * bg2 * wmax / (I * I)) - beta2 - half_delta);
  double dE = dedx * m.rho * (x * 0.1) * 1e-3;
  double E2 = E - dE;
  if (!(E2 > mass)) return TKF_TRACK_PARTICLE_STOPPED;
  lam = copysign(1.0 / sqrt(E2 * E2 - mass * mass), lam);
  return 0;
}

// ------------------------------------------------------------------ fit of one track
template <class F>
__device__ void fit_track(const FitArgs& a, const F& fld, uint32_t i) {
  const uint32_t n = a.n_tracks;
  const uint32_t b0 = a.offsets[i], b1 = a.offsets[i + 1];
  double p[5], C[15];
  for (int j = 0; j < 5; ++j) p[j] = a.seed_par[size_t(j) * n + i];
  for (int j = 0; j < 15; ++j) C[j] = a.seed_cov[size_t(j) * n + i];
  uint32_t status = 0, attempts = 0, rejected = 0;
  double chi2 = 0.0;
  int N = 0;
  double dl[5], E[15];
  const double nan = __longlong_as_double(0x7ff8000000000000LL);

  const bool bad_offsets = b1 < b0 || b1 > a.n_meas;
  if (bad_offsets) {
    status = TKF_TRACK_BAD_INPUT;  // never read outside the measurement arrays
  } else {
    N = int(b1 - b0);
    for (int k = 0; k < N; ++k)
      if (a.sid[b0 + k] >= a.n_surf) status = TKF_TRACK_BAD_INPUT;
  }
  if (N == 0 && status == 0) {
    for (int j = 0; j < 5; ++j) a.par[size_t(j) * n + i] = p[j];
    for (int j = 0; j < 15; ++j) a.cov[size_t(j) * n + i] = C[j];
    a.chi2[i] = 0.0;
    a.ndf[i] = 0;
    a.status[i] = TKF_TRACK_TOO_FEW_HITS;
    if (a.steps) { a.steps[i] = 0; a.steps[n + i] = 0; }
    return;
  }
  if (status == 0) {
    bool fin = true;
    for (int j = 0; j < 5; ++j) fin = fin && isfinite(p[j]);
    for (int j = 0; j < 15; ++j) fin = fin && isfinite(C[j]);
    if (!fin) status = TKF_TRACK_NON_FINITE;
  }

  double P[5][5];  // G_k C_k|k (smoother recursion)
  Surf sp;         // surface of the previous measurement
  double h_ctrl = a.opt.h_max;

  for (int k = 0; k < N && !(status & kFatal); ++k) {
    const uint32_t m = b0 + k;
    const uint32_t id = a.sid[m];
    Surf s;
    load_surf(a.surf, id, s);
    double J[5][5];
    if (k > 0) {
      // ---- material of the previous surface, then propagation (paper Sec. 3: muon hypothesis)
      double sph, cph, sth, cth;
      sincos(p[2], &sph, &cph);
      sincos(p[3], &sth, &cth);
      double T[3] = {sth * cph, sth * sph, cth};
      double lam = p[4], th0sq;
      status |= material(sp, a.mat, a.opt.mass, T, lam, th0sq);
      if (status & kFatal) break;
      double r[3];
      for (int j = 0; j < 3; ++j) r[j] = sp.c[j] + p[0] * sp.u[j] + p[1] * sp.v[j];
      double dr[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
      double dT[3][3] = {{-sth * sph, sth * cph, 0.0}, {cth * cph, cth * sph, -sth}, {0, 0, 0}};
      double kend[3];
      status |= propagate(fld, a.opt, s, r, T, lam, dr, dT, h_ctrl, attempts, rejected, kend);
      if (status & kFatal) break;
      // ---- bound parameters at the target and the transport Jacobian (path correction)
      double tnorm = sqrt(dot3(T, T));
      double tn[3] = {T[0] / tnorm, T[1] / tnorm, T[2] / tnorm};
      double st2 = sqrt(tn[0] * tn[0] + tn[1] * tn[1]);
      double ct2 = tn[2], cp2 = tn[0] / st2, sp2 = tn[1] / st2;
      double inv_nT = 1.0 / dot3(s.n, T);
#pragma unroll
      for (int c = 0; c < 5; ++c) {
        double x[3], t[3];
        for (int j = 0; j < 3; ++j) {
          x[j] = (c == 0) ? sp.u[j] : (c == 1) ? sp.v[j] : dr[c - 2][j];
          t[j] = (c < 2) ? 0.0 : dT[c - 2][j];
        }
        double ds = -dot3(s.n, x) * inv_nT;
        for (int j = 0; j < 3; ++j) {
          x[j] += T[j] * ds;
          t[j] += kend[j] * ds;
        }
        J[0][c] = dot3(s.u, x);
        J[1][c] = dot3(s.v, x);
        J[2][c] = (-sp2 * t[0] + cp2 * t[1]) / st2;
        J[3][c] = ct2 * cp2 * t[0] + ct2 * sp2 * t[1] - st2 * t[2];
        J[4][c] = (c == 4) ? 1.0 : 0.0;
      }
      double d[3] = {r[0] - s.c[0], r[1] - s.c[1], r[2] - s.c[2]};
      p[0] = dot3(s.u, d);
      p[1] = dot3(s.v, d);
      p[2] = atan2(tn[1], tn[0]);
      p[3] = acos(tn[2]);
      p[4] = lam;
      // ---- C_pred = J (C + Q) J^T, Q = diag(0, 0, th0^2/sin^2(theta), th0^2, 0)
      C[S(2, 2)] += th0sq / (sth * sth);
      C[S(3, 3)] += th0sq;
      double M[5][5];
#pragma unroll
      for (int r0 = 0; r0 < 4; ++r0)
#pragma unroll
        for (int c0 = 0; c0 < 5; ++c0) {
          double acc = 0.0;
#pragma unroll
          for (int q = 0; q < 5; ++q) acc += J[r0][q] * C[S(q, c0)];
          M[r0][c0] = acc;
        }
#pragma unroll
      for (int c0 = 0; c0 < 5; ++c0) M[4][c0] = C[S(4, c0)];
#pragma unroll
      for (int r0 = 0; r0 < 5; ++r0)
#pragma unroll
        for (int c0 = r0; c0 < 5; ++c0) {
          double acc;
          if (c0 == 4) {
            acc = M[r0][4];
          } else {
            acc = 0.0;
#pragma unroll
            for (int q = 0; q < 5; ++q) acc += M[r0][q] * J[c0][q];
          }
          C[S(r0, c0)] = acc;
        }
      // ---- smoother: R = P J^T (in place; J row 4 is e_4)
#pragma unroll
      for (int r0 = 0; r0 < 5; ++r0) {
        double row[5];
#pragma unroll
        for (int c0 = 0; c0 < 4; ++c0) {
          double acc = 0.0;
#pragma unroll
          for (int q = 0; q < 5; ++q) acc += P[r0][q] * J[c0][q];
          row[c0] = acc;
        }
        row[4] = P[r0][4];
#pragma unroll
        for (int c0 = 0; c0 < 5; ++c0) P[r0][c0] = row[c0];
      }
    }
    // ---- gain-matrix update with H = [I2 0]; Joseph form (paper Sec. 2; Fruhwirth 1987)
    const double m0 = a.loc0[m], m1 = a.loc1[m];
    const double V00 = a.v00[m], V01 = a.v01[m], V11 = a.v11[m];
    const double S00 = C[S(0, 0)] + V00, S01 = C[S(0, 1)] + V01, S11 = C[S(1, 1)] + V11;
    const double det = S00 * S11 - S01 * S01;
    if (!(S00 > 0.0 && det > 0.0)) {
      status |= TKF_TRACK_UPDATE_NOT_SPD;
      break;
    }
    const double idet = 1.0 / det;
    const double Si00 = S11 * idet, Si01 = -S01 * idet, Si11 = S00 * idet;
    const double r0 = m0 - p[0], r1 = m1 - p[1];
    chi2 += r0 * (Si00 * r0 + Si01 * r1) + r1 * (Si01 * r0 + Si11 * r1);
    double K[5][2];
#pragma unroll
    for (int j = 0; j < 5; ++j) {
      const double U0 = C[S(j, 0)], U1 = C[S(j, 1)];
      K[j][0] = U0 * Si00 + U1 * Si01;
      K[j][1] = U0 * Si01 + U1 * Si11;
    }
#pragma unroll
    for (int j = 0; j < 5; ++j) p[j] += K[j][0] * r0 + K[j][1] * r1;
    {
      // X = (I - K H) C ; C' = X - (X H^T - K V) K^T
      double X[5][5];
#pragma unroll
      for (int r_ = 0; r_ < 5; ++r_)
#pragma unroll
        for (int c_ = 0; c_ < 5; ++c_) X[r_][c_] = C[S(r_, c_)] - K[r_][0] * C[S(0, c_)] - K[r_][1] * C[S(1, c_)];
      double Y[5][2];
#pragma unroll
      for (int r_ = 0; r_ < 5; ++r_) {
        Y[r_][0] = X[r_][0] - (K[r_][0] * V00 + K[r_][1] * V01);
        Y[r_][1] = X[r_][1] - (K[r_][0] * V01 + K[r_][1] * V11);
      }
#pragma unroll
      for (int r_ = 0; r_ < 5; ++r_)
#pragma unroll
        for (int c_ = r_; c_ < 5; ++c_) C[S(r_, c_)] = X[r_][c_] - Y[r_][0] * K[c_][0] - Y[r_][1] * K[c_][1];
    }
    if (p[2] > kPi) p[2] -= 2.0 * kPi;
    if (p[2] <= -kPi) p[2] += 2.0 * kPi;
    if (!(p[3] > 0.0 && p[3] < kPi)) {
      status |= TKF_TRACK_NON_FINITE;
      break;
    }
    if (k == 0) {
      // p_0|0 and C_0|0 start the smoothed sums; P_0 = C_0|0
#pragma unroll
      for (int j = 0; j < 5; ++j) dl[j] = p[j];
#pragma unroll
      for (int j = 0; j < 15; ++j) E[j] = C[j];
#pragma unroll
      for (int r_ = 0; r_ < 5; ++r_)
#pragma unroll
        for (int c_ = 0; c_ < 5; ++c_) P[r_][c_] = C[S(r_, c_)];
    } else {
      // W = R H^T S^-1; p_0|N += W r; C_0|N -= W (R H^T)^T; P = R - R H^T K^T
      double W[5][2];
#pragma unroll
      for (int j = 0; j < 5; ++j) {
        W[j][0] = P[j][0] * Si00 + P[j][1] * Si01;
        W[j][1] = P[j][0] * Si01 + P[j][1] * Si11;
        dl[j] += W[j][0] * r0 + W[j][1] * r1;
      }
#pragma unroll
      for (int r_ = 0; r_ < 5; ++r_)
#pragma unroll
        for (int c_ = r_; c_ < 5; ++c_) E[S(r_, c_)] -= W[r_][0] * P[c_][0] + W[r_][1] * P[c_][1];
#pragma unroll
      for (int r_ = 0; r_ < 5; ++r_) {
        const double R0 = P[r_][0], R1 = P[r_][1];
#pragma unroll
        for (int c_ = 0; c_ < 5; ++c_) P[r_][c_] -= R0 * K[c_][0] + R1 * K[c_][1];
      }
    }
    sp = s;
  }

  if (!(status & kFatal)) {
    if (dl[2] > kPi) dl[2] -= 2.0 * kPi;
    if (dl[2] <= -kPi) dl[2] += 2.0 * kPi;
    // positive definiteness of the smoothed covariance: all LDL^T pivots > 0
    double L[15];
#pragma unroll
    for (int j = 0; j < 15; ++j) L[j] = E[j];
    bool spd = true;
#pragma unroll
    for (int j = 0; j < 5; ++j) {
      double d = L[S(j, j)];
      spd = spd && (d > 0.0);
      double inv = 1.0 / d;
#pragma unroll
      for (int r_ = j + 1; r_ < 5; ++r_) {
        double f = L[S(j, r_)] * inv;
#pragma unroll
        for (int c_ = r_; c_ < 5; ++c_) L[S(r_, c_)] -= f * L[S(j, c_)];
      }
    }
    if (!spd) status |= TKF_TRACK_SMOOTHER_NOT_SPD;
    bool fin = isfinite(chi2);
#pragma unroll
    for (int j = 0; j < 5; ++j) fin = fin && isfinite(dl[j]);
#pragma unroll
    for (int j = 0; j < 15; ++j) fin = fin && isfinite(E[j]);
    if (!fin) status |= TKF_TRACK_NON_FINITE;
  }
  if (status & kFatal) {
#pragma unroll
    for (int j = 0; j < 5; ++j) dl[j] = nan;
#pragma unroll
    for (int j = 0; j < 15; ++j) E[j] = nan;
    chi2 = nan;
  }
  if (N < 3 && !bad_offsets) status |= TKF_TRACK_TOO_FEW_HITS;
#pragma unroll
  for (int j = 0; j < 5; ++j) a.par[size_t(j) * n + i] = dl[j];
#pragma unroll
  for (int j = 0; j < 15; ++j) a.cov[size_t(j) * n + i] = E[j];
  a.chi2[i] = chi2;
  a.ndf[i] = 2 * N;
  a.status[i] = status;
  if (a.steps) {
    a.steps[i] = attempts;
    a.steps[n + i] = rejected;
  }
}

template <class F>
__global__ void __launch_bounds__(128) fit_kernel(FitArgs a, F fld) {
  const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= a.n_tracks) return;
  fit_track(a, fld, i);
}

}  // namespace

cudaError_t launch_fit(const FitArgs& a, const FieldDev& f, int precision, cudaStream_t stream) {
  (void)precision;
  if (a.n_tracks == 0) return cudaSuccess;
  const int block = 128;
  const unsigned grid = (a.n_tracks + block - 1) / block;
  if (f.kind == TKF_FIELD_UNIFORM) {
    if (f.b[0] == 0.0 && f.b[1] == 0.0) {
      FieldUniformZ u{f.b[2]};
      fit_kernel<<<grid, block, 0, stream>>>(a, u);
    } else {
      FieldUniform u{{f.b[0], f.b[1], f.b[2]}};
      fit_kernel<<<grid, block, 0, stream>>>(a, u);
    }
  } else {
    FieldGrid g{f.grid, f.nr, f.nz, f.r0, f.z0, f.inv_dr, f.inv_dz};
    fit_kernel<<<grid, block, 0, stream>>>(a, g);
  }
  return cudaGetLastError();
}

}  // namespace tkf
