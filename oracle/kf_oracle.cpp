// kf_oracle.cpp -- TEST INFRASTRUCTURE, NOT PRODUCT CODE.
//
// A plain, slow, FP64 CPU Kalman-filter track fitter. Only tests/, the smoke()
// entry of __graft_entry__.py and the CPU-baseline leg of bench.py may load it.
// It shares no code, header, table or constant generator with the CUDA fitter.
//
// What it computes (paper Sec. 2, "Implementation", second paragraph): for each
// track candidate, the Kalman-filter fit with 4th-order Runge-Kutta-Nystrom (RKN)
// propagation and Jacobian transport between surfaces (refs Nystrom 1925,
// Bugge-Myrheim 1981, Lund et al. 2009a/b, Yeo et al. 2024), a gain-matrix update
// with a chi2 from the covariance-weighted spatial residual (ref Fruhwirth 1987),
// and the Rauch-Tung-Striebel (RTS) smoother (ref Rauch-Tung-Striebel 1965) so that
// the first-measurement parameters use every measurement. Material effects assume a
// muon (paper Sec. 3, first paragraph). The paper prints no formula for any of these;
// each formula below is the textbook form of the cited method, and every reading that
// the paper leaves open is marked "Reading:".
//
// Style: every matrix is a full dense array and every product is a plain triple
// loop; no structure (sparsity, symmetry, packing) is exploited, so that a reader can
// check each line against the textbook formula.
//
// Conventions fixed by reading, the same on both sides, each pinned by an invariant rather
// than by a printed value:
//   * the density-effect term of the Bethe formula (high-energy form): above its threshold
//     the mean excitation energy cancels and the loss takes the plasma-energy plateau form;
//   * the field gradient dB/dr, neglected in the Jacobian (exact in a uniform field): in a
//     map the Jacobian differs from finite differences only by a term linear in the gradient.

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <thread>
#include <vector>

namespace {

const double kKappa = 2.99792458e-4;  // c in GeV / (T mm): curvature = kKappa * B / p
const double kPi = 3.14159265358979323846;
const double kMe = 0.51099895e-3;     // electron mass, GeV
const double kBetheK = 0.307075;      // 4 pi N_A r_e^2 m_e c^2, MeV cm^2 / mol

// Per-track status bits (values fixed by the library interface).
const uint32_t kMaxSteps = 1u << 0;
const uint32_t kSurfaceMissed = 1u << 1;
const uint32_t kParticleStopped = 1u << 2;
const uint32_t kUpdateNotSpd = 1u << 3;
const uint32_t kSmootherNotSpd = 1u << 4;
const uint32_t kTooFewHits = 1u << 5;
const uint32_t kOutOfField = 1u << 6;
const uint32_t kBadInput = 1u << 7;
const uint32_t kStepUnderflow = 1u << 8;
const uint32_t kNonFinite = 1u << 9;
const uint32_t kFatal = ~(kTooFewHits | kOutOfField);

// Reading (navigation through surfaces without a measurement, Sec. 2): a track-state entry
// whose surface id carries this bit is a surface the track crosses without a measurement (a
// hole in a sensitive module, or a passive surface): the fit propagates to it and applies its
// material on leaving it, and makes no update there.
const uint32_t kNoMeasurement = 0x80000000u;
inline uint32_t surface_of(uint32_t sid) { return sid & ~kNoMeasurement; }
inline bool measured(uint32_t sid) { return (sid & kNoMeasurement) == 0; }

struct Surface {
  double u[3], v[3], n[3];  // local axes and normal (global frame); n = u x v
  double c[3];              // centre
  double t;                 // thickness, mm (0: no material)
  double X0;                // radiation length, mm
};

struct Field {
  int kind;  // 0 uniform, 1 r-z grid
  double B[3];
  int nr, nz;
  double r0, dr, z0, dz;
  const float* Br;  // [nz][nr]
  const float* Bz;  // [nz][nr]
};

// Learned step proposer (an addition, not in the paper): an MLP 12 -> 64 -> 64 -> 1 with SiLU
// activations whose weights are BF16 values; the forward pass is FP32 arithmetic.
struct Mlp {
  float W1[64][12], b1[64], W2[64][64], b2[64], w3[64], b3;
};

struct Opts {
  const Mlp* mlp;   // learned step proposals when not null
  double tol;       // RKN local error tolerance, mm
  double h_max;     // largest step, mm
  double h_min;     // smallest step-size control value, mm
  double surf_tol;  // distance to the target plane at which propagation stops, mm
  double mass;      // particle hypothesis, GeV
  uint32_t max_steps;
  double ZA, I_eV, rho, hwp_eV;  // material: Z/A, mean excitation, density g/cm3, plasma energy
  int smoother = 0;              // 0: RTS; 1: two-filter (forward filter, backward filter, weighted mean)
  double inflation = 1e3;        // two-filter: the backward filter starts from the last filtered
                                 // covariance times this factor
  std::vector<float>* records = nullptr;  // training records of the step proposer, when not null
};

// ---------------------------------------------------------------- dense algebra
void matmul(const double* A, const double* B, double* C, int n, int k, int m) {
  // C (n x m) = A (n x k) * B (k x m)
  std::vector<double> tmp(n * m, 0.0);
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < m; ++j) {
      double s = 0.0;
      for (int l = 0; l < k; ++l) s += A[i * k + l] * B[l * m + j];
      tmp[i * m + j] = s;
    }
  std::memcpy(C, tmp.data(), sizeof(double) * n * m);
}

void transpose(const double* A, double* At, int n, int m) {
  // At (m x n) = A (n x m)^T
  std::vector<double> tmp(n * m);
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < m; ++j) tmp[j * n + i] = A[i * m + j];
  std::memcpy(At, tmp.data(), sizeof(double) * n * m);
}

// Cholesky C = L L^T of an n x n matrix; false if not positive definite.
bool cholesky(const double* C, double* L, int n) {
  for (int i = 0; i < n * n; ++i) L[i] = 0.0;
  for (int j = 0; j < n; ++j) {
    double d = C[j * n + j];
    for (int k = 0; k < j; ++k) d -= L[j * n + k] * L[j * n + k];
    if (!(d > 0.0)) return false;
    L[j * n + j] = std::sqrt(d);
    for (int i = j + 1; i < n; ++i) {
      double s = C[i * n + j];
      for (int k = 0; k < j; ++k) s -= L[i * n + k] * L[j * n + k];
      L[i * n + j] = s / L[j * n + j];
    }
  }
  return true;
}

// Inverse of an SPD matrix by solving C X = I with its Cholesky factor.
bool spd_inverse(const double* C, double* Ci, int n) {
  std::vector<double> L(n * n);
  if (!cholesky(C, L.data(), n)) return false;
  for (int col = 0; col < n; ++col) {
    std::vector<double> y(n), x(n);
    for (int i = 0; i < n; ++i) {  // L y = e_col
      double s = (i == col) ? 1.0 : 0.0;
      for (int k = 0; k < i; ++k) s -= L[i * n + k] * y[k];
      y[i] = s / L[i * n + i];
    }
    for (int i = n - 1; i >= 0; --i) {  // L^T x = y
      double s = y[i];
      for (int k = i + 1; k < n; ++k) s -= L[k * n + i] * x[k];
      x[i] = s / L[i * n + i];
    }
    for (int i = 0; i < n; ++i) Ci[i * n + col] = x[i];
  }
  return true;
}

void symmetrize(double* C, int n) {
  for (int i = 0; i < n; ++i)
    for (int j = i + 1; j < n; ++j) {
      double a = 0.5 * (C[i * n + j] + C[j * n + i]);
      C[i * n + j] = a;
      C[j * n + i] = a;
    }
}

double wrap_phi(double phi) {
  // Reading: phi is kept in (-pi, pi].
  while (phi > kPi) phi -= 2.0 * kPi;
  while (phi <= -kPi) phi += 2.0 * kPi;
  return phi;
}

void cross(const double a[3], const double b[3], double out[3]) {
  out[0] = a[1] * b[2] - a[2] * b[1];
  out[1] = a[2] * b[0] - a[0] * b[2];
  out[2] = a[0] * b[1] - a[1] * b[0];
}

double dot3(const double a[3], const double b[3]) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }

// Matrix M(B) with M(B) T = T x B.
void cross_matrix(const double B[3], double M[9]) {
  M[0] = 0.0;   M[1] = B[2];  M[2] = -B[1];
  M[3] = -B[2]; M[4] = 0.0;   M[5] = B[0];
  M[6] = B[1];  M[7] = -B[0]; M[8] = 0.0;
}

// ---------------------------------------------------------------- field
// Uniform field, or bilinear interpolation in (r, z) of a tabulated solenoid map with
// B_x = B_r x / r, B_y = B_r y / r. Outside the grid B = 0 and the flag is raised.
void field_at(const Field& f, const double x[3], double B[3], bool* out_of_map) {
  if (f.kind == 0) {
    B[0] = f.B[0]; B[1] = f.B[1]; B[2] = f.B[2];
    return;
  }
  double r = std::sqrt(x[0] * x[0] + x[1] * x[1]);
  double fr = (r - f.r0) / f.dr;
  double fz = (x[2] - f.z0) / f.dz;
  if (!(fr >= 0.0 && fr <= double(f.nr - 1) && fz >= 0.0 && fz <= double(f.nz - 1))) {
    B[0] = B[1] = B[2] = 0.0;
    *out_of_map = true;
    return;
  }
  int ir = int(std::floor(fr));
  int iz = int(std::floor(fz));
  if (ir > f.nr - 2) ir = f.nr - 2;
  if (iz > f.nz - 2) iz = f.nz - 2;
  double a = fr - ir, b = fz - iz;
  double w00 = (1.0 - a) * (1.0 - b), w01 = a * (1.0 - b), w10 = (1.0 - a) * b, w11 = a * b;
  int i00 = iz * f.nr + ir, i01 = i00 + 1, i10 = i00 + f.nr, i11 = i10 + 1;
  double br = w00 * double(f.Br[i00]) + w01 * double(f.Br[i01]) + w10 * double(f.Br[i10]) + w11 * double(f.Br[i11]);
  double bz = w00 * double(f.Bz[i00]) + w01 * double(f.Bz[i01]) + w10 * double(f.Bz[i10]) + w11 * double(f.Bz[i11]);
  if (r > 0.0) {
    B[0] = br * x[0] / r;
    B[1] = br * x[1] / r;
  } else {
    B[0] = 0.0;
    B[1] = 0.0;
  }
  B[2] = bz;
}

// ---------------------------------------------------------------- RKN4 step
// One 4th-order Runge-Kutta-Nystrom step of length h for d2r/ds2 = kappa*lam*T x B(r)
// (Bugge-Myrheim / Lund 2009a form), with the 7x7 derivative D of the discrete map
// x = (r, T, lam) -> x' taken through the stages (Lund 2009b). dB/dr is neglected.
// The local error estimate is eps = h^2 * || k1 - k2 - k3 + k4 ||_1 (Lund 2009a).
struct Step {
  double r[3], T[3];
  double D[49];
  double eps;
  double dTds[3];  // k1 of the step (dT/ds at the start point)
};

void rkn_step(const Field& f, const double r[3], const double T[3], double lam, double h, Step& out,
              bool* oof) {
  double B1[3], B2[3], B4[3];
  field_at(f, r, B1, oof);
  double k1[3], k2[3], k3[3], k4[3], T2[3], T3[3], T4[3], r2[3], r4[3], c[3];
  cross(T, B1, c);
  for (int i = 0; i < 3; ++i) k1[i] = kKappa * lam * c[i];
  for (int i = 0; i < 3; ++i) {
    r2[i] = r[i] + 0.5 * h * T[i] + 0.125 * h * h * k1[i];
    T2[i] = T[i] + 0.5 * h * k1[i];
  }
  field_at(f, r2, B2, oof);
  cross(T2, B2, c);
  for (int i = 0; i < 3; ++i) k2[i] = kKappa * lam * c[i];
  for (int i = 0; i < 3; ++i) T3[i] = T[i] + 0.5 * h * k2[i];
  cross(T3, B2, c);
  for (int i = 0; i < 3; ++i) k3[i] = kKappa * lam * c[i];
  for (int i = 0; i < 3; ++i) {
    r4[i] = r[i] + h * T[i] + 0.5 * h * h * k3[i];
    T4[i] = T[i] + h * k3[i];
  }
  field_at(f, r4, B4, oof);
  cross(T4, B4, c);
  for (int i = 0; i < 3; ++i) k4[i] = kKappa * lam * c[i];

  for (int i = 0; i < 3; ++i) {
    out.r[i] = r[i] + h * T[i] + h * h / 6.0 * (k1[i] + k2[i] + k3[i]);
    out.T[i] = T[i] + h / 6.0 * (k1[i] + 2.0 * k2[i] + 2.0 * k3[i] + k4[i]);
    out.dTds[i] = k1[i];
  }
  double e = 0.0;
  for (int i = 0; i < 3; ++i) e += std::fabs(k1[i] - k2[i] - k3[i] + k4[i]);
  out.eps = h * h * e;

  // Stage derivatives w.r.t. T (3x3) and lam (3x1), by the chain rule.
  double M1[9], M2[9], M4[9], I3[9] = {1, 0, 0, 0, 1, 0, 0, 0, 1};
  cross_matrix(B1, M1);
  cross_matrix(B2, M2);
  cross_matrix(B4, M4);
  double dk1T[9], dk2T[9], dk3T[9], dk4T[9], dT2T[9], dT3T[9], dT4T[9];
  double dk1l[3], dk2l[3], dk3l[3], dk4l[3], dT2l[3], dT3l[3], dT4l[3];
  double tmp[9], c1[3], c2[3], c3[3], c4[3];
  for (int i = 0; i < 9; ++i) dk1T[i] = kKappa * lam * M1[i];
  cross(T, B1, c1);
  for (int i = 0; i < 3; ++i) dk1l[i] = kKappa * c1[i];
  for (int i = 0; i < 9; ++i) dT2T[i] = I3[i] + 0.5 * h * dk1T[i];
  for (int i = 0; i < 3; ++i) dT2l[i] = 0.5 * h * dk1l[i];
  matmul(M2, dT2T, tmp, 3, 3, 3);
  for (int i = 0; i < 9; ++i) dk2T[i] = kKappa * lam * tmp[i];
  cross(T2, B2, c2);
  matmul(M2, dT2l, tmp, 3, 3, 1);
  for (int i = 0; i < 3; ++i) dk2l[i] = kKappa * c2[i] + kKappa * lam * tmp[i];
  for (int i = 0; i < 9; ++i) dT3T[i] = I3[i] + 0.5 * h * dk2T[i];
  for (int i = 0; i < 3; ++i) dT3l[i] = 0.5 * h * dk2l[i];
  matmul(M2, dT3T, tmp, 3, 3, 3);
  for (int i = 0; i < 9; ++i) dk3T[i] = kKappa * lam * tmp[i];
  cross(T3, B2, c3);
  matmul(M2, dT3l, tmp, 3, 3, 1);
  for (int i = 0; i < 3; ++i) dk3l[i] = kKappa * c3[i] + kKappa * lam * tmp[i];
  for (int i = 0; i < 9; ++i) dT4T[i] = I3[i] + h * dk3T[i];
  for (int i = 0; i < 3; ++i) dT4l[i] = h * dk3l[i];
  matmul(M4, dT4T, tmp, 3, 3, 3);
  for (int i = 0; i < 9; ++i) dk4T[i] = kKappa * lam * tmp[i];
  cross(T4, B4, c4);
  matmul(M4, dT4l, tmp, 3, 3, 1);
  for (int i = 0; i < 3; ++i) dk4l[i] = kKappa * c4[i] + kKappa * lam * tmp[i];

  // D = [[I, dr'/dT, dr'/dlam], [0, dT'/dT, dT'/dlam], [0, 0, 1]]
  for (int i = 0; i < 49; ++i) out.D[i] = 0.0;
  for (int i = 0; i < 3; ++i) {
    out.D[i * 7 + i] = 1.0;
    for (int j = 0; j < 3; ++j) {
      double id = (i == j) ? 1.0 : 0.0;
      out.D[i * 7 + 3 + j] = h * id + h * h / 6.0 * (dk1T[i * 3 + j] + dk2T[i * 3 + j] + dk3T[i * 3 + j]);
      out.D[(3 + i) * 7 + 3 + j] =
          id + h / 6.0 * (dk1T[i * 3 + j] + 2.0 * dk2T[i * 3 + j] + 2.0 * dk3T[i * 3 + j] + dk4T[i * 3 + j]);
    }
    out.D[i * 7 + 6] = h * h / 6.0 * (dk1l[i] + dk2l[i] + dk3l[i]);
    out.D[(3 + i) * 7 + 6] = h / 6.0 * (dk1l[i] + 2.0 * dk2l[i] + 2.0 * dk3l[i] + dk4l[i]);
  }
  out.D[6 * 7 + 6] = 1.0;
}

// ---------------------------------------------------------------- propagation to a plane
// Adaptive RKN stepping from (r, T, lam) to the plane of surface s.
// Reading (step control, after Lund 2009a, with the usual safety factor 0.9): a step with
// eps > tol is rejected and h_ctrl becomes |h| * clamp(0.9 (tol/eps)^(1/4), 1/4, 4); an accepted
// step that was limited by h_ctrl sets h_ctrl = min(h_max, h_ctrl * clamp(0.9 (tol/eps)^(1/4), 1/4, 4)).
// Reading (surface targeting): each step aims at the plane's intersection with the parabola
// r + s T + s^2/2 k1 (k1 = dT/ds at the start point): s = 2 d / (a + sign(a) sqrt(a^2 + 2 b d)),
// d = n.(c - r), a = n.T, b = n.k1 (the straight-line d / a when a^2 + 2 b d < 0); the step is s if
// |s| < h_ctrl, else h_ctrl with the sign of s. Propagation stops when |n.(r - c)| <= surf_tol,
// closing the rest with a Taylor step. Reading: a plane more than 1 mm behind the start point
// (straight-line path d / a < -1 mm, or not finite) is a miss; overlapping modules can be crossed
// within a fraction of a millimetre, and the update may then leave the next plane just behind.
struct PropState {
  double h_ctrl;
  uint32_t attempts;  // all step attempts, this track
  uint32_t rejected;  // rejected attempts, this track
  double h_last;      // last accepted step length (an MLP input)
  bool use_mlp;       // unused by the oracle's propagation (the proposal is made per track)
  std::vector<float>* records = nullptr;  // training records (12 inputs, label), when not null
};

// MLP inputs at the start of a step, FP32: position (u, v, n components of r - c) / 1000 mm,
// direction (u, v, n components of T), q/p, B / 2 T, ln(last step / mm) / 5, and the
// straight-line path to the plane / 1000 mm clamped to [-2, 2].
void mlp_features(const Surface& s, const double r[3], const double T[3], double lam, const double B[3],
                  double h_last, double sl, float x[12]) {
  float d[3], t[3], u[3], v[3], n[3];
  for (int i = 0; i < 3; ++i) {
    d[i] = float(r[i] - s.c[i]);
    t[i] = float(T[i]);
    u[i] = float(s.u[i]);
    v[i] = float(s.v[i]);
    n[i] = float(s.n[i]);
  }
  x[0] = (u[0] * d[0] + u[1] * d[1] + u[2] * d[2]) * 1e-3f;
  x[1] = (v[0] * d[0] + v[1] * d[1] + v[2] * d[2]) * 1e-3f;
  x[2] = (n[0] * d[0] + n[1] * d[1] + n[2] * d[2]) * 1e-3f;
  x[3] = u[0] * t[0] + u[1] * t[1] + u[2] * t[2];
  x[4] = v[0] * t[0] + v[1] * t[1] + v[2] * t[2];
  x[5] = n[0] * t[0] + n[1] * t[1] + n[2] * t[2];
  x[6] = float(lam);
  x[7] = float(B[0]) * 0.5f;
  x[8] = float(B[1]) * 0.5f;
  x[9] = float(B[2]) * 0.5f;
  x[10] = std::log(float(h_last)) * 0.2f;
  float q = float(sl) * 1e-3f;
  x[11] = q < -2.0f ? -2.0f : (q > 2.0f ? 2.0f : q);
}

float silu(float z) { return z / (1.0f + std::exp(-z)); }

// BF16 rounding of an FP32 value (nearest, ties to even), returned as FP32.
float bf16_round(float x) {
  uint32_t u;
  std::memcpy(&u, &x, 4);
  u = (u + 0x7FFFu + ((u >> 16) & 1u)) & 0xFFFF0000u;
  float y;
  std::memcpy(&y, &u, 4);
  return y;
}

// The network's output is ln(h / mm) of the largest step within tolerance. Reading of "BF16
// weights, FP32 accumulate, dense layers on tensor cores": the operands of both dense layers
// are BF16 (the inputs and the first hidden layer's activations are rounded to BF16), each
// layer's products are exact and summed in FP32 (here: summed exactly, rounded once), and the
// bias is added in FP32; the 64 -> 1 output layer is FP32. Reading (proposal): the output is
// rounded to a 1/32 grid of ln h, and the proposal is 0.9 exp(k / 32), clamped to
// [h_min, h_max]; non-finite inputs propose h_max.
double mlp_propose(const Mlp& m, const float x[12], double h_min, double h_max) {
  float xb[12];
  for (int i = 0; i < 12; ++i) {
    if (!std::isfinite(x[i])) return h_max;
    xb[i] = bf16_round(x[i]);
  }
  float a1[64], a2[64];
  for (int j = 0; j < 64; ++j) {
    double acc = 0.0;
    for (int i = 0; i < 12; ++i) acc += double(m.W1[j][i]) * double(xb[i]);
    a1[j] = bf16_round(silu(float(acc) + m.b1[j]));
  }
  for (int j = 0; j < 64; ++j) {
    double acc = 0.0;
    for (int i = 0; i < 64; ++i) acc += double(m.W2[j][i]) * double(a1[i]);
    a2[j] = silu(float(acc) + m.b2[j]);
  }
  float out = m.b3;
  for (int i = 0; i < 64; ++i) out += m.w3[i] * a2[i];
  const float q = 0.9f * std::exp(std::nearbyint(out * 32.0f) / 32.0f);
  if (!std::isfinite(q)) return h_max;
  double h = q;
  if (h < h_min) h = h_min;
  if (h > h_max) h = h_max;
  return h;
}

void bound_to_free(const Surface& s, const double p[5], double r[3], double T[3]);

// Learned mode: the starting step-size control of a track, proposed from the seed state at the
// first surface s0, toward the second surface s1.
double propose_start(const Surface& s0, const Surface& s1, const Field& f, const Opts& o, const double* seed_par) {
  double r[3], T[3], B[3], diff[3];
  bound_to_free(s0, seed_par, r, T);
  bool oofm = false;
  field_at(f, r, B, &oofm);
  for (int i = 0; i < 3; ++i) diff[i] = s1.c[i] - r[i];
  float x[12];
  mlp_features(s1, r, T, seed_par[4], B, o.h_max, dot3(s1.n, diff) / dot3(s1.n, T), x);
  return mlp_propose(*o.mlp, x, o.h_min, o.h_max);
}

double step_factor(double q, double lo, double hi) {
  // clamp(0.9 q^(1/4), lo, hi) with q^(1/4) taken as sqrt(sqrt(q)).
  double f = 0.9 * std::sqrt(std::sqrt(q));
  if (f < lo) f = lo;
  if (f > hi) f = hi;
  return f;
}

uint32_t propagate(const Field& f, const Opts& o, const Surface& s, double r[3], double T[3], double lam,
                   double Dtot[49], double dxds[7], PropState& ps) {
  uint32_t status = 0;
  for (int i = 0; i < 49; ++i) Dtot[i] = (i % 8 == 0) ? 1.0 : 0.0;
  bool first = true;
  uint32_t n_here = 0;

  for (;;) {
    double diff[3] = {s.c[0] - r[0], s.c[1] - r[1], s.c[2] - r[2]};
    double dist = dot3(s.n, diff);
    if (std::fabs(dist) <= o.surf_tol) {
      // Reading: the remaining distance (at most surf_tol) is closed by a second-order Taylor
      // step of length s onto the plane: r += s T + s^2/2 k, T += s k (k = dT/ds here), whose
      // 7x7 derivative joins the transport (error O(kappa^2 s^2), below 1e-12 at s = 0.01 mm).
      double B[3], c[3], k[3];
      bool oofs = false;
      field_at(f, r, B, &oofs);
      if (oofs) status |= kOutOfField;
      cross(T, B, c);
      for (int i = 0; i < 3; ++i) k[i] = kKappa * lam * c[i];
      double a = dot3(s.n, T), b = dot3(s.n, k);
      double sp = dist / a, disc = a * a + 2.0 * b * dist;
      if (disc >= 0.0) {
        double q = 2.0 * dist / (a + std::copysign(std::sqrt(disc), a));
        if (std::isfinite(q)) sp = q;
      }
      double M[9], D[49];
      cross_matrix(B, M);
      for (int i = 0; i < 49; ++i) D[i] = (i % 8 == 0) ? 1.0 : 0.0;
      for (int i = 0; i < 3; ++i) {
        for (int j = 0; j < 3; ++j) {
          double id = (i == j) ? 1.0 : 0.0;
          D[i * 7 + 3 + j] = sp * id + 0.5 * sp * sp * kKappa * lam * M[i * 3 + j];
          D[(3 + i) * 7 + 3 + j] = id + sp * kKappa * lam * M[i * 3 + j];
        }
        D[i * 7 + 6] = 0.5 * sp * sp * kKappa * c[i];
        D[(3 + i) * 7 + 6] = sp * kKappa * c[i];
      }
      for (int i = 0; i < 3; ++i) {
        r[i] += sp * T[i] + 0.5 * sp * sp * k[i];
        T[i] += sp * k[i];
      }
      matmul(D, Dtot, Dtot, 7, 7, 7);
      break;
    }
    double a = dot3(s.n, T);
    double sl = dist / a;
    if (first && !(sl > -1.0 && std::isfinite(sl))) return status | kSurfaceMissed;
    first = false;
    if (n_here >= o.max_steps) return status | kMaxSteps;
    ++n_here;
    ++ps.attempts;
    double B0[3], c0[3], k1[3];
    bool oof0 = false;
    field_at(f, r, B0, &oof0);
    cross(T, B0, c0);
    for (int i = 0; i < 3; ++i) k1[i] = kKappa * lam * c0[i];
    double b = dot3(s.n, k1);
    double disc = a * a + 2.0 * b * dist;
    double sp = sl;
    if (disc >= 0.0) {
      sp = 2.0 * dist / (a + std::copysign(std::sqrt(disc), a));
      if (!std::isfinite(sp)) sp = sl;
    }
    double limit = ps.h_ctrl;
    bool limited = !(std::fabs(sp) < limit);
    double h = limited ? std::copysign(limit, sp) : sp;
    float feat[12];
    if (ps.records) mlp_features(s, r, T, lam, B0, ps.h_last, sl, feat);
    Step st;
    bool oof = false;
    rkn_step(f, r, T, lam, h, st, &oof);
    if (st.eps > o.tol) {
      ++ps.rejected;
      ps.h_ctrl = std::fabs(h) * step_factor(o.tol / st.eps, 0.25, 4.0);
      if (ps.h_ctrl < o.h_min) return status | kStepUnderflow;
      continue;
    }
    if (oof) status |= kOutOfField;
    for (int i = 0; i < 3; ++i) {
      r[i] = st.r[i];
      T[i] = st.T[i];
    }
    matmul(st.D, Dtot, Dtot, 7, 7, 7);
    // Training record (learned step proposer): an accepted step that the control limited gives
    // the inputs at its start and the label ln(|h| (tol/eps)^(1/4)), the largest step within
    // tolerance at this step's error constant.
    if (ps.records && limited && st.eps > 0.0) {
      ps.records->insert(ps.records->end(), feat, feat + 12);
      ps.records->push_back(float(std::log(std::fabs(h) * std::sqrt(std::sqrt(o.tol / st.eps)))));
    }
    if (limited) {
      double fac = (st.eps > 0.0) ? step_factor(o.tol / st.eps, 0.25, 4.0) : 4.0;
      ps.h_ctrl = std::min(o.h_max, std::fabs(h) * fac);
    }
    ps.h_last = std::fabs(h);
  }
  // dx/ds at the end point: (T, kappa*lam*T x B(r), 0).
  double B[3], c[3];
  bool oof = false;
  field_at(f, r, B, &oof);
  if (oof) status |= kOutOfField;
  cross(T, B, c);
  for (int i = 0; i < 3; ++i) {
    dxds[i] = T[i];
    dxds[3 + i] = kKappa * lam * c[i];
  }
  dxds[6] = 0.0;
  return status;
}

// ---------------------------------------------------------------- parametrisation
// Bound parameters on a plane: (l0, l1, phi, theta, q/p), with (l0, l1) = (u.(r-c), v.(r-c)),
// T = (sin th cos ph, sin th sin ph, cos th). Free parameters: (r, T, q/p).
void bound_to_free(const Surface& s, const double p[5], double r[3], double T[3]) {
  for (int i = 0; i < 3; ++i) r[i] = s.c[i] + p[0] * s.u[i] + p[1] * s.v[i];
  T[0] = std::sin(p[3]) * std::cos(p[2]);
  T[1] = std::sin(p[3]) * std::sin(p[2]);
  T[2] = std::cos(p[3]);
}

// Reading: T is renormalised only here, when converting to bound parameters.
void free_to_bound(const Surface& s, const double r[3], const double T[3], double lam, double p[5]) {
  double d[3] = {r[0] - s.c[0], r[1] - s.c[1], r[2] - s.c[2]};
  double nT = std::sqrt(dot3(T, T));
  double t[3] = {T[0] / nT, T[1] / nT, T[2] / nT};
  p[0] = dot3(s.u, d);
  p[1] = dot3(s.v, d);
  p[2] = std::atan2(t[1], t[0]);
  p[3] = std::acos(t[2]);
  p[4] = lam;
}

// d(free)/d(bound), 7x5.
void jac_bound_to_free(const Surface& s, const double p[5], double J[35]) {
  for (int i = 0; i < 35; ++i) J[i] = 0.0;
  double sp = std::sin(p[2]), cp = std::cos(p[2]), st = std::sin(p[3]), ct = std::cos(p[3]);
  for (int i = 0; i < 3; ++i) {
    J[i * 5 + 0] = s.u[i];
    J[i * 5 + 1] = s.v[i];
  }
  J[3 * 5 + 2] = -st * sp;
  J[4 * 5 + 2] = st * cp;
  J[5 * 5 + 2] = 0.0;
  J[3 * 5 + 3] = ct * cp;
  J[4 * 5 + 3] = ct * sp;
  J[5 * 5 + 3] = -st;
  J[6 * 5 + 4] = 1.0;
}

// d(bound)/d(free), 5x7, at the target plane (angles from the normalised direction).
// The angle rows are the tangent-space gradients of phi and theta.
void jac_free_to_bound(const Surface& s, const double T[3], double J[35]) {
  for (int i = 0; i < 35; ++i) J[i] = 0.0;
  double nT = std::sqrt(dot3(T, T));
  double t[3] = {T[0] / nT, T[1] / nT, T[2] / nT};
  double phi = std::atan2(t[1], t[0]), th = std::acos(t[2]);
  double sp = std::sin(phi), cp = std::cos(phi), st = std::sin(th), ct = std::cos(th);
  for (int i = 0; i < 3; ++i) {
    J[0 * 7 + i] = s.u[i];
    J[1 * 7 + i] = s.v[i];
  }
  J[2 * 7 + 3] = -sp / st;
  J[2 * 7 + 4] = cp / st;
  J[3 * 7 + 3] = ct * cp;
  J[3 * 7 + 4] = ct * sp;
  J[3 * 7 + 5] = -st;
  J[4 * 7 + 6] = 1.0;
}

// Path correction at the plane: the free state moves along dx/ds by
// ds = -n.dr / n.T when the intersection shifts, so P = I - dxds (n,0,0)^T / (n.T).
void path_correction(const Surface& s, const double T[3], const double dxds[7], double P[49]) {
  double nT = dot3(s.n, T);
  for (int i = 0; i < 7; ++i)
    for (int j = 0; j < 7; ++j) {
      double nj = (j < 3) ? s.n[j] : 0.0;
      P[i * 7 + j] = ((i == j) ? 1.0 : 0.0) - dxds[i] * nj / nT;
    }
}

// ---------------------------------------------------------------- material
// Highland (PDG) r.m.s. plane scattering angle for a path x in a layer of radiation
// length X0: theta0 = 13.6 MeV / (beta c p) * sqrt(x/X0) * (1 + 0.038 ln(x / (X0 beta^2))).
double highland(double p, double beta, double x, double X0) {
  return 0.0136 / (beta * p) * std::sqrt(x / X0) * (1.0 + 0.038 * std::log(x / (X0 * beta * beta)));
}

// Mean energy loss rate (Bethe, PDG) in MeV cm^2 / g for a unit-charge particle of mass m.
// Reading: density effect delta/2 = max(0, ln(hbar omega_p / I) + ln(beta gamma) - 1/2),
// the high-energy asymptote; no shell correction.
double bethe(double p, double m, const Opts& o) {
  double E = std::sqrt(p * p + m * m);
  double beta2 = (p * p) / (E * E);
  double gamma = E / m;
  double bg2 = (p / m) * (p / m);
  double me_m = kMe / m;
  double wmax = 2.0 * kMe * bg2 / (1.0 + 2.0 * gamma * me_m + me_m * me_m);  // GeV
  double I = o.I_eV * 1e-9;                                                   // GeV
  double half_delta = std::log(o.hwp_eV / o.I_eV) + 0.5 * std::log(bg2) - 0.5;
  if (half_delta < 0.0) half_delta = 0.0;
  return kBetheK * o.ZA / beta2 * (0.5 * std::log(2.0 * kMe * bg2 * wmax / (I * I)) - beta2 - half_delta);
}

// Thin-layer material at surface s, applied to the filtered state after the update.
// Adds theta0^2 / sin^2(theta) to Var(phi) and theta0^2 to Var(theta) (Q, full 5x5), and
// lowers |p| by the mean energy loss. Reading: no energy-loss variance; the material
// Jacobian is the identity. With `gain` (the backward filter's reversed particle, which crosses
// the layer against the flight direction) |p| rises by the mean loss instead. Reading: theta0
// and the loss are then evaluated at the reversed particle's momentum on arrival (the momentum
// after the crossing in the flight direction), which differs from the forward evaluation at
// second order in the loss.
uint32_t material(const Surface& s, const Opts& o, double p[5], double Q[25], bool gain = false) {
  for (int i = 0; i < 25; ++i) Q[i] = 0.0;
  if (!(s.t > 0.0)) return 0;
  double r[3], T[3];
  bound_to_free(s, p, r, T);
  double x = s.t / std::fabs(dot3(s.n, T));
  double mom = 1.0 / std::fabs(p[4]);
  double E = std::sqrt(mom * mom + o.mass * o.mass);
  double beta = mom / E;
  double th0 = highland(mom, beta, x, s.X0);
  double sth = std::sin(p[3]);
  Q[2 * 5 + 2] = th0 * th0 / (sth * sth);
  Q[3 * 5 + 3] = th0 * th0;
  double dE = bethe(mom, o.mass, o) * o.rho * (x * 0.1) * 1e-3;  // GeV
  double E2 = gain ? E + dE : E - dE;
  if (!(E2 > o.mass)) return kParticleStopped;
  double mom2 = std::sqrt(E2 * E2 - o.mass * o.mass);
  p[4] = std::copysign(1.0 / mom2, p[4]);
  return 0;
}

// ---------------------------------------------------------------- Kalman update
// Gain-matrix update with H = [I2 0]: S = V + H C H^T, K = C H^T S^-1, p' = p + K r,
// C' = (I - K H) C (I - K H)^T + K V K^T (Joseph form), chi2 = r^T S^-1 r with the
// predicted residual r = m - H p.
uint32_t kf_update(const double m[2], const double V[4], double p[5], double C[25], double* chi2) {
  double H[10] = {1, 0, 0, 0, 0, 0, 1, 0, 0, 0};
  double Ht[10];
  transpose(H, Ht, 2, 5);
  double HC[10], S[4], CHt[10];
  matmul(H, C, HC, 2, 5, 5);
  matmul(HC, Ht, S, 2, 5, 2);
  for (int i = 0; i < 4; ++i) S[i] += V[i];
  double det = S[0] * S[3] - S[1] * S[2];
  if (!(S[0] > 0.0 && det > 0.0)) return kUpdateNotSpd;
  double Si[4] = {S[3] / det, -S[1] / det, -S[2] / det, S[0] / det};
  matmul(C, Ht, CHt, 5, 5, 2);
  double K[10];
  matmul(CHt, Si, K, 5, 2, 2);
  double Hp[2];
  matmul(H, p, Hp, 2, 5, 1);
  double res[2] = {m[0] - Hp[0], m[1] - Hp[1]};
  double Kr[5];
  matmul(K, res, Kr, 5, 2, 1);
  for (int i = 0; i < 5; ++i) p[i] += Kr[i];
  double Sr[2];
  matmul(Si, res, Sr, 2, 2, 1);
  *chi2 = res[0] * Sr[0] + res[1] * Sr[1];
  double IKH[25], KH[25];
  matmul(K, H, KH, 5, 2, 5);
  for (int i = 0; i < 25; ++i) IKH[i] = ((i % 6) == 0 ? 1.0 : 0.0) - KH[i];
  double IKHt[25], A[25], B[25], Kt[10], KV[10], KVKt[25];
  transpose(IKH, IKHt, 5, 5);
  matmul(IKH, C, A, 5, 5, 5);
  matmul(A, IKHt, B, 5, 5, 5);
  transpose(K, Kt, 5, 2);
  matmul(K, V, KV, 5, 2, 2);
  matmul(KV, Kt, KVKt, 5, 2, 5);
  for (int i = 0; i < 25; ++i) C[i] = B[i] + KVKt[i];
  symmetrize(C, 5);
  return 0;
}

// ---------------------------------------------------------------- RTS smoother
// Backward pass k = N-2 .. 0 over stored filtered (pf, Cf) and predicted (pp, Cp) states
// and transport Jacobians J[k+1] (k -> k+1):
//   A_k = Cf_k J_{k+1}^T Cp_{k+1}^-1,
//   ps_k = pf_k + A_k (ps_{k+1} - pp_{k+1}),
//   Cs_k = Cf_k + A_k (Cs_{k+1} - Cp_{k+1}) A_k^T   (symmetrised).
// The phi component of a parameter difference is wrapped to (-pi, pi].
uint32_t rts(int N, const double* pf, const double* Cf, const double* pp, const double* Cp, const double* J,
             double* ps, double* Cs) {
  std::memcpy(ps + (N - 1) * 5, pf + (N - 1) * 5, sizeof(double) * 5);
  std::memcpy(Cs + (N - 1) * 25, Cf + (N - 1) * 25, sizeof(double) * 25);
  for (int k = N - 2; k >= 0; --k) {
    double Cpi[25], Jt[25], A[25], At[25], tmp[25], dC[25], dCs[25];
    if (!spd_inverse(Cp + (k + 1) * 25, Cpi, 5)) return kSmootherNotSpd;
    transpose(J + (k + 1) * 25, Jt, 5, 5);
    matmul(Cf + k * 25, Jt, tmp, 5, 5, 5);
    matmul(tmp, Cpi, A, 5, 5, 5);
    double dp[5], Adp[5];
    for (int i = 0; i < 5; ++i) dp[i] = ps[(k + 1) * 5 + i] - pp[(k + 1) * 5 + i];
    dp[2] = wrap_phi(dp[2]);
    matmul(A, dp, Adp, 5, 5, 1);
    for (int i = 0; i < 5; ++i) ps[k * 5 + i] = pf[k * 5 + i] + Adp[i];
    ps[k * 5 + 2] = wrap_phi(ps[k * 5 + 2]);
    for (int i = 0; i < 25; ++i) dC[i] = Cs[(k + 1) * 25 + i] - Cp[(k + 1) * 25 + i];
    transpose(A, At, 5, 5);
    matmul(A, dC, tmp, 5, 5, 5);
    matmul(tmp, At, dCs, 5, 5, 5);
    for (int i = 0; i < 25; ++i) Cs[k * 25 + i] = Cf[k * 25 + i] + dCs[i];
    symmetrize(Cs + k * 25, 5);
  }
  return 0;
}

// ---------------------------------------------------------------- one track
void unpack_cov(const double* packed, double C[25]) {
  int idx = 0;
  for (int i = 0; i < 5; ++i)
    for (int j = i; j < 5; ++j) {
      C[i * 5 + j] = packed[idx];
      C[j * 5 + i] = packed[idx];
      ++idx;
    }
}

void pack_cov(const double C[25], double* packed) {
  int idx = 0;
  for (int i = 0; i < 5; ++i)
    for (int j = i; j < 5; ++j) packed[idx++] = C[i * 5 + j];
}

struct TrackIn {
  uint32_t N;
  const double* meas;  // [N][5]: loc0, loc1, V00, V01, V11
  const uint32_t* sid;
  const double* seed_par;  // [5]
  const double* seed_cov;  // [15]
};

struct TrackOut {
  double par[5], cov[15], chi2;
  double cov_filt0[15];  // filtered covariance at the first surface
  int32_t ndf;
  uint32_t status;
  uint32_t attempts, rejected;
};

void fill_nan(TrackOut& out) {
  double nan = std::nan("");
  for (int i = 0; i < 5; ++i) out.par[i] = nan;
  for (int i = 0; i < 15; ++i) out.cov[i] = nan;
  out.chi2 = nan;
}

bool all_finite(const double* a, int n) {
  for (int i = 0; i < n; ++i)
    if (!std::isfinite(a[i])) return false;
  return true;
}

struct States {
  std::vector<double> pp, Cp, pf, Cf, J, ps, Cs;
};

// ---------------------------------------------------------------- two-filter smoother
// Reading of the optimal smoother (Sec. 4 ¶2: the smoothed parameters are the weighted mean of
// a forward and a backward filter; Fraser-Potter form). For the first-surface result:
//  * the forward filter runs as for RTS and gives the track's chi2;
//  * the backward filter is a Kalman filter of the reversed particle (l0, l1, phi + pi,
//    pi - theta, -q/p) -- the same trajectory traversed against the flight direction, so that
//    the ordinary propagation applies -- over the entries from the last to the first. It starts
//    from the forward filter's state at the last entry with that covariance times `inflation`
//    (it then carries 1/inflation of the forward information) and updates with every
//    measurement, the last one included. Before each earlier entry it propagates to it and then
//    applies that surface's material (scattering variance; the mean loss given back), because
//    the state on a surface is the one before its material in the flight direction;
//  * the result is the weighted mean, at the first surface, of the backward filtered state
//    (every measurement) and the seed (the prior there):
//    K = C_b (C_b + C_0)^-1, p = p_b + K (p_0 - p_b), C = (I - K) C_b.
// The reversal maps (phi, theta, q/p) to (phi + pi, pi - theta, -q/p): its Jacobian is
// diag(1, 1, 1, -1, -1), applied to the covariance on both sides.
void reverse_state(double p[5], double C[25]) {
  p[2] = wrap_phi(p[2] + kPi);
  p[3] = kPi - p[3];
  p[4] = -p[4];
  const double sgn[5] = {1, 1, 1, -1, -1};
  for (int r = 0; r < 5; ++r)
    for (int c = 0; c < 5; ++c) C[r * 5 + c] *= sgn[r] * sgn[c];
}

// Backward filter over entries N-1 .. 0 from (p_last, C_last), the forward filtered state at
// the last entry. On return (pb, Cb) is the backward filtered state at the first entry in the
// flight direction's parameters.
uint32_t backward_filter(const Surface* surf, const Field& f, const Opts& o, const TrackIn& in,
                         const double* p_last, const double* C_last, PropState& prop, double pb[5], double Cb[25]) {
  const int N = int(in.N);
  std::memcpy(pb, p_last, sizeof(double) * 5);
  for (int i = 0; i < 25; ++i) Cb[i] = C_last[i] * o.inflation;
  reverse_state(pb, Cb);
  uint32_t status = 0;
  for (int k = N - 1; k >= 0; --k) {
    const Surface& sk = surf[surface_of(in.sid[k])];
    if (k < N - 1) {
      const Surface& snext = surf[surface_of(in.sid[k + 1])];
      double r[3], T[3], Dtot[49], dxds[7], Jb2f[35], Jf2b[35], P[49], tmp[49], t75[35], J[25], Jt[25], t55[25];
      bound_to_free(snext, pb, r, T);
      jac_bound_to_free(snext, pb, Jb2f);
      status |= propagate(f, o, sk, r, T, pb[4], Dtot, dxds, prop);
      if (status & kFatal) return status;
      jac_free_to_bound(sk, T, Jf2b);
      path_correction(sk, T, dxds, P);
      matmul(P, Dtot, tmp, 7, 7, 7);
      matmul(tmp, Jb2f, t75, 7, 7, 5);
      matmul(Jf2b, t75, J, 5, 7, 5);
      const double lam = pb[4];
      free_to_bound(sk, r, T, lam, pb);
      transpose(J, Jt, 5, 5);
      matmul(J, Cb, t55, 5, 5, 5);
      matmul(t55, Jt, Cb, 5, 5, 5);
      double Q[25];
      status |= material(sk, o, pb, Q, true);
      if (status & kFatal) return status;
      for (int i = 0; i < 25; ++i) Cb[i] += Q[i];
      symmetrize(Cb, 5);
    }
    if (measured(in.sid[k])) {
      const double* mk = in.meas + 5 * k;
      double m[2] = {mk[0], mk[1]};
      double V[4] = {mk[2], mk[3], mk[3], mk[4]};
      double c2 = 0.0;
      status |= kf_update(m, V, pb, Cb, &c2);
      if (status & kFatal) return status;
    }
    pb[2] = wrap_phi(pb[2]);
    if (!(pb[3] > 0.0 && pb[3] < kPi)) return status | kNonFinite;
  }
  reverse_state(pb, Cb);
  return status;
}

// Weighted mean of two estimates of the same parameters: (p0, C0) and (pb, Cb).
uint32_t weighted_mean(const double p0[5], const double C0[25], const double pb[5], const double Cb[25], double ps[5],
                       double Cs[25]) {
  double S[25], Si[25], K[25], KCb[25];
  for (int i = 0; i < 25; ++i) S[i] = Cb[i] + C0[i];
  if (!spd_inverse(S, Si, 5)) return kSmootherNotSpd;
  matmul(Cb, Si, K, 5, 5, 5);
  double d[5], Kd[5];
  for (int i = 0; i < 5; ++i) d[i] = p0[i] - pb[i];
  d[2] = wrap_phi(d[2]);
  matmul(K, d, Kd, 5, 5, 1);
  for (int i = 0; i < 5; ++i) ps[i] = pb[i] + Kd[i];
  ps[2] = wrap_phi(ps[2]);
  matmul(K, Cb, KCb, 5, 5, 5);
  for (int i = 0; i < 25; ++i) Cs[i] = Cb[i] - KCb[i];
  symmetrize(Cs, 5);
  return 0;
}

void fit_track(const Surface* surf, uint32_t n_surf, const Field& f, const Opts& o, const TrackIn& in,
               TrackOut& out, States* keep = nullptr) {
  const int N = int(in.N);
  out.status = 0;
  out.attempts = out.rejected = 0;
  out.ndf = 0;
  for (int i = 0; i < 15; ++i) out.cov_filt0[i] = std::nan("");
  int M = 0;  // entries with a measurement
  bool bad = false;
  for (int k = 0; k < N; ++k) {
    bad = bad || surface_of(in.sid[k]) >= n_surf;
    M += measured(in.sid[k]) ? 1 : 0;
  }
  out.ndf = 2 * M;
  if (bad) {
    fill_nan(out);
    out.status = kBadInput;
    return;
  }
  if (M == 0) {  // nothing to fit: the seed is the result
    std::memcpy(out.par, in.seed_par, sizeof(double) * 5);
    std::memcpy(out.cov, in.seed_cov, sizeof(double) * 15);
    out.chi2 = 0.0;
    out.status = kTooFewHits;
    return;
  }
  if (!all_finite(in.seed_par, 5) || !all_finite(in.seed_cov, 15)) {
    fill_nan(out);
    out.status = kNonFinite;
    return;
  }
  std::vector<double> pp(N * 5), Cp(N * 25), pf(N * 5), Cf(N * 25), J(N * 25, 0.0), ps(N * 5), Cs(N * 25);
  std::memcpy(&pp[0], in.seed_par, sizeof(double) * 5);
  unpack_cov(in.seed_cov, &Cp[0]);
  PropState prop{o.h_max, 0, 0, o.h_max, true, o.records};
  if (o.mlp && N >= 2) {
    // Reading (learned mode): the step-size control has no error estimate before the first step,
    // so the network proposes its starting value (instead of h_max) from the seed state at the
    // first surface, toward the second surface; from then on the plain control adapts it from
    // the error estimates, and the error estimate judges every step.
    prop.h_ctrl = propose_start(surf[surface_of(in.sid[0])], surf[surface_of(in.sid[1])], f, o, in.seed_par);
  }
  double chi2 = 0.0;
  uint32_t status = 0;
  for (int k = 0; k < N; ++k) {
    const Surface& sk = surf[surface_of(in.sid[k])];
    if (k > 0) {
      const Surface& sprev = surf[surface_of(in.sid[k - 1])];
      double pm[5], Q[25];
      std::memcpy(pm, &pf[(k - 1) * 5], sizeof(pm));
      status |= material(sprev, o, pm, Q);
      if (status & kFatal) break;
      double r[3], T[3], Dtot[49], dxds[7], Jb2f[35], Jf2b[35], P[49], tmp[49], t75[35], t55[25];
      bound_to_free(sprev, pm, r, T);
      jac_bound_to_free(sprev, pm, Jb2f);
      status |= propagate(f, o, sk, r, T, pm[4], Dtot, dxds, prop);
      if (status & kFatal) break;
      jac_free_to_bound(sk, T, Jf2b);
      path_correction(sk, T, dxds, P);
      matmul(P, Dtot, tmp, 7, 7, 7);
      matmul(tmp, Jb2f, t75, 7, 7, 5);
      matmul(Jf2b, t75, &J[k * 25], 5, 7, 5);
      free_to_bound(sk, r, T, pm[4], &pp[k * 5]);
      double CQ[25], Jt[25];
      for (int i = 0; i < 25; ++i) CQ[i] = Cf[(k - 1) * 25 + i] + Q[i];
      transpose(&J[k * 25], Jt, 5, 5);
      matmul(&J[k * 25], CQ, t55, 5, 5, 5);
      matmul(t55, Jt, &Cp[k * 25], 5, 5, 5);
      symmetrize(&Cp[k * 25], 5);
    }
    std::memcpy(&pf[k * 5], &pp[k * 5], sizeof(double) * 5);
    std::memcpy(&Cf[k * 25], &Cp[k * 25], sizeof(double) * 25);
    if (measured(in.sid[k])) {  // else the filtered state is the predicted one
      const double* mk = in.meas + 5 * k;
      double m[2] = {mk[0], mk[1]};
      double V[4] = {mk[2], mk[3], mk[3], mk[4]};
      double c2 = 0.0;
      status |= kf_update(m, V, &pf[k * 5], &Cf[k * 25], &c2);
      if (status & kFatal) break;
      chi2 += c2;
    }
    if (k == 0) pack_cov(&Cf[0], out.cov_filt0);
    pf[k * 5 + 2] = wrap_phi(pf[k * 5 + 2]);
    if (!(pf[k * 5 + 3] > 0.0 && pf[k * 5 + 3] < kPi)) {
      status |= kNonFinite;
      break;
    }
  }
  if (o.smoother == 1 && !(status & kFatal)) {
    double pb[5], Cb[25], C0[25];
    status |= backward_filter(surf, f, o, in, &pf[(N - 1) * 5], &Cf[(N - 1) * 25], prop, pb, Cb);
    unpack_cov(in.seed_cov, C0);
    if (!(status & kFatal)) status |= weighted_mean(in.seed_par, C0, pb, Cb, &ps[0], &Cs[0]);
  }
  out.attempts = prop.attempts;
  out.rejected = prop.rejected;
  if (o.smoother == 0 && !(status & kFatal))
    status |= rts(N, &pf[0], &Cf[0], &pp[0], &Cp[0], &J[0], &ps[0], &Cs[0]);
  if (!(status & kFatal)) {
    double L[25];
    if (!cholesky(&Cs[0], L, 5)) status |= kSmootherNotSpd;
  }
  if (!(status & kFatal)) {
    std::memcpy(out.par, &ps[0], sizeof(double) * 5);
    pack_cov(&Cs[0], out.cov);
    out.chi2 = chi2;
    if (!all_finite(out.par, 5) || !all_finite(out.cov, 15) || !std::isfinite(chi2)) status |= kNonFinite;
  }
  if (status & kFatal) fill_nan(out);
  if (M < 3) status |= kTooFewHits;
  out.status = status;
  if (keep) {
    keep->pp = pp; keep->Cp = Cp; keep->pf = pf; keep->Cf = Cf; keep->J = J; keep->ps = ps; keep->Cs = Cs;
  }
}


// ---------------------------------------------------------------- track finding (CKF)
// Reading (Sec. 2, track finding; the paper describes the combinatorial Kalman filter as the
// step that follows seeding and precedes fitting, and prints no algorithm): starting from a
// seed (parameters and covariance on a sensitive surface), the filter navigates outward from
// surface to surface; on every sensitive surface it crosses, each measurement whose predicted
// chi2 passes a gate makes a branch (the best `kChildren` of them), and so does the
// "no measurement here" hypothesis (a hole) while the branch has fewer than max_holes
// consecutive holes. A beam of at most `beam` branches is kept after every step, ranked by
// measurement count (more first), then consecutive holes (fewer first), then chi2 (lower
// first), then the order the branches were made in. A branch ends when no surface lies ahead,
// when it would exceed its holes, or when it has max_entries entries; the best ended branch (same
// ranking) is the track candidate.
//
// Navigation (reading of the paper's navigator for a detector of layers): the modules are
// planar and tile barrel cylinders and endcap disks. From a state on a module, the candidates
// are the modules of the same layer around it (overlaps) and those of the layers whose outer
// face the straight line from the state reaches ahead, in order of path length; the module
// crossed first among them is taken (a layer is skipped once its face lies 20 mm beyond the
// best crossing found: barrel and endcap overlap). In a layer, the modules next to the crossing point (phi bin and row or
// ring, +-1 each; the point on the parabola x + s T + s^2/2 k at the straight-line path s, k the
// path's curvature vector) are candidates; one is crossed if the parabola meets its plane ahead
// within its half extents plus a margin for the helix's deviation from the parabola. The
// nearest candidate is propagated to
// with the RKN stepper; if the propagated point lies outside the module it is excluded and the
// navigation repeats (at most 4 exclusions a step).

constexpr int kChildren = 3;        // measurements a branch may take on one surface
constexpr int kCkfMaxEntries = 32;  // entries (measurements and holes) a candidate may have
// RKN attempts a propagation to the next module may take (the fit allows max_steps): a branch
// whose state cannot reach the module in as many (a seed with far too low a momentum curls)
// excludes it, as an out-of-bounds landing does
constexpr uint32_t kCkfMaxSteps = 100;

struct CkfOpts {
  double chi2_max;
  uint32_t beam, max_holes, max_entries;
};

struct CkfLayers {
  const double* layers;  // [n][8]
  uint32_t n;
  const double* rings;   // [m][4]
  std::vector<int> layer_of;  // surface id -> layer
};

struct Branch {
  double p[5], C[25];
  double h_ctrl;
  double chi2;
  uint32_t n_meas, holes, n_entries, status;
  uint32_t order;  // creation order (the last tie-break)
  int32_t sid;     // current surface (-1: none yet)
  bool done;
  uint32_t e_sid[kCkfMaxEntries];
  int32_t e_meas[kCkfMaxEntries];
};

bool branch_better(const Branch& a, const Branch& b) {
  if (a.n_meas != b.n_meas) return a.n_meas > b.n_meas;
  if (a.holes != b.holes) return a.holes < b.holes;
  if (a.chi2 != b.chi2) return a.chi2 < b.chi2;
  return a.order < b.order;
}

void build_layer_of(CkfLayers& L, uint32_t n_surf) {
  L.layer_of.assign(n_surf, -1);
  for (uint32_t li = 0; li < L.n; ++li) {
    const double* l = L.layers + 8 * li;
    if (l[0] == 0.0) {
      const uint32_t first = uint32_t(l[5]), cnt = uint32_t(l[2]) * uint32_t(l[3]);
      for (uint32_t k = 0; k < cnt && first + k < n_surf; ++k) L.layer_of[first + k] = int(li);
    } else {
      for (uint32_t k = 0; k < uint32_t(l[2]); ++k) {
        const double* rg = L.rings + 4 * (uint32_t(l[3]) + k);
        for (uint32_t ip = 0; ip < uint32_t(rg[1]) && uint32_t(rg[2]) + ip < n_surf; ++ip)
          L.layer_of[uint32_t(rg[2]) + ip] = int(li);
      }
    }
  }
}

// Modules of layer li next to the point q (phi bin and row or ring, +-1).
void layer_candidates(const CkfLayers& L, uint32_t li, const double q[3], std::vector<uint32_t>& out) {
  const double* l = L.layers + 8 * li;
  double phi = std::atan2(q[1], q[0]);
  if (phi < 0.0) phi += 2.0 * kPi;
  if (l[0] == 0.0) {
    const int nphi = int(l[2]), nrows = int(l[3]);
    const int ip0 = int(std::floor(phi / (2.0 * kPi / nphi) + 0.5));
    const int iz0 = int(std::floor(q[2] / l[4] + 0.5 * nrows));
    for (int iz = iz0 - 1; iz <= iz0 + 1; ++iz) {
      if (iz < 0 || iz >= nrows) continue;
      for (int d = -1; d <= 1; ++d) out.push_back(uint32_t(l[5]) + uint32_t(iz * nphi + ((ip0 + d) % nphi + nphi) % nphi));
    }
  } else {
    const int nr = int(l[2]);
    const double r = std::hypot(q[0], q[1]);
    const int k0 = int(std::floor((r - l[5]) / l[4]));
    for (int k = k0 - 1; k <= k0 + 1; ++k) {
      if (k < 0 || k >= nr) continue;
      const double* rg = L.rings + 4 * (uint32_t(l[3]) + uint32_t(k));
      const int nphi = int(rg[1]);
      const int ip0 = int(std::floor(phi / (2.0 * kPi / nphi) + 0.5));
      for (int d = -1; d <= 1; ++d) out.push_back(uint32_t(rg[2]) + uint32_t(((ip0 + d) % nphi + nphi) % nphi));
    }
  }
}

// Straight-line path from x along T to the outer face of layer li (the largest radius a flat
// barrel module reaches, or the |z| of a disk's modules, which sit at the nominal value and
// 1 mm beyond), if that lies ahead and its crossing point is within the layer's extent (margin
// 10 mm); else -1.
double layer_path(const CkfLayers& L, uint32_t li, const double x[3], const double T[3]) {
  const double* l = L.layers + 8 * li;
  double s;
  if (l[0] == 0.0) {
    const double a = T[0] * T[0] + T[1] * T[1], b = x[0] * T[0] + x[1] * T[1];
    // the outer face: flat modules at r and r + 1 mm reach out to sqrt((r + 1)^2 + half_u^2)
    const double rf = std::sqrt((l[1] + 1.0) * (l[1] + 1.0) + l[6] * l[6]);
    const double c = x[0] * x[0] + x[1] * x[1] - rf * rf;
    if (!(a > 0.0) || c >= 0.0) return -1.0;  // outward only: from inside the cylinder
    s = (-b + std::sqrt(b * b - a * c)) / a;
    if (std::fabs(x[2] + s * T[2]) > 0.5 * l[3] * l[4] + 10.0) return -1.0;
  } else {
    if (T[2] == 0.0) return -1.0;
    s = (l[1] + (l[1] > 0.0 ? 1.0 : -1.0) - x[2]) / T[2];  // the outer face (modules at |z| and |z| + 1 mm)
    if (!(s > 0.0)) return -1.0;
    const double r = std::hypot(x[0] + s * T[0], x[1] + s * T[1]);
    if (r < l[5] - 10.0 || r > l[5] + l[2] * l[4] + 10.0) return -1.0;
  }
  return s > 0.0 ? s : -1.0;
}

// Half extents (u, v) of a module: those of its layer.
void module_half(const CkfLayers& L, uint32_t id, double& hu, double& hv) {
  const int li = L.layer_of[id];
  hu = li >= 0 ? L.layers[8 * li + 6] : 1e300;
  hv = li >= 0 ? L.layers[8 * li + 7] : 1e300;
}

// The nearest module among `cand` (not in `skip`) crossed by the parabola x + s T + s^2/2 k (k the
// path curvature vector at x), within its half extents plus a margin for the helix's deviation
// from the parabola (1 mm + s^3 bend^2 / 6, bend = kappa |q/p| |B|); returns -1 if none.
int nearest_crossed(const CkfLayers& L, const Surface* surf, const std::vector<uint32_t>& cand, const double x[3],
                    const double T[3], const double k[3], double bend, const std::vector<uint32_t>& skip,
                    uint32_t n_surf, double* s_out) {
  int best = -1;
  double best_s = 0.0;
  for (uint32_t id : cand) {
    if (id >= n_surf || std::find(skip.begin(), skip.end(), id) != skip.end()) continue;
    const Surface& m = surf[id];
    // the parabola x + s T + s^2/2 k meets the plane n.(r - c) = 0 (straight line if it misses)
    double d[3] = {m.c[0] - x[0], m.c[1] - x[1], m.c[2] - x[2]};
    const double dist = dot3(m.n, d), a = dot3(m.n, T), b = dot3(m.n, k);
    if (a == 0.0) continue;
    double s = dist / a;
    const double disc = a * a + 2.0 * b * dist;
    if (disc >= 0.0) {
      const double q2 = 2.0 * dist / (a + std::copysign(std::sqrt(disc), a));
      if (std::isfinite(q2)) s = q2;
    }
    if (!(s > 1e-3)) continue;
    const double h = 0.5 * s * s;
    double q[3] = {x[0] + s * T[0] + h * k[0] - m.c[0], x[1] + s * T[1] + h * k[1] - m.c[1],
                   x[2] + s * T[2] + h * k[2] - m.c[2]};
    const double margin = 1.0 + s * s * s * bend * bend / 6.0;
    double hu, hv;
    module_half(L, id, hu, hv);
    if (std::fabs(dot3(m.u, q)) > hu + margin || std::fabs(dot3(m.v, q)) > hv + margin) continue;
    // crossings within 1e-6 mm of each other (coplanar overlapping modules) count as one
    // point: the lower id first, whatever the rounding
    if (best < 0 || s < best_s - 1e-6 || (std::fabs(s - best_s) <= 1e-6 && id < uint32_t(best))) {
      best = int(id);
      best_s = s;
    }
  }
  if (s_out) *s_out = best_s;
  return best;
}

// Next module from a state at position x, direction T on surface `cur` (-1: none): the nearest
// crossing among the current layer's modules around x (overlaps) and the modules of the layers
// ahead (a layer is skipped once its face lies 20 mm beyond the best crossing found: layers
// overlap where barrel and endcap meet).
int navigate(const CkfLayers& L, const Surface* surf, uint32_t n_surf, int cur, const double x[3], const double T[3],
             const double k[3], double bend, const std::vector<uint32_t>& skip) {
  std::vector<uint32_t> cand;
  int best = -1;
  double best_s = 0.0;
  if (cur >= 0 && L.layer_of[uint32_t(cur)] >= 0) {  // overlaps in the same layer
    layer_candidates(L, uint32_t(L.layer_of[uint32_t(cur)]), x, cand);
    std::vector<uint32_t> sk = skip;
    sk.push_back(uint32_t(cur));
    best = nearest_crossed(L, surf, cand, x, T, k, bend, sk, n_surf, &best_s);
  }
  std::vector<std::pair<double, uint32_t>> order;
  for (uint32_t li = 0; li < L.n; ++li) {
    if (cur >= 0 && L.layer_of[uint32_t(cur)] == int(li)) continue;
    const double s = layer_path(L, li, x, T);
    if (s > 0.0) order.push_back({s, li});
  }
  std::sort(order.begin(), order.end());
  for (const auto& sl : order) {
    if (best >= 0 && sl.first > best_s + 20.0) break;
    const double h = 0.5 * sl.first * sl.first;  // the parabola's point at the straight-line path
    double q[3] = {x[0] + sl.first * T[0] + h * k[0], x[1] + sl.first * T[1] + h * k[1],
                   x[2] + sl.first * T[2] + h * k[2]};
    cand.clear();
    layer_candidates(L, sl.second, q, cand);
    double sm = 0.0;
    const int m = nearest_crossed(L, surf, cand, x, T, k, bend, skip, n_surf, &sm);
    if (m >= 0 && (best < 0 || sm < best_s)) {
      best = m;
      best_s = sm;
    }
  }
  return best;
}

void find_track(const Surface* surf, uint32_t n_surf, const Field& f, const Opts& o_fit, const CkfOpts& co,
                const CkfLayers& L, const uint32_t* meas_off, const double* meas, uint32_t seed_sid,
                const double* seed_par, const double* seed_cov, Branch& best, bool& have_best) {
  Opts o = o_fit;
  o.max_steps = std::min(o.max_steps, kCkfMaxSteps);
  std::vector<Branch> active(1), children, ended;
  uint32_t order = 0;
  Branch& b0 = active[0];
  std::memcpy(b0.p, seed_par, sizeof(b0.p));
  unpack_cov(seed_cov, b0.C);
  b0.h_ctrl = o.h_max;
  b0.chi2 = 0.0;
  b0.n_meas = b0.holes = b0.n_entries = b0.status = 0;
  b0.order = order++;
  b0.sid = -1;
  b0.done = false;
  have_best = false;
  bool first_step = true;
  while (!active.empty()) {
    children.clear();
    for (Branch& br : active) {
      // ---- the next surface and the predicted state on it
      Branch nb = br;
      int target = -1;
      double pp[5], Cp[25];
      if (first_step) {
        target = int(seed_sid);
        std::memcpy(pp, br.p, sizeof(pp));
        std::memcpy(Cp, br.C, sizeof(Cp));
      } else {
        if (br.n_entries >= co.max_entries) {
          ended.push_back(br);
          continue;
        }
        const Surface& sc = surf[uint32_t(br.sid)];
        double pm[5], Q[25];
        std::memcpy(pm, br.p, sizeof(pm));
        const uint32_t stm = material(sc, o, pm, Q);
        if (stm & kFatal) {
          ended.push_back(br);
          continue;
        }
        double x[3], T[3], B[3];
        bound_to_free(sc, pm, x, T);
        bool oof = false;
        field_at(f, x, B, &oof);
        const double bend = kKappa * std::fabs(pm[4]) * std::sqrt(dot3(B, B));
        double kc[3];  // curvature vector of the path: kappa (q/p) T x B
        kc[0] = kKappa * pm[4] * (T[1] * B[2] - T[2] * B[1]);
        kc[1] = kKappa * pm[4] * (T[2] * B[0] - T[0] * B[2]);
        kc[2] = kKappa * pm[4] * (T[0] * B[1] - T[1] * B[0]);
        std::vector<uint32_t> skip;
        for (int tries = 0; tries < 4 && target < 0; ++tries) {
          const int m = navigate(L, surf, n_surf, br.sid, x, T, kc, bend, skip);
          if (m < 0) break;
          const Surface& sk = surf[uint32_t(m)];
          double r[3], Tt[3], Dtot[49], dxds[7], Jb2f[35], Jf2b[35], P[49], tmp[49], t75[35], J[25];
          std::memcpy(r, x, sizeof(r));
          std::memcpy(Tt, T, sizeof(Tt));
          jac_bound_to_free(sc, pm, Jb2f);
          PropState ps{br.h_ctrl, 0, 0, o.h_max, false};
          const uint32_t stp = propagate(f, o, sk, r, Tt, pm[4], Dtot, dxds, ps);
          if (stp & kFatal) {
            skip.push_back(uint32_t(m));
            continue;
          }
          double d[3] = {r[0] - sk.c[0], r[1] - sk.c[1], r[2] - sk.c[2]}, hu, hv;
          module_half(L, uint32_t(m), hu, hv);
          if (std::fabs(dot3(sk.u, d)) > hu || std::fabs(dot3(sk.v, d)) > hv) {
            skip.push_back(uint32_t(m));
            continue;
          }
          jac_free_to_bound(sk, Tt, Jf2b);
          path_correction(sk, Tt, dxds, P);
          matmul(P, Dtot, tmp, 7, 7, 7);
          matmul(tmp, Jb2f, t75, 7, 7, 5);
          matmul(Jf2b, t75, J, 5, 7, 5);
          free_to_bound(sk, r, Tt, pm[4], pp);
          double CQ[25], Jt[25], t55[25];
          for (int i = 0; i < 25; ++i) CQ[i] = br.C[i] + Q[i];
          transpose(J, Jt, 5, 5);
          matmul(J, CQ, t55, 5, 5, 5);
          matmul(t55, Jt, Cp, 5, 5, 5);
          symmetrize(Cp, 5);
          nb.h_ctrl = ps.h_ctrl;
          target = m;
        }
        if (target < 0) {  // nothing ahead: the branch ends
          ended.push_back(br);
          continue;
        }
      }
      // ---- branches on the target surface: compatible measurements, best kChildren by chi2
      nb.sid = target;
      std::vector<std::pair<double, uint32_t>> ok;
      for (uint32_t mi = meas_off[uint32_t(target)]; mi < meas_off[uint32_t(target) + 1]; ++mi) {
        const double* mk = meas + 5 * size_t(mi);
        double pt[5], Ct[25], c2 = 0.0;
        std::memcpy(pt, pp, sizeof(pt));
        std::memcpy(Ct, Cp, sizeof(Ct));
        const double m2[2] = {mk[0], mk[1]}, V[4] = {mk[2], mk[3], mk[3], mk[4]};
        if (kf_update(m2, V, pt, Ct, &c2) != 0) continue;
        if (c2 < co.chi2_max) ok.push_back({c2, mi});
      }
      std::sort(ok.begin(), ok.end());
      for (size_t j = 0; j < ok.size() && j < size_t(kChildren); ++j) {
        Branch ch = nb;
        const double* mk = meas + 5 * size_t(ok[j].second);
        const double m2[2] = {mk[0], mk[1]}, V[4] = {mk[2], mk[3], mk[3], mk[4]};
        std::memcpy(ch.p, pp, sizeof(ch.p));
        std::memcpy(ch.C, Cp, sizeof(ch.C));
        double c2 = 0.0;
        kf_update(m2, V, ch.p, ch.C, &c2);
        ch.p[2] = wrap_phi(ch.p[2]);
        ch.chi2 += c2;
        ch.n_meas += 1;
        ch.holes = 0;
        ch.e_sid[ch.n_entries] = uint32_t(target);
        ch.e_meas[ch.n_entries] = int32_t(ok[j].second);
        ch.n_entries += 1;
        ch.order = order++;
        children.push_back(ch);
      }
      if (nb.holes < co.max_holes) {
        Branch ch = nb;
        std::memcpy(ch.p, pp, sizeof(ch.p));
        std::memcpy(ch.C, Cp, sizeof(ch.C));
        ch.holes += 1;
        ch.e_sid[ch.n_entries] = uint32_t(target) | kNoMeasurement;
        ch.e_meas[ch.n_entries] = -1;
        ch.n_entries += 1;
        ch.order = order++;
        children.push_back(ch);
      } else if (ok.empty()) {
        ended.push_back(br);  // one hole too many: the branch ends before this surface
      }
    }
    first_step = false;
    std::stable_sort(children.begin(), children.end(), branch_better);
    if (children.size() > co.beam) children.resize(co.beam);
    active.swap(children);
  }
  for (const Branch& e : ended)
    if (!have_best || branch_better(e, best)) {
      best = e;
      have_best = true;
    }
}
}  // namespace

// ================================================================ C interface
extern "C" {

struct orc_field {
  int kind;
  double B[3];
  int nr, nz;
  double r0, dr, z0, dz;
  const float* Br;
  const float* Bz;
};

struct orc_opts {
  double tol, h_max, h_min, surf_tol, mass;
  uint32_t max_steps;
  double ZA, I_eV, rho, hwp_eV;
  const uint16_t* mlp_bf16;  // 5057 BF16 weights (W1, b1, W2, b2, w3, b3) or null
  int smoother;              // 0: RTS, 1: two-filter
  double inflation;          // two-filter: backward filter's starting covariance factor
};

static float bf16_to_float(uint16_t b) {
  uint32_t u = uint32_t(b) << 16;
  float f;
  std::memcpy(&f, &u, 4);
  return f;
}

static void unpack_mlp(const uint16_t* w, Mlp& m) {
  size_t k = 0;
  for (int j = 0; j < 64; ++j)
    for (int i = 0; i < 12; ++i) m.W1[j][i] = bf16_to_float(w[k++]);
  for (int j = 0; j < 64; ++j) m.b1[j] = bf16_to_float(w[k++]);
  for (int j = 0; j < 64; ++j)
    for (int i = 0; i < 64; ++i) m.W2[j][i] = bf16_to_float(w[k++]);
  for (int j = 0; j < 64; ++j) m.b2[j] = bf16_to_float(w[k++]);
  for (int i = 0; i < 64; ++i) m.w3[i] = bf16_to_float(w[k++]);
  m.b3 = bf16_to_float(w[k++]);
}

static Field to_field(const orc_field* f) {
  Field F;
  F.kind = f->kind;
  for (int i = 0; i < 3; ++i) F.B[i] = f->B[i];
  F.nr = f->nr; F.nz = f->nz;
  F.r0 = f->r0; F.dr = f->dr; F.z0 = f->z0; F.dz = f->dz;
  F.Br = f->Br; F.Bz = f->Bz;
  return F;
}

static Opts to_opts(const orc_opts* o, Mlp* storage) {
  Opts O;
  O.mlp = nullptr;
  if (o->mlp_bf16 && storage) {
    unpack_mlp(o->mlp_bf16, *storage);
    O.mlp = storage;
  }
  O.tol = o->tol; O.h_max = o->h_max; O.h_min = o->h_min; O.surf_tol = o->surf_tol; O.mass = o->mass;
  O.max_steps = o->max_steps;
  O.ZA = o->ZA; O.I_eV = o->I_eV; O.rho = o->rho; O.hwp_eV = o->hwp_eV;
  O.smoother = o->smoother;
  O.inflation = o->inflation;
  return O;
}

// surfaces: [n][14] = u[3], v[3], n[3], c[3], t, X0
static std::vector<Surface> to_surfaces(const double* s, uint32_t n) {
  std::vector<Surface> out(n);
  for (uint32_t i = 0; i < n; ++i) {
    const double* q = s + 14 * i;
    for (int j = 0; j < 3; ++j) {
      out[i].u[j] = q[j];
      out[i].v[j] = q[3 + j];
      out[i].n[j] = q[6 + j];
      out[i].c[j] = q[9 + j];
    }
    out[i].t = q[12];
    out[i].X0 = q[13];
  }
  return out;
}

// Fit n_tracks tracks. meas: [n_meas][5] (loc0, loc1, V00, V01, V11); seed_par [n][5];
// seed_cov [n][15] packed upper triangle; outputs in the same AoS layouts.
// steps (nullable): [n][2] = step attempts, rejected attempts. cov_filt0 (nullable): [n][15]
// filtered covariance at the first surface. n_threads >= 1.
// Fits every track; with `states_par` [n_meas][5] and `states_cov`, `states_cov_filt`
// [n_meas][15] (packed) not NULL it also writes every entry's smoothed state and filtered
// covariance (rows indexed like the measurements; NaN for a track whose status is fatal).
static int fit_batch(const double* surfaces, uint32_t n_surf, const orc_field* field, const orc_opts* opts,
                     uint32_t n_tracks, uint64_t n_meas, const uint32_t* offsets, const double* meas,
                     const uint32_t* sid, const double* seed_par, const double* seed_cov, double* out_par,
                     double* out_cov, double* chi2, int32_t* ndf, uint32_t* status, uint32_t* steps,
                     double* cov_filt0, double* states_par, double* states_cov, double* states_cov_filt,
                     int n_threads) {
  std::vector<Surface> surf = to_surfaces(surfaces, n_surf);
  Field F = to_field(field);
  Mlp mlp_store;
  Opts O = to_opts(opts, &mlp_store);
  const bool want_states = states_par && states_cov && states_cov_filt;
  auto work = [&](uint32_t lo, uint32_t hi) {
    for (uint32_t i = lo; i < hi; ++i) {
      TrackIn in;
      uint32_t a = offsets[i], b = offsets[i + 1];
      TrackOut out;
      States keep;
      if (b < a || b > n_meas) {
        fill_nan(out);
        for (int j = 0; j < 15; ++j) out.cov_filt0[j] = std::nan("");
        out.status = kBadInput;
        out.ndf = 0;
        out.attempts = out.rejected = 0;
      } else {
        in.N = b - a;
        in.meas = meas + 5 * size_t(a);
        in.sid = sid + a;
        in.seed_par = seed_par + 5 * size_t(i);
        in.seed_cov = seed_cov + 15 * size_t(i);
        fit_track(surf.data(), n_surf, F, O, in, out, want_states ? &keep : nullptr);
        if (want_states) {
          const bool ok = !(out.status & kFatal) && !keep.ps.empty();
          for (uint32_t k = 0; k < b - a; ++k) {
            const size_t e = size_t(a) + k;
            for (int j = 0; j < 5; ++j) states_par[5 * e + j] = ok ? keep.ps[5 * k + j] : std::nan("");
            if (ok) {
              pack_cov(&keep.Cs[25 * k], states_cov + 15 * e);
              pack_cov(&keep.Cf[25 * k], states_cov_filt + 15 * e);
            } else {
              for (int j = 0; j < 15; ++j) states_cov[15 * e + j] = states_cov_filt[15 * e + j] = std::nan("");
            }
          }
        }
      }
      std::memcpy(out_par + 5 * size_t(i), out.par, sizeof(double) * 5);
      std::memcpy(out_cov + 15 * size_t(i), out.cov, sizeof(double) * 15);
      chi2[i] = out.chi2;
      ndf[i] = out.ndf;
      status[i] = out.status;
      if (steps) {
        steps[2 * size_t(i)] = out.attempts;
        steps[2 * size_t(i) + 1] = out.rejected;
      }
      if (cov_filt0) std::memcpy(cov_filt0 + 15 * size_t(i), out.cov_filt0, sizeof(double) * 15);
    }
  };
  if (n_threads <= 1 || n_tracks < 2) {
    work(0, n_tracks);
    return 0;
  }
  std::vector<std::thread> th;
  uint32_t per = (n_tracks + n_threads - 1) / n_threads;
  for (int t = 0; t < n_threads; ++t) {
    uint32_t lo = std::min<uint32_t>(n_tracks, t * per), hi = std::min<uint32_t>(n_tracks, lo + per);
    if (lo < hi) th.emplace_back(work, lo, hi);
  }
  for (auto& x : th) x.join();
  return 0;
}

int orc_fit(const double* surfaces, uint32_t n_surf, const orc_field* field, const orc_opts* opts,
            uint32_t n_tracks, uint64_t n_meas, const uint32_t* offsets, const double* meas, const uint32_t* sid,
            const double* seed_par, const double* seed_cov, double* out_par, double* out_cov, double* chi2,
            int32_t* ndf, uint32_t* status, uint32_t* steps, double* cov_filt0, int n_threads) {
  return fit_batch(surfaces, n_surf, field, opts, n_tracks, n_meas, offsets, meas, sid, seed_par, seed_cov, out_par,
                   out_cov, chi2, ndf, status, steps, cov_filt0, nullptr, nullptr, nullptr, n_threads);
}

// orc_fit that also writes the smoothed state (and the filtered covariance) of every entry.
int orc_fit_all_states(const double* surfaces, uint32_t n_surf, const orc_field* field, const orc_opts* opts,
                   uint32_t n_tracks, uint64_t n_meas, const uint32_t* offsets, const double* meas,
                   const uint32_t* sid, const double* seed_par, const double* seed_cov, double* out_par,
                   double* out_cov, double* chi2, int32_t* ndf, uint32_t* status, uint32_t* steps,
                   double* cov_filt0, double* states_par, double* states_cov, double* states_cov_filt,
                   int n_threads) {
  return fit_batch(surfaces, n_surf, field, opts, n_tracks, n_meas, offsets, meas, sid, seed_par, seed_cov, out_par,
                   out_cov, chi2, ndf, status, steps, cov_filt0, states_par, states_cov, states_cov_filt, n_threads);
}

// Training records of the step proposer from the oracle's plain adaptive fit of every track,
// in track order: rec [cap][13] (12 inputs, label); returns the number of records (at most cap
// are written).
uint64_t orc_record_steps(const double* surfaces, uint32_t n_surf, const orc_field* field, const orc_opts* opts,
                          uint32_t n_tracks, uint64_t n_meas, const uint32_t* offsets, const double* meas,
                          const uint32_t* sid, const double* seed_par, const double* seed_cov, float* rec,
                          uint64_t cap) {
  std::vector<Surface> surf = to_surfaces(surfaces, n_surf);
  Field F = to_field(field);
  Mlp mlp_store;
  Opts O = to_opts(opts, &mlp_store);
  O.mlp = nullptr;  // the plain control makes the records
  std::vector<float> all;
  O.records = &all;
  for (uint32_t i = 0; i < n_tracks; ++i) {
    uint32_t a = offsets[i], b = offsets[i + 1];
    if (b < a || b > n_meas) continue;
    TrackIn in;
    in.N = b - a;
    in.meas = meas + 5 * size_t(a);
    in.sid = sid + a;
    in.seed_par = seed_par + 5 * size_t(i);
    in.seed_cov = seed_cov + 15 * size_t(i);
    TrackOut out;
    fit_track(surf.data(), n_surf, F, O, in, out);
  }
  const uint64_t n = all.size() / 13;
  std::memcpy(rec, all.data(), sizeof(float) * 13 * size_t(std::min(n, cap)));
  return n;
}

// ---- component entry points used by the oracle's own pins

void orc_field_at(const orc_field* field, const double* x, uint32_t n, double* B, uint8_t* oof) {
  Field F = to_field(field);
  for (uint32_t i = 0; i < n; ++i) {
    bool o = false;
    field_at(F, x + 3 * i, B + 3 * i, &o);
    oof[i] = o ? 1 : 0;
  }
}

// n_steps fixed steps of length h; writes the final (r, T) and the accumulated 7x7 D.
void orc_rkn_fixed(const orc_field* field, const double* r0, const double* T0, double lam, double h,
                   uint32_t n_steps, double* r_out, double* T_out, double* D_out) {
  Field F = to_field(field);
  double r[3] = {r0[0], r0[1], r0[2]}, T[3] = {T0[0], T0[1], T0[2]};
  double D[49];
  for (int i = 0; i < 49; ++i) D[i] = (i % 8 == 0) ? 1.0 : 0.0;
  for (uint32_t s = 0; s < n_steps; ++s) {
    Step st;
    bool oof = false;
    rkn_step(F, r, T, lam, h, st, &oof);
    for (int i = 0; i < 3; ++i) {
      r[i] = st.r[i];
      T[i] = st.T[i];
    }
    matmul(st.D, D, D, 7, 7, 7);
  }
  std::memcpy(r_out, r, sizeof(r));
  std::memcpy(T_out, T, sizeof(T));
  if (D_out) std::memcpy(D_out, D, sizeof(D));
}

// One RKN step: writes r', T', eps.
void orc_rkn_step(const orc_field* field, const double* r, const double* T, double lam, double h,
                  double* r_out, double* T_out, double* eps) {
  Field F = to_field(field);
  Step st;
  bool oof = false;
  rkn_step(F, r, T, lam, h, st, &oof);
  std::memcpy(r_out, st.r, sizeof(st.r));
  std::memcpy(T_out, st.T, sizeof(st.T));
  *eps = st.eps;
}

// Bound -> bound transport from surface a to surface b (no material, no update):
// par_out = f(par_in), J = d par_out / d par_in (5x5 row-major). Returns the status bits.
uint32_t orc_transport(const double* surfaces, uint32_t a, uint32_t b, const orc_field* field,
                       const orc_opts* opts, const double* par_in, double* par_out, double* J,
                       uint32_t* attempts) {
  std::vector<Surface> surf = to_surfaces(surfaces, std::max(a, b) + 1);
  Field F = to_field(field);
  Mlp mlp_store;
  Opts O = to_opts(opts, &mlp_store);
  double r[3], T[3], Dtot[49], dxds[7], Jb2f[35], Jf2b[35], P[49], tmp[49], t75[35];
  bound_to_free(surf[a], par_in, r, T);
  jac_bound_to_free(surf[a], par_in, Jb2f);
  PropState ps{O.h_max, 0, 0, O.h_max, true};
  uint32_t st = propagate(F, O, surf[b], r, T, par_in[4], Dtot, dxds, ps);
  if (attempts) *attempts = ps.attempts;
  if (st & kFatal) return st;
  jac_free_to_bound(surf[b], T, Jf2b);
  path_correction(surf[b], T, dxds, P);
  matmul(P, Dtot, tmp, 7, 7, 7);
  matmul(tmp, Jb2f, t75, 7, 7, 5);
  matmul(Jf2b, t75, J, 5, 7, 5);
  free_to_bound(surf[b], r, T, par_in[4], par_out);
  return st;
}

// Material model at one surface: theta0, and the q/p after the mean energy loss.
uint32_t orc_material(const double* surface14, const orc_opts* opts, const double* par, double* theta0,
                      double* qop_after, double* dedx_mev_cm2_g) {
  std::vector<Surface> s = to_surfaces(surface14, 1);
  Mlp mlp_store;
  Opts O = to_opts(opts, &mlp_store);
  double p[5], Q[25];
  std::memcpy(p, par, sizeof(p));
  uint32_t st = material(s[0], O, p, Q);
  *theta0 = std::sqrt(Q[3 * 5 + 3]);
  *qop_after = p[4];
  double mom = 1.0 / std::fabs(par[4]);
  *dedx_mev_cm2_g = bethe(mom, O.mass, O);
  return st;
}

// Linear-Gaussian chain through the oracle's own update and smoother: states x_k in R^5
// with x_k = J_k (x_{k-1} + w_{k-1}), w ~ N(0, Q_{k-1}), measured by H = [I2 0] with
// covariance V_k; prior x_0 ~ N(p0, C0). Writes the smoothed mean/cov of every state
// (ps [N][5], Cs [N][25]) and the chi2 sum; a step whose measurement is NaN has none.
// Returns status bits.
uint32_t orc_linear_chain(int N, const double* J, const double* Q, const double* p0, const double* C0,
                          const double* m, const double* V, double* ps, double* Cs, double* chi2_out,
                          double* pf_out, double* Cf_out) {
  std::vector<double> pp(N * 5), Cp(N * 25), pf(N * 5), Cf(N * 25);
  std::memcpy(&pp[0], p0, sizeof(double) * 5);
  std::memcpy(&Cp[0], C0, sizeof(double) * 25);
  double chi2 = 0.0;
  uint32_t st = 0;
  for (int k = 0; k < N; ++k) {
    if (k > 0) {
      const double* Jk = J + 25 * k;
      double CQ[25], Jt[25], t[25];
      for (int i = 0; i < 25; ++i) CQ[i] = Cf[(k - 1) * 25 + i] + Q[(k - 1) * 25 + i];
      matmul(Jk, &pf[(k - 1) * 5], &pp[k * 5], 5, 5, 1);
      transpose(Jk, Jt, 5, 5);
      matmul(Jk, CQ, t, 5, 5, 5);
      matmul(t, Jt, &Cp[k * 25], 5, 5, 5);
      symmetrize(&Cp[k * 25], 5);
    }
    std::memcpy(&pf[k * 5], &pp[k * 5], sizeof(double) * 5);
    std::memcpy(&Cf[k * 25], &Cp[k * 25], sizeof(double) * 25);
    double c2 = 0.0, mm[2] = {m[2 * k], m[2 * k + 1]};
    if (std::isnan(mm[0])) continue;  // a step without a measurement, as a hole in fit_track
    st |= kf_update(mm, V + 4 * k, &pf[k * 5], &Cf[k * 25], &c2);
    chi2 += c2;
  }
  // The linear chain has no angle wrap: undo wrap_phi's effect by keeping |phi| small.
  st |= rts(N, &pf[0], &Cf[0], &pp[0], &Cp[0], J, ps, Cs);
  *chi2_out = chi2;
  if (pf_out) std::memcpy(pf_out, &pf[0], sizeof(double) * 5 * N);
  if (Cf_out) std::memcpy(Cf_out, &Cf[0], sizeof(double) * 25 * N);
  return st;
}

// Inverse of a general n x n matrix by Gauss-Jordan elimination with partial pivoting.
static bool general_inverse(const double* A, double* Ai, int n) {
  std::vector<double> M(A, A + n * n);
  for (int i = 0; i < n * n; ++i) Ai[i] = (i % (n + 1) == 0) ? 1.0 : 0.0;
  for (int c = 0; c < n; ++c) {
    int piv = c;
    for (int r = c + 1; r < n; ++r)
      if (std::fabs(M[r * n + c]) > std::fabs(M[piv * n + c])) piv = r;
    if (!(std::fabs(M[piv * n + c]) > 0.0)) return false;
    for (int j = 0; j < n; ++j) {
      std::swap(M[c * n + j], M[piv * n + j]);
      std::swap(Ai[c * n + j], Ai[piv * n + j]);
    }
    const double d = M[c * n + c];
    for (int j = 0; j < n; ++j) {
      M[c * n + j] /= d;
      Ai[c * n + j] /= d;
    }
    for (int r = 0; r < n; ++r) {
      if (r == c) continue;
      const double f = M[r * n + c];
      for (int j = 0; j < n; ++j) {
        M[r * n + j] -= f * M[c * n + j];
        Ai[r * n + j] -= f * Ai[c * n + j];
      }
    }
  }
  return true;
}

// The two-filter smoother on the linear chain of orc_linear_chain: the forward filter, then the
// backward filter of x_k = J_{k+1}^-1 x_{k+1} - w_k (w_k ~ N(0, Q_k), the noise of step k seen
// from its far end) from the last filtered state with the covariance times `inflation`, then the
// weighted mean with the prior (p0, C0) at step 0. Returns the smoothed state at step 0.
uint32_t orc_linear_chain_two_filter(int N, const double* J, const double* Q, const double* p0, const double* C0,
                                     const double* m, const double* V, double inflation, double* ps0, double* Cs0) {
  std::vector<double> pf(N * 5), Cf(N * 25);
  double chi2 = 0.0;
  std::vector<double> ps(N * 5), Cs(N * 25);
  uint32_t st = orc_linear_chain(N, J, Q, p0, C0, m, V, &ps[0], &Cs[0], &chi2, &pf[0], &Cf[0]);
  st &= ~kSmootherNotSpd;  // only the forward filter is used
  double pb[5], Cb[25];
  std::memcpy(pb, &pf[(N - 1) * 5], sizeof(pb));
  for (int i = 0; i < 25; ++i) Cb[i] = Cf[(N - 1) * 25 + i] * inflation;
  for (int k = N - 1; k >= 0; --k) {
    if (k < N - 1) {
      double Ji[25], Jit[25], t[25], pn[5];
      if (!general_inverse(J + 25 * (k + 1), Ji, 5)) return st | kSmootherNotSpd;
      matmul(Ji, pb, pn, 5, 5, 1);
      std::memcpy(pb, pn, sizeof(pb));
      transpose(Ji, Jit, 5, 5);
      matmul(Ji, Cb, t, 5, 5, 5);
      matmul(t, Jit, Cb, 5, 5, 5);
      for (int i = 0; i < 25; ++i) Cb[i] += Q[k * 25 + i];
      symmetrize(Cb, 5);
    }
    double mm[2] = {m[2 * k], m[2 * k + 1]}, c2 = 0.0;
    if (std::isnan(mm[0])) continue;
    st |= kf_update(mm, V + 4 * k, pb, Cb, &c2);
  }
  st |= weighted_mean(p0, C0, pb, Cb, ps0, Cs0);
  return st;
}

// Fits one track and exports its per-measurement states: predicted (pp [N][5], Cp [N][25]),
// filtered (pf, Cf), smoothed (ps, Cs) and the transport Jacobians J [N][25] (J[0] unused).
uint32_t orc_fit_states(const double* surfaces, uint32_t n_surf, const orc_field* field, const orc_opts* opts,
                        uint32_t N, const double* meas, const uint32_t* sid, const double* seed_par,
                        const double* seed_cov, double* pp, double* Cp, double* pf, double* Cf, double* J,
                        double* ps, double* Cs, double* chi2) {
  std::vector<Surface> surf = to_surfaces(surfaces, n_surf);
  Field F = to_field(field);
  Mlp mlp_store;
  Opts O = to_opts(opts, &mlp_store);
  TrackIn in{N, meas, sid, seed_par, seed_cov};
  TrackOut out;
  States st;
  fit_track(surf.data(), n_surf, F, O, in, out, &st);
  if (st.pp.size() == size_t(N) * 5) {
    std::memcpy(pp, st.pp.data(), sizeof(double) * 5 * N);
    std::memcpy(Cp, st.Cp.data(), sizeof(double) * 25 * N);
    std::memcpy(pf, st.pf.data(), sizeof(double) * 5 * N);
    std::memcpy(Cf, st.Cf.data(), sizeof(double) * 25 * N);
    std::memcpy(J, st.J.data(), sizeof(double) * 25 * N);
    std::memcpy(ps, st.ps.data(), sizeof(double) * 5 * N);
    std::memcpy(Cs, st.Cs.data(), sizeof(double) * 25 * N);
  }
  *chi2 = out.chi2;
  return out.status;
}

// Raw network output (ln of the proposed step before the 0.9 factor and clamping) for n inputs
// x [n][12], with BF16 weights w (5057).
void orc_mlp_forward(const uint16_t* w, const float* x, uint32_t n, float* out) {
  Mlp m;
  unpack_mlp(w, m);
  for (uint32_t s = 0; s < n; ++s) {
    const float* xi = x + 12 * size_t(s);
    float a1[64], a2[64];
    for (int j = 0; j < 64; ++j) {
      float z = m.b1[j];
      for (int i = 0; i < 12; ++i) z += m.W1[j][i] * xi[i];
      a1[j] = silu(z);
    }
    for (int j = 0; j < 64; ++j) {
      float z = m.b2[j];
      for (int i = 0; i < 64; ++i) z += m.W2[j][i] * a1[i];
      a2[j] = silu(z);
    }
    float o = m.b3;
    for (int i = 0; i < 64; ++i) o += m.w3[i] * a2[i];
    out[s] = o;
  }
}

// Learned mode: each track's proposed starting step-size control (h_max where there are fewer
// than two measurements or a surface id is out of range).
void orc_propose_start(const double* surfaces, uint32_t n_surf, const orc_field* field, const orc_opts* opts,
                       uint32_t n_tracks, uint64_t n_meas, const uint32_t* offsets, const uint32_t* sid,
                       const double* seed_par, double* h0) {
  std::vector<Surface> surf = to_surfaces(surfaces, n_surf);
  Field F = to_field(field);
  Mlp mlp_store;
  Opts O = to_opts(opts, &mlp_store);
  for (uint32_t i = 0; i < n_tracks; ++i) {
    const uint32_t a = offsets[i], b = offsets[i + 1];
    h0[i] = O.h_max;
    if (!O.mlp || b < a || b - a < 2 || b > n_meas || surface_of(sid[a]) >= n_surf ||
        surface_of(sid[a + 1]) >= n_surf)
      continue;
    h0[i] = propose_start(surf[surface_of(sid[a])], surf[surface_of(sid[a + 1])], F, O, seed_par + 5 * size_t(i));
  }
}

// ---------------------------------------------------------------- seed estimation (helix through 3 hits)
// Reading (the paper lists track parameter estimation from a seed as a step of the chain,
// Sec. 2, and prints no method): three measurements of a track give three space points; the
// helix axis is z. In the transverse plane the circle through the points gives the radius R,
// the turning sense (hence the charge) and the direction at the first point; along a helix z is
// linear in the transverse arc length, which gives cot(theta) from points 1 and 3;
// p_T = kappa |B_z| R. The parameters are expressed on the surface of the first measurement (its
// measured local position, the direction angles, q/p). Exact for noise-free hits of a track in
// a uniform axial field without material.
// Status: 1 fewer than 3 measurements; 2 no curvature (collinear points in the transverse plane,
// or B_z = 0: a straight line, q/p = 0); 4 bad input (offsets or surface ids, or a first entry
// without a measurement).
static uint32_t helix_seed(const double r1[3], const double r2[3], const double r3[3], double bz, double par[3]) {
  // par: phi, theta, q/p at r1
  const double ax = r2[0] - r1[0], ay = r2[1] - r1[1], bx = r3[0] - r1[0], by = r3[1] - r1[1];
  const double a2 = ax * ax + ay * ay, b2 = bx * bx + by * by;
  // twice the signed area of the triangle: > 0 when 1 -> 2 -> 3 runs counterclockwise seen from +z
  const double D = 2.0 * (ax * by - ay * bx);
  uint32_t st = 0;
  double tx, ty, s13;
  if (!(std::fabs(D) > 1e-12 * (a2 + b2)) || bz == 0.0) {
    st = 2;  // the straight line from point 1 to point 3
    const double c13 = std::sqrt(b2);
    tx = bx / c13;
    ty = by / c13;
    s13 = c13;
    par[2] = 0.0;
  } else {
    // centre of the circle, relative to point 1
    const double cx = (by * a2 - ay * b2) / D, cy = (ax * b2 - bx * a2) / D;
    const double R = std::sqrt(cx * cx + cy * cy);
    // unit tangent at point 1 in the sense of travel: the radius vector (-cx, -cy) turned by
    // +90 degrees when counterclockwise, -90 when clockwise
    const double sg = D > 0.0 ? 1.0 : -1.0;
    tx = sg * cy / R;
    ty = -sg * cx / R;
    // transverse arc from point 1 to point 3 in the sense of travel (up to one full turn)
    const double u1x = -cx, u1y = -cy, u3x = bx - cx, u3y = by - cy;
    double ang = std::atan2(sg * (u1x * u3y - u1y * u3x), u1x * u3x + u1y * u3y);
    if (ang < 0.0) ang += 2.0 * kPi;
    s13 = R * ang;
    // F = q v x B: for B_z > 0 a positive charge turns clockwise seen from +z
    const double q = (D > 0.0) == (bz > 0.0) ? -1.0 : 1.0;
    const double pt = kKappa * std::fabs(bz) * R;
    const double cot = (r3[2] - r1[2]) / s13;
    par[2] = q / (pt * std::sqrt(1.0 + cot * cot));
  }
  par[0] = std::atan2(ty, tx);
  par[1] = std::atan2(s13, r3[2] - r1[2]);
  return st;
}

static void seed_track(const Surface* surf, uint32_t n_surf, const Field& F, const double* meas, const uint32_t* sid,
                       uint32_t N, int first_three, double par[5], double cov[15], uint32_t* status) {
  for (int j = 0; j < 5; ++j) par[j] = std::nan("");
  for (int j = 0; j < 15; ++j) cov[j] = 0.0;
  // entries without a measurement (holes, passive surfaces) give no space point; the seed is
  // expressed on the first entry's surface, which therefore needs its measurement
  std::vector<uint32_t> mi;
  for (uint32_t e = 0; e < N; ++e) {
    if (surface_of(sid[e]) >= n_surf) {
      *status = 4;
      return;
    }
    if (measured(sid[e])) mi.push_back(e);
  }
  if (N > 0 && !measured(sid[0])) {
    *status = 4;
    return;
  }
  const uint32_t M = uint32_t(mi.size());
  if (M < 3) {
    *status = 1;
    return;
  }
  // Reading (which three): the first, middle and last measurements of the candidate by default
  // (the longest lever arm the candidate offers); the first three on request, as for a seed
  // made of three inner space points.
  const uint32_t k[3] = {mi[0], mi[first_three ? 1u : (M - 1) / 2], mi[first_three ? 2u : M - 1]};
  double r[3][3], bz[3];
  for (int j = 0; j < 3; ++j) {
    const Surface& s = surf[sid[k[j]]];
    const double* m = meas + 5 * size_t(k[j]);
    for (int i = 0; i < 3; ++i) r[j][i] = s.c[i] + m[0] * s.u[i] + m[1] * s.v[i];
    double B[3];
    bool oof = false;
    field_at(F, r[j], B, &oof);
    bz[j] = B[2];
  }
  // Reading (field): the mean of B_z at the three points
  const double bmean = (bz[0] + bz[1] + bz[2]) / 3.0;
  double ang[3];
  *status = helix_seed(r[0], r[1], r[2], bmean, ang);
  par[0] = meas[0];
  par[1] = meas[1];
  par[2] = ang[0];
  par[3] = ang[1];
  par[4] = ang[2];

  // Reading (covariance: a prior for the fit, meant to be wide rather than narrow). The local
  // position is the first measurement's. sh2 is the mean per-coordinate hit variance. Multiple
  // scattering: the Highland angle theta0 of the first surface at normal incidence, at the
  // estimated momentum (1 GeV without curvature) and beta = 1, once per surface spanned. Angles:
  // the hit errors over the lever arm L (transverse L_T for phi) plus twice the scattering, and for
  // phi the bending angle L_T / 2R times the relative curvature error. Relative q/p error: hit
  // errors and scattering over the sagitta, the spread of B_z over the points, and a 1 % floor.
  // Without curvature var(q/p) = 1 GeV^-2. Angle variances are at most pi^2.
  double sh2 = 0.0;
  for (int j = 0; j < 3; ++j) sh2 += (meas[5 * k[j] + 2] + meas[5 * k[j] + 4]) / 6.0;
  const double dx = r[2][0] - r[0][0], dy = r[2][1] - r[0][1], dz = r[2][2] - r[0][2];
  const double LT2 = dx * dx + dy * dy, L2 = LT2 + dz * dz;
  const double p_est = *status == 0 ? std::fabs(1.0 / ang[2]) : 1.0;
  const Surface& s0 = surf[sid[0]];  // measured, so no flag bit
  const double th0 = (s0.t > 0.0 && s0.X0 > 0.0) ? highland(p_est, 1.0, s0.t, s0.X0) : 0.0;
  const double ms2 = double(k[2] - k[0]) * th0 * th0;
  const double sth = std::sin(ang[1]);
  double var_phi = 64.0 * sh2 / LT2 + 2.0 * ms2 / (sth * sth);
  double var_qop = 1.0;
  if (*status == 0) {
    const double R = p_est * sth / (kKappa * std::fabs(bmean));
    const double sag = LT2 / (8.0 * R);
    const double bmax = std::fmax(bz[0], std::fmax(bz[1], bz[2]));
    const double bmin = std::fmin(bz[0], std::fmin(bz[1], bz[2]));
    const double db = (bmax - bmin) / bmean;
    const double rel2 = 4.0 * sh2 / (sag * sag) + ms2 * LT2 / (16.0 * sag * sag) + db * db + 1e-4;
    var_qop = rel2 * ang[2] * ang[2];
    var_phi += LT2 / (4.0 * R * R) * rel2;
  }
  const double pi2 = kPi * kPi;
  cov[0] = meas[2];                                                 // (l0, l0)
  cov[1] = meas[3];                                                 // (l0, l1)
  cov[5] = meas[4];                                                 // (l1, l1)
  cov[9] = std::fmin(var_phi, pi2);                                 // (phi, phi)
  cov[12] = std::fmin(16.0 * sh2 / L2 + 2.0 * ms2, pi2);            // (theta, theta)
  cov[14] = var_qop;                                                // (q/p, q/p)
}

// Seed parameters [n][5] and packed covariances [n][15] of every track from three of its
// measurements (first_three = 0: first, middle, last; 1: the first three); status [n] as in
// seed_track.
void orc_estimate_seeds(const double* surfaces, uint32_t n_surf, const orc_field* field, uint32_t n_tracks,
                        uint64_t n_meas, const uint32_t* offsets, const double* meas, const uint32_t* sid,
                        int first_three, double* seed_par, double* seed_cov, uint32_t* status) {
  std::vector<Surface> surf = to_surfaces(surfaces, n_surf);
  Field F = to_field(field);
  for (uint32_t i = 0; i < n_tracks; ++i) {
    const uint32_t a = offsets[i], b = offsets[i + 1];
    if (b < a || b > n_meas) {
      for (int j = 0; j < 5; ++j) seed_par[5 * size_t(i) + j] = std::nan("");
      for (int j = 0; j < 15; ++j) seed_cov[15 * size_t(i) + j] = 0.0;
      status[i] = 4;
      continue;
    }
    seed_track(surf.data(), n_surf, F, meas + 5 * size_t(a), sid + a, b - a, first_three, seed_par + 5 * size_t(i),
               seed_cov + 15 * size_t(i), status + i);
  }
}

// Track finding: for every seed (surface id, parameters [5], packed covariance [15]) the best
// candidate of the combinatorial Kalman filter. Measurements [n_meas][5] are grouped by surface:
// those of surface s are meas_off[s] .. meas_off[s+1]-1. Outputs per seed: entries (surface ids,
// with bit 31 for holes, and measurement indices or -1) [n_seeds][max_entries], the entry and
// measurement counts and the chi2 sum; 0 entries when the seed surface is out of range.
void orc_find_tracks(const double* surfaces, uint32_t n_surf, const orc_field* field, const orc_opts* opts,
                     const double* layers, uint32_t n_layers, const double* rings, uint32_t n_meas,
                     const uint32_t* meas_off, const double* meas, uint32_t n_seeds, const uint32_t* seed_sid,
                     const double* seed_par, const double* seed_cov, double chi2_max, uint32_t beam,
                     uint32_t max_holes, uint32_t max_entries, uint32_t* out_n_entries, uint32_t* out_n_meas,
                     double* out_chi2, uint32_t* out_sid, int32_t* out_meas, int n_threads) {
  (void)n_meas;
  std::vector<Surface> surf = to_surfaces(surfaces, n_surf);
  Field F = to_field(field);
  Mlp mlp_store;
  Opts O = to_opts(opts, &mlp_store);
  CkfLayers L{layers, n_layers, rings, {}};
  build_layer_of(L, n_surf);
  CkfOpts co{chi2_max, beam < 1 ? 1u : beam, max_holes,
             max_entries < 1 ? 1u : (max_entries > uint32_t(kCkfMaxEntries) ? uint32_t(kCkfMaxEntries) : max_entries)};
  auto work = [&](uint32_t lo, uint32_t hi) {
    for (uint32_t i = lo; i < hi; ++i) {
      Branch best;
      bool have = false;
      uint32_t* es = out_sid + size_t(i) * max_entries;
      int32_t* em = out_meas + size_t(i) * max_entries;
      for (uint32_t j = 0; j < max_entries; ++j) {
        es[j] = 0;
        em[j] = -1;
      }
      out_n_entries[i] = out_n_meas[i] = 0;
      out_chi2[i] = 0.0;
      if (seed_sid[i] >= n_surf) continue;
      find_track(surf.data(), n_surf, F, O, co, L, meas_off, meas, seed_sid[i], seed_par + 5 * size_t(i),
                 seed_cov + 15 * size_t(i), best, have);
      if (!have) continue;
      out_n_entries[i] = best.n_entries;
      out_n_meas[i] = best.n_meas;
      out_chi2[i] = best.chi2;
      for (uint32_t j = 0; j < best.n_entries && j < max_entries; ++j) {
        es[j] = best.e_sid[j];
        em[j] = best.e_meas[j];
      }
    }
  };
  int nt = std::max(1, n_threads);
  std::vector<std::thread> th;
  for (int t = 0; t < nt; ++t) th.emplace_back(work, uint32_t(uint64_t(n_seeds) * t / nt), uint32_t(uint64_t(n_seeds) * (t + 1) / nt));
  for (auto& t : th) t.join();
}

// The helix-through-three-points step alone (for the pins): phi, theta, q/p and the status.
uint32_t orc_helix_seed(const double* r1, const double* r2, const double* r3, double bz, double* out) {
  return helix_seed(r1, r2, r3, bz, out);
}

// One gain-matrix update (for the chi2 identity pin).
uint32_t orc_update(const double* m, const double* V, double* p, double* C, double* chi2) {
  return kf_update(m, V, p, C, chi2);
}

}  // extern "C"
