#pragma once
// tkf_fit_impl.cuh -- Kalman-filter fit kernels for GB300 (sm_103a), included by the per-precision
// translation units tkf_fit_fp64.cu and tkf_fit_mixed.cu.
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

constexpr uint32_t kFatal = ~(TKF_TRACK_TOO_FEW_HITS | TKF_TRACK_OUT_OF_FIELD | TKF_TRACK_PROPOSAL_FALLBACK);

// Exact FP32 <-> FP64 conversions on the integer pipes. On GB300 the hardware conversion runs
// on the FP64 pipe (a warp instruction occupies it for 16 SM cycles), and the FP64 pipe bounds
// the mixed path; these give the IEEE results (round to nearest even) for every normal number
// and zero with a few integer operations. FP32 denormals become signed zero; out of range
// FP64 values (beyond the FP32 normals, infinities, NaN) become NaN, and FP32 infinities and
// NaN become FP64 NaN, so a non-finite value stays non-finite.
__device__ __forceinline__ double f2d(float x) {
  const uint32_t u = __float_as_uint(x), a = u & 0x7FFFFFFFu;
  const bool tiny = a < 0x00800000u, special = a >= 0x7F800000u;
  const uint32_t hi = tiny ? 0u : (special ? 0x7FF80000u : (a >> 3) + (896u << 20));  // bias 127 -> 1023
  return __hiloint2double(int((u & 0x80000000u) | hi), int(tiny ? 0u : (u << 29)));
}

__device__ __forceinline__ float d2f(double x) {
  const uint32_t hi = uint32_t(__double2hiint(x)), lo = uint32_t(__double2loint(x)), a = hi & 0x7FFFFFFFu;
  uint32_t m = ((a - 0x38000000u) << 3) | (lo >> 29);  // bias 1023 -> 127, top 23 mantissa bits
  // round to nearest even on the 29 dropped bits: up if above half, or at half with m odd
  m += (lo >> 28) & ((lo & 0x0FFFFFFFu ? 1u : 0u) | m) & 1u;
  m = a < 0x38100000u ? 0u : (a >= 0x47F00000u ? 0x7FC00000u : m);
  return __uint_as_float((hi & 0x80000000u) | m);
}

// index of (i, j) in the packed row-major upper triangle of a symmetric 5x5 matrix
__host__ __device__ constexpr int S(int i, int j) { return i <= j ? i * (9 - i) / 2 + j : j * (9 - j) / 2 + i; }

struct Surf {
  double u[3], v[3], n[3], c[3], t, x0, t_x0;
  float uf[3], vf[3], nf[3], tf, t_x0f;  // FP32 copies (mixed path)
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
  const float4* q = reinterpret_cast<const float4*>(p + 8);
  const float4 f0 = __ldg(q), f1 = __ldg(q + 1), f2 = __ldg(q + 2);
  s.uf[0] = f0.x; s.uf[1] = f0.y; s.uf[2] = f0.z;
  s.vf[0] = f0.w; s.vf[1] = f1.x; s.vf[2] = f1.y;
  s.nf[0] = f1.z; s.nf[1] = f1.w; s.nf[2] = f2.x;
  s.tf = f2.y; s.t_x0f = f2.z;
}

// Frame vectors of a surface read again from its record after the propagation, so that they do
// not stay in registers across it (the fit's register budget is capped). The loads are volatile:
// the compiler may not reuse the values of the earlier load, which would keep them live.
__device__ __forceinline__ double2 ld_nc_d2(const double2* p) {
  double2 v;
  asm volatile("ld.global.nc.v2.f64 {%0, %1}, [%2];" : "=d"(v.x), "=d"(v.y) : "l"(p));
  return v;
}
__device__ __forceinline__ float4 ld_nc_f4(const float4* p) {
  float4 v;
  asm volatile("ld.global.nc.v4.f32 {%0, %1, %2, %3}, [%4];" : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w) : "l"(p));
  return v;
}
// u and v in FP64
__device__ __forceinline__ void reload_uv(const double* __restrict__ g, uint32_t id, double u[3], double v[3]) {
  const double2* p = reinterpret_cast<const double2*>(g + size_t(id) * kSurfStride);
  const double2 a0 = ld_nc_d2(p), a1 = ld_nc_d2(p + 1), a2 = ld_nc_d2(p + 2);
  u[0] = a0.x; u[1] = a0.y; u[2] = a1.x;
  v[0] = a1.y; v[1] = a2.x; v[2] = a2.y;
}
// u and v in FP32
__device__ __forceinline__ void reload_uvf(const double* __restrict__ g, uint32_t id, float u[3], float v[3]) {
  const float4* q = reinterpret_cast<const float4*>(g + size_t(id) * kSurfStride + 16);
  const float4 f0 = ld_nc_f4(q), f1 = ld_nc_f4(q + 1);
  u[0] = f0.x; u[1] = f0.y; u[2] = f0.z;
  v[0] = f0.w; v[1] = f1.x; v[2] = f1.y;
}

__device__ __forceinline__ double dot3(const double a[3], const double b[3]) {
  return a[0] * b[0] + a[1] * b[1] + a[2] * b[2];
}

// ------------------------------------------------------------------ field policies
// Uniform field along z (the solenoid axis): T x B has no z component, so T_z, and with it
// theta, is constant along the path: the theta row of the transport Jacobian of the motion is
// exactly e_3 (kAlongZ). The FP64 path keeps the derivative of the discrete RKN map (whose
// final normalisation of T moves that row by the integration error, ~1e-9); the mixed path,
// whose FP32 Jacobian carries ~1e-7 of rounding there, sets the row to e_3.
struct FieldUniformZ {
  double bz;
  float bzf;
  static constexpr bool kUniform = true;
  static constexpr bool kAlongZ = true;
  __device__ __forceinline__ void at(const double*, double B[3], bool&) const {
    B[0] = 0.0; B[1] = 0.0; B[2] = bz;
  }
  __device__ __forceinline__ void atf(const float*, float B[3], bool&) const {
    B[0] = 0.0f; B[1] = 0.0f; B[2] = bzf;
  }
};

struct FieldUniform {
  double b[3];
  float bf[3];
  static constexpr bool kUniform = true;
  static constexpr bool kAlongZ = false;
  __device__ __forceinline__ void at(const double*, double B[3], bool&) const {
    B[0] = b[0]; B[1] = b[1]; B[2] = b[2];
  }
  __device__ __forceinline__ void atf(const float*, float B[3], bool&) const {
    B[0] = bf[0]; B[1] = bf[1]; B[2] = bf[2];
  }
};

// Bilinear (r, z) interpolation of the (B_r, B_z) grid, FP64 arithmetic on FP32 nodes.
struct FieldGrid {
  const float2* __restrict__ grid;
  int nr, nz;
  double r0, z0, inv_dr, inv_dz;
  float r0f, z0f, inv_drf, inv_dzf, rmaxf, zmaxf;  // FP32 copies: origin, 1/spacing, nr-1, nz-1
  static constexpr bool kUniform = false;
  static constexpr bool kAlongZ = false;
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
  // the same interpolation in FP32 (mixed precision)
  __device__ __forceinline__ void atf(const float* x, float B[3], bool& oof) const {
    const float r = sqrtf(x[0] * x[0] + x[1] * x[1]);
    const float fr = (r - r0f) * inv_drf;
    const float fz = (x[2] - z0f) * inv_dzf;
    if (!(fr >= 0.0f && fr <= rmaxf && fz >= 0.0f && fz <= zmaxf)) {
      B[0] = B[1] = B[2] = 0.0f;
      oof = true;
      return;
    }
    const int ir = min(int(fr), nr - 2);
    const int iz = min(int(fz), nz - 2);
    const float a = fr - ir, b = fz - iz;
    const float2* g = grid + size_t(iz) * nr + ir;
    const float2 g00 = __ldg(g), g01 = __ldg(g + 1), g10 = __ldg(g + nr), g11 = __ldg(g + nr + 1);
    const float br = (1.0f - b) * ((1.0f - a) * g00.x + a * g01.x) + b * ((1.0f - a) * g10.x + a * g11.x);
    const float bz = (1.0f - b) * ((1.0f - a) * g00.y + a * g01.y) + b * ((1.0f - a) * g10.y + a * g11.y);
    const float q = r > 0.0f ? br / r : 0.0f;
    B[0] = q * x[0];
    B[1] = q * x[1];
    B[2] = bz;
  }
};

template <class R>
__device__ __forceinline__ R dotr(const R a[3], const R b[3]) {
  return a[0] * b[0] + a[1] * b[1] + a[2] * b[2];
}

__device__ __forceinline__ void cross(const float a[3], const float b[3], float o[3]) {
  o[0] = a[1] * b[2] - a[2] * b[1];
  o[1] = a[2] * b[0] - a[0] * b[2];
  o[2] = a[0] * b[1] - a[1] * b[0];
}

__device__ __forceinline__ void cross(const double a[3], const double b[3], double o[3]) {
  o[0] = a[1] * b[2] - a[2] * b[1];
  o[1] = a[2] * b[0] - a[0] * b[2];
  o[2] = a[0] * b[1] - a[1] * b[0];
}

// clamp(0.9 q^(1/4), lo, hi) with the quarter root as two square roots
__device__ __forceinline__ double step_factor(double q, double lo, double hi) {
  double f = 0.9 * sqrt(sqrt(q));
  return fmin(fmax(f, lo), hi);
}

// Path length to the plane along the parabola r + s T + s^2/2 k (a = n.T, b = n.k, d = n.(c - r)),
// the straight-line d / a when the parabola misses the plane.
__device__ __forceinline__ double parabolic_path(double d, double a, double b) {
  double s = d / a;
  const double disc = a * a + 2.0 * b * d;
  if (disc >= 0.0) {
    const double q = 2.0 * d / (a + copysign(sqrt(disc), a));
    if (isfinite(q)) s = q;
  }
  return s;
}

// ------------------------------------------------------------------ learned step proposer
// Network inputs at the start of a step (FP32): u, v, n components of (r - c) / 1000 mm, of the
// direction, q/p, B / 2 T, ln(last step / mm) / 5, straight-line path / 1000 mm in [-2, 2].
__device__ __forceinline__ void mlp_features(const Surf& s, const double r[3], const float Tf[3], double lam,
                                             const float B[3], float h_last, float sl, float x[12]) {
  const float d[3] = {float(r[0] - s.c[0]), float(r[1] - s.c[1]), float(r[2] - s.c[2])};
  const float* u = s.uf;
  const float* v = s.vf;
  const float* n = s.nf;
  x[0] = (u[0] * d[0] + u[1] * d[1] + u[2] * d[2]) * 1e-3f;
  x[1] = (v[0] * d[0] + v[1] * d[1] + v[2] * d[2]) * 1e-3f;
  x[2] = (n[0] * d[0] + n[1] * d[1] + n[2] * d[2]) * 1e-3f;
  x[3] = u[0] * Tf[0] + u[1] * Tf[1] + u[2] * Tf[2];
  x[4] = v[0] * Tf[0] + v[1] * Tf[1] + v[2] * Tf[2];
  x[5] = n[0] * Tf[0] + n[1] * Tf[1] + n[2] * Tf[2];
  x[6] = float(lam);
  x[7] = B[0] * 0.5f;
  x[8] = B[1] * 0.5f;
  x[9] = B[2] * 0.5f;
  x[10] = logf(h_last) * 0.2f;
  x[11] = fminf(fmaxf(sl * 1e-3f, -2.0f), 2.0f);
}

// SiLU z sigmoid(z) with the fast exponential and division (a few ulp; the proposal grid
// absorbs the difference from the exactly rounded form)
__device__ __forceinline__ float silu_f(float z) { return __fdividef(z, 1.0f + __expf(-z)); }

// Step modes: plain adaptive control, learned proposals, or plain control with record capture.
constexpr int kPlain = 0, kLearned = 1, kRecord = 2;
// kStates: plain adaptive stepping that also stores every entry's filtered state (into the
// caller's all-states arrays) and predicted state with its transport Jacobian (into the
// workspace), for the backward RTS pass of tkf_states.cu.
constexpr int kStates = 3;

// Where learned proposals and training records go during one track's propagation.
struct StepLearn {
  float* rec;             // record buffer, or null
  uint32_t rec_cap;
  uint32_t* rec_count;
  float h_last;           // last accepted step (network input), per track
};

__device__ __forceinline__ void put_record(StepLearn& L, const float x[12], float label) {
  const uint32_t k = atomicAdd(L.rec_count, 1u);
  if (k < L.rec_cap) {
    float* o = L.rec + size_t(k) * kMlpRecord;
#pragma unroll
    for (int i = 0; i < 12; ++i) o[i] = x[i];
    o[12] = label;
  }
}

// ------------------------------------------------------------------ propagation
// Adaptive RKN4 stepping of (r, T, lam) to the plane of `s`, transporting the derivative
// columns of (phi, theta, q/p): dr[c], dT[c] (c = 0, 1, 2); a lane of a group-per-track fit
// carries one column (kCols = 1), with qcol = 1 for the q/p column (whose source term adds
// T x kappa B) and 0 otherwise, and steps the state like the other lanes of its group. Step control (Lund 2009a, safety
// factor 0.9): eps = h^2 |k1 - k2 - k3 + k4|_1; eps > tol rejects and sets
// h_ctrl = |h| clamp(0.9 (tol/eps)^1/4, 1/4, 4); an accepted step limited by h_ctrl sets
// h_ctrl = min(h_max, h_ctrl clamp(0.9 (tol/eps)^1/4, 1/4, 4)). Each step aims at the plane's
// intersection with the parabola r + s T + s^2/2 k1; within surf_tol a second-order Taylor
// step (state and columns) lands on the plane.
template <int kMode, int kCols, class F>
__device__ uint32_t propagate(const F& fld, const OptionsDev& o, const Surf& s, double r[3], double T[3],
                              double lam, double dr[kCols][3], double dT[kCols][3], double qcol, double& h_ctrl,
                              uint32_t& attempts, uint32_t& rejected, double kend[3], StepLearn& L) {
  uint32_t st = 0;
  bool first = true;
  uint32_t n_here = 0;
  const double lk = lam * kKappa;
  for (;;) {
    const double dist = s.n[0] * (s.c[0] - r[0]) + s.n[1] * (s.c[1] - r[1]) + s.n[2] * (s.c[2] - r[2]);
    const double a = dot3(s.n, T);
    bool oof = false;
    double B1[3], Bt1[3], k1[3];
    fld.at(r, B1, oof);
    for (int i = 0; i < 3; ++i) Bt1[i] = lk * B1[i];
    cross(T, Bt1, k1);
    if (fabs(dist) <= o.surf_tol) {
      // second-order Taylor step onto the plane, with the derivative columns
      if (oof) st |= TKF_TRACK_OUT_OF_FIELD;
      const double sp = parabolic_path(dist, a, dot3(s.n, k1)), sp2 = 0.5 * sp * sp;
#pragma unroll
      for (int c = 0; c < kCols; ++c) {
        double q[3];
        cross(dT[c], Bt1, q);
        if (kCols == 1 || c == 2) {
          double e[3], Bk[3] = {kKappa * B1[0], kKappa * B1[1], kKappa * B1[2]};
          cross(T, Bk, e);
          for (int i = 0; i < 3; ++i) q[i] += kCols == 1 ? qcol * e[i] : e[i];
        }
        for (int i = 0; i < 3; ++i) {
          dr[c][i] += sp * dT[c][i] + sp2 * q[i];
          dT[c][i] += sp * q[i];
        }
      }
      for (int i = 0; i < 3; ++i) {
        r[i] += sp * T[i] + sp2 * k1[i];
        T[i] += sp * k1[i];
      }
      break;
    }
    const double sl = dist / a;
    if (first && !(sl > -1.0 && isfinite(sl))) return st | TKF_TRACK_SURFACE_MISSED;
    first = false;
    if (n_here >= o.max_steps) return st | TKF_TRACK_MAX_STEPS;
    ++n_here;
    ++attempts;
    const double sp = parabolic_path(dist, a, dot3(s.n, k1));
    float x[kMode == kRecord ? 12 : 1];
    if constexpr (kMode == kRecord) {
      const float Tf[3] = {float(T[0]), float(T[1]), float(T[2])};
      const float Bf[3] = {float(B1[0]), float(B1[1]), float(B1[2])};
      mlp_features(s, r, Tf, lam, Bf, L.h_last, float(sl), x);
    }
    const double limit = h_ctrl;
    const bool limited = !(fabs(sp) < limit);
    const double h = limited ? copysign(limit, sp) : sp;
    const double h2 = 0.5 * h, h6 = h * (1.0 / 6.0);
    double B2[3], B4[3], Bt2[3], Bt4[3];
    double k2[3], k3[3], k4[3], T2[3], T3[3], T4[3];
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
      h_ctrl = fabs(h) * step_factor(o.tol / eps, 0.25, 4.0);
      if (h_ctrl < o.h_min) return st | TKF_TRACK_STEP_UNDERFLOW;
      continue;
    }
    if (oof) st |= TKF_TRACK_OUT_OF_FIELD;
    if constexpr (kMode == kRecord)  // steps the control limited: the proposals' domain
      if (limited && eps > 0.0) put_record(L, x, float(log(fabs(h) * sqrt(sqrt(o.tol / eps)))));
    // derivative columns through the accepted step (dB/dr neglected)
#pragma unroll
    for (int c = 0; c < kCols; ++c) {
      double q1[3], q2[3], q3[3], q4[3], u2[3], u3[3], u4[3];
      cross(dT[c], Bt1, q1);
      if (kCols == 1 || c == 2) {
        double e[3];
        double Bk1[3] = {kKappa * B1[0], kKappa * B1[1], kKappa * B1[2]};
        cross(T, Bk1, e);
        for (int i = 0; i < 3; ++i) q1[i] += kCols == 1 ? qcol * e[i] : e[i];
      }
      for (int i = 0; i < 3; ++i) u2[i] = dT[c][i] + h2 * q1[i];
      cross(u2, Bt2, q2);
      if (kCols == 1 || c == 2) {
        double e[3];
        double Bk2[3] = {kKappa * B2[0], kKappa * B2[1], kKappa * B2[2]};
        cross(T2, Bk2, e);
        for (int i = 0; i < 3; ++i) q2[i] += kCols == 1 ? qcol * e[i] : e[i];
      }
      for (int i = 0; i < 3; ++i) u3[i] = dT[c][i] + h2 * q2[i];
      cross(u3, Bt2, q3);
      if (kCols == 1 || c == 2) {
        double e[3];
        double Bk2[3] = {kKappa * B2[0], kKappa * B2[1], kKappa * B2[2]};
        cross(T3, Bk2, e);
        for (int i = 0; i < 3; ++i) q3[i] += kCols == 1 ? qcol * e[i] : e[i];
      }
      for (int i = 0; i < 3; ++i) u4[i] = dT[c][i] + h * q3[i];
      cross(u4, Bt4, q4);
      if (kCols == 1 || c == 2) {
        double e[3];
        double Bk4[3] = {kKappa * B4[0], kKappa * B4[1], kKappa * B4[2]};
        cross(T4, Bk4, e);
        for (int i = 0; i < 3; ++i) q4[i] += kCols == 1 ? qcol * e[i] : e[i];
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
      const double fac = (eps > 0.0) ? step_factor(o.tol / eps, 0.25, 4.0) : 4.0;
      h_ctrl = fmin(o.h_max, fabs(h) * fac);
    }
    if constexpr (kMode == kRecord) L.h_last = float(fabs(h));
  }
  double B[3], Bt[3];
  bool oof = false;
  fld.at(r, B, oof);
  if (oof) st |= TKF_TRACK_OUT_OF_FIELD;
  for (int i = 0; i < 3; ++i) Bt[i] = lk * B[i];
  cross(T, Bt, kend);
  return st;
}

// ------------------------------------------------------------------ propagation, mixed precision
// The same stepping, step control and targeting with the stage derivatives, the error estimate,
// the step control and the derivative columns in FP32; the position and direction are FP64
// anchors that accumulate each accepted step's FP32 increments, and the distance to the plane
// is taken in FP64 (sub-micron landing at metre-scale coordinates).
__device__ __forceinline__ float step_factor_f(float q) {
  return fminf(fmaxf(0.9f * sqrtf(sqrtf(q)), 0.25f), 4.0f);
}

__device__ __forceinline__ float parabolic_path_f(float d, float a, float b) {
  float s = d / a;
  const float disc = a * a + 2.0f * b * d;
  if (disc >= 0.0f) {
    const float q = 2.0f * d / (a + copysignf(sqrtf(disc), a));
    if (isfinite(q)) s = q;
  }
  return s;
}

// kRoll: the derivative-column loops are kept rolled (smaller code; the 64-register kernel,
// whose column state is in local memory anyway, runs faster so: measured).
template <int kMode, int kCols, class F, bool kRoll = false>
__device__ uint32_t propagate_mixed(const F& fld, const OptionsDev& o, const Surf& s, const float nf[3], double r[3],
                                    double T[3], double lam, float dr[kCols][3], float dT[kCols][3], float qcol,
                                    float& h_ctrl,
                                    uint32_t& attempts, uint32_t& rejected, float kend[3], StepLearn& L) {
  uint32_t st = 0;
  bool first = true;
  uint32_t n_here = 0;
  const float lk = d2f(lam * kKappa);
  const float tol = o.tol_f, h_min = o.h_min_f, h_max = o.h_max_f, surf_tol = o.surf_tol_f;
  for (;;) {
    const double dist = s.n[0] * (s.c[0] - r[0]) + s.n[1] * (s.c[1] - r[1]) + s.n[2] * (s.c[2] - r[2]);
    const float Tf[3] = {d2f(T[0]), d2f(T[1]), d2f(T[2])};
    float rf[3] = {0.0f, 0.0f, 0.0f};
    if (!F::kUniform || kMode == kRecord)
      for (int i = 0; i < 3; ++i) rf[i] = d2f(r[i]);
    const float a = dotr(nf, Tf), df = d2f(dist);
    bool oof = false;
    float B1[3], Bt1[3], k1[3];
    fld.atf(rf, B1, oof);
    for (int i = 0; i < 3; ++i) Bt1[i] = lk * B1[i];
    cross(Tf, Bt1, k1);
    if (fabsf(df) <= surf_tol) {
      if (oof) st |= TKF_TRACK_OUT_OF_FIELD;
      const float sp = parabolic_path_f(df, a, dotr(nf, k1)), sp2 = 0.5f * sp * sp;
#pragma unroll(kRoll ? 1 : kCols)
      for (int c = 0; c < kCols; ++c) {
        float q[3];
        cross(dT[c], Bt1, q);
        if (kCols == 1 || c == 2) {
          float e[3], Bk[3] = {float(kKappa) * B1[0], float(kKappa) * B1[1], float(kKappa) * B1[2]};
          cross(Tf, Bk, e);
          for (int i = 0; i < 3; ++i) q[i] += kCols == 1 ? qcol * e[i] : e[i];
        }
        for (int i = 0; i < 3; ++i) {
          dr[c][i] += sp * dT[c][i] + sp2 * q[i];
          dT[c][i] += sp * q[i];
        }
      }
      const double spd = f2d(sp);
      for (int i = 0; i < 3; ++i) {
        r[i] += spd * T[i] + f2d(sp2 * k1[i]);
        T[i] += f2d(sp * k1[i]);
      }
      break;
    }
    const float sl = df / a;
    if (first && !(sl > -1.0f && isfinite(sl))) return st | TKF_TRACK_SURFACE_MISSED;
    first = false;
    if (n_here >= o.max_steps) return st | TKF_TRACK_MAX_STEPS;
    ++n_here;
    ++attempts;
    const float sp = parabolic_path_f(df, a, dotr(nf, k1));
    float x[kMode == kRecord ? 12 : 1];
    if constexpr (kMode == kRecord) mlp_features(s, r, Tf, lam, B1, L.h_last, sl, x);
    const float limit = h_ctrl;
    const bool limited = !(fabsf(sp) < limit);
    const float h = limited ? copysignf(limit, sp) : sp;
    const float h2 = 0.5f * h, h6 = h * (1.0f / 6.0f);
    float B2[3], B4[3], Bt2[3], Bt4[3], k2[3], k3[3], k4[3], T2[3], T3[3], T4[3];
    if (F::kUniform) {
      for (int i = 0; i < 3; ++i) { B2[i] = B1[i]; Bt2[i] = Bt1[i]; }
    } else {
      float r2[3];
      for (int i = 0; i < 3; ++i) r2[i] = rf[i] + h2 * Tf[i] + 0.125f * h * h * k1[i];
      fld.atf(r2, B2, oof);
      for (int i = 0; i < 3; ++i) Bt2[i] = lk * B2[i];
    }
    for (int i = 0; i < 3; ++i) T2[i] = Tf[i] + h2 * k1[i];
    cross(T2, Bt2, k2);
    for (int i = 0; i < 3; ++i) T3[i] = Tf[i] + h2 * k2[i];
    cross(T3, Bt2, k3);
    if (F::kUniform) {
      for (int i = 0; i < 3; ++i) { B4[i] = B1[i]; Bt4[i] = Bt1[i]; }
    } else {
      float r4[3];
      for (int i = 0; i < 3; ++i) r4[i] = rf[i] + h * Tf[i] + 0.5f * h * h * k3[i];
      fld.atf(r4, B4, oof);
      for (int i = 0; i < 3; ++i) Bt4[i] = lk * B4[i];
    }
    for (int i = 0; i < 3; ++i) T4[i] = Tf[i] + h * k3[i];
    cross(T4, Bt4, k4);
    float eps = 0.0f;
    for (int i = 0; i < 3; ++i) eps += fabsf(k1[i] - k2[i] - k3[i] + k4[i]);
    eps *= h * h;
    if (eps > tol) {
      ++rejected;
      h_ctrl = fabsf(h) * step_factor_f(tol / eps);
      if (h_ctrl < h_min) return st | TKF_TRACK_STEP_UNDERFLOW;
      continue;
    }
    if (oof) st |= TKF_TRACK_OUT_OF_FIELD;
    if constexpr (kMode == kRecord)  // steps the control limited: the proposals' domain
      if (limited && eps > 0.0f) put_record(L, x, logf(fabsf(h) * sqrtf(sqrtf(tol / eps))));
#pragma unroll(kRoll ? 1 : kCols)
    for (int c = 0; c < kCols; ++c) {
      float q1[3], q2[3], q3[3], q4[3], u2[3], u3[3], u4[3];
      cross(dT[c], Bt1, q1);
      if (kCols == 1 || c == 2) {
        float e[3], Bk[3] = {float(kKappa) * B1[0], float(kKappa) * B1[1], float(kKappa) * B1[2]};
        cross(Tf, Bk, e);
        for (int i = 0; i < 3; ++i) q1[i] += kCols == 1 ? qcol * e[i] : e[i];
      }
      for (int i = 0; i < 3; ++i) u2[i] = dT[c][i] + h2 * q1[i];
      cross(u2, Bt2, q2);
      if (kCols == 1 || c == 2) {
        float e[3], Bk[3] = {float(kKappa) * B2[0], float(kKappa) * B2[1], float(kKappa) * B2[2]};
        cross(T2, Bk, e);
        for (int i = 0; i < 3; ++i) q2[i] += kCols == 1 ? qcol * e[i] : e[i];
      }
      for (int i = 0; i < 3; ++i) u3[i] = dT[c][i] + h2 * q2[i];
      cross(u3, Bt2, q3);
      if (kCols == 1 || c == 2) {
        float e[3], Bk[3] = {float(kKappa) * B2[0], float(kKappa) * B2[1], float(kKappa) * B2[2]};
        cross(T3, Bk, e);
        for (int i = 0; i < 3; ++i) q3[i] += kCols == 1 ? qcol * e[i] : e[i];
      }
      for (int i = 0; i < 3; ++i) u4[i] = dT[c][i] + h * q3[i];
      cross(u4, Bt4, q4);
      if (kCols == 1 || c == 2) {
        float e[3], Bk[3] = {float(kKappa) * B4[0], float(kKappa) * B4[1], float(kKappa) * B4[2]};
        cross(T4, Bk, e);
        for (int i = 0; i < 3; ++i) q4[i] += kCols == 1 ? qcol * e[i] : e[i];
      }
      for (int i = 0; i < 3; ++i) {
        dr[c][i] += h * dT[c][i] + h * h6 * (q1[i] + q2[i] + q3[i]);
        dT[c][i] += h6 * (q1[i] + 2.0f * q2[i] + 2.0f * q3[i] + q4[i]);
      }
    }
    const double hd = f2d(h);
    for (int i = 0; i < 3; ++i) {
      r[i] += hd * T[i] + f2d(h * h6 * (k1[i] + k2[i] + k3[i]));
      T[i] += f2d(h6 * (k1[i] + 2.0f * k2[i] + 2.0f * k3[i] + k4[i]));
    }
    if (limited) {
      const float fac = (eps > 0.0f) ? step_factor_f(tol / eps) : 4.0f;
      h_ctrl = fminf(h_max, fabsf(h) * fac);
    }
    if constexpr (kMode == kRecord) L.h_last = fabsf(h);
  }
  float B[3], Bt[3];
  bool oof = false;
  float rf[3] = {0.0f, 0.0f, 0.0f};
  if (!F::kUniform)
    for (int i = 0; i < 3; ++i) rf[i] = d2f(r[i]);
  const float Tf[3] = {d2f(T[0]), d2f(T[1]), d2f(T[2])};
  fld.atf(rf, B, oof);
  if (oof) st |= TKF_TRACK_OUT_OF_FIELD;
  for (int i = 0; i < 3; ++i) Bt[i] = lk * B[i];
  cross(Tf, Bt, kend);
  return st;
}

// ------------------------------------------------------------------ material
// Thin layer at surface s crossed with unit direction T: returns theta0^2 (Highland) and lowers
// |q/p| by the Bethe mean loss (density effect: high-energy asymptote). With p^2 = 1/lam^2:
//   1/(beta p) = E lam^2,  1/beta^2 = 1 + m^2 lam^2,  beta^2 gamma^2 = p^2 / m^2.
// Above beta gamma = exp(1/2 - ln(hbar omega_p / I)) the density term cancels ln(beta gamma) and
// the Bethe bracket needs one logarithm: 1/2 ln(2 m_e W_max / I^2) - ln(hbar omega_p / I) + 1/2 - beta^2.
// kGain: the reversed particle of the backward filter crosses the layer against the flight
// direction and regains the mean loss (theta0 and the loss at its momentum on arrival).
template <bool kGain = false>
__device__ __forceinline__ uint32_t material(const Surf& s, const MaterialDev& m, double mass, const double T[3],
                                             double& lam, double& th0sq) {
  th0sq = 0.0;
  if (!(s.t > 0.0)) return 0;
  const double inv_cos = 1.0 / fabs(dot3(s.n, T));
  const double x = s.t * inv_cos, xx0 = s.t_x0 * inv_cos;
  const double l2 = lam * lam;
  const double p2 = 1.0 / l2;
  const double m2 = mass * mass;
  const double E2 = p2 + m2, E = sqrt(E2);
  const double inv_beta2 = 1.0 + m2 * l2;
  const double beta2 = 1.0 / inv_beta2;
  const double hl = 1.0 + 0.038 * log(xx0 * inv_beta2);
  const double a = 0.0136 * E * l2;
  th0sq = a * a * xx0 * hl * hl;
  const double bg2 = p2 / m2;
  const double me_m = kMe / mass;
  const double wmax = 2.0 * kMe * bg2 / (1.0 + 2.0 * (E / mass) * me_m + me_m * me_m);
  const double I = m.i_ev * 1e-9;
  double bracket;
  if (bg2 > m.bg2_density)  // density term active: ln(beta gamma) cancels
    bracket = 0.5 * log(2.0 * kMe * wmax / (I * I)) - m.log_hwp_over_i + 0.5 - beta2;
  else
    bracket = 0.5 * log(2.0 * kMe * bg2 * wmax / (I * I)) - beta2;
  const double dedx = kBetheK * m.z_over_a * inv_beta2 * bracket;
  const double dE = dedx * m.rho * x * 1e-4;  // MeV cm^2/g * g/cm^3 * mm -> GeV
  const double Ef = kGain ? E + dE : E - dE;
  if (!(Ef > mass)) return TKF_TRACK_PARTICLE_STOPPED;
  lam = copysign(1.0 / sqrt((Ef - mass) * (Ef + mass)), lam);
  return 0;
}

// Material in mixed precision: theta0^2 and the mean loss dE in FP32; the new q/p as
// lam (1 - delta)^(-1/2) with delta = (2 E dE - dE^2) lam^2, i.e. lam + lam g in FP64 where
// g = (1 - delta)^(-1/2) - 1 is formed in FP32 (series for small delta).
// kGain as for `material`: delta = -(2 E dE + dE^2) lam^2 < 0.
template <bool kGain = false>
__device__ __forceinline__ uint32_t material_mixed(const Surf& s, const MaterialDev& m, const OptionsDev& o,
                                                   const float T[3], double& lam, float& th0sq) {
  th0sq = 0.0f;
  if (!(s.tf > 0.0f)) return 0;
  const float mass = o.mass_f;
  const float inv_cos = 1.0f / fabsf(dotr(s.nf, T));
  const float x = s.tf * inv_cos, xx0 = s.t_x0f * inv_cos;
  const float lf = d2f(lam), l2 = lf * lf;
  const float p2 = 1.0f / l2, m2 = mass * mass;
  const float E = sqrtf(p2 + m2);
  const float inv_beta2 = 1.0f + m2 * l2, beta2 = 1.0f / inv_beta2;
  const float hl = 1.0f + 0.038f * logf(xx0 * inv_beta2);
  const float aa = 0.0136f * E * l2;
  th0sq = aa * aa * xx0 * hl * hl;
  const float bg2 = p2 / m2;
  const float me_m = o.me_over_mass_f;
  const float wmax = 2.0f * float(kMe) * bg2 / (1.0f + 2.0f * (E / mass) * me_m + me_m * me_m);
  float bracket;
  if (bg2 > m.bg2_density_f)
    bracket = 0.5f * logf(m.two_me_over_i2_f * wmax) - m.log_hwp_over_i_f + 0.5f - beta2;
  else
    bracket = 0.5f * logf(m.two_me_over_i2_f * bg2 * wmax) - beta2;
  const float dE = m.dedx_scale_f * inv_beta2 * bracket * x;
  if (!kGain && !(dE < E - mass)) return TKF_TRACK_PARTICLE_STOPPED;
  const float delta = kGain ? -(2.0f * E * dE + dE * dE) * l2 : (2.0f * E * dE - dE * dE) * l2;
  const float g = (kGain ? fabsf(delta) < 0.01f : delta < 0.01f)
                      ? delta * (0.5f + delta * (0.375f + delta * (0.3125f + delta * (0.2734375f + delta * 0.24609375f))))
                      : rsqrtf(1.0f - delta) - 1.0f;
  lam += lam * f2d(g);
  return 0;
}

// sin and cos of a small angle: Taylor polynomials through x^9 / x^8 (truncation below
// 1e-19 for |x| < 1/16), else the library sincos.
__device__ __forceinline__ void small_sincos(double x, double& s, double& c) {
  if (fabs(x) < 0.0625) {
    const double x2 = x * x;
    s = x * (1.0 + x2 * (-1.0 / 6 + x2 * (1.0 / 120 + x2 * (-1.0 / 5040 + x2 * (1.0 / 362880)))));
    c = 1.0 + x2 * (-0.5 + x2 * (1.0 / 24 + x2 * (-1.0 / 720 + x2 * (1.0 / 40320 - x2 * (1.0 / 3628800)))));
  } else {
    sincos(x, &s, &c);
  }
}

// sin x and cos x - 1 of a small angle in FP32 (absolute errors ~1e-8 |x| and ~1e-8 x^2),
// FP64 sincos above 1/16.
__device__ __forceinline__ void small_sincos_m1(double x, double& s, double& cm1) {
  const float xf = d2f(x);
  if (fabsf(xf) < 0.0625f) {
    const float h = sinf(0.5f * xf);
    s = f2d(sinf(xf));
    cm1 = f2d(-2.0f * h * h);
  } else {
    double c;
    sincos(x, &s, &c);
    cm1 = c - 1.0;
  }
}

// ------------------------------------------------------------------ fit of one track
// For k >= 1 the absolute angles are never output, so the filtered direction is carried as
// (sin phi, cos phi, sin theta, cos theta): the predicted values come from the propagated
// direction and the update's increments are applied by the angle-addition identities.
// Smoother state of one track (P = G_k C_k|k, the smoothed sums E and dl): 45 doubles that
// are read and written once per measurement. kPlace 0 keeps them in registers (spilled to
// local memory when the register cap is low); 1 puts P, and 2 all of them, in this thread's
// slot of shared memory (an odd number of doubles a slot, so a warp's accesses hit distinct
// bank pairs), which frees registers for a register-capped kernel.
template <int kPlace, class U>
struct SmootherStore {
  U P_[25], E_[15];
  double dl_[5];
  __device__ __forceinline__ U& P(int r, int c) { return P_[r * 5 + c]; }
  __device__ __forceinline__ U& E(int j) { return E_[j]; }
  __device__ __forceinline__ double& dl(int j) { return dl_[j]; }
};
template <>
struct SmootherStore<1, double> {
  double* s;  // 25 doubles
  double E_[15], dl_[5];
  __device__ __forceinline__ double& P(int r, int c) { return s[r * 5 + c]; }
  __device__ __forceinline__ double& E(int j) { return E_[j]; }
  __device__ __forceinline__ double& dl(int j) { return dl_[j]; }
};
template <>
struct SmootherStore<2, double> {
  double* s;  // 45 doubles
  __device__ __forceinline__ double& P(int r, int c) { return s[r * 5 + c]; }
  __device__ __forceinline__ double& E(int j) { return s[25 + j]; }
  __device__ __forceinline__ double& dl(int j) { return s[40 + j]; }
};

// Precision of the covariance algebra (Joseph update, smoother, covariance transport results):
// FP64 in the FP64 (kPrec 0) and mixed (kPrec 1) paths, FP32 in the experimental kPrec 2.
template <int kPrec>
struct CovType {
  using type = double;
};
template <>
struct CovType<2> {
  using type = float;
};
template <class U>
__device__ __forceinline__ U cov_from_d(double x);
template <>
__device__ __forceinline__ double cov_from_d<double>(double x) { return x; }
template <>
__device__ __forceinline__ float cov_from_d<float>(double x) { return d2f(x); }
template <class U>
__device__ __forceinline__ U cov_from_f(float x);
template <>
__device__ __forceinline__ double cov_from_f<double>(float x) { return f2d(x); }
template <>
__device__ __forceinline__ float cov_from_f<float>(float x) { return x; }
__device__ __forceinline__ double cov_to_d(double x) { return x; }
__device__ __forceinline__ double cov_to_d(float x) { return f2d(x); }
__device__ __forceinline__ float cov_to_f(double x) { return d2f(x); }
__device__ __forceinline__ float cov_to_f(float x) { return x; }

// acc - (a0 b0 + a1 b1) as two fused multiply-adds (no separate multiply and add).
__device__ __forceinline__ double sub2(double acc, double a0, double b0, double a1, double b1) {
  return fma(-a1, b1, fma(-a0, b0, acc));
}
__device__ __forceinline__ float sub2(float acc, float a0, float b0, float a1, float b1) {
  return fmaf(-a1, b1, fmaf(-a0, b0, acc));
}
// acc + (a0 b0 + a1 b1) into an FP64 accumulator: fused in FP64, or the FP32 sum added.
__device__ __forceinline__ double add2d(double acc, double a0, double b0, double a1, double b1) {
  return fma(a1, b1, fma(a0, b0, acc));
}
__device__ __forceinline__ double add2d(double acc, float a0, float b0, float a1, float b1) {
  return acc + f2d(a0 * b0 + a1 * b1);
}

__host__ __device__ constexpr int state_doubles(int place) { return place == 0 ? 0 : (place == 1 ? 25 : 45); }

// ------------------------------------------------------------------ group-per-track helpers
// A group of kG lanes may share one track (kG = 4): every lane steps the state, the update and
// the smoother identically (same data, same instructions, so the group never diverges), lane g
// of the group transports derivative column g (g < 3), and lane r computes row r of the
// covariance transport J (C + Q) J^T; shuffles within the group (width kG) assemble the full
// Jacobian and covariance in every lane. Each element is computed by the same operations in the
// same order as in the one-lane-per-track fit, so both give identical results.
template <int kG, class T>
__device__ __forceinline__ T gshfl(uint32_t gmask, T v, int src) {
  if constexpr (kG == 1) {
    return v;
  } else {
    return __shfl_sync(gmask, v, src, kG);
  }
}

// a[gl] for a lane index gl in 0..3, by selects (no dynamic register indexing)
template <class T>
__device__ __forceinline__ T pick4(uint32_t gl, T a0, T a1, T a2, T a3) {
  return gl == 0 ? a0 : (gl == 1 ? a1 : (gl == 2 ? a2 : a3));
}

// Rows 0..3 of one Jacobian column at the target: the derivative (x, t) of position and
// direction, moved along T to the plane (path correction), in the target's bound frame.
template <class R>
__device__ __forceinline__ void jac_column(const R n[3], const R u[3], const R v[3], const R T[3], const R kend[3],
                                           R inv_nT, R sp2, R cp2, R st2, R ct2, R inv_st, R x[3], R t[3],
                                           R out[4]) {
  const R ds = -dotr(n, x) * inv_nT;
  for (int j = 0; j < 3; ++j) {
    x[j] += T[j] * ds;
    t[j] += kend[j] * ds;
  }
  out[0] = dotr(u, x);
  out[1] = dotr(v, x);
  out[2] = (-sp2 * t[0] + cp2 * t[1]) * inv_st;
  out[3] = ct2 * cp2 * t[0] + ct2 * sp2 * t[1] - st2 * t[2];
}

// C <- J C J^T for the 5x5 packed symmetric C (J row 4 = e_4), over rows 0..3 of J; with kG = 4
// lane gl computes row gl and the group exchanges the results.
// kZ: row 3 of J is e_3 (theta conserved, a field along z): that row and column are copies.
template <int kG, class R, bool kZ = false>
__device__ __forceinline__ void transport_cov(const R J[5][5], R Cw[15], uint32_t gl, uint32_t gmask) {
  if constexpr (kG == 1) {
    R M[5][5];
#pragma unroll
    for (int r0 = 0; r0 < 4; ++r0)
#pragma unroll
      for (int c0 = 0; c0 < 5; ++c0) {
        if (kZ && r0 == 3) {
          M[3][c0] = Cw[S(3, c0)];
          continue;
        }
        R acc = R(0);
#pragma unroll
        for (int q = 0; q < 5; ++q) acc += J[r0][q] * Cw[S(q, c0)];
        M[r0][c0] = acc;
      }
#pragma unroll
    for (int c0 = 0; c0 < 5; ++c0) M[4][c0] = Cw[S(4, c0)];
#pragma unroll
    for (int r0 = 0; r0 < 5; ++r0)
#pragma unroll
      for (int c0 = r0; c0 < 5; ++c0) {
        R acc;
        if (c0 == 4) {
          acc = M[r0][4];
        } else if (kZ && c0 == 3) {
          acc = M[r0][3];
        } else {
          acc = R(0);
#pragma unroll
          for (int q = 0; q < 5; ++q) acc += M[r0][q] * J[c0][q];
        }
        Cw[S(r0, c0)] = acc;
      }
  } else {
    static_assert(kG == 4, "groups of 4 lanes");
    R Jr[5], Mr[5], Cr[5];
#pragma unroll
    for (int q = 0; q < 5; ++q) Jr[q] = pick4(gl, J[0][q], J[1][q], J[2][q], J[3][q]);
#pragma unroll
    for (int c0 = 0; c0 < 5; ++c0) {
      R acc = R(0);
#pragma unroll
      for (int q = 0; q < 5; ++q) acc += Jr[q] * Cw[S(q, c0)];
      Mr[c0] = acc;
    }
#pragma unroll
    for (int c0 = 0; c0 < 4; ++c0) {
      R acc = R(0);
#pragma unroll
      for (int q = 0; q < 5; ++q) acc += Mr[q] * J[c0][q];
      Cr[c0] = acc;
    }
    Cr[4] = Mr[4];
#pragma unroll
    for (int r0 = 0; r0 < 4; ++r0)
#pragma unroll
      for (int c0 = r0; c0 < 5; ++c0) Cw[S(r0, c0)] = gshfl<kG>(gmask, Cr[c0], r0);
  }
}

// ---- gain-matrix update with H = [I2 0]; Joseph form (paper Sec. 2; Fruhwirth 1987), with the
// measurement of entry m: sets the gain K, the inverse residual covariance Si and the residual r,
// updates p and C and adds r^T Si r to chi2. Returns TKF_TRACK_UPDATE_NOT_SPD (state untouched)
// when the residual covariance is not positive definite.
template <int kG, class U>
__device__ __forceinline__ uint32_t kalman_update(const FitArgs& a, uint32_t m, double p[5], U C[15], U K[5][2],
                                                  U& Si00, U& Si01, U& Si11, U& r0, U& r1, double& chi2,
                                                  uint32_t gl, uint32_t gmask) {
  const double m0 = a.loc0[m], m1 = a.loc1[m];
  const U V00 = cov_from_d<U>(a.v00[m]), V01 = cov_from_d<U>(a.v01[m]), V11 = cov_from_d<U>(a.v11[m]);
  const U S00 = C[S(0, 0)] + V00, S01 = C[S(0, 1)] + V01, S11 = C[S(1, 1)] + V11;
  const U det = S00 * S11 - S01 * S01;
  if (!(S00 > U(0) && det > U(0))) return TKF_TRACK_UPDATE_NOT_SPD;
  const U idet = U(1) / det;
  Si00 = S11 * idet;
  Si01 = -S01 * idet;
  Si11 = S00 * idet;
  r0 = cov_from_d<U>(m0 - p[0]);
  r1 = cov_from_d<U>(m1 - p[1]);
  chi2 += cov_to_d(r0 * (Si00 * r0 + Si01 * r1) + r1 * (Si01 * r0 + Si11 * r1));
#pragma unroll
  for (int j = 0; j < 5; ++j) {
    const U U0 = C[S(j, 0)], U1 = C[S(j, 1)];
    K[j][0] = U0 * Si00 + U1 * Si01;
    K[j][1] = U0 * Si01 + U1 * Si11;
  }
#pragma unroll
  for (int j = 0; j < 5; ++j) p[j] = add2d(p[j], K[j][0], r0, K[j][1], r1);
  if constexpr (kG == 1) {
    // X = (I - K H) C ; C' = X - (X H^T - K V) K^T
    U X[5][5];
#pragma unroll
    for (int r_ = 0; r_ < 5; ++r_)
#pragma unroll
      for (int c_ = 0; c_ < 5; ++c_) X[r_][c_] = C[S(r_, c_)] - K[r_][0] * C[S(0, c_)] - K[r_][1] * C[S(1, c_)];
    U Y[5][2];
#pragma unroll
    for (int r_ = 0; r_ < 5; ++r_) {
      Y[r_][0] = sub2(X[r_][0], K[r_][0], V00, K[r_][1], V01);
      Y[r_][1] = sub2(X[r_][1], K[r_][0], V01, K[r_][1], V11);
    }
#pragma unroll
    for (int r_ = 0; r_ < 5; ++r_)
#pragma unroll
      for (int c_ = r_; c_ < 5; ++c_) C[S(r_, c_)] = X[r_][c_] - Y[r_][0] * K[c_][0] - Y[r_][1] * K[c_][1];
  } else {
    // the same, row gl in lane gl and row 4 in every lane, then exchanged
    const U Kg0 = pick4(gl, K[0][0], K[1][0], K[2][0], K[3][0]);
    const U Kg1 = pick4(gl, K[0][1], K[1][1], K[2][1], K[3][1]);
    U Xg[5], X4[5], Cn[5];
#pragma unroll
    for (int c_ = 0; c_ < 5; ++c_) {
      const U Cgc = pick4(gl, C[S(0, c_)], C[S(1, c_)], C[S(2, c_)], C[S(3, c_)]);
      Xg[c_] = Cgc - Kg0 * C[S(0, c_)] - Kg1 * C[S(1, c_)];
      X4[c_] = C[S(4, c_)] - K[4][0] * C[S(0, c_)] - K[4][1] * C[S(1, c_)];
    }
    const U Yg0 = sub2(Xg[0], Kg0, V00, Kg1, V01), Yg1 = sub2(Xg[1], Kg0, V01, Kg1, V11);
    const U Y40 = sub2(X4[0], K[4][0], V00, K[4][1], V01), Y41 = sub2(X4[1], K[4][0], V01, K[4][1], V11);
#pragma unroll
    for (int c_ = 0; c_ < 5; ++c_) Cn[c_] = Xg[c_] - Yg0 * K[c_][0] - Yg1 * K[c_][1];
    const U C44 = X4[4] - Y40 * K[4][0] - Y41 * K[4][1];
#pragma unroll
    for (int r_ = 0; r_ < 4; ++r_)
#pragma unroll
      for (int c_ = r_; c_ < 5; ++c_) C[S(r_, c_)] = gshfl<kG>(gmask, Cn[c_], r_);
    C[S(4, 4)] = C44;
  }
  return 0;
}

// Filtered direction: the predicted one (sp2, cp2, st2, ct2) turned by the update's angle
// increments p[2], p[3] (angle-addition identities). Returns false when theta leaves (0, pi).
template <bool kMixed>
__device__ __forceinline__ bool turn_direction(const double p[5], double sp2, double cp2, double st2, double ct2,
                                               double& sph, double& cph, double& sth, double& cth) {
  if constexpr (!kMixed) {
    double sd, cd, se, ce;
    small_sincos(p[2], sd, cd);
    small_sincos(p[3], se, ce);
    sph = sp2 * cd + cp2 * sd;
    cph = cp2 * cd - sp2 * sd;
    sth = st2 * ce + ct2 * se;
    cth = ct2 * ce - st2 * se;
  } else {
    // sin and (cos - 1) of the small increments in FP32, applied to the FP64 anchors
    double sd, cd1, se, ce1;
    small_sincos_m1(p[2], sd, cd1);
    small_sincos_m1(p[3], se, ce1);
    sph = sp2 + (sp2 * cd1 + cp2 * sd);
    cph = cp2 + (cp2 * cd1 - sp2 * sd);
    sth = st2 + (st2 * ce1 + ct2 * se);
    cth = ct2 + (ct2 * ce1 - st2 * se);
  }
  return sth > 0.0;
}

// ---- two-filter smoother (the optimal smoother of paper Sec. 4; Fraser-Potter form): after the
// forward filter, a backward Kalman filter of the reversed particle -- (phi + pi, pi - theta,
// -q/p): the same trajectory traversed against the flight direction, so that the ordinary
// propagation applies -- runs from the last entry to the first. It starts from the last filtered
// state with the covariance times the inflation factor, updates with every measurement, and
// after each propagation applies the material of the surface reached (the state on a surface is
// the one before its material in the flight direction). The result on the first surface is the
// weighted mean of the backward filtered state and the seed.

// The reversal's Jacobian is diag(1, 1, 1, -1, -1): the covariance elements that pair theta or
// q/p with one of the other three change sign.
__device__ __forceinline__ bool reversal_flips(int r, int c) { return (r >= 3) != (c >= 3); }

// Backward start: the forward filter's last state reversed, its covariance times `infl`, angle
// increments restarting at 0 (the direction is carried as sines and cosines).
template <class U>
__device__ __forceinline__ void reverse_for_backward(double p[5], U C[15], double& sph, double& cph, double& cth,
                                                     U infl) {
  sph = -sph;
  cph = -cph;
  cth = -cth;
  p[2] = 0.0;
  p[3] = 0.0;
  p[4] = -p[4];
#pragma unroll
  for (int r = 0; r < 5; ++r)
#pragma unroll
    for (int c = r; c < 5; ++c) C[S(r, c)] = (reversal_flips(r, c) ? -infl : infl) * C[S(r, c)];
}

// The material of surface s for the reversed particle arriving with direction (sp2, cp2, st2,
// ct2): the mean loss given back to q/p = p[4], the scattering variance added to C.
template <int kPrec>
__device__ __forceinline__ uint32_t arrival_material(const FitArgs& a, const Surf& s, double sp2, double cp2,
                                                     double st2, double ct2, double p[5],
                                                     typename CovType<kPrec>::type C[15]) {
  using U = typename CovType<kPrec>::type;
  double lam = p[4];
  uint32_t status;
  if constexpr (kPrec == 0) {
    const double T[3] = {st2 * cp2, st2 * sp2, ct2};
    double th0sq;
    status = material<true>(s, a.mat, a.opt.mass, T, lam, th0sq);
    C[S(2, 2)] += th0sq / (st2 * st2);
    C[S(3, 3)] += th0sq;
  } else {
    const float T[3] = {d2f(st2 * cp2), d2f(st2 * sp2), d2f(ct2)};
    float th0sq;
    status = material_mixed<true>(s, a.mat, a.opt, T, lam, th0sq);
    const float fst = d2f(st2);
    C[S(2, 2)] += cov_from_f<U>(th0sq / (fst * fst));
    C[S(3, 3)] += cov_from_f<U>(th0sq);
  }
  p[4] = lam;
  return status;
}

// The backward filter's state on the first surface back in the flight direction's parameters,
// and its weighted mean with the seed (p0, C0): K = Cb (Cb + C0)^-1, p = pb + K (p0 - pb),
// C = (I - K) Cb (I - K)^T + K C0 K^T (the symmetric form of (I - K) Cb), into st.dl / st.E.
template <int kPlace, class U>
__device__ __forceinline__ uint32_t combine_with_seed(const FitArgs& a, uint32_t i, const double p[5], const U C[15],
                                                      double sph, double cph, double sth, double cth,
                                                      SmootherStore<kPlace, U>& st) {
  const uint32_t n = a.stride;
  double pb[5] = {p[0], p[1], atan2(-sph, -cph), atan2(sth, -cth), -p[4]};
  U Cb[15], C0[15], L[15];
  double d[5];
#pragma unroll
  for (int r = 0; r < 5; ++r)
#pragma unroll
    for (int c = r; c < 5; ++c) Cb[S(r, c)] = reversal_flips(r, c) ? -C[S(r, c)] : C[S(r, c)];
#pragma unroll
  for (int j = 0; j < 15; ++j) {
    C0[j] = cov_from_d<U>(a.seed_cov[size_t(j) * n + i] * a.seed_cov_scale);
    L[j] = Cb[j] + C0[j];
  }
#pragma unroll
  for (int j = 0; j < 5; ++j) d[j] = a.seed_par[size_t(j) * n + i] - pb[j];
  if (d[2] > kPi) d[2] -= 2.0 * kPi;
  if (d[2] <= -kPi) d[2] += 2.0 * kPi;
  // Cb + C0 = L D L^T in place (unit lower L below the diagonal, D on it)
#pragma unroll
  for (int j = 0; j < 5; ++j) {
    if (!(L[S(j, j)] > U(0))) return TKF_TRACK_SMOOTHER_NOT_SPD;
    const U inv = U(1) / L[S(j, j)];
#pragma unroll
    for (int r = j + 1; r < 5; ++r) {
      const U f = L[S(j, r)] * inv;
#pragma unroll
      for (int c = r; c < 5; ++c) L[S(r, c)] -= f * L[S(j, c)];
    }
#pragma unroll
    for (int r = j + 1; r < 5; ++r) L[S(j, r)] *= inv;
  }
  // K^T = (Cb + C0)^-1 Cb: column c of K^T (row c of K) from row c of Cb
  U K[5][5];
#pragma unroll
  for (int c = 0; c < 5; ++c) {
    U x[5];
#pragma unroll
    for (int r = 0; r < 5; ++r) {
      U acc = Cb[S(c, r)];
#pragma unroll
      for (int q = 0; q < r; ++q) acc -= L[S(q, r)] * x[q];
      x[r] = acc;
    }
#pragma unroll
    for (int r = 0; r < 5; ++r) x[r] /= L[S(r, r)];
#pragma unroll
    for (int r = 4; r >= 0; --r) {
#pragma unroll
      for (int q = r + 1; q < 5; ++q) x[r] -= L[S(r, q)] * x[q];
    }
#pragma unroll
    for (int r = 0; r < 5; ++r) K[c][r] = x[r];
  }
#pragma unroll
  for (int r = 0; r < 5; ++r) {
    double acc = pb[r];
#pragma unroll
    for (int c = 0; c < 5; ++c) acc += cov_to_d(K[r][c]) * d[c];
    st.dl(r) = acc;
  }
  if (st.dl(2) > kPi) st.dl(2) -= 2.0 * kPi;
  if (st.dl(2) <= -kPi) st.dl(2) += 2.0 * kPi;
  // A = (I - K) Cb, B = K C0; C = A (I - K)^T + B K^T
  U A[5][5], B[5][5];
#pragma unroll
  for (int r = 0; r < 5; ++r)
#pragma unroll
    for (int c = 0; c < 5; ++c) {
      U acc = Cb[S(r, c)], acc0 = U(0);
#pragma unroll
      for (int q = 0; q < 5; ++q) {
        acc -= K[r][q] * Cb[S(q, c)];
        acc0 += K[r][q] * C0[S(q, c)];
      }
      A[r][c] = acc;
      B[r][c] = acc0;
    }
#pragma unroll
  for (int r = 0; r < 5; ++r)
#pragma unroll
    for (int c = r; c < 5; ++c) {
      U acc = A[r][c];
#pragma unroll
      for (int q = 0; q < 5; ++q) acc += B[r][q] * K[c][q] - A[r][q] * K[c][q];
      st.E(S(r, c)) = acc;
    }
  return 0;
}

// ---- all-states mode: the forward pass stores what the backward RTS pass needs.
// Filtered state of entry m into the all-states arrays (SoA [5][n_meas], [15][n_meas]); at
// the first entry p holds the angles, later the direction is carried as sines and cosines.
template <class U>
__device__ __forceinline__ void store_filtered(const FitArgs& a, uint32_t m, const double p[5], const U C[15],
                                               bool first, double sph, double cph, double sth, double cth) {
  const size_t nm = size_t(a.n_meas);
  a.states_par[m] = p[0];
  a.states_par[nm + m] = p[1];
  a.states_par[2 * nm + m] = first ? p[2] : atan2(sph, cph);
  a.states_par[3 * nm + m] = first ? p[3] : atan2(sth, cth);
  a.states_par[4 * nm + m] = p[4];
#pragma unroll
  for (int j = 0; j < 15; ++j) a.states_cov[size_t(j) * nm + m] = cov_to_d(C[j]);
}

// Predicted state, packed covariance and transport Jacobian (row-major) of entry m into the
// workspace: 45 doubles an entry, entry-major (kStatesScratch).
template <class U>
__device__ __forceinline__ void store_predicted(const FitArgs& a, uint32_t m, const double p[5], const U C[15],
                                                const U J[5][5], double sp2, double cp2, double st2, double ct2) {
  double* w = a.states_scratch + size_t(m) * kStatesScratch;
  w[0] = p[0];
  w[1] = p[1];
  w[2] = atan2(sp2, cp2);
  w[3] = atan2(st2, ct2);
  w[4] = p[4];
#pragma unroll
  for (int j = 0; j < 15; ++j) w[5 + j] = cov_to_d(C[j]);
#pragma unroll
  for (int r = 0; r < 5; ++r)
#pragma unroll
    for (int c = 0; c < 5; ++c) w[20 + 5 * r + c] = cov_to_d(J[r][c]);
}

template <int kPrec, int kMode, int kG, int kPlace, int kSmooth, bool kRoll, class F>
__device__ void fit_track(const FitArgs& a, const F& fld, uint32_t i,
                          SmootherStore<kPlace, typename CovType<kPrec>::type> st, uint32_t gl = 0,
                          uint32_t gmask = 0xffffffffu) {
  constexpr bool kMixed = kPrec != 0;
  static_assert(kG == 1 || kMode != kRecord, "record capture runs one lane per track");
  static_assert(kSmooth == 0 || (kG == 1 && kMode != kRecord), "the two-filter smoother runs one lane a track");
  static_assert(kMode != kStates || (kG == 1 && kSmooth == 0), "all-states output: one lane a track, RTS");
  const bool writer = kG == 1 || gl == 0;  // the lane that writes the group's results
  using U = typename CovType<kPrec>::type;
  const uint32_t n = a.stride;  // SoA row stride of seeds and outputs
  const uint32_t b0 = a.offsets[i], b1 = a.offsets[i + 1];
  double p[5];
  U C[15];
  for (int j = 0; j < 5; ++j) p[j] = a.seed_par[size_t(j) * n + i];
  for (int j = 0; j < 15; ++j) C[j] = cov_from_d<U>(a.seed_cov[size_t(j) * n + i] * a.seed_cov_scale);
  uint32_t status = 0, attempts = 0, rejected = 0;
  double chi2 = 0.0;
  int N = 0, M = 0;  // entries, and entries with a measurement
  const double nan = __longlong_as_double(0x7ff8000000000000LL);

  const bool bad_offsets = b1 < b0 || b1 > a.n_meas;
  if (bad_offsets) {
    status = TKF_TRACK_BAD_INPUT;  // never read outside the measurement arrays
  } else {
    N = int(b1 - b0);
    for (int k = 0; k < N; ++k) {
      const uint32_t sid = a.sid[b0 + k];
      if ((sid & ~TKF_SID_NO_MEASUREMENT) >= a.n_surf) status = TKF_TRACK_BAD_INPUT;
      M += (sid & TKF_SID_NO_MEASUREMENT) ? 0 : 1;
    }
  }
  if (M == 0 && status == 0) {  // nothing to fit (no entry, or no measurement): the seed
    if (!writer) return;
    for (int j = 0; j < 5; ++j) a.par[size_t(j) * n + i] = p[j];
    for (int j = 0; j < 15; ++j) a.cov[size_t(j) * n + i] = cov_to_d(C[j]);
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

  Surf sp;                       // surface of the previous measurement (FP64 path)
  uint32_t sid_prev = 0;         // its id (the mixed path reads the record again when needed)
  double sph = 0.0, cph = 1.0, sth = 1.0, cth = 0.0;  // filtered direction at sp
  // learned mode: the step-size control starts from the network's proposal for this track
  // (a negative value: the proposal pre-pass gave up; start from h_max and flag the track)
  float h_start = a.opt.h_max_f;
  if constexpr (kMode == kLearned) {
    h_start = a.h0[i];
    if (!(h_start > 0.0f)) {
      h_start = a.opt.h_max_f;
      status |= TKF_TRACK_PROPOSAL_FALLBACK;
    }
  }
  double h_ctrl = kMode == kLearned ? double(h_start) : a.opt.h_max;
  float h_ctrl_f = h_start;
  StepLearn learn{a.records, a.record_capacity, a.record_count, a.opt.h_max_f};
  // group-per-track: lane gl keeps row gl of P and of E (and its element of dl), every lane
  // keeps row 4 (gathered into `st` after the last measurement)
  U Pg[5], P4[5], Eg[5], E44 = U(0);
  double dlg = 0.0, dl4 = 0.0;
#pragma unroll
  for (int c = 0; c < 5; ++c) Pg[c] = P4[c] = Eg[c] = U(0);

  // kSmooth 1 (two-filter): a second pass runs the backward filter over the entries in reverse
  // (unrolled: each pass is compiled with its own direction)
  constexpr int kPasses = kSmooth == 1 ? 2 : 1;
  double chi2_bwd = 0.0;
#pragma unroll 1
  for (int pass = 0; pass < kPasses; ++pass) {
  const bool bwd = pass == 1;
  if (bwd) {
    if (status & kFatal) break;
    reverse_for_backward(p, C, sph, cph, cth, U(a.backward_inflation));
  }
  for (int ent = 0; ent < N && !(status & kFatal); ++ent) {
    const int k = bwd ? N - 1 - ent : ent;
    const uint32_t m = b0 + k;
    Surf s;
    const uint32_t sid_m = a.sid[m];
    const bool measured = (sid_m & TKF_SID_NO_MEASUREMENT) == 0;
    const uint32_t sid = sid_m & ~TKF_SID_NO_MEASUREMENT;
    load_surf(a.surf, sid, s);
    U J[5][5];
    double sp2 = 0.0, cp2 = 1.0, st2 = 1.0, ct2 = 0.0;  // predicted direction at s (ent >= 1)
    if (bwd && ent == 0) {  // the backward filter starts on this surface: no prediction
      sp2 = sph;
      cp2 = cph;
      st2 = sth;
      ct2 = cth;
    }
    if (ent > 0) {
      constexpr int kCols = kG == 1 ? 3 : 1;
      if constexpr (!kMixed) {
      // ---- material of the previous surface (muon hypothesis), then propagation
      double T[3] = {sth * cph, sth * sph, cth};
      double lam = p[4], th0sq = 0.0;
      if (!bwd) {
        status |= material(sp, a.mat, a.opt.mass, T, lam, th0sq);
        if (status & kFatal) break;
      }
      double r[3];
      for (int j = 0; j < 3; ++j) r[j] = sp.c[j] + p[0] * sp.u[j] + p[1] * sp.v[j];
      double dr[kCols][3], dT[kCols][3];
      const double dphi[3] = {-sth * sph, sth * cph, 0.0}, dtheta[3] = {cth * cph, cth * sph, -sth};
#pragma unroll
      for (int c = 0; c < kCols; ++c)
#pragma unroll
        for (int j = 0; j < 3; ++j) {
          const uint32_t col = kG == 1 ? uint32_t(c) : gl;  // this lane's column
          dr[c][j] = 0.0;
          dT[c][j] = col == 0 ? dphi[j] : (col == 1 ? dtheta[j] : 0.0);
        }
      const double qcol = gl == 2 ? 1.0 : 0.0;
      double kend[3];
      status |= propagate<kMode == kRecord ? kRecord : kPlain, kCols>(fld, a.opt, s, r, T, lam, dr, dT, qcol, h_ctrl,
                                                                      attempts, rejected, kend, learn);
      if (status & kFatal) break;
      // ---- bound parameters at the target and the transport Jacobian (path correction)
      const double inv_norm = 1.0 / sqrt(dot3(T, T));
      const double tn[3] = {T[0] * inv_norm, T[1] * inv_norm, T[2] * inv_norm};
      st2 = sqrt(tn[0] * tn[0] + tn[1] * tn[1]);
      const double inv_st = 1.0 / st2;
      ct2 = tn[2];
      cp2 = tn[0] * inv_st;
      sp2 = tn[1] * inv_st;
      const double inv_nT = 1.0 / dot3(s.n, T);
#pragma unroll
      for (int c = 0; c < 2 + kCols; ++c) {  // u, v, then this lane's derivative columns
        double x[3], t[3], out[4];
        for (int j = 0; j < 3; ++j) {
          x[j] = (c == 0) ? sp.u[j] : (c == 1) ? sp.v[j] : dr[c - 2][j];
          t[j] = (c < 2) ? 0.0 : dT[c - 2][j];
        }
        jac_column(s.n, s.u, s.v, T, kend, inv_nT, sp2, cp2, st2, ct2, inv_st, x, t, out);
        for (int rr = 0; rr < 4; ++rr) J[rr][c] = out[rr];
      }
      if constexpr (kG > 1) {
        const double own[4] = {J[0][2], J[1][2], J[2][2], J[3][2]};
#pragma unroll
        for (int c = 2; c < 5; ++c)
#pragma unroll
          for (int rr = 0; rr < 4; ++rr) J[rr][c] = gshfl<kG>(gmask, own[rr], c - 2);
      }
#pragma unroll
      for (int c = 0; c < 5; ++c) J[4][c] = (c == 4) ? 1.0 : 0.0;
      const double d[3] = {r[0] - s.c[0], r[1] - s.c[1], r[2] - s.c[2]};
      p[0] = dot3(s.u, d);
      p[1] = dot3(s.v, d);
      p[2] = 0.0;  // angles are carried as sines and cosines from here on
      p[3] = 0.0;
      p[4] = lam;
      // ---- C_pred = J (C + Q) J^T, Q = diag(0, 0, th0^2/sin^2(theta), th0^2, 0)
      if (!bwd) {
        C[S(2, 2)] += th0sq / (sth * sth);
        C[S(3, 3)] += th0sq;
      }
      transport_cov<kG>(J, C, gl, gmask);
      } else {
      // ---- mixed precision: material, propagation, Jacobian and covariance transport in FP32.
      // Only the ids of both surfaces stay live: their frames are read again after the
      // propagation, which keeps the state carried through it within the register cap.
      Surf sp;
      load_surf(a.surf, sid_prev, sp);
      const float Tm[3] = {d2f(sth * cph), d2f(sth * sph), d2f(cth)};
      double lam = p[4];
      float th0sq = 0.0f;
      if (!bwd) {
        status |= material_mixed(sp, a.mat, a.opt, Tm, lam, th0sq);
        if (status & kFatal) break;
      }
      double T[3] = {sth * cph, sth * sph, cth};
      double r[3];
      for (int j = 0; j < 3; ++j) r[j] = sp.c[j] + p[0] * sp.u[j] + p[1] * sp.v[j];
      const float fsth = d2f(sth), fcth = d2f(cth), fsph = d2f(sph), fcph = d2f(cph);
      float dr[kCols][3], dT[kCols][3];
      const float dphi[3] = {-fsth * fsph, fsth * fcph, 0.0f}, dtheta[3] = {fcth * fcph, fcth * fsph, -fsth};
#pragma unroll
      for (int c = 0; c < kCols; ++c)
#pragma unroll
        for (int j = 0; j < 3; ++j) {
          const uint32_t col = kG == 1 ? uint32_t(c) : gl;  // this lane's column
          dr[c][j] = 0.0f;
          dT[c][j] = col == 0 ? dphi[j] : (col == 1 ? dtheta[j] : 0.0f);
        }
      const float qcol = gl == 2 ? 1.0f : 0.0f;
      const float* nf = s.nf;
      // C + Q in FP32, formed before the propagation: only the FP32 copy is transported
      float Cf[15];
#pragma unroll
      for (int j = 0; j < 15; ++j) Cf[j] = cov_to_f(C[j]);
      if (!bwd) {
        Cf[S(2, 2)] += th0sq / (fsth * fsth);
        Cf[S(3, 3)] += th0sq;
      }
      float kend[3];
      status |= propagate_mixed<kMode == kRecord ? kRecord : kPlain, kCols, F, kRoll>(
          fld, a.opt, s, nf, r, T, lam, dr, dT, qcol, h_ctrl_f, attempts, rejected, kend, learn);
      if (status & kFatal) break;
      // direction at the target in FP64 from FP32-seeded Newton steps (relative error ~1e-14)
      const double t2 = dot3(T, T), e2 = t2 - 1.0;
      const double inv_norm = fabs(e2) < 1e-4 ? 1.0 - e2 * (0.5 - 0.375 * e2) : 1.0 / sqrt(t2);
      const double tn[3] = {T[0] * inv_norm, T[1] * inv_norm, T[2] * inv_norm};
      const double v = tn[0] * tn[0] + tn[1] * tn[1];
      double inv_st;
      if (v > 1e-12) {
        const float yf = sqrtf(d2f(v));
        double y = f2d(yf);
        y = fma(fma(-y, y, v), f2d(0.5f / yf), y);
        const float zf = 1.0f / d2f(y);
        double z = f2d(zf);
        z = z * fma(-y, z, 2.0);
        st2 = y;
        inv_st = z;
      } else {
        st2 = sqrt(v);
        inv_st = 1.0 / st2;
      }
      ct2 = tn[2];
      cp2 = tn[0] * inv_st;
      sp2 = tn[1] * inv_st;
      const float Tf[3] = {d2f(T[0]), d2f(T[1]), d2f(T[2])};
      float uf[3], vf[3], puf[3], pvf[3];
      reload_uvf(a.surf, sid, uf, vf);
      reload_uvf(a.surf, sid_prev, puf, pvf);
      const float inv_nT = 1.0f / dotr(nf, Tf);
      const float fst = d2f(st2), fct = d2f(ct2), fcp = d2f(cp2), fsp = d2f(sp2), finv_st = d2f(inv_st);
      float Jf[5][5];
#pragma unroll
      for (int c = 0; c < 2 + kCols; ++c) {  // u, v, then this lane's derivative columns
        float x[3], t[3], out[4];
        for (int j = 0; j < 3; ++j) {
          x[j] = (c == 0) ? puf[j] : (c == 1) ? pvf[j] : dr[c - 2][j];
          t[j] = (c < 2) ? 0.0f : dT[c - 2][j];
        }
        jac_column(nf, uf, vf, Tf, kend, inv_nT, fsp, fcp, fst, fct, finv_st, x, t, out);
        for (int rr = 0; rr < 4; ++rr) Jf[rr][c] = out[rr];
      }
      if constexpr (kG > 1) {
        const float own[4] = {Jf[0][2], Jf[1][2], Jf[2][2], Jf[3][2]};
#pragma unroll
        for (int c = 2; c < 5; ++c)
#pragma unroll
          for (int rr = 0; rr < 4; ++rr) Jf[rr][c] = gshfl<kG>(gmask, own[rr], c - 2);
      }
#pragma unroll
      for (int c = 0; c < 5; ++c) Jf[4][c] = (c == 4) ? 1.0f : 0.0f;
      if constexpr (F::kAlongZ) {  // theta is conserved: its row is e_3 (FP32 noise otherwise)
#pragma unroll
        for (int c = 0; c < 5; ++c) Jf[3][c] = (c == 3) ? 1.0f : 0.0f;
      }
      const double d[3] = {r[0] - s.c[0], r[1] - s.c[1], r[2] - s.c[2]};
      double su[3], sv[3];
      reload_uv(a.surf, sid, su, sv);
      p[0] = dot3(su, d);
      p[1] = dot3(sv, d);
      p[2] = 0.0;
      p[3] = 0.0;
      p[4] = lam;
      // C_pred = J (C + Q) J^T in FP32
      transport_cov<kG, float, F::kAlongZ>(Jf, Cf, gl, gmask);
#pragma unroll
      for (int j = 0; j < 15; ++j) C[j] = cov_from_f<U>(Cf[j]);
#pragma unroll
      for (int r0 = 0; r0 < 5; ++r0)
#pragma unroll
        for (int c0 = 0; c0 < 5; ++c0) J[r0][c0] = cov_from_f<U>(Jf[r0][c0]);
      }
      if (bwd) {  // the material of the surface reached, crossed against the flight direction
        status |= arrival_material<kPrec>(a, s, sp2, cp2, st2, ct2, p, C);
        if (status & kFatal) break;
      }
      if constexpr (kMode == kStates) store_predicted(a, m, p, C, J, sp2, cp2, st2, ct2);
      // ---- smoother: R = P J^T (in place; J row 4 is e_4); the row loop stays rolled in the
      // 64-register kernel (smaller code; measured faster), unrolled otherwise
      if constexpr (kSmooth == 1) {
      } else if constexpr (kG == 1) {
#pragma unroll(kRoll ? 1 : 5)
      for (int r0 = 0; r0 < 5; ++r0) {
        U row[5];
#pragma unroll
        for (int c0 = 0; c0 < 4; ++c0) {
          if (kMixed && F::kAlongZ && c0 == 3) {  // J row 3 is e_3 (mixed path, field along z)
            row[3] = st.P(r0, 3);
            continue;
          }
          U acc = 0;
#pragma unroll
          for (int q = 0; q < 5; ++q) acc += st.P(r0, q) * J[c0][q];
          row[c0] = acc;
        }
        row[4] = st.P(r0, 4);
#pragma unroll
        for (int c0 = 0; c0 < 5; ++c0) st.P(r0, c0) = row[c0];
      }
      } else {
        U rg[5], r4[5];
#pragma unroll
        for (int c0 = 0; c0 < 4; ++c0) {
          if (kMixed && F::kAlongZ && c0 == 3) {  // J row 3 is e_3 (mixed path, field along z)
            rg[3] = Pg[3];
            r4[3] = P4[3];
            continue;
          }
          U acc = 0, acc4 = 0;
#pragma unroll
          for (int q = 0; q < 5; ++q) {
            acc += Pg[q] * J[c0][q];
            acc4 += P4[q] * J[c0][q];
          }
          rg[c0] = acc;
          r4[c0] = acc4;
        }
        rg[4] = Pg[4];
        r4[4] = P4[4];
#pragma unroll
        for (int c0 = 0; c0 < 5; ++c0) {
          Pg[c0] = rg[c0];
          P4[c0] = r4[c0];
        }
      }
    }
    // ---- gain-matrix update with H = [I2 0]; Joseph form (paper Sec. 2; Fruhwirth 1987).
    // An entry without a measurement has none: the gain, the inverse residual covariance and
    // the residual stay 0, so the filtered state is the predicted one and the smoother terms
    // below add exact zeros.
    U Si00 = U(0), Si01 = U(0), Si11 = U(0), r0 = U(0), r1 = U(0);
    U K[5][2];
#pragma unroll
    for (int j = 0; j < 5; ++j) K[j][0] = K[j][1] = U(0);
    if (measured) {
      // the track's chi2 is the forward filter's; the backward filter's goes to chi2_bwd
      status |= kalman_update<kG>(a, m, p, C, K, Si00, Si01, Si11, r0, r1, bwd ? chi2_bwd : chi2, gl, gmask);
      if (status & kFatal) break;
    }  // measured
    if (!bwd && k == 0) {
      if (p[2] > kPi) p[2] -= 2.0 * kPi;
      if (p[2] <= -kPi) p[2] += 2.0 * kPi;
      if (!(p[3] > 0.0 && p[3] < kPi)) {
        status |= TKF_TRACK_NON_FINITE;
        break;
      }
      sincos(p[2], &sph, &cph);
      sincos(p[3], &sth, &cth);
      // p_0|0 and C_0|0 start the smoothed sums; P_0 = C_0|0
      if constexpr (kSmooth == 1) {
      } else if constexpr (kG == 1) {
#pragma unroll
      for (int j = 0; j < 5; ++j) st.dl(j) = p[j];
#pragma unroll
      for (int j = 0; j < 15; ++j) st.E(j) = C[j];
#pragma unroll
      for (int r_ = 0; r_ < 5; ++r_)
#pragma unroll
        for (int c_ = 0; c_ < 5; ++c_) st.P(r_, c_) = C[S(r_, c_)];
      } else {
        dlg = pick4(gl, p[0], p[1], p[2], p[3]);
        dl4 = p[4];
#pragma unroll
        for (int c_ = 0; c_ < 5; ++c_) {
          Pg[c_] = Eg[c_] = pick4(gl, C[S(0, c_)], C[S(1, c_)], C[S(2, c_)], C[S(3, c_)]);
          P4[c_] = C[S(4, c_)];
        }
        E44 = C[S(4, 4)];
      }
    } else {
      // filtered direction: predicted angles plus the update's increments p[2], p[3]
      if (!turn_direction<kMixed>(p, sp2, cp2, st2, ct2, sph, cph, sth, cth)) {  // theta left (0, pi)
        status |= TKF_TRACK_NON_FINITE;
        break;
      }
      // W = R H^T S^-1; p_0|N += W r; C_0|N -= W (R H^T)^T; P = R - R H^T K^T
      if constexpr (kSmooth == 1) {
      } else if constexpr (kG == 1) {
      U W[5][2];
#pragma unroll
      for (int j = 0; j < 5; ++j) {
        W[j][0] = st.P(j, 0) * Si00 + st.P(j, 1) * Si01;
        W[j][1] = st.P(j, 0) * Si01 + st.P(j, 1) * Si11;
        st.dl(j) = add2d(st.dl(j), W[j][0], r0, W[j][1], r1);
      }
#pragma unroll
      for (int r_ = 0; r_ < 5; ++r_)
#pragma unroll
        for (int c_ = r_; c_ < 5; ++c_)
          st.E(S(r_, c_)) = sub2(st.E(S(r_, c_)), W[r_][0], st.P(c_, 0), W[r_][1], st.P(c_, 1));
#pragma unroll
      for (int r_ = 0; r_ < 5; ++r_) {
        const U R0 = st.P(r_, 0), R1 = st.P(r_, 1);
#pragma unroll
        for (int c_ = 0; c_ < 5; ++c_) st.P(r_, c_) = sub2(st.P(r_, c_), R0, K[c_][0], R1, K[c_][1]);
      }
      } else {
        // rows gl and 4; columns 0 and 1 of R from every row's lane
        const U Wg0 = Pg[0] * Si00 + Pg[1] * Si01, Wg1 = Pg[0] * Si01 + Pg[1] * Si11;
        const U W40 = P4[0] * Si00 + P4[1] * Si01, W41 = P4[0] * Si01 + P4[1] * Si11;
        dlg = add2d(dlg, Wg0, r0, Wg1, r1);
        dl4 = add2d(dl4, W40, r0, W41, r1);
        U R0c[5], R1c[5];
#pragma unroll
        for (int c_ = 0; c_ < 4; ++c_) {
          R0c[c_] = gshfl<kG>(gmask, Pg[0], c_);
          R1c[c_] = gshfl<kG>(gmask, Pg[1], c_);
        }
        R0c[4] = P4[0];
        R1c[4] = P4[1];
#pragma unroll
        for (int c_ = 0; c_ < 5; ++c_) Eg[c_] = sub2(Eg[c_], Wg0, R0c[c_], Wg1, R1c[c_]);
        E44 = sub2(E44, W40, R0c[4], W41, R1c[4]);
        const U Rg0 = Pg[0], Rg1 = Pg[1], R40 = P4[0], R41 = P4[1];
#pragma unroll
        for (int c_ = 0; c_ < 5; ++c_) {
          Pg[c_] = sub2(Pg[c_], Rg0, K[c_][0], Rg1, K[c_][1]);
          P4[c_] = sub2(P4[c_], R40, K[c_][0], R41, K[c_][1]);
        }
      }
    }
    if constexpr (kMode == kStates) store_filtered(a, m, p, C, k == 0, sph, cph, sth, cth);
    if constexpr (!kMixed) sp = s;
    sid_prev = sid;
  }
  }  // passes
  if constexpr (kSmooth == 1) {
    if (!(status & kFatal)) status |= combine_with_seed(a, i, p, C, sph, cph, sth, cth, st);
  }
  if constexpr (kG > 1) {
    // the smoothed sums into every lane's full store (rows 0..3 from their lanes)
#pragma unroll
    for (int r_ = 0; r_ < 4; ++r_) {
      st.dl(r_) = gshfl<kG>(gmask, dlg, r_);
#pragma unroll
      for (int c_ = r_; c_ < 5; ++c_) st.E(S(r_, c_)) = gshfl<kG>(gmask, Eg[c_], r_);
    }
    st.dl(4) = dl4;
    st.E(S(4, 4)) = E44;
  }

  if (!(status & kFatal)) {
    if (st.dl(2) > kPi) st.dl(2) -= 2.0 * kPi;
    if (st.dl(2) <= -kPi) st.dl(2) += 2.0 * kPi;
    // positive definiteness of the smoothed covariance: all LDL^T pivots > 0
    U L[15];
#pragma unroll
    for (int j = 0; j < 15; ++j) L[j] = st.E(j);
    bool spd = true;
#pragma unroll
    for (int j = 0; j < 5; ++j) {
      const U d = L[S(j, j)];
      spd = spd && (d > U(0));
      const U inv = U(1) / d;
#pragma unroll
      for (int r_ = j + 1; r_ < 5; ++r_) {
        const U f = L[S(j, r_)] * inv;
#pragma unroll
        for (int c_ = r_; c_ < 5; ++c_) L[S(r_, c_)] -= f * L[S(j, c_)];
      }
    }
    if (!spd) status |= TKF_TRACK_SMOOTHER_NOT_SPD;
    bool fin = isfinite(chi2);
#pragma unroll
    for (int j = 0; j < 5; ++j) fin = fin && isfinite(st.dl(j));
#pragma unroll
    for (int j = 0; j < 15; ++j) fin = fin && isfinite(st.E(j));
    if (!fin) status |= TKF_TRACK_NON_FINITE;
  }
  if (status & kFatal) {
#pragma unroll
    for (int j = 0; j < 5; ++j) st.dl(j) = nan;
#pragma unroll
    for (int j = 0; j < 15; ++j) st.E(j) = U(nan);
    chi2 = nan;
  }
  if (M < 3 && !bad_offsets) status |= TKF_TRACK_TOO_FEW_HITS;
  if (!writer) return;
#pragma unroll
  for (int j = 0; j < 5; ++j) a.par[size_t(j) * n + i] = st.dl(j);
#pragma unroll
  for (int j = 0; j < 15; ++j) a.cov[size_t(j) * n + i] = cov_to_d(st.E(j));
  a.chi2[i] = chi2;
  a.ndf[i] = 2 * M;
  a.status[i] = status;
  if (a.steps) {
    a.steps[i] = attempts;
    a.steps[n + i] = rejected;
  }
}

// Persistent fit: each warp takes the next `tpw` (1..32) tracks of the ordered list from a
// global counter, one per lane; lanes tpw..31 idle. Fewer tracks per warp spread a small batch
// over more warps and schedulers. kRegs caps the registers a thread (255, 128 or 64): below
// 255 part of the per-track state lives in local memory (L1), and an SM holds 16 or 32 warps
// instead of 8, which hides more of the latency between the FP64 and FP32 phases.
__host__ __device__ constexpr int reg_block_threads(int regs) { return regs >= 255 ? 256 : 128; }
__host__ __device__ constexpr int reg_min_blocks(int regs) { return regs >= 255 ? 1 : 65536 / (regs * 128); }

// Where the smoother state lives per register cap (measured): 255 registers hold it; at 128 the
// whole state goes to shared memory (184 KB an SM at 16 warps; spills fall from 1.2 to 0.4 KB a
// thread, launch -3 %); at 64 registers it stays with the spilled state (shared memory for 32
// warps would take the L1 capacity those spills need: launch +6 %).
__host__ __device__ constexpr int reg_state_place(int regs) { return regs == 128 ? 2 : 0; }

// kG lanes a track (1, or 4 for the group-per-track mapping): a warp takes tpw <= 32 / kG tracks
// at a time, lanes g kG .. g kG + kG - 1 fit track base + g together.
template <int kPrec, int kMode, int kRegs, int kG, int kSmooth, class F>
__global__ void __launch_bounds__(reg_block_threads(kRegs), reg_min_blocks(kRegs))
    fit_persistent_kernel(FitArgs a, F fld, const uint32_t* __restrict__ perm, uint32_t* __restrict__ counter,
                          uint32_t tpw) {
  constexpr int kPlace = kPrec == 2 ? 0 : reg_state_place(kRegs);
  extern __shared__ double smem_state[];
  SmootherStore<kPlace, typename CovType<kPrec>::type> st{};
  if constexpr (kPlace != 0) st.s = smem_state + threadIdx.x * state_doubles(kPlace);
  const uint32_t lane = threadIdx.x & 31u;
  const uint32_t g = lane / kG, gl = lane % kG;
  const uint32_t gmask = kG == 1 ? 0xffffffffu : ((1u << kG) - 1u) << (g * kG);
  for (;;) {
    uint32_t base = 0;
    if (lane == 0) base = atomicAdd(counter, tpw);
    base = __shfl_sync(0xffffffffu, base, 0);
    if (base >= a.n_tracks) break;
    const uint32_t j = base + g;
    if (g < tpw && j < a.n_tracks)
      fit_track<kPrec, kMode, kG, kPlace, kSmooth, kRegs == 64>(a, fld, perm[j], st, gl, gmask);
  }
}

inline FieldGrid grid_policy(const FieldDev& f) {
  return FieldGrid{f.grid, f.nr, f.nz, f.r0, f.z0, f.inv_dr, f.inv_dz, float(f.r0), float(f.z0), float(f.inv_dr),
                   float(f.inv_dz), float(f.nr - 1), float(f.nz - 1)};
}

// ------------------------------------------------------------------ learned pre-pass on tensor cores
// Each track's starting step-size control comes from the network, evaluated on the seed state
// at the first surface toward the second. The two dense layers run on the fifth-generation
// tensor cores (tcgen05.mma, BF16 operands from shared memory, FP32 accumulators in tensor
// memory); bias, SiLU and the 64 -> 1 output layer run on the CUDA cores. A CTA of 128 threads
// takes tiles of 128 tracks (one track per thread and per accumulator row):
//   features (FP32, rounded to BF16) -> A1 [128 x 16]      layer 1: D = A1 W1^T   (M128 N64 K16)
//   SiLU(D + b1) rounded to BF16    -> A2 [128 x 64]       layer 2: D = A2 W2^T   (4 x K16)
//   out = b3 + w3 . SiLU(D + b2);  h0 = 0.9 exp(round(32 out) / 32), clamped to [h_min, h_max].
// The proposal is rounded to a 1/32 grid in ln h: the control only needs a rough start, and
// the grid makes the proposal insensitive to the accumulation order of the tensor cores.
// Operand layout: K-major, no swizzle, 8 x 16-byte core matrices; the core matrix (row group g,
// K group q) of a [rows x K] operand sits at (g * K/8 + q) * 128 bytes, so consecutive K
// groups are 128 bytes apart (leading byte offset) and row groups K/8 * 128 bytes (stride byte
// offset).
constexpr int kPropTile = 128;
constexpr uint32_t kPropWaitLimit = 1u << 20;  // mbarrier polls (100 ns apart) before a tile gives up

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ uint32_t bf16_rne(float x) {
  uint32_t u = __float_as_uint(x);
  u += 0x7FFFu + ((u >> 16) & 1u);
  return u >> 16;
}

__device__ __forceinline__ float bf16_value(uint32_t b) { return __uint_as_float(b << 16); }

// Shared-memory matrix descriptor: start address, leading and stride byte offsets (all >> 4),
// the fixed version field 0b001 at bit 46, no swizzle.
__device__ __forceinline__ uint64_t umma_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  return uint64_t((saddr >> 4) & 0x3FFFu) | (uint64_t((lbo >> 4) & 0x3FFFu) << 16) |
         (uint64_t((sbo >> 4) & 0x3FFFu) << 32) | (uint64_t(1) << 46);
}

// Instruction descriptor of kind::f16: FP32 accumulator (bit 4), BF16 A (bit 7) and B (bit 10),
// both K-major, N >> 3 at bit 17, M >> 4 at bit 24.
constexpr uint32_t kIdescM128N64 = (1u << 4) | (1u << 7) | (1u << 10) | ((64u >> 3) << 17) | ((128u >> 4) << 24);

__device__ __forceinline__ void tc_mma(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d_tmem),
      "l"(adesc), "l"(bdesc), "r"(kIdescM128N64), "r"(accumulate)
      : "memory");
}

// Instruction descriptor of kind::f16 (BF16 A and B, K-major, FP32 accumulator) for an M x N tile.
__host__ __device__ constexpr uint32_t umma_idesc_bf16(uint32_t m, uint32_t n) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((n >> 3) << 17) | ((m >> 4) << 24);
}

__device__ __forceinline__ void tc_mma_id(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                          uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d_tmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}

__device__ __forceinline__ void tc_commit(uint64_t* mbar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_addr(mbar))
               : "memory");
}

// Waits for the mbarrier phase of the given parity to complete: a non-blocking test every
// 100 ns, at most kPropWaitLimit times (about 0.1 s); false if it never completed.
__device__ __forceinline__ bool mbar_wait(uint64_t* mbar, uint32_t parity) {
  for (uint32_t it = 0; it < kPropWaitLimit; ++it) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(done)
        : "r"(smem_addr(mbar)), "r"(parity)
        : "memory");
    if (done) return true;
    __nanosleep(100);
  }
  return false;
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// 32 consecutive FP32 accumulator columns of this thread's row (lane) of tensor memory.
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float v[32]) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
      "%15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]),
        "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
        "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr)
      : "memory");
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int k = 0; k < 32; ++k) v[k] = __uint_as_float(r[k]);
}

// Byte offset of element (row, k) in a K-major no-swizzle operand with `kgroups` groups of 8 along K.
__device__ __forceinline__ uint32_t core_offset(int row, int k, int kgroups) {
  return uint32_t(((row >> 3) * kgroups + (k >> 3)) * 128 + (row & 7) * 16 + (k & 7) * 2);
}

struct __align__(1024) PropSmem {
  uint8_t a2[kPropTile * 64 * 2];  // layer-2 activations, 16 KB
  uint8_t a1[kPropTile * 16 * 2];  // features, 4 KB
  uint8_t w2[64 * 64 * 2];         // W2 (N = 64 outputs x K = 64), 8 KB
  uint8_t w1[64 * 16 * 2];         // W1 (N = 64 x K = 16, inputs 12..15 zero), 2 KB
  float b1[64], b2[64], w3[64], b3;
  uint64_t mbar;
  uint32_t tmem_base;
};

template <class F>
__global__ void __launch_bounds__(kPropTile) propose_start_tc_kernel(FitArgs a, F fld, float* __restrict__ h0) {
  __shared__ PropSmem sm;
  const int tid = threadIdx.x, warp = tid >> 5;
  // weights: BF16-representable FP32 values, converted exactly
  for (int e = tid; e < 64 * 16; e += kPropTile) {
    const int j = e >> 4, i = e & 15;
    const uint32_t b = i < 12 ? (__float_as_uint(a.mlp[j * 12 + i]) >> 16) : 0u;
    *reinterpret_cast<uint16_t*>(sm.w1 + core_offset(j, i, 2)) = uint16_t(b);
  }
  for (int e = tid; e < 64 * 64; e += kPropTile) {
    const int j = e >> 6, i = e & 63;
    *reinterpret_cast<uint16_t*>(sm.w2 + core_offset(j, i, 8)) = uint16_t(__float_as_uint(a.mlp[832 + e]) >> 16);
  }
  if (tid < 64) {
    sm.b1[tid] = a.mlp[768 + tid];
    sm.b2[tid] = a.mlp[4928 + tid];
    sm.w3[tid] = a.mlp[4992 + tid];
  }
  if (tid == 0) {
    sm.b3 = a.mlp[5056];
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(&sm.mbar)) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {  // 64 accumulator columns, reused by both layers
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 64;" ::"r"(smem_addr(&sm.tmem_base))
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  fence_async_smem();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = sm.tmem_base;
  const uint32_t t_row = tmem + (uint32_t(warp * 32) << 16);  // this warp's 32 lanes
  const uint64_t d_a1 = umma_desc(smem_addr(sm.a1), 128, 256), d_w1 = umma_desc(smem_addr(sm.w1), 128, 256);
  uint32_t phase = 0;
  bool failed = false;
  const uint32_t n = a.n_tracks, n_tiles = (n + kPropTile - 1) / kPropTile;

  uint32_t tile = blockIdx.x;
  for (; tile < n_tiles && !failed; tile += gridDim.x) {
    const uint32_t i = tile * kPropTile + tid;
    bool ok = false;
    float x[12] = {0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f};
    if (i < n) {
      const uint32_t b0 = a.offsets[i], b1 = a.offsets[i + 1];
      const uint32_t id0 = b1 >= b0 + 2 && b1 <= a.n_meas ? a.sid[b0] & ~TKF_SID_NO_MEASUREMENT : a.n_surf;
      const uint32_t id1 = b1 >= b0 + 2 && b1 <= a.n_meas ? a.sid[b0 + 1] & ~TKF_SID_NO_MEASUREMENT : a.n_surf;
      ok = id0 < a.n_surf && id1 < a.n_surf;
      if (ok) {
        Surf s0, s1;
        load_surf(a.surf, id0, s0);
        load_surf(a.surf, id1, s1);
        float p[5];
        for (int j = 0; j < 5; ++j) p[j] = float(a.seed_par[size_t(j) * a.stride + i]);
        float sph, cph, sth, cth;
        sincosf(p[2], &sph, &cph);
        sincosf(p[3], &sth, &cth);
        const float Tf[3] = {sth * cph, sth * sph, cth};
        // position relative to the target surface's origin, FP32 (features are BF16 anyway)
        float d[3], rf[3];
        for (int j = 0; j < 3; ++j) {
          rf[j] = float(s0.c[j]) + p[0] * s0.uf[j] + p[1] * s0.vf[j];
          d[j] = float(s0.c[j] - s1.c[j]) + p[0] * s0.uf[j] + p[1] * s0.vf[j];
        }
        float B[3];
        bool oof = false;
        fld.atf(rf, B, oof);
        const float sl = -(s1.nf[0] * d[0] + s1.nf[1] * d[1] + s1.nf[2] * d[2]) /
                         (s1.nf[0] * Tf[0] + s1.nf[1] * Tf[1] + s1.nf[2] * Tf[2]);
        x[0] = (s1.uf[0] * d[0] + s1.uf[1] * d[1] + s1.uf[2] * d[2]) * 1e-3f;
        x[1] = (s1.vf[0] * d[0] + s1.vf[1] * d[1] + s1.vf[2] * d[2]) * 1e-3f;
        x[2] = (s1.nf[0] * d[0] + s1.nf[1] * d[1] + s1.nf[2] * d[2]) * 1e-3f;
        x[3] = s1.uf[0] * Tf[0] + s1.uf[1] * Tf[1] + s1.uf[2] * Tf[2];
        x[4] = s1.vf[0] * Tf[0] + s1.vf[1] * Tf[1] + s1.vf[2] * Tf[2];
        x[5] = s1.nf[0] * Tf[0] + s1.nf[1] * Tf[1] + s1.nf[2] * Tf[2];
        x[6] = p[4];
        x[7] = B[0] * 0.5f;
        x[8] = B[1] * 0.5f;
        x[9] = B[2] * 0.5f;
        x[10] = logf(a.opt.h_max_f) * 0.2f;
        x[11] = fminf(fmaxf(sl * 1e-3f, -2.0f), 2.0f);
        for (int j = 0; j < 12; ++j) ok = ok && isfinite(x[j]);
        if (!ok)
          for (int j = 0; j < 12; ++j) x[j] = 0.0f;
      }
    }
    {  // row tid of A1: two 16-byte chunks (K 0..7, 8..15)
      uint4 c0, c1;
      c0.x = bf16_rne(x[0]) | (bf16_rne(x[1]) << 16);
      c0.y = bf16_rne(x[2]) | (bf16_rne(x[3]) << 16);
      c0.z = bf16_rne(x[4]) | (bf16_rne(x[5]) << 16);
      c0.w = bf16_rne(x[6]) | (bf16_rne(x[7]) << 16);
      c1.x = bf16_rne(x[8]) | (bf16_rne(x[9]) << 16);
      c1.y = bf16_rne(x[10]) | (bf16_rne(x[11]) << 16);
      c1.z = 0u;
      c1.w = 0u;
      *reinterpret_cast<uint4*>(sm.a1 + core_offset(tid, 0, 2)) = c0;
      *reinterpret_cast<uint4*>(sm.a1 + core_offset(tid, 8, 2)) = c1;
    }
    fence_async_smem();
    tc_fence_before();
    __syncthreads();
    if (tid == 0 && !a.test_stall_proposals) {
      tc_fence_after();
      tc_mma(tmem, d_a1, d_w1, 0u);
      tc_commit(&sm.mbar);
    }
    bool done = mbar_wait(&sm.mbar, phase);
    phase ^= 1u;
    __syncwarp();  // the tensor-memory loads are warp-collective
    tc_fence_after();
    float v[32];
#pragma unroll
    for (int half = 0; half < 2; ++half) {
      tmem_ld32(t_row + uint32_t(half * 32), v);
#pragma unroll
      for (int q = 0; q < 4; ++q) {  // K groups 4 half + q of A2's row tid
        uint32_t w[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          const int j0 = half * 32 + q * 8 + 2 * e;
          const float z0 = v[q * 8 + 2 * e] + sm.b1[j0], z1 = v[q * 8 + 2 * e + 1] + sm.b1[j0 + 1];
          w[e] = bf16_rne(silu_f(z0)) | (bf16_rne(silu_f(z1)) << 16);
        }
        *reinterpret_cast<uint4*>(sm.a2 + core_offset(tid, half * 32 + q * 8, 8)) = make_uint4(w[0], w[1], w[2], w[3]);
      }
    }
    fence_async_smem();
    tc_fence_before();
    __syncthreads();
    if (tid == 0 && !a.test_stall_proposals) {
      tc_fence_after();
#pragma unroll
      for (int k = 0; k < 4; ++k)
        tc_mma(tmem, umma_desc(smem_addr(sm.a2) + k * 256, 128, 1024), umma_desc(smem_addr(sm.w2) + k * 256, 128, 1024),
               k > 0 ? 1u : 0u);
      tc_commit(&sm.mbar);
    }
    done = mbar_wait(&sm.mbar, phase) && done;
    phase ^= 1u;
    __syncwarp();
    tc_fence_after();
    float out = sm.b3;
#pragma unroll
    for (int half = 0; half < 2; ++half) {
      tmem_ld32(t_row + uint32_t(half * 32), v);
#pragma unroll
      for (int k = 0; k < 32; ++k) out = fmaf(sm.w3[half * 32 + k], silu_f(v[k] + sm.b2[half * 32 + k]), out);
    }
    tc_fence_before();
    failed = __syncthreads_or(!done) != 0;
    if (i < n) {
      float h = a.opt.h_max_f;
      if (ok) {
        const float q = 0.9f * expf(rintf(out * 32.0f) * (1.0f / 32.0f));
        h = isfinite(q) ? fminf(fmaxf(q, a.opt.h_min_f), a.opt.h_max_f) : a.opt.h_max_f;
      }
      h0[i] = failed ? -1.0f : h;  // -1: no proposal (the fit starts from h_max and flags it)
    }
  }
  if (failed) {  // the tiles this CTA did not reach get no proposal either
    for (; tile < n_tiles; tile += gridDim.x) {
      const uint32_t i = tile * kPropTile + tid;
      if (i < n) h0[i] = -1.0f;
    }
    mbar_wait(&sm.mbar, phase ^ 1u);  // give an MMA still in flight a bounded time to finish
  }
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 64;" ::"r"(tmem) : "memory");
  }
}

template <class F>
cudaError_t launch_propose(const FitArgs& a, const F& fld, float* h0, cudaStream_t stream) {
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  const uint32_t tiles = (a.n_tracks + kPropTile - 1) / kPropTile;
  const uint32_t grid = tiles < uint32_t(4 * sms) ? tiles : uint32_t(4 * sms);
  propose_start_tc_kernel<<<grid, kPropTile, 0, stream>>>(a, fld, h0);
  return cudaGetLastError();
}

inline cudaError_t propose_fields(const FitArgs& a, const FieldDev& f, float* h0, cudaStream_t stream) {
  if (f.kind == TKF_FIELD_UNIFORM) {
    if (f.b[0] == 0.0 && f.b[1] == 0.0) return launch_propose(a, FieldUniformZ{f.b[2], float(f.b[2])}, h0, stream);
    return launch_propose(a, FieldUniform{{f.b[0], f.b[1], f.b[2]}, {float(f.b[0]), float(f.b[1]), float(f.b[2])}}, h0,
                          stream);
  }
  return launch_propose(a, grid_policy(f), h0, stream);
}

// Launches the persistent fit for one precision, step mode, lanes a track, smoother and field.
template <int kPrec, int kMode, int kRegs, int kG, int kSmooth, class F>
cudaError_t launch_persistent(const FitArgs& a, const F& fld, const uint32_t* perm, uint32_t* counter,
                              LaunchShape shape, cudaStream_t stream) {
  if (shape.threads > reg_block_threads(kRegs) || shape.tracks_per_warp * kG > 32) return cudaErrorInvalidConfiguration;
  const int place = kPrec == 2 ? 0 : reg_state_place(kRegs);
  const size_t smem = size_t(shape.threads) * state_doubles(place) * sizeof(double);
  fit_persistent_kernel<kPrec, kMode, kRegs, kG, kSmooth>
      <<<shape.blocks, shape.threads, smem, stream>>>(a, fld, perm, counter, uint32_t(shape.tracks_per_warp));
  return cudaGetLastError();
}

// Record capture (training only) is built with the full register file and one lane a track; the
// all-states mode with one lane a track at every register cap.
template <int kPrec, int kRegs, int kG, int kSmooth, class F>
cudaError_t launch_mode(const FitArgs& a, const F& fld, int mode, const uint32_t* perm, uint32_t* counter,
                        LaunchShape shape, cudaStream_t stream) {
  if (mode == kLearned)
    return launch_persistent<kPrec, kLearned, kRegs, kG, kSmooth>(a, fld, perm, counter, shape, stream);
  if (mode == kRecord) {
    if constexpr (kRegs == 255 && kPrec != 2 && kG == 1 && kSmooth == 0)
      return launch_persistent<kPrec, kRecord, kRegs, kG, kSmooth>(a, fld, perm, counter, shape, stream);
    return cudaErrorInvalidValue;
  }
  if (mode == kStates) {  // all-states output: one lane a track, RTS, any register cap
    if constexpr (kG == 1 && kSmooth == 0)
      return launch_persistent<kPrec, kStates, kRegs, kG, kSmooth>(a, fld, perm, counter, shape, stream);
    return cudaErrorInvalidValue;
  }
  return launch_persistent<kPrec, kPlain, kRegs, kG, kSmooth>(a, fld, perm, counter, shape, stream);
}

template <int kPrec, int kRegs, int kG = 1, int kSmooth = 0>
cudaError_t launch_fields(const FitArgs& a, const FieldDev& f, int mode, const uint32_t* perm, uint32_t* counter,
                          LaunchShape shape, cudaStream_t stream) {
  if (f.kind == TKF_FIELD_UNIFORM) {
    if (f.b[0] == 0.0 && f.b[1] == 0.0)
      return launch_mode<kPrec, kRegs, kG, kSmooth>(a, FieldUniformZ{f.b[2], float(f.b[2])}, mode, perm, counter, shape,
                                           stream);
    return launch_mode<kPrec, kRegs, kG, kSmooth>(
        a, FieldUniform{{f.b[0], f.b[1], f.b[2]}, {float(f.b[0]), float(f.b[1]), float(f.b[2])}}, mode, perm, counter,
        shape, stream);
  }
  return launch_mode<kPrec, kRegs, kG, kSmooth>(a, grid_policy(f), mode, perm, counter, shape, stream);
}

}  // namespace
}  // namespace tkf
