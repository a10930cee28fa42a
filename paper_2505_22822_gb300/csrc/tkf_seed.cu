// tkf_seed.cu -- track parameter estimation: the starting parameters of every track from the
// helix through three of its measurements (the step between seeding and track finding or
// fitting in the chain of Sec. 2; the paper prints no method, the construction and the prior
// covariance are stated in include/tkf.h at tkf_estimate_seeds).
//
// One thread per track, FP64 throughout. Per track the kernel reads its two offsets, its
// surface ids, three measurements (loc0, loc1, v00, v01, v11: 40 bytes each) and writes 20
// doubles and a status word (164 bytes); surfaces and the field grid are small and stay in
// L1/L2. The measurement loads are gathers (one 8-byte value per 32-byte sector and array), so
// the DRAM traffic of the inputs is set by sectors, not bytes.

#include "tkf_fit_impl.cuh"

namespace tkf {
namespace {

constexpr int kSeedBlock = 256;

// The FP64 pipe bounds this kernel (a warp instruction holds it for 16 SM cycles on GB300),
// so the arithmetic below takes one reciprocal where the plain formulas divide repeatedly,
// sin(theta) from the arc and dz instead of a sine, and the Highland factor of a surface from
// its record (computed once when the geometry is created).

// phi, theta and q/p at point r1 of the helix (axis z, field bz) through r1, r2, r3 in the
// order of travel; also the radius (0 without curvature) and sin(theta). Returns
// TKF_SEED_NO_CURVATURE for collinear points or bz = 0.
__device__ uint32_t helix_three_points(const double r1[3], const double r2[3], const double r3[3], double bz,
                                       double out[3], double& radius, double& sin_theta) {
  const double ax = r2[0] - r1[0], ay = r2[1] - r1[1];
  const double bx = r3[0] - r1[0], by = r3[1] - r1[1];
  const double a2 = ax * ax + ay * ay, b2 = bx * bx + by * by;
  const double area2 = 2.0 * (ax * by - ay * bx);  // > 0: counterclockwise seen from +z
  const double dz = r3[2] - r1[2];
  double tx, ty, arc;
  uint32_t st = 0;
  if (!(fabs(area2) > 1e-12 * (a2 + b2)) || bz == 0.0) {
    st = TKF_SEED_NO_CURVATURE;
    arc = sqrt(b2);
    const double inv = 1.0 / arc;
    tx = bx * inv;
    ty = by * inv;
    radius = 0.0;
    out[2] = 0.0;
  } else {
    // circumcentre relative to r1, from |c|^2 = |c - a|^2 = |c - b|^2
    const double inv_area2 = 1.0 / area2;
    const double cx = (by * a2 - ay * b2) * inv_area2;
    const double cy = (ax * b2 - bx * a2) * inv_area2;
    const double R = sqrt(cx * cx + cy * cy);
    const double turn_over_R = (area2 > 0.0 ? 1.0 : -1.0) / R;
    tx = cy * turn_over_R;  // tangent: the radius vector -c rotated by +-90 degrees
    ty = -cx * turn_over_R;
    // signed angle swept from r1 to r3 about the centre, in the sense of travel, in [0, 2 pi)
    const double ux = -cx, uy = -cy, wx = bx - cx, wy = by - cy;
    double swept = atan2((area2 > 0.0 ? 1.0 : -1.0) * (ux * wy - uy * wx), ux * wx + uy * wy);
    if (swept < 0.0) swept += 2.0 * kPi;
    arc = R * swept;
    radius = R;
    // a positive charge circles clockwise about +z when bz > 0 (F = q v x B); p = p_T / sin(theta)
    const double charge = (area2 > 0.0) == (bz > 0.0) ? -1.0 : 1.0;
    out[2] = charge * arc / (kKappa * fabs(bz) * R * sqrt(arc * arc + dz * dz));
  }
  out[0] = atan2(ty, tx);
  out[1] = atan2(arc, dz);
  sin_theta = arc / sqrt(arc * arc + dz * dz);
  return st;
}

template <class F>
__device__ uint32_t seed_one(const SeedArgs& a, const F& fld, uint32_t i, double par[5], double cov[15]) {
  const double nan = __longlong_as_double(0x7ff8000000000000LL);
  for (int j = 0; j < 5; ++j) par[j] = nan;
  for (int j = 0; j < 15; ++j) cov[j] = 0.0;
  const uint32_t b0 = a.offsets[i], b1 = a.offsets[i + 1];
  if (b1 < b0 || b1 > a.n_meas) return TKF_SEED_BAD_INPUT;
  const uint32_t N = b1 - b0;
  // entries without a measurement (holes, passive surfaces) give no space point; the first
  // entry carries the seed and needs its measurement
  // (no early exit inside the scan, so that the unrolled loads are all in flight together)
  uint32_t M = 0;
  bool bad = false;
#pragma unroll 4
  for (uint32_t e = 0; e < N; ++e) {
    const uint32_t sid = __ldg(a.sid + b0 + e);
    bad |= (sid & ~TKF_SID_NO_MEASUREMENT) >= a.n_surf;
    M += (sid >> 31) ^ 1u;
  }
  if (bad || (N > 0 && (__ldg(a.sid + b0) & TKF_SID_NO_MEASUREMENT))) return TKF_SEED_BAD_INPUT;
  if (M < 3) return TKF_SEED_TOO_FEW_HITS;
  // the measured entries number 0, j1, j2 of the M
  const uint32_t j1 = a.first_three ? 1u : (M - 1) / 2, j2 = a.first_three ? 2u : M - 1;
  uint32_t m[3] = {b0, b0, b0};
  if (M == N) {
    m[1] = b0 + j1;
    m[2] = b0 + j2;
  } else {
    for (uint32_t e = 0, c = 0; e < N; ++e) {
      if (a.sid[b0 + e] & TKF_SID_NO_MEASUREMENT) continue;
      if (c == j1) m[1] = b0 + e;
      if (c == j2) m[2] = b0 + e;
      ++c;
    }
  }
  double r[3][3], bzs[3], sh2 = 0.0, highland = 0.0;
  for (int j = 0; j < 3; ++j) {
    const uint32_t id = a.sid[m[j]];
    const double* rec = a.surf + size_t(id) * kSurfStride;
    const double l0 = a.loc0[m[j]], l1 = a.loc1[m[j]];
    for (int c = 0; c < 3; ++c) r[j][c] = __ldg(rec + 9 + c) + l0 * __ldg(rec + c) + l1 * __ldg(rec + 3 + c);
    double B[3];
    bool oof = false;
    fld.at(r[j], B, oof);
    bzs[j] = B[2];
    sh2 += (a.v00[m[j]] + a.v11[m[j]]) * (1.0 / 6.0);
    if (j == 0) highland = __ldg(rec + 15);
  }
  const double bz = (bzs[0] + bzs[1] + bzs[2]) * (1.0 / 3.0);
  double h[3], R, sin_theta;
  const uint32_t st = helix_three_points(r[0], r[1], r[2], bz, h, R, sin_theta);
  par[0] = a.loc0[b0];
  par[1] = a.loc1[b0];
  par[2] = h[0];
  par[3] = h[1];
  par[4] = h[2];

  // prior covariance: see tkf_estimate_seeds in include/tkf.h
  const double dx = r[2][0] - r[0][0], dy = r[2][1] - r[0][1], dz = r[2][2] - r[0][2];
  const double lt2 = dx * dx + dy * dy, l2 = lt2 + dz * dz;
  const double inv_lt2 = 1.0 / lt2;
  const double th0 = st == 0 ? 0.0136 * fabs(h[2]) * highland : 0.0136 * highland;  // 1 GeV without curvature
  const double ms2 = double(m[2] - m[0]) * th0 * th0;
  const double inv_s2 = 1.0 / (sin_theta * sin_theta);
  double var_phi = 64.0 * sh2 * inv_lt2 + 2.0 * ms2 * inv_s2;
  double var_qop = 1.0;
  if (st == 0) {
    // sagitta s = lt2 / 8R: 1 / s^2 = 64 R^2 / lt2^2
    const double inv_sag2 = 64.0 * R * R * inv_lt2 * inv_lt2;
    const double spread = (fmax(bzs[0], fmax(bzs[1], bzs[2])) - fmin(bzs[0], fmin(bzs[1], bzs[2]))) / bz;
    const double rel2 = (4.0 * sh2 + ms2 * lt2 * (1.0 / 16.0)) * inv_sag2 + spread * spread + 1e-4;
    var_qop = rel2 * h[2] * h[2];
    var_phi += lt2 / (4.0 * R * R) * rel2;
  }
  const double pi2 = kPi * kPi;
  cov[S(0, 0)] = a.v00[b0];
  cov[S(0, 1)] = a.v01[b0];
  cov[S(1, 1)] = a.v11[b0];
  cov[S(2, 2)] = fmin(var_phi, pi2);
  cov[S(3, 3)] = fmin(16.0 * sh2 / l2 + 2.0 * ms2, pi2);
  cov[S(4, 4)] = var_qop;
  return st;
}

template <class F>
__global__ void __launch_bounds__(kSeedBlock) estimate_seeds_kernel(const SeedArgs a, const F fld) {
  const uint32_t n = a.n_tracks;
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    double par[5], cov[15];
    const uint32_t st = seed_one(a, fld, i, par, cov);
    for (int j = 0; j < 5; ++j) a.par[size_t(j) * n + i] = par[j];
    for (int j = 0; j < 15; ++j) a.cov[size_t(j) * n + i] = cov[j];
    a.status[i] = st;
  }
}

// One wave of resident blocks (grid-stride beyond it), so that no partial last wave idles SMs.
template <class F>
cudaError_t launch_seeds(const SeedArgs& a, const F& fld, int sm_count, cudaStream_t stream) {
  int per_sm = 0;
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, estimate_seeds_kernel<F>, kSeedBlock, 0);
  if (e != cudaSuccess) return e;
  const uint32_t need = (a.n_tracks + kSeedBlock - 1) / kSeedBlock;
  const uint32_t wave = uint32_t(sm_count > 0 ? sm_count : 1) * uint32_t(per_sm > 0 ? per_sm : 1);
  estimate_seeds_kernel<<<need < wave ? need : wave, kSeedBlock, 0, stream>>>(a, fld);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_estimate_seeds(const SeedArgs& a, const FieldDev& f, int sm_count, cudaStream_t stream) {
  if (f.kind == TKF_FIELD_UNIFORM) {
    if (f.b[0] == 0.0 && f.b[1] == 0.0) return launch_seeds(a, FieldUniformZ{f.b[2], float(f.b[2])}, sm_count, stream);
    return launch_seeds(a, FieldUniform{{f.b[0], f.b[1], f.b[2]}, {float(f.b[0]), float(f.b[1]), float(f.b[2])}},
                        sm_count, stream);
  }
  return launch_seeds(a, grid_policy(f), sm_count, stream);
}

}  // namespace tkf
