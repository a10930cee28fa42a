// tkf_ckf.cu -- track finding with a combinatorial Kalman filter (the step of the chain of
// Sec. 2 between seeding and fitting; the algorithm and the navigation read for this library
// are stated in include/tkf.h at tkf_find_tracks).
//
// The search runs as phases over all seeds (below): the fit's RKN propagation, material and
// gain-matrix update; FP64 throughout, or (kMixed) with the propagation, material and covariance
// transport in FP32 around FP64 anchors as in the fit's mixed path (navigation, gate and update
// decide in FP64; FP32 screens with error bounds skip FP64 evaluations whose outcome is already
// certain). A seed's branches live in a workspace of global memory (a branch: state, direction,
// covariance and counters, 240 bytes); a branch's entries are not copied with it: each entry is a
// node of the seed's history tree (surface, measurement, parent node), written once when the
// beam keeps the branch, and the candidate's entries are read back along the parent links. The
// navigation tables are built once a call and copied into each prediction block's shared memory;
// the module records and measurements are gathered through L1/L2.

#include "tkf_fit_impl.cuh"

namespace tkf {
namespace {

constexpr int kCkfChildren = 3;         // measurements a branch may take on one surface
constexpr int kCkfMaxLayers = 32;
constexpr int kCkfBlock = 128;
// RKN attempts a propagation to the next module may take: a branch whose state cannot reach
// the module in as many (a seed with far too low a momentum curls) excludes it
constexpr uint32_t kCkfMaxSteps = 100;

struct CkfBranch {
  double p[5];     // l0, l1, (angle increments, 0 between steps), q/p
  double dir[4];   // filtered direction: sin phi, cos phi, sin theta, cos theta
  double C[15];
  double h_ctrl, chi2;
  uint32_t n_meas, holes, n_entries, order;
  int32_t sid;     // current surface, -1 before the seed surface
  int32_t node;    // history node of its last entry (-1: no entry yet)
  uint32_t e_sid;  // a child's own entry (surface, measurement or -1), made into a node when
  int32_t e_meas;  // the beam keeps the child
};

// An entry of a seed's history tree: node (step, q) is the entry of the q-th branch the beam
// kept after that step.
struct CkfNode {
  uint32_t sid;
  int32_t meas;
  int32_t parent;  // node of the previous entry, -1: none
};

// Per seed: two areas of children (a step's beam lives in one, its children are written to the
// other), then the best ended branch.
__host__ __device__ __forceinline__ uint32_t area_slots(uint32_t beam) { return beam * (kCkfChildren + 1); }
__host__ __device__ __forceinline__ uint32_t slots_per_seed(uint32_t beam) { return 2 * area_slots(beam) + 1; }
__host__ __device__ __forceinline__ uint32_t ckf_steps(uint32_t max_entries) { return max_entries + 2; }

// ranking of branches: more measurements, fewer consecutive holes, lower chi2, created earlier
__device__ __forceinline__ bool better(const CkfBranch& a, const CkfBranch& b) {
  if (a.n_meas != b.n_meas) return a.n_meas > b.n_meas;
  if (a.holes != b.holes) return a.holes < b.holes;
  if (a.chi2 != b.chi2) return a.chi2 < b.chi2;
  return a.order < b.order;
}

__device__ __forceinline__ void copy_branch(CkfBranch& d, const CkfBranch& s) {
  for (int j = 0; j < 5; ++j) d.p[j] = s.p[j];
  for (int j = 0; j < 4; ++j) d.dir[j] = s.dir[j];
  for (int j = 0; j < 15; ++j) d.C[j] = s.C[j];
  d.h_ctrl = s.h_ctrl;
  d.chi2 = s.chi2;
  d.n_meas = s.n_meas;
  d.holes = s.holes;
  d.n_entries = s.n_entries;
  d.order = s.order;
  d.sid = s.sid;
  d.node = s.node;
  d.e_sid = s.e_sid;
  d.e_meas = s.e_meas;
}

constexpr int kCkfMaxRings = 256;  // ring rows kept in shared memory (more: read from global)

// Navigation tables of a block, in shared memory: the layer rows, the ring rows (when they fit),
// the barrel layers' outer face radii, and the layer ids in the order in which a straight line
// meets them: barrel layers by face radius, disks by face z (ties: lower id first). The FP32
// screens read their operands from FP32 rows, the same values as converting the FP64 rows at each
// use: per layer float(n_phi / 2 pi) (barrels), the pitch, the inner radius (disks) and the
// modules' half extents, the outer face radius (barrels), the radial extent test's bounds (disks);
// per ring float(n_phi / 2 pi).
constexpr int kLayF = 8;  // floats a layer: phi bins a radian, pitch, r_inner, half_u, half_v, face_r,
                          // then the extent test's bounds: barrels n_rows row_pitch / 2 + 10, 0;
                          // disks r_inner - 10, r_inner + n_rings ring_pitch + 10
struct alignas(16) NavTables {
  double lay[kCkfMaxLayers * 8];
  double ring[kCkfMaxRings * 4];
  double face_r[kCkfMaxLayers];
  float lay_f[kCkfMaxLayers * kLayF];
  float ring_f[kCkfMaxRings];
  const double* rings;     // `ring`, or the global table when it does not fit
  const float* rings_f;    // `ring_f`, or NULL when the rings do not fit
  int bar[kCkfMaxLayers], dsk[kCkfMaxLayers];
  int nbar, ndsk;
};

__device__ __forceinline__ float phi_bins_per_radian(double n_phi) { return float(n_phi / (2.0 * kPi)); }

// outer face radius of a barrel layer (its flat modules reach sqrt((r + 1)^2 + half_u^2))
__device__ __forceinline__ double barrel_face(const double* l) { return sqrt((l[1] + 1.0) * (l[1] + 1.0) + l[6] * l[6]); }

__device__ void build_nav_tables(const CkfArgs& a, NavTables& nt) {
  const bool ring_fit = a.n_rings <= uint32_t(kCkfMaxRings);
  for (uint32_t j = threadIdx.x; j < 8 * a.n_layers; j += blockDim.x) nt.lay[j] = a.layers[j];
  if (ring_fit)
    for (uint32_t j = threadIdx.x; j < 4 * a.n_rings; j += blockDim.x) nt.ring[j] = a.rings[j];
  if (threadIdx.x == 0) {
    nt.rings = ring_fit ? nt.ring : a.rings;
    nt.rings_f = ring_fit ? nt.ring_f : nullptr;
  }
  __syncthreads();
  for (uint32_t li = threadIdx.x; li < a.n_layers; li += blockDim.x) {
    const double* l = nt.lay + 8 * li;
    nt.face_r[li] = l[0] == 0.0 ? barrel_face(l) : 0.0;
    float* lf = nt.lay_f + kLayF * li;
    lf[0] = l[0] == 0.0 ? phi_bins_per_radian(double(int(l[2]))) : 0.0f;
    lf[1] = d2f(l[4]);
    lf[2] = d2f(l[5]);
    lf[3] = d2f(l[6]);
    lf[4] = d2f(l[7]);
    lf[5] = d2f(nt.face_r[li]);
    lf[6] = l[0] == 0.0 ? d2f(0.5 * l[3] * l[4] + 10.0) : d2f(l[5] - 10.0);
    lf[7] = l[0] == 0.0 ? 0.0f : d2f(l[5] + l[2] * l[4] + 10.0);
  }
  if (ring_fit)
    for (uint32_t k = threadIdx.x; k < a.n_rings; k += blockDim.x) nt.ring_f[k] = phi_bins_per_radian(double(int(nt.ring[4 * k + 1])));
  __syncthreads();
  if (threadIdx.x == 0) {
    int nb = 0, nd = 0;
    for (uint32_t li = 0; li < a.n_layers; ++li) {  // insertion in id order: stable for ties
      const double* l = nt.lay + 8 * li;
      if (l[0] == 0.0) {
        int pos = nb++;
        for (; pos > 0 && nt.face_r[nt.bar[pos - 1]] > nt.face_r[li]; --pos) nt.bar[pos] = nt.bar[pos - 1];
        nt.bar[pos] = int(li);
      } else {
        const double z = l[1] + (l[1] > 0.0 ? 1.0 : -1.0);
        int pos = nd++;
        for (; pos > 0; --pos) {
          const double* lp = nt.lay + 8 * nt.dsk[pos - 1];
          if (!(lp[1] + (lp[1] > 0.0 ? 1.0 : -1.0) > z)) break;
          nt.dsk[pos] = nt.dsk[pos - 1];
        }
        nt.dsk[pos] = int(li);
      }
    }
    nt.nbar = nb;
    nt.ndsk = nd;
  }
  __syncthreads();
}

__device__ __forceinline__ void module_half(const CkfArgs& a, const NavTables& nt, uint32_t id, double& hu,
                                            double& hv) {
  const int li = a.layer_of[id];
  hu = li >= 0 ? nt.lay[8 * li + 6] : 1e300;
  hv = li >= 0 ? nt.lay[8 * li + 7] : 1e300;
}

// floor(v) from an FP32 evaluation vf within `err` of the FP64 value v: decided (true, in `out`)
// when vf lies farther than err from every integer, so that floor(v) = floor(vf); else the
// caller evaluates v in FP64. (vf - floor(vf) and floor(vf) + 1 - vf are exact for |vf| < 2^23.)
__device__ __forceinline__ bool floor_sure(float vf, float err, int& out) {
  const float f = floorf(vf);
  if (fabsf(vf) < 8388608.0f && vf - f > err && f + 1.0f - vf > err) {
    out = int(f);
    return true;
  }
  return false;
}

// ip0 + d taken modulo nphi, as ((ip0 + d) % nphi + nphi) % nphi
__device__ __forceinline__ uint32_t wrap_bin(int ip0, int d, int nphi) {
  int ip = ip0 + d;
  if (ip0 >= 0 && ip0 <= nphi) {
    if (ip < 0) ip += nphi;
    if (ip >= nphi) ip -= nphi;
    return uint32_t(ip);
  }
  return uint32_t((ip % nphi + nphi) % nphi);
}

// modules of layer li around the point q: phi bin and row (barrel) or ring (disk), +-1 each.
// Each bin index is floor() of an FP64 expression (the angle phi in [0, 2 pi) from atan2, the row
// z / pitch + rows / 2, the ring (hypot - r0) / pitch); it is first evaluated in FP32 with a bound
// on the difference from the FP64 value (the FP32 inputs, atan2f / hypotf within 3 ulp, the wrap
// by 2 pi and the products and sums: a few 1e-7 relative, bounded here by 4e-6 of the bin count
// or of the magnitudes), and the FP64 value is computed only when the FP32 one lies within that
// bound of a bin edge. Near phi = 0 the two may wrap differently (bin 0 against bin nphi): the
// modules +-1 around either are the same, taken in the same order.
__device__ __noinline__ int layer_candidates(const NavTables& nt, uint32_t li, const double q[3], uint32_t out[9]) {
  const double* l = nt.lay + 8 * li;
  const float phf0 = atan2f(d2f(q[1]), d2f(q[0]));
  const float phf = phf0 < 0.0f ? phf0 + float(2.0 * kPi) : phf0;
  double phi = -1.0;  // the FP64 angle in [0, 2 pi), on first need
  const float* lf = nt.lay_f + kLayF * li;
  auto phi_bin = [&](int nphi, float per_rad) -> int {
    int b;
    if (floor_sure(phf * per_rad + 0.5f, 4e-6f * float(nphi + 1), b)) return b;
    if (phi < 0.0) {
      phi = atan2(q[1], q[0]);
      if (phi < 0.0) phi += 2.0 * kPi;
    }
    return int(floor(phi / (2.0 * kPi / nphi) + 0.5));
  };
  int n = 0;
  if (l[0] == 0.0) {
    const int nphi = int(l[2]), nrows = int(l[3]);
    const int ip0 = phi_bin(nphi, lf[0]);
    const float zq = d2f(q[2]) / lf[1];
    int iz0;
    if (!floor_sure(zq + 0.5f * float(nrows), 4e-6f * (1.0f + fabsf(zq) + float(nrows)), iz0))
      iz0 = int(floor(q[2] / l[4] + 0.5 * nrows));
    for (int iz = iz0 - 1; iz <= iz0 + 1; ++iz) {
      if (iz < 0 || iz >= nrows) continue;
      for (int d = -1; d <= 1; ++d) out[n++] = uint32_t(l[5]) + uint32_t(iz * nphi) + wrap_bin(ip0, d, nphi);
    }
  } else {
    const int nr = int(l[2]);
    const float rq = hypotf(d2f(q[0]), d2f(q[1])), r0f = lf[2], pf = lf[1];
    int k0;
    if (!floor_sure((rq - r0f) / pf, 4e-6f * (1.0f + (rq + fabsf(r0f)) / pf), k0))
      k0 = int(floor((hypot(q[0], q[1]) - l[5]) / l[4]));
    for (int k = k0 - 1; k <= k0 + 1; ++k) {
      if (k < 0 || k >= nr) continue;
      const uint32_t row = uint32_t(l[3]) + uint32_t(k);
      const double* rg = nt.rings + 4 * row;
      const int nphi = int(rg[1]);
      const int ip0 = phi_bin(nphi, nt.rings_f ? nt.rings_f[row] : phi_bins_per_radian(double(nphi)));
      for (int d = -1; d <= 1; ++d) out[n++] = uint32_t(rg[2]) + wrap_bin(ip0, d, nphi);
    }
  }
  return n;
}

// straight-line path to the outer face of layer li if ahead and within its extent, else -1
// (face_r: the barrel layers' outer face radii, computed once a block). xf, Tf: FP32 copies of x
// and T for three screens that return -1 only where the FP64 evaluation surely does: a barrel face
// the point lies outside (|x_perp|^2 - r_face^2 >= 0); a barrel face reached beyond the layer's
// z extent; a disk face reached outside its radial extent. Each FP32 quantity is within a few
// 2^-24 of its magnitudes of the FP64 one (the copies, one rounding an operation, sqrtf and the
// division correctly rounded); the bounds below take 1e-6 relative (about 17 units) plus 1e-3 mm
// for the rounding of the stored bounds.
//
// The z extent: where the line, in its direction of travel, passes z_l = +-(z_max + 1e-3 mm +
// 1e-6 |z|), it is still surely inside the face radius. The squared distance from the axis is a
// convex function of the path, so from inside at the start (c < 0; else the FP64 test returns -1
// anyway) the face is met beyond z_l, past z_max by more than the FP64 rounding of x_z + s T_z.
// Reached at path (z_l - x_z) / T_z; the error of that path carries the rounding of z_l - x_z
// divided by |T_z| into the transverse position.
__device__ double layer_path(const NavTables& nt, uint32_t li, const double x[3], const double T[3],
                             const float xf[3], const float Tf[3]) {
  const double* l = nt.lay + 8 * li;
  const float* lf = nt.lay_f + kLayF * li;
  double s;
  if (l[0] == 0.0) {
    const float p2f = xf[0] * xf[0] + xf[1] * xf[1], f2f = lf[5] * lf[5];
    if (p2f - f2f > 1e-6f * (p2f + f2f)) return -1.0;
    if (Tf[2] != 0.0f) {
      const float zl = copysignf(lf[6] + 1e-3f + 1e-6f * fabsf(xf[2]), Tf[2]);
      const float dzf = zl - xf[2];
      if (Tf[2] > 0.0f ? dzf <= 0.0f : dzf >= 0.0f) return -1.0;  // beyond z_l already, moving away
      const float szf = dzf / Tf[2], tp = fabsf(Tf[0]) + fabsf(Tf[1]);
      const float px = fmaf(szf, Tf[0], xf[0]), py = fmaf(szf, Tf[1], xf[1]);
      const float rq = sqrtf(px * px + py * py);
      const float e = 1e-6f * (fabsf(xf[0]) + fabsf(xf[1]) + szf * tp + rq +
                               (fabsf(zl) + fabsf(xf[2])) * tp / fabsf(Tf[2])) + 1e-3f;
      if (rq + e < lf[5]) return -1.0;
    }
    const double aa = T[0] * T[0] + T[1] * T[1], b = x[0] * T[0] + x[1] * T[1];
    const double rf = nt.face_r[li];
    const double c = x[0] * x[0] + x[1] * x[1] - rf * rf;
    if (!(aa > 0.0) || c >= 0.0) return -1.0;
    s = (-b + sqrt(b * b - aa * c)) / aa;
    if (fabs(x[2] + s * T[2]) > 0.5 * l[3] * l[4] + 10.0) return -1.0;
  } else {
    const double dz = l[1] + (l[1] > 0.0 ? 1.0 : -1.0) - x[2];
    // behind or parallel (opposite or zero signs): the quotient would not be > 0
    if (!((dz > 0.0 && T[2] > 0.0) || (dz < 0.0 && T[2] < 0.0))) return -1.0;
    // the radius where the line meets the face, in FP32 (an overflow or NaN screens nothing)
    const float sf = d2f(dz) / Tf[2];
    const float px = fmaf(sf, Tf[0], xf[0]), py = fmaf(sf, Tf[1], xf[1]);
    const float rq = sqrtf(px * px + py * py);
    const float e = 1e-6f * (fabsf(xf[0]) + fabsf(xf[1]) + fabsf(sf) * (fabsf(Tf[0]) + fabsf(Tf[1])) + rq) + 1e-3f;
    if (rq + e < lf[6] || rq - e > lf[7]) return -1.0;
    s = dz / T[2];
    if (!(s > 0.0)) return -1.0;
    const double r = hypot(x[0] + s * T[0], x[1] + s * T[1]);
    if (r < l[5] - 10.0 || r > l[5] + l[2] * l[4] + 10.0) return -1.0;
  }
  return s > 0.0 ? s : -1.0;
}

__device__ __forceinline__ bool listed(const uint32_t* v, int n, uint32_t id) {
  for (int j = 0; j < n; ++j)
    if (v[j] == id) return true;
  return false;
}

// True when the parabola x + s T + s^2/2 k surely crosses the plane of a module outside its half
// extents plus the helix margin: an FP32 evaluation whose every rounding is covered by `err`
// (below), so that the FP64 test of nearest_crossed rejects the module too. `f`: the record's
// FP32 block (frame u, v, n at 0, 3, 6; centre c at 11); xf: the FP32 copy of x, xn its L1 norm.
// The offset d = c - x is formed in FP32 from the two copies: besides the rounding of the
// difference (relative 2^-24, as a conversion of the FP64 offset would have), it carries the
// copies' rounding, at most 2^-24 (|c|_1 + |x|_1) in L1 norm (ecx, taken twice over). That error
// moves q by as much, and the crossing's path by at most ecx / |an + bn s| <= 2 ecx / |an| (the
// screen keeps disc = (an + bn s)^2 above an^2 / 4; taken as 2.5 ecx / |an|). Grazing incidence
// (|n.T| <= 0.05) and near-tangent solutions (disc <= an^2 / 4) are left to FP64.
__device__ __forceinline__ bool surely_outside(const float* __restrict__ f, const float xf[3], float xn,
                                               const float Tf[3], const float kf[3], float knorm, float bendf,
                                               float huf, float hvf) {
  const float uf[3] = {f[0], f[1], f[2]}, vf[3] = {f[3], f[4], f[5]}, nf[3] = {f[6], f[7], f[8]};
  const float cf[3] = {f[11], f[12], f[13]};
  const float df[3] = {cf[0] - xf[0], cf[1] - xf[1], cf[2] - xf[2]};
  const float an = dotr(nf, Tf);
  if (!(fabsf(an) > 0.05f)) return false;
  const float dist = dotr(nf, df), bn = dotr(nf, kf);
  const float disc = an * an + 2.0f * bn * dist;
  if (!(disc > 0.25f * an * an)) return false;
  const float sf = 2.0f * dist / (an + copysignf(sqrtf(disc), an));
  if (!isfinite(sf)) return false;
  const float as = fabsf(sf), h = 0.5f * sf * sf;
  const float q[3] = {-df[0] + sf * Tf[0] + h * kf[0], -df[1] + sf * Tf[1] + h * kf[1], -df[2] + sf * Tf[2] + h * kf[2]};
  const float dn = fabsf(df[0]) + fabsf(df[1]) + fabsf(df[2]), qn = fabsf(q[0]) + fabsf(q[1]) + fabsf(q[2]);
  const float ecx = 1.2e-7f * (fabsf(cf[0]) + fabsf(cf[1]) + fabsf(cf[2]) + xn);
  // error of s: relative 1e-5 plus the propagated rounding of dist (through an and disc) and the
  // copies' error ecx, then that of q (d, the products, the sums) and of the projections
  const float rs = 1e-5f + 2e-6f * fabsf(bn) * dn / (an * an);
  const float ds = rs * as + (1e-5f * dn + 2.5f * ecx) / fabsf(an);
  const float err = 1e-3f + ecx + ds * (1.0f + (as + ds) * knorm) + 1e-6f * (dn + qn);
  const float sup = (as + ds) * 1.00001f;
  const float margin = (1.0f + sup * sup * sup * bendf * bendf / 6.0f) * 1.00001f;
  return fabsf(dotr(uf, q)) - err > huf + margin || fabsf(dotr(vf, q)) - err > hvf + margin;
}

// nearest of `cand` crossed by the parabola x + s T + s^2/2 k within bounds and margin
// (xf, Tf, kf: FP32 copies of x, T, k)
__device__ __noinline__ int nearest_crossed(const CkfArgs& a, const NavTables& nt, const uint32_t* cand, int nc,
                                            const double x[3], const double T[3], const double k[3], double bend,
                                            const float xf[3], const float Tf[3], const float kf[3],
                                            const uint32_t* skip, int nskip, double& s_out) {
  int best = -1;
  double best_s = 0.0;
  const float knorm = (fabsf(kf[0]) + fabsf(kf[1]) + fabsf(kf[2])) * 1.00001f, bendf = d2f(bend) * 1.00001f;
  const float xn = fabsf(xf[0]) + fabsf(xf[1]) + fabsf(xf[2]);
  for (int j = 0; j < nc; ++j) {
    const uint32_t id = cand[j];
    if (id >= a.n_surf || listed(skip, nskip, id)) continue;
    const double* rec = a.surf + size_t(id) * kSurfStride;
    // half extents of the module's layer (outside the layer structure: unbounded)
    const int li = a.layer_of[id];
    const float huf = li >= 0 ? nt.lay_f[kLayF * li + 3] : INFINITY, hvf = li >= 0 ? nt.lay_f[kLayF * li + 4] : INFINITY;
    if (surely_outside(reinterpret_cast<const float*>(rec + 16), xf, xn, Tf, kf, knorm, bendf, huf, hvf)) continue;
    const double hu = li >= 0 ? nt.lay[8 * li + 6] : 1e300, hv = li >= 0 ? nt.lay[8 * li + 7] : 1e300;
    const double c[3] = {rec[9], rec[10], rec[11]};
    const double d[3] = {c[0] - x[0], c[1] - x[1], c[2] - x[2]};
    const double u[3] = {rec[0], rec[1], rec[2]}, v[3] = {rec[3], rec[4], rec[5]};
    const double n[3] = {rec[6], rec[7], rec[8]};
    const double dist = dot3(n, d), an = dot3(n, T), bn = dot3(n, k);
    if (an == 0.0) continue;
    // the nearer root of an s + bn s^2 / 2 = dist, else (no real root, or an overflow) the
    // straight-line path dist / an
    double s;
    bool root = false;
    const double disc = an * an + 2.0 * bn * dist;
    if (disc >= 0.0) {
      const double q2 = 2.0 * dist / (an + copysign(sqrt(disc), an));
      if (isfinite(q2)) {
        s = q2;
        root = true;
      }
    }
    if (!root) s = dist / an;
    if (!(s > 1e-3)) continue;
    const double h = 0.5 * s * s;
    const double q[3] = {x[0] + s * T[0] + h * k[0] - c[0], x[1] + s * T[1] + h * k[1] - c[1],
                         x[2] + s * T[2] + h * k[2] - c[2]};
    const double margin = 1.0 + s * s * s * bend * bend / 6.0;
    if (fabs(dot3(u, q)) > hu + margin || fabs(dot3(v, q)) > hv + margin) continue;
    // crossings within 1e-6 mm of each other (coplanar overlapping modules): the lower id
    if (best < 0 || s < best_s - 1e-6 || (fabs(s - best_s) <= 1e-6 && id < uint32_t(best))) {
      best = int(id);
      best_s = s;
    }
  }
  s_out = best_s;
  return best;
}

// the next module from (x, T) on surface `cur`: the nearest crossing among the current layer's
// modules around x and the modules of the layers ahead, taken in order of face path (ties:
// lower index first) until a layer's face lies more than 20 mm beyond the nearest crossing
// found. A straight line meets the barrel faces in order of radius and the disk faces in
// order of z (ascending for T_z > 0, descending for T_z < 0), so the layers ahead come from
// merging those two orders, and a face path is computed only when the merge reaches it.
__device__ int navigate(const CkfArgs& a, int cur, const double x[3], const double T[3], const double k[3],
                        double bend, const uint32_t* skip, int nskip, const NavTables& nt) {
  uint32_t cand[9];
  int best = -1;
  double best_s = 0.0;
  const float xf[3] = {d2f(x[0]), d2f(x[1]), d2f(x[2])}, Tf[3] = {d2f(T[0]), d2f(T[1]), d2f(T[2])};
  const float kf[3] = {d2f(k[0]), d2f(k[1]), d2f(k[2])};
  const int cur_layer = cur >= 0 ? a.layer_of[cur] : -1;
  if (cur_layer >= 0) {
    uint32_t sk[5];
    for (int j = 0; j < nskip; ++j) sk[j] = skip[j];
    sk[nskip] = uint32_t(cur);
    const int nc = layer_candidates(nt, uint32_t(cur_layer), x, cand);
    best = nearest_crossed(a, nt, cand, nc, x, T, k, bend, xf, Tf, kf, sk, nskip + 1, best_s);
  }
  // the head of each order: the next layer ahead (face path > 0, within its extent) and its path
  int pb = 0, pd = 0, lb = -1, ld = -1;
  double sb = 0.0, sd = 0.0;
  const int dstep = T[2] > 0.0 ? 1 : -1;  // direction of the disk order
  int dpos = T[2] > 0.0 ? 0 : nt.ndsk - 1;
  const bool disks = T[2] != 0.0;
  auto next_barrel = [&]() {
    lb = -1;
    while (pb < nt.nbar) {
      const int li = nt.bar[pb++];
      if (li == cur_layer) continue;
      const double s = layer_path(nt, uint32_t(li), x, T, xf, Tf);
      if (s > 0.0) {
        lb = li;
        sb = s;
        return;
      }
    }
  };
  auto next_disk = [&]() {
    ld = -1;
    while (disks && pd < nt.ndsk) {
      const int li = nt.dsk[dpos];
      dpos += dstep;
      ++pd;
      if (li == cur_layer) continue;
      const double s = layer_path(nt, uint32_t(li), x, T, xf, Tf);
      if (s > 0.0) {
        ld = li;
        sd = s;
        return;
      }
    }
  };
  next_barrel();
  next_disk();
  while (lb >= 0 || ld >= 0) {
    const bool take_b = ld < 0 || (lb >= 0 && (sb < sd || (sb == sd && lb < ld)));
    const int pick = take_b ? lb : ld;
    const double sl = take_b ? sb : sd;
    if (best >= 0 && sl > best_s + 20.0) break;
    const double h = 0.5 * sl * sl;
    const double q[3] = {x[0] + sl * T[0] + h * k[0], x[1] + sl * T[1] + h * k[1], x[2] + sl * T[2] + h * k[2]};
    const int nc = layer_candidates(nt, uint32_t(pick), q, cand);
    double sm = 0.0;
    const int m = nearest_crossed(a, nt, cand, nc, x, T, k, bend, xf, Tf, kf, skip, nskip, sm);
    if (m >= 0 && (best < 0 || sm < best_s)) {
      best = m;
      best_s = sm;
    }
    if (take_b)
      next_barrel();
    else
      next_disk();
  }
  return best;
}

// From a branch's filtered state on its surface: material, navigation, RKN propagation and
// covariance transport to the next module; returns its id (-1: none ahead, or stopped).
template <bool kMixed, class F>
__device__ int predict(const CkfArgs& a, const F& fld, const NavTables& nt, const CkfBranch& br, double pp[5],
                       double pdir[4], double Cp[15], double& h_ctrl) {
  Surf sc;
  load_surf(a.surf, uint32_t(br.sid), sc);
  const double sph = br.dir[0], cph = br.dir[1], sth = br.dir[2], cth = br.dir[3];
  const double T0[3] = {sth * cph, sth * sph, cth};
  double lam = br.p[4], th0sq;
  if constexpr (kMixed) {
    const float Tm[3] = {d2f(T0[0]), d2f(T0[1]), d2f(T0[2])};
    float th0sq_f;
    if (material_mixed(sc, a.mat, a.opt, Tm, lam, th0sq_f) & ~(TKF_TRACK_OUT_OF_FIELD)) return -1;
    th0sq = f2d(th0sq_f);
  } else {
    if (material(sc, a.mat, a.opt.mass, T0, lam, th0sq) & ~(TKF_TRACK_OUT_OF_FIELD)) return -1;
  }
  double x[3];
  for (int j = 0; j < 3; ++j) x[j] = sc.c[j] + br.p[0] * sc.u[j] + br.p[1] * sc.v[j];
  double B[3];
  bool oof = false;
  fld.at(x, B, oof);
  const double bend = kKappa * fabs(lam) * sqrt(dot3(B, B));
  const double kc[3] = {kKappa * lam * (T0[1] * B[2] - T0[2] * B[1]), kKappa * lam * (T0[2] * B[0] - T0[0] * B[2]),
                        kKappa * lam * (T0[0] * B[1] - T0[1] * B[0])};
  uint32_t skip[4];
  int nskip = 0;
  for (int tries = 0; tries < 4; ++tries) {
    const int m = navigate(a, br.sid, x, T0, kc, bend, skip, nskip, nt);
    if (m < 0) return -1;
    Surf s;
    load_surf(a.surf, uint32_t(m), s);
    if constexpr (kMixed) {
      double r[3] = {x[0], x[1], x[2]}, T[3] = {T0[0], T0[1], T0[2]};
      const float fsth = d2f(sth), fcth = d2f(cth), fsph = d2f(sph), fcph = d2f(cph);
      float dr[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
      float dT[3][3] = {{-fsth * fsph, fsth * fcph, 0.0f}, {fcth * fcph, fcth * fsph, -fsth}, {0, 0, 0}};
      float kend[3], h = float(br.h_ctrl);
      uint32_t att = 0, rej = 0;
      StepLearn learn{nullptr, 0, nullptr, 0.0f};
      const uint32_t st =
          propagate_mixed<kPlain, 3>(fld, a.opt, s, s.nf, r, T, lam, dr, dT, 0.0f, h, att, rej, kend, learn);
      const double d[3] = {r[0] - s.c[0], r[1] - s.c[1], r[2] - s.c[2]};
      double hu, hv;
      module_half(a, nt, uint32_t(m), hu, hv);
      if ((st & ~TKF_TRACK_OUT_OF_FIELD) || fabs(dot3(s.u, d)) > hu || fabs(dot3(s.v, d)) > hv) {
        skip[nskip++] = uint32_t(m);
        continue;
      }
      // bound parameters (FP64 from the anchors) and the transport Jacobian in FP32
      const double inv_norm = 1.0 / sqrt(dot3(T, T));
      const double tn[3] = {T[0] * inv_norm, T[1] * inv_norm, T[2] * inv_norm};
      const double st2 = sqrt(tn[0] * tn[0] + tn[1] * tn[1]), inv_st = 1.0 / st2;
      const double ct2 = tn[2], cp2 = tn[0] * inv_st, sp2 = tn[1] * inv_st;
      const float Tf[3] = {d2f(T[0]), d2f(T[1]), d2f(T[2])};
      const float inv_nT = 1.0f / dotr(s.nf, Tf);
      const float fst = d2f(st2), fct = d2f(ct2), fcp = d2f(cp2), fsp = d2f(sp2), finv_st = d2f(inv_st);
      float J[5][5];
      for (int c = 0; c < 5; ++c) {
        float xx[3], tt[3], out[4];
        for (int j = 0; j < 3; ++j) {
          xx[j] = (c == 0) ? sc.uf[j] : (c == 1) ? sc.vf[j] : dr[c - 2][j];
          tt[j] = (c < 2) ? 0.0f : dT[c - 2][j];
        }
        jac_column(s.nf, s.uf, s.vf, Tf, kend, inv_nT, fsp, fcp, fst, fct, finv_st, xx, tt, out);
        for (int rr = 0; rr < 4; ++rr) J[rr][c] = out[rr];
        J[4][c] = (c == 4) ? 1.0f : 0.0f;
      }
      pp[0] = dot3(s.u, d);
      pp[1] = dot3(s.v, d);
      pp[2] = 0.0;  // the angles as the predicted direction (increments from here on)
      pp[3] = 0.0;
      pdir[0] = sp2;
      pdir[1] = cp2;
      pdir[2] = st2;
      pdir[3] = ct2;
      pp[4] = lam;
      float Cf[15];
      for (int j = 0; j < 15; ++j) Cf[j] = d2f(br.C[j]);
      Cf[S(2, 2)] += d2f(th0sq) / (fsth * fsth);
      Cf[S(3, 3)] += d2f(th0sq);
      transport_cov<1>(J, Cf, 0u, 0xffffffffu);
      for (int j = 0; j < 15; ++j) Cp[j] = f2d(Cf[j]);
      h_ctrl = double(h);
      return m;
    } else {
      double r[3] = {x[0], x[1], x[2]}, T[3] = {T0[0], T0[1], T0[2]};
      double dr[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
      double dT[3][3] = {{-sth * sph, sth * cph, 0.0}, {cth * cph, cth * sph, -sth}, {0, 0, 0}};
      double kend[3], h = br.h_ctrl;
      uint32_t att = 0, rej = 0;
      StepLearn learn{nullptr, 0, nullptr, 0.0f};
      const uint32_t st = propagate<kPlain, 3>(fld, a.opt, s, r, T, lam, dr, dT, 0.0, h, att, rej, kend, learn);
      const double d[3] = {r[0] - s.c[0], r[1] - s.c[1], r[2] - s.c[2]};
      double hu, hv;
      module_half(a, nt, uint32_t(m), hu, hv);
      if ((st & ~TKF_TRACK_OUT_OF_FIELD) || fabs(dot3(s.u, d)) > hu || fabs(dot3(s.v, d)) > hv) {
        skip[nskip++] = uint32_t(m);
        continue;
      }
      // bound parameters and the transport Jacobian at the target (path correction)
      const double inv_norm = 1.0 / sqrt(dot3(T, T));
      const double tn[3] = {T[0] * inv_norm, T[1] * inv_norm, T[2] * inv_norm};
      const double st2 = sqrt(tn[0] * tn[0] + tn[1] * tn[1]), inv_st = 1.0 / st2;
      const double ct2 = tn[2], cp2 = tn[0] * inv_st, sp2 = tn[1] * inv_st;
      const double inv_nT = 1.0 / dot3(s.n, T);
      double J[5][5];
      for (int c = 0; c < 5; ++c) {
        double xx[3], tt[3], out[4];
        for (int j = 0; j < 3; ++j) {
          xx[j] = (c == 0) ? sc.u[j] : (c == 1) ? sc.v[j] : dr[c - 2][j];
          tt[j] = (c < 2) ? 0.0 : dT[c - 2][j];
        }
        jac_column(s.n, s.u, s.v, T, kend, inv_nT, sp2, cp2, st2, ct2, inv_st, xx, tt, out);
        for (int rr = 0; rr < 4; ++rr) J[rr][c] = out[rr];
        J[4][c] = (c == 4) ? 1.0 : 0.0;
      }
      pp[0] = dot3(s.u, d);
      pp[1] = dot3(s.v, d);
      pp[2] = 0.0;  // the angles as the predicted direction (increments from here on)
      pp[3] = 0.0;
      pdir[0] = sp2;
      pdir[1] = cp2;
      pdir[2] = st2;
      pdir[3] = ct2;
      pp[4] = lam;
      for (int j = 0; j < 15; ++j) Cp[j] = br.C[j];
      Cp[S(2, 2)] += th0sq / (sth * sth);
      Cp[S(3, 3)] += th0sq;
      transport_cov<1>(J, Cp, 0u, 0xffffffffu);
      h_ctrl = h;
      return m;
    }
  }
  return -1;
}

// predicted chi2 of a measurement (no update)
__device__ __forceinline__ bool meas_chi2(const double pp[5], const double Cp[15], double m0, double m1, double V00,
                                          double V01, double V11, double& chi2) {
  const double S00 = Cp[S(0, 0)] + V00, S01 = Cp[S(0, 1)] + V01, S11 = Cp[S(1, 1)] + V11;
  const double det = S00 * S11 - S01 * S01;
  if (!(S00 > 0.0 && det > 0.0)) return false;
  const double idet = 1.0 / det;
  const double Si00 = S11 * idet, Si01 = -S01 * idet, Si11 = S00 * idet;
  const double r0 = m0 - pp[0], r1 = m1 - pp[1];
  chi2 = r0 * (Si00 * r0 + Si01 * r1) + r1 * (Si01 * r0 + Si11 * r1);
  return true;
}

// gain-matrix update, Joseph form (as in the fit)
__device__ void update(double p[5], double C[15], double m0, double m1, double V00, double V01, double V11,
                       double& chi2) {
  const double S00 = C[S(0, 0)] + V00, S01 = C[S(0, 1)] + V01, S11 = C[S(1, 1)] + V11;
  const double idet = 1.0 / (S00 * S11 - S01 * S01);
  const double Si00 = S11 * idet, Si01 = -S01 * idet, Si11 = S00 * idet;
  const double r0 = m0 - p[0], r1 = m1 - p[1];
  chi2 = r0 * (Si00 * r0 + Si01 * r1) + r1 * (Si01 * r0 + Si11 * r1);
  double K[5][2];
  for (int j = 0; j < 5; ++j) {
    const double U0 = C[S(j, 0)], U1 = C[S(j, 1)];
    K[j][0] = U0 * Si00 + U1 * Si01;
    K[j][1] = U0 * Si01 + U1 * Si11;
  }
  for (int j = 0; j < 5; ++j) p[j] += K[j][0] * r0 + K[j][1] * r1;
  double X[5][5];
  for (int r_ = 0; r_ < 5; ++r_)
    for (int c_ = 0; c_ < 5; ++c_) X[r_][c_] = C[S(r_, c_)] - K[r_][0] * C[S(0, c_)] - K[r_][1] * C[S(1, c_)];
  double Y[5][2];
  for (int r_ = 0; r_ < 5; ++r_) {
    Y[r_][0] = X[r_][0] - (K[r_][0] * V00 + K[r_][1] * V01);
    Y[r_][1] = X[r_][1] - (K[r_][0] * V01 + K[r_][1] * V11);
  }
  for (int r_ = 0; r_ < 5; ++r_)
    for (int c_ = r_; c_ < 5; ++c_) C[S(r_, c_)] = X[r_][c_] - Y[r_][0] * K[c_][0] - Y[r_][1] * K[c_][1];
  if (p[2] > kPi) p[2] -= 2.0 * kPi;
  if (p[2] <= -kPi) p[2] += 2.0 * kPi;
}

// Seeds in the order of their direction, so that the lanes of a warp cross the same modules and
// diverge less: a counting sort over 32 x 32 bins of (theta, phi). The order within a bin is the
// atomics' and affects no result: every seed is found on its own and written at its own index.
constexpr int kCkfOrderBins = 1024;

__device__ __forceinline__ uint32_t direction_bin(const double* __restrict__ seed_par, uint32_t n, uint32_t i) {
  const double ph = (seed_par[2 * size_t(n) + i] + kPi) * (16.0 / kPi), th = seed_par[3 * size_t(n) + i] * (32.0 / kPi);
  const uint32_t bp = ph >= 0.0 && ph < 32.0 ? uint32_t(ph) : (ph >= 32.0 ? 31u : 0u);  // NaN: bin 0
  const uint32_t bt = th >= 0.0 && th < 32.0 ? uint32_t(th) : (th >= 32.0 ? 31u : 0u);
  return bt * 32u + bp;
}

__global__ void ckf_order_hist_kernel(const double* __restrict__ seed_par, uint32_t n, uint32_t* __restrict__ hist) {
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    atomicAdd(&hist[direction_bin(seed_par, n, i)], 1u);
}

// exclusive prefix sum of the bins, one block of kCkfOrderBins threads
__global__ void __launch_bounds__(kCkfOrderBins) ckf_order_scan_kernel(uint32_t* __restrict__ hist) {
  __shared__ uint32_t v[kCkfOrderBins];
  const uint32_t t = threadIdx.x;
  const uint32_t own = hist[t];
  v[t] = own;
  __syncthreads();
  for (uint32_t d = 1; d < uint32_t(kCkfOrderBins); d <<= 1) {
    const uint32_t add = t >= d ? v[t - d] : 0u;
    __syncthreads();
    v[t] += add;
    __syncthreads();
  }
  hist[t] = v[t] - own;
}

__global__ void ckf_order_scatter_kernel(const double* __restrict__ seed_par, uint32_t n, uint32_t* __restrict__ hist,
                                         uint32_t* __restrict__ perm) {
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    perm[atomicAdd(&hist[direction_bin(seed_par, n, i)], 1u)] = i;
}

__global__ void ckf_meas_f32_kernel(const double* __restrict__ loc0, const double* __restrict__ loc1,
                                    const double* __restrict__ v00, const double* __restrict__ v11, uint32_t n,
                                    float4* __restrict__ out) {
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    out[i] = make_float4(float(loc0[i]), float(loc1[i]), float(v00[i]), float(v11[i]));
}

// ---- the search as phases: every step of every seed is three launches over all seeds,
// (1) one thread per branch slot predicts its branch to the next module, (2) one thread per slot
// gates that module's measurements and makes the branch's children, (3) one thread per seed
// numbers the children in creation order, keeps the best ended branch and the beam. Every
// thread of a launch runs the same phase, so the lanes of a warp stay in step (one thread per
// seed running all phases of its branches in turn left two thirds of the lanes idle), and the
// branches of a seed are predicted in parallel. The arithmetic of every branch, the order in
// which children are made and the ranking are those of the sequential search, so the candidates
// are the same.

// One branch's prediction for the current step, and the children it made.
struct alignas(16) CkfPred {
  double pp[5], pdir[4], Cp[15], h;
  int32_t target;  // next module; -1: the branch ends (nothing ahead, or the entries are full); -2: no branch
  uint32_t nk;     // children with a measurement
  uint32_t hole;   // 1: a child with a hole
  uint32_t pad;
};

// The doubles of a prediction (pp, pdir, Cp, h) and of a branch (p, dir, C, h_ctrl, chi2) are
// contiguous from the start of their 16-byte aligned records: a thread moves them with 16-byte
// accesses, which a warp of scattered records issues in half the memory transactions.
static_assert(offsetof(CkfPred, h) == 24 * sizeof(double), "prediction doubles contiguous");
static_assert(offsetof(CkfBranch, chi2) == 25 * sizeof(double) && sizeof(CkfBranch) % 16 == 0,
              "branch doubles contiguous, records 16-byte aligned");

__device__ __forceinline__ void load_pred(const CkfPred& pr, double pp[5], double pdir[4], double Cp[15], double& h) {
  const double2* q = reinterpret_cast<const double2*>(&pr);
  double v[26];
#pragma unroll
  for (int j = 0; j < 12; ++j) {
    const double2 w = q[j];
    v[2 * j] = w.x;
    v[2 * j + 1] = w.y;
  }
  v[24] = pr.h;
#pragma unroll
  for (int j = 0; j < 5; ++j) pp[j] = v[j];
#pragma unroll
  for (int j = 0; j < 4; ++j) pdir[j] = v[5 + j];
#pragma unroll
  for (int j = 0; j < 15; ++j) Cp[j] = v[9 + j];
  h = v[24];
}

__device__ __forceinline__ void store_pred(CkfPred& pr, const double pp[5], const double pdir[4], const double Cp[15],
                                           double h) {
  double v[24];
#pragma unroll
  for (int j = 0; j < 5; ++j) v[j] = pp[j];
#pragma unroll
  for (int j = 0; j < 4; ++j) v[5 + j] = pdir[j];
#pragma unroll
  for (int j = 0; j < 15; ++j) v[9 + j] = Cp[j];
  double2* q = reinterpret_cast<double2*>(&pr);
#pragma unroll
  for (int j = 0; j < 12; ++j) q[j] = make_double2(v[2 * j], v[2 * j + 1]);
  pr.h = h;
}

// a child's doubles: parameters, direction, covariance, step control and chi2
__device__ __forceinline__ void store_child(CkfBranch& ch, const double p[5], const double dir[4], const double C[15],
                                            double h, double chi2) {
  double v[26];
#pragma unroll
  for (int j = 0; j < 5; ++j) v[j] = p[j];
#pragma unroll
  for (int j = 0; j < 4; ++j) v[5 + j] = dir[j];
#pragma unroll
  for (int j = 0; j < 15; ++j) v[9 + j] = C[j];
  v[24] = h;
  v[25] = chi2;
  double2* q = reinterpret_cast<double2*>(&ch);
#pragma unroll
  for (int j = 0; j < 13; ++j) q[j] = make_double2(v[2 * j], v[2 * j + 1]);
}

// Per-seed search state.
struct CkfSeed {
  uint32_t n_act;   // branches in the beam (0: the search is over)
  uint32_t order;   // creation counter of the children
  uint32_t have_best;
  uint32_t first;   // 1 before the first step (the seed's own surface)
  uint32_t area;    // the children area that holds the beam (0 or 1)
  uint8_t act[8];   // the beam's slots, in rank order
};

struct CkfWork {
  CkfBranch* slots;  // per seed: two areas of B (C + 1) children, then the best ended branch
  CkfPred* pred;     // per seed: B
  CkfSeed* seeds;    // per seed
  uint32_t* list;    // the branch slots (t B + bi) in the beam, for the next step's phases 1 and 2
  uint32_t* count;   // their number
  uint32_t* next;    // the prediction's next chunk of the list (reset with count)
  CkfNode* nodes;    // per seed: ckf_steps(max_entries) x B history nodes
  const NavTables* nav;  // the navigation tables, built once a call (pointers fixed up per block)
};

// Appends each seed's beam slots to the list for the next step: in seed order within a block
// (an exclusive scan of the beam sizes), blocks in any order. Every thread of the block calls it.
__device__ void append_beam(const CkfWork& w, uint32_t t, uint32_t n_act, uint32_t B) {
  __shared__ uint32_t part[kCkfBlock];
  __shared__ uint32_t base;
  const uint32_t tid = threadIdx.x;
  part[tid] = n_act;
  __syncthreads();
  for (uint32_t d = 1; d < kCkfBlock; d <<= 1) {
    const uint32_t add = tid >= d ? part[tid - d] : 0u;
    __syncthreads();
    part[tid] += add;
    __syncthreads();
  }
  if (tid == kCkfBlock - 1) base = part[tid] ? atomicAdd(w.count, part[tid]) : 0u;
  __syncthreads();
  const uint32_t at = base + part[tid] - n_act;
  for (uint32_t q = 0; q < n_act; ++q) w.list[at + q] = t * B + q;
}

__device__ __forceinline__ CkfBranch* seed_slots(const CkfWork& w, uint32_t t, uint32_t B) {
  return w.slots + size_t(t) * slots_per_seed(B);
}

__device__ __forceinline__ CkfNode* seed_nodes(const CkfArgs& a, const CkfWork& w, uint32_t t) {
  return w.nodes + size_t(t) * ckf_steps(a.max_entries) * a.beam;
}

// Outputs of seed i from its best ended branch: its entries read back along the history tree
// from its last node (slot t's nodes).
__device__ void write_candidate(const CkfArgs& a, const CkfWork& w, uint32_t t, uint32_t i, const CkfBranch* best,
                                bool have_best) {
  const uint32_t n = a.n_seeds;
  const uint32_t ne = have_best ? best->n_entries : 0;
  a.n_entries[i] = ne;
  a.n_meas_out[i] = have_best ? best->n_meas : 0;
  a.chi2[i] = have_best ? best->chi2 : 0.0;
  for (uint32_t j = ne; j < a.max_entries; ++j) {
    a.entry_sid[size_t(j) * n + i] = 0u;
    a.entry_meas[size_t(j) * n + i] = -1;
  }
  const CkfNode* nodes = seed_nodes(a, w, t);
  const uint32_t n_nodes = ckf_steps(a.max_entries) * a.beam;
  int32_t at = have_best ? best->node : -1;
  for (uint32_t j = ne; j-- > 0;) {
    const bool ok = at >= 0 && uint32_t(at) < n_nodes;
    const CkfNode nd = ok ? nodes[at] : CkfNode{0u, -1, -1};
    a.entry_sid[size_t(j) * n + i] = nd.sid;
    a.entry_meas[size_t(j) * n + i] = nd.meas;
    at = nd.parent;
  }
}

__device__ void init_seed(const CkfArgs& a, const CkfWork& w, uint32_t t, CkfSeed& st);
__device__ uint32_t beam_seed(const CkfArgs& a, const CkfWork& w, uint32_t t, uint32_t step, uint32_t last);

// The seed's starting branch (thread t finds seed perm[t]); a seed on a missing surface or event
// gets no candidate at once.
__global__ void __launch_bounds__(kCkfBlock) ckf_init_kernel(const CkfArgs a, CkfWork w) {
  const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
  const bool live = t < a.n_seeds;
  CkfSeed st{0u, 1u, 0u, 1u, 0u, {0, 0, 0, 0, 0, 0, 0, 0}};
  if (live) init_seed(a, w, t, st);
  append_beam(w, t, st.n_act, a.beam);
}

__device__ void init_seed(const CkfArgs& a, const CkfWork& w, uint32_t t, CkfSeed& st) {
  const uint32_t i = a.perm[t], n = a.n_seeds;
  const uint32_t seed_sid = a.seed_sid[i];
  const uint32_t ev = a.seed_event ? a.seed_event[i] : 0u;
  if (seed_sid < a.n_surf && ev < a.n_events) {
    CkfBranch& b0 = seed_slots(w, t, a.beam)[0];
    for (int j = 0; j < 5; ++j) b0.p[j] = a.seed_par[size_t(j) * n + i];
    sincos(b0.p[2], &b0.dir[0], &b0.dir[1]);
    sincos(b0.p[3], &b0.dir[2], &b0.dir[3]);
    b0.p[2] = 0.0;
    b0.p[3] = 0.0;
    for (int j = 0; j < 15; ++j) b0.C[j] = a.seed_cov[size_t(j) * n + i];
    b0.h_ctrl = a.opt.h_max;
    b0.chi2 = 0.0;
    b0.n_meas = b0.holes = b0.n_entries = 0;
    b0.order = 0;
    b0.sid = -1;
    b0.node = -1;
    st.n_act = 1;
    st.area = 0;
    st.act[0] = 0;
  } else {
    write_candidate(a, w, t, i, nullptr, false);
  }
  w.seeds[t] = st;
}

// The navigation tables, built by one block once a call; the prediction's blocks copy them.
__global__ void __launch_bounds__(kCkfBlock) ckf_nav_kernel(const CkfArgs a, NavTables* __restrict__ out) {
  __shared__ NavTables nt;
  build_nav_tables(a, nt);
  const uint4* src = reinterpret_cast<const uint4*>(&nt);
  uint4* dst = reinterpret_cast<uint4*>(out);
  for (uint32_t j = threadIdx.x; j < sizeof(NavTables) / 16; j += blockDim.x) dst[j] = src[j];
}

// Phase 1: the prediction of the branch at list entry k (beam slot g = t B + bi).
template <bool kMixed, class F>
__device__ __forceinline__ void predict_branch(const CkfArgs& a, const F& fld, const NavTables& nt, const CkfWork& w,
                                               uint32_t k) {
  const uint32_t B = a.beam;
  const uint32_t g = w.list[k];  // a branch slot in the beam
  const uint32_t t = g / B, bi = g % B;
  const CkfSeed st = w.seeds[t];
  CkfPred& pr = w.pred[g];
  const CkfBranch& br = seed_slots(w, t, B)[st.act[bi]];
  int target;
  if (st.first) {
    target = int(a.seed_sid[a.perm[t]]);
    store_pred(pr, br.p, br.dir, br.C, br.h_ctrl);
  } else {
    double pp[5], pdir[4], Cp[15], h = br.h_ctrl;
    target = br.n_entries >= a.max_entries ? -1 : predict<kMixed>(a, fld, nt, br, pp, pdir, Cp, h);
    if (target >= 0) store_pred(pr, pp, pdir, Cp, h);
  }
  pr.target = target;
}

// One wave of resident blocks: each copies the navigation tables once, then takes chunks of
// blockDim.x list entries from a counter until the list is done (branches differ in their work,
// so the chunks balance the blocks). No block waits on another.
template <bool kMixed, class F>
__global__ void __launch_bounds__(kCkfBlock) ckf_predict_kernel(const CkfArgs a, const F fld, CkfWork w) {
  __shared__ NavTables nt;
  __shared__ uint32_t chunk;
  const uint32_t count = *w.count;
  if (blockIdx.x * blockDim.x >= count) return;  // more blocks than chunks: none for this one
  const uint4* src = reinterpret_cast<const uint4*>(w.nav);
  uint4* dst = reinterpret_cast<uint4*>(&nt);
  for (uint32_t j = threadIdx.x; j < sizeof(NavTables) / 16; j += blockDim.x) dst[j] = src[j];
  __syncthreads();
  if (threadIdx.x == 0) {
    const bool ring_fit = a.n_rings <= uint32_t(kCkfMaxRings);
    nt.rings = ring_fit ? nt.ring : a.rings;
    nt.rings_f = ring_fit ? nt.ring_f : nullptr;
  }
  for (;;) {
    if (threadIdx.x == 0) chunk = atomicAdd(w.next, blockDim.x);
    __syncthreads();  // (the first one also publishes the ring pointers)
    const uint32_t b0 = chunk;
    __syncthreads();
    if (b0 >= count) break;
    if (b0 + threadIdx.x < count) predict_branch<kMixed>(a, fld, nt, w, b0 + threadIdx.x);
  }
}

// Phase 2: the gate over the predicted module's measurements and the children of branch bi.
__global__ void __launch_bounds__(kCkfBlock, 4) ckf_gate_kernel(const CkfArgs a, CkfWork w) {
  const uint32_t B = a.beam;
  const uint32_t k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= *w.count) return;
  const uint32_t g = w.list[k];
  const uint32_t t = g / B, bi = g % B;
  CkfPred& pr = w.pred[g];
  const int target = pr.target;
  if (target < 0) {
    pr.nk = 0;
    pr.hole = 0;
    return;
  }
  const uint32_t i = a.perm[t];
  const uint32_t ev = a.seed_event ? a.seed_event[i] : 0u;
  const uint32_t* __restrict__ moff = a.meas_off + size_t(ev) * (a.n_surf + 1);  // this event's offsets
  const CkfSeed st = w.seeds[t];
  CkfBranch* slots = seed_slots(w, t, B);
  const CkfBranch& br = slots[st.act[bi]];
  // the children go to the other area: the beam kernel keeps its choice there
  CkfBranch* kids = slots + (st.area ^ 1u) * area_slots(B) + bi * (kCkfChildren + 1);
  const double br_chi2 = br.chi2;
  const uint32_t br_meas = br.n_meas, br_holes = br.holes, br_entries = br.n_entries;
  const int32_t br_node = br.node;
  double pp[5], pdir[4], Cp[15], h;
  load_pred(pr, pp, pdir, Cp, h);
  // the (at most 3) compatible measurements with the lowest chi2 (ties: lower index)
  double kc2[kCkfChildren];
  uint32_t km[kCkfChildren];
  int nk = 0;
  const uint32_t m_end = moff[target + 1] < a.n_meas ? moff[target + 1] : a.n_meas;
  // chi2 = r^T S^-1 r >= r0^2 / S00 and >= r1^2 / S11 (S positive definite): a measurement
  // whose residual fails the gate in one coordinate alone is skipped before the full chi2.
  // The margin keeps the skip exact under rounding (the full test would reject it too).
  const double gate = a.chi2_max * (1.0 + 1e-6);
  // the same bound first in FP32, on FP32 copies of the measurements: it skips only where
  // the rounding of every FP32 operand (at most 1e-6 of |loc| + |p| + |r| in the residual,
  // 1e-4 of S) cannot bring the residual back inside the gate
  const float p0f = d2f(pp[0]), p1f = d2f(pp[1]), c00f = d2f(Cp[S(0, 0)]), c11f = d2f(Cp[S(1, 1)]);
  const float gatef = float(a.chi2_max) * 1.0001f;
  // eight measurements at a time: their FP32 copies loaded together (the loop waits on the
  // loads, not the arithmetic), screened into a mask, the survivors taken in index order
  for (uint32_t base = moff[target]; base < m_end; base += 8) {
    float4 mf[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) mf[u] = base + u < m_end ? a.meas_f[base + u] : make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    uint32_t pass = 0;
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const float r0f = mf[u].x - p0f, r1f = mf[u].y - p1f;
      const float e0 = fabsf(r0f) - 1e-6f * (fabsf(mf[u].x) + fabsf(p0f) + fabsf(r0f));
      const float e1 = fabsf(r1f) - 1e-6f * (fabsf(mf[u].y) + fabsf(p1f) + fabsf(r1f));
      const bool out = (e0 > 0.0f && e0 * e0 > gatef * (c00f + mf[u].z)) || (e1 > 0.0f && e1 * e1 > gatef * (c11f + mf[u].w));
      if (base + u < m_end && !out) pass |= 1u << u;
    }
    while (pass) {
      const uint32_t mi = base + uint32_t(__ffs(pass) - 1);
      pass &= pass - 1u;
      const double q0 = a.loc0[mi] - pp[0], q1 = a.loc1[mi] - pp[1];
      if (q0 * q0 > gate * (Cp[S(0, 0)] + a.v00[mi]) || q1 * q1 > gate * (Cp[S(1, 1)] + a.v11[mi])) continue;
      double c2;
      if (!meas_chi2(pp, Cp, a.loc0[mi], a.loc1[mi], a.v00[mi], a.v01[mi], a.v11[mi], c2)) continue;
      if (!(c2 < a.chi2_max)) continue;
      int pos = nk;
      while (pos > 0 && (c2 < kc2[pos - 1] || (c2 == kc2[pos - 1] && mi < km[pos - 1]))) --pos;
      if (pos >= kCkfChildren) continue;
      for (int q = (nk < kCkfChildren ? nk : kCkfChildren - 1); q > pos; --q) {
        kc2[q] = kc2[q - 1];
        km[q] = km[q - 1];
      }
      kc2[pos] = c2;
      km[pos] = mi;
      if (nk < kCkfChildren) ++nk;
    }
  }
  for (int q = 0; q < nk; ++q) {
    double p[5], C[15];
    for (int j = 0; j < 5; ++j) p[j] = pp[j];
    for (int j = 0; j < 15; ++j) C[j] = Cp[j];
    const uint32_t mi = km[q];
    double c2;
    update(p, C, a.loc0[mi], a.loc1[mi], a.v00[mi], a.v01[mi], a.v11[mi], c2);
    // filtered direction: the predicted one turned by the update's angle increments
    double sd, cd, se, ce;
    small_sincos(p[2], sd, cd);
    small_sincos(p[3], se, ce);
    CkfBranch& ch = kids[q];
    const double dir[4] = {pdir[0] * cd + pdir[1] * sd, pdir[1] * cd - pdir[0] * sd, pdir[2] * ce + pdir[3] * se,
                           pdir[3] * ce - pdir[2] * se};
    p[2] = 0.0;
    p[3] = 0.0;
    store_child(ch, p, dir, C, h, br_chi2 + c2);
    ch.n_meas = br_meas + 1;
    ch.holes = 0;
    ch.n_entries = br_entries + 1;
    ch.sid = target;
    ch.node = br_node;
    ch.e_sid = uint32_t(target);
    ch.e_meas = int32_t(mi);
  }
  uint32_t hole = 0;
  if (br_holes < a.max_holes) {
    CkfBranch& ch = kids[nk];
    store_child(ch, pp, pdir, Cp, h, br_chi2);
    ch.n_meas = br_meas;
    ch.holes = br_holes + 1;
    ch.n_entries = br_entries + 1;
    ch.sid = target;
    ch.node = br_node;
    ch.e_sid = uint32_t(target) | TKF_SID_NO_MEASUREMENT;
    ch.e_meas = -1;
    hole = 1;
  }
  pr.nk = uint32_t(nk);
  pr.hole = hole;
}

// Phase 3, one thread per seed: the children numbered in creation order (branch by branch,
// measurements by chi2, then the hole), the best ended branch, the beam of the best B children.
// `step`: the step's index (the row of history nodes it writes); `last`: the final step; the
// candidate is written when the search is over.
__global__ void __launch_bounds__(kCkfBlock) ckf_beam_kernel(const CkfArgs a, CkfWork w, uint32_t step,
                                                             uint32_t last) {
  const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
  uint32_t n_next = 0;
  if (t < a.n_seeds) n_next = beam_seed(a, w, t, step, last);
  append_beam(w, t, n_next, a.beam);
}

// The beam of seed slot t after a step; returns its size (0: the search is over). The kept
// children stay where the gate wrote them (the other area becomes the beam's); each gets its
// entry as history node (step, rank).
__device__ uint32_t beam_seed(const CkfArgs& a, const CkfWork& w, uint32_t t, uint32_t step, uint32_t last) {
  CkfSeed st = w.seeds[t];
  if (st.n_act == 0) return 0;  // over (candidate written)
  const uint32_t B = a.beam;
  CkfBranch* slots = seed_slots(w, t, B);
  const uint32_t kid_area = (st.area ^ 1u) * area_slots(B);
  CkfBranch* kids = slots + kid_area;
  CkfBranch* best = slots + 2 * area_slots(B);
  const CkfPred* pr = w.pred + size_t(t) * B;
  uint32_t kid_at[8 * (kCkfChildren + 1)];
  uint32_t n_kids = 0;
  for (uint32_t bi = 0; bi < st.n_act; ++bi) {
    const CkfBranch& br = slots[st.act[bi]];
    const uint32_t nc = pr[bi].target < 0 ? 0u : pr[bi].nk + pr[bi].hole;
    for (uint32_t q = 0; q < nc; ++q) {
      const uint32_t k = bi * (kCkfChildren + 1) + q;
      kids[k].order = st.order++;
      kid_at[n_kids++] = k;
    }
    // a branch ends when nothing lies ahead, or when one hole too many would follow with no
    // compatible measurement
    const bool ends = pr[bi].target < 0 || (pr[bi].nk == 0 && pr[bi].hole == 0);
    if (ends && (!st.have_best || better(br, *best))) {
      copy_branch(*best, br);
      st.have_best = 1;
    }
  }
  st.first = 0;
  // the beam: the best B children, in rank order
  const uint32_t n_act = n_kids < B ? n_kids : B;
  CkfNode* nodes = seed_nodes(a, w, t) + size_t(step) * B;
  uint32_t taken = 0;
  for (uint32_t q = 0; q < n_act; ++q) {
    int pick = -1;
    for (uint32_t j = 0; j < n_kids; ++j)
      if (!((taken >> j) & 1u) && (pick < 0 || better(kids[kid_at[j]], kids[kid_at[pick]]))) pick = int(j);
    taken |= 1u << pick;
    CkfBranch& k = kids[kid_at[pick]];
    nodes[q] = CkfNode{k.e_sid, k.e_meas, k.node};
    k.node = int32_t(step * B + q);
    st.act[q] = uint8_t(kid_area + kid_at[pick]);
  }
  st.area ^= 1u;
  st.n_act = last ? 0u : n_act;
  if (st.n_act == 0) write_candidate(a, w, t, a.perm[t], best, st.have_best != 0);
  w.seeds[t] = st;
  return st.n_act;
}

// Workspace layout (byte offsets): branch slots, the seed-order histogram and permutation, FP32
// copies of the measurements (16-byte aligned), the predictions of every beam slot, the per-seed
// states, the list of beam slots, its count and the prediction's chunk counter, the history nodes,
// the navigation tables (16-byte aligned).
struct CkfLayout {
  size_t hist, meas_f, pred, seeds, list, count, nodes, nav, total;
  CkfLayout(uint32_t n_seeds, uint32_t beam, uint32_t n_meas, uint32_t max_entries) {
    hist = size_t(n_seeds) * slots_per_seed(beam) * sizeof(CkfBranch);
    meas_f = hist + ((sizeof(uint32_t) * (kCkfOrderBins + size_t(n_seeds)) + 15) & ~size_t(15));
    pred = meas_f + sizeof(float4) * size_t(n_meas);
    seeds = pred + sizeof(CkfPred) * size_t(n_seeds) * beam;
    list = (seeds + sizeof(CkfSeed) * size_t(n_seeds) + 7) & ~size_t(7);
    count = list + sizeof(uint32_t) * size_t(n_seeds) * beam;
    nodes = count + 2 * sizeof(uint32_t);
    nav = (nodes + sizeof(CkfNode) * size_t(n_seeds) * ckf_steps(max_entries) * beam + 15) & ~size_t(15);
    total = nav + sizeof(NavTables);
  }
};

template <class F>
cudaError_t launch_ckf(const CkfArgs& a_in, const F& fld, cudaStream_t stream) {
  CkfArgs a = a_in;
  if (a.opt.max_steps > kCkfMaxSteps) a.opt.max_steps = kCkfMaxSteps;
  const CkfLayout L(a.n_seeds, a.beam, a.n_meas, a.max_entries);
  char* base = static_cast<char*>(a.ws);
  // the seed order: histogram, scan and scatter
  uint32_t* hist = reinterpret_cast<uint32_t*>(base + L.hist);
  uint32_t* perm = hist + kCkfOrderBins;
  cudaError_t e = cudaMemsetAsync(hist, 0, sizeof(uint32_t) * kCkfOrderBins, stream);
  if (e != cudaSuccess) return e;
  const unsigned og = (a.n_seeds + 255) / 256 < 1024 ? (a.n_seeds + 255) / 256 : 1024;
  ckf_order_hist_kernel<<<og, 256, 0, stream>>>(a.seed_par, a.n_seeds, hist);
  ckf_order_scan_kernel<<<1, kCkfOrderBins, 0, stream>>>(hist);
  ckf_order_scatter_kernel<<<og, 256, 0, stream>>>(a.seed_par, a.n_seeds, hist, perm);
  a.perm = perm;
  // FP32 copies of the measurements for the gate's first bound
  float4* mf = reinterpret_cast<float4*>(base + L.meas_f);
  if (a.n_meas > 0) {
    const unsigned mg = (a.n_meas + 255) / 256 < 4096 ? (a.n_meas + 255) / 256 : 4096;
    ckf_meas_f32_kernel<<<mg, 256, 0, stream>>>(a.loc0, a.loc1, a.v00, a.v11, a.n_meas, mf);
  }
  a.meas_f = mf;
  CkfWork w;
  w.slots = reinterpret_cast<CkfBranch*>(base);
  w.pred = reinterpret_cast<CkfPred*>(base + L.pred);
  w.seeds = reinterpret_cast<CkfSeed*>(base + L.seeds);
  w.list = reinterpret_cast<uint32_t*>(base + L.list);
  w.count = reinterpret_cast<uint32_t*>(base + L.count);
  w.next = w.count + 1;
  w.nodes = reinterpret_cast<CkfNode*>(base + L.nodes);
  NavTables* nav = reinterpret_cast<NavTables*>(base + L.nav);
  w.nav = nav;
  const unsigned gs = (a.n_seeds + kCkfBlock - 1) / kCkfBlock;
  const unsigned gb = unsigned((size_t(a.n_seeds) * a.beam + kCkfBlock - 1) / kCkfBlock);
  // the prediction: one wave of resident blocks at most
  int dev = 0, sms = 0, per_sm = 0;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
  if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
  e = a.mixed ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, ckf_predict_kernel<true, F>, kCkfBlock, 0)
              : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, ckf_predict_kernel<false, F>, kCkfBlock, 0);
  if (e != cudaSuccess) return e;
  const unsigned wave = unsigned(sms > 0 ? sms : 1) * unsigned(per_sm > 0 ? per_sm : 1);
  const unsigned gp = gb < wave ? gb : wave;
  if ((e = cudaMemsetAsync(w.count, 0, 2 * sizeof(uint32_t), stream)) != cudaSuccess) return e;
  ckf_nav_kernel<<<1, kCkfBlock, 0, stream>>>(a, nav);
  ckf_init_kernel<<<gs, kCkfBlock, 0, stream>>>(a, w);
  // every step adds an entry to each surviving branch: at most max_entries + 2 steps
  const uint32_t n_steps = ckf_steps(a.max_entries);
  for (uint32_t step = 0; step < n_steps; ++step) {
    if (a.mixed)
      ckf_predict_kernel<true><<<gp, kCkfBlock, 0, stream>>>(a, fld, w);
    else
      ckf_predict_kernel<false><<<gp, kCkfBlock, 0, stream>>>(a, fld, w);
    ckf_gate_kernel<<<gb, kCkfBlock, 0, stream>>>(a, w);
    if ((e = cudaMemsetAsync(w.count, 0, 2 * sizeof(uint32_t), stream)) != cudaSuccess) return e;
    ckf_beam_kernel<<<gs, kCkfBlock, 0, stream>>>(a, w, step, step + 1 == n_steps ? 1u : 0u);
  }
  return cudaGetLastError();
}

}  // namespace

size_t ckf_workspace_bytes(uint32_t n_seeds, uint32_t beam, uint32_t n_meas, uint32_t max_entries) {
  return CkfLayout(n_seeds, beam, n_meas, max_entries).total;
}

cudaError_t launch_find_tracks(const CkfArgs& a, const FieldDev& f, cudaStream_t stream) {
  if (a.n_layers > uint32_t(kCkfMaxLayers)) return cudaErrorInvalidValue;
  if (f.kind == TKF_FIELD_UNIFORM) {
    if (f.b[0] == 0.0 && f.b[1] == 0.0) return launch_ckf(a, FieldUniformZ{f.b[2], float(f.b[2])}, stream);
    return launch_ckf(a, FieldUniform{{f.b[0], f.b[1], f.b[2]}, {float(f.b[0]), float(f.b[1]), float(f.b[2])}},
                      stream);
  }
  return launch_ckf(a, grid_policy(f), stream);
}

}  // namespace tkf
