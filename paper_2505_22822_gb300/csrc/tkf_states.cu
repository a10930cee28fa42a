// tkf_states.cu -- the all-states output: the Rauch-Tung-Striebel backward pass (paper Sec. 2:
// the smoother makes every state use every measurement) over the states the forward fit
// stored, so that every entry of every track gets its smoothed parameters and covariance.
//
// The first-surface result of tkf_fit needs no stored states (the smoother is evaluated
// forward there); this pass is what an all-states request adds. Per track, k = N-2 .. 0:
//   A_k    = Cf_k J_{k+1}^T Cp_{k+1}^-1                  (Cp_{k+1} by its Cholesky factor)
//   ps_k   = pf_k + A_k (ps_{k+1} - pp_{k+1})            (phi difference wrapped)
//   Cs_k   = Cf_k + A_k (Cs_{k+1} - Cp_{k+1}) A_k^T
// with the filtered state (pf, Cf) read from the all-states arrays, where the forward pass left
// it, and the predicted state (pp, Cp) and transport Jacobian J from the workspace. Each result
// overwrites the filtered state it came from; the last entry's smoothed state is its filtered
// one. FP64 throughout (the paper attributes its FP32 fit's mismatch to this smoother).

#include "tkf_internal.cuh"

namespace tkf {
namespace {

constexpr double kPi = 3.14159265358979323846;
constexpr uint32_t kFatal = ~(TKF_TRACK_TOO_FEW_HITS | TKF_TRACK_OUT_OF_FIELD | TKF_TRACK_PROPOSAL_FALLBACK);

__host__ __device__ constexpr int P(int i, int j) { return i <= j ? i * (9 - i) / 2 + j : j * (9 - j) / 2 + i; }

__device__ __forceinline__ double wrap_pi(double x) {
  if (x > kPi) x -= 2.0 * kPi;
  if (x <= -kPi) x += 2.0 * kPi;
  return x;
}

__device__ void nan_entries(const FitArgs& a, uint32_t b0, uint32_t b1) {
  const double nan = __longlong_as_double(0x7ff8000000000000LL);
  const size_t nm = size_t(a.n_meas);
  for (uint32_t e = b0; e < b1; ++e) {
    for (int j = 0; j < 5; ++j) a.states_par[size_t(j) * nm + e] = nan;
    for (int j = 0; j < 15; ++j) a.states_cov[size_t(j) * nm + e] = nan;
  }
}

// Thread k takes track perm[k]: the fit's order (most entries first), so that the lanes of a warp
// run backward passes of the same length.
__global__ void __launch_bounds__(128) smooth_states_kernel(FitArgs a, const uint32_t* __restrict__ perm) {
  const size_t nm = size_t(a.n_meas);
  for (uint32_t k = blockIdx.x * blockDim.x + threadIdx.x; k < a.n_tracks; k += gridDim.x * blockDim.x) {
    const uint32_t i = perm[k];
    const uint32_t b0 = a.offsets[i], b1 = a.offsets[i + 1];
    if (b1 < b0 || b1 > a.n_meas) continue;  // bad offsets: the track has no entries to write
    const uint32_t N = b1 - b0;
    if (N == 0) continue;
    uint32_t M = 0;
    for (uint32_t e = b0; e < b1; ++e) M += (a.sid[e] & TKF_SID_NO_MEASUREMENT) ? 0u : 1u;
    const uint32_t status = a.status[i];
    if (M == 0 || (status & kFatal)) {  // no fit (the seed was returned), or a failed one
      nan_entries(a, b0, b1);
      continue;
    }
    double ps[5], Cs[15];
    for (int j = 0; j < 5; ++j) ps[j] = a.states_par[size_t(j) * nm + b1 - 1];
    for (int j = 0; j < 15; ++j) Cs[j] = a.states_cov[size_t(j) * nm + b1 - 1];
    bool spd = true;
    for (int k = int(N) - 2; k >= 0 && spd; --k) {
      const uint32_t e = b0 + uint32_t(k);
      const double* w = a.states_scratch + size_t(e + 1) * kStatesScratch;
      double pf[5], Cf[15], pp[5], Cp[15], J[5][5];
      for (int j = 0; j < 5; ++j) pf[j] = a.states_par[size_t(j) * nm + e];
      for (int j = 0; j < 15; ++j) Cf[j] = a.states_cov[size_t(j) * nm + e];
      for (int j = 0; j < 5; ++j) pp[j] = w[j];
      for (int j = 0; j < 15; ++j) Cp[j] = w[5 + j];
      for (int r = 0; r < 5; ++r)
        for (int c = 0; c < 5; ++c) J[r][c] = w[20 + 5 * r + c];
      // B = J Cf, then X = Cp^-1 B = A^T (Cp, Cf symmetric); row 4 of J is e_4
      double X[5][5];
      for (int r = 0; r < 4; ++r)
        for (int c = 0; c < 5; ++c) {
          double acc = 0.0;
          for (int q = 0; q < 5; ++q) acc += J[r][q] * Cf[P(q, c)];
          X[r][c] = acc;
        }
      for (int c = 0; c < 5; ++c) X[4][c] = Cf[P(4, c)];
      // Cholesky Cp = L L^T, with the reciprocals of its diagonal (one division a row)
      double L[5][5], inv[5];
      for (int r = 0; r < 5; ++r)
        for (int c = 0; c <= r; ++c) {
          double acc = Cp[P(r, c)];
          for (int q = 0; q < c; ++q) acc -= L[r][q] * L[c][q];
          if (r == c) {
            spd = spd && acc > 0.0;
            L[r][r] = sqrt(acc);
            inv[r] = 1.0 / L[r][r];
          } else {
            L[r][c] = acc * inv[c];
          }
        }
      if (!spd) break;
      for (int c = 0; c < 5; ++c) {  // solve L L^T x = column c of B
        for (int r = 0; r < 5; ++r) {
          double acc = X[r][c];
          for (int q = 0; q < r; ++q) acc -= L[r][q] * X[q][c];
          X[r][c] = acc * inv[r];
        }
        for (int r = 4; r >= 0; --r) {
          double acc = X[r][c];
          for (int q = r + 1; q < 5; ++q) acc -= L[q][r] * X[q][c];
          X[r][c] = acc * inv[r];
        }
      }
      // A = X^T: A[r][c] = X[c][r]
      double dp[5];
      for (int j = 0; j < 5; ++j) dp[j] = ps[j] - pp[j];
      dp[2] = wrap_pi(dp[2]);
      for (int r = 0; r < 5; ++r) {
        double acc = pf[r];
        for (int c = 0; c < 5; ++c) acc += X[c][r] * dp[c];
        ps[r] = acc;
      }
      ps[2] = wrap_pi(ps[2]);
      // Cs = Cf + A (Cs - Cp) A^T: G = A D (5 x 5), then the upper triangle of G A^T
      double G[5][5];
      for (int r = 0; r < 5; ++r)
        for (int c = 0; c < 5; ++c) {
          double acc = 0.0;
          for (int q = 0; q < 5; ++q) acc += X[q][r] * (Cs[P(q, c)] - Cp[P(q, c)]);
          G[r][c] = acc;
        }
      for (int r = 0; r < 5; ++r)
        for (int c = r; c < 5; ++c) {
          double acc = 0.0;
          for (int q = 0; q < 5; ++q) acc += G[r][q] * X[q][c];
          Cs[P(r, c)] = Cf[P(r, c)] + acc;
        }
      for (int j = 0; j < 5; ++j) a.states_par[size_t(j) * nm + e] = ps[j];
      for (int j = 0; j < 15; ++j) a.states_cov[size_t(j) * nm + e] = Cs[j];
    }
    if (!spd) {  // a predicted covariance that is not positive definite: the track fails
      const double nan = __longlong_as_double(0x7ff8000000000000LL);
      a.status[i] = status | TKF_TRACK_SMOOTHER_NOT_SPD;
      for (int j = 0; j < 5; ++j) a.par[size_t(j) * a.stride + i] = nan;
      for (int j = 0; j < 15; ++j) a.cov[size_t(j) * a.stride + i] = nan;
      a.chi2[i] = nan;
      nan_entries(a, b0, b1);
    }
  }
}

}  // namespace

cudaError_t launch_smooth_states(const FitArgs& a, const uint32_t* perm, cudaStream_t stream) {
  if (a.n_tracks == 0) return cudaSuccess;
  const unsigned blocks = (a.n_tracks + 127) / 128;
  smooth_states_kernel<<<blocks, 128, 0, stream>>>(a, perm);
  return cudaGetLastError();
}

}  // namespace tkf
