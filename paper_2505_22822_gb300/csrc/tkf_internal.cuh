// tkf_internal.cuh -- handle layouts and kernel arguments shared by the API and the kernels.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "tkf.h"

namespace tkf {

// Device surface record: 16 doubles (128 B, one aligned L2 line pair) per surface:
//   [0..2] u, [3..5] v, [6..8] n, [9..11] c, [12] thickness, [13] x0, [14] t / x0, [15] 0.
constexpr int kSurfStride = 16;

// Material constants folded for the kernels.
struct MaterialDev {
  double z_over_a, i_ev, rho, hwp_ev;
  double log_hwp_over_i;  // ln(hbar omega_p / I)
  double bg2_density;     // (beta gamma)^2 above which the density-effect term is positive
};

struct FieldDev {
  int kind;          // tkf_field_kind
  double b[3];       // uniform field, T
  int nr, nz;        // grid
  double r0, dr, z0, dz;
  double inv_dr, inv_dz;
  const float2* grid;  // [nz][nr] (B_r, B_z)
};

struct OptionsDev {
  double tol, h_max, h_min, surf_tol, mass;
  uint32_t max_steps;
};

struct FitArgs {
  uint32_t n_tracks;
  uint64_t n_meas;
  const uint32_t* __restrict__ offsets;
  const double* __restrict__ loc0;
  const double* __restrict__ loc1;
  const double* __restrict__ v00;
  const double* __restrict__ v01;
  const double* __restrict__ v11;
  const uint32_t* __restrict__ sid;
  const double* __restrict__ seed_par;
  const double* __restrict__ seed_cov;
  double* __restrict__ par;
  double* __restrict__ cov;
  double* __restrict__ chi2;
  int32_t* __restrict__ ndf;
  uint32_t* __restrict__ status;
  uint32_t* __restrict__ steps;
  const double* __restrict__ surf;  // n_surf * kSurfStride
  uint32_t n_surf;
  MaterialDev mat;
  OptionsDev opt;
};

// Scratch of one fit launch: work counter, key histogram, sort keys, track permutation.
struct Workspace {
  uint32_t* counter = nullptr;
  uint32_t* hist = nullptr;
  uint32_t* keys = nullptr;
  uint32_t* perm = nullptr;
};
size_t workspace_bytes(uint32_t n_tracks);
Workspace carve_workspace(void* base, uint32_t n_tracks);

// Enqueues the fit of every track in `a` on `stream`: track ordering, then the persistent fit.
cudaError_t launch_fit(const FitArgs& a, const FieldDev& field, int precision, const Workspace& ws, int sm_count,
                       cudaStream_t stream);

}  // namespace tkf

struct tkf_context_s {
  int device = 0;
  int sm_count = 0;
  std::string last_error;
  // fit workspace (ordering scratch), grown on demand and reused by later calls
  void* ws = nullptr;
  size_t ws_bytes = 0;
  // staging for tkf_fit_host
  void* stage = nullptr;
  size_t stage_bytes = 0;
};

struct tkf_geometry_s {
  tkf_context ctx = nullptr;
  int device = 0;
  double* d_surf = nullptr;
  uint32_t n = 0;
  tkf::MaterialDev mat{};
};

struct tkf_field_s {
  tkf_context ctx = nullptr;
  int device = 0;
  tkf::FieldDev f{};
  float2* d_grid = nullptr;
};

struct tkf_mlp_s {
  tkf_context ctx = nullptr;
  int device = 0;
};
