// tkf_internal.cuh -- handle layouts and kernel arguments shared by the API and the kernels.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <array>
#include <map>
#include <string>
#include <utility>

#include "tkf.h"

namespace tkf {

// Device surface record: 24 doubles (192 B) per surface:
//   [0..2] u, [3..5] v, [6..8] n, [9..11] c, [12] thickness, [13] x0, [14] t / x0,
//   [15] sqrt(t / x0) (1 + 0.038 ln(t / x0)) (the Highland factor at normal incidence, beta = 1;
//   0 without material),
//   then 16 floats: u, v, n, thickness, t / x0 (FP32 copies for the mixed path), c (FP32 copy for
//   the navigation's screens), 2 x 0.
constexpr int kSurfStride = 24;

// Material constants folded for the kernels.
struct MaterialDev {
  double z_over_a, i_ev, rho, hwp_ev;
  double log_hwp_over_i;  // ln(hbar omega_p / I)
  double bg2_density;     // (beta gamma)^2 above which the density-effect term is positive
  // FP32 copies for the mixed path
  float log_hwp_over_i_f, bg2_density_f;
  float two_me_over_i2_f;  // 2 m_e / I^2, 1/GeV
  float dedx_scale_f;      // K Z/A rho 1e-4: MeV cm^2/g -> GeV per mm of path
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
  // FP32 copies for the mixed path
  float tol_f, h_max_f, h_min_f, mass_f, me_over_mass_f, surf_tol_f;
};

struct FitArgs {
  uint32_t n_tracks;
  uint32_t stride;  // row stride of the SoA seed and output arrays: n_tracks, or a whole batch's for a chunk of it
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
  double seed_cov_scale;  // factor on every seed covariance element (1: as given)
  int smoother;               // TKF_SMOOTHER_RTS or TKF_SMOOTHER_TWO_FILTER
  double backward_inflation;  // two-filter: factor on the backward filter's starting covariance
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
  const float* __restrict__ mlp;     // FP32 (BF16-rounded) step-proposer weights, or null
  const float* __restrict__ h0;      // learned mode: per-track starting step-size control
  float* __restrict__ records;       // training-record capture, or null
  uint32_t record_capacity;
  uint32_t* __restrict__ record_count;
  bool test_stall_proposals;  // test of the timeout path: the pre-pass issues no tensor-core work
  // all-states output (or null): every entry's smoothed state, SoA [5][n_meas] and [15][n_meas];
  // the forward pass writes the filtered states there first
  double* __restrict__ states_par;
  double* __restrict__ states_cov;
  double* __restrict__ states_scratch;  // workspace: kStatesScratch doubles per entry
};

// Per entry for the backward RTS pass: predicted parameters (5), packed covariance (15) and the
// transport Jacobian from the previous entry (25, row-major).
constexpr int kStatesScratch = 45;

constexpr int kMlpParams = TKF_MLP_PARAMS;
constexpr int kMlpRecord = TKF_MLP_RECORD;

// Scratch of one fit launch: work counter, key histogram, sort keys, track permutation.
struct Workspace {
  uint32_t* counter = nullptr;
  uint32_t* hist = nullptr;
  uint32_t* keys = nullptr;
  uint32_t* perm = nullptr;
  float* h0 = nullptr;  // learned mode: per-track starting step size (only when space was reserved)
  double* states = nullptr;  // all-states output: kStatesScratch doubles per entry (when reserved)
};
size_t workspace_bytes(uint32_t n_tracks, bool learned, uint64_t states_entries = 0);
Workspace carve_workspace(void* base, uint32_t n_tracks, bool learned, uint64_t states_entries = 0);
// Backward RTS pass of the all-states output (tkf_states.cu), after the fit on the same stream;
// perm: the fit's track order.
cudaError_t launch_smooth_states(const FitArgs& a, const uint32_t* perm, cudaStream_t stream);
cudaError_t launch_propose_start(const FitArgs& a, const FieldDev& f, float* h0, cudaStream_t stream);

// Seed parameter estimation (tkf_seed.cu): one thread per track, outputs in the fit's seed layout.
struct SeedArgs {
  uint32_t n_tracks;
  uint64_t n_meas;
  const uint32_t* __restrict__ offsets;
  const double* __restrict__ loc0;
  const double* __restrict__ loc1;
  const double* __restrict__ v00;
  const double* __restrict__ v01;
  const double* __restrict__ v11;
  const uint32_t* __restrict__ sid;
  const double* __restrict__ surf;  // n_surf * kSurfStride
  uint32_t n_surf;
  uint32_t first_three;  // 0: first, middle, last measurement; 1: the first three
  double* __restrict__ par;  // [5][n_tracks]
  double* __restrict__ cov;  // [15][n_tracks]
  uint32_t* __restrict__ status;
};
cudaError_t launch_estimate_seeds(const SeedArgs& a, const FieldDev& f, int sm_count, cudaStream_t stream);

// Track finding (tkf_ckf.cu): one thread per seed, branch store in a workspace.
struct CkfArgs {
  uint32_t n_seeds;
  const uint32_t* __restrict__ seed_sid;
  const double* __restrict__ seed_par;  // [5][n_seeds]
  const double* __restrict__ seed_cov;  // [15][n_seeds]
  const uint32_t* __restrict__ meas_off;    // [n_events][n_surf + 1]
  uint32_t n_meas;  // measurement rows: offsets beyond are clamped (never read past the arrays)
  const uint32_t* __restrict__ seed_event;  // event of each seed, or null (one event)
  uint32_t n_events;
  const double* __restrict__ loc0;
  const double* __restrict__ loc1;
  const double* __restrict__ v00;
  const double* __restrict__ v01;
  const double* __restrict__ v11;
  const double* __restrict__ surf;
  uint32_t n_surf;
  const double* __restrict__ layers;
  uint32_t n_layers;
  const double* __restrict__ rings;
  uint32_t n_rings;
  const int32_t* __restrict__ layer_of;
  MaterialDev mat;
  OptionsDev opt;
  double chi2_max;
  uint32_t beam, max_holes, max_entries;
  bool mixed;  // TKF_MIXED: propagation, material and covariance transport in FP32
  uint32_t* __restrict__ n_entries;
  uint32_t* __restrict__ n_meas_out;
  double* __restrict__ chi2;
  uint32_t* __restrict__ entry_sid;   // [max_entries][n_seeds]
  int32_t* __restrict__ entry_meas;   // [max_entries][n_seeds]
  void* ws;                           // branch store, then the seed order
  const uint32_t* __restrict__ perm;  // seed found by each thread (set by the launch)
  const float4* __restrict__ meas_f;  // FP32 loc0, loc1, V00, V11 (set by the launch)
};
size_t ckf_workspace_bytes(uint32_t n_seeds, uint32_t beam, uint32_t n_meas, uint32_t max_entries);
cudaError_t launch_find_tracks(const CkfArgs& a, const FieldDev& f, cudaStream_t stream);

// Launch shape of the persistent fit: threads per block, blocks in the grid, tracks a warp
// takes at a time (1..32 / group), the register cap of the kernel variant (255, or 128 / 64
// for the mixed path, whose blocks then have at most 128 threads) and the lanes a track.
struct LaunchShape {
  int threads = 128;
  int blocks = 0;
  int tracks_per_warp = 32;
  int regs = 255;
  int group = 1;  // lanes a track: 1, or 4 (group-per-track: FP64 and mixed, 255 registers)
};

// Persistent fit launches per precision; mode 0 plain, 1 learned proposals, 2 record capture.
cudaError_t launch_fit_fp64(const FitArgs& a, const FieldDev& f, int mode, const uint32_t* perm, uint32_t* counter,
                            LaunchShape shape, cudaStream_t stream);
cudaError_t launch_fit_fp64_r128(const FitArgs& a, const FieldDev& f, int mode, const uint32_t* perm,
                                 uint32_t* counter, LaunchShape shape, cudaStream_t stream);
cudaError_t launch_fit_fp64_r64(const FitArgs& a, const FieldDev& f, int mode, const uint32_t* perm,
                                uint32_t* counter, LaunchShape shape, cudaStream_t stream);
cudaError_t launch_fit_mixed(const FitArgs& a, const FieldDev& f, int mode, const uint32_t* perm, uint32_t* counter,
                             LaunchShape shape, cudaStream_t stream);
cudaError_t launch_fit_mixed_r128(const FitArgs& a, const FieldDev& f, int mode, const uint32_t* perm,
                                  uint32_t* counter, LaunchShape shape, cudaStream_t stream);
cudaError_t launch_fit_mixed_r64(const FitArgs& a, const FieldDev& f, int mode, const uint32_t* perm,
                                 uint32_t* counter, LaunchShape shape, cudaStream_t stream);
cudaError_t launch_fit_mixed32(const FitArgs& a, const FieldDev& f, int mode, const uint32_t* perm, uint32_t* counter,
                               LaunchShape shape, cudaStream_t stream);
cudaError_t launch_fit_group(const FitArgs& a, const FieldDev& f, int precision, int mode, const uint32_t* perm,
                             uint32_t* counter, LaunchShape shape, cudaStream_t stream);
// Two-filter smoother (a.smoother == TKF_SMOOTHER_TWO_FILTER): one lane a track; 255 registers,
// or 128 / 64 (shape.regs) in FP64 and mixed precision.
cudaError_t launch_fit_two_filter(const FitArgs& a, const FieldDev& f, int precision, int mode, const uint32_t* perm,
                                  uint32_t* counter, LaunchShape shape, cudaStream_t stream);
cudaError_t launch_fit_two_filter_mixed_capped(const FitArgs& a, const FieldDev& f, int mode, const uint32_t* perm,
                                               uint32_t* counter, LaunchShape shape, cudaStream_t stream);
cudaError_t launch_fit_two_filter_fp64_capped(const FitArgs& a, const FieldDev& f, int mode, const uint32_t* perm,
                                              uint32_t* counter, LaunchShape shape, cudaStream_t stream);
cudaError_t launch_fit_two_filter_mixed(const FitArgs& a, const FieldDev& f, int mode, const uint32_t* perm,
                                        uint32_t* counter, LaunchShape shape, cudaStream_t stream);
cudaError_t launch_fit_two_filter_mixed32(const FitArgs& a, const FieldDev& f, int mode, const uint32_t* perm,
                                          uint32_t* counter, LaunchShape shape, cudaStream_t stream);

// Enqueues the fit of every track in `a` on `stream`: track ordering, then the persistent fit.
// With `timing`, events timing[0] and timing[1] are recorded right before and after the
// persistent fit kernel. Learned mode: the starting proposals come from the pre-pass, or, with
// `h0_given`, from that array (one per track of `a`, written by an earlier pre-pass on the device).
cudaError_t launch_fit(const FitArgs& a, const FieldDev& field, int precision, const Workspace& ws, LaunchShape shape,
                       cudaStream_t stream, const cudaEvent_t* timing = nullptr, const float* h0_given = nullptr);

}  // namespace tkf

// chunks of the host-buffer pipeline (tkf_fit_host) at most
constexpr int kHostChunksMax = 8;

struct tkf_context_s;

namespace tkf {

// Launch policy (tkf_policy.cu). The block shape of a call: the explicit one of the options,
// the context's tuned one for the launch class (timing the candidates on the first call when
// TKF_FIT_AUTOTUNE is set), else the default.
bool valid_block_shape(uint32_t threads, uint32_t blocks_per_sm, uint32_t tracks_per_warp, uint32_t max_registers,
                       uint32_t lanes_per_track, int precision, bool record);
cudaError_t resolve_shape(tkf_context_s* ctx, const FitArgs& a, const FieldDev& f, int precision, const Workspace& ws,
                          const tkf_fit_options* o, cudaStream_t stream, LaunchShape* out);
// Direct launch, or through the context's CUDA graph when `use_graph` (captured on the second
// consecutive call with identical arguments, replayed after that).
cudaError_t launch_with_policy(tkf_context_s* ctx, const FitArgs& a, const FieldDev& f, int precision,
                               const Workspace& ws, LaunchShape shape, bool use_graph, cudaStream_t stream,
                               const cudaEvent_t* timing);
void load_tune_cache(tkf_context_s* ctx);
// The launch shape used without tuning or explicit options.
LaunchShape default_launch_shape(int precision, bool record, int sm_count);
void release_graph(tkf_context_s* ctx);

}  // namespace tkf

struct tkf_context_s {
  int device = 0;
  int sm_count = 0;
  std::string last_error;
  // autotuner: best (threads, blocks per SM, tracks per warp, registers, lanes a track) per launch class;
  // optional cache file
  std::map<std::string, std::array<int, 5>> tuned;
  std::string tune_cache_path;
  // CUDA graph of the last repeated launch sequence
  cudaGraphExec_t graph_exec = nullptr;
  std::string graph_key, pending_key;
  // host-buffer entry point: copy streams and events of its chunk pipeline (created on first use)
  cudaStream_t h2d_stream = nullptr, d2h_stream = nullptr, fit2_stream = nullptr;
  cudaEvent_t chunk_in[kHostChunksMax] = {}, chunk_fit[kHostChunksMax] = {};
  cudaEvent_t props_in = nullptr, props_done = nullptr;  // learned mode: the batch's proposal pre-pass
  // fit workspace (ordering scratch), grown on demand and reused by later calls
  void* ws = nullptr;
  size_t ws_bytes = 0;
  // scratch of the network's training kernels
  void* train_ws = nullptr;
  size_t train_bytes = 0;
  // staging for tkf_fit_host
  void* stage = nullptr;
  size_t stage_bytes = 0;
  // branch store of track finding
  void* ckf_ws = nullptr;
  size_t ckf_ws_bytes = 0;
  // device address of tkf_fit_noalloc's static scratch on this context's device (NULL: not found)
  void* noalloc_scratch = nullptr;
};

struct tkf_geometry_s {
  tkf_context ctx = nullptr;
  int device = 0;
  double* d_surf = nullptr;
  uint32_t n = 0;
  tkf::MaterialDev mat{};
  // navigation (track finding): layer rows, ring rows, layer of every surface (-1: none)
  double* d_layers = nullptr;
  double* d_rings = nullptr;
  int32_t* d_layer_of = nullptr;
  uint32_t n_layers = 0, n_rings = 0;
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
  float* d_weights = nullptr;  // TKF_MLP_PARAMS FP32 values, each a BF16 value
};

namespace tkf {
// Training scratch size and launches (tkf_mlp.cu).
size_t mlp_train_scratch_bytes(uint32_t batch);
cudaError_t mlp_loss_grad(const float* params, const float* x, int x_stride, const float* y, int y_stride,
                          uint32_t n, float* grad, float* loss, void* scratch, cudaStream_t stream);
cudaError_t mlp_train(const float* records, uint32_t n, uint32_t batch, uint32_t epochs, float lr, float beta1,
                      float beta2, float eps, float* params, float* moments, uint32_t* adam_t, float* epoch_loss,
                      void* scratch, cudaStream_t stream);
cudaError_t mlp_forward(const float* params, const float* x, uint32_t n, float* out, cudaStream_t stream);
cudaError_t mlp_init(float* params, uint64_t seed, cudaStream_t stream);
size_t mlp_calibrate_scratch_bytes(uint32_t n);
// shift: DEVICE double receiving the bias shift
cudaError_t mlp_calibrate(float* params, const float* records, uint32_t n, double quantile, double* shift,
                          void* scratch, cudaStream_t stream);
cudaError_t mlp_round_bf16(const float* in, float* out, uint32_t* bad, cudaStream_t stream);
}  // namespace tkf
