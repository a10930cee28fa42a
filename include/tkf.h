/*
 * tkf.h -- C interface of the batched Kalman-filter track fitter for NVIDIA GB300 (sm_103a).
 *
 * The library fits track candidates as the paper describes its fitting stage (Sec. 2,
 * "Implementation", second paragraph): each track's parameters and covariance are
 * propagated between detector surfaces with the 4th-order Runge-Kutta-Nystrom method and
 * Jacobian transport, the Kalman filter adds each measurement with a chi2 from the
 * covariance-weighted spatial residual, and the Rauch-Tung-Striebel smoother makes the
 * parameters at the first measurement use every measurement. Material effects assume a
 * muon (Sec. 3, first paragraph). Geometry and field are uploaded once; per batch, only
 * measurements and seeds go in and fitted parameters come out (Sec. 2, third paragraph).
 *
 * Conventions
 *   Units: mm, GeV, tesla, radians; q/p in e/GeV.
 *   Bound parameters on a surface: (l0, l1, phi, theta, q/p), where (l0, l1) are the
 *   coordinates of the intersection along the surface's local axes u and v, and the unit
 *   direction is (sin(theta) cos(phi), sin(theta) sin(phi), cos(theta)); phi in (-pi, pi].
 *   Covariances are stored as the 15-element upper triangle in row-major order:
 *   (00, 01, 02, 03, 04, 11, 12, 13, 14, 22, 23, 24, 33, 34, 44).
 *   Device arrays are structure-of-arrays: component j of track i is at [j * n_tracks + i].
 *
 * Errors
 *   Every entry point returns a tkf_status. An argument error returns a nonzero code and
 *   enqueues nothing; tkf_last_error() then describes it. Numerical failures of single
 *   tracks never fail a call: they are reported in that track's status word.
 *
 * Threading
 *   A context is used by one host thread at a time, and its fits must not overlap on the
 *   device: they share the context's workspace, so give each concurrent stream its own
 *   context. Handles are freed by the matching *_destroy call, after all work that uses them
 *   has completed.
 */
#ifndef TKF_H_
#define TKF_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum tkf_status {
  TKF_OK = 0,
  TKF_ERR_INVALID_ARG = 1, /* null pointer, bad size, bad option, bad layout */
  TKF_ERR_BAD_HANDLE = 2,  /* handle null or from another context/device */
  TKF_ERR_DEVICE = 3,      /* no usable CUDA device, or a CUDA call failed */
  TKF_ERR_OOM = 4,         /* device or host allocation failed */
  TKF_ERR_UNSUPPORTED = 5  /* valid request this build cannot serve */
} tkf_status;

/* Per-track status bits written to tkf_fit_outputs.status. A track with any bit other than
 * TKF_TRACK_TOO_FEW_HITS, TKF_TRACK_OUT_OF_FIELD or TKF_TRACK_PROPOSAL_FALLBACK set has NaN
 * parameters, covariance and chi2. */
#define TKF_TRACK_MAX_STEPS (1u << 0)        /* more than max_steps step attempts to one surface */
#define TKF_TRACK_SURFACE_MISSED (1u << 1)   /* next surface more than 1 mm behind, or parallel */
#define TKF_TRACK_PARTICLE_STOPPED (1u << 2) /* mean energy loss left E <= mass */
#define TKF_TRACK_UPDATE_NOT_SPD (1u << 3)   /* residual covariance S not positive definite */
#define TKF_TRACK_SMOOTHER_NOT_SPD (1u << 4) /* smoothed covariance not positive definite */
#define TKF_TRACK_TOO_FEW_HITS (1u << 5)     /* fewer than 3 measurements (ndf < 6) */
#define TKF_TRACK_OUT_OF_FIELD (1u << 6)     /* a field sample fell outside the map (B = 0 used) */
#define TKF_TRACK_BAD_INPUT (1u << 7)        /* surface id out of range, or offsets decreasing */
#define TKF_TRACK_STEP_UNDERFLOW (1u << 8)   /* step size control fell below h_min */
#define TKF_TRACK_NON_FINITE (1u << 9)       /* NaN/Inf in the seed or the result, theta left (0, pi) */
#define TKF_TRACK_PROPOSAL_FALLBACK (1u << 10) /* learned mode: no proposal (the tensor-core pre-pass
                                                  timed out), the control started from h_max */

typedef struct tkf_context_s* tkf_context;
typedef struct tkf_geometry_s* tkf_geometry;
typedef struct tkf_field_s* tkf_field;
typedef struct tkf_mlp_s* tkf_mlp;

/* ---------------------------------------------------------------------------- context */

/* Creates a context on CUDA device `device` (the caller's current device if < 0). The
 * context owns a small device workspace (grown on demand, reused) and its launch settings.
 * Errors: TKF_ERR_INVALID_ARG (out == NULL), TKF_ERR_DEVICE (no such device),
 * TKF_ERR_UNSUPPORTED (device is not compute capability 10.3). */
tkf_status tkf_context_create(int device, tkf_context* out);
void tkf_context_destroy(tkf_context ctx);

/* Text of the last error on this context (valid until the next call on it). A NULL
 * context returns the last error of a create call. */
const char* tkf_last_error(tkf_context ctx);

/* ---------------------------------------------------------------------------- geometry */

/* One planar detector surface (paper Sec. 2: tracking geometry resident on the device). */
typedef struct tkf_surface_desc {
  double rot[9];     /* row-major 3x3 rotation; its columns are u, v and n = u x v (global frame) */
  double center[3];  /* origin of the local frame, mm */
  double thickness;  /* mm; 0 disables material effects on this surface */
  double x0;         /* radiation length of its material, mm */
} tkf_surface_desc;

/* Material constants of every surface (Bethe mean energy loss). */
typedef struct tkf_material {
  double z_over_a;        /* Z/A */
  double i_ev;            /* mean excitation energy, eV */
  double rho_g_cm3;       /* density, g/cm^3 */
  double hbar_omega_p_ev; /* plasma energy, eV (density-effect term) */
} tkf_material;

/* Silicon: Z/A 0.49848, I 173 eV, rho 2.329 g/cm^3, plasma energy 31.05 eV (PDG). */
void tkf_material_silicon(tkf_material* m);

/* Copies `n` host surface descriptions to device memory owned by the new handle (uploaded
 * once, paper Sec. 2). `material` may be NULL (silicon). The copy is synchronous.
 * Errors: TKF_ERR_INVALID_ARG (NULL pointers, n == 0, a rotation that is not orthonormal
 * to 1e-9, thickness < 0, x0 <= 0), TKF_ERR_OOM, TKF_ERR_DEVICE. */
tkf_status tkf_geometry_create(tkf_context ctx, const tkf_surface_desc* surfaces, uint32_t n,
                               const tkf_material* material, tkf_geometry* out);
void tkf_geometry_destroy(tkf_geometry geo);

/* ---------------------------------------------------------------------------- field */

typedef enum tkf_field_kind {
  TKF_FIELD_UNIFORM = 0, /* constant b_tesla */
  TKF_FIELD_RZ_GRID = 1  /* axially symmetric map: B_r, B_z on an (r, z) grid */
} tkf_field_kind;

/* Magnetic field (paper Sec. 3: a 2 T solenoid along z). For TKF_FIELD_RZ_GRID the nodes
 * are r = r0 + i dr (i < nr) and z = z0 + j dz (j < nz); br and bz are host arrays of
 * nz * nr floats, row-major [j][i], in tesla. The field at a point is the bilinear
 * interpolation in (r, z), with B_x = B_r x / r, B_y = B_r y / r (0 on the axis); outside
 * the grid it is 0 and the track is flagged TKF_TRACK_OUT_OF_FIELD. */
typedef struct tkf_field_desc {
  int kind;           /* tkf_field_kind */
  double b_tesla[3];  /* TKF_FIELD_UNIFORM */
  uint32_t nr, nz;    /* TKF_FIELD_RZ_GRID: >= 2 each */
  double r0, dr, z0, dz;
  const float* br;
  const float* bz;
} tkf_field_desc;

/* Copies the field to device memory owned by the new handle (synchronous).
 * Errors: TKF_ERR_INVALID_ARG (NULL, unknown kind, nr or nz < 2, dr or dz <= 0, r0 < 0,
 * NULL grid arrays), TKF_ERR_OOM, TKF_ERR_DEVICE. */
tkf_status tkf_field_create(tkf_context ctx, const tkf_field_desc* desc, tkf_field* out);
void tkf_field_destroy(tkf_field field);

/* ---------------------------------------------------------------------------- fit */

typedef enum tkf_precision {
  TKF_FP64 = 0,  /* every step in FP64 */
  TKF_MIXED = 1, /* propagation and transport in FP32 around FP64 anchors; update and
                    smoother in FP64 */
  TKF_MIXED_FP32 = 2 /* experimental, outside the FP64-update policy of TKF_MIXED: the mixed
                        path with the covariance algebra (Joseph update, smoother, covariance
                        transport results) in FP32 as well; FP64 is left only for the position
                        and direction anchors and the smoothed parameters. No record capture. */
} tkf_precision;

typedef enum tkf_step_mode {
  TKF_STEP_ADAPTIVE = 0, /* RKN step-size control from the local error estimate */
  TKF_STEP_LEARNED = 1   /* a small MLP proposes the starting step; the error estimate judges */
} tkf_step_mode;

typedef struct tkf_fit_options {
  int precision;       /* tkf_precision */
  int step_mode;       /* tkf_step_mode */
  double tol;          /* RKN local error tolerance, mm (default 1e-4) */
  double h_max;        /* largest step, mm (default 1000) */
  double h_min;        /* smallest step-size control value, mm (default 1e-4) */
  double surf_tol;     /* within this distance of the target plane a Taylor step lands on it, mm (1e-2) */
  uint32_t max_steps;  /* step attempts per surface (default 10000) */
  double mass;         /* particle hypothesis, GeV (default: muon, 0.1056583755) */
  tkf_mlp mlp;         /* step proposer for TKF_STEP_LEARNED, else NULL */
  /* Optional training-record capture (TKF_STEP_ADAPTIVE only): for every accepted RKN step
   * that the step-size control limited (the steps a proposer is asked about) and that has a
   * nonzero error estimate, TKF_MLP_RECORD floats are appended to `records` (DEVICE,
   * record_capacity records): the TKF_MLP_INPUTS network inputs at the step start and the
   * label ln(|h| (tol/eps)^(1/4) / mm), the largest step within tolerance. *record_count
   * (DEVICE, zeroed by the caller) counts every record, also those beyond the capacity. */
  float* records;
  uint32_t record_capacity;
  uint32_t* record_count;
  /* Launch policy (no effect on the results: every track's arithmetic is the same under any
   * launch shape). flags: TKF_FIT_AUTOTUNE and/or TKF_FIT_GRAPH, default 0. block_threads
   * (32, 64, 128 or 256) and blocks_per_sm (1..32) fix the persistent kernel's block shape
   * when both are nonzero (with the full register file unless max_registers says otherwise);
   * tracks_per_warp (1..32) fixes how many tracks a warp takes at a time, one per lane, when
   * nonzero; max_registers (255, or 128 / 64 for TKF_FP64 and TKF_MIXED and 128 for
   * TKF_MIXED_FP32, without record capture, blocks of at most 128 threads) picks the kernel
   * variant capped at that many registers a thread, which keeps part of the per-track state in
   * local memory (at 128 the smoother state in shared memory) and holds more warps per SM. With
   * all four 0 the shape is the tuned one of this launch class when TKF_FIT_AUTOTUNE is set,
   * else FP64: 128 threads x 2 blocks per SM, 255 registers; mixed: 128 x 4, 128 registers;
   * 32 tracks per warp. An explicit part disables tuning; the other parts take defaults. */
  uint32_t flags;
  uint32_t block_threads;
  uint32_t blocks_per_sm;
  uint32_t tracks_per_warp;
  uint32_t max_registers;
  /* Optional kernel timing: NULL, or two cudaEvent_t (begin, end; created by the caller)
   * that tkf_fit records on its stream right before and right after the persistent fit
   * kernel, so that cudaEventElapsedTime gives that kernel's duration alone (without the
   * ordering and proposal launches). A call with events launches directly (no graph). */
  void* const* kernel_events;
  /* Factor applied to every seed covariance element before the fit (default 1; must be > 0
   * and finite). A refit from an earlier pass's result (whose covariance already holds the
   * information of these measurements) inflates it, for example by 100, so that the
   * measurements are not counted twice. */
  double seed_cov_scale;
  /* Lanes a track (launch policy, no effect on the results): 0 = the default or tuned mapping,
   * 1 = one lane a track, 4 = group-per-track (TKF_FP64 or TKF_MIXED, 255 registers, no record
   * capture; at most 8 tracks a warp). In a group every lane steps the state, update and
   * smoother; lane g transports derivative column g and computes row g of the covariance
   * transport, exchanged by warp shuffles, which shortens each track's critical path when a
   * batch is too small to fill the GPU one lane a track. TKF_FIT_AUTOTUNE also times the group
   * mapping for small batches. */
  uint32_t lanes_per_track;
  /* Smoother that gives the first-surface result: TKF_SMOOTHER_RTS (default) or
   * TKF_SMOOTHER_TWO_FILTER, the optimal smoother of Sec. 4 (weighted mean of a forward and a
   * backward filter). The two-filter form runs, after the forward filter (whose chi2 is the
   * track's), a backward Kalman filter of the reversed particle (phi + pi, pi - theta, -q/p)
   * from the last entry to the first: it starts from the last filtered state with that
   * covariance times backward_inflation, updates with every measurement, and before each
   * earlier entry propagates to it and applies that surface's material (the scattering
   * variance; the mean energy loss given back). The result is the weighted mean of the
   * backward filtered state at the first surface and the seed. It propagates every track twice;
   * no per-measurement state is kept. One lane a track (lanes_per_track 0 or 1), no record
   * capture; 255 registers, or max_registers 128 / 64 in TKF_FP64 and TKF_MIXED. Default block
   * shape 128 threads x 2 blocks per SM (x 4 or x 8 when capped at 128 / 64) unless one is
   * given; TKF_FIT_AUTOTUNE times the block shapes and register caps as for RTS (one lane a
   * track), cached apart from RTS. */
  int smoother;
  /* TKF_SMOOTHER_TWO_FILTER: factor on the last filtered covariance that starts the backward
   * filter (default 1e3; finite and >= 1). The start then holds 1/backward_inflation of the
   * forward filter's information; larger factors let the first backward updates move the state
   * (and its linearisation) further. */
  double backward_inflation;
} tkf_fit_options;

#define TKF_SMOOTHER_RTS 0
#define TKF_SMOOTHER_TWO_FILTER 1

/* Autotuning: the first call of a launch class (precision, step mode, field kind, batch size
 * rounded down to a power of two, SM count) times every candidate launch shape on the call's
 * own inputs (six block shapes at 255 registers, and for the FP64 and mixed paths three each at
 * 128 and 64 registers; below one track per lane of every resident warp also 16, 8 and 4 tracks per
 * warp; each candidate runs the whole fit into the call's outputs, then the call runs with the
 * fastest shape) and keeps the winner in the context. The call synchronizes its stream while
 * tuning. If the environment variable TKF_AUTOTUNE_CACHE names a file when the context is
 * created, tuned shapes are read from it and every new one is written back (JSON object:
 * class -> [threads, blocks per SM, tracks per warp, registers]); an unreadable or unwritable
 * file is ignored. Skipped (defaults used) while the stream is capturing and in record-capture
 * mode. */
#define TKF_FIT_AUTOTUNE 1u
/* Graph replay: the ordering and fit launches of a call are captured into a CUDA graph on the
 * second consecutive call with identical arguments (every pointer, size, option, handle and
 * the block shape) and replayed as one graph launch by every further identical call; any
 * change of argument launches directly again. Needs a stream other than the legacy default
 * stream (ignored there and while the caller is itself capturing the stream). */
#define TKF_FIT_GRAPH 2u
/* For tests of the failure path of the learned mode's tensor-core pre-pass: the pre-pass
 * issues no tensor-core work, so its bounded waits for it run out (about 0.1 s); every track
 * then gets no proposal, starts from h_max and carries TKF_TRACK_PROPOSAL_FALLBACK. */
#define TKF_FIT_TEST_PROPOSAL_TIMEOUT (1u << 31)

void tkf_fit_options_default(tkf_fit_options* opts);

/* Surface-id flag of a track entry without a measurement (Sec. 2: the navigation passes every
 * surface a track crosses): a hole in a sensitive module, or a passive surface. The fit
 * propagates to the surface (sid & ~TKF_SID_NO_MEASUREMENT) and applies its material on
 * leaving it, and makes no update there; loc0, loc1, v00, v01, v11 of the entry are not read.
 * ndf counts measurements only. */
#define TKF_SID_NO_MEASUREMENT 0x80000000u

/* Inputs of one batch, all DEVICE pointers owned by the caller (read only).
 * Track i has the entries offsets[i] .. offsets[i+1]-1, ordered along the track.
 * Entry m: local position (loc0[m], loc1[m]) on surface sid[m] and its covariance
 * [[v00, v01], [v01, v11]] (mm^2), or a surface crossed without a measurement (sid[m] with
 * TKF_SID_NO_MEASUREMENT). The seed of track i is given on the surface of its first entry:
 * seed_par (5 x n_tracks) and seed_cov (15 x n_tracks, packed). */
typedef struct tkf_fit_inputs {
  uint32_t n_tracks;
  uint64_t n_meas;
  const uint32_t* offsets; /* n_tracks + 1 */
  const double* loc0;
  const double* loc1;
  const double* v00;
  const double* v01;
  const double* v11;
  const uint32_t* sid;
  const double* seed_par;
  const double* seed_cov;
} tkf_fit_inputs;

/* Outputs, DEVICE pointers owned by the caller (written). par (5 x n) and cov (15 x n) are
 * the smoothed parameters and covariance on the surface of the first measurement; chi2 is
 * the sum over measurements of the predicted-residual chi2, the first one taken against the
 * seed; ndf = 2 * (number of measurements) (the seed enters as a prior). steps, if not NULL,
 * receives 2 x n counters: step attempts [0, n) and rejected attempts [n, 2n).
 *
 * Optional all-states output (paper Sec. 2: the smoother lets every state use every
 * measurement): states_par (5 x n_meas) and states_cov (15 x n_meas, packed like cov), both
 * NULL or both set, receive the smoothed parameters and covariance at EVERY entry of every
 * track, in the measurements' indexing (entry k of track i at column offsets[i] + k; phi in
 * (-pi, pi], angles at entries without a measurement too). They come from the
 * Rauch-Tung-Striebel backward pass over stored filtered and predicted states and transport
 * Jacobians (A_k = C_k|k J_{k+1}^T C_{k+1|k}^-1, Cholesky), FP64, in a second kernel after the
 * fit; the context's workspace then also holds 360 bytes per measurement row. The entry-0 state
 * equals par / cov up to rounding (par / cov come from the forward-evaluated smoother). Rows of
 * a track whose status is fatal, or that has no measurement, are NaN; a predicted covariance that
 * is not positive definite in the backward pass sets TKF_TRACK_SMOOTHER_NOT_SPD (and NaN outputs)
 * as it does in the textbook smoother. Requires TKF_STEP_ADAPTIVE without record capture, the
 * RTS smoother and tkf_fit (not tkf_fit_host or tkf_fit_noalloc; TKF_ERR_UNSUPPORTED otherwise).
 * It runs one lane a track (lanes_per_track is ignored): by default 128 threads x 2 blocks per
 * SM at 255 registers; max_registers 128 / 64 (x 4 / x 8 blocks) where the precision has them;
 * TKF_FIT_AUTOTUNE times the one-lane shapes and register caps, cached apart from the plain fit.
 * NULL keeps the default path, unchanged and as fast. */
typedef struct tkf_fit_outputs {
  double* par;
  double* cov;
  double* chi2;
  int32_t* ndf;
  uint32_t* status;
  uint32_t* steps;
  double* states_par;
  double* states_cov;
} tkf_fit_outputs;

/* Fits every track of the batch, asynchronously on `stream` (a cudaStream_t; NULL is the
 * legacy default stream). Nothing is copied between host and device. Device pointers must
 * be 8-byte aligned and stay valid until the stream reaches this work.
 * Errors (nothing enqueued): TKF_ERR_INVALID_ARG (NULL required pointers, n_meas too large
 * for 32-bit offsets, bad options or block shape, misaligned pointers), TKF_ERR_BAD_HANDLE,
 * TKF_ERR_UNSUPPORTED (TKF_STEP_LEARNED without an mlp), TKF_ERR_DEVICE (launch, capture or
 * graph failure). Offsets are read on the device: a decreasing pair flags
 * TKF_TRACK_BAD_INPUT. The call blocks on the stream only when the context's workspace must
 * grow and while autotuning (TKF_FIT_AUTOTUNE, first call of a launch class). */
tkf_status tkf_fit(tkf_context ctx, tkf_geometry geo, tkf_field field, const tkf_fit_options* opts,
                   const tkf_fit_inputs* in, const tkf_fit_outputs* out, void* stream);

/* The same fit from HOST arrays: copies the inputs to a device staging area owned by the
 * context (grown on demand), fits, and copies the outputs back; returns when the outputs are
 * in host memory. Batches of at least 131,072 tracks are cut into chunks of consecutive tracks
 * (a twentieth of the batch first, then up to four equal chunks, each with its own launch
 * shape) pipelined over two copy streams of the context, `stream` and a second
 * compute stream (a chunk fits while its predecessor finishes its tail): the copy-in of a chunk
 * and the copy-out of the previous one overlap the fit of the current one (results identical
 * to one piece). A chunk copies the measurements between the least and the greatest of its
 * tracks' offsets, grown onto what earlier chunks copied as one interval (no byte twice). In
 * TKF_STEP_LEARNED the offsets, surface ids and seed parameters of the whole batch go first and
 * one proposal pre-pass serves every chunk. Page-locked host memory gives asynchronous copies.
 * `stream` is synchronized first (its earlier work must not use the staging area) and at the
 * end. Pointers as in tkf_fit_inputs / tkf_fit_outputs but in host memory. Errors as tkf_fit,
 * plus TKF_ERR_OOM. */
tkf_status tkf_fit_host(tkf_context ctx, tkf_geometry geo, tkf_field field,
                        const tkf_fit_options* opts, const tkf_fit_inputs* host_in,
                        const tkf_fit_outputs* host_out, void* stream);

/* ---------------------------------------------------------------------------- seed parameter estimation */

/* Track parameter estimation (Sec. 2 places it between seeding and track finding and prints no
 * method; this is the helix through three space points). For each track, three of its
 * measurements become space points r = c + loc0 u + loc1 v on their surfaces. In the plane
 * transverse to z the circle through them gives the radius R, the sense of turning (hence the
 * charge: F = q v x B) and the direction at the first point; z is linear in the transverse arc
 * length along a helix, which gives theta from points 1 and 3 (the arc followed in the sense
 * of travel, up to one full turn); p_T = 2.99792458e-4 |B_z| R (GeV, T, mm) with B_z the mean
 * of the field's z component at the three points. The result is expressed on the surface of
 * the track's first measurement: (loc0, loc1) = that measurement, phi, theta, q/p. It is exact
 * for noise-free hits of a track in a uniform axial field without material.
 *
 * Covariance (a prior for the fit, meant to be wide rather than narrow; all off-diagonal
 * elements 0 but (loc0, loc1)): the first measurement's 2x2 covariance; with sh2 the mean
 * per-coordinate hit variance of the three, L and L_T the 3D and transverse distances of points
 * 1 and 3, theta0 the Highland angle of the first surface (t / X0, normal incidence, beta = 1)
 * at the estimated momentum (1 GeV without curvature) and ms2 = (k3 - k1) theta0^2 for the
 * measurement indices k1 < k3 of points 1 and 3:
 *   var(theta) = 16 sh2 / L^2 + 2 ms2,
 *   rel2 = 4 sh2 / s^2 + ms2 L_T^2 / (16 s^2) + (dB / B_z)^2 + 1e-4   (s = L_T^2 / 8R, the
 *          sagitta; dB the spread of B_z over the three points),
 *   var(phi) = 64 sh2 / L_T^2 + 2 ms2 / sin^2(theta) + L_T^2 / (4 R^2) rel2,
 *   var(q/p) = rel2 (q/p)^2;
 * without curvature the last term of var(phi) is left out and var(q/p) = 1 GeV^-2; the angle
 * variances are capped at pi^2.
 *
 * `which` selects the measurements: TKF_SEED_FIRST_MIDDLE_LAST (the first, the one at index
 * (N - 1) / 2 and the last of the N; the longest lever arm of a candidate) or
 * TKF_SEED_FIRST_THREE (as for a seed of three inner space points). */
#define TKF_SEED_FIRST_MIDDLE_LAST 0u
#define TKF_SEED_FIRST_THREE 1u

/* Seed status bits: fewer than 3 measurements (parameters NaN, covariance 0); no curvature
 * (collinear points in the transverse plane, or B_z = 0: a straight line, q/p = 0); offsets
 * decreasing or beyond n_meas, or a surface id out of range (parameters NaN, covariance 0). */
#define TKF_SEED_TOO_FEW_HITS 1u
#define TKF_SEED_NO_CURVATURE 2u
#define TKF_SEED_BAD_INPUT 4u

/* Outputs, DEVICE pointers owned by the caller (written), in the layout of the fit's seed
 * inputs, so that they can be passed to tkf_fit as tkf_fit_inputs.seed_par / seed_cov. */
typedef struct tkf_seed_outputs {
  double* par;      /* 5 x n_tracks: loc0, loc1, phi, theta, q/p */
  double* cov;      /* 15 x n_tracks, packed upper triangle */
  uint32_t* status; /* n_tracks */
} tkf_seed_outputs;

/* Estimates the starting parameters of every track of the batch from its measurements,
 * asynchronously on `stream` (a cudaStream_t; NULL is the legacy default stream). Reads
 * offsets, loc0, loc1, v00, v01, v11 and sid of `in` (DEVICE pointers; seed_par and seed_cov
 * are not read and may be NULL). Device pointers must be 8-byte aligned and stay valid until
 * the stream reaches this work. One kernel launch, no allocation.
 * Errors (nothing enqueued): TKF_ERR_BAD_HANDLE (NULL context, geometry or field from another
 * context), TKF_ERR_INVALID_ARG (unknown `which`, NULL required pointers, misaligned pointers,
 * n_meas too large for 32-bit offsets), TKF_ERR_DEVICE (launch failure). Bad offsets or surface
 * ids are reported per track in `status`. */
tkf_status tkf_estimate_seeds(tkf_context ctx, tkf_geometry geo, tkf_field field, uint32_t which,
                              const tkf_fit_inputs* in, const tkf_seed_outputs* out, void* stream);

/* ---------------------------------------------------------------------------- track finding */

/* Track finding with a combinatorial Kalman filter (Sec. 2 places it after seeding and before
 * fitting, and prints no algorithm; this is the reading implemented). From a seed (parameters
 * and covariance on a sensitive surface) the filter navigates outward module by module. On
 * every module it crosses, each of the (at most 3) measurements with the lowest predicted chi2
 * below chi2_max makes a branch, and so does a hole (no measurement) while the branch has fewer
 * than max_holes consecutive holes. After every step a beam of the best `beam` branches is kept
 * (ranked by measurement count, more first; then consecutive holes, fewer first; then chi2,
 * lower first; then creation order). A branch ends when no module lies ahead, when a further
 * hole would exceed max_holes with no compatible measurement, or at max_entries entries; the
 * best ended branch is the seed's candidate. Propagation, material and the gain-matrix update
 * are the fit's (FP64, TKF_STEP_ADAPTIVE).
 *
 * Navigation uses the layer structure of the geometry (tkf_geometry_set_layers): from a state
 * on a module, the candidates are the modules of the same layer around the state (overlaps) and
 * those of the layers whose outer face the straight line from the state reaches ahead, in order
 * of path length; in a layer, the modules next to the crossing point (phi bin and row or ring,
 * +-1 each; the point on the parabola x + s T + s^2/2 k at the straight-line path s, k the
 * path's curvature vector kappa (q/p) T x B). A module is crossed if the parabola meets its plane
 * ahead (s > 1e-3 mm) within its half extents plus 1 mm + s^3 (kappa |q/p| |B|)^2 / 6; the
 * nearest is taken (crossings within 1e-6 mm of each other, coplanar overlapping modules, go to
 * the lower surface id; a layer is skipped once its face lies 20 mm beyond the best crossing).
 * The RKN propagation to it must end within its half extents in at most min(max_steps, 100)
 * attempts, else it is excluded and the navigation repeats (at most 4 exclusions). Surfaces
 * outside the layer structure are never candidates. */
#define TKF_CKF_MAX_ENTRIES 32u

/* Layer structure for navigation, host arrays copied to the device (replacing an earlier one).
 * layers [n_layers][8]:
 *   barrel cylinder: {0, r, n_phi, n_rows, row_pitch, first, half_u, half_v}: module (row iz,
 *     phi bin ip) has surface id first + iz n_phi + ip, its centre at phi 2 pi ip / n_phi and
 *     z = (iz - (n_rows - 1) / 2) row_pitch; modules at radius r or r + 1 mm, normal radial;
 *   endcap disk: {1, z, n_rings, first_ring, ring_pitch, r_inner, half_u, half_v}: rings
 *     first_ring .. first_ring + n_rings - 1 of `rings`, ring k covering radii from
 *     r_inner + k ring_pitch; modules at z or z + sign(z) 1 mm, normal along z;
 * rings [n_rings][4]: {r_centre, n_phi, first, 0}: module ip has surface id first + ip.
 * half_u, half_v: half extents of the layer's modules along their u and v axes (mm).
 * At most 32 layers. Errors: TKF_ERR_BAD_HANDLE, TKF_ERR_INVALID_ARG (NULL pointers, more than
 * 32 layers, surface ids or ring rows out of range), TKF_ERR_OOM / TKF_ERR_DEVICE. */
tkf_status tkf_geometry_set_layers(tkf_geometry geo, const double* layers, uint32_t n_layers, const double* rings,
                                   uint32_t n_rings);

typedef struct tkf_ckf_options {
  double chi2_max;      /* gate on the predicted chi2 of a measurement (2 dof; default 15) */
  uint32_t beam;        /* branches kept after every step (1..8; default 3) */
  uint32_t max_holes;   /* consecutive holes a branch may have (default 2) */
  uint32_t max_entries; /* entries (measurements and holes) of a candidate, 1..TKF_CKF_MAX_ENTRIES (24) */
} tkf_ckf_options;

void tkf_ckf_options_default(tkf_ckf_options* o);

/* Inputs, DEVICE pointers owned by the caller (read only): seeds (surface id, parameters 5 x n,
 * packed covariance 15 x n, the fit's seed layout) and the measurements of the event grouped by
 * surface: those of surface s are meas_offsets[s] .. meas_offsets[s+1]-1 (n_surfaces + 1
 * offsets, non-decreasing). Several events in one call (n_events > 1): meas_offsets holds
 * n_events consecutive arrays of n_surfaces + 1 offsets, all into the same measurement arrays,
 * and seed_event[i] (DEVICE, n_seeds) is the event of seed i, whose measurements alone it
 * searches; a seed whose event is >= n_events gets no candidate. One launch over the seeds of
 * many events fills the GPU where one event's seeds leave most of it idle. n_events 0 or 1
 * with seed_event NULL: one event. */
typedef struct tkf_ckf_inputs {
  uint32_t n_seeds;
  const uint32_t* seed_sid;
  const double* seed_par;
  const double* seed_cov;
  uint32_t n_meas;
  const uint32_t* meas_offsets;
  const double* loc0;
  const double* loc1;
  const double* v00;
  const double* v01;
  const double* v11;
  uint32_t n_events;
  const uint32_t* seed_event;
} tkf_ckf_inputs;

/* Outputs, DEVICE pointers owned by the caller (written): per seed the candidate's entry count,
 * measurement count and chi2 sum, and its entries in order, max_entries x n_seeds: entry_sid
 * (surface id, TKF_SID_NO_MEASUREMENT for a hole) and entry_meas (measurement index, -1 for a
 * hole); unused entries are 0 / -1. A seed whose surface is out of range gets 0 entries. The
 * entries are a fit input as they stand (holes included). */
typedef struct tkf_ckf_outputs {
  uint32_t* n_entries;
  uint32_t* n_meas;
  double* chi2;
  uint32_t* entry_sid;
  int32_t* entry_meas;
} tkf_ckf_outputs;

/* Finds the candidate of every seed, asynchronously on `stream`. fit_opts gives the propagation
 * and material options (step mode TKF_STEP_ADAPTIVE; launch policy fields ignored) and the
 * precision: TKF_FP64, or TKF_MIXED with the propagation, material and covariance transport in
 * FP32 around FP64 anchors as in the fit's mixed path (navigation, chi2 gate and update stay
 * FP64). The branch store (about 7 KB a seed at beam 3: branches and their history) is a workspace of the
 * context, grown on demand (the call then synchronizes the stream). Errors: TKF_ERR_BAD_HANDLE,
 * TKF_ERR_INVALID_ARG (NULL pointers, options out of range, no layer structure), TKF_ERR_OOM,
 * TKF_ERR_DEVICE. */
tkf_status tkf_find_tracks(tkf_context ctx, tkf_geometry geo, tkf_field field, const tkf_fit_options* fit_opts,
                           const tkf_ckf_options* ckf_opts, const tkf_ckf_inputs* in, const tkf_ckf_outputs* out,
                           void* stream);

/* ---------------------------------------------------------------------------- learned step proposer */

/* A learned addition to the paper's method (which has no learned component): before a track's
 * first RKN step, where the step-size control has no error estimate yet, a network proposes the
 * control's starting value from the seed state and the field at the first surface, toward the
 * second (the plain control starts from h_max and sheds it by rejected steps). From then on the
 * plain control adapts the value from the error estimates, and every step is accepted only if
 * the RKN error estimate passes, so proposals never loosen the tolerance. (Proposing every
 * control-limited step was measured to take more steps: once it exists, the control's own
 * estimate from the last step's error is the better predictor.) The proposals run in a
 * separate pre-pass kernel over all tracks.
 *
 * Network: TKF_MLP_INPUTS inputs -> 64 SiLU -> 64 SiLU -> 1 output, the natural log of the
 * largest step within tolerance in mm (proposal = 0.9 exp(output), clamped to [h_min, h_max]).
 * Inputs, at the step start: u, v, n components of (r - c_target) / 1000 mm; u, v, n components
 * of the direction; q/p (e/GeV); B / 2 T (global x, y, z); ln(last accepted step / mm) / 5; the
 * straight-line path to the target plane / 1000 mm, clamped to [-2, 2].
 * Parameter layout (TKF_MLP_PARAMS values): W1 [64][12] row-major, b1 [64], W2 [64][64],
 * b2 [64], w3 [64], b3 [1]. Inference uses BF16 weights and FP32 arithmetic.
 * For the starting proposal the inputs are taken at the seed state on the first surface, with
 * the second surface as the target and h_max as the last step. */
#define TKF_MLP_INPUTS 12
#define TKF_MLP_RECORD 13
#define TKF_MLP_PARAMS 5057

/* Uploads BF16 weights (host, n = TKF_MLP_PARAMS 16-bit patterns) into a handle for
 * tkf_fit_options.mlp. Errors: TKF_ERR_INVALID_ARG (NULL, n != TKF_MLP_PARAMS, a non-finite
 * weight), TKF_ERR_OOM, TKF_ERR_DEVICE. */
tkf_status tkf_mlp_load(tkf_context ctx, const uint16_t* bf16_weights, size_t n, tkf_mlp* out);
/* The same from trained FP32 parameters (DEVICE, n = TKF_MLP_PARAMS): each is rounded to BF16
 * (nearest, ties to even) by a kernel on `stream`; the call waits for it. Errors as
 * tkf_mlp_load (a non-finite parameter: TKF_ERR_INVALID_ARG, no handle). */
tkf_status tkf_mlp_load_f32(tkf_context ctx, const float* params, size_t n, tkf_mlp* out, void* stream);
void tkf_mlp_destroy(tkf_mlp mlp);

/* Initial FP32 parameters (DEVICE, n = TKF_MLP_PARAMS) for training, on `stream`: weights
 * uniform in (-1/sqrt(fan_in), 1/sqrt(fan_in)) from SplitMix64 of (seed, parameter index)
 * (fan_in 12 for W1, 64 for W2 and w3), biases 0. Deterministic for a seed. */
tkf_status tkf_mlp_init(tkf_context ctx, float* params, size_t n, uint64_t seed, void* stream);

/* Calibration after training: shifts the output bias b3 of the FP32 parameters (DEVICE, in
 * place) by the `quantile` (0..1) of the residuals label - output over the training records
 * (DEVICE [n][TKF_MLP_RECORD]), so that proposals 0.9 exp(output) rarely exceed the largest
 * step within tolerance (a rejected proposal costs an attempt, a short one only a little
 * length). The network's outputs and the residuals are FP32; the quantile interpolates
 * linearly between the order statistics at positions floor and ceil of quantile (n - 1),
 * which a radix select finds on the device; the shift is added to b3 in FP64 and rounded to
 * FP32, and returned in *shift (HOST). Waits for the work on `stream`. Scratch comes from the
 * context. Errors: TKF_ERR_INVALID_ARG (NULL, n = 0, quantile outside [0, 1]), TKF_ERR_OOM,
 * TKF_ERR_DEVICE. */
tkf_status tkf_mlp_calibrate(tkf_context ctx, float* params, const float* records, uint32_t n, double quantile,
                             double* shift, void* stream);

typedef struct tkf_mlp_train_options {
  uint32_t batch;   /* records per Adam step (1..8192); the last partial batch is dropped */
  uint32_t epochs;  /* passes over the records, in their given order */
  float lr, beta1, beta2, eps;  /* Adam (Kingma & Ba 2015); e.g. 1e-3, 0.9, 0.999, 1e-8 */
} tkf_mlp_train_options;

/* Trains FP32 parameters in place with mean-squared-error loss and Adam, with the library's
 * own forward, backward and update kernels, on `stream`. Every dense contraction of a step
 * runs on the tensor cores with BF16 operands (rounded to nearest even from FP32) and FP32
 * accumulation: the two layers, the backpropagation through layer 2 (dA1 = dZ2 W2), and the
 * weight and bias gradients of both layers (dW2 = dZ2^T A1, dW1 = dZ1^T X, sums of dZ2 and dZ1);
 * bias, SiLU, its derivative, the output layer and its gradient, and Adam are FP32 on the CUDA
 * cores; partial gradients of 128-sample tiles are summed in a fixed order (deterministic).
 * All pointers are DEVICE memory:
 * records [n][TKF_MLP_RECORD] (inputs, label), params [TKF_MLP_PARAMS], adam_moments
 * [2][TKF_MLP_PARAMS] (first and second moments; zero them before the first call),
 * epoch_loss [epochs] (mean loss of each epoch). *adam_t (HOST) counts the Adam steps taken so
 * far (0 before the first call) and is advanced. Scratch comes from the context workspace.
 * Errors: TKF_ERR_INVALID_ARG (NULL, batch out of range or larger than n), TKF_ERR_OOM,
 * TKF_ERR_DEVICE. */
tkf_status tkf_mlp_train(tkf_context ctx, const float* records, uint32_t n, const tkf_mlp_train_options* opts,
                         float* params, float* adam_moments, uint32_t* adam_t, float* epoch_loss, void* stream);

/* Mean squared error of the network on n samples (x [n][TKF_MLP_INPUTS], y [n], DEVICE) and
 * its gradient grad [TKF_MLP_PARAMS] (DEVICE), by the training kernels of tkf_mlp_train (BF16
 * operands in the contractions); loss is one DEVICE float. For checks of the training
 * kernels. Errors as tkf_mlp_train. */
tkf_status tkf_mlp_loss_grad(tkf_context ctx, const float* params, const float* x, const float* y, uint32_t n,
                             float* grad, float* loss, void* stream);

/* Raw outputs out [n] (DEVICE) of the network with FP32 params for x [n][TKF_MLP_INPUTS]. */
tkf_status tkf_mlp_forward(tkf_context ctx, const float* params, const float* x, uint32_t n, float* out,
                           void* stream);

/* Learned mode, the proposal pre-pass alone: h0[i] (DEVICE, n_tracks floats) receives the
 * starting step-size control that tkf_fit uses for track i with these options (opts->mlp
 * required, step_mode TKF_STEP_LEARNED): the network, its two dense layers on the tensor cores
 * (BF16 operands, FP32 accumulation), evaluated on the seed state at the first surface toward
 * the second; 0.9 exp(output rounded to a 1/32 grid), clamped to [h_min, h_max]; h_max for
 * tracks with fewer than two measurements or a bad surface id; -1 if the pre-pass timed out
 * waiting for its tensor-core work. For inspection and tests; asynchronous on `stream`.
 * Errors: as tkf_fit, TKF_ERR_INVALID_ARG for a NULL h0. The learned step proposer has no
 * counterpart in the paper. */
tkf_status tkf_propose_start(tkf_context ctx, tkf_geometry geo, tkf_field field, const tkf_fit_options* opts,
                             const tkf_fit_inputs* in, float* h0, void* stream);

/* ---------------------------------------------------------------------------- allocation-free fit */

/* The paper has no counterpart to this entry point. It is the fit of tkf_fit for callers that
 * may not allocate device memory while running: for example an online trigger or
 * reconstruction process that reserves all of its GPU memory at start-up and forbids later
 * allocations, or a host framework whose own memory pool owns the device. It calls no
 * cudaMalloc, cudaFree or other allocating routine: its scratch (work counter, sort keys and
 * track permutation, 16 MB) is a static device array of the library, held on every GPU that
 * loads the library until the process exits.
 *   - Batches are limited to TKF_NOALLOC_MAX_TRACKS tracks; a larger n_tracks returns
 *     TKF_ERR_INVALID_ARG with a message, and nothing is enqueued.
 *   - tkf_context_create looks up the array's device address on the context's device
 *     (cudaGetSymbolAddress) and keeps it in the context; the calls themselves look up nothing.
 *   - Every call on a device shares the one array: calls whose work overlaps on the GPU
 *     (different streams, or different contexts, without ordering) race and give wrong
 *     results. Serialize them.
 *   - It ignores the flags TKF_FIT_AUTOTUNE and TKF_FIT_GRAPH (both allocate); it launches with
 *     the shape tkf_fit uses without tuning (the explicit one of the options, else the default).
 *   - Learned step mode (TKF_STEP_LEARNED) returns TKF_ERR_UNSUPPORTED: it needs a per-track
 *     starting step, for which the static scratch has no room.
 *   - TKF_ERR_DEVICE if the array's address was not found when the context was created.
 * Arguments, outputs and the other errors are those of tkf_fit. */
#define TKF_NOALLOC_MAX_TRACKS 2097152u
tkf_status tkf_fit_noalloc(tkf_context ctx, tkf_geometry geo, tkf_field field, const tkf_fit_options* opts,
                           const tkf_fit_inputs* in, const tkf_fit_outputs* out, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* TKF_H_ */
