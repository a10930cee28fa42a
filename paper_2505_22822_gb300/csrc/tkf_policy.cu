// tkf_policy.cu -- launch policy of the fit: launch-shape autotuning and CUDA-graph replay.
//
// Neither changes what a track computes: every thread fits its own tracks with the same
// arithmetic whatever the launch shape, and a graph replays exactly the launches that a
// direct call makes.

#include <errno.h>
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <array>
#include <string>

#include "tkf_internal.cuh"

namespace tkf {
namespace {

// Candidates: (threads per block, blocks per SM, registers a thread). With 255 registers an SM
// holds 8 warps: the first four shapes fill it, the next two use half of it (less contention
// for the FP64 pipe and the L1 per warp). The FP64 and mixed paths also have kernels capped at
// 128 and 64 registers (16 and 32 warps an SM, part of the per-track state in local memory, the
// smoother state in shared memory at 128): more warps hide more latency, at the cost of spill
// traffic, and which balance wins depends on the precision, the field and the tracks.
struct Candidate {
  int threads, blocks_per_sm, regs;
};
constexpr Candidate kCandidates[] = {{32, 8, 255},   {64, 4, 255},   {128, 2, 255}, {256, 1, 255},
                                     {64, 2, 255},   {128, 1, 255},  {128, 4, 128}, {64, 8, 128},
                                     {32, 16, 128},  {128, 8, 64},   {64, 16, 64},  {32, 32, 64}};
// Tracks per warp: below one track per lane of every resident warp, fewer tracks per warp
// spread the batch over more schedulers. Small batches also try four lanes a track (full
// register file, FP64 and mixed, 8 to 1 tracks a warp): every lane of a group transports one
// derivative column and one row of the covariance transport, which shortens each track's
// critical path when the batch cannot fill the GPU one lane a track.
constexpr int kTracksPerWarp[] = {32, 16, 8, 4};
constexpr int kGroupTracksPerWarp[] = {8, 4, 2, 1};
constexpr int kResidentWarpsPerSm = 8;

// Defaults without tuning: FP64 128 x 2 at 255 registers; mixed 128 x 4 at 128 registers (the
// best single shape over the uniform-field and field-map batches); record capture keeps the
// full register file (its kernels exist only there).
std::array<int, 5> default_shape(int precision, bool record) {
  if (precision == TKF_MIXED && !record) return {128, 4, 32, 128, 1};
  return {128, 2, 32, 255, 1};
}

// Lanes a track the kernels of a precision and mode exist with.
bool has_group(int precision, bool record, int group) {
  if (group == 1) return true;
  return group == 4 && !record && (precision == TKF_FP64 || precision == TKF_MIXED);
}

// Register caps the kernels of a precision exist at.
bool has_regs(int precision, int regs) {
  if (regs == 255) return true;
  if (precision == TKF_MIXED || precision == TKF_FP64) return regs == 128 || regs == 64;
  if (precision == TKF_MIXED_FP32) return regs == 128;
  return false;
}

// The two-filter smoother's register caps: 255, and 128 / 64 in FP64 and mixed precision.
bool has_two_filter_regs(int precision, int regs) {
  return regs == 255 || ((precision == TKF_MIXED || precision == TKF_FP64) && (regs == 128 || regs == 64));
}

int field_class(const FieldDev& f) {
  if (f.kind != TKF_FIELD_UNIFORM) return 2;
  return (f.b[0] == 0.0 && f.b[1] == 0.0) ? 0 : 1;
}

int fit_mode(const FitArgs& a) { return a.mlp ? 1 : (a.records ? 2 : (a.states_par ? 3 : 0)); }

std::string tune_key(const FitArgs& a, const FieldDev& f, int precision, int sm_count) {
  static const char* kField[] = {"uz", "u", "grid"};
  int lg = 0;
  while ((2u << lg) <= a.n_tracks && lg < 31) ++lg;
  char buf[96];
  snprintf(buf, sizeof(buf), "%s%s.%s.%s.n%d.sm%d",
           precision == TKF_MIXED ? "mixed" : (precision == TKF_MIXED_FP32 ? "mixed_fp32" : "fp64"),
           a.smoother == TKF_SMOOTHER_TWO_FILTER ? "_two_filter" : "",
           fit_mode(a) == 1 ? "learned" : (fit_mode(a) == 2 ? "record" : (fit_mode(a) == 3 ? "states" : "adaptive")),
           kField[field_class(f)], lg,
           sm_count);
  return buf;
}

LaunchShape make_shape(const std::array<int, 5>& c, int sm_count) {
  LaunchShape s;
  s.threads = c[0];
  s.blocks = c[1] * sm_count;
  s.tracks_per_warp = c[2];
  s.regs = c[3];
  s.group = c[4];
  return s;
}

// Cache file: one JSON object, "class": [threads, blocks_per_sm, tracks_per_warp, registers,
// lanes_per_track].
void save_cache(const tkf_context ctx) {
  if (ctx->tune_cache_path.empty()) return;
  const std::string tmp = ctx->tune_cache_path + ".tmp";
  FILE* fp = fopen(tmp.c_str(), "w");
  if (!fp) return;
  fprintf(fp, "{\n");
  size_t k = 0;
  for (const auto& kv : ctx->tuned)
    fprintf(fp, "  \"%s\": [%d, %d, %d, %d, %d]%s\n", kv.first.c_str(), kv.second[0], kv.second[1], kv.second[2],
            kv.second[3], kv.second[4], ++k < ctx->tuned.size() ? "," : "");
  fprintf(fp, "}\n");
  const bool ok = fclose(fp) == 0;
  if (ok) rename(tmp.c_str(), ctx->tune_cache_path.c_str());
}

bool valid_shape(int threads, int bps, int regs) {
  return (threads == 32 || threads == 64 || threads == 128 || (threads == 256 && regs == 255)) && bps >= 1 &&
         bps <= 32 && (regs == 255 || regs == 128 || regs == 64);
}

// Times every candidate on the call's inputs: one warm-up fit, then the best of two fits each.
cudaError_t tune(tkf_context ctx, const FitArgs& a, const FieldDev& f, int precision, const Workspace& ws,
                 cudaStream_t stream, std::array<int, 5>* best) {
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  float best_ms = INFINITY;
  const bool two_filter = a.smoother == TKF_SMOOTHER_TWO_FILTER;  // one lane a track, its own caps
  const bool one_lane = two_filter || a.states_par != nullptr;     // the all-states mode: one lane too
  *best = one_lane ? std::array<int, 5>{128, 2, 32, 255, 1} : default_shape(precision, a.records != nullptr);
  if (e == cudaSuccess) e = launch_fit(a, f, precision, ws, make_shape(*best, ctx->sm_count), stream);
  const bool small = a.n_tracks < uint32_t(32 * kResidentWarpsPerSm * ctx->sm_count);
  const bool record = a.records != nullptr;
  for (int group : {1, 4}) {
    if (group != 1 && (one_lane || !small || !has_group(precision, record, group))) break;
    for (const int tpw : (group == 1 ? kTracksPerWarp : kGroupTracksPerWarp)) {
    if (group == 1 && tpw != 32 && !small) break;
    for (const Candidate& c : kCandidates) {
      if (e != cudaSuccess) break;
      if (!has_regs(precision, c.regs) || (group != 1 && c.regs != 255)) continue;
      if (two_filter && !has_two_filter_regs(precision, c.regs)) continue;
      const std::array<int, 5> cand = {c.threads, c.blocks_per_sm, tpw, c.regs, group};
      const LaunchShape s = make_shape(cand, ctx->sm_count);
      for (int rep = 0; rep < 2 && e == cudaSuccess; ++rep) {
        e = cudaEventRecord(e0, stream);
        if (e == cudaSuccess) e = launch_fit(a, f, precision, ws, s, stream);
        if (e == cudaSuccess) e = cudaEventRecord(e1, stream);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        float ms = 0.0f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        if (e == cudaSuccess && ms < best_ms) {
          best_ms = ms;
          *best = cand;
        }
      }
    }
    }
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  return e;
}

// Byte string of every launch argument: equal strings mean identical launches.
struct KeyWriter {
  std::string s;
  template <class T>
  void put(const T& v) {
    s.append(reinterpret_cast<const char*>(&v), sizeof(T));
  }
};

std::string graph_key(const FitArgs& a, const FieldDev& f, int precision, const Workspace& ws, LaunchShape shape) {
  KeyWriter k;
  k.put(precision);
  k.put(shape.threads);
  k.put(shape.blocks);
  k.put(shape.tracks_per_warp);
  k.put(shape.regs);
  k.put(shape.group);
  k.put(a.n_tracks);
  k.put(a.stride);
  k.put(a.n_meas);
  const void* ptrs[] = {a.offsets, a.loc0,   a.loc1,  a.v00,      a.v01,     a.v11,
                        a.sid,     a.seed_par, a.seed_cov, a.par,   a.cov,     a.chi2,
                        a.ndf,     a.status, a.steps, a.surf,     a.mlp,     a.records,
                        a.record_count, ws.counter, ws.hist, ws.keys, ws.perm, ws.h0, f.grid,
                        a.states_par, a.states_cov, ws.states};
  for (const void* p : ptrs) k.put(p);
  k.put(a.n_surf);
  k.put(a.record_capacity);
  k.put(a.test_stall_proposals);
  k.put(a.smoother);
  const double dm[] = {a.mat.z_over_a, a.mat.i_ev, a.mat.rho, a.mat.hwp_ev, a.mat.log_hwp_over_i, a.mat.bg2_density,
                       a.opt.tol, a.opt.h_max, a.opt.h_min, a.opt.surf_tol, a.opt.mass, a.seed_cov_scale, a.backward_inflation, f.b[0], f.b[1], f.b[2],
                       f.r0, f.dr, f.z0, f.dz, f.inv_dr, f.inv_dz};
  for (double d : dm) k.put(d);
  const float fm[] = {a.mat.log_hwp_over_i_f, a.mat.bg2_density_f, a.mat.two_me_over_i2_f, a.mat.dedx_scale_f,
                      a.opt.tol_f, a.opt.h_max_f, a.opt.h_min_f, a.opt.mass_f, a.opt.me_over_mass_f,
                      a.opt.surf_tol_f};
  for (float x : fm) k.put(x);
  k.put(a.opt.max_steps);
  k.put(f.kind);
  k.put(f.nr);
  k.put(f.nz);
  return k.s;
}

}  // namespace

void load_tune_cache(tkf_context ctx) {
  const char* path = getenv("TKF_AUTOTUNE_CACHE");
  if (!path || !*path) return;
  ctx->tune_cache_path = path;
  FILE* fp = fopen(path, "r");
  if (!fp) return;
  std::string text;
  char buf[4096];
  size_t n;
  while ((n = fread(buf, 1, sizeof(buf), fp)) > 0) text.append(buf, n);
  fclose(fp);
  // entries "class": [threads, blocks_per_sm, tracks_per_warp, registers(, lanes_per_track)];
  // anything else is skipped
  size_t pos = 0;
  while ((pos = text.find('"', pos)) != std::string::npos) {
    const size_t end = text.find('"', pos + 1);
    if (end == std::string::npos) break;
    const std::string key = text.substr(pos + 1, end - pos - 1);
    const size_t lb = text.find('[', end);
    const size_t next = text.find('"', end + 1);
    pos = end + 1;
    if (lb == std::string::npos || (next != std::string::npos && next < lb)) continue;
    int t = 0, b = 0, w = 0, r = 0, g = 1;
    const int got = sscanf(text.c_str() + lb, "[ %d , %d , %d , %d , %d ]", &t, &b, &w, &r, &g);
    if (got == 4) g = 1;
    if (got >= 4 && valid_shape(t, b, r) && (g == 1 || (g == 4 && r == 255)) && w >= 1 && w * g <= 32)
      ctx->tuned[key] = {t, b, w, r, g};
  }
}

void release_graph(tkf_context ctx) {
  if (ctx->graph_exec) cudaGraphExecDestroy(ctx->graph_exec);
  ctx->graph_exec = nullptr;
  ctx->graph_key.clear();
  ctx->pending_key.clear();
}

bool valid_block_shape(uint32_t threads, uint32_t blocks_per_sm, uint32_t tracks_per_warp, uint32_t max_registers,
                       uint32_t lanes_per_track, int precision, bool record) {
  if (tracks_per_warp > 32) return false;
  if (lanes_per_track > 1) {
    if (!has_group(precision, record, int(lanes_per_track))) return false;
    if (tracks_per_warp * lanes_per_track > 32 || (max_registers != 0 && max_registers != 255)) return false;
  }
  if (max_registers != 0 && max_registers != 255 && max_registers != 128 && max_registers != 64) return false;
  if (max_registers != 0 && (!has_regs(precision, int(max_registers)) || (max_registers != 255 && record)))
    return false;
  if (threads == 0 && blocks_per_sm == 0) return true;
  return valid_shape(int(threads), int(blocks_per_sm), max_registers ? int(max_registers) : 255);
}

cudaError_t resolve_shape(tkf_context ctx, const FitArgs& a, const FieldDev& f, int precision, const Workspace& ws,
                          const tkf_fit_options* o, cudaStream_t stream, LaunchShape* out) {
  // record capture exists at 255 registers, one lane a track; the all-states output defaults to it
  const bool full_file = a.records != nullptr || a.states_par != nullptr;
  std::array<int, 5> shape = default_shape(precision, full_file);
  const bool explicit_block = o->block_threads && o->blocks_per_sm;
  if (explicit_block) {
    shape[0] = int(o->block_threads);
    shape[1] = int(o->blocks_per_sm);
    shape[3] = 255;  // an explicit block shape runs the full register file unless told otherwise
  }
  if (o->lanes_per_track > 1) {
    shape[4] = int(o->lanes_per_track);
    shape[3] = 255;
    shape[2] = 32 / shape[4];
  }
  if (o->tracks_per_warp) shape[2] = int(o->tracks_per_warp);
  if (o->max_registers) shape[3] = int(o->max_registers);
  *out = make_shape(shape, ctx->sm_count);
  if (a.states_par) {  // one lane a track; 255 registers unless capped
    if (!explicit_block) {
      out->threads = 128;
      out->blocks = 2 * ctx->sm_count;
    }
    out->regs = o->max_registers && has_regs(precision, int(o->max_registers)) ? int(o->max_registers) : 255;
    out->group = 1;
    if (out->regs != 255 && !explicit_block)  // a capped kernel: 128 threads, the SM's registers full
      out->blocks = (65536 / (out->regs * 128)) * ctx->sm_count;
  }
  if (a.smoother == TKF_SMOOTHER_TWO_FILTER) {  // one lane a track; 255 registers unless capped
    if (!explicit_block) {
      out->threads = 128;
      out->blocks = 2 * ctx->sm_count;
    }
    out->regs = o->max_registers && has_two_filter_regs(precision, int(o->max_registers)) ? int(o->max_registers) : 255;
    out->group = 1;
    if (out->regs != 255 && !explicit_block)  // a capped kernel: 128 threads, the SM's registers full
      out->blocks = (65536 / (out->regs * 128)) * ctx->sm_count;
  }
  const bool any_explicit = explicit_block || o->tracks_per_warp || o->max_registers || o->lanes_per_track;
  if (any_explicit || !(o->flags & TKF_FIT_AUTOTUNE) || a.records) return cudaSuccess;
  const std::string key = tune_key(a, f, precision, ctx->sm_count);
  auto it = ctx->tuned.find(key);
  if (it != ctx->tuned.end()) {
    *out = make_shape(it->second, ctx->sm_count);
    return cudaSuccess;
  }
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  cudaError_t e = cudaStreamIsCapturing(stream, &cs);
  if (e != cudaSuccess || cs != cudaStreamCaptureStatusNone) return e;
  std::array<int, 5> best;
  e = tune(ctx, a, f, precision, ws, stream, &best);
  if (e != cudaSuccess) return e;
  ctx->tuned[key] = best;
  save_cache(ctx);
  *out = make_shape(best, ctx->sm_count);
  return cudaSuccess;
}

LaunchShape default_launch_shape(int precision, bool record, int sm_count) {
  return make_shape(default_shape(precision, record), sm_count);
}

cudaError_t launch_with_policy(tkf_context ctx, const FitArgs& a, const FieldDev& f, int precision,
                               const Workspace& ws, LaunchShape shape, bool use_graph, cudaStream_t stream,
                               const cudaEvent_t* timing) {
  if (!use_graph || timing || stream == nullptr || stream == cudaStreamLegacy)
    return launch_fit(a, f, precision, ws, shape, stream, timing);
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  cudaError_t e = cudaStreamIsCapturing(stream, &cs);
  if (e != cudaSuccess) return e;
  if (cs != cudaStreamCaptureStatusNone) return launch_fit(a, f, precision, ws, shape, stream);
  std::string key = graph_key(a, f, precision, ws, shape);
  if (ctx->graph_exec && key == ctx->graph_key) return cudaGraphLaunch(ctx->graph_exec, stream);
  if (key != ctx->pending_key) {
    // first call with these arguments: launch directly and remember them
    ctx->pending_key = std::move(key);
    return launch_fit(a, f, precision, ws, shape, stream);
  }
  // second consecutive call with these arguments: capture, instantiate (or update), launch
  cudaGraph_t g = nullptr;
  e = cudaStreamBeginCapture(stream, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) return e;
  const cudaError_t le = launch_fit(a, f, precision, ws, shape, stream);
  e = cudaStreamEndCapture(stream, &g);
  if (le != cudaSuccess || e != cudaSuccess) {
    if (g) cudaGraphDestroy(g);
    return le != cudaSuccess ? le : e;
  }
  if (ctx->graph_exec) {
    cudaGraphExecUpdateResultInfo info;
    if (cudaGraphExecUpdate(ctx->graph_exec, g, &info) != cudaSuccess) {
      cudaGetLastError();
      cudaGraphExecDestroy(ctx->graph_exec);
      ctx->graph_exec = nullptr;
    }
  }
  if (!ctx->graph_exec) {
    e = cudaGraphInstantiate(&ctx->graph_exec, g, 0);
    if (e != cudaSuccess) {
      cudaGraphDestroy(g);
      ctx->graph_exec = nullptr;
      ctx->graph_key.clear();
      return e;
    }
  }
  cudaGraphDestroy(g);
  ctx->graph_key = std::move(key);
  ctx->pending_key.clear();
  return cudaGraphLaunch(ctx->graph_exec, stream);
}

}  // namespace tkf
