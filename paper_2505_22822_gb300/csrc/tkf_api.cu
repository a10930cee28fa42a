// tkf_api.cu -- the C interface declared in include/tkf.h: handles, validation, launches.

#include <cuda_runtime.h>
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <new>
#include <string>
#include <vector>

#include "tkf_internal.cuh"

namespace {

thread_local std::string g_create_error;

tkf_status fail(tkf_context ctx, tkf_status code, const std::string& msg) {
  if (ctx)
    ctx->last_error = msg;
  else
    g_create_error = msg;
  return code;
}

tkf_status cuda_fail(tkf_context ctx, cudaError_t e, const char* what) {
  std::string m = std::string(what) + ": " + cudaGetErrorString(e);
  return fail(ctx, e == cudaErrorMemoryAllocation ? TKF_ERR_OOM : TKF_ERR_DEVICE, m);
}

// Makes the context's device current for the duration of a call and restores the caller's.
struct DeviceGuard {
  int prev = -1;
  bool ok = true;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    if (prev != dev) ok = cudaSetDevice(dev) == cudaSuccess;
  }
  ~DeviceGuard() {
    int cur = -1;
    if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
  }
};

bool aligned8(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 7u) == 0; }

// Device address of the allocation-free entry point's static scratch on the current device
// (defined with the array, at the end of this file).
cudaError_t noalloc_scratch_address(void** out);

// Host-buffer entry point: a batch of at least two kHostChunkMinTracks is cut into a small first
// chunk and up to four chunks of at least kHostChunkMinTracks tracks, whose copies overlap the
// fits of their neighbours.
constexpr size_t kHostChunkMinTracks = 65536;

}  // namespace

extern "C" {

tkf_status tkf_context_create(int device, tkf_context* out) {
  if (!out) return fail(nullptr, TKF_ERR_INVALID_ARG, "tkf_context_create: out is NULL");
  *out = nullptr;
  int n = 0;
  cudaError_t e = cudaGetDeviceCount(&n);
  if (e != cudaSuccess || n == 0) {
    cudaGetLastError();
    return fail(nullptr, TKF_ERR_DEVICE, std::string("tkf_context_create: no CUDA device (") +
                                             (e == cudaSuccess ? "count 0" : cudaGetErrorString(e)) + ")");
  }
  if (device < 0) {
    if (cudaGetDevice(&device) != cudaSuccess) return fail(nullptr, TKF_ERR_DEVICE, "cudaGetDevice failed");
  }
  if (device >= n) return fail(nullptr, TKF_ERR_DEVICE, "tkf_context_create: device index out of range");
  cudaDeviceProp prop;
  if (cudaGetDeviceProperties(&prop, device) != cudaSuccess)
    return fail(nullptr, TKF_ERR_DEVICE, "cudaGetDeviceProperties failed");
  if (!(prop.major == 10 && prop.minor == 3))
    return fail(nullptr, TKF_ERR_UNSUPPORTED,
                "tkf_context_create: this library is built for sm_103a (GB300); device is sm_" +
                    std::to_string(prop.major) + std::to_string(prop.minor));
  tkf_context c = new (std::nothrow) tkf_context_s();
  if (!c) return fail(nullptr, TKF_ERR_OOM, "tkf_context_create: host allocation failed");
  c->device = device;
  c->sm_count = prop.multiProcessorCount;
  {
    // the allocation-free entry point's scratch: its device address in this device's context
    // (host code cannot use the array's name as a device address); a failure only disables
    // tkf_fit_noalloc on this context
    DeviceGuard g(device);
    if (!g.ok || noalloc_scratch_address(&c->noalloc_scratch) != cudaSuccess) {
      c->noalloc_scratch = nullptr;
      cudaGetLastError();
    }
  }
  tkf::load_tune_cache(c);
  *out = c;
  return TKF_OK;
}

void tkf_context_destroy(tkf_context ctx) {
  if (!ctx) return;
  if (ctx->stage || ctx->ws || ctx->train_ws || ctx->graph_exec || ctx->h2d_stream || ctx->ckf_ws) {
    DeviceGuard g(ctx->device);
    tkf::release_graph(ctx);
    for (int c = 0; c < kHostChunksMax; ++c) {
      if (ctx->chunk_in[c]) cudaEventDestroy(ctx->chunk_in[c]);
      if (ctx->chunk_fit[c]) cudaEventDestroy(ctx->chunk_fit[c]);
    }
    if (ctx->props_in) cudaEventDestroy(ctx->props_in);
    if (ctx->props_done) cudaEventDestroy(ctx->props_done);
    if (ctx->h2d_stream) cudaStreamDestroy(ctx->h2d_stream);
    if (ctx->d2h_stream) cudaStreamDestroy(ctx->d2h_stream);
    if (ctx->fit2_stream) cudaStreamDestroy(ctx->fit2_stream);
    if (ctx->stage) cudaFree(ctx->stage);
    if (ctx->ws) cudaFree(ctx->ws);
    if (ctx->train_ws) cudaFree(ctx->train_ws);
    if (ctx->ckf_ws) cudaFree(ctx->ckf_ws);
  }
  delete ctx;
}

const char* tkf_last_error(tkf_context ctx) {
  return ctx ? ctx->last_error.c_str() : g_create_error.c_str();
}

void tkf_material_silicon(tkf_material* m) {
  if (!m) return;
  m->z_over_a = 0.49848;
  m->i_ev = 173.0;
  m->rho_g_cm3 = 2.329;
  m->hbar_omega_p_ev = 31.05;
}

tkf_status tkf_geometry_create(tkf_context ctx, const tkf_surface_desc* s, uint32_t n, const tkf_material* mat,
                               tkf_geometry* out) {
  if (!ctx) return fail(nullptr, TKF_ERR_BAD_HANDLE, "tkf_geometry_create: NULL context");
  if (!out || !s || n == 0) return fail(ctx, TKF_ERR_INVALID_ARG, "tkf_geometry_create: NULL pointer or n == 0");
  *out = nullptr;
  tkf_material m;
  if (mat)
    m = *mat;
  else
    tkf_material_silicon(&m);
  if (!(m.z_over_a > 0 && m.i_ev > 0 && m.rho_g_cm3 > 0 && m.hbar_omega_p_ev > 0))
    return fail(ctx, TKF_ERR_INVALID_ARG, "tkf_geometry_create: material constants must be positive");
  double* host = new (std::nothrow) double[size_t(n) * tkf::kSurfStride];
  if (!host) return fail(ctx, TKF_ERR_OOM, "tkf_geometry_create: host allocation failed");
  for (uint32_t i = 0; i < n; ++i) {
    const tkf_surface_desc& d = s[i];
    double col[3][3];  // col[c] = column c of rot
    for (int c = 0; c < 3; ++c)
      for (int r = 0; r < 3; ++r) col[c][r] = d.rot[r * 3 + c];
    bool ok = true;
    for (int a = 0; a < 3; ++a)
      for (int b = 0; b < 3; ++b) {
        double dp = col[a][0] * col[b][0] + col[a][1] * col[b][1] + col[a][2] * col[b][2];
        if (fabs(dp - (a == b ? 1.0 : 0.0)) > 1e-9) ok = false;
      }
    // n must be u x v (right-handed frame)
    double cx = col[0][1] * col[1][2] - col[0][2] * col[1][1];
    double cy = col[0][2] * col[1][0] - col[0][0] * col[1][2];
    double cz = col[0][0] * col[1][1] - col[0][1] * col[1][0];
    if (fabs(cx - col[2][0]) > 1e-9 || fabs(cy - col[2][1]) > 1e-9 || fabs(cz - col[2][2]) > 1e-9) ok = false;
    if (!ok || !(d.thickness >= 0.0) || !(d.x0 > 0.0) || !isfinite(d.center[0]) || !isfinite(d.center[1]) ||
        !isfinite(d.center[2])) {
      delete[] host;
      return fail(ctx, TKF_ERR_INVALID_ARG,
                  "tkf_geometry_create: surface " + std::to_string(i) +
                      " has a non-orthonormal or left-handed frame, negative thickness or x0 <= 0");
    }
    double* o = host + size_t(i) * tkf::kSurfStride;
    for (int r = 0; r < 3; ++r) {
      o[r] = col[0][r];
      o[3 + r] = col[1][r];
      o[6 + r] = col[2][r];
      o[9 + r] = d.center[r];
    }
    o[12] = d.thickness;
    o[13] = d.x0;
    o[14] = d.thickness / d.x0;
    o[15] = (d.thickness > 0.0) ? sqrt(o[14]) * (1.0 + 0.038 * log(o[14])) : 0.0;
    float* f = reinterpret_cast<float*>(o + 16);
    for (int r = 0; r < 3; ++r) {
      f[r] = float(col[0][r]);
      f[3 + r] = float(col[1][r]);
      f[6 + r] = float(col[2][r]);
    }
    f[9] = float(d.thickness);
    f[10] = float(d.thickness / d.x0);
    for (int r = 0; r < 3; ++r) f[11 + r] = float(d.center[r]);
    f[14] = 0.0f;
    f[15] = 0.0f;
  }
  DeviceGuard g(ctx->device);
  if (!g.ok) {
    delete[] host;
    return fail(ctx, TKF_ERR_DEVICE, "tkf_geometry_create: cudaSetDevice failed");
  }
  double* dev = nullptr;
  cudaError_t e = cudaMalloc(&dev, size_t(n) * tkf::kSurfStride * sizeof(double));
  if (e != cudaSuccess) {
    delete[] host;
    return cuda_fail(ctx, e, "tkf_geometry_create: cudaMalloc");
  }
  e = cudaMemcpy(dev, host, size_t(n) * tkf::kSurfStride * sizeof(double), cudaMemcpyHostToDevice);
  delete[] host;
  if (e != cudaSuccess) {
    cudaFree(dev);
    return cuda_fail(ctx, e, "tkf_geometry_create: cudaMemcpy");
  }
  tkf_geometry h = new (std::nothrow) tkf_geometry_s();
  if (!h) {
    cudaFree(dev);
    return fail(ctx, TKF_ERR_OOM, "tkf_geometry_create: host allocation failed");
  }
  h->ctx = ctx;
  h->device = ctx->device;
  h->d_surf = dev;
  h->n = n;
  h->mat.z_over_a = m.z_over_a;
  h->mat.i_ev = m.i_ev;
  h->mat.rho = m.rho_g_cm3;
  h->mat.hwp_ev = m.hbar_omega_p_ev;
  h->mat.log_hwp_over_i = log(m.hbar_omega_p_ev / m.i_ev);
  h->mat.bg2_density = exp(1.0 - 2.0 * h->mat.log_hwp_over_i);
  h->mat.log_hwp_over_i_f = float(h->mat.log_hwp_over_i);
  h->mat.bg2_density_f = float(h->mat.bg2_density);
  const double I = m.i_ev * 1e-9;
  h->mat.two_me_over_i2_f = float(2.0 * 0.51099895e-3 / (I * I));
  h->mat.dedx_scale_f = float(0.307075 * m.z_over_a * m.rho_g_cm3 * 1e-4);
  *out = h;
  return TKF_OK;
}

void tkf_geometry_destroy(tkf_geometry geo) {
  if (!geo) return;
  DeviceGuard g(geo->device);
  cudaFree(geo->d_surf);
  if (geo->d_layers) cudaFree(geo->d_layers);
  if (geo->d_rings) cudaFree(geo->d_rings);
  if (geo->d_layer_of) cudaFree(geo->d_layer_of);
  delete geo;
}

tkf_status tkf_geometry_set_layers(tkf_geometry geo, const double* layers, uint32_t n_layers, const double* rings,
                                   uint32_t n_rings) {
  if (!geo) return fail(nullptr, TKF_ERR_BAD_HANDLE, "tkf_geometry_set_layers: NULL geometry");
  tkf_context ctx = geo->ctx;
  if (!layers || n_layers == 0 || (n_rings && !rings))
    return fail(ctx, TKF_ERR_INVALID_ARG, "tkf_geometry_set_layers: NULL or empty layer table");
  if (n_layers > 32) return fail(ctx, TKF_ERR_INVALID_ARG, "tkf_geometry_set_layers: more than 32 layers");
  // the layer of every surface; every module id and ring row must be in range
  std::vector<int32_t> layer_of(geo->n, -1);
  for (uint32_t li = 0; li < n_layers; ++li) {
    const double* l = layers + 8 * size_t(li);
    bool ok = (l[0] == 0.0 || l[0] == 1.0) && l[2] >= 1.0 && l[3] >= (l[0] == 0.0 ? 1.0 : 0.0) && l[4] > 0.0 &&
              l[6] > 0.0 && l[7] > 0.0;
    if (ok && l[0] == 0.0) {
      const double cnt = l[2] * l[3];
      ok = l[5] >= 0.0 && l[5] + cnt <= double(geo->n);
      for (uint32_t k = 0; ok && k < uint32_t(cnt); ++k) layer_of[uint32_t(l[5]) + k] = int32_t(li);
    } else if (ok) {
      ok = l[3] >= 0.0 && l[3] + l[2] <= double(n_rings);
      for (uint32_t k = 0; ok && k < uint32_t(l[2]); ++k) {
        const double* rg = rings + 4 * (size_t(l[3]) + k);
        ok = rg[1] >= 1.0 && rg[2] >= 0.0 && rg[2] + rg[1] <= double(geo->n);
        for (uint32_t ip = 0; ok && ip < uint32_t(rg[1]); ++ip) layer_of[uint32_t(rg[2]) + ip] = int32_t(li);
      }
    }
    if (!ok)
      return fail(ctx, TKF_ERR_INVALID_ARG,
                  "tkf_geometry_set_layers: layer " + std::to_string(li) + " malformed or out of range");
  }
  DeviceGuard g(geo->device);
  if (!g.ok) return fail(ctx, TKF_ERR_DEVICE, "tkf_geometry_set_layers: cudaSetDevice failed");
  double *dl = nullptr, *dr = nullptr;
  int32_t* dlo = nullptr;
  cudaError_t e = cudaMalloc(&dl, sizeof(double) * 8 * n_layers);
  if (e == cudaSuccess) e = cudaMalloc(&dr, sizeof(double) * 4 * (n_rings ? n_rings : 1));
  if (e == cudaSuccess) e = cudaMalloc(&dlo, sizeof(int32_t) * (geo->n ? geo->n : 1));
  if (e == cudaSuccess) e = cudaMemcpy(dl, layers, sizeof(double) * 8 * n_layers, cudaMemcpyHostToDevice);
  if (e == cudaSuccess && n_rings) e = cudaMemcpy(dr, rings, sizeof(double) * 4 * n_rings, cudaMemcpyHostToDevice);
  if (e == cudaSuccess && geo->n)
    e = cudaMemcpy(dlo, layer_of.data(), sizeof(int32_t) * geo->n, cudaMemcpyHostToDevice);
  if (e != cudaSuccess) {
    if (dl) cudaFree(dl);
    if (dr) cudaFree(dr);
    if (dlo) cudaFree(dlo);
    return cuda_fail(ctx, e, "tkf_geometry_set_layers: upload");
  }
  if (geo->d_layers) cudaFree(geo->d_layers);
  if (geo->d_rings) cudaFree(geo->d_rings);
  if (geo->d_layer_of) cudaFree(geo->d_layer_of);
  geo->d_layers = dl;
  geo->d_rings = dr;
  geo->d_layer_of = dlo;
  geo->n_layers = n_layers;
  geo->n_rings = n_rings;
  return TKF_OK;
}

void tkf_ckf_options_default(tkf_ckf_options* o) {
  if (!o) return;
  o->chi2_max = 15.0;
  o->beam = 3;
  o->max_holes = 2;
  o->max_entries = 24;
}

tkf_status tkf_field_create(tkf_context ctx, const tkf_field_desc* d, tkf_field* out) {
  if (!ctx) return fail(nullptr, TKF_ERR_BAD_HANDLE, "tkf_field_create: NULL context");
  if (!d || !out) return fail(ctx, TKF_ERR_INVALID_ARG, "tkf_field_create: NULL pointer");
  *out = nullptr;
  tkf::FieldDev f{};
  f.kind = d->kind;
  float2* dev = nullptr;
  if (d->kind == TKF_FIELD_UNIFORM) {
    for (int i = 0; i < 3; ++i) {
      if (!isfinite(d->b_tesla[i])) return fail(ctx, TKF_ERR_INVALID_ARG, "tkf_field_create: non-finite field");
      f.b[i] = d->b_tesla[i];
    }
  } else if (d->kind == TKF_FIELD_RZ_GRID) {
    if (d->nr < 2 || d->nz < 2 || !(d->dr > 0) || !(d->dz > 0) || !(d->r0 >= 0) || !d->br || !d->bz ||
        !isfinite(d->z0))
      return fail(ctx, TKF_ERR_INVALID_ARG,
                  "tkf_field_create: grid needs nr, nz >= 2, dr, dz > 0, r0 >= 0 and both arrays");
    size_t cnt = size_t(d->nr) * d->nz;
    if (cnt > (size_t(1) << 31)) return fail(ctx, TKF_ERR_INVALID_ARG, "tkf_field_create: grid too large");
    float2* host = new (std::nothrow) float2[cnt];
    if (!host) return fail(ctx, TKF_ERR_OOM, "tkf_field_create: host allocation failed");
    for (size_t i = 0; i < cnt; ++i) host[i] = make_float2(d->br[i], d->bz[i]);
    DeviceGuard g(ctx->device);
    cudaError_t e = cudaMalloc(&dev, cnt * sizeof(float2));
    if (e != cudaSuccess) {
      delete[] host;
      return cuda_fail(ctx, e, "tkf_field_create: cudaMalloc");
    }
    e = cudaMemcpy(dev, host, cnt * sizeof(float2), cudaMemcpyHostToDevice);
    delete[] host;
    if (e != cudaSuccess) {
      cudaFree(dev);
      return cuda_fail(ctx, e, "tkf_field_create: cudaMemcpy");
    }
    f.nr = int(d->nr);
    f.nz = int(d->nz);
    f.r0 = d->r0;
    f.dr = d->dr;
    f.z0 = d->z0;
    f.dz = d->dz;
    f.inv_dr = 1.0 / d->dr;
    f.inv_dz = 1.0 / d->dz;
    f.grid = dev;
  } else {
    return fail(ctx, TKF_ERR_INVALID_ARG, "tkf_field_create: unknown field kind");
  }
  tkf_field h = new (std::nothrow) tkf_field_s();
  if (!h) {
    if (dev) cudaFree(dev);
    return fail(ctx, TKF_ERR_OOM, "tkf_field_create: host allocation failed");
  }
  h->ctx = ctx;
  h->device = ctx->device;
  h->f = f;
  h->d_grid = dev;
  *out = h;
  return TKF_OK;
}

void tkf_field_destroy(tkf_field field) {
  if (!field) return;
  if (field->d_grid) {
    DeviceGuard g(field->device);
    cudaFree(field->d_grid);
  }
  delete field;
}

void tkf_fit_options_default(tkf_fit_options* o) {
  if (!o) return;
  o->precision = TKF_FP64;
  o->step_mode = TKF_STEP_ADAPTIVE;
  o->tol = 1e-4;
  o->h_max = 1000.0;
  o->h_min = 1e-4;
  o->surf_tol = 1e-2;
  o->max_steps = 10000;
  o->mass = 0.1056583755;
  o->mlp = nullptr;
  o->records = nullptr;
  o->record_capacity = 0;
  o->record_count = nullptr;
  o->flags = 0;
  o->block_threads = 0;
  o->blocks_per_sm = 0;
  o->tracks_per_warp = 0;
  o->max_registers = 0;
  o->kernel_events = nullptr;
  o->seed_cov_scale = 1.0;
  o->lanes_per_track = 0;
  o->smoother = TKF_SMOOTHER_RTS;
  o->backward_inflation = 1e3;
}

// Validation shared by the fit entry points; `out` may be NULL only when `need_out` is false.
static tkf_status check_common(tkf_context ctx, tkf_geometry geo, tkf_field field, const tkf_fit_options* o,
                               const tkf_fit_inputs* in, const tkf_fit_outputs* out, const char* fn,
                               bool need_out = true) {
  if (!ctx) return fail(nullptr, TKF_ERR_BAD_HANDLE, std::string(fn) + ": NULL context");
  if (!geo || !field || geo->ctx != ctx || field->ctx != ctx)
    return fail(ctx, TKF_ERR_BAD_HANDLE, std::string(fn) + ": geometry or field handle NULL or from another context");
  if (!o || !in || (need_out && !out))
    return fail(ctx, TKF_ERR_INVALID_ARG, std::string(fn) + ": NULL options, inputs or outputs");
  if (!(o->precision == TKF_FP64 || o->precision == TKF_MIXED || o->precision == TKF_MIXED_FP32))
    return fail(ctx, TKF_ERR_INVALID_ARG, std::string(fn) + ": unknown precision");
  if (o->precision == TKF_MIXED_FP32 && o->records)
    return fail(ctx, TKF_ERR_UNSUPPORTED, std::string(fn) + ": record capture runs in TKF_FP64 or TKF_MIXED");
  if (!(o->step_mode == TKF_STEP_ADAPTIVE || o->step_mode == TKF_STEP_LEARNED))
    return fail(ctx, TKF_ERR_INVALID_ARG, std::string(fn) + ": unknown step mode");
  if (o->step_mode == TKF_STEP_LEARNED && !o->mlp)
    return fail(ctx, TKF_ERR_UNSUPPORTED, std::string(fn) + ": TKF_STEP_LEARNED needs an mlp handle");
  if (o->step_mode == TKF_STEP_LEARNED && o->mlp->ctx != ctx)
    return fail(ctx, TKF_ERR_BAD_HANDLE, std::string(fn) + ": mlp handle from another context");
  if (o->records && (!o->record_count || o->record_capacity == 0 || o->step_mode != TKF_STEP_ADAPTIVE))
    return fail(ctx, TKF_ERR_INVALID_ARG,
                std::string(fn) + ": record capture needs record_count, a capacity and TKF_STEP_ADAPTIVE");
  if (!(o->tol > 0) || !(o->h_max > 0) || !(o->h_min > 0) || !(o->h_min <= o->h_max) || !(o->surf_tol > 0) ||
      o->max_steps == 0 || !(o->mass > 0) || !isfinite(o->h_max))
    return fail(ctx, TKF_ERR_INVALID_ARG,
                std::string(fn) + ": options need tol, h_max, h_min, surf_tol, mass > 0, h_min <= h_max, max_steps > 0");
  if (!(o->seed_cov_scale > 0) || !isfinite(o->seed_cov_scale))
    return fail(ctx, TKF_ERR_INVALID_ARG, std::string(fn) + ": seed_cov_scale must be positive and finite");
  if (!(o->smoother == TKF_SMOOTHER_RTS || o->smoother == TKF_SMOOTHER_TWO_FILTER))
    return fail(ctx, TKF_ERR_INVALID_ARG, std::string(fn) + ": unknown smoother");
  if (o->smoother == TKF_SMOOTHER_TWO_FILTER) {
    if (!(o->backward_inflation >= 1.0) || !isfinite(o->backward_inflation))
      return fail(ctx, TKF_ERR_INVALID_ARG, std::string(fn) + ": backward_inflation must be finite and >= 1");
    const bool capped = o->max_registers == 128 || o->max_registers == 64;
    if (o->records || o->lanes_per_track > 1 || (o->max_registers != 0 && o->max_registers != 255 && !capped) ||
        (capped && o->precision == TKF_MIXED_FP32))
      return fail(ctx, TKF_ERR_UNSUPPORTED,
                  std::string(fn) + ": TKF_SMOOTHER_TWO_FILTER runs one lane a track without record capture, at "
                                    "255 registers (or 128 / 64 in TKF_FP64 and TKF_MIXED)");
  }
  if ((o->flags & ~(TKF_FIT_AUTOTUNE | TKF_FIT_GRAPH | TKF_FIT_TEST_PROPOSAL_TIMEOUT)) != 0)
    return fail(ctx, TKF_ERR_INVALID_ARG, std::string(fn) + ": unknown flag");
  if (!tkf::valid_block_shape(o->block_threads, o->blocks_per_sm, o->tracks_per_warp, o->max_registers,
                              o->lanes_per_track, o->precision, o->records != nullptr))
    return fail(ctx, TKF_ERR_INVALID_ARG,
                std::string(fn) + ": block shape needs threads 32, 64, 128 or 256 (at most 128 below 255 registers) "
                                  "and 1..32 blocks per SM (or 0, 0), 0..32 tracks per warp, and max_registers 0, 255, "
                                  "or 128 / 64 for the mixed path without record capture; lanes_per_track 0, 1, or 4 "
                                  "(TKF_FP64 or TKF_MIXED, 255 registers, at most 8 tracks per warp, no record capture)");
  if (in->n_meas > 0xffffffffull)
    return fail(ctx, TKF_ERR_INVALID_ARG, std::string(fn) + ": n_meas exceeds 32-bit offsets");
  if (in->n_tracks == 0) return TKF_OK;
  if (!in->offsets || !in->seed_par || !in->seed_cov)
    return fail(ctx, TKF_ERR_INVALID_ARG, std::string(fn) + ": NULL required pointer");
  if (out && (!out->par || !out->cov || !out->chi2 || !out->ndf || !out->status))
    return fail(ctx, TKF_ERR_INVALID_ARG, std::string(fn) + ": NULL required pointer");
  if (out && (!out->states_par != !out->states_cov))
    return fail(ctx, TKF_ERR_INVALID_ARG, std::string(fn) + ": states_par and states_cov must both be set or both NULL");
  if (out && out->states_par &&
      (o->step_mode != TKF_STEP_ADAPTIVE || o->records || o->smoother != TKF_SMOOTHER_RTS))
    return fail(ctx, TKF_ERR_UNSUPPORTED,
                std::string(fn) + ": the all-states output needs TKF_STEP_ADAPTIVE without record capture and the "
                                  "RTS smoother");
  if (out && (!aligned8(out->states_par) || !aligned8(out->states_cov)))
    return fail(ctx, TKF_ERR_INVALID_ARG, std::string(fn) + ": states pointer not 8-byte aligned");
  if (in->n_meas > 0 && (!in->loc0 || !in->loc1 || !in->v00 || !in->v01 || !in->v11 || !in->sid))
    return fail(ctx, TKF_ERR_INVALID_ARG, std::string(fn) + ": NULL measurement pointer");
  const void* ptrs[] = {in->loc0, in->loc1, in->v00, in->v01, in->v11, in->seed_par, in->seed_cov,
                        out ? out->par : nullptr, out ? out->cov : nullptr, out ? out->chi2 : nullptr};
  for (const void* p : ptrs)
    if (!aligned8(p)) return fail(ctx, TKF_ERR_INVALID_ARG, std::string(fn) + ": pointer not 8-byte aligned");
  return TKF_OK;
}

static tkf::FitArgs make_args(tkf_geometry geo, const tkf_fit_options* o, const tkf_fit_inputs* in,
                              const tkf_fit_outputs* out) {
  tkf::FitArgs a{};
  a.n_tracks = in->n_tracks;
  a.stride = in->n_tracks;
  a.n_meas = in->n_meas;
  a.offsets = in->offsets;
  a.loc0 = in->loc0;
  a.loc1 = in->loc1;
  a.v00 = in->v00;
  a.v01 = in->v01;
  a.v11 = in->v11;
  a.sid = in->sid;
  a.seed_par = in->seed_par;
  a.seed_cov = in->seed_cov;
  a.seed_cov_scale = o->seed_cov_scale;
  a.smoother = o->smoother;
  a.backward_inflation = o->backward_inflation;
  if (out) {
    a.par = out->par;
    a.cov = out->cov;
    a.chi2 = out->chi2;
    a.ndf = out->ndf;
    a.status = out->status;
    a.steps = out->steps;
    a.states_par = out->states_par;
    a.states_cov = out->states_cov;
  }
  a.surf = geo->d_surf;
  a.n_surf = geo->n;
  a.mat = geo->mat;
  a.opt.tol = o->tol;
  a.opt.h_max = o->h_max;
  a.opt.h_min = o->h_min;
  a.opt.surf_tol = o->surf_tol;
  a.opt.mass = o->mass;
  a.opt.max_steps = o->max_steps;
  a.opt.tol_f = float(o->tol);
  a.opt.h_max_f = float(o->h_max);
  a.opt.h_min_f = float(o->h_min);
  a.opt.mass_f = float(o->mass);
  a.opt.me_over_mass_f = float(0.51099895e-3 / o->mass);
  a.opt.surf_tol_f = float(o->surf_tol);
  a.mlp = (o->step_mode == TKF_STEP_LEARNED && o->mlp) ? o->mlp->d_weights : nullptr;
  a.records = (o->step_mode == TKF_STEP_ADAPTIVE) ? o->records : nullptr;
  a.record_capacity = o->record_capacity;
  a.record_count = o->record_count;
  a.test_stall_proposals = (o->flags & TKF_FIT_TEST_PROPOSAL_TIMEOUT) != 0;
  return a;
}

// Enqueues the fit of `a` (device pointers) on `stream`: grows the workspace if needed, picks
// the launch shape, launches directly or through the graph cache.
static tkf_status fit_enqueue(tkf_context ctx, tkf_field field, const tkf_fit_options* o, const tkf::FitArgs& a,
                              cudaStream_t st, bool allow_graph, const char* fn) {
  const bool learned = o->step_mode == TKF_STEP_LEARNED;
  const uint64_t states = a.states_par ? a.n_meas : 0;  // rows of the all-states scratch
  const size_t need = tkf::workspace_bytes(a.n_tracks, learned, states);
  if (need > ctx->ws_bytes) {
    // the old workspace may still be in use by earlier work on this context's stream
    cudaError_t e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(ctx, e, (std::string(fn) + ": stream synchronize").c_str());
    if (ctx->ws) cudaFree(ctx->ws);
    ctx->ws = nullptr;
    ctx->ws_bytes = 0;
    e = cudaMalloc(&ctx->ws, need);
    if (e != cudaSuccess) return cuda_fail(ctx, e, (std::string(fn) + ": workspace cudaMalloc").c_str());
    ctx->ws_bytes = need;
  }
  tkf::Workspace ws = tkf::carve_workspace(ctx->ws, a.n_tracks, learned, states);
  tkf::LaunchShape shape;
  cudaError_t e = tkf::resolve_shape(ctx, a, field->f, o->precision, ws, o, st, &shape);
  if (e != cudaSuccess) return cuda_fail(ctx, e, (std::string(fn) + ": autotune").c_str());
  const cudaEvent_t* timing = reinterpret_cast<const cudaEvent_t*>(o->kernel_events);
  e = tkf::launch_with_policy(ctx, a, field->f, o->precision, ws, shape,
                              allow_graph && (o->flags & TKF_FIT_GRAPH) != 0, st, timing);
  if (e != cudaSuccess) return cuda_fail(ctx, e, (std::string(fn) + ": launch").c_str());
  return TKF_OK;
}

tkf_status tkf_fit(tkf_context ctx, tkf_geometry geo, tkf_field field, const tkf_fit_options* o,
                   const tkf_fit_inputs* in, const tkf_fit_outputs* out, void* stream) {
  tkf_status s = check_common(ctx, geo, field, o, in, out, "tkf_fit");
  if (s != TKF_OK || in->n_tracks == 0) return s;
  DeviceGuard g(ctx->device);
  if (!g.ok) return fail(ctx, TKF_ERR_DEVICE, "tkf_fit: cudaSetDevice failed");
  return fit_enqueue(ctx, field, o, make_args(geo, o, in, out), static_cast<cudaStream_t>(stream), true, "tkf_fit");
}

tkf_status tkf_propose_start(tkf_context ctx, tkf_geometry geo, tkf_field field, const tkf_fit_options* o,
                             const tkf_fit_inputs* in, float* h0, void* stream) {
  tkf_status s = check_common(ctx, geo, field, o, in, nullptr, "tkf_propose_start", false);
  if (s != TKF_OK) return s;
  if (o->step_mode != TKF_STEP_LEARNED)
    return fail(ctx, TKF_ERR_INVALID_ARG, "tkf_propose_start: needs TKF_STEP_LEARNED and an mlp handle");
  if (in->n_tracks == 0) return TKF_OK;
  if (!h0) return fail(ctx, TKF_ERR_INVALID_ARG, "tkf_propose_start: NULL h0");
  DeviceGuard g(ctx->device);
  if (!g.ok) return fail(ctx, TKF_ERR_DEVICE, "tkf_propose_start: cudaSetDevice failed");
  tkf::FitArgs a = make_args(geo, o, in, nullptr);
  cudaError_t e = tkf::launch_propose_start(a, field->f, h0, static_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return cuda_fail(ctx, e, "tkf_propose_start: launch");
  return TKF_OK;
}

tkf_status tkf_estimate_seeds(tkf_context ctx, tkf_geometry geo, tkf_field field, uint32_t which,
                              const tkf_fit_inputs* in, const tkf_seed_outputs* out, void* stream) {
  const char* fn = "tkf_estimate_seeds";
  if (!ctx) return fail(nullptr, TKF_ERR_BAD_HANDLE, std::string(fn) + ": NULL context");
  if (!geo || !field || geo->ctx != ctx || field->ctx != ctx)
    return fail(ctx, TKF_ERR_BAD_HANDLE, std::string(fn) + ": geometry or field handle NULL or from another context");
  if (!in || !out) return fail(ctx, TKF_ERR_INVALID_ARG, std::string(fn) + ": NULL inputs or outputs");
  if (which != TKF_SEED_FIRST_MIDDLE_LAST && which != TKF_SEED_FIRST_THREE)
    return fail(ctx, TKF_ERR_INVALID_ARG, std::string(fn) + ": unknown measurement selection");
  if (in->n_meas > 0xffffffffull)
    return fail(ctx, TKF_ERR_INVALID_ARG, std::string(fn) + ": n_meas exceeds 32-bit offsets");
  if (in->n_tracks == 0) return TKF_OK;
  if (!in->offsets || !out->par || !out->cov || !out->status)
    return fail(ctx, TKF_ERR_INVALID_ARG, std::string(fn) + ": NULL required pointer");
  if (in->n_meas > 0 && (!in->loc0 || !in->loc1 || !in->v00 || !in->v01 || !in->v11 || !in->sid))
    return fail(ctx, TKF_ERR_INVALID_ARG, std::string(fn) + ": NULL measurement pointer");
  const void* ptrs[] = {in->loc0, in->loc1, in->v00, in->v01, in->v11, out->par, out->cov};
  for (const void* p : ptrs)
    if (!aligned8(p)) return fail(ctx, TKF_ERR_INVALID_ARG, std::string(fn) + ": pointer not 8-byte aligned");
  DeviceGuard g(ctx->device);
  if (!g.ok) return fail(ctx, TKF_ERR_DEVICE, std::string(fn) + ": cudaSetDevice failed");
  tkf::SeedArgs a{};
  a.n_tracks = in->n_tracks;
  a.n_meas = in->n_meas;
  a.offsets = in->offsets;
  a.loc0 = in->loc0;
  a.loc1 = in->loc1;
  a.v00 = in->v00;
  a.v01 = in->v01;
  a.v11 = in->v11;
  a.sid = in->sid;
  a.surf = geo->d_surf;
  a.n_surf = geo->n;
  a.first_three = which == TKF_SEED_FIRST_THREE ? 1u : 0u;
  a.par = out->par;
  a.cov = out->cov;
  a.status = out->status;
  cudaError_t e = tkf::launch_estimate_seeds(a, field->f, ctx->sm_count, static_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return cuda_fail(ctx, e, (std::string(fn) + ": launch").c_str());
  return TKF_OK;
}

tkf_status tkf_find_tracks(tkf_context ctx, tkf_geometry geo, tkf_field field, const tkf_fit_options* o,
                           const tkf_ckf_options* co, const tkf_ckf_inputs* in, const tkf_ckf_outputs* out,
                           void* stream) {
  const char* fn = "tkf_find_tracks";
  if (!ctx) return fail(nullptr, TKF_ERR_BAD_HANDLE, std::string(fn) + ": NULL context");
  if (!geo || !field || geo->ctx != ctx || field->ctx != ctx)
    return fail(ctx, TKF_ERR_BAD_HANDLE, std::string(fn) + ": geometry or field handle NULL or from another context");
  if (!o || !co || !in || !out) return fail(ctx, TKF_ERR_INVALID_ARG, std::string(fn) + ": NULL argument");
  if (!(o->precision == TKF_FP64 || o->precision == TKF_MIXED) || o->step_mode != TKF_STEP_ADAPTIVE)
    return fail(ctx, TKF_ERR_INVALID_ARG, std::string(fn) + ": needs TKF_FP64 or TKF_MIXED, and TKF_STEP_ADAPTIVE");
  if (!(o->tol > 0) || !(o->h_max > 0) || !(o->h_min > 0) || !(o->h_min <= o->h_max) || !(o->surf_tol > 0) ||
      o->max_steps == 0 || !(o->mass > 0) || !isfinite(o->h_max))
    return fail(ctx, TKF_ERR_INVALID_ARG, std::string(fn) + ": fit options out of range");
  if (!(co->chi2_max >= 0) || co->beam < 1 || co->beam > 8 || co->max_entries < 1 ||
      co->max_entries > TKF_CKF_MAX_ENTRIES)
    return fail(ctx, TKF_ERR_INVALID_ARG,
                std::string(fn) + ": ckf options need chi2_max >= 0, beam 1..8, max_entries 1..TKF_CKF_MAX_ENTRIES");
  if (!geo->d_layers) return fail(ctx, TKF_ERR_INVALID_ARG, std::string(fn) + ": geometry has no layer structure");
  if (in->n_seeds == 0) return TKF_OK;
  if (!in->seed_sid || !in->seed_par || !in->seed_cov || !in->meas_offsets || !out->n_entries || !out->n_meas ||
      !out->chi2 || !out->entry_sid || !out->entry_meas)
    return fail(ctx, TKF_ERR_INVALID_ARG, std::string(fn) + ": NULL required pointer");
  if (in->n_meas > 0 && (!in->loc0 || !in->loc1 || !in->v00 || !in->v01 || !in->v11))
    return fail(ctx, TKF_ERR_INVALID_ARG, std::string(fn) + ": NULL measurement pointer");
  if (in->n_events > 1 && !in->seed_event)
    return fail(ctx, TKF_ERR_INVALID_ARG, std::string(fn) + ": several events need seed_event");
  const void* ptrs[] = {in->seed_par, in->seed_cov, in->loc0, in->loc1, in->v00, in->v01, in->v11, out->chi2};
  for (const void* p : ptrs)
    if (!aligned8(p)) return fail(ctx, TKF_ERR_INVALID_ARG, std::string(fn) + ": pointer not 8-byte aligned");
  DeviceGuard g(ctx->device);
  if (!g.ok) return fail(ctx, TKF_ERR_DEVICE, std::string(fn) + ": cudaSetDevice failed");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const size_t need = tkf::ckf_workspace_bytes(in->n_seeds, co->beam, in->n_meas, co->max_entries);
  if (need > ctx->ckf_ws_bytes) {
    cudaError_t e = cudaStreamSynchronize(st);  // the old store may still be in use
    if (e != cudaSuccess) return cuda_fail(ctx, e, (std::string(fn) + ": stream synchronize").c_str());
    if (ctx->ckf_ws) cudaFree(ctx->ckf_ws);
    ctx->ckf_ws = nullptr;
    ctx->ckf_ws_bytes = 0;
    e = cudaMalloc(&ctx->ckf_ws, need);
    if (e != cudaSuccess) return cuda_fail(ctx, e, (std::string(fn) + ": branch store cudaMalloc").c_str());
    ctx->ckf_ws_bytes = need;
  }
  tkf_fit_inputs dummy_in{};
  tkf::FitArgs fa = make_args(geo, o, &dummy_in, nullptr);
  tkf::CkfArgs a{};
  a.n_seeds = in->n_seeds;
  a.seed_sid = in->seed_sid;
  a.seed_par = in->seed_par;
  a.seed_cov = in->seed_cov;
  a.meas_off = in->meas_offsets;
  a.n_meas = in->n_meas;
  a.seed_event = in->seed_event;
  a.n_events = in->seed_event ? (in->n_events > 1 ? in->n_events : 1u) : 1u;
  a.loc0 = in->loc0;
  a.loc1 = in->loc1;
  a.v00 = in->v00;
  a.v01 = in->v01;
  a.v11 = in->v11;
  a.surf = geo->d_surf;
  a.n_surf = geo->n;
  a.layers = geo->d_layers;
  a.n_layers = geo->n_layers;
  a.rings = geo->d_rings;
  a.n_rings = geo->n_rings;
  a.layer_of = geo->d_layer_of;
  a.mat = fa.mat;
  a.opt = fa.opt;
  a.chi2_max = co->chi2_max;
  a.beam = co->beam;
  a.max_holes = co->max_holes;
  a.max_entries = co->max_entries;
  a.mixed = o->precision == TKF_MIXED;
  a.n_entries = out->n_entries;
  a.n_meas_out = out->n_meas;
  a.chi2 = out->chi2;
  a.entry_sid = out->entry_sid;
  a.entry_meas = out->entry_meas;
  a.ws = ctx->ckf_ws;
  cudaError_t e = tkf::launch_find_tracks(a, field->f, st);
  if (e != cudaSuccess) return cuda_fail(ctx, e, (std::string(fn) + ": launch").c_str());
  return TKF_OK;
}

tkf_status tkf_fit_host(tkf_context ctx, tkf_geometry geo, tkf_field field, const tkf_fit_options* o,
                        const tkf_fit_inputs* hin, const tkf_fit_outputs* hout, void* stream) {
  tkf_status s = check_common(ctx, geo, field, o, hin, hout, "tkf_fit_host");
  if (s == TKF_OK && hout->states_par)
    return fail(ctx, TKF_ERR_UNSUPPORTED, "tkf_fit_host: the all-states output is available through tkf_fit");
  if (s != TKF_OK || hin->n_tracks == 0) return s;
  DeviceGuard g(ctx->device);
  if (!g.ok) return fail(ctx, TKF_ERR_DEVICE, "tkf_fit_host: cudaSetDevice failed");
  const size_t n = hin->n_tracks, m = hin->n_meas;
  auto up = [](size_t b) { return (b + 255) & ~size_t(255); };
  const size_t b_off = up((n + 1) * 4), b_meas = up(m * 8), b_sid = up(m * 4), b_seedp = up(5 * n * 8),
               b_seedc = up(15 * n * 8), b_par = up(5 * n * 8), b_cov = up(15 * n * 8), b_n8 = up(n * 8),
               b_n4 = up(n * 4), b_steps = hout->steps ? up(2 * n * 4) : 0,
               b_h0 = o->step_mode == TKF_STEP_LEARNED ? up(n * 4) : 0;
  const size_t total =
      b_off + 5 * b_meas + b_sid + b_seedp + b_seedc + b_par + b_cov + b_n8 + 2 * b_n4 + b_steps + b_h0;
  if (total > ctx->stage_bytes) {
    if (ctx->stage) cudaFree(ctx->stage);
    ctx->stage = nullptr;
    ctx->stage_bytes = 0;
    cudaError_t e = cudaMalloc(&ctx->stage, total);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "tkf_fit_host: staging cudaMalloc");
    ctx->stage_bytes = total;
  }
  char* p = static_cast<char*>(ctx->stage);
  auto take = [&p](size_t b) {
    char* q = p;
    p += b;
    return q;
  };
  tkf_fit_inputs din = *hin;
  tkf_fit_outputs dout{};
  din.offsets = reinterpret_cast<uint32_t*>(take(b_off));
  din.loc0 = reinterpret_cast<double*>(take(b_meas));
  din.loc1 = reinterpret_cast<double*>(take(b_meas));
  din.v00 = reinterpret_cast<double*>(take(b_meas));
  din.v01 = reinterpret_cast<double*>(take(b_meas));
  din.v11 = reinterpret_cast<double*>(take(b_meas));
  din.sid = reinterpret_cast<uint32_t*>(take(b_sid));
  din.seed_par = reinterpret_cast<double*>(take(b_seedp));
  din.seed_cov = reinterpret_cast<double*>(take(b_seedc));
  dout.par = reinterpret_cast<double*>(take(b_par));
  dout.cov = reinterpret_cast<double*>(take(b_cov));
  dout.chi2 = reinterpret_cast<double*>(take(b_n8));
  dout.ndf = reinterpret_cast<int32_t*>(take(b_n4));
  dout.status = reinterpret_cast<uint32_t*>(take(b_n4));
  dout.steps = hout->steps ? reinterpret_cast<uint32_t*>(take(b_steps)) : nullptr;
  float* h0_all = b_h0 ? reinterpret_cast<float*>(take(b_h0)) : nullptr;  // learned mode: the proposals
  // Pipeline over chunks of tracks: the copy-in of chunk c + 1 (h2d stream) and the copy-out of
  // chunk c - 1 (d2h stream) overlap the fit of chunk c (the caller's stream). Each chunk is the
  // tracks [t0, t1) with the measurements they can reference, copied to the same positions of
  // full-size staging arrays, so offsets stay absolute; seeds and outputs are SoA rows of the
  // full batch, so a chunk's fit runs with the batch's row stride.
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  cudaError_t e = cudaSuccess;
  if (!ctx->h2d_stream) {
    e = cudaStreamCreateWithFlags(&ctx->h2d_stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&ctx->d2h_stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&ctx->fit2_stream, cudaStreamNonBlocking);
    for (int c = 0; c < kHostChunksMax && e == cudaSuccess; ++c) {
      e = cudaEventCreateWithFlags(&ctx->chunk_in[c], cudaEventDisableTiming);
      if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ctx->chunk_fit[c], cudaEventDisableTiming);
    }
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ctx->props_in, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ctx->props_done, cudaEventDisableTiming);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "tkf_fit_host: stream or event creation");
  }
  // chunk schedule: a small first chunk (a twentieth of the batch), so that the first fit starts
  // soon after the first copies, then up to four equal chunks (large chunks keep the persistent
  // fit's tail short)
  uint32_t chunks = 1;
  size_t bound[kHostChunksMax + 1] = {0, n};
  if (n >= size_t(kHostChunkMinTracks) * 2) {
    const size_t big = n / kHostChunkMinTracks < 4 ? n / kHostChunkMinTracks : 4;
    const size_t first = n / 20;
    chunks = uint32_t(big) + 1;
    bound[1] = first;
    for (size_t c = 1; c <= big; ++c) bound[c + 1] = first + (n - first) * c / big;
  }
  size_t max_chunk = 0;
  for (uint32_t c = 0; c < chunks; ++c) max_chunk = bound[c + 1] - bound[c] > max_chunk ? bound[c + 1] - bound[c] : max_chunk;
  tkf::FitArgs full = make_args(geo, o, &din, &dout);
  const bool learned = o->step_mode == TKF_STEP_LEARNED;
  // one workspace per chunk (sized for the largest)
  const size_t chunk_ws = (tkf::workspace_bytes(uint32_t(max_chunk + 1), learned) + 255) & ~size_t(255);
  tkf::LaunchShape chunk_shape;
  if (chunks > 1 && chunks * chunk_ws > ctx->ws_bytes) {
    e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "tkf_fit_host: stream synchronize");
    if (ctx->ws) cudaFree(ctx->ws);
    ctx->ws = nullptr;
    ctx->ws_bytes = 0;
    e = cudaMalloc(&ctx->ws, chunks * chunk_ws);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "tkf_fit_host: workspace cudaMalloc");
    ctx->ws_bytes = chunks * chunk_ws;
  }
  // the staging buffers may still be in use by an earlier call's work (also one that stopped on
  // an error with copies in flight)
  e = cudaStreamSynchronize(st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->h2d_stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->d2h_stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->fit2_stream);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "tkf_fit_host: stream synchronize");
  auto h2d = [&](void* dst, const void* src, size_t bytes) {
    if (e == cudaSuccess && bytes) e = cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, ctx->h2d_stream);
  };
  auto d2h = [&](void* dst, const void* src, size_t bytes) {
    if (e == cudaSuccess && bytes) e = cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToHost, ctx->d2h_stream);
  };
  // `cols` consecutive doubles of each of `rows` rows of a [rows][n] matrix
  auto h2d_rows = [&](double* dst, const double* src, size_t cols, size_t rows) {
    if (e == cudaSuccess && cols)
      e = cudaMemcpy2DAsync(dst, n * 8, src, n * 8, cols * 8, rows, cudaMemcpyHostToDevice, ctx->h2d_stream);
  };
  auto d2h_rows = [&](double* dst, const double* src, size_t cols, size_t rows) {
    if (e == cudaSuccess && cols)
      e = cudaMemcpy2DAsync(dst, n * 8, src, n * 8, cols * 8, rows, cudaMemcpyDeviceToHost, ctx->d2h_stream);
  };
  // measurements copied so far: one interval [cov_lo, cov_hi), grown by every chunk, so that no
  // byte is copied twice while an earlier chunk's fit may read it
  size_t cov_lo = 0, cov_hi = 0;
  // Learned mode in chunks: the proposals of the whole batch come first, from the offsets,
  // surface ids and seed parameters copied ahead of everything else, in one pre-pass while the
  // GPU has nothing else to do; the chunks' fits then follow one another with no pre-pass
  // between them (a pre-pass could start only in the tail of the previous chunk's fit, which
  // holds every SM).
  const bool props_first = h0_all && chunks > 1;
  if (props_first) {
    h2d(const_cast<uint32_t*>(din.offsets), hin->offsets, (n + 1) * 4);
    h2d(const_cast<uint32_t*>(din.sid), hin->sid, m * 4);
    h2d(const_cast<double*>(din.seed_par), hin->seed_par, 5 * n * 8);
    if (e == cudaSuccess) e = cudaEventRecord(ctx->props_in, ctx->h2d_stream);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(st, ctx->props_in, 0);
    if (e == cudaSuccess) e = tkf::launch_propose_start(full, field->f, h0_all, st);
    if (e == cudaSuccess) e = cudaEventRecord(ctx->props_done, st);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(ctx->fit2_stream, ctx->props_done, 0);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "tkf_fit_host: proposal pre-pass");
  }
  auto h2d_meas = [&](size_t a0, size_t a1) {
    if (a1 <= a0) return;
    const size_t k = a1 - a0;
    h2d(const_cast<double*>(din.loc0) + a0, hin->loc0 + a0, k * 8);
    h2d(const_cast<double*>(din.loc1) + a0, hin->loc1 + a0, k * 8);
    h2d(const_cast<double*>(din.v00) + a0, hin->v00 + a0, k * 8);
    h2d(const_cast<double*>(din.v01) + a0, hin->v01 + a0, k * 8);
    h2d(const_cast<double*>(din.v11) + a0, hin->v11 + a0, k * 8);
    if (!props_first) h2d(const_cast<uint32_t*>(din.sid) + a0, hin->sid + a0, k * 4);
  };
  for (uint32_t c = 0; c < chunks; ++c) {
    const size_t t0 = bound[c], t1 = bound[c + 1], nt = t1 - t0;
    // the measurements the chunk's tracks can reference lie between the least and the greatest
    // of their offsets (a track whose range is reversed or beyond n_meas reads none: the kernel
    // flags it); scanned here, while the earlier chunks' copies and fits run
    size_t lo = m, hi = 0;
    for (size_t i = t0; i <= t1; ++i) {
      const size_t v = hin->offsets[i] < m ? hin->offsets[i] : m;
      lo = v < lo ? v : lo;
      hi = v > hi ? v : hi;
    }
    if (c == 0) {
      cov_lo = cov_hi = lo;
    }
    const size_t new_lo = lo < cov_lo ? lo : cov_lo, new_hi = hi > cov_hi ? hi : cov_hi;
    // offsets [t0, t1]: offsets[t0] came with the previous chunk (all of them first in learned mode)
    if (!props_first)
      h2d(const_cast<uint32_t*>(din.offsets) + t0 + (c ? 1 : 0), hin->offsets + t0 + (c ? 1 : 0),
          (nt + (c ? 0 : 1)) * 4);
    h2d_meas(new_lo, cov_lo);
    h2d_meas(cov_hi, new_hi);
    cov_lo = new_lo;
    cov_hi = new_hi;
    // the chunk's columns of the SoA seed matrices: one strided copy each
    if (!props_first) h2d_rows(const_cast<double*>(din.seed_par) + t0, hin->seed_par + t0, nt, 5);
    h2d_rows(const_cast<double*>(din.seed_cov) + t0, hin->seed_cov + t0, nt, 15);
    // chunks alternate between the caller's stream and a second compute stream, each with a
    // workspace of its own, so that a chunk's fit fills the SMs its predecessor's tail leaves
    const cudaStream_t cs = (chunks > 1 && (c & 1u)) ? ctx->fit2_stream : st;
    if (e == cudaSuccess) e = cudaEventRecord(ctx->chunk_in[c], ctx->h2d_stream);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(cs, ctx->chunk_in[c], 0);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "tkf_fit_host: host-to-device copy");
    tkf::FitArgs a = full;
    a.n_tracks = uint32_t(nt);
    a.offsets += t0;
    a.seed_par += t0;
    a.seed_cov += t0;
    a.par += t0;
    a.cov += t0;
    a.chi2 += t0;
    a.ndf += t0;
    a.status += t0;
    if (a.steps) a.steps += t0;
    if (chunks == 1) {
      s = fit_enqueue(ctx, field, o, a, st, true, "tkf_fit_host");
      if (s != TKF_OK) return s;
    } else {
      const tkf::Workspace wsc = tkf::carve_workspace(static_cast<char*>(ctx->ws) + c * chunk_ws, nt, learned);
      // each chunk its own launch shape (the small first chunk and the large ones tune apart); a
      // tuning run launches on `stream`, which therefore waits for the chunk's inputs first
      if (c > 0 && (e = cudaStreamWaitEvent(st, ctx->chunk_in[c], 0)) != cudaSuccess)
        return cuda_fail(ctx, e, "tkf_fit_host: stream wait");
      if ((e = tkf::resolve_shape(ctx, a, field->f, o->precision, wsc, o, st, &chunk_shape)) != cudaSuccess)
        return cuda_fail(ctx, e, "tkf_fit_host: autotune");
      if ((e = tkf::launch_fit(a, field->f, o->precision, wsc, chunk_shape, cs, nullptr,
                               props_first ? h0_all + t0 : nullptr)) != cudaSuccess)
        return cuda_fail(ctx, e, "tkf_fit_host: launch");
    }
    e = cudaEventRecord(ctx->chunk_fit[c], cs);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(ctx->d2h_stream, ctx->chunk_fit[c], 0);
    d2h_rows(hout->par + t0, dout.par + t0, nt, 5);
    d2h_rows(hout->cov + t0, dout.cov + t0, nt, 15);
    d2h(hout->chi2 + t0, dout.chi2 + t0, nt * 8);
    d2h(hout->ndf + t0, dout.ndf + t0, nt * 4);
    d2h(hout->status + t0, dout.status + t0, nt * 4);
    if (hout->steps && e == cudaSuccess && nt)
      e = cudaMemcpy2DAsync(hout->steps + t0, n * 4, dout.steps + t0, n * 4, nt * 4, 2, cudaMemcpyDeviceToHost,
                            ctx->d2h_stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "tkf_fit_host: device-to-host copy");
  }
  e = cudaStreamSynchronize(ctx->d2h_stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->fit2_stream);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "tkf_fit_host: stream synchronize");
  return TKF_OK;
}

}  // extern "C"

// ============================================================================ learned step proposer
extern "C" {

// A handle around device FP32 weights that hold BF16 values (takes ownership of `dev`).
static tkf_status make_mlp(tkf_context ctx, float* dev, tkf_mlp* out, const char* fn) {
  tkf_mlp h = new (std::nothrow) tkf_mlp_s();
  if (!h) {
    cudaFree(dev);
    return fail(ctx, TKF_ERR_OOM, std::string(fn) + ": host allocation failed");
  }
  h->ctx = ctx;
  h->device = ctx->device;
  h->d_weights = dev;
  *out = h;
  return TKF_OK;
}

tkf_status tkf_mlp_load(tkf_context ctx, const uint16_t* w, size_t n, tkf_mlp* out) {
  if (!ctx) return fail(nullptr, TKF_ERR_BAD_HANDLE, "tkf_mlp_load: NULL context");
  if (!w || !out) return fail(ctx, TKF_ERR_INVALID_ARG, "tkf_mlp_load: NULL pointer");
  *out = nullptr;
  if (n != TKF_MLP_PARAMS)
    return fail(ctx, TKF_ERR_INVALID_ARG, "tkf_mlp_load: expected " + std::to_string(TKF_MLP_PARAMS) +
                                              " BF16 weights, got " + std::to_string(n));
  float host[TKF_MLP_PARAMS];
  for (int k = 0; k < TKF_MLP_PARAMS; ++k) {
    const uint32_t u = uint32_t(w[k]) << 16;
    float f;
    memcpy(&f, &u, 4);
    if (!isfinite(f)) return fail(ctx, TKF_ERR_INVALID_ARG, "tkf_mlp_load: non-finite weight " + std::to_string(k));
    host[k] = f;
  }
  DeviceGuard g(ctx->device);
  float* dev = nullptr;
  cudaError_t e = cudaMalloc(&dev, sizeof(host));
  if (e != cudaSuccess) return cuda_fail(ctx, e, "tkf_mlp_load: cudaMalloc");
  e = cudaMemcpy(dev, host, sizeof(host), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) {
    cudaFree(dev);
    return cuda_fail(ctx, e, "tkf_mlp_load: cudaMemcpy");
  }
  return make_mlp(ctx, dev, out, "tkf_mlp_load");
}

tkf_status tkf_mlp_load_f32(tkf_context ctx, const float* params, size_t n, tkf_mlp* out, void* stream) {
  if (!ctx) return fail(nullptr, TKF_ERR_BAD_HANDLE, "tkf_mlp_load_f32: NULL context");
  if (!params || !out) return fail(ctx, TKF_ERR_INVALID_ARG, "tkf_mlp_load_f32: NULL pointer");
  *out = nullptr;
  if (n != TKF_MLP_PARAMS)
    return fail(ctx, TKF_ERR_INVALID_ARG, "tkf_mlp_load_f32: expected " + std::to_string(TKF_MLP_PARAMS) +
                                              " FP32 parameters, got " + std::to_string(n));
  DeviceGuard g(ctx->device);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  float* dev = nullptr;
  cudaError_t e = cudaMalloc(&dev, sizeof(float) * TKF_MLP_PARAMS + 16);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "tkf_mlp_load_f32: cudaMalloc");
  uint32_t* bad = reinterpret_cast<uint32_t*>(dev + TKF_MLP_PARAMS);
  uint32_t bad_h = 0;
  e = cudaMemsetAsync(bad, 0, sizeof(uint32_t), st);
  if (e == cudaSuccess) e = tkf::mlp_round_bf16(params, dev, bad, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&bad_h, bad, sizeof(uint32_t), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) {
    cudaFree(dev);
    return cuda_fail(ctx, e, "tkf_mlp_load_f32: rounding");
  }
  if (bad_h) {
    cudaFree(dev);
    return fail(ctx, TKF_ERR_INVALID_ARG, "tkf_mlp_load_f32: non-finite parameter");
  }
  return make_mlp(ctx, dev, out, "tkf_mlp_load_f32");
}

tkf_status tkf_mlp_init(tkf_context ctx, float* params, size_t n, uint64_t seed, void* stream) {
  if (!ctx) return fail(nullptr, TKF_ERR_BAD_HANDLE, "tkf_mlp_init: NULL context");
  if (!params) return fail(ctx, TKF_ERR_INVALID_ARG, "tkf_mlp_init: NULL pointer");
  if (n != TKF_MLP_PARAMS)
    return fail(ctx, TKF_ERR_INVALID_ARG, "tkf_mlp_init: expected " + std::to_string(TKF_MLP_PARAMS) + " parameters");
  DeviceGuard g(ctx->device);
  cudaError_t e = tkf::mlp_init(params, seed, static_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return cuda_fail(ctx, e, "tkf_mlp_init: launch");
  return TKF_OK;
}

tkf_status tkf_mlp_calibrate(tkf_context ctx, float* params, const float* records, uint32_t n, double quantile,
                             double* shift, void* stream) {
  if (!ctx) return fail(nullptr, TKF_ERR_BAD_HANDLE, "tkf_mlp_calibrate: NULL context");
  if (!params || !records || !shift) return fail(ctx, TKF_ERR_INVALID_ARG, "tkf_mlp_calibrate: NULL pointer");
  if (n == 0 || !(quantile >= 0.0 && quantile <= 1.0))
    return fail(ctx, TKF_ERR_INVALID_ARG, "tkf_mlp_calibrate: need n > 0 and 0 <= quantile <= 1");
  DeviceGuard g(ctx->device);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const size_t need = tkf::mlp_calibrate_scratch_bytes(n) + 64;  // the shift, then the scratch
  if (need > ctx->train_bytes) {
    cudaError_t e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "tkf_mlp_calibrate: scratch");
    if (ctx->train_ws) cudaFree(ctx->train_ws);
    ctx->train_ws = nullptr;
    ctx->train_bytes = 0;
    e = cudaMalloc(&ctx->train_ws, need);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "tkf_mlp_calibrate: scratch");
    ctx->train_bytes = need;
  }
  double* d_shift = reinterpret_cast<double*>(ctx->train_ws);
  void* scratch = static_cast<char*>(ctx->train_ws) + 64;
  cudaError_t e = tkf::mlp_calibrate(params, records, n, quantile, d_shift, scratch, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(shift, d_shift, sizeof(double), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "tkf_mlp_calibrate: launch");
  return TKF_OK;
}

void tkf_mlp_destroy(tkf_mlp m) {
  if (!m) return;
  DeviceGuard g(m->device);
  cudaFree(m->d_weights);
  delete m;
}

static tkf_status train_scratch(tkf_context ctx, uint32_t batch, void** out, cudaStream_t stream, const char* fn) {
  const size_t need = tkf::mlp_train_scratch_bytes(batch);
  if (need > ctx->train_bytes) {
    cudaError_t e = cudaStreamSynchronize(stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, fn);
    if (ctx->train_ws) cudaFree(ctx->train_ws);
    ctx->train_ws = nullptr;
    ctx->train_bytes = 0;
    e = cudaMalloc(&ctx->train_ws, need);
    if (e != cudaSuccess) return cuda_fail(ctx, e, fn);
    ctx->train_bytes = need;
  }
  *out = ctx->train_ws;
  return TKF_OK;
}

tkf_status tkf_mlp_train(tkf_context ctx, const float* records, uint32_t n, const tkf_mlp_train_options* o,
                         float* params, float* moments, uint32_t* adam_t, float* epoch_loss, void* stream) {
  if (!ctx) return fail(nullptr, TKF_ERR_BAD_HANDLE, "tkf_mlp_train: NULL context");
  if (!records || !o || !params || !moments || !adam_t || !epoch_loss)
    return fail(ctx, TKF_ERR_INVALID_ARG, "tkf_mlp_train: NULL pointer");
  if (o->batch == 0 || o->batch > 8192 || o->batch > n || o->epochs == 0 || !(o->lr > 0) || !(o->beta1 >= 0) ||
      !(o->beta1 < 1) || !(o->beta2 >= 0) || !(o->beta2 < 1) || !(o->eps > 0))
    return fail(ctx, TKF_ERR_INVALID_ARG,
                "tkf_mlp_train: need 1 <= batch <= min(8192, n), epochs > 0, lr > 0, 0 <= beta < 1, eps > 0");
  DeviceGuard g(ctx->device);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  void* scratch = nullptr;
  tkf_status s = train_scratch(ctx, o->batch, &scratch, st, "tkf_mlp_train: scratch");
  if (s != TKF_OK) return s;
  cudaError_t e = tkf::mlp_train(records, n, o->batch, o->epochs, o->lr, o->beta1, o->beta2, o->eps, params, moments,
                                 adam_t, epoch_loss, scratch, st);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "tkf_mlp_train: launch");
  return TKF_OK;
}

tkf_status tkf_mlp_loss_grad(tkf_context ctx, const float* params, const float* x, const float* y, uint32_t n,
                             float* grad, float* loss, void* stream) {
  if (!ctx) return fail(nullptr, TKF_ERR_BAD_HANDLE, "tkf_mlp_loss_grad: NULL context");
  if (!params || !x || !y || !grad || !loss || n == 0 || n > 65536)
    return fail(ctx, TKF_ERR_INVALID_ARG, "tkf_mlp_loss_grad: NULL pointer, or n not in 1..65536");
  DeviceGuard g(ctx->device);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  void* scratch = nullptr;
  tkf_status s = train_scratch(ctx, n, &scratch, st, "tkf_mlp_loss_grad: scratch");
  if (s != TKF_OK) return s;
  cudaError_t e = tkf::mlp_loss_grad(params, x, TKF_MLP_INPUTS, y, 1, n, grad, loss, scratch, st);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "tkf_mlp_loss_grad: launch");
  return TKF_OK;
}

tkf_status tkf_mlp_forward(tkf_context ctx, const float* params, const float* x, uint32_t n, float* out,
                           void* stream) {
  if (!ctx) return fail(nullptr, TKF_ERR_BAD_HANDLE, "tkf_mlp_forward: NULL context");
  if (!params || !x || !out) return fail(ctx, TKF_ERR_INVALID_ARG, "tkf_mlp_forward: NULL pointer");
  if (n == 0) return TKF_OK;
  DeviceGuard g(ctx->device);
  cudaError_t e = tkf::mlp_forward(params, x, n, out, static_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return cuda_fail(ctx, e, "tkf_mlp_forward: launch");
  return TKF_OK;
}

}  // extern "C"

// ============================================================================ allocation-free fit
// Some callers cannot allocate device memory once they are running: an online trigger or
// reconstruction process that reserves all of its GPU memory at start-up and forbids later
// allocations (their latency and fragmentation are not allowed on the event path), or a host
// framework whose own pool allocator owns the whole device. tkf_fit_noalloc serves them: its
// scratch (work counter, key histogram, sort keys, track permutation) is this file-scope
// array, which every GPU that loads the library holds until the process exits.

namespace {

constexpr uint32_t kNoallocMaxTracks = TKF_NOALLOC_MAX_TRACKS;
constexpr size_t kNoallocWords = 1 + 1024 + 2 * size_t(kNoallocMaxTracks) + 64;

static __device__ __align__(256) uint32_t g_noalloc_scratch[kNoallocWords];

// Looked up by tkf_context_create, with the context's device current, and kept in the context
// (a context is tied to one device; a new context after a device reset looks it up again).
cudaError_t noalloc_scratch_address(void** out) { return cudaGetSymbolAddress(out, g_noalloc_scratch); }

}  // namespace

extern "C" tkf_status tkf_fit_noalloc(tkf_context ctx, tkf_geometry geo, tkf_field field, const tkf_fit_options* o,
                                      const tkf_fit_inputs* in, const tkf_fit_outputs* out, void* stream) {
  tkf_status s = check_common(ctx, geo, field, o, in, out, "tkf_fit_noalloc");
  if (s == TKF_OK && out->states_par)
    return fail(ctx, TKF_ERR_UNSUPPORTED, "tkf_fit_noalloc: the all-states output needs workspace; use tkf_fit");
  if (s != TKF_OK || in->n_tracks == 0) return s;
  if (in->n_tracks > kNoallocMaxTracks)
    return fail(ctx, TKF_ERR_INVALID_ARG,
                "tkf_fit_noalloc: n_tracks " + std::to_string(in->n_tracks) + " exceeds the maximum " +
                    std::to_string(kNoallocMaxTracks) + " of the static scratch; use tkf_fit or split the batch");
  if (o->step_mode == TKF_STEP_LEARNED)
    return fail(ctx, TKF_ERR_UNSUPPORTED,
                "tkf_fit_noalloc: learned step mode needs a per-track starting step, for which the static "
                "scratch has no room; use tkf_fit");
  if (!ctx->noalloc_scratch)
    return fail(ctx, TKF_ERR_DEVICE, "tkf_fit_noalloc: the static scratch's device address was not found when "
                                     "the context was created");
  DeviceGuard g(ctx->device);
  if (!g.ok) return fail(ctx, TKF_ERR_DEVICE, "tkf_fit_noalloc: cudaSetDevice failed");
  tkf::FitArgs a = make_args(geo, o, in, out);
  // the launch clears the counter and histogram before use (the array keeps the last call's data)
  tkf::Workspace ws = tkf::carve_workspace(ctx->noalloc_scratch, in->n_tracks, false);
  // the launch shape of tkf_fit for these options, without tuning (tuning and graphs allocate)
  tkf_fit_options untuned = *o;
  untuned.flags &= ~uint32_t(TKF_FIT_AUTOTUNE);
  tkf::LaunchShape shape;
  cudaError_t e = tkf::resolve_shape(ctx, a, field->f, o->precision, ws, &untuned, static_cast<cudaStream_t>(stream),
                                     &shape);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "tkf_fit_noalloc: launch shape");
  e = tkf::launch_fit(a, field->f, o->precision, ws, shape, static_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return cuda_fail(ctx, e, "tkf_fit_noalloc: launch");
  return TKF_OK;
}
