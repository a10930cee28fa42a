// tkf_order.cu -- track ordering for the fit (counting sort into a permutation) and the launch
// sequence: ordering kernels, then the persistent fit of the requested precision and mode.

#include "tkf_internal.cuh"

namespace tkf {
namespace {

// ------------------------------------------------------------------ track ordering
// Counting sort of the tracks by key = (most measurements first, then lowest seed pT first,
// then |cos theta|): warps then hold tracks with the same number of measurements, similar step
// counts and similar distances between surfaces (barrel or endcap), and the work queue hands
// out the longest tracks first.
constexpr int kPtBins = 8;
constexpr int kNBins = 32;
constexpr int kEtaBins = 4;
constexpr int kKeyBins = kPtBins * kNBins * kEtaBins;

__global__ void __launch_bounds__(256) order_keys_kernel(const uint32_t* __restrict__ offsets,
                                                         const double* __restrict__ seed_par, uint32_t n,
                                                         uint32_t stride, uint32_t* __restrict__ keys,
                                                         uint32_t* __restrict__ hist) {
  __shared__ uint32_t h[kKeyBins];
  for (int b = threadIdx.x; b < kKeyBins; b += blockDim.x) h[b] = 0;
  __syncthreads();
  // each block takes one contiguous range of the tracks (one histogram flush a block)
  const uint32_t per = (n + gridDim.x - 1) / gridDim.x;
  const uint32_t r0 = blockIdx.x * per, r1 = min(n, r0 + per);
  for (uint32_t i = r0 + threadIdx.x; i < r1; i += blockDim.x) {
    const uint32_t b0 = offsets[i], b1 = offsets[i + 1];
    const uint32_t nh = b1 >= b0 ? min(b1 - b0, uint32_t(kNBins - 1)) : 0u;
    const float qop = float(seed_par[size_t(4) * stride + i]);
    const float th = float(seed_par[size_t(3) * stride + i]);
    const float sth = fabsf(sinf(th));
    const float pt = (qop != 0.0f) ? sth / fabsf(qop) : 1e30f;
    int pb = (pt > 0.0f) ? int(floorf(log2f(pt))) + 2 : 0;  // octaves from 1/4 GeV
    pb = pb < 0 ? 0 : (pb >= kPtBins ? kPtBins - 1 : pb);
    const float ac = fabsf(cosf(th)) * float(kEtaBins);
    const int eb = ac >= 0.0f && ac < float(kEtaBins) ? int(ac) : kEtaBins - 1;  // NaN: last bin
    const uint32_t key = ((uint32_t(kNBins - 1) - nh) * kPtBins + uint32_t(pb)) * kEtaBins + uint32_t(eb);
    keys[i] = key;
    atomicAdd(&h[key], 1u);
  }
  __syncthreads();
  for (int b = threadIdx.x; b < kKeyBins; b += blockDim.x)
    if (h[b]) atomicAdd(&hist[b], h[b]);
}

// exclusive scan of the kKeyBins histogram in place (one block of kKeyBins threads)
__global__ void __launch_bounds__(kKeyBins) order_scan_kernel(uint32_t* __restrict__ hist) {
  __shared__ uint32_t v[kKeyBins];
  const int t = threadIdx.x;
  v[t] = hist[t];
  __syncthreads();
  for (int off = 1; off < kKeyBins; off <<= 1) {
    const uint32_t x = t >= off ? v[t - off] : 0u;
    __syncthreads();
    v[t] += x;
    __syncthreads();
  }
  hist[t] = v[t] - hist[t];
}

// Scatter in two levels: each block takes one contiguous range of the tracks, counts its keys in
// shared memory, reserves its range of every key with one global atomic (the per-track global
// atomics contended on the few most common keys), then places its tracks within those ranges.
// Tracks of a key land in block order of arrival; the fit of a track does not depend on its place.
__global__ void __launch_bounds__(256) order_scatter_kernel(const uint32_t* __restrict__ keys, uint32_t n,
                                                            uint32_t* __restrict__ base, uint32_t* __restrict__ perm) {
  __shared__ uint32_t cnt[kKeyBins];
  __shared__ uint32_t off[kKeyBins];
  for (int b = threadIdx.x; b < kKeyBins; b += blockDim.x) cnt[b] = 0;
  __syncthreads();
  const uint32_t per = (n + gridDim.x - 1) / gridDim.x;
  const uint32_t r0 = blockIdx.x * per, r1 = min(n, r0 + per);
  for (uint32_t i = r0 + threadIdx.x; i < r1; i += blockDim.x) atomicAdd(&cnt[keys[i]], 1u);
  __syncthreads();
  for (int b = threadIdx.x; b < kKeyBins; b += blockDim.x) {
    if (cnt[b]) off[b] = atomicAdd(&base[b], cnt[b]);
    cnt[b] = 0;  // from here on: the next free rank of the key within the block's range
  }
  __syncthreads();
  for (uint32_t i = r0 + threadIdx.x; i < r1; i += blockDim.x) {
    const uint32_t key = keys[i];
    perm[off[key] + atomicAdd(&cnt[key], 1u)] = i;
  }
}

}  // namespace

namespace {
// bytes of the ordering scratch (and the learned mode's starting steps), rounded up to 256
size_t order_bytes(uint32_t n_tracks, bool learned) {
  const size_t b = 256 + sizeof(uint32_t) * (kKeyBins + (learned ? 3 : 2) * size_t(n_tracks)) + 256;
  return (b + 255) / 256 * 256;
}
}  // namespace

size_t workspace_bytes(uint32_t n_tracks, bool learned, uint64_t states_entries) {
  return order_bytes(n_tracks, learned) + sizeof(double) * kStatesScratch * size_t(states_entries);
}

Workspace carve_workspace(void* base, uint32_t n_tracks, bool learned, uint64_t states_entries) {
  Workspace w;
  uint32_t* p = static_cast<uint32_t*>(base);
  w.counter = p;          // 1 word, followed directly by the histogram (one memset clears both)
  w.hist = p + 1;
  w.keys = p + 1 + kKeyBins;
  w.perm = w.keys + n_tracks;
  if (learned) w.h0 = reinterpret_cast<float*>(w.perm + n_tracks);
  if (states_entries)
    w.states = reinterpret_cast<double*>(static_cast<char*>(base) + order_bytes(n_tracks, learned));
  return w;
}

cudaError_t launch_fit(const FitArgs& a, const FieldDev& f, int precision, const Workspace& ws, LaunchShape shape,
                       cudaStream_t stream, const cudaEvent_t* timing, const float* h0_given) {
  if (a.n_tracks == 0) return cudaSuccess;
  const uint32_t n = a.n_tracks;
  cudaError_t e = cudaMemsetAsync(ws.counter, 0, sizeof(uint32_t) * (1 + kKeyBins), stream);
  if (e != cudaSuccess) return e;
  // at most 1,216 blocks (8 an SM on GB300), each over one contiguous range of the tracks
  const unsigned g256 = (n + 255) / 256 < 1216u ? (n + 255) / 256 : 1216u;
  order_keys_kernel<<<g256, 256, 0, stream>>>(a.offsets, a.seed_par, n, a.stride, ws.keys, ws.hist);
  order_scan_kernel<<<1, kKeyBins, 0, stream>>>(ws.hist);
  order_scatter_kernel<<<g256, 256, 0, stream>>>(ws.keys, n, ws.hist, ws.perm);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  // learned, record capture, all-states output, or plain
  const int mode = a.mlp ? 1 : (a.records ? 2 : (a.states_par ? 3 : 0));
  FitArgs b = a;
  if (mode == 3) {
    if (!ws.states) return cudaErrorInvalidValue;
    b.states_scratch = ws.states;
  }
  if (mode == 1 && h0_given) {  // proposals already made for these tracks
    b.h0 = h0_given;
  } else if (mode == 1) {  // network proposals of each track's starting step size
    if (!ws.h0) return cudaErrorInvalidValue;
    e = launch_propose_start(a, f, ws.h0, stream);
    if (e != cudaSuccess) return e;
    b.h0 = ws.h0;
  }
  if (timing && (e = cudaEventRecord(timing[0], stream)) != cudaSuccess) return e;
  e = a.smoother == TKF_SMOOTHER_TWO_FILTER
          ? launch_fit_two_filter(b, f, precision, mode, ws.perm, ws.counter, shape, stream)
      : shape.group == 4            ? launch_fit_group(b, f, precision, mode, ws.perm, ws.counter, shape, stream)
      : precision == TKF_MIXED      ? launch_fit_mixed(b, f, mode, ws.perm, ws.counter, shape, stream)
      : precision == TKF_MIXED_FP32 ? launch_fit_mixed32(b, f, mode, ws.perm, ws.counter, shape, stream)
                                    : launch_fit_fp64(b, f, mode, ws.perm, ws.counter, shape, stream);
  if (e != cudaSuccess) return e;
  if (timing && (e = cudaEventRecord(timing[1], stream)) != cudaSuccess) return e;
  if (mode == 3) e = launch_smooth_states(b, ws.perm, stream);  // backward RTS over the stored states
  return e;
}

}  // namespace tkf
