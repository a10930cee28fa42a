// tkf_mlp.cu -- training and inference kernels of the learned step proposer (FP32).
//
// Network: 12 inputs -> 64 SiLU -> 64 SiLU -> 1, parameters packed as W1 [64][12], b1 [64],
// W2 [64][64], b2 [64], w3 [64], b3. Loss: mean squared error. Optimiser: Adam
// (Kingma & Ba 2015). One training step on a batch of B samples is four launches:
//   forward   (one thread per sample; activations kept for the backward pass),
//   backward  (one thread per sample; dL/dz of both hidden layers and of the output),
//   reduce    (one thread per parameter; sums over the batch, no atomics: deterministic),
//   adam      (one thread per parameter).
// Around training: seeded initialisation, calibration of the output bias (a quantile of the
// training residuals, by a radix select on the device) and rounding to the BF16 weights the
// fit's inference uses.
// The paper has no learned component; the learned step proposer is an addition to its method.

#include <math.h>

#include "tkf_internal.cuh"

namespace tkf {
namespace {

constexpr int kIn = 12, kHid = 64;
constexpr int oW1 = 0, oB1 = 768, oW2 = 832, oB2 = 4928, oW3 = 4992, oB3 = 5056;

__device__ __forceinline__ float sigm(float z) { return 1.0f / (1.0f + expf(-z)); }

// Per-sample activations: z1, a1, z2, a2 (4 x 64 floats), then out.
struct Act {
  float* z1;
  float* a1;
  float* z2;
  float* a2;
  float* out;
  float* dz1;
  float* dz2;
  float* dout;
};

__global__ void __launch_bounds__(128) mlp_forward_kernel(const float* __restrict__ p, const float* __restrict__ x,
                                                          int x_stride, uint32_t n, Act act) {
  __shared__ float w[kMlpParams];
  for (int k = threadIdx.x; k < kMlpParams; k += blockDim.x) w[k] = p[k];
  __syncthreads();
  const uint32_t s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= n) return;
  float in[kIn];
  for (int i = 0; i < kIn; ++i) in[i] = x[size_t(s) * x_stride + i];
  float a1[kHid];
  for (int j = 0; j < kHid; ++j) {
    float z = w[oB1 + j];
    for (int i = 0; i < kIn; ++i) z = fmaf(w[oW1 + j * kIn + i], in[i], z);
    const float a = z * sigm(z);
    a1[j] = a;
    if (act.z1) {
      act.z1[size_t(s) * kHid + j] = z;
      act.a1[size_t(s) * kHid + j] = a;
    }
  }
  float out = w[oB3];
  for (int j = 0; j < kHid; ++j) {
    float z = w[oB2 + j];
    for (int i = 0; i < kHid; ++i) z = fmaf(w[oW2 + j * kHid + i], a1[i], z);
    const float a = z * sigm(z);
    if (act.z2) {
      act.z2[size_t(s) * kHid + j] = z;
      act.a2[size_t(s) * kHid + j] = a;
    }
    out = fmaf(w[oW3 + j], a, out);
  }
  act.out[s] = out;
}

// dL/dout = 2 (out - y) / B; dz2 = dout w3 silu'(z2); dz1 = (W2^T dz2) silu'(z1). The squared
// residual of each sample goes to sq[s] for the loss.
__global__ void __launch_bounds__(128) mlp_backward_kernel(const float* __restrict__ p, const float* __restrict__ y,
                                                           int y_stride, uint32_t n, Act act, float* __restrict__ sq) {
  __shared__ float w[kMlpParams];
  for (int k = threadIdx.x; k < kMlpParams; k += blockDim.x) w[k] = p[k];
  __syncthreads();
  const uint32_t s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= n) return;
  const float r = act.out[s] - y[size_t(s) * y_stride];
  sq[s] = r * r;
  const float dout = 2.0f * r / float(n);
  act.dout[s] = dout;
  float dz2[kHid];
  for (int j = 0; j < kHid; ++j) {
    const float z = act.z2[size_t(s) * kHid + j];
    const float sg = sigm(z);
    dz2[j] = dout * w[oW3 + j] * sg * (1.0f + z * (1.0f - sg));
    act.dz2[size_t(s) * kHid + j] = dz2[j];
  }
  for (int i = 0; i < kHid; ++i) {
    float da = 0.0f;
    for (int j = 0; j < kHid; ++j) da = fmaf(w[oW2 + j * kHid + i], dz2[j], da);
    const float z = act.z1[size_t(s) * kHid + i];
    const float sg = sigm(z);
    act.dz1[size_t(s) * kHid + i] = da * sg * (1.0f + z * (1.0f - sg));
  }
}

// Gradient of every parameter: a sum over the batch of (output gradient x input activation).
__global__ void __launch_bounds__(256) mlp_reduce_kernel(const float* __restrict__ x, int x_stride, uint32_t n,
                                                         Act act, float* __restrict__ grad) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= kMlpParams) return;
  float g = 0.0f;
  if (k < oB1) {
    const int j = k / kIn, i = k % kIn;
    for (uint32_t s = 0; s < n; ++s) g = fmaf(act.dz1[size_t(s) * kHid + j], x[size_t(s) * x_stride + i], g);
  } else if (k < oW2) {
    const int j = k - oB1;
    for (uint32_t s = 0; s < n; ++s) g += act.dz1[size_t(s) * kHid + j];
  } else if (k < oB2) {
    const int j = (k - oW2) / kHid, i = (k - oW2) % kHid;
    for (uint32_t s = 0; s < n; ++s) g = fmaf(act.dz2[size_t(s) * kHid + j], act.a1[size_t(s) * kHid + i], g);
  } else if (k < oW3) {
    const int j = k - oB2;
    for (uint32_t s = 0; s < n; ++s) g += act.dz2[size_t(s) * kHid + j];
  } else if (k < oB3) {
    const int i = k - oW3;
    for (uint32_t s = 0; s < n; ++s) g = fmaf(act.dout[s], act.a2[size_t(s) * kHid + i], g);
  } else {
    for (uint32_t s = 0; s < n; ++s) g += act.dout[s];
  }
  grad[k] = g;
}

// Sum of the per-sample squared residuals / n (one block), written to *loss, and, if epoch_acc is
// not null, added to it with weight 1 / n_batches.
__global__ void __launch_bounds__(256) mlp_loss_kernel(const float* __restrict__ sq, uint32_t n, float* __restrict__ loss,
                                                       float* __restrict__ epoch_acc, float inv_batches) {
  __shared__ float part[256];
  float acc = 0.0f;
  for (uint32_t s = threadIdx.x; s < n; s += blockDim.x) acc += sq[s];
  part[threadIdx.x] = acc;
  __syncthreads();
  for (int off = 128; off > 0; off >>= 1) {
    if (threadIdx.x < off) part[threadIdx.x] += part[threadIdx.x + off];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    const float l = part[0] / float(n);
    if (loss) *loss = l;
    if (epoch_acc) *epoch_acc += l * inv_batches;
  }
}

__global__ void __launch_bounds__(256) mlp_adam_kernel(float* __restrict__ p, const float* __restrict__ g,
                                                       float* __restrict__ m, float* __restrict__ v, float lr,
                                                       float beta1, float beta2, float eps, float c1, float c2) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= kMlpParams) return;
  const float gk = g[k];
  const float mk = beta1 * m[k] + (1.0f - beta1) * gk;
  const float vk = beta2 * v[k] + (1.0f - beta2) * gk * gk;
  m[k] = mk;
  v[k] = vk;
  p[k] -= lr * (mk / c1) / (sqrtf(vk / c2) + eps);
}

struct Scratch {
  Act act;
  float* sq;
  float* grad;
};

Scratch carve(void* base, uint32_t batch) {
  float* f = static_cast<float*>(base);
  Scratch s;
  const size_t h = size_t(batch) * kHid;
  s.act.z1 = f;
  s.act.a1 = f + h;
  s.act.z2 = f + 2 * h;
  s.act.a2 = f + 3 * h;
  s.act.dz1 = f + 4 * h;
  s.act.dz2 = f + 5 * h;
  s.act.out = f + 6 * h;
  s.act.dout = s.act.out + batch;
  s.sq = s.act.dout + batch;
  s.grad = s.sq + batch;
  return s;
}

cudaError_t batch_grad(const float* params, const float* x, int x_stride, const float* y, int y_stride, uint32_t n,
                       const Scratch& sc, float* grad, float* loss, float* epoch_acc, float inv_batches,
                       cudaStream_t stream) {
  const unsigned gs = (n + 127) / 128;
  mlp_forward_kernel<<<gs, 128, 0, stream>>>(params, x, x_stride, n, sc.act);
  mlp_backward_kernel<<<gs, 128, 0, stream>>>(params, y, y_stride, n, sc.act, sc.sq);
  mlp_reduce_kernel<<<(kMlpParams + 255) / 256, 256, 0, stream>>>(x, x_stride, n, sc.act, grad);
  mlp_loss_kernel<<<1, 256, 0, stream>>>(sc.sq, n, loss, epoch_acc, inv_batches);
  return cudaGetLastError();
}

// ---- initialisation: W ~ U(-1/sqrt(fan_in), 1/sqrt(fan_in)) from SplitMix64 of (seed, index), b = 0
__device__ __forceinline__ uint64_t splitmix64(uint64_t x) {
  x += 0x9E3779B97F4A7C15ull;
  x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
  x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
  return x ^ (x >> 31);
}

__global__ void __launch_bounds__(256) mlp_init_kernel(float* __restrict__ p, uint64_t seed) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= kMlpParams) return;
  const bool weight = k < oB1 || (k >= oW2 && k < oB2) || (k >= oW3 && k < oB3);
  if (!weight) {
    p[k] = 0.0f;
    return;
  }
  const float fan_in = k < oB1 ? float(kIn) : float(kHid);
  const uint64_t r = splitmix64(seed * 0x100000001B3ull + uint64_t(k));
  const float u = float(r >> 40) * (1.0f / 16777216.0f);  // [0, 1), 24 bits
  p[k] = (2.0f * u - 1.0f) * rsqrtf(fan_in);
}

// ---- calibration: residual = label - output, shifted bias b3 += quantile of the residuals
// order-preserving map of an FP32 value to an unsigned key, and back
__device__ __forceinline__ uint32_t order_key(float f) {
  const uint32_t u = __float_as_uint(f);
  return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}
__device__ __forceinline__ float from_order_key(uint32_t k) {
  return __uint_as_float((k & 0x80000000u) ? (k & 0x7fffffffu) : ~k);
}

__global__ void __launch_bounds__(256) residual_keys_kernel(const float* __restrict__ rec, uint32_t n,
                                                            const float* __restrict__ out, uint32_t* __restrict__ keys) {
  const uint32_t s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s < n) keys[s] = order_key(rec[size_t(s) * kMlpRecord + 12] - out[s]);
}

// The k0-th and k1-th smallest keys (0-based) by a radix select, 8 bits a pass from the top:
// each pass counts the keys that share the digits chosen so far by their next digit and keeps
// the bucket that holds the wanted rank. One block; every loop is bounded by n or 256.
__global__ void __launch_bounds__(1024) select_kernel(const uint32_t* __restrict__ keys, uint32_t n, uint32_t k0,
                                                      uint32_t k1, uint32_t* __restrict__ sel) {
  __shared__ uint32_t hist[256];
  __shared__ uint32_t s_prefix, s_rank;
  for (int which = 0; which < 2; ++which) {
    uint32_t prefix = 0, mask = 0, rank = which ? k1 : k0;
    for (int pass = 0; pass < 4; ++pass) {
      const int shift = 24 - 8 * pass;
      for (int b = threadIdx.x; b < 256; b += blockDim.x) hist[b] = 0;
      __syncthreads();
      for (uint32_t i = threadIdx.x; i < n; i += blockDim.x) {
        const uint32_t key = keys[i];
        if ((key & mask) == prefix) atomicAdd(&hist[(key >> shift) & 255u], 1u);
      }
      __syncthreads();
      if (threadIdx.x == 0) {
        uint32_t acc = 0;
        int d = 0;
        for (; d < 255; ++d) {
          if (acc + hist[d] > rank) break;
          acc += hist[d];
        }
        s_prefix = prefix | (uint32_t(d) << shift);
        s_rank = rank - acc;
      }
      __syncthreads();
      prefix = s_prefix;
      rank = s_rank;
      mask |= 255u << shift;
      __syncthreads();
    }
    if (threadIdx.x == 0) sel[which] = prefix;
    __syncthreads();
  }
}

// The quantile by linear interpolation between the two order statistics around
// position q (n - 1) (FP64), added to the output bias (FP64, rounded to FP32).
__global__ void shift_bias_kernel(float* __restrict__ p, const uint32_t* __restrict__ sel, double frac,
                                  double* __restrict__ shift) {
  const double v0 = from_order_key(sel[0]), v1 = from_order_key(sel[1]);
  const double q = v0 + frac * (v1 - v0);
  p[oB3] = float(double(p[oB3]) + q);
  *shift = q;
}

// ---- BF16 weights: round to nearest even; a non-finite value sets *bad
__global__ void __launch_bounds__(256) round_bf16_kernel(const float* __restrict__ in, float* __restrict__ out,
                                                         uint32_t* __restrict__ bad) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= kMlpParams) return;
  const float x = in[k];
  if (!isfinite(x)) atomicOr(bad, 1u);
  const uint32_t u = __float_as_uint(x);
  out[k] = __uint_as_float((u + 0x7FFFu + ((u >> 16) & 1u)) & 0xFFFF0000u);
}

}  // namespace

cudaError_t mlp_init(float* params, uint64_t seed, cudaStream_t stream) {
  mlp_init_kernel<<<(kMlpParams + 255) / 256, 256, 0, stream>>>(params, seed);
  return cudaGetLastError();
}

size_t mlp_calibrate_scratch_bytes(uint32_t n) { return sizeof(float) * 2 * size_t(n) + 64; }

cudaError_t mlp_calibrate(float* params, const float* records, uint32_t n, double quantile, double* shift,
                          void* scratch, cudaStream_t stream) {
  float* out = static_cast<float*>(scratch);
  uint32_t* keys = reinterpret_cast<uint32_t*>(out + n);
  uint32_t* sel = keys + n;
  Act act{};
  act.out = out;
  const unsigned g = (n + 255) / 256;
  mlp_forward_kernel<<<(n + 127) / 128, 128, 0, stream>>>(params, records, kMlpRecord, n, act);
  residual_keys_kernel<<<g, 256, 0, stream>>>(records, n, out, keys);
  const double pos = quantile * double(n - 1);
  const uint32_t k0 = uint32_t(floor(pos));
  const uint32_t k1 = k0 + 1 < n ? k0 + 1 : k0;
  select_kernel<<<1, 1024, 0, stream>>>(keys, n, k0, k1, sel);
  shift_bias_kernel<<<1, 1, 0, stream>>>(params, sel, pos - double(k0), shift);
  return cudaGetLastError();
}

cudaError_t mlp_round_bf16(const float* in, float* out, uint32_t* bad, cudaStream_t stream) {
  round_bf16_kernel<<<(kMlpParams + 255) / 256, 256, 0, stream>>>(in, out, bad);
  return cudaGetLastError();
}

size_t mlp_train_scratch_bytes(uint32_t batch) {
  return sizeof(float) * (size_t(batch) * (6 * kHid + 3) + kMlpParams) + 256;
}

cudaError_t mlp_loss_grad(const float* params, const float* x, int x_stride, const float* y, int y_stride,
                          uint32_t n, float* grad, float* loss, void* scratch, cudaStream_t stream) {
  Scratch sc = carve(scratch, n);
  return batch_grad(params, x, x_stride, y, y_stride, n, sc, grad, loss, nullptr, 0.0f, stream);
}

cudaError_t mlp_train(const float* records, uint32_t n, uint32_t batch, uint32_t epochs, float lr, float beta1,
                      float beta2, float eps, float* params, float* moments, uint32_t* adam_t, float* epoch_loss,
                      void* scratch, cudaStream_t stream) {
  Scratch sc = carve(scratch, batch);
  const uint32_t nb = n / batch;
  cudaError_t e = cudaMemsetAsync(epoch_loss, 0, sizeof(float) * epochs, stream);
  if (e != cudaSuccess) return e;
  for (uint32_t ep = 0; ep < epochs; ++ep) {
    for (uint32_t b = 0; b < nb; ++b) {
      const float* rec = records + size_t(b) * batch * kMlpRecord;
      e = batch_grad(params, rec, kMlpRecord, rec + 12, kMlpRecord, batch, sc, sc.grad, nullptr, epoch_loss + ep,
                     1.0f / float(nb), stream);
      if (e != cudaSuccess) return e;
      const uint32_t t = ++(*adam_t);
      const float c1 = 1.0f - powf(beta1, float(t)), c2 = 1.0f - powf(beta2, float(t));
      mlp_adam_kernel<<<(kMlpParams + 255) / 256, 256, 0, stream>>>(params, sc.grad, moments, moments + kMlpParams,
                                                                     lr, beta1, beta2, eps, c1, c2);
      e = cudaGetLastError();
      if (e != cudaSuccess) return e;
    }
  }
  return cudaSuccess;
}

cudaError_t mlp_forward(const float* params, const float* x, uint32_t n, float* out, cudaStream_t stream) {
  Act act{};
  act.out = out;
  mlp_forward_kernel<<<(n + 127) / 128, 128, 0, stream>>>(params, x, kIn, n, act);
  return cudaGetLastError();
}

}  // namespace tkf
