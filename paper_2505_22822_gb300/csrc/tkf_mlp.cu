// tkf_mlp.cu -- training and inference kernels of the learned step proposer (FP32).
//
// Network: 12 inputs -> 64 SiLU -> 64 SiLU -> 1, parameters packed as W1 [64][12], b1 [64],
// W2 [64][64], b2 [64], w3 [64], b3. Loss: mean squared error. Optimiser: Adam
// (Kingma & Ba 2015). One training step on a batch of B samples is four launches:
//   forward   (one thread per sample; activations kept for the backward pass),
//   backward  (one thread per sample; dL/dz of both hidden layers and of the output),
//   reduce    (one thread per parameter; sums over the batch, no atomics: deterministic),
//   adam      (one thread per parameter).
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

}  // namespace

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
