// tkf_mlp.cu -- training and inference kernels of the learned step proposer.
//
// Network: 12 inputs -> 64 SiLU -> 64 SiLU -> 1, parameters packed as W1 [64][12], b1 [64],
// W2 [64][64], b2 [64], w3 [64], b3 (FP32 master copy). Loss: mean squared error. Optimiser:
// Adam (Kingma & Ba 2015). One training step on a batch of B samples is two launches:
//   mlp_train_tc_kernel: one CTA per 128 samples; the forward and backward pass with every
//     dense contraction on the tensor cores (tcgen05.mma kind::f16, BF16 operands, FP32
//     accumulation in tensor memory): the two layers, the backpropagation through layer 2, and
//     the weight gradients of both layers together with the bias gradients (one M128 N96 K128
//     product per CTA); the output layer, bias, SiLU and its derivative on the CUDA cores in
//     FP32; each CTA writes its partial gradient;
//   mlp_reduce_adam_kernel: one thread per parameter; the partials summed in CTA order (no
//     atomics: deterministic), then the Adam step.
// Around training: seeded initialisation, calibration of the output bias (a quantile of the
// training residuals, by a radix select on the device) and rounding to the BF16 weights the
// fit's inference uses.
// The paper has no learned component; the learned step proposer is an addition to its method.

#include <math.h>

#include "tkf_fit_impl.cuh"

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

// ---- training on the tensor cores
// One CTA of 128 threads per tile of 128 samples, thread s = sample s = accumulator row s.
// Operands in shared memory are K-major, no swizzle, 8 x 16-byte core matrices (core_offset);
// a K16 step of an operand with g groups of 8 along K starts 256 bytes further, its K groups
// are 128 bytes apart and its row groups g x 128 bytes apart.
//   xa  [128 x 16]   features (12, then zeros)           layer 1:  Z1 = X W1^T       M128 N64 K16
//   a1  [128 x 64]   SiLU(Z1 + b1)                        layer 2:  Z2 = A1 W2^T      M128 N64 K64
//   dz2 [128 x 64]   dL/dZ2 = dout w3 SiLU'(Z2 + b2)      back:     dA1 = dZ2 W2      M128 N64 K64
//   ag  [128 x 128]  rows 0..63: dZ2^T, rows 64..127: dZ1^T (dZ1 = dA1 SiLU'(Z1 + b1)); K = samples
//   bg  [96 x 128]   rows 0..63: A1^T, 64..79: X^T, 80: ones, 81..95: zeros
//   gradients:       G = ag bg^T                          M128 N96 K128
//     G[j][i] = dW2[j][i] (j, i < 64), G[64 + j][64 + q] = dW1[j][q], G[r][80] = db2 / db1.
// w3 and b3 get their gradients on the CUDA cores (FP32, a fixed-order sum over the tile).
// BF16 operands are rounded to nearest even from the FP32 values; the products are exact and
// summed in FP32.
constexpr int kTile = 128;
constexpr uint32_t kIdescN64 = umma_idesc_bf16(128, 64);
constexpr uint32_t kIdescN96 = umma_idesc_bf16(128, 96);
static_assert(kIdescN64 == kIdescM128N64, "instruction descriptor");

struct __align__(1024) TrainSmem {
  uint8_t ag[128 * 128 * 2];  // 32 KB
  uint8_t bg[96 * 128 * 2];   // 24 KB
  uint8_t a1[128 * 64 * 2];   // 16 KB
  uint8_t dz2[128 * 64 * 2];  // 16 KB
  uint8_t w2[64 * 64 * 2];    // W2 (N = outputs j, K = inputs i)
  uint8_t w2t[64 * 64 * 2];   // W2^T (N = i, K = j)
  uint8_t xa[128 * 16 * 2];
  uint8_t w1[64 * 16 * 2];    // W1 (N = j, K = inputs, 12..15 zero)
  float red[66][kTile];       // per-sample dout a2[j] (j < 64), dout, squared residual
  float b1[64], b2[64], w3[64], b3;
  uint64_t mbar;
  uint32_t tmem_base;
};

__device__ __forceinline__ void st_bf16(uint8_t* base, uint32_t off, float v) {
  *reinterpret_cast<uint16_t*>(base + off) = uint16_t(bf16_rne(v));
}

// Issues `nk` K16 steps of D = A B^T into tensor memory (thread 0), commits them to the
// mbarrier and waits (every thread, bounded). Returns false if the wait ran out.
__device__ bool tc_stage(TrainSmem& sm, uint32_t tmem, const uint8_t* a, uint32_t a_sbo, const uint8_t* b,
                         uint32_t b_sbo, int nk, uint32_t idesc, uint32_t& phase, bool stall) {
  fence_async_smem();
  tc_fence_before();
  __syncthreads();
  if (threadIdx.x == 0 && !stall) {
    tc_fence_after();
    for (int k = 0; k < nk; ++k)
      tc_mma_id(tmem, umma_desc(smem_addr(a) + k * 256, 128, a_sbo), umma_desc(smem_addr(b) + k * 256, 128, b_sbo),
                idesc, k > 0 ? 1u : 0u);
    tc_commit(&sm.mbar);
  }
  const bool done = mbar_wait(&sm.mbar, phase);
  phase ^= 1u;
  __syncwarp();
  tc_fence_after();
  return __syncthreads_or(!done) == 0;
}

// Forward and backward pass of one tile; the CTA's partial gradient (TKF_MLP_PARAMS floats) and
// its sum of squared residuals go to part[blockIdx.x] and sq[blockIdx.x]. `inv_n`: 1 / batch
// size (dL/dout = 2 r / n). A wait that ran out leaves NaN partials (and so NaN losses).
__global__ void __launch_bounds__(kTile, 1) mlp_train_tc_kernel(const float* __restrict__ p, const float* __restrict__ x,
                                                                 int x_stride, const float* __restrict__ y, int y_stride,
                                                                 uint32_t n, float inv_n, float* __restrict__ part,
                                                                 float* __restrict__ sq) {
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  // the operands at a 1024-byte boundary (the launch reserves the slack)
  const uint32_t pad = (1024u - (smem_addr(smem_raw) & 1023u)) & 1023u;
  TrainSmem& sm = *reinterpret_cast<TrainSmem*>(smem_raw + pad);
  const int tid = threadIdx.x, warp = tid >> 5;
  // weights as BF16 operands (both orientations of W2), biases and w3 in FP32
  for (int e = tid; e < 64 * 16; e += kTile) {
    const int j = e >> 4, i = e & 15;
    st_bf16(sm.w1, core_offset(j, i, 2), i < kIn ? p[oW1 + j * kIn + i] : 0.0f);
  }
  for (int e = tid; e < 64 * 64; e += kTile) {
    const int j = e >> 6, i = e & 63;
    const float w = p[oW2 + e];
    st_bf16(sm.w2, core_offset(j, i, 8), w);
    st_bf16(sm.w2t, core_offset(i, j, 8), w);
  }
  if (tid < 64) {
    sm.b1[tid] = p[oB1 + tid];
    sm.b2[tid] = p[oB2 + tid];
    sm.w3[tid] = p[oW3 + tid];
  }
  if (tid == 0) {
    sm.b3 = p[oB3];
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(&sm.mbar)) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {  // 128 accumulator columns: each stage writes from column 0
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 128;" ::"r"(smem_addr(&sm.tmem_base))
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  // this sample's inputs (rows beyond the batch: zeros, and no gradient)
  const uint32_t s = blockIdx.x * kTile + tid;
  const bool live = s < n;
  float xv[kIn], yv = 0.0f;
  for (int i = 0; i < kIn; ++i) xv[i] = live ? x[size_t(s) * x_stride + i] : 0.0f;
  if (live) yv = y[size_t(s) * y_stride];
  for (int i = 0; i < 16; ++i) {
    const float v = i < kIn ? xv[i] : 0.0f;
    st_bf16(sm.xa, core_offset(tid, i, 2), v);
    st_bf16(sm.bg, core_offset(64 + i, tid, 16), v);  // X^T
  }
  st_bf16(sm.bg, core_offset(80, tid, 16), 1.0f);  // ones: the bias gradients
  for (int r = 81; r < 96; ++r) st_bf16(sm.bg, core_offset(r, tid, 16), 0.0f);
  fence_async_smem();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = sm.tmem_base;
  const uint32_t t_row = tmem + (uint32_t(warp * 32) << 16);  // this warp's 32 lanes
  uint32_t phase = 0;
  bool ok = true;
  float v[32], d1[64];  // d1: SiLU'(Z1 + b1) of this sample
  // layer 1
  ok = tc_stage(sm, tmem, sm.xa, 256, sm.w1, 256, 1, kIdescN64, phase, false);
  if (ok) {
    for (int half = 0; half < 2; ++half) {
      tmem_ld32(t_row + uint32_t(half * 32), v);
      for (int k = 0; k < 32; ++k) {
        const int j = half * 32 + k;
        const float z = v[k] + sm.b1[j], sg = sigm(z), a = z * sg;
        d1[j] = sg * (1.0f + z * (1.0f - sg));
        st_bf16(sm.a1, core_offset(tid, j, 8), a);
        st_bf16(sm.bg, core_offset(j, tid, 16), a);  // A1^T
      }
    }
    // layer 2
    ok = tc_stage(sm, tmem, sm.a1, 1024, sm.w2, 1024, 4, kIdescN64, phase, false);
  }
  if (ok) {
    float z2[64], a2[64];
    float out = sm.b3;
    for (int half = 0; half < 2; ++half) {
      tmem_ld32(t_row + uint32_t(half * 32), v);
      for (int k = 0; k < 32; ++k) {
        const int j = half * 32 + k;
        z2[j] = v[k] + sm.b2[j];
        a2[j] = z2[j] * sigm(z2[j]);
        out = fmaf(sm.w3[j], a2[j], out);
      }
    }
    const float r = live ? out - yv : 0.0f;
    const float dout = 2.0f * r * inv_n;
    for (int j = 0; j < 64; ++j) {
      const float sg = sigm(z2[j]);
      const float dz = dout * sm.w3[j] * (sg * (1.0f + z2[j] * (1.0f - sg)));
      st_bf16(sm.dz2, core_offset(tid, j, 8), dz);
      st_bf16(sm.ag, core_offset(j, tid, 16), dz);  // dZ2^T
      sm.red[j][tid] = dout * a2[j];
    }
    sm.red[64][tid] = dout;
    sm.red[65][tid] = r * r;
    // backpropagation through layer 2
    ok = tc_stage(sm, tmem, sm.dz2, 1024, sm.w2t, 1024, 4, kIdescN64, phase, false);
  }
  if (ok) {
    for (int half = 0; half < 2; ++half) {
      tmem_ld32(t_row + uint32_t(half * 32), v);
      for (int k = 0; k < 32; ++k) {
        const int i = half * 32 + k;
        st_bf16(sm.ag, core_offset(64 + i, tid, 16), v[k] * d1[i]);  // dZ1^T
      }
    }
    // weight and bias gradients of both layers: G = ag bg^T over the tile's samples
    ok = tc_stage(sm, tmem, sm.ag, 2048, sm.bg, 2048, 8, kIdescN96, phase, false);
  }
  float* g = part + size_t(blockIdx.x) * kMlpParams;
  const float nan = __int_as_float(0x7fc00000);
  if (ok) {
    // row tid of G: dW2 row tid and db2 (tid < 64), or dW1 row tid - 64 and db1
    for (int c = 0; c < 3; ++c) {
      tmem_ld32(t_row + uint32_t(c * 32), v);
      for (int k = 0; k < 32; ++k) {
        const int col = c * 32 + k;
        if (tid < 64) {
          if (col < 64) g[oW2 + tid * 64 + col] = v[k];
          if (col == 80) g[oB2 + tid] = v[k];
        } else {
          if (col >= 64 && col < 64 + kIn) g[oW1 + (tid - 64) * kIn + (col - 64)] = v[k];
          if (col == 80) g[oB1 + tid - 64] = v[k];
        }
      }
    }
    // w3, b3 and the squared residuals: sums over the tile in sample order
    if (tid < 66) {
      float acc = 0.0f;
      for (int t = 0; t < kTile; ++t) acc += sm.red[tid][t];
      if (tid < 64)
        g[oW3 + tid] = acc;
      else if (tid == 64)
        g[oB3] = acc;
      else
        sq[blockIdx.x] = acc;
    }
  } else {
    for (int k = tid; k < kMlpParams; k += kTile) g[k] = nan;
    if (tid == 0) sq[blockIdx.x] = nan;
    mbar_wait(&sm.mbar, phase ^ 1u);  // give an MMA still in flight a bounded time to finish
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 128;" ::"r"(tmem) : "memory");
  }
}

// Sum of the CTAs' partial gradients (in CTA order), written to grad, then (when m is not
// null) one Adam step of the parameters; thread 0 also writes the batch's mean squared residual
// to *loss and adds it, weighted, to *epoch_acc.
__global__ void __launch_bounds__(256) mlp_reduce_adam_kernel(const float* __restrict__ part,
                                                              const float* __restrict__ sq, uint32_t n_cta, float inv_n,
                                                              float* __restrict__ grad, float* __restrict__ p,
                                                              float* __restrict__ m, float* __restrict__ v, float lr,
                                                              float beta1, float beta2, float eps, float c1, float c2,
                                                              float* __restrict__ loss, float* __restrict__ epoch_acc,
                                                              float inv_batches) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k == 0) {
    float l = 0.0f;
    for (uint32_t c = 0; c < n_cta; ++c) l += sq[c];
    l *= inv_n;
    if (loss) *loss = l;
    if (epoch_acc) *epoch_acc += l * inv_batches;
  }
  if (k >= kMlpParams) return;
  float gk = 0.0f;
  for (uint32_t c = 0; c < n_cta; ++c) gk += part[size_t(c) * kMlpParams + k];
  if (grad) grad[k] = gk;
  if (!m) return;
  const float mk = beta1 * m[k] + (1.0f - beta1) * gk;
  const float vk = beta2 * v[k] + (1.0f - beta2) * gk * gk;
  m[k] = mk;
  v[k] = vk;
  p[k] -= lr * (mk / c1) / (sqrtf(vk / c2) + eps);
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
  const size_t n_cta = (size_t(batch) + kTile - 1) / kTile;
  return sizeof(float) * (n_cta * (kMlpParams + 1) + kMlpParams) + 256;
}

namespace {
// Partial gradients [n_cta][params], per-CTA squared residuals [n_cta], the summed gradient.
struct TrainScratch {
  float* part;
  float* sq;
  float* grad;
};
TrainScratch carve_train(void* base, uint32_t batch) {
  const size_t n_cta = (size_t(batch) + kTile - 1) / kTile;
  float* f = static_cast<float*>(base);
  return TrainScratch{f, f + n_cta * kMlpParams, f + n_cta * (kMlpParams + 1)};
}

cudaError_t train_tile_launch(const float* params, const float* x, int x_stride, const float* y, int y_stride,
                              uint32_t n, const TrainScratch& sc, cudaStream_t stream) {
  static_assert(sizeof(TrainSmem) + 1024 <= 227 * 1024, "shared memory");
  const size_t smem = sizeof(TrainSmem) + 1024;  // + alignment slack
  cudaError_t e = cudaFuncSetAttribute(mlp_train_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
  if (e != cudaSuccess) return e;
  const unsigned n_cta = (n + kTile - 1) / kTile;
  mlp_train_tc_kernel<<<n_cta, kTile, smem, stream>>>(params, x, x_stride, y, y_stride, n, 1.0f / float(n), sc.part,
                                                      sc.sq);
  return cudaGetLastError();
}
}  // namespace

cudaError_t mlp_loss_grad(const float* params, const float* x, int x_stride, const float* y, int y_stride,
                          uint32_t n, float* grad, float* loss, void* scratch, cudaStream_t stream) {
  const TrainScratch sc = carve_train(scratch, n);
  cudaError_t e = train_tile_launch(params, x, x_stride, y, y_stride, n, sc, stream);
  if (e != cudaSuccess) return e;
  const unsigned n_cta = (n + kTile - 1) / kTile;
  mlp_reduce_adam_kernel<<<(kMlpParams + 255) / 256, 256, 0, stream>>>(
      sc.part, sc.sq, n_cta, 1.0f / float(n), grad, nullptr, nullptr, nullptr, 0.0f, 0.0f, 0.0f, 0.0f, 1.0f, 1.0f, loss,
      nullptr, 0.0f);
  return cudaGetLastError();
}

cudaError_t mlp_train(const float* records, uint32_t n, uint32_t batch, uint32_t epochs, float lr, float beta1,
                      float beta2, float eps, float* params, float* moments, uint32_t* adam_t, float* epoch_loss,
                      void* scratch, cudaStream_t stream) {
  const TrainScratch sc = carve_train(scratch, batch);
  const uint32_t nb = n / batch;
  const unsigned n_cta = (batch + kTile - 1) / kTile;
  cudaError_t e = cudaMemsetAsync(epoch_loss, 0, sizeof(float) * epochs, stream);
  if (e != cudaSuccess) return e;
  for (uint32_t ep = 0; ep < epochs; ++ep) {
    for (uint32_t b = 0; b < nb; ++b) {
      const float* rec = records + size_t(b) * batch * kMlpRecord;
      e = train_tile_launch(params, rec, kMlpRecord, rec + 12, kMlpRecord, batch, sc, stream);
      if (e != cudaSuccess) return e;
      const uint32_t t = ++(*adam_t);
      const float c1 = 1.0f - powf(beta1, float(t)), c2 = 1.0f - powf(beta2, float(t));
      mlp_reduce_adam_kernel<<<(kMlpParams + 255) / 256, 256, 0, stream>>>(
          sc.part, sc.sq, n_cta, 1.0f / float(batch), sc.grad, params, moments, moments + kMlpParams, lr, beta1, beta2,
          eps, c1, c2, nullptr, epoch_loss + ep, 1.0f / float(nb));
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
