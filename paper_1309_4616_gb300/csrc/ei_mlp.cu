// The schedule network: inference and training kernels (FP32).
//
// A 12-64-64-64-2 fully connected network with ReLU hidden layers and a
// linear output proposes, for a phi_1 call at a candidate substep count, the
// Leja degree the a posteriori estimate will need (output 0, as a fraction
// of m_max) and the logit of meeting it within m_max (output 1).  It replaces
// the conservative a priori choice of the substep count (Sec. III-C); the a
// posteriori estimate still accepts or rejects its proposal.
//
// Parameters are one flat FP32 vector: per layer, W (out x in, row major)
// then b.  The loss of a batch is the mean over its rows of
//   mask k(e) e^2 + lam (softplus(o_1) - y_1 o_1),   e = o_0 - y_0,
// k(e) = kappa for e < 0 and 1 otherwise; Adam (Kingma and Ba) trains it.
//
// The network is tiny (9282 parameters): no tensor cores, plain FP32 FMA.
// Weights live in shared memory with odd row strides (13 and 65), so a warp
// reading a row of W (lanes over inputs) or a column (lanes over outputs)
// touches 32 distinct banks.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <string.h>

#include <vector>

#include "ei.h"
#include "ei_internal.h"

namespace ei {
namespace {

constexpr int kIn = EI_MLP_INPUTS, kH = 64, kOut = EI_MLP_OUTPUTS;
constexpr int kW0 = 0, kB0 = kW0 + kH * kIn;
constexpr int kW1 = kB0 + kH, kB1 = kW1 + kH * kH;
constexpr int kW2 = kB1 + kH, kB2 = kW2 + kH * kH;
constexpr int kW3 = kB2 + kH, kB3 = kW3 + kOut * kH;
constexpr int kNP = kB3 + kOut;
static_assert(kNP == EI_MLP_PARAMS, "parameter count");
constexpr int kS0 = kIn + 1;  // padded row strides in shared memory
constexpr int kS = kH + 1;

struct SmemW {
  float w0[kH * kS0];
  float b0[kH];
  float w1[kH * kS];
  float b1[kH];
  float w2[kH * kS];
  float b2[kH];
  float w3[kOut * kS];
  float b3[kOut];
};

__device__ void load_weights(SmemW& W, const float* __restrict__ th) {
  for (int k = threadIdx.x; k < kH * kIn; k += blockDim.x)
    W.w0[(k / kIn) * kS0 + k % kIn] = th[kW0 + k];
  for (int k = threadIdx.x; k < kH * kH; k += blockDim.x) {
    W.w1[(k / kH) * kS + k % kH] = th[kW1 + k];
    W.w2[(k / kH) * kS + k % kH] = th[kW2 + k];
  }
  for (int k = threadIdx.x; k < kOut * kH; k += blockDim.x)
    W.w3[(k / kH) * kS + k % kH] = th[kW3 + k];
  for (int k = threadIdx.x; k < kH; k += blockDim.x) {
    W.b0[k] = th[kB0 + k];
    W.b1[k] = th[kB1 + k];
    W.b2[k] = th[kB2 + k];
  }
  if (threadIdx.x < kOut) W.b3[threadIdx.x] = th[kB3 + threadIdx.x];
}

// One hidden layer for one row, by one warp: lane computes units lane and
// lane + 32 of relu(W h + b).
template <int NIN, int STRIDE>
__device__ __forceinline__ void warp_layer(const float* __restrict__ w, const float* __restrict__ b,
                                           const float* h, float* out, int lane) {
#pragma unroll
  for (int half = 0; half < 2; ++half) {
    const int u = lane + 32 * half;
    float z = b[u];
#pragma unroll 8
    for (int i = 0; i < NIN; ++i) z = fmaf(w[u * STRIDE + i], h[i], z);
    out[u] = fmaxf(z, 0.0f);
  }
}

// Forward pass of one row by one warp.  x: kIn inputs (shared); h1, h2, h3:
// the hidden activations (shared, kH each).  Returns the outputs in o0, o1
// (all lanes).
__device__ __forceinline__ void warp_forward(const SmemW& W, const float* x, float* h1, float* h2,
                                             float* h3, int lane, float& o0, float& o1) {
  warp_layer<kIn, kS0>(W.w0, W.b0, x, h1, lane);
  __syncwarp();
  warp_layer<kH, kS>(W.w1, W.b1, h1, h2, lane);
  __syncwarp();
  warp_layer<kH, kS>(W.w2, W.b2, h2, h3, lane);
  __syncwarp();
  float s0 = W.w3[lane] * h3[lane] + W.w3[lane + 32] * h3[lane + 32];
  float s1 = W.w3[kS + lane] * h3[lane] + W.w3[kS + lane + 32] * h3[lane + 32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    s0 += __shfl_xor_sync(0xffffffffu, s0, o);
    s1 += __shfl_xor_sync(0xffffffffu, s1, o);
  }
  o0 = W.b3[0] + s0;
  o1 = W.b3[1] + s1;
}

constexpr int kFwdThreads = 256;
constexpr int kFwdWarps = kFwdThreads / 32;

__global__ void __launch_bounds__(kFwdThreads) k_mlp_forward(const float* __restrict__ theta,
                                                             const float* __restrict__ X,
                                                             int64_t B, float* __restrict__ O) {
  __shared__ SmemW W;
  __shared__ float buf[kFwdWarps][kS0 + 3 * kH];
  load_weights(W, theta);
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  float* x = buf[warp];
  float* h1 = x + kS0;
  float* h2 = h1 + kH;
  float* h3 = h2 + kH;
  for (int64_t r = (int64_t)blockIdx.x * kFwdWarps + warp; r < B;
       r += (int64_t)gridDim.x * kFwdWarps) {
    if (lane < kIn) x[lane] = X[r * kIn + lane];
    __syncwarp();
    float o0, o1;
    warp_forward(W, x, h1, h2, h3, lane, o0, o1);
    if (lane == 0) {
      O[r * kOut] = o0;
      O[r * kOut + 1] = o1;
    }
    __syncwarp();
  }
}

// Training: each block takes kRows rows, runs forward and backward for them
// (one warp per row at a time), keeps every activation H_l and gradient
// G_l = dL/dZ_l in shared memory, then forms its partial gradient
// dW_l = sum_r G_l[r] (x) H_l[r], db_l = sum_r G_l[r] and writes it to
// gpart[block]; its rows' loss sum goes to lpart[block].
constexpr int kRows = 32;
constexpr int kGradThreads = 256;

struct SmemRows {
  float x[kRows * kS0];
  float h1[kRows * kS], h2[kRows * kS], h3[kRows * kS];
  float g0[kRows * kS], g1[kRows * kS], g2[kRows * kS];
  float g3[kRows * kOut];
  float loss[kGradThreads / 32];
};

__device__ __forceinline__ float softplus_f(float z) {
  return fmaxf(z, 0.0f) + log1pf(expf(-fabsf(z)));
}

__global__ void __launch_bounds__(kGradThreads)
    k_mlp_grad(const float* __restrict__ theta, const float* __restrict__ X,
               const float* __restrict__ Y, const float* __restrict__ mask, int64_t B,
               float lam, float kappa, float* __restrict__ gpart, float* __restrict__ lpart) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  SmemW& W = *reinterpret_cast<SmemW*>(smem_raw);
  SmemRows& R = *reinterpret_cast<SmemRows*>(smem_raw + sizeof(SmemW));
  load_weights(W, theta);
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nwarps = kGradThreads / 32;
  const int64_t r0 = (int64_t)blockIdx.x * kRows;
  const float invB = 1.0f / (float)B;
  float lsum = 0.0f;
  for (int rr = warp; rr < kRows; rr += nwarps) {
    const int64_t r = r0 + rr;
    const bool valid = r < B;
    float* x = R.x + rr * kS0;
    float* h1 = R.h1 + rr * kS;
    float* h2 = R.h2 + rr * kS;
    float* h3 = R.h3 + rr * kS;
    if (lane < kIn) x[lane] = valid ? X[r * kIn + lane] : 0.0f;
    __syncwarp();
    float o0, o1;
    warp_forward(W, x, h1, h2, h3, lane, o0, o1);
    // output gradient (rows beyond B contribute nothing)
    float go0 = 0.0f, go1 = 0.0f;
    if (valid) {
      const float y0 = Y[r * kOut], y1 = Y[r * kOut + 1], mk = mask[r];
      const float e = o0 - y0;
      const float k = e < 0.0f ? kappa : 1.0f;
      if (lane == 0) lsum += mk * k * e * e + lam * (softplus_f(o1) - y1 * o1);
      go0 = 2.0f * mk * k * e * invB;
      go1 = lam * (1.0f / (1.0f + expf(-o1)) - y1) * invB;
    }
    if (lane == 0) {
      R.g3[rr * kOut] = go0;
      R.g3[rr * kOut + 1] = go1;
    }
    // G_2 = relu'(Z_2) (W_3^T G_3), G_1 = relu'(Z_1) (W_2^T G_2), G_0 = relu'(Z_0) (W_1^T G_1)
    float* g2 = R.g2 + rr * kS;
    float* g1 = R.g1 + rr * kS;
    float* g0 = R.g0 + rr * kS;
#pragma unroll
    for (int half = 0; half < 2; ++half) {
      const int u = lane + 32 * half;
      const float t = W.w3[u] * go0 + W.w3[kS + u] * go1;
      g2[u] = h3[u] > 0.0f ? t : 0.0f;
    }
    __syncwarp();
#pragma unroll
    for (int half = 0; half < 2; ++half) {
      const int u = lane + 32 * half;
      float t = 0.0f;
#pragma unroll 8
      for (int k = 0; k < kH; ++k) t = fmaf(W.w2[k * kS + u], g2[k], t);
      g1[u] = h2[u] > 0.0f ? t : 0.0f;
    }
    __syncwarp();
#pragma unroll
    for (int half = 0; half < 2; ++half) {
      const int u = lane + 32 * half;
      float t = 0.0f;
#pragma unroll 8
      for (int k = 0; k < kH; ++k) t = fmaf(W.w1[k * kS + u], g1[k], t);
      g0[u] = h1[u] > 0.0f ? t : 0.0f;
    }
    __syncwarp();
  }
  // per-warp loss (rows in order), then the block's in warp order
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) lsum += __shfl_xor_sync(0xffffffffu, lsum, o);
  if (lane == 0) R.loss[warp] = lsum;
  __syncthreads();
  if (threadIdx.x == 0) {
    float t = 0.0f;
    for (int w = 0; w < nwarps; ++w) t += R.loss[w];
    lpart[blockIdx.x] = t;
  }
  // partial gradient of this block's rows
  float* gout = gpart + (int64_t)blockIdx.x * kNP;
  for (int p = threadIdx.x; p < kNP; p += blockDim.x) {
    const float* G;
    const float* H;
    int gs, hs, u, i;  // row strides of G and H; unit u, input i (i < 0: bias)
    if (p < kB0) {
      G = R.g0; gs = kS; H = R.x; hs = kS0; u = p / kIn; i = p % kIn;
    } else if (p < kW1) {
      G = R.g0; gs = kS; H = nullptr; hs = 0; u = p - kB0; i = -1;
    } else if (p < kB1) {
      G = R.g1; gs = kS; H = R.h1; hs = kS; u = (p - kW1) / kH; i = (p - kW1) % kH;
    } else if (p < kW2) {
      G = R.g1; gs = kS; H = nullptr; hs = 0; u = p - kB1; i = -1;
    } else if (p < kB2) {
      G = R.g2; gs = kS; H = R.h2; hs = kS; u = (p - kW2) / kH; i = (p - kW2) % kH;
    } else if (p < kW3) {
      G = R.g2; gs = kS; H = nullptr; hs = 0; u = p - kB2; i = -1;
    } else if (p < kB3) {
      G = R.g3; gs = kOut; H = R.h3; hs = kS; u = (p - kW3) / kH; i = (p - kW3) % kH;
    } else {
      G = R.g3; gs = kOut; H = nullptr; hs = 0; u = p - kB3; i = -1;
    }
    float acc = 0.0f;
    if (i >= 0) {
#pragma unroll 8
      for (int r = 0; r < kRows; ++r) acc = fmaf(G[r * gs + u], H[r * hs + i], acc);
    } else {
#pragma unroll 8
      for (int r = 0; r < kRows; ++r) acc += G[r * gs + u];
    }
    gout[p] = acc;
  }
}

// Sum of the block partials in block order (deterministic); then either the
// gradient is written out, or Adam updates theta, m and v.  Thread 0 of block
// 0 also sums the loss partials.
__global__ void k_mlp_reduce(const float* __restrict__ gpart, const float* __restrict__ lpart,
                             int nblocks, int64_t B, float* __restrict__ grad,
                             float* __restrict__ theta, float* __restrict__ m,
                             float* __restrict__ v, float lr, float b1, float b2, float c1,
                             float c2, float eps, double* __restrict__ loss_out) {
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < kNP; p += gridDim.x * blockDim.x) {
    float g = 0.0f;
    for (int b = 0; b < nblocks; ++b) g += gpart[(int64_t)b * kNP + p];
    if (grad) grad[p] = g;
    if (theta) {
      const float mi = b1 * m[p] + (1.0f - b1) * g;
      const float vi = b2 * v[p] + (1.0f - b2) * g * g;
      m[p] = mi;
      v[p] = vi;
      theta[p] -= lr * (mi * c1) / (sqrtf(vi * c2) + eps);
    }
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    double t = 0.0;
    for (int b = 0; b < nblocks; ++b) t += (double)lpart[b];
    *loss_out = t / (double)B;
  }
}

}  // namespace
}  // namespace ei

using namespace ei;

struct ei_mlp {
  int device = 0;
  cudaStream_t stream = nullptr;
  float* theta = nullptr;  // device parameters
  float* m = nullptr;      // Adam moments
  float* v = nullptr;
  float* gpart = nullptr;  // per-block partial gradients
  float* lpart = nullptr;
  int64_t part_blocks = 0;
  double* d_loss = nullptr;
  double* h_loss = nullptr;  // pinned
  float* d_x = nullptr;      // small staging for the library's own inference
  float* d_o = nullptr;
  float* h_xo = nullptr;     // pinned: inputs then outputs
  int64_t t = 0;             // Adam step count
  ei_mlp_decision dec{};
  float* big_x = nullptr;    // staging of many-row inference (mlp_infer_rows)
  float* big_o = nullptr;
  float* big_h = nullptr;    // pinned
  int64_t big_rows = 0;
};

namespace {

size_t grad_smem() { return sizeof(SmemW) + sizeof(SmemRows); }

ei_status grow_parts(ei_mlp* M, int64_t nb) {
  if (nb <= M->part_blocks) return EI_OK;
  cudaFree(M->gpart);
  cudaFree(M->lpart);
  M->gpart = nullptr;
  M->lpart = nullptr;
  M->part_blocks = 0;
  if (cudaMalloc(&M->gpart, sizeof(float) * kNP * nb) != cudaSuccess ||
      cudaMalloc(&M->lpart, sizeof(float) * nb) != cudaSuccess) {
    cudaGetLastError();
    return EI_ERR_NOMEM;
  }
  M->part_blocks = nb;
  return EI_OK;
}

ei_status launch_grad(ei_mlp* M, const float* x, const float* y, const float* mask, int64_t B,
                      double lam, double kappa, int64_t* nb_out) {
  const int64_t nb = (B + kRows - 1) / kRows;
  if (nb > (1 << 24)) return EI_ERR_INVALID_ARG;
  ei_status rs = grow_parts(M, nb);
  if (rs != EI_OK) return rs;
  if (cudaFuncSetAttribute(k_mlp_grad, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)grad_smem()) != cudaSuccess)
    return EI_ERR_CUDA;
  k_mlp_grad<<<(unsigned)nb, kGradThreads, grad_smem(), M->stream>>>(
      M->theta, x, y, mask, B, (float)lam, (float)kappa, M->gpart, M->lpart);
  if (cudaGetLastError() != cudaSuccess) return EI_ERR_CUDA;
  *nb_out = nb;
  return EI_OK;
}

}  // namespace

// Library-internal: the network's outputs for `rows` host feature rows
// (FP64, kIn each) -> host outputs (FP32 rounding, kOut each).  Synchronises
// the model's stream.
namespace ei {
ei_status mlp_infer_host(const ei_mlp* Mc, const double* feat, int rows, float* out) {
  ei_mlp* M = const_cast<ei_mlp*>(Mc);
  if (rows < 1 || rows > EI_MLP_MAX_Q + 1) return EI_ERR_INVALID_ARG;
  for (int i = 0; i < rows * kIn; ++i) M->h_xo[i] = (float)feat[i];
  if (cudaMemcpyAsync(M->d_x, M->h_xo, sizeof(float) * rows * kIn, cudaMemcpyHostToDevice,
                      M->stream) != cudaSuccess)
    return EI_ERR_CUDA;
  k_mlp_forward<<<1, kFwdThreads, 0, M->stream>>>(M->theta, M->d_x, rows, M->d_o);
  if (cudaGetLastError() != cudaSuccess) return EI_ERR_CUDA;
  float* ho = M->h_xo + (EI_MLP_MAX_Q + 1) * kIn;
  if (cudaMemcpyAsync(ho, M->d_o, sizeof(float) * rows * kOut, cudaMemcpyDeviceToHost,
                      M->stream) != cudaSuccess ||
      cudaStreamSynchronize(M->stream) != cudaSuccess)
    return EI_ERR_CUDA;
  memcpy(out, ho, sizeof(float) * rows * kOut);
  return EI_OK;
}
const ei_mlp_decision& mlp_decision(const ei_mlp* M) { return M->dec; }

// Any number of rows: staging buffers grow as needed (pinned host, device).
ei_status mlp_infer_rows(const ei_mlp* Mc, const double* feat, int64_t rows, float* out) {
  ei_mlp* M = const_cast<ei_mlp*>(Mc);
  if (rows < 1) return EI_ERR_INVALID_ARG;
  if (rows > M->big_rows) {
    cudaFree(M->big_x);
    cudaFree(M->big_o);
    cudaFreeHost(M->big_h);
    M->big_x = M->big_o = M->big_h = nullptr;
    M->big_rows = 0;
    if (cudaMalloc(&M->big_x, sizeof(float) * rows * kIn) != cudaSuccess ||
        cudaMalloc(&M->big_o, sizeof(float) * rows * kOut) != cudaSuccess ||
        cudaMallocHost(&M->big_h, sizeof(float) * rows * (kIn + kOut)) != cudaSuccess) {
      cudaGetLastError();
      return EI_ERR_NOMEM;
    }
    M->big_rows = rows;
  }
  for (int64_t i = 0; i < rows * kIn; ++i) M->big_h[i] = (float)feat[i];
  float* ho = M->big_h + rows * kIn;
  if (cudaMemcpyAsync(M->big_x, M->big_h, sizeof(float) * rows * kIn, cudaMemcpyHostToDevice,
                      M->stream) != cudaSuccess)
    return EI_ERR_CUDA;
  if (ei_mlp_forward(M, M->big_x, rows, M->big_o) != EI_OK) return EI_ERR_CUDA;
  if (cudaMemcpyAsync(ho, M->big_o, sizeof(float) * rows * kOut, cudaMemcpyDeviceToHost,
                      M->stream) != cudaSuccess ||
      cudaStreamSynchronize(M->stream) != cudaSuccess)
    return EI_ERR_CUDA;
  memcpy(out, ho, sizeof(float) * rows * kOut);
  return EI_OK;
}
}  // namespace ei

extern "C" {

ei_status ei_mlp_create(ei_mlp** out, int device, void* stream) {
  if (!out) return EI_ERR_INVALID_ARG;
  *out = nullptr;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
    cudaGetLastError();
    return device < 0 ? EI_ERR_INVALID_ARG : EI_ERR_CUDA;
  }
  if (cudaSetDevice(device) != cudaSuccess) return EI_ERR_CUDA;
  ei_mlp* M = new ei_mlp();
  M->device = device;
  M->stream = (cudaStream_t)stream;
  M->dec.z_min = 0.0;
  M->dec.rho_m = 0.05;
  M->dec.delta_m = 2.0;
  M->dec.q_max = EI_MLP_MAX_Q;
  const int rows = EI_MLP_MAX_Q + 1;
  if (cudaMalloc(&M->theta, sizeof(float) * kNP) != cudaSuccess ||
      cudaMalloc(&M->m, sizeof(float) * kNP) != cudaSuccess ||
      cudaMalloc(&M->v, sizeof(float) * kNP) != cudaSuccess ||
      cudaMalloc(&M->d_loss, sizeof(double)) != cudaSuccess ||
      cudaMalloc(&M->d_x, sizeof(float) * rows * kIn) != cudaSuccess ||
      cudaMalloc(&M->d_o, sizeof(float) * rows * kOut) != cudaSuccess ||
      cudaMallocHost(&M->h_loss, sizeof(double)) != cudaSuccess ||
      cudaMallocHost(&M->h_xo, sizeof(float) * rows * (kIn + kOut)) != cudaSuccess) {
    cudaGetLastError();
    ei_mlp_destroy(M);
    return EI_ERR_NOMEM;
  }
  if (cudaMemset(M->theta, 0, sizeof(float) * kNP) != cudaSuccess ||
      cudaMemset(M->m, 0, sizeof(float) * kNP) != cudaSuccess ||
      cudaMemset(M->v, 0, sizeof(float) * kNP) != cudaSuccess) {
    ei_mlp_destroy(M);
    return EI_ERR_CUDA;
  }
  *out = M;
  return EI_OK;
}

void ei_mlp_destroy(ei_mlp* M) {
  if (!M) return;
  cudaSetDevice(M->device);
  if (M->stream) cudaStreamSynchronize(M->stream);
  cudaFree(M->theta);
  cudaFree(M->m);
  cudaFree(M->v);
  cudaFree(M->gpart);
  cudaFree(M->lpart);
  cudaFree(M->d_loss);
  cudaFree(M->d_x);
  cudaFree(M->d_o);
  cudaFreeHost(M->h_loss);
  cudaFreeHost(M->h_xo);
  cudaFree(M->big_x);
  cudaFree(M->big_o);
  cudaFreeHost(M->big_h);
  delete M;
}

ei_status ei_mlp_set_params(ei_mlp* M, const float* theta) {
  if (!M || !theta) return EI_ERR_INVALID_ARG;
  for (int i = 0; i < kNP; ++i)
    if (!isfinite(theta[i])) return EI_ERR_NONFINITE;
  if (cudaSetDevice(M->device) != cudaSuccess ||
      cudaMemcpyAsync(M->theta, theta, sizeof(float) * kNP, cudaMemcpyHostToDevice, M->stream) !=
          cudaSuccess ||
      cudaMemsetAsync(M->m, 0, sizeof(float) * kNP, M->stream) != cudaSuccess ||
      cudaMemsetAsync(M->v, 0, sizeof(float) * kNP, M->stream) != cudaSuccess ||
      cudaStreamSynchronize(M->stream) != cudaSuccess)
    return EI_ERR_CUDA;
  M->t = 0;
  return EI_OK;
}

ei_status ei_mlp_get_params(ei_mlp* M, float* theta) {
  if (!M || !theta) return EI_ERR_INVALID_ARG;
  if (cudaSetDevice(M->device) != cudaSuccess ||
      cudaMemcpyAsync(theta, M->theta, sizeof(float) * kNP, cudaMemcpyDeviceToHost, M->stream) !=
          cudaSuccess ||
      cudaStreamSynchronize(M->stream) != cudaSuccess)
    return EI_ERR_CUDA;
  return EI_OK;
}

ei_status ei_mlp_set_decision(ei_mlp* M, const ei_mlp_decision* d) {
  if (!M || !d || !isfinite(d->z_min) || !isfinite(d->rho_m) || !isfinite(d->delta_m) ||
      d->rho_m < 0 || d->q_max < 0 || d->q_max > EI_MLP_MAX_Q)
    return EI_ERR_INVALID_ARG;
  M->dec = *d;
  return EI_OK;
}

ei_status ei_mlp_get_decision(const ei_mlp* M, ei_mlp_decision* d) {
  if (!M || !d) return EI_ERR_INVALID_ARG;
  *d = M->dec;
  return EI_OK;
}

ei_status ei_mlp_forward(ei_mlp* M, const float* x, int64_t B, float* out) {
  if (!M || B < 0 || (B > 0 && (!x || !out))) return EI_ERR_INVALID_ARG;
  if (B == 0) return EI_OK;
  if (cudaSetDevice(M->device) != cudaSuccess) return EI_ERR_CUDA;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int64_t want = (B + kFwdWarps - 1) / kFwdWarps;
  const int64_t cap = (int64_t)(sms > 0 ? sms : 1) * 8;
  const unsigned grid = (unsigned)(want < cap ? want : cap);
  k_mlp_forward<<<grid, kFwdThreads, 0, M->stream>>>(M->theta, x, B, out);
  if (cudaGetLastError() != cudaSuccess) return EI_ERR_CUDA;
  return EI_OK;
}

ei_status ei_mlp_loss_grad(ei_mlp* M, const float* x, const float* y, const float* mask,
                           int64_t B, double lam, double kappa, double* loss, float* grad) {
  if (!M || B < 1 || !x || !y || !mask || !grad || !(lam >= 0) || !(kappa > 0) ||
      !isfinite(lam) || !isfinite(kappa))
    return EI_ERR_INVALID_ARG;
  if (cudaSetDevice(M->device) != cudaSuccess) return EI_ERR_CUDA;
  int64_t nb = 0;
  ei_status rs = launch_grad(M, x, y, mask, B, lam, kappa, &nb);
  if (rs != EI_OK) return rs;
  k_mlp_reduce<<<(kNP + 255) / 256, 256, 0, M->stream>>>(
      M->gpart, M->lpart, (int)nb, B, grad, nullptr, nullptr, nullptr, 0.f, 0.f, 0.f, 0.f, 0.f,
      0.f, M->d_loss);
  if (cudaGetLastError() != cudaSuccess) return EI_ERR_CUDA;
  if (loss) {
    if (cudaMemcpyAsync(M->h_loss, M->d_loss, sizeof(double), cudaMemcpyDeviceToHost,
                        M->stream) != cudaSuccess ||
        cudaStreamSynchronize(M->stream) != cudaSuccess)
      return EI_ERR_CUDA;
    *loss = *M->h_loss;
  }
  return EI_OK;
}

ei_status ei_mlp_train_step(ei_mlp* M, const float* x, const float* y, const float* mask,
                            int64_t B, double lam, double kappa, double lr, double* loss) {
  if (!M || B < 1 || !x || !y || !mask || !(lam >= 0) || !(kappa > 0) || !(lr > 0) ||
      !isfinite(lam) || !isfinite(kappa) || !isfinite(lr))
    return EI_ERR_INVALID_ARG;
  if (cudaSetDevice(M->device) != cudaSuccess) return EI_ERR_CUDA;
  int64_t nb = 0;
  ei_status rs = launch_grad(M, x, y, mask, B, lam, kappa, &nb);
  if (rs != EI_OK) return rs;
  const double b1 = 0.9, b2 = 0.999, eps = 1e-8;
  M->t += 1;
  const double c1 = 1.0 / (1.0 - pow(b1, (double)M->t));
  const double c2 = 1.0 / (1.0 - pow(b2, (double)M->t));
  k_mlp_reduce<<<(kNP + 255) / 256, 256, 0, M->stream>>>(
      M->gpart, M->lpart, (int)nb, B, nullptr, M->theta, M->m, M->v, (float)lr, (float)b1,
      (float)b2, (float)c1, (float)c2, (float)eps, M->d_loss);
  if (cudaGetLastError() != cudaSuccess) return EI_ERR_CUDA;
  if (loss) {
    if (cudaMemcpyAsync(M->h_loss, M->d_loss, sizeof(double), cudaMemcpyDeviceToHost,
                        M->stream) != cudaSuccess ||
        cudaStreamSynchronize(M->stream) != cudaSuccess)
      return EI_ERR_CUDA;
    *loss = *M->h_loss;
  }
  return EI_OK;
}

}  // extern "C"
