// Learned (s, m) selector: a small FP32 MLP 8 -> 64 -> 64 -> 52 (21 logits for s = 0..20,
// 31 for m = 2..32), ReLU, trained with cross-entropy on both heads by hand-written kernels:
//   mlp_forward_kernel  one thread per sample, weights in shared memory
//   mlp_grad_kernel     one thread per sample for the forward/backward activations, then one
//                       thread per weight for the batch reduction of the weight gradients;
//                       each block adds its partial gradient into the global buffer
//   adam_kernel         Adam update of the flat parameter vector
// The training loop (phikron_selector_train) keeps features and labels on the device and
// draws a random permutation per epoch on the host.  The trained parameters become the
// process-wide model used by plans made with PHIKRON_SELECT_MLP.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>
#include <random>
#include <vector>

#include "common.h"
#include "profile.h"

namespace phikron {
namespace mlp {

constexpr int IN = 8, H = 64, OS = 21, OM = 31, OUT = OS + OM;
constexpr int NPARAM = IN * H + H + H * H + H + H * OUT + OUT;  // 8116
constexpr int OFF_W1 = 0, OFF_B1 = IN * H, OFF_W2 = OFF_B1 + H, OFF_B2 = OFF_W2 + H * H,
              OFF_W3 = OFF_B2 + H, OFF_B3 = OFF_W3 + H * OUT;
constexpr int SPB = 64;  // samples per block

namespace {

__global__ void __launch_bounds__(SPB) mlp_forward_kernel(const float* __restrict__ params,
                                                          const float* __restrict__ X, int count,
                                                          float* __restrict__ logits, int* __restrict__ s_out,
                                                          int* __restrict__ m_out) {
  __shared__ float w[NPARAM];
  for (int i = threadIdx.x; i < NPARAM; i += SPB) w[i] = params[i];
  __syncthreads();
  const int n = blockIdx.x * SPB + threadIdx.x;
  if (n >= count) return;
  float x[IN], h1[H], h2[H];
#pragma unroll
  for (int i = 0; i < IN; ++i) x[i] = X[(size_t)n * IN + i];
#pragma unroll 4
  for (int j = 0; j < H; ++j) {
    float a = w[OFF_B1 + j];
#pragma unroll
    for (int i = 0; i < IN; ++i) a = fmaf(x[i], w[OFF_W1 + i * H + j], a);
    h1[j] = fmaxf(a, 0.f);
  }
#pragma unroll 4
  for (int j = 0; j < H; ++j) {
    float a = w[OFF_B2 + j];
#pragma unroll
    for (int i = 0; i < H; ++i) a = fmaf(h1[i], w[OFF_W2 + i * H + j], a);
    h2[j] = fmaxf(a, 0.f);
  }
  int bs = 0, bm = 0;
  float vs = -INFINITY, vm = -INFINITY;
  for (int j = 0; j < OUT; ++j) {
    float a = w[OFF_B3 + j];
#pragma unroll
    for (int i = 0; i < H; ++i) a = fmaf(h2[i], w[OFF_W3 + i * OUT + j], a);
    if (logits) logits[(size_t)n * OUT + j] = a;
    if (j < OS) {
      if (a > vs) { vs = a; bs = j; }
    } else if (a > vm) {
      vm = a;
      bm = j - OS;
    }
  }
  if (s_out) s_out[n] = bs;
  if (m_out) m_out[n] = bm + 2;
}

// Gradient of the mean loss over `count` samples idx[0..count) (or 0..count when idx is null);
// grad must be zeroed by the caller; loss_sum accumulates the summed per-sample loss.
__global__ void __launch_bounds__(SPB) mlp_grad_kernel(const float* __restrict__ params,
                                                       const float* __restrict__ X, const int* __restrict__ ys,
                                                       const int* __restrict__ ym, const int* __restrict__ idx,
                                                       int count, float inv_batch, float* __restrict__ grad,
                                                       float* __restrict__ loss_sum) {
  extern __shared__ float sm[];
  float* w = sm;                      // NPARAM
  float* sx = w + NPARAM;             // SPB x IN
  float* s1 = sx + SPB * IN;          // SPB x H   (h1 after ReLU)
  float* s2 = s1 + SPB * H;           // SPB x H   (h2 after ReLU)
  float* sd = s2 + SPB * H;           // SPB x OUT (dLoss/dlogits)
  float* g2 = sd + SPB * OUT;         // SPB x H   (dLoss/dpre2)
  float* g1 = g2 + SPB * H;           // SPB x H   (dLoss/dpre1)
  const int t = threadIdx.x;
  for (int i = t; i < NPARAM; i += SPB) w[i] = params[i];
  __syncthreads();
  const int n = blockIdx.x * SPB + t;
  const bool live = n < count;
  const int src = live ? (idx ? idx[n] : n) : 0;
  float lsum = 0.f;
  {
    float x[IN];
#pragma unroll
    for (int i = 0; i < IN; ++i) {
      x[i] = live ? X[(size_t)src * IN + i] : 0.f;
      sx[t * IN + i] = x[i];
    }
    for (int j = 0; j < H; ++j) {
      float a = w[OFF_B1 + j];
#pragma unroll
      for (int i = 0; i < IN; ++i) a = fmaf(x[i], w[OFF_W1 + i * H + j], a);
      s1[t * H + j] = fmaxf(a, 0.f);
    }
    for (int j = 0; j < H; ++j) {
      float a = w[OFF_B2 + j];
      for (int i = 0; i < H; ++i) a = fmaf(s1[t * H + i], w[OFF_W2 + i * H + j], a);
      s2[t * H + j] = fmaxf(a, 0.f);
    }
    float o[OUT];
    for (int j = 0; j < OUT; ++j) {
      float a = w[OFF_B3 + j];
      for (int i = 0; i < H; ++i) a = fmaf(s2[t * H + i], w[OFF_W3 + i * OUT + j], a);
      o[j] = a;
    }
    // softmax cross-entropy on both heads; d = (p - onehot) / batch
    for (int head = 0; head < 2; ++head) {
      const int b = head ? OS : 0, len = head ? OM : OS;
      const int label = head ? (live ? ym[src] - 2 : 0) : (live ? ys[src] : 0);
      float mx = -INFINITY;
      for (int j = 0; j < len; ++j) mx = fmaxf(mx, o[b + j]);
      float den = 0.f;
      for (int j = 0; j < len; ++j) den += __expf(o[b + j] - mx);
      for (int j = 0; j < len; ++j) {
        const float pj = __expf(o[b + j] - mx) / den;
        sd[t * OUT + b + j] = live ? (pj - (j == label ? 1.f : 0.f)) * inv_batch : 0.f;
      }
      if (live) lsum += logf(den) + mx - o[b + label];
    }
    for (int i = 0; i < H; ++i) {
      float a = 0.f;
      for (int j = 0; j < OUT; ++j) a = fmaf(sd[t * OUT + j], w[OFF_W3 + i * OUT + j], a);
      g2[t * H + i] = s2[t * H + i] > 0.f ? a : 0.f;
    }
    for (int i = 0; i < H; ++i) {
      float a = 0.f;
      for (int j = 0; j < H; ++j) a = fmaf(g2[t * H + j], w[OFF_W2 + i * H + j], a);
      g1[t * H + i] = s1[t * H + i] > 0.f ? a : 0.f;
    }
  }
  // block reduction of the loss
  for (int o = 16; o > 0; o >>= 1) lsum += __shfl_xor_sync(0xffffffffu, lsum, o);
  if ((t & 31) == 0) atomicAdd(loss_sum, lsum);
  __syncthreads();
  // weight gradients: one thread per parameter, summed over the block's samples
  for (int q = t; q < NPARAM; q += SPB) {
    float a = 0.f;
    if (q < OFF_B1) {
      const int i = q / H, j = q % H;
      for (int s = 0; s < SPB; ++s) a = fmaf(sx[s * IN + i], g1[s * H + j], a);
    } else if (q < OFF_W2) {
      const int j = q - OFF_B1;
      for (int s = 0; s < SPB; ++s) a += g1[s * H + j];
    } else if (q < OFF_B2) {
      const int i = (q - OFF_W2) / H, j = (q - OFF_W2) % H;
      for (int s = 0; s < SPB; ++s) a = fmaf(s1[s * H + i], g2[s * H + j], a);
    } else if (q < OFF_W3) {
      const int j = q - OFF_B2;
      for (int s = 0; s < SPB; ++s) a += g2[s * H + j];
    } else if (q < OFF_B3) {
      const int i = (q - OFF_W3) / OUT, j = (q - OFF_W3) % OUT;
      for (int s = 0; s < SPB; ++s) a = fmaf(s2[s * H + i], sd[s * OUT + j], a);
    } else {
      const int j = q - OFF_B3;
      for (int s = 0; s < SPB; ++s) a += sd[s * OUT + j];
    }
    atomicAdd(&grad[q], a);
  }
}

__global__ void adam_kernel(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m1,
                            float* __restrict__ m2, int n, float lr, float b1, float b2, float eps, float c1,
                            float c2) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const float gi = g[i];
    const float a = b1 * m1[i] + (1.f - b1) * gi;
    const float b = b2 * m2[i] + (1.f - b2) * gi * gi;
    m1[i] = a;
    m2[i] = b;
    p[i] -= lr * (a / c1) / (sqrtf(b / c2) + eps);
  }
}

size_t grad_smem() { return sizeof(float) * (NPARAM + SPB * (IN + 4 * H + OUT)); }

// process-wide trained model
std::mutex g_model_mu;
std::vector<float> g_model;

}  // namespace

int forward(const float* dparams, const float* dX, int count, float* dlogits, int* ds, int* dm, cudaStream_t st) {
  if (count <= 0) return PHIKRON_OK;
  launch_begin(KC_OTHER, st);
  mlp_forward_kernel<<<(count + SPB - 1) / SPB, SPB, 0, st>>>(dparams, dX, count, dlogits, ds, dm);
  launch_end(st);
  PK_CHECK_LAUNCH();
  return PHIKRON_OK;
}

int grad(const float* dparams, const float* dX, const int* dys, const int* dym, const int* didx, int count,
         float inv_batch, float* dgrad, float* dloss, cudaStream_t st) {
  if (count <= 0) return PHIKRON_OK;
  static bool attr = false;
  if (!attr) {
    PK_TRY_CUDA(cudaFuncSetAttribute(mlp_grad_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)grad_smem()));
    attr = true;
  }
  launch_begin(KC_OTHER, st);
  mlp_grad_kernel<<<(count + SPB - 1) / SPB, SPB, grad_smem(), st>>>(dparams, dX, dys, dym, didx, count, inv_batch,
                                                                     dgrad, dloss);
  launch_end(st);
  PK_CHECK_LAUNCH();
  return PHIKRON_OK;
}

int adam(float* dp, const float* dg, float* dm1, float* dm2, int step, float lr, cudaStream_t st) {
  const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
  const float c1 = 1.f - std::pow(b1, (float)step), c2 = 1.f - std::pow(b2, (float)step);
  launch_begin(KC_OTHER, st);
  adam_kernel<<<32, 256, 0, st>>>(dp, dg, dm1, dm2, NPARAM, lr, b1, b2, eps, c1, c2);
  launch_end(st);
  PK_CHECK_LAUNCH();
  return PHIKRON_OK;
}

bool model(std::vector<float>* out) {
  std::lock_guard<std::mutex> lk(g_model_mu);
  if ((int)g_model.size() != NPARAM) return false;
  *out = g_model;
  return true;
}

void set_model(const float* p) {
  std::lock_guard<std::mutex> lk(g_model_mu);
  g_model.assign(p, p + NPARAM);
}

}  // namespace mlp
}  // namespace phikron

using namespace phikron;

namespace {

template <typename T>
struct DevBuf {
  T* p = nullptr;
  ~DevBuf() {
    if (p) cudaFree(p);
  }
  int alloc(size_t n) {
    if (cudaMalloc(&p, sizeof(T) * std::max<size_t>(n, 1)) != cudaSuccess) {
      cudaGetLastError();
      p = nullptr;
      set_error("selector: device allocation failed");
      return PHIKRON_ENOMEM;
    }
    return PHIKRON_OK;
  }
};

}  // namespace

extern "C" {

int phikron_selector_param_count(void) { return mlp::NPARAM; }

int phikron_selector_set_model(const float* params, int n) {
  clear_error();
  if (!params || n != mlp::NPARAM) {
    set_error("phikron_selector_set_model: need phikron_selector_param_count() floats");
    return PHIKRON_EINVAL;
  }
  for (int i = 0; i < n; ++i)
    if (!std::isfinite(params[i])) {
      set_error("phikron_selector_set_model: non-finite parameter");
      return PHIKRON_EINVAL;
    }
  mlp::set_model(params);
  return PHIKRON_OK;
}

int phikron_selector_get_model(float* params, int n) {
  clear_error();
  std::vector<float> m;
  if (!params || n != mlp::NPARAM || !mlp::model(&m)) {
    set_error("phikron_selector_get_model: no model set, or wrong size");
    return PHIKRON_EINVAL;
  }
  std::memcpy(params, m.data(), sizeof(float) * n);
  return PHIKRON_OK;
}

int phikron_selector_forward(const float* params, const float* X, int count, float* logits, int* s, int* m,
                             void* stream) {
  clear_error();
  if (!params || !X || count < 0) {
    set_error("phikron_selector_forward: bad arguments");
    return PHIKRON_EINVAL;
  }
  return mlp::forward(params, X, count, logits, s, m, static_cast<cudaStream_t>(stream));
}

int phikron_selector_grad(const float* params, const float* X, const int* ys, const int* ym, int count, float* grad,
                          float* loss, void* stream) {
  clear_error();
  if (!params || !X || !ys || !ym || !grad || !loss || count <= 0) {
    set_error("phikron_selector_grad: bad arguments");
    return PHIKRON_EINVAL;
  }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  PK_TRY_CUDA(cudaMemsetAsync(grad, 0, sizeof(float) * mlp::NPARAM, st));
  PK_TRY_CUDA(cudaMemsetAsync(loss, 0, sizeof(float), st));
  return mlp::grad(params, X, ys, ym, nullptr, count, 1.0f / count, grad, loss, st);
}

int phikron_selector_train(const float* X_host, const int* ys_host, const int* ym_host, int count, int epochs,
                           int batch, float lr, unsigned seed, const float* init_params_host, float* params_out_host,
                           float* final_loss) {
  clear_error();
  if (!X_host || !ys_host || !ym_host || count < 1 || epochs < 1 || batch < 1 || !(lr > 0.f)) {
    set_error("phikron_selector_train: bad arguments");
    return PHIKRON_EINVAL;
  }
  for (int i = 0; i < count; ++i)
    if (ys_host[i] < 0 || ys_host[i] > 20 || ym_host[i] < 2 || ym_host[i] > 32) {
      set_error("phikron_selector_train: labels need s in 0..20 and m in 2..32");
      return PHIKRON_EINVAL;
    }
  const int NP = mlp::NPARAM;
  std::vector<float> p0(NP);
  if (init_params_host) {
    std::memcpy(p0.data(), init_params_host, sizeof(float) * NP);
  } else {  // He initialisation, zero biases
    std::mt19937 rng(seed);
    auto fill = [&](int off, int fan_in, int cnt) {
      std::normal_distribution<float> nd(0.f, std::sqrt(2.f / fan_in));
      for (int i = 0; i < cnt; ++i) p0[off + i] = nd(rng);
    };
    fill(mlp::OFF_W1, mlp::IN, mlp::IN * mlp::H);
    fill(mlp::OFF_W2, mlp::H, mlp::H * mlp::H);
    fill(mlp::OFF_W3, mlp::H, mlp::H * mlp::OUT);
  }
  DevBuf<float> dX, dp, dg, dm1, dm2, dl;
  DevBuf<int> dys, dym, didx;
  PK_RET(dX.alloc((size_t)count * mlp::IN));
  PK_RET(dys.alloc(count));
  PK_RET(dym.alloc(count));
  PK_RET(didx.alloc(count));
  PK_RET(dp.alloc(NP));
  PK_RET(dg.alloc(NP));
  PK_RET(dm1.alloc(NP));
  PK_RET(dm2.alloc(NP));
  PK_RET(dl.alloc(1));
  PK_TRY_CUDA(cudaMemcpy(dX.p, X_host, sizeof(float) * count * mlp::IN, cudaMemcpyHostToDevice));
  PK_TRY_CUDA(cudaMemcpy(dys.p, ys_host, sizeof(int) * count, cudaMemcpyHostToDevice));
  PK_TRY_CUDA(cudaMemcpy(dym.p, ym_host, sizeof(int) * count, cudaMemcpyHostToDevice));
  PK_TRY_CUDA(cudaMemcpy(dp.p, p0.data(), sizeof(float) * NP, cudaMemcpyHostToDevice));
  PK_TRY_CUDA(cudaMemset(dm1.p, 0, sizeof(float) * NP));
  PK_TRY_CUDA(cudaMemset(dm2.p, 0, sizeof(float) * NP));
  cudaStream_t st = nullptr;
  std::vector<int> perm(count);
  for (int i = 0; i < count; ++i) perm[i] = i;
  std::mt19937 rng(seed ^ 0x9e3779b9u);
  int step = 0;
  float last = 0.f;
  for (int ep = 0; ep < epochs; ++ep) {
    std::shuffle(perm.begin(), perm.end(), rng);
    PK_TRY_CUDA(cudaMemcpy(didx.p, perm.data(), sizeof(int) * count, cudaMemcpyHostToDevice));
    PK_TRY_CUDA(cudaMemsetAsync(dl.p, 0, sizeof(float), st));
    for (int b0 = 0; b0 < count; b0 += batch) {
      const int bn = std::min(batch, count - b0);
      PK_TRY_CUDA(cudaMemsetAsync(dg.p, 0, sizeof(float) * NP, st));
      PK_RET(mlp::grad(dp.p, dX.p, dys.p, dym.p, didx.p + b0, bn, 1.0f / bn, dg.p, dl.p, st));
      PK_RET(mlp::adam(dp.p, dg.p, dm1.p, dm2.p, ++step, lr, st));
    }
    PK_TRY_CUDA(cudaMemcpy(&last, dl.p, sizeof(float), cudaMemcpyDeviceToHost));
    last /= count;
  }
  std::vector<float> out(NP);
  PK_TRY_CUDA(cudaMemcpy(out.data(), dp.p, sizeof(float) * NP, cudaMemcpyDeviceToHost));
  for (float v : out)
    if (!std::isfinite(v)) {
      set_error("phikron_selector_train: training diverged (non-finite parameters)");
      return PHIKRON_ENOTCONVERGED;
    }
  mlp::set_model(out.data());
  if (params_out_host) std::memcpy(params_out_host, out.data(), sizeof(float) * NP);
  if (final_loss) *final_loss = last;
  return PHIKRON_OK;
}

}  // extern "C"
