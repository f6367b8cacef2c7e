// Mixed-precision apply path (PHIKRON_PREC_OZAKI_BF16): plan-time slicing of the 1D
// exponentials, float-float elementwise kernels, and the orchestration of Algorithm 1 +
// the modified squaring of Eq. (29) on top of the tensor-core mode products (tc_mode.cu).
//
// State vectors between passes are float-float pairs (hi, lo) of FP32 (~48-bit
// significand), 8 bytes per unknown like float64, so every buffer of the float64 plan is
// reused.  Node weights, the squaring recurrence and the final float64 outputs are formed
// with compensated FP32 arithmetic (two-sum / FMA two-product) and integer bit assembly:
// no float64 instruction runs per element, because GB300's float64 rate is ~1/64 of FP32.
// Each kernel that writes a state vector also records an exponent e with |v| < 2^e
// (atomicMax over the vector), which the next mode product uses to cut its digits.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "mixed.h"
#include "plan.h"
#include "profile.h"

namespace phikron {

namespace {

constexpr int KC = 32;
constexpr int SLICE_BYTES = 128 * KC * 2;

__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = a + b;
  const float bb = s - a;
  e = (a - (s - bb)) + (b - bb);
}

__device__ __forceinline__ void fast_two_sum(float a, float b, float& s, float& e) {
  s = a + b;
  e = b - (s - a);
}

// acc += c * t  in float-float
__device__ __forceinline__ void ff_fma(float2& acc, float2 c, float2 t) {
  const float p = c.x * t.x;
  float pe = fmaf(c.x, t.x, -p);
  pe = fmaf(c.x, t.y, pe);
  pe = fmaf(c.y, t.x, pe);
  float s, e;
  two_sum(acc.x, p, s, e);
  e += acc.y + pe;
  fast_two_sum(s, e, acc.x, acc.y);
}

// acc += t
__device__ __forceinline__ void ff_add(float2& acc, float2 t) {
  float s, e;
  two_sum(acc.x, t.x, s, e);
  e += acc.y + t.y;
  fast_two_sum(s, e, acc.x, acc.y);
}

// float-float -> float64 by integer assembly of the 53-bit significand (no float64 ops).
// Requires |lo| <= ulp(hi)/2 (normalised pair).
__device__ __forceinline__ double ff_to_f64(float hi, float lo) {
  const uint32_t bh = __float_as_uint(hi);
  const int eh = (int)((bh >> 23) & 0xFF);
  if (eh == 0) return 0.0;
  uint64_t M = (uint64_t)((bh & 0x7FFFFFu) | 0x800000u) << 29;  // 53-bit significand of hi
  int E = eh - 127 + 1023;
  const uint32_t bl = __float_as_uint(lo);
  const int el = (int)((bl >> 23) & 0xFF);
  if (el != 0) {
    const uint64_t ml = (uint64_t)((bl & 0x7FFFFFu) | 0x800000u);
    const int sh = el - eh + 29;  // lo in units of hi's 53-bit ulp
    uint64_t L;
    if (sh >= 0)
      L = ml << sh;
    else if (sh > -40)
      L = (ml + (1ull << (-sh - 1))) >> (-sh);
    else
      L = 0;
    if (((bh ^ bl) >> 31) == 0) {
      M += L;
      if (M >> 53) {  // carry (cannot happen for normalised pairs; kept for safety)
        M >>= 1;
        ++E;
      }
    } else {
      M -= L;
      while (M && !(M >> 52)) {
        M <<= 1;
        --E;
      }
    }
  }
  const uint64_t bits = ((uint64_t)(bh >> 31) << 63) | ((uint64_t)E << 52) | (M & 0xFFFFFFFFFFFFFull);
  return __longlong_as_double((long long)bits);
}

__device__ __forceinline__ int exp_plus1(float x) { return (int)((__float_as_uint(x) >> 23) & 0xFF) - 126; }

__device__ __forceinline__ void warp_max_atomic(int v, int* slot) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = max(v, __shfl_xor_sync(0xffffffffu, v, o));
  if ((threadIdx.x & 31) == 0 && slot && v > -1000) atomicMax(slot, v);
}

constexpr int MAXP = 20;

template <int P_, bool OUT_F64>
__global__ void ff_weighted_sum_kernel(const float2* __restrict__ T, long long T_stride,
                                       const float2* __restrict__ coef, int m, long long N,
                                       void* __restrict__ Y, long long Y_stride, int* __restrict__ out_exp) {
  extern __shared__ float2 cs[];  // P_ * m coefficients
  for (int i = threadIdx.x; i < P_ * m; i += blockDim.x) cs[i] = coef[i];
  __syncthreads();
  int emax[P_];
#pragma unroll
  for (int j = 0; j < P_; ++j) emax[j] = -1000;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N;
       i += (long long)gridDim.x * blockDim.x) {
    float2 acc[P_];
#pragma unroll
    for (int j = 0; j < P_; ++j) acc[j] = make_float2(0.f, 0.f);
    for (int k = 0; k < m; ++k) {
      const float2 t = T[k * T_stride + i];
#pragma unroll
      for (int j = 0; j < P_; ++j) ff_fma(acc[j], cs[j * m + k], t);
    }
#pragma unroll
    for (int j = 0; j < P_; ++j) {
      if (OUT_F64)
        reinterpret_cast<double*>(Y)[j * Y_stride + i] = ff_to_f64(acc[j].x, acc[j].y);
      else
        reinterpret_cast<float2*>(Y)[j * Y_stride + i] = acc[j];
      if (acc[j].x != 0.f) emax[j] = max(emax[j], exp_plus1(acc[j].x));
    }
  }
  if (!OUT_F64) {
#pragma unroll
    for (int j = 0; j < P_; ++j) warp_max_atomic(emax[j], out_exp ? out_exp + j : nullptr);
  }
}

struct InvFact {
  float2 f[MAXP + 1];  // 1/k! as float-float
};

template <int P_, bool OUT_F64>
__global__ void ff_squaring_kernel(const float2* __restrict__ Z, const float2* __restrict__ Y,
                                   void* __restrict__ Yn, long long N, long long stride,
                                   int* __restrict__ out_exp, InvFact inv) {
  int emax[P_];
#pragma unroll
  for (int j = 0; j < P_; ++j) emax[j] = -1000;
  for (long long x = blockIdx.x * (long long)blockDim.x + threadIdx.x; x < N;
       x += (long long)gridDim.x * blockDim.x) {
    float2 y[P_];
#pragma unroll
    for (int j = 0; j < P_; ++j) y[j] = Y[j * stride + x];
    float sc = 1.0f;
#pragma unroll
    for (int q = 1; q <= P_; ++q) {
      sc *= 0.5f;
      float2 acc = Z[(q - 1) * stride + x];
#pragma unroll
      for (int j = 1; j <= q; ++j) {
        const int d = q - j;
        if (d <= 1)
          ff_add(acc, y[j - 1]);
        else
          ff_fma(acc, inv.f[d], y[j - 1]);
      }
      acc.x *= sc;
      acc.y *= sc;
      if (OUT_F64)
        reinterpret_cast<double*>(Yn)[(q - 1) * stride + x] = ff_to_f64(acc.x, acc.y);
      else
        reinterpret_cast<float2*>(Yn)[(q - 1) * stride + x] = acc;
      if (acc.x != 0.f) emax[q - 1] = max(emax[q - 1], exp_plus1(acc.x));
    }
  }
  if (!OUT_F64) {
#pragma unroll
    for (int j = 0; j < P_; ++j) warp_max_atomic(emax[j], out_exp ? out_exp + j : nullptr);
  }
}

__global__ void f64_exponent_kernel(const double* __restrict__ v, long long N, int* __restrict__ slot) {
  int e = -1000;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N;
       i += (long long)gridDim.x * blockDim.x) {
    const uint64_t b = (uint64_t)__double_as_longlong(v[i]);
    const int ex = (int)((b >> 52) & 0x7FF);
    if (ex != 0) e = max(e, ex - 1022);  // |x| < 2^{ex - 1023 + 1}
  }
  warp_max_atomic(e, slot);
}

int ew_grid(long long N) {
  long long b = (N + 255) / 256;
  return (int)std::max(1LL, std::min(b, 152LL * 8));
}

template <int P_>
int launch_ws(const float2* T, long long Ts, const float2* coef, int m, long long N, void* Y, long long Ys,
              int out_f64, int* out_exp, cudaStream_t st) {
  const size_t sm = sizeof(float2) * P_ * m;
  launch_begin(KC_WEIGHTED, st);
  if (out_f64)
    ff_weighted_sum_kernel<P_, true><<<ew_grid(N), 256, sm, st>>>(T, Ts, coef, m, N, Y, Ys, out_exp);
  else
    ff_weighted_sum_kernel<P_, false><<<ew_grid(N), 256, sm, st>>>(T, Ts, coef, m, N, Y, Ys, out_exp);
  launch_end(st);
  PK_CHECK_LAUNCH();
  return PHIKRON_OK;
}

template <int P_>
int launch_sq(const float2* Z, const float2* Y, void* Yn, long long N, long long stride, int out_f64,
              int* out_exp, const InvFact& inv, cudaStream_t st) {
  launch_begin(KC_SQUARING, st);
  if (out_f64)
    ff_squaring_kernel<P_, true><<<ew_grid(N), 256, 0, st>>>(Z, Y, Yn, N, stride, out_exp, inv);
  else
    ff_squaring_kernel<P_, false><<<ew_grid(N), 256, 0, st>>>(Z, Y, Yn, N, stride, out_exp, inv);
  launch_end(st);
  PK_CHECK_LAUNCH();
  return PHIKRON_OK;
}

InvFact make_invfact() {
  InvFact r;
  double f = 1.0;
  for (int k = 0; k <= MAXP; ++k) {
    if (k > 1) f *= k;
    const double v = 1.0 / f;
    const float hi = (float)v;
    r.f[k] = make_float2(hi, (float)(v - (double)hi));
  }
  return r;
}

}  // namespace

#define PK_DISPATCH_P(p, CALL)                                                                     \
  switch (p) {                                                                                     \
    case 1: { constexpr int PP = 1; return CALL; }                                                 \
    case 2: { constexpr int PP = 2; return CALL; }                                                 \
    case 3: { constexpr int PP = 3; return CALL; }                                                 \
    case 4: { constexpr int PP = 4; return CALL; }                                                 \
    case 5: { constexpr int PP = 5; return CALL; }                                                 \
    case 6: { constexpr int PP = 6; return CALL; }                                                 \
    case 7: { constexpr int PP = 7; return CALL; }                                                 \
    case 8: { constexpr int PP = 8; return CALL; }                                                 \
    default: set_error("mixed path: l_max must be <= 8"); return PHIKRON_ENOTSUP;                  \
  }

int ff_weighted_sum(const float2* T, long long T_stride, const float2* coef, int p, int m, long long N,
                    void* Y, long long Y_stride, int out_f64, int* out_exp, cudaStream_t st) {
  PK_DISPATCH_P(p, launch_ws<PP>(T, T_stride, coef, m, N, Y, Y_stride, out_f64, out_exp, st));
}

int ff_squaring_combine(const float2* Z, const float2* Y, void* Yn, int p, long long N, long long stride,
                        int out_f64, int* out_exp, cudaStream_t st) {
  static const InvFact inv = make_invfact();
  PK_DISPATCH_P(p, launch_sq<PP>(Z, Y, Yn, N, stride, out_f64, out_exp, inv, st));
}

int f64_exponent(const double* v, long long N, int* slot, cudaStream_t st) {
  launch_begin(KC_CONVERT, st);
  f64_exponent_kernel<<<ew_grid(N), 256, 0, st>>>(v, N, slot);
  launch_end(st);
  PK_CHECK_LAUNCH();
  return PHIKRON_OK;
}

// ----------------------------------------------------------------------------- host slicing

size_t sliced_bytes(int n, int slices) {
  const int nchunks = (n + KC - 1) / KC;
  return (size_t)nchunks * slices * SLICE_BYTES;
}

void slice_matrix_host(const double* E, int n, int slices, uint8_t* out, int* rexp) {
  const int nchunks = (n + KC - 1) / KC;
  std::memset(out, 0, sliced_bytes(n, slices));
  for (int i = 0; i < 128; ++i) rexp[i] = 0;
  for (int i = 0; i < n; ++i) {
    double mx = 0.0;
    for (int k = 0; k < n; ++k) mx = std::max(mx, std::fabs(E[(size_t)i * n + k]));
    int f = 0;
    if (mx > 0.0) {
      std::frexp(mx, &f);  // mx = frac * 2^f, frac in [0.5, 1) -> mx < 2^f
    }
    rexp[i] = f;
    for (int k = 0; k < n; ++k) {
      const double x = E[(size_t)i * n + k];
      const double a = std::ldexp(std::fabs(x), 64 - f);  // in [0, 2^64)
      uint64_t F = (a >= 18446744073709551616.0) ? ~0ull : (uint64_t)a;
      const uint64_t half = 1ull << (63 - 8 * slices);  // round to nearest at the last digit
      F = (F > ~0ull - half) ? ~0ull : F + half;
      const int c = k / KC, kk = k % KC;
      const size_t off = (size_t)(i >> 3) * 512 + (size_t)(kk >> 3) * 128 + (size_t)(i & 7) * 16 +
                         (size_t)(kk & 7) * 2;
      for (int s = 0; s < slices; ++s) {
        const int t = s + 1;
        const uint32_t d = (uint32_t)((F >> (64 - 8 * t)) & 0xFFu);
        const float v = std::ldexp((float)d, -8 * t) * (x < 0 ? -1.0f : 1.0f);
        uint32_t bits;
        std::memcpy(&bits, &v, 4);
        const uint16_t bf = (uint16_t)(bits >> 16);
        uint8_t* dst = out + ((size_t)c * slices + s) * SLICE_BYTES + off;
        std::memcpy(dst, &bf, 2);
      }
    }
  }
}

// ----------------------------------------------------------------------------- plan state

struct MixedState {
  int slices = 5;
  int nsm = 148;
  uint8_t* dSl[3] = {nullptr, nullptr, nullptr};  // per unique factor: nexp matrices
  int* dRexp[3] = {nullptr, nullptr, nullptr};
  size_t mat_bytes[3] = {0, 0, 0};
  float2* dCoefFF = nullptr;
  int* dSlots = nullptr;
  int nslots = 0;
  int* dStatus = nullptr;
};

static void mixed_free(void* p) { delete static_cast<MixedState*>(p); }

int precision_setup(Plan& P) {
  if (P.opts.precision == PHIKRON_PREC_FP64) return PHIKRON_OK;
  if (P.opts.precision != PHIKRON_PREC_OZAKI_BF16) {
    set_error("precision mode not supported");
    return PHIKRON_ENOTSUP;
  }
  for (int d = 0; d < P.dims; ++d) {
    if (P.n[d] < 16 || P.n[d] > 128 || P.n[d] % 16 != 0) {
      set_error("mixed path: every n[d] must be a multiple of 16 in 16..128");
      return PHIKRON_ENOTSUP;
    }
  }
  if (P.p > 8) {
    set_error("mixed path: l_max must be <= 8");
    return PHIKRON_ENOTSUP;
  }
  MixedState* M = new MixedState();
  P.mixed = M;
  P.mixed_free = mixed_free;
  int slices = P.opts.slices;
  if (slices <= 0) {
    slices = (P.tol >= 1e-5) ? 3 : (P.tol >= 1e-7) ? 4 : (P.tol >= 1e-10) ? 5 : 6;
  }
  if (slices < 3 || slices > 6) {
    set_error("mixed path: slices must be 3..6");
    return PHIKRON_EINVAL;
  }
  M->slices = slices;
  int dev = 0;
  PK_TRY_CUDA(cudaGetDevice(&dev));
  PK_TRY_CUDA(cudaDeviceGetAttribute(&M->nsm, cudaDevAttrMultiProcessorCount, dev));

  // slice every 1D exponential (plan time, host)
  for (int u = 0; u < P.nuniq; ++u) {
    const int nd = P.n[P.uniq_rep[u]];
    const size_t nn = (size_t)nd * nd;
    std::vector<double> h(nn * P.nexp);
    PK_TRY_CUDA(cudaMemcpy(h.data(), P.dExp[u], sizeof(double) * nn * P.nexp, cudaMemcpyDeviceToHost));
    const size_t mb = sliced_bytes(nd, slices);
    std::vector<uint8_t> sl(mb * P.nexp);
    std::vector<int> rx(128 * P.nexp);
    for (int e = 0; e < P.nexp; ++e) slice_matrix_host(h.data() + nn * e, nd, slices, sl.data() + mb * e, rx.data() + 128 * e);
    PK_RET(P.alloc((void**)&M->dSl[u], sl.size()));
    PK_RET(P.alloc((void**)&M->dRexp[u], sizeof(int) * rx.size()));
    PK_TRY_CUDA(cudaMemcpy(M->dSl[u], sl.data(), sl.size(), cudaMemcpyHostToDevice));
    PK_TRY_CUDA(cudaMemcpy(M->dRexp[u], rx.data(), sizeof(int) * rx.size(), cudaMemcpyHostToDevice));
    M->mat_bytes[u] = mb;
  }
  // node weights as float-float
  std::vector<float2> cf(P.coef.size());
  for (size_t i = 0; i < P.coef.size(); ++i) {
    const float hi = (float)P.coef[i];
    cf[i] = make_float2(hi, (float)(P.coef[i] - (double)hi));
  }
  PK_RET(P.alloc((void**)&M->dCoefFF, sizeof(float2) * std::max<size_t>(1, cf.size())));
  if (!cf.empty())
    PK_TRY_CUDA(cudaMemcpy(M->dCoefFF, cf.data(), sizeof(float2) * cf.size(), cudaMemcpyHostToDevice));
  // exponent slots: v + per pass per vector + Y + per squaring step
  const int nv = std::max(P.m + 1, std::max(P.p, 1));
  M->nslots = 1 + 3 * nv + P.p + P.s * (3 * P.p + P.p) + 16;
  PK_RET(P.alloc((void**)&M->dSlots, sizeof(int) * M->nslots));
  PK_RET(P.alloc((void**)&M->dStatus, sizeof(int)));
  PK_TRY_CUDA(cudaMemset(M->dStatus, 0, sizeof(int)));
  return PHIKRON_OK;
}

namespace {

struct ChainVec {
  const void* in;       // input of the first pass
  int in_slot;          // slot index of the input exponent
  int mat;              // matrix index e in the per-factor exponential arrays
  void* out;            // final destination
  bool out_f64;         // final destination is float64
  int out_slot;         // slot index for the final output exponent (-1: none)
};

// Kronecker action (x)_d E_d on a batch of vectors, one pass per axis (Eq. (8)).
int kron_chain_mixed(Plan& P, MixedState& M, const std::vector<ChainVec>& vecs, bool first_in_f64,
                     float2* bufA, float2* bufB, int& slot_next, cudaStream_t st) {
  const long long N = P.N;
  const int nvec = (int)vecs.size();
  std::vector<int> cur_slot(nvec);
  for (int j = 0; j < nvec; ++j) cur_slot[j] = vecs[j].in_slot;
  for (int d = 0; d < P.dims; ++d) {
    long long B0 = 1, R = 1;
    for (int q = 0; q < d; ++q) B0 *= P.n[q];
    for (int q = d + 1; q < P.dims; ++q) R *= P.n[q];
    const int u = P.uniq_of[d];
    const bool last = (d == P.dims - 1);
    float2* dstbuf = (d % 2 == 0) ? bufA : bufB;
    const float2* srcbuf = (d % 2 == 0) ? bufB : bufA;
    for (int j0 = 0; j0 < nvec; j0 += MAX_MODE_JOBS) {
      ModePass pass{};
      pass.n = P.n[d];
      pass.R = R;
      pass.B0 = B0;
      pass.in_f64 = (d == 0) ? (first_in_f64 ? 1 : 0) : 0;
      const int cnt = std::min(MAX_MODE_JOBS, nvec - j0);
      pass.njobs = cnt;
      for (int q = 0; q < cnt; ++q) {
        const int j = j0 + q;
        ModeJob& J = pass.jobs[q];
        J.in = (d == 0) ? vecs[j].in : (const void*)(srcbuf + (size_t)j * N);
        J.in_exp = M.dSlots + cur_slot[j];
        J.eslices = M.dSl[u] + M.mat_bytes[u] * (size_t)vecs[j].mat;
        J.rexp = M.dRexp[u] + 128 * vecs[j].mat;
        if (last) {
          J.out = vecs[j].out;
          J.out_f64 = vecs[j].out_f64 ? 1 : 0;
          J.out_exp = (vecs[j].out_slot >= 0) ? M.dSlots + vecs[j].out_slot : nullptr;
        } else {
          J.out = dstbuf + (size_t)j * N;
          J.out_f64 = 0;
          J.out_exp = M.dSlots + slot_next + j;
        }
      }
      PK_RET(tc::mode_pass(pass, M.slices, M.dStatus, M.nsm, st));
    }
    if (!last) {
      for (int j = 0; j < nvec; ++j) cur_slot[j] = slot_next + j;
      slot_next += nvec;
    }
  }
  return PHIKRON_OK;
}

}  // namespace

int apply_mixed(Plan& P, const double* V, double* Out, cudaStream_t st) {
  MixedState& M = *static_cast<MixedState*>(P.mixed);
  const long long N = P.N;
  const int p = P.p, m = P.m, s = P.s;
  float2* W1 = reinterpret_cast<float2*>(P.dW1);
  float2* W2 = reinterpret_cast<float2*>(P.dW2);
  float2* Y = reinterpret_cast<float2*>(P.dY);
  float2* Yn = reinterpret_cast<float2*>(P.dYn);
  PK_TRY_CUDA(cudaMemsetAsync(M.dSlots, 0x80, sizeof(int) * M.nslots, st));
  PK_RET(f64_exponent(V, N, M.dSlots + 0, st));
  int slot_next = 1;
  // chain buffers: the last pass writes the chain's destination, so intermediates must
  // avoid it; with dims passes the intermediates alternate bufA (d even) / bufB (d odd).
  // node phase destination for the m node actions: W1 when dims is odd (last pass d=dims-1
  // even -> writes bufA... ) -- choose the pair so the destination is never an input.
  std::vector<ChainVec> vecs;
  if (p == 0) {
    vecs.push_back({V, 0, m, Out, true, -1});
    return kron_chain_mixed(P, M, vecs, true, W1, W2, slot_next, st);
  }
  // node actions (k < m) to T, phi_0 (matrix index m = exp(M^d)) straight to Out[0]
  // intermediates: d=0 -> bufA, d=1 -> bufB, final (d = dims-1) -> destination.
  // dims = 3: bufA = W1, bufB = W2, destination T = W1 (read from W2 in the last pass).
  // dims = 2: bufA = W1, destination T = W2 (read from W1).
  float2* T = (P.dims == 3) ? W1 : W2;
  const int slotT = slot_next;
  slot_next += m;
  for (int k = 0; k < m; ++k) vecs.push_back({V, 0, k, T + (size_t)k * N, false, slotT + k});
  vecs.push_back({V, 0, m, Out, true, -1});
  PK_RET(kron_chain_mixed(P, M, vecs, true, W1, W2, slot_next, st));
  // weighted sums over the nodes (Algorithm 1, second step)
  const int slotY = slot_next;
  slot_next += p;
  if (s == 0) {
    return ff_weighted_sum(T, N, M.dCoefFF, p, m, N, Out + N, N, 1, nullptr, st);
  }
  PK_RET(ff_weighted_sum(T, N, M.dCoefFF, p, m, N, Y, N, 0, M.dSlots + slotY, st));
  int ycur = slotY;
  for (int t = 0; t < s; ++t) {
    // Z_i = (x)_d G_{t,d} y_i, i = 1..p
    std::vector<ChainVec> zv;
    float2* Z = (P.dims == 3) ? W1 : W2;
    for (int i = 0; i < p; ++i) zv.push_back({Y + (size_t)i * N, ycur + i, m + 1 + t, Z + (size_t)i * N, false, -1});
    PK_RET(kron_chain_mixed(P, M, zv, false, W1, W2, slot_next, st));
    const bool last = (t == s - 1);
    const int slotYn = slot_next;
    slot_next += p;
    if (last) {
      PK_RET(ff_squaring_combine(Z, Y, Out + N, p, N, N, 1, nullptr, st));
    } else {
      PK_RET(ff_squaring_combine(Z, Y, Yn, p, N, N, 0, M.dSlots + slotYn, st));
      std::swap(Y, Yn);
      ycur = slotYn;
    }
  }
  if (slot_next > M.nslots) {
    set_error("mixed path: exponent slot overflow");
    return PHIKRON_EINVAL;
  }
  return PHIKRON_OK;
}

int mixed_slices(const Plan& P) { return static_cast<const MixedState*>(P.mixed)->slices; }

int mixed_status(Plan& P, int* status) {
  if (!P.mixed) {
    *status = 0;
    return PHIKRON_OK;
  }
  MixedState& M = *static_cast<MixedState*>(P.mixed);
  PK_TRY_CUDA(cudaMemcpy(status, M.dStatus, sizeof(int), cudaMemcpyDeviceToHost));
  PK_TRY_CUDA(cudaMemset(M.dStatus, 0, sizeof(int)));
  return PHIKRON_OK;
}

}  // namespace phikron
