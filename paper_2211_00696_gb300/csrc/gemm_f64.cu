// Float64 building blocks on the DFMA pipe: a strided batched GEMM, the mode product of
// Eq. (8) built on it, the node-weighted sums of Algorithm 1 and the modified squaring
// combination of Eq. (29) / Algorithm 6.
//
// GB300 executes float64 at ~1.2 TFLOP/s (about 2 DFMA per clock per SM), so every
// float64 contraction here is bound by the FP64 pipe, not by memory: a 64x64 register
// tile with a 16-deep shared-memory K stage keeps the pipe busy with ample margin
// (arithmetic intensity 8 flop per staged byte against a pipe that needs < 1).
#include <cstdio>

#include "checked.cuh"
#include "common.h"
#include "profile.h"

PK_CHK_BIND(gemm_f64)

namespace phikron {

namespace {

using chk::ld_ck;
using chk::st_ck;

constexpr int BM = 64, BN = 64, BK = 16, NT = 256;

__global__ void __launch_bounds__(NT) gemm_f64_kernel(GemmF64 g, int tiles_n, long long nbatch) {
  __shared__ double As[BK][BM + 1];
  __shared__ double Bs[BK][BN + 1];
  const int tid = threadIdx.x;
  const int tx = tid & 15, ty = tid >> 4;
  const int tm = blockIdx.x / tiles_n, tn = blockIdx.x % tiles_n;
  const long long z = (long long)blockIdx.y + (long long)gridDim.y * blockIdx.z;
  if (z >= nbatch) return;
  const long long b = z / g.nb0, i0 = z % g.nb0;
  const double* A = g.A + b * g.sAb + i0 * g.sAi0;
  const double* B = g.B + b * g.sBb + i0 * g.sBi0;
  double* C = g.C + b * g.sCb + i0 * g.sCi0;
  const int m0 = tm * BM, n0 = tn * BN;

  double acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = 0.0;

  const bool a_k_fast = (g.sAk == 1);
  const bool b_n_fast = (g.sBn == 1);
  for (int k0 = 0; k0 < g.K; k0 += BK) {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int e = tid + NT * q;
      int ii, kk;
      if (a_k_fast) { ii = e / BK; kk = e % BK; } else { kk = e / BM; ii = e % BM; }
      const int gi = m0 + ii, gk = k0 + kk;
      As[kk][ii] = (gi < g.M && gk < g.K) ? ld_ck(A + gi * g.sAm + gk * g.sAk, chk::SITE_F64_LOAD) : 0.0;
      int jj, kb;
      if (b_n_fast) { kb = e / BN; jj = e % BN; } else { jj = e / BK; kb = e % BK; }
      const int gj = n0 + jj, gkb = k0 + kb;
      Bs[kb][jj] = (gj < g.N && gkb < g.K) ? ld_ck(B + gkb * g.sBk + gj * g.sBn, chk::SITE_F64_LOAD) : 0.0;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      double a[4], bv[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[kk][ty + 16 * i];
#pragma unroll
      for (int j = 0; j < 4; ++j) bv[j] = Bs[kk][tx + 16 * j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fma(a[i], bv[j], acc[i][j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int gi = m0 + ty + 16 * i;
    if (gi >= g.M) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int gj = n0 + tx + 16 * j;
      if (gj >= g.N) continue;
      double* c = C + gi * g.sCm + gj * g.sCn;
      const double v = g.alpha * acc[i][j];
      if (PK_CK(c, sizeof(double), chk::SITE_F64_STORE)) *c = (g.beta == 0.0) ? v : fma(g.beta, *c, v);
    }
  }
}

__global__ void weighted_sum_kernel(const double* __restrict__ T, long long T_stride,
                                    const double* __restrict__ coef, int p, int m, long long N,
                                    double* __restrict__ Y, long long Y_stride) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N;
       i += (long long)gridDim.x * blockDim.x) {
    double acc[20];
#pragma unroll
    for (int j = 0; j < 20; ++j) acc[j] = 0.0;
    for (int k = 0; k < m; ++k) {
      const double t = ld_ck(T + k * T_stride + i, chk::SITE_F64_LOAD);
#pragma unroll
      for (int j = 0; j < 20; ++j)
        if (j < p) acc[j] = fma(ld_ck(coef + j * m + k, chk::SITE_F64_LOAD), t, acc[j]);
    }
#pragma unroll
    for (int j = 0; j < 20; ++j)
      if (j < p) st_ck(Y + j * Y_stride + i, acc[j], chk::SITE_F64_STORE);
  }
}

__device__ __forceinline__ double inv_factorial(int k) {
  double f = 1.0;
  for (int q = 2; q <= k; ++q) f *= q;
  return 1.0 / f;
}

__global__ void squaring_combine_kernel(const double* __restrict__ Z, const double* __restrict__ Y,
                                        double* __restrict__ Yn, int p, long long N, long long stride) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N;
       i += (long long)gridDim.x * blockDim.x) {
    double y[20];
#pragma unroll
    for (int j = 0; j < 20; ++j)
      if (j < p) y[j] = ld_ck(Y + j * stride + i, chk::SITE_F64_LOAD);
    double scale = 1.0;
#pragma unroll
    for (int q = 1; q <= 20; ++q) {
      if (q > p) break;
      scale *= 0.5;
      double acc = ld_ck(Z + (q - 1) * stride + i, chk::SITE_F64_LOAD);
      for (int j = 1; j <= q; ++j) acc = fma(y[j - 1], inv_factorial(q - j), acc);
      st_ck(Yn + (q - 1) * stride + i, scale * acc, chk::SITE_F64_STORE);
    }
  }
}

int grid_for(long long N, int threads) {
  long long b = (N + threads - 1) / threads;
  if (b > 152LL * 32) b = 152LL * 32;
  if (b < 1) b = 1;
  return static_cast<int>(b);
}

}  // namespace

int gemm_f64(const GemmF64& g, cudaStream_t st) {
  if (g.M <= 0 || g.N <= 0 || g.nb <= 0 || g.nb0 <= 0) return PHIKRON_OK;
  const int tiles_m = (g.M + BM - 1) / BM, tiles_n = (g.N + BN - 1) / BN;
  const long long nbatch = (long long)g.nb * g.nb0;
  const long long tiles = (long long)tiles_m * tiles_n;
  if (tiles > 0x7fffffffLL) {
    set_error("gemm_f64: too many tiles");
    return PHIKRON_EINVAL;
  }
  dim3 grid((unsigned)tiles, (unsigned)(nbatch < 65535 ? nbatch : 65535),
            (unsigned)((nbatch + 65534) / 65535));
  if (g.K <= 0) {
    // empty contraction: C = beta*C (only beta == 0 is used by callers)
  }
  launch_begin(KC_GEMM_F64, st);
  gemm_f64_kernel<<<grid, NT, 0, st>>>(g, tiles_n, nbatch);
  launch_end(st);
  PK_CHECK_LAUNCH();
  return PHIKRON_OK;
}

int mode_product_f64(const double* in, long long in_sb, double* out, long long out_sb,
                     const double* E, long long E_sb, int nbatch, long long B0, int n,
                     long long R, cudaStream_t st) {
  GemmF64 g{};
  g.alpha = 1.0;
  g.beta = 0.0;
  g.nb = nbatch;
  if (R > 1) {
    // out_{b,i0} (n x R) = E_b (n x n) * in_{b,i0} (n x R)
    g.A = E; g.sAb = E_sb; g.sAi0 = 0; g.sAm = n; g.sAk = 1;
    g.B = in; g.sBb = in_sb; g.sBi0 = (long long)n * R; g.sBk = R; g.sBn = 1;
    g.C = out; g.sCb = out_sb; g.sCi0 = (long long)n * R; g.sCm = R; g.sCn = 1;
    g.M = n; g.N = static_cast<int>(R); g.K = n;
    if (B0 > 0x7fffffffLL) return PHIKRON_EINVAL;
    g.nb0 = static_cast<int>(B0);
  } else {
    // out_b (B0 x n) = in_b (B0 x n) * E_b^T
    if (B0 > 0x7fffffffLL) return PHIKRON_EINVAL;
    g.A = in; g.sAb = in_sb; g.sAi0 = 0; g.sAm = n; g.sAk = 1;
    g.B = E; g.sBb = E_sb; g.sBi0 = 0; g.sBk = 1; g.sBn = n;
    g.C = out; g.sCb = out_sb; g.sCi0 = 0; g.sCm = n; g.sCn = 1;
    g.M = static_cast<int>(B0); g.N = n; g.K = n;
    g.nb0 = 1;
  }
  return gemm_f64(g, st);
}

int weighted_sum_f64(const double* T, long long T_stride, const double* coef, int p, int m,
                     long long N, double* Y, long long Y_stride, cudaStream_t st) {
  if (p < 1 || p > 20) {
    set_error("weighted_sum_f64: p must be in 1..20");
    return PHIKRON_EINVAL;
  }
  launch_begin(KC_WEIGHTED, st);
  weighted_sum_kernel<<<grid_for(N, 256), 256, 0, st>>>(T, T_stride, coef, p, m, N, Y, Y_stride);
  launch_end(st);
  PK_CHECK_LAUNCH();
  return PHIKRON_OK;
}

int squaring_combine_f64(const double* Z, const double* Y, double* Yn, int p, long long N,
                         long long stride, cudaStream_t st) {
  if (p < 1 || p > 20) {
    set_error("squaring_combine_f64: p must be in 1..20");
    return PHIKRON_EINVAL;
  }
  launch_begin(KC_SQUARING, st);
  squaring_combine_kernel<<<grid_for(N, 256), 256, 0, st>>>(Z, Y, Yn, p, N, stride);
  launch_end(st);
  PK_CHECK_LAUNCH();
  return PHIKRON_OK;
}

}  // namespace phikron
