// K1: batched float64 matrix exponential exp(c_b * A_b) by Taylor scaling and squaring, with
// the degree-18 Taylor polynomial evaluated by the Paterson-Stockmeyer scheme (GEMMs only).
//
// The paper needs 1D exponentials exp((1 - x_k) 2^{-s} M^d) at every quadrature node and
// exp(2^{t-s} M^d) for the squaring steps (Algorithm 6; Eq. (7)-(8)), and leaves the
// algorithm for them unspecified (MATLAB's expm).  Here:
//   * B = 2^{-s_b} c_b A_b with s_b = max(0, ceil(log2 ||c_b A_b||_1)), so ||B||_1 <= 1.  The
//     Taylor remainder of degree 18 then obeys ||R(B)|| <= e ||B||^19/19! <= 2.3e-17, and
//     ||e^B|| >= e^{-1}, so the truncation is below the float64 unit roundoff relative to the
//     result; the s_b squarings follow.
//   * T18(B) = C0 + B4 (C1 + B4 (C2 + B4 (C3 + B4 C4))) with C_j = sum_{i<4} B^i/(4j+i)!
//     (C4 = I/16! + B/17! + B^2/18!): B^2, B^3, B^4 and four Horner products, 7 GEMMs.
//   * s_b comes from the host-side norm, so no device round trip is needed.  The batch is
//     processed in descending order of s_b, so the matrices still being squared at step t
//     form a prefix and each squaring is one batched GEMM over that prefix.
//   * There is no linear solve (a Pade denominator solve is sequential in n and, with one CTA
//     per matrix, dominated plan time for n >= 1024).
#include <algorithm>
#include <cmath>
#include <vector>

#include "checked.cuh"
#include "common.h"

PK_CHK_BIND(expm)

namespace phikron {

namespace {

constexpr double kTheta = 1.0;  // ||B||_1 bound for the degree-18 Taylor polynomial
constexpr int kDeg = 18;
constexpr int kChunk = 256;

struct ScaleArgs {
  double s[kChunk];
  int src[kChunk];
};

// out[b0 + j] = scale[j] * in[src[j]] for j < count  (gather into the processing order)
__global__ void scale_batch_kernel(const double* __restrict__ in, double* __restrict__ out,
                                   long long nn, int b0, int count, ScaleArgs sc) {
  const int bl = blockIdx.y;
  if (bl >= count) return;
  const long long off = (long long)(b0 + bl) * nn;
  const long long ioff = (long long)sc.src[bl] * nn;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < nn;
       i += (long long)gridDim.x * blockDim.x)
    chk::st_ck(out + off + i, sc.s[bl] * chk::ld_ck(in + ioff + i, chk::SITE_PLAN), chk::SITE_PLAN);
}

// out = c0*X0 + c1*X1 + c2*X2 + c3*X3 + cI*I  (batched; null X with zero coefficient skipped)
__global__ void lincomb_kernel(double* __restrict__ out, const double* __restrict__ X0,
                               const double* __restrict__ X1, const double* __restrict__ X2,
                               const double* __restrict__ X3, double c0, double c1, double c2,
                               double c3, double cI, int n, long long total) {
  const long long nn = (long long)n * n;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    double v = 0.0;
    if (X0) v = fma(c0, chk::ld_ck(X0 + e, chk::SITE_PLAN), v);
    if (X1) v = fma(c1, chk::ld_ck(X1 + e, chk::SITE_PLAN), v);
    if (X2) v = fma(c2, chk::ld_ck(X2 + e, chk::SITE_PLAN), v);
    if (X3) v = fma(c3, chk::ld_ck(X3 + e, chk::SITE_PLAN), v);
    const long long w = e % nn;
    if ((w / n) == (w % n)) v += cI;
    chk::st_ck(out + e, v, chk::SITE_PLAN);
  }
}

int ew_grid(long long total) {
  long long b = (total + 255) / 256;
  return static_cast<int>(std::max(1LL, std::min(b, 152LL * 16)));
}

// C = A*B (+ beta*C) for `count` contiguous n x n row-major matrices
int bgemm(const double* A, const double* B, double* C, int count, int n, double beta,
          cudaStream_t st) {
  GemmF64 g{};
  const long long nn = (long long)n * n;
  g.A = A; g.sAb = nn; g.sAi0 = 0; g.sAm = n; g.sAk = 1;
  g.B = B; g.sBb = nn; g.sBi0 = 0; g.sBk = n; g.sBn = 1;
  g.C = C; g.sCb = nn; g.sCi0 = 0; g.sCm = n; g.sCn = 1;
  g.M = n; g.N = n; g.K = n; g.nb = count; g.nb0 = 1;
  g.alpha = 1.0; g.beta = beta;
  return gemm_f64(g, st);
}

}  // namespace

size_t expm_workspace_bytes(int count, int n) {
  return (size_t)6 * (size_t)count * (size_t)n * (size_t)n * sizeof(double);
}

int expm_batched(int count, int n, const double* A, const double* scale_host,
                 const double* norms1_host, double* E, void* ws, cudaStream_t st) {
  if (count <= 0) return PHIKRON_OK;
  if (n < 1 || !A || !E || !ws || !scale_host || !norms1_host) {
    set_error("expm_batched: bad arguments");
    return PHIKRON_EINVAL;
  }
  std::vector<int> sp(count), order(count);
  int sp_max = 0;
  for (int b = 0; b < count; ++b) {
    const double e = std::fabs(scale_host[b]) * norms1_host[b];
    if (!std::isfinite(e)) {
      set_error("expm_batched: non-finite norm or scale");
      return PHIKRON_EINVAL;
    }
    sp[b] = (e > kTheta) ? static_cast<int>(std::ceil(std::log2(e / kTheta))) : 0;
    sp_max = std::max(sp_max, sp[b]);
    order[b] = b;
  }
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return sp[a] > sp[b]; });

  // 1/k!, k = 0..18
  double inv[kDeg + 1];
  inv[0] = 1.0;
  for (int k = 1; k <= kDeg; ++k) inv[k] = inv[k - 1] / k;

  const long long nn = (long long)n * n;
  const long long total = nn * count;
  double* w = static_cast<double*>(ws);
  double* B = w;
  double* B2 = w + total;
  double* B3 = w + 2 * total;
  double* B4 = w + 3 * total;
  double* H = w + 4 * total;
  double* T1 = w + 5 * total;

  for (int b0 = 0; b0 < count; b0 += kChunk) {
    const int c = std::min(kChunk, count - b0);
    ScaleArgs sa;
    for (int i = 0; i < c; ++i) {
      const int src = order[b0 + i];
      sa.s[i] = scale_host[src] * std::ldexp(1.0, -sp[src]);
      sa.src[i] = src;
    }
    dim3 grid(static_cast<unsigned>(std::min<long long>((nn + 255) / 256, 1024)), c);
    scale_batch_kernel<<<grid, 256, 0, st>>>(A, B, nn, b0, c, sa);
    PK_CHECK_LAUNCH();
  }
  const int g = ew_grid(total);
  PK_RET(bgemm(B, B, B2, count, n, 0.0, st));
  PK_RET(bgemm(B2, B, B3, count, n, 0.0, st));
  PK_RET(bgemm(B2, B2, B4, count, n, 0.0, st));
  // H = C4 = I/16! + B/17! + B^2/18!
  lincomb_kernel<<<g, 256, 0, st>>>(H, B, B2, nullptr, nullptr, inv[17], inv[18], 0.0, 0.0, inv[16], n, total);
  PK_CHECK_LAUNCH();
  // H <- C_j + B4 H for j = 3, 2, 1, 0 (C_j preloaded into the destination, beta = 1)
  double* cur = H;
  double* nxt = T1;
  for (int j = 3; j >= 0; --j) {
    lincomb_kernel<<<g, 256, 0, st>>>(nxt, B, B2, B3, nullptr, inv[4 * j + 1], inv[4 * j + 2], inv[4 * j + 3], 0.0,
                                      inv[4 * j], n, total);
    PK_CHECK_LAUNCH();
    PK_RET(bgemm(B4, cur, nxt, count, n, 1.0, st));
    std::swap(cur, nxt);
  }
  // undo the scaling: R <- R^2, s_b times; matrices with s_b > t form the prefix of length
  // cnt(t), squared by one batched GEMM while the others stay where they are
  double* bufs[2] = {cur, nxt};
  for (int t = 0; t < sp_max; ++t) {
    int cnt = 0;
    while (cnt < count && sp[order[cnt]] > t) ++cnt;
    PK_RET(bgemm(bufs[t & 1], bufs[t & 1], bufs[(t + 1) & 1], cnt, n, 0.0, st));
  }
  for (int i = 0; i < count; ++i) {
    const int b = order[i];
    PK_TRY_CUDA(cudaMemcpyAsync(E + (long long)b * nn, bufs[sp[b] & 1] + (long long)i * nn,
                                nn * sizeof(double), cudaMemcpyDeviceToDevice, st));
  }
  return PHIKRON_OK;
}

}  // namespace phikron
