// K1: batched float64 matrix exponential exp(c_b * A_b) by Pade [13/13] scaling and
// squaring (Higham, SIAM J. Matrix Anal. Appl. 26 (2005), the published method).
//
// The paper needs 1D exponentials exp((1 - x_k) 2^{-s} M^d) at every quadrature node and
// exp(2^{t-s} M^d) for the squaring steps (Algorithm 6; Eq. (7)-(8)), and leaves the
// algorithm for them unspecified (MATLAB's expm).  Here:
//   * Pade coefficients come from the closed form b_j = (2m-j)! m! / ((2m)! j! (m-j)!),
//     evaluated by the ratio b_j/b_{j-1} = (m-j+1)/((2m-j+1) j) with b_0 = 1 (any common
//     factor cancels in (V-U)^{-1}(V+U)).
//   * theta_13 = 5.371920351148152 is the published backward-error threshold for m = 13.
//   * Degree 13 for every matrix and a squaring count per matrix,
//     s_b = max(0, ceil(log2(eta_b/theta_13))), where eta_b = |c_b| ||A_b||_1 comes from the
//     host, so no device round trip is needed to choose them.  The batch is processed in
//     descending order of s_b, so the matrices still being squared at step t form a prefix
//     and each squaring is one batched GEMM over that prefix.
//   * Every contraction runs on the FP64 GEMM; (V-U) R = V+U is solved with one CTA per
//     matrix by Gaussian elimination with partial pivoting.
#include <algorithm>
#include <cmath>
#include <vector>

#include "common.h"

namespace phikron {

namespace {

constexpr double kTheta13 = 5.371920351148152;
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
    out[off + i] = sc.s[bl] * in[ioff + i];
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
    if (X0) v = fma(c0, X0[e], v);
    if (X1) v = fma(c1, X1[e], v);
    if (X2) v = fma(c2, X2[e], v);
    if (X3) v = fma(c3, X3[e], v);
    const long long w = e % nn;
    if ((w / n) == (w % n)) v += cI;
    out[e] = v;
  }
}

// P <- V - U, Q <- V + U (batched)
__global__ void pq_kernel(const double* __restrict__ U, const double* __restrict__ V,
                          double* __restrict__ P, double* __restrict__ Q, long long total) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const double u = U[e], v = V[e];
    P[e] = v - u;
    Q[e] = v + u;
  }
}

// Solve P X = Q in place (X overwrites Q) for one n x n system per CTA, Gaussian
// elimination with partial pivoting followed by back substitution.
__global__ void __launch_bounds__(256) lu_solve_kernel(double* __restrict__ Pall,
                                                       double* __restrict__ Qall, int n) {
  double* P = Pall + (long long)blockIdx.x * n * n;
  double* Q = Qall + (long long)blockIdx.x * n * n;
  __shared__ double red_v[256];
  __shared__ int red_i[256];
  __shared__ int piv_s;
  const int tid = threadIdx.x, nt = blockDim.x;
  for (int k = 0; k < n; ++k) {
    double best = -1.0;
    int bi = k;
    for (int i = k + tid; i < n; i += nt) {
      const double a = fabs(P[(long long)i * n + k]);
      if (a > best) { best = a; bi = i; }
    }
    red_v[tid] = best;
    red_i[tid] = bi;
    __syncthreads();
    for (int o = nt / 2; o > 0; o >>= 1) {
      if (tid < o) {
        if (red_v[tid + o] > red_v[tid] ||
            (red_v[tid + o] == red_v[tid] && red_i[tid + o] < red_i[tid])) {
          red_v[tid] = red_v[tid + o];
          red_i[tid] = red_i[tid + o];
        }
      }
      __syncthreads();
    }
    if (tid == 0) piv_s = red_i[0];
    __syncthreads();
    const int piv = piv_s;
    if (piv != k) {
      for (int j = tid; j < n; j += nt) {
        double t = P[(long long)k * n + j];
        P[(long long)k * n + j] = P[(long long)piv * n + j];
        P[(long long)piv * n + j] = t;
        t = Q[(long long)k * n + j];
        Q[(long long)k * n + j] = Q[(long long)piv * n + j];
        Q[(long long)piv * n + j] = t;
      }
    }
    __syncthreads();
    const double inv = 1.0 / P[(long long)k * n + k];
    for (int i = k + 1 + tid; i < n; i += nt) P[(long long)i * n + k] *= inv;
    __syncthreads();
    const int rows = n - k - 1;
    const int wp = n - k - 1;  // P columns k+1..n-1
    const long long work = (long long)rows * (wp + n);
    for (long long e = tid; e < work; e += nt) {
      const int r = static_cast<int>(e / (wp + n));
      const int c = static_cast<int>(e % (wp + n));
      const int i = k + 1 + r;
      const double l = P[(long long)i * n + k];
      if (c < wp) {
        const int j = k + 1 + c;
        P[(long long)i * n + j] -= l * P[(long long)k * n + j];
      } else {
        const int j = c - wp;
        Q[(long long)i * n + j] -= l * Q[(long long)k * n + j];
      }
    }
    __syncthreads();
  }
  for (int k = n - 1; k >= 0; --k) {
    const double inv = 1.0 / P[(long long)k * n + k];
    for (int j = tid; j < n; j += nt) Q[(long long)k * n + j] *= inv;
    __syncthreads();
    const long long work = (long long)k * n;
    for (long long e = tid; e < work; e += nt) {
      const int i = static_cast<int>(e / n), j = static_cast<int>(e % n);
      Q[(long long)i * n + j] -= P[(long long)i * n + k] * Q[(long long)k * n + j];
    }
    __syncthreads();
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
  return (size_t)9 * (size_t)count * (size_t)n * (size_t)n * sizeof(double);
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
    sp[b] = (e > kTheta13) ? static_cast<int>(std::ceil(std::log2(e / kTheta13))) : 0;
    sp_max = std::max(sp_max, sp[b]);
    order[b] = b;
  }
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return sp[a] > sp[b]; });

  // Pade [13/13] coefficients b_0..b_13 with b_0 = 1
  double bc[14];
  bc[0] = 1.0;
  for (int j = 1; j <= 13; ++j) bc[j] = bc[j - 1] * (13.0 - j + 1.0) / ((26.0 - j + 1.0) * j);

  const long long nn = (long long)n * n;
  const long long total = nn * count;
  double* w = static_cast<double*>(ws);
  double* B = w;
  double* B2 = w + total;
  double* B4 = w + 2 * total;
  double* B6 = w + 3 * total;
  double* T1 = w + 4 * total;
  double* U = w + 5 * total;
  double* V = w + 6 * total;
  double* P = w + 7 * total;
  double* Q = w + 8 * total;

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
  PK_RET(bgemm(B2, B2, B4, count, n, 0.0, st));
  PK_RET(bgemm(B4, B2, B6, count, n, 0.0, st));
  // U = B * (B6*(b13 B6 + b11 B4 + b9 B2) + b7 B6 + b5 B4 + b3 B2 + b1 I)
  lincomb_kernel<<<g, 256, 0, st>>>(T1, B6, B4, B2, nullptr, bc[13], bc[11], bc[9], 0.0, 0.0, n, total);
  PK_CHECK_LAUNCH();
  lincomb_kernel<<<g, 256, 0, st>>>(V, B6, B4, B2, nullptr, bc[7], bc[5], bc[3], 0.0, bc[1], n, total);
  PK_CHECK_LAUNCH();
  PK_RET(bgemm(B6, T1, V, count, n, 1.0, st));  // V holds the bracket for U
  PK_RET(bgemm(B, V, U, count, n, 0.0, st));
  // V = B6*(b12 B6 + b10 B4 + b8 B2) + b6 B6 + b4 B4 + b2 B2 + b0 I
  lincomb_kernel<<<g, 256, 0, st>>>(T1, B6, B4, B2, nullptr, bc[12], bc[10], bc[8], 0.0, 0.0, n, total);
  PK_CHECK_LAUNCH();
  lincomb_kernel<<<g, 256, 0, st>>>(V, B6, B4, B2, nullptr, bc[6], bc[4], bc[2], 0.0, bc[0], n, total);
  PK_CHECK_LAUNCH();
  PK_RET(bgemm(B6, T1, V, count, n, 1.0, st));
  pq_kernel<<<g, 256, 0, st>>>(U, V, P, Q, total);
  PK_CHECK_LAUNCH();
  lu_solve_kernel<<<count, 256, 0, st>>>(P, Q, n);
  PK_CHECK_LAUNCH();
  // undo the scaling: R <- R^2, s_b times; matrices with s_b > t form the prefix of length
  // cnt(t), squared by one batched GEMM while the others stay where they are
  double* bufs[2] = {Q, T1};
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
