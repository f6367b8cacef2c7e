// Internal declarations shared by the phikron translation units (not part of the C ABI).
#pragma once

#include <cstddef>
#include <cstdint>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/phikron.h"

namespace phikron {

// ----------------------------------------------------------------------------- errors
void set_error(const std::string& msg);
void clear_error();

#define PK_TRY_CUDA(call)                                                                  \
  do {                                                                                     \
    cudaError_t e_ = (call);                                                               \
    if (e_ != cudaSuccess) {                                                               \
      ::phikron::set_error(std::string(#call) + ": " + cudaGetErrorString(e_));            \
      return PHIKRON_ECUDA;                                                                \
    }                                                                                      \
  } while (0)

#define PK_CHECK_LAUNCH()                                                                  \
  do {                                                                                     \
    cudaError_t e_ = cudaGetLastError();                                                   \
    if (e_ != cudaSuccess) {                                                               \
      ::phikron::set_error(std::string("kernel launch: ") + cudaGetErrorString(e_));       \
      return PHIKRON_ECUDA;                                                                \
    }                                                                                      \
  } while (0)

#define PK_RET(call)                                                                       \
  do {                                                                                     \
    int r_ = (call);                                                                       \
    if (r_ != PHIKRON_OK) return r_;                                                       \
  } while (0)

// ----------------------------------------------------------------------------- allocation
// Every device buffer of plans, sequences, batches and integrators comes from device_malloc,
// and every library object from a host allocation that first asks alloc_fault(): both fail
// with PHIKRON_ENOMEM (and a message naming `who`) when the allocation is refused.  Fault
// injection for tests of the failure paths: with the environment variable
// PHIKRON_FAIL_ALLOC_AFTER = k set, the library's allocations after the first k (counted from
// the moment the variable took that value) are refused.
bool alloc_fault();
int device_malloc(void** p, size_t bytes, const char* who);
// Frees a buffer from device_malloc (null is ignored); the library's count of live device
// buffers (phikron_live_device_buffers) follows both.
void device_free(void* p);

// true if the address ranges [a, a + n) and [b, b + n) of n float64 share an element
inline bool ranges_overlap(const void* a, const void* b, long long n) {
  const uintptr_t x = reinterpret_cast<uintptr_t>(a), y = reinterpret_cast<uintptr_t>(b);
  const uintptr_t len = static_cast<uintptr_t>(n) * sizeof(double);
  return x < y + len && y < x + len;
}

// ----------------------------------------------------------------------------- planner
namespace planner {
int log_quaderr(double n, int p, double alpha, double beta, int rule, double* out);
int quadnodes(double eps, int p, double alpha, double beta, int rule, int* n);
int setup_quadrature(double eps, int p, double alpha, double beta, int rule, int* s, int* m,
                     int* cost);
int gauss_legendre(int m, double* x, double* w);
int clenshaw_curtis(int n, double* x, double* w);
}  // namespace planner

// ----------------------------------------------------------------------------- selector
namespace selector {
double criterion(double zlo, double zhi, int p, int s, int m, int npts);
int search(double zlo, double zhi, int p, double tol, int npts, int* s, int* m, int* cost);
}  // namespace selector
namespace mlp {
int forward(const float* dparams, const float* dX, int count, float* dlogits, int* ds, int* dm, cudaStream_t st);
bool model(std::vector<float>* out);
}  // namespace mlp
// 8 selector features: log10(tau ||A^d||_inf) (d = 1..3; -6 for a missing axis), log2(n_d)/8,
// l_max/4, -log10(tol)/10
void selector_features(int dims, const int* n, const double* tau_norm_inf, int p, double tol, float* out);

// ----------------------------------------------------------------------------- fp64 GEMM
// C[z](i, j) = alpha * sum_k A[z](i, k) * B[z](k, j) + beta * C[z](i, j), where the batch
// index z = b * nb0 + i0 selects base offsets b*s?b + i0*s?i0 and the element (i, k) of A
// sits at A[offset + i*sAm + k*sAk] (likewise B, C).  All strides in elements.
struct GemmF64 {
  const double* A; long long sAb, sAi0; long long sAm, sAk;
  const double* B; long long sBb, sBi0; long long sBk, sBn;
  double* C;       long long sCb, sCi0; long long sCm, sCn;
  int M, N, K;
  int nb, nb0;
  double alpha, beta;
};
int gemm_f64(const GemmF64& g, cudaStream_t st);

// Mode-d product of a batch of tensors (Eq. (8) as a Tucker/mode product):
//   out[b][i0][i][r] = sum_k E_b[i][k] * in[b][i0][k][r],  i, k < n, i0 < B0, r < R.
// in/out/E of batch b at in + b*in_sb, out + b*out_sb, E + b*E_sb (E_sb may be 0).
int mode_product_f64(const double* in, long long in_sb, double* out, long long out_sb,
                     const double* E, long long E_sb, int nbatch, long long B0, int n,
                     long long R, cudaStream_t st);

// ----------------------------------------------------------------------------- expm (K1)
size_t expm_workspace_bytes(int count, int n);
int expm_batched(int count, int n, const double* A, const double* scale_host,
                 const double* norms1_host, double* E, void* ws, cudaStream_t st);

// ----------------------------------------------------------------------------- combine (K3)
// Y[j][i] = sum_k coef[j*m + k] * T[k][i]   (j < p, k < m, i < N), coef on the DEVICE.
int weighted_sum_f64(const double* T, long long T_stride, const double* coef, int p, int m,
                     long long N, double* Y, long long Y_stride, cudaStream_t st);
// Modified squaring step (Eq. (29)), i = 1..p:
//   Yn[i-1] = 2^{-i} (Z[i-1] + sum_{j=1}^{i} Y[j-1] / (i-j)!)
int squaring_combine_f64(const double* Z, const double* Y, double* Yn, int p, long long N,
                         long long stride, cudaStream_t st);

}  // namespace phikron
