// Mixed-precision (split-BF16 tensor-core) apply path: shared declarations.
#pragma once

#include <cstdint>

#include "common.h"

namespace phikron {

// One mode product of a pass: out = E x_d in (Eq. (8)), see tc_mode.cu.
struct ModeJob {
  const void* in;          // float64 (pass.in_f64) or float2 (hi, lo) vector(s)
  const int* in_exp;       // e with |in| < 2^e for the whole vector
  const uint8_t* eslices;  // E as [chunk][slice][128 rows x 32 K bf16, core-matrix layout]
  const int* rexp;         // per-row exponents f_i of E (|E[i][k]| < 2^{f_i})
  void* out;               // float2 or float64 (out_f64)
  int* out_exp;            // receives max exponent of out (atomicMax), or null
  int out_f64;
  int pad_;
};

constexpr int MAX_MODE_JOBS = 24;

struct ModePass {
  ModeJob jobs[MAX_MODE_JOBS];
  int njobs;
  int n;            // size of the contracted axis (E is n x n)
  long long R;      // product of the faster axes (1 for the fastest axis)
  long long B0;     // product of the slower axes
  int in_f64;       // inputs are float64 (else float-float)
};

namespace tc {
int mode_pass(const ModePass& P, int slices, int* status, int nsm, cudaStream_t st);
}

// float-float elementwise kernels (mixed.cu)
// Y_j = sum_k coef[j][k] T_k (float-float coefficients on the device), j < p, k < m.
int ff_weighted_sum(const float2* T, long long T_stride, const float2* coef, int p, int m, long long N,
                    void* Y, long long Y_stride, int out_f64, int* out_exp, cudaStream_t st);
// Yn_i = 2^{-i}(Z_i + sum_{j<=i} Y_j/(i-j)!), i = 1..p  (Eq. (29)).
int ff_squaring_combine(const float2* Z, const float2* Y, void* Yn, int p, long long N, long long stride,
                        int out_f64, int* out_exp, cudaStream_t st);
// slot = e with |v| < 2^e over a float64 vector (integer ops only).
int f64_exponent(const double* v, long long N, int* slot, cudaStream_t st);

// Host: cut an n x n float64 matrix into `slices` BF16 digit slices in the kernel's layout.
// out: nchunks*slices*8192 bytes; rexp: 128 ints (rows >= n get 0).
void slice_matrix_host(const double* E, int n, int slices, uint8_t* out, int* rexp);
size_t sliced_bytes(int n, int slices);

}  // namespace phikron
