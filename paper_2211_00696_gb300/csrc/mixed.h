// Mixed-precision (split-BF16 tensor-core) apply path: shared declarations.
#pragma once

#include <cstdint>

#include "common.h"

namespace phikron {

// One mode product (Eq. (8)) of one vector by one matrix, see tc_mode.cu.  Inputs and outputs
// are either direct device pointers or (tab >= 0) a byte offset into an entry of the pass's
// device pointer table, which holds the caller's V / Out pointers of the current apply.
struct GJob {
  const void* in;          // float64 (pass shape in_f64) or float2 (hi, lo) vector
  const int* in_exp;       // e with |in| < 2^e for the whole vector
  const uint8_t* eslices;  // E as [row block][chunk32][slice][128 rows x 32 K bf16 core-matrix layout]
  const int* rexp;         // [row block][128] row exponents f_i of E (|E[i][k]| < 2^{f_i})
  void* out;               // float2 or float64 (out_f64)
  int* out_exp;            // receives the max exponent of out (atomicMax), or null
  long long R, B0;         // product of faster / slower axes than the contracted one
  long long tile_begin;    // first tile of this job in its pass
  long long tab_off_in, tab_off_out;  // byte offsets when in_tab / out_tab >= 0
  int n;                   // contracted size (E is n x n), multiple of 16, <= 4096
  int out_f64;
  int in_tab, out_tab;     // pointer-table entries, or -1
  const uint8_t* xslices;  // the input's digit slices, cut once for all jobs that share it
                           // ([128-fiber block][chunk32][slice] shared-memory images), or null
};

struct GPass {
  const GJob* jobs;        // device array, sorted by tile_begin
  int njobs;
  long long total_tiles;
  const void* const* ptrtab;
  unsigned long long wait_ns;  // limit of every bounded mbarrier wait (wall clock)
  const void* tmaps;       // raw-ring passes: one 128-byte TMA tensor map per job (its input)
};

struct PassShape {
  int slices;              // digit slices per operand (3..6)
  int sub;                 // K chunk = 32 * sub (1, or 2 with 3 slices)
  int grid;                // CTAs (persistent, 1 per SM at most)
  bool in_f64, trans;
  bool ws;                 // warp-specialised kernel (producer / MMA / epilogue warps)
  bool db;                 // double-buffered 128 x 64 tiles (needs n >= 64 in every job)
  bool rr;                 // raw-ring kernel (float-float input, every job's input 16-byte
                           // aligned and direct; <= 5 slices warp-specialised, <= 4 double-buffered)
  bool pc;                 // float64 first pass from pre-cut input slices (GJob::xslices)
};

// Shared-memory operand layout of one 128-row x 32-K BF16 slice (8 KiB), K-major, used by the
// host slicing of E and by the kernels' digit cutting and MMA descriptors: the 64-byte swizzle
// (8-row x 64-byte atoms of 512 B; the 16-byte chunk g of row r sits at chunk g ^ ((r >> 1) & 3)).
constexpr bool kSwizzle64 = true;
__host__ __device__ inline unsigned chunk_offset(int row, int g) {
  return kSwizzle64 ? (unsigned)(row * 64 + ((g ^ ((row >> 1) & 3)) * 16))
                    : (unsigned)((row >> 3) * 512 + g * 128 + (row & 7) * 16);
}

constexpr int MAX_PTRS = 128;
struct PtrArgs {
  void* p[MAX_PTRS];
  int n;
};

namespace tc {
int mode_pass(const GPass& P, const PassShape& S, int* status, cudaStream_t st);
int set_ptrtab(void** tab, const PtrArgs& args, cudaStream_t st);
// The digit slices of each job's float64 input (transposed first pass of a chain: B0 = 1),
// cut once into job.xslices in the shared-memory image the mode kernel's MMAs read
int precut_pass(const GPass& P, int slices, int* status, cudaStream_t st);
// bytes of a job's pre-cut slices
size_t precut_bytes(long long R, int n, int slices);
// TMA tensor maps (128 bytes each, job order) of the inputs of a raw-ring mode pass's jobs
// (boxes of `fibers` = 128 fibers for the warp-specialised kernel, 64 for the double-buffered one)
int encode_raw_maps(const GJob* jobs, int njobs, bool trans, int fibers, uint8_t* out);
size_t smem_bytes(int ks, int sub);
}  // namespace tc

// fibers per tile of a pass: 64 for the double-buffered kernel, 128 otherwise
inline long long tile_fibers(const PassShape& s) { return s.db ? 64 : 128; }

// Fused last mode pass of the node phase (fused.cu): for every output tile the kernel runs the
// last mode product of every node of its unit one after the other and folds the weighted ones
// into the p sums y_j = sum_k c_{j,k} T_k of Algorithm 1 (Sec. 3.1) in TMEM, so that the node
// products T_k never reach HBM; "direct" nodes (phi_0, and phi_0 at tau/2) are stored as they
// are.  Contraction over the fastest axis (R = 1), float-float inputs, n <= 128, p <= 4.
constexpr int FW_MAXP = 4;     // weighted outputs a fused pass holds in TMEM
constexpr int FW_MAXN = 128;   // contracted size (one E row block)

struct FNode {
  const float2* in;        // the node's input vector (float-float)
  const int* in_exp;       // e with |in| < 2^e
  const uint8_t* eslices;  // E sliced as for GJob (n <= 128: one row block)
  const int* rexp;         // the 128 row exponents of E
  void* out;               // direct node: float64 output vector (or table entry + offset)
  long long tab_off_out;
  int out_tab;             // -1: `out` is a direct pointer
  int direct;              // 1: store the product; 0: weighted node `k`
  int k;
  int pad_;
};

struct FJob {
  long long B0;            // fibers (product of the slower axes)
  long long tile_begin;    // first tile (32 fibers) of this job in its pass
  int n;                   // contracted size (multiple of 16, <= FW_MAXN)
  int node0, nnodes;       // nodes [node0, node0 + nnodes): the m weighted ones first
  int m;                   // weighted nodes (columns of coef)
  const float2* coef;      // p x m float-float weights, (j-1)*m + k
  void* out;               // y_j at out + (j-1)*stride elements: float2, or float64 (out_f64)
  void* out2;              // optional float64 copy of y_j (half-step outputs), or null
  long long stride, tab_off_out, tab_off_out2;
  int out_tab, out2_tab;   // pointer-table entries, or -1
  int out_f64;
  int pad_;
  int* out_exp;            // p exponent slots (float2 outputs), or null
};

struct FPass {
  const FJob* jobs;        // device array, sorted by tile_begin
  const FNode* nodes;      // device array
  int njobs;
  long long total_tiles;
  const void* const* ptrtab;
  unsigned long long wait_ns;
};

namespace fused {
// Runs one fused pass with `slices` digit slices and p weighted outputs on `grid` CTAs.
int launch(const FPass& P, int slices, int p, int grid, int* status, cudaStream_t st);
// Fibers per tile of a fused pass.
constexpr int kFibers = 32;
}  // namespace fused

// Grouped float-float elementwise jobs (mixed.cu): weighted sums of Algorithm 1, modified
// squaring of Eq. (29), and the exponent scan of a float64 input.
struct EJob {
  const float2* a;         // weighted: T (m vectors); squaring: Z (p vectors)
  const float2* b;         // squaring: Y (p vectors); unused for weighted sums
  const float2* coef;      // weighted: p x m float-float coefficients
  const double* v;         // exponent scan: float64 input (or table)
  void* out;               // p vectors (float2), or float64 (out_f64)
  void* out2;              // optional float64 copy (half-step outputs), or null
  int* out_exp;            // p slots (float2 outputs), or null
  long long N, stride;     // vector length; stride between consecutive vectors of a/b/out/out2
  long long block_begin;   // first block of this job in its launch
  long long tab_off_out, tab_off_out2, tab_off_v;
  int m;
  int out_f64;
  int out_tab, out2_tab, v_tab;
  int pad_;
};

}  // namespace phikron
