// Launch sequences of the mixed-precision apply: one sequence runs Algorithm 1 + Algorithm 6
// (+ phi_0, + optional half-step outputs) for a set of "units" (one unit = one right-hand
// side of one plan), grouping every unit's work of a stage into one persistent launch.  The
// single-plan apply is a sequence of one unit; the batched apply groups all plans x RHS.
#pragma once

#include <vector>

#include "mixed.h"

namespace phikron {

struct Plan;

enum StepKind { STEP_MODE = 0, STEP_WEIGHTED = 1, STEP_SQUARING = 2, STEP_EXPSCAN = 3, STEP_FUSED = 4, STEP_PRECUT = 5 };

struct Step {
  int kind;
  size_t off;        // first job in the job table of its kind
  int count;         // jobs
  long long total;   // tiles (mode) or blocks (elementwise)
  int p;
  PassShape shape;
  long long tmap_off = -1;   // raw-ring mode pass: first tensor map (index) in Seq::dTmaps
};

struct Seq {
  std::vector<Step> steps;
  GJob* dG = nullptr;
  EJob* dE = nullptr;
  FJob* dF = nullptr;      // fused node passes: jobs and their nodes
  FNode* dFN = nullptr;
  uint8_t* dTmaps = nullptr;   // TMA tensor maps of the raw-ring passes' inputs (128 B each)
  bool fused = false;      // the node phase ends in a fused weighted pass
  int* dSlots = nullptr;
  int nslots = 0;
  void** dPtrtab = nullptr;
  int* dStatus = nullptr;
  int p = 0, ninst = 0;
  bool half = false;
  size_t njobs_mode = 0;
  cudaGraphExec_t exec = nullptr;
  unsigned long long wait_ns = 2000000000ull;  // limit of the kernels' bounded waits
  size_t device_bytes = 0;
  std::vector<void*> allocs;
  ~Seq();
};

struct SeqUnit {
  const Plan* plan;
  int inst, rhs;
  float2 *W1, *W2, *Y, *Yn;   // work buffers: W* hold max(m+2, p) vectors, Y* hold p
};

struct SeqConfig {
  bool half = false;      // also write phi_l(-tau/2 A) v (state before the last squaring)
  int slices = 5;
  int sub = 1;            // K chunk = 32*sub
  int grid = 148;         // CTAs per mode pass
  bool big_first = false; // order the jobs of a pass by decreasing tile count
  bool graph = true;      // capture the sequence as a CUDA graph
  bool ws = true;         // warp-specialised mode kernel
  bool db = false;        // double-buffered 128 x 64-tile mode kernel where every n >= 64
  bool fuse = true;       // fold Algorithm 1's weights into the last node pass where it applies
  bool rr = true;         // raw-ring warp-specialised kernel where it applies
};

struct MixedView {
  const uint8_t* sl;
  const int* rexp;
  size_t mat_bytes;
  int rexp_stride;
  const float2* coef;
  int slices, nsm;
};

// Mode-kernel variant when nothing is tuned: the warp-specialised kernel, unless the environment
// variable PHIKRON_MODE_KERNEL names another ("db": double-buffered 128 x 64 tiles where every
// contracted size is at least 64; "classic": the single-role kernel).
bool mode_kernel_ws_default();
bool mode_kernel_db_default();
// Fused node-weight pass where it applies if the environment variable PHIKRON_FUSED_WEIGHTS is
// "1" (measured slower than the separate passes on the 128^3 workload; see fused.cu).
bool fused_weights_default();
// Raw-ring mode kernel where it applies, unless PHIKRON_RAW_RING is "0".
bool raw_ring_default();

const MixedView mixed_view(const Plan& P, int d);
int seq_build(Seq& S, std::vector<SeqUnit>& units, int ninst, const SeqConfig& cfg);
int seq_launch_all(Seq& S, cudaStream_t st);
int seq_run(Seq& S, const PtrArgs& args, cudaStream_t st);
int seq_status(Seq& S, int* status);

}  // namespace phikron
