// Per-kernel CUDA-event timing and launch counting for the apply path.
//
// An apply installs its plan's Profiler as the thread's current one; every kernel launch
// site brackets its launch with launch_begin/launch_end.  Launches are always counted;
// when timing is enabled a pair of events is recorded on the launch stream around the
// kernel, so the measured interval is that kernel's execution on its own stream.
#pragma once

#include <cuda_runtime.h>

#include <vector>

#include "../../include/phikron.h"

namespace phikron {

enum KernelClass {
  KC_GEMM_F64 = 0,     // float64 mode products (DFMA)
  KC_WEIGHTED = 1,     // node-weighted sums (Algorithm 1)
  KC_SQUARING = 2,     // modified squaring combination (Eq. (29))
  KC_TC_MODE = 3,      // tensor-core mode products (tcgen05)
  KC_CONVERT = 4,      // precision conversions / splits
  KC_OTHER = 5,
  KC_COUNT = 6
};

struct Profiler {
  bool timing = false;
  long long launches = 0;
  long long launches_by_class[KC_COUNT] = {0, 0, 0, 0, 0, 0};
  std::vector<cudaEvent_t> ev;    // 2 per recorded launch
  std::vector<int> cls;
  size_t used = 0;                // recorded launches
  ~Profiler() {
    for (cudaEvent_t e : ev) cudaEventDestroy(e);
  }
};

extern thread_local Profiler* tl_prof;

// Starts counting (and, for max_timed > 0, timing the first max_timed) launches; profiler_end
// adds the counts and the summed event times per class to *out and stops timing.
int profiler_begin(Profiler& pr, int max_timed);
int profiler_end(Profiler& pr, struct ::phikron_profile* out);

inline void launch_begin(int c, cudaStream_t st) {
  Profiler* p = tl_prof;
  if (!p) return;
  p->launches++;
  p->launches_by_class[c]++;
  if (p->timing && p->used < p->cls.size()) {
    cudaEventRecord(p->ev[2 * p->used], st);
    p->cls[p->used] = c;
  }
}

inline void launch_end(cudaStream_t st) {
  Profiler* p = tl_prof;
  if (!p || !p->timing || p->used >= p->cls.size()) return;
  cudaEventRecord(p->ev[2 * p->used + 1], st);
  p->used++;
}

struct ProfScope {
  Profiler* prev;
  explicit ProfScope(Profiler* p) : prev(tl_prof) { tl_prof = p; }
  ~ProfScope() { tl_prof = prev; }
};

}  // namespace phikron
