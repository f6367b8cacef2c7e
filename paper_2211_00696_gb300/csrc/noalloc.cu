// phikron_kron_apply_f64_noalloc: phikron_kron_apply_f64 without a caller-provided work
// buffer and without any device allocation.
//
// Who needs this: callers that must not allocate device memory at call time -- a host
// framework that owns every byte of device memory through its own pool and forbids raw
// cudaMalloc, or a latency-critical loop where cudaMalloc/cudaFree would add an implicit
// device synchronisation.  Such callers still pass their inputs and outputs; the
// intermediate between mode products lives in a fixed array that the library embeds.
//
// The scratch is a file-scope __device__ array of kMaxElems float64 (8 MiB).  Every GPU
// that loads the library holds it until the process exits.  In host code the array's name
// is only a host-side stand-in, so its device address is looked up once per device with
// cudaGetSymbolAddress (with that device current) on the first call made on that device.
// That first call is a warm-up: with lazy module loading it is the call that loads the
// library's device code (and so creates the array) on that device, which can allocate and
// synchronise; make it before any stream capture and outside latency-critical loops.  Later
// calls allocate nothing.  The address is cached per device ordinal for the life of the
// process: cudaDeviceReset (which destroys the context that holds the array) is not
// supported between calls.  All calls share the one array and it keeps whatever the
// previous call wrote; the mode-product chain writes every scratch element before reading
// it, so nothing needs clearing.  Calls whose executions overlap on the GPU (different
// streams, or different host threads) race on the array: serialise them.  V and Out must
// not overlap (PHIKRON_EINVAL).
#include <mutex>

#include "checked.cuh"
#include "common.h"

namespace phikron {
namespace {

constexpr long long kMaxElems = 1LL << 20;  // 1,048,576 float64 = 8 MiB
__device__ __align__(256) double g_scratch[kMaxElems];

constexpr int kMaxDevices = 64;
double* g_scratch_dev[kMaxDevices] = {};
std::mutex g_scratch_mu;

int scratch_address(double** out) {
  int dev = -1;
  PK_TRY_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) {
    set_error("phikron_kron_apply_f64_noalloc: device ordinal out of range");
    return PHIKRON_EINVAL;
  }
  std::lock_guard<std::mutex> lock(g_scratch_mu);
  if (!g_scratch_dev[dev]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
    if (e != cudaSuccess || !p) {
      set_error(std::string("phikron_kron_apply_f64_noalloc: cudaGetSymbolAddress: ") + cudaGetErrorString(e));
      return PHIKRON_ECUDA;
    }
    g_scratch_dev[dev] = static_cast<double*>(p);
    chk::add(p, sizeof(double) * kMaxElems);
  }
  *out = g_scratch_dev[dev];
  return PHIKRON_OK;
}

}  // namespace
}  // namespace phikron

using namespace phikron;

extern "C" long long phikron_noalloc_max_elements(void) { return kMaxElems; }

extern "C" int phikron_kron_apply_f64_noalloc(int dims, const int* n, const double* const* E, const double* V,
                                              double* Out, void* stream) {
  clear_error();
  if (dims < 1 || dims > PHIKRON_MAX_DIMS || !n || !E || !V || !Out) {
    set_error("phikron_kron_apply_f64_noalloc: bad arguments");
    return PHIKRON_EINVAL;
  }
  long long N = 1;
  for (int d = 0; d < dims; ++d) {
    if (n[d] < 1 || !E[d]) {
      set_error("phikron_kron_apply_f64_noalloc: bad size or matrix pointer");
      return PHIKRON_EINVAL;
    }
    N *= n[d];
  }
  if (N > kMaxElems) {
    set_error("phikron_kron_apply_f64_noalloc: prod n[d] = " + std::to_string(N) +
              " exceeds the built-in scratch of " + std::to_string(kMaxElems) + " float64");
    return PHIKRON_EINVAL;
  }
  // a mode product reads its whole input while it writes its output (with an odd number of
  // factors the first one writes Out while reading V)
  if (ranges_overlap(V, Out, N)) {
    set_error("phikron_kron_apply_f64_noalloc: V and Out must not overlap");
    return PHIKRON_EINVAL;
  }
  double* work = nullptr;
  PK_RET(scratch_address(&work));
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  chk::Range r[PHIKRON_MAX_DIMS + 2];
  for (int d = 0; d < dims; ++d) r[d] = {E[d], sizeof(double) * (size_t)n[d] * n[d]};
  r[dims] = {V, sizeof(double) * (size_t)N};
  r[dims + 1] = {Out, sizeof(double) * (size_t)N};
  chk::CallScope cs(st, r, dims + 2);
  PK_RET(cs.rc);
  const double* cur = V;
  for (int d = 0; d < dims; ++d) {
    long long B0 = 1, R = 1;
    for (int q = 0; q < d; ++q) B0 *= n[q];
    for (int q = d + 1; q < dims; ++q) R *= n[q];
    // the last mode lands in Out; the modes before it alternate between Out and the scratch
    double* dst = (((dims - 1 - d) % 2) == 0) ? Out : work;
    PK_RET(mode_product_f64(cur, 0, dst, 0, E[d], 0, 1, B0, n[d], R, st));
    cur = dst;
  }
  return PHIKRON_OK;
}
