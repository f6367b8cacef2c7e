// Host side of the bounds-checked build (see checked.cuh): the registry of device ranges the
// kernels may touch, the caller-buffer ranges of the current call, and the violation record.
// In the default build every function here is a no-op and phikron_checked() returns 0.
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "checked.cuh"
#include "common.h"

namespace phikron {
namespace chk {

#ifdef PHIKRON_CHECKED

// one binder per translation unit with kernels (PK_CHK_BIND)
int chk_bind_tc_mode(void*);
int chk_bind_fused(void*);
int chk_bind_mixed(void*);
int chk_bind_gemm_f64(void*);
int chk_bind_erk(void*);
int chk_bind_api(void*);
int chk_bind_expm(void*);

namespace {

struct Host {
  std::mutex mu;
  State* dstate = nullptr;   // device copy
  void* zero = nullptr;
  std::vector<unsigned long long> lo, hi;   // library part
  bool failed = false;
};

Host& host() {
  static Host h;
  return h;
}

// bytes cut off the end of every library range (PHIKRON_CHECKED_SHRINK): makes the checks
// refuse accesses to the last bytes of real allocations, so that a test sees the violation
// path without any access outside memory the library owns
size_t shrink() {
  const char* v = std::getenv("PHIKRON_CHECKED_SHRINK");
  return v ? (size_t)std::strtoull(v, nullptr, 10) : 0;
}

int upload_lib(Host& h) {
  const int n = (int)h.lo.size();
  if (n > kLibRanges) {
    set_error("checked build: more than 1024 registered device ranges");
    return PHIKRON_ENOMEM;
  }
  if (n > 0) {
    PK_TRY_CUDA(cudaMemcpy(h.dstate->lo, h.lo.data(), sizeof(unsigned long long) * n, cudaMemcpyHostToDevice));
    PK_TRY_CUDA(cudaMemcpy(h.dstate->hi, h.hi.data(), sizeof(unsigned long long) * n, cudaMemcpyHostToDevice));
  }
  PK_TRY_CUDA(cudaMemcpy(&h.dstate->nlib, &n, sizeof(int), cudaMemcpyHostToDevice));
  return PHIKRON_OK;
}

// allocates the device state and binds every translation unit to it (once)
int ensure(Host& h) {
  if (h.dstate) return PHIKRON_OK;
  if (h.failed) return PHIKRON_ECUDA;
  h.failed = true;
  PK_TRY_CUDA(cudaMalloc(&h.dstate, sizeof(State)));
  PK_TRY_CUDA(cudaMemset(h.dstate, 0, sizeof(State)));
  PK_TRY_CUDA(cudaMalloc(&h.zero, kZeroBytes));
  PK_TRY_CUDA(cudaMemset(h.zero, 0, kZeroBytes));
  PK_TRY_CUDA(cudaMemcpy(&h.dstate->zero, &h.zero, sizeof(void*), cudaMemcpyHostToDevice));
  h.lo.push_back(reinterpret_cast<unsigned long long>(h.zero));
  h.hi.push_back(reinterpret_cast<unsigned long long>(h.zero) + kZeroBytes);
  void* s = h.dstate;
  for (int (*bind)(void*) : {chk_bind_tc_mode, chk_bind_fused, chk_bind_mixed, chk_bind_gemm_f64, chk_bind_erk,
                             chk_bind_api, chk_bind_expm}) {
    const int e = bind(s);
    if (e != 0) {
      set_error(std::string("checked build: binding the device state: ") + cudaGetErrorString((cudaError_t)e));
      return PHIKRON_ECUDA;
    }
  }
  h.failed = false;
  return upload_lib(h);
}

struct CallArgs {
  unsigned long long lo[kCallRanges], hi[kCallRanges];
  int n;
};

__global__ void call_ranges_kernel(State* s, const __grid_constant__ CallArgs a) {
  for (int i = threadIdx.x; i < a.n; i += blockDim.x) {
    s->lo[kLibRanges + i] = a.lo[i];
    s->hi[kLibRanges + i] = a.hi[i];
  }
  if (threadIdx.x == 0) s->ncall = a.n;
}

}  // namespace

bool enabled() { return true; }

void add(const void* p, size_t bytes) {
  if (!p) return;
  Host& h = host();
  std::lock_guard<std::mutex> g(h.mu);
  if (ensure(h) != PHIKRON_OK) return;
  const size_t k = shrink();
  const unsigned long long a = reinterpret_cast<unsigned long long>(p);
  h.lo.push_back(a);
  h.hi.push_back(a + (bytes > k ? bytes - k : bytes));
  upload_lib(h);
}

void remove(const void* p) {
  if (!p) return;
  Host& h = host();
  std::lock_guard<std::mutex> g(h.mu);
  if (!h.dstate) return;
  const unsigned long long a = reinterpret_cast<unsigned long long>(p);
  for (size_t i = 0; i < h.lo.size(); ++i) {
    if (h.lo[i] == a) {
      h.lo.erase(h.lo.begin() + i);
      h.hi.erase(h.hi.begin() + i);
      upload_lib(h);
      return;
    }
  }
}

thread_local int t_depth = 0;
std::vector<Range> t_calls;   // guarded by Host::mu

CallScope::CallScope(cudaStream_t st, const Range* r, int n) {
  Host& h = host();
  std::lock_guard<std::mutex> g(h.mu);
  const int depth = t_depth++;
  if (depth == 0) t_calls.clear();
  saved = t_calls.size();
  if ((rc = ensure(h)) != PHIKRON_OK) return;
  for (int i = 0; i < n; ++i)
    if (r[i].p && r[i].bytes > 0) t_calls.push_back(r[i]);
  if ((int)t_calls.size() > kCallRanges) {
    set_error("checked build: more than 192 caller buffers in one call");
    rc = PHIKRON_EINVAL;
    return;
  }
  CallArgs a{};
  a.n = (int)t_calls.size();
  for (int i = 0; i < a.n; ++i) {
    a.lo[i] = reinterpret_cast<unsigned long long>(t_calls[i].p);
    a.hi[i] = a.lo[i] + t_calls[i].bytes;
  }
  call_ranges_kernel<<<1, 64, 0, st>>>(h.dstate, a);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    set_error(std::string("checked build: registering caller buffers: ") + cudaGetErrorString(e));
    rc = PHIKRON_ECUDA;
  }
}

// a nested scope's ranges leave the host list (the device copy keeps them until the next
// registration: extra ranges of buffers that are still alive only widen the checks)
CallScope::~CallScope() {
  Host& h = host();
  std::lock_guard<std::mutex> g(h.mu);
  --t_depth;
  if (t_calls.size() > saved) t_calls.resize(saved);
}

int status() {
  Host& h = host();
  std::lock_guard<std::mutex> g(h.mu);
  if (!h.dstate) return PHIKRON_OK;
  int site = 0;
  unsigned long long addr = 0, bytes = 0;
  PK_TRY_CUDA(cudaMemcpy(&site, &h.dstate->site, sizeof(int), cudaMemcpyDeviceToHost));
  if (site == 0) return PHIKRON_OK;
  PK_TRY_CUDA(cudaMemcpy(&addr, &h.dstate->addr, sizeof(addr), cudaMemcpyDeviceToHost));
  PK_TRY_CUDA(cudaMemcpy(&bytes, &h.dstate->bytes, sizeof(bytes), cudaMemcpyDeviceToHost));
  set_error(std::string("checked build: out-of-range access at ") + phikron_checked_site_name(site) + " (" +
            std::to_string(bytes) + " bytes at 0x" + [&] {
              char b[32];
              std::snprintf(b, sizeof(b), "%llx", addr);
              return std::string(b);
            }() + ")");
  return PHIKRON_EBOUNDS;
}

int read_and_clear(int* site, unsigned long long* addr, unsigned long long* bytes, int* count) {
  Host& h = host();
  std::lock_guard<std::mutex> g(h.mu);
  *site = 0;
  *addr = *bytes = 0;
  *count = 0;
  if (!h.dstate) return PHIKRON_OK;
  PK_TRY_CUDA(cudaMemcpy(site, &h.dstate->site, sizeof(int), cudaMemcpyDeviceToHost));
  PK_TRY_CUDA(cudaMemcpy(count, &h.dstate->count, sizeof(int), cudaMemcpyDeviceToHost));
  PK_TRY_CUDA(cudaMemcpy(addr, &h.dstate->addr, sizeof(*addr), cudaMemcpyDeviceToHost));
  PK_TRY_CUDA(cudaMemcpy(bytes, &h.dstate->bytes, sizeof(*bytes), cudaMemcpyDeviceToHost));
  const int zero[2] = {0, 0};
  PK_TRY_CUDA(cudaMemcpy(&h.dstate->site, zero, sizeof(zero), cudaMemcpyHostToDevice));   // site, count
  return PHIKRON_OK;
}

#else

bool enabled() { return false; }
void add(const void*, size_t) {}
void remove(const void*) {}
CallScope::CallScope(cudaStream_t, const Range*, int) {}
CallScope::~CallScope() {}
int status() { return PHIKRON_OK; }
int read_and_clear(int* site, unsigned long long* addr, unsigned long long* bytes, int* count) {
  *site = 0;
  *addr = *bytes = 0;
  *count = 0;
  return PHIKRON_OK;
}

#endif

}  // namespace chk
}  // namespace phikron

extern "C" {

int phikron_checked(void) { return phikron::chk::enabled() ? 1 : 0; }

int phikron_checked_violation(int* site, unsigned long long* addr, unsigned long long* bytes, int* count) {
  phikron::clear_error();
  if (!site || !addr || !bytes || !count) {
    phikron::set_error("phikron_checked_violation: NULL argument");
    return PHIKRON_EINVAL;
  }
  return phikron::chk::read_and_clear(site, addr, bytes, count);
}

const char* phikron_checked_site_name(int site) {
  static const char* const names[phikron::chk::SITE_COUNT] = {
      "none",
      "mode kernel operand load",
      "mode kernel output store",
      "mode kernel E-slice bulk copy",
      "mode kernel row exponents",
      "mode kernel exponent slot",
      "job, node or pointer table",
      "fused pass raw-X bulk copy",
      "fused pass E-slice bulk copy",
      "fused pass output store",
      "fused pass weights or row exponents",
      "float-float elementwise load",
      "float-float elementwise store",
      "float-float elementwise exponent slot",
      "float64 path load",
      "float64 path store",
      "integrator elementwise kernel",
      "plan-time kernel",
  };
  return (site >= 0 && site < phikron::chk::SITE_COUNT) ? names[site] : "unknown";
}

}  // extern "C"
