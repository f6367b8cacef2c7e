// Bounds-checked build (PHIKRON_CHECKED): the stand-in for a memory checker on a pool where
// compute-sanitizer is not available.  Compiled with -DPHIKRON_CHECKED into
// libphikron_checked.so; the default library compiles every check below to `true`.
//
// The host keeps a registry of the device ranges a kernel may touch: every allocation the
// library makes (device_malloc), its static device arrays, and the caller's buffers of the
// current call (registered on the call's stream before its kernels).  Each global load, store,
// atomic and bulk copy of the apply-path kernels asks check(address, bytes, site) first.  A
// range outside every registered one is recorded (first site, address and size, and a count)
// in the device state and the access is skipped: loads read zeros, stores and atomics do not
// happen, and a bulk copy reads a registered block of zeros instead, so that its mbarrier
// still completes.  Nothing traps: phikron_check_status reports PHIKRON_EBOUNDS and
// phikron_checked_violation returns the record.
//
// Device code sees the state through a pointer per translation unit (no relocatable device
// code is needed): every unit with kernels instantiates PK_CHK_BIND(name), and the host binds
// all of them once.
#pragma once

#include <cuda_runtime.h>

#include <cstddef>

namespace phikron {
namespace chk {

constexpr int kLibRanges = 1024;   // library allocations and static arrays
constexpr int kCallRanges = 192;   // caller buffers of the current call
constexpr int kRanges = kLibRanges + kCallRanges;
constexpr unsigned kZeroBytes = 128 * 1024;   // the largest bulk copy of any kernel

struct State {
  unsigned long long lo[kRanges], hi[kRanges];  // [lo, hi); hi == 0: free slot
  int nlib, ncall;                               // scan bounds of the two parts
  int site;                                      // first violation's site (0: none)
  int count;                                     // violations since the last read
  unsigned long long addr, bytes;                // first violation's range
  const void* zero;                              // kZeroBytes of zeros (registered)
};

// Access sites (phikron_checked_site_name gives the text).
enum Site : int {
  SITE_NONE = 0,
  SITE_MODE_LOAD = 1,      // mode kernels: operand values X
  SITE_MODE_STORE = 2,     // mode kernels: outputs
  SITE_MODE_ECOPY = 3,     // mode kernels: bulk copy of E digit slices
  SITE_MODE_REXP = 4,      // mode kernels: row exponents of E
  SITE_MODE_EXP = 5,       // mode kernels: exponent slots (input read, output atomicMax)
  SITE_TABLE = 6,          // job / node tables and the pointer table of a launch
  SITE_FUSED_XCOPY = 7,    // fused pass: bulk copy of a tile's raw X
  SITE_FUSED_ECOPY = 8,    // fused pass: bulk copy of E digit slices
  SITE_FUSED_STORE = 9,    // fused pass: y_j and direct outputs
  SITE_FUSED_READ = 10,    // fused pass: weights and row exponents
  SITE_EW_LOAD = 11,       // float-float elementwise kernels: loads
  SITE_EW_STORE = 12,      // float-float elementwise kernels: stores
  SITE_EW_EXP = 13,        // float-float elementwise kernels: exponent slots
  SITE_F64_LOAD = 14,      // float64 path: loads
  SITE_F64_STORE = 15,     // float64 path: stores
  SITE_ERK = 16,           // exponential integrators' elementwise kernels
  SITE_PLAN = 17,          // plan-time kernels (expm, quadrature error)
  SITE_COUNT = 18
};

#ifdef PHIKRON_CHECKED
static __device__ State* g_state = nullptr;

// true if [p, p + bytes) lies inside one registered range; else records the violation
static __device__ __noinline__ bool check(const void* p, unsigned long long bytes, int site) {
  State* s = g_state;
  if (!s) return true;
  const unsigned long long a = reinterpret_cast<unsigned long long>(p), b = a + bytes;
  const int nl = s->nlib, nc = s->ncall;
  for (int i = 0; i < nl; ++i)
    if (a >= s->lo[i] && b <= s->hi[i]) return true;
  for (int i = kLibRanges; i < kLibRanges + nc; ++i)
    if (a >= s->lo[i] && b <= s->hi[i]) return true;
  if (atomicCAS(&s->site, 0, site) == 0) {
    s->addr = a;
    s->bytes = bytes;
  }
  atomicAdd(&s->count, 1);
  return false;
}

// the source of a bulk copy: src if its range is registered, else the zero block
static __device__ __forceinline__ const void* copy_src(const void* src, unsigned long long bytes, int site) {
  if (check(src, bytes, site)) return src;
  return g_state->zero;
}

#define PK_CK(p, bytes, site) (::phikron::chk::check((const void*)(p), (unsigned long long)(bytes), (site)))
#define PK_CK_SRC(p, bytes, site) (::phikron::chk::copy_src((const void*)(p), (unsigned long long)(bytes), (site)))
// at global scope, once per translation unit with kernels
#define PK_CHK_BIND(name)                                                                     \
  namespace phikron {                                                                         \
  namespace chk {                                                                             \
  int chk_bind_##name(void* s) { return (int)cudaMemcpyToSymbol(g_state, &s, sizeof(s)); }   \
  }                                                                                           \
  }
#else
#define PK_CK(p, bytes, site) true
#define PK_CK_SRC(p, bytes, site) (p)
#define PK_CHK_BIND(name)
#endif

// a store that the checked build drops when it falls outside the registered ranges
template <class T>
__device__ __forceinline__ void st_ck(T* p, T v, int site) {
  if (PK_CK(p, sizeof(T), site)) *p = v;
}

// a load that reads zero in the checked build when it falls outside the registered ranges
template <class T>
__device__ __forceinline__ T ld_ck(const T* p, int site) {
  return PK_CK(p, sizeof(T), site) ? *p : T{};
}

// ---------------------------------------------------------------- host side (checked.cu)

struct Range {
  const void* p;
  size_t bytes;
};

// whether this library was built with the checks
bool enabled();
// a library allocation / static array comes and goes (no-ops in the default build)
void add(const void* p, size_t bytes);
void remove(const void* p);
// The caller's buffers of an entry point, registered on its stream before its kernels for the
// lifetime of the scope: an outermost call replaces the previous call's ranges, a nested one
// (an integrator step calling phikron_apply) adds to them.
struct CallScope {
  CallScope(cudaStream_t st, const Range* r, int n);
  ~CallScope();
  int rc = 0;        // PHIKRON_OK, or the error of the registration
  size_t saved = 0;  // host list length before this scope's ranges (restored at its end)
};
// PHIKRON_EBOUNDS if a violation is recorded (the record stays until read by
// phikron_checked_violation), else PHIKRON_OK
int status();
// the record (site 0 = none), cleared by the read
int read_and_clear(int* site, unsigned long long* addr, unsigned long long* bytes, int* count);

}  // namespace chk
}  // namespace phikron
