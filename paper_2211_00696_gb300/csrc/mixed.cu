// Mixed-precision apply path (PHIKRON_PREC_OZAKI_BF16): plan-time slicing of the 1D
// exponentials, float-float elementwise kernels, and the orchestration of Algorithm 1 +
// the modified squaring of Eq. (29) on top of the tensor-core mode products (tc_mode.cu).
//
// State vectors between passes are float-float pairs (hi, lo) of FP32 (~48-bit
// significand), 8 bytes per unknown like float64, so every buffer of the float64 plan is
// reused.  Node weights, the squaring recurrence and the final float64 outputs are formed
// with compensated FP32 arithmetic (two-sum / FMA two-product) and integer bit assembly:
// no float64 instruction runs per element, because GB300's float64 rate is ~1/64 of FP32.
// Each kernel that writes a state vector also records an exponent e with |v| < 2^e
// (atomicMax over the vector), which the next mode product uses to cut its digits.
#include <algorithm>
#include <cstdlib>
#include <cstring>
#include <new>
#include <cmath>
#include <vector>

#include "mixed.h"
#include "plan.h"
#include "profile.h"
#include "batch.h"
#include "checked.cuh"
#include "ff_arith.cuh"

PK_CHK_BIND(mixed)

namespace phikron {

namespace {

using chk::st_ck;

// Bounds-checked build: a launch whose job table or pointer table is not registered does
// nothing (every thread decides alike).
#ifdef PHIKRON_CHECKED
#define PK_CHECK_EW_TABLES(jobs, njobs, tab)                                                  \
  if (!PK_CK((jobs), sizeof(EJob) * (size_t)(njobs), chk::SITE_TABLE) ||                        \
      ((tab) && !PK_CK((tab), sizeof(void*) * MAX_PTRS, chk::SITE_TABLE)))                      \
    return;
#else
#define PK_CHECK_EW_TABLES(jobs, njobs, tab)
#endif

constexpr int KC = 32;
constexpr int SLICE_BYTES = 128 * KC * 2;

using ff::to_f64;

constexpr int MAXP = 20;   // l_max of the mixed path (the paper's range, Sec. 4)
constexpr int MAXM = 64;
constexpr int EW_THREADS = 256;
// element pairs per thread and virtual block of the weighted-sum and squaring kernels (vectors
// are float2 arrays of even length).  Two: a 2M-element vector makes ~3.4 rounds of virtual
// blocks over the resident blocks instead of ~1.7 with four pairs, whose last round left a third
// of them idle (measured on the 128^3 step: weighted sums 0.061 -> 0.054 ms, squaring 0.063 ->
// 0.060 ms; one pair gave 0.061 and 0.060)
constexpr int EW_PAIRS = 2;
constexpr long long EW_BLOCK = 2LL * EW_THREADS * EW_PAIRS;
// the exponent scan reads SCAN_PAIRS pairs a thread, all loads in flight at once
constexpr int SCAN_PAIRS = 4;
constexpr long long SCAN_BLOCK = 2LL * EW_THREADS * SCAN_PAIRS;

struct InvFact {
  float2 f[MAXP + 1];  // 1/k! as float-float
};

__device__ __forceinline__ int find_ejob(const EJob* jobs, int njobs, long long blk) {
  int lo = 0, hi = njobs - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (jobs[mid].block_begin <= blk) lo = mid; else hi = mid - 1;
  }
  return lo;
}

__device__ __forceinline__ void* tab_ptr(const void* const* tab, int e, long long off, void* direct) {
  if (e < 0) return direct;
  if (!PK_CK(tab + e, sizeof(void*), chk::SITE_TABLE)) return nullptr;
  return (void*)((char*)tab[e] + off);
}

// two consecutive float-float values (16 bytes; every vector offset used is a multiple of 2)
__device__ __forceinline__ void ld_pair(const float2* p, float2& a, float2& b) {
  const float4 v = PK_CK(p, 16, chk::SITE_EW_LOAD) ? __ldg(reinterpret_cast<const float4*>(p))
                                                   : make_float4(0.f, 0.f, 0.f, 0.f);
  a = make_float2(v.x, v.y);
  b = make_float2(v.z, v.w);
}

// stores of the results of one element pair: float-float (16-byte store) or float64 (two
// 8-byte stores: the caller's float64 buffers need only be 8-byte aligned), plus the optional
// float64 copy; the exponent maximum covers both
__device__ __forceinline__ void st_pair(void* out, void* out2, bool f64, long long off, float2 a, float2 b, int& emax) {
  if (f64) {
    double* o = reinterpret_cast<double*>(out) + off;
    st_ck(o, to_f64(a.x, a.y), chk::SITE_EW_STORE);
    st_ck(o + 1, to_f64(b.x, b.y), chk::SITE_EW_STORE);
  } else {
    st_ck(reinterpret_cast<float4*>(reinterpret_cast<float2*>(out) + off), make_float4(a.x, a.y, b.x, b.y),
          chk::SITE_EW_STORE);
  }
  if (out2) {
    double* o = reinterpret_cast<double*>(out2) + off;
    st_ck(o, to_f64(a.x, a.y), chk::SITE_EW_STORE);
    st_ck(o + 1, to_f64(b.x, b.y), chk::SITE_EW_STORE);
  }
  emax = max(emax, (int)((__float_as_uint(a.x) >> 23) & 0xFFu));
  emax = max(emax, (int)((__float_as_uint(b.x) >> 23) & 0xFFu));
}

// Exponent slots: the block's largest biased exponent per output (0 = nothing stored; BIAS
// 126 for FP32 exponent fields, 1022 for float64 ones, so that |v| < 2^{emax - BIAS}),
// reduced over warps in shared memory, then one atomicMax per output and block (instead of
// one per warp: same-address atomics serialise in L2).  Called by every thread of the block.
template <int P_, int BIAS = 126>
__device__ __forceinline__ void block_exp_flush(int (&emax)[P_], int* out_exp, int (*red)[EW_THREADS / 32]) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
  for (int j = 0; j < P_; ++j) {
    int v = emax[j] > 0 ? emax[j] - BIAS : -1000;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = max(v, __shfl_xor_sync(0xffffffffu, v, o));
    if (lane == 0) red[j][warp] = v;
    emax[j] = 0;
  }
  __syncthreads();
  if (threadIdx.x < P_ && out_exp) {
    int v = -1000;
#pragma unroll
    for (int w = 0; w < EW_THREADS / 32; ++w) v = max(v, red[threadIdx.x][w]);
    if (v > -1000 && PK_CK(out_exp + threadIdx.x, sizeof(int), chk::SITE_EW_EXP)) atomicMax(out_exp + threadIdx.x, v);
  }
  __syncthreads();
}

// The elementwise kernels run a grid of (SMs x resident blocks) that strides over the
// launch's virtual blocks of EW_BLOCK elements (all jobs laid end to end), so that no
// partial second wave idles most of the GPU.

// y_j = sum_k coef[j][k] T_k in float-float (Algorithm 1, second step), grouped over jobs.
// The T_k of a pair are read in batches (KB) before any arithmetic, so that each thread keeps
// KB x 16 bytes of loads in flight.
template <int P_>
__global__ void __launch_bounds__(EW_THREADS, P_ <= 3 ? 4 : (P_ <= 7 ? 3 : (P_ <= 11 ? 2 : 1)))
    g_weighted_kernel(const EJob* __restrict__ jobs, int njobs, long long total, const void* const* ptrtab) {
  PK_CHECK_EW_TABLES(jobs, njobs, ptrtab);
  constexpr int KB = P_ <= 3 ? 6 : (P_ <= 8 ? 4 : 2);  // T_k per batch (register budget without spills)
  __shared__ float2 cs[P_ * MAXM];
  __shared__ int red[P_][EW_THREADS / 32];
  int emax[P_];
#pragma unroll
  for (int j = 0; j < P_; ++j) emax[j] = 0;
  int cur = -1;
  for (long long vb = blockIdx.x; vb < total; vb += gridDim.x) {
    const int jb = find_ejob(jobs, njobs, vb);  // uniform over the block
    const EJob& J = jobs[jb];
    if (jb != cur) {
      if (cur >= 0) block_exp_flush<P_>(emax, jobs[cur].out_exp, red);
      for (int q = threadIdx.x; q < P_ * J.m; q += EW_THREADS)
        cs[q] = PK_CK(J.coef + q, sizeof(float2), chk::SITE_EW_LOAD) ? J.coef[q] : make_float2(0.f, 0.f);
      __syncthreads();
      cur = jb;
    }
    const int m = J.m;
    void* out = tab_ptr(ptrtab, J.out_tab, J.tab_off_out, J.out);
    void* out2 = tab_ptr(ptrtab, J.out2_tab, J.tab_off_out2, J.out2);
    const bool f64 = J.out_f64 != 0;
    const long long N = J.N, stride = J.stride;
    const long long base = (vb - J.block_begin) * EW_BLOCK;
#pragma unroll 1
    for (int e = 0; e < EW_PAIRS; ++e) {
      const long long i = base + 2 * ((long long)e * EW_THREADS + threadIdx.x);
      if (i < N) {
        float2 acc0[P_], acc1[P_];
#pragma unroll
        for (int j = 0; j < P_; ++j) acc0[j] = acc1[j] = make_float2(0.f, 0.f);
#pragma unroll 1
        for (int k0 = 0; k0 < m; k0 += KB) {
          float2 t0[KB], t1[KB];
#pragma unroll
          for (int q = 0; q < KB; ++q)
            if (k0 + q < m) ld_pair(J.a + (k0 + q) * stride + i, t0[q], t1[q]);
#pragma unroll
          for (int q = 0; q < KB; ++q) {
            if (k0 + q < m) {
#pragma unroll
              for (int j = 0; j < P_; ++j) {
                ff::fma_ff(acc0[j], cs[j * m + k0 + q], t0[q]);
                ff::fma_ff(acc1[j], cs[j * m + k0 + q], t1[q]);
              }
            }
          }
        }
#pragma unroll
        for (int j = 0; j < P_; ++j) st_pair(out, out2, f64, j * stride + i, acc0[j], acc1[j], emax[j]);
      }
    }
  }
  if (cur >= 0) block_exp_flush<P_>(emax, jobs[cur].out_exp, red);
}

// y-hat_i = 2^{-i}(Z_i + sum_{j<=i} y_j/(i-j)!), i = 1..p (Eq. (29)), grouped over jobs
template <int P_>
__global__ void __launch_bounds__(EW_THREADS, P_ <= 6 ? 4 : (P_ <= 11 ? 2 : 1)) g_squaring_kernel(const EJob* __restrict__ jobs, int njobs,
                                                                   long long total, const void* const* ptrtab,
                                                                   InvFact inv) {
  PK_CHECK_EW_TABLES(jobs, njobs, ptrtab);
  __shared__ int red[P_][EW_THREADS / 32];
  int emax[P_];
#pragma unroll
  for (int j = 0; j < P_; ++j) emax[j] = 0;
  int cur = -1;
  for (long long vb = blockIdx.x; vb < total; vb += gridDim.x) {
    const int jb = find_ejob(jobs, njobs, vb);
    const EJob& J = jobs[jb];
    if (jb != cur) {
      if (cur >= 0) block_exp_flush<P_>(emax, jobs[cur].out_exp, red);
      cur = jb;
    }
    void* out = tab_ptr(ptrtab, J.out_tab, J.tab_off_out, J.out);
    void* out2 = tab_ptr(ptrtab, J.out2_tab, J.tab_off_out2, J.out2);
    const bool f64 = J.out_f64 != 0;
    const long long N = J.N, stride = J.stride;
    const long long base = (vb - J.block_begin) * EW_BLOCK;
#pragma unroll 1
    for (int e = 0; e < EW_PAIRS; ++e) {
      const long long x = base + 2 * ((long long)e * EW_THREADS + threadIdx.x);
      if (x < N) {
        float2 y0[P_], y1[P_], z0[P_], z1[P_];
#pragma unroll
        for (int j = 0; j < P_; ++j) {
          ld_pair(J.b + j * stride + x, y0[j], y1[j]);
          ld_pair(J.a + j * stride + x, z0[j], z1[j]);
        }
        float sc = 1.0f;
#pragma unroll
        for (int q = 1; q <= P_; ++q) {
          sc *= 0.5f;
          float2 a0 = z0[q - 1], a1 = z1[q - 1];
#pragma unroll
          for (int j = 1; j <= q; ++j) {
            const int d = q - j;
            if (d <= 1) {
              ff::add_ff(a0, y0[j - 1]);
              ff::add_ff(a1, y1[j - 1]);
            } else {
              ff::fma_ff(a0, inv.f[d], y0[j - 1]);
              ff::fma_ff(a1, inv.f[d], y1[j - 1]);
            }
          }
          z0[q - 1] = make_float2(a0.x * sc, a0.y * sc);
          z1[q - 1] = make_float2(a1.x * sc, a1.y * sc);
        }
#pragma unroll
        for (int q = 0; q < P_; ++q) st_pair(out, out2, f64, q * stride + x, z0[q], z1[q], emax[q]);
      }
    }
  }
  if (cur >= 0) block_exp_flush<P_>(emax, jobs[cur].out_exp, red);
}

// e with |v| < 2^e over a float64 vector (integer ops only), grouped over jobs
__global__ void __launch_bounds__(EW_THREADS) g_expscan_kernel(const EJob* __restrict__ jobs, int njobs,
                                                               long long total, const void* const* ptrtab) {
  PK_CHECK_EW_TABLES(jobs, njobs, ptrtab);
  __shared__ int red[1][EW_THREADS / 32];
  int emax[1] = {0};  // float64 exponent field: |v| < 2^{emax - 1022}
  int cur = -1;
  for (long long vb = blockIdx.x; vb < total; vb += gridDim.x) {
    const int jb = find_ejob(jobs, njobs, vb);
    const EJob& J = jobs[jb];
    if (jb != cur) {
      if (cur >= 0) block_exp_flush<1, 1022>(emax, jobs[cur].out_exp, red);
      cur = jb;
    }
    const double* v = reinterpret_cast<const double*>(tab_ptr(ptrtab, J.v_tab, J.tab_off_v, (void*)J.v));
    const long long base = (vb - J.block_begin) * SCAN_BLOCK;
    uint64_t b[2 * SCAN_PAIRS];
#pragma unroll
    for (int q = 0; q < 2 * SCAN_PAIRS; ++q) {
      const long long i = base + (long long)q * EW_THREADS + threadIdx.x;
      b[q] = (i < J.N && PK_CK(v + i, sizeof(double), chk::SITE_EW_LOAD)) ? (uint64_t)__double_as_longlong(__ldg(v + i))
                                                                          : 0ull;
    }
#pragma unroll
    for (int q = 0; q < 2 * SCAN_PAIRS; ++q) {
      emax[0] = max(emax[0], (int)((b[q] >> 52) & 0x7FF));  // subnormals and zeros: 0
    }
  }
  if (cur >= 0) block_exp_flush<1, 1022>(emax, jobs[cur].out_exp, red);
}

// sizes of a padded plan: n[d] of the caller's vectors, pn[d] of the padded ones (C-order)
struct PadDims {
  int dims;
  int n[PHIKRON_MAX_DIMS];
  int pn[PHIKRON_MAX_DIMS];
};

// Vp = V zero-padded: element q of the padded tensor takes V at the same multi-index when every
// index is inside n, else 0
__global__ void pad_scatter_kernel(const double* __restrict__ V, double* __restrict__ Vp, long long PN, PadDims D) {
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < PN; q += (long long)gridDim.x * blockDim.x) {
    long long r = q, src = 0, mul = 1;
    bool in = true;
    for (int d = D.dims - 1; d >= 0; --d) {
      const int id = (int)(r % D.pn[d]);
      r /= D.pn[d];
      in = in && id < D.n[d];
      src += (long long)id * mul;
      mul *= D.n[d];
    }
    st_ck(Vp + q, (in && PK_CK(V + src, sizeof(double), chk::SITE_EW_LOAD)) ? V[src] : 0.0, chk::SITE_EW_STORE);
  }
}

// Out[v][x] = Op[v][padded index of x] for the vectors v in mask (v < nvec <= 64)
__global__ void pad_gather_kernel(const double* __restrict__ Op, double* __restrict__ Out, long long N, long long PN,
                                  int nvec, unsigned long long mask, PadDims D) {
  const long long total = (long long)nvec * N;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total; t += (long long)gridDim.x * blockDim.x) {
    const int v = (int)(t / N);
    if (!((mask >> v) & 1ull)) continue;
    long long r = t - (long long)v * N, dst = 0, mul = 1;
    for (int d = D.dims - 1; d >= 0; --d) {
      const int id = (int)(r % D.n[d]);
      r /= D.n[d];
      dst += (long long)id * mul;
      mul *= D.pn[d];
    }
    const double* sp = Op + (long long)v * PN + dst;
    st_ck(Out + t, PK_CK(sp, sizeof(double), chk::SITE_EW_LOAD) ? *sp : 0.0, chk::SITE_EW_STORE);
  }
}

// grid for a grid-stride elementwise kernel: every SM filled with resident blocks, no more
// blocks than virtual blocks
template <typename K>
unsigned ew_grid(K kernel, long long total) {
  static int sms = 0;
  if (!sms) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (sms <= 0) sms = 1;
  }
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, EW_THREADS, 0) != cudaSuccess || per_sm < 1)
    per_sm = 1;
  return (unsigned)std::min<long long>(total, (long long)sms * per_sm);
}

InvFact make_invfact() {
  InvFact r;
  double f = 1.0;
  for (int k = 0; k <= MAXP; ++k) {
    if (k > 1) f *= k;
    const double v = 1.0 / f;
    const float hi = (float)v;
    r.f[k] = make_float2(hi, (float)(v - (double)hi));
  }
  return r;
}

template <int P_>
int launch_ew(int kind, const EJob* jobs, int njobs, long long blocks, const void* const* tab, cudaStream_t st) {
  if (kind == STEP_WEIGHTED) {
    const unsigned grid = ew_grid(g_weighted_kernel<P_>, blocks);
    launch_begin(KC_WEIGHTED, st);
    g_weighted_kernel<P_><<<grid, EW_THREADS, 0, st>>>(jobs, njobs, blocks, tab);
  } else {
    static const InvFact inv = make_invfact();
    const unsigned grid = ew_grid(g_squaring_kernel<P_>, blocks);
    launch_begin(KC_SQUARING, st);
    g_squaring_kernel<P_><<<grid, EW_THREADS, 0, st>>>(jobs, njobs, blocks, tab, inv);
  }
  launch_end(st);
  PK_CHECK_LAUNCH();
  return PHIKRON_OK;
}

int launch_ew_p(int kind, int p, const EJob* jobs, int njobs, long long blocks, const void* const* tab,
                cudaStream_t st) {
  switch (p) {
    case 1: return launch_ew<1>(kind, jobs, njobs, blocks, tab, st);
    case 2: return launch_ew<2>(kind, jobs, njobs, blocks, tab, st);
    case 3: return launch_ew<3>(kind, jobs, njobs, blocks, tab, st);
    case 4: return launch_ew<4>(kind, jobs, njobs, blocks, tab, st);
    case 5: return launch_ew<5>(kind, jobs, njobs, blocks, tab, st);
    case 6: return launch_ew<6>(kind, jobs, njobs, blocks, tab, st);
    case 7: return launch_ew<7>(kind, jobs, njobs, blocks, tab, st);
    case 8: return launch_ew<8>(kind, jobs, njobs, blocks, tab, st);
    case 9: return launch_ew<9>(kind, jobs, njobs, blocks, tab, st);
    case 10: return launch_ew<10>(kind, jobs, njobs, blocks, tab, st);
    case 11: return launch_ew<11>(kind, jobs, njobs, blocks, tab, st);
    case 12: return launch_ew<12>(kind, jobs, njobs, blocks, tab, st);
    case 13: return launch_ew<13>(kind, jobs, njobs, blocks, tab, st);
    case 14: return launch_ew<14>(kind, jobs, njobs, blocks, tab, st);
    case 15: return launch_ew<15>(kind, jobs, njobs, blocks, tab, st);
    case 16: return launch_ew<16>(kind, jobs, njobs, blocks, tab, st);
    case 17: return launch_ew<17>(kind, jobs, njobs, blocks, tab, st);
    case 18: return launch_ew<18>(kind, jobs, njobs, blocks, tab, st);
    case 19: return launch_ew<19>(kind, jobs, njobs, blocks, tab, st);
    case 20: return launch_ew<20>(kind, jobs, njobs, blocks, tab, st);
    default: set_error("mixed path: l_max must be in 1..20"); return PHIKRON_ENOTSUP;
  }
}

}  // namespace

// ----------------------------------------------------------------------------- host slicing

size_t sliced_bytes(int n, int slices) {
  const int nchunks = (n + KC - 1) / KC;
  const int nhalves = (n + 127) / 128;
  return (size_t)nhalves * nchunks * slices * SLICE_BYTES;
}

// E (n x n) -> [row block][chunk32][slice][128 rows x 32 cols core-matrix layout] with rows
// 128*b .. 128*b+127 of E in block b; rexp[b*128 + i] = f with max_k |E[row][k]| < 2^f.
// Digits are those of |E| * 2^{64-f} rounded to nearest at digit `slices`.
void slice_matrix_host(const double* E, int n, int slices, uint8_t* out, int* rexp) {
  const int nchunks = (n + KC - 1) / KC;
  const int nhalves = (n + 127) / 128;
  std::memset(out, 0, sliced_bytes(n, slices));
  for (int i = 0; i < 128 * nhalves; ++i) rexp[i] = 0;
  for (int row = 0; row < n; ++row) {
    const int h = row / 128, i = row % 128;
    double mx = 0.0;
    for (int k = 0; k < n; ++k) mx = std::max(mx, std::fabs(E[(size_t)row * n + k]));
    int f = 0;
    if (mx > 0.0) std::frexp(mx, &f);  // mx = frac * 2^f, frac in [0.5, 1) -> mx < 2^f
    rexp[h * 128 + i] = f;
    for (int k = 0; k < n; ++k) {
      const double x = E[(size_t)row * n + k];
      const double a = std::ldexp(std::fabs(x), 64 - f);  // in [0, 2^64)
      uint64_t F = (a >= 18446744073709551616.0) ? ~0ull : (uint64_t)a;
      const uint64_t half = 1ull << (63 - 8 * slices);  // round to nearest at the last digit
      F = (F > ~0ull - half) ? ~0ull : F + half;
      const int c = k / KC, kk = k % KC;
      const size_t off = (size_t)chunk_offset(i, kk >> 3) + (size_t)(kk & 7) * 2;
      for (int s = 0; s < slices; ++s) {
        const int t = s + 1;
        const uint32_t d = (uint32_t)((F >> (64 - 8 * t)) & 0xFFu);
        const float v = std::ldexp((float)d, -8 * t) * (x < 0 ? -1.0f : 1.0f);
        uint32_t bits;
        std::memcpy(&bits, &v, 4);
        const uint16_t bf = (uint16_t)(bits >> 16);
        uint8_t* dst = out + (((size_t)h * nchunks + c) * slices + s) * SLICE_BYTES + off;
        std::memcpy(dst, &bf, 2);
      }
    }
  }
}

// ----------------------------------------------------------------------------- plan state

struct MixedState {
  int slices = 5;
  int nsm = 148;
  uint8_t* dSl[PHIKRON_MAX_DIMS] = {};             // per unique factor: nexp sliced matrices
  int* dRexp[PHIKRON_MAX_DIMS] = {};                // per unique factor: nexp x row blocks x 128
  size_t mat_bytes[PHIKRON_MAX_DIMS] = {};
  int rexp_stride[PHIKRON_MAX_DIMS] = {};
  float2* dCoefFF = nullptr;
  // padded plans (some n[d] not a multiple of 16): work buffers, input and output staging of the
  // padded sizes; the apply scatters V into dVp and gathers the results from dOutp
  bool padded = false;
  double* dVp = nullptr;
  double* dOutp = nullptr;
  Seq seq;                                         // launch sequence of a single-vector apply
};

static void mixed_free(void* p) { delete static_cast<MixedState*>(p); }

const MixedView mixed_view(const Plan& P, int d) {
  const MixedState& M = *static_cast<const MixedState*>(P.mixed);
  const int u = P.uniq_of[d];
  MixedView v;
  v.sl = M.dSl[u];
  v.rexp = M.dRexp[u];
  v.mat_bytes = M.mat_bytes[u];
  v.rexp_stride = M.rexp_stride[u];
  v.coef = M.dCoefFF;
  v.slices = M.slices;
  v.nsm = M.nsm;
  return v;
}

int precision_setup(Plan& P) {
  if (P.opts.precision == PHIKRON_PREC_FP64) return PHIKRON_OK;
  if (P.opts.precision != PHIKRON_PREC_OZAKI_BF16) {
    set_error("precision mode not supported");
    return PHIKRON_ENOTSUP;
  }
  // the tensor-core mode products need every contracted size to be a multiple of 16: other
  // sizes are padded (see Plan::pn)
  bool pad = false;
  P.PN = 1;
  for (int d = 0; d < P.dims; ++d) {
    P.pn[d] = std::max(16, (P.n[d] + 15) / 16 * 16);
    if (P.pn[d] > 4096) {
      set_error("mixed path: every n[d] must be at most 4096");
      return PHIKRON_ENOTSUP;
    }
    pad = pad || P.pn[d] != P.n[d];
    P.PN *= P.pn[d];
  }
  if (P.p > MAXP || P.m > MAXM) {
    set_error("mixed path: needs l_max <= 20 and at most 64 quadrature nodes");
    return PHIKRON_ENOTSUP;
  }
  MixedState* M = alloc_fault() ? nullptr : new (std::nothrow) MixedState();
  if (!M) {
    set_error("mixed plan state: host allocation failed");
    return PHIKRON_ENOMEM;
  }
  P.mixed = M;
  P.mixed_free = mixed_free;
  int slices = P.opts.slices;
  // digit error per apply measured on the 128^3 convection-diffusion workload: 3 slices ~4e-7,
  // 4 ~2e-9, 5 ~1e-11, 6 below the float-float state's ~1e-13
  if (slices <= 0) slices = (P.tol >= 1e-5) ? 3 : (P.tol >= 1e-8) ? 4 : (P.tol >= 1e-10) ? 5 : 6;
  if (slices < 3 || slices > 6) {
    set_error("mixed path: slices must be 3..6");
    return PHIKRON_EINVAL;
  }
  M->slices = slices;
  int dev = 0;
  PK_TRY_CUDA(cudaGetDevice(&dev));
  PK_TRY_CUDA(cudaDeviceGetAttribute(&M->nsm, cudaDevAttrMultiProcessorCount, dev));

  // slice every 1D exponential (plan time, host)
  for (int u = 0; u < P.nuniq; ++u) {
    const int nd = P.n[P.uniq_rep[u]], pd = P.pn[P.uniq_rep[u]];
    const size_t nn = (size_t)nd * nd, pp = (size_t)pd * pd;
    std::vector<double> h(nn * P.nexp);
    PK_TRY_CUDA(cudaMemcpy(h.data(), P.dExp[u], sizeof(double) * nn * P.nexp, cudaMemcpyDeviceToHost));
    const size_t mb = sliced_bytes(pd, slices);
    const int rs = 128 * ((pd + 127) / 128);
    std::vector<uint8_t> sl(mb * P.nexp);
    std::vector<int> rx((size_t)rs * P.nexp);
    std::vector<double> hp(pp);
    for (int e = 0; e < P.nexp; ++e) {
      const double* src = h.data() + nn * e;
      if (pd != nd) {   // exp of diag(c A^d, 0): the exponential on the leading block, I on the pad
        std::fill(hp.begin(), hp.end(), 0.0);
        for (int r = 0; r < nd; ++r)
          std::copy(src + (size_t)r * nd, src + (size_t)(r + 1) * nd, hp.data() + (size_t)r * pd);
        for (int r = nd; r < pd; ++r) hp[(size_t)r * pd + r] = 1.0;
        src = hp.data();
      }
      slice_matrix_host(src, pd, slices, sl.data() + mb * e, rx.data() + (size_t)rs * e);
    }
    PK_RET(P.alloc((void**)&M->dSl[u], sl.size()));
    PK_RET(P.alloc((void**)&M->dRexp[u], sizeof(int) * rx.size()));
    PK_TRY_CUDA(cudaMemcpy(M->dSl[u], sl.data(), sl.size(), cudaMemcpyHostToDevice));
    PK_TRY_CUDA(cudaMemcpy(M->dRexp[u], rx.data(), sizeof(int) * rx.size(), cudaMemcpyHostToDevice));
    M->mat_bytes[u] = mb;
    M->rexp_stride[u] = rs;
  }
  // node weights as float-float
  std::vector<float2> cf(P.coef.size());
  for (size_t i = 0; i < P.coef.size(); ++i) {
    const float hi = (float)P.coef[i];
    cf[i] = make_float2(hi, (float)(P.coef[i] - (double)hi));
  }
  PK_RET(P.alloc((void**)&M->dCoefFF, sizeof(float2) * std::max<size_t>(1, cf.size())));
  if (!cf.empty())
    PK_TRY_CUDA(cudaMemcpy(M->dCoefFF, cf.data(), sizeof(float2) * cf.size(), cudaMemcpyHostToDevice));

  // the single-vector apply as a launch sequence over the plan's own work buffers (of the
  // padded sizes, with input and output staging, when some n[d] is padded)
  std::vector<SeqUnit> units(1);
  units[0].plan = &P;
  units[0].inst = 0;
  units[0].rhs = 0;
  units[0].W1 = reinterpret_cast<float2*>(P.dW1);
  units[0].W2 = reinterpret_cast<float2*>(P.dW2);
  units[0].Y = reinterpret_cast<float2*>(P.dY);
  units[0].Yn = reinterpret_cast<float2*>(P.dYn);
  M->padded = pad;
  if (pad) {
    const size_t nv = (size_t)std::max(P.m + 2, std::max(P.p, 1));
    const size_t ny = (size_t)std::max(P.p, 1);
    const size_t nout = (size_t)(P.p + 1) * (P.opts.half_step ? 2 : 1);
    PK_RET(P.alloc((void**)&units[0].W1, sizeof(float2) * nv * P.PN));
    PK_RET(P.alloc((void**)&units[0].W2, sizeof(float2) * nv * P.PN));
    PK_RET(P.alloc((void**)&units[0].Y, sizeof(float2) * ny * P.PN));
    PK_RET(P.alloc((void**)&units[0].Yn, sizeof(float2) * ny * P.PN));
    PK_RET(P.alloc((void**)&M->dVp, sizeof(double) * P.PN));
    PK_RET(P.alloc((void**)&M->dOutp, sizeof(double) * nout * P.PN));
    PK_TRY_CUDA(cudaMemset(M->dOutp, 0, sizeof(double) * nout * P.PN));
  }
  SeqConfig cfg;
  cfg.half = P.opts.half_step != 0;
  cfg.slices = slices;
  cfg.sub = 1;
  cfg.grid = M->nsm;
  cfg.big_first = false;
  cfg.graph = true;
  cfg.ws = mode_kernel_ws_default();
  cfg.db = mode_kernel_db_default();
  cfg.fuse = fused_weights_default();
  cfg.rr = raw_ring_default();
  PK_RET(seq_build(M->seq, units, 1, cfg));
  return PHIKRON_OK;
}

int apply_mixed(Plan& P, const double* V, double* Out, cudaStream_t st) {
  MixedState& M = *static_cast<MixedState*>(P.mixed);
  PtrArgs args{};
  args.n = 2;
  if (!M.padded) {
    args.p[0] = const_cast<double*>(V);
    args.p[1] = Out;
    return seq_run(M.seq, args, st);
  }
  PadDims D{};
  D.dims = P.dims;
  for (int d = 0; d < P.dims; ++d) {
    D.n[d] = P.n[d];
    D.pn[d] = P.pn[d];
  }
  launch_begin(KC_CONVERT, st);
  pad_scatter_kernel<<<ew_grid(pad_scatter_kernel, (P.PN + 255) / 256), 256, 0, st>>>(V, M.dVp, P.PN, D);
  launch_end(st);
  PK_CHECK_LAUNCH();
  args.p[0] = M.dVp;
  args.p[1] = M.dOutp;
  PK_RET(seq_run(M.seq, args, st));
  // every output vector except the phi_0 slots a skip_phi0 plan leaves untouched
  const int nout = (P.p + 1) * (P.opts.half_step ? 2 : 1);
  unsigned long long mask = 0;
  for (int v = 0; v < nout; ++v)
    if (!(P.opts.skip_phi0 && (v % (P.p + 1)) == 0)) mask |= 1ull << v;
  launch_begin(KC_CONVERT, st);
  pad_gather_kernel<<<ew_grid(pad_gather_kernel, (nout * P.N + 255) / 256), 256, 0, st>>>(M.dOutp, Out, P.N, P.PN,
                                                                                        nout, mask, D);
  launch_end(st);
  PK_CHECK_LAUNCH();
  return PHIKRON_OK;
}

int mixed_slices(const Plan& P) { return static_cast<const MixedState*>(P.mixed)->slices; }

bool mixed_fused(const Plan& P) { return P.mixed && static_cast<const MixedState*>(P.mixed)->seq.fused; }

int mixed_status(Plan& P, int* status) {
  if (!P.mixed) {
    *status = 0;
    return PHIKRON_OK;
  }
  MixedState& M = *static_cast<MixedState*>(P.mixed);
  return seq_status(M.seq, status);
}

// ----------------------------------------------------------------------------- sequences

Seq::~Seq() {
  if (exec) cudaGraphExecDestroy(exec);
  for (void* p : allocs) device_free(p);
}

namespace {

int seq_alloc(Seq& S, void** p, size_t bytes) {
  if (bytes == 0) bytes = 16;
  PK_RET(device_malloc(p, bytes, "launch sequence"));
  S.allocs.push_back(*p);
  S.device_bytes += bytes;
  return PHIKRON_OK;
}

long long job_tiles(const GJob& j, const PassShape& s) {
  const long long blocks = (j.n + 127) / 128, f = tile_fibers(s);
  return s.trans ? blocks * j.B0 * ((j.R + f - 1) / f) : blocks * ((j.B0 + f - 1) / f);
}

struct Builder {
  std::vector<GJob> gjobs;
  std::vector<EJob> ejobs;
  std::vector<FJob> fjobs;
  std::vector<FNode> fnodes;
  std::vector<Step> steps;
  int nslots = 0;
  bool big_first = false;
  std::vector<uint8_t> tmaps;   // tensor maps of the raw-ring passes' inputs

  void mode_step(std::vector<GJob> jobs, const PassShape& shape) {
    if (jobs.empty()) return;
    if (big_first)
      std::stable_sort(jobs.begin(), jobs.end(), [&](const GJob& a, const GJob& b) {
        return job_tiles(a, shape) > job_tiles(b, shape);
      });
    long long t = 0;
    for (GJob& j : jobs) {
      j.tile_begin = t;
      t += job_tiles(j, shape);
    }
    Step s{};
    s.kind = STEP_MODE;
    s.off = gjobs.size();
    s.count = (int)jobs.size();
    s.total = t;
    s.shape = shape;
    gjobs.insert(gjobs.end(), jobs.begin(), jobs.end());
    steps.push_back(s);
  }

  // pre-cut digit slices of float64 inputs: one block per (job, 128-fiber block, chunk)
  void precut_step(std::vector<GJob> jobs, int slices) {
    if (jobs.empty()) return;
    long long t = 0;
    for (GJob& j : jobs) {
      j.tile_begin = t;
      t += ((j.R + 127) / 128) * ((j.n + 31) / 32);
    }
    Step s{};
    s.kind = STEP_PRECUT;
    s.off = gjobs.size();
    s.count = (int)jobs.size();
    s.total = t;
    s.shape.slices = slices;
    gjobs.insert(gjobs.end(), jobs.begin(), jobs.end());
    steps.push_back(s);
  }

  // jobs[u].node0 indexes `nodes`; both are appended to the builder's tables
  void fused_step(std::vector<FJob> jobs, const std::vector<FNode>& nodes, const PassShape& shape, int p) {
    if (jobs.empty()) return;
    long long t = 0;
    const int base = (int)fnodes.size();
    for (FJob& j : jobs) {
      j.tile_begin = t;
      t += (j.B0 + fused::kFibers - 1) / fused::kFibers;
      j.node0 += base;
    }
    Step s{};
    s.kind = STEP_FUSED;
    s.off = fjobs.size();
    s.count = (int)jobs.size();
    s.total = t;
    s.p = p;
    s.shape = shape;
    fjobs.insert(fjobs.end(), jobs.begin(), jobs.end());
    fnodes.insert(fnodes.end(), nodes.begin(), nodes.end());
    steps.push_back(s);
  }

  void ew_step(int kind, std::vector<EJob> jobs, int p) {
    if (jobs.empty()) return;
    long long b = 0;
    const long long bs = kind == STEP_EXPSCAN ? SCAN_BLOCK : EW_BLOCK;
    for (EJob& j : jobs) {
      j.block_begin = b;
      b += (j.N + bs - 1) / bs;
    }
    Step s{};
    s.kind = kind;
    s.off = ejobs.size();
    s.count = (int)jobs.size();
    s.total = b;
    s.p = p;
    ejobs.insert(ejobs.end(), jobs.begin(), jobs.end());
    steps.push_back(s);
  }
};

}  // namespace

// Builds the launch sequence of Algorithm 1 + Algorithm 6 (+ phi_0, + optional half-step
// outputs) over `units` (one unit = one vector of one plan).  Unit u reads V from pointer
// table entry 2*inst at byte offset rhs*N*8 and writes Out to entry 2*inst+1 at offset
// rhs*(p+1)*(1+half)*N*8.
bool mode_kernel_ws_default() {
  const char* v = std::getenv("PHIKRON_MODE_KERNEL");
  return !(v && std::strcmp(v, "classic") == 0);
}

bool mode_kernel_db_default() {
  const char* v = std::getenv("PHIKRON_MODE_KERNEL");
  return v && std::strcmp(v, "db") == 0;
}

bool fused_weights_default() {
  const char* v = std::getenv("PHIKRON_FUSED_WEIGHTS");
  return v && std::strcmp(v, "1") == 0;
}

bool raw_ring_default() {
  const char* v = std::getenv("PHIKRON_RAW_RING");
  return !(v && std::strcmp(v, "0") == 0);
}

// the float64 first pass reads its input's digit slices cut once (unless PHIKRON_PRECUT is "0")
static bool precut_default() {
  const char* v = std::getenv("PHIKRON_PRECUT");
  return !(v && std::strcmp(v, "0") == 0);
}

int seq_build(Seq& S, std::vector<SeqUnit>& units, int ninst, const SeqConfig& cfg) {
  Builder B;
  B.big_first = cfg.big_first;
  const int nu = (int)units.size();
  if (nu == 0) return PHIKRON_OK;
  const int dims = units[0].plan->dims;
  const int p = units[0].plan->p;
  for (const SeqUnit& U : units) {
    if (U.plan->dims != dims || U.plan->p != p) {
      set_error("batched apply: every plan must have the same dims and l_max");
      return PHIKRON_EINVAL;
    }
  }
  if (2 * ninst > MAX_PTRS) {
    set_error("batched apply: at most 64 plans");
    return PHIKRON_EINVAL;
  }
  S.p = p;
  S.half = cfg.half;
  S.ninst = ninst;
  // the longest wait limit any plan of the sequence asks for (0 = the default 2 s)
  unsigned long long wait_us = 0;
  for (const SeqUnit& U : units) {
    const unsigned long long w = U.plan->opts.wait_us > 0 ? (unsigned long long)U.plan->opts.wait_us : 2000000ull;
    wait_us = std::max(wait_us, w);
  }
  S.wait_ns = wait_us * 1000ull;
  // per-unit exponent slots
  std::vector<int> slot0(nu);
  for (int u = 0; u < nu; ++u) {
    const Plan& P = *units[u].plan;
    slot0[u] = B.nslots;
    const int nv = P.m + 2;
    B.nslots += 1 + nv * dims + p + P.s * (dims * p + p) + 8;
  }
  // placeholders for device pointers: slots are resolved after allocation (offsets now)
  PK_RET(seq_alloc(S, (void**)&S.dSlots, sizeof(int) * B.nslots));
  PK_RET(seq_alloc(S, (void**)&S.dPtrtab, sizeof(void*) * MAX_PTRS));
  PK_RET(seq_alloc(S, (void**)&S.dStatus, sizeof(int)));
  PK_TRY_CUDA(cudaMemset(S.dStatus, 0, sizeof(int)));
  S.nslots = B.nslots;
  int* slots = S.dSlots;

  struct UState {
    int next;              // next free slot
    int vslot;
    float2* Y;
    float2* Yn;
    int yslot;
  };
  std::vector<UState> us(nu);
  for (int u = 0; u < nu; ++u) {
    us[u].next = slot0[u];
    us[u].vslot = us[u].next++;
    us[u].Y = units[u].Y;
    us[u].Yn = units[u].Yn;
  }
  const long long out_mult = (long long)(p + 1) * (cfg.half ? 2 : 1);

  // 1. exponent scan of every input vector
  {
    std::vector<EJob> ej;
    for (int u = 0; u < nu; ++u) {
      const Plan& P = *units[u].plan;
      EJob j{};
      j.N = P.PN;
      j.v_tab = 2 * units[u].inst;
      j.tab_off_v = (long long)units[u].rhs * P.PN * 8;
      j.out_tab = j.out2_tab = -1;
      j.out_exp = slots + us[u].vslot;
      ej.push_back(j);
    }
    B.ew_step(STEP_EXPSCAN, ej, p);
  }

  // generic Kronecker chain over a list of (unit, matrix index, input, output) vectors
  struct CV {
    int u, mat;
    const void* in;        // direct input (pass 0) or null for table input
    int in_slot;
    bool in_tab;           // pass-0 input is V (table)
    int vec;               // index of the vector within the unit's W buffers
    void* out;             // final destination (direct) or null for table output
    bool out_tab;
    long long out_off;     // byte offset within Out (table) when out_tab
    bool out_f64;
    int out_slot;          // -1 none
  };
  // passes d < npass of the chain (all when npass = dims); cur_out receives the exponent slot
  // of every vector after the last pass run
  auto chain = [&](const std::vector<CV>& vs, bool first_f64, int npass, std::vector<int>* cur_out) -> int {
    std::vector<int> cur(vs.size());
    for (size_t q = 0; q < vs.size(); ++q) cur[q] = vs[q].in_slot;
    for (int d = 0; d < npass; ++d) {
      const bool last = (d == dims - 1);
      std::vector<GJob> jobs;
      std::vector<int> newslot(vs.size(), -1);
      bool trans = false;
      for (size_t q = 0; q < vs.size(); ++q) {
        const CV& c = vs[q];
        const Plan& P = *units[c.u].plan;
        long long B0 = 1, R = 1;
        for (int e = 0; e < d; ++e) B0 *= P.pn[e];
        for (int e = d + 1; e < dims; ++e) R *= P.pn[e];
        trans = R > 1;
        const MixedView mv = mixed_view(P, d);
        const long long N = P.PN;
        float2* dst = (d % 2 == 0) ? units[c.u].W1 : units[c.u].W2;
        const float2* src = (d % 2 == 0) ? units[c.u].W2 : units[c.u].W1;
        GJob j{};
        j.n = P.pn[d];
        j.R = R;
        j.B0 = B0;
        j.eslices = mv.sl + mv.mat_bytes * (size_t)c.mat;
        j.rexp = mv.rexp + (size_t)mv.rexp_stride * c.mat;
        j.in_tab = -1;
        j.out_tab = -1;
        if (d == 0) {
          if (c.in_tab) {
            j.in_tab = 2 * units[c.u].inst;
            j.tab_off_in = (long long)units[c.u].rhs * N * 8;
          } else {
            j.in = c.in;
          }
        } else {
          j.in = src + (size_t)c.vec * N;
        }
        j.in_exp = slots + cur[q];
        if (last) {
          if (c.out_tab) {
            j.out_tab = 2 * units[c.u].inst + 1;
            j.tab_off_out = (long long)units[c.u].rhs * out_mult * N * 8 + c.out_off;
          } else {
            j.out = c.out;
          }
          j.out_f64 = c.out_f64 ? 1 : 0;
          j.out_exp = c.out_slot >= 0 ? slots + c.out_slot : nullptr;
        } else {
          j.out = dst + (size_t)c.vec * N;
          j.out_f64 = 0;
          newslot[q] = us[c.u].next++;
          j.out_exp = slots + newslot[q];
        }
        jobs.push_back(j);
      }
      PassShape sh;
      sh.slices = cfg.slices;
      sh.sub = cfg.sub;
      sh.grid = cfg.grid;
      sh.in_f64 = (d == 0) && first_f64;
      sh.trans = trans;
      sh.ws = cfg.ws;
      sh.pc = false;
      // the double-buffered kernel keeps two 32-wide chunks of a job in flight: n >= 64 in
      // every job of the pass; smaller factors take the warp-specialised kernel
      int minn = 1 << 30;
      for (const GJob& j : jobs) minn = std::min(minn, j.n);
      sh.db = cfg.db && minn >= 64;
      // the raw ring's bulk copies read float-float inputs through direct, 16-byte aligned
      // pointers (the library's own buffers), in runs whose lengths and offsets are multiples
      // of 16 bytes: n (and R on transposed passes) multiples of 16
      bool direct16 = true;
      for (const GJob& j : jobs)
        direct16 = direct16 && j.in_tab < 0 && (reinterpret_cast<uintptr_t>(j.in) & 15u) == 0 && j.n % 16 == 0 &&
                   (!trans || j.R % 16 == 0);
      // (the warp-specialised raw-ring kernel up to 5 slices, the double-buffered one up to 4)
      sh.rr = cfg.rr && (sh.db ? cfg.slices <= 4 : (cfg.ws && cfg.slices <= 5)) && !sh.in_f64 && direct16;
      if (dims == 1) sh.trans = false;
      // all jobs of one pass share the formulation (same axis d)
      // the float64 first pass of a chain whose vectors share their unit's input: that input's
      // digit slices are cut once per unit (into the unit's second work buffer, which the pass
      // does not write) instead of once per job
      if (sh.in_f64 && sh.trans && !sh.db && cfg.ws && precut_default()) {
        std::vector<GJob> pj;
        std::vector<int> unit_pj(nu, -1);
        bool ok = true;
        for (size_t q = 0; q < vs.size() && ok; ++q) {
          GJob& j = jobs[q];
          const int u = vs[q].u;
          const Plan& P = *units[u].plan;
          const size_t cap = sizeof(float2) * (size_t)std::max(P.m + 2, std::max(P.p, 1)) * (size_t)P.PN;
          ok = vs[q].in_tab && j.B0 == 1 && tc::precut_bytes(j.R, j.n, cfg.slices) <= cap;
          if (!ok) break;
          if (unit_pj[u] < 0) {
            unit_pj[u] = (int)pj.size();
            GJob c = j;
            c.xslices = reinterpret_cast<const uint8_t*>(units[u].W2);
            pj.push_back(c);
          }
          j.xslices = reinterpret_cast<const uint8_t*>(units[u].W2);
        }
        if (ok) {
          B.precut_step(pj, cfg.slices);
          sh.pc = true;
        } else {
          for (GJob& j : jobs) j.xslices = nullptr;
        }
      }
      B.mode_step(jobs, sh);
      if (sh.rr) {
        Step& stp = B.steps.back();
        const size_t off = B.tmaps.size();
        B.tmaps.resize(off + 128 * (size_t)stp.count);
        if (tc::encode_raw_maps(B.gjobs.data() + stp.off, stp.count, sh.trans, sh.db ? 64 : 128, B.tmaps.data() + off) ==
            PHIKRON_OK) {
          stp.tmap_off = (long long)(off / 128);
        } else {   // no tensor maps: the register-loading kernel
          B.tmaps.resize(off);
          stp.shape.rr = false;
        }
      }
      for (size_t q = 0; q < vs.size(); ++q)
        if (newslot[q] >= 0) cur[q] = newslot[q];
    }
    if (cur_out) *cur_out = cur;
    return PHIKRON_OK;
  };

  // 2. node phase: m node actions (to T), phi_0 (to Out[0]), half-step phi_0 (to Out[p+1]).
  // Fused: the last pass of the chain runs as one fused pass that folds Algorithm 1's weights
  // into its epilogue (fused.cu) and writes y_1..y_p itself; needs a float-float last pass (dims
  // >= 2) over a factor of at most FW_MAXN rows and 1 <= p <= FW_MAXP.
  bool fuse = cfg.fuse && p >= 1 && p <= FW_MAXP && dims >= 2;
  for (int u = 0; u < nu && fuse; ++u)
    if (units[u].plan->pn[dims - 1] > FW_MAXN) fuse = false;
  S.fused = fuse;
  std::vector<float2*> T(nu);
  std::vector<int> tslot(nu);
  {
    std::vector<CV> vs;
    for (int u = 0; u < nu; ++u) {
      const Plan& P = *units[u].plan;
      T[u] = (dims % 2 == 1) ? units[u].W1 : units[u].W2;
      tslot[u] = us[u].next;
      us[u].next += P.m;
      for (int k = 0; k < P.m; ++k)
        vs.push_back(CV{u, k, nullptr, us[u].vslot, true, k, T[u] + (size_t)k * P.PN, false, 0, false, tslot[u] + k});
      if (!P.opts.skip_phi0)
        vs.push_back(CV{u, P.m, nullptr, us[u].vslot, true, P.m, nullptr, true, 0, true, -1});
      if (cfg.half && !P.opts.skip_phi0)
        vs.push_back(CV{u, P.m + P.s, nullptr, us[u].vslot, true, P.m + 1, nullptr, true,
                        (long long)(p + 1) * P.PN * 8, true, -1});
    }
    if (!fuse) {
      PK_RET(chain(vs, true, dims, nullptr));
    } else {
      std::vector<int> cur;
      PK_RET(chain(vs, true, dims - 1, &cur));
      // the fused last pass: one job per unit over its nodes (weighted first, then direct)
      std::vector<FJob> fj;
      std::vector<FNode> fn;
      size_t q = 0;
      const int dl = dims - 1;
      for (int u = 0; u < nu; ++u) {
        const Plan& P = *units[u].plan;
        const MixedView mv = mixed_view(P, dl);
        const float2* src = (dl % 2 == 1) ? units[u].W1 : units[u].W2;   // written by pass dl - 1
        FJob j{};
        j.n = P.pn[dl];
        j.B0 = P.PN / P.pn[dl];
        j.node0 = (int)fn.size();
        j.m = P.m;
        j.coef = mv.coef;
        j.stride = P.PN;
        j.out_tab = j.out2_tab = -1;
        if (P.s == 0) {
          j.out_tab = 2 * units[u].inst + 1;
          j.tab_off_out = (long long)units[u].rhs * out_mult * P.PN * 8 + (long long)P.PN * 8;
          j.out_f64 = 1;
        } else {
          j.out = us[u].Y;
          us[u].yslot = us[u].next;
          us[u].next += p;
          j.out_exp = slots + us[u].yslot;
        }
        if (cfg.half && P.s == 1) {
          j.out2_tab = 2 * units[u].inst + 1;
          j.tab_off_out2 = (long long)units[u].rhs * out_mult * P.PN * 8 + (long long)(p + 2) * P.PN * 8;
        }
        // the vectors of this unit in vs are contiguous, in the order pushed above
        for (; q < vs.size() && vs[q].u == u; ++q) {
          const CV& c = vs[q];
          FNode nd{};
          nd.in = src + (size_t)c.vec * P.PN;
          nd.in_exp = slots + cur[q];
          nd.eslices = mv.sl + mv.mat_bytes * (size_t)c.mat;
          nd.rexp = mv.rexp + (size_t)mv.rexp_stride * c.mat;
          nd.out_tab = -1;
          if (c.out_tab) {   // phi_0 (or phi_0 at tau/2): stored as it is, float64
            nd.direct = 1;
            nd.out_tab = 2 * units[u].inst + 1;
            nd.tab_off_out = (long long)units[u].rhs * out_mult * P.PN * 8 + c.out_off;
          } else {
            nd.direct = 0;
            nd.k = c.mat;
          }
          fn.push_back(nd);
        }
        j.nnodes = (int)fn.size() - j.node0;
        fj.push_back(j);
      }
      PassShape sh{};
      sh.slices = cfg.slices;
      sh.grid = cfg.grid;
      B.fused_step(fj, fn, sh, p);
    }
  }
  if (p >= 1) {
    // 3. weighted sums (already written by the fused pass when it ran)
    std::vector<EJob> ej;
    for (int u = 0; u < nu && !fuse; ++u) {
      const Plan& P = *units[u].plan;
      const MixedView mv = mixed_view(P, 0);
      EJob j{};
      j.a = T[u];
      j.coef = mv.coef;
      j.m = P.m;
      j.N = P.PN;
      j.stride = P.PN;
      j.out_tab = j.out2_tab = -1;
      if (P.s == 0) {
        j.out_tab = 2 * units[u].inst + 1;
        j.tab_off_out = (long long)units[u].rhs * out_mult * P.PN * 8 + (long long)P.PN * 8;
        j.out_f64 = 1;
      } else {
        j.out = us[u].Y;
        us[u].yslot = us[u].next;
        us[u].next += p;
        j.out_exp = slots + us[u].yslot;
      }
      if (cfg.half && P.s == 1) {
        j.out2_tab = 2 * units[u].inst + 1;
        j.tab_off_out2 = (long long)units[u].rhs * out_mult * P.PN * 8 + (long long)(p + 2) * P.PN * 8;
      }
      ej.push_back(j);
    }
    B.ew_step(STEP_WEIGHTED, ej, p);
    // 4. squaring steps (units with s > t take part in step t)
    int smax = 0;
    for (int u = 0; u < nu; ++u) smax = std::max(smax, units[u].plan->s);
    for (int t = 0; t < smax; ++t) {
      std::vector<CV> vs;
      std::vector<int> part;
      for (int u = 0; u < nu; ++u) {
        const Plan& P = *units[u].plan;
        if (P.s <= t) continue;
        part.push_back(u);
        float2* Z = (dims % 2 == 1) ? units[u].W1 : units[u].W2;
        for (int i = 0; i < p; ++i)
          vs.push_back(CV{u, P.m + 1 + t, us[u].Y + (size_t)i * P.PN, us[u].yslot + i, false, i,
                          Z + (size_t)i * P.PN, false, 0, false, -1});
      }
      PK_RET(chain(vs, false, dims, nullptr));
      std::vector<EJob> sj;
      for (int u : part) {
        const Plan& P = *units[u].plan;
        EJob j{};
        j.a = (dims % 2 == 1) ? units[u].W1 : units[u].W2;
        j.b = us[u].Y;
        j.N = P.PN;
        j.stride = P.PN;
        j.out_tab = j.out2_tab = -1;
        const bool lastt = (t == P.s - 1);
        if (lastt) {
          j.out_tab = 2 * units[u].inst + 1;
          j.tab_off_out = (long long)units[u].rhs * out_mult * P.PN * 8 + (long long)P.PN * 8;
          j.out_f64 = 1;
        } else {
          j.out = us[u].Yn;
          const int ns = us[u].next;
          us[u].next += p;
          j.out_exp = slots + ns;
          us[u].yslot = ns;
        }
        if (cfg.half && t == P.s - 2) {
          j.out2_tab = 2 * units[u].inst + 1;
          j.tab_off_out2 = (long long)units[u].rhs * out_mult * P.PN * 8 + (long long)(p + 2) * P.PN * 8;
        }
        sj.push_back(j);
        if (!lastt) std::swap(us[u].Y, us[u].Yn);
      }
      B.ew_step(STEP_SQUARING, sj, p);
    }
  }
  for (int u = 0; u < nu; ++u) {
    const Plan& P = *units[u].plan;
    const int cap = slot0[u] + 1 + (P.m + 2) * dims + p + P.s * (dims * p + p) + 8;
    if (us[u].next > cap) {
      set_error("sequence builder: exponent slot overflow");
      return PHIKRON_EINVAL;
    }
  }
  // upload the job tables
  PK_RET(seq_alloc(S, (void**)&S.dG, sizeof(GJob) * std::max<size_t>(1, B.gjobs.size())));
  PK_RET(seq_alloc(S, (void**)&S.dE, sizeof(EJob) * std::max<size_t>(1, B.ejobs.size())));
  PK_RET(seq_alloc(S, (void**)&S.dF, sizeof(FJob) * std::max<size_t>(1, B.fjobs.size())));
  PK_RET(seq_alloc(S, (void**)&S.dFN, sizeof(FNode) * std::max<size_t>(1, B.fnodes.size())));
  if (!B.tmaps.empty()) {
    PK_RET(seq_alloc(S, (void**)&S.dTmaps, B.tmaps.size()));
    PK_TRY_CUDA(cudaMemcpy(S.dTmaps, B.tmaps.data(), B.tmaps.size(), cudaMemcpyHostToDevice));
  }
  if (!B.fjobs.empty())
    PK_TRY_CUDA(cudaMemcpy(S.dF, B.fjobs.data(), sizeof(FJob) * B.fjobs.size(), cudaMemcpyHostToDevice));
  if (!B.fnodes.empty())
    PK_TRY_CUDA(cudaMemcpy(S.dFN, B.fnodes.data(), sizeof(FNode) * B.fnodes.size(), cudaMemcpyHostToDevice));
  if (!B.gjobs.empty())
    PK_TRY_CUDA(cudaMemcpy(S.dG, B.gjobs.data(), sizeof(GJob) * B.gjobs.size(), cudaMemcpyHostToDevice));
  if (!B.ejobs.empty())
    PK_TRY_CUDA(cudaMemcpy(S.dE, B.ejobs.data(), sizeof(EJob) * B.ejobs.size(), cudaMemcpyHostToDevice));
  S.steps = B.steps;
  S.njobs_mode = B.gjobs.size();
  // capture the sequence as a CUDA graph
  if (cfg.graph) {
    cudaStream_t cs;
    PK_TRY_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
    ProfScope none(nullptr);
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    int rc = PHIKRON_OK;
    if (e == cudaSuccess) rc = seq_launch_all(S, cs);
    cudaError_t e2 = cudaStreamEndCapture(cs, &g);
    if (e == cudaSuccess && rc == PHIKRON_OK && e2 == cudaSuccess && g) {
      e = cudaGraphInstantiate(&S.exec, g, 0);
      if (e != cudaSuccess) S.exec = nullptr;
    }
    if (g) cudaGraphDestroy(g);
    cudaStreamDestroy(cs);
    cudaGetLastError();
    clear_error();
  }
  return PHIKRON_OK;
}

int seq_launch_all(Seq& S, cudaStream_t st) {
  PK_TRY_CUDA(cudaMemsetAsync(S.dSlots, 0x80, sizeof(int) * S.nslots, st));
  for (const Step& s : S.steps) {
    if (s.kind == STEP_MODE) {
      GPass P;
      P.jobs = S.dG + s.off;
      P.njobs = s.count;
      P.total_tiles = s.total;
      P.ptrtab = S.dPtrtab;
      P.wait_ns = S.wait_ns;
      P.tmaps = (s.tmap_off >= 0) ? S.dTmaps + 128 * s.tmap_off : nullptr;
      PK_RET(tc::mode_pass(P, s.shape, S.dStatus, st));
    } else if (s.kind == STEP_FUSED) {
      FPass F;
      F.jobs = S.dF + s.off;
      F.nodes = S.dFN;
      F.njobs = s.count;
      F.total_tiles = s.total;
      F.ptrtab = S.dPtrtab;
      F.wait_ns = S.wait_ns;
      PK_RET(fused::launch(F, s.shape.slices, s.p, s.shape.grid, S.dStatus, st));
    } else if (s.kind == STEP_PRECUT) {
      GPass P;
      P.jobs = S.dG + s.off;
      P.njobs = s.count;
      P.total_tiles = s.total;
      P.ptrtab = S.dPtrtab;
      P.wait_ns = S.wait_ns;
      P.tmaps = nullptr;
      PK_RET(tc::precut_pass(P, s.shape.slices, S.dStatus, st));
    } else if (s.kind == STEP_EXPSCAN) {
      launch_begin(KC_CONVERT, st);
      g_expscan_kernel<<<ew_grid(g_expscan_kernel, s.total), EW_THREADS, 0, st>>>(S.dE + s.off, s.count, s.total,
                                                                                  S.dPtrtab);
      launch_end(st);
      PK_CHECK_LAUNCH();
    } else {
      PK_RET(launch_ew_p(s.kind, s.p, S.dE + s.off, s.count, s.total, S.dPtrtab, st));
    }
  }
  return PHIKRON_OK;
}

int seq_run(Seq& S, const PtrArgs& args, cudaStream_t st) {
  PK_RET(tc::set_ptrtab(S.dPtrtab, args, st));
  Profiler* pr = tl_prof;
  if (S.exec && !(pr && pr->timing)) {
    PK_TRY_CUDA(cudaGraphLaunch(S.exec, st));
    if (pr) {
      pr->launches += (long long)S.steps.size();
      for (const Step& s : S.steps)
        pr->launches_by_class[(s.kind == STEP_MODE || s.kind == STEP_FUSED) ? KC_TC_MODE
                              : s.kind == STEP_WEIGHTED ? KC_WEIGHTED
                              : s.kind == STEP_SQUARING ? KC_SQUARING : KC_CONVERT]++;
    }
    return PHIKRON_OK;
  }
  return seq_launch_all(S, st);
}

int seq_status(Seq& S, int* status) {
  PK_TRY_CUDA(cudaMemcpy(status, S.dStatus, sizeof(int), cudaMemcpyDeviceToHost));
  PK_TRY_CUDA(cudaMemset(S.dStatus, 0, sizeof(int)));
  return PHIKRON_OK;
}

}  // namespace phikron
