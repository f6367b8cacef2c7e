// K2 (mixed precision): mode products of Eq. (8) on the tcgen05 tensor cores with exact
// BF16 slice products (Ozaki-style splitting), accumulated in TMEM.
//
// A mode product out[b][i0][i][r] = sum_k E[i][k] in[b][i0][k][r] is computed with both
// operands cut into KS "digit" slices:
//   in  ~ 2^{eX}   * sum_t x_t,  x_t = integer * 2^{-8t}, |integer| <= 256   (per-vector
//        exponent eX; float64 input: the sign-magnitude digits of |in| 2^{-eX} rounded to
//        nearest at digit KS, cut with integer ops; float-float input: signed digits from
//        FP32 round-to-nearest remainders)
//   E   ~ 2^{f_i}  * sum_s e_s,  e_s likewise                           (per-row exponent f_i)
// Every slice value is exactly representable in BF16.  The slice pairs (s, t) with
// s + t <= KS + 1 are multiplied on the tensor cores (kind::f16, BF16 inputs, FP32
// accumulation): level 2 = (1,1) and level 3 = (1,2)+(2,1) sums are exact in FP32 (at most
// 2 * 255^2 * 128 < 2^24), level 4 has its own accumulator (rounding 2^-24 of a
// 2^-16-relative term) and levels >= 5 share a fourth (2^-24 of 2^-24).  Four accumulators
// of 128 FP32 columns fill the 512 TMEM columns.  A single accumulator for levels >= 4
// would take ~K/16 * (#pairs) FP32 roundings of a 2^-16-relative term per output and
// leave a ~1e-10 floor.  The epilogue adds the accumulators in float-float (compensated
// FP32) arithmetic and scales by 2^{eX + f_i}.  Result accuracy per product is
// about 2^{1-8 KS} relative to ||E||_inf max|in|: KS = 3 ~ FP32, KS = 5 ~ 1e-12.
//
// No float64 arithmetic runs per element (GB300 executes float64 at ~1/64 of FP32): float64
// digits are cut from the bit patterns with integer shifts, float-float digits with FP32
// adds, and the state between passes is float-float (hi, lo) FP32 pairs.
//
// Two formulations share one kernel:
//   TRANS (R > 1, contraction over a non-fastest axis):  D[r][i] = sum_k X^T[r][k] E[i][k]
//       A = X^T tile (128 r-rows, K-major, transposed while slicing), B = E (n rows).
//       TMEM lane = r, column = i; stores out[i][r] coalesced over lanes.
//   NORMAL (R = 1, contraction over the fastest axis):   D[i][row] = sum_k E[i][k] X[row][k]
//       A = E (128 rows, zero-padded), B = X tile (128 rows).  TMEM lane = i, column = row;
//       stores out[row][i] coalesced over lanes.
// K (= n) is processed in chunks of 32 through a shared-memory ring of stages (two in the
// single-role kernel, up to three in the warp-specialised ones): while the tensor cores work
// on chunk c, the producer threads cut the next chunks (with the raw values of the following
// chunk -- or of the next tile's first chunk -- already in flight), and the E slices of each
// chunk arrive by one asynchronous bulk copy (TMA).  Operands use
// the 64-byte-swizzled K-major layout (one 64-byte row of 32 BF16 per operand row, its four
// 16-byte pieces permuted by bits 1-2 of the row; SBO = 512 B between 8-row groups); the
// no-swizzle canonical layout (8-row x 16-byte core matrices, LBO = 128 B) remains
// selectable through kSwizzle64.  The warp-specialised and double-buffered variants below
// are the ones the library launches by default.
//
// Every wait on an mbarrier is bounded; on expiry the kernel records PHIKRON_ETIMEOUT in the
// status word, waits (bounded) for its own tensor-core work, frees its TMEM and returns.
#include <algorithm>
#include <cstdint>
#include <cstring>

#include <cuda.h>

#include "checked.cuh"
#include "common.h"
#include "mixed.h"
#include "profile.h"
#include "tc_common.cuh"

PK_CHK_BIND(tc_mode)

namespace phikron {
namespace tc {

namespace {

constexpr int NTHREADS = 512;

// Bounds-checked build: a launch whose job table or pointer table is not registered does
// nothing (every thread of the CTA decides alike, before any barrier or TMEM allocation).
#ifdef PHIKRON_CHECKED
#define PK_CHECK_TABLES(P)                                                                  \
  if (!PK_CK((P).jobs, sizeof(GJob) * (size_t)(P).njobs, chk::SITE_TABLE) ||                  \
      ((P).ptrtab && !PK_CK((P).ptrtab, sizeof(void*) * MAX_PTRS, chk::SITE_TABLE)))          \
    return;
#else
#define PK_CHECK_TABLES(P)
#endif

using chk::st_ck;

// input / output base of a job: direct, or a pointer-table entry plus offset
__device__ __forceinline__ const void* job_in(const GPass& P, const GJob& J) {
  if (J.in_tab < 0) return J.in;
  if (!PK_CK(P.ptrtab + J.in_tab, sizeof(void*), chk::SITE_TABLE)) return nullptr;
  return (const void*)((const char*)P.ptrtab[J.in_tab] + J.tab_off_in);
}

__device__ __forceinline__ void* job_out(const GPass& P, const GJob& J) {
  if (J.out_tab < 0) return J.out;
  if (!PK_CK(P.ptrtab + J.out_tab, sizeof(void*), chk::SITE_TABLE)) return nullptr;
  return (void*)((char*)P.ptrtab[J.out_tab] + J.tab_off_out);
}

// exponent of a job's input (all-zero input: 0)
__device__ __forceinline__ int job_in_exp(const GJob& J) {
  const int eX = PK_CK(J.in_exp, sizeof(int), chk::SITE_MODE_EXP) ? *J.in_exp : -1000;
  return eX < -600 ? 0 : eX;
}

__device__ __forceinline__ void out_exp_max(int* out_exp, int v) {
  if (out_exp && PK_CK(out_exp, sizeof(int), chk::SITE_MODE_EXP)) atomicMax(out_exp, v);
}

// Raw operand values of one thread for one 32-wide K sub-chunk: 8 consecutive k of its row.
template <bool IN_F64>
struct Raw {
  double d[IN_F64 ? 8 : 1];
  float2 f[IN_F64 ? 1 : 8];
};

struct TileCtx {
  int job;
  int rb;            // which 128-row block of E (n > 128)
  int n, nsub;         // contracted size, number of 32-wide K sub-chunks
  long long R, B0;
  long long b0, r0, row0;
  int eX;
  long long in_base, gr;
  bool valid_row;
  const void* in;
  void* out;
};

__device__ __forceinline__ int find_job(const GPass& P, long long tile) {
  int lo = 0, hi = P.njobs - 1;  // last job with tile_begin <= tile
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (P.jobs[mid].tile_begin <= tile) lo = mid; else hi = mid - 1;
  }
  return lo;
}

template <bool TRANS>
__device__ __forceinline__ TileCtx tile_ctx(const GPass& P, long long tile, int orow) {
  TileCtx t;
  t.job = find_job(P, tile);
  const GJob& J = P.jobs[t.job];
  t.n = J.n;
  t.nsub = (J.n + 31) / 32;
  t.R = J.R;
  t.B0 = J.B0;
  const long long tj = tile - J.tile_begin;
  const long long rtiles = TRANS ? (J.R + 127) / 128 : 1;
  const long long per_rb = TRANS ? J.B0 * rtiles : (J.B0 + 127) / 128;
  t.rb = (int)(tj / per_rb);
  const long long th = tj % per_rb;
  t.b0 = t.r0 = t.row0 = 0;
  if (TRANS) {
    t.b0 = th / rtiles;
    t.r0 = (th % rtiles) * 128;
  } else {
    t.row0 = th * 128;
  }
  t.eX = job_in_exp(J);
  t.in_base = TRANS ? t.b0 * (long long)J.n * J.R : 0;
  t.gr = TRANS ? t.r0 + orow : t.row0 + orow;
  t.valid_row = TRANS ? (t.gr < J.R) : (t.gr < J.B0);
  t.in = job_in(P, J);
  t.out = job_out(P, J);
  return t;
}

template <bool IN_F64, bool TRANS>
__device__ __forceinline__ void load_raw(const TileCtx& t, int sub, int kq, Raw<IN_F64>& raw) {
#pragma unroll
  for (int e = 0; e < 8; ++e) {
    const int k = sub * 32 + kq * 8 + e;
    const long long idx = TRANS ? t.in_base + (long long)k * t.R + t.gr : t.gr * (long long)t.n + k;
    const bool ok = t.valid_row && k < t.n && PK_CK((const char*)t.in + 8 * idx, 8, chk::SITE_MODE_LOAD);
    if (IN_F64)
      raw.d[e] = ok ? __ldg(reinterpret_cast<const double*>(t.in) + idx) : 0.0;
    else
      raw.f[e] = ok ? __ldg(reinterpret_cast<const float2*>(t.in) + idx) : make_float2(0.f, 0.f);
  }
}

// One tile = 128 operand rows (r for TRANS, X rows for NORMAL) x one 128-row block of E,
// accumulated over the full contraction K = n in chunks of 32*SUB.
template <int KS, int SUB, bool IN_F64, bool TRANS>
__global__ void __launch_bounds__(NTHREADS, 1) mode_kernel(const __grid_constant__ GPass P, int* status) {
  PK_CHECK_TABLES(P);
  const unsigned long long wl = P.wait_ns;  // limit of every bounded wait
  extern __shared__ __align__(1024) uint8_t smem[];
  // [stage 0: X slices SUB*KS*8K | E slices SUB*KS*8K][stage 1: ...][mbarriers][scales][tmem]
  constexpr int HALF_BYTES = SUB * KS * SLICE_BYTES;
  constexpr int STAGE_BYTES = 2 * HALF_BYTES;
  uint64_t* mbar_mma = reinterpret_cast<uint64_t*>(smem + 2 * STAGE_BYTES);   // 2: MMAs of stage done
  uint64_t* mbar_e = mbar_mma + 2;                                             // 2: E slices of stage landed
  float* scale_s = reinterpret_cast<float*>(smem + 2 * STAGE_BYTES + 64);     // 128 floats: 2^{eX + f_i}
  uint32_t* tmem_s = reinterpret_cast<uint32_t*>(smem + 2 * STAGE_BYTES + 64 + 512);

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int orow = tid & 127;   // operand row owned by this thread (r for TRANS, row for NORMAL)
  const int kq = tid >> 7;      // which 8 of each 32-wide sub-chunk this thread cuts
  const long long total_tiles = P.total_tiles;

  if (tid == 0) {
    for (int q = 0; q < 4; ++q) asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mbar_mma[q])));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_s)),
                 "r"(512));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tmem_s;

  uint32_t it = 0;          // global chunk counter (stage = it & 1, use = it >> 1)
  bool aborted = false;
  int fail = 0;             // thread 0: an E-slice wait expired
  long long e_issued = -1, mma_issued = -1;  // thread 0: chunk of the latest E copy / MMA commit

  long long tile = blockIdx.x;
  TileCtx T;
  Raw<IN_F64> raw[SUB];
  if (tile < total_tiles) {
    T = tile_ctx<TRANS>(P, tile, orow);
#pragma unroll
    for (int q = 0; q < SUB; ++q) load_raw<IN_F64, TRANS>(T, q, kq, raw[q]);
  }
  for (; tile < total_tiles && !aborted; tile += gridDim.x) {
    const GJob& J = P.jobs[T.job];
    const int n = T.n;
    const int nchunks = (T.nsub + SUB - 1) / SUB;
    const int nrows_e = min(128, n - 128 * T.rb);   // E rows in this row block
    const uint8_t* ebase = J.eslices + (size_t)T.rb * (size_t)T.nsub * KS * SLICE_BYTES;
    if (tid < 128) {
      const int* rx = J.rexp + T.rb * 128 + tid;
      const int E = T.eX + ((tid < nrows_e && PK_CK(rx, sizeof(int), chk::SITE_MODE_REXP)) ? *rx : 0);
      scale_s[tid] = pow2f(E);
    }
    const uint32_t idesc = TRANS ? make_idesc(128, nrows_e) : make_idesc(128, 128);
    const int eb = 1011 + T.eX;           // float64 input: integer digit cutting
    const float xsc = pow2f_full(-T.eX);  // float-float input: FP32 slicing of X 2^{-eX}
    bool init[4] = {false, false, false, false};
    TileCtx Tn = T;
    const long long next_tile = tile + gridDim.x;
    for (int c = 0; c < nchunks; ++c, ++it) {
      const uint32_t st = it & 1u;
      uint8_t* sX = smem + st * STAGE_BYTES;
      uint8_t* sE = sX + HALF_BYTES;
      const int nsub_c = min(SUB, T.nsub - c * SUB);   // sub-chunks in this chunk
      int timed_out = fail;
      if (it >= 2) timed_out |= mbar_wait(smem_u32(&mbar_mma[st]), ((it >> 1) - 1) & 1u, wl) ? 0 : 1;
      if (__syncthreads_or(timed_out)) {  // block-uniform decision
        aborted = true;
        break;
      }
      if (tid == 0) {  // E slices of this chunk: one asynchronous bulk copy ([sub][slice][8 KB])
        const uint32_t bytes = (uint32_t)(nsub_c * KS * SLICE_BYTES);
        mbar_expect_tx(smem_u32(&mbar_e[st]), bytes);
        bulk_copy_g2s(smem_u32(sE), PK_CK_SRC(ebase + (size_t)c * SUB * KS * SLICE_BYTES, bytes, chk::SITE_MODE_ECOPY),
                      bytes, smem_u32(&mbar_e[st]));
        e_issued = it;
      }
      // raw values of the next chunk (or of the next tile's first chunk) go in flight now
      Raw<IN_F64> rawn[SUB];
      if (c + 1 < nchunks) {
#pragma unroll
        for (int q = 0; q < SUB; ++q)
          if ((c + 1) * SUB + q < T.nsub) load_raw<IN_F64, TRANS>(T, (c + 1) * SUB + q, kq, rawn[q]);
      } else if (next_tile < total_tiles) {
        Tn = tile_ctx<TRANS>(P, next_tile, orow);
#pragma unroll
        for (int q = 0; q < SUB; ++q)
          if (q < Tn.nsub) load_raw<IN_F64, TRANS>(Tn, q, kq, rawn[q]);
      }
#pragma unroll
      for (int q = 0; q < SUB; ++q) {
        if (q >= nsub_c) break;
        uint32_t pk[KS][4];
#pragma unroll
        for (int e = 0; e < 8; e += 2) {
          if (IN_F64) {
            uint32_t s0, s1;
            const uint64_t F0 = round_digits<KS>(fixed_f64(raw[q].d[e], eb, s0));
            const uint64_t F1 = round_digits<KS>(fixed_f64(raw[q].d[e + 1], eb, s1));
            uint32_t w[KS];
            cut_pair<KS>(F0, s0, F1, s1, w);
#pragma unroll
            for (int sl = 0; sl < KS; ++sl) pk[sl][e >> 1] = w[sl];
          } else {
            float2 v[KS];
            cut_ff_float2<KS>(make_float2(raw[q].f[e].x, raw[q].f[e + 1].x), make_float2(raw[q].f[e].y, raw[q].f[e + 1].y), xsc, v);
#pragma unroll
            for (int sl = 0; sl < KS; ++sl) pk[sl][e >> 1] = pack_bf16x2(v[sl].x, v[sl].y);
          }
        }
        const uint32_t off = chunk_offset(orow, kq);
#pragma unroll
        for (int sl = 0; sl < KS; ++sl)
          *reinterpret_cast<uint4*>(sX + (q * KS + sl) * SLICE_BYTES + off) =
              make_uint4(pk[sl][0], pk[sl][1], pk[sl][2], pk[sl][3]);
      }
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      __syncthreads();
      if (tid == 0) {
        if (!mbar_wait(smem_u32(&mbar_e[st]), (it >> 1) & 1u, wl)) {
          fail = 1;  // E never landed: skip the MMAs; the next vote aborts the block
        } else {
          asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
          const uint32_t xa = smem_u32(sX), ea = smem_u32(sE);
          for (int q = 0; q < nsub_c; ++q) {
#pragma unroll
            for (int s = 1; s <= KS; ++s) {          // E slice
#pragma unroll
              for (int t = 1; t <= KS; ++t) {        // X slice
                if (s + t > KS + 1) continue;
                const int L = s + t - 2;
                const int a = L < 3 ? L : 3;
                const uint32_t dacc = tmem + (uint32_t)(a * 128);
#pragma unroll
                for (int ks = 0; ks < 2; ++ks) {
                  const uint32_t xs = xa + (uint32_t)((q * KS + t - 1) * SLICE_BYTES) + ks * KSTEP_BYTES;
                  const uint32_t es = ea + (uint32_t)((q * KS + s - 1) * SLICE_BYTES) + ks * KSTEP_BYTES;
                  const uint64_t xd = make_desc(xs), ed = make_desc(es);
                  if (TRANS)
                    mma_bf16(dacc, xd, ed, idesc, init[a] ? 1u : 0u);
                  else
                    mma_bf16(dacc, ed, xd, idesc, init[a] ? 1u : 0u);
                  init[a] = true;
                }
              }
            }
          }
          mma_commit(smem_u32(&mbar_mma[st]));
          mma_issued = it;
        }
      }
#pragma unroll
      for (int a = 0; a < 4; ++a) init[a] = true;
#pragma unroll
      for (int q = 0; q < SUB; ++q) raw[q] = rawn[q];
    }
    if (aborted) break;
    // epilogue: wait for the last chunk's MMAs (covers every earlier MMA of this tile)
    {
      const uint32_t lastit = it - 1;
      int to = fail;
      to |= mbar_wait(smem_u32(&mbar_mma[lastit & 1u]), (lastit >> 1) & 1u, wl) ? 0 : 1;
      if (__syncthreads_or(to)) aborted = true;
    }
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (!aborted) {
      // warps w, w+4, w+8, w+12 share TMEM lanes 32*(w%4)..+31 and split the columns
      const uint32_t lane_base = tmem + ((uint32_t)((warp & 3) * 32) << 16);
      const int lrow = (warp & 3) * 32 + lane;  // TMEM lane of this thread
      const int cq = warp >> 2;
      int emax = 0;
      const int ncols = TRANS ? ((nrows_e + 15) & ~15) : 128;
      const int ngroups = ncols / 16;
      const int gbeg = (cq * ngroups) / 4, gend = ((cq + 1) * ngroups) / 4;
      float2* outFF = reinterpret_cast<float2*>(T.out);
      double* outF64 = reinterpret_cast<double*>(T.out);
      const long long out_base = TRANS ? T.b0 * (long long)n * T.R : 0;
      const float lane_scale = TRANS ? 1.0f : scale_s[lrow];
      for (int gq = gbeg; gq < gend; ++gq) {
        const int cc = gq * 16;
        float d2[16], d3[16], d4[16], d5[16];
        tmem_ld16(lane_base + (uint32_t)cc, d2);
        tmem_ld16(lane_base + 128u + (uint32_t)cc, d3);
        tmem_ld16(lane_base + 256u + (uint32_t)cc, d4);
        if (KS >= 4) {
          tmem_ld16(lane_base + 384u + (uint32_t)cc, d5);
        } else {  // KS = 3 has no pair at level >= 5: the fourth accumulator is never written
#pragma unroll
          for (int j = 0; j < 16; ++j) d5[j] = 0.0f;
        }
        tmem_wait_ld();
#pragma unroll
        for (int j = 0; j < 16; ++j) {
          const int col = cc + j;
          int il, i;
          long long oidx;
          bool ok;
          float sc;
          if (TRANS) {
            il = col;
            i = 128 * T.rb + il;
            const long long g = T.r0 + lrow;
            ok = (il < nrows_e) && (g < T.R);
            oidx = out_base + (long long)i * T.R + g;
            sc = scale_s[il];
          } else {
            il = lrow;
            i = 128 * T.rb + il;
            const long long g = T.row0 + col;
            ok = (il < nrows_e) && (g < T.B0);
            oidx = g * (long long)n + i;
            sc = lane_scale;
          }
          if (!ok) continue;
          // full two-sums at every step: D4 + D5 spans ~31 bits for 6 digits (a plain FP32
          // add would round at 2^-42 of D2), and an element whose leading digit is small has
          // |D2| < |D3 + ...|, where a fast two-sum would lose the error term
          float t45, e45, u, eu, hi, eh;
          two_sum(d4[j], d5[j], t45, e45);
          two_sum(d3[j], t45, u, eu);
          two_sum(d2[j], u, hi, eh);
          float lo = eh + (eu + e45);
          fast_two_sum(hi, lo, hi, lo);
          hi *= sc;
          lo *= sc;
          if (J.out_f64)
            st_ck(outF64 + oidx, ff_to_f64(hi, lo), chk::SITE_MODE_STORE);
          else
            st_ck(outFF + oidx, make_float2(hi, lo), chk::SITE_MODE_STORE);
          emax = max(emax, (int)((__float_as_uint(hi) >> 23) & 0xFFu));
        }
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) emax = max(emax, __shfl_xor_sync(0xffffffffu, emax, o));
      // |v| < 2^{biased - 126}; a zero vector keeps the slot's initial (very negative) value
      if (lane == 0 && emax > 0) out_exp_max(J.out_exp, emax - 126);
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    T = Tn;
  }
  if (aborted && tid == 0) {
    atomicExch(status, PHIKRON_ETIMEOUT);
    // the latest E copy and the latest MMA commit (which covers every earlier MMA of this
    // thread) complete without any other CTA: wait for both before shared memory and TMEM
    // are released (no later arrival touches those phases)
    if (mma_issued >= 0)
      mbar_wait(smem_u32(&mbar_mma[mma_issued & 1]), (uint32_t)(mma_issued >> 1) & 1u, CLEANUP_WAIT_NS);
    if (e_issued >= 0)
      mbar_wait(smem_u32(&mbar_e[e_issued & 1]), (uint32_t)(e_issued >> 1) & 1u, CLEANUP_WAIT_NS);
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512));
}

// ---------------------------------------------------------------- warp-specialised variant
// Roles of the warp-specialised kernel (15 warps = 480 threads; 32-wide K chunks):
//   warps 0-7   producers: cut the operand digits of each chunk into the stage ring;
//               producer thread 0 also starts the chunk's E bulk copy
//   warps 8-11  epilogue: drain the four TMEM accumulators (warp 8+q owns TMEM lanes 32q..32q+31,
//               all columns), float-float, scale, store, exponent of the output
//   warps 12,14 lane 0 issues the tcgen05 MMAs of accumulators {0, 3} (warp 12) and {1, 2}
//               (warp 14)
//   warp 13     lane 0 resolves each tile's context (job lookup, input exponent, pointers) into a
//               4-slot shared-memory ring ahead of the other roles, so that no role waits on a
//               chain of dependent global loads at a tile boundary
// The double-buffered variant further below uses the same roles.
// mbarriers: full_x[NST] (256 producer arrivals), full_e[NST] (bulk-copy bytes), empty[NST]
// (one MMA commit per issuing thread), tmem_full (likewise, after a tile), tmem_empty (128 epilogue
// arrivals), done (final commit of each issuing thread), slot_full[4] (scheduler),
// slot_empty[4] (every reader: 256 + 2 + 128).  The producers fill the ring for the next tile
// while the epilogue drains the current one.  Every wait is bounded; an expired wait sets a
// shared abort flag and the status word, every role stops at its next check, the epilogue
// decides by a vote so that its named barrier stays matched, and TMEM is freed only after
// both MMA threads saw their own MMAs complete.
constexpr int WS_EPI0 = 8, WS_MMA = 12, WS_SCHED = 13;
constexpr int WS_PROD = 256, WS_EPI = 128, WS_SLOTS = 4;
// The warp-specialised kernel issues its MMAs from two threads (warps 12 and 14, on different
// warp schedulers), each owning two of the four accumulators: one issuing thread that shares
// its scheduler with two digit-cutting warps gets a tcgen05.mma out only every ~100 cycles,
// while the tensor pipe retires one 128 x 128 x 16 MMA every 64.
constexpr int WS_MMA2 = 14, WS_ISSUERS = 2, WS_THREADS = 480;
constexpr int WS_SLOT_READERS = WS_PROD + WS_ISSUERS + WS_EPI;
constexpr int WS_MASK1 = 0b1001, WS_MASK2 = 0b0110;  // accumulators {0, 3} and {1, 2}

struct WsSlot {
  const void* in;
  void* out;
  const uint8_t* ebase;  // E slices of the tile's 128-row block
  const int* rexp;       // row exponents of that block
  int* out_exp;
  long long R, B0;
  long long base;        // TRANS: b0 * n * R (first element of the tile's slab); NORMAL: 0
  long long g0;          // first fiber of the tile: r0 (TRANS) or row0 (NORMAL)
  const uint8_t* xsl;    // pre-cut input slices of the tile ([chunk][slice] images), or null
  int n, nsub, rb, eX, nrows_e, out_f64;
};

// shared-memory layout after the stages
constexpr int WS_BAR_BYTES = 256, WS_SCALE_BYTES = 512, WS_SLOT_BYTES = 512;
static_assert(sizeof(WsSlot) * WS_SLOTS <= WS_SLOT_BYTES, "slot ring");

// Stages of the warp-specialised kernel's operand ring (X and E slices of one 32-wide chunk
// each): three up to 4 digit slices (3 x 64 KB), two above.  With two stages the producers
// can cut chunk c + 2 only after the MMAs of chunk c completed, and the tensor pipe waited
// for them on every tile's third and fourth chunk.
__host__ __device__ constexpr int ws_stages(int ks) { return ks <= 4 ? 3 : 2; }
static_assert(3 * 3 + 3 + 2 * WS_SLOTS <= WS_BAR_BYTES / 8, "mbarrier area");

size_t ws_smem_bytes(int ks) {
  return (size_t)ws_stages(ks) * 2 * ks * SLICE_BYTES + WS_BAR_BYTES + WS_SCALE_BYTES + WS_SLOT_BYTES + 32;
}

// Raw-ring variant (float-float passes up to 5 digit slices): the raw float-float operand of a
// 32-wide chunk (128 fibers x 32 K x 8 B = 32 KB) arrives in shared memory by TMA tensor copies
// that the scheduler warp issues up to ws_nraw chunks ahead, so that ~96 KB per SM are in flight
// without holding registers; the producers cut from shared memory into two operand stages.
// With loads issued by the producers themselves, one prefetched chunk (32 KB per SM, the
// register budget) at ~1.5 us of loaded latency capped the input near half the HBM bandwidth.
constexpr int WS_NRAW = 3;
// raw buffers of the warp-specialised kernel's ring: three up to 4 digit slices, two at 5
// (two 80 KB operand stages leave room for two)
__host__ __device__ constexpr int ws_nraw(int ks) { return ks <= 4 ? WS_NRAW : 2; }
constexpr int WS_RAW_BYTES = 128 * KC * 8;
constexpr int WS_RR_STAGES = 2;
static_assert(3 * WS_RR_STAGES + 3 + 2 * WS_SLOTS + 2 * WS_NRAW <= WS_BAR_BYTES / 8, "mbarrier area (raw ring)");

size_t ws_smem_bytes_rr(int ks) {
  return (size_t)WS_RR_STAGES * 2 * ks * SLICE_BYTES + (size_t)ws_nraw(ks) * WS_RAW_BYTES + WS_BAR_BYTES + WS_SCALE_BYTES +
         WS_SLOT_BYTES + 32;
}


// read slot tc % WS_SLOTS once it is filled, then release it
__device__ __forceinline__ bool ws_get(const WsSlot* slots, uint64_t* slot_full, uint64_t* slot_empty, uint32_t tc,
                                       WsSlot& out, unsigned long long wl) {
  const uint32_t q = tc % WS_SLOTS;
  const bool ok = mbar_wait(smem_u32(&slot_full[q]), (tc / WS_SLOTS) & 1u, wl);
  if (ok) out = slots[q];
  mbar_arrive(smem_u32(&slot_empty[q]));
  return ok;
}

// raw operand values of one thread: 8 consecutive k (from kc) of its operand row
template <bool IN_F64, bool TRANS>
__device__ __forceinline__ void ws_load(const WsSlot& S, int orow, int kc, Raw<IN_F64>& raw) {
  const long long gr = S.g0 + orow;
  const bool vr = TRANS ? (gr < S.R) : (gr < S.B0);
  if (!TRANS && !IN_F64) {
    // along a row of an internal float-float buffer: 16-byte loads (n is a multiple of 16 and
    // every row starts 16-byte aligned), half the L1 wavefronts of 8-byte loads
#pragma unroll
    for (int e = 0; e < 8; e += 2) {
      const int k = kc + e;
      const float2* src = reinterpret_cast<const float2*>(S.in) + gr * (long long)S.n + k;
      const bool ok = vr && k < S.n && PK_CK(src, 16, chk::SITE_MODE_LOAD);
      const float4 v = ok ? __ldg(reinterpret_cast<const float4*>(src)) : make_float4(0.f, 0.f, 0.f, 0.f);
      raw.f[e] = make_float2(v.x, v.y);
      raw.f[e + 1] = make_float2(v.z, v.w);
    }
    return;
  }
#pragma unroll
  for (int e = 0; e < 8; ++e) {
    const int k = kc + e;
    const long long idx = TRANS ? S.base + (long long)k * S.R + gr : gr * (long long)S.n + k;
    const bool ok = vr && k < S.n && PK_CK((const char*)S.in + 8 * idx, 8, chk::SITE_MODE_LOAD);
    if (IN_F64)
      raw.d[e] = ok ? __ldg(reinterpret_cast<const double*>(S.in) + idx) : 0.0;
    else
      raw.f[e] = ok ? __ldg(reinterpret_cast<const float2*>(S.in) + idx) : make_float2(0.f, 0.f);
  }
}


// Fastest-axis float-float passes: the raw values of chunk kc of a producer warp, loaded so that
// one load instruction covers two full 256-byte chunk rows (lane = 16-byte piece q = lane & 15
// of row 16 w + 2 j + lane / 16, j = 0..7): whole 32-byte sectors per request, where one row per
// lane and 16 bytes per request left half of every sector unused.  Piece j lands in
// raw[j / 4].f[2 (j % 4)] and .f[2 (j % 4) + 1] (values k = kc + 2q and kc + 2q + 1).
__device__ __forceinline__ void ws_load_rows(const WsSlot& S, int w, int lane, int kc, Raw<false>* raw) {
  const int q = lane & 15;
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    const long long gr = S.g0 + 16 * w + 2 * j + (lane >> 4);
    const int k = kc + 2 * q;
    const float2* src = reinterpret_cast<const float2*>(S.in) + gr * (long long)S.n + k;
    // n is a multiple of 16: k + 1 < n as well
    const bool ok = gr < S.B0 && k < S.n && PK_CK(src, 16, chk::SITE_MODE_LOAD);
    const float4 v = ok ? __ldg(reinterpret_cast<const float4*>(src)) : make_float4(0.f, 0.f, 0.f, 0.f);
    raw[j >> 2].f[2 * (j & 3)] = make_float2(v.x, v.y);
    raw[j >> 2].f[2 * (j & 3) + 1] = make_float2(v.z, v.w);
  }
}

// the slot of a tile of the warp-specialised kernel; job moves forward only (the tiles of a
// CTA increase)
template <int KS, bool TRANS>
__device__ __forceinline__ void ws_make_slot(const GPass& P, long long tile, int& job, WsSlot& S) {
  int lo = job, hi = P.njobs - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (P.jobs[mid].tile_begin <= tile) lo = mid; else hi = mid - 1;
  }
  job = lo;
  const GJob& J = P.jobs[job];
  const long long tj = tile - J.tile_begin;
  const long long rtiles = TRANS ? (J.R + 127) / 128 : 1;
  const long long per_rb = TRANS ? J.B0 * rtiles : (J.B0 + 127) / 128;
  const int rb = (int)(tj / per_rb);
  const long long th = tj % per_rb;
  S.in = job_in(P, J);
  S.out = job_out(P, J);
  const int nsub = (J.n + 31) / 32;
  S.ebase = J.eslices + (size_t)rb * (size_t)nsub * KS * SLICE_BYTES;
  S.rexp = J.rexp + 128 * rb;
  S.out_exp = J.out_exp;
  S.R = J.R;
  S.B0 = J.B0;
  S.base = TRANS ? (th / rtiles) * (long long)J.n * J.R : 0;
  S.g0 = TRANS ? (th % rtiles) * 128 : th * 128;
  S.xsl = J.xslices ? J.xslices + (size_t)(th % rtiles) * (size_t)nsub * KS * SLICE_BYTES : nullptr;
  S.n = J.n;
  S.nsub = nsub;
  S.rb = rb;
  S.eX = job_in_exp(J);
  S.nrows_e = min(128, J.n - 128 * rb);
  S.out_f64 = J.out_f64;
}

// TMA tensor copies (tile mode, no swizzle) of a box of the tensor map's global tensor into
// shared memory; elements outside the tensor arrive as zeros and count toward the bytes
__device__ __forceinline__ void tma_load_2d(uint32_t dst, const void* tmap, int x, int y, uint32_t mbar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
          dst),
      "l"(tmap), "r"(x), "r"(y), "r"(mbar)
      : "memory");
}

__device__ __forceinline__ void tma_load_3d(uint32_t dst, const void* tmap, int x, int y, int z, uint32_t mbar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];" ::
          "r"(dst),
      "l"(tmap), "r"(x), "r"(y), "r"(z), "r"(mbar)
      : "memory");
}

// Raw-ring variant: chunk c of a tile into raw buffer rbuf by one TMA copy (issued by one
// thread).  Fastest-axis passes: the job's input as a 2D tensor {n, B0} of 8-byte elements,
// box {32, 128} at (32 c, g0) -> 128 rows of 256 B.  Transposed passes: 3D {R, n, B0}, box
// {128, 32, 1} at (g0, 32 c, b0) -> 32 K rows of 1 KB.  The innermost coordinate (32 c resp.
// g0, a multiple of 128) times 8 bytes is a multiple of 16; fibers past R or B0 and K past n
// arrive as zeros.  The barrier expects the full 32 KB box.
template <bool TRANS>
__device__ __forceinline__ void ws_raw_tma(const GPass& P, int job, const WsSlot& S, int c, uint8_t* rbuf,
                                           uint64_t* full) {
  mbar_expect_tx(smem_u32(full), (uint32_t)WS_RAW_BYTES);
#ifdef PHIKRON_CHECKED
  const size_t in_bytes = 8ull * (size_t)S.n * (size_t)S.B0 * (size_t)(TRANS ? S.R : 1);
  if (!PK_CK(S.in, in_bytes, chk::SITE_MODE_LOAD)) {   // the zero block instead of the box
    bulk_copy_g2s(smem_u32(rbuf), chk::g_state->zero, (uint32_t)WS_RAW_BYTES, smem_u32(full));
    return;
  }
#endif
  const void* tm = static_cast<const uint8_t*>(P.tmaps) + 128 * (size_t)job;
  if (!TRANS)
    tma_load_2d(smem_u32(rbuf), tm, KC * c, (int)S.g0, smem_u32(full));
  else
    tma_load_3d(smem_u32(rbuf), tm, (int)S.g0, KC * c, (int)(S.base / ((long long)S.n * S.R)), smem_u32(full));
}

// The epilogue's work on TMEM columns [c0, c1) (multiples of 16) of lane et (lane_base = its
// lane quarter): the four level accumulators combined into float-float, scaled by the row
// exponents, stored (float-float or float64); returns the largest |hi| stored.  Run by whole
// warps (tcgen05.ld is warp-collective).
template <int KS, bool TRANS>
__device__ __forceinline__ float ws_epi_cols(const WsSlot& S, uint32_t lane_base, int et, int c0, int c1,
                                             const float* scale_s) {
  float mxf = 0.0f;  // largest |hi| stored (one FMNMX per element)
  if (TRANS) {
    // TMEM lane = fiber r, column = output row i of this row block; stores coalesce over lanes
    const long long g = S.g0 + et;
    const bool vg = g < S.R;
    const long long o0 = S.base + (long long)(128 * S.rb) * S.R + g;
    for (int cc = c0; cc < min(c1, S.nrows_e); cc += 16) {
      float d2[16], d3[16], d4[16], d5[16];
      tmem_ld16(lane_base + (uint32_t)cc, d2);
      tmem_ld16(lane_base + 128u + (uint32_t)cc, d3);
      tmem_ld16(lane_base + 256u + (uint32_t)cc, d4);
      if (KS >= 4) tmem_ld16(lane_base + 384u + (uint32_t)cc, d5);
      tmem_wait_ld();
      // the float64 / float-float choice is made per group, so that the 16 columns of the
      // unrolled body stay straight-line code the compiler can interleave
      if (vg && !S.out_f64) {
        float2* dst = reinterpret_cast<float2*>(S.out) + o0 + (long long)cc * S.R;
#pragma unroll
        for (int j = 0; j < 16; j += 2) {
          float2 hi, lo;
          ff_combine2<KS>(make_float2(d2[j], d2[j + 1]), make_float2(d3[j], d3[j + 1]),
                          make_float2(d4[j], d4[j + 1]),
                          KS >= 4 ? make_float2(d5[j], d5[j + 1]) : make_float2(0.0f, 0.0f), hi, lo);
          const float2 sc = *reinterpret_cast<const float2*>(scale_s + cc + j);
          hi = mul2(hi, sc);
          lo = mul2(lo, sc);
          st_ck(dst + (long long)j * S.R, make_float2(hi.x, lo.x), chk::SITE_MODE_STORE);
          st_ck(dst + (long long)(j + 1) * S.R, make_float2(hi.y, lo.y), chk::SITE_MODE_STORE);
          mxf = fmaxf(mxf, fmaxf(fabsf(hi.x), fabsf(hi.y)));
        }
      } else if (vg) {
        double* dst = reinterpret_cast<double*>(S.out) + o0 + (long long)cc * S.R;
#pragma unroll
        for (int j = 0; j < 16; j += 2) {
          float2 hi, lo;
          ff_combine2<KS>(make_float2(d2[j], d2[j + 1]), make_float2(d3[j], d3[j + 1]),
                          make_float2(d4[j], d4[j + 1]),
                          KS >= 4 ? make_float2(d5[j], d5[j + 1]) : make_float2(0.0f, 0.0f), hi, lo);
          const float2 sc = *reinterpret_cast<const float2*>(scale_s + cc + j);
          hi = mul2(hi, sc);
          lo = mul2(lo, sc);
          st_ck(dst + (long long)j * S.R, ff_to_f64(hi.x, lo.x), chk::SITE_MODE_STORE);
          st_ck(dst + (long long)(j + 1) * S.R, ff_to_f64(hi.y, lo.y), chk::SITE_MODE_STORE);
          mxf = fmaxf(mxf, fmaxf(fabsf(hi.x), fabsf(hi.y)));
        }
      }
    }
  } else {
    // TMEM lane = output row i of this row block, column = fiber; stores coalesce over lanes
    const bool vi = et < S.nrows_e;
    const int ncols = (int)min(128LL, S.B0 - S.g0);
    const float sc = scale_s[et];
    const long long o0 = S.g0 * (long long)S.n + 128 * S.rb + et;
    for (int cc = c0; cc < min(c1, ncols); cc += 16) {
      float d2[16], d3[16], d4[16], d5[16];
      tmem_ld16(lane_base + (uint32_t)cc, d2);
      tmem_ld16(lane_base + 128u + (uint32_t)cc, d3);
      tmem_ld16(lane_base + 256u + (uint32_t)cc, d4);
      if (KS >= 4) tmem_ld16(lane_base + 384u + (uint32_t)cc, d5);
      tmem_wait_ld();
      const int jn = min(16, ncols - cc);  // columns of this group inside the tile
      if (vi && !S.out_f64) {
        float2* dst = reinterpret_cast<float2*>(S.out) + o0 + (long long)cc * S.n;
#pragma unroll
        for (int j = 0; j < 16; j += 2) {
          float2 hi, lo;
          ff_combine2<KS>(make_float2(d2[j], d2[j + 1]), make_float2(d3[j], d3[j + 1]),
                          make_float2(d4[j], d4[j + 1]),
                          KS >= 4 ? make_float2(d5[j], d5[j + 1]) : make_float2(0.0f, 0.0f), hi, lo);
          hi = mul2(hi, make_float2(sc, sc));
          lo = mul2(lo, make_float2(sc, sc));
          if (j < jn) {
            st_ck(dst + (long long)j * S.n, make_float2(hi.x, lo.x), chk::SITE_MODE_STORE);
            mxf = fmaxf(mxf, fabsf(hi.x));
          }
          if (j + 1 < jn) {
            st_ck(dst + (long long)(j + 1) * S.n, make_float2(hi.y, lo.y), chk::SITE_MODE_STORE);
            mxf = fmaxf(mxf, fabsf(hi.y));
          }
        }
      } else if (vi) {
        double* dst = reinterpret_cast<double*>(S.out) + o0 + (long long)cc * S.n;
#pragma unroll
        for (int j = 0; j < 16; j += 2) {
          float2 hi, lo;
          ff_combine2<KS>(make_float2(d2[j], d2[j + 1]), make_float2(d3[j], d3[j + 1]),
                          make_float2(d4[j], d4[j + 1]),
                          KS >= 4 ? make_float2(d5[j], d5[j + 1]) : make_float2(0.0f, 0.0f), hi, lo);
          hi = mul2(hi, make_float2(sc, sc));
          lo = mul2(lo, make_float2(sc, sc));
          if (j < jn) {
            st_ck(dst + (long long)j * S.n, ff_to_f64(hi.x, lo.x), chk::SITE_MODE_STORE);
            mxf = fmaxf(mxf, fabsf(hi.x));
          }
          if (j + 1 < jn) {
            st_ck(dst + (long long)(j + 1) * S.n, ff_to_f64(hi.y, lo.y), chk::SITE_MODE_STORE);
            mxf = fmaxf(mxf, fabsf(hi.y));
          }
        }
      }
    }
  }
  return mxf;
}

template <int KS, bool IN_F64, bool TRANS, bool RR = false, bool PC = false>
__global__ void __launch_bounds__(WS_THREADS, 1) mode_kernel_ws(const __grid_constant__ GPass P, int* status) {
  static_assert(!RR || (!IN_F64 && KS <= 5), "raw ring: float-float passes up to 5 digit slices");
  static_assert(!PC || (IN_F64 && TRANS && !RR), "pre-cut input: the float64 first pass");
  PK_CHECK_TABLES(P);
  const unsigned long long wl = P.wait_ns;  // limit of every bounded wait
  extern __shared__ __align__(1024) uint8_t smem[];
  constexpr int HALF_BYTES = KS * SLICE_BYTES;
  constexpr int STAGE_BYTES = 2 * HALF_BYTES;
  constexpr int NST = RR ? WS_RR_STAGES : ws_stages(KS);
  constexpr int NRAW = RR ? ws_nraw(KS) : 0;
  constexpr int NRAW_DIV = RR ? ws_nraw(KS) : 1;   // ring index arithmetic (compiled, unused, without the ring)
  uint8_t* rawring = smem + NST * STAGE_BYTES;   // [NRAW] raw chunks (raw-ring variant)
  uint8_t* tail = rawring + NRAW * WS_RAW_BYTES;
  uint64_t* bars = reinterpret_cast<uint64_t*>(tail);
  uint64_t* full_x = bars;              // [NST]
  uint64_t* full_e = bars + NST;        // [NST]
  uint64_t* empty = bars + 2 * NST;     // [NST]
  uint64_t* tmem_full = bars + 3 * NST;
  uint64_t* tmem_empty = bars + 3 * NST + 1;
  uint64_t* done = bars + 3 * NST + 2;
  uint64_t* slot_full = bars + 3 * NST + 3;            // [WS_SLOTS]
  uint64_t* slot_empty = bars + 3 * NST + 3 + WS_SLOTS;  // [WS_SLOTS]
  uint64_t* raw_full = bars + 3 * NST + 3 + 2 * WS_SLOTS;   // [NRAW] raw chunk landed
  uint64_t* raw_empty = raw_full + NRAW;                   // [NRAW] producers read it
  float* scale_s = reinterpret_cast<float*>(tail + WS_BAR_BYTES);  // 128 floats
  WsSlot* slots = reinterpret_cast<WsSlot*>(tail + WS_BAR_BYTES + WS_SCALE_BYTES);
  uint32_t* tmem_s = reinterpret_cast<uint32_t*>(tail + WS_BAR_BYTES + WS_SCALE_BYTES + WS_SLOT_BYTES);
  volatile int* abort_s = reinterpret_cast<volatile int*>(tail + WS_BAR_BYTES + WS_SCALE_BYTES + WS_SLOT_BYTES + 16);

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const long long total_tiles = P.total_tiles;
  if (tid == 0) {
    for (int q = 0; q < NST; ++q) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&full_x[q])), "r"(PC ? 1 : WS_PROD));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&full_e[q])));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&empty[q])), "r"(WS_ISSUERS));
    }
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(tmem_full)), "r"(WS_ISSUERS));
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(tmem_empty)), "r"(WS_EPI));
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(done)), "r"(WS_ISSUERS));
    for (int q = 0; q < WS_SLOTS; ++q) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&slot_full[q])));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&slot_empty[q])), "r"(WS_SLOT_READERS));
    }
    for (int q = 0; q < NRAW; ++q) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&raw_full[q])));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&raw_empty[q])), "r"(WS_PROD));
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    *abort_s = 0;
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_s)),
                 "r"(512));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tmem_s;

  if (RR && warp < WS_EPI0) {
    // ------------------------------------------------------------ producers (raw ring)
    const int orow = tid & 127;
    const int kh = tid >> 7;
    const int q = lane & 15;
    uint32_t it = 0, tc = 0;
    int e_last = -1;          // thread 0: chunk of the latest E bulk copy
    bool stop = false;
    for (long long tile = blockIdx.x; tile < total_tiles && !stop; tile += gridDim.x, ++tc) {
      WsSlot S;
      if (!ws_get(slots, slot_full, slot_empty, tc, S, wl)) ws_fail(abort_s, status);
      if (*abort_s) break;
      const float xsc = pow2f_full(-S.eX);
      const int nr = (int)min(128LL, TRANS ? S.R - S.g0 : S.B0 - S.g0);   // valid fibers of the tile
      for (int c = 0; c < S.nsub; ++c, ++it) {
        const uint32_t st = it % NST, use = it / NST;
        const uint32_t r = it % NRAW_DIV, ru = it / NRAW_DIV;
        uint8_t* sX = smem + st * STAGE_BYTES;
        uint8_t* sE = sX + HALF_BYTES;
        const uint8_t* rb = rawring + r * WS_RAW_BYTES;
        const int kv = min(KC, S.n - KC * c);
        if (use >= 1 && !mbar_wait(smem_u32(&empty[st]), (use - 1) & 1u, wl)) ws_fail(abort_s, status);
        if (!mbar_wait(smem_u32(&raw_full[r]), ru & 1u, wl)) ws_fail(abort_s, status);
        if (*abort_s) { stop = true; break; }
        if (tid == 0) {
          e_last = (int)it;
          mbar_expect_tx(smem_u32(&full_e[st]), (uint32_t)HALF_BYTES);
          bulk_copy_g2s(smem_u32(sE), PK_CK_SRC(S.ebase + (size_t)c * HALF_BYTES, HALF_BYTES, chk::SITE_MODE_ECOPY),
                        (uint32_t)HALF_BYTES, smem_u32(&full_e[st]));
        }
        if constexpr (!TRANS) {
          // piece j: values k = 2q, 2q + 1 of row 16 w + 2 j + lane / 16 (16 lanes read a row's
          // 256 contiguous bytes) -> 4 bytes of every slice
          float4 v[8];
#pragma unroll
          for (int j = 0; j < 8; ++j) {
            const int row = 16 * warp + 2 * j + (lane >> 4);
            v[j] = (row < nr && 2 * q < kv) ? *reinterpret_cast<const float4*>(rb + row * 256 + q * 16)
                                            : make_float4(0.f, 0.f, 0.f, 0.f);
          }
          mbar_arrive(smem_u32(&raw_empty[r]));   // this thread's raw values are in registers
#pragma unroll
          for (int j = 0; j < 8; ++j) {
            float2 a[KS];
            cut_ff_float2<KS>(make_float2(v[j].x, v[j].z), make_float2(v[j].y, v[j].w), xsc, a);
            const int row = 16 * warp + 2 * j + (lane >> 4);
            const uint32_t off = chunk_offset(row, q >> 2) + (uint32_t)(q & 3) * 4u;
#pragma unroll
            for (int sl = 0; sl < KS; ++sl)
              *reinterpret_cast<uint32_t*>(sX + sl * SLICE_BYTES + off) = pack_bf16x2(a[sl].x, a[sl].y);
          }
        } else {
          // fiber orow, values k = 16 kh .. 16 kh + 15 (lanes read consecutive fibers)
          float2 f[16];
#pragma unroll
          for (int e = 0; e < 16; ++e) {
            const int k = 16 * kh + e;
            f[e] = (orow < nr && k < kv) ? *reinterpret_cast<const float2*>(rb + k * 1024 + orow * 8)
                                         : make_float2(0.f, 0.f);
          }
          mbar_arrive(smem_u32(&raw_empty[r]));
#pragma unroll
          for (int g2 = 0; g2 < 2; ++g2) {
            uint32_t pk[KS][4];
#pragma unroll
            for (int e = 0; e < 8; e += 2) {
              float2 a[KS];
              cut_ff_float2<KS>(make_float2(f[8 * g2 + e].x, f[8 * g2 + e + 1].x),
                                make_float2(f[8 * g2 + e].y, f[8 * g2 + e + 1].y), xsc, a);
#pragma unroll
              for (int sl = 0; sl < KS; ++sl) pk[sl][e >> 1] = pack_bf16x2(a[sl].x, a[sl].y);
            }
            const uint32_t off = chunk_offset(orow, 2 * kh + g2);
#pragma unroll
            for (int sl = 0; sl < KS; ++sl)
              *reinterpret_cast<uint4*>(sX + sl * SLICE_BYTES + off) = make_uint4(pk[sl][0], pk[sl][1], pk[sl][2], pk[sl][3]);
          }
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        mbar_arrive(smem_u32(&full_x[st]));
      }
    }
    if (tid == 0 && *abort_s) {
      // bulk copies still in flight must land before the CTA's shared memory is released
      for (int k = e_last; k >= 0 && k >= e_last - (NST - 1); --k)
        mbar_wait(smem_u32(&full_e[k % NST]), ((uint32_t)k / NST) & 1u, CLEANUP_WAIT_NS);
    }
  } else if (PC && warp < WS_EPI0) {
    // ------------------------------------------------------------ producers (pre-cut input)
    // the input's digit slices were cut once for all jobs: thread 0 brings each chunk's X and E
    // slices in by bulk copies; the other producer threads only read the slots
    uint32_t it = 0, tc = 0;
    int e_last = -1;
    bool stop = false;
    for (long long tile = blockIdx.x; tile < total_tiles && !stop; tile += gridDim.x, ++tc) {
      WsSlot S;
      if (!ws_get(slots, slot_full, slot_empty, tc, S, wl)) ws_fail(abort_s, status);
      if (*abort_s) break;
      if (tid != 0) continue;
      for (int c = 0; c < S.nsub; ++c, ++it) {
        const uint32_t st = it % NST, use = it / NST;
        uint8_t* sX = smem + st * STAGE_BYTES;
        uint8_t* sE = sX + HALF_BYTES;
        if (use >= 1 && !mbar_wait(smem_u32(&empty[st]), (use - 1) & 1u, wl)) ws_fail(abort_s, status);
        if (*abort_s) { stop = true; break; }
        e_last = (int)it;
        mbar_expect_tx(smem_u32(&full_e[st]), (uint32_t)HALF_BYTES);
        bulk_copy_g2s(smem_u32(sE), PK_CK_SRC(S.ebase + (size_t)c * HALF_BYTES, HALF_BYTES, chk::SITE_MODE_ECOPY),
                      (uint32_t)HALF_BYTES, smem_u32(&full_e[st]));
        mbar_expect_tx(smem_u32(&full_x[st]), (uint32_t)HALF_BYTES);
        bulk_copy_g2s(smem_u32(sX), PK_CK_SRC(S.xsl + (size_t)c * HALF_BYTES, HALF_BYTES, chk::SITE_MODE_LOAD),
                      (uint32_t)HALF_BYTES, smem_u32(&full_x[st]));
      }
    }
    if (tid == 0 && *abort_s) {
      // bulk copies still in flight must land before the CTA's shared memory is released
      for (int k = e_last; k >= 0 && k >= e_last - (NST - 1); --k) {
        mbar_wait(smem_u32(&full_e[k % NST]), ((uint32_t)k / NST) & 1u, CLEANUP_WAIT_NS);
        mbar_wait(smem_u32(&full_x[k % NST]), ((uint32_t)k / NST) & 1u, CLEANUP_WAIT_NS);
      }
    }
  } else if (!RR && !PC && warp < WS_EPI0) {
    // ------------------------------------------------------------ producers
    const int orow = tid & 127;
    const int kh = tid >> 7;  // k-groups 2*kh, 2*kh + 1 of every 32-wide chunk
    // fastest-axis float-float passes load and cut by row pieces (ws_load_rows)
    constexpr bool ROWS = !TRANS && !IN_F64;
    uint32_t it = 0, tc = 0;
    int e_last = -1;          // thread 0: chunk of the latest E bulk copy
    long long tile = blockIdx.x;
    WsSlot S, Sn;
    Raw<IN_F64> raw[2];
    bool have = false;
    if (tile < total_tiles) {
      have = ws_get(slots, slot_full, slot_empty, 0, S, wl);
      if (!have) {
        ws_fail(abort_s, status);
      } else {
        if constexpr (ROWS) {
          ws_load_rows(S, warp, lane, 0, raw);
        } else {
          ws_load<IN_F64, TRANS>(S, orow, 16 * kh, raw[0]);
          ws_load<IN_F64, TRANS>(S, orow, 16 * kh + 8, raw[1]);
        }
      }
    }
    for (; have && tile < total_tiles; tile += gridDim.x, ++tc) {
      const int nchunks = S.nsub;
      const int eb = 1011 + S.eX;
      const float xsc = pow2f_full(-S.eX);
      const bool has_next = tile + gridDim.x < total_tiles;
      bool stop = false;
      for (int c = 0; c < nchunks; ++c, ++it) {
        const uint32_t st = it % NST, use = it / NST;
        uint8_t* sX = smem + st * STAGE_BYTES;
        uint8_t* sE = sX + HALF_BYTES;
        // the next chunk's raw values go in flight before the wait for a free stage, so that
        // their latency overlaps the wait and this chunk's cutting
        Raw<IN_F64> rawn[2];
        if (c + 1 < nchunks) {
          if constexpr (ROWS) {
            ws_load_rows(S, warp, lane, 32 * (c + 1), rawn);
          } else {
            ws_load<IN_F64, TRANS>(S, orow, 32 * (c + 1) + 16 * kh, rawn[0]);
            ws_load<IN_F64, TRANS>(S, orow, 32 * (c + 1) + 16 * kh + 8, rawn[1]);
          }
        } else if (has_next) {
          if (ws_get(slots, slot_full, slot_empty, tc + 1, Sn, wl)) {
            if constexpr (ROWS) {
              ws_load_rows(Sn, warp, lane, 0, rawn);
            } else {
              ws_load<IN_F64, TRANS>(Sn, orow, 16 * kh, rawn[0]);
              ws_load<IN_F64, TRANS>(Sn, orow, 16 * kh + 8, rawn[1]);
            }
          } else {
            ws_fail(abort_s, status);
          }
        }
        if (use >= 1 && !mbar_wait(smem_u32(&empty[st]), (use - 1) & 1u, wl)) ws_fail(abort_s, status);
        if (*abort_s) { stop = true; break; }
        if (tid == 0) {
          e_last = (int)it;
          mbar_expect_tx(smem_u32(&full_e[st]), (uint32_t)HALF_BYTES);
          bulk_copy_g2s(smem_u32(sE), PK_CK_SRC(S.ebase + (size_t)c * HALF_BYTES, HALF_BYTES, chk::SITE_MODE_ECOPY),
                        (uint32_t)HALF_BYTES, smem_u32(&full_e[st]));
        }
        if constexpr (ROWS) {
          // piece j: values k = 2q, 2q + 1 of row 16 w + 2 j + lane / 16 -> 4 bytes of every slice
          const int q = lane & 15;
#pragma unroll
          for (int j = 0; j < 8; ++j) {
            const float2 a = raw[j >> 2].f[2 * (j & 3)], b = raw[j >> 2].f[2 * (j & 3) + 1];
            float2 v[KS];
            cut_ff_float2<KS>(make_float2(a.x, b.x), make_float2(a.y, b.y), xsc, v);
            const int r = 16 * warp + 2 * j + (lane >> 4);
            const uint32_t off = chunk_offset(r, q >> 2) + (uint32_t)(q & 3) * 4u;
#pragma unroll
            for (int sl = 0; sl < KS; ++sl)
              *reinterpret_cast<uint32_t*>(sX + sl * SLICE_BYTES + off) = pack_bf16x2(v[sl].x, v[sl].y);
          }
        } else {
#pragma unroll
        for (int g2 = 0; g2 < 2; ++g2) {
          uint32_t pk[KS][4];
#pragma unroll
          for (int e = 0; e < 8; e += 2) {
            if (IN_F64) {
              uint32_t s0, s1;
              const uint64_t F0 = round_digits<KS>(fixed_f64(raw[g2].d[e], eb, s0));
              const uint64_t F1 = round_digits<KS>(fixed_f64(raw[g2].d[e + 1], eb, s1));
              uint32_t w[KS];
              cut_pair<KS>(F0, s0, F1, s1, w);
#pragma unroll
              for (int sl = 0; sl < KS; ++sl) pk[sl][e >> 1] = w[sl];
            } else {
              float2 v[KS];
              cut_ff_float2<KS>(make_float2(raw[g2].f[e].x, raw[g2].f[e + 1].x), make_float2(raw[g2].f[e].y, raw[g2].f[e + 1].y), xsc, v);
#pragma unroll
              for (int sl = 0; sl < KS; ++sl) pk[sl][e >> 1] = pack_bf16x2(v[sl].x, v[sl].y);
            }
          }
          const int g = 2 * kh + g2;
          const uint32_t off = chunk_offset(orow, g);
#pragma unroll
          for (int sl = 0; sl < KS; ++sl)
            *reinterpret_cast<uint4*>(sX + sl * SLICE_BYTES + off) = make_uint4(pk[sl][0], pk[sl][1], pk[sl][2], pk[sl][3]);
        }
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        mbar_arrive(smem_u32(&full_x[st]));
        raw[0] = rawn[0];
        raw[1] = rawn[1];
      }
      if (stop) break;
      S = Sn;
    }
    if (tid == 0 && *abort_s) {
      // bulk copies still in flight must land before the CTA's shared memory is released
      for (int k = e_last; k >= 0 && k >= e_last - (NST - 1); --k)
        mbar_wait(smem_u32(&full_e[k % NST]), ((uint32_t)k / NST) & 1u, CLEANUP_WAIT_NS);
    }
  } else if (warp < WS_MMA) {
    // ------------------------------------------------------------ epilogue
    const int et = tid - WS_EPI0 * 32;   // 0..127 = TMEM lane
    const uint32_t lane_base = tmem + ((uint32_t)((et >> 5) * 32) << 16);
    uint32_t tc = 0;
    for (long long tile = blockIdx.x; tile < total_tiles; tile += gridDim.x, ++tc) {
      WsSlot S;
      bool ok = ws_get(slots, slot_full, slot_empty, tc, S, wl);
      asm volatile("bar.sync 1, 128;" ::: "memory");  // the previous tile's scale table is no longer read
      if (ok)
        scale_s[et] = pow2f(S.eX + ((et < S.nrows_e && PK_CK(S.rexp + et, sizeof(int), chk::SITE_MODE_REXP))
                                        ? S.rexp[et] : 0));
      ok = ok && mbar_wait(smem_u32(tmem_full), tc & 1u, wl);
      if (!ok) ws_fail(abort_s, status);
      // the vote is also the barrier after the scale writes; every epilogue thread decides alike
      if (epi_vote_any(!ok || *abort_s)) break;
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const float mxf = ws_epi_cols<KS, TRANS>(S, lane_base, et, 0, 128, scale_s);
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      mbar_arrive(smem_u32(tmem_empty));
      uint32_t mx = __float_as_uint(mxf);  // non-negative: bit patterns order like the values
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
      // |v| < 2^{biased - 126}; a zero vector keeps the slot's initial (very negative) value
      const int emax = (int)(mx >> 23);
      if (lane == 0 && emax > 0) out_exp_max(S.out_exp, emax - 126);
    }
  } else if (warp == WS_MMA || warp == WS_MMA2) {
    if (lane == 0) {
      // ---------------------------------------------------------- MMA issuers (two threads)
      const bool second = warp == WS_MMA2;
      uint32_t it = 0, tc = 0;
      bool issued = false;
      for (long long tile = blockIdx.x; tile < total_tiles; tile += gridDim.x, ++tc) {
        WsSlot S;
        if (!ws_get(slots, slot_full, slot_empty, tc, S, wl)) ws_fail(abort_s, status);
        if (tc >= 1 && !mbar_wait(smem_u32(tmem_empty), (tc - 1) & 1u, wl)) ws_fail(abort_s, status);
        if (*abort_s) break;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t idesc = TRANS ? make_idesc(128, S.nrows_e) : make_idesc(128, 128);
        bool stop = false;
        for (int c = 0; c < S.nsub; ++c, ++it) {
          const uint32_t st = it % NST, use = it / NST;
          if (!mbar_wait(smem_u32(&full_x[st]), use & 1u, wl) || !mbar_wait(smem_u32(&full_e[st]), use & 1u, wl))
            ws_fail(abort_s, status);
          if (*abort_s) { stop = true; break; }
          asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
          // descriptors built once per chunk; the issue loop only adds compile-time offsets
          // (start-address units of 16 bytes) to 32-bit low words
          const uint32_t xa = smem_u32(smem + st * STAGE_BYTES);
          const uint32_t xlo = desc_lo(xa), elo = desc_lo(xa + HALF_BYTES);
          if (second) {
            if (c == 0)
              issue_chunk<KS, true, !TRANS, 128, SLICE_BYTES, WS_MASK2>(tmem, xlo, elo, idesc);
            else
              issue_chunk<KS, false, !TRANS, 128, SLICE_BYTES, WS_MASK2>(tmem, xlo, elo, idesc);
          } else {
            if (c == 0)
              issue_chunk<KS, true, !TRANS, 128, SLICE_BYTES, WS_MASK1>(tmem, xlo, elo, idesc);
            else
              issue_chunk<KS, false, !TRANS, 128, SLICE_BYTES, WS_MASK1>(tmem, xlo, elo, idesc);
          }
          issued = true;
          mma_commit(smem_u32(&empty[st]));  // arrives once this thread's MMAs of the chunk are done
        }
        if (stop) break;
        mma_commit(smem_u32(tmem_full));
      }
      // every MMA this thread issued is complete before TMEM is released
      mma_commit(smem_u32(done));
      if (issued) mbar_wait(smem_u32(done), 0u, CLEANUP_WAIT_NS);
    }
  } else if (RR && warp == WS_SCHED) {
    // ------------------------------------------------------------ scheduler + raw copies (warp 13)
    int job = 0;
    uint32_t tc = 0, it = 0;
    long long r_last = -1;   // chunk of the latest raw copy
    bool stop = false;
    for (long long tile = blockIdx.x; tile < total_tiles && !stop; tile += gridDim.x, ++tc) {
      const uint32_t q = tc % WS_SLOTS;
      bool ok = tc < WS_SLOTS || mbar_wait(smem_u32(&slot_empty[q]), ((tc / WS_SLOTS) - 1) & 1u, wl);
      if (!ok) ws_fail(abort_s, status);
      if (__any_sync(0xffffffffu, !ok || *abort_s)) break;   // warp-uniform
      WsSlot L;
      ws_make_slot<KS, TRANS>(P, tile, job, L);   // every lane computes the same slot
      if (lane == 0) {
        slots[q] = L;
        mbar_arrive(smem_u32(&slot_full[q]));
      }
      for (int c = 0; c < L.nsub; ++c, ++it) {
        const uint32_t r = it % NRAW_DIV, ru = it / NRAW_DIV;
        ok = ru == 0 || mbar_wait(smem_u32(&raw_empty[r]), (ru - 1) & 1u, wl);
        if (!ok) ws_fail(abort_s, status);
        if (__any_sync(0xffffffffu, !ok || *abort_s)) { stop = true; break; }
        if (lane == 0) ws_raw_tma<TRANS>(P, job, L, c, rawring + r * WS_RAW_BYTES, &raw_full[r]);
        r_last = it;
      }
    }
    if (lane == 0 && *abort_s) {
      // raw copies still in flight must land before the CTA's shared memory is released
      for (long long k = r_last; k >= 0 && k >= r_last - (NRAW - 1); --k)
        mbar_wait(smem_u32(&raw_full[k % NRAW_DIV]), (uint32_t)(k / NRAW_DIV) & 1u, CLEANUP_WAIT_NS);
    }
  } else if (!RR && warp == WS_SCHED && lane == 0) {
    // ------------------------------------------------------------ scheduler (warp 13, lane 0)
    int job = 0;
    uint32_t tc = 0;
    for (long long tile = blockIdx.x; tile < total_tiles; tile += gridDim.x, ++tc) {
      const uint32_t q = tc % WS_SLOTS;
      if (tc >= WS_SLOTS && !mbar_wait(smem_u32(&slot_empty[q]), ((tc / WS_SLOTS) - 1) & 1u, wl))
        ws_fail(abort_s, status);
      if (*abort_s) break;
      ws_make_slot<KS, TRANS>(P, tile, job, slots[q]);
      mbar_arrive(smem_u32(&slot_full[q]));
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512));
}

// ---------------------------------------------------------------- pre-cut input slices
// One block per (job, 128-fiber block, 32-wide chunk): the digit slices of that chunk of the
// job's float64 input (transposed first pass: B0 = 1, element (k, r) at k * R + r), cut as the
// producers of the mode kernel cut them (same exponent, same integer digit cutting), written as
// the KS shared-memory images [slice][8 KB] the MMAs read.  Blocks are counted by tile_begin.
template <int KS>
__global__ void __launch_bounds__(WS_PROD) precut_kernel(const __grid_constant__ GPass P) {
  PK_CHECK_TABLES(P);
  const int tid = threadIdx.x;
  const int orow = tid & 127, kh = tid >> 7;
  for (long long blk = blockIdx.x; blk < P.total_tiles; blk += gridDim.x) {
    int lo = 0, hi = P.njobs - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (P.jobs[mid].tile_begin <= blk) lo = mid; else hi = mid - 1;
    }
    const GJob& J = P.jobs[lo];
    const int nsub = (J.n + 31) / 32;
    const long long jb = blk - J.tile_begin;
    const long long rt = jb / nsub;
    const int c = (int)(jb % nsub);
    const double* in = static_cast<const double*>(job_in(P, J));
    const int eb = 1011 + job_in_exp(J);
    const long long g = rt * 128 + orow;
    uint8_t* dst = const_cast<uint8_t*>(J.xslices) + (size_t)(rt * nsub + c) * KS * SLICE_BYTES;
    double dv[16];   // all of this thread's loads in flight before any cutting
#pragma unroll
    for (int e = 0; e < 16; ++e) {
      const int k = 32 * c + 16 * kh + e;
      const double* src = in + (long long)k * J.R + g;
      dv[e] = (g < J.R && k < J.n && PK_CK(src, sizeof(double), chk::SITE_MODE_LOAD)) ? __ldg(src) : 0.0;
    }
#pragma unroll
    for (int g2 = 0; g2 < 2; ++g2) {
      const double* d = dv + 8 * g2;
      uint32_t pk[KS][4];
#pragma unroll
      for (int e = 0; e < 8; e += 2) {
        uint32_t s0, s1;
        const uint64_t F0 = round_digits<KS>(fixed_f64(d[e], eb, s0));
        const uint64_t F1 = round_digits<KS>(fixed_f64(d[e + 1], eb, s1));
        uint32_t w[KS];
        cut_pair<KS>(F0, s0, F1, s1, w);
#pragma unroll
        for (int sl = 0; sl < KS; ++sl) pk[sl][e >> 1] = w[sl];
      }
      const uint32_t off = chunk_offset(orow, 2 * kh + g2);
#pragma unroll
      for (int sl = 0; sl < KS; ++sl)
        st_ck(reinterpret_cast<uint4*>(dst + sl * SLICE_BYTES + off), make_uint4(pk[sl][0], pk[sl][1], pk[sl][2], pk[sl][3]),
              chk::SITE_MODE_STORE);
    }
  }
}

// ---------------------------------------------------------------- double-buffered variant
// Tiles of 128 E rows x 64 fibers with E as the A operand (M = 128) and the fibers' digit
// slices as B (N = 64) in both orientations, so that one tile's four level accumulators take
// 4 x 64 TMEM columns and two tiles alternate between columns [0, 256) and [256, 512): the
// epilogue drains tile t while the MMAs of tile t+1 run.  Same roles as the warp-specialised
// kernel (8 producer, 4 epilogue, 2 MMA-issuing, 1 scheduler warp).  Producers hold three chunks
// (8 values a thread each) in registers, so the loads of chunk c+2 are in flight while chunk c
// is cut.  With fibers on the TMEM columns, a transposed pass's outputs (fiber = fastest
// index) are staged in shared memory and written back row by row, coalesced.  Every job of a
// pass needs n >= 64 (two or more 32-wide chunks).
constexpr int DB_XSLICE = 64 * KC * 2;       // one slice of a 64-fiber chunk: 4 KB
constexpr int DB_STAGE_PITCH = 528;          // bytes per staged output row (64 x 8 B + 16)
constexpr int DB_STAGE_BYTES = 128 * DB_STAGE_PITCH;

// stages of the double-buffered kernel's operand ring: three up to 4 digit slices, two above
__host__ __device__ constexpr int db_stages(int ks) { return ks <= 4 ? 3 : 2; }
static_assert(3 * 3 + 5 + 2 * WS_SLOTS <= WS_BAR_BYTES / 8, "mbarrier area (double-buffered kernel)");

size_t db_smem_bytes(int ks) {
  return (size_t)db_stages(ks) * ks * (DB_XSLICE + SLICE_BYTES) + DB_STAGE_BYTES + WS_BAR_BYTES + WS_SLOT_BYTES + 32;
}

// Raw-ring variant of the double-buffered kernel (float-float passes up to 4 slices): raw
// chunks of 64 fibers x 32 K (16 KB) by one TMA tensor copy each, three in flight, two stages
constexpr int DB_RAW_BYTES = 64 * KC * 8;
static_assert(3 * WS_RR_STAGES + 5 + 2 * WS_SLOTS + 2 * WS_NRAW <= WS_BAR_BYTES / 8, "mbarrier area (db raw ring)");

size_t db_smem_bytes_rr(int ks) {
  return (size_t)WS_RR_STAGES * ks * (DB_XSLICE + SLICE_BYTES) + DB_STAGE_BYTES + (size_t)WS_NRAW * DB_RAW_BYTES +
         WS_BAR_BYTES + WS_SLOT_BYTES + 32;
}

// chunk c of a 64-fiber tile into raw buffer rbuf by one TMA copy (see ws_raw_tma; boxes
// {32, 64} resp. {64, 32, 1}, tensor maps encoded for 64-fiber boxes)
template <bool TRANS>
__device__ __forceinline__ void db_raw_tma(const GPass& P, int job, const WsSlot& S, int c, uint8_t* rbuf,
                                           uint64_t* full) {
  mbar_expect_tx(smem_u32(full), (uint32_t)DB_RAW_BYTES);
#ifdef PHIKRON_CHECKED
  const size_t in_bytes = 8ull * (size_t)S.n * (size_t)S.B0 * (size_t)(TRANS ? S.R : 1);
  if (!PK_CK(S.in, in_bytes, chk::SITE_MODE_LOAD)) {
    bulk_copy_g2s(smem_u32(rbuf), chk::g_state->zero, (uint32_t)DB_RAW_BYTES, smem_u32(full));
    return;
  }
#endif
  const void* tm = static_cast<const uint8_t*>(P.tmaps) + 128 * (size_t)job;
  if (!TRANS)
    tma_load_2d(smem_u32(rbuf), tm, KC * c, (int)S.g0, smem_u32(full));
  else
    tma_load_3d(smem_u32(rbuf), tm, (int)S.g0, KC * c, (int)(S.base / ((long long)S.n * S.R)), smem_u32(full));
}

// 8 consecutive values (k = kc .. kc+7) of fiber g0 + fib
template <bool IN_F64, bool TRANS>
__device__ __forceinline__ void db_load(const WsSlot& S, int fib, int kc, Raw<IN_F64>& raw) {
  const long long gr = S.g0 + fib;
  const bool vr = TRANS ? (gr < S.R) : (gr < S.B0);
  if constexpr (!TRANS && !IN_F64) {
#pragma unroll
    for (int e = 0; e < 8; e += 2) {
      const int k = kc + e;
      const float2* src = reinterpret_cast<const float2*>(S.in) + gr * (long long)S.n + k;
      const bool ok = vr && k < S.n && PK_CK(src, 16, chk::SITE_MODE_LOAD);
      const float4 v = ok ? __ldg(reinterpret_cast<const float4*>(src)) : make_float4(0.f, 0.f, 0.f, 0.f);
      raw.f[e] = make_float2(v.x, v.y);
      raw.f[e + 1] = make_float2(v.z, v.w);
    }
  } else {
#pragma unroll
    for (int e = 0; e < 8; ++e) {
      const int k = kc + e;
      const long long idx = TRANS ? S.base + (long long)k * S.R + gr : gr * (long long)S.n + k;
      const bool ok = vr && k < S.n && PK_CK((const char*)S.in + 8 * idx, 8, chk::SITE_MODE_LOAD);
      if constexpr (IN_F64)
        raw.d[e] = ok ? __ldg(reinterpret_cast<const double*>(S.in) + idx) : 0.0;
      else
        raw.f[e] = ok ? __ldg(reinterpret_cast<const float2*>(S.in) + idx) : make_float2(0.f, 0.f);
    }
  }
}

// the slot of a 64-fiber tile of the double-buffered kernel (job moves forward only)
template <int KS, bool TRANS>
__device__ __forceinline__ void db_make_slot(const GPass& P, long long tile, int& job, WsSlot& S) {
  int lo = job, hi = P.njobs - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (P.jobs[mid].tile_begin <= tile) lo = mid; else hi = mid - 1;
  }
  job = lo;
  const GJob& J = P.jobs[job];
  const long long tj = tile - J.tile_begin;
  const long long rt = TRANS ? (J.R + 63) / 64 : 1;
  const long long per_rb = TRANS ? J.B0 * rt : (J.B0 + 63) / 64;
  const int rb = (int)(tj / per_rb);
  const long long th = tj % per_rb;
  S.in = job_in(P, J);
  S.out = job_out(P, J);
  const int nsub = (J.n + 31) / 32;
  S.ebase = J.eslices + (size_t)rb * (size_t)nsub * KS * SLICE_BYTES;
  S.rexp = J.rexp + 128 * rb;
  S.out_exp = J.out_exp;
  S.R = J.R;
  S.B0 = J.B0;
  S.base = TRANS ? (th / rt) * (long long)J.n * J.R : 0;
  S.g0 = TRANS ? (th % rt) * 64 : th * 64;
  S.n = J.n;
  S.nsub = nsub;
  S.rb = rb;
  S.eX = job_in_exp(J);
  S.nrows_e = min(128, J.n - 128 * rb);
  S.out_f64 = J.out_f64;
}

template <int KS, bool IN_F64, bool TRANS, bool RR = false>
__global__ void __launch_bounds__(WS_THREADS, 1) mode_kernel_db(const __grid_constant__ GPass P, int* status) {
  static_assert(!RR || (!IN_F64 && KS <= 4), "raw ring: float-float passes up to 4 digit slices");
  PK_CHECK_TABLES(P);
  const unsigned long long wl = P.wait_ns;  // limit of every bounded wait
  extern __shared__ __align__(1024) uint8_t smem[];
  constexpr int XBYTES = KS * DB_XSLICE;
  constexpr int STAGE = XBYTES + KS * SLICE_BYTES;
  constexpr int NST = RR ? WS_RR_STAGES : db_stages(KS);
  constexpr int NRAW = RR ? WS_NRAW : 0;
  constexpr int NRAW_DIV = RR ? WS_NRAW : 1;   // ring index arithmetic (compiled, unused, without the ring)
  uint8_t* staging = smem + NST * STAGE;
  uint8_t* rawring = staging + DB_STAGE_BYTES;   // [NRAW] raw chunks (raw-ring variant)
  uint8_t* tail = rawring + NRAW * DB_RAW_BYTES;
  uint64_t* bars = reinterpret_cast<uint64_t*>(tail);
  uint64_t* full_x = bars;                  // [NST]
  uint64_t* full_e = bars + NST;            // [NST]
  uint64_t* empty = bars + 2 * NST;         // [NST]
  uint64_t* tmem_full = bars + 3 * NST;     // [2] one per TMEM buffer
  uint64_t* tmem_empty = bars + 3 * NST + 2;  // [2]
  uint64_t* done = bars + 3 * NST + 4;
  uint64_t* slot_full = bars + 3 * NST + 5;             // [WS_SLOTS]
  uint64_t* slot_empty = bars + 3 * NST + 5 + WS_SLOTS; // [WS_SLOTS]
  uint64_t* raw_full = bars + 3 * NST + 5 + 2 * WS_SLOTS;  // [NRAW]
  uint64_t* raw_empty = raw_full + NRAW;                  // [NRAW]
  WsSlot* slots = reinterpret_cast<WsSlot*>(tail + WS_BAR_BYTES);
  uint32_t* tmem_s = reinterpret_cast<uint32_t*>(tail + WS_BAR_BYTES + WS_SLOT_BYTES);
  volatile int* abort_s = reinterpret_cast<volatile int*>(tail + WS_BAR_BYTES + WS_SLOT_BYTES + 16);

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const long long total_tiles = P.total_tiles;
  if (tid == 0) {
    for (int q = 0; q < NST; ++q) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&full_x[q])), "r"(WS_PROD));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&full_e[q])));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&empty[q])), "r"(WS_ISSUERS));
    }
    for (int q = 0; q < 2; ++q) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&tmem_full[q])), "r"(WS_ISSUERS));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&tmem_empty[q])), "r"(WS_EPI));
    }
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(done)), "r"(WS_ISSUERS));
    for (int q = 0; q < WS_SLOTS; ++q) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&slot_full[q])));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&slot_empty[q])), "r"(WS_SLOT_READERS));
    }
    for (int q = 0; q < NRAW; ++q) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&raw_full[q])));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&raw_empty[q])), "r"(WS_PROD));
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    *abort_s = 0;
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_s)),
                 "r"(512));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tmem_s;

  if (RR && warp < WS_EPI0) {
    // ------------------------------------------------------------ producers (raw ring)
    const int fib = tid & 63;   // fiber of the tile (transposed passes)
    const int kg = tid >> 6;    // k-group (8 values) of every 32-wide chunk (transposed passes)
    const int q = lane & 15;    // 16-byte piece of a row (fastest-axis passes)
    uint32_t it = 0, tc = 0;
    int e_last = -1;            // thread 0: chunk of the latest E bulk copy
    bool stop = false;
    for (long long tile = blockIdx.x; tile < total_tiles && !stop; tile += gridDim.x, ++tc) {
      WsSlot S;
      if (!ws_get(slots, slot_full, slot_empty, tc, S, wl)) ws_fail(abort_s, status);
      if (*abort_s) break;
      const float xsc = pow2f_full(-S.eX);
      const int nr = (int)min(64LL, TRANS ? S.R - S.g0 : S.B0 - S.g0);   // valid fibers of the tile
      for (int c = 0; c < S.nsub; ++c, ++it) {
        const uint32_t st = it % NST, use = it / NST;
        const uint32_t r = it % NRAW_DIV, ru = it / NRAW_DIV;
        uint8_t* sX = smem + st * STAGE;
        uint8_t* sE = sX + XBYTES;
        const uint8_t* rb = rawring + r * DB_RAW_BYTES;
        const int kv = min(KC, S.n - KC * c);
        if (use >= 1 && !mbar_wait(smem_u32(&empty[st]), (use - 1) & 1u, wl)) ws_fail(abort_s, status);
        if (!mbar_wait(smem_u32(&raw_full[r]), ru & 1u, wl)) ws_fail(abort_s, status);
        if (*abort_s) { stop = true; break; }
        if (tid == 0) {
          e_last = (int)it;
          mbar_expect_tx(smem_u32(&full_e[st]), (uint32_t)(KS * SLICE_BYTES));
          bulk_copy_g2s(smem_u32(sE),
                        PK_CK_SRC(S.ebase + (size_t)c * KS * SLICE_BYTES, KS * SLICE_BYTES, chk::SITE_MODE_ECOPY),
                        (uint32_t)(KS * SLICE_BYTES), smem_u32(&full_e[st]));
        }
        if constexpr (!TRANS) {
          // piece j: values k = 2q, 2q + 1 of row 8 w + 2 j + lane / 16 -> 4 bytes of every slice
          float4 v[4];
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            const int row = 8 * warp + 2 * j + (lane >> 4);
            v[j] = (row < nr && 2 * q < kv) ? *reinterpret_cast<const float4*>(rb + row * 256 + q * 16)
                                            : make_float4(0.f, 0.f, 0.f, 0.f);
          }
          mbar_arrive(smem_u32(&raw_empty[r]));
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            float2 a[KS];
            cut_ff_float2<KS>(make_float2(v[j].x, v[j].z), make_float2(v[j].y, v[j].w), xsc, a);
            const int row = 8 * warp + 2 * j + (lane >> 4);
            const uint32_t off = chunk_offset(row, q >> 2) + (uint32_t)(q & 3) * 4u;
#pragma unroll
            for (int sl = 0; sl < KS; ++sl)
              *reinterpret_cast<uint32_t*>(sX + sl * DB_XSLICE + off) = pack_bf16x2(a[sl].x, a[sl].y);
          }
        } else {
          // fiber fib, values k = 8 kg .. 8 kg + 7 (lanes read consecutive fibers)
          float2 f[8];
#pragma unroll
          for (int e = 0; e < 8; ++e) {
            const int k = 8 * kg + e;
            f[e] = (fib < nr && k < kv) ? *reinterpret_cast<const float2*>(rb + k * 512 + fib * 8)
                                        : make_float2(0.f, 0.f);
          }
          mbar_arrive(smem_u32(&raw_empty[r]));
          uint32_t pk[KS][4];
#pragma unroll
          for (int e = 0; e < 8; e += 2) {
            float2 a[KS];
            cut_ff_float2<KS>(make_float2(f[e].x, f[e + 1].x), make_float2(f[e].y, f[e + 1].y), xsc, a);
#pragma unroll
            for (int sl = 0; sl < KS; ++sl) pk[sl][e >> 1] = pack_bf16x2(a[sl].x, a[sl].y);
          }
          const uint32_t off = chunk_offset(fib, kg);
#pragma unroll
          for (int sl = 0; sl < KS; ++sl)
            *reinterpret_cast<uint4*>(sX + sl * DB_XSLICE + off) = make_uint4(pk[sl][0], pk[sl][1], pk[sl][2], pk[sl][3]);
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        mbar_arrive(smem_u32(&full_x[st]));
      }
    }
    if (tid == 0 && *abort_s) {
      // bulk copies still in flight must land before the CTA's shared memory is released
      for (int k = e_last; k >= 0 && k >= e_last - (NST - 1); --k)
        mbar_wait(smem_u32(&full_e[k % NST]), ((uint32_t)k / NST) & 1u, CLEANUP_WAIT_NS);
    }
  } else if (!RR && warp < WS_EPI0) {
    // ------------------------------------------------------------ producers
    const int fib = tid & 63;   // fiber of the tile
    const int kg = tid >> 6;    // k-group (8 values) of every 32-wide chunk
    uint32_t it = 0, tc = 0;
    int e_last = -1;            // thread 0: chunk of the latest E bulk copy
    long long tile = blockIdx.x;
    WsSlot S, Sn;
    Raw<IN_F64> r0, r1, r2;     // chunks it, it+1 and (in flight) it+2
    bool have = false;
    if (tile < total_tiles) {
      have = ws_get(slots, slot_full, slot_empty, 0, S, wl);
      if (!have) ws_fail(abort_s, status);
    }
    if (have) {
      db_load<IN_F64, TRANS>(S, fib, 8 * kg, r0);
      db_load<IN_F64, TRANS>(S, fib, 32 + 8 * kg, r1);
    }
    bool stop = false;
    for (; have && tile < total_tiles; tile += gridDim.x, ++tc) {
      const int nchunks = S.nsub;
      const int eb = 1011 + S.eX;
      const float xsc = pow2f_full(-S.eX);
      const bool has_next = tile + gridDim.x < total_tiles;
      bool have_next = false;
      for (int c = 0; c < nchunks; ++c, ++it) {
        const uint32_t st = it % NST, use = it / NST;
        uint8_t* sX = smem + st * STAGE;
        uint8_t* sE = sX + XBYTES;
        // chunk it + 2 in flight before the wait for a free stage
        if (c + 2 < nchunks) {
          db_load<IN_F64, TRANS>(S, fib, 32 * (c + 2) + 8 * kg, r2);
        } else {
          if (c + 2 == nchunks && has_next) {
            have_next = ws_get(slots, slot_full, slot_empty, tc + 1, Sn, wl);
            if (!have_next) ws_fail(abort_s, status);
          }
          if (have_next) db_load<IN_F64, TRANS>(Sn, fib, 32 * (c + 2 - nchunks) + 8 * kg, r2);
        }
        if (use >= 1 && !mbar_wait(smem_u32(&empty[st]), (use - 1) & 1u, wl)) ws_fail(abort_s, status);
        if (*abort_s) { stop = true; break; }
        if (tid == 0) {
          e_last = (int)it;
          mbar_expect_tx(smem_u32(&full_e[st]), (uint32_t)(KS * SLICE_BYTES));
          bulk_copy_g2s(smem_u32(sE),
                        PK_CK_SRC(S.ebase + (size_t)c * KS * SLICE_BYTES, KS * SLICE_BYTES, chk::SITE_MODE_ECOPY),
                        (uint32_t)(KS * SLICE_BYTES), smem_u32(&full_e[st]));
        }
        uint32_t pk[KS][4];
#pragma unroll
        for (int e = 0; e < 8; e += 2) {
          if (IN_F64) {
            uint32_t s0, s1;
            const uint64_t F0 = round_digits<KS>(fixed_f64(r0.d[e], eb, s0));
            const uint64_t F1 = round_digits<KS>(fixed_f64(r0.d[e + 1], eb, s1));
            uint32_t w[KS];
            cut_pair<KS>(F0, s0, F1, s1, w);
#pragma unroll
            for (int sl = 0; sl < KS; ++sl) pk[sl][e >> 1] = w[sl];
          } else {
            float2 v[KS];
            cut_ff_float2<KS>(make_float2(r0.f[e].x, r0.f[e + 1].x), make_float2(r0.f[e].y, r0.f[e + 1].y), xsc, v);
#pragma unroll
            for (int sl = 0; sl < KS; ++sl) pk[sl][e >> 1] = pack_bf16x2(v[sl].x, v[sl].y);
          }
        }
        const uint32_t off = chunk_offset(fib, kg);
#pragma unroll
        for (int sl = 0; sl < KS; ++sl)
          *reinterpret_cast<uint4*>(sX + sl * DB_XSLICE + off) = make_uint4(pk[sl][0], pk[sl][1], pk[sl][2], pk[sl][3]);
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        mbar_arrive(smem_u32(&full_x[st]));
        r0 = r1;
        r1 = r2;
      }
      if (stop) break;
      S = Sn;
    }
    if (tid == 0 && *abort_s) {
      // bulk copies still in flight must land before the CTA's shared memory is released
      for (int k = e_last; k >= 0 && k >= e_last - (NST - 1); --k)
        mbar_wait(smem_u32(&full_e[k % NST]), ((uint32_t)k / NST) & 1u, CLEANUP_WAIT_NS);
    }
  } else if (warp < WS_MMA) {
    // ------------------------------------------------------------ epilogue
    const int q4 = warp - WS_EPI0;     // TMEM lane quarter (= warp % 4)
    const int i = q4 * 32 + lane;      // E row of this thread (TMEM lane)
    uint32_t tc = 0;
    for (long long tile = blockIdx.x; tile < total_tiles; tile += gridDim.x, ++tc) {
      const uint32_t b = tc & 1u, u = tc >> 1;
      WsSlot S;
      bool ok = ws_get(slots, slot_full, slot_empty, tc, S, wl);
      ok = ok && mbar_wait(smem_u32(&tmem_full[b]), u & 1u, wl);
      if (!ok) ws_fail(abort_s, status);
      // every epilogue thread decides alike; the vote is also the barrier that frees the
      // staging area of the previous tile
      if (epi_vote_any(!ok || *abort_s)) break;
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t tb = tmem + 256u * b + ((uint32_t)(q4 * 32) << 16);
      const bool vi = i < S.nrows_e;
      const float sc = pow2f(S.eX + ((vi && PK_CK(S.rexp + i, sizeof(int), chk::SITE_MODE_REXP)) ? __ldg(S.rexp + i) : 0));
      const int ncols = TRANS ? (int)min(64LL, S.R - S.g0) : (int)min(64LL, S.B0 - S.g0);
      const bool f64 = S.out_f64 != 0;
      uint32_t mx = 0;
      for (int cc = 0; cc < ncols; cc += 16) {
        float d2[16], d3[16], d4[16], d5[16];
        tmem_ld16(tb + (uint32_t)cc, d2);
        tmem_ld16(tb + 64u + (uint32_t)cc, d3);
        tmem_ld16(tb + 128u + (uint32_t)cc, d4);
        if (KS >= 4) tmem_ld16(tb + 192u + (uint32_t)cc, d5);
        tmem_wait_ld();
        float hs[16], ls[16];
#pragma unroll
        for (int j = 0; j < 16; j += 2) {
          float2 hi, lo;
          ff_combine2<KS>(make_float2(d2[j], d2[j + 1]), make_float2(d3[j], d3[j + 1]),
                          make_float2(d4[j], d4[j + 1]),
                          KS >= 4 ? make_float2(d5[j], d5[j + 1]) : make_float2(0.0f, 0.0f), hi, lo);
          hi = mul2(hi, make_float2(sc, sc));
          lo = mul2(lo, make_float2(sc, sc));
          hs[j] = hi.x;
          hs[j + 1] = hi.y;
          ls[j] = lo.x;
          ls[j + 1] = lo.y;
          mx = max(mx, __float_as_uint(hi.x) & 0x7FFFFFFFu);
          mx = max(mx, __float_as_uint(hi.y) & 0x7FFFFFFFu);
        }
        if (TRANS) {
          // row i of the staged tile: 16 columns as 8 pairs of 16 bytes
          uint8_t* row = staging + i * DB_STAGE_PITCH + cc * 8;
          if (!f64) {
#pragma unroll
            for (int j = 0; j < 16; j += 2)
              *reinterpret_cast<float4*>(row + j * 8) = make_float4(hs[j], ls[j], hs[j + 1], ls[j + 1]);
          } else {
#pragma unroll
            for (int j = 0; j < 16; j += 2)
              *reinterpret_cast<double2*>(row + j * 8) =
                  make_double2(ff_to_f64(hs[j], ls[j]), ff_to_f64(hs[j + 1], ls[j + 1]));
          }
        } else if (vi) {
          const int jn = ncols - cc;  // >= 16 unless this is the tile's last group
          const long long o = (S.g0 + cc) * (long long)S.n + 128 * S.rb + i;
          if (!f64) {
            float2* dst = reinterpret_cast<float2*>(S.out) + o;
#pragma unroll
            for (int j = 0; j < 16; ++j)
              if (j < jn) st_ck(dst + (long long)j * S.n, make_float2(hs[j], ls[j]), chk::SITE_MODE_STORE);
          } else {
            double* dst = reinterpret_cast<double*>(S.out) + o;
#pragma unroll
            for (int j = 0; j < 16; ++j)
              if (j < jn) st_ck(dst + (long long)j * S.n, ff_to_f64(hs[j], ls[j]), chk::SITE_MODE_STORE);
          }
        }
      }
      // the accumulators of buffer b are free for tile t+2
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      mbar_arrive(smem_u32(&tmem_empty[b]));
      if (TRANS) {
        asm volatile("bar.sync 1, 128;" ::: "memory");  // the staged tile is complete
        // rows q4, q4+4, ...: 64 consecutive fibers = 512 contiguous bytes in the output
        const int nrows = S.nrows_e;
        for (int r = q4; r < nrows; r += 4) {
          const int c2 = 2 * lane;  // this lane's column pair
          if (c2 < ncols) {
            const long long o = S.base + (long long)(128 * S.rb + r) * S.R + S.g0 + c2;
            const uint8_t* src = staging + r * DB_STAGE_PITCH + c2 * 8;
            if (!f64) {
              st_ck(reinterpret_cast<float4*>(reinterpret_cast<float2*>(S.out) + o), *reinterpret_cast<const float4*>(src),
                    chk::SITE_MODE_STORE);
            } else {
              // the caller's float64 buffer need only be 8-byte aligned
              const double2 v = *reinterpret_cast<const double2*>(src);
              double* dst = reinterpret_cast<double*>(S.out) + o;
              st_ck(dst, v.x, chk::SITE_MODE_STORE);
              st_ck(dst + 1, v.y, chk::SITE_MODE_STORE);
            }
          }
        }
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
      // |v| < 2^{biased - 126}; a zero vector keeps the slot's initial (very negative) value
      const int emax = (int)(mx >> 23);
      if (lane == 0 && emax > 0) out_exp_max(S.out_exp, emax - 126);
    }
  } else if (warp == WS_MMA || warp == WS_MMA2) {
    if (lane == 0) {
      // ---------------------------------------------------------- MMA issuers (two threads)
      const bool second = warp == WS_MMA2;
      uint32_t it = 0, tc = 0;
      bool issued = false;
      const uint32_t idesc = make_idesc(128, 64);
      for (long long tile = blockIdx.x; tile < total_tiles; tile += gridDim.x, ++tc) {
        const uint32_t b = tc & 1u, u = tc >> 1;
        WsSlot S;
        if (!ws_get(slots, slot_full, slot_empty, tc, S, wl)) ws_fail(abort_s, status);
        if (u >= 1 && !mbar_wait(smem_u32(&tmem_empty[b]), (u - 1) & 1u, wl)) ws_fail(abort_s, status);
        if (*abort_s) break;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        bool stop = false;
        for (int c = 0; c < S.nsub; ++c, ++it) {
          const uint32_t st = it % NST, use = it / NST;
          if (!mbar_wait(smem_u32(&full_x[st]), use & 1u, wl) || !mbar_wait(smem_u32(&full_e[st]), use & 1u, wl))
            ws_fail(abort_s, status);
          if (*abort_s) { stop = true; break; }
          asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
          const uint32_t xa = smem_u32(smem + st * STAGE);
          const uint32_t xlo = desc_lo(xa), elo = desc_lo(xa + XBYTES);
          const uint32_t acc0 = tmem + 256u * b;
          if (second) {
            if (c == 0)
              issue_chunk<KS, true, true, 64, DB_XSLICE, WS_MASK2>(acc0, xlo, elo, idesc);
            else
              issue_chunk<KS, false, true, 64, DB_XSLICE, WS_MASK2>(acc0, xlo, elo, idesc);
          } else {
            if (c == 0)
              issue_chunk<KS, true, true, 64, DB_XSLICE, WS_MASK1>(acc0, xlo, elo, idesc);
            else
              issue_chunk<KS, false, true, 64, DB_XSLICE, WS_MASK1>(acc0, xlo, elo, idesc);
          }
          issued = true;
          mma_commit(smem_u32(&empty[st]));
        }
        if (stop) break;
        mma_commit(smem_u32(&tmem_full[b]));
      }
      // every MMA this thread issued is complete before TMEM is released
      mma_commit(smem_u32(done));
      if (issued) mbar_wait(smem_u32(done), 0u, CLEANUP_WAIT_NS);
    }
  } else if (RR && warp == WS_SCHED) {
    // ------------------------------------------------------------ scheduler + raw copies (warp 13)
    int job = 0;
    uint32_t tc = 0, it = 0;
    long long r_last = -1;   // chunk of the latest raw copy
    bool stop = false;
    for (long long tile = blockIdx.x; tile < total_tiles && !stop; tile += gridDim.x, ++tc) {
      const uint32_t q = tc % WS_SLOTS;
      bool ok = tc < WS_SLOTS || mbar_wait(smem_u32(&slot_empty[q]), ((tc / WS_SLOTS) - 1) & 1u, wl);
      if (!ok) ws_fail(abort_s, status);
      if (__any_sync(0xffffffffu, !ok || *abort_s)) break;   // warp-uniform
      WsSlot L;
      db_make_slot<KS, TRANS>(P, tile, job, L);   // every lane computes the same slot
      if (lane == 0) {
        slots[q] = L;
        mbar_arrive(smem_u32(&slot_full[q]));
      }
      for (int c = 0; c < L.nsub; ++c, ++it) {
        const uint32_t r = it % NRAW_DIV, ru = it / NRAW_DIV;
        ok = ru == 0 || mbar_wait(smem_u32(&raw_empty[r]), (ru - 1) & 1u, wl);
        if (!ok) ws_fail(abort_s, status);
        if (__any_sync(0xffffffffu, !ok || *abort_s)) { stop = true; break; }
        if (lane == 0) db_raw_tma<TRANS>(P, job, L, c, rawring + r * DB_RAW_BYTES, &raw_full[r]);
        r_last = it;
      }
    }
    if (lane == 0 && *abort_s) {
      // raw copies still in flight must land before the CTA's shared memory is released
      for (long long k = r_last; k >= 0 && k >= r_last - (NRAW - 1); --k)
        mbar_wait(smem_u32(&raw_full[k % NRAW_DIV]), (uint32_t)(k / NRAW_DIV) & 1u, CLEANUP_WAIT_NS);
    }
  } else if (!RR && warp == WS_SCHED && lane == 0) {
    // ------------------------------------------------------------ scheduler (64-fiber tiles)
    int job = 0;
    uint32_t tc = 0;
    for (long long tile = blockIdx.x; tile < total_tiles; tile += gridDim.x, ++tc) {
      const uint32_t q = tc % WS_SLOTS;
      if (tc >= WS_SLOTS && !mbar_wait(smem_u32(&slot_empty[q]), ((tc / WS_SLOTS) - 1) & 1u, wl))
        ws_fail(abort_s, status);
      if (*abort_s) break;
      db_make_slot<KS, TRANS>(P, tile, job, slots[q]);
      mbar_arrive(smem_u32(&slot_full[q]));
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512));
}

__global__ void ptrtab_set_kernel(void** tab, PtrArgs args) {
  const int i = threadIdx.x;
  if (i < args.n) st_ck(tab + i, args.p[i], chk::SITE_TABLE);
}

}  // namespace

size_t smem_bytes(int ks, int sub) {
  return (size_t)2 * 2 * sub * ks * SLICE_BYTES + 128 + 512 + 16 + 16 + 16;
}

template <int KS, int SUB, bool IN_F64, bool TRANS>
int launch_one(const GPass& P, int grid, bool ws, bool rr, bool pc, int* status, cudaStream_t st) {
  // the warp-specialised kernel is built for 32-wide K chunks only (its 15 warps leave ~128
  // registers a thread, too few for the doubled raw-value buffers of 64-wide chunks)
  const bool use_ws = ws && SUB == 1;
  size_t sm = use_ws ? ws_smem_bytes(KS) : smem_bytes(KS, SUB);
  auto kern = use_ws ? mode_kernel_ws<KS, IN_F64, TRANS> : mode_kernel<KS, SUB, IN_F64, TRANS>;
  if constexpr (!IN_F64 && KS <= 5 && SUB == 1) {
    if (use_ws && rr) {
      kern = mode_kernel_ws<KS, false, TRANS, true>;
      sm = ws_smem_bytes_rr(KS);
    }
  }
  if constexpr (IN_F64 && TRANS && SUB == 1) {
    if (use_ws && pc) kern = mode_kernel_ws<KS, true, true, false, true>;
  }
  const int threads = use_ws ? WS_THREADS : NTHREADS;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) {
    set_error(std::string("tc mode kernel smem attribute: ") + cudaGetErrorString(e));
    return PHIKRON_ECUDA;
  }
  launch_begin(KC_TC_MODE, st);
  kern<<<grid, threads, sm, st>>>(P, status);
  launch_end(st);
  PK_CHECK_LAUNCH();
  return PHIKRON_OK;
}

template <int KS, int SUB>
int launch_ks(const GPass& P, bool in_f64, bool trans, int grid, bool ws, bool rr, bool pc, int* status,
              cudaStream_t st) {
  if (in_f64)
    return trans ? launch_one<KS, SUB, true, true>(P, grid, ws, false, pc, status, st)
                 : launch_one<KS, SUB, true, false>(P, grid, ws, false, false, status, st);
  return trans ? launch_one<KS, SUB, false, true>(P, grid, ws, rr, false, status, st)
               : launch_one<KS, SUB, false, false>(P, grid, ws, rr, false, status, st);
}

template <int KS, bool IN_F64, bool TRANS>
int launch_db(const GPass& P, int grid, bool rr, int* status, cudaStream_t st) {
  size_t sm = db_smem_bytes(KS);
  auto kern = mode_kernel_db<KS, IN_F64, TRANS>;
  if constexpr (!IN_F64 && KS <= 4) {
    if (rr) {
      kern = mode_kernel_db<KS, false, TRANS, true>;
      sm = db_smem_bytes_rr(KS);
    }
  }
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) {
    set_error(std::string("tc mode kernel smem attribute: ") + cudaGetErrorString(e));
    return PHIKRON_ECUDA;
  }
  launch_begin(KC_TC_MODE, st);
  kern<<<grid, WS_THREADS, sm, st>>>(P, status);
  launch_end(st);
  PK_CHECK_LAUNCH();
  return PHIKRON_OK;
}

template <int KS>
int launch_db_ks(const GPass& P, bool in_f64, bool trans, int grid, bool rr, int* status, cudaStream_t st) {
  if (in_f64)
    return trans ? launch_db<KS, true, true>(P, grid, false, status, st)
                 : launch_db<KS, true, false>(P, grid, false, status, st);
  return trans ? launch_db<KS, false, true>(P, grid, rr, status, st)
               : launch_db<KS, false, false>(P, grid, rr, status, st);
}

int mode_pass(const GPass& P, const PassShape& S, int* status, cudaStream_t st) {
  if (P.njobs <= 0 || P.total_tiles <= 0) return PHIKRON_OK;
  const int grid = (int)std::min<long long>(P.total_tiles, S.grid);
  const bool rr = S.rr && P.tmaps != nullptr;   // the raw ring needs its tensor maps
  if (S.db) {
    switch (S.slices) {
      case 3: return launch_db_ks<3>(P, S.in_f64, S.trans, grid, rr, status, st);
      case 4: return launch_db_ks<4>(P, S.in_f64, S.trans, grid, rr, status, st);
      case 5: return launch_db_ks<5>(P, S.in_f64, S.trans, grid, rr, status, st);
      case 6: return launch_db_ks<6>(P, S.in_f64, S.trans, grid, rr, status, st);
      default: break;
    }
    set_error("tc mode pass: unsupported slice count");
    return PHIKRON_EINVAL;
  }
  if (S.sub == 1) {
    switch (S.slices) {
      case 3: return launch_ks<3, 1>(P, S.in_f64, S.trans, grid, S.ws, rr, S.pc, status, st);
      case 4: return launch_ks<4, 1>(P, S.in_f64, S.trans, grid, S.ws, rr, S.pc, status, st);
      case 5: return launch_ks<5, 1>(P, S.in_f64, S.trans, grid, S.ws, rr, S.pc, status, st);
      case 6: return launch_ks<6, 1>(P, S.in_f64, S.trans, grid, S.ws, rr, S.pc, status, st);
      default: break;
    }
  } else if (S.sub == 2 && S.slices == 3) {
    return launch_ks<3, 2>(P, S.in_f64, S.trans, grid, S.ws, false, false, status, st);
  }
  set_error("tc mode pass: unsupported (slices, sub-chunks) combination");
  return PHIKRON_EINVAL;
}

// TMA tensor maps of the inputs of a raw-ring pass's jobs (one 128-byte CUtensorMap each, in
// job order), encoded with the driver's cuTensorMapEncodeTiled (looked up through the runtime,
// no link against the driver library).  PHIKRON_ENOTSUP if the driver lacks it or refuses a map.
using EncodeTiled = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                 const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                 CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

int encode_raw_maps(const GJob* jobs, int njobs, bool trans, int fibers, uint8_t* out) {
  static EncodeTiled encode = nullptr;
  static bool looked = false;
  if (!looked) {
    looked = true;
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      encode = reinterpret_cast<EncodeTiled>(fn);
    cudaGetLastError();
  }
  if (!encode) return PHIKRON_ENOTSUP;
  static_assert(sizeof(CUtensorMap) == 128, "tensor map size");
  for (int j = 0; j < njobs; ++j) {
    const GJob& J = jobs[j];
    CUtensorMap m;
    const cuuint32_t estr[3] = {1, 1, 1};
    CUresult r;
    if (!trans) {
      const cuuint64_t dim[2] = {(cuuint64_t)J.n, (cuuint64_t)J.B0};
      const cuuint64_t str[1] = {(cuuint64_t)J.n * 8};
      const cuuint32_t box[2] = {(cuuint32_t)KC, (cuuint32_t)fibers};
      r = encode(&m, CU_TENSOR_MAP_DATA_TYPE_UINT64, 2, const_cast<void*>(J.in), dim, str, box, estr,
                 CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                 CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    } else {
      const cuuint64_t dim[3] = {(cuuint64_t)J.R, (cuuint64_t)J.n, (cuuint64_t)J.B0};
      const cuuint64_t str[2] = {(cuuint64_t)J.R * 8, (cuuint64_t)J.n * J.R * 8};
      const cuuint32_t box[3] = {(cuuint32_t)fibers, (cuuint32_t)KC, 1};
      r = encode(&m, CU_TENSOR_MAP_DATA_TYPE_UINT64, 3, const_cast<void*>(J.in), dim, str, box, estr,
                 CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                 CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    }
    if (r != CUDA_SUCCESS) return PHIKRON_ENOTSUP;
    std::memcpy(out + 128 * (size_t)j, &m, 128);
  }
  return PHIKRON_OK;
}

size_t precut_bytes(long long R, int n, int slices) {
  return (size_t)((R + 127) / 128) * (size_t)((n + 31) / 32) * (size_t)slices * SLICE_BYTES;
}

int precut_pass(const GPass& P, int slices, int* status, cudaStream_t st) {
  (void)status;
  if (P.njobs <= 0 || P.total_tiles <= 0) return PHIKRON_OK;
  int dev = 0, nsm = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  const unsigned grid = (unsigned)std::min<long long>(P.total_tiles, (long long)nsm * 4);
  launch_begin(KC_CONVERT, st);
  if (slices == 3) {
    precut_kernel<3><<<grid, WS_PROD, 0, st>>>(P);
  } else if (slices == 4) {
    precut_kernel<4><<<grid, WS_PROD, 0, st>>>(P);
  } else if (slices == 5) {
    precut_kernel<5><<<grid, WS_PROD, 0, st>>>(P);
  } else if (slices == 6) {
    precut_kernel<6><<<grid, WS_PROD, 0, st>>>(P);
  } else {
    launch_end(st);
    set_error("pre-cut input: 3 to 6 digit slices");
    return PHIKRON_EINVAL;
  }
  launch_end(st);
  PK_CHECK_LAUNCH();
  return PHIKRON_OK;
}

int set_ptrtab(void** tab, const PtrArgs& args, cudaStream_t st) {
  launch_begin(KC_OTHER, st);
  ptrtab_set_kernel<<<1, 128, 0, st>>>(tab, args);
  launch_end(st);
  PK_CHECK_LAUNCH();
  return PHIKRON_OK;
}

}  // namespace tc
}  // namespace phikron
