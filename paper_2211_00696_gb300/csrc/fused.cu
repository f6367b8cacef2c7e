// K2 with the node weights of Algorithm 1 in the epilogue: the last mode product of every
// quadrature node, fused with the weighted sums y_j = sum_k w_k x_k^{j-1}/(j-1)! T_k (Sec. 3.1,
// Algorithm 1), so that the node products T_k are never written to HBM.
//
// The pass contracts the fastest axis (Eq. (8) with R = 1): T_k[f][i] = sum_q E_k[i][q] X_k[f][q]
// for the fibers f of the slower axes.  One tile is 32 fibers x all n <= 128 rows of E; for its
// tile a CTA runs the nodes of the unit one after the other (the m weighted nodes in order, then
// the "direct" nodes phi_0 and phi_0 at tau/2, whose products are stored as they are).  Per node
// the digit-slice MMAs (tcgen05, kind::f16, M = 128 E rows, N = 32 fibers, the same exact BF16
// slice products as tc_mode.cu) fill four level accumulators of 32 TMEM columns; two such sets
// alternate, so the MMAs of node k+1 run while the epilogue drains node k.  The epilogue forms
// T_k in float-float exactly like the separate mode kernel and adds c_{j,k} T_k into p
// float-float sums held in the other 256 TMEM columns (hi and lo, 32 columns each, j <= 4); at
// the last weighted node it writes y_j (float-float, or float64 when no squaring follows), with
// the same operations in the same order as the separate weighted-sum kernel: the results are
// bitwise those of the unfused pass pair.
//
// X of a (tile, node) is 32 consecutive fibers of n float-float values: one contiguous block,
// brought into shared memory by one bulk copy (cp.async.bulk) that the scheduler thread issues
// ahead into a ring of raw buffers; the producer warps cut it into digit slices chunk by chunk
// (32 K values), next to the chunk's E slices (one bulk copy each).  Roles (15 warps):
//   warps 0-3   producers: digit slices of X; thread 0 also starts each chunk's E copy
//   warps 4-11  epilogue: warp w owns TMEM lanes 32 (w % 4) .. + 31 (= rows i of E) and the
//               columns (fibers) 16 h .. 16 h + 15, h = (w - 4) / 4 (two warps per lane quarter)
//   warps 12,14 lane 0 issues the MMAs of accumulators {0, 3} resp. {1, 2}
//   warp 13     lane 0: per (tile, node) context into a 4-slot ring, and the raw X copies
// Every mbarrier wait is bounded (FPass::wait_ns); on expiry the CTA records PHIKRON_ETIMEOUT,
// every role stops at its next check, and the CTA waits for its own bulk copies and MMAs before
// it releases TMEM.
//
// Per (tile, node) step the slice MMAs (80 of N = 32 at 4 digit slices) take ~2.7 us, which
// bounds the pass; the write-out of y_j and of the direct products comes on top once per tile.
// On the 128^3 convection-diffusion workload (11 node vectors, 4 digit slices) the pass takes
// ~0.15 ms against ~0.10 + 0.06 ms for the separate last mode pass and weighted sums.
#include <algorithm>
#include <cstdint>

#include "checked.cuh"
#include "common.h"
#include "mixed.h"
#include "profile.h"
#include "tc_common.cuh"

PK_CHK_BIND(fused)

namespace phikron {
namespace tc {
namespace {

constexpr int FW_FIB = fused::kFibers;         // fibers per tile (MMA N)
constexpr int FW_XSL = FW_FIB * KC * 2;        // one X slice of a chunk: 32 rows x 64 B
constexpr int FW_RAW = FW_FIB * FW_MAXN * 8;   // raw float-float X of a (tile, node): 32 KB
constexpr int FW_EPI0 = 4, FW_MMA = 12, FW_SCHED = 13, FW_MMA2 = 14;
constexpr int FW_THREADS = 480, FW_PROD = 128, FW_EPI = 256, FW_ISSUERS = 2, FW_SLOTS = 4;
constexpr int FW_SLOT_READERS = FW_PROD + FW_ISSUERS + FW_EPI;
constexpr int FW_MASK1 = 0b1001, FW_MASK2 = 0b0110;
constexpr int FW_BAR_BYTES = 256, FW_SLOT_BYTES = 512;
// TMEM columns: level accumulators of node buffer b at 128 b + 32 a (a = level 0..3); the
// float-float sums of y_j at 256 + 64 (j-1) (hi) and + 32 (lo)
constexpr uint32_t FW_SUMS = 256;

enum : int { FW_DIRECT = 1, FW_FIRST = 2, FW_LAST = 4, FW_END = 8 };

__host__ __device__ constexpr int fw_stages(int ks) { return ks == 3 ? 4 : (ks <= 5 ? 3 : 2); }
__host__ __device__ constexpr int fw_raws(int ks) { return ks <= 4 ? 3 : 2; }
__host__ __device__ constexpr int fw_stage_bytes(int ks) { return ks * (FW_XSL + SLICE_BYTES); }
static_assert(3 * 4 + 2 * 3 + 2 + 2 + 1 + 2 * FW_SLOTS <= FW_BAR_BYTES / 8, "mbarrier area");

size_t fw_smem_bytes(int ks) {
  return (size_t)fw_stages(ks) * fw_stage_bytes(ks) + (size_t)fw_raws(ks) * FW_RAW + FW_BAR_BYTES +
         FW_SLOT_BYTES + 32;
}

struct FwSlot {
  const float2* xsrc;      // X of the tile: fibers f0.. of the node's input, n values each
  const uint8_t* ebase;    // E slices of the node
  const int* rexp;         // row exponents of E
  double* dout;            // direct node: output at fiber f0 (float64)
  float2 c[FW_MAXP];       // weighted node k: c_{j,k}, j = 1..p
  long long f0;
  unsigned xbytes;
  int n, nsub, nfib, eX, flags, job;
};
static_assert(sizeof(FwSlot) * FW_SLOTS <= FW_SLOT_BYTES, "slot ring");

// reads slot sc once it is filled, then releases it: lane >= 0 for a whole warp (one arrival
// of count 32), lane < 0 for a single thread
__device__ __forceinline__ bool fw_get(const FwSlot* slots, uint64_t* slot_full, uint64_t* slot_empty, uint32_t sc,
                                       FwSlot& out, unsigned long long wl, int lane) {
  const uint32_t q = sc % FW_SLOTS;
  const bool ok = mbar_wait(smem_u32(&slot_full[q]), (sc / FW_SLOTS) & 1u, wl);
  if (ok) out = slots[q];
  if (lane >= 0)
    mbar_arrive_warp(smem_u32(&slot_empty[q]), lane);
  else
    mbar_arrive(smem_u32(&slot_empty[q]));
  return ok;
}

using chk::st_ck;

// pointer-table entry plus offset, or the direct pointer
__device__ __forceinline__ void* fw_tab(const FPass& P, int tab, long long off, void* direct) {
  if (tab < 0) return direct;
  if (!PK_CK(P.ptrtab + tab, sizeof(void*), chk::SITE_TABLE)) return nullptr;
  return (void*)((char*)P.ptrtab[tab] + off);
}

__device__ __forceinline__ void tmem_ld8(uint32_t taddr, float* v) {
  uint32_t r[8];
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
               : "r"(taddr));
#pragma unroll
  for (int j = 0; j < 8; ++j) v[j] = __uint_as_float(r[j]);
}

__device__ __forceinline__ void tmem_st8(uint32_t taddr, const float* v) {
  asm volatile("tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8};" ::"r"(taddr),
               "r"(__float_as_uint(v[0])), "r"(__float_as_uint(v[1])), "r"(__float_as_uint(v[2])),
               "r"(__float_as_uint(v[3])), "r"(__float_as_uint(v[4])), "r"(__float_as_uint(v[5])),
               "r"(__float_as_uint(v[6])), "r"(__float_as_uint(v[7]))
               : "memory");
}

__device__ __forceinline__ void tmem_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }

// Writes this warp's column half ch of nvec float-float vectors of a tile from TMEM (hi at
// sums + 64 v, lo 32 columns further, column = fiber) to y + v * stride + col * n + i: float-float (yff), float64 (y64) and/or a
// float64 copy (y2); with out_exp, the exponent of each vector's largest |hi| goes to
// out_exp[v].  It runs once or twice per tile, so its loops stay rolled: fully unrolled copies
// of it in the node loop cost instruction-cache misses on every tile.  Called by every lane of
// an epilogue warp.
__device__ __forceinline__ void fw_write_out(uint32_t sums, int nvec, int ch, bool vi, int i, int lane, int n, int nfib,
                                          long long stride, float2* yff, double* y64, double* y2, int* out_exp) {
#pragma unroll 1
  for (int v = 0; v < nvec; ++v) {
    uint32_t mx = 0;
#pragma unroll 1
    for (int g = 2 * ch; g < 2 * ch + 2; ++g) {   // this warp's half, 8 columns at a time
      float h[8], l[8];
      tmem_ld8(sums + 64u * v + 8u * g, h);
      tmem_ld8(sums + 64u * v + 32u + 8u * g, l);
      tmem_wait_ld();
      if (vi) {
        const long long o = (long long)v * stride + (long long)(8 * g) * n + i;
#pragma unroll
        for (int q = 0; q < 8; ++q) {
          if (8 * g + q < nfib) {
            const long long e = o + (long long)q * n;
            if (yff) st_ck(yff + e, make_float2(h[q], l[q]), chk::SITE_FUSED_STORE);
            if (y64 || y2) {
              const double d = ff::to_f64(h[q], l[q]);
              if (y64) st_ck(y64 + e, d, chk::SITE_FUSED_STORE);
              if (y2) st_ck(y2 + e, d, chk::SITE_FUSED_STORE);
            }
            mx = max(mx, __float_as_uint(h[q]) & 0x7FFFFFFFu);
          }
        }
      }
    }
    if (out_exp) {
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
      // |y| < 2^{biased - 126}; a zero output keeps the slot's initial (very negative) value
      const int emax = (int)(mx >> 23);
      if (lane == 0 && emax > 0 && PK_CK(out_exp + v, sizeof(int), chk::SITE_FUSED_STORE))
        atomicMax(out_exp + v, emax - 126);
    }
  }
}

template <int KS, int P_>
__global__ void __launch_bounds__(FW_THREADS, 1) fused_weights_kernel(const __grid_constant__ FPass P, int* status) {
  extern __shared__ __align__(1024) uint8_t smem[];
  constexpr int NST = fw_stages(KS);
  constexpr int NRAW = fw_raws(KS);
  constexpr int STAGE = fw_stage_bytes(KS);
  constexpr int XBYTES = KS * FW_XSL;
  uint8_t* rawbuf = smem + NST * STAGE;
  uint8_t* tail = rawbuf + NRAW * FW_RAW;
  uint64_t* bars = reinterpret_cast<uint64_t*>(tail);
  uint64_t* full_x = bars;                          // [NST]  producer arrivals
  uint64_t* full_e = bars + NST;                    // [NST]  E bulk copy bytes
  uint64_t* empty = bars + 2 * NST;                 // [NST]  MMA commits
  uint64_t* raw_full = bars + 3 * NST;              // [NRAW] X bulk copy bytes
  uint64_t* raw_empty = bars + 3 * NST + NRAW;      // [NRAW] producer arrivals
  uint64_t* tmem_full = bars + 3 * NST + 2 * NRAW;  // [2]    MMA commits
  uint64_t* tmem_empty = tmem_full + 2;             // [2]    epilogue arrivals
  uint64_t* done = tmem_empty + 2;
  uint64_t* slot_full = done + 1;                   // [FW_SLOTS]
  uint64_t* slot_empty = slot_full + FW_SLOTS;      // [FW_SLOTS]
  FwSlot* slots = reinterpret_cast<FwSlot*>(tail + FW_BAR_BYTES);
  uint32_t* tmem_s = reinterpret_cast<uint32_t*>(tail + FW_BAR_BYTES + FW_SLOT_BYTES);
  volatile int* abort_s = reinterpret_cast<volatile int*>(tail + FW_BAR_BYTES + FW_SLOT_BYTES + 16);

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const long long total_tiles = P.total_tiles;
#ifdef PHIKRON_CHECKED
  // a launch whose tables are not registered does nothing (uniform over the CTA)
  if (!PK_CK(P.jobs, sizeof(FJob) * (size_t)P.njobs, chk::SITE_TABLE) ||
      (P.ptrtab && !PK_CK(P.ptrtab, sizeof(void*) * MAX_PTRS, chk::SITE_TABLE)))
    return;
#endif
  const unsigned long long wl = P.wait_ns;
  if (tid == 0) {
    for (int q = 0; q < NST; ++q) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&full_x[q])), "r"(FW_PROD));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&full_e[q])));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&empty[q])), "r"(FW_ISSUERS));
    }
    for (int q = 0; q < NRAW; ++q) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&raw_full[q])));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&raw_empty[q])), "r"(FW_PROD));
    }
    for (int q = 0; q < 2; ++q) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&tmem_full[q])), "r"(FW_ISSUERS));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&tmem_empty[q])), "r"(FW_EPI));
    }
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(done)), "r"(FW_ISSUERS));
    for (int q = 0; q < FW_SLOTS; ++q) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&slot_full[q])));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&slot_empty[q])), "r"(FW_SLOT_READERS));
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

  if (warp < FW_EPI0) {
    // ------------------------------------------------------------ producers
    // a load instruction covers two fibers' 256-byte chunk rows (lane = 16-byte piece q of fiber
    // 8 w + 2 j + lane / 16, j = 0..3): consecutive shared-memory addresses, where one fiber per
    // four lanes put every lane of a warp on the same two bank groups
    const int q = lane & 15;   // K values 2q, 2q + 1 of every 32-wide chunk
    uint32_t sc = 0, it = 0;
    int e_last = -1;           // thread 0: chunk of the latest E bulk copy
    bool stop = false;
    for (long long tile = blockIdx.x; tile < total_tiles && !stop; tile += gridDim.x) {
      while (true) {
        FwSlot S;
        const uint32_t r = sc % NRAW;
        if (!fw_get(slots, slot_full, slot_empty, sc, S, wl, lane) ||
            !mbar_wait(smem_u32(&raw_full[r]), (sc / NRAW) & 1u, wl))
          ws_fail(abort_s, status);
        if (__any_sync(0xffffffffu, *abort_s)) { stop = true; break; }   // warp-uniform
        const float xsc = pow2f_full(-S.eX);
        const float2* raw = reinterpret_cast<const float2*>(rawbuf + r * FW_RAW);
        for (int c = 0; c < S.nsub; ++c, ++it) {
          const uint32_t st = it % NST, use = it / NST;
          uint8_t* sX = smem + st * STAGE;
          if (use >= 1 && !mbar_wait(smem_u32(&empty[st]), (use - 1) & 1u, wl)) ws_fail(abort_s, status);
          if (__any_sync(0xffffffffu, *abort_s)) { stop = true; break; }
          if (tid == 0) {
            e_last = (int)it;
            mbar_expect_tx(smem_u32(&full_e[st]), (uint32_t)(KS * SLICE_BYTES));
            bulk_copy_g2s(smem_u32(sX + XBYTES),
                          PK_CK_SRC(S.ebase + (size_t)c * KS * SLICE_BYTES, KS * SLICE_BYTES, chk::SITE_FUSED_ECOPY),
                          (uint32_t)(KS * SLICE_BYTES),
                          smem_u32(&full_e[st]));
          }
          const int k = c * KC + 2 * q;   // n is a multiple of 16: k < n covers k + 1
          float4 v[4];
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            const int f = 8 * warp + 2 * j + (lane >> 4);
            v[j] = (f < S.nfib && k < S.n) ? *reinterpret_cast<const float4*>(raw + (long long)f * S.n + k)
                                          : make_float4(0.f, 0.f, 0.f, 0.f);
          }
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            float2 a[KS];
            cut_ff_float2<KS>(make_float2(v[j].x, v[j].z), make_float2(v[j].y, v[j].w), xsc, a);
            const int f = 8 * warp + 2 * j + (lane >> 4);
            const uint32_t off = chunk_offset(f, q >> 2) + (uint32_t)(q & 3) * 4u;
#pragma unroll
            for (int sl = 0; sl < KS; ++sl)
              *reinterpret_cast<uint32_t*>(sX + sl * FW_XSL + off) = pack_bf16x2(a[sl].x, a[sl].y);
          }
          asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
          mbar_arrive_warp(smem_u32(&full_x[st]), lane);
        }
        if (stop) break;
        mbar_arrive_warp(smem_u32(&raw_empty[r]), lane);   // this warp is done with the raw X of step sc
        ++sc;
        if (S.flags & FW_END) break;
      }
    }
    if (tid == 0 && *abort_s) {
      // E copies still in flight land before the CTA's shared memory is released
      for (int k = e_last; k >= 0 && k >= e_last - (NST - 1); --k)
        mbar_wait(smem_u32(&full_e[k % NST]), ((uint32_t)k / NST) & 1u, CLEANUP_WAIT_NS);
    }
  } else if (warp < FW_MMA) {
    // ------------------------------------------------------------ epilogue
    const int i = (warp & 3) * 32 + lane;         // TMEM lane = row i of E = output index along the fastest axis
    const int ch = (warp - FW_EPI0) >> 2;         // column half: fibers 16 ch .. 16 ch + 15
    const uint32_t lane_base = tmem + ((uint32_t)((warp & 3) * 32) << 16);
    uint32_t sc = 0;
    bool stop = false;
    for (long long tile = blockIdx.x; tile < total_tiles && !stop; tile += gridDim.x) {
      while (true) {
        FwSlot S;
        const uint32_t b = sc & 1u;
        bool ok = fw_get(slots, slot_full, slot_empty, sc, S, wl, lane);
        ok = ok && mbar_wait(smem_u32(&tmem_full[b]), (sc >> 1) & 1u, wl);
        if (!ok) ws_fail(abort_s, status);
        if (epi_vote_any256(!ok || *abort_s)) { stop = true; break; }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const bool vi = i < S.n;
        const float scl =
            pow2f(S.eX + ((vi && PK_CK(S.rexp + i, sizeof(int), chk::SITE_FUSED_READ)) ? __ldg(S.rexp + i) : 0));
        const float2 sc2 = make_float2(scl, scl);
        const bool direct = (S.flags & FW_DIRECT) != 0;
        const bool first = (S.flags & FW_FIRST) != 0;
        const uint32_t lv = lane_base + 128u * b;
        const uint32_t sums = lane_base + FW_SUMS;
        // two groups of 8 columns (fibers) of this warp's half: a group's level values, T_k and
        // sums stay in registers
#pragma unroll
        for (int gg = 0; gg < 2; ++gg) {
          const int g = 2 * ch + gg;
          const int cc = 8 * g;
          float d2[8], d3[8], d4[8], d5[8];
          tmem_ld8(lv + (uint32_t)cc, d2);
          tmem_ld8(lv + 32u + (uint32_t)cc, d3);
          tmem_ld8(lv + 64u + (uint32_t)cc, d4);
          if (KS >= 4) tmem_ld8(lv + 96u + (uint32_t)cc, d5);
          tmem_wait_ld();
          if (gg == 1) {
            // this warp's column groups are in registers: its part of buffer b is free
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            mbar_arrive_warp(smem_u32(&tmem_empty[b]), lane);
          }
          float2 th[4], tl[4];   // T_k of columns (cc + 2q, cc + 2q + 1): hi pair, lo pair
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            const int j = 2 * q;
            float2 hi, lo;
            ff_combine2<KS>(make_float2(d2[j], d2[j + 1]), make_float2(d3[j], d3[j + 1]),
                            make_float2(d4[j], d4[j + 1]),
                            KS >= 4 ? make_float2(d5[j], d5[j + 1]) : make_float2(0.0f, 0.0f), hi, lo);
            th[q] = mul2(hi, sc2);
            tl[q] = mul2(lo, sc2);
          }
          if (direct) {
            // the product leaves through the write-out below: parked in the columns of y_1, free
            // since the tile's sums were written out at its last weighted node
            float h[8], l[8];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
              h[2 * q] = th[q].x;
              h[2 * q + 1] = th[q].y;
              l[2 * q] = tl[q].x;
              l[2 * q + 1] = tl[q].y;
            }
            tmem_st8(sums + (uint32_t)cc, h);
            tmem_st8(sums + 32u + (uint32_t)cc, l);
            continue;
          }
#pragma unroll
          for (int jj = 0; jj < P_; ++jj) {
            const uint32_t sa = sums + 64u * jj + (uint32_t)cc;
            float sh[8], sl[8];
            if (first) {
#pragma unroll
              for (int q = 0; q < 8; ++q) sh[q] = sl[q] = 0.0f;
            } else {
              tmem_ld8(sa, sh);
              tmem_ld8(sa + 32u, sl);
              tmem_wait_ld();
            }
            const float2 cj = S.c[jj];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
              float2 ah = make_float2(sh[2 * q], sh[2 * q + 1]), al = make_float2(sl[2 * q], sl[2 * q + 1]);
              ff::fma_ff2(ah, al, cj, th[q], tl[q]);
              sh[2 * q] = ah.x;
              sh[2 * q + 1] = ah.y;
              sl[2 * q] = al.x;
              sl[2 * q + 1] = al.y;
            }
            tmem_st8(sa, sh);
            tmem_st8(sa + 32u, sl);
          }
        }
        tmem_wait_st();   // the sums (or the parked product) are in TMEM before they are read
        if (direct) {
          fw_write_out(sums, 1, ch, vi, i, lane, S.n, S.nfib, 0, nullptr, S.dout, nullptr, nullptr);
        } else if (S.flags & FW_LAST) {
          const FJob& J = P.jobs[S.job];
          void* o = fw_tab(P, J.out_tab, J.tab_off_out, J.out);
          void* o2 = fw_tab(P, J.out2_tab, J.tab_off_out2, J.out2);
          const long long t0 = S.f0 * (long long)S.n;
          float2* yff = J.out_f64 ? nullptr : reinterpret_cast<float2*>(o) + t0;
          double* y64 = J.out_f64 ? reinterpret_cast<double*>(o) + t0 : nullptr;
          double* y2 = o2 ? reinterpret_cast<double*>(o2) + t0 : nullptr;
          fw_write_out(sums, P_, ch, vi, i, lane, S.n, S.nfib, J.stride, yff, y64, y2, J.out_exp);
        }
        ++sc;
        if (S.flags & FW_END) break;
      }
    }
  } else if (warp == FW_MMA || warp == FW_MMA2) {
    if (lane == 0) {
      // ---------------------------------------------------------- MMA issuers (two threads)
      const bool second = warp == FW_MMA2;
      const uint32_t idesc = make_idesc(128, FW_FIB);
      uint32_t sc = 0, it = 0;
      bool issued = false, stop = false;
      for (long long tile = blockIdx.x; tile < total_tiles && !stop; tile += gridDim.x) {
        while (true) {
          FwSlot S;
          const uint32_t b = sc & 1u, u = sc >> 1;
          if (!fw_get(slots, slot_full, slot_empty, sc, S, wl, -1)) ws_fail(abort_s, status);
          if (u >= 1 && !mbar_wait(smem_u32(&tmem_empty[b]), (u - 1) & 1u, wl)) ws_fail(abort_s, status);
          if (*abort_s) { stop = true; break; }
          asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
          const uint32_t acc0 = tmem + 128u * b;
          for (int c = 0; c < S.nsub; ++c, ++it) {
            const uint32_t st = it % NST, use = it / NST;
            if (!mbar_wait(smem_u32(&full_x[st]), use & 1u, wl) || !mbar_wait(smem_u32(&full_e[st]), use & 1u, wl))
              ws_fail(abort_s, status);
            if (*abort_s) { stop = true; break; }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t xa = smem_u32(smem + st * STAGE);
            const uint32_t xlo = desc_lo(xa), elo = desc_lo(xa + XBYTES);
            if (second) {
              if (c == 0)
                issue_chunk<KS, true, true, FW_FIB, FW_XSL, FW_MASK2>(acc0, xlo, elo, idesc);
              else
                issue_chunk<KS, false, true, FW_FIB, FW_XSL, FW_MASK2>(acc0, xlo, elo, idesc);
            } else {
              if (c == 0)
                issue_chunk<KS, true, true, FW_FIB, FW_XSL, FW_MASK1>(acc0, xlo, elo, idesc);
              else
                issue_chunk<KS, false, true, FW_FIB, FW_XSL, FW_MASK1>(acc0, xlo, elo, idesc);
            }
            issued = true;
            mma_commit(smem_u32(&empty[st]));
          }
          if (stop) break;
          mma_commit(smem_u32(&tmem_full[b]));
          ++sc;
          if (S.flags & FW_END) break;
        }
      }
      // every MMA this thread issued is complete before TMEM is released
      mma_commit(smem_u32(done));
      if (issued) mbar_wait(smem_u32(done), 0u, CLEANUP_WAIT_NS);
    }
  } else if (warp == FW_SCHED && lane == 0) {
    // ------------------------------------------------------------ scheduler + raw X copies
    int job = 0;
    uint32_t sc = 0;
    long long r_last = -1;   // step of the latest raw X copy
    bool stop = false;
    for (long long tile = blockIdx.x; tile < total_tiles && !stop; tile += gridDim.x) {
      int lo = job, hi = P.njobs - 1;   // tiles of this CTA increase: the job index only moves forward
      while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (P.jobs[mid].tile_begin <= tile) lo = mid; else hi = mid - 1;
      }
      job = lo;
      const FJob& J = P.jobs[job];
      const long long f0 = (tile - J.tile_begin) * FW_FIB;
      const int nfib = (int)min((long long)FW_FIB, J.B0 - f0);
      for (int nd = 0; nd < J.nnodes; ++nd, ++sc) {
        const uint32_t q = sc % FW_SLOTS;
        if (sc >= FW_SLOTS && !mbar_wait(smem_u32(&slot_empty[q]), ((sc / FW_SLOTS) - 1) & 1u, wl))
          ws_fail(abort_s, status);
        if (*abort_s) { stop = true; break; }
        if (!PK_CK(P.nodes + J.node0 + nd, sizeof(FNode), chk::SITE_TABLE)) {
          ws_fail(abort_s, status);   // no node to run: the CTA stops like on an expired wait
          stop = true;
          break;
        }
        const FNode& N = P.nodes[J.node0 + nd];
        FwSlot& S = slots[q];
        S.xsrc = N.in + f0 * J.n;
        S.ebase = N.eslices;
        S.rexp = N.rexp;
        S.dout = nullptr;
        int flags = 0;
        if (N.direct) {
          flags |= FW_DIRECT;
          double* o = reinterpret_cast<double*>(fw_tab(P, N.out_tab, N.tab_off_out, N.out));
          S.dout = o + f0 * J.n;
        } else {
          if (N.k == 0) flags |= FW_FIRST;
          if (N.k == J.m - 1) flags |= FW_LAST;
#pragma unroll
          for (int j = 0; j < P_; ++j) {
            const float2* cp = J.coef + j * J.m + N.k;
            S.c[j] = PK_CK(cp, sizeof(float2), chk::SITE_FUSED_READ) ? *cp : make_float2(0.f, 0.f);
          }
        }
        if (nd == J.nnodes - 1) flags |= FW_END;
        S.flags = flags;
        S.f0 = f0;
        S.n = J.n;
        S.nsub = (J.n + KC - 1) / KC;
        S.nfib = nfib;
        S.xbytes = (unsigned)(nfib * J.n * 8);
        const int eX = PK_CK(N.in_exp, sizeof(int), chk::SITE_FUSED_READ) ? *N.in_exp : -1000;
        S.eX = eX < -600 ? 0 : eX;  // all-zero input
        S.job = job;
        mbar_arrive(smem_u32(&slot_full[q]));
        // the raw X of this step: one bulk copy into the ring of raw buffers
        const uint32_t r = sc % NRAW, u = sc / NRAW;
        if (u >= 1 && !mbar_wait(smem_u32(&raw_empty[r]), (u - 1) & 1u, wl)) ws_fail(abort_s, status);
        if (*abort_s) { stop = true; break; }
        mbar_expect_tx(smem_u32(&raw_full[r]), S.xbytes);
        bulk_copy_g2s(smem_u32(rawbuf + r * FW_RAW), PK_CK_SRC(S.xsrc, S.xbytes, chk::SITE_FUSED_XCOPY), S.xbytes,
                      smem_u32(&raw_full[r]));
        r_last = sc;
      }
    }
    if (*abort_s) {
      // raw copies still in flight land before the CTA's shared memory is released
      for (long long k = r_last; k >= 0 && k >= r_last - (NRAW - 1); --k)
        mbar_wait(smem_u32(&raw_full[k % NRAW]), (uint32_t)(k / NRAW) & 1u, CLEANUP_WAIT_NS);
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512));
}

template <int KS, int P_>
int launch_fw(const FPass& P, int grid, int* status, cudaStream_t st) {
  const size_t sm = fw_smem_bytes(KS);
  auto kern = fused_weights_kernel<KS, P_>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) {
    set_error(std::string("fused mode kernel smem attribute: ") + cudaGetErrorString(e));
    return PHIKRON_ECUDA;
  }
  launch_begin(KC_TC_MODE, st);
  kern<<<grid, FW_THREADS, sm, st>>>(P, status);
  launch_end(st);
  PK_CHECK_LAUNCH();
  return PHIKRON_OK;
}

template <int KS>
int launch_fw_p(const FPass& P, int p, int grid, int* status, cudaStream_t st) {
  switch (p) {
    case 1: return launch_fw<KS, 1>(P, grid, status, st);
    case 2: return launch_fw<KS, 2>(P, grid, status, st);
    case 3: return launch_fw<KS, 3>(P, grid, status, st);
    case 4: return launch_fw<KS, 4>(P, grid, status, st);
    default: break;
  }
  set_error("fused mode pass: p must be in 1..4");
  return PHIKRON_EINVAL;
}

}  // namespace
}  // namespace tc

namespace fused {

int launch(const FPass& P, int slices, int p, int grid, int* status, cudaStream_t st) {
  if (P.njobs <= 0 || P.total_tiles <= 0) return PHIKRON_OK;
  grid = (int)std::min<long long>(P.total_tiles, grid);
  switch (slices) {
    case 3: return tc::launch_fw_p<3>(P, p, grid, status, st);
    case 4: return tc::launch_fw_p<4>(P, p, grid, status, st);
    case 5: return tc::launch_fw_p<5>(P, p, grid, status, st);
    case 6: return tc::launch_fw_p<6>(P, p, grid, status, st);
    default: break;
  }
  set_error("fused mode pass: unsupported slice count");
  return PHIKRON_EINVAL;
}

}  // namespace fused
}  // namespace phikron
