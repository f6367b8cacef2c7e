// Device building blocks shared by the tensor-core mode kernels (tc_mode.cu, fused.cu):
// tcgen05 shared-memory descriptors and MMA issue, mbarrier waits (every one bounded by a
// wall-clock limit), TMEM loads, bulk copies, the digit cutting of float64 and float-float
// operands into exact BF16 slices, and float-float (compensated FP32) arithmetic.  Internal
// to the library; each translation unit that includes it gets its own copies.
#pragma once

#include <cstdint>

#include "ff_arith.cuh"
#include "mixed.h"

namespace phikron {
namespace tc {
namespace {

constexpr int KC = 32;                    // K elements per chunk
constexpr int SLICE_BYTES = 128 * KC * 2; // one slice of a 128-row chunk: 8 KB

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ uint64_t make_desc(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFF);
  if (kSwizzle64) {
    // 64-byte swizzle, K-major: SBO = 512 B (next 8-row atom); LBO unused (one atom spans K)
    d |= (uint64_t)1 << 16;
    d |= (uint64_t)((512u >> 4) & 0x3FFF) << 32;
    d |= (uint64_t)4 << 61;  // layout type: 64-byte swizzle
  } else {
    // no swizzle, K-major: LBO = 128 B (next core matrix along K), SBO = 512 B (next 8 rows)
    d |= (uint64_t)((128u >> 4) & 0x3FFF) << 16;
    d |= (uint64_t)((512u >> 4) & 0x3FFF) << 32;
  }
  d |= (uint64_t)1 << 46;  // descriptor version for sm_100-class tensor cores
  return d;
}

// byte offset of the 16-element K-step ks (0 or 1) inside a slice
constexpr uint32_t KSTEP_BYTES = kSwizzle64 ? 32u : 256u;

__device__ __forceinline__ uint32_t make_idesc(int M, int N) {
  // kind::f16: D = F32 (bits 4-5 = 1), A = B = BF16 (bits 7-9, 10-12 = 1), both K-major,
  // N >> 3 at bits 17-22, M >> 4 at bits 24-28.
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t tmem_d, uint64_t ad, uint64_t bd, uint32_t idesc,
                                         uint32_t accumulate) {
  asm volatile(
      "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
      "l"(ad), "l"(bd), "r"(idesc), "r"(accumulate));
}

// The descriptor's high word (SBO, version, layout type) is the same for every operand of these
// kernels; only the start-address field of the low word moves.  Shared-memory addresses stay
// below 256 KB, so an offset added to the low word never carries out of that 14-bit field.
constexpr uint32_t DESC_HI = kSwizzle64 ? ((512u >> 4) | (1u << 14) | (4u << 29)) : ((512u >> 4) | (1u << 14));
constexpr uint32_t DESC_LBO = kSwizzle64 ? (1u << 16) : ((128u >> 4) << 16);

__device__ __forceinline__ uint32_t desc_lo(uint32_t saddr) { return ((saddr >> 4) & 0x3FFFu) | DESC_LBO; }

// one MMA from two descriptor low words; `accumulate` is a compile-time constant at every call
// site after unrolling, so the issue loop carries no per-MMA select or 64-bit arithmetic
__device__ __forceinline__ void mma_bf16_lo(uint32_t tmem_d, uint32_t a_lo, uint32_t b_lo, uint32_t idesc,
                                            uint32_t accumulate) {
  asm volatile(
      "{\n.reg .b64 da, db;\n.reg .b32 hi;\n.reg .pred p;\n"
      "mov.b32 hi, %4;\nmov.b64 da, {%1, hi};\nmov.b64 db, {%2, hi};\n"
      "setp.ne.b32 p, %5, 0;\n"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], da, db, %3, p;\n}\n" ::"r"(tmem_d),
      "r"(a_lo), "r"(b_lo), "r"(idesc), "n"(DESC_HI), "r"(accumulate));
}

// The slice-pair MMAs of one 32-wide K chunk: pairs (s, t) with s + t <= KS + 1, two K-steps
// each, level s + t - 2 into accumulator min(level, 3) (ACC_COLS columns apart).  FIRST: the
// tile's first chunk, where each accumulator's first MMA overwrites it -- the first touch of
// accumulator a is pair (1, a + 1) at K-step 0.  E_IS_A puts E in the A operand (M = output
// rows) and the input slices in B; otherwise the input slices are A.  XSLICE: bytes between
// input slices.  MASK: the accumulators this call issues for (bit a = accumulator a).
template <int KS, bool FIRST, bool E_IS_A, int ACC_COLS, int XSLICE, int MASK = 15>
__device__ __forceinline__ void issue_chunk(uint32_t acc0, uint32_t xlo, uint32_t elo, uint32_t idesc) {
#pragma unroll
  for (int s = 1; s <= KS; ++s) {
#pragma unroll
    for (int t = 1; t <= KS; ++t) {
      if (s + t > KS + 1) continue;
      const int L = s + t - 2;
      const int a = L < 3 ? L : 3;
      if (!((MASK >> a) & 1)) continue;  // accumulator issued by the other MMA thread
#pragma unroll
      for (int ks = 0; ks < 2; ++ks) {
        const uint32_t xd = xlo + (uint32_t)((((t - 1) * XSLICE) + ks * KSTEP_BYTES) >> 4);
        const uint32_t ed = elo + (uint32_t)((((s - 1) * SLICE_BYTES) + ks * KSTEP_BYTES) >> 4);
        const uint32_t accumulate = (FIRST && s == 1 && ks == 0 && t <= 4) ? 0u : 1u;
        if (E_IS_A)
          mma_bf16_lo(acc0 + (uint32_t)(a * ACC_COLS), ed, xd, idesc, accumulate);
        else
          mma_bf16_lo(acc0 + (uint32_t)(a * ACC_COLS), xd, ed, idesc, accumulate);
      }
    }
  }
}

__device__ __forceinline__ void mma_commit(uint32_t mbar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar)
               : "memory");
}

__device__ __forceinline__ bool mbar_try(uint32_t mbar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(mbar), "r"(parity)
      : "memory");
  return ok != 0;
}

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// bounded wait (wall clock, limit_ns nanoseconds); returns false on expiry
__device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t parity, unsigned long long limit_ns) {
  if (mbar_try(mbar, parity)) return true;
  const unsigned long long t0 = global_ns();
  while (true) {
    if (mbar_try(mbar, parity)) return true;
    if (global_ns() - t0 > limit_ns) return false;
  }
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float* v) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
#pragma unroll
  for (int j = 0; j < 16; ++j) v[j] = __uint_as_float(r[j]);
}

__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// ---------------------------------------------------------------- digit cutting (integer ops)
// F = |x| * 2^{64 - eX} as a 64-bit fixed-point integer (|x| < 2^eX); the digits d_t are the
// bytes of F, most significant first.

// float64 input; eb = 1011 + eX
__device__ __forceinline__ uint64_t fixed_f64(double x, int eb, uint32_t& sgn) {
  const uint64_t b = (uint64_t)__double_as_longlong(x);
  sgn = (uint32_t)(b >> 32) & 0x80000000u;
  const int ex = (int)((b >> 52) & 0x7FF);
  const uint64_t m = (b & 0xFFFFFFFFFFFFFull) | (ex ? (1ull << 52) : 0ull);
  const int sh = ex - eb;  // <= 11
  return sh >= 0 ? (m << sh) : (m >> min(-sh, 63));
}

// round to nearest at digit KS, saturating on carry-out
template <int KS>
__device__ __forceinline__ uint64_t round_digits(uint64_t F) {
  const uint64_t G = F + (1ull << (63 - 8 * KS));
  return G < F ? ~0ull : G;
}

// The signed slice value +-d_t 2^{-8t} as an FP32 whose upper 16 bits are its (exact) BF16:
// one byte permute puts d_t under the exponent of 2^23 (with the element's sign), one add
// removes 2^23, one multiply applies 2^{-8t}.
template <int T>
__device__ __forceinline__ float digit_value(uint32_t w1, uint32_t w0, uint32_t magic, float unmagic) {
  constexpr uint32_t byte = (T <= 4) ? (4 - T) : (8 - T);
  const uint32_t w = (T <= 4) ? w1 : w0;
  const float f = __uint_as_float(__byte_perm(w, magic, byte | 0x7540u)) + unmagic;
  return f * __uint_as_float((uint32_t)(127 - 8 * T) << 23);
}

template <int KS, int T = 1>
__device__ __forceinline__ void cut_pair(uint64_t F0, uint32_t s0, uint64_t F1, uint32_t s1, uint32_t* out) {
  if constexpr (T <= KS) {
    const float a = digit_value<T>((uint32_t)(F0 >> 32), (uint32_t)F0, 0x4B000000u | s0, s0 ? 8388608.0f : -8388608.0f);
    const float b = digit_value<T>((uint32_t)(F1 >> 32), (uint32_t)F1, 0x4B000000u | s1, s1 ? 8388608.0f : -8388608.0f);
    out[T - 1] = __byte_perm(__float_as_uint(a), __float_as_uint(b), 0x7632u);  // (bf16(b) << 16) | bf16(a)
    cut_pair<KS, T + 1>(F0, s0, F1, s1, out);
  }
}

// Float-float input: the slices come from FP32 arithmetic alone.  With X = (hi + lo) 2^{-eX}
// (|X| < 1), slice t is X's running remainder rounded to a multiple of 2^{-8t} by adding and
// subtracting 1.5 * 2^{23-8t} (round to nearest in FP32); the remainder update is exact.  lo
// joins the remainder before slice min(4, KS), where the FP32 add rounds at <= 2^-49.  Every
// slice is an integer of at most 256 times 2^{-8t}, exact in BF16, like the integer digits.
template <int KS>
__device__ __forceinline__ void cut_ff_float(float hi, float lo, float sc, float* v) {
  float r = __fmul_rn(hi, sc);
  const float l = __fmul_rn(lo, sc);
  constexpr int FOLD = KS < 4 ? KS : 4;
#pragma unroll
  for (int t = 1; t <= KS; ++t) {
    if (t == FOLD) r = __fadd_rn(r, l);
    const float M = __uint_as_float((uint32_t)(127 + 23 - 8 * t) << 23) * 1.5f;
    const float q = __fsub_rn(__fadd_rn(r, M), M);
    v[t - 1] = q;
    r = __fsub_rn(r, q);
  }
}

// Packed FP32x2 arithmetic (one instruction for two lanes, each lane IEEE round-to-nearest
// like the scalar FADD/FMUL): the digit cutting and the accumulator combination work on pairs
// of independent elements, so the producer and epilogue warps issue about half the FP32
// instructions.  a - b is one fused multiply-add, b * (-1) + a, rounded once like FSUB.
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 sub2(float2 a, float2 b) { return __ffma2_rn(b, make_float2(-1.0f, -1.0f), a); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }

// cut_ff_float for two elements at once (lane x: element (hi.x, lo.x), lane y: (hi.y, lo.y));
// bitwise the scalar results
template <int KS>
__device__ __forceinline__ void cut_ff_float2(float2 hi, float2 lo, float sc, float2* v) {
  const float2 sc2 = make_float2(sc, sc);
  float2 r = mul2(hi, sc2);
  const float2 l = mul2(lo, sc2);
  constexpr int FOLD = KS < 4 ? KS : 4;
#pragma unroll
  for (int t = 1; t <= KS; ++t) {
    if (t == FOLD) r = add2(r, l);
    const float Ms = __uint_as_float((uint32_t)(127 + 23 - 8 * t) << 23) * 1.5f;
    const float2 M = make_float2(Ms, Ms);
    const float2 q = sub2(add2(r, M), M);
    v[t - 1] = q;
    r = sub2(r, q);
  }
}

// two FP32 values exactly representable in BF16 -> (bf16(b) << 16) | bf16(a)
__device__ __forceinline__ uint32_t pack_bf16x2(float a, float b) {
  uint32_t d;
  asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(d) : "f"(b), "f"(a));
  return d;
}

// 2^e for e in [-149, 127] (subnormal scales included)
__device__ __forceinline__ float pow2f_full(int e) {
  e = e < -149 ? -149 : (e > 127 ? 127 : e);
  return e >= -126 ? __uint_as_float((uint32_t)(e + 127) << 23) : __uint_as_float(1u << (e + 149));
}

// ---------------------------------------------------------------- float-float helpers
using ff::two_sum;
using ff::fast_two_sum;
__device__ __forceinline__ double ff_to_f64(float hi, float lo) { return ff::to_f64(hi, lo); }

__device__ __forceinline__ float pow2f(int e) {
  e = e < -126 ? -126 : (e > 127 ? 127 : e);
  return __uint_as_float((uint32_t)(e + 127) << 23);
}



// ---------------------------------------------------------------- the kernel

__device__ __forceinline__ void bulk_copy_g2s(uint32_t dst, const void* src, uint32_t bytes, uint32_t mbar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
      "l"(src), "r"(bytes), "r"(mbar)
      : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t mbar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(mbar), "r"(bytes) : "memory");
}


__device__ __forceinline__ void mbar_arrive(uint32_t mbar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(mbar) : "memory");
}

// all 128 epilogue threads (named barrier 1): true if any of them passes true
__device__ __forceinline__ bool epi_vote_any(bool pred) {
  uint32_t r;
  asm volatile(
      "{\n.reg .pred p, q;\nsetp.ne.u32 q, %1, 0;\nbar.red.or.pred p, 1, 128, q;\nselp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(r)
      : "r"((uint32_t)pred)
      : "memory");
  return r != 0;
}

// all 256 epilogue threads (named barrier 1): true if any of them passes true
__device__ __forceinline__ bool epi_vote_any256(bool pred) {
  uint32_t r;
  asm volatile(
      "{\n.reg .pred p, q;\nsetp.ne.u32 q, %1, 0;\nbar.red.or.pred p, 1, 256, q;\nselp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(r)
      : "r"((uint32_t)pred)
      : "memory");
  return r != 0;
}

// one arrival of count 32 for the whole (converged) warp instead of 32 arrivals on one word
__device__ __forceinline__ void mbar_arrive_warp(uint32_t mbar, int lane) {
  __syncwarp();
  if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0], 32;" ::"r"(mbar) : "memory");
}

__device__ __forceinline__ void ws_fail(volatile int* abort_s, int* status) {
  *abort_s = 1;
  atomicExch(status, PHIKRON_ETIMEOUT);
}

// hi + lo ~ d2 + d3 + d4 + d5 (the level accumulators, largest first).  With at most 5 digit
// slices the products are exact to ~2^-40 of the vector's scale, so only d2 + d3 needs an
// error-free sum: d4 (~2^-16 of it) and d5 join the error term in plain FP32, which rounds at
// ~2^-40.  Six slices (~2^-48) keep error-free sums at every step.
template <int KS>
__device__ __forceinline__ void ff_combine(float d2, float d3, float d4, float d5, float& hi, float& lo) {
  if (KS <= 5) {
    float eh;
    two_sum(d2, d3, hi, eh);
    lo = eh + (d4 + d5);
  } else {
    float t45, e45, u, eu, eh;
    two_sum(d4, d5, t45, e45);
    two_sum(d3, t45, u, eu);
    two_sum(d2, u, hi, eh);
    lo = eh + (eu + e45);
  }
  fast_two_sum(hi, lo, hi, lo);
}

// ff_combine for two columns at once (packed FP32x2; bitwise the scalar results)
template <int KS>
__device__ __forceinline__ void ff_combine2(float2 d2, float2 d3, float2 d4, float2 d5, float2& hi, float2& lo) {
  float2 h, l;
  if (KS <= 5) {
    h = add2(d2, d3);
    const float2 bb = sub2(h, d2);
    const float2 eh = add2(sub2(d2, sub2(h, bb)), sub2(d3, bb));
    l = add2(eh, add2(d4, d5));
  } else {
    const float2 t45 = add2(d4, d5);
    const float2 b45 = sub2(t45, d4);
    const float2 e45 = add2(sub2(d4, sub2(t45, b45)), sub2(d5, b45));
    const float2 u = add2(d3, t45);
    const float2 bu = sub2(u, d3);
    const float2 eu = add2(sub2(d3, sub2(u, bu)), sub2(t45, bu));
    h = add2(d2, u);
    const float2 bh = sub2(h, d2);
    const float2 eh = add2(sub2(d2, sub2(h, bh)), sub2(u, bh));
    l = add2(eh, add2(eu, e45));
  }
  hi = add2(h, l);
  lo = sub2(l, sub2(hi, h));
}

// A bounded wait that follows an expired one (waiting for the CTA's own bulk copies and MMAs
// before its shared memory and TMEM are released): these complete without any other CTA, so
// the limit is long.
constexpr unsigned long long CLEANUP_WAIT_NS = 10000000000ull;

}  // namespace
}  // namespace tc
}  // namespace phikron
