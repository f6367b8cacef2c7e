// Float-float (compensated FP32) arithmetic shared by the mixed path's kernels: a value is an
// unevaluated sum hi + lo of two FP32 numbers with |lo| <= ulp(hi)/2 (~48-bit significand).
// Every product and sum is written with round-to-nearest intrinsics, so the compiler cannot
// contract a multiply and a later add into one fused operation: each kernel that forms the same
// float-float expression gets the same bits (the fused node-weight epilogue relies on this to
// reproduce the separate weighted-sum kernel exactly).  Internal to the library.
#pragma once

#include <cstdint>

namespace phikron {
namespace ff {

// s + e = a + b exactly (Knuth's two-sum)
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// s + e = a + b exactly when |a| >= |b| (or a == 0)
__device__ __forceinline__ void fast_two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  e = __fsub_rn(b, __fsub_rn(s, a));
}

// acc += c * t in float-float: the exact product c.x t.x (FMA residual) plus the cross terms,
// one two-sum with acc.x, the low parts added, renormalised
__device__ __forceinline__ void fma_ff(float2& acc, float2 c, float2 t) {
  const float p = __fmul_rn(c.x, t.x);
  float pe = __fmaf_rn(c.x, t.x, -p);
  pe = __fmaf_rn(c.x, t.y, pe);
  pe = __fmaf_rn(c.y, t.x, pe);
  float s, e;
  two_sum(acc.x, p, s, e);
  e = __fadd_rn(e, __fadd_rn(acc.y, pe));
  fast_two_sum(s, e, acc.x, acc.y);
}

// acc += t in float-float
__device__ __forceinline__ void add_ff(float2& acc, float2 t) {
  float s, e;
  two_sum(acc.x, t.x, s, e);
  e = __fadd_rn(e, __fadd_rn(acc.y, t.y));
  fast_two_sum(s, e, acc.x, acc.y);
}

// fma_ff on two independent accumulators with the same coefficient (packed FP32x2: one
// instruction per pair, each lane rounded like the scalar instruction, so bitwise fma_ff)
__device__ __forceinline__ void fma_ff2(float2& acc_hi, float2& acc_lo, float2 c, float2 t_hi, float2 t_lo) {
  const float2 cx = make_float2(c.x, c.x), cy = make_float2(c.y, c.y);
  const float2 p = __fmul2_rn(cx, t_hi);
  const float2 np = make_float2(-p.x, -p.y);
  float2 pe = __ffma2_rn(cx, t_hi, np);
  pe = __ffma2_rn(cx, t_lo, pe);
  pe = __ffma2_rn(cy, t_hi, pe);
  const float2 m1 = make_float2(-1.0f, -1.0f);
  // two_sum(acc_hi, p)
  const float2 s = __fadd2_rn(acc_hi, p);
  const float2 bb = __ffma2_rn(acc_hi, m1, s);                       // s - acc_hi
  const float2 e0 = __fadd2_rn(__ffma2_rn(__ffma2_rn(bb, m1, s), m1, acc_hi),  // acc_hi - (s - bb)
                               __ffma2_rn(bb, m1, p));                           // p - bb
  const float2 e = __fadd2_rn(e0, __fadd2_rn(acc_lo, pe));
  // fast_two_sum(s, e)
  acc_hi = __fadd2_rn(s, e);
  acc_lo = __ffma2_rn(__ffma2_rn(s, m1, acc_hi), m1, e);             // e - (hi - s)
}

// float-float -> float64 by integer assembly of the 53-bit significand (no float64 arithmetic);
// requires |lo| <= ulp(hi)/2
__device__ __forceinline__ double to_f64(float hi, float lo) {
  const uint32_t bh = __float_as_uint(hi);
  const int eh = (int)((bh >> 23) & 0xFF);
  if (eh == 0) return 0.0;
  uint64_t M = (uint64_t)((bh & 0x7FFFFFu) | 0x800000u) << 29;  // 53-bit significand of hi
  int E = eh - 127 + 1023;
  const uint32_t bl = __float_as_uint(lo);
  const int el = (int)((bl >> 23) & 0xFF);
  if (el != 0) {
    const uint64_t ml = (uint64_t)((bl & 0x7FFFFFu) | 0x800000u);
    const int sh = el - eh + 29;  // lo in units of hi's 53-bit ulp
    uint64_t L;
    if (sh >= 0)
      L = ml << sh;
    else if (sh > -40)
      L = (ml + (1ull << (-sh - 1))) >> (-sh);
    else
      L = 0;
    if (((bh ^ bl) >> 31) == 0) {
      M += L;
      if (M >> 53) {  // carry (cannot happen for normalised pairs; kept for safety)
        M >>= 1;
        ++E;
      }
    } else {
      M -= L;
      while (M && !(M >> 52)) {
        M <<= 1;
        --E;
      }
    }
  }
  const uint64_t bits = ((uint64_t)(bh >> 31) << 63) | ((uint64_t)E << 52) | (M & 0xFFFFFFFFFFFFFull);
  return __longlong_as_double((long long)bits);
}

}  // namespace ff
}  // namespace phikron
