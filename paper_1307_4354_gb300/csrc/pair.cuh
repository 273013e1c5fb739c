// FP32-pair ("double-single") arithmetic for the outer residual.  A value is
// hi + lo with two floats; products are split exactly with a fused
// multiply-add, sums of leading parts with Knuth's TwoSum (error-free), and
// the trailing parts are accumulated in plain float (Dekker 1971, Knuth
// TAOCP vol. 2 4.2.2).  About 48 significand bits on the FP32 pipe, whose
// rate on this part is 64 times that of FP64.  Packed forms work on two
// independent lanes per instruction (float2, Blackwell's paired FP32 ops).
#pragma once

#include <cstdint>

#include <cuda_runtime.h>

namespace cpm {

// float64 -> (hi, lo) with integer operations only: hi = d rounded to 24
// significand bits (the magnitude plus half a unit at bit 28, truncated: ties
// away from zero), lo = d - hi, an integer of at most 29 bits in units of
// d's last place, rounded to float.  |d| < 2^-126 gives (0, 0); below 2^-74
// lo is dropped (|lo| < 2^-98); |d| >= 2^128 gives hi = +-inf.
__device__ __forceinline__ float2 pair_split(double d) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(d);
  const unsigned long long mag = b & 0x7FFFFFFFFFFFFFFFull;
  const uint32_t sign = (uint32_t)(b >> 32) & 0x80000000u;
  const int e = (int)(mag >> 52);
  if (e < 1023 - 126) return make_float2(0.f, 0.f);
  const unsigned long long r = (mag + (1ull << 28)) & ~((1ull << 29) - 1ull);
  const int er = (int)(r >> 52);
  if (er > 1023 + 127) return make_float2(__int_as_float((int)(sign | 0x7F800000u)), 0.f);
  const uint32_t hb = sign | ((uint32_t)(er - 1023 + 127) << 23) | (uint32_t)((r >> 29) & 0x7FFFFFull);
  float lo = 0.f;
  if (e >= 949) {
    const int32_t rem = (int32_t)(long long)(mag - r);  // |rem| <= 2^28
    lo = __fmul_rn(__int2float_rn(rem), __int_as_float((e - 948) << 23));
    lo = __int_as_float(__float_as_int(lo) ^ (int)sign);
  }
  return make_float2(__int_as_float((int)hb), lo);
}

// float -> double by integer operations (exact for normal floats; zero and
// subnormal floats give zero, infinities and NaN stay so).
__device__ __forceinline__ double pair_f2d(float x) {
  const uint32_t b = (uint32_t)__float_as_int(x);
  const uint32_t ex = (b >> 23) & 0xFFu;
  const unsigned long long sign = (unsigned long long)(b & 0x80000000u) << 32;
  if (ex == 0) return __longlong_as_double((long long)sign);
  const unsigned long long e64 = ex == 0xFFu ? 0x7FFull : (unsigned long long)(ex + 896u);
  return __longlong_as_double((long long)(sign | (e64 << 52) | ((unsigned long long)(b & 0x7FFFFFu) << 29)));
}

// s + e == a + b exactly, s = fl(a + b).
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// s + e == a + b exactly for |a| >= |b|.
__device__ __forceinline__ void fast_two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  e = __fsub_rn(b, __fsub_rn(s, a));
}

// hi + lo as a double (one rounding).
__device__ __forceinline__ double pair_to_f64(float hi, float lo) { return pair_f2d(hi) + pair_f2d(lo); }

// (ah, al) (bh, bl) as a pair (leading product exact, the cross terms and the
// neglected al bl below 2^-46 of the product).
__device__ __forceinline__ void pair_mul(float ah, float al, float bh, float bl, float& ph, float& pl) {
  const float p = __fmul_rn(ah, bh);
  float e = __fmaf_rn(ah, bh, -p);
  e = __fmaf_rn(ah, bl, e);
  e = __fmaf_rn(al, bh, e);
  fast_two_sum(p, e, ph, pl);
}

// (ah, al) + (bh, bl) as a pair.
__device__ __forceinline__ void pair_add(float ah, float al, float bh, float bl, float& sh, float& sl) {
  float s, t;
  two_sum(ah, bh, s, t);
  fast_two_sum(s, __fadd_rn(t, __fadd_rn(al, bl)), sh, sl);
}

// ---- packed: two lanes per instruction.  There is no packed subtraction:
// a - b is formed as b * (-1) + a (one rounding, the same result).

// A pair per lane: (h.x, l.x) and (h.y, l.y).
struct Pair2 {
  float2 h, l;
};

// Broadcast or per-lane pair weight with its negated leading part.
struct PairW2 {
  float2 h, l, hn;
};
__device__ __forceinline__ PairW2 pw2(float2 w) {  // one pair (w.x, w.y) on both lanes
  return PairW2{make_float2(w.x, w.x), make_float2(w.y, w.y), make_float2(-w.x, -w.x)};
}
__device__ __forceinline__ PairW2 pw2(float2 w0, float2 w1) {  // lane 0: w0, lane 1: w1
  return PairW2{make_float2(w0.x, w1.x), make_float2(w0.y, w1.y), make_float2(-w0.x, -w1.x)};
}

// w x as a pair per lane (the first term of a sum).
__device__ __forceinline__ Pair2 pmul(const PairW2& w, float2 xh, float2 xl) {
  const float2 p = __fmul2_rn(w.h, xh);
  const float2 pn = __fmul2_rn(w.hn, xh);         // -p
  float2 e = __ffma2_rn(w.h, xh, pn);             // w.h xh - p, exact
  e = __ffma2_rn(w.h, xl, e);
  e = __ffma2_rn(w.l, xh, e);
  return Pair2{p, e};
}

// s += w x per lane: exact leading product, TwoSum into s.h, every error
// term into s.l (no renormalisation).
__device__ __forceinline__ void pmul_acc(const PairW2& w, float2 xh, float2 xl, Pair2& s) {
  const float2 m1 = make_float2(-1.f, -1.f);
  const float2 pn = __fmul2_rn(w.hn, xh);         // -p, p = fl(w.h xh)
  float2 e = __ffma2_rn(w.h, xh, pn);             // w.h xh - p, exact
  e = __ffma2_rn(w.h, xl, e);
  e = __ffma2_rn(w.l, xh, e);
  const float2 sn = __ffma2_rn(pn, m1, s.h);      // s.h + p
  const float2 bb = __ffma2_rn(s.h, m1, sn);      // sn - s.h
  float2 t1 = __ffma2_rn(bb, m1, sn);             // sn - bb
  t1 = __ffma2_rn(t1, m1, s.h);                   // s.h - (sn - bb)
  const float2 t2n = __fadd2_rn(pn, bb);          // -(p - bb)
  const float2 err = __ffma2_rn(t2n, m1, t1);     // TwoSum error
  s.l = __fadd2_rn(s.l, __fadd2_rn(err, e));
  s.h = sn;
}

}  // namespace cpm
