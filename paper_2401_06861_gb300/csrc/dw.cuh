// Double-word ("double-float") arithmetic on the FP32 pipe for FP64-accurate
// kernels: a value is an unevaluated sum h + l of two floats with
// |l| <= ulp(h) / 2.  GB300 issues FP32 at 64 times its FP64 rate, so
// products and sums of FP64 states run here instead of on the FP64 pipe.
//
// Methods (Joldes, Muller, Popescu, "Tight and rigorous error bounds for basic
// building blocks of double-word arithmetic", ACM TOMS 2017): the exact
// product of the high parts by one FMA (Dekker's TwoProduct with an FMA), the
// cross terms added in float, Knuth's TwoSum on the high parts and a final
// Fast2Sum.  Relative error of a product or sum: a few units of 2^-48.  The
// __f*_rn intrinsics keep the compiler from contracting or reassociating the
// error-free steps.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace nwq {

struct Dw {
  float h, l;
};

// Split a double into a float pair by integer operations (no FP64
// instruction): h = the top 24 significant bits, l = the next 23, rounded, so
// |x - h - l| <= 2^-47 |x|; magnitudes below 2^-103 become 0 and magnitudes of
// 2^128 or more become a signed infinity.
__device__ __forceinline__ Dw dw_split(double x) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const unsigned hi32 = (unsigned)(b >> 32), lo32 = (unsigned)b;
  const unsigned e = (hi32 >> 20) & 0x7ffu;
  // h: exponent rebiased 1023 -> 127, the top 23 fraction bits
  const unsigned hb = (hi32 & 0x80000000u) | (__funnelshift_l(lo32, hi32 - (896u << 20), 3) & 0x7fffffffu);
  // l: the other 29 fraction bits r (value r 2^(E-52)) as (2^(E-23) + q 2^(E-46)) - 2^(E-23),
  // q = r / 64 rounded (at most 2^23); exact by Sterbenz's lemma
  const unsigned mb = (hb & 0xff800000u) - (23u << 23);
  const unsigned q = ((lo32 & 0x1fffffffu) + 32u) >> 6;
  const float l = __fsub_rn(__int_as_float((int)(mb + q)), __int_as_float((int)mb));
  if (e < 920u) return Dw{0.f, 0.f};                                        // |x| < 2^-103
  if (e > 1150u) return Dw{__int_as_float((int)((hi32 & 0x80000000u) | 0x7f800000u)), 0.f};  // |x| >= 2^128
  return Dw{__int_as_float((int)hb), l};
}

__device__ __forceinline__ double dw_to_double(Dw a) { return (double)a.h + (double)a.l; }

// The exact product of two floats as a float pair (TwoProduct with an FMA).
__device__ __forceinline__ Dw two_prod(float a, float b) {
  const float p = __fmul_rn(a, b);
  return Dw{p, __fmaf_rn(a, b, -p)};
}

__device__ __forceinline__ Dw dw_neg(Dw a) { return Dw{-a.h, -a.l}; }

// The same value h + l with |l| <= ulp(h) / 2 (TwoSum, exact): the pairs a
// sweep writes leave their low parts unnormalised.
__device__ __forceinline__ Dw dw_norm(float h, float l) {
  const float s = __fadd_rn(h, l);
  const float v = __fsub_rn(s, h);
  return Dw{s, __fadd_rn(__fsub_rn(h, __fsub_rn(s, v)), __fsub_rn(l, v))};
}

__device__ __forceinline__ Dw dw_mul(Dw a, Dw b) {
  const float ph = __fmul_rn(a.h, b.h);
  float pl = __fmaf_rn(a.h, b.h, -ph);
  pl = __fmaf_rn(a.h, b.l, pl);
  pl = __fmaf_rn(a.l, b.h, pl);
  const float h = __fadd_rn(ph, pl);
  return Dw{h, __fsub_rn(pl, __fsub_rn(h, ph))};
}

__device__ __forceinline__ Dw dw_fma(Dw a, Dw b, Dw c) {  // a b + c
  const float ph = __fmul_rn(a.h, b.h);
  float pl = __fmaf_rn(a.h, b.h, -ph);
  pl = __fmaf_rn(a.h, b.l, pl);
  pl = __fmaf_rn(a.l, b.h, pl);
  const float s = __fadd_rn(ph, c.h);
  const float v = __fsub_rn(s, ph);
  float e = __fadd_rn(__fsub_rn(ph, __fsub_rn(s, v)), __fsub_rn(c.h, v));
  e = __fadd_rn(e, __fadd_rn(pl, c.l));
  const float h = __fadd_rn(s, e);
  return Dw{h, __fsub_rn(e, __fsub_rn(h, s))};
}

__device__ __forceinline__ Dw dw_add(Dw a, Dw b) {  // a + b (TwoSum of the high parts, then Fast2Sum)
  const float s = __fadd_rn(a.h, b.h);
  const float v = __fsub_rn(s, a.h);
  float e = __fadd_rn(__fsub_rn(a.h, __fsub_rn(s, v)), __fsub_rn(b.h, v));
  e = __fadd_rn(e, __fadd_rn(a.l, b.l));
  const float h = __fadd_rn(s, e);
  return Dw{h, __fsub_rn(e, __fsub_rn(h, s))};
}

// Compensated running sum (s, c) += v, the sign of v flipped when
// sg = 0x80000000: TwoSum on the running high part, its rounding error and
// the low parts collected in c.
__device__ __forceinline__ void dw_acc(float& s, float& c, Dw v, uint32_t sg) {
  const float vh = __int_as_float(__float_as_int(v.h) ^ (int)sg), vl = __int_as_float(__float_as_int(v.l) ^ (int)sg);
  const float t = __fadd_rn(s, vh);
  const float z = __fsub_rn(t, s);
  const float e = __fadd_rn(__fsub_rn(s, __fsub_rn(t, z)), __fsub_rn(vh, z));
  c = __fadd_rn(c, __fadd_rn(e, vl));
  s = t;
}

// (s, c) += a1 b1 + a2 b2 without renormalising the products: the exact high
// products (one FMA each for their rounding errors), the cross terms and the
// errors collected in float, TwoSum of the two high products, then TwoSum of
// that into the running sum s; every low-order part goes to c.
__device__ __forceinline__ void dw_acc_prod2(float& s, float& c, Dw a1, Dw b1, Dw a2, Dw b2) {
  const float p1 = __fmul_rn(a1.h, b1.h), p2 = __fmul_rn(a2.h, b2.h);
  float lo = __fadd_rn(__fmaf_rn(a1.h, b1.h, -p1), __fmaf_rn(a2.h, b2.h, -p2));
  lo = __fmaf_rn(a1.h, b1.l, lo);
  lo = __fmaf_rn(a1.l, b1.h, lo);
  lo = __fmaf_rn(a2.h, b2.l, lo);
  lo = __fmaf_rn(a2.l, b2.h, lo);
  const float h = __fadd_rn(p1, p2);
  const float v = __fsub_rn(h, p1);
  const float eh = __fadd_rn(__fsub_rn(p1, __fsub_rn(h, v)), __fsub_rn(p2, v));
  const float t = __fadd_rn(s, h);
  const float z = __fsub_rn(t, s);
  const float e = __fadd_rn(__fsub_rn(s, __fsub_rn(t, z)), __fsub_rn(h, z));
  c = __fadd_rn(c, __fadd_rn(e, __fadd_rn(eh, lo)));
  s = t;
}

}  // namespace nwq
