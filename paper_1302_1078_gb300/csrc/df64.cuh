// Double-precision multiply-accumulate on the FP32 pipe ("dual-pipe FP64").
//
// GB300's FP64 pipe retires 2 fused multiply-adds per clock per SM, against
// 128 on the FP32 pipe.  FP64 SpMM (and SpMV near the HBM roof) is therefore
// bound by the FP64 pipe.  A share of the products can be computed on the
// FP32 pipe instead, with enough precision for the library's accuracy bound
// (|y - y_exact| <= 1e-12 * sum |a x| per entry):
//
//   * split_f64: a double d becomes hi + lo, two floats, using integer
//     operations only (no FP64 conversion instruction):
//       - hi is d truncated to 24 significant bits;
//       - lo is the next 23 bits, made exact by subtracting a power of two
//         that shares lo's exponent (one FADD);
//       - |d - (hi + lo)| < 2^-46 |d|;
//       - valid when the exponent of d lies within [-38, 38], or when d is
//         zero; other operands are reported, so the caller can use the native
//         pipe for them.  The range keeps a product of two valid operands
//         within [2^-76, 2^78), so the product, its exact low part (about
//         2^-48 of it) and a sum of 48 such products are all normal floats.
//   * product: a*x = ah*xh + (ah*xl + al*xh) + O(2^-46 |a x|).  ah*xh is
//     split exactly into p + e1 with one FFMA (24 x 24 bits fit in 48); the
//     cross terms are added to e1 with two FFMAs.
//   * accumulation: Knuth's TwoSum keeps the running float sum s exact up to
//     a compensation float c, which also collects the low-order product
//     terms; a second TwoSum renormalises the pair after every term, which
//     keeps |c| below half an ulp of s, so each term adds at most about 2^-48 of the running
//     magnitude.  Over n terms the error stays below roughly
//     (n 2^-48 + 2^-44) sum |a x|: 2.9e-13 for n = 64.  Callers flush the
//     pair into a native double at least every 64 terms.
//
// Each emulated term is about 35 integer/FP32 instructions, so a mix of
// native and emulated terms keeps both pipes busy.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace gbs {

// Split d into hi + lo; returns false if d needs the native pipe (|d| outside
// [2^-38, 2^39) and not zero, or not finite).
__device__ __forceinline__ bool split_f64(double d, float& hi, float& lo) {
  const unsigned long long bits = static_cast<unsigned long long>(__double_as_longlong(d));
  const unsigned H = static_cast<unsigned>(bits >> 32), L = static_cast<unsigned>(bits);
  const unsigned e = (H >> 20) & 0x7FFu;
  const bool zero = ((H & 0x7FFFFFFFu) | L) == 0u;
  const bool ok = (e - (1023u - 38u)) <= 76u;  // unsigned wrap: e in [985, 1061]
  // hi: rebias the exponent in place (1023 -> 127), then shift mantissa and exponent up by 3
  const unsigned hb = H - ((1023u - 127u) << 20);
  unsigned fhi = __funnelshift_l(L, hb, 3);
  fhi = (fhi & 0x7FFFFFFFu) | (H & 0x80000000u);
  // lo: bits 28..6 of L under hi's exponent - 23, minus that power of two
  const unsigned elo = (fhi & 0xFF800000u) - (23u << 23);
  const unsigned flo = elo | ((L >> 6) & 0x007FFFFFu);
  const float h = __uint_as_float(fhi);
  const float l = __fsub_rn(__uint_as_float(flo), __uint_as_float(elo));
  hi = (ok && !zero) ? h : 0.0f;
  lo = (ok && !zero) ? l : 0.0f;
  return ok || zero;
}

// A float widened to double with integer operations only (exact; keeps the FP64 pipe, where
// GB300 also runs the conversion instruction, free for the products).  Handles zeros and
// subnormal floats; the accumulator never holds infinities or NaNs (operands are range-checked).
__device__ __forceinline__ double widen_f32(float f) {
  const unsigned u = __float_as_uint(f);
  const unsigned long long sign = static_cast<unsigned long long>(u & 0x80000000u) << 32;
  const unsigned e = (u >> 23) & 0xFFu;
  unsigned m = u & 0x007FFFFFu;
  unsigned long long bits;
  if (e != 0u) {
    bits = sign | (static_cast<unsigned long long>(e + (1023u - 127u)) << 52) |
           (static_cast<unsigned long long>(m) << 29);
  } else if (m == 0u) {
    bits = sign;
  } else {
    // subnormal: m * 2^-149 with the leading one of m at bit p
    const int p = 31 - __clz(m);
    m &= ~(1u << p);
    bits = sign | (static_cast<unsigned long long>(p + (1023 - 149)) << 52) |
           (static_cast<unsigned long long>(m) << (52 - p));
  }
  return __longlong_as_double(static_cast<long long>(bits));
}

// Float-float accumulator of products of split doubles.
struct DFAcc {
  float s = 0.0f, c = 0.0f;
  __device__ __forceinline__ void add(float ah, float al, float xh, float xl) {
    const float p = __fmul_rn(ah, xh);
    const float e1 = __fmaf_rn(ah, xh, -p);  // exact: ah*xh = p + e1
    float t = __fmaf_rn(ah, xl, e1);
    t = __fmaf_rn(al, xh, t);
    const float sn = __fadd_rn(s, p);
    const float bp = __fsub_rn(sn, s);
    const float err = __fadd_rn(__fsub_rn(s, __fsub_rn(sn, bp)), __fsub_rn(p, bp));
    const float cn = __fadd_rn(c, __fadd_rn(err, t));
    // renormalise the pair with a second TwoSum (exact whatever the magnitudes)
    const float s2 = __fadd_rn(sn, cn);
    const float b2 = __fsub_rn(s2, sn);
    c = __fadd_rn(__fsub_rn(sn, __fsub_rn(s2, b2)), __fsub_rn(cn, b2));
    s = s2;
  }
  // s + c is exact in double (at most 48 significant bits): one FP64 add
  __device__ __forceinline__ double value() const { return widen_f32(s) + widen_f32(c); }
  // add another accumulator's pair (the lanes of one row), renormalised like add()
  __device__ __forceinline__ void merge(const DFAcc& o) {
    const float sn = __fadd_rn(s, o.s);
    const float bp = __fsub_rn(sn, s);
    const float err = __fadd_rn(__fsub_rn(s, __fsub_rn(sn, bp)), __fsub_rn(o.s, bp));
    const float cn = __fadd_rn(c, __fadd_rn(err, o.c));
    const float s2 = __fadd_rn(sn, cn);
    const float b2 = __fsub_rn(s2, sn);
    c = __fadd_rn(__fsub_rn(sn, __fsub_rn(s2, b2)), __fsub_rn(cn, b2));
    s = s2;
  }
  __device__ __forceinline__ void reset() {
    s = 0.0f;
    c = 0.0f;
  }
};

}  // namespace gbs
