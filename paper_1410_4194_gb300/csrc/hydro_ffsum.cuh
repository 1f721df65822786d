// hydro_ffsum.cuh -- float-float sums of the mixed-precision update and their
// conversion to one double without an FP64 add (GB300 issues FP64 adds on its
// FP64 pipe at 1/64 of the float rate; the update of the mixed path is bound by
// that pipe).
#pragma once
#include "hydro_math.cuh"

namespace hydro {

// a + b as an unevaluated sum s + e of two floats, exactly (Knuth's TwoSum,
// round-to-nearest without overflow)
__device__ __forceinline__ float two_sum(float a, float b, float& e) {
  const float s = a + b;
  const float bb = s - a;
  e = (a - (s - bb)) + (b - bb);
  return s;
}

// hi + lo of a float-float pair as one double, in integer arithmetic, in place
// of f2d(hi) + f2d(lo).  The pair is first renormalised by TwoSum (s + t =
// hi + lo exactly, |t| <= ulp(s)/2).  s's 24-bit significand fills the top of
// the double's 53; t's significand (a subnormal t's without the leading one)
// is added or subtracted at its place below, with one guard bit: since
// |t| <= 2^(e_s - 24), it reaches at most 5 bits into the 29 zero bits that
// follow s's, so a sum never carries out, and a difference only borrows below
// 2^52 when s is a power of two, where the guard bit becomes the last bit of
// the result one binade lower.  Bits of t below the result's last place are
// dropped: the result is within one ulp of the exact sum (an FP64 add would be
// within half an ulp).  A zero or subnormal s counts as zero, as in f2d; a
// non-finite s converts as it is.
__device__ __forceinline__ double ff_to_double(float hi, float lo) {
  float t;
  const float s = two_sum(hi, lo, t);
  const unsigned sb = __float_as_uint(s), tb = __float_as_uint(t);
  const unsigned es = sb >> 23 & 0xffu, et = tb >> 23 & 0xffu;
  if (es == 0xffu || es == 0u || (tb & 0x7fffffffu) == 0u) return f2d(s);
  const unsigned long long mt = et ? (1ull << 23) | (tb & 0x7fffffu) : (tb & 0x7fffffu);
  // place of t's last bit above the guard bit under the double's last place
  const int k = (int)(et ? et : 1u) - (int)es + 30;
  const unsigned long long sig_s = ((1ull << 52) | ((unsigned long long)(sb & 0x7fffffu) << 29)) << 1;
  const unsigned long long sig_t = k >= 0 ? mt << k : (k > -24 ? mt >> -k : 0ull);
  unsigned long long sig = ((sb ^ tb) & 0x80000000u) ? sig_s - sig_t : sig_s + sig_t;
  unsigned long long e = es + 896u;  // double exponent field of s
  if (sig >= (1ull << 53))
    sig >>= 1;  // drop the guard bit
  else
    e -= 1;  // s a power of two less t: the guard bit is the last place
  const unsigned long long sign = (unsigned long long)(sb & 0x80000000u) << 32;
  return __longlong_as_double((long long)(sign | e << 52 | (sig & ((1ull << 52) - 1))));
}

}  // namespace hydro
