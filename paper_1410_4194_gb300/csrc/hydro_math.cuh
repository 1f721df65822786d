// hydro_math.cuh -- device arithmetic of one CTU step, templated on the
// arithmetic type T (double for the FP64 path, float for the reconstruction and
// Riemann stages of the mixed path).
//
//   * cons/prim conversion of the ideal gas (Sec. 2.1);
//   * the characteristic-limited slope of one cell (App. A.2: differences,
//     projection onto the characteristic fields, MC limiter, back-projection);
//   * PPMC face states with characteristic tracing (App. A.3);
//   * the exact Riemann solver with Newton iteration and ten-case sampling
//     (App. B.1).
//
// GB300 executes FP64 at two FMA per clock per SM, 1/64 of its FP32 rate, and a
// library pow() costs about a hundred FP64 FMA slots, a division or square root
// about ten.  The arithmetic below therefore evaluates the paper's formulas
// through algebraic identities that remove most of those operations; every
// result equals the printed formula up to rounding:
//   * (p/p_k)^z with z = (gamma-1)/(2 gamma) = 1/k (gamma = 5/3 -> k = 5,
//     gamma = 7/5 -> k = 7) is a k-th root: an FP32 seed from the SFU
//     (log2/exp2) refined by Newton steps for the reciprocal root,
//     t <- t + (t/k)(1 - r t^k), then r^(1/k) = r t^(k-1); any other gamma uses pow;
//   * FP64 divisions and square roots by Newton iteration from SFU seeds, and
//     FP64 comparisons on the integer pipe (both below);
//   * f_L, f_R at the final pressure reuse the last Newton evaluation when
//     that step left p unchanged;
//   * f'_k on a rarefaction: (p/p_k)^(-(gamma+1)/(2gamma)) / (rho_k a_k)
//     = x (a_k/gamma) / p with x = (p/p_k)^z, since -(gamma+1)/(2gamma) = z - 1 and
//     p_k/(rho_k a_k) = a_k/gamma;
//   * rarefaction star density rho_k (p/p_k)^(1/gamma) = rho_k r / x^2, since
//     1/gamma = 1 - 2z; the fan exponents 2gamma/(gamma-1) = k and
//     2/(gamma-1) = k - 2 are integer powers;
//   * the Newton stopping test 2|p_{n+1}-p_n|/|p_{n+1}+p_n| < tol is evaluated as
//     2|p_{n+1}-p_n| < tol |p_{n+1}+p_n|;
//   * divisions by a, a^2, rho and 6 become products with reciprocals computed
//     once per cell;
//   * of the six traced-parabola integrals of PPMC only those whose wave moves
//     toward the face (the sign tests of App. A.3) are formed.
// With the template switch S (strict) set, every function below instead performs
// the printed formulas operation by operation in the order of the CPU reference
// (divisions, pow), which reproduces that reference bit for bit wherever CUDA's
// pow rounds as the host's does; the FP64 "strict" mode of the library uses it
// to check reproducibility.
//
// Readings where the printed formulas are garbled (shared with the CPU
// reference): xi0 = (-rho du/a + dp/a^2)/2; w6 = 6 w_i - 3 (W_L + W_R);
// B = T^m_L - T^p_L and D = T^p_R - T^0_R with T the traced-parabola integrals;
// right fan sound speed 2/(gamma+1) (a_R - (gamma-1) u_R/2) with u = -a.  Newton:
// tolerance 1e-6, at most 50 iterations, iterates floored at 1e-20, u^m from
// f_L, f_R at the final p^m.
#pragma once
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

namespace hydro {

constexpr int kNG = 4;             // ghost layers per active side
constexpr double kPFloor = 1e-20;  // pressure floor (Sec. 2.4.1)
constexpr double kP0Floor = 1e-6;  // floor of the Newton start value (App. B.1)
constexpr double kNewtonTol = 1e-6;
constexpr int kNewtonMax = 50;

enum : int { kFlagNewton = 1, kFlagNonPhys = 2 };

// gamma-derived constants, computed once on the host in double
template <typename T>
struct GasT {
  T gamma, gm1, gp1;
  T z;        // (gamma-1)/(2 gamma)
  T inv_g;    // 1/gamma
  T inv_gm1;  // 1/(gamma-1)
  T fan_d;    // 2/(gamma-1)
  T fan_p;    // 2 gamma/(gamma-1)
  T two_gp1;  // 2/(gamma+1)
  T half_gm1; // (gamma-1)/2
  T half_gp1; // (gamma+1)/2
  T sh_a;     // (gamma+1)/(2 gamma)
  T sh_b;     // (gamma-1)/(2 gamma)
  T gm1_gp1;  // (gamma-1)/(gamma+1)
  int k;      // z = 1/k exactly for k = 5 or 7, else 0
};

template <typename T>
inline GasT<T> make_gas(double g) {
  GasT<T> c;
  c.gamma = T(g);
  c.gm1 = T(g - 1.0);
  c.gp1 = T(g + 1.0);
  c.z = T((g - 1.0) / (2.0 * g));
  c.inv_g = T(1.0 / g);
  c.inv_gm1 = T(1.0 / (g - 1.0));
  c.fan_d = T(2.0 / (g - 1.0));
  c.fan_p = T(2.0 * g / (g - 1.0));
  c.two_gp1 = T(2.0 / (g + 1.0));
  c.half_gm1 = T((g - 1.0) / 2.0);
  c.half_gp1 = T((g + 1.0) / 2.0);
  c.sh_a = T((g + 1.0) / (2.0 * g));
  c.sh_b = T((g - 1.0) / (2.0 * g));
  c.gm1_gp1 = T((g - 1.0) / (g + 1.0));
  const double kk = 2.0 * g / (g - 1.0);
  const int ki = (int)(kk + 0.5);
  c.k = ((ki == 5 || ki == 7) && fabs(kk - ki) < 1e-12 * ki) ? ki : 0;
  return c;
}

__device__ __forceinline__ double xpow(double x, double y) { return pow(x, y); }
__device__ __forceinline__ float xpow(float x, float y) { return powf(x, y); }
__device__ __forceinline__ double xsqrt(double x) { return sqrt(x); }
__device__ __forceinline__ float xsqrt(float x) { return sqrtf(x); }
__device__ __forceinline__ double xabs(double x) { return fabs(x); }
__device__ __forceinline__ float xabs(float x) { return fabsf(x); }
__device__ __forceinline__ double xfma(double a, double b, double c) { return fma(a, b, c); }
// a rounded product that contraction cannot fuse into a following add
__device__ __forceinline__ double mul_rn(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ float mul_rn(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ float xfma(float a, float b, float c) { return fmaf(a, b, c); }

// min/max with the tie and signed-zero behaviour of "(b < a) ? b : a"
template <typename T> __device__ __forceinline__ T tmin(T a, T b) { return (b < a) ? b : a; }
template <typename T> __device__ __forceinline__ T tmax(T a, T b) { return (a < b) ? b : a; }

// Comparisons of FP64 values through their bit patterns.  GB300 issues an FP64
// compare (and so an FP64 min, max or sign test) on the FP64 pipe; these issue
// on the integer pipe.  ord(x) maps a double to a 64-bit integer with the same
// order (negative values get their magnitude bits inverted), so a < b is
// ord(a) < ord(b); the sign tests read the bits directly.  For every non-NaN
// operand the result equals the IEEE comparison, except that the ordered
// comparison puts -0 below +0 (vmin/vmax may then return -0 where IEEE returns
// +0, the same value).  With S (strict) set, and for float, these are the
// plain IEEE comparisons.
__device__ __forceinline__ long long ord(double x) {
  const long long b = __double_as_longlong(x);
  return b ^ ((b >> 63) & 0x7fffffffffffffffLL);
}
template <bool S, typename T>
__device__ __forceinline__ bool lt(T a, T b) {
  if constexpr (S || sizeof(T) == 4) return a < b;
  else return ord(a) < ord(b);
}
// float: the min/max instructions (one instruction against a compare and a
// select; they differ from the compare-and-select only for NaN operands and in
// which zero of +0/-0 they return)
template <bool S, typename T>
__device__ __forceinline__ T vmin(T a, T b) {
  if constexpr (sizeof(T) == 4) return fminf(a, b);
  else return lt<S>(b, a) ? b : a;
}
template <bool S, typename T>
__device__ __forceinline__ T vmax(T a, T b) {
  if constexpr (sizeof(T) == 4) return fmaxf(a, b);
  else return lt<S>(a, b) ? b : a;
}
// larger of two non-negative doubles (a NaN counts as absent, as in the
// IEEE "(a < b) ? b : a" with the NaN second), on the integer pipe: the bit
// patterns of non-negative doubles order like the values, and a NaN's exceeds
// infinity's
__device__ __forceinline__ double max_nonneg(double a, double b) {
  const long long ka = __double_as_longlong(a), kb = __double_as_longlong(b);
  return (kb > ka && kb <= 0x7ff0000000000000LL) ? b : a;
}
// the same with S (strict): IEEE comparisons, else integer ones (same result)
template <bool S>
__device__ __forceinline__ double max_nn(double v, double w) {
  if constexpr (S) return tmax(v, w);
  else return max_nonneg(v, w);
}
__device__ __forceinline__ bool bits_equal(double a, double b) {
  return __double_as_longlong(a) == __double_as_longlong(b);
}
__device__ __forceinline__ bool bits_equal(float a, float b) {
  return __float_as_int(a) == __float_as_int(b);
}
template <bool S, typename T>
__device__ __forceinline__ bool neg(T x) {  // x < 0
  if constexpr (S || sizeof(T) == 4) return x < T(0);
  else return (unsigned long long)__double_as_longlong(x) > 0x8000000000000000ull;
}
template <bool S, typename T>
__device__ __forceinline__ bool pos(T x) {  // x > 0
  if constexpr (S || sizeof(T) == 4) return x > T(0);
  else return __double_as_longlong(x) > 0;
}
template <bool S, typename T>
__device__ __forceinline__ bool nonpos(T x) {  // x <= 0
  if constexpr (S || sizeof(T) == 4) return x <= T(0);
  else return __double_as_longlong(x) <= 0;
}
template <bool S, typename T>
__device__ __forceinline__ bool nonneg(T x) {  // x >= 0
  if constexpr (S || sizeof(T) == 4) return x >= T(0);
  else return (unsigned long long)__double_as_longlong(x) <= 0x8000000000000000ull;
}

// The two 32-bit halves of a double and back, through PTX moves that the
// compiler cannot see through: a bit test written on the whole 64-bit pattern
// (e.g. "bits << 1 != 0") can otherwise be turned back into an FP64 compare,
// which GB300 issues on its FP64 pipe.
__device__ __forceinline__ void split_bits(double x, unsigned& lo, unsigned& hi) {
  asm("mov.b64 {%0, %1}, %2;" : "=r"(lo), "=r"(hi) : "d"(x));
}
__device__ __forceinline__ double join_bits(unsigned lo, unsigned hi) {
  double x;
  asm("mov.b64 %0, {%1, %2};" : "=d"(x) : "r"(lo), "r"(hi));
  return x;
}
// x with its sign flipped where smask is 0x80000000 (0 leaves x): a negation
// chosen per lane, on the integer pipe
__device__ __forceinline__ double flip_sign(double x, unsigned smask) {
  unsigned lo, hi;
  split_bits(x, lo, hi);
  return join_bits(lo, hi ^ smask);
}
// |x| and, for the limiters, the sign of c given to a non-negative m (c < 0:
// -m, else m) by sign-bit moves on the integer pipe.  An FP64 absolute value
// or negation that the compiler cannot fold into an arithmetic instruction's
// operand (its result feeds a compare or a select) otherwise takes an FP64
// issue slot: on supersonic turbulence the slope kernel ran 32% slower.  With
// S (strict), and for float, the library operations.
template <bool S, typename T>
__device__ __forceinline__ T vabs(T x) {
  if constexpr (S || sizeof(T) == 4) {
    return xabs(x);
  } else {
    unsigned lo, hi;
    split_bits(x, lo, hi);
    return join_bits(lo, hi & 0x7fffffffu);
  }
}
template <bool S, typename T>
__device__ __forceinline__ T sign_of(T c, T m) {
  if constexpr (S || sizeof(T) == 4) return neg<S>(c) ? -m : m;
  else return flip_sign(m, neg<S>(c) ? 0x80000000u : 0u);
}

// Sign tests of a product x*y from the factors' sign bits and zero tests, on
// the integer pipe: an FP64 multiply formed only for its sign costs a full slot
// of the FP64 pipe.  They equal the tests of the rounded product except where
// that product underflows to zero (|x y| < 2^-1074, counted here as nonzero)
// and for NaN factors.  With S (strict), and for float, the product is formed.
template <bool S, typename T>
__device__ __forceinline__ bool prod_pos(T x, T y) {  // x*y > 0
  if constexpr (S || sizeof(T) == 4) {
    return x * y > T(0);
  } else {
    unsigned xl, xh, yl, yh;
    split_bits(x, xl, xh);
    split_bits(y, yl, yh);
    return ((xh << 1) | xl) != 0u && ((yh << 1) | yl) != 0u && (int)(xh ^ yh) >= 0;
  }
}
template <bool S, typename T>
__device__ __forceinline__ bool prod_neg(T x, T y) {  // x*y < 0
  if constexpr (S || sizeof(T) == 4) {
    return x * y < T(0);
  } else {
    unsigned xl, xh, yl, yh;
    split_bits(x, xl, xh);
    split_bits(y, yl, yh);
    return ((xh << 1) | xl) != 0u && ((yh << 1) | yl) != 0u && (int)(xh ^ yh) < 0;
  }
}
template <bool S, typename T>
__device__ __forceinline__ bool prod_nonpos(T x, T y) {  // x*y <= 0
  if constexpr (S || sizeof(T) == 4) return x * y <= T(0);
  else return !prod_pos<S>(x, y);
}

// Sign tests of a product of two differences (a - b)(c - d) without forming
// either difference: a difference of two finite doubles is zero only when they
// are equal (subnormals are not flushed), so its sign is the order of a and b,
// which the ordered bit patterns give on the integer pipe.  Equal to the tests
// of the rounded product except where that product underflows to zero, where
// +0 meets -0 (counted here as unequal), and for NaN.
template <bool S, typename T>
__device__ __forceinline__ bool diffs_prod_nonpos(T a, T b, T c, T d) {  // (a-b)(c-d) <= 0
  if constexpr (S || sizeof(T) == 4) {
    return nonpos<S>((a - b) * (c - d));
  } else {
    const long long oa = ord(a), ob = ord(b), oc = ord(c), od = ord(d);
    return !((oa > ob && oc > od) || (oa < ob && oc < od));
  }
}
template <bool S, typename T>
__device__ __forceinline__ bool diffs_prod_pos(T a, T b, T c, T d) {  // (a-b)(c-d) > 0
  if constexpr (S || sizeof(T) == 4) {
    return pos<S>((a - b) * (c - d));
  } else {
    const long long oa = ord(a), ob = ord(b), oc = ord(c), od = ord(d);
    return (oa > ob && oc > od) || (oa < ob && oc < od);
  }
}
template <bool S, typename T>
__device__ __forceinline__ bool diffs_prod_neg(T a, T b, T c, T d) {  // (a-b)(c-d) < 0
  if constexpr (S || sizeof(T) == 4) {
    return neg<S>((a - b) * (c - d));
  } else {
    const long long oa = ord(a), ob = ord(b), oc = ord(c), od = ord(d);
    return (oa > ob && oc < od) || (oa < ob && oc > od);
  }
}

// x/2 and 2x in integer arithmetic, the IEEE products exactly: a normal
// operand with a normal result moves its exponent field by one; infinities and
// NaN come back unchanged; halving the smallest normals and the subnormals
// shifts the magnitude right by one bit, rounding the dropped bit to even;
// doubling a subnormal shifts it left (exact), doubling the largest binade
// overflows to infinity.  half<S>(x) and twice<S>(x) use them; with S, and for
// float, the multiply itself.
__device__ __forceinline__ double half_bits(double x) {
  unsigned lo, hi;
  split_bits(x, lo, hi);
  const unsigned ex = (hi >> 20) & 0x7ffu;
  if (ex - 2u <= 2044u) return join_bits(lo, hi - (1u << 20));  // 2 <= ex <= 2046
  if (ex == 0x7ffu) return x;
  const unsigned sign = hi & 0x80000000u, mh = hi & 0x7fffffffu;
  unsigned l = (lo >> 1) | (mh << 31), h = mh >> 1;
  if ((lo & 1u) & l) {  // dropped bit 1 and kept bit 1: round up to even
    l += 1u;
    h += (l == 0u) ? 1u : 0u;
  }
  return join_bits(l, sign | h);
}
__device__ __forceinline__ double twice_bits(double x) {
  unsigned lo, hi;
  split_bits(x, lo, hi);
  const unsigned ex = (hi >> 20) & 0x7ffu;
  if (ex - 1u <= 2044u) return join_bits(lo, hi + (1u << 20));  // 1 <= ex <= 2045
  if (ex == 0x7ffu) return x;
  const unsigned sign = hi & 0x80000000u;
  if (ex == 0x7feu) return join_bits(0u, sign | 0x7ff00000u);
  return join_bits(lo << 1, sign | ((hi << 1) & 0x7fffffffu) | (lo >> 31));  // subnormal
}
template <bool S, typename T>
__device__ __forceinline__ T half(T x) {
  if constexpr (S || sizeof(T) == 4) return T(0.5) * x;
  else return half_bits(x);
}
template <bool S, typename T>
__device__ __forceinline__ T twice(T x) {
  if constexpr (S || sizeof(T) == 4) return T(2) * x;
  else return twice_bits(x);
}

// ---------------------------------------------------------------------------
// float <-> double conversion in integer arithmetic.  GB300 issues the
// hardware conversions (cvt.f64.f32, cvt.rn.f32.f64) on its FP64 pipe, at the
// FP64 rate; these rebuild the IEEE 754 bit fields with integer operations and
// selects (no branch, so nothing of the FP64 pipe is issued).  For normal
// values, zeros and infinities they return the bits of the hardware
// conversion with round to nearest even; subnormal values are flushed to a
// zero of the same sign (as the .ftz conversions do), NaN stays NaN, and a
// double beyond the float range becomes an infinity, as IEEE rounding gives.
// hydro_check_conversions() checks them against the hardware on the GPU.

// widening: float fields (1, 8, 23) -> double fields (1, 11, 52), the exponent
// rebiased by 1023 - 127 = 896 (255, infinity or NaN, maps to 2047) and the
// fraction shifted left by 29
__device__ __forceinline__ double f2d(float x) {
  const unsigned b = __float_as_uint(x);
  const unsigned e = b >> 23 & 0xffu;
  const unsigned sign = b & 0x80000000u;
  const unsigned frac_hi = b >> 3 & 0xfffffu;
  unsigned hi = sign | ((e + 896u) << 20) | frac_hi;
  unsigned lo = b << 29;
  hi = (e == 255u) ? (sign | 0x7ff00000u | frac_hi) : hi;
  hi = (e == 0u) ? sign : hi;
  lo = (e == 0u) ? 0u : lo;
  return __hiloint2double((int)hi, (int)lo);
}

// narrowing with round to nearest, ties to even: keep the top 23 of the 52
// fraction bits and round on the 29 discarded ones (a carry out of the
// fraction increments the exponent, and out of the largest exponent gives
// infinity, as IEEE rounding does)
__device__ __forceinline__ float d2f(double x) {
  const unsigned hi = (unsigned)__double2hiint(x), lo = (unsigned)__double2loint(x);
  const unsigned e = hi >> 20 & 0x7ffu;
  const unsigned sign = hi & 0x80000000u;
  const unsigned m = (hi & 0xfffffu) << 3 | lo >> 29;
  const unsigned rest = lo & 0x1fffffffu;
  unsigned f = sign | ((e - 896u) << 23) | m;
  f += (rest > 0x10000000u || (rest == 0x10000000u && (m & 1u))) ? 1u : 0u;
  f = (e > 1150u) ? (sign | 0x7f800000u) : f;  // beyond the float range
  f = (e == 2047u && ((hi & 0xfffffu) | lo)) ? (sign | 0x7fc00000u) : f;  // NaN
  f = (e < 897u) ? sign : f;  // zero, or a float subnormal: flushed
  return __uint_as_float(f);
}

// ---------------------------------------------------------------------------
// FP64 reciprocal, quotient, square root and reciprocal square root by
// Newton-Raphson iteration from SFU seeds.  An IEEE FP64 division or square
// root costs about ten FP64 issue slots on GB300; these cost four to eight.
// Seeds: rcp.approx.ftz.f64 (reciprocal, relative error near 2^-23, issued on
// the SFU) and the float reciprocal square root of the operand scaled by an
// even power of two into [1, 4) (so that every positive normal double has a
// seed).  Iterations:
//   reciprocal   one third-order step r <- r (1 + e + e^2), e = 1 - b r: the
//                series of 1/(1 - e) = 1/(b r) cut after e^2, leaving the
//                seed's error cubed (~2^-69);
//   quotient     a Newton step for r (r <- r + r e, error squared), q = a r,
//                then q <- q + r (a - b q) (Markstein's correction with the
//                residual formed exactly by fma);
//   square root  s = x y, then s <- s + (y/2)(x - s^2), twice (each step
//                multiplies the error by the seed's);
//   rsqrt        one third-order step y <- y (1 + e/2 + 3 e^2/8), e = 1 - x y^2:
//                the binomial series of (1 - e)^(-1/2) = 1/(y sqrt(x)) cut
//                after e^2 (error (5/2) times the seed's cubed, ~2^-64).
// A third-order step costs three (reciprocal) or five (rsqrt) FP64 issue slots
// against four and six for two Newton steps: either way what is left is the
// final rounding and, for rsqrt, the rounding of x y inside the residual (an
// absolute ~2^-53 in e).
// Results are within an ulp or two of the correctly rounded value for
// positive normal operands (the only ones the solver passes); zero, infinite
// and NaN operands are not handled.  The float overloads (mixed precision) are
// the SFU approximations rcp/sqrt/rsqrt.approx and the approximate quotient
// a * rcp(b), each within about two ulp, in place of the IEEE-rounded
// operations' multi-instruction sequences: the mixed path's accuracy bar is an
// L1 difference of 1e-5 to FP64, four hundred times the float ulp.
__device__ __forceinline__ double rcp_seed(double b) {
  double r;
  asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(r) : "d"(b));
  return r;
}
// y ~ 1/sqrt(x), relative error ~2^-22, for positive normal x
__device__ __forceinline__ double rsqrt_seed(double x) {
  const int hi = __double2hiint(x);
  const int k = ((hi >> 20) - 1023) >> 1;  // x = m 2^(2k), m in [1, 4)
  const double m = __hiloint2double(hi - (k << 21), __double2loint(x));
  const double ym = f2d(rsqrtf(d2f(m)));
  return __hiloint2double(__double2hiint(ym) - (k << 20), __double2loint(ym));
}
__device__ __forceinline__ double nr_rcp(double b) {
  const double r = rcp_seed(b);
  const double e = fma(-b, r, 1.0);
  return fma(r, fma(e, e, e), r);
}
__device__ __forceinline__ double nr_div(double a, double b) {
  double r = rcp_seed(b);
  r = fma(r, fma(-b, r, 1.0), r);
  const double q = a * r;
  return fma(r, fma(-b, q, a), q);
}
__device__ __forceinline__ double nr_sqrt(double x) {
  const double y = rsqrt_seed(x);
  const double hy = half_bits(y);
  double s = x * y;
  s = fma(hy, fma(-s, s, x), s);
  return fma(hy, fma(-s, s, x), s);
}
__device__ __forceinline__ double nr_rsqrt(double x) {
  const double y = rsqrt_seed(x);
  const double e = fma(-x * y, y, 1.0);
  return fma(y * e, fma(e, 0.375, 0.5), y);
}
__device__ __forceinline__ float nr_rcp(float b) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(b));
  return r;
}
__device__ __forceinline__ float nr_div(float a, float b) { return a * nr_rcp(b); }
__device__ __forceinline__ float nr_sqrt(float x) {
  float r;
  asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}
__device__ __forceinline__ float nr_rsqrt(float x) {
  float r;
  asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}

// x^K by squaring (K is small)
template <int K, typename T>
__device__ __forceinline__ T ipow(T x) {
  if constexpr (K == 0) {
    return T(1);
  } else if constexpr (K == 1) {
    return x;
  } else {
    const T h = ipow<K / 2>(x);
    if constexpr (K % 2 == 0)
      return h * h;
    else
      return h * h * x;
  }
}

// r^(1/K), correctly rounded, for r in [1e-30, 1e30].
//   1. t ~ r^(-1/K) from an SFU seed (log2/exp2 in float) and one Newton step
//      t <- t + (t/K)(1 - r t^K)  (relative error ~1e-13 in double);
//   2. y = r t^(K-1) ~ r^(1/K), then one Newton step for y^K = r with the
//      residual r - y^K formed exactly in double-double arithmetic (products
//      split by fma); the correction delta = (r - y^K) t^(K-1) / K is ~1e-13 y and
//      is itself accurate to ~1e-26 y, so y + delta rounds to the correctly
//      rounded root.
// Measured faster in the solver than a second reciprocal-root step without the
// correction.  r = 1 gives exactly 1.  In float (mixed path) one Newton step is
// enough for float accuracy.  Double arguments within 2^-20 of 1 take a short
// series instead (below).
template <int K, typename T>
__device__ __forceinline__ T kth_root(T r) {
  if constexpr (sizeof(T) == 8) {
    // near 1 (1 - 2^-20 < r < 1 + 2^-20, e.g. equal pressures up to rounding;
    // tested on the bit pattern): the series 1 + e/K - (K-1) e^2/(2K^2),
    // e = r - 1 exact (Sterbenz); the next term, (K-1)(2K-1) e^3/(6K^3) < 1e-19,
    // is below an ulp
    const long long rb = __double_as_longlong(r);
    if (rb > 0x3feffffe00000000LL && rb < 0x3ff0000100000000LL) {
      const T e = r - T(1);
      return xfma(e, xfma(e, T(-(K - 1) / (2.0 * K * K)), T(1.0 / K)), T(1));
    }
  }
  float lr;
  if constexpr (sizeof(T) == 4)
    lr = __log2f(r);
  else
    lr = __log2f(d2f(r));
  T t;
  if constexpr (sizeof(T) == 4)
    t = exp2f(lr * (-1.0f / (float)K));
  else
    t = f2d(exp2f(lr * (-1.0f / (float)K)));
  const T invK = T(1.0 / K);
  {
    const T e = xfma(-r, ipow<K>(t), T(1));
    t = xfma(t * invK, e, t);
  }
  if constexpr (sizeof(T) == 4) {
    return r * ipow<K - 1>(t);
  } else {
    const T tk1 = ipow<K - 1>(t);
    const T y = r * tk1;
    // y^K as hi + lo (double-double), by repeated exact products
    T hi = y, lo = T(0);
#pragma unroll
    for (int i = 1; i < K; ++i) {
      const T p = hi * y;
      lo = xfma(hi, y, -p) + lo * y;
      hi = p;
    }
    const T res = (r - hi) - lo;  // r - hi is exact (Sterbenz: hi ~ r)
    return xfma(res * tk1, invK, y);
  }
}

// (p/p_k)^z
template <typename T>
__device__ __forceinline__ T pow_z(T r, const GasT<T>& g) {
  if (lt<false>(T(1e-30), r) && lt<false>(r, T(1e30))) {
    if (g.k == 5) return kth_root<5>(r);
    if (g.k == 7) return kth_root<7>(r);
  }
  return xpow(r, g.z);
}

// s^(2/(gamma-1)) and s^(2 gamma/(gamma-1)) of the rarefaction fan
template <typename T>
__device__ __forceinline__ void fan_powers(T s, const GasT<T>& g, T& pd, T& pp) {
  if (g.k == 5) {
    pd = ipow<3>(s);
    pp = pd * s * s;
  } else if (g.k == 7) {
    pd = ipow<5>(s);
    pp = pd * s * s;
  } else {
    pd = xpow(s, g.fan_d);
    pp = xpow(s, g.fan_p);
  }
}

// ---------------------------------------------------------------------------
// ideal-gas conversion in sweep order (rho, normal, t1, t2, E | p)
template <bool S = false, typename T>
__device__ __forceinline__ void cons2prim(const T U[5], const GasT<T>& g, T W[5], T& inv_d) {
  const T d = U[0];
  T vn, v1, v2;
  if constexpr (S) {
    inv_d = T(0);
    vn = U[1] / d;
    v1 = U[2] / d;
    v2 = U[3] / d;
  } else {
    inv_d = nr_rcp(d);
    vn = U[1] * inv_d;
    v1 = U[2] * inv_d;
    v2 = U[3] * inv_d;
  }
  const T p = g.gm1 * (U[4] - half<S>(d) * (vn * vn + v1 * v1 + v2 * v2));
  W[0] = d;
  W[1] = vn;
  W[2] = v1;
  W[3] = v2;
  W[4] = vmax<S>(p, T(kPFloor));
}

template <bool S = false, typename T>
__device__ __forceinline__ void prim2cons(const T W[5], const GasT<T>& g, T U[5]) {
  const T d = W[0];
  U[0] = d;
  U[1] = d * W[1];
  U[2] = d * W[2];
  U[3] = d * W[3];
  if constexpr (S) {
    U[4] = W[4] / g.gm1 + half<S>(d) * (W[1] * W[1] + W[2] * W[2] + W[3] * W[3]);
  } else {
    // rho V^2/2 as (m . v)/2 with the momenta just formed, the halving on the
    // integer pipe and p/(gamma-1) folded into the last multiply-add: one FP64
    // issue slot fewer than rho/2 (v . v) + p/(gamma-1)
    U[4] = fma(W[4], g.inv_gm1, half<S>(U[1] * W[1] + U[2] * W[2] + U[3] * W[3]));
  }
}

// ---------------------------------------------------------------------------
// App. A.2: characteristic projection of a primitive difference
template <bool S, typename T>
__device__ __forceinline__ void char_project(const T dw[5], T rho, T a, T inv_a, T inv_a2,
                                             T xi[5]) {
  T dpa2, rdu_a;
  if constexpr (S) {
    dpa2 = dw[4] / (a * a);
    rdu_a = rho * dw[1] / a;
  } else {
    dpa2 = dw[4] * inv_a2;
    rdu_a = rho * dw[1] * inv_a;
  }
  xi[0] = half<S>(-rdu_a + dpa2);
  xi[1] = dw[0] - dpa2;
  xi[2] = dw[2];
  xi[3] = dw[3];
  xi[4] = half<S>(rdu_a + dpa2);
}

// limited slope of the cell c from its neighbours m (c-1) and p (c+1)
template <bool S = false, typename T>
__device__ __forceinline__ void limited_slope(const T wm[5], const T wc[5], const T wp[5], T a,
                                              T inv_a, T inv_rho, T dw[5]) {
  const T inv_a2 = inv_a * inv_a;
  T xl[5], xr[5], xc[5], dl[5], dr[5], dc[5];
#pragma unroll
  for (int q = 0; q < 5; ++q) {
    dl[q] = wc[q] - wm[q];
    dr[q] = wp[q] - wc[q];
  }
  char_project<S>(dl, wc[0], a, inv_a, inv_a2, xl);
  char_project<S>(dr, wc[0], a, inv_a, inv_a2, xr);
  bool keep[5], any = false;
#pragma unroll
  for (int q = 0; q < 5; ++q) {
    keep[q] = prod_pos<S>(xl[q], xr[q]);
    any = any || keep[q];
  }
  if constexpr (!S && sizeof(T) == 8) {
    // no characteristic slope kept: the back-projection of zeros is +0
    if (!any) {
#pragma unroll
      for (int q = 0; q < 5; ++q) dw[q] = T(0);
      return;
    }
  }
  T xi[5] = {T(0), T(0), T(0), T(0), T(0)};
  // the centred difference is projected only where the limiter keeps a slope
  // (in FP64; in strict mode and in float always, as printed)
  if (S || sizeof(T) == 4 || any) {
#pragma unroll
    for (int q = 0; q < 5; ++q) dc[q] = half<S>(wp[q] - wm[q]);
    char_project<S>(dc, wc[0], a, inv_a, inv_a2, xc);
#pragma unroll
    for (int q = 0; q < 5; ++q) {
      if (keep[q]) {
        const T m = vmin<S>(vmin<S>(vabs<S>(xc[q]), twice<S>(vabs<S>(xl[q]))),
                            twice<S>(vabs<S>(xr[q])));
        xi[q] = sign_of<S>(xc[q], m);
      }
    }
  }
  dw[0] = xi[0] + xi[1] + xi[4];
  dw[1] = (S ? a / wc[0] : a * inv_rho) * (-xi[0] + xi[4]);
  dw[2] = xi[2];
  dw[3] = xi[3];
  dw[4] = a * a * (xi[0] + xi[4]);
}

// ---------------------------------------------------------------------------
// The characteristic corrections of App. A.3 in the fast FP64 path.  The
// contact term E (left face, lambda^0 < 0) excludes the contact term D (right
// face, lambda^0 > 0), and the acoustic term B (left face, lambda^p < 0)
// excludes C (right face, lambda^m > 0).  Each pair is computed once with
// operands chosen per lane: the face's traced reference state and wave speed,
// and the negations that tell the two formulas apart, applied to sign bits on
// the integer pipe.  A warp whose cells take different members of a pair (on
// supersonic turbulent data, most warps) then issues the FP64 work once
// instead of once for each branch.  Every member keeps its printed operation
// order (E = T^m_L - T^0_L, the halvings exact).  The corrections are added
// to the reference states in place, contact term first, each where it applies
// (a face state no correction reaches takes no addition of zero), so a face
// that both a contact and an acoustic term reach sums them one after the
// other rather than first with each other.
// lm, l0, lp: lambda^m, lambda^0, lambda^p of the cell; the reference-state
// integrals are T^m_L = hAm gM and T^p_R = hBp gP; WL, WR: the reference
// states at the left and right face, corrected on return.
__device__ __forceinline__ void ppmc_corrections_fast(double rho, double a, double inv_a,
                                                      double inv_a2, double inv_rho, double dtdx,
                                                      double lm, double l0, double lp,
                                                      const double dw[5], const double w6[5],
                                                      double hAm, double hBp, const double gM[5],
                                                      const double gP[5], double WL[5],
                                                      double WR[5]) {
  const double c23 = 2.0 / 3.0;
  const bool cE = neg<false>(l0), cD = pos<false>(l0);
  if (cE || cD) {
    // E: T^m_L - (alpha^0/2)(dw + w6 (1 + (2/3) alpha^0)), into s_L;
    // D: T^p_R - (beta^0/2)(dw - w6 (1 - (2/3) beta^0)), into s_R
    const unsigned sm = cE ? 0u : 0x80000000u;
    const double c = dtdx * l0;
    const double k = fma(flip_sign(c23, sm), c, 1.0);
    const double hc = half_bits(c);
    double X[5];
#pragma unroll
    for (int q = 0; q < 5; ++q) {
      if (q == 1) continue;
      const double t = (cE ? hAm : hBp) * (cE ? gM[q] : gP[q]);  // T^m_L or T^p_R
      X[q] = fma(-hc, fma(flip_sign(w6[q], sm), k, dw[q]), t);
    }
    X[0] = fma(-X[4], inv_a2, X[0]);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      if (q == 1) continue;
      const double v = (cE ? WL[q] : WR[q]) + X[q];
      WL[q] = cE ? v : WL[q];
      WR[q] = cE ? WR[q] : v;
    }
  }
  const bool cB = neg<false>(lp), cC = pos<false>(lm);
  if (cB || cC) {
    // B: T^m_L - T^p_L (alpha^p), into s_L; C: T^p_R - T^m_R (beta^m), into s_R
    const unsigned sm = cB ? 0u : 0x80000000u;
    const double c = dtdx * (cB ? lp : lm);
    const double k = fma(flip_sign(c23, sm), c, 1.0);
    const double hc = half_bits(c);
    const double h = cB ? hAm : hBp;
    const double X1 = fma(-hc, fma(flip_sign(w6[1], sm), k, dw[1]), h * (cB ? gM[1] : gP[1]));
    const double X4 = fma(-hc, fma(flip_sign(w6[4], sm), k, dw[4]), h * (cB ? gM[4] : gP[4]));
    const double rX1 = flip_sign(rho, sm) * X1;  // rho B1, or -(rho C1)
    double sc[5];
    sc[0] = half_bits(fma(X4, inv_a2, rX1 * inv_a));
    sc[1] = half_bits(fma(flip_sign(X4, sm), inv_a * inv_rho, X1));
    sc[4] = half_bits(fma(rX1, a, X4));
#pragma unroll
    for (int q = 0; q < 5; ++q) {
      if (q == 2 || q == 3) continue;
      const double v = (cB ? WL[q] : WR[q]) + sc[q];
      WL[q] = cB ? v : WL[q];
      WR[q] = cB ? WR[q] : v;
    }
  }
}

// ---------------------------------------------------------------------------
// App. A.3: PPMC.  The parabola's value at the face between cells j and j+1
// (Eq. parabolic_interpolation) from their averages and limited slopes; the
// same expression, and so the same double, for the right face of cell j and
// the left face of cell j+1, which lets neighbouring cells share it.
template <bool S = false, typename T>
__device__ __forceinline__ T ppmc_face(T w_left, T w_right, T s_left, T s_right) {
  if constexpr (S)
    return T(0.5) * (w_right + w_left) - (s_right - s_left) / T(6);
  else
    return half<S>(w_right + w_left) - (s_right - s_left) * T(1.0 / 6.0);
}

// PPMC of cell i from its face values: w_m, w_c, w_p: primitive averages of
// cells i-1, i, i+1; L, R: the parabola's values at its left and right faces
// (ppmc_face); a, inv_a, inv_rho of cell i.  Outputs the traced states at the
// left (WsL) and right (WsR) face of cell i, pressure floored.
template <bool S = false, typename T>
__device__ __forceinline__ void ppmc_states_faces(const T w_m[5], const T w_c[5], const T w_p[5],
                                                  const T Lf[5], const T Rf[5], T a, T inv_a,
                                                  T inv_rho, T dtdx, T WsL[5], T WsR[5]) {
  T dw[5], w6[5];
#pragma unroll
  for (int q = 0; q < 5; ++q) {
    const T wi = w_c[q];
    T L = Lf[q], R = Rf[q];
    if (diffs_prod_nonpos<S>(R, wi, wi, L)) {
      L = wi;
      R = wi;
    }
    if constexpr (!S && sizeof(T) == 8) {
      // 3 w_i - 2 W as one FMA on the exact doubling (a single rounding)
      const T sl = fma(T(3), wi, -twice_bits(R));
      if (diffs_prod_neg<S>(R, L, L, sl)) L = sl;
      const T sr = fma(T(3), wi, -twice_bits(L));
      if (diffs_prod_neg<S>(R, L, sr, R)) R = sr;
    } else {
      if (diffs_prod_neg<S>(R, L, L, T(3) * wi - T(2) * R)) L = T(3) * wi - T(2) * R;
      if (diffs_prod_neg<S>(R, L, T(3) * wi - T(2) * L, R)) R = T(3) * wi - T(2) * L;
    }
    L = vmin<S>(vmax<S>(wi, w_m[q]), vmax<S>(vmin<S>(wi, w_m[q]), L));
    R = vmin<S>(vmax<S>(wi, w_p[q]), vmax<S>(vmin<S>(wi, w_p[q]), R));
    WsL[q] = L;
    WsR[q] = R;
    dw[q] = R - L;
    w6[q] = T(6) * wi - T(3) * (L + R);
  }
  const T rho = w_c[0];
  const T un = w_c[1];
  const T lm = un - a, l0 = un, lp = un + a;
  const T am = dtdx * vmin<S>(lm, T(0)), bp = dtdx * vmax<S>(lp, T(0));
  const T c23 = T(2.0 / 3.0);
  const T inv_a2 = inv_a * inv_a;
  // integral of the parabola over the domain of dependence of the fastest
  // left-going (m) and right-going (p) waves, T^m_L = (alpha^m/2) gM and
  // T^p_R = (beta^p/2) gP: the reference states W_L - T^m_L, W_R - T^p_R
  T gM[5], gP[5];
#pragma unroll
  for (int q = 0; q < 5; ++q) {
    gM[q] = dw[q] + w6[q] * (T(1) + c23 * am);
    gP[q] = dw[q] - w6[q] * (T(1) - c23 * bp);
  }
  if constexpr (!S && sizeof(T) == 8) {
    // fast FP64: each reference state as one FMA (the product T^m_L is
    // formed only where a correction needs it)
    const T hAm = half<S>(am), hBp = half<S>(bp);
#pragma unroll
    for (int q = 0; q < 5; ++q) {
      WsL[q] = fma(-hAm, gM[q], WsL[q]);
      WsR[q] = fma(-hBp, gP[q], WsR[q]);
    }
    ppmc_corrections_fast(rho, a, inv_a, inv_a2, inv_rho, dtdx, lm, l0, lp, dw, w6, hAm, hBp, gM,
                          gP, WsL, WsR);
  } else {
    T tLm[5], tRp[5];
#pragma unroll
    for (int q = 0; q < 5; ++q) {
      tLm[q] = half<S>(am) * gM[q];
      tRp[q] = half<S>(bp) * gP[q];
    }
    T sL[5] = {T(0), T(0), T(0), T(0), T(0)};
    T sR[5] = {T(0), T(0), T(0), T(0), T(0)};
    if (neg<S>(l0)) {  // contact and advected velocities reach the left face: E
      const T a0 = dtdx * l0;
      T E[5];
#pragma unroll
      for (int q = 0; q < 5; ++q)
        E[q] = tLm[q] - half<S>(a0) * (dw[q] + w6[q] * (T(1) + c23 * a0));
      sL[0] = sL[0] + (E[0] - (S ? E[4] / (a * a) : E[4] * inv_a2));
      sL[2] = sL[2] + E[2];
      sL[3] = sL[3] + E[3];
    }
    if (neg<S>(lp)) {  // right acoustic wave reaches the left face: B
      const T ap = dtdx * lp;
      const T B1 = tLm[1] - half<S>(ap) * (dw[1] + w6[1] * (T(1) + c23 * ap));
      const T B4 = tLm[4] - half<S>(ap) * (dw[4] + w6[4] * (T(1) + c23 * ap));
      if constexpr (S) {
        sL[0] = sL[0] + T(0.5) * (rho * B1 / a + B4 / (a * a));
        sL[1] = sL[1] + T(0.5) * (B1 + B4 / (a * rho));
      } else {
        sL[0] = sL[0] + T(0.5) * (rho * B1 * inv_a + B4 * inv_a2);
        sL[1] = sL[1] + T(0.5) * (B1 + B4 * (inv_a * inv_rho));
      }
      sL[4] = sL[4] + T(0.5) * (rho * B1 * a + B4);
    }
    if (pos<S>(lm)) {  // left acoustic wave reaches the right face: C
      const T bm = dtdx * lm;
      const T C1 = tRp[1] - half<S>(bm) * (dw[1] - w6[1] * (T(1) - c23 * bm));
      const T C4 = tRp[4] - half<S>(bm) * (dw[4] - w6[4] * (T(1) - c23 * bm));
      if constexpr (S) {
        sR[0] = sR[0] + T(0.5) * (-(rho * C1) / a + C4 / (a * a));
        sR[1] = sR[1] + T(0.5) * (C1 - C4 / (a * rho));
      } else {
        sR[0] = sR[0] + T(0.5) * (-(rho * C1) * inv_a + C4 * inv_a2);
        sR[1] = sR[1] + T(0.5) * (C1 - C4 * (inv_a * inv_rho));
      }
      sR[4] = sR[4] + T(0.5) * (-(rho * C1 * a) + C4);
    }
    if (pos<S>(l0)) {  // contact and advected velocities reach the right face: D
      const T b0 = dtdx * l0;
      T D[5];
#pragma unroll
      for (int q = 0; q < 5; ++q)
        D[q] = tRp[q] - half<S>(b0) * (dw[q] - w6[q] * (T(1) - c23 * b0));
      sR[0] = sR[0] + (D[0] - (S ? D[4] / (a * a) : D[4] * inv_a2));
      sR[2] = sR[2] + D[2];
      sR[3] = sR[3] + D[3];
    }
#pragma unroll
    for (int q = 0; q < 5; ++q) {
      WsL[q] = (WsL[q] - tLm[q]) + sL[q];
      WsR[q] = (WsR[q] - tRp[q]) + sR[q];
    }
  }
  WsL[4] = vmax<S>(WsL[4], T(kPFloor));
  WsR[4] = vmax<S>(WsR[4], T(kPFloor));
}

// PPMC of cell i from the averages and limited slopes of cells i-1, i, i+1
// (s_m, s_c, s_p), both face values formed here.
template <bool S = false, typename T>
__device__ __forceinline__ void ppmc_states(const T w_m[5], const T w_c[5], const T w_p[5],
                                            const T s_m[5], const T s_c[5], const T s_p[5], T a,
                                            T inv_a, T inv_rho, T dtdx, T WsL[5], T WsR[5]) {
  T Lf[5], Rf[5];
#pragma unroll
  for (int q = 0; q < 5; ++q) {
    Lf[q] = ppmc_face<S>(w_m[q], w_c[q], s_m[q], s_c[q]);
    Rf[q] = ppmc_face<S>(w_c[q], w_p[q], s_c[q], s_p[q]);
  }
  ppmc_states_faces<S>(w_m, w_c, w_p, Lf, Rf, a, inv_a, inv_rho, dtdx, WsL, WsR);
}

// ---------------------------------------------------------------------------
// The other reconstructions of App. A / Sec. 2.2.1 (PPMP, PLMC, PLMP; PCM needs
// no arithmetic).  Arguments in sweep order; S selects the printed operation
// order (strict) as for PPMC.

// primitive-variable slope of one cell: left, right and centred differences
// and the MC limiter (Eqs. diffs, vanLeer_limiter), each variable alone
template <bool S = false, typename T>
__device__ __forceinline__ void prim_slope(const T wm[5], const T wc[5], const T wp[5], T dw[5]) {
#pragma unroll
  for (int q = 0; q < 5; ++q) {
    T s = T(0);
    // the differences are formed only where the limiter keeps a slope
    if (diffs_prod_pos<S>(wc[q], wm[q], wp[q], wc[q])) {
      const T dL = wc[q] - wm[q];
      const T dR = wp[q] - wc[q];
      const T dC = half<S>(wp[q] - wm[q]);
      const T m = vmin<S>(vmin<S>(vabs<S>(dC), twice<S>(vabs<S>(dL))), twice<S>(vabs<S>(dR)));
      s = sign_of<S>(dC, m);
    }
    dw[q] = s;
  }
}

// Euler flux along the sweep of a primitive state (Eq. x_flux)
template <bool S = false, typename T>
__device__ __forceinline__ void euler_flux(const T W[5], const GasT<T>& g, T F[5]) {
  const T E = (S ? W[4] / g.gm1 : W[4] * g.inv_gm1) +
              half<S>(W[0]) * (W[1] * W[1] + W[2] * W[2] + W[3] * W[3]);
  const T m = W[0] * W[1];
  F[0] = m;
  F[1] = m * W[1] + W[4];
  F[2] = m * W[2];
  F[3] = m * W[3];
  F[4] = (E + W[4]) * W[1];
}

// PLMP (App. A.1): W_L = w - dw/2, W_R = w + dw/2 from the limited primitive
// slope dw of the cell, converted to conserved variables and evolved half a
// step with the fluxes of the two boundary values (Eqs. plmp_evolution_L/R).
// Returns the conserved U*_L, U*_R.
template <bool S = false, typename T>
__device__ __forceinline__ void plmp_states(const T wc[5], const T dw[5], T dtdx,
                                            const GasT<T>& g, T UsL[5], T UsR[5]) {
  T WL[5], WR[5];
#pragma unroll
  for (int q = 0; q < 5; ++q) {
    WL[q] = wc[q] - T(0.5) * dw[q];
    WR[q] = wc[q] + T(0.5) * dw[q];
  }
  WL[4] = vmax<S>(WL[4], T(kPFloor));
  WR[4] = vmax<S>(WR[4], T(kPFloor));
  T UL[5], UR[5], FL[5], FR[5];
  prim2cons<S>(WL, g, UL);
  prim2cons<S>(WR, g, UR);
  euler_flux<S>(WL, g, FL);
  euler_flux<S>(WR, g, FR);
  const T h = T(0.5) * dtdx;
#pragma unroll
  for (int q = 0; q < 5; ++q) {
    UsL[q] = UL[q] + h * (FL[q] - FR[q]);
    UsR[q] = UR[q] + h * (FL[q] - FR[q]);
  }
}

// PLMC (App. A.2): boundary values from the characteristic-limited slope dw of
// the cell (limited_slope), bounded by the neighbouring averages, the slope
// recomputed as W_R - W_L, the integral under the linear profile over the
// fastest wave's domain of dependence and the corrections s_L, s_R of the
// other waves that move toward each face.
template <bool S = false, typename T>
__device__ __forceinline__ void plmc_states(const T wm[5], const T wc[5], const T wp[5],
                                            const T dwc[5], T a, T inv_a, T inv_rho, T dtdx,
                                            T WsL[5], T WsR[5]) {
  T WL[5], WR[5], dw[5];
#pragma unroll
  for (int q = 0; q < 5; ++q) {
    const T LA = wc[q] - T(0.5) * dwc[q];
    const T RA = wc[q] + T(0.5) * dwc[q];
    WL[q] = vmin<S>(vmax<S>(wc[q], wm[q]), vmax<S>(vmin<S>(wc[q], wm[q]), LA));
    WR[q] = vmin<S>(vmax<S>(wc[q], wp[q]), vmax<S>(vmin<S>(wc[q], wp[q]), RA));
    dw[q] = WR[q] - WL[q];
  }
  const T d = wc[0];
  const T u = wc[1];
  const T lm = u - a, l0 = u, lp = u + a;
  const T a2 = a * a;
  const T inv_a2 = inv_a * inv_a;
  T sL[5] = {T(0), T(0), T(0), T(0), T(0)};
  T sR[5] = {T(0), T(0), T(0), T(0), T(0)};
  if (neg<S>(l0)) {  // contact (and advected transverse velocities)
    sL[0] = sL[0] + (lm - l0) * (dw[0] - (S ? dw[4] / a2 : dw[4] * inv_a2));
    sL[2] = sL[2] + (lm - l0) * dw[2];
    sL[3] = sL[3] + (lm - l0) * dw[3];
  }
  if (neg<S>(lp)) {  // right acoustic wave
    if constexpr (S) {
      sL[0] = sL[0] + half<S>(lm - lp) * (d * dw[1] / a + dw[4] / a2);
      sL[1] = sL[1] + half<S>(lm - lp) * (dw[1] + dw[4] / (a * d));
    } else {
      sL[0] = sL[0] + half<S>(lm - lp) * (d * dw[1] * inv_a + dw[4] * inv_a2);
      sL[1] = sL[1] + half<S>(lm - lp) * (dw[1] + dw[4] * (inv_a * inv_rho));
    }
    sL[4] = sL[4] + half<S>(lm - lp) * (d * dw[1] * a + dw[4]);
  }
  if (pos<S>(lm)) {  // left acoustic wave
    if constexpr (S) {
      sR[0] = sR[0] + half<S>(lp - lm) * (-(d * dw[1]) / a + dw[4] / a2);
      sR[1] = sR[1] + half<S>(lp - lm) * (dw[1] - dw[4] / (a * d));
    } else {
      sR[0] = sR[0] + half<S>(lp - lm) * (-(d * dw[1]) * inv_a + dw[4] * inv_a2);
      sR[1] = sR[1] + half<S>(lp - lm) * (dw[1] - dw[4] * (inv_a * inv_rho));
    }
    sR[4] = sR[4] + half<S>(lp - lm) * (-(d * dw[1] * a) + dw[4]);
  }
  if (pos<S>(l0)) {  // contact (and advected transverse velocities)
    sR[0] = sR[0] + (lp - l0) * (dw[0] - (S ? dw[4] / a2 : dw[4] * inv_a2));
    sR[2] = sR[2] + (lp - l0) * dw[2];
    sR[3] = sR[3] + (lp - l0) * dw[3];
  }
  const T am = dtdx * vmin<S>(lm, T(0)), bp = dtdx * vmax<S>(lp, T(0));
  const T h = T(0.5) * dtdx;
#pragma unroll
  for (int q = 0; q < 5; ++q) {
    WsL[q] = (WL[q] - half<S>(am) * dw[q]) + h * sL[q];
    WsR[q] = (WR[q] - half<S>(bp) * dw[q]) + h * sR[q];
  }
  WsL[4] = vmax<S>(WsL[4], T(kPFloor));
  WsR[4] = vmax<S>(WsR[4], T(kPFloor));
}

// PPMP shock flattening coefficient F~_k (App. A.4) from p_{k-2..k+2} and the
// normal velocities u_{k-1}, u_{k+1}: zero for a relative pressure jump across
// k-1..k+1 below a third or diverging flow, else max(0, min(1, 10 (S - 3/4)))
// with S = (p_{k+1} - p_{k-1}) / (p_{k+2} - p_{k-2}) (a vanishing denominator
// gives S = +-inf, i.e. F~ = 1 for a positive numerator, else 0)
template <bool S = false, typename T>
__device__ __forceinline__ T flatten_tilde(const T p[5], T um, T up) {
  const T num = p[3] - p[1];
  if constexpr (S) {
    const T jump = xabs(num) / tmin(p[3], p[1]);
    if (jump < T(1.0 / 3.0) || up - um > T(0)) return T(0);
    const T St = num / (p[4] - p[0]);
    return tmax(T(0), tmin(T(1), T(10) * (St - T(0.75))));
  } else {
    if (lt<S>(T(3) * xabs(num), vmin<S>(p[3], p[1])) || pos<S>(up - um)) return T(0);
    const T den = p[4] - p[0];
    if (bits_equal(vabs<S>(den), T(0))) return pos<S>(num) ? T(1) : T(0);
    const T St = nr_div(num, den);
    return vmax<S>(T(0), vmin<S>(T(1), T(10) * (St - T(0.75))));
  }
}

// PPMP for cell i (App. A.4): w[0..6] the primitive states of cells i-3..i+3,
// sm, sc, sp the limited primitive slopes of cells i-1, i, i+1 (prim_slope);
// a, inv_a, inv_rho of cell i; dx the cell width.  Steps in the paper's order:
// parabolic interpolation, density steepening at contacts (concavity test
// d2rho_{i-1} d2rho_{i+1} < 0, as in the method the paper follows; see the
// CPU reference), shock flattening, monotonicity, the integrals under the
// parabola for the three characteristics, the reference states and the CW84
// corrections chi.  Fast mode: division-free forms of the jump tests, the
// undivided second differences in the concavity test and eta (dx cancels),
// reciprocals and square roots by Newton iteration.
template <bool S = false, typename T>
__device__ __forceinline__ void ppmp_states(const T w[7][5], const T sm[5], const T sc[5],
                                            const T sp[5], T a, T dtdx, T dx,
                                            const GasT<T>& g, T WsL[5], T WsR[5]) {
  const T* wim = w[2];
  const T* wi = w[3];
  const T* wip = w[4];
  T WL[5], WR[5];
#pragma unroll
  for (int q = 0; q < 5; ++q) {
    if constexpr (S) {
      WL[q] = T(0.5) * (wi[q] + wim[q]) - (sc[q] - sm[q]) / T(6);
      WR[q] = T(0.5) * (wip[q] + wi[q]) - (sp[q] - sc[q]) / T(6);
    } else {
      WL[q] = half<S>(wi[q] + wim[q]) - (sc[q] - sm[q]) * T(1.0 / 6.0);
      WR[q] = half<S>(wip[q] + wi[q]) - (sp[q] - sc[q]) * T(1.0 / 6.0);
    }
  }
  // contact discontinuity steepening of the density
  {
    T eta = T(0);
    bool steep;
    if constexpr (S) {
      const T rjump = xabs(wip[0] - wim[0]) / tmin(wip[0], wim[0]);
      const T pjump = xabs(wip[4] - wim[4]) / tmin(wip[4], wim[4]);
      const T dx2 = dx * dx;
      const T d2m = (wi[0] - T(2) * wim[0] + w[1][0]) / (T(6) * dx2);
      const T d2p = (w[5][0] - T(2) * wip[0] + wi[0]) / (T(6) * dx2);
      steep = rjump > T(0.01) && pjump < T(0.1) * g.gamma * rjump && d2m * d2p < T(0);
      if (steep) {
        const T eta_t = -((d2p - d2m) * dx2) / (wip[0] - wim[0]);
        eta = tmax(T(0), tmin(T(20) * eta_t - T(1), T(1)));
      }
    } else {
      const T dr = vabs<S>(wip[0] - wim[0]), mr = vmin<S>(wip[0], wim[0]);
      const T dp = xabs(wip[4] - wim[4]), mp = vmin<S>(wip[4], wim[4]);
      const T e2m = wi[0] - T(2) * wim[0] + w[1][0];
      const T e2p = w[5][0] - T(2) * wip[0] + wi[0];
      steep = lt<S>(T(0.01) * mr, dr) && lt<S>(dp * mr, T(0.1) * g.gamma * dr * mp) &&
              prod_neg<S>(e2m, e2p);
      if (steep) {
        const T eta_t = -nr_div(e2p - e2m, T(6) * (wip[0] - wim[0]));
        eta = vmax<S>(T(0), vmin<S>(T(20) * eta_t - T(1), T(1)));
      }
    }
    if (steep) {
      WL[0] = WL[0] * (T(1) - eta) + (wim[0] + T(0.5) * sm[0]) * eta;
      WR[0] = WR[0] * (T(1) - eta) + (wip[0] - T(0.5) * sp[0]) * eta;
    }
  }
  // shock flattening
  {
    T pm[5], pc[5], pp[5];
#pragma unroll
    for (int k = 0; k < 5; ++k) {
      pm[k] = w[k][4];
      pc[k] = w[k + 1][4];
      pp[k] = w[k + 2][4];
    }
    const T Fm = flatten_tilde<S>(pm, w[1][1], w[3][1]);
    const T Fc = flatten_tilde<S>(pc, w[2][1], w[4][1]);
    const T Fp = flatten_tilde<S>(pp, w[3][1], w[5][1]);
    const T F = neg<S>(wip[4] - wim[4]) ? vmax<S>(Fc, Fp) : vmax<S>(Fc, Fm);
#pragma unroll
    for (int q = 0; q < 5; ++q) {
      WL[q] = F * wi[q] + (T(1) - F) * WL[q];
      WR[q] = F * wi[q] + (T(1) - F) * WR[q];
    }
  }
  // monotonicity
  T dw[5], w6[5];
#pragma unroll
  for (int q = 0; q < 5; ++q) {
    T L = WL[q], R = WR[q];
    if (diffs_prod_nonpos<S>(R, wi[q], wi[q], L)) {
      L = wi[q];
      R = wi[q];
    }
    if constexpr (!S && sizeof(T) == 8) {  // one FMA on the exact doubling, as in PPMC
      const T sl = fma(T(3), wi[q], -twice_bits(R));
      if (diffs_prod_neg<S>(R, L, L, sl)) L = sl;
      const T sr = fma(T(3), wi[q], -twice_bits(L));
      if (diffs_prod_neg<S>(R, L, sr, R)) R = sr;
    } else {
      if (diffs_prod_neg<S>(R, L, L, T(3) * wi[q] - T(2) * R)) L = T(3) * wi[q] - T(2) * R;
      if (diffs_prod_neg<S>(R, L, T(3) * wi[q] - T(2) * L, R)) R = T(3) * wi[q] - T(2) * L;
    }
    WL[q] = L;
    WR[q] = R;
    dw[q] = R - L;
    w6[q] = T(6) * (wi[q] - T(0.5) * (L + R));
  }
  // characteristic tracing (CW84): boundary values integrated over each wave's
  // domain of dependence
  const T u = wi[1];
  const T lm = u - a, l0 = u, lp = u + a;
  const T am = dtdx * vmin<S>(lm, T(0)), a0 = dtdx * vmin<S>(l0, T(0)),
          ap = dtdx * vmin<S>(lp, T(0));
  const T bm = dtdx * vmax<S>(lm, T(0)), b0 = dtdx * vmax<S>(l0, T(0)),
          bp = dtdx * vmax<S>(lp, T(0));
  const T c23 = T(2.0 / 3.0);
  T WLm[5], WL0[5], WLp[5], WRm[5], WR0[5], WRp[5];
#pragma unroll
  for (int q = 0; q < 5; ++q) {
    WLm[q] = WL[q] - half<S>(am) * (dw[q] + w6[q] * (T(1) + c23 * am));
    WL0[q] = WL[q] - half<S>(a0) * (dw[q] + w6[q] * (T(1) + c23 * a0));
    WLp[q] = WL[q] - half<S>(ap) * (dw[q] + w6[q] * (T(1) + c23 * ap));
    WRm[q] = WR[q] - half<S>(bm) * (dw[q] - w6[q] * (T(1) - c23 * bm));
    WR0[q] = WR[q] - half<S>(b0) * (dw[q] - w6[q] * (T(1) - c23 * b0));
    WRp[q] = WR[q] - half<S>(bp) * (dw[q] - w6[q] * (T(1) - c23 * bp));
  }
  // reference states and Lagrangian impedances C = rho a of the reference states
  T chiLp, chiRm, chiL0, chiR0, CL, CR, irL, irR;
  if constexpr (S) {
    const T aL = xsqrt(g.gamma * tmax(WLm[4], T(kPFloor)) / WLm[0]);
    const T aR = xsqrt(g.gamma * tmax(WRp[4], T(kPFloor)) / WRp[0]);
    CL = WLm[0] * aL;
    CR = WRp[0] * aR;
    chiLp = -(T(1) / (T(2) * CL)) * ((WLm[1] - WLp[1]) + (WLm[4] - WLp[4]) / CL);
    chiRm = (T(1) / (T(2) * CR)) * ((WRp[1] - WRm[1]) - (WRp[4] - WRm[4]) / CR);
    chiL0 = (WLm[4] - WL0[4]) / (CL * CL) + T(1) / WLm[0] - T(1) / WL0[0];
    chiR0 = (WRp[4] - WR0[4]) / (CR * CR) + T(1) / WRp[0] - T(1) / WR0[0];
    irL = T(1) / WLm[0];
    irR = T(1) / WRp[0];
  } else {
    // C = sqrt(gamma p rho): one reciprocal square root gives C and 1/C
    const T xL = g.gamma * vmax<S>(WLm[4], T(kPFloor)) * WLm[0];
    const T xR = g.gamma * vmax<S>(WRp[4], T(kPFloor)) * WRp[0];
    const T iCL = nr_rsqrt(xL), iCR = nr_rsqrt(xR);
    CL = xL * iCL;
    CR = xR * iCR;
    irL = nr_rcp(WLm[0]);
    irR = nr_rcp(WRp[0]);
    chiLp = -T(0.5) * iCL * ((WLm[1] - WLp[1]) + (WLm[4] - WLp[4]) * iCL);
    chiRm = T(0.5) * iCR * ((WRp[1] - WRm[1]) - (WRp[4] - WRm[4]) * iCR);
    chiL0 = (WLm[4] - WL0[4]) * (iCL * iCL) + irL - nr_rcp(WL0[0]);
    chiR0 = (WRp[4] - WR0[4]) * (iCR * iCR) + irR - nr_rcp(WR0[0]);
  }
  if (pos<S>(l0)) chiL0 = T(0);
  if (pos<S>(lp)) chiLp = T(0);
  if (neg<S>(lm)) chiRm = T(0);
  if (neg<S>(l0)) chiR0 = T(0);
  if constexpr (S) {
    WsL[0] = T(1) / (T(1) / WLm[0] - chiL0 - chiLp);
    WsR[0] = T(1) / (T(1) / WRp[0] - chiRm - chiR0);
  } else {
    WsL[0] = nr_rcp(irL - chiL0 - chiLp);
    WsR[0] = nr_rcp(irR - chiRm - chiR0);
  }
  WsL[1] = WLm[1] + CL * chiLp;
  WsL[2] = WL0[2];
  WsL[3] = WL0[3];
  WsL[4] = vmax<S>(WLm[4] + CL * CL * chiLp, T(kPFloor));
  WsR[1] = WRp[1] - CR * chiRm;
  WsR[2] = WR0[2];
  WsR[3] = WR0[3];
  WsR[4] = vmax<S>(WRp[4] + CR * CR * chiRm, T(kPFloor));
}

// ---------------------------------------------------------------------------
// Roe solver with the HLLE fallback (Sec. 2.2.2, App. B.2) and the H
// correction (App. C).  Inputs in sweep order: conserved U and primitive W of
// each side (W with the pressure floor, inv_d = 1/rho); etaH >= 0 replaces every
// |lambda| of the Roe coefficients by max(|lambda|, etaH) (0: no correction).
// Readings as in the CPU reference: s_3 carries C_3 w~; a "negative"
// intermediate density or pressure is < 0; a Roe average without a real sound
// speed takes the HLLE flux.

template <bool S = false, typename T>
__device__ __forceinline__ void hlle_flux(const T UL[5], const T UR[5], const T WL[5],
                                          const T WR[5], T inv_dL, T inv_dR, const T FL[5],
                                          const T FR[5], T lm, T lp, const GasT<T>& g, T F[5]) {
  T aL, aR;
  if constexpr (S) {
    aL = xsqrt(g.gamma * WL[4] / WL[0]);
    aR = xsqrt(g.gamma * WR[4] / WR[0]);
  } else {
    aL = nr_sqrt(g.gamma * WL[4] * inv_dL);
    aR = nr_sqrt(g.gamma * WR[4] * inv_dR);
  }
  const T bm = vmin<S>(vmin<S>(lm, WL[1] - aL), T(0));
  const T bp = vmax<S>(vmax<S>(lp, WR[1] + aR), T(0));
  // bp = bm = 0 (no real Roe sound speed, u~ = 0, both states moving
  // supersonically toward the face: cold gas at a reflecting wall): the
  // quotient is 0/0; its symmetric limit 0 gives (F_L + F_R)/2
  const T den = bp - bm;
  const T k = !pos<S>(den) ? T(0) : (S ? (bp + bm) / den : nr_div(bp + bm, den));
#pragma unroll
  for (int q = 0; q < 5; ++q) {
    const T FLh = FL[q] - bm * UL[q];
    const T FRh = FR[q] - bp * UR[q];
    F[q] = half<S>((FLh + FRh) + (FLh - FRh) * k);
  }
}

// an intermediate state with rho < 0 or p < 0 (fast: p < 0 as 2 E rho < |m|^2
// for rho > 0)
template <bool S = false, typename T>
__device__ __forceinline__ bool negative_state(const T U[5], const GasT<T>& g) {
  const T m2 = U[1] * U[1] + U[2] * U[2] + U[3] * U[3];
  if constexpr (S) {
    const T p = g.gm1 * (U[4] - T(0.5) * m2 / U[0]);
    return U[0] < T(0) || p < T(0);
  } else {
    return neg<S>(U[0]) || lt<S>(twice<S>(U[4]) * U[0], m2);
  }
}

template <bool S = false, typename T>
__device__ __forceinline__ void riemann_roe(const T UL[5], const T UR[5], const T WL[5],
                                            const T WR[5], T inv_dL, T inv_dR, T etaH,
                                            const GasT<T>& g, T F[5]) {
  T FL[5], FR[5];
  euler_flux<S>(WL, g, FL);
  euler_flux<S>(WR, g, FR);
  T u, v, w, H;
  if constexpr (S) {
    const T sL = xsqrt(WL[0]), sR = xsqrt(WR[0]);
    const T HL = (UL[4] + WL[4]) / WL[0];
    const T HR = (UR[4] + WR[4]) / WR[0];
    u = (sL * WL[1] + sR * WR[1]) / (sL + sR);
    v = (sL * WL[2] + sR * WR[2]) / (sL + sR);
    w = (sL * WL[3] + sR * WR[3]) / (sL + sR);
    H = (sL * HL + sR * HR) / (sL + sR);
  } else {
    const T sL = nr_sqrt(WL[0]), sR = nr_sqrt(WR[0]);
    const T HL = (UL[4] + WL[4]) * inv_dL;
    const T HR = (UR[4] + WR[4]) * inv_dR;
    const T ir = nr_rcp(sL + sR);
    // the normal velocity from two rounded products, not one contracted
    // multiply-add: mirror-image states (a reflecting wall) then give u~ = 0
    // exactly, as in the printed formula's arithmetic, and the HLLE fallback's
    // wave bounds stay at the wall (a contracted form leaves the product's
    // rounding error, ~1e-18, which turns the symmetric wall flux into an
    // upwind one)
    u = (mul_rn(sL, WL[1]) + mul_rn(sR, WR[1])) * ir;
    v = (sL * WL[2] + sR * WR[2]) * ir;
    w = (sL * WL[3] + sR * WR[3]) * ir;
    H = (sL * HL + sR * HR) * ir;
  }
  const T V2 = u * u + v * v + w * w;
  const T a2 = g.gm1 * (H - half<S>(V2));
  if (!pos<S>(a2)) {
    hlle_flux<S>(UL, UR, WL, WR, inv_dL, inv_dR, FL, FR, u, u, g, F);
    return;
  }
  const T a = S ? xsqrt(a2) : nr_sqrt(a2);
  const T lm = u - a, l0 = u, lp = u + a;
  if (nonneg<S>(lm)) {
#pragma unroll
    for (int q = 0; q < 5; ++q) F[q] = FL[q];
    return;
  }
  if (nonpos<S>(lp)) {
#pragma unroll
    for (int q = 0; q < 5; ++q) F[q] = FR[q];
    return;
  }
  T dU[5];
#pragma unroll
  for (int q = 0; q < 5; ++q) dU[q] = UR[q] - UL[q];
  const T gp = g.gm1;
  T Na, ia2;
  if constexpr (S) {
    Na = T(1) / (T(2) * a2);
    ia2 = T(0);
  } else {
    ia2 = nr_rcp(a2);
    Na = T(0.5) * ia2;
  }
  const T xi0 = dU[0] * Na * (T(0.5) * gp * V2 + u * a) - dU[1] * Na * (gp * u + a) -
                dU[2] * Na * gp * v - dU[3] * Na * gp * w + dU[4] * Na * gp;
  const T xi1 = -dU[0] * v + dU[2];
  const T xi2 = -dU[0] * w + dU[3];
  T xi3;
  if constexpr (S)
    xi3 = dU[0] * (T(1) - Na * gp * V2) + dU[1] * gp * u / a2 + dU[2] * gp * v / a2 +
          dU[3] * gp * w / a2 - dU[4] * gp / a2;
  else
    xi3 = dU[0] * (T(1) - Na * gp * V2) + (dU[1] * u + dU[2] * v + dU[3] * w - dU[4]) * (gp * ia2);
  const T xi4 = dU[0] * Na * (T(0.5) * gp * V2 - u * a) - dU[1] * Na * (gp * u - a) -
                dU[2] * Na * gp * v - dU[3] * Na * gp * w + dU[4] * Na * gp;
  const T alm = vmax<S>(vabs<S>(lm), etaH), al0 = vmax<S>(vabs<S>(l0), etaH),
          alp = vmax<S>(vabs<S>(lp), etaH);
  const T C0 = xi0 * alm, C1 = xi1 * al0, C2 = xi2 * al0, C3 = xi3 * al0, C4 = xi4 * alp;
  T s[5];
  s[0] = C0 + C3 + C4;
  s[1] = C0 * (u - a) + C3 * u + C4 * (u + a);
  s[2] = C0 * v + C1 + C3 * v + C4 * v;
  s[3] = C0 * w + C2 + C3 * w + C4 * w;
  s[4] = C0 * (H - u * a) + C1 * v + C2 * w + T(0.5) * C3 * V2 + C4 * (H + u * a);
#pragma unroll
  for (int q = 0; q < 5; ++q) F[q] = half<S>(FL[q] + FR[q] - s[q]);
  // intermediate states: a negative density or pressure takes the HLLE flux
  T Um[5];
  Um[0] = UL[0] + xi0;
  Um[1] = UL[1] + xi0 * (u - a);
  Um[2] = UL[2] + xi0 * v;
  Um[3] = UL[3] + xi0 * w;
  Um[4] = UL[4] + xi0 * (H - u * a);
  bool fail = lt<S>(lm, l0) && negative_state<S>(Um, g);
  if (!fail && lt<S>(l0, lp)) {
    Um[0] = Um[0] + xi3;
    Um[1] = Um[1] + xi3 * u;
    Um[2] = Um[2] + xi1 + xi3 * v;
    Um[3] = Um[3] + xi2 + xi3 * w;
    Um[4] = Um[4] + xi1 * v + xi2 * w + T(0.5) * xi3 * V2;
    fail = negative_state<S>(Um, g);
  }
  if (fail) hlle_flux<S>(UL, UR, WL, WR, inv_dL, inv_dR, FL, FR, lm, lp, g, F);
}

// H-correction quantity of a face (App. C): half the largest jump of a
// characteristic speed, max(|(u_R + a_R) - (u_L + a_L)|, |(u_R - a_R) - (u_L - a_L)|)/2
// (the paper prints the u + a term; see the CPU reference for the reading)
template <bool S = false, typename T>
__device__ __forceinline__ T h_eta(const T WL[5], const T WR[5], T inv_dL, T inv_dR,
                                   const GasT<T>& g) {
  T aL, aR;
  if constexpr (S) {
    aL = xsqrt(g.gamma * WL[4] / WL[0]);
    aR = xsqrt(g.gamma * WR[4] / WR[0]);
  } else {
    aL = nr_sqrt(g.gamma * WL[4] * inv_dL);
    aR = nr_sqrt(g.gamma * WR[4] * inv_dR);
  }
  return half<S>(vmax<S>(vabs<S>((WR[1] + aR) - (WL[1] + aL)),
                         vabs<S>((WR[1] - aR) - (WL[1] - aL))));
}

// ---------------------------------------------------------------------------
// App. B.1: exact Riemann solver
template <typename T>
struct RSide {
  T d, u, p, a;
  T inv_p;  // 1/p_k
  T A, B;   // A_k = 2/((gamma+1) rho_k), B_k = (gamma-1)/(gamma+1) p_k
  T inv_A;  // 1/A_k = (gamma+1) rho_k / 2
  T cf;     // 2 a_k/(gamma-1)
  T cdp;    // a_k/(gamma p_k): f' on a rarefaction is cdp (p/p_k)^(z-1)
};

// pressure function f_k, its derivative, and x = (p/p_k)^z on a rarefaction
// (0 on a shock)
template <bool S, typename T>
__device__ __forceinline__ void side_f(T p, T inv_p, const RSide<T>& s, const GasT<T>& g, T& f,
                                       T& fd, T& x) {
  if (!lt<S>(s.p, p)) {  // p <= p_k
    if constexpr (S) {
      const T r = p / s.p;
      x = xpow(r, g.z);
      f = T(2) * s.a / g.gm1 * (x - T(1));
      fd = T(1) / (s.d * s.a) * xpow(r, -g.sh_a);
    } else {
      x = pow_z(p * s.inv_p, g);
      f = s.cf * (x - T(1));
      fd = x * (s.a * g.inv_g) * inv_p;  // a_k/gamma = p_k/(rho_k a_k)
    }
  } else {
    x = T(0);
    if constexpr (S) {
      const T q = xsqrt(s.A / (p + s.B));
      f = (p - s.p) * q;
      fd = q * (T(1) - (p - s.p) / (T(2) * (s.B + p)));
    } else {
      // q = sqrt(A/(p+B)) as the reciprocal square root of (p+B)/A, then
      // 1/(p+B) = q^2/A
      const T q = nr_rsqrt((p + s.B) * s.inv_A);
      const T ipb = q * q * s.inv_A;
      const T dp = p - s.p;
      f = dp * q;
      fd = q * (T(1) - half<S>(dp) * ipb);
    }
  }
}

template <bool S, typename T>
__device__ __forceinline__ void side_f_only(T p, const RSide<T>& s, const GasT<T>& g, T& f, T& x) {
  if (!lt<S>(s.p, p)) {  // p <= p_k
    if constexpr (S) {
      x = xpow(p / s.p, g.z);
      f = T(2) * s.a / g.gm1 * (x - T(1));
    } else {
      x = pow_z(p * s.inv_p, g);
      f = s.cf * (x - T(1));
    }
  } else {
    if constexpr (!S)
      f = (p - s.p) * nr_rsqrt((p + s.B) * s.inv_A);
    else
      f = (p - s.p) * xsqrt(s.A / (p + s.B));
    x = T(0);
  }
}

// INV: inv_d = 1/rho is given; without it (fast FP64) the sound speed is
// a = x / sqrt(x rho) with x = gamma p, as a product with the reciprocal square
// root y = 1/sqrt(x rho) (nine FP64 issue slots against eleven for 1/rho and
// then sqrt(x/rho)), and the rarefaction derivative's factor a/(gamma p) is y
// itself
template <bool S, typename T, bool INV = true>
__device__ __forceinline__ void make_side(const T W[5], T inv_d, const GasT<T>& g, RSide<T>& s) {
  s.d = W[0];
  s.u = W[1];
  s.p = W[4];
  if constexpr (S) {
    s.a = xsqrt(g.gamma * s.p / s.d);
    s.inv_p = T(0);
    s.A = T(2) / (g.gp1 * s.d);
    s.inv_A = T(0);
  } else {
    s.inv_p = nr_rcp(s.p);
    if constexpr (INV || sizeof(T) == 4) {
      s.a = nr_sqrt(g.gamma * s.p * inv_d);
      s.cdp = s.a * g.inv_g * s.inv_p;
    } else {
      const T x = g.gamma * s.p;
      const T y = nr_rsqrt(x * s.d);
      s.a = x * y;
      s.cdp = y;
    }
    s.A = g.two_gp1 * inv_d;
    s.inv_A = g.half_gp1 * s.d;
  }
  s.B = g.gm1_gp1 * s.p;
  s.cf = S ? T(2) * s.a * g.inv_gm1 : s.a * g.fan_d;  // fan_d = 2 inv_gm1 exactly
  if constexpr (S) s.cdp = T(0);
}

// t = sigma^(-1/m) for sigma in [1e-30, 1e30], with m = K where rare, else 2
// (the two forms of side_eval, chosen per lane).  The seed comes from the float
// log2 and exp2, with relative error delta ~2^-22 near sigma = 1 and up to
// ~2^-19 at the ends of the range (the float exponent log2(sigma)/m keeps fewer
// fraction bits there).  One third-order step follows:
//   t <- t (1 + e/m + (m+1) e^2/(2 m^2)),  e = 1 - sigma t^m,
// the binomial series of (1 - e)^(-1/m) = (exact root)/t cut after e^2.  It
// leaves a relative error of (m+1)(2m+1)/6 delta^3 (below 2^-54 for m = 5 at
// the range's ends) beside the rounding of e (~2^-53 absolute from the
// products forming t^m).  Two Newton steps t <- t + (t/m) e reach the same
// accuracy with five more FP64 issue slots.
template <int K>
__device__ __forceinline__ double rroot_seeded(double sig, bool rare) {
  const float nm = rare ? -1.0f / K : -0.5f;
  const double t = f2d(exp2f(__log2f(d2f(sig)) * nm));
  const double c1 = rare ? 1.0 / K : 0.5;
  const double c2 = rare ? (K + 1) / (2.0 * K * K) : 0.375;
  const double t2 = t * t, t4 = t2 * t2;
  const double tK = (K == 5) ? t4 * t : t4 * t2 * t;
  const double e = fma(-sig, rare ? tK : t2, 1.0);
  return fma(t * e, fma(e, c2, c1), t);
}

// Pressure function of one side without a branch between its two forms, for
// gamma with z = (gamma-1)/(2 gamma) = 1/K (fast FP64 path, used for K = 5).  On
// GB300 the FP64 pipe runs at 1/64 of the float rate and a warp whose lanes
// take both the rarefaction and the shock form issues both: on turbulent data
// nine warps in ten hold both kinds of sides.  Here both forms are one
// reciprocal-root iteration t = sigma^(-1/m) with lane-selected operands:
//   rarefaction (p <= p_k): sigma = p/p_k, m = K: x = (p/p_k)^(1/K) = sigma t^(K-1),
//     f = cf (x - 1), f' = cdp t^(K-1)  (= x a_k/(gamma p), as x/r = t^(K-1));
//   shock: sigma = (p + B_k)/A_k, m = 2: q = sqrt(A_k/(p + B_k)) = t,
//     f = (p - p_k) q, f' = q (1 - (p - p_k)/(2 (p + B_k))), 1/(p + B_k) = t^2/A_k;
// t from rroot_seeded (a float seed and one third-order step), within an ulp
// or so.  A side whose ratio p/p_k lies within 2^-20 of 1 (equal pressures up to
// rounding: uniform regions, where the two-shock start value can land an ulp
// on either side of p_k) takes the rarefaction form's short series on either
// branch: the shock and rarefaction forms of f agree there to within
// (gamma+1)|3 gamma - 5| e^3 sqrt(p_k/rho)/(96 gamma^(5/2)), e = p/p_k - 1
// (third-order contact; zero for gamma = 5/3), below the rounding of f_L + f_R
// + u_R - u_L, and f' to O(e^2), which only scales the Newton step.  A sigma
// outside [1e-30, 1e30] (beyond the float seed's range) takes side_f.
// FD: also f'.  x = 0 on a shock side (the sampling of a shock side does not
// use it).
template <int K, bool FD>
__device__ __forceinline__ void side_eval(double p, const RSide<double>& s,
                                          const GasT<double>& g, double& f, double& fd,
                                          double& x) {
  const bool rare = !lt<false>(s.p, p);  // p <= p_k
  const double r = p * s.inv_p;
  const long long rb = __double_as_longlong(r);
  if (rb > 0x3feffffe00000000LL && rb < 0x3ff0000100000000LL) {
    // (1 + e)^(1/K) and (1 + e)^(1/K - 1) to second order, e = r - 1 exact
    // (Sterbenz); the third-order terms are below 1e-18
    const double e = r - 1.0;
    x = fma(e, fma(e, -(K - 1) / (2.0 * K * K), 1.0 / K), 1.0);
    f = s.cf * (x - 1.0);
    if (FD) fd = s.cdp * fma(e, fma(e, (K - 1) * (2.0 * K - 1) / (2.0 * K * K), -(K - 1.0) / K), 1.0);
    return;
  }
  const double sig = rare ? r : (p + s.B) * s.inv_A;
  if (!(lt<false>(1e-30, sig) && lt<false>(sig, 1e30))) {
    side_f<false>(p, nr_rcp(p), s, g, f, fd, x);
    return;
  }
  const double t = rroot_seeded<K>(sig, rare);
  const double t2 = t * t, t4 = t2 * t2;
  const double tK1 = (K == 5) ? t4 : t4 * t2;  // t^(K-1)
  x = rare ? r * tK1 : 0.0;
  const double dp = p - s.p;
  f = (rare ? s.cf : dp) * (rare ? x - 1.0 : t);
  if (FD) fd = (rare ? s.cdp : t) * (rare ? tK1 : fma(-half<false>(dp), t2 * s.inv_A, 1.0));
}

// sampled state on a rarefaction side at x/t = 0 past the head: star state
// (x = (pm/p_k)^z from the final pressure-function evaluation) or fan; sgn = +1
// for the left side, -1 for the right
template <bool S, bool LEFT, typename T>
__device__ __forceinline__ void sample_raref(const RSide<T>& k, T pm, T um, T x, const GasT<T>& g,
                                             T& d, T& u, T& ps) {
  const T sgn = LEFT ? T(1) : T(-1);
  const bool star = LEFT ? neg<S>(um - k.a * x) : nonneg<S>(um + k.a * x);
  if (star) {  // star state between the fan tail and the contact
    // rho_k (p*/p_k)^(1/gamma); with z = 1/K, 1/gamma = (K-2)/K, so in FP64
    // this is rho_k x^(K-2) (x^3 for gamma = 5/3, x^5 for 7/5: three or four
    // FP64 issue slots against eight for the quotient rho_k r / x^2; Sedov 256^3
    // 46.53 -> 45.65 ms a step); float keeps the quotient (an SFU reciprocal)
    if constexpr (S) {
      d = k.d * xpow(pm / k.p, g.inv_g);
    } else {
      if (sizeof(T) == 8 && g.k == 5) {
        d = k.d * (x * x * x);
      } else if (sizeof(T) == 8 && g.k == 7) {
        const T x2 = x * x;
        d = k.d * (x2 * x2 * x);
      } else {
        d = nr_div(k.d * (pm * k.inv_p), x * x);
      }
    }
    u = um;
    ps = pm;
  } else {  // inside the fan
    const T a = g.two_gp1 * (k.a + sgn * g.half_gm1 * k.u);
    if constexpr (S) {
      d = k.d * xpow(a / k.a, g.fan_d);
      ps = k.p * xpow(a / k.a, g.fan_p);
    } else {
      T pd, pp;
      fan_powers(nr_div(a, k.a), g, pd, pp);
      d = k.d * pd;
      ps = k.p * pp;
    }
    u = sgn * a;
  }
}

// sampled state on a shock side: data state if the shock has not crossed
// x/t = 0, else the post-shock state
template <bool S, typename T>
__device__ __forceinline__ void sample_shock(const RSide<T>& k, T pm, T um, T sgn,
                                             const GasT<T>& g, T& d, T& u, T& ps) {
  const T r = S ? pm / k.p : pm * k.inv_p;
  const T arg = S ? g.sh_a * pm / k.p + g.sh_b : g.sh_a * r + g.sh_b;
  const T sk = k.u - sgn * k.a * (S ? xsqrt(arg) : nr_sqrt(arg));
  if (nonneg<S>(sgn * sk)) {
    d = k.d; u = k.u; ps = k.p;
  } else {
    if constexpr (S)
      d = k.d * (pm / k.p + g.gm1_gp1) / (pm / k.p * g.gm1_gp1 + T(1));
    else
      d = nr_div(k.d * (r + g.gm1_gp1), r * g.gm1_gp1 + T(1));
    u = um;
    ps = pm;
  }
}

// The sampling at x/t = 0 in the fast FP64 path: the side the contact leaves
// behind (left for u* >= 0, right otherwise) is sampled by one code path with
// its operands chosen per lane, the side's state and the signs that mirror
// the right-side formulas into the left-side ones (applied to sign bits on the
// integer pipe).  On data where the contact moves either way within a warp
// (supersonic turbulence) the warp then issues each sampling formula once
// instead of once for each side.  Every test and formula is the side's own,
// operation for operation: the head test u_R + a_R <= 0 is -u_R - a_R >= 0,
// the tail test u* + a_R x >= 0 is -u* - a_R x <= 0, and so on.
template <typename T>
__device__ __forceinline__ void sample_fast(const RSide<T>& L, const RSide<T>& R, T pm, T um,
                                            T xL, T xR, const GasT<T>& g, T& d, T& u, T& ps) {
  const bool left = nonneg<false>(um);
  const unsigned sm = left ? 0u : 0x80000000u;
  const T kd = left ? L.d : R.d, ku = left ? L.u : R.u, kp = left ? L.p : R.p;
  const T ka = left ? L.a : R.a, kip = left ? L.inv_p : R.inv_p;
  const T x = left ? xL : xR;
  if (!lt<false>(kp, pm)) {  // rarefaction
    if (nonneg<false>(flip_sign(ku, sm) - ka)) {  // x/t = 0 ahead of the head: data state
      d = kd; u = ku; ps = kp;
      return;
    }
    const T tail = fma(-ka, x, flip_sign(um, sm));  // u* - a* (left), -(u* + a*) (right)
    if (left ? neg<false>(tail) : nonpos<false>(tail)) {  // star state (see sample_raref)
      if (g.k == 5) {
        d = kd * (x * x * x);
      } else if (g.k == 7) {
        const T x2 = x * x;
        d = kd * (x2 * x2 * x);
      } else {
        d = nr_div(kd * (pm * kip), x * x);
      }
      u = um;
      ps = pm;
    } else {  // inside the fan
      const T a = g.two_gp1 * fma(flip_sign(g.half_gm1, sm), ku, ka);
      T pd, pp;
      fan_powers(nr_div(a, ka), g, pd, pp);
      d = kd * pd;
      ps = kp * pp;
      u = flip_sign(a, sm);
    }
  } else {  // shock
    const T r = pm * kip;
    const T sk = fma(-flip_sign(ka, sm), nr_sqrt(g.sh_a * r + g.sh_b), ku);
    if (nonneg<false>(flip_sign(sk, sm))) {  // the shock has not crossed x/t = 0
      d = kd; u = ku; ps = kp;
    } else {
      d = nr_div(kd * (r + g.gm1_gp1), r * g.gm1_gp1 + T(1));
      u = um;
      ps = pm;
    }
  }
}

// Exact Riemann flux from primitive states in sweep order (inv_d = 1/rho of
// each side, unused when strict); returns the status flags.  K = 5 or 7: the
// fast FP64 form for z = 1/K (side_eval); K = 0: any gamma, strict or float.
template <bool S, typename T, int K, bool INV = true>
__device__ __forceinline__ int riemann_exact_k(const T WL[5], const T WR[5], T inv_dL, T inv_dR,
                                               const GasT<T>& g, T F[5]) {
  RSide<T> L, R;
  make_side<S, T, INV>(WL, inv_dL, g, L);
  make_side<S, T, INV>(WR, inv_dR, g, R);
  if constexpr (K == 5) {
    // gamma = 5/3: B_k = p_k (gamma-1)/(gamma+1) = p_k/4 exactly, by moving
    // the exponent (p_k is at least the 1e-20 floor, a normal number)
    L.B = half_bits(half_bits(L.p));
    R.B = half_bits(half_bits(R.p));
  }
  // primitive-variable estimate, then the two-shock estimate as Newton start
  T pt = half<S>(L.p + R.p) +
         half<S>(half<S>(half<S>(L.u - R.u))) * (L.d + R.d) * (L.a + R.a);  // (1/8) du, exact
  if (neg<S>(pt)) pt = T(0);
  T gL, gR, p;
  if constexpr (!S) {
    gL = nr_rsqrt((pt + L.B) * L.inv_A);
    gR = nr_rsqrt((pt + R.B) * R.inv_A);
    p = nr_div(gL * L.p + gR * R.p - (R.u - L.u), gL + gR);
  } else {
    gL = xsqrt(L.A / (pt + L.B));
    gR = xsqrt(R.A / (pt + R.B));
    p = (gL * L.p + gR * R.p - (R.u - L.u)) / (gL + gR);
  }
  if (lt<S>(p, T(kP0Floor))) p = T(kP0Floor);
  T fL, fR, dfL, dfR, xL, xR;
  int flags = kFlagNewton;
  T prev_step = T(0);  // float path: the previous Newton step
  bool same = false;   // the last step left p unchanged (bit for bit)
  for (int it = 0; it < kNewtonMax; ++it) {
    if constexpr (K != 0) {
      side_eval<K, true>(p, L, g, fL, dfL, xL);
      side_eval<K, true>(p, R, g, fR, dfR, xR);
    } else {
      const T ip = S ? T(0) : nr_rcp(p);
      side_f<S>(p, ip, L, g, fL, dfL, xL);
      side_f<S>(p, ip, R, g, fR, dfR, xR);
    }
    const T F = fL + fR + R.u - L.u;
    T pn = p - (S ? F / (dfL + dfR) : nr_div(F, dfL + dfR));
    if (lt<S>(pn, T(kPFloor))) pn = T(kPFloor);
    same = bits_equal(pn, p);
    bool done;
    if constexpr (S)
      done = T(2) * xabs(pn - p) / xabs(pn + p) < T(kNewtonTol);
    else
      // 2|d| < tol |s| as |d| < (tol/2) |s|: both sides halved exactly
      done = lt<S>(vabs<S>(pn - p), T(0.5 * kNewtonTol) * xabs(pn + p));
    if constexpr (sizeof(T) == 4) {
      // In float the residual f_L + f_R + u_R - u_L carries the rounding error of
      // its terms; near the root the Newton steps that noise produces can stay
      // above the relative tolerance forever (a two-point cycle, e.g. when p*
      // is small against the velocities).  Newton's quadratic convergence never
      // reverses the step without at least halving it, rounding noise does: a
      // step that reverses and does not shrink by half, or a residual at the
      // rounding level of its terms, means float has converged as far as it can.
      const T step = pn - p;
      done = done || (step * prev_step < T(0) && xabs(step) >= T(0.5) * xabs(prev_step)) ||
             xabs(F) <= T(4.0 * 1.1920929e-7) * (xabs(fL) + xabs(fR) + xabs(L.u) + xabs(R.u));
      prev_step = step;
    }
    p = pn;
    if (done) {
      flags = 0;
      break;
    }
  }
  // f_L, f_R and x at the final p (already in hand when the last step left p
  // unchanged, the usual case for smooth data)
  if (!same) {
    if constexpr (K != 0) {
      T unused;
      side_eval<K, false>(p, L, g, fL, unused, xL);
      side_eval<K, false>(p, R, g, fR, unused, xR);
    } else {
      side_f_only<S>(p, L, g, fL, xL);
      side_f_only<S>(p, R, g, fR, xR);
    }
  }
  const T pm = p;
  const T um = half<S>(L.u + R.u + fR - fL);

  T d, u, ps;
  if constexpr (!S && sizeof(T) == 8) {
    sample_fast(L, R, pm, um, xL, xR, g, d, u, ps);
  } else if (nonneg<S>(um)) {
    if (!lt<S>(L.p, pm)) {  // left rarefaction
      if (nonneg<S>(L.u - L.a)) {
        d = L.d; u = L.u; ps = L.p;
      } else {
        sample_raref<S, true>(L, pm, um, xL, g, d, u, ps);
      }
    } else {
      sample_shock<S>(L, pm, um, T(1), g, d, u, ps);
    }
  } else {
    if (!lt<S>(R.p, pm)) {  // right rarefaction
      if (nonpos<S>(R.u + R.a)) {
        d = R.d; u = R.u; ps = R.p;
      } else {
        sample_raref<S, false>(R, pm, um, xR, g, d, u, ps);
      }
    } else {
      sample_shock<S>(R, pm, um, T(-1), g, d, u, ps);
    }
  }
  const bool left = nonneg<S>(u);
  const T v = left ? WL[2] : WR[2];
  const T w = left ? WL[3] : WR[3];
  T Ep;  // E + p
  if constexpr (!S && sizeof(T) == 8) {
    // E + p = p gamma/(gamma-1) + rho V^2/2, gamma/(gamma-1) = fan_p/2 exactly
    Ep = fma(ps, half<S>(g.fan_p), half<S>(d) * (u * u + v * v + w * w));
  } else {
    const T E = (S ? ps / g.gm1 : ps * g.inv_gm1) + half<S>(d) * (u * u + v * v + w * w);
    Ep = E + ps;
  }
  const T mf = d * u;
  F[0] = mf;
  F[1] = mf * u + ps;
  F[2] = mf * v;
  F[3] = mf * w;
  F[4] = Ep * u;
  return flags;
}

// The fast FP64 path takes the branch-free pressure functions for gamma = 5/3
// (K = 5, every three-dimensional workload here).  Other gamma keep the
// correctly rounded k-th root of side_f: for K = 7 the branch-free form's t^6
// and t^7 add two roundings (the fast/strict difference after 10 steps grew
// from 2e-15 to 1.1e-14 of a variable's scale), and a second copy of the solver
// in every Riemann kernel cost 0.2-0.3% on Sedov 256^3 (code size).
// INV = false: inv_dL, inv_dR are not given (fast FP64 only; see make_side).
template <bool S = false, typename T, bool INV = true>
__device__ __forceinline__ int riemann_exact(const T WL[5], const T WR[5], T inv_dL, T inv_dR,
                                             const GasT<T>& g, T F[5]) {
  if constexpr (!S && sizeof(T) == 8) {
    if (g.k == 5) return riemann_exact_k<false, T, 5, INV>(WL, WR, inv_dL, inv_dR, g, F);
  }
  return riemann_exact_k<S, T, 0, INV>(WL, WR, inv_dL, inv_dR, g, F);
}

}  // namespace hydro
