// hydro_selfcheck.cu -- hydro_check_conversions(): the integer-arithmetic
// float <-> double conversions of hydro_math.cuh against the hardware ones
// (bit for bit in the normal range, zeros and infinities; subnormals flushed
// to a signed zero; NaN to NaN); hydro_check_scaling(): its integer halving,
// doubling and sign tests against the FP64 arithmetic, and the float-float to
// double conversion of hydro_ffsum.cuh against the FP64 add;
// hydro_check_newton(): its Newton-refined FP64 reciprocal, quotient, square
// root, reciprocal square root and the pressure function's reciprocal roots,
// in ulps from CUDA's correctly rounded operations or from the exact root;
// hydro_probe_fp64_rate(): the device's measured FP64 FMA throughput, the
// denominator of the FP64 kernels' roofline.
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/hydro.h"
#include "hydro_internal.h"
#include "hydro_ffsum.cuh"
#include "hydro_math.cuh"

namespace {

constexpr int kThreads = 256;
constexpr unsigned kBlocks = 152 * 8;
constexpr unsigned long long kNarrowSamples = 1ull << 30;

__device__ __forceinline__ void count(bool bad, unsigned long long* slot) {
  const unsigned m = __ballot_sync(0xffffffffu, bad);
  if ((threadIdx.x & 31) == 0 && m) atomicAdd(slot, (unsigned long long)__popc(m));
}

// every float bit pattern: the hardware's bits for normal values, zeros and
// infinities; a zero of the same sign for subnormals; NaN for NaN
__global__ void __launch_bounds__(kThreads) k_check_widen(unsigned long long* bad) {
  const unsigned long long n = 1ull << 32;
  const unsigned long long stride = (unsigned long long)gridDim.x * kThreads;
  for (unsigned long long i = (unsigned long long)blockIdx.x * kThreads + threadIdx.x; i < n;
       i += stride) {
    const unsigned bits = (unsigned)i;
    const float x = __uint_as_float(bits);
    const double a = hydro::f2d(x), b = (double)x;
    const unsigned e = bits >> 23 & 0xffu;
    bool ok;
    if (isnan(x))
      ok = isnan(a);
    else if (e == 0u)
      ok = __double_as_longlong(a) == (long long)((unsigned long long)(bits & 0x80000000u) << 32);
    else
      ok = __double_as_longlong(a) == __double_as_longlong(b);
    count(!ok, bad);
  }
}

// splitmix64 (Steele, Lea and Flood, 2014) as a counter-based bit source
__device__ __forceinline__ unsigned long long mix64(unsigned long long z) {
  z += 0x9e3779b97f4a7c15ull;
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
  return z ^ (z >> 31);
}

// doubles: a quarter with any bit pattern, a quarter with exponents around the
// float range (biased 860..1190), a quarter of those with the 29 discarded
// fraction bits at or next to the rounding tie, a quarter near 1 with ties
__global__ void __launch_bounds__(kThreads) k_check_narrow(unsigned long long* bad) {
  const unsigned long long stride = (unsigned long long)gridDim.x * kThreads;
  for (unsigned long long i = (unsigned long long)blockIdx.x * kThreads + threadIdx.x;
       i < kNarrowSamples; i += stride) {
    unsigned long long b = mix64(i);
    const unsigned kind = (unsigned)(i & 3);
    const unsigned long long r = mix64(i ^ 0x5bd1e995ull);
    if (kind >= 1) {
      const unsigned long long e = (kind == 3) ? 1023ull - 2 + (r % 5) : 860ull + (r % 331);
      b = (b & 0x800fffffffffffffull) | (e << 52);
    }
    if (kind >= 2) {
      const unsigned long long low = 0x10000000ull + ((r >> 20) % 3) - 1;  // tie - 1, tie, tie + 1
      b = (b & ~0x1fffffffull) | low;
    }
    const double x = __longlong_as_double((long long)b);
    const float a = hydro::d2f(x), c = __double2float_rn(x);
    const unsigned e = (unsigned)(b >> 52) & 0x7ffu;
    bool ok;
    if (isnan(x))
      ok = isnan(a);
    else if (e < 897u)  // below the float normal range: a zero of the same sign
      ok = __float_as_uint(a) == (unsigned)(b >> 32 & 0x80000000ull);
    else
      ok = __float_as_uint(a) == __float_as_uint(c);
    count(!ok, bad);
  }
}

// doubles for the scaling checks: a quarter with any bit pattern, the rest
// with exponent fields at the edges of the range (0, 1, 2, 2045, 2046, 2047)
// or near the middle, the fraction random or with its low bit set
__device__ __forceinline__ double scaling_sample(unsigned long long i) {
  unsigned long long b = mix64(i * 3 + 1);
  const unsigned long long r = mix64(i * 3 + 2);
  if ((i & 3) != 0) {
    const unsigned long long edge[8] = {0, 1, 2, 2045, 2046, 2047, 1023, 1022};
    const unsigned long long e = edge[r & 7];
    b = (b & 0x800fffffffffffffull) | (e << 52);
    if (r & 8) b |= 1ull;
  }
  return __longlong_as_double((long long)b);
}

__global__ void __launch_bounds__(kThreads) k_check_scaling(unsigned long long* bad) {
  const unsigned long long stride = (unsigned long long)gridDim.x * kThreads;
  for (unsigned long long i = (unsigned long long)blockIdx.x * kThreads + threadIdx.x;
       i < kNarrowSamples; i += stride) {
    const double x = scaling_sample(i), y = scaling_sample(i ^ 0x9e3779b9ull);
    const double h = hydro::half<false>(x), t = hydro::twice<false>(x);
    const double hm = x * 0.5, tm = x * 2.0;
    const bool okh = isnan(x) ? isnan(h) : __double_as_longlong(h) == __double_as_longlong(hm);
    const bool okt = isnan(x) ? isnan(t) : __double_as_longlong(t) == __double_as_longlong(tm);
    // the product's sign tests, except where it underflows to zero or is NaN
    const double p = x * y;
    bool oks = true;
    if (!isnan(p) && !(p == 0.0 && x != 0.0 && y != 0.0))
      oks = hydro::prod_pos<false>(x, y) == (p > 0.0) && hydro::prod_neg<false>(x, y) == (p < 0.0) &&
            hydro::prod_nonpos<false>(x, y) == (p <= 0.0);
    // the sign tests of a product of differences (a-b)(c-d), from the operands'
    // order, except where the rounded product underflows, is NaN, or a
    // difference meets +0 against -0 (equal values, unequal patterns)
    const double a = x, b = (i & 16) ? a : (i & 4) ? y : scaling_sample(i + 0x51ed27ull);
    const double c = scaling_sample(i ^ 0x2545f491ull), e = (i & 8) ? a : scaling_sample(i + 7);
    const double pd = (a - b) * (c - e);
    bool okd = true;
    const bool zero_mix = (a == b && __double_as_longlong(a) != __double_as_longlong(b)) ||
                          (c == e && __double_as_longlong(c) != __double_as_longlong(e));
    if (!isnan(pd) && !zero_mix && !(pd == 0.0 && a != b && c != e))
      okd = hydro::diffs_prod_pos<false>(a, b, c, e) == (pd > 0.0) &&
            hydro::diffs_prod_neg<false>(a, b, c, e) == (pd < 0.0) &&
            hydro::diffs_prod_nonpos<false>(a, b, c, e) == (pd <= 0.0);
    // a float-float pair as one double: within one ulp of the FP64 sum (the
    // second member drawn up to 16 ulp of the first, or much smaller)
    const float fh = __uint_as_float((unsigned)mix64(i ^ 0x7f4a7c15ull) & 0x7f7fffffu |
                                     ((unsigned)i & 0x80000000u)) ;
    const unsigned efh = __float_as_uint(fh) >> 23 & 0xffu;
    const unsigned r2 = (unsigned)mix64(i + 0x94d049bbull);
    const int de = 19 + (int)(r2 % 28u);  // lo 19..46 binades below hi
    float fl = 0.f;
    if (efh > (unsigned)de + 1u)
      fl = __uint_as_float(((efh - de) << 23) | (r2 >> 9 & 0x7fffffu) | (r2 << 31));
    bool okf = true;
    if (efh >= 2u && efh <= 253u) {
      const double ref = (double)fh + (double)fl;
      const double got = hydro::ff_to_double(fh, fl);
      const double ulp = fabs(ref) * 2.220446049250313e-16;
      okf = fabs(got - ref) <= ulp;
    }
    count(!okh, bad);
    count(!okt, bad + 1);
    count(!(oks && okd), bad + 2);
    count(!okf, bad + 3);
  }
}

// distance in ulps between two positive finite doubles
__device__ __forceinline__ unsigned long long ulps(double a, double b) {
  const long long x = __double_as_longlong(a), y = __double_as_longlong(b);
  return (unsigned long long)(x > y ? x - y : y - x);
}

// the nearest double to sigma^(-1/m), from t within a few ulps of it: the
// residual 1 - sigma t^m in double-double arithmetic (products split by fma,
// 1 - s exact by Sterbenz as s lies within a factor 2 of 1), then
// t (1 - res)^(-1/m) = t (1 + res/m + O(res^2)) rounded once; res ~ 2^-52, so
// the dropped terms are ~2^-105 of t
__device__ __forceinline__ double root_reference(double t, double sig, int m) {
  double hi = t, lo = 0.0;
  for (int i = 1; i < m; ++i) {
    const double p = hi * t;
    lo = fma(hi, t, -p) + lo * t;
    hi = p;
  }
  const double s = sig * hi;
  const double sl = fma(sig, hi, -s) + sig * lo;
  const double res = (1.0 - s) - sl;
  return fma(t, res / m, t);
}

// a positive normal double with the exponent drawn from [-emax, emax] and a
// random fraction; one case in eight with the fraction all zeros (a power of
// two) and one in eight all ones (just below one)
__device__ __forceinline__ double newton_sample(unsigned long long i, unsigned emax) {
  const unsigned long long r = mix64(i);
  const unsigned long long e = 1023ull - emax + (mix64(i ^ 0x2545f491ull) % (2ull * emax + 1));
  unsigned long long f = r & 0xfffffffffffffull;
  if ((r >> 61) == 0) f = 0;
  if ((r >> 61) == 1) f = 0xfffffffffffffull;
  return __longlong_as_double((long long)((e << 52) | f));
}

constexpr unsigned long long kNewtonSamples = 1ull << 26;

// largest ulp distances: 0 nr_rcp against __drcp_rn, 1 nr_div against
// __ddiv_rn, 2 nr_sqrt against __dsqrt_rn, 3 nr_rsqrt against the nearest
// double to x^(-1/2), 4 and 5 rroot_seeded<5> (rarefaction form m = 5, shock
// form m = 2) against the nearest double to sigma^(-1/m), sigma in
// [1e-30, 1e30] (the range the pressure function hands it)
__global__ void __launch_bounds__(kThreads) k_check_newton(unsigned long long* worst) {
  unsigned long long w[6] = {0, 0, 0, 0, 0, 0};
  const unsigned long long stride = (unsigned long long)gridDim.x * kThreads;
  for (unsigned long long i = (unsigned long long)blockIdx.x * kThreads + threadIdx.x;
       i < kNewtonSamples; i += stride) {
    const double b = newton_sample(8 * i, 500), x = newton_sample(8 * i + 1, 500);
    const double a = newton_sample(8 * i + 2, 200), c = newton_sample(8 * i + 3, 200);
    // sigma over the binades -99..99, kept strictly inside (1e-30, 1e30)
    const double sig = fmin(fmax(newton_sample(8 * i + 4, 99), nextafter(1e-30, 1.0)),
                            nextafter(1e30, 1.0));
    const double y = hydro::nr_rsqrt(x);
    const double t5 = hydro::rroot_seeded<5>(sig, true);
    const double t2 = hydro::rroot_seeded<5>(sig, false);
    const unsigned long long d[6] = {
        ulps(hydro::nr_rcp(b), __drcp_rn(b)), ulps(hydro::nr_div(a, c), __ddiv_rn(a, c)),
        ulps(hydro::nr_sqrt(x), __dsqrt_rn(x)), ulps(y, root_reference(y, x, 2)),
        ulps(t5, root_reference(t5, sig, 5)), ulps(t2, root_reference(t2, sig, 2))};
#pragma unroll
    for (int k = 0; k < 6; ++k) w[k] = d[k] > w[k] ? d[k] : w[k];
  }
#pragma unroll
  for (int k = 0; k < 6; ++k) atomicMax(worst + k, w[k]);
}

// FP64 FMA throughput: every thread runs kChains independent chains
// x <- x * b + c of kRateIters fused multiply-adds each (b, c from the host, so
// nothing folds); the sum is stored only if it equals a value it cannot take,
// which keeps the chains live without writing memory
constexpr int kChains = 8;
constexpr int kRateIters = 4096;
constexpr unsigned kRateBlocks = 152 * 8;
__device__ double g_rate_sink;

__global__ void __launch_bounds__(kThreads) k_fp64_rate(double b, double c, double never) {
  double x[kChains];
#pragma unroll
  for (int k = 0; k < kChains; ++k) x[k] = (double)(threadIdx.x + k);
  for (int i = 0; i < kRateIters; ++i) {
#pragma unroll
    for (int k = 0; k < kChains; ++k) x[k] = fma(x[k], b, c);
  }
  double s = 0.0;
#pragma unroll
  for (int k = 0; k < kChains; ++k) s += x[k];
  if (s == never) g_rate_sink = s;
}

}  // namespace

extern "C" int hydro_probe_fp64_rate(double* flops_per_s, void* stream) {
  if (!flops_per_s) return HYDRO_EINVAL;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaEventCreate(&e0) != cudaSuccess) return HYDRO_ECUDA;
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return HYDRO_ECUDA;
  }
  int rc = HYDRO_OK;
  float best_ms = -1.0f;
  // a warm-up launch, then the fastest of three timed ones
  for (int rep = 0; rep < 4 && rc == HYDRO_OK; ++rep) {
    if (cudaEventRecord(e0, st) != cudaSuccess) rc = HYDRO_ECUDA;
    k_fp64_rate<<<kRateBlocks, kThreads, 0, st>>>(0.999999, 1e-7, -1.0);
    if (cudaGetLastError() != cudaSuccess || cudaEventRecord(e1, st) != cudaSuccess ||
        cudaEventSynchronize(e1) != cudaSuccess)
      rc = HYDRO_ECUDA;
    float ms = 0.0f;
    if (rc == HYDRO_OK && cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) rc = HYDRO_ECUDA;
    if (rc == HYDRO_OK && rep > 0 && (best_ms < 0.0f || ms < best_ms)) best_ms = ms;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc != HYDRO_OK) return rc;
  if (!(best_ms > 0.0f)) return HYDRO_ECUDA;
  const double fmas = (double)kRateBlocks * kThreads * kChains * kRateIters;
  *flops_per_s = 2.0 * fmas / (best_ms * 1e-3);
  return HYDRO_OK;
}

extern "C" int hydro_check_scaling(unsigned long long* mismatches, void* stream) {
  if (!mismatches) return HYDRO_EINVAL;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  unsigned long long* d = nullptr;
  if (cudaMalloc(&d, 4 * sizeof(unsigned long long)) != cudaSuccess) return HYDRO_ECUDA;
  int rc = HYDRO_OK;
  if (cudaMemsetAsync(d, 0, 4 * sizeof(unsigned long long), st) != cudaSuccess) rc = HYDRO_ECUDA;
  if (rc == HYDRO_OK) {
    k_check_scaling<<<kBlocks, kThreads, 0, st>>>(d);
    if (cudaGetLastError() != cudaSuccess) rc = HYDRO_ECUDA;
  }
  if (rc == HYDRO_OK &&
      (cudaMemcpyAsync(mismatches, d, 4 * sizeof(unsigned long long), cudaMemcpyDeviceToHost,
                       st) != cudaSuccess ||
       cudaStreamSynchronize(st) != cudaSuccess))
    rc = HYDRO_ECUDA;
  cudaFree(d);
  return rc;
}

extern "C" int hydro_check_newton(unsigned long long* max_ulp, void* stream) {
  if (!max_ulp) return HYDRO_EINVAL;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  unsigned long long* d = nullptr;
  if (cudaMalloc(&d, 6 * sizeof(unsigned long long)) != cudaSuccess) return HYDRO_ECUDA;
  int rc = HYDRO_OK;
  if (cudaMemsetAsync(d, 0, 6 * sizeof(unsigned long long), st) != cudaSuccess) rc = HYDRO_ECUDA;
  if (rc == HYDRO_OK) {
    k_check_newton<<<kBlocks, kThreads, 0, st>>>(d);
    if (cudaGetLastError() != cudaSuccess) rc = HYDRO_ECUDA;
  }
  if (rc == HYDRO_OK &&
      (cudaMemcpyAsync(max_ulp, d, 6 * sizeof(unsigned long long), cudaMemcpyDeviceToHost,
                       st) != cudaSuccess ||
       cudaStreamSynchronize(st) != cudaSuccess))
    rc = HYDRO_ECUDA;
  cudaFree(d);
  return rc;
}

extern "C" int hydro_check_conversions(unsigned long long* mismatches, void* stream) {
  if (!mismatches) return HYDRO_EINVAL;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  unsigned long long* d = nullptr;
  if (cudaMalloc(&d, 2 * sizeof(unsigned long long)) != cudaSuccess) return HYDRO_ECUDA;
  int rc = HYDRO_OK;
  if (cudaMemsetAsync(d, 0, 2 * sizeof(unsigned long long), st) != cudaSuccess) rc = HYDRO_ECUDA;
  if (rc == HYDRO_OK) {
    k_check_widen<<<kBlocks, kThreads, 0, st>>>(d);
    k_check_narrow<<<kBlocks, kThreads, 0, st>>>(d + 1);
    if (cudaGetLastError() != cudaSuccess) rc = HYDRO_ECUDA;
  }
  if (rc == HYDRO_OK &&
      (cudaMemcpyAsync(mismatches, d, 2 * sizeof(unsigned long long), cudaMemcpyDeviceToHost,
                       st) != cudaSuccess ||
       cudaStreamSynchronize(st) != cudaSuccess))
    rc = HYDRO_ECUDA;
  cudaFree(d);
  return rc;
}

// Host check of the multiply-high division the kernels use for index
// arithmetic (FastDiv in hydro_internal.h): every divisor 1..2^16, then
// divisors spread up to 2^31 - 1 by a counter-based hash, each against
// numerators at the edges (0, d - 1, d, d + 1, multiples of d near 2^31 - 1,
// 2^31 - 1 itself) and hashed numerators below 2^31.
extern "C" long long hydro_check_fastdiv(void) {
  auto mix = [](unsigned long long x) {  // splitmix64 finaliser
    x += 0x9e3779b97f4a7c15ull;
    x = (x ^ (x >> 30)) * 0xbf58476d1ce4e5b9ull;
    x = (x ^ (x >> 27)) * 0x94d049bb133111ebull;
    return x ^ (x >> 31);
  };
  const unsigned kMax = 0x7fffffffu;
  long long bad = 0;
  auto check = [&](unsigned d) {
    const hydro::FastDiv f = hydro::make_fastdiv(d);
    auto one = [&](unsigned n) {
      if (n > kMax) return;
      if (hydro::fast_div(n, f) != n / d) ++bad;
    };
    one(0);
    one(d - 1);
    one(d);
    one(d + 1);
    const unsigned top = kMax / d;
    for (unsigned k = top > 2 ? top - 2 : 0; k <= top; ++k) {
      one(k * d);
      if (k * d > 0) one(k * d - 1);
      if (k * d < kMax) one(k * d + 1);
    }
    one(kMax);
    for (unsigned i = 0; i < 64; ++i) one((unsigned)(mix(((unsigned long long)d << 8) + i) & kMax));
  };
  for (unsigned d = 1; d <= 65536; ++d) check(d);
  for (unsigned i = 0; i < 200000; ++i) {
    unsigned d = (unsigned)(mix(0x5eedull + i) & kMax);
    if (d == 0) d = 1;
    check(d);
  }
  for (unsigned k = 0; k < 31; ++k) {
    check(1u << k);
    check((1u << k) + 1);
    if (k > 0) check((1u << k) - 1);
  }
  return bad;
}
