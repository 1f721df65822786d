// hydro_math.cuh -- device arithmetic of one CTU step, templated on the
// arithmetic type T (double for the FP64 path, float for the reconstruction and
// Riemann stages of the mixed path).
//
//   * cons/prim conversion of the ideal gas (Sec. 2.1);
//   * the characteristic-limited slope of one cell (App. A.2, Eqs. diffs,
//     plmc_lim_slopes and the PLMC projection);
//   * PPMC face states with characteristic tracing (App. A.3);
//   * the exact Riemann solver with Newton iteration and ten-case sampling
//     (App. B.1).
//
// Readings where the paper's printed formulas are garbled (the same readings
// as the CPU reference): xi0 = (-rho du/a + dp/a^2)/2; w6 = 6 w_i - 3 (W_L + W_R);
// B = T^m_L - T^p_L and D = T^p_R - T^0_R with T the traced-parabola integrals;
// the right fan sound speed 2/(gamma+1) (a_R - (gamma-1) u_R/2) with u = -a.
// Newton: tolerance 1e-6, at most 50 iterations, iterates floored at 1e-20,
// u^m from f_L, f_R at the final p^m.
#pragma once
#include <cuda_runtime.h>
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
  T zd;       // -(gamma+1)/(2 gamma)
  T inv_g;    // 1/gamma
  T fan_d;    // 2/(gamma-1)
  T fan_p;    // 2 gamma/(gamma-1)
  T two_gp1;  // 2/(gamma+1)
  T half_gm1; // (gamma-1)/2
  T sh_a;     // (gamma+1)/(2 gamma)
  T sh_b;     // (gamma-1)/(2 gamma)
  T gm1_gp1;  // (gamma-1)/(gamma+1)
};

template <typename T>
inline GasT<T> make_gas(double g) {
  GasT<T> c;
  c.gamma = T(g);
  c.gm1 = T(g - 1.0);
  c.gp1 = T(g + 1.0);
  c.z = T((g - 1.0) / (2.0 * g));
  c.zd = T(-(g + 1.0) / (2.0 * g));
  c.inv_g = T(1.0 / g);
  c.fan_d = T(2.0 / (g - 1.0));
  c.fan_p = T(2.0 * g / (g - 1.0));
  c.two_gp1 = T(2.0 / (g + 1.0));
  c.half_gm1 = T((g - 1.0) / 2.0);
  c.sh_a = T((g + 1.0) / (2.0 * g));
  c.sh_b = T((g - 1.0) / (2.0 * g));
  c.gm1_gp1 = T((g - 1.0) / (g + 1.0));
  return c;
}

__device__ __forceinline__ double xpow(double x, double y) { return pow(x, y); }
__device__ __forceinline__ float xpow(float x, float y) { return powf(x, y); }
__device__ __forceinline__ double xsqrt(double x) { return sqrt(x); }
__device__ __forceinline__ float xsqrt(float x) { return sqrtf(x); }
__device__ __forceinline__ double xabs(double x) { return fabs(x); }
__device__ __forceinline__ float xabs(float x) { return fabsf(x); }

// min/max with the tie and signed-zero behaviour of "(b < a) ? b : a"
template <typename T> __device__ __forceinline__ T tmin(T a, T b) { return (b < a) ? b : a; }
template <typename T> __device__ __forceinline__ T tmax(T a, T b) { return (a < b) ? b : a; }

// ---------------------------------------------------------------------------
// ideal-gas conversion in sweep order (rho, normal, t1, t2, E | p)
template <typename T>
__device__ __forceinline__ void cons2prim(const T U[5], const GasT<T>& g, T W[5]) {
  const T d = U[0];
  const T vn = U[1] / d, v1 = U[2] / d, v2 = U[3] / d;
  const T p = g.gm1 * (U[4] - T(0.5) * d * (vn * vn + v1 * v1 + v2 * v2));
  W[0] = d;
  W[1] = vn;
  W[2] = v1;
  W[3] = v2;
  W[4] = tmax(p, T(kPFloor));
}

template <typename T>
__device__ __forceinline__ void prim2cons(const T W[5], const GasT<T>& g, T U[5]) {
  const T d = W[0];
  U[0] = d;
  U[1] = d * W[1];
  U[2] = d * W[2];
  U[3] = d * W[3];
  U[4] = W[4] / g.gm1 + T(0.5) * d * (W[1] * W[1] + W[2] * W[2] + W[3] * W[3]);
}

// ---------------------------------------------------------------------------
// App. A.2: project a primitive difference onto the characteristic fields of a
// cell with density rho and sound speed a
template <typename T>
__device__ __forceinline__ void char_project(const T dw[5], T rho, T a, T xi[5]) {
  const T a2 = a * a;
  const T dpa2 = dw[4] / a2;
  const T rdu_a = rho * dw[1] / a;
  xi[0] = T(0.5) * (-rdu_a + dpa2);
  xi[1] = dw[0] - dpa2;
  xi[2] = dw[2];
  xi[3] = dw[3];
  xi[4] = T(0.5) * (rdu_a + dpa2);
}

// limited slope of the cell c from its neighbours m (c-1) and p (c+1)
template <typename T>
__device__ __forceinline__ void limited_slope(const T wm[5], const T wc[5], const T wp[5], T a,
                                              T dw[5]) {
  T dl[5], dr[5], dc[5];
#pragma unroll
  for (int q = 0; q < 5; ++q) {
    dl[q] = wc[q] - wm[q];
    dr[q] = wp[q] - wc[q];
    dc[q] = T(0.5) * (wp[q] - wm[q]);
  }
  T xl[5], xr[5], xc[5], xi[5];
  char_project(dl, wc[0], a, xl);
  char_project(dr, wc[0], a, xr);
  char_project(dc, wc[0], a, xc);
#pragma unroll
  for (int q = 0; q < 5; ++q) {
    T s = T(0);
    if (xl[q] * xr[q] > T(0)) {
      const T m = tmin(tmin(xabs(xc[q]), T(2) * xabs(xl[q])), T(2) * xabs(xr[q]));
      s = (xc[q] < T(0)) ? -m : m;
    }
    xi[q] = s;
  }
  dw[0] = xi[0] + xi[1] + xi[4];
  dw[1] = a / wc[0] * (-xi[0] + xi[4]);
  dw[2] = xi[2];
  dw[3] = xi[3];
  dw[4] = a * a * (xi[0] + xi[4]);
}

// ---------------------------------------------------------------------------
// App. A.3: PPMC.  w_m, w_c, w_p: primitive averages of cells i-1, i, i+1;
// s_m, s_c, s_p: their limited slopes; a: sound speed of cell i.  Outputs the
// traced states at the left (WsL) and right (WsR) face of cell i, pressure
// floored.
template <typename T>
__device__ __forceinline__ void ppmc_states(const T w_m[5], const T w_c[5], const T w_p[5],
                                            const T s_m[5], const T s_c[5], const T s_p[5], T a,
                                            T dtdx, T WsL[5], T WsR[5]) {
  T dw[5], w6[5], WL[5], WR[5];
#pragma unroll
  for (int q = 0; q < 5; ++q) {
    const T wi = w_c[q];
    T L = T(0.5) * (wi + w_m[q]) - (s_c[q] - s_m[q]) / T(6);
    T R = T(0.5) * (w_p[q] + wi) - (s_p[q] - s_c[q]) / T(6);
    if ((R - wi) * (wi - L) <= T(0)) {
      L = wi;
      R = wi;
    }
    if ((R - L) * (L - (T(3) * wi - T(2) * R)) < T(0)) L = T(3) * wi - T(2) * R;
    if ((R - L) * ((T(3) * wi - T(2) * L) - R) < T(0)) R = T(3) * wi - T(2) * L;
    L = tmin(tmax(wi, w_m[q]), tmax(tmin(wi, w_m[q]), L));
    R = tmin(tmax(wi, w_p[q]), tmax(tmin(wi, w_p[q]), R));
    WL[q] = L;
    WR[q] = R;
    dw[q] = R - L;
    w6[q] = T(6) * wi - T(3) * (L + R);
  }
  const T rho = w_c[0];
  const T un = w_c[1];
  const T lm = un - a, l0 = un, lp = un + a;
  const T am = dtdx * tmin(lm, T(0)), a0 = dtdx * tmin(l0, T(0)), ap = dtdx * tmin(lp, T(0));
  const T bm = dtdx * tmax(lm, T(0)), b0 = dtdx * tmax(l0, T(0)), bp = dtdx * tmax(lp, T(0));
  const T c23 = T(2.0 / 3.0);
  const T a2 = a * a;
  T E[5], B[5], C[5], D[5];
#pragma unroll
  for (int q = 0; q < 5; ++q) {
    const T tLm = T(0.5) * am * (dw[q] + w6[q] * (T(1) + c23 * am));
    const T tL0 = T(0.5) * a0 * (dw[q] + w6[q] * (T(1) + c23 * a0));
    const T tLp = T(0.5) * ap * (dw[q] + w6[q] * (T(1) + c23 * ap));
    const T tRm = T(0.5) * bm * (dw[q] - w6[q] * (T(1) - c23 * bm));
    const T tR0 = T(0.5) * b0 * (dw[q] - w6[q] * (T(1) - c23 * b0));
    const T tRp = T(0.5) * bp * (dw[q] - w6[q] * (T(1) - c23 * bp));
    WsL[q] = WL[q] - tLm;
    WsR[q] = WR[q] - tRp;
    E[q] = tLm - tL0;
    B[q] = tLm - tLp;
    C[q] = tRp - tRm;
    D[q] = tRp - tR0;
  }
  T sL[5] = {T(0), T(0), T(0), T(0), T(0)};
  T sR[5] = {T(0), T(0), T(0), T(0), T(0)};
  if (l0 < T(0)) {
    sL[0] = sL[0] + (E[0] - E[4] / a2);
    sL[2] = sL[2] + E[2];
    sL[3] = sL[3] + E[3];
  }
  if (lp < T(0)) {
    sL[0] = sL[0] + T(0.5) * (rho * B[1] / a + B[4] / a2);
    sL[1] = sL[1] + T(0.5) * (B[1] + B[4] / (a * rho));
    sL[4] = sL[4] + T(0.5) * (rho * B[1] * a + B[4]);
  }
  if (lm > T(0)) {
    sR[0] = sR[0] + T(0.5) * (-(rho * C[1]) / a + C[4] / a2);
    sR[1] = sR[1] + T(0.5) * (C[1] - C[4] / (a * rho));
    sR[4] = sR[4] + T(0.5) * (-(rho * C[1] * a) + C[4]);
  }
  if (l0 > T(0)) {
    sR[0] = sR[0] + (D[0] - D[4] / a2);
    sR[2] = sR[2] + D[2];
    sR[3] = sR[3] + D[3];
  }
#pragma unroll
  for (int q = 0; q < 5; ++q) {
    WsL[q] = WsL[q] + sL[q];
    WsR[q] = WsR[q] + sR[q];
  }
  WsL[4] = tmax(WsL[4], T(kPFloor));
  WsR[4] = tmax(WsR[4], T(kPFloor));
}

// ---------------------------------------------------------------------------
// App. B.1: pressure function of one side and its derivative
template <typename T>
__device__ __forceinline__ void pressure_fn(T p, T dk, T pk, T ak, T Ak, T Bk, const GasT<T>& g,
                                            T& f, T& fd) {
  if (p <= pk) {
    const T r = p / pk;
    f = T(2) * ak / g.gm1 * (xpow(r, g.z) - T(1));
    fd = T(1) / (dk * ak) * xpow(r, g.zd);
  } else {
    const T q = xsqrt(Ak / (p + Bk));
    f = (p - pk) * q;
    fd = q * (T(1) - (p - pk) / (T(2) * (Bk + p)));
  }
}

// Exact Riemann flux from primitive states in sweep order; returns the flags.
template <typename T>
__device__ __forceinline__ int riemann_exact(const T WL[5], const T WR[5], const GasT<T>& g,
                                             T F[5]) {
  const T dL = WL[0], uL = WL[1], pL = WL[4];
  const T dR = WR[0], uR = WR[1], pR = WR[4];
  const T aL = xsqrt(g.gamma * pL / dL);
  const T aR = xsqrt(g.gamma * pR / dR);
  T pt = T(0.5) * (pL + pR) + T(0.125) * (uL - uR) * (dL + dR) * (aL + aR);
  if (pt < T(0)) pt = T(0);
  const T AL = T(2) / (g.gp1 * dL), AR = T(2) / (g.gp1 * dR);
  const T BL = g.gm1_gp1 * pL, BR = g.gm1_gp1 * pR;
  const T gL = xsqrt(AL / (pt + BL)), gR = xsqrt(AR / (pt + BR));
  T p = (gL * pL + gR * pR - (uR - uL)) / (gL + gR);
  if (p < T(kP0Floor)) p = T(kP0Floor);
  T fL, fR, dfL, dfR;
  int flags = kFlagNewton;
  for (int it = 0; it < kNewtonMax; ++it) {
    pressure_fn(p, dL, pL, aL, AL, BL, g, fL, dfL);
    pressure_fn(p, dR, pR, aR, AR, BR, g, fR, dfR);
    T pn = p - (fL + fR + uR - uL) / (dfL + dfR);
    if (pn < T(kPFloor)) pn = T(kPFloor);
    const T delta = T(2) * xabs(pn - p) / xabs(pn + p);
    p = pn;
    if (delta < T(kNewtonTol)) {
      flags = 0;
      break;
    }
  }
  pressure_fn(p, dL, pL, aL, AL, BL, g, fL, dfL);
  pressure_fn(p, dR, pR, aR, AR, BR, g, fR, dfR);
  const T pm = p;
  const T um = T(0.5) * (uL + uR + fR - fL);

  T d, u, ps;
  if (um >= T(0)) {
    if (pm <= pL) {
      if (uL - aL >= T(0)) {
        d = dL; u = uL; ps = pL;
      } else if (um - aL * xpow(pm / pL, g.z) < T(0)) {
        d = dL * xpow(pm / pL, g.inv_g); u = um; ps = pm;
      } else {
        const T a = g.two_gp1 * (aL + g.half_gm1 * uL);
        d = dL * xpow(a / aL, g.fan_d); u = a; ps = pL * xpow(a / aL, g.fan_p);
      }
    } else {
      const T sL = uL - aL * xsqrt(g.sh_a * pm / pL + g.sh_b);
      if (sL >= T(0)) {
        d = dL; u = uL; ps = pL;
      } else {
        d = dL * (pm / pL + g.gm1_gp1) / (pm / pL * g.gm1_gp1 + T(1));
        u = um; ps = pm;
      }
    }
  } else {
    if (pm <= pR) {
      if (uR + aR <= T(0)) {
        d = dR; u = uR; ps = pR;
      } else if (um + aR * xpow(pm / pR, g.z) >= T(0)) {
        d = dR * xpow(pm / pR, g.inv_g); u = um; ps = pm;
      } else {
        const T a = g.two_gp1 * (aR - g.half_gm1 * uR);
        d = dR * xpow(a / aR, g.fan_d); u = -a; ps = pR * xpow(a / aR, g.fan_p);
      }
    } else {
      const T sR = uR + aR * xsqrt(g.sh_a * pm / pR + g.sh_b);
      if (sR <= T(0)) {
        d = dR; u = uR; ps = pR;
      } else {
        d = dR * (pm / pR + g.gm1_gp1) / (pm / pR * g.gm1_gp1 + T(1));
        u = um; ps = pm;
      }
    }
  }
  const bool left = u >= T(0);
  const T v = left ? WL[2] : WR[2];
  const T w = left ? WL[3] : WR[3];
  const T E = ps / g.gm1 + T(0.5) * d * (u * u + v * v + w * w);
  const T mf = d * u;
  F[0] = mf;
  F[1] = mf * u + ps;
  F[2] = mf * v;
  F[3] = mf * w;
  F[4] = (E + ps) * u;
  return flags;
}

}  // namespace hydro
