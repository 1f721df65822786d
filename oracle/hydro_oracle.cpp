// hydro_oracle.cpp -- TEST INFRASTRUCTURE, NOT PART OF THE PRODUCT PATH.
//
// Plain, slow CPU reference ("oracle") for one unsplit six-solve CTU step of the
// 3D Euler equations (Schneider & Robertson, "Cholla", Sec. 2.3, Eqs.
// simple_conserved_update / transverse_evolution / conserved_update), with PPMC
// reconstruction (App. A.3, slopes from App. A.2) and the exact Riemann solver of
// Toro ch. 4 as the paper gives it (App. B.1).  Everything is FP64 and follows
// the paper's steps in the paper's order and notation: every intermediate of the
// method (cell primitives w, face states U*, first fluxes F*, CTU fluxes
// F^{n+1/2}) is a full-grid array, nothing is fused, blocked or reordered.
//
// Only the test suite, the smoke check and the benchmark's CPU-baseline leg load
// this library.  It shares no source, header, table or helper with the CUDA path.
//
// Build: g++ -std=c++17 -O2 -ffp-contract=off -fopenmp -shared -fPIC.  No
// fast-math, no fused multiply-add: every operation is one IEEE round-to-nearest
// operation; divisions and square roots are correctly rounded, pow is libm's.
//
// Readings of the paper adopted here (each is a reading, not a printed fact):
//  * ghost depth NG = 4 per active side; PPMC needs 3 (App. A.3 stencil).
//  * transmissive boundary = every ghost copies the outermost real cell; reflective
//    = mirror copy with the normal momentum negated (Sec. 3.1); inflow = a fixed
//    prescribed primitive state; ghosts are filled x, then y, then z, each pass
//    over the already-filled ghosts of earlier axes (this fills edges and corners
//    the way the x->y->z exchange of Sec. 3.5.2 does).
//  * Noh boundary (Sec. 4.3.1, outer faces of the octant): a ghost cell takes the
//    analytic solution at the start of the step, time t, at its own centre x
//    (r = |x| over the active axes, n of them): rho = rho0 (1 + V t / r)^(n-1),
//    velocity V toward the origin, E = p0/(gamma-1) + rho V^2 / 2 (the printed
//    energy with V = 1); rho0, V, p0 are the face's prescribed state
//    (rho0, V, -, -, p0); t starts at 0 and advances by each step's dt.
//  * dt is taken from the state at the start of the step over real cells and
//    active axes (Eq. calc_dt_3D); an axis with one cell is inactive (no ghosts,
//    no sweep, no transverse term), so the step reduces to 2D/1D CTU (Sec. 2.3).
//  * the 1e-20 pressure floor (Sec. 2.4.1) applies to every derived pressure: cell
//    primitives, the PPMC face states, the states fed to each Riemann solve and
//    each Newton iterate.  Stored conserved variables are never modified.
//  * PLMC projection: xi0 = 0.5(-rho du/a + dp/a^2) (the printed sign of the rho
//    du/a term makes projection followed by back-projection lose dp; App. A.2).
//  * PPMC: w6 = 6 w_i - 3 (W_L + W_R) (the cell mean of the parabola is w_i);
//    B uses alpha^m in its first bracket and D uses the "beta" form with minus
//    signs in both brackets, so that E, B, C, D are differences of the traced
//    states W^k (App. A.3).  Slopes of cells i-1, i, i+1 use each cell's own rho
//    and a and are not clipped to the neighbours (PPMC step one).
//  * MC limiter: zero unless xi_L xi_R > 0, sgn(0) = +1 (App. A.1).
//  * Newton: tolerance 1e-6, at most 50 iterations (cap sets a status flag and
//    keeps the last iterate); an iterate below the floor is raised to it; u^m uses
//    f_L, f_R evaluated at the final p^m.
//  * Right-hand rarefaction fan: a = 2/(gamma+1) (a_R - (gamma-1) u_R / 2), u = -a
//    (the printed "+" breaks continuity at the fan head u_R + a_R = 0); the right
//    shock speed is s_R (printed "s_LR").
//  * Interface energy: E = p/(gamma-1) + rho (u^2 + v_k^2 + w_k^2)/2; transverse
//    velocities are taken from the left state when the sampled u >= 0.
//  * Velocity order of a sweep is cyclic: x (u,v,w), y (v,w,u), z (w,u,v); the
//    transverse terms of an x face are added y then z, of a y face z then x, of a
//    z face x then y; the update adds the x, then y, then z flux differences.

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <limits>
#include <vector>
#ifdef _OPENMP
#include <omp.h>
#endif

namespace {

constexpr int NG = 4;
constexpr double P_FLOOR = 1e-20;
constexpr double P0_FLOOR = 1e-6;
constexpr double NEWTON_TOL = 1e-6;
constexpr int NEWTON_MAX = 50;

enum : int { FLAG_NEWTON = 1, FLAG_NONPHYS = 2 };
enum : int { BC_PERIODIC = 0, BC_REFLECT = 1, BC_OUTFLOW = 2, BC_INFLOW = 3, BC_NOH = 4 };

// ---------------------------------------------------------------------------
// Operation-counting scalar.  The same templated code runs on `double` (the
// oracle proper) and on `CR` (a double that counts each arithmetic operation) so
// that the algorithmic FP64 operation count per cell update can be measured on
// any workload.  Counting runs single-threaded.
struct OpCount {
  uint64_t add = 0, mul = 0, div = 0, sqrt = 0, pow = 0, cmp = 0;
};
OpCount g_ops;
// Counts are also kept per stage of the step: 0 primitives and dt, 1 PPMC
// (without its slopes), 2 first Riemann solves, 3 transverse half-step and
// second Riemann solves, 4 conserved update, 5 limited slopes.  g_units holds
// the number of cells or faces each stage processed.
constexpr int kStages = 6;
OpCount g_stage_ops[kStages];
uint64_t g_units[kStages];
int g_stage = 0;

struct CR {
  double v;
  CR() : v(0.0) {}
  CR(double x) : v(x) {}
};
#define ORACLE_COUNT(field) (++g_ops.field, ++g_stage_ops[g_stage].field)
inline CR operator+(CR a, CR b) { ORACLE_COUNT(add); return CR(a.v + b.v); }
inline CR operator-(CR a, CR b) { ORACLE_COUNT(add); return CR(a.v - b.v); }
inline CR operator-(CR a) { return CR(-a.v); }
inline CR operator*(CR a, CR b) { ORACLE_COUNT(mul); return CR(a.v * b.v); }
inline CR operator/(CR a, CR b) { ORACLE_COUNT(div); return CR(a.v / b.v); }
inline bool operator<(CR a, CR b) { ORACLE_COUNT(cmp); return a.v < b.v; }
inline bool operator>(CR a, CR b) { ORACLE_COUNT(cmp); return a.v > b.v; }
inline bool operator<=(CR a, CR b) { ORACLE_COUNT(cmp); return a.v <= b.v; }
inline bool operator>=(CR a, CR b) { ORACLE_COUNT(cmp); return a.v >= b.v; }
inline CR sqrt(CR a) { ORACLE_COUNT(sqrt); return CR(std::sqrt(a.v)); }
inline CR pow(CR a, CR b) { ORACLE_COUNT(pow); return CR(std::pow(a.v, b.v)); }
inline CR fabs(CR a) { ORACLE_COUNT(cmp); return CR(std::fabs(a.v)); }
#undef ORACLE_COUNT

// stage bookkeeping; does nothing for the plain double oracle
inline void set_stage(double*, int) {}
inline void set_stage(CR*, int s) { g_stage = s; }
inline void add_units(double*, int) {}
inline void add_units(CR*, int s) { ++g_units[s]; }
inline double val(CR a) { return a.v; }
inline double val(double a) { return a; }
// the double overloads sit beside the counted ones so that templated code picks
// the exact match for R = double
using std::fabs;
using std::pow;
using std::sqrt;

template <class R> inline R mn(R a, R b) { return (b < a) ? b : a; }
template <class R> inline R mx(R a, R b) { return (a < b) ? b : a; }
// sgn(x) = -1 for x < 0, else +1 (App. A.1)
template <class R> inline R sgn(R x) { return (x < R(0.0)) ? R(-1.0) : R(1.0); }

// Constants that depend on gamma only (computed once, not per operation).
struct Gas {
  double gamma, gm1, gp1;
  double z;        // (gamma-1)/(2 gamma), rarefaction exponent
  double zd;       // -(gamma+1)/(2 gamma), exponent of f' on a rarefaction
  double inv_g;    // 1/gamma
  double g_fan_d;  // 2/(gamma-1)
  double g_fan_p;  // 2 gamma/(gamma-1)
  double two_gp1;  // 2/(gamma+1)
  double half_gm1; // (gamma-1)/2
  double sh_a;     // (gamma+1)/(2 gamma)
  double sh_b;     // (gamma-1)/(2 gamma)
  double gm1_gp1;  // (gamma-1)/(gamma+1)
  explicit Gas(double g) {
    gamma = g; gm1 = g - 1.0; gp1 = g + 1.0;
    z = (g - 1.0) / (2.0 * g);
    zd = -(g + 1.0) / (2.0 * g);
    inv_g = 1.0 / g;
    g_fan_d = 2.0 / (g - 1.0);
    g_fan_p = 2.0 * g / (g - 1.0);
    two_gp1 = 2.0 / (g + 1.0);
    half_gm1 = (g - 1.0) / 2.0;
    sh_a = (g + 1.0) / (2.0 * g);
    sh_b = (g - 1.0) / (2.0 * g);
    gm1_gp1 = (g - 1.0) / (g + 1.0);
  }
};

// Velocity order of a sweep along axis d: (normal, t1, t2) as global components.
constexpr int PERM[3][3] = {{0, 1, 2}, {1, 2, 0}, {2, 0, 1}};

// ---------------------------------------------------------------------------
// Conserved <-> primitive (Sec. 2.1: u = [rho, rho u, rho v, rho w, E],
// w = [rho, u, v, w, p], p = (gamma-1) rho e, E = rho (V^2/2 + e)).  Vectors are in
// the sweep's rotated order (rho, normal, t1, t2, energy-or-pressure).
template <class R>
void cons_to_prim(const R U[5], const Gas& g, R W[5]) {
  const R d = U[0];
  const R u = U[1] / d, v = U[2] / d, w = U[3] / d;
  R p = R(g.gm1) * (U[4] - R(0.5) * d * (u * u + v * v + w * w));
  W[0] = d; W[1] = u; W[2] = v; W[3] = w;
  W[4] = mx(p, R(P_FLOOR));
}

template <class R>
void prim_to_cons(const R W[5], const Gas& g, R U[5]) {
  const R d = W[0], u = W[1], v = W[2], w = W[3], p = W[4];
  U[0] = d; U[1] = d * u; U[2] = d * v; U[3] = d * w;
  U[4] = p / R(g.gm1) + R(0.5) * d * (u * u + v * v + w * w);
}

// ---------------------------------------------------------------------------
// Exact Riemann solver (App. B.1, after Toro ch. 4).
template <class R>
struct RiemannResult {
  R F[5];    // flux, rotated order
  R pm, um;  // star pressure and velocity
  R ws[5];   // sampled primitive state at x/t = 0 (rotated order)
  int iters;
  int flags;
};

// Pressure function f_k and its derivative (Eq. pressure_functions and the
// derivative that follows it).
template <class R>
void pressure_function(R p, R dk, R pk, R ak, R Ak, R Bk, const Gas& g, R& f, R& fd) {
  if (p <= pk) {  // rarefaction
    const R ratio = p / pk;
    f = R(2.0) * ak / R(g.gm1) * (pow(ratio, R(g.z)) - R(1.0));
    fd = R(1.0) / (dk * ak) * pow(ratio, R(g.zd));
  } else {        // shock
    const R q = sqrt(Ak / (p + Bk));
    f = (p - pk) * q;
    fd = q * (R(1.0) - (p - pk) / (R(2.0) * (Bk + p)));
  }
}

template <class R>
void riemann_exact_prim(const R WL[5], const R WR[5], const Gas& g, RiemannResult<R>& out) {
  const R dL = WL[0], uL = WL[1], pL = WL[4];
  const R dR = WR[0], uR = WR[1], pR = WR[4];
  out.flags = 0;
  // sound speeds
  const R aL = sqrt(R(g.gamma) * pL / dL);
  const R aR = sqrt(R(g.gamma) * pR / dR);
  // primitive-variable (PVRS) estimate, not below zero
  R pt = R(0.5) * (pL + pR) + R(0.125) * (uL - uR) * (dL + dR) * (aL + aR);
  if (pt < R(0.0)) pt = R(0.0);
  // two-shock estimate p0, floored at 1e-6
  const R AL = R(2.0) / (R(g.gp1) * dL), AR = R(2.0) / (R(g.gp1) * dR);
  const R BL = R(g.gm1_gp1) * pL, BR = R(g.gm1_gp1) * pR;
  const R gL = sqrt(AL / (pt + BL)), gR = sqrt(AR / (pt + BR));
  R p0 = (gL * pL + gR * pR - (uR - uL)) / (gL + gR);
  if (p0 < R(P0_FLOOR)) p0 = R(P0_FLOOR);
  // Newton-Raphson iteration on f_L + f_R + u_R - u_L = 0
  R p = p0, fL, fR, dfL, dfR;
  int it = 0;
  bool converged = false;
  while (it < NEWTON_MAX) {
    pressure_function(p, dL, pL, aL, AL, BL, g, fL, dfL);
    pressure_function(p, dR, pR, aR, AR, BR, g, fR, dfR);
    R pn = p - (fL + fR + uR - uL) / (dfL + dfR);
    if (pn < R(P_FLOOR)) pn = R(P_FLOOR);
    const R delta = R(2.0) * fabs(pn - p) / fabs(pn + p);
    p = pn;
    ++it;
    if (delta < R(NEWTON_TOL)) { converged = true; break; }
  }
  if (!converged) out.flags |= FLAG_NEWTON;
  out.iters = it;
  // star velocity from the pressure functions at the final p^m
  pressure_function(p, dL, pL, aL, AL, BL, g, fL, dfL);
  pressure_function(p, dR, pR, aR, AR, BR, g, fR, dfR);
  const R pm = p;
  const R um = R(0.5) * (uL + uR + fR - fL);
  out.pm = pm;
  out.um = um;

  // sample the solution at the interface (ten cases)
  R d, u, pp;
  if (um >= R(0.0)) {
    if (pm <= pL) {  // left rarefaction
      if (uL - aL >= R(0.0)) {
        d = dL; u = uL; pp = pL;
      } else if (um - aL * pow(pm / pL, R(g.z)) < R(0.0)) {
        d = dL * pow(pm / pL, R(g.inv_g)); u = um; pp = pm;
      } else {
        const R a = R(g.two_gp1) * (aL + R(g.half_gm1) * uL);
        d = dL * pow(a / aL, R(g.g_fan_d)); u = a; pp = pL * pow(a / aL, R(g.g_fan_p));
      }
    } else {          // left shock
      const R sL = uL - aL * sqrt(R(g.sh_a) * pm / pL + R(g.sh_b));
      if (sL >= R(0.0)) {
        d = dL; u = uL; pp = pL;
      } else {
        d = dL * (pm / pL + R(g.gm1_gp1)) / (pm / pL * R(g.gm1_gp1) + R(1.0));
        u = um; pp = pm;
      }
    }
  } else {
    if (pm <= pR) {  // right rarefaction
      if (uR + aR <= R(0.0)) {
        d = dR; u = uR; pp = pR;
      } else if (um + aR * pow(pm / pR, R(g.z)) >= R(0.0)) {
        d = dR * pow(pm / pR, R(g.inv_g)); u = um; pp = pm;
      } else {
        const R a = R(g.two_gp1) * (aR - R(g.half_gm1) * uR);
        d = dR * pow(a / aR, R(g.g_fan_d)); u = -a; pp = pR * pow(a / aR, R(g.g_fan_p));
      }
    } else {          // right shock
      const R sR = uR + aR * sqrt(R(g.sh_a) * pm / pR + R(g.sh_b));
      if (sR <= R(0.0)) {
        d = dR; u = uR; pp = pR;
      } else {
        d = dR * (pm / pR + R(g.gm1_gp1)) / (pm / pR * R(g.gm1_gp1) + R(1.0));
        u = um; pp = pm;
      }
    }
  }
  // transverse velocities are advected: left state if u >= 0, else right
  const R v = (u >= R(0.0)) ? WL[2] : WR[2];
  const R w = (u >= R(0.0)) ? WL[3] : WR[3];
  out.ws[0] = d; out.ws[1] = u; out.ws[2] = v; out.ws[3] = w; out.ws[4] = pp;
  // flux (Eq. x_flux with E = p/(gamma-1) + rho V^2/2)
  const R E = pp / R(g.gm1) + R(0.5) * d * (u * u + v * v + w * w);
  const R mflux = d * u;
  out.F[0] = mflux;
  out.F[1] = mflux * u + pp;
  out.F[2] = mflux * v;
  out.F[3] = mflux * w;
  out.F[4] = (E + pp) * u;
}

template <class R>
int riemann_exact_cons(const R UL[5], const R UR[5], const Gas& g, R F[5]) {
  R WL[5], WR[5];
  cons_to_prim(UL, g, WL);
  cons_to_prim(UR, g, WR);
  RiemannResult<R> res;
  riemann_exact_prim(WL, WR, g, res);
  for (int q = 0; q < 5; ++q) F[q] = res.F[q];
  return res.flags;
}

// ---------------------------------------------------------------------------
// PLMC slope of one cell (App. A.2: differences, characteristic projection with the
// cell's own rho and a, MC limiter on each characteristic, back-projection).
template <class R>
void project(const R dv[5], R d, R a, R x[5]) {
  x[0] = R(0.5) * (-(d * dv[1]) / a + dv[4] / (a * a));
  x[1] = dv[0] - dv[4] / (a * a);
  x[2] = dv[2];
  x[3] = dv[3];
  x[4] = R(0.5) * (d * dv[1] / a + dv[4] / (a * a));
}

template <class R>
void plmc_slope(const R wm[5], const R wc[5], const R wp[5], const Gas& g, R dw[5]) {
  const R d = wc[0];
  const R a = sqrt(R(g.gamma) * wc[4] / d);
  R dL[5], dR[5], dC[5];
  for (int q = 0; q < 5; ++q) {
    dL[q] = wc[q] - wm[q];
    dR[q] = wp[q] - wc[q];
    dC[q] = R(0.5) * (wp[q] - wm[q]);
  }
  R xL[5], xR[5], xC[5], xi[5];
  project(dL, d, a, xL);
  project(dR, d, a, xR);
  project(dC, d, a, xC);
  for (int q = 0; q < 5; ++q) {
    if (xL[q] * xR[q] > R(0.0)) {
      const R lim = mn(mn(fabs(xC[q]), R(2.0) * fabs(xL[q])), R(2.0) * fabs(xR[q]));
      xi[q] = sgn(xC[q]) * lim;
    } else {
      xi[q] = R(0.0);
    }
  }
  dw[0] = xi[0] + xi[1] + xi[4];
  dw[1] = a / d * (-xi[0] + xi[4]);
  dw[2] = xi[2];
  dw[3] = xi[3];
  dw[4] = a * a * (xi[0] + xi[4]);
}

// PPMC for cell i (App. A.3).  w[0..4] are the primitive states of cells
// i-2..i+2 in rotated order; dtdx = dt/dx along the sweep.  Returns the
// time-evolved left-face state W*_L and right-face state W*_R of cell i.
template <class R>
void ppmc_cell(const R (*w)[5], R dtdx, const Gas& g, R WsL[5], R WsR[5]) {
  R dwm[5], dwc[5], dwp[5];
  set_stage((R*)nullptr, 5);
  plmc_slope(w[0], w[1], w[2], g, dwm);  // cell i-1
  plmc_slope(w[1], w[2], w[3], g, dwc);  // cell i
  plmc_slope(w[2], w[3], w[4], g, dwp);  // cell i+1
  for (int k = 0; k < 3; ++k) add_units((R*)nullptr, 5);
  set_stage((R*)nullptr, 1);
  const R* wim = w[1];
  const R* wi = w[2];
  const R* wip = w[3];

  R WL[5], WR[5], dw[5], w6[5];
  for (int q = 0; q < 5; ++q) {
    // parabolic interpolation (Eq. parabolic_interpolation)
    R L = R(0.5) * (wi[q] + wim[q]) - (dwc[q] - dwm[q]) / R(6.0);
    R Rr = R(0.5) * (wip[q] + wi[q]) - (dwp[q] - dwc[q]) / R(6.0);
    // local extremum (Eq. max_min)
    if ((Rr - wi[q]) * (wi[q] - L) <= R(0.0)) { L = wi[q]; Rr = wi[q]; }
    // steep gradients (Eq. steep_gradient), in the printed order
    if ((Rr - L) * (L - (R(3.0) * wi[q] - R(2.0) * Rr)) < R(0.0)) L = R(3.0) * wi[q] - R(2.0) * Rr;
    if ((Rr - L) * ((R(3.0) * wi[q] - R(2.0) * L) - Rr) < R(0.0)) Rr = R(3.0) * wi[q] - R(2.0) * L;
    // bound by the neighbouring averages
    L = mn(mx(wi[q], wim[q]), mx(mn(wi[q], wim[q]), L));
    Rr = mn(mx(wi[q], wip[q]), mx(mn(wi[q], wip[q]), Rr));
    WL[q] = L;
    WR[q] = Rr;
    dw[q] = Rr - L;
    w6[q] = R(6.0) * wi[q] - R(3.0) * (L + Rr);
  }

  // characteristic speeds of cell i and the CW84 Courant fractions
  const R d = wi[0];
  const R a = sqrt(R(g.gamma) * wi[4] / d);
  const R u = wi[1];
  const R lm = u - a, l0 = u, lp = u + a;
  const R am = dtdx * mn(lm, R(0.0)), a0 = dtdx * mn(l0, R(0.0)), ap = dtdx * mn(lp, R(0.0));
  const R bm = dtdx * mx(lm, R(0.0)), b0 = dtdx * mx(l0, R(0.0)), bp = dtdx * mx(lp, R(0.0));
  const R two3 = R(2.0 / 3.0);

  R TL_m[5], TL_0[5], TL_p[5], TR_m[5], TR_0[5], TR_p[5];
  for (int q = 0; q < 5; ++q) {
    // integral under the parabola over the domain of dependence of each wave
    TL_m[q] = R(0.5) * am * (dw[q] + w6[q] * (R(1.0) + two3 * am));
    TL_0[q] = R(0.5) * a0 * (dw[q] + w6[q] * (R(1.0) + two3 * a0));
    TL_p[q] = R(0.5) * ap * (dw[q] + w6[q] * (R(1.0) + two3 * ap));
    TR_m[q] = R(0.5) * bm * (dw[q] - w6[q] * (R(1.0) - two3 * bm));
    TR_0[q] = R(0.5) * b0 * (dw[q] - w6[q] * (R(1.0) - two3 * b0));
    TR_p[q] = R(0.5) * bp * (dw[q] - w6[q] * (R(1.0) - two3 * bp));
  }
  R WtL[5], WtR[5], E[5], B[5], C[5], D[5];
  for (int q = 0; q < 5; ++q) {
    WtL[q] = WL[q] - TL_m[q];  // Eq. integration_PPMC
    WtR[q] = WR[q] - TR_p[q];
    E[q] = TL_m[q] - TL_0[q];
    B[q] = TL_m[q] - TL_p[q];
    C[q] = TR_p[q] - TR_m[q];
    D[q] = TR_p[q] - TR_0[q];
  }
  const R a2 = a * a;
  R sL[5] = {R(0.0), R(0.0), R(0.0), R(0.0), R(0.0)};
  R sR[5] = {R(0.0), R(0.0), R(0.0), R(0.0), R(0.0)};
  if (l0 < R(0.0)) {  // contact (and advected transverse velocities)
    sL[0] = sL[0] + (E[0] - E[4] / a2);
    sL[2] = sL[2] + E[2];
    sL[3] = sL[3] + E[3];
  }
  if (lp < R(0.0)) {  // right-moving acoustic wave reaching the left face
    sL[0] = sL[0] + R(0.5) * (d * B[1] / a + B[4] / a2);
    sL[1] = sL[1] + R(0.5) * (B[1] + B[4] / (a * d));
    sL[4] = sL[4] + R(0.5) * (d * B[1] * a + B[4]);
  }
  if (lm > R(0.0)) {  // left-moving acoustic wave reaching the right face
    sR[0] = sR[0] + R(0.5) * (-(d * C[1]) / a + C[4] / a2);
    sR[1] = sR[1] + R(0.5) * (C[1] - C[4] / (a * d));
    sR[4] = sR[4] + R(0.5) * (-(d * C[1] * a) + C[4]);
  }
  if (l0 > R(0.0)) {  // contact (and advected transverse velocities)
    sR[0] = sR[0] + (D[0] - D[4] / a2);
    sR[2] = sR[2] + D[2];
    sR[3] = sR[3] + D[3];
  }
  for (int q = 0; q < 5; ++q) {
    WsL[q] = WtL[q] + sL[q];
    WsR[q] = WtR[q] + sR[q];
  }
  WsL[4] = mx(WsL[4], R(P_FLOOR));
  WsR[4] = mx(WsR[4], R(P_FLOOR));
}

// ---------------------------------------------------------------------------
// The other reconstructions of App. A and Sec. 2.2.1.  Stencils are in rotated
// order (rho, normal velocity, two transverse velocities, p).

// primitive-variable slope of one cell: left, right and centred differences
// (Eq. diffs) and the MC limiter (Eq. vanLeer_limiter), each variable alone
template <class R>
void plm_prim_slope(const R wm[5], const R wc[5], const R wp[5], R dw[5]) {
  for (int q = 0; q < 5; ++q) {
    const R dL = wc[q] - wm[q];
    const R dR = wp[q] - wc[q];
    const R dC = R(0.5) * (wp[q] - wm[q]);
    if (dL * dR > R(0.0))
      dw[q] = sgn(dC) * mn(mn(fabs(dC), R(2.0) * fabs(dL)), R(2.0) * fabs(dR));
    else
      dw[q] = R(0.0);
  }
}

// Euler flux along the sweep of a primitive state (Eq. x_flux)
template <class R>
void euler_flux(const R W[5], const Gas& g, R F[5]) {
  const R E = W[4] / R(g.gm1) + R(0.5) * W[0] * (W[1] * W[1] + W[2] * W[2] + W[3] * W[3]);
  const R m = W[0] * W[1];
  F[0] = m;
  F[1] = m * W[1] + W[4];
  F[2] = m * W[2];
  F[3] = m * W[3];
  F[4] = (E + W[4]) * W[1];
}

// PLMP (App. A.1): boundary values from the limited primitive slopes
// (W_L = w - dw/2, W_R = w + dw/2), converted to conserved variables and evolved
// half a step with the fluxes of the two boundary values (Eqs.
// plmp_evolution_L, plmp_evolution_R).  w[0..2]: cells i-1, i, i+1.
template <class R>
void plmp_cell(const R w[3][5], R dtdx, const Gas& g, R UsL[5], R UsR[5]) {
  R dw[5], WL[5], WR[5];
  set_stage((R*)nullptr, 5);
  add_units((R*)nullptr, 5);
  plm_prim_slope(w[0], w[1], w[2], dw);
  set_stage((R*)nullptr, 1);
  for (int q = 0; q < 5; ++q) {
    WL[q] = w[1][q] - R(0.5) * dw[q];
    WR[q] = w[1][q] + R(0.5) * dw[q];
  }
  WL[4] = mx(WL[4], R(P_FLOOR));
  WR[4] = mx(WR[4], R(P_FLOOR));
  R UL[5], UR[5], FL[5], FR[5];
  prim_to_cons(WL, g, UL);
  prim_to_cons(WR, g, UR);
  euler_flux(WL, g, FL);
  euler_flux(WR, g, FR);
  const R h = R(0.5) * dtdx;
  for (int q = 0; q < 5; ++q) {
    UsL[q] = UL[q] + h * (FL[q] - FR[q]);
    UsR[q] = UR[q] + h * (FL[q] - FR[q]);
  }
}

// PLMC (App. A.2): characteristic-limited slope (plmc_slope), boundary values
// W_{L,A}, W_{R,A} (Eq. plm_interpolation) bounded by the neighbouring averages,
// the slope recomputed as W_R - W_L, integration under the linear profile over
// the fastest wave's domain of dependence, and the corrections s_L, s_R for the
// other waves moving toward each face.  w[0..2]: cells i-1, i, i+1.
template <class R>
void plmc_cell(const R w[3][5], R dtdx, const Gas& g, R WsL[5], R WsR[5]) {
  R dw[5];
  set_stage((R*)nullptr, 5);
  add_units((R*)nullptr, 5);
  plmc_slope(w[0], w[1], w[2], g, dw);
  set_stage((R*)nullptr, 1);
  const R* wim = w[0];
  const R* wi = w[1];
  const R* wip = w[2];
  R WL[5], WR[5];
  for (int q = 0; q < 5; ++q) {
    const R LA = wi[q] - R(0.5) * dw[q];
    const R RA = wi[q] + R(0.5) * dw[q];
    const R LB = mx(mn(wi[q], wim[q]), LA);
    WL[q] = mn(mx(wi[q], wim[q]), LB);
    const R RB = mx(mn(wi[q], wip[q]), RA);
    WR[q] = mn(mx(wi[q], wip[q]), RB);
    dw[q] = WR[q] - WL[q];
  }
  const R d = wi[0];
  const R a = sqrt(R(g.gamma) * wi[4] / d);
  const R u = wi[1];
  const R lm = u - a, l0 = u, lp = u + a;
  const R a2 = a * a;
  R sL[5] = {R(0.0), R(0.0), R(0.0), R(0.0), R(0.0)};
  R sR[5] = {R(0.0), R(0.0), R(0.0), R(0.0), R(0.0)};
  if (l0 < R(0.0)) {  // contact (and advected transverse velocities)
    sL[0] = sL[0] + (lm - l0) * (dw[0] - dw[4] / a2);
    sL[2] = sL[2] + (lm - l0) * dw[2];
    sL[3] = sL[3] + (lm - l0) * dw[3];
  }
  if (lp < R(0.0)) {  // right acoustic wave
    sL[0] = sL[0] + R(0.5) * (lm - lp) * (d * dw[1] / a + dw[4] / a2);
    sL[1] = sL[1] + R(0.5) * (lm - lp) * (dw[1] + dw[4] / (a * d));
    sL[4] = sL[4] + R(0.5) * (lm - lp) * (d * dw[1] * a + dw[4]);
  }
  if (lm > R(0.0)) {  // left acoustic wave
    sR[0] = sR[0] + R(0.5) * (lp - lm) * (-(d * dw[1]) / a + dw[4] / a2);
    sR[1] = sR[1] + R(0.5) * (lp - lm) * (dw[1] - dw[4] / (a * d));
    sR[4] = sR[4] + R(0.5) * (lp - lm) * (-(d * dw[1] * a) + dw[4]);
  }
  if (l0 > R(0.0)) {  // contact (and advected transverse velocities)
    sR[0] = sR[0] + (lp - l0) * (dw[0] - dw[4] / a2);
    sR[2] = sR[2] + (lp - l0) * dw[2];
    sR[3] = sR[3] + (lp - l0) * dw[3];
  }
  const R am = dtdx * mn(lm, R(0.0)), bp = dtdx * mx(lp, R(0.0));
  const R h = R(0.5) * dtdx;
  for (int q = 0; q < 5; ++q) {
    WsL[q] = (WL[q] - R(0.5) * am * dw[q]) + h * sL[q];
    WsR[q] = (WR[q] - R(0.5) * bp * dw[q]) + h * sR[q];
  }
  WsL[4] = mx(WsL[4], R(P_FLOOR));
  WsR[4] = mx(WsR[4], R(P_FLOOR));
}

// flattening coefficient F~_k of cell k from p_{k-2..k+2} and the normal
// velocities u_{k-1}, u_{k+1} (App. A.4, shock flattening).  The two conditions
// that zero F~ are tested first, so the steepness ratio is only formed across a
// pressure jump of at least a third (its denominator may still vanish, which
// gives an infinite ratio and F~ = 0 or 1 by its sign).
template <class R>
R flatten_tilde(const R p[5], R um, R up) {
  const R jump = fabs(p[3] - p[1]) / mn(p[3], p[1]);
  if (jump < R(1.0 / 3.0) || up - um > R(0.0)) return R(0.0);
  const R S = (p[3] - p[1]) / (p[4] - p[0]);
  return mx(R(0.0), mn(R(1.0), R(10.0) * (S - R(0.75))));
}

// PPMP for cell i (App. A.4).  w[0..6] are the primitive states of cells
// i-3..i+3 in rotated order; dtdx = dt/dx along the sweep; dx the cell width.
// Steps in the paper's order: parabolic interpolation with MC-limited
// primitive slopes, contact steepening of the density, shock flattening,
// monotonicity, the integrals under the parabola for the three
// characteristics, reference states and the corrections chi.
template <class R>
void ppmp_cell(const R w[7][5], R dtdx, R dx, const Gas& g, R WsL[5], R WsR[5]) {
  R dwm[5], dwc[5], dwp[5];
  set_stage((R*)nullptr, 5);
  plm_prim_slope(w[1], w[2], w[3], dwm);  // cell i-1
  plm_prim_slope(w[2], w[3], w[4], dwc);  // cell i
  plm_prim_slope(w[3], w[4], w[5], dwp);  // cell i+1
  for (int k = 0; k < 3; ++k) add_units((R*)nullptr, 5);
  set_stage((R*)nullptr, 1);
  const R* wim = w[2];
  const R* wi = w[3];
  const R* wip = w[4];
  R WL[5], WR[5];
  for (int q = 0; q < 5; ++q) {  // parabolic interpolation
    WL[q] = R(0.5) * (wi[q] + wim[q]) - (dwc[q] - dwm[q]) / R(6.0);
    WR[q] = R(0.5) * (wip[q] + wi[q]) - (dwp[q] - dwc[q]) / R(6.0);
  }
  // contact discontinuity steepening of the density
  {
    const R rjump = fabs(wip[0] - wim[0]) / mn(wip[0], wim[0]);
    const R pjump = fabs(wip[4] - wim[4]) / mn(wip[4], wim[4]);
    const R dx2 = dx * dx;
    const R d2m = (wi[0] - R(2.0) * wim[0] + w[1][0]) / (R(6.0) * dx2);   // cell i-1
    const R d2p = (w[5][0] - R(2.0) * wip[0] + wi[0]) / (R(6.0) * dx2);  // cell i+1
    // the concavity test: d2m d2p < 0 (opposite curvature on the two sides, the
    // inflection of a smeared contact), as in the method the paper follows
    // (CW84, FLASH); the printed "> 0 (same concavity)" disables steepening of
    // smeared contacts and contradicts the paper's own Sod result (contact over
    // two zones with PPMP, three to four with PPMC, Sec. 4.1.1)
    if (rjump > R(0.01) && pjump < R(0.1) * R(g.gamma) * rjump && d2m * d2p < R(0.0)) {
      const R eta_t = -((d2p - d2m) * dx2) / (wip[0] - wim[0]);
      const R eta = mx(R(0.0), mn(R(20.0) * eta_t - R(1.0), R(1.0)));
      WL[0] = WL[0] * (R(1.0) - eta) + (wim[0] + R(0.5) * dwm[0]) * eta;
      WR[0] = WR[0] * (R(1.0) - eta) + (wip[0] - R(0.5) * dwp[0]) * eta;
    }
  }
  // shock flattening
  {
    R pm[5], pc[5], pp[5];
    for (int s = 0; s < 5; ++s) {
      pm[s] = w[s][4];
      pc[s] = w[s + 1][4];
      pp[s] = w[s + 2][4];
    }
    const R Fm = flatten_tilde(pm, w[1][1], w[3][1]);  // cell i-1
    const R Fc = flatten_tilde(pc, w[2][1], w[4][1]);  // cell i
    const R Fp = flatten_tilde(pp, w[3][1], w[5][1]);  // cell i+1
    const R F = (wip[4] - wim[4] < R(0.0)) ? mx(Fc, Fp) : mx(Fc, Fm);
    for (int q = 0; q < 5; ++q) {
      WL[q] = F * wi[q] + (R(1.0) - F) * WL[q];
      WR[q] = F * wi[q] + (R(1.0) - F) * WR[q];
    }
  }
  // monotonicity (the third rule sets W_R; the printed "W_L" is a slip)
  R dw[5], w6[5];
  for (int q = 0; q < 5; ++q) {
    R L = WL[q], Rr = WR[q];
    if ((Rr - wi[q]) * (wi[q] - L) <= R(0.0)) { L = wi[q]; Rr = wi[q]; }
    if ((Rr - L) * (L - (R(3.0) * wi[q] - R(2.0) * Rr)) < R(0.0)) L = R(3.0) * wi[q] - R(2.0) * Rr;
    if ((Rr - L) * ((R(3.0) * wi[q] - R(2.0) * L) - Rr) < R(0.0)) Rr = R(3.0) * wi[q] - R(2.0) * L;
    WL[q] = L;
    WR[q] = Rr;
    dw[q] = Rr - L;
    w6[q] = R(6.0) * (wi[q] - R(0.5) * (L + Rr));
  }
  // characteristic speeds, Courant fractions, traced boundary values
  const R d = wi[0];
  const R a = sqrt(R(g.gamma) * wi[4] / d);
  const R u = wi[1];
  const R lm = u - a, l0 = u, lp = u + a;
  const R am = dtdx * mn(lm, R(0.0)), a0 = dtdx * mn(l0, R(0.0)), ap = dtdx * mn(lp, R(0.0));
  const R bm = dtdx * mx(lm, R(0.0)), b0 = dtdx * mx(l0, R(0.0)), bp = dtdx * mx(lp, R(0.0));
  const R two3 = R(2.0 / 3.0);
  R WLm[5], WL0[5], WLp[5], WRm[5], WR0[5], WRp[5];
  for (int q = 0; q < 5; ++q) {
    WLm[q] = WL[q] - R(0.5) * am * (dw[q] + w6[q] * (R(1.0) + two3 * am));
    WL0[q] = WL[q] - R(0.5) * a0 * (dw[q] + w6[q] * (R(1.0) + two3 * a0));
    WLp[q] = WL[q] - R(0.5) * ap * (dw[q] + w6[q] * (R(1.0) + two3 * ap));
    WRm[q] = WR[q] - R(0.5) * bm * (dw[q] - w6[q] * (R(1.0) - two3 * bm));
    WR0[q] = WR[q] - R(0.5) * b0 * (dw[q] - w6[q] * (R(1.0) - two3 * b0));
    WRp[q] = WR[q] - R(0.5) * bp * (dw[q] - w6[q] * (R(1.0) - two3 * bp));
  }
  // reference states: rho, u, p from the fastest wave toward each face, the
  // transverse velocities from the advection speed; sound speeds of the
  // reference states (their pressures floored before the square root)
  const R aL = sqrt(R(g.gamma) * mx(WLm[4], R(P_FLOOR)) / WLm[0]);
  const R aR = sqrt(R(g.gamma) * mx(WRp[4], R(P_FLOOR)) / WRp[0]);
  const R CL = WLm[0] * aL;
  const R CR = WRp[0] * aR;
  // corrections (CW84): chi^p_L = -(1/(2 C_L)) [(u^m - u^p) + (p^m - p^p)/C_L]
  // (the printed "-" before the pressure term and "p^m + p^p" are slips),
  // chi^m_R with rho^p_R for the printed "rho^p_s"
  R chiLp = -(R(1.0) / (R(2.0) * CL)) * ((WLm[1] - WLp[1]) + (WLm[4] - WLp[4]) / CL);
  R chiRm = (R(1.0) / (R(2.0) * CR)) * ((WRp[1] - WRm[1]) - (WRp[4] - WRm[4]) / CR);
  R chiL0 = (WLm[4] - WL0[4]) / (CL * CL) + R(1.0) / WLm[0] - R(1.0) / WL0[0];
  R chiR0 = (WRp[4] - WR0[4]) / (CR * CR) + R(1.0) / WRp[0] - R(1.0) / WR0[0];
  if (l0 > R(0.0)) chiL0 = R(0.0);
  if (lp > R(0.0)) chiLp = R(0.0);
  if (lm < R(0.0)) chiRm = R(0.0);
  if (l0 < R(0.0)) chiR0 = R(0.0);
  WsL[0] = R(1.0) / (R(1.0) / WLm[0] - chiL0 - chiLp);
  WsL[1] = WLm[1] + CL * chiLp;
  WsL[2] = WL0[2];
  WsL[3] = WL0[3];
  WsL[4] = mx(WLm[4] + CL * CL * chiLp, R(P_FLOOR));
  WsR[0] = R(1.0) / (R(1.0) / WRp[0] - chiRm - chiR0);
  WsR[1] = WRp[1] - CR * chiRm;
  WsR[2] = WR0[2];
  WsR[3] = WR0[3];
  WsR[4] = mx(WRp[4] + CR * CR * chiRm, R(P_FLOOR));
}

// ---------------------------------------------------------------------------
// Roe solver with the HLLE fallback (Sec. 2.2.2, App. B.2) on conserved input
// states in sweep order.  etaH >= 0 is the H correction (App. C): every |lambda|
// of the Roe coefficients is replaced by max(|lambda|, etaH); 0 leaves them.
// Readings: the printed "C_3 2~" of s_3 is C_3 w~; "negative" density or
// pressure of an intermediate state means < 0; a Roe average with
// (gamma-1)(H~ - V~^2/2) <= 0 has no sound speed and takes the HLLE flux, with
// u~ for both Roe eigenvalues; HLLE bounds b^p = b^m = 0 (possible only then,
// with u~ = 0 and both states moving supersonically toward the interface, as
// cold gas at a reflecting wall) take the ratio (b^p + b^m)/(b^p - b^m) as its
// symmetric limit 0, i.e. the flux (F_L + F_R)/2 (the printed quotient is 0/0).
template <class R>
void roe_hlle_flux(const R UL[5], const R UR[5], const R WL[5], const R WR[5], const R FL[5],
                   const R FR[5], R lm, R lp, const Gas& g, R F[5]) {
  const R aL = sqrt(R(g.gamma) * WL[4] / WL[0]);
  const R aR = sqrt(R(g.gamma) * WR[4] / WR[0]);
  const R bm = mn(mn(lm, WL[1] - aL), R(0.0));
  const R bp = mx(mx(lp, WR[1] + aR), R(0.0));
  const R k = (bp - bm > R(0.0)) ? (bp + bm) / (bp - bm) : R(0.0);
  for (int q = 0; q < 5; ++q) {
    const R FLh = FL[q] - bm * UL[q];
    const R FRh = FR[q] - bp * UR[q];
    F[q] = R(0.5) * ((FLh + FRh) + (FLh - FRh) * k);
  }
}

template <class R>
bool negative_state(const R U[5], const Gas& g) {
  const R p = R(g.gm1) * (U[4] - R(0.5) * (U[1] * U[1] + U[2] * U[2] + U[3] * U[3]) / U[0]);
  return U[0] < R(0.0) || p < R(0.0);
}

template <class R>
int riemann_roe_cons(const R UL[5], const R UR[5], const Gas& g, R etaH, R F[5]) {
  R WL[5], WR[5], FL[5], FR[5];
  cons_to_prim(UL, g, WL);
  cons_to_prim(UR, g, WR);
  euler_flux(WL, g, FL);
  euler_flux(WR, g, FR);
  // Roe averages (weights sqrt(rho)); enthalpy H = (E + p)/rho
  const R sL = sqrt(WL[0]), sR = sqrt(WR[0]);
  const R HL = (UL[4] + WL[4]) / WL[0];
  const R HR = (UR[4] + WR[4]) / WR[0];
  const R u = (sL * WL[1] + sR * WR[1]) / (sL + sR);
  const R v = (sL * WL[2] + sR * WR[2]) / (sL + sR);
  const R w = (sL * WL[3] + sR * WR[3]) / (sL + sR);
  const R H = (sL * HL + sR * HR) / (sL + sR);
  const R V2 = u * u + v * v + w * w;
  const R a2 = R(g.gm1) * (H - R(0.5) * V2);
  if (!(a2 > R(0.0))) {
    roe_hlle_flux(UL, UR, WL, WR, FL, FR, u, u, g, F);
    return 0;
  }
  const R a = sqrt(a2);
  const R lm = u - a, l0 = u, lp = u + a;
  if (lm >= R(0.0)) {  // supersonic to the right
    for (int q = 0; q < 5; ++q) F[q] = FL[q];
    return 0;
  }
  if (lp <= R(0.0)) {  // supersonic to the left
    for (int q = 0; q < 5; ++q) F[q] = FR[q];
    return 0;
  }
  R dU[5];
  for (int q = 0; q < 5; ++q) dU[q] = UR[q] - UL[q];
  const R gp = R(g.gm1);
  const R Na = R(1.0) / (R(2.0) * a2);
  // wave strengths (projection on the left eigenvectors)
  const R xi0 = dU[0] * Na * (R(0.5) * gp * V2 + u * a) - dU[1] * Na * (gp * u + a) -
                dU[2] * Na * gp * v - dU[3] * Na * gp * w + dU[4] * Na * gp;
  const R xi1 = -dU[0] * v + dU[2];
  const R xi2 = -dU[0] * w + dU[3];
  const R xi3 = dU[0] * (R(1.0) - Na * gp * V2) + dU[1] * gp * u / a2 + dU[2] * gp * v / a2 +
                dU[3] * gp * w / a2 - dU[4] * gp / a2;
  const R xi4 = dU[0] * Na * (R(0.5) * gp * V2 - u * a) - dU[1] * Na * (gp * u - a) -
                dU[2] * Na * gp * v - dU[3] * Na * gp * w + dU[4] * Na * gp;
  // coefficients C = xi |lambda| (H correction: |lambda| -> max(|lambda|, etaH))
  const R alm = mx(fabs(lm), etaH), al0 = mx(fabs(l0), etaH), alp = mx(fabs(lp), etaH);
  const R C0 = xi0 * alm, C1 = xi1 * al0, C2 = xi2 * al0, C3 = xi3 * al0, C4 = xi4 * alp;
  R s[5];
  s[0] = C0 + C3 + C4;
  s[1] = C0 * (u - a) + C3 * u + C4 * (u + a);
  s[2] = C0 * v + C1 + C3 * v + C4 * v;
  s[3] = C0 * w + C2 + C3 * w + C4 * w;
  s[4] = C0 * (H - u * a) + C1 * v + C2 * w + R(0.5) * C3 * V2 + C4 * (H + u * a);
  for (int q = 0; q < 5; ++q) F[q] = R(0.5) * (FL[q] + FR[q] - s[q]);
  // intermediate states: negative density or pressure -> HLLE flux
  bool fail = false;
  R UmL[5];
  UmL[0] = UL[0] + xi0;
  UmL[1] = UL[1] + xi0 * (u - a);
  UmL[2] = UL[2] + xi0 * v;
  UmL[3] = UL[3] + xi0 * w;
  UmL[4] = UL[4] + xi0 * (H - u * a);
  if (l0 > lm && negative_state(UmL, g)) fail = true;
  if (!fail && lp > l0) {
    R UmR[5];
    UmR[0] = UmL[0] + xi3;
    UmR[1] = UmL[1] + xi3 * u;
    UmR[2] = UmL[2] + xi1 + xi3 * v;
    UmR[3] = UmL[3] + xi2 + xi3 * w;
    UmR[4] = UmL[4] + xi1 * v + xi2 * w + R(0.5) * xi3 * V2;
    if (negative_state(UmR, g)) fail = true;
  }
  if (fail) roe_hlle_flux(UL, UR, WL, WR, FL, FR, lm, lp, g, F);
  return 0;
}

// H-correction quantity of a face (App. C): half the largest jump of a
// characteristic speed between the right and the left input state,
// max(|(u_R + a_R) - (u_L + a_L)|, |(u_R - a_R) - (u_L - a_L)|) / 2.  The paper
// prints only the u + a term; the method it cites (Sanders et al. 1998) takes
// the maximum over the characteristic families, and the u + a term alone is
// not invariant under reflection (a mirrored flow would get different
// dissipation).  The jump of u is never the largest.
template <class R>
R h_eta(const R UL[5], const R UR[5], const Gas& g) {
  R WL[5], WR[5];
  cons_to_prim(UL, g, WL);
  cons_to_prim(UR, g, WR);
  const R aL = sqrt(R(g.gamma) * WL[4] / WL[0]);
  const R aR = sqrt(R(g.gamma) * WR[4] / WR[0]);
  return R(0.5) * mx(fabs((WR[1] + aR) - (WL[1] + aL)), fabs((WR[1] - aR) - (WL[1] - aL)));
}

// ---------------------------------------------------------------------------
// Reconstructions (Sec. 2.2.1): PPMC is the method of the benchmarked path.
enum { RECON_PPMC = 0, RECON_PPMP = 1, RECON_PLMC = 2, RECON_PLMP = 3, RECON_PCM = 4 };
// Riemann solvers (Sec. 2.2.2): exact (the benchmarked path) or Roe with the
// HLLE fallback and, in the second set, the H correction (App. B.2, C)
enum { SOLVER_EXACT = 0, SOLVER_ROE = 1 };

// ---------------------------------------------------------------------------
// Grid: conserved variables as five padded planes [5][N2][N1][N0], x fastest.
template <class R>
struct Grid {
  int n[3], gh[3], N[3];
  double dx, gamma;
  int bc[6];
  double inflow_prim[6][5];
  int recon = RECON_PPMC;  // reconstruction of App. A / Sec. 2.2.1
  int solver = SOLVER_EXACT;
  double time = 0.0;       // t at the start of the next step (Noh boundary)
  size_t ncell;
  std::vector<R> u;

  Grid(const int nn[3], double dx_, double gamma_, const int bc_[6]) : dx(dx_), gamma(gamma_) {
    for (int d = 0; d < 3; ++d) {
      n[d] = nn[d];
      gh[d] = (nn[d] > 1) ? NG : 0;
      N[d] = n[d] + 2 * gh[d];
    }
    for (int f = 0; f < 6; ++f) {
      bc[f] = bc_[f];
      for (int q = 0; q < 5; ++q) inflow_prim[f][q] = 0.0;
    }
    ncell = (size_t)N[0] * N[1] * N[2];
    u.assign(5 * ncell, R(0.0));
  }
  size_t idx(int i, int j, int k) const { return ((size_t)k * N[1] + j) * N[0] + i; }
  size_t stride(int d) const { return d == 0 ? 1 : (d == 1 ? (size_t)N[0] : (size_t)N[0] * N[1]); }
};

template <class R>
void fill_ghosts(Grid<R>& G) {
  const Gas g(G.gamma);
  for (int d = 0; d < 3; ++d) {
    if (G.gh[d] == 0) continue;
    // ranges: axes filled earlier cover their full padded range, later axes only real
    int lo[3], hi[3];
    for (int t = 0; t < 3; ++t) {
      if (t < d) { lo[t] = 0; hi[t] = G.N[t]; }
      else { lo[t] = G.gh[t]; hi[t] = G.gh[t] + G.n[t]; }
    }
    for (int side = 0; side < 2; ++side) {
      const int type = G.bc[2 * d + side];
      double Uin[5] = {0, 0, 0, 0, 0};
      if (type == BC_INFLOW) {
        const double* W = G.inflow_prim[2 * d + side];
        Uin[0] = W[0]; Uin[1] = W[0] * W[1]; Uin[2] = W[0] * W[2]; Uin[3] = W[0] * W[3];
        Uin[4] = W[4] / (G.gamma - 1.0) + 0.5 * W[0] * (W[1] * W[1] + W[2] * W[2] + W[3] * W[3]);
      }
      int nact = 0;
      for (int t = 0; t < 3; ++t) nact += G.n[t] > 1 ? 1 : 0;
      for (int gd = 1; gd <= G.gh[d]; ++gd) {
        const int tgt = side == 0 ? G.gh[d] - gd : G.gh[d] + G.n[d] - 1 + gd;
        int src = 0;
        switch (type) {
          case BC_PERIODIC: src = side == 0 ? G.gh[d] + G.n[d] - gd : G.gh[d] + gd - 1; break;
          case BC_REFLECT: src = side == 0 ? G.gh[d] + gd - 1 : G.gh[d] + G.n[d] - gd; break;
          case BC_OUTFLOW: src = side == 0 ? G.gh[d] : G.gh[d] + G.n[d] - 1; break;
          default: src = -1; break;
        }
        int c[3];
        for (c[2] = (d == 2 ? 0 : lo[2]); c[2] < (d == 2 ? 1 : hi[2]); ++c[2])
          for (c[1] = (d == 1 ? 0 : lo[1]); c[1] < (d == 1 ? 1 : hi[1]); ++c[1])
            for (c[0] = (d == 0 ? 0 : lo[0]); c[0] < (d == 0 ? 1 : hi[0]); ++c[0]) {
              int ct[3] = {c[0], c[1], c[2]}, cs[3] = {c[0], c[1], c[2]};
              ct[d] = tgt;
              cs[d] = src;
              const size_t it = G.idx(ct[0], ct[1], ct[2]);
              if (type == BC_NOH) {
                const double* P = G.inflow_prim[2 * d + side];
                double x[3] = {0, 0, 0}, r2 = 0.0;
                for (int t = 0; t < 3; ++t) {
                  if (G.n[t] <= 1) continue;
                  x[t] = (ct[t] - G.gh[t] + 0.5) * G.dx;
                  r2 += x[t] * x[t];
                }
                const double r = std::sqrt(r2);
                const double rho = P[0] * std::pow(1.0 + P[1] * G.time / r, nact - 1);
                G.u[it] = R(rho);
                for (int t = 0; t < 3; ++t) G.u[(1 + t) * G.ncell + it] = R(-rho * P[1] * x[t] / r);
                G.u[4 * G.ncell + it] = R(P[4] / (G.gamma - 1.0) + 0.5 * rho * P[1] * P[1]);
                continue;
              }
              for (int q = 0; q < 5; ++q) {
                if (type == BC_INFLOW) {
                  G.u[q * G.ncell + it] = R(Uin[q]);
                } else {
                  const size_t is = G.idx(cs[0], cs[1], cs[2]);
                  R val_ = G.u[q * G.ncell + is];
                  if (type == BC_REFLECT && q == 1 + d) val_ = -val_;
                  G.u[q * G.ncell + it] = val_;
                }
              }
            }
      }
    }
  }
  (void)g;
}

template <class R>
R compute_dt_min(const Grid<R>& G) {
  const Gas g(G.gamma);
  double best = std::numeric_limits<double>::infinity();
  R bestR = R(best);
  for (int k = G.gh[2]; k < G.gh[2] + G.n[2]; ++k)
    for (int j = G.gh[1]; j < G.gh[1] + G.n[1]; ++j)
      for (int i = G.gh[0]; i < G.gh[0] + G.n[0]; ++i) {
        const size_t c = G.idx(i, j, k);
        R U[5], W[5];
        for (int q = 0; q < 5; ++q) U[q] = G.u[q * G.ncell + c];
        cons_to_prim(U, g, W);
        const R a = sqrt(R(g.gamma) * W[4] / W[0]);
        for (int d = 0; d < 3; ++d) {
          if (G.n[d] <= 1) continue;
          const R t = R(G.dx) / (fabs(W[1 + d]) + a);
          if (t < bestR) bestR = t;
        }
      }
  return bestR;
}

// One CTU step with a given dt (Sec. 2.3 steps 1-5).  Returns status flags.
template <class R>
int ctu_step(Grid<R>& G, double dt_in, bool threaded) {
  const Gas g(G.gamma);
  const size_t nc = G.ncell;
  const R dt = R(dt_in);
  const R dtdx = dt / R(G.dx);
  const R hdtdx = R(0.5) * dtdx;
  int flags = 0;

  fill_ghosts(G);

  // cell-average primitives (global order) of every padded cell
  set_stage((R*)nullptr, 0);
  std::vector<R> W(5 * nc);
#pragma omp parallel for if (threaded) schedule(static)
  for (long c = 0; c < (long)nc; ++c) {
    R U[5], Wc[5];
    for (int q = 0; q < 5; ++q) U[q] = G.u[q * nc + c];
    cons_to_prim(U, g, Wc);
    for (int q = 0; q < 5; ++q) W[q * nc + c] = Wc[q];
    add_units((R*)nullptr, 0);
  }

  bool active[3];
  for (int d = 0; d < 3; ++d) active[d] = G.n[d] > 1;

  // face arrays, indexed by the padded index of the cell right of the face
  // (eta: the H-correction quantity of each face, Roe solver only)
  const bool roe = G.solver == SOLVER_ROE;
  std::vector<R> UL[3], UR[3], F1[3], F2[3], eta[3];
  for (int d = 0; d < 3; ++d) {
    if (!active[d]) continue;
    UL[d].assign(5 * nc, R(0.0));
    UR[d].assign(5 * nc, R(0.0));
    F1[d].assign(5 * nc, R(0.0));
    F2[d].assign(5 * nc, R(0.0));
    if (roe) eta[d].assign(nc, R(0.0));
  }

  // steps 1-2: reconstruction and the first set of Riemann solves, one axis at
  // a time.  Reconstructed cells along the sweep: padded index 3 .. N-4 (every
  // stencil, up to i-3..i+3 for PPMP, lies inside the padded grid; these are
  // the cells whose face states the fluxes of the real cells need).
  for (int d = 0; d < 3; ++d) {
    if (!active[d]) continue;
    const size_t sd = G.stride(d);
    const int* P = PERM[d];
#pragma omp parallel for if (threaded) schedule(static)
    for (int k = 0; k < G.N[2]; ++k)
      for (int j = 0; j < G.N[1]; ++j)
        for (int i = 0; i < G.N[0]; ++i) {
          const int c3[3] = {i, j, k};
          if (c3[d] < 3 || c3[d] > G.N[d] - 4) continue;
          const size_t c = G.idx(i, j, k);
          R w[7][5];
          for (int s = 0; s < 7; ++s) {
            const size_t cs = c + (size_t)((long)(s - 3) * (long)sd);
            w[s][0] = W[0 * nc + cs];
            w[s][1] = W[(1 + P[0]) * nc + cs];
            w[s][2] = W[(1 + P[1]) * nc + cs];
            w[s][3] = W[(1 + P[2]) * nc + cs];
            w[s][4] = W[4 * nc + cs];
          }
          R WsL[5], WsR[5], UsL[5], UsR[5];
          set_stage((R*)nullptr, 1);
          add_units((R*)nullptr, 1);
          switch (G.recon) {
            case RECON_PPMP:
              ppmp_cell(w, dtdx, R(G.dx), g, WsL, WsR);
              prim_to_cons(WsL, g, UsL);
              prim_to_cons(WsR, g, UsR);
              break;
            case RECON_PLMC:
              plmc_cell(&w[2], dtdx, g, WsL, WsR);
              prim_to_cons(WsL, g, UsL);
              prim_to_cons(WsR, g, UsR);
              break;
            case RECON_PLMP:
              plmp_cell(&w[2], dtdx, g, UsL, UsR);
              break;
            case RECON_PCM:  // U*_R(i-1/2) = U*_L(i+1/2) = u_i
              UsL[0] = G.u[0 * nc + c];
              UsL[4] = G.u[4 * nc + c];
              for (int s = 0; s < 3; ++s) UsL[1 + s] = G.u[(1 + P[s]) * nc + c];
              for (int q = 0; q < 5; ++q) UsR[q] = UsL[q];
              break;
            default:
              ppmc_cell(&w[1], dtdx, g, WsL, WsR);
              prim_to_cons(WsL, g, UsL);
              prim_to_cons(WsR, g, UsR);
              break;
          }
          // left face of cell i is the right state of face i-1/2; right face of
          // cell i is the left state of face i+1/2
          const size_t cr = c + sd;
          UR[d][0 * nc + c] = UsL[0];
          UR[d][4 * nc + c] = UsL[4];
          UL[d][0 * nc + cr] = UsR[0];
          UL[d][4 * nc + cr] = UsR[4];
          for (int s = 0; s < 3; ++s) {
            UR[d][(1 + P[s]) * nc + c] = UsL[1 + s];
            UL[d][(1 + P[s]) * nc + cr] = UsR[1 + s];
          }
        }
    int fl = 0;
#pragma omp parallel for if (threaded) schedule(static) reduction(| : fl)
    for (int k = 0; k < G.N[2]; ++k)
      for (int j = 0; j < G.N[1]; ++j)
        for (int i = 0; i < G.N[0]; ++i) {
          const int c3[3] = {i, j, k};
          if (c3[d] < 4 || c3[d] > G.N[d] - 4) continue;
          const size_t f = G.idx(i, j, k);
          R ULr[5], URr[5], Fr[5];
          ULr[0] = UL[d][0 * nc + f]; URr[0] = UR[d][0 * nc + f];
          ULr[4] = UL[d][4 * nc + f]; URr[4] = UR[d][4 * nc + f];
          for (int s = 0; s < 3; ++s) {
            ULr[1 + s] = UL[d][(1 + P[s]) * nc + f];
            URr[1 + s] = UR[d][(1 + P[s]) * nc + f];
          }
          set_stage((R*)nullptr, 2);
          add_units((R*)nullptr, 2);
          if (roe) {
            fl |= riemann_roe_cons(ULr, URr, g, R(0.0), Fr);
            eta[d][f] = h_eta(ULr, URr, g);
          } else {
            fl |= riemann_exact_cons(ULr, URr, g, Fr);
          }
          F1[d][0 * nc + f] = Fr[0];
          F1[d][4 * nc + f] = Fr[4];
          for (int s = 0; s < 3; ++s) F1[d][(1 + P[s]) * nc + f] = Fr[1 + s];
        }
    flags |= fl;
  }

  // steps 3-4: transverse half-step (Eq. transverse_evolution) and the second
  // set of Riemann solves
  for (int d = 0; d < 3; ++d) {
    if (!active[d]) continue;
    const size_t sd = G.stride(d);
    const int* P = PERM[d];
    const int t1 = P[1], t2 = P[2];  // transverse axes in cyclic order
    int fl = 0;
#pragma omp parallel for if (threaded) schedule(static) reduction(| : fl)
    for (int k = 0; k < G.N[2]; ++k)
      for (int j = 0; j < G.N[1]; ++j)
        for (int i = 0; i < G.N[0]; ++i) {
          const int c3[3] = {i, j, k};
          if (c3[d] < 4 || c3[d] > G.N[d] - 4) continue;
          bool ok = true;
          for (int t = 0; t < 3; ++t)
            if (t != d && active[t] && (c3[t] < 4 || c3[t] > G.N[t] - 5)) ok = false;
          if (!ok) continue;
          const size_t f = G.idx(i, j, k);
          const size_t cl = f - sd;  // cell left of the face
          const size_t cr = f;       // cell right of the face
          set_stage((R*)nullptr, 3);
          add_units((R*)nullptr, 3);
          R UhL[5], UhR[5];
          for (int q = 0; q < 5; ++q) {
            UhL[q] = UL[d][q * nc + f];
            UhR[q] = UR[d][q * nc + f];
          }
          const int tt[2] = {t1, t2};
          for (int m = 0; m < 2; ++m) {
            const int t = tt[m];
            if (!active[t]) continue;
            const size_t st = G.stride(t);
            for (int q = 0; q < 5; ++q) {
              UhL[q] = UhL[q] + hdtdx * (F1[t][q * nc + cl] - F1[t][q * nc + cl + st]);
              UhR[q] = UhR[q] + hdtdx * (F1[t][q * nc + cr] - F1[t][q * nc + cr + st]);
            }
          }
          R ULr[5], URr[5], Fr[5];
          ULr[0] = UhL[0]; URr[0] = UhR[0];
          ULr[4] = UhL[4]; URr[4] = UhR[4];
          for (int s = 0; s < 3; ++s) {
            ULr[1 + s] = UhL[1 + P[s]];
            URr[1 + s] = UhR[1 + P[s]];
          }
          if (roe) {
            // H correction (App. C): the largest eta of this face and of the
            // transverse faces of the two cells it separates (nine in 3D)
            R etaH = eta[d][f];
            for (int m = 0; m < 2; ++m) {
              const int t = tt[m];
              if (!active[t]) continue;
              const size_t st = G.stride(t);
              etaH = mx(etaH, eta[t][cl]);
              etaH = mx(etaH, eta[t][cl + st]);
              etaH = mx(etaH, eta[t][cr]);
              etaH = mx(etaH, eta[t][cr + st]);
            }
            fl |= riemann_roe_cons(ULr, URr, g, etaH, Fr);
          } else {
            fl |= riemann_exact_cons(ULr, URr, g, Fr);
          }
          F2[d][0 * nc + f] = Fr[0];
          F2[d][4 * nc + f] = Fr[4];
          for (int s = 0; s < 3; ++s) F2[d][(1 + P[s]) * nc + f] = Fr[1 + s];
        }
    flags |= fl;
  }

  // step 5: conserved update of the real cells (Eq. conserved_update)
  set_stage((R*)nullptr, 4);
  int fl = 0;
#pragma omp parallel for if (threaded) schedule(static) reduction(| : fl)
  for (int k = G.gh[2]; k < G.gh[2] + G.n[2]; ++k)
    for (int j = G.gh[1]; j < G.gh[1] + G.n[1]; ++j)
      for (int i = G.gh[0]; i < G.gh[0] + G.n[0]; ++i) {
        const size_t c = G.idx(i, j, k);
        add_units((R*)nullptr, 4);
        for (int q = 0; q < 5; ++q) {
          R un = G.u[q * nc + c];
          for (int d = 0; d < 3; ++d) {
            if (!active[d]) continue;
            const size_t sd = G.stride(d);
            un = un + dtdx * (F2[d][q * nc + c] - F2[d][q * nc + c + sd]);
          }
          G.u[q * nc + c] = un;
          if (std::isnan(val(un))) fl |= FLAG_NONPHYS;
        }
        if (!(val(G.u[c]) > 0.0)) fl |= FLAG_NONPHYS;
      }
  flags |= fl;
  return flags;
}

struct Handle {
  Grid<double> G;
  Handle(const int n[3], double dx, double gamma, const int bc[6]) : G(n, dx, gamma, bc) {}
};

}  // namespace

// ---------------------------------------------------------------------------
// C interface used by the tests (ctypes).  Conserved state layout for set/get:
// five planes [5][nz][ny][nx] of real cells, x fastest.
extern "C" {

void* oracle_init(int nx, int ny, int nz, double dx, double gamma, const int* bc) {
  const int n[3] = {nx, ny, nz};
  for (int d = 0; d < 3; ++d) {
    if (n[d] < 1 || (n[d] > 1 && n[d] < NG)) return nullptr;
    if (n[d] > 1 && ((bc[2 * d] == BC_PERIODIC) != (bc[2 * d + 1] == BC_PERIODIC))) return nullptr;
  }
  if (!(dx > 0.0) || !(gamma > 1.0)) return nullptr;
  return new Handle(n, dx, gamma, bc);
}

void oracle_free(void* h) { delete static_cast<Handle*>(h); }

int oracle_set_inflow(void* h, int face, const double* prim) {
  if (!h || face < 0 || face > 5) return -1;
  for (int q = 0; q < 5; ++q) static_cast<Handle*>(h)->G.inflow_prim[face][q] = prim[q];
  return 0;
}

// Riemann solver: 0 exact (default), 1 Roe (HLLE fallback, H correction in the
// second set)
int oracle_set_solver(void* h, int solver) {
  if (!h || solver < SOLVER_EXACT || solver > SOLVER_ROE) return -1;
  static_cast<Handle*>(h)->G.solver = solver;
  return 0;
}

// reconstruction: 0 PPMC (default), 1 PPMP, 2 PLMC, 3 PLMP, 4 PCM
int oracle_set_recon(void* h, int recon) {
  if (!h || recon < RECON_PPMC || recon > RECON_PCM) return -1;
  static_cast<Handle*>(h)->G.recon = recon;
  return 0;
}

int oracle_set_state(void* h, const double* u) {
  auto& G = static_cast<Handle*>(h)->G;
  const size_t nreal = (size_t)G.n[0] * G.n[1] * G.n[2];
  for (int q = 0; q < 5; ++q)
    for (int k = 0; k < G.n[2]; ++k)
      for (int j = 0; j < G.n[1]; ++j)
        for (int i = 0; i < G.n[0]; ++i)
          G.u[q * G.ncell + G.idx(i + G.gh[0], j + G.gh[1], k + G.gh[2])] =
              u[q * nreal + ((size_t)k * G.n[1] + j) * G.n[0] + i];
  return 0;
}

int oracle_get_state(void* h, double* u) {
  auto& G = static_cast<Handle*>(h)->G;
  const size_t nreal = (size_t)G.n[0] * G.n[1] * G.n[2];
  for (int q = 0; q < 5; ++q)
    for (int k = 0; k < G.n[2]; ++k)
      for (int j = 0; j < G.n[1]; ++j)
        for (int i = 0; i < G.n[0]; ++i)
          u[q * nreal + ((size_t)k * G.n[1] + j) * G.n[0] + i] =
              G.u[q * G.ncell + G.idx(i + G.gh[0], j + G.gh[1], k + G.gh[2])];
  return 0;
}

double oracle_compute_dt(void* h, double cfl) {
  return cfl * compute_dt_min(static_cast<Handle*>(h)->G);
}

int oracle_step_dt(void* h, double dt) {
  auto& G = static_cast<Handle*>(h)->G;
  const int flags = ctu_step(G, dt, true);
  G.time += dt;
  return flags;
}

// time at the start of the next step (used by the Noh boundary); starts at 0
int oracle_set_time(void* h, double t) {
  if (!h) return -1;
  static_cast<Handle*>(h)->G.time = t;
  return 0;
}
double oracle_get_time(void* h) { return static_cast<Handle*>(h)->G.time; }

// Padded conserved state after the ghost fill of the current state, for the
// boundary tests: [5][N2][N1][N0] with N = n + 8 on active axes.
int oracle_fill_ghosts(void* h, double* upad) {
  auto& G = static_cast<Handle*>(h)->G;
  fill_ghosts(G);
  std::memcpy(upad, G.u.data(), sizeof(double) * 5 * G.ncell);
  return 0;
}

int oracle_set_threads(int n) {
#ifdef _OPENMP
  omp_set_num_threads(n > 0 ? n : omp_get_num_procs());  // 0: every processor
  return omp_get_max_threads();
#else
  (void)n;
  return 1;
#endif
}

// Exact Riemann solver on n primitive state pairs (rotated order, [n][5] each).
int oracle_riemann_prim(int n, const double* WL, const double* WR, double gamma, double* F,
                        double* pm, double* um, double* ws, int* iters) {
  const Gas g(gamma);
  int flags = 0;
  for (int i = 0; i < n; ++i) {
    RiemannResult<double> r;
    riemann_exact_prim(WL + 5 * i, WR + 5 * i, g, r);
    for (int q = 0; q < 5; ++q) {
      if (F) F[5 * i + q] = r.F[q];
      if (ws) ws[5 * i + q] = r.ws[q];
    }
    if (pm) pm[i] = r.pm;
    if (um) um[i] = r.um;
    if (iters) iters[i] = r.iters;
    flags |= r.flags;
  }
  return flags;
}

// Exact Riemann solver on n conserved state pairs (rotated order, [n][5] each),
// as the CTU step calls it (conversion to primitives with the pressure floor).
int oracle_riemann_cons(int n, const double* UL, const double* UR, double gamma, double* F) {
  const Gas g(gamma);
  int flags = 0;
  for (int i = 0; i < n; ++i) flags |= riemann_exact_cons(UL + 5 * i, UR + 5 * i, g, F + 5 * i);
  return flags;
}

// PPMC on n five-cell stencils w[n][5 cells][5 prims] (rotated order).
int oracle_ppmc(int n, const double* w, double dtdx, double gamma, double* WsL, double* WsR) {
  const Gas g(gamma);
  for (int i = 0; i < n; ++i) {
    double st[5][5];
    for (int s = 0; s < 5; ++s)
      for (int q = 0; q < 5; ++q) st[s][q] = w[25 * i + 5 * s + q];
    ppmc_cell(st, dtdx, g, WsL + 5 * i, WsR + 5 * i);
  }
  return 0;
}

// Any reconstruction on seven-cell primitive stencils w[n][7 cells i-3..i+3][5]
// (rotated order); returns the conserved face states of the centre cell at its
// left (UsL) and right (UsR) face, each [n][5].  PCM returns the conserved
// form of w_i at both faces.
int oracle_reconstruct(int n, int recon, const double* w, double dtdx, double dx, double gamma,
                       double* UsL, double* UsR) {
  if (recon < RECON_PPMC || recon > RECON_PCM) return -1;
  const Gas g(gamma);
  for (int i = 0; i < n; ++i) {
    double st[7][5], WsL[5], WsR[5];
    for (int s = 0; s < 7; ++s)
      for (int q = 0; q < 5; ++q) st[s][q] = w[35 * i + 5 * s + q];
    double* L = UsL + 5 * i;
    double* R = UsR + 5 * i;
    switch (recon) {
      case RECON_PPMP: ppmp_cell(st, dtdx, dx, g, WsL, WsR); break;
      case RECON_PLMC: plmc_cell(&st[2], dtdx, g, WsL, WsR); break;
      case RECON_PLMP: plmp_cell(&st[2], dtdx, g, L, R); continue;
      case RECON_PCM:
        for (int q = 0; q < 5; ++q) WsL[q] = WsR[q] = st[3][q];
        break;
      default: ppmc_cell(&st[1], dtdx, g, WsL, WsR); break;
    }
    prim_to_cons(WsL, g, L);
    prim_to_cons(WsR, g, R);
  }
  return 0;
}

// Roe solver (with the HLLE fallback) on n interfaces: conserved states [n][5]
// in sweep order, etaH [n] (0: no H correction); fluxes F [n][5].
int oracle_riemann_roe(int n, const double* UL, const double* UR, const double* etaH,
                       double gamma, double* F) {
  const Gas g(gamma);
  for (int i = 0; i < n; ++i)
    riemann_roe_cons(UL + 5 * i, UR + 5 * i, g, etaH ? etaH[i] : 0.0, F + 5 * i);
  return 0;
}

// Algorithmic operation count of one CTU step with the given dt on the current
// state (the state itself is not changed).  counts = {add/sub, mul, div, sqrt,
// pow, compare/min/max/abs}; returns the step's status flags.
int oracle_count_step(void* h, double dt, double* counts) {
  const auto& G0 = static_cast<Handle*>(h)->G;
  Grid<CR> G(G0.n, G0.dx, G0.gamma, G0.bc);
  for (int f = 0; f < 6; ++f)
    for (int q = 0; q < 5; ++q) G.inflow_prim[f][q] = G0.inflow_prim[f][q];
  G.recon = G0.recon;
  G.solver = G0.solver;
  G.time = G0.time;
  for (size_t i = 0; i < G0.u.size(); ++i) G.u[i] = CR(G0.u[i]);
  g_ops = OpCount();
  for (int k = 0; k < kStages; ++k) {
    g_stage_ops[k] = OpCount();
    g_units[k] = 0;
  }
  g_stage = 0;
  const int fl = ctu_step(G, dt, false);
  counts[0] = (double)g_ops.add;
  counts[1] = (double)g_ops.mul;
  counts[2] = (double)g_ops.div;
  counts[3] = (double)g_ops.sqrt;
  counts[4] = (double)g_ops.pow;
  counts[5] = (double)g_ops.cmp;
  return fl;
}

// Per-stage version of oracle_count_step: counts[stage*6 + kind] with the kinds
// of oracle_count_step and units[stage] cells or faces processed, for the six
// stages (0 primitives and the dt minimum, 1 PPMC without slopes, 2 first
// Riemann solves, 3 transverse half-step + second Riemann solves, 4 update,
// 5 limited slopes -- the oracle computes three per PPMC cell).
int oracle_count_step_stages(void* h, double dt, double* counts, double* units) {
  const auto& G0 = static_cast<Handle*>(h)->G;
  Grid<CR> G(G0.n, G0.dx, G0.gamma, G0.bc);
  for (int f = 0; f < 6; ++f)
    for (int q = 0; q < 5; ++q) G.inflow_prim[f][q] = G0.inflow_prim[f][q];
  G.recon = G0.recon;
  G.solver = G0.solver;
  G.time = G0.time;
  for (size_t i = 0; i < G0.u.size(); ++i) G.u[i] = CR(G0.u[i]);
  g_ops = OpCount();
  for (int k = 0; k < kStages; ++k) {
    g_stage_ops[k] = OpCount();
    g_units[k] = 0;
  }
  g_stage = 0;
  (void)compute_dt_min(G);
  const int fl = ctu_step(G, dt, false);
  for (int k = 0; k < kStages; ++k) {
    const OpCount& c = g_stage_ops[k];
    const uint64_t v[6] = {c.add, c.mul, c.div, c.sqrt, c.pow, c.cmp};
    for (int q = 0; q < 6; ++q) counts[6 * k + q] = (double)v[q];
    units[k] = (double)g_units[k];
  }
  return fl;
}

}  // extern "C"
