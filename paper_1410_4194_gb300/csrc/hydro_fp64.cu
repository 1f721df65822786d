// hydro_fp64.cu -- FP64 kernels of one CTU step (Sec. 2.3) on sm_103a.
//
// Built with --fmad=false: every a*b+c of this file is a rounded multiply and a
// rounded add, as in the CPU reference, so the FP64 path differs from it only
// through pow() (CUDA's versus the host libm's, a few ulp).
//
// One launch per stage, one thread per cell or face, x fastest so that every
// load and store of a warp is coalesced (neighbours along y or z are whole rows
// apart; each of those loads is still a coalesced row segment).  FP64
// arithmetic, not memory, bounds this path on GB300 (two FP64 FMA per clock per
// SM), so every intermediate -- primitives, slopes, face states, first fluxes
// -- is computed once and stored in HBM rather than recomputed by neighbours:
// the extra traffic is a few percent of what HBM delivers in the same time.
//
// Stages of one step (each a kernel below):
//   k_prims      ghost cells by index remap (Sec. 3.1) + primitives + dt minimum
//   k_set_dt     dt = cfl * min (Eq. calc_dt_3D) or a fixed dt; dt/dx
//   k_slopes<d>  limited characteristic slopes along axis d (App. A.2)
//   k_ppmc<d>    traced face states W* of every cell (App. A.3)
//   k_riemann1<d> first fluxes F* (Sec. 2.3 step 2; App. B.1)
//   k_riemann2<d> transverse half-step (Eq. transverse_evolution) + CTU fluxes
//   k_update     conserved update (Eq. conserved_update) + positivity check
#include <math.h>

#include "hydro_internal.h"
#include "hydro_math.cuh"

namespace hydro {
namespace {

constexpr int kThreads = 256;
using Gas = GasT<double>;

__device__ __forceinline__ void box_coords(const Box& b, long long t, int c[3]) {
  const long long n0 = b.n[0], n01 = (long long)b.n[0] * b.n[1];
  c[2] = b.lo[2] + (int)(t / n01);
  const long long r = t - (long long)(c[2] - b.lo[2]) * n01;
  c[1] = b.lo[1] + (int)(r / n0);
  c[0] = b.lo[0] + (int)(r - (long long)(c[1] - b.lo[1]) * n0);
}

__device__ __forceinline__ long long pidx(const Geom& G, const int c[3]) {
  return c[0] + c[1] * G.s[1] + c[2] * G.s[2];
}

// order of the velocity components in a sweep along axis D: (normal, t1, t2)
template <int D> struct Perm {
  static constexpr int n = D, t1 = (D + 1) % 3, t2 = (D + 2) % 3;
};

// load primitive cell c in sweep order (rho, v_n, v_t1, v_t2, p)
template <int D>
__device__ __forceinline__ void load_prim(const double* __restrict__ W, long long ps, long long c,
                                          double w[5]) {
  w[0] = W[c];
  w[1] = W[(1 + Perm<D>::n) * ps + c];
  w[2] = W[(1 + Perm<D>::t1) * ps + c];
  w[3] = W[(1 + Perm<D>::t2) * ps + c];
  w[4] = W[4 * ps + c];
}

// load/store a global-order 5-vector plane set in sweep order
template <int D>
__device__ __forceinline__ void load_rot(const double* __restrict__ A, long long ps, long long c,
                                         double v[5]) {
  v[0] = A[c];
  v[1] = A[(1 + Perm<D>::n) * ps + c];
  v[2] = A[(1 + Perm<D>::t1) * ps + c];
  v[3] = A[(1 + Perm<D>::t2) * ps + c];
  v[4] = A[4 * ps + c];
}
template <int D>
__device__ __forceinline__ void store_rot(double* __restrict__ A, long long ps, long long c,
                                          const double v[5]) {
  A[c] = v[0];
  A[(1 + Perm<D>::n) * ps + c] = v[1];
  A[(1 + Perm<D>::t1) * ps + c] = v[2];
  A[(1 + Perm<D>::t2) * ps + c] = v[3];
  A[4 * ps + c] = v[4];
}

__device__ __forceinline__ int* rec_flags(double* rec) { return reinterpret_cast<int*>(rec + 4); }

// block-wide minimum of a positive double, then one atomicMin on its bits
__device__ __forceinline__ void block_min_to(double v, unsigned long long* slot) {
  __shared__ double warp_min[kThreads / 32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const double w = __shfl_xor_sync(0xffffffffu, v, o);
    v = tmin(v, w);
  }
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) warp_min[wid] = v;
  __syncthreads();
  if (wid == 0) {
    v = (lane < (int)(blockDim.x >> 5)) ? warp_min[lane] : __longlong_as_double(0x7ff0000000000000ll);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const double w = __shfl_xor_sync(0xffffffffu, v, o);
      v = tmin(v, w);
    }
    if (lane == 0 && v >= 0.0) atomicMin(slot, (unsigned long long)__double_as_longlong(v));
  }
}

// ---------------------------------------------------------------------------
// Primitives of every padded cell.  A ghost cell takes the value the
// boundary passes x, then y, then z would give it: a mapped real cell (periodic
// wrap, mirror, or the outermost cell) with the normal momentum of every
// reflective axis negated, unless an inflow axis is involved, in which case the
// last inflow face (in x, y, z order) provides the state and only the
// reflective axes after it negate their momentum.
__global__ void __launch_bounds__(kThreads) k_prims(Geom G, Bufs B, BcDesc bc, Gas g, int want_dt) {
  const long long total = (long long)G.N[0] * G.N[1] * G.N[2];
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  double local = __longlong_as_double(0x7ff0000000000000ll);
  if (t < total) {
    int c[3];
    c[2] = (int)(t / G.s[2]);
    c[1] = (int)((t - c[2] * G.s[2]) / G.s[1]);
    c[0] = (int)(t - c[2] * G.s[2] - c[1] * G.s[1]);
    int src[3];
    int neg = 0, inflow_face = -1;
    bool real = true;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      const int n = G.n[d];
      const int r = c[d] - G.g[d];
      if (r >= 0 && r < n) {
        src[d] = r;
        continue;
      }
      real = false;
      const bool lo = r < 0;
      const int depth = lo ? -r : r - n + 1;
      const int face = 2 * d + (lo ? 0 : 1);
      switch (bc.type[face]) {
        case 0:  // periodic
          src[d] = lo ? n - depth : depth - 1;
          break;
        case 1:  // reflective
          src[d] = lo ? depth - 1 : n - depth;
          neg |= 1 << d;
          break;
        case 2:  // outflow
          src[d] = lo ? 0 : n - 1;
          break;
        default:  // inflow
          src[d] = 0;
          inflow_face = face;
          neg = 0;
          break;
      }
    }
    double U[5];
    if (inflow_face >= 0) {
#pragma unroll
      for (int q = 0; q < 5; ++q) U[q] = bc.inflow[inflow_face][q];
    } else {
      const long long rs = src[0] + (long long)G.n[0] * (src[1] + (long long)G.n[1] * src[2]);
#pragma unroll
      for (int q = 0; q < 5; ++q) U[q] = B.u[q * G.nreal + rs];
    }
#pragma unroll
    for (int d = 0; d < 3; ++d)
      if (neg & (1 << d)) U[1 + d] = -U[1 + d];
    // primitives in the CPU reference's operation order (divisions), then the
    // per-cell reciprocals the later stages multiply by
    const double d = U[0];
    double W[5];
    W[0] = d;
    W[1] = U[1] / d;
    W[2] = U[2] / d;
    W[3] = U[3] / d;
    W[4] = tmax(g.gm1 * (U[4] - 0.5 * d * (W[1] * W[1] + W[2] * W[2] + W[3] * W[3])), kPFloor);
    const double a = sqrt(g.gamma * W[4] / d);
#pragma unroll
    for (int q = 0; q < 5; ++q) B.W[q * G.ps + t] = W[q];
    B.W[5 * G.ps + t] = a;
    B.W[6 * G.ps + t] = 1.0 / a;
    B.W[7 * G.ps + t] = 1.0 / d;
    if (want_dt && real) {
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        if (G.n[d] > 1) {
          const double tc = G.dx / (fabs(W[1 + d]) + a);
          local = tmin(local, tc);
        }
      }
    }
  }
  if (want_dt) block_min_to(local, reinterpret_cast<unsigned long long*>(B.rec));
}

__global__ void k_set_dt(double* rec, double cfl, double fixed_dt, double dx) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    const double dt = (fixed_dt > 0.0) ? fixed_dt : cfl * rec[0];
    const double dtdx = dt / dx;
    rec[1] = dt;
    rec[2] = dtdx;
    rec[3] = 0.5 * dtdx;
  }
}

template <int D, bool S>
__global__ void __launch_bounds__(kThreads) k_slopes(Geom G, Bufs B, Box box, Gas g) {
  const long long count = (long long)box.n[0] * box.n[1] * box.n[2];
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= count) return;
  int c3[3];
  box_coords(box, t, c3);
  const long long c = pidx(G, c3);
  const long long s = G.s[D];
  double wm[5], wc[5], wp[5], dw[5];
  load_prim<D>(B.W, G.ps, c - s, wm);
  load_prim<D>(B.W, G.ps, c, wc);
  load_prim<D>(B.W, G.ps, c + s, wp);
  const double a = B.W[5 * G.ps + c];
  const double inv_a = B.W[6 * G.ps + c];
  const double inv_rho = B.W[7 * G.ps + c];
  limited_slope<S>(wm, wc, wp, a, inv_a, inv_rho, dw);
#pragma unroll
  for (int q = 0; q < 5; ++q) B.S[q * G.ps + c] = dw[q];
}

template <int D, bool S>
__global__ void __launch_bounds__(kThreads) k_ppmc(Geom G, Bufs B, Box box, Gas g) {
  const long long count = (long long)box.n[0] * box.n[1] * box.n[2];
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= count) return;
  int c3[3];
  box_coords(box, t, c3);
  const long long c = pidx(G, c3);
  const long long s = G.s[D];
  double wm[5], wc[5], wp[5], sm[5], sc[5], sp[5];
  load_prim<D>(B.W, G.ps, c - s, wm);
  load_prim<D>(B.W, G.ps, c, wc);
  load_prim<D>(B.W, G.ps, c + s, wp);
#pragma unroll
  for (int q = 0; q < 5; ++q) {
    sm[q] = B.S[q * G.ps + c - s];
    sc[q] = B.S[q * G.ps + c];
    sp[q] = B.S[q * G.ps + c + s];
  }
  const double a = B.W[5 * G.ps + c];
  const double inv_a = B.W[6 * G.ps + c];
  const double inv_rho = B.W[7 * G.ps + c];
  const double dtdx = B.rec[2];
  double WsL[5], WsR[5];
  ppmc_states<S>(wm, wc, wp, sm, sc, sp, a, inv_a, inv_rho, dtdx, WsL, WsR);
  // the left face of cell c is the right state of face c; its right face is the
  // left state of face c+1.  Stored as primitives W*, or (strict) as the
  // conserved U* the paper passes between kernels.
  if constexpr (S) {
    double UsL[5], UsR[5];
    prim2cons<true>(WsL, g, UsL);
    prim2cons<true>(WsR, g, UsR);
    store_rot<D>(B.UR[D], G.ps, c, UsL);
    store_rot<D>(B.UL[D], G.ps, c + s, UsR);
  } else {
    store_rot<D>(B.UR[D], G.ps, c, WsL);
    store_rot<D>(B.UL[D], G.ps, c + s, WsR);
  }
}

template <int D, bool S>
__global__ void __launch_bounds__(kThreads) k_riemann1(Geom G, Bufs B, Box box, Gas g) {
  const long long count = (long long)box.n[0] * box.n[1] * box.n[2];
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= count) return;
  int c3[3];
  box_coords(box, t, c3);
  const long long f = pidx(G, c3);
  double WL[5], WR[5], F[5];
  int fl;
  if constexpr (S) {
    double UL[5], UR[5], idL, idR;
    load_rot<D>(B.UL[D], G.ps, f, UL);
    load_rot<D>(B.UR[D], G.ps, f, UR);
    cons2prim<true>(UL, g, WL, idL);
    cons2prim<true>(UR, g, WR, idR);
    fl = riemann_exact<true>(WL, WR, idL, idR, g, F);
  } else {
    load_rot<D>(B.UL[D], G.ps, f, WL);
    load_rot<D>(B.UR[D], G.ps, f, WR);
    fl = riemann_exact<false>(WL, WR, 1.0 / WL[0], 1.0 / WR[0], g, F);
  }
  store_rot<D>(B.F1[D], G.ps, f, F);
  if (fl) atomicOr(rec_flags(B.rec), fl);
}

template <int D, bool S>
__global__ void __launch_bounds__(kThreads) k_riemann2(Geom G, Bufs B, Box box, Gas g) {
  const long long count = (long long)box.n[0] * box.n[1] * box.n[2];
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= count) return;
  int c3[3];
  box_coords(box, t, c3);
  const long long f = pidx(G, c3);
  const long long ps = G.ps;
  const long long cl = f - G.s[D], cr = f;
  const double h = B.rec[3];
  double UhL[5], UhR[5];
  if constexpr (S) {  // U* stored conserved
#pragma unroll
    for (int q = 0; q < 5; ++q) {
      UhL[q] = B.UL[D][q * ps + f];
      UhR[q] = B.UR[D][q * ps + f];
    }
  } else {  // U* from the stored W* (global order)
    double WsL[5], WsR[5];
#pragma unroll
    for (int q = 0; q < 5; ++q) {
      WsL[q] = B.UL[D][q * ps + f];
      WsR[q] = B.UR[D][q * ps + f];
    }
    prim2cons(WsL, g, UhL);
    prim2cons(WsR, g, UhR);
  }
  constexpr int T1 = Perm<D>::t1, T2 = Perm<D>::t2;
  if (G.n[T1] > 1) {
    const double* F = B.F1[T1];
    const long long st = G.s[T1];
#pragma unroll
    for (int q = 0; q < 5; ++q) {
      UhL[q] = UhL[q] + h * (F[q * ps + cl] - F[q * ps + cl + st]);
      UhR[q] = UhR[q] + h * (F[q * ps + cr] - F[q * ps + cr + st]);
    }
  }
  if (G.n[T2] > 1) {
    const double* F = B.F1[T2];
    const long long st = G.s[T2];
#pragma unroll
    for (int q = 0; q < 5; ++q) {
      UhL[q] = UhL[q] + h * (F[q * ps + cl] - F[q * ps + cl + st]);
      UhR[q] = UhR[q] + h * (F[q * ps + cr] - F[q * ps + cr + st]);
    }
  }
  double UL[5], UR[5], WL[5], WR[5], Fx[5], idL, idR;
  UL[0] = UhL[0]; UL[1] = UhL[1 + D]; UL[2] = UhL[1 + T1]; UL[3] = UhL[1 + T2]; UL[4] = UhL[4];
  UR[0] = UhR[0]; UR[1] = UhR[1 + D]; UR[2] = UhR[1 + T1]; UR[3] = UhR[1 + T2]; UR[4] = UhR[4];
  cons2prim<S>(UL, g, WL, idL);
  cons2prim<S>(UR, g, WR, idR);
  const int fl = riemann_exact<S>(WL, WR, idL, idR, g, Fx);
  // CTU flux of this face replaces its (now consumed) left state
  store_rot<D>(B.UL[D], ps, f, Fx);
  if (fl) atomicOr(rec_flags(B.rec), fl);
}

__global__ void __launch_bounds__(kThreads) k_update(Geom G, Bufs B) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= G.nreal) return;
  const int i = (int)(t % G.n[0]);
  const int j = (int)((t / G.n[0]) % G.n[1]);
  const int k = (int)(t / ((long long)G.n[0] * G.n[1]));
  const long long c = (i + G.g[0]) + (j + G.g[1]) * G.s[1] + (k + G.g[2]) * G.s[2];
  const double dtdx = B.rec[2];
  int fl = 0;
#pragma unroll
  for (int q = 0; q < 5; ++q) {
    double un = B.u[q * G.nreal + t];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      if (G.n[d] > 1) {
        const double* F = B.UL[d];
        un = un + dtdx * (F[q * G.ps + c] - F[q * G.ps + c + G.s[d]]);
      }
    }
    B.u[q * G.nreal + t] = un;
    if (isnan(un)) fl = kFlagNonPhys;
    if (q == 0 && !(un > 0.0)) fl = kFlagNonPhys;
  }
  if (fl) atomicOr(rec_flags(B.rec), fl);
}

// ---- building blocks on SoA device arrays -----------------------------------
__global__ void k_riemann_soa(int n, const double* __restrict__ UL, const double* __restrict__ UR,
                              Gas g, double* __restrict__ F, int* flags) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n) return;
  double L[5], R[5], WL[5], WR[5], Fx[5], idL, idR;
#pragma unroll
  for (int q = 0; q < 5; ++q) {
    L[q] = UL[(long long)q * n + t];
    R[q] = UR[(long long)q * n + t];
  }
  cons2prim(L, g, WL, idL);
  cons2prim(R, g, WR, idR);
  const int fl = riemann_exact<false>(WL, WR, idL, idR, g, Fx);
#pragma unroll
  for (int q = 0; q < 5; ++q) F[(long long)q * n + t] = Fx[q];
  if (fl && flags) atomicOr(flags, fl);
}

__global__ void k_ppmc_soa(int n, const double* __restrict__ w, double dtdx, Gas g,
                           double* __restrict__ WsL, double* __restrict__ WsR) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n) return;
  double st[5][5], a[5], ia[5], ir[5];
#pragma unroll
  for (int s = 0; s < 5; ++s) {
#pragma unroll
    for (int q = 0; q < 5; ++q) st[s][q] = w[((long long)s * 5 + q) * n + t];
    a[s] = sqrt(g.gamma * st[s][4] / st[s][0]);
    ia[s] = 1.0 / a[s];
    ir[s] = 1.0 / st[s][0];
  }
  double sm[5], sc[5], sp[5], L[5], R[5];
  limited_slope(st[0], st[1], st[2], a[1], ia[1], ir[1], sm);
  limited_slope(st[1], st[2], st[3], a[2], ia[2], ir[2], sc);
  limited_slope(st[2], st[3], st[4], a[3], ia[3], ir[3], sp);
  ppmc_states(st[1], st[2], st[3], sm, sc, sp, a[2], ia[2], ir[2], dtdx, L, R);
#pragma unroll
  for (int q = 0; q < 5; ++q) {
    WsL[(long long)q * n + t] = L[q];
    WsR[(long long)q * n + t] = R[q];
  }
}

inline unsigned blocks_for(long long count) {
  return (unsigned)((count + kThreads - 1) / kThreads);
}

// Range of an axis for a stage: real cells [g, g+n-1] widened by lo/hi (an
// inactive axis is always the single index 0).
inline void axis_range(const Geom& G, int d, int lo_off, int hi_off, int& lo, int& n) {
  if (G.n[d] <= 1) {
    lo = 0;
    n = 1;
    return;
  }
  lo = G.g[d] + lo_off;
  n = G.n[d] + hi_off - lo_off;
}

inline Box make_box(const Geom& G, int axis, int lo_d, int hi_d, int lo_o, int hi_o) {
  Box b;
  for (int d = 0; d < 3; ++d) {
    if (d == axis)
      axis_range(G, d, lo_d, hi_d, b.lo[d], b.n[d]);
    else
      axis_range(G, d, lo_o, hi_o, b.lo[d], b.n[d]);
  }
  return b;
}

inline long long box_count(const Box& b) { return (long long)b.n[0] * b.n[1] * b.n[2]; }

}  // namespace

cudaError_t fp64_prims(const Geom& G, const Bufs& B, const BcDesc& bc, double gamma, bool want_dt,
                       cudaStream_t st) {
  if (want_dt) {
    cudaError_t e = cudaMemsetAsync(B.rec, 0x7f, sizeof(double), st);
    if (e != cudaSuccess) return e;
  }
  const long long total = (long long)G.N[0] * G.N[1] * G.N[2];
  k_prims<<<blocks_for(total), kThreads, 0, st>>>(G, B, bc, make_gas<double>(gamma), want_dt ? 1 : 0);
  return cudaGetLastError();
}

cudaError_t fp64_set_dt(const Geom& G, const Bufs& B, double cfl, double fixed_dt, cudaStream_t st) {
  k_set_dt<<<1, 32, 0, st>>>(B.rec, cfl, fixed_dt, G.dx);
  return cudaGetLastError();
}

// Ranges (padded coordinates; "others" are the two axes across the sweep):
//   slopes   d in [g-2, g+n+1], others in [g-1, g+n]
//   ppmc     d in [g-1, g+n],   others in [g-1, g+n]
//   riemann1 faces d in [g, g+n], others in [g-1, g+n]
//   riemann2 faces d in [g, g+n], others real
// which is exactly what the CTU fluxes of the real cells need.
Box stage_box(const Geom& G, int stage, int axis) {
  switch (stage) {
    case kStageSlopes: return make_box(G, axis, -2, 2, -1, 1);
    case kStagePpmc: return make_box(G, axis, -1, 1, -1, 1);
    case kStageRiemann1: return make_box(G, axis, 0, 1, -1, 1);
    default: return make_box(G, axis, 0, 1, 0, 0);
  }
}

long long stage_units(const Geom& G, int stage, int axis) {
  if (stage == kStagePrims) return (long long)G.N[0] * G.N[1] * G.N[2];
  if (stage == kStageUpdate) return G.nreal;
  if (stage == kStageSetDt) return 1;
  return box_count(stage_box(G, stage, axis));
}

cudaError_t fp64_stage(const Geom& G, const Bufs& B, int stage, int axis, double gamma,
                       bool strict, cudaStream_t st) {
  const Gas g = make_gas<double>(gamma);
  const Box b = stage_box(G, stage, axis);
  const unsigned nb = blocks_for(box_count(b));
#define HYDRO_LAUNCH_AXIS(K)                                                      \
  if (strict) {                                                                   \
    switch (axis) {                                                               \
      case 0: K<0, true><<<nb, kThreads, 0, st>>>(G, B, b, g); break;            \
      case 1: K<1, true><<<nb, kThreads, 0, st>>>(G, B, b, g); break;            \
      default: K<2, true><<<nb, kThreads, 0, st>>>(G, B, b, g); break;           \
    }                                                                             \
  } else {                                                                        \
    switch (axis) {                                                               \
      case 0: K<0, false><<<nb, kThreads, 0, st>>>(G, B, b, g); break;           \
      case 1: K<1, false><<<nb, kThreads, 0, st>>>(G, B, b, g); break;           \
      default: K<2, false><<<nb, kThreads, 0, st>>>(G, B, b, g); break;          \
    }                                                                             \
  }
  switch (stage) {
    case kStageSlopes: HYDRO_LAUNCH_AXIS(k_slopes) break;
    case kStagePpmc: HYDRO_LAUNCH_AXIS(k_ppmc) break;
    case kStageRiemann1: HYDRO_LAUNCH_AXIS(k_riemann1) break;
    case kStageRiemann2: HYDRO_LAUNCH_AXIS(k_riemann2) break;
    default: return cudaErrorInvalidValue;
  }
#undef HYDRO_LAUNCH_AXIS
  return cudaGetLastError();
}

cudaError_t fp64_update(const Geom& G, const Bufs& B, cudaStream_t st) {
  k_update<<<blocks_for(G.nreal), kThreads, 0, st>>>(G, B);
  return cudaGetLastError();
}

cudaError_t fp64_riemann_soa(int n, const double* UL, const double* UR, double gamma, double* F,
                             int* flags, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  k_riemann_soa<<<blocks_for(n), kThreads, 0, st>>>(n, UL, UR, make_gas<double>(gamma), F, flags);
  return cudaGetLastError();
}

cudaError_t fp64_ppmc_soa(int n, const double* w, double dtdx, double gamma, double* WsL,
                          double* WsR, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  k_ppmc_soa<<<blocks_for(n), kThreads, 0, st>>>(n, w, dtdx, make_gas<double>(gamma), WsL, WsR);
  return cudaGetLastError();
}

}  // namespace hydro
