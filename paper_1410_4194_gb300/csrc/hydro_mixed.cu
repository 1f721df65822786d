// hydro_mixed.cu -- the mixed-precision CTU step (HYDRO_MIXED).
//
// Float32: the characteristic slopes, PPMC reconstruction and tracing, and both
// sets of exact Riemann solves (App. A.2, A.3, B.1) -- the bulk of the
// arithmetic, on GB300's FP32 pipe (64 times the FP64 rate).
// Float64, where the step's stability needs it:
//   * primitives of the FP64 state: the internal energy E - rho v^2/2 (the
//     cancellation of total and kinetic energy at high Mach), the pressure
//     floor and the CFL time-step reduction;
//   * the transverse half-step U^{n+1/2} = U* + dt/(2dx) (G*_{-} - G*_{+}) + ...
//     (Eq. transverse_evolution), a conserved flux accumulation, and the
//     recovery of the primitives of U^{n+1/2} (internal energy again);
//   * the conserved update (Eq. conserved_update), accumulated from the float
//     CTU fluxes into the FP64 state.
// Intermediates (primitives, slopes, face states, fluxes) are float, which
// halves their HBM traffic.  Compiled with FMA contraction.
#include "../../include/hydro.h"
#include "hydro_kernels.cuh"

namespace hydro {
namespace {

using GasF = GasT<float>;
using GasD = GasT<double>;

// resident 256-thread blocks per SM for the stencil and Riemann stages: the
// float kernels fit 64 registers (4 blocks, 50% of the warp slots) with a few
// bytes of spill, which measured ~1% faster than 3 blocks at 72-80 registers
constexpr int kMinBlocksMixed = 4;

// float views of the step's work arrays (same slab as the FP64 path)
struct BufsF {
  double* u;      // FP64 state, real cells [5][nz][ny][nx]
  float* W;       // padded primitives [8][ps]: rho, vx, vy, vz, p, a, 1/a, 1/rho
  float* S;       // padded slopes [5][ps] (sweep order)
  float* UL[3];   // per axis: primitive left states W*_L [5][ps]; then F^{n+1/2}
  float* UR[3];   // per axis: primitive right states W*_R [5][ps]
  float* F1[3];   // per axis: first fluxes F* [5][ps]
  double* rec;    // step record (dt, flags)
};

__host__ __device__ inline BufsF float_view(const Bufs& B) {
  BufsF F;
  F.u = B.u;
  F.W = reinterpret_cast<float*>(B.W);
  F.S = reinterpret_cast<float*>(B.S);
  for (int d = 0; d < 3; ++d) {
    F.UL[d] = reinterpret_cast<float*>(B.UL[d]);
    F.UR[d] = reinterpret_cast<float*>(B.UR[d]);
    F.F1[d] = reinterpret_cast<float*>(B.F1[d]);
  }
  F.rec = B.rec;
  return F;
}

template <int D>
__device__ __forceinline__ void load_prim_f(const float* __restrict__ W, long long ps, long long c,
                                            float w[5]) {
  w[0] = W[c];
  w[1] = W[(1 + Perm<D>::n) * ps + c];
  w[2] = W[(1 + Perm<D>::t1) * ps + c];
  w[3] = W[(1 + Perm<D>::t2) * ps + c];
  w[4] = W[4 * ps + c];
}
template <int D>
__device__ __forceinline__ void store_rot_f(float* __restrict__ A, long long ps, long long c,
                                            const float v[5]) {
  A[c] = v[0];
  A[(1 + Perm<D>::n) * ps + c] = v[1];
  A[(1 + Perm<D>::t1) * ps + c] = v[2];
  A[(1 + Perm<D>::t2) * ps + c] = v[3];
  A[4 * ps + c] = v[4];
}

__device__ __forceinline__ void block_max_to(double v, unsigned long long* slot) {
  __shared__ double warp_max[kThreads / 32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = max_nonneg(v, __shfl_xor_sync(0xffffffffu, v, o));
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) warp_max[wid] = v;
  __syncthreads();
  if (wid == 0) {
    v = (lane < (int)(blockDim.x >> 5)) ? warp_max[lane] : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = max_nonneg(v, __shfl_xor_sync(0xffffffffu, v, o));
    if (lane == 0 && v > 0.0) atomicMax(slot, (unsigned long long)__double_as_longlong(v));
  }
}

// primitives in FP64 (ghosts by index remap, as in the FP64 path), stored as
// float; dt reduction in FP64
__device__ __forceinline__ double prims_mixed_body(const Geom& G, const BufsF& B, const BcDesc& bc,
                                                   const GasD& g, int want_dt, long long t) {
  double local = 0.0;
  {
    int c[3];
    padded_coords(G, t, c);
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
        case 0: src[d] = lo ? n - depth : depth - 1; break;
        case 1: src[d] = lo ? depth - 1 : n - depth; neg |= 1 << d; break;
        case 2: src[d] = lo ? 0 : n - 1; break;
        default: src[d] = 0; inflow_face = face; neg = 0; break;
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
    // 1/rho: float reciprocal of the rounded density refined by one Newton
    // step r <- r + r (1 - rho r) in FP64 (relative error below 2^-44)
    const float df = d2f(U[0]);
    const float rf = __frcp_rn(df);
    double r = f2d(rf);
    r = fma(r, fma(-U[0], r, 1.0), r);
    double v[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) v[d] = U[1 + d] * r;
    // FP64 internal energy E - (rho v) . v / 2 and the pressure floor
    const double ke2 = U[1] * v[0] + U[2] * v[1] + U[3] * v[2];
    const double p = vmax<false>(g.gm1 * fma(-0.5, ke2, U[4]), kPFloor);
    // a = sqrt(gamma p / rho): float reciprocal square root of x = a^2 refined
    // by one Newton step, a = x y (1 + (1 - x y^2)/2) (relative error ~1e-13)
    const double x = g.gamma * p * r;
    const double y = f2d(rsqrtf(d2f(x)));
    const double xy = x * y;
    const double a = fma(0.5 * xy, fma(-xy, y, 1.0), xy);
    const float af = d2f(a);
    B.W[t] = df;
#pragma unroll
    for (int d = 0; d < 3; ++d) B.W[(1 + d) * G.ps + t] = d2f(v[d]);
    B.W[4 * G.ps + t] = d2f(p);
    B.W[5 * G.ps + t] = af;
    B.W[6 * G.ps + t] = __frcp_rn(af);
    B.W[7 * G.ps + t] = rf;
    if (want_dt && real) {
#pragma unroll
      for (int d = 0; d < 3; ++d)
        if (G.n[d] > 1) local = max_nonneg(local, fabs(v[d]) + a);
    }
  }
  return local;
}

template <int BS>
__global__ void __launch_bounds__(BS) kb_prims_mixed(BatchLaunch L) {
  const BatchItem it = batch_item(L);
  const Geom& G = it.d->G;
  const BufsF F = float_view(it.d->B);
  const long long total = (long long)G.N[0] * G.N[1] * G.N[2];
  const double local = (it.t < total) ? prims_mixed_body(G, F, it.d->bc, it.d->gd, 1, it.t) : 0.0;
  block_max_to(local, reinterpret_cast<unsigned long long*>(F.rec));
}

template <int D>
__device__ __forceinline__ void ppmc_mixed_body(const Geom& G, const BufsF& B, const Box& box,
    long long t) {
  int c3[3];
  box_coords(box, t, c3);
  const long long c = pidx(G, c3);
  const long long s = G.s[D];
  // the limited slopes of cells c-1, c, c+1 are formed here in float (cheap
  // next to the FP64 stages) rather than read from a slope pass: this saves
  // the slope planes' HBM round trip and a launch per axis
  float w2m[5], wm[5], wc[5], wp[5], w2p[5], sm[5], sc[5], sp[5];
  load_prim_f<D>(B.W, G.ps, c - 2 * s, w2m);
  load_prim_f<D>(B.W, G.ps, c - s, wm);
  load_prim_f<D>(B.W, G.ps, c, wc);
  load_prim_f<D>(B.W, G.ps, c + s, wp);
  load_prim_f<D>(B.W, G.ps, c + 2 * s, w2p);
  limited_slope(w2m, wm, wc, B.W[5 * G.ps + c - s], B.W[6 * G.ps + c - s],
                B.W[7 * G.ps + c - s], sm);
  limited_slope(wm, wc, wp, B.W[5 * G.ps + c], B.W[6 * G.ps + c], B.W[7 * G.ps + c], sc);
  limited_slope(wc, wp, w2p, B.W[5 * G.ps + c + s], B.W[6 * G.ps + c + s],
                B.W[7 * G.ps + c + s], sp);
  const float dtdx = (float)B.rec[2];
  float WsL[5], WsR[5];
  ppmc_states(wm, wc, wp, sm, sc, sp, B.W[5 * G.ps + c], B.W[6 * G.ps + c], B.W[7 * G.ps + c],
              dtdx, WsL, WsR);
  store_rot_f<D>(B.UR[D], G.ps, c, WsL);
  store_rot_f<D>(B.UL[D], G.ps, c + s, WsR);
}


template <int D>
__device__ __forceinline__ void riemann1_mixed_body(const Geom& G, const BufsF& B, const Box& box, const GasF& g,
    long long t) {
  int c3[3];
  box_coords(box, t, c3);
  const long long f = pidx(G, c3);
  float WL[5], WR[5], F[5];
  load_prim_f<D>(B.UL[D], G.ps, f, WL);
  load_prim_f<D>(B.UR[D], G.ps, f, WR);
  const int fl = riemann_exact(WL, WR, 1.0f / WL[0], 1.0f / WR[0], g, F);
  store_rot_f<D>(B.F1[D], G.ps, f, F);
  if (fl) atomicOr(rec_flags(B.rec), fl);
}


// One side of a face at the transverse half-step (Eq. transverse_evolution):
// U^{n+1/2} = U* + h (G*(c) - G*(c + e_t1)) + h (H*(c) - H*(c + e_t2)), h =
// dt/(2 dx), accumulated in FP64 from the float face state W* (converted
// exactly to U*: rho v is an exact product of two floats, E from p/(gamma-1)
// and the kinetic energy) and the float flux differences, then the FP64
// recovery of its primitives: internal energy E - |m|^2/(2 rho) with 1/rho from
// a float seed and one Newton step (relative error below 2^-44).  The float
// difference of two float fluxes has the rounding error of the fluxes
// themselves.  Returns the primitives in sweep order and 1/rho, in float.
template <int D>
__device__ __forceinline__ void half_step_side(const Geom& G, const BufsF& B, const float* __restrict__ Ws,
                                               long long f, long long c, double h, const GasD& gd,
                                               float w[5], float& inv_d) {
  const long long ps = G.ps;
  double U[5];
  {
    const double d = f2d(Ws[f]);
    double v[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      v[i] = f2d(Ws[(1 + i) * ps + f]);
      U[1 + i] = d * v[i];
    }
    const double ke2 = U[1] * v[0] + U[2] * v[1] + U[3] * v[2];
    U[0] = d;
    U[4] = fma(0.5, ke2, f2d(Ws[4 * ps + f]) * gd.inv_gm1);
  }
  constexpr int T1 = Perm<D>::t1, T2 = Perm<D>::t2;
  if (G.n[T1] > 1) {
    const float* F = B.F1[T1];
    const long long st = G.s[T1];
#pragma unroll
    for (int q = 0; q < 5; ++q) U[q] = fma(h, f2d(F[q * ps + c] - F[q * ps + c + st]), U[q]);
  }
  if (G.n[T2] > 1) {
    const float* F = B.F1[T2];
    const long long st = G.s[T2];
#pragma unroll
    for (int q = 0; q < 5; ++q) U[q] = fma(h, f2d(F[q * ps + c] - F[q * ps + c + st]), U[q]);
  }
  const float df = d2f(U[0]);
  const float rf = __frcp_rn(df);
  double r = f2d(rf);
  r = fma(r, fma(-U[0], r, 1.0), r);
  const double m2 = U[1] * U[1] + U[2] * U[2] + U[3] * U[3];
  const double p = gd.gm1 * fma(-0.5 * m2, r, U[4]);
  // the floor applied to the rounded pressure equals the rounded floored
  // pressure: rounding is monotonic, so it commutes with the maximum
  w[0] = df;
  w[1] = d2f(U[1 + D]) * rf;
  w[2] = d2f(U[1 + T1]) * rf;
  w[3] = d2f(U[1 + T2]) * rf;
  w[4] = tmax(d2f(p), (float)kPFloor);
  inv_d = rf;
}

// transverse half-step in FP64, second Riemann solve in float
template <int D>
__device__ __forceinline__ void riemann2_mixed_body(const Geom& G, const BufsF& B, const Box& box, const GasD& gd, const GasF& g,
    long long t) {
  int c3[3];
  box_coords(box, t, c3);
  const long long f = pidx(G, c3);
  const double h = B.rec[3];
  float wl[5], wr[5], idL, idR, Fx[5];
  half_step_side<D>(G, B, B.UL[D], f, f - G.s[D], h, gd, wl, idL);
  half_step_side<D>(G, B, B.UR[D], f, f, h, gd, wr, idR);
  const int fl = riemann_exact(wl, wr, idL, idR, g, Fx);
  store_rot_f<D>(B.UL[D], G.ps, f, Fx);
  if (fl) atomicOr(rec_flags(B.rec), fl);
}


// conserved update in FP64 from the float CTU fluxes
__device__ __forceinline__ void update_mixed_body(const Geom& G, const BufsF& B, long long t) {
  const long long c = real_to_padded(G, t);
  const double dtdx = B.rec[2];
  int fl = 0;
#pragma unroll
  for (int q = 0; q < 5; ++q) {
    double un = B.u[q * G.nreal + t];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      if (G.n[d] > 1) {
        const float* F = B.UL[d];
        un = un + dtdx * (f2d(F[q * G.ps + c]) - f2d(F[q * G.ps + c + G.s[d]]));
      }
    }
    B.u[q * G.nreal + t] = un;
    const long long b = __double_as_longlong(un);
    if ((b & 0x7fffffffffffffffLL) > 0x7ff0000000000000LL) fl = kFlagNonPhys;  // NaN
    if (q == 0 && b <= 0) fl = kFlagNonPhys;  // rho <= 0 (or a NaN with the sign bit)
  }
  if (fl) atomicOr(rec_flags(B.rec), fl);
}


template <int BS>
__global__ void __launch_bounds__(BS) kb_update_mixed(BatchLaunch L) {
  const BatchItem it = batch_item(L);
  if (it.t < it.d->G.nreal) update_mixed_body(it.d->G, float_view(it.d->B), it.t);
}

#define HYDRO_BATCH_MIXED(NAME, STAGE_IDX, CALL)                                           \
  template <int D, int BS>                                                                  \
  __global__ void __launch_bounds__(BS, kMinBlocksMixed * kThreads / BS) NAME(BatchLaunch L) {  \
    const BatchItem it = batch_item(L);                                                     \
    const Box& box = it.d->box[STAGE_IDX][D];                                               \
    if (it.t < (long long)box.n[0] * box.n[1] * box.n[2]) {                                 \
      const BufsF F = float_view(it.d->B);                                                  \
      CALL;                                                                                 \
    }                                                                                       \
  }
HYDRO_BATCH_MIXED(kb_ppmc_mixed, 1, ppmc_mixed_body<D>(it.d->G, F, box, it.t))
HYDRO_BATCH_MIXED(kb_riemann1_mixed, 2, riemann1_mixed_body<D>(it.d->G, F, box, it.d->gf, it.t))
HYDRO_BATCH_MIXED(kb_riemann2_mixed, 3,
                  riemann2_mixed_body<D>(it.d->G, F, box, it.d->gd, it.d->gf, it.t))
#undef HYDRO_BATCH_MIXED


}  // namespace

cudaError_t batch_prims_mixed(const BatchLaunch& L, int bs, unsigned blocks, cudaStream_t st) {
  if (blocks == 0) return cudaSuccess;
  if (bs == 128)
    kb_prims_mixed<128><<<blocks, 128, 0, st>>>(L);
  else
    kb_prims_mixed<256><<<blocks, 256, 0, st>>>(L);
  return cudaGetLastError();
}

cudaError_t batch_update_mixed(const BatchLaunch& L, int bs, unsigned blocks, cudaStream_t st) {
  if (blocks == 0) return cudaSuccess;
  if (bs == 128)
    kb_update_mixed<128><<<blocks, 128, 0, st>>>(L);
  else
    kb_update_mixed<256><<<blocks, 256, 0, st>>>(L);
  return cudaGetLastError();
}

cudaError_t batch_stage_mixed(const BatchLaunch& L, int stage, int axis, int bs, unsigned blocks,
                              cudaStream_t st) {
  if (blocks == 0) return cudaSuccess;
#define HYDRO_BATCH_MIXED_AXIS(K)                                                   \
  if (bs == 128) {                                                                  \
    switch (axis) {                                                                 \
      case 0: K<0, 128><<<blocks, 128, 0, st>>>(L); break;                         \
      case 1: K<1, 128><<<blocks, 128, 0, st>>>(L); break;                         \
      default: K<2, 128><<<blocks, 128, 0, st>>>(L); break;                        \
    }                                                                               \
  } else {                                                                          \
    switch (axis) {                                                                 \
      case 0: K<0, 256><<<blocks, 256, 0, st>>>(L); break;                         \
      case 1: K<1, 256><<<blocks, 256, 0, st>>>(L); break;                         \
      default: K<2, 256><<<blocks, 256, 0, st>>>(L); break;                        \
    }                                                                               \
  }
  switch (stage) {
    case kStageSlopes: return cudaSuccess;  // formed inside the PPMC kernel
    case kStagePpmc: HYDRO_BATCH_MIXED_AXIS(kb_ppmc_mixed) break;
    case kStageRiemann1: HYDRO_BATCH_MIXED_AXIS(kb_riemann1_mixed) break;
    case kStageRiemann2: HYDRO_BATCH_MIXED_AXIS(kb_riemann2_mixed) break;
    default: return cudaErrorInvalidValue;
  }
#undef HYDRO_BATCH_MIXED_AXIS
  return cudaGetLastError();
}


}  // namespace hydro
