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

#include "../../include/hydro.h"
#include "hydro_kernels.cuh"
#include "hydro_run.h"

namespace hydro {
namespace {

// block-wide maximum of a non-negative double (NaN ignored), then one
// atomicMax on its bits (non-negative doubles order like their bit patterns)
template <bool S>
__device__ __forceinline__ void block_max_to(double v, unsigned long long* slot) {
  __shared__ double warp_max[kThreads / 32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const double w = __shfl_xor_sync(0xffffffffu, v, o);
    v = max_nn<S>(v, w);
  }
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) warp_max[wid] = v;
  __syncthreads();
  if (wid == 0) {
    v = (lane < (int)(blockDim.x >> 5)) ? warp_max[lane] : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const double w = __shfl_xor_sync(0xffffffffu, v, o);
      v = max_nn<S>(v, w);
    }
    if (lane == 0 && v > 0.0) atomicMax(slot, (unsigned long long)__double_as_longlong(v));
  }
}

// ---------------------------------------------------------------------------
// Primitives of every padded cell.  A ghost cell takes the value the
// boundary passes x, then y, then z would give it (boundary_state).
// returns this cell's |v_d| + a maximum (0 for ghosts or when !want_dt).
// S (strict): the CPU reference's operation order with IEEE divisions and
// square root; otherwise 1/rho and 1/a by Newton iteration (nr_rcp, nr_rsqrt)
// and fused multiply-adds.
template <bool S, bool NOH>
__device__ __forceinline__ double prims_body(const Geom& G, const Bufs& B, const BcDesc& bc,
                                             const Gas& g, int want_dt, long long t) {
  double local = 0.0;
  {
    int c[3];
    padded_coords(G, t, c);
    double U[5];
    int neg;
    const bool real = boundary_state<NOH>(G, B.u, bc, g.gm1, B.rec[5], c, U, neg);
#pragma unroll
    for (int d = 0; d < 3; ++d)
      if (neg & (1 << d)) U[1 + d] = -U[1 + d];
    // primitives, then the per-cell reciprocals the later stages multiply by
    const double d = U[0];
    double W[5], a, inv_a, inv_d;
    W[0] = d;
    if constexpr (S) {  // the CPU reference's operation order (divisions)
      W[1] = U[1] / d;
      W[2] = U[2] / d;
      W[3] = U[3] / d;
      W[4] = tmax(g.gm1 * (U[4] - 0.5 * d * (W[1] * W[1] + W[2] * W[2] + W[3] * W[3])), kPFloor);
      a = sqrt(g.gamma * W[4] / d);
      inv_a = 1.0 / a;
      inv_d = 1.0 / d;
    } else {  // E - (rho v).v/2 with v = (rho v)/rho; a = x/sqrt(x), x = gamma p/rho
      inv_d = nr_rcp(d);
      W[1] = U[1] * inv_d;
      W[2] = U[2] * inv_d;
      W[3] = U[3] * inv_d;
      const double ke2 = fma(U[1], W[1], fma(U[2], W[2], U[3] * W[3]));
      W[4] = vmax<false>(g.gm1 * fma(-0.5, ke2, U[4]), kPFloor);
      const double x = g.gamma * W[4] * inv_d;
      inv_a = nr_rsqrt(x);
      a = x * inv_a;
    }
#pragma unroll
    for (int q = 0; q < 5; ++q) B.W[q * G.ps + t] = W[q];
    B.W[5 * G.ps + t] = a;
    B.W[6 * G.ps + t] = inv_a;
    B.W[7 * G.ps + t] = inv_d;
    // Eq. calc_dt_3D: min over cells and axes of dx/(|v_d| + a) equals
    // dx / max(|v_d| + a) exactly, because rounding and the quotient are
    // monotone; so the cells contribute a maximum and one division follows
    if (want_dt && real) {
      if constexpr (S) {
#pragma unroll
        for (int d = 0; d < 3; ++d)
          if (G.n[d] > 1) local = tmax(local, fabs(W[1 + d]) + a);
      } else {
        // max_d (|v_d| + a) as (max_d |v_d|) + a, the same double (adding a
        // is monotone under rounding): the maximum on the integer pipe, one
        // FP64 add; a NaN counts as absent, as in the maxima
        double vm = 0.0;
#pragma unroll
        for (int d = 0; d < 3; ++d)
          if (G.n[d] > 1) vm = max_nonneg(vm, vabs<false>(W[1 + d]));
        local = max_nonneg(local, vm + a);
      }
    }
  }
  return local;
}

template <bool NOH>
__global__ void __launch_bounds__(kThreads) k_prims(Geom G, Bufs B, BcDesc bc, Gas g, int want_dt) {
  const long long total = (long long)G.N[0] * G.N[1] * G.N[2];
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const double local = (t < total) ? prims_body<true, NOH>(G, B, bc, g, want_dt, t) : 0.0;
  if (want_dt) block_max_to<true>(local, reinterpret_cast<unsigned long long*>(B.rec));
}

template <int BS, bool NOH>
__global__ void __launch_bounds__(BS) kb_prims(BatchLaunch L) {
  const BatchItem it = batch_item(L);
  const Geom& G = it.d->G;
  const long long total = (long long)G.N[0] * G.N[1] * G.N[2];
  const double local =
      (it.t < total) ? prims_body<false, NOH>(G, it.d->B, it.d->bc, it.d->gd, 1, it.t) : 0.0;
  block_max_to<false>(local, reinterpret_cast<unsigned long long*>(it.d->B.rec));
}

// advance: the step's time advance t <- t + dt (record [5]); the step's
// primitive kernel has read t by then, the next step's reads t + dt
__global__ void k_set_dt(double* rec, double cfl, double fixed_dt, double dx, int advance) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    const double dt = (fixed_dt > 0.0) ? fixed_dt : cfl * (dx / rec[0]);
    const double dtdx = dt / dx;
    rec[1] = dt;
    rec[2] = dtdx;
    rec[3] = 0.5 * dtdx;
    if (advance) rec[5] = rec[5] + dt;
  }
}

// Device-driven runs (hydro_run.h: a CUDA graph whose WHILE node repeats the
// step).  The step's dt is the CFL dt cut back to reach the end time exactly,
// the host loop's rule: t + dt >= t_end gives dt = t_end - t and t = t_end.
__global__ void k_set_dt_to_end(double* rec, double cfl, double dx) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    double dt = cfl * (dx / rec[0]);
    const double t = rec[5], t_end = rec[8];
    const bool last = t + dt >= t_end;
    if (last) dt = t_end - t;
    const double dtdx = dt / dx;
    rec[1] = dt;
    rec[2] = dtdx;
    rec[3] = 0.5 * dtdx;
    rec[5] = last ? t_end : t + dt;
  }
}

// the loop runs while t < t_end, steps are left and no step raised a flag;
// at most `chunk` steps a graph launch bound the time one launch holds the GPU
__global__ void k_run_begin(double* rec, cudaGraphConditionalHandle cond) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    rec[10] = 0.0;
    cudaGraphSetConditional(cond, (rec[5] < rec[8] && rec[9] >= 1.0) ? 1u : 0u);
  }
}

__global__ void k_run_next(double* rec, cudaGraphConditionalHandle cond, double chunk) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    const int flags = *rec_flags(rec);
    const double left = rec[9] - 1.0, taken = rec[10] + 1.0;
    rec[9] = left;
    rec[10] = taken;
    const bool go = flags == 0 && rec[5] < rec[8] && left >= 1.0 && taken < chunk;
    cudaGraphSetConditional(cond, go ? 1u : 0u);
  }
}

// S (strict): u + dt/dx (F_- - F_+) rounded as the CPU reference rounds it;
// otherwise with a fused multiply-add and the NaN test on the bit pattern
template <bool S>
__device__ __forceinline__ void update_body(const Geom& G, const Bufs& B, long long t) {
  const long long c = real_to_padded(G, t);
  const double dtdx = B.rec[2];
  int fl = 0;
#pragma unroll
  for (int q = 0; q < 5; ++q) {
    double un = B.u[q * G.nreal + t];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      if (G.n[d] > 1) {
        const double* F = B.UL[d];
        if constexpr (S)
          un = un + dtdx * (F[q * G.ps + c] - F[q * G.ps + c + G.s[d]]);
        else
          un = fma(dtdx, F[q * G.ps + c] - F[q * G.ps + c + G.s[d]], un);
      }
    }
    B.u[q * G.nreal + t] = un;
    if constexpr (S) {
      if (isnan(un)) fl = kFlagNonPhys;
      if (q == 0 && !(un > 0.0)) fl = kFlagNonPhys;
    } else {
      const long long b = __double_as_longlong(un);
      if ((b & 0x7fffffffffffffffLL) > 0x7ff0000000000000LL) fl = kFlagNonPhys;  // NaN
      if (q == 0 && b <= 0) fl = kFlagNonPhys;  // rho <= 0 (or a NaN with the sign bit)
    }
  }
  if (fl) atomicOr(rec_flags(B.rec), fl);
}

__global__ void __launch_bounds__(kThreads) k_update(Geom G, Bufs B) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t < G.nreal) update_body<true>(G, B, t);
}

template <int BS>
__global__ void __launch_bounds__(BS) kb_update(BatchLaunch L) {
  const BatchItem it = batch_item(L);
  if (it.t < it.d->G.nreal) update_body<false>(it.d->G, it.d->B, it.t);
}

// per grid: dt = cfl * dx / max(|v_d| + a) (or the fixed dt), dt/dx, history
__global__ void k_batch_set_dt(const GridDesc* descs, int ngrids, double cfl, double* dt_hist) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= ngrids) return;
  double* rec = descs[i].B.rec;
  const double dx = descs[i].G.dx;
  const double dt = cfl * (dx / rec[0]);
  const double dtdx = dt / dx;
  rec[0] = 0.0;  // the next step's primitive kernel reduces into a zeroed slot
  rec[1] = dt;
  rec[2] = dtdx;
  rec[3] = 0.5 * dtdx;
  rec[5] = rec[5] + dt;  // the grid's time
  if (dt_hist) dt_hist[i] = dt;
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


}  // namespace

cudaError_t fp64_prims(const Geom& G, const Bufs& B, const BcDesc& bc, double gamma, bool want_dt,
                       cudaStream_t st) {
  if (want_dt) {
    cudaError_t e = cudaMemsetAsync(B.rec, 0, sizeof(double), st);
    if (e != cudaSuccess) return e;
  }
  const long long total = (long long)G.N[0] * G.N[1] * G.N[2];
  if (has_noh(bc))
    k_prims<true><<<blocks_for(total), kThreads, 0, st>>>(G, B, bc, make_gas<double>(gamma),
                                                          want_dt ? 1 : 0);
  else
    k_prims<false><<<blocks_for(total), kThreads, 0, st>>>(G, B, bc, make_gas<double>(gamma),
                                                           want_dt ? 1 : 0);
  return cudaGetLastError();
}

cudaError_t fp64_set_dt(const Geom& G, const Bufs& B, double cfl, double fixed_dt, cudaStream_t st,
                        bool advance_time) {
  k_set_dt<<<1, 32, 0, st>>>(B.rec, cfl, fixed_dt, G.dx, advance_time ? 1 : 0);
  return cudaGetLastError();
}

cudaError_t set_dt_to_end(const Geom& G, const Bufs& B, double cfl, cudaStream_t st) {
  k_set_dt_to_end<<<1, 32, 0, st>>>(B.rec, cfl, G.dx);
  return cudaGetLastError();
}

cudaError_t run_begin(double* rec, cudaGraphConditionalHandle cond, cudaStream_t st) {
  k_run_begin<<<1, 32, 0, st>>>(rec, cond);
  return cudaGetLastError();
}

cudaError_t run_next(double* rec, cudaGraphConditionalHandle cond, double chunk, cudaStream_t st) {
  k_run_next<<<1, 32, 0, st>>>(rec, cond, chunk);
  return cudaGetLastError();
}

Box stage_box_of(const Geom& G, int stage, int axis) { return stage_box(G, stage, axis); }

void fill_desc(GridDesc& d, double gamma) {
  d.gd = make_gas<double>(gamma);
  d.gf = make_gas<float>(gamma);
  for (int s = kStageSlopes; s <= kStageRiemann2; ++s)
    for (int a = 0; a < 3; ++a) d.box[s - kStageSlopes][a] = stage_box(d.G, s, a);
  for (int a = 0; a < 3; ++a) {
    for (int which = 0; which < 2; ++which) {
      Box b = d.box[(which ? kStageRiemann2 : kStagePpmc) - kStageSlopes][a];
      b.n[a] = (b.n[a] + kPpmcSeg - 1) / kPpmcSeg;
      b.div0 = make_fastdiv((unsigned)b.n[0]);
      b.div01 = make_fastdiv((unsigned)b.n[0] * (unsigned)b.n[1]);
      (which ? d.seg2 : d.seg)[a] = b;
    }
  }
}

bool build_launch_tables(const GridDesc* desc, const int* order, int n, int bs, int* tab,
                         unsigned* blocks) {
  for (int k = 0; k < kLaunchKinds; ++k) {
    long long acc = 0;
    for (int i = 0; i < n; ++i) {
      const GridDesc& g = desc[order[i]];
      long long units;
      if (k == 0) {
        units = (long long)g.G.N[0] * g.G.N[1] * g.G.N[2];
      } else if (k == 1) {
        units = g.G.nreal;
      } else if (k >= ppmc_seg_kind(1)) {
        // kPpmcSegThreads a block whatever bs is: one compiled kernel, so the
        // rounding of its fused multiply-adds does not depend on the schedule
        const bool r2 = k >= riemann2_seg_kind(1);
        const int axis = k - (r2 ? riemann2_seg_kind(1) : ppmc_seg_kind(1)) + 1;
        const long long segs = g.G.n[axis] > 1 ? box_count((r2 ? g.seg2 : g.seg)[axis]) : 0;
        units = (segs + kPpmcSegThreads - 1) / kPpmcSegThreads * bs;
      } else {
        const int stage = kStageSlopes + (k - 2) / 3, axis = (k - 2) % 3;
        units = g.G.n[axis] > 1 ? box_count(g.box[stage - kStageSlopes][axis]) : 0;
      }
      tab[(size_t)k * (n + 1) + i] = (int)acc;
      acc += (units + bs - 1) / bs;
    }
    if (acc > 0x7fffffffLL) return false;
    tab[(size_t)k * (n + 1) + n] = (int)acc;
    blocks[k] = (unsigned)acc;
  }
  for (int i = 0; i < n; ++i) tab[(size_t)kLaunchKinds * (n + 1) + i] = order[i];
  return true;
}

long long stage_units(const Geom& G, int stage, int axis) {
  if (stage == kStagePrims) return (long long)G.N[0] * G.N[1] * G.N[2];
  if (stage == kStageUpdate) return G.nreal;
  if (stage == kStageSetDt) return 1;
  return box_count(stage_box(G, stage, axis));
}

cudaError_t fp64_stage_strict(const Geom& G, const Bufs& B, int recon, int solver, int stage,
                              int axis, double gamma, cudaStream_t st) {
  return launch_axis_stage<true>(G, B, recon, solver, stage, axis, gamma, st);
}

cudaError_t batch_prims(const BatchLaunch& L, int precision, int bs, unsigned blocks, cudaStream_t st,
                        bool noh) {
  if (precision == HYDRO_MIXED) return batch_prims_mixed(L, bs, blocks, st, noh);
  if (blocks == 0) return cudaSuccess;
  if (bs == 128) {
    if (noh)
      kb_prims<128, true><<<blocks, 128, 0, st>>>(L);
    else
      kb_prims<128, false><<<blocks, 128, 0, st>>>(L);
  } else {
    if (noh)
      kb_prims<256, true><<<blocks, 256, 0, st>>>(L);
    else
      kb_prims<256, false><<<blocks, 256, 0, st>>>(L);
  }
  return cudaGetLastError();
}

cudaError_t batch_update(const BatchLaunch& L, int precision, int bs, unsigned blocks,
                         cudaStream_t st) {
  if (precision == HYDRO_MIXED) return batch_update_mixed(L, bs, blocks, st);
  if (blocks == 0) return cudaSuccess;
  if (bs == 128)
    kb_update<128><<<blocks, 128, 0, st>>>(L);
  else
    kb_update<256><<<blocks, 256, 0, st>>>(L);
  return cudaGetLastError();
}

cudaError_t batch_set_dt(const GridDesc* descs, int ngrids, double cfl, double* dt_hist,
                         cudaStream_t st) {
  k_batch_set_dt<<<(ngrids + 127) / 128, 128, 0, st>>>(descs, ngrids, cfl, dt_hist);
  return cudaGetLastError();
}

cudaError_t batch_stage(const BatchLaunch& L, int precision, int recon, int solver, int stage,
                        int axis, int bs, unsigned blocks, cudaStream_t st) {
  return precision == HYDRO_MIXED
             ? batch_stage_mixed(L, stage, axis, bs, blocks, st)
             : batch_stage_fp64(L, recon, solver, stage, axis, bs, blocks, st);
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
