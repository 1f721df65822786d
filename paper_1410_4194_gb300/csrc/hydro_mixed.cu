// hydro_mixed.cu -- the mixed-precision CTU step (HYDRO_MIXED).
//
// Float32: the characteristic slopes, PPMC reconstruction and tracing, and both
// sets of exact Riemann solves (App. A.2, A.3, B.1) -- the bulk of the
// arithmetic, on GB300's FP32 pipe (64 times the FP64 rate).
// Float, too: the transverse half-step (Eq. transverse_evolution), written for
// the increments of the face state so that its pressure recovery has no
// cancellation of total and kinetic energy (see half_step_side).
// Float64, where the step's stability needs it:
//   * primitives of the FP64 state: the internal energy, as rho E - |m|^2/2
//     (the cancellation of total and kinetic energy at high Mach), the
//     pressure floor and the CFL time-step reduction;
//   * the conserved update (Eq. conserved_update), accumulated from the float
//     CTU fluxes into the FP64 state.
// Intermediates (primitives, face states, fluxes) are float, in float4
// vector planes (see Face5), which halves their HBM traffic; the PPMC kernel
// forms the limited slopes it needs itself.  The float divisions and square
// roots of the solver are the SFU approximations (nr_* in hydro_math.cuh).
// Compiled with FMA contraction.
#include "../../include/hydro.h"
#include "hydro_ffsum.cuh"
#include "hydro_kernels.cuh"

namespace hydro {
namespace {

using GasF = GasT<float>;
using GasD = GasT<double>;

// resident threads per SM for the stencil and Riemann stages, in units of 256
// (a block is 128 or 256 threads), by measurement on Sedov 256^3: PPMC at 4
// (64 registers; 3 is 6% slower; 5 takes 48 registers and spills, 1% faster on
// Sedov but 5% slower on Mach-5 turbulence), the first Riemann set at 6 (40 registers: its Newton
// iteration is a latency chain that more resident warps hide; 14% faster than
// at 4), the second with the bound of 3 (the compiler then takes 64 registers
// instead of 56 and the kernel runs 8% faster; 4 is slower), the primitives at
// 6 and the update at 6 (40 registers and a 56-byte spill, 4% faster than at 5,
// which was 14% faster than 4)
constexpr int kMinBlocksPpmc = 4, kMinBlocksRiemann1 = 6, kMinBlocksRiemann2 = 3;
constexpr int kMinBlocksPrims = 6, kMinBlocksUpdate = 6;

// A five-value face quantity (a primitive state or a flux, x/y/z components
// in axis order) in vector form: values 0-3 in one float4 plane, value 4 in
// one float plane.  A thread moves a face with one 16-byte and one 4-byte
// access, each coalesced across its warp, instead of five 4-byte ones.
struct Face5 {
  float4* v;
  float* e;
};
// The primitives of a padded cell as two float4 planes: (rho, vx, vy, vz) and
// (p, a, 1/a, 1/rho).
struct Prim8 {
  float4* a;
  float4* b;
};

// float views of the step's work arrays, carved from the same slab as the
// FP64 path (each FP64 array has room for its float vector form)
struct BufsF {
  double* u;      // FP64 state, real cells [5][nz][ny][nx]
  Prim8 W;        // padded primitives
  Face5 UL[3];    // per axis: left states W*_L of the faces; then F^{n+1/2}
  Face5 UR[3];    // per axis: right states W*_R of the faces
  Face5 F1[3];    // per axis: first fluxes F*
  double* rec;    // step record (dt, flags)
};

__host__ __device__ inline Face5 face_view(double* base, long long ps) {
  Face5 f;
  f.v = reinterpret_cast<float4*>(base);
  f.e = base ? reinterpret_cast<float*>(f.v + ps) : nullptr;
  return f;
}

__host__ __device__ inline BufsF float_view(const Bufs& B, long long ps) {
  BufsF F;
  F.u = B.u;
  F.W.a = reinterpret_cast<float4*>(B.W);
  F.W.b = F.W.a + ps;
  for (int d = 0; d < 3; ++d) {
    F.UL[d] = face_view(B.UL[d], ps);
    F.UR[d] = face_view(B.UR[d], ps);
    F.F1[d] = face_view(B.F1[d], ps);
  }
  F.rec = B.rec;
  return F;
}

// the primitives of cell c in sweep order, and a, 1/a, 1/rho
template <int D>
__device__ __forceinline__ void load_prim_f(const Prim8& W, long long c, float w[5], float& a,
                                            float& ia, float& ir) {
  const float4 x = __ldg(W.a + c), y = __ldg(W.b + c);
  const float v[3] = {x.y, x.z, x.w};
  w[0] = x.x;
  w[1] = v[Perm<D>::n];
  w[2] = v[Perm<D>::t1];
  w[3] = v[Perm<D>::t2];
  w[4] = y.x;
  a = y.y;
  ia = y.z;
  ir = y.w;
}
// a face quantity in axis order (flux differences) or in sweep order (states)
__device__ __forceinline__ void load_face_xyz(const Face5& A, long long c, float w[5]) {
  const float4 x = __ldg(A.v + c);
  w[0] = x.x;
  w[1] = x.y;
  w[2] = x.z;
  w[3] = x.w;
  w[4] = __ldg(A.e + c);
}
template <int D>
__device__ __forceinline__ void load_face(const Face5& A, long long c, float w[5]) {
  float x[5];
  load_face_xyz(A, c, x);
  w[0] = x[0];
  w[1] = x[1 + Perm<D>::n];
  w[2] = x[1 + Perm<D>::t1];
  w[3] = x[1 + Perm<D>::t2];
  w[4] = x[4];
}
template <int D>
__device__ __forceinline__ void store_face(const Face5& A, long long c, const float w[5]) {
  float x[3];
  x[Perm<D>::n] = w[1];
  x[Perm<D>::t1] = w[2];
  x[Perm<D>::t2] = w[3];
  A.v[c] = make_float4(w[0], x[0], x[1], x[2]);
  A.e[c] = w[4];
}

// What a cell keeps for the FP64 signal speed of the CFL condition.
struct DtCand {
  double m[3], d, re;  // momentum, density, rho times the internal energy
  float s;             // float estimate of max_d |v_d| + a; -1 for cells outside dt
};

// primitives from the FP64 state (ghosts by index remap, as in the FP64 path),
// stored as float.  The cancellation of total and kinetic energy at high Mach
// is taken in FP64: rho e = rho E - |m|^2/2, whose only rounding is that of
// its fused multiply-add (|m|^2/2 exact).  The division of rho e by rho that
// remains is well conditioned, so the pressure is (rho e)(gamma-1)/rho with
// the float reciprocal of the rounded density (five FP64 instructions a cell,
// where forming e = E - |m|^2 (1/rho)/2 needed an FP64 reciprocal first); the
// velocities and the sound speed are formed in float from rounded operands.
// Every stored value is within a few float ulps of its FP64 value.
template <bool NOH>
__device__ __forceinline__ void prims_mixed_body(const Geom& G, const BufsF& B, const BcDesc& bc,
                                                 const GasD& g, const GasF& gf, int want_dt,
                                                 long long t, DtCand& cand) {
  int c[3];
  padded_coords(G, t, c);
  double U[5];
  int neg;
  const bool real = boundary_state<NOH>(G, B.u, bc, g.gm1, B.rec[5], c, U, neg);
  // a reflected momentum is negated in float (U keeps the source cell's sign:
  // only |m|^2 and |v| use it in FP64)
  float mf[3];
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    mf[d] = d2f(U[1 + d]);
    if (neg & (1 << d)) mf[d] = -mf[d];
  }
  const float df = d2f(U[0]);
  const float rf = __frcp_rn(df);
  // FP64 rho e = rho E - |m|^2/2 (m2/2 exact), then the pressure and its floor
  const double m2 = fma(U[1], U[1], fma(U[2], U[2], U[3] * U[3]));
  const double re = fma(U[0], U[4], -half_bits(m2));
  const double p = vmax<false>(re * f2d(gf.gm1 * rf), kPFloor);
  const float pf = d2f(p);
  const float af = sqrtf(gf.gamma * pf * rf);
  float vf[3];
#pragma unroll
  for (int d = 0; d < 3; ++d) vf[d] = mf[d] * rf;
  B.W.a[t] = make_float4(df, vf[0], vf[1], vf[2]);
  B.W.b[t] = make_float4(pf, af, __frcp_rn(af), rf);
  cand.s = -1.f;
  if (want_dt && real) {
    float m = 0.f;
#pragma unroll
    for (int d = 0; d < 3; ++d)
      if (G.n[d] > 1) m = fmaxf(m, fabsf(vf[d]));
    cand.s = m + af;
#pragma unroll
    for (int d = 0; d < 3; ++d) cand.m[d] = U[1 + d];
    cand.d = U[0];
    cand.re = re;
  }
}

// FP64 signal speed max_d |v_d| + a of a cell: 1/rho (nr_rcp, to FP64
// precision), the floored pressure (gamma-1)(rho e)(1/rho), and a =
// sqrt(gamma p / rho) from a float reciprocal square root of x = a^2 refined
// by one Newton step, a = x y (1 + (1 - x y^2)/2) (relative error ~1e-13);
// max_d |v_d| as (max_d |m_d|)(1/rho) (multiplying by 1/rho > 0 is monotone,
// so the largest product is the product of the largest), the maximum on the
// integer pipe.  One lane a block takes this path, and each of its FP64
// instructions holds the FP64 pipe as long as a full warp's: eleven of them.
__device__ __forceinline__ double signal_speed_fp64(const Geom& G, const GasD& g, const DtCand& c) {
  const double r = nr_rcp(c.d);
  const double p = vmax<false>(g.gm1 * (c.re * r), kPFloor);
  const double x = g.gamma * p * r;
  const double y = f2d(rsqrtf(d2f(x)));
  const double xy = x * y;
  const double a = fma(half_bits(xy), fma(-xy, y, 1.0), xy);
  double mmax = 0.0;
#pragma unroll
  for (int d = 0; d < 3; ++d)
    if (G.n[d] > 1) mmax = max_nonneg(mmax, vabs<false>(c.m[d]));
  return mmax * r + a;
}

// The CFL reduction: each block evaluates the FP64 signal speed of one cell,
// the first (lowest thread) that holds the block's largest float estimate,
// and the grid takes the largest of those.  The float estimate of a cell is
// within 5 x 2^-24 of its FP64 value (roundings of m, p, 1/rho, gamma, the
// products, the square root and the sum), so the chosen cell's FP64 signal
// speed is within 10 x 2^-24 of the FP64 maximum, and is it exactly unless two
// cells' float estimates tie while their FP64 values differ (a uniform region
// ties with identical FP64 values).  A NaN estimate counts as absent, as in the FP64
// reduction.  The choice is a maximum over 64-bit keys, the estimate's bits
// (non-negative floats order like their bit patterns) above the complement of
// the thread index: one warp-shuffle reduction, each warp's winner parks its
// operands in shared memory, and a single barrier before warp 0 finishes.
template <int BS, bool NOH>
__global__ void __launch_bounds__(BS, kMinBlocksPrims * kThreads / BS) kb_prims_mixed(BatchLaunch L) {
  constexpr int kWarps = BS / 32;
  __shared__ unsigned long long warp_key[kWarps];
  __shared__ DtCand warp_cand[kWarps];
  const BatchItem it = batch_item(L);
  const Geom& G = it.d->G;
  const BufsF F = float_view(it.d->B, it.d->G.ps);
  const long long total = (long long)G.N[0] * G.N[1] * G.N[2];
  DtCand cand;
  cand.s = -1.f;
  if (it.t < total) prims_mixed_body<NOH>(G, F, it.d->bc, it.d->gd, it.d->gf, 1, it.t, cand);
  const unsigned long long key =
      (cand.s >= 0.f) ? ((unsigned long long)__float_as_uint(cand.s) << 32) | (~threadIdx.x & 0xffffffffu)
                      : 0ull;
  unsigned long long wk = key;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long other = __shfl_xor_sync(0xffffffffu, wk, o);
    wk = other > wk ? other : wk;
  }
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (key != 0ull && key == wk) {  // the warp's winner (keys are distinct)
    warp_key[wid] = wk;
    warp_cand[wid] = cand;
  } else if (wk == 0ull && lane == 0) {
    warp_key[wid] = 0ull;
  }
  __syncthreads();
  if (wid == 0) {
    const unsigned long long k = lane < kWarps ? warp_key[lane] : 0ull;
    unsigned long long bk = k;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const unsigned long long other = __shfl_xor_sync(0xffffffffu, bk, o);
      bk = other > bk ? other : bk;
    }
    if (bk != 0ull && k == bk) {
      const double sp = signal_speed_fp64(G, it.d->gd, warp_cand[lane]);
      if (sp > 0.0)
        atomicMax(reinterpret_cast<unsigned long long*>(F.rec),
                  (unsigned long long)__double_as_longlong(sp));
    }
  }
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
  float a2m, ia2m, ir2m, am, iam, irm, ac, iac, irc, ap, iap, irp, a2p, ia2p, ir2p;
  load_prim_f<D>(B.W, c - 2 * s, w2m, a2m, ia2m, ir2m);
  load_prim_f<D>(B.W, c - s, wm, am, iam, irm);
  load_prim_f<D>(B.W, c, wc, ac, iac, irc);
  load_prim_f<D>(B.W, c + s, wp, ap, iap, irp);
  load_prim_f<D>(B.W, c + 2 * s, w2p, a2p, ia2p, ir2p);
  limited_slope(w2m, wm, wc, am, iam, irm, sm);
  limited_slope(wm, wc, wp, ac, iac, irc, sc);
  limited_slope(wc, wp, w2p, ap, iap, irp, sp);
  const float dtdx = (float)B.rec[2];
  float WsL[5], WsR[5];
  ppmc_states(wm, wc, wp, sm, sc, sp, ac, iac, irc, dtdx, WsL, WsR);
  store_face<D>(B.UR[D], c, WsL);
  store_face<D>(B.UL[D], c + s, WsR);
}


// PPMC along y or z for a segment of up to kPpmcSeg consecutive cells of a
// column: the thread keeps a sliding window of primitives and limited slopes in
// registers, so a segment of K cells loads K + 4 cells (instead of 5K) and forms
// K + 2 limited slopes (instead of 3K).  The cells of a warp are 32 x-adjacent
// columns, so every load and store stays a coalesced row.  Per cell the same
// formulas as ppmc_mixed_body (the compiler may fuse a different set of
// multiply-adds in the two kernels, so the face states agree to rounding).
// Measured on Sedov 256^3 against one thread a cell: a y or z sweep 0.368 ->
// 0.347 ms; K = 2 and K = 8 (107 registers) gained less.
template <int D>
__device__ __forceinline__ void ppmc_mixed_seg_body(const Geom& G, const BufsF& B, const Box& seg,
                                                    const Box& box, long long t) {
  int c3[3];
  box_coords(seg, t, c3);
  const int k0 = box.lo[D] + (c3[D] - seg.lo[D]) * kPpmcSeg;  // first cell along D
  const int kn = min(kPpmcSeg, box.lo[D] + box.n[D] - k0);     // cells in this segment
  c3[D] = k0;
  const long long s = G.s[D];
  const long long c0 = pidx(G, c3);
  const float dtdx = (float)B.rec[2];
  // window: cells k-1, k, k+1 (primitives, a, 1/a, 1/rho) and their slopes
  float wm[5], wc[5], wp[5], sm[5], sc[5], sp[5];
  float am, iam, irm, ac, iac, irc, ap, iap, irp;
  {
    float w2[5], a2, ia2, ir2;
    load_prim_f<D>(B.W, c0 - 2 * s, w2, a2, ia2, ir2);
    load_prim_f<D>(B.W, c0 - s, wm, am, iam, irm);
    load_prim_f<D>(B.W, c0, wc, ac, iac, irc);
    load_prim_f<D>(B.W, c0 + s, wp, ap, iap, irp);
    limited_slope(w2, wm, wc, am, iam, irm, sm);
    limited_slope(wm, wc, wp, ac, iac, irc, sc);
  }
#pragma unroll
  for (int k = 0; k < kPpmcSeg; ++k) {
    if (k >= kn) break;
    const long long c = c0 + k * s;
    float w2p[5], a2p, ia2p, ir2p;
    load_prim_f<D>(B.W, c + 2 * s, w2p, a2p, ia2p, ir2p);
    limited_slope(wc, wp, w2p, ap, iap, irp, sp);
    float WsL[5], WsR[5];
    ppmc_states(wm, wc, wp, sm, sc, sp, ac, iac, irc, dtdx, WsL, WsR);
    store_face<D>(B.UR[D], c, WsL);
    store_face<D>(B.UL[D], c + s, WsR);
    // slide the window by one cell
#pragma unroll
    for (int q = 0; q < 5; ++q) {
      wm[q] = wc[q];
      wc[q] = wp[q];
      wp[q] = w2p[q];
      sm[q] = sc[q];
      sc[q] = sp[q];
    }
    am = ac; iam = iac; irm = irc;
    ac = ap; iac = iap; irc = irp;
    ap = a2p; iap = ia2p; irp = ir2p;
  }
}

template <int D>
__device__ __forceinline__ void riemann1_mixed_body(const Geom& G, const BufsF& B, const Box& box, const GasF& g,
    long long t) {
  int c3[3];
  box_coords(box, t, c3);
  const long long f = pidx(G, c3);
  float WL[5], WR[5], F[5];
  load_face<D>(B.UL[D], f, WL);
  load_face<D>(B.UR[D], f, WR);
  const int fl = riemann_exact(WL, WR, nr_rcp(WL[0]), nr_rcp(WR[0]), g, F);
  store_face<D>(B.F1[D], f, F);
  if (fl) atomicOr(rec_flags(B.rec), fl);
}


// One side of a face at the transverse half-step (Eq. transverse_evolution):
// U^{n+1/2} = U* + h (G*(c) - G*(c + e_t1)) + h (H*(c) - H*(c + e_t2)), h =
// dt/(2 dx), in float, written for the increments dU = (d rho, d m, d E) so
// that no total or kinetic energy of the state is ever formed.  With v the
// velocity of the face state W*, rho' = rho + d rho and q = d m - v d rho:
//   v' = v + q / rho'
//   p' = p + (gamma - 1) (dE - v.q - |v|^2 d rho / 2 - |q|^2 / (2 rho'))
// which is the primitive recovery of U* + dU rearranged exactly (the kinetic
// energy |m'|^2 / (2 rho') expanded about |m|^2 / (2 rho)).  The internal
// energy is then never the small difference of two large energies: every term
// is an increment of the size of the flux differences, whose float rounding
// (the fluxes are float) already bounds the result's accuracy.  Returns the
// primitives in sweep order and 1/rho', in float.
template <int D>
__device__ __forceinline__ void half_step_side(const Geom& G, const BufsF& B, const Face5& Ws,
                                               long long f, long long c, float h, const GasF& g,
                                               float w[5], float& inv_d) {
  float ws[5];  // the face state, x/y/z velocity order
  load_face_xyz(Ws, f, ws);
  const float d = ws[0];
  const float v[3] = {ws[1], ws[2], ws[3]};
  const float p = ws[4];
  float dU[5] = {0.f, 0.f, 0.f, 0.f, 0.f};
  constexpr int T1 = Perm<D>::t1, T2 = Perm<D>::t2;
  if (G.n[T1] > 1) {
    float a[5], b[5];
    load_face_xyz(B.F1[T1], c, a);
    load_face_xyz(B.F1[T1], c + G.s[T1], b);
#pragma unroll
    for (int q = 0; q < 5; ++q) dU[q] = h * (a[q] - b[q]);
  }
  if (G.n[T2] > 1) {
    float a[5], b[5];
    load_face_xyz(B.F1[T2], c, a);
    load_face_xyz(B.F1[T2], c + G.s[T2], b);
#pragma unroll
    for (int q = 0; q < 5; ++q) dU[q] = fmaf(h, a[q] - b[q], dU[q]);
  }
  const float dn = d + dU[0];
  const float rn = nr_rcp(dn);
  float qv[3];
#pragma unroll
  for (int i = 0; i < 3; ++i) qv[i] = fmaf(-v[i], dU[0], dU[1 + i]);
  const float vq = fmaf(v[0], qv[0], fmaf(v[1], qv[1], v[2] * qv[2]));
  const float v2 = fmaf(v[0], v[0], fmaf(v[1], v[1], v[2] * v[2]));
  const float q2 = fmaf(qv[0], qv[0], fmaf(qv[1], qv[1], qv[2] * qv[2]));
  const float de = dU[4] - vq - 0.5f * fmaf(v2, dU[0], q2 * rn);
  w[0] = dn;
  w[1] = fmaf(qv[D], rn, v[D]);
  w[2] = fmaf(qv[T1], rn, v[T1]);
  w[3] = fmaf(qv[T2], rn, v[T2]);
  w[4] = tmax(fmaf(g.gm1, de, p), (float)kPFloor);
  inv_d = rn;
}

// transverse half-step and second Riemann solve, all in float
template <int D>
__device__ __forceinline__ void riemann2_mixed_body(const Geom& G, const BufsF& B, const Box& box, const GasF& g,
    long long t) {
  int c3[3];
  box_coords(box, t, c3);
  const long long f = pidx(G, c3);
  const float h = (float)B.rec[3];
  float wl[5], wr[5], idL, idR, Fx[5];
  half_step_side<D>(G, B, B.UL[D], f, f - G.s[D], h, g, wl, idL);
  half_step_side<D>(G, B, B.UR[D], f, f, h, g, wr, idR);
  const int fl = riemann_exact(wl, wr, idL, idR, g, Fx);
  store_face<D>(B.UL[D], f, Fx);
  if (fl) atomicOr(rec_flags(B.rec), fl);
}



// conserved update in FP64 from the float CTU fluxes.  Per variable the flux
// differences of the active axes are summed in float-float arithmetic: each
// difference F(c) - F(c + e_d) is an exact pair, the pairs are added with
// TwoSum into hi + lo, and only the low-order remainders (each below 2^-24 of
// the value it came from) are rounded, to float, so hi + lo carries the sum to
// within about 2^-45 of the largest difference.  Two FP64 operations then
// apply it:
// u + dt/dx (hi + lo).  Neighbour cells see the same float flux with opposite
// sign, so the step conserves to FP64 rounding.
__device__ __forceinline__ void update_mixed_body(const Geom& G, const BufsF& B, long long t) {
  const long long c = real_to_padded(G, t);
  const double dtdx = B.rec[2];
  // every load is issued before the first store (the state and the flux
  // planes are distinct arrays), so that a thread has all of them in flight
  double u[5];
  float fc[3][5], fn[3][5];
#pragma unroll
  for (int q = 0; q < 5; ++q) u[q] = B.u[q * G.nreal + t];
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    if (G.n[d] > 1) {
      load_face_xyz(B.UL[d], c, fc[d]);
      load_face_xyz(B.UL[d], c + G.s[d], fn[d]);
    } else {
#pragma unroll
      for (int q = 0; q < 5; ++q) fc[d][q] = fn[d][q] = 0.f;
    }
  }
  int fl = 0;
#pragma unroll
  for (int q = 0; q < 5; ++q) {
    float hi = 0.f, lo = 0.f;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      float e1, e2;
      const float s = two_sum(fc[d][q], -fn[d][q], e1);
      hi = two_sum(hi, s, e2);
      lo += e1 + e2;
    }
    u[q] = fma(dtdx, ff_to_double(hi, lo), u[q]);
    const long long b = __double_as_longlong(u[q]);
    if ((b & 0x7fffffffffffffffLL) > 0x7ff0000000000000LL) fl = kFlagNonPhys;  // NaN
    if (q == 0 && b <= 0) fl = kFlagNonPhys;  // rho <= 0 (or a NaN with the sign bit)
  }
#pragma unroll
  for (int q = 0; q < 5; ++q) B.u[q * G.nreal + t] = u[q];
  if (fl) atomicOr(rec_flags(B.rec), fl);
}


template <int BS>
__global__ void __launch_bounds__(BS, kMinBlocksUpdate * kThreads / BS) kb_update_mixed(BatchLaunch L) {
  const BatchItem it = batch_item(L);
  if (it.t < it.d->G.nreal) update_mixed_body(it.d->G, float_view(it.d->B, it.d->G.ps), it.t);
}

#define HYDRO_BATCH_MIXED(NAME, STAGE_IDX, MINB, CALL)                                     \
  template <int D, int BS>                                                                  \
  __global__ void __launch_bounds__(BS, MINB * kThreads / BS) NAME(BatchLaunch L) {         \
    const BatchItem it = batch_item(L);                                                     \
    const Box& box = it.d->box[STAGE_IDX][D];                                               \
    if (it.t < (long long)box.n[0] * box.n[1] * box.n[2]) {                                 \
      const BufsF F = float_view(it.d->B, it.d->G.ps);                                      \
      CALL;                                                                                 \
    }                                                                                       \
  }
HYDRO_BATCH_MIXED(kb_ppmc_mixed, 1, kMinBlocksPpmc, ppmc_mixed_body<D>(it.d->G, F, box, it.t))
HYDRO_BATCH_MIXED(kb_riemann1_mixed, 2, kMinBlocksRiemann1,
                  riemann1_mixed_body<D>(it.d->G, F, box, it.d->gf, it.t))
HYDRO_BATCH_MIXED(kb_riemann2_mixed, 3, kMinBlocksRiemann2,
                  riemann2_mixed_body<D>(it.d->G, F, box, it.d->gf, it.t))
#undef HYDRO_BATCH_MIXED

// the segmented PPMC along y (D = 1) or z (D = 2); units: segments of seg[D].
// Two 256-thread blocks an SM (104 registers; at three the window spills)
constexpr int kMinBlocksPpmcSeg = 2;
template <int D, int BS>
__global__ void __launch_bounds__(BS, kMinBlocksPpmcSeg * kThreads / BS) kb_ppmc_mixed_seg(BatchLaunch L) {
  const BatchItem it = batch_item(L);
  const Box& seg = it.d->seg[D];
  if (it.t < (long long)seg.n[0] * seg.n[1] * seg.n[2]) {
    const BufsF F = float_view(it.d->B, it.d->G.ps);
    ppmc_mixed_seg_body<D>(it.d->G, F, seg, it.d->box[1][D], it.t);
  }
}


}  // namespace

cudaError_t batch_prims_mixed(const BatchLaunch& L, int bs, unsigned blocks, cudaStream_t st,
                              bool noh) {
  if (blocks == 0) return cudaSuccess;
  if (bs == 128) {
    if (noh)
      kb_prims_mixed<128, true><<<blocks, 128, 0, st>>>(L);
    else
      kb_prims_mixed<128, false><<<blocks, 128, 0, st>>>(L);
  } else {
    if (noh)
      kb_prims_mixed<256, true><<<blocks, 256, 0, st>>>(L);
    else
      kb_prims_mixed<256, false><<<blocks, 256, 0, st>>>(L);
  }
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

cudaError_t batch_ppmc_mixed_seg(const BatchLaunch& L, int axis, unsigned blocks, cudaStream_t st) {
  if (blocks == 0) return cudaSuccess;
  if (axis == 1)
    kb_ppmc_mixed_seg<1, kPpmcSegThreads><<<blocks, kPpmcSegThreads, 0, st>>>(L);
  else
    kb_ppmc_mixed_seg<2, kPpmcSegThreads><<<blocks, kPpmcSegThreads, 0, st>>>(L);
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
