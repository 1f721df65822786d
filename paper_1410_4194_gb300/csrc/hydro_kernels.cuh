// hydro_kernels.cuh -- the per-axis stage kernels of the FP64 step (slopes,
// PPMC, first Riemann fluxes, transverse half-step + CTU fluxes), templated on
// the sweep axis D and on the strict switch S of hydro_math.cuh.  Included by
// two translation units: hydro_fp64_fast.cu (S = false, compiled with fused
// multiply-add contraction) and hydro_fp64_strict.cu (S = true, compiled without
// it so that every a*b+c rounds twice, as the CPU reference does).
#pragma once
#include "../../include/hydro.h"
#include "hydro_internal.h"
#include "hydro_math.cuh"

namespace hydro {
namespace {

constexpr int kThreads = 256;
// three 256-thread blocks per SM (<= 85 registers a thread): the FP64 pipe is
// the bottleneck, more resident warps hide its dependent-issue latency
constexpr int kMinBlocks = 3;
using Gas = GasT<double>;

// 32-bit index arithmetic: hydro_init and hydro_batch_init reject grids of
// 2^31 or more padded cells, so every box index fits
__device__ __forceinline__ void box_coords(const Box& b, long long t, int c[3]) {
  const unsigned n0 = (unsigned)b.n[0], n01 = (unsigned)b.n[0] * (unsigned)b.n[1];
  const unsigned tt = (unsigned)t;
  const unsigned k = fast_div(tt, b.div01);
  const unsigned r = tt - k * n01;
  const unsigned j = fast_div(r, b.div0);
  c[2] = b.lo[2] + (int)k;
  c[1] = b.lo[1] + (int)j;
  c[0] = b.lo[0] + (int)(r - j * n0);
}

// (i, j, k) of padded cell t: t = i + s1 j + s2 k
__device__ __forceinline__ void padded_coords(const Geom& G, long long t, int c[3]) {
  const unsigned tt = (unsigned)t, s1 = (unsigned)G.s[1], s2 = (unsigned)G.s[2];
  const unsigned k = fast_div(tt, G.div_s2);
  const unsigned r = tt - k * s2;
  const unsigned j = fast_div(r, G.div_s1);
  c[2] = (int)k;
  c[1] = (int)j;
  c[0] = (int)(r - j * s1);
}

// padded index of real cell t (t = i + nx j + nx ny k over the real cells)
__device__ __forceinline__ long long real_to_padded(const Geom& G, long long t) {
  const unsigned tt = (unsigned)t, n0 = (unsigned)G.n[0], n1 = (unsigned)G.n[1];
  const unsigned q = fast_div(tt, G.div_n0);
  const unsigned i = tt - q * n0;
  const unsigned k = fast_div(q, G.div_n1);
  const unsigned j = q - k * n1;
  return (long long)(i + G.g[0]) + (long long)(j + G.g[1]) * G.s[1] + (long long)(k + G.g[2]) * G.s[2];
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


template <int D, bool S>
__device__ __forceinline__ void slopes_body(const Geom& G, const Bufs& B, const Box& box,
    const Gas& g, long long t) {
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
__global__ void __launch_bounds__(kThreads, kMinBlocks) k_slopes(Geom G, Bufs B, Box box, Gas g) {
  const long long count = (long long)box.n[0] * box.n[1] * box.n[2];
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t < count) slopes_body<D, S>(G, B, box, g, t);
}

template <int D, bool S>
__device__ __forceinline__ void ppmc_body(const Geom& G, const Bufs& B, const Box& box,
    const Gas& g, long long t) {
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

// PPMC along x (fast FP64) with the face values shared through the warp.
// Lane l takes cell 31 k + l of the box (k: the warp's chunk; x runs fastest),
// forms the parabola's value at its cell's left face and takes its right
// face's value from lane l + 1, which holds the next cell of the row; the last
// cell of a row forms its own.  A warp so forms 32 face values for 31 cells
// instead of 62 (lane 31 only supplies one), the same doubles (ppmc_face).
// 31 cells a warp need 32/31 of a one-thread-a-cell launch: a warp takes the
// chunks k, k + W, k + 2W, ... (W warps in the grid's launch).
template <int BS>
__device__ __forceinline__ void ppmc_x_shared_body(const Geom& G, const Bufs& B, const Box& box,
                                                   long long t) {
  const long long count = (long long)box.n[0] * box.n[1] * box.n[2];
  const long long nchunk = (count + 30) / 31;
  const long long nwarp = (count + BS - 1) / BS * (BS / 32);
  const int lane = threadIdx.x & 31;
  const long long ps = G.ps, s = G.s[0];
  const double dtdx = B.rec[2];
  for (long long k = t >> 5; k < nchunk; k += nwarp) {  // the same trips for the whole warp
    const long long cell = 31 * k + lane;
    const bool have = cell < count;
    int c3[3] = {0, 0, 0};
    long long c = 0;
    double wm[5], wc[5], sc[5], Lf[5];
    if (have) {
      box_coords(box, cell, c3);
      c = pidx(G, c3);
      load_prim<0>(B.W, ps, c - s, wm);
      load_prim<0>(B.W, ps, c, wc);
#pragma unroll
      for (int q = 0; q < 5; ++q) {
        sc[q] = B.S[q * ps + c];
        Lf[q] = ppmc_face<false>(wm[q], wc[q], B.S[q * ps + c - s], sc[q]);
      }
    } else {
#pragma unroll
      for (int q = 0; q < 5; ++q) Lf[q] = 0.0;
    }
    double Rf[5];
#pragma unroll
    for (int q = 0; q < 5; ++q) Rf[q] = __shfl_down_sync(0xffffffffu, Lf[q], 1);
    if (have && lane < 31) {
      double wp[5];
      load_prim<0>(B.W, ps, c + s, wp);
      if (c3[0] == box.lo[0] + box.n[0] - 1) {  // the row's last cell: its own right face
#pragma unroll
        for (int q = 0; q < 5; ++q) Rf[q] = ppmc_face<false>(wc[q], wp[q], sc[q], B.S[q * ps + c + s]);
      }
      const double a = B.W[5 * ps + c], inv_a = B.W[6 * ps + c], inv_rho = B.W[7 * ps + c];
      double WsL[5], WsR[5];
      ppmc_states_faces<false>(wm, wc, wp, Lf, Rf, a, inv_a, inv_rho, dtdx, WsL, WsR);
      store_rot<0>(B.UR[0], ps, c, WsL);
      store_rot<0>(B.UL[0], ps, c + s, WsR);
    }
  }
}

// PPMC along y or z (fast FP64) for a segment of up to kPpmcSeg consecutive
// cells of a column: a cell's right face value is the next cell's left one
// (ppmc_face), so a segment of K cells forms K + 1 face values instead of 2K,
// and the averages and slopes slide through registers (K + 2 cells loaded
// instead of 3K).  The cells of a warp are 32 x-adjacent columns, so every load
// and store stays a coalesced row.
template <int D>
__device__ __forceinline__ void ppmc_seg_body(const Geom& G, const Bufs& B, const Box& seg,
                                              const Box& box, long long t) {
  int c3[3];
  box_coords(seg, t, c3);
  const int k0 = box.lo[D] + (c3[D] - seg.lo[D]) * kPpmcSeg;  // first cell along D
  const int kn = min(kPpmcSeg, box.lo[D] + box.n[D] - k0);     // cells in this segment
  c3[D] = k0;
  const long long ps = G.ps, s = G.s[D];
  const long long c0 = pidx(G, c3);
  const double dtdx = B.rec[2];
  double wm[5], wc[5], sc[5], Lf[5];
  load_prim<D>(B.W, ps, c0 - s, wm);
  load_prim<D>(B.W, ps, c0, wc);
#pragma unroll
  for (int q = 0; q < 5; ++q) {
    sc[q] = B.S[q * ps + c0];
    Lf[q] = ppmc_face<false>(wm[q], wc[q], B.S[q * ps + c0 - s], sc[q]);
  }
#pragma unroll 1
  for (int k = 0; k < kn; ++k) {
    const long long c = c0 + k * s;
    double wp[5], sp[5], Rf[5];
    load_prim<D>(B.W, ps, c + s, wp);
#pragma unroll
    for (int q = 0; q < 5; ++q) {
      sp[q] = B.S[q * ps + c + s];
      Rf[q] = ppmc_face<false>(wc[q], wp[q], sc[q], sp[q]);
    }
    const double a = B.W[5 * ps + c], inv_a = B.W[6 * ps + c], inv_rho = B.W[7 * ps + c];
    double WsL[5], WsR[5];
    ppmc_states_faces<false>(wm, wc, wp, Lf, Rf, a, inv_a, inv_rho, dtdx, WsL, WsR);
    store_rot<D>(B.UR[D], ps, c, WsL);
    store_rot<D>(B.UL[D], ps, c + s, WsR);
#pragma unroll
    for (int q = 0; q < 5; ++q) {
      wm[q] = wc[q];
      wc[q] = wp[q];
      sc[q] = sp[q];
      Lf[q] = Rf[q];
    }
  }
}

template <int D, bool S>
__global__ void __launch_bounds__(kThreads, kMinBlocks) k_ppmc(Geom G, Bufs B, Box box, Gas g) {
  const long long count = (long long)box.n[0] * box.n[1] * box.n[2];
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t < count) ppmc_body<D, S>(G, B, box, g, t);
}

// store the face states of cell c: its left face is the right state of face c,
// its right face the left state of face c+1; primitives W* (fast) or the
// conserved U* (strict, as the paper passes them between kernels)
template <int D, bool S>
__device__ __forceinline__ void store_face_states(const Geom& G, const Bufs& B, const Gas& g,
                                                  long long c, const double WsL[5],
                                                  const double WsR[5]) {
  const long long s = G.s[D];
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

// limited primitive slope of every cell of the box (PPMP, PLMP)
template <int D, bool S>
__device__ __forceinline__ void prim_slopes_body(const Geom& G, const Bufs& B, const Box& box,
    const Gas& g, long long t) {
  int c3[3];
  box_coords(box, t, c3);
  const long long c = pidx(G, c3);
  const long long s = G.s[D];
  double wm[5], wc[5], wp[5], dw[5];
  load_prim<D>(B.W, G.ps, c - s, wm);
  load_prim<D>(B.W, G.ps, c, wc);
  load_prim<D>(B.W, G.ps, c + s, wp);
  prim_slope<S>(wm, wc, wp, dw);
#pragma unroll
  for (int q = 0; q < 5; ++q) B.S[q * G.ps + c] = dw[q];
}

// PPMP face states of cell c (stencil c-3..c+3)
template <int D, bool S>
__device__ __forceinline__ void ppmp_body(const Geom& G, const Bufs& B, const Box& box,
    const Gas& g, long long t) {
  int c3[3];
  box_coords(box, t, c3);
  const long long c = pidx(G, c3);
  const long long s = G.s[D];
  double w[7][5], sm[5], sc[5], sp[5];
#pragma unroll
  for (int k = 0; k < 7; ++k) load_prim<D>(B.W, G.ps, c + (k - 3) * s, w[k]);
#pragma unroll
  for (int q = 0; q < 5; ++q) {
    sm[q] = B.S[q * G.ps + c - s];
    sc[q] = B.S[q * G.ps + c];
    sp[q] = B.S[q * G.ps + c + s];
  }
  double WsL[5], WsR[5];
  ppmp_states<S>(w, sm, sc, sp, B.W[5 * G.ps + c], B.rec[2], G.dx, g, WsL, WsR);
  store_face_states<D, S>(G, B, g, c, WsL, WsR);
}

// PLMC face states of cell c (characteristic slope of c from the slope stage)
template <int D, bool S>
__device__ __forceinline__ void plmc_body(const Geom& G, const Bufs& B, const Box& box,
    const Gas& g, long long t) {
  int c3[3];
  box_coords(box, t, c3);
  const long long c = pidx(G, c3);
  const long long s = G.s[D];
  double wm[5], wc[5], wp[5], dw[5];
  load_prim<D>(B.W, G.ps, c - s, wm);
  load_prim<D>(B.W, G.ps, c, wc);
  load_prim<D>(B.W, G.ps, c + s, wp);
#pragma unroll
  for (int q = 0; q < 5; ++q) dw[q] = B.S[q * G.ps + c];
  double WsL[5], WsR[5];
  plmc_states<S>(wm, wc, wp, dw, B.W[5 * G.ps + c], B.W[6 * G.ps + c], B.W[7 * G.ps + c],
                 B.rec[2], WsL, WsR);
  store_face_states<D, S>(G, B, g, c, WsL, WsR);
}

// PLMP face states of cell c (primitive slope of c from the slope stage); the
// half-step evolution gives conserved states, stored as such (strict) or as
// their primitives (fast)
template <int D, bool S>
__device__ __forceinline__ void plmp_body(const Geom& G, const Bufs& B, const Box& box,
    const Gas& g, long long t) {
  int c3[3];
  box_coords(box, t, c3);
  const long long c = pidx(G, c3);
  const long long s = G.s[D];
  double wc[5], dw[5], UsL[5], UsR[5];
  load_prim<D>(B.W, G.ps, c, wc);
#pragma unroll
  for (int q = 0; q < 5; ++q) dw[q] = B.S[q * G.ps + c];
  plmp_states<S>(wc, dw, B.rec[2], g, UsL, UsR);
  if constexpr (S) {
    store_rot<D>(B.UR[D], G.ps, c, UsL);
    store_rot<D>(B.UL[D], G.ps, c + s, UsR);
  } else {
    double WsL[5], WsR[5], idL, idR;
    cons2prim<false>(UsL, g, WsL, idL);
    cons2prim<false>(UsR, g, WsR, idR);
    store_rot<D>(B.UR[D], G.ps, c, WsL);
    store_rot<D>(B.UL[D], G.ps, c + s, WsR);
  }
}

// PCM face states of cell c: the cell average at both faces (stored as its
// primitives, or in strict mode converted back to conserved variables -- a
// rounding-level round trip of the cell's conserved average, so strict PCM is
// not operation-identical to the CPU reference)
template <int D, bool S>
__device__ __forceinline__ void pcm_body(const Geom& G, const Bufs& B, const Box& box,
    const Gas& g, long long t) {
  int c3[3];
  box_coords(box, t, c3);
  const long long c = pidx(G, c3);
  double wc[5];
  load_prim<D>(B.W, G.ps, c, wc);
  store_face_states<D, S>(G, B, g, c, wc, wc);
}

#define HYDRO_SINGLE_WRAPPER(NAME, BODY)                                                 \
  template <int D, bool S>                                                               \
  __global__ void __launch_bounds__(kThreads, kMinBlocks) NAME(Geom G, Bufs B, Box box, Gas g) { \
    const long long count = (long long)box.n[0] * box.n[1] * box.n[2];                   \
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;                \
    if (t < count) BODY<D, S>(G, B, box, g, t);                                          \
  }
HYDRO_SINGLE_WRAPPER(k_prim_slopes, prim_slopes_body)
HYDRO_SINGLE_WRAPPER(k_ppmp, ppmp_body)
HYDRO_SINGLE_WRAPPER(k_plmc, plmc_body)
HYDRO_SINGLE_WRAPPER(k_plmp, plmp_body)
HYDRO_SINGLE_WRAPPER(k_pcm, pcm_body)
#undef HYDRO_SINGLE_WRAPPER

// first Riemann set at face f: the exact solver, or (ROE) the Roe solver with
// the HLLE fallback, which also stores the face's H-correction eta
template <int D, bool S, bool ROE = false>
__device__ __forceinline__ void riemann1_body(const Geom& G, const Bufs& B, const Box& box,
    const Gas& g, long long t) {
  int c3[3];
  box_coords(box, t, c3);
  const long long f = pidx(G, c3);
  double UL[5], UR[5], WL[5], WR[5], F[5], idL, idR;
  int fl = 0;
  if constexpr (S) {
    load_rot<D>(B.UL[D], G.ps, f, UL);
    load_rot<D>(B.UR[D], G.ps, f, UR);
    cons2prim<true>(UL, g, WL, idL);
    cons2prim<true>(UR, g, WR, idR);
  } else {
    load_rot<D>(B.UL[D], G.ps, f, WL);
    load_rot<D>(B.UR[D], G.ps, f, WR);
    idL = idR = 0.0;
    if constexpr (ROE) {
      idL = nr_rcp(WL[0]);
      idR = nr_rcp(WR[0]);
      prim2cons(WL, g, UL);
      prim2cons(WR, g, UR);
    }
  }
  if constexpr (ROE) {
    riemann_roe<S>(UL, UR, WL, WR, idL, idR, 0.0, g, F);
    B.eta[D][f] = h_eta<S>(WL, WR, idL, idR, g);
  } else if constexpr (S) {
    fl = riemann_exact<S>(WL, WR, idL, idR, g, F);
  } else {
    // the face states are primitives: the solver needs 1/rho only for the
    // sound speeds, which it forms without it
    fl = riemann_exact<S, double, false>(WL, WR, idL, idR, g, F);
  }
  store_rot<D>(B.F1[D], G.ps, f, F);
  if (fl) atomicOr(rec_flags(B.rec), fl);
}
template <int D, bool S>
__device__ __forceinline__ void riemann1_roe_body(const Geom& G, const Bufs& B, const Box& box,
    const Gas& g, long long t) {
  riemann1_body<D, S, true>(G, B, box, g, t);
}

template <int D, bool S>
__global__ void __launch_bounds__(kThreads, kMinBlocks) k_riemann1(Geom G, Bufs B, Box box, Gas g) {
  const long long count = (long long)box.n[0] * box.n[1] * box.n[2];
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t < count) riemann1_body<D, S>(G, B, box, g, t);
}

// transverse half-step and second Riemann set at face f; with ROE the Roe
// solver with the H correction: eta^H is the largest eta of this face and of
// the transverse faces of the two cells it separates (nine faces in 3D)
template <int D, bool S, bool ROE = false>
__device__ __forceinline__ void riemann2_body(const Geom& G, const Bufs& B, const Box& box,
    const Gas& g, long long t) {
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
  int fl = 0;
  if constexpr (ROE) {
    double etaH = B.eta[D][f];
    if (G.n[T1] > 1) {
      const double* e = B.eta[T1];
      const long long st = G.s[T1];
      etaH = max_nn<S>(etaH, e[cl]);
      etaH = max_nn<S>(etaH, e[cl + st]);
      etaH = max_nn<S>(etaH, e[cr]);
      etaH = max_nn<S>(etaH, e[cr + st]);
    }
    if (G.n[T2] > 1) {
      const double* e = B.eta[T2];
      const long long st = G.s[T2];
      etaH = max_nn<S>(etaH, e[cl]);
      etaH = max_nn<S>(etaH, e[cl + st]);
      etaH = max_nn<S>(etaH, e[cr]);
      etaH = max_nn<S>(etaH, e[cr + st]);
    }
    riemann_roe<S>(UL, UR, WL, WR, idL, idR, etaH, g, Fx);
  } else if constexpr (S) {
    fl = riemann_exact<S>(WL, WR, idL, idR, g, Fx);
  } else {
    // the sound speeds from reciprocal square roots of gamma p rho, as in the
    // first set (one FP64 issue slot a side fewer than sqrt(gamma p / rho))
    fl = riemann_exact<S, double, false>(WL, WR, idL, idR, g, Fx);
  }
  // CTU flux of this face replaces its (now consumed) left state
  store_rot<D>(B.UL[D], ps, f, Fx);
  if (fl) atomicOr(rec_flags(B.rec), fl);
}
// The transverse half-step and second set of exact solves (fast FP64) along y
// or z for a segment of up to kPpmcSeg consecutive faces of a column.  The
// cell between faces f and f + s supplies the right state of face f and the
// left state of face f + s, and both take its transverse flux differences:
// formed once here and added to both states in the order of riemann2_body
// (the same doubles), where one face a thread forms each cell's differences
// twice.  The next face's left state is formed before the current face's solve,
// so five doubles are carried across it.  The cells of a warp are 32
// x-adjacent columns, so every load and store stays a coalesced row.
template <int D>
__device__ __forceinline__ void riemann2_seg_body(const Geom& G, const Bufs& B, const Box& seg,
                                                  const Box& box, const Gas& g, long long t) {
  int c3[3];
  box_coords(seg, t, c3);
  const int k0 = box.lo[D] + (c3[D] - seg.lo[D]) * kPpmcSeg;  // first face along D
  const int kn = min(kPpmcSeg, box.lo[D] + box.n[D] - k0);     // faces in this segment
  c3[D] = k0;
  const long long ps = G.ps, s = G.s[D];
  const long long f0 = pidx(G, c3);
  const double h = B.rec[3];
  constexpr int T1 = Perm<D>::t1, T2 = Perm<D>::t2;
  const bool act1 = G.n[T1] > 1, act2 = G.n[T2] > 1;
  const double* Fa = B.F1[T1];
  const double* Fb = B.F1[T2];
  const long long sa = G.s[T1], sb = G.s[T2];
  double UhL[5];
  {
    double Ws[5];
#pragma unroll
    for (int q = 0; q < 5; ++q) Ws[q] = B.UL[D][q * ps + f0];
    prim2cons(Ws, g, UhL);
    const long long cl = f0 - s;
    if (act1) {
#pragma unroll
      for (int q = 0; q < 5; ++q) UhL[q] = UhL[q] + h * (Fa[q * ps + cl] - Fa[q * ps + cl + sa]);
    }
    if (act2) {
#pragma unroll
      for (int q = 0; q < 5; ++q) UhL[q] = UhL[q] + h * (Fb[q * ps + cl] - Fb[q * ps + cl + sb]);
    }
  }
#pragma unroll 1
  for (int k = 0; k < kn; ++k) {
    const long long f = f0 + k * s;  // the cell f lies between faces f and f + s
    const bool next = k + 1 < kn;
    double UhR[5], UhN[5], Ws[5];
#pragma unroll
    for (int q = 0; q < 5; ++q) Ws[q] = B.UR[D][q * ps + f];
    prim2cons(Ws, g, UhR);
    if (next) {
#pragma unroll
      for (int q = 0; q < 5; ++q) Ws[q] = B.UL[D][q * ps + f + s];
      prim2cons(Ws, g, UhN);
    }
    if (act1) {
#pragma unroll
      for (int q = 0; q < 5; ++q) {
        const double dq = Fa[q * ps + f] - Fa[q * ps + f + sa];
        UhR[q] = UhR[q] + h * dq;
        if (next) UhN[q] = UhN[q] + h * dq;
      }
    }
    if (act2) {
#pragma unroll
      for (int q = 0; q < 5; ++q) {
        const double dq = Fb[q * ps + f] - Fb[q * ps + f + sb];
        UhR[q] = UhR[q] + h * dq;
        if (next) UhN[q] = UhN[q] + h * dq;
      }
    }
    double UL[5], UR[5], WL[5], WR[5], Fx[5], idL, idR;
    UL[0] = UhL[0]; UL[1] = UhL[1 + D]; UL[2] = UhL[1 + T1]; UL[3] = UhL[1 + T2]; UL[4] = UhL[4];
    UR[0] = UhR[0]; UR[1] = UhR[1 + D]; UR[2] = UhR[1 + T1]; UR[3] = UhR[1 + T2]; UR[4] = UhR[4];
    cons2prim<false>(UL, g, WL, idL);
    cons2prim<false>(UR, g, WR, idR);
    const int fl = riemann_exact<false, double, false>(WL, WR, idL, idR, g, Fx);
    // CTU flux of this face replaces its (now consumed) left state
    store_rot<D>(B.UL[D], ps, f, Fx);
    if (fl) atomicOr(rec_flags(B.rec), fl);
#pragma unroll
    for (int q = 0; q < 5; ++q) UhL[q] = UhN[q];
  }
}

template <int D, bool S>
__device__ __forceinline__ void riemann2_roe_body(const Geom& G, const Bufs& B, const Box& box,
    const Gas& g, long long t) {
  riemann2_body<D, S, true>(G, B, box, g, t);
}

template <int D, bool S>
__global__ void __launch_bounds__(kThreads, kMinBlocks) k_riemann2(Geom G, Bufs B, Box box, Gas g) {
  const long long count = (long long)box.n[0] * box.n[1] * box.n[2];
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t < count) riemann2_body<D, S>(G, B, box, g, t);
}
template <int D, bool S>
__global__ void __launch_bounds__(kThreads, kMinBlocks) k_riemann1_roe(Geom G, Bufs B, Box box, Gas g) {
  const long long count = (long long)box.n[0] * box.n[1] * box.n[2];
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t < count) riemann1_roe_body<D, S>(G, B, box, g, t);
}
template <int D, bool S>
__global__ void __launch_bounds__(kThreads, kMinBlocks) k_riemann2_roe(Geom G, Bufs B, Box box, Gas g) {
  const long long count = (long long)box.n[0] * box.n[1] * box.n[2];
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t < count) riemann2_roe_body<D, S>(G, B, box, g, t);
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
  b.div0 = make_fastdiv((unsigned)b.n[0]);
  b.div01 = make_fastdiv((unsigned)b.n[0] * (unsigned)b.n[1]);
  return b;
}

inline long long box_count(const Box& b) { return (long long)b.n[0] * b.n[1] * b.n[2]; }

// The conserved state of padded cell c (coordinates c[3]): a real cell's, or
// for a ghost the value the boundary passes x, then y, then z give it.  Each
// ghost axis maps the coordinate to a real cell (periodic wrap, mirror, or the
// outermost cell) and a reflective axis negates its normal momentum; an inflow
// or Noh axis ends the chain: its state replaces the mapped cell's and only
// the reflective axes after it negate their momentum.  The Noh state (Sec.
// 4.3.1: rho0 (1 + V t/r)^(n-1), velocity V toward the origin, E = p0/(gamma-1)
// + rho V^2/2, n the active axes) is taken at the position the passes reach:
// the cell's own coordinates on the Noh axis and the axes before it, the
// mapped ones after it.  Returns whether the cell is real; neg receives the
// axes (bit d) whose momentum component the caller negates, in the precision
// it works in.  NOH: whether the grid has a Noh face (the kernels are compiled
// both ways so that the other grids carry none of its code or registers).
template <bool NOH>
__device__ __forceinline__ bool boundary_state(const Geom& G, const double* __restrict__ u,
                                               const BcDesc& bc, double gm1, double time,
                                               const int c[3], double U[5], int& neg_out) {
  int src[3];
  int neg = 0, fixed_face = -1, noh_axis = -1;
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
      case 4:  // Noh: analytic, at this coordinate
        if constexpr (NOH) {
          src[d] = r;
          fixed_face = face;
          noh_axis = d;
          neg = 0;
        }
        break;
      default:  // inflow
        src[d] = 0;
        fixed_face = face;
        noh_axis = -1;
        neg = 0;
        break;
    }
  }
  if (NOH && noh_axis >= 0) {
    const double* P = bc.prim[fixed_face];
    double x[3], r2 = 0.0;
    int nact = 0;
#pragma unroll
    for (int t = 0; t < 3; ++t) {
      x[t] = 0.0;
      if (G.n[t] > 1) {
        ++nact;
        x[t] = ((t <= noh_axis ? c[t] - G.g[t] : src[t]) + 0.5) * G.dx;
        r2 += x[t] * x[t];
      }
    }
    const double rr = sqrt(r2);
    const double b = 1.0 + P[1] * time / rr;
    double bn = 1.0;  // b^(n-1), n <= 3: exact products as pow rounds them
    for (int k = 1; k < nact; ++k) bn = k == 1 ? b : bn * b;
    const double rho = P[0] * bn;
    U[0] = rho;
#pragma unroll
    for (int t = 0; t < 3; ++t) U[1 + t] = -rho * P[1] * x[t] / rr;
    U[4] = P[4] / gm1 + 0.5 * rho * P[1] * P[1];
  } else if (fixed_face >= 0) {
#pragma unroll
    for (int q = 0; q < 5; ++q) U[q] = bc.inflow[fixed_face][q];
  } else {
    const long long rs = src[0] + (long long)G.n[0] * (src[1] + (long long)G.n[1] * src[2]);
#pragma unroll
    for (int q = 0; q < 5; ++q) U[q] = u[q * G.nreal + rs];
  }
  neg_out = neg;
  return real;
}


// ---- batched launches: one launch, the blocks of every grid ----------------
// grid slot of block b: the last i with prefix[i] <= b
__device__ __forceinline__ int find_slot(const int* __restrict__ prefix, int n, int b) {
  int lo = 0, hi = n;
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (prefix[mid] <= b)
      lo = mid;
    else
      hi = mid;
  }
  return lo;
}

// the grid of this block and the index t of this thread within that grid's box
struct BatchItem {
  const GridDesc* d;
  long long t;
};
__device__ __forceinline__ BatchItem batch_item(const BatchLaunch& L) {
  const int slot = find_slot(L.prefix, L.ngrids, (int)blockIdx.x);
  BatchItem it;
  it.d = L.descs + L.order[slot];
  it.t = (long long)((int)blockIdx.x - L.prefix[slot]) * blockDim.x + threadIdx.x;
  return it;
}

#define HYDRO_BATCH_WRAPPER(NAME, BODY, STAGE_IDX)                                             \
  template <int D, bool S, int BS>                                                             \
  __global__ void __launch_bounds__(BS, kMinBlocks * kThreads / BS) NAME(BatchLaunch L) {     \
    const BatchItem it = batch_item(L);                                                        \
    const Box& box = it.d->box[STAGE_IDX][D];                                                  \
    if (it.t < (long long)box.n[0] * box.n[1] * box.n[2])                                      \
      BODY<D, S>(it.d->G, it.d->B, box, it.d->gd, it.t);                                       \
  }
HYDRO_BATCH_WRAPPER(kb_slopes, slopes_body, 0)
HYDRO_BATCH_WRAPPER(kb_prim_slopes, prim_slopes_body, 0)
HYDRO_BATCH_WRAPPER(kb_ppmc, ppmc_body, 1)
HYDRO_BATCH_WRAPPER(kb_ppmp, ppmp_body, 1)
HYDRO_BATCH_WRAPPER(kb_plmc, plmc_body, 1)
HYDRO_BATCH_WRAPPER(kb_plmp, plmp_body, 1)
HYDRO_BATCH_WRAPPER(kb_pcm, pcm_body, 1)
// The Riemann sets with their own register budgets, by measurement on Sedov
// 256^3 and Mach-5 turbulence 256^3: the first set at 64 registers (1024
// resident threads an SM), 1.8% faster than at 80 (768 threads); the second
// at 72 (896 threads with 128-thread blocks, 768 with 256), 0.4-0.6% faster
// than at 80 and 1% faster than at 96 (640 threads); the reconstruction and
// slope kernels gain nothing from 640 or 896 threads.  The budget is a
// register count, the same for both block sizes, so that both compile to the
// same code and a grid's results do not depend on its block size (bit for
// bit; a bound in resident threads would give 256-thread blocks 80 registers).
#define HYDRO_BATCH_WRAPPER_R(NAME, BODY, STAGE_IDX, REGS)                                     \
  template <int D, bool S, int BS>                                                             \
  __global__ void __maxnreg__(REGS) NAME(BatchLaunch L) {                                      \
    const BatchItem it = batch_item(L);                                                        \
    const Box& box = it.d->box[STAGE_IDX][D];                                                  \
    if (it.t < (long long)box.n[0] * box.n[1] * box.n[2])                                      \
      BODY<D, S>(it.d->G, it.d->B, box, it.d->gd, it.t);                                       \
  }
// PPMC (fast FP64) along x with the face values shared through the warp (one
// launch of the x PPMC stage's blocks; see ppmc_x_shared_body) and along y, z
// by segments (units: the segments of seg[D], kPpmcSegThreads a block for any
// schedule).  Both at 128 registers (512 resident threads an SM): at the
// one-cell kernel's 80 their windows and face values spill, which cost more
// than the extra warps gave (measured, one GB300: Sedov 256^3 PPMC 7.31 ->
// 7.21 ms a step, turbulence 256^3 10.64 -> 10.47).
constexpr int kPpmcSharedThreadsPerSM = 512;
template <int BS>
__global__ void __launch_bounds__(BS, kPpmcSharedThreadsPerSM / BS) kb_ppmc_xs(BatchLaunch L) {
  const BatchItem it = batch_item(L);
  ppmc_x_shared_body<BS>(it.d->G, it.d->B, it.d->box[1][0], it.t);
}
template <int D>
__global__ void __launch_bounds__(kPpmcSegThreads, kPpmcSharedThreadsPerSM / kPpmcSegThreads)
    kb_ppmc_seg(BatchLaunch L) {
  const BatchItem it = batch_item(L);
  const Box& seg = it.d->seg[D];
  if (it.t < (long long)seg.n[0] * seg.n[1] * seg.n[2])
    ppmc_seg_body<D>(it.d->G, it.d->B, seg, it.d->box[1][D], it.t);
}
// the fast FP64 second Riemann set along y, z by segments (units: the segments
// of seg2[D], kPpmcSegThreads a block for any schedule)
constexpr int kRiemann2SegRegs = 96;
template <int D>
__global__ void __maxnreg__(kRiemann2SegRegs) kb_riemann2_seg(BatchLaunch L) {
  const BatchItem it = batch_item(L);
  const Box& seg = it.d->seg2[D];
  if (it.t < (long long)seg.n[0] * seg.n[1] * seg.n[2])
    riemann2_seg_body<D>(it.d->G, it.d->B, seg, it.d->box[3][D], it.d->gd, it.t);
}
HYDRO_BATCH_WRAPPER_R(kb_riemann1, riemann1_body, 2, 64)
HYDRO_BATCH_WRAPPER_R(kb_riemann2, riemann2_body, 3, 72)
#undef HYDRO_BATCH_WRAPPER_R
HYDRO_BATCH_WRAPPER(kb_riemann1_roe, riemann1_roe_body, 2)
HYDRO_BATCH_WRAPPER(kb_riemann2_roe, riemann2_roe_body, 3)
#undef HYDRO_BATCH_WRAPPER

// Ranges (padded coordinates; "others" are the two axes across the sweep):
//   slopes   d in [g-2, g+n+1], others in [g-1, g+n]
//   ppmc     d in [g-1, g+n],   others in [g-1, g+n]
//   riemann1 faces d in [g, g+n], others in [g-1, g+n]
//   riemann2 faces d in [g, g+n], others real
// which is exactly what the CTU fluxes of the real cells need.
inline Box stage_box(const Geom& G, int stage, int axis) {
  switch (stage) {
    case kStageSlopes: return make_box(G, axis, -2, 2, -1, 1);
    case kStagePpmc: return make_box(G, axis, -1, 1, -1, 1);
    case kStageRiemann1: return make_box(G, axis, 0, 1, -1, 1);
    default: return make_box(G, axis, 0, 1, 0, 0);
  }
}

// kernels of the slope and reconstruction stages for each reconstruction:
// PPMC and PLMC take characteristic slopes, PPMP and PLMP primitive ones, PCM
// none (its slope stage launches nothing)
template <bool S>
cudaError_t launch_axis_stage(const Geom& G, const Bufs& B, int recon, int solver, int stage,
                              int axis, double gamma, cudaStream_t st) {
  const Gas g = make_gas<double>(gamma);
  const Box b = stage_box(G, stage, axis);
  const unsigned nb = blocks_for(box_count(b));
  if (nb == 0) return cudaSuccess;
#define HYDRO_LAUNCH_AXIS(K)                                                 \
  switch (axis) {                                                            \
    case 0: K<0, S><<<nb, kThreads, 0, st>>>(G, B, b, g); break;            \
    case 1: K<1, S><<<nb, kThreads, 0, st>>>(G, B, b, g); break;            \
    default: K<2, S><<<nb, kThreads, 0, st>>>(G, B, b, g); break;           \
  }
  switch (stage) {
    case kStageSlopes:
      if (recon == HYDRO_RECON_PCM) return cudaSuccess;
      if (recon == HYDRO_RECON_PPMP || recon == HYDRO_RECON_PLMP) {
        HYDRO_LAUNCH_AXIS(k_prim_slopes)
      } else {
        HYDRO_LAUNCH_AXIS(k_slopes)
      }
      break;
    case kStagePpmc:
      switch (recon) {
        case HYDRO_RECON_PPMP: HYDRO_LAUNCH_AXIS(k_ppmp) break;
        case HYDRO_RECON_PLMC: HYDRO_LAUNCH_AXIS(k_plmc) break;
        case HYDRO_RECON_PLMP: HYDRO_LAUNCH_AXIS(k_plmp) break;
        case HYDRO_RECON_PCM: HYDRO_LAUNCH_AXIS(k_pcm) break;
        default: HYDRO_LAUNCH_AXIS(k_ppmc) break;
      }
      break;
    case kStageRiemann1:
      if (solver == HYDRO_RIEMANN_ROE) {
        HYDRO_LAUNCH_AXIS(k_riemann1_roe)
      } else {
        HYDRO_LAUNCH_AXIS(k_riemann1)
      }
      break;
    case kStageRiemann2:
      if (solver == HYDRO_RIEMANN_ROE) {
        HYDRO_LAUNCH_AXIS(k_riemann2_roe)
      } else {
        HYDRO_LAUNCH_AXIS(k_riemann2)
      }
      break;
    default: return cudaErrorInvalidValue;
  }
#undef HYDRO_LAUNCH_AXIS
  return cudaGetLastError();
}

template <bool S>
cudaError_t launch_batch_stage(const BatchLaunch& L, int recon, int solver, int stage, int axis,
                               int bs, unsigned blocks, cudaStream_t st) {
  if (blocks == 0) return cudaSuccess;
#define HYDRO_BATCH_AXIS(K)                                                              \
  if (bs == 128) {                                                                       \
    switch (axis) {                                                                      \
      case 0: K<0, S, 128><<<blocks, 128, 0, st>>>(L); break;                           \
      case 1: K<1, S, 128><<<blocks, 128, 0, st>>>(L); break;                           \
      default: K<2, S, 128><<<blocks, 128, 0, st>>>(L); break;                          \
    }                                                                                    \
  } else {                                                                               \
    switch (axis) {                                                                      \
      case 0: K<0, S, 256><<<blocks, 256, 0, st>>>(L); break;                           \
      case 1: K<1, S, 256><<<blocks, 256, 0, st>>>(L); break;                           \
      default: K<2, S, 256><<<blocks, 256, 0, st>>>(L); break;                          \
    }                                                                                    \
  }
  switch (stage) {
    case kStageSlopes:
      if (recon == HYDRO_RECON_PCM) return cudaSuccess;
      if (recon == HYDRO_RECON_PPMP || recon == HYDRO_RECON_PLMP) {
        HYDRO_BATCH_AXIS(kb_prim_slopes)
      } else {
        HYDRO_BATCH_AXIS(kb_slopes)
      }
      break;
    case kStagePpmc:
      switch (recon) {
        case HYDRO_RECON_PPMP: HYDRO_BATCH_AXIS(kb_ppmp) break;
        case HYDRO_RECON_PLMC: HYDRO_BATCH_AXIS(kb_plmc) break;
        case HYDRO_RECON_PLMP: HYDRO_BATCH_AXIS(kb_plmp) break;
        case HYDRO_RECON_PCM: HYDRO_BATCH_AXIS(kb_pcm) break;
        default:
          if (!S && axis == 0) {  // face values shared through the warp
            if (bs == 128)
              kb_ppmc_xs<128><<<blocks, 128, 0, st>>>(L);
            else
              kb_ppmc_xs<256><<<blocks, 256, 0, st>>>(L);
          } else {
            HYDRO_BATCH_AXIS(kb_ppmc)
          }
          break;
      }
      break;
    case kStageRiemann1:
      if (solver == HYDRO_RIEMANN_ROE) {
        HYDRO_BATCH_AXIS(kb_riemann1_roe)
      } else {
        HYDRO_BATCH_AXIS(kb_riemann1)
      }
      break;
    case kStageRiemann2:
      if (solver == HYDRO_RIEMANN_ROE) {
        HYDRO_BATCH_AXIS(kb_riemann2_roe)
      } else {
        HYDRO_BATCH_AXIS(kb_riemann2)
      }
      break;
    default: return cudaErrorInvalidValue;
  }
#undef HYDRO_BATCH_AXIS
  return cudaGetLastError();
}

}  // namespace
}  // namespace hydro
