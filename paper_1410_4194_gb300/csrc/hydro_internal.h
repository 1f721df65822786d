// hydro_internal.h -- host-side types shared by the C-ABI and the kernel files.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "hydro_math.cuh"

namespace hydro {

// Division of a 32-bit index n < 2^31 by a fixed divisor d (1 <= d < 2^31)
// with a multiply-high and a shift instead of an integer division (which the
// GPU evaluates as a ~20-instruction sequence): for d not a power of two, with
// 2^(s-1) < d < 2^s and m = ceil(2^(31+s) / d) < 2^32,
//   floor(n / d) = floor(n m / 2^(31+s))
// because n m / 2^(31+s) = n/d + n r / (d 2^(31+s)) with 0 < r < d adds less
// than n / 2^(31+s) < 2^-s < 1/d, too little to reach the next integer (the
// round-up method of division by invariant integers); for d = 2^k, m = 0 and
// the quotient is n >> k.
struct FastDiv {
  unsigned m;  // multiplier, 0 for a power of two
  int sh;      // shift after the multiply-high (s - 1), or k
};
inline FastDiv make_fastdiv(unsigned d) {
  FastDiv f;
  int s = 0;
  while ((1u << s) < d) ++s;  // d <= 2^s
  if ((1u << s) == d) {
    f.m = 0;
    f.sh = s;
  } else {
    const unsigned long long two = 1ull << (31 + s);
    f.m = (unsigned)((two + d - 1) / d);
    f.sh = s - 1;
  }
  return f;
}
__host__ __device__ __forceinline__ unsigned fast_div(unsigned n, FastDiv f) {
#ifdef __CUDA_ARCH__
  return f.m ? (__umulhi(n, f.m) >> f.sh) : (n >> f.sh);
#else
  return f.m ? (unsigned)(((unsigned long long)n * f.m) >> 32) >> f.sh : (n >> f.sh);
#endif
}

// Geometry of one grid.  Padded arrays carry kNG ghost layers on each side of
// an active axis (an axis with one cell has none) and are laid out x fastest.
struct Geom {
  int n[3];          // real cells per axis
  int g[3];          // ghost layers per side (4 on active axes, 0 otherwise)
  int N[3];          // padded extent per axis
  long long s[3];    // padded strides: 1, N0, N0*N1
  long long ps;      // plane stride of padded arrays (multiple of 32)
  long long nreal;   // nx*ny*nz
  double dx;
  FastDiv div_s1, div_s2;  // by the padded strides s[1], s[2]
  FastDiv div_n0, div_n1;  // by the real extents n[0], n[1]
};
// fill the divisors of a geometry whose extents and strides are set
inline void geom_divisors(Geom& G) {
  G.div_s1 = make_fastdiv((unsigned)G.s[1]);
  G.div_s2 = make_fastdiv((unsigned)G.s[2]);
  G.div_n0 = make_fastdiv((unsigned)G.n[0]);
  G.div_n1 = make_fastdiv((unsigned)G.n[1]);
}

// Boundary description passed to the primitive kernel by value.
struct BcDesc {
  int type[6];          // HYDRO_BC_* per face x-, x+, y-, y+, z-, z+
  double inflow[6][5];  // conserved inflow state per face (rho, mx, my, mz, E)
  double prim[6][5];    // the prescribed state as given: inflow (rho, u, v, w, p),
                        // Noh (rho0, V, -, -, p0)
};
// whether a grid has a Noh face (the primitive kernels are compiled with and
// without the Noh case)
inline bool has_noh(const BcDesc& bc) {
  for (int f = 0; f < 6; ++f)
    if (bc.type[f] == HYDRO_BC_NOH) return true;
  return false;
}

// Device buffers of the FP64 path.
struct Bufs {
  double* u;       // real cells [5][nz][ny][nx]
  double* W;       // padded primitives [8][ps]: rho, vx, vy, vz, p, a, 1/a, 1/rho
  double* S;       // padded limited slopes [5][ps] of the current sweep (sweep order)
  double* UL[3];   // per axis: primitive left states W*_L of faces [5][ps]; reused for F^{n+1/2}
  double* UR[3];   // per axis: primitive right states W*_R of faces [5][ps]
  double* F1[3];   // per axis: first fluxes F* [5][ps]
  double* eta[3];  // per axis: H-correction eta of each face [ps] (Roe solver only, else null)
  // 64-byte step record on the device: [0] max of |v_d| + a (bits), [1] dt, [2] dt/dx,
  // [3] dt/(2 dx), [4] flags (int in the low word), [5] time t at the start of
  // the next step (advanced by the dt kernel after the step's primitive kernel
  // has read it; read by the Noh boundary)
  double* rec;
};

// Box of cells (or faces: a face carries the index of the cell to its right).
struct Box {
  int lo[3];
  int n[3];
  FastDiv div0, div01;  // by n[0] and n[0] n[1]
};

// Everything a batched launch needs about one grid, in device memory.  The
// mixed path reads the work arrays of B through float views.
struct GridDesc {
  Geom G;
  Bufs B;
  BcDesc bc;
  GasT<double> gd;  // gamma-derived constants, formed on the host
  GasT<float> gf;
  Box box[4][3];    // [stage - kStageSlopes][axis]: units of the per-axis stages
  Box seg[3];       // PPMC along y and z: the PPMC box with segments of kPpmcSeg
                    // cells along the sweep axis as units (seg[0] unused)
  Box seg2[3];      // the fast FP64 second Riemann set along y and z: its face box
                    // with segments of kPpmcSeg faces along the sweep axis as units
};

// A batched launch covers the blocks of all grids: grid order[i] owns blocks
// [prefix[i], prefix[i+1]); blocks never straddle grids.
struct BatchLaunch {
  const GridDesc* descs;
  const int* prefix;  // ngrids + 1 block offsets
  const int* order;   // grid index of each prefix slot
  int ngrids;
};

// Stages of one step; each is one kernel launch (per axis for the sweep stages).
enum Stage : int {
  kStagePrims = 0,     // ghost remap + primitives (+ dt minimum)
  kStageSetDt = 1,     // dt, dt/dx
  kStageSlopes = 2,    // limited slopes along an axis
  kStagePpmc = 3,      // traced face states along an axis
  kStageRiemann1 = 4,  // first fluxes along an axis
  kStageRiemann2 = 5,  // transverse half-step + CTU fluxes along an axis
  kStageUpdate = 6,    // conserved update
  kNumStages = 7
};

// Units (cells or faces) one launch of a stage processes.
long long stage_units(const Geom& G, int stage, int axis);

// padded cells of a grid of n[3] real cells (kNG ghost layers per active side)
inline long long padded_cells(const int n[3]) {
  long long c = 1;
  for (int d = 0; d < 3; ++d) c *= (n[d] > 1) ? (long long)n[d] + 2 * kNG : 1;
  return c;
}
// Cells or faces of a per-axis stage (kStageSlopes..kStageRiemann2).
Box stage_box_of(const Geom& G, int stage, int axis);

// Launch kinds of a (batched) step: 0 primitives, 1 update, then the four
// per-axis stages x three axes, then PPMC by segments along y and z, then the
// fast FP64 second Riemann set by segments along y and z.
constexpr int kLaunchKinds = 2 + 4 * 3 + 2 + 2;
inline int ppmc_seg_kind(int axis) { return 2 + 4 * 3 + (axis - 1); }
inline int riemann2_seg_kind(int axis) { return 2 + 4 * 3 + 2 + (axis - 1); }
// cells a thread of the segmented mixed PPMC kernels reconstructs along the
// sweep axis (y or z)
constexpr int kPpmcSeg = 4;
constexpr int kPpmcSegThreads = 128;  // threads a block of those kernels, for any schedule
inline int launch_kind(int stage, int axis) { return 2 + (stage - kStageSlopes) * 3 + axis; }
// Fill a descriptor's stage boxes and gas constants from its geometry and gamma.
void fill_desc(GridDesc& d, double gamma);
// Block-prefix tables of every launch kind for the grids in `order`, bs threads
// a block: tab = [kLaunchKinds][n+1] offsets followed by the n grid indices;
// blocks[kind] = total blocks.  Returns false if a launch would exceed 2^31 blocks.
bool build_launch_tables(const GridDesc* desc, const int* order, int n, int bs, int* tab,
                         unsigned* blocks);

// FP64 launchers (hydro_fp64.cu).  Every launcher enqueues on `st` and returns
// the launch error.
cudaError_t fp64_prims(const Geom& G, const Bufs& B, const BcDesc& bc, double gamma, bool want_dt,
                       cudaStream_t st);
// advance_time: add dt to the grid's time (a step; not a dt query)
cudaError_t fp64_set_dt(const Geom& G, const Bufs& B, double cfl, double fixed_dt, cudaStream_t st,
                        bool advance_time = true);
// one launch of a per-axis stage in the reference operation order (strict mode);
// the fast FP64 and mixed paths use the batched launchers below with one grid
cudaError_t fp64_stage_strict(const Geom& G, const Bufs& B, int recon, int solver, int stage,
                              int axis, double gamma, cudaStream_t st);
cudaError_t fp64_update(const Geom& G, const Bufs& B, cudaStream_t st);

// Batched launchers: one launch covers the given stage of every grid of a
// batch, with `bs` threads a block (128 or 256).  Precision HYDRO_FP64 or
// HYDRO_MIXED.  blocks = the batch's total block count for this stage/axis.
// noh: some grid of the launch has a Noh face
cudaError_t batch_prims(const BatchLaunch& L, int precision, int bs, unsigned blocks, cudaStream_t st,
                        bool noh = false);
cudaError_t batch_set_dt(const GridDesc* descs, int ngrids, double cfl, double* dt_hist,
                         cudaStream_t st);
cudaError_t batch_stage(const BatchLaunch& L, int precision, int recon, int solver, int stage,
                        int axis, int bs, unsigned blocks, cudaStream_t st);
cudaError_t batch_update(const BatchLaunch& L, int precision, int bs, unsigned blocks,
                         cudaStream_t st);
// batched building blocks in the fast FP64 and the mixed translation units
cudaError_t batch_stage_fp64(const BatchLaunch& L, int recon, int solver, int stage, int axis,
                             int bs, unsigned blocks, cudaStream_t st);
cudaError_t batch_stage_mixed(const BatchLaunch& L, int stage, int axis, int bs, unsigned blocks,
                              cudaStream_t st);
cudaError_t batch_prims_mixed(const BatchLaunch& L, int bs, unsigned blocks, cudaStream_t st,
                              bool noh);
cudaError_t batch_update_mixed(const BatchLaunch& L, int bs, unsigned blocks, cudaStream_t st);
// the mixed PPMC along y (axis 1) or z (axis 2) by segments (launch kind
// ppmc_seg_kind(axis), kPpmcSegThreads a block)
cudaError_t batch_ppmc_mixed_seg(const BatchLaunch& L, int axis, unsigned blocks, cudaStream_t st);
// the fast FP64 PPMC along y or z by segments (the same launch kind and blocks)
cudaError_t batch_ppmc_fp64_seg(const BatchLaunch& L, int axis, unsigned blocks, cudaStream_t st);
// the fast FP64 second Riemann set (exact solver) along y or z by segments
// (launch kind riemann2_seg_kind(axis), kPpmcSegThreads a block)
cudaError_t batch_riemann2_fp64_seg(const BatchLaunch& L, int axis, unsigned blocks,
                                    cudaStream_t st);
cudaError_t fp64_riemann_soa(int n, const double* UL, const double* UR, double gamma, double* F,
                             int* flags, cudaStream_t st);
cudaError_t fp64_ppmc_soa(int n, const double* w, double dtdx, double gamma, double* WsL,
                          double* WsR, cudaStream_t st);

}  // namespace hydro
