// hydro_internal.h -- host-side types shared by the C-ABI and the kernel files.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "hydro_math.cuh"

namespace hydro {

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
};

// Boundary description passed to the primitive kernel by value.
struct BcDesc {
  int type[6];          // HYDRO_BC_* per face x-, x+, y-, y+, z-, z+
  double inflow[6][5];  // conserved inflow state per face (rho, mx, my, mz, E)
};

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
  // [3] dt/(2 dx), [4] flags (int in the low word)
  double* rec;
};

// Box of cells (or faces: a face carries the index of the cell to its right).
struct Box {
  int lo[3];
  int n[3];
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
// per-axis stages x three axes.
constexpr int kLaunchKinds = 2 + 4 * 3;
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
cudaError_t fp64_set_dt(const Geom& G, const Bufs& B, double cfl, double fixed_dt, cudaStream_t st);
// one launch of a per-axis stage in the reference operation order (strict mode);
// the fast FP64 and mixed paths use the batched launchers below with one grid
cudaError_t fp64_stage_strict(const Geom& G, const Bufs& B, int recon, int solver, int stage,
                              int axis, double gamma, cudaStream_t st);
cudaError_t fp64_update(const Geom& G, const Bufs& B, cudaStream_t st);

// Batched launchers: one launch covers the given stage of every grid of a
// batch, with `bs` threads a block (128 or 256).  Precision HYDRO_FP64 or
// HYDRO_MIXED.  blocks = the batch's total block count for this stage/axis.
cudaError_t batch_prims(const BatchLaunch& L, int precision, int bs, unsigned blocks, cudaStream_t st);
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
cudaError_t batch_prims_mixed(const BatchLaunch& L, int bs, unsigned blocks, cudaStream_t st);
cudaError_t batch_update_mixed(const BatchLaunch& L, int bs, unsigned blocks, cudaStream_t st);
cudaError_t fp64_riemann_soa(int n, const double* UL, const double* UR, double gamma, double* F,
                             int* flags, cudaStream_t st);
cudaError_t fp64_ppmc_soa(int n, const double* w, double dtdx, double gamma, double* WsL,
                          double* WsR, cudaStream_t st);

}  // namespace hydro
