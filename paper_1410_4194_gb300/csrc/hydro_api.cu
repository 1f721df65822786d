// hydro_api.cu -- the C-ABI of include/hydro.h: handle, device memory, the
// order of the stage launches of one CTU step (Sec. 2.3), errors.
//
// All device memory of a handle is one allocation carved into 256-byte aligned
// planes.  The conserved state stays resident in HBM between steps; a step
// reads back only a 64-byte record (dt and status flags) so that hydro_step()
// can return dt, as the paper's host loop does after its reduction (Sec. 3.4).
#include <cuda_runtime.h>
#include <cmath>
#include <stdio.h>
#include <string.h>

#include <new>

#include <nvtx3/nvToolsExt.h>

#include "../../include/hydro.h"
#include "hydro_internal.h"
#include "hydro_run.h"
#include "hydro_math.cuh"

using namespace hydro;

struct hydro_s {
  Geom G;
  Bufs B;
  BcDesc bc;
  double gamma;
  int precision;
  int recon;
  int solver;
  double* eta_buf;  // H-correction planes (one per active axis), allocated for the Roe solver
  int device;
  cudaStream_t stream;
  bool have_state;
  int last_error;
  char cuda_err[256];
  void* slab;
  size_t slab_bytes;
  double* host_rec;  // pinned copy of the device step record
  // tracing: per-stage device time (CUDA events around each launch) and counts
  bool profile;
  int nev;
  cudaEvent_t ev[2 * 64];
  int ev_stage[64];
  long long ev_units[64];
  double stage_ms[kNumStages];
  long long stage_launches[kNumStages];
  long long stage_units_sum[kNumStages];
  long long launches_total;
  // the fast FP64 and mixed paths launch the batched kernels over this one grid
  GridDesc desc;
  GridDesc* d_desc;
  int* d_tab;
  unsigned blocks[kLaunchKinds];
  int bs;          // threads a block of the fast FP64 and mixed launches (128 or 256)
  int bs_choice;   // 0 = chosen from the grid size, else the caller's 128 or 256
  // device-driven runs (hydro_advance): the captured loop graph, the settings it
  // was captured with, and the private stream it was captured on
  cudaStream_t cap_stream;
  cudaGraphExec_t run_exec;
  double run_cfl;
  int run_precision, run_recon, run_solver;
  long long run_launches_per_step;
};

namespace {

int fail(hydro_t h, int code) {
  if (h) h->last_error = code;
  return code;
}

int cuda_fail(hydro_t h, cudaError_t e) {
  if (h) {
    snprintf(h->cuda_err, sizeof(h->cuda_err), "%s: %s", cudaGetErrorName(e), cudaGetErrorString(e));
    h->last_error = HYDRO_ECUDA;
  }
  return HYDRO_ECUDA;
}

#define CK(h, call)                              \
  do {                                           \
    cudaError_t e_ = (call);                     \
    if (e_ != cudaSuccess) return cuda_fail(h, e_); \
  } while (0)

int use_device(hydro_t h) {
  int cur = -1;
  cudaError_t e = cudaGetDevice(&cur);
  if (e != cudaSuccess) return cuda_fail(h, e);
  if (cur != h->device) {
    e = cudaSetDevice(h->device);
    if (e != cudaSuccess) return cuda_fail(h, e);
  }
  return HYDRO_OK;
}

size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

bool active(const Geom& G, int d) { return G.n[d] > 1; }

// Tracing: when enabled, every launch is bracketed by two events on the
// handle's stream, and by an NVTX range named after its stage for external
// profilers; times are folded into per-stage totals once the step has
// completed (hydro_step waits for its record anyway).
const char* const kStageRange[kNumStages] = {"hydro prims+dt", "hydro dt",       "hydro slopes",
                                             "hydro reconstruction", "hydro riemann1",
                                             "hydro riemann2", "hydro update"};

int mark_begin(hydro_t h, int stage, int axis) {
  ++h->launches_total;
  if (!h->profile || h->nev >= 64) return HYDRO_OK;
  nvtxRangePushA(kStageRange[stage]);
  const int k = h->nev;
  h->ev_stage[k] = stage;
  h->ev_units[k] = stage_units(h->G, stage, axis);
  CK(h, cudaEventRecord(h->ev[2 * k], h->stream));
  return HYDRO_OK;
}

int mark_end(hydro_t h) {
  if (!h->profile || h->nev >= 64) return HYDRO_OK;
  nvtxRangePop();
  CK(h, cudaEventRecord(h->ev[2 * h->nev + 1], h->stream));
  ++h->nev;
  return HYDRO_OK;
}

int fold_events(hydro_t h) {
  for (int k = 0; k < h->nev; ++k) {
    float ms = 0.f;
    CK(h, cudaEventElapsedTime(&ms, h->ev[2 * k], h->ev[2 * k + 1]));
    h->stage_ms[h->ev_stage[k]] += ms;
    h->stage_launches[h->ev_stage[k]] += 1;
    h->stage_units_sum[h->ev_stage[k]] += h->ev_units[k];
  }
  h->nev = 0;
  return HYDRO_OK;
}

BatchLaunch one_grid(hydro_t h, int kind) {
  BatchLaunch L;
  L.descs = h->d_desc;
  L.prefix = h->d_tab + 2 * kind;
  L.order = h->d_tab + 2 * kLaunchKinds;
  L.ngrids = 1;
  return L;
}

#define STAGE(h, stage, axis, call)          \
  do {                                       \
    int rc_ = mark_begin(h, stage, axis);    \
    if (rc_) return rc_;                     \
    cudaError_t e_ = (call);                 \
    if (e_ != cudaSuccess) return cuda_fail(h, e_); \
    rc_ = mark_end(h);                       \
    if (rc_) return rc_;                     \
  } while (0)

// Enqueue one full step; dt from the CFL condition when fixed_dt <= 0, cut back
// to the end time in the record's slot 8 when to_end is set.
// keep_flags: leave the status word of earlier steps (asynchronous steps, whose
// status is read by hydro_sync).
int enqueue_step(hydro_t h, double cfl, double fixed_dt, bool to_end = false,
                 bool keep_flags = false) {
  const Geom& G = h->G;
  const Bufs& B = h->B;
  cudaStream_t st = h->stream;
  h->nev = 0;
  if (!keep_flags) CK(h, cudaMemsetAsync(B.rec + 4, 0, sizeof(double), st));
  if (h->precision == HYDRO_FP64_STRICT) {
    STAGE(h, kStagePrims, 0, fp64_prims(G, B, h->bc, h->gamma, fixed_dt <= 0.0, st));
    STAGE(h, kStageSetDt, 0,
          to_end ? set_dt_to_end(G, B, cfl, st) : fp64_set_dt(G, B, cfl, fixed_dt, st));
    for (int d = 0; d < 3; ++d) {
      if (!active(G, d)) continue;
      for (int s = kStageSlopes; s <= kStageRiemann1; ++s) {
        if (s == kStageSlopes && h->recon == HYDRO_RECON_PCM) continue;  // no slopes
        STAGE(h, s, d, fp64_stage_strict(G, B, h->recon, h->solver, s, d, h->gamma, st));
      }
    }
    for (int d = 0; d < 3; ++d)
      if (active(G, d))
        STAGE(h, kStageRiemann2, d,
              fp64_stage_strict(G, B, h->recon, h->solver, kStageRiemann2, d, h->gamma, st));
    STAGE(h, kStageUpdate, 0, fp64_update(G, B, st));
    return HYDRO_OK;
  }
  // fast FP64 or mixed: the batched kernels over this single grid (256 threads)
  const int P = h->precision;
  CK(h, cudaMemsetAsync(B.rec, 0, sizeof(double), st));
  STAGE(h, kStagePrims, 0, batch_prims(one_grid(h, 0), P, h->bs, h->blocks[0], st, has_noh(h->bc)));
  STAGE(h, kStageSetDt, 0,
        to_end ? set_dt_to_end(G, B, cfl, st) : fp64_set_dt(G, B, cfl, fixed_dt, st));
  for (int d = 0; d < 3; ++d) {
    if (!active(G, d)) continue;
    for (int s = kStageSlopes; s <= kStageRiemann1; ++s) {
      // no slope pass for PCM; the mixed PPMC kernel forms its own slopes
      if (s == kStageSlopes && (h->recon == HYDRO_RECON_PCM || P == HYDRO_MIXED)) continue;
      if (s == kStagePpmc && d > 0 && (P == HYDRO_MIXED || h->recon == HYDRO_RECON_PPMC)) {
        const int k = ppmc_seg_kind(d);  // PPMC by segments along y and z
        STAGE(h, s, d,
              P == HYDRO_MIXED ? batch_ppmc_mixed_seg(one_grid(h, k), d, h->blocks[k], st)
                               : batch_ppmc_fp64_seg(one_grid(h, k), d, h->blocks[k], st));
        continue;
      }
      const int k = launch_kind(s, d);
      STAGE(h, s, d,
            batch_stage(one_grid(h, k), P, h->recon, h->solver, s, d, h->bs, h->blocks[k], st));
    }
  }
  for (int d = 0; d < 3; ++d) {
    if (!active(G, d)) continue;
    if (d > 0 && P == HYDRO_FP64 && h->solver == HYDRO_RIEMANN_EXACT) {  // by segments
      const int k = riemann2_seg_kind(d);
      STAGE(h, kStageRiemann2, d, batch_riemann2_fp64_seg(one_grid(h, k), d, h->blocks[k], st));
      continue;
    }
    const int k = launch_kind(kStageRiemann2, d);
    STAGE(h, kStageRiemann2, d,
          batch_stage(one_grid(h, k), P, h->recon, h->solver, kStageRiemann2, d, h->bs,
                      h->blocks[k], st));
  }
  STAGE(h, kStageUpdate, 0, batch_update(one_grid(h, 1), P, h->bs, h->blocks[1], st));
  return HYDRO_OK;
}

int read_record(hydro_t h, int n = 8) {
  CK(h, cudaMemcpyAsync(h->host_rec, h->B.rec, n * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
  CK(h, cudaStreamSynchronize(h->stream));
  return HYDRO_OK;
}

double run_step(hydro_t h, double cfl, double fixed_dt) {
  if (!h) return (double)HYDRO_EINVAL;
  h->last_error = HYDRO_OK;
  if (!h->have_state) return (double)fail(h, HYDRO_ENOSTATE);
  if (fixed_dt <= 0.0 && !(cfl > 0.0)) return (double)fail(h, HYDRO_EINVAL);
  int rc = use_device(h);
  if (rc) return (double)rc;
  rc = enqueue_step(h, cfl, fixed_dt);
  if (rc) return (double)rc;
  rc = read_record(h);
  if (rc) return (double)rc;
  if (h->profile) {
    rc = fold_events(h);
    if (rc) return (double)rc;
  }
  int flags;
  memcpy(&flags, h->host_rec + 4, sizeof(int));
  if (flags & kFlagNonPhys) return (double)fail(h, HYDRO_ENONPHYS);
  if (flags & kFlagNewton) return (double)fail(h, HYDRO_ENEWTON);
  return h->host_rec[1];
}

// Threads a block when the caller left the choice to the library: 128.  Timed
// against 256 on Sedov grids from 32^3 to 256^3 and on a 512-cell tube, 128 was
// never slower: equal for FP64 at 128^3 and up, 3% faster for mixed precision at
// 256^3, and 5-30% faster on small grids, which spread over twice as many SMs
// (one warp per SM sub-partition instead of two on the FP64 pipe).
int auto_block_size(const Geom&) { return 128; }

// Launch tables of the one-grid descriptor for bs threads a block, copied to
// the device (synchronously: no launch of this handle may be reading them).
int set_block_size(hydro_t h, int bs) {
  int tab[2 * kLaunchKinds + 1];
  unsigned blocks[kLaunchKinds];
  const int zero = 0;
  if (!build_launch_tables(&h->desc, &zero, 1, bs, tab, blocks)) return fail(h, HYDRO_EINVAL);
  if (h->stream) CK(h, cudaStreamSynchronize(h->stream));
  CK(h, cudaMemcpy(h->d_tab, tab, sizeof(tab), cudaMemcpyHostToDevice));
  for (int k = 0; k < kLaunchKinds; ++k) h->blocks[k] = blocks[k];
  h->bs = bs;
  return HYDRO_OK;
}

void drop_run_graph(hydro_t h) {
  if (h->run_exec) {
    if (h->stream) cudaStreamSynchronize(h->stream);
    else cudaDeviceSynchronize();
    cudaGraphExecDestroy(h->run_exec);
  }
  h->run_exec = nullptr;
}

// Steps a graph launch may take: about 2^26 cell updates (a fraction of a
// second even in FP64), at least one step and at most 4096.
double run_chunk(const Geom& G) {
  const long long c = (1ll << 26) / (G.nreal > 0 ? G.nreal : 1);
  return (double)(c < 1 ? 1 : (c > 4096 ? 4096 : c));
}

// Capture the loop graph of device-driven runs: a kernel that sets the loop
// condition, then a WHILE node whose body is one step (the stage launches of
// enqueue_step with the end-time dt) and the kernel that updates the condition.
// Captured on a private stream (the handle's stream may be the legacy default
// stream, which cannot be captured), without tracing events.
int capture_run_graph(hydro_t h, double cfl) {
  drop_run_graph(h);
  if (!h->cap_stream) CK(h, cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking));
  cudaStream_t cs = h->cap_stream;
  cudaGraph_t graph = nullptr;
  CK(h, cudaGraphCreate(&graph, 0));
  int rc = HYDRO_OK;
  cudaError_t e = cudaSuccess;
  cudaGraphConditionalHandle cond = 0;
  cudaGraphNode_t begin = nullptr, loop = nullptr;
  size_t nnodes = 1;
  cudaGraphNodeParams cp = {cudaGraphNodeTypeConditional};
  const cudaStream_t user_stream = h->stream;
  const bool profile = h->profile;
  const long long launches0 = h->launches_total;
  e = cudaGraphConditionalHandleCreate(&cond, graph, 0, cudaGraphCondAssignDefault);
  if (e == cudaSuccess)
    e = cudaStreamBeginCaptureToGraph(cs, graph, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal);
  if (e == cudaSuccess) {
    cudaError_t e1 = run_begin(h->B.rec, cond, cs);
    cudaGraph_t g_out = nullptr;
    e = cudaStreamEndCapture(cs, &g_out);
    if (e == cudaSuccess) e = e1;
  }
  if (e == cudaSuccess) e = cudaGraphGetNodes(graph, &begin, &nnodes);
  if (e == cudaSuccess && nnodes != 1) e = cudaErrorInvalidValue;
  if (e == cudaSuccess) {
    cp.conditional.handle = cond;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    e = cudaGraphAddNode(&loop, graph, &begin, nullptr, 1, &cp);
  }
  if (e == cudaSuccess)
    e = cudaStreamBeginCaptureToGraph(cs, cp.conditional.phGraph_out[0], nullptr, nullptr, 0,
                                      cudaStreamCaptureModeThreadLocal);
  if (e == cudaSuccess) {
    h->stream = cs;
    h->profile = false;
    rc = enqueue_step(h, cfl, 0.0, true);
    cudaError_t e1 = rc ? cudaSuccess : run_next(h->B.rec, cond, run_chunk(h->G), cs);
    h->stream = user_stream;
    h->profile = profile;
    h->run_launches_per_step = h->launches_total - launches0 + 1;
    h->launches_total = launches0;
    cudaGraph_t g_out = nullptr;
    e = cudaStreamEndCapture(cs, &g_out);
    if (e == cudaSuccess) e = e1;
  }
  if (rc == HYDRO_OK && e == cudaSuccess) e = cudaGraphInstantiate(&h->run_exec, graph, 0);
  cudaGraphDestroy(graph);
  if (rc) return rc;
  if (e != cudaSuccess) {
    h->run_exec = nullptr;
    return cuda_fail(h, e);
  }
  h->run_cfl = cfl;
  h->run_precision = h->precision;
  h->run_recon = h->recon;
  h->run_solver = h->solver;
  return HYDRO_OK;
}

}  // namespace

extern "C" {

int hydro_init(hydro_t* out, int nx, int ny, int nz, double dx, double gamma, const int bc[6]) {
  if (!out) return HYDRO_EINVAL;
  *out = nullptr;
  if (!bc || !(dx > 0.0) || !(gamma > 1.0)) return HYDRO_EINVAL;
  const int n[3] = {nx, ny, nz};
  for (int d = 0; d < 3; ++d) {
    if (n[d] < 1 || (n[d] > 1 && n[d] < kNG)) return HYDRO_EINVAL;
    if (n[d] > 1 && (bc[2 * d] < 0 || bc[2 * d] > HYDRO_BC_NOH || bc[2 * d + 1] < 0 ||
                     bc[2 * d + 1] > HYDRO_BC_NOH))
      return HYDRO_EINVAL;
    if (n[d] > 1 && ((bc[2 * d] == HYDRO_BC_PERIODIC) != (bc[2 * d + 1] == HYDRO_BC_PERIODIC)))
      return HYDRO_EINVAL;
  }
  if (padded_cells(n) >= (1ll << 31)) return HYDRO_EINVAL;  // kernels index in 32 bits
  hydro_t h = new (std::nothrow) hydro_s();
  if (!h) return HYDRO_ENOMEM;
  h->profile = false;
  h->nev = 0;
  h->launches_total = 0;
  for (int k = 0; k < kNumStages; ++k) {
    h->stage_ms[k] = 0.0;
    h->stage_launches[k] = 0;
    h->stage_units_sum[k] = 0;
  }
  memset(h->cuda_err, 0, sizeof(h->cuda_err));
  h->gamma = gamma;
  h->precision = HYDRO_FP64;
  h->recon = HYDRO_RECON_PPMC;
  h->solver = HYDRO_RIEMANN_EXACT;
  h->eta_buf = nullptr;
  h->stream = nullptr;
  h->cap_stream = nullptr;
  h->run_exec = nullptr;
  h->have_state = false;
  h->last_error = HYDRO_OK;
  cudaError_t e = cudaGetDevice(&h->device);
  if (e != cudaSuccess) {
    delete h;
    return HYDRO_ECUDA;
  }
  Geom& G = h->G;
  for (int d = 0; d < 3; ++d) {
    G.n[d] = n[d];
    G.g[d] = n[d] > 1 ? kNG : 0;
    G.N[d] = n[d] + 2 * G.g[d];
  }
  G.s[0] = 1;
  G.s[1] = G.N[0];
  G.s[2] = (long long)G.N[0] * G.N[1];
  G.ps = (long long)align_up((size_t)G.N[0] * G.N[1] * G.N[2], 32);
  G.nreal = (long long)nx * ny * nz;
  geom_divisors(G);
  G.dx = dx;
  for (int f = 0; f < 6; ++f) {
    h->bc.type[f] = (n[f / 2] > 1) ? bc[f] : HYDRO_BC_PERIODIC;
    for (int q = 0; q < 5; ++q) h->bc.inflow[f][q] = 0.0;
  }
  // one slab: u, W (8 planes), S (5), per active axis UL/UR/F1 (15), record
  int nact = 0;
  for (int d = 0; d < 3; ++d) nact += active(G, d) ? 1 : 0;
  const size_t plane = (size_t)G.ps * sizeof(double);
  const size_t ubytes = align_up((size_t)G.nreal * 5 * sizeof(double), 256);
  const size_t total = ubytes + plane * (8 + 5 + 15 * (size_t)nact) + 256;
  h->slab_bytes = total;
  e = cudaMalloc(&h->slab, total);
  if (e != cudaSuccess) {
    cudaGetLastError();
    delete h;
    return HYDRO_ENOMEM;
  }
  e = cudaMallocHost((void**)&h->host_rec, 16 * sizeof(double));
  if (e != cudaSuccess) {
    cudaFree(h->slab);
    delete h;
    return HYDRO_ENOMEM;
  }
  char* p = static_cast<char*>(h->slab);
  Bufs& B = h->B;
  B.u = reinterpret_cast<double*>(p);
  p += ubytes;
  B.W = reinterpret_cast<double*>(p);
  p += 8 * plane;
  B.S = reinterpret_cast<double*>(p);
  p += 5 * plane;
  for (int d = 0; d < 3; ++d) {
    B.UL[d] = B.UR[d] = B.F1[d] = nullptr;
    if (!active(G, d)) continue;
    B.UL[d] = reinterpret_cast<double*>(p);
    p += 5 * plane;
    B.UR[d] = reinterpret_cast<double*>(p);
    p += 5 * plane;
    B.F1[d] = reinterpret_cast<double*>(p);
    p += 5 * plane;
  }
  B.rec = reinterpret_cast<double*>(p);
  // one-grid descriptor and launch tables for the batched kernels
  memset(&h->desc, 0, sizeof(h->desc));
  h->desc.G = G;
  h->desc.B = B;
  h->desc.bc = h->bc;
  fill_desc(h->desc, gamma);
  int tab[2 * kLaunchKinds + 1];
  const int zero = 0;
  h->d_desc = nullptr;
  h->d_tab = nullptr;
  h->bs_choice = 0;
  h->bs = auto_block_size(G);
  if (!build_launch_tables(&h->desc, &zero, 1, h->bs, tab, h->blocks)) {
    cudaFreeHost(h->host_rec);
    cudaFree(h->slab);
    delete h;
    return HYDRO_EINVAL;
  }
  e = cudaMemset(h->slab, 0, total);
  if (e == cudaSuccess) e = cudaMalloc(&h->d_desc, sizeof(GridDesc));
  if (e == cudaSuccess) e = cudaMalloc(&h->d_tab, sizeof(tab));
  if (e == cudaSuccess) e = cudaMemcpy(h->d_desc, &h->desc, sizeof(GridDesc), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(h->d_tab, tab, sizeof(tab), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) {
    cudaGetLastError();
    if (h->d_desc) cudaFree(h->d_desc);
    if (h->d_tab) cudaFree(h->d_tab);
    cudaFreeHost(h->host_rec);
    cudaFree(h->slab);
    delete h;
    return e == cudaErrorMemoryAllocation ? HYDRO_ENOMEM : HYDRO_ECUDA;
  }
  *out = h;
  return HYDRO_OK;
}

int hydro_set_inflow(hydro_t h, int face, const double prim[5]) {
  if (!h) return HYDRO_EINVAL;
  h->last_error = HYDRO_OK;
  if (face < 0 || face > 5 || !prim) return fail(h, HYDRO_EINVAL);
  if (!(prim[0] > 0.0) || !(prim[4] >= 0.0)) return fail(h, HYDRO_EINVAL);
  double* U = h->bc.inflow[face];
  for (int q = 0; q < 5; ++q) h->bc.prim[face][q] = prim[q];
  U[0] = prim[0];
  U[1] = prim[0] * prim[1];
  U[2] = prim[0] * prim[2];
  U[3] = prim[0] * prim[3];
  U[4] = prim[4] / (h->gamma - 1.0) + 0.5 * prim[0] * (prim[1] * prim[1] + prim[2] * prim[2] + prim[3] * prim[3]);
  h->desc.bc = h->bc;
  int rc = use_device(h);
  if (rc) return rc;
  drop_run_graph(h);  // the strict path takes the boundary description by value
  CK(h, cudaMemcpy(&h->d_desc->bc, &h->bc, sizeof(BcDesc), cudaMemcpyHostToDevice));
  return HYDRO_OK;
}

int hydro_set_time(hydro_t h, double t) {
  if (!h) return HYDRO_EINVAL;
  h->last_error = HYDRO_OK;
  if (!std::isfinite(t) || t < 0.0) return fail(h, HYDRO_EINVAL);
  int rc = use_device(h);
  if (rc) return rc;
  CK(h, cudaStreamSynchronize(h->stream));
  CK(h, cudaMemcpy(h->B.rec + 5, &t, sizeof(double), cudaMemcpyHostToDevice));
  return HYDRO_OK;
}

double hydro_get_time(hydro_t h) {
  if (!h) return (double)HYDRO_EINVAL;
  h->last_error = HYDRO_OK;
  int rc = use_device(h);
  if (rc) return (double)rc;
  rc = read_record(h);
  if (rc) return (double)rc;
  return h->host_rec[5];
}

int hydro_set_precision(hydro_t h, int mode) {
  if (!h) return HYDRO_EINVAL;
  h->last_error = HYDRO_OK;
  if (mode != HYDRO_FP64 && mode != HYDRO_FP64_STRICT && mode != HYDRO_MIXED)
    return fail(h, HYDRO_EINVAL);
  if (mode == HYDRO_MIXED && (h->recon != HYDRO_RECON_PPMC || h->solver != HYDRO_RIEMANN_EXACT))
    return fail(h, HYDRO_EINVAL);
  h->precision = mode;
  return HYDRO_OK;
}

int hydro_set_reconstruction(hydro_t h, int recon) {
  if (!h) return HYDRO_EINVAL;
  h->last_error = HYDRO_OK;
  if (recon < HYDRO_RECON_PPMC || recon > HYDRO_RECON_PCM) return fail(h, HYDRO_EINVAL);
  if (recon != HYDRO_RECON_PPMC && h->precision == HYDRO_MIXED) return fail(h, HYDRO_EINVAL);
  h->recon = recon;
  return HYDRO_OK;
}

int hydro_set_riemann_solver(hydro_t h, int solver) {
  if (!h) return HYDRO_EINVAL;
  h->last_error = HYDRO_OK;
  if (solver != HYDRO_RIEMANN_EXACT && solver != HYDRO_RIEMANN_ROE) return fail(h, HYDRO_EINVAL);
  if (solver != HYDRO_RIEMANN_EXACT && h->precision == HYDRO_MIXED) return fail(h, HYDRO_EINVAL);
  if (solver == HYDRO_RIEMANN_ROE && !h->eta_buf) {
    int rc = use_device(h);
    if (rc) return rc;
    int nact = 0;
    for (int d = 0; d < 3; ++d) nact += active(h->G, d) ? 1 : 0;
    const size_t plane = (size_t)h->G.ps * sizeof(double);
    cudaError_t e = cudaMalloc(&h->eta_buf, plane * (size_t)nact);
    if (e != cudaSuccess) {
      cudaGetLastError();
      h->eta_buf = nullptr;
      return fail(h, HYDRO_ENOMEM);
    }
    double* p = h->eta_buf;
    for (int d = 0; d < 3; ++d) {
      h->B.eta[d] = nullptr;
      if (!active(h->G, d)) continue;
      h->B.eta[d] = p;
      p += h->G.ps;
    }
    h->desc.B = h->B;
    CK(h, cudaMemcpy(h->d_desc, &h->desc, sizeof(GridDesc), cudaMemcpyHostToDevice));
  }
  h->solver = solver;
  return HYDRO_OK;
}

int hydro_set_block_size(hydro_t h, int bs) {
  if (!h) return HYDRO_EINVAL;
  h->last_error = HYDRO_OK;
  if (bs != 0 && bs != 128 && bs != 256) return fail(h, HYDRO_EINVAL);
  int rc = use_device(h);
  if (rc) return rc;
  const int want = bs ? bs : auto_block_size(h->G);
  if (want != h->bs) {
    drop_run_graph(h);
    rc = set_block_size(h, want);
    if (rc) return rc;
  }
  h->bs_choice = bs;
  return HYDRO_OK;
}

int hydro_block_size(hydro_t h) {
  if (!h) return HYDRO_EINVAL;
  h->last_error = HYDRO_OK;
  return h->bs;
}

int hydro_set_stream(hydro_t h, void* stream) {
  if (!h) return HYDRO_EINVAL;
  h->last_error = HYDRO_OK;
  h->stream = static_cast<cudaStream_t>(stream);
  return HYDRO_OK;
}

int hydro_set_state(hydro_t h, const double* u, int on_device) {
  if (!h) return HYDRO_EINVAL;
  h->last_error = HYDRO_OK;
  if (!u) return fail(h, HYDRO_EINVAL);
  int rc = use_device(h);
  if (rc) return rc;
  const size_t bytes = (size_t)h->G.nreal * 5 * sizeof(double);
  CK(h, cudaMemcpyAsync(h->B.u, u, bytes, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                        h->stream));
  CK(h, cudaStreamSynchronize(h->stream));
  h->have_state = true;
  return HYDRO_OK;
}

int hydro_get_state(hydro_t h, double* u, int on_device) {
  if (!h) return HYDRO_EINVAL;
  h->last_error = HYDRO_OK;
  if (!u) return fail(h, HYDRO_EINVAL);
  if (!h->have_state) return fail(h, HYDRO_ENOSTATE);
  int rc = use_device(h);
  if (rc) return rc;
  const size_t bytes = (size_t)h->G.nreal * 5 * sizeof(double);
  CK(h, cudaMemcpyAsync(u, h->B.u, bytes, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                        h->stream));
  CK(h, cudaStreamSynchronize(h->stream));
  return HYDRO_OK;
}

double hydro_step(hydro_t h, double cfl) { return run_step(h, cfl, 0.0); }

int hydro_set_state_async(hydro_t h, const double* u, int on_device) {
  if (!h) return HYDRO_EINVAL;
  h->last_error = HYDRO_OK;
  if (!u) return fail(h, HYDRO_EINVAL);
  int rc = use_device(h);
  if (rc) return rc;
  const size_t bytes = (size_t)h->G.nreal * 5 * sizeof(double);
  CK(h, cudaMemcpyAsync(h->B.u, u, bytes, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                        h->stream));
  h->have_state = true;
  return HYDRO_OK;
}

int hydro_get_state_async(hydro_t h, double* u, int on_device) {
  if (!h) return HYDRO_EINVAL;
  h->last_error = HYDRO_OK;
  if (!u) return fail(h, HYDRO_EINVAL);
  if (!h->have_state) return fail(h, HYDRO_ENOSTATE);
  int rc = use_device(h);
  if (rc) return rc;
  const size_t bytes = (size_t)h->G.nreal * 5 * sizeof(double);
  CK(h, cudaMemcpyAsync(u, h->B.u, bytes, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                        h->stream));
  return HYDRO_OK;
}

int hydro_step_async(hydro_t h, double cfl) {
  if (!h) return HYDRO_EINVAL;
  h->last_error = HYDRO_OK;
  if (!h->have_state) return fail(h, HYDRO_ENOSTATE);
  if (!(cfl > 0.0)) return fail(h, HYDRO_EINVAL);
  int rc = use_device(h);
  if (rc) return rc;
  // not traced: the events of a step are folded only once it has completed
  const bool profile = h->profile;
  h->profile = false;
  rc = enqueue_step(h, cfl, 0.0, false, true);
  h->profile = profile;
  return rc;
}

int hydro_sync(hydro_t h, double* dt_out) {
  if (!h) return HYDRO_EINVAL;
  h->last_error = HYDRO_OK;
  int rc = use_device(h);
  if (rc) return rc;
  rc = read_record(h);  // waits for the handle's stream
  if (rc) return rc;
  if (dt_out) *dt_out = h->host_rec[1];
  int flags;
  memcpy(&flags, h->host_rec + 4, sizeof(int));
  if (flags) {
    CK(h, cudaMemsetAsync(h->B.rec + 4, 0, sizeof(double), h->stream));
    CK(h, cudaStreamSynchronize(h->stream));
  }
  if (flags & kFlagNonPhys) return fail(h, HYDRO_ENONPHYS);
  if (flags & kFlagNewton) return fail(h, HYDRO_ENEWTON);
  return HYDRO_OK;
}

double hydro_step_dt(hydro_t h, double dt) {
  if (!h) return (double)HYDRO_EINVAL;
  if (!(dt > 0.0)) return (double)fail(h, HYDRO_EINVAL);
  return run_step(h, 0.0, dt);
}

int hydro_advance(hydro_t h, double cfl, double t_end, long long max_steps, long long* steps_out) {
  if (!h) return HYDRO_EINVAL;
  h->last_error = HYDRO_OK;
  if (steps_out) *steps_out = 0;
  if (!h->have_state) return fail(h, HYDRO_ENOSTATE);
  if (!(cfl > 0.0) || std::isnan(t_end) || max_steps < 0 || max_steps > (1ll << 52))
    return fail(h, HYDRO_EINVAL);
  int rc = use_device(h);
  if (rc) return rc;
  const bool same = h->run_exec && h->run_cfl == cfl && h->run_precision == h->precision &&
                    h->run_recon == h->recon && h->run_solver == h->solver;
  if (!same) {
    rc = capture_run_graph(h, cfl);
    if (rc) return rc;
  }
  // end time and step budget into the record (the pinned copy is not touched
  // again before the stream has read it: read_record below waits on the stream)
  h->host_rec[8] = t_end;
  h->host_rec[9] = (double)max_steps;
  CK(h, cudaMemcpyAsync(h->B.rec + 8, h->host_rec + 8, 2 * sizeof(double), cudaMemcpyHostToDevice,
                        h->stream));
  long long done = 0;
  for (;;) {
    nvtxRangePushA("hydro advance (graph launch)");
    const cudaError_t le = cudaGraphLaunch(h->run_exec, h->stream);
    nvtxRangePop();
    CK(h, le);
    rc = read_record(h, 11);
    if (rc) return rc;
    const long long n = (long long)h->host_rec[10];
    done += n;
    h->launches_total += 1 + n * h->run_launches_per_step;
    if (steps_out) *steps_out = done;
    int flags;
    memcpy(&flags, h->host_rec + 4, sizeof(int));
    if (n > 0 && (flags & kFlagNonPhys)) return fail(h, HYDRO_ENONPHYS);
    if (n > 0 && (flags & kFlagNewton)) return fail(h, HYDRO_ENEWTON);
    if (n == 0 || !(h->host_rec[5] < t_end) || h->host_rec[9] < 1.0) break;
  }
  return HYDRO_OK;
}

double hydro_compute_dt(hydro_t h, double cfl) {
  if (!h) return (double)HYDRO_EINVAL;
  h->last_error = HYDRO_OK;
  if (!h->have_state) return (double)fail(h, HYDRO_ENOSTATE);
  if (!(cfl > 0.0)) return (double)fail(h, HYDRO_EINVAL);
  int rc = use_device(h);
  if (rc) return (double)rc;
  cudaError_t e;
  if (h->precision == HYDRO_FP64_STRICT) {
    e = fp64_prims(h->G, h->B, h->bc, h->gamma, true, h->stream);
  } else {
    e = cudaMemsetAsync(h->B.rec, 0, sizeof(double), h->stream);
    if (e == cudaSuccess)
      e = batch_prims(one_grid(h, 0), h->precision, h->bs, h->blocks[0], h->stream, has_noh(h->bc));
  }
  if (e != cudaSuccess) return (double)cuda_fail(h, e);
  e = fp64_set_dt(h->G, h->B, cfl, 0.0, h->stream, false);
  if (e != cudaSuccess) return (double)cuda_fail(h, e);
  h->launches_total += 2;
  rc = read_record(h);
  if (rc) return (double)rc;
  return h->host_rec[1];
}

int hydro_last_error(hydro_t h) { return h ? h->last_error : HYDRO_EINVAL; }

const char* hydro_error_string(int code) {
  switch (code) {
    case HYDRO_OK: return "ok";
    case HYDRO_EINVAL: return "invalid argument";
    case HYDRO_ENOMEM: return "out of memory";
    case HYDRO_ECUDA: return "CUDA runtime error";
    case HYDRO_ENONPHYS: return "non-physical state (rho <= 0 or NaN) after the step";
    case HYDRO_ENEWTON: return "Riemann Newton iteration reached its cap";
    case HYDRO_ENOSTATE: return "no state set";
    default: return "unknown error";
  }
}

const char* hydro_cuda_error_string(hydro_t h) { return h ? h->cuda_err : ""; }

int hydro_profile(hydro_t h, int enable) {
  if (!h) return HYDRO_EINVAL;
  h->last_error = HYDRO_OK;
  int rc = use_device(h);
  if (rc) return rc;
  if (enable && !h->profile) {
    for (int k = 0; k < 2 * 64; ++k) CK(h, cudaEventCreate(&h->ev[k]));
    h->profile = true;
  } else if (!enable && h->profile) {
    CK(h, cudaStreamSynchronize(h->stream));
    for (int k = 0; k < 2 * 64; ++k) cudaEventDestroy(h->ev[k]);
    h->profile = false;
  }
  for (int k = 0; k < kNumStages; ++k) {
    h->stage_ms[k] = 0.0;
    h->stage_launches[k] = 0;
    h->stage_units_sum[k] = 0;
  }
  h->launches_total = 0;
  h->nev = 0;
  return HYDRO_OK;
}

int hydro_profile_read(hydro_t h, int nstages, double* ms, long long* launches, long long* units,
                       long long* launches_total) {
  if (!h) return HYDRO_EINVAL;
  h->last_error = HYDRO_OK;
  if (nstages < 0 || nstages > kNumStages) return fail(h, HYDRO_EINVAL);
  for (int k = 0; k < nstages; ++k) {
    if (ms) ms[k] = h->stage_ms[k];
    if (launches) launches[k] = h->stage_launches[k];
    if (units) units[k] = h->stage_units_sum[k];
  }
  if (launches_total) *launches_total = h->launches_total;
  return HYDRO_OK;
}

void hydro_free(hydro_t h) {
  if (!h) return;
  int cur = -1;
  if (cudaGetDevice(&cur) == cudaSuccess && cur != h->device) cudaSetDevice(h->device);
  if (h->stream) cudaStreamSynchronize(h->stream);
  else cudaDeviceSynchronize();
  drop_run_graph(h);
  if (h->cap_stream) cudaStreamDestroy(h->cap_stream);
  if (h->profile)
    for (int k = 0; k < 2 * 64; ++k) cudaEventDestroy(h->ev[k]);
  cudaFree(h->slab);
  if (h->eta_buf) cudaFree(h->eta_buf);
  cudaFree(h->d_desc);
  cudaFree(h->d_tab);
  cudaFreeHost(h->host_rec);
  if (cur >= 0 && cur != h->device) cudaSetDevice(cur);
  delete h;
}

int hydro_riemann_exact(int n, const double* UL, const double* UR, double gamma, double* F,
                        int* flags, void* stream) {
  if (n < 0 || (n > 0 && (!UL || !UR || !F)) || !(gamma > 1.0)) return HYDRO_EINVAL;
  cudaError_t e = fp64_riemann_soa(n, UL, UR, gamma, F, flags, static_cast<cudaStream_t>(stream));
  return e == cudaSuccess ? HYDRO_OK : HYDRO_ECUDA;
}

int hydro_ppmc(int n, const double* w, double dtdx, double gamma, double* WsL, double* WsR,
               void* stream) {
  if (n < 0 || (n > 0 && (!w || !WsL || !WsR)) || !(gamma > 1.0) || !(dtdx >= 0.0))
    return HYDRO_EINVAL;
  cudaError_t e = fp64_ppmc_soa(n, w, dtdx, gamma, WsL, WsR, static_cast<cudaStream_t>(stream));
  return e == cudaSuccess ? HYDRO_OK : HYDRO_ECUDA;
}

}  // extern "C"
