// hydro_batch.cu -- many independent grids of uneven sizes advanced together.
//
// The paper suggests running many problems at once on the GPUs (Sec. 5); here
// each stage of the CTU step (Sec. 2.3) is one launch over the blocks of every
// grid of a batch (a block never straddles two grids, so the per-block dt
// reduction still lands in its own grid's record), every grid keeps its own
// dt, and nsteps steps are captured once into a CUDA graph and replayed with a
// single graph launch.  The schedule -- thread-block size and the order in which
// the grids' blocks are laid out -- is chosen by measurement (autotuner below)
// and remembered per batch shape and device in a small text cache.
#include <cuda_runtime.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>
#include <sys/stat.h>

#include <algorithm>
#include <new>
#include <string>
#include <vector>

#include "../../include/hydro.h"
#include "hydro_internal.h"

using namespace hydro;

namespace {

struct Schedule {
  int bs = 128;    // threads a block (the single-grid default; the autotuner may pick 256)
  int order = 0;   // 0: grids in the given order, 1: largest grid first
};

}  // namespace

struct hydro_batch_s {
  int ngrids = 0;
  int precision = HYDRO_FP64;
  int recon = HYDRO_RECON_PPMC;
  int solver = HYDRO_RIEMANN_EXACT;
  double* eta_buf = nullptr;       // H-correction planes of every grid (Roe solver)
  int device = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  std::vector<GridDesc> desc;      // host copy
  GridDesc* d_desc = nullptr;      // device copy
  void* slab = nullptr;
  double* recs = nullptr;          // [ngrids][8] step records (inside the slab)
  std::vector<char> have_state;
  Schedule sched;
  bool tuned = false;
  // launch tables for the current schedule: per kind, ngrids+1 block offsets
  int* d_tables = nullptr;         // [kLaunchKinds][ngrids+1] then order [ngrids]
  unsigned blocks[kLaunchKinds] = {0};
  bool axis_used[3] = {false, false, false};
  // dt history of the last call: [nsteps][ngrids]
  double* d_dt = nullptr;
  int dt_cap = 0;
  // captured graph of the last call shape
  cudaGraphExec_t gexec = nullptr;
  int g_nsteps = -1;
  double g_cfl = -1.0;
  int g_precision = -1;
  int g_recon = -1;
  int g_solver = -1;
  Schedule g_sched;
  int last_error = HYDRO_OK;
  char cuda_err[256] = {0};
  float tune_ms[4] = {0, 0, 0, 0};
};

namespace {

int bfail(hydro_batch_t h, int code) {
  if (h) h->last_error = code;
  return code;
}

int bcuda(hydro_batch_t h, cudaError_t e) {
  if (h) {
    snprintf(h->cuda_err, sizeof(h->cuda_err), "%s: %s", cudaGetErrorName(e), cudaGetErrorString(e));
    h->last_error = HYDRO_ECUDA;
  }
  return HYDRO_ECUDA;
}

#define BCK(h, call)                               \
  do {                                             \
    cudaError_t e_ = (call);                       \
    if (e_ != cudaSuccess) return bcuda(h, e_);    \
  } while (0)

size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

// build and upload the launch tables of a schedule
int build_tables(hydro_batch_t h, const Schedule& s) {
  const int n = h->ngrids;
  std::vector<int> order(n);
  for (int i = 0; i < n; ++i) order[i] = i;
  if (s.order == 1)
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
      return h->desc[a].G.nreal > h->desc[b].G.nreal;
    });
  std::vector<int> tab((size_t)kLaunchKinds * (n + 1) + n);
  if (!build_launch_tables(h->desc.data(), order.data(), n, s.bs, tab.data(), h->blocks))
    return bfail(h, HYDRO_EINVAL);
  BCK(h, cudaMemcpy(h->d_tables, tab.data(), tab.size() * sizeof(int), cudaMemcpyHostToDevice));
  h->sched = s;
  return HYDRO_OK;
}

BatchLaunch launch_of(hydro_batch_t h, int kind) {
  BatchLaunch L;
  L.descs = h->d_desc;
  L.prefix = h->d_tables + (size_t)kind * (h->ngrids + 1);
  L.order = h->d_tables + (size_t)kLaunchKinds * (h->ngrids + 1);
  L.ngrids = h->ngrids;
  return L;
}

// one step of every grid; dt of step `step` into d_dt[step][grid]
int enqueue_step(hydro_batch_t h, double cfl, int step) {
  cudaStream_t st = h->stream;
  const int bs = h->sched.bs;
  BCK(h, batch_prims(launch_of(h, 0), h->precision, bs, h->blocks[0], st));
  BCK(h, batch_set_dt(h->d_desc, h->ngrids, cfl, h->d_dt + (size_t)step * h->ngrids, st));
  for (int d = 0; d < 3; ++d) {
    if (!h->axis_used[d]) continue;
    for (int s = kStageSlopes; s <= kStageRiemann1; ++s) {
      const int kind = launch_kind(s, d);
      // no slope pass for PCM; the mixed PPMC kernel forms its own slopes
      if (s == kStageSlopes && (h->recon == HYDRO_RECON_PCM || h->precision == HYDRO_MIXED))
        continue;
      if (s == kStagePpmc && d > 0 &&
          (h->precision == HYDRO_MIXED || h->recon == HYDRO_RECON_PPMC)) {  // by segments along y, z
        const int k = ppmc_seg_kind(d);
        BCK(h, h->precision == HYDRO_MIXED
                   ? batch_ppmc_mixed_seg(launch_of(h, k), d, h->blocks[k], st)
                   : batch_ppmc_fp64_seg(launch_of(h, k), d, h->blocks[k], st));
        continue;
      }
      BCK(h, batch_stage(launch_of(h, kind), h->precision, h->recon, h->solver, s, d, bs,
                         h->blocks[kind], st));
    }
  }
  for (int d = 0; d < 3; ++d) {
    if (!h->axis_used[d]) continue;
    if (d > 0 && h->precision == HYDRO_FP64 && h->solver == HYDRO_RIEMANN_EXACT) {  // by segments
      const int kind = riemann2_seg_kind(d);
      BCK(h, batch_riemann2_fp64_seg(launch_of(h, kind), d, h->blocks[kind], st));
      continue;
    }
    const int kind = launch_kind(kStageRiemann2, d);
    BCK(h, batch_stage(launch_of(h, kind), h->precision, h->recon, h->solver, kStageRiemann2, d,
                       bs, h->blocks[kind], st));
  }
  BCK(h, batch_update(launch_of(h, 1), h->precision, bs, h->blocks[1], st));
  return HYDRO_OK;
}

int ensure_dt(hydro_batch_t h, int nsteps) {
  if (nsteps <= h->dt_cap) return HYDRO_OK;
  if (h->d_dt) cudaFree(h->d_dt);
  h->d_dt = nullptr;
  cudaError_t e = cudaMalloc(&h->d_dt, (size_t)nsteps * h->ngrids * sizeof(double));
  if (e != cudaSuccess) {
    cudaGetLastError();
    h->dt_cap = 0;
    return bfail(h, HYDRO_ENOMEM);
  }
  h->dt_cap = nsteps;
  return HYDRO_OK;
}

int read_flags(hydro_batch_t h, int* any) {
  std::vector<double> r((size_t)h->ngrids * 8);
  BCK(h, cudaMemcpyAsync(r.data(), h->recs, r.size() * sizeof(double), cudaMemcpyDeviceToHost,
                         h->stream));
  BCK(h, cudaStreamSynchronize(h->stream));
  int f = 0;
  for (int i = 0; i < h->ngrids; ++i) {
    int fi;
    memcpy(&fi, &r[(size_t)i * 8 + 4], sizeof(int));
    f |= fi;
  }
  *any = f;
  return HYDRO_OK;
}

// ---- autotuner cache -------------------------------------------------------
std::string cache_path() {
  const char* p = getenv("HYDRO_TUNE_CACHE");
  if (p && *p) return p;
  const char* home = getenv("HOME");
  return std::string(home ? home : "/tmp") + "/.cache/hydro_gb300_batch_tune.txt";
}

std::string shape_key(hydro_batch_t h) {
  // FNV-1a over the grid sizes (and a non-default reconstruction), plus
  // precision and device name
  unsigned long long x = 1469598103934665603ULL;
  auto mix = [&](long long v) {
    for (int b = 0; b < 8; ++b) {
      x ^= (unsigned long long)((v >> (8 * b)) & 0xff);
      x *= 1099511628211ULL;
    }
  };
  mix(h->ngrids);
  for (const GridDesc& g : h->desc)
    for (int d = 0; d < 3; ++d) mix(g.G.n[d]);
  if (h->recon != HYDRO_RECON_PPMC) mix(1000 + h->recon);
  if (h->solver != HYDRO_RIEMANN_EXACT) mix(2000 + h->solver);
  cudaDeviceProp prop;
  char name[64] = "unknown";
  if (cudaGetDeviceProperties(&prop, h->device) == cudaSuccess) {
    snprintf(name, sizeof(name), "%s", prop.name);
    for (char* c = name; *c; ++c)
      if (*c == ' ') *c = '_';
  }
  char key[160];
  snprintf(key, sizeof(key), "%016llx_p%d_%s", x, h->precision, name);
  return key;
}

bool cache_lookup(const std::string& key, Schedule* s) {
  FILE* f = fopen(cache_path().c_str(), "r");
  if (!f) return false;
  char k[200];
  int bs, order;
  float ms;
  bool found = false;
  while (fscanf(f, "%199s %d %d %f", k, &bs, &order, &ms) == 4) {
    if (key == k && (bs == 128 || bs == 256) && (order == 0 || order == 1)) {
      s->bs = bs;
      s->order = order;
      found = true;
    }
  }
  fclose(f);
  return found;
}

void cache_store(const std::string& key, const Schedule& s, float ms) {
  const std::string path = cache_path();
  // create the parent directories (the cache is optional: failures are ignored)
  for (size_t pos = path.find('/', 1); pos != std::string::npos; pos = path.find('/', pos + 1))
    mkdir(path.substr(0, pos).c_str(), 0755);
  FILE* f = fopen(path.c_str(), "a");
  if (!f) return;
  fprintf(f, "%s %d %d %.4f\n", key.c_str(), s.bs, s.order, ms);
  fclose(f);
}

}  // namespace

extern "C" {

int hydro_batch_init(hydro_batch_t* out, int ngrids, const int* dims, const double* dx,
                     const double* gamma, const int* bc) {
  if (!out) return HYDRO_EINVAL;
  *out = nullptr;
  if (ngrids < 1 || !dims || !dx || !gamma || !bc) return HYDRO_EINVAL;
  for (int i = 0; i < ngrids; ++i) {
    if (!(dx[i] > 0.0) || !(gamma[i] > 1.0)) return HYDRO_EINVAL;
    for (int d = 0; d < 3; ++d) {
      const int n = dims[3 * i + d];
      const int b0 = bc[6 * i + 2 * d], b1 = bc[6 * i + 2 * d + 1];
      if (n < 1 || (n > 1 && n < kNG)) return HYDRO_EINVAL;
      if (n > 1 && (b0 < 0 || b0 > 3 || b1 < 0 || b1 > 3)) return HYDRO_EINVAL;
      if (n > 1 && ((b0 == HYDRO_BC_PERIODIC) != (b1 == HYDRO_BC_PERIODIC))) return HYDRO_EINVAL;
    }
    if (padded_cells(dims + 3 * i) >= (1ll << 31)) return HYDRO_EINVAL;  // 32-bit indices
  }
  hydro_batch_t h = new (std::nothrow) hydro_batch_s();
  if (!h) return HYDRO_ENOMEM;
  h->ngrids = ngrids;
  if (cudaGetDevice(&h->device) != cudaSuccess) {
    delete h;
    return HYDRO_ECUDA;
  }
  h->desc.resize(ngrids);
  h->have_state.assign(ngrids, 0);
  // geometry and slab layout of every grid
  std::vector<size_t> off(ngrids);
  size_t total = align_up((size_t)ngrids * 8 * sizeof(double), 256);  // records first
  for (int i = 0; i < ngrids; ++i) {
    GridDesc& g = h->desc[i];
    memset(&g, 0, sizeof(g));
    Geom& G = g.G;
    for (int d = 0; d < 3; ++d) {
      G.n[d] = dims[3 * i + d];
      G.g[d] = G.n[d] > 1 ? kNG : 0;
      G.N[d] = G.n[d] + 2 * G.g[d];
      if (G.n[d] > 1) h->axis_used[d] = true;
    }
    G.s[0] = 1;
    G.s[1] = G.N[0];
    G.s[2] = (long long)G.N[0] * G.N[1];
    G.ps = (long long)align_up((size_t)G.N[0] * G.N[1] * G.N[2], 32);
    G.nreal = (long long)G.n[0] * G.n[1] * G.n[2];
    geom_divisors(G);
    G.dx = dx[i];
    for (int f = 0; f < 6; ++f) g.bc.type[f] = (G.n[f / 2] > 1) ? bc[6 * i + f] : HYDRO_BC_PERIODIC;
    fill_desc(g, gamma[i]);
    int nact = 0;
    for (int d = 0; d < 3; ++d) nact += G.n[d] > 1 ? 1 : 0;
    off[i] = total;
    total += align_up((size_t)G.nreal * 5 * sizeof(double), 256) +
             (size_t)G.ps * sizeof(double) * (8 + 5 + 15 * (size_t)nact);
  }
  cudaError_t e = cudaMalloc(&h->slab, total);
  if (e != cudaSuccess) {
    cudaGetLastError();
    delete h;
    return HYDRO_ENOMEM;
  }
  char* base = static_cast<char*>(h->slab);
  h->recs = reinterpret_cast<double*>(base);
  for (int i = 0; i < ngrids; ++i) {
    GridDesc& g = h->desc[i];
    const Geom& G = g.G;
    const size_t plane = (size_t)G.ps * sizeof(double);
    char* p = base + off[i];
    Bufs& B = g.B;
    B.u = reinterpret_cast<double*>(p);
    p += align_up((size_t)G.nreal * 5 * sizeof(double), 256);
    B.W = reinterpret_cast<double*>(p);
    p += 8 * plane;
    B.S = reinterpret_cast<double*>(p);
    p += 5 * plane;
    for (int d = 0; d < 3; ++d) {
      B.UL[d] = B.UR[d] = B.F1[d] = nullptr;
      if (G.n[d] <= 1) continue;
      B.UL[d] = reinterpret_cast<double*>(p);
      p += 5 * plane;
      B.UR[d] = reinterpret_cast<double*>(p);
      p += 5 * plane;
      B.F1[d] = reinterpret_cast<double*>(p);
      p += 5 * plane;
    }
    B.rec = h->recs + (size_t)i * 8;
  }
  e = cudaMalloc(&h->d_desc, sizeof(GridDesc) * ngrids);
  if (e == cudaSuccess)
    e = cudaMalloc(&h->d_tables, sizeof(int) * ((size_t)kLaunchKinds * (ngrids + 1) + ngrids));
  if (e == cudaSuccess) e = cudaMemset(h->slab, 0, total);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking);
  if (e == cudaSuccess) {
    h->own_stream = true;
    e = cudaMemcpy(h->d_desc, h->desc.data(), sizeof(GridDesc) * ngrids, cudaMemcpyHostToDevice);
  }
  if (e != cudaSuccess || build_tables(h, Schedule()) != HYDRO_OK) {
    hydro_batch_free(h);
    return e == cudaErrorMemoryAllocation ? HYDRO_ENOMEM : HYDRO_ECUDA;
  }
  *out = h;
  return HYDRO_OK;
}

int hydro_batch_set_inflow(hydro_batch_t h, int grid, int face, const double prim[5]) {
  if (!h) return HYDRO_EINVAL;
  h->last_error = HYDRO_OK;
  if (grid < 0 || grid >= h->ngrids || face < 0 || face > 5 || !prim) return bfail(h, HYDRO_EINVAL);
  if (!(prim[0] > 0.0) || !(prim[4] >= 0.0)) return bfail(h, HYDRO_EINVAL);
  const double gm1 = (double)h->desc[grid].gd.gm1;
  double* U = h->desc[grid].bc.inflow[face];
  for (int q = 0; q < 5; ++q) h->desc[grid].bc.prim[face][q] = prim[q];
  U[0] = prim[0];
  U[1] = prim[0] * prim[1];
  U[2] = prim[0] * prim[2];
  U[3] = prim[0] * prim[3];
  U[4] = prim[4] / gm1 + 0.5 * prim[0] * (prim[1] * prim[1] + prim[2] * prim[2] + prim[3] * prim[3]);
  BCK(h, cudaMemcpy(&h->d_desc[grid].bc, &h->desc[grid].bc, sizeof(BcDesc), cudaMemcpyHostToDevice));
  return HYDRO_OK;
}

int hydro_batch_set_precision(hydro_batch_t h, int mode) {
  if (!h) return HYDRO_EINVAL;
  h->last_error = HYDRO_OK;
  if (mode != HYDRO_FP64 && mode != HYDRO_MIXED) return bfail(h, HYDRO_EINVAL);
  if (mode == HYDRO_MIXED && (h->recon != HYDRO_RECON_PPMC || h->solver != HYDRO_RIEMANN_EXACT))
    return bfail(h, HYDRO_EINVAL);
  if (mode != h->precision) h->tuned = false;
  h->precision = mode;
  return HYDRO_OK;
}

int hydro_batch_set_reconstruction(hydro_batch_t h, int recon) {
  if (!h) return HYDRO_EINVAL;
  h->last_error = HYDRO_OK;
  if (recon < HYDRO_RECON_PPMC || recon > HYDRO_RECON_PCM) return bfail(h, HYDRO_EINVAL);
  if (recon != HYDRO_RECON_PPMC && h->precision == HYDRO_MIXED) return bfail(h, HYDRO_EINVAL);
  if (recon != h->recon) h->tuned = false;
  h->recon = recon;
  return HYDRO_OK;
}

int hydro_batch_set_riemann_solver(hydro_batch_t h, int solver) {
  if (!h) return HYDRO_EINVAL;
  h->last_error = HYDRO_OK;
  if (solver != HYDRO_RIEMANN_EXACT && solver != HYDRO_RIEMANN_ROE) return bfail(h, HYDRO_EINVAL);
  if (solver != HYDRO_RIEMANN_EXACT && h->precision == HYDRO_MIXED) return bfail(h, HYDRO_EINVAL);
  if (solver == HYDRO_RIEMANN_ROE && !h->eta_buf) {
    if (cudaSetDevice(h->device) != cudaSuccess) return bfail(h, HYDRO_ECUDA);
    size_t planes = 0;
    for (const GridDesc& g : h->desc)
      for (int d = 0; d < 3; ++d)
        if (g.G.n[d] > 1) planes += (size_t)g.G.ps;
    cudaError_t e = cudaMalloc(&h->eta_buf, planes * sizeof(double));
    if (e != cudaSuccess) {
      cudaGetLastError();
      h->eta_buf = nullptr;
      return bfail(h, HYDRO_ENOMEM);
    }
    double* p = h->eta_buf;
    for (GridDesc& g : h->desc)
      for (int d = 0; d < 3; ++d) {
        g.B.eta[d] = nullptr;
        if (g.G.n[d] <= 1) continue;
        g.B.eta[d] = p;
        p += g.G.ps;
      }
    e = cudaMemcpy(h->d_desc, h->desc.data(), sizeof(GridDesc) * h->ngrids,
                   cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return bcuda(h, e);
  }
  if (solver != h->solver) h->tuned = false;
  h->solver = solver;
  return HYDRO_OK;
}

int hydro_batch_set_stream(hydro_batch_t h, void* stream) {
  if (!h) return HYDRO_EINVAL;
  h->last_error = HYDRO_OK;
  if (!stream) return bfail(h, HYDRO_EINVAL);  // graph capture needs a non-default stream
  if (h->own_stream) cudaStreamDestroy(h->stream);
  h->own_stream = false;
  h->stream = static_cast<cudaStream_t>(stream);
  if (h->gexec) cudaGraphExecDestroy(h->gexec);
  h->gexec = nullptr;
  return HYDRO_OK;
}

int hydro_batch_set_state(hydro_batch_t h, int grid, const double* u, int on_device) {
  if (!h) return HYDRO_EINVAL;
  h->last_error = HYDRO_OK;
  if (grid < 0 || grid >= h->ngrids || !u) return bfail(h, HYDRO_EINVAL);
  const GridDesc& g = h->desc[grid];
  BCK(h, cudaMemcpyAsync(g.B.u, u, (size_t)g.G.nreal * 5 * sizeof(double),
                         on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, h->stream));
  BCK(h, cudaStreamSynchronize(h->stream));
  h->have_state[grid] = 1;
  return HYDRO_OK;
}

int hydro_batch_get_state(hydro_batch_t h, int grid, double* u, int on_device) {
  if (!h) return HYDRO_EINVAL;
  h->last_error = HYDRO_OK;
  if (grid < 0 || grid >= h->ngrids || !u) return bfail(h, HYDRO_EINVAL);
  if (!h->have_state[grid]) return bfail(h, HYDRO_ENOSTATE);
  const GridDesc& g = h->desc[grid];
  BCK(h, cudaMemcpyAsync(u, g.B.u, (size_t)g.G.nreal * 5 * sizeof(double),
                         on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, h->stream));
  BCK(h, cudaStreamSynchronize(h->stream));
  return HYDRO_OK;
}

// Capture (when the call shape changed) and launch the graph of nsteps steps.
static int launch_steps(hydro_batch_t h, double cfl, int nsteps) {
  if (nsteps < 1 || !(cfl > 0.0)) return bfail(h, HYDRO_EINVAL);
  for (int i = 0; i < h->ngrids; ++i)
    if (!h->have_state[i]) return bfail(h, HYDRO_ENOSTATE);
  int rc = ensure_dt(h, nsteps);
  if (rc) return rc;
  const bool same = h->gexec && h->g_nsteps == nsteps && h->g_cfl == cfl &&
                    h->g_precision == h->precision && h->g_recon == h->recon &&
                    h->g_solver == h->solver &&
                    h->g_sched.bs == h->sched.bs && h->g_sched.order == h->sched.order;
  if (!same) {
    if (h->gexec) cudaGraphExecDestroy(h->gexec);
    h->gexec = nullptr;
    cudaGraph_t graph = nullptr;
    BCK(h, cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal));
    int erc = HYDRO_OK;
    cudaError_t e = cudaMemsetAsync(h->recs, 0, (size_t)h->ngrids * 8 * sizeof(double), h->stream);
    if (e != cudaSuccess) erc = bcuda(h, e);
    for (int s = 0; s < nsteps && erc == HYDRO_OK; ++s) erc = enqueue_step(h, cfl, s);
    e = cudaStreamEndCapture(h->stream, &graph);
    if (erc != HYDRO_OK) {
      if (graph) cudaGraphDestroy(graph);
      return erc;
    }
    if (e != cudaSuccess) return bcuda(h, e);
    e = cudaGraphInstantiate(&h->gexec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) {
      h->gexec = nullptr;
      return bcuda(h, e);
    }
    h->g_nsteps = nsteps;
    h->g_cfl = cfl;
    h->g_precision = h->precision;
    h->g_recon = h->recon;
    h->g_solver = h->solver;
    h->g_sched = h->sched;
  }
  BCK(h, cudaGraphLaunch(h->gexec, h->stream));
  return HYDRO_OK;
}

// the status word of the last graph launch (waits for the stream)
static int status_of(hydro_batch_t h) {
  int flags = 0;
  const int rc = read_flags(h, &flags);
  if (rc) return rc;
  if (flags & kFlagNonPhys) return bfail(h, HYDRO_ENONPHYS);
  if (flags & kFlagNewton) return bfail(h, HYDRO_ENEWTON);
  return HYDRO_OK;
}

int hydro_batch_step(hydro_batch_t h, double cfl, int nsteps, double* dt_out) {
  if (!h) return HYDRO_EINVAL;
  h->last_error = HYDRO_OK;
  int rc = launch_steps(h, cfl, nsteps);
  if (rc) return rc;
  if (dt_out)
    BCK(h, cudaMemcpyAsync(dt_out, h->d_dt, (size_t)nsteps * h->ngrids * sizeof(double),
                           cudaMemcpyDeviceToHost, h->stream));
  return status_of(h);
}

int hydro_batch_step_async(hydro_batch_t h, double cfl, int nsteps) {
  if (!h) return HYDRO_EINVAL;
  h->last_error = HYDRO_OK;
  return launch_steps(h, cfl, nsteps);
}

int hydro_batch_sync(hydro_batch_t h) {
  if (!h) return HYDRO_EINVAL;
  h->last_error = HYDRO_OK;
  return status_of(h);
}

int hydro_batch_set_state_async(hydro_batch_t h, int grid, const double* u, int on_device) {
  if (!h) return HYDRO_EINVAL;
  h->last_error = HYDRO_OK;
  if (grid < 0 || grid >= h->ngrids || !u) return bfail(h, HYDRO_EINVAL);
  const GridDesc& g = h->desc[grid];
  BCK(h, cudaMemcpyAsync(g.B.u, u, (size_t)g.G.nreal * 5 * sizeof(double),
                         on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, h->stream));
  h->have_state[grid] = 1;
  return HYDRO_OK;
}

int hydro_batch_get_state_async(hydro_batch_t h, int grid, double* u, int on_device) {
  if (!h) return HYDRO_EINVAL;
  h->last_error = HYDRO_OK;
  if (grid < 0 || grid >= h->ngrids || !u) return bfail(h, HYDRO_EINVAL);
  if (!h->have_state[grid]) return bfail(h, HYDRO_ENOSTATE);
  const GridDesc& g = h->desc[grid];
  BCK(h, cudaMemcpyAsync(u, g.B.u, (size_t)g.G.nreal * 5 * sizeof(double),
                         on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, h->stream));
  return HYDRO_OK;
}

int hydro_batch_autotune(hydro_batch_t h, int use_cache, int* block_size, int* order,
                         float* ms_per_step) {
  if (!h) return HYDRO_EINVAL;
  h->last_error = HYDRO_OK;
  for (int i = 0; i < h->ngrids; ++i)
    if (!h->have_state[i]) return bfail(h, HYDRO_ENOSTATE);
  const std::string key = shape_key(h);
  Schedule best;
  float best_ms = -1.f;
  bool hit = use_cache && cache_lookup(key, &best);
  if (!hit) {
    // keep the states: every candidate runs from the same state, restored after
    size_t bytes = 0;
    for (const GridDesc& g : h->desc) bytes += (size_t)g.G.nreal * 5 * sizeof(double);
    double* backup = nullptr;
    cudaError_t e = cudaMalloc(&backup, bytes);
    if (e != cudaSuccess) {
      cudaGetLastError();
      return bfail(h, HYDRO_ENOMEM);
    }
    int rc = ensure_dt(h, 1);
    if (rc) {
      cudaFree(backup);
      return rc;
    }
    size_t o = 0;
    for (const GridDesc& g : h->desc) {
      const size_t b = (size_t)g.G.nreal * 5 * sizeof(double);
      e = cudaMemcpyAsync(reinterpret_cast<char*>(backup) + o, g.B.u, b, cudaMemcpyDeviceToDevice,
                          h->stream);
      o += b;
    }
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    const Schedule cands[4] = {{256, 0}, {256, 1}, {128, 0}, {128, 1}};
    for (int c = 0; c < 4 && rc == HYDRO_OK; ++c) {
      rc = build_tables(h, cands[c]);
      if (rc) break;
      // one untimed step, then two timed ones (zeroed records each step)
      float ms = 0.f;
      for (int rep = 0; rep < 3 && rc == HYDRO_OK; ++rep) {
        cudaMemsetAsync(h->recs, 0, (size_t)h->ngrids * 8 * sizeof(double), h->stream);
        if (rep == 1) cudaEventRecord(e0, h->stream);
        rc = enqueue_step(h, 0.3, 0);
      }
      cudaEventRecord(e1, h->stream);
      cudaEventSynchronize(e1);
      cudaEventElapsedTime(&ms, e0, e1);
      h->tune_ms[c] = ms / 2.f;
      if (best_ms < 0.f || ms / 2.f < best_ms) {
        best_ms = ms / 2.f;
        best = cands[c];
      }
      o = 0;  // restore the states
      for (const GridDesc& g : h->desc) {
        const size_t b = (size_t)g.G.nreal * 5 * sizeof(double);
        cudaMemcpyAsync(g.B.u, reinterpret_cast<char*>(backup) + o, b, cudaMemcpyDeviceToDevice,
                        h->stream);
        o += b;
      }
    }
    cudaStreamSynchronize(h->stream);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(backup);
    if (rc) return rc;
    e = cudaGetLastError();
    if (e != cudaSuccess) return bcuda(h, e);
    cache_store(key, best, best_ms);
  }
  const int rc = build_tables(h, best);
  if (rc) return rc;
  h->tuned = true;
  if (block_size) *block_size = best.bs;
  if (order) *order = best.order;
  if (ms_per_step) *ms_per_step = best_ms;
  return HYDRO_OK;
}

int hydro_batch_last_error(hydro_batch_t h) { return h ? h->last_error : HYDRO_EINVAL; }

const char* hydro_batch_cuda_error_string(hydro_batch_t h) { return h ? h->cuda_err : ""; }

void hydro_batch_free(hydro_batch_t h) {
  if (!h) return;
  if (h->stream) cudaStreamSynchronize(h->stream);
  if (h->gexec) cudaGraphExecDestroy(h->gexec);
  if (h->d_dt) cudaFree(h->d_dt);
  if (h->d_tables) cudaFree(h->d_tables);
  if (h->d_desc) cudaFree(h->d_desc);
  if (h->slab) cudaFree(h->slab);
  if (h->eta_buf) cudaFree(h->eta_buf);
  if (h->own_stream && h->stream) cudaStreamDestroy(h->stream);
  delete h;
}

}  // extern "C"
