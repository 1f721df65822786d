// hydro_noalloc.cu -- hydro_compute_dt_noalloc(): the CFL time-step reduction
// of a caller-held state without any device allocation.
//
// Callers that cannot call cudaMalloc -- for example code whose device memory is
// owned entirely by another allocator (a framework's caching pool that has
// already reserved the device), or a latency-critical path where an allocation,
// which can synchronize the device, is not acceptable -- still need the time
// step of a state they hold.  This variant of the library's dt reduction keeps
// its scratch (one partial maximum per thread block) in a file-scope device
// array instead of memory allocated per handle.
//
// The scratch array holds kMaxBlocks doubles (512 KiB), so a state may have at
// most kMaxBlocks * kThreads = 2^24 cells.  Every GPU that loads this library
// holds the array until the process exits.  All calls share it: calls that
// overlap on the GPU (different streams without ordering between them) race on
// it and may return each other's result.  A call writes every partial it later
// reads before reading it, so nothing has to start at zero.
//
// Host code cannot use the array's name as a device address; the first call on
// each device looks the address up with cudaGetSymbolAddress (with that device
// current) and caches it for the life of the process.  That first call should
// come before any stream capture, and the entry point must not be used across
// a cudaDeviceReset (the module, and with it the array, may move).
//
// A cell whose density is not positive, or a NaN anywhere in a cell, makes the
// result NaN (the maxima below keep a NaN once they meet one), so such a state
// cannot silently yield a dt from its other cells.
//
// Built with --fmad=false: the per-cell arithmetic is the operation order of
// the library's strict primitive kernel, so the result equals hydro_compute_dt's
// in HYDRO_FP64_STRICT bit for bit; HYDRO_FP64 forms 1/rho and 1/a by Newton
// iteration with fused multiply-adds and agrees to a few ulp.
#include <cuda_runtime.h>

#include <mutex>

#include "../../include/hydro.h"
#include "hydro_math.cuh"

namespace {

constexpr int kThreads = 256;
constexpr int kMaxBlocks = 65536;
constexpr int kMaxDevices = 64;

static __device__ __align__(256) double g_dt_partials[kMaxBlocks];

std::mutex g_mutex;
double* g_partials_addr[kMaxDevices] = {nullptr};

// maximum that keeps a NaN: once v is NaN it stays NaN, and a NaN x replaces v
__device__ __forceinline__ double max_keep_nan(double v, double x) {
  return (x > v || x != x) ? x : v;
}

// per block: max over its cells and active axes of |v_d| + a (Eq. calc_dt_3D;
// min dx/(|v_d| + a) = dx / max(|v_d| + a) exactly); NaN for a cell with
// rho <= 0 or a NaN field
__global__ void __launch_bounds__(kThreads)
k_dt_partials(const double* __restrict__ u, long long nreal, int active, double gamma, double gm1,
              double* __restrict__ partials) {
  __shared__ double warp_max[kThreads / 32];
  const long long t = (long long)blockIdx.x * kThreads + threadIdx.x;
  double v = 0.0;
  if (t < nreal) {
    const double d = u[t];
    const double vel[3] = {u[nreal + t] / d, u[2 * nreal + t] / d, u[3 * nreal + t] / d};
    // the floor keeps a NaN pressure NaN ((NaN < floor) is false)
    const double p = hydro::tmax(
        gm1 * (u[4 * nreal + t] - 0.5 * d * (vel[0] * vel[0] + vel[1] * vel[1] + vel[2] * vel[2])),
        hydro::kPFloor);
    const double a = sqrt(gamma * p / d);
#pragma unroll
    for (int k = 0; k < 3; ++k)
      if (active & (1 << k)) v = max_keep_nan(v, fabs(vel[k]) + a);
    if (!(d > 0.0)) v = __longlong_as_double(0x7ff8000000000000ll);  // quiet NaN
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = max_keep_nan(v, __shfl_xor_sync(0xffffffffu, v, o));
  if ((threadIdx.x & 31) == 0) warp_max[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x < 32) {
    v = threadIdx.x < kThreads / 32 ? warp_max[threadIdx.x] : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = max_keep_nan(v, __shfl_xor_sync(0xffffffffu, v, o));
    if (threadIdx.x == 0) partials[blockIdx.x] = v;
  }
}

// one block: maximum of the partials, then dt = cfl * (dx / max) (NaN when a
// partial is NaN)
__global__ void __launch_bounds__(1024)
k_dt_finish(const double* __restrict__ partials, int nblocks, double dx, double cfl,
            double* __restrict__ dt_out) {
  __shared__ double warp_max[32];
  double v = 0.0;
  for (int i = threadIdx.x; i < nblocks; i += 1024) v = max_keep_nan(v, partials[i]);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = max_keep_nan(v, __shfl_xor_sync(0xffffffffu, v, o));
  if ((threadIdx.x & 31) == 0) warp_max[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x < 32) {
    v = warp_max[threadIdx.x];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = max_keep_nan(v, __shfl_xor_sync(0xffffffffu, v, o));
    if (threadIdx.x == 0) dt_out[0] = cfl * (dx / v);
  }
}

// device address of the scratch array on the current device (set-up on the
// first call per device)
cudaError_t partials_address(double** out) {
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lock(g_mutex);
  if (dev >= 0 && dev < kMaxDevices && g_partials_addr[dev]) {
    *out = g_partials_addr[dev];
    return cudaSuccess;
  }
  void* ptr = nullptr;
  e = cudaGetSymbolAddress(&ptr, g_dt_partials);
  if (e != cudaSuccess) return e;
  if (dev >= 0 && dev < kMaxDevices) g_partials_addr[dev] = static_cast<double*>(ptr);
  *out = static_cast<double*>(ptr);
  return cudaSuccess;
}

}  // namespace

extern "C" int hydro_compute_dt_noalloc(const double* u, int nx, int ny, int nz, double dx,
                                        double gamma, double cfl, double* dt_out, void* stream) {
  if (!u || !dt_out || nx < 1 || ny < 1 || nz < 1 || !(dx > 0.0) || !(gamma > 1.0) || !(cfl > 0.0))
    return HYDRO_EINVAL;
  const long long nreal = (long long)nx * ny * nz;
  const long long nblocks = (nreal + kThreads - 1) / kThreads;
  if (nblocks > kMaxBlocks) return HYDRO_EINVAL;  // more than 2^24 cells
  const int active = (nx > 1 ? 1 : 0) | (ny > 1 ? 2 : 0) | (nz > 1 ? 4 : 0);
  double* partials = nullptr;
  if (partials_address(&partials) != cudaSuccess) return HYDRO_ECUDA;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  k_dt_partials<<<(unsigned)nblocks, kThreads, 0, st>>>(u, nreal, active, gamma, gamma - 1.0,
                                                        partials);
  if (cudaGetLastError() != cudaSuccess) return HYDRO_ECUDA;
  k_dt_finish<<<1, 1024, 0, st>>>(partials, (int)nblocks, dx, cfl, dt_out);
  if (cudaGetLastError() != cudaSuccess) return HYDRO_ECUDA;
  return HYDRO_OK;
}
