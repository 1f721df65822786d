// hydro_fp64_fast.cu -- the FP64 stage kernels (batched launches over one or
// many grids) with the algebraic rewrites of hydro_math.cuh (S = false),
// compiled with fused multiply-add contraction:
// every a*b+c becomes one DFMA, which both halves the instruction count of
// those expressions on GB300's FP64 pipe and rounds once instead of twice.
#include "hydro_kernels.cuh"

namespace hydro {

cudaError_t batch_stage_fp64(const BatchLaunch& L, int recon, int solver, int stage, int axis,
                             int bs, unsigned blocks, cudaStream_t st) {
  return launch_batch_stage<false>(L, recon, solver, stage, axis, bs, blocks, st);
}

cudaError_t batch_ppmc_fp64_seg(const BatchLaunch& L, int axis, unsigned blocks, cudaStream_t st) {
  if (blocks == 0) return cudaSuccess;
  if (axis == 1)
    kb_ppmc_seg<1><<<blocks, kPpmcSegThreads, 0, st>>>(L);
  else
    kb_ppmc_seg<2><<<blocks, kPpmcSegThreads, 0, st>>>(L);
  return cudaGetLastError();
}

cudaError_t batch_riemann2_fp64_seg(const BatchLaunch& L, int axis, unsigned blocks,
                                    cudaStream_t st) {
  if (blocks == 0) return cudaSuccess;
  if (axis == 1)
    kb_riemann2_seg<1><<<blocks, kPpmcSegThreads, 0, st>>>(L);
  else
    kb_riemann2_seg<2><<<blocks, kPpmcSegThreads, 0, st>>>(L);
  return cudaGetLastError();
}

}  // namespace hydro
