// hydro_run.h -- launchers of the device-driven run (hydro_advance): a CUDA
// graph whose conditional WHILE node repeats one step.  A single grid's step
// record has room for 32 doubles; the run uses slots [8] end time, [9] steps
// left, [10] steps taken in the current graph launch.
#pragma once
#include <cuda_runtime.h>

#include "hydro_internal.h"

namespace hydro {

// The step's dt: the CFL dt cut back to t_end - t when t + dt >= t_end (then
// the time becomes t_end exactly, else t + dt).
cudaError_t set_dt_to_end(const Geom& G, const Bufs& B, double cfl, cudaStream_t st);
// Loop condition before the first step (t < t_end and a step left) ...
cudaError_t run_begin(double* rec, cudaGraphConditionalHandle cond, cudaStream_t st);
// ... and after each step (also: no status flag, fewer than `chunk` steps taken
// in this graph launch).
cudaError_t run_next(double* rec, cudaGraphConditionalHandle cond, double chunk, cudaStream_t st);

}  // namespace hydro
