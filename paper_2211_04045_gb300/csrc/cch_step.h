// cch_step.h -- host launchers of the per-iteration kernels (cch_step.cu).
#pragma once
#include "cch_host.h"

namespace cch {
int coop_grid(int threads, int which);
void step_init(Runtime& R, cudaStream_t st, int mode);
void output_scene(Runtime& R, int s, cudaStream_t st);
void set_any_search(Runtime& R, cudaStream_t st);
cudaError_t iteration(Runtime& R, int cur, cudaStream_t st);
void output(Runtime& R, cudaStream_t st);
void reset_accept(Runtime& R, cudaStream_t st);
// pre-passes (cch_prepass.cu)
void normal_flow(Runtime& R, const double* x, double* y, double* tmp, double sb, double alpha, int iters,
                 cudaStream_t st);
void friction(Runtime& R, double mu, double reach, double sep, double* out, cudaStream_t st);
}  // namespace cch
