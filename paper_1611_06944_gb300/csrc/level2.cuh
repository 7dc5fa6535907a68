// The third level of the coarse solve (level2.cu).
#pragma once

#include "coarse.cuh"

namespace hdcr {

struct Level2;
void level2_free(Level2* l);
// builds (or rebuilds) the third level of co from nvec2/2 coarse noise vectors (C128, device)
int level2_build(hdcr_coarse* co, const hdcr_level2_params* p, const void* noise, cudaStream_t st);
// x = A^{-1} b by flexible GCR preconditioned with the level-2 V-cycle (coarse vectors in R)
template <typename R>
int level2_solve(const hdcr_coarse* co, const cpx<R>* b, cpx<R>* x, double tol, int max_iter, int* iters,
                 cudaStream_t st);

}  // namespace hdcr
