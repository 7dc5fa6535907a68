// The shared-memory (TMA-staged) FP32 operator of dwf_tma.cu, as extra
// variants of the FP32 autotuner in dwf_x2.cu.
#pragma once

#include "dwf_x2.cuh"
#include "reduce.cuh"

namespace hdcr {

constexpr int TMA_SHAPES = 1;  // column shapes (Lx, TY, TZ): (16, 4, 2)

// whether column shape ``shape`` applies to the lattice and the fields' alignment
bool tma_shape_fits(int shape, const Geom& g, const void* in, const void* out);
// H in for nrhs fields with epilogue epi (X2_STORE, X2_DOT with rs/result, X2_CHEB with ch)
int launch_g5dwf_tma(int shape, int epi, const Geom& g, float diag, float mf, const cpx<float>* U,
                     const cpx<float>* in, cpx<float>* out, int nrhs, RedScratch rs, double* result, X2Cheb ch,
                     cudaStream_t st);
// reads and clears the device flag a TMA-stencil CTA sets when a copy did not arrive in time
int tma_take_timeouts(int* flag);

}  // namespace hdcr
