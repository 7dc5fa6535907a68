// Tensor-core (tcgen05) projection of the FP32 coarse-operator build.
#pragma once

#include "coarse.cuh"

namespace hdcr {

constexpr int TC_MAX_SPLIT = 16;  // CTAs sharing one block's contraction

// Operands of one projection A[a][leg] = X_a^dag Y_a, for every block a:
//   field = 1: X, Y are nvec fields in the psi[x4][c][s] layout and kappa runs
//              over the block's 4d sites (x fastest) times the 12*Ls components;
//   field = 0: X, Y are [v][a][K] arrays, contiguous per vector and block.
struct TcSrc {
  const cpx<float>* X;
  const cpx<float>* Y;
  long long K;  // kappa per block
  int field;
  Geom g;
  BlockGeom bg;
};

// A[a][leg][j][k] = sum_kappa conj(X_j) Y_k for every block; *err is set when a
// wait on the tensor cores ran out of time.  nvec <= 64.  With part non-null
// (room for TC_MAX_SPLIT * Vc * nvec^2 complex) long contractions are
// split over several CTAs per block and summed by a second kernel.  npass = 3
// keeps the products at FP32 accuracy (TF32 hi/lo splits); npass = 1 takes the
// TF32-rounded operands once (relative error of a product about 2^-11).
int tc_project_splits(const TcSrc& S);
int launch_tc_project(const TcSrc& S, cpx<float>* A, int nvec, int leg, cpx<float>* part, int* err, int npass,
                      cudaStream_t st);

}  // namespace hdcr
