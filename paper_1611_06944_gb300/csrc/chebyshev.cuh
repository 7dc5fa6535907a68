// Chebyshev smoother and low-pass filter on H^2 (Section 4, Fig. 1).
#pragma once

#include <vector>

#include "krylov.cuh"

namespace hdcr {

template <typename R>
struct ChebWork {
  cpx<R>* t0 = nullptr;  // recurrence terms
  cpx<R>* t1 = nullptr;
  cpx<R>* h1 = nullptr;  // H t
  cpx<R>* h2 = nullptr;  // H^2 t
  double* n2 = nullptr;  // device scalar for rescaling
};

template <typename R>
int cheb_work_alloc(ChebWork<R>* w, long long n);
template <typename R>
void cheb_work_free(ChebWork<R>* w);

// coefficients c_0..c_order of the truncated Chebyshev series of 1/y on [lo, hi]
std::vector<double> cheb_inverse_coeffs(double lo, double hi, int order);

// out = H p(H^2) r;  adds the stencil applications made to *matvecs
template <typename R>
int cheb_smoother(const FineOp<R>& H, const cpx<R>* r, cpx<R>* out, const std::vector<double>& c, double lo,
                  double hi, ChebWork<R>& w, cudaStream_t st, int* matvecs);

// x <- T_order(t(H^2)) x / |.|, t mapping [lam_cut^2, lam_max^2] onto [-1, 1]
template <typename R>
int cheb_filter(const FineOp<R>& H, cpx<R>* x, int order, double lam_cut, double lam_max, ChebWork<R>& w,
                RedScratch rs, cudaStream_t st);

// The same filter on nrhs fields x at once (stencil launches over all of them; in
// FP32 each step's recurrence is fused into the second stencil).  work holds
// 4 * nrhs fields, n2 one device double.  The fields share one rescaling: the
// result is x scaled by a common factor, not normalised field by field.
template <typename R>
int cheb_filter_multi(const FineOp<R>& H, cpx<R>* x, int nrhs, int order, double lam_cut, double lam_max,
                      cpx<R>* work, double* n2, RedScratch rs, cudaStream_t st);

template <typename R>
void rescale_copy(const cpx<R>* in, cpx<R>* out, long long n, R s, cudaStream_t st);

}  // namespace hdcr
