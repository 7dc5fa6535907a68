// Conjugate residual (Section 3) on the fine operator, with all scalars kept
// on the device so that fixed-length runs (smoother, subspace smoothing) need
// no host synchronisation.
#pragma once

#include "blas.cuh"

namespace hdcr {

template <typename R>
struct FineOp {
  Geom g;
  double M5, mf;
  const cpx<R>* U;
  long long n() const { return g.V5 * 12; }  // complex entries of one field
};

// device scalars of one CR run
struct CRDev {
  double gamma;      // <r, H r>
  double gamma_new;  // <r', H r'>
  double ApAp;       // |Ap|^2
  double rr;         // |r|^2
  double bb;         // |b|^2
  double tr;         // |b - H x|^2 (true residual)
  double pad[2];
};

template <typename R>
struct CRWork {
  cpx<R>* r;
  cpx<R>* p;
  cpx<R>* Ar;
  cpx<R>* Ap;
  RedBuffers rb;  // rb.scal holds one CRDev
  CRDev* dev() const { return reinterpret_cast<CRDev*>(rb.scal); }
};

template <typename R>
int crwork_alloc(CRWork<R>* w, long long n);
template <typename R>
void crwork_free(CRWork<R>* w);

struct CRConfig {
  double tol = 1e-10;   // relative residual target (convergence mode)
  int max_iter = 10000;
  int fixed_iters = -1; // >= 0: run exactly this many iterations, no test, no host sync
  bool x_zero = false;  // x is zero on entry: skip the initial H x
  int check_every = 4;  // host convergence test every k iterations
};

struct CRResult {
  int iters = 0;
  int matvecs = 0;
  bool converged = false;
  double rel_resid = -1.0;  // recursive |r|/|b| at the last check
};

template <typename R>
int cr_run(const FineOp<R>& H, const cpx<R>* b, cpx<R>* x, CRWork<R>& w, const CRConfig& cfg,
           CRResult* res, cudaStream_t st);

// |b - H x|^2 into *result (device double), using tmp as workspace.
template <typename R>
int true_residual2(const FineOp<R>& H, const cpx<R>* b, const cpx<R>* x, cpx<R>* tmp, RedScratch rs,
                   double* result, cudaStream_t st);

// out = H in, and Re <in, out> into *result (device double).
template <typename R>
int launch_g5dwf_dot(const FineOp<R>& H, const cpx<R>* in, cpx<R>* out, RedScratch rs, double* result,
                     cudaStream_t st);

double* pinned_ring();  // per host thread, 1024 doubles of pinned memory
constexpr int PINNED_RING = 1024;

}  // namespace hdcr
