// Conjugate residual (Section 3) on the fine operator, with all scalars kept
// on the device so that fixed-length runs (smoother, subspace smoothing) need
// no host synchronisation.
#pragma once

#include "blas.cuh"

namespace hdcr {

// out = H in, and Re <in, out> into *result (device double).
template <typename R>
int launch_g5dwf_dot(const Geom& g, double M5, double mf, const cpx<R>* U, const cpx<R>* in,
                     cpx<R>* out, RedScratch rs, double* result, cudaStream_t st);

// The continued-fraction overlap operator (overlap.cu): its coefficients, and
// out = H_cf in (nrhs fields), with Re <in, out> into *dot when dot is set (nrhs 1).
struct CFCoef;
template <typename R>
int launch_cf(const Geom& g, double M5, const CFCoef& cf, const cpx<R>* U, const cpx<R>* in, cpx<R>* out, int nrhs,
              RedScratch rs, double* dot, cudaStream_t st);

// An operator usable by cr_run: n() complex entries per vector, apply, and
// apply with Re <in, out> reduced into a device double.
template <typename R>
struct FineOp {
  Geom g;
  double M5, mf;
  const cpx<R>* U;
  int nrhs = 1;  // fields a vector of this operator spans (one launch applies H to all)
  // set: the continued-fraction operator of Section 3 (its N components where the
  // domain-wall operator has s) instead of Gamma5 D_dwf; mf is then unused
  const CFCoef* cf = nullptr;
  long long n() const { return g.V5 * 12 * nrhs; }  // complex entries of one vector
  int apply(const cpx<R>* in, cpx<R>* out, cudaStream_t st) const {
    if (cf) return launch_cf<R>(g, M5, *cf, U, in, out, nrhs, RedScratch{nullptr, nullptr}, nullptr, st);
    return launch_g5dwf<R>(g, M5, mf, U, in, out, nrhs, st);
  }
  int apply_dot(const cpx<R>* in, cpx<R>* out, RedScratch rs, double* res, cudaStream_t st) const {
    if (cf) return launch_cf<R>(g, M5, *cf, U, in, out, 1, rs, res, st);
    return launch_g5dwf_dot<R>(g, M5, mf, U, in, out, rs, res, st);
  }
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

// A CUDA graph of check_every consecutive CR iterations (update of x and r, copy of
// |r|^2 to the host, H r with <r, H r>, update of p and H p) on fixed buffers,
// captured once on a library stream and replayed on the run's stream: in
// convergence mode the iterations between two host checks then cost one launch.
// Replays give the same bits as the eager launches (the same kernels in the same
// order).  Owned by the caller, who keeps it while the buffers it names stay the
// same (cr_run re-captures when they change) and frees it with cr_graph_free.
struct CRGraph {
  cudaGraphExec_t exec = nullptr;
  const void* key[6] = {};
  long long n = 0;
  int ck = 0;
  unsigned long long kernels = 0;  // kernels one replay launches
};
void cr_graph_free(CRGraph* g);
// the current device's stream for captures (created once, non-blocking)
int capture_stream(cudaStream_t* s);

struct CRConfig {
  double tol = 1e-10;   // relative residual target (convergence mode)
  int max_iter = 10000;
  int fixed_iters = -1; // >= 0: run exactly this many iterations, no test, no host sync
  bool x_zero = false;  // x is zero on entry: skip the initial H x
  int check_every = 4;  // host convergence test every k iterations
  CRGraph* graph = nullptr;  // convergence mode: replay the iterations from this graph
};

struct CRResult {
  int iters = 0;
  int matvecs = 0;
  bool converged = false;
  double rel_resid = -1.0;  // recursive |r|/|b| at the last check
};

double* pinned_ring();  // per host thread, 1024 doubles of pinned memory
constexpr int PINNED_RING = 1024;

// BLAS steps of CR (cr.cu), n complex entries, scalars in CRDev
template <typename R>
int launch_cr_setup_r(const cpx<R>* b, const cpx<R>* Hx, cpx<R>* r, cpx<R>* p, long long n,
                      RedScratch rs, CRDev* s, cudaStream_t st);
template <typename R>
int launch_cr_setup_ap(const cpx<R>* Ar, cpx<R>* Ap, long long n, RedScratch rs, CRDev* s, cudaStream_t st);
template <typename R>
int launch_cr_update_xr(cpx<R>* x, cpx<R>* r, const cpx<R>* p, const cpx<R>* Ap, long long n,
                        RedScratch rs, CRDev* s, cudaStream_t st);
template <typename R>
int launch_cr_update_p(const cpx<R>* r, cpx<R>* p, const cpx<R>* Ar, cpx<R>* Ap, long long n,
                       RedScratch rs, CRDev* s, cudaStream_t st);
// |b - y|^2 into *result
template <typename R>
int launch_diff_norm(const cpx<R>* b, const cpx<R>* y, long long n, RedScratch rs, double* result,
                     cudaStream_t st);

// |b - A x|^2 into *result (device double), using tmp as workspace.
template <typename R, class Op>
int true_residual2(const Op& A, const cpx<R>* b, const cpx<R>* x, cpx<R>* tmp, RedScratch rs,
                   double* result, cudaStream_t st) {
  HDCR_TRY(A.apply(x, tmp, st));
  return launch_diff_norm<R>(b, tmp, A.n(), rs, result, st);
}

// Conjugate residual on A x = b (Section 3).  In convergence mode the host
// reads |r|^2 every cfg.check_every iterations; with cfg.fixed_iters >= 0 the
// run is a fixed sequence of launches with no host synchronisation.
template <typename R, class Op>
int cr_run(const Op& A, const cpx<R>* b, cpx<R>* x, CRWork<R>& w, const CRConfig& cfg, CRResult* res,
           cudaStream_t st) {
  const long long n = A.n();
  CRDev* s = w.dev();
  RedScratch rs = w.rb.rs;
  CRResult out;
  const bool fixed = cfg.fixed_iters >= 0;
  if (!cfg.x_zero) {
    HDCR_TRY(A.apply(x, w.Ar, st));
    out.matvecs++;
  }
  HDCR_TRY(launch_cr_setup_r<R>(b, cfg.x_zero ? nullptr : w.Ar, w.r, w.p, n, rs, s, st));
  const int niter = fixed ? cfg.fixed_iters : cfg.max_iter;
  if (niter == 0) {
    if (res) *res = out;
    return HDCR_OK;
  }
  double* ring = nullptr;
  double scale2 = 0.0;
  if (!fixed) {
    ring = pinned_ring();
    if (!ring) {
      set_error("pinned host buffer unavailable");
      return HDCR_ERR_NO_MEMORY;
    }
    HDCR_CUDA_TRY(cudaMemcpyAsync(ring, &s->rr, 2 * sizeof(double), cudaMemcpyDeviceToHost, st));
    HDCR_CUDA_TRY(cudaStreamSynchronize(st));
    scale2 = ring[1] > 0.0 ? ring[1] : ring[0];  // |b|^2, or |r0|^2 when b = 0
    if (!(scale2 == scale2) || scale2 > 1e300) {
      set_error("CR: non-finite right-hand side or initial residual");
      return HDCR_ERR_NONFINITE;
    }
    if (scale2 == 0.0 || ring[0] <= cfg.tol * cfg.tol * scale2) {
      out.converged = true;
      out.rel_resid = scale2 > 0 ? sqrt(ring[0] / scale2) : 0.0;
      if (res) *res = out;
      return HDCR_OK;
    }
  }
  HDCR_TRY(A.apply_dot(w.r, w.Ar, rs, &s->gamma, st));
  out.matvecs++;
  HDCR_TRY(launch_cr_setup_ap<R>(w.Ar, w.Ap, n, rs, s, st));
  const int ck = cfg.check_every > 0 ? (cfg.check_every < PINNED_RING ? cfg.check_every : PINNED_RING) : 1;
  int k0 = 0;  // iterations done by graph replays
  if (!fixed && cfg.graph) {
    CRGraph* gr = cfg.graph;
    const void* key[6] = {x, w.r, w.p, w.Ar, w.Ap, ring};
    bool same = gr->exec && gr->n == n && gr->ck == ck;
    for (int i = 0; i < 6 && same; ++i) same = gr->key[i] == key[i];
    if (!same) {
      cr_graph_free(gr);
      cudaStream_t cs;
      HDCR_TRY(capture_stream(&cs));
      const unsigned long long before = launches_so_far();
      HDCR_CUDA_TRY(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
      int cap = HDCR_OK;
      for (int i = 0; i < ck && cap == HDCR_OK; ++i) {
        cap = launch_cr_update_xr<R>(x, w.r, w.p, w.Ap, n, rs, s, cs);
        if (cap == HDCR_OK && cudaMemcpyAsync(ring + i, &s->rr, sizeof(double), cudaMemcpyDeviceToHost, cs) !=
                                  cudaSuccess)
          cap = HDCR_ERR_CUDA;
        if (cap == HDCR_OK) cap = A.apply_dot(w.r, w.Ar, rs, &s->gamma_new, cs);
        if (cap == HDCR_OK) cap = launch_cr_update_p<R>(w.r, w.p, w.Ar, w.Ap, n, rs, s, cs);
      }
      cudaGraph_t graph = nullptr;
      const cudaError_t ee = cudaStreamEndCapture(cs, &graph);
      if (cap == HDCR_OK && ee == cudaSuccess) {
        if (cudaGraphInstantiate(&gr->exec, graph, 0) != cudaSuccess) gr->exec = nullptr;
      }
      if (graph) cudaGraphDestroy(graph);
      cudaGetLastError();
      gr->kernels = launches_so_far() - before;
      uncount_launches(gr->kernels);  // captured, not launched
      gr->n = n;
      gr->ck = ck;
      for (int i = 0; i < 6; ++i) gr->key[i] = key[i];
    }
    // whole chunks from the graph while they fit under niter; the rest runs eagerly below
    while (gr->exec && k0 + ck <= niter) {
      HDCR_CUDA_TRY(cudaGraphLaunch(gr->exec, st));
      count_launches(gr->kernels);
      k0 += ck;
      out.iters = k0;
      out.matvecs += ck;
      HDCR_CUDA_TRY(cudaStreamSynchronize(st));
      for (int i = 0; i < ck; ++i) {
        const double rr = ring[i];
        if (!(rr == rr) || rr > 1e300) {
          set_error("CR: non-finite residual at iteration %d", k0 - ck + i + 1);
          if (res) *res = out;
          return HDCR_ERR_NONFINITE;
        }
        out.rel_resid = sqrt(rr / scale2);
        if (rr <= cfg.tol * cfg.tol * scale2) {
          out.converged = true;
          break;
        }
      }
      if (out.converged) {
        if (res) *res = out;
        return HDCR_OK;
      }
    }
  }
  int pending = 0;
  for (int k = k0; k < niter; ++k) {
    HDCR_TRY(launch_cr_update_xr<R>(x, w.r, w.p, w.Ap, n, rs, s, st));
    out.iters = k + 1;
    if (!fixed) {
      HDCR_CUDA_TRY(cudaMemcpyAsync(ring + pending, &s->rr, sizeof(double), cudaMemcpyDeviceToHost, st));
      ++pending;
      if (pending == ck || k == niter - 1) {
        HDCR_CUDA_TRY(cudaStreamSynchronize(st));
        for (int i = 0; i < pending; ++i) {
          const double rr = ring[i];
          if (!(rr == rr) || rr > 1e300) {
            set_error("CR: non-finite residual at iteration %d", k + 2 - pending + i);
            if (res) *res = out;
            return HDCR_ERR_NONFINITE;
          }
          out.rel_resid = sqrt(rr / scale2);
          if (rr <= cfg.tol * cfg.tol * scale2) {
            out.converged = true;
            break;
          }
        }
        pending = 0;
        if (out.converged) break;
      }
    }
    if (k == niter - 1) break;
    HDCR_TRY(A.apply_dot(w.r, w.Ar, rs, &s->gamma_new, st));
    out.matvecs++;
    HDCR_TRY(launch_cr_update_p<R>(w.r, w.p, w.Ar, w.Ap, n, rs, s, st));
  }
  if (res) *res = out;
  return HDCR_OK;
}

}  // namespace hdcr
