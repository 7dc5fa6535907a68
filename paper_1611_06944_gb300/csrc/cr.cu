// Conjugate residual on H = Gamma5 D_dwf (Section 3):
//
//   r = b - H x,  p = r,  Ar = H r,  Ap = Ar,  gamma = <r, Ar>
//   repeat:  alpha = gamma / |Ap|^2;  x += alpha p;  r -= alpha Ap
//            Ar = H r;  gamma' = <r, Ar>;  beta = gamma' / gamma
//            p = r + beta p;  Ap = Ar + beta Ap
//
// Three kernels per iteration: the x/r update (with |r|^2), the stencil with
// the <r, Ar> reduction fused into it, and the p/Ap update (with |Ap|^2).
// alpha and beta are formed inside the kernels from device scalars; the
// reduction epilogues (last block) advance those scalars.
#include <chrono>

#include <mutex>

#include "dwf_stencil.cuh"
#include "krylov.cuh"

namespace hdcr {

template <typename R, int LS>
__global__ void __launch_bounds__(RED_THREADS, 2) g5dwf_dot_kernel(Geom g, R diag, R mf,
                                                                   const cpx<R>* __restrict__ U,
                                                                   const cpx<R>* __restrict__ in,
                                                                   cpx<R>* __restrict__ out, RedScratch rs,
                                                                   double* result) {
  const int ls = ls_of<LS>(g);
  double acc_d[1] = {0.0};
  for (long long i5 = (long long)blockIdx.x * blockDim.x + threadIdx.x; i5 < g.V5;
       i5 += (long long)gridDim.x * blockDim.x) {
    const int x4 = (int)(i5 / ls);
    const int s = (int)(i5 - (long long)x4 * ls);
    cpx<R> acc[4][3];
    dwf_site<R, LS>(g, diag, mf, U, in, x4, s, acc);
    store_g5r5<R, LS>(g, out, x4, s, acc);
    // <in, out> at the output site (x4, Ls-1-s), where out = gamma5 acc
    const cpx<R>* o = in + (unsigned)(x4 * 12 * ls + (ls - 1 - s));
#pragma unroll
    for (int sp = 0; sp < 4; ++sp)
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        const cpx<R> a = ld(o + (3 * sp + c) * ls);
        // Re conj(a) (gamma5 acc): the sign of gamma5 folded into a, two FMAs
        const double ar = sp >= 2 ? -(double)a.re : (double)a.re, ai = sp >= 2 ? -(double)a.im : (double)a.im;
        acc_d[0] = fma(ar, (double)acc[sp][c].re, fma(ai, (double)acc[sp][c].im, acc_d[0]));
      }
  }
  double tot[1];
  if (grid_reduce<1>(acc_d, rs, tot)) *result = tot[0];
}

template <typename R>
__global__ void __launch_bounds__(RED_THREADS) cr_setup_r_kernel(const cpx<R>* __restrict__ b,
                                                                 const cpx<R>* __restrict__ Hx,
                                                                 cpx<R>* __restrict__ r,
                                                                 cpx<R>* __restrict__ p, long long n,
                                                                 RedScratch rs, CRDev* s) {
  double acc[2] = {0.0, 0.0};
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const cpx<R> bv = ld(b + i);
    cpx<R> rv = bv;
    if (Hx) rv = bv - ld(Hx + i);
    st(r + i, rv);
    st(p + i, rv);
    acc[0] = fma((double)rv.re, (double)rv.re, fma((double)rv.im, (double)rv.im, acc[0]));
    acc[1] = fma((double)bv.re, (double)bv.re, fma((double)bv.im, (double)bv.im, acc[1]));
  }
  double tot[2];
  if (grid_reduce<2>(acc, rs, tot)) {
    s->rr = tot[0];
    s->bb = tot[1];
  }
}

template <typename R>
__global__ void __launch_bounds__(RED_THREADS) cr_setup_ap_kernel(const cpx<R>* __restrict__ Ar,
                                                                  cpx<R>* __restrict__ Ap, long long n,
                                                                  RedScratch rs, CRDev* s) {
  double acc[1] = {0.0};
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const cpx<R> v = ld(Ar + i);
    st(Ap + i, v);
    acc[0] = fma((double)v.re, (double)v.re, fma((double)v.im, (double)v.im, acc[0]));
  }
  double tot[1];
  if (grid_reduce<1>(acc, rs, tot)) s->ApAp = tot[0];
}

template <typename R>
__global__ void __launch_bounds__(RED_THREADS) cr_update_xr_kernel(cpx<R>* __restrict__ x,
                                                                   cpx<R>* __restrict__ r,
                                                                   const cpx<R>* __restrict__ p,
                                                                   const cpx<R>* __restrict__ Ap,
                                                                   long long n, RedScratch rs, CRDev* s) {
  const double den = s->ApAp;
  const R alpha = (R)(den > 0.0 ? s->gamma / den : 0.0);
  double acc[1] = {0.0};
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    cpx<R> xv = ld(x + i), rv = ld(r + i);
    const cpx<R> pv = ld(p + i), av = ld(Ap + i);
    xv.re = fma(alpha, pv.re, xv.re);
    xv.im = fma(alpha, pv.im, xv.im);
    rv.re = fma(-alpha, av.re, rv.re);
    rv.im = fma(-alpha, av.im, rv.im);
    st(x + i, xv);
    st(r + i, rv);
    acc[0] = fma((double)rv.re, (double)rv.re, fma((double)rv.im, (double)rv.im, acc[0]));
  }
  double tot[1];
  if (grid_reduce<1>(acc, rs, tot)) s->rr = tot[0];
}

template <typename R>
__global__ void __launch_bounds__(RED_THREADS) cr_update_p_kernel(const cpx<R>* __restrict__ r,
                                                                  cpx<R>* __restrict__ p,
                                                                  const cpx<R>* __restrict__ Ar,
                                                                  cpx<R>* __restrict__ Ap, long long n,
                                                                  RedScratch rs, CRDev* s) {
  const double gam = s->gamma;
  const R beta = (R)(gam != 0.0 ? s->gamma_new / gam : 0.0);
  double acc[1] = {0.0};
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const cpx<R> rv = ld(r + i), arv = ld(Ar + i);
    cpx<R> pv = ld(p + i), apv = ld(Ap + i);
    pv.re = fma(beta, pv.re, rv.re);
    pv.im = fma(beta, pv.im, rv.im);
    apv.re = fma(beta, apv.re, arv.re);
    apv.im = fma(beta, apv.im, arv.im);
    st(p + i, pv);
    st(Ap + i, apv);
    acc[0] = fma((double)apv.re, (double)apv.re, fma((double)apv.im, (double)apv.im, acc[0]));
  }
  double tot[1];
  if (grid_reduce<1>(acc, rs, tot)) {
    s->ApAp = tot[0];
    s->gamma = s->gamma_new;
  }
}

template <typename R>
__global__ void __launch_bounds__(RED_THREADS) diff_norm_kernel(const cpx<R>* __restrict__ b,
                                                                const cpx<R>* __restrict__ Hx, long long n,
                                                                RedScratch rs, double* result) {
  double acc[1] = {0.0};
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const cpx<R> d = ld(b + i) - ld(Hx + i);
    acc[0] = fma((double)d.re, (double)d.re, fma((double)d.im, (double)d.im, acc[0]));
  }
  double tot[1];
  if (grid_reduce<1>(acc, rs, tot)) *result = tot[0];
}

// ------------------------------------------------------------------- host side
double* pinned_ring() {
  static thread_local double* ring = nullptr;
  if (!ring) {
    if (cudaHostAlloc((void**)&ring, sizeof(double) * PINNED_RING, cudaHostAllocPortable) != cudaSuccess) {
      ring = nullptr;
      cudaGetLastError();
    }
  }
  return ring;
}

template <typename R>
int crwork_alloc(CRWork<R>* w, long long n) {
  void* p = nullptr;
  const size_t bytes = sizeof(cpx<R>) * (size_t)n * 4;
  cudaError_t e = cudaMalloc(&p, bytes);
  if (e != cudaSuccess) {
    set_error("CR workspace: cudaMalloc(%zu) failed: %s", bytes, cudaGetErrorString(e));
    return HDCR_ERR_NO_MEMORY;
  }
  w->r = (cpx<R>*)p;
  w->p = w->r + n;
  w->Ar = w->p + n;
  w->Ap = w->Ar + n;
  int s = red_buffers_alloc(&w->rb, (int)(sizeof(CRDev) / sizeof(double)));
  if (s != HDCR_OK) {
    cudaFree(p);
    return s;
  }
  return HDCR_OK;
}

template <typename R>
void crwork_free(CRWork<R>* w) {
  if (w->r) cudaFree(w->r);
  w->r = nullptr;
  red_buffers_free(&w->rb);
}

template <typename R>
int launch_g5dwf_dot(const Geom& g, double M5, double mf, const cpx<R>* U, const cpx<R>* in,
                     cpx<R>* out, RedScratch rs, double* result, cudaStream_t st) {
  int slot;
  stencil_timer_begin(sizeof(R) == 8 ? 0 : 1, g.V5, st, &slot);
  if (sizeof(R) == 4 && g5dwf_x2_ok(g, in, out)) {
    const int s = launch_g5dwf_x2(g, M5, mf, (const cpx<float>*)U, (const cpx<float>*)in, (cpx<float>*)out, 1, &rs,
                                  result, st);
    stencil_timer_end(slot, st);
    return s;
  }
  HDCR_DISPATCH_LS(g.Ls, (g5dwf_dot_kernel<R, LSC><<<red_blocks(g.V5 * 4), RED_THREADS, 0, st>>>(
                             g, (R)(5.0 - M5), (R)mf, U, in, out, rs, result)));
  stencil_timer_end(slot, st);
  HDCR_LAUNCH_CHECK();
  return HDCR_OK;
}

template <typename R>
int launch_cr_setup_r(const cpx<R>* b, const cpx<R>* Hx, cpx<R>* r, cpx<R>* p, long long n,
                      RedScratch rs, CRDev* s, cudaStream_t st) {
  cr_setup_r_kernel<R><<<red_blocks(n), RED_THREADS, 0, st>>>(b, Hx, r, p, n, rs, s); count_launch();
  HDCR_LAUNCH_CHECK();
  return HDCR_OK;
}
template <typename R>
int launch_cr_setup_ap(const cpx<R>* Ar, cpx<R>* Ap, long long n, RedScratch rs, CRDev* s, cudaStream_t st) {
  cr_setup_ap_kernel<R><<<red_blocks(n), RED_THREADS, 0, st>>>(Ar, Ap, n, rs, s); count_launch();
  HDCR_LAUNCH_CHECK();
  return HDCR_OK;
}
template <typename R>
int launch_cr_update_xr(cpx<R>* x, cpx<R>* r, const cpx<R>* p, const cpx<R>* Ap, long long n,
                        RedScratch rs, CRDev* s, cudaStream_t st) {
  cr_update_xr_kernel<R><<<red_blocks(n), RED_THREADS, 0, st>>>(x, r, p, Ap, n, rs, s); count_launch();
  HDCR_LAUNCH_CHECK();
  return HDCR_OK;
}
template <typename R>
int launch_cr_update_p(const cpx<R>* r, cpx<R>* p, const cpx<R>* Ar, cpx<R>* Ap, long long n,
                       RedScratch rs, CRDev* s, cudaStream_t st) {
  cr_update_p_kernel<R><<<red_blocks(n), RED_THREADS, 0, st>>>(r, p, Ar, Ap, n, rs, s); count_launch();
  HDCR_LAUNCH_CHECK();
  return HDCR_OK;
}
template <typename R>
int launch_diff_norm(const cpx<R>* b, const cpx<R>* y, long long n, RedScratch rs, double* result,
                     cudaStream_t st) {
  diff_norm_kernel<R><<<red_blocks(n), RED_THREADS, 0, st>>>(b, y, n, rs, result); count_launch();
  HDCR_LAUNCH_CHECK();
  return HDCR_OK;
}

#define HDCR_INST_CR(R)                                                                              \
  template int crwork_alloc<R>(CRWork<R>*, long long);                                              \
  template void crwork_free<R>(CRWork<R>*);                                                         \
  template int launch_g5dwf_dot<R>(const Geom&, double, double, const cpx<R>*, const cpx<R>*,        \
                                   cpx<R>*, RedScratch, double*, cudaStream_t);                     \
  template int launch_cr_setup_r<R>(const cpx<R>*, const cpx<R>*, cpx<R>*, cpx<R>*, long long,      \
                                    RedScratch, CRDev*, cudaStream_t);                              \
  template int launch_cr_setup_ap<R>(const cpx<R>*, cpx<R>*, long long, RedScratch, CRDev*,          \
                                     cudaStream_t);                                                 \
  template int launch_cr_update_xr<R>(cpx<R>*, cpx<R>*, const cpx<R>*, const cpx<R>*, long long,    \
                                      RedScratch, CRDev*, cudaStream_t);                            \
  template int launch_cr_update_p<R>(const cpx<R>*, cpx<R>*, const cpx<R>*, cpx<R>*, long long,     \
                                     RedScratch, CRDev*, cudaStream_t);                             \
  template int launch_diff_norm<R>(const cpx<R>*, const cpx<R>*, long long, RedScratch, double*,    \
                                   cudaStream_t);
HDCR_INST_CR(double)
HDCR_INST_CR(float)

void cr_graph_free(CRGraph* g) {
  if (g->exec) cudaGraphExecDestroy(g->exec);
  *g = CRGraph();
}

int capture_stream(cudaStream_t* s) {
  static std::mutex mu;
  static cudaStream_t streams[64] = {};
  int dev = 0;
  HDCR_CUDA_TRY(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64) {
    set_error("capture stream: device %d beyond the 64 supported", dev);
    return HDCR_ERR_BAD_ARG;
  }
  std::lock_guard<std::mutex> lock(mu);
  if (!streams[dev]) HDCR_CUDA_TRY(cudaStreamCreateWithFlags(&streams[dev], cudaStreamNonBlocking));
  *s = streams[dev];
  return HDCR_OK;
}

template <typename R>
static int cr_solve_impl(const Geom& g, const hdcr_dwf_params* p, const void* U, const void* b, void* x,
                         double tol, int max_iter, hdcr_solve_stats* stats, cudaStream_t st) {
  const auto t0 = std::chrono::steady_clock::now();
  FineOp<R> H{g, p->M5, p->mf, (const cpx<R>*)U};
  CRWork<R> w;
  HDCR_TRY(crwork_alloc<R>(&w, H.n()));
  CRConfig cfg;
  cfg.tol = tol;
  cfg.max_iter = max_iter;
  cfg.check_every = sizeof(R) == 8 ? 2 : 8;
  CRGraph graph;  // the iterations between host checks replay from one CUDA graph
  cfg.graph = &graph;
  CRResult res;
  int s = cr_run<R>(H, (const cpx<R>*)b, (cpx<R>*)x, w, cfg, &res, st);
  cr_graph_free(&graph);
  double tr = -1.0;
  if (s == HDCR_OK) {
    s = true_residual2<R>(H, (const cpx<R>*)b, (const cpx<R>*)x, w.Ar, w.rb.rs, &w.dev()->tr, st);
    double* ring = pinned_ring();
    if (s == HDCR_OK && ring) {
      cudaError_t e = cudaMemcpyAsync(ring, &w.dev()->bb, 2 * sizeof(double), cudaMemcpyDeviceToHost, st);
      if (e == cudaSuccess) e = cudaStreamSynchronize(st);
      if (e != cudaSuccess)
        s = cuda_status(e, "CR true residual");
      else
        tr = ring[0] > 0 ? sqrt(ring[1] / ring[0]) : 0.0;
    }
  }
  cudaStreamSynchronize(st);
  crwork_free<R>(&w);
  if (s == HDCR_OK && !res.converged) {
    set_error("CR: not converged after %d iterations (|r|/|b| = %g)", res.iters, res.rel_resid);
    s = HDCR_ERR_NOT_CONVERGED;
  }
  if (stats) {
    stats->status = s;
    stats->iters = res.iters;
    stats->fine_matvecs = res.matvecs + 1;
    stats->fine_matvecs_lo = 0;
    stats->coarse_matvecs = 0;
    stats->restarts = 0;
    stats->true_resid = tr;
    stats->t_total = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    stats->t_smoother = 0.0;
    stats->t_coarse = 0.0;
  }
  return s;
}

}  // namespace hdcr

using namespace hdcr;

extern "C" int hdcr_cr_solve(const hdcr_geom* gp, const hdcr_dwf_params* p, const void* U, const void* b,
                             void* x, int dtype, double tol, int max_iter, hdcr_solve_stats* stats,
                             void* stream) {
  Geom g;
  HDCR_TRY(make_geom(gp, &g));
  if (!p || !U || !b || !x || b == x || !(tol > 0.0) || max_iter < 1) {
    set_error("hdcr_cr_solve: bad pointer, tol or max_iter");
    return HDCR_ERR_BAD_ARG;
  }
  if (dtype == HDCR_C128) return cr_solve_impl<double>(g, p, U, b, x, tol, max_iter, stats, as_stream(stream));
  if (dtype == HDCR_C64) return cr_solve_impl<float>(g, p, U, b, x, tol, max_iter, stats, as_stream(stream));
  set_error("hdcr_cr_solve: unknown dtype %d", dtype);
  return HDCR_ERR_BAD_ARG;
}
