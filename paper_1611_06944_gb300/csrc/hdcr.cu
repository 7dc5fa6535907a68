// HDCR solve (Section 4): flexible GCR(m) on H in FP64, preconditioned by the
// two-level V-cycle
//     z1 = S r;   z2 = z1 + P A^{-1} P^dag (r - H z1);   z = z2 + S (r - H z2)
// with S a fixed number of CR steps from zero and A^{-1} a CR solve on the
// coarse operator to a loose tolerance.  For a fixed linear S and an exact
// coarse solve this equals M_outer = S P_L + P_R S + Q - S P_L H S.  The
// preconditioner is nonlinear (CR), which is why the outer iteration is the
// flexible variant.  The preconditioner runs in FP64 or FP32 (inner_dtype);
// the outer orthogonalisation, updates and the true residual are FP64.
// Smoother: CR steps from zero (nonlinear) or the Chebyshev polynomial
// S = H p(H^2) of Section 4 (linear).  Coarse solve: CR on the coarse operator
// or its dense inverse.
#include <chrono>
#include <mutex>
#include <vector>

#include "host_io.cuh"
#include "level2.cuh"
#include "chebyshev.cuh"
#include "coarse.cuh"

namespace hdcr {

// ------------------------------------------------------------------ kernels
template <typename R>
__global__ void sub_kernel(const cpx<R>* __restrict__ a, const cpx<R>* __restrict__ b, cpx<R>* __restrict__ out,
                           long long n) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    st(out + i, ld(a + i) - ld(b + i));
}

template <typename R>
__global__ void add_kernel(cpx<R>* __restrict__ y, const cpx<R>* __restrict__ x, long long n) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    st(y + i, ld(y + i) + ld(x + i));
}

// w -= beta wj;  z -= beta zj   (beta complex, device)
__global__ void axpy2_neg_kernel(cpx<double>* __restrict__ w, const cpx<double>* __restrict__ wj,
                                 cpx<double>* __restrict__ z, const cpx<double>* __restrict__ zj, long long n,
                                 const double* __restrict__ beta) {
  const double br = beta[0], bi = beta[1];
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const cpx<double> a = wj[i], c = zj[i];
    cpx<double> u = w[i], v = z[i];
    u.re = fma(-br, a.re, fma(bi, a.im, u.re));
    u.im = fma(-br, a.im, fma(-bi, a.re, u.im));
    v.re = fma(-br, c.re, fma(bi, c.im, v.re));
    v.im = fma(-br, c.im, fma(-bi, c.re, v.im));
    w[i] = u;
    z[i] = v;
  }
}

// w /= |w|, z /= |w|
__global__ void scale2_kernel(cpx<double>* __restrict__ w, cpx<double>* __restrict__ z, long long n,
                              const double* __restrict__ n2) {
  const double s = *n2 > 0.0 ? 1.0 / sqrt(*n2) : 0.0;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const cpx<double> a = w[i], c = z[i];
    w[i] = cpx<double>(a.re * s, a.im * s);
    z[i] = cpx<double>(c.re * s, c.im * s);
  }
}

// x += a z;  r -= a w;  |r|^2 -> *rr
__global__ void __launch_bounds__(RED_THREADS) fgcr_update_kernel(cpx<double>* __restrict__ x,
                                                                  const cpx<double>* __restrict__ z,
                                                                  cpx<double>* __restrict__ r,
                                                                  const cpx<double>* __restrict__ w, long long n,
                                                                  const double* __restrict__ a, RedScratch rs,
                                                                  double* rr) {
  const double ar = a[0], ai = a[1];
  double acc[1] = {0.0};
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const cpx<double> zv = z[i], wv = w[i];
    cpx<double> xv = x[i], rv = r[i];
    xv.re = fma(ar, zv.re, fma(-ai, zv.im, xv.re));
    xv.im = fma(ar, zv.im, fma(ai, zv.re, xv.im));
    rv.re = fma(-ar, wv.re, fma(ai, wv.im, rv.re));
    rv.im = fma(-ar, wv.im, fma(-ai, wv.re, rv.im));
    x[i] = xv;
    r[i] = rv;
    acc[0] = fma((double)rv.re, (double)rv.re, fma((double)rv.im, (double)rv.im, acc[0]));
  }
  double tot[1];
  if (grid_reduce<1>(acc, rs, tot)) *rr = tot[0];
}

// ------------------------------------------------------------------ workspace
struct SolveCache {
  int restart = 0;
  int inner = -1;
  long long fs = 0, cs = 0;
  void* mem = nullptr;
  // FP64 outer
  cpx<double>* Z = nullptr;  // restart fields
  cpx<double>* W = nullptr;  // restart fields
  cpx<double>* r = nullptr;
  cpx<double>* tmp = nullptr;
  // inner precision (R): r_in, z_in, t1, t2, e; coarse rhs / solution
  void* r_in = nullptr;
  void* z_in = nullptr;
  void* t1 = nullptr;
  void* t2 = nullptr;
  void* e = nullptr;
  void* c_rhs = nullptr;
  void* c_sol = nullptr;
  void* U_in = nullptr;  // links in the inner precision (FP32 mode)
  void* sw = nullptr;    // CRWork<R> of the smoother
  void* cw = nullptr;    // CRWork<R> of the coarse solve
  void* chw = nullptr;   // ChebWork<R> of the Chebyshev smoother
  std::vector<double> cheb_c;
  RedBuffers rb{};       // outer reductions; scal: [0..127] MGS coefficients, 128.. scalars
  cudaEvent_t ev[6] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
  CRGraph cgraph;        // the coarse CR's iterations between host checks, replayed every V-cycle
};

template <typename R>
static void free_inner(SolveCache* c) {
  if (c->sw) {
    crwork_free<R>((CRWork<R>*)c->sw);
    delete (CRWork<R>*)c->sw;
  }
  if (c->cw) {
    crwork_free<R>((CRWork<R>*)c->cw);
    delete (CRWork<R>*)c->cw;
  }
  if (c->chw) {
    cheb_work_free<R>((ChebWork<R>*)c->chw);
    delete (ChebWork<R>*)c->chw;
  }
  c->sw = c->cw = c->chw = nullptr;
}

void solve_cache_free(SolveCache* c) {
  if (!c) return;
  if (c->inner == HDCR_C128) free_inner<double>(c);
  if (c->inner == HDCR_C64) free_inner<float>(c);
  cr_graph_free(&c->cgraph);
  if (c->mem) cudaFree(c->mem);
  red_buffers_free(&c->rb);
  for (int i = 0; i < 6; ++i)
    if (c->ev[i]) cudaEventDestroy(c->ev[i]);
  delete c;
}

template <typename R>
static int alloc_cache(const hdcr_coarse* co, int restart, SolveCache** out) {
  SolveCache* c = new SolveCache();
  c->restart = restart;
  c->inner = sizeof(R) == 8 ? HDCR_C128 : HDCR_C64;
  c->fs = co->g.V5 * 12;
  c->cs = (long long)co->bg.Vc * co->nvec;
  const size_t f64 = sizeof(cpx<double>) * c->fs, fin = sizeof(cpx<R>) * c->fs, cin = sizeof(cpx<R>) * c->cs;
  const size_t bytes = f64 * (2 * restart + 2) + fin * 5 + cin * 2 + sizeof(cpx<R>) * (size_t)co->g.V4 * 36 + 1024;
  cudaError_t e = cudaMalloc(&c->mem, bytes);
  if (e != cudaSuccess) {
    delete c;
    set_error("HDCR workspace: cudaMalloc(%zu) failed: %s", bytes, cudaGetErrorString(e));
    return HDCR_ERR_NO_MEMORY;
  }
  char* p = (char*)c->mem;
  auto take = [&](size_t b) {
    void* q = p;
    p += (b + 255) & ~(size_t)255;
    return q;
  };
  c->Z = (cpx<double>*)take(f64 * restart);
  c->W = (cpx<double>*)take(f64 * restart);
  c->r = (cpx<double>*)take(f64);
  c->tmp = (cpx<double>*)take(f64);
  c->r_in = take(fin);
  c->z_in = take(fin);
  c->t1 = take(fin);
  c->t2 = take(fin);
  c->e = take(fin);
  c->c_rhs = take(cin);
  c->c_sol = take(cin);
  c->U_in = take(sizeof(cpx<R>) * (size_t)co->g.V4 * 36);
  int s = red_buffers_alloc(&c->rb, 192);
  CRWork<R>* sw = new CRWork<R>();
  CRWork<R>* cw = new CRWork<R>();
  ChebWork<R>* chw = new ChebWork<R>();
  c->sw = sw;
  c->cw = cw;
  c->chw = chw;
  if (s == HDCR_OK) s = crwork_alloc<R>(sw, c->fs);
  if (s == HDCR_OK) s = crwork_alloc<R>(cw, c->cs);
  if (s == HDCR_OK) s = cheb_work_alloc<R>(chw, c->fs);
  for (int i = 0; i < 6 && s == HDCR_OK; ++i) {
    if (cudaEventCreate(&c->ev[i]) != cudaSuccess) s = HDCR_ERR_CUDA;
  }
  if (s != HDCR_OK) {
    solve_cache_free(c);  // frees whatever part was allocated
    return s;
  }
  *out = c;
  return HDCR_OK;
}

struct VStats {
  int fine = 0;          // inner-precision fine applies
  int coarse = 0;        // coarse stencil applies
  int coarse_dense = 0;  // dense coarse solves
  int coarse_fail = 0;
};

// out = S r (out must not alias r or the workspaces)
template <typename R>
static int smooth(const FineOp<R>& H, SolveCache* c, const hdcr_solve_params* prm, const cpx<R>* r, cpx<R>* out,
                  VStats* vs, cudaStream_t st) {
  if (prm->smoother_kind == HDCR_SMOOTHER_CHEBYSHEV)
    return cheb_smoother<R>(H, r, out, c->cheb_c, prm->cheb_lo, prm->cheb_hi, *(ChebWork<R>*)c->chw, st, &vs->fine);
  CRWork<R>& sw = *(CRWork<R>*)c->sw;
  CRConfig cfg;
  cfg.fixed_iters = prm->smoother_order;
  cfg.x_zero = true;
  CRResult res;
  HDCR_CUDA_TRY(cudaMemsetAsync(out, 0, sizeof(cpx<R>) * c->fs, st));
  HDCR_TRY(cr_run<R>(H, r, out, sw, cfg, &res, st));
  vs->fine += res.matvecs;
  return HDCR_OK;
}

// c_sol = A^{-1} c_rhs (coarse vectors in R)
template <typename R>
static int coarse_solve(const hdcr_coarse* co, SolveCache* c, const hdcr_solve_params* prm, VStats* vs,
                        cudaStream_t st) {
  if (prm->coarse_solver == HDCR_COARSE_RECURSIVE) {
    int it = 0;
    HDCR_TRY(level2_solve<R>(co, (const cpx<R>*)c->c_rhs, (cpx<R>*)c->c_sol, prm->coarse_tol, prm->coarse_max, &it,
                             st));
    vs->coarse += it;
    return HDCR_OK;
  }
  if (prm->coarse_solver == HDCR_COARSE_DENSE) {
    vs->coarse_dense++;
    return launch_dense_solve<R>(co, (const cpx<R>*)c->c_rhs, (cpx<R>*)c->c_sol, 1, st);
  }
  CRWork<R>& cw = *(CRWork<R>*)c->cw;
  HDCR_CUDA_TRY(cudaMemsetAsync(c->c_sol, 0, sizeof(cpx<R>) * c->cs, st));
  CRConfig ccfg;
  ccfg.tol = prm->coarse_tol;
  ccfg.max_iter = prm->coarse_max;
  ccfg.x_zero = true;
  ccfg.check_every = 8;
  ccfg.graph = &c->cgraph;
  CoarseOp<R> A{co};
  CRResult res;
  HDCR_TRY(cr_run<R>(A, (const cpx<R>*)c->c_rhs, (cpx<R>*)c->c_sol, cw, ccfg, &res, st));
  vs->coarse += res.matvecs;
  if (!res.converged) vs->coarse_fail++;
  return HDCR_OK;
}

// z = B r in precision R (r, z in R)
template <typename R>
static int vcycle(const hdcr_coarse* co, const FineOp<R>& H, SolveCache* c, const hdcr_solve_params* prm,
                  const cpx<R>* r, cpx<R>* z, VStats* vs, cudaStream_t st) {
  const long long fs = c->fs;
  cpx<R>* t1 = (cpx<R>*)c->t1;
  cpx<R>* t2 = (cpx<R>*)c->t2;
  cpx<R>* e = (cpx<R>*)c->e;
  const int nb = num_blocks(fs, 256, 4096);
  if (prm->cycle == HDCR_CYCLE_POST) {
    // z1 = P A^{-1} P^dag r;  z = z1 + S (r - H z1)
    HDCR_CUDA_TRY(cudaEventRecord(c->ev[0], st));
    HDCR_CUDA_TRY(cudaEventRecord(c->ev[1], st));
    HDCR_CUDA_TRY(cudaEventRecord(c->ev[2], st));
    HDCR_TRY(launch_restrict<R>(co->sub, r, (cpx<R>*)c->c_rhs, 1, st));
    HDCR_TRY(coarse_solve<R>(co, c, prm, vs, st));
    HDCR_TRY(launch_prolong<R>(co->sub, (const cpx<R>*)c->c_sol, (const cpx<R>*)nullptr, z, 1, st));
    HDCR_CUDA_TRY(cudaEventRecord(c->ev[3], st));
    HDCR_TRY(H.apply(z, t1, st));
    vs->fine++;
    sub_kernel<R><<<nb, 256, 0, st>>>(r, t1, t2, fs); count_launch();
    HDCR_LAUNCH_CHECK();
    HDCR_CUDA_TRY(cudaEventRecord(c->ev[4], st));
    HDCR_TRY(smooth<R>(H, c, prm, t2, e, vs, st));
    add_kernel<R><<<nb, 256, 0, st>>>(z, e, fs); count_launch();
    HDCR_LAUNCH_CHECK();
    HDCR_CUDA_TRY(cudaEventRecord(c->ev[5], st));
    return HDCR_OK;
  }
  // z1 = S r
  HDCR_CUDA_TRY(cudaEventRecord(c->ev[0], st));
  HDCR_TRY(smooth<R>(H, c, prm, r, z, vs, st));
  HDCR_CUDA_TRY(cudaEventRecord(c->ev[1], st));
  // r1 = r - H z1;  z2 = z1 + P A^{-1} P^dag r1
  HDCR_TRY(H.apply(z, t1, st));
  vs->fine++;
  sub_kernel<R><<<nb, 256, 0, st>>>(r, t1, t2, fs); count_launch();
  HDCR_LAUNCH_CHECK();
  HDCR_CUDA_TRY(cudaEventRecord(c->ev[2], st));
  HDCR_TRY(launch_restrict<R>(co->sub, t2, (cpx<R>*)c->c_rhs, 1, st));
  HDCR_TRY(coarse_solve<R>(co, c, prm, vs, st));
  HDCR_TRY(launch_prolong<R>(co->sub, (const cpx<R>*)c->c_sol, z, z, 1, st));
  HDCR_CUDA_TRY(cudaEventRecord(c->ev[3], st));
  // r2 = r - H z2;  z = z2 + S r2
  HDCR_TRY(H.apply(z, t1, st));
  vs->fine++;
  sub_kernel<R><<<nb, 256, 0, st>>>(r, t1, t2, fs); count_launch();
  HDCR_LAUNCH_CHECK();
  HDCR_CUDA_TRY(cudaEventRecord(c->ev[4], st));
  HDCR_TRY(smooth<R>(H, c, prm, t2, e, vs, st));
  add_kernel<R><<<nb, 256, 0, st>>>(z, e, fs); count_launch();
  HDCR_LAUNCH_CHECK();
  HDCR_CUDA_TRY(cudaEventRecord(c->ev[5], st));
  return HDCR_OK;
}

template <typename R>
static int solve_impl(const hdcr_coarse* co, SolveCache* c, const void* U, const cpx<double>* b, cpx<double>* x,
                      const hdcr_solve_params* prm, hdcr_solve_stats* stats, cudaStream_t st) {
  const auto t0 = std::chrono::steady_clock::now();
  const long long fs = c->fs;
  const int nb = num_blocks(fs, 256, 4096);
  FineOp<double> H64{co->g, co->M5, co->mf, (const cpx<double>*)U};
  H64.cf = co->cf;
  const cpx<R>* Uin = (const cpx<R>*)U;
  if (sizeof(R) != 8) {
    HDCR_TRY(launch_convert(U, HDCR_C128, c->U_in, HDCR_C64, (long long)co->g.V4 * 36, st));
    Uin = (const cpx<R>*)c->U_in;
  }
  FineOp<R> Hin{co->g, co->M5, co->mf, Uin};
  Hin.cf = co->cf;
  if (prm->smoother_kind == HDCR_SMOOTHER_CHEBYSHEV)
    c->cheb_c = cheb_inverse_coeffs(prm->cheb_lo, prm->cheb_hi, prm->smoother_order);
  double* scal = c->rb.scal;    // [0, 2*restart): MGS coefficients; 128: |w|^2; 130: a; 132: |r|^2; 133: |b|^2
  RedScratch rs = c->rb.rs;
  double* ring = pinned_ring();
  if (!ring) {
    set_error("pinned host buffer unavailable");
    return HDCR_ERR_NO_MEMORY;
  }
  // r = b - H x, |b|^2
  HDCR_TRY(H64.apply(x, c->tmp, st));
  sub_kernel<double><<<nb, 256, 0, st>>>(b, c->tmp, c->r, fs); count_launch();
  HDCR_LAUNCH_CHECK();
  HDCR_TRY(launch_norm2<double>(b, fs, rs, scal + 133, st));
  HDCR_TRY(launch_norm2<double>(c->r, fs, rs, scal + 132, st));
  HDCR_CUDA_TRY(cudaMemcpyAsync(ring, scal + 132, 2 * sizeof(double), cudaMemcpyDeviceToHost, st));
  HDCR_CUDA_TRY(cudaStreamSynchronize(st));
  const double bb = ring[1];
  double rr = ring[0];
  int fine64 = 1, iters = 0, restarts = 0, status = HDCR_OK;
  VStats vs;
  double t_smooth = 0.0, t_coarse = 0.0;
  if (!(bb == bb) || !(rr == rr) || bb > 1e300) {
    set_error("hdcr_solve: non-finite right-hand side or initial residual");
    return HDCR_ERR_NONFINITE;
  }
  const double tol2 = prm->tol * prm->tol * bb;
  bool converged = bb == 0.0 || rr <= tol2;
  while (!converged && iters < prm->max_outer) {
    int i = 0;
    for (; i < prm->restart && iters < prm->max_outer; ++i) {
      cpx<double>* z = c->Z + (long long)i * fs;
      cpx<double>* w = c->W + (long long)i * fs;
      // z = B r
      if (sizeof(R) == 8) {
        HDCR_TRY(vcycle<R>(co, Hin, c, prm, (const cpx<R>*)c->r, (cpx<R>*)z, &vs, st));
      } else {
        HDCR_TRY(launch_convert(c->r, HDCR_C128, c->r_in, HDCR_C64, fs, st));
        HDCR_TRY(vcycle<R>(co, Hin, c, prm, (const cpx<R>*)c->r_in, (cpx<R>*)c->z_in, &vs, st));
        HDCR_TRY(launch_convert(c->z_in, HDCR_C64, z, HDCR_C128, fs, st));
      }
      // w = H z, orthogonalised against the earlier w_j (same coefficients on z)
      HDCR_TRY(H64.apply(z, w, st));
      fine64++;
      for (int j = 0; j < i; ++j) {
        HDCR_TRY(launch_cdot<double>(c->W + (long long)j * fs, w, fs, rs, scal + 2 * j, st));
        axpy2_neg_kernel<<<nb, 256, 0, st>>>(w, c->W + (long long)j * fs, z, c->Z + (long long)j * fs, fs,
                                             scal + 2 * j); count_launch();
        HDCR_LAUNCH_CHECK();
      }
      HDCR_TRY(launch_norm2<double>(w, fs, rs, scal + 128, st));
      scale2_kernel<<<nb, 256, 0, st>>>(w, z, fs, scal + 128); count_launch();
      HDCR_LAUNCH_CHECK();
      HDCR_TRY(launch_cdot<double>(w, c->r, fs, rs, scal + 130, st));
      fgcr_update_kernel<<<red_blocks(fs), RED_THREADS, 0, st>>>(x, z, c->r, w, fs, scal + 130, rs, scal + 132); count_launch();
      HDCR_LAUNCH_CHECK();
      HDCR_CUDA_TRY(cudaMemcpyAsync(ring, scal + 132, sizeof(double), cudaMemcpyDeviceToHost, st));
      HDCR_CUDA_TRY(cudaStreamSynchronize(st));
      float ms = 0.f;
      if (cudaEventElapsedTime(&ms, c->ev[0], c->ev[1]) == cudaSuccess) t_smooth += ms * 1e-3;
      if (cudaEventElapsedTime(&ms, c->ev[4], c->ev[5]) == cudaSuccess) t_smooth += ms * 1e-3;
      if (cudaEventElapsedTime(&ms, c->ev[2], c->ev[3]) == cudaSuccess) t_coarse += ms * 1e-3;
      ++iters;
      rr = ring[0];
      if (!(rr == rr) || rr > 1e300) {
        set_error("hdcr_solve: non-finite residual at outer iteration %d", iters);
        status = HDCR_ERR_NONFINITE;
        break;
      }
      if (rr <= tol2) break;
    }
    if (status != HDCR_OK) break;
    // true residual (restart or convergence check)
    HDCR_TRY(H64.apply(x, c->tmp, st));
    fine64++;
    sub_kernel<double><<<nb, 256, 0, st>>>(b, c->tmp, c->r, fs); count_launch();
    HDCR_LAUNCH_CHECK();
    HDCR_TRY(launch_norm2<double>(c->r, fs, rs, scal + 132, st));
    HDCR_CUDA_TRY(cudaMemcpyAsync(ring, scal + 132, sizeof(double), cudaMemcpyDeviceToHost, st));
    HDCR_CUDA_TRY(cudaStreamSynchronize(st));
    rr = ring[0];
    ++restarts;
    if (!(rr == rr)) {
      status = HDCR_ERR_NONFINITE;
      set_error("hdcr_solve: non-finite true residual");
      break;
    }
    converged = rr <= tol2;
  }
  if (status == HDCR_OK && !converged) {
    set_error("hdcr_solve: not converged after %d outer iterations (|r|/|b| = %g)", iters,
              bb > 0 ? sqrt(rr / bb) : 0.0);
    status = HDCR_ERR_NOT_CONVERGED;
  }
  if (stats) {
    stats->status = status;
    stats->iters = iters;
    stats->fine_matvecs = fine64 + (sizeof(R) == 8 ? vs.fine : 0);
    stats->fine_matvecs_lo = sizeof(R) == 8 ? 0 : vs.fine;
    stats->coarse_matvecs = vs.coarse + vs.coarse_dense;
    stats->restarts = restarts;
    stats->true_resid = bb > 0 ? sqrt(rr / bb) : 0.0;
    stats->t_total = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    stats->t_smoother = t_smooth;
    stats->t_coarse = t_coarse;
  }
  return status;
}

}  // namespace hdcr

using namespace hdcr;

// The solve workspace is cached per coarse handle (created on first use,
// released by hdcr_coarse_destroy).  Solves on one handle must not overlap.
static std::mutex g_cache_mutex;
static std::vector<std::pair<const hdcr_coarse*, SolveCache*>> g_cache;

static SolveCache** cache_slot(const hdcr_coarse* co) {
  for (auto& p : g_cache)
    if (p.first == co) return &p.second;
  g_cache.push_back({co, nullptr});
  return &g_cache.back().second;
}

namespace hdcr {
void solve_cache_release(const hdcr_coarse* co) {
  std::lock_guard<std::mutex> lock(g_cache_mutex);
  for (size_t i = 0; i < g_cache.size(); ++i)
    if (g_cache[i].first == co) {
      solve_cache_free(g_cache[i].second);
      g_cache.erase(g_cache.begin() + i);
      return;
    }
}
}  // namespace hdcr

static int solve_entry(hdcr_coarse* co, const void* U, const void* b, void* x, const hdcr_solve_params* prm,
                       hdcr_solve_stats* stats, void* stream) {
  HDCR_TRY(coarse_check(co));
  if (!U || !b || !x || !prm || b == x) {
    set_error("hdcr_solve: null pointer or b == x");
    return HDCR_ERR_BAD_ARG;
  }
  if (!(prm->tol > 0.0) || prm->max_outer < 1 || prm->restart < 1 || prm->restart > 64 ||
      prm->smoother_order < 0 || !(prm->coarse_tol > 0.0) || prm->coarse_max < 1 ||
      (prm->smoother_kind != HDCR_SMOOTHER_CR && prm->smoother_kind != HDCR_SMOOTHER_CHEBYSHEV) ||
      (prm->coarse_solver != HDCR_COARSE_CR && prm->coarse_solver != HDCR_COARSE_DENSE &&
       prm->coarse_solver != HDCR_COARSE_RECURSIVE) ||
      (prm->cycle != HDCR_CYCLE_SYMMETRIC && prm->cycle != HDCR_CYCLE_POST)) {
    set_error("hdcr_solve: bad parameters");
    return HDCR_ERR_BAD_ARG;
  }
  if (prm->smoother_kind == HDCR_SMOOTHER_CHEBYSHEV &&
      (prm->smoother_order < 1 || !(prm->cheb_lo > 0.0) || !(prm->cheb_hi > prm->cheb_lo))) {
    set_error("hdcr_solve: Chebyshev smoother needs order >= 1 and 0 < cheb_lo < cheb_hi");
    return HDCR_ERR_BAD_ARG;
  }
  if (prm->inner_dtype != HDCR_C128 && prm->inner_dtype != HDCR_C64) {
    set_error("hdcr_solve: unknown inner dtype %d", prm->inner_dtype);
    return HDCR_ERR_BAD_ARG;
  }
  if (co->dtype != prm->inner_dtype || co->sub->dtype != prm->inner_dtype) {
    set_error("hdcr_solve: basis (%d) and coarse operator (%d) must be stored in the inner dtype %d",
              co->sub->dtype, co->dtype, prm->inner_dtype);
    return HDCR_ERR_BAD_ARG;
  }
  if (prm->coarse_solver == HDCR_COARSE_DENSE && !co->Ainv) HDCR_TRY(coarse_invert(co, as_stream(stream)));
  if (prm->coarse_solver == HDCR_COARSE_RECURSIVE && !co->l2) {
    set_error("hdcr_solve: the recursive coarse solve needs a third level (hdcr_coarse_build_level2)");
    return HDCR_ERR_BAD_ARG;
  }
  cudaStream_t st = as_stream(stream);
  SolveCache* cache = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_cache_mutex);
    SolveCache** slot = cache_slot(co);
    if (*slot && ((*slot)->inner != prm->inner_dtype || (*slot)->restart < prm->restart)) {
      solve_cache_free(*slot);
      *slot = nullptr;
    }
    if (!*slot) {
      int s = prm->inner_dtype == HDCR_C128 ? alloc_cache<double>(co, prm->restart, slot)
                                            : alloc_cache<float>(co, prm->restart, slot);
      if (s != HDCR_OK) return s;
    }
    cache = *slot;
  }
  if (prm->inner_dtype == HDCR_C128)
    return solve_impl<double>(co, cache, U, (const cpx<double>*)b, (cpx<double>*)x, prm, stats, st);
  return solve_impl<float>(co, cache, U, (const cpx<double>*)b, (cpx<double>*)x, prm, stats, st);
}

extern "C" int hdcr_solve(hdcr_coarse* co, const void* U, const void* b, void* x,
                          const hdcr_solve_params* prm, hdcr_solve_stats* stats, void* stream) {
  HDCR_TRY(coarse_check(co));
  if (!U || !b || !x || b == x) {
    set_error("hdcr_solve: null pointer or b == x");
    return HDCR_ERR_BAD_ARG;
  }
  // links, source and solution given in host memory are staged through the device
  cudaStream_t st = as_stream(stream);
  const size_t field = (size_t)co->g.V5 * 12 * 16;
  Staged su, sb, sx;
  HDCR_TRY(su.in(U, (size_t)co->g.V4 * 36 * 16, st));
  HDCR_TRY(sb.in(b, field, st));
  HDCR_TRY(sx.out(x, field, st, true));
  const int s = solve_entry(co, su.ptr(), sb.ptr(), sx.ptr(), prm, stats, stream);
  HDCR_TRY(sx.finish());
  if (sx.ptr() != x) HDCR_CUDA_TRY(cudaStreamSynchronize(st));
  return s;
}
