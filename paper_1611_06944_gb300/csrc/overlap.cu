// The continued-fraction overlap operator of Section 3: the Hermitian-indefinite
// block-tridiagonal matrix in the Hermitian Wilson kernel H = gamma5 D_W that the
// paper prints for five components (diagonal H, -H, H, -H, R gamma5 + beta_0 H,
// scalar couplings 1/sqrt(beta_i beta_{i+1}) and 1/sqrt(beta_{N-2})), for any
// number N of components.
//
// The N components are stored where a domain-wall field stores s (psi[x4][c][i],
// the geometry's Ls = N), so the kernel is the domain-wall one's 4d Wilson part
// per component -- one thread per (4d site, component), the links broadcast to
// the N threads of a site -- followed by gamma5, the component's factor on H, the
// two scalar couplings and, on the last component, R gamma5.  CR on it uses the
// Krylov machinery of the domain-wall operator (krylov.cuh).
#include <chrono>

#include "dwf_stencil.cuh"
#include "krylov.cuh"

namespace hdcr {

constexpr int CF_MAX = 16;

struct CFCoef {
  int n;
  double R;
  double scale[CF_MAX];  // factor of H on component i: (-1)^i, beta_0 on the last
  double coup[CF_MAX];   // coupling between components i and i + 1
};

template <typename R>
__global__ void __launch_bounds__(256) cf_kernel(Geom g, R m0, CFCoef cf, const cpx<R>* __restrict__ U,
                                                 const cpx<R>* __restrict__ in, cpx<R>* __restrict__ out, int nrhs,
                                                 RedScratch rs, double* dot) {
  const int n = g.Ls;
  const long long V5 = g.V5;
  double d = 0.0;
  for (long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x; idx < V5 * nrhs;
       idx += (long long)gridDim.x * blockDim.x) {
    const int r = (int)(idx / V5);
    const int i5 = (int)(idx - (long long)r * V5);
    const int x4 = i5 / n;
    const int s = i5 - x4 * n;
    const cpx<R>* src = in + (long long)r * 12 * V5;
    cpx<R>* dst = out + (long long)r * 12 * V5;
    int co[4];
    x4_coords(g, x4, co);
    const cpx<R>* self = src + (unsigned)(x4 * 12 * n + s);
    cpx<R> acc[4][3];
#pragma unroll
    for (int sp = 0; sp < 4; ++sp)
#pragma unroll
      for (int c = 0; c < 3; ++c) acc[sp][c] = m0 * ld(self + (3 * sp + c) * n);
    hop_full<R, 0, 0, +1>(g, U, src, x4, s, co, acc);
    hop_full<R, 0, 0, -1>(g, U, src, x4, s, co, acc);
    hop_full<R, 0, 1, +1>(g, U, src, x4, s, co, acc);
    hop_full<R, 0, 1, -1>(g, U, src, x4, s, co, acc);
    hop_full<R, 0, 2, +1>(g, U, src, x4, s, co, acc);
    hop_full<R, 0, 2, -1>(g, U, src, x4, s, co, acc);
    hop_full<R, 0, 3, +1>(g, U, src, x4, s, co, acc);
    hop_full<R, 0, 3, -1>(g, U, src, x4, s, co, acc);
    // out = scale_s gamma5 D_W psi + couplings (+ R gamma5 psi on the last component)
    const R sc = (R)cf.scale[s];
    const R cm = s > 0 ? (R)cf.coup[s - 1] : (R)0, cp = s + 1 < n ? (R)cf.coup[s] : (R)0;
    const R rl = s == n - 1 ? (R)cf.R : (R)0;
    cpx<R>* o = dst + (unsigned)(x4 * 12 * n + s);
#pragma unroll
    for (int sp = 0; sp < 4; ++sp)
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        const int k = 3 * sp + c;
        const R g5 = sp < 2 ? (R)1 : (R)-1;
        const cpx<R> v = ld(self + k * n);
        cpx<R> y(g5 * (sc * acc[sp][c].re + rl * v.re), g5 * (sc * acc[sp][c].im + rl * v.im));
        if (s > 0) {
          const cpx<R> a = ld(self + k * n - 1);
          y.re += cm * a.re;
          y.im += cm * a.im;
        }
        if (s + 1 < n) {
          const cpx<R> b = ld(self + k * n + 1);
          y.re += cp * b.re;
          y.im += cp * b.im;
        }
        st(o + k * n, y);
        if (dot) d += (double)v.re * y.re + (double)v.im * y.im;
      }
  }
  if (dot) {
    double v[1] = {d};
    double tot[1];
    if (grid_reduce<1>(v, rs, tot)) *dot = tot[0];
  }
}

template <typename R>
int launch_cf(const Geom& g, double M5, const CFCoef& cf, const cpx<R>* U, const cpx<R>* in, cpx<R>* out, int nrhs,
              RedScratch rs, double* dot, cudaStream_t st) {
  const long long n = g.V5 * nrhs;
  // the reducing form runs at most RED_MAX_BLOCKS CTAs (sites grid-stride)
  const int blocks = dot ? red_blocks(n) : num_blocks(n, 256);
  cf_kernel<R><<<blocks, 256, 0, st>>>(g, (R)(4.0 - M5), cf, U, in, out, nrhs, rs, dot);
  count_launch();
  HDCR_LAUNCH_CHECK();
  return HDCR_OK;
}

// the operator for cr_run
template <typename R>
struct CFOp {
  Geom g;
  double M5;
  CFCoef cf;
  const cpx<R>* U;
  long long n() const { return g.V5 * 12; }
  int apply(const cpx<R>* in, cpx<R>* out, cudaStream_t st) const {
    RedScratch none{nullptr, nullptr};
    return launch_cf<R>(g, M5, cf, U, in, out, 1, none, nullptr, st);
  }
  int apply_dot(const cpx<R>* in, cpx<R>* out, RedScratch rs, double* res, cudaStream_t st) const {
    return launch_cf<R>(g, M5, cf, U, in, out, 1, rs, res, st);
  }
};

static int cf_coef(const hdcr_geom* gp, const hdcr_cf_params* p, Geom* g, CFCoef* cf) {
  HDCR_TRY(make_geom(gp, g));
  if (!p || p->ncomp < 2 || p->ncomp > CF_MAX || p->ncomp != g->Ls) {
    set_error("continued-fraction operator: ncomp = %d must equal the geometry's Ls = %d and lie in 2..%d",
              p ? p->ncomp : -1, g->Ls, CF_MAX);
    return HDCR_ERR_BAD_ARG;
  }
  const int n = p->ncomp;
  for (int i = 0; i < n - 1; ++i)
    if (!(p->beta[i] > 0.0)) {
      set_error("continued-fraction operator: beta[%d] = %g must be positive", i, p->beta[i]);
      return HDCR_ERR_BAD_ARG;
    }
  cf->n = n;
  cf->R = p->R;
  for (int i = 0; i < CF_MAX; ++i) cf->scale[i] = cf->coup[i] = 0.0;
  for (int i = 0; i < n; ++i) cf->scale[i] = (i % 2 == 0) ? 1.0 : -1.0;
  cf->scale[n - 1] = p->beta[0];
  for (int i = 0; i < n - 2; ++i) cf->coup[i] = 1.0 / sqrt(p->beta[i] * p->beta[i + 1]);
  cf->coup[n - 2] = 1.0 / sqrt(p->beta[n - 2]);
  return HDCR_OK;
}

template <typename R>
static int cf_solve_impl(const Geom& g, double M5, const CFCoef& cf, const void* U, const void* b, void* x, double tol,
                         int max_iter, hdcr_solve_stats* stats, cudaStream_t st) {
  const auto t0 = std::chrono::steady_clock::now();
  CFOp<R> A{g, M5, cf, (const cpx<R>*)U};
  CRWork<R> w;
  HDCR_TRY(crwork_alloc<R>(&w, A.n()));
  CRConfig cfg;
  cfg.tol = tol;
  cfg.max_iter = max_iter;
  cfg.check_every = 4;
  CRGraph graph;
  cfg.graph = &graph;
  CRResult res;
  int s = cr_run<R>(A, (const cpx<R>*)b, (cpx<R>*)x, w, cfg, &res, st);
  cr_graph_free(&graph);
  double tr = -1.0;
  if (s == HDCR_OK) {
    s = true_residual2<R>(A, (const cpx<R>*)b, (const cpx<R>*)x, w.Ar, w.rb.rs, &w.dev()->tr, st);
    double* ring = pinned_ring();
    if (s == HDCR_OK && ring) {
      cudaError_t e = cudaMemcpyAsync(ring, &w.dev()->bb, 2 * sizeof(double), cudaMemcpyDeviceToHost, st);
      if (e == cudaSuccess) e = cudaStreamSynchronize(st);
      if (e != cudaSuccess)
        s = cuda_status(e, "continued-fraction CR true residual");
      else
        tr = ring[0] > 0 ? sqrt(ring[1] / ring[0]) : 0.0;
    }
  }
  cudaStreamSynchronize(st);
  crwork_free<R>(&w);
  if (s == HDCR_OK && !res.converged) {
    set_error("continued-fraction CR: not converged after %d iterations (|r|/|b| = %g)", res.iters, res.rel_resid);
    s = HDCR_ERR_NOT_CONVERGED;
  }
  if (stats) {
    *stats = hdcr_solve_stats();
    stats->status = s;
    stats->iters = res.iters;
    stats->fine_matvecs = res.matvecs + 1;
    stats->true_resid = tr;
    stats->t_total = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  }
  return s;
}

}  // namespace hdcr

using namespace hdcr;

extern "C" int hdcr_apply_cf_overlap(const hdcr_geom* gp, double M5, const hdcr_cf_params* p, const void* U,
                                     const void* in, void* out, int dtype, int nrhs, void* stream) {
  Geom g;
  CFCoef cf;
  HDCR_TRY(cf_coef(gp, p, &g, &cf));
  if (!U || !in || !out || in == out || nrhs < 1) {
    set_error("hdcr_apply_cf_overlap: bad pointers or nrhs");
    return HDCR_ERR_BAD_ARG;
  }
  RedScratch none{nullptr, nullptr};
  if (dtype == HDCR_C128)
    return launch_cf<double>(g, M5, cf, (const cpx<double>*)U, (const cpx<double>*)in, (cpx<double>*)out, nrhs, none,
                             nullptr, as_stream(stream));
  if (dtype == HDCR_C64)
    return launch_cf<float>(g, M5, cf, (const cpx<float>*)U, (const cpx<float>*)in, (cpx<float>*)out, nrhs, none,
                            nullptr, as_stream(stream));
  set_error("hdcr_apply_cf_overlap: unknown dtype %d", dtype);
  return HDCR_ERR_BAD_ARG;
}

extern "C" int hdcr_cf_cr_solve(const hdcr_geom* gp, double M5, const hdcr_cf_params* p, const void* U, const void* b,
                                void* x, int dtype, double tol, int max_iter, hdcr_solve_stats* stats,
                                void* stream) {
  Geom g;
  CFCoef cf;
  HDCR_TRY(cf_coef(gp, p, &g, &cf));
  if (!U || !b || !x || b == x || !(tol > 0.0) || max_iter < 1) {
    set_error("hdcr_cf_cr_solve: bad pointer, tol or max_iter");
    return HDCR_ERR_BAD_ARG;
  }
  if (dtype == HDCR_C128) return cf_solve_impl<double>(g, M5, cf, U, b, x, tol, max_iter, stats, as_stream(stream));
  if (dtype == HDCR_C64) return cf_solve_impl<float>(g, M5, cf, U, b, x, tol, max_iter, stats, as_stream(stream));
  set_error("hdcr_cf_cr_solve: unknown dtype %d", dtype);
  return HDCR_ERR_BAD_ARG;
}
