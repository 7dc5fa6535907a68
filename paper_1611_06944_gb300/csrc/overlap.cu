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

#include "chebyshev.cuh"
#include "coarse.cuh"
#include "dwf_stencil.cuh"
#include "host_io.cuh"
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

template int launch_cf<double>(const Geom&, double, const CFCoef&, const cpx<double>*, const cpx<double>*,
                               cpx<double>*, int, RedScratch, double*, cudaStream_t);
template int launch_cf<float>(const Geom&, double, const CFCoef&, const cpx<float>*, const cpx<float>*,
                              cpx<float>*, int, RedScratch, double*, cudaStream_t);

void cf_coef_free(CFCoef* cf) { delete cf; }

static int cf_coef_of(const Geom* g, const hdcr_cf_params* p, CFCoef* cf) {
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

static int cf_coef(const hdcr_geom* gp, const hdcr_cf_params* p, Geom* g, CFCoef* cf) {
  HDCR_TRY(make_geom(gp, g));
  return cf_coef_of(g, p, cf);
}

template <typename R>
static int cf_solve_impl(const Geom& g, double M5, const CFCoef& cf, const void* U, const void* b, void* x, double tol,
                         int max_iter, hdcr_solve_stats* stats, cudaStream_t st) {
  const auto t0 = std::chrono::steady_clock::now();
  FineOp<R> A{g, M5, 0.0, (const cpx<R>*)U};
  A.cf = &cf;
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

// ------------------------------------------------------------------ two-level method
// The site-local part of H_cf (part < 0: the diagonal (4 - M5) psi, the couplings of
// the components and R gamma5 on the last one, with the factor of H) or its hop d
// alone (part = d = 2 mu + (0 forward, 1 backward)): H_cf is their sum.
template <typename R>
__global__ void __launch_bounds__(256) cf_part_kernel(Geom g, R m0, CFCoef cf, const cpx<R>* __restrict__ U,
                                                      const cpx<R>* __restrict__ in, cpx<R>* __restrict__ out,
                                                      int part) {
  const int n = g.Ls;
  for (long long i5 = (long long)blockIdx.x * blockDim.x + threadIdx.x; i5 < g.V5;
       i5 += (long long)gridDim.x * blockDim.x) {
    const int x4 = (int)(i5 / n);
    const int s = (int)(i5 - (long long)x4 * n);
    int co[4];
    x4_coords(g, x4, co);
    const cpx<R>* self = in + (unsigned)(x4 * 12 * n + s);
    cpx<R> acc[4][3];
#pragma unroll
    for (int sp = 0; sp < 4; ++sp)
#pragma unroll
      for (int c = 0; c < 3; ++c) acc[sp][c] = part < 0 ? m0 * ld(self + (3 * sp + c) * n) : cpx<R>((R)0, (R)0);
    switch (part) {
      case 0: hop_full<R, 0, 0, +1>(g, U, in, x4, s, co, acc); break;
      case 1: hop_full<R, 0, 0, -1>(g, U, in, x4, s, co, acc); break;
      case 2: hop_full<R, 0, 1, +1>(g, U, in, x4, s, co, acc); break;
      case 3: hop_full<R, 0, 1, -1>(g, U, in, x4, s, co, acc); break;
      case 4: hop_full<R, 0, 2, +1>(g, U, in, x4, s, co, acc); break;
      case 5: hop_full<R, 0, 2, -1>(g, U, in, x4, s, co, acc); break;
      case 6: hop_full<R, 0, 3, +1>(g, U, in, x4, s, co, acc); break;
      case 7: hop_full<R, 0, 3, -1>(g, U, in, x4, s, co, acc); break;
      default: break;
    }
    const bool local = part < 0;
    const R sc = (R)cf.scale[s];
    const R cm = local && s > 0 ? (R)cf.coup[s - 1] : (R)0, cp = local && s + 1 < n ? (R)cf.coup[s] : (R)0;
    const R rl = local && s == n - 1 ? (R)cf.R : (R)0;
    cpx<R>* o = out + (unsigned)(x4 * 12 * n + s);
#pragma unroll
    for (int sp = 0; sp < 4; ++sp)
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        const int k = 3 * sp + c;
        const R g5 = sp < 2 ? (R)1 : (R)-1;
        const cpx<R> v = ld(self + k * n);
        cpx<R> y(g5 * (sc * acc[sp][c].re + rl * v.re), g5 * (sc * acc[sp][c].im + rl * v.im));
        if (cm != (R)0) {
          const cpx<R> a = ld(self + k * n - 1);
          y.re += cm * a.re;
          y.im += cm * a.im;
        }
        if (cp != (R)0) {
          const cpx<R> b = ld(self + k * n + 1);
          y.re += cp * b.re;
          y.im += cp * b.im;
        }
        st(o + k * n, y);
      }
  }
}

// plus = (1 + gamma5)/2 in, minus = (1 - gamma5)/2 in: the 4d chirality of every
// site and fifth coordinate (the upper and the lower two spins in the chiral basis)
template <typename R>
__global__ void g5_split_kernel(const cpx<R>* __restrict__ in, cpx<R>* __restrict__ plus, cpx<R>* __restrict__ minus,
                                long long n, int ls) {
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
    const int c = (int)((e / ls) % 12);
    const cpx<R> v = ld(in + e);
    const cpx<R> z((R)0, (R)0);
    st(plus + e, c < 6 ? v : z);
    st(minus + e, c < 6 ? z : v);
  }
}

constexpr int CFP_J = 4;  // basis vectors per projection CTA

// Column k of the little operator from Y = (part of H_cf) phi_k: for block a and
// CFP_J vectors j, the sum over the block's sites of conj(phi_j) Y, split for a hop
// part d into the sites on the block's face in the hop's direction (leg d, written)
// and the rest (the self leg, added); the local part adds all of it to the self leg.
__global__ void __launch_bounds__(RED_THREADS) cf_project_kernel(Geom g, BlockGeom bg, const cpx<double>* __restrict__ phi,
                                                                 const cpx<double>* __restrict__ Y,
                                                                 cpx<double>* __restrict__ A, int nvec, int k,
                                                                 int part) {
  const int a = blockIdx.x;
  const int j0 = blockIdx.y * CFP_J;
  const long long fs = g.V5 * 12;
  const int per = 12 * g.Ls;
  const int nel = bg.bvol * per;
  const int mu = part >= 0 ? part / 2 : 0;
  const bool fwd = part >= 0 && part % 2 == 0;
  double acc[4 * CFP_J];  // per j: self (re, im), face (re, im)
#pragma unroll
  for (int i = 0; i < 4 * CFP_J; ++i) acc[i] = 0.0;
  for (int e = threadIdx.x; e < nel; e += RED_THREADS) {
    const int site = e / per;
    const long long i5 = block_site(g, bg, a, (long long)site * g.Ls);
    const int x4 = (int)(i5 / g.Ls);
    bool face = false;
    if (part >= 0) {
      int co[4];
      x4_coords(g, x4, co);
      face = co[mu] % bg.b[mu] == (fwd ? bg.b[mu] - 1 : 0);
    }
    const unsigned off = (unsigned)x4 * (unsigned)per + (unsigned)(e - site * per);
    const cpx<double> q = Y[off];
#pragma unroll
    for (int i = 0; i < CFP_J; ++i) {
      if (j0 + i >= nvec) continue;
      const cpx<double> p = phi[(long long)(j0 + i) * fs + off];
      const double re = p.re * q.re + p.im * q.im, im = p.re * q.im - p.im * q.re;
      if (face) {
        acc[4 * i + 2] += re;
        acc[4 * i + 3] += im;
      } else {
        acc[4 * i] += re;
        acc[4 * i + 1] += im;
      }
    }
  }
  block_reduce<4 * CFP_J>(acc);
  if (threadIdx.x == 0) {
    const int leg = part >= 0 ? leg_of(mu, fwd ? +1 : -1) : 0;
    for (int i = 0; i < CFP_J; ++i) {
      const int j = j0 + i;
      if (j >= nvec) continue;
      cpx<double>* a0 = A + (((long long)a * NLEGS + 0) * nvec + j) * nvec + k;
      a0->re += acc[4 * i];
      a0->im += acc[4 * i + 1];
      if (part >= 0) A[(((long long)a * NLEGS + leg) * nvec + j) * nvec + k] = cpx<double>(acc[4 * i + 2], acc[4 * i + 3]);
    }
  }
}

static int cf_build_impl(const hdcr_subspace* sub, double M5, const CFCoef& cf, const cpx<double>* U, cudaStream_t st,
                         hdcr_coarse** out) {
  const Geom& g = sub->g;
  const BlockGeom& bg = sub->bg;
  const int nvec = sub->nvec;
  const long long fs = g.V5 * 12;
  hdcr_coarse* co = new hdcr_coarse();
  co->sub = sub;
  co->g = g;
  co->bg = bg;
  co->nvec = nvec;
  co->dtype = HDCR_C128;
  co->M5 = M5;
  co->mf = 0.0;
  co->cf = new CFCoef(cf);
  cudaGetDevice(&co->device);
  cpx<double>* Y = nullptr;
  int s = HDCR_OK;
  const size_t abytes = sizeof(cpx<double>) * (size_t)bg.Vc * NLEGS * nvec * nvec;
  cudaError_t e = cudaMalloc(&co->A, abytes);
  if (e == cudaSuccess) e = cudaMalloc(&co->nbr, sizeof(int) * bg.Vc * NLEGS);
  if (e == cudaSuccess) e = cudaMalloc(&Y, sizeof(cpx<double>) * fs);
  if (e == cudaSuccess) e = cudaMemsetAsync(co->A, 0, abytes, st);
  if (e != cudaSuccess) s = cuda_status(e, "continued-fraction coarse operator storage");
  if (s == HDCR_OK) s = fill_neighbour_table(bg, co->nbr, st);
  const cpx<double>* phi = (const cpx<double>*)sub->vecs;
  for (int k = 0; k < nvec && s == HDCR_OK; ++k) {
    for (int part = -1; part < 8 && s == HDCR_OK; ++part) {
      cf_part_kernel<double><<<num_blocks(g.V5, 256), 256, 0, st>>>(g, 4.0 - M5, cf, U, phi + (long long)k * fs, Y,
                                                                   part);
      cf_project_kernel<<<dim3(bg.Vc, (nvec + CFP_J - 1) / CFP_J), RED_THREADS, 0, st>>>(g, bg, phi, Y,
                                                                                         (cpx<double>*)co->A, nvec,
                                                                                         k, part);
      count_launches(2);
      e = cudaGetLastError();
      if (e != cudaSuccess) s = cuda_status(e, "continued-fraction coarse operator build");
    }
  }
  if (s == HDCR_OK) {
    e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) s = cuda_status(e, "continued-fraction coarse operator build");
  }
  if (Y) cudaFree(Y);
  if (s != HDCR_OK) {
    hdcr_coarse_destroy(co);
    return s;
  }
  *out = co;
  return HDCR_OK;
}

// x <- the subspace filter (CR steps on H_cf x = 0, or the Chebyshev filter on H_cf^2) in place
template <typename R>
static int cf_filter_impl(const Geom& g, double M5, const CFCoef& cf, const void* U, void* x,
                          const hdcr_subspace_params* sp, cudaStream_t st) {
  FineOp<R> H{g, M5, 0.0, (const cpx<R>*)U};
  H.cf = &cf;
  const long long n = H.n();
  int s = HDCR_OK;
  if (sp->kind == HDCR_SUBSPACE_CR_SMOOTH) {
    CRWork<R> w;
    HDCR_TRY(crwork_alloc<R>(&w, n));
    cpx<R>* zero = nullptr;
    cudaError_t e = cudaMalloc(&zero, sizeof(cpx<R>) * n);
    if (e == cudaSuccess) e = cudaMemsetAsync(zero, 0, sizeof(cpx<R>) * n, st);
    if (e != cudaSuccess) s = cuda_status(e, "continued-fraction filter workspace");
    CRConfig cfg;
    cfg.fixed_iters = sp->order;
    if (s == HDCR_OK) s = cr_run<R>(H, zero, (cpx<R>*)x, w, cfg, nullptr, st);
    cudaStreamSynchronize(st);
    if (zero) cudaFree(zero);
    crwork_free<R>(&w);
    return s;
  }
  ChebWork<R> cw;
  HDCR_TRY(cheb_work_alloc<R>(&cw, n));
  RedBuffers rb{{nullptr, nullptr}, nullptr, 0, nullptr};
  s = red_buffers_alloc(&rb, 2);
  if (s == HDCR_OK) s = cheb_filter<R>(H, (cpx<R>*)x, sp->order, sp->lam_cut, sp->lam_max, cw, rb.rs, st);
  cudaStreamSynchronize(st);
  red_buffers_free(&rb);
  cheb_work_free<R>(&cw);
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

extern "C" int hdcr_cf_filter(const hdcr_geom* gp, double M5, const hdcr_cf_params* p, const void* U, void* x,
                              int dtype, const hdcr_subspace_params* sp, void* stream) {
  Geom g;
  CFCoef cf;
  HDCR_TRY(cf_coef(gp, p, &g, &cf));
  if (!U || !x || !sp || sp->order < 0 ||
      (sp->kind != HDCR_SUBSPACE_CR_SMOOTH && sp->kind != HDCR_SUBSPACE_CHEBYSHEV) ||
      (sp->kind == HDCR_SUBSPACE_CHEBYSHEV && (sp->order < 1 || !(sp->lam_cut > 0.0) || !(sp->lam_max > sp->lam_cut)))) {
    set_error("hdcr_cf_filter: null pointer or bad filter parameters");
    return HDCR_ERR_BAD_ARG;
  }
  if (dtype == HDCR_C128) return cf_filter_impl<double>(g, M5, cf, U, x, sp, as_stream(stream));
  if (dtype == HDCR_C64) return cf_filter_impl<float>(g, M5, cf, U, x, sp, as_stream(stream));
  set_error("hdcr_cf_filter: unknown dtype %d", dtype);
  return HDCR_ERR_BAD_ARG;
}

extern "C" int hdcr_cf_build_coarse_op(const hdcr_subspace* sub, double M5, const hdcr_cf_params* p, const void* U,
                                       void* stream, hdcr_coarse** out) {
  HDCR_TRY(subspace_check(sub));
  if (!p || !U || !out) {
    set_error("hdcr_cf_build_coarse_op: null pointer");
    return HDCR_ERR_BAD_ARG;
  }
  *out = nullptr;
  if (sub->dtype != HDCR_C128) {
    set_error("hdcr_cf_build_coarse_op: the basis must be stored as C128");
    return HDCR_ERR_BAD_ARG;
  }
  CFCoef cf;
  HDCR_TRY(cf_coef_of(&sub->g, p, &cf));
  cudaStream_t st = as_stream(stream);
  Staged su;  // links given in host memory are staged through the device
  HDCR_TRY(su.in(U, (size_t)sub->g.V4 * 36 * 16, st));
  return cf_build_impl(sub, M5, cf, (const cpx<double>*)su.ptr(), st, out);
}

extern "C" int hdcr_gamma5_split(const hdcr_geom* gp, const void* in, void* plus, void* minus, int dtype, int nfields,
                                 void* stream) {
  Geom g;
  HDCR_TRY(make_geom(gp, &g));
  if (!in || !plus || !minus || plus == minus || nfields < 1) {
    set_error("hdcr_gamma5_split: bad pointers or nfields");
    return HDCR_ERR_BAD_ARG;
  }
  const long long n = g.V5 * 12 * nfields;
  cudaStream_t st = as_stream(stream);
  if (dtype == HDCR_C128)
    g5_split_kernel<double><<<num_blocks(n, 256, 8192), 256, 0, st>>>((const cpx<double>*)in, (cpx<double>*)plus,
                                                                     (cpx<double>*)minus, n, g.Ls);
  else if (dtype == HDCR_C64)
    g5_split_kernel<float><<<num_blocks(n, 256, 8192), 256, 0, st>>>((const cpx<float>*)in, (cpx<float>*)plus,
                                                                    (cpx<float>*)minus, n, g.Ls);
  else {
    set_error("hdcr_gamma5_split: unknown dtype %d", dtype);
    return HDCR_ERR_BAD_ARG;
  }
  count_launch();
  HDCR_LAUNCH_CHECK();
  return HDCR_OK;
}
