// Red-black (even-odd) preconditioned CGNE: the comparison solver of Section 5
// (Table 1), on the same operator, in FP64.
//
// 4d sites are coloured by parity (x + y + z + t) mod 2 (every extent even); the
// fifth dimension is site-local.  D_dwf = M5 + D_hop with M5 = (5 - M5) - P_- S_+
// - P_+ S_- (the site-local part, walls included) and D_hop the 4d hops, which
// join opposite parities.  With the Schur complement on the odd sites,
//     S = M5 - D_oe M5^{-1} D_eo,
// D x = eta is solved as eta~_o = eta_o - D_oe M5^{-1} eta_e, S x_o = eta~_o (CG on
// S^dag S with S^dag = Gamma5 S Gamma5), x_e = M5^{-1} (eta_e - D_eo x_o).  The
// HDCR problem H x = b is D x = Gamma5 b.
//
// Fields are full-lattice arrays in the library layout; a half-lattice operand
// lives on the sites of its parity and is zero elsewhere (every buffer is zeroed
// once and each kernel writes only the sites of its output parity).
//
// M5^{-1} per (4d site, spin-colour) over the fifth coordinate: for the upper
// spins M5 = a - N + mf e_0 e_{Ls-1}^T (a = 5 - M5, N the shift s-1 -> s), a
// lower-bidiagonal matrix plus the wall corner.  Forward substitution gives
// z = (a - N)^{-1} b, and the corner is taken out exactly (Sherman-Morrison with
// (a - N)^{-1} e_0 = (a^{-1}, ..., a^{-Ls})):
//     y = z - [mf z(Ls-1) / (1 + mf a^{-Ls})] (a^{-1}, a^{-2}, ..., a^{-Ls}).
// The lower spins are the same with s reversed.
#include <chrono>

#include "blas.cuh"
#include "dwf_stencil.cuh"
#include "krylov.cuh"

namespace hdcr {

// 4d site of parity ``par`` number h (x in steps of two, fastest)
__device__ __forceinline__ int rb_site(const Geom& g, int h, int par, int co[4]) {
  const int hx = g.L[0] >> 1;
  const int k = h % hx;
  int r = h / hx;
  co[1] = r % g.L[1];
  r /= g.L[1];
  co[2] = r % g.L[2];
  co[3] = r / g.L[2];
  co[0] = 2 * k + ((par + co[1] + co[2] + co[3]) & 1);
  return x4_index(g, co);
}

// out = D_hop in on the sites of parity par (in read on the other parity)
template <int LS>
__global__ void __launch_bounds__(256) rb_hop_kernel(Geom g, const cpx<double>* __restrict__ U,
                                                     const cpx<double>* __restrict__ in,
                                                     cpx<double>* __restrict__ out, int par) {
  const int ls = ls_of<LS>(g);
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= g.V5 / 2) return;
  const int h = (int)(i / ls), s = (int)(i - (long long)h * ls);
  int co[4];
  const int x4 = rb_site(g, h, par, co);
  cpx<double> acc[4][3];
#pragma unroll
  for (int sp = 0; sp < 4; ++sp)
#pragma unroll
    for (int c = 0; c < 3; ++c) acc[sp][c] = cpx<double>(0.0, 0.0);
  hop_full<double, LS, 0, +1>(g, U, in, x4, s, co, acc);
  hop_full<double, LS, 0, -1>(g, U, in, x4, s, co, acc);
  hop_full<double, LS, 1, +1>(g, U, in, x4, s, co, acc);
  hop_full<double, LS, 1, -1>(g, U, in, x4, s, co, acc);
  hop_full<double, LS, 2, +1>(g, U, in, x4, s, co, acc);
  hop_full<double, LS, 2, -1>(g, U, in, x4, s, co, acc);
  hop_full<double, LS, 3, +1>(g, U, in, x4, s, co, acc);
  hop_full<double, LS, 3, -1>(g, U, in, x4, s, co, acc);
  cpx<double>* o = out + (unsigned)(x4 * 12 * ls + s);
#pragma unroll
  for (int sp = 0; sp < 4; ++sp)
#pragma unroll
    for (int c = 0; c < 3; ++c) st(o + (3 * sp + c) * ls, acc[sp][c]);
}

constexpr int RB_M5 = 0, RB_M5INV = 1, RB_M5_MINUS = 2;  // out = M5 in, M5^{-1} in, M5 in - sub

// one thread per (4d site of parity par, spin-colour component): the run over s
template <int MODE>
__global__ void __launch_bounds__(256) rb_m5_kernel(Geom g, const cpx<double>* __restrict__ in,
                                                    const cpx<double>* __restrict__ sub,
                                                    cpx<double>* __restrict__ out, int par, double a, double mf) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (long long)(g.V4 / 2) * 12) return;
  const int h = (int)(i / 12), c = (int)(i - (long long)h * 12);
  int co[4];
  const int x4 = rb_site(g, h, par, co);
  const int ls = g.Ls;
  const unsigned base = (unsigned)((x4 * 12 + c) * ls);
  const cpx<double>* b = in + base;
  cpx<double>* y = out + base;
  const bool upper = c < 6;  // P_+ components: coupled to s - 1; P_- to s + 1
  if (MODE != RB_M5INV) {
    for (int s = 0; s < ls; ++s) {
      cpx<double> v = a * b[s];
      if (upper) {
        const cpx<double> w = s > 0 ? b[s - 1] : (-mf) * b[ls - 1];
        v = v - w;
      } else {
        const cpx<double> w = s + 1 < ls ? b[s + 1] : (-mf) * b[0];
        v = v - w;
      }
      if (MODE == RB_M5_MINUS) v = v - sub[base + s];
      y[s] = v;
    }
    return;
  }
  // inverse: substitution along the bidiagonal, then the wall corner
  const double ia = 1.0 / a;
  double aLs = 1.0;  // a^{-Ls}
  for (int s = 0; s < ls; ++s) aLs *= ia;
  if (upper) {
    cpx<double> z = ia * b[0];
    y[0] = z;
    for (int s = 1; s < ls; ++s) {
      z = ia * (b[s] + z);
      y[s] = z;
    }
    const double f = mf / (1.0 + mf * aLs);
    const cpx<double> gam = f * z;  // z = z(Ls-1)
    double w = ia;
    for (int s = 0; s < ls; ++s) {
      y[s] = y[s] - w * gam;
      w *= ia;
    }
  } else {
    cpx<double> z = ia * b[ls - 1];
    y[ls - 1] = z;
    for (int s = ls - 2; s >= 0; --s) {
      z = ia * (b[s] + z);
      y[s] = z;
    }
    const double f = mf / (1.0 + mf * aLs);
    const cpx<double> gam = f * z;  // z = z(0)
    double w = ia;
    for (int s = ls - 1; s >= 0; --s) {
      y[s] = y[s] - w * gam;
      w *= ia;
    }
  }
}

// out = in1 + c2 in2 on the sites of parity par (in2 may be null: out = in1 there)
__global__ void rb_lincomb_kernel(Geom g, const cpx<double>* __restrict__ in1, const cpx<double>* __restrict__ in2,
                                  double c2, cpx<double>* __restrict__ out, int par) {
  const long long per = 12LL * g.Ls;
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (long long)(g.V4 / 2) * per) return;
  const int h = (int)(i / per);
  const long long rem = i - (long long)h * per;
  int co[4];
  const int x4 = rb_site(g, h, par, co);
  const long long o = (long long)x4 * per + rem;
  cpx<double> v = in1[o];
  if (in2) {
    const cpx<double> w = in2[o];
    v = cpx<double>(v.re + c2 * w.re, v.im + c2 * w.im);
  }
  out[o] = v;
}

// device scalars of the CG on S^dag S
struct RBDev {
  double rr[2];  // |r|^2 of the current and next iteration (by iteration parity)
  double qq;     // |S p|^2
  double tt;     // |t|^2, t the Schur residual
  double ee;     // |eta|^2
  double pad[3];
};

// x += alpha p; t -= alpha q; r -= alpha Ap with alpha = rr[k] / qq; |r|^2 -> rr[k^1], |t|^2 -> tt
__global__ void __launch_bounds__(RED_THREADS) rb_update_kernel(cpx<double>* __restrict__ x,
                                                                const cpx<double>* __restrict__ p,
                                                                cpx<double>* __restrict__ t,
                                                                const cpx<double>* __restrict__ q,
                                                                cpx<double>* __restrict__ r,
                                                                const cpx<double>* __restrict__ Ap, long long n,
                                                                RBDev* d, int k, RedScratch rs) {
  const double alpha = d->qq > 0.0 ? d->rr[k] / d->qq : 0.0;
  double acc[2] = {0.0, 0.0};
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const cpx<double> pv = p[i], qv = q[i], av = Ap[i];
    cpx<double> xv = x[i], tv = t[i], rv = r[i];
    xv.re += alpha * pv.re;
    xv.im += alpha * pv.im;
    tv.re -= alpha * qv.re;
    tv.im -= alpha * qv.im;
    rv.re -= alpha * av.re;
    rv.im -= alpha * av.im;
    x[i] = xv;
    t[i] = tv;
    r[i] = rv;
    acc[0] = fma(rv.re, rv.re, fma(rv.im, rv.im, acc[0]));
    acc[1] = fma(tv.re, tv.re, fma(tv.im, tv.im, acc[1]));
  }
  double tot[2];
  if (grid_reduce<2>(acc, rs, tot)) {
    d->rr[k ^ 1] = tot[0];
    d->tt = tot[1];
  }
}

// p = r + (rr[k^1] / rr[k]) p
__global__ void rb_p_kernel(const cpx<double>* __restrict__ r, cpx<double>* __restrict__ p, long long n,
                            const RBDev* d, int k) {
  const double beta = d->rr[k] > 0.0 ? d->rr[k ^ 1] / d->rr[k] : 0.0;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const cpx<double> rv = r[i], pv = p[i];
    p[i] = cpx<double>(rv.re + beta * pv.re, rv.im + beta * pv.im);
  }
}

namespace {

struct RBWork {
  void* mem = nullptr;
  cpx<double> *eta, *a, *b2, *xo, *t, *r, *p, *q, *Ap, *g1, *g2;
  RedBuffers rb{};
  RBDev* dev() const { return reinterpret_cast<RBDev*>(rb.scal); }
};

struct RBOp {
  Geom g;
  double a, mf;
  const cpx<double>* U;
  RBWork* w;
  long long n() const { return g.V5 * 12; }

  int hop(const cpx<double>* in, cpx<double>* out, int par, cudaStream_t st) const {
    const long long n = g.V5 / 2;
    HDCR_DISPATCH_LS(g.Ls, (rb_hop_kernel<LSC><<<num_blocks(n, 256), 256, 0, st>>>(g, U, in, out, par)));
    HDCR_LAUNCH_CHECK();
    return HDCR_OK;
  }
  template <int MODE>
  int m5(const cpx<double>* in, const cpx<double>* sub, cpx<double>* out, int par, cudaStream_t st) const {
    const long long n = (long long)(g.V4 / 2) * 12;
    rb_m5_kernel<MODE><<<num_blocks(n, 256), 256, 0, st>>>(g, in, sub, out, par, a, mf);
    count_launch();
    HDCR_LAUNCH_CHECK();
    return HDCR_OK;
  }
  int lincomb(const cpx<double>* in1, const cpx<double>* in2, double c2, cpx<double>* out, int par,
              cudaStream_t st) const {
    const long long n = (long long)(g.V4 / 2) * 12 * g.Ls;
    rb_lincomb_kernel<<<num_blocks(n, 256), 256, 0, st>>>(g, in1, in2, c2, out, par);
    count_launch();
    HDCR_LAUNCH_CHECK();
    return HDCR_OK;
  }
  // out_o = S v_o = M5 v_o - D_oe M5^{-1} D_eo v_o (uses w->a, w->b2 on the even sites)
  int schur(const cpx<double>* v, cpx<double>* out, cudaStream_t st) const {
    HDCR_TRY(hop(v, w->a, 0, st));
    HDCR_TRY(m5<RB_M5INV>(w->a, nullptr, w->b2, 0, st));
    HDCR_TRY(hop(w->b2, w->a, 1, st));
    return m5<RB_M5_MINUS>(v, w->a, out, 1, st);
  }
  // out = S^dag v = Gamma5 S Gamma5 v (uses w->g1, w->g2)
  int schur_dag(const cpx<double>* v, cpx<double>* out, cudaStream_t st) const {
    HDCR_TRY(launch_gamma5_r5<double>(g, v, w->g1, 1, st));
    HDCR_TRY(schur(w->g1, w->g2, st));
    return launch_gamma5_r5<double>(g, w->g2, out, 1, st);
  }
};

}  // namespace

static int rb_solve_impl(const Geom& g, const hdcr_dwf_params* prm, const cpx<double>* U, const cpx<double>* bvec,
                         cpx<double>* x, double tol, int max_iter, hdcr_solve_stats* stats, cudaStream_t st) {
  const auto t0 = std::chrono::steady_clock::now();
  const long long n = g.V5 * 12;
  double* ring = pinned_ring();
  if (!ring) {
    set_error("pinned host buffer unavailable");
    return HDCR_ERR_NO_MEMORY;
  }
  RBWork w;
  const size_t fb = sizeof(cpx<double>) * (size_t)n;
  HDCR_CUDA_TRY(cudaMalloc(&w.mem, fb * 11));
  cpx<double>* base = (cpx<double>*)w.mem;
  cpx<double>** slots[11] = {&w.eta, &w.a, &w.b2, &w.xo, &w.t, &w.r, &w.p, &w.q, &w.Ap, &w.g1, &w.g2};
  for (int i = 0; i < 11; ++i) *slots[i] = base + (size_t)i * n;
  int s = red_buffers_alloc(&w.rb, 8);
  if (s != HDCR_OK) {
    cudaFree(w.mem);
    return s;
  }
  RBOp S{g, 5.0 - prm->M5, prm->mf, U, &w};
  RBDev* d = w.dev();
  RedScratch rs = w.rb.rs;
  const int nb = num_blocks(n, 256, 4096);
  int iters = 0;
  double tr = -1.0, rel = -1.0;
  bool converged = false;
  auto body = [&]() -> int {
    HDCR_CUDA_TRY(cudaMemsetAsync(w.mem, 0, fb * 11, st));
    // eta = Gamma5 b;  t = eta~_o = eta_o - (D_oe M5^{-1} eta_e)_o
    HDCR_TRY(launch_gamma5_r5<double>(g, bvec, w.eta, 1, st));
    HDCR_TRY(launch_norm2<double>(w.eta, n, rs, &d->ee, st));
    HDCR_TRY(S.m5<RB_M5INV>(w.eta, nullptr, w.b2, 0, st));
    HDCR_TRY(S.hop(w.b2, w.a, 1, st));
    HDCR_TRY(S.lincomb(w.eta, w.a, -1.0, w.t, 1, st));
    // r = S^dag t, p = r
    HDCR_TRY(S.schur_dag(w.t, w.r, st));
    HDCR_CUDA_TRY(cudaMemcpyAsync(w.p, w.r, fb, cudaMemcpyDeviceToDevice, st));
    HDCR_TRY(launch_norm2<double>(w.r, n, rs, &d->rr[0], st));
    HDCR_TRY(launch_norm2<double>(w.t, n, rs, &d->tt, st));
    HDCR_CUDA_TRY(cudaMemcpyAsync(ring, &d->tt, 2 * sizeof(double), cudaMemcpyDeviceToHost, st));  // tt, ee
    HDCR_CUDA_TRY(cudaStreamSynchronize(st));
    const double ee = ring[1];
    if (!(ee == ee) || ee > 1e300) {
      set_error("red-black CGNE: non-finite right-hand side");
      return HDCR_ERR_NONFINITE;
    }
    const double stop2 = tol * tol * ee;
    converged = ee == 0.0 || ring[0] <= stop2;
    constexpr int CHECK = 4;
    for (int k = 0; !converged && k < max_iter; ++k) {
      const int par = k & 1;
      HDCR_TRY(S.schur(w.p, w.q, st));
      HDCR_TRY(launch_norm2<double>(w.q, n, rs, &d->qq, st));
      HDCR_TRY(S.schur_dag(w.q, w.Ap, st));
      rb_update_kernel<<<red_blocks(n), RED_THREADS, 0, st>>>(w.xo, w.p, w.t, w.q, w.r, w.Ap, n, d, par, rs);
      count_launch();
      rb_p_kernel<<<nb, 256, 0, st>>>(w.r, w.p, n, d, par);
      count_launch();
      HDCR_LAUNCH_CHECK();
      iters = k + 1;
      if (iters % CHECK == 0 || iters == max_iter) {
        HDCR_CUDA_TRY(cudaMemcpyAsync(ring, &d->tt, sizeof(double), cudaMemcpyDeviceToHost, st));
        HDCR_CUDA_TRY(cudaStreamSynchronize(st));
        if (!(ring[0] == ring[0])) {
          set_error("red-black CGNE: non-finite residual at iteration %d", iters);
          return HDCR_ERR_NONFINITE;
        }
        rel = ee > 0 ? sqrt(ring[0] / ee) : 0.0;
        converged = ring[0] <= stop2;
      }
    }
    // x_e = M5^{-1} (eta_e - D_eo x_o); x = x_o + x_e
    HDCR_TRY(S.hop(w.xo, w.a, 0, st));
    HDCR_TRY(S.lincomb(w.eta, w.a, -1.0, w.g1, 0, st));
    HDCR_TRY(S.m5<RB_M5INV>(w.g1, nullptr, w.b2, 0, st));
    HDCR_CUDA_TRY(cudaMemcpyAsync(x, w.xo, fb, cudaMemcpyDeviceToDevice, st));
    HDCR_TRY(S.lincomb(w.b2, nullptr, 0.0, x, 0, st));
    // true residual |b - H x| / |b|
    FineOp<double> H{g, prm->M5, prm->mf, U};
    HDCR_TRY(true_residual2<double>(H, bvec, x, w.g2, rs, &d->pad[0], st));
    HDCR_CUDA_TRY(cudaMemcpyAsync(ring, &d->pad[0], sizeof(double), cudaMemcpyDeviceToHost, st));
    HDCR_CUDA_TRY(cudaStreamSynchronize(st));
    tr = ee > 0 ? sqrt(ring[0] / ee) : 0.0;
    return HDCR_OK;
  };
  s = body();
  cudaStreamSynchronize(st);
  red_buffers_free(&w.rb);
  cudaFree(w.mem);
  if (s == HDCR_OK && !converged) {
    set_error("red-black CGNE: not converged after %d iterations (|r|/|b| = %g)", iters, rel);
    s = HDCR_ERR_NOT_CONVERGED;
  }
  if (stats) {
    stats->status = s;
    stats->iters = iters;
    // applications of D_dwf's hops, counted in whole-lattice units: S and S^dag take
    // two half-lattice hops each; set-up and reconstruction one each; the true residual one H
    stats->fine_matvecs = 2 * iters + 2;
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

extern "C" int hdcr_cgne_rb_solve(const hdcr_geom* gp, const hdcr_dwf_params* p, const void* U, const void* b,
                                  void* x, double tol, int max_iter, hdcr_solve_stats* stats, void* stream) {
  Geom g;
  HDCR_TRY(make_geom(gp, &g));
  if (!p || !U || !b || !x || b == x || !(tol > 0.0) || max_iter < 1) {
    set_error("hdcr_cgne_rb_solve: bad pointer, tol or max_iter");
    return HDCR_ERR_BAD_ARG;
  }
  for (int mu = 0; mu < 4; ++mu)
    if (g.L[mu] % 2) {
      set_error("hdcr_cgne_rb_solve: every extent must be even (L[%d] = %d)", mu, g.L[mu]);
      return HDCR_ERR_BAD_GEOMETRY;
    }
  if (!(5.0 - p->M5 != 0.0)) {
    set_error("hdcr_cgne_rb_solve: M5 = 5 makes the site-local part singular");
    return HDCR_ERR_BAD_ARG;
  }
  return rb_solve_impl(g, p, (const cpx<double>*)U, (const cpx<double>*)b, (cpx<double>*)x, tol, max_iter, stats,
                       as_stream(stream));
}
