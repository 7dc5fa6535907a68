// Chebyshev polynomials of H^2 (Section 4 and Fig. 1):
//
//  * smoother  S r = H p(H^2) r, p the truncated Chebyshev series of 1/y on
//    [lo, hi] ("an order 10 Chebyshev polynomial approximation to 1/x in the
//    range [1.0, 64.0]"; the interval is read as one for y = H^2, whose top
//    edge lambda_max(H)^2 is about 64);
//  * filter    T_n(t(H^2)) x, t mapping [lam_cut^2, lam_max^2] onto [-1, 1]:
//    the low-pass filter applied to Gaussian noise to build the subspace.
//
// Both run the three-term recurrence T_{k+1} = 2 t T_k - T_{k-1} on vectors;
// one fused kernel per step forms T_{k+1} from H^2 T_k and accumulates the
// series, so a step costs two stencil launches and one BLAS pass.
#include <math.h>

#include <vector>

#include "chebyshev.cuh"

namespace hdcr {

std::vector<double> cheb_inverse_coeffs(double lo, double hi, int order) {
  // c_k = (2/m) sum_j f(y_j) cos(k theta_j), theta_j = pi (j + 1/2) / m, m = 4 (order + 1)
  const int m = 4 * (order + 1);
  std::vector<double> c(order + 1, 0.0);
  for (int j = 0; j < m; ++j) {
    const double th = M_PI * (j + 0.5) / m;
    const double y = 0.5 * (hi + lo) + 0.5 * (hi - lo) * cos(th);
    const double f = 1.0 / y;
    for (int k = 0; k <= order; ++k) c[k] += f * cos(k * th);
  }
  for (int k = 0; k <= order; ++k) c[k] *= 2.0 / m;
  return c;
}

// next = 2 (a w + b cur) - prev (written over prev);  acc = acc0 * acc + ck * next
template <typename R>
__global__ void cheb_step_kernel(const cpx<R>* __restrict__ w, const cpx<R>* __restrict__ cur,
                                 cpx<R>* __restrict__ prev, cpx<R>* __restrict__ acc, long long n, R a, R b,
                                 R ck, int with_acc) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const cpx<R> wv = ld(w + i), cv = ld(cur + i), pv = ld(prev + i);
    cpx<R> nx;
    nx.re = (R)2 * fma(a, wv.re, b * cv.re) - pv.re;
    nx.im = (R)2 * fma(a, wv.im, b * cv.im) - pv.im;
    st(prev + i, nx);
    if (with_acc) {
      cpx<R> av = ld(acc + i);
      av.re = fma(ck, nx.re, av.re);
      av.im = fma(ck, nx.im, av.im);
      st(acc + i, av);
    }
  }
}

// cur = a w + b v (first step, T_1);  acc = c0/2 v + c1 cur
template <typename R>
__global__ void cheb_first_kernel(const cpx<R>* __restrict__ w, const cpx<R>* __restrict__ v,
                                  cpx<R>* __restrict__ cur, cpx<R>* __restrict__ acc, long long n, R a, R b,
                                  R c0h, R c1, int with_acc) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const cpx<R> wv = ld(w + i), vv = ld(v + i);
    cpx<R> t;
    t.re = fma(a, wv.re, b * vv.re);
    t.im = fma(a, wv.im, b * vv.im);
    st(cur + i, t);
    if (with_acc) {
      cpx<R> av;
      av.re = fma(c1, t.re, c0h * vv.re);
      av.im = fma(c1, t.im, c0h * vv.im);
      st(acc + i, av);
    }
  }
}

// u *= 1/sqrt(*n2), v *= 1/sqrt(*n2)
template <typename R>
__global__ void rescale2_kernel(cpx<R>* __restrict__ u, cpx<R>* __restrict__ v, long long n, const double* n2) {
  const R s = (R)(*n2 > 0.0 ? 1.0 / sqrt(*n2) : 1.0);
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const cpx<R> a = ld(u + i);
    st(u + i, cpx<R>(s * a.re, s * a.im));
    if (v) {
      const cpx<R> c = ld(v + i);
      st(v + i, cpx<R>(s * c.re, s * c.im));
    }
  }
}

template <typename R>
int cheb_work_alloc(ChebWork<R>* w, long long n) {
  void* p = nullptr;
  cudaError_t e = cudaMalloc(&p, sizeof(cpx<R>) * n * 4 + 256);
  if (e != cudaSuccess) return cuda_status(e, "Chebyshev workspace");
  w->t0 = (cpx<R>*)p;
  w->t1 = w->t0 + n;
  w->h1 = w->t1 + n;
  w->h2 = w->h1 + n;
  w->n2 = (double*)(w->h2 + n);
  return HDCR_OK;
}

template <typename R>
void cheb_work_free(ChebWork<R>* w) {
  if (w->t0) cudaFree(w->t0);
  w->t0 = nullptr;
}

template <typename R>
int cheb_smoother(const FineOp<R>& H, const cpx<R>* r, cpx<R>* out, const std::vector<double>& c, double lo,
                  double hi, ChebWork<R>& w, cudaStream_t st, int* matvecs) {
  const long long n = H.n();
  const int nb = num_blocks(n, 256, 4096);
  const int order = (int)c.size() - 1;
  const R a = (R)(2.0 / (hi - lo)), b = (R)(-(hi + lo) / (hi - lo));
  // v = H r (held in t0 = T_0 v)
  HDCR_TRY(H.apply(r, w.t0, st));
  int mv = 1;
  if (order == 0) {
    rescale_copy(w.t0, out, n, (R)(0.5 * c[0]), st);
    *matvecs += mv;
    return HDCR_OK;
  }
  // T_1 v = t(H^2) v
  HDCR_TRY(H.apply(w.t0, w.h1, st));
  HDCR_TRY(H.apply(w.h1, w.h2, st));
  mv += 2;
  cheb_first_kernel<R><<<nb, 256, 0, st>>>(w.h2, w.t0, w.t1, out, n, a, b, (R)(0.5 * c[0]), (R)c[1], 1); count_launch();
  HDCR_LAUNCH_CHECK();
  cpx<R>* prev = w.t0;
  cpx<R>* cur = w.t1;
  for (int k = 2; k <= order; ++k) {
    HDCR_TRY(H.apply(cur, w.h1, st));
    mv += 2;
    if constexpr (sizeof(R) == 8) {
      if (!H.cf && H.nrhs == 1) {  // the step fused into the second application (domain-wall FP64)
        HDCR_TRY(launch_g5dwf_cheb(H.g, H.M5, H.mf, (const cpx<double>*)H.U, (const cpx<double>*)w.h1,
                                   (const cpx<double>*)cur, (cpx<double>*)prev, (cpx<double>*)out, (double)a,
                                   (double)b, c[k], st));
        cpx<R>* t = prev;
        prev = cur;
        cur = t;
        continue;
      }
    } else {
      if (!H.cf && g5dwf_x2_ok(H.g, w.h1, prev) && g5dwf_x2_ok(H.g, cur, out)) {  // the same in FP32
        int slot;
        stencil_timer_begin(1, H.g.V5 * H.nrhs, st, &slot);
        const int s = launch_g5dwf_x2_cheb(H.g, H.M5, H.mf, (const cpx<float>*)H.U, (const cpx<float>*)w.h1,
                                           (const cpx<float>*)cur, (cpx<float>*)prev, (float)a, (float)b, H.nrhs,
                                           st, (cpx<float>*)out, (float)c[k]);
        stencil_timer_end(slot, st);
        HDCR_TRY(s);
        cpx<R>* t = prev;
        prev = cur;
        cur = t;
        continue;
      }
    }
    HDCR_TRY(H.apply(w.h1, w.h2, st));
    cheb_step_kernel<R><<<nb, 256, 0, st>>>(w.h2, cur, prev, out, n, a, b, (R)c[k], 1); count_launch();
    HDCR_LAUNCH_CHECK();
    cpx<R>* t = prev;
    prev = cur;
    cur = t;
  }
  *matvecs += mv;
  return HDCR_OK;
}

template <typename R>
__global__ void scale_copy_kernel(const cpx<R>* __restrict__ in, cpx<R>* __restrict__ out, long long n, R s) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const cpx<R> v = ld(in + i);
    st(out + i, cpx<R>(s * v.re, s * v.im));
  }
}

template <typename R>
void rescale_copy(const cpx<R>* in, cpx<R>* out, long long n, R s, cudaStream_t st) {
  scale_copy_kernel<R><<<num_blocks(n, 256, 4096), 256, 0, st>>>(in, out, n, s); count_launch();
}

template <typename R>
int cheb_filter(const FineOp<R>& H, cpx<R>* x, int order, double lam_cut, double lam_max, ChebWork<R>& w,
                RedScratch rs, cudaStream_t st) {
  const long long n = H.n();
  const int nb = num_blocks(n, 256, 4096);
  const double lo = lam_cut * lam_cut, hi = lam_max * lam_max;
  const R a = (R)(2.0 / (hi - lo)), b = (R)(-(hi + lo) / (hi - lo));
  // T_0 = x (copy into t0), T_1 = t(H^2) x
  rescale_copy(x, w.t0, n, (R)1, st);
  HDCR_TRY(H.apply(w.t0, w.h1, st));
  HDCR_TRY(H.apply(w.h1, w.h2, st));
  cheb_first_kernel<R><<<nb, 256, 0, st>>>(w.h2, w.t0, w.t1, nullptr, n, a, b, (R)0, (R)0, 0); count_launch();
  HDCR_LAUNCH_CHECK();
  cpx<R>* prev = w.t0;
  cpx<R>* cur = w.t1;
  for (int k = 2; k <= order; ++k) {
    HDCR_TRY(H.apply(cur, w.h1, st));
    HDCR_TRY(H.apply(w.h1, w.h2, st));
    cheb_step_kernel<R><<<nb, 256, 0, st>>>(w.h2, cur, prev, nullptr, n, a, b, (R)0, 0); count_launch();
    HDCR_LAUNCH_CHECK();
    cpx<R>* t = prev;
    prev = cur;
    cur = t;
    if (k % 8 == 0) {  // keep the growing recurrence in range: common rescale of both terms
      HDCR_TRY(launch_norm2<R>(cur, n, rs, w.n2, st));
      rescale2_kernel<R><<<nb, 256, 0, st>>>(cur, prev, n, w.n2); count_launch();
      HDCR_LAUNCH_CHECK();
    }
  }
  HDCR_TRY(launch_norm2<R>(cur, n, rs, w.n2, st));
  rescale2_kernel<R><<<nb, 256, 0, st>>>(cur, (cpx<R>*)nullptr, n, w.n2); count_launch();
  HDCR_LAUNCH_CHECK();
  rescale_copy(cur, x, n, (R)1, st);
  return HDCR_OK;
}

template <typename R>
int cheb_filter_multi(const FineOp<R>& H, cpx<R>* x, int nrhs, int order, double lam_cut, double lam_max,
                      cpx<R>* work, double* n2, RedScratch rs, cudaStream_t st) {
  const long long n = H.n(), N = n * nrhs;
  const int nb = num_blocks(N, 256, 8192);
  const double lo = lam_cut * lam_cut, hi = lam_max * lam_max;
  const R a = (R)(2.0 / (hi - lo)), b = (R)(-(hi + lo) / (hi - lo));
  cpx<R>* t0 = work;
  cpx<R>* t1 = work + N;
  cpx<R>* h1 = work + 2 * N;
  cpx<R>* h2 = work + 3 * N;  // the unfused path only
  bool fused = false;
  if constexpr (sizeof(R) == 4) fused = g5dwf_x2_ok(H.g, x, work) && g5dwf_x2_ok(H.g, work + N, work + 2 * N);
  const void* U = H.U;
  // T_0 = x, T_1 = a H^2 x + b x
  rescale_copy(x, t0, N, (R)1, st);
  HDCR_TRY(launch_g5dwf<R>(H.g, H.M5, H.mf, U, t0, h1, nrhs, st));
  if (fused) {
    HDCR_CUDA_TRY(cudaMemsetAsync(t1, 0, sizeof(cpx<R>) * N, st));
    HDCR_TRY(launch_g5dwf_x2_cheb(H.g, H.M5, H.mf, (const cpx<float>*)U, (const cpx<float>*)h1,
                                  (const cpx<float>*)t0, (cpx<float>*)t1, (float)(0.5 * a), (float)(0.5 * b), nrhs,
                                  st));
  } else {
    HDCR_TRY(launch_g5dwf<R>(H.g, H.M5, H.mf, U, h1, h2, nrhs, st));
    cheb_first_kernel<R><<<nb, 256, 0, st>>>(h2, t0, t1, nullptr, N, a, b, (R)0, (R)0, 0); count_launch();
    HDCR_LAUNCH_CHECK();
  }
  cpx<R>* prev = t0;
  cpx<R>* cur = t1;
  for (int k = 2; k <= order; ++k) {
    // T_k = 2 t(H^2) T_{k-1} - T_{k-2}, written over T_{k-2}
    HDCR_TRY(launch_g5dwf<R>(H.g, H.M5, H.mf, U, cur, h1, nrhs, st));
    if (fused) {
      HDCR_TRY(launch_g5dwf_x2_cheb(H.g, H.M5, H.mf, (const cpx<float>*)U, (const cpx<float>*)h1,
                                    (const cpx<float>*)cur, (cpx<float>*)prev, (float)a, (float)b, nrhs, st));
    } else {
      HDCR_TRY(launch_g5dwf<R>(H.g, H.M5, H.mf, U, h1, h2, nrhs, st));
      cheb_step_kernel<R><<<nb, 256, 0, st>>>(h2, cur, prev, nullptr, N, a, b, (R)0, 0); count_launch();
      HDCR_LAUNCH_CHECK();
    }
    cpx<R>* t = prev;
    prev = cur;
    cur = t;
    if (k % 8 == 0) {  // keep the growing recurrence in range: one common rescale of both terms
      HDCR_TRY(launch_norm2<R>(cur, N, rs, n2, st));
      rescale2_kernel<R><<<nb, 256, 0, st>>>(cur, prev, N, n2); count_launch();
      HDCR_LAUNCH_CHECK();
    }
  }
  HDCR_TRY(launch_norm2<R>(cur, N, rs, n2, st));
  rescale2_kernel<R><<<nb, 256, 0, st>>>(cur, (cpx<R>*)nullptr, N, n2); count_launch();
  HDCR_LAUNCH_CHECK();
  rescale_copy(cur, x, N, (R)1, st);
  return HDCR_OK;
}

#define HDCR_INST_CHEB(R)                                                                            \
  template int cheb_work_alloc<R>(ChebWork<R>*, long long);                                         \
  template int cheb_filter_multi<R>(const FineOp<R>&, cpx<R>*, int, int, double, double, cpx<R>*, double*,  \
                                    RedScratch, cudaStream_t);                                      \
  template void cheb_work_free<R>(ChebWork<R>*);                                                    \
  template int cheb_smoother<R>(const FineOp<R>&, const cpx<R>*, cpx<R>*, const std::vector<double>&, \
                                double, double, ChebWork<R>&, cudaStream_t, int*);                  \
  template int cheb_filter<R>(const FineOp<R>&, cpx<R>*, int, double, double, ChebWork<R>&,         \
                              RedScratch, cudaStream_t);                                            \
  template void rescale_copy<R>(const cpx<R>*, cpx<R>*, long long, R, cudaStream_t);
HDCR_INST_CHEB(double)
HDCR_INST_CHEB(float)

}  // namespace hdcr
