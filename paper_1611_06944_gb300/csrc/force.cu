// Gauge-link force of a solve through H = Gamma5 D_dwf (the gradient the
// paper does not write down).  With H x = b, H y = eta and w = Gamma5 y, the
// loss Re(eta^dag x) changes by dL = Re sum_{x,mu} tr(dU_mu(x) F_mu(x)) with
//
//   F_mu(x) = 1/2 sum_s [ B + C^dag ],
//   B_ba = sum_alpha [(1 - gamma_mu) x(x+mu, s)]_{alpha b} conj(w(x, s)_{alpha a}),
//   C_ba = sum_alpha [(1 + gamma_mu) x(x, s)]_{alpha b}    conj(w(x+mu, s)_{alpha a}),
//
// the t-boundary phase entering through x(x+mu) and w(x+mu).
// One thread per link (mu, x4) sums over s and spin.  With GRAD the kernel
// stores the gradient of the loss with respect to the link instead:
// conj(F_ba) at [a][b], i.e. dL/dRe U_ab + i dL/dIm U_ab.
#include "dwf_stencil.cuh"
#include "host_io.cuh"

namespace hdcr {

// (1 - SG gamma_mu) psi for the spinor at p (component c at p + c*ls), chiral basis
template <typename R>
__device__ __forceinline__ void proj_full(const cpx<R>* __restrict__ p, int ls, int mu, int sg,
                                          cpx<R> (&o)[4][3]) {
  cpx<R> u0[3], u1[3], d0[3], d1[3];
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    u0[c] = ld(p + (0 + c) * ls);
    u1[c] = ld(p + (3 + c) * ls);
    d0[c] = ld(p + (6 + c) * ls);
    d1[c] = ld(p + (9 + c) * ls);
  }
  // gamma_mu psi = (G d, G^dag... ) written out per direction:
  //   gamma_k: upper = -i sigma_k d, lower = +i sigma_k u;  gamma_t: upper = d, lower = u
  cpx<R> gu0[3], gu1[3], gd0[3], gd1[3];
  if (mu == 3) {
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      gu0[c] = d0[c];
      gu1[c] = d1[c];
      gd0[c] = u0[c];
      gd1[c] = u1[c];
    }
  } else {
    cpx<R> a0[3], a1[3], b0[3], b1[3];
    if (mu == 0) {
      i_sigma<R, 0>(d0, d1, a0, a1);
      i_sigma<R, 0>(u0, u1, b0, b1);
    } else if (mu == 1) {
      i_sigma<R, 1>(d0, d1, a0, a1);
      i_sigma<R, 1>(u0, u1, b0, b1);
    } else {
      i_sigma<R, 2>(d0, d1, a0, a1);
      i_sigma<R, 2>(u0, u1, b0, b1);
    }
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      gu0[c] = cpx<R>(-a0[c].re, -a0[c].im);
      gu1[c] = cpx<R>(-a1[c].re, -a1[c].im);
      gd0[c] = b0[c];
      gd1[c] = b1[c];
    }
  }
  const R s = (R)sg;
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    o[0][c] = cpx<R>(u0[c].re - s * gu0[c].re, u0[c].im - s * gu0[c].im);
    o[1][c] = cpx<R>(u1[c].re - s * gu1[c].re, u1[c].im - s * gu1[c].im);
    o[2][c] = cpx<R>(d0[c].re - s * gd0[c].re, d0[c].im - s * gd0[c].im);
    o[3][c] = cpx<R>(d1[c].re - s * gd1[c].re, d1[c].im - s * gd1[c].im);
  }
}

template <typename R, bool GRAD>
__global__ void __launch_bounds__(128) force_kernel(Geom g, const cpx<R>* __restrict__ x,
                                                    const cpx<R>* __restrict__ w, cpx<R>* __restrict__ F) {
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= 4LL * g.V4) return;
  const int mu = (int)(idx / g.V4);
  const int x4 = (int)(idx - (long long)mu * g.V4);
  int co[4];
  x4_coords(g, x4, co);
  int nc[4] = {co[0], co[1], co[2], co[3]};
  R ph = (R)1;
  nc[mu] = co[mu] + 1;
  if (nc[mu] == g.L[mu]) {
    nc[mu] = 0;
    if (mu == 3) ph = (R)g.bc_t;
  }
  const int y4 = x4_index(g, nc);
  const int ls = g.Ls;
  double acc[3][3][2];
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int b = 0; b < 3; ++b) acc[a][b][0] = acc[a][b][1] = 0.0;
  for (int s = 0; s < ls; ++s) {
    const cpx<R>* xs = x + (unsigned)(x4 * 12 * ls + s);
    const cpx<R>* xf = x + (unsigned)(y4 * 12 * ls + s);
    const cpx<R>* ws = w + (unsigned)(x4 * 12 * ls + s);
    const cpx<R>* wf = w + (unsigned)(y4 * 12 * ls + s);
    cpx<R> h[4][3], q[4][3];
    proj_full<R>(xf, ls, mu, +1, h);  // (1 - gamma_mu) x(x+mu)
    proj_full<R>(xs, ls, mu, -1, q);  // (1 + gamma_mu) x(x)
#pragma unroll
    for (int al = 0; al < 4; ++al) {
      cpx<R> wv[3], wfv[3];
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        wv[c] = ld(ws + (3 * al + c) * ls);
        wfv[c] = ld(wf + (3 * al + c) * ls);
      }
#pragma unroll
      for (int b = 0; b < 3; ++b)
#pragma unroll
        for (int a = 0; a < 3; ++a) {
          // B_ba += h_{al b} conj(w_{al a});  (C^dag)_ba = conj(C_ab) += conj(q_{al a}) w(x+mu)_{al b}
          const cpx<R> hb = h[al][b], wa = wv[a], qa = q[al][a], wb = wfv[b];
          acc[b][a][0] += (double)hb.re * wa.re + (double)hb.im * wa.im + (double)qa.re * wb.re +
                          (double)qa.im * wb.im;
          acc[b][a][1] += (double)hb.im * wa.re - (double)hb.re * wa.im + (double)qa.re * wb.im -
                          (double)qa.im * wb.re;
        }
    }
  }
  cpx<R>* out = F + (long long)idx * 9;
  const double sc = 0.5 * (double)ph;
#pragma unroll
  for (int b = 0; b < 3; ++b)
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      if (GRAD)
        st(out + 3 * a + b, cpx<R>((R)(sc * acc[b][a][0]), (R)(-sc * acc[b][a][1])));
      else
        st(out + 3 * b + a, cpx<R>((R)(sc * acc[b][a][0]), (R)(sc * acc[b][a][1])));
    }
}

template <typename R, bool GRAD>
int launch_force(const Geom& g, const void* x, const void* w, void* F, cudaStream_t st) {
  const long long n = 4LL * g.V4;
  force_kernel<R, GRAD><<<num_blocks(n, 128), 128, 0, st>>>(g, (const cpx<R>*)x, (const cpx<R>*)w, (cpx<R>*)F);
  count_launch();
  HDCR_LAUNCH_CHECK();
  return HDCR_OK;
}

}  // namespace hdcr

using namespace hdcr;

template <bool GRAD>
static int gauge_force_call(const char* name, const hdcr_geom* gp, const void* x, const void* w, void* F,
                            int dtype, void* stream) {
  Geom g;
  HDCR_TRY(make_geom(gp, &g));
  if (!x || !w || !F) {
    set_error("%s: null pointer", name);
    return HDCR_ERR_BAD_ARG;
  }
  const size_t cb = dtype_complex_bytes(dtype);
  if (!cb) {
    set_error("%s: unknown dtype %d", name, dtype);
    return HDCR_ERR_BAD_ARG;
  }
  // fields given in host memory are staged through the device
  cudaStream_t st = as_stream(stream);
  Staged sx, sw, sf;
  HDCR_TRY(sx.in(x, (size_t)g.V5 * 12 * cb, st));
  HDCR_TRY(sw.in(w, (size_t)g.V5 * 12 * cb, st));
  HDCR_TRY(sf.out(F, (size_t)g.V4 * 36 * cb, st, false));
  if (dtype == HDCR_C128)
    HDCR_TRY((launch_force<double, GRAD>(g, sx.ptr(), sw.ptr(), sf.ptr(), st)));
  else
    HDCR_TRY((launch_force<float, GRAD>(g, sx.ptr(), sw.ptr(), sf.ptr(), st)));
  return sf.finish();
}

extern "C" int hdcr_gauge_force(const hdcr_geom* gp, const void* x, const void* w, void* F, int dtype,
                                void* stream) {
  return gauge_force_call<false>("hdcr_gauge_force", gp, x, w, F, dtype, stream);
}

extern "C" int hdcr_gauge_grad(const hdcr_geom* gp, const void* x, const void* w, void* G, int dtype,
                               void* stream) {
  return gauge_force_call<true>("hdcr_gauge_grad", gp, x, w, G, dtype, stream);
}
