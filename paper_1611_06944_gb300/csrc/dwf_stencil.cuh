// Per-site body of the domain-wall stencil, shared by the plain operator
// kernel and the fused solver kernels.
//
//   (D_dwf psi)(x,s) = (5 - M5) psi(x,s)
//        - 1/2 sum_mu [(1 - gamma_mu) U_mu(x) psi(x+mu,s) + (1 + gamma_mu) U_mu(x-mu)^dag psi(x-mu,s)]
//        - P_- psi(x,s+1) - P_+ psi(x,s-1),   psi(Ls) = -mf psi(0), psi(-1) = -mf psi(Ls-1)
//   (H psi)(x,s) = gamma5 (D_dwf psi)(x, Ls-1-s)                     (Section 3)
//
// Chiral basis: psi = (u, d) with u = spins 0,1 and d = spins 2,3.
//   (1 - gamma_k) psi = (h, -i sigma_k h),  h = u + i sigma_k d   (k = x, y, z)
//   (1 + gamma_k) psi = (h, +i sigma_k h),  h = u - i sigma_k d
//   (1 - gamma_t) psi = (h, -h),            h = u - d
//   (1 + gamma_t) psi = (h, +h),            h = u + d
// so each hop multiplies only the two components of h by the link.
//
// Field layout psi[x4][c][s] (see hdcr_internal.cuh): a pointer to component 0
// of site (x4, s) reaches component c at offset c*Ls.  The Ls template
// parameter LS makes those offsets immediates (LS = 0: runtime Ls).
#pragma once

#include "hdcr_internal.cuh"

namespace hdcr {

template <int LS>
__device__ __forceinline__ int ls_of(const Geom& g) {
  return LS > 0 ? LS : g.Ls;
}

// (o0, o1) = i sigma_K (w0, w1) for colour vectors w0, w1
template <typename R, int K>
__device__ __forceinline__ void i_sigma(const cpx<R> (&w0)[3], const cpx<R> (&w1)[3], cpx<R> (&o0)[3],
                                        cpx<R> (&o1)[3]) {
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    if (K == 0) {
      o0[c] = times_i(w1[c]);
      o1[c] = times_i(w0[c]);
    } else if (K == 1) {
      o0[c] = w1[c];
      o1[c] = cpx<R>(-w0[c].re, -w0[c].im);
    } else {
      o0[c] = times_i(w0[c]);
      o1[c] = cpx<R>(w1[c].im, -w1[c].re);
    }
  }
}

// neighbour x4 index and boundary phase for the hop x -> x + SIGN*mu
template <int MU, int SIGN>
__device__ __forceinline__ int neighbour(const Geom& g, const int co[4], int* phase) {
  int nc[4] = {co[0], co[1], co[2], co[3]};
  *phase = 1;
  if (SIGN > 0) {
    nc[MU] = co[MU] + 1;
    if (nc[MU] == g.L[MU]) {
      nc[MU] = 0;
      if (MU == 3) *phase = g.bc_t;
    }
  } else {
    nc[MU] = co[MU] - 1;
    if (nc[MU] < 0) {
      nc[MU] = g.L[MU] - 1;
      if (MU == 3) *phase = g.bc_t;
    }
  }
  return x4_index(g, nc);
}

// acc += coef * [(1 -+ gamma_mu) U psi(nbr)] for the hop (MU, SIGN); nb points at
// component 0 of the neighbour site, Ul at the link (U_mu(x) for SIGN > 0,
// U_mu(x-mu), used as its adjoint, for SIGN < 0)
template <typename R, int MU, int SIGN>
__device__ __forceinline__ void wilson_hop(const cpx<R>* __restrict__ Ul, const cpx<R>* __restrict__ nb, int ls,
                                           R coef, cpx<R> (&acc)[4][3]) {
  cpx<R> h[2][3];
  {
    cpx<R> u0[3], u1[3], d0[3], d1[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      u0[c] = ld(nb + (0 + c) * ls);
      u1[c] = ld(nb + (3 + c) * ls);
      d0[c] = ld(nb + (6 + c) * ls);
      d1[c] = ld(nb + (9 + c) * ls);
    }
    if (MU == 3) {
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        h[0][c] = SIGN > 0 ? u0[c] - d0[c] : u0[c] + d0[c];
        h[1][c] = SIGN > 0 ? u1[c] - d1[c] : u1[c] + d1[c];
      }
    } else {
      cpx<R> t0[3], t1[3];
      i_sigma<R, MU>(d0, d1, t0, t1);
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        h[0][c] = SIGN > 0 ? u0[c] + t0[c] : u0[c] - t0[c];
        h[1][c] = SIGN > 0 ? u1[c] + t1[c] : u1[c] - t1[c];
      }
    }
  }
  cpx<R> m[3][3];
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int b = 0; b < 3; ++b) m[a][b] = ld(Ul + 3 * a + b);
  cpx<R> hp[2][3];
#pragma unroll
  for (int sp = 0; sp < 2; ++sp)
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      cpx<R> t((R)0, (R)0);
#pragma unroll
      for (int b = 0; b < 3; ++b) {
        if (SIGN > 0)
          t = cmadd(t, m[a][b], h[sp][b]);
        else
          t = cjmadd(t, m[b][a], h[sp][b]);
      }
      hp[sp][a] = t;
    }
  cpx<R> lo[2][3];
  if (MU == 3) {
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      lo[0][c] = hp[0][c];
      lo[1][c] = hp[1][c];
    }
  } else {
    i_sigma<R, MU>(hp[0], hp[1], lo[0], lo[1]);
  }
  // lower = -lo for (1 - gamma), +lo for (1 + gamma)
  const R cl = SIGN > 0 ? -coef : coef;
#pragma unroll
  for (int sp = 0; sp < 2; ++sp)
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      acc[sp][c].re = fma(coef, hp[sp][c].re, acc[sp][c].re);
      acc[sp][c].im = fma(coef, hp[sp][c].im, acc[sp][c].im);
      acc[2 + sp][c].re = fma(cl, lo[sp][c].re, acc[2 + sp][c].re);
      acc[2 + sp][c].im = fma(cl, lo[sp][c].im, acc[2 + sp][c].im);
    }
}

template <typename R, int LS, int MU, int SIGN>
__device__ __forceinline__ void hop_full(const Geom& g, const cpx<R>* __restrict__ U,
                                         const cpx<R>* __restrict__ in, int x4, int s, const int co[4],
                                         cpx<R> (&acc)[4][3]) {
  int ph;
  const int ls = ls_of<LS>(g);
  const int y4 = neighbour<MU, SIGN>(g, co, &ph);
  const cpx<R>* Ul = U + (unsigned)((MU * g.V4 + (SIGN > 0 ? x4 : y4)) * 9);
  const cpx<R>* nb = in + (unsigned)(y4 * 12 * ls + s);
  wilson_hop<R, MU, SIGN>(Ul, nb, ls, (R)(-0.5 * ph), acc);
}

// The diagonal and fifth-dimension part: acc = (5 - M5) psi(x,s) - P_- psi(x,s+1) - P_+ psi(x,s-1).
// self points at component 0 of site (x4, s).
template <typename R, int LS>
__device__ __forceinline__ void local_part(const Geom& g, R diag, R mf, const cpx<R>* __restrict__ self, int s,
                                           cpx<R> (&acc)[4][3]) {
  const int ls = ls_of<LS>(g);
#pragma unroll
  for (int sp = 0; sp < 4; ++sp)
#pragma unroll
    for (int c = 0; c < 3; ++c) acc[sp][c] = diag * ld(self + (3 * sp + c) * ls);
  {
    const bool wall = (s + 1 == ls);
    const cpx<R>* p = wall ? self - (ls - 1) : self + 1;
    const R w = wall ? -mf : (R)1;
#pragma unroll
    for (int sp = 2; sp < 4; ++sp)
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        cpx<R> v = ld(p + (3 * sp + c) * ls);
        acc[sp][c].re = fma(-w, v.re, acc[sp][c].re);
        acc[sp][c].im = fma(-w, v.im, acc[sp][c].im);
      }
  }
  {
    const bool wall = (s == 0);
    const cpx<R>* p = wall ? self + (ls - 1) : self - 1;
    const R w = wall ? -mf : (R)1;
#pragma unroll
    for (int sp = 0; sp < 2; ++sp)
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        cpx<R> v = ld(p + (3 * sp + c) * ls);
        acc[sp][c].re = fma(-w, v.re, acc[sp][c].re);
        acc[sp][c].im = fma(-w, v.im, acc[sp][c].im);
      }
  }
}

// acc = (D_dwf psi)(x4, s) for the 5d site (x4, s)
template <typename R, int LS>
__device__ __forceinline__ void dwf_site(const Geom& g, R diag, R mf, const cpx<R>* __restrict__ U,
                                         const cpx<R>* __restrict__ in, int x4, int s, cpx<R> (&acc)[4][3]) {
  const int ls = ls_of<LS>(g);
  int co[4];
  x4_coords(g, x4, co);
  local_part<R, LS>(g, diag, mf, in + (unsigned)(x4 * 12 * ls + s), s, acc);
  hop_full<R, LS, 0, +1>(g, U, in, x4, s, co, acc);
  hop_full<R, LS, 0, -1>(g, U, in, x4, s, co, acc);
  hop_full<R, LS, 1, +1>(g, U, in, x4, s, co, acc);
  hop_full<R, LS, 1, -1>(g, U, in, x4, s, co, acc);
  hop_full<R, LS, 2, +1>(g, U, in, x4, s, co, acc);
  hop_full<R, LS, 2, -1>(g, U, in, x4, s, co, acc);
  hop_full<R, LS, 3, +1>(g, U, in, x4, s, co, acc);
  hop_full<R, LS, 3, -1>(g, U, in, x4, s, co, acc);
}

// out(x4, Ls-1-s) = gamma5 acc
template <typename R, int LS>
__device__ __forceinline__ void store_g5r5(const Geom& g, cpx<R>* __restrict__ out, int x4, int s,
                                           const cpx<R> (&acc)[4][3]) {
  const int ls = ls_of<LS>(g);
  cpx<R>* o = out + (unsigned)(x4 * 12 * ls + (ls - 1 - s));
#pragma unroll
  for (int sp = 0; sp < 4; ++sp)
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      cpx<R> v = acc[sp][c];
      if (sp >= 2) v = cpx<R>(-v.re, -v.im);
      st(o + (3 * sp + c) * ls, v);
    }
}

// Dispatch a kernel template on the fifth-dimension extent: LS = 16, 8 or runtime.
#define HDCR_DISPATCH_LS(ls, KERNEL_CALL) \
  do {                                    \
    if ((ls) == 16) {                     \
      constexpr int LSC = 16;             \
      KERNEL_CALL;                        \
      count_launch();                     \
    } else if ((ls) == 8) {               \
      constexpr int LSC = 8;              \
      KERNEL_CALL;                        \
      count_launch();                     \
    } else {                              \
      constexpr int LSC = 0;              \
      KERNEL_CALL;                        \
      count_launch();                     \
    }                                     \
  } while (0)

}  // namespace hdcr
