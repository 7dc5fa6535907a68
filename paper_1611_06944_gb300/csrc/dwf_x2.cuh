// The two-site hop of the packed FP32 operator (Section 3's hopping term), shared
// by the FP32 kernel (dwf_x2.cu) and the FP16-storage kernel (dwf_h16.cu): the
// pair of fifth-dimension sites (s, s+1) of one 4d site in two float2 lanes,
// the spin projection, the SU(3) multiply on the packed FP32 pipe and the
// accumulation into the upper / Gamma5-signed lower spins.
#pragma once

#include "dwf_stencil.cuh"

namespace hdcr {

struct cx2 {
  float2 re, im;  // lanes: sites s and s+1
};

__device__ __forceinline__ float2 f2(float a) { return make_float2(a, a); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 sub2(float2 a, float2 b) { return __ffma2_rn(b, make_float2(-1.f, -1.f), a); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }

__device__ __forceinline__ float4 ld4(const cpx<float>* p) { return __ldg(reinterpret_cast<const float4*>(p)); }

// a + S b and a + S i b for the pair (a, b given as two consecutive complex numbers)
template <int S>
__device__ __forceinline__ cx2 comb(float4 a, float4 b) {
  cx2 h;
  h.re = make_float2(a.x + S * b.x, a.z + S * b.z);
  h.im = make_float2(a.y + S * b.y, a.w + S * b.w);
  return h;
}
template <int S>
__device__ __forceinline__ cx2 comb_i(float4 a, float4 b) {
  cx2 h;
  h.re = make_float2(a.x - S * b.y, a.z - S * b.w);
  h.im = make_float2(a.y + S * b.x, a.w + S * b.z);
  return h;
}

// acc_up += coef hp,  acc_lo -= cl lo  (lower accumulated with the Gamma5 sign),
// for one hop (MU, SIGN): h = (1 -+ gamma_mu) projection of the neighbour pair
// nb (nb(c) = component c of the pair as (re_s, im_s, re_s+1, im_s+1)), hp = U h
// (SIGN > 0) or U^dag h (SIGN < 0) with the link L (row-major 3x3).
template <int MU, int SIGN, class Pair>
__device__ __forceinline__ void hop_x2(const cpx<float>* __restrict__ L, const Pair& nb, float coef,
                                       cx2 (&up)[2][3], cx2 (&lo)[2][3]) {
  cx2 h[2][3];
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const float4 u0 = nb(0 + c), u1 = nb(3 + c);
    const float4 d0 = nb(6 + c), d1 = nb(9 + c);
    constexpr int S = SIGN;
    if (MU == 3) {
      h[0][c] = comb<-S>(u0, d0);
      h[1][c] = comb<-S>(u1, d1);
    } else if (MU == 0) {
      h[0][c] = comb_i<S>(u0, d1);
      h[1][c] = comb_i<S>(u1, d0);
    } else if (MU == 1) {
      h[0][c] = comb<S>(u0, d1);
      h[1][c] = comb<-S>(u1, d0);
    } else {
      h[0][c] = comb_i<S>(u0, d0);
      h[1][c] = comb_i<-S>(u1, d1);
    }
  }
  // hp = U h (forward) or U^dag h (backward); each element broadcast to both lanes
  cx2 hp[2][3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    float2 pr[2], nr[2], pi[2], ni[2];
#pragma unroll
    for (int b = 0; b < 3; ++b) {
      const cpx<float> lc = ld(L + (SIGN > 0 ? 3 * a + b : 3 * b + a));
      const float4 l = make_float4(lc.re, lc.re, lc.im, lc.im);
      const float2 mr = make_float2(l.x, l.y), mi = make_float2(l.z, l.w);
#pragma unroll
      for (int sp = 0; sp < 2; ++sp) {
        const cx2 x = h[sp][b];
        if (SIGN > 0) {  // re = mr xr - mi xi, im = mr xi + mi xr
          pr[sp] = b == 0 ? mul2(mr, x.re) : fma2(mr, x.re, pr[sp]);
          nr[sp] = b == 0 ? mul2(mi, x.im) : fma2(mi, x.im, nr[sp]);
          pi[sp] = b == 0 ? mul2(mr, x.im) : fma2(mr, x.im, pi[sp]);
          pi[sp] = fma2(mi, x.re, pi[sp]);
        } else {  // conj: re = mr xr + mi xi, im = mr xi - mi xr
          pr[sp] = b == 0 ? mul2(mr, x.re) : fma2(mr, x.re, pr[sp]);
          pr[sp] = fma2(mi, x.im, pr[sp]);
          pi[sp] = b == 0 ? mul2(mr, x.im) : fma2(mr, x.im, pi[sp]);
          ni[sp] = b == 0 ? mul2(mi, x.re) : fma2(mi, x.re, ni[sp]);
        }
      }
    }
#pragma unroll
    for (int sp = 0; sp < 2; ++sp) {
      if (SIGN > 0) {
        hp[sp][a].re = sub2(pr[sp], nr[sp]);
        hp[sp][a].im = pi[sp];
      } else {
        hp[sp][a].re = pr[sp];
        hp[sp][a].im = sub2(pi[sp], ni[sp]);
      }
    }
  }
  // upper += coef hp; true lower += cl lo with cl = -coef (SIGN > 0) or +coef,
  // lo = hp (t) or i sigma_mu hp; the stored lower is minus the true one
  const float2 cp = f2(coef), cm = f2(-coef);
  const float2 gl = SIGN > 0 ? cp : cm;  // -cl: factor on lo for the negated lower
  const float2 gn = SIGN > 0 ? cm : cp;  // +cl
#pragma unroll
  for (int c = 0; c < 3; ++c) {
#pragma unroll
    for (int sp = 0; sp < 2; ++sp) {
      up[sp][c].re = fma2(cp, hp[sp][c].re, up[sp][c].re);
      up[sp][c].im = fma2(cp, hp[sp][c].im, up[sp][c].im);
    }
    const cx2 a = hp[0][c], b = hp[1][c];
    if (MU == 3) {  // lo = (a, b)
      lo[0][c].re = fma2(gl, a.re, lo[0][c].re);
      lo[0][c].im = fma2(gl, a.im, lo[0][c].im);
      lo[1][c].re = fma2(gl, b.re, lo[1][c].re);
      lo[1][c].im = fma2(gl, b.im, lo[1][c].im);
    } else if (MU == 0) {  // lo = (i b, i a):  (i z) = (-z.im, z.re)
      lo[0][c].re = fma2(gn, b.im, lo[0][c].re);
      lo[0][c].im = fma2(gl, b.re, lo[0][c].im);
      lo[1][c].re = fma2(gn, a.im, lo[1][c].re);
      lo[1][c].im = fma2(gl, a.re, lo[1][c].im);
    } else if (MU == 1) {  // lo = (b, -a)
      lo[0][c].re = fma2(gl, b.re, lo[0][c].re);
      lo[0][c].im = fma2(gl, b.im, lo[0][c].im);
      lo[1][c].re = fma2(gn, a.re, lo[1][c].re);
      lo[1][c].im = fma2(gn, a.im, lo[1][c].im);
    } else {  // lo = (i a, -i b):  (-i z) = (z.im, -z.re)
      lo[0][c].re = fma2(gn, a.im, lo[0][c].re);
      lo[0][c].im = fma2(gl, a.re, lo[0][c].im);
      lo[1][c].re = fma2(gl, b.im, lo[1][c].re);
      lo[1][c].im = fma2(gn, b.re, lo[1][c].im);
    }
  }
}

// The order in which every FP32 kernel variant adds up one output pair, so that
// all variants give the same bits: first the hops y+, y-, z+, z-, t- (the ones the
// shared-memory kernel reads from its halo and its previous plane), then x+, x-,
// t+, then the diagonal and fifth-dimension terms.  NB(d) is the accessor of the
// neighbour pair of hop d = 2 mu + (0 forward, 1 backward), LK(d) its link and
// CF(d) its factor -1/2 times the boundary phase.
template <class Hop>
__device__ __forceinline__ void hops_first(const Hop& h, cx2 (&up)[2][3], cx2 (&lo)[2][3]) {
  hop_x2<1, +1>(h.link(2), h.nb(2), h.coef(2), up, lo);
  hop_x2<1, -1>(h.link(3), h.nb(3), h.coef(3), up, lo);
  hop_x2<2, +1>(h.link(4), h.nb(4), h.coef(4), up, lo);
  hop_x2<2, -1>(h.link(5), h.nb(5), h.coef(5), up, lo);
  hop_x2<3, -1>(h.link(7), h.nb(7), h.coef(7), up, lo);
}
template <class Hop>
__device__ __forceinline__ void hops_second(const Hop& h, cx2 (&up)[2][3], cx2 (&lo)[2][3]) {
  hop_x2<0, +1>(h.link(0), h.nb(0), h.coef(0), up, lo);
  hop_x2<0, -1>(h.link(1), h.nb(1), h.coef(1), up, lo);
  hop_x2<3, +1>(h.link(6), h.nb(6), h.coef(6), up, lo);
}

__device__ __forceinline__ void zero_acc(cx2 (&up)[2][3], cx2 (&lo)[2][3]) {
#pragma unroll
  for (int sp = 0; sp < 2; ++sp)
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      up[sp][c].re = up[sp][c].im = lo[sp][c].re = lo[sp][c].im = make_float2(0.f, 0.f);
    }
}

// Adds the diagonal and fifth-dimension terms of the pair (s0, s0+1), lane by lane:
//   upper(s) += diag psi(s) - w psi(s-1),  lower(s) += diag psi(s) - w psi(s+1)
// (the lower accumulated negated, i.e. with the Gamma5 sign).  q[c]: the pair's
// component c as (re_s0, im_s0, re_s0+1, im_s0+1); prv[c] = psi(s0-1) for the
// upper components c < 6 with weight w0, nxt[c] = psi(s0+2) for the lower ones
// c >= 6 (index c - 6) with weight w1 (1, or -mf at a wall).
__device__ __forceinline__ void local_x2(const float4 (&q)[12], const cpx<float> (&prv)[6],
                                         const cpx<float> (&nxt)[6], float w0, float w1, float diag,
                                         cx2 (&up)[2][3], cx2 (&lo)[2][3]) {
#pragma unroll
  for (int c = 0; c < 6; ++c) {
    const int sp = c / 3, cc = c % 3;
    up[sp][cc].re = add2(up[sp][cc].re, make_float2(fmaf(-w0, prv[c].re, diag * q[c].x), fmaf(-1.f, q[c].x, diag * q[c].z)));
    up[sp][cc].im = add2(up[sp][cc].im, make_float2(fmaf(-w0, prv[c].im, diag * q[c].y), fmaf(-1.f, q[c].y, diag * q[c].w)));
  }
#pragma unroll
  for (int c = 6; c < 12; ++c) {
    const int sp = c / 3 - 2, cc = c % 3;
    lo[sp][cc].re = add2(lo[sp][cc].re, make_float2(fmaf(-diag, q[c].x, q[c].z), fmaf(-diag, q[c].z, w1 * nxt[c - 6].re)));
    lo[sp][cc].im = add2(lo[sp][cc].im, make_float2(fmaf(-diag, q[c].y, q[c].w), fmaf(-diag, q[c].w, w1 * nxt[c - 6].im)));
  }
}

constexpr int X2_STORE = 0, X2_DOT = 1, X2_CHEB = 2;  // epilogues of the kernels

// Chebyshev step of the epilogue X2_CHEB: out <- nx = 2 (a H in + b cur) - out,
// and, when acc is set, acc += ck nx (the smoother's running sum)
struct X2Cheb {
  const cpx<float>* cur;
  float a, b;
  cpx<float>* acc = nullptr;
  float ck = 0.f;
};

// Writes the pair to its output sites: out(Ls-1-s) = gamma5 acc(s), i.e. the pair
// at Ls-2-s0 with its lanes swapped; o, i and cur point at that output pair of
// out, in and ch.cur (component stride ls).  X2_DOT returns Re <in, H in> of the
// two output sites (products summed in FP32 within each spin half, where the
// terms share the sign of Gamma5, the halves combined in FP64); X2_CHEB writes
// 2 (a H in + b cur) - prev over prev = out and adds ck times it to acc when set.
template <int EPI>
__device__ __forceinline__ double store_x2(const cx2 (&up)[2][3], const cx2 (&lo)[2][3], cpx<float>* o,
                                           const cpx<float>* i, const cpx<float>* cur, float ca, float cb,
                                           int ls, cpx<float>* acc = nullptr, float ck = 0.f) {
  float d[2] = {0.f, 0.f};
#pragma unroll
  for (int c = 0; c < 12; ++c) {
    const cx2 v = c < 6 ? up[c / 3][c % 3] : lo[c / 3 - 2][c % 3];
    float4 r = make_float4(v.re.y, v.im.y, v.re.x, v.im.x);
    if constexpr (EPI == X2_CHEB) {
      const float4 cv = ld4(cur + c * ls), pv = ld4(o + c * ls);
      r = make_float4(2.f * fmaf(ca, r.x, cb * cv.x) - pv.x, 2.f * fmaf(ca, r.y, cb * cv.y) - pv.y,
                      2.f * fmaf(ca, r.z, cb * cv.z) - pv.z, 2.f * fmaf(ca, r.w, cb * cv.w) - pv.w);
      if (acc) {
        const float4 av = ld4(acc + c * ls);
        *reinterpret_cast<float4*>(acc + c * ls) =
            make_float4(fmaf(ck, r.x, av.x), fmaf(ck, r.y, av.y), fmaf(ck, r.z, av.z), fmaf(ck, r.w, av.w));
      }
    }
    *reinterpret_cast<float4*>(o + c * ls) = r;
    if (EPI == X2_DOT) {
      const float4 a = ld4(i + c * ls);
      float& e = d[c < 6 ? 0 : 1];
      e = fmaf(a.x, r.x, e);
      e = fmaf(a.y, r.y, e);
      e = fmaf(a.z, r.z, e);
      e = fmaf(a.w, r.w, e);
    }
  }
  return EPI == X2_DOT ? (double)d[0] + (double)d[1] : 0.0;
}

// Per-CTA data: for each of the SITES 4d sites of the CTA's tile and each hop
// d = 2 mu + (0 forward, 1 backward) the neighbour site, the boundary factor
// and the link (U_mu(x) forward, U_mu(x - mu) backward) as an index into U.
template <int SITES>
struct X2Stage {
  int x4[SITES];
  int nb[SITES][8];
  float coef[SITES][8];
  int li[SITES][8];
};

// Tile shapes of the CTA: TX x TY x TZ x TT 4d sites (x fastest), the tiles
// laid out over the lattice in the same order; TY == 0 marks the linear tile of
// TX consecutive 4d sites, which fits any volume.  A tile shares the hops that
// stay inside it through L1 (the Ls/2 threads of a site, and the sites of the
// tile, run on one SM at the same time).
template <int TX, int TY, int TZ, int TT>
struct Tile {
  static constexpr bool linear = TY == 0;
  static constexpr int sites = linear ? TX : TX * TY * TZ * TT;
  // 4d index of site `site` of tile `grp`, or -1 past the end of the lattice
  __device__ static int site_x4(const Geom& g, int grp, int site) {
    if constexpr (linear) {
      const int x4 = grp * TX + site;
      return x4 < g.V4 ? x4 : -1;
    } else {
      const int nx = g.L[0] / TX, ny = g.L[1] / TY, nz = g.L[2] / TZ;
      int r = grp;
      const int gx = r % nx; r /= nx;
      const int gy = r % ny; r /= ny;
      const int gz = r % nz;
      const int gt = r / nz;
      int q = site;
      const int sx = q % TX; q /= TX;
      const int sy = q % TY; q /= TY;
      const int sz = q % TZ;
      const int st = q / TZ;
      const int c[4] = {gx * TX + sx, gy * TY + sy, gz * TZ + sz, gt * TT + st};
      return c[3] < g.L[3] ? x4_index(g, c) : -1;
    }
  }
  __host__ static bool fits(const Geom& g) {
    if (linear) return true;
    return g.L[0] % TX == 0 && g.L[1] % TY == 0 && g.L[2] % TZ == 0 && g.L[3] % TT == 0;
  }
  __host__ __device__ static int tiles(const Geom& g) { return (g.V4 + sites - 1) / sites; }
};

// Neighbours, boundary factors and link indices of the sites of tile grp.
template <typename T>
__device__ __forceinline__ void stage_sites(const Geom& g, int grp, X2Stage<T::sites>& sm) {
  for (int t = threadIdx.x; t < T::sites * 8; t += blockDim.x) {
    const int site = t >> 3, d = t & 7, mu = d >> 1;
    const int x4 = T::site_x4(g, grp, site);
    int nb = 0, li = 0;
    float cf = 0.f;
    if (x4 >= 0) {
      // coordinate mu of x4 and the index stride of direction mu (no dynamic indexing)
      const int L0 = g.L[0], L1 = g.L[1], L2 = g.L[2], L3 = g.L[3];
      const int lm = mu == 0 ? L0 : mu == 1 ? L1 : mu == 2 ? L2 : L3;
      const int stride = mu == 0 ? 1 : mu == 1 ? L0 : mu == 2 ? L0 * L1 : L0 * L1 * L2;
      const int cm = (x4 / stride) % lm;
      int ph = 1;
      if (d & 1) {
        nb = cm == 0 ? x4 + (lm - 1) * stride : x4 - stride;
        if (cm == 0 && mu == 3) ph = g.bc_t;
      } else {
        nb = cm == lm - 1 ? x4 - (lm - 1) * stride : x4 + stride;
        if (cm == lm - 1 && mu == 3) ph = g.bc_t;
      }
      li = mu * g.V4 + ((d & 1) ? nb : x4);
      cf = -0.5f * (float)ph;
    }
    if (d == 0) sm.x4[site] = x4;
    sm.nb[site][d] = nb;
    sm.coef[site][d] = cf;
    sm.li[site][d] = li;
  }
  __syncthreads();
}

// component c of a pair in an FP32 field: psi[x4][c][s] with q at (x4, 0, s0)
struct PairF32 {
  const cpx<float>* q;
  int ls;
  __device__ __forceinline__ float4 operator()(int c) const { return ld4(q + c * ls); }
};

}  // namespace hdcr
