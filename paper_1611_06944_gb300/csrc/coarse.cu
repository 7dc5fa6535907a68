// Little Dirac operator A^{ab}_{jk} = <phi_j^a | H | phi_k^b> (Eq. 4.5), its
// 9-point application, and the restriction / prolongation P^dag, P (Eq. 4.3).
//
// Build.  H splits into the part that stays inside a block (leg 0: the local
// terms and the hops between sites of one block) and the hops that leave a
// block towards a +- mu.  Blocks span the whole fifth dimension, so the s-hops
// and Gamma5's R5 stay inside a block.
//   leg 0:   Y_k = H_0 phi_k on every site, A[a][0][j][k] = sum_{x in a} phi_j^dag Y_k
//            for j <= k (A^{aa} is Hermitian; the rest is mirrored).  The FP32
//            build instead applies all of H to the nvec fields at once (the
//            packed stencil), projects, and subtracts the outward legs below.
//   leg +mu: only the +mu face of block a takes part, and there the hop result
//            is (hp; lo(hp)) after Gamma5 with hp = -1/2 U_mu(x) h (h the
//            two-spinor projection of phi_k(x + mu)), lo = i sigma_mu (or 1 for
//            t).  So A[a][+mu][j][k] = sum_face phit_j^dag hp_k with the
//            six-component projected basis phit = phi_up + lo^dag phi_lo taken at
//            the reflected s (R5): half the components of a full projection.
//   leg -mu: H is Hermitian, so A[a][-mu] = (A[a - mu][+mu])^dag.
// On a coarse extent of 2 the legs +mu and -mu reach the same coarse site and
// are both kept.
#include <algorithm>
#include <vector>

#include "host_io.cuh"
#include "level2.cuh"
#include "coarse.cuh"
#include "coarse_tc.cuh"
#include "dwf_stencil.cuh"

namespace hdcr {

int coarse_check(const hdcr_coarse* co) {
  if (!co || !co->A || !co->nbr || !co->sub) {
    set_error("invalid coarse-operator handle");
    return HDCR_ERR_BAD_ARG;
  }
  return HDCR_OK;
}

// ------------------------------------------------------------ leg stencil
template <typename R>
__device__ __forceinline__ bool crosses(const BlockGeom& bg, const int co[4], int mu, int sign) {
  const int r = co[mu] % bg.b[mu];
  return sign > 0 ? (r == bg.b[mu] - 1) : (r == 0);
}

// leg 0: local terms + hops that stay inside the block, every site
template <typename R>
__global__ void __launch_bounds__(256) leg_self_kernel(Geom g, BlockGeom bg, R diag, R mf,
                                                       const cpx<R>* __restrict__ U,
                                                       const cpx<R>* __restrict__ vecs,
                                                       cpx<R>* __restrict__ Y, int nvec) {
  const long long total = g.V5 * nvec;
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= total) return;
  const int k = (int)(idx / g.V5);
  const long long i5 = idx - (long long)k * g.V5;
  const cpx<R>* in = vecs + (long long)k * 12 * g.V5;
  const int x4 = (int)(i5 / g.Ls);
  const int s = (int)(i5 - (long long)x4 * g.Ls);
  int co[4];
  x4_coords(g, x4, co);
  cpx<R> acc[4][3];
  local_part<R, 0>(g, diag, mf, in + fidx(g, 0, i5), s, acc);
  if (!crosses<R>(bg, co, 0, +1)) hop_full<R, 0, 0, +1>(g, U, in, x4, s, co, acc);
  if (!crosses<R>(bg, co, 0, -1)) hop_full<R, 0, 0, -1>(g, U, in, x4, s, co, acc);
  if (!crosses<R>(bg, co, 1, +1)) hop_full<R, 0, 1, +1>(g, U, in, x4, s, co, acc);
  if (!crosses<R>(bg, co, 1, -1)) hop_full<R, 0, 1, -1>(g, U, in, x4, s, co, acc);
  if (!crosses<R>(bg, co, 2, +1)) hop_full<R, 0, 2, +1>(g, U, in, x4, s, co, acc);
  if (!crosses<R>(bg, co, 2, -1)) hop_full<R, 0, 2, -1>(g, U, in, x4, s, co, acc);
  if (!crosses<R>(bg, co, 3, +1)) hop_full<R, 0, 3, +1>(g, U, in, x4, s, co, acc);
  if (!crosses<R>(bg, co, 3, -1)) hop_full<R, 0, 3, -1>(g, U, in, x4, s, co, acc);
  store_g5r5<R, 0>(g, Y + (long long)k * 12 * g.V5, x4, s, acc);
}

// ------------------------------------------------------------ projection
// local site index l (0 <= l < nsites) of the leg's site set in block a -> fine 5d index
__device__ __forceinline__ long long leg_local_site(const Geom& g, const BlockGeom& bg, int a, int leg,
                                                    long long l) {
  if (leg == 0) return block_site(g, bg, a, l);
  const int mu = (leg - 1) >> 1;
  const int sign = ((leg - 1) & 1) ? -1 : +1;
  // enumerate the block with extent 1 in mu, then place the mu coordinate on the face
  const int s = (int)(l % g.Ls);
  long long r = l / g.Ls;
  int ac[4];
  coarse_coords(bg, a, ac);
  int c[4];
#pragma unroll
  for (int nu = 0; nu < 4; ++nu) {
    const int ext = nu == mu ? 1 : bg.b[nu];
    const int loc = (int)(r % ext);
    r /= ext;
    c[nu] = ac[nu] * bg.b[nu] + (nu == mu ? (sign > 0 ? bg.b[nu] - 1 : 0) : loc);
  }
  return (long long)x4_index(g, c) * g.Ls + s;
}

constexpr int PROJ_THREADS = 256;
constexpr int PROJ_MAXP = 16;  // (j, k) pairs per thread: nvec <= 64

template <typename R>
__global__ void __launch_bounds__(PROJ_THREADS) project_kernel(Geom g, BlockGeom bg,
                                                               const cpx<R>* __restrict__ phi,
                                                               const cpx<R>* __restrict__ Y,
                                                               cpx<R>* __restrict__ A, int nvec, int leg,
                                                               int T, bool upper) {
  extern __shared__ unsigned char smem_raw[];
  cpx<R>* sphi = reinterpret_cast<cpx<R>*>(smem_raw);   // [nvec][12][T]
  cpx<R>* sy = sphi + (size_t)nvec * 12 * T;            // [nvec][12][T]
  const int a = blockIdx.x;
  const long long fs = g.V5 * 12;
  const long long nsites = leg == 0 ? bg.K5 : bg.K5 / bg.b[(leg - 1) >> 1];
  const int npairs = nvec * nvec;
  double acc[PROJ_MAXP][2];
#pragma unroll
  for (int i = 0; i < PROJ_MAXP; ++i) acc[i][0] = acc[i][1] = 0.0;
  const int nload = nvec * 12 * T;
  for (long long l0 = 0; l0 < nsites; l0 += T) {
    const int tn = (int)min((long long)T, nsites - l0);
    for (int e = threadIdx.x; e < nload; e += PROJ_THREADS) {
      const int t = e % T;
      const int c = (e / T) % 12;
      const int v = e / (12 * T);
      cpx<R> p((R)0, (R)0), q((R)0, (R)0);
      if (t < tn) {
        const long long i5 = leg_local_site(g, bg, a, leg, l0 + t);
        const long long off = (long long)v * fs + fidx(g, c, i5);
        p = ld(phi + off);
        q = ld(Y + off);
      }
      sphi[e] = p;
      sy[e] = q;
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < PROJ_MAXP; ++i) {
      const int pr = threadIdx.x + i * PROJ_THREADS;
      if (pr < npairs && !(upper && pr / nvec > pr % nvec)) {
        const int j = pr / nvec, k = pr % nvec;
        const cpx<R>* pj = sphi + (size_t)j * 12 * T;
        const cpx<R>* yk = sy + (size_t)k * 12 * T;
        cpx<R> sum((R)0, (R)0);
        for (int e = 0; e < 12 * T; ++e) sum = cjmadd(sum, pj[e], yk[e]);
        acc[i][0] += (double)sum.re;
        acc[i][1] += (double)sum.im;
      }
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < PROJ_MAXP; ++i) {
    const int pr = threadIdx.x + i * PROJ_THREADS;
    if (pr < npairs && !(upper && pr / nvec > pr % nvec)) {
      const int j = pr / nvec, k = pr % nvec;
      A[(((long long)a * NLEGS + leg) * nvec + j) * nvec + k] = cpx<R>((R)acc[i][0], (R)acc[i][1]);
    }
  }
}

// ------------------------------------------------------------ forward legs
// Face site l of the +MU face of block a: the local sites of the block with
// the MU coordinate fixed to the block's last, l = ((x4 local) * Ls + s).
template <int MU>
__device__ __forceinline__ long long face_site(const Geom& g, const BlockGeom& bg, int a, long long l) {
  return leg_local_site(g, bg, a, leg_of(MU, +1), l);
}

// For vector v and face site (x, s) of the +MU face of block a, both operands of
// the leg's projection (layout [v][a][l][6]):
//   pt = phi_up + lo^dag phi_lo at (x, Ls-1-s),  lo^dag = -i sigma_MU (MU < 3) or 1,
//   hf = -1/2 (phase) U_MU(x) h(x + MU, s), h the two-spinor of the (1 - gamma_MU)
//        projection of phi_v.
template <typename R, int MU>
__global__ void __launch_bounds__(256) face_kernel(Geom g, BlockGeom bg, const cpx<R>* __restrict__ U,
                                                   const cpx<R>* __restrict__ phi, cpx<R>* __restrict__ pt,
                                                   cpx<R>* __restrict__ hf, int nvec, long long nf) {
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long per = (long long)bg.Vc * nf;
  if (idx >= per * nvec) return;
  const int v = (int)(idx / per);
  const long long r = idx - (long long)v * per;
  const int a = (int)(r / nf);
  const long long l = r - (long long)a * nf;
  const long long i5 = face_site<MU>(g, bg, a, l);
  const int x4 = (int)(i5 / g.Ls);
  const int s = (int)(i5 - (long long)x4 * g.Ls);
  const int ls = g.Ls;
  const cpx<R>* field = phi + (long long)v * 12 * g.V5;
  {
    const cpx<R>* p = field + (unsigned)(x4 * 12 * ls + (ls - 1 - s));
    cpx<R> u0[3], u1[3], d0[3], d1[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      u0[c] = ld(p + (0 + c) * ls);
      u1[c] = ld(p + (3 + c) * ls);
      d0[c] = ld(p + (6 + c) * ls);
      d1[c] = ld(p + (9 + c) * ls);
    }
    cpx<R> o0[3], o1[3];
    if (MU == 3) {
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        o0[c] = u0[c] + d0[c];
        o1[c] = u1[c] + d1[c];
      }
    } else {
      cpx<R> t0[3], t1[3];
      i_sigma<R, MU>(d0, d1, t0, t1);
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        o0[c] = u0[c] - t0[c];
        o1[c] = u1[c] - t1[c];
      }
    }
    cpx<R>* q = pt + idx * 6;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      st(q + c, o0[c]);
      st(q + 3 + c, o1[c]);
    }
  }
  int co[4];
  x4_coords(g, x4, co);
  int ph;
  const int y4 = neighbour<MU, +1>(g, co, &ph);
  const cpx<R>* nb = field + (unsigned)(y4 * 12 * ls + s);
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
        h[0][c] = u0[c] - d0[c];
        h[1][c] = u1[c] - d1[c];
      }
    } else {
      cpx<R> t0[3], t1[3];
      i_sigma<R, MU>(d0, d1, t0, t1);
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        h[0][c] = u0[c] + t0[c];
        h[1][c] = u1[c] + t1[c];
      }
    }
  }
  const cpx<R>* Ul = U + (unsigned)((MU * g.V4 + x4) * 9);
  const R coef = (R)(-0.5 * ph);
  cpx<R>* q = hf + idx * 6;
#pragma unroll
  for (int sp = 0; sp < 2; ++sp)
#pragma unroll
    for (int aa = 0; aa < 3; ++aa) {
      cpx<R> t((R)0, (R)0);
#pragma unroll
      for (int b = 0; b < 3; ++b) t = cmadd(t, ld(Ul + 3 * aa + b), h[sp][b]);
      st(q + 3 * sp + aa, coef * t);
    }
}

// A[a][leg][j][k] = sum_e conj(X[j][a][e]) Y[k][a][e], e < K (contiguous per vector and block)
template <typename R>
__global__ void __launch_bounds__(PROJ_THREADS) face_project_kernel(const cpx<R>* __restrict__ X,
                                                                    const cpx<R>* __restrict__ Y, long long K,
                                                                    cpx<R>* __restrict__ A, int Vc, int nvec,
                                                                    int leg, int T) {
  extern __shared__ unsigned char smem_raw[];
  cpx<R>* sx = reinterpret_cast<cpx<R>*>(smem_raw);  // [nvec][T]
  cpx<R>* sy = sx + (size_t)nvec * T;                // [nvec][T]
  const int a = blockIdx.x;
  const int npairs = nvec * nvec;
  double acc[PROJ_MAXP][2];
#pragma unroll
  for (int i = 0; i < PROJ_MAXP; ++i) acc[i][0] = acc[i][1] = 0.0;
  for (long long e0 = 0; e0 < K; e0 += T) {
    const int tn = (int)min((long long)T, K - e0);
    for (int e = threadIdx.x; e < nvec * T; e += PROJ_THREADS) {
      const int v = e / T, t = e - v * T;
      cpx<R> p((R)0, (R)0), q((R)0, (R)0);
      if (t < tn) {
        const long long off = ((long long)v * Vc + a) * K + e0 + t;
        p = ld(X + off);
        q = ld(Y + off);
      }
      sx[e] = p;
      sy[e] = q;
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < PROJ_MAXP; ++i) {
      const int pr = threadIdx.x + i * PROJ_THREADS;
      if (pr < npairs) {
        const int j = pr / nvec, k = pr % nvec;
        const cpx<R>* xj = sx + (size_t)j * T;
        const cpx<R>* yk = sy + (size_t)k * T;
        cpx<R> sum((R)0, (R)0);
        for (int e = 0; e < T; ++e) sum = cjmadd(sum, xj[e], yk[e]);
        acc[i][0] += (double)sum.re;
        acc[i][1] += (double)sum.im;
      }
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < PROJ_MAXP; ++i) {
    const int pr = threadIdx.x + i * PROJ_THREADS;
    if (pr < npairs) {
      const int j = pr / nvec, k = pr % nvec;
      A[(((long long)a * NLEGS + leg) * nvec + j) * nvec + k] = cpx<R>((R)acc[i][0], (R)acc[i][1]);
    }
  }
}

// The legs not computed directly: A[a][0][j][k] = conj(A[a][0][k][j]) for j > k, and
// A[a][-mu][j][k] = conj(A[a - mu][+mu][k][j]).
template <typename R>
__global__ void complete_legs_kernel(cpx<R>* __restrict__ A, const int* __restrict__ nbr, int Vc, int nvec,
                                     bool leg0) {
  const long long n2 = (long long)nvec * nvec;
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (long long)Vc * 5 * n2) return;
  const int a = (int)(idx / (5 * n2));
  const long long r = idx - (long long)a * 5 * n2;
  const int w = (int)(r / n2);  // 0: leg 0, 1..4: leg (mu = w-1, -)
  const int j = (int)((r - (long long)w * n2) / nvec), k = (int)(r % nvec);
  cpx<R> v;
  int leg;
  if (w == 0) {
    if (!leg0 || j <= k) return;
    leg = 0;
    v = A[(((long long)a * NLEGS) * nvec + k) * nvec + j];
  } else {
    const int mu = w - 1;
    leg = leg_of(mu, -1);
    const int b = nbr[a * NLEGS + leg];
    v = A[(((long long)b * NLEGS + leg_of(mu, +1)) * nvec + k) * nvec + j];
  }
  A[(((long long)a * NLEGS + leg) * nvec + j) * nvec + k] = cpx<R>(v.re, -v.im);
}

// Leg 0 from the projection of the whole of H: over block a, sum_x phi_j^dag (H phi_k)
// (phi_k holding every block's vector k) is A^{aa} plus every leg that reaches a
// neighbour block, so A[a][0] = P - sum_{leg > 0} A[a][leg]; the result is made
// exactly Hermitian, (d + d^dag) / 2.  One thread per pair j <= k.
template <typename R>
__global__ void subtract_legs_kernel(cpx<R>* __restrict__ A, int Vc, int nvec) {
  const long long n2 = (long long)nvec * nvec;
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (long long)Vc * n2) return;
  const int a = (int)(idx / n2);
  const int j = (int)((idx - (long long)a * n2) / nvec), k = (int)(idx % nvec);
  if (j > k) return;
  cpx<R>* Aa = A + (long long)a * NLEGS * n2;
  cpx<R> d1 = Aa[(long long)j * nvec + k], d2 = Aa[(long long)k * nvec + j];
  for (int leg = 1; leg < NLEGS; ++leg) {
    d1 = d1 - Aa[leg * n2 + (long long)j * nvec + k];
    d2 = d2 - Aa[leg * n2 + (long long)k * nvec + j];
  }
  const cpx<R> h((R)0.5 * (d1.re + d2.re), (R)0.5 * (d1.im - d2.im));
  Aa[(long long)j * nvec + k] = h;
  Aa[(long long)k * nvec + j] = cpx<R>(h.re, -h.im);
}

// ------------------------------------------------------------ coarse apply
template <typename R>
__global__ void coarse_apply_kernel(const cpx<R>* __restrict__ A, const int* __restrict__ nbr,
                                    const cpx<R>* __restrict__ in, cpx<R>* __restrict__ out, int Vc, int nvec,
                                    int nrhs) {
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long n = (long long)Vc * nvec;
  if (idx >= n * nrhs) return;
  const int r = (int)(idx / n);
  const long long rem = idx - (long long)r * n;
  const int a = (int)(rem / nvec);
  const int j = (int)(rem - (long long)a * nvec);
  const cpx<R>* x = in + (long long)r * n;
  cpx<R> acc((R)0, (R)0);
  for (int d = 0; d < NLEGS; ++d) {
    const cpx<R>* row = A + (((long long)a * NLEGS + d) * nvec + j) * nvec;
    const cpx<R>* xb = x + (long long)nbr[a * NLEGS + d] * nvec;
    for (int k = 0; k < nvec; ++k) acc = cmadd(acc, ld(row + k), ld(xb + k));
  }
  st(out + idx, acc);
}

template <typename R>
__global__ void __launch_bounds__(RED_THREADS) cdot_re_kernel(const cpx<R>* __restrict__ u,
                                                              const cpx<R>* __restrict__ v, long long n,
                                                              RedScratch rs, double* result) {
  double acc[1] = {0.0};
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const cpx<R> a = ld(u + i), b = ld(v + i);
    acc[0] = fma((double)a.re, (double)b.re, fma((double)a.im, (double)b.im, acc[0]));
  }
  double tot[1];
  if (grid_reduce<1>(acc, rs, tot)) *result = tot[0];
}

// ------------------------------------------------------------ restrict / prolong
constexpr int RP_KC = 8;  // basis vectors per restrict CTA

template <typename R>
__global__ void __launch_bounds__(RED_THREADS) restrict_kernel(Geom g, BlockGeom bg,
                                                               const cpx<R>* __restrict__ phi,
                                                               const cpx<R>* __restrict__ fine,
                                                               cpx<R>* __restrict__ coarse, int nvec,
                                                               bool table) {
  extern __shared__ int sx4[];  // the block's 4d sites (bvol of them), when ``table``
  const int a = blockIdx.x;
  const int k0 = blockIdx.y * RP_KC;
  const int r = blockIdx.z;
  const long long fs = g.V5 * 12;
  const cpx<R>* v = fine + (long long)r * fs;
  if (table) {
    for (int i = threadIdx.x; i < bg.bvol; i += RED_THREADS)
      sx4[i] = (int)(block_site(g, bg, a, (long long)i * g.Ls) / g.Ls);
    __syncthreads();
  }
  // each thread sums its elements in R (FP32 for an FP32 basis: the result is
  // stored in FP32, and FP64 arithmetic would bind the kernel to the slow FP64
  // pipe); the threads' partial sums are added in FP64
  R tacc[2 * RP_KC];
#pragma unroll
  for (int i = 0; i < 2 * RP_KC; ++i) tacc[i] = (R)0;
  // elements in the order (4d site of the block, component, s): one 4d site's 12 Ls
  // elements are contiguous in the field, so the index is one 32-bit division and a
  // table lookup
  const int per = 12 * g.Ls;
  const int nel = bg.bvol * per;
  for (int e = threadIdx.x; e < nel; e += RED_THREADS) {
    const int site = e / per;
    const unsigned x4 = table ? (unsigned)sx4[site] : (unsigned)(block_site(g, bg, a, (long long)site * g.Ls) / g.Ls);
    const unsigned off = x4 * (unsigned)per + (unsigned)(e - site * per);
    const cpx<R> q = ld(v + off);
#pragma unroll
    for (int i = 0; i < RP_KC; ++i) {
      if (k0 + i < nvec) {
        const cpx<R> p = ld(phi + (long long)(k0 + i) * fs + off);
        // conj(p) q accumulated with four FMAs
        tacc[2 * i] = fma(p.re, q.re, fma(p.im, q.im, tacc[2 * i]));
        tacc[2 * i + 1] = fma(p.re, q.im, fma(-p.im, q.re, tacc[2 * i + 1]));
      }
    }
  }
  double acc[2 * RP_KC];
#pragma unroll
  for (int i = 0; i < 2 * RP_KC; ++i) acc[i] = (double)tacc[i];
  block_reduce<2 * RP_KC>(acc);
  if (threadIdx.x == 0) {
#pragma unroll
    for (int i = 0; i < RP_KC; ++i)
      if (k0 + i < nvec)
        coarse[((long long)r * bg.Vc + a) * nvec + k0 + i] = cpx<R>((R)acc[2 * i], (R)acc[2 * i + 1]);
  }
}

// fine = fine_in + sum_k phi_k c[a][k]   (fine_in may be null)
template <typename R>
__global__ void prolong_kernel(Geom g, BlockGeom bg, const cpx<R>* __restrict__ phi,
                               const cpx<R>* __restrict__ coarse, const cpx<R>* __restrict__ fine_in,
                               cpx<R>* __restrict__ fine, int nvec, int nrhs) {
  const long long fs = g.V5 * 12;
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= fs * nrhs) return;
  const int r = (int)(idx / fs);
  const long long e = idx - (long long)r * fs;   // element (x4*12 + c)*Ls + s
  const int x4 = (int)(e / (12LL * g.Ls));
  int co[4];
  x4_coords(g, x4, co);
  int ac[4];
  for (int mu = 0; mu < 4; ++mu) ac[mu] = co[mu] / bg.b[mu];
  const int a = ((ac[3] * bg.Lc[2] + ac[2]) * bg.Lc[1] + ac[1]) * bg.Lc[0] + ac[0];
  const cpx<R>* cf = coarse + ((long long)r * bg.Vc + a) * nvec;
  cpx<R> acc((R)0, (R)0);
  if (fine_in) acc = ld(fine_in + idx);
  for (int k = 0; k < nvec; ++k) acc = cmadd(acc, ld(phi + (long long)k * fs + e), ld(cf + k));
  st(fine + idx, acc);
}

// ---------------------------------------------------------------- launchers
template <typename R>
int launch_restrict(const hdcr_subspace* sub, const cpx<R>* fine, cpx<R>* coarse, int nrhs, cudaStream_t st) {
  dim3 grid(sub->bg.Vc, (sub->nvec + RP_KC - 1) / RP_KC, nrhs);
  // the table of the block's 4d sites in shared memory when it fits (48 KB), else
  // the sites are worked out per element
  const bool table = sub->bg.bvol <= 12 * 1024;
  const size_t smem = table ? sizeof(int) * (size_t)sub->bg.bvol : 0;
  restrict_kernel<R><<<grid, RED_THREADS, smem, st>>>(sub->g, sub->bg, (const cpx<R>*)sub->vecs, fine, coarse,
                                                      sub->nvec, table); count_launch();
  HDCR_LAUNCH_CHECK();
  return HDCR_OK;
}

template <typename R>
int launch_prolong(const hdcr_subspace* sub, const cpx<R>* coarse, const cpx<R>* fine_in, cpx<R>* fine,
                   int nrhs, cudaStream_t st) {
  const long long n = sub->g.V5 * 12 * nrhs;
  prolong_kernel<R><<<num_blocks(n, 256), 256, 0, st>>>(sub->g, sub->bg, (const cpx<R>*)sub->vecs, coarse,
                                                        fine_in, fine, sub->nvec, nrhs); count_launch();
  HDCR_LAUNCH_CHECK();
  return HDCR_OK;
}

template <typename R>
int launch_coarse_apply(const hdcr_coarse* co, const cpx<R>* in, cpx<R>* out, int nrhs, cudaStream_t st) {
  const long long n = (long long)co->bg.Vc * co->nvec * nrhs;
  coarse_apply_kernel<R><<<num_blocks(n, 128), 128, 0, st>>>((const cpx<R>*)co->A, co->nbr, in, out,
                                                             co->bg.Vc, co->nvec, nrhs); count_launch();
  HDCR_LAUNCH_CHECK();
  return HDCR_OK;
}

template <typename R>
int CoarseOp<R>::apply_dot(const cpx<R>* in, cpx<R>* out, RedScratch rs, double* res, cudaStream_t st) const {
  HDCR_TRY(launch_coarse_apply<R>(co, in, out, 1, st));
  const long long n = this->n();
  cdot_re_kernel<R><<<red_blocks(n), RED_THREADS, 0, st>>>(in, out, n, rs, res); count_launch();
  HDCR_LAUNCH_CHECK();
  return HDCR_OK;
}

#define HDCR_INST_COARSE(R)                                                                            \
  template int launch_restrict<R>(const hdcr_subspace*, const cpx<R>*, cpx<R>*, int, cudaStream_t);   \
  template int launch_prolong<R>(const hdcr_subspace*, const cpx<R>*, const cpx<R>*, cpx<R>*, int,    \
                                 cudaStream_t);                                                       \
  template int launch_coarse_apply<R>(const hdcr_coarse*, const cpx<R>*, cpx<R>*, int, cudaStream_t); \
  template struct CoarseOp<R>;
HDCR_INST_COARSE(double)
HDCR_INST_COARSE(float)

template <typename R, int MU>
static int launch_forward_leg(const Geom& g, const BlockGeom& bg, const cpx<R>* U, const cpx<R>* phi, cpx<R>* pt,
                              cpx<R>* hf, cpx<R>* A, int nvec, cpx<R>* part, int* err, int npass, cudaStream_t st) {
  const long long nf = bg.K5 / bg.b[MU];
  const long long n = (long long)bg.Vc * nf * nvec;
  face_kernel<R, MU><<<num_blocks(n, 256), 256, 0, st>>>(g, bg, U, phi, pt, hf, nvec, nf); count_launch();
  if constexpr (sizeof(R) == 4) {
    const TcSrc src{pt, hf, nf * 6, 0, g, bg};
    return launch_tc_project(src, A, nvec, leg_of(MU, +1), part, err, npass, st);
  } else {
    int T = (int)(48 * 1024 / (2 * (size_t)nvec * sizeof(cpx<R>)));
    if (T > 256) T = 256;
    const size_t smem = 2 * (size_t)nvec * T * sizeof(cpx<R>);
    face_project_kernel<R><<<bg.Vc, PROJ_THREADS, smem, st>>>(pt, hf, nf * 6, A, bg.Vc, nvec, leg_of(MU, +1), T); count_launch();
    HDCR_LAUNCH_CHECK();
    return HDCR_OK;
  }
}

template <typename R>
static int build_legs(const hdcr_subspace* sub, double M5, double mf, const cpx<R>* U, const cpx<R>* phi,
                      cpx<R>* Y, cpx<R>* face_work, cpx<R>* A, cpx<R>* part, cpx<R>* part2, int* err, int npass,
                      bool full_y, cudaStream_t st, cudaStream_t sf, cudaEvent_t fork) {
  const Geom& g = sub->g;
  const BlockGeom& bg = sub->bg;
  const int nvec = sub->nvec;
  // leg 0: in-block part of H on every site, upper triangle of the projection
  int T = (int)(48 * 1024 / (2 * (size_t)nvec * 12 * sizeof(cpx<R>)));
  if (T < 1) T = 1;
  if (T > 16) T = 16;
  const size_t smem = 2 * (size_t)nvec * 12 * T * sizeof(cpx<R>);
  const long long n = g.V5 * nvec;
  if (full_y) {
    HDCR_TRY(launch_g5dwf<R>(g, M5, mf, U, phi, Y, nvec, st));
  } else {
    leg_self_kernel<R><<<num_blocks(n, 256), 256, 0, st>>>(g, bg, (R)(5.0 - M5), (R)mf, U, phi, Y, nvec); count_launch();
    HDCR_LAUNCH_CHECK();
  }
  // forward legs on the block faces (six-component projections), on sf: they need
  // only phi and U, and run while st applies H and projects leg 0
  if (fork) HDCR_CUDA_TRY(cudaStreamWaitEvent(sf, fork, 0));
  long long nfmax = 0;
  for (int mu = 0; mu < 4; ++mu) nfmax = std::max(nfmax, bg.K5 / bg.b[mu]);
  cpx<R>* pt = face_work;
  cpx<R>* hf = face_work + (size_t)nvec * bg.Vc * nfmax * 6;
  HDCR_TRY((launch_forward_leg<R, 0>(g, bg, U, phi, pt, hf, A, nvec, part2, err, npass, sf)));
  HDCR_TRY((launch_forward_leg<R, 1>(g, bg, U, phi, pt, hf, A, nvec, part2, err, npass, sf)));
  HDCR_TRY((launch_forward_leg<R, 2>(g, bg, U, phi, pt, hf, A, nvec, part2, err, npass, sf)));
  HDCR_TRY((launch_forward_leg<R, 3>(g, bg, U, phi, pt, hf, A, nvec, part2, err, npass, sf)));
  if constexpr (sizeof(R) == 4) {
    const TcSrc src{phi, Y, bg.K5 * 12, 1, g, bg};
    HDCR_TRY(launch_tc_project(src, A, nvec, 0, part, err, npass, st));
  } else {
    project_kernel<R><<<bg.Vc, PROJ_THREADS, smem, st>>>(g, bg, phi, Y, A, nvec, 0, T, true); count_launch();
    HDCR_LAUNCH_CHECK();
  }
  return HDCR_OK;
}

// The nine legs of A.  The face legs go to a second stream (forked after the
// caller's earlier work on st and joined before the legs are completed); they
// write other legs of A and their own partial sums.  On any failure the second
// stream is drained before returning, so no kernel outlives the buffers.
template <typename R>
static int build_op(const hdcr_subspace* sub, double M5, double mf, const cpx<R>* U, const cpx<R>* phi,
                    cpx<R>* Y, cpx<R>* face_work, cpx<R>* A, const int* nbr, cpx<R>* part, cpx<R>* part2, int* err,
                    int npass, cudaStream_t st) {
  const BlockGeom& bg = sub->bg;
  const int nvec = sub->nvec;
  // FP32 with the packed stencil available: Y = H phi over all nvec fields in one
  // launch (the fastest FP32 stencil), leg 0 recovered afterwards by subtracting the
  // outward legs; otherwise Y = the in-block part of H only
  const bool full_y = sizeof(R) == 4 && g5dwf_x2_ok(sub->g, phi, Y);
  cudaStream_t s2 = nullptr;
  cudaEvent_t fork = nullptr, join = nullptr;
  bool two = cudaStreamCreateWithFlags(&s2, cudaStreamNonBlocking) == cudaSuccess;
  two = two && cudaEventCreateWithFlags(&fork, cudaEventDisableTiming) == cudaSuccess &&
        cudaEventCreateWithFlags(&join, cudaEventDisableTiming) == cudaSuccess &&
        cudaEventRecord(fork, st) == cudaSuccess;
  cudaGetLastError();  // a failed optional call above leaves no sticky error
  int status = build_legs<R>(sub, M5, mf, U, phi, Y, face_work, A, part, two ? part2 : part, err, npass, full_y,
                             st, two ? s2 : st, two ? fork : nullptr);
  if (two) {
    if (status == HDCR_OK) {
      const cudaError_t e = cudaEventRecord(join, s2);
      if (e == cudaSuccess) {
        const cudaError_t w = cudaStreamWaitEvent(st, join, 0);
        if (w != cudaSuccess) status = cuda_status(w, "coarse build: join of the face legs");
      } else {
        status = cuda_status(e, "coarse build: join of the face legs");
      }
    }
    if (status != HDCR_OK) cudaStreamSynchronize(s2);
  }
  if (s2) cudaStreamDestroy(s2);
  if (fork) cudaEventDestroy(fork);
  if (join) cudaEventDestroy(join);
  HDCR_TRY(status);
  // lower triangle of leg 0 and the backward legs from Hermiticity
  const long long nc = (long long)bg.Vc * 5 * nvec * nvec;
  complete_legs_kernel<R><<<num_blocks(nc, 256), 256, 0, st>>>(A, nbr, bg.Vc, nvec, !full_y); count_launch();
  HDCR_LAUNCH_CHECK();
  if (full_y) {
    const long long n2 = (long long)bg.Vc * nvec * nvec;
    subtract_legs_kernel<R><<<num_blocks(n2, 256), 256, 0, st>>>(A, bg.Vc, nvec); count_launch();
    HDCR_LAUNCH_CHECK();
  }
  return HDCR_OK;
}

}  // namespace hdcr

namespace hdcr {

int fill_neighbour_table(const BlockGeom& bg, int* nbr, cudaStream_t st) {
  std::vector<int> hn((size_t)bg.Vc * NLEGS);
  for (int a = 0; a < bg.Vc; ++a) {
    int c[4];
    coarse_coords(bg, a, c);
    hn[(size_t)a * NLEGS] = a;
    for (int mu = 0; mu < 4; ++mu)
      for (int sg = 0; sg < 2; ++sg) {
        int d[4] = {c[0], c[1], c[2], c[3]};
        d[mu] = (c[mu] + (sg == 0 ? 1 : -1) + bg.Lc[mu]) % bg.Lc[mu];
        hn[(size_t)a * NLEGS + leg_of(mu, sg == 0 ? 1 : -1)] =
            ((d[3] * bg.Lc[2] + d[2]) * bg.Lc[1] + d[1]) * bg.Lc[0] + d[0];
      }
  }
  cudaError_t e = cudaMemcpyAsync(nbr, hn.data(), sizeof(int) * hn.size(), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_status(e, "coarse neighbour table");
  return HDCR_OK;
}

}  // namespace hdcr

using namespace hdcr;

static int build_coarse_op_entry(const hdcr_subspace* sub, const hdcr_dwf_params* p, const void* U,
                                 int op_dtype, void* stream, hdcr_coarse** out) {
  HDCR_TRY(subspace_check(sub));
  if (!p || !U || !out) {
    set_error("hdcr_build_coarse_op: null pointer");
    return HDCR_ERR_BAD_ARG;
  }
  if (op_dtype != HDCR_C128 && op_dtype != HDCR_C64 && op_dtype != HDCR_C64_FAST && op_dtype != HDCR_C128_TC) {
    set_error("hdcr_build_coarse_op: unknown dtype %d", op_dtype);
    return HDCR_ERR_BAD_ARG;
  }
  // HDCR_C64_FAST: stored as C64, tensor-core products in one TF32 pass;
  // HDCR_C128_TC: built as C64 with the three-pass (FP32-exact) products, stored as C128
  const int npass = op_dtype == HDCR_C64_FAST ? 1 : 3;
  const bool store_c128 = op_dtype == HDCR_C128_TC;
  if (op_dtype == HDCR_C64_FAST || op_dtype == HDCR_C128_TC) op_dtype = HDCR_C64;
  if (sub->nvec > 64) {
    set_error("hdcr_build_coarse_op: nvec = %d above the supported 64", sub->nvec);
    return HDCR_ERR_BAD_ARG;
  }
  *out = nullptr;
  cudaStream_t st = as_stream(stream);
  const Geom& g = sub->g;
  const BlockGeom& bg = sub->bg;
  const int nvec = sub->nvec;
  const size_t cb = dtype_complex_bytes(op_dtype);
  const long long fs = g.V5 * 12;
  // workspace: Y (nvec fields), and basis / links converted to the build precision when needed
  const bool conv_phi = sub->dtype != op_dtype;
  const bool conv_u = op_dtype != HDCR_C128;
  long long nfmax = 0;
  for (int mu = 0; mu < 4; ++mu) nfmax = std::max(nfmax, bg.K5 / bg.b[mu]);
  const size_t face_bytes = cb * (size_t)2 * nvec * bg.Vc * nfmax * 6;
  // partial projections of the split tensor-core contractions (FP32 builds)
  // (two sets: the face legs run on their own stream)
  const size_t part_bytes = op_dtype == HDCR_C64 ? 2 * sizeof(cpx<float>) * TC_MAX_SPLIT * (size_t)bg.Vc * nvec * nvec : 0;
  const size_t a_bytes = cb * (size_t)bg.Vc * NLEGS * nvec * nvec;
  size_t bytes = cb * (size_t)fs * nvec + face_bytes + 256 + part_bytes + (store_c128 ? a_bytes : 0);
  if (conv_phi) bytes += cb * (size_t)fs * nvec;
  if (conv_u) bytes += cb * (size_t)g.V4 * 36;
  std::lock_guard<std::mutex> lock(sub->build_mu);
  if (sub->build_ws_bytes < bytes) {
    if (sub->build_ws) cudaFree(sub->build_ws);
    sub->build_ws = nullptr;
    sub->build_ws_bytes = 0;
    HDCR_CUDA_TRY(cudaMalloc(&sub->build_ws, bytes));
    sub->build_ws_bytes = bytes;
  }
  char* wp = (char*)sub->build_ws;
  void* Y = wp;
  wp += cb * (size_t)fs * nvec;
  void* face_work = wp;
  wp += face_bytes;
  int* err = (int*)wp;  // time-out flag of the tensor-core projections
  wp += 256;
  void* part = wp;
  wp += part_bytes;
  void* A_build = nullptr;  // the FP32 operator before its conversion (HDCR_C128_TC)
  if (store_c128) {
    A_build = wp;
    wp += a_bytes;
  }
  cudaMemsetAsync(err, 0, sizeof(int), st);
  const void* phi = sub->vecs;
  if (conv_phi) {
    phi = wp;
    launch_convert(sub->vecs, sub->dtype, wp, op_dtype, fs * nvec, st);
    wp += cb * (size_t)fs * nvec;
  }
  const void* Ub = U;
  if (conv_u) {
    Ub = wp;
    launch_convert(U, HDCR_C128, wp, op_dtype, (long long)g.V4 * 36, st);
  }
  hdcr_coarse* co = new hdcr_coarse();
  co->sub = sub;
  co->g = g;
  co->bg = bg;
  co->nvec = nvec;
  co->dtype = store_c128 ? HDCR_C128 : op_dtype;
  co->M5 = p->M5;
  co->mf = p->mf;
  cudaGetDevice(&co->device);
  int s = HDCR_OK;
  cudaError_t e = cudaMalloc(&co->A, dtype_complex_bytes(co->dtype) * (size_t)bg.Vc * NLEGS * nvec * nvec);
  if (!store_c128) A_build = co->A;
  if (e == cudaSuccess) e = cudaMalloc(&co->nbr, sizeof(int) * bg.Vc * NLEGS);
  if (e != cudaSuccess) s = cuda_status(e, "coarse operator storage");
  if (s == HDCR_OK) s = fill_neighbour_table(bg, co->nbr, st);
  if (s == HDCR_OK) {
    if (op_dtype == HDCR_C128)
      s = build_op<double>(sub, p->M5, p->mf, (const cpx<double>*)Ub, (const cpx<double>*)phi, (cpx<double>*)Y,
                           (cpx<double>*)face_work, (cpx<double>*)co->A, co->nbr, nullptr, nullptr, err, 3, st);
    else
      s = build_op<float>(sub, p->M5, p->mf, (const cpx<float>*)Ub, (const cpx<float>*)phi, (cpx<float>*)Y,
                          (cpx<float>*)face_work, (cpx<float>*)A_build, co->nbr, (cpx<float>*)part,
                          (cpx<float>*)part + TC_MAX_SPLIT * (size_t)bg.Vc * nvec * nvec, err, npass, st);
    if (s == HDCR_OK && store_c128)
      s = launch_convert(A_build, HDCR_C64, co->A, HDCR_C128, (long long)bg.Vc * NLEGS * nvec * nvec, st);
  }
  if (s == HDCR_OK) {
    int herr = 0;
    e = cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
      s = cuda_status(e, "coarse operator build");
    } else if (herr) {
      set_error("coarse operator build: a tensor-core projection timed out");
      s = HDCR_ERR_TIMEOUT;
    }
  }
  if (s != HDCR_OK) {
    hdcr_coarse_destroy(co);
    return s;
  }
  *out = co;
  return HDCR_OK;
}

extern "C" int hdcr_coarse_get_op(const hdcr_coarse* co, void* out, void* stream) {
  HDCR_TRY(coarse_check(co));
  if (!out) {
    set_error("hdcr_coarse_get_op: null output");
    return HDCR_ERR_BAD_ARG;
  }
  const long long n = (long long)co->bg.Vc * NLEGS * co->nvec * co->nvec;
  return launch_convert(co->A, co->dtype, out, HDCR_C128, n, as_stream(stream));
}

extern "C" int hdcr_apply_coarse(const hdcr_coarse* co, const void* in, void* out, int dtype, int nrhs,
                                 void* stream) {
  HDCR_TRY(coarse_check(co));
  if (!in || !out || in == out || nrhs < 1) {
    set_error("hdcr_apply_coarse: bad pointers or nrhs");
    return HDCR_ERR_BAD_ARG;
  }
  if (dtype != co->dtype) {
    set_error("hdcr_apply_coarse: vector dtype %d differs from the operator's %d", dtype, co->dtype);
    return HDCR_ERR_BAD_ARG;
  }
  if (dtype == HDCR_C128)
    return launch_coarse_apply<double>(co, (const cpx<double>*)in, (cpx<double>*)out, nrhs, as_stream(stream));
  return launch_coarse_apply<float>(co, (const cpx<float>*)in, (cpx<float>*)out, nrhs, as_stream(stream));
}

extern "C" int hdcr_restrict(const hdcr_subspace* sub, const void* fine, void* coarse, int dtype, int nrhs,
                             void* stream) {
  HDCR_TRY(subspace_check(sub));
  if (!fine || !coarse || nrhs < 1 || nrhs > 65535) {
    set_error("hdcr_restrict: bad pointers or nrhs");
    return HDCR_ERR_BAD_ARG;
  }
  if (dtype != sub->dtype) {
    set_error("hdcr_restrict: vector dtype %d differs from the basis storage %d", dtype, sub->dtype);
    return HDCR_ERR_BAD_ARG;
  }
  if (dtype == HDCR_C128)
    return launch_restrict<double>(sub, (const cpx<double>*)fine, (cpx<double>*)coarse, nrhs, as_stream(stream));
  return launch_restrict<float>(sub, (const cpx<float>*)fine, (cpx<float>*)coarse, nrhs, as_stream(stream));
}

extern "C" int hdcr_prolong(const hdcr_subspace* sub, const void* coarse, void* fine, int dtype, int nrhs,
                            void* stream) {
  HDCR_TRY(subspace_check(sub));
  if (!fine || !coarse || nrhs < 1) {
    set_error("hdcr_prolong: bad pointers or nrhs");
    return HDCR_ERR_BAD_ARG;
  }
  if (dtype != sub->dtype) {
    set_error("hdcr_prolong: vector dtype %d differs from the basis storage %d", dtype, sub->dtype);
    return HDCR_ERR_BAD_ARG;
  }
  if (dtype == HDCR_C128)
    return launch_prolong<double>(sub, (const cpx<double>*)coarse, nullptr, (cpx<double>*)fine, nrhs,
                                  as_stream(stream));
  return launch_prolong<float>(sub, (const cpx<float>*)coarse, nullptr, (cpx<float>*)fine, nrhs,
                               as_stream(stream));
}

extern "C" void hdcr_coarse_destroy(hdcr_coarse* co) {
  if (!co) return;
  solve_cache_release(co);
  multi_cache_release(co);
  if (co->A) cudaFree(co->A);
  if (co->nbr) cudaFree(co->nbr);
  if (co->Ainv) cudaFree(co->Ainv);
  if (co->dws) cudaFree(co->dws);
  level2_free(co->l2);
  cf_coef_free(co->cf);
  delete co;
}

extern "C" int hdcr_build_coarse_op(const hdcr_subspace* sub, const hdcr_dwf_params* p, const void* U,
                                    int op_dtype, void* stream, hdcr_coarse** out) {
  HDCR_TRY(subspace_check(sub));
  Staged su;  // links given in host memory are staged through the device
  HDCR_TRY(su.in(U, (size_t)sub->g.V4 * 36 * 16, as_stream(stream)));
  return build_coarse_op_entry(sub, p, su.ptr(), op_dtype, stream, out);
}
