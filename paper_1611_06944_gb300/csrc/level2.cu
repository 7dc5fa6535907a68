// A third level for the coarse solve: the two-level construction of Section 4
// applied to the little Dirac operator A itself (Section 5 names recursion as the
// way to solve the coarse system more exactly).
//
//  1. n2/2 noise vectors on the coarse lattice (drawn by the caller), each smoothed
//     by a fixed number of CR steps on A x = 0 and normalised;
//  2. split by the coarse Gamma5: the level-1 basis vectors have definite Gamma5
//     chirality (the nvec/2 P_+ vectors first), so P^dag Gamma5 P = diag(+1 x nvec/2,
//     -1 x nvec/2) on every coarse site;
//  3. blocks of b2 coarse sites times all nvec components, modified Gram-Schmidt
//     twice per block in FP64 (one CTA per block);
//  4. A2 = P2^dag A P2 on the level-2 lattice, 9 legs: for each leg the coarse
//     stencil restricted to the hops that leave a level-2 block in that direction
//     (the self leg: every other hop) is applied to all n2 basis vectors in one
//     launch and projected block by block;
//  5. A2's dense inverse (the FP32 Gauss-Jordan of coarse_dense.cu);
//  6. the coarse solve of the V-cycle (HDCR_COARSE_RECURSIVE): flexible GCR(8) on A
//     preconditioned by z1 = S r, z2 = z1 + P2 A2^{-1} P2^dag (r - A z1),
//     z = z2 + S (r - A z2), S a fixed number of CR steps on A from zero.  The GCR's
//     orthogonalisation runs on device scalars; the host reads one residual norm
//     per iteration.
//
// Layouts: level-2 basis phi2[n2][Vc][nvec] (coarse vectors, block-orthonormal
// within each level-2 block), A2[B][leg][j][k], level-2 vectors c2[B][j],
// B = ((t2*Z2 + z2)*Y2 + y2)*X2 + x2.
#include <cmath>
#include <vector>

#include "coarse.cuh"
#include "host_io.cuh"
#include "level2.cuh"

namespace hdcr {

namespace {

struct L2Geom {
  int Lc[4], b[4], L2[4];
  int Vc, Vc2, nvec, bvol;
};

__host__ __device__ inline int l2_block_of(const L2Geom& q, int a) {
  int c[4];
  c[0] = a % q.Lc[0];
  int r = a / q.Lc[0];
  c[1] = r % q.Lc[1];
  r /= q.Lc[1];
  c[2] = r % q.Lc[2];
  c[3] = r / q.Lc[2];
  return (((c[3] / q.b[3]) * q.L2[2] + c[2] / q.b[2]) * q.L2[1] + c[1] / q.b[1]) * q.L2[0] + c[0] / q.b[0];
}

// coarse site of local site l (x fastest) of level-2 block B
__device__ inline int l2_site(const L2Geom& q, int B, int l) {
  int bc[4];
  bc[0] = B % q.L2[0];
  int r = B / q.L2[0];
  bc[1] = r % q.L2[1];
  r /= q.L2[1];
  bc[2] = r % q.L2[2];
  bc[3] = r / q.L2[2];
  int c[4];
  c[0] = bc[0] * q.b[0] + l % q.b[0];
  int t = l / q.b[0];
  c[1] = bc[1] * q.b[1] + t % q.b[1];
  t /= q.b[1];
  c[2] = bc[2] * q.b[2] + t % q.b[2];
  c[3] = bc[3] * q.b[3] + t / q.b[2];
  return ((c[3] * q.Lc[2] + c[2]) * q.Lc[1] + c[1]) * q.Lc[0] + c[0];
}

// whether the coarse hop (mu, sign) from site a leaves its level-2 block
__device__ inline bool l2_crosses(const L2Geom& q, int a, int mu, int sign) {
  int c[4];
  c[0] = a % q.Lc[0];
  int r = a / q.Lc[0];
  c[1] = r % q.Lc[1];
  r /= q.Lc[1];
  c[2] = r % q.Lc[2];
  c[3] = r / q.Lc[2];
  const int m = c[mu] % q.b[mu];
  return sign > 0 ? m == q.b[mu] - 1 : m == 0;
}

// out[r][a][j] = sum over the selected legs of A[a][leg] in[r][nbr(a, leg)]; mode 0: the
// self leg and every hop that stays inside the level-2 block; mode d > 0: leg d where it
// leaves the block
template <typename R>
__global__ void l2_masked_apply_kernel(const cpx<R>* __restrict__ A, const int* __restrict__ nbr, L2Geom q,
                                       int mode, const cpx<R>* __restrict__ in, cpx<R>* __restrict__ out,
                                       int nrhs) {
  const long long n = (long long)q.Vc * q.nvec;
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= n * nrhs) return;
  const int r = (int)(idx / n);
  const long long rem = idx - (long long)r * n;
  const int a = (int)(rem / q.nvec);
  const int j = (int)(rem - (long long)a * q.nvec);
  const cpx<R>* x = in + (long long)r * n;
  cpx<R> acc((R)0, (R)0);
  for (int d = 0; d < NLEGS; ++d) {
    bool use;
    if (d == 0) {
      use = mode == 0;
    } else {
      const int mu = (d - 1) >> 1, sg = (d - 1) & 1 ? -1 : 1;
      const bool cross = l2_crosses(q, a, mu, sg);
      use = mode == 0 ? !cross : (mode == d && cross);
    }
    if (!use) continue;
    const cpx<R>* row = A + (((long long)a * NLEGS + d) * q.nvec + j) * q.nvec;
    const cpx<R>* xb = x + (long long)nbr[a * NLEGS + d] * q.nvec;
    for (int k = 0; k < q.nvec; ++k) acc = cmadd(acc, ld(row + k), ld(xb + k));
  }
  st(out + idx, acc);
}

// A2[B][leg][j][k] = sum_{a in B, i} conj(phi2[j][a][i]) Y[k][a][i]
template <typename R>
__global__ void l2_project_kernel(const cpx<R>* __restrict__ phi2, const cpx<R>* __restrict__ Y, L2Geom q, int n2,
                                  int leg, cpx<R>* __restrict__ A2) {
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (long long)q.Vc2 * n2 * n2) return;
  const int k = (int)(idx % n2);
  const int j = (int)((idx / n2) % n2);
  const int B = (int)(idx / ((long long)n2 * n2));
  const long long cs = (long long)q.Vc * q.nvec;
  double re = 0.0, im = 0.0;
  for (int l = 0; l < q.bvol; ++l) {
    const long long o = (long long)l2_site(q, B, l) * q.nvec;
    for (int i = 0; i < q.nvec; ++i) {
      const cpx<R> p = ld(phi2 + (long long)j * cs + o + i), y = ld(Y + (long long)k * cs + o + i);
      re += (double)p.re * y.re + (double)p.im * y.im;
      im += (double)p.re * y.im - (double)p.im * y.re;
    }
  }
  st(A2 + (((long long)B * NLEGS + leg) * n2 + j) * n2 + k, cpx<R>((R)re, (R)im));
}

// c2[r][B][j] = sum_{a in B, i} conj(phi2[j][a][i]) v[r][a][i]
template <typename R>
__global__ void l2_restrict_kernel(const cpx<R>* __restrict__ phi2, const cpx<R>* __restrict__ v, L2Geom q, int n2,
                                   cpx<R>* __restrict__ c2, int nrhs) {
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (long long)nrhs * q.Vc2 * n2) return;
  const int j = (int)(idx % n2);
  const int B = (int)((idx / n2) % q.Vc2);
  const int r = (int)(idx / ((long long)n2 * q.Vc2));
  const long long cs = (long long)q.Vc * q.nvec;
  double re = 0.0, im = 0.0;
  for (int l = 0; l < q.bvol; ++l) {
    const long long o = (long long)l2_site(q, B, l) * q.nvec;
    for (int i = 0; i < q.nvec; ++i) {
      const cpx<R> p = ld(phi2 + (long long)j * cs + o + i), y = ld(v + (long long)r * cs + o + i);
      re += (double)p.re * y.re + (double)p.im * y.im;
      im += (double)p.re * y.im - (double)p.im * y.re;
    }
  }
  st(c2 + idx, cpx<R>((R)re, (R)im));
}

// v[r][a][i] = (add ? v[r][a][i] : 0) + sum_j c2[r][B(a)][j] phi2[j][a][i]
template <typename R>
__global__ void l2_prolong_kernel(const cpx<R>* __restrict__ phi2, const cpx<R>* __restrict__ c2, L2Geom q, int n2,
                                  cpx<R>* __restrict__ v, int nrhs, bool add) {
  const long long cs = (long long)q.Vc * q.nvec;
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (long long)nrhs * cs) return;
  const int r = (int)(idx / cs);
  const long long e = idx - (long long)r * cs;
  const int a = (int)(e / q.nvec);
  const int B = l2_block_of(q, a);
  const cpx<R>* c = c2 + ((long long)r * q.Vc2 + B) * n2;
  double re = 0.0, im = 0.0;
  for (int j = 0; j < n2; ++j) {
    const cpx<R> p = ld(phi2 + (long long)j * cs + e), cj = ld(c + j);
    re += (double)cj.re * p.re - (double)cj.im * p.im;
    im += (double)cj.re * p.im + (double)cj.im * p.re;
  }
  if (add) {
    const cpx<R> o = ld(v + idx);
    re += o.re;
    im += o.im;
  }
  st(v + idx, cpx<R>((R)re, (R)im));
}

// (1 +- Gamma5c)/2 of h smoothed vectors s: phi[0..h) the + halves, phi[h..2h) the - halves (FP64)
template <typename R>
__global__ void l2_split_kernel(const cpx<R>* __restrict__ s, int h, long long cs, int nvec,
                                cpx<double>* __restrict__ phi) {
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (long long)h * cs) return;
  const int i = (int)(idx % nvec);
  const cpx<R> v = ld(s + idx);
  const cpx<double> vd((double)v.re, (double)v.im), z(0.0, 0.0);
  const bool plus = i < nvec / 2;
  const long long v0 = idx / cs, e = idx - v0 * cs;
  st(phi + v0 * cs + e, plus ? vd : z);
  st(phi + (v0 + h) * cs + e, plus ? z : vd);
}

// Modified Gram-Schmidt, twice, in every level-2 block (one CTA per block), FP64, in
// place; *rank = 1 + (first dependent vector's index) when a vector has nothing left
__global__ void __launch_bounds__(256) l2_block_gs_kernel(cpx<double>* __restrict__ phi, L2Geom q, int n2,
                                                          int* __restrict__ rank) {
  __shared__ double red[2][8];
  const int B = blockIdx.x;
  const long long cs = (long long)q.Vc * q.nvec;
  const int K2 = q.bvol * q.nvec;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  auto elem = [&](int v, int e) -> cpx<double>* {
    return phi + (long long)v * cs + (long long)l2_site(q, B, e / q.nvec) * q.nvec + e % q.nvec;
  };
  // sum over the CTA of (re, im)
  auto csum = [&](double re, double im, double* ore, double* oim) {
    for (int off = 16; off > 0; off >>= 1) {
      re += __shfl_down_sync(0xffffffffu, re, off);
      im += __shfl_down_sync(0xffffffffu, im, off);
    }
    __syncthreads();
    if (lane == 0) {
      red[0][warp] = re;
      red[1][warp] = im;
    }
    __syncthreads();
    double a = 0.0, b = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
      a += red[0][w];
      b += red[1][w];
    }
    *ore = a;
    *oim = b;
  };
  for (int k = 0; k < n2; ++k) {
    double n0, dummy;
    {
      double s = 0.0;
      for (int e = tid; e < K2; e += blockDim.x) {
        const cpx<double> v = *elem(k, e);
        s += v.re * v.re + v.im * v.im;
      }
      csum(s, 0.0, &n0, &dummy);
    }
    for (int pass = 0; pass < 2; ++pass)
      for (int j = 0; j < k; ++j) {
        double re = 0.0, im = 0.0;
        for (int e = tid; e < K2; e += blockDim.x) {
          const cpx<double> p = *elem(j, e), v = *elem(k, e);
          re += p.re * v.re + p.im * v.im;
          im += p.re * v.im - p.im * v.re;
        }
        double dr, di;
        csum(re, im, &dr, &di);
        for (int e = tid; e < K2; e += blockDim.x) {
          cpx<double>* v = elem(k, e);
          const cpx<double> p = *elem(j, e);
          v->re -= dr * p.re - di * p.im;
          v->im -= dr * p.im + di * p.re;
        }
        __syncthreads();
      }
    double nn;
    {
      double s = 0.0;
      for (int e = tid; e < K2; e += blockDim.x) {
        const cpx<double> v = *elem(k, e);
        s += v.re * v.re + v.im * v.im;
      }
      csum(s, 0.0, &nn, &dummy);
    }
    if (!(nn > 1e-24 * n0)) {
      if (tid == 0) atomicCAS(rank, 0, 1 + k);
      return;
    }
    const double inv = 1.0 / sqrt(nn);
    for (int e = tid; e < K2; e += blockDim.x) {
      cpx<double>* v = elem(k, e);
      v->re *= inv;
      v->im *= inv;
    }
    __syncthreads();
  }
}

// y -= c x with c = (s[0], s[1]) (device); with conj_neg, c = -(s[0], s[1]) and y += ... (same)
template <typename R>
__global__ void l2_axpy_dev_kernel(cpx<R>* __restrict__ y, const cpx<R>* __restrict__ x, const double* __restrict__ s,
                                   double sign, long long n) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double cr = sign * s[0], ci = sign * s[1];
  const cpx<R> a = ld(x + i), b = ld(y + i);
  st(y + i, cpx<R>((R)(b.re + cr * a.re - ci * a.im), (R)(b.im + cr * a.im + ci * a.re)));
}

// y *= 1 / sqrt(*nrm2) for two vectors
template <typename R>
__global__ void l2_scale2_kernel(cpx<R>* __restrict__ u, cpx<R>* __restrict__ w, const double* __restrict__ nrm2,
                                 long long n) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double f = 1.0 / sqrt(*nrm2);
  const cpx<R> a = ld(u + i), b = ld(w + i);
  st(u + i, cpx<R>((R)(a.re * f), (R)(a.im * f)));
  st(w + i, cpx<R>((R)(b.re * f), (R)(b.im * f)));
}

template <typename R>
__global__ void l2_normalise_kernel(cpx<R>* __restrict__ u, const double* __restrict__ nrm2, long long n) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double f = 1.0 / sqrt(*nrm2);
  const cpx<R> a = ld(u + i);
  st(u + i, cpx<R>((R)(a.re * f), (R)(a.im * f)));
}

template <typename Ri, typename Ro>
__global__ void l2_copy_kernel(const cpx<Ri>* __restrict__ in, cpx<Ro>* __restrict__ out, long long n) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const cpx<Ri> a = ld(in + i);
  st(out + i, cpx<Ro>((Ro)a.re, (Ro)a.im));
}

// r = b - y
template <typename R>
__global__ void l2_sub_kernel(const cpx<R>* __restrict__ b, const cpx<R>* __restrict__ y, cpx<R>* __restrict__ r,
                              long long n) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const cpx<R> a = ld(b + i), c = ld(y + i);
  st(r + i, cpx<R>(a.re - c.re, a.im - c.im));
}

constexpr int L2_RESTART = 8;

}  // namespace

// The third level attached to a coarse handle.
struct Level2 {
  L2Geom q{};
  int n2 = 0, smooth = 0, dtype = 0;
  void* phi2 = nullptr;     // [n2][Vc][nvec] in the level-1 precision
  hdcr_coarse* co2 = nullptr;
  // workspace of the recursive coarse solve (level-1 precision): Z, W (restart each), r, t1, t2, x,
  // level-2 vectors c2, e2
  void* ws = nullptr;
  void* crw = nullptr;      // CRWork of the smoother
  RedBuffers rb{};          // scalars: [0, 2 * restart) MGS coefficients, 2*restart.. norms
};

void level2_free(Level2* l) {
  if (!l) return;
  if (l->crw) {
    if (l->dtype == HDCR_C128) {
      crwork_free<double>((CRWork<double>*)l->crw);
      delete (CRWork<double>*)l->crw;
    } else {
      crwork_free<float>((CRWork<float>*)l->crw);
      delete (CRWork<float>*)l->crw;
    }
  }
  if (l->phi2) cudaFree(l->phi2);
  if (l->ws) cudaFree(l->ws);
  red_buffers_free(&l->rb);
  if (l->co2) {
    if (l->co2->A) cudaFree(l->co2->A);
    if (l->co2->nbr) cudaFree(l->co2->nbr);
    if (l->co2->Ainv) cudaFree(l->co2->Ainv);
    if (l->co2->dws) cudaFree(l->co2->dws);
    delete l->co2;
  }
  delete l;
}

namespace {

template <typename R>
int l2_vcycle(const hdcr_coarse* co, Level2* l, const cpx<R>* r, cpx<R>* z, cudaStream_t st);

template <typename R>
int build_impl(hdcr_coarse* co, const hdcr_level2_params* p, const void* noise, Level2* l, cudaStream_t st) {
  const L2Geom& q = l->q;
  const long long cs = (long long)q.Vc * q.nvec;
  const int n2 = l->n2, h = n2 / 2;
  const int nb = 256;
  // 1. smoothing: CR steps on A x = 0 from each noise vector, normalised
  cpx<R>* s = nullptr;
  cpx<R>* zero = nullptr;
  cpx<double>* phi = nullptr;
  HDCR_CUDA_TRY(cudaMalloc(&s, sizeof(cpx<R>) * (size_t)(h * cs + cs)));
  zero = s + h * cs;
  int status = HDCR_OK;
  auto fail = [&](int st_) {
    if (status == HDCR_OK) status = st_;
  };
  if (cudaMalloc(&phi, sizeof(cpx<double>) * (size_t)(n2 * cs)) != cudaSuccess) fail(HDCR_ERR_NO_MEMORY);
  if (status == HDCR_OK && cudaMemsetAsync(zero, 0, sizeof(cpx<R>) * cs, st) != cudaSuccess) fail(HDCR_ERR_CUDA);
  CRWork<R>* cw = (CRWork<R>*)l->crw;
  if (status == HDCR_OK) {
    l2_copy_kernel<double, R><<<num_blocks(h * cs, nb), nb, 0, st>>>((const cpx<double>*)noise, s, h * cs);
    count_launch();
    CoarseOp<R> A{co};
    CRConfig cfg;
    cfg.fixed_iters = p->smooth_iters;
    for (int v = 0; v < h && status == HDCR_OK; ++v) {
      CRResult res;
      fail(cr_run<R>(A, zero, s + v * cs, *cw, cfg, &res, st));
      if (status != HDCR_OK) break;
      fail(launch_norm2<R>(s + v * cs, cs, l->rb.rs, l->rb.scal, st));
      l2_normalise_kernel<R><<<num_blocks(cs, nb), nb, 0, st>>>(s + v * cs, l->rb.scal, cs);
      count_launch();
    }
  }
  // 2. chiral split; 3. block Gram-Schmidt (FP64)
  int* rank = nullptr;
  if (status == HDCR_OK) {
    l2_split_kernel<R><<<num_blocks(h * cs, nb), nb, 0, st>>>(s, h, cs, q.nvec, phi);
    count_launch();
    rank = reinterpret_cast<int*>(l->rb.scal + 60);
    if (cudaMemsetAsync(rank, 0, sizeof(int), st) != cudaSuccess) fail(HDCR_ERR_CUDA);
    l2_block_gs_kernel<<<q.Vc2, 256, 0, st>>>(phi, q, n2, rank);
    count_launch();
    l2_copy_kernel<double, R><<<num_blocks(n2 * cs, nb), nb, 0, st>>>(phi, (cpx<R>*)l->phi2, n2 * cs);
    count_launch();
    int hr = 0;
    if (cudaMemcpyAsync(&hr, rank, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess) {
      fail(HDCR_ERR_CUDA);
    } else if (hr) {
      set_error("level-2 subspace: vector %d is linearly dependent in a level-2 block", hr - 1);
      fail(HDCR_ERR_RANK_DEFICIENT);
    }
  }
  // 4. A2: the masked stencil on all n2 basis vectors, projected leg by leg (Y reuses phi's room)
  if (status == HDCR_OK) {
    cpx<R>* Y = reinterpret_cast<cpx<R>*>(phi);
    for (int d = 0; d < NLEGS && status == HDCR_OK; ++d) {
      l2_masked_apply_kernel<R><<<num_blocks(n2 * cs, 128), 128, 0, st>>>((const cpx<R>*)co->A, co->nbr, q, d,
                                                                          (const cpx<R>*)l->phi2, Y, n2);
      count_launch();
      const long long np = (long long)q.Vc2 * n2 * n2;
      l2_project_kernel<R><<<num_blocks(np, 128), 128, 0, st>>>((const cpx<R>*)l->phi2, Y, q, n2, d,
                                                               (cpx<R>*)l->co2->A);
      count_launch();
    }
    if (cudaGetLastError() != cudaSuccess) fail(HDCR_ERR_CUDA);
  }
  cudaStreamSynchronize(st);
  cudaFree(s);
  if (phi) cudaFree(phi);
  // 5. the dense inverse of A2
  if (status == HDCR_OK) status = coarse_invert(l->co2, st);
  return status;
}

}  // namespace

int level2_build(hdcr_coarse* co, const hdcr_level2_params* p, const void* noise, cudaStream_t st) {
  const int n1 = co->nvec;
  if (!p || !noise || p->nvec2 < 2 || p->nvec2 % 2 || p->nvec2 > 64 || p->smooth_iters < 0 || p->cycle_smooth < 0) {
    set_error("hdcr_coarse_build_level2: bad parameters (nvec2 even in 2..64, iterations >= 0)");
    return HDCR_ERR_BAD_ARG;
  }
  Level2* l = new Level2();
  L2Geom& q = l->q;
  q.Vc = co->bg.Vc;
  q.nvec = n1;
  q.Vc2 = 1;
  q.bvol = 1;
  for (int mu = 0; mu < 4; ++mu) {
    q.Lc[mu] = co->bg.Lc[mu];
    q.b[mu] = p->block[mu];
    if (q.b[mu] < 1 || q.Lc[mu] % q.b[mu] || q.Lc[mu] / q.b[mu] < 2) {
      set_error("hdcr_coarse_build_level2: block %d does not divide the coarse extent %d into >= 2", q.b[mu],
                q.Lc[mu]);
      delete l;
      return HDCR_ERR_BAD_GEOMETRY;
    }
    q.L2[mu] = q.Lc[mu] / q.b[mu];
    q.Vc2 *= q.L2[mu];
    q.bvol *= q.b[mu];
  }
  l->n2 = p->nvec2;
  l->smooth = p->cycle_smooth;
  l->dtype = co->dtype;
  const size_t cb = dtype_complex_bytes(co->dtype);
  const long long cs = (long long)q.Vc * n1;
  const int n2 = l->n2;
  int s = HDCR_OK;
  // level-2 handle: A2 in the level-1 precision, its neighbour table
  hdcr_coarse* c2 = new hdcr_coarse();
  l->co2 = c2;
  c2->sub = co->sub;
  c2->nvec = n2;
  c2->dtype = co->dtype;
  c2->bg.Vc = q.Vc2;
  for (int mu = 0; mu < 4; ++mu) {
    c2->bg.Lc[mu] = q.L2[mu];
    c2->bg.b[mu] = q.b[mu];
  }
  c2->M5 = co->M5;
  c2->mf = co->mf;
  c2->device = co->device;
  if (cudaMalloc(&c2->A, cb * (size_t)q.Vc2 * NLEGS * n2 * n2) != cudaSuccess ||
      cudaMalloc(&c2->nbr, sizeof(int) * (size_t)q.Vc2 * NLEGS) != cudaSuccess ||
      cudaMalloc(&l->phi2, cb * (size_t)n2 * cs) != cudaSuccess ||
      cudaMalloc(&l->ws, cb * (size_t)((2 * L2_RESTART + 4) * cs + 2 * (long long)q.Vc2 * n2)) != cudaSuccess) {
    cudaGetLastError();
    s = HDCR_ERR_NO_MEMORY;
    set_error("hdcr_coarse_build_level2: out of device memory");
  }
  if (s == HDCR_OK) s = red_buffers_alloc(&l->rb, 64);
  if (s == HDCR_OK) {
    std::vector<int> hn((size_t)q.Vc2 * NLEGS);
    for (int B = 0; B < q.Vc2; ++B) {
      int c[4];
      c[0] = B % q.L2[0];
      int r = B / q.L2[0];
      c[1] = r % q.L2[1];
      r /= q.L2[1];
      c[2] = r % q.L2[2];
      c[3] = r / q.L2[2];
      hn[(size_t)B * NLEGS] = B;
      for (int mu = 0; mu < 4; ++mu)
        for (int sg = 0; sg < 2; ++sg) {
          int d[4] = {c[0], c[1], c[2], c[3]};
          d[mu] = (d[mu] + (sg == 0 ? 1 : q.L2[mu] - 1)) % q.L2[mu];
          hn[(size_t)B * NLEGS + leg_of(mu, sg == 0 ? 1 : -1)] = ((d[3] * q.L2[2] + d[2]) * q.L2[1] + d[1]) * q.L2[0] + d[0];
        }
    }
    if (cudaMemcpyAsync(c2->nbr, hn.data(), sizeof(int) * hn.size(), cudaMemcpyHostToDevice, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
      s = cuda_status(cudaGetLastError(), "level-2 neighbour table");
  }
  if (s == HDCR_OK) {
    if (co->dtype == HDCR_C128) {
      CRWork<double>* w = new CRWork<double>();
      l->crw = w;
      s = crwork_alloc<double>(w, cs);
      if (s == HDCR_OK) s = build_impl<double>(co, p, noise, l, st);
    } else {
      CRWork<float>* w = new CRWork<float>();
      l->crw = w;
      s = crwork_alloc<float>(w, cs);
      if (s == HDCR_OK) s = build_impl<float>(co, p, noise, l, st);
    }
  }
  if (s != HDCR_OK) {
    level2_free(l);
    return s;
  }
  level2_free(co->l2);
  co->l2 = l;
  return HDCR_OK;
}

namespace {

// z = B2 r: the V-cycle one level down (smoother CR steps on A, exact level-2 correction)
template <typename R>
int l2_vcycle(const hdcr_coarse* co, Level2* l, const cpx<R>* r, cpx<R>* z, cudaStream_t st) {
  const L2Geom& q = l->q;
  const long long cs = (long long)q.Vc * q.nvec;
  const int nb = 256;
  cpx<R>* base = (cpx<R>*)l->ws;
  cpx<R>* t1 = base + (2 * L2_RESTART + 1) * cs;
  cpx<R>* t2 = t1 + cs;
  cpx<R>* c2 = base + (2 * L2_RESTART + 4) * cs;
  cpx<R>* e2 = c2 + (long long)q.Vc2 * l->n2;
  CoarseOp<R> A{co};
  CRWork<R>& cw = *(CRWork<R>*)l->crw;
  CRConfig cfg;
  cfg.fixed_iters = l->smooth;
  cfg.x_zero = true;
  // z1 = S r
  HDCR_CUDA_TRY(cudaMemsetAsync(z, 0, sizeof(cpx<R>) * cs, st));
  HDCR_TRY(cr_run<R>(A, r, z, cw, cfg, nullptr, st));
  // z2 = z1 + P2 A2^{-1} P2^dag (r - A z1)
  HDCR_TRY(A.apply(z, t1, st));
  l2_sub_kernel<R><<<num_blocks(cs, nb), nb, 0, st>>>(r, t1, t2, cs);
  count_launch();
  l2_restrict_kernel<R><<<num_blocks((long long)q.Vc2 * l->n2, 128), 128, 0, st>>>((const cpx<R>*)l->phi2, t2, q,
                                                                                  l->n2, c2, 1);
  count_launch();
  HDCR_TRY(launch_dense_solve<R>(l->co2, c2, e2, 1, st));
  l2_prolong_kernel<R><<<num_blocks(cs, nb), nb, 0, st>>>((const cpx<R>*)l->phi2, e2, q, l->n2, z, 1, true);
  count_launch();
  // z = z2 + S (r - A z2)
  HDCR_TRY(A.apply(z, t1, st));
  l2_sub_kernel<R><<<num_blocks(cs, nb), nb, 0, st>>>(r, t1, t2, cs);
  count_launch();
  HDCR_CUDA_TRY(cudaMemsetAsync(t1, 0, sizeof(cpx<R>) * cs, st));
  HDCR_TRY(cr_run<R>(A, t2, t1, cw, cfg, nullptr, st));
  l2_axpy_dev_kernel<R><<<num_blocks(cs, nb), nb, 0, st>>>(z, t1, l->rb.scal + 62, 1.0, cs);  // scal[62] = (1, 0)
  count_launch();
  HDCR_LAUNCH_CHECK();
  return HDCR_OK;
}

}  // namespace

// x = A^{-1} b (coarse vectors in R) by flexible GCR(8) on A preconditioned with the
// level-2 V-cycle, to |b - A x| <= tol |b| or max_iter iterations.
template <typename R>
int level2_solve(const hdcr_coarse* co, const cpx<R>* b, cpx<R>* x, double tol, int max_iter, int* iters,
                 cudaStream_t st) {
  Level2* l = co->l2;
  if (!l) {
    set_error("recursive coarse solve: no third level (call hdcr_coarse_build_level2)");
    return HDCR_ERR_BAD_ARG;
  }
  const L2Geom& q = l->q;
  const long long cs = (long long)q.Vc * q.nvec;
  const int nb = 256;
  cpx<R>* base = (cpx<R>*)l->ws;
  cpx<R>* Z = base;
  cpx<R>* W = base + L2_RESTART * cs;
  cpx<R>* r = base + 2 * L2_RESTART * cs;
  cpx<R>* t1 = r + cs;
  double* sc = l->rb.scal;  // [0, 16): MGS coefficients (re, im); 16: |w|^2; 18: <w, r>; 20: |r|^2; 21: |b|^2
  RedScratch rs = l->rb.rs;
  CoarseOp<R> A{co};
  const double one[2] = {1.0, 0.0};
  HDCR_CUDA_TRY(cudaMemcpyAsync(sc + 62, one, 2 * sizeof(double), cudaMemcpyHostToDevice, st));
  HDCR_CUDA_TRY(cudaMemsetAsync(x, 0, sizeof(cpx<R>) * cs, st));
  l2_copy_kernel<R, R><<<num_blocks(cs, nb), nb, 0, st>>>(b, r, cs);
  count_launch();
  HDCR_TRY(launch_norm2<R>(b, cs, rs, sc + 21, st));
  double* ring = pinned_ring();
  if (!ring) {
    set_error("pinned host buffer unavailable");
    return HDCR_ERR_NO_MEMORY;
  }
  HDCR_CUDA_TRY(cudaMemcpyAsync(ring, sc + 21, sizeof(double), cudaMemcpyDeviceToHost, st));
  HDCR_CUDA_TRY(cudaStreamSynchronize(st));
  const double bb = ring[0];
  if (!(bb == bb) || bb > 1e300) {
    set_error("recursive coarse solve: non-finite right-hand side");
    return HDCR_ERR_NONFINITE;
  }
  int it = 0;
  if (bb == 0.0) {
    *iters = 0;
    return HDCR_OK;
  }
  bool conv = false;
  while (!conv && it < max_iter) {
    for (int i = 0; i < L2_RESTART && it < max_iter; ++i, ++it) {
      cpx<R>* z = Z + i * cs;
      cpx<R>* w = W + i * cs;
      HDCR_TRY(l2_vcycle<R>(co, l, r, z, st));
      HDCR_TRY(A.apply(z, w, st));
      for (int j = 0; j < i; ++j) {  // modified Gram-Schmidt, coefficients on the device
        HDCR_TRY(launch_cdot<R>(W + j * cs, w, cs, rs, sc + 2 * j, st));
        l2_axpy_dev_kernel<R><<<num_blocks(cs, nb), nb, 0, st>>>(w, W + j * cs, sc + 2 * j, -1.0, cs);
        l2_axpy_dev_kernel<R><<<num_blocks(cs, nb), nb, 0, st>>>(z, Z + j * cs, sc + 2 * j, -1.0, cs);
        count_launches(2);
      }
      HDCR_TRY(launch_norm2<R>(w, cs, rs, sc + 16, st));
      l2_scale2_kernel<R><<<num_blocks(cs, nb), nb, 0, st>>>(z, w, sc + 16, cs);
      count_launch();
      HDCR_TRY(launch_cdot<R>(w, r, cs, rs, sc + 18, st));
      l2_axpy_dev_kernel<R><<<num_blocks(cs, nb), nb, 0, st>>>(x, z, sc + 18, 1.0, cs);
      l2_axpy_dev_kernel<R><<<num_blocks(cs, nb), nb, 0, st>>>(r, w, sc + 18, -1.0, cs);
      count_launches(2);
      HDCR_TRY(launch_norm2<R>(r, cs, rs, sc + 20, st));
      HDCR_CUDA_TRY(cudaMemcpyAsync(ring, sc + 20, sizeof(double), cudaMemcpyDeviceToHost, st));
      HDCR_CUDA_TRY(cudaStreamSynchronize(st));
      const double rr = ring[0];
      if (!(rr == rr) || rr > 1e300) {
        set_error("recursive coarse solve: non-finite residual");
        return HDCR_ERR_NONFINITE;
      }
      if (rr <= tol * tol * bb) {
        conv = true;
        ++it;
        break;
      }
    }
    if (!conv) {  // restart from the true residual
      HDCR_TRY(A.apply(x, t1, st));
      l2_sub_kernel<R><<<num_blocks(cs, nb), nb, 0, st>>>(b, t1, r, cs);
      count_launch();
    }
  }
  HDCR_LAUNCH_CHECK();
  *iters = it;
  return HDCR_OK;
}
template int level2_solve<double>(const hdcr_coarse*, const cpx<double>*, cpx<double>*, double, int, int*,
                                  cudaStream_t);
template int level2_solve<float>(const hdcr_coarse*, const cpx<float>*, cpx<float>*, double, int, int*,
                                 cudaStream_t);

}  // namespace hdcr

using namespace hdcr;

extern "C" int hdcr_coarse_build_level2(hdcr_coarse* co, const hdcr_level2_params* p, const void* noise,
                                        void* stream) {
  HDCR_TRY(coarse_check(co));
  if (!p || !noise) {
    set_error("hdcr_coarse_build_level2: null pointer");
    return HDCR_ERR_BAD_ARG;
  }
  cudaStream_t st = as_stream(stream);
  Staged sn;  // noise given in host memory is staged through the device
  HDCR_TRY(sn.in(noise, (size_t)(p->nvec2 > 0 ? p->nvec2 / 2 : 0) * co->bg.Vc * co->nvec * 16, st));
  return level2_build(co, p, sn.ptr(), st);
}

extern "C" int hdcr_coarse_level2_info(const hdcr_coarse* co, int* nvec2, int L2[4]) {
  HDCR_TRY(coarse_check(co));
  if (!nvec2 || !L2) {
    set_error("hdcr_coarse_level2_info: null pointer");
    return HDCR_ERR_BAD_ARG;
  }
  if (!co->l2) {
    *nvec2 = 0;
    return HDCR_OK;
  }
  *nvec2 = co->l2->n2;
  for (int mu = 0; mu < 4; ++mu) L2[mu] = co->l2->q.L2[mu];
  return HDCR_OK;
}

extern "C" int hdcr_coarse_level2_get(const hdcr_coarse* co, void* vectors, void* op, void* stream) {
  HDCR_TRY(coarse_check(co));
  if (!co->l2 || !vectors || !op) {
    set_error("hdcr_coarse_level2_get: no third level or null pointer");
    return HDCR_ERR_BAD_ARG;
  }
  const Level2* l = co->l2;
  cudaStream_t st = as_stream(stream);
  const long long nv = (long long)l->n2 * l->q.Vc * l->q.nvec;
  const long long na = (long long)l->q.Vc2 * NLEGS * l->n2 * l->n2;
  HDCR_TRY(launch_convert(l->phi2, l->dtype, vectors, HDCR_C128, nv, st));
  HDCR_TRY(launch_convert(l->co2->A, l->dtype, op, HDCR_C128, na, st));
  return HDCR_OK;
}

extern "C" int hdcr_coarse_solve_level2(const hdcr_coarse* co, const void* in, void* out, double tol, int max_iter,
                                        int* iters, void* stream) {
  HDCR_TRY(coarse_check(co));
  if (!in || !out || in == out || !(tol > 0.0) || max_iter < 1 || !iters) {
    set_error("hdcr_coarse_solve_level2: bad pointers, tol or max_iter");
    return HDCR_ERR_BAD_ARG;
  }
  if (co->dtype == HDCR_C128)
    return level2_solve<double>(co, (const cpx<double>*)in, (cpx<double>*)out, tol, max_iter, iters,
                                as_stream(stream));
  return level2_solve<float>(co, (const cpx<float>*)in, (cpx<float>*)out, tol, max_iter, iters, as_stream(stream));
}
