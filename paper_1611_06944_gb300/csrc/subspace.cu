// Subspace of the two-level preconditioner (Section 4):
//   noise -> a fixed number of CR steps on H x = 0 ("inverse iteration applied
//   to Gaussian noise") -> normalise -> chiral split with Gamma5 = gamma5 R5
//   -> restriction to blocks (Eq. 4.1) -> block orthonormalisation, so that
//   P_S = sum |phi_k^b><phi_k^b| (Eq. 4.3) is a projector (Cholesky QR twice,
//   Gram-Schmidt for ill-conditioned blocks).
// All of it runs in FP64; the basis is then stored in the requested dtype.
#include <vector>

#include "host_io.cuh"
#include "chebyshev.cuh"
#include "coarse.cuh"

namespace hdcr {

int make_block_geom(const Geom& g, const int block[4], BlockGeom* out) {
  if (!block) {
    set_error("block pointer is NULL");
    return HDCR_ERR_BAD_ARG;
  }
  out->Vc = 1;
  out->bvol = 1;
  for (int mu = 0; mu < 4; ++mu) {
    if (block[mu] < 1 || g.L[mu] % block[mu] != 0) {
      set_error("block extent %d does not divide L[%d] = %d", block[mu], mu, g.L[mu]);
      return HDCR_ERR_BAD_GEOMETRY;
    }
    if (g.L[mu] / block[mu] < 2) {
      set_error("coarse extent L[%d]/b = %d must be at least 2", mu, g.L[mu] / block[mu]);
      return HDCR_ERR_BAD_GEOMETRY;
    }
    out->b[mu] = block[mu];
    out->Lc[mu] = g.L[mu] / block[mu];
    out->Vc *= out->Lc[mu];
    out->bvol *= block[mu];
  }
  out->K5 = (long long)out->bvol * g.Ls;
  return HDCR_OK;
}

int subspace_check(const hdcr_subspace* sub) {
  if (!sub || !sub->vecs || sub->nvec < 2) {
    set_error("invalid subspace handle");
    return HDCR_ERR_BAD_ARG;
  }
  return HDCR_OK;
}

// ------------------------------------------------------------------ kernels
// v *= 1 / sqrt(*n2)
__global__ void scale_rsqrt_kernel(cpx<double>* __restrict__ v, long long n, const double* n2) {
  const double s = 1.0 / sqrt(*n2);
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    cpx<double> a = v[i];
    v[i] = cpx<double>(a.re * s, a.im * s);
  }
}

// plus = (x + Gamma5 x)/2, minus = (x - Gamma5 x)/2, Gamma5 = gamma5 R5
__global__ void gamma5_split_kernel(Geom g, const cpx<double>* __restrict__ x, cpx<double>* __restrict__ plus,
                                    cpx<double>* __restrict__ minus) {
  const long long n = g.V5 * 12;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < n;
       e += (long long)gridDim.x * blockDim.x) {
    const long long row = e / g.Ls;   // x4*12 + c
    const int s = (int)(e - row * g.Ls);
    const int c = (int)(row % 12);
    const cpx<double> a = x[e];
    cpx<double> b = x[row * g.Ls + (g.Ls - 1 - s)];
    if (c >= 6) b = cpx<double>(-b.re, -b.im);
    plus[e] = cpx<double>(0.5 * (a.re + b.re), 0.5 * (a.im + b.im));
    minus[e] = cpx<double>(0.5 * (a.re - b.re), 0.5 * (a.im - b.im));
  }
}

constexpr int GS_THREADS = 256;

// sum over the block of conj(u) v (both fields in plane layout), broadcast to all threads
__device__ __forceinline__ void block_dot(const Geom& g, const BlockGeom& bg, int a, const cpx<double>* u,
                                          const cpx<double>* v, double* bcast, double out[2]) {
  double acc[2] = {0.0, 0.0};
  for (long long l = threadIdx.x; l < bg.K5; l += GS_THREADS) {
    const unsigned o = fidx(g, 0, block_site(g, bg, a, l));
#pragma unroll 4
    for (int c = 0; c < 12; ++c) {
      const cpx<double> p = u[o + c * g.Ls], q = v[o + c * g.Ls];
      acc[0] += p.re * q.re + p.im * q.im;
      acc[1] += p.re * q.im - p.im * q.re;
    }
  }
  block_reduce<2>(acc);
  if (threadIdx.x == 0) {
    bcast[0] = acc[0];
    bcast[1] = acc[1];
  }
  __syncthreads();
  out[0] = bcast[0];
  out[1] = bcast[1];
  __syncthreads();
}

// Modified Gram-Schmidt, applied twice, inside each block (one CTA per block, the
// blocks of ``list`` or all of them), in the fixed order k = 0..nvec-1.  Rank
// deficiency sets *status.  Used for the blocks the Cholesky QR below leaves.
__global__ void __launch_bounds__(GS_THREADS) block_gs_kernel(Geom g, BlockGeom bg, cpx<double>* vecs,
                                                              int nvec, double rank_tol, int* status,
                                                              const int* list) {
  __shared__ double bcast[2];
  const int a = list ? list[blockIdx.x] : blockIdx.x;
  const long long fs = g.V5 * 12;
  for (int k = 0; k < nvec; ++k) {
    cpx<double>* vk = vecs + (long long)k * fs;
    double n0[2];
    block_dot(g, bg, a, vk, vk, bcast, n0);
    for (int pass = 0; pass < 2; ++pass) {
      for (int j = 0; j < k; ++j) {
        const cpx<double>* vj = vecs + (long long)j * fs;
        double d[2];
        block_dot(g, bg, a, vj, vk, bcast, d);
        for (long long l = threadIdx.x; l < bg.K5; l += GS_THREADS) {
          const unsigned o = fidx(g, 0, block_site(g, bg, a, l));
#pragma unroll 4
          for (int c = 0; c < 12; ++c) {
            const unsigned e = o + c * g.Ls;
            const cpx<double> p = vj[e];
            cpx<double> q = vk[e];
            q.re -= d[0] * p.re - d[1] * p.im;
            q.im -= d[0] * p.im + d[1] * p.re;
            vk[e] = q;
          }
        }
        __syncthreads();
      }
    }
    double n1[2];
    block_dot(g, bg, a, vk, vk, bcast, n1);
    double scale = 0.0;
    if (n1[0] > rank_tol * rank_tol * n0[0] && n1[0] > 0.0) {
      scale = 1.0 / sqrt(n1[0]);
    } else if (threadIdx.x == 0) {
      atomicExch(status, 1 + a);
    }
    for (long long l = threadIdx.x; l < bg.K5; l += GS_THREADS) {
      const unsigned o = fidx(g, 0, block_site(g, bg, a, l));
      for (int c = 0; c < 12; ++c) {
        const unsigned e = o + c * g.Ls;
        vk[e] = cpx<double>(vk[e].re * scale, vk[e].im * scale);
      }
    }
    __syncthreads();
  }
}

// ------------------------------------------------------------------ Cholesky QR
// The same orthonormalisation by two rounds of Cholesky QR per block: the Gram
// matrix G = V^dag V of the block's nvec vectors, G = R^dag R (R upper triangular,
// positive real diagonal), V <- V R^{-1}.  The QR factor with a positive real
// diagonal is unique, so in exact arithmetic this is the Gram-Schmidt result; the
// second round removes what the first left of the rounding (about cond(V)^2 eps).
// It reads each vector twice per round instead of twice per pair of vectors, so
// it runs at the FP64 rate instead of the memory rate.  A block whose pivot
// falls below CQR_TOL of its diagonal entry (condition number above ~1e4) is
// left to the Gram-Schmidt kernel, which also decides rank deficiency.
constexpr int CQR_E = 96;         // elements (site x component) of a block per chunk
constexpr int CQR_MAXV = 64;      // largest nvec handled (else Gram-Schmidt throughout)
constexpr int CQR_TILES = 3;      // 2 x 2 Gram tiles per thread: (nvec/2)(nvec/2+1)/2 <= 3 * 256
constexpr double CQR_TOL = 1e-8;

// offset of element le of block a: elements ordered by the block's 4d sites, then
// component and s, so one 4d site's 12 Ls elements are contiguous in the field
__device__ __forceinline__ unsigned cqr_off(const Geom& g, const BlockGeom& bg, int a, long long le) {
  const int per = 12 * g.Ls;
  const long long r = le / per;
  const int rem = (int)(le - r * per);
  const long long i5 = block_site(g, bg, a, r * g.Ls);  // s = 0 of the block's 4d site r
  return (unsigned)((i5 / g.Ls) * per + rem);
}

__device__ __forceinline__ void cqr_tile(int t, int nt, int* j, int* k) {
  int row = 0;  // tiles (tj, tk), tj <= tk, row by row
  while (t >= nt - row) {
    t -= nt - row;
    ++row;
  }
  *j = 2 * row;
  *k = 2 * (row + t);
}

// part[a][q] = sum over share q of block a of conj(v_j) v_k (upper 2x2 tiles)
__global__ void __launch_bounds__(GS_THREADS) cqr_gram_kernel(Geom g, BlockGeom bg, const cpx<double>* __restrict__ vecs,
                                                              int nvec, int S, const int* __restrict__ skip,
                                                              cpx<double>* __restrict__ part) {
  extern __shared__ cpx<double> xs[];  // [nvec][CQR_E]
  const int a = blockIdx.x, q = blockIdx.y;
  if (skip[a]) return;
  const long long fs = g.V5 * 12;
  const long long ne = bg.K5 * 12;
  const long long e0 = ne * q / S, e1 = ne * (q + 1) / S;
  const int nt = nvec / 2, ntiles = nt * (nt + 1) / 2;
  double acc[CQR_TILES][8];
  int tj[CQR_TILES], tk[CQR_TILES];
#pragma unroll
  for (int i = 0; i < CQR_TILES; ++i) {
    const int t = threadIdx.x + i * GS_THREADS;
    tj[i] = tk[i] = -1;
    if (t < ntiles) cqr_tile(t, nt, &tj[i], &tk[i]);
#pragma unroll
    for (int m = 0; m < 8; ++m) acc[i][m] = 0.0;
  }
  for (long long c0 = e0; c0 < e1; c0 += CQR_E) {
    const int n = (int)(e1 - c0 < CQR_E ? e1 - c0 : CQR_E);
    __syncthreads();
    for (int i = threadIdx.x; i < nvec * CQR_E; i += GS_THREADS) {
      const int k = i / CQR_E, e = i - k * CQR_E;
      xs[i] = e < n ? vecs[(long long)k * fs + cqr_off(g, bg, a, c0 + e)] : cpx<double>(0.0, 0.0);
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < CQR_TILES; ++i) {
      if (tj[i] < 0) continue;
      const cpx<double>* x0 = xs + tj[i] * CQR_E;
      const cpx<double>* x1 = x0 + CQR_E;
      const cpx<double>* y0 = xs + tk[i] * CQR_E;
      const cpx<double>* y1 = y0 + CQR_E;
      double* A = acc[i];
      for (int e = 0; e < n; ++e) {
        const cpx<double> u0 = x0[e], u1 = x1[e], w0 = y0[e], w1 = y1[e];
        A[0] = fma(u0.re, w0.re, fma(u0.im, w0.im, A[0]));
        A[1] = fma(u0.re, w0.im, fma(-u0.im, w0.re, A[1]));
        A[2] = fma(u0.re, w1.re, fma(u0.im, w1.im, A[2]));
        A[3] = fma(u0.re, w1.im, fma(-u0.im, w1.re, A[3]));
        A[4] = fma(u1.re, w0.re, fma(u1.im, w0.im, A[4]));
        A[5] = fma(u1.re, w0.im, fma(-u1.im, w0.re, A[5]));
        A[6] = fma(u1.re, w1.re, fma(u1.im, w1.im, A[6]));
        A[7] = fma(u1.re, w1.im, fma(-u1.im, w1.re, A[7]));
      }
    }
  }
  cpx<double>* P = part + ((long long)a * S + q) * nvec * nvec;
#pragma unroll
  for (int i = 0; i < CQR_TILES; ++i) {
    if (tj[i] < 0) continue;
    P[tj[i] * nvec + tk[i]] = cpx<double>(acc[i][0], acc[i][1]);
    P[tj[i] * nvec + tk[i] + 1] = cpx<double>(acc[i][2], acc[i][3]);
    P[(tj[i] + 1) * nvec + tk[i]] = cpx<double>(acc[i][4], acc[i][5]);
    P[(tj[i] + 1) * nvec + tk[i] + 1] = cpx<double>(acc[i][6], acc[i][7]);
  }
}

// G = sum_q part[a][q] (fixed order), G = R^dag R, rinv[a] = R^{-1}; one warp per
// block.  A pivot below CQR_TOL of its diagonal sets skip[a] (the block goes to
// Gram-Schmidt).
__global__ void __launch_bounds__(32) cqr_chol_kernel(int nvec, int S, const cpx<double>* __restrict__ part,
                                                      cpx<double>* __restrict__ rinv, int* __restrict__ skip) {
  extern __shared__ cpx<double> G[];  // [nvec][nvec]: G, then R in the upper triangle; diag G in d0
  double* d0 = reinterpret_cast<double*>(G + nvec * nvec);
  const int a = blockIdx.x, lane = threadIdx.x;
  if (skip[a]) return;
  const cpx<double>* P = part + (long long)a * S * nvec * nvec;
  for (int i = lane; i < nvec * nvec; i += 32) {
    const int j = i / nvec, k = i - j * nvec;
    if (j > k) continue;
    cpx<double> v(0.0, 0.0);
    for (int q = 0; q < S; ++q) {
      const cpx<double> w = P[(long long)q * nvec * nvec + i];
      v.re += w.re;
      v.im += w.im;
    }
    G[i] = v;
    if (j == k) d0[j] = v.re;
  }
  __syncwarp();
  bool ok = true;
  for (int k = 0; k < nvec && ok; ++k) {
    // pivot: G_kk - sum_{i<k} |R_ik|^2
    double dk = G[k * nvec + k].re;
    for (int i = 0; i < k; ++i) dk -= G[i * nvec + k].re * G[i * nvec + k].re + G[i * nvec + k].im * G[i * nvec + k].im;
    ok = dk > CQR_TOL * d0[k] && d0[k] > 0.0;
    if (!ok) break;
    const double rkk = sqrt(dk);
    __syncwarp();
    // row k of R: R_kj = (G_kj - sum_{i<k} conj(R_ik) R_ij) / R_kk, j > k
    for (int j = k + 1 + lane; j < nvec; j += 32) {
      double re = G[k * nvec + j].re, im = G[k * nvec + j].im;
      for (int i = 0; i < k; ++i) {
        const cpx<double> r1 = G[i * nvec + k], r2 = G[i * nvec + j];
        re -= r1.re * r2.re + r1.im * r2.im;
        im -= r1.re * r2.im - r1.im * r2.re;
      }
      G[k * nvec + j] = cpx<double>(re / rkk, im / rkk);
    }
    __syncwarp();
    if (lane == 0) G[k * nvec + k] = cpx<double>(rkk, 0.0);
    __syncwarp();
  }
  if (!ok) {
    if (lane == 0) skip[a] = 1;
    return;
  }
  // R^{-1} column by column (lane j): X_jj = 1/R_jj, X_ij = -(sum_{m=i+1..j} R_im X_mj) / R_ii
  cpx<double>* X = rinv + (long long)a * nvec * nvec;
  for (int j = lane; j < nvec; j += 32) {
    for (int i = j + 1; i < nvec; ++i) X[i * nvec + j] = cpx<double>(0.0, 0.0);
    X[j * nvec + j] = cpx<double>(1.0 / G[j * nvec + j].re, 0.0);
    for (int i = j - 1; i >= 0; --i) {
      double re = 0.0, im = 0.0;
      for (int m = i + 1; m <= j; ++m) {
        const cpx<double> r = G[i * nvec + m], x = X[m * nvec + j];
        re += r.re * x.re - r.im * x.im;
        im += r.re * x.im + r.im * x.re;
      }
      const double inv = -1.0 / G[i * nvec + i].re;
      X[i * nvec + j] = cpx<double>(re * inv, im * inv);
    }
  }
}

// v_k <- sum_{j<=k} v_j rinv_jk for the elements of share q of block a
__global__ void __launch_bounds__(GS_THREADS) cqr_apply_kernel(Geom g, BlockGeom bg, cpx<double>* __restrict__ vecs,
                                                               int nvec, int S, const int* __restrict__ skip,
                                                               const cpx<double>* __restrict__ rinv) {
  extern __shared__ cpx<double> sh[];  // rinv [nvec][nvec], then xs [nvec][CQR_E]
  const int a = blockIdx.x, q = blockIdx.y;
  if (skip[a]) return;
  cpx<double>* Ri = sh;
  cpx<double>* xs = sh + nvec * nvec;
  const cpx<double>* X = rinv + (long long)a * nvec * nvec;
  for (int i = threadIdx.x; i < nvec * nvec; i += GS_THREADS) Ri[i] = X[i];
  const long long fs = g.V5 * 12;
  const long long ne = bg.K5 * 12;
  const long long e0 = ne * q / S, e1 = ne * (q + 1) / S;
  for (long long c0 = e0; c0 < e1; c0 += CQR_E) {
    const int n = (int)(e1 - c0 < CQR_E ? e1 - c0 : CQR_E);
    __syncthreads();
    for (int i = threadIdx.x; i < nvec * CQR_E; i += GS_THREADS) {
      const int k = i / CQR_E, e = i - k * CQR_E;
      if (e < n) xs[i] = vecs[(long long)k * fs + cqr_off(g, bg, a, c0 + e)];
    }
    __syncthreads();
    for (int i = threadIdx.x; i < nvec * CQR_E; i += GS_THREADS) {
      const int k = i / CQR_E, e = i - k * CQR_E;
      if (e >= n) continue;
      double re = 0.0, im = 0.0;
      for (int j = 0; j <= k; ++j) {
        const cpx<double> v = xs[j * CQR_E + e], r = Ri[j * nvec + k];
        re = fma(v.re, r.re, fma(-v.im, r.im, re));
        im = fma(v.re, r.im, fma(v.im, r.re, im));
      }
      vecs[(long long)k * fs + cqr_off(g, bg, a, c0 + e)] = cpx<double>(re, im);
    }
  }
}

// Two rounds of Cholesky QR over every block that allows it; *flagged receives the
// blocks left for Gram-Schmidt (device list, count on the host).
static int cholesky_qr2(const Geom& g, const BlockGeom& bg, cpx<double>* vecs, int nvec, cudaStream_t st,
                        int** list_out, int* nlist) {
  *list_out = nullptr;
  *nlist = 0;
  const int Vc = bg.Vc;
  int dev = 0, sms = 0;
  HDCR_CUDA_TRY(cudaGetDevice(&dev));
  HDCR_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  int S = (4 * sms + Vc - 1) / Vc;  // shares of a block, so that the grid covers the SMs about four times
  if (S < 1) S = 1;
  if (S > 8) S = 8;
  const size_t nn = (size_t)nvec * nvec;
  cpx<double>* part = nullptr;
  cpx<double>* rinv = nullptr;
  int* skip = nullptr;
  cudaError_t e = cudaMallocAsync(&part, sizeof(cpx<double>) * nn * Vc * S, st);
  if (e == cudaSuccess) e = cudaMallocAsync(&rinv, sizeof(cpx<double>) * nn * Vc, st);
  // skip flags [0, Vc), then the list of flagged blocks handed to the caller
  if (e == cudaSuccess) e = cudaMallocAsync(&skip, sizeof(int) * (2 * (size_t)Vc + 1), st);
  if (e == cudaSuccess) e = cudaMemsetAsync(skip, 0, sizeof(int) * (2 * (size_t)Vc + 1), st);
  const size_t smem_gram = sizeof(cpx<double>) * (size_t)nvec * CQR_E;
  const size_t smem_chol = sizeof(cpx<double>) * nn + sizeof(double) * nvec;
  const size_t smem_apply = sizeof(cpx<double>) * (nn + (size_t)nvec * CQR_E);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(cqr_gram_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_gram);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(cqr_chol_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_chol);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(cqr_apply_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_apply);
  for (int round = 0; round < 2 && e == cudaSuccess; ++round) {
    cqr_gram_kernel<<<dim3(Vc, S), GS_THREADS, smem_gram, st>>>(g, bg, vecs, nvec, S, skip, part);
    cqr_chol_kernel<<<Vc, 32, smem_chol, st>>>(nvec, S, part, rinv, skip);
    cqr_apply_kernel<<<dim3(Vc, S), GS_THREADS, smem_apply, st>>>(g, bg, vecs, nvec, S, skip, rinv);
    count_launches(3);
    e = cudaGetLastError();
  }
  std::vector<int> hs(Vc);
  if (e == cudaSuccess) e = cudaMemcpyAsync(hs.data(), skip, sizeof(int) * Vc, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e == cudaSuccess) {
    std::vector<int> list;
    for (int a = 0; a < Vc; ++a)
      if (hs[a]) list.push_back(a);
    if (!list.empty()) {
      int* dl = skip + Vc;  // the second half of the flag buffer holds the list
      e = cudaMemcpyAsync(dl, list.data(), sizeof(int) * list.size(), cudaMemcpyHostToDevice, st);
      if (e == cudaSuccess) e = cudaStreamSynchronize(st);
      *list_out = dl;
      *nlist = (int)list.size();
    }
  }
  cudaFreeAsync(part, st);
  cudaFreeAsync(rinv, st);
  if (e != cudaSuccess || *nlist == 0) cudaFreeAsync(skip, st);
  if (e != cudaSuccess) {
    *list_out = nullptr;
    return cuda_status(e, "block Cholesky QR");
  }
  return HDCR_OK;
}

// ---------------------------------------------------------------- host side
// Takes ownership of ``vecs`` (freed on every failure, kept or converted on success).
static int orthonormalise_and_store(const Geom& g, const BlockGeom& bg, cpx<double>* vecs, int nvec,
                                    int store_dtype, cudaStream_t st, hdcr_subspace** out) {
  int* dstatus = nullptr;
  cudaError_t e0 = cudaMalloc(&dstatus, sizeof(int));
  if (e0 != cudaSuccess) {
    cudaFree(vecs);
    return cuda_status(e0, "subspace status flag");
  }
  cudaMemsetAsync(dstatus, 0, sizeof(int), st);
  // Cholesky QR where the blocks allow it, Gram-Schmidt for the rest (all of them
  // when nvec is above the Cholesky kernels' limit)
  int* list = nullptr;
  int nlist = bg.Vc;
  if (nvec <= CQR_MAXV) {
    const int s = cholesky_qr2(g, bg, vecs, nvec, st, &list, &nlist);
    if (s != HDCR_OK) {
      cudaFree(dstatus);
      cudaFree(vecs);
      return s;
    }
  }
  if (nlist > 0) {
    block_gs_kernel<<<nlist, GS_THREADS, 0, st>>>(g, bg, vecs, nvec, 1e-12, dstatus, list);
    count_launch();
  }
  cudaError_t e = cudaGetLastError();
  if (list) cudaFreeAsync(list - bg.Vc, st);  // the list sits behind the skip flags of cholesky_qr2
  int hstatus = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&hstatus, dstatus, sizeof(int), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  cudaFree(dstatus);
  if (e != cudaSuccess) {
    cudaFree(vecs);
    return cuda_status(e, "block orthonormalisation");
  }
  if (hstatus != 0) {
    cudaFree(vecs);
    set_error("subspace vectors are linearly dependent in block %d", hstatus - 1);
    return HDCR_ERR_RANK_DEFICIENT;
  }
  hdcr_subspace* sub = new hdcr_subspace();
  sub->g = g;
  sub->bg = bg;
  sub->nvec = nvec;
  sub->dtype = store_dtype;
  cudaGetDevice(&sub->device);
  const long long n = (long long)nvec * g.V5 * 12;
  if (store_dtype == HDCR_C128) {
    sub->vecs = vecs;  // keep the FP64 buffer
  } else {
    void* p = nullptr;
    e = cudaMalloc(&p, n * sizeof(cpx<float>));
    if (e != cudaSuccess) {
      cudaFree(vecs);
      delete sub;
      return cuda_status(e, "subspace storage");
    }
    int s = launch_convert(vecs, HDCR_C128, p, HDCR_C64, n, st);
    if (s == HDCR_OK) {
      e = cudaStreamSynchronize(st);
      if (e != cudaSuccess) s = cuda_status(e, "subspace convert");
    }
    cudaFree(vecs);
    if (s != HDCR_OK) {
      cudaFree(p);
      delete sub;
      return s;
    }
    sub->vecs = p;
  }
  *out = sub;
  return HDCR_OK;
}

// step 1 for one vector: filter x (precision R, in place) towards the low modes of H
template <typename R>
static int filter_one(const FineOp<R>& H, cpx<R>* x, const cpx<R>* zero, const hdcr_subspace_params* sp,
                      CRWork<R>& w, ChebWork<R>& cw, cudaStream_t st) {
  if (sp->kind == HDCR_SUBSPACE_CR_SMOOTH) {
    CRConfig cfg;
    cfg.fixed_iters = sp->order;
    return cr_run<R>(H, zero, x, w, cfg, nullptr, st);
  }
  return cheb_filter<R>(H, x, sp->order, sp->lam_cut, sp->lam_max, cw, w.rb.rs, st);
}

// step 1 with the Chebyshev filter: all nvec/2 noise fields through one run of
// the recurrence (multi-field stencil launches), then each is normalised and split
template <typename R>
static int filter_all_cheb(const Geom& g, const hdcr_dwf_params* p, const void* U, const void* noise,
                           const hdcr_subspace_params* sp, cpx<double>* vecs, cudaStream_t st) {
  const long long fs = g.V5 * 12;
  const int half = sp->nvec / 2;
  const bool f64 = sizeof(R) == 8;
  // x (half fields), recurrence work (4 * half fields), x64 scratch, U in R
  const size_t bytes = sizeof(cpx<R>) * fs * half * 5 + sizeof(cpx<double>) * fs +
                       (f64 ? 0 : sizeof(cpx<R>) * g.V4 * 36) + 1024;
  void* mem = nullptr;
  HDCR_CUDA_TRY(cudaMalloc(&mem, bytes));
  cpx<R>* x = (cpx<R>*)mem;
  cpx<R>* work = x + fs * half;
  cpx<double>* x64 = (cpx<double>*)(work + 4 * fs * half);
  const cpx<R>* Ur = (const cpx<R>*)U;
  if (!f64) {
    cpx<R>* u32 = (cpx<R>*)(x64 + fs);
    launch_convert(U, HDCR_C128, u32, HDCR_C64, (long long)g.V4 * 36, st);
    Ur = u32;
  }
  RedBuffers rb{{nullptr, nullptr}, nullptr, 0, nullptr};
  int s = red_buffers_alloc(&rb, 2);
  FineOp<R> H{g, p->M5, p->mf, Ur};
  if (s == HDCR_OK) s = launch_convert(noise, HDCR_C128, x, f64 ? HDCR_C128 : HDCR_C64, fs * half, st);
  if (s == HDCR_OK) s = cheb_filter_multi<R>(H, x, half, sp->order, sp->lam_cut, sp->lam_max, work, rb.scal, rb.rs, st);
  for (int i = 0; i < half && s == HDCR_OK; ++i) {
    s = launch_convert(x + (long long)i * fs, f64 ? HDCR_C128 : HDCR_C64, x64, HDCR_C128, fs, st);
    if (s == HDCR_OK) s = launch_norm2<double>(x64, fs, rb.rs, rb.scal + 1, st);
    if (s != HDCR_OK) break;
    scale_rsqrt_kernel<<<num_blocks(fs, 256, 4096), 256, 0, st>>>(x64, fs, rb.scal + 1); count_launch();
    gamma5_split_kernel<<<num_blocks(fs, 256, 4096), 256, 0, st>>>(g, x64, vecs + (long long)i * fs,
                                                                   vecs + (long long)(i + half) * fs); count_launch();
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) s = cuda_status(e, "subspace filtering");
  }
  cudaStreamSynchronize(st);
  red_buffers_free(&rb);
  cudaFree(mem);
  return s;
}

template <typename R>
static int filter_all(const Geom& g, const hdcr_dwf_params* p, const void* U, const void* noise,
                      const hdcr_subspace_params* sp, cpx<double>* vecs, cudaStream_t st) {
  const long long fs = g.V5 * 12;
  const int half = sp->nvec / 2;
  const bool f64 = sizeof(R) == 8;
  // x (R), zero (R), x64 scratch, U in R
  const size_t bytes = sizeof(cpx<R>) * fs * 2 + sizeof(cpx<double>) * fs + (f64 ? 0 : sizeof(cpx<R>) * g.V4 * 36) + 512;
  void* mem = nullptr;
  HDCR_CUDA_TRY(cudaMalloc(&mem, bytes));
  cpx<R>* x = (cpx<R>*)mem;
  cpx<R>* zero = x + fs;
  cpx<double>* x64 = (cpx<double>*)(zero + fs);
  const cpx<R>* Ur = (const cpx<R>*)U;
  if (!f64) {
    cpx<R>* u32 = (cpx<R>*)(x64 + fs);
    launch_convert(U, HDCR_C128, u32, HDCR_C64, (long long)g.V4 * 36, st);
    Ur = u32;
  }
  CRWork<R> w;
  ChebWork<R> cw;
  int s = crwork_alloc<R>(&w, fs);
  if (s == HDCR_OK && sp->kind == HDCR_SUBSPACE_CHEBYSHEV) s = cheb_work_alloc<R>(&cw, fs);
  FineOp<R> H{g, p->M5, p->mf, Ur};
  cudaMemsetAsync(zero, 0, sizeof(cpx<R>) * fs, st);
  for (int i = 0; i < half && s == HDCR_OK; ++i) {
    const cpx<double>* src = (const cpx<double>*)noise + (long long)i * fs;
    s = launch_convert(src, HDCR_C128, x, f64 ? HDCR_C128 : HDCR_C64, fs, st);
    if (s == HDCR_OK) s = filter_one<R>(H, x, zero, sp, w, cw, st);
    if (s == HDCR_OK) s = launch_convert(x, f64 ? HDCR_C128 : HDCR_C64, x64, HDCR_C128, fs, st);
    if (s == HDCR_OK) s = launch_norm2<double>(x64, fs, w.rb.rs, &w.dev()->tr, st);
    if (s != HDCR_OK) break;
    scale_rsqrt_kernel<<<num_blocks(fs, 256, 4096), 256, 0, st>>>(x64, fs, &w.dev()->tr); count_launch();
    gamma5_split_kernel<<<num_blocks(fs, 256, 4096), 256, 0, st>>>(g, x64, vecs + (long long)i * fs,
                                                                   vecs + (long long)(i + half) * fs); count_launch();
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) s = cuda_status(e, "subspace filtering");
  }
  cudaStreamSynchronize(st);
  crwork_free<R>(&w);
  cheb_work_free<R>(&cw);
  cudaFree(mem);
  return s;
}

static int build_subspace_impl(const Geom& g, const BlockGeom& bg, const hdcr_dwf_params* p, const void* U,
                               const void* noise, const hdcr_subspace_params* sp, cudaStream_t st,
                               hdcr_subspace** out) {
  const long long fs = g.V5 * 12;
  cpx<double>* vecs = nullptr;
  HDCR_CUDA_TRY(cudaMalloc(&vecs, sizeof(cpx<double>) * fs * sp->nvec));
  int s;
  if (sp->kind == HDCR_SUBSPACE_CHEBYSHEV)
    s = sp->filter_dtype == HDCR_C128 ? filter_all_cheb<double>(g, p, U, noise, sp, vecs, st)
                                      : filter_all_cheb<float>(g, p, U, noise, sp, vecs, st);
  else
    s = sp->filter_dtype == HDCR_C128 ? filter_all<double>(g, p, U, noise, sp, vecs, st)
                                      : filter_all<float>(g, p, U, noise, sp, vecs, st);
  if (s != HDCR_OK) {
    cudaFree(vecs);
    return s;
  }
  return orthonormalise_and_store(g, bg, vecs, sp->nvec, sp->store_dtype, st, out);
}

}  // namespace hdcr

using namespace hdcr;

static int subspace_args(const hdcr_geom* gp, const int block[4], int nvec, int store_dtype, Geom* g,
                         BlockGeom* bg) {
  HDCR_TRY(make_geom(gp, g));
  HDCR_TRY(make_block_geom(*g, block, bg));
  if (nvec < 2 || nvec % 2 != 0 || nvec > 256) {
    set_error("nvec = %d must be even, 2..256", nvec);
    return HDCR_ERR_BAD_ARG;
  }
  if (store_dtype != HDCR_C128 && store_dtype != HDCR_C64) {
    set_error("unknown storage dtype %d", store_dtype);
    return HDCR_ERR_BAD_ARG;
  }
  return HDCR_OK;
}

extern "C" int hdcr_build_subspace(const hdcr_geom* gp, const hdcr_dwf_params* p, const void* U,
                                   const void* noise, const hdcr_subspace_params* sp, void* stream,
                                   hdcr_subspace** out) {
  if (!sp) {
    set_error("hdcr_build_subspace: null parameters");
    return HDCR_ERR_BAD_ARG;
  }
  Geom g;
  BlockGeom bg;
  HDCR_TRY(subspace_args(gp, sp->block, sp->nvec, sp->store_dtype, &g, &bg));
  if (!p || !U || !noise || !out || sp->order < 0 ||
      (sp->kind != HDCR_SUBSPACE_CR_SMOOTH && sp->kind != HDCR_SUBSPACE_CHEBYSHEV) ||
      (sp->filter_dtype != HDCR_C128 && sp->filter_dtype != HDCR_C64)) {
    set_error("hdcr_build_subspace: null pointer or bad parameters");
    return HDCR_ERR_BAD_ARG;
  }
  if (sp->kind == HDCR_SUBSPACE_CHEBYSHEV && (sp->order < 1 || !(sp->lam_cut > 0.0) || !(sp->lam_max > sp->lam_cut))) {
    set_error("hdcr_build_subspace: Chebyshev filter needs order >= 1 and 0 < lam_cut < lam_max");
    return HDCR_ERR_BAD_ARG;
  }
  *out = nullptr;
  cudaStream_t st = as_stream(stream);
  Staged su, sn;
  HDCR_TRY(su.in(U, (size_t)g.V4 * 36 * 16, st));
  HDCR_TRY(sn.in(noise, (size_t)(sp->nvec / 2) * g.V5 * 12 * 16, st));
  return build_subspace_impl(g, bg, p, su.ptr(), sn.ptr(), sp, st, out);
}

extern "C" int hdcr_subspace_from_vectors(const hdcr_geom* gp, const int block[4], int nvec,
                                          const void* vectors, int store_dtype, void* stream,
                                          hdcr_subspace** out) {
  Geom g;
  BlockGeom bg;
  HDCR_TRY(subspace_args(gp, block, nvec, store_dtype, &g, &bg));
  if (!vectors || !out) {
    set_error("hdcr_subspace_from_vectors: null pointer");
    return HDCR_ERR_BAD_ARG;
  }
  *out = nullptr;
  cudaStream_t st = as_stream(stream);
  const long long n = (long long)nvec * g.V5 * 12;
  cpx<double>* vecs = nullptr;
  HDCR_CUDA_TRY(cudaMalloc(&vecs, sizeof(cpx<double>) * n));
  cudaMemcpyAsync(vecs, vectors, sizeof(cpx<double>) * n, cudaMemcpyDeviceToDevice, st);
  return orthonormalise_and_store(g, bg, vecs, nvec, store_dtype, st, out);
}

extern "C" int hdcr_subspace_info(const hdcr_subspace* sub, int* nvec, int coarse_L[4], int* dtype) {
  HDCR_TRY(subspace_check(sub));
  if (nvec) *nvec = sub->nvec;
  if (coarse_L)
    for (int mu = 0; mu < 4; ++mu) coarse_L[mu] = sub->bg.Lc[mu];
  if (dtype) *dtype = sub->dtype;
  return HDCR_OK;
}

extern "C" int hdcr_subspace_get_vectors(const hdcr_subspace* sub, void* out, void* stream) {
  HDCR_TRY(subspace_check(sub));
  if (!out) {
    set_error("hdcr_subspace_get_vectors: null output");
    return HDCR_ERR_BAD_ARG;
  }
  const long long n = (long long)sub->nvec * sub->g.V5 * 12;
  return launch_convert(sub->vecs, sub->dtype, out, HDCR_C128, n, as_stream(stream));
}

extern "C" void hdcr_subspace_destroy(hdcr_subspace* sub) {
  if (!sub) return;
  if (sub->vecs) cudaFree(sub->vecs);
  if (sub->build_ws) cudaFree(sub->build_ws);
  delete sub;
}
