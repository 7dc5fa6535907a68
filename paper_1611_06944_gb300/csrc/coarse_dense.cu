// Dense inverse of the little Dirac operator, so that the coarse inverse of
// Eq. 4.6 (Q = P A^{-1} P^dag) is applied exactly up to FP32 rounding.
//
// The coarse operator is small (Vc * nvec unknowns: 6144 on a 4^4 coarse
// lattice with 24 vectors) but Hermitian indefinite with eigenvalues close to
// zero, where a Krylov solve to a loose residual leaves the important
// directions unresolved.  The whole matrix is assembled from the 9-point
// stencil, inverted in place by Gauss-Jordan elimination with partial (row)
// pivoting, and applied as a matrix-vector product.
//
// Elimination step k: one CTA finds the pivot row (largest |a_ik|, lowest
// index on ties), swaps it into row k, saves column k and scales row k by the
// inverse pivot; then the grid applies the rank-1 update to every other row.
// The row interchanges are undone at the end by swapping columns in reverse
// order.
#include <vector>

#include "coarse.cuh"

namespace hdcr {

constexpr int GJ_THREADS = 1024;

// assemble the dense matrix D[(a, j)][(b, k)] from the 9 legs (legs reaching the same b add up)
__global__ void assemble_dense_kernel(const cpx<float>* __restrict__ A, const int* __restrict__ nbr, int Vc,
                                      int nvec, cpx<float>* __restrict__ D) {
  const long long n = (long long)Vc * nvec;
  const long long total = (long long)Vc * NLEGS * nvec * nvec;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const int k = (int)(e % nvec);
    long long r = e / nvec;
    const int j = (int)(r % nvec);
    r /= nvec;
    const int d = (int)(r % NLEGS);
    const int a = (int)(r / NLEGS);
    const int b = nbr[a * NLEGS + d];
    const cpx<float> v = A[e];
    float* dst = reinterpret_cast<float*>(D + ((long long)a * nvec + j) * n + (long long)b * nvec + k);
    atomicAdd(dst, v.re);
    atomicAdd(dst + 1, v.im);
  }
}

__global__ void __launch_bounds__(GJ_THREADS) gj_pivot_kernel(cpx<float>* __restrict__ M, int n, int k,
                                                              cpx<float>* __restrict__ ck,
                                                              cpx<float>* __restrict__ rk, int* __restrict__ perm,
                                                              int* __restrict__ status) {
  __shared__ float sv[GJ_THREADS / 32];
  __shared__ int si[GJ_THREADS / 32];
  __shared__ int piv;
  __shared__ float ipr, ipi;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  // argmax |M[i][k]|^2 over i >= k, lowest index on ties
  float best = -1.f;
  int bi = n;
  for (int i = k + tid; i < n; i += GJ_THREADS) {
    const cpx<float> v = M[(long long)i * n + k];
    const float m = v.re * v.re + v.im * v.im;
    if (m > best || (m == best && i < bi)) {
      best = m;
      bi = i;
    }
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    const float ob = __shfl_down_sync(0xffffffffu, best, off);
    const int oi = __shfl_down_sync(0xffffffffu, bi, off);
    if (ob > best || (ob == best && oi < bi)) {
      best = ob;
      bi = oi;
    }
  }
  if (lane == 0) {
    sv[warp] = best;
    si[warp] = bi;
  }
  __syncthreads();
  if (tid == 0) {
    float b = -1.f;
    int ii = n;
    for (int w = 0; w < GJ_THREADS / 32; ++w)
      if (sv[w] > b || (sv[w] == b && si[w] < ii)) {
        b = sv[w];
        ii = si[w];
      }
    piv = ii;
    perm[k] = ii;
    if (!(b > 0.f) || !(b < 3.0e38f)) atomicExch(status, 1 + k);
  }
  __syncthreads();
  const int p = piv;
  if (p != k && p < n) {
    for (int j = tid; j < n; j += GJ_THREADS) {
      const cpx<float> a = M[(long long)k * n + j], b = M[(long long)p * n + j];
      M[(long long)k * n + j] = b;
      M[(long long)p * n + j] = a;
    }
  }
  __syncthreads();
  if (tid == 0) {
    const cpx<float> d = M[(long long)k * n + k];
    const float m = d.re * d.re + d.im * d.im;
    const float inv = m > 0.f ? 1.f / m : 0.f;
    ipr = d.re * inv;
    ipi = -d.im * inv;
  }
  __syncthreads();
  const float pr = ipr, pi = ipi;
  for (int i = tid; i < n; i += GJ_THREADS) ck[i] = M[(long long)i * n + k];
  __syncthreads();
  for (int j = tid; j < n; j += GJ_THREADS) {
    cpx<float> v;
    if (j == k) {
      v = cpx<float>(pr, pi);
    } else {
      const cpx<float> a = M[(long long)k * n + j];
      v = cpx<float>(a.re * pr - a.im * pi, a.re * pi + a.im * pr);
    }
    rk[j] = v;
    M[(long long)k * n + j] = v;
  }
}

// M[i][j] -= ck[i] rk[j] (j != k), M[i][k] = -ck[i] rk[k], for every i != k
__global__ void gj_update_kernel(cpx<float>* __restrict__ M, int n, int k, const cpx<float>* __restrict__ ck,
                                 const cpx<float>* __restrict__ rk) {
  const long long total = (long long)n * n;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(e / n);
    if (i == k) continue;
    const int j = (int)(e - (long long)i * n);
    const cpx<float> c = ck[i], r = rk[j];
    if (j == k) {
      M[e] = cpx<float>(-(c.re * r.re - c.im * r.im), -(c.re * r.im + c.im * r.re));
    } else {
      cpx<float> m = M[e];
      m.re -= c.re * r.re - c.im * r.im;
      m.im -= c.re * r.im + c.im * r.re;
      M[e] = m;
    }
  }
}

__global__ void swap_columns_kernel(cpx<float>* __restrict__ M, int n, int a, int b) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const cpx<float> u = M[(long long)i * n + a], v = M[(long long)i * n + b];
    M[(long long)i * n + a] = v;
    M[(long long)i * n + b] = u;
  }
}

// y[r] = M x[r] (vectors in R, matrix FP32); one warp per row, coalesced row reads
template <typename R>
__global__ void dense_gemv_kernel(const cpx<float>* __restrict__ M, int n, const cpx<R>* __restrict__ x,
                                  cpx<R>* __restrict__ y, int nrhs) {
  const int warps = blockDim.x >> 5;
  const int lane = threadIdx.x & 31;
  const long long row0 = (long long)blockIdx.x * warps + (threadIdx.x >> 5);
  for (long long rr = row0; rr < (long long)n * nrhs; rr += (long long)gridDim.x * warps) {
    const int r = (int)(rr / n);
    const long long i = rr - (long long)r * n;
    const cpx<float>* row = M + i * n;
    const cpx<R>* xv = x + (long long)r * n;
    float sr = 0.f, si = 0.f;
    for (int j = lane; j < n; j += 32) {
      const cpx<float> m = row[j];
      const cpx<R> v = ld(xv + j);
      const float vr = (float)v.re, vi = (float)v.im;
      sr = fmaf(m.re, vr, sr);
      sr = fmaf(-m.im, vi, sr);
      si = fmaf(m.re, vi, si);
      si = fmaf(m.im, vr, si);
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
      sr += __shfl_down_sync(0xffffffffu, sr, off);
      si += __shfl_down_sync(0xffffffffu, si, off);
    }
    if (lane == 0) st(y + rr, cpx<R>((R)sr, (R)si));
  }
}

template <typename R>
int launch_dense_solve(const hdcr_coarse* co, const cpx<R>* in, cpx<R>* out, int nrhs, cudaStream_t st) {
  const int n = co->bg.Vc * co->nvec;
  const long long rows = (long long)n * nrhs;
  dense_gemv_kernel<R><<<num_blocks(rows, 8, 152 * 16), 256, 0, st>>>((const cpx<float>*)co->Ainv, n, in, out,
                                                                       nrhs); count_launch();
  HDCR_LAUNCH_CHECK();
  return HDCR_OK;
}
template int launch_dense_solve<double>(const hdcr_coarse*, const cpx<double>*, cpx<double>*, int, cudaStream_t);
template int launch_dense_solve<float>(const hdcr_coarse*, const cpx<float>*, cpx<float>*, int, cudaStream_t);

int coarse_invert(hdcr_coarse* co, cudaStream_t st) {
  const int Vc = co->bg.Vc, nvec = co->nvec;
  const long long n = (long long)Vc * nvec;
  if (n > 32768) {
    set_error("dense coarse inverse: %lld unknowns above the supported 32768", n);
    return HDCR_ERR_BAD_ARG;
  }
  if (co->Ainv) return HDCR_OK;
  const size_t mbytes = sizeof(cpx<float>) * (size_t)n * n;
  void* M = nullptr;
  void* aux = nullptr;
  HDCR_CUDA_TRY(cudaMalloc(&M, mbytes));
  const size_t abytes = sizeof(cpx<float>) * (size_t)(2 * n + (long long)Vc * NLEGS * nvec * nvec) +
                        sizeof(int) * (size_t)(n + 1) + 1024;
  cudaError_t e = cudaMalloc(&aux, abytes);
  if (e != cudaSuccess) {
    cudaFree(M);
    return cuda_status(e, "dense coarse inverse workspace");
  }
  cpx<float>* ck = (cpx<float>*)aux;
  cpx<float>* rk = ck + n;
  cpx<float>* A32 = rk + n;
  int* perm = (int*)(A32 + (long long)Vc * NLEGS * nvec * nvec);
  int* status = perm + n;
  int s = HDCR_OK;
  cudaMemsetAsync(M, 0, mbytes, st);
  cudaMemsetAsync(status, 0, sizeof(int), st);
  s = launch_convert(co->A, co->dtype, A32, HDCR_C64, (long long)Vc * NLEGS * nvec * nvec, st);
  if (s == HDCR_OK) {
    assemble_dense_kernel<<<num_blocks((long long)Vc * NLEGS * nvec * nvec, 256, 8192), 256, 0, st>>>(
        A32, co->nbr, Vc, nvec, (cpx<float>*)M); count_launch();
    const int ub = num_blocks(n * n, 256, 152 * 16);
    for (int k = 0; k < n; ++k) {
      gj_pivot_kernel<<<1, GJ_THREADS, 0, st>>>((cpx<float>*)M, (int)n, k, ck, rk, perm, status); count_launch();
      gj_update_kernel<<<ub, 256, 0, st>>>((cpx<float>*)M, (int)n, k, ck, rk); count_launch();
    }
    e = cudaGetLastError();
    if (e != cudaSuccess) s = cuda_status(e, "Gauss-Jordan elimination");
  }
  std::vector<int> hperm(n);
  int hstatus = 0;
  if (s == HDCR_OK) {
    e = cudaMemcpyAsync(hperm.data(), perm, sizeof(int) * n, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&hstatus, status, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) s = cuda_status(e, "Gauss-Jordan pivots");
  }
  if (s == HDCR_OK && hstatus != 0) {
    set_error("dense coarse inverse: zero or non-finite pivot at column %d", hstatus - 1);
    s = HDCR_ERR_NONFINITE;
  }
  if (s == HDCR_OK) {
    for (long long k = n - 1; k >= 0; --k)
      if (hperm[k] != k)
        swap_columns_kernel<<<num_blocks(n, 256, 1024), 256, 0, st>>>((cpx<float>*)M, (int)n, (int)k, hperm[k]); count_launch();
    e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) s = cuda_status(e, "dense coarse inverse");
  }
  cudaFree(aux);
  if (s != HDCR_OK) {
    cudaFree(M);
    return s;
  }
  co->Ainv = M;
  return HDCR_OK;
}

}  // namespace hdcr

using namespace hdcr;

extern "C" int hdcr_coarse_invert(hdcr_coarse* co, void* stream) {
  HDCR_TRY(coarse_check(co));
  return coarse_invert(co, as_stream(stream));
}

extern "C" int hdcr_coarse_solve_dense(const hdcr_coarse* co, const void* in, void* out, int nrhs, void* stream) {
  HDCR_TRY(coarse_check(co));
  if (!co->Ainv) {
    set_error("hdcr_coarse_solve_dense: call hdcr_coarse_invert first");
    return HDCR_ERR_BAD_ARG;
  }
  if (!in || !out || in == out || nrhs < 1) {
    set_error("hdcr_coarse_solve_dense: bad pointers or nrhs");
    return HDCR_ERR_BAD_ARG;
  }
  return launch_dense_solve<float>(co, (const cpx<float>*)in, (cpx<float>*)out, nrhs, as_stream(stream));
}
