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
// Blocked elimination.  Step k of Gauss-Jordan multiplies the matrix from the
// left by S_k (the row interchange) and E_k = I + u_k e_k^T, and overwrites
// column k with E_k e_k.  For a panel of P consecutive steps the interchanges can
// be moved to the front, so the panel acts on every other column j as
// col_j <- (I + U K^T) col_j, K^T selecting the panel's rows and U (n x P)
// accumulating the u_k (with later interchanges applied to its rows).  The P
// steps on the panel's own columns run as one grid-wide launch each (a thread
// per row; the last CTA to finish also picks the next pivot), then the rank-P
// update of all other columns is one complex GEMM on the tensor cores
// (coarse_gemm.cuh: cuBLAS, FP32 emulated on BF16 tensor cores).  The panel is
// wide (P = 128) so that the update's K is long enough for the tensor cores and
// the n/P passes over the matrix stay few.  The row interchanges amount to a
// permutation of the inverse's columns, which the matrix-vector product applies
// as a gather of the input vector; for several right-hand sides the vectors are
// gathered once and multiplied by the matrix in one GEMM, which reads the
// matrix once.
#include <climits>
#include <utility>
#include <vector>

#include "coarse.cuh"
#include "coarse_gemm.cuh"

namespace hdcr {

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

constexpr int GJ_P = 128;     // panel width
constexpr int GJ_ROWS = 64;   // rows (threads) per CTA of the panel kernels
constexpr int GJ_MAX_N = 32768;
constexpr int GJ_MAX_CTAS = GJ_MAX_N / GJ_ROWS;

// Workspace of the elimination.  The panel is held column-major (element (i, c)
// at c*n + i) so that a thread per row reads and writes coalesced, in two
// buffers: step l reads buffer l&1 and writes buffer (l+1)&1, so no CTA
// overwrites a row another CTA still has to read.
struct GJWork {
  cpx<float>* W[2];    // panel columns
  cpx<float>* U[2];    // accumulated multipliers (column c < l filled after step l)
  cpx<float>* T;       // panel rows of M after the interchanges, [GJ_P][n]
  float* cand_m;       // per-CTA pivot candidates
  int* cand_i;
  unsigned int* counter;  // zero between launches
  int* perm;           // perm[k]: row interchanged with row k at step k
  int* status;         // 1 + k of the first zero or non-finite pivot
  unsigned int* bar;   // grid barrier of the panel kernel: arrivals, generation, time-out flag
};

__device__ __forceinline__ float pivot_metric(cpx<float> v) {
  const float m = v.re * v.re + v.im * v.im;
  return m == m ? m : INFINITY;  // a NaN wins the search and is then reported
}

__device__ __forceinline__ void better(float& m, int& i, float om, int oi) {
  if (om > m || (om == m && oi < i)) {
    m = om;
    i = oi;
  }
}

// Grid-wide barrier of the cooperative panel kernel (all its CTAs are resident):
// generation counting, every wait bounded.  A CTA that gives up sets bar[2]; the
// kernel's result is then discarded (the host reports TIMEOUT).
__device__ __forceinline__ bool gj_grid_barrier(unsigned int* bar, unsigned int& gen) {
  __shared__ bool timed_out;
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    const unsigned int arrived = atomicAdd(&bar[0], 1u) + 1u;
    if (arrived == gridDim.x) {
      bar[0] = 0u;
      __threadfence();
      atomicExch(&bar[1], gen + 1u);
    } else {
      for (int it = 0; ((volatile unsigned int*)bar)[1] == gen; ++it) {
        if (it > (1 << 22)) {
          atomicExch(&bar[2], 1u);
          break;
        }
        if (it > 32) __nanosleep(64);
      }
    }
    __threadfence();
    timed_out = ((volatile unsigned int*)bar)[2] != 0u;  // one reading for the whole CTA
  }
  __syncthreads();
  ++gen;
  return !timed_out;
}

// a complex FP32 number read through L2 only: other CTAs wrote it during this launch,
// so a line this SM cached earlier may be stale
__device__ __forceinline__ cpx<float> ldcg_c(const cpx<float>* p) {
  const float2 v = __ldcg(reinterpret_cast<const float2*>(p));
  return cpx<float>(v.x, v.y);
}

constexpr int GJ_PARTS = 16;                   // threads sharing a row in the panel kernel
constexpr int GJ_COOP_T = GJ_ROWS * GJ_PARTS;  // threads per CTA of the panel kernel

// argmax over the CTA's threads, written to the CTA's candidate slot
__device__ __forceinline__ void gj_cta_candidate(float m, int i, const GJWork& w) {
  __shared__ float sm[GJ_COOP_T / 32];
  __shared__ int si[GJ_COOP_T / 32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int off = 16; off > 0; off >>= 1)
    better(m, i, __shfl_down_sync(0xffffffffu, m, off), __shfl_down_sync(0xffffffffu, i, off));
  if (lane == 0) {
    sm[warp] = m;
    si[warp] = i;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int q = 1; q < GJ_COOP_T / 32; ++q) better(m, i, sm[q], si[q]);
    w.cand_m[blockIdx.x] = m;
    w.cand_i[blockIdx.x] = i;
  }
}

// the pivot of step k from every CTA's candidate (each CTA reduces them all, in the
// same order, so all agree); CTA 0 records it
__device__ __forceinline__ int gj_grid_pivot(int k, const GJWork& w) {
  __shared__ float sm[GJ_COOP_T / 32];
  __shared__ int si[GJ_COOP_T / 32];
  __shared__ int piv;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  float m = -1.f;
  int i = INT_MAX;
  for (int b = threadIdx.x; b < (int)gridDim.x; b += GJ_COOP_T) better(m, i, __ldcg(w.cand_m + b), __ldcg(w.cand_i + b));
#pragma unroll
  for (int off = 16; off > 0; off >>= 1)
    better(m, i, __shfl_down_sync(0xffffffffu, m, off), __shfl_down_sync(0xffffffffu, i, off));
  if (lane == 0) {
    sm[warp] = m;
    si[warp] = i;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int q = 1; q < GJ_COOP_T / 32; ++q) better(m, i, sm[q], si[q]);
    if (!(m > 0.f) || !(m < 3.0e38f)) {
      if (blockIdx.x == 0) atomicCAS(w.status, 0, 1 + k);
      i = k;  // carry on without an interchange; the result is discarded
    }
    if (blockIdx.x == 0) w.perm[k] = i;
    piv = i;
  }
  __syncthreads();
  return piv;
}

// One whole panel in one cooperative launch: W = M[:, k0:k0+pw], U = 0, then the pw
// steps of gj_step_kernel with the pivot searches and the hand-over between steps
// done through a grid barrier instead of a launch per step.  Each row is shared by
// GJ_PARTS threads, which take every GJ_PARTS-th panel column (rows grid-stride).
__global__ void __launch_bounds__(GJ_COOP_T) gj_panel_coop_kernel(const cpx<float>* __restrict__ M, int n, int k0,
                                                                  int pw, GJWork w) {
  __shared__ cpx<float> rk[GJ_P], ruk[GJ_P];
  __shared__ cpx<float> rp[GJ_P], rup[GJ_P];
  unsigned int gen = ((volatile unsigned int*)w.bar)[1];
  const int t = threadIdx.x;
  const int rl = t % GJ_ROWS, part = t / GJ_ROWS;  // row of the CTA's chunk, column share
  const int stride = gridDim.x * GJ_ROWS;
  float m = -1.f;
  int bi = INT_MAX;
  for (int i = blockIdx.x * GJ_ROWS + rl; i < n; i += stride) {
    const cpx<float>* row = M + (long long)i * n + k0;
    for (int c = part; c < GJ_P; c += GJ_PARTS) {
      const cpx<float> v = c < pw ? row[c] : cpx<float>(0.f, 0.f);
      w.W[0][(long long)c * n + i] = v;
      w.U[0][(long long)c * n + i] = cpx<float>(0.f, 0.f);
      w.U[1][(long long)c * n + i] = cpx<float>(0.f, 0.f);
      if (c == 0 && i >= k0) better(m, bi, pivot_metric(v), i);
    }
  }
  for (int l = 0; l < pw; ++l) {
    const int k = k0 + l;
    gj_cta_candidate(m, bi, w);
    if (!gj_grid_barrier(w.bar, gen)) return;  // a barrier timed out: give up (the result is discarded)
    const int p = gj_grid_pivot(k, w);
    const bool odd = l & 1;
    const cpx<float>* Win = odd ? w.W[1] : w.W[0];
    const cpx<float>* Uin = odd ? w.U[1] : w.U[0];
    cpx<float>* Wout = odd ? w.W[0] : w.W[1];
    cpx<float>* Uout = odd ? w.U[0] : w.U[1];
    for (int c = t; c < GJ_P; c += GJ_COOP_T) {
      rk[c] = ldcg_c(Win + (long long)c * n + p);
      ruk[c] = ldcg_c(Uin + (long long)c * n + p);
      rp[c] = ldcg_c(Win + (long long)c * n + k);
      rup[c] = ldcg_c(Uin + (long long)c * n + k);
    }
    __syncthreads();
    const cpx<float> d = rk[l];
    const float dm = d.re * d.re + d.im * d.im;
    const float inv = dm > 0.f ? 1.f / dm : 0.f;
    const cpx<float> pinv(d.re * inv, -d.im * inv);
    m = -1.f;
    bi = INT_MAX;
    for (int i = blockIdx.x * GJ_ROWS + rl; i < n; i += stride) {
      const bool is_k = i == k, is_p = i == p && p != k;
      auto wsrc = [&](int c) { return is_k ? rk[c] : (is_p ? rp[c] : ldcg_c(Win + (long long)c * n + i)); };
      auto usrc = [&](int c) { return is_k ? ruk[c] : (is_p ? rup[c] : ldcg_c(Uin + (long long)c * n + i)); };
      const cpx<float> wl = wsrc(l);  // every part of the row forms the same multiplier
      const cpx<float> u = is_k ? cpx<float>(pinv.re - 1.f, pinv.im)
                                : cpx<float>(-(wl.re * pinv.re - wl.im * pinv.im), -(wl.re * pinv.im + wl.im * pinv.re));
      for (int c = part; c < pw; c += GJ_PARTS) {
        cpx<float> v;
        if (c == l) {
          v = cpx<float>(u.re + (is_k ? 1.f : 0.f), u.im);
        } else {
          v = wsrc(c);
          const cpx<float> r = rk[c];
          v.re += u.re * r.re - u.im * r.im;
          v.im += u.re * r.im + u.im * r.re;
        }
        Wout[(long long)c * n + i] = v;
        if (c == l + 1 && i > k) better(m, bi, pivot_metric(v), i);
      }
      for (int c = part; c < l; c += GJ_PARTS) {
        cpx<float> v = usrc(c);
        const cpx<float> r = ruk[c];
        v.re += u.re * r.re - u.im * r.im;
        v.im += u.re * r.im + u.im * r.re;
        Uout[(long long)c * n + i] = v;
      }
      if (l % GJ_PARTS == part) Uout[(long long)l * n + i] = u;
    }
    __syncthreads();  // rk .. rup are refilled by the next step
  }
}

__device__ __forceinline__ float tf32_trunc(float x) { return __uint_as_float(__float_as_uint(x) & 0xFFFFE000u); }

// The operands of the rank-pw update as three-term TF32 products (3xTF32): with
// x = hi(x) + lo(x), hi the TF32 truncation, U T ~ hi(U) hi(T) + hi(U) lo(T) + lo(U) hi(T),
// which one GEMM with K = 3 pw computes from Ucat = [hi U | hi U | lo U] and
// Tcat = [hi T | lo T | hi T] (both n x 3pw, column-major with leading dimension n).
__global__ void gj_split3_kernel(const cpx<float>* __restrict__ U, const cpx<float>* __restrict__ T, int n, int pw,
                                 cpx<float>* __restrict__ Ucat, cpx<float>* __restrict__ Tcat) {
  const long long total = (long long)n * pw;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const cpx<float> u = U[e], t = T[e];
    const cpx<float> uh(tf32_trunc(u.re), tf32_trunc(u.im)), th(tf32_trunc(t.re), tf32_trunc(t.im));
    const cpx<float> ul(u.re - uh.re, u.im - uh.im), tl(t.re - th.re, t.im - th.im);
    Ucat[e] = uh;
    Ucat[e + total] = uh;
    Ucat[e + 2 * total] = ul;
    Tcat[e] = th;
    Tcat[e + total] = tl;
    Tcat[e + 2 * total] = th;
  }
}

// End of a panel, before the update: the panel's row interchanges on every
// column outside it (a thread per column applies them in order) and the panel's
// rows copied to T.
__global__ void gj_panel_swap_kernel(cpx<float>* __restrict__ M, int n, int k0, int pw, GJWork w) {
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x) {
    if (j >= k0 && j < k0 + pw) continue;
    for (int l = 0; l < pw; ++l) {
      const int k = k0 + l, p = w.perm[k];
      if (p != k) {
        const cpx<float> a = M[(long long)k * n + j], b = M[(long long)p * n + j];
        M[(long long)k * n + j] = b;
        M[(long long)p * n + j] = a;
      }
    }
    for (int l = 0; l < pw; ++l) w.T[(long long)l * n + j] = M[(long long)(k0 + l) * n + j];
  }
}

// After the update (which also touched the panel's columns): the eliminated panel
// columns written into M.
__global__ void gj_panel_store_kernel(cpx<float>* __restrict__ M, int n, int k0, int pw,
                                      const cpx<float>* __restrict__ Wfin) {
  const long long total = (long long)n * pw;
  for (long long f = (long long)blockIdx.x * blockDim.x + threadIdx.x; f < total;
       f += (long long)gridDim.x * blockDim.x) {
    const int c = (int)(f / n), i = (int)(f - (long long)c * n);
    M[(long long)i * n + k0 + c] = Wfin[f];
  }
}

// y[r] = M x[r][pi] (vectors in R, matrix FP32, pi the column gather index);
// one warp per row, coalesced row reads
template <typename R>
__global__ void dense_gemv_kernel(const cpx<float>* __restrict__ M, const int* __restrict__ pi, int n,
                                  const cpx<R>* __restrict__ x, cpx<R>* __restrict__ y, int nrhs) {
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
      const cpx<R> v = ld(xv + __ldg(pi + j));
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

// xg[r][j] = x[r][pi[j]] in FP32
template <typename R>
__global__ void dense_gather_kernel(const cpx<R>* __restrict__ x, const int* __restrict__ pi, int n, int nrhs,
                                    cpx<float>* __restrict__ xg) {
  const long long total = (long long)n * nrhs;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const int r = (int)(e / n), j = (int)(e - (long long)r * n);
    const cpx<R> v = ld(x + (long long)r * n + __ldg(pi + j));
    st(xg + e, cpx<float>((float)v.re, (float)v.im));
  }
}

template <typename R>
__global__ void dense_out_kernel(const cpx<float>* __restrict__ y32, cpx<R>* __restrict__ y, long long total) {
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const cpx<float> v = ld(y32 + e);
    st(y + e, cpx<R>((R)v.re, (R)v.im));
  }
}

int dense_solve_prepare(hdcr_coarse* co, int nrhs) {
  if (nrhs <= 1) return HDCR_OK;
  HDCR_TRY(gemm_prepare());
  const size_t n = (size_t)co->bg.Vc * co->nvec;
  const size_t need = sizeof(cpx<float>) * n * (size_t)nrhs * 2;
  if (co->dws_bytes >= need) return HDCR_OK;
  if (co->dws) cudaFree(co->dws);
  co->dws = nullptr;
  co->dws_bytes = 0;
  HDCR_CUDA_TRY(cudaMalloc(&co->dws, need));
  co->dws_bytes = need;
  return HDCR_OK;
}

template <typename R>
int launch_dense_solve(const hdcr_coarse* co, const cpx<R>* in, cpx<R>* out, int nrhs, cudaStream_t st) {
  const int n = co->bg.Vc * co->nvec;
  const cpx<float>* M = (const cpx<float>*)co->Ainv;
  const int* pi = (const int*)(M + (long long)n * n);
  if (nrhs == 1) {  // one vector: a bandwidth-bound matrix-vector product on the CUDA cores
    dense_gemv_kernel<R><<<num_blocks(n, 8, 152 * 16), 256, 0, st>>>(M, pi, n, in, out, 1);
    count_launch();
    HDCR_LAUNCH_CHECK();
    return HDCR_OK;
  }
  // several: gather once, one GEMM on the tensor cores (the matrix is read once)
  const long long tot = (long long)n * nrhs;
  if (co->dws_bytes < sizeof(cpx<float>) * (size_t)tot * 2) {
    set_error("dense coarse solve: workspace for %d right-hand sides not prepared", nrhs);
    return HDCR_ERR_BAD_ARG;
  }
  cpx<float>* xg = (cpx<float>*)co->dws;
  cpx<float>* y32 = sizeof(R) == 4 ? (cpx<float>*)out : xg + tot;
  dense_gather_kernel<R><<<num_blocks(tot, 256, 4096), 256, 0, st>>>(in, pi, n, nrhs, xg);
  count_launch();
  HDCR_LAUNCH_CHECK();
  // out (column-major n x nrhs) = M xg, M row-major = (its column-major view)^T
  HDCR_TRY(cgemm_tc('T', 'N', n, nrhs, n, 1.f, M, n, xg, n, 0.f, y32, n, st, TC_BF16X9));
  if (sizeof(R) == 8) {
    dense_out_kernel<R><<<num_blocks(tot, 256, 4096), 256, 0, st>>>(y32, out, tot);
    count_launch();
    HDCR_LAUNCH_CHECK();
  }
  return HDCR_OK;
}
template int launch_dense_solve<double>(const hdcr_coarse*, const cpx<double>*, cpx<double>*, int, cudaStream_t);
template int launch_dense_solve<float>(const hdcr_coarse*, const cpx<float>*, cpx<float>*, int, cudaStream_t);

int coarse_invert(hdcr_coarse* co, cudaStream_t st) {
  const int Vc = co->bg.Vc, nvec = co->nvec;
  const long long n = (long long)Vc * nvec;
  if (n > GJ_MAX_N) {
    set_error("dense coarse inverse: %lld unknowns above the supported %d", n, GJ_MAX_N);
    return HDCR_ERR_BAD_ARG;
  }
  if (co->Ainv) return HDCR_OK;
  // the inverse (n x n, FP32 complex) followed by its column gather index (n ints)
  const size_t mbytes = sizeof(cpx<float>) * (size_t)n * n;
  void* M = nullptr;
  void* aux = nullptr;
  HDCR_CUDA_TRY(cudaMalloc(&M, mbytes + sizeof(int) * (size_t)n));
  const long long na = (long long)Vc * NLEGS * nvec * nvec;
  const size_t abytes = sizeof(cpx<float>) * (size_t)(11 * n * GJ_P + na) +
                        sizeof(float) * GJ_MAX_CTAS + sizeof(int) * (size_t)(GJ_MAX_CTAS + n + 5) + 256;
  cudaError_t e = cudaMalloc(&aux, abytes);
  if (e != cudaSuccess) {
    cudaFree(M);
    return cuda_status(e, "dense coarse inverse workspace");
  }
  GJWork w;
  cpx<float>* base = (cpx<float>*)aux;
  w.W[0] = base;
  w.W[1] = base + n * GJ_P;
  w.U[0] = base + 2 * n * GJ_P;
  w.U[1] = base + 3 * n * GJ_P;
  w.T = base + 4 * n * GJ_P;
  cpx<float>* Ucat = base + 5 * n * GJ_P;
  cpx<float>* Tcat = base + 8 * n * GJ_P;
  cpx<float>* A32 = base + 11 * n * GJ_P;
  w.cand_m = (float*)(A32 + na);
  w.cand_i = (int*)(w.cand_m + GJ_MAX_CTAS);
  w.perm = w.cand_i + GJ_MAX_CTAS;
  w.status = w.perm + n;
  w.counter = (unsigned int*)(w.status + 1);
  w.bar = w.counter + 1;
  int s = HDCR_OK;
  e = cudaMemsetAsync(M, 0, mbytes, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(w.status, 0, 5 * sizeof(int), st);  // status, counter, barrier
  if (e != cudaSuccess) s = cuda_status(e, "dense coarse inverse: clear");
  if (s == HDCR_OK) s = launch_convert(co->A, co->dtype, A32, HDCR_C64, na, st);
  if (s == HDCR_OK) {
    assemble_dense_kernel<<<num_blocks(na, 256, 8192), 256, 0, st>>>(A32, co->nbr, Vc, nvec, (cpx<float>*)M); count_launch();
    // the panel kernel runs cooperatively: as many CTAs as fit on the device at once
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, gj_panel_coop_kernel, GJ_COOP_T, 0);
    long long ctas = (n + GJ_ROWS - 1) / GJ_ROWS;
    if (ctas > (long long)sms * per_sm) ctas = (long long)sms * per_sm;
    if (ctas > GJ_MAX_CTAS) ctas = GJ_MAX_CTAS;
    s = gemm_prepare();
    for (long long k0 = 0; k0 < n && s == HDCR_OK; k0 += GJ_P) {
      const int pw = (int)(n - k0 < GJ_P ? n - k0 : GJ_P);
      const cpx<float>* Mc = (const cpx<float>*)M;
      int ni = (int)n, k0i = (int)k0, pwi = pw;
      void* args[] = {(void*)&Mc, (void*)&ni, (void*)&k0i, (void*)&pwi, (void*)&w};
      e = cudaLaunchCooperativeKernel((const void*)gj_panel_coop_kernel, dim3((unsigned)ctas), dim3(GJ_COOP_T), args,
                                      0, st);
      count_launch();
      if (e != cudaSuccess) {
        s = cuda_status(e, "Gauss-Jordan panel (cooperative launch)");
        break;
      }
      gj_panel_swap_kernel<<<num_blocks(n, 256, 4096), 256, 0, st>>>((cpx<float>*)M, (int)n, (int)k0, pw, w);
      count_launch();
      // M[i][j] += sum_c U[i][c] T[c][j]: in the column-major view (M^T) that is T^T U^T, with
      // T^T (n x pw) and U (n x pw) both stored column-major with leading dimension n; as
      // three TF32 products in one GEMM of K = 3 pw on the tensor cores
      gj_split3_kernel<<<num_blocks(n * pw, 256, 4096), 256, 0, st>>>(w.U[pw & 1], w.T, (int)n, pw, Ucat, Tcat);
      count_launch();
      s = cgemm_tc('N', 'T', (int)n, (int)n, 3 * pw, 1.f, Tcat, n, Ucat, n, 1.f, (cpx<float>*)M, n, st, TC_TF32);
      gj_panel_store_kernel<<<num_blocks(n * pw, 256, 4096), 256, 0, st>>>((cpx<float>*)M, (int)n, (int)k0, pw,
                                                                          w.W[pw & 1]);
      count_launch();
    }
    e = cudaGetLastError();
    if (e != cudaSuccess) s = cuda_status(e, "Gauss-Jordan elimination");
  }
  std::vector<int> hperm(n);
  int hstatus = 0, htimeout = 0;
  if (s == HDCR_OK) {
    e = cudaMemcpyAsync(hperm.data(), w.perm, sizeof(int) * n, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&hstatus, w.status, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&htimeout, w.bar + 2, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) s = cuda_status(e, "Gauss-Jordan pivots");
  }
  if (s == HDCR_OK && htimeout != 0) {
    set_error("dense coarse inverse: a grid barrier of the panel kernel timed out");
    s = HDCR_ERR_TIMEOUT;
  }
  if (s == HDCR_OK && hstatus != 0) {
    set_error("dense coarse inverse: zero or non-finite pivot at column %d", hstatus - 1);
    s = HDCR_ERR_NONFINITE;
  }
  if (s == HDCR_OK) {
    // Undoing the interchanges (columns k <-> perm[k], k from n-1 down to 0) makes
    // column j of the inverse column idx[j] of M; M x[pi] with pi = idx^{-1}
    // then equals the inverse applied to x.
    std::vector<int> idx(n), pi(n);
    for (long long j = 0; j < n; ++j) idx[j] = (int)j;
    for (long long k = n - 1; k >= 0; --k) std::swap(idx[k], idx[hperm[k]]);
    for (long long j = 0; j < n; ++j) pi[idx[j]] = (int)j;
    e = cudaMemcpyAsync((char*)M + mbytes, pi.data(), sizeof(int) * n, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
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
  // the workspace of several right-hand sides is internal state of the handle
  HDCR_TRY(dense_solve_prepare(const_cast<hdcr_coarse*>(co), nrhs));
  return launch_dense_solve<float>(co, (const cpx<float>*)in, (cpx<float>*)out, nrhs, as_stream(stream));
}
