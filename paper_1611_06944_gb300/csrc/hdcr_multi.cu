// Multi-right-hand-side HDCR solve (Section 4, batched): nrhs independent
// flexible GCR(m) solves of H x_r = b_r advanced in lockstep.  Every
// application of H, every Chebyshev smoother step, the restriction, the dense
// coarse solve and the prolongation is one launch over all nrhs fields, so each
// link the stencil loads serves every right-hand side.  The outer iteration is
// FP64 with its scalars on the device, one set per right-hand side, reduced by
// batched kernels in a fixed order (deterministic).  The V-cycle runs in the
// inner precision; with the Chebyshev smoother and the dense coarse solve it is
// a fixed sequence of launches, which is captured once into a CUDA graph (on a
// private stream) and replayed on the caller's stream every outer iteration.
#include <chrono>
#include <mutex>
#include <vector>

#include "chebyshev.cuh"
#include "coarse.cuh"

namespace hdcr {

constexpr int MB_BLOCKS = 128;  // blocks per right-hand side of a batched reduction
constexpr int MB_THREADS = 256;
constexpr int MB_MAX_RHS = 64;

// ------------------------------------------------------------------ kernels
__device__ __forceinline__ double warp_sum_d(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// sum of (a, b) over the block, valid in thread 0 (fixed order)
__device__ __forceinline__ void block_sum2(double& a, double& b) {
  __shared__ double sa[32], sb[32];
  a = warp_sum_d(a);
  b = warp_sum_d(b);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0) {
    sa[w] = a;
    sb[w] = b;
  }
  __syncthreads();
  if (w == 0) {
    const int nw = blockDim.x >> 5;
    a = l < nw ? sa[l] : 0.0;
    b = l < nw ? sb[l] : 0.0;
    a = warp_sum_d(a);
    b = warp_sum_d(b);
  }
}

// part[r][blk] = partial sum of conj(u_r) v_r over the block's slice (grid: MB_BLOCKS x nrhs)
__global__ void __launch_bounds__(MB_THREADS) mdot_part_kernel(const cpx<double>* __restrict__ u,
                                                               const cpx<double>* __restrict__ v, long long n,
                                                               double2* __restrict__ part) {
  const long long off = (long long)blockIdx.y * n;
  double a = 0.0, b = 0.0;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const cpx<double> x = u[off + i], y = v[off + i];
    a = fma((double)x.re, (double)y.re, fma((double)x.im, (double)y.im, a));
    b = fma((double)x.re, (double)y.im, fma(-(double)x.im, (double)y.re, b));
  }
  block_sum2(a, b);
  if (threadIdx.x == 0) part[blockIdx.y * gridDim.x + blockIdx.x] = make_double2(a, b);
}

// out[r * stride + {0, 1}] = sum of the nblk partials of right-hand side r (grid: nrhs)
__global__ void __launch_bounds__(MB_THREADS) mdot_final_kernel(const double2* __restrict__ part, int nblk,
                                                                double* __restrict__ out, int stride) {
  double a = 0.0, b = 0.0;
  for (int t = threadIdx.x; t < nblk; t += blockDim.x) {
    const double2 p = part[blockIdx.x * nblk + t];
    a += p.x;
    b += p.y;
  }
  block_sum2(a, b);
  if (threadIdx.x == 0) {
    out[blockIdx.x * stride] = a;
    out[blockIdx.x * stride + 1] = b;
  }
}

// w_r -= beta_r wj_r;  z_r -= beta_r zj_r   (beta_r = sc[r * ss], complex)
__global__ void maxpy2_neg_kernel(cpx<double>* __restrict__ w, const cpx<double>* __restrict__ wj,
                                  cpx<double>* __restrict__ z, const cpx<double>* __restrict__ zj, long long n,
                                  const double* __restrict__ sc, int ss) {
  const long long off = (long long)blockIdx.y * n;
  const double br = sc[blockIdx.y * ss], bi = sc[blockIdx.y * ss + 1];
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const cpx<double> a = wj[off + i], c = zj[off + i];
    cpx<double> u = w[off + i], v = z[off + i];
    u.re = fma(-br, a.re, fma(bi, a.im, u.re));
    u.im = fma(-br, a.im, fma(-bi, a.re, u.im));
    v.re = fma(-br, c.re, fma(bi, c.im, v.re));
    v.im = fma(-br, c.im, fma(-bi, c.re, v.im));
    w[off + i] = u;
    z[off + i] = v;
  }
}

// w_r /= |w_r|, z_r /= |w_r|   (|w_r|^2 = sc[r * ss])
__global__ void mscale2_kernel(cpx<double>* __restrict__ w, cpx<double>* __restrict__ z, long long n,
                               const double* __restrict__ sc, int ss) {
  const long long off = (long long)blockIdx.y * n;
  const double n2 = sc[blockIdx.y * ss];
  const double s = n2 > 0.0 ? 1.0 / sqrt(n2) : 0.0;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const cpx<double> a = w[off + i], c = z[off + i];
    w[off + i] = cpx<double>(a.re * s, a.im * s);
    z[off + i] = cpx<double>(c.re * s, c.im * s);
  }
}

// x_r += a_r z_r;  r_r -= a_r w_r;  partial |r_r|^2 into part (a_r = sc[r * ss])
__global__ void __launch_bounds__(MB_THREADS) mfgcr_update_kernel(cpx<double>* __restrict__ x,
                                                                  const cpx<double>* __restrict__ z,
                                                                  cpx<double>* __restrict__ r,
                                                                  const cpx<double>* __restrict__ w, long long n,
                                                                  const double* __restrict__ sc, int ss,
                                                                  double2* __restrict__ part) {
  const long long off = (long long)blockIdx.y * n;
  const double ar = sc[blockIdx.y * ss], ai = sc[blockIdx.y * ss + 1];
  double acc = 0.0, zero = 0.0;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const cpx<double> zv = z[off + i], wv = w[off + i];
    cpx<double> xv = x[off + i], rv = r[off + i];
    xv.re = fma(ar, zv.re, fma(-ai, zv.im, xv.re));
    xv.im = fma(ar, zv.im, fma(ai, zv.re, xv.im));
    rv.re = fma(-ar, wv.re, fma(ai, wv.im, rv.re));
    rv.im = fma(-ar, wv.im, fma(-ai, wv.re, rv.im));
    x[off + i] = xv;
    r[off + i] = rv;
    acc = fma((double)rv.re, (double)rv.re, fma((double)rv.im, (double)rv.im, acc));
  }
  block_sum2(acc, zero);
  if (threadIdx.x == 0) part[blockIdx.y * gridDim.x + blockIdx.x] = make_double2(acc, 0.0);
}

template <typename R>
__global__ void msub_kernel(const cpx<R>* __restrict__ a, const cpx<R>* __restrict__ b, cpx<R>* __restrict__ out,
                            long long n) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    st(out + i, ld(a + i) - ld(b + i));
}

template <typename R>
__global__ void madd_kernel(cpx<R>* __restrict__ y, const cpx<R>* __restrict__ x, long long n) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    st(y + i, ld(y + i) + ld(x + i));
}

// ------------------------------------------------------------------ workspace
struct MultiCache {
  int nrhs = 0, restart = 0, inner = -1;
  long long fs = 0, N = 0, cs = 0;  // one field, nrhs fields, one coarse vector (complex entries)
  void* mem = nullptr;
  cpx<double>* Z = nullptr;  // restart x nrhs fields
  cpx<double>* W = nullptr;
  cpx<double>* r = nullptr;  // nrhs fields
  cpx<double>* tmp = nullptr;
  void *r_in = nullptr, *z_in = nullptr, *t1 = nullptr, *t2 = nullptr, *e = nullptr;  // nrhs fields, inner
  void *c_rhs = nullptr, *c_sol = nullptr;                                            // nrhs coarse vectors
  void* U_in = nullptr;                                                               // links, inner precision
  void* chw = nullptr;                                                                // ChebWork<R> over nrhs
  double* sc = nullptr;     // nrhs x SC device scalars
  double2* part = nullptr;  // nrhs x MB_BLOCKS partial sums
  double* rr = nullptr;     // nrhs x 2: |r_r|^2 (stride 2)
  double* bb = nullptr;     // nrhs x 2: |b_r|^2
  double* host = nullptr;   // pinned, 2 * nrhs
  int SC = 0;
  std::vector<double> cheb_c;
  // captured V-cycle
  cudaStream_t cap = nullptr;
  cudaGraphExec_t exec = nullptr;
  unsigned long long graph_kernels = 0;
  int graph_fine = 0;
  const void* key_U = nullptr;
  const void* key_Ainv = nullptr;
  const void* key_dws = nullptr;  // the dense solve's workspace the graph was captured with
  double key_lo = 0, key_hi = 0;
  int key_order = -1, key_cycle = -1;
};

template <typename R>
static void multi_free_inner(MultiCache* c) {
  if (c->chw) {
    cheb_work_free<R>((ChebWork<R>*)c->chw);
    delete (ChebWork<R>*)c->chw;
    c->chw = nullptr;
  }
}

static void multi_cache_free(MultiCache* c) {
  if (!c) return;
  if (c->inner == HDCR_C128) multi_free_inner<double>(c);
  if (c->inner == HDCR_C64) multi_free_inner<float>(c);
  if (c->exec) cudaGraphExecDestroy(c->exec);
  if (c->cap) cudaStreamDestroy(c->cap);
  if (c->host) cudaFreeHost(c->host);
  if (c->mem) cudaFree(c->mem);
  delete c;
}

template <typename R>
static int multi_alloc(const hdcr_coarse* co, int nrhs, int restart, MultiCache** out) {
  MultiCache* c = new MultiCache();
  c->nrhs = nrhs;
  c->restart = restart;
  c->inner = sizeof(R) == 8 ? HDCR_C128 : HDCR_C64;
  c->fs = co->g.V5 * 12;
  c->N = c->fs * nrhs;
  c->cs = (long long)co->bg.Vc * co->nvec;
  c->SC = 2 * restart + 8;
  const size_t f64 = sizeof(cpx<double>) * (size_t)c->N, fin = sizeof(cpx<R>) * (size_t)c->N;
  const size_t cin = sizeof(cpx<R>) * (size_t)(c->cs * nrhs);
  const size_t bytes = f64 * (2 * (size_t)restart + 2) + fin * 5 + cin * 2 + sizeof(cpx<R>) * (size_t)co->g.V4 * 36 +
                       sizeof(double) * (size_t)(nrhs * c->SC + 4 * nrhs) + sizeof(double2) * nrhs * MB_BLOCKS +
                       16 * 256;
  cudaError_t e = cudaMalloc(&c->mem, bytes);
  if (e != cudaSuccess) {
    delete c;
    set_error("multi-RHS HDCR workspace: cudaMalloc(%zu) failed: %s", bytes, cudaGetErrorString(e));
    return HDCR_ERR_NO_MEMORY;
  }
  char* p = (char*)c->mem;
  auto take = [&](size_t b) {
    void* q = p;
    p += (b + 255) & ~(size_t)255;
    return q;
  };
  c->Z = (cpx<double>*)take(f64 * restart);
  c->W = (cpx<double>*)take(f64 * restart);
  c->r = (cpx<double>*)take(f64);
  c->tmp = (cpx<double>*)take(f64);
  c->r_in = take(fin);
  c->z_in = take(fin);
  c->t1 = take(fin);
  c->t2 = take(fin);
  c->e = take(fin);
  c->c_rhs = take(cin);
  c->c_sol = take(cin);
  c->U_in = take(sizeof(cpx<R>) * (size_t)co->g.V4 * 36);
  c->sc = (double*)take(sizeof(double) * (size_t)nrhs * c->SC);
  c->rr = (double*)take(sizeof(double) * 2 * nrhs);
  c->bb = (double*)take(sizeof(double) * 2 * nrhs);
  c->part = (double2*)take(sizeof(double2) * nrhs * MB_BLOCKS);
  int s = HDCR_OK;
  if (cudaMallocHost(&c->host, sizeof(double) * 2 * nrhs) != cudaSuccess) s = HDCR_ERR_NO_MEMORY;
  ChebWork<R>* chw = new ChebWork<R>();
  c->chw = chw;
  if (s == HDCR_OK) s = cheb_work_alloc<R>(chw, c->N);
  if (s == HDCR_OK && cudaStreamCreateWithFlags(&c->cap, cudaStreamNonBlocking) != cudaSuccess) s = HDCR_ERR_CUDA;
  if (s != HDCR_OK) {
    if (s == HDCR_ERR_NO_MEMORY) set_error("multi-RHS HDCR workspace: out of memory");
    multi_cache_free(c);
    return s;
  }
  *out = c;
  return HDCR_OK;
}

// batched <u_r, v_r> into out[r * stride] (2 doubles each)
static void mdot(const cpx<double>* u, const cpx<double>* v, long long n, int nrhs, double2* part, double* out,
                 int stride, cudaStream_t st) {
  mdot_part_kernel<<<dim3(MB_BLOCKS, nrhs), MB_THREADS, 0, st>>>(u, v, n, part);
  count_launch();
  mdot_final_kernel<<<nrhs, MB_THREADS, 0, st>>>(part, MB_BLOCKS, out, stride);
  count_launch();
}

// z = B r over all nrhs fields in precision R (fixed launch sequence, no host sync)
template <typename R>
static int mvcycle(const hdcr_coarse* co, const FineOp<R>& H, MultiCache* c, const hdcr_solve_params* prm,
                   const cpx<R>* r, cpx<R>* z, int* fine, cudaStream_t st) {
  const long long N = c->N;
  cpx<R>* t1 = (cpx<R>*)c->t1;
  cpx<R>* t2 = (cpx<R>*)c->t2;
  cpx<R>* e = (cpx<R>*)c->e;
  ChebWork<R>& w = *(ChebWork<R>*)c->chw;
  const int nb = num_blocks(N, 256, 8192);
  if (prm->cycle == HDCR_CYCLE_POST) {
    // z1 = P A^{-1} P^dag r;  z = z1 + S (r - H z1)
    HDCR_TRY(launch_restrict<R>(co->sub, r, (cpx<R>*)c->c_rhs, c->nrhs, st));
    HDCR_TRY(launch_dense_solve<R>(co, (const cpx<R>*)c->c_rhs, (cpx<R>*)c->c_sol, c->nrhs, st));
    HDCR_TRY(launch_prolong<R>(co->sub, (const cpx<R>*)c->c_sol, (const cpx<R>*)nullptr, z, c->nrhs, st));
  } else {
    // z1 = S r;  z2 = z1 + P A^{-1} P^dag (r - H z1)
    HDCR_TRY(cheb_smoother<R>(H, r, z, c->cheb_c, prm->cheb_lo, prm->cheb_hi, w, st, fine));
    HDCR_TRY(H.apply(z, t1, st));
    (*fine)++;
    msub_kernel<R><<<nb, 256, 0, st>>>(r, t1, t2, N);
    count_launch();
    HDCR_LAUNCH_CHECK();
    HDCR_TRY(launch_restrict<R>(co->sub, t2, (cpx<R>*)c->c_rhs, c->nrhs, st));
    HDCR_TRY(launch_dense_solve<R>(co, (const cpx<R>*)c->c_rhs, (cpx<R>*)c->c_sol, c->nrhs, st));
    HDCR_TRY(launch_prolong<R>(co->sub, (const cpx<R>*)c->c_sol, z, z, c->nrhs, st));
  }
  // z = z2 + S (r - H z2)
  HDCR_TRY(H.apply(z, t1, st));
  (*fine)++;
  msub_kernel<R><<<nb, 256, 0, st>>>(r, t1, t2, N);
  count_launch();
  HDCR_LAUNCH_CHECK();
  HDCR_TRY(cheb_smoother<R>(H, t2, e, c->cheb_c, prm->cheb_lo, prm->cheb_hi, w, st, fine));
  madd_kernel<R><<<nb, 256, 0, st>>>(z, e, N);
  count_launch();
  HDCR_LAUNCH_CHECK();
  return HDCR_OK;
}

// z_in = B r over all fields: the inner-precision copy of r (FP32 mode) and the V-cycle
template <typename R>
static int mprecondition(const hdcr_coarse* co, const FineOp<R>& H, MultiCache* c, const hdcr_solve_params* prm,
                         int* fine, cudaStream_t st) {
  const cpx<R>* rin = (const cpx<R>*)c->r;
  if (sizeof(R) != 8) {
    HDCR_TRY(launch_convert(c->r, HDCR_C128, c->r_in, HDCR_C64, c->N, st));
    rin = (const cpx<R>*)c->r_in;
  }
  return mvcycle<R>(co, H, c, prm, rin, (cpx<R>*)c->z_in, fine, st);
}

// Capture the preconditioner into a CUDA graph on the cache's private stream.
template <typename R>
static int capture_vcycle(const hdcr_coarse* co, const FineOp<R>& H, MultiCache* c, const hdcr_solve_params* prm) {
  if (c->exec) {
    cudaGraphExecDestroy(c->exec);
    c->exec = nullptr;
  }
  const unsigned long long k0 = launches_so_far();
  HDCR_CUDA_TRY(cudaStreamBeginCapture(c->cap, cudaStreamCaptureModeThreadLocal));
  int fine = 0;
  const int s = mprecondition<R>(co, H, c, prm, &fine, c->cap);
  cudaGraph_t graph = nullptr;
  const cudaError_t ee = cudaStreamEndCapture(c->cap, &graph);
  if (s != HDCR_OK) {
    if (graph) cudaGraphDestroy(graph);
    return s;
  }
  if (ee != cudaSuccess) return cuda_status(ee, "cudaStreamEndCapture (V-cycle)");
  const cudaError_t ei = cudaGraphInstantiate(&c->exec, graph, 0);
  cudaGraphDestroy(graph);
  if (ei != cudaSuccess) {
    c->exec = nullptr;
    return cuda_status(ei, "cudaGraphInstantiate (V-cycle)");
  }
  c->graph_kernels = launches_so_far() - k0;
  c->graph_fine = fine;
  return HDCR_OK;
}

template <typename R>
static int solve_multi_impl(const hdcr_coarse* co, MultiCache* c, const void* U, const cpx<double>* b,
                            cpx<double>* x, const hdcr_solve_params* prm, int use_graph, hdcr_solve_stats* stats,
                            cudaStream_t st) {
  const auto t0 = std::chrono::steady_clock::now();
  const int nrhs = c->nrhs;
  const long long fs = c->fs, N = c->N;
  const int nb = num_blocks(N, 256, 8192);
  const dim3 gb(num_blocks(fs, 256, MB_BLOCKS * 4), nrhs);
  FineOp<double> H64{co->g, co->M5, co->mf, (const cpx<double>*)U, nrhs};
  const cpx<R>* Uin = (const cpx<R>*)U;
  if (sizeof(R) != 8) {
    HDCR_TRY(launch_convert(U, HDCR_C128, c->U_in, HDCR_C64, (long long)co->g.V4 * 36, st));
    Uin = (const cpx<R>*)c->U_in;
  }
  FineOp<R> Hin{co->g, co->M5, co->mf, Uin, nrhs};
  c->cheb_c = cheb_inverse_coeffs(prm->cheb_lo, prm->cheb_hi, prm->smoother_order);
  double* sc = c->sc;
  const int SC = c->SC;
  const int I_N2 = 2 * c->restart, I_A = 2 * c->restart + 2;
  // r = b - H x, |b_r|^2, |r_r|^2
  HDCR_TRY(H64.apply(x, c->tmp, st));
  msub_kernel<double><<<nb, 256, 0, st>>>(b, c->tmp, c->r, N);
  count_launch();
  HDCR_LAUNCH_CHECK();
  mdot(b, b, fs, nrhs, c->part, c->bb, 2, st);
  mdot(c->r, c->r, fs, nrhs, c->part, c->rr, 2, st);
  HDCR_LAUNCH_CHECK();
  std::vector<double> bb(nrhs), rr(nrhs), tol2(nrhs);
  HDCR_CUDA_TRY(cudaMemcpyAsync(c->host, c->bb, sizeof(double) * 2 * nrhs, cudaMemcpyDeviceToHost, st));
  HDCR_CUDA_TRY(cudaStreamSynchronize(st));
  for (int q = 0; q < nrhs; ++q) bb[q] = c->host[2 * q];
  HDCR_CUDA_TRY(cudaMemcpyAsync(c->host, c->rr, sizeof(double) * 2 * nrhs, cudaMemcpyDeviceToHost, st));
  HDCR_CUDA_TRY(cudaStreamSynchronize(st));
  bool converged = true;
  for (int q = 0; q < nrhs; ++q) {
    rr[q] = c->host[2 * q];
    if (!(bb[q] == bb[q]) || !(rr[q] == rr[q]) || bb[q] > 1e300) {
      set_error("hdcr_solve_multi: non-finite right-hand side %d or its initial residual", q);
      return HDCR_ERR_NONFINITE;
    }
    tol2[q] = prm->tol * prm->tol * bb[q];
    if (!(bb[q] == 0.0 || rr[q] <= tol2[q])) converged = false;
  }
  // the graph bakes in U (FP64 inner), the dense inverse and the smoother: re-capture when they change
  const bool graph_ok = use_graph && c->exec && c->key_U == U && c->key_Ainv == co->Ainv && c->key_dws == co->dws &&
                        c->key_order == prm->smoother_order && c->key_lo == prm->cheb_lo &&
                        c->key_hi == prm->cheb_hi && c->key_cycle == prm->cycle;
  bool have_graph = graph_ok;
  int fine64 = 1, fine_in = 0, iters = 0, restarts = 0, status = HDCR_OK;
  while (!converged && iters < prm->max_outer) {
    int i = 0;
    for (; i < prm->restart && iters < prm->max_outer; ++i) {
      cpx<double>* z = c->Z + (long long)i * N;
      cpx<double>* w = c->W + (long long)i * N;
      // z = B r (the first V-cycle of a solve runs eagerly, which also tunes the stencil tiles)
      if (have_graph) {
        HDCR_CUDA_TRY(cudaGraphLaunch(c->exec, st));
        count_launches(c->graph_kernels);
        fine_in += c->graph_fine;
      } else {
        HDCR_TRY(mprecondition<R>(co, Hin, c, prm, &fine_in, st));
        if (use_graph) {
          HDCR_TRY(capture_vcycle<R>(co, Hin, c, prm));
          c->key_U = U;
          c->key_Ainv = co->Ainv;
          c->key_dws = co->dws;
          c->key_order = prm->smoother_order;
          c->key_lo = prm->cheb_lo;
          c->key_hi = prm->cheb_hi;
          c->key_cycle = prm->cycle;
          have_graph = true;
        }
      }
      if (sizeof(R) == 8) {
        HDCR_CUDA_TRY(cudaMemcpyAsync(z, c->z_in, sizeof(cpx<double>) * N, cudaMemcpyDeviceToDevice, st));
      } else {
        HDCR_TRY(launch_convert(c->z_in, HDCR_C64, z, HDCR_C128, N, st));
      }
      // w = H z, orthogonalised against the earlier w_j (same coefficients on z), per right-hand side
      HDCR_TRY(H64.apply(z, w, st));
      fine64++;
      for (int j = 0; j < i; ++j) {
        mdot(c->W + (long long)j * N, w, fs, nrhs, c->part, sc + 2 * j, SC, st);
        maxpy2_neg_kernel<<<gb, 256, 0, st>>>(w, c->W + (long long)j * N, z, c->Z + (long long)j * N, fs, sc + 2 * j,
                                              SC);
        count_launch();
        HDCR_LAUNCH_CHECK();
      }
      mdot(w, w, fs, nrhs, c->part, sc + I_N2, SC, st);
      mscale2_kernel<<<gb, 256, 0, st>>>(w, z, fs, sc + I_N2, SC);
      count_launch();
      mdot(w, c->r, fs, nrhs, c->part, sc + I_A, SC, st);
      mfgcr_update_kernel<<<dim3(MB_BLOCKS, nrhs), MB_THREADS, 0, st>>>(x, z, c->r, w, fs, sc + I_A, SC, c->part);
      count_launch();
      mdot_final_kernel<<<nrhs, MB_THREADS, 0, st>>>(c->part, MB_BLOCKS, c->rr, 2);
      count_launch();
      HDCR_LAUNCH_CHECK();
      HDCR_CUDA_TRY(cudaMemcpyAsync(c->host, c->rr, sizeof(double) * 2 * nrhs, cudaMemcpyDeviceToHost, st));
      HDCR_CUDA_TRY(cudaStreamSynchronize(st));
      ++iters;
      bool all = true;
      for (int q = 0; q < nrhs; ++q) {
        rr[q] = c->host[2 * q];
        if (!(rr[q] == rr[q]) || rr[q] > 1e300) {
          set_error("hdcr_solve_multi: non-finite residual of right-hand side %d at outer iteration %d", q, iters);
          status = HDCR_ERR_NONFINITE;
        }
        if (rr[q] > tol2[q]) all = false;
      }
      if (status != HDCR_OK || all) break;
    }
    if (status != HDCR_OK) break;
    // true residuals (restart or convergence check)
    HDCR_TRY(H64.apply(x, c->tmp, st));
    fine64++;
    msub_kernel<double><<<nb, 256, 0, st>>>(b, c->tmp, c->r, N);
    count_launch();
    mdot(c->r, c->r, fs, nrhs, c->part, c->rr, 2, st);
    HDCR_LAUNCH_CHECK();
    HDCR_CUDA_TRY(cudaMemcpyAsync(c->host, c->rr, sizeof(double) * 2 * nrhs, cudaMemcpyDeviceToHost, st));
    HDCR_CUDA_TRY(cudaStreamSynchronize(st));
    ++restarts;
    converged = true;
    for (int q = 0; q < nrhs; ++q) {
      rr[q] = c->host[2 * q];
      if (!(rr[q] == rr[q])) {
        status = HDCR_ERR_NONFINITE;
        set_error("hdcr_solve_multi: non-finite true residual of right-hand side %d", q);
      }
      if (rr[q] > tol2[q]) converged = false;
    }
    if (status != HDCR_OK) break;
  }
  if (status == HDCR_OK && !converged) {
    set_error("hdcr_solve_multi: not converged after %d outer iterations", iters);
    status = HDCR_ERR_NOT_CONVERGED;
  }
  if (stats) {
    const double t = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    for (int q = 0; q < nrhs; ++q) {
      hdcr_solve_stats& s = stats[q];
      s.status = status;
      s.iters = iters;
      s.fine_matvecs = fine64 + (sizeof(R) == 8 ? fine_in : 0);
      s.fine_matvecs_lo = sizeof(R) == 8 ? 0 : fine_in;
      s.coarse_matvecs = iters;  // one dense coarse solve per V-cycle
      s.restarts = restarts;
      s.true_resid = bb[q] > 0 ? sqrt(rr[q] / bb[q]) : 0.0;
      s.t_total = t;
      s.t_smoother = 0.0;
      s.t_coarse = 0.0;
    }
  }
  return status;
}

// ------------------------------------------------------------------ cache per coarse handle
static std::mutex g_mcache_mutex;
static std::vector<std::pair<const hdcr_coarse*, MultiCache*>> g_mcache;

void multi_cache_release(const hdcr_coarse* co) {
  std::lock_guard<std::mutex> lock(g_mcache_mutex);
  for (size_t i = 0; i < g_mcache.size(); ++i)
    if (g_mcache[i].first == co) {
      multi_cache_free(g_mcache[i].second);
      g_mcache.erase(g_mcache.begin() + i);
      return;
    }
}

}  // namespace hdcr

using namespace hdcr;

extern "C" int hdcr_solve_multi(hdcr_coarse* co, const void* U, const void* b, void* x, int nrhs,
                                const hdcr_solve_params* prm, int use_graph, hdcr_solve_stats* stats,
                                void* stream) {
  HDCR_TRY(coarse_check(co));
  if (!U || !b || !x || !prm || b == x || nrhs < 1 || nrhs > MB_MAX_RHS) {
    set_error("hdcr_solve_multi: null pointer, b == x or nrhs outside 1..%d", MB_MAX_RHS);
    return HDCR_ERR_BAD_ARG;
  }
  if (co->cf) {
    set_error("hdcr_solve_multi: the batched solve runs the domain-wall operator only (use hdcr_solve)");
    return HDCR_ERR_BAD_ARG;
  }
  if (!(prm->tol > 0.0) || prm->max_outer < 1 || prm->restart < 1 || prm->restart > 64 ||
      prm->smoother_kind != HDCR_SMOOTHER_CHEBYSHEV || prm->smoother_order < 1 || !(prm->cheb_lo > 0.0) ||
      !(prm->cheb_hi > prm->cheb_lo) || prm->coarse_solver != HDCR_COARSE_DENSE ||
      (prm->cycle != HDCR_CYCLE_SYMMETRIC && prm->cycle != HDCR_CYCLE_POST)) {
    set_error("hdcr_solve_multi: needs tol > 0, 1 <= restart <= 64, the Chebyshev smoother (order >= 1, "
              "0 < cheb_lo < cheb_hi), the dense coarse solve and a known cycle");
    return HDCR_ERR_BAD_ARG;
  }
  if (prm->inner_dtype != HDCR_C128 && prm->inner_dtype != HDCR_C64) {
    set_error("hdcr_solve_multi: unknown inner dtype %d", prm->inner_dtype);
    return HDCR_ERR_BAD_ARG;
  }
  if (co->dtype != prm->inner_dtype || co->sub->dtype != prm->inner_dtype) {
    set_error("hdcr_solve_multi: basis (%d) and coarse operator (%d) must be stored in the inner dtype %d",
              co->sub->dtype, co->dtype, prm->inner_dtype);
    return HDCR_ERR_BAD_ARG;
  }
  if ((co->g.V5 * 12) * (long long)nrhs >= (1LL << 31)) {
    set_error("hdcr_solve_multi: nrhs fields must hold fewer than 2^31 complex numbers");
    return HDCR_ERR_BAD_ARG;
  }
  cudaStream_t st = as_stream(stream);
  if (!co->Ainv) HDCR_TRY(coarse_invert(co, st));
  HDCR_TRY(dense_solve_prepare(co, nrhs));  // before any capture: the coarse solve then allocates nothing
  MultiCache* cache = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_mcache_mutex);
    MultiCache** slot = nullptr;
    for (auto& p : g_mcache)
      if (p.first == co) slot = &p.second;
    if (!slot) {
      g_mcache.push_back({co, nullptr});
      slot = &g_mcache.back().second;
    }
    if (*slot && ((*slot)->inner != prm->inner_dtype || (*slot)->restart < prm->restart || (*slot)->nrhs != nrhs)) {
      multi_cache_free(*slot);
      *slot = nullptr;
    }
    if (!*slot) {
      int s = prm->inner_dtype == HDCR_C128 ? multi_alloc<double>(co, nrhs, prm->restart, slot)
                                            : multi_alloc<float>(co, nrhs, prm->restart, slot);
      if (s != HDCR_OK) return s;
    }
    cache = *slot;
  }
  if (prm->inner_dtype == HDCR_C128)
    return solve_multi_impl<double>(co, cache, U, (const cpx<double>*)b, (cpx<double>*)x, prm, use_graph, stats, st);
  return solve_multi_impl<float>(co, cache, U, (const cpx<double>*)b, (cpx<double>*)x, prm, use_graph, stats, st);
}
