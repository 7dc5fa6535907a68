// Subspace of the two-level preconditioner (Section 4):
//   noise -> a fixed number of CR steps on H x = 0 ("inverse iteration applied
//   to Gaussian noise") -> normalise -> chiral split with Gamma5 = gamma5 R5
//   -> restriction to blocks (Eq. 4.1) -> block orthonormalisation, so that
//   P_S = sum |phi_k^b><phi_k^b| (Eq. 4.3) is a projector.
// All of it runs in FP64; the basis is then stored in the requested dtype.
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

// Modified Gram-Schmidt, applied twice, inside each block (one CTA per block),
// in the fixed order k = 0..nvec-1.  Rank deficiency sets *status.
__global__ void __launch_bounds__(GS_THREADS) block_gs_kernel(Geom g, BlockGeom bg, cpx<double>* vecs,
                                                              int nvec, double rank_tol, int* status) {
  __shared__ double bcast[2];
  const int a = blockIdx.x;
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
  block_gs_kernel<<<bg.Vc, GS_THREADS, 0, st>>>(g, bg, vecs, nvec, 1e-12, dstatus); count_launch();
  cudaError_t e = cudaGetLastError();
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
