// Projections of the FP32 coarse-operator build on the tensor cores (tcgen05).
//
// For one block a and one leg the projection is a complex inner-product matrix
// A_jk = sum_kappa conj(X_j(kappa)) Y_k(kappa) over the leg's sites and spin-colour
// components (Eq. 4.5): a GEMM with small M = N = nvec and long K.  It is run as
// the real GEMM
//     C = P Q^T,  P = [Re X ; Im X] (2 nvec x K),  Q = [Re Y ; Im Y] (2 nvec x K),
//     Re A_jk = C[j][k] + C[n+j][n+k],   Im A_jk = C[j][n+k] - C[n+j][k],
// with P as the M operand (M = 64 for nvec <= 32, else 128; rows beyond 2 nvec
// are zero) and Q as the N = 16 * ceil(2 nvec / 16) operand, both K-major in
// shared memory, and the FP32 accumulator C in tensor memory.  The products use kind::tf32 in three
// passes (x = hi + lo with hi the TF32 truncation of x: hi*hi + hi*lo + lo*hi),
// which keeps the products at FP32 accuracy.  The tensor cores add into their
// FP32 accumulator without rounding to nearest, so a long sum drifts; each
// accumulator therefore takes TCP_SEG chunks only, alternating between two
// tensor-memory accumulators, and the segments are added up in FP32 registers
// (round to nearest) while the next segment runs.
//
// One CTA per block and share of K (a few CTAs split a long K; a second kernel
// adds their partial results in a fixed order).  K streams through shared
// memory in chunks of 32; each thread keeps its share of the next three chunks
// in flight in registers while the current one is split, stored in the
// canonical no-swizzle K-major layout
// (8-row x 16-byte core matrices) and handed to the MMA issued by thread 0.
// Two shared-memory stages alternate; an mbarrier per stage, signalled by
// tcgen05.commit, says when it may be refilled, so each chunk needs one CTA
// barrier only (between the stores and the MMA issue).  Every wait is bounded: on time-out the
// kernel records an error, stops issuing, waits (bounded) for what it issued,
// frees its tensor memory and returns.
#include "coarse.cuh"
#include "coarse_tc.cuh"

namespace hdcr {

constexpr int TCP_THREADS = 256;
constexpr int TCP_KC = 32;                  // kappa per chunk: 4 MMAs of K = 8
constexpr int TCP_SBO = (TCP_KC / 4) * 128; // bytes between 8-row core-matrix groups
constexpr int TCP_SEG = 16;                 // chunks accumulated in tensor memory before being added up in FP32

// MMA M: 64 when the 2 nvec rows of P fit, else 128; N = np
__host__ __device__ inline int tcp_m(int nvec) { return 2 * nvec <= 64 ? 64 : 128; }
__host__ __device__ inline int tcp_np(int nvec) { return (2 * nvec + 15) / 16 * 16; }
// one stage: the hi (and, with three passes, lo) parts of both operands for TCP_KC kappa
__host__ __device__ inline int tcp_stage_bytes(int m, int np, int npass) {
  return (npass == 3 ? 2 : 1) * (m + np) * TCP_KC * 4;
}
// shared-memory stages: two with three passes (at M = 64 that is 80 KB with the
// totals, so two CTAs share an SM; three stages needed 115 KB and left one CTA,
// 8 warps, per SM), three with one pass (65 KB).  Staging the operands through
// shared memory with asynchronous copies instead of the register prefetch measured
// slower on GB300 (one CTA per SM at eight chunks ahead, or two at three).
__host__ __device__ constexpr int tcp_nst(int m, int npass) { return npass == 3 ? 2 : 3; }
// dynamic shared memory: the stages, then the FP32 totals C[np][np + 1] (rows < 2 nvec <= np carry data)
__host__ __device__ inline int tcp_smem_bytes(int m, int np, int npass) {
  return tcp_nst(m, npass) * tcp_stage_bytes(m, np, npass) + np * (np + 1) * 4;
}

// stride between the vectors of an operand
__device__ __forceinline__ long long tc_vec_stride(const TcSrc& S) {
  return S.field ? 12 * S.g.V5 : (long long)S.bg.Vc * S.K;
}

// byte offset of element (row, k) in a K-major no-swizzle tile of TCP_KC columns
__device__ __forceinline__ int tile_off(int row, int k) {
  return (row >> 3) * TCP_SBO + (k >> 2) * 128 + (row & 7) * 16 + (k & 3) * 4;
}

__device__ __forceinline__ unsigned long long smem_desc(uint32_t addr) {
  // start address >> 4 (bits 0-13), leading (K-direction) byte offset 128 >> 4
  // (bits 16-29), stride (8-row) byte offset >> 4 (bits 32-45), version 1
  // (bits 46-48), no swizzle (bits 61-63 = 0)
  return (unsigned long long)((addr & 0x3FFFF) >> 4) | ((unsigned long long)(128 >> 4) << 16) |
         ((unsigned long long)(TCP_SBO >> 4) << 32) | (1ull << 46);
}

__device__ __forceinline__ uint32_t idesc_tf32(int m, int n) {
  // D F32 (bits 4-5 = 1), A and B TF32 (bits 7-9, 10-12 = 2), both K-major,
  // N >> 3 (bits 17-22), M >> 4 (bits 24-28)
  return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(m >> 4) << 24);
}

// tensor-memory lane of accumulator row r: row r itself for M = 128; for M = 64
// rows 16w .. 16w+15 sit in lanes 32w .. 32w+15 (measured on GB300)
template <int M>
__device__ __forceinline__ int acc_row_of_lane(int lane) {
  if (M == 128) return lane;
  return (lane & 31) < 16 ? 16 * (lane >> 5) + (lane & 31) : -1;
}

__device__ __forceinline__ void mma_tf32(uint32_t d, unsigned long long a, unsigned long long b, uint32_t idesc,
                                         int acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(d),
      "l"(a), "l"(b), "r"(idesc), "r"(acc)
      : "memory");
}

__device__ __forceinline__ bool mbar_test(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\tmbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}

// bounded wait on an mbarrier phase (about a second at most)
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
  for (int it = 0; it < (1 << 22); ++it) {
    if (mbar_test(bar, parity)) return true;
    __nanosleep(256);
  }
  return false;
}

__device__ __forceinline__ float tf32_hi(float x) { return __uint_as_float(__float_as_uint(x) & 0xFFFFE000u); }
// x rounded to the nearest TF32 value (ties away from zero), for the single-pass products
__device__ __forceinline__ float tf32_rna(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}

// Per chunk every thread owns up to TPT tasks: task t = (vector v, quad q) loads
// the four complex numbers kappa = 4q .. 4q+3 of X_v and Y_v (two 16-byte loads
// each) and stores the TF32 hi / lo parts of their real and imaginary rows as
// one 16-byte row of a core matrix each.  t -> v8 = t & 7, q = (t >> 3) & 7,
// v = 8 (t >> 6) + v8: the eight threads of a quarter warp write eight rows of
// one core matrix (no bank conflicts) and read eight 32-byte sectors.
// The loads run three chunks ahead in registers.
template <int TPT, int M, int NPASS, int TCP_NST = tcp_nst(M, NPASS)>
__global__ void __launch_bounds__(TCP_THREADS, TPT == 1 ? 2 : 1) tc_project_kernel(TcSrc S,
                                                                                  cpx<float>* __restrict__ A,
                                                                                  int nvec, int leg,
                                                                                  cpx<float>* __restrict__ part,
                                                                                  int* __restrict__ err) {
  extern __shared__ __align__(1024) unsigned char dsm[];
  __shared__ uint32_t tmem_slot;
  __shared__ __align__(8) unsigned long long bars[TCP_NST];
  __shared__ int abort_flag;
  const int a = blockIdx.x;
  const int tid = threadIdx.x;
  const int np = tcp_np(nvec);
  const int stage_bytes = tcp_stage_bytes(M, np, NPASS);
  const int a_bytes = M * TCP_KC * 4;
  // two accumulators of np columns each
  const uint32_t ncols = 2 * np <= 32 ? 32u : 2 * np <= 64 ? 64u : 2 * np <= 128 ? 128u : 256u;
  // zero both stages (the pad rows stay zero) and the totals, set up barriers and tensor memory
  for (int i = tid; i < tcp_smem_bytes(M, np, NPASS) / 16; i += TCP_THREADS)
    reinterpret_cast<float4*>(dsm)[i] = make_float4(0.f, 0.f, 0.f, 0.f);
  float* C = reinterpret_cast<float*>(dsm + TCP_NST * stage_bytes);  // FP32 totals per accumulator row
  const int cst = np + 1;
  if (tid == 0) {
    abort_flag = 0;
    for (int s = 0; s < TCP_NST; ++s)
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"((uint32_t)__cvta_generic_to_shared(&bars[s]))
                   : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (tid < 32) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     (uint32_t)__cvta_generic_to_shared(&tmem_slot)),
                 "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_slot;
  const uint32_t smem0 = (uint32_t)__cvta_generic_to_shared(dsm);
  const uint32_t idesc = idesc_tf32(M, np);
  // this CTA's share of the chunks (split-K over blockIdx.y)
  const long long ntot = (S.K + TCP_KC - 1) / TCP_KC;
  const long long cbeg = ntot * blockIdx.y / gridDim.y, cend = ntot * (blockIdx.y + 1) / gridDim.y;
  const long long nchunks = cend - cbeg;

  // the thread's tasks: all share q (so one kappa per chunk), vectors v0 + 32 i
  const int q = (tid >> 3) & 7;
  const int v0 = (tid >> 6) * 8 + (tid & 7);
  const long long vstride = tc_vec_stride(S);
  // site offset of kappa = 32 (cbeg + ch) + 4q, followed chunk by chunk: in the field
  // layout kappa = l * w + r over the block's 4d sites l, advanced without division
  const int w = 12 * S.g.Ls;
  long long kap = cbeg * TCP_KC + 4 * q;
  int l = S.field ? (int)(kap / w) : 0;
  int r = S.field ? (int)(kap - (long long)l * w) : 0;
  int lsite = -1;
  long long sbase = 0;
  auto site_off = [&]() -> long long {
    if (!S.field) return (long long)a * S.K + kap;
    if (l != lsite) {
      lsite = l;
      int ac[4];
      coarse_coords(S.bg, a, ac);
      int c[4];
      int t = l;
      c[0] = ac[0] * S.bg.b[0] + t % S.bg.b[0];
      t /= S.bg.b[0];
      c[1] = ac[1] * S.bg.b[1] + t % S.bg.b[1];
      t /= S.bg.b[1];
      c[2] = ac[2] * S.bg.b[2] + t % S.bg.b[2];
      c[3] = ac[3] * S.bg.b[3] + t / S.bg.b[2];
      sbase = (long long)x4_index(S.g, c) * w;
    }
    return sbase + r;
  };
  auto advance = [&]() {
    kap += TCP_KC;
    if (S.field) {
      r += TCP_KC;
      while (r >= w) {
        r -= w;
        ++l;
      }
    }
  };
  // four complex numbers of X and Y (zero beyond K) for every task of the thread
  auto load = [&](float4 (&xv)[TPT][2], float4 (&yv)[TPT][2]) {
    const long long so = site_off();
    const int avail = (int)min((long long)4, S.K - kap);
#pragma unroll
    for (int i = 0; i < TPT; ++i) {
      xv[i][0] = xv[i][1] = yv[i][0] = yv[i][1] = make_float4(0.f, 0.f, 0.f, 0.f);
      const int v = v0 + 32 * i;
      if (v < nvec && avail > 0) {
        const float4* px = reinterpret_cast<const float4*>(S.X + (long long)v * vstride + so);
        const float4* py = reinterpret_cast<const float4*>(S.Y + (long long)v * vstride + so);
        xv[i][0] = __ldg(px);
        yv[i][0] = __ldg(py);
        if (avail > 2) {
          xv[i][1] = __ldg(px + 1);
          yv[i][1] = __ldg(py + 1);
        }
        if (avail == 1 || avail == 3) {  // the last complex number lies beyond K
          if (avail == 1) {
            xv[i][0].z = xv[i][0].w = yv[i][0].z = yv[i][0].w = 0.f;
          } else {
            xv[i][1].z = xv[i][1].w = yv[i][1].z = yv[i][1].w = 0.f;
          }
        }
      }
    }
    advance();
  };
  // add accumulator (sg & 1) into the FP32 totals (warps 0-3 own tensor-memory lanes 0-127)
  auto flush = [&](long long sg) {
    // warp-uniform: skipped by a whole warp once a wait has timed out (the result is then discarded)
    if (tid < 128 && __all_sync(0xffffffffu, abort_flag == 0)) {
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const int wq = tid >> 5;
      for (int cg = 0; cg < np / 16; ++cg) {
        uint32_t rr[16];
        const uint32_t taddr = tmem + ((uint32_t)(32 * wq) << 16) + (uint32_t)((sg & 1) * np + cg * 16);
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
            : "=r"(rr[0]), "=r"(rr[1]), "=r"(rr[2]), "=r"(rr[3]), "=r"(rr[4]), "=r"(rr[5]), "=r"(rr[6]),
              "=r"(rr[7]), "=r"(rr[8]), "=r"(rr[9]), "=r"(rr[10]), "=r"(rr[11]), "=r"(rr[12]), "=r"(rr[13]),
              "=r"(rr[14]), "=r"(rr[15])
            : "r"(taddr));
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
        const int row = acc_row_of_lane<M>(tid);
        if (row >= 0 && row < 2 * nvec)
#pragma unroll
          for (int i = 0; i < 16; ++i) C[row * cst + cg * 16 + i] += __uint_as_float(rr[i]);
      }
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    }
  };
  // hi / lo rows of four consecutive kappa: 16 bytes at tile_off(row, 4q) (one pass: the
  // TF32-rounded values only)
  auto put = [&](unsigned char* hi, unsigned char* lo, int row, float e0, float e1, float e2, float e3) {
    const int o = tile_off(row, 4 * q);
    if constexpr (NPASS == 3) {
      const float4 h = make_float4(tf32_hi(e0), tf32_hi(e1), tf32_hi(e2), tf32_hi(e3));
      *reinterpret_cast<float4*>(hi + o) = h;
      *reinterpret_cast<float4*>(lo + o) = make_float4(e0 - h.x, e1 - h.y, e2 - h.z, e3 - h.w);
    } else {
      *reinterpret_cast<float4*>(hi + o) = make_float4(tf32_rna(e0), tf32_rna(e1), tf32_rna(e2), tf32_rna(e3));
    }
  };
  constexpr int OPS = NPASS == 3 ? 2 : 1;  // hi (+ lo) tiles per operand
  long long flushed = 0;  // segments added into C so far
  float4 xa[TPT][2], ya[TPT][2], xb[TPT][2], yb[TPT][2], xc[TPT][2], yc[TPT][2];
  long long issued = -1;  // last chunk whose MMAs were committed
  // One chunk: refill its stage from the registers (xv, yv), reload them with chunk
  // ch + 3, hand the stage to the MMA.  The three register sets keep their roles
  // (the loop below is unrolled three times), so no register copy waits on a
  // load in flight.  Returns false once a wait has timed out.
  auto step = [&](long long ch, float4 (&xv)[TPT][2], float4 (&yv)[TPT][2]) -> bool {
    const int s = (int)(ch % TCP_NST);
    unsigned char* st = dsm + s * stage_bytes;
    // every thread waits itself for the MMAs that last read this stage (chunk ch - NST)
    if (ch >= TCP_NST && !abort_flag) {
      if (!mbar_wait((uint32_t)__cvta_generic_to_shared(&bars[s]), (uint32_t)(((ch - TCP_NST) / TCP_NST) & 1)))
        abort_flag = 1;
    }
    // the segment that ended with chunk ch - NST is complete (waited for above): add it up
    if (ch % TCP_SEG == TCP_NST - 1 && ch > TCP_SEG) {
      flush(flushed);
      ++flushed;
    }
    unsigned char* qb = st + OPS * a_bytes;
    const int qbytes = np * TCP_KC * 4;
#pragma unroll
    for (int i = 0; i < TPT; ++i) {
      const int v = v0 + 32 * i;
      if (v < nvec) {
        const float4 x0 = xv[i][0], x1 = xv[i][1], y0 = yv[i][0], y1 = yv[i][1];
        put(st, st + a_bytes, v, x0.x, x0.z, x1.x, x1.z);
        put(st, st + a_bytes, nvec + v, x0.y, x0.w, x1.y, x1.w);
        put(qb, qb + qbytes, v, y0.x, y0.z, y1.x, y1.z);
        put(qb, qb + qbytes, nvec + v, y0.y, y0.w, y1.y, y1.w);
      }
    }
    if (ch + 3 < nchunks) load(xv, yv);
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    if (abort_flag) return false;
    if (tid == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t ahi = smem0 + s * stage_bytes, alo = ahi + a_bytes;
      const uint32_t bhi = ahi + OPS * a_bytes, blo = bhi + np * TCP_KC * 4;
      const uint32_t d = tmem + (uint32_t)(((ch / TCP_SEG) & 1) * np);
      const bool first = ch % TCP_SEG == 0;
#pragma unroll
      for (int ks = 0; ks < TCP_KC / 8; ++ks) {
        const uint32_t off = ks * 256;  // two core matrices along K per MMA
        mma_tf32(d, smem_desc(ahi + off), smem_desc(bhi + off), idesc, (!first || ks > 0) ? 1 : 0);
        if constexpr (NPASS == 3) {
          mma_tf32(d, smem_desc(ahi + off), smem_desc(blo + off), idesc, 1);
          mma_tf32(d, smem_desc(alo + off), smem_desc(bhi + off), idesc, 1);
        }
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                       (uint32_t)__cvta_generic_to_shared(&bars[s]))
                   : "memory");
    }
    issued = ch;
    return true;
  };
  // chunks 0, 1, 2 in flight before the first step; chunk c is always loaded into
  // set c % 3
  if (nchunks > 0) load(xa, ya);
  if (nchunks > 1) load(xb, yb);
  if (nchunks > 2) load(xc, yc);
  for (long long ch = 0; ch < nchunks; ch += 3) {
    if (!step(ch, xa, ya)) break;
    if (ch + 1 >= nchunks || !step(ch + 1, xb, yb)) break;
    if (ch + 2 >= nchunks || !step(ch + 2, xc, yc)) break;
  }
  // wait for the last committed chunk (its commit covers every earlier MMA)
  bool done = issued >= 0;
  if (done)
    done = mbar_wait((uint32_t)__cvta_generic_to_shared(&bars[issued % TCP_NST]),
                     (uint32_t)((issued / TCP_NST) & 1));
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  const bool good = __syncthreads_and(done && !abort_flag) != 0;
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (!good && tid == 0) atomicExch(err, 1);
  // the segments not yet added up (at most the last two)
  if (good) {
    const long long last = (nchunks - 1) / TCP_SEG;
    for (long long sg = flushed; sg <= last; ++sg) flush(sg);
  }
  __syncthreads();
  if (good) {
    for (int p = tid; p < nvec * nvec; p += TCP_THREADS) {
      const int j = p / nvec, k = p - j * nvec;
      const float re = C[j * cst + k] + C[(nvec + j) * cst + nvec + k];
      const float im = C[j * cst + nvec + k] - C[(nvec + j) * cst + k];
      if (part)
        part[(((long long)blockIdx.y * S.bg.Vc + a) * nvec + j) * nvec + k] = cpx<float>(re, im);
      else
        A[(((long long)a * NLEGS + leg) * nvec + j) * nvec + k] = cpx<float>(re, im);
    }
  }
  if (tid < 32) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(ncols) : "memory");
  }
}

// A[a][leg] = sum over the splits of the partial projections, in split order
__global__ void tc_reduce_kernel(const cpx<float>* __restrict__ part, int nsplit, cpx<float>* __restrict__ A, int Vc,
                                 int nvec, int leg) {
  const long long n2 = (long long)nvec * nvec;
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (long long)Vc * n2) return;
  const int a = (int)(idx / n2);
  const long long jk = idx - (long long)a * n2;
  float re = 0.f, im = 0.f;
  for (int s = 0; s < nsplit; ++s) {
    const cpx<float> v = part[(long long)s * Vc * n2 + idx];
    re += v.re;
    im += v.im;
  }
  A[((long long)a * NLEGS + leg) * n2 + jk] = cpx<float>(re, im);
}

int tc_project_splits(const TcSrc& S) {
  // enough CTAs for about four per SM, at least 16 chunks each
  int dev = 0, sms = 152;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    sms = 152;
  const long long nch = (S.K + TCP_KC - 1) / TCP_KC;
  long long sp = (4LL * sms + S.bg.Vc - 1) / S.bg.Vc;
  if (sp > nch / 16) sp = nch / 16;
  if (sp > TC_MAX_SPLIT) sp = TC_MAX_SPLIT;
  return sp < 1 ? 1 : (int)sp;
}

int launch_tc_project(const TcSrc& S, cpx<float>* A, int nvec, int leg, cpx<float>* part, int* err, int npass,
                      cudaStream_t st) {
  if (nvec > 64 || (npass != 1 && npass != 3)) {
    set_error("tensor-core projection: nvec = %d above the supported 64, or %d passes", nvec, npass);
    return HDCR_ERR_BAD_ARG;
  }
  const int m = tcp_m(nvec), np = tcp_np(nvec);
  const int smem = tcp_smem_bytes(m, np, npass);
  // the kernel for this size, allowed the dynamic shared memory of its largest nvec
  // (set on every call: the setting is per device, the value the same for every
  // caller, and the call is cheap beside the launch)
  void (*kern)(TcSrc, cpx<float>*, int, int, cpx<float>*, int*);
  if (npass == 3)
    kern = nvec <= 32 ? tc_project_kernel<1, 64, 3> : tc_project_kernel<2, 128, 3>;
  else
    kern = nvec <= 32 ? tc_project_kernel<1, 64, 1> : tc_project_kernel<2, 128, 1>;
  const int smem_max = nvec <= 32 ? tcp_smem_bytes(64, tcp_np(32), npass) : tcp_smem_bytes(128, tcp_np(64), npass);
  HDCR_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_max));
  const int sp = part ? tc_project_splits(S) : 1;
  const dim3 grid(S.bg.Vc, sp);
  cpx<float>* pp = sp > 1 ? part : nullptr;
  kern<<<grid, TCP_THREADS, smem, st>>>(S, A, nvec, leg, pp, err);
  count_launch();
  HDCR_LAUNCH_CHECK();
  if (sp > 1) {
    const long long n = (long long)S.bg.Vc * nvec * nvec;
    tc_reduce_kernel<<<num_blocks(n, 256), 256, 0, st>>>(part, sp, A, S.bg.Vc, nvec, leg); count_launch();
    HDCR_LAUNCH_CHECK();
  }
  return HDCR_OK;
}

}  // namespace hdcr
