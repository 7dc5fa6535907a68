// FP32 operator H = Gamma5 D_dwf (Section 3) with the spinors staged in shared
// memory by the tensor memory accelerator (TMA): 2.5-dimensional blocking.
//
// Why: every spinor of the field is read by nine output sites (itself and its
// eight 4d neighbours).  Gathered from L2 site by site, as the other FP32
// kernel does, those reads move several times the field's bytes from L2 to the
// SMs and the warps wait on them.  Here a CTA owns a column of the lattice --
// whole x-rows, TY x TZ of them in (y, z), one quad of fifth-dimension sites
// (s = 4q .. 4q+3) -- and marches along t.  Three consecutive t-planes of the
// column sit in shared memory (t-1, t, t+1), together with the four (y, z)
// faces next to plane t; each plane is loaded once by a TMA tensor copy and
// serves as t+1, t and t-1 in turn, so the L2 reads per output plane are the
// column's plane plus its faces.  The x-hops wrap inside the row.
//
// Shared-memory layout of a box: [z][y][component c][x][one quad of s], i.e.
// 32 bytes per (site, component), so the 16 threads x 2 pairs of an x-row read
// one component as 512 contiguous bytes (no bank conflicts).  The tensor map
// describes the field (psi[x4][c][s], FP32 complex) as a 5-dimensional FP32
// tensor (s-and-re/im: 2 Ls, x: Lx, c: 12, y: Ly, z + Lz (t + Lt r): Lz Lt nrhs)
// whose dimension order differs from the memory order, which gives the
// component-major box layout above in one copy.
//
// Each thread owns one pair (s0, s0+1) of one site, as the packed kernel of
// dwf_x2.cu does, with the same hop arithmetic and the same order of the sums
// (hops_first, hops_second, local_x2, store_x2), so both kernels give the same
// bits.  The step over plane t is split in two halves around one CTA barrier:
// the hops that read the faces and plane t-1 (y+-, z+-, t-) first; then one
// thread issues the copies of the next plane's faces and of plane t+2 into the
// buffers just freed, and the remaining hops (x+-, t+) and the fifth-dimension
// terms run while they fly.  The fifth-dimension neighbours across the quad's
// edges (s = 4q-1, 4q+4) are read from global memory.
//
// Every wait on a copy is bounded (well under a second); a CTA that gives up
// sets a device flag, waits (again bounded) for the copies it still has in
// flight and leaves.  The autotuner reads the flag and drops the variant.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <atomic>
#include <mutex>

#include "dwf_x2.cuh"
#include "dwf_tma.cuh"
#include "reduce.cuh"

namespace hdcr {

namespace {

static __device__ int g_tma_timeout;  // set by a CTA whose copy did not arrive in time

// ------------------------------------------------------------------ PTX helpers
__device__ __forceinline__ uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint32_t bar) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar) : "memory");
}

__device__ __forceinline__ void mbar_expect(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

__device__ __forceinline__ bool mbar_ready(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\tmbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}

// bounded wait for the phase with the given parity to complete (a few hundred ms at most)
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
  for (int i = 0; i < (1 << 21); ++i) {
    if (mbar_ready(bar, parity)) return true;
    if (i > 64) __nanosleep(64);
  }
  return false;
}

__device__ __forceinline__ void tma_load(uint32_t dst, const CUtensorMap* map, uint32_t bar, int c0, int c3,
                                         int c4) {
  asm volatile(
      "cp.async.bulk.tensor.5d.shared::cluster.global.tile.mbarrier::complete_tx::bytes "
      "[%0], [%1, {%3, %4, %5, %6, %7}], [%2];" ::"r"(dst),
      "l"(reinterpret_cast<unsigned long long>(map)), "r"(bar), "r"(c0), "r"(0), "r"(0), "r"(c3), "r"(c4)
      : "memory");
}

// ------------------------------------------------------------------ geometry of a variant
template <int LX, int TY, int TZ>
struct Shape {
  static constexpr int sites = LX * TY * TZ;
  static constexpr int threads = 2 * sites;
  static constexpr int site_bytes = 12 * 32;  // 12 components x one quad of s (4 FP32 complex)
  static constexpr int cstride = LX * 32;     // bytes between components of one site in a box
  static constexpr int plane = sites * site_bytes;
  static constexpr int yface = LX * TZ * site_bytes;
  static constexpr int zface = LX * TY * site_bytes;
  static constexpr int off_halo = 3 * plane;
  static constexpr int off_bar = off_halo + 2 * yface + 2 * zface;
  static constexpr int smem = off_bar + 64;
};

template <int CS>
struct PairS {
  const char* b;  // component 0 of the pair in shared memory
  __device__ __forceinline__ float4 operator()(int c) const {
    return *reinterpret_cast<const float4*>(b + c * CS);
  }
};

// Neighbours of one pair in the staged buffers (hop d = 2 mu + backward)
template <int LX, int TY, int TZ>
struct SmemHops {
  typedef Shape<LX, TY, TZ> S;
  const char* prev;
  const char* mid;
  const char* next;
  const char* halo;
  const cpx<float>* U;
  int x, yy, zz, p;
  int x4, V4, sx, sy, sz, st;  // site index and the index strides of x, y, z, t
  int xm, ym, zm, tm;          // index offsets of the backward neighbours (wrapped)
  float ct_f, ct_b;            // factors of the t hops (boundary phase)
  __device__ __forceinline__ int off(int xi, int yi, int zi) const {
    return (((zi * TY + yi) * 12) * LX + xi) * 32 + p * 16;
  }
  __device__ __forceinline__ PairS<S::cstride> nb(int d) const {
    const char* b;
    switch (d) {
      case 0: b = mid + off(x + 1 == LX ? 0 : x + 1, yy, zz); break;
      case 1: b = mid + off(x == 0 ? LX - 1 : x - 1, yy, zz); break;
      case 2: b = yy + 1 < TY ? mid + off(x, yy + 1, zz) : halo + S::yface + ((zz * 12) * LX + x) * 32 + p * 16; break;
      case 3: b = yy > 0 ? mid + off(x, yy - 1, zz) : halo + ((zz * 12) * LX + x) * 32 + p * 16; break;
      case 4:
        b = zz + 1 < TZ ? mid + off(x, yy, zz + 1)
                        : halo + 2 * S::yface + S::zface + ((yy * 12) * LX + x) * 32 + p * 16;
        break;
      case 5: b = zz > 0 ? mid + off(x, yy, zz - 1) : halo + 2 * S::yface + ((yy * 12) * LX + x) * 32 + p * 16; break;
      case 6: b = next + off(x, yy, zz); break;
      default: b = prev + off(x, yy, zz); break;
    }
    return PairS<S::cstride>{b};
  }
  __device__ __forceinline__ const cpx<float>* link(int d) const {
    const int mu = d >> 1;
    int y4 = x4;
    if (d & 1) y4 += mu == 0 ? xm : mu == 1 ? ym : mu == 2 ? zm : tm;
    return U + (unsigned)((mu * V4 + y4) * 9);
  }
  __device__ __forceinline__ float coef(int d) const { return d == 6 ? ct_f : d == 7 ? ct_b : -0.5f; }
};

struct TmaArgs {
  Geom g;
  float diag, mf;
  const cpx<float>* U;
  const cpx<float>* in;
  cpx<float>* out;
  int tc;     // planes per unit
  int units;  // quads x (y, z) tiles x t-chunks x right-hand sides
  RedScratch rs;
  double* result;
  X2Cheb ch;
};

template <int LS, int EPI, int LX, int TY, int TZ>
__global__ void __launch_bounds__(2 * LX * TY * TZ, 1)
    g5dwf_tma_kernel(const __grid_constant__ CUtensorMap mplane, const __grid_constant__ CUtensorMap myface,
                     const __grid_constant__ CUtensorMap mzface, TmaArgs a) {
  typedef Shape<LX, TY, TZ> S;
  constexpr int Q = LS / 4;
  extern __shared__ __align__(128) char smem[];
  const Geom& g = a.g;
  const int Ly = g.L[1], Lz = g.L[2], Lt = g.L[3];
  const int nyt = Ly / TY, nzt = Lz / TZ, nch = Lt / a.tc;
  const uint32_t sbase = smem_addr(smem);
  const uint32_t bar0 = sbase + S::off_bar;  // plane slots 0..2 at +0, +8, +16; faces at +24
  const uint32_t barh = bar0 + 24;
  const int tid = threadIdx.x;
  const int p = tid & 1, sidx = tid >> 1, x = sidx % LX, row = sidx / LX, yy = row % TY, zz = row / TY;
  if (tid == 0) {
    for (int i = 0; i < 4; ++i) mbar_init(bar0 + 8 * i);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  uint32_t par = 0u;                   // bit i: parity of the next phase of barrier i
  uint32_t pend = 0u;                  // barriers with a copy in flight (bit i: barrier i)
  bool ok = true;
  double dot = 0.0;
  const long long fsize = g.V5 * 12;
  const int sx = 1, sy = g.L[0], sz = g.L[0] * Ly, st = sz * Lz;

  for (int u = blockIdx.x; u < a.units && ok; u += gridDim.x) {
    int rem = u;
    const int q = rem % Q;
    rem /= Q;
    const int yz = rem % (nyt * nzt);
    rem /= nyt * nzt;
    const int ch = rem % nch;
    const int r = rem / nch;
    const int y0 = (yz % nyt) * TY, z0 = (yz / nyt) * TZ, t0 = ch * a.tc;
    const int t1 = t0 + a.tc;
    auto tplane = [&](int t) { return (t + Lt) % Lt; };
    auto c4 = [&](int z, int t) { return z + Lz * (tplane(t) + Lt * r); };
    auto slot = [&](int t) { return (t - t0 + 1) % 3; };
    // copies, issued by thread 0 (every thread tracks the same pending set)
    auto issue_plane = [&](int t) {
      const int sl = slot(t);
      if (tid == 0) {
        mbar_expect(bar0 + 8 * sl, S::plane);
        tma_load(sbase + sl * S::plane, &mplane, bar0 + 8 * sl, 8 * q, y0, c4(z0, t));
      }
      pend |= 1u << sl;
    };
    auto issue_faces = [&](int t) {
      if (tid == 0) {
        mbar_expect(barh, 2 * S::yface + 2 * S::zface);
        const uint32_t h = sbase + S::off_halo;
        tma_load(h, &myface, barh, 8 * q, (y0 + Ly - 1) % Ly, c4(z0, t));
        tma_load(h + S::yface, &myface, barh, 8 * q, (y0 + TY) % Ly, c4(z0, t));
        tma_load(h + 2 * S::yface, &mzface, barh, 8 * q, y0, c4((z0 + Lz - 1) % Lz, t));
        tma_load(h + 2 * S::yface + S::zface, &mzface, barh, 8 * q, y0, c4((z0 + TZ) % Lz, t));
      }
      pend |= 8u;
    };
    auto wait = [&](int i) {  // a copy that did not arrive stays pending
      if (!(pend >> i & 1u)) return;
      if (!mbar_wait(bar0 + 8 * i, par >> i & 1u)) {
        ok = false;
        return;
      }
      par ^= 1u << i;
      pend &= ~(1u << i);
    };
    if (tid == 0) asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    issue_plane(t0 - 1);
    issue_plane(t0);
    issue_faces(t0);
    issue_plane(t0 + 1);
    wait(slot(t0 - 1));
    wait(slot(t0));
    wait(3);

    const int x4base = ((0 * Lz + z0 + zz) * Ly + y0 + yy) * g.L[0] + x;  // at t = 0
    const int s0 = 4 * q + 2 * p;
    for (int t = t0; t < t1; ++t) {
      const int x4 = x4base + t * st;
      SmemHops<LX, TY, TZ> h;
      h.prev = smem + slot(t - 1) * S::plane;
      h.mid = smem + slot(t) * S::plane;
      h.next = smem + slot(t + 1) * S::plane;
      h.halo = smem + S::off_halo;
      h.U = a.U;
      h.x = x, h.yy = yy, h.zz = zz, h.p = p;
      h.x4 = x4, h.V4 = g.V4, h.sx = sx, h.sy = sy, h.sz = sz, h.st = st;
      h.xm = x == 0 ? (LX - 1) * sx : -sx;
      h.ym = y0 + yy == 0 ? (Ly - 1) * sy : -sy;
      h.zm = z0 + zz == 0 ? (Lz - 1) * sz : -sz;
      h.tm = t == 0 ? (Lt - 1) * st : -st;
      h.ct_f = t == Lt - 1 ? -0.5f * (float)g.bc_t : -0.5f;
      h.ct_b = t == 0 ? -0.5f * (float)g.bc_t : -0.5f;
      cx2 up[2][3], lo[2][3];
      zero_acc(up, lo);
      hops_first(h, up, lo);
      ok = __syncthreads_and(ok);  // the faces and plane t-1 are free; a time-out anywhere stops the CTA
      if (!ok) break;
      if (t + 1 < t1) {
        if (tid == 0) asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        issue_faces(t + 1);
        issue_plane(t + 2);
      }
      wait(slot(t + 1));
      hops_second(h, up, lo);
      // diagonal and fifth-dimension terms: the partner pair from shared memory,
      // the neighbours across the quad's edges (or the walls) from global memory
      {
        const cpx<float>* gin = a.in + (long long)r * fsize + (unsigned)(x4 * 12 * LS);
        const char* self = h.mid + h.off(x, yy, zz);
        const char* other = self + (p ? -16 : 16);
        float4 qv[12];
#pragma unroll
        for (int c = 0; c < 12; ++c) qv[c] = *reinterpret_cast<const float4*>(self + c * S::cstride);
        const bool wl = p == 0 && q == 0, wr = p == 1 && q == Q - 1;
        const int gs = p == 0 ? (q == 0 ? LS - 1 : s0 - 1) : (q == Q - 1 ? 0 : s0 + 2);
        const int gc = p == 0 ? 0 : 6;
        cpx<float> pv[6], nv[6];
#pragma unroll
        for (int c = 0; c < 6; ++c) {
          const cpx<float> gv = ld(gin + (gc + c) * LS + gs);
          const float4 ov = *reinterpret_cast<const float4*>(other + (p ? c : c + 6) * S::cstride);
          pv[c] = p ? cpx<float>(ov.z, ov.w) : gv;
          nv[c] = p ? gv : cpx<float>(ov.x, ov.y);
        }
        local_x2(qv, pv, nv, wl ? -a.mf : 1.f, wr ? -a.mf : 1.f, a.diag, up, lo);
      }
      {
        const long long ro = (long long)r * fsize + (unsigned)(x4 * 12 * LS + (LS - 2 - s0));
        dot += store_x2<EPI>(up, lo, a.out + ro, a.in + ro, EPI == X2_CHEB ? a.ch.cur + ro : nullptr, a.ch.a,
                             a.ch.b, LS, EPI == X2_CHEB && a.ch.acc ? a.ch.acc + ro : nullptr, a.ch.ck);
      }
      if (t + 1 < t1) wait(3);
    }
    ok = __syncthreads_and(ok);  // every read of this unit's buffers is done before the next unit's copies
  }
  if (!ok) {
    if (tid == 0) atomicExch(&g_tma_timeout, 1);
    // let the copies still in flight land before the CTA leaves (bounded)
    for (int i = 0; i < 4; ++i)
      if (pend >> i & 1u) mbar_wait(bar0 + 8 * i, par >> i & 1u);
    __syncthreads();
  }
  if (EPI == X2_DOT) {
    double v[1] = {dot};
    double tot[1];
    if (grid_reduce<1>(v, a.rs, tot)) *a.result = tot[0];
  }
}

// ------------------------------------------------------------------ host side
PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;
std::once_flag g_encode_once;

int encode_fn(PFN_cuTensorMapEncodeTiled_v12000* fn) {
  std::call_once(g_encode_once, [] {
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      g_encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(f);
  });
  if (!g_encode) {
    set_error("TMA stencil: cuTensorMapEncodeTiled is not available from the driver");
    return HDCR_ERR_CUDA;
  }
  *fn = g_encode;
  return HDCR_OK;
}

// the field as the 5-d FP32 tensor of the kernel's comment, box (8, Lx, 12, by, bz)
int make_map(CUtensorMap* m, const Geom& g, const void* base, int nrhs, int by, int bz) {
  PFN_cuTensorMapEncodeTiled_v12000 enc;
  HDCR_TRY(encode_fn(&enc));
  const cuuint64_t Ls = (cuuint64_t)g.Ls;
  const cuuint64_t dims[5] = {2 * Ls, (cuuint64_t)g.L[0], 12, (cuuint64_t)g.L[1],
                              (cuuint64_t)g.L[2] * g.L[3] * (cuuint64_t)nrhs};
  const cuuint64_t site = 12 * Ls * 8;  // bytes per 4d site
  const cuuint64_t strides[4] = {site, Ls * 8, site * g.L[0], site * g.L[0] * g.L[1]};
  const cuuint32_t box[5] = {8, (cuuint32_t)g.L[0], 12, (cuuint32_t)by, (cuuint32_t)bz};
  const cuuint32_t es[5] = {1, 1, 1, 1, 1};
  const CUresult r = enc(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 5, const_cast<void*>(base), dims, strides, box, es,
                         CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                         CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) {
    set_error("TMA stencil: cuTensorMapEncodeTiled failed (%d)", (int)r);
    return HDCR_ERR_CUDA;
  }
  return HDCR_OK;
}

template <int LX, int TY, int TZ>
bool shape_fits(const Geom& g) {
  return (g.Ls == 16 || g.Ls == 8) && g.L[0] == LX && g.L[1] % TY == 0 && g.L[2] % TZ == 0 && g.L[3] >= 2;
}

// planes per unit: fewest (waves x (planes + 2 start-up planes)) over the divisors of Lt
int pick_chunk(const Geom& g, long long per_chunk_units, int sms) {
  int best = g.L[3];
  long long best_cost = -1;
  for (int tc = g.L[3]; tc >= 2; --tc) {
    if (g.L[3] % tc) continue;
    const long long units = per_chunk_units * (g.L[3] / tc);
    const long long waves = (units + sms - 1) / sms;
    const long long cost = waves * (tc + 2);
    if (best_cost < 0 || cost < best_cost) {
      best_cost = cost;
      best = tc;
    }
  }
  return best;
}

template <int EPI, int LX, int TY, int TZ>
int launch_shape(const Geom& g, float diag, float mf, const cpx<float>* U, const cpx<float>* in, cpx<float>* out,
                 int nrhs, RedScratch rs, double* result, X2Cheb ch, cudaStream_t st) {
  typedef Shape<LX, TY, TZ> S;
  static_assert(S::smem <= 227 * 1024, "shared memory of the TMA stencil");
  static_assert(S::threads <= RED_THREADS, "the reducing epilogue sums at most RED_THREADS threads");
  int dev = 0, sms = 0;
  HDCR_CUDA_TRY(cudaGetDevice(&dev));
  HDCR_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  CUtensorMap mp, my, mz;
  HDCR_TRY(make_map(&mp, g, in, nrhs, TY, TZ));
  HDCR_TRY(make_map(&my, g, in, nrhs, 1, TZ));
  HDCR_TRY(make_map(&mz, g, in, nrhs, TY, 1));
  TmaArgs a;
  a.g = g;
  a.diag = diag;
  a.mf = mf;
  a.U = U;
  a.in = in;
  a.out = out;
  const long long per_chunk = (long long)(g.Ls / 4) * (g.L[1] / TY) * (g.L[2] / TZ) * nrhs;
  a.tc = pick_chunk(g, per_chunk, sms);
  a.units = (int)(per_chunk * (g.L[3] / a.tc));
  a.rs = rs;
  a.result = result;
  a.ch = ch;
  const int grid = a.units < sms ? a.units : sms;
  // the dynamic shared-memory limit is a per-device attribute of each kernel: set it
  // once per device (a race only sets it twice)
  static std::atomic<unsigned long long> configured16{0}, configured8{0};
  const unsigned long long bit = dev < 64 ? 1ull << dev : 0ull;
  if (g.Ls == 16) {
    auto k = g5dwf_tma_kernel<16, EPI, LX, TY, TZ>;
    if (!bit || !(configured16.load() & bit)) {
      HDCR_CUDA_TRY(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, S::smem));
      configured16.fetch_or(bit);
    }
    k<<<grid, S::threads, S::smem, st>>>(mp, my, mz, a);
  } else {
    auto k = g5dwf_tma_kernel<8, EPI, LX, TY, TZ>;
    if (!bit || !(configured8.load() & bit)) {
      HDCR_CUDA_TRY(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, S::smem));
      configured8.fetch_or(bit);
    }
    k<<<grid, S::threads, S::smem, st>>>(mp, my, mz, a);
  }
  count_launch();
  HDCR_LAUNCH_CHECK();
  return HDCR_OK;
}

// the shapes: (Lx, TY, TZ)
#define HDCR_TMA_SHAPES(V) V(0, 16, 4, 2)

}  // namespace

bool tma_shape_fits(int shape, const Geom& g, const void* in, const void* out) {
  if ((((uintptr_t)in) | ((uintptr_t)out)) & 15) return false;
  switch (shape) {
#define HDCR_TMA_FITS(K, A, B, C) \
  case K:                         \
    return shape_fits<A, B, C>(g);
    HDCR_TMA_SHAPES(HDCR_TMA_FITS)
#undef HDCR_TMA_FITS
    default:
      return false;
  }
}

int launch_g5dwf_tma(int shape, int epi, const Geom& g, float diag, float mf, const cpx<float>* U,
                     const cpx<float>* in, cpx<float>* out, int nrhs, RedScratch rs, double* result, X2Cheb ch,
                     cudaStream_t st) {
  switch (shape) {
#define HDCR_TMA_CASE(K, A, B, C)                                                                                \
  case K:                                                                                                        \
    if (epi == X2_DOT) return launch_shape<X2_DOT, A, B, C>(g, diag, mf, U, in, out, nrhs, rs, result, ch, st);  \
    if (epi == X2_CHEB) return launch_shape<X2_CHEB, A, B, C>(g, diag, mf, U, in, out, nrhs, rs, result, ch, st); \
    return launch_shape<X2_STORE, A, B, C>(g, diag, mf, U, in, out, nrhs, rs, result, ch, st);
    HDCR_TMA_SHAPES(HDCR_TMA_CASE)
#undef HDCR_TMA_CASE
    default:
      set_error("TMA stencil: unknown shape %d", shape);
      return HDCR_ERR_BAD_ARG;
  }
}

int tma_take_timeouts(int* flag) {
  int z = 0;
  HDCR_CUDA_TRY(cudaMemcpyFromSymbol(flag, g_tma_timeout, sizeof(int)));
  if (*flag) HDCR_CUDA_TRY(cudaMemcpyToSymbol(g_tma_timeout, &z, sizeof(int)));
  return HDCR_OK;
}

}  // namespace hdcr
