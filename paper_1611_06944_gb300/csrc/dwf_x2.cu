// FP32 fine operator H = Gamma5 D_dwf (Section 3) on the packed FP32 pipe.
//
// Each thread owns the two fifth-dimension sites (s, s+1), s even, of one 4d
// site and keeps every complex number of the pair as two float2 lanes
// (re_s, re_s+1) and (im_s, im_s+1).  The two sites see the same gauge link,
// so the SU(3) multiply of a hop is one packed FMA per real multiply-add for
// both sites (fma.rn.f32x2), and each spinor component is one 16-byte load of
// two consecutive complex numbers of the psi[x4][c][s] layout.
//
// A CTA covers a tile of 4d sites (16 to 64 of them, x fastest) and all their
// fifth-dimension pairs.  The neighbour indices, boundary factors and link
// offsets of its sites are worked out once into shared memory; the spinors and
// the link elements themselves are read straight from global memory, where the
// Ls/2 threads of a 4d site read the same link address (one broadcast per
// quarter warp) and the hops that stay inside the tile hit L1.  The tile shape
// is picked per lattice by a small autotuner (below).  Staging the links in
// shared memory instead, or sharing them between the threads with shuffles,
// measured slower on GB300.
//
// The projection onto the two-spinor h of a hop and the fifth-dimension terms
// are formed lane by lane in scalar FP32 (they write the packed registers
// directly); the lower spin components are accumulated with the sign of Gamma5
// already applied, and the store writes the pair at Ls-2-s with its lanes
// swapped (the R5 reflection).
#include <map>
#include <mutex>
#include <tuple>

#include "dwf_tma.cuh"
#include "dwf_x2.cuh"
#include "reduce.cuh"

namespace hdcr {

constexpr int X2_MAX_LP = 8;   // fifth-dimension pairs per 4d site (Ls <= 16)

// Neighbours of one pair for the shared hop order: spinors and links read
// straight from global memory, indices from the CTA's staged site data.
struct GlobalHops {
  const cpx<float>* in;
  const cpx<float>* U;
  const int* nbs;
  const int* lis;
  const float* cfs;
  int ls, s0;
  __device__ __forceinline__ PairF32 nb(int d) const { return PairF32{in + (unsigned)(nbs[d] * 12 * ls + s0), ls}; }
  __device__ __forceinline__ const cpx<float>* link(int d) const { return U + (unsigned)(lis[d] * 9); }
  __device__ __forceinline__ float coef(int d) const { return cfs[d]; }
};

// One pass of H over the pair (x4, s0, s0+1) of one right-hand side, in the
// shared order of dwf_x2.cuh, with the epilogue EPI (store_x2).
template <int LS, int EPI, typename Stage>
__device__ __forceinline__ void site_pair(const Geom& g, const cpx<float>* __restrict__ U, const Stage& sm,
                                          int site, int x4, int p, float diag, float mf,
                                          const cpx<float>* __restrict__ in, cpx<float>* __restrict__ out,
                                          double* dot, const X2Cheb& ch) {
  const int ls = ls_of<LS>(g);
  const int s0 = 2 * p;
  const unsigned base = (unsigned)(x4 * 12 * ls);
  cx2 up[2][3], lo[2][3];
  zero_acc(up, lo);
  const GlobalHops h{in, U, sm.nb[site], sm.li[site], sm.coef[site], ls, s0};
  hops_first(h, up, lo);
  hops_second(h, up, lo);
  {
    const cpx<float>* self = in + base + s0;
    const bool wl = s0 == 0, wr = s0 + 2 == ls;
    const cpx<float>* prv = in + base + (wl ? ls - 1 : s0 - 1);
    const cpx<float>* nxt = in + base + (wr ? 0 : s0 + 2);
    float4 q[12];
    cpx<float> pv[6], nv[6];
#pragma unroll
    for (int c = 0; c < 12; ++c) q[c] = ld4(self + c * ls);
#pragma unroll
    for (int c = 0; c < 6; ++c) {
      pv[c] = ld(prv + c * ls);
      nv[c] = ld(nxt + (c + 6) * ls);
    }
    local_x2(q, pv, nv, wl ? -mf : 1.f, wr ? -mf : 1.f, diag, up, lo);
  }
  const unsigned ob = base + (unsigned)(ls - 2 - s0);
  *dot += store_x2<EPI>(up, lo, out + ob, in + ob, EPI == X2_CHEB ? ch.cur + ob : nullptr, ch.a, ch.b, ls,
                        EPI == X2_CHEB && ch.acc ? ch.acc + ob : nullptr, ch.ck);
}

// blockDim = T::sites * Ls/2: thread (site, p) = (tid / (Ls/2), tid % (Ls/2)).
// A CTA loops over tiles (grid-stride).  With gridDim.y > 1 the right-hand side
// is blockIdx.y, so the CTAs sweep the lattice one field after the other and the
// neighbours a field's tiles share stay in L2; with gridDim.y == 1 a CTA loops
// over all nrhs fields of its tile.  Every tile shape runs 16 warps per SM at 128
// registers a thread.
template <int LS, int EPI, typename T>
__global__ void __launch_bounds__(T::sites * 8, 64 / T::sites) g5dwf_x2_kernel(
    Geom g, float diag, float mf, const cpx<float>* __restrict__ U, const cpx<float>* __restrict__ in,
    cpx<float>* __restrict__ out, int nrhs, RedScratch rs, double* result, X2Cheb ch) {
  __shared__ X2Stage<T::sites> sm;
  const int ls = ls_of<LS>(g);
  const int lp = ls >> 1;
  const int site = threadIdx.x / lp, p = threadIdx.x - site * lp;
  const int groups = T::tiles(g);
  const long long fsize = g.V5 * 12;
  double dot = 0.0;
  for (int grp = blockIdx.x; grp < groups; grp += gridDim.x) {
    stage_sites<T>(g, grp, sm);
    const int x4 = sm.x4[site];
    const int r0 = gridDim.y > 1 ? (int)blockIdx.y : 0, r1 = gridDim.y > 1 ? (int)blockIdx.y + 1 : nrhs;
    if (x4 >= 0) {
      for (int r = r0; r < r1; ++r)
        if constexpr (EPI == X2_CHEB)
          site_pair<LS, EPI>(g, U, sm, site, x4, p, diag, mf, in + r * fsize, out + r * fsize, &dot,
                             X2Cheb{ch.cur + r * fsize, ch.a, ch.b, ch.acc ? ch.acc + r * fsize : nullptr, ch.ck});
        else
          site_pair<LS, EPI>(g, U, sm, site, x4, p, diag, mf, in + r * fsize, out + r * fsize, &dot, ch);
    }
    __syncthreads();  // the per-site data is refilled for the next tile
  }
  if (EPI == X2_DOT) {
    double v[1] = {dot};
    double tot[1];
    if (grid_reduce<1>(v, rs, tot)) *result = tot[0];
  }
}

// ------------------------------------------------------------------ tile variants
// Variant k of the kernel: the tile shapes tried by the autotuner.  All keep
// 16 warps per SM; they differ in which neighbours a CTA finds in L1.
#define HDCR_X2_TILES(V)   \
  V(0, 16, 0, 0, 0)        \
  V(1, 4, 4, 1, 1)         \
  V(2, 8, 2, 1, 1)         \
  V(3, 32, 0, 0, 0)        \
  V(4, 16, 2, 1, 1)        \
  V(5, 16, 4, 1, 1)
constexpr int X2_L1_VARIANTS = 6;
// variants X2_L1_VARIANTS.. are the shared-memory (TMA-staged) kernel of dwf_tma.cu,
// one per column shape
constexpr int X2_VARIANTS = X2_L1_VARIANTS + TMA_SHAPES;

template <int EPI, typename T>
static void x2_launch(const Geom& g, int blocks, float diag, float mf, const cpx<float>* U, const cpx<float>* in,
                      cpx<float>* out, int nrhs, RedScratch rs, double* result, X2Cheb ch, cudaStream_t st) {
  const int threads = T::sites * (g.Ls / 2);
  // one grid row per right-hand side, except for the reducing epilogue (one row)
  const dim3 grid(blocks, EPI == X2_DOT || nrhs > 65535 ? 1 : nrhs);
  if (g.Ls == 16) {
    g5dwf_x2_kernel<16, EPI, T><<<grid, threads, 0, st>>>(g, diag, mf, U, in, out, nrhs, rs, result, ch);
  } else if (g.Ls == 8) {
    g5dwf_x2_kernel<8, EPI, T><<<grid, threads, 0, st>>>(g, diag, mf, U, in, out, nrhs, rs, result, ch);
  } else if constexpr (T::linear && T::sites == 16) {  // other Ls: the default tile only
    g5dwf_x2_kernel<0, EPI, T><<<grid, threads, 0, st>>>(g, diag, mf, U, in, out, nrhs, rs, result, ch);
  } else {
    return;
  }
  count_launch();
}

// Whether variant v applies to the lattice (and the fields' alignment), its tile
// count, and a launch of it.
static bool x2_variant_fits(int v, const Geom& g, const void* in, const void* out, int* tiles, int* sites) {
  if (v >= X2_L1_VARIANTS) {
    *tiles = *sites = 0;
    return tma_shape_fits(v - X2_L1_VARIANTS, g, in, out);
  }
  switch (v) {
#define HDCR_X2_FITS(K, A, B, C, D)        \
  case K: {                               \
    typedef Tile<A, B, C, D> T;           \
    *tiles = T::tiles(g);                 \
    *sites = T::sites;                    \
    return T::fits(g) && T::sites * (g.Ls / 2) <= 512 && (K == 0 || g.Ls == 8 || g.Ls == 16); \
  }
    HDCR_X2_TILES(HDCR_X2_FITS)
#undef HDCR_X2_FITS
    default:
      return false;
  }
}

template <int EPI>
static int x2_launch_variant(int v, const Geom& g, int blocks, float diag, float mf, const cpx<float>* U,
                             const cpx<float>* in, cpx<float>* out, int nrhs, RedScratch rs, double* result,
                             X2Cheb ch, cudaStream_t st) {
  if (v >= X2_L1_VARIANTS)
    return launch_g5dwf_tma(v - X2_L1_VARIANTS, EPI, g, diag, mf, U, in, out, nrhs, rs, result, ch, st);
  switch (v) {
#define HDCR_X2_CASE(K, A, B, C, D)                                                            \
  case K:                                                                                      \
    x2_launch<EPI, Tile<A, B, C, D>>(g, blocks, diag, mf, U, in, out, nrhs, rs, result, ch, st); \
    break;
    HDCR_X2_TILES(HDCR_X2_CASE)
#undef HDCR_X2_CASE
    default:
      break;
  }
  return HDCR_OK;
}

// ------------------------------------------------------------------ autotuner
// The tile shape of the FP32 operator is chosen per (device, lattice, Ls,
// nrhs) the first time a plain application of H meets that key outside a
// stream capture: every fitting variant is run on the call's own fields (the
// result does not depend on the tile, so ``out`` ends as the call leaves it)
// and timed with CUDA events on the call's stream, and the fastest is kept for
// every later call with that key (all epilogues).  Until then, and when the
// tuner is off, the linear 16-site tile runs.
namespace {
struct TuneKey {
  int dev, L[4], Ls, nrhs;
  bool operator<(const TuneKey& o) const {
    return std::tie(dev, L[0], L[1], L[2], L[3], Ls, nrhs) <
           std::tie(o.dev, o.L[0], o.L[1], o.L[2], o.L[3], o.Ls, o.nrhs);
  }
};
struct TuneEntry {
  int variant;
  float us[X2_VARIANTS];
};
std::mutex g_tune_mu;
std::map<TuneKey, TuneEntry> g_tune;
int g_tune_mode = 1;       // 1: tune on first use, 0: default tile only
int g_force_variant = -1;  // >= 0: run this variant where it fits (diagnostics)

TuneKey tune_key(const Geom& g, int nrhs) {
  TuneKey k;
  cudaGetDevice(&k.dev);
  for (int i = 0; i < 4; ++i) k.L[i] = g.L[i];
  k.Ls = g.Ls;
  k.nrhs = nrhs;
  return k;
}
}  // namespace

static int x2_tune(const Geom& g, float diag, float mf, const cpx<float>* U, const cpx<float>* in, cpx<float>* out,
                   int nrhs, cudaStream_t st, TuneEntry* e) {
  cudaEvent_t a, b;
  HDCR_CUDA_TRY(cudaEventCreate(&a));
  if (cudaEventCreate(&b) != cudaSuccess) {
    cudaEventDestroy(a);
    return cuda_status(cudaErrorMemoryAllocation, "cudaEventCreate");
  }
  RedScratch none{nullptr, nullptr};
  const X2Cheb nc{nullptr, 0.f, 0.f};
  e->variant = 0;
  float best = 1e30f;
  int status = HDCR_OK;
  for (int v = 0; v < X2_VARIANTS && status == HDCR_OK; ++v) {
    int tiles, sites;
    e->us[v] = -1.f;
    if (!x2_variant_fits(v, g, in, out, &tiles, &sites)) continue;
    constexpr int reps = 3;
    // a variant that cannot be launched here (e.g. no tensor-map support) is skipped
    if (x2_launch_variant<X2_STORE>(v, g, tiles, diag, mf, U, in, out, nrhs, none, nullptr, nc, st) != HDCR_OK) {
      cudaGetLastError();
      continue;
    }
    cudaEventRecord(a, st);
    for (int r = 0; r < reps; ++r)
      x2_launch_variant<X2_STORE>(v, g, tiles, diag, mf, U, in, out, nrhs, none, nullptr, nc, st);
    cudaEventRecord(b, st);
    cudaError_t err = cudaEventSynchronize(b);
    float ms = 0.f;
    if (err == cudaSuccess) err = cudaEventElapsedTime(&ms, a, b);
    if (err == cudaSuccess) err = cudaGetLastError();
    if (err != cudaSuccess) {
      status = cuda_status(err, "stencil autotune");
      break;
    }
    if (v >= X2_L1_VARIANTS) {  // a shared-memory variant whose copies timed out is not used
      int flag = 0;
      status = tma_take_timeouts(&flag);
      if (status != HDCR_OK) break;
      if (flag) continue;
    }
    e->us[v] = ms * 1e3f / reps;
    if (e->us[v] < best) {
      best = e->us[v];
      e->variant = v;
    }
  }
  // every variant wrote ``out``; rewrite it with the chosen one (the variants agree bit for
  // bit, but a dropped variant may have left it half written)
  if (status == HDCR_OK) {
    int tiles, sites;
    x2_variant_fits(e->variant, g, in, out, &tiles, &sites);
    status = x2_launch_variant<X2_STORE>(e->variant, g, tiles, diag, mf, U, in, out, nrhs, none, nullptr, nc, st);
  }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  return status;
}

// The variant for this call: forced, tuned (tuning now if allowed), or the default.
static int x2_pick(const Geom& g, float diag, float mf, const cpx<float>* U, const cpx<float>* in, cpx<float>* out,
                   int nrhs, bool may_tune, cudaStream_t st, int* variant) {
  int tiles, sites;
  *variant = 0;
  std::lock_guard<std::mutex> lock(g_tune_mu);
  if (g_force_variant >= 0) {
    if (x2_variant_fits(g_force_variant, g, in, out, &tiles, &sites)) *variant = g_force_variant;
    return HDCR_OK;
  }
  if (!g_tune_mode) return HDCR_OK;
  const TuneKey k = tune_key(g, nrhs);
  auto it = g_tune.find(k);
  if (it != g_tune.end()) {
    *variant = it->second.variant;
    return HDCR_OK;
  }
  if (!may_tune) return HDCR_OK;
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(st, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) return HDCR_OK;
  TuneEntry e;
  HDCR_TRY(x2_tune(g, diag, mf, U, in, out, nrhs, st, &e));
  g_tune[k] = e;
  *variant = e.variant;
  return HDCR_OK;
}

// Whether the packed kernel applies: even Ls up to 16, 16-byte aligned fields.
bool g5dwf_x2_ok(const Geom& g, const void* in, const void* out) {
  return (g.Ls % 2 == 0) && g.Ls <= 2 * X2_MAX_LP && ((((uintptr_t)in) | ((uintptr_t)out)) & 15) == 0;
}

int launch_g5dwf_x2(const Geom& g, double M5, double mf, const cpx<float>* U, const cpx<float>* in, cpx<float>* out,
                    int nrhs, RedScratch* rs, double* result, cudaStream_t st) {
  const float diag = (float)(5.0 - M5), fmf = (float)mf;
  const X2Cheb none_ch{nullptr, 0.f, 0.f};
  int v, tiles, sites;
  HDCR_TRY(x2_pick(g, diag, fmf, U, in, out, nrhs, true, st, &v));
  if (!x2_variant_fits(v, g, in, out, &tiles, &sites)) {  // a tuned shared-memory variant, misaligned fields
    v = 0;
    x2_variant_fits(v, g, in, out, &tiles, &sites);
  }
  if (rs) {
    const int blocks = tiles < RED_MAX_BLOCKS ? tiles : RED_MAX_BLOCKS;
    HDCR_TRY(x2_launch_variant<X2_DOT>(v, g, blocks, diag, fmf, U, in, out, nrhs, *rs, result, none_ch, st));
  } else {
    RedScratch none{nullptr, nullptr};
    HDCR_TRY(x2_launch_variant<X2_STORE>(v, g, tiles, diag, fmf, U, in, out, nrhs, none, nullptr, none_ch, st));
  }
  HDCR_LAUNCH_CHECK();
  return HDCR_OK;
}

int launch_g5dwf_x2_cheb(const Geom& g, double M5, double mf, const cpx<float>* U, const cpx<float>* in,
                         const cpx<float>* cur, cpx<float>* prev, float a, float b, int nrhs, cudaStream_t st,
                         cpx<float>* acc, float ck) {
  const float diag = (float)(5.0 - M5), fmf = (float)mf;
  int v, tiles, sites;
  HDCR_TRY(x2_pick(g, diag, fmf, U, in, prev, nrhs, false, st, &v));  // prev is read: no tuning here
  if (!x2_variant_fits(v, g, in, prev, &tiles, &sites)) {
    v = 0;
    x2_variant_fits(v, g, in, prev, &tiles, &sites);
  }
  RedScratch none{nullptr, nullptr};
  HDCR_TRY(x2_launch_variant<X2_CHEB>(v, g, tiles, diag, fmf, U, in, prev, nrhs, none, nullptr,
                                      X2Cheb{cur, a, b, acc, ck}, st));
  HDCR_LAUNCH_CHECK();
  return HDCR_OK;
}

int x2_tune_mode(int mode, int force_variant) {
  std::lock_guard<std::mutex> lock(g_tune_mu);
  if (mode == 2) {
    g_tune.clear();
  } else {
    g_tune_mode = mode != 0;
  }
  g_force_variant = force_variant;
  return HDCR_OK;
}

int x2_tune_info(const Geom& g, int nrhs, int* variant, float* us, int nus) {
  std::lock_guard<std::mutex> lock(g_tune_mu);
  auto it = g_tune.find(tune_key(g, nrhs));
  if (it == g_tune.end()) {
    *variant = -1;
    return HDCR_OK;
  }
  *variant = it->second.variant;
  for (int i = 0; i < nus; ++i) us[i] = i < X2_VARIANTS ? it->second.us[i] : -1.f;
  return HDCR_OK;
}

}  // namespace hdcr
