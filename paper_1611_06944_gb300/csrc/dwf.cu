// Fine operator H = Gamma5 D_dwf (arXiv:1611.06944 Section 3) and the field
// utilities around it (Gamma5, layout and precision conversion).
//
// One thread per 5d site (x4, s) with s fastest, so the Ls threads of a 4d
// site are neighbours in a warp: each gauge link is fetched once per warp
// (broadcast) and reused across the fifth dimension.  In the field layout
// psi[x4][c][s] every component load is a run of Ls consecutive complex
// numbers across those threads (coalesced), at an immediate offset c*Ls from
// one base address per site when Ls is a compile-time constant.  The 4d hops use the
// chiral-basis spin projection (two spin components go through the SU(3)
// multiply instead of four) and the s-hops read only the projected half of
// the neighbour spinor (P_+ = upper, P_- = lower spins in the chiral basis).
#include <mutex>
#include <vector>

#include "host_io.cuh"
#include "blas.cuh"
#include "dwf_stencil.cuh"

namespace hdcr {

template <typename R, int LS>
__global__ void __launch_bounds__(256, 2) g5dwf_kernel(Geom g, R diag, R mf, const cpx<R>* __restrict__ U,
                                                       const cpx<R>* __restrict__ in, cpx<R>* __restrict__ out,
                                                       int nrhs) {
  const int ls = ls_of<LS>(g);
  const long long V5 = g.V5;
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= V5 * nrhs) return;
  const int r = (int)(idx / V5);
  const int i5 = (int)(idx - (long long)r * V5);
  const int x4 = i5 / ls;
  const int s = i5 - x4 * ls;
  in += (long long)r * 12 * V5;
  out += (long long)r * 12 * V5;
  cpx<R> acc[4][3];
  dwf_site<R, LS>(g, diag, mf, U, in, x4, s, acc);
  store_g5r5<R, LS>(g, out, x4, s, acc);
}

// One step of the Chebyshev smoother's recurrence fused into the FP64 operator:
// with h = H in at every element, prev <- nx = 2 (a h + b cur) - prev and
// acc += ck nx (the same arithmetic, in the same order, as the separate step
// kernel after a plain application, so the same bits).  The separate pass over
// four fields does not happen; the epilogue's own loads are not hidden behind
// the FP64 arithmetic, so a launch takes about 0.2 ms longer than a plain one
// (16^4 x 16), a small net gain.
template <int LS>
__global__ void __launch_bounds__(256, 2) g5dwf_cheb_kernel(Geom g, double diag, double mf,
                                                            const cpx<double>* __restrict__ U,
                                                            const cpx<double>* __restrict__ in,
                                                            const cpx<double>* __restrict__ cur,
                                                            cpx<double>* __restrict__ prev,
                                                            cpx<double>* __restrict__ acc_out, double a, double b,
                                                            double ck) {
  const int ls = ls_of<LS>(g);
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= g.V5) return;
  const int i5 = (int)idx;
  const int x4 = i5 / ls;
  const int s = i5 - x4 * ls;
  cpx<double> acc[4][3];
  dwf_site<double, LS>(g, diag, mf, U, in, x4, s, acc);
  const unsigned o0 = (unsigned)(x4 * 12 * ls + (ls - 1 - s));  // the R5 reflection of store_g5r5
#pragma unroll
  for (int sp = 0; sp < 4; ++sp)
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      cpx<double> h = acc[sp][c];
      if (sp >= 2) h = cpx<double>(-h.re, -h.im);
      const unsigned o = o0 + (3 * sp + c) * ls;
      const cpx<double> cv = ld(cur + o), pv = ld(prev + o);
      cpx<double> nx;
      nx.re = 2.0 * fma(a, h.re, b * cv.re) - pv.re;
      nx.im = 2.0 * fma(a, h.im, b * cv.im) - pv.im;
      st(prev + o, nx);
      cpx<double> av = ld(acc_out + o);
      av.re = fma(ck, nx.re, av.re);
      av.im = fma(ck, nx.im, av.im);
      st(acc_out + o, av);
    }
}

template <typename R>
__global__ void gamma5_r5_kernel(Geom g, const cpx<R>* __restrict__ in, cpx<R>* __restrict__ out,
                                 int nfields) {
  // element e = ((f*V4 + x4)*12 + c)*Ls + s in the field layout
  const long long n = g.V5 * 12 * nfields;
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n) return;
  const int s = (int)(e % g.Ls);
  const long long row = e / g.Ls;      // (f*V4 + x4)*12 + c
  const int c = (int)(row % 12);
  cpx<R> v = ld(in + e);
  if (c >= 6) v = cpx<R>(-v.re, -v.im);
  st(out + row * g.Ls + (g.Ls - 1 - s), v);
}

// natural[f][x4][s][c] <-> field[f][x4][c][s]
template <typename R>
__global__ void pack_kernel(Geom g, const cpx<R>* __restrict__ nat, cpx<R>* __restrict__ pl, int nfields) {
  const long long n = g.V5 * 12 * nfields;
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;  // natural order
  if (idx >= n) return;
  const int c = (int)(idx % 12);
  const long long fi5 = idx / 12;     // f*V5 + i5
  const int s = (int)(fi5 % g.Ls);
  const long long fx4 = fi5 / g.Ls;   // f*V4 + x4
  st(pl + (fx4 * 12 + c) * g.Ls + s, ld(nat + idx));
}

template <typename R>
__global__ void unpack_kernel(Geom g, const cpx<R>* __restrict__ pl, cpx<R>* __restrict__ nat, int nfields) {
  const long long n = g.V5 * 12 * nfields;
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;  // natural order
  if (idx >= n) return;
  const int c = (int)(idx % 12);
  const long long fi5 = idx / 12;
  const int s = (int)(fi5 % g.Ls);
  const long long fx4 = fi5 / g.Ls;
  st(nat + idx, ld(pl + (fx4 * 12 + c) * g.Ls + s));
}

template <typename Ri, typename Ro>
__global__ void convert_kernel(const cpx<Ri>* __restrict__ in, cpx<Ro>* __restrict__ out, long long n) {
  long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  cpx<Ri> v = ld(in + i);
  st(out + i, cpx<Ro>((Ro)v.re, (Ro)v.im));
}

// ------------------------------------------------------------ stencil timer
// While enabled, every stencil launch is bracketed by CUDA events recorded on
// its own stream; hdcr_stencil_timer_read() adds up the elapsed times per
// precision.  Up to TIMER_PAIRS launches are recorded between resets.
namespace {
constexpr int TIMER_PAIRS = 16384;
struct StencilTimer {
  std::mutex mu;
  bool enabled = false;
  std::vector<cudaEvent_t> ev;  // 2 per launch
  std::vector<int> kind;        // 0 = FP64, 1 = FP32, 2 = FP16 storage, 3 = FP64 with a smoother step
  std::vector<long long> sites;
  int used = 0;
  long long all_launches[4] = {0, 0, 0, 0};  // every launch while enabled, timed or not
  long long all_sites[4] = {0, 0, 0, 0};
};
StencilTimer g_timer;
}  // namespace

void stencil_timer_begin(int kind, long long sites, cudaStream_t st, int* slot) {
  *slot = -1;
  std::lock_guard<std::mutex> lock(g_timer.mu);
  if (!g_timer.enabled) return;
  // launches captured into a CUDA graph are not timed (their events would not
  // be recorded by a replay)
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(st, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) return;
  g_timer.all_launches[kind]++;
  g_timer.all_sites[kind] += sites;
  if (g_timer.used >= TIMER_PAIRS) return;
  const int i = g_timer.used++;
  if ((int)g_timer.kind.size() <= i) {
    cudaEvent_t a, b;
    if (cudaEventCreate(&a) != cudaSuccess || cudaEventCreate(&b) != cudaSuccess) {
      g_timer.used--;
      return;
    }
    g_timer.ev.push_back(a);
    g_timer.ev.push_back(b);
    g_timer.kind.push_back(kind);
    g_timer.sites.push_back(sites);
  }
  g_timer.kind[i] = kind;
  g_timer.sites[i] = sites;
  cudaEventRecord(g_timer.ev[2 * i], st);
  *slot = i;
}

void stencil_timer_end(int slot, cudaStream_t st) {
  if (slot < 0) return;
  std::lock_guard<std::mutex> lock(g_timer.mu);
  cudaEventRecord(g_timer.ev[2 * slot + 1], st);
}

// ------------------------------------------------------------ host launchers
template <typename R>
int launch_g5dwf(const Geom& g, double M5, double mf, const void* U, const void* in, void* out,
                 int nrhs, cudaStream_t st) {
  const int threads = 256;
  const long long n = g.V5 * nrhs;
  int slot;
  stencil_timer_begin(sizeof(R) == 8 ? 0 : 1, n, st, &slot);
  if (sizeof(R) == 4 && g5dwf_x2_ok(g, in, out)) {
    const int s = launch_g5dwf_x2(g, M5, mf, (const cpx<float>*)U, (const cpx<float>*)in, (cpx<float>*)out, nrhs,
                                  nullptr, nullptr, st);
    stencil_timer_end(slot, st);
    return s;
  }
  HDCR_DISPATCH_LS(g.Ls, (g5dwf_kernel<R, LSC><<<num_blocks(n, threads), threads, 0, st>>>(
                             g, (R)(5.0 - M5), (R)mf, (const cpx<R>*)U, (const cpx<R>*)in, (cpx<R>*)out, nrhs)));
  stencil_timer_end(slot, st);
  HDCR_LAUNCH_CHECK();
  return HDCR_OK;
}
template int launch_g5dwf<double>(const Geom&, double, double, const void*, const void*, void*, int,
                                  cudaStream_t);

int launch_g5dwf_cheb(const Geom& g, double M5, double mf, const cpx<double>* U, const cpx<double>* in,
                      const cpx<double>* cur, cpx<double>* prev, cpx<double>* acc, double a, double b, double ck,
                      cudaStream_t st) {
  const int threads = 256;
  int slot;
  stencil_timer_begin(3, g.V5, st, &slot);
  HDCR_DISPATCH_LS(g.Ls, (g5dwf_cheb_kernel<LSC><<<num_blocks(g.V5, threads), threads, 0, st>>>(
                             g, 5.0 - M5, mf, U, in, cur, prev, acc, a, b, ck)));
  stencil_timer_end(slot, st);
  HDCR_LAUNCH_CHECK();
  return HDCR_OK;
}
template int launch_g5dwf<float>(const Geom&, double, double, const void*, const void*, void*, int,
                                 cudaStream_t);

template <typename R>
int launch_gamma5_r5(const Geom& g, const void* in, void* out, int nfields, cudaStream_t st) {
  const long long n = g.V5 * 12 * nfields;
  gamma5_r5_kernel<R><<<num_blocks(n, 256), 256, 0, st>>>(g, (const cpx<R>*)in, (cpx<R>*)out, nfields); count_launch();
  HDCR_LAUNCH_CHECK();
  return HDCR_OK;
}
template int launch_gamma5_r5<double>(const Geom&, const void*, void*, int, cudaStream_t);
template int launch_gamma5_r5<float>(const Geom&, const void*, void*, int, cudaStream_t);

int launch_convert(const void* in, int idt, void* out, int odt, long long n, cudaStream_t st) {
  const int b = num_blocks(n, 256);
  if (idt == HDCR_C128 && odt == HDCR_C64)
    convert_kernel<double, float><<<b, 256, 0, st>>>((const cpx<double>*)in, (cpx<float>*)out, n);
  else if (idt == HDCR_C64 && odt == HDCR_C128)
    convert_kernel<float, double><<<b, 256, 0, st>>>((const cpx<float>*)in, (cpx<double>*)out, n);
  else if (idt == HDCR_C128 && odt == HDCR_C128)
    convert_kernel<double, double><<<b, 256, 0, st>>>((const cpx<double>*)in, (cpx<double>*)out, n);
  else if (idt == HDCR_C64 && odt == HDCR_C64)
    convert_kernel<float, float><<<b, 256, 0, st>>>((const cpx<float>*)in, (cpx<float>*)out, n);
  else {
    set_error("hdcr_convert: unknown dtype pair %d -> %d", idt, odt);
    return HDCR_ERR_BAD_ARG;
  }
  count_launch();
  HDCR_LAUNCH_CHECK();
  return HDCR_OK;
}

}  // namespace hdcr

// ===================================================================== C ABI
using namespace hdcr;

extern "C" int hdcr_apply_g5dwf(const hdcr_geom* gp, const hdcr_dwf_params* p, const void* U,
                                const void* in, void* out, int dtype, int nrhs, void* stream) {
  Geom g;
  HDCR_TRY(make_geom(gp, &g));
  if (!p || !U || !in || !out || nrhs < 1) {
    set_error("hdcr_apply_g5dwf: null pointer or nrhs < 1");
    return HDCR_ERR_BAD_ARG;
  }
  if (in == out) {
    set_error("hdcr_apply_g5dwf: in and out must not overlap");
    return HDCR_ERR_BAD_ARG;
  }
  if (dtype == HDCR_H16) {
    if (g.Ls % 2 || g.Ls > 16 || ((((uintptr_t)in) | ((uintptr_t)out)) & 15) || nrhs > 65535) {
      set_error("hdcr_apply_g5dwf: FP16 storage needs an even Ls <= 16, 16-byte aligned fields, nrhs <= 65535");
      return HDCR_ERR_BAD_ARG;
    }
    int slot;
    stencil_timer_begin(2, g.V5 * nrhs, as_stream(stream), &slot);
    const int s = launch_g5dwf_h16(g, p->M5, p->mf, (const cpx<float>*)U, in, out, nrhs, as_stream(stream));
    stencil_timer_end(slot, as_stream(stream));
    return s;
  }
  if (dtype == HDCR_C128) return launch_g5dwf<double>(g, p->M5, p->mf, U, in, out, nrhs, as_stream(stream));
  if (dtype == HDCR_C64) return launch_g5dwf<float>(g, p->M5, p->mf, U, in, out, nrhs, as_stream(stream));
  set_error("hdcr_apply_g5dwf: unknown dtype %d", dtype);
  return HDCR_ERR_BAD_ARG;
}

extern "C" int hdcr_stencil_tune(int mode, int force_variant) {
  if (mode < 0 || mode > 2 || force_variant < -1 || force_variant >= 64) {
    set_error("hdcr_stencil_tune: mode must be 0, 1 or 2 and force_variant >= -1");
    return HDCR_ERR_BAD_ARG;
  }
  return x2_tune_mode(mode, force_variant);
}

extern "C" int hdcr_stencil_tune_info(const hdcr_geom* gp, int nrhs, int* variant, float* us, int nus) {
  Geom g;
  HDCR_TRY(make_geom(gp, &g));
  if (!variant || nrhs < 1 || nus < 0 || (nus > 0 && !us)) {
    set_error("hdcr_stencil_tune_info: bad arguments");
    return HDCR_ERR_BAD_ARG;
  }
  return x2_tune_info(g, nrhs, variant, us, nus);
}

static int gamma5_r5_entry(const hdcr_geom* gp, const void* in, void* out, int dtype, int nfields,
                           void* stream) {
  Geom g;
  HDCR_TRY(make_geom(gp, &g));
  if (!in || !out || nfields < 1 || in == out) {
    set_error("hdcr_apply_gamma5_r5: bad pointers or nfields");
    return HDCR_ERR_BAD_ARG;
  }
  if (dtype == HDCR_C128) return launch_gamma5_r5<double>(g, in, out, nfields, as_stream(stream));
  if (dtype == HDCR_C64) return launch_gamma5_r5<float>(g, in, out, nfields, as_stream(stream));
  set_error("hdcr_apply_gamma5_r5: unknown dtype %d", dtype);
  return HDCR_ERR_BAD_ARG;
}

static int planes_common(const hdcr_geom* gp, const void* a, void* b, int dtype, int nfields,
                         Geom* g) {
  HDCR_TRY(make_geom(gp, g));
  if (!a || !b || nfields < 1 || a == b) {
    set_error("layout conversion: bad pointers or nfields");
    return HDCR_ERR_BAD_ARG;
  }
  if (dtype != HDCR_C128 && dtype != HDCR_C64) {
    set_error("layout conversion: unknown dtype %d", dtype);
    return HDCR_ERR_BAD_ARG;
  }
  return HDCR_OK;
}

extern "C" int hdcr_fermion_pack(const hdcr_geom* gp, const void* natural, void* packed,
                                      int dtype, int nfields, void* stream) {
  Geom g;
  HDCR_TRY(planes_common(gp, natural, packed, dtype, nfields, &g));
  const long long n = g.V5 * 12 * nfields;
  cudaStream_t st = as_stream(stream);
  if (dtype == HDCR_C128)
    pack_kernel<double><<<num_blocks(n, 256), 256, 0, st>>>(g, (const cpx<double>*)natural,
                                                                 (cpx<double>*)packed, nfields);
  else
    pack_kernel<float><<<num_blocks(n, 256), 256, 0, st>>>(g, (const cpx<float>*)natural,
                                                                (cpx<float>*)packed, nfields); count_launch();
  HDCR_LAUNCH_CHECK();
  return HDCR_OK;
}

extern "C" int hdcr_fermion_unpack(const hdcr_geom* gp, const void* packed, void* natural,
                                        int dtype, int nfields, void* stream) {
  Geom g;
  HDCR_TRY(planes_common(gp, packed, natural, dtype, nfields, &g));
  const long long n = g.V5 * 12 * nfields;
  cudaStream_t st = as_stream(stream);
  if (dtype == HDCR_C128)
    unpack_kernel<double><<<num_blocks(n, 256), 256, 0, st>>>(g, (const cpx<double>*)packed,
                                                                   (cpx<double>*)natural, nfields);
  else
    unpack_kernel<float><<<num_blocks(n, 256), 256, 0, st>>>(g, (const cpx<float>*)packed,
                                                                  (cpx<float>*)natural, nfields); count_launch();
  HDCR_LAUNCH_CHECK();
  return HDCR_OK;
}

extern "C" int hdcr_convert(const void* in, int in_dtype, void* out, int out_dtype, size_t n,
                            void* stream) {
  if (!in || !out || n == 0) {
    set_error("hdcr_convert: null pointer or n == 0");
    return HDCR_ERR_BAD_ARG;
  }
  return launch_convert(in, in_dtype, out, out_dtype, (long long)n, as_stream(stream));
}

extern "C" int hdcr_stencil_timer(int enable) {
  std::lock_guard<std::mutex> lock(g_timer.mu);
  g_timer.enabled = enable != 0;
  if (g_timer.enabled) {
    g_timer.used = 0;
    for (int k = 0; k < 3; ++k) g_timer.all_launches[k] = g_timer.all_sites[k] = 0;
  }
  return HDCR_OK;
}

static int timer_kind(int dtype) {
  return dtype == HDCR_C128 ? 0 : dtype == HDCR_C64 ? 1 : dtype == HDCR_H16 ? 2 : dtype == HDCR_TIMER_C128_CHEB ? 3 : -1;
}

extern "C" int hdcr_stencil_timer_count(int dtype, long long* launches, long long* sites) {
  const int k = timer_kind(dtype);
  if (!launches || !sites || k < 0) {
    set_error("hdcr_stencil_timer_count: bad arguments");
    return HDCR_ERR_BAD_ARG;
  }
  std::lock_guard<std::mutex> lock(g_timer.mu);
  *launches = g_timer.all_launches[k];
  *sites = g_timer.all_sites[k];
  return HDCR_OK;
}

extern "C" int hdcr_stencil_timer_read(int dtype, double* total_ms, long long* launches, long long* sites) {
  const int want = timer_kind(dtype);
  if (!total_ms || !launches || !sites || want < 0) {
    set_error("hdcr_stencil_timer_read: bad arguments");
    return HDCR_ERR_BAD_ARG;
  }
  std::lock_guard<std::mutex> lock(g_timer.mu);
  double ms = 0.0;
  long long nl = 0, ns = 0;
  for (int i = 0; i < g_timer.used; ++i) {
    if (g_timer.kind[i] != want) continue;
    HDCR_CUDA_TRY(cudaEventSynchronize(g_timer.ev[2 * i + 1]));
    float t = 0.f;
    HDCR_CUDA_TRY(cudaEventElapsedTime(&t, g_timer.ev[2 * i], g_timer.ev[2 * i + 1]));
    ms += t;
    nl++;
    ns += g_timer.sites[i];
  }
  *total_ms = ms;
  *launches = nl;
  *sites = ns;
  return HDCR_OK;
}

extern "C" int hdcr_apply_gamma5_r5(const hdcr_geom* gp, const void* in, void* out, int dtype,
                                    int nfields, void* stream) {
  Geom g;
  HDCR_TRY(make_geom(gp, &g));
  const size_t cb = dtype_complex_bytes(dtype);
  if (!cb || nfields < 1) return gamma5_r5_entry(gp, in, out, dtype, nfields, stream);
  // fields given in host memory are staged through the device
  cudaStream_t st = as_stream(stream);
  Staged si, so;
  HDCR_TRY(si.in(in, (size_t)nfields * g.V5 * 12 * cb, st));
  HDCR_TRY(so.out(out, (size_t)nfields * g.V5 * 12 * cb, st, false));
  HDCR_TRY(gamma5_r5_entry(gp, si.ptr(), so.ptr(), dtype, nfields, stream));
  return so.finish();
}
