// Fine operator H = Gamma5 D_dwf (arXiv:1611.06944 Section 3) and the field
// utilities around it (Gamma5, layout and precision conversion).
//
// One thread per 5d site (x4, s) with s fastest, so the Ls threads of a 4d
// site are neighbours in a warp: each gauge link is fetched once per warp
// (broadcast) and reused across the fifth dimension, and every spinor plane
// load is a coalesced 8/16-byte access across the warp.  The 4d hops use the
// chiral-basis spin projection (two spin components go through the SU(3)
// multiply instead of four) and the s-hops read only the projected half of
// the neighbour spinor (P_+ = upper, P_- = lower spins in the chiral basis).
#include "dwf_stencil.cuh"

namespace hdcr {

template <typename R>
__global__ void __launch_bounds__(256) g5dwf_kernel(Geom g, R diag, R mf,
                                                    const cpx<R>* __restrict__ U,
                                                    const cpx<R>* __restrict__ in,
                                                    cpx<R>* __restrict__ out, int nrhs) {
  const long long V5 = g.V5;
  long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= V5 * nrhs) return;
  const int r = (int)(idx / V5);
  const long long i5 = idx - (long long)r * V5;
  in += (long long)r * 12 * V5;
  out += (long long)r * 12 * V5;
  cpx<R> acc[4][3];
  dwf_site<R>(g, diag, mf, U, in, i5, acc);
  store_g5r5<R>(g, out, i5, acc);
}

template <typename R>
__global__ void gamma5_r5_kernel(Geom g, const cpx<R>* __restrict__ in, cpx<R>* __restrict__ out,
                                 int nfields) {
  const long long V5 = g.V5;
  long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= V5 * 12 * nfields) return;
  const long long f = idx / (12 * V5);
  const long long rem = idx - f * 12 * V5;
  const int c = (int)(rem / V5);
  const long long i5 = rem - (long long)c * V5;
  const int s = (int)(i5 % g.Ls);
  const long long o5 = i5 - s + (g.Ls - 1 - s);
  cpx<R> v = ld(in + f * 12 * V5 + rem);
  if (c >= 6) v = cpx<R>(-v.re, -v.im);
  st(out + f * 12 * V5 + (long long)c * V5 + o5, v);
}

template <typename R>
__global__ void to_planes_kernel(long long V5, const cpx<R>* __restrict__ nat, cpx<R>* __restrict__ pl,
                                 int nfields) {
  long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;  // natural order
  if (idx >= V5 * 12 * nfields) return;
  const long long f = idx / (12 * V5);
  const long long rem = idx - f * 12 * V5;
  const long long i5 = rem / 12;
  const int c = (int)(rem - i5 * 12);
  st(pl + f * 12 * V5 + (long long)c * V5 + i5, ld(nat + idx));
}

template <typename R>
__global__ void from_planes_kernel(long long V5, const cpx<R>* __restrict__ pl, cpx<R>* __restrict__ nat,
                                   int nfields) {
  long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;  // natural order
  if (idx >= V5 * 12 * nfields) return;
  const long long f = idx / (12 * V5);
  const long long rem = idx - f * 12 * V5;
  const long long i5 = rem / 12;
  const int c = (int)(rem - i5 * 12);
  st(nat + idx, ld(pl + f * 12 * V5 + (long long)c * V5 + i5));
}

template <typename Ri, typename Ro>
__global__ void convert_kernel(const cpx<Ri>* __restrict__ in, cpx<Ro>* __restrict__ out, long long n) {
  long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  cpx<Ri> v = ld(in + i);
  st(out + i, cpx<Ro>((Ro)v.re, (Ro)v.im));
}

// ------------------------------------------------------------ host launchers
template <typename R>
int launch_g5dwf(const Geom& g, double M5, double mf, const void* U, const void* in, void* out,
                 int nrhs, cudaStream_t st) {
  const int threads = 256;
  const long long n = g.V5 * nrhs;
  g5dwf_kernel<R><<<num_blocks(n, threads), threads, 0, st>>>(
      g, (R)(5.0 - M5), (R)mf, (const cpx<R>*)U, (const cpx<R>*)in, (cpx<R>*)out, nrhs);
  HDCR_LAUNCH_CHECK();
  return HDCR_OK;
}
template int launch_g5dwf<double>(const Geom&, double, double, const void*, const void*, void*, int,
                                  cudaStream_t);
template int launch_g5dwf<float>(const Geom&, double, double, const void*, const void*, void*, int,
                                 cudaStream_t);

template <typename R>
int launch_gamma5_r5(const Geom& g, const void* in, void* out, int nfields, cudaStream_t st) {
  const long long n = g.V5 * 12 * nfields;
  gamma5_r5_kernel<R><<<num_blocks(n, 256), 256, 0, st>>>(g, (const cpx<R>*)in, (cpx<R>*)out, nfields);
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
  if (dtype == HDCR_C128) return launch_g5dwf<double>(g, p->M5, p->mf, U, in, out, nrhs, as_stream(stream));
  if (dtype == HDCR_C64) return launch_g5dwf<float>(g, p->M5, p->mf, U, in, out, nrhs, as_stream(stream));
  set_error("hdcr_apply_g5dwf: unknown dtype %d", dtype);
  return HDCR_ERR_BAD_ARG;
}

extern "C" int hdcr_apply_gamma5_r5(const hdcr_geom* gp, const void* in, void* out, int dtype,
                                    int nfields, void* stream) {
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

extern "C" int hdcr_fermion_to_planes(const hdcr_geom* gp, const void* natural, void* planes,
                                      int dtype, int nfields, void* stream) {
  Geom g;
  HDCR_TRY(planes_common(gp, natural, planes, dtype, nfields, &g));
  const long long n = g.V5 * 12 * nfields;
  cudaStream_t st = as_stream(stream);
  if (dtype == HDCR_C128)
    to_planes_kernel<double><<<num_blocks(n, 256), 256, 0, st>>>(g.V5, (const cpx<double>*)natural,
                                                                 (cpx<double>*)planes, nfields);
  else
    to_planes_kernel<float><<<num_blocks(n, 256), 256, 0, st>>>(g.V5, (const cpx<float>*)natural,
                                                                (cpx<float>*)planes, nfields);
  HDCR_LAUNCH_CHECK();
  return HDCR_OK;
}

extern "C" int hdcr_fermion_from_planes(const hdcr_geom* gp, const void* planes, void* natural,
                                        int dtype, int nfields, void* stream) {
  Geom g;
  HDCR_TRY(planes_common(gp, planes, natural, dtype, nfields, &g));
  const long long n = g.V5 * 12 * nfields;
  cudaStream_t st = as_stream(stream);
  if (dtype == HDCR_C128)
    from_planes_kernel<double><<<num_blocks(n, 256), 256, 0, st>>>(g.V5, (const cpx<double>*)planes,
                                                                   (cpx<double>*)natural, nfields);
  else
    from_planes_kernel<float><<<num_blocks(n, 256), 256, 0, st>>>(g.V5, (const cpx<float>*)planes,
                                                                  (cpx<float>*)natural, nfields);
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
