// FP16 storage of the fermion fields for the FP32 operator H = Gamma5 D_dwf
// (Section 3): half-precision storage, FP32 arithmetic.
//
// Storage (HDCR_H16): a field of 12 V5 complex numbers is kept as 12 V5 half2
// (FP16 real and imaginary parts) in the psi[x4][c][s] layout, followed by V5
// FP32 scales, one per 5d site (x4, s) at index x4 * Ls + s.  A component is its
// half2 times its site's scale.  The encoder takes the scale to be the largest
// |re|, |im| among the site's 24 reals, so every stored half lies in [-1, 1] and
// is rounded to 2^-11 of the site's largest entry.  52 bytes a site (fields of
// nrhs follow one another).
//
// The kernel is the packed FP32 one (two fifth-dimension sites per thread, the
// hop arithmetic of dwf_x2.cuh) with one 8-byte load of two half2 per component,
// one 8-byte load of the pair's scales per site visited, and the result encoded
// site by site on the way out.
#include <cuda_fp16.h>

#include "blas.cuh"
#include "dwf_x2.cuh"

namespace hdcr {

constexpr int H16_SITES = 16;  // 4d sites per CTA (the linear tile)

// element offsets of one H16 field of geometry g (in half2 / float units)
struct H16Field {
  const __half2* h;
  const float* n;
};

__device__ __forceinline__ float2 h2f(uint32_t v) {
  __half2 x;
  memcpy(&x, &v, 4);
  return __half22float2(x);
}

__device__ __forceinline__ uint32_t f2h(float a, float b) {
  const __half2 x = __floats2half2_rn(a, b);
  uint32_t v;
  memcpy(&v, &x, 4);
  return v;
}

// component c of a pair (s0, s0+1) in an H16 field: q at (x4, 0, s0) in units of
// two half2, n0 and n1 the pair's scales
struct PairH16 {
  const uint2* q;
  float n0, n1;
  int hls;  // Ls / 2
  __device__ __forceinline__ float4 operator()(int c) const {
    const uint2 r = __ldg(q + c * hls);
    const float2 a = h2f(r.x), b = h2f(r.y);
    return make_float4(a.x * n0, a.y * n0, b.x * n1, b.y * n1);
  }
};

__device__ __forceinline__ PairH16 h16_pair(const H16Field& f, int x4, int s0, int ls) {
  const float2 nn = __ldg(reinterpret_cast<const float2*>(f.n + x4 * ls + s0));
  return PairH16{reinterpret_cast<const uint2*>(f.h + (unsigned)(x4 * 12 * ls + s0)), nn.x, nn.y, ls >> 1};
}

// one complex number (x4, c, s) of an H16 field, decoded
__device__ __forceinline__ cpx<float> h16_one(const H16Field& f, int x4, int c, int s, int ls, float n) {
  uint32_t v;
  const __half2 x = __ldg(f.h + (unsigned)((x4 * 12 + c) * ls + s));
  memcpy(&v, &x, 4);
  const float2 a = h2f(v);
  return cpx<float>(a.x * n, a.y * n);
}

// blockDim = 16 * Ls/2; one CTA per 16 consecutive 4d sites and right-hand side blockIdx.y
template <int LS>
__global__ void __launch_bounds__(128, 4) g5dwf_h16_kernel(Geom g, float diag, float mf,
                                                           const cpx<float>* __restrict__ U,
                                                           const unsigned char* __restrict__ in,
                                                           unsigned char* __restrict__ out) {
  __shared__ X2Stage<H16_SITES> sm;
  typedef Tile<H16_SITES, 0, 0, 0> T;
  const int ls = ls_of<LS>(g);
  const int lp = ls >> 1;
  const int site = threadIdx.x / lp, p = threadIdx.x - site * lp;
  const long long fbytes = 52 * g.V5;  // one field
  const H16Field fin{reinterpret_cast<const __half2*>(in + blockIdx.y * fbytes),
                     reinterpret_cast<const float*>(in + blockIdx.y * fbytes + 48 * g.V5)};
  __half2* hout = reinterpret_cast<__half2*>(out + blockIdx.y * fbytes);
  float* nout = reinterpret_cast<float*>(out + blockIdx.y * fbytes + 48 * g.V5);
  stage_sites<T>(g, blockIdx.x, sm);
  const int x4 = sm.x4[site];
  if (x4 < 0) return;
  const int s0 = 2 * p;
  cx2 up[2][3], lo[2][3];
  {
    // diagonal and fifth-dimension terms (as in the FP32 kernel)
    const bool wl = s0 == 0, wr = s0 + 2 == ls;
    const int sp_ = wl ? ls - 1 : s0 - 1, sn_ = wr ? 0 : s0 + 2;
    const float np_ = __ldg(fin.n + x4 * ls + sp_), nn_ = __ldg(fin.n + x4 * ls + sn_);
    const float w0 = wl ? -mf : 1.f, w1 = wr ? -mf : 1.f;
    const PairH16 self = h16_pair(fin, x4, s0, ls);
#pragma unroll
    for (int c = 0; c < 6; ++c) {
      const float4 q = self(c);
      const cpx<float> v = h16_one(fin, x4, c, sp_, ls, np_);
      const int sp = c / 3, cc = c % 3;
      up[sp][cc].re = make_float2(fmaf(-w0, v.re, diag * q.x), fmaf(-1.f, q.x, diag * q.z));
      up[sp][cc].im = make_float2(fmaf(-w0, v.im, diag * q.y), fmaf(-1.f, q.y, diag * q.w));
    }
#pragma unroll
    for (int c = 6; c < 12; ++c) {
      const float4 q = self(c);
      const cpx<float> v = h16_one(fin, x4, c, sn_, ls, nn_);
      const int sp = c / 3 - 2, cc = c % 3;
      lo[sp][cc].re = make_float2(fmaf(-diag, q.x, q.z), fmaf(-diag, q.z, w1 * v.re));
      lo[sp][cc].im = make_float2(fmaf(-diag, q.y, q.w), fmaf(-diag, q.w, w1 * v.im));
    }
  }
  const int* nbs = sm.nb[site];
  const float* cfs = sm.coef[site];
  hop_x2<0, +1>(U + (unsigned)(sm.li[site][0] * 9), h16_pair(fin, nbs[0], s0, ls), cfs[0], up, lo);
  hop_x2<0, -1>(U + (unsigned)(sm.li[site][1] * 9), h16_pair(fin, nbs[1], s0, ls), cfs[1], up, lo);
  hop_x2<1, +1>(U + (unsigned)(sm.li[site][2] * 9), h16_pair(fin, nbs[2], s0, ls), cfs[2], up, lo);
  hop_x2<1, -1>(U + (unsigned)(sm.li[site][3] * 9), h16_pair(fin, nbs[3], s0, ls), cfs[3], up, lo);
  hop_x2<2, +1>(U + (unsigned)(sm.li[site][4] * 9), h16_pair(fin, nbs[4], s0, ls), cfs[4], up, lo);
  hop_x2<2, -1>(U + (unsigned)(sm.li[site][5] * 9), h16_pair(fin, nbs[5], s0, ls), cfs[5], up, lo);
  hop_x2<3, +1>(U + (unsigned)(sm.li[site][6] * 9), h16_pair(fin, nbs[6], s0, ls), cfs[6], up, lo);
  hop_x2<3, -1>(U + (unsigned)(sm.li[site][7] * 9), h16_pair(fin, nbs[7], s0, ls), cfs[7], up, lo);
  // out(Ls-1-s) = gamma5 acc(s): lane y (site s0+1) lands at Ls-2-s0, lane x at Ls-1-s0;
  // each output site is encoded with its own scale
  float my = 0.f, mx = 0.f;
#pragma unroll
  for (int c = 0; c < 12; ++c) {
    const cx2 v = c < 6 ? up[c / 3][c % 3] : lo[c / 3 - 2][c % 3];
    my = fmaxf(my, fmaxf(fabsf(v.re.y), fabsf(v.im.y)));
    mx = fmaxf(mx, fmaxf(fabsf(v.re.x), fabsf(v.im.x)));
  }
  const float iy = my > 0.f ? 1.f / my : 0.f, ix = mx > 0.f ? 1.f / mx : 0.f;
  const int so = ls - 2 - s0;
  uint2* ho = reinterpret_cast<uint2*>(hout + (unsigned)(x4 * 12 * ls + so));
#pragma unroll
  for (int c = 0; c < 12; ++c) {
    const cx2 v = c < 6 ? up[c / 3][c % 3] : lo[c / 3 - 2][c % 3];
    ho[c * lp] = make_uint2(f2h(v.re.y * iy, v.im.y * iy), f2h(v.re.x * ix, v.im.x * ix));
  }
  *reinterpret_cast<float2*>(nout + x4 * ls + so) = make_float2(my, mx);
}

// encode: one thread per 5d site (x4, s) of field f
template <typename R>
__global__ void h16_encode_kernel(Geom g, const cpx<R>* __restrict__ in, unsigned char* __restrict__ out,
                                  int nfields) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= g.V5 * nfields) return;
  const long long f = i / g.V5;
  const long long i5 = i - f * g.V5;
  const int x4 = (int)(i5 / g.Ls), s = (int)(i5 - (long long)x4 * g.Ls);
  const cpx<R>* src = in + f * 12 * g.V5;
  __half2* h = reinterpret_cast<__half2*>(out + f * 52 * g.V5);
  float* n = reinterpret_cast<float*>(out + f * 52 * g.V5 + 48 * g.V5);
  float v[24];
  float m = 0.f;
#pragma unroll
  for (int c = 0; c < 12; ++c) {
    const cpx<R> z = ld(src + fidx(g, c, i5));
    v[2 * c] = (float)z.re;
    v[2 * c + 1] = (float)z.im;
    m = fmaxf(m, fmaxf(fabsf(v[2 * c]), fabsf(v[2 * c + 1])));
  }
  const float inv = m > 0.f ? 1.f / m : 0.f;
#pragma unroll
  for (int c = 0; c < 12; ++c) h[fidx(g, c, i5)] = __floats2half2_rn(v[2 * c] * inv, v[2 * c + 1] * inv);
  n[i5] = m;
}

template <typename R>
__global__ void h16_decode_kernel(Geom g, const unsigned char* __restrict__ in, cpx<R>* __restrict__ out,
                                  int nfields) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= g.V5 * nfields) return;
  const long long f = i / g.V5;
  const long long i5 = i - f * g.V5;
  const __half2* h = reinterpret_cast<const __half2*>(in + f * 52 * g.V5);
  const float m = reinterpret_cast<const float*>(in + f * 52 * g.V5 + 48 * g.V5)[i5];
  cpx<R>* dst = out + f * 12 * g.V5;
#pragma unroll
  for (int c = 0; c < 12; ++c) {
    const float2 a = __half22float2(h[fidx(g, c, i5)]);
    st(dst + fidx(g, c, i5), cpx<R>((R)(a.x * m), (R)(a.y * m)));
  }
}

int launch_g5dwf_h16(const Geom& g, double M5, double mf, const cpx<float>* U, const void* in, void* out, int nrhs,
                     cudaStream_t st) {
  const dim3 grid((g.V4 + H16_SITES - 1) / H16_SITES, nrhs);
  const int threads = H16_SITES * (g.Ls / 2);
  const float diag = (float)(5.0 - M5), fmf = (float)mf;
  const unsigned char* pi = (const unsigned char*)in;
  unsigned char* po = (unsigned char*)out;
  if (g.Ls == 16)
    g5dwf_h16_kernel<16><<<grid, threads, 0, st>>>(g, diag, fmf, U, pi, po);
  else if (g.Ls == 8)
    g5dwf_h16_kernel<8><<<grid, threads, 0, st>>>(g, diag, fmf, U, pi, po);
  else
    g5dwf_h16_kernel<0><<<grid, threads, 0, st>>>(g, diag, fmf, U, pi, po);
  count_launch();
  HDCR_LAUNCH_CHECK();
  return HDCR_OK;
}

}  // namespace hdcr

using namespace hdcr;

static int h16_common(const hdcr_geom* gp, const void* a, const void* b, int dtype, int n, Geom* g) {
  HDCR_TRY(make_geom(gp, g));
  if (!a || !b || a == b || n < 1 || n > 65535) {
    set_error("FP16 field conversion: bad pointers or field count");
    return HDCR_ERR_BAD_ARG;
  }
  if (dtype != HDCR_C128 && dtype != HDCR_C64) {
    set_error("FP16 field conversion: dtype %d is not C128 or C64", dtype);
    return HDCR_ERR_BAD_ARG;
  }
  if (((uintptr_t)a | (uintptr_t)b) & 15) {
    set_error("FP16 field conversion: buffers must be 16-byte aligned");
    return HDCR_ERR_BAD_ARG;
  }
  return HDCR_OK;
}

extern "C" int hdcr_fermion_encode_h16(const hdcr_geom* gp, const void* in, int in_dtype, void* out, int nfields,
                                       void* stream) {
  Geom g;
  HDCR_TRY(h16_common(gp, in, out, in_dtype, nfields, &g));
  const long long n = g.V5 * nfields;
  cudaStream_t st = as_stream(stream);
  if (in_dtype == HDCR_C128)
    h16_encode_kernel<double><<<num_blocks(n, 256), 256, 0, st>>>(g, (const cpx<double>*)in, (unsigned char*)out,
                                                                  nfields);
  else
    h16_encode_kernel<float><<<num_blocks(n, 256), 256, 0, st>>>(g, (const cpx<float>*)in, (unsigned char*)out,
                                                                 nfields);
  count_launch();
  HDCR_LAUNCH_CHECK();
  return HDCR_OK;
}

extern "C" int hdcr_fermion_decode_h16(const hdcr_geom* gp, const void* in, void* out, int out_dtype, int nfields,
                                       void* stream) {
  Geom g;
  HDCR_TRY(h16_common(gp, in, out, out_dtype, nfields, &g));
  const long long n = g.V5 * nfields;
  cudaStream_t st = as_stream(stream);
  if (out_dtype == HDCR_C128)
    h16_decode_kernel<double><<<num_blocks(n, 256), 256, 0, st>>>(g, (const unsigned char*)in, (cpx<double>*)out,
                                                                  nfields);
  else
    h16_decode_kernel<float><<<num_blocks(n, 256), 256, 0, st>>>(g, (const unsigned char*)in, (cpx<float>*)out,
                                                                 nfields);
  count_launch();
  HDCR_LAUNCH_CHECK();
  return HDCR_OK;
}
