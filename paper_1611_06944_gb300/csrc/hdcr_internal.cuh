// Internal definitions shared by the CUDA sources of libhdcr: lattice geometry,
// complex arithmetic, error reporting and launch helpers.
//
// Field layouts (the C ABI documents the same):
//   fermion  psi[x4][c][s]: for every 4d site x4 = ((t*Lz + z)*Ly + y)*Lx + x
//            the 12 components c = 3*spin + colour, each a run of Ls
//            interleaved complex numbers over the fifth coordinate s.  The
//            logical 5d site index is i5 = x4*Ls + s; element (c, i5) sits at
//            fidx(c, i5) = (x4*12 + c)*Ls + s.  nrhs fields follow one another.
//   gauge    U[mu][x4][a][b], a 3x3 colour matrix per link, row-major.
//   coarse   c[a][k] (coarse site a, basis index k), op A[a][leg][j][k].
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <stdio.h>
#include <string>

#include "../../include/hdcr.h"

namespace hdcr {

// ------------------------------------------------------------------ errors
void set_error(const char* fmt, ...);
int cuda_status(cudaError_t e, const char* what);

#define HDCR_CUDA_TRY(expr)                                       \
  do {                                                            \
    cudaError_t _e = (expr);                                      \
    if (_e != cudaSuccess) return ::hdcr::cuda_status(_e, #expr); \
  } while (0)

#define HDCR_TRY(expr)          \
  do {                          \
    int _s = (expr);            \
    if (_s != HDCR_OK) return _s; \
  } while (0)

#define HDCR_LAUNCH_CHECK() HDCR_CUDA_TRY(cudaGetLastError())

// number of kernels this library has launched in the process (a diagnostic)
void count_launch();
void count_launches(unsigned long long n);  // kernels a replayed CUDA graph launched
void uncount_launches(unsigned long long n);  // kernels counted while captured, not launched
unsigned long long launches_so_far();

// --------------------------------------------------------------- geometry
struct Geom {
  int L[4];      // x, y, z, t
  int Ls;
  int bc_t;      // +1 periodic, -1 antiperiodic in t
  int V4;
  long long V5;
};

int make_geom(const hdcr_geom* g, Geom* out);

__host__ __device__ inline void x4_coords(const Geom& g, int x4, int c[4]) {
  c[0] = x4 % g.L[0];
  int r = x4 / g.L[0];
  c[1] = r % g.L[1];
  r /= g.L[1];
  c[2] = r % g.L[2];
  c[3] = r / g.L[2];
}

__host__ __device__ inline int x4_index(const Geom& g, const int c[4]) {
  return ((c[3] * g.L[2] + c[2]) * g.L[1] + c[1]) * g.L[0] + c[0];
}

// offset of component c of 5d site i5 in a fermion field (fits in 32 bits: make_geom
// rejects fields of 2^31 complex numbers or more)
__host__ __device__ inline unsigned fidx(const Geom& g, int c, long long i5) {
  const unsigned x4 = (unsigned)(i5 / g.Ls);
  const unsigned s = (unsigned)(i5 - (long long)x4 * g.Ls);
  return (x4 * 12u + (unsigned)c) * (unsigned)g.Ls + s;
}

// --------------------------------------------------------------- complex
template <typename R> struct V2;
template <> struct V2<double> { typedef double2 t; };
template <> struct V2<float> { typedef float2 t; };

template <typename R>
struct cpx {
  R re, im;
  __host__ __device__ cpx() {}
  __host__ __device__ cpx(R a, R b) : re(a), im(b) {}
};

template <typename R>
__device__ __forceinline__ cpx<R> ld(const cpx<R>* p) {
  typedef typename V2<R>::t T2;
  T2 v = __ldg(reinterpret_cast<const T2*>(p));
  return cpx<R>(v.x, v.y);
}
template <typename R>
__device__ __forceinline__ void st(cpx<R>* p, cpx<R> a) {
  typedef typename V2<R>::t T2;
  T2 v;
  v.x = a.re;
  v.y = a.im;
  *reinterpret_cast<T2*>(p) = v;
}
template <typename R>
__device__ __forceinline__ cpx<R> operator+(cpx<R> a, cpx<R> b) { return cpx<R>(a.re + b.re, a.im + b.im); }
template <typename R>
__device__ __forceinline__ cpx<R> operator-(cpx<R> a, cpx<R> b) { return cpx<R>(a.re - b.re, a.im - b.im); }
template <typename R>
__device__ __forceinline__ cpx<R> operator*(R s, cpx<R> a) { return cpx<R>(s * a.re, s * a.im); }
// i * a
template <typename R>
__device__ __forceinline__ cpx<R> times_i(cpx<R> a) { return cpx<R>(-a.im, a.re); }
// acc + a * b
template <typename R>
__device__ __forceinline__ cpx<R> cmadd(cpx<R> acc, cpx<R> a, cpx<R> b) {
  acc.re = fma(a.re, b.re, acc.re);
  acc.re = fma(-a.im, b.im, acc.re);
  acc.im = fma(a.re, b.im, acc.im);
  acc.im = fma(a.im, b.re, acc.im);
  return acc;
}
// acc + conj(a) * b
template <typename R>
__device__ __forceinline__ cpx<R> cjmadd(cpx<R> acc, cpx<R> a, cpx<R> b) {
  acc.re = fma(a.re, b.re, acc.re);
  acc.re = fma(a.im, b.im, acc.re);
  acc.im = fma(a.re, b.im, acc.im);
  acc.im = fma(-a.im, b.re, acc.im);
  return acc;
}

// ---------------------------------------------------------- launch helpers
inline int num_blocks(long long n, int threads, int cap = 1 << 30) {
  long long b = (n + threads - 1) / threads;
  if (b > cap) b = cap;
  if (b < 1) b = 1;
  return (int)b;
}

inline cudaStream_t as_stream(void* s) { return reinterpret_cast<cudaStream_t>(s); }

size_t dtype_complex_bytes(int dtype);

}  // namespace hdcr
