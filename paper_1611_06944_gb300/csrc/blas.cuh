// Host-side declarations of the kernel launchers shared between translation units.
#pragma once

#include "reduce.cuh"

namespace hdcr {

template <typename R>
int launch_g5dwf(const Geom& g, double M5, double mf, const void* U, const void* in, void* out,
                 int nrhs, cudaStream_t st);
template <typename R>
int launch_gamma5_r5(const Geom& g, const void* in, void* out, int nfields, cudaStream_t st);
int launch_convert(const void* in, int idt, void* out, int odt, long long n, cudaStream_t st);

// FP32 operator on the packed two-site kernel (dwf_x2.cu); with rs non-null it
// also reduces Re <in, H in> into *result.  g5dwf_x2_ok says whether it applies.
bool g5dwf_x2_ok(const Geom& g, const void* in, const void* out);
int launch_g5dwf_x2(const Geom& g, double M5, double mf, const cpx<float>* U, const cpx<float>* in, cpx<float>* out,
                    int nrhs, RedScratch* rs, double* result, cudaStream_t st);
// prev <- nx = 2 (a H in + b cur) - prev for nrhs fields (a Chebyshev step fused into the
// FP32 stencil), and acc += ck nx when acc is set
int launch_g5dwf_x2_cheb(const Geom& g, double M5, double mf, const cpx<float>* U, const cpx<float>* in,
                         const cpx<float>* cur, cpx<float>* prev, float a, float b, int nrhs, cudaStream_t st,
                         cpx<float>* acc = nullptr, float ck = 0.f);
// FP64 operator with one Chebyshev smoother step fused into its epilogue (dwf.cu):
// prev <- nx = 2 (a H in + b cur) - prev, acc += ck nx (one field)
int launch_g5dwf_cheb(const Geom& g, double M5, double mf, const cpx<double>* U, const cpx<double>* in,
                      const cpx<double>* cur, cpx<double>* prev, cpx<double>* acc, double a, double b, double ck,
                      cudaStream_t st);
// FP32 operator on FP16-stored fields (dwf_h16.cu): nrhs fields of 52 V5 bytes each
int launch_g5dwf_h16(const Geom& g, double M5, double mf, const cpx<float>* U, const void* in, void* out, int nrhs,
                     cudaStream_t st);
// tile-shape autotuner of the FP32 operator: mode 1 tunes on first use, 0 keeps the
// default tile, 2 forgets what was tuned; force_variant >= 0 pins one variant
int x2_tune_mode(int mode, int force_variant);
int x2_tune_info(const Geom& g, int nrhs, int* variant, float* us, int nus);

template <typename R>
int launch_cdot(const void* u, const void* v, long long n, RedScratch rs, double* result, cudaStream_t st);
template <typename R>
int launch_norm2(const void* u, long long n, RedScratch rs, double* result, cudaStream_t st);

int device_red_scratch(RedScratch* out);

// stencil timer (dwf.cu): bracket one stencil launch with events when enabled
void stencil_timer_begin(int kind, long long sites, cudaStream_t st, int* slot);
void stencil_timer_end(int slot, cudaStream_t st);

}  // namespace hdcr
