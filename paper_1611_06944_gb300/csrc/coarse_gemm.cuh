// Plain complex FP32 GEMMs of the coarse level on the tensor cores, through cuBLAS:
// the rank-P updates of the dense coarse inverse (3xTF32: operands split into TF32
// hi / lo parts by the caller, one TF32 GEMM over the three products) and its
// application to several right-hand sides at once (cuBLAS's FP32 emulation on BF16
// tensor cores, three BF16 parts per operand).  Both keep FP32 accuracy and
// accumulate in FP32.
#pragma once

#include "hdcr_internal.cuh"

namespace hdcr {

// tensor-core precision of a GEMM: FP32 emulated by three BF16 parts per operand, or one
// TF32 pass (for operands the caller split into TF32 hi / lo parts itself, 3xTF32)
enum TcMode { TC_BF16X9 = 0, TC_TF32 = 1 };

// C = alpha op(A) op(B) + beta C, column-major complex FP32 (cuBLAS conventions; ta, tb:
// 'N' or 'T'), on stream st.  The first call on a device creates its cuBLAS handle with
// a fixed workspace; make it outside a stream capture (gemm_prepare).
int cgemm_tc(char ta, char tb, int m, int n, int k, float alpha, const cpx<float>* A, long long lda,
             const cpx<float>* B, long long ldb, float beta, cpx<float>* C, long long ldc, cudaStream_t st,
             TcMode mode);
// creates the current device's cuBLAS handle now (outside any capture)
int gemm_prepare();
// GEMMs that cuBLAS would not run on the emulated path and that ran in plain FP32 instead
unsigned long long gemm_fallbacks();

}  // namespace hdcr
