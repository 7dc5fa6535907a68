// Plain complex FP32 GEMMs of the coarse level on the tensor cores, through cuBLAS:
// the rank-P updates of the dense coarse inverse and its application to several
// right-hand sides at once.  The products use cuBLAS's FP32 emulation on BF16
// tensor cores (each FP32 operand split into three BF16 parts, FP32
// accumulation), which keeps FP32 accuracy.
#pragma once

#include "hdcr_internal.cuh"

namespace hdcr {

// C = alpha op(A) op(B) + beta C, column-major complex FP32 (cuBLAS conventions; ta, tb:
// 'N' or 'T'), on stream st.  The first call on a device creates its cuBLAS handle with
// a fixed workspace; make it outside a stream capture (gemm_prepare).
int cgemm_tc(char ta, char tb, int m, int n, int k, float alpha, const cpx<float>* A, long long lda,
             const cpx<float>* B, long long ldb, float beta, cpx<float>* C, long long ldc, cudaStream_t st);
// creates the current device's cuBLAS handle now (outside any capture)
int gemm_prepare();
// GEMMs that cuBLAS would not run on the emulated path and that ran in plain FP32 instead
unsigned long long gemm_fallbacks();

}  // namespace hdcr
