// cuBLAS handles and the complex FP32 tensor-core GEMM of the coarse level
// (see coarse_gemm.cuh).  One handle per device, created on first use with a
// library-owned workspace set explicitly, so that later calls allocate nothing
// (they may run inside a CUDA-graph capture).
#include <cublas_v2.h>

#include <atomic>
#include <mutex>

#include "coarse_gemm.cuh"

namespace hdcr {

namespace {
constexpr int MAX_DEV = 64;
constexpr size_t WS_BYTES = 256u << 20;
std::mutex g_mu;
cublasHandle_t g_handle[MAX_DEV] = {};
void* g_ws[MAX_DEV] = {};
std::atomic<unsigned long long> g_fallbacks{0};
std::atomic<unsigned long long> g_calls{0};

int blas_status(cublasStatus_t s, const char* what) {
  set_error("%s: cuBLAS status %d", what, (int)s);
  return s == CUBLAS_STATUS_ALLOC_FAILED ? HDCR_ERR_NO_MEMORY : HDCR_ERR_CUDA;
}

int handle_of(cublasHandle_t* h) {
  int dev = 0;
  HDCR_CUDA_TRY(cudaGetDevice(&dev));
  if (dev < 0 || dev >= MAX_DEV) {
    set_error("cuBLAS handle: device %d beyond the %d supported", dev, MAX_DEV);
    return HDCR_ERR_BAD_ARG;
  }
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_handle[dev]) {
    cublasHandle_t hh;
    cublasStatus_t s = cublasCreate(&hh);
    if (s != CUBLAS_STATUS_SUCCESS) return blas_status(s, "cublasCreate");
    void* ws = nullptr;
    cudaError_t e = cudaMalloc(&ws, WS_BYTES);
    if (e != cudaSuccess) {
      cublasDestroy(hh);
      return cuda_status(e, "cuBLAS workspace");
    }
    s = cublasSetWorkspace(hh, ws, WS_BYTES);
    if (s == CUBLAS_STATUS_SUCCESS) s = cublasSetEmulationStrategy(hh, CUBLAS_EMULATION_STRATEGY_EAGER);
    if (s != CUBLAS_STATUS_SUCCESS) {
      cublasDestroy(hh);
      cudaFree(ws);
      return blas_status(s, "cuBLAS handle set-up");
    }
    g_handle[dev] = hh;
    g_ws[dev] = ws;
  }
  *h = g_handle[dev];
  return HDCR_OK;
}
}  // namespace

unsigned long long gemm_fallbacks() { return g_fallbacks.load(); }

int gemm_prepare() {
  cublasHandle_t h;
  return handle_of(&h);
}

int cgemm_tc(char ta, char tb, int m, int n, int k, float alpha, const cpx<float>* A, long long lda,
             const cpx<float>* B, long long ldb, float beta, cpx<float>* C, long long ldc, cudaStream_t st,
             TcMode mode) {
  if (m == 0 || n == 0) return HDCR_OK;
  cublasHandle_t h;
  HDCR_TRY(handle_of(&h));
  // cuBLAS calls on one handle from several host threads are serialised here (the
  // stream and the call must go together)
  std::lock_guard<std::mutex> lock(g_mu);
  cublasStatus_t s = cublasSetStream(h, st);
  if (s != CUBLAS_STATUS_SUCCESS) return blas_status(s, "cublasSetStream");
  g_calls.fetch_add(1);
  const cuComplex a = make_cuComplex(alpha, 0.f), b = make_cuComplex(beta, 0.f);
  const cublasOperation_t oa = ta == 'T' ? CUBLAS_OP_T : CUBLAS_OP_N, ob = tb == 'T' ? CUBLAS_OP_T : CUBLAS_OP_N;
  const cublasComputeType_t ct =
      mode == TC_TF32 ? CUBLAS_COMPUTE_32F_FAST_TF32 : CUBLAS_COMPUTE_32F_EMULATED_16BFX9;
  s = cublasGemmEx(h, oa, ob, m, n, k, &a, A, CUDA_C_32F, (int)lda, B, CUDA_C_32F, (int)ldb, &b, C, CUDA_C_32F,
                   (int)ldc, ct, CUBLAS_GEMM_DEFAULT);
  if (s == CUBLAS_STATUS_NOT_SUPPORTED) {
    // a shape the emulated path does not take (e.g. its workspace would not fit): plain FP32
    g_fallbacks.fetch_add(1);
    s = cublasGemmEx(h, oa, ob, m, n, k, &a, A, CUDA_C_32F, (int)lda, B, CUDA_C_32F, (int)ldb, &b, C, CUDA_C_32F,
                     (int)ldc, CUBLAS_COMPUTE_32F, CUBLAS_GEMM_DEFAULT);
  }
  if (s != CUBLAS_STATUS_SUCCESS) return blas_status(s, "cublasGemmEx (complex FP32 on the tensor cores)");
  count_launch();
  return HDCR_OK;
}

}  // namespace hdcr

using namespace hdcr;

extern "C" int hdcr_tc_gemm_info(unsigned long long* calls, unsigned long long* fallbacks) {
  if (!calls || !fallbacks) {
    set_error("hdcr_tc_gemm_info: null pointer");
    return HDCR_ERR_BAD_ARG;
  }
  *calls = g_calls.load();
  *fallbacks = g_fallbacks.load();
  return HDCR_OK;
}
