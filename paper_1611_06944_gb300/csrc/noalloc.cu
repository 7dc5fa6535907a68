// hdcr_cdot_noalloc: the inner product of hdcr_cdot for callers that must not
// allocate device memory.
//
// hdcr_cdot keeps its partial sums in a buffer that the library allocates with
// cudaMalloc on first use.  Some callers cannot let a library allocate: callers
// that hand all device memory to their own pool or allocator up front and keep
// a fixed budget, and callers in a runtime that forbids allocations after
// start-up (a cudaMalloc there fails or stalls the caller's other streams).
// This entry point keeps its scratch in a fixed array compiled into the library
// instead, so a call only launches kernels and sets one word.
//
// The device address of the array is looked up once per device and kept for
// the life of the process; after a cudaDeviceReset (or any other destruction
// of the device's primary context) that address is stale, so no call may
// follow a device reset.
//
// Scratch: one FP64 (re, im) partial sum per block of NOALLOC_BLOCK complex
// entries plus a completion counter, NOALLOC_MAX_BLOCKS blocks at most (1 MiB),
// so n may not exceed NOALLOC_MAX_BLOCKS * NOALLOC_BLOCK = 268,435,456.  The
// array lives on every GPU that loads the library until the process exits.
#include <mutex>

#include "reduce.cuh"

namespace hdcr {

constexpr long long NOALLOC_BLOCK = 4096;     // complex entries per thread block
constexpr int NOALLOC_MAX_BLOCKS = 65536;
constexpr int NOALLOC_MAX_DEVICES = 64;

// partial sums (2 per block) followed by the completion counter
static __device__ __align__(256) double g_noalloc_scratch[2 * NOALLOC_MAX_BLOCKS + 32];

template <typename R>
__global__ void __launch_bounds__(RED_THREADS) cdot_noalloc_kernel(const cpx<R>* __restrict__ u,
                                                                   const cpx<R>* __restrict__ v, long long n,
                                                                   RedScratch rs, double* result) {
  double acc[2] = {0.0, 0.0};
  const long long begin = (long long)blockIdx.x * NOALLOC_BLOCK;
  const long long end = begin + NOALLOC_BLOCK < n ? begin + NOALLOC_BLOCK : n;
  for (long long i = begin + threadIdx.x; i < end; i += RED_THREADS) {
    const cpx<R> a = ld(u + i), b = ld(v + i);
    acc[0] += (double)a.re * b.re + (double)a.im * b.im;
    acc[1] += (double)a.re * b.im - (double)a.im * b.re;
  }
  double tot[2];
  if (grid_reduce<2>(acc, rs, tot)) {
    result[0] = tot[0];
    result[1] = tot[1];
  }
}

// device address of the static scratch, looked up once per device
static std::mutex g_noalloc_mutex;
static double* g_noalloc_ptr[NOALLOC_MAX_DEVICES] = {nullptr};

static int noalloc_scratch(RedScratch* rs) {
  int dev = 0;
  HDCR_CUDA_TRY(cudaGetDevice(&dev));
  if (dev < 0 || dev >= NOALLOC_MAX_DEVICES) {
    set_error("hdcr_cdot_noalloc: device %d beyond the %d supported", dev, NOALLOC_MAX_DEVICES);
    return HDCR_ERR_BAD_ARG;
  }
  std::lock_guard<std::mutex> lock(g_noalloc_mutex);
  if (!g_noalloc_ptr[dev]) {
    double* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress((void**)&p, g_noalloc_scratch);
    if (e != cudaSuccess) return cuda_status(e, "cudaGetSymbolAddress(noalloc scratch)");
    g_noalloc_ptr[dev] = p;
  }
  rs->partials = g_noalloc_ptr[dev];
  rs->counter = reinterpret_cast<unsigned int*>(g_noalloc_ptr[dev] + 2 * NOALLOC_MAX_BLOCKS);
  return HDCR_OK;
}

}  // namespace hdcr

using namespace hdcr;

extern "C" int hdcr_cdot_noalloc(const void* u, const void* v, size_t n, int dtype, double* result,
                                 void* stream) {
  if (!u || !v || !result || n == 0) {
    set_error("hdcr_cdot_noalloc: null pointer or n == 0");
    return HDCR_ERR_BAD_ARG;
  }
  if (n > (size_t)NOALLOC_MAX_BLOCKS * (size_t)NOALLOC_BLOCK) {
    set_error("hdcr_cdot_noalloc: n = %zu exceeds the static scratch limit of %lld complex entries", n,
              (long long)NOALLOC_MAX_BLOCKS * NOALLOC_BLOCK);
    return HDCR_ERR_BAD_ARG;
  }
  if (dtype != HDCR_C128 && dtype != HDCR_C64) {
    set_error("hdcr_cdot_noalloc: unknown dtype %d", dtype);
    return HDCR_ERR_BAD_ARG;
  }
  RedScratch rs;
  HDCR_TRY(noalloc_scratch(&rs));
  cudaStream_t st = as_stream(stream);
  // the completion counter must start at zero: clear it on the caller's stream
  HDCR_CUDA_TRY(cudaMemsetAsync(rs.counter, 0, sizeof(unsigned int), st));
  const int blocks = (int)((n + NOALLOC_BLOCK - 1) / NOALLOC_BLOCK);
  if (dtype == HDCR_C128)
    cdot_noalloc_kernel<double><<<blocks, RED_THREADS, 0, st>>>((const cpx<double>*)u, (const cpx<double>*)v,
                                                                 (long long)n, rs, result);
  else
    cdot_noalloc_kernel<float><<<blocks, RED_THREADS, 0, st>>>((const cpx<float>*)u, (const cpx<float>*)v,
                                                                (long long)n, rs, result);
  count_launch();
  HDCR_LAUNCH_CHECK();
  return HDCR_OK;
}
