// Host buffers at the C ABI: the entry points that take fields or links
// (hdcr_build_subspace, hdcr_build_coarse_op, hdcr_solve, hdcr_apply_gamma5_r5,
// hdcr_gauge_force, hdcr_gauge_grad) accept host pointers as well as device
// pointers.  A host argument (pinned or pageable, as reported by
// cudaPointerGetAttributes) is staged through a stream-ordered device buffer:
// inputs are copied in on the call's stream before the work, outputs copied back
// after it, and the buffer is freed on the stream.  Pinned buffers make the
// copies asynchronous; the caller synchronises the stream before reading a host
// output of an asynchronous call.
#pragma once

#include "hdcr_internal.cuh"

namespace hdcr {

inline bool is_host_pointer(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return true;  // not known to CUDA: ordinary host memory
  }
  return a.type == cudaMemoryTypeHost || a.type == cudaMemoryTypeUnregistered;
}

class Staged {
 public:
  Staged() = default;
  Staged(const Staged&) = delete;
  Staged& operator=(const Staged&) = delete;
  ~Staged() {
    if (dev_) cudaFreeAsync(dev_, st_);
  }
  // an input of ``bytes`` bytes: the device pointer to use is ptr()
  int in(const void* p, size_t bytes, cudaStream_t st) { return setup(const_cast<void*>(p), bytes, st, true); }
  // an output (copied back by finish()); ``copy_in`` also stages its initial contents
  int out(void* p, size_t bytes, cudaStream_t st, bool copy_in) { return setup(p, bytes, st, copy_in); }
  void* ptr() const { return dev_ ? dev_ : user_; }
  // copies an output back to the host buffer (no-op for device pointers)
  int finish() {
    if (!dev_) return HDCR_OK;
    HDCR_CUDA_TRY(cudaMemcpyAsync(user_, dev_, bytes_, cudaMemcpyDeviceToHost, st_));
    return HDCR_OK;
  }

 private:
  int setup(void* p, size_t bytes, cudaStream_t st, bool copy_in) {
    user_ = p;
    bytes_ = bytes;
    st_ = st;
    if (!p || !is_host_pointer(p)) return HDCR_OK;
    HDCR_CUDA_TRY(cudaMallocAsync(&dev_, bytes, st));
    if (copy_in) HDCR_CUDA_TRY(cudaMemcpyAsync(dev_, p, bytes, cudaMemcpyHostToDevice, st));
    return HDCR_OK;
  }
  void* user_ = nullptr;
  void* dev_ = nullptr;
  size_t bytes_ = 0;
  cudaStream_t st_ = nullptr;
};

}  // namespace hdcr
