// Moebius domain wall with c5 = 0 (Section 3: the Shamir operator of this library is
// the Moebius/Cayley form with c = 0, b = 1).  With b5 != 1 the 4d part is scaled,
//     D = b5 D_W + D_5,   (D psi)(s) = (b5 D_W + 1) psi(s) - P_- psi(s+1) - P_+ psi(s-1).
// b5 D_W = b5 (4 - M5) - (b5 / 2) sum_mu [hops with U], and the hops are linear in
// the links, so D is the Shamir operator of links b5 U and wall height
//     M5' = 4 - b5 (4 - M5)        (diagonal 5 - M5' = b5 (4 - M5) + 1).
// The conversion below scales the links on the device and returns M5'; every
// kernel of the library then applies to the Moebius operator unchanged.
#include "hdcr_internal.cuh"

namespace hdcr {

template <typename R>
__global__ void scale_links_kernel(const cpx<R>* __restrict__ in, cpx<R>* __restrict__ out, long long n, R b5) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const cpx<R> v = ld(in + i);
    st(out + i, cpx<R>(b5 * v.re, b5 * v.im));
  }
}

}  // namespace hdcr

using namespace hdcr;

extern "C" int hdcr_mobius_to_shamir(const hdcr_dwf_params* mobius, double b5, const void* U, void* U_out,
                                     int dtype, size_t n, hdcr_dwf_params* shamir, void* stream) {
  if (!mobius || !U || !U_out || !shamir || n == 0 || !(b5 > 0.0)) {
    set_error("hdcr_mobius_to_shamir: null pointer, n == 0 or b5 <= 0");
    return HDCR_ERR_BAD_ARG;
  }
  if (dtype != HDCR_C128 && dtype != HDCR_C64) {
    set_error("hdcr_mobius_to_shamir: dtype %d is not C128 or C64", dtype);
    return HDCR_ERR_BAD_ARG;
  }
  cudaStream_t st = as_stream(stream);
  const int blocks = num_blocks((long long)n, 256, 4096);
  if (dtype == HDCR_C128)
    scale_links_kernel<double><<<blocks, 256, 0, st>>>((const cpx<double>*)U, (cpx<double>*)U_out, (long long)n, b5);
  else
    scale_links_kernel<float><<<blocks, 256, 0, st>>>((const cpx<float>*)U, (cpx<float>*)U_out, (long long)n,
                                                      (float)b5);
  count_launch();
  HDCR_LAUNCH_CHECK();
  shamir->M5 = 4.0 - b5 * (4.0 - mobius->M5);
  shamir->mf = mobius->mf;
  return HDCR_OK;
}
