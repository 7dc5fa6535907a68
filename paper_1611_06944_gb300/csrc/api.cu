// Runtime pieces of the C ABI: status strings, per-thread error messages and
// geometry validation.
#include <stdarg.h>
#include <string.h>

#include <atomic>

#include "hdcr_internal.cuh"

namespace hdcr {

static thread_local char g_last_error[512] = "";
static std::atomic<unsigned long long> g_launches{0};

void count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }
void count_launches(unsigned long long n) { g_launches.fetch_add(n, std::memory_order_relaxed); }
void uncount_launches(unsigned long long n) { g_launches.fetch_sub(n, std::memory_order_relaxed); }
unsigned long long launches_so_far() { return g_launches.load(std::memory_order_relaxed); }

void set_error(const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_last_error, sizeof(g_last_error), fmt, ap);
  va_end(ap);
}

int cuda_status(cudaError_t e, const char* what) {
  set_error("%s: %s (%s)", what, cudaGetErrorString(e), cudaGetErrorName(e));
  return e == cudaErrorMemoryAllocation ? HDCR_ERR_NO_MEMORY : HDCR_ERR_CUDA;
}

int make_geom(const hdcr_geom* gp, Geom* g) {
  if (!gp) {
    set_error("geometry pointer is NULL");
    return HDCR_ERR_BAD_ARG;
  }
  long long v4 = 1;
  for (int mu = 0; mu < 4; ++mu) {
    if (gp->L[mu] < 1) {
      set_error("lattice extent L[%d] = %d must be >= 1", mu, gp->L[mu]);
      return HDCR_ERR_BAD_GEOMETRY;
    }
    g->L[mu] = gp->L[mu];
    v4 *= gp->L[mu];
  }
  if (gp->Ls < 2) {
    set_error("Ls = %d must be >= 2", gp->Ls);
    return HDCR_ERR_BAD_GEOMETRY;
  }
  if (gp->bc_t != 1 && gp->bc_t != -1) {
    set_error("bc_t = %d must be +1 or -1", gp->bc_t);
    return HDCR_ERR_BAD_GEOMETRY;
  }
  if (v4 * gp->Ls * 12 >= (1LL << 31)) {
    set_error("lattice too large: a field must hold fewer than 2^31 complex numbers");
    return HDCR_ERR_BAD_GEOMETRY;
  }
  g->Ls = gp->Ls;
  g->bc_t = gp->bc_t;
  g->V4 = (int)v4;
  g->V5 = v4 * gp->Ls;
  return HDCR_OK;
}

size_t dtype_complex_bytes(int dtype) {
  if (dtype == HDCR_C128) return 16;
  if (dtype == HDCR_C64) return 8;
  return 0;
}

}  // namespace hdcr

extern "C" const char* hdcr_strerror(int status) {
  switch (status) {
    case HDCR_OK: return "ok";
    case HDCR_ERR_BAD_ARG: return "bad argument";
    case HDCR_ERR_BAD_GEOMETRY: return "bad geometry";
    case HDCR_ERR_NOT_CONVERGED: return "not converged";
    case HDCR_ERR_NONFINITE: return "non-finite value";
    case HDCR_ERR_RANK_DEFICIENT: return "rank-deficient subspace";
    case HDCR_ERR_CUDA: return "CUDA error";
    case HDCR_ERR_TIMEOUT: return "device wait timed out";
    case HDCR_ERR_NO_MEMORY: return "out of memory";
    default: return "unknown status";
  }
}

extern "C" const char* hdcr_last_error(void) { return hdcr::g_last_error; }

extern "C" int hdcr_version(void) { return 100; }

extern "C" unsigned long long hdcr_launch_count(void) { return hdcr::g_launches.load(std::memory_order_relaxed); }
