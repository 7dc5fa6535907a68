// Block geometry, subspace and coarse-operator handles (Section 4).
//
// A block is b = (bx, by, bz, bt) 4d sites times the whole fifth dimension.
// Coarse site a = ((tc*Zc + zc)*Yc + yc)*Xc + xc; inside block a the local
// 5d site l runs with s fastest, then x, y, z, t (so a block row of bx*Ls
// fine sites is contiguous in every plane).
#pragma once

#include <mutex>

#include "krylov.cuh"

namespace hdcr {

constexpr int NLEGS = 9;  // self + 8 nearest coarse neighbours

struct BlockGeom {
  int b[4];
  int Lc[4];
  int Vc;
  int bvol;
  long long K5;  // fine 5d sites per block
};

int make_block_geom(const Geom& g, const int block[4], BlockGeom* out);

__host__ __device__ inline void coarse_coords(const BlockGeom& bg, int a, int c[4]) {
  c[0] = a % bg.Lc[0];
  int r = a / bg.Lc[0];
  c[1] = r % bg.Lc[1];
  r /= bg.Lc[1];
  c[2] = r % bg.Lc[2];
  c[3] = r / bg.Lc[2];
}

// fine 5d index of local site l of block a
__host__ __device__ inline long long block_site(const Geom& g, const BlockGeom& bg, int a, long long l) {
  const int s = (int)(l % g.Ls);
  long long r = l / g.Ls;
  int ac[4];
  coarse_coords(bg, a, ac);
  int c[4];
  c[0] = ac[0] * bg.b[0] + (int)(r % bg.b[0]);
  r /= bg.b[0];
  c[1] = ac[1] * bg.b[1] + (int)(r % bg.b[1]);
  r /= bg.b[1];
  c[2] = ac[2] * bg.b[2] + (int)(r % bg.b[2]);
  c[3] = ac[3] * bg.b[3] + (int)(r / bg.b[2]);
  return (long long)x4_index(g, c) * g.Ls + s;
}

// leg index of the hop to coarse neighbour a + sign*mu
__host__ __device__ inline int leg_of(int mu, int sign) { return 1 + 2 * mu + (sign > 0 ? 0 : 1); }

}  // namespace hdcr

// Opaque handles of the C ABI.
struct hdcr_subspace {
  hdcr::Geom g;
  hdcr::BlockGeom bg;
  int nvec;
  int dtype;      // storage of the basis vectors (HDCR_C128 / HDCR_C64)
  void* vecs;     // nvec fields, plane layout, block-orthonormal
  int device;
  // scratch of hdcr_build_coarse_op, kept for the next build from this basis (a
  // rebuild after a gauge update needs no allocation); builds from one subspace
  // are serialised on build_mu
  mutable std::mutex build_mu;
  mutable void* build_ws = nullptr;
  mutable size_t build_ws_bytes = 0;
};

namespace hdcr {
struct Level2;
struct CFCoef;
void cf_coef_free(CFCoef* cf);
}

struct hdcr_coarse {
  const hdcr_subspace* sub;  // borrowed: must outlive the coarse handle
  hdcr::Geom g;
  hdcr::BlockGeom bg;
  int nvec;
  int dtype;    // of A
  void* A;      // [Vc][9][nvec][nvec]
  int* nbr;     // [Vc][9] coarse site reached by each leg
  void* Ainv;   // dense inverse (FP32 complex, n = Vc*nvec, n x n) then its column gather index (n ints)
  void* dws;    // workspace of the multi-right-hand-side dense solve (grown on demand)
  size_t dws_bytes;
  hdcr::Level2* l2;  // third level of the coarse solve (hdcr_coarse_build_level2), or null
  hdcr::CFCoef* cf;  // set: built on the continued-fraction operator (hdcr_cf_build_coarse_op)
  double M5, mf;
  int device;
};

namespace hdcr {

// restrict / prolong with vector precision R and basis precision R (same dtype)
template <typename R>
int launch_restrict(const hdcr_subspace* sub, const cpx<R>* fine, cpx<R>* coarse, int nrhs, cudaStream_t st);
// fine = (add ? fine_in : 0) + P coarse
template <typename R>
int launch_prolong(const hdcr_subspace* sub, const cpx<R>* coarse, const cpx<R>* fine_in, cpx<R>* fine,
                   int nrhs, cudaStream_t st);
template <typename R>
int launch_coarse_apply(const hdcr_coarse* co, const cpx<R>* in, cpx<R>* out, int nrhs, cudaStream_t st);
// nbr[a][leg]: the coarse site each leg of site a reaches (device array of Vc * 9 ints)
int fill_neighbour_table(const BlockGeom& bg, int* nbr, cudaStream_t st);

template <typename R>
struct CoarseOp {
  const hdcr_coarse* co;
  long long n() const { return (long long)co->bg.Vc * co->nvec; }
  int apply(const cpx<R>* in, cpx<R>* out, cudaStream_t st) const {
    return launch_coarse_apply<R>(co, in, out, 1, st);
  }
  int apply_dot(const cpx<R>* in, cpx<R>* out, RedScratch rs, double* res, cudaStream_t st) const;
};

int coarse_check(const hdcr_coarse* co);
int coarse_invert(hdcr_coarse* co, cudaStream_t st);
// makes the dense solve of nrhs right-hand sides ready to run without allocating
// (workspace and cuBLAS handle); call outside a stream capture
int dense_solve_prepare(hdcr_coarse* co, int nrhs);
template <typename R>
int launch_dense_solve(const hdcr_coarse* co, const cpx<R>* in, cpx<R>* out, int nrhs, cudaStream_t st);
void solve_cache_release(const hdcr_coarse* co);  // frees the cached solve workspace
void multi_cache_release(const hdcr_coarse* co);  // frees the multi-RHS solve workspace and graph
int subspace_check(const hdcr_subspace* sub);

}  // namespace hdcr
