/*
 * hdcr.h -- C ABI of libhdcr, a GB300 (sm_103a) implementation of the hot path
 * of the hierarchically deflated conjugate residual (HDCR) solver for 5d
 * domain-wall fermions (Yamaguchi & Boyle, arXiv:1611.06944).
 *
 * Conventions for every call
 * --------------------------
 *  - Return value: HDCR_OK (0) or a negative HDCR_ERR_* status.  No C++
 *    exception crosses the ABI.  hdcr_strerror() names a status and
 *    hdcr_last_error() gives the message of the last failing call of the
 *    calling host thread.
 *  - Field pointers are DEVICE pointers owned by the caller (e.g. the data of
 *    a torch tensor) unless a parameter says otherwise.  The library never
 *    frees them.  Handles (hdcr_subspace*, hdcr_coarse*) are owned by the
 *    library: create and destroy them in pairs.
 *  - ``stream`` is a cudaStream_t passed as void* (NULL = legacy default
 *    stream).  Calls are asynchronous on that stream unless stated otherwise;
 *    solves synchronise the stream because they return statistics.
 *  - Calls are made on the CUDA device current on the calling thread.
 *
 * Layouts
 * -------
 *  Complex numbers are interleaved (re, im) pairs of the dtype's real type:
 *  HDCR_C128 = double, HDCR_C64 = float.
 *  4d site index  x4 = ((t*Lz + z)*Ly + y)*Lx + x   (x fastest).
 *  Gauge field    U[mu][x4][a][b], mu = 0..3 <-> x, y, z, t, a 3x3 colour
 *                 matrix U_mu(x)_{ab} per link, row-major; the link leaves x
 *                 in the +mu direction.  4 * V4 * 9 complex.
 *  Fermion field  psi[c][i5]: 12 planes c = 3*spin + colour, each holding
 *                 V5 complex, i5 = x4*Ls + s.  Several fields (nrhs, nvec)
 *                 follow one another, each 12*V5 complex.
 *  Spin basis     chiral: gamma_k = [[0, -i sigma_k], [i sigma_k, 0]] (k = x,y,z),
 *                 gamma_t = [[0, 1], [1, 0]], gamma5 = diag(1, 1, -1, -1).
 *  Coarse field   c[a][k], a = ((tc*Zc + zc)*Yc + yc)*Xc + xc, k < nvec.
 *  Coarse op      A[a][leg][j][k], leg 0 = self, leg 1 + 2*mu (+mu), 2 + 2*mu (-mu).
 */
#ifndef HDCR_H
#define HDCR_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ------------------------------------------------------------- statuses */
#define HDCR_OK 0
#define HDCR_ERR_BAD_ARG (-1)        /* null pointer, bad size or dtype       */
#define HDCR_ERR_BAD_GEOMETRY (-2)   /* lattice, Ls or block not admissible   */
#define HDCR_ERR_NOT_CONVERGED (-3)  /* solve hit its iteration cap           */
#define HDCR_ERR_NONFINITE (-4)      /* NaN/Inf met in a residual or scalar   */
#define HDCR_ERR_RANK_DEFICIENT (-5) /* subspace vectors dependent in a block */
#define HDCR_ERR_CUDA (-6)           /* a CUDA runtime call failed            */
#define HDCR_ERR_TIMEOUT (-7)        /* a bounded device wait gave up         */
#define HDCR_ERR_NO_MEMORY (-8)      /* device or host allocation failed      */

/* --------------------------------------------------------------- dtypes */
#define HDCR_C128 0 /* complex double */
#define HDCR_C64 1  /* complex float  */

typedef struct {
  int L[4]; /* Lx, Ly, Lz, Lt (4d extents, each >= 1)                     */
  int Ls;   /* extent of the fifth dimension (>= 2)                        */
  int bc_t; /* +1 periodic or -1 antiperiodic time boundary for fermions   */
} hdcr_geom;

typedef struct {
  double M5; /* domain-wall height; the 4d Wilson mass is -M5              */
  double mf; /* quark mass coupling the two walls                          */
} hdcr_dwf_params;

/* Statistics returned by the solves. */
typedef struct {
  int status;           /* HDCR_OK or the error the solve ended with            */
  int iters;            /* outer iterations (CR: iterations)                    */
  int fine_matvecs;     /* applications of H at the solve's outer precision      */
  int fine_matvecs_lo;  /* applications of H at the inner precision (mixed)     */
  int coarse_matvecs;   /* applications of the coarse operator                   */
  int restarts;         /* FGCR restarts / defect-correction cycles              */
  double true_resid;    /* |b - H x| / |b| recomputed in FP64 at the end         */
  double t_total;       /* wall seconds of the solve (host clock, stream synced) */
  double t_smoother;    /* seconds in the fine smoother (event timed)            */
  double t_coarse;      /* seconds in restrict + coarse solve + prolong          */
} hdcr_solve_stats;

const char* hdcr_strerror(int status);
const char* hdcr_last_error(void);
int hdcr_version(void); /* 10000*major + 100*minor + patch */

/* ---------------------------------------------------------------- fine operator
 * hdcr_apply_g5dwf: out = H in with H = Gamma5 D_dwf = gamma5 R5 D_dwf
 * (arXiv:1611.06944 Section 3), D_dwf the Shamir domain-wall operator
 *   (D_dwf psi)(x,s) = (5 - M5) psi(x,s)
 *        - 1/2 sum_mu [(1 - gamma_mu) U_mu(x) psi(x+mu,s) + (1 + gamma_mu) U_mu(x-mu)^dag psi(x-mu,s)]
 *        - P_- psi(x,s+1) - P_+ psi(x,s-1),
 * walls psi(x,Ls) = -mf psi(x,0), psi(x,-1) = -mf psi(x,Ls-1), P_pm = (1 pm gamma5)/2,
 * R5 psi(s) = psi(Ls-1-s).  U and the nrhs fields in/out share ``dtype``.
 * ``in`` and ``out`` must not overlap.  Errors: BAD_ARG, BAD_GEOMETRY, CUDA.
 */
int hdcr_apply_g5dwf(const hdcr_geom* g, const hdcr_dwf_params* p, const void* U,
                     const void* in, void* out, int dtype, int nrhs, void* stream);

/* out = Gamma5 in = gamma5 R5 in (Section 3), nfields fields; in == out not allowed. */
int hdcr_apply_gamma5_r5(const hdcr_geom* g, const void* in, void* out, int dtype,
                         int nfields, void* stream);

/* Layout conversion between the natural array layout psi[x4][s][spin][colour]
 * (complex, as a (Lt,Lz,Ly,Lx,Ls,4,3) tensor) and the plane layout above. */
int hdcr_fermion_to_planes(const hdcr_geom* g, const void* natural, void* planes,
                           int dtype, int nfields, void* stream);
int hdcr_fermion_from_planes(const hdcr_geom* g, const void* planes, void* natural,
                             int dtype, int nfields, void* stream);

/* Precision conversion of n complex numbers (device to device). */
int hdcr_convert(const void* in, int in_dtype, void* out, int out_dtype, size_t n,
                 void* stream);

/* ---------------------------------------------------------------- reductions
 * Inner products used by the Krylov solvers (Section 3), accumulated in FP64
 * with a fixed, deterministic reduction order for a given n.
 * result (DEVICE pointer, 2 doubles): sum_i conj(u_i) v_i as (re, im).
 * hdcr_norm2 writes 1 double: sum_i |u_i|^2.  n = number of complex entries.
 * They use a library-owned scratch area of the current device: calls that
 * overlap on the GPU (different streams) race on it.
 */
int hdcr_cdot(const void* u, const void* v, size_t n, int dtype, double* result,
              void* stream);
int hdcr_norm2(const void* u, size_t n, int dtype, double* result, void* stream);

/* ---------------------------------------------------------------- CR solve
 * Conjugate residual (Section 3) on H x = b, unpreconditioned, all in ``dtype``
 * (inner products in FP64).  x holds the initial guess on entry.  Stops when the
 * recursively updated residual satisfies |r| <= tol |b| and then recomputes the
 * true residual in FP64 into stats->true_resid.  max_iter caps the iterations
 * (NOT_CONVERGED when reached).  Synchronises ``stream``.  Workspace (5 fields)
 * is allocated and freed by the call.
 */
int hdcr_cr_solve(const hdcr_geom* g, const hdcr_dwf_params* p, const void* U,
                  const void* b, void* x, int dtype, double tol, int max_iter,
                  hdcr_solve_stats* stats, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* HDCR_H */
