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
 *    frees them.  hdcr_build_subspace, hdcr_build_coarse_op, hdcr_solve,
 *    hdcr_apply_gamma5_r5, hdcr_gauge_force and hdcr_gauge_grad also accept
 *    HOST pointers for their links and fields (pinned or pageable, told apart
 *    by cudaPointerGetAttributes): the call stages each host argument through
 *    a stream-ordered device buffer, copying inputs in before the work and
 *    outputs back after it on ``stream``; with pinned memory the copies are
 *    asynchronous, so synchronise the stream before reading a host output of
 *    an asynchronous call (hdcr_solve synchronises itself).  Handles (hdcr_subspace*, hdcr_coarse*) are owned by the
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
 *  Fermion field  psi[x4][c][s]: for each 4d site the 12 components
 *                 c = 3*spin + colour, each a run of Ls complex numbers over
 *                 the fifth coordinate s (element offset (x4*12 + c)*Ls + s).
 *                 The 5d site index is i5 = x4*Ls + s.  Several fields
 *                 (nrhs, nvec) follow one another, each 12*V5 complex.
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
/* hdcr_build_coarse_op only: complex float storage, projections with one pass of
 * TF32 tensor-core products (FP32 accumulation), relative error about 1e-3 */
#define HDCR_C64_FAST 2
/* hdcr_build_coarse_op only: complex double storage, built as C64 with the
 * three-pass (FP32-exact) tensor-core products from the FP32-rounded basis and
 * links, relative error about 1e-7.  For solves whose coarse correction is the
 * FP32 dense inverse, which rounds A to FP32 anyway. */
#define HDCR_C128_TC 4
/* FP16 storage of a fermion field (the precision form's half-precision
 * storage; arithmetic stays FP32): 12*V5 half2 (FP16 re, im) in the field
 * layout below, followed by V5 FP32 scales, one per 5d site (x4, s) at index
 * x4*Ls + s; a component is its half2 times its site's scale, chosen by the
 * encoder as the largest |re|, |im| of the site's 24 reals (so halves lie in
 * [-1, 1], rounded to 2^-11 of that value).  52*V5 bytes a field; nfields
 * fields follow one another.  Used by hdcr_apply_g5dwf (with C64 links) and the
 * two conversions below. */
#define HDCR_H16 3

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
/* Number of CUDA kernels the library has launched in this process (all
 * devices, all threads); a diagnostic for counting launches per step. */
unsigned long long hdcr_launch_count(void);
/* Stencil timer: hdcr_stencil_timer(1) resets and starts recording CUDA
 * events around every application of H (on the launching stream, at most
 * 16384 launches); hdcr_stencil_timer(0) stops.  hdcr_stencil_timer_read adds
 * up the recorded launches of one precision (HDCR_C128, HDCR_C64 or HDCR_H16;
 * HDCR_TIMER_C128_CHEB: the FP64 applications that carry a fused Chebyshev
 * smoother step, which HDCR_C128 leaves out): total device milliseconds, number
 * of launches and 5d sites processed.  It waits for the recorded events. */
#define HDCR_TIMER_C128_CHEB 100
int hdcr_stencil_timer(int enable);
int hdcr_stencil_timer_read(int dtype, double* total_ms, long long* launches, long long* sites);
/* Every application of H of one precision since the timer was started,
 * including those beyond the 16384 that carry events: launches and 5d sites. */
int hdcr_stencil_timer_count(int dtype, long long* launches, long long* sites);
/* Measured FMA rate of the current device (a property of the machine, used as
 * the roofline denominator of the arithmetic-bound FP64 operator; not a step of
 * the method): every SM runs long chains of independent fused multiply-adds of
 * one precision (HDCR_C128: FP64, HDCR_C64: FP32), five launches are timed with
 * CUDA events on ``stream`` and *tflops receives 2 x FMAs / second / 1e12.
 * Synchronises ``stream``.  Errors: BAD_ARG, CUDA. */
int hdcr_probe_fma_rate(int dtype, double* tflops, void* stream);
/* The coarse level's complex FP32 GEMMs (the rank-128 updates of the dense coarse
 * inverse, its application to several right-hand sides) run on the tensor cores
 * through cuBLAS's FP32 emulation on BF16 (three BF16 parts per operand, FP32
 * accumulation).  Diagnostic: how many such GEMMs the process issued, and how many
 * of them cuBLAS declined on that path and ran in plain FP32 instead. */
int hdcr_tc_gemm_info(unsigned long long* calls, unsigned long long* fallbacks);

/* ---------------------------------------------------------------- fine operator
 * hdcr_apply_g5dwf: out = H in with H = Gamma5 D_dwf = gamma5 R5 D_dwf
 * (arXiv:1611.06944 Section 3), D_dwf the Shamir domain-wall operator
 *   (D_dwf psi)(x,s) = (5 - M5) psi(x,s)
 *        - 1/2 sum_mu [(1 - gamma_mu) U_mu(x) psi(x+mu,s) + (1 + gamma_mu) U_mu(x-mu)^dag psi(x-mu,s)]
 *        - P_- psi(x,s+1) - P_+ psi(x,s-1),
 * walls psi(x,Ls) = -mf psi(x,0), psi(x,-1) = -mf psi(x,Ls-1), P_pm = (1 pm gamma5)/2,
 * R5 psi(s) = psi(Ls-1-s).  U and the nrhs fields in/out share ``dtype``, except
 * for HDCR_H16: fields in FP16 storage (even Ls <= 16, 16-byte aligned), U C64,
 * arithmetic FP32, each output site re-encoded with its own scale.
 * ``in`` and ``out`` must not overlap.  Errors: BAD_ARG, BAD_GEOMETRY, CUDA.
 */
int hdcr_apply_g5dwf(const hdcr_geom* g, const hdcr_dwf_params* p, const void* U,
                     const void* in, void* out, int dtype, int nrhs, void* stream);

/* Tile-shape autotuner of the FP32 operator (a property of this library, not a
 * step of the method).  The FP32 kernel runs one CTA per tile of 4d sites;
 * several tile shapes are compiled in.  With the tuner on (mode 1, the
 * default) the first plain FP32 application of H (hdcr_apply_g5dwf, or the
 * solvers' own calls) for a given (device, lattice, Ls, nrhs), outside a
 * stream capture, runs and event-times every tile shape that divides the
 * lattice on the call's own fields and stream (synchronising it once), and
 * keeps the fastest for every later FP32 call with that key.  Results do not
 * depend on the tile.  mode 0 keeps the default linear tile of 16 consecutive
 * 4d sites, mode 2 forgets every tuned choice.  force_variant >= 0 runs that
 * variant wherever it fits (diagnostics), -1 restores tuning.
 * hdcr_stencil_tune_info: the variant chosen for (g, nrhs) or -1 if none yet,
 * and the measured microseconds per launch of the first ``nus`` variants
 * (-1 where a variant does not fit).  Errors: BAD_ARG. */
int hdcr_stencil_tune(int mode, int force_variant);
int hdcr_stencil_tune_info(const hdcr_geom* g, int nrhs, int* variant, float* us, int nus);

/* FP16-storage conversions (HDCR_H16 above) of nfields fields between C128 or C64
 * (``dtype``) and the FP16 form; buffers 16-byte aligned, distinct.  Errors: BAD_ARG. */
int hdcr_fermion_encode_h16(const hdcr_geom* g, const void* in, int in_dtype, void* out, int nfields,
                            void* stream);
int hdcr_fermion_decode_h16(const hdcr_geom* g, const void* in, void* out, int out_dtype, int nfields,
                            void* stream);

/* hdcr_mobius_to_shamir: the Moebius domain-wall operator with c5 = 0 and scale b5
 * (Section 3: the Shamir operator above is the Moebius/Cayley form with c = 0,
 * b = 1), D = b5 D_W + D_5, i.e. (D psi)(s) = (b5 D_W + 1) psi(s) - P_- psi(s+1)
 * - P_+ psi(s-1), equals the Shamir operator of this library with links b5 U and
 * wall height M5' = 4 - b5 (4 - M5) (D_W's hops are linear in the links).  This
 * call writes U_out = b5 U (n complex numbers, 4*V4*9 for a gauge field, device
 * memory, dtype C128 or C64; U_out may equal U) and *shamir = {M5', mf}; with them
 * every other call of the library (operator, solves, subspace, coarse operator)
 * applies to the Moebius operator.  The gauge force of a solve computed with the
 * scaled links is the gradient with respect to U_out; with respect to U it is b5
 * times that.  b5 > 0.  Errors: BAD_ARG. */
int hdcr_mobius_to_shamir(const hdcr_dwf_params* mobius, double b5, const void* U, void* U_out,
                          int dtype, size_t n, hdcr_dwf_params* shamir, void* stream);

/* out = Gamma5 in = gamma5 R5 in (Section 3), nfields fields; in == out not allowed. */
int hdcr_apply_gamma5_r5(const hdcr_geom* g, const void* in, void* out, int dtype,
                         int nfields, void* stream);

/* Layout conversion between the natural array layout psi[x4][s][spin][colour]
 * (complex, a (Lt,Lz,Ly,Lx,Ls,4,3) tensor) and the library layout above. */
int hdcr_fermion_pack(const hdcr_geom* g, const void* natural, void* packed, int dtype,
                      int nfields, void* stream);
int hdcr_fermion_unpack(const hdcr_geom* g, const void* packed, void* natural, int dtype,
                        int nfields, void* stream);

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

/* hdcr_cdot_noalloc: the same inner product as hdcr_cdot, for callers that may
 * not let the library allocate device memory -- for example a caller that hands
 * all device memory to its own pool at start-up and keeps a fixed budget, or a
 * runtime that forbids allocations after start-up.  The paper has no
 * counterpart: this is an interface of the library, not a step of the method.
 * Its scratch (one FP64 partial sum per 4096 entries and a completion counter,
 * 1 MiB) is a fixed array compiled into the library, held on every GPU that
 * loads the library until the process exits; the call allocates nothing and
 * only launches kernels and clears the counter on ``stream``.  n may not exceed
 * HDCR_NOALLOC_MAX_N (BAD_ARG otherwise).  The first call on a device looks up
 * the array's device address with that device current and keeps it for the
 * life of the process; make no call after a device reset (the kept address
 * would be stale).  All
 * calls share the one array: calls that overlap on the GPU (different streams)
 * race and give wrong results.  result: DEVICE pointer to 2 doubles. */
#define HDCR_NOALLOC_MAX_N 268435456
int hdcr_cdot_noalloc(const void* u, const void* v, size_t n, int dtype, double* result,
                      void* stream);

/* ---------------------------------------------------------------- CR solve
 * Conjugate residual (Section 3) on H x = b, unpreconditioned, all in ``dtype``
 * (inner products in FP64).  x holds the initial guess on entry.  Stops when the
 * recursively updated residual satisfies |r| <= tol |b| and then recomputes the
 * true residual |b - H x| / |b| (FP64 accumulation) into stats->true_resid.
 * max_iter caps the iterations (NOT_CONVERGED when reached; x then holds the
 * last iterate).  Synchronises ``stream``.  Workspace (4 fields) is allocated
 * and freed by the call.
 */
int hdcr_cr_solve(const hdcr_geom* g, const hdcr_dwf_params* p, const void* U,
                  const void* b, void* x, int dtype, double tol, int max_iter,
                  hdcr_solve_stats* stats, void* stream);

/* ---------------------------------------------------------------- red-black CGNE
 * hdcr_cgne_rb_solve: H x = b by the comparison solver of Section 5 (Table 1's
 * red-black preconditioned CGNE): with the 4d sites coloured by parity (x+y+z+t) mod 2 and
 * D_dwf = M5 + D_hop (M5 the site-local part, D_hop the 4d hops, which join
 * opposite parities), D x = Gamma5 b is reduced to the odd sites,
 *   S x_o = eta_o - D_oe M5^{-1} eta_e,   S = M5 - D_oe M5^{-1} D_eo,  eta = Gamma5 b,
 * solved by conjugate gradient on S^dag S (S^dag = Gamma5 S Gamma5), and
 * x_e = M5^{-1} (eta_e - D_eo x_o).  FP64 throughout; U, b, x are C128; x is
 * output (zero initial guess).  Every extent L[mu] must be even.  Stops when the
 * Schur residual |eta~_o - S x_o| (the full residual) <= tol |b|, then recomputes
 * |b - H x| / |b| into stats->true_resid.  stats->fine_matvecs counts
 * whole-lattice applications of the hopping term (2 per iteration + 2).
 * Synchronises ``stream``; workspace (11 fields) is allocated and freed by the
 * call.  Errors: BAD_ARG, BAD_GEOMETRY (an odd extent), NOT_CONVERGED, NONFINITE,
 * CUDA, NO_MEMORY. */
int hdcr_cgne_rb_solve(const hdcr_geom* g, const hdcr_dwf_params* p, const void* U, const void* b,
                       void* x, double tol, int max_iter, hdcr_solve_stats* stats, void* stream);

/* ---------------------------------------------------------------- subspace
 * hdcr_build_subspace: the near-null-space basis of Section 4.
 *   1. each of the nvec/2 Gaussian noise fields (``noise``: nvec/2 C128
 *      fields, drawn by the caller) is filtered towards the low modes of H and
 *      normalised, by one of the paper's approaches (Section 4):
 *        HDCR_SUBSPACE_CR_SMOOTH  ``order`` conjugate-residual steps on H x = 0
 *                                 from the noise ("inverse iteration applied to
 *                                 Gaussian noise");
 *        HDCR_SUBSPACE_CHEBYSHEV  the Chebyshev low-pass filter of Fig. 1,
 *                                 T_order(t(H^2)) x with t mapping
 *                                 [lam_cut^2, lam_max^2] onto [-1, 1];
 *      in ``filter_dtype`` precision;
 *   2. chiral split with Gamma5 = gamma5 R5: v -> (1 + Gamma5) v / 2 and
 *      (1 - Gamma5) v / 2 (the nvec/2 "+" vectors first, then the "-" ones);
 *   3. restriction to blocks of block[0..3] sites times the full fifth
 *      dimension (Eq. 4.1);
 *   4. modified Gram-Schmidt, applied twice, in each block in the order
 *      k = 0..nvec-1 (FP64), so that P_S of Eq. 4.3 is a projector.
 * The basis is stored in ``store_dtype``.  U is C128.  Every L[mu] must be a
 * multiple of block[mu] with L[mu]/block[mu] >= 2; nvec even, 2..256.
 * Errors: BAD_ARG, BAD_GEOMETRY, RANK_DEFICIENT (a vector has nothing left
 * after orthogonalisation: |v| < 1e-12 |v0|), CUDA, NO_MEMORY.
 * Synchronises ``stream``.  On success *out receives a new handle.
 */
#define HDCR_SUBSPACE_CR_SMOOTH 0
#define HDCR_SUBSPACE_CHEBYSHEV 1

typedef struct {
  int nvec;           /* basis size after the chiral split (even)            */
  int block[4];       /* block extents bx, by, bz, bt                        */
  int kind;           /* HDCR_SUBSPACE_CR_SMOOTH or HDCR_SUBSPACE_CHEBYSHEV  */
  int order;          /* CR steps, or Chebyshev polynomial order (>= 1)      */
  double lam_cut;     /* Chebyshev filter: |lambda| below which modes grow   */
  double lam_max;     /* Chebyshev filter: upper edge of the spectrum of |H| */
  int filter_dtype;   /* precision of step 1: HDCR_C128 or HDCR_C64          */
  int store_dtype;    /* storage of the basis: HDCR_C128 or HDCR_C64         */
} hdcr_subspace_params;

typedef struct hdcr_subspace hdcr_subspace;
int hdcr_build_subspace(const hdcr_geom* g, const hdcr_dwf_params* p, const void* U,
                        const void* noise, const hdcr_subspace_params* sp, void* stream,
                        hdcr_subspace** out);
/* A subspace from nvec given fields (C128, already split): steps 3-4 only. */
int hdcr_subspace_from_vectors(const hdcr_geom* g, const int block[4], int nvec,
                               const void* vectors, int store_dtype, void* stream,
                               hdcr_subspace** out);
int hdcr_subspace_info(const hdcr_subspace* sub, int* nvec, int coarse_L[4], int* dtype);
/* Copies the nvec block-orthonormal basis fields (C128) into ``out`` (device). */
int hdcr_subspace_get_vectors(const hdcr_subspace* sub, void* out, void* stream);
void hdcr_subspace_destroy(hdcr_subspace* sub);

/* P^dag and P of Eq. 4.3: coarse[r][a][k] = <phi_k^a, fine_r> and
 * fine_r = sum_{a,k} coarse[r][a][k] phi_k^a, for nrhs fields.  ``dtype`` must
 * equal the basis storage dtype. */
int hdcr_restrict(const hdcr_subspace* sub, const void* fine, void* coarse, int dtype, int nrhs,
                  void* stream);
int hdcr_prolong(const hdcr_subspace* sub, const void* coarse, void* fine, int dtype, int nrhs,
                 void* stream);

/* ---------------------------------------------------------------- coarse operator
 * hdcr_build_coarse_op: little Dirac operator A^{ab}_{jk} = <phi_j^a | H | phi_k^b>
 * (Eq. 4.5), nonzero only for b = a and the 8 nearest coarse neighbours (the
 * sparsity noted after Eq. 4.6), stored as A[a][leg][j][k] in ``op_dtype``
 * (HDCR_C64_FAST: stored as C64, built with single-pass TF32 products, for the
 * mixed-precision solve whose FP64 outer iteration recovers the accuracy;
 * HDCR_C128_TC: stored as C128, built by the FP32-exact tensor-core path).  Leg
 * (mu, +-) collects the fine hops from block a into block a +- mu; on a coarse
 * extent of 2 the two legs of mu reach the same coarse site and both apply.  U
 * is C128 (converted internally when op_dtype is C64).  The subspace handle is
 * borrowed and must outlive the coarse handle.  Synchronises ``stream``.
 * Errors: BAD_ARG (nvec > 64), CUDA, NO_MEMORY.
 */
typedef struct hdcr_coarse hdcr_coarse;
int hdcr_build_coarse_op(const hdcr_subspace* sub, const hdcr_dwf_params* p, const void* U,
                         int op_dtype, void* stream, hdcr_coarse** out);
/* Copies A (C128, [Vc][9][nvec][nvec]) into ``out`` (device). */
int hdcr_coarse_get_op(const hdcr_coarse* co, void* out, void* stream);
/* out[r][a] = sum_leg A[a][leg] in[r][a + leg], 9-point coarse stencil; dtype = op dtype. */
int hdcr_apply_coarse(const hdcr_coarse* co, const void* in, void* out, int dtype, int nrhs,
                      void* stream);
/* Dense inverse of the coarse operator (the whole (Vc*nvec)^2 matrix, FP32
 * complex, Gauss-Jordan elimination with partial pivoting), kept in the handle
 * and used by hdcr_solve's HDCR_COARSE_DENSE solver.  Q = P A^{-1} P^dag of
 * Eq. 4.6 applied exactly up to FP32 rounding.  Memory: 8 (Vc*nvec)^2 bytes.
 * Synchronises ``stream``.  Errors: BAD_ARG (Vc*nvec > 32768), NONFINITE
 * (singular pivot), CUDA, NO_MEMORY. */
int hdcr_coarse_invert(hdcr_coarse* co, void* stream);
/* out = A^{-1} in (C64, nrhs coarse vectors) with the dense inverse. */
int hdcr_coarse_solve_dense(const hdcr_coarse* co, const void* in, void* out, int nrhs,
                            void* stream);
void hdcr_coarse_destroy(hdcr_coarse* co);

/* ---------------------------------------------------------------- third level
 * hdcr_coarse_build_level2: the two-level construction of Section 4 applied to
 * the coarse operator A itself (Section 5: recursion solves the coarse system
 * more exactly).  nvec2/2 Gaussian noise vectors on the coarse lattice (``noise``:
 * C128 coarse vectors [v][a][k], drawn by the caller) are each smoothed by
 * ``smooth_iters`` CR steps on A x = 0 and normalised, split by the coarse Gamma5
 * (+1 on the first nvec/2 basis components of a site, -1 on the rest: the level-1
 * basis vectors have definite Gamma5 chirality), restricted to blocks of
 * block[0..3] coarse sites times all nvec components and orthonormalised by
 * modified Gram-Schmidt twice per block (FP64); then A2 = P2^dag A P2 (9 legs on
 * the level-2 lattice) is built and inverted densely (FP32).  The level is kept
 * in the coarse handle (rebuilt by a new call, freed with it) and used by
 * hdcr_solve's HDCR_COARSE_RECURSIVE solver, whose V-cycle one level down takes
 * ``cycle_smooth`` CR steps on A as its smoother.  Every block[mu] must divide
 * the coarse extent into >= 2; nvec2 even, 2..64.  Synchronises ``stream``.
 * Errors: BAD_ARG, BAD_GEOMETRY, RANK_DEFICIENT, NONFINITE, CUDA, NO_MEMORY. */
typedef struct {
  int nvec2;         /* level-2 basis size after the split (even)          */
  int block[4];      /* level-2 block in coarse sites                      */
  int smooth_iters;  /* CR steps smoothing each level-2 noise vector       */
  int cycle_smooth;  /* CR steps of the smoother of the recursive V-cycle  */
} hdcr_level2_params;
int hdcr_coarse_build_level2(hdcr_coarse* co, const hdcr_level2_params* p, const void* noise,
                             void* stream);
/* nvec2 (0 without a third level) and the level-2 lattice extents. */
int hdcr_coarse_level2_info(const hdcr_coarse* co, int* nvec2, int L2[4]);
/* Copies the level-2 basis (C128, [nvec2][Vc][nvec]) and A2 (C128,
 * [Vc2][9][nvec2][nvec2]) into device buffers. */
int hdcr_coarse_level2_get(const hdcr_coarse* co, void* vectors, void* op, void* stream);
/* out = A^{-1} in (one coarse vector in the coarse operator's dtype) by the
 * recursive solver to |in - A out| <= tol |in|; *iters receives the GCR
 * iterations.  Synchronises ``stream``.  Errors: BAD_ARG, NONFINITE, CUDA. */
int hdcr_coarse_solve_level2(const hdcr_coarse* co, const void* in, void* out, double tol,
                             int max_iter, int* iters, void* stream);

/* ---------------------------------------------------------------- HDCR solve
 * hdcr_solve: H x = b (Section 4) by flexible GCR(restart) in FP64 on H,
 * preconditioned by the two-level V-cycle
 *     z1 = S r;  z2 = z1 + P A^{-1} P^dag (r - H z1);  z = z2 + S (r - H z2).
 * For a linear smoother and an exact coarse solve this is the composite
 * M_outer = S P_L + P_R S + Q - S P_L H S of Section 4 (``cycle`` =
 * HDCR_CYCLE_SYMMETRIC).  HDCR_CYCLE_POST drops the first smoothing:
 *     z1 = P A^{-1} P^dag r;  z = z1 + S (r - H z1),
 * whose error propagator is (1 - S H)(1 - Q H): half the smoother's fine
 * applications per cycle, not Hermitian (flexible GCR does not need it).
 * Smoothers:
 *   HDCR_SMOOTHER_CR         ``smoother_order`` CR steps from zero (nonlinear);
 *   HDCR_SMOOTHER_CHEBYSHEV  S = H p(H^2), p the order-``smoother_order``
 *                            Chebyshev approximation of 1/y on
 *                            [cheb_lo, cheb_hi] (Section 4: order 10 on [1, 64]).
 * Coarse solvers: HDCR_COARSE_CR (CR on A to ``coarse_tol``, cap
 * ``coarse_max``), HDCR_COARSE_DENSE (the dense inverse of
 * hdcr_coarse_invert, computed on first use) or HDCR_COARSE_RECURSIVE (flexible
 * GCR on A to ``coarse_tol``, cap ``coarse_max``, preconditioned by the third
 * level built by hdcr_coarse_build_level2).  inner_dtype C128 runs the
 * smoother and coarse correction in FP64 (the dense inverse is FP32 in either
 * case); C64 runs them in FP32 (FP32 basis and coarse operator required) while
 * the outer FGCR, its orthogonalisation and the true residual stay FP64.  The
 * solve ends when the true residual |b - H x| / |b| <= tol.  U and b, x are
 * C128; x holds the initial guess.  Synchronises ``stream``.  Solves on one
 * coarse handle must not overlap (they share its cached workspace).
 * Errors: BAD_ARG, NOT_CONVERGED (max_outer reached), NONFINITE, CUDA, NO_MEMORY.
 */
#define HDCR_SMOOTHER_CR 0
#define HDCR_SMOOTHER_CHEBYSHEV 1
#define HDCR_COARSE_CR 0
#define HDCR_COARSE_DENSE 1
#define HDCR_COARSE_RECURSIVE 2 /* FGCR on A with the third level (hdcr_coarse_build_level2) */
#define HDCR_CYCLE_SYMMETRIC 0  /* smoother before and after the coarse correction */
#define HDCR_CYCLE_POST 1       /* coarse correction, then the smoother            */

typedef struct {
  double tol;         /* true relative residual target, e.g. 1e-10           */
  int max_outer;      /* cap on outer iterations                             */
  int restart;        /* FGCR restart length (1..64)                         */
  int smoother_kind;  /* HDCR_SMOOTHER_CR or HDCR_SMOOTHER_CHEBYSHEV         */
  int smoother_order; /* CR steps or Chebyshev order (>= 0)                  */
  double cheb_lo;     /* Chebyshev smoother interval on H^2                  */
  double cheb_hi;
  int coarse_solver;  /* HDCR_COARSE_CR or HDCR_COARSE_DENSE                 */
  double coarse_tol;  /* relative residual of the coarse CR, e.g. 1e-4       */
  int coarse_max;     /* cap on coarse CR iterations                         */
  int inner_dtype;    /* HDCR_C128 or HDCR_C64                               */
  int cycle;          /* HDCR_CYCLE_SYMMETRIC or HDCR_CYCLE_POST             */
} hdcr_solve_params;

int hdcr_solve(hdcr_coarse* co, const void* U, const void* b, void* x,
               const hdcr_solve_params* params, hdcr_solve_stats* stats, void* stream);

/* hdcr_solve_multi: nrhs solves H x_r = b_r (r = 0..nrhs-1) by the method of
 * hdcr_solve, advanced in lockstep so that every application of H, every
 * smoother step, P^dag, the coarse solve and P is one launch over all nrhs
 * fields (Section 4's solve, batched over right-hand sides, e.g. the 12
 * spin-colour point sources of a propagator).  b and x hold nrhs C128 fields
 * one after the other (x: initial guesses); U is C128.  Each right-hand side
 * has its own flexible GCR coefficients; the iteration stops when every true
 * residual |b_r - H x_r| / |b_r| <= tol, so iteration counts are shared.
 * Requires the Chebyshev smoother and the dense coarse solve (the V-cycle is
 * then a fixed sequence of launches); with use_graph != 0 the V-cycle is
 * captured once into a CUDA graph on a library stream and replayed on
 * ``stream`` every outer iteration (re-captured when U, the smoother or the
 * coarse inverse change).  stats: nrhs entries (t_smoother and t_coarse are 0).
 * nrhs 1..64.  Workspace (2 restart + ~9 fields per right-hand side) is cached
 * on the coarse handle; solves on one handle must not overlap.  Synchronises
 * ``stream``.  Errors: as hdcr_solve. */
int hdcr_solve_multi(hdcr_coarse* co, const void* U, const void* b, void* x, int nrhs,
                     const hdcr_solve_params* params, int use_graph, hdcr_solve_stats* stats,
                     void* stream);

/* ---------------------------------------------------------------- continued-fraction overlap
 * hdcr_apply_cf_overlap: out = H_cf in for the continued-fraction form of the
 * overlap operator (Section 3), which the paper prints for five components as the
 * Hermitian-indefinite block-tridiagonal matrix with diagonal blocks H, -H, H, -H,
 * R gamma5 + beta_0 H and scalar off-diagonal blocks 1/sqrt(beta_0 beta_1),
 * 1/sqrt(beta_1 beta_2), 1/sqrt(beta_2 beta_3), 1/sqrt(beta_3), where H = gamma5 D_W is
 * the Hermitian Wilson kernel with mass -M5 (the 4d part of D_dwf above).  For
 * ncomp = N components (2..16): diagonal (-1)^i H for i < N-1 and R gamma5 + beta_0 H
 * last, coupling 1/sqrt(beta_i beta_{i+1}) between i and i+1 for i < N-2 and
 * 1/sqrt(beta_{N-2}) between N-2 and N-1 (beta[0..N-2] > 0).  The N components are
 * stored as the fifth coordinate of a fermion field: g->Ls must equal ncomp.  U and
 * the nrhs fields share ``dtype`` (C128 or C64).  Errors: BAD_ARG, BAD_GEOMETRY. */
typedef struct {
  int ncomp;        /* N, the number of components (2..16)  */
  double beta[15];  /* beta_0 .. beta_{N-2}                  */
  double R;         /* coefficient of gamma5 on the last one */
} hdcr_cf_params;
int hdcr_apply_cf_overlap(const hdcr_geom* g, double M5, const hdcr_cf_params* cf, const void* U,
                          const void* in, void* out, int dtype, int nrhs, void* stream);
/* CR (Section 3) on H_cf x = b in ``dtype``, as hdcr_cr_solve: x holds the initial
 * guess, the true residual |b - H_cf x| / |b| is recomputed into stats->true_resid;
 * the iterations between host checks replay from a captured CUDA graph.
 * Synchronises ``stream``.  Errors: BAD_ARG, NOT_CONVERGED, NONFINITE, CUDA. */
int hdcr_cf_cr_solve(const hdcr_geom* g, double M5, const hdcr_cf_params* cf, const void* U,
                     const void* b, void* x, int dtype, double tol, int max_iter,
                     hdcr_solve_stats* stats, void* stream);
/* The two-level method on the continued-fraction operator (Section 4's
 * construction with H_cf in place of H).
 * hdcr_cf_filter: the subspace filter on H_cf, in place on one field x of
 * ``dtype``: sp->kind HDCR_SUBSPACE_CR_SMOOTH (sp->order CR steps on H_cf x = 0)
 * or HDCR_SUBSPACE_CHEBYSHEV (T_order(t(H_cf^2)), t mapping [lam_cut^2, lam_max^2]
 * onto [-1, 1], then normalised); the other fields of sp are ignored.  The
 * filtered fields, split by 4d chirality (hdcr_gamma5_split) and
 * block-orthonormalised by hdcr_subspace_from_vectors on the same geometry (its
 * Ls = the number of components), form the basis.  Synchronises
 * ``stream``.  Errors: BAD_ARG, CUDA, NO_MEMORY.
 * hdcr_cf_build_coarse_op: A^{ab}_jk = <phi_j^a | H_cf | phi_k^b> on that basis
 * (stored C128, legs as for hdcr_build_coarse_op: the hops leaving the block per
 * leg, everything else, the components' couplings and R gamma5 included, in the
 * self leg).  The handle keeps the operator: hdcr_solve (inner dtype C128),
 * hdcr_apply_coarse, hdcr_coarse_invert and the coarse solves then run on H_cf;
 * hdcr_solve_multi refuses it.  The basis must be stored C128; U is C128 (device
 * or host).  Synchronises ``stream``.  Errors: BAD_ARG, CUDA, NO_MEMORY. */
int hdcr_cf_filter(const hdcr_geom* g, double M5, const hdcr_cf_params* cf, const void* U, void* x,
                   int dtype, const hdcr_subspace_params* sp, void* stream);
/* plus = (1 + gamma5)/2 in, minus = (1 - gamma5)/2 in for nfields fields: the 4d
 * chirality at every site and fifth coordinate (spins 0, 1 and 2, 3 of the chiral
 * basis; no R5 reflection).  The split that makes the continued-fraction basis work:
 * without it the two-level solve on H_cf stalls (measured); with the filtered fields
 * split this way it converges.  Asynchronous on ``stream``.  Errors: BAD_ARG. */
int hdcr_gamma5_split(const hdcr_geom* g, const void* in, void* plus, void* minus, int dtype, int nfields,
                      void* stream);
int hdcr_cf_build_coarse_op(const hdcr_subspace* sub, double M5, const hdcr_cf_params* cf, const void* U,
                            void* stream, hdcr_coarse** out);

/* ---------------------------------------------------------------- gauge force
 * hdcr_gauge_force: the gauge-link gradient of a solve (not in the paper;
 * derived from the operator above).  For H x = b and H y = eta, with
 * w = Gamma5 y, the loss Re(eta^dag x) changes by Re sum tr(dU_mu(x) F_mu(x)) with
 *   F_mu(x) = 1/2 sum_s [ B + C^dag ],
 *   B_ba = sum_alpha [(1 - gamma_mu) x(x+mu,s)]_{alpha b} conj(w(x,s)_{alpha a}),
 *   C_ba = sum_alpha [(1 + gamma_mu) x(x,s)]_{alpha b} conj(w(x+mu,s)_{alpha a})
 * (the t-boundary phase enters through x(x+mu), w(x+mu)).  x, w: one field each;
 * F: 4*V4*9 complex in the gauge layout, F[mu][x4][b][a] = (F_mu(x))_ba.  The
 * gradient of the loss with respect to Re U_ab + i Im U_ab is conj(F_ba).
 */
int hdcr_gauge_force(const hdcr_geom* g, const void* x, const void* w, void* F, int dtype,
                     void* stream);
/* hdcr_gauge_grad: the same sum as hdcr_gauge_force, stored as the gradient of
 * the loss with respect to the links in the gauge layout:
 * G[mu][x4][a][b] = conj((F_mu(x))_ba) = dL/dRe U_ab + i dL/dIm U_ab (the
 * convention of torch's complex autograd).  Errors: BAD_ARG, BAD_GEOMETRY. */
int hdcr_gauge_grad(const hdcr_geom* g, const void* x, const void* w, void* G, int dtype,
                    void* stream);

#ifdef __cplusplus
}
#endif

#endif /* HDCR_H */
