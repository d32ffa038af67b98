/*
 * gmres_gb300.h -- C ABI of the GB300 (sm_103a) deflated restarted GMRES(m) library.
 *
 * Method: Ioannidis et al., "On the performance of various parallel GMRES
 * implementations on CPU and GPU clusters", arXiv:1906.04051.
 *   Sec. 3.2, Eqs. 10-15  restarted GMRES(m): Arnoldi basis V_m of K_m(A, r0/||r0||),
 *                         least squares min ||beta e1 - Hbar_m y|| by plane rotations,
 *                         residual estimate |gamma_{k+1}|, restart with x_m as new x0,
 *                         stop when ||b - A x|| / ||b - A x0|| falls below tol.
 *   Sec. 3.3, Eqs. 16-18  right preconditioning A M^-1 z = b, x = M^-1 z, with the
 *                         deflation preconditioner M^-1 = I + U (|mu| T^-1 - I) U^T,
 *                         T = U^T A U, mu the largest eigenvalue of A estimated from the
 *                         Ritz values of H_m.
 *   Sec. 3.1, Eqs. 2-9    Galerkin finite-element assembly with Dirichlet rows replaced
 *                         by u_i = 0: bilinear Q1 elements on the unit square
 *                         (convection-diffusion), and the paper's 3-D Bratu problem on
 *                         27-node hexahedra solved by Newton's method.
 *
 * Conventions shared by every entry point
 *   - Pointers named "device" must point to memory of the current CUDA device; the
 *     library never dereferences them on the host.  Host pointers are marked "host".
 *   - A "stream" argument is a cudaStream_t passed as void* (NULL = legacy default
 *     stream).  All device work of a call is enqueued on that stream.
 *   - Matrices are CSR with int32 row pointers and int32 column indices, columns strictly
 *     ascending within each row, no duplicates, values in FP64.
 *   - Negative status = error: nothing about the outputs is guaranteed.  A positive
 *     status (GMRES_NOT_CONVERGED) is a normal return: x holds the last iterate and the
 *     info struct is valid.
 *   - No entry point falls back to the CPU: every arithmetic step runs in this library's
 *     CUDA kernels.
 */
#ifndef GMRES_GB300_H
#define GMRES_GB300_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct gmres_s* gmres_t; /* opaque handle: owns device copies and workspace */

typedef enum {
  GMRES_OK = 0,
  GMRES_NOT_CONVERGED = 1,        /* maxit Arnoldi steps done without reaching tol */
  GMRES_ERR_INVALID_ARG = -1,     /* bad size, pointer, option, CSR or aggregate map */
  GMRES_ERR_CUDA = -2,            /* a CUDA runtime call failed; see gmres_last_error */
  GMRES_ERR_OOM = -3,             /* device allocation failed */
  GMRES_ERR_SINGULAR_COARSE = -4, /* empty aggregate (zero column of W), singular T, or
                                     no usable Ritz estimate of mu */
  GMRES_ERR_NAN = -5,             /* NaN/Inf met in a residual or Hessenberg entry */
  GMRES_ERR_TIMEOUT = -6          /* opts.timeout_ms elapsed (checked at restarts), or a
                                     bounded device wait ran out (a basis copy, or the
                                     grid barrier of GMRES_ORTHO_MGS) */
} gmres_status;

/* Matrix A (Eq. 1), n x n.  All arrays device, read during gmres_create only: the
 * library keeps its own copies, so the caller may free them afterwards. */
typedef struct {
  int32_t n;
  int64_t nnz;
  const int32_t* rowptr; /* n+1 entries, rowptr[0] = 0, rowptr[n] = nnz, nnz < 2^31 */
  const int32_t* col;    /* nnz entries in [0, n), strictly ascending per row */
  const double* val;     /* nnz entries */
} gmres_csr;

/* Deflation space W (Eq. 17), in one of two forms.
 * Aggregates: agg (device, n entries) gives the aggregate of each row in [0, r), or -1
 * for none; W holds their r indicator columns and the library forms
 * U = W diag(1/sqrt|agg_p|), which has orthonormal columns, and T = U^T A U.
 * 1 <= r <= 6144; every aggregate must be non-empty.
 * Dense columns: dense (device, n x r column-major, column c at dense + c n), agg NULL,
 * 1 <= r <= 32 (approximate eigenvectors, say): the library keeps a copy and, at the
 * first solve, orthonormalises the columns in order into U (two classical Gram-Schmidt
 * passes each; GMRES_ERR_INVALID_ARG if a column lies in the span of the previous ones)
 * and forms A U, T = U^T A U and T^-1.  GMRES_DEFL_EBP, FP64, forward single-system
 * solves.
 * r = 0 (agg and dense may be NULL) disables deflation. */
typedef struct {
  int32_t r;
  const int32_t* agg;
  const double* dense;
} gmres_defl;

typedef enum {
  GMRES_FP64 = 0,        /* everything in FP64 */
  GMRES_FP32_INNER = 1,  /* each restart cycle (inner solve) runs SpMV and Arnoldi in
                            FP32 with an FP32 basis; H, Givens, the true residual
                            r = b - A x and the update of x with its coarse correction
                            stay FP64 (iterative refinement: one inner cycle per
                            refinement); the coarse solve of each step, whose result the
                            FP32 SpMV reads in FP32, runs in FP32 (an FP32 copy of T^-1)
                            where the step is fused, in FP64 elsewhere */
  GMRES_BF16_BASIS = 2   /* as GMRES_FP32_INNER, with the basis V stored in BF16 and
                            FP32 accumulation */
} gmres_precision;

typedef enum {
  GMRES_DEFL_EBP = 0,       /* M^-1 = I + U (|mu| T^-1 - I) U^T  (Eq. 17, the paper's) */
  GMRES_DEFL_PROJECTOR = 1, /* P = I - A U T^-1 U^T: GMRES on P A xh = P b, then
                               x = xh + U T^-1 U^T (b - A xh); P A W = 0.  The true
                               residual of x equals P (b - A xh), which the stopping test
                               uses (single-system solves; not in gmres_batch_solve) */
  GMRES_DEFL_NONE = 2,
  GMRES_DEFL_ADAPTIVE = 3   /* the paper's adaptive EBP (Sec. 3.3, Eq. 19): U starts empty;
                               after every restart cycle the eigenvector of the cycle's
                               H_k for its smallest-modulus eigenvalue (inverse power
                               method; a complex pair gives two vectors) is mapped through
                               the basis, u = V_k z, orthonormalised against U and
                               appended; with rmax columns in U, the direction of the
                               largest-modulus eigenvalue of T = U^T A U (two for a
                               complex pair) leaves first: U keeps the complement of
                               that eigenvalue's left eigenvector, a T-invariant
                               subspace.  W (gmres_defl) must be empty; FP64 only;
                               single-system solves */
} gmres_deflation_mode;

typedef enum {
  GMRES_MU_RITZ_FIRST_CYCLE = 0, /* cycle 1 runs with M = I; |mu| = largest modulus of
                                    the eigenvalues of its H_k (Ritz values, Sec. 3.3) */
  GMRES_MU_USER = 1,             /* |mu| = |opts.mu_user| */
  GMRES_MU_NORM_INF = 2          /* |mu| = max_i sum_j |a_ij| (an upper bound) */
} gmres_mu_mode;

typedef enum {
  GMRES_ORTHO_CGS2 = 0,     /* classical Gram-Schmidt applied twice (three pipelined passes
                               over the basis per Arnoldi step) */
  GMRES_ORTHO_MGS = 1,      /* the paper's modified Gram-Schmidt (Sec. 3.2, Eq. 13): one
                               projection after the other, in one cooperative kernel per
                               step that keeps w in shared memory; half the FMAs of CGS2.
                               FP64 single-system solves with n <= 28,000 x the SM count */
  GMRES_ORTHO_MGS_LOWSYNC = 2 /* the same projections as MGS in the inverse compact WY
                               form: one reduction gives V^T w and V^T v_j, h solves
                               (I + L) h = V^T w with L the strictly lower part of V^T V,
                               and w -= V h; two passes over the basis per step, 3k FMAs
                               per row instead of CGS2's 4k.  FP64 and FP32 inner solves,
                               single-system and batched */
} gmres_ortho;

typedef enum {
  GMRES_DOT_FP64 = 0,  /* the basis multi-dot in FP64 FMAs */
  GMRES_DOT_DF32 = 1   /* the multi-dot V^T [w, v_j] of the one-reduction MGS step in
                          double-FP32 on the FP32 pipe: each FP64 operand split into two
                          floats (47 significant bits), products exact by FMA (Dekker's
                          two-product), sums by Knuth's TwoSum, each block's totals rounded
                          to FP64 once; magnitudes below 2^-126 count as 0.  The rest of the
                          step (SpMV, update, norm, H, rotations) stays FP64.  FP64 solves
                          with GMRES_ORTHO_MGS_LOWSYNC only (GMRES_ERR_INVALID_ARG
                          otherwise); applied where the step runs fused (a diagonal-structured
                          A, aggregate or no deflation), FP64 FMAs elsewhere */
} gmres_dot_arith;

typedef struct {
  int32_t precision;        /* gmres_precision */
  int32_t deflation_mode;   /* gmres_deflation_mode */
  int32_t mu_mode;          /* gmres_mu_mode */
  double mu_user;
  int32_t fixed_iterations; /* 1: no convergence test; exactly maxit Arnoldi steps
                               (the fixed 50 x 100 protocol of Sec. 4) */
  double r0_norm_ref;       /* > 0: reference norm for the relative tolerance instead of
                               ||b - A x0|| (resume after a restart boundary) */
  int32_t timeout_ms;       /* > 0: give up with GMRES_ERR_TIMEOUT after this long */
  double inner_tol;         /* mixed precision: a cycle ends once its own residual
                               estimate falls by this factor (0 = 1e-4 FP32, 1e-2 BF16) */
  int32_t profile;          /* 1: bracket every phase with CUDA events (gmres_profile) */
  int32_t rmax;             /* GMRES_DEFL_ADAPTIVE: most columns of U, 1..32 (paper: 20) */
  int32_t ninv;             /* GMRES_DEFL_ADAPTIVE: inverse power iterations per restart */
  int32_t ortho;            /* gmres_ortho (default CGS2) */
  int32_t dot_arith;        /* gmres_dot_arith (default GMRES_DOT_FP64) */
} gmres_opts;

/* Phases reported by gmres_profile (kernel groups of one solve). */
typedef enum {
  GMRES_PH_SETUP = 0,     /* gmres_create (host wall time, ms) */
  GMRES_PH_RESIDUAL = 1,  /* r = b - A x in FP64 and the restart decision (Eq. 15) */
  GMRES_PH_SPMV = 2,      /* w = A M^-1 v_j (Eqs. 16-17) */
  GMRES_PH_DOT1 = 3,      /* CGS2 pass 1: h = V^T w */
  GMRES_PH_UPD1DOT2 = 4,  /* CGS2 pass 2: w -= V h, h' = V^T w */
  GMRES_PH_UPD2NORM = 5,  /* CGS2 pass 3: w -= V h', ||w|| and the plane rotations */
  GMRES_PH_DEFL = 6,      /* U^T v and the coarse correction (Eqs. 17-18) */
  GMRES_PH_CYCLE_END = 7, /* back substitution and x += M^-1 V y (Eq. 11) */
  GMRES_PH_RITZ = 8,      /* |mu| from the Ritz values of H_k */
  GMRES_PH_PROJ_FINAL = 9,/* projector: x = xh + U T^-1 U^T (b - A xh) */
  GMRES_PH_ADAPT = 10,    /* adaptive deflation: the update of U, A U, T, T^-1 */
  GMRES_PH_MGS = 11,      /* modified Gram-Schmidt step: projections, ||w||, rotations */
  GMRES_PH_ARNOLDI = 12,  /* a whole step in one kernel: SpMV, one-reduction MGS, ||w||,
                             rotations (Eqs. 10, 12-14) */
  GMRES_PH_COUNT = 13
} gmres_phase;

typedef struct {
  int64_t iters;        /* Arnoldi steps done */
  int64_t cycles;       /* restart cycles (= refinements in mixed precision) */
  int64_t refinements;  /* FP64 residual recomputations after an inner cycle */
  double rel_res_est;   /* |gamma_{k+1}| / rho0 of the last step (Eq. 14) */
  double rel_res_true;  /* ||b - A x|| / rho0 in FP64 at return (Eq. 15) */
  double mu;            /* |mu| used by the EBP preconditioner (0 if none) */
  float ms_total;       /* device time of the solve, CUDA events on the handle stream */
  int32_t status;       /* same as the return value */
} gmres_info;

/* Fills *o with the defaults: FP64, EBP, Ritz mu, no fixed iterations, no timeout. */
void gmres_opts_default(gmres_opts* o);

/* Setup (Eqs. 17-18): validates and copies A and the aggregate map, builds the
 * aggregate permutation, U's scaling, T = U^T A U and T^-1 (band LU with partial pivoting
 * when T is narrowly banded, as for a structured partition into aggregates; Gauss-Jordan
 * with partial pivoting otherwise), all on the device.  *h receives the handle.  W may be NULL (no deflation).
 * o may be NULL (defaults).  Synchronises the stream before returning.
 * Errors: INVALID_ARG (n <= 0, null pointers, unsorted/out-of-range CSR, agg out of
 * range, r > 6144), SINGULAR_COARSE (empty aggregate, zero pivot in T), OOM, CUDA. */
gmres_status gmres_create(gmres_t* h, const gmres_csr* A, const gmres_defl* W,
                          const gmres_opts* o, void* stream);

/* Solves A x = b by deflated GMRES(m) (Sec. 3.2-3.3).  b (device, n), x0 (device, n,
 * may be NULL = zero), x (device, n, may alias x0).  m: restart length, 1 <= m <= 64.
 * tol >= 0: relative residual target.  maxit >= 0: total Arnoldi steps.  info (host,
 * may be NULL).  Returns after the stream is synchronised.  Workspace is owned by the
 * handle and grown on demand: calls on one handle must not overlap. */
gmres_status gmres_solve(gmres_t h, const double* b, const double* x0, int32_t m,
                         double tol, int64_t maxit, double* x, gmres_info* info);

/* Same solve as gmres_solve, but on success the call allocates no memory, on the device or
 * the host (an error records its message in the handle, as every entry point does): the
 * workspace it needs (Krylov basis, working vectors, control block, reduction
 * partials) is carved from one 32 MiB array in the library's static device memory, which
 * every device that loads the library holds until the process exits.  Intended for
 * callers that must not allocate once set up: real-time loops with a frozen memory
 * budget, or processes where a framework's caching allocator owns the device memory and
 * an extra cudaMalloc could fail or fragment it.  The handle (from gmres_create, which
 * does allocate) provides A and the deflation data.  The paper has no counterpart.
 * Limits: the workspace must fit in 32 MiB, otherwise GMRES_ERR_INVALID_ARG with a
 * message naming the size.  It is the basis, (m+1) round_up(n, 256) elements of 8 bytes
 * (FP64), 4 (FP32) or 2 (BF16), plus two FP64 vectors of round_up(n, 256) entries, plus
 * the reduction partials, 8 x 144 x 8 x (number of SMs) bytes (1.4 MB on a 152-SM GPU),
 * plus a few kilobytes (control block, aggregate sums).  The first call on a device looks
 * up the array's device address (cudaGetSymbolAddress) with that device current and
 * caches it (thread-safe): make that first call before any stream capture.  A
 * cudaDeviceReset after that first call is not supported (the cached address would be
 * stale).  Every call on every handle shares the one
 * array and it keeps the previous call's contents (the call clears what must start at
 * zero): calls that overlap on the GPU, in any stream, race and give wrong results, so
 * serialise them.  ms_total in info is host wall time.  Arguments, outputs and errors as
 * gmres_solve; the per-phase profile of gmres_profile is not updated.  Handles with
 * GMRES_DEFL_ADAPTIVE, a dense W or an orthogonalisation other than GMRES_ORTHO_CGS2 are
 * refused with GMRES_ERR_INVALID_ARG (their workspace does not fit the fixed array). */
gmres_status gmres_solve_noalloc(gmres_t h, const double* b, const double* x0, int32_t m,
                                 double tol, int64_t maxit, double* x, gmres_info* info);

/* Adjoint solve A^T lam = g with the transposed preconditioner
 * M^-T = I + U (|mu| T^-T - I) U^T (same U; T^T = U^T A^T U).  The transpose of A is
 * built on the first call and kept.  Arguments as gmres_solve.  A handle with a dense W
 * is refused with GMRES_ERR_INVALID_ARG. */
gmres_status gmres_adjoint_solve(gmres_t h, const double* g, const double* lam0, int32_t m,
                                 double tol, int64_t maxit, double* lam, gmres_info* info);

/* Solves count independent systems, system i with handle hs[i] (host array), in one
 * persistent launch on `stream`.  b, x0, x: host arrays of count device pointers (x0
 * may be NULL, or contain NULLs).  infos: host array of count entries, may be NULL.
 * All handles must use the same precision, the same orthogonalisation (GMRES_ORTHO_CGS2,
 * or GMRES_ORTHO_MGS_LOWSYNC with an FP64 or FP32 basis), and W as aggregates (or no W)
 * with deflation_mode EBP or NONE; otherwise GMRES_ERR_INVALID_ARG before any launch.
 * Returns the worst status. */
gmres_status gmres_batch_solve(int32_t count, gmres_t const* hs, const double* const* b,
                               const double* const* x0, int32_t m, double tol,
                               int64_t maxit, double* const* x, gmres_info* infos,
                               void* stream);

/* Per-phase device time (ms, from CUDA events on the handle stream while profiling is on;
 * the setup entry is host wall time) and kernel launch counts (always counted) summed
 * since the last reset.  ms and launches (host, GMRES_PH_COUNT entries each) may be NULL.
 * reset != 0 zeroes the sums after reading them.  enable: 1 on, 0 off, -1 unchanged.
 * Host-only; never blocks. */
gmres_status gmres_profile(gmres_t h, int32_t enable, int32_t reset, double* ms,
                           int64_t* launches);

/* Device data layout chosen at create (host-only, never blocks).  No counterpart in the
 * paper: it reports how the operator and the deflation space are stored. */
typedef struct gmres_layout {
  int64_t n, nnz;     /* order and stored entries of A */
  int32_t r;          /* deflation vectors (aggregates); 0 without deflation */
  int32_t npieces;    /* runs of at most 1024 nodes in which U^T x is summed */
  int32_t ndiag;      /* diagonals of A in diagonal storage; 0: A is kept in CSR only */
  int32_t adapt_q;    /* GMRES_DEFL_ADAPTIVE: columns of U after the last solve, else 0 */
  int64_t nau;        /* entries of A W (coarse part of the deflated SpMV) */
  int64_t ldv;        /* rows per basis column in device memory (n rounded up) */
  int32_t spmv_lanes; /* CSR SpMV: lanes per row (4 for rows of 16+ entries on average;
                         0: a thread per row, or diagonal storage) */
  int32_t coarse_band; /* T^-1 from the band LU: T's band width kl + ku + 1; 0: Gauss-Jordan
                          (or no aggregates) */
} gmres_layout;
gmres_status gmres_layout_query(gmres_t h, gmres_layout* out);

/* The dense deflation space of a handle: the adaptive one left by the last solve of a
 * GMRES_DEFL_ADAPTIVE handle (Sec. 3.3, Eqs. 17-19), or the orthonormalised dense W given
 * at create (after the first solve): U (orthonormal, n x q) and T = U^T A U (q x q).  q (host,
 * required) receives the column count, at most opts.rmax.  U (device, may be NULL)
 * receives column c at U + c * ldu (ldu >= n); T (device, may be NULL) receives
 * T[i * q + j] = u_i^T A u_j.  Call with both NULL to learn q first.  Synchronises the
 * handle's stream.  The space belongs to the handle and is rebuilt (from empty) by the
 * next solve (adaptive).  Errors: INVALID_ARG (no dense space, null q, ldu < n), CUDA. */
gmres_status gmres_adaptive_space(gmres_t h, int32_t* q, double* U, int64_t ldu, double* T);

gmres_status gmres_set_stream(gmres_t h, void* stream);
/* Message of the last error on this handle (or of the last failed create when h is
 * NULL).  Owned by the library, valid until the next call on the handle. */
const char* gmres_last_error(gmres_t h);
void gmres_destroy(gmres_t h);

/* ---- Q1 Galerkin assembly on the device (Sec. 3.1, Eqs. 6-8) -------------------------
 * Unit square, n x n square elements, node (i, j) -> j*(n+1)+i.  A has the mesh
 * connectivity pattern; each boundary row is replaced by u_i = 0 (one entry 1.0,
 * b_i = 0); interior rows keep their couplings to boundary columns. */

/* nnz of the assembled matrix: 9 (n-1)^2 + 4 n. */
int64_t q1_nnz(int32_t n);

/* kappa (device, n*n, element (ei, ej) at ej*n+ei): per-element diffusion coefficient.
 * (bx, by): convection vector.  f (device, (n+1)^2): nodal load values, b = M f on
 * interior rows (consistent mass matrix).  u (device, (n+1)^2, may be NULL): a nodal
 * linearisation point, b -= K u on interior rows.  Outputs (device): rowptr
 * ((n+1)^2 + 1 entries), col and val (q1_nnz(n) entries), b ((n+1)^2 entries).
 * Deterministic: the same inputs give bitwise identical outputs.
 * Errors: INVALID_ARG (n < 1, null pointer, nnz >= 2^31), CUDA. */
gmres_status q1_assemble(int32_t n, const double* kappa, double bx, double by,
                         const double* f, const double* u, int32_t* rowptr, int32_t* col,
                         double* val, double* b, void* stream);

/* Adjoint of the assembly with respect to kappa: grad_e = - lam^T (dA/dkappa_e) x
 * = - sum_{i in e, i interior} lam_i (K1 x_e)_i, where K1 is the unit-kappa element
 * stiffness.  lam, x (device, (n+1)^2), grad (device, n*n). */
gmres_status q1_kappa_grad(int32_t n, const double* lam, const double* x, double* grad,
                           void* stream);

/* ---- The paper's benchmark: 3-D Bratu problem (Sec. 3.1, Eqs. 2-9) -------------------
 * lap u + lambda exp(u) = 0 on the unit cube, u = 0 on the x- and y-faces, du/dz = 0 on
 * the z-faces; Galerkin method with n^3 cubic 27-node (triquadratic) elements,
 * M = 2n + 1 nodes per direction, node (I, J, K) -> (K M + J) M + I, N = M^3.  Newton's
 * method solves J(u) du = -R(u) (Eq. 9) with this library's GMRES(m).  Rows of x- and
 * y-face nodes are replaced by du_i = 0 (one entry 1.0, b_i = 0); the other rows keep
 * their couplings to those columns (the pattern is the mesh connectivity, as counted by
 * the paper's Table 1).  The element integrals use 3 x 3 x 3 Gauss-Legendre points. */

/* nnz of the Newton matrix: M (4M - 4) + S^2 (S + 6), S = 8n - 5 (Table 1: 1,603,945 at
 * n = 15, 108,583,705 at n = 60). */
int64_t q2_nnz(int32_t n);

/* The Newton system at u (device, N entries; NULL: u = 0): rowptr (N + 1), col and val
 * (q2_nnz(n) entries; columns ascending), b = -R(u) (N).  All device, caller-owned.
 * Deterministic.  Errors: INVALID_ARG (n < 1, null output, non-finite lambda, nnz or
 * N >= 2^31), CUDA. */
gmres_status q2_bratu_assemble(int32_t n, double lambda, const double* u, int32_t* rowptr,
                               int32_t* col, double* val, double* b, void* stream);

typedef struct {
  int32_t newton_iters;   /* Newton steps taken */
  int32_t status;         /* GMRES_OK when ||du||_inf <= newton_tol, else why it stopped */
  int64_t gmres_iters;    /* Arnoldi steps over all linear solves */
  double du_inf;          /* max |du_i| of the last step */
  double last_rel_res;    /* true relative residual of the last linear solve */
  float ms_total;         /* device time of the whole Newton iteration */
  float ms_assemble;      /* of which assembly */
  float ms_solve;         /* of which GMRES solves (setup excluded) */
  int32_t reserved;
  int64_t step_iters[32]; /* GMRES steps of Newton steps 1..32 */
  double step_du[32];     /* ||du||_inf of Newton steps 1..32 */
} q2_newton_info;

/* Newton's method for the Bratu problem from u (device, N entries, updated in place):
 * per step the system is assembled, a handle is created with opts and W (W may be NULL;
 * its aggregates index the N nodes), GMRES(m) solves J du = -R from du = 0 to tol
 * (relative; a step whose solve stops at maxit is still taken: inexact Newton), and
 * u += du.  Stops when max |du_i| <= newton_tol (status GMRES_OK) or after max_newton
 * steps (GMRES_NOT_CONVERGED).  Allocates its CSR and vectors for the call.  Errors:
 * INVALID_ARG, the errors of gmres_create and gmres_solve (message in
 * gmres_last_error(NULL)), NAN, CUDA. */
gmres_status q2_bratu_newton(int32_t n, double lambda, const gmres_opts* opts,
                             const gmres_defl* W, int32_t m, double tol, int64_t maxit,
                             double newton_tol, int32_t max_newton, double* u,
                             q2_newton_info* info, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* GMRES_GB300_H */
