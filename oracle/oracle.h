/*
 * oracle.h -- plain, sequential FP64 CPU oracle for deflated restarted GMRES(m).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path may include, link or call
 * this code: only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline leg use
 * it.  It shares no source, header, table or helper with the CUDA library.
 *
 * Every routine follows the paper (Ioannidis et al., arXiv:1906.04051) step by step,
 * in FP64, with no blocking, fusion or reordering:
 *   - Q1 Galerkin assembly with Dirichlet row replacement      (Sec. 3.1, Eqs. 6-8)
 *   - the paper's 3-D Bratu Newton system on Q2 hexahedra       (Sec. 3.1, Eqs. 2-9)
 *   - restarted GMRES(m), Arnoldi + Givens least squares       (Sec. 3.2, Eqs. 10-15)
 *   - right preconditioning by deflation M^-1 = I + U(|mu|T^-1 - I)U^T, T = U^T A U
 *                                                              (Sec. 3.3, Eqs. 16-18)
 *   - mu from the Ritz values of H_m                           (Sec. 3.3)
 * Orthogonalisation is classical Gram-Schmidt applied twice (CGS2) by default, with the
 * paper's modified Gram-Schmidt (Sec. 3.2) as a second path.
 */
#ifndef GMRES_ORACLE_H
#define GMRES_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- Q1 finite elements on the unit square, n x n elements, (n+1)^2 nodes ---- */
int64_t orc_q1_nnz(int32_t n);
/* Element matrices for a square element of side h (local node l = a + 2b, a,b in {0,1}):
 * K1 = int grad(phi_i).grad(phi_j) (kappa = 1), C = int phi_i (beta.grad phi_j), M = int phi_i phi_j.
 * All 4x4 row-major. */
void orc_q1_element(double h, double bx, double by, double* K1, double* C, double* M);
/* Assemble A (CSR, ascending columns) and b = M f - K u on interior rows; boundary rows
 * are replaced by u_i = 0 (Sec. 3.1).  kappa: n*n per-element values (element (ei,ej) at
 * ej*n+ei); f, u: nodal values, u may be NULL.  Returns 0. */
int orc_q1_assemble(int32_t n, const double* kappa, double bx, double by, const double* f,
                    const double* u, int32_t* rowptr, int32_t* col, double* val, double* b);
/* dL/dkappa_e = - sum_{i in e, i interior} lam_i (K1 x_e)_i  (adjoint of the assembly). */
void orc_q1_kappa_grad(int32_t n, const double* lam, const double* x, double* grad);

/* ---- 3-D Bratu problem (Sec. 3.1, Eqs. 2-9): lap u + lambda exp(u) = 0 on the unit
 * cube, u = 0 on the x- and y-faces, du/dz = 0 on the z-faces; n x n x n elements with
 * 27 nodes (triquadratic), M = 2n + 1 nodes per direction, node (I, J, K) ->
 * (K M + J) M + I ---- */
int64_t orc_q2_nnz(int32_t n);
/* Element Jacobian J_e (27x27 row-major) and residual R_e (27) for nodal values ue
 * (NULL: zero), local node l = a + 3b + 9c, by 3x3x3 Gauss-Legendre quadrature. */
void orc_q2_element(double h, double lambda, const double* ue, double* Je, double* Re);
/* The Newton system J(u) du = -R(u) (Eq. 9): A = J (CSR, ascending columns, the mesh
 * connectivity pattern), b = -R.  Rows of x- and y-face nodes are replaced by du_i = 0
 * (one stored 1.0, b_i = 0); the other rows keep their couplings to those columns.
 * u may be NULL (u = 0).  Returns 0. */
int orc_q2_bratu_assemble(int32_t n, double lambda, const double* u, int32_t* rowptr,
                          int32_t* col, double* val, double* b);

/* ---- sparse / dense kernels ---- */
void orc_spmv(int32_t N, const int32_t* rowptr, const int32_t* col, const double* val,
              const double* x, double* y);
void orc_transpose(int32_t N, const int32_t* rowptr, const int32_t* col, const double* val,
                   int32_t* rowptr_t, int32_t* col_t, double* val_t);
/* LU with partial pivoting, row-major n x n in place.  Returns 0, or k+1 if the k-th
 * pivot is exactly zero. */
int orc_lu_factor(int32_t n, double* a, int32_t* piv);
void orc_lu_solve(int32_t n, const double* lu, const int32_t* piv, double* b);
/* Eigenvalues of an upper Hessenberg matrix (row-major) by the Francis double-shift QR
 * iteration.  Returns 0, or -1 if the iteration did not converge. */
int orc_hessenberg_eigs(int32_t n, const double* h, double* wr, double* wi);

/* ---- deflation (Sec. 3.3) with U = W diag(1/sqrt|agg_p|), W = aggregate indicators ---- */
typedef struct orc_defl orc_defl;
/* agg[i] in [0,r) or -1.  Forms T = U^T A U and its LU.  Returns NULL on an empty
 * aggregate or a singular T (status in *err: -4). */
orc_defl* orc_defl_create(int32_t N, const int32_t* rowptr, const int32_t* col,
                          const double* val, int32_t r, const int32_t* agg, int* err);
void orc_defl_destroy(orc_defl* d);
void orc_defl_T(const orc_defl* d, double* T);                      /* r*r row-major */
void orc_defl_apply_Minv(const orc_defl* d, double mu, const double* v, double* z);
void orc_defl_apply_P(const orc_defl* d, const double* w, double* out); /* (I - AU T^-1 U^T) w */

/* ---- GMRES(m) ---- */
enum { ORC_CGS2 = 0, ORC_MGS = 1 };
enum { ORC_DEFL_NONE = 0, ORC_DEFL_EBP = 1, ORC_DEFL_PROJECTOR = 2, ORC_DEFL_ADAPTIVE = 3 };
enum { ORC_MU_RITZ_FIRST_CYCLE = 0, ORC_MU_USER = 1, ORC_MU_NORM_INF = 2 };

typedef struct {
  int32_t m;
  double tol;
  int64_t maxit;            /* total Arnoldi steps */
  int32_t ortho;            /* ORC_CGS2 / ORC_MGS */
  int32_t defl_mode;        /* ORC_DEFL_* */
  int32_t mu_mode;          /* ORC_MU_* */
  double mu_user;
  int32_t fixed_iterations; /* 1: no convergence test, exactly maxit steps */
  double r0_norm_ref;       /* > 0: reference norm for the relative tolerance */
  /* ORC_DEFL_ADAPTIVE (Sec. 3.3, Eq. 19): U starts empty and grows by the inverse-power
   * eigenvectors of each cycle's H_k mapped through V_k, at most rmax columns */
  int32_t rmax;             /* upper limit on the columns of U (paper: 20) */
  int32_t ninv;             /* inverse power iterations per restart */
  double* u_out;            /* N x rmax column-major (may be NULL): the final U */
  /* a deflation space given as dense columns instead of aggregates (Eqs. 16-18 with this
   * U): W is N x w_cols column-major, U its orthonormalisation (two classical
   * Gram-Schmidt passes per column, in order), fixed for the whole solve; the
   * preconditioner and mu are those of ORC_DEFL_EBP.  w_cols = 0: none. */
  const double* w_dense;
  int32_t w_cols;
} orc_opts;

typedef struct {
  int64_t iters, cycles;
  int32_t status;           /* 0 converged, 1 not converged, <0 error */
  double rel_res_est, rel_res_true, mu;
  int32_t q;                /* columns of U at the end (ORC_DEFL_ADAPTIVE) */
} orc_info;

/* Inverse power method on a k x k upper Hessenberg H (row-major; Sec. 3.3): iterates
 * z <- H^-1 z / ||H^-1 z|| ninv times from the normalised all-ones vector (LU with
 * partial pivoting between the two rows each column touches; a zero pivot is replaced
 * by 1e-14 max|H|), then sign-normalises z (its largest-magnitude entry positive, the
 * first one on ties).  If z is not an eigenvector to within ||Hz - (z^T H z) z|| <=
 * 1e-3 ||Hz|| (the smallest eigenvalues form a complex pair), one more iterate is
 * orthonormalised against z and returned as z2: the pair spans the pair's invariant
 * subspace.  Returns the number of vectors (1 or 2), 0 if k < 1. */
int orc_hess_invvec(int32_t k, const double* H, int32_t ninv, double* z1, double* z2);

/* The drop step of the adaptive deflation when U is full (Sec. 3.3: the vectors that
 * correspond to the largest eigenvalues of T_r leave the space).  T: q x q (row stride
 * ldt).  Its eigenvalue lambda of largest modulus (Householder reduction to Hessenberg
 * form, then orc_hessenberg_eigs; the first on ties) has a left eigenvector y (T^T y =
 * lambda y; inverse iteration, three solves from all ones, on the real 2q x 2q form when
 * lambda is complex).  The real vectors c with y^T c = 0 form a T-invariant subspace
 * that carries the other eigenvalues; Qc (q x (q-p), row-major, orthonormal columns) is
 * a basis of it (the last q - p columns of the Householder QR factor of [Re y, Im y]) and
 * Tn = Qc^T T Qc ((q-p) x (q-p)).  Returns p (1, or 2 for a complex pair) or -1 when
 * the QR iteration fails. */
int orc_adapt_drop(int32_t q, const double* T, int32_t ldt, double* Qc, double* Tn);

/* Solves A x = b.  d may be NULL (no deflation).  hist (2*maxit doubles, may be NULL)
 * receives, per Arnoldi step, (step index j within its cycle, |gamma_{j+1}| / rho0). */
int orc_gmres(int32_t N, const int32_t* rowptr, const int32_t* col, const double* val,
              const orc_defl* d, const double* b, const double* x0, const orc_opts* o,
              double* x, orc_info* info, double* hist);

/* k Arnoldi steps on the operator of the chosen deflation mode (A M^-1, or P A), from
 * v0 (normalised inside).  V: N*(k+1) column-major, H: (k+1)*k row-major.  Returns the
 * number of steps done (< k on breakdown). */
int orc_arnoldi(int32_t N, const int32_t* rowptr, const int32_t* col, const double* val,
                const orc_defl* d, int32_t defl_mode, double mu, int32_t ortho,
                const double* v0, int32_t k, double* V, double* H);

#ifdef __cplusplus
}
#endif
#endif
