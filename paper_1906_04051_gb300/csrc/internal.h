// internal.h -- host-side launchers shared between the library's translation units.
#pragma once

#include <cuda_runtime.h>

#include "common.cuh"

namespace gg {

int grid_for(long long work, int threads, int max_blocks);
// rows of w per block of the modified Gram-Schmidt kernel (one block per SM), 0 if n
// does not fit in its shared memory
int mgs_rows(int n, int sms);

// fem.cu
cudaError_t launch_q1_assemble(int n, const double* kappa, double bx, double by,
                               const double* f, const double* u, int* rowptr, int* col,
                               double* val, double* b, cudaStream_t st);
cudaError_t launch_q1_kappa_grad(int n, const double* lam, const double* x, double* grad,
                                 cudaStream_t st);
cudaError_t launch_transpose(int n, int nnz, const int* rowptr, const int* col,
                             const double* val, int* rowptr_t, int* col_t, double* val_t,
                             int* scratch, cudaStream_t st);

// setup.cu
cudaError_t launch_validate(int n, long long nnz, const int* rowptr, const int* col,
                            const int* agg, int r, int* err, cudaStream_t st);
int agg_chunks(int n);
// pieces cut at the row ranges of a grid of `grid` blocks over `units` units of 256 rows
// (the fused Arnoldi kernel's partition; grid 0: no cuts), with each block's piece list
cudaError_t launch_agg_perm(int n, int r, const int* agg, int* counts, int* aggptr, int* cnt,
                            int* perm, int* agg_piece, int* piece_start, double* uscale,
                            int units, int grid, int* bcnt, int* blk_piece_start,
                            int* blk_piece, int* err, cudaStream_t st);
cudaError_t launch_coarse_T(int r, const int* rowptr, const int* col, const double* val,
                            const int* agg, const int* perm, const int* aggptr,
                            const double* uscale, double* T, cudaStream_t st);
size_t gj_aux_bytes(int r);
// T^-1 and T^-T: band LU when T is narrowly banded, else Gauss-Jordan (band: kl, ku and
// whether the band path ran, out; nlaunch: the kernels it enqueued)
cudaError_t launch_coarse_inverse(int r, const double* T, double* G, void* aux, double* Tinv,
                                  double* TinvT, int* err, int* band, int* nlaunch,
                                  cudaStream_t st);
cudaError_t launch_gauss_jordan(int r, const double* T, double* G, void* aux, double* Tinv,
                                double* TinvT, int* err, cudaStream_t st);
cudaError_t launch_norm_inf(int n, const int* rowptr, const double* val,
                            unsigned long long* out, cudaStream_t st);
cudaError_t launch_to_float(long long n, const double* a, float* b, cudaStream_t st);
int au_scan_blocks(int n);
cudaError_t launch_au_rows(int n, const int* rowptr, const int* col, const int* agg, int* cnt,
                           int* bsum, int* aurp, cudaStream_t st);
// A W row pointers padded with nau to `total` entries; *tmax = most entries per tile of
// `unit` rows
cudaError_t launch_au_tiles(int n, long long total, int unit, int* aurp, int* tmax,
                            cudaStream_t st);
cudaError_t launch_au_fill(int n, const int* rowptr, const int* col, const double* val,
                           const int* agg, const int* aurp, int* aucol, double* auval,
                           float* auval32, cudaStream_t st);
// the first two A W entries of each row in two row-indexed planes (see setup.cu)
cudaError_t launch_au_planes(int n, const int* aurp, const int* aucol, const double* auval,
                             const float* auval32, int* pcol, double* pval, float* pval32,
                             cudaStream_t st);
cudaError_t launch_dia_detect(int n, const int* rowptr, const int* col, int* slots, int* count,
                              cudaStream_t st);
int dia_empty_slot();
cudaError_t launch_dia_fill(int n, const int* rowptr, const int* col, const double* val,
                            const DiaOffsets& offs, long long ldd, double* dval, float* dval32,
                            cudaStream_t st);
cudaError_t launch_ext_csr(int n, const int* rowptr, const int* col, const double* val,
                           const float* val32, const int* aurp, const int* aucol,
                           const double* auval, const float* auval32, int* xrp, int* xcol,
                           double* xval, float* xval32, cudaStream_t st);

// arnoldi.cu: one restart cycle's kernels, by precision
enum Prec { P_FP64 = 0, P_FP32 = 1, P_BF16 = 2 };

struct OpDev {           // one operator (A or A^T) as the kernels see it
  int n;
  const int* rowptr;
  const int* col;
  const double* val;     // FP64 values (true residual, FP64 inner)
  const float* val32;    // FP32 copy (FP32 inner), may be null
  Defl defl;
  // diagonal storage (dia.nd = 0: none), ldd elements per diagonal
  DiaOffsets dia;
  long long ldd;
  const double* dval;
  const float* dval32;
  // rows [A | A W] (column n + a = aggregate a), for the deflated SpMV of a step
  const int* xrp;
  const int* xcol;
  const double* xval;
  const float* xval32;
  // lanes per row of the CSR SpMV (0: a thread per row); set for long rows
  int vec;
  int au_tile_max;       // most A W entries in a tile of 256 rows
};

struct CycleArgs {
  OpDev op;
  Ctl ctl;
  void* V;               // basis storage (double / float / bf16), column stride ldv
  long long ldv;
  void* w;               // working vector (double for FP64, float otherwise)
  double* t;             // FP64 scratch vector (x update)
  int prec;
  int m;                 // restart length of this solve (<= ctl.ldh)
  int proj;              // deflation projector instead of the EBP preconditioner
  int sms;               // multiprocessors of the device
  int grid_small;        // blocks of the coarse GEMV
  int pdl;               // step kernels with programmatic dependent launch
  int ortho;             // gmres_ortho
  int dot_arith;         // gmres_dot_arith (the fused FP64 step's multi-dot)
  unsigned* gbar;        // grid barrier words of the MGS and fused kernels (4 words)
};

// Phases of a solve; each launch_phase call enqueues the kernels of one phase.
enum Phase {
  PH_SETUP = 0,     // gmres_create: validation, aggregates, T, T^-1
  PH_RESIDUAL,      // r = b - A x in FP64, u_0, stopping decision
  PH_SPMV,          // w = A M^-1 v_j
  PH_DOT1,          // CGS2 pass 1
  PH_UPD1DOT2,      // CGS2 pass 2
  PH_UPD2NORM,      // CGS2 pass 3 + Givens
  PH_DEFL,          // U^T v_j and the coarse correction
  PH_CYCLE_END,     // back substitution and x update
  PH_RITZ,          // |mu| from the Ritz values
  PH_PROJ_FINAL,    // projector: x = xh + U T^-1 U^T (b - A xh)
  PH_ADAPT,         // adaptive deflation: update of U, A U, T, T^-1 after a cycle
  PH_MGS,           // modified Gram-Schmidt step (one cooperative kernel)
  PH_ARNOLDI,       // the Arnoldi steps of a cycle in one persistent kernel (fused.cu)
  PH_COUNT
};
// c = M^T x over ncols FP64 columns of M (leading dimension ldm), pipelined multi-dot with
// the given epilogue (adaptive deflation)
cudaError_t launch_udots(const CycleArgs& a, const double* M, long long ldm, int ncols,
                         const double* x, DotEpi epi, cudaStream_t st);
cudaError_t launch_phase(const CycleArgs& a, int ph, int j, bool defl, double* x,
                         const double* b, cudaStream_t st, int* launches);
// fused.cu: SpMV, one-reduction MGS projections, ||w|| and the rotations of step j in one
// cooperative kernel (diagonal storage, EBP deflation or none, FP64 or FP32)
bool arnoldi_fusable(const CycleArgs& a);
// one launch runs the jmax steps of a restart cycle (fewer when the cycle ends early)
cudaError_t launch_arnoldi(const CycleArgs& a, int jmax, bool defl, cudaStream_t st);
// Control-block initialisation for a new solve.
cudaError_t launch_init(const CycleArgs& a, double tol, double inner_tol, double r0ref,
                        double mu, int fixed, int mixed, long long maxit, cudaStream_t st);

}  // namespace gg
