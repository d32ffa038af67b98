// handle.h -- host-side state of a gmres_t handle and its workspace helpers, shared by
// the single-system driver (solver.cu) and the batched driver (batch.cu).
#pragma once

#include <algorithm>

#include <chrono>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "common.cuh"
#include "internal.h"

using namespace gg;

extern thread_local std::string g_create_error;

struct DevMem {
  void* p = nullptr;
  size_t bytes = 0;
  DevMem() = default;
  DevMem(const DevMem&) = delete;
  DevMem& operator=(const DevMem&) = delete;
  ~DevMem() { release(); }
  void release() {
    if (p) cudaFree(p);
    p = nullptr;
    bytes = 0;
  }
  cudaError_t ensure(size_t n) {
    if (n <= bytes && p) return cudaSuccess;
    release();
    cudaError_t e = cudaMalloc(&p, n ? n : 16);
    if (e == cudaSuccess) bytes = n;
    return e;
  }
  template <typename T> T* as() const { return static_cast<T*>(p); }
};

struct Meta {  // mirrors the device status block
  double scal[S_NSCAL];
  long long counts[C_NCOUNT];
  int flags[F_NFLAGS];
};

struct OpHost {
  DevMem rowptr, col, val, val32, tinv, tinv32;  // tinv32: FP32 copy (FP32 / BF16 solves)
  DevMem aurp, aucol, auval, auval32;  // A W in CSR (projector, residual)
  DevMem aup_col, aup_val, aup_val32;  // its first two entries per row, two planes of n
  DevMem xrp, xcol, xval, xval32;      // [A | A W] rows (deflated SpMV of a step)
  DevMem dval, dval32;                 // diagonal storage (banded operators)
  long long nau = 0;                   // entries of A W
  int au_tile_max = 0;                 // most A W entries in a tile of 256 rows
  DiaOffsets dia{};
  long long ldd = 0;
  bool ready = false;
};

struct gmres_s {
  int n = 0;
  long long nnz = 0;
  cudaStream_t stream = nullptr;
  gmres_opts opts{};
  int sms = 152;
  std::string err;
  OpHost fwd, adj;
  // deflation (shared by A and A^T)
  int r = 0, npieces = 0;
  DevMem agg, perm, piece_start, agg_piece, uscale;
  int tband[3] = {0, 0, 0};           // T's lower and upper bandwidth, band LU used (create)
  int coarse_band = 0;                // kl + ku + 1 when T^-1 came from the band LU, else 0
  int blk_grid = 0;                   // blocks of the fused kernel the pieces are cut for
  DevMem blk_piece_start, blk_piece;  // each block's pieces
  double mu_norminf = 0.0;
  // workspace
  int ldh = 0, prec_ws = -1;
  long long ldv = 0;
  DevMem V, w, t, dctl, meta, part, part2, tickets, cpart, sdefl;
  // adaptive deflation (GMRES_DEFL_ADAPTIVE): U, A U (ldv x rmax), T (rmax x rmax),
  // T^-1 (q x q), a work vector, small scratch; aq columns in use
  DevMem aU, aAU, aT, aTinv, au, asmall;
  DevMem gbar;  // grid barrier words of the modified Gram-Schmidt and fused Arnoldi kernels
  DevMem lmat;  // strictly lower part of V^T V (one-reduction MGS)
  // a deflation space given as dense columns W (n x dense_r), orthonormalised into the
  // dense-space buffers above (aU, aAU, aT, aTinv) at the first solve
  DevMem wdense;
  int dense_r = 0;
  bool dense_built = false;
  int aq = 0;
  Meta* hmeta = nullptr;  // pinned
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  // per-phase profiling: events bracket each phase when enabled; launches always counted
  bool prof_on = false;
  std::vector<cudaEvent_t> pev;
  std::vector<int> pph;
  int pused = 0;
  double pms[PH_COUNT] = {0};
  long long plaunch[PH_COUNT] = {0};
  ~gmres_s() {
    for (cudaEvent_t e : pev) cudaEventDestroy(e);
  }
};

inline gmres_status fail(gmres_s* h, gmres_status s, const std::string& msg) {
  if (h) h->err = msg;
  else g_create_error = msg;
  return s;
}

inline gmres_status cuda_fail(gmres_s* h, cudaError_t e, const char* where) {
  std::string m = std::string(where) + ": " + cudaGetErrorString(e);
  return fail(h, e == cudaErrorMemoryAllocation ? GMRES_ERR_OOM : GMRES_ERR_CUDA, m);
}

#define CK(h, expr)                                   \
  do {                                                \
    cudaError_t e_ = (expr);                          \
    if (e_ != cudaSuccess) return cuda_fail(h, e_, #expr); \
  } while (0)

inline int prec_of(int precision) {
  return precision == GMRES_FP32_INNER ? P_FP32 : (precision == GMRES_BF16_BASIS ? P_BF16 : P_FP64);
}

inline size_t basis_elem(int prec) { return prec == P_FP64 ? 8 : (prec == P_FP32 ? 4 : 2); }

constexpr int kLdp = 144;  // >= 2 kMaxK + 1 (two dot sets), multiple of 16

// Entries of the coarse correction s' (FP64, then its FP32 copy right after): one per
// aggregate, or per column of the adaptive space (at most kMaxAdapt), plus one.
inline int sdefl_len(const gmres_s* h) { return (h->r > kMaxAdapt ? h->r : kMaxAdapt) + 1; }

// Lays out the control block for restart length ldh and returns the Ctl view.
inline gmres_status ensure_workspace(gmres_s* h, int m, int prec) {
  const int ldh = m > h->ldh ? m : h->ldh;
  // columns padded to 256 rows: the pipelined passes copy whole 256-row-aligned tiles,
  // and the padding rows stay zero (never written after this memset)
  const long long ldv = ((long long)h->n + 255) / 256 * 256;
  const int max_grid = h->sms * 8;
  if (ldh != h->ldh || prec != h->prec_ws) {
    const size_t vbytes = basis_elem(prec) * (size_t)ldv * (ldh + 1);
    CK(h, h->V.ensure(vbytes));
    CK(h, cudaMemsetAsync(h->V.p, 0, vbytes, h->stream));
    const size_t nd = 2 * (size_t)(ldh + 1) * ldh + 8 * (size_t)(ldh + 1);
    CK(h, h->dctl.ensure(sizeof(double) * nd));
    h->ldh = ldh;
    h->prec_ws = prec;
    h->ldv = ldv;
  }
  if (!h->w.p) {
    CK(h, h->w.ensure(sizeof(double) * (size_t)ldv));
    CK(h, cudaMemsetAsync(h->w.p, 0, sizeof(double) * (size_t)ldv, h->stream));
  }
  CK(h, h->t.ensure(sizeof(double) * (size_t)ldv));
  CK(h, h->part.ensure(sizeof(double) * (size_t)max_grid * kLdp));
  CK(h, h->part2.ensure(sizeof(double) * (size_t)kMaxGroups * kLdp));
  if (!h->tickets.p) {
    CK(h, h->tickets.ensure(sizeof(unsigned) * (1 + kMaxGroups)));
    CK(h, cudaMemsetAsync(h->tickets.p, 0, sizeof(unsigned) * (1 + kMaxGroups), h->stream));
  }
  CK(h, h->cpart.ensure(sizeof(double) * (size_t)(h->npieces + 1)));
  CK(h, h->sdefl.ensure(12 * (size_t)sdefl_len(h)));
  CK(h, h->gbar.ensure(4 * sizeof(unsigned)));
  if (h->opts.ortho == GMRES_ORTHO_MGS_LOWSYNC)
    CK(h, h->lmat.ensure(sizeof(double) * (size_t)kMaxK * kMaxK));
  if ((h->opts.deflation_mode == GMRES_DEFL_ADAPTIVE || h->dense_r > 0) && !h->aU.p) {
    const size_t col = sizeof(double) * (size_t)ldv;
    const size_t R = (size_t)h->opts.rmax;
    CK(h, h->aU.ensure(col * R));
    CK(h, h->aAU.ensure(col * R));
    CK(h, h->au.ensure(col));
    CK(h, cudaMemsetAsync(h->aU.p, 0, col * R, h->stream));
    CK(h, cudaMemsetAsync(h->aAU.p, 0, col * R, h->stream));
    CK(h, cudaMemsetAsync(h->au.p, 0, col, h->stream));
    CK(h, h->aT.ensure(sizeof(double) * R * R));
    CK(h, h->aTinv.ensure(sizeof(double) * R * R));
    CK(h, h->asmall.ensure(sizeof(double) * (2 * kMaxK + 2 * (kMaxAdapt + 1) + 2 +
                                             kMaxAdapt * kMaxAdapt) +
                           (4 + kMaxAdapt) * sizeof(int)));
  }
  CK(h, h->meta.ensure(sizeof(Meta)));
  if (!h->hmeta) CK(h, cudaMallocHost(&h->hmeta, sizeof(Meta)));
  if (!h->ev0) CK(h, cudaEventCreate(&h->ev0));
  if (!h->ev1) CK(h, cudaEventCreate(&h->ev1));
  return GMRES_OK;
}

inline Ctl make_ctl(gmres_s* h) {
  Ctl c{};
  const int ldh = h->ldh;
  double* d = h->dctl.as<double>();
  c.H = d;
  d += (size_t)(ldh + 1) * ldh;
  c.Hr = d;
  d += (size_t)(ldh + 1) * ldh;
  c.g = d; d += ldh + 1;
  c.cs = d; d += ldh + 1;
  c.sn = d; d += ldh + 1;
  c.y = d; d += ldh + 1;
  c.sigma = d; d += ldh + 1;
  c.h = d; d += ldh + 1;
  c.coef = d;
  Meta* m = h->meta.as<Meta>();
  c.scal = m->scal;
  c.counts = m->counts;
  c.flags = m->flags;
  c.ticket = h->tickets.as<unsigned>();
  c.part = h->part.as<double>();
  c.part2 = h->part2.as<double>();
  c.cpart = h->cpart.as<double>();
  c.sdefl = h->sdefl.as<double>();
  c.sdefl32 = reinterpret_cast<float*>(h->sdefl.as<double>() + sdefl_len(h));
  c.ldh = ldh;
  c.ldp = kLdp;
  c.L = h->lmat.as<double>();
  return c;
}

// Diagonal storage of operator o when it has at most kMaxDiag distinct diagonals and they
// are at least 80 % filled (the Q1 stencils: 9 diagonals, 99.6 % filled); otherwise the
// CSR kernels are used.
inline gmres_status build_dia(gmres_s* h, OpHost& o) {
  cudaStream_t st = h->stream;
  const int n = h->n;
  o.dia.nd = 0;
  DevMem slots;
  CK(h, slots.ensure(sizeof(int) * 65));
  int* sl = slots.as<int>();
  CK(h, launch_dia_detect(n, o.rowptr.as<int>(), o.col.as<int>(), sl, sl + 64, st));
  int hs[65];
  CK(h, cudaMemcpyAsync(hs, sl, sizeof(hs), cudaMemcpyDeviceToHost, st));
  CK(h, cudaStreamSynchronize(st));
  if (hs[64] > kMaxDiag || hs[64] < 1) return GMRES_OK;
  DiaOffsets offs{};
  for (int i = 0; i < 64; ++i)
    if (hs[i] != dia_empty_slot()) offs.off[offs.nd++] = hs[i];
  std::sort(offs.off, offs.off + offs.nd);
  if ((double)h->nnz < 0.8 * (double)offs.nd * (double)n) return GMRES_OK;
  // rows padded to 256 (kernels copy whole 256-row-aligned tiles of the diagonals)
  const long long ldd = ((long long)n + 255) / 256 * 256;
  const size_t cnt = (size_t)offs.nd * (size_t)ldd;
  CK(h, o.dval.ensure(sizeof(double) * cnt));
  CK(h, cudaMemsetAsync(o.dval.p, 0, sizeof(double) * cnt, st));
  const bool f32 = h->opts.precision != GMRES_FP64;
  if (f32) {
    CK(h, o.dval32.ensure(sizeof(float) * cnt));
    CK(h, cudaMemsetAsync(o.dval32.p, 0, sizeof(float) * cnt, st));
  }
  CK(h, launch_dia_fill(n, o.rowptr.as<int>(), o.col.as<int>(), o.val.as<double>(), offs, ldd,
                        o.dval.as<double>(), f32 ? o.dval32.as<float>() : nullptr, st));
  CK(h, cudaStreamSynchronize(st));
  o.dia = offs;
  o.ldd = ldd;
  return GMRES_OK;
}

// A W of operator o in CSR (count, scan, fill; one host read of the entry count)
inline gmres_status build_au(gmres_s* h, OpHost& o) {
  cudaStream_t st = h->stream;
  const int n = h->n;
  DevMem cnt, bsum;
  CK(h, cnt.ensure(sizeof(int) * (size_t)n));
  CK(h, bsum.ensure(sizeof(int) * (size_t)(au_scan_blocks(n) + 1)));
  // row pointers padded past n up to whole 256-row tiles (+ 8): tile copies stay defined
  const long long ptot = ((long long)n + 255) / 256 * 256 + 8;
  CK(h, o.aurp.ensure(sizeof(int) * (size_t)ptot));
  CK(h, launch_au_rows(n, o.rowptr.as<int>(), o.col.as<int>(), h->agg.as<int>(), cnt.as<int>(),
                       bsum.as<int>(), o.aurp.as<int>(), st));
  CK(h, launch_au_tiles(n, ptot, 256, o.aurp.as<int>(), bsum.as<int>(), st));
  int hv[2] = {0, 0};
  CK(h, cudaMemcpyAsync(&hv[0], o.aurp.as<int>() + n, sizeof(int), cudaMemcpyDeviceToHost, st));
  CK(h, cudaMemcpyAsync(&hv[1], bsum.as<int>(), sizeof(int), cudaMemcpyDeviceToHost, st));
  CK(h, cudaStreamSynchronize(st));
  const int nau = hv[0];
  o.nau = nau;
  o.au_tile_max = hv[1];
  // 8 entries of slack: tile copies round their range out to 16-byte boundaries
  const size_t cap = (size_t)nau + 8;
  CK(h, o.aucol.ensure(sizeof(int) * cap));
  CK(h, o.auval.ensure(sizeof(double) * cap));
  if (h->opts.precision != GMRES_FP64) CK(h, o.auval32.ensure(sizeof(float) * cap));
  CK(h, launch_au_fill(n, o.rowptr.as<int>(), o.col.as<int>(), o.val.as<double>(),
                       h->agg.as<int>(), o.aurp.as<int>(), o.aucol.as<int>(),
                       o.auval.as<double>(),
                       h->opts.precision != GMRES_FP64 ? o.auval32.as<float>() : nullptr, st));
  const bool f32 = h->opts.precision != GMRES_FP64;
  CK(h, o.aup_col.ensure(sizeof(int) * 2 * (size_t)n));
  CK(h, o.aup_val.ensure(sizeof(double) * 2 * (size_t)n));
  if (f32) CK(h, o.aup_val32.ensure(sizeof(float) * 2 * (size_t)n));
  CK(h, launch_au_planes(n, o.aurp.as<int>(), o.aucol.as<int>(), o.auval.as<double>(),
                         f32 ? o.auval32.as<float>() : nullptr, o.aup_col.as<int>(),
                         o.aup_val.as<double>(), f32 ? o.aup_val32.as<float>() : nullptr, st));
  if (h->opts.deflation_mode == GMRES_DEFL_EBP) {
    const long long nnz = h->nnz;
    CK(h, o.xrp.ensure(sizeof(int) * (size_t)(n + 1)));
    CK(h, o.xcol.ensure(sizeof(int) * (size_t)(nnz + nau)));
    CK(h, o.xval.ensure(sizeof(double) * (size_t)(nnz + nau)));
    if (f32) CK(h, o.xval32.ensure(sizeof(float) * (size_t)(nnz + nau)));
    CK(h, launch_ext_csr(n, o.rowptr.as<int>(), o.col.as<int>(), o.val.as<double>(),
                         f32 ? o.val32.as<float>() : nullptr, o.aurp.as<int>(),
                         o.aucol.as<int>(), o.auval.as<double>(),
                         f32 ? o.auval32.as<float>() : nullptr, o.xrp.as<int>(),
                         o.xcol.as<int>(), o.xval.as<double>(),
                         f32 ? o.xval32.as<float>() : nullptr, st));
  }
  CK(h, cudaStreamSynchronize(st));
  return GMRES_OK;
}

inline OpDev make_op(gmres_s* h, OpHost& o) {
  OpDev op{};
  op.n = h->n;
  op.rowptr = o.rowptr.as<int>();
  op.col = o.col.as<int>();
  op.val = o.val.as<double>();
  op.val32 = o.val32.as<float>();
  op.defl.r = h->r;
  op.defl.agg = h->agg.as<int>();
  op.defl.perm = h->perm.as<int>();
  op.defl.piece_start = h->piece_start.as<int>();
  op.defl.agg_piece = h->agg_piece.as<int>();
  op.defl.uscale = h->uscale.as<double>();
  op.defl.tinv = o.tinv.as<double>();
  op.defl.tinv32 = o.tinv32.as<float>();
  op.defl.npieces = h->npieces;
  op.defl.blk_piece_start = h->blk_piece_start.as<int>();
  op.defl.blk_piece = h->blk_piece.as<int>();
  op.defl.blk_grid = h->blk_grid;
  op.defl.aurp = o.aurp.as<int>();
  op.defl.aucol = o.aucol.as<int>();
  op.defl.auval = o.auval.as<double>();
  op.defl.auval32 = o.auval32.as<float>();
  op.defl.aup_col = o.aup_col.as<int>();
  op.defl.aup_val = o.aup_val.as<double>();
  op.defl.aup_val32 = o.aup_val32.as<float>();
  op.dia = o.dia;
  op.ldd = o.ldd;
  op.dval = o.dval.as<double>();
  op.dval32 = o.dval32.as<float>();
  op.xrp = o.xrp.as<int>();
  op.xcol = o.xcol.as<int>();
  op.xval = o.xval.as<double>();
  op.xval32 = o.xval32.as<float>();
  op.vec = (o.dia.nd == 0 && h->nnz >= (long long)kVecMinRowLen * h->n) ? kVecLanes : 0;
  op.au_tile_max = o.au_tile_max;
  return op;
}

inline gmres_status read_meta(gmres_s* h) {
  CK(h, cudaMemcpyAsync(h->hmeta, h->meta.p, sizeof(Meta), cudaMemcpyDeviceToHost, h->stream));
  CK(h, cudaStreamSynchronize(h->stream));
  return GMRES_OK;
}


namespace gg {
// batch.cu
gmres_status batch_solve_impl(int count, gmres_t const* hs, const double* const* b,
                              const double* const* x0, int m, double tol, long long maxit,
                              double* const* x, gmres_info* infos, cudaStream_t st,
                              long long* launches);
void batch_forget(gmres_t h);
// after a restart cycle: grows the adaptive deflation space (adaptive.cu)
// U, A U, T and T^-1 of a handle from its dense columns W (first solve only)
gmres_status dense_build(gmres_s* h, CycleArgs& a);
gmres_status adapt_update(gmres_s* h, CycleArgs& a);

}  // namespace gg
