// handle.h -- host-side state of a gmres_t handle and its workspace helpers, shared by
// the single-system driver (solver.cu) and the batched driver (batch.cu).
#pragma once

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
  DevMem rowptr, col, val, val32, tinv;
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
  double mu_norminf = 0.0;
  // workspace
  int ldh = 0, prec_ws = -1;
  long long ldv = 0;
  DevMem V, w, t, dctl, meta, part, part2, tickets, cpart, sdefl;
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

constexpr int kLdp = 80;  // >= kMaxK + 1, multiple of 16

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
  CK(h, h->sdefl.ensure(12 * (size_t)(h->r + 1)));
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
  c.sdefl32 = reinterpret_cast<float*>(h->sdefl.as<double>() + (h->r + 1));
  c.ldh = ldh;
  c.ldp = kLdp;
  return c;
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
  op.defl.npieces = h->npieces;
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
}  // namespace gg
