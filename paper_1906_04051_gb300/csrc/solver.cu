// solver.cu -- C ABI of the library: handle lifetime, setup orchestration and the
// restart / refinement driver of deflated GMRES(m) (Sec. 3.2-3.3).
//
// The driver enqueues one restart cycle at a time (m Arnoldi steps, the cycle end and
// the true residual) and reads back a 272-byte status block once per cycle; every
// decision inside a cycle (Givens, stopping tests, breakdown) is taken on the device, so
// steps after an early exit return at once.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "handle.h"

thread_local std::string g_create_error;

namespace {

// Starts a profiled segment of phase ph (no-op unless profiling is on).
cudaError_t prof_mark(gmres_s* h, int ph) {
  if (!h->prof_on) return cudaSuccess;
  if (h->pused == (int)h->pev.size()) {
    cudaEvent_t e;
    cudaError_t err = cudaEventCreate(&e);
    if (err != cudaSuccess) return err;
    h->pev.push_back(e);
    h->pph.push_back(-1);
  }
  cudaError_t err = cudaEventRecord(h->pev[h->pused], h->stream);
  h->pph[h->pused] = ph;
  ++h->pused;
  return err;
}

// After a stream synchronisation: adds the closed segments to the phase totals and keeps
// the last event open as the start of the next segment.
void prof_flush(gmres_s* h, bool close) {
  if (!h->prof_on || h->pused == 0) return;
  for (int i = 0; i + 1 < h->pused; ++i) {
    float ms = 0.f;
    if (h->pph[i] >= 0 && cudaEventElapsedTime(&ms, h->pev[i], h->pev[i + 1]) == cudaSuccess)
      h->pms[h->pph[i]] += ms;
  }
  if (close) {
    h->pused = 0;
    return;
  }
  std::swap(h->pev[0], h->pev[h->pused - 1]);
  h->pph[0] = h->pph[h->pused - 1];
  h->pused = 1;
}

cudaError_t phase(gmres_s* h, const CycleArgs& a, int ph, int j, bool defl, double* x,
                  const double* b) {
  cudaError_t e = prof_mark(h, ph);
  if (e != cudaSuccess) return e;
  int nl = 0;
  e = launch_phase(a, ph, j, defl, x, b, h->stream, &nl);
  h->plaunch[ph] += nl;
  return e;
}

gmres_status run(gmres_s* h, OpHost& o, const double* b, const double* x0, int m, double tol,
                 long long maxit, double* x, gmres_info* info) {
  if (!b || !x) return fail(h, GMRES_ERR_INVALID_ARG, "b and x must be device pointers");
  if (m < 1 || m > kMaxM) return fail(h, GMRES_ERR_INVALID_ARG, "m must be in [1, 64]");
  if (!(tol >= 0.0) || maxit < 0) return fail(h, GMRES_ERR_INVALID_ARG, "tol >= 0, maxit >= 0");
  const int prec = prec_of(h->opts.precision);
  gmres_status s = ensure_workspace(h, m, prec);
  if (s != GMRES_OK) return s;
  cudaStream_t st = h->stream;
  const size_t nb = sizeof(double) * (size_t)h->n;
  if (x != x0) {
    if (x0) CK(h, cudaMemcpyAsync(x, x0, nb, cudaMemcpyDeviceToDevice, st));
    else CK(h, cudaMemsetAsync(x, 0, nb, st));
  }
  CycleArgs a{};
  a.op = make_op(h, o);
  a.ctl = make_ctl(h);
  a.V = h->V.p;
  a.ldv = h->ldv;
  a.w = h->w.p;
  a.t = h->t.as<double>();
  a.prec = prec;
  a.m = m;
  a.sms = h->sms;
  a.grid_small = h->r > 0 ? grid_for(h->r, 8, h->sms) : 1;
  a.pdl = h->prof_on ? 0 : 1;  // per-phase events would serialise the launches anyway
  a.proj = (h->r > 0 && h->opts.deflation_mode == GMRES_DEFL_PROJECTOR) ? 1 : 0;
  a.ortho = h->opts.ortho;
  a.dot_arith = h->opts.dot_arith;
  a.gbar = h->gbar.as<unsigned>();
  const bool mgs = a.ortho == GMRES_ORTHO_MGS;
  if (mgs) {
    if (mgs_rows(h->n, h->sms) == 0)
      return fail(h, GMRES_ERR_INVALID_ARG, "GMRES_ORTHO_MGS: n exceeds 220 KiB of w per SM");
    CK(h, cudaMemsetAsync(h->gbar.p, 0, 4 * sizeof(unsigned), st));
  }

  const bool ebp = h->r > 0 && h->opts.deflation_mode == GMRES_DEFL_EBP;
  const bool ada = h->opts.deflation_mode == GMRES_DEFL_ADAPTIVE;  // U grows from empty
  const bool dw = h->dense_r > 0;  // U from the caller's dense columns, fixed
  if (ada) h->aq = 0;
  // the whole step in one persistent kernel where it applies (fused.cu)
  const bool fused = !mgs && !ada && !dw && arnoldi_fusable(a);
  if (fused) CK(h, cudaMemsetAsync(h->gbar.p, 0, 4 * sizeof(unsigned), st));
  const int mu_mode = h->opts.mu_mode;
  double mu = 0.0;
  if (mu_mode == GMRES_MU_USER) mu = std::fabs(h->opts.mu_user);
  if (mu_mode == GMRES_MU_NORM_INF) mu = h->mu_norminf;
  const bool mixed = prec != P_FP64;
  double inner_tol = h->opts.inner_tol;
  if (!(inner_tol > 0.0)) inner_tol = prec == P_BF16 ? 1e-2 : 1e-4;
  const auto t_start = std::chrono::steady_clock::now();

  CK(h, cudaEventRecord(h->ev0, st));
  CK(h, launch_init(a, tol, inner_tol, h->opts.r0_norm_ref, mu, h->opts.fixed_iterations ? 1 : 0,
                    mixed ? 1 : 0, maxit, st));
  h->plaunch[PH_RESIDUAL] += 1;  // the init kernel is counted with the first residual
  if (dw && !h->dense_built) {  // U, A U, T, T^-1 from W, once per handle
    s = dense_build(h, a);
    if (s != GMRES_OK) return s;
    h->dense_built = true;
  }
  CK(h, phase(h, a, PH_RESIDUAL, 0, false, x, b));
  s = read_meta(h);
  if (s != GMRES_OK) return s;
  prof_flush(h, false);
  int cycle = 0;
  gmres_status status = GMRES_OK;
  while (!h->hmeta->flags[F_STOP]) {
    const bool mu_known = mu_mode != GMRES_MU_RITZ_FIRST_CYCLE || cycle > 0;
    const bool defl_cycle = (ebp || ((ada || dw) && h->aq > 0)) && mu_known;
    if (ada || dw) {  // this cycle's dense deflation space (adaptive: empty at first)
      a.op.defl.ud = h->aU.as<double>();
      a.op.defl.aud = h->aAU.as<double>();
      a.op.defl.tinv_a = h->aTinv.as<double>();
      a.op.defl.ldu = h->ldv;
      a.op.defl.qd = defl_cycle ? h->aq : 0;
    }
    if (defl_cycle) CK(h, phase(h, a, PH_DEFL, 0, true, x, b));
    const long long left = maxit - h->hmeta->counts[C_STEPS];
    const int jmax = (int)(left < m ? left : m);
    // the whole cycle in one launch where the step fuses; each step's coarse solve for the
    // next step inside it
    if (fused && jmax > 0) CK(h, phase(h, a, PH_ARNOLDI, jmax, defl_cycle, x, b));
    for (int j = 0; j < (fused ? 0 : jmax); ++j) {
      CK(h, phase(h, a, PH_SPMV, j, defl_cycle, x, b));
      if (mgs) {
        CK(h, phase(h, a, PH_MGS, j, defl_cycle, x, b));
      } else if (a.ortho == GMRES_ORTHO_MGS_LOWSYNC) {  // pass 1 + solve, then pass 3
        CK(h, phase(h, a, PH_DOT1, j, defl_cycle, x, b));
        CK(h, phase(h, a, PH_UPD2NORM, j, defl_cycle, x, b));
      } else {
        CK(h, phase(h, a, PH_DOT1, j, defl_cycle, x, b));
        CK(h, phase(h, a, PH_UPD1DOT2, j, defl_cycle, x, b));
        CK(h, phase(h, a, PH_UPD2NORM, j, defl_cycle, x, b));
      }
      if (defl_cycle) CK(h, phase(h, a, PH_DEFL, j + 1, true, x, b));
    }
    CK(h, phase(h, a, PH_CYCLE_END, 0, defl_cycle, x, b));
    if ((ebp || ada || dw) && mu_mode == GMRES_MU_RITZ_FIRST_CYCLE && cycle == 0)
      CK(h, phase(h, a, PH_RITZ, 0, false, x, b));
    if (ada) {  // grow U from this cycle's H_k and basis (Sec. 3.3, Eq. 19)
      CK(h, prof_mark(h, PH_ADAPT));
      s = adapt_update(h, a);
      if (s != GMRES_OK) return s;
    }
    CK(h, phase(h, a, PH_RESIDUAL, 0, false, x, b));
    s = read_meta(h);
    if (s != GMRES_OK) return s;
    prof_flush(h, false);
    ++cycle;
    if (h->opts.timeout_ms > 0 && !h->hmeta->flags[F_STOP]) {
      const double ms = std::chrono::duration<double, std::milli>(
                            std::chrono::steady_clock::now() - t_start).count();
      if (ms > h->opts.timeout_ms) {
        status = fail(h, GMRES_ERR_TIMEOUT, "timeout_ms elapsed");
        break;
      }
    }
  }
  if (a.proj && status == GMRES_OK && h->hmeta->flags[F_STATUS] >= 0)
    CK(h, phase(h, a, PH_PROJ_FINAL, 0, false, x, b));
  CK(h, prof_mark(h, -1));
  CK(h, cudaEventRecord(h->ev1, st));
  CK(h, cudaEventSynchronize(h->ev1));
  float ms = 0.f;
  cudaEventElapsedTime(&ms, h->ev0, h->ev1);
  prof_flush(h, true);
  if (status == GMRES_OK) status = (gmres_status)h->hmeta->flags[F_STATUS];
  if (status == GMRES_ERR_NAN) h->err = "NaN or Inf in the residual or Hessenberg matrix";
  if (status == GMRES_ERR_SINGULAR_COARSE) h->err = "no usable Ritz estimate of mu";
  if (info) {
    info->iters = h->hmeta->counts[C_STEPS];
    info->cycles = h->hmeta->counts[C_CYCLES];
    info->refinements = h->hmeta->counts[C_REFINE];
    info->rel_res_est = h->hmeta->scal[S_EST];
    info->rel_res_true = h->hmeta->scal[S_TRUE];
    info->mu = (ebp || ada || dw) ? h->hmeta->scal[S_MU] : 0.0;
    info->ms_total = ms;
    info->status = status;
  }
  return status;
}

// ---------------------------------------------------------------------------------------
// Allocation-free solve.  The per-solve workspace (Krylov basis, working vectors, control
// block, reduction partials) lives in one file-scope device array instead of memory
// owned by the handle, so a successful call allocates nothing on the device or the host.
// It is meant for callers that must not allocate once set up: a real-time loop with a
// frozen memory budget, or a process whose device memory is owned by another allocator
// (a framework's caching allocator) where an extra cudaMalloc could fail or fragment.
// The handle (gmres_create, which does allocate) still holds A and the deflation data.
// ---------------------------------------------------------------------------------------
constexpr size_t kNoAllocBytes = (size_t)32 << 20;  // 32 MiB, held by every device that
                                                    // loads the library until exit
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

constexpr int kNoAllocMaxDevices = 64;
unsigned char* g_noalloc_ptr[kNoAllocMaxDevices] = {nullptr};
std::mutex g_noalloc_mu;  // guards g_noalloc_ptr (first calls from several host threads)

// Device address of the scratch array for the current device.  In host code the array's
// name is only a host-side stand-in, so the address is looked up once per device (with
// that device current) and cached.  This first lookup on a device is the only set-up
// step; make the first call on each device before any stream capture.  The cache is not
// invalidated by cudaDeviceReset, which is therefore not supported after that first call.
cudaError_t noalloc_scratch(unsigned char** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kNoAllocMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  if (!g_noalloc_ptr[dev]) {
    void* ptr = nullptr;
    e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_noalloc_ptr[dev] = static_cast<unsigned char*>(ptr);
  }
  *out = g_noalloc_ptr[dev];
  return cudaSuccess;
}

gmres_status run_noalloc(gmres_s* h, OpHost& o, const double* b, const double* x0, int m,
                         double tol, long long maxit, double* x, gmres_info* info) {
  if (!b || !x) return fail(h, GMRES_ERR_INVALID_ARG, "b and x must be device pointers");
  if (h->opts.deflation_mode == GMRES_DEFL_ADAPTIVE)
    return fail(h, GMRES_ERR_INVALID_ARG, "gmres_solve_noalloc: GMRES_DEFL_ADAPTIVE allocates its space");
  if (h->opts.ortho != GMRES_ORTHO_CGS2)
    return fail(h, GMRES_ERR_INVALID_ARG, "gmres_solve_noalloc: CGS2 only");
  if (h->dense_r > 0)
    return fail(h, GMRES_ERR_INVALID_ARG, "gmres_solve_noalloc: dense W allocates its space");
  if (m < 1 || m > kMaxM) return fail(h, GMRES_ERR_INVALID_ARG, "m must be in [1, 64]");
  if (!(tol >= 0.0) || maxit < 0) return fail(h, GMRES_ERR_INVALID_ARG, "tol >= 0, maxit >= 0");
  const int prec = prec_of(h->opts.precision);
  const long long ldv = ((long long)h->n + 255) / 256 * 256;
  const int max_grid = h->sms * 8;
  // carve the workspace out of the static array, 256-byte aligned pieces
  size_t off = 0;
  auto take = [&](size_t bytes) {
    const size_t at = off;
    off += (bytes + 255) / 256 * 256;
    return at;
  };
  const size_t oV = take(basis_elem(prec) * (size_t)ldv * (m + 1));
  const size_t oW = take(sizeof(double) * (size_t)ldv);
  const size_t oT = take(sizeof(double) * (size_t)ldv);
  const size_t oCtl = take(sizeof(double) * (2 * (size_t)(m + 1) * m + 8 * (size_t)(m + 1)));
  const size_t oMeta = take(sizeof(Meta));
  const size_t oPart = take(sizeof(double) * (size_t)max_grid * kLdp);
  const size_t oPart2 = take(sizeof(double) * (size_t)kMaxGroups * kLdp);
  const size_t oTick = take(sizeof(unsigned) * (1 + kMaxGroups));
  const size_t oCpart = take(sizeof(double) * (size_t)(h->npieces + 1));
  const size_t oSdefl = take(12 * (size_t)sdefl_len(h));
  if (off > kNoAllocBytes)
    return fail(h, GMRES_ERR_INVALID_ARG,
                "gmres_solve_noalloc: workspace of " + std::to_string(off) +
                    " bytes exceeds the 33554432-byte static scratch (about (m+1)*n basis "
                    "elements); use gmres_solve");
  unsigned char* base = nullptr;
  CK(h, noalloc_scratch(&base));
  cudaStream_t st = h->stream;
  // everything that must start at zero (the previous call's contents are otherwise kept):
  // ticket counters, and the basis and working vector, whose padding rows past n are read
  CK(h, cudaMemsetAsync(base + oTick, 0, sizeof(unsigned) * (1 + kMaxGroups), st));
  CK(h, cudaMemsetAsync(base + oV, 0, oW + sizeof(double) * (size_t)ldv - oV, st));
  const size_t nb = sizeof(double) * (size_t)h->n;
  if (x != x0) {
    if (x0) CK(h, cudaMemcpyAsync(x, x0, nb, cudaMemcpyDeviceToDevice, st));
    else CK(h, cudaMemsetAsync(x, 0, nb, st));
  }
  CycleArgs a{};
  a.op = make_op(h, o);
  Ctl& c = a.ctl;
  double* d = reinterpret_cast<double*>(base + oCtl);
  c.H = d; d += (size_t)(m + 1) * m;
  c.Hr = d; d += (size_t)(m + 1) * m;
  c.g = d; d += m + 1;
  c.cs = d; d += m + 1;
  c.sn = d; d += m + 1;
  c.y = d; d += m + 1;
  c.sigma = d; d += m + 1;
  c.h = d; d += m + 1;
  c.coef = d;
  Meta* meta = reinterpret_cast<Meta*>(base + oMeta);
  c.scal = meta->scal;
  c.counts = meta->counts;
  c.flags = meta->flags;
  c.ticket = reinterpret_cast<unsigned*>(base + oTick);
  c.part = reinterpret_cast<double*>(base + oPart);
  c.part2 = reinterpret_cast<double*>(base + oPart2);
  c.cpart = reinterpret_cast<double*>(base + oCpart);
  c.sdefl = reinterpret_cast<double*>(base + oSdefl);
  c.sdefl32 = reinterpret_cast<float*>(c.sdefl + sdefl_len(h));
  c.ldh = m;
  c.ldp = kLdp;
  c.L = nullptr;
  a.V = base + oV;
  a.ldv = ldv;
  a.w = base + oW;
  a.t = reinterpret_cast<double*>(base + oT);
  a.prec = prec;
  a.m = m;
  a.sms = h->sms;
  a.grid_small = h->r > 0 ? grid_for(h->r, 8, h->sms) : 1;
  a.pdl = h->prof_on ? 0 : 1;  // per-phase events would serialise the launches anyway
  a.proj = (h->r > 0 && h->opts.deflation_mode == GMRES_DEFL_PROJECTOR) ? 1 : 0;

  const bool ebp = h->r > 0 && h->opts.deflation_mode == GMRES_DEFL_EBP;
  const int mu_mode = h->opts.mu_mode;
  double mu = 0.0;
  if (mu_mode == GMRES_MU_USER) mu = std::fabs(h->opts.mu_user);
  if (mu_mode == GMRES_MU_NORM_INF) mu = h->mu_norminf;
  const bool mixed = prec != P_FP64;
  double inner_tol = h->opts.inner_tol;
  if (!(inner_tol > 0.0)) inner_tol = prec == P_BF16 ? 1e-2 : 1e-4;
  const auto t_start = std::chrono::steady_clock::now();
  Meta hm;  // status block read back into host stack memory
  auto read = [&]() -> gmres_status {
    CK(h, cudaMemcpyAsync(&hm, meta, sizeof(Meta), cudaMemcpyDeviceToHost, st));
    CK(h, cudaStreamSynchronize(st));
    return GMRES_OK;
  };
  CK(h, launch_init(a, tol, inner_tol, h->opts.r0_norm_ref, mu, h->opts.fixed_iterations ? 1 : 0,
                    mixed ? 1 : 0, maxit, st));
  CK(h, launch_phase(a, PH_RESIDUAL, 0, false, x, b, st, nullptr));
  gmres_status s = read();
  if (s != GMRES_OK) return s;
  int cycle = 0;
  gmres_status status = GMRES_OK;
  while (!hm.flags[F_STOP]) {
    const bool defl_cycle = ebp && (mu_mode != GMRES_MU_RITZ_FIRST_CYCLE || cycle > 0);
    if (defl_cycle) CK(h, launch_phase(a, PH_DEFL, 0, true, x, b, st, nullptr));
    const long long left = maxit - hm.counts[C_STEPS];
    const int jmax = (int)(left < m ? left : m);
    for (int j = 0; j < jmax; ++j) {
      CK(h, launch_phase(a, PH_SPMV, j, defl_cycle, x, b, st, nullptr));
      CK(h, launch_phase(a, PH_DOT1, j, defl_cycle, x, b, st, nullptr));
      CK(h, launch_phase(a, PH_UPD1DOT2, j, defl_cycle, x, b, st, nullptr));
      CK(h, launch_phase(a, PH_UPD2NORM, j, defl_cycle, x, b, st, nullptr));
      if (defl_cycle) CK(h, launch_phase(a, PH_DEFL, j + 1, true, x, b, st, nullptr));
    }
    CK(h, launch_phase(a, PH_CYCLE_END, 0, defl_cycle, x, b, st, nullptr));
    if (ebp && mu_mode == GMRES_MU_RITZ_FIRST_CYCLE && cycle == 0)
      CK(h, launch_phase(a, PH_RITZ, 0, false, x, b, st, nullptr));
    CK(h, launch_phase(a, PH_RESIDUAL, 0, false, x, b, st, nullptr));
    s = read();
    if (s != GMRES_OK) return s;
    ++cycle;
    if (h->opts.timeout_ms > 0 && !hm.flags[F_STOP]) {
      const double ms = std::chrono::duration<double, std::milli>(
                            std::chrono::steady_clock::now() - t_start).count();
      if (ms > h->opts.timeout_ms) {
        status = fail(h, GMRES_ERR_TIMEOUT, "timeout_ms elapsed");
        break;
      }
    }
  }
  if (a.proj && status == GMRES_OK && hm.flags[F_STATUS] >= 0) {
    CK(h, launch_phase(a, PH_PROJ_FINAL, 0, false, x, b, st, nullptr));
    CK(h, cudaStreamSynchronize(st));
  }
  if (status == GMRES_OK) status = (gmres_status)hm.flags[F_STATUS];
  if (status == GMRES_ERR_NAN) h->err = "NaN or Inf in the residual or Hessenberg matrix";
  if (status == GMRES_ERR_SINGULAR_COARSE) h->err = "no usable Ritz estimate of mu";
  if (info) {
    info->iters = hm.counts[C_STEPS];
    info->cycles = hm.counts[C_CYCLES];
    info->refinements = hm.counts[C_REFINE];
    info->rel_res_est = hm.scal[S_EST];
    info->rel_res_true = hm.scal[S_TRUE];
    info->mu = ebp ? hm.scal[S_MU] : 0.0;
    info->ms_total = (float)std::chrono::duration<double, std::milli>(
                         std::chrono::steady_clock::now() - t_start).count();
    info->status = status;
  }
  return status;
}

}  // namespace

extern "C" {

void gmres_opts_default(gmres_opts* o) {
  if (!o) return;
  std::memset(o, 0, sizeof(*o));
  o->precision = GMRES_FP64;
  o->deflation_mode = GMRES_DEFL_EBP;
  o->mu_mode = GMRES_MU_RITZ_FIRST_CYCLE;
  o->rmax = 20;
  o->ninv = 20;
}

gmres_status gmres_create(gmres_t* out, const gmres_csr* A, const gmres_defl* W,
                          const gmres_opts* o, void* stream) {
  if (!out || !A) return fail(nullptr, GMRES_ERR_INVALID_ARG, "null handle or matrix");
  *out = nullptr;
  if (A->n <= 0 || !A->rowptr || !A->col || !A->val || A->nnz < 0 || A->nnz >= (1LL << 31))
    return fail(nullptr, GMRES_ERR_INVALID_ARG, "invalid CSR description");
  const bool dense_w = W && W->r > 0 && W->dense;  // W as dense columns
  const int r = (W && W->r > 0 && !dense_w) ? W->r : 0;  // aggregates
  const int dr = dense_w ? W->r : 0;
  if (r > kMaxR) return fail(nullptr, GMRES_ERR_INVALID_ARG, "r exceeds 6144");
  if (r > 0 && !W->agg) return fail(nullptr, GMRES_ERR_INVALID_ARG, "agg is null");
  if (dense_w && W->agg)
    return fail(nullptr, GMRES_ERR_INVALID_ARG, "give W as aggregates or as dense columns, not both");
  if (dr > kMaxAdapt) return fail(nullptr, GMRES_ERR_INVALID_ARG, "dense W: r exceeds 32");
  gmres_opts opts;
  if (o) opts = *o;
  else gmres_opts_default(&opts);
  if (opts.precision < 0 || opts.precision > 2 || opts.deflation_mode < 0 ||
      opts.deflation_mode > 3 || opts.mu_mode < 0 || opts.mu_mode > 2 || opts.ortho < 0 ||
      opts.ortho > 2 || opts.dot_arith < 0 || opts.dot_arith > 1)
    return fail(nullptr, GMRES_ERR_INVALID_ARG, "invalid option value");
  if (opts.dot_arith == GMRES_DOT_DF32 &&
      (opts.precision != GMRES_FP64 || opts.ortho != GMRES_ORTHO_MGS_LOWSYNC))
    return fail(nullptr, GMRES_ERR_INVALID_ARG,
                "GMRES_DOT_DF32: FP64 solves with GMRES_ORTHO_MGS_LOWSYNC only");
  if (opts.ortho == GMRES_ORTHO_MGS && opts.precision != GMRES_FP64)
    return fail(nullptr, GMRES_ERR_INVALID_ARG, "GMRES_ORTHO_MGS is FP64 only");
  if (opts.ortho == GMRES_ORTHO_MGS_LOWSYNC && opts.precision == GMRES_BF16_BASIS)
    return fail(nullptr, GMRES_ERR_INVALID_ARG, "GMRES_ORTHO_MGS_LOWSYNC: FP64 or FP32 inner");
  if (dense_w && (opts.deflation_mode != GMRES_DEFL_EBP || opts.precision != GMRES_FP64))
    return fail(nullptr, GMRES_ERR_INVALID_ARG, "dense W: GMRES_DEFL_EBP and FP64 only");
  if (dense_w) opts.rmax = dr;  // the dense-space buffers hold exactly its columns
  if (opts.deflation_mode == GMRES_DEFL_ADAPTIVE) {
    if (r > 0 || dense_w)
      return fail(nullptr, GMRES_ERR_INVALID_ARG,
                  "GMRES_DEFL_ADAPTIVE builds U itself: pass no aggregates");
    if (opts.precision != GMRES_FP64)
      return fail(nullptr, GMRES_ERR_INVALID_ARG, "GMRES_DEFL_ADAPTIVE is FP64 only");
    if (opts.rmax < 1 || opts.rmax > kMaxAdapt || opts.ninv < 1 || opts.ninv > 1000)
      return fail(nullptr, GMRES_ERR_INVALID_ARG, "rmax must be in [1, 32], ninv in [1, 1000]");
  }

  gmres_s* h = new gmres_s();
  const auto t_setup = std::chrono::steady_clock::now();
  h->n = A->n;
  h->nnz = A->nnz;
  h->stream = static_cast<cudaStream_t>(stream);
  h->opts = opts;
  h->r = r;
  int dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&h->sms, cudaDevAttrMultiProcessorCount, dev);
  auto bail = [&](gmres_status s) {
    g_create_error = h->err;
    delete h;
    return s;
  };
#define CKC(expr)                                  \
  do {                                             \
    cudaError_t e_ = (expr);                       \
    if (e_ != cudaSuccess) return bail(cuda_fail(h, e_, #expr)); \
  } while (0)
  cudaStream_t st = h->stream;
  const int n = h->n;
  const long long nnz = h->nnz;
  CKC(h->fwd.rowptr.ensure(sizeof(int) * (size_t)(n + 1)));
  CKC(h->fwd.col.ensure(sizeof(int) * (size_t)nnz));
  CKC(h->fwd.val.ensure(sizeof(double) * (size_t)nnz));
  CKC(cudaMemcpyAsync(h->fwd.rowptr.p, A->rowptr, sizeof(int) * (size_t)(n + 1),
                      cudaMemcpyDeviceToDevice, st));
  CKC(cudaMemcpyAsync(h->fwd.col.p, A->col, sizeof(int) * (size_t)nnz, cudaMemcpyDeviceToDevice, st));
  CKC(cudaMemcpyAsync(h->fwd.val.p, A->val, sizeof(double) * (size_t)nnz,
                      cudaMemcpyDeviceToDevice, st));
  if (r > 0) {
    CKC(h->agg.ensure(sizeof(int) * (size_t)n));
    CKC(cudaMemcpyAsync(h->agg.p, W->agg, sizeof(int) * (size_t)n, cudaMemcpyDeviceToDevice, st));
  }
  if (dense_w) {
    h->dense_r = dr;
    CKC(h->wdense.ensure(sizeof(double) * (size_t)n * dr));
    CKC(cudaMemcpyAsync(h->wdense.p, W->dense, sizeof(double) * (size_t)n * dr,
                        cudaMemcpyDeviceToDevice, st));
  }
  DevMem err;
  CKC(err.ensure(sizeof(int) * 4));
  CKC(cudaMemsetAsync(err.p, 0, sizeof(int) * 4, st));
  CKC(launch_validate(n, nnz, h->fwd.rowptr.as<int>(), h->fwd.col.as<int>(),
                      r > 0 ? h->agg.as<int>() : nullptr, r, err.as<int>(), st));
  int herr[4] = {0, 0, 0, 0};
  int inv_launches = 0;  // kernels of the coarse inverse (band LU or Gauss-Jordan)
  CKC(cudaMemcpyAsync(herr, err.p, sizeof(herr), cudaMemcpyDeviceToHost, st));
  CKC(cudaStreamSynchronize(st));
  if (herr[0] & 1) return bail(fail(h, GMRES_ERR_INVALID_ARG, "CSR rows not sorted/in range"));
  if (herr[0] & 2) return bail(fail(h, GMRES_ERR_INVALID_ARG, "aggregate index out of range"));
  if (opts.precision != GMRES_FP64) {
    CKC(h->fwd.val32.ensure(sizeof(float) * (size_t)nnz));
    CKC(launch_to_float(nnz, h->fwd.val.as<double>(), h->fwd.val32.as<float>(), st));
  }
  if (r > 0) {
    const int nb = agg_chunks(n);
    DevMem counts, aggptr, cnt, T, G, fac;
    // the fused kernel's grid: min(units of kPartUnit rows of the padded columns, SMs); its
    // row ranges cut pieces too
    const long long units = ((long long)n + 255) / 256 * 256 / kPartUnit;
    const int bg = (int)std::min<long long>(units, h->sms);
    const long long max_pieces =
        std::min<long long>((long long)n / kPiece + r + 1 + (long long)(bg - 1) * r, (long long)n + r + 1);
    DevMem bcnt;
    CKC(bcnt.ensure(sizeof(int) * (size_t)bg));
    CKC(h->blk_piece_start.ensure(sizeof(int) * (size_t)(bg + 1)));
    CKC(h->blk_piece.ensure(sizeof(int) * (size_t)max_pieces));
    h->blk_grid = bg;
    CKC(counts.ensure(sizeof(int) * (size_t)nb * r));
    CKC(aggptr.ensure(sizeof(int) * (size_t)(r + 1)));
    CKC(cnt.ensure(sizeof(int) * (size_t)r));
    CKC(h->perm.ensure(sizeof(int) * (size_t)n));
    CKC(h->agg_piece.ensure(sizeof(int) * (size_t)(r + 1)));
    CKC(h->piece_start.ensure(sizeof(int) * (size_t)(max_pieces + 1)));
    CKC(h->uscale.ensure(sizeof(double) * (size_t)r));
    CKC(launch_agg_perm(n, r, h->agg.as<int>(), counts.as<int>(), aggptr.as<int>(),
                        cnt.as<int>(), h->perm.as<int>(), h->agg_piece.as<int>(),
                        h->piece_start.as<int>(), h->uscale.as<double>(), (int)units, bg,
                        bcnt.as<int>(), h->blk_piece_start.as<int>(), h->blk_piece.as<int>(),
                        err.as<int>(), st));
    CKC(T.ensure(sizeof(double) * (size_t)r * r));
    CKC(G.ensure(sizeof(double) * 2 * (size_t)r * r));
    CKC(fac.ensure(gj_aux_bytes(r)));
    CKC(h->fwd.tinv.ensure(sizeof(double) * (size_t)r * r));
    CKC(h->adj.tinv.ensure(sizeof(double) * (size_t)r * r));
    CKC(launch_coarse_T(r, h->fwd.rowptr.as<int>(), h->fwd.col.as<int>(),
                        h->fwd.val.as<double>(), h->agg.as<int>(), h->perm.as<int>(),
                        aggptr.as<int>(), h->uscale.as<double>(), T.as<double>(), st));
    CKC(launch_coarse_inverse(r, T.as<double>(), G.as<double>(), fac.p,
                              h->fwd.tinv.as<double>(), h->adj.tinv.as<double>(), err.as<int>(),
                              h->tband, &inv_launches, st));
    h->coarse_band = h->tband[2] ? h->tband[0] + h->tband[1] + 1 : 0;
    if (opts.precision != GMRES_FP64) {  // the FP32 coarse solve of the fused FP32 step
      CKC(h->fwd.tinv32.ensure(sizeof(float) * (size_t)r * r));
      CKC(h->adj.tinv32.ensure(sizeof(float) * (size_t)r * r));
      CKC(launch_to_float((long long)r * r, h->fwd.tinv.as<double>(), h->fwd.tinv32.as<float>(), st));
      CKC(launch_to_float((long long)r * r, h->adj.tinv.as<double>(), h->adj.tinv32.as<float>(), st));
    }
    int np = 0;
    CKC(cudaMemcpyAsync(&np, h->agg_piece.as<int>() + r, sizeof(int), cudaMemcpyDeviceToHost, st));
    CKC(cudaMemcpyAsync(herr, err.p, sizeof(herr), cudaMemcpyDeviceToHost, st));
    CKC(cudaStreamSynchronize(st));
    if (herr[0] & 4) return bail(fail(h, GMRES_ERR_SINGULAR_COARSE, "empty aggregate (zero column of W)"));
    if (herr[0] & 8) return bail(fail(h, GMRES_ERR_SINGULAR_COARSE, "T = U^T A U is singular"));
    h->npieces = np;
  }
  if (r > 0 && opts.deflation_mode != GMRES_DEFL_NONE) {
    const gmres_status s_au = build_au(h, h->fwd);
    if (s_au != GMRES_OK) return bail(s_au);
  }
  {
    const gmres_status s_dia = build_dia(h, h->fwd);
    if (s_dia != GMRES_OK) return bail(s_dia);
  }
  if (opts.mu_mode == GMRES_MU_NORM_INF) {
    DevMem mx;
    CKC(mx.ensure(sizeof(unsigned long long)));
    CKC(cudaMemsetAsync(mx.p, 0, sizeof(unsigned long long), st));
    CKC(launch_norm_inf(n, h->fwd.rowptr.as<int>(), h->fwd.val.as<double>(),
                        mx.as<unsigned long long>(), st));
    unsigned long long bits = 0;
    CKC(cudaMemcpyAsync(&bits, mx.p, sizeof(bits), cudaMemcpyDeviceToHost, st));
    CKC(cudaStreamSynchronize(st));
    std::memcpy(&h->mu_norminf, &bits, sizeof(double));
  }
  h->fwd.ready = true;
  h->prof_on = opts.profile != 0;
  h->pms[PH_SETUP] = std::chrono::duration<double, std::milli>(
                         std::chrono::steady_clock::now() - t_setup).count();
  // kernels enqueued by the setup: validation, FP32 copy, aggregate permutation (4),
  // coarse matrix, its inverse (band width + band LU + substitutions, or Gauss-Jordan), A W
  // (count, three scan passes, fill, planes), the rows [A | A W] (2), diagonal storage
  // (detect, fill), infinity norm
  h->plaunch[PH_SETUP] = 1 + (opts.precision != GMRES_FP64 ? 1 : 0) +
                         (r > 0 ? 4 + 1 + 1 + (long long)inv_launches : 0) +
                         (r > 0 && opts.precision != GMRES_FP64 ? 2 : 0) +
                         (r > 0 && opts.deflation_mode != GMRES_DEFL_NONE ? 6 : 0) +
                         (r > 0 && opts.deflation_mode == GMRES_DEFL_EBP ? 2 : 0) +
                         1 + (h->fwd.dia.nd > 0 ? 1 : 0) +
                         (opts.mu_mode == GMRES_MU_NORM_INF ? 1 : 0);
#undef CKC
  *out = h;
  return GMRES_OK;
}

gmres_status gmres_solve(gmres_t h, const double* b, const double* x0, int32_t m, double tol,
                         int64_t maxit, double* x, gmres_info* info) {
  if (!h) return fail(nullptr, GMRES_ERR_INVALID_ARG, "null handle");
  return run(h, h->fwd, b, x0, m, tol, maxit, x, info);
}

gmres_status gmres_solve_noalloc(gmres_t h, const double* b, const double* x0, int32_t m,
                                 double tol, int64_t maxit, double* x, gmres_info* info) {
  if (!h) return fail(nullptr, GMRES_ERR_INVALID_ARG, "null handle");
  return run_noalloc(h, h->fwd, b, x0, m, tol, maxit, x, info);
}

gmres_status gmres_adjoint_solve(gmres_t h, const double* g, const double* lam0, int32_t m,
                                 double tol, int64_t maxit, double* lam, gmres_info* info) {
  if (!h) return fail(nullptr, GMRES_ERR_INVALID_ARG, "null handle");
  if (h->dense_r > 0)
    return fail(h, GMRES_ERR_INVALID_ARG, "gmres_adjoint_solve: not with a dense W");
  if (!h->adj.ready) {
    cudaStream_t st = h->stream;
    const int n = h->n;
    const long long nnz = h->nnz;
    CK(h, h->adj.rowptr.ensure(sizeof(int) * (size_t)(n + 1)));
    CK(h, h->adj.col.ensure(sizeof(int) * (size_t)nnz));
    CK(h, h->adj.val.ensure(sizeof(double) * (size_t)nnz));
    DevMem scratch;
    CK(h, scratch.ensure(sizeof(int) * (size_t)(n + 1)));
    CK(h, launch_transpose(n, (int)nnz, h->fwd.rowptr.as<int>(), h->fwd.col.as<int>(),
                           h->fwd.val.as<double>(), h->adj.rowptr.as<int>(),
                           h->adj.col.as<int>(), h->adj.val.as<double>(), scratch.as<int>(), st));
    if (h->opts.precision != GMRES_FP64) {
      CK(h, h->adj.val32.ensure(sizeof(float) * (size_t)nnz));
      CK(h, launch_to_float(nnz, h->adj.val.as<double>(), h->adj.val32.as<float>(), st));
    }
    CK(h, cudaStreamSynchronize(st));
    if (h->r > 0 && h->opts.deflation_mode != GMRES_DEFL_NONE) {
      const gmres_status s_au = build_au(h, h->adj);
      if (s_au != GMRES_OK) return s_au;
    }
    const gmres_status s_dia = build_dia(h, h->adj);
    if (s_dia != GMRES_OK) return s_dia;
    h->adj.ready = true;
  }
  return run(h, h->adj, g, lam0, m, tol, maxit, lam, info);
}

gmres_status gmres_batch_solve(int32_t count, gmres_t const* hs, const double* const* b,
                               const double* const* x0, int32_t m, double tol, int64_t maxit,
                               double* const* x, gmres_info* infos, void* stream) {
  if (count < 0 || (count > 0 && (!hs || !b || !x)))
    return fail(nullptr, GMRES_ERR_INVALID_ARG, "invalid batch arguments");
  return gg::batch_solve_impl(count, hs, b, x0, m, tol, maxit, x, infos,
                              static_cast<cudaStream_t>(stream), nullptr);
}

gmres_status gmres_profile(gmres_t h, int32_t enable, int32_t reset, double* ms,
                           int64_t* launches) {
  if (!h) return fail(nullptr, GMRES_ERR_INVALID_ARG, "null handle");
  if (ms)
    for (int i = 0; i < PH_COUNT; ++i) ms[i] = h->pms[i];
  if (launches)
    for (int i = 0; i < PH_COUNT; ++i) launches[i] = h->plaunch[i];
  if (reset)
    for (int i = 0; i < PH_COUNT; ++i) {
      h->pms[i] = 0.0;
      h->plaunch[i] = 0;
    }
  if (enable >= 0) h->prof_on = enable != 0;
  return GMRES_OK;
}

gmres_status gmres_layout_query(gmres_t h, gmres_layout* out) {
  if (!h) return fail(nullptr, GMRES_ERR_INVALID_ARG, "null handle");
  if (!out) return fail(h, GMRES_ERR_INVALID_ARG, "gmres_layout_query: null output");
  std::memset(out, 0, sizeof(*out));
  out->n = h->n;
  out->nnz = h->nnz;
  out->r = h->r;
  out->npieces = h->npieces;
  out->ndiag = h->fwd.dia.nd;
  out->nau = h->fwd.nau;
  out->ldv = h->ldv;
  out->adapt_q = (h->opts.deflation_mode == GMRES_DEFL_ADAPTIVE || h->dense_r > 0) ? h->aq : 0;
  out->spmv_lanes = (h->fwd.dia.nd == 0 && h->nnz >= (long long)kVecMinRowLen * h->n) ? kVecLanes : 0;
  out->coarse_band = h->coarse_band;
  return GMRES_OK;
}

gmres_status gmres_adaptive_space(gmres_t h, int32_t* q, double* U, int64_t ldu, double* T) {
  if (!h) return fail(nullptr, GMRES_ERR_INVALID_ARG, "null handle");
  if (h->opts.deflation_mode != GMRES_DEFL_ADAPTIVE && h->dense_r == 0)
    return fail(h, GMRES_ERR_INVALID_ARG, "gmres_adaptive_space: the handle has no dense space");
  if (!q) return fail(h, GMRES_ERR_INVALID_ARG, "gmres_adaptive_space: null q");
  if (U && ldu < h->n) return fail(h, GMRES_ERR_INVALID_ARG, "gmres_adaptive_space: ldu < n");
  const int nq = h->aU.p ? h->aq : 0;
  *q = nq;
  if (nq == 0) return GMRES_OK;
  cudaStream_t st = h->stream;
  const size_t d = sizeof(double);
  if (U)
    CK(h, cudaMemcpy2DAsync(U, d * (size_t)ldu, h->aU.p, d * (size_t)h->ldv, d * (size_t)h->n, nq,
                            cudaMemcpyDeviceToDevice, st));
  if (T)
    CK(h, cudaMemcpy2DAsync(T, d * (size_t)nq, h->aT.p, d * (size_t)h->opts.rmax, d * (size_t)nq,
                            nq, cudaMemcpyDeviceToDevice, st));
  CK(h, cudaStreamSynchronize(st));
  return GMRES_OK;
}

gmres_status gmres_set_stream(gmres_t h, void* stream) {
  if (!h) return fail(nullptr, GMRES_ERR_INVALID_ARG, "null handle");
  h->stream = static_cast<cudaStream_t>(stream);
  return GMRES_OK;
}

const char* gmres_last_error(gmres_t h) {
  return h ? h->err.c_str() : g_create_error.c_str();
}

void gmres_destroy(gmres_t h) {
  if (!h) return;
  gg::batch_forget(h);
  if (h->stream) cudaStreamSynchronize(h->stream);
  else cudaDeviceSynchronize();
  if (h->hmeta) cudaFreeHost(h->hmeta);
  if (h->ev0) cudaEventDestroy(h->ev0);
  if (h->ev1) cudaEventDestroy(h->ev1);
  delete h;
}

int64_t q1_nnz(int32_t n) {
  if (n < 1) return 0;
  return 9LL * (n - 1) * (n - 1) + 4LL * n;
}

gmres_status q1_assemble(int32_t n, const double* kappa, double bx, double by, const double* f,
                         const double* u, int32_t* rowptr, int32_t* col, double* val, double* b,
                         void* stream) {
  if (n < 1 || !kappa || !f || !rowptr || !col || !val || !b)
    return fail(nullptr, GMRES_ERR_INVALID_ARG, "q1_assemble: invalid arguments");
  if (q1_nnz(n) >= (1LL << 31) || (long long)(n + 1) * (n + 1) >= (1LL << 31))
    return fail(nullptr, GMRES_ERR_INVALID_ARG, "q1_assemble: mesh too large for int32 CSR");
  cudaError_t e = launch_q1_assemble(n, kappa, bx, by, f, u, rowptr, col, val, b,
                                     static_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return cuda_fail(nullptr, e, "q1_assemble");
  return GMRES_OK;
}

gmres_status q1_kappa_grad(int32_t n, const double* lam, const double* x, double* grad,
                           void* stream) {
  if (n < 1 || !lam || !x || !grad)
    return fail(nullptr, GMRES_ERR_INVALID_ARG, "q1_kappa_grad: invalid arguments");
  cudaError_t e = launch_q1_kappa_grad(n, lam, x, grad, static_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return cuda_fail(nullptr, e, "q1_kappa_grad");
  return GMRES_OK;
}

}  // extern "C"
