// batch.cu -- many independent deflated GMRES(m) solves in one CUDA-graph launch.
//
// Every phase kernel runs over a flattened list of row tiles drawn from all systems, so
// each launch spreads every system's work over all SMs (on GB300 one SM retires only two
// FP64 FMAs per clock: a system of 66k unknowns cannot be left to one SM).  Block b owns
// the contiguous tile range [b T / G, (b+1) T / G); it accumulates a system's partial sums
// over its tiles of that system and, when the system changes, stores them in the
// system's slot b - (first block touching the system).  The last block to fill a
// system's slots (per-system ticket) reduces them in slot order and runs the system's
// epilogue (projection coefficients, plane rotations, restart decision), so results are
// deterministic and no block waits on another.
//
// All systems advance in lock step through restart cycles; a system that converged or
// ended its cycle early is skipped by every tile of it.  The cycle's kernel sequence is
// captured once into the body of a conditional `while` graph node, and a last kernel sets
// the loop condition (any system still running), so the whole solve is one graph launch.
#include <algorithm>
#include <map>
#include <memory>

#include "handle.h"
#include "kernels.cuh"

namespace gg {

namespace {

struct BSys {
  int n;
  int tile0_s, ntile_s;  // 256-row tiles: SpMV, residual, x update
  int tile0_p, ntile_p;  // TR-row tiles: CGS2 passes
  int piece0;            // first global piece of the aggregate sums
  int ebp;               // EBP deflation configured
  int mu_mode;
  double mu_init;
  const int* rowptr;
  const int* col;
  const double* val;
  const float* val32;
  const double* b;
  double* x;
  void* V;
  long long ldv;
  void* w;
  double* t;
  Defl defl;
  Ctl ctl;
};

struct BTab {
  const BSys* sys;
  int count;
  const int* tile_sys_s;
  int T_s;
  const int* tile_sys_p;
  int T_p;
  const int* piece_sys;
  int P;
  int TR;
  int m;
};

// block range of a grid of G blocks over T tiles, and the block owning tile t
__device__ __forceinline__ int range_lo(int b, int G, int T) {
  return (int)(((long long)b * T) / G);
}
__device__ __forceinline__ int block_of(int t, int G, int T) {
  return (int)(((long long)t * G + G - 1) / T);
}

// Stores this block's ncols partial sums of system S in its slot; the last contributor
// reduces all slots (slot order) into tot and returns true.
__device__ bool sys_flush(const BSys& S, int t_first, int nt, int T, const double* sred,
                          int ncols, double* tot) {
  __shared__ unsigned s_last;
  const int G = gridDim.x;
  const int blo = block_of(t_first, G, T), bhi = block_of(t_first + nt - 1, G, T);
  const int nslots = bhi - blo + 1, slot = (int)blockIdx.x - blo;
  double* part = S.ctl.part;
  const int ldp = S.ctl.ldp;
  for (int c = threadIdx.x; c < ncols; c += blockDim.x) part[(size_t)slot * ldp + c] = sred[c];
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0)
    s_last = (atomicAdd(S.ctl.ticket, 1u) == (unsigned)nslots - 1u) ? 1u : 0u;
  __syncthreads();
  if (!s_last) return false;
  __threadfence();
  reduce_rows(part, nslots, ncols, ldp, tot);
  if (threadIdx.x == 0) *S.ctl.ticket = 0u;
  __syncthreads();
  return true;
}

// column sums of the warp-slice accumulators (eight slices, one per warp) with shuffles:
// flushes are rare (a few per block and kernel), so their FP64 cost does not matter
template <typename TACC>
__device__ void flush_cols(const TACC (&acc)[kSliceCols], int nw, int k, double* swarp,
                           double* sred) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
  for (int i = 0; i < kSliceCols; ++i)
    if (i < nw) {
      const double v = warp_sum((double)acc[i]);
      if (lane == 0) swarp[warp * kSliceCols + i] = v;
    }
  __syncthreads();
  for (int c = threadIdx.x; c < k; c += blockDim.x)
    sred[c] = swarp[(c % kSlices) * kSliceCols + c / kSlices];
  __syncthreads();
}

__device__ __forceinline__ bool sys_step_active(const BSys& S) {
  return !S.ctl.flags[F_CYCLE_DONE];
}
__device__ __forceinline__ bool sys_live(const BSys& S) { return !S.ctl.flags[F_STOP]; }

// ---------------------------------------------------------------------------------------
__global__ void kb_init(BTab tab, double tol, double inner_tol, int fixed, int mixed,
                        long long maxit) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= tab.count) return;
  Ctl ctl = tab.sys[s].ctl;
  init_ctl(ctl, tol, inner_tol, 0.0, tab.sys[s].mu_init, fixed, mixed, maxit);
  ctl.flags[F_DEFL_ON] =
      (tab.sys[s].ebp && tab.sys[s].mu_mode != GMRES_MU_RITZ_FIRST_CYCLE) ? 1 : 0;
}

// true residual (Eq. 15) of every live system, then its restart decision
template <typename TV>
__global__ void __launch_bounds__(kSpmvRows) kb_residual(BTab tab) {
  __shared__ double sval[kSpmvCap];
  __shared__ int scol[kSpmvCap];
  __shared__ double sbuf[kSpmvRows / 32];
  __shared__ double sred[2], tot[2];
  const int T = tab.T_s;
  const int lo = range_lo(blockIdx.x, gridDim.x, T), hi = range_lo(blockIdx.x + 1, gridDim.x, T);
  int t = lo;
  while (t < hi) {
    const int s = tab.tile_sys_s[t];
    const BSys& S = tab.sys[s];
    const int t_end = min(hi, S.tile0_s + S.ntile_s);
    if (!sys_live(S)) {
      t = t_end;
      continue;
    }
    double n1 = 0.0, n2 = 0.0;
    TV* V0 = static_cast<TV*>(S.V);
    for (; t < t_end; ++t) {
      const int r0 = (t - S.tile0_s) * kSpmvRows;
      double acc, accd;
      const double* x = S.x;
      spmv_tile<double, double, false>(S.n, r0, S.rowptr, S.col, S.val, sval, scol,
                                       [&](int c) { return __ldg(x + c); }, nullptr,
                                       (const double*)nullptr, acc, accd);
      const int row = r0 + threadIdx.x;
      if (row < S.n) {
        const double r = __ldg(S.b + row) - acc;
        n1 += r * r;
        if constexpr (sizeof(TV) == sizeof(double)) {
          V0[row] = r;
        } else {
          const TV st = st_round<TV>((float)r);
          V0[row] = st;
          const double sv = (double)to_f<TV>(st);
          n2 += sv * sv;
        }
      }
    }
    const double b1 = block_sum(n1, sbuf);
    const double b2 = (sizeof(TV) == sizeof(double)) ? b1 : block_sum(n2, sbuf);
    if (threadIdx.x == 0) {
      sred[0] = b1;
      sred[1] = b2;
    }
    __syncthreads();
    if (sys_flush(S, S.tile0_s, S.ntile_s, T, sred, 2, tot) && threadIdx.x == 0) {
      Ctl ctl = S.ctl;
      residual_decide(ctl, sqrt(tot[0]), sqrt(tot[1]));
    }
    __syncthreads();
  }
}

// w = A M^-1 v_j of every system still in its cycle
template <typename TA, typename TV, typename TACC>
__global__ void __launch_bounds__(kSpmvRows) kb_spmv(BTab tab, int j) {
  __shared__ TA sval[kSpmvCap];
  __shared__ int scol[kSpmvCap];
  const int T = tab.T_s;
  const int lo = range_lo(blockIdx.x, gridDim.x, T), hi = range_lo(blockIdx.x + 1, gridDim.x, T);
  for (int t = lo; t < hi; ++t) {
    const BSys& S = tab.sys[tab.tile_sys_s[t]];
    if (!sys_step_active(S)) continue;
    const int r0 = (t - S.tile0_s) * kSpmvRows;
    const TV* xj = static_cast<const TV*>(S.V) + (size_t)j * S.ldv;
    const TA* val;
    const TACC* sd;
    if constexpr (sizeof(TA) == sizeof(double)) val = S.val;
    else val = S.val32;
    if constexpr (sizeof(TACC) == sizeof(double)) sd = S.ctl.sdefl;
    else sd = S.ctl.sdefl32;
    const TACC sigma = (TACC)S.ctl.sigma[j];
    TACC acc, accd;
    auto xg = [&](int c) { return ld_as<TACC, TV>(xj + c); };
    if (S.ctl.flags[F_DEFL_ON])
      spmv_tile<TA, TACC, true>(S.n, r0, S.rowptr, S.col, val, sval, scol, xg, S.defl.agg, sd,
                                acc, accd);
    else
      spmv_tile<TA, TACC, false>(S.n, r0, S.rowptr, S.col, val, sval, scol, xg, nullptr, sd,
                                 acc, accd);
    const int row = r0 + threadIdx.x;
    if (row < S.n) static_cast<TACC*>(S.w)[row] = sigma * acc + accd;
  }
}

// ---- pipelined passes over the tiles of all systems (CGS2, one-reduction MGS) ---------
template <typename TV, typename TACC>
struct BRing {
  unsigned char* base;
  uint64_t* bars;
  int k, TR, S;
  size_t stage_bytes;
  __device__ TV* vt(int st) const { return reinterpret_cast<TV*>(base + (size_t)st * stage_bytes); }
  __device__ TACC* wt(int st) const {
    return reinterpret_cast<TACC*>(base + (size_t)st * stage_bytes + (size_t)k * TR * sizeof(TV));
  }
  // warp 0: tile t of system Sy into stage st; an idle system's tile completes the phase
  // with a plain arrival
  __device__ void issue(int st, const BSys& Sy, int t) const {
    const int lane = threadIdx.x & 31;
    if (!sys_step_active(Sy)) {
      if (lane == 0) mbar_arrive_expect_tx(&bars[st], 0);
      return;
    }
    const long long r0 = (long long)(t - Sy.tile0_p) * TR;
    const uint32_t vb = (uint32_t)(TR * sizeof(TV)), wb = (uint32_t)(TR * sizeof(TACC));
    if (lane == 0) mbar_arrive_expect_tx(&bars[st], (uint32_t)k * vb + wb);
    __syncwarp();
    const TV* V = static_cast<const TV*>(Sy.V);
    TV* dst = vt(st);
    for (int c = lane; c < k; c += 32)
      bulk_g2s(dst + (size_t)c * TR, V + (size_t)c * Sy.ldv + r0, vb, &bars[st]);
    if (lane == 0) bulk_g2s(wt(st), static_cast<const TACC*>(Sy.w) + r0, wb, &bars[st]);
  }
};

// Streams the block's tile range through the ring; calls begin(S) when a live system
// starts, body(st, S, r0) per tile and end(S) after its last tile in this block.
template <typename TV, typename TACC, typename FB, typename FT, typename FE>
__device__ bool bring_run(const BRing<TV, TACC>& R, const BTab& tab, FB&& begin, FT&& body,
                          FE&& end) {
  const int T = tab.T_p;
  const int lo = range_lo(blockIdx.x, gridDim.x, T), hi = range_lo(blockIdx.x + 1, gridDim.x, T);
  const int nt = hi - lo;
  if (threadIdx.x == 0) {
    for (int st = 0; st < R.S; ++st) mbar_init(&R.bars[st], 1);
    mbar_fence_init();
  }
  __syncthreads();
  if (threadIdx.x < 32)
    for (int i = 0; i < nt && i < R.S; ++i) R.issue(i, tab.sys[tab.tile_sys_p[lo + i]], lo + i);
  int cur = -1;
  bool ok = true;
  int i = 0;
  for (; i < nt; ++i) {
    const int t = lo + i;
    const int s = tab.tile_sys_p[t];
    const BSys& S = tab.sys[s];
    const int st = i % R.S;
    ok = __syncthreads_and(mbar_wait(&R.bars[st], (uint32_t)((i / R.S) & 1)));
    if (!ok) break;
    if (s != cur) {
      if (cur >= 0 && sys_step_active(tab.sys[cur])) end(tab.sys[cur]);
      cur = s;
      if (sys_step_active(S)) begin(S);
    }
    if (sys_step_active(S)) body(st, S, (long long)(t - S.tile0_p) * R.TR);
    __syncthreads();
    if (threadIdx.x < 32 && i + R.S < nt)
      R.issue(st, tab.sys[tab.tile_sys_p[lo + i + R.S]], lo + i + R.S);
  }
  if (!ok) {
    for (int q = i; q < nt && q < i + R.S; ++q) mbar_wait(&R.bars[q % R.S], (uint32_t)((q / R.S) & 1));
    if (threadIdx.x == 0)
      for (int s = 0; s < tab.count; ++s) {
        tab.sys[s].ctl.flags[F_STATUS] = GMRES_ERR_TIMEOUT;
        tab.sys[s].ctl.flags[F_STOP] = 1;
        tab.sys[s].ctl.flags[F_CYCLE_DONE] = 1;
      }
    return false;
  }
  if (cur >= 0 && sys_step_active(tab.sys[cur])) end(tab.sys[cur]);
  return true;
}

template <typename TV, typename TACC>
__global__ void __launch_bounds__(kThreads) kb_pass1(BTab tab, int k) {
  extern __shared__ __align__(128) unsigned char smraw[];
  __shared__ uint64_t bars[kMaxStages];
  __shared__ double swarp[kSlices * kSliceCols];
  __shared__ double sred[kMaxK], tot[kMaxK];
  const int TR = tab.TR;
  const size_t sb = ring_stage_bytes(k, TR, sizeof(TV), sizeof(TACC));
  const BRing<TV, TACC> R{smraw, bars, k, TR, ring_stages(sb), sb};
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nw = slice_cols(k, warp, kSlices);
  TACC acc[kSliceCols];
  auto begin = [&](const BSys&) {
#pragma unroll
    for (int i = 0; i < kSliceCols; ++i) acc[i] = 0;
  };
  auto body = [&](int st, const BSys&, long long) {
#define GG_B1(NW) tile_dot<NW, TV, TACC>(acc, R.vt(st), R.wt(st), TR, warp, lane)
    GG_SLICE_SWITCH(nw, GG_B1)
#undef GG_B1
  };
  auto end = [&](const BSys& S) {
    flush_cols(acc, nw, k, swarp, sred);
    if (sys_flush(S, S.tile0_p, S.ntile_p, tab.T_p, sred, k, tot)) {
      for (int c = threadIdx.x; c < k; c += blockDim.x) {
        const double hc = S.ctl.sigma[c] * tot[c];
        S.ctl.h[c] = hc;
        S.ctl.coef[c] = S.ctl.sigma[c] * hc;
      }
    }
    __syncthreads();
  };
  bring_run(R, tab, begin, body, end);
}

// One-reduction MGS (the paper's projections, Eq. 13, in the inverse compact WY form), pass
// 1: one sweep over the basis tiles gives g = V^T w and the dots of the newest column u_j
// (the tile's column k - 1, already in shared memory) with all columns; the system's last
// block stores g_c = sigma_c (v_c . w) in h and the new row of L, v_j . v_c = sigma_j
// sigma_c (u_j . u_c) for c < j.  FP64 and FP32 bases (the second multi-dot reads the tile's
// column as the accumulator type).
template <typename TV, typename TACC>
__global__ void __launch_bounds__(kThreads) kb_pass1_icwy(BTab tab, int k) {
  static_assert(sizeof(TV) == sizeof(TACC), "u_j is read from the tile as TACC");
  extern __shared__ __align__(128) unsigned char smraw[];
  __shared__ uint64_t bars[kMaxStages];
  __shared__ double swarp[kSlices * kSliceCols];
  __shared__ double sred[2 * kMaxK], tot[2 * kMaxK];
  const int TR = tab.TR;
  const size_t sb = ring_stage_bytes(k, TR, sizeof(TV), sizeof(TACC));
  const BRing<TV, TACC> R{smraw, bars, k, TR, ring_stages(sb), sb};
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nw = slice_cols(k, warp, kSlices);
  TACC acc[kSliceCols], acc2[kSliceCols];
  auto begin = [&](const BSys&) {
#pragma unroll
    for (int i = 0; i < kSliceCols; ++i) acc[i] = acc2[i] = 0;
  };
  auto body = [&](int st, const BSys&, long long) {
#define GG_B1I(NW)                                                                        \
  {                                                                                       \
    tile_dot<NW, TV, TACC>(acc, R.vt(st), R.wt(st), TR, warp, lane);                      \
    tile_dot<NW, TV, TACC>(acc2, R.vt(st), (const TACC*)(R.vt(st) + (size_t)(k - 1) * TR), \
                           TR, warp, lane);                                               \
  }
    GG_SLICE_SWITCH(nw, GG_B1I)
#undef GG_B1I
  };
  auto end = [&](const BSys& S) {
    flush_cols(acc, nw, k, swarp, sred);
    flush_cols(acc2, nw, k, swarp, sred + k);
    if (sys_flush(S, S.tile0_p, S.ntile_p, tab.T_p, sred, 2 * k, tot)) {
      const double sj = S.ctl.sigma[k - 1];
      for (int c = threadIdx.x; c < k; c += blockDim.x) {
        S.ctl.h[c] = S.ctl.sigma[c] * tot[c];
        if (c < k - 1) S.ctl.L[(size_t)(k - 1) * kMaxK + c] = sj * S.ctl.sigma[c] * tot[k + c];
      }
    }
    __syncthreads();
  };
  bring_run(R, tab, begin, body, end);
}

// One-reduction MGS, the solve, a block per system in its cycle: (I + L) h = g by forward
// substitution in one warp (L staged in shared memory), then coef_c = sigma_c h_c for the
// update pass
__global__ void __launch_bounds__(256) kb_icwy_solve(BTab tab, int k) {
  __shared__ double sL[kMaxK * kMaxK];
  const BSys& S = tab.sys[blockIdx.x];
  if (!sys_step_active(S)) return;
  const Ctl& ctl = S.ctl;
  for (int t = threadIdx.x; t < k * k; t += blockDim.x) {
    const int i = t / k, c = t % k;
    sL[i * kMaxK + c] = c < i ? ctl.L[(size_t)i * kMaxK + c] : 0.0;
  }
  __syncthreads();
  if (threadIdx.x >= 32) return;
  const int lane = threadIdx.x;
  double g[3];
#pragma unroll
  for (int q = 0; q < 3; ++q) g[q] = lane + 32 * q < k ? ctl.h[lane + 32 * q] : 0.0;
  for (int c = 0; c < k; ++c) {
    const double hc = __shfl_sync(0xffffffffu, c < 32 ? g[0] : (c < 64 ? g[1] : g[2]), c & 31);
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      const int i = lane + 32 * q;
      if (i > c && i < k) g[q] -= sL[i * kMaxK + c] * hc;
    }
  }
#pragma unroll
  for (int q = 0; q < 3; ++q) {
    const int i = lane + 32 * q;
    if (i < k) {
      ctl.h[i] = g[q];
      ctl.coef[i] = ctl.sigma[i] * g[q];
    }
  }
}

template <typename TV, typename TACC>
__global__ void __launch_bounds__(kThreads) kb_pass2(BTab tab, int k) {
  constexpr int VN = Vec<TV>::n;
  extern __shared__ __align__(128) unsigned char smraw[];
  __shared__ uint64_t bars[kMaxStages];
  __shared__ double swarp[kSlices * kSliceCols];
  __shared__ double sred[kMaxK], tot[kMaxK];
  __shared__ TACC scoef[kMaxK];
  __shared__ __align__(16) TACC spart[4 * 256];
  __shared__ __align__(16) TACC sw2[256];
  const int TR = tab.TR;
  const size_t sb = ring_stage_bytes(k, TR, sizeof(TV), sizeof(TACC));
  const BRing<TV, TACC> R{smraw, bars, k, TR, ring_stages(sb), sb};
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nw = slice_cols(k, warp, kSlices);
  const int P = update_splits<TACC>(TR, VN), ng = TR / VN;
  TACC acc[kSliceCols];
  auto begin = [&](const BSys& S) {
#pragma unroll
    for (int i = 0; i < kSliceCols; ++i) acc[i] = 0;
    for (int c = threadIdx.x; c < k; c += blockDim.x) scoef[c] = (TACC)S.ctl.coef[c];
    __syncthreads();
  };
  auto body = [&](int st, const BSys& S, long long r0) {
    const TV* sV = R.vt(st);
    const TACC* sw = R.wt(st);
    tile_update<TV, TACC>(sV, TR, k, scoef, spart, P);
    __syncthreads();
    if ((int)threadIdx.x < ng) {
      const int r = threadIdx.x * VN;
      TACC* w = static_cast<TACC*>(S.w);
      TACC wn[VN];
      tile_combine<VN, TACC>(sw, spart, TR, P, r, wn);
      st_acc<VN>(sw2 + r, wn);
#pragma unroll
      for (int e = 0; e < VN; ++e)
        if (r0 + r + e < S.n) w[r0 + r + e] = wn[e];
    }
    __syncthreads();
#define GG_B2(NW) tile_dot<NW, TV, TACC>(acc, sV, sw2, TR, warp, lane)
    GG_SLICE_SWITCH(nw, GG_B2)
#undef GG_B2
  };
  auto end = [&](const BSys& S) {
    flush_cols(acc, nw, k, swarp, sred);
    if (sys_flush(S, S.tile0_p, S.ntile_p, tab.T_p, sred, k, tot)) {
      for (int c = threadIdx.x; c < k; c += blockDim.x) {
        const double h2 = S.ctl.sigma[c] * tot[c];
        S.ctl.h[c] += h2;
        S.ctl.coef[c] = S.ctl.sigma[c] * h2;
      }
    }
    __syncthreads();
  };
  bring_run(R, tab, begin, body, end);
}

template <typename TV, typename TACC>
__global__ void __launch_bounds__(kThreads) kb_pass3(BTab tab, int k) {
  constexpr int VN = Vec<TV>::n;
  extern __shared__ __align__(128) unsigned char smraw[];
  __shared__ uint64_t bars[kMaxStages];
  __shared__ TACC scoef[kMaxK];
  __shared__ __align__(16) TACC spart[4 * 256];
  __shared__ double sbuf[kThreads / 32];
  __shared__ double sred[1], tot[1];
  const int TR = tab.TR;
  const size_t sb = ring_stage_bytes(k, TR, sizeof(TV), sizeof(TACC));
  const BRing<TV, TACC> R{smraw, bars, k, TR, ring_stages(sb), sb};
  const int P = update_splits<TACC>(TR, VN), ng = TR / VN;
  TACC nrm = 0;
  auto begin = [&](const BSys& S) {
    nrm = 0;
    for (int c = threadIdx.x; c < k; c += blockDim.x) scoef[c] = (TACC)S.ctl.coef[c];
    __syncthreads();
  };
  auto body = [&](int st, const BSys& S, long long r0) {
    const TV* sV = R.vt(st);
    const TACC* sw = R.wt(st);
    tile_update<TV, TACC>(sV, TR, k, scoef, spart, P);
    __syncthreads();
    if ((int)threadIdx.x < ng) {
      const int r = threadIdx.x * VN;
      TV* vout = static_cast<TV*>(S.V) + (size_t)k * S.ldv;
      TACC wnv[VN];
      tile_combine<VN, TACC>(sw, spart, TR, P, r, wnv);
#pragma unroll
      for (int e = 0; e < VN; ++e) {
        if (r0 + r + e < S.n) {
          const TACC wn = wnv[e];
          TV stv;
          if constexpr (sizeof(TV) == sizeof(TACC)) {
            stv = (TV)wn;
          } else {
            stv = st_round<TV>((float)wn);
          }
          vout[r0 + r + e] = stv;
          const TACC sv = cv<TACC, TV>(stv);
          nrm += sv * sv;
        }
      }
    }
  };
  auto end = [&](const BSys& S) {
    const double bs = block_sum((double)nrm, sbuf);
    if (threadIdx.x == 0) sred[0] = bs;
    __syncthreads();
    if (sys_flush(S, S.tile0_p, S.ntile_p, tab.T_p, sred, 1, tot)) {
      Ctl ctl = S.ctl;
      givens_step(ctl, k - 1, tab.m, sqrt(tot[0]));
    }
    __syncthreads();
  };
  bring_run(R, tab, begin, body, end);
}

// ---- deflation: U^T x per system (warp per piece), then the coarse correction ----------
// mode 0: x = basis column j of a system in its cycle, scale sigma_j;
// mode 1: x = t of a live system at the cycle end, scale 1.
template <typename TV>
__global__ void __launch_bounds__(kThreads) kb_aggsum(BTab tab, int j, int mode) {
  const int lane = threadIdx.x & 31;
  const int p = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (p >= tab.P) return;
  const BSys& S = tab.sys[tab.piece_sys[p]];
  if (!S.ctl.flags[F_DEFL_ON] || (mode == 0 ? !sys_step_active(S) : !sys_live(S))) return;
  const int lp = p - S.piece0;
  const int s = S.defl.piece_start[lp], e = S.defl.piece_start[lp + 1];
  double acc = 0.0;
  if (mode == 0) {
    const TV* x = static_cast<const TV*>(S.V) + (size_t)j * S.ldv;
    for (int q = s + lane; q < e; q += 32) acc += ld_as<double, TV>(x + S.defl.perm[q]);
  } else {
    for (int q = s + lane; q < e; q += 32) acc += __ldg(S.t + S.defl.perm[q]);
  }
  acc = warp_sum(acc);
  if (lane == 0) S.ctl.cpart[lp] = acc;
}

__global__ void __launch_bounds__(kThreads) kb_coarse(BTab tab, int j, int mode) {
  extern __shared__ double sc[];
  const BSys& S = tab.sys[blockIdx.x];
  if (!S.ebp || !S.ctl.flags[F_DEFL_ON] || (mode == 0 ? !sys_step_active(S) : !sys_live(S)))
    return;
  const Defl& d = S.defl;
  const double scale = mode == 0 ? S.ctl.sigma[j] : 1.0;
  const double mu = S.ctl.scal[S_MU];
  for (int a = threadIdx.x; a < d.r; a += blockDim.x) {
    double s = 0.0;
    for (int p = d.agg_piece[a]; p < d.agg_piece[a + 1]; ++p) s += S.ctl.cpart[p];
    sc[a] = scale * d.uscale[a] * s;
  }
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  for (int a = warp; a < d.r; a += nwarps) {
    const double* row = d.tinv + (size_t)a * d.r;
    double acc = 0.0;
    for (int b = lane; b < d.r; b += 32) acc += __ldg(row + b) * sc[b];
    acc = warp_sum(acc);
    if (lane == 0) {
      const double sd = d.uscale[a] * (mu * acc - sc[a]);
      S.ctl.sdefl[a] = sd;
      S.ctl.sdefl32[a] = (float)sd;
    }
  }
}

// ---- cycle end -------------------------------------------------------------------------
__global__ void kb_backsolve(BTab tab) {
  __shared__ double R[kMaxM * kMaxM];
  __shared__ double sg[kMaxM], sy[kMaxM];
  const BSys& S = tab.sys[blockIdx.x];
  if (!sys_live(S)) return;
  Ctl ctl = S.ctl;
  backsolve_block(ctl, R, sg, sy);
}

template <typename TV>
__global__ void __launch_bounds__(kThreads) kb_xupdate(BTab tab) {
  __shared__ double scoef[kMaxK];
  const int T = tab.T_s;
  const int lo = range_lo(blockIdx.x, gridDim.x, T), hi = range_lo(blockIdx.x + 1, gridDim.x, T);
  int cur = -1;
  for (int t = lo; t < hi; ++t) {
    const int s = tab.tile_sys_s[t];
    const BSys& S = tab.sys[s];
    if (!sys_live(S)) continue;
    const int k = S.ctl.flags[F_K];
    if (s != cur) {
      __syncthreads();
      for (int c = threadIdx.x; c < k; c += blockDim.x) scoef[c] = S.ctl.coef[c];
      __syncthreads();
      cur = s;
    }
    const int row = (t - S.tile0_s) * kSpmvRows + threadIdx.x;
    if (row >= S.n) continue;
    const TV* V = static_cast<const TV*>(S.V);
    double p0 = 0.0, p1 = 0.0;
    int c = 0;
    for (; c + 1 < k; c += 2) {
      p0 += ld_as<double, TV>(V + (size_t)c * S.ldv + row) * scoef[c];
      p1 += ld_as<double, TV>(V + (size_t)(c + 1) * S.ldv + row) * scoef[c + 1];
    }
    if (c < k) p0 += ld_as<double, TV>(V + (size_t)c * S.ldv + row) * scoef[c];
    if (S.ctl.flags[F_DEFL_ON]) S.t[row] = p0 + p1;
    else S.x[row] += p0 + p1;
  }
}

__global__ void __launch_bounds__(kThreads) kb_xapply(BTab tab) {
  const int T = tab.T_s;
  const int lo = range_lo(blockIdx.x, gridDim.x, T), hi = range_lo(blockIdx.x + 1, gridDim.x, T);
  for (int t = lo; t < hi; ++t) {
    const BSys& S = tab.sys[tab.tile_sys_s[t]];
    if (!sys_live(S) || !S.ctl.flags[F_DEFL_ON]) continue;
    const int row = (t - S.tile0_s) * kSpmvRows + threadIdx.x;
    if (row >= S.n) continue;
    const int a = S.defl.agg[row];
    S.x[row] += S.t[row] + (a >= 0 ? S.ctl.sdefl[a] : 0.0);
  }
}

// |mu| from the Ritz values of the first cycle, then the EBP correction is switched on
__global__ void kb_ritz(BTab tab) {
  __shared__ double A[kMaxM * kMaxM];
  __shared__ double smod;
  __shared__ int sfail;
  const BSys& S = tab.sys[blockIdx.x];
  if (!sys_live(S) || !S.ebp || S.mu_mode != GMRES_MU_RITZ_FIRST_CYCLE || S.ctl.flags[F_DEFL_ON])
    return;
  Ctl ctl = S.ctl;
  ritz_warp(ctl, A, smod, sfail);
  __syncwarp();
  if (threadIdx.x == 0 && !ctl.flags[F_STOP]) ctl.flags[F_DEFL_ON] = 1;
}

// loop condition of the graph: any system still running
__global__ void kb_setcond(BTab tab, cudaGraphConditionalHandle handle) {
  __shared__ int any;
  if (threadIdx.x == 0) any = 0;
  __syncthreads();
  for (int s = threadIdx.x; s < tab.count; s += blockDim.x)
    if (sys_live(tab.sys[s])) atomicOr(&any, 1);
  __syncthreads();
  if (threadIdx.x == 0) cudaGraphSetConditional(handle, any ? 1u : 0u);
}

// ---- host side -------------------------------------------------------------------------
template <typename TV, typename TA, typename TACC>
struct BKern {
  static size_t ring_smem(int k, int TR) {
    const size_t sb = ring_stage_bytes(k, TR, sizeof(TV), sizeof(TACC));
    return (size_t)ring_stages(sb) * sb;
  }
  static cudaError_t prepare(int TR, int m) {
    // the stage count adapts to k, so the largest ring is not always the last step's
    int mx = 0;
    for (int k = 1; k <= m + 1; ++k) mx = std::max(mx, (int)ring_smem(k, TR));
    cudaError_t e = cudaFuncSetAttribute(kb_pass1<TV, TACC>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
    if constexpr (sizeof(TV) == sizeof(TACC))
      if (e == cudaSuccess)
        e = cudaFuncSetAttribute(kb_pass1_icwy<TV, TACC>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(kb_pass2<TV, TACC>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(kb_pass3<TV, TACC>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
    return e;
  }
  static int occupancy(const void* f, size_t smem) {
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, f, kThreads, smem) != cudaSuccess || n < 1) n = 1;
    return n;
  }
  // one restart cycle of every system; returns the number of kernels enqueued, or -1
  // with *err / *where set when a launch fails
  static int cycle(const BTab& tab, int sms, int bps_pass, int max_r, bool lowsync,
                   cudaStream_t st, cudaError_t* err, const char** where) {
    const int m = tab.m;
    auto grid = [&](int T, int per_sm) { return std::max(1, std::min(T, per_sm * sms)); };
    const int gs = grid(tab.T_s, 4);
    const int gpieces = std::max(1, (tab.P + 7) / 8);
    const size_t csm = sizeof(double) * (size_t)std::max(1, max_r);
    int nl = 0;
    kb_aggsum<TV><<<gpieces, kThreads, 0, st>>>(tab, 0, 0);
    if ((*err = cudaGetLastError()) != cudaSuccess) { *where = "kb_aggsum"; return -1; }
    kb_coarse<<<tab.count, kThreads, csm, st>>>(tab, 0, 0);
    if ((*err = cudaGetLastError()) != cudaSuccess) { *where = "kb_coarse"; return -1; }
    nl += 2;
    for (int j = 0; j < m; ++j) {
      const int k = j + 1;
      const size_t rs = ring_smem(k, tab.TR);
      kb_spmv<TA, TV, TACC><<<gs, kSpmvRows, 0, st>>>(tab, j);
      if ((*err = cudaGetLastError()) != cudaSuccess) { *where = "kb_spmv"; return -1; }
      const int gp3 = grid(tab.T_p, std::min(bps_pass, occupancy((const void*)kb_pass3<TV, TACC>, rs)));
      bool icwy = false;
      if constexpr (sizeof(TV) == sizeof(TACC)) {
        if (lowsync) {  // one-reduction MGS: one multi-dot pass, the solve, the update
          icwy = true;
          const int gp1 =
              grid(tab.T_p, std::min(bps_pass, occupancy((const void*)kb_pass1_icwy<TV, TACC>, rs)));
          kb_pass1_icwy<TV, TACC><<<gp1, kThreads, rs, st>>>(tab, k);
          if ((*err = cudaGetLastError()) != cudaSuccess) { *where = "kb_pass1_icwy"; return -1; }
          kb_icwy_solve<<<tab.count, 256, 0, st>>>(tab, k);
          if ((*err = cudaGetLastError()) != cudaSuccess) { *where = "kb_icwy_solve"; return -1; }
        }
      }
      if (!icwy) {  // CGS2: pass 1, pass 2, then the update
        const int gp1 = grid(tab.T_p, std::min(bps_pass, occupancy((const void*)kb_pass1<TV, TACC>, rs)));
        const int gp2 = grid(tab.T_p, std::min(bps_pass, occupancy((const void*)kb_pass2<TV, TACC>, rs)));
        kb_pass1<TV, TACC><<<gp1, kThreads, rs, st>>>(tab, k);
        if ((*err = cudaGetLastError()) != cudaSuccess) { *where = "kb_pass1"; return -1; }
        kb_pass2<TV, TACC><<<gp2, kThreads, rs, st>>>(tab, k);
        if ((*err = cudaGetLastError()) != cudaSuccess) { *where = "kb_pass2"; return -1; }
      }
      kb_pass3<TV, TACC><<<gp3, kThreads, rs, st>>>(tab, k);
      if ((*err = cudaGetLastError()) != cudaSuccess) { *where = "kb_pass3"; return -1; }
      kb_aggsum<TV><<<gpieces, kThreads, 0, st>>>(tab, k, 0);
      if ((*err = cudaGetLastError()) != cudaSuccess) { *where = "kb_aggsum"; return -1; }
      kb_coarse<<<tab.count, kThreads, csm, st>>>(tab, k, 0);
      if ((*err = cudaGetLastError()) != cudaSuccess) { *where = "kb_coarse"; return -1; }
      nl += 6;
    }
    kb_backsolve<<<tab.count, 128, 0, st>>>(tab);
    if ((*err = cudaGetLastError()) != cudaSuccess) { *where = "kb_backsolve"; return -1; }
    kb_xupdate<TV><<<gs, kThreads, 0, st>>>(tab);
    if ((*err = cudaGetLastError()) != cudaSuccess) { *where = "kb_xupdate"; return -1; }
    kb_aggsum<TV><<<gpieces, kThreads, 0, st>>>(tab, 0, 1);
    if ((*err = cudaGetLastError()) != cudaSuccess) { *where = "kb_aggsum"; return -1; }
    kb_coarse<<<tab.count, kThreads, csm, st>>>(tab, 0, 1);
    if ((*err = cudaGetLastError()) != cudaSuccess) { *where = "kb_coarse"; return -1; }
    kb_xapply<<<gs, kThreads, 0, st>>>(tab);
    if ((*err = cudaGetLastError()) != cudaSuccess) { *where = "kb_xapply"; return -1; }
    kb_ritz<<<tab.count, 32, 0, st>>>(tab);
    if ((*err = cudaGetLastError()) != cudaSuccess) { *where = "kb_ritz"; return -1; }
    kb_residual<TV><<<grid(tab.T_s, 4), kSpmvRows, 0, st>>>(tab);
    if ((*err = cudaGetLastError()) != cudaSuccess) { *where = "kb_residual"; return -1; }
    nl += 7;
    return nl;
  }
  static void prologue(const BTab& tab, int sms, double tol, double inner_tol, int fixed,
                       int mixed, long long maxit, cudaStream_t st) {
    kb_init<<<(tab.count + 31) / 32, 32, 0, st>>>(tab, tol, inner_tol, fixed, mixed, maxit);
    kb_residual<TV><<<std::max(1, std::min(tab.T_s, 4 * sms)), kSpmvRows, 0, st>>>(tab);
  }
};

struct BatchCtx {
  std::vector<gmres_s*> hs;
  int m = 0, prec = 0, TR = 0, bps = 0, max_r = 0, count = 0, ortho = 0;
  BTab tab{};
  DevMem dsys, dtile_s, dtile_p, dpiece;
  std::vector<BSys> hsys;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  int kernels_per_cycle = 0;
  cudaStream_t cap = nullptr;
  ~BatchCtx() {
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
    if (cap) cudaStreamDestroy(cap);
  }
};

// Cached batch contexts.  Deliberately never destroyed at process exit: no CUDA call may
// run from a static destructor once the runtime is being torn down.
std::vector<std::unique_ptr<BatchCtx>>& batch_cache() {
  static auto* c = new std::vector<std::unique_ptr<BatchCtx>>();
  return *c;
}

template <typename K>
int run_cycle(const BatchCtx& c, int sms, cudaStream_t st, cudaError_t* err, const char** where) {
  return K::cycle(c.tab, sms, c.bps, c.max_r, c.ortho == GMRES_ORTHO_MGS_LOWSYNC, st, err, where);
}

int dispatch_cycle(const BatchCtx& c, int sms, cudaStream_t st, cudaError_t* err,
                   const char** where) {
  switch (c.prec) {
    case P_FP64: return run_cycle<BKern<double, double, double>>(c, sms, st, err, where);
    case P_FP32: return run_cycle<BKern<float, float, float>>(c, sms, st, err, where);
    default: return run_cycle<BKern<__nv_bfloat16, float, float>>(c, sms, st, err, where);
  }
}

void dispatch_prologue(const BatchCtx& c, int sms, double tol, double inner_tol, int fixed,
                       int mixed, long long maxit, cudaStream_t st) {
  switch (c.prec) {
    case P_FP64: BKern<double, double, double>::prologue(c.tab, sms, tol, inner_tol, fixed, mixed, maxit, st); break;
    case P_FP32: BKern<float, float, float>::prologue(c.tab, sms, tol, inner_tol, fixed, mixed, maxit, st); break;
    default: BKern<__nv_bfloat16, float, float>::prologue(c.tab, sms, tol, inner_tol, fixed, mixed, maxit, st); break;
  }
}

cudaError_t dispatch_prepare(int prec, int TR, int m) {
  switch (prec) {
    case P_FP64: return BKern<double, double, double>::prepare(TR, m);
    case P_FP32: return BKern<float, float, float>::prepare(TR, m);
    default: return BKern<__nv_bfloat16, float, float>::prepare(TR, m);
  }
}

int vec_rows(int prec) { return prec == P_FP64 ? 2 : (prec == P_FP32 ? 4 : 8); }

// Builds the tile tables for pass tiles of TR rows and uploads the system table.
cudaError_t build_tables(BatchCtx& c, cudaStream_t st) {
  std::vector<int> ts, tp, ps;
  for (int s = 0; s < c.count; ++s) {
    BSys& S = c.hsys[s];
    S.tile0_s = (int)ts.size();
    S.ntile_s = (S.n + kSpmvRows - 1) / kSpmvRows;
    ts.insert(ts.end(), S.ntile_s, s);
    S.tile0_p = (int)tp.size();
    S.ntile_p = (S.n + c.TR - 1) / c.TR;
    tp.insert(tp.end(), S.ntile_p, s);
    S.piece0 = (int)ps.size();
    ps.insert(ps.end(), S.defl.npieces, s);
  }
  cudaError_t e;
  if ((e = c.dsys.ensure(sizeof(BSys) * c.hsys.size())) != cudaSuccess) return e;
  if ((e = c.dtile_s.ensure(sizeof(int) * ts.size())) != cudaSuccess) return e;
  if ((e = c.dtile_p.ensure(sizeof(int) * tp.size())) != cudaSuccess) return e;
  if ((e = c.dpiece.ensure(sizeof(int) * std::max<size_t>(1, ps.size()))) != cudaSuccess) return e;
  if ((e = cudaMemcpyAsync(c.dsys.p, c.hsys.data(), sizeof(BSys) * c.hsys.size(),
                           cudaMemcpyHostToDevice, st)) != cudaSuccess) return e;
  if ((e = cudaMemcpyAsync(c.dtile_s.p, ts.data(), sizeof(int) * ts.size(), cudaMemcpyHostToDevice, st)) != cudaSuccess) return e;
  if ((e = cudaMemcpyAsync(c.dtile_p.p, tp.data(), sizeof(int) * tp.size(), cudaMemcpyHostToDevice, st)) != cudaSuccess) return e;
  if (!ps.empty() && (e = cudaMemcpyAsync(c.dpiece.p, ps.data(), sizeof(int) * ps.size(),
                                          cudaMemcpyHostToDevice, st)) != cudaSuccess) return e;
  c.tab.sys = c.dsys.as<BSys>();
  c.tab.count = c.count;
  c.tab.tile_sys_s = c.dtile_s.as<int>();
  c.tab.T_s = (int)ts.size();
  c.tab.tile_sys_p = c.dtile_p.as<int>();
  c.tab.T_p = (int)tp.size();
  c.tab.piece_sys = c.dpiece.as<int>();
  c.tab.P = (int)ps.size();
  c.tab.TR = c.TR;
  c.tab.m = c.m;
  return cudaStreamSynchronize(st);
}

// Captures prologue-free solve: a while node whose body is one restart cycle of every
// system followed by the loop-condition kernel.
cudaError_t build_graph(BatchCtx& c, int sms, const char** failed) {
  cudaError_t e;
  if (c.exec) {
    cudaGraphExecDestroy(c.exec);
    c.exec = nullptr;
  }
  if (c.graph) {
    cudaGraphDestroy(c.graph);
    c.graph = nullptr;
  }
  if (!c.cap && (e = cudaStreamCreateWithFlags(&c.cap, cudaStreamNonBlocking)) != cudaSuccess) return e;
  if ((e = cudaGraphCreate(&c.graph, 0)) != cudaSuccess) return e;
  cudaGraphConditionalHandle handle;
  if ((e = cudaGraphConditionalHandleCreate(&handle, c.graph, 1, cudaGraphCondAssignDefault)) != cudaSuccess)
    return e;
  cudaGraphNodeParams p{};
  p.type = cudaGraphNodeTypeConditional;
  p.conditional.handle = handle;
  p.conditional.type = cudaGraphCondTypeWhile;
  p.conditional.size = 1;
  cudaGraphNode_t node;
  if ((e = cudaGraphAddNode(&node, c.graph, nullptr, nullptr, 0, &p)) != cudaSuccess) return e;
  cudaGraph_t body = p.conditional.phGraph_out[0];
  if ((e = cudaStreamBeginCaptureToGraph(c.cap, body, nullptr, nullptr, 0,
                                         cudaStreamCaptureModeRelaxed)) != cudaSuccess)
    return e;
  cudaError_t le = cudaSuccess;
  const char* where = "";
  c.kernels_per_cycle = dispatch_cycle(c, sms, c.cap, &le, &where);
  if (c.kernels_per_cycle >= 0) {
    kb_setcond<<<1, 256, 0, c.cap>>>(c.tab, handle);
    le = cudaGetLastError();
    where = "kb_setcond";
    c.kernels_per_cycle += 1;
  }
  cudaGraph_t captured;
  e = cudaStreamEndCapture(c.cap, &captured);  // always ends the capture
  if (le != cudaSuccess) {
    *failed = where;
    return le;
  }
  if (e != cudaSuccess) return e;
  return cudaGraphInstantiate(&c.exec, c.graph, 0);
}

}  // namespace

// Batched solve entry (called by gmres_batch_solve).
gmres_status batch_solve_impl(int count, gmres_t const* hs, const double* const* b,
                              const double* const* x0, int m, double tol, long long maxit,
                              double* const* x, gmres_info* infos, cudaStream_t st,
                              long long* launches) {
  if (count == 0) return GMRES_OK;
  if (m < 1 || m > kMaxM) return fail(nullptr, GMRES_ERR_INVALID_ARG, "m must be in [1, 64]");
  if (!(tol >= 0.0) || maxit < 0) return fail(nullptr, GMRES_ERR_INVALID_ARG, "tol >= 0, maxit >= 0");
  const int prec = prec_of(hs[0]->opts.precision);
  for (int i = 0; i < count; ++i) {
    if (!hs[i] || !b[i] || !x[i]) return fail(nullptr, GMRES_ERR_INVALID_ARG, "null handle or vector in batch");
    if (prec_of(hs[i]->opts.precision) != prec)
      return fail(nullptr, GMRES_ERR_INVALID_ARG, "all handles of a batch must use one precision");
    if (hs[i]->r > 0 && hs[i]->opts.deflation_mode == GMRES_DEFL_PROJECTOR)
      return fail(nullptr, GMRES_ERR_INVALID_ARG, "deflation_mode PROJECTOR is not available");
    if (hs[i]->opts.deflation_mode == GMRES_DEFL_ADAPTIVE)
      return fail(nullptr, GMRES_ERR_INVALID_ARG,
                  "deflation_mode ADAPTIVE is for single-system solves");
    if (hs[i]->opts.ortho != hs[0]->opts.ortho)
      return fail(nullptr, GMRES_ERR_INVALID_ARG, "all handles of a batch must use one ortho");
    if (hs[i]->opts.ortho == GMRES_ORTHO_MGS)
      return fail(nullptr, GMRES_ERR_INVALID_ARG,
                  "the batched solve orthogonalises by CGS2 or the one-reduction MGS");
    if (hs[i]->dense_r > 0)
      return fail(nullptr, GMRES_ERR_INVALID_ARG, "dense W is for single-system solves");
  }
  int sms = hs[0]->sms;
  // workspaces of the handles serve the batch (allocated on the batch stream)
  for (int i = 0; i < count; ++i) {
    cudaStream_t keep = hs[i]->stream;
    hs[i]->stream = st;
    gmres_status s = ensure_workspace(hs[i], m, prec);
    hs[i]->stream = keep;
    if (s != GMRES_OK) return fail(nullptr, s, hs[i]->err);
  }
  // context: cached per handle list and m
  BatchCtx* ctx = nullptr;
  for (auto& c : batch_cache())
    if (c->m == m && c->prec == prec && c->count == count && c->ortho == hs[0]->opts.ortho &&
        std::equal(c->hs.begin(), c->hs.end(), hs))
      ctx = c.get();
  const bool fresh = ctx == nullptr;
  if (fresh) {
    batch_cache().push_back(std::make_unique<BatchCtx>());
    ctx = batch_cache().back().get();
    ctx->hs.assign(hs, hs + count);
    ctx->m = m;
    ctx->prec = prec;
    ctx->count = count;
    ctx->ortho = hs[0]->opts.ortho;
  }
  ctx->hsys.resize(count);
  int max_r = 0;
  for (int i = 0; i < count; ++i) {
    gmres_s* h = hs[i];
    BSys& S = ctx->hsys[i];
    S = BSys{};
    S.n = h->n;
    S.ebp = (h->r > 0 && h->opts.deflation_mode == GMRES_DEFL_EBP) ? 1 : 0;
    S.mu_mode = h->opts.mu_mode;
    S.mu_init = h->opts.mu_mode == GMRES_MU_USER ? std::fabs(h->opts.mu_user)
                : (h->opts.mu_mode == GMRES_MU_NORM_INF ? h->mu_norminf : 0.0);
    OpDev op = make_op(h, h->fwd);
    S.rowptr = op.rowptr;
    S.col = op.col;
    S.val = op.val;
    S.val32 = op.val32;
    S.b = b[i];
    S.x = x[i];
    S.V = h->V.p;
    S.ldv = h->ldv;
    S.w = h->w.p;
    S.t = h->t.as<double>();
    S.defl = op.defl;
    if (!S.ebp) S.defl.npieces = 0;
    S.ctl = make_ctl(h);
    max_r = std::max(max_r, h->r);
    const size_t nb = sizeof(double) * (size_t)h->n;
    cudaError_t e = (x0 && x0[i] && x0[i] != x[i])
                        ? cudaMemcpyAsync(x[i], x0[i], nb, cudaMemcpyDeviceToDevice, st)
                        : (!(x0 && x0[i]) ? cudaMemsetAsync(x[i], 0, nb, st) : cudaSuccess);
    if (e != cudaSuccess) return cuda_fail(nullptr, e, "batch x0");
  }
  ctx->max_r = max_r;
  cudaError_t e;
  const bool mixed = prec != P_FP64;
  const double inner_tol = prec == P_BF16 ? 1e-2 : 1e-4;
  if (fresh) {
    // autotuner: pass tile height x blocks per SM, timed on one restart cycle of this batch
    const int lo = 32 * vec_rows(prec);
    std::vector<std::pair<int, int>> cand;
    for (int tr = 256; tr >= lo; tr >>= 1)
      for (int bps : {4, 2})
        if (ring_stage_bytes(m + 1, tr, basis_elem(prec), prec == P_FP64 ? 8 : 4) <= 48 * 1024)
          cand.push_back({tr, bps});
    if (cand.empty()) cand.push_back({lo, 2});
    float best = 1e30f;
    int best_i = 0;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    for (size_t ci = 0; ci < cand.size(); ++ci) {
      ctx->TR = cand[ci].first;
      ctx->bps = cand[ci].second;
      if ((e = dispatch_prepare(prec, ctx->TR, m)) != cudaSuccess) return cuda_fail(nullptr, e, "batch prepare");
      if ((e = build_tables(*ctx, st)) != cudaSuccess) return cuda_fail(nullptr, e, "batch tables");
      dispatch_prologue(*ctx, sms, 0.0, inner_tol, 1, mixed ? 1 : 0, m, st);
      cudaEventRecord(e0, st);
      cudaError_t le = cudaSuccess;
      const char* where = "";
      if (dispatch_cycle(*ctx, sms, st, &le, &where) < 0) {
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        return cuda_fail(nullptr, le, where);
      }
      cudaEventRecord(e1, st);
      if ((e = cudaEventSynchronize(e1)) != cudaSuccess) return cuda_fail(nullptr, e, "batch autotune");
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      if (ms < best) {
        best = ms;
        best_i = (int)ci;
      }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    ctx->TR = cand[best_i].first;
    ctx->bps = cand[best_i].second;
    if ((e = dispatch_prepare(prec, ctx->TR, m)) != cudaSuccess) return cuda_fail(nullptr, e, "batch prepare");
    if ((e = build_tables(*ctx, st)) != cudaSuccess) return cuda_fail(nullptr, e, "batch tables");
    const char* failed = "";
    if ((e = build_graph(*ctx, sms, &failed)) != cudaSuccess) {
      const std::string msg = std::string("batch graph ") + failed;
      batch_forget(hs[0]);
      return cuda_fail(nullptr, e, msg.c_str());
    }
    // restore the initial guesses the autotuner overwrote
    for (int i = 0; i < count; ++i) {
      const size_t nb = sizeof(double) * (size_t)hs[i]->n;
      e = (x0 && x0[i] && x0[i] != x[i]) ? cudaMemcpyAsync(x[i], x0[i], nb, cudaMemcpyDeviceToDevice, st)
                                         : (!(x0 && x0[i]) ? cudaMemsetAsync(x[i], 0, nb, st) : cudaSuccess);
      if (e != cudaSuccess) return cuda_fail(nullptr, e, "batch x0");
    }
  } else {
    if ((e = build_tables(*ctx, st)) != cudaSuccess) return cuda_fail(nullptr, e, "batch tables");
  }
  dispatch_prologue(*ctx, sms, tol, inner_tol, 0, mixed ? 1 : 0, maxit, st);
  if ((e = cudaGraphLaunch(ctx->exec, st)) != cudaSuccess) return cuda_fail(nullptr, e, "batch graph launch");
  if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return cuda_fail(nullptr, e, "batch solve");
  if (launches) *launches = 2 + 1;  // prologue kernels + one graph launch
  gmres_status worst = GMRES_OK;
  for (int i = 0; i < count; ++i) {
    Meta hm;
    if ((e = cudaMemcpy(&hm, hs[i]->meta.p, sizeof(Meta), cudaMemcpyDeviceToHost)) != cudaSuccess)
      return cuda_fail(nullptr, e, "batch status");
    const gmres_status si = (gmres_status)hm.flags[F_STATUS];
    if (infos) {
      infos[i].iters = hm.counts[C_STEPS];
      infos[i].cycles = hm.counts[C_CYCLES];
      infos[i].refinements = hm.counts[C_REFINE];
      infos[i].rel_res_est = hm.scal[S_EST];
      infos[i].rel_res_true = hm.scal[S_TRUE];
      infos[i].mu = hm.scal[S_MU];
      infos[i].ms_total = 0.f;
      infos[i].status = si;
    }
    if (si < 0) {
      if (worst >= 0 || si < worst) worst = si;
    } else if (worst >= 0 && si > worst) {
      worst = si;
    }
  }
  return worst;
}

// drops cached batch contexts that reference h (called by gmres_destroy)
void batch_forget(gmres_t h) {
  auto& c = batch_cache();
  c.erase(std::remove_if(c.begin(), c.end(),
                         [&](const std::unique_ptr<BatchCtx>& p) {
                           return std::find(p->hs.begin(), p->hs.end(), h) != p->hs.end();
                         }),
          c.end());
}

}  // namespace gg
