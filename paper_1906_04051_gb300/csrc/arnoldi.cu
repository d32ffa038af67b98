// arnoldi.cu -- the kernels of one restart cycle of deflated GMRES(m) (Sec. 3.2-3.3).
//
// Basis storage.  Column c of V holds u_c, and the orthonormal Arnoldi vector is
// v_c = sigma_c u_c: the 1/||w|| scaling of Eq. 13 is applied lazily through the
// per-column scale sigma_c (folded into the projection coefficients, the SpMV gather and
// the x update), which saves one full pass over each new column.
//
// Step j (k = j + 1 columns), all on one stream, each kernel returning at once when the
// cycle has already ended on the device:
//   spmv    w = A z,  z = M^-1 v_j = v_j + U (|mu| T^-1 - I) U^T v_j  (Eqs. 16-17), with
//           the correction gathered as s[agg[col]] inside the SpMV
//   dot1    h  = V^T w                                (CGS2 pass 1)
//   upd1dot2 w -= V h,  h' = V^T w,  h += h'          (CGS2 pass 2, V read once)
//   upd2norm w -= V h', u_{j+1} = w, h_{j+1,j} = ||w|| (Eq. 13) and, in the last block,
//           the plane rotations, gamma update and stopping tests (Eqs. 12, 14)
//   aggsum + coarse: U^T v_{j+1} and s = U (|mu| T^-1 - I) U^T v_{j+1} for the next step
// Cycle end: back substitution R y = g, x += M^-1 V y (Eq. 11 with Eq. 16), then the
// true residual r = b - A x in FP64 (Eq. 15), which also starts the next cycle.
//
// All floating-point reductions are formed in a fixed order (deterministic).
#include <utility>

#include "internal.h"
#include "kernels.cuh"

#include <type_traits>

namespace gg {

namespace {

// w = sigma_j A u_j, or with deflation w = sigma_j [A | A W] [u_j; s'] = A (v_j + U s) with
// s' = s / sigma_j the coarse correction of u_j (the extended rows carry the A W entries
// with column index N + a).  A thread per row reads its entries straight from global
// memory, four at a time (L1 absorbs the strided access), which keeps many independent
// loads in flight without staging or block barriers.
template <typename TA, typename TV, typename TACC, bool DEFL>
__global__ void __launch_bounds__(kThreads)
    k_spmv_step(int N, const int* __restrict__ rowptr, const int* __restrict__ col,
                const TA* __restrict__ val, const TV* __restrict__ x, int j,
                const TACC* __restrict__ sdefl, TACC* __restrict__ w, Ctl ctl, Defl d) {
  pdl_wait();
  pdl_trigger();
  if (ctl.flags[F_CYCLE_DONE]) return;
  const TACC sigma = (TACC)ctl.sigma[j];
  auto g = [&](int c) -> TACC {
    if constexpr (DEFL) return c < N ? ld_as<TACC, TV>(x + c) : sdefl[c - N];
    else return ld_as<TACC, TV>(x + c);
  };
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x) {
    const int rs = __ldg(rowptr + i), re = __ldg(rowptr + i + 1);
    TACC acc0 = 0, acc1 = 0;
    int k = rs;
    for (; k + 3 < re; k += 4) {
      int c[4];
      TACC v[4], xv[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        c[u] = __ldg(col + k + u);
        v[u] = (TACC)__ldg(val + k + u);
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) xv[u] = g(c[u]);
      acc0 += v[0] * xv[0];
      acc1 += v[1] * xv[1];
      acc0 += v[2] * xv[2];
      acc1 += v[3] * xv[3];
    }
    for (; k < re; ++k) acc0 += (TACC)__ldg(val + k) * g(__ldg(col + k));
    if (DEFL && d.qd > 0)  // adaptive deflation: A U dense (the rows are plain A)
      for (int t = 0; t < d.qd; ++t) acc1 += (TACC)d.aud[(size_t)t * d.ldu + i] * sdefl[t];
    w[i] = sigma * (acc0 + acc1);
  }
}

// The same product for long rows (finite elements of higher order: the 27-node hexahedra
// of the paper's benchmark couple a node with 27 to 125 others).  A group of kVecLanes
// consecutive lanes takes kVecRows consecutive rows in turn, striding through each row's
// entries (two independent chains per lane), and the partial sums meet by shuffles.  The
// FP64 pipe is nearly as tight as HBM here (12 bytes per FMA), so lanes must not idle:
// few lanes per row keep the shuffle adds rare, and taking rows in pairs evens out the
// alternating vertex / mid-edge row lengths between the groups of a warp.  The loop bound
// is the warp's first group, so every lane takes part in every shuffle.
template <typename TA, typename TV, typename TACC, bool DEFL>
__global__ void __launch_bounds__(kThreads)
    k_spmv_vec(int N, const int* __restrict__ rowptr, const int* __restrict__ col,
               const TA* __restrict__ val, const TV* __restrict__ x, int j,
               const TACC* __restrict__ sdefl, TACC* __restrict__ w, Ctl ctl, Defl d) {
  constexpr int G = kVecLanes, R = kVecRows;
  constexpr int GPW = 32 / G;  // groups per warp
  pdl_wait();
  pdl_trigger();
  if (ctl.flags[F_CYCLE_DONE]) return;
  const TACC sigma = (TACC)ctl.sigma[j];
  auto g = [&](int c) -> TACC {
    if constexpr (DEFL) return c < N ? ld_as<TACC, TV>(x + c) : sdefl[c - N];
    else return ld_as<TACC, TV>(x + c);
  };
  const int sub = threadIdx.x & (G - 1);
  const long long gid = (blockIdx.x * (long long)blockDim.x + threadIdx.x) / G;
  const long long groups = (long long)gridDim.x * blockDim.x / G;
  const long long nb = (N + R - 1) / R;
  for (long long base = gid & ~(long long)(GPW - 1); base < nb; base += groups) {
    const long long bund = base + (gid & (GPW - 1));
    TACC acc[R];
#pragma unroll
    for (int r = 0; r < R; ++r) acc[r] = 0;
    if (bund < nb) {
#pragma unroll
      for (int r = 0; r < R; ++r) {
        const long long row = bund * R + r;
        if (row < N) {
          const int rs = __ldg(rowptr + row), re = __ldg(rowptr + row + 1);
          TACC a2 = 0;
          int k = rs + sub;
          for (; k + G < re; k += 2 * G) {
            const int c0 = __ldg(col + k), c1 = __ldg(col + k + G);
            const TACC v0 = (TACC)__ldg(val + k), v1 = (TACC)__ldg(val + k + G);
            acc[r] += v0 * g(c0);
            a2 += v1 * g(c1);
          }
          if (k < re) acc[r] += (TACC)__ldg(val + k) * g(__ldg(col + k));
          if (DEFL && d.qd > 0)  // adaptive deflation: A U dense, split over the lanes
            for (int t = sub; t < d.qd; t += G) a2 += (TACC)d.aud[(size_t)t * d.ldu + row] * sdefl[t];
          acc[r] += a2;
        }
      }
    }
#pragma unroll
    for (int r = 0; r < R; ++r)
#pragma unroll
      for (int o = G / 2; o > 0; o >>= 1) acc[r] += __shfl_xor_sync(0xffffffffu, acc[r], o);
    if (bund < nb && sub < R) {
      TACC a = acc[0];
#pragma unroll
      for (int r = 1; r < R; ++r)
        if (sub == r) a = acc[r];
      const long long row = bund * R + sub;
      if (row < N) w[row] = sigma * a;
    }
  }
}

// The same product with A in diagonal storage: row i sums dval[q][i] x[i + off_q] over the
// nd diagonals (coalesced loads of the values and of the shifted x; an index past either
// end is clamped to a valid row, where the stored value is 0), plus the A W row.  Each
// thread takes kDiaRows rows (independent FMA chains).  With deflation the kernels
// between the step's basis column and this SpMV (U^T v, T^-1 c) do not write x or the
// operator, so the diagonal part runs before pdl_wait() and overlaps the coarse solve;
// only the A W part needs its output s'.
constexpr int kDiaRows = 4;

template <typename TA, typename TV, typename TACC>
__device__ __forceinline__ TACC dia_row(int i, int N, const int* soff, int nd, long long ldd,
                                        const TA* __restrict__ dval, const TV* __restrict__ x) {
  TACC acc = 0;
  int q = 0;
  for (; q + 3 < nd; q += 4) {
    int c[4];
    TACC a[4], xv[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) c[u] = min(max(i + soff[q + u], 0), N - 1);
#pragma unroll
    for (int u = 0; u < 4; ++u) a[u] = (TACC)__ldg(dval + (q + u) * ldd + i);
#pragma unroll
    for (int u = 0; u < 4; ++u) xv[u] = ld_as<TACC, TV>(x + c[u]);
#pragma unroll
    for (int u = 0; u < 4; ++u) acc += a[u] * xv[u];
  }
  for (; q < nd; ++q) {
    const int c = min(max(i + soff[q], 0), N - 1);
    acc += (TACC)__ldg(dval + q * ldd + i) * ld_as<TACC, TV>(x + c);
  }
  return acc;
}

template <typename TA, typename TV, typename TACC, bool DEFL>
__global__ void __launch_bounds__(kThreads)
    k_spmv_dia(int N, DiaOffsets dia, long long ldd, const TA* __restrict__ dval,
               const TV* __restrict__ x, int j, Defl d, const TA* __restrict__ auval,
               const TACC* __restrict__ sdefl, TACC* __restrict__ w, Ctl ctl) {
  __shared__ int soff[kMaxDiag];
#pragma unroll
  for (int q = 0; q < kMaxDiag; ++q)
    if ((int)threadIdx.x == q) soff[q] = dia.off[q];
  __syncthreads();
  const int nd = dia.nd;
  const int i0 = blockIdx.x * blockDim.x * kDiaRows + threadIdx.x;
  TACC acc[kDiaRows];
  if constexpr (DEFL) {
#pragma unroll
    for (int u = 0; u < kDiaRows; ++u) {
      const int i = i0 + u * blockDim.x;
      acc[u] = i < N ? dia_row<TA, TV, TACC>(i, N, soff, nd, ldd, dval, x) : (TACC)0;
    }
  }
  pdl_wait();
  pdl_trigger();
  if (ctl.flags[F_CYCLE_DONE]) return;
  if constexpr (!DEFL) {
#pragma unroll
    for (int u = 0; u < kDiaRows; ++u) {
      const int i = i0 + u * blockDim.x;
      acc[u] = i < N ? dia_row<TA, TV, TACC>(i, N, soff, nd, ldd, dval, x) : (TACC)0;
    }
  }
  const TACC sigma = (TACC)ctl.sigma[j];
  if constexpr (DEFL) {
    if (d.qd > 0) {  // adaptive deflation: A U dense
#pragma unroll
      for (int u = 0; u < kDiaRows; ++u) {
        const int i = i0 + u * blockDim.x;
        if (i < N)
          for (int t = 0; t < d.qd; ++t) acc[u] += (TACC)d.aud[(size_t)t * d.ldu + i] * sdefl[t];
      }
    } else {
      // the A W rows of the thread's kDiaRows rows, each level of the gather (row
      // pointers, first entries, s' at their aggregates) issued for all rows at once; the
      // rare further entries of a row follow one by one
      int e0[kDiaRows], e1[kDiaRows], ac[kDiaRows];
      TACC av[kDiaRows], sv[kDiaRows];
#pragma unroll
      for (int u = 0; u < kDiaRows; ++u) {
        const int i = i0 + u * blockDim.x;
        e0[u] = i < N ? __ldg(d.aurp + i) : 0;
        e1[u] = i < N ? __ldg(d.aurp + i + 1) : 0;
      }
#pragma unroll
      for (int u = 0; u < kDiaRows; ++u) {
        const bool has = e0[u] < e1[u];
        av[u] = has ? (TACC)__ldg(auval + e0[u]) : (TACC)0;
        ac[u] = has ? __ldg(d.aucol + e0[u]) : 0;
      }
#pragma unroll
      for (int u = 0; u < kDiaRows; ++u) sv[u] = e0[u] < e1[u] ? sdefl[ac[u]] : (TACC)0;
#pragma unroll
      for (int u = 0; u < kDiaRows; ++u) {
        TACC aw = av[u] * sv[u];
        for (int e = e0[u] + 1; e < e1[u]; ++e) aw += (TACC)__ldg(auval + e) * sdefl[__ldg(d.aucol + e)];
        acc[u] += aw;
      }
    }
  }
#pragma unroll
  for (int u = 0; u < kDiaRows; ++u) {
    const int i = i0 + u * blockDim.x;
    if (i < N) w[i] = sigma * acc[u];
  }
}

// CGS2 pass 1 (pipelined): h_c = sigma_c (u_c . w), coef_c = sigma_c h_c.  The same
// multi-dot c = M^T x serves the adaptive deflation space (columns of U or A U) with
// another epilogue (DotEpi).
template <typename TV, typename TACC>
__global__ void __launch_bounds__(kThreads)
    k_pass1(int N, const TV* __restrict__ V, long long ldv, int k, int TR,
            const TACC* __restrict__ w, Ctl ctl, DotEpi epi) {
  extern __shared__ __align__(128) unsigned char smraw[];
  __shared__ uint64_t bars[kMaxStages];
  __shared__ double swarp[kSlices * kSliceCols];
  __shared__ double sred[kMaxK];
  __shared__ double tot[kMaxK];
  const size_t sb = ring_stage_bytes(k, TR, sizeof(TV), sizeof(TACC));
  const Ring<TV, TACC> R{smraw, bars, k, TR, ring_stages(sb), sb};
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nw = slice_cols(k, warp, kSlices);
  TACC acc[kSliceCols];
#pragma unroll
  for (int i = 0; i < kSliceCols; ++i) acc[i] = 0;
  // w is the predecessor's (the SpMV's) output: its slices are copied after the wait
  const bool ok = ring_run(R, N, V, ldv, w, ctl, false, [] {}, [&](int st, long long) {
#define GG_P1(NW) tile_dot<NW, TV, TACC>(acc, R.vt(st), R.wt(st), TR, warp, lane)
    GG_SLICE_SWITCH(nw, GG_P1)
#undef GG_P1
  }, epi.skip_slot);
  if (!ok) return;
  reduce_slices(acc, nw, k, kSlices, reinterpret_cast<double*>(smraw), swarp, sred);
  if (!last_block_reduce(sred, k, ctl.part, ctl.part2, ctl.ldp, ctl.ticket, tot)) return;
  if (epi.mode == kEpiCoarse) {  // s = |mu| T^-1 c - c (adaptive deflation, Eq. 17)
    const double mu = fabs(ctl.scal[S_MU]);
    for (int t = threadIdx.x; t < k; t += blockDim.x) {
      double y = 0.0;
      for (int u = 0; u < k; ++u) y += epi.tinv[(size_t)t * epi.ldt + u] * tot[u];
      const double sv = mu * y - tot[t];
      ctl.sdefl[t] = sv;
      ctl.sdefl32[t] = (float)sv;
    }
    return;
  }
  if (epi.mode == kEpiRaw) {
    for (int t = threadIdx.x; t < k; t += blockDim.x) epi.out[t] = tot[t];
    return;
  }
  for (int c = threadIdx.x; c < k; c += blockDim.x) {
    const double hc = ctl.sigma[c] * tot[c];
    ctl.h[c] = hc;
    ctl.coef[c] = ctl.sigma[c] * hc;
  }
}

// One-reduction MGS, pass 1: the multi-dot of pass 1 that also forms the dots of the
// newest basis column u_j with all columns from the tile already in shared memory, so
// one reduction gives g = V^T w and the new row of L (v_j . v_c, c < j).  (A separate
// kernel from k_pass1 so that CGS2's pass keeps its own register allocation.)
template <typename TV, typename TACC>
__global__ void __launch_bounds__(kThreads, sizeof(TV) == 8 ? 3 : 2)
    k_pass1_icwy(int N, const TV* __restrict__ V, long long ldv, int k, int TR,
                 const TACC* __restrict__ w, Ctl ctl, DotEpi epi) {
  extern __shared__ __align__(128) unsigned char smraw[];
  __shared__ uint64_t bars[kMaxStages];
  __shared__ double swarp[kSlices * kSliceCols];
  __shared__ double sred[2 * kMaxK];  // the block's sums: g (k), then the L row (k)
  // the grid totals live in the ring's memory, free once the block's slices are reduced,
  // so that the static shared memory still allows three blocks per SM
  double* tot = reinterpret_cast<double*>(smraw);
  const size_t sb = ring_stage_bytes(k, TR, sizeof(TV), sizeof(TACC));
  const Ring<TV, TACC> R{smraw, bars, k, TR, ring_stages(sb), sb};
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nw = slice_cols(k, warp, kSlices);
  TACC acc[kSliceCols], acc2[kSliceCols];
#pragma unroll
  for (int i = 0; i < kSliceCols; ++i) acc[i] = 0;
#pragma unroll
  for (int i = 0; i < kSliceCols; ++i) acc2[i] = 0;
  // w is the predecessor's (the SpMV's) output: its slices are copied after the wait;
  // the second multi-dot takes the tile's newest column u_j in the place of w
  const bool ok = ring_run(R, N, V, ldv, w, ctl, false, [] {}, [&](int st, long long) {
#define GG_P1(NW)                                                                        \
  {                                                                                      \
    tile_dot<NW, TV, TACC>(acc, R.vt(st), R.wt(st), TR, warp, lane);                     \
    tile_dot<NW, TV, TACC>(acc2, R.vt(st), (const TACC*)(R.vt(st) + (size_t)(k - 1) * TR), \
                           TR, warp, lane);                                              \
  }
    GG_SLICE_SWITCH(nw, GG_P1)
#undef GG_P1
  }, epi.skip_slot);
  if (!ok) return;
  reduce_slices(acc, nw, k, kSlices, reinterpret_cast<double*>(smraw), swarp, sred);
  reduce_slices(acc2, nw, k, kSlices, reinterpret_cast<double*>(smraw), swarp, sred + k);
  if (!last_block_reduce(sred, 2 * k, ctl.part, ctl.part2, ctl.ldp, ctl.ticket, tot)) return;
  // g_c = v_c . w into h (the solve kernel turns it into the MGS coefficients) and the
  // new row of L: v_j . v_c = sigma_j sigma_c (u_j . u_c), c < j
  const double sj = ctl.sigma[k - 1];
  for (int c = threadIdx.x; c < k; c += blockDim.x) {
    ctl.h[c] = ctl.sigma[c] * tot[c];
    if (c < k - 1) ctl.L[(size_t)(k - 1) * kMaxK + c] = sj * ctl.sigma[c] * tot[k + c];
  }
}

// One-reduction MGS, the solve: (I + L) h = g with L strictly lower triangular (k x k of
// the cycle's rows), by forward substitution in one warp (entries i, i+32, i+64 of h in
// lane i's registers, column by column: h_c is final when reached, the rows below drop
// L[i][c] h_c), L staged in shared memory by the whole block first; then h = the MGS
// projection coefficients and coef_c = sigma_c h_c for the update pass.
__global__ void __launch_bounds__(256) k_icwy_solve(Ctl ctl, int k) {
  __shared__ double sL[kMaxK * kMaxK];
  pdl_wait();
  pdl_trigger();
  if (ctl.flags[F_CYCLE_DONE]) return;
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

// CGS2 pass 2 (pipelined): w -= sum_c coef_c u_c; h'_c = sigma_c (u_c . w); h += h'.
template <typename TV, typename TACC>
__global__ void __launch_bounds__(kThreads)
    k_pass2(int N, const TV* __restrict__ V, long long ldv, int k, int TR,
            TACC* __restrict__ w, Ctl ctl) {
  constexpr int VN = Vec<TV>::n;
  extern __shared__ __align__(128) unsigned char smraw[];
  __shared__ uint64_t bars[kMaxStages];
  __shared__ double swarp[kSlices * kSliceCols];
  __shared__ double sred[kMaxK];
  __shared__ double tot[kMaxK];
  __shared__ TACC scoef[kMaxK];
  __shared__ __align__(16) TACC spart[4 * 256];
  __shared__ __align__(16) TACC sw2[256];
  const size_t sb = ring_stage_bytes(k, TR, sizeof(TV), sizeof(TACC));
  const Ring<TV, TACC> R{smraw, bars, k, TR, ring_stages(sb), sb};
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nw = slice_cols(k, warp, kSlices);
  const int P = update_splits<TACC>(TR, VN);
  const int ng = TR / VN;
  TACC acc[kSliceCols];
#pragma unroll
  for (int i = 0; i < kSliceCols; ++i) acc[i] = 0;
  // w (the SpMV's output) is final before the wait; the coefficients are pass 1's output
  auto post = [&] {
    for (int c = threadIdx.x; c < k; c += blockDim.x) scoef[c] = (TACC)ctl.coef[c];
  };
  const bool ok = ring_run(R, N, V, ldv, (const TACC*)w, ctl, true, post, [&](int st, long long r0) {
    const TV* sV = R.vt(st);
    const TACC* sw = R.wt(st);
    tile_update<TV, TACC>(sV, TR, k, scoef, spart, P);
    __syncthreads();
    if ((int)threadIdx.x < ng) {
      const int r = threadIdx.x * VN;
      TACC wn[VN];
      tile_combine<VN, TACC>(sw, spart, TR, P, r, wn);
      st_acc<VN>(sw2 + r, wn);
#pragma unroll
      for (int e = 0; e < VN; ++e)
        if (r0 + r + e < N) w[r0 + r + e] = wn[e];
    }
    __syncthreads();
#define GG_P2(NW) tile_dot<NW, TV, TACC>(acc, sV, sw2, TR, warp, lane)
    GG_SLICE_SWITCH(nw, GG_P2)
#undef GG_P2
  });
  if (!ok) return;
  reduce_slices(acc, nw, k, kSlices, reinterpret_cast<double*>(smraw), swarp, sred);
  if (!last_block_reduce(sred, k, ctl.part, ctl.part2, ctl.ldp, ctl.ticket, tot)) return;
  for (int c = threadIdx.x; c < k; c += blockDim.x) {
    const double h2 = ctl.sigma[c] * tot[c];
    ctl.h[c] += h2;
    ctl.coef[c] = ctl.sigma[c] * h2;
  }
}

// CGS2 pass 3 (pipelined): u_{j+1} = w - sum_c coef_c u_c (stored), h_{j+1,j} = ||u_{j+1}||,
// then the plane rotations and stopping tests in the last block.
template <typename TV, typename TACC>
__global__ void __launch_bounds__(kThreads)
    k_pass3(int N, TV* __restrict__ V, long long ldv, int k, int TR,
            const TACC* __restrict__ w, Ctl ctl, int m) {
  constexpr int VN = Vec<TV>::n;
  extern __shared__ __align__(128) unsigned char smraw[];
  __shared__ uint64_t bars[kMaxStages];
  __shared__ TACC scoef[kMaxK];
  __shared__ __align__(16) TACC spart[4 * 256];
  __shared__ double sbuf[kThreads / 32];
  __shared__ double sred[1];
  __shared__ double tot[1];
  const size_t sb = ring_stage_bytes(k, TR, sizeof(TV), sizeof(TACC));
  const Ring<TV, TACC> R{smraw, bars, k, TR, ring_stages(sb), sb};
  // after the wait: pass 2's coefficients, and the rotations of Eq. 12 that do not need
  // h_{j+1,j}, off the critical path (the last block has the fewest tiles when they do
  // not divide evenly)
  auto post = [&] {
    for (int c = threadIdx.x; c < k; c += blockDim.x) scoef[c] = (TACC)ctl.coef[c];
    if (blockIdx.x == gridDim.x - 1) givens_prep(ctl, k - 1);
  };
  const int P = update_splits<TACC>(TR, VN);
  const int ng = TR / VN;
  TV* __restrict__ vout = V + (size_t)k * ldv;
  TACC nrm = 0;
  // w is pass 2's output: its slices are copied after the wait
  const bool ok = ring_run(R, N, (const TV*)V, ldv, w, ctl, false, post, [&](int st, long long r0) {
    const TV* sV = R.vt(st);
    const TACC* sw = R.wt(st);
    tile_update<TV, TACC>(sV, TR, k, scoef, spart, P);
    __syncthreads();
    if ((int)threadIdx.x < ng) {
      const int r = threadIdx.x * VN;
      TACC wnv[VN];
      tile_combine<VN, TACC>(sw, spart, TR, P, r, wnv);
#pragma unroll
      for (int e = 0; e < VN; ++e) {
        if (r0 + r + e < N) {
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
  });
  if (!ok) return;
  const double bs = block_sum((double)nrm, sbuf);
  if (threadIdx.x == 0) sred[0] = bs;
  __syncthreads();
  if (!last_block_reduce(sred, 1, ctl.part, ctl.part2, ctl.ldp, ctl.ticket, tot)) return;
  givens_finish(ctl, k - 1, m, sqrt(tot[0]));
}

// --------------------------------------------------------------------------------------
// Modified Gram-Schmidt (the paper's orthogonalisation, Sec. 3.2, Eq. 13): for c = 0..j,
// h_c = v_c . w, then w -= h_c v_c, each projection on the w left by the previous one.
// One cooperative kernel per Arnoldi step, one block per SM: each block keeps its
// contiguous slice of w on chip (registers, or shared memory for large n) for the whole
// step, so the basis is read once and w never leaves the chip; the only traffic is V
// (k columns) plus w in and u_{j+1} out.  Each projection needs the full dot product before the update, so every column
// ends with a grid barrier; the blocks' partial sums are then added by every block in
// the same fixed order (bitwise identical h_c everywhere, deterministic runs).  The last
// round is ||w||: u_{j+1} = w is stored (v_{j+1} = sigma_{j+1} u_{j+1}) and block 0 applies
// the plane rotations (Eq. 12).  The barrier's waits are bounded: a block that waits
// longer than about a second records GMRES_ERR_TIMEOUT and returns.
// --------------------------------------------------------------------------------------
constexpr int kMgsThreads = 512;
constexpr long long kBarrierSpins = 1LL << 21;  // polls of an L2 word: about a second

// Grid-wide barrier for a cooperative launch (all blocks co-resident): bar[0] counts
// arrivals, bar[1] is the generation that the last arrival advances.
__device__ __forceinline__ bool grid_barrier(unsigned* bar, unsigned& gen) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    int ok = 1;
    __threadfence();
    const unsigned arrived = atomicAdd(&bar[0], 1u);
    if (arrived == gridDim.x - 1) {
      atomicExch(&bar[0], 0u);
      __threadfence();
      atomicExch(&bar[1], gen + 1u);
    } else {
      long long spins = 0;
      while (*(volatile unsigned*)&bar[1] == gen) {
        if (++spins > kBarrierSpins) {
          ok = 0;
          break;
        }
      }
    }
    __threadfence();
    s_ok = ok;
  }
  __syncthreads();
  ++gen;
  return s_ok != 0;
}

// After each barrier the update with column c and the dot with column c+1 share one
// pass over the rows (w_r -= coef_c u_c[r]; part += w_r u_{c+1}[r]), so a column costs one
// pass and one barrier.  RPT > 0: each thread keeps its RPT rows of w and of the current
// column in registers (n <= SMs x threads x RPT); RPT = 0: w in shared memory and each
// column read twice (the second time from L1/L2).
template <int RPT>
__global__ void __launch_bounds__(kMgsThreads, 1)
    k_mgs(int N, double* __restrict__ V, long long ldv, int k, const double* __restrict__ w,
          Ctl ctl, int m, unsigned* bar, int rows) {
  extern __shared__ __align__(16) double sw[];  // RPT = 0: this block's rows of w
  __shared__ double sred[kMgsThreads / 32];
  __shared__ double stot;
  if (ctl.flags[F_CYCLE_DONE]) return;  // set before the launch: the same in every block
  unsigned gen = *(volatile unsigned*)&bar[1];  // nobody advances it before all arrive
  const int b = blockIdx.x, G = gridDim.x, T = blockDim.x, t = threadIdx.x;
  const long long r0 = (long long)b * rows;
  const int nr = (int)max(0LL, min((long long)rows, (long long)N - r0));
  double wr[RPT > 0 ? RPT : 1], ur[RPT > 0 ? RPT : 1];
  double part = 0.0;
  {  // w in, and the first dot (with u_0, or ||w||^2 when k = 0)
    const double* u = V + r0;
    if constexpr (RPT > 0) {
#pragma unroll
      for (int i = 0; i < RPT; ++i) {
        const int r = t + i * T;
        wr[i] = r < nr ? w[r0 + r] : 0.0;
        ur[i] = (r < nr && k > 0) ? u[r] : 0.0;
        part += k > 0 ? wr[i] * ur[i] : wr[i] * wr[i];
      }
    } else {
      for (int r = t; r < nr; r += T) {
        const double x = w[r0 + r];
        sw[r] = x;
        part += k > 0 ? x * u[r] : x * x;
      }
    }
  }
  for (int c = 0; c <= k; ++c) {  // round c: the dot with u_c (c < k) or ||w||^2 (c = k)
    const double bs = block_sum(part, sred);
    if (t == 0) __stcg(&ctl.part[(size_t)b * ctl.ldp + c], bs);
    if (!grid_barrier(bar, gen)) {
      if (t == 0) {
        ctl.flags[F_STATUS] = GMRES_ERR_TIMEOUT;
        ctl.flags[F_STOP] = 1;
        ctl.flags[F_CYCLE_DONE] = 1;
      }
      return;
    }
    if (t < 32) {  // every block: the same ordered sum of the G partials
      double x = 0.0;
      for (int i = t; i < G; i += 32) x += __ldcg(&ctl.part[(size_t)i * ctl.ldp + c]);
      x = warp_sum(x);
      if (t == 0) stot = x;
    }
    __syncthreads();
    const double tot = stot;
    if (c == k) {  // u_{j+1} = w is stored; v_{j+1} = sigma_{j+1} u_{j+1}
      double* vout = V + (size_t)k * ldv + r0;
      if constexpr (RPT > 0) {
#pragma unroll
        for (int i = 0; i < RPT; ++i)
          if (t + i * T < nr) vout[t + i * T] = wr[i];
      } else {
        for (int r = t; r < nr; r += T) vout[r] = sw[r];
      }
      if (b == 0) givens_step(ctl, k - 1, m, sqrt(tot));
      break;
    }
    const double sig = ctl.sigma[c];
    const double hc = sig * tot;  // v_c . w with v_c = sigma_c u_c
    if (b == 0 && t == 0) ctl.h[c] = hc;
    const double coef = sig * hc;
    const double* u = V + (size_t)c * ldv + r0;
    const double* un = u + ldv;  // u_{c+1}
    const bool last = c + 1 == k;
    part = 0.0;
    if constexpr (RPT > 0) {
#pragma unroll
      for (int i = 0; i < RPT; ++i) {
        const int r = t + i * T;
        const double nu = (r < nr && !last) ? un[r] : 0.0;
        wr[i] -= coef * ur[i];
        part += last ? wr[i] * wr[i] : wr[i] * nu;
        ur[i] = nu;
      }
    } else {
      for (int r = t; r < nr; r += T) {
        const double x = sw[r] - coef * u[r];
        sw[r] = x;
        part += last ? x * x : x * un[r];
      }
    }
  }
}

// --------------------------------------------------------------------------------------
// Deflation: c = scale U^T x by pieces (warp per piece), then s = U (|mu| T^-1 - I) c.
// --------------------------------------------------------------------------------------
// Piece sums: a warp per piece, up to 32 gathers in flight per lane (pieces hold at most
// kPiece = 1024 nodes, so one batch), four accumulators per lane (short FP64 chains).
template <typename TX>
__global__ void __launch_bounds__(kThreads)
    k_aggsum(const TX* __restrict__ x, Defl d, double* __restrict__ cpart, const int* flags,
             int skip_slot) {
  const int lane = threadIdx.x & 31;
  const int p = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const bool live = p < d.npieces;
  const int s = live ? d.piece_start[p] : 0, e = live ? d.piece_start[p + 1] : 0;
  // the permutation is static: the first batch of indexes is loaded before the wait
  int q[32];
#pragma unroll
  for (int u = 0; u < 32; ++u) {
    const int t = s + lane + 32 * u;
    q[u] = t < e ? __ldg(d.perm + t) : -1;
  }
  pdl_wait();
  pdl_trigger();
  if (!live || (skip_slot >= 0 && flags[skip_slot])) return;
  double acc[4] = {0.0, 0.0, 0.0, 0.0};
  for (int t0 = s; t0 < e; t0 += 32 * 32) {
    if (t0 != s) {
#pragma unroll
      for (int u = 0; u < 32; ++u) {
        const int t = t0 + lane + 32 * u;
        q[u] = t < e ? __ldg(d.perm + t) : -1;
      }
    }
    double v[32];
#pragma unroll
    for (int u = 0; u < 32; ++u) v[u] = q[u] >= 0 ? ld_as<double, TX>(x + q[u]) : 0.0;
#pragma unroll
    for (int u = 0; u < 32; ++u) acc[u & 3] += v[u];
  }
  const double sum = warp_sum((acc[0] + acc[1]) + (acc[2] + acc[3]));
  if (lane == 0) cpart[p] = sum;
}

// c_a = scale uscale_a sum(pieces of a) into shared memory (piece sums staged through
// shared memory when they fit), then y = T^-1 c by a warp per row (32 loads in flight
// per lane, four accumulators) and s_a = uscale_a (|mu| y_a - c_a), or s_a = uscale_a y_a
// for the deflation projector.
constexpr int kCoarseStage = 4096;  // piece sums staged in shared memory (32 KB)

__global__ void __launch_bounds__(kThreads)
    k_coarse(Defl d, const double* __restrict__ cpart, const double* __restrict__ scale_ptr,
             Ctl ctl, int skip_slot, int proj) {
  extern __shared__ double sc[];                 // r entries
  __shared__ double spc[kCoarseStage];
  const int r = d.r;
  const int lane = threadIdx.x & 31;
  const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int nw = (gridDim.x * blockDim.x) >> 5;
  // T^-1 is static: the first 32 entries per lane of the warp's first row are loaded
  // before the wait
  double t[32];
  {
    const double* row = d.tinv + (size_t)(gw < r ? gw : 0) * r;
#pragma unroll
    for (int u = 0; u < 32; ++u) {
      const int b = lane + 32 * u;
      t[u] = (gw < r && b < r) ? __ldg(row + b) : 0.0;
    }
  }
  pdl_wait();
  pdl_trigger();
  if (skip_slot >= 0 && ctl.flags[skip_slot]) return;
  const double scale = scale_ptr ? *scale_ptr : 1.0;
  const double mu = ctl.scal[S_MU];
  const bool staged = d.npieces <= kCoarseStage;
  if (staged)
    for (int p = threadIdx.x; p < d.npieces; p += blockDim.x) spc[p] = __ldg(cpart + p);
  __syncthreads();
  const double* pc = staged ? spc : cpart;
#pragma unroll 4
  for (int a = threadIdx.x; a < r; a += blockDim.x) {
    const int lo = __ldg(d.agg_piece + a), hi = __ldg(d.agg_piece + a + 1);
    const double us = __ldg(d.uscale + a);
    double sum = 0.0;
    for (int q = lo; q < hi; ++q) sum += pc[q];
    sc[a] = scale * us * sum;
  }
  __syncthreads();
  for (int a = gw; a < r; a += nw) {
    const double* row = d.tinv + (size_t)a * r;
    double acc[4] = {0.0, 0.0, 0.0, 0.0};
    for (int b0 = 0; b0 < r; b0 += 32 * 32) {
      if (a != gw || b0 != 0) {
#pragma unroll
        for (int u = 0; u < 32; ++u) {
          const int b = b0 + lane + 32 * u;
          t[u] = b < r ? __ldg(row + b) : 0.0;
        }
      }
#pragma unroll
      for (int u = 0; u < 32; ++u) {
        const int b = b0 + lane + 32 * u;
        if (b < r) acc[u & 3] += t[u] * sc[b];
      }
    }
    const double y = warp_sum((acc[0] + acc[1]) + (acc[2] + acc[3]));
    if (lane == 0) {
      const double us = __ldg(d.uscale + a);
      const double sd = proj ? us * y : us * (mu * y - sc[a]);
      ctl.sdefl[a] = sd;
      ctl.sdefl32[a] = (float)sd;
    }
  }
}

// --------------------------------------------------------------------------------------
// Deflation projector P = I - A U T^-1 U^T (GMRES on P A xh = P b): the coarse correction
// A (U y) is gathered over the CSR as s[agg[col]], with s = U y from k_coarse (proj mode).
// --------------------------------------------------------------------------------------
// vec -= A U y for every row (a step's w = P A v, skip when the cycle has ended)
template <typename TA, typename TACC>
__global__ void __launch_bounds__(kThreads)
    k_proj_sub(int N, Defl d, const TA* __restrict__ auval, const TACC* __restrict__ sdefl,
               TACC* __restrict__ vec, Ctl ctl) {
  pdl_wait();
  pdl_trigger();
  if (ctl.flags[F_CYCLE_DONE]) return;
  for (int row = blockIdx.x * blockDim.x + threadIdx.x; row < N; row += gridDim.x * blockDim.x)
    vec[row] -= au_row<TA, TACC>(row, d.aurp, d.aucol, auval, sdefl);
}

// r = t - A U y (t = b - A xh in FP64), stored as the cycle's start vector, with the
// restart decision on ||P (b - A xh)|| = ||b - A x|| (Eq. 15)
template <typename TV>
__global__ void __launch_bounds__(kSpmvRows)
    k_proj_resid(int N, Defl d, const double* __restrict__ t, TV* __restrict__ V0, Ctl ctl) {
  if (ctl.flags[F_STOP]) return;
  __shared__ double sbuf[kSpmvRows / 32];
  __shared__ double sred[2];
  __shared__ double tot[2];
  double n1 = 0.0, n2 = 0.0;
  for (int row = blockIdx.x * blockDim.x + threadIdx.x; row < N; row += gridDim.x * blockDim.x) {
    const double r = t[row] - au_row<double, double>(row, d.aurp, d.aucol, d.auval, ctl.sdefl);
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
  double b1 = block_sum(n1, sbuf);
  double b2 = (sizeof(TV) == sizeof(double)) ? b1 : block_sum(n2, sbuf);
  if (threadIdx.x == 0) {
    sred[0] = b1;
    sred[1] = b2;
  }
  __syncthreads();
  if (!last_block_reduce(sred, 2, ctl.part, ctl.part2, ctl.ldp, ctl.ticket, tot)) return;
  if (threadIdx.x == 0) residual_decide(ctl, sqrt(tot[0]), sqrt(tot[1]));
}

// x += U y (the coarse component x = xh + U T^-1 U^T (b - A xh) at the end of the solve)
__global__ void __launch_bounds__(kThreads)
    k_xcoarse(int N, double* __restrict__ x, const int* __restrict__ agg, Ctl ctl) {
  if (ctl.flags[F_STATUS] < 0) return;
  for (int row = blockIdx.x * blockDim.x + threadIdx.x; row < N; row += gridDim.x * blockDim.x) {
    const int a = agg[row];
    if (a >= 0) x[row] += ctl.sdefl[a];
  }
}

// --------------------------------------------------------------------------------------
// Cycle end
// --------------------------------------------------------------------------------------
__global__ void k_backsolve(Ctl ctl) {
  __shared__ double R[kMaxM * kMaxM];
  __shared__ double sg[kMaxM], sy[kMaxM];
  if (ctl.flags[F_STOP]) return;
  backsolve_block(ctl, R, sg, sy);
}

// t = V_k (sigma o y) in FP64; x += t directly, or t kept for the deflation correction.
template <typename TV, bool DEFL>
__global__ void __launch_bounds__(kThreads)
    k_xupdate(int N, const TV* __restrict__ V, long long ldv, double* __restrict__ x,
              double* __restrict__ t, Ctl ctl) {
  if (ctl.flags[F_STOP]) return;
  __shared__ double scoef[kMaxK];
  const int k = ctl.flags[F_K];
  for (int c = threadIdx.x; c < k; c += blockDim.x) scoef[c] = ctl.coef[c];
  __syncthreads();
  for (int row = blockIdx.x * blockDim.x + threadIdx.x; row < N; row += gridDim.x * blockDim.x) {
    double p0 = 0.0, p1 = 0.0, p2 = 0.0, p3 = 0.0;
    int c = 0;
    for (; c + 3 < k; c += 4) {
      const double v0 = ld_as<double, TV>(V + (size_t)c * ldv + row);
      const double v1 = ld_as<double, TV>(V + (size_t)(c + 1) * ldv + row);
      const double v2 = ld_as<double, TV>(V + (size_t)(c + 2) * ldv + row);
      const double v3 = ld_as<double, TV>(V + (size_t)(c + 3) * ldv + row);
      p0 += v0 * scoef[c];
      p1 += v1 * scoef[c + 1];
      p2 += v2 * scoef[c + 2];
      p3 += v3 * scoef[c + 3];
    }
    for (; c < k; ++c) p0 += ld_as<double, TV>(V + (size_t)c * ldv + row) * scoef[c];
    const double tv = (p0 + p1) + (p2 + p3);
    if (DEFL) t[row] = tv;
    else x[row] += tv;
  }
}

__global__ void __launch_bounds__(kThreads)
    k_xapply(int N, double* __restrict__ x, const double* __restrict__ t,
             const int* __restrict__ agg, Ctl ctl) {
  if (ctl.flags[F_STOP]) return;
  for (int row = blockIdx.x * blockDim.x + threadIdx.x; row < N; row += gridDim.x * blockDim.x) {
    const int a = agg[row];
    x[row] += t[row] + (a >= 0 ? ctl.sdefl[a] : 0.0);
  }
}

// x += t + U s with the dense adaptive U (s in ctl.sdefl)
__global__ void __launch_bounds__(kThreads)
    k_xapply_dense(int N, double* __restrict__ x, const double* __restrict__ t, Defl d, Ctl ctl) {
  if (ctl.flags[F_STOP]) return;
  for (int row = blockIdx.x * blockDim.x + threadIdx.x; row < N; row += gridDim.x * blockDim.x) {
    double v = t[row];
    for (int q = 0; q < d.qd; ++q) v += d.ud[(size_t)q * d.ldu + row] * ctl.sdefl[q];
    x[row] += v;
  }
}

// True residual in FP64 (Eq. 15): r = b - A x, u_0 = r stored in the basis precision,
// rho0 on the first call, convergence / maxit decision, and the start of a new cycle.
// With proj_t != null (deflation projector) the unprojected residual goes to proj_t, its
// norm only sets rho0 on the first call, and k_proj_resid takes the decision.
template <typename TV>
__global__ void __launch_bounds__(kSpmvRows)
    k_residual(int N, const int* __restrict__ rowptr, const int* __restrict__ col,
               const double* __restrict__ val, const double* __restrict__ x,
               const double* __restrict__ b, TV* __restrict__ V0, Ctl ctl,
               double* __restrict__ proj_t, int force) {
  if (!force && ctl.flags[F_STOP]) return;
  __shared__ double sval[kSpmvCap];
  __shared__ int scol[kSpmvCap];
  __shared__ double sbuf[kSpmvRows / 32];
  __shared__ double sred[2];
  __shared__ double tot[2];
  double n1 = 0.0, n2 = 0.0;
  const int tiles = (N + kSpmvRows - 1) / kSpmvRows;
  for (int t = blockIdx.x; t < tiles; t += gridDim.x) {
    double acc, accd;
    spmv_tile<double, double, false>(
        N, t * kSpmvRows, rowptr, col, val, sval, scol, [&](int c) { return __ldg(x + c); },
        nullptr, (const double*)nullptr, acc, accd);
    const int row = t * kSpmvRows + threadIdx.x;
    if (row < N) {
      const double r = __ldg(b + row) - acc;
      n1 += r * r;
      if (proj_t) {
        proj_t[row] = r;
      } else if constexpr (sizeof(TV) == sizeof(double)) {
        V0[row] = r;
      } else {
        const TV st = st_round<TV>((float)r);
        V0[row] = st;
        const double sv = (double)to_f<TV>(st);
        n2 += sv * sv;
      }
    }
  }
  double b1 = block_sum(n1, sbuf);
  double b2 = (sizeof(TV) == sizeof(double)) ? b1 : block_sum(n2, sbuf);
  if (threadIdx.x == 0) {
    sred[0] = b1;
    sred[1] = b2;
  }
  __syncthreads();
  if (!last_block_reduce(sred, 2, ctl.part, ctl.part2, ctl.ldp, ctl.ticket, tot)) return;
  if (threadIdx.x != 0) return;
  if (proj_t) {
    if (!ctl.flags[F_RHO0_SET]) {
      ctl.scal[S_RHO0] = ctl.scal[S_R0REF] > 0.0 ? ctl.scal[S_R0REF] : sqrt(tot[0]);
      ctl.flags[F_RHO0_SET] = 1;
    }
    return;
  }
  residual_decide(ctl, sqrt(tot[0]), sqrt(tot[1]));
}

// --------------------------------------------------------------------------------------
// |mu| from the Ritz values of H_k (Sec. 3.3): eigenvalues of the k x k Hessenberg matrix
// by the Francis double-shift QR iteration, one warp; lanes share the row and column
// updates of each reflector.
// --------------------------------------------------------------------------------------
__global__ void k_ritz(Ctl ctl) {
  __shared__ double A[kMaxM * kMaxM];
  __shared__ double smod;
  __shared__ int sfail;
  if (ctl.flags[F_STOP]) return;
  ritz_warp(ctl, A, smod, sfail);
}

__global__ void k_init(Ctl ctl, double tol, double inner_tol, double r0ref, double mu,
                       int fixed, int mixed, long long maxit) {
  if (threadIdx.x != 0) return;
  init_ctl(ctl, tol, inner_tol, r0ref, mu, fixed, mixed, maxit);
}

// ---- per-precision dispatch -----------------------------------------------------------
// Grid of a streaming kernel: one wave of resident blocks (occupancy calculator), never
// more blocks than tiles.
template <typename F>
int resident_grid(F kernel, int threads, size_t smem, int sms) {
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, smem) != cudaSuccess ||
      per_sm < 1)
    per_sm = 1;
  if (per_sm > 8) per_sm = 8;
  return per_sm * sms;
}

// Blocks for `tiles` tiles with at most gmax resident blocks: every block gets the same
// number of tiles (up to one), so no wave ends with a partial tail.
inline int balanced(int tiles, int gmax) {
  if (tiles < 1) return 1;
  const int per = (tiles + gmax - 1) / gmax;
  return (tiles + per - 1) / per;
}

// Launch with programmatic stream serialisation (the kernel may start while its
// predecessor finishes; see pdl_wait) when pdl, else as a plain launch.  Launch errors
// surface through cudaGetLastError like those of <<<>>>.
template <typename... Exp, typename... Act>
void launch_k(bool pdl, void (*kern)(Exp...), int grid, int block, size_t smem,
              cudaStream_t st, Act&&... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)grid);
  cfg.blockDim = dim3((unsigned)block);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = pdl ? 1 : 0;
  cudaLaunchKernelEx(&cfg, kern, std::forward<Act>(args)...);
}

template <typename TV, typename TA, typename TACC>
struct Kern {
  struct Grids {
    int spmv_d = 0, spmv_n = 0, resid = 0, xupd_d = 0, xupd_n = 0, xapply = 0;
    int tr[kMaxK + 1] = {0};
    int p1[kMaxK + 1] = {0}, p2[kMaxK + 1] = {0}, p3[kMaxK + 1] = {0}, p1i[kMaxK + 1] = {0};
  };
  // Tile height of the pipelined passes (256/128/64 rows, at least 32 16-byte vectors):
  // the largest whose stage fits 40 KB, so that a double-buffered ring leaves room for
  // three resident blocks per SM (the FP64 passes rely on other blocks to fill the FP64
  // pipe while one block waits at a barrier).
  static int tile_rows(int k) {
    const int lo = 32 * Vec<TV>::n;
    for (int tr = 256; tr > lo; tr >>= 1)
      if (ring_stage_bytes(k, tr, sizeof(TV), sizeof(TACC)) <= kStageBytes) return tr;
    return lo;
  }
  static size_t ring_smem(int k) {
    const size_t sb = ring_stage_bytes(k, tile_rows(k), sizeof(TV), sizeof(TACC));
    const size_t need = (size_t)ring_stages(sb) * sb;
    const size_t reduce = sizeof(double) * kSlices * kSliceCols * 33;  // reused after the ring
    return need > reduce ? need : (reduce + 127) / 128 * 128;
  }
  static Grids& grids(int sms) {
    static Grids g;
    static int for_sms = -1;
    if (for_sms != sms) {
      g.spmv_d = resident_grid(k_proj_sub<TA, TACC>, kThreads, 0, sms);
      g.resid = resident_grid(k_residual<TV>, kSpmvRows, 0, sms);
      g.xupd_d = resident_grid(k_xupdate<TV, true>, kThreads, 0, sms);
      g.xupd_n = resident_grid(k_xupdate<TV, false>, kThreads, 0, sms);
      g.xapply = resident_grid(k_xapply, kThreads, 0, sms);
      for (int k = 1; k <= kMaxK; ++k) {
        g.tr[k] = tile_rows(k);
        g.p1[k] = resident_grid(k_pass1<TV, TACC>, kThreads, ring_smem(k), sms);
        if constexpr (std::is_same<TV, TACC>::value)
          g.p1i[k] = resident_grid(k_pass1_icwy<TV, TACC>, kThreads, ring_smem(k), sms);
        g.p2[k] = resident_grid(k_pass2<TV, TACC>, kThreads, ring_smem(k), sms);
        g.p3[k] = resident_grid(k_pass3<TV, TACC>, kThreads, ring_smem(k), sms);
      }
      for_sms = sms;
    }
    return g;
  }
  static const TA* vals(const CycleArgs& a) {
    if constexpr (sizeof(TA) == sizeof(double)) return a.op.val;
    else return a.op.val32;
  }
  static const TA* dvals(const CycleArgs& a) {
    if constexpr (sizeof(TA) == sizeof(double)) return a.op.dval;
    else return a.op.dval32;
  }
  static const TA* xvals(const CycleArgs& a) {
    if constexpr (sizeof(TA) == sizeof(double)) return a.op.xval;
    else return a.op.xval32;
  }
  static const TA* auvals(const CycleArgs& a) {
    if constexpr (sizeof(TA) == sizeof(double)) return a.op.defl.auval;
    else return a.op.defl.auval32;
  }
  static const TACC* sdefl(const CycleArgs& a) {
    if constexpr (sizeof(TACC) == sizeof(double)) return a.ctl.sdefl;
    else return a.ctl.sdefl32;
  }

  // c = scale U^T x, then s = U (|mu| T^-1 - I) c (proj: s = U T^-1 c); c sits after the
  // piece sums in the cpart buffer
  template <typename TX>
  static void coarse(const CycleArgs& a, const TX* x, const double* scale, int skip, int proj,
                     cudaStream_t st, bool pdl = false) {
    const Defl& d = a.op.defl;
    const int gp = d.npieces > 0 ? (d.npieces + 7) / 8 : 1;
    launch_k(pdl, k_aggsum<TX>, gp, kThreads, 0, st, x, d, a.ctl.cpart, (const int*)a.ctl.flags,
             skip);
    const int rows = (d.r + 7) / 8;
    const int gc = rows < 2 * a.sms ? rows : 2 * a.sms;
    launch_k(pdl, k_coarse, gc > 0 ? gc : 1, kThreads, sizeof(double) * d.r, st, d,
             (const double*)a.ctl.cpart, scale, a.ctl, skip, proj);
  }

  // c = M^T x over ncols columns of M (leading dimension ldm) with the pipelined multi-dot
  // (FP64), finished by epi
  static void udots(const CycleArgs& a, const double* M, long long ldm, int ncols,
                    const double* x, DotEpi epi, bool pdl, cudaStream_t st) {
    if constexpr (sizeof(TV) == sizeof(double) && sizeof(TACC) == sizeof(double)) {
      const Grids& g = grids(a.sms);
      const int tr = g.tr[ncols];
      launch_k(pdl, k_pass1<TV, TACC>, grid_for((a.op.n + tr - 1) / tr, 1, g.p1[ncols]),
               kThreads, ring_smem(ncols), st, a.op.n, (const TV*)M, ldm, ncols, tr,
               (const TACC*)x, a.ctl, epi);
    }
  }

  static cudaError_t phase(const CycleArgs& a, int ph, int j, bool defl, double* x,
                           const double* b, cudaStream_t st, int* launches) {
    const int N = a.op.n;
    const int sms = a.sms;
    const Grids& g = grids(sms);
    const TV* V = static_cast<const TV*>(a.V);
    TV* Vm = static_cast<TV*>(a.V);
    TACC* w = static_cast<TACC*>(a.w);
    const int k = j + 1;
    const Defl& d = a.op.defl;
    int nl = 0;
    switch (ph) {
      case PH_SPMV: {
        const TV* xj = V + (size_t)j * a.ldv;
        const bool pdl = a.pdl != 0;
        // The CSR kernels gather x and are launched in plain stream order: started early
        // under programmatic dependent launch they made a GMRES(50) step 1.8x (lanes per
        // row) to 2.7x (thread per row) slower on the 3-D Bratu matrices.
        constexpr bool pdl_csr = false;
        const int gd = grid_for((N + kThreads - 1) / kThreads, 1, 8 * sms);
        if (a.op.dia.nd > 0) {  // banded A: diagonal storage
          const int gdd = (N + kThreads * kDiaRows - 1) / (kThreads * kDiaRows);
          if (defl && !a.proj)
            launch_k(pdl, k_spmv_dia<TA, TV, TACC, true>, gdd, kThreads, 0, st, N, a.op.dia,
                     a.op.ldd, dvals(a), xj, j, d, auvals(a), sdefl(a), w, a.ctl);
          else
            launch_k(pdl, k_spmv_dia<TA, TV, TACC, false>, gdd, kThreads, 0, st, N, a.op.dia,
                     a.op.ldd, dvals(a), xj, j, d, auvals(a), sdefl(a), w, a.ctl);
        } else if (a.op.vec) {  // long rows: kVecLanes lanes per row, rows in pairs
          const int gv = grid_for((long long)N * kVecLanes / kVecRows, kThreads, 64 * sms);
          if (defl && !a.proj && d.qd > 0)
            launch_k(pdl_csr, k_spmv_vec<TA, TV, TACC, true>, gv, kThreads, 0, st, N, a.op.rowptr,
                     a.op.col, vals(a), xj, j, sdefl(a), w, a.ctl, d);
          else if (defl && !a.proj)
            launch_k(pdl_csr, k_spmv_vec<TA, TV, TACC, true>, gv, kThreads, 0, st, N, a.op.xrp,
                     a.op.xcol, xvals(a), xj, j, sdefl(a), w, a.ctl, d);
          else
            launch_k(pdl_csr, k_spmv_vec<TA, TV, TACC, false>, gv, kThreads, 0, st, N,
                     a.op.rowptr, a.op.col, vals(a), xj, j, sdefl(a), w, a.ctl, d);
        } else if (defl && !a.proj && d.qd > 0) {  // adaptive: plain rows + A U dense
          launch_k(pdl_csr, k_spmv_step<TA, TV, TACC, true>, gd, kThreads, 0, st, N, a.op.rowptr,
                   a.op.col, vals(a), xj, j, sdefl(a), w, a.ctl, d);
        } else if (defl && !a.proj) {
          launch_k(pdl_csr, k_spmv_step<TA, TV, TACC, true>, gd, kThreads, 0, st, N, a.op.xrp,
                   a.op.xcol, xvals(a), xj, j, sdefl(a), w, a.ctl, d);
        } else {
          launch_k(pdl_csr, k_spmv_step<TA, TV, TACC, false>, gd, kThreads, 0, st, N, a.op.rowptr,
                   a.op.col, vals(a), xj, j, sdefl(a), w, a.ctl, d);
        }
        nl = 1;
        if (a.proj) {  // w = P A v_j = A v_j - A U T^-1 U^T A v_j
          coarse(a, (const TACC*)w, nullptr, F_CYCLE_DONE, 1, st, pdl);
          launch_k(pdl, k_proj_sub<TA, TACC>, g.spmv_d, kThreads, 0, st, N, d, auvals(a),
                   sdefl(a), w, a.ctl);
          nl = 4;
        }
        break;
      }
      case PH_DOT1: {
        const int tr = g.tr[k];
        if (a.ortho == GMRES_ORTHO_MGS_LOWSYNC) {  // one reduction, then the triangular solve
          if constexpr (std::is_same<TV, TACC>::value) {
            launch_k(a.pdl != 0, k_pass1_icwy<TV, TACC>, grid_for((N + tr - 1) / tr, 1, g.p1i[k]),
                     kThreads, ring_smem(k), st, N, V, a.ldv, k, tr, (const TACC*)w, a.ctl,
                     DotEpi{kEpiIcwy, nullptr, 0, nullptr, F_CYCLE_DONE});
            launch_k(a.pdl != 0, k_icwy_solve, 1, 256, 0, st, a.ctl, k);
            nl = 2;
          } else {
            return cudaErrorInvalidValue;
          }
          break;
        }
        launch_k(a.pdl != 0, k_pass1<TV, TACC>, grid_for((N + tr - 1) / tr, 1, g.p1[k]),
                 kThreads, ring_smem(k), st, N, V, a.ldv, k, tr, (const TACC*)w, a.ctl,
                 DotEpi{kEpiArnoldi, nullptr, 0, nullptr, F_CYCLE_DONE});
        nl = 1;
        break;
      }
      case PH_UPD1DOT2: {
        const int tr = g.tr[k];
        launch_k(a.pdl != 0, k_pass2<TV, TACC>, grid_for((N + tr - 1) / tr, 1, g.p2[k]),
                 kThreads, ring_smem(k), st, N, V, a.ldv, k, tr, w, a.ctl);
        nl = 1;
        break;
      }
      case PH_UPD2NORM: {
        const int tr = g.tr[k];
        launch_k(a.pdl != 0, k_pass3<TV, TACC>, grid_for((N + tr - 1) / tr, 1, g.p3[k]),
                 kThreads, ring_smem(k), st, N, Vm, a.ldv, k, tr, (const TACC*)w, a.ctl, a.m);
        nl = 1;
        break;
      }
      case PH_MGS: {  // modified Gram-Schmidt step on w = A M^-1 v_j (FP64)
        if constexpr (sizeof(TV) == sizeof(double) && sizeof(TACC) == sizeof(double)) {
          int rows = mgs_rows(N, sms);
          if (rows == 0) return cudaErrorInvalidValue;
          const int rpt = (rows + kMgsThreads - 1) / kMgsThreads;
          void (*kern)(int, double*, long long, int, const double*, Ctl, int, unsigned*, int) =
              rpt <= 4 ? k_mgs<4> : rpt <= 8 ? k_mgs<8> : rpt <= 16 ? k_mgs<16> : k_mgs<0>;
          const size_t smem = rpt <= 16 ? 0 : sizeof(double) * (size_t)rows;  // see prepare()
          int kk = k, Nn = N, m = a.m;
          double* Vd = reinterpret_cast<double*>(Vm);
          long long ldv = a.ldv;
          const double* wd = reinterpret_cast<const double*>(w);
          Ctl ctl = a.ctl;
          unsigned* bar = a.gbar;
          void* args[] = {&Nn, &Vd, &ldv, &kk, &wd, &ctl, &m, &bar, &rows};
          cudaError_t e = cudaLaunchCooperativeKernel((const void*)kern, dim3(sms),
                                                      dim3(kMgsThreads), args, smem, st);
          if (e != cudaSuccess) return e;
          nl = 1;
        } else {
          return cudaErrorInvalidValue;
        }
        break;
      }
      case PH_DEFL: {  // U^T v_j and the correction for column j
        const TV* xj = V + (size_t)j * a.ldv;
        if (d.qd > 0) {  // adaptive: one multi-dot over the dense U, then s' = |mu| T^-1 c - c
          if constexpr (sizeof(TV) == sizeof(double))
            udots(a, d.ud, d.ldu, d.qd, (const double*)xj,
                  DotEpi{kEpiCoarse, d.tinv_a, d.qd, nullptr, F_CYCLE_DONE}, a.pdl != 0, st);
          nl = 1;
        } else {
          coarse(a, xj, nullptr, F_CYCLE_DONE, 0, st, a.pdl != 0);  // s' = s / sigma_j
          nl = 2;
        }
        break;
      }
      case PH_CYCLE_END: {
        k_backsolve<<<1, 128, 0, st>>>(a.ctl);
        const int tiles = (N + kThreads - 1) / kThreads;
        if (defl && d.qd > 0) {  // adaptive: x += t + U s, s = |mu| T^-1 U^T t - U^T t
          k_xupdate<TV, true><<<grid_for(tiles, 1, g.xupd_d), kThreads, 0, st>>>(N, V, a.ldv, x,
                                                                                a.t, a.ctl);
          udots(a, d.ud, d.ldu, d.qd, a.t,
                DotEpi{kEpiCoarse, d.tinv_a, d.qd, nullptr, F_STOP}, false, st);
          k_xapply_dense<<<grid_for(tiles, 1, g.xapply), kThreads, 0, st>>>(N, x, a.t, d, a.ctl);
          nl = 4;
        } else if (defl) {
          k_xupdate<TV, true><<<grid_for(tiles, 1, g.xupd_d), kThreads, 0, st>>>(N, V, a.ldv, x,
                                                                                a.t, a.ctl);
          coarse(a, (const double*)a.t, nullptr, F_STOP, 0, st);
          k_xapply<<<grid_for(tiles, 1, g.xapply), kThreads, 0, st>>>(N, x, a.t, d.agg, a.ctl);
          nl = 5;
        } else {
          k_xupdate<TV, false><<<grid_for(tiles, 1, g.xupd_n), kThreads, 0, st>>>(N, V, a.ldv,
                                                                                 x, a.t, a.ctl);
          nl = 2;
        }
        break;
      }
      case PH_RESIDUAL: {
        const int tiles = (N + kSpmvRows - 1) / kSpmvRows;
        if (a.proj) {  // r = P (b - A xh), the true residual of x = xh + U T^-1 U^T (b - A xh)
          k_residual<TV><<<balanced(tiles, g.resid), kSpmvRows, 0, st>>>(
              N, a.op.rowptr, a.op.col, a.op.val, x, b, Vm, a.ctl, a.t, 0);
          coarse(a, (const double*)a.t, nullptr, F_STOP, 1, st);
          k_proj_resid<TV><<<balanced(tiles, g.resid), kSpmvRows, 0, st>>>(N, d, a.t, Vm, a.ctl);
          nl = 4;
        } else {
          k_residual<TV><<<balanced(tiles, g.resid), kSpmvRows, 0, st>>>(
              N, a.op.rowptr, a.op.col, a.op.val, x, b, Vm, a.ctl, nullptr, 0);
          nl = 1;
        }
        break;
      }
      case PH_PROJ_FINAL: {  // x = xh + U T^-1 U^T (b - A xh)
        const int tiles = (N + kSpmvRows - 1) / kSpmvRows;
        k_residual<TV><<<balanced(tiles, g.resid), kSpmvRows, 0, st>>>(
            N, a.op.rowptr, a.op.col, a.op.val, x, b, Vm, a.ctl, a.t, 1);
        coarse(a, (const double*)a.t, nullptr, -1, 1, st);
        k_xcoarse<<<grid_for((N + kThreads - 1) / kThreads, 1, g.xapply), kThreads, 0, st>>>(
            N, x, d.agg, a.ctl);
        nl = 4;
        break;
      }
      case PH_RITZ:
        k_ritz<<<1, 32, 0, st>>>(a.ctl);
        nl = 1;
        break;
      case PH_ARNOLDI: {  // the steps of a cycle in one persistent kernel (fused.cu; j = steps)
        const cudaError_t e = launch_arnoldi(a, j, defl, st);
        if (e != cudaSuccess) return e;
        nl = 1;
        break;
      }
      default:
        return cudaErrorInvalidValue;
    }
    if (launches) *launches += nl;
    return cudaGetLastError();
  }

  static cudaError_t prepare() {
    // the passes may need more than the default 48 KB of dynamic shared memory
    cudaError_t e = cudaSuccess;
    size_t mx = 0;
    for (int k = 1; k <= kMaxK; ++k) mx = ring_smem(k) > mx ? ring_smem(k) : mx;
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(k_pass1<TV, TACC>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)mx);
    if constexpr (std::is_same<TV, TACC>::value)
      if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_pass1_icwy<TV, TACC>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)mx);
    if constexpr (sizeof(TV) == sizeof(double))  // w of the MGS kernel, large n
      if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_mgs<0>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)(220 * 1024));
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(k_pass2<TV, TACC>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)mx);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(k_pass3<TV, TACC>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)mx);
    return e;
  }
};

using K64 = Kern<double, double, double>;
using K32 = Kern<float, float, float>;
using K16 = Kern<__nv_bfloat16, float, float>;

}  // namespace

static cudaError_t prepare_all() {
  static cudaError_t once = [] {
    cudaError_t e = K64::prepare();
    if (e == cudaSuccess) e = K32::prepare();
    if (e == cudaSuccess) e = K16::prepare();
    return e;
  }();
  return once;
}

cudaError_t launch_init(const CycleArgs& a, double tol, double inner_tol, double r0ref,
                        double mu, int fixed, int mixed, long long maxit, cudaStream_t st) {
  cudaError_t e = prepare_all();
  if (e != cudaSuccess) return e;
  k_init<<<1, 32, 0, st>>>(a.ctl, tol, inner_tol, r0ref, mu, fixed, mixed, maxit);
  return cudaGetLastError();
}

cudaError_t launch_udots(const CycleArgs& a, const double* M, long long ldm, int ncols,
                         const double* x, DotEpi epi, cudaStream_t st) {
  cudaError_t e = prepare_all();
  if (e != cudaSuccess) return e;
  K64::udots(a, M, ldm, ncols, x, epi, false, st);
  return cudaGetLastError();
}

// rows of w per block of the modified Gram-Schmidt kernel, 0 if n does not fit
int mgs_rows(int n, int sms) {
  const long long rows = ((long long)n + sms - 1) / sms;
  return rows * (long long)sizeof(double) <= 220 * 1024 ? (int)rows : 0;
}

cudaError_t launch_phase(const CycleArgs& a, int ph, int j, bool defl, double* x,
                         const double* b, cudaStream_t st, int* launches) {
  switch (a.prec) {
    case P_FP64: return K64::phase(a, ph, j, defl, x, b, st, launches);
    case P_FP32: return K32::phase(a, ph, j, defl, x, b, st, launches);
    default: return K16::phase(a, ph, j, defl, x, b, st, launches);
  }
}

}  // namespace gg
