// kernels.cuh -- device building blocks shared by the single-system kernels (arnoldi.cu)
// and the batched kernels (batch.cu): the staged SpMV tile, warp-slice multi-dots and
// their deterministic reduction, the bulk-copy tile ring, the vector shared-memory
// loads, the plane rotations (Eqs. 12, 14), the restart decision (Eq. 15), the back
// substitution (Eq. 12), the Ritz estimate of |mu| (Sec. 3.3) and the control-block
// initialisation.
#pragma once

#include <cfloat>

#include "common.cuh"
#include "tma.cuh"

namespace gg {

namespace {

// Programmatic dependent launch (the step kernels are launched with programmatic stream
// serialisation): pdl_wait() blocks until the previous kernel in the stream has
// completed and its writes are visible; pdl_trigger() lets the next kernel start its
// own prologue.  Each step kernel triggers only after its own wait, so when a kernel
// starts, every kernel before its immediate predecessor has completed: the prologue
// before pdl_wait() may read anything the predecessor does not write (static operator
// data, basis columns of earlier steps), never its outputs.  Launched without the
// attribute, both are no-ops.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() {
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

constexpr int kSpmvRows = 256;   // rows per SpMV tile (one per thread)
constexpr int kSpmvCap = 2560;   // CSR entries staged in shared memory per chunk

// --------------------------------------------------------------------------------------
// SpMV tile: rows [r0, r0 + 256) of A, one thread per row.  The tile's CSR entries are
// staged through shared memory with coalesced loads; x is gathered from global memory.
// acc  = sum_k a_ik x(col_k);  accd = sum_k a_ik s(agg(col_k))  (when DEFL)
// --------------------------------------------------------------------------------------
template <typename TA, typename TACC, bool DEFL, typename XG>
__device__ __forceinline__ void spmv_tile(int N, int r0, const int* __restrict__ rowptr,
                                          const int* __restrict__ col,
                                          const TA* __restrict__ val, TA* sval, int* scol,
                                          XG xg, const int* __restrict__ agg,
                                          const TACC* __restrict__ sdefl, TACC& acc,
                                          TACC& accd) {
  const int row = r0 + threadIdx.x;
  const int last = min(r0 + kSpmvRows, N);
  const int rs = row < N ? __ldg(rowptr + row) : 0;
  const int re = row < N ? __ldg(rowptr + row + 1) : 0;
  const int base = __ldg(rowptr + r0);
  const int end = __ldg(rowptr + last);
  acc = 0;
  accd = 0;
  for (int cs = base; cs < end; cs += kSpmvCap) {
    const int ce = min(cs + kSpmvCap, end);
    __syncthreads();
#pragma unroll 4
    for (int k = cs + threadIdx.x; k < ce; k += blockDim.x) {
      sval[k - cs] = __ldg(val + k);
      scol[k - cs] = __ldg(col + k);
    }
    __syncthreads();
    const int a = max(rs, cs), b = min(re, ce);
    int k = a;
    for (; k + 3 < b; k += 4) {  // four independent gathers in flight
      const int c0 = scol[k - cs], c1 = scol[k + 1 - cs], c2 = scol[k + 2 - cs],
                c3 = scol[k + 3 - cs];
      const TACC x0 = xg(c0), x1 = xg(c1), x2 = xg(c2), x3 = xg(c3);
      const TACC v0 = (TACC)sval[k - cs], v1 = (TACC)sval[k + 1 - cs],
                 v2 = (TACC)sval[k + 2 - cs], v3 = (TACC)sval[k + 3 - cs];
      acc += v0 * x0;
      acc += v1 * x1;
      acc += v2 * x2;
      acc += v3 * x3;
      if (DEFL) {
        const int p0 = __ldg(agg + c0), p1 = __ldg(agg + c1), p2 = __ldg(agg + c2),
                  p3 = __ldg(agg + c3);
        if (p0 >= 0) accd += v0 * sdefl[p0];
        if (p1 >= 0) accd += v1 * sdefl[p1];
        if (p2 >= 0) accd += v2 * sdefl[p2];
        if (p3 >= 0) accd += v3 * sdefl[p3];
      }
    }
    for (; k < b; ++k) {
      const int c = scol[k - cs];
      const TACC v = (TACC)sval[k - cs];
      acc += v * xg(c);
      if (DEFL) {
        const int p = __ldg(agg + c);
        if (p >= 0) accd += v * sdefl[p];
      }
    }
  }
}

// Coarse part of a deflated SpMV row: (A U s)_i = sum over the aggregates a met in row i
// of (A W)_ia * s_a, with A W stored in CSR (usually one entry per row), s = U-scaled
// coarse correction indexed by aggregate.
template <typename TA, typename TACC>
__device__ __forceinline__ TACC au_row(int row, const int* __restrict__ aurp,
                                       const int* __restrict__ aucol,
                                       const TA* __restrict__ auval,
                                       const TACC* __restrict__ s) {
  const int b = __ldg(aurp + row), e = __ldg(aurp + row + 1);
  TACC acc = 0;
  for (int q = b; q < e; ++q) acc += (TACC)__ldg(auval + q) * s[__ldg(aucol + q)];
  return acc;
}

// Number of columns of warp slice `slice` among k columns dealt round-robin to nslice
// slices.  Each warp runs an instance unrolled for exactly that many columns (a
// warp-uniform switch), so no floating-point instruction is issued under a false
// predicate: on GB300 a warp-wide FP64 FMA holds the narrow FP64 pipe for many cycles
// whether or not its lanes are enabled.
__device__ __forceinline__ int slice_cols(int k, int slice, int nslice) {
  return (k - slice + nslice - 1) / nslice;
}

#define GG_SLICE_SWITCH(nw, CALL)      \
  switch (nw) {                        \
    case 1: CALL(1); break;            \
    case 2: CALL(2); break;            \
    case 3: CALL(3); break;            \
    case 4: CALL(4); break;            \
    case 5: CALL(5); break;            \
    case 6: CALL(6); break;            \
    case 7: CALL(7); break;            \
    case 8: CALL(8); break;            \
    case 9: CALL(9); break;            \
    default: break;                    \
  }

// Per-block column sums of the warp-slice accumulators.  Lanes store their live
// accumulators (nw of them) transposed in shared memory; each (warp, column) pair is then
// summed by two threads, 16 lane values each as a pairwise tree, and one shuffle: the
// dependent chain of FP64 adds is 5 deep instead of 32 (a lone FP64 add costs the
// narrow FP64 pipe as much as a full warp's).  Row groups are then added in a fixed
// order.
__device__ __forceinline__ double tree16(const double* v) {
  double a[8];
#pragma unroll
  for (int i = 0; i < 8; ++i) a[i] = v[2 * i] + v[2 * i + 1];
#pragma unroll
  for (int i = 0; i < 4; ++i) a[i] = a[2 * i] + a[2 * i + 1];
  return (a[0] + a[1]) + (a[2] + a[3]);
}

template <typename TACC>
__device__ __forceinline__ void reduce_slices(const TACC (&acc)[kSliceCols], int nw, int k,
                                              int nslice, double* sbuf /* 8*9*33 */,
                                              double* swarp /* 8*9 */, double* sred) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nrg = kSlices / nslice;
#pragma unroll
  for (int i = 0; i < kSliceCols; ++i)
    if (i < nw) sbuf[(warp * kSliceCols + i) * 33 + lane] = (double)acc[i];
  __syncthreads();
  for (int t0 = 0; t0 < 2 * kSlices * kSliceCols; t0 += blockDim.x) {
    const int t = t0 + (int)threadIdx.x;
    const int pair = t >> 1, half = t & 1;
    double s = 0.0;
    bool live = false;
    if (pair < kSlices * kSliceCols) {
      const int wv = pair / kSliceCols, i = pair % kSliceCols;
      live = i < slice_cols(k, wv % nslice, nslice);
      if (live) s = tree16(sbuf + (size_t)pair * 33 + half * 16);
    }
    s += __shfl_xor_sync(0xffffffffu, s, 1);
    if (live && half == 0) swarp[pair] = s;
  }
  __syncthreads();
  for (int c = threadIdx.x; c < k; c += blockDim.x) {
    const int sl = c % nslice, i = c / nslice;
    double sum = 0.0;
    for (int g = 0; g < nrg; ++g) sum += swarp[(g * nslice + sl) * kSliceCols + i];
    sred[c] = sum;
  }
  __syncthreads();
}

// Plane rotations and stopping tests of step j (Eqs. 12, 14), by warp 0 of the calling
// block (the other threads return at once).  Lane l holds rows 2l and 2l+1 of the new
// Hessenberg column (j < kMaxM = 64).  Applying the j earlier rotations is a linear
// recurrence in the value carried down the column,
//   t_0 = h_0,  t_{i+1} = -sn_i t_i + cs_i h_{i+1},  rotated h_i = cs_i t_i + sn_i h_{i+1},
// so the carried values come from a warp scan of the affine maps t -> -sn_i t + cs_i h_{i+1}
// (5 shuffle levels) instead of a 2j-deep chain of dependent FP64 operations on one
// thread; the divisions of the new rotation and of 1/||w|| run in one SIMT division.
__device__ __forceinline__ void affine_compose(double& A, double& B, double Ae, double Be) {
  // (A, B) <- (A, B) o (Ae, Be): t -> A (Ae t + Be) + B
  B = fma(A, Be, B);
  A = A * Ae;
}

// First half, independent of h_{j+1,j} (it only needs h from the projections): the
// earlier rotations applied to column j (rows < j of H written), the unrotated column
// stored in Hr, and t_j and sum h_ij^2 left in the scalar slots for the second half.
__device__ void givens_prep(Ctl& ctl, int j) {
  if (threadIdx.x >= 32) return;
  const unsigned full = 0xffffffffu;
  const int lane = threadIdx.x;
  const int ldh = ctl.ldh;
  const int i0 = 2 * lane, i1 = 2 * lane + 1;
  const double h0 = i0 <= j ? ctl.h[i0] : 0.0;
  const double h1 = i1 <= j ? ctl.h[i1] : 0.0;
  const double c0 = i0 < j ? ctl.cs[i0] : 1.0, s0 = i0 < j ? ctl.sn[i0] : 0.0;
  const double c1 = i1 < j ? ctl.cs[i1] : 1.0, s1 = i1 < j ? ctl.sn[i1] : 0.0;
  if (i0 <= j) ctl.Hr[(size_t)i0 * ldh + j] = h0;
  if (i1 <= j) ctl.Hr[(size_t)i1 * ldh + j] = h1;
  const double hsq = warp_sum(fma(h1, h1, h0 * h0));
  const double h2 = __shfl_down_sync(full, h0, 1);  // h_{2l+2}
  // maps of rotations 2l and 2l+1 (identity past j - 1) and their composition
  const double a0 = i0 < j ? -s0 : 1.0, b0 = i0 < j ? c0 * h1 : 0.0;
  const double a1 = i1 < j ? -s1 : 1.0, b1 = i1 < j ? c1 * h2 : 0.0;
  double A = a1, B = b1;
  affine_compose(A, B, a0, b0);
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {  // inclusive scan, later maps applied last
    const double Ap = __shfl_up_sync(full, A, d), Bp = __shfl_up_sync(full, B, d);
    if (lane >= d) affine_compose(A, B, Ap, Bp);
  }
  double PA = __shfl_up_sync(full, A, 1), PB = __shfl_up_sync(full, B, 1);
  if (lane == 0) {
    PA = 1.0;
    PB = 0.0;
  }
  const double t0 = __shfl_sync(full, h0, 0);
  const double tc0 = fma(PA, t0, PB);       // t_{2l}
  const double tc1 = fma(a0, tc0, b0);      // t_{2l+1}
  const double r0 = fma(c0, tc0, s0 * h1);  // rotated h_{2l}
  const double r1 = fma(c1, tc1, s1 * h2);  // rotated h_{2l+1}
  if (i0 < j) ctl.H[(size_t)i0 * ldh + j] = r0;
  if (i1 < j) ctl.H[(size_t)i1 * ldh + j] = r1;
  const double a = __shfl_sync(full, (j & 1) ? tc1 : tc0, j >> 1);
  if (lane == 0) {
    ctl.scal[S_GIV_A] = a;
    ctl.scal[S_GIV_HN2] = hsq;
  }
}

// Second half: the new rotation from t_j and h_{j+1,j}, gamma update, 1 / ||w|| for the
// lazy normalisation, and the stopping tests (Eqs. 12, 14), by warp 0.
__device__ void givens_finish(Ctl& ctl, int j, int m, double hnext) {
  if (threadIdx.x >= 32) return;
  const unsigned full = 0xffffffffu;
  const int lane = threadIdx.x;
  const int ldh = ctl.ldh;
  const double a = __ldcg(&ctl.scal[S_GIV_A]);
  const double hn2 = fma(hnext, hnext, __ldcg(&ctl.scal[S_GIV_HN2]));
  const double gj = ctl.g[j];
  if (lane == 0) ctl.Hr[(size_t)(j + 1) * ldh + j] = hnext;
  double rho = 0.0;
  if (lane == 0 && hnext != 0.0) rho = hypot(a, hnext);
  rho = __shfl_sync(full, rho, 0);
  // lane 0: cs_j = a / rho, lane 1: sn_j = hnext / rho, lane 2: sigma_{j+1} = 1 / hnext
  double q = 0.0;
  if (lane < 3) {
    const double num = lane == 0 ? a : (lane == 1 ? hnext : 1.0);
    const double den = lane == 2 ? hnext : rho;
    const bool use = lane == 2 ? (hnext > 0.0) : (hnext != 0.0);
    q = use ? num / den : (lane == 0 ? 1.0 : 0.0);
  }
  const double c = __shfl_sync(full, q, 0), sn = __shfl_sync(full, q, 1);
  const double sig = __shfl_sync(full, q, 2);
  if (lane == 0) {
    ctl.H[(size_t)j * ldh + j] = hnext != 0.0 ? rho : a;
    ctl.H[(size_t)(j + 1) * ldh + j] = 0.0;
    const double sg1 = -sn * gj, sg0 = c * gj;
    ctl.cs[j] = c;
    ctl.sn[j] = sn;
    ctl.g[j] = sg0;
    ctl.g[j + 1] = sg1;
    const long long steps = ++ctl.counts[C_STEPS];
    ctl.flags[F_K] = j + 1;
    const double est = fabs(sg1) / ctl.scal[S_RHO0];
    ctl.scal[S_EST] = est;
    ctl.sigma[j + 1] = sig;
    bool done = false;
    if (!isfinite(hnext) || !isfinite(est)) {
      ctl.flags[F_STATUS] = GMRES_ERR_NAN;
      ctl.flags[F_STOP] = 1;
      done = true;
    }
    if (hnext <= 1e-14 * sqrt(hn2)) done = true;  // breakdown: the Krylov space is invariant
    if (!ctl.flags[F_FIXED] && est <= ctl.scal[S_TOL]) done = true;
    if (ctl.flags[F_MIXED] && fabs(sg1) <= ctl.scal[S_INNER_TOL] * ctl.scal[S_BETA_CYCLE])
      done = true;
    if (steps >= ctl.counts[C_MAXIT]) done = true;
    if (j + 1 >= m) done = true;
    if (done) ctl.flags[F_CYCLE_DONE] = 1;
  }
}

__device__ void givens_step(Ctl& ctl, int j, int m, double hnext) {
  givens_prep(ctl, j);
  __syncwarp();
  givens_finish(ctl, j, m, hnext);
}

// --------------------------------------------------------------------------------------
// Pipelined CGS2 passes.  Tiles of TR rows x k basis columns (plus the matching piece of
// w) are copied into a ring of 2-4 shared-memory stages by bulk asynchronous copies
// (one per column segment, issued by one thread, completed through an mbarrier per
// stage), so the copies of the next tile are in flight while the current one is
// computed.  Rows past n are zero padding of V and w (ldv and the w buffer are rounded
// up to 256 rows and zeroed at allocation), so tiles need no row guards when reading.
// --------------------------------------------------------------------------------------
constexpr int kMaxStages = 4;
constexpr size_t kStageBytes = 40 * 1024;  // preferred stage size
constexpr size_t kRingBytes = 60 * 1024;   // ring per block (three blocks per SM)

template <typename TV, typename TACC>
struct Ring {
  unsigned char* base;
  uint64_t* bars;
  int k, TR, S;
  size_t stage_bytes;
  __device__ TV* vt(int st) const { return reinterpret_cast<TV*>(base + (size_t)st * stage_bytes); }
  __device__ TACC* wt(int st) const {
    return reinterpret_cast<TACC*>(base + (size_t)st * stage_bytes + (size_t)k * TR * sizeof(TV));
  }
  // warp 0: tile starting at row r0 into stage st (lane 0 announces the bytes of the whole
  // stage, the lanes issue the column segments; the slice of w too when with_w)
  __device__ void issue_v(int st, long long r0, const TV* V, long long ldv, const TACC* w,
                          bool with_w) const {
    const int lane = threadIdx.x & 31;
    const uint32_t vb = (uint32_t)(TR * sizeof(TV)), wb = (uint32_t)(TR * sizeof(TACC));
    if (lane == 0) mbar_arrive_expect_tx(&bars[st], (uint32_t)k * vb + wb);
    __syncwarp();
    TV* dst = vt(st);
    for (int c = lane; c < k; c += 32)
      bulk_g2s(dst + (size_t)c * TR, V + (size_t)c * ldv + r0, vb, &bars[st]);
    if (with_w && lane == 0) bulk_g2s(wt(st), w + r0, wb, &bars[st]);
  }
  // warp 0: the slice of w of a stage whose columns were issued without it
  __device__ void issue_w(int st, long long r0, const TACC* w) const {
    if ((threadIdx.x & 31) == 0)
      bulk_g2s(wt(st), w + r0, (uint32_t)(TR * sizeof(TACC)), &bars[st]);
  }
};

__host__ __device__ inline size_t ring_stage_bytes(int k, int TR, size_t sv, size_t sa) {
  return ((size_t)k * TR * sv + (size_t)TR * sa + 127) / 128 * 128;
}

// stages that fit the ring budget (2..4)
__host__ __device__ inline int ring_stages(size_t stage_bytes) {
  int S = (int)(kRingBytes / stage_bytes);
  return S < 2 ? 2 : (S > kMaxStages ? kMaxStages : S);
}

// Streams this block's tiles (blockIdx.x, +gridDim.x, ...) through the ring and calls
// body(stage, r0) for each.  The copies of the basis columns for the first stages are
// issued before pdl_wait() (the columns 0..k-1 are final by then); the slice of w joins
// them before the wait too when w_early (w is not written by the predecessor), after it
// otherwise.  After the wait, post_wait() runs on all threads (loads of the
// predecessor's outputs); when flags[skip_slot] is set (by default the cycle has ended)
// the copies in flight are drained and false is returned, as it is (after recording GMRES_ERR_TIMEOUT and draining, with a
// bound) when a copy never completes.
template <typename TV, typename TACC, typename F, typename PW>
__device__ bool ring_run(const Ring<TV, TACC>& R, int N, const TV* V, long long ldv,
                         const TACC* w, Ctl& ctl, bool w_early, PW&& post_wait, F&& body,
                         int skip_slot = F_CYCLE_DONE) {
  __shared__ int s_pre;
  const int tiles = (N + R.TR - 1) / R.TR;
  const int nt = (int)blockIdx.x < tiles ? (tiles - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;
  const int first = nt < R.S ? nt : R.S;
  auto r0_of = [&](int i) { return (long long)(blockIdx.x + (size_t)i * gridDim.x) * R.TR; };
  if (threadIdx.x == 0) {
    for (int st = 0; st < R.S; ++st) mbar_init(&R.bars[st], 1);
    mbar_fence_init();
    // a cycle that has visibly ended already needs no prefetch (a stale read only costs
    // a wasted prefetch; the decision below is taken after the wait)
    s_pre = (skip_slot >= 0 && *(volatile const int*)&ctl.flags[skip_slot]) ? 0 : 1;
  }
  __syncthreads();
  const bool pre = s_pre != 0;
  if (pre && threadIdx.x < 32)
    for (int i = 0; i < first; ++i) R.issue_v(i, r0_of(i), V, ldv, w, w_early);
  pdl_wait();
  pdl_trigger();
  const bool done = skip_slot >= 0 && ctl.flags[skip_slot] != 0;
  if (pre && !w_early && threadIdx.x < 32)
    for (int i = 0; i < first; ++i) R.issue_w(i, r0_of(i), w);
  if (done) {
    if (pre)
      for (int i = 0; i < first; ++i) mbar_wait(&R.bars[i], 0u);
    __syncthreads();
    return false;
  }
  if (!pre && threadIdx.x < 32)
    for (int i = 0; i < first; ++i) R.issue_v(i, r0_of(i), V, ldv, w, true);
  post_wait();
  __syncthreads();
  int i = 0;
  bool ok = true;
  for (; i < nt; ++i) {
    const int st = i % R.S;
    ok = __syncthreads_and(mbar_wait(&R.bars[st], (uint32_t)((i / R.S) & 1)));
    if (!ok) break;
    body(st, r0_of(i));
    __syncthreads();
    if (threadIdx.x < 32 && i + R.S < nt) R.issue_v(st, r0_of(i + R.S), V, ldv, w, true);
  }
  if (!ok) {
    for (int j = i; j < nt && j < i + R.S; ++j)
      mbar_wait(&R.bars[j % R.S], (uint32_t)((j / R.S) & 1));
    if (threadIdx.x == 0) {
      ctl.flags[F_STATUS] = GMRES_ERR_TIMEOUT;
      ctl.flags[F_STOP] = 1;
      ctl.flags[F_CYCLE_DONE] = 1;
    }
    __syncthreads();
  }
  return ok;
}

// 16-byte vectors of the basis type: VN consecutive rows per shared-memory load.
template <typename TV> struct Vec;
template <> struct Vec<double> { static constexpr int n = 2; };
template <> struct Vec<float> { static constexpr int n = 4; };
template <> struct Vec<__nv_bfloat16> { static constexpr int n = 8; };

template <typename TACC>
__device__ __forceinline__ void ld_vec(const double* p, TACC (&o)[2]) {
  const double2 v = *reinterpret_cast<const double2*>(p);
  o[0] = (TACC)v.x;
  o[1] = (TACC)v.y;
}
template <typename TACC>
__device__ __forceinline__ void ld_vec(const float* p, TACC (&o)[4]) {
  const float4 v = *reinterpret_cast<const float4*>(p);
  o[0] = v.x;
  o[1] = v.y;
  o[2] = v.z;
  o[3] = v.w;
}
template <typename TACC>
__device__ __forceinline__ void ld_vec(const __nv_bfloat16* p, TACC (&o)[8]) {
  const uint4 v = *reinterpret_cast<const uint4*>(p);
  const __nv_bfloat162* h = reinterpret_cast<const __nv_bfloat162*>(&v);
#pragma unroll
  for (int e = 0; e < 4; ++e) {
    const float2 f = __bfloat1622float2(h[e]);
    o[2 * e] = f.x;
    o[2 * e + 1] = f.y;
  }
}
// VN accumulator-type values from shared memory (16-byte aligned)
template <int VN>
__device__ __forceinline__ void ld_acc(const double* p, double (&o)[VN]) {
#pragma unroll
  for (int e = 0; e < VN; e += 2) {
    const double2 v = *reinterpret_cast<const double2*>(p + e);
    o[e] = v.x;
    o[e + 1] = v.y;
  }
}
template <int VN>
__device__ __forceinline__ void ld_acc(const float* p, float (&o)[VN]) {
#pragma unroll
  for (int e = 0; e < VN; e += 4) {
    const float4 v = *reinterpret_cast<const float4*>(p + e);
    o[e] = v.x;
    o[e + 1] = v.y;
    o[e + 2] = v.z;
    o[e + 3] = v.w;
  }
}
// the inverse: VN values to shared memory (16-byte aligned)
template <int VN>
__device__ __forceinline__ void acc_store(double* p, const double (&v)[VN]) {
#pragma unroll
  for (int e = 0; e < VN; e += 2) *reinterpret_cast<double2*>(p + e) = make_double2(v[e], v[e + 1]);
}
template <int VN>
__device__ __forceinline__ void acc_store(float* p, const float (&v)[VN]) {
#pragma unroll
  for (int e = 0; e < VN; e += 4)
    *reinterpret_cast<float4*>(p + e) = make_float4(v[e], v[e + 1], v[e + 2], v[e + 3]);
}

// VN accumulator-type values to shared memory (16-byte aligned)
template <int VN>
__device__ __forceinline__ void st_acc(double* p, const double (&v)[VN]) {
#pragma unroll
  for (int e = 0; e < VN; e += 2) *reinterpret_cast<double2*>(p + e) = make_double2(v[e], v[e + 1]);
}
template <int VN>
__device__ __forceinline__ void st_acc(float* p, const float (&v)[VN]) {
#pragma unroll
  for (int e = 0; e < VN; e += 4)
    *reinterpret_cast<float4*>(p + e) = make_float4(v[e], v[e + 1], v[e + 2], v[e + 3]);
}

// Combine of a tile's update: for the VN rows at r, wn = sw - sum_q spart[q] (vector
// shared-memory accesses: no bank conflicts).
template <int VN, typename TACC>
__device__ __forceinline__ void tile_combine(const TACC* sw, const TACC* spart, int TR, int P,
                                             int r, TACC (&wn)[VN]) {
  TACC acc[VN];
  ld_acc<VN>(spart + r, acc);
  for (int q = 1; q < P; ++q) {
    TACC t[VN];
    ld_acc<VN>(spart + q * TR + r, t);
#pragma unroll
    for (int e = 0; e < VN; ++e) acc[e] += t[e];
  }
  TACC wv[VN];
  ld_acc<VN>(sw + r, wv);
#pragma unroll
  for (int e = 0; e < VN; ++e) wn[e] = wv[e] - acc[e];
}

// Dot phase of a tile: warp `slice` owns columns slice, slice+8, ... (NW of them) and its
// lanes sweep all TR rows, VN rows per 16-byte load.
template <int NW, typename TV, typename TACC>
__device__ __forceinline__ void tile_dot(TACC (&acc)[kSliceCols], const TV* sV, const TACC* sw,
                                         int TR, int slice, int lane) {
  constexpr int VN = Vec<TV>::n;
  for (int r = lane * VN; r < TR; r += 32 * VN) {
    TACC wv[VN];
    ld_acc<VN>(sw + r, wv);
#pragma unroll
    for (int i = 0; i < NW; ++i) {
      TACC v[VN];
      ld_vec(sV + (size_t)(slice + kSlices * i) * TR + r, v);
#pragma unroll
      for (int e = 0; e < VN; ++e) acc[i] += v[e] * wv[e];
    }
  }
}

// Update phase of a tile: thread (sub, group) sums columns [sub*kq, ...) of coef_c u_c for
// the VN rows of its group; partials land in spart[sub][row].  Returns the threads used.
template <typename TV, typename TACC>
__device__ __forceinline__ void tile_update(const TV* sV, int TR, int k, const TACC* scoef,
                                            TACC* spart, int P) {
  constexpr int VN = Vec<TV>::n;
  const int ng = TR / VN;
  if ((int)threadIdx.x >= ng * P) return;
  const int sub = threadIdx.x / ng, r = (threadIdx.x % ng) * VN;
  const int kq = (k + P - 1) / P;
  const int c0 = sub * kq, c1 = min(k, c0 + kq);
  TACC p[VN];
#pragma unroll
  for (int e = 0; e < VN; ++e) p[e] = 0;
  for (int c = c0; c < c1; ++c) {
    TACC v[VN];
    ld_vec(sV + (size_t)c * TR + r, v);
    const TACC cf = scoef[c];
#pragma unroll
    for (int e = 0; e < VN; ++e) p[e] += v[e] * cf;
  }
  st_acc<VN>(spart + sub * TR + r, p);
}

template <typename TACC> __host__ __device__ constexpr int update_splits(int TR, int VN) {
  // column subsets per row group: FP64 keeps the combine short (the FP64 pipe is the
  // bound), FP32 spreads the work over more threads
  return (kThreads / (TR / VN)) < (sizeof(TACC) == 8 ? 2 : 4) ? (kThreads / (TR / VN))
                                                              : (sizeof(TACC) == 8 ? 2 : 4);
}

// Restart decision after a true residual (Eq. 15): rho0 on the first call, NaN, tolerance
// and maxit tests, and the start of a new cycle (g = beta_s e1, sigma_0 = 1/beta_s).
__device__ void residual_decide(Ctl& ctl, double beta, double beta_s) {
  if (!ctl.flags[F_RHO0_SET]) {
    ctl.scal[S_RHO0] = ctl.scal[S_R0REF] > 0.0 ? ctl.scal[S_R0REF] : beta;
    ctl.flags[F_RHO0_SET] = 1;
  }
  const double rho0 = ctl.scal[S_RHO0];
  const double rel = rho0 > 0.0 ? beta / rho0 : 0.0;
  ctl.scal[S_BETA] = beta;
  ctl.scal[S_TRUE] = rel;
  ctl.flags[F_K] = 0;
  ctl.flags[F_CYCLE_DONE] = 1;
  if (!isfinite(beta) || !isfinite(beta_s)) {
    ctl.flags[F_STATUS] = GMRES_ERR_NAN;
    ctl.flags[F_STOP] = 1;
    return;
  }
  if (beta == 0.0 || (!ctl.flags[F_FIXED] && rel <= ctl.scal[S_TOL])) {
    ctl.flags[F_STATUS] = GMRES_OK;
    ctl.flags[F_STOP] = 1;
    return;
  }
  if (ctl.counts[C_STEPS] >= ctl.counts[C_MAXIT]) {
    ctl.flags[F_STATUS] = GMRES_NOT_CONVERGED;
    ctl.flags[F_STOP] = 1;
    return;
  }
  ctl.counts[C_REFINE]++;
  ctl.g[0] = beta_s;
  for (int i = 1; i <= ctl.ldh; ++i) ctl.g[i] = 0.0;
  ctl.sigma[0] = 1.0 / beta_s;
  ctl.scal[S_BETA_CYCLE] = beta_s;
  ctl.flags[F_CYCLE_DONE] = 0;
}

// Back substitution R_k y = g (Eq. 12) on a shared-memory copy of R; coef = sigma o y.
// Block-wide (at least one warp); R (kMaxM^2 doubles), sg, sy (kMaxM each) are
// shared-memory scratch.  The substitution runs column by column in warp 0: y_i = s_i / R_ii
// (s_i times the reciprocal of R_ii, all reciprocals formed up front), then s_l -= R_li y_i
// for every l < i at once, the lanes holding s in registers (k <= 64: two rows per lane).
// On GB300 a dependent FP64 operation costs a few dozen cycles and a division about ten of
// them, so the chain is k multiplies and multiply-adds instead of k^2 / 2 multiply-adds
// and k divisions in one thread.
__device__ void backsolve_block(Ctl& ctl, double* R, double* sg, double* sy) {
  static_assert(kMaxM <= 64, "two rows per lane");
  const int k = ctl.flags[F_K];
  const int ldh = ctl.ldh;
  for (int t = threadIdx.x; t < k * k; t += blockDim.x) {
    const int i = t / k, l = t % k;
    R[t] = l >= i ? ctl.H[(size_t)i * ldh + l] : 0.0;
  }
  for (int i = threadIdx.x; i < k; i += blockDim.x) sg[i] = ctl.g[i];
  __syncthreads();
  if (threadIdx.x < 32) {
    const int lane = threadIdx.x;
    double rinv[2], sl[2];
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      const int i = lane + 32 * q;
      rinv[q] = i < k ? 1.0 / R[i * k + i] : 0.0;
      sl[q] = i < k ? sg[i] : 0.0;
    }
    for (int i = k - 1; i >= 0; --i) {
      const int o = i & 31;
      const double si = __shfl_sync(0xffffffffu, i < 32 ? sl[0] : sl[1], o);
      const double ri = __shfl_sync(0xffffffffu, i < 32 ? rinv[0] : rinv[1], o);
      const double yi = si * ri;
      if (lane == o) sy[i] = yi;
#pragma unroll
      for (int q = 0; q < 2; ++q) {
        const int l = lane + 32 * q;
        if (l < i) sl[q] = fma(-R[l * k + i], yi, sl[q]);
      }
    }
    if (lane == 0) ctl.counts[C_CYCLES]++;
  }
  __syncthreads();
  for (int i = threadIdx.x; i < k; i += blockDim.x) {
    ctl.y[i] = sy[i];
    ctl.coef[i] = ctl.sigma[i] * sy[i];
  }
}

// Eigenvalues of the n x n upper Hessenberg matrix A in shared memory (row stride n,
// overwritten) by the Francis double-shift QR iteration, run by one warp (lanes 0..31 of
// the calling warp).  On return (after a __syncwarp) smod holds the largest eigenvalue
// modulus and (sre, sim) that eigenvalue (sim >= 0 for a complex pair; among equal
// moduli the one of lowest position on the diagonal); sfail = 1 if the iteration did not
// converge within 60 n sweeps.
__device__ void hqr_warp(double* A, int n, double& sre, double& sim, double& smod, int& sfail) {
  const int lane = threadIdx.x & 31;
#define AA(i, j) A[(i) * n + (j)]
  if (lane == 0) { smod = 0.0; sre = 0.0; sim = 0.0; sfail = 0; }
  __syncwarp();
  // eigenvalues are found from the bottom of the diagonal upwards, so ">=" keeps the
  // lowest-positioned one among equal moduli
  auto take = [&](double re, double im) {
    const double md = im == 0.0 ? fabs(re) : hypot(re, im);
    if (md >= smod) { smod = md; sre = re; sim = fabs(im); }
  };
  double an = 0.0;
  for (int t = lane; t < n * n; t += 32)
    if (t % n >= t / n - 1) an += fabs(A[t]);
  an = warp_sum(an);
  int hi = n - 1, its = 0, total = 0;
  while (hi >= 0) {
    int l;
    for (l = hi; l > 0; --l) {
      double s = fabs(AA(l - 1, l - 1)) + fabs(AA(l, l));
      if (s == 0.0) s = an;
      if (fabs(AA(l, l - 1)) <= DBL_EPSILON * s) break;
    }
    __syncwarp();
    if (l > 0 && lane == 0) AA(l, l - 1) = 0.0;
    __syncwarp();
    if (l == hi) {
      if (lane == 0) take(AA(hi, hi), 0.0);
      __syncwarp();
      --hi;
      its = 0;
      continue;
    }
    if (l == hi - 1) {
      const double a = AA(hi - 1, hi - 1), b = AA(hi - 1, hi), c = AA(hi, hi - 1), d = AA(hi, hi);
      const double p = 0.5 * (a - d), disc = p * p + b * c, mid = 0.5 * (a + d);
      if (lane == 0) {
        if (disc >= 0.0) {
          const double q = sqrt(disc);
          const double l1 = mid + (p >= 0.0 ? q : -q);
          const double l2 = (l1 != 0.0) ? (a * d - b * c) / l1 : mid - (p >= 0.0 ? q : -q);
          take(l2, 0.0);  // position hi
          take(l1, 0.0);  // position hi - 1
        } else {
          take(mid, sqrt(-disc));
        }
      }
      __syncwarp();
      hi -= 2;
      its = 0;
      continue;
    }
    if (++total > 60 * n) {
      if (lane == 0) sfail = 1;
      break;
    }
    double s, t;
    if (its == 10 || its == 20) {
      const double w = fabs(AA(hi, hi - 1)) + fabs(AA(hi - 1, hi - 2));
      const double sig = AA(hi, hi) + 0.75 * w;
      s = 2.0 * sig;
      t = sig * sig;
    } else {
      s = AA(hi - 1, hi - 1) + AA(hi, hi);
      t = AA(hi - 1, hi - 1) * AA(hi, hi) - AA(hi - 1, hi) * AA(hi, hi - 1);
    }
    ++its;
    double x = AA(l, l) * AA(l, l) + AA(l, l + 1) * AA(l + 1, l) - s * AA(l, l) + t;
    double y = AA(l + 1, l) * (AA(l, l) + AA(l + 1, l + 1) - s);
    double z = AA(l + 1, l) * AA(l + 2, l + 1);
    for (int k = l; k <= hi - 2; ++k) {
      const double nrm = sqrt(x * x + y * y + z * z);
      if (nrm != 0.0) {
        const double alpha = (x >= 0.0) ? -nrm : nrm;
        const double v0 = x - alpha, v1 = y, v2 = z;
        const double beta = 2.0 / (v0 * v0 + v1 * v1 + v2 * v2);
        const int c0 = (k > l) ? k - 1 : l;
        __syncwarp();
        for (int jj = c0 + lane; jj <= hi; jj += 32) {
          const double dd = beta * (v0 * AA(k, jj) + v1 * AA(k + 1, jj) + v2 * AA(k + 2, jj));
          AA(k, jj) -= dd * v0;
          AA(k + 1, jj) -= dd * v1;
          AA(k + 2, jj) -= dd * v2;
        }
        __syncwarp();
        if (k > l && lane == 0) {
          AA(k + 1, k - 1) = 0.0;
          AA(k + 2, k - 1) = 0.0;
        }
        __syncwarp();
        const int r1 = (k + 3 < hi) ? k + 3 : hi;
        for (int ii = l + lane; ii <= r1; ii += 32) {
          const double dd = beta * (AA(ii, k) * v0 + AA(ii, k + 1) * v1 + AA(ii, k + 2) * v2);
          AA(ii, k) -= dd * v0;
          AA(ii, k + 1) -= dd * v1;
          AA(ii, k + 2) -= dd * v2;
        }
        __syncwarp();
      }
      x = AA(k + 1, k);
      y = AA(k + 2, k);
      if (k < hi - 2) z = AA(k + 3, k);
      __syncwarp();
    }
    const double nrm = sqrt(x * x + y * y);
    if (nrm != 0.0) {
      const double alpha = (x >= 0.0) ? -nrm : nrm;
      const double v0 = x - alpha, v1 = y;
      const double beta = 2.0 / (v0 * v0 + v1 * v1);
      const int c0 = (hi - 2 > l) ? hi - 2 : l;
      __syncwarp();
      for (int jj = c0 + lane; jj <= hi; jj += 32) {
        const double dd = beta * (v0 * AA(hi - 1, jj) + v1 * AA(hi, jj));
        AA(hi - 1, jj) -= dd * v0;
        AA(hi, jj) -= dd * v1;
      }
      __syncwarp();
      if (hi - 2 >= l && lane == 0) AA(hi, hi - 2) = 0.0;
      __syncwarp();
      for (int ii = l + lane; ii <= hi; ii += 32) {
        const double dd = beta * (AA(ii, hi - 1) * v0 + AA(ii, hi) * v1);
        AA(ii, hi - 1) -= dd * v0;
        AA(ii, hi) -= dd * v1;
      }
      __syncwarp();
    }
  }
#undef AA
  __syncwarp();
}

// |mu| from the Ritz values of the cycle's H_k (one warp; A is kMaxM^2 doubles of shared
// scratch): the largest eigenvalue modulus.
__device__ void ritz_warp(Ctl& ctl, double* A, double& smod, int& sfail) {
  const int n = ctl.flags[F_K];
  const int lane = threadIdx.x & 31;
  if (n <= 0) return;
  const int ldh = ctl.ldh;
  // the Hessenberg block as built; entries below the subdiagonal are never written, so they
  // are taken as the zeros they are (not read from memory)
  for (int t = lane; t < n * n; t += 32) {
    const int i = t / n, c = t % n;
    A[t] = i <= c + 1 ? ctl.Hr[(size_t)i * ldh + c] : 0.0;
  }
  __syncwarp();
  __shared__ double sre, sim;
  hqr_warp(A, n, sre, sim, smod, sfail);
  if (lane == 0) {
    if (sfail || !(smod > 0.0) || !isfinite(smod)) {
      ctl.flags[F_STATUS] = GMRES_ERR_SINGULAR_COARSE;
      ctl.flags[F_STOP] = 1;
    } else {
      ctl.scal[S_MU] = smod;
    }
  }
}


__device__ void init_ctl(Ctl& ctl, double tol, double inner_tol, double r0ref, double mu,
                       int fixed, int mixed, long long maxit) {
  for (int i = 0; i < S_NSCAL; ++i) ctl.scal[i] = 0.0;
  for (int i = 0; i < F_NFLAGS; ++i) ctl.flags[i] = 0;
  for (int i = 0; i < C_NCOUNT; ++i) ctl.counts[i] = 0;
  ctl.scal[S_TOL] = tol;
  ctl.scal[S_INNER_TOL] = inner_tol;
  ctl.scal[S_R0REF] = r0ref;
  ctl.scal[S_MU] = mu;
  ctl.flags[F_FIXED] = fixed;
  ctl.flags[F_MIXED] = mixed;
  ctl.flags[F_STATUS] = GMRES_NOT_CONVERGED;
  ctl.flags[F_CYCLE_DONE] = 1;
  ctl.counts[C_MAXIT] = maxit;
  for (int i = 0; i < 1 + kMaxGroups; ++i) ctl.ticket[i] = 0u;
}

}  // namespace

}  // namespace gg
