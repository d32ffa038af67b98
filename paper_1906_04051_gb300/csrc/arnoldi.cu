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
#include <cfloat>

#include "common.cuh"
#include "internal.h"
#include "tma.cuh"

namespace gg {

namespace {

constexpr int kSpmvRows = 256;   // rows per SpMV tile (one per thread)
constexpr int kSpmvCap = 2560;   // CSR entries staged in shared memory per chunk
constexpr int kTile2 = 128;      // rows per tile of CGS2 pass 2

template <typename TACC> struct AccOf;

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
    for (int k = a; k < b; ++k) {
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

template <typename TA, typename TV, typename TACC, bool DEFL>
__global__ void __launch_bounds__(kSpmvRows)
    k_spmv_step(int N, const int* __restrict__ rowptr, const int* __restrict__ col,
                const TA* __restrict__ val, const TV* __restrict__ x, int j,
                const int* __restrict__ agg, const TACC* __restrict__ sdefl,
                TACC* __restrict__ w, Ctl ctl) {
  if (ctl.flags[F_CYCLE_DONE]) return;
  __shared__ TA sval[kSpmvCap];
  __shared__ int scol[kSpmvCap];
  const TACC sigma = (TACC)ctl.sigma[j];
  const int tiles = (N + kSpmvRows - 1) / kSpmvRows;
  for (int t = blockIdx.x; t < tiles; t += gridDim.x) {
    TACC acc, accd;
    spmv_tile<TA, TACC, DEFL>(
        N, t * kSpmvRows, rowptr, col, val, sval, scol,
        [&](int c) { return ld_as<TACC, TV>(x + c); }, agg, sdefl, acc, accd);
    const int row = t * kSpmvRows + threadIdx.x;
    if (row < N) w[row] = sigma * acc + accd;
  }
}

// --------------------------------------------------------------------------------------
// Multi-dot reduction helpers: warps split into nslice column slices x nrg row groups.
// --------------------------------------------------------------------------------------
__device__ __forceinline__ int slices_for(int k) {
  return k >= 8 ? 8 : (k >= 4 ? 4 : (k >= 2 ? 2 : 1));
}

// Number of columns of warp slice `slice` among k columns dealt round-robin to nslice
// slices.  Each warp runs an instance unrolled for exactly that many columns (a
// warp-uniform switch), so no floating-point instruction is issued under a false
// predicate: on GB300 a warp-wide FP64 FMA holds the narrow FP64 pipe for many cycles
// whether or not its lanes are enabled.
__device__ __forceinline__ int slice_cols(int k, int slice, int nslice) {
  return (k - slice + nslice - 1) / nslice;
}

// acc[i] += (column slice + nslice*i of V at `row`) * wv, for i < NW.
template <int NW, typename TV, typename TACC>
__device__ __forceinline__ void slice_fma(TACC (&acc)[kSliceCols], const TV* __restrict__ V,
                                          long long ldv, int slice, int nslice, int row,
                                          TACC wv) {
  TACC v[NW > 0 ? NW : 1];
#pragma unroll
  for (int i = 0; i < NW; ++i) v[i] = ld_as<TACC, TV>(V + (size_t)(slice + nslice * i) * ldv + row);
#pragma unroll
  for (int i = 0; i < NW; ++i) acc[i] += v[i] * wv;
}

// same, V from a shared-memory tile laid out [column][row of tile]
template <int NW, typename TV, typename TACC>
__device__ __forceinline__ void slice_fma_smem(TACC (&acc)[kSliceCols], const TV* sV, int ld,
                                               int slice, int nslice, int rr, TACC wv) {
#pragma unroll
  for (int i = 0; i < NW; ++i) acc[i] += cv<TACC, TV>(sV[(slice + nslice * i) * ld + rr]) * wv;
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
// accumulators (nw of them) transposed in shared memory and one thread adds the 32 lane
// values of a (warp, column) pair, which costs far fewer FP64 instructions than a
// shuffle tree on every lane; row groups are then added in a fixed order.
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
  for (int t = threadIdx.x; t < kSlices * kSliceCols; t += blockDim.x) {
    const int wv = t / kSliceCols, i = t % kSliceCols;
    if (i < slice_cols(k, wv % nslice, nslice)) {
      const double* src = sbuf + (size_t)t * 33;
      double s = 0.0;
      for (int l = 0; l < 32; ++l) s += src[l];
      swarp[t] = s;
    }
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

// CGS2 pass 1: h_c = sigma_c (u_c . w), coef_c = sigma_c h_c.
template <typename TV, typename TACC>
__global__ void __launch_bounds__(kThreads)
    k_dot1(int N, const TV* __restrict__ V, long long ldv, int k, const TACC* __restrict__ w,
           Ctl ctl) {
  if (ctl.flags[F_CYCLE_DONE]) return;
  __shared__ double sbuf[kSlices * kSliceCols * 33];
  __shared__ double swarp[kSlices * kSliceCols];
  __shared__ double sred[kMaxK];
  __shared__ double tot[kMaxK];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nslice = slices_for(k), nrg = kSlices / nslice;
  const int slice = warp % nslice, rg = warp / nslice;
  TACC acc[kSliceCols];
#pragma unroll
  for (int i = 0; i < kSliceCols; ++i) acc[i] = 0;
  const int nw = slice_cols(k, slice, nslice);
  const int tiles = (N + 255) / 256;
  for (int t = blockIdx.x; t < tiles; t += gridDim.x) {
    for (int q = rg; q < 8; q += nrg) {
      const int row = t * 256 + q * 32 + lane;
      if (row < N) {
        const TACC wv = w[row];
#define GG_DOT1(NW) slice_fma<NW, TV, TACC>(acc, V, ldv, slice, nslice, row, wv)
        GG_SLICE_SWITCH(nw, GG_DOT1)
#undef GG_DOT1
      }
    }
  }
  reduce_slices(acc, nw, k, nslice, sbuf, swarp, sred);
  if (!last_block_reduce(sred, k, ctl.part, ctl.part2, ctl.ldp, ctl.ticket, tot)) return;
  for (int c = threadIdx.x; c < k; c += blockDim.x) {
    const double hc = ctl.sigma[c] * tot[c];
    ctl.h[c] = hc;
    ctl.coef[c] = ctl.sigma[c] * hc;
  }
}

// CGS2 pass 2: w -= sum_c coef_c u_c, then h'_c = sigma_c (u_c . w), h += h'.
// The tile of V is read from global memory once, kept in shared memory for the dot.
template <typename TV, typename TACC>
__global__ void __launch_bounds__(kThreads)
    k_upd1dot2(int N, const TV* __restrict__ V, long long ldv, int k, TACC* __restrict__ w,
               Ctl ctl) {
  if (ctl.flags[F_CYCLE_DONE]) return;
  extern __shared__ __align__(16) unsigned char smraw[];
  TACC* sw = reinterpret_cast<TACC*>(smraw);           // kTile2
  TACC* spart = sw + kTile2;                            // 2 * kTile2
  TV* sV = reinterpret_cast<TV*>(spart + 2 * kTile2);   // k * kTile2
  __shared__ double sbuf[kSlices * kSliceCols * 33];
  __shared__ double swarp[kSlices * kSliceCols];
  __shared__ double sred[kMaxK];
  __shared__ double tot[kMaxK];
  __shared__ TACC scoef[kMaxK];
  for (int c = threadIdx.x; c < k; c += blockDim.x) scoef[c] = (TACC)ctl.coef[c];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nslice = slices_for(k), nrg = kSlices / nslice;
  const int slice = warp % nslice, rg = warp / nslice;
  const int nw = slice_cols(k, slice, nslice);
  const int half = threadIdx.x >> 7, rl = threadIdx.x & (kTile2 - 1);
  const int kh = (k + 1) >> 1;
  const int c0 = half * kh, c1 = min(k, c0 + kh);
  TACC acc[kSliceCols];
#pragma unroll
  for (int i = 0; i < kSliceCols; ++i) acc[i] = 0;
  __syncthreads();
  const int tiles = (N + kTile2 - 1) / kTile2;
  for (int t = blockIdx.x; t < tiles; t += gridDim.x) {
    const int row = t * kTile2 + rl;
    TACC p = 0;
    if (row < N) {
#pragma unroll 4
      for (int c = c0; c < c1; ++c) {
        const TV v = V[(size_t)c * ldv + row];
        sV[c * kTile2 + rl] = v;
        p += cv<TACC, TV>(v) * scoef[c];
      }
    } else {
      for (int c = c0; c < c1; ++c) sV[c * kTile2 + rl] = zero_of<TV>();
    }
    spart[half * kTile2 + rl] = p;
    __syncthreads();
    if (half == 0) {
      TACC wn = 0;
      if (row < N) {
        wn = w[row] - (spart[rl] + spart[kTile2 + rl]);
        w[row] = wn;
      }
      sw[rl] = wn;
    }
    __syncthreads();
    for (int q = rg; q < kTile2 / 32; q += nrg) {
      const int rr = q * 32 + lane;
      const TACC wv = sw[rr];
#define GG_DOT2(NW) slice_fma_smem<NW, TV, TACC>(acc, sV, kTile2, slice, nslice, rr, wv)
      GG_SLICE_SWITCH(nw, GG_DOT2)
#undef GG_DOT2
    }
    __syncthreads();
  }
  reduce_slices(acc, nw, k, nslice, sbuf, swarp, sred);
  if (!last_block_reduce(sred, k, ctl.part, ctl.part2, ctl.ldp, ctl.ticket, tot)) return;
  for (int c = threadIdx.x; c < k; c += blockDim.x) {
    const double h2 = ctl.sigma[c] * tot[c];
    ctl.h[c] += h2;
    ctl.coef[c] = ctl.sigma[c] * h2;
  }
}

// Plane rotations and stopping tests of step j (Eqs. 12, 14), by the whole block: the
// column, rotations and gamma are staged in shared memory, one thread applies the
// rotations there (no dependent global-memory round trips), then all threads store.
__device__ void givens_step(Ctl& ctl, int j, int m, double hnext) {
  __shared__ double sh[kMaxK + 1], scs[kMaxK], ssn[kMaxK], sg[2];
  __shared__ int sdone;
  const int ldh = ctl.ldh;
  for (int i = threadIdx.x; i <= j; i += blockDim.x) {
    const double hi = ctl.h[i];
    sh[i] = hi;
    ctl.Hr[(size_t)i * ldh + j] = hi;
    if (i < j) {
      scs[i] = ctl.cs[i];
      ssn[i] = ctl.sn[i];
    }
  }
  if (threadIdx.x == 0) {
    ctl.Hr[(size_t)(j + 1) * ldh + j] = hnext;
    sg[0] = ctl.g[j];
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double hn2 = hnext * hnext;
    for (int i = 0; i <= j; ++i) hn2 += sh[i] * sh[i];
    for (int i = 0; i < j; ++i) {
      const double a = sh[i], b = sh[i + 1];
      sh[i] = scs[i] * a + ssn[i] * b;
      sh[i + 1] = -ssn[i] * a + scs[i] * b;
    }
    const double a = sh[j];
    double c = 1.0, sn = 0.0;
    if (hnext != 0.0) {
      const double rho = hypot(a, hnext);
      c = a / rho;
      sn = hnext / rho;
      sh[j] = rho;
    }
    sh[j + 1] = 0.0;
    scs[j] = c;
    ssn[j] = sn;
    const double gj = sg[0];
    sg[1] = -sn * gj;
    sg[0] = c * gj;
    const long long steps = ++ctl.counts[C_STEPS];
    ctl.flags[F_K] = j + 1;
    const double est = fabs(sg[1]) / ctl.scal[S_RHO0];
    ctl.scal[S_EST] = est;
    ctl.sigma[j + 1] = hnext > 0.0 ? 1.0 / hnext : 0.0;
    bool done = false;
    if (!isfinite(hnext) || !isfinite(est)) {
      ctl.flags[F_STATUS] = GMRES_ERR_NAN;
      ctl.flags[F_STOP] = 1;
      done = true;
    }
    if (hnext <= 1e-14 * sqrt(hn2)) done = true;  // breakdown: the Krylov space is invariant
    if (!ctl.flags[F_FIXED] && est <= ctl.scal[S_TOL]) done = true;
    if (ctl.flags[F_MIXED] && fabs(sg[1]) <= ctl.scal[S_INNER_TOL] * ctl.scal[S_BETA_CYCLE])
      done = true;
    if (steps >= ctl.counts[C_MAXIT]) done = true;
    if (j + 1 >= m) done = true;
    sdone = done ? 1 : 0;
  }
  __syncthreads();
  for (int i = threadIdx.x; i <= j + 1; i += blockDim.x) ctl.H[(size_t)i * ldh + j] = sh[i];
  if (threadIdx.x == 0) {
    ctl.cs[j] = scs[j];
    ctl.sn[j] = ssn[j];
    ctl.g[j] = sg[0];
    ctl.g[j + 1] = sg[1];
    if (sdone) ctl.flags[F_CYCLE_DONE] = 1;
  }
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
  // warp 0: tile starting at row r0 into stage st (lane 0 announces the bytes, the lanes
  // issue the column segments)
  __device__ void issue(int st, long long r0, const TV* V, long long ldv, const TACC* w) const {
    const int lane = threadIdx.x & 31;
    const uint32_t vb = (uint32_t)(TR * sizeof(TV)), wb = (uint32_t)(TR * sizeof(TACC));
    if (lane == 0) mbar_arrive_expect_tx(&bars[st], (uint32_t)k * vb + wb);
    __syncwarp();
    TV* dst = vt(st);
    for (int c = lane; c < k; c += 32)
      bulk_g2s(dst + (size_t)c * TR, V + (size_t)c * ldv + r0, vb, &bars[st]);
    if (lane == 0) bulk_g2s(wt(st), w + r0, wb, &bars[st]);
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
// body(stage, r0) for each.  Returns false (after recording GMRES_ERR_TIMEOUT and waiting,
// with a bound, for this block's copies still in flight) if a copy never completes.
template <typename TV, typename TACC, typename F>
__device__ bool ring_run(const Ring<TV, TACC>& R, int N, const TV* V, long long ldv,
                         const TACC* w, Ctl& ctl, F&& body) {
  const int tiles = (N + R.TR - 1) / R.TR;
  const int nt = (int)blockIdx.x < tiles ? (tiles - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;
  if (threadIdx.x == 0) {
    for (int st = 0; st < R.S; ++st) mbar_init(&R.bars[st], 1);
    mbar_fence_init();
  }
  __syncthreads();
  if (threadIdx.x < 32)
    for (int i = 0; i < nt && i < R.S; ++i)
      R.issue(i, (long long)(blockIdx.x + (size_t)i * gridDim.x) * R.TR, V, ldv, w);
  int i = 0;
  bool ok = true;
  for (; i < nt; ++i) {
    const int st = i % R.S;
    ok = __syncthreads_and(mbar_wait(&R.bars[st], (uint32_t)((i / R.S) & 1)));
    if (!ok) break;
    body(st, (long long)(blockIdx.x + (size_t)i * gridDim.x) * R.TR);
    __syncthreads();
    if (threadIdx.x < 32 && i + R.S < nt)
      R.issue(st, (long long)(blockIdx.x + (size_t)(i + R.S) * gridDim.x) * R.TR, V, ldv, w);
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
#pragma unroll
  for (int e = 0; e < VN; ++e) spart[sub * TR + r + e] = p[e];
}

template <typename TACC> __host__ __device__ constexpr int update_splits(int TR, int VN) {
  // column subsets per row group: FP64 keeps the combine short (the FP64 pipe is the
  // bound), FP32 spreads the work over more threads
  return (kThreads / (TR / VN)) < (sizeof(TACC) == 8 ? 2 : 4) ? (kThreads / (TR / VN))
                                                              : (sizeof(TACC) == 8 ? 2 : 4);
}

// CGS2 pass 1 (pipelined): h_c = sigma_c (u_c . w), coef_c = sigma_c h_c.
template <typename TV, typename TACC>
__global__ void __launch_bounds__(kThreads)
    k_pass1(int N, const TV* __restrict__ V, long long ldv, int k, int TR,
            const TACC* __restrict__ w, Ctl ctl) {
  if (ctl.flags[F_CYCLE_DONE]) return;
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
  const bool ok = ring_run(R, N, V, ldv, w, ctl, [&](int st, long long) {
#define GG_P1(NW) tile_dot<NW, TV, TACC>(acc, R.vt(st), R.wt(st), TR, warp, lane)
    GG_SLICE_SWITCH(nw, GG_P1)
#undef GG_P1
  });
  if (!ok) return;
  reduce_slices(acc, nw, k, kSlices, reinterpret_cast<double*>(smraw), swarp, sred);
  if (!last_block_reduce(sred, k, ctl.part, ctl.part2, ctl.ldp, ctl.ticket, tot)) return;
  for (int c = threadIdx.x; c < k; c += blockDim.x) {
    const double hc = ctl.sigma[c] * tot[c];
    ctl.h[c] = hc;
    ctl.coef[c] = ctl.sigma[c] * hc;
  }
}

// CGS2 pass 2 (pipelined): w -= sum_c coef_c u_c; h'_c = sigma_c (u_c . w); h += h'.
template <typename TV, typename TACC>
__global__ void __launch_bounds__(kThreads)
    k_pass2(int N, const TV* __restrict__ V, long long ldv, int k, int TR,
            TACC* __restrict__ w, Ctl ctl) {
  if (ctl.flags[F_CYCLE_DONE]) return;
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
  for (int c = threadIdx.x; c < k; c += blockDim.x) scoef[c] = (TACC)ctl.coef[c];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nw = slice_cols(k, warp, kSlices);
  const int P = update_splits<TACC>(TR, VN);
  const int ng = TR / VN;
  TACC acc[kSliceCols];
#pragma unroll
  for (int i = 0; i < kSliceCols; ++i) acc[i] = 0;
  const bool ok = ring_run(R, N, V, ldv, (const TACC*)w, ctl, [&](int st, long long r0) {
    const TV* sV = R.vt(st);
    const TACC* sw = R.wt(st);
    tile_update<TV, TACC>(sV, TR, k, scoef, spart, P);
    __syncthreads();
    if ((int)threadIdx.x < ng) {
      const int r = threadIdx.x * VN;
#pragma unroll
      for (int e = 0; e < VN; ++e) {
        TACC acc_p = spart[r + e];
        for (int q = 1; q < P; ++q) acc_p += spart[q * TR + r + e];
        const TACC wn = sw[r + e] - acc_p;
        sw2[r + e] = wn;
        if (r0 + r + e < N) w[r0 + r + e] = wn;
      }
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
  if (ctl.flags[F_CYCLE_DONE]) return;
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
  for (int c = threadIdx.x; c < k; c += blockDim.x) scoef[c] = (TACC)ctl.coef[c];
  const int P = update_splits<TACC>(TR, VN);
  const int ng = TR / VN;
  TV* __restrict__ vout = V + (size_t)k * ldv;
  TACC nrm = 0;
  const bool ok = ring_run(R, N, (const TV*)V, ldv, w, ctl, [&](int st, long long r0) {
    const TV* sV = R.vt(st);
    const TACC* sw = R.wt(st);
    tile_update<TV, TACC>(sV, TR, k, scoef, spart, P);
    __syncthreads();
    if ((int)threadIdx.x < ng) {
      const int r = threadIdx.x * VN;
#pragma unroll
      for (int e = 0; e < VN; ++e) {
        if (r0 + r + e < N) {
          TACC acc_p = spart[r + e];
          for (int q = 1; q < P; ++q) acc_p += spart[q * TR + r + e];
          const TACC wn = sw[r + e] - acc_p;
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
  givens_step(ctl, k - 1, m, sqrt(tot[0]));
}

// CGS2 pass 3: u_{j+1} = w - sum_c coef_c u_c (stored), h_{j+1,j} = ||u_{j+1}||.
template <typename TV, typename TACC>
__global__ void __launch_bounds__(kThreads)
    k_upd2norm(int N, TV* __restrict__ V, long long ldv, int k, const TACC* __restrict__ w,
               Ctl ctl, int m) {
  if (ctl.flags[F_CYCLE_DONE]) return;
  __shared__ TACC scoef[kMaxK];
  __shared__ double sbuf[kThreads / 32];
  __shared__ double sred[1];
  __shared__ double tot[1];
  for (int c = threadIdx.x; c < k; c += blockDim.x) scoef[c] = (TACC)ctl.coef[c];
  __syncthreads();
  TV* __restrict__ vout = V + (size_t)k * ldv;
  TACC nrm = 0;
  for (int row = blockIdx.x * blockDim.x + threadIdx.x; row < N; row += gridDim.x * blockDim.x) {
    TACC p0 = 0, p1 = 0, p2 = 0, p3 = 0;
    int c = 0;
    for (; c + 3 < k; c += 4) {
      const TACC v0 = ld_as<TACC, TV>(V + (size_t)c * ldv + row);
      const TACC v1 = ld_as<TACC, TV>(V + (size_t)(c + 1) * ldv + row);
      const TACC v2 = ld_as<TACC, TV>(V + (size_t)(c + 2) * ldv + row);
      const TACC v3 = ld_as<TACC, TV>(V + (size_t)(c + 3) * ldv + row);
      p0 += v0 * scoef[c];
      p1 += v1 * scoef[c + 1];
      p2 += v2 * scoef[c + 2];
      p3 += v3 * scoef[c + 3];
    }
    for (; c < k; ++c) p0 += ld_as<TACC, TV>(V + (size_t)c * ldv + row) * scoef[c];
    const TACC wn = w[row] - ((p0 + p1) + (p2 + p3));
    TV st;
    if constexpr (sizeof(TV) == sizeof(TACC)) {
      st = (TV)wn;
    } else {
      st = st_round<TV>((float)wn);
    }
    vout[row] = st;
    const TACC sv = cv<TACC, TV>(st);
    nrm += sv * sv;
  }
  const double bs = block_sum((double)nrm, sbuf);
  if (threadIdx.x == 0) sred[0] = bs;
  __syncthreads();
  if (!last_block_reduce(sred, 1, ctl.part, ctl.part2, ctl.ldp, ctl.ticket, tot)) return;
  givens_step(ctl, k - 1, m, sqrt(tot[0]));
}

// --------------------------------------------------------------------------------------
// Deflation: U^T x by pieces (warp per piece), then s = U (|mu| T^-1 - I) c.
// --------------------------------------------------------------------------------------
template <typename TX>
__global__ void __launch_bounds__(kThreads)
    k_aggsum(const TX* __restrict__ x, Defl d, double* __restrict__ cpart, const int* flags,
             int skip_slot) {
  if (flags[skip_slot]) return;
  const int lane = threadIdx.x & 31;
  const int p = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (p >= d.npieces) return;
  const int s = d.piece_start[p], e = d.piece_start[p + 1];
  double acc = 0.0;
  for (int t = s + lane; t < e; t += 32) acc += ld_as<double, TX>(x + d.perm[t]);
  acc = warp_sum(acc);
  if (lane == 0) cpart[p] = acc;
}

// c_a = scale uscale_a sum(pieces of a);  s_a = uscale_a (|mu| (T^-1 c)_a - c_a).
__global__ void __launch_bounds__(kThreads)
    k_coarse(Defl d, const double* __restrict__ cpart, const double* __restrict__ scale_ptr,
             Ctl ctl, int skip_slot) {
  if (ctl.flags[skip_slot]) return;
  extern __shared__ double sc[];
  const double scale = scale_ptr ? *scale_ptr : 1.0;
  const double mu = ctl.scal[S_MU];
  const int r = d.r;
  for (int a = threadIdx.x; a < r; a += blockDim.x) {
    double s = 0.0;
    for (int p = d.agg_piece[a]; p < d.agg_piece[a + 1]; ++p) s += cpart[p];
    sc[a] = scale * d.uscale[a] * s;
  }
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int nw = (gridDim.x * blockDim.x) >> 5;
  for (int a = gw; a < r; a += nw) {
    const double* row = d.tinv + (size_t)a * r;
    double acc = 0.0;
    for (int b = lane; b < r; b += 32) acc += __ldg(row + b) * sc[b];
    acc = warp_sum(acc);
    if (lane == 0) {
      const double sd = d.uscale[a] * (mu * acc - sc[a]);
      ctl.sdefl[a] = sd;
      ctl.sdefl32[a] = (float)sd;
    }
  }
}

// --------------------------------------------------------------------------------------
// Cycle end
// --------------------------------------------------------------------------------------
// Back substitution R_k y = g (Eq. 12) on a shared-memory copy of R; coef = sigma o y.
__global__ void k_backsolve(Ctl ctl) {
  __shared__ double R[kMaxM * kMaxM];
  __shared__ double sg[kMaxM], sy[kMaxM];
  if (ctl.flags[F_STOP]) return;
  const int k = ctl.flags[F_K];
  const int ldh = ctl.ldh;
  for (int t = threadIdx.x; t < k * k; t += blockDim.x) {
    const int i = t / k, l = t % k;
    R[t] = l >= i ? ctl.H[(size_t)i * ldh + l] : 0.0;
  }
  for (int i = threadIdx.x; i < k; i += blockDim.x) sg[i] = ctl.g[i];
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int i = k - 1; i >= 0; --i) {
      double s = sg[i];
      for (int l = i + 1; l < k; ++l) s -= R[i * k + l] * sy[l];
      sy[i] = s / R[i * k + i];
    }
    ctl.counts[C_CYCLES]++;
  }
  __syncthreads();
  for (int i = threadIdx.x; i < k; i += blockDim.x) {
    ctl.y[i] = sy[i];
    ctl.coef[i] = ctl.sigma[i] * sy[i];
  }
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

// True residual in FP64 (Eq. 15): r = b - A x, u_0 = r stored in the basis precision,
// rho0 on the first call, convergence / maxit decision, and the start of a new cycle.
template <typename TV>
__global__ void __launch_bounds__(kSpmvRows)
    k_residual(int N, const int* __restrict__ rowptr, const int* __restrict__ col,
               const double* __restrict__ val, const double* __restrict__ x,
               const double* __restrict__ b, TV* __restrict__ V0, Ctl ctl) {
  if (ctl.flags[F_STOP]) return;
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
  double b1 = block_sum(n1, sbuf);
  double b2 = (sizeof(TV) == sizeof(double)) ? b1 : block_sum(n2, sbuf);
  if (threadIdx.x == 0) {
    sred[0] = b1;
    sred[1] = b2;
  }
  __syncthreads();
  if (!last_block_reduce(sred, 2, ctl.part, ctl.part2, ctl.ldp, ctl.ticket, tot)) return;
  if (threadIdx.x != 0) return;
  const double beta = sqrt(tot[0]);
  const double beta_s = sqrt(tot[1]);
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
  const int n = ctl.flags[F_K];
  const int lane = threadIdx.x;
  if (n <= 0) return;
  const int ldh = ctl.ldh;
#define AA(i, j) A[(i) * n + (j)]
  for (int t = lane; t < n * n; t += 32) AA(t / n, t % n) = ctl.Hr[(size_t)(t / n) * ldh + t % n];
  if (lane == 0) { smod = 0.0; sfail = 0; }
  __syncwarp();
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
      if (lane == 0) smod = fmax(smod, fabs(AA(hi, hi)));
      __syncwarp();
      --hi;
      its = 0;
      continue;
    }
    if (l == hi - 1) {
      const double a = AA(hi - 1, hi - 1), b = AA(hi - 1, hi), c = AA(hi, hi - 1), d = AA(hi, hi);
      const double p = 0.5 * (a - d), disc = p * p + b * c, mid = 0.5 * (a + d);
      double m2;
      if (disc >= 0.0) {
        const double q = sqrt(disc);
        const double l1 = mid + (p >= 0.0 ? q : -q);
        const double l2 = (l1 != 0.0) ? (a * d - b * c) / l1 : mid - (p >= 0.0 ? q : -q);
        m2 = fmax(fabs(l1), fabs(l2));
      } else {
        m2 = hypot(mid, sqrt(-disc));
      }
      if (lane == 0) smod = fmax(smod, m2);
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
  if (lane == 0) {
    if (sfail || !(smod > 0.0) || !isfinite(smod)) {
      ctl.flags[F_STATUS] = GMRES_ERR_SINGULAR_COARSE;
      ctl.flags[F_STOP] = 1;
    } else {
      ctl.scal[S_MU] = smod;
    }
  }
}

__global__ void k_init(Ctl ctl, double tol, double inner_tol, double r0ref, double mu,
                       int fixed, int mixed, long long maxit) {
  if (threadIdx.x != 0) return;
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

template <typename TV, typename TA, typename TACC>
struct Kern {
  struct Grids {
    int spmv_d = 0, spmv_n = 0, dot1 = 0, upd2 = 0, resid = 0, xupd_d = 0, xupd_n = 0,
        xapply = 0, aggsum = 0;
    int upd1[kMaxK + 1] = {0};
    int tr[kMaxK + 1] = {0};
    int p1[kMaxK + 1] = {0}, p2[kMaxK + 1] = {0}, p3[kMaxK + 1] = {0};
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
      g.spmv_d = resident_grid(k_spmv_step<TA, TV, TACC, true>, kSpmvRows, 0, sms);
      g.spmv_n = resident_grid(k_spmv_step<TA, TV, TACC, false>, kSpmvRows, 0, sms);
      g.dot1 = resident_grid(k_dot1<TV, TACC>, kThreads, 0, sms);
      g.upd2 = resident_grid(k_upd2norm<TV, TACC>, kThreads, 0, sms);
      g.resid = resident_grid(k_residual<TV>, kSpmvRows, 0, sms);
      g.xupd_d = resident_grid(k_xupdate<TV, true>, kThreads, 0, sms);
      g.xupd_n = resident_grid(k_xupdate<TV, false>, kThreads, 0, sms);
      g.xapply = resident_grid(k_xapply, kThreads, 0, sms);
      for (int k = 1; k <= kMaxK; ++k) {
        g.upd1[k] = resident_grid(k_upd1dot2<TV, TACC>, kThreads, smem_upd1(k), sms);
        g.tr[k] = tile_rows(k);
        g.p1[k] = resident_grid(k_pass1<TV, TACC>, kThreads, ring_smem(k), sms);
        g.p2[k] = resident_grid(k_pass2<TV, TACC>, kThreads, ring_smem(k), sms);
        g.p3[k] = resident_grid(k_pass3<TV, TACC>, kThreads, ring_smem(k), sms);
      }
      for_sms = sms;
    }
    return g;
  }
  static size_t smem_upd1(int k) {
    return sizeof(TACC) * 3 * kTile2 + sizeof(TV) * (size_t)k * kTile2;
  }
  static const TA* vals(const CycleArgs& a) {
    if constexpr (sizeof(TA) == sizeof(double)) return a.op.val;
    else return a.op.val32;
  }
  static const TACC* sdefl(const CycleArgs& a) {
    if constexpr (sizeof(TACC) == sizeof(double)) return a.ctl.sdefl;
    else return a.ctl.sdefl32;
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
        const int tiles = (N + kSpmvRows - 1) / kSpmvRows;
        const TV* xj = V + (size_t)j * a.ldv;
        if (defl)
          k_spmv_step<TA, TV, TACC, true><<<balanced(tiles, g.spmv_d), kSpmvRows, 0, st>>>(
              N, a.op.rowptr, a.op.col, vals(a), xj, j, d.agg, sdefl(a), w, a.ctl);
        else
          k_spmv_step<TA, TV, TACC, false><<<balanced(tiles, g.spmv_n), kSpmvRows, 0, st>>>(
              N, a.op.rowptr, a.op.col, vals(a), xj, j, nullptr, sdefl(a), w, a.ctl);
        nl = 1;
        break;
      }
      case PH_DOT1: {
        const int tr = g.tr[k];
        k_pass1<TV, TACC><<<grid_for((N + tr - 1) / tr, 1, g.p1[k]), kThreads, ring_smem(k), st>>>(
            N, V, a.ldv, k, tr, w, a.ctl);
        nl = 1;
        break;
      }
      case PH_UPD1DOT2: {
        const int tr = g.tr[k];
        k_pass2<TV, TACC><<<grid_for((N + tr - 1) / tr, 1, g.p2[k]), kThreads, ring_smem(k), st>>>(
            N, V, a.ldv, k, tr, w, a.ctl);
        nl = 1;
        break;
      }
      case PH_UPD2NORM: {
        const int tr = g.tr[k];
        k_pass3<TV, TACC><<<grid_for((N + tr - 1) / tr, 1, g.p3[k]), kThreads, ring_smem(k), st>>>(
            N, Vm, a.ldv, k, tr, w, a.ctl, a.m);
        nl = 1;
        break;
      }
      case PH_DEFL: {  // U^T v_j and the correction for column j
        const TV* xj = V + (size_t)j * a.ldv;
        k_aggsum<TV><<<(d.npieces + 7) / 8, kThreads, 0, st>>>(xj, d, a.ctl.cpart, a.ctl.flags,
                                                              F_CYCLE_DONE);
        k_coarse<<<a.grid_small, kThreads, sizeof(double) * d.r, st>>>(
            d, a.ctl.cpart, a.ctl.sigma + j, a.ctl, F_CYCLE_DONE);
        nl = 2;
        break;
      }
      case PH_CYCLE_END: {
        k_backsolve<<<1, 128, 0, st>>>(a.ctl);
        const int tiles = (N + kThreads - 1) / kThreads;
        if (defl) {
          k_xupdate<TV, true><<<grid_for(tiles, 1, g.xupd_d), kThreads, 0, st>>>(N, V, a.ldv, x,
                                                                                a.t, a.ctl);
          k_aggsum<double><<<(d.npieces + 7) / 8, kThreads, 0, st>>>(a.t, d, a.ctl.cpart,
                                                                    a.ctl.flags, F_STOP);
          k_coarse<<<a.grid_small, kThreads, sizeof(double) * d.r, st>>>(d, a.ctl.cpart,
                                                                        nullptr, a.ctl, F_STOP);
          k_xapply<<<grid_for(tiles, 1, g.xapply), kThreads, 0, st>>>(N, x, a.t, d.agg, a.ctl);
          nl = 5;
        } else {
          k_xupdate<TV, false><<<grid_for(tiles, 1, g.xupd_n), kThreads, 0, st>>>(N, V, a.ldv,
                                                                                 x, a.t, a.ctl);
          nl = 2;
        }
        break;
      }
      case PH_RESIDUAL:
        k_residual<TV><<<balanced((N + kSpmvRows - 1) / kSpmvRows, g.resid), kSpmvRows, 0,
                         st>>>(N, a.op.rowptr, a.op.col, a.op.val, x, b, Vm, a.ctl);
        nl = 1;
        break;
      case PH_RITZ:
        k_ritz<<<1, 32, 0, st>>>(a.ctl);
        nl = 1;
        break;
      default:
        return cudaErrorInvalidValue;
    }
    if (launches) *launches += nl;
    return cudaGetLastError();
  }

  static cudaError_t prepare() {
    // the passes may need more than the default 48 KB of dynamic shared memory
    cudaError_t e = cudaFuncSetAttribute(k_upd1dot2<TV, TACC>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem_upd1(kMaxK));
    size_t mx = 0;
    for (int k = 1; k <= kMaxK; ++k) mx = ring_smem(k) > mx ? ring_smem(k) : mx;
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(k_pass1<TV, TACC>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)mx);
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

cudaError_t launch_phase(const CycleArgs& a, int ph, int j, bool defl, double* x,
                         const double* b, cudaStream_t st, int* launches) {
  switch (a.prec) {
    case P_FP64: return K64::phase(a, ph, j, defl, x, b, st, launches);
    case P_FP32: return K32::phase(a, ph, j, defl, x, b, st, launches);
    default: return K16::phase(a, ph, j, defl, x, b, st, launches);
  }
}

}  // namespace gg
