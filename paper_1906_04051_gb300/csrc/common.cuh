// common.cuh -- shared device helpers of the GB300 GMRES library (sm_103a).
//
// Reductions here are deterministic: every partial sum is formed in a fixed order
// (per-lane strided loops, then an xor-shuffle tree, then fixed-order combination of
// warps and blocks), so two runs with the same launch shape give bitwise equal results.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/gmres_gb300.h"

namespace gg {

constexpr int kWarp = 32;
constexpr int kMaxM = 64;               // largest restart length m
constexpr int kMaxK = kMaxM + 1;        // basis columns held in a cycle
constexpr int kMaxAdapt = 32;           // most columns of the adaptive deflation space
constexpr int kVecLanes = 4;          // lanes per row of the CSR SpMV for long rows
constexpr int kVecRows = 2;           // consecutive rows per lane group (taken in turn)
constexpr int kVecMinRowLen = 16;     // mean row length from which it is used
constexpr int kMaxR = 6144;             // largest number of deflation aggregates
constexpr int kThreads = 256;           // threads of the streaming kernels
constexpr int kSlices = 8;              // column slices of a multi-dot (one per warp)
constexpr int kSliceCols = (kMaxK + kSlices - 1) / kSlices;  // 9 accumulators / thread
constexpr int kPiece = 1024;            // nodes per piece of an aggregate sum
// rows per unit of the fused Arnoldi kernel's row partition (block b owns the units
// [floor(b U / G), floor((b + 1) U / G)) of the U = ldv / kPartUnit): the FP32 chunk of 128
// rows, so that no block owns more than 128 rows above the mean
constexpr int kPartUnit = 128;

// ---- named slots of the solver control block (device memory) ----
enum ScalarSlot {
  S_RHO0 = 0,     // reference norm of the relative tolerance (Eq. 15)
  S_BETA,         // true residual norm at the start of the current cycle
  S_BETA_CYCLE,   // norm of the stored start vector (g_0 of the cycle)
  S_MU,           // |mu| of the EBP preconditioner
  S_TOL,
  S_INNER_TOL,
  S_EST,          // |gamma_{k+1}| / rho0 of the last step
  S_TRUE,         // true relative residual of the last residual evaluation
  S_R0REF,        // user reference norm (0 = none)
  S_GIV_A,        // t_j: entry j of the step's column after the earlier rotations
  S_GIV_HN2,      // sum of h_ij^2 over i <= j (breakdown test)
  S_NSCAL = 16
};
enum FlagSlot {
  F_CYCLE_DONE = 0,  // the current cycle has ended (remaining step launches return)
  F_STOP,            // the solve has ended
  F_STATUS,          // gmres_status of the solve so far
  F_K,               // Arnoldi steps done in the current cycle
  F_FIXED,           // fixed-iteration protocol
  F_MIXED,           // inner-tolerance test active (mixed precision)
  F_RHO0_SET,
  F_DEFL_ON,         // the EBP correction is active (batched driver; set by the Ritz step)
  F_NFLAGS = 16
};
enum CountSlot { C_STEPS = 0, C_CYCLES, C_REFINE, C_MAXIT, C_QDEF, C_NCOUNT = 8 };  // C_QDEF: columns of the adaptive U

// Device control block: all pointers into library-owned device memory.
struct Ctl {
  double* H;      // (ldh+1) x ldh row-major, Hessenberg columns after rotation (R)
  double* Hr;     // same shape, Hessenberg as built (for the Ritz values)
  double* g;      // ldh+1: rotated right-hand side beta e1
  double* cs;     // ldh: rotation cosines
  double* sn;     // ldh: rotation sines
  double* y;      // ldh: least-squares solution of the cycle
  double* sigma;  // ldh+1: basis scales, v_c = sigma_c * V[:, c]
  double* h;      // ldh+1: projection coefficients of the current column
  double* coef;   // ldh+1: coefficients of the pending basis update
  double* part;   // [max_grid][ldp] per-block partial sums
  double* part2;  // [kMaxGroups][ldp] per-group partial sums
  double* scal;   // S_NSCAL scalars
  double* cpart;  // per-piece partial sums of an aggregate reduction
  double* sdefl;  // r: correction per aggregate, z = v + sdefl[agg]
  float* sdefl32; // r: FP32 copy for the FP32 inner kernels
  int* flags;     // F_NFLAGS
  unsigned* ticket;         // 1 + kMaxGroups last-block counters (zero between kernels)
  long long* counts;        // C_NCOUNT
  int ldh;        // m of the workspace
  int ldp;        // leading dimension of part (>= 2 kMaxK + 1)
  double* L;      // one-reduction MGS: kMaxK x kMaxK, L[i][c] = v_i . v_c (c < i) of the cycle
};

// Epilogue of a multi-dot kernel: the Arnoldi coefficients, the adaptive deflation's
// coarse correction s = |mu| T^-1 c - c (into ctl.sdefl), or the raw dots (into out).
enum { kEpiArnoldi = 0, kEpiCoarse = 1, kEpiRaw = 2, kEpiIcwy = 3 };
struct DotEpi {
  int mode;
  const double* tinv;  // kEpiCoarse: k x k, row stride ldt
  int ldt;
  double* out;         // kEpiRaw
  int skip_slot;       // flag that ends the launch at once (F_CYCLE_DONE, F_STOP, -1)
};

// Deflation data of one operator (A or A^T).
// Diagonal storage of a banded operator: a_{i, i + off[d]} = dval[d * ldd + i].
constexpr int kMaxDiag = 32;
struct DiaOffsets {
  int nd;
  int off[kMaxDiag];
};

struct Defl {
  int r;                  // number of aggregates (0 = none)
  const int* agg;         // N
  const int* perm;        // nodes sorted by aggregate, then index
  const int* piece_start; // npieces + 1 offsets into perm
  const int* agg_piece;   // r + 1 offsets into the piece list
  const double* uscale;   // r: 1/sqrt|agg_p|
  const double* tinv;     // r x r row-major T^-1
  const float* tinv32;    // its FP32 copy (FP32 / BF16 solves), may be null
  int npieces;
  // the pieces of each block of the fused Arnoldi kernel (a grid of blk_grid blocks owning
  // consecutive row ranges; pieces are split at those ranges): block b's pieces are
  // blk_piece[blk_piece_start[b] .. blk_piece_start[b + 1]), in aggregate order
  const int* blk_piece_start;
  const int* blk_piece;
  int blk_grid;
  // A W (W = the 0/1 aggregate indicator) in CSR: row i holds, for each aggregate a met
  // in row i of A, the sum of the row's entries in the columns of a
  const int* aurp;        // N + 1
  const int* aucol;       // aggregate ids
  const double* auval;
  const float* auval32;   // FP32 copy (FP32 inner), may be null
  // the same rows' first two entries in two planes of n (plane q at q * n): column -1 when
  // absent; plane 1 holds -(column) - 2 when the row has more entries (from aurp[i] + 2)
  const int* aup_col;
  const double* aup_val;
  const float* aup_val32;  // may be null
  // adaptive deflation: U and A U dense (qd columns of ldu rows), T^-1 (qd x qd); the
  // step's coarse term is sum_t aud[t][i] s'_t instead of the A W row
  const double* ud;
  const double* aud;
  const double* tinv_a;
  long long ldu;
  int qd;
};

// ---- element-type helpers ----
template <typename T> __device__ __forceinline__ float to_f(T v);
template <> __device__ __forceinline__ float to_f<float>(float v) { return v; }
template <> __device__ __forceinline__ float to_f<__nv_bfloat16>(__nv_bfloat16 v) {
  return __bfloat162float(v);
}

template <typename TACC, typename T> __device__ __forceinline__ TACC ld_as(const T* p);
template <> __device__ __forceinline__ double ld_as<double, double>(const double* p) { return __ldg(p); }
template <> __device__ __forceinline__ float ld_as<float, float>(const float* p) { return __ldg(p); }
template <> __device__ __forceinline__ float ld_as<float, __nv_bfloat16>(const __nv_bfloat16* p) {
  return __bfloat162float(__ldg(p));
}
template <> __device__ __forceinline__ double ld_as<double, float>(const float* p) {
  return (double)__ldg(p);
}
template <> __device__ __forceinline__ double ld_as<double, __nv_bfloat16>(const __nv_bfloat16* p) {
  return (double)__bfloat162float(__ldg(p));
}

// value conversion (registers / shared memory)
template <typename TACC, typename T> __device__ __forceinline__ TACC cv(T v);
template <> __device__ __forceinline__ double cv<double, double>(double v) { return v; }
template <> __device__ __forceinline__ float cv<float, float>(float v) { return v; }
template <> __device__ __forceinline__ float cv<float, __nv_bfloat16>(__nv_bfloat16 v) {
  return __bfloat162float(v);
}
template <> __device__ __forceinline__ double cv<double, float>(float v) { return (double)v; }
template <> __device__ __forceinline__ double cv<double, __nv_bfloat16>(__nv_bfloat16 v) {
  return (double)__bfloat162float(v);
}

template <typename T> __device__ __forceinline__ T zero_of() { return T(0); }
template <> __device__ __forceinline__ __nv_bfloat16 zero_of<__nv_bfloat16>() {
  return __float2bfloat16_rn(0.0f);
}

// plain (coherent) load: for data written earlier in the same kernel launch
template <typename TACC, typename T> __device__ __forceinline__ TACC ld_cg(const T* p);
template <> __device__ __forceinline__ double ld_cg<double, double>(const double* p) { return __ldcg(p); }
template <> __device__ __forceinline__ float ld_cg<float, float>(const float* p) { return __ldcg(p); }

template <typename T> __device__ __forceinline__ T st_round(float v);
template <> __device__ __forceinline__ float st_round<float>(float v) { return v; }
template <> __device__ __forceinline__ __nv_bfloat16 st_round<__nv_bfloat16>(float v) {
  return __float2bfloat16_rn(v);
}

template <typename T> __device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

template <typename T> __device__ __forceinline__ T warp_max(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

__device__ __forceinline__ bool finite_d(double v) { return isfinite(v); }

// Block-wide sum of one value per thread (fixed tree); result valid in all threads.
template <typename T>
__device__ __forceinline__ T block_sum(T v, T* sbuf /* >= blockDim/32 */) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  v = warp_sum(v);
  __syncthreads();
  if (lane == 0) sbuf[warp] = v;
  __syncthreads();
  T t = 0;
  const int nw = blockDim.x >> 5;
  for (int w = 0; w < nw; ++w) t += sbuf[w];
  return t;
}

constexpr int kGroup = 32;      // blocks per first-level group of a grid reduction
constexpr int kMaxGroups = 64;  // groups per grid (grid <= kGroup * kMaxGroups)

// dst[c] = sum_{r < nrows} src[r * ldp + c] for c < ncols, in a fixed order: the Q
// threads of a column (Q a power of two, consecutive lanes) sum rows q, q + Q, ... with
// two accumulators and independent loads, then combine by shuffles (no block barriers).
__device__ __forceinline__ void reduce_rows(const double* src, int nrows, int ncols, int ldp,
                                            double* dst) {
  int Q = 1;
  while (Q * 2 <= 32 && Q * 2 * ncols <= (int)blockDim.x) Q *= 2;
  const int lanes = ncols * Q;
  const int rounds = (lanes + blockDim.x - 1) / blockDim.x;
  for (int rd = 0; rd < rounds; ++rd) {
    const int idx = rd * blockDim.x + threadIdx.x;
    const int c = idx / Q, q = idx % Q;
    double s0 = 0.0, s1 = 0.0;
    if (c < ncols) {
      int r = q;
      for (; r + Q < nrows; r += 2 * Q) {
        s0 += __ldcg(src + (size_t)r * ldp + c);
        s1 += __ldcg(src + (size_t)(r + Q) * ldp + c);
      }
      if (r < nrows) s0 += __ldcg(src + (size_t)r * ldp + c);
    }
    double v = s0 + s1;
    for (int o = 1; o < Q; o <<= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (c < ncols && q == 0) dst[c] = v;
  }
  __syncthreads();
}

// Grid-wide deterministic reduction of per-block vectors.  Each block writes its ncols
// partials (smem sred) to part[blockIdx.x * ldp + c].  The last block of each group of
// kGroup blocks (ticket counters) sums its group into part2[group]; the last group to
// finish sums the group partials into tot[c] (shared memory), resets the counters and
// returns true.  Every other block returns false.  No block ever waits on another.
__device__ __forceinline__ bool last_block_reduce(const double* sred, int ncols, double* part,
                                                  double* part2, int ldp, unsigned* tickets,
                                                  double* tot) {
  __shared__ unsigned s_last;
  const int G = gridDim.x, b = blockIdx.x;
  const int ng = (G + kGroup - 1) / kGroup, g = b / kGroup;
  const int gs = (G - g * kGroup) < kGroup ? (G - g * kGroup) : kGroup;
  for (int c = threadIdx.x; c < ncols; c += blockDim.x) part[(size_t)b * ldp + c] = sred[c];
  __syncthreads();
  if (threadIdx.x == 0) {  // the block's writes are ordered before thread 0's fence
    __threadfence();
    s_last = (atomicAdd(&tickets[1 + g], 1u) == (unsigned)gs - 1u) ? 1u : 0u;
    if (s_last) __threadfence();
  }
  __syncthreads();
  if (!s_last) return false;
  reduce_rows(part + (size_t)g * kGroup * ldp, gs, ncols, ldp, tot);
  for (int c = threadIdx.x; c < ncols; c += blockDim.x) part2[(size_t)g * ldp + c] = tot[c];
  __syncthreads();
  if (threadIdx.x == 0) {
    tickets[1 + g] = 0u;
    __threadfence();
    s_last = (atomicAdd(&tickets[0], 1u) == (unsigned)ng - 1u) ? 1u : 0u;
    if (s_last) __threadfence();
  }
  __syncthreads();
  if (!s_last) return false;
  reduce_rows(part2, ng, ncols, ldp, tot);
  if (threadIdx.x == 0) tickets[0] = 0u;
  __syncthreads();
  return true;
}

}  // namespace gg
