// fused.cu -- the Arnoldi steps of a restart cycle of deflated GMRES(m) in one persistent
// kernel: per step the SpMV w = A M^-1 v_j (Eq. 10 with Eqs. 16-17), the paper's modified
// Gram-Schmidt projections (Eq. 13) in their one-reduction form, ||w||, the plane rotations
// with the stopping tests (Eqs. 12, 14) and the coarse solve of the next step's
// preconditioner (Eq. 17: s' = U (|mu| T^-1 - I) U^T v_{j+1}).
//
// One block of 16 warps per multiprocessor, launched cooperatively (every block resident).
// Block b owns a contiguous range of rows (a multiple of 128) for the whole cycle, taken in
// super-tiles of at most RS rows whose slices of w and u_j stay in shared memory.  A step:
//   1. SpMV of the super-tile's rows (diagonal storage; the coarse correction through the
//      A W rows, s' staged in shared memory): w into shared memory (and global memory when
//      the update reads it there), u_j next to it.  Step 0's diagonal part runs before the
//      programmatic-launch wait, overlapping the coarse-solve kernel that produces its s'.
//   2. Multi-dot g = V^T w and the new row of L (u_j . u_c), streamed from HBM against the
//      shared-memory slices (FP64: four warps per column; FP32: row chunks over column
//      groups; double-FP32 on request).
//   3. Grid barrier 1; every block adds the G partial sums in the same order (identical
//      totals in every block) and solves (I + L) h = g itself.
//   4. Update of its rows, u_{j+1} = w - V (sigma o h), in the reverse order of step 2 (the
//      columns read last are the likeliest to be in L2); partial sums of ||u_{j+1}||^2 and
//      of u_{j+1} over the block's pieces of aggregates (U^T u_{j+1}).
//   5. Grid barrier 2; block 0 adds the norm partials and applies the rotations and the
//      stopping tests; the other blocks form c = U^T u_{j+1} from the piece sums and share
//      the rows of y = T^-1 c, giving s' for step j + 1.
//   6. A split barrier: each block arrives once its share of step 5 is published, forms the
//      diagonal part of the next step's SpMV (it needs only u_{j+1}), then waits for all
//      arrivals and reads the same stopping decision and sigma_{j+1}.
// Every reduction is formed in a fixed order: runs are bitwise reproducible.  The per-phase
// register budgets (loads in flight) are set so that the kernel needs no local memory:
// with 220 KB of shared memory per block, spilled registers would live in L2.
//
// The basis is streamed with plain vectorised loads rather than bulk asynchronous copies:
// measured on GB300, a multiprocessor fed by bulk copies reached about 10 bytes per clock,
// against the 22 that the HBM copy bandwidth asks of each of the 152.
#include <algorithm>
#include <type_traits>
#include <utility>

#include "internal.h"
#include "kernels.cuh"

namespace gg {

namespace {

constexpr int kArnWarps = 16;
constexpr int kArnThreads = kArnWarps * 32;
constexpr int kArnUnit = kPartUnit;              // rows per unit of the row partition
constexpr size_t kArnSmem = 220 * 1024;          // dynamic shared memory
// reductions: lane-wise totals [2][kMaxK][33] (FP64) or warp sums [2][16][kMaxK] (FP32)
constexpr size_t kArnScratch = 2 * kMaxK * 33 * sizeof(double);
constexpr size_t kArnStaging = 2 * 2 * 16 * 32 * sizeof(double);  // FP64 multi-dot staging
constexpr long long kArnSpins = 1LL << 21;       // polls of the barrier word: about a second
constexpr int kArnNormCol = 2 * kMaxK;           // column of ctl.part holding the norm partials
constexpr int kArnAwRows64 = 6;  // rows per thread of an A W gather batch: FP64 (CSR rows)
constexpr int kArnAwRows32 = 7;  // FP32 (row-indexed planes)
// 16-byte basis loads in flight per lane in the multi-dot: FP32 (bound by HBM) asks for
// more bytes in flight than FP64 (bound by its FMA pipe)
template <typename TV> constexpr int arn_loads() { return sizeof(TV) == 8 ? 6 : 12; }

template <typename TV, typename TACC>
struct ArnArgs {
  int N;          // rows of A
  int units;      // ldv / kArnUnit
  int jmax, m;    // steps of this cycle (<= m), restart length
  int pre;        // the predecessor is the coarse solve of step 0: the diagonal part of
                  // its SpMV may run before the wait
  int defl;       // add the coarse correction A W s'
  int r;          // aggregates (entries of s')
  int RS;         // rows per super-tile (a multiple of kArnUnit)
  long long ldv, ldd;
  const TV* V;    // basis, column-major (ldv)
  TACC* w;        // working vector
  DiaOffsets dia;
  const TACC* dval;
  const int* aurp;
  const int* aucol;
  const TACC* auval;
  const int* aup_col;   // the rows' first two A W entries, two planes of N
  const TACC* aup_val;
  const TACC* sdefl;  // s' in the step's precision (step 0: from the coarse-solve kernel)
  // the coarse solve of the next step, in the kernel: pieces of aggregates (nodes perm
  // [piece_start[p], piece_start[p + 1]), each inside one block's rows), block b's pieces
  // blk_piece[blk_piece_start[b] ...], T^-1 (r x r, row-major)
  const int* perm;
  const int* piece_start;
  const int* agg_piece;
  const int* blk_piece_start;
  const int* blk_piece;
  const double* uscale;
  const double* tinv;
  const float* tinv32;  // FP32 copy of T^-1 (FP32 basis)
  Ctl ctl;
  unsigned* gbar;  // [0] arrivals, [1] generation
};

// rows VN elements at a time (16-byte loads of the basis type)
template <typename TV> struct ArnVec { static constexpr int n = Vec<TV>::n; };

// Grid barrier (cooperative launch: every block resident).  Thread 0 arrives on bar[0];
// the last arrival resets it and advances the generation bar[1]; the others poll the
// generation with a bound and report false when it never moves.
__device__ __forceinline__ bool arn_grid_sync(unsigned* bar, unsigned gen) {
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
        if (++spins > kArnSpins) {
          ok = 0;
          break;
        }
      }
    }
    __threadfence();
    s_ok = ok;
  }
  __syncthreads();
  return s_ok != 0;
}

// Split grid barrier on a counter that only grows (bar[2]): a block arrives once its share
// of a phase is published, carries on with work that does not need the other blocks'
// shares, and waits later until the counter reaches the target (G arrivals per phase,
// counted from the value read at the kernel's start; compared modulo 2^32).
__device__ __forceinline__ void arn_arrive(unsigned* cnt) {
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    atomicAdd(cnt, 1u);
  }
}

__device__ __forceinline__ bool arn_wait(const unsigned* cnt, unsigned target) {
  __shared__ int s_ok;
  if (threadIdx.x == 0) {
    int ok = 1;
    long long spins = 0;
    while ((int)(*(volatile const unsigned*)cnt - target) < 0) {
      if (++spins > kArnSpins) {
        ok = 0;
        break;
      }
    }
    __threadfence();
    s_ok = ok;
  }
  __syncthreads();
  return s_ok != 0;
}

// dst[c] = sum_{r < nrows} src[r * ldp + c] for c < ncols, in a fixed order: the Q threads
// of a column (consecutive lanes) take rows q, q + Q, ..., each issuing up to 8 loads at
// once before adding them, then combine by shuffles; ends with a block barrier.  (FP64 adds
// issue at a quarter-warp per clock on GB300: the trees are kept short.)
__device__ __forceinline__ void arn_reduce_cols(const double* src, int nrows, int ncols, int ldp,
                                                double* dst) {
  constexpr int L = 8;
  int Q = 1;
  while (Q * 2 <= 32 && Q * 2 * ncols <= (int)blockDim.x) Q *= 2;
  const int rounds = (ncols * Q + blockDim.x - 1) / blockDim.x;
  for (int rd = 0; rd < rounds; ++rd) {
    const int idx = rd * blockDim.x + threadIdx.x;
    const int c = idx / Q, q = idx % Q;
    double sum = 0.0;
    if (c < ncols) {
      for (int r0 = q; r0 < nrows; r0 += L * Q) {
        double v[L];
#pragma unroll
        for (int u = 0; u < L; ++u) {
          const int r = r0 + u * Q;
          v[u] = r < nrows ? __ldcg(src + (size_t)r * ldp + c) : 0.0;
        }
#pragma unroll
        for (int h = L / 2; h > 0; h >>= 1)
#pragma unroll
          for (int u = 0; u < h; ++u) v[u] += v[u + h];
        sum += v[0];
      }
    }
    for (int o = 1; o < Q; o <<= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
    if (c < ncols && q == 0) dst[c] = sum;
  }
  __syncthreads();
}

// 16-byte vector load of VN basis elements from global memory, read-only and streamed past
// L1 (the basis is read once per pass; L1 is mostly carved out for shared memory here)
template <typename TV, typename TACC, int VN>
__device__ __forceinline__ void arn_ldg(const TV* p, TACC (&o)[VN]) {
  if constexpr (std::is_same<TV, double>::value) {
    double x, y;
    asm volatile("ld.global.nc.L1::no_allocate.v2.f64 {%0, %1}, [%2];"
                 : "=d"(x), "=d"(y)
                 : "l"(p));
    o[0] = (TACC)x;
    o[1] = (TACC)y;
  } else if constexpr (std::is_same<TV, float>::value) {
    float x, y, z, w;
    asm volatile("ld.global.nc.L1::no_allocate.v4.f32 {%0, %1, %2, %3}, [%4];"
                 : "=f"(x), "=f"(y), "=f"(z), "=f"(w)
                 : "l"(p));
    o[0] = x; o[1] = y; o[2] = z; o[3] = w;
  } else {
    const uint4 v = __ldg(reinterpret_cast<const uint4*>(p));
    const __nv_bfloat162* h = reinterpret_cast<const __nv_bfloat162*>(&v);
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const float2 f = __bfloat1622float2(h[e]);
      o[2 * e] = f.x;
      o[2 * e + 1] = f.y;
    }
  }
}

// An FP64 operator value read with the L2 evict-first priority: the diagonals (76 MB at
// 1M rows) then give way to the basis columns, which the update re-reads right after the
// multi-dot (measured on q1-n1024: FP64 step 236.4 to 228.0 us at the fixed 100-step
// protocol; the FP32 step, whose 38 MB of diagonals stay useful in L2 across steps, went
// from 76.9 to 80.0 us with the same hint and keeps plain loads)
__device__ __forceinline__ double arn_ld_evict_first(const double* p) {
  unsigned long long pol;
  asm("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol));
  double v;
  asm volatile("ld.global.nc.L2::cache_hint.f64 %0, [%1], %2;" : "=d"(v) : "l"(p), "l"(pol));
  return v;
}

template <typename TV, typename TACC, int VN>
__device__ __forceinline__ void arn_stv(TV* p, const TACC (&v)[VN]) {
  if constexpr (std::is_same<TV, double>::value) {
    *reinterpret_cast<double2*>(p) = make_double2(v[0], v[1]);
  } else if constexpr (std::is_same<TV, float>::value) {
    *reinterpret_cast<float4*>(p) = make_float4(v[0], v[1], v[2], v[3]);
  } else {
    uint4 o;
    __nv_bfloat162* h = reinterpret_cast<__nv_bfloat162*>(&o);
#pragma unroll
    for (int e = 0; e < 4; ++e) h[e] = __floats2bfloat162_rn(v[2 * e], v[2 * e + 1]);
    *reinterpret_cast<uint4*>(p) = o;
  }
}

// a grid barrier that never completed: the solve stops with GMRES_ERR_TIMEOUT
__device__ __forceinline__ void arn_timeout(Ctl& ctl) {
  if (threadIdx.x == 0) {
    ctl.flags[F_STATUS] = GMRES_ERR_TIMEOUT;
    ctl.flags[F_STOP] = 1;
    ctl.flags[F_CYCLE_DONE] = 1;
  }
}

// a basis entry written earlier in this launch, read through L2 as FP64
__device__ __forceinline__ double arn_ldcg_d(const double* p) { return __ldcg(p); }
__device__ __forceinline__ double arn_ldcg_d(const float* p) { return (double)__ldcg(p); }

// ---- double-FP32 arithmetic for the FP64 multi-dot (GMRES_DOT_DF32) ---------------------
// GB300 issues FP64 FMAs at 2 lanes per clock and multiprocessor, FP32 FMAs at 128: the
// FP64 multi-dot is bound by its FMA pipe, not by HBM.  In the double-FP32 form each FP64
// operand is split into two floats, x ~ hi + lo, with integer operations only (hi = x with
// its significand cut to 24 bits, lo = the remaining 29 bits rounded to 24: 47 significant
// bits in all); a product takes the exact product of the high parts by an FMA (Dekker's
// two-product), the two cross terms in FP32 (lo * lo, below 2^-46 of the product, is
// dropped), and the running sum is a pair (s, c) advanced by Knuth's TwoSum, every rounding
// error gathered in c.  Magnitudes between 2^-126 and 2^127 split exactly as stated; smaller
// ones become 0 (an absolute error below 2^-126), larger ones infinity.
__device__ __forceinline__ void arn_df_split(double v, float& hi, float& lo) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(v);
  const unsigned h32 = (unsigned)(b >> 32), l32 = (unsigned)b;
  const unsigned sgn = h32 & 0x80000000u;
  const unsigned ah = h32 & 0x7fffffffu;
  const int E = (int)(ah >> 20);  // biased FP64 exponent
  // exponent and top 23 significand bits, rebiased from 1023 to 127 (mod 2^32)
  unsigned hb = ((ah << 3) | (l32 >> 29)) - (896u << 23);
  const unsigned m29 = l32 & 0x1fffffffu;  // the significand bits below hi's
  const unsigned fb = __float_as_uint(__uint2float_rn(m29));
  const unsigned lb = fb + ((unsigned)(E - 1075) << 23);  // m29 * 2^(E - 1075)
  const bool okh = E >= 897;
  const bool okl = okh && m29 != 0u && (int)(fb >> 23) + E - 1075 >= 1;
  hb = E > 1150 ? 0x7f800000u : hb;
  hi = __uint_as_float(okh ? (hb | sgn) : sgn);
  lo = __uint_as_float(okl ? (lb | sgn) : 0u);
}

// (s, c) += (ah + al) (bh + bl); the _rn intrinsics keep the compiler from contracting the
// error-free steps into FMAs
__device__ __forceinline__ void arn_df_fma(float& s, float& c, float ah, float al, float bh,
                                           float bl) {
  const float p = __fmul_rn(ah, bh);
  float e = __fmaf_rn(ah, bh, -p);  // exact: p + e = ah bh
  e = __fmaf_rn(ah, bl, e);
  e = __fmaf_rn(al, bh, e);
  const float t = __fadd_rn(s, p);  // TwoSum: t + err = s + p exactly
  const float bp = __fsub_rn(t, s);
  const float err = __fadd_rn(__fsub_rn(s, __fsub_rn(t, bp)), __fsub_rn(p, bp));
  s = t;
  c = __fadd_rn(c, __fadd_rn(err, e));
}

// (s, c) += (s2, c2)
__device__ __forceinline__ void arn_df_add(float& s, float& c, float s2, float c2) {
  const float t = __fadd_rn(s, s2);
  const float bp = __fsub_rn(t, s);
  const float err = __fadd_rn(__fsub_rn(s, __fsub_rn(t, bp)), __fsub_rn(s2, bp));
  s = t;
  c = __fadd_rn(__fadd_rn(c, c2), err);
}

// The same over partials stored as double-FP32 pairs (two floats per slot): TwoSum on the
// FP32 pipe in a fixed order, L loads in flight per thread, rounded to FP64 once per column.
template <int L>
__device__ __forceinline__ void arn_reduce_cols_df(const double* src, int nrows, int ncols,
                                                   int ldp, double* dst) {
  int Q = 1;
  while (Q * 2 <= 32 && Q * 2 * ncols <= (int)blockDim.x) Q *= 2;
  const int rounds = (ncols * Q + blockDim.x - 1) / blockDim.x;
  for (int rd = 0; rd < rounds; ++rd) {
    const int idx = rd * blockDim.x + threadIdx.x;
    const int c = idx / Q, q = idx % Q;
    float hs = 0.f, hc = 0.f;
    if (c < ncols) {
      for (int r0 = q; r0 < nrows; r0 += L * Q) {
        float2 v[L];
#pragma unroll
        for (int u = 0; u < L; ++u) {
          const int r = r0 + u * Q;
          v[u] = r < nrows ? __ldcg(reinterpret_cast<const float2*>(src + (size_t)r * ldp + c))
                           : make_float2(0.f, 0.f);
        }
#pragma unroll
        for (int u = 0; u < L; ++u) arn_df_add(hs, hc, v[u].x, v[u].y);
      }
    }
    for (int o = 1; o < Q; o <<= 1) {
      const float a2 = __shfl_xor_sync(0xffffffffu, hs, o);
      const float b2 = __shfl_xor_sync(0xffffffffu, hc, o);
      arn_df_add(hs, hc, a2, b2);
    }
    if (c < ncols && q == 0) dst[c] = (double)hs + (double)hc;
  }
  __syncthreads();
}

// Multi-dot of an FP64 basis in double-FP32 (row order): warp w takes the chunks w, w + 16,
// ... of 64 rows of the super-tile and, per pass, G columns at the same rows (one 16-byte
// load per column and lane, all issued before the products); w and u_j come split from
// shared memory (float2 hi, lo per row).  At the end of a pass the lanes' pairs of each
// column meet by a shuffle tree of TwoSums and lane 0 adds them into dfp[warp][c][set]:
// no FP64 instruction in the loop.
constexpr int kArnDfGroup = 6;

__device__ __forceinline__ void arn_dots_df(float* dfp, const double* V, long long ldv, int k,
                                            long long s0, int nch, const float2* Ws,
                                            const float2* Us, int warp, int lane) {
  constexpr int G = kArnDfGroup;
  for (int g0 = 0; g0 < k; g0 += G) {
    const int gc = k - g0 < G ? k - g0 : G;
    float s1[G], c1[G], s2[G], c2[G];
#pragma unroll
    for (int q = 0; q < G; ++q) s1[q] = c1[q] = s2[q] = c2[q] = 0.f;
    const double* col = V + (size_t)g0 * ldv + s0 + (size_t)lane * 2;
    for (int ch = warp; ch < nch; ch += kArnWarps) {
      const int r = ch * 64 + lane * 2;
      double v[G][2];
#pragma unroll
      for (int q = 0; q < G; ++q)
        if (q < gc) arn_ldg<double, double, 2>(col + (size_t)q * ldv + (size_t)ch * 64, v[q]);
      const float4 wv = *reinterpret_cast<const float4*>(Ws + r);
      const float4 uv = *reinterpret_cast<const float4*>(Us + r);
#pragma unroll
      for (int q = 0; q < G; ++q)
        if (q < gc) {
          float h0, l0, h1, l1;
          arn_df_split(v[q][0], h0, l0);
          arn_df_split(v[q][1], h1, l1);
          arn_df_fma(s1[q], c1[q], h0, l0, wv.x, wv.y);
          arn_df_fma(s1[q], c1[q], h1, l1, wv.z, wv.w);
          arn_df_fma(s2[q], c2[q], h0, l0, uv.x, uv.y);
          arn_df_fma(s2[q], c2[q], h1, l1, uv.z, uv.w);
        }
    }
#pragma unroll
    for (int q = 0; q < G; ++q)
      if (q < gc) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
          const float a = __shfl_xor_sync(0xffffffffu, s1[q], o);
          const float b = __shfl_xor_sync(0xffffffffu, c1[q], o);
          const float d = __shfl_xor_sync(0xffffffffu, s2[q], o);
          const float e = __shfl_xor_sync(0xffffffffu, c2[q], o);
          arn_df_add(s1[q], c1[q], a, b);
          arn_df_add(s2[q], c2[q], d, e);
        }
        if (lane == 0) {
          float* p = dfp + ((size_t)warp * kMaxK + g0 + q) * 4;
          float a = p[0], b = p[1];
          arn_df_add(a, b, s1[q], c1[q]);
          p[0] = a;
          p[1] = b;
          a = p[2];
          b = p[3];
          arn_df_add(a, b, s2[q], c2[q]);
          p[2] = a;
          p[3] = b;
        }
      }
  }
}

// Diagonal part of the SpMV for B rows (row0 + b * stride) at once: all loads of the B
// rows are issued before their products (ND > 0: ND diagonals, unrolled; ND = 0: nd at
// run time, four at a time).  x indexes are clamped to a valid row, where the stored
// value is 0.
template <int B, int ND, typename TV, typename TACC>
__device__ __forceinline__ void arn_dia_rows(TACC (&acc)[B], long long row0, long long stride,
                                             long long Nn, int nd, const int* off,
                                             long long ldd, const TACC* __restrict__ dval,
                                             const TV* __restrict__ x) {
  constexpr int NQ = ND > 0 ? ND : 4;
#pragma unroll
  for (int b = 0; b < B; ++b) acc[b] = 0;
  for (int q0 = 0; q0 < (ND > 0 ? ND : nd); q0 += NQ) {
    TACC av[B][NQ], xv[B][NQ];
#pragma unroll
    for (int b = 0; b < B; ++b) {
      const long long row = row0 + b * stride;
      const long long rr = row < Nn ? row : Nn - 1;
#pragma unroll
      for (int u = 0; u < NQ; ++u) {
        const int q = q0 + u;
        const bool live = ND > 0 || q < nd;
        const long long c = min(max(rr + off[live ? q : 0], 0LL), Nn - 1);
        if constexpr (sizeof(TACC) == 8)
          av[b][u] = live ? arn_ld_evict_first(dval + (size_t)q * ldd + rr) : (TACC)0;
        else
          av[b][u] = live ? __ldg(dval + (size_t)q * ldd + rr) : (TACC)0;
        xv[b][u] = live ? ld_as<TACC, TV>(x + c) : (TACC)0;
      }
    }
#pragma unroll
    for (int b = 0; b < B; ++b)
#pragma unroll
      for (int u = 0; u < NQ; ++u) acc[b] += av[b][u] * xv[b][u];
  }
}

// Multi-dot in row-chunk order (FP32 basis): warp w takes the chunks w, w + 16, ... of the
// super-tile and, per unit, a group of up to G columns at one chunk: one 16-byte load per
// column and lane for the same rows, so the loads in flight of a warp fall in one row window
// of many columns (on GB300 this streams about twice as fast as a warp reading one column
// through many consecutive chunks).  Units run group by group, the warp's chunks in order,
// and the next unit's G loads are issued before the current one is consumed (two units in
// flight).  At a group's last chunk the lanes' partial sums of each column are added by a
// shuffle tree and lane 0 accumulates them into wsum[set][warp][c].  (G = 6 with two units
// in flight: measured on q1-n1024, 20 us at k = 26 against 21 for 10 columns, one unit at a
// time; 8 columns do not fit the register budget, nor 6 beside the run-time diagonal count
// of the general banded instantiation, which takes 5.)
template <int ND> constexpr int arn_group() { return ND == 9 ? 6 : 5; }

template <typename TV, typename TACC, int G>
__device__ __forceinline__ void arn_dots_rows(double* wsum, const TV* V, long long ldv, int k,
                                              long long s0, int nch, const TACC* Ws,
                                              const TACC* Us, int warp, int lane) {
  constexpr int VN = ArnVec<TV>::n;
  const int nqw = warp < nch ? (nch - 1 - warp) / kArnWarps + 1 : 0;  // chunks of this warp
  const int ng = (k + G - 1) / G;
  const int TU = ng * nqw;
  if (TU == 0) return;
  TACC a1[G], a2[G];
#pragma unroll
  for (int u = 0; u < G; ++u) {
    a1[u] = 0;
    a2[u] = 0;
  }
  auto load_unit = [&](int un, TACC (&b)[G][VN]) {
    const int g = un / nqw, qi = un - g * nqw;
    const int g0 = g * G;
    const int gc = k - g0 < G ? k - g0 : G;
    const TV* col = V + (size_t)g0 * ldv + s0 + (size_t)lane * VN +
                    (size_t)(warp + qi * kArnWarps) * 32 * VN;
#pragma unroll
    for (int u = 0; u < G; ++u)
      if (u < gc) arn_ldg<TV, TACC, VN>(col + (size_t)u * ldv, b[u]);
  };
  auto consume = [&](int un, const TACC (&b)[G][VN]) {
    const int g = un / nqw, qi = un - g * nqw;
    const int g0 = g * G;
    const int gc = k - g0 < G ? k - g0 : G;
    const size_t off = (size_t)(warp + qi * kArnWarps) * 32 * VN;
    TACC wv[VN], uv[VN];
    ld_acc<VN>(Ws + off + lane * VN, wv);
    ld_acc<VN>(Us + off + lane * VN, uv);
#pragma unroll
    for (int u = 0; u < G; ++u)
      if (u < gc)
#pragma unroll
        for (int e = 0; e < VN; ++e) {
          a1[u] += b[u][e] * wv[e];
          a2[u] += b[u][e] * uv[e];
        }
    if (qi == nqw - 1) {  // the group's last chunk in this warp
#pragma unroll
      for (int u = 0; u < G; ++u) {
        if (u < gc) {
          const TACC t1 = warp_sum(a1[u]), t2 = warp_sum(a2[u]);
          if (lane == 0) {
            float2* p1 = reinterpret_cast<float2*>(wsum) + (size_t)warp * kMaxK + g0 + u;
            float2* p2 = reinterpret_cast<float2*>(wsum) + (size_t)(kArnWarps + warp) * kMaxK + g0 + u;
            float2 a1v = *p1, a2v = *p2;
            arn_df_add(a1v.x, a1v.y, (float)t1, 0.f);
            arn_df_add(a2v.x, a2v.y, (float)t2, 0.f);
            *p1 = a1v;
            *p2 = a2v;
          }
        }
        a1[u] = 0;
        a2[u] = 0;
      }
    }
  };
  TACC bA[G][VN], bB[G][VN];
  load_unit(0, bA);
  for (int un = 0; un < TU; un += 2) {
    if (un + 1 < TU) load_unit(un + 1, bB);
    consume(un, bA);
    if (un + 2 < TU) load_unit(un + 2, bA);
    if (un + 1 < TU) consume(un + 1, bB);
  }
}

// Multi-dot of an FP64 basis: the 16 warps form 4 groups; group cg takes the columns
// cg, cg + 4, ... one after the other, and its 4 warps stream each column together, warp ws
// taking the chunks ws, ws + 4, ... (D chunks in flight per warp, the stream running on
// across column boundaries).  Four warps on one column keep long contiguous runs of the
// column in flight, which DRAM serves about twice as fast as one warp per column.  When a
// column ends, the group's 4 lane-wise partial sums meet in shared memory (double-buffered
// staging, one named barrier of the group) and warp ws = 0 adds them, in warp order, into
// the lane-wise totals sbuf[set][c][lane]: one FP64 add per lane, warp and column.
template <typename TV, typename TACC>
__device__ __forceinline__ void arn_dots_group4(double* sbuf, double* stg, const TV* V,
                                                long long ldv, int k, long long s0, int nch,
                                                const TACC* Ws, const TACC* Us, int warp,
                                                int lane) {
  constexpr int VN = ArnVec<TV>::n;
  constexpr int D = arn_loads<TV>();
  const int cg = warp >> 2, ws = warp & 3;
  const int ncg = cg < k ? (k - cg + 3) / 4 : 0;  // columns of this group
  const int cpw = (nch - ws + 3) / 4;              // chunks of this warp per column
  const int T = ncg * cpw;
  if (ncg == 0) return;  // the same in the group's four warps
  if (T == 0) {  // no chunk of this warp (nch < 4): zeros at the group's column ends
    for (int i = 0; i < ncg; ++i) {
      double* sb = stg + (size_t)(i & 1) * 2 * kArnWarps * 32;
      sb[(0 * kArnWarps + warp) * 32 + lane] = 0.0;
      sb[(1 * kArnWarps + warp) * 32 + lane] = 0.0;
      asm volatile("bar.sync %0, 128;" ::"r"(1 + cg) : "memory");
    }
    return;
  }
  // load side: a pointer that steps 4 chunks down the column, then on to the group's next
  // column (no division per load)
  const size_t step = (size_t)4 * 32 * VN;
  const long long jump = 4 * ldv - (long long)cpw * (long long)step;
  const TV* pl = V + (size_t)cg * ldv + s0 + (size_t)ws * 32 * VN + lane * VN;
  int lq = 0;
  auto next_load = [&](TACC (&o)[VN]) {
    arn_ldg<TV, TACC, VN>(pl, o);
    pl += step;
    if (++lq == cpw) {
      lq = 0;
      pl += jump;
    }
  };
  TACC buf[D][VN];
#pragma unroll
  for (int d = 0; d < D; ++d)
    if (d < T) next_load(buf[d]);
  TACC a1[VN], a2[VN];  // one chain per vector element (FP64 latency hidden by ILP)
#pragma unroll
  for (int e = 0; e < VN; ++e) {
    a1[e] = 0;
    a2[e] = 0;
  }
  int i = 0, qi = 0;  // column of the group and chunk of the warp being consumed
  const TACC* pw = Ws + (size_t)ws * 32 * VN + lane * VN;
  const TACC* pu = Us + (size_t)ws * 32 * VN + lane * VN;
  for (int t0 = 0; t0 < T; t0 += D) {
#pragma unroll
    for (int d = 0; d < D; ++d) {
      const int t = t0 + d;
      if (t < T) {
        TACC wv[VN], uv[VN];
        ld_acc<VN>(pw + (size_t)qi * step, wv);
        ld_acc<VN>(pu + (size_t)qi * step, uv);
#pragma unroll
        for (int e = 0; e < VN; ++e) {
          a1[e] += buf[d][e] * wv[e];
          a2[e] += buf[d][e] * uv[e];
        }
        if (t + D < T) next_load(buf[d]);
        if (++qi == cpw) {  // column cg + 4 i is done in this warp
          double* sb = stg + (size_t)(i & 1) * 2 * kArnWarps * 32;
          double s1 = 0.0, s2 = 0.0;
#pragma unroll
          for (int e = 0; e < VN; ++e) {
            s1 += (double)a1[e];
            s2 += (double)a2[e];
            a1[e] = 0;
            a2[e] = 0;
          }
          sb[(0 * kArnWarps + warp) * 32 + lane] = s1;
          sb[(1 * kArnWarps + warp) * 32 + lane] = s2;
          asm volatile("bar.sync %0, 128;" ::"r"(1 + cg) : "memory");
          if (ws == 0) {
            const int c = cg + 4 * i;
#pragma unroll
            for (int set = 0; set < 2; ++set) {
              const double* g = sb + (size_t)(set * kArnWarps + 4 * cg) * 32 + lane;
              sbuf[((size_t)set * kMaxK + c) * 33 + lane] += ((g[0] + g[32]) + (g[64] + g[96]));
            }
          }
          qi = 0;
          ++i;
        }
      }
    }
  }
}

// Diagonal part of step j's SpMV for the rows [s0, s1) of a super-tile: (A v_j) into Ws and
// u_j into Us (shared memory, from row s0; zeros past N)
template <int ND, typename TV, typename TACC>
__device__ __forceinline__ void arn_diag(const ArnArgs<TV, TACC>& a, int j, long long s0,
                                         long long s1, TACC* Ws, TACC* Us) {
  constexpr int B = sizeof(TACC) == 8 ? 2 : 4;  // SpMV rows per thread and batch
  const long long N = a.N;
  const TV* xj = a.V + (size_t)j * a.ldv;
  const int nd = ND > 0 ? ND : a.dia.nd;
  for (long long i0 = s0 + threadIdx.x; i0 < s1; i0 += (long long)B * kArnThreads) {
    TACC v[B];
    arn_dia_rows<B, ND, TV, TACC>(v, i0, kArnThreads, N, nd, a.dia.off, a.ldd, a.dval, xj);
#pragma unroll
    for (int b = 0; b < B; ++b) {
      const long long row = i0 + (long long)b * kArnThreads;
      if (row < s1) {
        Ws[row - s0] = row < N ? v[b] : (TACC)0;
        Us[row - s0] = row < N ? ld_as<TACC, TV>(xj + row) : (TACC)0;
      }
    }
  }
}

// SpMV, coarse correction and multi-dot of step j over the block's super-tiles (a function
// of its own, so that the cycle loop's state stays out of these loops' registers)
template <typename TV, typename TACC, int ND, bool DF>
__device__ __forceinline__ void arn_front(const ArnArgs<TV, TACC>& a, int j, TACC sig, bool waited,
                                       bool first_diag_done, TACC* Ws, TACC* Us, TACC* Ss,
                                       double* sbuf, double* stg) {
  constexpr int VN = ArnVec<TV>::n;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int t = threadIdx.x;
  const int G = gridDim.x, bid = blockIdx.x;
  const long long R0 = (long long)bid * a.units / G * kArnUnit;
  const long long R1 = (long long)(bid + 1) * a.units / G * kArnUnit;
  const long long N = a.N;
  const int k = j + 1;
  const bool multi = R1 - R0 > a.RS;  // w goes through global memory to the update
  for (long long s0 = R0; s0 < R1; s0 += a.RS) {
    const long long s1 = s0 + a.RS < R1 ? s0 + a.RS : R1;
    // ---- 1. SpMV of the super-tile's rows: w and u_j into shared memory (the first
    // super-tile's may have been formed during the previous step's coarse solve) ---------
    if (!(first_diag_done && s0 == R0)) arn_diag<ND, TV, TACC>(a, j, s0, s1, Ws, Us);
    // + A W s' (the row's A W entries, s' from shared memory), the scale sigma_j; w also to
    // global memory when the update reads it there.
    if constexpr (sizeof(TACC) == 8) {
      // FP64 (every FP64 instruction costs the scarce FP64 pipe): the CSR rows, kArnAwRows64
      // rows per thread at once, each level of the gather (row pointers, then the first entry
      // of every row) issued for all of them; s' is staged pre-scaled by sigma_j, so that
      // w = sigma_j Ws + sum a_iq (sigma_j s'_q) takes one multiply-add per entry and row
      if (!waited) {  // s' (the coarse solve's output) is read from here on
        pdl_wait();
        pdl_trigger();
        waited = true;
      }
      if (a.defl && s0 == R0)
        for (int q = t; q < a.r; q += kArnThreads) Ss[q] = sig * __ldcg(a.sdefl + q);
      __syncthreads();
      constexpr int AWR = kArnAwRows64;
      for (long long i0 = s0 + t; i0 < s1; i0 += (long long)AWR * kArnThreads) {
        int e0[AWR], e1[AWR];
#pragma unroll
        for (int b = 0; b < AWR; ++b) {
          const long long row = i0 + (long long)b * kArnThreads;
          const bool live = a.defl && row < N && row < s1;
          e0[b] = live ? __ldg(a.aurp + row) : 0;
          e1[b] = live ? __ldg(a.aurp + row + 1) : 0;
        }
        TACC av[AWR];
        int ac[AWR];
#pragma unroll
        for (int b = 0; b < AWR; ++b) {
          const bool has = e0[b] < e1[b];
          av[b] = has ? __ldg(a.auval + e0[b]) : (TACC)0;
          ac[b] = has ? __ldg(a.aucol + e0[b]) : 0;
        }
#pragma unroll
        for (int b = 0; b < AWR; ++b) {
          const long long row = i0 + (long long)b * kArnThreads;
          if (row < s1) {
            TACC wv = 0;
            if (row < N) {
              TACC aw = a.defl ? av[b] * Ss[ac[b]] : (TACC)0;
              for (int e = e0[b] + 1; e < e1[b]; ++e) aw += __ldg(a.auval + e) * Ss[__ldg(a.aucol + e)];
              wv = fma(sig, Ws[row - s0], aw);
            }
            Ws[row - s0] = wv;
            if ((multi || DF) && row < N) a.w[row] = wv;
          }
        }
      }
    } else {
      // FP32: a row's first two A W entries from the row-indexed planes (one level of loads,
      // kArnAwRows32 rows per thread at once); the first batch's loads are issued before s'
      // is read, since they do not depend on it
      constexpr int AWR = kArnAwRows32;
      TACC av0[AWR], av1[AWR];
      int ac0[AWR], ac1[AWR];
      auto aw_load = [&](long long i0) {
#pragma unroll
        for (int b = 0; b < AWR; ++b) {
          const long long row = i0 + (long long)b * kArnThreads;
          const bool live = a.defl && row < N && row < s1;
          ac0[b] = live ? __ldg(a.aup_col + row) : -1;
          ac1[b] = live ? __ldg(a.aup_col + N + row) : -1;
          av0[b] = live ? __ldg(a.aup_val + row) : (TACC)0;
          av1[b] = live ? __ldg(a.aup_val + N + row) : (TACC)0;
        }
      };
      auto aw_apply = [&](long long i0) {
#pragma unroll
        for (int b = 0; b < AWR; ++b) {
          const long long row = i0 + (long long)b * kArnThreads;
          if (row < s1) {
            // absent entries carry the value 0 (and read s'_0, which is finite)
            TACC aw = 0;
            if (a.defl) {
              aw = av0[b] * Ss[ac0[b] >= 0 ? ac0[b] : 0];
              aw += av1[b] * Ss[ac1[b] >= 0 ? ac1[b] : (ac1[b] == -1 ? 0 : -ac1[b] - 2)];
              if (ac1[b] < -1) {  // the row's third and later entries (rare)
                const int e1 = __ldg(a.aurp + row + 1);
#pragma unroll 1
                for (int e = __ldg(a.aurp + row) + 2; e < e1; ++e)
                  aw += __ldg(a.auval + e) * Ss[__ldg(a.aucol + e)];
              }
            }
            const TACC wv = row < N ? sig * (Ws[row - s0] + aw) : (TACC)0;
            Ws[row - s0] = wv;
            if ((multi || DF) && row < N) a.w[row] = wv;
          }
        }
      };
      aw_load(s0 + t);
      if (!waited) {  // s' (the coarse solve's output) is read from here on
        pdl_wait();
        pdl_trigger();
        waited = true;
      }
      if (a.defl && s0 == R0)
        for (int q = t; q < a.r; q += kArnThreads) Ss[q] = __ldcg(a.sdefl + q);
      __syncthreads();
      for (long long i0 = s0 + t; i0 < s1; i0 += (long long)AWR * kArnThreads) {
        if (i0 != s0 + t) aw_load(i0);
        aw_apply(i0);
      }
    }
    __syncthreads();
    const int nch = (int)((s1 - s0) / (32 * VN));
    if constexpr (DF) {
      // w and u_j split in place (float2 hi, lo in the 8 bytes of each double); the
      // update reads w from global memory
      for (long long q = t; q < s1 - s0; q += kArnThreads) {
        float h1, l1, h2, l2;
        arn_df_split((double)Ws[q], h1, l1);
        arn_df_split((double)Us[q], h2, l2);
        reinterpret_cast<float2*>(Ws)[q] = make_float2(h1, l1);
        reinterpret_cast<float2*>(Us)[q] = make_float2(h2, l2);
      }
      __syncthreads();
      arn_dots_df(reinterpret_cast<float*>(sbuf), reinterpret_cast<const double*>(a.V), a.ldv,
                  k, s0, nch, reinterpret_cast<const float2*>(Ws),
                  reinterpret_cast<const float2*>(Us), warp, lane);
    } else if constexpr (sizeof(TV) == 8) {
      // FP64 (its FMA pipe is the bound and its adds are dear): lane-wise partial sums
      // per column, four warps per column
      arn_dots_group4<TV, TACC>(sbuf, stg, a.V, a.ldv, k, s0, nch, Ws, Us, warp, lane);
    } else {
        arn_dots_rows<TV, TACC, arn_group<ND>()>(sbuf, a.V, a.ldv, k, s0, nch, Ws, Us, warp, lane);
    }
    __syncthreads();  // the slices are rewritten by the next super-tile
  }
}

// u_{j+1} = w - V (sigma o h) over the block's rows (also into ush, indexed from the block's
// first row, when given); returns the warp's part of ||u_{j+1}||^2 (in every lane)
template <typename TV, typename TACC, int ND, bool DF>
__device__ __forceinline__ double arn_update(const ArnArgs<TV, TACC>& a, int k, const TACC* Ws,
                                          const TACC* scoef, TACC* ush) {
  constexpr int VN = ArnVec<TV>::n;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int G = gridDim.x, bid = blockIdx.x;
  const long long R0 = (long long)bid * a.units / G * kArnUnit;
  const long long R1 = (long long)(bid + 1) * a.units / G * kArnUnit;
  const long long N = a.N;
  TV* __restrict__ vout = const_cast<TV*>(a.V) + (size_t)k * a.ldv;
  double nrm = 0.0;       // FP64 basis
  float ns = 0.f, nc = 0.f;  // FP32 basis: a double-FP32 pair (FP64 adds are dear)
  {
    constexpr int U = sizeof(TV) == 4 ? 8 : (ND == 9 && !DF ? 13 : 10);  // basis loads in flight per lane
    const int chunk = 32 * VN;
    const long long nch = (R1 - R0) / chunk;
    const bool wsm = !DF && R1 - R0 <= a.RS;  // the block's w is still in shared memory
    for (long long q = nch - 1 - warp; q >= 0; q -= kArnWarps) {
      const long long r = R0 + q * chunk + (long long)lane * VN;
      TACC wv[VN], p[VN];
      if (wsm) {
        ld_acc<VN>(Ws + (r - R0), wv);
      } else {
#pragma unroll
        for (int e = 0; e < VN; ++e) wv[e] = r + e < N ? __ldcg(a.w + r + e) : (TACC)0;
      }
#pragma unroll
      for (int e = 0; e < VN; ++e) p[e] = 0;
      for (int c0 = 0; c0 < k; c0 += U) {
        TACC v[U][VN];
#pragma unroll
        for (int u = 0; u < U; ++u)
          if (c0 + u < k) arn_ldg<TV, TACC, VN>(a.V + (size_t)(c0 + u) * a.ldv + r, v[u]);
#pragma unroll
        for (int u = 0; u < U; ++u)
          if (c0 + u < k) {
            const TACC cf = scoef[c0 + u];
#pragma unroll
            for (int e = 0; e < VN; ++e) p[e] += v[u][e] * cf;
          }
      }
      TACC un[VN];
#pragma unroll
      for (int e = 0; e < VN; ++e) un[e] = wv[e] - p[e];
      arn_stv<TV, TACC, VN>(vout + r, un);
      if (ush) acc_store<VN>(ush + (r - R0), un);  // for the piece sums
      TACC s = 0;
#pragma unroll
      for (int e = 0; e < VN; ++e) s += un[e] * un[e];
      if constexpr (sizeof(TACC) == 8) nrm += s;
      else arn_df_add(ns, nc, s, 0.f);
    }
  }
  if constexpr (sizeof(TACC) == 8) {
    return warp_sum(nrm);
  } else {  // the warp's total in double-FP32, rounded once
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const float a2 = __shfl_xor_sync(0xffffffffu, ns, o);
      const float b2 = __shfl_xor_sync(0xffffffffu, nc, o);
      arn_df_add(ns, nc, a2, b2);
    }
    return (double)ns + (double)nc;
  }
}

// Sums of u_{j+1} over this block's aggregate pieces (c of the next step's coarse solve, by
// pieces, a warp each).  The pieces' bounds are loaded up front (lane i < 8 holds the
// warp's i-th piece), then per piece the node indexes and the values: from the shared-memory
// copy of the block's rows when there is one (ush, from row R0), else through L2 (this
// block wrote them just before).  Fixed order throughout.
template <typename TV, typename TACC>
__device__ __forceinline__ void arn_piece_sums(const ArnArgs<TV, TACC>& a, const TV* vout,
                                               const TACC* ush, long long R0) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int bid = blockIdx.x;
  const int p0 = __ldg(a.blk_piece_start + bid), p1 = __ldg(a.blk_piece_start + bid + 1);
  for (int base = p0 + warp; base < p1; base += kArnWarps * 8) {
    const int pi = base + kArnWarps * lane;
    int mp = -1, ms = 0, me = 0;
    if (lane < 8 && pi < p1) {
      mp = __ldg(a.blk_piece + pi);
      ms = __ldg(a.piece_start + mp);
      me = __ldg(a.piece_start + mp + 1);
    }
    for (int i = 0; i < 8; ++i) {
      const int p = __shfl_sync(0xffffffffu, mp, i);
      const int s = __shfl_sync(0xffffffffu, ms, i), e = __shfl_sync(0xffffffffu, me, i);
      if (p < 0) break;
      double acc[2] = {0.0, 0.0};
      for (int o = s; o < e; o += 32 * 8) {
        int node[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          const int q = o + lane + 32 * u;
          node[u] = q < e ? __ldg(a.perm + q) : -1;
        }
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          double v = 0.0;
          if (node[u] >= 0) v = ush ? (double)ush[node[u] - R0] : arn_ldcg_d(vout + node[u]);
          acc[u & 1] += v;
        }
      }
      const double sum = warp_sum(acc[0] + acc[1]);
      if (lane == 0) {
        if constexpr (sizeof(TACC) == 8) {
          __stcg(a.ctl.cpart + p, sum);
        } else {  // the pair the FP32 coarse solve reads
          const float hs = (float)sum;
          __stcg(reinterpret_cast<float2*>(a.ctl.cpart + p), make_float2(hs, (float)(sum - (double)hs)));
        }
      }
    }
  }
}

// The same sums from the staged node list: a warp per piece, values from the shared-memory
// copy of u_{j+1}.  FP64 rows add in FP64; FP32 rows in double-FP32 (TwoSum on the FP32
// pipe, exact to about 2^-48 of the sum's magnitude), rounded to FP64 once per piece.
constexpr int kArnMaxBlkPieces = 256;

template <typename TACC>
__device__ __forceinline__ void arn_piece_sums_staged(double* cpart, const TACC* ush,
                                                      const unsigned short* snode,
                                                      const int* spid, const int* spls, int np) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int i = warp; i < np; i += kArnWarps) {
    const int ls = spls[i], le = spls[i + 1];
    double sum;
    if constexpr (sizeof(TACC) == 8) {
      double acc[2] = {0.0, 0.0};
      for (int q = ls + lane; q < le; q += 64) {
        acc[0] += (double)ush[snode[q]];
        if (q + 32 < le) acc[1] += (double)ush[snode[q + 32]];
      }
      sum = warp_sum(acc[0] + acc[1]);
    } else {
      float hs = 0.f, hc = 0.f;
      for (int q = ls + lane; q < le; q += 32) arn_df_add(hs, hc, (float)ush[snode[q]], 0.f);
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        const float a2 = __shfl_xor_sync(0xffffffffu, hs, o);
        const float b2 = __shfl_xor_sync(0xffffffffu, hc, o);
        arn_df_add(hs, hc, a2, b2);
      }
      // an FP32 basis keeps the pair (two floats in the slot) for the FP32 coarse solve
      if (lane == 0) __stcg(reinterpret_cast<float2*>(cpart + spid[i]), make_float2(hs, hc));
      continue;
    }
    if (lane == 0) __stcg(cpart + spid[i], sum);
  }
}

template <typename TV, typename TACC, int ND, bool DF>
__global__ void __launch_bounds__(kArnThreads, 1)
    k_arnoldi(const __grid_constant__ ArnArgs<TV, TACC> a) {
  static_assert(std::is_same<TV, TACC>::value, "w and u_j slices share the basis element type");
  static_assert(!DF || sizeof(TV) == 8, "the double-FP32 multi-dot takes an FP64 basis");
  constexpr int VN = ArnVec<TV>::n;
  constexpr int B = sizeof(TACC) == 8 ? 2 : 4;  // SpMV rows per thread and batch
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ double tot[2 * kMaxK + 1];
  __shared__ double sred[2 * kMaxK];
  __shared__ double sg[kMaxK];
  __shared__ TACC scoef[kMaxK];
  __shared__ double snrm[kArnWarps];
  __shared__ double ssig[kMaxK + 1];
  // the control block is read from the grid-constant parameter (no register copy)
  Ctl& ctl = const_cast<Ctl&>(a.ctl);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int t = threadIdx.x;
  const int G = gridDim.x, bid = blockIdx.x;
  const long long R0 = (long long)bid * a.units / G * kArnUnit;
  const long long R1 = (long long)(bid + 1) * a.units / G * kArnUnit;
  const long long N = a.N;
  // shared memory: w and u_j of a super-tile, s' (r), reduction scratch, the rows of L
  // (stride kMaxK), the FP64 multi-dot staging
  TACC* Ws = reinterpret_cast<TACC*>(smem);
  TACC* Us = Ws + a.RS;
  TACC* Ss = Us + a.RS;
  double* scratch = reinterpret_cast<double*>(
      smem + ((2 * (size_t)a.RS + (size_t)a.r) * sizeof(TACC) + 127) / 128 * 128);
  double* sL = scratch + kArnScratch / sizeof(double);
  double* stg = sL + (size_t)kMaxK * kMaxK;
  double* sbuf = scratch;
  double* sc = reinterpret_cast<double*>(smem);  // c of the coarse solve (w, u_j are dead)

  if (!a.pre) {
    pdl_wait();
    pdl_trigger();
  }
  // the flag is final here (set by the previous cycle's last step, reset by the residual
  // kernel before this one started): the same value in every block
  if (__ldcg(&ctl.flags[F_CYCLE_DONE])) {
    if (a.pre) {
      pdl_wait();
      pdl_trigger();
    }
    return;
  }
  unsigned gen = *(volatile unsigned*)&a.gbar[1];  // advanced only once all arrive
  // the split barrier's counter: no block arrives before every block has passed the first
  // grid barrier, so all read the same base
  const unsigned cbase = *(volatile unsigned*)&a.gbar[2];
  for (int q = t; q < kMaxK * kMaxK; q += kArnThreads) sL[q] = 0.0;
  if (t == 0) ssig[0] = __ldcg(&ctl.sigma[0]);
  // the block's aggregate pieces for the whole cycle: their ids, local starts and nodes (as
  // offsets from R0, 16 bits) in shared memory, past the rows of u_j's slice, when the
  // block's rows fit one super-tile with room to spare (else the sums read perm from L2)
  __shared__ int spid[kArnMaxBlkPieces];
  __shared__ int spls[kArnMaxBlkPieces + 1];
  const long long nrows = R1 - R0;
  unsigned short* snode = reinterpret_cast<unsigned short*>(Us + nrows);
  const int bp0 = a.defl ? __ldg(a.blk_piece_start + bid) : 0;
  const int bp1 = a.defl ? __ldg(a.blk_piece_start + bid + 1) : 0;
  const bool staged = a.defl && bp1 - bp0 <= kArnMaxBlkPieces && nrows <= 65536 &&
                      (size_t)nrows * sizeof(TACC) + (size_t)nrows * 2 <= (size_t)a.RS * sizeof(TACC);
  if (staged) {
    if (warp == 0) {  // ids and sizes 32 at a time, local starts by a warp scan
      int run = 0;
      for (int i0 = 0; i0 < bp1 - bp0; i0 += 32) {
        const int i = i0 + lane;
        int p = 0, n = 0;
        if (i < bp1 - bp0) {
          p = __ldg(a.blk_piece + bp0 + i);
          n = __ldg(a.piece_start + p + 1) - __ldg(a.piece_start + p);
        }
        int inc = n;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
          const int v = __shfl_up_sync(0xffffffffu, inc, o);
          if (lane >= o) inc += v;
        }
        if (i < bp1 - bp0) {
          spid[i] = p;
          spls[i] = run + inc - n;
        }
        run += __shfl_sync(0xffffffffu, inc, 31);
      }
      if (lane == 0) spls[bp1 - bp0] = run;
    }
    __syncthreads();
    for (int i = warp; i < bp1 - bp0; i += kArnWarps) {
      const int p = spid[i];
      const int s = __ldg(a.piece_start + p), ls = spls[i], n = spls[i + 1] - ls;
      for (int q = lane; q < n; q += 32) snode[ls + q] = (unsigned short)(__ldg(a.perm + s + q) - R0);
    }
  }
  // FP32 basis: the coarse solve's static data for the cycle (the aggregates' piece ranges,
  // their scales, this block's rows of T^-1 when every warp has at most one) staged once in
  // shared memory past the rows of w's slice, when it fits
  int* sap = nullptr;       // agg_piece, r + 1
  float* sus = nullptr;     // uscale, r
  float* stinv = nullptr;   // the block's rows of T^-1 (warp w: row (b - 1) + (G - 1) w)
  if constexpr (sizeof(TACC) == 4) {
    const int nwr = G == 1 ? kArnWarps : (G - 1) * kArnWarps;  // warps sharing the rows
    const int rows = (a.defl && bid > 0 && a.r <= nwr && bid - 1 < a.r)
                         ? min(kArnWarps, (a.r - (bid - 1) + G - 2) / (G - 1)) : 0;
    const size_t need = (size_t)(a.r + 1) * 4 + (size_t)a.r * 4 + (size_t)rows * a.r * 4;
    if (a.defl && G > 1 && a.RS > nrows && (size_t)(a.RS - nrows) * sizeof(TACC) >= need + 16) {
      sap = reinterpret_cast<int*>(Ws + nrows);
      sus = reinterpret_cast<float*>(sap + a.r + 1);
      stinv = rows > 0 ? sus + a.r : nullptr;
      for (int q = t; q <= a.r; q += kArnThreads) sap[q] = __ldg(a.agg_piece + q);
      for (int q = t; q < a.r; q += kArnThreads) sus[q] = (float)__ldg(a.uscale + q);
      for (int q = t; q < rows * a.r; q += kArnThreads) {
        const int w = q / a.r, b = q % a.r;
        stinv[q] = __ldg(a.tinv32 + (size_t)((bid - 1) + (G - 1) * w) * a.r + b);
      }
    }
  }
  bool waited = !a.pre;
  __syncthreads();

  for (int j = 0; j < a.jmax; ++j) {
    const int k = j + 1;
    const TACC sig = (TACC)ssig[j];
    // partial sums of the multi-dot in shared memory, so that they persist across
    // super-tiles (FP64: lane-wise per column; FP32: per warp and column; double-FP32:
    // pairs per warp and column)
    for (int q = t; q < 2 * kMaxK * 33; q += kArnThreads) sbuf[q] = 0.0;
    arn_front<TV, TACC, ND, DF>(a, j, sig, waited, j > 0, Ws, Us, Ss, sbuf, stg);
    waited = true;
    // per-block column sums (fixed order)
    if constexpr (DF) {  // the 16 warps' pairs of each column in warp order, then FP64 once
      for (int q = t; q < 2 * k; q += kArnThreads) {
        const int set = q / k, c = q % k;
        const float* dfp = reinterpret_cast<const float*>(sbuf);
        float s = 0.f, cc = 0.f;
        for (int w = 0; w < kArnWarps; ++w) {
          const float* p = dfp + ((size_t)w * kMaxK + c) * 4 + 2 * set;
          arn_df_add(s, cc, p[0], p[1]);
        }
        sred[q] = (double)s + (double)cc;
      }
    } else if constexpr (sizeof(TV) == 8) {  // the 32 lane-wise totals of each column, pairwise
      for (int q0 = 0; q0 < 2 * k; q0 += kArnThreads / 2) {
        const int q = q0 + (t >> 1), half = t & 1;
        double v = 0.0;
        if (q < 2 * k) {
          const int set = q / k, c = q % k;
          v = tree16(sbuf + ((size_t)set * kMaxK + c) * 33 + half * 16);
        }
        v += __shfl_xor_sync(0xffffffffu, v, 1);
        if (q < 2 * k && half == 0) sred[q] = v;
      }
    } else {  // the 16 warps' pairs of each column in warp order, kept as a pair
      for (int q = t; q < 2 * k; q += kArnThreads) {
        const int set = q / k, c = q % k;
        const float2* ws = reinterpret_cast<const float2*>(sbuf);
        float hs = 0.f, hc = 0.f;
        for (int w = 0; w < kArnWarps; ++w) {
          const float2 v = ws[(size_t)(set * kArnWarps + w) * kMaxK + c];
          arn_df_add(hs, hc, v.x, v.y);
        }
        reinterpret_cast<float2*>(sred)[q] = make_float2(hs, hc);
      }
    }
    __syncthreads();
    // the partials: FP64 values, or double-FP32 pairs (two floats in the slot) for an FP32
    // basis, whose cross-block sums then run on the FP32 pipe
    for (int c = t; c < 2 * k; c += kArnThreads) __stcg(&ctl.part[(size_t)bid * ctl.ldp + c], sred[c]);
    // ---- 3. grid barrier; identical totals in every block; (I + L) h = g ----------------
    if (!arn_grid_sync(a.gbar, gen++)) {
      arn_timeout(ctl);
      return;
    }
    if constexpr (sizeof(TV) == 4)
      // (a thread's 152 / 8 rows of partials in one batch of loads)
      arn_reduce_cols_df<24>(ctl.part, G, 2 * k, ctl.ldp, tot);  // ends with __syncthreads
    else
      arn_reduce_cols(ctl.part, G, 2 * k, ctl.ldp, tot);
    {
      // the new row of L: v_j . v_c = sigma_j sigma_c (u_j . u_c), c < j; g_c = sigma_c (u_c . w)
      const double sj = ssig[k - 1];
      for (int c = t; c < k; c += kArnThreads) {
        if (c < k - 1) sL[(size_t)(k - 1) * kMaxK + c] = sj * ssig[c] * tot[k + c];
        sg[c] = ssig[c] * tot[c];
      }
      __syncthreads();
      if (warp == 0) {  // forward substitution: h_c final when reached (entries c, c+32, c+64)
        // sL[i][c] = 0 for c >= i, so rows at or above c take a zero update; only the
        // 32-row groups below k are touched (one FP64 FMA per group and column)
        const int nq = (k + 31) >> 5;
        double g[3];
#pragma unroll
        for (int q = 0; q < 3; ++q) g[q] = lane + 32 * q < k ? sg[lane + 32 * q] : 0.0;
        for (int c = 0; c < k; ++c) {
          const double hc = __shfl_sync(0xffffffffu, c < 32 ? g[0] : (c < 64 ? g[1] : g[2]), c & 31);
#pragma unroll
          for (int q = 0; q < 3; ++q) {
            const int i = lane + 32 * q;
            if (q < nq) g[q] -= (i < k ? sL[(size_t)i * kMaxK + c] : 0.0) * hc;
          }
        }
#pragma unroll
        for (int q = 0; q < 3; ++q) {
          const int i = lane + 32 * q;
          if (i < k) {
            scoef[i] = (TACC)(ssig[i] * g[q]);
            if (bid == 0) {
              ctl.h[i] = g[q];
              if (i < k - 1) ctl.L[(size_t)(k - 1) * kMaxK + i] = sL[(size_t)(k - 1) * kMaxK + i];
            }
          }
        }
      }
      __syncthreads();
    }
    // ---- 4. update u_{j+1} = w - V (sigma o h) and ||u_{j+1}||^2 ------------------------
    TV* __restrict__ vout = const_cast<TV*>(a.V) + (size_t)k * a.ldv;
    // a shared-memory copy of u_{j+1} for the piece sums when the block's rows fit one
    // super-tile (u_j's slice is dead by now)
    TACC* ush = (a.defl && k < a.jmax && R1 - R0 <= a.RS) ? Us : nullptr;
    double nrm = arn_update<TV, TACC, ND, DF>(a, k, Ws, scoef, ush);
    // ---- 5. norm partial; partial sums of u_{j+1} over this block's aggregate pieces ----
    {
      // the warp sums (formed by the update), then warp 0 adds the 16 of them (a block-wide
      // final loop would issue 16 FP64 adds in every warp)
      if (lane == 0) snrm[warp] = nrm;
      __syncthreads();  // also orders this block's stores of u_{j+1} before the piece sums
      if (warp == 0) {
        double bs = lane < kArnWarps ? snrm[lane] : 0.0;
#pragma unroll
        for (int o = kArnWarps / 2; o > 0; o >>= 1) bs += __shfl_xor_sync(0xffffffffu, bs, o);
        if (lane == 0) __stcg(&ctl.part[(size_t)bid * ctl.ldp + kArnNormCol], bs);
      }
      if (a.defl && k < a.jmax) {
        if (staged && ush)
          arn_piece_sums_staged(ctl.cpart, ush, snode, spid, spls, bp1 - bp0);
        else
          arn_piece_sums(a, vout, ush, R0);
      }
    }
    if (!arn_grid_sync(a.gbar, gen++)) {
      arn_timeout(ctl);
      return;
    }
    const bool coarse = a.defl && k < a.jmax && (bid > 0 || G == 1);
    // ---- 6. ||u_{j+1}|| and the plane rotations with the stopping tests (block 0); the next
    // step's coarse solve s' = U (|mu| T^-1 - I) U^T u_{j+1} (the other blocks) -------------
    if (bid == 0) {
      arn_reduce_cols(ctl.part + kArnNormCol, G, 1, ctl.ldp, tot);
      givens_step(ctl, j, a.m, sqrt(tot[0]));
    }
    if (coarse) {
      // y = T^-1 c: a warp per row, the rows dealt round-robin over blocks 1 .. G-1 (warp w
      // of block b takes rows (b - 1) + (G - 1) (w + 16 i)) so that each block has few; all
      // to block 0 when it is alone.  TQ loads in flight per lane (a whole row up to 1024)
      constexpr int TQ = 32;
      const int gw = G == 1 ? warp : (bid - 1) + (G - 1) * warp;
      const int nw = G == 1 ? kArnWarps : (G - 1) * kArnWarps;
      if constexpr (sizeof(TACC) == 8) {
        // c_a = uscale_a (sum of a's pieces, in piece order), every aggregate in every block
        for (int q = t; q < a.r; q += kArnThreads) {
          const int p0 = __ldg(a.agg_piece + q), p1 = __ldg(a.agg_piece + q + 1);
          double sum = 0.0;
          for (int pb = p0; pb < p1; pb += 8) {
            double v[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) v[u] = pb + u < p1 ? __ldcg(ctl.cpart + pb + u) : 0.0;
#pragma unroll
            for (int u = 0; u < 8; ++u) sum += v[u];
          }
          sc[q] = __ldg(a.uscale + q) * sum;
        }
        __syncthreads();
        const double mu = __ldcg(&ctl.scal[S_MU]);
        for (int row = gw; row < a.r; row += nw) {
          const double* tr = a.tinv + (size_t)row * a.r;
          double acc[2] = {0.0, 0.0};
          for (int b0 = 0; b0 < a.r; b0 += 32 * TQ) {
            double tv[TQ];
#pragma unroll
            for (int u = 0; u < TQ; ++u) {
              const int b = b0 + lane + 32 * u;
              tv[u] = b < a.r ? __ldg(tr + b) : 0.0;
            }
#pragma unroll
            for (int u = 0; u < TQ; ++u) {
              const int b = b0 + lane + 32 * u;
              if (b < a.r) acc[u & 1] += tv[u] * sc[b];
            }
          }
          const double y = warp_sum(acc[0] + acc[1]);
          if (lane == 0) {
            const double sd = __ldg(a.uscale + row) * (mu * y - sc[row]);
            __stcg(ctl.sdefl + row, sd);
            __stcg(ctl.sdefl32 + row, (float)sd);
          }
        }
      } else {
        // FP32 basis: s' is used in FP32, so the coarse solve runs in FP32 too (c from the
        // double-FP32 piece pairs, rounded once; the FP32 copy of T^-1; FP32 sums)
        float* scf = reinterpret_cast<float*>(sc);
        for (int q = t; q < a.r; q += kArnThreads) {
          const int p0 = sap ? sap[q] : __ldg(a.agg_piece + q);
          const int p1 = sap ? sap[q + 1] : __ldg(a.agg_piece + q + 1);
          float hs = 0.f, hc = 0.f;
          for (int pb = p0; pb < p1; pb += 8) {
            float2 v[8];
#pragma unroll
            for (int u = 0; u < 8; ++u)
              v[u] = pb + u < p1 ? __ldcg(reinterpret_cast<const float2*>(ctl.cpart + pb + u))
                                 : make_float2(0.f, 0.f);
#pragma unroll
            for (int u = 0; u < 8; ++u) arn_df_add(hs, hc, v[u].x, v[u].y);
          }
          scf[q] = (sus ? sus[q] : (float)__ldg(a.uscale + q)) * (hs + hc);
        }
        __syncthreads();
        const float mu = (float)__ldcg(&ctl.scal[S_MU]);
        for (int row = gw; row < a.r; row += nw) {
          // the row from shared memory when staged (a plain load), else from global memory
          const float* tr = stinv ? stinv + (size_t)warp * a.r : a.tinv32 + (size_t)row * a.r;
          float acc[4] = {0.f, 0.f, 0.f, 0.f};
          for (int b0 = 0; b0 < a.r; b0 += 32 * TQ) {
            float tv[TQ];
#pragma unroll
            for (int u = 0; u < TQ; ++u) {
              const int b = b0 + lane + 32 * u;
              tv[u] = b < a.r ? tr[b] : 0.f;
            }
#pragma unroll
            for (int u = 0; u < TQ; ++u) {
              const int b = b0 + lane + 32 * u;
              if (b < a.r) acc[u & 3] += tv[u] * scf[b];
            }
          }
          const float y = warp_sum((acc[0] + acc[1]) + (acc[2] + acc[3]));
          if (lane == 0) {
            const float sd = (sus ? sus[row] : (float)__ldg(a.uscale + row)) * (mu * y - scf[row]);
            __stcg(ctl.sdefl + row, (double)sd);
            __stcg(ctl.sdefl32 + row, sd);
          }
        }
      }
    }
    // this block's s' rows and (block 0) the rotations are published: arrive, then form the
    // diagonal part of the next step's SpMV for the first super-tile, which needs only
    // u_{j+1} (complete since the barrier), not s' or sigma_{j+1} (it overwrites c); then
    // wait for every block's arrival
    arn_arrive(&a.gbar[2]);
    if (k < a.jmax) arn_diag<ND, TV, TACC>(a, k, R0, R0 + a.RS < R1 ? R0 + a.RS : R1, Ws, Us);
    if (!arn_wait(&a.gbar[2], cbase + (unsigned)G * (unsigned)k)) {
      arn_timeout(ctl);
      return;
    }
    // the rotations' outputs are visible to every block: the same decision everywhere
    if (t == 0) ssig[k] = __ldcg(&ctl.sigma[k]);
    const int done = __ldcg(&ctl.flags[F_CYCLE_DONE]);
    __syncthreads();
    if (done) break;
  }
}

template <typename TV, typename TACC>
struct Arn {
  // rows of a super-tile: w and u_j slices, s' and the reduction scratch in kArnSmem
  static long long super_rows(int r) {
    const size_t fixed = ((size_t)r * sizeof(TACC) + 127) / 128 * 128 + kArnScratch +
                         sizeof(double) * kMaxK * kMaxK + kArnStaging + 256;
    if (fixed >= kArnSmem) return 0;
    return (long long)((kArnSmem - fixed) / (2 * sizeof(TACC))) / kArnUnit * kArnUnit;
  }
  template <int ND, bool DF>
  static cudaError_t prepare() {
    return cudaFuncSetAttribute(k_arnoldi<TV, TACC, ND, DF>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kArnSmem);
  }
  template <int ND, bool DF>
  static cudaError_t launch_nd(const CycleArgs& c, const ArnArgs<TV, TACC>& p, cudaStream_t st) {
    static cudaError_t prep = prepare<ND, DF>();
    if (prep != cudaSuccess) return prep;
    const int grid = p.units < c.sms ? p.units : c.sms;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)grid);
    cfg.blockDim = dim3((unsigned)kArnThreads);
    cfg.dynamicSmemBytes = kArnSmem;
    cfg.stream = st;
    cudaLaunchAttribute at[2];
    at[0].id = cudaLaunchAttributeCooperative;
    at[0].val.cooperative = 1;
    at[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[1].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    // a cooperative launch with programmatic serialisation; should the runtime refuse the
    // pair, the kernel runs cooperatively in plain stream order from then on (same result)
    static bool pdl_ok = true;
    cfg.numAttrs = (c.pdl && pdl_ok) ? 2 : 1;
    cudaError_t e = cudaLaunchKernelEx(&cfg, k_arnoldi<TV, TACC, ND, DF>, p);
    if (e != cudaSuccess && cfg.numAttrs == 2) {
      (void)cudaGetLastError();
      pdl_ok = false;
      cfg.numAttrs = 1;
      e = cudaLaunchKernelEx(&cfg, k_arnoldi<TV, TACC, ND, DF>, p);
    }
    return e;
  }
  static cudaError_t launch(const CycleArgs& c, int jmax, bool defl, cudaStream_t st) {
    ArnArgs<TV, TACC> p{};
    p.N = c.op.n;
    p.units = (int)(c.ldv / kArnUnit);
    p.jmax = jmax;
    p.m = c.m;
    p.pre = (defl && c.pdl) ? 1 : 0;
    p.defl = defl ? 1 : 0;
    p.r = defl ? c.op.defl.r : 0;
    p.RS = (int)super_rows(p.r);
    if (p.RS < kArnUnit) return cudaErrorInvalidValue;  // arnoldi_fusable rules this out
    p.ldv = c.ldv;
    p.ldd = c.op.ldd;
    p.V = static_cast<const TV*>(c.V);
    p.w = static_cast<TACC*>(c.w);
    p.dia = c.op.dia;
    if constexpr (sizeof(TACC) == 8) {
      p.dval = c.op.dval;
      p.auval = c.op.defl.auval;
      p.aup_val = c.op.defl.aup_val;
      p.sdefl = c.ctl.sdefl;
    } else {
      p.dval = c.op.dval32;
      p.auval = c.op.defl.auval32;
      p.aup_val = c.op.defl.aup_val32;
      p.sdefl = c.ctl.sdefl32;
    }
    p.aurp = c.op.defl.aurp;
    p.aup_col = c.op.defl.aup_col;
    p.aucol = c.op.defl.aucol;
    p.perm = c.op.defl.perm;
    p.piece_start = c.op.defl.piece_start;
    p.agg_piece = c.op.defl.agg_piece;
    p.blk_piece_start = c.op.defl.blk_piece_start;
    p.blk_piece = c.op.defl.blk_piece;
    p.uscale = c.op.defl.uscale;
    p.tinv = c.op.defl.tinv;
    p.tinv32 = c.op.defl.tinv32;
    p.ctl = c.ctl;
    p.gbar = c.gbar;
    // the 9-point stencils of the Q1 systems take an unrolled instantiation
    if constexpr (sizeof(TV) == 8) {
      if (c.dot_arith == GMRES_DOT_DF32)
        return c.op.dia.nd == 9 ? launch_nd<9, true>(c, p, st) : launch_nd<0, true>(c, p, st);
    }
    return c.op.dia.nd == 9 ? launch_nd<9, false>(c, p, st) : launch_nd<0, false>(c, p, st);
  }
};

}  // namespace

bool arnoldi_fusable(const CycleArgs& a) {
  if (!(a.ortho == GMRES_ORTHO_MGS_LOWSYNC && a.op.dia.nd > 0 && !a.proj &&
        a.op.defl.qd == 0 && a.ldv % kArnUnit == 0 && a.m + 1 <= kMaxK &&
        (a.prec == P_FP64 || a.prec == P_FP32)))
    return false;
  const int r = a.op.defl.r;
  // with deflation: the pieces split at this kernel's block rows (built at setup for a
  // grid of min(units, SMs) blocks)
  if (r > 0 && (!a.op.defl.blk_piece_start ||
                a.op.defl.blk_grid != (int)std::min<long long>(a.ldv / kArnUnit, a.sms)))
    return false;
  if (r > 0 && a.prec == P_FP32 && !a.op.defl.tinv32) return false;  // its FP32 coarse solve
  const long long rs = a.prec == P_FP64 ? Arn<double, double>::super_rows(r)
                                        : Arn<float, float>::super_rows(r);
  // c (r doubles) lives where w and u_j do
  const size_t esz = a.prec == P_FP64 ? sizeof(double) : sizeof(float);
  return rs >= kArnUnit && (size_t)r * sizeof(double) <= 2 * (size_t)rs * esz;
}

cudaError_t launch_arnoldi(const CycleArgs& a, int jmax, bool defl, cudaStream_t st) {
  switch (a.prec) {
    case P_FP64: return Arn<double, double>::launch(a, jmax, defl, st);
    case P_FP32: return Arn<float, float>::launch(a, jmax, defl, st);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace gg
