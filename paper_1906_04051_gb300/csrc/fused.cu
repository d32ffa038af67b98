// fused.cu -- a whole Arnoldi step of deflated GMRES(m) in one persistent kernel: the
// SpMV w = A M^-1 v_j (Eq. 10 with Eqs. 16-17), the paper's modified Gram-Schmidt
// projections (Eq. 13) in their one-reduction form, ||w|| and the plane rotations with the
// stopping tests (Eqs. 12, 14).
//
// One block per multiprocessor, launched cooperatively (every block resident).  Block b
// owns a contiguous range of rows (a multiple of 256) for the whole step:
//   1. SpMV of its rows into w (diagonal storage; the coarse correction through the A W
//      rows).  With deflation the diagonal part runs before the programmatic-launch wait,
//      overlapping the coarse solve that produces s'.
//   2. Multi-dot over the basis tiles of its rows: g = V^T w and the new row of L
//      (u_j . u_c), by 16 consumer warps (one column slice each) from a ring of
//      shared-memory stages that a producer warp fills with bulk asynchronous copies; each
//      stage has a full and an empty mbarrier, so no block barrier sits in the loop.
//   3. Grid barrier; every block adds the G partial sums in the same order (identical
//      totals in every block) and solves (I + L) h = g itself.
//   4. Update of its rows, u_{j+1} = w - V (sigma o h): each lane owns rows and reads the
//      basis straight from global memory, in the reverse order of step 2 so that the
//      tiles read last are still in L2; partial sums of ||u_{j+1}||^2.
//   5. The last block to finish (ticket counter) adds the norm partials and applies the
//      plane rotations and stopping tests (Eqs. 12, 14).
// Every reduction is formed in a fixed order: runs are bitwise reproducible.
#include <type_traits>
#include <utility>

#include "internal.h"
#include "kernels.cuh"

namespace gg {

namespace {

constexpr int kArnCW = 16;                       // consumer warps (one column slice each)
constexpr int kArnThreads = (kArnCW + 1) * 32;   // plus the producer warp
constexpr int kArnSliceCols = (kMaxK + kArnCW - 1) / kArnCW;  // 5 accumulators per set
constexpr int kArnMaxStages = 8;
constexpr int kArnUnit = 256;                    // rows per unit of the row partition
constexpr size_t kArnRing = 200 * 1024;          // the ring (dynamic shared memory)
// preferred stage size: FP64 (bound by its FMA pipe) keeps 128-row tiles longer, so that a
// tile's SpMV rows occupy four warps (one per scheduler); FP32 (bound by HBM) keeps stages
// small enough for six or more in the ring
template <typename TV> constexpr size_t arn_stage_cap() { return sizeof(TV) == 8 ? 48 * 1024 : 28 * 1024; }
constexpr long long kArnSpins = 1LL << 21;       // polls of the barrier word: about a second
constexpr int kArnNormCol = 2 * kMaxK;           // column of ctl.part holding the norm partials

template <typename TV, typename TACC>
struct ArnArgs {
  int N;          // rows of A
  int units;      // ldv / kArnUnit
  int j, k, m;    // step, basis columns in use (j + 1), restart length
  int TR, S;      // tile rows, ring stages
  int pre;        // the predecessor is the coarse solve: the basis and operator tiles may be
                  // prefetched before the wait
  int defl;       // add the coarse correction A W s'
  unsigned stage_bytes;
  // byte offsets of a stage's parts: basis tile (k columns), diagonals (nd), x windows,
  // A W row pointers, A W columns, A W values, and w (computed in place)
  unsigned offD, offX, offP, offC, offA, offW;
  int awcap;      // A W entries reserved per stage (a multiple of 4)
  int ng;         // x windows: groups of diagonals whose offsets lie close together
  int wlo[kMaxDiag];   // window g starts at row r0 + wlo[g] (elements, 16-byte aligned)
  int wlen[kMaxDiag];  // its length (elements, 16-byte multiple)
  int woff[kMaxDiag];  // its place in the stage's window part (elements)
  int gq[kMaxDiag + 1];  // diagonals gq[g] .. gq[g+1]-1 (sorted offsets) use window g
  long long ldv, ldd;
  const TV* V;    // basis, column-major (ldv)
  TACC* w;        // working vector
  DiaOffsets dia;
  const TACC* dval;
  const int* aurp;
  const int* aucol;
  const TACC* auval;
  const TACC* sdefl;
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

// Barrier of the first nthreads threads on named barrier id, returning the AND of v.
__device__ __forceinline__ bool bar_and(int id, int nthreads, bool v) {
  int r;
  asm volatile(
      "{\n .reg .pred p, q;\n setp.ne.u32 q, %1, 0;\n bar.red.and.pred p, %2, %3, q;\n"
      " selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(r)
      : "r"((int)v), "r"(id), "r"(nthreads)
      : "memory");
  return r != 0;
}

// Copy range of x window g for the tile at row r0: [cs, ce) clamped into [0, ldv) and
// never shorter than one 16-byte chunk (E elements), placed at element dpos of the window's
// part of the stage.  Element i of x is then read at  xb + clamp(i, cs, ce - 1), with
// xb = woff + dpos - cs: outside [0, n) the diagonal entries are 0, so the clamped (finite)
// value they meet contributes nothing.
struct ArnWin {
  long long cs, ce;
  long long xb;
};

__host__ __device__ __forceinline__ ArnWin arn_win(int wlo, int wlen, int woff, long long r0,
                                                   long long ldv, int E) {
  const long long start = r0 + wlo, end = start + wlen;
  ArnWin w;
  w.cs = start < 0 ? 0 : start;
  w.ce = end > ldv ? ldv : end;
  long long dpos = w.cs - start;
  if (w.ce - w.cs < E) {  // (almost) outside [0, ldv): one chunk at the window's start
    w.cs = start < 0 ? 0 : ldv - E;
    w.ce = w.cs + E;
    dpos = 0;
  }
  w.xb = woff + dpos - w.cs;
  return w;
}

// Multi-dot of one stage by consumer warp `sl` (columns sl, sl + 16, ...; NW of them):
// acc += V_c . w and acc2 += V_c . u_j over the stage's TR rows.
template <int NW, typename TV, typename TACC>
__device__ __forceinline__ void arn_dots(TACC (&acc)[kArnSliceCols], TACC (&acc2)[kArnSliceCols],
                                         const unsigned char* st, const TACC* sw, int k, int TR,
                                         int sl, int lane) {
  constexpr int VN = ArnVec<TV>::n;
  const TV* sV = reinterpret_cast<const TV*>(st);
  const TV* su = sV + (size_t)(k - 1) * TR;
  for (int r = lane * VN; r < TR; r += 32 * VN) {
    TACC wv[VN], uv[VN];
    ld_acc<VN>(sw + r, wv);
    ld_vec(su + r, uv);
#pragma unroll
    for (int i = 0; i < NW; ++i) {
      TACC v[VN];
      ld_vec(sV + (size_t)(sl + kArnCW * i) * TR + r, v);
#pragma unroll
      for (int e = 0; e < VN; ++e) {
        acc[i] += v[e] * wv[e];
        acc2[i] += v[e] * uv[e];
      }
    }
  }
}

#define GG_ARN_SWITCH(nw, CALL) \
  switch (nw) {                 \
    case 1: CALL(1); break;     \
    case 2: CALL(2); break;     \
    case 3: CALL(3); break;     \
    case 4: CALL(4); break;     \
    case 5: CALL(5); break;     \
    default: break;             \
  }

// 16-byte vector load / store of VN basis elements from global memory
template <typename TV, typename TACC, int VN>
__device__ __forceinline__ void arn_ldg(const TV* p, TACC (&o)[VN]) {
  if constexpr (std::is_same<TV, double>::value) {
    const double2 v = __ldg(reinterpret_cast<const double2*>(p));
    o[0] = (TACC)v.x;
    o[1] = (TACC)v.y;
  } else if constexpr (std::is_same<TV, float>::value) {
    const float4 v = __ldg(reinterpret_cast<const float4*>(p));
    o[0] = v.x; o[1] = v.y; o[2] = v.z; o[3] = v.w;
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

template <typename TACC, int VN>
__device__ __forceinline__ void arn_ldw(const TACC* p, TACC (&o)[VN]) {  // w: coherent loads
  if constexpr (sizeof(TACC) == 8) {
#pragma unroll
    for (int e = 0; e < VN; e += 2) {
      const double2 v = __ldcg(reinterpret_cast<const double2*>(p + e));
      o[e] = v.x;
      o[e + 1] = v.y;
    }
  } else {
#pragma unroll
    for (int e = 0; e < VN; e += 4) {
      const float4 v = __ldcg(reinterpret_cast<const float4*>(p + e));
      o[e] = v.x; o[e + 1] = v.y; o[e + 2] = v.z; o[e + 3] = v.w;
    }
  }
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

template <typename TV, typename TACC>
__global__ void __launch_bounds__(kArnThreads, 1)
    k_arnoldi(const __grid_constant__ ArnArgs<TV, TACC> a) {
  constexpr int VN = ArnVec<TV>::n;
  constexpr int E = 16 / (int)sizeof(TV);  // elements per 16-byte chunk of x
  extern __shared__ __align__(128) unsigned char ring[];
  __shared__ uint64_t full[kArnMaxStages], empty[kArnMaxStages];
  __shared__ double tot[2 * kMaxK + 1];
  __shared__ double sred[2 * kMaxK];
  __shared__ double sg[kMaxK];
  __shared__ TACC scoef[kMaxK];
  __shared__ double snrm[kArnThreads / 32];
  __shared__ unsigned s_last;
  Ctl ctl = a.ctl;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const bool prod = warp == kArnCW;
  const int ct = threadIdx.x;  // consumer thread index (warps 0..kArnCW-1)
  const int G = gridDim.x, bid = blockIdx.x;
  const long long R0 = (long long)bid * a.units / G * kArnUnit;
  const long long R1 = (long long)(bid + 1) * a.units / G * kArnUnit;
  const int k = a.k, TR = a.TR, S = a.S, nd = a.dia.nd;
  const int nt = (int)((R1 - R0) / TR);
  const int N = a.N;

  if (!a.pre) {
    pdl_wait();
    pdl_trigger();
  }
  // the flag is final here: set only by the previous step's rotations (complete before
  // this kernel's predecessor started when pre, waited for otherwise); the same value in
  // every block, so the whole grid returns together
  if (__ldcg(&ctl.flags[F_CYCLE_DONE])) {
    if (a.pre) {
      pdl_wait();
      pdl_trigger();
    }
    return;
  }
  const unsigned gen = *(volatile unsigned*)&a.gbar[1];  // advanced only once all arrive
  if (threadIdx.x == 0) {
    for (int s = 0; s < S; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], kArnCW);
    }
    mbar_fence_init();
  }
  __syncthreads();

  const TV* xj = a.V + (size_t)a.j * a.ldv;
  const uint32_t vbytes = (uint32_t)(TR * sizeof(TV)), dbytes = (uint32_t)(TR * sizeof(TACC));
  auto stage = [&](int s) { return ring + (size_t)s * a.stage_bytes; };

  // ---- 1-2. SpMV and multi-dot, tile by tile, from the ring ------------------------
  // Stage of tile i (rows r0 .. r0 + TR): the basis tile (columns 0..k-1), the diagonals,
  // the x windows and the A W rows, all copied by the producer warp; the consumers form
  // w for the tile's rows in the stage (and in global memory for the update), meet at a
  // named barrier, and run the multi-dot.
  TACC acc[kArnSliceCols], acc2[kArnSliceCols];
#pragma unroll
  for (int i = 0; i < kArnSliceCols; ++i) {
    acc[i] = 0;
    acc2[i] = 0;
  }
  bool ok = true;
  if (prod) {
    // A W row pointers at the tile boundaries, 32 tiles per refresh (lane l: tile base + l)
    int ap0 = 0, ap1 = 0, abase_tile = -32;
    for (int i = 0; i < nt; ++i) {
      const int s = i % S;
      if (i >= S) {  // stage s was last used by tile i - S: all consumer warps released it
        if (!mbar_wait(&empty[s], (uint32_t)(((i / S) - 1) & 1))) {
          ok = false;
          break;
        }
      }
      const long long r0 = R0 + (long long)i * TR;
      int abase = 0, acnt = 0;
      if (a.defl) {
        if (i - abase_tile >= 32) {
          abase_tile = i;
          const long long t0 = R0 + (long long)(i + lane) * TR, t1 = t0 + TR;
          ap0 = __ldg(a.aurp + (t0 < R1 ? t0 : R1));
          ap1 = __ldg(a.aurp + (t1 < R1 ? t1 : R1));
        }
        const int e0 = __shfl_sync(0xffffffffu, ap0, i - abase_tile);
        const int e1 = __shfl_sync(0xffffffffu, ap1, i - abase_tile);
        abase = e0 & ~3;
        acnt = (e1 - abase + 3) & ~3;
      }
      unsigned char* st = stage(s);
      if (lane == 0) {
        uint32_t bytes = (uint32_t)k * vbytes + (uint32_t)nd * dbytes;
        for (int g = 0; g < a.ng; ++g) {
          const ArnWin wg = arn_win(a.wlo[g], a.wlen[g], a.woff[g], r0, a.ldv, E);
          bytes += (uint32_t)((wg.ce - wg.cs) * (long long)sizeof(TV));
        }
        if (a.defl)
          bytes += (uint32_t)((TR + 4) * sizeof(int)) +
                   (uint32_t)acnt * (uint32_t)(sizeof(int) + sizeof(TACC));
        mbar_arrive_expect_tx(&full[s], bytes);
      }
      __syncwarp();
      for (int c = lane; c < k; c += 32)
        bulk_g2s(st + (size_t)c * vbytes, a.V + (size_t)c * a.ldv + r0, vbytes, &full[s]);
      for (int q = lane; q < nd; q += 32)
        bulk_g2s(st + a.offD + (size_t)q * dbytes, a.dval + (size_t)q * a.ldd + r0, dbytes,
                 &full[s]);
      for (int g = lane; g < a.ng; g += 32) {
        const ArnWin wg = arn_win(a.wlo[g], a.wlen[g], a.woff[g], r0, a.ldv, E);
        bulk_g2s(st + a.offX + (size_t)(wg.xb + wg.cs) * sizeof(TV), xj + wg.cs,
                 (uint32_t)((wg.ce - wg.cs) * (long long)sizeof(TV)), &full[s]);
      }
      if (a.defl) {
        if (lane == 0)
          bulk_g2s(st + a.offP, a.aurp + r0, (uint32_t)((TR + 4) * sizeof(int)), &full[s]);
        if (lane == 1 && acnt > 0)
          bulk_g2s(st + a.offC, a.aucol + abase, (uint32_t)(acnt * sizeof(int)), &full[s]);
        if (lane == 2 && acnt > 0)
          bulk_g2s(st + a.offA, a.auval + abase, (uint32_t)(acnt * sizeof(TACC)), &full[s]);
      }
    }
  } else {
    if (a.pre) {  // s' (the coarse solve's output) is read below
      pdl_wait();
      pdl_trigger();
    }
    const int nw = slice_cols(k, warp, kArnCW);
    const TACC sig = (TACC)__ldcg(&ctl.sigma[a.j]);
    for (int i = 0; i < nt; ++i) {
      const int s = i % S;
      const bool okw = mbar_wait(&full[s], (uint32_t)((i / S) & 1));
      const unsigned char* st = stage(s);
      TACC* sw = reinterpret_cast<TACC*>(const_cast<unsigned char*>(st) + a.offW);
      const long long r0 = R0 + (long long)i * TR;
      if (okw && ct < TR) {  // row r0 + ct of w = sigma_j (A u_j + A W s')
        const long long row = r0 + ct;
        TACC v = 0;
        if (row < N) {
          const TACC* sD = reinterpret_cast<const TACC*>(st + a.offD);
          const TV* sX = reinterpret_cast<const TV*>(st + a.offX);
          TACC p0 = 0, p1 = 0;
          int q = 0;
          for (int g = 0; g < a.ng; ++g) {
            const ArnWin wg = arn_win(a.wlo[g], a.wlen[g], a.woff[g], r0, a.ldv, E);
            const int qe = a.gq[g + 1];
            for (; q < qe; ++q) {
              long long xi = row + a.dia.off[q];
              xi = xi < wg.cs ? wg.cs : (xi >= wg.ce ? wg.ce - 1 : xi);
              const TACC t = sD[(size_t)q * TR + ct] * cv<TACC, TV>(sX[wg.xb + xi]);
              if (q & 1) p1 += t;
              else p0 += t;
            }
          }
          v = p0 + p1;
          if (a.defl) {
            const int* sP = reinterpret_cast<const int*>(st + a.offP);
            const int* sC = reinterpret_cast<const int*>(st + a.offC);
            const TACC* sA = reinterpret_cast<const TACC*>(st + a.offA);
            const int ab = sP[0] & ~3;
            const int e1 = sP[ct + 1] - ab;
            TACC aw = 0;
            for (int e = sP[ct] - ab; e < e1; ++e) aw += sA[e] * __ldg(a.sdefl + sC[e]);
            v += aw;
          }
          v *= sig;
          a.w[row] = v;
        }
        sw[ct] = v;  // rows past n stay 0
      }
      // the tile's w is complete; every consumer warp learns whether all copies arrived
      if (!bar_and(1, kArnCW * 32, okw)) {
        ok = false;
        break;
      }
#define GG_ARN_DOTS(NW) arn_dots<NW, TV, TACC>(acc, acc2, st, sw, k, TR, warp, lane)
      GG_ARN_SWITCH(nw, GG_ARN_DOTS)
#undef GG_ARN_DOTS
      __syncwarp();
      if (lane == 0) mbar_arrive(&empty[s]);
    }
  }
  if (!__syncthreads_and(ok)) {
    // a copy never completed: drain what is still in flight (bounded), report, return
    if (threadIdx.x == 0) {
      for (int i = 0; i < nt; ++i) mbar_wait(&full[i % S], (uint32_t)((i / S) & 1));
      ctl.flags[F_STATUS] = GMRES_ERR_TIMEOUT;
      ctl.flags[F_STOP] = 1;
      ctl.flags[F_CYCLE_DONE] = 1;
    }
    __syncthreads();
    return;
  }
  // per-block column sums: each column belongs to one warp; lanes' values transposed
  // through shared memory (the ring is free now) and summed 16 at a time by lane pairs
  {
    double* sbuf = reinterpret_cast<double*>(ring);  // [2][kArnCW][kArnSliceCols][33]
    if (!prod) {
      const int nw = slice_cols(k, warp, kArnCW);
#pragma unroll
      for (int i = 0; i < kArnSliceCols; ++i)
        if (i < nw) {
          sbuf[((0 * kArnCW + warp) * kArnSliceCols + i) * 33 + lane] = (double)acc[i];
          sbuf[((1 * kArnCW + warp) * kArnSliceCols + i) * 33 + lane] = (double)acc2[i];
        }
      __syncwarp();
      const int p = lane >> 1, half = lane & 1;  // pair p: set p / 5, accumulator p % 5
      const int set = p / kArnSliceCols, i = p % kArnSliceCols;
      double v = 0.0;
      const bool live = p < 2 * kArnSliceCols && i < nw;
      if (live) v = tree16(sbuf + ((set * kArnCW + warp) * kArnSliceCols + i) * 33 + half * 16);
      v += __shfl_xor_sync(0xffffffffu, v, 1);
      if (live && half == 0) sred[set * k + warp + kArnCW * i] = v;
    }
    __syncthreads();
    for (int c = threadIdx.x; c < 2 * k; c += blockDim.x)
      __stcg(&ctl.part[(size_t)bid * ctl.ldp + c], sred[c]);
  }
  // ---- 3. grid barrier; identical totals in every block; (I + L) h = g --------------
  if (!arn_grid_sync(a.gbar, gen)) {
    if (threadIdx.x == 0) {
      ctl.flags[F_STATUS] = GMRES_ERR_TIMEOUT;
      ctl.flags[F_STOP] = 1;
      ctl.flags[F_CYCLE_DONE] = 1;
    }
    return;
  }
  reduce_rows(ctl.part, G, 2 * k, ctl.ldp, tot);  // ends with __syncthreads
  {
    double* sL = reinterpret_cast<double*>(ring);  // k x k, strictly lower part used
    const double sj = __ldcg(&ctl.sigma[k - 1]);
    for (int t = threadIdx.x; t < k * k; t += blockDim.x) {
      const int i = t / k, c = t % k;
      double v = 0.0;
      if (c < i) v = i < k - 1 ? __ldcg(&ctl.L[(size_t)i * kMaxK + c])
                               : sj * __ldcg(&ctl.sigma[c]) * tot[k + c];
      sL[t] = v;
    }
    for (int c = threadIdx.x; c < k; c += blockDim.x) sg[c] = __ldcg(&ctl.sigma[c]) * tot[c];
    __syncthreads();
    if (warp == 0) {  // forward substitution: h_c final when reached (entries c, c+32, c+64)
      double g[3];
#pragma unroll
      for (int q = 0; q < 3; ++q) g[q] = lane + 32 * q < k ? sg[lane + 32 * q] : 0.0;
      for (int c = 0; c < k; ++c) {
        const double hc = __shfl_sync(0xffffffffu, c < 32 ? g[0] : (c < 64 ? g[1] : g[2]), c & 31);
#pragma unroll
        for (int q = 0; q < 3; ++q) {
          const int i = lane + 32 * q;
          if (i > c && i < k) g[q] -= sL[i * k + c] * hc;
        }
      }
#pragma unroll
      for (int q = 0; q < 3; ++q) {
        const int i = lane + 32 * q;
        if (i < k) {
          const double sc = __ldcg(&ctl.sigma[i]);
          scoef[i] = (TACC)(sc * g[q]);
          if (bid == 0) {
            ctl.h[i] = g[q];
            if (i < k - 1) ctl.L[(size_t)(k - 1) * kMaxK + i] = sL[(k - 1) * k + i];
          }
        }
      }
    }
    __syncthreads();
  }
  // ---- 4. update u_{j+1} = w - V (sigma o h) and ||u_{j+1}||^2 ----------------------
  double nrm = 0.0;
  if (!prod) {
    constexpr int U = sizeof(TV) == 8 ? 8 : 12;  // basis loads in flight per lane
    const int chunk = 32 * VN;
    const long long nch = (R1 - R0) / chunk;
    TV* __restrict__ vout = const_cast<TV*>(a.V) + (size_t)k * a.ldv;
    for (long long q = nch - 1 - warp; q >= 0; q -= kArnCW) {
      const long long r = R0 + q * chunk + (long long)lane * VN;
      TACC wv[VN], p[VN];
      arn_ldw<TACC, VN>(a.w + r, wv);
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
      if constexpr (std::is_same<TV, TACC>::value) {
        TACC s = 0;
#pragma unroll
        for (int e = 0; e < VN; ++e) s += un[e] * un[e];
        nrm += (double)s;
      } else {  // the norm of the stored (rounded) vector
        TACC s = 0;
#pragma unroll
        for (int e = 0; e < VN; ++e) {
          const TACC sv = cv<TACC, TV>(st_round<TV>((float)un[e]));
          s += sv * sv;
        }
        nrm += (double)s;
      }
    }
  }
  // ---- 5. norm partials; the last block applies the rotations -----------------------
  {
    const double bs = block_sum(nrm, snrm);
    if (threadIdx.x == 0) {
      __stcg(&ctl.part[(size_t)bid * ctl.ldp + kArnNormCol], bs);
      __threadfence();
      s_last = (atomicAdd(&ctl.ticket[0], 1u) == (unsigned)G - 1u) ? 1u : 0u;
      if (s_last) __threadfence();
    }
    __syncthreads();
    if (!s_last) return;
    reduce_rows(ctl.part + kArnNormCol, G, 1, ctl.ldp, tot);
    if (threadIdx.x == 0) ctl.ticket[0] = 0u;
    givens_step(ctl, k - 1, a.m, sqrt(tot[0]));
  }
}

template <typename TV, typename TACC>
struct Arn {
  struct Layout {
    int TR, S, ng, awcap;
    unsigned offD, offX, offP, offC, offA, offW, bytes;
    int wlo[kMaxDiag], wlen[kMaxDiag], woff[kMaxDiag], gq[kMaxDiag + 1];
  };
  static unsigned up(size_t b) { return (unsigned)((b + 127) / 128 * 128); }
  // x windows: diagonals whose sorted offsets lie within kArnGap of the previous one share
  // a window; for tile rows TR, window g covers rows [r0 + wlo, r0 + wlo + wlen)
  static Layout layout(const CycleArgs& c, int k, int TR, bool defl, int au_tile_max) {
    constexpr int E = 16 / (int)sizeof(TV);
    constexpr int kArnGap = 32;
    Layout L{};
    L.TR = TR;
    const DiaOffsets& d = c.op.dia;
    int woff = 0;
    for (int q = 0; q < d.nd;) {
      int qe = q + 1;
      while (qe < d.nd && d.off[qe] - d.off[qe - 1] <= kArnGap) ++qe;
      const int lo = d.off[q], hi = d.off[qe - 1];
      auto fdiv = [](int a, int b) { return (a >= 0 ? a / b : -((-a + b - 1) / b)); };
      const int wlo = fdiv(lo, E) * E;
      const int whi = fdiv(TR + hi + E - 1, E) * E;
      L.wlo[L.ng] = wlo;
      L.wlen[L.ng] = whi - wlo;
      L.woff[L.ng] = woff;
      L.gq[L.ng] = q;
      woff += whi - wlo;
      ++L.ng;
      q = qe;
    }
    L.gq[L.ng] = d.nd;
    L.awcap = defl ? (au_tile_max + 8 + 3) / 4 * 4 : 0;
    size_t off = up((size_t)k * TR * sizeof(TV));
    L.offD = (unsigned)off;
    off += up((size_t)d.nd * TR * sizeof(TACC));
    L.offX = (unsigned)off;
    off += up((size_t)woff * sizeof(TV));
    L.offP = (unsigned)off;
    off += defl ? up((size_t)(TR + 4) * sizeof(int)) : 0;
    L.offC = (unsigned)off;
    off += up((size_t)L.awcap * sizeof(int));
    L.offA = (unsigned)off;
    off += up((size_t)L.awcap * sizeof(TACC));
    L.offW = (unsigned)off;
    off += up((size_t)TR * sizeof(TACC));
    L.bytes = (unsigned)off;
    const int S = (int)(kArnRing / off);
    L.S = S > kArnMaxStages ? kArnMaxStages : S;
    return L;
  }
  // tile rows: the largest of 256 / 128 / 64 whose stage fits the cap, and at least one
  // full sweep of a warp (32 lanes x one 16-byte vector)
  static Layout pick(const CycleArgs& c, int k, bool defl, int au_tile_max) {
    constexpr int lo = 32 * ArnVec<TV>::n;
    Layout L = layout(c, k, kArnUnit, defl, au_tile_max);
    for (int tr = kArnUnit / 2; tr >= lo && L.bytes > arn_stage_cap<TV>(); tr >>= 1)
      L = layout(c, k, tr, defl, au_tile_max);
    return L;
  }
  static cudaError_t prepare() {
    return cudaFuncSetAttribute(k_arnoldi<TV, TACC>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)kArnRing);
  }
  static cudaError_t launch(const CycleArgs& c, int j, bool defl, cudaStream_t st) {
    static cudaError_t prep = prepare();
    if (prep != cudaSuccess) return prep;
    ArnArgs<TV, TACC> p{};
    const Layout L = pick(c, j + 1, defl, c.op.au_tile_max);
    if (L.S < 2) return cudaErrorInvalidValue;  // arnoldi_fusable keeps this from happening
    p.N = c.op.n;
    p.units = (int)(c.ldv / kArnUnit);
    p.j = j;
    p.k = j + 1;
    p.m = c.m;
    p.TR = L.TR;
    p.S = L.S;
    p.stage_bytes = L.bytes;
    p.offD = L.offD;
    p.offX = L.offX;
    p.offP = L.offP;
    p.offC = L.offC;
    p.offA = L.offA;
    p.offW = L.offW;
    p.awcap = L.awcap;
    p.ng = L.ng;
    for (int g = 0; g < L.ng; ++g) {
      p.wlo[g] = L.wlo[g];
      p.wlen[g] = L.wlen[g];
      p.woff[g] = L.woff[g];
    }
    for (int g = 0; g <= L.ng; ++g) p.gq[g] = L.gq[g];
    p.pre = (defl && c.pdl) ? 1 : 0;
    p.defl = defl ? 1 : 0;
    p.ldv = c.ldv;
    p.ldd = c.op.ldd;
    p.V = static_cast<const TV*>(c.V);
    p.w = static_cast<TACC*>(c.w);
    p.dia = c.op.dia;
    if constexpr (sizeof(TACC) == 8) {
      p.dval = c.op.dval;
      p.auval = c.op.defl.auval;
      p.sdefl = c.ctl.sdefl;
    } else {
      p.dval = c.op.dval32;
      p.auval = c.op.defl.auval32;
      p.sdefl = c.ctl.sdefl32;
    }
    p.aurp = c.op.defl.aurp;
    p.aucol = c.op.defl.aucol;
    p.ctl = c.ctl;
    p.gbar = c.gbar;
    const int grid = p.units < c.sms ? p.units : c.sms;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)grid);
    cfg.blockDim = dim3((unsigned)kArnThreads);
    cfg.dynamicSmemBytes = kArnRing;
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
    cudaError_t e = cudaLaunchKernelEx(&cfg, k_arnoldi<TV, TACC>, p);
    if (e != cudaSuccess && cfg.numAttrs == 2) {
      (void)cudaGetLastError();
      pdl_ok = false;
      cfg.numAttrs = 1;
      e = cudaLaunchKernelEx(&cfg, k_arnoldi<TV, TACC>, p);
    }
    return e;
  }
};

}  // namespace

bool arnoldi_fusable(const CycleArgs& a) {
  if (!(a.ortho == GMRES_ORTHO_MGS_LOWSYNC && a.op.dia.nd > 0 && !a.proj &&
        a.op.defl.qd == 0 && a.ldv % kArnUnit == 0 && a.m + 1 <= kMaxK &&
        a.op.ldd % kArnUnit == 0 && (a.prec == P_FP64 || a.prec == P_FP32)))
    return false;
  // the widest stage (k = m + 1 columns) must leave a ring of at least two stages
  const bool defl = a.op.defl.r > 0;
  if (a.prec == P_FP64) return Arn<double, double>::pick(a, a.m + 1, defl, a.op.au_tile_max).S >= 2;
  return Arn<float, float>::pick(a, a.m + 1, defl, a.op.au_tile_max).S >= 2;
}

cudaError_t launch_arnoldi(const CycleArgs& a, int j, bool defl, cudaStream_t st) {
  switch (a.prec) {
    case P_FP64: return Arn<double, double>::launch(a, j, defl, st);
    case P_FP32: return Arn<float, float>::launch(a, j, defl, st);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace gg
