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
constexpr size_t kArnStageCap = 28 * 1024;       // preferred stage size (FP64 tiles)
constexpr long long kArnSpins = 1LL << 21;       // polls of the barrier word: about a second
constexpr int kArnNormCol = 2 * kMaxK;           // column of ctl.part holding the norm partials

template <typename TV, typename TACC>
struct ArnArgs {
  int N;          // rows of A
  int units;      // ldv / kArnUnit
  int j, k, m;    // step, basis columns in use (j + 1), restart length
  int TR, S;      // tile rows, ring stages
  int pre;        // the predecessor is the coarse solve: the SpMV's diagonal part and the
                  // basis prefetch may run before the wait
  int defl;       // add the coarse correction A W s'
  unsigned stage_bytes;
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

// Diagonal part of SpMV row i: sum_q dval[q][i] x[i + off_q] (index clamped to a valid
// row, where the stored value is 0).
template <typename TA, typename TV, typename TACC>
__device__ __forceinline__ TACC arn_dia_row(long long i, int N, const int* soff, int nd,
                                            long long ldd, const TA* __restrict__ dval,
                                            const TV* __restrict__ x) {
  TACC acc0 = 0, acc1 = 0;
  int q = 0;
  for (; q + 3 < nd; q += 4) {
    TACC av[4], xv[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const long long c = min(max(i + soff[q + u], 0LL), (long long)N - 1);
      av[u] = (TACC)__ldg(dval + (size_t)(q + u) * ldd + i);
      xv[u] = ld_as<TACC, TV>(x + c);
    }
    acc0 += av[0] * xv[0];
    acc1 += av[1] * xv[1];
    acc0 += av[2] * xv[2];
    acc1 += av[3] * xv[3];
  }
  for (; q < nd; ++q) {
    const long long c = min(max(i + soff[q], 0LL), (long long)N - 1);
    acc0 += (TACC)__ldg(dval + (size_t)q * ldd + i) * ld_as<TACC, TV>(x + c);
  }
  return acc0 + acc1;
}

// Multi-dot of one stage by consumer warp `sl` (columns sl, sl + 16, ...; NW of them):
// acc += V_c . w and acc2 += V_c . u_j over the stage's TR rows.
template <int NW, typename TV, typename TACC>
__device__ __forceinline__ void arn_dots(TACC (&acc)[kArnSliceCols], TACC (&acc2)[kArnSliceCols],
                                         const unsigned char* st, int k, int TR, int sl,
                                         int lane) {
  constexpr int VN = ArnVec<TV>::n;
  const TV* sV = reinterpret_cast<const TV*>(st);
  const TV* su = sV + (size_t)(k - 1) * TR;
  const TACC* sw = reinterpret_cast<const TACC*>(st + (size_t)k * TR * sizeof(TV));
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
  extern __shared__ __align__(128) unsigned char ring[];
  __shared__ uint64_t full[kArnMaxStages], empty[kArnMaxStages];
  __shared__ double tot[2 * kMaxK + 1];
  __shared__ double sred[2 * kMaxK];
  __shared__ double sg[kMaxK];
  __shared__ TACC scoef[kMaxK];
  __shared__ int soff[kMaxDiag];
  __shared__ double snrm[kArnThreads / 32];
  __shared__ unsigned s_last;
  Ctl ctl = a.ctl;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const bool prod = warp == kArnCW;
  const int ct = threadIdx.x;  // consumer thread index (warps 0..kArnCW-1)
  const int G = gridDim.x, bid = blockIdx.x;
  const long long R0 = (long long)bid * a.units / G * kArnUnit;
  const long long R1 = (long long)(bid + 1) * a.units / G * kArnUnit;
  const int k = a.k, TR = a.TR, S = a.S;
  const int nt = (int)((R1 - R0) / TR);
  const int N = a.N;
  const long long Rn = R1 < N ? R1 : N;  // rows of A in this block's range

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
  if (threadIdx.x < kMaxDiag) soff[threadIdx.x] = a.dia.off[threadIdx.x];
  if (threadIdx.x == 0) {
    for (int s = 0; s < S; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], kArnCW);
    }
    mbar_fence_init();
  }
  __syncthreads();

  const TV* xj = a.V + (size_t)a.j * a.ldv;
  const uint32_t vbytes = (uint32_t)(TR * sizeof(TV)), wbytes = (uint32_t)(TR * sizeof(TACC));
  auto stage = [&](int s) { return ring + (size_t)s * a.stage_bytes; };
  const int first = nt < S ? nt : S;
  // ---- 1. SpMV (producer: the first stages' basis columns meanwhile) ----------------
  if (prod) {
    if (lane == 0)
      for (int i = 0; i < first; ++i) mbar_arrive_expect_tx(&full[i], (uint32_t)k * vbytes + wbytes);
    __syncwarp();
    for (int i = 0; i < first; ++i) {
      const long long r0 = R0 + (long long)i * TR;
      TV* dst = reinterpret_cast<TV*>(stage(i));
      for (int c = lane; c < k; c += 32)
        bulk_g2s(dst + (size_t)c * TR, a.V + (size_t)c * a.ldv + r0, vbytes, &full[i]);
    }
  } else {
    const TACC sig = (TACC)__ldcg(&ctl.sigma[a.j]);
    for (long long i = R0 + ct; i < Rn; i += kArnCW * 32) {
      const TACC v = arn_dia_row<TACC, TV, TACC>(i, N, soff, a.dia.nd, a.ldd, a.dval, xj);
      a.w[i] = a.defl ? v : sig * v;
    }
  }
  if (a.pre) {
    pdl_wait();
    pdl_trigger();
  }
  if (!prod) {
    if (a.defl) {  // + A W s' (s' from the coarse solve), then the scale sigma_j
      const TACC sig = (TACC)__ldcg(&ctl.sigma[a.j]);
      for (long long i = R0 + ct; i < Rn; i += kArnCW * 32)
        a.w[i] = sig * (a.w[i] + au_row<TACC, TACC>((int)i, a.aurp, a.aucol, a.auval, a.sdefl));
    }
    // the slices of w are read below by the bulk-copy (async) proxy
    asm volatile("fence.proxy.async.global;" ::: "memory");
  }
  __syncthreads();

  // ---- 2. multi-dot over the ring ---------------------------------------------------
  TACC acc[kArnSliceCols], acc2[kArnSliceCols];
#pragma unroll
  for (int i = 0; i < kArnSliceCols; ++i) {
    acc[i] = 0;
    acc2[i] = 0;
  }
  bool ok = true;
  if (prod) {
    if (lane == 0)
      for (int i = 0; i < first; ++i)
        bulk_g2s(stage(i) + (size_t)k * vbytes, a.w + R0 + (long long)i * TR, wbytes, &full[i]);
    for (int i = first; i < nt; ++i) {
      const int s = i % S;
      // stage s was last used by tile i - S: all consumer warps must have released it
      if (!mbar_wait(&empty[s], (uint32_t)(((i / S) - 1) & 1))) {
        ok = false;
        break;
      }
      const long long r0 = R0 + (long long)i * TR;
      if (lane == 0) mbar_arrive_expect_tx(&full[s], (uint32_t)k * vbytes + wbytes);
      __syncwarp();
      TV* dst = reinterpret_cast<TV*>(stage(s));
      for (int c = lane; c < k; c += 32)
        bulk_g2s(dst + (size_t)c * TR, a.V + (size_t)c * a.ldv + r0, vbytes, &full[s]);
      if (lane == 0) bulk_g2s(stage(s) + (size_t)k * vbytes, a.w + r0, wbytes, &full[s]);
    }
  } else {
    const int nw = slice_cols(k, warp, kArnCW);
    for (int i = 0; i < nt; ++i) {
      const int s = i % S;
      if (!mbar_wait(&full[s], (uint32_t)((i / S) & 1))) {
        ok = false;
        break;
      }
#define GG_ARN_DOTS(NW) arn_dots<NW, TV, TACC>(acc, acc2, stage(s), k, TR, warp, lane)
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
  static size_t stage_bytes(int k, int TR) {
    return ((size_t)k * TR * sizeof(TV) + (size_t)TR * sizeof(TACC) + 127) / 128 * 128;
  }
  // tile rows: FP64 keeps stages near kArnStageCap (its passes are bound by the FP64 pipe,
  // so more stages matter less than short tiles); FP32 and BF16 take 256-row tiles, which
  // keeps every lane of a slice busy (32 lanes x 4 or 8 rows of a 16-byte load)
  static int tile_rows(int k) {
    constexpr int lo = 2 * 32 * ArnVec<TV>::n;  // two row sweeps of a warp at least
    int tr = kArnUnit;
    if (sizeof(TV) == 8)
      while (tr > lo && stage_bytes(k, tr) > kArnStageCap) tr >>= 1;
    return tr < lo ? lo : tr;
  }
  static cudaError_t prepare() {
    return cudaFuncSetAttribute(k_arnoldi<TV, TACC>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)kArnRing);
  }
  static cudaError_t launch(const CycleArgs& c, int j, bool defl, cudaStream_t st) {
    static cudaError_t prep = prepare();
    if (prep != cudaSuccess) return prep;
    ArnArgs<TV, TACC> p{};
    p.N = c.op.n;
    p.units = (int)(c.ldv / kArnUnit);
    p.j = j;
    p.k = j + 1;
    p.m = c.m;
    p.TR = tile_rows(p.k);
    const size_t sb = stage_bytes(p.k, p.TR);
    int S = (int)(kArnRing / sb);
    p.S = S > kArnMaxStages ? kArnMaxStages : S;
    p.stage_bytes = (unsigned)sb;
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
  return a.ortho == GMRES_ORTHO_MGS_LOWSYNC && a.op.dia.nd > 0 && !a.proj &&
         a.op.defl.qd == 0 && a.ldv % kArnUnit == 0 && a.m + 1 <= kMaxK &&
         (a.prec == P_FP64 || a.prec == P_FP32);
}

cudaError_t launch_arnoldi(const CycleArgs& a, int j, bool defl, cudaStream_t st) {
  switch (a.prec) {
    case P_FP64: return Arn<double, double>::launch(a, j, defl, st);
    case P_FP32: return Arn<float, float>::launch(a, j, defl, st);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace gg
