// setup.cu -- gmres_create's device work (Sec. 3.3, Eqs. 17-18): CSR validation, the
// aggregate permutation and piece list used by U^T v, U's column scaling, the coarse
// matrix T = U^T A U and its inverse by Gauss-Jordan elimination with partial pivoting.
//
// Every step is deterministic: integer counting, stable sequential placement inside a
// block, and floating-point sums taken in a fixed order.
#include "common.cuh"
#include "internal.h"

namespace gg {

namespace {

// ---- validation: sets err bits (1 = CSR structure, 2 = agg out of range) ----
__global__ void k_validate(int n, long long nnz, const int* __restrict__ rowptr,
                           const int* __restrict__ col, const int* __restrict__ agg, int r,
                           int* __restrict__ err) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const int s = rowptr[i], e = rowptr[i + 1];
    bool bad = (s > e) || (s < 0) || ((long long)e > nnz);
    if (i == 0 && s != 0) bad = true;
    if (i == n - 1 && (long long)e != nnz) bad = true;
    if (!bad) {
      int prev = -1;
      for (int k = s; k < e; ++k) {
        const int c = col[k];
        if (c < 0 || c >= n || c <= prev) { bad = true; break; }
        prev = c;
      }
    }
    if (bad) atomicOr(err, 1);
    if (agg) {
      const int a = agg[i];
      if (a < -1 || a >= r) atomicOr(err, 2);
    }
  }
}

// ---- aggregate permutation: per-chunk counts, scan, stable scatter ----
constexpr int kChunk = 16384;  // nodes per counting block

__global__ void k_agg_count(int n, int r, const int* __restrict__ agg, int* __restrict__ counts) {
  extern __shared__ int scnt[];
  for (int a = threadIdx.x; a < r; a += blockDim.x) scnt[a] = 0;
  __syncthreads();
  const int base = blockIdx.x * kChunk;
  const int end = min(n, base + kChunk);
  for (int i = base + threadIdx.x; i < end; i += blockDim.x) {
    const int a = agg[i];
    if (a >= 0) atomicAdd(&scnt[a], 1);
  }
  __syncthreads();
  for (int a = threadIdx.x; a < r; a += blockDim.x) counts[(size_t)blockIdx.x * r + a] = scnt[a];
}

// Single block: counts[b][a] -> global start offsets of chunk b's nodes of aggregate a;
// aggptr[a] (r+1) -> start of aggregate a in perm; cnt[a] -> size of aggregate a.
__global__ void k_agg_scan(int r, int nb, int* __restrict__ counts, int* __restrict__ aggptr,
                           int* __restrict__ cnt) {
  for (int a = threadIdx.x; a < r; a += blockDim.x) {
    int run = 0;
    for (int b = 0; b < nb; ++b) {
      const int c = counts[(size_t)b * r + a];
      counts[(size_t)b * r + a] = run;
      run += c;
    }
    cnt[a] = run;
  }
  __syncthreads();
  if (threadIdx.x == 0) {  // r <= 6144: a sequential scan is cheap and exact
    int run = 0;
    for (int a = 0; a < r; ++a) {
      aggptr[a] = run;
      run += cnt[a];
    }
    aggptr[r] = run;
  }
  __syncthreads();
  for (int a = threadIdx.x; a < r; a += blockDim.x) {
    const int base = aggptr[a];
    for (int b = 0; b < nb; ++b) counts[(size_t)b * r + a] += base;
  }
}

// Stable: the chunk's nodes of each aggregate land in increasing index order.  One warp
// takes 32 consecutive nodes at a time; the lanes of equal aggregate find each other
// (match), take consecutive slots in lane order, and the lowest of them advances the
// aggregate's offset.
__global__ void k_agg_scatter(int n, int r, const int* __restrict__ agg,
                              const int* __restrict__ counts, int* __restrict__ perm) {
  extern __shared__ int soff[];
  for (int a = threadIdx.x; a < r; a += blockDim.x) soff[a] = counts[(size_t)blockIdx.x * r + a];
  __syncthreads();
  if (threadIdx.x < 32) {
    const int lane = threadIdx.x;
    const int base = blockIdx.x * kChunk;
    const int end = min(n, base + kChunk);
    for (int i0 = base; i0 < end; i0 += 32) {
      const int i = i0 + lane;
      const int a = i < end ? agg[i] : -1;
      const unsigned peers = __match_any_sync(0xffffffffu, a);
      const int off = a >= 0 ? soff[a] : 0;
      __syncwarp();
      if (a >= 0) {
        perm[off + __popc(peers & ((1u << lane) - 1u))] = i;
        if (lane == __ffs(peers) - 1) soff[a] = off + __popc(peers);
      }
      __syncwarp();
    }
  }
}

// Pieces: aggregate a's range of perm (its nodes in increasing order) is cut where the
// nodes pass from one block's rows to the next block's, for a grid of G blocks owning the
// row ranges [floor(b U / G), floor((b + 1) U / G)) x kPartUnit of U = ldv / kPartUnit units
// (the fused Arnoldi kernel's partition; G = 0: no cuts), and every part into ranges of at
// most kPiece nodes.  piece_walk counts a's pieces and, given out, writes their starts.
__device__ __forceinline__ long long part_block(long long row, int U, int G) {
  return ((row / kPartUnit + 1) * G + U - 1) / U - 1;
}

__device__ int piece_walk(const int* __restrict__ perm, int s, int e, int U, int G, int* out) {
  int np = 0;
  for (int t = s; t < e;) {
    int te = e;
    if (G > 0) {
      const long long b = part_block(perm[t], U, G);
      const long long rend = (b + 1) * U / G * kPartUnit;
      int lo = t + 1, hi = e;  // the first node at or past rend
      while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (perm[mid] < rend) lo = mid + 1;
        else hi = mid;
      }
      te = lo;
    }
    for (int q = t; q < te; q += kPiece) {
      if (out) out[np] = q;
      ++np;
    }
    t = te;
  }
  return np;
}

// one block of 1024 threads: pieces per aggregate, their exclusive scan (agg_piece), the
// piece starts, 1 / sqrt|a|
__global__ void __launch_bounds__(1024)
    k_pieces(int r, int U, int G, const int* __restrict__ perm, const int* __restrict__ aggptr,
             const int* __restrict__ cnt, int* __restrict__ agg_piece,
             int* __restrict__ piece_start, double* __restrict__ uscale, int* __restrict__ err) {
  __shared__ int ssum[1024];
  const int t = threadIdx.x;
  const int per = (r + 1023) / 1024;  // consecutive aggregates per thread
  const int a0 = t * per, a1 = min(r, a0 + per);
  int mine = 0;
  for (int a = a0; a < a1; ++a) {
    const int np = piece_walk(perm, aggptr[a], aggptr[a + 1], U, G, nullptr);
    agg_piece[a] = np;
    mine += np;
  }
  ssum[t] = mine;
  __syncthreads();
  for (int o = 1; o < 1024; o <<= 1) {  // inclusive scan of the threads' totals
    const int v = t >= o ? ssum[t - o] : 0;
    __syncthreads();
    ssum[t] += v;
    __syncthreads();
  }
  int run = ssum[t] - mine;
  for (int a = a0; a < a1; ++a) {
    const int np = agg_piece[a];
    agg_piece[a] = run;
    piece_walk(perm, aggptr[a], aggptr[a + 1], U, G, piece_start + run);
    run += np;
    if (cnt[a] == 0) atomicOr(err, 4);
    uscale[a] = cnt[a] > 0 ? 1.0 / sqrt((double)cnt[a]) : 0.0;
  }
  if (t == 1023) {
    agg_piece[r] = ssum[1023];
    piece_start[ssum[1023]] = aggptr[r];
  }
}

// The pieces of each block of that grid, in piece (aggregate) order: block b counts the
// pieces whose first node lies in its rows, then (second launch) writes their indexes
// from its offset by a stable block-wide compaction.
__global__ void k_blk_count(int U, const int* __restrict__ perm,
                            const int* __restrict__ piece_start, const int* __restrict__ agg_piece,
                            int r, int* __restrict__ bcnt) {
  __shared__ int swarp[32];
  const int np = agg_piece[r];
  const int G = gridDim.x;
  int c = 0;
  for (int p = threadIdx.x; p < np; p += blockDim.x)
    c += part_block(perm[piece_start[p]], U, G) == blockIdx.x ? 1 : 0;
  for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
  if ((threadIdx.x & 31) == 0) swarp[threadIdx.x >> 5] = c;
  __syncthreads();
  if (threadIdx.x == 0) {
    int s = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += swarp[w];
    bcnt[blockIdx.x] = s;
  }
}

__global__ void k_blk_fill(int U, const int* __restrict__ perm, const int* __restrict__ piece_start,
                           const int* __restrict__ agg_piece, int r, const int* __restrict__ bcnt,
                           int* __restrict__ blk_piece_start, int* __restrict__ blk_piece) {
  __shared__ int swarp[32];
  __shared__ int s_base;
  const int np = agg_piece[r];
  const int G = gridDim.x, b = blockIdx.x;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  if (threadIdx.x == 0) {
    int off = 0;
    for (int q = 0; q < b; ++q) off += bcnt[q];
    blk_piece_start[b] = off;
    if (b == G - 1) blk_piece_start[G] = off + bcnt[b];
    s_base = off;
  }
  __syncthreads();
  for (int p0 = 0; p0 < np; p0 += blockDim.x) {
    const int p = p0 + threadIdx.x;
    const bool mine = p < np && part_block(perm[piece_start[p]], U, G) == b;
    const unsigned bal = __ballot_sync(0xffffffffu, mine);
    if (lane == 0) swarp[warp] = __popc(bal);
    __syncthreads();
    int before = 0, total = 0;
    for (int w = 0; w < nw; ++w) {
      before += w < warp ? swarp[w] : 0;
      total += swarp[w];
    }
    if (mine) blk_piece[s_base + before + __popc(bal & ((1u << lane) - 1u))] = p;
    __syncthreads();
    if (threadIdx.x == 0) s_base += total;
    __syncthreads();
  }
}

// T row of aggregate p: sum_{i in p} sum_{k in row i, agg(col_k) = q} a_ik, in perm order.
// Small r: lanes take nodes round-robin into private rows, summed in lane order.
// Large r: the aggregates the block meets are found first; when there are at most kTLocal
// of them (the neighbours of a structured partition: 9) the lanes keep private sums of
// just those, summed in lane order; else lane 0 accumulates sequentially.
constexpr int kTLocal = 32;
__global__ void k_T_rows(int r, const int* __restrict__ rowptr, const int* __restrict__ col,
                         const double* __restrict__ val, const int* __restrict__ agg,
                         const int* __restrict__ perm, const int* __restrict__ aggptr,
                         const double* __restrict__ uscale, double* __restrict__ T) {
  extern __shared__ double srow[];
  const int p = blockIdx.x, lane = threadIdx.x;
  const int s = aggptr[p], e = aggptr[p + 1];
  const bool lane_rows = (r * 32 * (int)sizeof(double)) <= 48 * 1024;
  const int nrows = lane_rows ? 32 : 1;
  for (int t = lane; t < nrows * r; t += 32) srow[t] = 0.0;
  __syncwarp();
  if (lane_rows) {
    double* mine = srow + (size_t)lane * r;
    for (int t = s + lane; t < e; t += 32) {
      const int i = perm[t];
      for (int k = rowptr[i]; k < rowptr[i + 1]; ++k) {
        const int q = agg[col[k]];
        if (q >= 0) mine[q] += val[k];
      }
    }
    __syncwarp();
    for (int q = lane; q < r; q += 32) {
      double acc = 0.0;
      for (int l = 0; l < 32; ++l) acc += srow[(size_t)l * r + q];
      T[(size_t)p * r + q] = acc * uscale[p] * uscale[q];
    }
  } else {
    // the aggregates that row block p meets, as a bitmap, then their ranks (a prefix of the
    // words' popcounts) and list
    const int nw = (r + 31) / 32;
    unsigned* bm = reinterpret_cast<unsigned*>(srow + r);
    int* pre = reinterpret_cast<int*>(bm + nw);
    int* qlist = pre + nw;  // kTLocal
    double* priv = reinterpret_cast<double*>(qlist + kTLocal + (kTLocal & 1));
    __shared__ int s_nq;
    for (int w = lane; w < nw; w += 32) bm[w] = 0u;
    __syncwarp();
    for (int t = s + lane; t < e; t += 32) {
      const int i = perm[t];
      for (int k = rowptr[i]; k < rowptr[i + 1]; ++k) {
        const int q = agg[col[k]];
        if (q >= 0) atomicOr(&bm[q >> 5], 1u << (q & 31));
      }
    }
    __syncwarp();
    if (lane == 0) {
      int run = 0;
      for (int w = 0; w < nw; ++w) {
        pre[w] = run;
        unsigned m = bm[w];
        while (m) {
          const int b = __ffs(m) - 1;
          if (run < kTLocal) qlist[run] = w * 32 + b;
          ++run;
          m &= m - 1u;
        }
      }
      s_nq = run;
    }
    __syncwarp();
    const int nq = s_nq;
    if (nq <= kTLocal) {
      // lane l sums the nodes l, l + 32, ... (perm order) into its own slots, one per met
      // aggregate; the lanes' sums are then added in lane order
      for (int q = 0; q < nq; ++q) priv[lane * (kTLocal + 1) + q] = 0.0;
      for (int t = s + lane; t < e; t += 32) {
        const int i = perm[t];
        for (int k = rowptr[i]; k < rowptr[i + 1]; ++k) {
          const int q = agg[col[k]];
          if (q >= 0) {
            const int rk = pre[q >> 5] + __popc(bm[q >> 5] & ((1u << (q & 31)) - 1u));
            priv[lane * (kTLocal + 1) + rk] += val[k];
          }
        }
      }
      __syncwarp();
      for (int q = lane; q < r; q += 32)
        if (!(bm[q >> 5] & (1u << (q & 31)))) T[(size_t)p * r + q] = 0.0;
      for (int lq = lane; lq < nq; lq += 32) {
        double acc = 0.0;
        for (int l = 0; l < 32; ++l) acc += priv[l * (kTLocal + 1) + lq];
        const int q = qlist[lq];
        T[(size_t)p * r + q] = acc * uscale[p] * uscale[q];
      }
      return;
    }
    // many aggregates met: lane 0 accumulates sequentially, the warp loads each row's entries
    for (int t = s; t < e; ++t) {
      const int i = perm[t];
      const int ks = rowptr[i], ke = rowptr[i + 1];
      for (int k0 = ks; k0 < ke; k0 += 32) {
        const int k = k0 + lane;
        int q = -1;
        double v = 0.0;
        if (k < ke) {
          q = agg[col[k]];
          v = val[k];
        }
        const int cntk = min(32, ke - k0);
        for (int l = 0; l < cntk; ++l) {
          const int ql = __shfl_sync(0xffffffffu, q, l);
          const double vl = __shfl_sync(0xffffffffu, v, l);
          if (lane == 0 && ql >= 0) srow[ql] += vl;
        }
      }
    }
    __syncwarp();
    for (int q = lane; q < r; q += 32) T[(size_t)p * r + q] = srow[q] * uscale[p] * uscale[q];
  }
}

// ---- T^-1 by Gauss-Jordan elimination with partial pivoting on G = [T | I] (r x 2r,
// row-major), without row exchanges: the pivot of step k is the row p_k, among the rows
// not yet used as pivots, with the largest |G_ik| (the lowest index on ties).  Row p_k is
// normalised lazily (its factor 1/G_{p_k k} is kept as a pending row scale and applied
// when the row is next updated), and its identity entry is placed in right-hand column
// r + k when the row becomes the pivot, so the right-hand columns in use at step k are
// exactly [r, r + k] and every step updates r entries per row.  With P the pivot
// permutation (P e_k = e_{p_k}) the right half ends as P T^-1 P, from which T^-1 is read
// back.  Each step is one kernel; every block reduces the previous step's per-block
// pivot candidates itself (deterministic: fixed tie rule, fixed update order).
constexpr int kGjMaxBlocks = 1024;  // blocks of a Gauss-Jordan step

struct GjAux {
  double* pinv;     // r: 1 / pivot of step k
  double* pscale;   // r: pending row scale (1 unless the row was the last pivot)
  double* cval;     // per-block pivot candidates, two buffers (by step parity)
  int* piv;         // r: pivot row of step k
  int* slot;        // r: step at which row i was the pivot
  int* used;        // r: row i has been a pivot
  int* cidx;
  int* err;
};

__global__ void k_gj_init(int r, const double* __restrict__ T, double* __restrict__ G,
                          GjAux x) {
  const long long tot = 2LL * r * r;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < tot;
       t += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(t / (2 * r)), j = (int)(t % (2 * r));
    G[t] = j < r ? T[(size_t)i * r + j] : 0.0;
  }
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < r; i += gridDim.x * blockDim.x) {
    x.pscale[i] = 1.0;
    x.used[i] = 0;
  }
}

// (value, index) argmax: larger value, then lower index
__device__ __forceinline__ void argmax_merge(double& v, int& i, double ov, int oi) {
  if (ov > v || (ov == v && oi < i)) {
    v = ov;
    i = oi;
  }
}

// block-wide argmax; the result is valid in thread 0
__device__ void block_argmax(double& v, int& i) {
  __shared__ double sv[32];
  __shared__ int si[32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const double ov = __shfl_xor_sync(0xffffffffu, v, o);
    const int oi = __shfl_xor_sync(0xffffffffu, i, o);
    argmax_merge(v, i, ov, oi);
  }
  __syncthreads();
  if (lane == 0) {
    sv[warp] = v;
    si[warp] = i;
  }
  __syncthreads();
  if (warp == 0) {
    v = lane < nw ? sv[lane] : -1.0;
    i = lane < nw ? si[lane] : 0x7fffffff;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const double ov = __shfl_xor_sync(0xffffffffu, v, o);
      const int oi = __shfl_xor_sync(0xffffffffu, i, o);
      argmax_merge(v, i, ov, oi);
    }
  }
}

// pivot of column 0: per-block candidate slots of the "previous step" (buffer 1), with
// the column's argmax in slot 0 and no candidate elsewhere (one block)
__global__ void k_gj_first(int r, const double* __restrict__ G, GjAux x, int nslots) {
  double v = -1.0;
  int i = 0x7fffffff;
  for (int t = threadIdx.x; t < r; t += blockDim.x)
    argmax_merge(v, i, fabs(G[(size_t)t * 2 * r]), t);
  block_argmax(v, i);
  double* cv = x.cval + kGjMaxBlocks;
  int* ci = x.cidx + kGjMaxBlocks;
  for (int b = threadIdx.x; b < nslots; b += blockDim.x) {
    cv[b] = -1.0;
    ci[b] = 0x7fffffff;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    cv[0] = v;
    ci[0] = i;
  }
}

// Step k.  Every block first reduces the previous step's per-block candidates to the
// pivot row p_k (the same result in every block, so no block waits on another) and
// forms 1/G_{p_k k}; block 0 records the pivot and the block owning row p_k places its
// identity entry.  Then every row i != p_k gets
//   row_i <- s_i row_i - (s_i G_ik / G_{p_k k}) row_{p_k}   (s_i its pending scale)
// over the active columns [k+1, r) and [r, r + k], a warp per row, and the rows not yet
// used propose |G_{i,k+1}| for the next step (candidate buffers alternate by step).
constexpr int kGjRowsPerBlock = 8;  // warps of a step block

__global__ void __launch_bounds__(32 * kGjRowsPerBlock)
    k_gj_step(int r, int k, double* __restrict__ G, GjAux x) {
  extern __shared__ double sprow[];  // active part of the pivot row: r entries
  __shared__ int s_p;
  __shared__ double s_ip;
  const int ld = 2 * r;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  {
    const double* cv = x.cval + (size_t)((k + 1) & 1) * kGjMaxBlocks;
    const int* ci = x.cidx + (size_t)((k + 1) & 1) * kGjMaxBlocks;
    double v = -1.0;
    int i = 0x7fffffff;
    for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x) argmax_merge(v, i, cv[b], ci[b]);
    block_argmax(v, i);
    if (threadIdx.x == 0) {
      if (!(v > 0.0) || i >= r) {  // singular: record it, keep the bookkeeping consistent
        if (blockIdx.x == 0) atomicOr(x.err, 8);
        i = 0;
        while (i < r && x.used[i]) ++i;
        if (i >= r) i = 0;
      }
      const double pv = G[(size_t)i * ld + k];
      s_p = i;
      s_ip = pv != 0.0 ? 1.0 / pv : 0.0;
    }
    __syncthreads();
  }
  const int p = s_p;
  const double ip = s_ip;
  const int nl = r - k - 1;  // active left columns k+1 .. r-1, then right columns r .. r+k
  const double* prow = G + (size_t)p * ld;
  for (int c = threadIdx.x; c < r; c += blockDim.x)
    sprow[c] = c < nl ? prow[k + 1 + c] : (c - nl == k ? 1.0 : prow[r + (c - nl)]);
  if (threadIdx.x == 0) {
    if (blockIdx.x == 0) {
      x.piv[k] = p;
      x.pinv[k] = ip;
      x.pscale[p] = ip;  // row p_k is normalised when it is next updated
      x.slot[p] = k;
      x.used[p] = 1;
    }
    if ((p / kGjRowsPerBlock) % (int)gridDim.x == (int)blockIdx.x) G[(size_t)p * ld + r + k] = 1.0;
  }
  __syncthreads();
  double bv = -1.0;
  int bi = 0x7fffffff;
  for (int i = blockIdx.x * kGjRowsPerBlock + warp; i < r; i += gridDim.x * kGjRowsPerBlock) {
    if (i == p) continue;
    double* row = G + (size_t)i * ld;
    const double ps = x.pscale[i];
    const double f = ps * row[k] * ip;
    const bool cand = k + 1 < r && !x.used[i];
    for (int c0 = 0; c0 < r; c0 += 32 * 16) {
      double v[16];
#pragma unroll
      for (int u = 0; u < 16; ++u) {
        const int c = c0 + lane + 32 * u;
        v[u] = c < r ? (c < nl ? row[k + 1 + c] : row[r + (c - nl)]) : 0.0;
      }
      if (ps != 1.0) {  // the previous pivot row: apply its pending scale (warp-uniform)
#pragma unroll
        for (int u = 0; u < 16; ++u) v[u] *= ps;
      }
#pragma unroll
      for (int u = 0; u < 16; ++u) {
        const int c = c0 + lane + 32 * u;
        if (c < r) {
          const double nv = fma(-f, sprow[c], v[u]);
          if (c < nl) row[k + 1 + c] = nv;
          else row[r + (c - nl)] = nv;
          if (c == 0 && cand) argmax_merge(bv, bi, fabs(nv), i);
        }
      }
    }
    if (ps != 1.0) {
      __syncwarp();  // every lane has read pscale[i] before it is reset
      if (lane == 0) x.pscale[i] = 1.0;
    }
  }
  block_argmax(bv, bi);
  if (threadIdx.x == 0) {
    x.cval[(size_t)(k & 1) * kGjMaxBlocks + blockIdx.x] = bv;
    x.cidx[(size_t)(k & 1) * kGjMaxBlocks + blockIdx.x] = bi;
  }
}

// ---------------------------------------------------------------------------------------
// The same Gauss-Jordan elimination in one cooperative kernel (r small enough that every
// block keeps its rows of [T | slots] in shared memory): block b owns the rows b, b + G, ...
// and each step costs one grid barrier instead of one launch.  At the end of step k - 1
// every block proposes its largest |G_{i,k}| over its unused rows and copies that row's
// active part (left columns k .. r-1, then slots 0 .. k-1) into its candidate slot; after
// the barrier every block picks the same pivot (largest value, then lowest row) from the G
// proposals, reads the winning row, normalises it (its identity entry goes to slot k) and
// eliminates column k from its own rows, exactly r entries per row.
// ---------------------------------------------------------------------------------------
constexpr int kGjPThreads = 512;
constexpr long long kGjSpins = 1LL << 21;  // polls of the barrier word: about a second

struct GjP {
  // candidates of step k in buffer k & 1 (the step-(k+1) proposals of a block that has
  // finished step k must not overwrite what a slower block still reads for step k)
  double* cval;    // 2 x kGjMaxBlocks candidate values
  int* cidx;       // 2 x kGjMaxBlocks candidate rows
  double* crow;    // 2 x G x r candidate rows (active parts)
  int* piv;        // r: pivot row of step k
  int* slot;       // r: step at which row i was the pivot
  unsigned* bar;   // 2 words: arrivals, generation
  int* err;
};

__device__ __forceinline__ bool gj_grid_sync(unsigned* bar, unsigned& gen) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    int ok = 1;
    __threadfence();
    if (atomicAdd(&bar[0], 1u) == gridDim.x - 1) {
      atomicExch(&bar[0], 0u);
      __threadfence();
      atomicExch(&bar[1], gen + 1u);
    } else {
      long long spins = 0;
      while (*(volatile unsigned*)&bar[1] == gen)
        if (++spins > kGjSpins) {
          ok = 0;
          break;
        }
    }
    __threadfence();
    s_ok = ok;
  }
  __syncthreads();
  ++gen;
  return s_ok != 0;
}

__global__ void __launch_bounds__(kGjPThreads, 1)
    k_gj_persistent(int r, const double* __restrict__ T, GjP x, double* __restrict__ Tinv,
                    double* __restrict__ TinvT) {
  extern __shared__ double gsm[];
  __shared__ int s_used[64];
  __shared__ int s_p, s_src;
  __shared__ double s_ip;
  const int G = gridDim.x, b = blockIdx.x, t = threadIdx.x;
  const int nq = (r - b + G - 1) / G;  // rows b, b + G, ... of this block
  double* rows = gsm;                  // nq x 2r: left columns [0, r), slots [r, 2r)
  double* prow = gsm + (size_t)nq * 2 * r;
  unsigned gen = *(volatile unsigned*)&x.bar[1];
  for (int q = t; q < nq; q += blockDim.x) s_used[q] = 0;
  for (long long e = t; e < (long long)nq * 2 * r; e += blockDim.x) {
    const int q = (int)(e / (2 * r)), c = (int)(e % (2 * r));
    rows[e] = c < r ? T[(size_t)(b + q * G) * r + c] : 0.0;
  }
  __syncthreads();
  // proposal for step k: largest |left[k]| over the unused rows, and that row's active part
  auto propose = [&](int k) {
    if (t < 32) {
      double v = -1.0;
      int i = 0x7fffffff;
      for (int q = t; q < nq; q += 32)
        if (!s_used[q]) argmax_merge(v, i, fabs(rows[(size_t)q * 2 * r + k]), b + q * G);
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        const double ov = __shfl_xor_sync(0xffffffffu, v, o);
        const int oi = __shfl_xor_sync(0xffffffffu, i, o);
        argmax_merge(v, i, ov, oi);
      }
      if (t == 0) {
        x.cval[(size_t)(k & 1) * kGjMaxBlocks + b] = v;
        x.cidx[(size_t)(k & 1) * kGjMaxBlocks + b] = i;
        s_p = i;
      }
    }
    __syncthreads();
    const int i = s_p;
    if (i < r) {
      const double* row = rows + (size_t)((i - b) / G) * 2 * r;
      double* dst = x.crow + ((size_t)(k & 1) * G + b) * r;
      for (int c = t; c < r; c += blockDim.x)
        dst[c] = c < r - k ? row[k + c] : row[r + (c - (r - k))];
    }
  };
  propose(0);
  for (int k = 0; k < r; ++k) {
    if (!gj_grid_sync(x.bar, gen)) {
      if (t == 0) atomicOr(x.err, 16);
      return;
    }
    if (t < 32) {  // the pivot: largest candidate, then lowest row (the same in every block)
      double v = -1.0;
      int i = 0x7fffffff, src = 0;
      const double* cv = x.cval + (size_t)(k & 1) * kGjMaxBlocks;
      const int* ci = x.cidx + (size_t)(k & 1) * kGjMaxBlocks;
      for (int q = t; q < G; q += 32) {
        const double ov = __ldcg(cv + q);
        const int oi = __ldcg(ci + q);
        if (ov > v || (ov == v && oi < i)) {
          v = ov;
          i = oi;
          src = q;
        }
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        const double ov = __shfl_xor_sync(0xffffffffu, v, o);
        const int oi = __shfl_xor_sync(0xffffffffu, i, o);
        const int os = __shfl_xor_sync(0xffffffffu, src, o);
        if (ov > v || (ov == v && oi < i)) {
          v = ov;
          i = oi;
          src = os;
        }
      }
      if (t == 0) {
        if (!(v > 0.0) || i >= r) {  // singular: record it and stop
          if (b == 0) atomicOr(x.err, 8);
          s_p = -1;
        } else {
          s_p = i;
          s_ip = 1.0 / __ldcg(x.crow + ((size_t)(k & 1) * G + src) * r);
          if (b == 0) {
            x.piv[k] = i;
            x.slot[i] = k;
          }
        }
      }
      if (t == 0) s_src = src;
    }
    __syncthreads();
    const int p = s_p;
    if (p < 0) return;
    const double ip = s_ip;
    const double* crow = x.crow + ((size_t)(k & 1) * G + s_src) * r;
    // the normalised pivot row: left columns k+1 .. r-1 at prow[0 ..), slots 0 .. k at
    // prow[r - k - 1 ..] (slot k: the identity entry 1 / pivot)
    const int nl = r - k - 1;
    for (int c = t; c < r; c += blockDim.x)
      prow[c] = c < nl ? __ldcg(crow + 1 + c) * ip : (c - nl < k ? __ldcg(crow + 1 + c) * ip : ip);
    __syncthreads();
    // eliminate column k from every own row but the pivot; the pivot row becomes prow
    for (int q = 0; q < nq; ++q) {
      double* row = rows + (size_t)q * 2 * r;
      const bool piv = b + q * G == p;
      const double f = row[k];
      for (int c = t; c < r; c += blockDim.x) {
        double* dst = c < nl ? row + k + 1 + c : row + r + (c - nl);
        *dst = piv ? prow[c] : fma(-f, prow[c], *dst);
      }
      if (piv && t == 0) s_used[q] = 1;
    }
    __syncthreads();
    if (k + 1 < r) propose(k + 1);
  }
  if (!gj_grid_sync(x.bar, gen)) {
    if (t == 0) atomicOr(x.err, 16);
    return;
  }
  // own rows: row p = piv[k] holds row k of T^-1 with column j at slot(j)
  for (long long e = t; e < (long long)nq * r; e += blockDim.x) {
    const int q = (int)(e / r), j = (int)(e % r);
    const int i = b + q * G;
    const int k = __ldcg(x.slot + i);
    const double v = rows[(size_t)q * 2 * r + r + __ldcg(x.slot + j)];
    Tinv[(size_t)k * r + j] = v;
    if (TinvT) TinvT[(size_t)j * r + k] = v;
  }
}

// T^-1[a][c] = s(p_a) G[p_a][r + slot(c)]  (and its transpose)
__global__ void k_gj_extract(int r, const double* __restrict__ G, GjAux x,
                             double* __restrict__ Tinv, double* __restrict__ TinvT) {
  const long long tot = (long long)r * r;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < tot;
       t += (long long)gridDim.x * blockDim.x) {
    const int a = (int)(t / r), c = (int)(t % r);
    const int pa = x.piv[a];
    const double v = x.pscale[pa] * G[(size_t)pa * 2 * r + r + x.slot[c]];
    Tinv[t] = v;
    if (TinvT) TinvT[(size_t)c * r + a] = v;
  }
}

__global__ void k_norm_inf(int n, const int* __restrict__ rowptr, const double* __restrict__ val,
                           unsigned long long* __restrict__ out) {
  double best = 0.0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int k = rowptr[i]; k < rowptr[i + 1]; ++k) s += fabs(val[k]);
    best = fmax(best, s);
  }
  best = warp_max(best);
  // non-negative doubles order like their bit patterns: the max is order-independent
  if ((threadIdx.x & 31) == 0) atomicMax(out, (unsigned long long)__double_as_longlong(best));
}

__global__ void k_to_float(long long n, const double* __restrict__ a, float* __restrict__ b) {
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n;
       t += (long long)gridDim.x * blockDim.x)
    b[t] = (float)a[t];
}

// ---- coarse rows AU: per row i and aggregate a met in row i, (AU W^-1)_ia = sum of a_ik
// over the row's entries whose column lies in aggregate a (unscaled, U = W diag(uscale)).
// Entries of a row are kept in order of first occurrence; each sum runs in CSR order.
__device__ __forceinline__ bool first_of_agg(const int* __restrict__ col,
                                             const int* __restrict__ agg, int s, int k, int a) {
  for (int q = s; q < k; ++q)
    if (agg[col[q]] == a) return false;
  return true;
}

__global__ void k_au_count(int n, const int* __restrict__ rowptr, const int* __restrict__ col,
                           const int* __restrict__ agg, int* __restrict__ cnt) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const int s = rowptr[i], e = rowptr[i + 1];
    int c = 0;
    for (int k = s; k < e; ++k) {
      const int a = agg[col[k]];
      if (a >= 0 && first_of_agg(col, agg, s, k, a)) ++c;
    }
    cnt[i] = c;
  }
}

// exclusive scan of cnt[0, n) into out[0, n], out[n] = total; 1024 entries per block
constexpr int kScanBlock = 1024;

__device__ __forceinline__ int block_excl_scan(int v, int* sw /* 32 */, int* total) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) sw[warp] = x;
  __syncthreads();
  if (warp == 0) {
    int t = lane < (int)(blockDim.x >> 5) ? sw[lane] : 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, t, o);
      if (lane >= o) t += y;
    }
    sw[lane] = t;
  }
  __syncthreads();
  const int before = warp > 0 ? sw[warp - 1] : 0;
  *total = sw[31];
  __syncthreads();
  return before + x - v;
}

__global__ void __launch_bounds__(kScanBlock)
    k_scan_sums(int n, const int* __restrict__ cnt, int* __restrict__ bsum) {
  __shared__ int sw[32];
  const int i = blockIdx.x * kScanBlock + threadIdx.x;
  int tot;
  block_excl_scan(i < n ? cnt[i] : 0, sw, &tot);
  if (threadIdx.x == 0) bsum[blockIdx.x] = tot;
}

// one block: bsum[0, nb) -> exclusive offsets, bsum[nb] = total
__global__ void __launch_bounds__(kScanBlock) k_scan_top(int nb, int* __restrict__ bsum) {
  __shared__ int sw[32];
  __shared__ int carry;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  for (int b0 = 0; b0 < nb; b0 += kScanBlock) {
    const int b = b0 + threadIdx.x;
    const int v = b < nb ? bsum[b] : 0;
    int tot;
    const int ex = block_excl_scan(v, sw, &tot);
    if (b < nb) bsum[b] = carry + ex;
    __syncthreads();
    if (threadIdx.x == 0) carry += tot;
    __syncthreads();
  }
  if (threadIdx.x == 0) bsum[nb] = carry;
}

__global__ void __launch_bounds__(kScanBlock)
    k_scan_apply(int n, int nb, const int* __restrict__ cnt, const int* __restrict__ bsum,
                 int* __restrict__ out) {
  __shared__ int sw[32];
  const int i = blockIdx.x * kScanBlock + threadIdx.x;
  int tot;
  const int ex = block_excl_scan(i < n ? cnt[i] : 0, sw, &tot);
  if (i < n) out[i] = bsum[blockIdx.x] + ex;
  if (blockIdx.x == 0 && threadIdx.x == 0) out[n] = bsum[nb];
}

__global__ void k_au_fill(int n, const int* __restrict__ rowptr, const int* __restrict__ col,
                          const double* __restrict__ val, const int* __restrict__ agg,
                          const int* __restrict__ aurp, int* __restrict__ aucol,
                          double* __restrict__ auval, float* __restrict__ auval32) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const int s = rowptr[i], e = rowptr[i + 1];
    int q = aurp[i];
    for (int k = s; k < e; ++k) {
      const int a = agg[col[k]];
      if (a < 0 || !first_of_agg(col, agg, s, k, a)) continue;
      double sum = 0.0;
      for (int k2 = k; k2 < e; ++k2)
        if (agg[col[k2]] == a) sum += val[k2];
      aucol[q] = a;
      auval[q] = sum;
      if (auval32) auval32[q] = (float)sum;
      ++q;
    }
  }
}

// ---- extended rows [A | A W] for the deflated SpMV: row i holds A's entries, then its
// A W entries with column index n + a (a = aggregate) ----
__global__ void k_ext_rows(int n, const int* __restrict__ rowptr, const int* __restrict__ aurp,
                           int* __restrict__ xrp) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i <= n; i += gridDim.x * blockDim.x)
    xrp[i] = rowptr[i] + aurp[i];
}

__global__ void k_ext_fill(int n, const int* __restrict__ rowptr, const int* __restrict__ col,
                           const double* __restrict__ val, const float* __restrict__ val32,
                           const int* __restrict__ aurp, const int* __restrict__ aucol,
                           const double* __restrict__ auval, const float* __restrict__ auval32,
                           const int* __restrict__ xrp, int* __restrict__ xcol,
                           double* __restrict__ xval, float* __restrict__ xval32) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    int q = xrp[i];
    for (int k = rowptr[i]; k < rowptr[i + 1]; ++k, ++q) {
      xcol[q] = col[k];
      xval[q] = val[k];
      if (xval32) xval32[q] = val32[k];
    }
    for (int k = aurp[i]; k < aurp[i + 1]; ++k, ++q) {
      xcol[q] = n + aucol[k];
      xval[q] = auval[k];
      if (xval32) xval32[q] = auval32[k];
    }
  }
}

// ---- diagonal storage: the distinct offsets col - row of A (a lock-free insert into a
// 64-slot open-addressing table; more than kMaxDiag distinct offsets sets the overflow
// count), then dval[d * ldd + i] = a_{i, i + off_d} (0 where the entry is absent) ----
constexpr int kDiagSlots = 64;
constexpr int kDiagEmpty = (int)0x80000000;

__global__ void k_dia_detect(int n, const int* __restrict__ rowptr, const int* __restrict__ col,
                             int* __restrict__ slots, int* __restrict__ count) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    for (int k = rowptr[i]; k < rowptr[i + 1]; ++k) {
      const int off = col[k] - i;
      int h = (int)(((unsigned)off * 2654435761u) >> 26);  // 6 bits
      for (int probe = 0; probe < kDiagSlots; ++probe, h = (h + 1) & (kDiagSlots - 1)) {
        const int cur = *(volatile int*)(slots + h);
        if (cur == off) break;
        if (cur == kDiagEmpty) {
          const int prev = atomicCAS(slots + h, kDiagEmpty, off);
          if (prev == kDiagEmpty) {
            atomicAdd(count, 1);
            break;
          }
          if (prev == off) break;
        }
      }
      if (*(volatile int*)count > kMaxDiag) return;  // too many: no diagonal storage
    }
  }
}

__global__ void k_dia_fill(int n, const int* __restrict__ rowptr, const int* __restrict__ col,
                           const double* __restrict__ val, DiaOffsets offs, long long ldd,
                           double* __restrict__ dval, float* __restrict__ dval32) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    for (int k = rowptr[i]; k < rowptr[i + 1]; ++k) {
      const int off = col[k] - i;
      int d = 0;
      while (d < offs.nd && offs.off[d] != off) ++d;
      if (d == offs.nd) continue;  // cannot happen after a complete detection
      dval[d * ldd + i] = val[k];
      if (dval32) dval32[d * ldd + i] = (float)val[k];
    }
  }
}

}  // namespace

cudaError_t launch_validate(int n, long long nnz, const int* rowptr, const int* col,
                            const int* agg, int r, int* err, cudaStream_t st) {
  k_validate<<<grid_for(n, 256, 152 * 8), 256, 0, st>>>(n, nnz, rowptr, col, agg, r, err);
  return cudaGetLastError();
}

int agg_chunks(int n) { return (n + kChunk - 1) / kChunk; }

cudaError_t launch_agg_perm(int n, int r, const int* agg, int* counts /* chunks*r */,
                            int* aggptr /* r+1 */, int* cnt /* r */, int* perm,
                            int* agg_piece /* r+1 */, int* piece_start, double* uscale,
                            int units, int grid, int* bcnt /* grid */,
                            int* blk_piece_start /* grid+1 */, int* blk_piece, int* err,
                            cudaStream_t st) {
  const int nb = agg_chunks(n);
  const size_t sm = sizeof(int) * (size_t)r;
  k_agg_count<<<nb, 256, sm, st>>>(n, r, agg, counts);
  k_agg_scan<<<1, 1024, 0, st>>>(r, nb, counts, aggptr, cnt);
  k_agg_scatter<<<nb, 32, sm, st>>>(n, r, agg, counts, perm);
  k_pieces<<<1, 1024, 0, st>>>(r, units, grid, perm, aggptr, cnt, agg_piece, piece_start, uscale,
                               err);
  if (grid > 0) {
    k_blk_count<<<grid, 256, 0, st>>>(units, perm, piece_start, agg_piece, r, bcnt);
    k_blk_fill<<<grid, 256, 0, st>>>(units, perm, piece_start, agg_piece, r, bcnt,
                                     blk_piece_start, blk_piece);
  }
  return cudaGetLastError();
}

cudaError_t launch_coarse_T(int r, const int* rowptr, const int* col, const double* val,
                            const int* agg, const int* perm, const int* aggptr,
                            const double* uscale, double* T, cudaStream_t st) {
  const bool lane_rows = (r * 32 * (int)sizeof(double)) <= 48 * 1024;
  // large r: the sequential row, the bitmap and its prefix, the list, the private sums
  const size_t sm = lane_rows ? sizeof(double) * (size_t)r * 32
                              : sizeof(double) * (size_t)r + 2 * sizeof(int) * ((r + 31) / 32) +
                                    sizeof(int) * (kTLocal + (kTLocal & 1)) +
                                    sizeof(double) * 32 * (kTLocal + 1);
  if (sm > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(k_T_rows, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)sm);
    if (e != cudaSuccess) return e;
  }
  k_T_rows<<<r, 32, sm, st>>>(r, rowptr, col, val, agg, perm, aggptr, uscale, T);
  return cudaGetLastError();
}

size_t gj_aux_bytes(int r) {
  return sizeof(double) * (2 * (size_t)r + 2 * kGjMaxBlocks) +
         sizeof(int) * (3 * (size_t)r + 2 * kGjMaxBlocks) + 4 * sizeof(unsigned);
}

namespace {
// shared memory of the cooperative Gauss-Jordan kernel on `grid` blocks
size_t gj_persistent_smem(int r, int grid) {
  const size_t nq = ((size_t)r + grid - 1) / grid;
  return sizeof(double) * (nq * 2 * (size_t)r + (size_t)r);
}
}  // namespace

// ---- T^-1 of a banded T (kl sub-, ku super-diagonals, small against r): band LU with
// partial pivoting (row interchanges within the kl rows below the diagonal), then the r
// columns of T^-1 by forward and back substitution.  The aggregates of a structured
// partition couple only with their neighbours (a 32 x 32 grid of aggregates under a
// 9-point operator: kl = ku = 33), so the factorisation costs r (kl + ku) kl FMA instead
// of the r^3 of Gauss-Jordan.
__global__ void k_band_width(int r, const double* __restrict__ T, int* __restrict__ bw) {
  int lo = 0, up = 0;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < (long long)r * r;
       e += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(e / r), j = (int)(e % r);
    if (T[e] != 0.0) {
      lo = max(lo, i - j);
      up = max(up, j - i);
    }
  }
  for (int o = 16; o > 0; o >>= 1) {
    lo = max(lo, __shfl_xor_sync(0xffffffffu, lo, o));
    up = max(up, __shfl_xor_sync(0xffffffffu, up, o));
  }
  if ((threadIdx.x & 31) == 0) {
    atomicMax(&bw[0], lo);
    atomicMax(&bw[1], up);
  }
}

// One block.  The active window (rows k .. k + kl, columns k .. k + kl + ku) lives in shared
// memory, entry (i, j) at win[(i mod R) C + (j mod C)] with R = kl + 1, C = kl + ku + 1 (the
// upper band widens by kl under interchanges).  Step k: pivot = the largest |a_ik| over the
// window's rows (lowest row on ties), swap, multipliers, rank-1 update of the window; row k
// (of U) and column k (of L) leave for global memory, and row k + R enters from T.
// Outputs: U row k at Ub[k C .. k C + C) (U_{k,k+t}), 1 / U_kk at dinv[k], the multipliers
// of step k at Lm[k kl .. k kl + kl), the pivot row at piv[k].
// A block on one multiprocessor issues FP64 at 2 lanes per clock, so the scalar steps stay
// off that pipe where they can: the pivot is chosen by the magnitudes' bit patterns (for
// finite doubles |a| < |b| exactly when the bits of |a| are below those of |b|, as
// unsigned integers), the multipliers take one multiply by 1 / U_kk, and the row entering
// the window is loaded a step ahead.
constexpr int kBandThreads = 256;

__global__ void __launch_bounds__(kBandThreads, 1)
    k_band_lu(int r, int kl, int ku, const double* __restrict__ T, double* __restrict__ Ub,
              double* __restrict__ dinv, double* __restrict__ Lm, int* __restrict__ piv,
              int* __restrict__ err) {
  extern __shared__ double win[];
  __shared__ int s_p;
  __shared__ int s_sing;
  __shared__ double s_rp;
  const int R = kl + 1, C = kl + ku + 1;
  const int t = threadIdx.x, lane = t & 31;
  // the update's 2-D split: 64 columns x 4 row groups
  const int tx = t & 63, ty = t >> 6;
  for (int e = t; e < R * C; e += kBandThreads) {
    const int i = e / C, j = e % C;
    win[e] = (i < r && j < r) ? T[(size_t)i * r + j] : 0.0;
  }
  // thread q < C holds entry (k + R, k + 1 + q) of T, the row that enters after step k
  double nxt = 0.0;
  auto fetch_row = [&](int k) {
    const int nrow = k + R, j = k + 1 + t;
    nxt = (t < C && nrow < r && j < r) ? __ldg(T + (size_t)nrow * r + j) : 0.0;
  };
  fetch_row(0);
  __syncthreads();
  constexpr unsigned long long kMag = 0x7fffffffffffffffULL, kInf = 0x7ff0000000000000ULL;
  int kr = 0, kc = 0;  // window slots of row k and column k (k mod R, k mod C)
  for (int k = 0; k < r; ++k) {
    const int nr = min(kl, r - 1 - k), nc = min(kl + ku, r - 1 - k);  // rows, columns past k
    // slot of row k + di (0 <= di <= R - 1) and column k + dj (0 <= dj <= C)
    auto rs = [&](int di) { const int v = kr + di; return v >= R ? v - R : v; };
    auto cs = [&](int dj) { const int v = kc + dj; return v >= C ? v - C : v; };
    if (t < 32) {
      unsigned long long key = 0;
      int idx = 0x7fffffff;
      for (int di = lane; di <= nr; di += 32) {
        const unsigned long long m =
            (unsigned long long)__double_as_longlong(win[rs(di) * C + kc]) & kMag;
        if (m > key || (m == key && k + di < idx)) {
          key = m;
          idx = k + di;
        }
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long ok = __shfl_xor_sync(0xffffffffu, key, o);
        const int oi = __shfl_xor_sync(0xffffffffu, idx, o);
        if (ok > key || (ok == key && oi < idx)) {
          key = ok;
          idx = oi;
        }
      }
      if (lane == 0) {
        const bool good = key > 0 && key < kInf;  // nonzero and finite
        s_p = idx;
        s_sing = !good;
        if (good) s_rp = 1.0 / win[rs(idx - k) * C + kc];
      }
    }
    __syncthreads();
    if (s_sing) {
      if (t == 0) atomicOr(err, 8);
      return;
    }
    const int p = s_p;
    const double rp = s_rp;
    if (p != k) {
      double* r0 = win + rs(0) * C;
      double* r1 = win + rs(p - k) * C;
      for (int dj = t; dj <= nc; dj += kBandThreads) {
        const int c = cs(dj);
        const double a = r0[c];
        r0[c] = r1[c];
        r1[c] = a;
      }
    }
    __syncthreads();
    for (int di = 1 + t; di <= nr; di += kBandThreads) {
      double* e = win + rs(di) * C + kc;
      const double l = *e * rp;
      *e = l;
      Lm[(size_t)k * kl + (di - 1)] = l;
    }
    for (int q = t; q < C; q += kBandThreads) Ub[(size_t)k * C + q] = q <= nc ? win[rs(0) * C + cs(q)] : 0.0;
    if (t == 0) {
      piv[k] = p;
      dinv[k] = rp;
    }
    __syncthreads();
    {
      // a_ij -= l_i u_kj over rows k + 1 .. k + nr, columns k + 1 .. k + nc
      const double* urow = win + rs(0) * C;
      double u0 = 0.0, u1 = 0.0;
      int c0 = 0, c1 = 0;
      const bool h0 = 1 + tx <= nc, h1 = 65 + tx <= nc;
      if (h0) { c0 = cs(1 + tx); u0 = urow[c0]; }
      if (h1) { c1 = cs(65 + tx); u1 = urow[c1]; }
      for (int di = 1 + ty; di <= nr; di += kBandThreads / 64) {
        double* row = win + rs(di) * C;
        const double l = row[kc];
        if (h0) row[c0] = fma(-l, u0, row[c0]);
        if (h1) row[c1] = fma(-l, u1, row[c1]);
      }
    }
    __syncthreads();
    // row k's slot takes row k + R (its entries lie in columns k + 1 .. k + C), column k's
    // slot takes column k + C (zero in the rows already in the window)
    if (t < C) win[rs(0) * C + cs(1 + t)] = nxt;
    fetch_row(k + 1);
    for (int di = 1 + t; di <= kl; di += kBandThreads) win[rs(di) * C + kc] = 0.0;
    __syncthreads();
    kr = kr + 1 == R ? 0 : kr + 1;
    kc = kc + 1 == C ? 0 : kc + 1;
  }
}

// Column j of T^-1 (one warp): x = e_j; forward, for k = 0 .. r - 2: swap x_k and x_piv[k],
// x_{k+1..k+kl} -= l_k x_k (k starts at j - kl: x stays 0 above); back, for i = r - 1 .. 0:
// x_i = x_i / U_ii, x_{i-t} -= U_{i-t,i} x_i.  The factors of the next kBandAhead steps are
// loaded ahead of the substitution chain.  Writes column j of T^-1 and row j of T^-T.
constexpr int kBandAhead = 8;
constexpr int kBandWarps = 4;

__global__ void __launch_bounds__(32 * kBandWarps)
    k_band_inv(int r, int kl, int ku, const double* __restrict__ Ub,
               const double* __restrict__ dinv, const double* __restrict__ Lm,
               const int* __restrict__ piv, double* __restrict__ Tinv,
               double* __restrict__ TinvT) {
  extern __shared__ double xs[];
  const int C = kl + ku + 1;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int j = blockIdx.x * kBandWarps + warp;
  if (j >= r) return;
  double* x = xs + (size_t)warp * r;
  for (int i = lane; i < r; i += 32) x[i] = i == j ? 1.0 : 0.0;
  __syncwarp();
  constexpr int D = kBandAhead;
  // forward: each lane takes the multipliers t = lane, lane + 32 (kl <= 64)
  {
    const int k0 = j - kl > 0 ? j - kl : 0;
    double la[D], lb[D];
    int pv[D];
    auto fetch = [&](int k, int d) {
      const bool ok = k < r - 1;
      pv[d] = ok ? __ldg(piv + k) : k;
      la[d] = ok && lane < kl ? __ldg(Lm + (size_t)k * kl + lane) : 0.0;
      lb[d] = ok && lane + 32 < kl ? __ldg(Lm + (size_t)k * kl + lane + 32) : 0.0;
    };
#pragma unroll
    for (int d = 0; d < D; ++d) fetch(k0 + d, d);
    for (int k = k0; k < r - 1; k += D) {
#pragma unroll
      for (int d = 0; d < D; ++d) {
        const int kk = k + d;
        if (kk < r - 1) {
          const int p = pv[d];
          if (p != kk) {
            const double a = x[kk], b = x[p];
            __syncwarp();
            if (lane == 0) {
              x[kk] = b;
              x[p] = a;
            }
            __syncwarp();
          }
          const double xk = x[kk];
          if (lane < kl && kk + 1 + lane < r) x[kk + 1 + lane] = fma(-la[d], xk, x[kk + 1 + lane]);
          if (lane + 32 < kl && kk + 33 + lane < r)
            x[kk + 33 + lane] = fma(-lb[d], xk, x[kk + 33 + lane]);
          __syncwarp();
          fetch(kk + D, d);
        }
      }
    }
  }
  // back: column i of U above the diagonal, U_{i-t,i} = Ub[(i - t) C + t], t = 1 .. C - 1:
  // lane takes t = 1 + lane + 32 s, s < 3 (C <= 97)
  {
    double u[D][3], dv[D];
    auto fetch = [&](int i, int d) {
      dv[d] = i >= 0 ? __ldg(dinv + i) : 0.0;
#pragma unroll
      for (int s = 0; s < 3; ++s) {
        const int tt = 1 + lane + 32 * s;
        u[d][s] = (i >= 0 && tt < C && tt <= i) ? __ldg(Ub + (size_t)(i - tt) * C + tt) : 0.0;
      }
    };
#pragma unroll
    for (int d = 0; d < D; ++d) fetch(r - 1 - d, d);
    for (int i0 = r - 1; i0 >= 0; i0 -= D) {
#pragma unroll
      for (int d = 0; d < D; ++d) {
        const int i = i0 - d;
        if (i >= 0) {
          const double xi = x[i] * dv[d];
          if (lane == 0) {
            Tinv[(size_t)i * r + j] = xi;
            TinvT[(size_t)j * r + i] = xi;
          }
#pragma unroll
          for (int s = 0; s < 3; ++s) {
            const int tt = 1 + lane + 32 * s;
            if (tt < C && tt <= i) x[i - tt] = fma(-u[d][s], xi, x[i - tt]);
          }
          __syncwarp();
          fetch(i - D, d);
        }
      }
    }
  }
}

// the band path's limits: window and multipliers within the kernels' shapes, the band
// narrow against r (a dense T takes Gauss-Jordan)
static bool band_ok(int r, int kl, int ku) {
  const int C = kl + ku + 1;
  return kl <= 64 && C <= 97 && C <= 128 && 2 * C <= r &&
         sizeof(double) * (size_t)(kl + 1) * C <= 200 * 1024 &&
         sizeof(double) * (size_t)r * kBandWarps <= 200 * 1024;
}

cudaError_t launch_band_inverse(int r, int kl, int ku, double* work, double* Tinv,
                                double* TinvT, const double* T, int* err, cudaStream_t st) {
  const int C = kl + ku + 1;
  double* Ub = work;                         // r x C
  double* Lm = Ub + (size_t)r * C;           // r x kl
  double* dinv = Lm + (size_t)r * kl;        // r
  int* piv = reinterpret_cast<int*>(dinv + r);
  const size_t sm = sizeof(double) * (size_t)(kl + 1) * C;
  static cudaError_t a1 = cudaFuncSetAttribute(k_band_lu, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
  static cudaError_t a2 = cudaFuncSetAttribute(k_band_inv, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
  if (a1 != cudaSuccess) return a1;
  if (a2 != cudaSuccess) return a2;
  k_band_lu<<<1, kBandThreads, sm, st>>>(r, kl, ku, T, Ub, dinv, Lm, piv, err);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_band_inv<<<(r + kBandWarps - 1) / kBandWarps, 32 * kBandWarps,
               sizeof(double) * (size_t)r * kBandWarps, st>>>(r, kl, ku, Ub, dinv, Lm, piv,
                                                              Tinv, TinvT);
  return cudaGetLastError();
}

// kernels a Gauss-Jordan inversion enqueues: one cooperative launch when every block's
// rows fit its shared memory, else init, first pivot, one per column and the extraction
static int gj_launches(int r) {
  int dev = 0, sms = 152;
  if (cudaGetDevice(&dev) == cudaSuccess)
    (void)cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int grid = r < sms ? r : sms;
  return (gj_persistent_smem(r, grid) <= 200 * 1024 && (r + grid - 1) / grid <= 63) ? 1 : 3 + r;
}

cudaError_t launch_gauss_jordan(int r, const double* T, double* G /* r*2r */, void* aux,
                                double* Tinv, double* TinvT, int* err, cudaStream_t st) {
  GjAux x;
  double* d = static_cast<double*>(aux);
  x.pinv = d;
  x.pscale = d + r;
  x.cval = d + 2 * (size_t)r;
  int* q = reinterpret_cast<int*>(d + 2 * (size_t)r + 2 * kGjMaxBlocks);
  x.piv = q;
  x.slot = q + r;
  x.used = q + 2 * (size_t)r;
  x.cidx = q + 3 * (size_t)r;
  x.err = err;
  cudaError_t e;
  {  // one cooperative kernel when every block's rows fit in shared memory
    int dev = 0, sms = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess)
      return e;
    const int grid = r < sms ? r : sms;
    const size_t psm = gj_persistent_smem(r, grid);
    if (psm <= 200 * 1024 && (r + grid - 1) / grid <= 63) {
      static cudaError_t attr = cudaFuncSetAttribute(
          k_gj_persistent, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
      if (attr != cudaSuccess) return attr;
      GjP p;
      p.cval = x.cval;
      p.cidx = x.cidx;
      p.crow = G;  // 2 x grid x r doubles of the r x 2r work matrix (grid <= r)
      p.piv = x.piv;
      p.slot = x.slot;
      p.bar = reinterpret_cast<unsigned*>(x.cidx + 2 * kGjMaxBlocks);
      p.err = err;
      if ((e = cudaMemsetAsync(p.bar, 0, 2 * sizeof(unsigned), st)) != cudaSuccess) return e;
      cudaLaunchConfig_t cfg = {};
      cfg.gridDim = dim3((unsigned)grid);
      cfg.blockDim = dim3((unsigned)kGjPThreads);
      cfg.dynamicSmemBytes = psm;
      cfg.stream = st;
      cudaLaunchAttribute at[1];
      at[0].id = cudaLaunchAttributeCooperative;
      at[0].val.cooperative = 1;
      cfg.attrs = at;
      cfg.numAttrs = 1;
      return cudaLaunchKernelEx(&cfg, k_gj_persistent, r, T, p, Tinv, TinvT);
    }
  }
  const size_t sm = sizeof(double) * (size_t)r;
  if (sm > 48 * 1024) {
    e = cudaFuncSetAttribute(k_gj_step, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
  }
  int gs = (r + kGjRowsPerBlock - 1) / kGjRowsPerBlock;
  if (gs > kGjMaxBlocks) gs = kGjMaxBlocks;
  k_gj_init<<<grid_for(2LL * r * r, 256, 152 * 8), 256, 0, st>>>(r, T, G, x);
  k_gj_first<<<1, 1024, 0, st>>>(r, G, x, gs);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  // one launch per column, captured into a CUDA graph (launch gaps of a plain loop of r
  // kernels would dominate)
  cudaStream_t cap;
  if ((e = cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking)) != cudaSuccess) return e;
  cudaGraph_t g = nullptr;
  cudaGraphExec_t ex = nullptr;
  e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeRelaxed);
  if (e == cudaSuccess) {
    for (int k = 0; k < r; ++k)
      k_gj_step<<<gs, 32 * kGjRowsPerBlock, sm, cap>>>(r, k, G, x);
    const cudaError_t le = cudaGetLastError();
    e = cudaStreamEndCapture(cap, &g);
    if (e == cudaSuccess) e = le;
  }
  if (e == cudaSuccess) e = cudaGraphInstantiate(&ex, g, 0);
  if (e == cudaSuccess) e = cudaGraphLaunch(ex, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (ex) cudaGraphExecDestroy(ex);
  if (g) cudaGraphDestroy(g);
  cudaStreamDestroy(cap);
  if (e != cudaSuccess) return e;
  k_gj_extract<<<grid_for((long long)r * r, 256, 152 * 8), 256, 0, st>>>(r, G, x, Tinv, TinvT);
  return cudaGetLastError();
}

// T^-1 (and T^-T): the band path when T is narrowly banded, Gauss-Jordan otherwise.  G
// (r x 2r doubles) is the work matrix of either.  Reads T's bandwidth back to the host;
// band (3 ints, may be null) receives kl, ku and 1 if the band path ran (else 0).
cudaError_t launch_coarse_inverse(int r, const double* T, double* G, void* aux, double* Tinv,
                                  double* TinvT, int* err, int* band, int* nlaunch,
                                  cudaStream_t st) {
  int* bw = reinterpret_cast<int*>(G);
  cudaError_t e = cudaMemsetAsync(bw, 0, 2 * sizeof(int), st);
  if (e != cudaSuccess) return e;
  k_band_width<<<grid_for((long long)r * r, 256, 152 * 4), 256, 0, st>>>(r, T, bw);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  int hb[2] = {0, 0};
  if ((e = cudaMemcpyAsync(hb, bw, sizeof(hb), cudaMemcpyDeviceToHost, st)) != cudaSuccess) return e;
  if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return e;
  const bool use_band = band_ok(r, hb[0], hb[1]);
  if (band) {
    band[0] = hb[0];
    band[1] = hb[1];
    band[2] = use_band ? 1 : 0;
  }
  if (use_band) {
    if (nlaunch) *nlaunch = 3;
    return launch_band_inverse(r, hb[0], hb[1], G, Tinv, TinvT, T, err, st);
  }
  if (nlaunch) *nlaunch = gj_launches(r);
  return launch_gauss_jordan(r, T, G, aux, Tinv, TinvT, err, st);
}

cudaError_t launch_norm_inf(int n, const int* rowptr, const double* val,
                            unsigned long long* out, cudaStream_t st) {
  k_norm_inf<<<grid_for(n, 256, 152 * 4), 256, 0, st>>>(n, rowptr, val, out);
  return cudaGetLastError();
}

cudaError_t launch_to_float(long long n, const double* a, float* b, cudaStream_t st) {
  k_to_float<<<grid_for(n, 256, 152 * 8), 256, 0, st>>>(n, a, b);
  return cudaGetLastError();
}

}  // namespace gg

namespace gg {

int au_scan_blocks(int n) { return (n + kScanBlock - 1) / kScanBlock; }

namespace {
// Row pointers of A W past n set to nau (up to `total` entries), so that kernels copying
// whole tiles of rows read defined values; tmax = the most A W entries in any tile of
// `unit` rows.
__global__ void k_au_tiles(int n, long long total, int unit, int* __restrict__ aurp,
                           int* __restrict__ tmax) {
  const int nau = aurp[n];
  const long long stride = (long long)gridDim.x * blockDim.x;
  const long long t0 = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  for (long long i = t0; i < total; i += stride)
    if (i > n) aurp[i] = nau;
  for (long long t = t0; t * unit < n; t += stride) {
    const long long e = (t + 1) * unit < n ? (t + 1) * unit : n;
    atomicMax(tmax, aurp[e] - aurp[t * unit]);
  }
}
}  // namespace

cudaError_t launch_au_tiles(int n, long long total, int unit, int* aurp, int* tmax,
                            cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(tmax, 0, sizeof(int), st);
  if (e != cudaSuccess) return e;
  k_au_tiles<<<grid_for(total, 256, 152 * 8), 256, 0, st>>>(n, total, unit, aurp, tmax);
  return cudaGetLastError();
}

cudaError_t launch_au_rows(int n, const int* rowptr, const int* col, const int* agg,
                           int* cnt /* n */, int* bsum /* blocks + 1 */, int* aurp /* n + 1 */,
                           cudaStream_t st) {
  const int nb = au_scan_blocks(n);
  k_au_count<<<grid_for(n, 256, 152 * 8), 256, 0, st>>>(n, rowptr, col, agg, cnt);
  k_scan_sums<<<nb, kScanBlock, 0, st>>>(n, cnt, bsum);
  k_scan_top<<<1, kScanBlock, 0, st>>>(nb, bsum);
  k_scan_apply<<<nb, kScanBlock, 0, st>>>(n, nb, cnt, bsum, aurp);
  return cudaGetLastError();
}

cudaError_t launch_au_fill(int n, const int* rowptr, const int* col, const double* val,
                           const int* agg, const int* aurp, int* aucol, double* auval,
                           float* auval32, cudaStream_t st) {
  k_au_fill<<<grid_for(n, 256, 152 * 8), 256, 0, st>>>(n, rowptr, col, val, agg, aurp, aucol,
                                                       auval, auval32);
  return cudaGetLastError();
}

// ---- the first two A W entries of every row in two planes of n (row-indexed, no row
// pointer to chase): plane 0 the first entry, plane 1 the second; column -1 where a row has
// fewer entries, and -(column) - 2 in plane 1 when the row has more than two (the rest
// are read from the CSR rows, from entry aurp[i] + 2) ----
__global__ void k_au_planes(int n, const int* __restrict__ aurp, const int* __restrict__ aucol,
                            const double* __restrict__ auval, const float* __restrict__ auval32,
                            int* __restrict__ pcol, double* __restrict__ pval,
                            float* __restrict__ pval32) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const int s = aurp[i], e = aurp[i + 1];
    for (int q = 0; q < 2; ++q) {
      const bool has = s + q < e;
      int c = has ? aucol[s + q] : -1;
      if (q == 1 && e - s > 2) c = -c - 2;
      pcol[(size_t)q * n + i] = c;
      pval[(size_t)q * n + i] = has ? auval[s + q] : 0.0;
      if (pval32) pval32[(size_t)q * n + i] = has ? auval32[s + q] : 0.f;
    }
  }
}

cudaError_t launch_au_planes(int n, const int* aurp, const int* aucol, const double* auval,
                             const float* auval32, int* pcol, double* pval, float* pval32,
                             cudaStream_t st) {
  k_au_planes<<<grid_for(n, 256, 152 * 8), 256, 0, st>>>(n, aurp, aucol, auval, auval32, pcol,
                                                         pval, pval32);
  return cudaGetLastError();
}

cudaError_t launch_ext_csr(int n, const int* rowptr, const int* col, const double* val,
                           const float* val32, const int* aurp, const int* aucol,
                           const double* auval, const float* auval32, int* xrp, int* xcol,
                           double* xval, float* xval32, cudaStream_t st) {
  k_ext_rows<<<grid_for(n + 1LL, 256, 152 * 8), 256, 0, st>>>(n, rowptr, aurp, xrp);
  k_ext_fill<<<grid_for(n, 256, 152 * 8), 256, 0, st>>>(n, rowptr, col, val, val32, aurp, aucol,
                                                        auval, auval32, xrp, xcol, xval, xval32);
  return cudaGetLastError();
}

cudaError_t launch_dia_detect(int n, const int* rowptr, const int* col, int* slots /* 64 */,
                              int* count, cudaStream_t st) {
  int init[kDiagSlots];
  for (int i = 0; i < kDiagSlots; ++i) init[i] = kDiagEmpty;
  cudaError_t e = cudaMemcpyAsync(slots, init, sizeof(init), cudaMemcpyHostToDevice, st);
  if (e != cudaSuccess) return e;
  if ((e = cudaMemsetAsync(count, 0, sizeof(int), st)) != cudaSuccess) return e;
  if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return e;  // init is a stack array
  k_dia_detect<<<grid_for(n, 256, 152 * 8), 256, 0, st>>>(n, rowptr, col, slots, count);
  return cudaGetLastError();
}

int dia_empty_slot() { return kDiagEmpty; }

cudaError_t launch_dia_fill(int n, const int* rowptr, const int* col, const double* val,
                            const DiaOffsets& offs, long long ldd, double* dval, float* dval32,
                            cudaStream_t st) {
  k_dia_fill<<<grid_for(n, 256, 152 * 8), 256, 0, st>>>(n, rowptr, col, val, offs, ldd, dval,
                                                        dval32);
  return cudaGetLastError();
}

}  // namespace gg
