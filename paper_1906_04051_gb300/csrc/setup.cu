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

__global__ void k_agg_scatter(int n, int r, const int* __restrict__ agg,
                              const int* __restrict__ counts, int* __restrict__ perm) {
  extern __shared__ int soff[];
  for (int a = threadIdx.x; a < r; a += blockDim.x) soff[a] = counts[(size_t)blockIdx.x * r + a];
  __syncthreads();
  if (threadIdx.x == 0) {  // stable: nodes of the chunk in increasing index order
    const int base = blockIdx.x * kChunk;
    const int end = min(n, base + kChunk);
    for (int i = base; i < end; ++i) {
      const int a = agg[i];
      if (a >= 0) perm[soff[a]++] = i;
    }
  }
}

// pieces: aggregate a is split into ceil(cnt_a / kPiece) consecutive ranges of perm
__global__ void k_pieces(int r, const int* __restrict__ aggptr, const int* __restrict__ cnt,
                         int* __restrict__ agg_piece, int* __restrict__ piece_start,
                         double* __restrict__ uscale, int* __restrict__ err) {
  if (threadIdx.x == 0) {
    int np = 0;
    for (int a = 0; a < r; ++a) {
      agg_piece[a] = np;
      const int c = cnt[a];
      if (c == 0) atomicOr(err, 4);
      for (int s = 0; s < c; s += kPiece) piece_start[np++] = aggptr[a] + s;
    }
    agg_piece[r] = np;
    piece_start[np] = aggptr[r];
  }
  __syncthreads();
  for (int a = threadIdx.x; a < r; a += blockDim.x)
    uscale[a] = cnt[a] > 0 ? 1.0 / sqrt((double)cnt[a]) : 0.0;
}

// T row of aggregate p: sum_{i in p} sum_{k in row i, agg(col_k) = q} a_ik, in perm order.
// Small r: lanes take nodes round-robin into private rows, summed in lane order.
// Large r: lane 0 accumulates sequentially, the warp loads each row's entries.
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

// ---- Gauss-Jordan inverse of T on the augmented r x 2r matrix G = [T | I] ----
__global__ void k_gj_init(int r, const double* __restrict__ T, double* __restrict__ G) {
  const long long tot = 2LL * r * r;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < tot;
       t += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(t / (2 * r)), j = (int)(t % (2 * r));
    G[t] = j < r ? T[(size_t)i * r + j] : (j - r == i ? 1.0 : 0.0);
  }
}

// Pivot step for column k, run by one block: the largest |G_ik| over i >= k (first on
// ties; candidates come from pmax/pidx partials when given, else from a scan), row swap
// k <-> p, scaling of row k, and the elimination factors fac_i = G_ik (fac_k = 0).
__device__ void gj_pivot_block(int r, int k, double* __restrict__ G, double* __restrict__ fac,
                               int* __restrict__ err) {
  __shared__ double sv[32];
  __shared__ int si[32];
  __shared__ int s_piv;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int ld = 2 * r;
  double best = -1.0;
  int bi = r;
  for (int i = k + threadIdx.x; i < r; i += blockDim.x) {
    const double v = fabs(__ldcg(&G[(size_t)i * ld + k]));
    if (v > best) { best = v; bi = i; }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const double ov = __shfl_xor_sync(0xffffffffu, best, o);
    const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
    if (ov > best || (ov == best && oi < bi)) { best = ov; bi = oi; }
  }
  if (lane == 0) { sv[warp] = best; si[warp] = bi; }
  __syncthreads();
  if (threadIdx.x == 0) {
    double b = -1.0;
    int p = r;
    for (int w = 0; w < nw; ++w)
      if (sv[w] > b || (sv[w] == b && si[w] < p)) { b = sv[w]; p = si[w]; }
    if (!(b > 0.0) || p >= r) { atomicOr(err, 8); p = k; }
    s_piv = p;
  }
  __syncthreads();
  const int p = s_piv;
  if (p != k)
    for (int j = threadIdx.x; j < ld; j += blockDim.x) {
      const double t = __ldcg(&G[(size_t)k * ld + j]);
      G[(size_t)k * ld + j] = __ldcg(&G[(size_t)p * ld + j]);
      G[(size_t)p * ld + j] = t;
    }
  __syncthreads();
  const double piv = __ldcg(&G[(size_t)k * ld + k]);
  const double inv = (piv != 0.0) ? 1.0 / piv : 0.0;
  __syncthreads();
  for (int j = threadIdx.x; j < ld; j += blockDim.x)
    if (j != k) G[(size_t)k * ld + j] = __ldcg(&G[(size_t)k * ld + j]) * inv;
  __syncthreads();
  if (threadIdx.x == 0) G[(size_t)k * ld + k] = 1.0;
  for (int i = threadIdx.x; i < r; i += blockDim.x)
    fac[i] = (i == k) ? 0.0 : __ldcg(&G[(size_t)i * ld + k]);
}

__global__ void k_gj_pivot0(int r, double* __restrict__ G, double* __restrict__ fac,
                            int* __restrict__ err) {
  gj_pivot_block(r, 0, G, fac, err);
}

// Step k: G_ij -= fac_i G_kj for i != k over columns [k, 2r) (row swaps move the identity
// columns of the right half, so all of it stays active); each block owns whole rows.  The
// last block to finish (ticket) performs the pivot step of column k + 1.
__global__ void __launch_bounds__(1024)
    k_gj_step(int r, int k, double* __restrict__ G, double* __restrict__ fac,
              unsigned* __restrict__ ticket, int* __restrict__ err) {
  __shared__ unsigned s_last;
  const int ld = 2 * r;
  for (int i = blockIdx.x; i < r; i += gridDim.x) {
    const double f = fac[i];
    if (f == 0.0) continue;
    const double* prow = G + (size_t)k * ld;
    double* row = G + (size_t)i * ld;
    for (int j = k + threadIdx.x; j < ld; j += blockDim.x) row[j] -= f * __ldcg(prow + j);
  }
  if (k + 1 >= r) return;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) s_last = (atomicAdd(ticket, 1u) == gridDim.x - 1) ? 1u : 0u;
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  gj_pivot_block(r, k + 1, G, fac, err);
  if (threadIdx.x == 0) *ticket = 0u;
}

__global__ void k_gj_extract(int r, const double* __restrict__ G, double* __restrict__ Tinv,
                             double* __restrict__ TinvT) {
  const long long tot = (long long)r * r;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < tot;
       t += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(t / r), j = (int)(t % r);
    const double v = G[(size_t)i * 2 * r + r + j];
    Tinv[t] = v;
    if (TinvT) TinvT[(size_t)j * r + i] = v;
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
                            int* err, cudaStream_t st) {
  const int nb = agg_chunks(n);
  const size_t sm = sizeof(int) * (size_t)r;
  k_agg_count<<<nb, 256, sm, st>>>(n, r, agg, counts);
  k_agg_scan<<<1, 1024, 0, st>>>(r, nb, counts, aggptr, cnt);
  k_agg_scatter<<<nb, 32, sm, st>>>(n, r, agg, counts, perm);
  k_pieces<<<1, 256, 0, st>>>(r, aggptr, cnt, agg_piece, piece_start, uscale, err);
  return cudaGetLastError();
}

cudaError_t launch_coarse_T(int r, const int* rowptr, const int* col, const double* val,
                            const int* agg, const int* perm, const int* aggptr,
                            const double* uscale, double* T, cudaStream_t st) {
  const bool lane_rows = (r * 32 * (int)sizeof(double)) <= 48 * 1024;
  const size_t sm = sizeof(double) * (size_t)r * (lane_rows ? 32 : 1);
  if (sm > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(k_T_rows, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)sm);
    if (e != cudaSuccess) return e;
  }
  k_T_rows<<<r, 32, sm, st>>>(r, rowptr, col, val, agg, perm, aggptr, uscale, T);
  return cudaGetLastError();
}

cudaError_t launch_gauss_jordan(int r, const double* T, double* G /* r*2r */, double* fac,
                                double* Tinv, double* TinvT, int* err, cudaStream_t st) {
  // one launch per column, captured into a CUDA graph (launch gaps of a plain loop of r
  // kernels would dominate for r ~ 1000)
  unsigned* ticket = reinterpret_cast<unsigned*>(fac + r);  // fac has r + 1 doubles
  cudaError_t e = cudaMemsetAsync(ticket, 0, sizeof(unsigned), st);
  if (e != cudaSuccess) return e;
  k_gj_init<<<grid_for(2LL * r * r, 256, 152 * 8), 256, 0, st>>>(r, T, G);
  k_gj_pivot0<<<1, 1024, 0, st>>>(r, G, fac, err);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  int dev = 0, sms = 152;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int grid = r < 2 * sms ? r : 2 * sms;
  cudaStream_t cap;
  if ((e = cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking)) != cudaSuccess) return e;
  cudaGraph_t g = nullptr;
  cudaGraphExec_t ex = nullptr;
  e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeRelaxed);
  if (e == cudaSuccess) {
    for (int k = 0; k < r; ++k) k_gj_step<<<grid, 256, 0, cap>>>(r, k, G, fac, ticket, err);
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
  k_gj_extract<<<grid_for((long long)r * r, 256, 152 * 8), 256, 0, st>>>(r, G, Tinv, TinvT);
  return cudaGetLastError();
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
