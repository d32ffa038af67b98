// adaptive.cu -- the paper's adaptive deflation update (Sec. 3.3, Eq. 19), FP64.
//
// After every restart cycle of k steps: the eigenvector z of the cycle's k x k Hessenberg
// matrix H_k for its smallest-modulus eigenvalue (inverse power method; a complex pair of
// smallest eigenvalues gives two vectors spanning its invariant subspace), u = V_k z,
// orthonormalised against U (two classical Gram-Schmidt passes) and appended to U; A u is
// appended to A U and T = U^T A U grows by a row and a column.  With rmax columns already
// in U, the direction of T's largest-modulus eigenvalue leaves first (two directions for
// a complex pair): U keeps the complement of that eigenvalue's left eigenvector(s), a
// T-invariant subspace carrying the other eigenvalues, in the basis U H_0 (H_1) given by
// Householder reflectors that map the dropped directions onto single coordinates (rank-1
// updates of U and A U instead of a dense rotation), T <- H T H without those rows and
// columns.  T^-1 follows.  Arithmetic runs in the kernels below and in the pipelined
// multi-dot of arnoldi.cu; the host only sequences them and reads the few scalars that
// decide the branches (vector count, norms, the number of dropped directions).  A
// deflation space given as dense columns W is built by the same steps (dense_build).
#include <cmath>
#include <cstring>

#include "handle.h"
#include "kernels.cuh"

namespace gg {

namespace {

// ---- inverse power method on H_k, one warp ------------------------------------------
// Same steps as the oracle's: LU of the Hessenberg matrix with partial pivoting between
// the two rows a column touches (a zero pivot becomes 1e-14 max|H|), ninv iterations
// z <- H^-1 z / ||H^-1 z|| from the normalised all-ones vector, the sign making the
// largest-magnitude entry positive (the first on ties); if ||Hz - (z^T H z) z|| >
// 1e-3 ||Hz|| one more iterate, orthonormalised against z, is the second vector.
// z lives in registers, entry i in lane i % 32 (z0: i < 32, z1: i >= 32); the two
// triangular solves are chains of k dependent steps, so each step is a shuffle and an
// FMA, with the factors read from shared memory off the chain.

struct WZ {  // a vector of k <= 64 entries spread over the warp
  double z0, z1;
};

__device__ __forceinline__ double wz_get(const WZ& v, int i) {
  return __shfl_sync(0xffffffffu, i < 32 ? v.z0 : v.z1, i & 31);
}

// z <- U^-1 L^-1 P z for the factors of the Hessenberg LU: sw[j] (rows j and j+1
// exchanged at step j), l[j] (multiplier of step j), Ut (U transposed: Ut[c * 64 + r] =
// U[r][c]) and rd (1 / U[i][i]).
__device__ void warp_hess_solve(int k, const double* Ut, const int* sw, const double* l,
                                const double* rd, WZ& z, int lane) {
  // forward: the row operations of the factorisation in order; c carries the current
  // entry j, which step j finalises
  double c = wz_get(z, 0);
  WZ f{0.0, 0.0};
  for (int j = 0; j + 1 < k; ++j) {
    const double o = wz_get(z, j + 1);  // not yet touched by the chain
    const double lj = l[j];
    double fin, nxt;
    if (sw[j]) {
      fin = o;
      nxt = c - lj * o;
    } else {
      fin = c;
      nxt = o - lj * c;
    }
    if (lane == (j & 31)) (j < 32 ? f.z0 : f.z1) = fin;
    c = nxt;
  }
  if (lane == ((k - 1) & 31)) (k - 1 < 32 ? f.z0 : f.z1) = c;
  // backward, by columns: x_i = y_i / u_ii, then the rows above drop u_ri x_i
  for (int i = k - 1; i >= 0; --i) {
    const double xi = wz_get(f, i) * rd[i];
    if (lane == (i & 31)) (i < 32 ? f.z0 : f.z1) = xi;
    const double* col = Ut + i * 64;
    if (lane < i) f.z0 -= col[lane] * xi;
    if (lane + 32 < i) f.z1 -= col[lane + 32] * xi;
  }
  z = f;
}

__device__ void warp_normalise_sign(int k, WZ& z, int lane) {
  const double a0 = lane < k ? z.z0 : 0.0, a1 = lane + 32 < k ? z.z1 : 0.0;
  const double s = warp_sum(a0 * a0 + a1 * a1);
  const double inv = 1.0 / sqrt(s);
  z.z0 = a0 * inv;
  z.z1 = a1 * inv;
  // largest magnitude, first index on ties
  double bv = -1.0;
  int bi = 0x7fffffff;
  if (lane < k) {
    bv = fabs(z.z0);
    bi = lane;
  }
  if (lane + 32 < k && fabs(z.z1) > bv) {
    bv = fabs(z.z1);
    bi = lane + 32;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const double ov = __shfl_xor_sync(0xffffffffu, bv, o);
    const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
    if (ov > bv || (ov == bv && oi < bi)) {
      bv = ov;
      bi = oi;
    }
  }
  if (wz_get(z, bi) < 0.0) {
    z.z0 = -z.z0;
    z.z1 = -z.z1;
  }
}

__global__ void k_adapt_z(Ctl ctl, int ninv, double* __restrict__ zout, int* __restrict__ iv) {
  static_assert(kMaxM <= 64, "the register layout holds 64 entries");
  __shared__ double a[kMaxM * kMaxM];  // the LU factors in place, U transposed afterwards
  __shared__ double l[kMaxM], rd[kMaxM];
  __shared__ int sw[kMaxM];
  const int lane = threadIdx.x;
  const int k = ctl.flags[F_K];
  if (k < 1 || k > kMaxM) {
    if (lane == 0) iv[0] = 0;
    return;
  }
  const int ldh = ctl.ldh;
  double hmax = 0.0;
  for (int t = lane; t < k * k; t += 32) {
    const int i = t / k, c = t % k;
    const double v = i <= c + 1 ? ctl.Hr[(size_t)i * ldh + c] : 0.0;  // below: never written
    a[t] = v;
    hmax = fmax(hmax, fabs(v));
  }
  hmax = warp_max(hmax);
  const double eps = hmax > 0.0 ? 1e-14 * hmax : 1e-300;
  __syncwarp();
  // Hessenberg LU with partial pivoting between rows j and j+1
  for (int j = 0; j < k; ++j) {
    const bool swp = j + 1 < k && fabs(a[(j + 1) * k + j]) > fabs(a[j * k + j]);
    if (swp)
      for (int c = j + lane; c < k; c += 32) {
        const double t = a[j * k + c];
        a[j * k + c] = a[(j + 1) * k + c];
        a[(j + 1) * k + c] = t;
      }
    __syncwarp();
    if (lane == 0) {
      sw[j] = swp ? 1 : 0;
      l[j] = 0.0;
      if (a[j * k + j] == 0.0) a[j * k + j] = eps;
      if (j + 1 < k) l[j] = a[(j + 1) * k + j] / a[j * k + j];
    }
    __syncwarp();
    if (j + 1 < k) {
      const double lj = l[j];
      for (int c = j + 1 + lane; c < k; c += 32) a[(j + 1) * k + c] -= lj * a[j * k + c];
      __syncwarp();
      if (lane == 0) a[(j + 1) * k + j] = 0.0;
    }
    __syncwarp();
  }
  // U transposed into registers' order of access (column i contiguous), reciprocal pivots
  double ut[kMaxM * kMaxM / 32];
  int nt = 0;
  for (int t = lane; t < k * k; t += 32) ut[nt++] = a[t];
  __syncwarp();
  nt = 0;
  for (int t = lane; t < k * k; t += 32) {
    const int r = t / k, c = t % k;
    a[c * 64 + r] = r <= c ? ut[nt] : 0.0;
    ++nt;
  }
  __syncwarp();
  for (int i = lane; i < k; i += 32) rd[i] = 1.0 / a[i * 64 + i];
  __syncwarp();
  WZ z{lane < k ? 1.0 / sqrt((double)k) : 0.0, lane + 32 < k ? 1.0 / sqrt((double)k) : 0.0};
  for (int it = 0; it < ninv; ++it) {
    warp_hess_solve(k, a, sw, l, rd, z, lane);
    warp_normalise_sign(k, z, lane);
  }
  // eigenvector test with the Rayleigh quotient rho = z^T H z
  double rho = 0.0, nhz = 0.0, hz0 = 0.0, hz1 = 0.0;
  for (int c = 0; c < k; ++c) {
    const double zc = wz_get(z, c);
    // H z over the Hessenberg entries (row i has columns c >= i - 1)
    if (lane < k && lane <= c + 1) hz0 += ctl.Hr[(size_t)lane * ldh + c] * zc;
    if (lane + 32 < k && lane + 32 <= c + 1) hz1 += ctl.Hr[(size_t)(lane + 32) * ldh + c] * zc;
  }
  rho = warp_sum(z.z0 * hz0 + z.z1 * hz1);
  nhz = warp_sum(hz0 * hz0 + hz1 * hz1);
  const double r0 = hz0 - rho * z.z0, r1 = hz1 - rho * z.z1;
  const double res = warp_sum(r0 * r0 + r1 * r1);
  int nvec = 1;
  WZ z2{0.0, 0.0};
  if (sqrt(res) > 1e-3 * sqrt(nhz)) {
    z2 = z;
    warp_hess_solve(k, a, sw, l, rd, z2, lane);
    const double c = warp_sum(z.z0 * z2.z0 + z.z1 * z2.z1);
    z2.z0 -= c * z.z0;
    z2.z1 -= c * z.z1;
    warp_normalise_sign(k, z2, lane);
    nvec = 2;
  }
  for (int i = lane; i < kMaxK; i += 32) {
    const bool lo = i < 32;
    zout[i] = i < k ? (lo ? z.z0 : z.z1) : 0.0;
    zout[kMaxK + i] = (nvec == 2 && i < k) ? (lo ? z2.z0 : z2.z1) : 0.0;
  }
  if (lane == 0) iv[0] = nvec;
}

// u = V_k z (the basis columns as stored, v_c = sigma_c u_c: z is scaled by sigma here)
__global__ void __launch_bounds__(kThreads)
    k_adapt_vz(int N, const double* __restrict__ V, long long ldv, const double* __restrict__ z,
               Ctl ctl, double* __restrict__ u) {
  __shared__ double sz[kMaxK];
  const int k = ctl.flags[F_K];
  for (int c = threadIdx.x; c < k; c += blockDim.x) sz[c] = z[c] * ctl.sigma[c];
  __syncthreads();
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int c = 0; c < k; ++c) s += V[(size_t)c * ldv + i] * sz[c];
    u[i] = s;
  }
}

// out = ||u||_2 (deterministic grid reduction)
__global__ void __launch_bounds__(kThreads)
    k_adapt_norm(int N, const double* __restrict__ u, Ctl ctl, double* __restrict__ out) {
  __shared__ double sbuf[kThreads / 32];
  __shared__ double sred[1];
  __shared__ double tot[1];
  double s = 0.0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x)
    s += u[i] * u[i];
  const double bs = block_sum(s, sbuf);
  if (threadIdx.x == 0) sred[0] = bs;
  __syncthreads();
  if (!last_block_reduce(sred, 1, ctl.part, ctl.part2, ctl.ldp, ctl.ticket, tot)) return;
  if (threadIdx.x == 0) *out = sqrt(tot[0]);
}

// u -= U c (q columns)
__global__ void __launch_bounds__(kThreads)
    k_adapt_axpy(int N, double* __restrict__ u, const double* __restrict__ U, long long ldu,
                 int q, const double* __restrict__ c) {
  __shared__ double sc[kMaxAdapt + 1];
  for (int t = threadIdx.x; t < q; t += blockDim.x) sc[t] = c[t];
  __syncthreads();
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x) {
    double v = u[i];
    for (int t = 0; t < q; ++t) v -= U[(size_t)t * ldu + i] * sc[t];
    u[i] = v;
  }
}

// dst = u / nrm
__global__ void __launch_bounds__(kThreads)
    k_adapt_scale(int N, const double* __restrict__ u, const double* __restrict__ nrm,
                  double* __restrict__ dst) {
  const double inv = 1.0 / *nrm;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x)
    dst[i] = u[i] * inv;
}

// y = A x in FP64 (CSR): kVecLanes lanes per row, kVecRows consecutive rows per lane
// group (the layout of the step's SpMV for long rows; short rows lose little by it)
__global__ void __launch_bounds__(kThreads)
    k_adapt_spmv(int N, const int* __restrict__ rowptr, const int* __restrict__ col,
                 const double* __restrict__ val, const double* __restrict__ x,
                 double* __restrict__ y) {
  constexpr int G = kVecLanes, R = kVecRows, GPW = 32 / G;
  const int sub = threadIdx.x & (G - 1);
  const long long gid = (blockIdx.x * (long long)blockDim.x + threadIdx.x) / G;
  const long long groups = (long long)gridDim.x * blockDim.x / G;
  const long long nb = (N + R - 1) / R;
  for (long long base = gid & ~(long long)(GPW - 1); base < nb; base += groups) {
    const long long bund = base + (gid & (GPW - 1));
    double acc[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
      acc[r] = 0.0;
      const long long row = bund * R + r;
      if (bund < nb && row < N)
        for (int e = __ldg(rowptr + row) + sub; e < __ldg(rowptr + row + 1); e += G)
          acc[r] += __ldg(val + e) * x[__ldg(col + e)];
    }
#pragma unroll
    for (int r = 0; r < R; ++r)
#pragma unroll
      for (int o = G / 2; o > 0; o >>= 1) acc[r] += __shfl_xor_sync(0xffffffffu, acc[r], o);
    if (bund < nb && sub < R) {
      double v = acc[0];
#pragma unroll
      for (int r = 1; r < R; ++r)
        if (sub == r) v = acc[r];
      if (bund * R + sub < N) y[bund * R + sub] = v;
    }
  }
}

// T (row stride ldt): column q from c1 (q+1 entries), row q from c2 (q entries)
__global__ void k_adapt_tset(double* __restrict__ T, int ldt, int q, const double* __restrict__ c1,
                             const double* __restrict__ c2) {
  for (int i = threadIdx.x; i <= q; i += blockDim.x) T[(size_t)i * ldt + q] = c1[i];
  for (int i = threadIdx.x; i < q; i += blockDim.x) T[(size_t)q * ldt + i] = c2[i];
}

// ---- drop step at rmax, one warp --------------------------------------------------
// T (q x q, row stride ldt): Householder reduction of a copy to Hessenberg form, Francis
// QR (hqr_warp) for the eigenvalue lambda = a + i b of largest modulus, its left
// eigenvector y (T^T y = lambda y) by three inverse iterations from all ones on the real
// form [[T^T - a I, b I], [-b I, T^T - a I]] (LU with partial pivoting, first index on
// ties; a pivot of modulus <= 1e-14 max|entry| becomes that bound), then p Householder
// reflectors H_c = I - beta_c v_c v_c^T mapping the columns of Y = [Re y (, Im y)] onto
// single coordinates jd_c (the columns of Q = H_0 ... H_{p-1} other than jd_c span
// {c : y^T c = 0}); T <- Q^T T Q with rows and columns jd_c removed, the dropped slots
// below q - p refilled from the kept coordinates above.  Qc receives v_0 (, v_1) and
// beta_0, beta_1 for k_adapt_reflect; out[0] = p (1, or 2 for a complex pair), out[1] = 1
// if the QR iteration did not converge, out[2 + s] = the coordinate that slot s keeps.
__global__ void __launch_bounds__(32)
    k_adapt_drop(double* __restrict__ T, int ldt, int q, double* __restrict__ Qc,
                 int* __restrict__ out) {
  constexpr int Q = kMaxAdapt;
  __shared__ double M[4 * Q * Q];  // Hessenberg copy, then the shifted system, then Qc | T Qc
  __shared__ double T0[Q * Q];
  __shared__ double y[2 * Q], hv[2][Q], hb[2], sv[Q];
  __shared__ int piv[2 * Q];
  __shared__ double sre, sim, smod;
  __shared__ int sfail;
  const int lane = threadIdx.x;
  for (int t = lane; t < q * q; t += 32) {
    const double v = T[(size_t)(t / q) * ldt + t % q];
    T0[t] = v;
    M[t] = v;
  }
  __syncwarp();
  // Householder reduction of M (row stride q) to upper Hessenberg form
  for (int k = 0; k + 2 < q; ++k) {
    const int len = q - k - 1;
    const double x = lane < len ? M[(k + 1 + lane) * q + k] : 0.0;
    const double nx = sqrt(warp_sum(x * x));
    if (nx == 0.0) continue;
    const double x0 = __shfl_sync(0xffffffffu, x, 0);
    const double alpha = x0 >= 0.0 ? -nx : nx;
    const double v = lane < len ? x - (lane == 0 ? alpha : 0.0) : 0.0;
    const double vv = warp_sum(v * v);
    if (vv == 0.0) continue;
    const double beta = 2.0 / vv;
    sv[lane] = v;
    __syncwarp();
    if (lane < q) {  // (I - beta v v^T) on rows k+1.., column lane
      double sd = 0.0;
      for (int i = 0; i < len; ++i) sd += sv[i] * M[(k + 1 + i) * q + lane];
      for (int i = 0; i < len; ++i) M[(k + 1 + i) * q + lane] -= beta * sd * sv[i];
    }
    __syncwarp();
    if (lane < q) {  // on columns k+1.., row lane
      double sd = 0.0;
      for (int j = 0; j < len; ++j) sd += M[lane * q + k + 1 + j] * sv[j];
      for (int j = 0; j < len; ++j) M[lane * q + k + 1 + j] -= beta * sd * sv[j];
    }
    __syncwarp();
    if (lane == 0) M[(k + 1) * q + k] = alpha;
    if (lane >= 1 && lane < len) M[(k + 1 + lane) * q + k] = 0.0;
    __syncwarp();
  }
  hqr_warp(M, q, sre, sim, smod, sfail);
  if (sfail) {
    if (lane == 0) {
      out[0] = 0;
      out[1] = 1;
    }
    return;
  }
  const double la = sre, lb = sim;
  const int p = lb != 0.0 ? 2 : 1, n2 = p * q;
  // the shifted real system (row stride n2)
  double mx = 0.0;
  for (int t = lane; t < n2 * n2; t += 32) {
    const int i = t / n2, j = t % n2, bi = i / q, ii = i % q, bj = j / q, jj = j % q;
    double v;
    if (bi == bj) v = T0[jj * q + ii] - (ii == jj ? la : 0.0);
    else if (bi == 0) v = ii == jj ? lb : 0.0;
    else v = ii == jj ? -lb : 0.0;
    M[t] = v;
    mx = fmax(mx, fabs(v));
  }
  mx = warp_max(mx);
  const double eps = mx > 0.0 ? 1e-14 * mx : 1e-300;
  __syncwarp();
  for (int k = 0; k < n2; ++k) {
    double bv = -1.0;
    int bi = n2;
    for (int i = k + lane; i < n2; i += 32) {
      const double a = fabs(M[i * n2 + k]);
      if (a > bv) { bv = a; bi = i; }
    }
    for (int o = 16; o > 0; o >>= 1) {
      const double ov = __shfl_xor_sync(0xffffffffu, bv, o);
      const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
      if (ov > bv || (ov == bv && oi < bi)) { bv = ov; bi = oi; }
    }
    if (bi >= n2) bi = k;  // no comparable entry (NaN column): keep the row order
    if (lane == 0) piv[k] = bi;
    if (bi != k)
      for (int j = lane; j < n2; j += 32) {
        const double t = M[k * n2 + j];
        M[k * n2 + j] = M[bi * n2 + j];
        M[bi * n2 + j] = t;
      }
    __syncwarp();
    if (lane == 0 && fabs(M[k * n2 + k]) <= eps) M[k * n2 + k] = eps;
    __syncwarp();
    const double pv = M[k * n2 + k];
    for (int i = k + 1 + lane; i < n2; i += 32) {
      const double l = M[i * n2 + k] / pv;
      M[i * n2 + k] = l;
      for (int j = k + 1; j < n2; ++j) M[i * n2 + j] -= l * M[k * n2 + j];
    }
    __syncwarp();
  }
  for (int i = lane; i < n2; i += 32) y[i] = 1.0;
  __syncwarp();
  for (int it = 0; it < 3; ++it) {
    if (lane == 0)
      for (int k = 0; k < n2; ++k)
        if (piv[k] != k) {
          const double t = y[k];
          y[k] = y[piv[k]];
          y[piv[k]] = t;
        }
    __syncwarp();
    for (int j = 0; j < n2; ++j) {  // L (unit diagonal), by columns
      const double yj = y[j];
      for (int i = j + 1 + lane; i < n2; i += 32) y[i] -= M[i * n2 + j] * yj;
      __syncwarp();
    }
    for (int i = n2 - 1; i >= 0; --i) {  // U, by columns
      if (lane == 0) y[i] /= M[i * n2 + i];
      __syncwarp();
      const double yi = y[i];
      for (int r = lane; r < i; r += 32) y[r] -= M[r * n2 + i] * yi;
      __syncwarp();
    }
    double ss = 0.0;
    for (int i = lane; i < n2; i += 32) ss += y[i] * y[i];
    const double inv = 1.0 / sqrt(warp_sum(ss));
    for (int i = lane; i < n2; i += 32) y[i] *= inv;
    __syncwarp();
  }
  // Householder reflectors H_c = I - beta_c v_c v_c^T, c < p, each mapping column c of
  // Y = [Re y (, Im y)] (after the earlier reflectors) onto a coordinate jd_c, chosen as
  // its largest entry among the coordinates not yet taken; v_c vanishes on those, so
  // Q = H_0 ... H_{p-1} has Q e_{jd_c} spanning span(Y) and its other columns spanning
  // the complement {c : y^T c = 0}.  U Q is then U with p rank-1 updates, and T's
  // new coordinates are Q^T T Q with rows and columns jd_c removed.
  double yc[2];
  yc[0] = lane < q ? y[lane] : 0.0;
  yc[1] = (p == 2 && lane < q) ? y[q + lane] : 0.0;
  int used = -1;
  for (int c = 0; c < p; ++c) {
    const double x = (lane < q && lane != used) ? yc[c] : 0.0;
    double bv = fabs(x);
    int bi = lane < q && lane != used ? lane : 64;
    for (int o = 16; o > 0; o >>= 1) {
      const double ov = __shfl_xor_sync(0xffffffffu, bv, o);
      const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
      if (ov > bv || (ov == bv && oi < bi)) {
        bv = ov;
        bi = oi;
      }
    }
    const int jc = bi < q ? bi : 0;
    const double nx = sqrt(warp_sum(x * x));
    const double xj = __shfl_sync(0xffffffffu, x, jc);
    const double alpha = xj >= 0.0 ? -nx : nx;
    const double v = x - (lane == jc ? alpha : 0.0);
    const double vv = warp_sum(v * v);
    const double beta = vv > 0.0 ? 2.0 / vv : 0.0;
    hv[c][lane] = v;
    if (lane == 0) {
      hb[c] = beta;
      piv[c] = jc;
    }
    if (c + 1 < p) {
      const double sd = warp_sum(v * yc[c + 1]);
      yc[c + 1] -= beta * sd * v;
    }
    used = jc;
  }
  __syncwarp();
  // T <- H_c T H_c for c = 0..p-1 (T0, row stride q)
  for (int c = 0; c < p; ++c) {
    const double bt = hb[c];
    if (lane < q) {  // left: column lane
      double sd = 0.0;
      for (int i = 0; i < q; ++i) sd += hv[c][i] * T0[i * q + lane];
      for (int i = 0; i < q; ++i) T0[i * q + lane] -= bt * sd * hv[c][i];
    }
    __syncwarp();
    if (lane < q) {  // right: row lane
      double sd = 0.0;
      for (int jj = 0; jj < q; ++jj) sd += T0[lane * q + jj] * hv[c][jj];
      for (int jj = 0; jj < q; ++jj) T0[lane * q + jj] -= bt * sd * hv[c][jj];
    }
    __syncwarp();
  }
  // slots of the kept coordinates: a dropped slot below nc takes the next kept
  // coordinate at or above nc; map[s] = source coordinate of slot s
  const int nc = q - p;
  if (lane == 0) {
    int src = nc;
    for (int sl = 0; sl < nc; ++sl) {
      bool drop = false;
      for (int c = 0; c < p; ++c) drop = drop || piv[c] == sl;
      if (!drop) {
        piv[8 + sl] = sl;
        continue;
      }
      for (;; ++src) {
        bool dsrc = false;
        for (int c = 0; c < p; ++c) dsrc = dsrc || piv[c] == src;
        if (!dsrc) break;
      }
      piv[8 + sl] = src++;
    }
  }
  __syncwarp();
  if (lane < nc)
    for (int i = 0; i < nc; ++i) T[(size_t)i * ldt + lane] = T0[piv[8 + i] * q + piv[8 + lane]];
  // reflectors and the slot map for k_adapt_reflect and the column moves
  for (int c = 0; c < p; ++c) Qc[c * Q + lane] = hv[c][lane];
  if (lane == 0) {
    Qc[2 * Q] = hb[0];
    Qc[2 * Q + 1] = p == 2 ? hb[1] : 0.0;
    out[0] = p;
    out[1] = 0;
  }
  if (lane < nc) out[2 + lane] = piv[8 + lane];
}

// U <- U H_0 ... H_{p-1} and A U <- A U H_0 ... H_{p-1} in place (q columns), thread per
// row: w = X v_c, X -= beta_c w v_c^T.  QT >= q bounds the unrolled column loops.
template <int QT>
__global__ void __launch_bounds__(kThreads)
    k_adapt_reflect(int N, double* __restrict__ U, double* __restrict__ AU, long long ld, int q,
                    int p, const double* __restrict__ hvec) {
  __shared__ double sv[2][kMaxAdapt], sb[2];
  for (int t = threadIdx.x; t < 2 * kMaxAdapt; t += blockDim.x)
    sv[t / kMaxAdapt][t % kMaxAdapt] = (t / kMaxAdapt) < p ? hvec[t] : 0.0;
  if (threadIdx.x < 2) sb[threadIdx.x] = hvec[2 * kMaxAdapt + threadIdx.x];
  __syncthreads();
  for (int row = blockIdx.x * blockDim.x + threadIdx.x; row < N; row += gridDim.x * blockDim.x)
    for (int pass = 0; pass < 2; ++pass) {
      double* X = pass == 0 ? U : AU;
      double u[QT];
#pragma unroll
      for (int t = 0; t < QT; ++t) u[t] = t < q ? X[(size_t)t * ld + row] : 0.0;
      for (int c = 0; c < p; ++c) {
        double w = 0.0;
#pragma unroll
        for (int t = 0; t < QT; ++t) w += u[t] * sv[c][t];
        w *= sb[c];
#pragma unroll
        for (int t = 0; t < QT; ++t) u[t] -= w * sv[c][t];
      }
#pragma unroll
      for (int t = 0; t < QT; ++t)
        if (t < q) X[(size_t)t * ld + row] = u[t];
    }
}

// Tinv (q x q, row stride q) = T^-1 by Gauss-Jordan with partial pivoting, one block;
// bit 0 of *bad is set when a pivot is zero
__global__ void k_adapt_tinv(const double* __restrict__ T, int ldt, int q,
                             double* __restrict__ Tinv, int* __restrict__ bad) {
  __shared__ double G[kMaxAdapt][2 * kMaxAdapt + 1];
  __shared__ int sp;
  for (int t = threadIdx.x; t < q * 2 * q; t += blockDim.x) {
    const int i = t / (2 * q), j = t % (2 * q);
    G[i][j] = j < q ? T[(size_t)i * ldt + j] : (j - q == i ? 1.0 : 0.0);
  }
  __syncthreads();
  for (int k = 0; k < q; ++k) {
    if (threadIdx.x == 0) {
      int p = k;
      for (int i = k + 1; i < q; ++i)
        if (fabs(G[i][k]) > fabs(G[p][k])) p = i;
      if (G[p][k] == 0.0) *bad = 1;
      sp = p;
    }
    __syncthreads();
    const int p = sp;
    if (p != k)
      for (int j = threadIdx.x; j < 2 * q; j += blockDim.x) {
        const double t = G[k][j];
        G[k][j] = G[p][j];
        G[p][j] = t;
      }
    __syncthreads();
    const double piv = G[k][k];
    __syncthreads();
    for (int j = threadIdx.x; j < 2 * q; j += blockDim.x) G[k][j] = piv != 0.0 ? G[k][j] / piv : 0.0;
    __syncthreads();
    for (int t = threadIdx.x; t < q * 2 * q; t += blockDim.x) {
      const int i = t / (2 * q), j = t % (2 * q);
      if (i != k && j != k) G[i][j] -= G[i][k] * G[k][j];
    }
    __syncthreads();
    for (int i = threadIdx.x; i < q; i += blockDim.x)
      if (i != k) G[i][k] = 0.0;
    __syncthreads();
  }
  for (int t = threadIdx.x; t < q * q; t += blockDim.x) Tinv[t] = G[t / q][q + t % q];
}

}  // namespace

// The dense space from the caller's columns W (the same steps as an update of the
// adaptive space, without the eigenvector and the drop): each column orthonormalised
// against the previous ones by two multi-dot passes, appended with A u and T's new row
// and column; then T^-1.
gmres_status dense_build(gmres_s* h, CycleArgs& a) {
  cudaStream_t st = h->stream;
  const int N = h->n;
  const long long ld = h->ldv;
  const int R = h->opts.rmax;  // = the number of columns of W
  double* U = h->aU.as<double>();
  double* AU = h->aAU.as<double>();
  double* T = h->aT.as<double>();
  double* Tinv = h->aTinv.as<double>();
  double* u = h->au.as<double>();
  double* sm = h->asmall.as<double>();
  double* c1 = sm + 2 * kMaxK;
  double* c2 = c1 + kMaxAdapt + 1;
  double* nrm = c2 + kMaxAdapt + 1;
  double* qc = nrm + 2;
  int* iv = reinterpret_cast<int*>(qc + kMaxAdapt * kMaxAdapt);
  const int tiles = (N + kThreads - 1) / kThreads;
  const int grid = grid_for(tiles, 1, 8 * h->sms);
  const Ctl& ctl = a.ctl;
  const double* W = h->wdense.as<double>();
  int q = 0;
  for (int c = 0; c < h->dense_r; ++c) {
    CK(h, cudaMemcpyAsync(u, W + (size_t)c * N, sizeof(double) * N, cudaMemcpyDeviceToDevice, st));
    k_adapt_norm<<<grid, kThreads, 0, st>>>(N, u, ctl, nrm);
    for (int pass = 0; pass < 2 && q > 0; ++pass) {
      CK(h, launch_udots(a, U, ld, q, u, DotEpi{kEpiRaw, nullptr, 0, c1, -1}, st));
      k_adapt_axpy<<<grid, kThreads, 0, st>>>(N, u, U, ld, q, c1);
    }
    k_adapt_norm<<<grid, kThreads, 0, st>>>(N, u, ctl, nrm + 1);
    CK(h, cudaGetLastError());
    double hn[2];
    CK(h, cudaMemcpyAsync(hn, nrm, sizeof(hn), cudaMemcpyDeviceToHost, st));
    CK(h, cudaStreamSynchronize(st));
    if (!(hn[1] > 1e-10 * hn[0]))
      return fail(h, GMRES_ERR_INVALID_ARG,
                  "dense W: column " + std::to_string(c) + " lies in the span of the previous ones");
    k_adapt_scale<<<grid, kThreads, 0, st>>>(N, u, nrm + 1, U + (size_t)q * ld);
    k_adapt_spmv<<<grid_for((long long)N * kVecLanes / kVecRows, kThreads, 64 * h->sms), kThreads,
                   0, st>>>(N, a.op.rowptr, a.op.col, a.op.val, U + (size_t)q * ld,
                            AU + (size_t)q * ld);
    CK(h, launch_udots(a, U, ld, q + 1, AU + (size_t)q * ld, DotEpi{kEpiRaw, nullptr, 0, c1, -1}, st));
    if (q > 0)
      CK(h, launch_udots(a, AU, ld, q, U + (size_t)q * ld, DotEpi{kEpiRaw, nullptr, 0, c2, -1}, st));
    k_adapt_tset<<<1, 64, 0, st>>>(T, R, q, c1, c2);
    CK(h, cudaGetLastError());
    ++q;
  }
  CK(h, cudaMemsetAsync(iv + 1, 0, sizeof(int), st));
  k_adapt_tinv<<<1, 256, 0, st>>>(T, R, q, Tinv, iv + 1);
  int bad = 0;
  CK(h, cudaMemcpyAsync(&bad, iv + 1, sizeof(int), cudaMemcpyDeviceToHost, st));
  CK(h, cudaStreamSynchronize(st));
  if (bad) return fail(h, GMRES_ERR_SINGULAR_COARSE, "dense W: T = U^T A U is singular");
  h->aq = q;
  return GMRES_OK;
}

// One update of the adaptive deflation space after a cycle (see the file comment).
gmres_status adapt_update(gmres_s* h, CycleArgs& a) {
  cudaStream_t st = h->stream;
  const int N = h->n;
  const long long ld = h->ldv;
  const int R = h->opts.rmax;
  double* U = h->aU.as<double>();
  double* AU = h->aAU.as<double>();
  double* T = h->aT.as<double>();
  double* Tinv = h->aTinv.as<double>();
  double* u = h->au.as<double>();
  double* sm = h->asmall.as<double>();
  double* z = sm;                        // 2 x kMaxK
  double* c1 = z + 2 * kMaxK;            // kMaxAdapt + 1
  double* c2 = c1 + kMaxAdapt + 1;       // kMaxAdapt + 1
  double* nrm = c2 + kMaxAdapt + 1;      // 2
  double* qc = nrm + 2;                  // reflectors of the drop step (2 kMaxAdapt + 2)
  int* iv = reinterpret_cast<int*>(qc + kMaxAdapt * kMaxAdapt);  // nvec, bad, p, fail, map
  const int tiles = (N + kThreads - 1) / kThreads;
  const int grid = grid_for(tiles, 1, 8 * h->sms);
  const Ctl& ctl = a.ctl;
  long long nl = 0;

  k_adapt_z<<<1, 32, 0, st>>>(ctl, h->opts.ninv, z, iv);
  CK(h, cudaGetLastError());
  ++nl;
  int hiv[2] = {0, 0};
  CK(h, cudaMemcpyAsync(hiv, iv, sizeof(hiv), cudaMemcpyDeviceToHost, st));
  CK(h, cudaStreamSynchronize(st));
  const int nvec = hiv[0];
  int q = h->aq;
  for (int v = 0; v < nvec; ++v) {
    k_adapt_vz<<<grid, kThreads, 0, st>>>(N, static_cast<const double*>(a.V), ld,
                                          z + (size_t)v * kMaxK, ctl, u);
    k_adapt_norm<<<grid, kThreads, 0, st>>>(N, u, ctl, nrm);
    nl += 2;
    for (int pass = 0; pass < 2 && q > 0; ++pass) {
      launch_udots(a, U, ld, q, u, DotEpi{kEpiRaw, nullptr, 0, c1, -1}, st);
      k_adapt_axpy<<<grid, kThreads, 0, st>>>(N, u, U, ld, q, c1);
      nl += 2;
    }
    k_adapt_norm<<<grid, kThreads, 0, st>>>(N, u, ctl, nrm + 1);
    ++nl;
    CK(h, cudaGetLastError());
    double hn[2];
    CK(h, cudaMemcpyAsync(hn, nrm, sizeof(hn), cudaMemcpyDeviceToHost, st));
    CK(h, cudaStreamSynchronize(st));
    if (!(hn[1] > 1e-10 * hn[0])) continue;  // already in span(U)
    if (q == R) {  // U is full: the direction(s) of T's largest eigenvalue leave first
      k_adapt_drop<<<1, 32, 0, st>>>(T, R, q, qc, iv + 2);
      CK(h, cudaGetLastError());
      int hd[2 + kMaxAdapt] = {0};
      CK(h, cudaMemcpyAsync(hd, iv + 2, sizeof(hd), cudaMemcpyDeviceToHost, st));
      CK(h, cudaStreamSynchronize(st));
      if (hd[1] || hd[0] < 1 || hd[0] > q)
        return fail(h, GMRES_ERR_SINGULAR_COARSE,
                    "adaptive deflation: the QR iteration on T = U^T A U did not converge");
      const int p = hd[0], nc = q - p;
      if (q <= 8)
        k_adapt_reflect<8><<<grid, kThreads, 0, st>>>(N, U, AU, ld, q, p, qc);
      else if (q <= 16)
        k_adapt_reflect<16><<<grid, kThreads, 0, st>>>(N, U, AU, ld, q, p, qc);
      else if (q <= 24)
        k_adapt_reflect<24><<<grid, kThreads, 0, st>>>(N, U, AU, ld, q, p, qc);
      else
        k_adapt_reflect<32><<<grid, kThreads, 0, st>>>(N, U, AU, ld, q, p, qc);
      nl += 2;
      for (int sl = 0; sl < nc; ++sl)  // the dropped slots below nc take kept columns
        if (hd[2 + sl] != sl) {
          CK(h, cudaMemcpyAsync(U + (size_t)sl * ld, U + (size_t)hd[2 + sl] * ld,
                                sizeof(double) * N, cudaMemcpyDeviceToDevice, st));
          CK(h, cudaMemcpyAsync(AU + (size_t)sl * ld, AU + (size_t)hd[2 + sl] * ld,
                                sizeof(double) * N, cudaMemcpyDeviceToDevice, st));
        }
      q = nc;
    }
    k_adapt_scale<<<grid, kThreads, 0, st>>>(N, u, nrm + 1, U + (size_t)q * ld);
    k_adapt_spmv<<<grid_for((long long)N * kVecLanes / kVecRows, kThreads, 64 * h->sms), kThreads,
                   0, st>>>(N, a.op.rowptr, a.op.col, a.op.val, U + (size_t)q * ld,
                            AU + (size_t)q * ld);
    nl += 2;
    launch_udots(a, U, ld, q + 1, AU + (size_t)q * ld, DotEpi{kEpiRaw, nullptr, 0, c1, -1}, st);
    ++nl;
    if (q > 0) {
      launch_udots(a, AU, ld, q, U + (size_t)q * ld, DotEpi{kEpiRaw, nullptr, 0, c2, -1}, st);
      ++nl;
    }
    k_adapt_tset<<<1, 64, 0, st>>>(T, R, q, c1, c2);
    ++nl;
    ++q;
  }
  if (q > 0) {
    CK(h, cudaMemsetAsync(iv + 1, 0, sizeof(int), st));
    k_adapt_tinv<<<1, 256, 0, st>>>(T, R, q, Tinv, iv + 1);
    ++nl;
    CK(h, cudaMemcpyAsync(hiv, iv, sizeof(hiv), cudaMemcpyDeviceToHost, st));
    CK(h, cudaStreamSynchronize(st));
    if (hiv[1]) return fail(h, GMRES_ERR_SINGULAR_COARSE, "T = U^T A U of the adaptive space is singular");
  }
  CK(h, cudaGetLastError());
  h->aq = q;
  h->plaunch[PH_ADAPT] += nl;
  return GMRES_OK;
}

}  // namespace gg
