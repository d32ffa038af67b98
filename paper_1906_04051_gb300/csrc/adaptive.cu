// adaptive.cu -- the paper's adaptive deflation update (Sec. 3.3, Eq. 19), FP64.
//
// After every restart cycle of k steps: the eigenvector z of the cycle's k x k Hessenberg
// matrix H_k for its smallest-modulus eigenvalue (inverse power method; a complex pair of
// smallest eigenvalues gives two vectors spanning its invariant subspace), u = V_k z,
// orthonormalised against U (two classical Gram-Schmidt passes) and appended to U; A u is
// appended to A U and T = U^T A U grows by a row and a column.  With rmax columns already
// in U, the direction of T's largest-modulus eigenvalue leaves first (two directions for
// a complex pair): U <- U Qc, A U <- A U Qc, T <- Qc^T T Qc, where Qc is an orthonormal
// basis of the complement of that eigenvalue's left eigenvector(s), a T-invariant
// subspace carrying the other eigenvalues.  T^-1 follows.  Arithmetic runs in the
// kernels below and in the pipelined multi-dot of arnoldi.cu; the host only sequences
// them and reads the few scalars that decide the branches (vector count, norms, the
// number of dropped directions).
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
__device__ void warp_hess_solve(int k, const double* a, const int* sw, const double* l,
                                double* z, int lane) {
  // forward: the row operations of the factorisation, in order (lane 0)
  if (lane == 0)
    for (int j = 0; j + 1 < k; ++j) {
      if (sw[j]) {
        const double t = z[j];
        z[j] = z[j + 1];
        z[j + 1] = t;
      }
      z[j + 1] -= l[j] * z[j];
    }
  __syncwarp();
  // backward, by columns: z_i /= a_ii, then the rows above drop a_ri z_i
  for (int i = k - 1; i >= 0; --i) {
    if (lane == 0) z[i] /= a[i * k + i];
    __syncwarp();
    const double zi = z[i];
    for (int r = lane; r < i; r += 32) z[r] -= a[r * k + i] * zi;
    __syncwarp();
  }
}

__device__ void warp_normalise_sign(int k, double* z, int lane) {
  double s = 0.0;
  for (int i = lane; i < k; i += 32) s += z[i] * z[i];
  s = warp_sum(s);
  const double inv = 1.0 / sqrt(s);
  __syncwarp();
  for (int i = lane; i < k; i += 32) z[i] *= inv;
  __syncwarp();
  // largest magnitude, first index on ties
  double bv = -1.0;
  int bi = 0x7fffffff;
  for (int i = lane; i < k; i += 32)
    if (fabs(z[i]) > bv) {
      bv = fabs(z[i]);
      bi = i;
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
  const bool neg = z[bi] < 0.0;
  __syncwarp();
  if (neg)
    for (int i = lane; i < k; i += 32) z[i] = -z[i];
  __syncwarp();
}

__global__ void k_adapt_z(Ctl ctl, int ninv, double* __restrict__ zout, int* __restrict__ iv) {
  __shared__ double a[kMaxM * kMaxM];  // the LU factors (H itself is read from ctl.Hr)
  __shared__ double l[kMaxM], z[kMaxM], z2[kMaxM], hz[kMaxM];
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
    const double v = ctl.Hr[(size_t)i * ldh + c];
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
  for (int i = lane; i < k; i += 32) z[i] = 1.0 / sqrt((double)k);
  __syncwarp();
  for (int it = 0; it < ninv; ++it) {
    warp_hess_solve(k, a, sw, l, z, lane);
    warp_normalise_sign(k, z, lane);
  }
  // eigenvector test with the Rayleigh quotient
  double rho = 0.0, nhz = 0.0;
  for (int i = lane; i < k; i += 32) {
    double s = 0.0;
    for (int c = 0; c < k; ++c) s += ctl.Hr[(size_t)i * ldh + c] * z[c];
    hz[i] = s;
    rho += z[i] * s;
    nhz += s * s;
  }
  rho = warp_sum(rho);
  nhz = warp_sum(nhz);
  __syncwarp();
  double res = 0.0;
  for (int i = lane; i < k; i += 32) res += (hz[i] - rho * z[i]) * (hz[i] - rho * z[i]);
  res = warp_sum(res);
  int nvec = 1;
  if (sqrt(res) > 1e-3 * sqrt(nhz)) {
    for (int i = lane; i < k; i += 32) z2[i] = z[i];
    __syncwarp();
    warp_hess_solve(k, a, sw, l, z2, lane);
    double c = 0.0;
    for (int i = lane; i < k; i += 32) c += z[i] * z2[i];
    c = warp_sum(c);
    __syncwarp();
    for (int i = lane; i < k; i += 32) z2[i] -= c * z[i];
    __syncwarp();
    warp_normalise_sign(k, z2, lane);
    nvec = 2;
  }
  for (int i = lane; i < kMaxK; i += 32) {
    zout[i] = i < k ? z[i] : 0.0;
    zout[kMaxK + i] = (nvec == 2 && i < k) ? z2[i] : 0.0;
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

// y = A x in FP64 (CSR, thread per row)
__global__ void __launch_bounds__(kThreads)
    k_adapt_spmv(int N, const int* __restrict__ rowptr, const int* __restrict__ col,
                 const double* __restrict__ val, const double* __restrict__ x,
                 double* __restrict__ y) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int e = __ldg(rowptr + i); e < __ldg(rowptr + i + 1); ++e)
      s += __ldg(val + e) * x[__ldg(col + e)];
    y[i] = s;
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
// ties; a pivot of modulus <= 1e-14 max|entry| becomes that bound), Householder QR of
// Y = [Re y (, Im y)] and Qc = (H_0 ... H_{p-1})[:, p:] (row stride kMaxAdapt), the
// orthonormal basis of {c : y^T c = 0}; T's leading (q-p) x (q-p) block becomes
// Qc^T T Qc.  out[0] = p (1, or 2 for a complex pair), out[1] = 1 if the QR iteration
// did not converge.
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
  // Householder QR of Y = [y[0..q) (, y[q..2q))]; lane i holds row i
  double yc[2];
  yc[0] = lane < q ? y[lane] : 0.0;
  yc[1] = (p == 2 && lane < q) ? y[q + lane] : 0.0;
  for (int c = 0; c < p; ++c) {
    const double x = (lane >= c && lane < q) ? yc[c] : 0.0;
    const double nx = sqrt(warp_sum(x * x));
    const double x0 = __shfl_sync(0xffffffffu, yc[c], c);
    const double alpha = x0 >= 0.0 ? -nx : nx;
    const double v = (lane >= c && lane < q) ? x - (lane == c ? alpha : 0.0) : 0.0;
    const double vv = warp_sum(v * v);
    const double beta = vv > 0.0 ? 2.0 / vv : 0.0;
    hv[c][lane] = v;
    if (lane == 0) hb[c] = beta;
    if (c + 1 < p) {
      const double sd = warp_sum(v * yc[c + 1]);
      if (lane >= c && lane < q) yc[c + 1] -= beta * sd * v;
    }
  }
  __syncwarp();
  const int nc = q - p;
  double* Qs = M;          // q x nc, row stride Q
  double* Ws = M + Q * Q;  // T Qc, row stride Q
  if (lane < nc) {         // column lane of (H_0 ... H_{p-1}) E, E = I[:, p:]
    for (int i = 0; i < q; ++i) Qs[i * Q + lane] = i == p + lane ? 1.0 : 0.0;
    for (int c = p - 1; c >= 0; --c) {
      double sd = 0.0;
      for (int i = c; i < q; ++i) sd += hv[c][i] * Qs[i * Q + lane];
      for (int i = c; i < q; ++i) Qs[i * Q + lane] -= hb[c] * sd * hv[c][i];
    }
    for (int i = 0; i < q; ++i) {
      double sd = 0.0;
      for (int l = 0; l < q; ++l) sd += T0[i * q + l] * Qs[l * Q + lane];
      Ws[i * Q + lane] = sd;
    }
  }
  __syncwarp();
  if (lane < nc) {
    for (int i = 0; i < nc; ++i) {
      double sd = 0.0;
      for (int l = 0; l < q; ++l) sd += Qs[l * Q + i] * Ws[l * Q + lane];
      T[(size_t)i * ldt + lane] = sd;
    }
    for (int i = 0; i < q; ++i) Qc[i * Q + lane] = Qs[i * Q + lane];
  }
  if (lane == 0) {
    out[0] = p;
    out[1] = 0;
  }
}

// U <- U Qc and A U <- A U Qc in place (q columns to nc), thread per row
__global__ void __launch_bounds__(kThreads)
    k_adapt_rotate(int N, double* __restrict__ U, double* __restrict__ AU, long long ld, int q,
                   int nc, const double* __restrict__ Qc) {
  __shared__ double sq[kMaxAdapt * kMaxAdapt];
  for (int t = threadIdx.x; t < q * kMaxAdapt; t += blockDim.x) sq[t] = Qc[t];
  __syncthreads();
  for (int row = blockIdx.x * blockDim.x + threadIdx.x; row < N; row += gridDim.x * blockDim.x)
    for (int pass = 0; pass < 2; ++pass) {
      double* X = pass == 0 ? U : AU;
      double u[kMaxAdapt];
#pragma unroll
      for (int t = 0; t < kMaxAdapt; ++t) u[t] = t < q ? X[(size_t)t * ld + row] : 0.0;
      for (int c = 0; c < nc; ++c) {
        double sd = 0.0;
#pragma unroll
        for (int t = 0; t < kMaxAdapt; ++t)
          if (t < q) sd += u[t] * sq[t * kMaxAdapt + c];
        X[(size_t)c * ld + row] = sd;
      }
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
  double* qc = nrm + 2;                  // kMaxAdapt x kMaxAdapt
  int* iv = reinterpret_cast<int*>(qc + kMaxAdapt * kMaxAdapt);  // nvec, bad, p, fail
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
      int hd[2] = {0, 0};
      CK(h, cudaMemcpyAsync(hd, iv + 2, sizeof(hd), cudaMemcpyDeviceToHost, st));
      CK(h, cudaStreamSynchronize(st));
      if (hd[1] || hd[0] < 1 || hd[0] > q)
        return fail(h, GMRES_ERR_SINGULAR_COARSE,
                    "adaptive deflation: the QR iteration on T = U^T A U did not converge");
      const int nc = q - hd[0];
      k_adapt_rotate<<<grid, kThreads, 0, st>>>(N, U, AU, ld, q, nc, qc);
      nl += 2;
      q = nc;
    }
    k_adapt_scale<<<grid, kThreads, 0, st>>>(N, u, nrm + 1, U + (size_t)q * ld);
    k_adapt_spmv<<<grid, kThreads, 0, st>>>(N, a.op.rowptr, a.op.col, a.op.val,
                                            U + (size_t)q * ld, AU + (size_t)q * ld);
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
