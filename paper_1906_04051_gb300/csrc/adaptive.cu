// adaptive.cu -- the paper's adaptive deflation update (Sec. 3.3, Eq. 19), FP64.
//
// After every restart cycle of k steps: the eigenvector z of the cycle's k x k Hessenberg
// matrix H_k for its smallest-modulus eigenvalue (inverse power method; a complex pair of
// smallest eigenvalues gives two vectors spanning its invariant subspace), u = V_k z,
// orthonormalised against U (two classical Gram-Schmidt passes) and appended to U; A u is
// appended to A U and T = U^T A U grows by a row and a column; beyond rmax columns the
// column with the largest |T_jj| is dropped first (the last column takes its place).
// T^-1 follows.  Arithmetic runs in the kernels below and in the pipelined multi-dot of
// arnoldi.cu; the host only sequences them and reads the few scalars that decide the
// branches (vector count, norms, T's diagonal).
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

// T: row and column last move to jd (the dropped column's place)
__global__ void k_adapt_tmove(double* __restrict__ T, int ldt, int last, int jd) {
  __shared__ double row[kMaxAdapt], colv[kMaxAdapt];
  for (int j = threadIdx.x; j <= last; j += blockDim.x) {
    row[j] = T[(size_t)last * ldt + j];
    colv[j] = T[(size_t)j * ldt + last];
  }
  __syncthreads();
  for (int j = threadIdx.x; j <= last; j += blockDim.x) {
    T[(size_t)jd * ldt + j] = row[j];
    T[(size_t)j * ldt + jd] = colv[j];
  }
  __syncthreads();
  if (threadIdx.x == 0) T[(size_t)jd * ldt + jd] = T[(size_t)last * ldt + last];
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
  int* iv = reinterpret_cast<int*>(nrm + 2);  // nvec, bad
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
    if (q == R) {  // r > rmax: deflate the column whose |T_jj| is largest
      double d[kMaxAdapt];
      for (int j = 0; j < q; ++j)
        CK(h, cudaMemcpyAsync(d + j, T + (size_t)j * R + j, sizeof(double), cudaMemcpyDeviceToHost,
                              st));
      CK(h, cudaStreamSynchronize(st));
      int jd = 0;
      for (int j = 1; j < q; ++j)
        if (std::fabs(d[j]) > std::fabs(d[jd])) jd = j;
      const int last = q - 1;
      if (jd != last) {
        CK(h, cudaMemcpyAsync(U + (size_t)jd * ld, U + (size_t)last * ld, sizeof(double) * N,
                              cudaMemcpyDeviceToDevice, st));
        CK(h, cudaMemcpyAsync(AU + (size_t)jd * ld, AU + (size_t)last * ld, sizeof(double) * N,
                              cudaMemcpyDeviceToDevice, st));
        k_adapt_tmove<<<1, 32, 0, st>>>(T, R, last, jd);
        ++nl;
      }
      q = last;
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
