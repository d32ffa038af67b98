// fem.cu -- Q1 Galerkin assembly on the device (Sec. 3.1, Eqs. 6-8), the adjoint of the
// assembly with respect to the element coefficients, and the CSR transpose used by the
// adjoint solve.
//
// Assembly is row-parallel and gather-based: the thread of row i visits the (at most
// four) elements around node i, so no two threads write the same entry and the result
// is bitwise deterministic.  The sparsity pattern (mesh connectivity, boundary rows
// replaced by u_i = 0) has a closed-form row pointer, so no scan is needed.
#include <cstdio>

#include "common.cuh"
#include "internal.h"

namespace gg {

namespace {

// 1-D integrals of the linear shape functions l0 = 1 - s, l1 = s on [0, 1]:
//   S[a][c] = int l_a' l_c',  Mr[a][c] = int l_a l_c,  G[a][c] = int l_a l_c'.
__device__ __forceinline__ double S1(int a, int c) { return a == c ? 1.0 : -1.0; }
__device__ __forceinline__ double Mr1(int a, int c) { return a == c ? (1.0 / 3.0) : (1.0 / 6.0); }
__device__ __forceinline__ double G1(int /*a*/, int c) { return c == 1 ? 0.5 : -0.5; }

// Element matrices of a square of side h for local nodes (a, b) (test) and (c, d) (trial):
// unit-kappa stiffness, convection with beta, and mass.
__device__ __forceinline__ double elem_K1(int a, int b, int c, int d) {
  return S1(a, c) * Mr1(b, d) + Mr1(a, c) * S1(b, d);
}
__device__ __forceinline__ double elem_C(double h, double bx, double by, int a, int b, int c,
                                         int d) {
  return h * (bx * G1(a, c) * Mr1(b, d) + by * Mr1(a, c) * G1(b, d));
}
__device__ __forceinline__ double elem_M(double h, int a, int b, int c, int d) {
  return h * h * Mr1(a, c) * Mr1(b, d);
}

__device__ __forceinline__ bool on_boundary(int n, int i, int j) {
  return i == 0 || j == 0 || i == n || j == n;
}

// Entries of the CSR before row (i, j): grid rows 0 and n hold n+1 one-entry rows,
// interior grid rows hold 2 boundary rows and n-1 nine-entry rows.
__device__ __forceinline__ long long q1_row_start(int n, int i, int j) {
  const long long interior_line = 2 + 9LL * (n - 1);
  long long before;
  if (j == 0) return i;
  before = (n + 1) + (long long)(j - 1) * interior_line;
  if (j == n) return before + i;
  if (i == 0) return before;
  return before + 1 + 9LL * (i - 1);
}

__global__ void k_q1_assemble(int n, const double* __restrict__ kappa, double bx, double by,
                              const double* __restrict__ f, const double* __restrict__ u,
                              int* __restrict__ rowptr, int* __restrict__ col,
                              double* __restrict__ val, double* __restrict__ b) {
  const int np = n + 1;
  const long long N = (long long)np * np;
  const double h = 1.0 / n;
  for (long long row = blockIdx.x * (long long)blockDim.x + threadIdx.x; row < N;
       row += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(row % np), j = (int)(row / np);
    const long long start = q1_row_start(n, i, j);
    rowptr[row] = (int)start;
    if (row == N - 1) rowptr[N] = (int)(start + 1);
    if (on_boundary(n, i, j)) {
      col[start] = (int)row;
      val[start] = 1.0;
      b[row] = 0.0;
      continue;
    }
    double bi = 0.0;
    long long pos = start;
    for (int dj = -1; dj <= 1; ++dj)
      for (int di = -1; di <= 1; ++di) {
        const int i2 = i + di, j2 = j + dj;
        double a_ij = 0.0;
        // elements (ei, ej) containing both (i, j) and (i2, j2), visited in a fixed order
        for (int ej = max(j, j2) - 1; ej <= min(j, j2); ++ej)
          for (int ei = max(i, i2) - 1; ei <= min(i, i2); ++ei) {
            const int a = i - ei, bb = j - ej, c = i2 - ei, d = j2 - ej;
            const double ke = kappa[(long long)ej * n + ei];
            const double kac = ke * elem_K1(a, bb, c, d) + elem_C(h, bx, by, a, bb, c, d);
            a_ij += kac;
            const long long node2 = (long long)j2 * np + i2;
            bi += elem_M(h, a, bb, c, d) * f[node2];
            if (u) bi -= kac * u[node2];
          }
        col[pos] = (int)((long long)j2 * np + i2);
        val[pos] = a_ij;
        ++pos;
      }
    b[row] = bi;
  }
}

__global__ void k_q1_kappa_grad(int n, const double* __restrict__ lam,
                                const double* __restrict__ x, double* __restrict__ grad) {
  const int np = n + 1;
  const long long ne = (long long)n * n;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < ne;
       e += (long long)gridDim.x * blockDim.x) {
    const int ei = (int)(e % n), ej = (int)(e / n);
    double xe[4];
#pragma unroll
    for (int l = 0; l < 4; ++l) xe[l] = x[(long long)(ej + (l >> 1)) * np + ei + (l & 1)];
    double gsum = 0.0;
#pragma unroll
    for (int l = 0; l < 4; ++l) {
      const int a = l & 1, bb = l >> 1;
      if (on_boundary(n, ei + a, ej + bb)) continue;
      double kx = 0.0;
#pragma unroll
      for (int q = 0; q < 4; ++q) kx += elem_K1(a, bb, q & 1, q >> 1) * xe[q];
      gsum += lam[(long long)(ej + bb) * np + ei + a] * kx;
    }
    grad[e] = -gsum;
  }
}

// ---- transpose: counts -> scan -> scatter -> per-row sort (deterministic result) ----
__global__ void k_count_cols(int nnz, const int* __restrict__ col, int* __restrict__ cnt) {
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < nnz; k += gridDim.x * blockDim.x)
    atomicAdd(&cnt[col[k]], 1);
}

// exclusive scan of cnt[0..n) into out[0..n], single block of 1024 threads, chunked
__global__ void k_scan_single(int n, const int* __restrict__ cnt, int* __restrict__ out) {
  __shared__ int sblock[1024];
  __shared__ int carry;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  for (int base = 0; base < n; base += 1024 * 8) {
    int local[8];
    int s = 0;
#pragma unroll
    for (int t = 0; t < 8; ++t) {
      const int idx = base + threadIdx.x * 8 + t;
      local[t] = idx < n ? cnt[idx] : 0;
      s += local[t];
    }
    sblock[threadIdx.x] = s;
    __syncthreads();
    for (int off = 1; off < 1024; off <<= 1) {  // Hillis-Steele inclusive scan
      const int v = threadIdx.x >= off ? sblock[threadIdx.x - off] : 0;
      __syncthreads();
      sblock[threadIdx.x] += v;
      __syncthreads();
    }
    int run = carry + sblock[threadIdx.x] - s;
#pragma unroll
    for (int t = 0; t < 8; ++t) {
      const int idx = base + threadIdx.x * 8 + t;
      if (idx < n) out[idx] = run;
      run += local[t];
    }
    __syncthreads();
    if (threadIdx.x == 1023) carry += sblock[1023];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[n] = carry;
}

__global__ void k_scatter_t(int n, const int* __restrict__ rowptr, const int* __restrict__ col,
                            const double* __restrict__ val, int* __restrict__ next,
                            int* __restrict__ colt, double* __restrict__ valt) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    for (int k = rowptr[i]; k < rowptr[i + 1]; ++k) {
      const int p = atomicAdd(&next[col[k]], 1);
      colt[p] = i;
      valt[p] = val[k];
    }
}

__global__ void k_sort_rows(int n, const int* __restrict__ rowptr, int* __restrict__ col,
                            double* __restrict__ val) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const int s = rowptr[i], e = rowptr[i + 1];
    for (int k = s + 1; k < e; ++k) {  // insertion sort: FEM rows are short
      const int c = col[k];
      const double v = val[k];
      int t = k - 1;
      while (t >= s && col[t] > c) {
        col[t + 1] = col[t];
        val[t + 1] = val[t];
        --t;
      }
      col[t + 1] = c;
      val[t + 1] = v;
    }
  }
}

}  // namespace

int grid_for(long long work, int threads, int max_blocks) {
  long long b = (work + threads - 1) / threads;
  if (b < 1) b = 1;
  if (b > max_blocks) b = max_blocks;
  return (int)b;
}

cudaError_t launch_q1_assemble(int n, const double* kappa, double bx, double by,
                               const double* f, const double* u, int* rowptr, int* col,
                               double* val, double* b, cudaStream_t st) {
  const long long N = (long long)(n + 1) * (n + 1);
  k_q1_assemble<<<grid_for(N, 256, 152 * 16), 256, 0, st>>>(n, kappa, bx, by, f, u, rowptr,
                                                            col, val, b);
  return cudaGetLastError();
}

cudaError_t launch_q1_kappa_grad(int n, const double* lam, const double* x, double* grad,
                                 cudaStream_t st) {
  k_q1_kappa_grad<<<grid_for((long long)n * n, 256, 152 * 16), 256, 0, st>>>(n, lam, x, grad);
  return cudaGetLastError();
}

cudaError_t launch_transpose(int n, int nnz, const int* rowptr, const int* col,
                             const double* val, int* rowptr_t, int* col_t, double* val_t,
                             int* scratch /* n+1 ints */, cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(scratch, 0, sizeof(int) * (size_t)(n + 1), st);
  if (e != cudaSuccess) return e;
  k_count_cols<<<grid_for(nnz, 256, 152 * 8), 256, 0, st>>>(nnz, col, scratch);
  k_scan_single<<<1, 1024, 0, st>>>(n, scratch, rowptr_t);
  e = cudaMemcpyAsync(scratch, rowptr_t, sizeof(int) * (size_t)n, cudaMemcpyDeviceToDevice, st);
  if (e != cudaSuccess) return e;
  k_scatter_t<<<grid_for(n, 256, 152 * 8), 256, 0, st>>>(n, rowptr, col, val, scratch, col_t,
                                                          val_t);
  k_sort_rows<<<grid_for(n, 256, 152 * 8), 256, 0, st>>>(n, rowptr_t, col_t, val_t);
  return cudaGetLastError();
}

}  // namespace gg
