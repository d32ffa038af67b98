// bratu.cu -- the paper's benchmark problem on the device: the 3-D Bratu equation
// lap u + lambda exp(u) = 0 on the unit cube (Sec. 3.1, Eqs. 2-9), u = 0 on the x- and
// y-faces, du/dz = 0 on the z-faces, discretised by the Galerkin method with 27-node
// triquadratic hexahedra; the Newton system J(u) du = -R(u) and a Newton driver whose
// linear solves are this library's deflated GMRES(m).
//
// Mesh: n^3 cubes of side h = 1/n, M = 2n + 1 nodes per direction, node (I, J, K) ->
// (K M + J) M + I.  Rows of x- and y-face nodes are replaced by du_i = 0 (one stored
// 1.0, b_i = 0); the other rows keep their couplings to those columns (the pattern is the
// mesh connectivity, which the paper's Table 1 counts).
//
// Assembly is row-parallel and gather-based (no atomics, bitwise deterministic): the
// thread of row i visits the 1, 2, 4 or 8 elements around node i.  Per element it forms
// the exp(u_h) values at the 3 x 3 x 3 Gauss-Legendre points by sum factorisation and the
// row of the element Jacobian
//   J_e[l][m] = - int grad phi_m . grad phi_l + lambda int exp(u_h) phi_m phi_l,
// the stiffness part from the exact 1-D integrals of the quadratic Lagrange functions
// (h (S x M x M + M x S x M + M x M x S)), the exp part by the quadrature, again by sum
// factorisation (243 FMA per row and element instead of 729).
#include <cmath>
#include <cstring>

#include "handle.h"
#include "kernels.cuh"

namespace gg {

namespace {

// Coupled nodes of node I along one direction (a vertex node, even I, shares elements
// with the nodes within 2 of it, a mid-edge node with those within 1), clamped to the
// mesh.
__device__ __forceinline__ void q2_range(int M, int I, int& lo, int& hi) {
  const int r = (I & 1) ? 1 : 2;
  lo = I - r < 0 ? 0 : I - r;
  hi = I + r > M - 1 ? M - 1 : I + r;
}

// Entries of the rows 1..I-1 of an interior line, per unit of the other two counts:
// interior nodes couple with 3 (odd) or 5 (even) nodes along the line.
__device__ __forceinline__ long long q2_px(int I) {
  return I >= 1 ? 3LL * (I / 2) + 5LL * ((I - 1) / 2) : 0;
}

__device__ __forceinline__ int q2_cz(int M, int K) {  // along z every node is a row
  return ((K & 1) || K == 0 || K == M - 1) ? 3 : 5;
}

// First CSR entry of row (I, J, K) in closed form (planes, then lines, then nodes);
// Sx = 8n - 5 entries per interior line and unit of the other two counts.
__device__ __forceinline__ long long q2_row_start(int n, int I, int J, int K) {
  const int M = 2 * n + 1;
  const long long Sx = 8LL * n - 5;
  long long base = (long long)K * (4 * M - 4) + Sx * Sx * (K == 0 ? 0 : 3 + q2_px(K));
  if (J == 0) return base + I;
  base += M + 2LL * (J - 1) + (long long)q2_cz(M, K) * Sx * q2_px(J);
  if (J == M - 1) return base + I;
  if (I == 0) return base;
  return base + 1 + (long long)((J & 1) ? 3 : 5) * q2_cz(M, K) * q2_px(I);
}

struct Q2Tab {
  double P[3][3];  // P[g][a]: 1-D quadratic Lagrange function a at Gauss point g
  double w[3];     // 1-D Gauss weights on [0, 1]
  double S[3][3];  // exact int p_a' p_c' on [0, 1]
  double Mm[3][3]; // exact int p_a p_c on [0, 1]
};

__device__ void q2_tables(Q2Tab& t) {
  const double gs = sqrt(0.6);
  const double xg[3] = {0.5 * (1.0 - gs), 0.5, 0.5 * (1.0 + gs)};
  for (int g = 0; g < 3; ++g) {
    const double s = xg[g];
    t.P[g][0] = (1.0 - s) * (1.0 - 2.0 * s);
    t.P[g][1] = 4.0 * s * (1.0 - s);
    t.P[g][2] = s * (2.0 * s - 1.0);
  }
  t.w[0] = 5.0 / 18.0;
  t.w[1] = 8.0 / 18.0;
  t.w[2] = 5.0 / 18.0;
  const double S3[3][3] = {{7.0, -8.0, 1.0}, {-8.0, 16.0, -8.0}, {1.0, -8.0, 7.0}};
  const double M30[3][3] = {{4.0, 2.0, -1.0}, {2.0, 16.0, 2.0}, {-1.0, 2.0, 4.0}};
  for (int a = 0; a < 3; ++a)
    for (int c = 0; c < 3; ++c) {
      t.S[a][c] = S3[a][c] / 3.0;
      t.Mm[a][c] = M30[a][c] / 30.0;
    }
}

// Row of J (values) and b = -R for the rows of the mesh; rowptr and col as well.
__global__ void __launch_bounds__(128)
    k_q2_assemble(int n, double lambda, const double* __restrict__ u, int* __restrict__ rowptr,
                  int* __restrict__ col, double* __restrict__ val, double* __restrict__ b) {
  __shared__ Q2Tab tab;
  if (threadIdx.x == 0) q2_tables(tab);
  __syncthreads();
  const int M = 2 * n + 1;
  const long long N = (long long)M * M * M;
  const double h = 1.0 / n, h3 = h * h * h;
  for (long long row = blockIdx.x * (long long)blockDim.x + threadIdx.x; row < N;
       row += (long long)gridDim.x * blockDim.x) {
    const int I = (int)(row % M), J = (int)((row / M) % M), K = (int)(row / ((long long)M * M));
    const long long start = q2_row_start(n, I, J, K);
    rowptr[row] = (int)start;
    if (row == N - 1) rowptr[N] = (int)(start + 1);
    if (I == 0 || J == 0 || I == M - 1 || J == M - 1) {  // x- and y-faces: du_i = 0
      col[start] = (int)row;
      val[start] = 1.0;
      b[row] = 0.0;
      continue;
    }
    int a0, a1, b0, b1, c0, c1;
    q2_range(M, I, a0, a1);
    q2_range(M, J, b0, b1);
    q2_range(M, K, c0, c1);
    const int nx = a1 - a0 + 1, ny = b1 - b0 + 1;
    {
      long long p = start;
      for (int k = c0; k <= c1; ++k)
        for (int jj = b0; jj <= b1; ++jj)
          for (int i = a0; i <= a1; ++i) {
            col[p] = (int)(((long long)k * M + jj) * M + i);
            val[p] = 0.0;
            ++p;
          }
    }
    double bi = 0.0;
    // elements around the node: two per direction for a vertex node (clamped), one for
    // a mid-edge node; visited in a fixed order
    const int ex0 = (I & 1) ? (I - 1) / 2 : max(I / 2 - 1, 0), ex1 = (I & 1) ? ex0 : min(I / 2, n - 1);
    const int ey0 = (J & 1) ? (J - 1) / 2 : max(J / 2 - 1, 0), ey1 = (J & 1) ? ey0 : min(J / 2, n - 1);
    const int ez0 = (K & 1) ? (K - 1) / 2 : max(K / 2 - 1, 0), ez1 = (K & 1) ? ez0 : min(K / 2, n - 1);
    for (int ez = ez0; ez <= ez1; ++ez)
      for (int ey = ey0; ey <= ey1; ++ey)
        for (int ex = ex0; ex <= ex1; ++ex) {
          const int la = I - 2 * ex, lb = J - 2 * ey, lc = K - 2 * ez;  // local node of the row
          double ue[27];
          for (int c = 0; c < 3; ++c)
            for (int bb = 0; bb < 3; ++bb)
              for (int a = 0; a < 3; ++a) {
                const long long g = ((long long)(2 * ez + c) * M + 2 * ey + bb) * M + 2 * ex + a;
                ue[a + 3 * bb + 9 * c] = u ? u[g] : 0.0;
              }
          // u_h at the Gauss points: contract x, then y, then z
          double t1[27], t2[27];
          for (int c = 0; c < 3; ++c)
            for (int bb = 0; bb < 3; ++bb)
              for (int gx = 0; gx < 3; ++gx) {
                double s = 0.0;
                for (int a = 0; a < 3; ++a) s += tab.P[gx][a] * ue[a + 3 * bb + 9 * c];
                t1[gx + 3 * bb + 9 * c] = s;
              }
          for (int c = 0; c < 3; ++c)
            for (int gy = 0; gy < 3; ++gy)
              for (int gx = 0; gx < 3; ++gx) {
                double s = 0.0;
                for (int bb = 0; bb < 3; ++bb) s += tab.P[gy][bb] * t1[gx + 3 * bb + 9 * c];
                t2[gx + 3 * gy + 9 * c] = s;
              }
          // E[g] = w_g exp(u_h(g)) phi_l(g) (row's local node l = (la, lb, lc))
          double E[27], rexp = 0.0;
          for (int gz = 0; gz < 3; ++gz)
            for (int gy = 0; gy < 3; ++gy)
              for (int gx = 0; gx < 3; ++gx) {
                double ug = 0.0;
                for (int c = 0; c < 3; ++c) ug += tab.P[gz][c] * t2[gx + 3 * gy + 9 * c];
                const double e = tab.w[gx] * tab.w[gy] * tab.w[gz] * h3 * exp(ug) *
                                 tab.P[gx][la] * tab.P[gy][lb] * tab.P[gz][lc];
                E[gx + 3 * gy + 9 * gz] = e;
                rexp += e;
              }
          // Q[m] = sum_g E[g] phi_m(g): contract gx -> a', gy -> b', gz -> c'
          for (int gz = 0; gz < 3; ++gz)
            for (int gy = 0; gy < 3; ++gy)
              for (int a = 0; a < 3; ++a) {
                double s = 0.0;
                for (int gx = 0; gx < 3; ++gx) s += E[gx + 3 * gy + 9 * gz] * tab.P[gx][a];
                t1[a + 3 * gy + 9 * gz] = s;
              }
          for (int gz = 0; gz < 3; ++gz)
            for (int bb = 0; bb < 3; ++bb)
              for (int a = 0; a < 3; ++a) {
                double s = 0.0;
                for (int gy = 0; gy < 3; ++gy) s += t1[a + 3 * gy + 9 * gz] * tab.P[gy][bb];
                t2[a + 3 * bb + 9 * gz] = s;
              }
          double ku = 0.0;  // (K_e u_e)_l
          for (int c = 0; c < 3; ++c)
            for (int bb = 0; bb < 3; ++bb)
              for (int a = 0; a < 3; ++a) {
                double q = 0.0;
                for (int gz = 0; gz < 3; ++gz) q += t2[a + 3 * bb + 9 * gz] * tab.P[gz][c];
                const double kl = h * (tab.S[la][a] * tab.Mm[lb][bb] * tab.Mm[lc][c] +
                                       tab.Mm[la][a] * tab.S[lb][bb] * tab.Mm[lc][c] +
                                       tab.Mm[la][a] * tab.Mm[lb][bb] * tab.S[lc][c]);
                ku += kl * ue[a + 3 * bb + 9 * c];
                const int gi = 2 * ex + a, gj = 2 * ey + bb, gk = 2 * ez + c;
                const long long slot = ((long long)(gk - c0) * ny + (gj - b0)) * nx + (gi - a0);
                val[start + slot] += -kl + lambda * q;
              }
          bi -= -ku + lambda * rexp;  // b = -R, R_l = -(K u)_l + lambda int exp(u) phi_l
        }
    b[row] = bi;
  }
}

// u += du; *dmax = max |du| (bit pattern of a non-negative double orders like an
// unsigned integer; a NaN orders above every finite value)
__global__ void __launch_bounds__(kThreads)
    k_newton_update(long long N, double* __restrict__ u, const double* __restrict__ du,
                    unsigned long long* __restrict__ dmax) {
  double m = 0.0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N;
       i += (long long)gridDim.x * blockDim.x) {
    const double d = du[i];
    u[i] += d;
    const double a = fabs(d);
    m = (a > m || a != a) ? a : m;
  }
  unsigned long long bits = (unsigned long long)__double_as_longlong(m);
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long ob = __shfl_xor_sync(0xffffffffu, bits, o);
    bits = ob > bits ? ob : bits;
  }
  if ((threadIdx.x & 31) == 0) atomicMax(dmax, bits);
}

struct DevBuf {  // scratch owned by one call
  void* p = nullptr;
  ~DevBuf() {
    if (p) cudaFree(p);
  }
};

}  // namespace

}  // namespace gg

using namespace gg;

extern "C" {

int64_t q2_nnz(int32_t n) {
  if (n < 1) return 0;
  const long long M = 2LL * n + 1, Sx = 8LL * n - 5;
  return M * (4 * M - 4) + Sx * Sx * (Sx + 6);
}

gmres_status q2_bratu_assemble(int32_t n, double lambda, const double* u, int32_t* rowptr,
                               int32_t* col, double* val, double* b, void* stream) {
  if (n < 1 || !rowptr || !col || !val || !b)
    return fail(nullptr, GMRES_ERR_INVALID_ARG, "q2_bratu_assemble: invalid arguments");
  const long long M = 2LL * n + 1, N = M * M * M;
  if (q2_nnz(n) >= (1LL << 31) || N >= (1LL << 31))
    return fail(nullptr, GMRES_ERR_INVALID_ARG, "q2_bratu_assemble: mesh too large for int32 CSR");
  if (!std::isfinite(lambda))
    return fail(nullptr, GMRES_ERR_INVALID_ARG, "q2_bratu_assemble: lambda must be finite");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  k_q2_assemble<<<grid_for(N, 128, 152 * 16), 128, 0, st>>>(n, lambda, u, rowptr, col, val, b);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(nullptr, e, "q2_bratu_assemble");
  return GMRES_OK;
}

gmres_status q2_bratu_newton(int32_t n, double lambda, const gmres_opts* opts,
                             const gmres_defl* W, int32_t m, double tol, int64_t maxit,
                             double newton_tol, int32_t max_newton, double* u,
                             q2_newton_info* info, void* stream) {
  if (n < 1 || !u || max_newton < 1 || !(newton_tol >= 0.0))
    return fail(nullptr, GMRES_ERR_INVALID_ARG, "q2_bratu_newton: invalid arguments");
  const long long M = 2LL * n + 1, N = M * M * M;
  const long long nnz = q2_nnz(n);
  if (nnz >= (1LL << 31) || N >= (1LL << 31))
    return fail(nullptr, GMRES_ERR_INVALID_ARG, "q2_bratu_newton: mesh too large for int32 CSR");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  q2_newton_info inf;
  std::memset(&inf, 0, sizeof(inf));
  inf.status = GMRES_NOT_CONVERGED;
  DevBuf brp, bcol, bval, bb, bdu, bmax;
  const size_t d = sizeof(double);
  cudaError_t e = cudaSuccess;
  if ((e = cudaMalloc(&brp.p, sizeof(int) * (size_t)(N + 1))) != cudaSuccess ||
      (e = cudaMalloc(&bcol.p, sizeof(int) * (size_t)nnz)) != cudaSuccess ||
      (e = cudaMalloc(&bval.p, d * (size_t)nnz)) != cudaSuccess ||
      (e = cudaMalloc(&bb.p, d * (size_t)N)) != cudaSuccess ||
      (e = cudaMalloc(&bdu.p, d * (size_t)N)) != cudaSuccess ||
      (e = cudaMalloc(&bmax.p, sizeof(unsigned long long))) != cudaSuccess)
    return cuda_fail(nullptr, e, "q2_bratu_newton: allocation");
  cudaEvent_t ev[4];
  for (auto& x : ev)
    if ((e = cudaEventCreate(&x)) != cudaSuccess) return cuda_fail(nullptr, e, "q2_bratu_newton");
  auto done = [&](gmres_status s) {
    for (auto& x : ev) cudaEventDestroy(x);
    if (info) *info = inf;
    return s;
  };
  gmres_csr csr{(int32_t)N, nnz, static_cast<int*>(brp.p), static_cast<int*>(bcol.p),
                static_cast<double*>(bval.p)};
  cudaEventRecord(ev[0], st);
  for (int it = 0; it < max_newton; ++it) {
    cudaEventRecord(ev[2], st);
    gmres_status s = q2_bratu_assemble(n, lambda, u, static_cast<int*>(brp.p),
                                       static_cast<int*>(bcol.p), static_cast<double*>(bval.p),
                                       static_cast<double*>(bb.p), stream);
    if (s != GMRES_OK) return done(s);
    cudaEventRecord(ev[3], st);
    gmres_t hs = nullptr;
    s = gmres_create(&hs, &csr, W, opts, stream);
    if (s != GMRES_OK) {
      g_create_error = std::string("q2_bratu_newton: ") + g_create_error;
      return done(s);
    }
    gmres_info gi;
    s = gmres_solve(hs, static_cast<double*>(bb.p), nullptr, m, tol, maxit,
                    static_cast<double*>(bdu.p), &gi);
    if (s != GMRES_OK && s != GMRES_NOT_CONVERGED) {
      g_create_error = std::string("q2_bratu_newton: ") + gmres_last_error(hs);
      gmres_destroy(hs);
      return done(s);
    }
    gmres_destroy(hs);
    float ms_a = 0.f;
    cudaEventSynchronize(ev[3]);
    cudaEventElapsedTime(&ms_a, ev[2], ev[3]);
    inf.ms_assemble += ms_a;
    inf.ms_solve += gi.ms_total;
    inf.gmres_iters += gi.iters;
    inf.last_rel_res = gi.rel_res_true;
    unsigned long long hbits = 0;
    if ((e = cudaMemsetAsync(bmax.p, 0, sizeof(unsigned long long), st)) != cudaSuccess)
      return done(cuda_fail(nullptr, e, "q2_bratu_newton"));
    k_newton_update<<<grid_for(N, kThreads, 152 * 8), kThreads, 0, st>>>(
        N, u, static_cast<double*>(bdu.p), static_cast<unsigned long long*>(bmax.p));
    if ((e = cudaMemcpyAsync(&hbits, bmax.p, sizeof(hbits), cudaMemcpyDeviceToHost, st)) !=
            cudaSuccess ||
        (e = cudaStreamSynchronize(st)) != cudaSuccess)
      return done(cuda_fail(nullptr, e, "q2_bratu_newton"));
    double dn;
    std::memcpy(&dn, &hbits, sizeof(dn));
    if (it < 32) {
      inf.step_iters[it] = gi.iters;
      inf.step_du[it] = dn;
    }
    inf.newton_iters = it + 1;
    inf.du_inf = dn;
    if (!std::isfinite(dn)) {
      inf.status = GMRES_ERR_NAN;
      g_create_error = "q2_bratu_newton: NaN or Inf in the Newton update";
      break;
    }
    if (dn <= newton_tol) {
      inf.status = GMRES_OK;
      break;
    }
  }
  cudaEventRecord(ev[1], st);
  cudaEventSynchronize(ev[1]);
  cudaEventElapsedTime(&inf.ms_total, ev[0], ev[1]);
  return done((gmres_status)inf.status);
}

}  // extern "C"
