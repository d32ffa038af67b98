/*
 * oracle.c -- plain, sequential FP64 CPU oracle for deflated restarted GMRES(m).
 *
 * TEST INFRASTRUCTURE ONLY (tests/, __graft_entry__.smoke(), bench.py's CPU baseline).
 * It shares no code with the CUDA library.  Written for a reader who checks it against
 * the paper (arXiv:1906.04051) by eye: one loop per mathematical operation, FP64 only,
 * no blocking, fusion or reordering.
 */
#include "oracle.h"

#include <float.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------------------------ */
/* Q1 Galerkin finite elements (Sec. 3.1, Eqs. 6-8, written for the bilinear square).   */
/* ------------------------------------------------------------------------------------ */

int64_t orc_q1_nnz(int32_t n) {
  /* interior rows couple to the 3x3 node patch; boundary rows hold only u_i = 0 */
  int64_t interior = (int64_t)(n - 1) * (n - 1);
  int64_t boundary = (int64_t)(n + 1) * (n + 1) - interior;
  return 9 * interior + boundary;
}

void orc_q1_element(double h, double bx, double by, double* K1, double* C, double* M) {
  /* 1-D linear shape functions l0 = 1 - s, l1 = s on [0,1]:
   *   S[a][c] = int l_a' l_c'    Mr[a][c] = int l_a l_c    G[a][c] = int l_a l_c'
   * The 2-D bilinear functions are phi_(a,b) = l_a(x/h) l_b(y/h).  On a square of side
   * h the Jacobian factors cancel in the stiffness, give h for convection, h^2 for mass. */
  const double S[2][2] = {{1.0, -1.0}, {-1.0, 1.0}};
  const double Mr[2][2] = {{1.0 / 3.0, 1.0 / 6.0}, {1.0 / 6.0, 1.0 / 3.0}};
  const double G[2][2] = {{-0.5, 0.5}, {-0.5, 0.5}};
  for (int a = 0; a < 2; ++a)
    for (int b = 0; b < 2; ++b)
      for (int c = 0; c < 2; ++c)
        for (int d = 0; d < 2; ++d) {
          int i = a + 2 * b, j = c + 2 * d;
          K1[4 * i + j] = S[a][c] * Mr[b][d] + Mr[a][c] * S[b][d];
          C[4 * i + j] = h * (bx * G[a][c] * Mr[b][d] + by * Mr[a][c] * G[b][d]);
          M[4 * i + j] = h * h * Mr[a][c] * Mr[b][d];
        }
}

static int is_boundary(int32_t n, int32_t i, int32_t j) {
  return i == 0 || j == 0 || i == n || j == n;
}

int orc_q1_assemble(int32_t n, const double* kappa, double bx, double by, const double* f,
                    const double* u, int32_t* rowptr, int32_t* col, double* val, double* b) {
  const int32_t np = n + 1;
  const int32_t N = np * np;
  /* sparsity pattern: mesh connectivity, node (i,j) -> j*(n+1)+i, columns ascending */
  int64_t pos = 0;
  for (int32_t j = 0; j < np; ++j)
    for (int32_t i = 0; i < np; ++i) {
      int32_t row = j * np + i;
      rowptr[row] = (int32_t)pos;
      if (is_boundary(n, i, j)) {
        col[pos] = row;
        val[pos] = 1.0; /* Dirichlet row replaced by u_i = 0 */
        ++pos;
      } else {
        for (int dj = -1; dj <= 1; ++dj)
          for (int di = -1; di <= 1; ++di) {
            col[pos] = (j + dj) * np + (i + di);
            val[pos] = 0.0;
            ++pos;
          }
      }
    }
  rowptr[N] = (int32_t)pos;
  for (int32_t k = 0; k < N; ++k) b[k] = 0.0;

  double K1[16], C[16], M[16];
  orc_q1_element(1.0 / n, bx, by, K1, C, M);
  /* element loop: scatter K_e = kappa_e K1 + C into interior rows, b += M_e f_e - K_e u_e */
  for (int32_t ej = 0; ej < n; ++ej)
    for (int32_t ei = 0; ei < n; ++ei) {
      double ke = kappa[ej * n + ei];
      int32_t gi[4], ii[4], jj[4];
      for (int l = 0; l < 4; ++l) {
        ii[l] = ei + (l & 1);
        jj[l] = ej + (l >> 1);
        gi[l] = jj[l] * np + ii[l];
      }
      for (int a = 0; a < 4; ++a) {
        if (is_boundary(n, ii[a], jj[a])) continue;
        int32_t row = gi[a];
        for (int c = 0; c < 4; ++c) {
          double kac = ke * K1[4 * a + c] + C[4 * a + c];
          int32_t k;
          for (k = rowptr[row]; k < rowptr[row + 1]; ++k)
            if (col[k] == gi[c]) break;
          val[k] += kac;
          b[row] += M[4 * a + c] * f[gi[c]];
          if (u) b[row] -= kac * u[gi[c]];
        }
      }
    }
  return 0;
}

void orc_q1_kappa_grad(int32_t n, const double* lam, const double* x, double* grad) {
  /* A depends on kappa_e only through the interior rows of element e: dA/dkappa_e = K1
   * scattered into those rows; b does not depend on kappa.  dL/dkappa_e = -lam^T dA x. */
  const int32_t np = n + 1;
  double K1[16], C[16], M[16];
  orc_q1_element(1.0 / n, 0.0, 0.0, K1, C, M);
  for (int32_t ej = 0; ej < n; ++ej)
    for (int32_t ei = 0; ei < n; ++ei) {
      double g = 0.0;
      for (int a = 0; a < 4; ++a) {
        int32_t ia = ei + (a & 1), ja = ej + (a >> 1);
        if (is_boundary(n, ia, ja)) continue;
        double kx = 0.0;
        for (int c = 0; c < 4; ++c) {
          int32_t ic = ei + (c & 1), jc = ej + (c >> 1);
          kx += K1[4 * a + c] * x[jc * np + ic];
        }
        g += lam[ja * np + ia] * kx;
      }
      grad[ej * n + ei] = -g;
    }
}

/* ------------------------------------------------------------------------------------ */
/* Sparse and dense building blocks                                                      */
/* ------------------------------------------------------------------------------------ */

/* ------------------------------------------------------------------------------------ */
/* 3-D Bratu problem on 27-node triquadratic hexahedra (Sec. 3.1, Eqs. 2-9)              */
/* ------------------------------------------------------------------------------------ */

/* Nodes per direction M = 2n + 1; node (I, J, K) -> (K M + J) M + I.  Along one
 * direction a vertex node (even index) shares elements with the nodes within 2 of it,
 * a mid-edge node (odd index) only with those within 1. */
static void q2_range(int32_t M, int32_t I, int32_t* lo, int32_t* hi) {
  const int32_t r = (I % 2 == 0) ? 2 : 1;
  *lo = I - r < 0 ? 0 : I - r;
  *hi = I + r > M - 1 ? M - 1 : I + r;
}

static int q2_dirichlet(int32_t M, int32_t I, int32_t J) {
  return I == 0 || J == 0 || I == M - 1 || J == M - 1; /* x- and y-faces (Eqs. 3-4) */
}

int64_t orc_q2_nnz(int32_t n) {
  const int32_t M = 2 * n + 1;
  int64_t nnz = 0;
  for (int32_t K = 0; K < M; ++K)
    for (int32_t J = 0; J < M; ++J)
      for (int32_t I = 0; I < M; ++I) {
        if (q2_dirichlet(M, I, J)) {
          nnz += 1;
          continue;
        }
        int32_t a0, a1, b0, b1, c0, c1;
        q2_range(M, I, &a0, &a1);
        q2_range(M, J, &b0, &b1);
        q2_range(M, K, &c0, &c1);
        nnz += (int64_t)(a1 - a0 + 1) * (b1 - b0 + 1) * (c1 - c0 + 1);
      }
  return nnz;
}

void orc_q2_element(double h, double lambda, const double* ue, double* Je, double* Re) {
  /* Element of side h, local node l = a + 3 b + 9 c (a, b, c in {0, 1, 2} along x, y, z).
   * 1-D quadratic Lagrange functions on [0,1] with nodes 0, 1/2, 1:
   *   p0 = (1 - s)(1 - 2 s), p1 = 4 s (1 - s), p2 = s (2 s - 1).
   * R_e[l] = - int grad(u_h) . grad(phi_l) + lambda int exp(u_h) phi_l        (Eq. 7)
   * J_e[l][m] = dR_e[l]/du_m = - int grad(phi_m) . grad(phi_l)
   *                            + lambda int exp(u_h) phi_m phi_l               (Eq. 9)
   * integrated by the 3 x 3 x 3 Gauss-Legendre rule (exact for the polynomial parts). */
  const double gs = sqrt(0.6);
  const double xg[3] = {0.5 * (1.0 - gs), 0.5, 0.5 * (1.0 + gs)};
  const double wg[3] = {5.0 / 18.0, 8.0 / 18.0, 5.0 / 18.0};
  double P[3][3], D[3][3]; /* P[g][a] = p_a(x_g), D[g][a] = p_a'(x_g) */
  for (int g = 0; g < 3; ++g) {
    const double t = xg[g];
    P[g][0] = (1.0 - t) * (1.0 - 2.0 * t);
    P[g][1] = 4.0 * t * (1.0 - t);
    P[g][2] = t * (2.0 * t - 1.0);
    D[g][0] = 4.0 * t - 3.0;
    D[g][1] = 4.0 - 8.0 * t;
    D[g][2] = 4.0 * t - 1.0;
  }
  for (int l = 0; l < 27 * 27; ++l) Je[l] = 0.0;
  for (int l = 0; l < 27; ++l) Re[l] = 0.0;
  for (int gz = 0; gz < 3; ++gz)
    for (int gy = 0; gy < 3; ++gy)
      for (int gx = 0; gx < 3; ++gx) {
        const double w = wg[gx] * wg[gy] * wg[gz] * h * h * h;
        double phi[27], dx[27], dy[27], dz[27];
        for (int c = 0; c < 3; ++c)
          for (int b = 0; b < 3; ++b)
            for (int a = 0; a < 3; ++a) {
              const int l = a + 3 * b + 9 * c;
              phi[l] = P[gx][a] * P[gy][b] * P[gz][c];
              dx[l] = D[gx][a] * P[gy][b] * P[gz][c] / h;
              dy[l] = P[gx][a] * D[gy][b] * P[gz][c] / h;
              dz[l] = P[gx][a] * P[gy][b] * D[gz][c] / h;
            }
        double ug = 0.0, ux = 0.0, uy = 0.0, uz = 0.0;
        for (int l = 0; l < 27; ++l) {
          const double v = ue ? ue[l] : 0.0;
          ug += v * phi[l];
          ux += v * dx[l];
          uy += v * dy[l];
          uz += v * dz[l];
        }
        const double eg = exp(ug);
        for (int l = 0; l < 27; ++l) {
          Re[l] += w * (-(ux * dx[l] + uy * dy[l] + uz * dz[l]) + lambda * eg * phi[l]);
          for (int m = 0; m < 27; ++m)
            Je[l * 27 + m] += w * (-(dx[m] * dx[l] + dy[m] * dy[l] + dz[m] * dz[l]) +
                                   lambda * eg * phi[m] * phi[l]);
        }
      }
}

int orc_q2_bratu_assemble(int32_t n, double lambda, const double* u, int32_t* rowptr,
                          int32_t* col, double* val, double* b) {
  const int32_t M = 2 * n + 1;
  const int32_t N = M * M * M;
  /* pattern: mesh connectivity, columns ascending; Dirichlet rows hold du_i = 0 (Sec. 3.1) */
  int64_t pos = 0;
  for (int32_t K = 0; K < M; ++K)
    for (int32_t J = 0; J < M; ++J)
      for (int32_t I = 0; I < M; ++I) {
        const int32_t row = (K * M + J) * M + I;
        rowptr[row] = (int32_t)pos;
        if (q2_dirichlet(M, I, J)) {
          col[pos] = row;
          val[pos] = 1.0;
          ++pos;
          continue;
        }
        int32_t a0, a1, b0, b1, c0, c1;
        q2_range(M, I, &a0, &a1);
        q2_range(M, J, &b0, &b1);
        q2_range(M, K, &c0, &c1);
        for (int32_t k = c0; k <= c1; ++k)
          for (int32_t j = b0; j <= b1; ++j)
            for (int32_t i = a0; i <= a1; ++i) {
              col[pos] = (k * M + j) * M + i;
              val[pos] = 0.0;
              ++pos;
            }
      }
  rowptr[N] = (int32_t)pos;
  for (int32_t r = 0; r < N; ++r) b[r] = 0.0;
  /* element loop: J = sum_e J_e, b = -R = -sum_e R_e on the rows that are not Dirichlet */
  double Je[27 * 27], Re[27], ue[27];
  int32_t gid[27];
  int dir[27];
  for (int32_t ez = 0; ez < n; ++ez)
    for (int32_t ey = 0; ey < n; ++ey)
      for (int32_t ex = 0; ex < n; ++ex) {
        for (int c = 0; c < 3; ++c)
          for (int bb = 0; bb < 3; ++bb)
            for (int a = 0; a < 3; ++a) {
              const int l = a + 3 * bb + 9 * c;
              const int32_t I = 2 * ex + a, J = 2 * ey + bb, K = 2 * ez + c;
              gid[l] = (K * M + J) * M + I;
              dir[l] = q2_dirichlet(M, I, J);
              ue[l] = u ? u[gid[l]] : 0.0;
            }
        orc_q2_element(1.0 / n, lambda, ue, Je, Re);
        for (int l = 0; l < 27; ++l) {
          if (dir[l]) continue;
          const int32_t row = gid[l];
          b[row] -= Re[l];
          for (int m = 0; m < 27; ++m) {
            int32_t lo = rowptr[row], hi = rowptr[row + 1] - 1; /* binary search */
            while (lo < hi) {
              const int32_t mid = (lo + hi) / 2;
              if (col[mid] < gid[m]) lo = mid + 1;
              else hi = mid;
            }
            val[lo] += Je[l * 27 + m];
          }
        }
      }
  return 0;
}

void orc_spmv(int32_t N, const int32_t* rowptr, const int32_t* col, const double* val,
              const double* x, double* y) {
  for (int32_t i = 0; i < N; ++i) {
    double s = 0.0;
    for (int32_t k = rowptr[i]; k < rowptr[i + 1]; ++k) s += val[k] * x[col[k]];
    y[i] = s;
  }
}

void orc_transpose(int32_t N, const int32_t* rowptr, const int32_t* col, const double* val,
                   int32_t* rowptr_t, int32_t* col_t, double* val_t) {
  for (int32_t i = 0; i <= N; ++i) rowptr_t[i] = 0;
  for (int32_t k = 0; k < rowptr[N]; ++k) rowptr_t[col[k] + 1]++;
  for (int32_t i = 0; i < N; ++i) rowptr_t[i + 1] += rowptr_t[i];
  int32_t* next = (int32_t*)malloc(sizeof(int32_t) * (size_t)(N > 0 ? N : 1));
  for (int32_t i = 0; i < N; ++i) next[i] = rowptr_t[i];
  /* rows visited in ascending order, so every transposed row comes out sorted */
  for (int32_t i = 0; i < N; ++i)
    for (int32_t k = rowptr[i]; k < rowptr[i + 1]; ++k) {
      int32_t p = next[col[k]]++;
      col_t[p] = i;
      val_t[p] = val[k];
    }
  free(next);
}

static double dot(const double* a, const double* b, int32_t n) {
  double s = 0.0;
  for (int32_t i = 0; i < n; ++i) s += a[i] * b[i];
  return s;
}

static double nrm2(const double* a, int32_t n) { return sqrt(dot(a, a, n)); }

int orc_lu_factor(int32_t n, double* a, int32_t* piv) {
  /* Gaussian elimination with partial pivoting (outer-product form) */
  for (int32_t k = 0; k < n; ++k) {
    int32_t p = k;
    for (int32_t i = k + 1; i < n; ++i)
      if (fabs(a[(size_t)i * n + k]) > fabs(a[(size_t)p * n + k])) p = i;
    piv[k] = p;
    if (a[(size_t)p * n + k] == 0.0) return k + 1;
    if (p != k)
      for (int32_t j = 0; j < n; ++j) {
        double t = a[(size_t)k * n + j];
        a[(size_t)k * n + j] = a[(size_t)p * n + j];
        a[(size_t)p * n + j] = t;
      }
    for (int32_t i = k + 1; i < n; ++i) {
      double l = a[(size_t)i * n + k] / a[(size_t)k * n + k];
      a[(size_t)i * n + k] = l;
      for (int32_t j = k + 1; j < n; ++j) a[(size_t)i * n + j] -= l * a[(size_t)k * n + j];
    }
  }
  return 0;
}

void orc_lu_solve(int32_t n, const double* lu, const int32_t* piv, double* b) {
  for (int32_t k = 0; k < n; ++k)
    if (piv[k] != k) {
      double t = b[k];
      b[k] = b[piv[k]];
      b[piv[k]] = t;
    }
  for (int32_t i = 0; i < n; ++i)
    for (int32_t j = 0; j < i; ++j) b[i] -= lu[(size_t)i * n + j] * b[j];
  for (int32_t i = n - 1; i >= 0; --i) {
    for (int32_t j = i + 1; j < n; ++j) b[i] -= lu[(size_t)i * n + j] * b[j];
    b[i] /= lu[(size_t)i * n + i];
  }
}

/* Eigenvalues of the 2x2 block [[a, b], [c, d]]. */
static void eig2(double a, double b, double c, double d, double* r1, double* i1, double* r2,
                 double* i2) {
  double p = 0.5 * (a - d);
  double disc = p * p + b * c;
  double mid = 0.5 * (a + d);
  if (disc >= 0.0) {
    double q = sqrt(disc);
    double l1 = mid + (p >= 0.0 ? q : -q);
    double det = a * d - b * c;
    double l2 = (l1 != 0.0) ? det / l1 : mid - (p >= 0.0 ? q : -q);
    *r1 = l1; *i1 = 0.0;
    *r2 = l2; *i2 = 0.0;
  } else {
    double q = sqrt(-disc);
    *r1 = mid; *i1 = q;
    *r2 = mid; *i2 = -q;
  }
}

int orc_hessenberg_eigs(int32_t n, const double* h, double* wr, double* wi) {
  /* Francis double-shift QR iteration (implicit, with bulge chasing by 3x3 Householder
   * reflectors), deflating at negligible subdiagonals.  Only the active diagonal block
   * is transformed: the eigenvalues alone are wanted. */
  double* a = (double*)malloc(sizeof(double) * (size_t)n * n);
  memcpy(a, h, sizeof(double) * (size_t)n * n);
#define A(i, j) a[(size_t)(i) * n + (j)]
  double anorm = 0.0;
  for (int32_t i = 0; i < n; ++i)
    for (int32_t j = (i > 0 ? i - 1 : 0); j < n; ++j) anorm += fabs(A(i, j));
  int32_t hi = n - 1;
  int its = 0, total = 0;
  while (hi >= 0) {
    int32_t l;
    for (l = hi; l > 0; --l) {
      double s = fabs(A(l - 1, l - 1)) + fabs(A(l, l));
      if (s == 0.0) s = anorm;
      if (fabs(A(l, l - 1)) <= DBL_EPSILON * s) {
        A(l, l - 1) = 0.0;
        break;
      }
    }
    if (l == hi) {
      wr[hi] = A(hi, hi);
      wi[hi] = 0.0;
      --hi;
      its = 0;
      continue;
    }
    if (l == hi - 1) {
      eig2(A(hi - 1, hi - 1), A(hi - 1, hi), A(hi, hi - 1), A(hi, hi), &wr[hi - 1], &wi[hi - 1],
           &wr[hi], &wi[hi]);
      hi -= 2;
      its = 0;
      continue;
    }
    if (++total > 60 * n) {
      free(a);
      return -1;
    }
    /* shifts: the eigenvalues of the trailing 2x2 block, as the roots of x^2 - s x + t;
     * an exceptional shift breaks rare cycles after 10 and 20 sweeps without deflation */
    double s, t;
    if (its == 10 || its == 20) {
      double w = fabs(A(hi, hi - 1)) + fabs(A(hi - 1, hi - 2));
      double sig = A(hi, hi) + 0.75 * w;
      s = 2.0 * sig;
      t = sig * sig;
    } else {
      s = A(hi - 1, hi - 1) + A(hi, hi);
      t = A(hi - 1, hi - 1) * A(hi, hi) - A(hi - 1, hi) * A(hi, hi - 1);
    }
    ++its;
    /* first column of (H - s1 I)(H - s2 I) restricted to the block */
    double x = A(l, l) * A(l, l) + A(l, l + 1) * A(l + 1, l) - s * A(l, l) + t;
    double y = A(l + 1, l) * (A(l, l) + A(l + 1, l + 1) - s);
    double z = A(l + 1, l) * A(l + 2, l + 1);
    for (int32_t k = l; k <= hi - 2; ++k) {
      double nrm = sqrt(x * x + y * y + z * z);
      if (nrm != 0.0) {
        double alpha = (x >= 0.0) ? -nrm : nrm; /* reflector maps (x,y,z) to alpha e1 */
        double v0 = x - alpha, v1 = y, v2 = z;
        double beta = 2.0 / (v0 * v0 + v1 * v1 + v2 * v2);
        int32_t c0 = (k > l) ? k - 1 : l;
        for (int32_t j = c0; j <= hi; ++j) {
          double dd = beta * (v0 * A(k, j) + v1 * A(k + 1, j) + v2 * A(k + 2, j));
          A(k, j) -= dd * v0;
          A(k + 1, j) -= dd * v1;
          A(k + 2, j) -= dd * v2;
        }
        if (k > l) {
          A(k + 1, k - 1) = 0.0;
          A(k + 2, k - 1) = 0.0;
        }
        int32_t r1 = (k + 3 < hi) ? k + 3 : hi;
        for (int32_t i = l; i <= r1; ++i) {
          double dd = beta * (A(i, k) * v0 + A(i, k + 1) * v1 + A(i, k + 2) * v2);
          A(i, k) -= dd * v0;
          A(i, k + 1) -= dd * v1;
          A(i, k + 2) -= dd * v2;
        }
      }
      x = A(k + 1, k);
      y = A(k + 2, k);
      if (k < hi - 2) z = A(k + 3, k);
    }
    /* last reflector acts on rows/columns hi-1, hi */
    double nrm = sqrt(x * x + y * y);
    if (nrm != 0.0) {
      double alpha = (x >= 0.0) ? -nrm : nrm;
      double v0 = x - alpha, v1 = y;
      double beta = 2.0 / (v0 * v0 + v1 * v1);
      int32_t c0 = (hi - 2 > l) ? hi - 2 : l;
      for (int32_t j = c0; j <= hi; ++j) {
        double dd = beta * (v0 * A(hi - 1, j) + v1 * A(hi, j));
        A(hi - 1, j) -= dd * v0;
        A(hi, j) -= dd * v1;
      }
      if (hi - 2 >= l) A(hi, hi - 2) = 0.0;
      for (int32_t i = l; i <= hi; ++i) {
        double dd = beta * (A(i, hi - 1) * v0 + A(i, hi) * v1);
        A(i, hi - 1) -= dd * v0;
        A(i, hi) -= dd * v1;
      }
    }
  }
#undef A
  free(a);
  return 0;
}

/* ------------------------------------------------------------------------------------ */
/* Deflation preconditioner (Sec. 3.3, Eqs. 17-18)                                       */
/* ------------------------------------------------------------------------------------ */

struct orc_defl {
  int32_t N, r;
  const int32_t *rowptr, *col;
  const double* val;
  int32_t* agg;     /* copy of the aggregate map */
  double* uscale;   /* 1/sqrt|agg_p|: U = W diag(uscale) has orthonormal columns */
  double* T;        /* U^T A U, r x r row-major */
  double* lu;       /* LU of T */
  int32_t* piv;
};

static void defl_Ut(const orc_defl* d, const double* v, double* c) { /* c = U^T v */
  for (int32_t p = 0; p < d->r; ++p) c[p] = 0.0;
  for (int32_t i = 0; i < d->N; ++i)
    if (d->agg[i] >= 0) c[d->agg[i]] += v[i];
  for (int32_t p = 0; p < d->r; ++p) c[p] *= d->uscale[p];
}

static void defl_U_add(const orc_defl* d, const double* y, double* v) { /* v += U y */
  for (int32_t i = 0; i < d->N; ++i)
    if (d->agg[i] >= 0) v[i] += d->uscale[d->agg[i]] * y[d->agg[i]];
}

orc_defl* orc_defl_create(int32_t N, const int32_t* rowptr, const int32_t* col,
                          const double* val, int32_t r, const int32_t* agg, int* err) {
  *err = 0;
  orc_defl* d = (orc_defl*)calloc(1, sizeof(orc_defl));
  d->N = N;
  d->r = r;
  d->rowptr = rowptr;
  d->col = col;
  d->val = val;
  d->agg = (int32_t*)malloc(sizeof(int32_t) * (size_t)N);
  memcpy(d->agg, agg, sizeof(int32_t) * (size_t)N);
  d->uscale = (double*)calloc((size_t)r, sizeof(double));
  int64_t* count = (int64_t*)calloc((size_t)r, sizeof(int64_t));
  for (int32_t i = 0; i < N; ++i)
    if (agg[i] >= 0) count[agg[i]]++;
  for (int32_t p = 0; p < r; ++p) {
    if (count[p] == 0) *err = -4; /* a zero column of W */
    d->uscale[p] = count[p] > 0 ? 1.0 / sqrt((double)count[p]) : 0.0;
  }
  free(count);
  d->T = (double*)calloc((size_t)r * r, sizeof(double));
  d->lu = (double*)malloc(sizeof(double) * (size_t)r * r);
  d->piv = (int32_t*)malloc(sizeof(int32_t) * (size_t)r);
  if (*err) {
    orc_defl_destroy(d);
    return NULL;
  }
  /* T = U^T A U: entry (p,q) sums a_ij over i in p, j in q, scaled by uscale_p uscale_q */
  for (int32_t i = 0; i < N; ++i) {
    int32_t p = agg[i];
    if (p < 0) continue;
    for (int32_t k = rowptr[i]; k < rowptr[i + 1]; ++k) {
      int32_t q = agg[col[k]];
      if (q < 0) continue;
      d->T[(size_t)p * r + q] += val[k] * d->uscale[p] * d->uscale[q];
    }
  }
  memcpy(d->lu, d->T, sizeof(double) * (size_t)r * r);
  if (orc_lu_factor(r, d->lu, d->piv) != 0) {
    *err = -4;
    orc_defl_destroy(d);
    return NULL;
  }
  return d;
}

void orc_defl_destroy(orc_defl* d) {
  if (!d) return;
  free(d->agg);
  free(d->uscale);
  free(d->T);
  free(d->lu);
  free(d->piv);
  free(d);
}

void orc_defl_T(const orc_defl* d, double* T) {
  memcpy(T, d->T, sizeof(double) * (size_t)d->r * d->r);
}

void orc_defl_apply_Minv(const orc_defl* d, double mu, const double* v, double* z) {
  /* z = M^-1 v = v + U (|mu| T^-1 - I) U^T v   (Eq. 17) */
  double* c = (double*)malloc(sizeof(double) * (size_t)d->r);
  double* y = (double*)malloc(sizeof(double) * (size_t)d->r);
  defl_Ut(d, v, c);
  memcpy(y, c, sizeof(double) * (size_t)d->r);
  orc_lu_solve(d->r, d->lu, d->piv, y); /* y = T^-1 c */
  for (int32_t p = 0; p < d->r; ++p) y[p] = fabs(mu) * y[p] - c[p];
  memcpy(z, v, sizeof(double) * (size_t)d->N);
  defl_U_add(d, y, z);
  free(c);
  free(y);
}

void orc_defl_apply_P(const orc_defl* d, const double* w, double* out) {
  /* out = P w = w - A U T^-1 U^T w, the deflation projector with E = W^T A W taken in
   * the orthonormal basis U of span(W) (P does not depend on that basis). */
  double* c = (double*)malloc(sizeof(double) * (size_t)d->r);
  double* t = (double*)calloc((size_t)d->N, sizeof(double));
  double* at = (double*)malloc(sizeof(double) * (size_t)d->N);
  defl_Ut(d, w, c);
  orc_lu_solve(d->r, d->lu, d->piv, c);
  defl_U_add(d, c, t);
  orc_spmv(d->N, d->rowptr, d->col, d->val, t, at);
  for (int32_t i = 0; i < d->N; ++i) out[i] = w[i] - at[i];
  free(c);
  free(t);
  free(at);
}

/* ------------------------------------------------------------------------------------ */
/* Adaptive deflation (Sec. 3.3, Eq. 19): U grows by eigenvectors of H_m mapped through V */
/* ------------------------------------------------------------------------------------ */

/* LU of a k x k upper Hessenberg matrix (row-major, in place): column j only has rows j
 * and j+1 below the diagonal, so partial pivoting compares those two rows. */
static void hess_lu(int32_t k, double* a, int32_t* sw, double* l, double eps) {
  for (int32_t j = 0; j < k; ++j) {
    sw[j] = 0;
    l[j] = 0.0;
    if (j + 1 < k && fabs(a[(size_t)(j + 1) * k + j]) > fabs(a[(size_t)j * k + j])) {
      for (int32_t c = j; c < k; ++c) {
        double t = a[(size_t)j * k + c];
        a[(size_t)j * k + c] = a[(size_t)(j + 1) * k + c];
        a[(size_t)(j + 1) * k + c] = t;
      }
      sw[j] = 1;
    }
    if (a[(size_t)j * k + j] == 0.0) a[(size_t)j * k + j] = eps;
    if (j + 1 < k) {
      l[j] = a[(size_t)(j + 1) * k + j] / a[(size_t)j * k + j];
      for (int32_t c = j + 1; c < k; ++c) a[(size_t)(j + 1) * k + c] -= l[j] * a[(size_t)j * k + c];
      a[(size_t)(j + 1) * k + j] = 0.0;
    }
  }
}

static void hess_solve(int32_t k, const double* a, const int32_t* sw, const double* l, double* z) {
  for (int32_t j = 0; j + 1 < k; ++j) {
    if (sw[j]) {
      double t = z[j];
      z[j] = z[j + 1];
      z[j + 1] = t;
    }
    z[j + 1] -= l[j] * z[j];
  }
  for (int32_t i = k - 1; i >= 0; --i) {
    double s = z[i];
    for (int32_t c = i + 1; c < k; ++c) s -= a[(size_t)i * k + c] * z[c];
    z[i] = s / a[(size_t)i * k + i];
  }
}

static void normalise_sign(int32_t k, double* z) {
  double nz = nrm2(z, k);
  for (int32_t i = 0; i < k; ++i) z[i] /= nz;
  int32_t im = 0;
  for (int32_t i = 1; i < k; ++i)
    if (fabs(z[i]) > fabs(z[im])) im = i;
  if (z[im] < 0.0)
    for (int32_t i = 0; i < k; ++i) z[i] = -z[i];
}

int orc_hess_invvec(int32_t k, const double* H, int32_t ninv, double* z1, double* z2) {
  if (k < 1) return 0;
  double* a = (double*)malloc(sizeof(double) * (size_t)k * k);
  double* l = (double*)malloc(sizeof(double) * (size_t)k);
  int32_t* sw = (int32_t*)malloc(sizeof(int32_t) * (size_t)k);
  double* hz = (double*)malloc(sizeof(double) * (size_t)k);
  double hmax = 0.0;
  for (int32_t i = 0; i < k * k; ++i) hmax = fabs(H[i]) > hmax ? fabs(H[i]) : hmax;
  memcpy(a, H, sizeof(double) * (size_t)k * k);
  hess_lu(k, a, sw, l, hmax > 0.0 ? 1e-14 * hmax : 1e-300);
  for (int32_t i = 0; i < k; ++i) z1[i] = 1.0 / sqrt((double)k);
  for (int32_t it = 0; it < ninv; ++it) {
    hess_solve(k, a, sw, l, z1);
    normalise_sign(k, z1);
  }
  /* eigenvector test with the Rayleigh quotient rho = z^T H z */
  double rho = 0.0, nhz = 0.0, res = 0.0;
  for (int32_t i = 0; i < k; ++i) {
    double s = 0.0;
    for (int32_t c = 0; c < k; ++c) s += H[(size_t)i * k + c] * z1[c];
    hz[i] = s;
    rho += z1[i] * s;
    nhz += s * s;
  }
  for (int32_t i = 0; i < k; ++i) res += (hz[i] - rho * z1[i]) * (hz[i] - rho * z1[i]);
  int nvec = 1;
  if (sqrt(res) > 1e-3 * sqrt(nhz)) {
    /* a complex pair: the next iterate completes a basis of its invariant subspace */
    memcpy(z2, z1, sizeof(double) * (size_t)k);
    hess_solve(k, a, sw, l, z2);
    double c = dot(z1, z2, k);
    for (int32_t i = 0; i < k; ++i) z2[i] -= c * z1[i];
    normalise_sign(k, z2);
    nvec = 2;
  }
  free(a);
  free(l);
  free(sw);
  free(hz);
  return nvec;
}

/* Reduction of a general n x n matrix (row-major, in place) to upper Hessenberg form by
 * Householder similarity transformations; the eigenvalues are unchanged. */
static void hessenberg_reduce(int32_t n, double* a) {
  double* v = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
  for (int32_t k = 0; k + 2 < n; ++k) {
    const int32_t len = n - k - 1;
    double nx = 0.0;
    for (int32_t i = 0; i < len; ++i) nx += a[(size_t)(k + 1 + i) * n + k] * a[(size_t)(k + 1 + i) * n + k];
    nx = sqrt(nx);
    if (nx == 0.0) continue;
    const double x0 = a[(size_t)(k + 1) * n + k];
    const double alpha = x0 >= 0.0 ? -nx : nx;
    double vv = 0.0;
    for (int32_t i = 0; i < len; ++i) {
      v[i] = a[(size_t)(k + 1 + i) * n + k] - (i == 0 ? alpha : 0.0);
      vv += v[i] * v[i];
    }
    if (vv == 0.0) continue;
    const double beta = 2.0 / vv;
    for (int32_t j = 0; j < n; ++j) { /* rows k+1.. : (I - beta v v^T) A */
      double s = 0.0;
      for (int32_t i = 0; i < len; ++i) s += v[i] * a[(size_t)(k + 1 + i) * n + j];
      for (int32_t i = 0; i < len; ++i) a[(size_t)(k + 1 + i) * n + j] -= beta * s * v[i];
    }
    for (int32_t i = 0; i < n; ++i) { /* columns k+1.. : A (I - beta v v^T) */
      double s = 0.0;
      for (int32_t j = 0; j < len; ++j) s += a[(size_t)i * n + k + 1 + j] * v[j];
      for (int32_t j = 0; j < len; ++j) a[(size_t)i * n + k + 1 + j] -= beta * s * v[j];
    }
    a[(size_t)(k + 1) * n + k] = alpha;
    for (int32_t i = k + 2; i < n; ++i) a[(size_t)i * n + k] = 0.0;
  }
  free(v);
}

int orc_adapt_drop(int32_t q, const double* T, int32_t ldt, double* Qc, double* Tn) {
  if (q < 1) return -1;
  double* h = (double*)malloc(sizeof(double) * (size_t)q * q);
  double* wr = (double*)malloc(sizeof(double) * (size_t)q);
  double* wi = (double*)malloc(sizeof(double) * (size_t)q);
  for (int32_t i = 0; i < q; ++i)
    for (int32_t j = 0; j < q; ++j) h[(size_t)i * q + j] = T[(size_t)i * ldt + j];
  hessenberg_reduce(q, h);
  const int e = orc_hessenberg_eigs(q, h, wr, wi);
  free(h);
  if (e != 0) {
    free(wr);
    free(wi);
    return -1;
  }
  /* the eigenvalue of largest modulus (the first one on ties), a + i b with b >= 0 */
  int32_t best = 0;
  double bmod = -1.0;
  for (int32_t i = 0; i < q; ++i) {
    const double md = hypot(wr[i], wi[i]);
    if (md > bmod) {
      bmod = md;
      best = i;
    }
  }
  const double la = wr[best], lb = fabs(wi[best]);
  free(wr);
  free(wi);
  const int32_t p = lb != 0.0 ? 2 : 1;
  /* left eigenvector y (T^T y = lambda y) by inverse iteration on the real form of
   * T^T - lambda I: [[T^T - a I, b I], [-b I, T^T - a I]] [y_r; y_i] = rhs */
  const int32_t n2 = p * q;
  double* M = (double*)calloc((size_t)n2 * n2, sizeof(double));
  for (int32_t i = 0; i < q; ++i)
    for (int32_t j = 0; j < q; ++j) {
      const double tv = T[(size_t)j * ldt + i] - (i == j ? la : 0.0);
      M[(size_t)i * n2 + j] = tv;
      if (p == 2) M[(size_t)(q + i) * n2 + q + j] = tv;
    }
  if (p == 2)
    for (int32_t i = 0; i < q; ++i) {
      M[(size_t)i * n2 + q + i] = lb;
      M[(size_t)(q + i) * n2 + i] = -lb;
    }
  double mmax = 0.0;
  for (int32_t i = 0; i < n2 * n2; ++i) mmax = fabs(M[i]) > mmax ? fabs(M[i]) : mmax;
  const double eps = mmax > 0.0 ? 1e-14 * mmax : 1e-300;
  int32_t* piv = (int32_t*)malloc(sizeof(int32_t) * (size_t)n2);
  for (int32_t k = 0; k < n2; ++k) { /* LU, partial pivoting; a tiny pivot becomes eps */
    int32_t pr = k;
    for (int32_t i = k + 1; i < n2; ++i)
      if (fabs(M[(size_t)i * n2 + k]) > fabs(M[(size_t)pr * n2 + k])) pr = i;
    piv[k] = pr;
    if (pr != k)
      for (int32_t j = 0; j < n2; ++j) {
        const double t = M[(size_t)k * n2 + j];
        M[(size_t)k * n2 + j] = M[(size_t)pr * n2 + j];
        M[(size_t)pr * n2 + j] = t;
      }
    if (fabs(M[(size_t)k * n2 + k]) <= eps) M[(size_t)k * n2 + k] = eps;
    for (int32_t i = k + 1; i < n2; ++i) {
      const double l = M[(size_t)i * n2 + k] / M[(size_t)k * n2 + k];
      M[(size_t)i * n2 + k] = l;
      for (int32_t j = k + 1; j < n2; ++j) M[(size_t)i * n2 + j] -= l * M[(size_t)k * n2 + j];
    }
  }
  double* y = (double*)malloc(sizeof(double) * (size_t)n2);
  for (int32_t i = 0; i < n2; ++i) y[i] = 1.0;
  for (int it = 0; it < 3; ++it) {
    orc_lu_solve(n2, M, piv, y);
    const double ny = nrm2(y, n2);
    for (int32_t i = 0; i < n2; ++i) y[i] /= ny;
  }
  free(M);
  free(piv);
  /* Householder QR of Y = [y_r (, y_i)]: Q = H_0 ... H_{p-1}; the last q - p columns of
   * Q are an orthonormal basis of the vectors c with y^T c = 0 */
  double* Y = (double*)malloc(sizeof(double) * (size_t)q * p);
  double* hv = (double*)calloc((size_t)q * p, sizeof(double));
  double hb[2] = {0.0, 0.0};
  for (int32_t i = 0; i < q; ++i)
    for (int32_t c = 0; c < p; ++c) Y[(size_t)i * p + c] = y[(size_t)c * q + i];
  for (int32_t c = 0; c < p; ++c) {
    double nx = 0.0;
    for (int32_t i = c; i < q; ++i) nx += Y[(size_t)i * p + c] * Y[(size_t)i * p + c];
    nx = sqrt(nx);
    const double x0 = Y[(size_t)c * p + c];
    const double alpha = x0 >= 0.0 ? -nx : nx;
    double vv = 0.0;
    for (int32_t i = c; i < q; ++i) {
      hv[(size_t)c * q + i] = Y[(size_t)i * p + c] - (i == c ? alpha : 0.0);
      vv += hv[(size_t)c * q + i] * hv[(size_t)c * q + i];
    }
    hb[c] = vv > 0.0 ? 2.0 / vv : 0.0;
    for (int32_t c2 = c + 1; c2 < p; ++c2) {
      double sd = 0.0;
      for (int32_t i = c; i < q; ++i) sd += hv[(size_t)c * q + i] * Y[(size_t)i * p + c2];
      for (int32_t i = c; i < q; ++i) Y[(size_t)i * p + c2] -= hb[c] * sd * hv[(size_t)c * q + i];
    }
  }
  const int32_t nc = q - p;
  for (int32_t i = 0; i < q; ++i)
    for (int32_t c = 0; c < nc; ++c) Qc[(size_t)i * nc + c] = (i == p + c) ? 1.0 : 0.0;
  for (int32_t c = p - 1; c >= 0; --c)
    for (int32_t j = 0; j < nc; ++j) {
      double sd = 0.0;
      for (int32_t i = c; i < q; ++i) sd += hv[(size_t)c * q + i] * Qc[(size_t)i * nc + j];
      for (int32_t i = c; i < q; ++i) Qc[(size_t)i * nc + j] -= hb[c] * sd * hv[(size_t)c * q + i];
    }
  free(Y);
  free(hv);
  free(y);
  /* Tn = Qc^T T Qc */
  double* W = (double*)malloc(sizeof(double) * (size_t)q * (nc > 0 ? nc : 1));
  for (int32_t i = 0; i < q; ++i)
    for (int32_t j = 0; j < nc; ++j) {
      double sd = 0.0;
      for (int32_t l = 0; l < q; ++l) sd += T[(size_t)i * ldt + l] * Qc[(size_t)l * nc + j];
      W[(size_t)i * nc + j] = sd;
    }
  for (int32_t i = 0; i < nc; ++i)
    for (int32_t j = 0; j < nc; ++j) {
      double sd = 0.0;
      for (int32_t l = 0; l < q; ++l) sd += Qc[(size_t)l * nc + i] * W[(size_t)l * nc + j];
      Tn[(size_t)i * nc + j] = sd;
    }
  free(W);
  return p;
}

/* Dense deflation space of the adaptive variant: U (N x q, orthonormal), A U, T = U^T A U
 * and its LU; at most rmax columns. */
typedef struct {
  int32_t N, rmax, q;
  double *U, *AU, *T, *lu;
  int32_t* piv;
} adapt_space;

static void adapt_apply_Minv(const adapt_space* s, double mu, const double* v, double* z) {
  /* z = v + U (|mu| T^-1 - I) U^T v  (Eq. 17 with the current U) */
  double* c = (double*)malloc(sizeof(double) * (size_t)(s->q + 1));
  double* y = (double*)malloc(sizeof(double) * (size_t)(s->q + 1));
  for (int32_t t = 0; t < s->q; ++t) c[t] = dot(s->U + (size_t)t * s->N, v, s->N);
  memcpy(y, c, sizeof(double) * (size_t)s->q);
  orc_lu_solve(s->q, s->lu, s->piv, y);
  for (int32_t t = 0; t < s->q; ++t) y[t] = fabs(mu) * y[t] - c[t];
  memcpy(z, v, sizeof(double) * (size_t)s->N);
  for (int32_t t = 0; t < s->q; ++t)
    for (int32_t i = 0; i < s->N; ++i) z[i] += y[t] * s->U[(size_t)t * s->N + i];
  free(c);
  free(y);
}

/* After a cycle of k steps: the inverse-power eigenvector(s) z of H_k give u = V_k z
 * (Eq. 19), orthonormalised against U (two classical Gram-Schmidt passes) and appended;
 * at rmax columns the direction of T's largest-modulus eigenvalue (two for a complex
 * pair) is deflated first: U <- U Qc with Qc spanning the complement of its left
 * eigenvector (orc_adapt_drop).  T and its LU follow U. */
static int adapt_update(adapt_space* s, int32_t N, const int32_t* rowptr, const int32_t* col,
                        const double* val, const double* V, const double* Hr, int32_t m,
                        int32_t k, int32_t ninv) {
  if (k < 1) return 0;
  double* hk = (double*)malloc(sizeof(double) * (size_t)k * k);
  double* z = (double*)malloc(sizeof(double) * 2 * (size_t)k);
  double* u = (double*)malloc(sizeof(double) * (size_t)N);
  double* c = (double*)malloc(sizeof(double) * (size_t)(s->rmax + 1));
  for (int32_t i = 0; i < k; ++i)
    for (int32_t l = 0; l < k; ++l) hk[(size_t)i * k + l] = Hr[(size_t)i * m + l];
  const int nz = orc_hess_invvec(k, hk, ninv, z, z + k);
  const int32_t R = s->rmax;
  for (int v = 0; v < nz; ++v) {
    const double* zv = z + (size_t)v * k;
    for (int32_t i = 0; i < N; ++i) u[i] = 0.0;
    for (int32_t l = 0; l < k; ++l)
      for (int32_t i = 0; i < N; ++i) u[i] += zv[l] * V[(size_t)l * N + i];
    const double n0 = nrm2(u, N);
    for (int pass = 0; pass < 2; ++pass) {
      for (int32_t t = 0; t < s->q; ++t) c[t] = dot(s->U + (size_t)t * N, u, N);
      for (int32_t t = 0; t < s->q; ++t)
        for (int32_t i = 0; i < N; ++i) u[i] -= c[t] * s->U[(size_t)t * N + i];
    }
    const double n1 = nrm2(u, N);
    if (!(n1 > 1e-10 * n0)) continue; /* already in span(U) */
    for (int32_t i = 0; i < N; ++i) u[i] /= n1;
    if (s->q == R) { /* r > rmax: deflate the direction of T's largest eigenvalue */
      const int32_t q0 = s->q;
      double* Qc = (double*)malloc(sizeof(double) * (size_t)q0 * q0);
      double* Tn = (double*)malloc(sizeof(double) * (size_t)q0 * q0);
      const int p = orc_adapt_drop(q0, s->T, R, Qc, Tn);
      if (p < 0) {
        free(Qc);
        free(Tn);
        free(hk);
        free(z);
        free(u);
        free(c);
        return 1;
      }
      const int32_t nc = q0 - p;
      double* row = (double*)malloc(sizeof(double) * (size_t)q0);
      for (int pass = 0; pass < 2; ++pass) { /* U <- U Qc, then A U <- A U Qc */
        double* X = pass == 0 ? s->U : s->AU;
        for (int32_t i = 0; i < N; ++i) {
          for (int32_t t = 0; t < q0; ++t) row[t] = X[(size_t)t * N + i];
          for (int32_t cc = 0; cc < nc; ++cc) {
            double sd = 0.0;
            for (int32_t t = 0; t < q0; ++t) sd += row[t] * Qc[(size_t)t * nc + cc];
            X[(size_t)cc * N + i] = sd;
          }
        }
      }
      for (int32_t i = 0; i < nc; ++i)
        for (int32_t j = 0; j < nc; ++j) s->T[(size_t)i * R + j] = Tn[(size_t)i * nc + j];
      free(row);
      free(Qc);
      free(Tn);
      s->q = nc;
    }
    const int32_t q = s->q;
    memcpy(s->U + (size_t)q * N, u, sizeof(double) * (size_t)N);
    orc_spmv(N, rowptr, col, val, u, s->AU + (size_t)q * N);
    for (int32_t i = 0; i < q; ++i) {
      s->T[(size_t)i * R + q] = dot(s->U + (size_t)i * N, s->AU + (size_t)q * N, N);
      s->T[(size_t)q * R + i] = dot(s->U + (size_t)q * N, s->AU + (size_t)i * N, N);
    }
    s->T[(size_t)q * R + q] = dot(s->U + (size_t)q * N, s->AU + (size_t)q * N, N);
    s->q = q + 1;
  }
  int err = 0;
  if (s->q > 0) {
    for (int32_t i = 0; i < s->q; ++i)
      for (int32_t j = 0; j < s->q; ++j) s->lu[(size_t)i * s->q + j] = s->T[(size_t)i * R + j];
    err = orc_lu_factor(s->q, s->lu, s->piv);
  }
  free(hk);
  free(z);
  free(u);
  free(c);
  return err;
}

/* U from the caller's columns W (N x nw): each column orthonormalised against the
 * previous ones by two classical Gram-Schmidt passes and appended with A u and T's new
 * row and column; then the LU of T.  Returns 1 if a column lies in the span of the
 * previous ones (||u|| <= 1e-10 ||w_c|| after the passes) or T is singular. */
static int adapt_fill(adapt_space* s, int32_t N, const int32_t* rowptr, const int32_t* col,
                      const double* val, const double* W, int32_t nw) {
  const int32_t R = s->rmax;
  double* u = (double*)malloc(sizeof(double) * (size_t)N);
  double* c = (double*)malloc(sizeof(double) * (size_t)(R + 1));
  int err = 0;
  for (int32_t cc = 0; cc < nw && !err; ++cc) {
    memcpy(u, W + (size_t)cc * N, sizeof(double) * (size_t)N);
    const double n0 = nrm2(u, N);
    for (int pass = 0; pass < 2; ++pass) {
      for (int32_t t = 0; t < s->q; ++t) c[t] = dot(s->U + (size_t)t * N, u, N);
      for (int32_t t = 0; t < s->q; ++t)
        for (int32_t i = 0; i < N; ++i) u[i] -= c[t] * s->U[(size_t)t * N + i];
    }
    const double n1 = nrm2(u, N);
    if (!(n1 > 1e-10 * n0)) {
      err = 1;
      break;
    }
    const int32_t q = s->q;
    for (int32_t i = 0; i < N; ++i) s->U[(size_t)q * N + i] = u[i] / n1;
    orc_spmv(N, rowptr, col, val, s->U + (size_t)q * N, s->AU + (size_t)q * N);
    for (int32_t i = 0; i < q; ++i) {
      s->T[(size_t)i * R + q] = dot(s->U + (size_t)i * N, s->AU + (size_t)q * N, N);
      s->T[(size_t)q * R + i] = dot(s->U + (size_t)q * N, s->AU + (size_t)i * N, N);
    }
    s->T[(size_t)q * R + q] = dot(s->U + (size_t)q * N, s->AU + (size_t)q * N, N);
    s->q = q + 1;
  }
  if (!err) {
    for (int32_t i = 0; i < s->q; ++i)
      for (int32_t j = 0; j < s->q; ++j) s->lu[(size_t)i * s->q + j] = s->T[(size_t)i * R + j];
    err = orc_lu_factor(s->q, s->lu, s->piv) != 0;
  }
  free(u);
  free(c);
  return err;
}

/* ------------------------------------------------------------------------------------ */
/* GMRES(m) (Sec. 3.2, Eqs. 10-15) with right deflation preconditioning (Eq. 16)         */
/* ------------------------------------------------------------------------------------ */

/* Operator of the Krylov space: w = A M^-1 v (EBP), w = P A v (projector) or w = A v. */
static void apply_op(int32_t N, const int32_t* rowptr, const int32_t* col, const double* val,
                     const orc_defl* d, int mode, double mu, const double* v, double* w,
                     double* tmp) {
  if (mode == ORC_DEFL_EBP) {
    orc_defl_apply_Minv(d, mu, v, tmp);
    orc_spmv(N, rowptr, col, val, tmp, w);
  } else if (mode == ORC_DEFL_PROJECTOR) {
    orc_spmv(N, rowptr, col, val, v, tmp);
    orc_defl_apply_P(d, tmp, w);
  } else {
    orc_spmv(N, rowptr, col, val, v, w);
  }
}

/* Orthogonalise w against V[:,0..j] (column-major, leading dimension N); hcol receives
 * the j+1 projection coefficients and hcol[j+1] = ||w|| afterwards. */
static void orthogonalise(int32_t N, const double* V, int32_t j, int ortho, double* w,
                          double* hcol) {
  if (ortho == ORC_MGS) {
    for (int32_t i = 0; i <= j; ++i) {
      const double* vi = V + (size_t)i * N;
      hcol[i] = dot(vi, w, N);
      for (int32_t t = 0; t < N; ++t) w[t] -= hcol[i] * vi[t];
    }
  } else {
    /* CGS2: two classical Gram-Schmidt passes, the coefficients of both accumulate */
    for (int32_t i = 0; i <= j; ++i) hcol[i] = 0.0;
    double* hp = (double*)malloc(sizeof(double) * (size_t)(j + 1));
    for (int pass = 0; pass < 2; ++pass) {
      for (int32_t i = 0; i <= j; ++i) hp[i] = dot(V + (size_t)i * N, w, N);
      for (int32_t i = 0; i <= j; ++i) {
        const double* vi = V + (size_t)i * N;
        for (int32_t t = 0; t < N; ++t) w[t] -= hp[i] * vi[t];
      }
      for (int32_t i = 0; i <= j; ++i) hcol[i] += hp[i];
    }
    free(hp);
  }
  hcol[j + 1] = nrm2(w, N);
}

int orc_arnoldi(int32_t N, const int32_t* rowptr, const int32_t* col, const double* val,
                const orc_defl* d, int32_t defl_mode, double mu, int32_t ortho,
                const double* v0, int32_t k, double* V, double* H) {
  double* w = (double*)malloc(sizeof(double) * (size_t)N);
  double* tmp = (double*)malloc(sizeof(double) * (size_t)N);
  double* hcol = (double*)malloc(sizeof(double) * (size_t)(k + 1));
  memset(H, 0, sizeof(double) * (size_t)(k + 1) * k);
  double beta = nrm2(v0, N);
  for (int32_t t = 0; t < N; ++t) V[t] = v0[t] / beta;
  int32_t done = 0;
  for (int32_t j = 0; j < k; ++j) {
    apply_op(N, rowptr, col, val, d, defl_mode, mu, V + (size_t)j * N, w, tmp);
    orthogonalise(N, V, j, ortho, w, hcol);
    for (int32_t i = 0; i <= j + 1; ++i) H[(size_t)i * k + j] = hcol[i];
    done = j + 1;
    if (hcol[j + 1] == 0.0) break;
    for (int32_t t = 0; t < N; ++t) V[(size_t)(j + 1) * N + t] = w[t] / hcol[j + 1];
  }
  free(w);
  free(tmp);
  free(hcol);
  return done;
}

static int has_nan(double v) { return v != v || isinf(v); }

int orc_gmres(int32_t N, const int32_t* rowptr, const int32_t* col, const double* val,
              const orc_defl* d, const double* b, const double* x0, const orc_opts* o,
              double* x, orc_info* info, double* hist) {
  const int32_t m = o->m;
  const int growing = o->defl_mode == ORC_DEFL_ADAPTIVE;  /* U grows after every cycle */
  const int given = !growing && o->w_dense && o->w_cols > 0; /* U from the caller's W */
  const int adaptive = growing || given;                    /* a dense U, A U, T */
  const int mode = adaptive ? ORC_DEFL_ADAPTIVE : (d ? o->defl_mode : ORC_DEFL_NONE);
  memset(info, 0, sizeof(*info));
  adapt_space as = {0};
  if (adaptive) {
    as.N = N;
    as.rmax = given ? o->w_cols : (o->rmax > 0 ? o->rmax : 20);
    as.U = (double*)malloc(sizeof(double) * (size_t)N * as.rmax);
    as.AU = (double*)malloc(sizeof(double) * (size_t)N * as.rmax);
    as.T = (double*)calloc((size_t)as.rmax * as.rmax, sizeof(double));
    as.lu = (double*)malloc(sizeof(double) * (size_t)as.rmax * as.rmax);
    as.piv = (int32_t*)malloc(sizeof(int32_t) * (size_t)as.rmax);
  }
  double* V = (double*)malloc(sizeof(double) * (size_t)N * (m + 1));
  double* H = (double*)calloc((size_t)(m + 1) * m, sizeof(double));  /* rotated */
  double* Hr = (double*)calloc((size_t)(m + 1) * m, sizeof(double)); /* as built */
  double* cs = (double*)malloc(sizeof(double) * (size_t)m);
  double* sn = (double*)malloc(sizeof(double) * (size_t)m);
  double* g = (double*)malloc(sizeof(double) * (size_t)(m + 1));
  double* y = (double*)malloc(sizeof(double) * (size_t)m);
  double* hcol = (double*)malloc(sizeof(double) * (size_t)(m + 1));
  double* w = (double*)malloc(sizeof(double) * (size_t)N);
  double* tmp = (double*)malloc(sizeof(double) * (size_t)N);
  double* r = (double*)malloc(sizeof(double) * (size_t)N);

  for (int32_t i = 0; i < N; ++i) x[i] = x0 ? x0[i] : 0.0;

  if (given && adapt_fill(&as, N, rowptr, col, val, o->w_dense, o->w_cols)) {
    /* a column of W lies in the span of the previous ones (or U^T A U is singular) */
    free(as.U);
    free(as.AU);
    free(as.T);
    free(as.lu);
    free(as.piv);
    free(V);
    free(H);
    free(Hr);
    free(cs);
    free(sn);
    free(g);
    free(y);
    free(hcol);
    free(w);
    free(tmp);
    free(r);
    info->status = -1;
    return -1;
  }

  /* mu (Sec. 3.3): the largest eigenvalue, estimated from the Ritz values of H_m of the
   * first cycle, which runs with M = I; or given; or bounded by the infinity norm. */
  double mu = 0.0;
  int defl_on = (mode == ORC_DEFL_PROJECTOR);
  if (mode == ORC_DEFL_EBP || mode == ORC_DEFL_ADAPTIVE) {
    if (o->mu_mode == ORC_MU_USER) {
      mu = o->mu_user;
      defl_on = 1;
    } else if (o->mu_mode == ORC_MU_NORM_INF) {
      for (int32_t i = 0; i < N; ++i) {
        double s = 0.0;
        for (int32_t k = rowptr[i]; k < rowptr[i + 1]; ++k) s += fabs(val[k]);
        if (s > mu) mu = s;
      }
      defl_on = 1;
    }
  }

  /* residual of the current iterate; with the projector, b - A x = P (b - A xhat) */
  #define TRUE_RESIDUAL()                                   \
    do {                                                     \
      orc_spmv(N, rowptr, col, val, x, tmp);                 \
      for (int32_t i_ = 0; i_ < N; ++i_) r[i_] = b[i_] - tmp[i_]; \
      if (mode == ORC_DEFL_PROJECTOR) {                      \
        orc_defl_apply_P(d, r, tmp);                         \
        memcpy(r, tmp, sizeof(double) * (size_t)N);          \
      }                                                      \
    } while (0)

  /* reference norm rho0 = ||b - A x0|| of the original system (Eq. 15) */
  orc_spmv(N, rowptr, col, val, x, tmp);
  for (int32_t i = 0; i < N; ++i) r[i] = b[i] - tmp[i];
  double rho0 = o->r0_norm_ref > 0.0 ? o->r0_norm_ref : nrm2(r, N);
  int status = 1;
  int64_t steps = 0, cycles = 0;
  double est = 1.0, truerel = 1.0;
  if (has_nan(rho0)) {
    status = -5;
    goto done;
  }
  if (rho0 == 0.0) {
    status = 0;
    est = truerel = 0.0;
    goto done;
  }
  if (mode == ORC_DEFL_PROJECTOR) TRUE_RESIDUAL();

  for (;;) {
    double beta = nrm2(r, N);
    truerel = beta / rho0;
    if (has_nan(beta)) {
      status = -5;
      break;
    }
    if (beta == 0.0 || (!o->fixed_iterations && truerel <= o->tol)) {
      status = 0;
      break;
    }
    if (steps >= o->maxit) {
      status = 1;
      break;
    }
    /* one cycle of GMRES(m): Arnoldi from v1 = r/beta, g = beta e1 */
    for (int32_t i = 0; i < N; ++i) V[i] = r[i] / beta;
    for (int32_t i = 0; i <= m; ++i) g[i] = 0.0;
    g[0] = beta;
    int32_t k = 0;
    int use_defl = defl_on ? mode : ORC_DEFL_NONE;
    const int dense = adaptive && defl_on && as.q > 0; /* M^-1 with the current U */
    for (int32_t j = 0; j < m && steps < o->maxit; ++j) {
      if (adaptive) {
        if (dense) {
          adapt_apply_Minv(&as, mu, V + (size_t)j * N, tmp);
          orc_spmv(N, rowptr, col, val, tmp, w);
        } else {
          orc_spmv(N, rowptr, col, val, V + (size_t)j * N, w);
        }
      } else {
        apply_op(N, rowptr, col, val, d, use_defl, mu, V + (size_t)j * N, w, tmp);
      }
      orthogonalise(N, V, j, o->ortho, w, hcol);
      double hnext = hcol[j + 1];
      double hn2 = 0.0;
      for (int32_t i = 0; i <= j + 1; ++i) {
        Hr[(size_t)i * m + j] = hcol[i];
        H[(size_t)i * m + j] = hcol[i];
        hn2 += hcol[i] * hcol[i];
      }
      if (has_nan(hnext)) {
        status = -5;
        goto done;
      }
      /* apply the previous plane rotations to the new column (Eq. 12) */
      for (int32_t i = 0; i < j; ++i) {
        double a = H[(size_t)i * m + j], bb = H[(size_t)(i + 1) * m + j];
        H[(size_t)i * m + j] = cs[i] * a + sn[i] * bb;
        H[(size_t)(i + 1) * m + j] = -sn[i] * a + cs[i] * bb;
      }
      /* new rotation annihilating h_{j+1,j} */
      double a = H[(size_t)j * m + j];
      if (hnext == 0.0) {
        cs[j] = 1.0;
        sn[j] = 0.0;
      } else {
        double rho = hypot(a, hnext);
        cs[j] = a / rho;
        sn[j] = hnext / rho;
        H[(size_t)j * m + j] = rho;
      }
      H[(size_t)(j + 1) * m + j] = 0.0;
      g[j + 1] = -sn[j] * g[j];
      g[j] = cs[j] * g[j];
      ++steps;
      k = j + 1;
      est = fabs(g[j + 1]) / rho0; /* ||b - A x_k|| = |gamma_{k+1}|  (Eq. 14) */
      if (hist) {
        hist[2 * (steps - 1)] = (double)j;
        hist[2 * (steps - 1) + 1] = est;
      }
      if (hnext <= 1e-14 * sqrt(hn2)) break; /* (lucky) breakdown: K_j is invariant */
      if (!o->fixed_iterations && est <= o->tol) break;
      for (int32_t i = 0; i < N; ++i) V[(size_t)(j + 1) * N + i] = w[i] / hnext;
    }
    /* least squares solution by back substitution with R_k (Eq. 12) */
    for (int32_t i = k - 1; i >= 0; --i) {
      double s = g[i];
      for (int32_t l = i + 1; l < k; ++l) s -= H[(size_t)i * m + l] * y[l];
      y[i] = s / H[(size_t)i * m + i];
    }
    /* x += M^-1 V_k y  (Eqs. 11 and 16) */
    for (int32_t i = 0; i < N; ++i) w[i] = 0.0;
    for (int32_t l = 0; l < k; ++l)
      for (int32_t i = 0; i < N; ++i) w[i] += y[l] * V[(size_t)l * N + i];
    if (use_defl == ORC_DEFL_EBP) {
      orc_defl_apply_Minv(d, mu, w, tmp);
      for (int32_t i = 0; i < N; ++i) x[i] += tmp[i];
    } else if (dense) {
      adapt_apply_Minv(&as, mu, w, tmp);
      for (int32_t i = 0; i < N; ++i) x[i] += tmp[i];
    } else {
      for (int32_t i = 0; i < N; ++i) x[i] += w[i];
    }
    ++cycles;
    if ((mode == ORC_DEFL_EBP || mode == ORC_DEFL_ADAPTIVE) && !defl_on) {
      /* Ritz values of H_k from the first cycle give |mu| */
      double* hk = (double*)malloc(sizeof(double) * (size_t)k * k);
      double* wr = (double*)malloc(sizeof(double) * (size_t)k);
      double* wi = (double*)malloc(sizeof(double) * (size_t)k);
      for (int32_t i = 0; i < k; ++i)
        for (int32_t l = 0; l < k; ++l) hk[(size_t)i * k + l] = Hr[(size_t)i * m + l];
      int e = orc_hessenberg_eigs(k, hk, wr, wi);
      mu = 0.0;
      for (int32_t i = 0; i < k; ++i) {
        double md = hypot(wr[i], wi[i]);
        if (md > mu) mu = md;
      }
      free(hk);
      free(wr);
      free(wi);
      if (e != 0 || mu == 0.0) {
        status = -4;
        break;
      }
      defl_on = 1;
    }
    /* grow U from this cycle's Hessenberg matrix and basis (Sec. 3.3, Eq. 19) */
    if (growing && adapt_update(&as, N, rowptr, col, val, V, Hr, m, k, o->ninv > 0 ? o->ninv : 20)) {
      status = -4;
      break;
    }
    TRUE_RESIDUAL();
  }
  #undef TRUE_RESIDUAL

done:
  if (mode == ORC_DEFL_PROJECTOR && status >= 0) {
    /* x = xhat + U T^-1 U^T (b - A xhat): adds the coarse component */
    orc_spmv(N, rowptr, col, val, x, tmp);
    for (int32_t i = 0; i < N; ++i) r[i] = b[i] - tmp[i];
    double* c = (double*)malloc(sizeof(double) * (size_t)d->r);
    defl_Ut(d, r, c);
    orc_lu_solve(d->r, d->lu, d->piv, c);
    defl_U_add(d, c, x);
    free(c);
  }
  if (status >= 0 && rho0 > 0.0) {
    orc_spmv(N, rowptr, col, val, x, tmp);
    for (int32_t i = 0; i < N; ++i) r[i] = b[i] - tmp[i];
    truerel = nrm2(r, N) / rho0;
  }
  info->iters = steps;
  info->cycles = cycles;
  info->status = status;
  info->rel_res_est = est;
  info->rel_res_true = truerel;
  info->mu = mu;
  if (adaptive) {
    info->q = as.q;
    if (o->u_out) memcpy(o->u_out, as.U, sizeof(double) * (size_t)N * as.q);
    free(as.U);
    free(as.AU);
    free(as.T);
    free(as.lu);
    free(as.piv);
  }
  free(V);
  free(H);
  free(Hr);
  free(cs);
  free(sn);
  free(g);
  free(y);
  free(hcol);
  free(w);
  free(tmp);
  free(r);
  return status;
}
