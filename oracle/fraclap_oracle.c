/*
 * FP64 CPU oracle for the fractional Poisson eigenfunction-expansion method.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * CPU-baseline leg of the benchmark may load this library.  It shares no code,
 * header or constant with the CUDA path.
 *
 * What it computes (arXiv:1911.11906):
 *   - Sec. II, eq. (discrete_laplace): the discrete Laplace eigenproblem.  With
 *     a nodal finite-difference discretisation the mass matrix is the identity,
 *     so K phi = theta phi with K the 5-point (2-D) or 7-point (3-D) Dirichlet
 *     Laplacian scaled by 1/h^2.
 *   - Sec. II, the sums g and v after eq. (discrete_laplace):
 *     v = sum_k theta_k^{-alpha/2} <f, phi_k> phi_k  (eq. poisson_solution).
 *   - Sec. II, eq. (diffusion_solution): the fractional diffusion solution
 *     u(t) = sum_k exp(-mu theta_k^{alpha/2} t) <u0, phi_k> phi_k.
 *   - Sec. II, eq. (discrete_laplace) with a finite-element basis: bilinear
 *     (2-D) / trilinear (3-D) elements give K and M, the generalised problem
 *     K phi = theta M phi is reduced by the Cholesky factor of M, and the
 *     apply takes the M-inner product.
 *   - Sec. III-D-2 (exact eigenvalue counting): the number of eigenvalues
 *     below sigma equals the number of negative pivots of the LDL^T
 *     factorisation of A - sigma I (Sylvester's law of inertia); the same
 *     count on the tridiagonal T (Sturm sequence) and bisection on it.
 *
 * The eigendecomposition is the plain textbook route, written from the
 * mathematics: Householder reduction to tridiagonal form with the orthogonal
 * factor accumulated, then implicit symmetric QR steps with a Wilkinson shift
 * applied through Givens rotations; cyclic Jacobi for tiny matrices.
 * Everything is IEEE double.  Matrices are column-major: a(i, j) = a[i + j*lda].
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

#define ORACLE_OK 0
#define ORACLE_EINVAL (-1)
#define ORACLE_ENOCONV (-2)
#define ORACLE_ENOMEM (-3)
#define ORACLE_EZEROPIVOT (-4)

int oracle_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

/* ------------------------------------------------------------------------ */
/* Assembly: Sec. II eq. (discrete_laplace) with nodal FD, Dirichlet zero     */
/* outside the mask.  Row i of A: (2*dim/h^2) on the diagonal, -1/h^2 for     */
/* every face neighbour that is also a dof.  Columns ascending within a row.  */
/* ------------------------------------------------------------------------ */

/* Numbers the dofs: idx[g] = dof number of grid node g, -1 outside.  Returns n. */
int64_t oracle_number_dofs(const uint8_t* mask, int64_t ngrid, int32_t* idx) {
  int64_t n = 0;
  for (int64_t g = 0; g < ngrid; ++g) idx[g] = mask[g] ? (int32_t)(n++) : -1;
  return n;
}

/* Fills the CSR of A.  ext = (nx, ny, nz), nz = 1 for dim = 2.
 * rowptr has n+1 entries; col/val have room for (2*dim+1)*n entries.
 * Returns nnz. */
int64_t oracle_assemble_csr(const int32_t* idx, int dim, const int64_t* ext, double h,
                            int64_t* rowptr, int32_t* col, double* val) {
  const int64_t nx = ext[0], ny = ext[1], nz = (dim == 3) ? ext[2] : 1;
  const double diag = (double)(2 * dim) / (h * h);
  const double off = -1.0 / (h * h);
  int64_t nnz = 0, row = 0;
  for (int64_t z = 0; z < nz; ++z)
    for (int64_t y = 0; y < ny; ++y)
      for (int64_t x = 0; x < nx; ++x) {
        const int64_t g = x + nx * (y + ny * z);
        if (idx[g] < 0) continue;
        rowptr[row] = nnz;
        /* neighbours in ascending grid (hence dof) order */
        int64_t nb[7];
        int cnt = 0;
        if (dim == 3 && z > 0) nb[cnt++] = g - nx * ny;
        if (y > 0) nb[cnt++] = g - nx;
        if (x > 0) nb[cnt++] = g - 1;
        nb[cnt++] = g;
        if (x + 1 < nx) nb[cnt++] = g + 1;
        if (y + 1 < ny) nb[cnt++] = g + nx;
        if (dim == 3 && z + 1 < nz) nb[cnt++] = g + nx * ny;
        for (int t = 0; t < cnt; ++t) {
          const int32_t c = idx[nb[t]];
          if (c < 0) continue;
          col[nnz] = c;
          val[nnz] = (nb[t] == g) ? diag : off;
          ++nnz;
        }
        ++row;
      }
  rowptr[row] = nnz;
  return nnz;
}

/* y = A x for the CSR matrix (alpha = -2 of the apply is this product). */
void oracle_spmv(int64_t n, const int64_t* rowptr, const int32_t* col, const double* val,
                 const double* x, double* y) {
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < n; ++i) {
    double s = 0.0;
    for (int64_t p = rowptr[i]; p < rowptr[i + 1]; ++p) s += val[p] * x[col[p]];
    y[i] = s;
  }
}

/* ------------------------------------------------------------------------ */
/* Householder reduction to tridiagonal form, A = Q T Q^T.                    */
/* Step k annihilates A(k+2:n-1, k) with H_k = I - tau_k v_k v_k^T,           */
/* v_k(k+1) = 1, applied on both sides of the trailing matrix through the     */
/* symmetric rank-2 update A22 -= v w^T + w v^T with                          */
/* p = tau A22 v, w = p - (tau/2)(p^T v) v.  Q = H_0 H_1 ... H_{n-3}.           */
/* A (full symmetric storage) is overwritten.                                */
/* ------------------------------------------------------------------------ */
int oracle_tridiagonalize(int64_t n, double* A, int64_t lda, double* d, double* e,
                          double* Q, int64_t ldq) {
  if (n < 1 || lda < n || (Q && ldq < n)) return ORACLE_EINVAL;
  double* tau = (double*)calloc((size_t)(n > 1 ? n : 1), sizeof(double));
  double* p = (double*)malloc(sizeof(double) * (size_t)n);
  if (!tau || !p) { free(tau); free(p); return ORACLE_ENOMEM; }
#define AA(i, j) A[(i) + (j) * lda]
  for (int64_t k = 0; k + 2 < n; ++k) {
    const int64_t m = n - k - 1;        /* length of x = A(k+1:n-1, k) */
    double* x = &AA(k + 1, k);
    double tail = 0.0;
    for (int64_t i = 1; i < m; ++i) tail += x[i] * x[i];
    if (tail == 0.0) {                  /* already reduced: H_k = I */
      tau[k] = 0.0;
      for (int64_t i = 1; i < m; ++i) x[i] = 0.0;
      continue;
    }
    const double x0 = x[0];
    const double alpha = sqrt(x0 * x0 + tail);
    const double beta = (x0 >= 0.0) ? -alpha : alpha;   /* H x = beta e_1 */
    const double v0 = x0 - beta;
    tau[k] = (beta - x0) / beta;
    for (int64_t i = 1; i < m; ++i) x[i] /= v0;       /* v = (1, x(1:)/v0) */
    x[0] = 1.0;
    const double* v = x;
    const double t = tau[k];
    /* p = tau * A22 v   (A22 symmetric: use its columns) */
#pragma omp parallel for schedule(static)
    for (int64_t j = 0; j < m; ++j) {
      const double* aj = &AA(k + 1, k + 1 + j);
      double s = 0.0;
      for (int64_t i = 0; i < m; ++i) s += aj[i] * v[i];
      p[j] = t * s;
    }
    double pv = 0.0;
    for (int64_t i = 0; i < m; ++i) pv += p[i] * v[i];
    const double half = 0.5 * t * pv;
    for (int64_t i = 0; i < m; ++i) p[i] -= half * v[i];   /* p is now w */
#pragma omp parallel for schedule(static)
    for (int64_t j = 0; j < m; ++j) {
      double* aj = &AA(k + 1, k + 1 + j);
      const double vj = v[j], wj = p[j];
      for (int64_t i = 0; i < m; ++i) aj[i] -= v[i] * wj + p[i] * vj;
    }
    /* store the reduced column: T(k+1,k) = beta, v kept below it for Q */
    x[0] = beta;   /* v(0) = 1 is implicit */
  }
  for (int64_t k = 0; k < n; ++k) d[k] = AA(k, k);
  for (int64_t k = 0; k + 1 < n; ++k) e[k] = AA(k + 1, k);
  if (Q) {
    /* backward accumulation: Q = H_0 (H_1 (... H_{n-3})) */
    for (int64_t j = 0; j < n; ++j)
      for (int64_t i = 0; i < n; ++i) Q[i + j * ldq] = (i == j) ? 1.0 : 0.0;
    for (int64_t k = n - 3; k >= 0; --k) {
      if (tau[k] == 0.0) continue;
      const int64_t m = n - k - 1;
      const double* vs = &AA(k + 2, k);   /* v(1:m-1); v(0) = 1 */
      const double t = tau[k];
#pragma omp parallel for schedule(static)
      for (int64_t j = 0; j < m; ++j) {
        double* qj = &Q[(k + 1) + (k + 1 + j) * ldq];
        double s = qj[0];
        for (int64_t i = 1; i < m; ++i) s += vs[i - 1] * qj[i];
        s *= t;
        qj[0] -= s;
        for (int64_t i = 1; i < m; ++i) qj[i] -= s * vs[i - 1];
      }
    }
  }
#undef AA
  free(tau);
  free(p);
  return ORACLE_OK;
}

/* ------------------------------------------------------------------------ */
/* Symmetric tridiagonal eigensolver: implicit QR steps with Wilkinson shift. */
/* T has diagonal d(0:n-1) and off-diagonal e(0:n-2), e(i) = T(i+1, i).       */
/* Each step on an unreduced block [l, hi] chases the bulge with rotations    */
/* P_k = [c s; -s c] acting on rows/columns (k, k+1): T <- P T P^T and the    */
/* eigenvector block Z <- Z P^T.  The rotations of one step are recorded and  */
/* then applied to the rows of Z (rows are independent).  On return d holds   */
/* the eigenvalues in ascending order and Z the matching eigenvectors.        */
/* ------------------------------------------------------------------------ */
static void apply_rotations_to_rows(int64_t nrows, double* Z, int64_t ldz, int64_t l,
                                    int64_t hi, const double* cs, const double* sn) {
  const int64_t blk = 64;
  const int64_t nblk = (nrows + blk - 1) / blk;
#pragma omp parallel for schedule(static)
  for (int64_t b = 0; b < nblk; ++b) {
    const int64_t r0 = b * blk, r1 = (r0 + blk < nrows) ? r0 + blk : nrows;
    for (int64_t k = l; k < hi; ++k) {
      const double c = cs[k - l], s = sn[k - l];
      double* zk = &Z[k * ldz];
      double* zk1 = &Z[(k + 1) * ldz];
      for (int64_t r = r0; r < r1; ++r) {
        const double a = zk[r], bb = zk1[r];
        zk[r] = c * a + s * bb;
        zk1[r] = -s * a + c * bb;
      }
    }
  }
}

static int negligible(double e, double d0, double d1) {
  return fabs(e) <= 0.5 * 2.220446049250313e-16 * (fabs(d0) + fabs(d1)) || e == 0.0;
}

int oracle_tridiag_eig(int64_t n, double* d, double* e, double* Z, int64_t ldz,
                       int64_t zrows, int64_t max_steps) {
  if (n < 1) return ORACLE_EINVAL;
  double* cs = (double*)malloc(sizeof(double) * (size_t)(n + 1));
  double* sn = (double*)malloc(sizeof(double) * (size_t)(n + 1));
  if (!cs || !sn) { free(cs); free(sn); return ORACLE_ENOMEM; }
  int64_t steps = 0;
  int64_t hi = n - 1;
  while (hi > 0) {
    if (negligible(e[hi - 1], d[hi - 1], d[hi])) {
      e[hi - 1] = 0.0;
      --hi;
      continue;
    }
    int64_t l = hi - 1;
    while (l > 0 && !negligible(e[l - 1], d[l - 1], d[l])) --l;
    if (l > 0) e[l - 1] = 0.0;
    if (++steps > max_steps) { free(cs); free(sn); return ORACLE_ENOCONV; }
    /* Wilkinson shift from the trailing 2x2 block of [l, hi] */
    const double a = d[hi - 1], b = e[hi - 1], c = d[hi];
    const double delta = 0.5 * (a - c);
    const double rr = hypot(delta, b);
    const double mu = c - b * b / (delta + (delta >= 0.0 ? rr : -rr));
    double x = d[l] - mu, z = e[l];
    for (int64_t k = l; k < hi; ++k) {
      double r = hypot(x, z);
      double cc = 1.0, ss = 0.0;
      if (r != 0.0) { cc = x / r; ss = z / r; }
      if (k > l) e[k - 1] = r;          /* bulge at (k+1, k-1) removed */
      const double dk = d[k], dk1 = d[k + 1], ek = e[k];
      d[k] = cc * cc * dk + 2.0 * cc * ss * ek + ss * ss * dk1;
      d[k + 1] = ss * ss * dk - 2.0 * cc * ss * ek + cc * cc * dk1;
      e[k] = cc * ss * (dk1 - dk) + (cc * cc - ss * ss) * ek;
      cs[k - l] = cc;
      sn[k - l] = ss;
      if (k + 1 < hi) {
        x = e[k];
        z = ss * e[k + 1];               /* new bulge at (k+2, k) */
        e[k + 1] = cc * e[k + 1];
      }
    }
    if (Z) apply_rotations_to_rows(zrows, Z, ldz, l, hi, cs, sn);
  }
  free(cs);
  free(sn);
  /* selection sort to ascending order (stable enough; n^2 compares only) */
  for (int64_t i = 0; i + 1 < n; ++i) {
    int64_t kmin = i;
    for (int64_t j = i + 1; j < n; ++j) if (d[j] < d[kmin]) kmin = j;
    if (kmin != i) {
      const double t = d[i]; d[i] = d[kmin]; d[kmin] = t;
      if (Z)
        for (int64_t r = 0; r < zrows; ++r) {
          const double q = Z[r + i * ldz];
          Z[r + i * ldz] = Z[r + kmin * ldz];
          Z[r + kmin * ldz] = q;
        }
    }
  }
  return ORACLE_OK;
}

/* Full eigendecomposition A = V diag(lam) V^T (A is not modified). */
int oracle_eig_full(int64_t n, const double* A, int64_t lda, double* lam, double* V,
                    int64_t ldv) {
  if (n < 1 || lda < n || ldv < n) return ORACLE_EINVAL;
  double* W = (double*)malloc(sizeof(double) * (size_t)n * (size_t)n);
  double* e = (double*)calloc((size_t)n, sizeof(double));
  if (!W || !e) { free(W); free(e); return ORACLE_ENOMEM; }
  for (int64_t j = 0; j < n; ++j) memcpy(&W[j * n], &A[j * lda], sizeof(double) * (size_t)n);
  int rc = oracle_tridiagonalize(n, W, n, lam, e, V, ldv);
  if (rc == ORACLE_OK) rc = oracle_tridiag_eig(n, lam, e, V, ldv, n, 30 * n + 30);
  free(W);
  free(e);
  return rc;
}

/* ------------------------------------------------------------------------ */
/* Cyclic Jacobi for tiny symmetric matrices (an independent second route).   */
/* Each rotation zeroes a(p, q); sweeps stop when the off-diagonal Frobenius  */
/* norm falls below 1e-15 ||A||_F.  Eigenvalues sorted ascending.             */
/* ------------------------------------------------------------------------ */
int oracle_eig_jacobi(int64_t n, const double* A, int64_t lda, double* lam, double* V,
                      int64_t ldv, int max_sweeps) {
  if (n < 1 || lda < n || ldv < n) return ORACLE_EINVAL;
  double* a = (double*)malloc(sizeof(double) * (size_t)n * (size_t)n);
  if (!a) return ORACLE_ENOMEM;
  double fro = 0.0;
  for (int64_t j = 0; j < n; ++j)
    for (int64_t i = 0; i < n; ++i) {
      a[i + j * n] = A[i + j * lda];
      fro += a[i + j * n] * a[i + j * n];
      V[i + j * ldv] = (i == j) ? 1.0 : 0.0;
    }
  fro = sqrt(fro);
  int sweep = 0;
  for (;; ++sweep) {
    double off = 0.0;
    for (int64_t j = 0; j < n; ++j)
      for (int64_t i = 0; i < n; ++i)
        if (i != j) off += a[i + j * n] * a[i + j * n];
    if (sqrt(off) <= 1e-15 * fro || fro == 0.0) break;
    if (sweep >= max_sweeps) { free(a); return ORACLE_ENOCONV; }
    for (int64_t p = 0; p + 1 < n; ++p)
      for (int64_t q = p + 1; q < n; ++q) {
        const double apq = a[p + q * n];
        if (apq == 0.0) continue;
        /* choose t = tan(theta) with a'(p,q) = 0, |theta| <= pi/4 */
        const double theta = (a[q + q * n] - a[p + p * n]) / (2.0 * apq);
        const double t = (theta >= 0.0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
        const double c = 1.0 / sqrt(t * t + 1.0), s = t * c;
        /* A <- J^T A J with J = [c s; -s c] in the (p, q) plane */
        for (int64_t k = 0; k < n; ++k) {      /* columns p, q */
          const double akp = a[k + p * n], akq = a[k + q * n];
          a[k + p * n] = c * akp - s * akq;
          a[k + q * n] = s * akp + c * akq;
        }
        for (int64_t k = 0; k < n; ++k) {      /* rows p, q */
          const double apk = a[p + k * n], aqk = a[q + k * n];
          a[p + k * n] = c * apk - s * aqk;
          a[q + k * n] = s * apk + c * aqk;
        }
        for (int64_t k = 0; k < n; ++k) {      /* V <- V J */
          const double vkp = V[k + p * ldv], vkq = V[k + q * ldv];
          V[k + p * ldv] = c * vkp - s * vkq;
          V[k + q * ldv] = s * vkp + c * vkq;
        }
      }
  }
  for (int64_t i = 0; i < n; ++i) lam[i] = a[i + i * n];
  for (int64_t i = 0; i + 1 < n; ++i) {
    int64_t kmin = i;
    for (int64_t j = i + 1; j < n; ++j) if (lam[j] < lam[kmin]) kmin = j;
    if (kmin != i) {
      const double t = lam[i]; lam[i] = lam[kmin]; lam[kmin] = t;
      for (int64_t r = 0; r < n; ++r) {
        const double q = V[r + i * ldv];
        V[r + i * ldv] = V[r + kmin * ldv];
        V[r + kmin * ldv] = q;
      }
    }
  }
  free(a);
  return ORACLE_OK;
}

/* ------------------------------------------------------------------------ */
/* Banded LDL^T of A - sigma I without pivoting (Sec. III-D-2).               */
/* The half-bandwidth bw is the largest i - j over the nonzeros of the CSR.   */
/* Band storage: B[(i - j) + j*(bw+1)] for 0 <= i - j <= bw.                  */
/* ------------------------------------------------------------------------ */
static int64_t csr_bandwidth(int64_t n, const int64_t* rowptr, const int32_t* col) {
  int64_t bw = 0;
  for (int64_t i = 0; i < n; ++i)
    for (int64_t p = rowptr[i]; p < rowptr[i + 1]; ++p)
      if (i - col[p] > bw) bw = i - col[p];
  return bw;
}

/* Factorises in place; dpiv receives the pivots, B keeps L below the diagonal. */
static int band_ldlt(int64_t n, int64_t bw, double* B, double* dpiv) {
  const int64_t ld = bw + 1;
  double* l = (double*)malloc(sizeof(double) * (size_t)ld);
  if (!l) return ORACLE_ENOMEM;
  for (int64_t j = 0; j < n; ++j) {
    const double dj = B[0 + j * ld];
    dpiv[j] = dj;
    if (dj == 0.0) { free(l); return ORACLE_EZEROPIVOT; }
    const int64_t last = (j + bw < n - 1) ? j + bw : n - 1;
    for (int64_t i = j + 1; i <= last; ++i) {
      l[i - j] = B[(i - j) + j * ld] / dj;
    }
    /* trailing update: B(i, k) -= l_i * d_j * l_k for j < k <= i <= last */
    for (int64_t k = j + 1; k <= last; ++k) {
      const double lk = l[k - j] * dj;
      for (int64_t i = k; i <= last; ++i) B[(i - k) + k * ld] -= l[i - j] * lk;
    }
    for (int64_t i = j + 1; i <= last; ++i) B[(i - j) + j * ld] = l[i - j];
  }
  free(l);
  return ORACLE_OK;
}

static double* csr_to_band(int64_t n, const int64_t* rowptr, const int32_t* col,
                           const double* val, double sigma, int64_t* bw_out) {
  const int64_t bw = csr_bandwidth(n, rowptr, col);
  const int64_t ld = bw + 1;
  double* B = (double*)calloc((size_t)ld * (size_t)n, sizeof(double));
  if (!B) return NULL;
  for (int64_t i = 0; i < n; ++i)
    for (int64_t p = rowptr[i]; p < rowptr[i + 1]; ++p) {
      const int64_t j = col[p];
      if (j <= i) B[(i - j) + j * ld] += val[p];
    }
  for (int64_t j = 0; j < n; ++j) B[j * ld] -= sigma;
  *bw_out = bw;
  return B;
}

/* Number of eigenvalues of A strictly below sigma (negative pivots of
 * A - sigma I = L D L^T).  Returns a negative error code on failure. */
int64_t oracle_count_below(int64_t n, const int64_t* rowptr, const int32_t* col,
                           const double* val, double sigma) {
  int64_t bw;
  double* B = csr_to_band(n, rowptr, col, val, sigma, &bw);
  double* dp = (double*)malloc(sizeof(double) * (size_t)n);
  if (!B || !dp) { free(B); free(dp); return ORACLE_ENOMEM; }
  const int rc = band_ldlt(n, bw, B, dp);
  int64_t neg = 0;
  if (rc == ORACLE_OK)
    for (int64_t j = 0; j < n; ++j) neg += (dp[j] < 0.0);
  free(B);
  free(dp);
  return rc == ORACLE_OK ? neg : rc;
}

/* Direct solve A u = f through the banded LDL^T (the alpha = 2 special case). */
int oracle_band_solve(int64_t n, const int64_t* rowptr, const int32_t* col,
                      const double* val, const double* f, double* u) {
  int64_t bw;
  double* B = csr_to_band(n, rowptr, col, val, 0.0, &bw);
  double* dp = (double*)malloc(sizeof(double) * (size_t)n);
  if (!B || !dp) { free(B); free(dp); return ORACLE_ENOMEM; }
  int rc = band_ldlt(n, bw, B, dp);
  if (rc == ORACLE_OK) {
    const int64_t ld = bw + 1;
    for (int64_t i = 0; i < n; ++i) u[i] = f[i];
    for (int64_t j = 0; j < n; ++j) {          /* L y = f */
      const int64_t last = (j + bw < n - 1) ? j + bw : n - 1;
      for (int64_t i = j + 1; i <= last; ++i) u[i] -= B[(i - j) + j * ld] * u[j];
    }
    for (int64_t j = 0; j < n; ++j) u[j] /= dp[j];   /* D z = y */
    for (int64_t j = n - 1; j >= 0; --j) {     /* L^T u = z */
      const int64_t last = (j + bw < n - 1) ? j + bw : n - 1;
      double s = u[j];
      for (int64_t i = j + 1; i <= last; ++i) s -= B[(i - j) + j * ld] * u[i];
      u[j] = s;
    }
  }
  free(B);
  free(dp);
  return rc;
}

/* ------------------------------------------------------------------------ */
/* Spectral apply, Sec. II (sums after eq. discrete_laplace):                 */
/*   W = V^T F,  u_j = V (lam^{-alpha_j/2} .* W(:, f_j)).                      */
/* pow() in double decides every multiplier.                                  */
/* ------------------------------------------------------------------------ */
int oracle_frac_apply(int64_t n, const double* V, int64_t ldv, const double* lam,
                      const double* F, int64_t ldf, int64_t m, const int32_t* pair_f,
                      const double* pair_alpha, int64_t k, double* U, int64_t ldu) {
  if (n < 0 || m < 0 || k < 0 || ldv < n || ldf < n || ldu < n) return ORACLE_EINVAL;
  for (int64_t j = 0; j < k; ++j)
    if (pair_f[j] < 0 || pair_f[j] >= m) return ORACLE_EINVAL;
  if (n == 0 || k == 0) return ORACLE_OK;
  double* W = (double*)malloc(sizeof(double) * (size_t)n * (size_t)(m ? m : 1));
  if (!W) return ORACLE_ENOMEM;
  /* W(i, c) = <v_i, f_c> */
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < n; ++i) {
    const double* vi = &V[i * ldv];
    for (int64_t c = 0; c < m; ++c) {
      const double* fc = &F[c * ldf];
      double s = 0.0;
      for (int64_t r = 0; r < n; ++r) s += vi[r] * fc[r];
      W[i + c * n] = s;
    }
  }
  double* coef = (double*)malloc(sizeof(double) * (size_t)n);
  if (!coef) { free(W); return ORACLE_ENOMEM; }
  for (int64_t j = 0; j < k; ++j) {
    const double ex = -0.5 * pair_alpha[j];
    const double* w = &W[(int64_t)pair_f[j] * n];
    for (int64_t i = 0; i < n; ++i) coef[i] = pow(lam[i], ex) * w[i];
    double* u = &U[j * ldu];
    /* u = sum_i coef_i v_i, rows split into independent chunks */
    const int64_t blk = 256, nblk = (n + blk - 1) / blk;
#pragma omp parallel for schedule(static)
    for (int64_t b = 0; b < nblk; ++b) {
      const int64_t r0 = b * blk, r1 = (r0 + blk < n) ? r0 + blk : n;
      for (int64_t r = r0; r < r1; ++r) u[r] = 0.0;
      for (int64_t i = 0; i < n; ++i) {
        const double ci = coef[i];
        const double* vi = &V[i * ldv];
        for (int64_t r = r0; r < r1; ++r) u[r] += vi[r] * ci;
      }
    }
  }
  free(coef);
  free(W);
  return ORACLE_OK;
}

/* ------------------------------------------------------------------------ */
/* Fractional diffusion, Sec. II eq. diffusion_solution: the solution of     */
/*   du/dt + mu (-Laplacian)^{alpha/2} u = 0,  u(0) = u0,                    */
/* at time t is sum_i exp(-mu lam_i^{alpha/2} t) <u0, v_i> v_i.              */
/* Pair j takes initial state U0(:, pair_f[j]), order pair_alpha[j] and      */
/* time pair_t[j]; mu is shared.  pow() and exp() in double decide every     */
/* multiplier.                                                               */
/* ------------------------------------------------------------------------ */
int oracle_frac_diffusion(int64_t n, const double* V, int64_t ldv, const double* lam,
                          const double* U0, int64_t ldu0, int64_t m, const int32_t* pair_f,
                          const double* pair_alpha, const double* pair_t, double mu, int64_t k,
                          double* U, int64_t ldu) {
  if (n < 0 || m < 0 || k < 0 || ldv < n || ldu0 < n || ldu < n) return ORACLE_EINVAL;
  for (int64_t j = 0; j < k; ++j)
    if (pair_f[j] < 0 || pair_f[j] >= m) return ORACLE_EINVAL;
  if (n == 0 || k == 0) return ORACLE_OK;
  double* W = (double*)malloc(sizeof(double) * (size_t)n * (size_t)(m ? m : 1));
  if (!W) return ORACLE_ENOMEM;
  /* W(i, c) = <u0_c, v_i>: the expansion coefficients of each initial state */
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < n; ++i) {
    const double* vi = &V[i * ldv];
    for (int64_t c = 0; c < m; ++c) {
      const double* uc = &U0[c * ldu0];
      double s = 0.0;
      for (int64_t r = 0; r < n; ++r) s += vi[r] * uc[r];
      W[i + c * n] = s;
    }
  }
  double* coef = (double*)malloc(sizeof(double) * (size_t)n);
  if (!coef) { free(W); return ORACLE_ENOMEM; }
  for (int64_t j = 0; j < k; ++j) {
    const double half = 0.5 * pair_alpha[j], t = pair_t[j];
    const double* w = &W[(int64_t)pair_f[j] * n];
    /* each mode decays with its own rate mu lam_i^{alpha/2} */
    for (int64_t i = 0; i < n; ++i) coef[i] = exp(-mu * pow(lam[i], half) * t) * w[i];
    double* u = &U[j * ldu];
    const int64_t blk = 256, nblk = (n + blk - 1) / blk;
#pragma omp parallel for schedule(static)
    for (int64_t b = 0; b < nblk; ++b) {
      const int64_t r0 = b * blk, r1 = (r0 + blk < n) ? r0 + blk : n;
      for (int64_t r = r0; r < r1; ++r) u[r] = 0.0;
      for (int64_t i = 0; i < n; ++i) {
        const double ci = coef[i];
        const double* vi = &V[i * ldv];
        for (int64_t r = r0; r < r1; ++r) u[r] += vi[r] * ci;
      }
    }
  }
  free(coef);
  free(W);
  return ORACLE_OK;
}

/* ======================================================================== */
/* The generalised problem K phi = theta M phi of Sec. II eq.               */
/* (discrete_laplace) with K_ij = <grad e_i, grad e_j>, M_ij = <e_i, e_j>    */
/* for piecewise bilinear (2-D) / trilinear (3-D) basis functions e_i on the */
/* grid cells: e_i is 1 at node i, 0 at every other node, and multilinear on */
/* each cell.  The cells tile the unit square/cube (node indices -1..m per   */
/* axis); nodes outside the mask are Dirichlet zeros, so K and M are the     */
/* principal submatrices of the full-grid matrices on the dofs.              */
/* ======================================================================== */

/* 1-D integrals over one cell [0, h] of the two linear hats (local nodes 0
 * and 1): int e_a e_b = h/3 (a = b) or h/6; int e_a' e_b' = 1/h or -1/h. */
static double hat_mass(int a, int b, double h) { return (a == b) ? h / 3.0 : h / 6.0; }
static double hat_stiff(int a, int b, double h) { return (a == b) ? 1.0 / h : -1.0 / h; }

/* Integrals over one cell of the products of two multilinear basis
 * functions with local corners a, b in {0,1}^dim: the mass is the product of
 * the 1-D mass integrals, the stiffness sums over the axis d carrying the
 * derivative (1-D stiffness along d, 1-D mass along the others). */
static void cell_integrals(int dim, const int* a, const int* b, double h, double* k, double* m) {
  double mass = 1.0, stiff = 0.0;
  for (int d = 0; d < dim; ++d) mass *= hat_mass(a[d], b[d], h);
  for (int d = 0; d < dim; ++d) {
    double t = hat_stiff(a[d], b[d], h);
    for (int e = 0; e < dim; ++e)
      if (e != d) t *= hat_mass(a[e], b[e], h);
    stiff += t;
  }
  *k = stiff;
  *m = mass;
}

/* CSR of K and M (same pattern: every node of the 3^dim box around a dof
 * that is itself a dof), columns ascending.  rowptr has n+1 entries, col,
 * valK, valM room for 3^dim * n.  Each entry sums the cell integrals over
 * the cells that hold both nodes.  Returns nnz. */
int64_t oracle_assemble_fem(const int32_t* idx, int dim, const int64_t* ext, double h,
                            int64_t* rowptr, int32_t* col, double* valK, double* valM) {
  const int64_t nx = ext[0], ny = ext[1], nz = (dim == 3) ? ext[2] : 1;
  int64_t nnz = 0, row = 0;
  for (int64_t z = 0; z < nz; ++z)
    for (int64_t y = 0; y < ny; ++y)
      for (int64_t x = 0; x < nx; ++x) {
        const int64_t g = x + nx * (y + ny * z);
        if (idx[g] < 0) continue;
        rowptr[row] = nnz;
        const int64_t p[3] = {x, y, z};
        const int zlo = (dim == 3) ? -1 : 0, zhi = (dim == 3) ? 1 : 0;
        for (int oz = zlo; oz <= zhi; ++oz)
          for (int oy = -1; oy <= 1; ++oy)
            for (int ox = -1; ox <= 1; ++ox) {
              const int64_t q[3] = {x + ox, y + oy, z + oz};
              if (q[0] < 0 || q[0] >= nx || q[1] < 0 || q[1] >= ny || q[2] < 0 || q[2] >= nz) continue;
              const int32_t c = idx[q[0] + nx * (q[1] + ny * q[2])];
              if (c < 0) continue;
              /* cells (lower corner s) that contain both p and q: per axis
               * s_d in [max(p_d, q_d) - 1, min(p_d, q_d)] */
              double K = 0.0, M = 0.0;
              int64_t lo[3], hi[3];
              for (int d = 0; d < 3; ++d) {
                const int64_t mx = p[d] > q[d] ? p[d] : q[d], mn = p[d] < q[d] ? p[d] : q[d];
                lo[d] = mx - 1;
                hi[d] = mn;
              }
              if (dim == 2) { lo[2] = hi[2] = 0; }
              for (int64_t sz = lo[2]; sz <= hi[2]; ++sz)
                for (int64_t sy = lo[1]; sy <= hi[1]; ++sy)
                  for (int64_t sx = lo[0]; sx <= hi[0]; ++sx) {
                    const int64_t s[3] = {sx, sy, sz};
                    int a[3], b[3];
                    for (int d = 0; d < 3; ++d) {
                      a[d] = (int)(p[d] - s[d]);
                      b[d] = (int)(q[d] - s[d]);
                    }
                    double kk, mm;
                    cell_integrals(dim, a, b, h, &kk, &mm);
                    K += kk;
                    M += mm;
                  }
              col[nnz] = c;
              valK[nnz] = K;
              valM[nnz] = M;
              ++nnz;
            }
        ++row;
      }
  rowptr[row] = nnz;
  return nnz;
}

/* Dense Cholesky M = L L^T (lower triangle of M read, L written to the
 * lower triangle of Lo, zeros above).  Column by column:
 * l_jj = sqrt(m_jj - sum_k l_jk^2), l_ij = (m_ij - sum_k l_ik l_jk) / l_jj. */
static int dense_cholesky(int64_t n, const double* M, int64_t ldm, double* Lo, int64_t ldl) {
  for (int64_t j = 0; j < n; ++j) {
    for (int64_t i = 0; i < j; ++i) Lo[i + j * ldl] = 0.0;
    double s = M[j + j * ldm];
    for (int64_t k = 0; k < j; ++k) s -= Lo[j + k * ldl] * Lo[j + k * ldl];
    if (!(s > 0.0)) return ORACLE_EZEROPIVOT;
    const double ljj = sqrt(s);
    Lo[j + j * ldl] = ljj;
#pragma omp parallel for schedule(static)
    for (int64_t i = j + 1; i < n; ++i) {
      double t = M[i + j * ldm];
      for (int64_t k = 0; k < j; ++k) t -= Lo[i + k * ldl] * Lo[j + k * ldl];
      Lo[i + j * ldl] = t / ljj;
    }
  }
  return ORACLE_OK;
}

/* Generalised eigendecomposition K Phi = M Phi diag(theta), Phi^T M Phi = I,
 * theta ascending (K symmetric, M symmetric positive definite, both dense
 * with full storage).  Reduction to the standard problem: M = L L^T,
 * C = L^-1 K L^-T, C = Z diag(theta) Z^T (oracle_eig_full), Phi = L^-T Z. */
int oracle_eig_pencil(int64_t n, const double* K, int64_t ldk, const double* M, int64_t ldm,
                      double* theta, double* Phi, int64_t ldp) {
  if (n < 1 || ldk < n || ldm < n || ldp < n) return ORACLE_EINVAL;
  double* L = (double*)malloc(sizeof(double) * (size_t)n * (size_t)n);
  double* C = (double*)malloc(sizeof(double) * (size_t)n * (size_t)n);
  if (!L || !C) { free(L); free(C); return ORACLE_ENOMEM; }
  int rc = dense_cholesky(n, M, ldm, L, n);
  if (rc == ORACLE_OK) {
    /* Y = L^-1 K (forward substitution on every column of K) */
#pragma omp parallel for schedule(static)
    for (int64_t c = 0; c < n; ++c) {
      double* y = &C[c * n];
      for (int64_t i = 0; i < n; ++i) {
        double t = K[i + c * ldk];
        for (int64_t k = 0; k < i; ++k) t -= L[i + k * n] * y[k];
        y[i] = t / L[i + i * n];
      }
    }
    /* C = Y L^-T = (L^-1 Y^T)^T: forward substitution on every row of Y */
    double* T = (double*)malloc(sizeof(double) * (size_t)n * (size_t)n);
    if (!T) rc = ORACLE_ENOMEM;
    if (rc == ORACLE_OK) {
#pragma omp parallel for schedule(static)
      for (int64_t r = 0; r < n; ++r) {
        double* t = &T[r * n];  /* column r of T = row r of Y L^-T */
        for (int64_t i = 0; i < n; ++i) {
          double s = C[r + i * n];
          for (int64_t k = 0; k < i; ++k) s -= L[i + k * n] * t[k];
          t[i] = s / L[i + i * n];
        }
      }
      /* C(r, i) = T(i, r), symmetrised (C is symmetric up to rounding) */
      for (int64_t i = 0; i < n; ++i)
        for (int64_t r = 0; r < n; ++r) C[r + i * n] = 0.5 * (T[i + r * n] + T[r + i * n]);
      free(T);
      rc = oracle_eig_full(n, C, n, theta, Phi, ldp);
    }
    if (rc == ORACLE_OK) {
      /* Phi = L^-T Z: back substitution on every column */
#pragma omp parallel for schedule(static)
      for (int64_t c = 0; c < n; ++c) {
        double* z = &Phi[c * ldp];
        for (int64_t i = n - 1; i >= 0; --i) {
          double t = z[i];
          for (int64_t k = i + 1; k < n; ++k) t -= L[k + i * n] * z[k];
          z[i] = t / L[i + i * n];
        }
      }
    }
  }
  free(L);
  free(C);
  return rc;
}

/* Number of generalised eigenvalues below sigma: the negative pivots of the
 * LDL^T factorisation of K - sigma M (Sylvester's law of inertia for the
 * congruence L^-1 (K - sigma M) L^-T = C - sigma I).  K and M share the CSR
 * pattern. */
int64_t oracle_count_below_pencil(int64_t n, const int64_t* rowptr, const int32_t* col,
                                  const double* valK, const double* valM, double sigma) {
  const int64_t nnz = rowptr[n];
  double* v = (double*)malloc(sizeof(double) * (size_t)(nnz > 0 ? nnz : 1));
  if (!v) return ORACLE_ENOMEM;
  for (int64_t p = 0; p < nnz; ++p) v[p] = valK[p] - sigma * valM[p];
  const int64_t r = oracle_count_below(n, rowptr, col, v, 0.0);
  free(v);
  return r;
}

/* Spectral apply of the generalised problem, the sum v after eq.
 * (discrete_laplace) with the M-inner product: <f, phi_k> = phi_k^T M f for
 * the nodal vector f, so W = Phi^T (M F) and u_j = Phi (theta^{-alpha_j/2} .*
 * W(:, f_j)).  M in CSR. */
int oracle_frac_apply_mass(int64_t n, const double* Phi, int64_t ldp, const double* theta,
                           const int64_t* rowptr, const int32_t* col, const double* valM,
                           const double* F, int64_t ldf, int64_t m, const int32_t* pair_f,
                           const double* pair_alpha, int64_t k, double* U, int64_t ldu) {
  if (n < 0 || m < 0 || k < 0 || ldp < n || ldf < n || ldu < n) return ORACLE_EINVAL;
  for (int64_t j = 0; j < k; ++j)
    if (pair_f[j] < 0 || pair_f[j] >= m) return ORACLE_EINVAL;
  if (n == 0 || k == 0) return ORACLE_OK;
  double* B = (double*)malloc(sizeof(double) * (size_t)n * (size_t)(m ? m : 1));
  if (!B) return ORACLE_ENOMEM;
  for (int64_t c = 0; c < m; ++c) oracle_spmv(n, rowptr, col, valM, &F[c * ldf], &B[c * n]);
  const int rc = oracle_frac_apply(n, Phi, ldp, theta, B, n, m, pair_f, pair_alpha, k, U, ldu);
  free(B);
  return rc;
}

/* ======================================================================== */
/* Inertia of a symmetric tridiagonal T (d[0..n-1], off-diagonal e[0..n-2]) */
/* and bisection (Sec. III-D-2 applied to T = Q^T A Q, which is congruent   */
/* to A, so the counts are those of A).                                     */
/* ======================================================================== */

/* Number of eigenvalues of T strictly below sigma: the negative pivots of
 * T - sigma I = L D L^T, q_0 = d_0 - sigma, q_i = d_i - sigma - e_{i-1}^2 / q_{i-1}.
 * An exact zero pivot is replaced by a tiny negative number (sigma moved up by
 * an amount far below the resolution of any eigenvalue). */
int64_t oracle_sturm_count(int64_t n, const double* d, const double* e, double sigma) {
  if (n < 1) return ORACLE_EINVAL;
  int64_t neg = 0;
  double q = 0.0;
  for (int64_t i = 0; i < n; ++i) {
    q = (i == 0) ? d[0] - sigma : d[i] - sigma - e[i - 1] * e[i - 1] / q;
    if (q == 0.0) q = -1e-300;
    neg += (q < 0.0);
  }
  return neg;
}

/* Eigenvalues number k0..k1 (0-based, ascending) of T by bisection on the
 * Sturm count, starting from the Gershgorin interval; each stops when the
 * interval holds no representable midpoint or is within 2 eps of its
 * magnitude.  lam receives k1 - k0 + 1 values. */
int oracle_bisect(int64_t n, const double* d, const double* e, int64_t k0, int64_t k1, double* lam) {
  if (n < 1 || k0 < 0 || k1 >= n || k0 > k1) return ORACLE_EINVAL;
  double glo = d[0], ghi = d[0];
  for (int64_t i = 0; i < n; ++i) {
    const double r = (i > 0 ? fabs(e[i - 1]) : 0.0) + (i + 1 < n ? fabs(e[i]) : 0.0);
    if (d[i] - r < glo) glo = d[i] - r;
    if (d[i] + r > ghi) ghi = d[i] + r;
  }
  const double pad = 2.220446049250313e-16 * (fabs(glo) + fabs(ghi)) + 1e-300;
  glo -= pad;
  ghi += pad;
#pragma omp parallel for schedule(dynamic, 1)
  for (int64_t k = k0; k <= k1; ++k) {
    double lo = glo, hi = ghi;  /* count(lo) <= k < count(hi) */
    for (int it = 0; it < 4096; ++it) {
      const double mid = 0.5 * (lo + hi);
      if (mid <= lo || mid >= hi) break;
      if (hi - lo <= 2.0 * 2.220446049250313e-16 * fmax(fabs(lo), fabs(hi))) break;
      if (oracle_sturm_count(n, d, e, mid) > k) hi = mid;
      else lo = mid;
    }
    lam[k - k0] = 0.5 * (lo + hi);
  }
  return ORACLE_OK;
}
