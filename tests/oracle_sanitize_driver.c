/*
 * Exercises every entry point of the C oracle on tiny and edge-case inputs,
 * for a build with AddressSanitizer and UndefinedBehaviorSanitizer (see
 * tests/test_oracle_sanitize.py).  Return codes and a few values are checked
 * here; the numerics themselves are pinned by the Python tests.  Exit status
 * 0 and "ok" on success.
 */
#include <math.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

int64_t oracle_number_dofs(const uint8_t* mask, int64_t ngrid, int32_t* idx);
int64_t oracle_assemble_csr(const int32_t* idx, int dim, const int64_t* ext, double h,
                            int64_t* rowptr, int32_t* col, double* val);
void oracle_spmv(int64_t n, const int64_t* rowptr, const int32_t* col, const double* val,
                 const double* x, double* y);
int oracle_tridiagonalize(int64_t n, double* A, int64_t lda, double* d, double* e, double* Q,
                          int64_t ldq);
int oracle_tridiag_eig(int64_t n, double* d, double* e, double* Z, int64_t ldz, int64_t zrows,
                       int64_t max_steps);
int oracle_eig_full(int64_t n, const double* A, int64_t lda, double* lam, double* V, int64_t ldv);
int oracle_eig_jacobi(int64_t n, const double* A, int64_t lda, double* lam, double* V,
                      int64_t ldv, int max_sweeps);
int64_t oracle_count_below(int64_t n, const int64_t* rowptr, const int32_t* col,
                           const double* val, double sigma);
int oracle_band_solve(int64_t n, const int64_t* rowptr, const int32_t* col, const double* val,
                      const double* f, double* u);
int oracle_frac_apply(int64_t n, const double* V, int64_t ldv, const double* lam, const double* F,
                      int64_t ldf, int64_t m, const int32_t* pair_f, const double* pair_alpha,
                      int64_t k, double* U, int64_t ldu);
int oracle_frac_diffusion(int64_t n, const double* V, int64_t ldv, const double* lam,
                          const double* U0, int64_t ldu0, int64_t m, const int32_t* pair_f,
                          const double* pair_alpha, const double* pair_t, double mu, int64_t k,
                          double* U, int64_t ldu);

int64_t oracle_assemble_fem(const int32_t* idx, int dim, const int64_t* ext, double h, int64_t* rowptr,
                            int32_t* col, double* valK, double* valM);
int oracle_eig_pencil(int64_t n, const double* K, int64_t ldk, const double* M, int64_t ldm,
                      double* theta, double* Phi, int64_t ldp);
int64_t oracle_count_below_pencil(int64_t n, const int64_t* rowptr, const int32_t* col,
                                  const double* valK, const double* valM, double sigma);
int oracle_frac_apply_mass(int64_t n, const double* Phi, int64_t ldp, const double* theta,
                           const int64_t* rowptr, const int32_t* col, const double* valM,
                           const double* F, int64_t ldf, int64_t m, const int32_t* pair_f,
                           const double* pair_alpha, int64_t k, double* U, int64_t ldu);

int64_t oracle_sturm_count(int64_t n, const double* d, const double* e, double sigma);
int oracle_bisect(int64_t n, const double* d, const double* e, int64_t k0, int64_t k1, double* lam);

static int failures = 0;
#define CHECK(cond)                                                   \
  do {                                                                \
    if (!(cond)) {                                                    \
      fprintf(stderr, "check failed at line %d: %s\n", __LINE__, #cond); \
      ++failures;                                                     \
    }                                                                 \
  } while (0)

/* Assembles a mask (x fastest) and returns n; the CSR arrays are malloc'd. */
static int64_t assemble(const uint8_t* mask, int dim, const int64_t ext[3], double h, int64_t** rowptr,
                        int32_t** col, double** val) {
  const int64_t ngrid = ext[0] * ext[1] * ext[2];
  int32_t* idx = malloc(sizeof(int32_t) * (size_t)ngrid);
  const int64_t n = oracle_number_dofs(mask, ngrid, idx);
  *rowptr = malloc(sizeof(int64_t) * (size_t)(n + 1));
  const int64_t cap = (2 * dim + 1) * (n > 0 ? n : 1);
  *col = malloc(sizeof(int32_t) * (size_t)cap);
  *val = malloc(sizeof(double) * (size_t)cap);
  const int64_t nnz = oracle_assemble_csr(idx, dim, ext, h, *rowptr, *col, *val);
  CHECK(nnz >= n && nnz <= cap);
  free(idx);
  return n;
}

static void dense_from_csr(int64_t n, const int64_t* rowptr, const int32_t* col, const double* val,
                           double* A) {
  memset(A, 0, sizeof(double) * (size_t)(n * n));
  for (int64_t i = 0; i < n; ++i)
    for (int64_t p = rowptr[i]; p < rowptr[i + 1]; ++p) A[i + (int64_t)col[p] * n] = val[p];
}

/* The finite-element generalised problem on the same mask. */
static void run_fem(const uint8_t* mask, int dim, const int64_t ext[3], double h) {
  const int64_t ngrid = ext[0] * ext[1] * ext[2];
  int32_t* idx = malloc(sizeof(int32_t) * (size_t)ngrid);
  const int64_t n = oracle_number_dofs(mask, ngrid, idx);
  const int64_t cap = (dim == 3 ? 27 : 9) * (n > 0 ? n : 1);
  int64_t* rowptr = malloc(sizeof(int64_t) * (size_t)(n + 1));
  int32_t* col = malloc(sizeof(int32_t) * (size_t)cap);
  double* vk = malloc(sizeof(double) * (size_t)cap);
  double* vm = malloc(sizeof(double) * (size_t)cap);
  const int64_t nnz = oracle_assemble_fem(idx, dim, ext, h, rowptr, col, vk, vm);
  CHECK(nnz >= n && nnz <= cap);
  if (n > 0) {
    double* K = malloc(sizeof(double) * (size_t)(n * n));
    double* M = malloc(sizeof(double) * (size_t)(n * n));
    double* Phi = malloc(sizeof(double) * (size_t)(n * n));
    double* th = malloc(sizeof(double) * (size_t)n);
    dense_from_csr(n, rowptr, col, vk, K);
    dense_from_csr(n, rowptr, col, vm, M);
    CHECK(oracle_eig_pencil(n, K, n, M, n, th, Phi, n) == 0);
    CHECK(oracle_count_below_pencil(n, rowptr, col, vk, vm, 0.5 * th[0]) == 0);
    CHECK(oracle_count_below_pencil(n, rowptr, col, vk, vm, 2.0 * th[n - 1]) == n);
    double* F = malloc(sizeof(double) * (size_t)(2 * n));
    double* U = malloc(sizeof(double) * (size_t)(3 * n));
    for (int64_t i = 0; i < 2 * n; ++i) F[i] = cos(0.7 * (double)i);
    int32_t pf[3] = {1, 0, 1};
    double pa[3] = {1.0, 0.0, 2.0};
    CHECK(oracle_frac_apply_mass(n, Phi, n, th, rowptr, col, vm, F, n, 2, pf, pa, 3, U, n) == 0);
    int32_t bad[1] = {-1};
    CHECK(oracle_frac_apply_mass(n, Phi, n, th, rowptr, col, vm, F, n, 2, bad, pa, 1, U, n) != 0);
    /* an indefinite "mass" matrix has no Cholesky factor */
    for (int64_t i = 0; i < n * n; ++i) M[i] = -M[i];
    CHECK(oracle_eig_pencil(n, K, n, M, n, th, Phi, n) != 0);
    free(K);
    free(M);
    free(Phi);
    free(th);
    free(F);
    free(U);
  }
  free(idx);
  free(rowptr);
  free(col);
  free(vk);
  free(vm);
}

static void run_problem(const uint8_t* mask, int dim, const int64_t ext[3], double h) {
  run_fem(mask, dim, ext, h);
  int64_t* rowptr;
  int32_t* col;
  double* val;
  const int64_t n = assemble(mask, dim, ext, h, &rowptr, &col, &val);
  if (n == 0) {
    CHECK(rowptr[0] == 0);
    CHECK(oracle_eig_full(0, NULL, 1, NULL, NULL, 1) != 0);
    free(rowptr);
    free(col);
    free(val);
    return;
  }
  double* A = malloc(sizeof(double) * (size_t)(n * n));
  double* V = malloc(sizeof(double) * (size_t)(n * n));
  double* V2 = malloc(sizeof(double) * (size_t)(n * n));
  double* lam = malloc(sizeof(double) * (size_t)n);
  double* lam2 = malloc(sizeof(double) * (size_t)n);
  double* d = malloc(sizeof(double) * (size_t)n);
  double* e = calloc((size_t)n, sizeof(double));
  double* x = malloc(sizeof(double) * (size_t)n);
  double* y = malloc(sizeof(double) * (size_t)n);
  dense_from_csr(n, rowptr, col, val, A);
  for (int64_t i = 0; i < n; ++i) x[i] = 1.0 + 0.25 * (double)(i % 5);
  oracle_spmv(n, rowptr, col, val, x, y);

  double* W = malloc(sizeof(double) * (size_t)(n * n));
  memcpy(W, A, sizeof(double) * (size_t)(n * n));
  CHECK(oracle_tridiagonalize(n, W, n, d, e, V, n) == 0);
  {
    double* tl = malloc(sizeof(double) * (size_t)n);
    CHECK(oracle_bisect(n, d, e, 0, n - 1, tl) == 0);
    CHECK(oracle_sturm_count(n, d, e, tl[0] - 1.0) == 0);
    CHECK(oracle_sturm_count(n, d, e, tl[n - 1] + 1.0) == n);
    CHECK(oracle_bisect(n, d, e, 0, n, tl) != 0);
    free(tl);
  }
  CHECK(oracle_tridiag_eig(n, d, e, V, n, n, 30 * n + 30) == 0);
  CHECK(oracle_eig_full(n, A, n, lam, V, n) == 0);
  CHECK(oracle_eig_jacobi(n, A, n, lam2, V2, n, 100) == 0);
  for (int64_t i = 0; i < n; ++i) CHECK(fabs(lam[i] - lam2[i]) <= 1e-10 * lam[n - 1]);
  CHECK(oracle_count_below(n, rowptr, col, val, 0.5 * lam[0]) == 0);
  CHECK(oracle_count_below(n, rowptr, col, val, 2.0 * lam[n - 1]) == n);

  double* u = malloc(sizeof(double) * (size_t)n);
  CHECK(oracle_band_solve(n, rowptr, col, val, x, u) == 0);

  const int64_t m = 2, k = 3;
  double* F = malloc(sizeof(double) * (size_t)(n * m));
  for (int64_t i = 0; i < n * m; ++i) F[i] = sin(0.3 * (double)i);
  int32_t pf[3] = {0, 1, 1};
  double pa[3] = {0.5, 2.0, -2.0};
  double pt[3] = {0.0, 1e-3, 0.4};
  double* U = malloc(sizeof(double) * (size_t)(n * k));
  CHECK(oracle_frac_apply(n, V, n, lam, F, n, m, pf, pa, k, U, n) == 0);
  CHECK(oracle_frac_diffusion(n, V, n, lam, F, n, m, pf, pa, pt, 1.5, k, U, n) == 0);
  int32_t bad[1] = {2};
  CHECK(oracle_frac_apply(n, V, n, lam, F, n, m, bad, pa, 1, U, n) != 0);
  CHECK(oracle_frac_diffusion(n, V, n, lam, F, n, m, bad, pa, pt, 1.0, 1, U, n) != 0);
  CHECK(oracle_frac_apply(n, V, n, lam, F, n, m, pf, pa, 0, U, n) == 0);
  CHECK(oracle_frac_apply(n, V, n - 1 > 0 ? n - 1 : 0, lam, F, n, m, pf, pa, k, U, n) != 0 || n == 1);
  /* an iteration cap of zero steps must report failure when there is work to do */
  if (n > 1) {
    memcpy(W, A, sizeof(double) * (size_t)(n * n));
    CHECK(oracle_tridiagonalize(n, W, n, d, e, NULL, n) == 0);
    CHECK(oracle_tridiag_eig(n, d, e, NULL, 1, 0, 0) != 0);
  }

  free(F);
  free(U);
  free(u);
  free(W);
  free(A);
  free(V);
  free(V2);
  free(lam);
  free(lam2);
  free(d);
  free(e);
  free(x);
  free(y);
  free(rowptr);
  free(col);
  free(val);
}

int main(void) {
  /* 2-D: 5 x 4 grid with two holes */
  const uint8_t m2[20] = {1, 1, 1, 1, 1, 1, 0, 1, 1, 1, 1, 1, 1, 0, 1, 1, 1, 1, 1, 1};
  const int64_t e2[3] = {5, 4, 1};
  run_problem(m2, 2, e2, 1.0 / 6.0);
  /* 3-D: 3 x 3 x 2 block with one hole */
  uint8_t m3[18];
  for (int i = 0; i < 18; ++i) m3[i] = (i == 4) ? 0 : 1;
  const int64_t e3[3] = {3, 3, 2};
  run_problem(m3, 3, e3, 0.25);
  /* single node, and an empty mask */
  const uint8_t one[1] = {1};
  const int64_t e1[3] = {1, 1, 1};
  run_problem(one, 2, e1, 0.5);
  const uint8_t none[4] = {0, 0, 0, 0};
  const int64_t e4[3] = {2, 2, 1};
  run_problem(none, 2, e4, 1.0 / 3.0);
  /* 1-D strip: 33 nodes */
  uint8_t strip[33];
  memset(strip, 1, sizeof(strip));
  const int64_t es[3] = {33, 1, 1};
  run_problem(strip, 2, es, 1.0 / 34.0);
  if (failures) {
    fprintf(stderr, "%d checks failed\n", failures);
    return 1;
  }
  printf("ok\n");
  return 0;
}
