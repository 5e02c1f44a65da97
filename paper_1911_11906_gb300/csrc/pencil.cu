// The generalised problem K phi = theta M phi of Sec. II eq. (discrete_laplace)
// with a symmetric positive definite mass matrix M (finite elements), and its
// spectral apply with the M-inner product: the coefficient of a nodal vector
// f on phi_i is phi_i^T M f, so u_j = Phi diag(theta^{-alpha_j/2}) Phi^T M f_j.
//
// Reduction to the standard problem on the GPU: M = L D L^T by the banded
// factorisation without pivoting (M is banded in the natural dof order; the
// factor fills only the band), then
//   C = D^-1/2 L^-1 K L^-T D^-1/2 (two banded forward solves with n
//       right-hand sides around one transpose, then a diagonal scaling),
//   C = Z diag(theta) Z^T by eig_full,
//   Phi = L^-T D^-1/2 Z (a scaling, then one banded backward solve),
// so that Phi^T M Phi = I and K Phi = M Phi diag(theta).  The banded solves
// give each right-hand side column to one thread and keep its last b + 1
// values in a shared-memory ring; the factor is read row-wise (forward) or
// column-wise (backward), the same addresses for the whole warp.
#include "internal.cuh"

namespace fraclap {
namespace {

constexpr int PS_NT_MAX = 64;
constexpr size_t kRingSmemMax = 200 * 1024;

// X <- L^-1 X with L unit lower of half-bandwidth ld - 1 (row band Lr); one
// column per thread, its last ld values in a shared ring (stride blockDim).
__global__ void __launch_bounds__(PS_NT_MAX)
band_fwd_solve(const double* __restrict__ Lr, int64_t ld, int64_t n, double* X, int64_t ldx, int64_t ncols) {
  extern __shared__ double ring[];  // ld x blockDim.x
  const int nt = blockDim.x;
  const int64_t j = (int64_t)blockIdx.x * nt + threadIdx.x;
  const bool active = j < ncols;
  double* x = X + (active ? j : 0) * ldx;
  double* R = ring + threadIdx.x;
  int64_t ipos = 0;  // i % ld
  for (int64_t i = 0; i < n; ++i) {
    double t = active ? x[i] : 0.0;
    const int64_t kmin = (i >= ld - 1) ? i - (ld - 1) : 0;
    const double* Li = Lr + i * ld;
    int64_t pos = ipos - (i - kmin);
    if (pos < 0) pos += ld;
    for (int64_t k = kmin; k < i; ++k) {
      t -= Li[i - k] * R[pos * nt];
      pos = (pos + 1 == ld) ? 0 : pos + 1;
    }
    R[ipos * nt] = t;
    if (active) x[i] = t;
    ipos = (ipos + 1 == ld) ? 0 : ipos + 1;
  }
}

// X <- L^-T X with L unit lower of half-bandwidth ld - 1 (column band Lb).
__global__ void __launch_bounds__(PS_NT_MAX)
band_bwd_solve(const double* __restrict__ Lb, int64_t ld, int64_t n, double* X, int64_t ldx, int64_t ncols) {
  extern __shared__ double ring[];
  const int nt = blockDim.x;
  const int64_t j = (int64_t)blockIdx.x * nt + threadIdx.x;
  const bool active = j < ncols;
  double* x = X + (active ? j : 0) * ldx;
  double* R = ring + threadIdx.x;
  int64_t ipos = (n - 1) % ld;  // i % ld
  for (int64_t i = n - 1; i >= 0; --i) {
    double t = active ? x[i] : 0.0;
    const int64_t kmax = (i + ld - 1 < n - 1) ? i + ld - 1 : n - 1;
    const double* Li = Lb + i * ld;
    int64_t pos = (ipos + 1 == ld) ? 0 : ipos + 1;
    for (int64_t k = i + 1; k <= kmax; ++k) {
      t -= Li[k - i] * R[pos * nt];
      pos = (pos + 1 == ld) ? 0 : pos + 1;
    }
    R[ipos * nt] = t;
    if (active) x[i] = t;
    ipos = (ipos == 0) ? ld - 1 : ipos - 1;
  }
}

// Y = K as a full symmetric matrix from its lower triangle.
__global__ void sym_from_lower(const double* K, int64_t ldk, int64_t n, double* Y, int64_t ldy) {
  const int64_t total = n * n;
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < total; p += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = p % n, j = p / n;
    Y[i + j * ldy] = (i >= j) ? K[i + j * ldk] : K[j + i * ldk];
  }
}

// B = A^T (n x n), 32 x 32 tiles through shared memory.  Block (32, 8).
__global__ void transpose_sq(const double* A, int64_t lda, int64_t n, double* B, int64_t ldb) {
  __shared__ double tile[32][33];
  const int64_t i0 = (int64_t)blockIdx.x * 32, j0 = (int64_t)blockIdx.y * 32;
  for (int q = threadIdx.y; q < 32; q += 8) {
    const int64_t i = i0 + threadIdx.x, j = j0 + q;
    if (i < n && j < n) tile[q][threadIdx.x] = A[i + j * lda];
  }
  __syncthreads();
  for (int q = threadIdx.y; q < 32; q += 8) {
    const int64_t i = j0 + threadIdx.x, j = i0 + q;  // B(i, j) = A(j, i)
    if (i < n && j < n) B[i + j * ldb] = tile[threadIdx.x][q];
  }
}

__global__ void inv_sqrt(const double* D, int64_t n, double* r) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) r[i] = 1.0 / sqrt(D[i]);
}

// C(i, j) *= r_i r_j (rows only when cols_too == 0).
__global__ void scale_rows_cols(double* C, int64_t ldc, int64_t n, int64_t ncols, const double* r, int cols_too) {
  const int64_t total = n * ncols;
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < total; p += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = p % n, j = p / n;
    const double s = cols_too ? r[i] * r[j] : r[i];
    C[i + j * ldc] *= s;
  }
}

// B(:, c) = M F(:, c) for the CSR matrix M; one thread per (row, column).
__global__ void csr_spmm(int64_t n, const int64_t* rowptr, const int32_t* col, const double* val, const double* F,
                         int64_t ldf, int64_t m, double* B, int64_t ldb) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t c = blockIdx.y;
  if (i >= n || c >= m) return;
  double s = 0.0;
  for (int64_t p = rowptr[i]; p < rowptr[i + 1]; ++p) s += val[p] * F[col[p] + c * ldf];
  B[i + c * ldb] = s;
}

struct PencilWork {
  double *Lb, *Lr, *D, *r, *C;
};

void pencil_take(Arena* ar, int64_t n, int64_t b, PencilWork* w) {
  const int64_t ld = b + 1;
  w->Lb = ar->take<double>(n * ld);
  w->Lr = ar->take<double>(n * ld);
  w->D = ar->take<double>(n);
  w->r = ar->take<double>(n);
  w->C = ar->take<double>(n * n);
}

size_t eig_ws_for(const fraclap_ctx* ctx, int64_t n) { return fraclap_eig_workspace_bytes(ctx, n); }

int band_solve_launch(fraclap_ctx* ctx, bool forward, const double* L, int64_t ld, int64_t n, double* X,
                      int64_t ldx, int64_t ncols, cudaStream_t st) {
  int nt = PS_NT_MAX;  // columns per CTA: as many as the ring of ld values each leaves room for
  while (nt > 4 && (size_t)ld * nt * sizeof(double) > kRingSmemMax) nt /= 2;
  const size_t smem = (size_t)ld * nt * sizeof(double);
  FL_CHECK(ctx, smem <= kRingSmemMax, FRACLAP_ERR_UNSUPPORTED, "eig_pencil: half-bandwidth %lld too large",
           (long long)(ld - 1));
  auto kern = forward ? band_fwd_solve : band_bwd_solve;
  FL_CUDA(ctx, cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kRingSmemMax));
  FL_CHECK(ctx, cdiv(ncols, nt) <= INT32_MAX, FRACLAP_ERR_UNSUPPORTED, "eig_pencil: too many columns");
  kern<<<(unsigned)cdiv(ncols, nt), nt, smem, st>>>(L, ld, n, X, ldx, ncols);
  count_launch(ctx);
  FL_CUDA(ctx, cudaGetLastError());
  return 0;
}

}  // namespace
}  // namespace fraclap

using namespace fraclap;

extern "C" size_t fraclap_eig_pencil_workspace_bytes(const fraclap_ctx* ctx, int64_t n, int64_t half_bandwidth) {
  if (!ctx || n <= 0 || half_bandwidth < 0) return 0;
  const int64_t b = std::min<int64_t>(half_bandwidth, n - 1);
  Arena ar;
  PencilWork w;
  pencil_take(&ar, n, b, &w);
  return ar.off + std::max(band_ldlt_ws(n, b), eig_ws_for(ctx, n)) + 1024;
}

extern "C" int eig_pencil(fraclap_ctx* ctx, const double* K_dev, int64_t ldk, int64_t n, const int64_t* rowptr_dev,
                          const int32_t* col_dev, const double* valM_dev, int64_t half_bandwidth, double* theta_dev,
                          double* Phi_dev, int64_t ldp, void* work_dev, size_t work_bytes,
                          fraclap_stream_t stream) {
  if (!ctx) return FRACLAP_ERR_INVALID_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  FL_CHECK(ctx, n >= 0, FRACLAP_ERR_INVALID_ARG, "eig_pencil: n < 0");
  if (n == 0) return 0;
  FL_CHECK(ctx, K_dev && rowptr_dev && col_dev && valM_dev && theta_dev && Phi_dev, FRACLAP_ERR_INVALID_ARG,
           "eig_pencil: null pointer");
  FL_CHECK(ctx, ldk >= n && ldp >= n, FRACLAP_ERR_INVALID_ARG, "eig_pencil: leading dimension < n");
  FL_CHECK(ctx, half_bandwidth >= 0, FRACLAP_ERR_INVALID_ARG, "eig_pencil: negative half-bandwidth");
  const int64_t b = std::min<int64_t>(half_bandwidth, n - 1), ld = b + 1;
  Arena ar;
  FL_TRY(get_workspace(ctx, work_dev, work_bytes, fraclap_eig_pencil_workspace_bytes(ctx, n, half_bandwidth), &ar));
  PencilWork w;
  pencil_take(&ar, n, b, &w);
  FL_CHECK(ctx, w.C != nullptr, FRACLAP_ERR_ALLOC, "eig_pencil: workspace too small");
  Arena tail = ar;  // the band factorisation's scratch, later the eigensolver's workspace
  FL_TRY(band_ldlt(ctx, n, rowptr_dev, col_dev, valM_dev, b, w.Lb, w.Lr, w.D, &tail, st));
  const unsigned g = (unsigned)std::min<int64_t>(cdiv(n * n, 256), 152 * 16);
  inv_sqrt<<<(unsigned)cdiv(n, 256), 256, 0, st>>>(w.D, n, w.r);
  count_launch(ctx);
  // Y = L^-1 K in the output buffer, then C = L^-1 Y^T = L^-1 K L^-T, scaled
  sym_from_lower<<<g, 256, 0, st>>>(K_dev, ldk, n, Phi_dev, ldp);
  count_launch(ctx);
  FL_TRY(band_solve_launch(ctx, true, w.Lr, ld, n, Phi_dev, ldp, n, st));
  transpose_sq<<<dim3((unsigned)cdiv(n, 32), (unsigned)cdiv(n, 32)), dim3(32, 8), 0, st>>>(Phi_dev, ldp, n, w.C, n);
  count_launch(ctx);
  FL_TRY(band_solve_launch(ctx, true, w.Lr, ld, n, w.C, n, n, st));
  scale_rows_cols<<<g, 256, 0, st>>>(w.C, n, n, n, w.r, 1);
  count_launch(ctx);
  FL_CUDA(ctx, cudaGetLastError());
  // C = Z diag(theta) Z^T (lower triangle of C read), Z into the output buffer
  const size_t rest = ar.cap - ar.off;
  FL_TRY(eig_full(ctx, w.C, n, n, theta_dev, Phi_dev, ldp, ar.base + ar.off, rest, nullptr, stream));
  // Phi = L^-T D^-1/2 Z
  scale_rows_cols<<<g, 256, 0, st>>>(Phi_dev, ldp, n, n, w.r, 0);
  count_launch(ctx);
  FL_TRY(band_solve_launch(ctx, false, w.Lb, ld, n, Phi_dev, ldp, n, st));
  return 0;
}

extern "C" size_t fraclap_apply_mass_workspace_bytes(const fraclap_ctx* ctx, int64_t n, int64_t m, int64_t k) {
  if (n < 0 || m < 0 || k < 0) return 0;
  return align256(sizeof(double) * (size_t)std::max<int64_t>(n, 1) * (size_t)std::max<int64_t>(m, 1)) +
         fraclap_apply_workspace_bytes_ctx(ctx, n, m, k) + 512;
}

extern "C" int frac_apply_mass(fraclap_ctx* ctx, const double* Phi_dev, int64_t ldp, const double* theta_dev,
                               int64_t n, const int64_t* rowptr_dev, const int32_t* col_dev, const double* valM_dev,
                               const double* F_dev, int64_t ldf, int64_t m, const int32_t* pair_f_dev,
                               const double* pair_alpha_dev, int64_t k, double* U_dev, int64_t ldu, void* work_dev,
                               size_t work_bytes, fraclap_stream_t stream) {
  if (!ctx) return FRACLAP_ERR_INVALID_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  FL_CHECK(ctx, n >= 0 && m >= 0 && k >= 0, FRACLAP_ERR_INVALID_ARG, "frac_apply_mass: negative size");
  if (n == 0 || k == 0) return 0;
  FL_CHECK(ctx, m >= 1 && m <= 65535, FRACLAP_ERR_UNSUPPORTED, "frac_apply_mass: 1..65535 forcings");
  FL_CHECK(ctx, rowptr_dev && col_dev && valM_dev && F_dev, FRACLAP_ERR_INVALID_ARG, "frac_apply_mass: null pointer");
  FL_CHECK(ctx, ldf >= n, FRACLAP_ERR_INVALID_ARG, "frac_apply_mass: ldf < n");
  Arena ar;
  FL_TRY(get_workspace(ctx, work_dev, work_bytes, fraclap_apply_mass_workspace_bytes(ctx, n, m, k), &ar));
  double* B = ar.take<double>(n * m);
  FL_CHECK(ctx, B != nullptr, FRACLAP_ERR_ALLOC, "frac_apply_mass: workspace too small");
  csr_spmm<<<dim3((unsigned)cdiv(n, 256), (unsigned)m), 256, 0, st>>>(n, rowptr_dev, col_dev, valM_dev, F_dev, ldf,
                                                                    m, B, n);
  count_launch(ctx);
  FL_CUDA(ctx, cudaGetLastError());
  return frac_apply(ctx, Phi_dev, ldp, theta_dev, n, B, n, m, pair_f_dev, pair_alpha_dev, k, U_dev, ldu,
                    ar.base + ar.off, ar.cap - ar.off, stream);
}
