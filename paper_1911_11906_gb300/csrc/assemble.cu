// fd_assemble: the nodal finite-difference form of Sec. II,
// eq. (discrete_laplace) (M = I, K = 5-/7-point Laplacian / h^2, homogeneous
// Dirichlet conditions of eq. (continuous_eigenproblem)).
// fem_assemble: the same equation with piecewise bilinear (2-D) / trilinear
// (3-D) basis functions on the grid cells: K_ij = <grad e_i, grad e_j> and
// M_ij = <e_i, e_j> (each a sum of cell integrals over the cells holding both
// nodes), on the 3^dim box of neighbours.
//
// HBM-bound integer work: a three-phase exclusive scan numbers the dofs
// (block counts, one-block scan of the counts, local scans plus offsets), a
// second scan turns per-row nonzero counts into the CSR row pointer, and a
// fill kernel writes each row's columns in ascending order.  The optional
// dense copy is a zero fill plus a scatter of the CSR entries.
#include "internal.cuh"

namespace fraclap {
namespace {

constexpr int SCAN_NT = 256, SCAN_ITEMS = 16, SCAN_TILE = SCAN_NT * SCAN_ITEMS;

struct Grid3 {
  int64_t nx, ny, nz;
  int dim;
};

// Number of in-mask neighbours (+1 for the node itself) of grid node g.
__device__ __forceinline__ int row_nnz(const uint8_t* mask, const Grid3& G, int64_t g) {
  const int64_t x = g % G.nx, y = (g / G.nx) % G.ny, z = g / (G.nx * G.ny);
  int c = 1;
  if (x > 0 && mask[g - 1]) ++c;
  if (x + 1 < G.nx && mask[g + 1]) ++c;
  if (y > 0 && mask[g - G.nx]) ++c;
  if (y + 1 < G.ny && mask[g + G.nx]) ++c;
  if (G.dim == 3) {
    if (z > 0 && mask[g - G.nx * G.ny]) ++c;
    if (z + 1 < G.nz && mask[g + G.nx * G.ny]) ++c;
  }
  return c;
}

// value of element i of the scanned sequence
struct MaskCount {
  const uint8_t* mask;
  __device__ int64_t operator()(int64_t i) const { return mask[i] ? 1 : 0; }
};
struct RowCount {  // per dof: nonzeros of its row (dofs listed by grid order)
  const uint8_t* mask;
  Grid3 G;
  __device__ int64_t operator()(int64_t g) const { return mask[g] ? row_nnz(mask, G, g) : 0; }
};

// In-mask nodes of the 3^dim box around grid node g (the node itself included):
// the row length of the finite-element matrices.
__device__ __forceinline__ int box_nnz(const uint8_t* mask, const Grid3& G, int64_t g) {
  const int64_t x = g % G.nx, y = (g / G.nx) % G.ny, z = g / (G.nx * G.ny);
  const int zr = (G.dim == 3) ? 1 : 0;
  int c = 0;
  for (int oz = -zr; oz <= zr; ++oz)
    for (int oy = -1; oy <= 1; ++oy)
      for (int ox = -1; ox <= 1; ++ox) {
        const int64_t qx = x + ox, qy = y + oy, qz = z + oz;
        if (qx < 0 || qx >= G.nx || qy < 0 || qy >= G.ny || qz < 0 || qz >= G.nz) continue;
        c += mask[qx + G.nx * (qy + G.ny * qz)] ? 1 : 0;
      }
  return c;
}
struct BoxRowCount {
  const uint8_t* mask;
  Grid3 G;
  __device__ int64_t operator()(int64_t g) const { return mask[g] ? box_nnz(mask, G, g) : 0; }
};

// Phase 1: per-tile totals.
template <class F>
__global__ void scan_tile_sums(F f, int64_t len, int64_t* tile_sum) {
  __shared__ int64_t warp_tot[SCAN_NT / 32];
  const int64_t base = (int64_t)blockIdx.x * SCAN_TILE;
  int64_t s = 0;
  for (int i = 0; i < SCAN_ITEMS; ++i) {
    const int64_t g = base + (int64_t)i * SCAN_NT + threadIdx.x;
    if (g < len) s += f(g);
  }
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) warp_tot[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    int64_t t = 0;
    for (int w = 0; w < SCAN_NT / 32; ++w) t += warp_tot[w];
    tile_sum[blockIdx.x] = t;
  }
}

// Phase 2: exclusive scan of the tile sums (one block); total -> *total.
__global__ void scan_tile_offsets(int64_t* tile_sum, int64_t ntiles, int64_t* total) {
  __shared__ int64_t buf[SCAN_NT];
  int64_t carry = 0;
  for (int64_t base = 0; base < ntiles; base += SCAN_NT) {
    const int64_t i = base + threadIdx.x;
    const int64_t v = (i < ntiles) ? tile_sum[i] : 0;
    buf[threadIdx.x] = v;
    __syncthreads();
    for (int o = 1; o < SCAN_NT; o <<= 1) {  // Hillis-Steele inclusive scan
      const int64_t add = (threadIdx.x >= (unsigned)o) ? buf[threadIdx.x - o] : 0;
      __syncthreads();
      buf[threadIdx.x] += add;
      __syncthreads();
    }
    if (i < ntiles) tile_sum[i] = carry + buf[threadIdx.x] - v;
    const int64_t blk_total = buf[SCAN_NT - 1];
    __syncthreads();
    carry += blk_total;
  }
  if (threadIdx.x == 0) *total = carry;
}

// Phase 3 for dof numbering: idx[g] = dof number or -1.
__global__ void number_dofs(const uint8_t* mask, int64_t len, const int64_t* tile_off,
                            int32_t* idx) {
  __shared__ int64_t buf[SCAN_NT];
  const int64_t base = (int64_t)blockIdx.x * SCAN_TILE + (int64_t)threadIdx.x * SCAN_ITEMS;
  int64_t local = 0;
  for (int i = 0; i < SCAN_ITEMS; ++i) {
    const int64_t g = base + i;
    if (g < len && mask[g]) ++local;
  }
  buf[threadIdx.x] = local;
  __syncthreads();
  for (int o = 1; o < SCAN_NT; o <<= 1) {
    const int64_t add = (threadIdx.x >= (unsigned)o) ? buf[threadIdx.x - o] : 0;
    __syncthreads();
    buf[threadIdx.x] += add;
    __syncthreads();
  }
  int64_t run = tile_off[blockIdx.x] + buf[threadIdx.x] - local;
  for (int i = 0; i < SCAN_ITEMS; ++i) {
    const int64_t g = base + i;
    if (g < len) idx[g] = mask[g] ? (int32_t)(run++) : -1;
  }
}

// Phase 3 for the row pointer: rowptr[idx[g]] = exclusive prefix of row counts.
template <class RC>
__global__ void write_rowptr(RC rc, const uint8_t* mask, int64_t len, const int64_t* tile_off,
                             const int32_t* idx, int64_t* rowptr, int64_t n) {
  __shared__ int64_t buf[SCAN_NT];
  const int64_t base = (int64_t)blockIdx.x * SCAN_TILE + (int64_t)threadIdx.x * SCAN_ITEMS;
  int64_t local = 0;
  for (int i = 0; i < SCAN_ITEMS; ++i) {
    const int64_t g = base + i;
    if (g < len && mask[g]) local += rc(g);
  }
  buf[threadIdx.x] = local;
  __syncthreads();
  for (int o = 1; o < SCAN_NT; o <<= 1) {
    const int64_t add = (threadIdx.x >= (unsigned)o) ? buf[threadIdx.x - o] : 0;
    __syncthreads();
    buf[threadIdx.x] += add;
    __syncthreads();
  }
  int64_t run = tile_off[blockIdx.x] + buf[threadIdx.x] - local;
  for (int i = 0; i < SCAN_ITEMS; ++i) {
    const int64_t g = base + i;
    if (g < len && mask[g]) {
      rowptr[idx[g]] = run;
      run += rc(g);
    }
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) rowptr[n] = 0;  // overwritten by the total below
}

__global__ void set_last(int64_t* rowptr, int64_t n, const int64_t* total) { rowptr[n] = *total; }

// CSR fill: one thread per grid node.
__global__ void fill_csr(const uint8_t* mask, Grid3 G, int64_t len, const int32_t* idx,
                         const int64_t* rowptr, int32_t* col, double* val, double diag, double off,
                         double* A, int64_t lda) {
  const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= len || !mask[g]) return;
  const int64_t x = g % G.nx, y = (g / G.nx) % G.ny, z = g / (G.nx * G.ny);
  const int64_t plane = G.nx * G.ny;
  int64_t nb[7];
  int cnt = 0;
  if (G.dim == 3 && z > 0) nb[cnt++] = g - plane;
  if (y > 0) nb[cnt++] = g - G.nx;
  if (x > 0) nb[cnt++] = g - 1;
  nb[cnt++] = g;
  if (x + 1 < G.nx) nb[cnt++] = g + 1;
  if (y + 1 < G.ny) nb[cnt++] = g + G.nx;
  if (G.dim == 3 && z + 1 < G.nz) nb[cnt++] = g + plane;
  const int32_t row = idx[g];
  int64_t p = rowptr[row];
  for (int t = 0; t < cnt; ++t) {
    const int64_t q = nb[t];
    if (!mask[q]) continue;
    const int32_t c = idx[q];
    const double v = (q == g) ? diag : off;
    col[p] = c;
    val[p] = v;
    if (A) A[(int64_t)row + (int64_t)c * lda] = v;
    ++p;
  }
}

// 1-D integrals over one cell [0, h] of the linear hats at local corners a, b:
// int e_a e_b = h/3 (a = b) or h/6, int e_a' e_b' = 1/h (a = b) or -1/h.
__device__ __forceinline__ double hat_m(int a, int b, double h) { return a == b ? __ddiv_rn(h, 3.0) : __ddiv_rn(h, 6.0); }
__device__ __forceinline__ double hat_k(int a, int b, double h) { return a == b ? __ddiv_rn(1.0, h) : __ddiv_rn(-1.0, h); }

// Finite-element CSR fill: one thread per grid node; row entries in
// ascending dof order (z, then y, then x offsets).  Entry (p, q) sums, over
// the cells s (lower corners, z outermost) holding both nodes, the cell's
// mass integral prod_d m(a_d, b_d) and stiffness integral
// sum_d k(a_d, b_d) prod_{e != d} m(a_e, b_e), with a = p - s, b = q - s;
// explicit roundings keep every product and sum a separate operation.
__global__ void fill_fem(const uint8_t* mask, Grid3 G, int64_t len, const int32_t* idx, const int64_t* rowptr,
                         int32_t* col, double* valK, double* valM, double h, double* Kd, double* Md, int64_t ld) {
  const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= len || !mask[g]) return;
  const int64_t p[3] = {g % G.nx, (g / G.nx) % G.ny, g / (G.nx * G.ny)};
  const int dim = G.dim, zr = (dim == 3) ? 1 : 0;
  const int32_t row = idx[g];
  int64_t pos = rowptr[row];
  for (int oz = -zr; oz <= zr; ++oz)
    for (int oy = -1; oy <= 1; ++oy)
      for (int ox = -1; ox <= 1; ++ox) {
        const int64_t q[3] = {p[0] + ox, p[1] + oy, p[2] + oz};
        if (q[0] < 0 || q[0] >= G.nx || q[1] < 0 || q[1] >= G.ny || q[2] < 0 || q[2] >= G.nz) continue;
        const int64_t gq = q[0] + G.nx * (q[1] + G.ny * q[2]);
        if (!mask[gq]) continue;
        int64_t lo[3], hi[3];
        for (int d = 0; d < 3; ++d) {
          lo[d] = (p[d] > q[d] ? p[d] : q[d]) - 1;
          hi[d] = (p[d] < q[d] ? p[d] : q[d]);
        }
        if (dim == 2) lo[2] = hi[2] = 0;
        double K = 0.0, M = 0.0;
        for (int64_t sz = lo[2]; sz <= hi[2]; ++sz)
          for (int64_t sy = lo[1]; sy <= hi[1]; ++sy)
            for (int64_t sx = lo[0]; sx <= hi[0]; ++sx) {
              const int64_t sc[3] = {sx, sy, sz};
              int a[3], b[3];
              for (int d = 0; d < 3; ++d) {
                a[d] = (int)(p[d] - sc[d]);
                b[d] = (int)(q[d] - sc[d]);
              }
              double mass = 1.0, stiff = 0.0;
              for (int d = 0; d < dim; ++d) mass = __dmul_rn(mass, hat_m(a[d], b[d], h));
              for (int d = 0; d < dim; ++d) {
                double t = hat_k(a[d], b[d], h);
                for (int e = 0; e < dim; ++e)
                  if (e != d) t = __dmul_rn(t, hat_m(a[e], b[e], h));
                stiff = __dadd_rn(stiff, t);
              }
              K = __dadd_rn(K, stiff);
              M = __dadd_rn(M, mass);
            }
        const int32_t c = idx[gq];
        col[pos] = c;
        valK[pos] = K;
        valM[pos] = M;
        if (Kd) Kd[(int64_t)row + (int64_t)c * ld] = K;
        if (Md) Md[(int64_t)row + (int64_t)c * ld] = M;
        ++pos;
      }
}

}  // namespace
}  // namespace fraclap

using namespace fraclap;

extern "C" int fd_assemble(fraclap_ctx* ctx, const uint8_t* mask_dev, int dim, const int64_t ext[3],
                           double h, int32_t* idx_dev, int64_t* n_out, int64_t* nnz_out,
                           int64_t* rowptr_dev, int32_t* col_dev, double* val_dev,
                           double* A_dense_dev, int64_t lda, fraclap_stream_t stream) {
  if (!ctx) return FRACLAP_ERR_INVALID_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  StageTimer timer(ctx, kStageAssemble, st);
  FL_CHECK(ctx, ext && (dim == 2 || dim == 3), FRACLAP_ERR_INVALID_ARG, "fd_assemble: dim must be 2 or 3");
  FL_CHECK(ctx, ext[0] >= 0 && ext[1] >= 0 && ext[2] >= 1 && (dim == 3 || ext[2] == 1),
           FRACLAP_ERR_INVALID_ARG, "fd_assemble: bad extents");
  FL_CHECK(ctx, h > 0.0 && h == h, FRACLAP_ERR_INVALID_ARG, "fd_assemble: h must be positive");
  const int64_t len = ext[0] * ext[1] * ext[2];
  FL_CHECK(ctx, len < ((int64_t)1 << 31), FRACLAP_ERR_UNSUPPORTED, "fd_assemble: grid too large");
  FL_CHECK(ctx, len == 0 || (mask_dev && idx_dev), FRACLAP_ERR_INVALID_ARG, "fd_assemble: null mask/idx");
  Grid3 G{ext[0], ext[1], ext[2], dim};
  const int64_t ntiles = cdiv(len, SCAN_TILE);

  // scratch: tile sums + totals, in the context workspace
  Arena ar;
  const size_t need = align256(sizeof(int64_t) * (size_t)(ntiles + 1)) + 256;
  FL_TRY(get_workspace(ctx, nullptr, 0, need, &ar));
  int64_t* tile = ar.take<int64_t>(ntiles + 1);
  int64_t* total = ar.take<int64_t>(2);

  if (rowptr_dev == nullptr) {
    FL_CHECK(ctx, n_out && nnz_out, FRACLAP_ERR_INVALID_ARG, "fd_assemble: null n_out/nnz_out");
    if (len == 0) { *n_out = 0; *nnz_out = 0; return 0; }
    scan_tile_sums<<<(unsigned)ntiles, SCAN_NT, 0, st>>>(MaskCount{mask_dev}, len, tile);
    count_launch(ctx);
    scan_tile_offsets<<<1, SCAN_NT, 0, st>>>(tile, ntiles, total);
    count_launch(ctx);
    number_dofs<<<(unsigned)ntiles, SCAN_NT, 0, st>>>(mask_dev, len, tile, idx_dev);
    count_launch(ctx);
    scan_tile_sums<<<(unsigned)ntiles, SCAN_NT, 0, st>>>(RowCount{mask_dev, G}, len, tile);
    count_launch(ctx);
    scan_tile_offsets<<<1, SCAN_NT, 0, st>>>(tile, ntiles, total + 1);
    count_launch(ctx);
    FL_CUDA(ctx, cudaGetLastError());
    int64_t host[2];
    FL_CUDA(ctx, cudaMemcpyAsync(host, total, sizeof(host), cudaMemcpyDeviceToHost, st));
    FL_CUDA(ctx, cudaStreamSynchronize(st));
    *n_out = host[0];
    *nnz_out = host[1];
    return 0;
  }
  // fill call: n from the host argument when given, else recount
  int64_t n = (n_out && *n_out >= 0) ? *n_out : -1;
  FL_CHECK(ctx, n >= 0, FRACLAP_ERR_INVALID_ARG, "fd_assemble: fill call needs *n_out from the first call");
  FL_CHECK(ctx, n == 0 || (col_dev && val_dev), FRACLAP_ERR_INVALID_ARG, "fd_assemble: null CSR buffers");
  FL_CHECK(ctx, !A_dense_dev || lda >= n, FRACLAP_ERR_INVALID_ARG, "fd_assemble: lda < n");
  if (len == 0) {
    FL_CUDA(ctx, cudaMemsetAsync(rowptr_dev, 0, sizeof(int64_t), st));
    return 0;
  }
  scan_tile_sums<<<(unsigned)ntiles, SCAN_NT, 0, st>>>(RowCount{mask_dev, G}, len, tile);
  count_launch(ctx);
  scan_tile_offsets<<<1, SCAN_NT, 0, st>>>(tile, ntiles, total + 1);
  count_launch(ctx);
  write_rowptr<<<(unsigned)ntiles, SCAN_NT, 0, st>>>(RowCount{mask_dev, G}, mask_dev, len, tile, idx_dev,
                                                     rowptr_dev, n);
  count_launch(ctx);
  set_last<<<1, 1, 0, st>>>(rowptr_dev, n, total + 1);
  count_launch(ctx);
  if (A_dense_dev && n > 0)
    FL_CUDA(ctx, cudaMemset2DAsync(A_dense_dev, (size_t)lda * sizeof(double), 0,
                                   (size_t)n * sizeof(double), (size_t)n, st));
  const double h2 = h * h;
  const double diag = (2.0 * dim) / h2, off = -1.0 / h2;
  fill_csr<<<(unsigned)cdiv(len, 256), 256, 0, st>>>(mask_dev, G, len, idx_dev, rowptr_dev, col_dev,
                                                    val_dev, diag, off, A_dense_dev, lda);
  count_launch(ctx);
  FL_CUDA(ctx, cudaGetLastError());
  return 0;
}

extern "C" int fem_assemble(fraclap_ctx* ctx, const uint8_t* mask_dev, int dim, const int64_t ext[3], double h,
                            int32_t* idx_dev, int64_t* n_out, int64_t* nnz_out, int64_t* rowptr_dev,
                            int32_t* col_dev, double* valK_dev, double* valM_dev, double* K_dense_dev,
                            double* M_dense_dev, int64_t ld, fraclap_stream_t stream) {
  if (!ctx) return FRACLAP_ERR_INVALID_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  StageTimer timer(ctx, kStageAssemble, st);
  FL_CHECK(ctx, ext && (dim == 2 || dim == 3), FRACLAP_ERR_INVALID_ARG, "fem_assemble: dim must be 2 or 3");
  FL_CHECK(ctx, ext[0] >= 0 && ext[1] >= 0 && ext[2] >= 1 && (dim == 3 || ext[2] == 1),
           FRACLAP_ERR_INVALID_ARG, "fem_assemble: bad extents");
  FL_CHECK(ctx, h > 0.0 && h == h, FRACLAP_ERR_INVALID_ARG, "fem_assemble: h must be positive");
  const int64_t len = ext[0] * ext[1] * ext[2];
  FL_CHECK(ctx, len < ((int64_t)1 << 31), FRACLAP_ERR_UNSUPPORTED, "fem_assemble: grid too large");
  FL_CHECK(ctx, len == 0 || (mask_dev && idx_dev), FRACLAP_ERR_INVALID_ARG, "fem_assemble: null mask/idx");
  Grid3 G{ext[0], ext[1], ext[2], dim};
  const int64_t ntiles = cdiv(len, SCAN_TILE);
  Arena ar;
  const size_t need = align256(sizeof(int64_t) * (size_t)(ntiles + 1)) + 256;
  FL_TRY(get_workspace(ctx, nullptr, 0, need, &ar));
  int64_t* tile = ar.take<int64_t>(ntiles + 1);
  int64_t* total = ar.take<int64_t>(2);
  if (rowptr_dev == nullptr) {
    FL_CHECK(ctx, n_out && nnz_out, FRACLAP_ERR_INVALID_ARG, "fem_assemble: null n_out/nnz_out");
    if (len == 0) { *n_out = 0; *nnz_out = 0; return 0; }
    scan_tile_sums<<<(unsigned)ntiles, SCAN_NT, 0, st>>>(MaskCount{mask_dev}, len, tile);
    count_launch(ctx);
    scan_tile_offsets<<<1, SCAN_NT, 0, st>>>(tile, ntiles, total);
    count_launch(ctx);
    number_dofs<<<(unsigned)ntiles, SCAN_NT, 0, st>>>(mask_dev, len, tile, idx_dev);
    count_launch(ctx);
    scan_tile_sums<<<(unsigned)ntiles, SCAN_NT, 0, st>>>(BoxRowCount{mask_dev, G}, len, tile);
    count_launch(ctx);
    scan_tile_offsets<<<1, SCAN_NT, 0, st>>>(tile, ntiles, total + 1);
    count_launch(ctx);
    FL_CUDA(ctx, cudaGetLastError());
    int64_t host[2];
    FL_CUDA(ctx, cudaMemcpyAsync(host, total, sizeof(host), cudaMemcpyDeviceToHost, st));
    FL_CUDA(ctx, cudaStreamSynchronize(st));
    *n_out = host[0];
    *nnz_out = host[1];
    return 0;
  }
  const int64_t n = (n_out && *n_out >= 0) ? *n_out : -1;
  FL_CHECK(ctx, n >= 0, FRACLAP_ERR_INVALID_ARG, "fem_assemble: fill call needs *n_out from the first call");
  FL_CHECK(ctx, n == 0 || (col_dev && valK_dev && valM_dev), FRACLAP_ERR_INVALID_ARG, "fem_assemble: null CSR buffers");
  FL_CHECK(ctx, (!K_dense_dev && !M_dense_dev) || ld >= n, FRACLAP_ERR_INVALID_ARG, "fem_assemble: ld < n");
  if (len == 0) {
    FL_CUDA(ctx, cudaMemsetAsync(rowptr_dev, 0, sizeof(int64_t), st));
    return 0;
  }
  scan_tile_sums<<<(unsigned)ntiles, SCAN_NT, 0, st>>>(BoxRowCount{mask_dev, G}, len, tile);
  count_launch(ctx);
  scan_tile_offsets<<<1, SCAN_NT, 0, st>>>(tile, ntiles, total + 1);
  count_launch(ctx);
  write_rowptr<<<(unsigned)ntiles, SCAN_NT, 0, st>>>(BoxRowCount{mask_dev, G}, mask_dev, len, tile, idx_dev,
                                                     rowptr_dev, n);
  count_launch(ctx);
  set_last<<<1, 1, 0, st>>>(rowptr_dev, n, total + 1);
  count_launch(ctx);
  for (double* D : {K_dense_dev, M_dense_dev})
    if (D && n > 0)
      FL_CUDA(ctx, cudaMemset2DAsync(D, (size_t)ld * sizeof(double), 0, (size_t)n * sizeof(double), (size_t)n, st));
  fill_fem<<<(unsigned)cdiv(len, 256), 256, 0, st>>>(mask_dev, G, len, idx_dev, rowptr_dev, col_dev, valK_dev,
                                                    valM_dev, h, K_dense_dev, M_dense_dev, ld);
  count_launch(ctx);
  FL_CUDA(ctx, cudaGetLastError());
  return 0;
}
