// Ogita-Aishima iterative refinement of a full symmetric eigendecomposition
// (T. Ogita, K. Aishima, JJIAM 35, 2018; clustered eigenvalues: JJIAM 36,
// 2019), written from the method's mathematics.  One iteration, with X the
// current approximate eigenvector matrix (FP64, n x n):
//   R = I - X^T X,  S = X^T A X   (FP64-accurate products on the tensor
//                                  cores, lower triangles)
//   l_i = s_ii / (1 - r_ii)
//   delta = 2 (||S - diag(l)||_2 + ||A||_2 ||R||_2)   (2-norms by power
//          iteration, x2, capped by the Frobenius norms; ||A||_2 <= Gershgorin)
//   E_ij = (s_ij + l_j r_ij) / (l_j - l_i)   off the clusters
//        = r_ij / 2                           inside them and on the diagonal
//   X <- X + X E                               (X E in FP32 precision: its
//                                              error is removed next time)
// then the columns are sorted by l, and every cluster is diagonalised on the
// pencil (X_c^T A X_c, X_c^T X_c): after the first-order update X_c is
// orthonormal only to second order in the outer coefficients, and the plain
// problem of X_c^T A X_c would leave mixing of order l |X_c^T X_c - I| / gap.
// A cluster is a run of sorted positions joined by "unsafe" pairs:
// |l_j - l_i| <= delta (the method's own test), or a first-order coefficient
// above the context's threshold (1e-3 by default), whose second-order error
// would spoil the quadratic convergence when the starting vectors are only
// FP32-accurate (this safeguard is ours).  Inside a run of more than 64
// positions the pairs are tested again by the first-order coefficient alone
// (ours too): delta is a bound on the whole coupling matrix, and where the
// spectrum is denser than delta it chains most of it into one cluster.  Using the lower triangles of R and
// S as symmetric matrices keeps E_ij + E_ji = r_ij, so orthogonality improves
// to first order exactly.  A enters only through products with its CSR form
// (5/7 nonzeros per row).  The eigenvalues returned are the Rayleigh
// quotients of the refined vectors.
#include <string.h>

#include <algorithm>

#include "internal.cuh"

namespace fraclap {
namespace {

// Y(:, j) = A X(:, j) for j < ncols; A in CSR.  grid (rows / 128, column chunks)
__global__ void spmm_csr(int64_t n, const int64_t* __restrict__ rowptr,
                         const int32_t* __restrict__ col, const double* __restrict__ val,
                         const double* X, int64_t ldx, int64_t ncols, double* Y, int64_t ldy) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int64_t p0 = rowptr[i], p1 = rowptr[i + 1];
  for (int64_t j = blockIdx.y; j < ncols; j += gridDim.y) {
    const double* x = X + j * ldx;
    double s = 0.0;
    for (int64_t p = p0; p < p1; ++p) s = fma(val[p], x[col[p]], s);
    Y[i + j * ldy] = s;
  }
}

// R(i,i) += 1 (R holds -X^T X on entry).
__global__ void add_identity(double* R, int64_t ldr, int64_t n) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) R[i + i * ldr] += 1.0;
}

__global__ void ritz_values(const double* S, int64_t lds, const double* R, int64_t ldr, int64_t n,
                            double* lt) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) lt[i] = S[i + i * lds] / (1.0 - R[i + i * ldr]);
}

// Partial sums of ||S - diag(l)||_F^2 and ||R||_F^2 over the lower triangles.
__global__ void frob_norms(const double* S, int64_t lds, const double* R, int64_t ldr,
                           const double* lt, int64_t n, double* acc) {
  double s2 = 0.0, r2 = 0.0;
  const int64_t total = n * n;
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < total;
       p += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = p % n, j = p / n;
    if (i < j) continue;
    const double s = S[i + j * lds], r = R[i + j * ldr];
    if (i == j) {
      s2 += (s - lt[i]) * (s - lt[i]);
      r2 += r * r;
    } else {
      s2 += 2.0 * s * s;
      r2 += 2.0 * r * r;
    }
  }
  __shared__ double red[2][32];
  s2 = warp_sum(s2);
  r2 = warp_sum(r2);
  if ((threadIdx.x & 31) == 0) {
    red[0][threadIdx.x >> 5] = s2;
    red[1][threadIdx.x >> 5] = r2;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0.0, b = 0.0;
    for (unsigned w = 0; w < blockDim.x / 32; ++w) {
      a += red[0][w];
      b += red[1][w];
    }
    atomicAdd(acc, a);
    atomicAdd(acc + 1, b);
  }
}


// y = M x for the symmetric M stored in its lower triangle, in segments of
// kSymvSeg 32 x 32 tiles (no atomics): CTA (row strip I, segment s) sums the
// row part y_row(i) = sum_{j <= i} M(i, j) x_j over the tiles J in
// [s G, s G + G) with J <= I into P[s n + i]; CTA (column strip J, segment s)
// sums the strictly lower column part y_col(j) = sum_{i > j} M(i, j) x_i
// over the tiles I in [J + s G, J + s G + G) into Q[s n + j]; segments
// without tiles write zeros, and reduce_segments adds the segments of each
// entry in a fixed order.  Thread (row lane, column group w) reads coalesced
// 256-byte column segments.  Block 256 = 32 x 8, grid 2 nt S.
constexpr int kSymvSeg = 16;
__global__ void __launch_bounds__(256) symv_segments(const double* M, int64_t ldm, int64_t n, const double* x,
                                                     double* P, double* Q, int S) {
  __shared__ double red[8][33];
  const int64_t nt = (n + 31) / 32;
  const int tx = threadIdx.x & 31, w = threadIdx.x >> 5;
  int64_t b = blockIdx.x;
  const bool colpass = b >= nt * S;
  if (colpass) b -= nt * S;
  const int64_t strip = b / S;
  const int seg = (int)(b % S);
  if (!colpass) {
    const int64_t I = strip, gi = I * 32 + tx;
    const int64_t J0 = (int64_t)seg * kSymvSeg, J1 = (J0 + kSymvSeg - 1 < I) ? J0 + kSymvSeg - 1 : I;
    double sum = 0.0;
    if (gi < n)
      for (int64_t J = J0; J <= J1; ++J)
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const int64_t gj = J * 32 + w * 4 + q;
          if (gj <= gi) sum = fma(M[gi + gj * ldm], x[gj], sum);
        }
    red[w][tx] = sum;
    __syncthreads();
    if (w == 0 && gi < n) {
      double t = 0.0;
#pragma unroll
      for (int q = 0; q < 8; ++q) t += red[q][tx];
      P[(int64_t)seg * n + gi] = t;
    }
  } else {
    const int64_t J = strip;
    const int64_t I0 = J + (int64_t)seg * kSymvSeg, I1 = (I0 + kSymvSeg - 1 < nt - 1) ? I0 + kSymvSeg - 1 : nt - 1;
    double acc[4] = {0.0, 0.0, 0.0, 0.0};
    for (int64_t I = I0; I <= I1; ++I) {
      const int64_t gi = I * 32 + tx;
      if (gi >= n) continue;
      const double xi = x[gi];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int64_t gj = J * 32 + w * 4 + q;
        if (gi > gj) acc[q] = fma(M[gi + gj * ldm], xi, acc[q]);
      }
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const double v = warp_sum(acc[q]);
      const int64_t gj = J * 32 + w * 4 + q;
      if (tx == 0 && gj < n) Q[(int64_t)seg * n + gj] = v;
    }
  }
}
// y_i = sum_s P[s n + i] + sum_s Q[s n + i] - shift_i x_i (into P's first
// segment), and each CTA's sum of y_i^2 into part[blockIdx.x].  Block 256.
__global__ void reduce_segments(double* P, const double* Q, int S, const double* shift, const double* x,
                                int64_t n, double* part) {
  __shared__ double red[8];
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  double y2 = 0.0;
  if (i < n) {
    double y = 0.0;
    for (int q = 0; q < S; ++q) y += P[(int64_t)q * n + i];
    for (int q = 0; q < S; ++q) y += Q[(int64_t)q * n + i];
    y -= shift ? shift[i] * x[i] : 0.0;
    P[i] = y;
    y2 = y * y;
  }
  y2 = warp_sum(y2);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = y2;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < 8; ++w) t += red[w];
    part[blockIdx.x] = t;
  }
}
// |y| from the CTAs' partial sums (added in order), x = y / |y|, *est = |y|.
__global__ void normalize_parts(const double* y, const double* part, int nparts, int64_t n, double* x, double* est) {
  __shared__ double nrm_sh;
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int q = 0; q < nparts; ++q) t += part[q];
    nrm_sh = sqrt(t);
  }
  __syncthreads();
  const double nrm = nrm_sh;
  const double inv = (nrm > 0.0) ? 1.0 / nrm : 0.0;
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) x[i] = y[i] * inv;
  if (threadIdx.x == 0) *est = nrm;
}


__global__ void start_vec(double* x, int64_t n) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) {
    // deterministic, sign-varying start with components in every direction
    const uint64_t h = (uint64_t)(i + 1) * 0x9E3779B97F4A7C15ull;
    x[i] = ((double)(h >> 11) * (1.0 / 9007199254740992.0) - 0.5) / sqrt((double)n);
  }
}

// Gershgorin bound of ||A||_2 (max absolute row sum), atomically maxed as bits.
__global__ void gershgorin(int64_t n, const int64_t* rowptr, const double* val,
                           unsigned long long* out) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double s = 0.0;
  for (int64_t p = rowptr[i]; p < rowptr[i + 1]; ++p) s += fabs(val[p]);
  atomicMax(out, (unsigned long long)__double_as_longlong(s));  // non-negative doubles order as bits
}

// Largest cluster diagonalised by the batched Jacobi step (one CTA each).
constexpr int kMaxCluster = 64;

// delta = 2 (||S - D||_2 + ||A||_2 ||R||_2) with the 2-norms of S - D and R
// estimated by power iteration (times a safety factor 2, the estimates being
// lower bounds) and capped by their Frobenius norms; ||A||_2 by Gershgorin.
__global__ void cluster_threshold(const double* acc, const double* est, const unsigned long long* nA,
                                  double* delta) {
  const double na = __longlong_as_double((long long)*nA);
  const double s2 = fmin(2.0 * est[0], sqrt(acc[0]));
  const double r2 = fmin(2.0 * est[1], sqrt(acc[1]));
  *delta = 2.0 * (s2 + na * r2);
}

// Unsafe pairs: |l_j - l_i| <= delta, or a first-order coefficient
// |s_ij + l r_ij| / |l_j - l_i| above tau.  Each unsafe pair (i, j) stretches
// the span starting at its smaller sorted position to its larger one.
// Second pass (big != nullptr, and only if big[n] is set): for two positions
// inside the same cluster of the first pass that is larger than kMaxCluster
// (big[pos] = its index, else -1) only the per-pair test decides.  delta
// bounds the coupling norm of the whole matrix, and where the spectrum is
// denser than delta (3-D grids at n ~ 3e4) it chains thousands of pairs
// whose first-order coefficients are all small.
__global__ void unsafe_spans(const double* S, int64_t lds, const double* R, int64_t ldr,
                             const double* lt, const int* rank, const double* delta, double tau,
                             int64_t n, const int* big, int* reach) {
  if (big && !big[n]) return;
  const int64_t total = n * n;
  const double dl = *delta;
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < total;
       p += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = p % n, j = p / n;
    if (i <= j) continue;  // strictly lower triangle
    const double g = fabs(lt[j] - lt[i]);
    const double s = S[i + j * lds], r = R[i + j * ldr];
    const double num = fmax(fabs(s + lt[j] * r), fabs(s + lt[i] * r));
    const int a = min(rank[i], rank[j]), b = max(rank[i], rank[j]);
    const bool inner = big && big[a] >= 0 && big[a] == big[b];
    // equal estimates always join (the first-order formula would divide by zero)
    if ((!inner && g <= dl) || num > tau * g || g == 0.0) atomicMax(reach + a, b);
  }
}

// reach[pos] = pos; a second pass (flag != nullptr) runs only if *flag is set.
__global__ void init_reach(int* reach, int64_t n, const int* flag) {
  if (flag && !*flag) return;
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) reach[i] = (int)i;
}

// big[pos] = cluster index of pos if its cluster has more than kMaxCluster
// members, else -1; big[n] = 1 if there is such a cluster (zeroed before).
__global__ void mark_big(const int* cid, const int* list, int64_t n, int* big) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int c = cid[i];
  const bool b = c >= 0 && list[2 * c + 1] > kMaxCluster;
  big[i] = b ? c : -1;
  if (b) big[n] = 1;
}

// Merges the spans (sorted positions) into clusters: cid[pos] = cluster
// index or -1; list = (start, size) pairs, clusters in position order;
// *count.  A second pass (flag != nullptr) runs only if *flag is set.
// reach[k] >= k, so with the prefix maximum M[k] = max(reach[0..k]) a
// cluster (or a lone position) ends at k exactly when M[k] = k: nothing at
// or before k reaches past it.  One CTA of kMergeThreads threads, each over
// a run of consecutive positions: a block scan of the runs' maxima gives
// M, a block scan of the counts of cluster starts gives the indices
// (n <= 65535).
constexpr int kMergeThreads = 1024;
__device__ __forceinline__ int block_scan_exclusive(int v, bool is_max, int* sh) {
  // exclusive scan (max or sum) over the CTA's threads in thread order
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int x = v;
  for (int o = 1; o < 32; o <<= 1) {
    const int y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x = is_max ? max(x, y) : x + y;
  }
  if (lane == 31) sh[warp] = x;
  __syncthreads();
  if (warp == 0) {
    int w = (lane < (int)(blockDim.x >> 5)) ? sh[lane] : (is_max ? INT_MIN : 0);
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, w, o);
      if (lane >= o) w = is_max ? max(w, y) : w + y;
    }
    sh[lane] = w;  // inclusive over warps
  }
  __syncthreads();
  const int before_warp = (warp == 0) ? (is_max ? INT_MIN : 0) : sh[warp - 1];
  const int excl_in_warp = __shfl_up_sync(0xffffffffu, x, 1);
  const int mine = (lane == 0) ? (is_max ? INT_MIN : 0) : excl_in_warp;
  const int r = is_max ? max(before_warp, mine) : before_warp + mine;
  __syncthreads();  // sh is reused by the next scan
  return r;
}
__global__ void __launch_bounds__(kMergeThreads) merge_spans(const int* reach, int64_t n, int* cid, int* list,
                                                             int* count, const int* flag) {
  if (flag && !*flag) return;
  __shared__ int sh[32];
  const int nn = (int)n;
  const int run = (nn + kMergeThreads - 1) / kMergeThreads;
  const int k0 = min(nn, (int)threadIdx.x * run), k1 = min(nn, k0 + run);
  // M[k] for the run: the maximum reach before it, then the running maximum
  int m = INT_MIN;
  for (int k = k0; k < k1; ++k) m = max(m, reach[k]);
  const int before = block_scan_exclusive(m, true, sh);
  // starts of clusters (segments of more than one position) in the run
  int cnt = 0;
  {
    int M = before;  // M[k0 - 1] (INT_MIN for the first run)
    for (int k = k0; k < k1; ++k) {
      const bool start = (k == 0) || (M == k - 1);
      M = max(M, reach[k]);
      if (start && M != k) ++cnt;
    }
  }
  const int first = block_scan_exclusive(cnt, false, sh);
  // cluster of each position and the clusters' starts; a run that does not
  // begin at a start continues the last cluster started before it
  {
    int M = before, c = first;
    bool in_cl = false;
    for (int k = k0; k < k1; ++k) {
      const bool start = (k == 0) || (M == k - 1);
      M = max(M, reach[k]);
      if (start) {
        in_cl = (M != k);
        if (in_cl) list[2 * c++] = k;
      } else if (k == k0) {
        in_cl = true;
      }
      cid[k] = in_cl ? c - 1 : -1;
    }
  }
  __syncthreads();  // every start is in list before the sizes are formed
  {
    int M = before, c = first;
    bool in_cl = false;
    for (int k = k0; k < k1; ++k) {
      const bool start = (k == 0) || (M == k - 1);
      M = max(M, reach[k]);
      if (start) {
        in_cl = (M != k);
        if (in_cl) ++c;
      } else if (k == k0) {
        in_cl = true;
      }
      if (in_cl && M == k) list[2 * (c - 1) + 1] = k - list[2 * (c - 1)] + 1;  // the cluster ends at k
    }
  }
  if (threadIdx.x == kMergeThreads - 1) *count = first + cnt;
}

// E (FP32) and X32 (FP32 copy of X); pairs inside one cluster get r_ij / 2.
// Tile by tile, every global access coalesced: a tile at
// or below the diagonal stages its own entries of R and S (the diagonal tile
// takes the mirror of its upper half from the staged lower half), a tile
// above it stages the tile below the diagonal that holds its entries, read
// transposed from shared memory.  Block 32 x 8, grid (nt, nt).
__global__ void __launch_bounds__(256) correction_tiles(const double* S, int64_t lds, const double* R,
                                                        int64_t ldr, const double* lt, const int* rank,
                                                        const int* cid, int64_t n, float* E, int64_t lde,
                                                        const double* X, int64_t ldx, float* X32) {
  __shared__ double rs[32][33], ss[32][33];  // [column offset][row offset] of the staged lower tile
  __shared__ double li[32], lj[32];
  __shared__ int ci[32], cj[32];
  const int tx = threadIdx.x, ty = threadIdx.y;
  const int64_t i0 = (int64_t)blockIdx.x * 32, j0 = (int64_t)blockIdx.y * 32;
  const bool below = blockIdx.x >= blockIdx.y;
  const int64_t a0 = below ? i0 : j0, b0 = below ? j0 : i0;  // staged tile: rows a0.., columns b0..
  for (int c = ty; c < 32; c += 8) {
    const int64_t a = a0 + tx, b = b0 + c;
    const bool in = a < n && b < n;
    rs[c][tx] = in ? R[a + b * ldr] : 0.0;
    ss[c][tx] = in ? S[a + b * lds] : 0.0;
  }
  if (ty == 0) {
    const int64_t i = i0 + tx, j = j0 + tx;
    li[tx] = (i < n) ? lt[i] : 0.0;
    ci[tx] = (i < n) ? cid[rank[i]] : -1;
    lj[tx] = (j < n) ? lt[j] : 0.0;
    cj[tx] = (j < n) ? cid[rank[j]] : -1;
  }
  __syncthreads();
  for (int c = ty; c < 32; c += 8) {
    const int64_t i = i0 + tx, j = j0 + c;
    if (i >= n || j >= n) continue;
    // the lower-triangle element (max(i, j), min(i, j)) in the staged tile
    const bool mine = below && (blockIdx.x != blockIdx.y || tx >= c);
    const double r = mine ? rs[c][tx] : rs[tx][c];
    const double sv = mine ? ss[c][tx] : ss[tx][c];
    double e;
    if (i == j || (ci[tx] >= 0 && ci[tx] == cj[c])) {
      e = 0.5 * r;
    } else {
      e = (sv + lj[c] * r) / (lj[c] - li[tx]);
    }
    E[i + j * lde] = (float)e;
    X32[i + j * n] = (float)X[i + j * ldx];
  }
}
__global__ void add_correction(double* X, int64_t ldx, const float* P, int64_t n) {
  const int64_t total = n * n;
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < total;
       p += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = p % n, j = p / n;
    X[i + j * ldx] += (double)P[p];
  }
}

// rank of l_i in ascending order (ties by index); O(n^2) comparisons, one thread per i
// rank[i] = #{j : lt[j] < lt[i] or (lt[j] == lt[i] and j < i)}, a permutation.
// Thread per i, the j range split over blockIdx.y in chunks staged in shared
// memory, the chunk counts added into rank (zeroed before; integer sums, so
// the order of the additions does not matter).  Block 256, grid
// (ceil(n / 256), ceil(n / kRankChunk)).
constexpr int kRankChunk = 1024;
__global__ void __launch_bounds__(256) ranks(const double* lt, int64_t n, int* rank) {
  __shared__ double sl[kRankChunk];
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t j0 = (int64_t)blockIdx.y * kRankChunk;
  const int64_t j1 = (j0 + kRankChunk < n) ? j0 + kRankChunk : n;
  for (int64_t j = j0 + threadIdx.x; j < j1; j += blockDim.x) sl[j - j0] = lt[j];
  __syncthreads();
  if (i >= n) return;
  const double v = lt[i];
  int r = 0;
  for (int64_t j = j0; j < j1; ++j) {
    const double u = sl[j - j0];
    r += (u < v) || (u == v && j < i);
  }
  if (r) atomicAdd(rank + i, r);
}

// Xs(:, rank[j]) = X(:, j); ls(rank[j]) = l_j.  grid (rows / 256, n)
__global__ void permute_columns(const double* X, int64_t ldx, const int* rank, int64_t n,
                                double* Xs, const double* lt, double* ls) {
  const int64_t j = blockIdx.y;
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t dst = rank[j];
  if (i < n) Xs[i + dst * n] = X[i + j * ldx];
  if (i == 0) ls[dst] = lt[j];
}

__global__ void copy_columns(const double* Xs, int64_t n, double* X, int64_t ldx) {
  const int64_t total = n * n;
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < total;
       p += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = p % n, j = p / n;
    X[i + j * ldx] = Xs[p];
  }
}

// Cyclic Jacobi on one symmetric c x c block (c <= 64), one CTA.
// In: Sc (ld c).  Out: Q (ld c, eigenvectors in columns), w (eigenvalues),
// both ascending.
// Stop after the iteration that starts with ||R||_2 and ||S - D||_2 / ||A||_2 below this
// (its quadratic step lands at rounding level).
constexpr double kConvergedR = 3e-9;
// BF16 slices per operand in the refinement's residual products (7: FP64).
constexpr int kRefineSlices = 7;
constexpr int kRefineFirstSlices = 5;   // first iteration (40 bits)
constexpr int kRefineSecondSlices = 6;  // second iteration (48 bits)

__device__ void cluster_jacobi_body(const double* Sc, const double* Bc, int c, double* Q, double* w,
                                    int32_t* status) {
  // Rayleigh-Ritz on the pencil (S, B), B = X_c^T X_c: B = L L^T (Cholesky),
  // C = L^-1 S L^-T, C = Y diag(mu) Y^T by parallel-order Jacobi (each round
  // applies c/2 disjoint rotations at once, round-robin pairing; for odd c
  // one index sits out each round), and Q = L^-T Y, so that X_c Q has
  // orthonormal columns even though X_c is orthonormal only to first order.
  __shared__ double a[kMaxCluster][kMaxCluster + 1];
  __shared__ double q[kMaxCluster][kMaxCluster + 1];
  __shared__ double l[kMaxCluster][kMaxCluster + 1];
  __shared__ double rc[kMaxCluster / 2], rs[kMaxCluster / 2];
  __shared__ int rp[kMaxCluster / 2], rq[kMaxCluster / 2];
  __shared__ double red[2][32];
  __shared__ int s_done;
  __shared__ int perm[kMaxCluster];
  const int tid = threadIdx.x, nt = blockDim.x;
  for (int p = tid; p < c * c; p += nt) {
    const int i = p % c, j = p / c;
    a[i][j] = 0.5 * (Sc[i + j * c] + Sc[j + i * c]);
    l[i][j] = 0.5 * (Bc[i + j * c] + Bc[j + i * c]);
  }
  __syncthreads();
  // Cholesky, column by column, in place in the lower triangle of l
  for (int j = 0; j < c; ++j) {
    if (tid == 0) {
      double d = l[j][j];
      for (int k = 0; k < j; ++k) d -= l[j][k] * l[j][k];
      if (!(d > 0.0)) {
        raise_status(status, FRACLAP_ERR_NO_CONVERGENCE);
        d = 1.0;
      }
      l[j][j] = sqrt(d);
    }
    __syncthreads();
    for (int i = j + 1 + tid; i < c; i += nt) {
      double v = l[i][j];
      for (int k = 0; k < j; ++k) v -= l[i][k] * l[j][k];
      l[i][j] = v / l[j][j];
    }
    __syncthreads();
  }
  // W = L^-1 S (in place in a, one column per thread)
  for (int m = tid; m < c; m += nt)
    for (int i = 0; i < c; ++i) {
      double v = a[i][m];
      for (int k = 0; k < i; ++k) v -= l[i][k] * a[k][m];
      a[i][m] = v / l[i][i];
    }
  __syncthreads();
  // C = L^-1 W^T (into q), then a = C symmetrised and q = I
  for (int m = tid; m < c; m += nt)
    for (int i = 0; i < c; ++i) {
      double v = a[m][i];
      for (int k = 0; k < i; ++k) v -= l[i][k] * q[k][m];
      q[i][m] = v / l[i][i];
    }
  __syncthreads();
  for (int p = tid; p < c * c; p += nt) {
    const int i = p % c, j = p / c;
    a[i][j] = 0.5 * (q[i][j] + q[j][i]);
  }
  __syncthreads();
  for (int p = tid; p < c * c; p += nt) {
    const int i = p % c, j = p / c;
    q[i][j] = (i == j) ? 1.0 : 0.0;
  }
  __syncthreads();
  const int m = c + (c & 1);  // players; index c is a bye when c is odd
  const int np = m / 2;
  for (int sweep = 0; sweep < 50; ++sweep) {
    double off = 0.0, fro = 0.0;
    for (int p = tid; p < c * c; p += nt) {
      const int i = p % c, j = p / c;
      const double v = a[i][j] * a[i][j];
      fro += v;
      if (i != j) off += v;
    }
    off = warp_sum(off);
    fro = warp_sum(fro);
    if ((tid & 31) == 0) {
      red[0][tid >> 5] = off;
      red[1][tid >> 5] = fro;
    }
    __syncthreads();
    if (tid == 0) {
      double o = 0.0, f = 0.0;
      for (int u = 0; u < nt / 32; ++u) {
        o += red[0][u];
        f += red[1][u];
      }
      s_done = (o <= 1e-30 * f) || f == 0.0;
    }
    __syncthreads();
    if (s_done) break;
    for (int r = 0; r + 1 < m; ++r) {
      if (tid < np) {
        int p, qq;
        if (tid == 0) {
          p = r;
          qq = m - 1;
        } else {
          p = (r + tid) % (m - 1);
          qq = (r - tid + (m - 1)) % (m - 1);
        }
        if (p > qq) {
          const int tmp = p;
          p = qq;
          qq = tmp;
        }
        double cs = 1.0, sn = 0.0;
        if (qq < c) {
          const double apq = a[p][qq];
          if (fabs(apq) > 1e-18 * (fabs(a[p][p]) + fabs(a[qq][qq]))) {
            const double theta = (a[qq][qq] - a[p][p]) / (2.0 * apq);
            const double t = (theta >= 0.0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
            cs = 1.0 / sqrt(t * t + 1.0);
            sn = t * cs;
          }
        }
        rp[tid] = p;
        rq[tid] = qq;
        rc[tid] = cs;
        rs[tid] = sn;
      }
      __syncthreads();
      for (int e = tid; e < np * c; e += nt) {  // columns p, q of A and of Q
        const int k = e / c, i = e % c;
        const double sn = rs[k];
        if (sn != 0.0) {
          const int p = rp[k], qq = rq[k];
          const double cs = rc[k];
          const double xp = a[i][p], xq = a[i][qq];
          a[i][p] = cs * xp - sn * xq;
          a[i][qq] = sn * xp + cs * xq;
          const double vp = q[i][p], vq = q[i][qq];
          q[i][p] = cs * vp - sn * vq;
          q[i][qq] = sn * vp + cs * vq;
        }
      }
      __syncthreads();
      for (int e = tid; e < np * c; e += nt) {  // rows p, q of A
        const int k = e / c, j = e % c;
        const double sn = rs[k];
        if (sn != 0.0) {
          const int p = rp[k], qq = rq[k];
          const double cs = rc[k];
          const double xp = a[p][j], xq = a[qq][j];
          a[p][j] = cs * xp - sn * xq;
          a[qq][j] = sn * xp + cs * xq;
        }
      }
      __syncthreads();
    }
    if (sweep == 49 && tid == 0) raise_status(status, FRACLAP_ERR_NO_CONVERGENCE);
  }
  // Q = L^-T Y (in place in q, one column per thread)
  for (int m = tid; m < c; m += nt)
    for (int i = c - 1; i >= 0; --i) {
      double v = q[i][m];
      for (int k = i + 1; k < c; ++k) v -= l[k][i] * q[k][m];
      q[i][m] = v / l[i][i];
    }
  __syncthreads();
  // ascending order (selection by thread 0), then write out
  if (tid == 0) {
    for (int i = 0; i < c; ++i) perm[i] = i;
    for (int i = 0; i + 1 < c; ++i) {
      int mm = i;
      for (int j = i + 1; j < c; ++j)
        if (a[perm[j]][perm[j]] < a[perm[mm]][perm[mm]]) mm = j;
      const int t = perm[i];
      perm[i] = perm[mm];
      perm[mm] = t;
    }
  }
  __syncthreads();
  for (int p = tid; p < c * c; p += nt) {
    const int i = p % c, j = p / c;
    Q[i + j * c] = q[i][perm[j]];
  }
  if (tid < c) w[tid] = a[perm[tid]][perm[tid]];
}

// S_q += X_q^T (A X_q) and B_q += X_q^T X_q over the row range of
// blockIdx.y (of gridDim.y), for every small cluster q (cinfo: size, first
// column, offset of its columns in AXc).  One CTA per (cluster, row range);
// rows are staged 32 at a time and the work is n c^2 per cluster.  S_q and
// B_q (ld c) must be zero on entry.
constexpr int kGramThreads = 256;
__global__ void __launch_bounds__(kGramThreads) cluster_gram(const double* X, int64_t ldx, const double* AXc,
                                                             int64_t n, const int* cinfo, double* Sall,
                                                             double* Ball) {
  constexpr int RB = 32, NT = kGramThreads, MO = kMaxCluster * kMaxCluster / NT;
  __shared__ double xs[RB][kMaxCluster + 1], ys[RB][kMaxCluster + 1];
  __shared__ double red[NT];
  const int q = blockIdx.x, tid = threadIdx.x;
  const int c = cinfo[3 * q], i0 = cinfo[3 * q + 1], off = cinfo[3 * q + 2];
  const int P = c * c;
  const int groups = (P >= NT) ? 1 : NT / P;
  const int64_t rows = (n + gridDim.y - 1) / gridDim.y;
  const int64_t rbeg = (int64_t)blockIdx.y * rows;
  const int64_t rend = (rbeg + rows < n) ? rbeg + rows : n;
  double acc[MO], accb[MO];
#pragma unroll
  for (int mo = 0; mo < MO; ++mo) {
    acc[mo] = 0.0;
    accb[mo] = 0.0;
  }
  for (int64_t r0 = rbeg; r0 < rend; r0 += RB) {
    for (int e = tid; e < RB * c; e += NT) {
      const int rr = e % RB, cc = e / RB;
      const int64_t r = r0 + rr;
      xs[rr][cc] = (r < rend) ? X[r + (int64_t)(i0 + cc) * ldx] : 0.0;
      ys[rr][cc] = (r < rend) ? AXc[r + (int64_t)(off + cc) * n] : 0.0;
    }
    __syncthreads();
    if (groups > 1) {
      if (tid < groups * P) {
        const int o = tid % P, gr = tid / P, i = o % c, j = o / c;
        double sum = acc[0], sumb = accb[0];
        for (int rr = gr; rr < RB; rr += groups) {
          sum = fma(xs[rr][i], ys[rr][j], sum);
          sumb = fma(xs[rr][i], xs[rr][j], sumb);
        }
        acc[0] = sum;
        accb[0] = sumb;
      }
    } else {
#pragma unroll
      for (int mo = 0; mo < MO; ++mo) {
        const int o = tid + NT * mo;
        if (o < P) {
          const int i = o % c, j = o / c;
          double sum = acc[mo], sumb = accb[mo];
#pragma unroll 8
          for (int rr = 0; rr < RB; ++rr) {
            sum = fma(xs[rr][i], ys[rr][j], sum);
            sumb = fma(xs[rr][i], xs[rr][j], sumb);
          }
          acc[mo] = sum;
          accb[mo] = sumb;
        }
      }
    }
    __syncthreads();
  }
  double* S = Sall + (int64_t)q * kMaxCluster * kMaxCluster;
  double* Bq = Ball + (int64_t)q * kMaxCluster * kMaxCluster;
  if (groups > 1) {
    for (int which = 0; which < 2; ++which) {
      red[tid] = (tid < groups * P) ? (which ? accb[0] : acc[0]) : 0.0;
      __syncthreads();
      if (tid < P) {
        double sum = 0.0;
        for (int gr = 0; gr < groups; ++gr) sum += red[tid + gr * P];
        atomicAdd((which ? Bq : S) + tid, sum);  // o = i + j c
      }
      __syncthreads();
    }
  } else {
#pragma unroll
    for (int mo = 0; mo < MO; ++mo) {
      const int o = tid + NT * mo;
      if (o < P) {
        atomicAdd(S + o, acc[mo]);
        atomicAdd(Bq + o, accb[mo]);
      }
    }
  }
}

// X_q <- X_q Q_q in place for every small cluster q; one CTA per (64 rows,
// cluster): the rows are staged in shared memory, so each thread reads only
// staged values before it writes its outputs.
__global__ void __launch_bounds__(256) cluster_rotate(double* X, int64_t ldx, int64_t n, const int* cinfo,
                                                      const double* Qall) {
  constexpr int RB = 64;
  __shared__ double xs[RB][kMaxCluster + 1];
  __shared__ double qs[kMaxCluster][kMaxCluster + 1];
  const int q = blockIdx.y, tid = threadIdx.x;
  const int c = cinfo[3 * q], i0 = cinfo[3 * q + 1];
  const int64_t r0 = (int64_t)blockIdx.x * RB;
  const double* Qq = Qall + (int64_t)q * kMaxCluster * kMaxCluster;
  for (int e = tid; e < RB * c; e += 256) {
    const int rr = e % RB, cc = e / RB;
    const int64_t r = r0 + rr;
    xs[rr][cc] = (r < n) ? X[r + (int64_t)(i0 + cc) * ldx] : 0.0;
  }
  for (int e = tid; e < c * c; e += 256) qs[e % c][e / c] = Qq[e];
  __syncthreads();
  const int rr = tid % RB, part = tid / RB;
  const int64_t r = r0 + rr;
  if (r < n) {
    for (int j = part; j < c; j += 256 / RB) {
      double sum = 0.0;
      for (int i = 0; i < c; ++i) sum = fma(xs[rr][i], qs[i][j], sum);
      X[r + (int64_t)(i0 + j) * ldx] = sum;
    }
  }
}

// AXc(:, t) = A X(:, src[t]) for the concatenated cluster columns t < T.
__global__ void spmm_csr_cols(int64_t n, const int64_t* __restrict__ rowptr,
                              const int32_t* __restrict__ col, const double* __restrict__ val,
                              const double* X, int64_t ldx, const int* src, int64_t T, double* Y) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int64_t p0 = rowptr[i], p1 = rowptr[i + 1];
  for (int64_t t = blockIdx.y; t < T; t += gridDim.y) {
    const double* x = X + (int64_t)src[t] * ldx;
    double s = 0.0;
    for (int64_t p = p0; p < p1; ++p) s = fma(val[p], x[col[p]], s);
    Y[i + t * n] = s;
  }
}

// One CTA per cluster: cinfo[3q] = size, cinfo[3q+1] = first sorted position;
// S_q, B_q, Q_q at Sall/Ball/Qall + q * 64 * 64 (ld = size).
__global__ void cluster_jacobi_batched(const double* Sall, const double* Ball, const int* cinfo, double* Qall,
                                       double* lambda, int32_t* status) {
  const int q = blockIdx.x;
  const int c = cinfo[3 * q], s0 = cinfo[3 * q + 1];
  const int64_t o = (int64_t)q * kMaxCluster * kMaxCluster;
  cluster_jacobi_body(Sall + o, Ball + o, c, Qall + o, lambda + s0, status);
}

// Pencil (S, I + G) to first order in G = B - I: C = S - (G S + S G) / 2
// (from the product P = G S), Q = Y - G Y / 2 (from P = G Y).  c x c, ld c.
__global__ void pencil_first_order(const double* S, const double* P, int64_t c, double* Cout) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= c * c) return;
  const int64_t i = t % c, j = t / c;
  Cout[t] = 0.5 * (S[i + j * c] + S[j + i * c]) - 0.5 * (P[i + j * c] + P[j + i * c]);
}
__global__ void vectors_first_order(double* Y, const double* P, int64_t c) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t < c * c) Y[t] -= 0.5 * P[t];
}
__global__ void minus_identity(double* G, int64_t c) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < c) G[i + i * c] -= 1.0;
}

// l_j = (x_j^T (A x_j)) / (x_j^T x_j); one block per column.
__global__ void rayleigh(const double* X, int64_t ldx, const double* AX, int64_t ldax, int64_t n,
                         double* l) {
  const int64_t j = blockIdx.x;
  const double* x = X + j * ldx;
  const double* y = AX + j * ldax;
  double num = 0.0, den = 0.0;
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
    num = fma(x[i], y[i], num);
    den = fma(x[i], x[i], den);
  }
  __shared__ double red[2][32];
  num = warp_sum(num);
  den = warp_sum(den);
  if ((threadIdx.x & 31) == 0) {
    red[0][threadIdx.x >> 5] = num;
    red[1][threadIdx.x >> 5] = den;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0.0, b = 0.0;
    for (unsigned w = 0; w < blockDim.x / 32; ++w) {
      a += red[0][w];
      b += red[1][w];
    }
    l[j] = a / b;
  }
}

}  // namespace

// Largest cluster the refinement diagonalises (clusters above 64 go through
// the FP64 dense eigensolver of this library; its workspace is sized for n).
constexpr int64_t kMaxBigCluster = 65535;

// Scratch of the batched small-cluster step: S_q, B_q and Q_q (64 x 64 each) for
// up to n/2 + 1 clusters, the column map and the cluster table.
static int64_t small_cluster_doubles(int64_t n) {
  const int64_t ns = n / 2 + 1;
  return 3 * ns * kMaxCluster * kMaxCluster + (n + 64) / 2 + (3 * ns + 64) / 2 + 64;
}

size_t refine_ws(const fraclap_ctx* ctx, int64_t n) {
  Arena ar;
  ar.take<double>(n * n);      // AX, then sorted X
  ar.take<double>(n * n);      // R
  ar.take<double>(n * n);      // S
  ar.take<float>(n * n);       // E
  ar.take<float>(n * n);       // X32
  ar.take<float>(n * n);       // P
  ar.take<double>(n);          // l
  ar.take<double>(n);          // sorted l
  ar.take<int>(n);             // ranks
  ar.take<int>(n);             // span reach
  ar.take<int>(n);             // cluster id per sorted position
  ar.take<int>(n + 1);         // big-cluster marks + flag
  ar.take<int>(2 * n + 2);     // cluster list + count
  ar.take<double>(8);          // norms, delta
  const int64_t cmax = std::min<int64_t>(n, kMaxBigCluster);
  ar.take<double>(4 * cmax * cmax + cmax);
  ar.take<double>(small_cluster_doubles(n));
  return ar.off + std::max(cluster_eig_ws(ctx, cmax), ozaki_ws(n, n, n, kRefineSlices));
}

int refine_run(fraclap_ctx* ctx, int64_t n, const int64_t* rowptr, const int32_t* col,
               const double* val, double* X, int64_t ldx, double* lambda, int iters, Arena* ar,
               cudaStream_t st) {
  double* AX = ar->take<double>(n * n);
  double* R = ar->take<double>(n * n);
  double* S = ar->take<double>(n * n);
  float* E = ar->take<float>(n * n);
  float* X32 = ar->take<float>(n * n);
  float* P = ar->take<float>(n * n);
  double* lt = ar->take<double>(n);
  double* ls = ar->take<double>(n);
  int* rank = ar->take<int>(n);
  int* reach = ar->take<int>(n);
  int* cid = ar->take<int>(n);
  int* bigm = ar->take<int>(n + 1);
  int* clist = ar->take<int>(2 * n + 2);
  double* scal = ar->take<double>(8);
  ctx->refine_stats.clear();
  const int64_t cmax = std::min<int64_t>(n, kMaxBigCluster);
  double* cbuf = ar->take<double>(4 * cmax * cmax + cmax);
  double* sbuf = ar->take<double>(small_cluster_doubles(n));
  Arena car = *ar;  // workspace of the dense eigensolver used on big clusters
  FL_CHECK(ctx, cbuf != nullptr, FRACLAP_ERR_ALLOC, "refine: workspace too small");
  const unsigned rows = (unsigned)cdiv(n, 128);
  const unsigned flat = (unsigned)std::min<int64_t>(cdiv(n * n, 256), 152 * 16);
  unsigned long long* nA = reinterpret_cast<unsigned long long*>(scal + 2);
  double* delta = scal + 3;
  using D64 = GemmDescT<double>;
  using D32 = GemmDescT<float>;
  bool converged = false;
  StageSpan span(ctx, st);
  for (int it = 0; it < iters && !converged; ++it) {
    // AX = A X
    span.start(kStageRefineNorms);
    spmm_csr<<<dim3(rows, (unsigned)std::min<int64_t>(n, 4096)), 128, 0, st>>>(n, rowptr, col, val, X, ldx, n, AX, n);
    count_launch(ctx);
    span.stop();
    // The first iteration starts from FP32 vectors (|R| ~ 1e-5) and the second
    // from |R| ~ 1e-6..1e-5: their products need about 40 and 48 bits, the later
    // iterations remove their error.  An iteration run with fewer slices never
    // counts as the converged (last) one.
    const int slices_it = (it + 1 >= iters) ? kRefineSlices
                          : (it == 0 ? kRefineFirstSlices : (it == 1 ? kRefineSecondSlices : kRefineSlices));
    // R = I - X^T X, S = X^T (A X): lower triangles, FP64-accurate products
    // from BF16 tensor-core slices (the slices live in the scratch arena)
    {
      StageTimer tm(ctx, kStageResidualGemm, st);
      Arena oz = *ar;
      FL_TRY(ozaki_gemm(ctx, true, false, n, n, n, -1.0, X, ldx, X, ldx, 0.0, R, n, slices_it, true, &oz, st));
    }
    add_identity<<<(unsigned)cdiv(n, 256), 256, 0, st>>>(R, n, n);
    count_launch(ctx);
    {
      StageTimer tm(ctx, kStageResidualGemm, st);
      Arena oz = *ar;
      FL_TRY(ozaki_gemm(ctx, true, false, n, n, n, 1.0, X, ldx, AX, n, 0.0, S, n, slices_it, true, &oz, st));
    }
    span.start(kStageRefineNorms);
    ritz_values<<<(unsigned)cdiv(n, 256), 256, 0, st>>>(S, n, R, n, n, lt);
    count_launch(ctx);
    FL_CUDA(ctx, cudaMemsetAsync(scal, 0, 8 * sizeof(double), st));
    frob_norms<<<flat, 256, 0, st>>>(S, n, R, n, lt, n, scal);
    count_launch(ctx);
    gershgorin<<<(unsigned)cdiv(n, 256), 256, 0, st>>>(n, rowptr, val, nA);
    count_launch(ctx);
    {  // 2-norm estimates of S - diag(l) and R (power iteration)
      double* xv = ls;              // reuse: n doubles
      double* yv = AX;              // reuse: first n doubles
      for (int which = 0; which < 2; ++which) {
        const double* M = which == 0 ? S : R;
        const double* shift = which == 0 ? lt : nullptr;
        start_vec<<<(unsigned)cdiv(n, 256), 256, 0, st>>>(xv, n);
        count_launch(ctx);
        const int64_t nt = cdiv(n, 32);
        const int S = (int)cdiv(nt, kSymvSeg);
        const unsigned nb = (unsigned)cdiv(n, 256);
        double* yc = AX + (int64_t)S * n;     // the segments' partial sums: 2 S n doubles of the n x n scratch
        double* part = yc + (int64_t)S * n;  // nb CTA sums of y^2
        for (int pit = 0; pit < 12; ++pit) {
          symv_segments<<<(unsigned)(2 * nt * S), 256, 0, st>>>(M, n, n, xv, yv, yc, S);
          reduce_segments<<<nb, 256, 0, st>>>(yv, yc, S, shift, xv, n, part);
          normalize_parts<<<1, 1024, 0, st>>>(yv, part, (int)nb, n, xv, scal + 4 + which);
          for (int q = 0; q < 3; ++q) count_launch(ctx);
        }
      }
    }
    cluster_threshold<<<1, 1, 0, st>>>(scal, scal + 4, nA, delta);
    count_launch(ctx);
    span.start(kStageRefineUpdate);
    // clusters from unsafe pairs, in sorted order
    FL_CUDA(ctx, cudaMemsetAsync(rank, 0, sizeof(int) * n, st));
    ranks<<<dim3((unsigned)cdiv(n, 256), (unsigned)cdiv(n, kRankChunk)), 256, 0, st>>>(lt, n, rank);
    count_launch(ctx);
    init_reach<<<(unsigned)cdiv(n, 256), 256, 0, st>>>(reach, n, nullptr);
    count_launch(ctx);
    unsafe_spans<<<flat, 256, 0, st>>>(S, n, R, n, lt, rank, delta, ctx->refine_tau, n, nullptr, reach);
    count_launch(ctx);
    merge_spans<<<1, kMergeThreads, 0, st>>>(reach, n, cid, clist + 1, clist, nullptr);
    count_launch(ctx);
    // second pass inside clusters above kMaxCluster (device-side no-op without one)
    FL_CUDA(ctx, cudaMemsetAsync(bigm + n, 0, sizeof(int), st));
    mark_big<<<(unsigned)cdiv(n, 256), 256, 0, st>>>(cid, clist + 1, n, bigm);
    init_reach<<<(unsigned)cdiv(n, 256), 256, 0, st>>>(reach, n, bigm + n);
    unsafe_spans<<<flat, 256, 0, st>>>(S, n, R, n, lt, rank, delta, ctx->refine_tau, n, bigm, reach);
    merge_spans<<<1, kMergeThreads, 0, st>>>(reach, n, cid, clist + 1, clist, bigm + n);
    for (int q = 0; q < 4; ++q) count_launch(ctx);
    correction_tiles<<<dim3((unsigned)cdiv(n, 32), (unsigned)cdiv(n, 32)), dim3(32, 8), 0, st>>>(
        S, n, R, n, lt, rank, cid, n, E, n, X, ldx, X32);
    count_launch(ctx);
    // X += X E  (product in FP32)
    FL_TRY(gemm<float>(ctx, false, false, kGemmPlain, D32{n, n, n, X32, n, E, n, P, n, nullptr, 0, nullptr, 0, 0, 1.0, 0.0}, 1, st));
    add_correction<<<flat, 256, 0, st>>>(X, ldx, P, n);
    count_launch(ctx);
    span.start(kStageRefineSort);
    // sort the columns by l
    FL_CHECK(ctx, n <= 65535, FRACLAP_ERR_UNSUPPORTED, "refine: n too large");
    permute_columns<<<dim3((unsigned)cdiv(n, 256), (unsigned)n), 256, 0, st>>>(X, ldx, rank, n, AX, lt, ls);
    count_launch(ctx);
    copy_columns<<<flat, 256, 0, st>>>(AX, n, X, ldx);
    count_launch(ctx);
    FL_CUDA(ctx, cudaMemcpyAsync(lambda, ls, sizeof(double) * n, cudaMemcpyDeviceToDevice, st));
    span.stop();
    int ncl = 0;
    double hs[8];
    FL_CUDA(ctx, cudaMemcpyAsync(&ncl, clist, sizeof(int), cudaMemcpyDeviceToHost, st));
    FL_CUDA(ctx, cudaMemcpyAsync(hs, scal, sizeof(hs), cudaMemcpyDeviceToHost, st));
    FL_CUDA(ctx, cudaStreamSynchronize(st));
    std::vector<int> cl(2 * (size_t)std::max(ncl, 0));
    if (ncl > 0) {  // on the caller's stream: other streams keep running
      FL_CUDA(ctx, cudaMemcpyAsync(cl.data(), clist + 1, sizeof(int) * 2 * ncl, cudaMemcpyDeviceToHost, st));
      FL_CUDA(ctx, cudaStreamSynchronize(st));
    }
    {
      unsigned long long nab;
      memcpy(&nab, &hs[2], sizeof(nab));
      double na;
      memcpy(&na, &nab, sizeof(na));
      int cmaxseen = 0;
      for (int q = 0; q < ncl; ++q) cmaxseen = std::max(cmaxseen, cl[2 * q + 1]);
      const double row[8] = {hs[3], hs[4], hs[5], sqrt(hs[0]), sqrt(hs[1]), na, (double)ncl, (double)cmaxseen};
      ctx->refine_stats.insert(ctx->refine_stats.end(), row, row + 8);
      // converged: this iteration started with small residuals, so its
      // quadratic step leaves them at rounding level
      converged = (hs[5] <= kConvergedR) && (hs[4] <= kConvergedR * na) && slices_it == kRefineSlices;
    }
    span.start(kStageRefineClusters);
    if (ncl > 0) {
      // clusters up to kMaxCluster: batched (gather A X_c, S_c = X_c^T A X_c,
      // Jacobi per CTA, X_c Q_c, scatter); larger ones one by one through the
      // dense FP64 eigensolver.
      std::vector<int> src, cinfo;
      int64_t T = 0;
      double* AXc = R;                      // n x T (R and S are free here)
      double* Sall = sbuf;                  // nsmall x 64 x 64
      std::vector<int> big;
      for (int q = 0; q < ncl; ++q) {
        const int i0 = cl[2 * q], c = cl[2 * q + 1];
        if (c > kMaxCluster) { big.push_back(q); continue; }
        cinfo.push_back(c);
        cinfo.push_back(i0);
        cinfo.push_back((int)T);
        for (int t = 0; t < c; ++t) src.push_back(i0 + t);
        T += c;
      }
      const int64_t ns = (int64_t)cinfo.size() / 3;
      if (ns > 0) {
        double* Ball = Sall + ns * kMaxCluster * kMaxCluster;
        double* Qall = Ball + ns * kMaxCluster * kMaxCluster;
        int* d_src = reinterpret_cast<int*>(Qall + ns * kMaxCluster * kMaxCluster);
        int* d_cinfo = d_src + ((T + 63) / 64) * 64;
        FL_CUDA(ctx, cudaMemcpyAsync(d_src, src.data(), sizeof(int) * T, cudaMemcpyHostToDevice, st));
        FL_CUDA(ctx, cudaMemcpyAsync(d_cinfo, cinfo.data(), sizeof(int) * 3 * ns, cudaMemcpyHostToDevice, st));
        FL_CHECK(ctx, ns <= 65535 && T <= 65535, FRACLAP_ERR_UNSUPPORTED, "refine: too many clustered columns");
        spmm_csr_cols<<<dim3(rows, (unsigned)std::min<int64_t>(T, 4096)), 128, 0, st>>>(n, rowptr, col, val, X, ldx,
                                                                                       d_src, T, AXc);
        count_launch(ctx);
        FL_CUDA(ctx, cudaMemsetAsync(Sall, 0, sizeof(double) * 2 * ns * kMaxCluster * kMaxCluster, st));
        cluster_gram<<<dim3((unsigned)ns, 4), kGramThreads, 0, st>>>(X, ldx, AXc, n, d_cinfo, Sall, Ball);
        count_launch(ctx);
        cluster_jacobi_batched<<<(unsigned)ns, 256, 0, st>>>(Sall, Ball, d_cinfo, Qall, lambda, ctx->d_status);
        count_launch(ctx);
        cluster_rotate<<<dim3((unsigned)cdiv(n, 64), (unsigned)ns), 256, 0, st>>>(X, ldx, n, d_cinfo, Qall);
        count_launch(ctx);
        // the host vectors must outlive the asynchronous copies
        FL_CUDA(ctx, cudaStreamSynchronize(st));
      }
      // Big clusters: the pencil (S_c, B_c), B_c = X_c^T X_c = I + G, to
      // first order in G (the basis is orthonormal to second order in the
      // first-order coefficients), through the dense FP64 eigensolver.
      double* Sc = cbuf;
      double* Qc = Sc + cmax * cmax;
      double* Gc = Qc + cmax * cmax;
      double* Pc = Gc + cmax * cmax;
      double* AXb = R;
      double* Xn = S;
      if (!big.empty()) span.start(kStageRefineBigClusters);
      for (int q : big) {
        const int i0 = cl[2 * q], c = cl[2 * q + 1];
        FL_CHECK(ctx, c <= cmax, FRACLAP_ERR_UNSUPPORTED,
                 "refine: a cluster of %d eigenvalues exceeds %lld", c, (long long)cmax);
        double* Xc = X + (int64_t)i0 * ldx;
        const unsigned cg = (unsigned)cdiv((int64_t)c * c, 256);
        const int ksplit = (int)cdiv(n, 512);
        spmm_csr<<<dim3(rows, (unsigned)std::min(c, 4096)), 128, 0, st>>>(n, rowptr, col, val, Xc, ldx, c, AXb, n);
        count_launch(ctx);
        FL_CUDA(ctx, cudaMemsetAsync(Sc, 0, sizeof(double) * c * c, st));
        FL_CUDA(ctx, cudaMemsetAsync(Gc, 0, sizeof(double) * c * c, st));
        FL_TRY(gemm<double>(ctx, true, false, kGemmPlain, D64{c, c, n, Xc, ldx, AXb, n, Sc, c, nullptr, 0, nullptr, 0, 0, 1.0, 1.0}, ksplit, st));
        FL_TRY(gemm<double>(ctx, true, false, kGemmPlain, D64{c, c, n, Xc, ldx, Xc, ldx, Gc, c, nullptr, 0, nullptr, 0, 0, 1.0, 1.0}, ksplit, st));
        minus_identity<<<(unsigned)cdiv(c, 256), 256, 0, st>>>(Gc, c);
        count_launch(ctx);
        FL_TRY(gemm<double>(ctx, false, false, kGemmPlain, D64{c, c, c, Gc, c, Sc, c, Pc, c, nullptr, 0, nullptr, 0, 0, 1.0, 0.0}, 1, st));
        pencil_first_order<<<cg, 256, 0, st>>>(Sc, Pc, c, Qc);
        count_launch(ctx);
        Arena sub = car;
        FL_TRY(cluster_eig(ctx, Qc, c, lambda + i0, Sc, &sub, st));  // Y into Sc
        FL_TRY(gemm<double>(ctx, false, false, kGemmPlain, D64{c, c, c, Gc, c, Sc, c, Pc, c, nullptr, 0, nullptr, 0, 0, 1.0, 0.0}, 1, st));
        vectors_first_order<<<cg, 256, 0, st>>>(Sc, Pc, c);
        count_launch(ctx);
        FL_TRY(gemm<double>(ctx, false, false, kGemmPlain, D64{n, c, c, Xc, ldx, Sc, c, Xn, n, nullptr, 0, nullptr, 0, 0, 1.0, 0.0}, 1, st));
        FL_CUDA(ctx, cudaMemcpy2DAsync(Xc, ldx * sizeof(double), Xn, n * sizeof(double), n * sizeof(double), c,
                                       cudaMemcpyDeviceToDevice, st));
      }
    }
    FL_CUDA(ctx, cudaGetLastError());
  }
  span.stop();
  if (iters > 0) {  // eigenvalues: Rayleigh quotients of the refined vectors, ascending
    spmm_csr<<<dim3(rows, (unsigned)std::min<int64_t>(n, 4096)), 128, 0, st>>>(n, rowptr, col, val, X, ldx, n, AX, n);
    count_launch(ctx);
    rayleigh<<<(unsigned)n, 256, 0, st>>>(X, ldx, AX, n, n, lt);
    count_launch(ctx);
    FL_CUDA(ctx, cudaMemsetAsync(rank, 0, sizeof(int) * n, st));
    ranks<<<dim3((unsigned)cdiv(n, 256), (unsigned)cdiv(n, kRankChunk)), 256, 0, st>>>(lt, n, rank);
    count_launch(ctx);
    permute_columns<<<dim3((unsigned)cdiv(n, 256), (unsigned)n), 256, 0, st>>>(X, ldx, rank, n, AX, lt, ls);
    count_launch(ctx);
    copy_columns<<<flat, 256, 0, st>>>(AX, n, X, ldx);
    count_launch(ctx);
    FL_CUDA(ctx, cudaMemcpyAsync(lambda, ls, sizeof(double) * n, cudaMemcpyDeviceToDevice, st));
    FL_CUDA(ctx, cudaGetLastError());
  }
  return 0;
}

}  // namespace fraclap
