// Stage 1 of the two-stage reduction: dense symmetric -> band of half-width b.
//
// Panel j (columns j0..j0+b-1) is factorised P = Q_j R with Q_j = I - V T V^T
// (compact WY) by a cooperative kernel: the panel's rows are split over the
// CTAs and stay in shared memory, and each Householder column costs one
// grid-wide reduction (the dot products of the pivot column with every later
// column, added by FP64 atomics, from which the reflector and its effect on
// the panel follow).  The
// trailing matrix is then updated as A22 <- Q^T A22 Q = A22 - W V^T - V W^T
// with X = A22 (V T), W = X - 1/2 V (T^T V^T X), through the GEMM engine
// (symmetric A22 read from its lower triangle; lower-triangular rank-2b
// update).  FP64 throughout; the Householder norms and scalings stay FP64.
#include <cooperative_groups.h>

#include "internal.cuh"

namespace fraclap {
namespace {

namespace cg = cooperative_groups;

constexpr int PQR_NT = 256;
constexpr int kClusterMax = 16;                  // CTAs of the cluster panel kernel (non-portable above 8)
constexpr int kPanelClusterSmemMax = 220 * 1024;  // panel rows one CTA of the cluster holds
constexpr int kPanelSmemMax = 180 * 1024;  // largest panel slice one CTA holds

// Cooperative panel QR.  P: m x bw panel (ld ldp) in the working matrix.
// On exit P holds R on and above its diagonal (the band block) and the
// reflectors below it; Vout gets the explicit unit lower-trapezoidal V
// (m x bw, ld ldv); tau[bw]; T: bw x bw upper triangular (ld bw).
template <class T>
__global__ void __launch_bounds__(PQR_NT)
panel_qr_kernel(T* P, int64_t ldp, int64_t m, int bw, T* Vout, int64_t ldv,
                double* tau, T* Tf, double* partials, double* gram, unsigned* bar,
                long long limit, int32_t* status, int64_t rows_per_cta) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* S = reinterpret_cast<T*>(smem_raw);  // rows_per_cta x bw, column-major (ld rows_per_cta)
  __shared__ double red[2 * 64 + 4];
  __shared__ double sw[64];
  __shared__ double s_coef[4];  // beta, v0, tau
  const unsigned G = gridDim.x;
  const int64_t rb = (int64_t)blockIdx.x * rows_per_cta;
  const int64_t re = (rb + rows_per_cta < m) ? rb + rows_per_cta : m;
  const int64_t nr = (re > rb) ? re - rb : 0;
  const int64_t ld = rows_per_cta;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarp = PQR_NT / 32;

  for (int c = 0; c < bw; ++c)
    for (int64_t r = tid; r < nr; r += PQR_NT) S[r + c * ld] = P[(rb + r) + c * ldp];
  __syncthreads();

  const int nref = (m < bw) ? (int)m : bw;
  const int stride = 2 * bw;
  for (int c = 0; c < nref; ++c) {
    // column sums over all CTAs: FP64 atomics into one of three buffers
    // (zeroed two columns ahead, after the barrier that ends its last use)
    double* acc = partials + (size_t)(c % 3) * stride;
    // partial dot products over this CTA's rows r >= c
    const int64_t r0 = (c > rb) ? c - rb : 0;  // first local row with global row >= c
    for (int j = c + warp; j < bw; j += nwarp) {
      double s = 0.0;
      for (int64_t r = r0 + lane; r < nr; r += 32) {
        const int64_t gr = rb + r;
        if (j == c && gr == c) continue;  // g_c is the tail sum of squares (rows > c)
        s += (double)S[r + c * ld] * (double)S[r + j * ld];
      }
      s = warp_sum(s);
      if (lane == 0 && s != 0.0) atomicAdd(acc + j, s);
    }
    if (c >= rb && c < re)
      for (int j = c + tid; j < bw; j += PQR_NT) acc[bw + j] = (double)S[(c - rb) + j * ld];
    if (!grid_barrier(bar, G, limit, status)) return;
    if (blockIdx.x == 0)
      for (int t = tid; t < stride; t += PQR_NT) partials[(size_t)((c + 2) % 3) * stride + t] = 0.0;
    for (int t = tid; t < 2 * (bw - c); t += PQR_NT) {
      const int slot = (t < bw - c) ? c + t : bw + c + (t - (bw - c));
      red[(t < bw - c) ? t : 64 + (t - (bw - c))] = __ldcg(acc + slot);
    }
    __syncthreads();
    if (tid == 0) {
      const double tail = red[0], x0 = red[64];
      double beta = x0, v0 = 1.0, tu = 0.0;
      if (tail > 0.0 && m - c > 1) {
        const double alpha = sqrt(x0 * x0 + tail);
        beta = (x0 >= 0.0) ? -alpha : alpha;
        v0 = x0 - beta;
        tu = (beta - x0) / beta;
      }
      s_coef[0] = beta;
      s_coef[1] = v0;
      s_coef[2] = tu;
      if (blockIdx.x == 0) tau[c] = tu;
    }
    __syncthreads();
    const double beta = s_coef[0], v0 = s_coef[1], tu = s_coef[2];
    // w_j = tau v^T p_j, v^T p_j = (g_j - beta p_j(c)) / v0
    for (int j = c + 1 + tid; j < bw; j += PQR_NT) {
      const double g = red[j - c], pc = red[64 + (j - c)];
      sw[j] = (tu == 0.0) ? 0.0 : tu * (g - beta * pc) / v0;
    }
    __syncthreads();
    // update own rows (global row >= c)
    const double inv_v0 = 1.0 / v0;
    for (int64_t r = r0 + tid; r < nr; r += PQR_NT) {
      const int64_t gr = rb + r;
      double vr;
      if (gr == c) {
        vr = 1.0;
        S[r + c * ld] = (T)beta;
      } else {
        vr = (tu == 0.0) ? 0.0 : (double)S[r + c * ld] * inv_v0;
        S[r + c * ld] = (T)vr;
      }
      if (tu != 0.0) {
        const T vt = (T)vr;
        for (int j = c + 1; j < bw; ++j) S[r + j * ld] -= vt * (T)sw[j];
      }
    }
    __syncthreads();
  }
  for (int c = nref; c < bw && blockIdx.x == 0 && tid == 0; ++c) tau[c] = 0.0;

  // write back the panel (R and the reflectors) and the explicit V
  for (int c = 0; c < bw; ++c)
    for (int64_t r = tid; r < nr; r += PQR_NT) {
      const int64_t gr = rb + r;
      const T s = S[r + c * ld];
      P[gr + c * ldp] = s;
      T v = T(0);
      if (c < nref) v = (gr < c) ? T(0) : (gr == c ? T(1) : s);
      Vout[gr + c * ldv] = v;
    }
  // Gram matrix V^T V (upper part) accumulated over CTAs
  for (int p = tid; p < bw * bw; p += PQR_NT) {
    const int i = p % bw, j = p / bw;
    if (i > j || j >= nref) continue;
    double s = 0.0;
    for (int64_t r = 0; r < nr; ++r) {
      const int64_t gr = rb + r;
      if (gr < j) continue;
      const double vi = (gr == i) ? 1.0 : (gr < i ? 0.0 : (double)S[r + i * ld]);
      const double vj = (gr == j) ? 1.0 : (double)S[r + j * ld];
      s += vi * vj;
    }
    if (s != 0.0) atomicAdd(&gram[i + j * bw], s);
  }
  if (!grid_barrier(bar, G, limit, status)) return;
  if (blockIdx.x != 0) return;
  // T: T(i,i) = tau_i, T(0:i, i) = -tau_i T(0:i,0:i) (V^T v_i)(0:i)
  __shared__ double Ts[64 * 64];
  __shared__ double y[64];
  for (int p = tid; p < bw * bw; p += PQR_NT) Ts[p] = 0.0;
  __syncthreads();
  for (int i = 0; i < bw; ++i) {
    const double ti = __ldcg(tau + i);
    if (tid < i) y[tid] = __ldcg(gram + tid + i * bw);
    __syncthreads();
    if (tid < i) {
      double s = 0.0;
      for (int q = tid; q < i; ++q) s += Ts[tid + q * bw] * y[q];
      Ts[tid + i * bw] = -ti * s;
    }
    if (tid == 0) Ts[i + i * bw] = ti;
    __syncthreads();
  }
  for (int p = tid; p < bw * bw; p += PQR_NT) Tf[p] = (T)Ts[p];
}

// The same panel factorisation on one thread-block cluster (up to 16 CTAs)
// when the panel fits in their shared memory: each column's partial sums are
// read from the other CTAs' shared memory (distributed shared memory) after
// one hardware cluster barrier, in the same rank order everywhere, instead of
// a grid-wide barrier and global atomics.  Partial sums are double-buffered
// by column parity, so one barrier per column suffices: a CTA writes the
// next column's partials only after the barrier that ends everyone's reads
// of the same buffer two columns back.  Writes R, the reflectors and the
// explicit V; the Gram matrix and T follow in separate kernels.
template <class T>
__global__ void __launch_bounds__(PQR_NT)
panel_qr_cluster_kernel(T* P, int64_t ldp, int64_t m, int bw, T* Vout, int64_t ldv, double* tau,
                        int64_t rows_per_cta) {
  cg::cluster_group cluster = cg::this_cluster();
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* S = reinterpret_cast<T*>(smem_raw);  // rows_per_cta x bw, column-major (ld rows_per_cta)
  __shared__ double part[2][2 * 64];
  __shared__ double red[2 * 64 + 4];
  __shared__ double sw[64];
  __shared__ T swt[64];  // sw in the working precision (converted once per column, not once per row)
  __shared__ double s_coef[4];
  const unsigned rank = cluster.block_rank(), CS = cluster.num_blocks();
  const int64_t rb = (int64_t)rank * rows_per_cta;
  const int64_t re = (rb + rows_per_cta < m) ? rb + rows_per_cta : m;
  const int64_t nr = (re > rb) ? re - rb : 0;
  const int64_t ld = rows_per_cta;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarp = PQR_NT / 32;

  for (int c = 0; c < bw; ++c)
    for (int64_t r = tid; r < nr; r += PQR_NT) S[r + c * ld] = P[(rb + r) + c * ldp];
  __syncthreads();

  const int nref = (m < bw) ? (int)m : bw;
  for (int c = 0; c < nref; ++c) {
    double* mine = part[c & 1];
    const int64_t r0 = (c > rb) ? c - rb : 0;  // first local row with global row >= c
    {
      // per-CTA partial dots in the working precision (FP64 work on ~m/16 rows
      // would occupy GB300's narrow FP64 pipe); the cluster sum is FP64.  A
      // warp takes columns j = c + warp + 8 q, all in one pass over its rows
      // (the pivot column read once, eight independent sums).
      constexpr int QMAX = 64 / 8;
      T sum[QMAX];
#pragma unroll
      for (int q = 0; q < QMAX; ++q) sum[q] = T(0);
      for (int64_t r = r0 + lane; r < nr; r += 32) {
        const int64_t gr = rb + r;
        const T pc = S[r + c * ld];
#pragma unroll
        for (int q = 0; q < QMAX; ++q) {
          const int j = c + warp + nwarp * q;
          if (j < bw && !(j == c && gr == c)) sum[q] += pc * S[r + j * ld];  // g_c: rows > c only
        }
      }
#pragma unroll
      for (int q = 0; q < QMAX; ++q) {
        T v = sum[q];
#pragma unroll
        for (int o = 16; o >= 1; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        const int j = c + warp + nwarp * q;
        if (lane == 0 && j < bw) mine[j] = (double)v;
      }
    }
    for (int j = c + tid; j < bw; j += PQR_NT) mine[bw + j] = (c >= rb && c < re) ? (double)S[(c - rb) + j * ld] : 0.0;
    cluster.sync();
    for (int t = tid; t < 2 * (bw - c); t += PQR_NT) {
      const int slot = (t < bw - c) ? c + t : bw + c + (t - (bw - c));
      double v[kClusterMax];  // all remote loads in flight, then the sum in rank order
#pragma unroll
      for (int q = 0; q < kClusterMax; ++q)
        v[q] = (q < (int)CS) ? cluster.map_shared_rank(&part[c & 1][0], q)[slot] : 0.0;
      double sum = 0.0;
#pragma unroll
      for (int q = 0; q < kClusterMax; ++q) sum += v[q];
      red[(t < bw - c) ? t : 64 + (t - (bw - c))] = sum;
    }
    __syncthreads();
    if (tid == 0) {
      const double tail = red[0], x0 = red[64];
      double beta = x0, v0 = 1.0, tu = 0.0;
      if (tail > 0.0 && m - c > 1) {
        const double alpha = sqrt(x0 * x0 + tail);
        beta = (x0 >= 0.0) ? -alpha : alpha;
        v0 = x0 - beta;
        tu = (beta - x0) / beta;
      }
      s_coef[0] = beta;
      s_coef[1] = 1.0 / v0;
      s_coef[2] = tu;
      if (rank == 0) tau[c] = tu;
    }
    __syncthreads();
    const double beta = s_coef[0], inv_v0 = s_coef[1], tu = s_coef[2];
    for (int j = c + 1 + tid; j < bw; j += PQR_NT) {
      const double g = red[j - c], pc = red[64 + (j - c)];
      sw[j] = (tu == 0.0) ? 0.0 : tu * (g - beta * pc) * inv_v0;
      swt[j] = (T)sw[j];
    }
    __syncthreads();
    for (int64_t r = r0 + tid; r < nr; r += PQR_NT) {
      const int64_t gr = rb + r;
      double vr;
      if (gr == c) {
        vr = 1.0;
        S[r + c * ld] = (T)beta;
      } else {
        vr = (tu == 0.0) ? 0.0 : (double)S[r + c * ld] * inv_v0;
        S[r + c * ld] = (T)vr;
      }
      if (tu != 0.0) {
        const T vt = (T)vr;
        for (int j = c + 1; j < bw; ++j) S[r + j * ld] -= vt * swt[j];
      }
    }
    __syncthreads();
  }
  for (int c = nref; c < bw && rank == 0 && tid == 0; ++c) tau[c] = 0.0;
  for (int c = 0; c < bw; ++c)
    for (int64_t r = tid; r < nr; r += PQR_NT) {
      const int64_t gr = rb + r;
      const T sv = S[r + c * ld];
      P[gr + c * ldp] = sv;
      T v = T(0);
      if (c < nref) v = (gr < c) ? T(0) : (gr == c ? T(1) : sv);
      Vout[gr + c * ldv] = v;
    }
  cluster.sync();  // no CTA leaves while another may still read its partial sums
}

// T of the compact WY form from tau and the Gram matrix G = V^T V (bw x bw).
// When every tau is nonzero, T^-1 = diag(1/tau) + strictly-upper(G)
// (Schreiber and Van Loan's form of H_1 ... H_bw = I - V T V^T): T is that
// triangle's inverse, formed row by row from the bottom, X(i, j) =
// -(1 / U(i, i)) sum_{i < k <= j} U(i, k) X(k, j), all columns of a row at
// once and each sum split over four lanes (one barrier per row).  Otherwise
// the column recurrence T(i, i) = tau_i, T(0:i, i) = -tau_i T(0:i, 0:i) G(0:i, i).
// One CTA of 256 threads.
template <class T>
__global__ void __launch_bounds__(PQR_NT) panel_t_kernel(const T* gram, const double* tau, int bw, T* Tf) {
  __shared__ double U[64][65];  // U(i, k), i <= k
  __shared__ double Ts[64 * 64];
  __shared__ double y[64];
  __shared__ int s_zero;
  const int tid = threadIdx.x;
  if (tid == 0) s_zero = 0;
  __syncthreads();
  for (int p = tid; p < bw * bw; p += PQR_NT) {
    const int i = p % bw, k = p / bw;
    if (i < k) U[i][k] = (double)gram[i + k * bw];
    else if (i == k) {
      const double t = tau[i];
      if (t == 0.0) s_zero = 1;
      U[i][i] = (t == 0.0) ? 1.0 : 1.0 / t;
    }
    Ts[p] = 0.0;
  }
  __syncthreads();
  if (!s_zero) {
    static_assert(PQR_NT == 256, "four lanes per column of a 64-wide panel");
    const int j = tid >> 2, part = tid & 3;  // column j, lanes 4j .. 4j + 3 of one warp
    for (int i = bw - 1; i >= 0; --i) {
      double sum = 0.0;
      if (j > i && j < bw)
        for (int k = i + 1 + part; k <= j; k += 4) sum += U[i][k] * Ts[k + j * bw];
      sum += __shfl_xor_sync(0xffffffffu, sum, 1);
      sum += __shfl_xor_sync(0xffffffffu, sum, 2);
      if (part == 0 && j < bw && j >= i) Ts[i + j * bw] = (j == i) ? 1.0 / U[i][i] : -sum / U[i][i];
      __syncthreads();
    }
  } else {
    for (int i = 0; i < bw; ++i) {
      const double ti = tau[i];
      if (tid < i) y[tid] = (double)gram[tid + i * bw];
      __syncthreads();
      if (tid < i) {
        double sum = 0.0;
        for (int q = tid; q < i; ++q) sum += Ts[tid + q * bw] * y[q];
        Ts[tid + i * bw] = -ti * sum;
      }
      if (tid == 0) Ts[i + i * bw] = ti;
      __syncthreads();
    }
  }
  for (int p = tid; p < bw * bw; p += PQR_NT) Tf[p] = (T)Ts[p];
}

// Band extraction: band(off, j) = A(j + off, j) for off <= b, 0 for b < off < ldb.
template <class T>
__global__ void extract_band(const T* A, int64_t lda, int64_t n, int b, T* band, int ldb) {
  const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= n * ldb) return;
  const int off = (int)(p % ldb);
  const int64_t j = p / ldb;
  const int64_t i = j + off;
  band[p] = (off <= b && i < n) ? A[i + j * lda] : T(0);
}

}  // namespace

int64_t stage1_panels(int64_t n, int b) { return (n > b) ? cdiv(n - b, b) : 0; }

template <class T>
int stage1_take(Arena* ar, int64_t n, int b, int G, Stage1T<T>* s) {
  s->npanel = stage1_panels(n, b);
  s->vtotal = 0;
  for (int64_t j = 0; j < s->npanel; ++j) s->vtotal += (n - j * b - b) * b;
  s->Vstore = ar->take<T>(s->vtotal);
  s->Tstore = ar->take<T>(s->npanel * b * b);
  s->tau = ar->take<double>(s->npanel * b);
  s->XT = ar->take<T>(n * b);
  s->X = ar->take<T>(n * b);
  s->Y = ar->take<T>((int64_t)b * b);
  s->Mm = ar->take<T>((int64_t)b * b);
  s->gram = ar->take<double>((int64_t)b * b);
  s->gramT = ar->take<T>((int64_t)b * b);
  s->partials = ar->take<double>(3 * 2 * (int64_t)b);
  return 0;
}

static int panel_grid(fraclap_ctx* ctx, int64_t m, int bw, size_t elem, int64_t* rows_per_cta,
                      size_t* smem) {
  int G = ctx->sm_count;
  if (m < (int64_t)G * 8) G = (int)cdiv(m, 8);
  if (G < 1) G = 1;
  *rows_per_cta = cdiv(m, G);
  G = (int)cdiv(m, *rows_per_cta);
  *smem = (size_t)(*rows_per_cta) * bw * elem;
  return G;
}

// Panel on one cluster, then G = V^T V (split over the rows) and T.  Returns
// 1 (nothing launched) when the panel does not fit in a cluster's shared
// memory or no cluster of that size can be resident; < 0 on a CUDA error.
template <class T>
int panel_cluster(fraclap_ctx* ctx, T* P, int64_t ldp, int64_t m, int b, T* V, double* tau, T* gramT, T* Tf,
                  cudaStream_t st) {
  // FP64 panels keep the grid kernel: spread over all SMs, their FP64 dot
  // products are not bound by one SM's narrow FP64 pipe
  if (sizeof(T) == 8) return 1;
  const int64_t cap = kPanelClusterSmemMax / ((int64_t)b * (int64_t)sizeof(T));
  const int limit = std::max(1, std::min(kClusterMax, ctx->sm_count));
  int CS = (int)std::max<int64_t>(cdiv(m, cap), std::min<int64_t>(limit, cdiv(m, 128)));
  if (CS > limit) return 1;
  const int64_t rows = cdiv(m, CS);
  CS = (int)cdiv(m, rows);
  const size_t smem = (size_t)rows * b * sizeof(T);
  FL_CUDA(ctx, cudaFuncSetAttribute(panel_qr_cluster_kernel<T>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1));
  FL_CUDA(ctx, cudaFuncSetAttribute(panel_qr_cluster_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    kPanelClusterSmemMax));
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)CS);
  cfg.blockDim = dim3(PQR_NT);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = (unsigned)CS;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  int clusters = 0;
  if (cudaOccupancyMaxActiveClusters(&clusters, panel_qr_cluster_kernel<T>, &cfg) != cudaSuccess || clusters < 1) {
    cudaGetLastError();
    return 1;
  }
  int bw = b;
  count_launch(ctx);
  FL_CUDA(ctx, cudaLaunchKernelEx(&cfg, panel_qr_cluster_kernel<T>, P, ldp, m, bw, V, m, tau, rows));
  using D = GemmDescT<T>;
  FL_CUDA(ctx, cudaMemsetAsync(gramT, 0, sizeof(T) * b * b, st));
  FL_TRY(gemm<T>(ctx, true, false, kGemmPlain, D{b, b, m, V, m, V, m, gramT, b, nullptr, 0, nullptr, 0, 0, 1.0, 1.0},
                 (int)std::min<int64_t>(cdiv(m, 512), 16), st));
  panel_t_kernel<T><<<1, PQR_NT, 0, st>>>(gramT, tau, b, Tf);
  count_launch(ctx);
  FL_CUDA(ctx, cudaGetLastError());
  return 0;
}

// Reduces Aw (n x n, lower triangle valid, overwritten) to band form and
// writes the band (ld 2b, offsets 0..2b-1, zero beyond b) to `band`.
template <class T>
int sy2sb_run(fraclap_ctx* ctx, T* Aw, int64_t n, int64_t lda, int b, T* band, Stage1T<T>* s,
              cudaStream_t st) {
  const int ldb = 2 * b;
  int64_t voff = 0;
  for (int64_t p = 0; p < s->npanel; ++p) {
    const int64_t j0 = p * b, m = n - j0 - b;
    T* P = Aw + (j0 + b) + j0 * lda;
    T* V = s->Vstore + voff;
    T* Tf = s->Tstore + p * b * b;
    const int crc = panel_cluster(ctx, P, lda, m, b, V, s->tau + p * b, s->gramT, Tf, st);
    if (crc < 0) return crc;
    if (crc == 0) {
      // done on one cluster
    } else {
    int64_t rows_per_cta;
    size_t smem;
    const int G = panel_grid(ctx, m, b, sizeof(T), &rows_per_cta, &smem);
    FL_CHECK(ctx, smem <= (size_t)kPanelSmemMax, FRACLAP_ERR_UNSUPPORTED, "sy2sb: panel too tall (%lld)", (long long)m);
    FL_CUDA(ctx, cudaMemsetAsync(s->gram, 0, sizeof(double) * b * b, st));
    FL_CUDA(ctx, cudaMemsetAsync(s->partials, 0, sizeof(double) * 3 * 2 * b, st));
    FL_CUDA(ctx, cudaMemsetAsync(ctx->d_barrier, 0, 2 * sizeof(unsigned), st));
    {
      double* tau = s->tau + p * b;
      int64_t ldp = lda, ldv = m, mm = m;
      int bw = b;
      double* partials = s->partials;
      double* gram = s->gram;
      unsigned* bar = ctx->d_barrier;
      long long limit = ctx->wait_cycles;
      int32_t* status = ctx->d_status;
      void* args[] = {&P, &ldp, &mm, &bw, &V, &ldv, &tau, &Tf, &partials, &gram, &bar, &limit, &status, &rows_per_cta};
      // the permitted maximum, not this panel's size: the attribute belongs to
      // the function, and concurrent callers on other streams share it
      FL_CUDA(ctx, cudaFuncSetAttribute(panel_qr_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, kPanelSmemMax));
      count_launch(ctx);
      FL_CUDA(ctx, cudaLaunchCooperativeKernel((void*)panel_qr_kernel<T>, dim3(G), dim3(PQR_NT), args, smem, st));
    }
    }
    T* A22 = Aw + (j0 + b) + (j0 + b) * lda;
    using D = GemmDescT<T>;
    // XT = V T  (m x b)
    FL_TRY(gemm<T>(ctx, false, false, kGemmPlain, D{m, b, b, V, m, Tf, b, s->XT, m, nullptr, 0, nullptr, 0, 0, 1.0, 0.0}, 1, st));
    // X = A22 XT (A22 symmetric, lower triangle)
    // (b columns only: split over the long dimension so that the grid fills the GPU)
    FL_CUDA(ctx, cudaMemsetAsync(s->X, 0, sizeof(T) * m * b, st));
    FL_TRY(gemm<T>(ctx, false, false, kGemmSymA, D{m, b, m, A22, lda, s->XT, m, s->X, m, nullptr, 0, nullptr, 0, 0, 1.0, 1.0}, (int)std::min<int64_t>(cdiv(m, 1024), 16), st));
    // Y = V^T X  (b x b), split over the long dimension
    FL_CUDA(ctx, cudaMemsetAsync(s->Y, 0, sizeof(T) * b * b, st));
    FL_TRY(gemm<T>(ctx, true, false, kGemmPlain, D{b, b, m, V, m, s->X, m, s->Y, b, nullptr, 0, nullptr, 0, 0, 1.0, 1.0}, (int)cdiv(m, 256), st));
    // Mm = T^T Y
    FL_TRY(gemm<T>(ctx, true, false, kGemmPlain, D{b, b, b, Tf, b, s->Y, b, s->Mm, b, nullptr, 0, nullptr, 0, 0, 1.0, 0.0}, 1, st));
    // W = X - 1/2 V Mm  (in X)
    FL_TRY(gemm<T>(ctx, false, false, kGemmPlain, D{m, b, b, V, m, s->Mm, b, s->X, m, nullptr, 0, nullptr, 0, 0, -0.5, 1.0}, 1, st));
    // A22 -= W V^T + V W^T  (lower triangle)
    FL_TRY(gemm<T>(ctx, false, true, kGemmLowerC, D{m, m, b, s->X, m, V, m, A22, lda, V, m, s->X, m, b, -1.0, 1.0}, 1, st));
    voff += m * b;
  }
  extract_band<T><<<(unsigned)cdiv(n * ldb, 256), 256, 0, st>>>(Aw, lda, n, b, band, ldb);
  count_launch(ctx);
  FL_CUDA(ctx, cudaGetLastError());
  return 0;
}

// Back-transformation by Q1 = Q_0 Q_1 ... Q_{p-1}: Z <- Q1 Z (n x ncols).
// Applied from the last panel to the first: Z(rows_j, :) -= V_j (T_j (V_j^T Z(rows_j, :))).
template <class T>
int q1_apply_run(fraclap_ctx* ctx, const Stage1T<T>* s, int64_t n, int b, T* Z, int64_t ldz,
                 int64_t ncols, T* W1, T* W2, cudaStream_t st) {
  int64_t voff = s->vtotal;
  using D = GemmDescT<T>;
  if (sizeof(T) == 4 && ctx->tc_scratch) {
    // tensor-core shapes (tall and wide products): W1^T = Z_r^T V (n x b),
    // W2^T = W1^T T^T, Z_r -= V W2 -- the same three products, transposed
    for (int64_t p = s->npanel - 1; p >= 0; --p) {
      const int64_t j0 = p * b, m = n - j0 - b;
      voff -= m * b;
      const T* V = s->Vstore + voff;
      const T* Tf = s->Tstore + p * b * b;
      T* Zr = Z + (j0 + b);
      FL_CUDA(ctx, cudaMemsetAsync(W1, 0, sizeof(T) * b * ncols, st));
      FL_TRY(gemm<T>(ctx, true, false, kGemmPlain, D{ncols, b, m, Zr, ldz, V, m, W1, ncols, nullptr, 0, nullptr, 0, 0, 1.0, 1.0}, (int)std::min<int64_t>(cdiv(m, 1024), 16), st));
      FL_TRY(gemm<T>(ctx, false, true, kGemmPlain, D{ncols, b, b, W1, ncols, Tf, b, W2, ncols, nullptr, 0, nullptr, 0, 0, 1.0, 0.0}, 1, st));
      FL_TRY(gemm<T>(ctx, false, true, kGemmPlain, D{m, ncols, b, V, m, W2, ncols, Zr, ldz, nullptr, 0, nullptr, 0, 0, -1.0, 1.0}, 1, st));
    }
    return 0;
  }
  for (int64_t p = s->npanel - 1; p >= 0; --p) {
    const int64_t j0 = p * b, m = n - j0 - b;
    voff -= m * b;
    const T* V = s->Vstore + voff;
    const T* Tf = s->Tstore + p * b * b;
    T* Zr = Z + (j0 + b);
    // W1 = V^T Zr  (b x ncols), split over the long dimension m
    FL_CUDA(ctx, cudaMemsetAsync(W1, 0, sizeof(T) * b * ncols, st));
    FL_TRY(gemm<T>(ctx, true, false, kGemmPlain, D{b, ncols, m, V, m, Zr, ldz, W1, b, nullptr, 0, nullptr, 0, 0, 1.0, 1.0}, (int)std::min<int64_t>(cdiv(m, 1024), 16), st));
    // W2 = T W1
    FL_TRY(gemm<T>(ctx, false, false, kGemmPlain, D{b, ncols, b, Tf, b, W1, b, W2, b, nullptr, 0, nullptr, 0, 0, 1.0, 0.0}, 1, st));
    // Zr -= V W2
    FL_TRY(gemm<T>(ctx, false, false, kGemmPlain, D{m, ncols, b, V, m, W2, b, Zr, ldz, nullptr, 0, nullptr, 0, 0, -1.0, 1.0}, 1, st));
  }
  return 0;
}

template int stage1_take<double>(Arena*, int64_t, int, int, Stage1T<double>*);
template int stage1_take<float>(Arena*, int64_t, int, int, Stage1T<float>*);
template int sy2sb_run<double>(fraclap_ctx*, double*, int64_t, int64_t, int, double*, Stage1T<double>*, cudaStream_t);
template int sy2sb_run<float>(fraclap_ctx*, float*, int64_t, int64_t, int, float*, Stage1T<float>*, cudaStream_t);
template int q1_apply_run<double>(fraclap_ctx*, const Stage1T<double>*, int64_t, int, double*, int64_t, int64_t, double*, double*, cudaStream_t);
template int q1_apply_run<float>(fraclap_ctx*, const Stage1T<float>*, int64_t, int, float*, int64_t, int64_t, float*, float*, cudaStream_t);

}  // namespace fraclap
