// FP64 GEMM engine.
//
// On GB300 the FP64 pipe delivers ~1.2 TFLOP/s for both DFMA and DMMA
// (measured: DFMA 1.20, mma.sync f64 1.05, cuBLAS DGEMM 1.10 TFLOP/s), i.e.
// about 2 FMA per clock per SM.  A 64x64 output tile with a 16-deep k step
// needs 1 KB of operands per 4096 FMAs, so a plain shared-memory tiled SIMT
// kernel is bound by the FP64 pipe, not by memory; the design goal is to keep
// that pipe busy (enough resident warps, 16 independent accumulators per
// thread) while supporting the operand forms the eigensolver needs: both
// transposes, a symmetric A read from its lower triangle, a lower-triangular
// C, a fused second product (symmetric rank-2k update), split-K with atomics
// and device-side batched descriptors.
#include <type_traits>

#include "internal.cuh"

namespace fraclap {
namespace {

constexpr int BM = 64, BN = 64, BK = 16, NT = 256;

template <class T, bool TA, int MODE>
__device__ __forceinline__ void load_a(T (*As)[BM + 1], const T* A, int64_t lda,
                                       int64_t M, int64_t K, int64_t m0, int64_t k0) {
  const int tid = threadIdx.x;
  if (MODE == kGemmSymA) {
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int m = tid % BM, k = tid / BM + 4 * i;
      const int64_t gm = m0 + m, gk = k0 + k;
      T v = T(0);
      if (gm < M && gk < K) v = (gm >= gk) ? A[gm + gk * lda] : A[gk + gm * lda];
      As[k][m] = v;
    }
  } else if (!TA) {
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int m = tid % BM, k = tid / BM + 4 * i;
      const int64_t gm = m0 + m, gk = k0 + k;
      As[k][m] = (gm < M && gk < K) ? A[gm + gk * lda] : T(0);
    }
  } else {
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int k = tid % BK, m = tid / BK + 16 * i;
      const int64_t gm = m0 + m, gk = k0 + k;
      As[k][m] = (gm < M && gk < K) ? A[gk + gm * lda] : T(0);
    }
  }
}

template <class T, bool TB>
__device__ __forceinline__ void load_b(T (*Bs)[BN + 1], const T* B, int64_t ldb,
                                       int64_t N, int64_t K, int64_t n0, int64_t k0) {
  const int tid = threadIdx.x;
  if (!TB) {
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int k = tid % BK, n = tid / BK + 16 * i;
      const int64_t gn = n0 + n, gk = k0 + k;
      Bs[k][n] = (gn < N && gk < K) ? B[gk + gn * ldb] : T(0);
    }
  } else {
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int n = tid % BN, k = tid / BN + 4 * i;
      const int64_t gn = n0 + n, gk = k0 + k;
      Bs[k][n] = (gn < N && gk < K) ? B[gn + gk * ldb] : T(0);
    }
  }
}

template <class T, bool TA, bool TB, int MODE>
__device__ __forceinline__ void accumulate(T (&acc)[4][4], T (*As)[BM + 1],
                                           T (*Bs)[BN + 1], const T* A, int64_t lda,
                                           const T* B, int64_t ldb, int64_t M, int64_t N,
                                           int64_t K, int64_t m0, int64_t n0, int64_t kbeg,
                                           int64_t kend) {
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
  for (int64_t k0 = kbeg; k0 < kend; k0 += BK) {
    load_a<T, TA, MODE>(As, A, lda, M, kend, m0, k0);
    load_b<T, TB>(Bs, B, ldb, N, kend, n0, k0);
    __syncthreads();
#pragma unroll
    for (int k = 0; k < BK; ++k) {
      T a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[k][ty + 16 * i];
#pragma unroll
      for (int j = 0; j < 4; ++j) b[j] = Bs[k][tx + 16 * j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
    }
    __syncthreads();
  }
}

template <class T, bool TA, bool TB, int MODE, bool ATOMIC>
__device__ __forceinline__ void gemm_tile(const GemmDescT<T>& d, int64_t m0, int64_t n0, int64_t kbeg,
                                          int64_t kend) {
  __shared__ T As[BK][BM + 1];
  __shared__ T Bs[BK][BN + 1];
  if (MODE == kGemmLowerC && m0 + BM - 1 < n0) return;  // tile entirely above the diagonal
  T acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = T(0);
  accumulate<T, TA, TB, MODE>(acc, As, Bs, d.A, d.lda, d.B, d.ldb, d.M, d.N, d.K, m0, n0, kbeg, kend);
  if (d.K2 > 0 && kbeg == 0)
    accumulate<T, TA, TB, MODE>(acc, As, Bs, d.A2, d.lda2, d.B2, d.ldb2, d.M, d.N, d.K2, m0, n0, 0,
                                d.K2);
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int64_t gm = m0 + ty + 16 * i;
    if (gm >= d.M) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int64_t gn = n0 + tx + 16 * j;
      if (gn >= d.N) continue;
      if (MODE == kGemmLowerC && gm < gn) continue;
      T* c = d.C + gm + gn * d.ldc;
      const T v = T(d.alpha) * acc[i][j];
      if (ATOMIC) {
        atomicAdd(c, v);
      } else {
        *c = (d.beta == 0.0) ? v : v + T(d.beta) * *c;
      }
    }
  }
}

template <class T, bool TA, bool TB, int MODE, bool ATOMIC>
__global__ void __launch_bounds__(NT) gemm_kernel(GemmDescT<T> d, int64_t kchunk) {
  const int64_t m0 = (int64_t)blockIdx.x * BM, n0 = (int64_t)blockIdx.y * BN;
  const int64_t kbeg = (int64_t)blockIdx.z * kchunk;
  const int64_t kend = (kbeg + kchunk < d.K) ? kbeg + kchunk : d.K;
  if (kbeg > 0 && kbeg >= d.K) return;  // z-slice 0 always runs (K = 0: C = beta C)
  gemm_tile<T, TA, TB, MODE, ATOMIC>(d, m0, n0, kbeg, kend);
}

template <class T, bool TA, bool TB>
__global__ void __launch_bounds__(NT) gemm_batched_kernel(const GemmDescT<T>* descs) {
  const GemmDescT<T> d = descs[blockIdx.z];
  const int64_t m0 = (int64_t)blockIdx.x * BM, n0 = (int64_t)blockIdx.y * BN;
  if (d.M <= 0 || d.N <= 0 || m0 >= d.M || n0 >= d.N) return;
  if (d.K <= 0) {  // C = beta C
    const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
    for (int i = 0; i < 4; ++i)
      for (int j = 0; j < 4; ++j) {
        const int64_t gm = m0 + ty + 16 * i, gn = n0 + tx + 16 * j;
        if (gm < d.M && gn < d.N) {
          T* c = d.C + gm + gn * d.ldc;
          *c = (d.beta == 0.0) ? T(0) : T(d.beta) * *c;
        }
      }
    return;
  }
  gemm_tile<T, TA, TB, kGemmPlain, false>(d, m0, n0, 0, d.K);
}

// ---------------------------------------------------------------------------
// FP32: 128 x 128 output tile, 8-deep k steps, 256 threads with 8 x 8 outputs
// each (rows 4 tx.. and 64 + 4 tx.., columns 4 ty.. and 64 + 4 ty..), read
// from shared memory as float4 (16 loads per 64 FMAs, against 8 per 16 on
// the 64 x 64 tile); the next k step is fetched into registers while the
// current one is multiplied (double-buffered shared memory, one barrier per
// step).  Plain and lower-C forms, fused second product, split-K, batched.
constexpr int SG_M = 128, SG_N = 128, SG_K = 8, SG_NT = 256, SG_LD = SG_M + 4;

template <bool TA, bool TB>
__device__ __forceinline__ void sg_fetch(const float* A, int64_t lda, const float* B, int64_t ldb, int64_t M,
                                         int64_t N, int64_t kend, int64_t m0, int64_t n0, int64_t k0,
                                         float (&ra)[4], float (&rb)[4]) {
  const int tid = threadIdx.x;
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    if (!TA) {
      const int64_t gm = m0 + tid % SG_M, gk = k0 + tid / SG_M + 2 * q;
      ra[q] = (gm < M && gk < kend) ? A[gm + gk * lda] : 0.0f;
    } else {
      const int64_t gk = k0 + tid % SG_K, gm = m0 + tid / SG_K + 32 * q;
      ra[q] = (gm < M && gk < kend) ? A[gk + gm * lda] : 0.0f;
    }
    if (!TB) {
      const int64_t gk = k0 + tid % SG_K, gn = n0 + tid / SG_K + 32 * q;
      rb[q] = (gn < N && gk < kend) ? B[gk + gn * ldb] : 0.0f;
    } else {
      const int64_t gn = n0 + tid % SG_N, gk = k0 + tid / SG_N + 2 * q;
      rb[q] = (gn < N && gk < kend) ? B[gn + gk * ldb] : 0.0f;
    }
  }
}

template <bool TA, bool TB>
__device__ __forceinline__ void sg_stash(float (*As)[SG_LD], float (*Bs)[SG_LD], const float (&ra)[4],
                                         const float (&rb)[4]) {
  const int tid = threadIdx.x;
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    if (!TA) As[tid / SG_M + 2 * q][tid % SG_M] = ra[q];
    else As[tid % SG_K][tid / SG_K + 32 * q] = ra[q];
    if (!TB) Bs[tid % SG_K][tid / SG_K + 32 * q] = rb[q];
    else Bs[tid / SG_N + 2 * q][tid % SG_N] = rb[q];
  }
}

template <bool TA, bool TB>
__device__ __forceinline__ void sg_accumulate(float (&acc)[8][8], float (*As)[SG_K][SG_LD],
                                              float (*Bs)[SG_K][SG_LD], const float* A, int64_t lda,
                                              const float* B, int64_t ldb, int64_t M, int64_t N, int64_t m0,
                                              int64_t n0, int64_t kbeg, int64_t kend) {
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
  float ra[4], rb[4];
  sg_fetch<TA, TB>(A, lda, B, ldb, M, N, kend, m0, n0, kbeg, ra, rb);
  __syncthreads();  // the buffers may still be read by a previous product
  sg_stash<TA, TB>(As[0], Bs[0], ra, rb);
  __syncthreads();
  int buf = 0;
  for (int64_t k0 = kbeg; k0 < kend; k0 += SG_K) {
    const bool more = k0 + SG_K < kend;
    if (more) sg_fetch<TA, TB>(A, lda, B, ldb, M, N, kend, m0, n0, k0 + SG_K, ra, rb);
#pragma unroll
    for (int k = 0; k < SG_K; ++k) {
      const float4 a0 = *reinterpret_cast<const float4*>(&As[buf][k][4 * tx]);
      const float4 a1 = *reinterpret_cast<const float4*>(&As[buf][k][64 + 4 * tx]);
      const float4 b0 = *reinterpret_cast<const float4*>(&Bs[buf][k][4 * ty]);
      const float4 b1 = *reinterpret_cast<const float4*>(&Bs[buf][k][64 + 4 * ty]);
      const float a[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
      const float b[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
      for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
    }
    if (more) sg_stash<TA, TB>(As[buf ^ 1], Bs[buf ^ 1], ra, rb);
    __syncthreads();
    buf ^= 1;
  }
}

template <bool TA, bool TB, int MODE, bool ATOMIC>
__device__ __forceinline__ void sg_tile(const GemmDescT<float>& d, int64_t m0, int64_t n0, int64_t kbeg,
                                        int64_t kend) {
  __shared__ __align__(16) float As[2][SG_K][SG_LD];
  __shared__ __align__(16) float Bs[2][SG_K][SG_LD];
  if (MODE == kGemmLowerC && m0 + SG_M - 1 < n0) return;  // tile entirely above the diagonal
  float acc[8][8];
#pragma unroll
  for (int i = 0; i < 8; ++i)
#pragma unroll
    for (int j = 0; j < 8; ++j) acc[i][j] = 0.0f;
  if (kend > kbeg) sg_accumulate<TA, TB>(acc, As, Bs, d.A, d.lda, d.B, d.ldb, d.M, d.N, m0, n0, kbeg, kend);
  if (d.K2 > 0 && kbeg == 0)
    sg_accumulate<TA, TB>(acc, As, Bs, d.A2, d.lda2, d.B2, d.ldb2, d.M, d.N, m0, n0, 0, d.K2);
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    const int64_t gn = n0 + (j < 4 ? 4 * ty + j : 64 + 4 * ty + j - 4);
    if (gn >= d.N) continue;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const int64_t gm = m0 + (i < 4 ? 4 * tx + i : 64 + 4 * tx + i - 4);
      if (gm >= d.M) continue;
      if (MODE == kGemmLowerC && gm < gn) continue;
      float* c = d.C + gm + gn * d.ldc;
      const float v = (float)d.alpha * acc[i][j];
      if (ATOMIC) atomicAdd(c, v);
      else *c = (d.beta == 0.0) ? v : v + (float)d.beta * *c;
    }
  }
}

template <bool TA, bool TB, int MODE, bool ATOMIC>
__global__ void __launch_bounds__(SG_NT, 2) sgemm_big_kernel(GemmDescT<float> d, int64_t kchunk) {
  const int64_t m0 = (int64_t)blockIdx.x * SG_M, n0 = (int64_t)blockIdx.y * SG_N;
  const int64_t kbeg = (int64_t)blockIdx.z * kchunk;
  const int64_t kend = (kbeg + kchunk < d.K) ? kbeg + kchunk : d.K;
  sg_tile<TA, TB, MODE, ATOMIC>(d, m0, n0, kbeg, kend);
}

template <bool TA, bool TB>
__global__ void __launch_bounds__(SG_NT, 2) sgemm_big_batched_kernel(const GemmDescT<float>* descs) {
  const GemmDescT<float> d = descs[blockIdx.z];
  const int64_t m0 = (int64_t)blockIdx.x * SG_M, n0 = (int64_t)blockIdx.y * SG_N;
  if (d.M <= 0 || d.N <= 0 || m0 >= d.M || n0 >= d.N) return;
  sg_tile<TA, TB, kGemmPlain, false>(d, m0, n0, 0, d.K > 0 ? d.K : 0);
}

// The large-tile FP32 kernel pays off once both output dimensions fill it.
inline bool sg_big(int64_t M, int64_t N) { return M >= 256 && N >= 256; }

template <class T, bool TA, bool TB, int MODE>
int launch(fraclap_ctx* ctx, const GemmDescT<T>& d, int split_k, cudaStream_t st) {
  if constexpr (std::is_same<T, float>::value && MODE != kGemmSymA) {
    if (sg_big(d.M, d.N)) {
      const int64_t gx = cdiv(d.M, SG_M), gy = cdiv(d.N, SG_N);
      FL_CHECK(ctx, gy <= 65535, FRACLAP_ERR_UNSUPPORTED, "gemm: N = %lld too large", (long long)d.N);
      if (split_k <= 1 || d.K2 > 0) {
        sgemm_big_kernel<TA, TB, MODE, false><<<dim3((unsigned)gx, (unsigned)gy, 1), SG_NT, 0, st>>>(
            d, d.K > 0 ? d.K : 1);
      } else {
        const int64_t kchunk = cdiv(cdiv(d.K, split_k), SG_K) * SG_K;
        const int64_t gz = cdiv(d.K, kchunk);
        sgemm_big_kernel<TA, TB, MODE, true><<<dim3((unsigned)gx, (unsigned)gy, (unsigned)gz), SG_NT, 0, st>>>(
            d, kchunk);
      }
      count_launch(ctx);
      FL_CUDA(ctx, cudaGetLastError());
      return 0;
    }
  }
  const int64_t gx = cdiv(d.M, BM), gy = cdiv(d.N, BN);
  FL_CHECK(ctx, gy <= 65535, FRACLAP_ERR_UNSUPPORTED, "gemm: N = %lld too large", (long long)d.N);
  if (split_k <= 1 || d.K2 > 0) {
    gemm_kernel<T, TA, TB, MODE, false><<<dim3((unsigned)gx, (unsigned)gy, 1), NT, 0, st>>>(
        d, d.K > 0 ? d.K : 1);
    count_launch(ctx);
  } else {
    int64_t kchunk = cdiv(cdiv(d.K, split_k), BK) * BK;
    const int64_t gz = cdiv(d.K, kchunk);
    gemm_kernel<T, TA, TB, MODE, true><<<dim3((unsigned)gx, (unsigned)gy, (unsigned)gz), NT, 0, st>>>(
        d, kchunk);
    count_launch(ctx);
  }
  FL_CUDA(ctx, cudaGetLastError());
  return 0;
}

}  // namespace

template <class T>
int gemm(fraclap_ctx* ctx, bool ta, bool tb, GemmMode mode, const GemmDescT<T>& d, int split_k,
         cudaStream_t st) {
  if (d.M <= 0 || d.N <= 0) return 0;
  FL_CHECK(ctx, mode != kGemmSymA || (!ta && d.M == d.K), FRACLAP_ERR_INVALID_ARG,
           "gemm: symmetric A must be square and untransposed");
  FL_CHECK(ctx, split_k <= 1 || d.beta == 1.0, FRACLAP_ERR_INVALID_ARG,
           "gemm: split-K accumulates into C (beta must be 1)");
  if constexpr (std::is_same<T, float>::value) {
    if ((d.K > 0 || d.K2 > 0) && tf32_route_fits(ctx, mode, d, split_k))
      return gemm_tf32x3(ctx, ta, tb, mode, d, split_k, st);
  }
  if (d.K <= 0 && d.K2 <= 0) {  // C = beta C
    GemmDescT<T> z = d;
    z.K = 0;
    z.K2 = 0;
    return launch<T, false, false, kGemmPlain>(ctx, z, 1, st);
  }
#define FL_GEMM_CASE(TA, TB)                                                           \
  if (ta == TA && tb == TB) {                                                          \
    if (mode == kGemmPlain) return launch<T, TA, TB, kGemmPlain>(ctx, d, split_k, st);  \
    if (mode == kGemmLowerC) return launch<T, TA, TB, kGemmLowerC>(ctx, d, split_k, st); \
  }
  FL_GEMM_CASE(false, false)
  FL_GEMM_CASE(false, true)
  FL_GEMM_CASE(true, false)
  FL_GEMM_CASE(true, true)
#undef FL_GEMM_CASE
  if (mode == kGemmSymA) {
    if (tb) return launch<T, false, true, kGemmSymA>(ctx, d, split_k, st);
    return launch<T, false, false, kGemmSymA>(ctx, d, split_k, st);
  }
  return set_error(ctx, FRACLAP_ERR_INVALID_ARG, "gemm: bad mode");
}

template <class T>
int gemm_batched(fraclap_ctx* ctx, bool ta, bool tb, const GemmDescT<T>* d_descs, int count,
                 int64_t max_m, int64_t max_n, cudaStream_t st) {
  if (count <= 0 || max_m <= 0 || max_n <= 0) return 0;
  if constexpr (std::is_same<T, float>::value) {
    if (sg_big(max_m, max_n)) {
      const int64_t gx = cdiv(max_m, SG_M), gy = cdiv(max_n, SG_N);
      FL_CHECK(ctx, gy <= 65535 && count <= 65535, FRACLAP_ERR_UNSUPPORTED, "gemm_batched: too large");
      dim3 grid((unsigned)gx, (unsigned)gy, (unsigned)count);
      if (!ta && !tb) sgemm_big_batched_kernel<false, false><<<grid, SG_NT, 0, st>>>(d_descs);
      else if (!ta && tb) sgemm_big_batched_kernel<false, true><<<grid, SG_NT, 0, st>>>(d_descs);
      else if (ta && !tb) sgemm_big_batched_kernel<true, false><<<grid, SG_NT, 0, st>>>(d_descs);
      else sgemm_big_batched_kernel<true, true><<<grid, SG_NT, 0, st>>>(d_descs);
      count_launch(ctx);
      FL_CUDA(ctx, cudaGetLastError());
      return 0;
    }
  }
  const int64_t gx = cdiv(max_m, BM), gy = cdiv(max_n, BN);
  FL_CHECK(ctx, gy <= 65535 && count <= 65535, FRACLAP_ERR_UNSUPPORTED, "gemm_batched: too large");
  dim3 grid((unsigned)gx, (unsigned)gy, (unsigned)count);
  if (!ta && !tb) gemm_batched_kernel<T, false, false><<<grid, NT, 0, st>>>(d_descs);
  else if (!ta && tb) gemm_batched_kernel<T, false, true><<<grid, NT, 0, st>>>(d_descs);
  else if (ta && !tb) gemm_batched_kernel<T, true, false><<<grid, NT, 0, st>>>(d_descs);
  else gemm_batched_kernel<T, true, true><<<grid, NT, 0, st>>>(d_descs);
  count_launch(ctx);
  FL_CUDA(ctx, cudaGetLastError());
  return 0;
}

template int gemm<double>(fraclap_ctx*, bool, bool, GemmMode, const GemmDescT<double>&, int, cudaStream_t);
template int gemm<float>(fraclap_ctx*, bool, bool, GemmMode, const GemmDescT<float>&, int, cudaStream_t);
template int gemm_batched<double>(fraclap_ctx*, bool, bool, const GemmDescT<double>*, int, int64_t, int64_t, cudaStream_t);
template int gemm_batched<float>(fraclap_ctx*, bool, bool, const GemmDescT<float>*, int, int64_t, int64_t, cudaStream_t);

}  // namespace fraclap
