// FP64-accurate GEMM from BF16 tensor-core products (Ozaki's error-free
// splitting: K. Ozaki, T. Ogita, S. Oishi, S. M. Rump, Numer. Algorithms 59,
// 2012), written from the method's mathematics.
//
// Every row i of op(A) is scaled by 2^-e_i (e_i: the exponent of its largest
// entry) and cut into s slices of 8 bits, A = sum_p 2^(e_i - 8p) A_p with A_p
// integer in [-255, 255] (exact in BF16); likewise every column j of op(B)
// with 2^f_j.  A product of two slices is an integer below 2^16, so a sum of
// 256 of them is exact in an FP32 accumulator: the tensor cores compute
// P_pq = A_p B_q exactly in K-chunks of 256, and the exact chunk sums are
// added, scaled by 2^-8(p+q), into an FP64 accumulator per output element
// (K/256 x pairs FP64 additions instead of K FP64 multiply-adds).  Pairs
// with p + q <= s + 1 are kept; the dropped tail and the slicing truncation
// are below 2^-8s relative to |row max| |column max| per term.  The result
// C = alpha 2^(e_i + f_j) sum + beta C is formed in FP64.
//
// The tensor-core step is mma.sync m16n8k16 (BF16 in, FP32 accumulate).
#include <cuda_bf16.h>

#include "internal.cuh"

namespace fraclap {
namespace {

constexpr int OZ_BM = 64, OZ_BN = 64, OZ_BK = 32, OZ_NT = 128, OZ_CHUNK = 256;
constexpr int OZ_LDS = OZ_BK / 2 + 4;  // shared row stride in 32-bit words (padded)

// Exponent of the largest |entry| of each row of op(A) (rows = M, length K).
// One block per row.
__global__ void row_exponents(const double* A, int64_t lda, bool trans, int64_t K, int* ex) {
  const int64_t i = blockIdx.x;
  double m = 0.0;
  for (int64_t k = threadIdx.x; k < K; k += blockDim.x) {
    const double v = trans ? A[k + i * lda] : A[i + k * lda];
    m = fmax(m, fabs(v));
  }
  __shared__ double red[32];
  for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (unsigned w = 0; w < blockDim.x / 32; ++w) t = fmax(t, red[w]);
    int e = 0;
    if (t > 0.0) frexp(t, &e);  // t = f 2^e, f in [0.5, 1): every |entry| < 2^e
    ex[i] = e;
  }
}

// Slices of op(A) (M x K): S[p][i][k] (k contiguous, Kp >= K, zero padded).
// One thread per (i, k); i fastest when A is not transposed (coalesced reads).
__global__ void make_slices(const double* A, int64_t lda, bool trans, int64_t M, int64_t K,
                            int64_t Kp, const int* ex, int s, __nv_bfloat16* S) {
  const int64_t total = M * Kp;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total;
       t += (int64_t)gridDim.x * blockDim.x) {
    int64_t i, k;
    if (trans) { k = t % Kp; i = t / Kp; } else { i = t % M; k = t / M; }
    double x = 0.0;
    if (k < K) x = ldexp(trans ? A[k + i * lda] : A[i + k * lda], -ex[i]);
    for (int p = 0; p < s; ++p) {
      const double y = x * 256.0;
      const double q = trunc(y);
      S[((int64_t)p * M + i) * Kp + k] = __float2bfloat16_rn((float)q);
      x = y - q;
    }
  }
}

__device__ __forceinline__ void mma_bf16(float (&c)[4], const uint32_t (&a)[4], const uint32_t (&b)[2]) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

// C tile 64 x 64 per CTA, 4 warps of 32 x 32 (2 x 4 mma tiles each).
__global__ void __launch_bounds__(OZ_NT)
ozaki_kernel(const __nv_bfloat16* __restrict__ SA, const __nv_bfloat16* __restrict__ SB,
             const int* __restrict__ ea, const int* __restrict__ eb, int64_t M, int64_t N,
             int64_t Kp, int s, double alpha, double beta, double* C, int64_t ldc, bool lower) {
  __shared__ uint32_t As[OZ_BM][OZ_LDS];
  __shared__ uint32_t Bs[OZ_BN][OZ_LDS];
  const int64_t m0 = (int64_t)blockIdx.x * OZ_BM, n0 = (int64_t)blockIdx.y * OZ_BN;
  if (lower && m0 + OZ_BM - 1 < n0) return;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int g = lane >> 2, tg = lane & 3;
  const int wm = (warp >> 1) * 32, wn = (warp & 1) * 32;
  double sum[2][4][4];
  float acc[2][4][4];
#pragma unroll
  for (int a = 0; a < 2; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b)
#pragma unroll
      for (int c = 0; c < 4; ++c) sum[a][b][c] = 0.0;

  for (int p = 0; p < s; ++p) {
    for (int q = 0; p + q < s; ++q) {  // slices p, q (0-based): p + q <= s - 1
      const __nv_bfloat16* Ap = SA + (int64_t)p * M * Kp;
      const __nv_bfloat16* Bq = SB + (int64_t)q * N * Kp;
      const double scale = ldexp(1.0, -8 * (p + q + 2));
      for (int64_t c0 = 0; c0 < Kp; c0 += OZ_CHUNK) {
#pragma unroll
        for (int a = 0; a < 2; ++a)
#pragma unroll
          for (int b = 0; b < 4; ++b)
#pragma unroll
            for (int c = 0; c < 4; ++c) acc[a][b][c] = 0.f;
        const int64_t cend = (c0 + OZ_CHUNK < Kp) ? c0 + OZ_CHUNK : Kp;
        for (int64_t k0 = c0; k0 < cend; k0 += OZ_BK) {
          // 64 rows x 32 bf16 = 64 x 16 words per operand; 128 threads x 8 words each
#pragma unroll
          for (int r = 0; r < 8; ++r) {
            const int idx = tid + r * OZ_NT;  // 0 .. 1023
            const int row = idx >> 4, w = idx & 15;
            const int64_t gm = m0 + row, gn = n0 + row;
            As[row][w] = (gm < M) ? reinterpret_cast<const uint32_t*>(Ap + gm * Kp + k0)[w] : 0u;
            Bs[row][w] = (gn < N) ? reinterpret_cast<const uint32_t*>(Bq + gn * Kp + k0)[w] : 0u;
          }
          __syncthreads();
#pragma unroll
          for (int kk = 0; kk < OZ_BK / 2; kk += 8) {  // two k16 steps (8 words each)
            uint32_t af[2][4], bf[4][2];
#pragma unroll
            for (int a = 0; a < 2; ++a) {
              const int r0 = wm + a * 16 + g;
              af[a][0] = As[r0][kk + tg];
              af[a][1] = As[r0 + 8][kk + tg];
              af[a][2] = As[r0][kk + tg + 4];
              af[a][3] = As[r0 + 8][kk + tg + 4];
            }
#pragma unroll
            for (int b = 0; b < 4; ++b) {
              const int c = wn + b * 8 + g;
              bf[b][0] = Bs[c][kk + tg];
              bf[b][1] = Bs[c][kk + tg + 4];
            }
#pragma unroll
            for (int a = 0; a < 2; ++a)
#pragma unroll
              for (int b = 0; b < 4; ++b) mma_bf16(acc[a][b], af[a], bf[b]);
          }
          __syncthreads();
        }
#pragma unroll
        for (int a = 0; a < 2; ++a)
#pragma unroll
          for (int b = 0; b < 4; ++b)
#pragma unroll
            for (int c = 0; c < 4; ++c) sum[a][b][c] = fma((double)acc[a][b][c], scale, sum[a][b][c]);
      }
    }
  }
  // epilogue: c0,c1 at (g, 2tg..), c2,c3 at (g + 8, 2tg..)
#pragma unroll
  for (int a = 0; a < 2; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b)
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        const int64_t gm = m0 + wm + a * 16 + g + ((c >> 1) << 3);
        const int64_t gn = n0 + wn + b * 8 + 2 * tg + (c & 1);
        if (gm >= M || gn >= N || (lower && gm < gn)) continue;
        const double v = ldexp(sum[a][b][c], ea[gm] + eb[gn]);
        double* cp = C + gm + gn * ldc;
        *cp = (beta == 0.0) ? alpha * v : alpha * v + beta * *cp;
      }
}

}  // namespace

size_t ozaki_ws(int64_t M, int64_t N, int64_t K, int s) {
  const int64_t Kp = cdiv(K, OZ_BK) * OZ_BK;
  Arena ar;
  ar.take<__nv_bfloat16>((int64_t)s * M * Kp);
  ar.take<__nv_bfloat16>((int64_t)s * N * Kp);
  ar.take<int>(M);
  ar.take<int>(N);
  return ar.off;
}

// C = alpha op(A) op(B) + beta C, FP64-accurate through s BF16 slices
// (s = 7 for full FP64 accuracy of the products).  lower: only C(i,j), i >= j.
int ozaki_gemm(fraclap_ctx* ctx, bool ta, bool tb, int64_t M, int64_t N, int64_t K, double alpha,
               const double* A, int64_t lda, const double* B, int64_t ldb, double beta, double* C,
               int64_t ldc, int s, bool lower, Arena* ar, cudaStream_t st) {
  if (M <= 0 || N <= 0) return 0;
  FL_CHECK(ctx, s >= 1 && s <= 8, FRACLAP_ERR_INVALID_ARG, "ozaki_gemm: slices must be 1..8");
  FL_CHECK(ctx, cdiv(N, OZ_BN) <= 65535, FRACLAP_ERR_UNSUPPORTED, "ozaki_gemm: N too large");
  const int64_t Kp = cdiv(std::max<int64_t>(K, 1), OZ_BK) * OZ_BK;
  __nv_bfloat16* SA = ar->take<__nv_bfloat16>((int64_t)s * M * Kp);
  __nv_bfloat16* SB = ar->take<__nv_bfloat16>((int64_t)s * N * Kp);
  int* ea = ar->take<int>(M);
  int* eb = ar->take<int>(N);
  FL_CHECK(ctx, eb != nullptr, FRACLAP_ERR_ALLOC, "ozaki_gemm: workspace too small");
  // op(A) rows: trans -> A stored K x M; op(B) columns = rows of op(B)^T
  row_exponents<<<(unsigned)M, 256, 0, st>>>(A, lda, ta, K, ea);
  count_launch(ctx);
  row_exponents<<<(unsigned)N, 256, 0, st>>>(B, ldb, !tb, K, eb);
  count_launch(ctx);
  const unsigned gs = (unsigned)std::min<int64_t>(cdiv(std::max(M, N) * Kp, 256), 152 * 32);
  make_slices<<<gs, 256, 0, st>>>(A, lda, ta, M, K, Kp, ea, s, SA);
  count_launch(ctx);
  make_slices<<<gs, 256, 0, st>>>(B, ldb, !tb, N, K, Kp, eb, s, SB);
  count_launch(ctx);
  dim3 grid((unsigned)cdiv(M, OZ_BM), (unsigned)cdiv(N, OZ_BN));
  ozaki_kernel<<<grid, OZ_NT, 0, st>>>(SA, SB, ea, eb, M, N, Kp, s, alpha, beta, C, ldc, lower);
  count_launch(ctx);
  FL_CUDA(ctx, cudaGetLastError());
  return 0;
}

}  // namespace fraclap

using namespace fraclap;

extern "C" size_t fraclap_dgemm_ozaki_workspace_bytes(int64_t m, int64_t n, int64_t k, int slices) {
  if (m < 0 || n < 0 || k < 0 || slices < 1 || slices > 8) return 0;
  return ozaki_ws(m, n, k, slices) + 1024;
}

extern "C" int fraclap_dgemm_ozaki(fraclap_ctx* ctx, int trans_a, int trans_b, int64_t m, int64_t n,
                                   int64_t k, double alpha, const double* A_dev, int64_t lda,
                                   const double* B_dev, int64_t ldb, double beta, double* C_dev,
                                   int64_t ldc, int slices, void* work_dev, size_t work_bytes,
                                   fraclap_stream_t stream) {
  if (!ctx) return FRACLAP_ERR_INVALID_ARG;
  FL_CHECK(ctx, m >= 0 && n >= 0 && k >= 0, FRACLAP_ERR_INVALID_ARG, "dgemm_ozaki: negative size");
  if (m == 0 || n == 0) return 0;
  FL_CHECK(ctx, C_dev && A_dev && B_dev, FRACLAP_ERR_INVALID_ARG, "dgemm_ozaki: null pointer");
  FL_CHECK(ctx, ldc >= m && lda >= (trans_a ? k : m) && ldb >= (trans_b ? n : k),
           FRACLAP_ERR_INVALID_ARG, "dgemm_ozaki: leading dimension too small");
  Arena ar;
  FL_TRY(get_workspace(ctx, work_dev, work_bytes, ozaki_ws(m, n, k, slices) + 1024, &ar));
  return ozaki_gemm(ctx, trans_a != 0, trans_b != 0, m, n, k, alpha, A_dev, lda, B_dev, ldb, beta,
                    C_dev, ldc, slices, false, &ar, (cudaStream_t)stream);
}
