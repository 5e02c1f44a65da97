// FP64-accurate GEMM from BF16 tensor-core products (Ozaki's error-free
// splitting: K. Ozaki, T. Ogita, S. Oishi, S. M. Rump, Numer. Algorithms 59,
// 2012), written from the method's mathematics.
//
// Every row i of op(A) is scaled by 2^-e_i (e_i: the exponent of its largest
// entry) and cut into slices of w bits, A = sum_p 2^(e_i - w p) A_p with A_p
// integer in (-2^w, 2^w) (exact in BF16 for w <= 8); likewise every column j
// of op(B) with 2^f_j.  A product of two slices is an integer below 2^2w, so a
// sum of 2^(24-2w) of them is exact in an FP32 accumulator: the tensor cores
// compute P_pq = A_p B_q exactly in K-chunks of that length, and the exact
// chunk sums are added, scaled by 2^-w(p+q), into an FP64 accumulator per
// output element.  w = 8 (chunks of 256) for short K; otherwise w = 7 (chunks
// of 1024) with ceil(8s/7) slices, which keeps the 8s bits and needs three
// times fewer FP64 additions.  Pairs with p + q <= slices + 1 are kept; the
// dropped tail and the slicing truncation are below about 2^-8s relative to
// |row max| |column max| per term.  The result
// C = alpha 2^(e_i + f_j) sum + beta C is formed in FP64.
//
// Two tensor-core kernels compute the slice products: the sm_103a one uses
// tcgen05.mma with operands brought into shared memory by TMA
// (cp.async.bulk.tensor, 128-byte swizzle) and the FP32 chunk accumulators in
// tensor memory (four buffers at 128 columns, two at 256), so that the
// draining and FP64 folding of finished chunks overlap the products of the
// next ones; a plain mma.sync m16n8k16 kernel is kept as the reference route
// for checking it.
#include <cuda.h>
#include <cuda_bf16.h>

#include <mutex>

#include "internal.cuh"
#include "tc_common.cuh"

namespace fraclap {
namespace {

using namespace tc;

constexpr int OZ_BM = 64, OZ_BN = 64, OZ_BK = 32, OZ_NT = 128;
constexpr int OZ_KPAD = 64;  // slice rows padded to a multiple of 64 (one TMA box)
constexpr int OZ_LDS = OZ_BK / 2 + 4;  // shared row stride in 32-bit words (padded)

// e with every |entry| < 2^e, from the largest |entry| t given as the bits
// of its IEEE pattern with the sign cleared.
__device__ __forceinline__ int exponent_above(unsigned long long t) {
  int e = 0;
  const int E = (int)(t >> 52);
  if (E > 0) e = E - 1022;  // t = f 2^e, f in [0.5, 1): every |entry| < 2^e
  else if (t != 0) frexp(__longlong_as_double((long long)t), &e);  // subnormal maximum
  return e;
}

// Exponent of the largest |entry| of each row of op(A) (rows = M, length K).
// One block per row.  The magnitudes are compared as the integers of their
// IEEE bit patterns with the sign cleared (the same order as the values), so
// the FP64 pipe is not used.
__global__ void row_exponents(const double* A, int64_t lda, bool trans, int64_t K, int* ex) {
  const int64_t i = blockIdx.x;
  unsigned long long m = 0;
  for (int64_t k = threadIdx.x; k < K; k += blockDim.x) {
    const double v = trans ? A[k + i * lda] : A[i + k * lda];
    const unsigned long long u = (unsigned long long)__double_as_longlong(v) & 0x7FFFFFFFFFFFFFFFull;
    m = u > m ? u : m;
  }
  __shared__ unsigned long long red[32];
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long v = __shfl_xor_sync(0xffffffffu, m, o);
    m = v > m ? v : m;
  }
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned long long t = 0;
    for (unsigned w = 0; w < blockDim.x / 32; ++w) t = red[w] > t ? red[w] : t;
    ex[i] = exponent_above(t);
  }
}

// The same for the rows of an untransposed column-major M x K operand, whose
// rows are strided: a thread per row over a chunk of kch columns (the reads
// of a warp are contiguous), the chunks' maxima merged by an integer
// atomicMax on the bit patterns (order-free, so the same maximum), then
// exponents_of_max.
constexpr int OZ_MAX_KCH = 64;
__global__ void row_absmax_strided(const double* A, int64_t lda, int64_t M, int64_t K, unsigned long long* mx) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= M) return;
  const int64_t k0 = (int64_t)blockIdx.y * OZ_MAX_KCH;
  const int64_t k1 = (k0 + OZ_MAX_KCH < K) ? k0 + OZ_MAX_KCH : K;
  unsigned long long m = 0;
  for (int64_t k = k0; k < k1; ++k) {
    const unsigned long long u = (unsigned long long)__double_as_longlong(A[i + k * lda]) & 0x7FFFFFFFFFFFFFFFull;
    m = u > m ? u : m;
  }
  if (m != 0) atomicMax(&mx[i], m);
}
__global__ void exponents_of_max(const unsigned long long* mx, int64_t M, int* ex) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < M) ex[i] = exponent_above(mx[i]);
}

// Slices of op(A) (M x K): S[p][i][k] (k contiguous, Kp >= K, zero padded).
// One thread per (i, k); i fastest when A is not transposed (coalesced reads).
// Slice p is the signed integer trunc(x 2^(w(p+1))) - 2^w trunc(x 2^(w p))
// of x = a 2^-e (|x| < 1): the w-bit digits of |x| with the sign of x.  When
// all s w bits fit in 64, |x| 2^(w s) is truncated once to an unsigned
// integer (exact: a power-of-two scaling, then a truncating conversion) and
// the digits are read off with shifts; otherwise the digits are peeled in
// FP64, which gives the same digits.
// The s digits of one entry a of row i (exponent e = ex[i]) into S[p * pstride].
__device__ __forceinline__ void write_digits(double a, int e, int s, int bits, __nv_bfloat16* S, int64_t pstride) {
  const int tb = bits * s;
  if (tb <= 64) {
    // floor(|a| 2^(tb - e)) from the bits: |a| = m 2^(E - 1075) (m with
    // its hidden bit; subnormals take E = 1), shifted exactly; below 2^tb
    // because |a| < 2^e
    const unsigned long long mask = (1ull << bits) - 1ull;
    const unsigned long long bitsA = (unsigned long long)__double_as_longlong(a);
    const int E = (int)((bitsA >> 52) & 0x7FF);
    const unsigned long long mant = (bitsA & 0xFFFFFFFFFFFFFull) | (E ? (1ull << 52) : 0ull);
    const int sh = (E ? E : 1) - 1075 + tb - e;
    const unsigned long long u = (sh >= 64 || sh <= -64) ? 0ull : (sh >= 0 ? (mant << sh) : (mant >> -sh));
    const float sg = (a < 0.0) ? -1.0f : 1.0f;
    for (int p = 0; p < s; ++p) {
      const unsigned long long dgt = (u >> (bits * (s - 1 - p))) & mask;
      S[p * pstride] = __float2bfloat16_rn(sg * (float)dgt);
    }
  } else {
    double x = ldexp(a, -e);
    for (int p = 0; p < s; ++p) {
      const double y = ldexp(x, bits);
      const double q = trunc(y);
      S[p * pstride] = __float2bfloat16_rn((float)q);
      x = y - q;
    }
  }
}

__global__ void make_slices(const double* A, int64_t lda, bool trans, int64_t M, int64_t K,
                            int64_t Kp, const int* ex, int s, int bits, __nv_bfloat16* S) {
  const int64_t total = M * Kp;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total;
       t += (int64_t)gridDim.x * blockDim.x) {
    int64_t i, k;
    if (trans) { k = t % Kp; i = t / Kp; } else { i = t % M; k = t / M; }
    const double a = (k < K) ? (trans ? A[k + i * lda] : A[i + k * lda]) : 0.0;
    write_digits(a, ex[i], s, bits, S + i * Kp + k, M * Kp);
  }
}

// The slices of an operand whose rows are contiguous (trans), for s * bits
// <= 64: a thread takes eight consecutive entries of a row and writes each
// digit's eight BF16 values as one 16-byte store (Kp is a multiple of 64, so
// every store is aligned); the digits are those of write_digits.
__global__ void make_slices_rows(const double* A, int64_t lda, int64_t M, int64_t K, int64_t Kp,
                                 const int* ex, int s, int bits, __nv_bfloat16* S) {
  const int64_t per_row = Kp / 8, total = M * per_row;
  const int tb = bits * s;
  const unsigned long long mask = (1ull << bits) - 1ull;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = t / per_row, k0 = (t % per_row) * 8;
    const int e = ex[i];
    unsigned long long u[8];
    float sg[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const double a = (k0 + q < K) ? A[k0 + q + i * lda] : 0.0;
      const unsigned long long bitsA = (unsigned long long)__double_as_longlong(a);
      const int E = (int)((bitsA >> 52) & 0x7FF);
      const unsigned long long mant = (bitsA & 0xFFFFFFFFFFFFFull) | (E ? (1ull << 52) : 0ull);
      const int sh = (E ? E : 1) - 1075 + tb - e;
      u[q] = (sh >= 64 || sh <= -64) ? 0ull : (sh >= 0 ? (mant << sh) : (mant >> -sh));
      sg[q] = (a < 0.0) ? -1.0f : 1.0f;
    }
    for (int p = 0; p < s; ++p) {
      const int rs = bits * (s - 1 - p);
      uint32_t w[4];
#pragma unroll
      for (int h = 0; h < 4; ++h) {
        const unsigned short lo =
            __bfloat16_as_ushort(__float2bfloat16_rn(sg[2 * h] * (float)((u[2 * h] >> rs) & mask)));
        const unsigned short hi =
            __bfloat16_as_ushort(__float2bfloat16_rn(sg[2 * h + 1] * (float)((u[2 * h + 1] >> rs) & mask)));
        w[h] = (uint32_t)lo | ((uint32_t)hi << 16);
      }
      *reinterpret_cast<uint4*>(S + ((int64_t)p * M + i) * Kp + k0) = make_uint4(w[0], w[1], w[2], w[3]);
    }
  }
}

// The same slices of an untransposed column-major operand (rows strided):
// 32 x 32 tiles of (i, k) staged in shared memory, read along i and written
// along k, so that both the FP64 reads and the BF16 writes are contiguous
// within a warp.  Block 32 x 8 threads; grid (ceil(M / 32), Kp / 32).
__global__ void make_slices_strided(const double* A, int64_t lda, int64_t M, int64_t K, int64_t Kp,
                                    const int* ex, int s, int bits, __nv_bfloat16* S) {
  __shared__ double tile[32][33];
  const int64_t i0 = (int64_t)blockIdx.x * 32, k0 = (int64_t)blockIdx.y * 32;
  for (int r = threadIdx.y; r < 32; r += 8) {
    const int64_t i = i0 + threadIdx.x, k = k0 + r;
    tile[r][threadIdx.x] = (i < M && k < K) ? A[i + k * lda] : 0.0;
  }
  __syncthreads();
  for (int r = threadIdx.y; r < 32; r += 8) {
    const int64_t i = i0 + r, k = k0 + threadIdx.x;
    if (i < M) write_digits(tile[threadIdx.x][r], ex[i], s, bits, S + i * Kp + k, M * Kp);
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
             int64_t Kp, int s, int bits, int64_t chunk, double alpha, double beta, double* C,
             int64_t ldc, bool lower) {
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
      const double scale = ldexp(1.0, -bits * (p + q + 2));
      for (int64_t c0 = 0; c0 < Kp; c0 += chunk) {
#pragma unroll
        for (int a = 0; a < 2; ++a)
#pragma unroll
          for (int b = 0; b < 4; ++b)
#pragma unroll
            for (int c = 0; c < 4; ++c) acc[a][b][c] = 0.f;
        const int64_t cend = (c0 + chunk < Kp) ? c0 + chunk : Kp;
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


// ----------------------------------------------------------------------------
// tcgen05 route: CTA tile 128 (rows of op(A)) x 128 (columns of op(B)).
// Warp 0: TMA producer; warp 1: TMEM owner and MMA issuer; warps 2-9:
// epilogue, two warps per TMEM lane quarter (lanes 32 (w % 4) ..), each
// thread one output row and 64 of the 128 columns.  Six 32 KB stages keep
// enough bytes in flight to cover the L2 latency.
// ----------------------------------------------------------------------------
// The tile width TCN (128, 192 or 256 columns of op(B)) is a schedule
// choice: a 128 x 256 tile moves 48 KB of slices per 4.2 MFLOP k-block
// instead of 32 KB per 2.1 MFLOP (1.33x fewer L2 bytes per flop), with four
// stages instead of six and the two accumulators filling all 512 TMEM
// columns, but its epilogue threads keep 128 integer sums each, more than
// their registers hold; 128 x 192 (40 KB per 3.1 MFLOP, five stages) keeps
// 96 per thread.
constexpr int TC_M = 128, TC_KB = 64;
constexpr int TC_EPI_WARPS = 8;
constexpr int TC_THREADS = 64 + 32 * TC_EPI_WARPS;
constexpr int TC_A_BYTES = TC_M * TC_KB * 2;
template <int TCN>
struct OzTile {
  static_assert(TCN == 128 || TCN == 192 || TCN == 256, "tile width 128, 192 or 256");
  static constexpr int STAGES = (TCN == 256) ? 4 : (TCN == 192) ? 5 : 6;
  static constexpr int B_BYTES = TCN * TC_KB * 2;
  static constexpr int STAGE_BYTES = TC_A_BYTES + B_BYTES;
  static constexpr int EPI_COLS = TCN * 4 / TC_EPI_WARPS;  // columns per epilogue thread
  // FP32 chunk accumulators in the 512 TMEM columns: four at 128 columns
  // (the MMA warp runs up to three chunks ahead of an epilogue that is
  // folding a finished diagonal into C), two at 192 or 256; the allocation
  // is the whole (power-of-two) 512 columns
  static constexpr int NBUF = 512 / TCN;
  static constexpr uint32_t TMEM_COLS = 512;
  // kind::f16 instruction descriptor: D F32, A and B BF16, both K-major, M 128, N TCN.
  static constexpr uint32_t IDESC = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(TCN >> 3) << 17) |
                                    ((uint32_t)(TC_M >> 4) << 24);
};

// 2^e for e in [-1022, 1023], from its bit pattern.
__device__ __forceinline__ double pow2i(int e) { return __longlong_as_double((long long)(e + 1023) << 52); }

// Order of the output tiles over the CTAs: groups of G consecutive tile rows;
// inside a group, the G rows of one tile column are consecutive CTAs, then
// the next column.  The CTAs resident at one time then cover a G x (152 / G)
// block of tiles, whose A rows and B columns L2 holds while every CTA of the
// block streams them (in the plain order a wave spans every tile row, so each
// slice pair re-streams all of A).  With `lower`, a group only has the columns
// up to its last row: tiles entirely above the diagonal are not enumerated.
// The host sizes the grid with the same count (ozaki_tile_count).  Tiles
// are TCM rows by TCN columns; with `lower`, a group of tile rows ending at
// tile row r needs the tile columns that start at or below row r TCM + TCM - 1.
__host__ __device__ inline int ozaki_group_cols(int g0, int Gg, int TN, int TCM, int TCN, bool lower) {
  if (!lower) return TN;
  const int64_t last_row = (int64_t)(g0 + Gg - 1) * TCM + TCM - 1;
  const int64_t c = last_row / TCN + 1;
  return (int)(c < TN ? c : TN);
}
__host__ __device__ inline int64_t ozaki_tile_count(int TM, int TN, int G, bool lower, int TCM, int TCN) {
  int64_t tot = 0;
  for (int g0 = 0; g0 < TM; g0 += G) {
    const int Gg = (TM - g0 < G) ? TM - g0 : G;
    tot += (int64_t)Gg * ozaki_group_cols(g0, Gg, TN, TCM, TCN, lower);
  }
  return tot;
}
__device__ __forceinline__ void ozaki_tile_of(int64_t idx, int TM, int TN, int G, bool lower, int TCM, int TCN,
                                              int* tm, int* tn) {
  int64_t base = 0;
  for (int g0 = 0; g0 < TM; g0 += G) {
    const int Gg = (TM - g0 < G) ? TM - g0 : G;
    const int ncol = ozaki_group_cols(g0, Gg, TN, TCM, TCN, lower);
    const int64_t cnt = (int64_t)Gg * ncol;
    if (idx < base + cnt) {
      const int r = (int)(idx - base);
      *tn = r / Gg;
      *tm = g0 + r % Gg;
      return;
    }
    base += cnt;
  }
  *tm = TM;  // past the end: no tile
  *tn = 0;
}

// CS = 2: a cluster of CS CTAs takes CS consecutive tile rows of one tile
// column.  They need the same B tile, so each CTA loads 1/CS of it (TCN / CS
// rows of op(B)) with one TMA multicast into the same stage of every CTA of
// the cluster: the L2-to-SM bytes per k-block drop from A + B to A + B / CS.
// A stage may then be refilled only once all CS CTAs have consumed it, so
// every MMA warp's stage-release commit is multicast to the empty barriers of
// the whole cluster, which count CS arrivals.  Every CTA of a cluster runs
// the whole pipeline (its peers need its share of B), also when its tile
// lies past the last row or above the diagonal; its epilogue then writes
// nothing.
template <int TCN, int CS>
__global__ void __launch_bounds__(TC_THREADS, 1)
ozaki_tc_kernel(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapB,
                const int* __restrict__ ea, const int* __restrict__ eb, int64_t M, int64_t N, int64_t Kp,
                int s, int bits, int64_t chunk, double alpha, double beta, double* C, int64_t ldc,
                int lower, int group, long long limit,
                int32_t* status) {
  constexpr int TC_N = TCN, TC_STAGES = OzTile<TCN>::STAGES, TC_B_BYTES = OzTile<TCN>::B_BYTES;
  constexpr int TC_STAGE_BYTES = OzTile<TCN>::STAGE_BYTES, TC_EPI_COLS = OzTile<TCN>::EPI_COLS;
  constexpr uint32_t TC_TMEM_COLS = OzTile<TCN>::TMEM_COLS, TC_IDESC = OzTile<TCN>::IDESC;
  constexpr int NBUF = OzTile<TCN>::NBUF;
  constexpr int B_ROWS = TCN / CS;  // rows of the B tile this CTA loads (and multicasts)
  static_assert(CS == 1 || CS == 2 || CS == 4, "cluster of 1, 2 or 4 CTAs");
  static_assert((B_ROWS * 128) % 1024 == 0, "a B share starts on a 128-byte-swizzle atom");
  (void)TC_B_BYTES;
  extern __shared__ __align__(1024) unsigned char tc_smem_raw[];
  unsigned char* smem = (unsigned char*)(((uintptr_t)tc_smem_raw + 1023) & ~(uintptr_t)1023);
  __shared__ __align__(8) uint64_t full_bar[TC_STAGES], empty_bar[TC_STAGES];
  __shared__ __align__(8) uint64_t acc_full[OzTile<TCN>::NBUF], acc_empty[OzTile<TCN>::NBUF], done_bar;
  __shared__ uint32_t tmem_base_sh;
  __shared__ int abort_sh;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int TM = (int)((M + TC_M - 1) / TC_M), TN = (int)((N + TC_N - 1) / TC_N);
  const int rank = (CS > 1) ? (int)cluster_ctarank() : 0;
  int tm, tn;
  if (CS == 1) {
    ozaki_tile_of((int64_t)blockIdx.x, TM, TN, group, lower != 0, TC_M, TC_N, &tm, &tn);
    if (tm >= TM || tn >= TN) return;
    if (lower && (int64_t)tm * TC_M + TC_M - 1 < (int64_t)tn * TC_N) return;  // tile above the diagonal
  } else {
    // the grid holds whole clusters of CS tile rows: no CTA leaves early
    int tc;
    ozaki_tile_of((int64_t)(blockIdx.x / CS), (TM + CS - 1) / CS, TN, group, lower != 0, CS * TC_M, TC_N, &tc, &tn);
    tm = tc * CS + rank;
  }
  const int64_t m0 = (int64_t)tm * TC_M, n0 = (int64_t)tn * TC_N;
  const int nchunk = (int)((Kp + chunk - 1) / chunk);

  if (threadIdx.x == 0) {
    for (int i = 0; i < TC_STAGES; ++i) {
      mbar_init(&full_bar[i], 1);
      mbar_init(&empty_bar[i], CS);
    }
    for (int i = 0; i < NBUF; ++i) {
      mbar_init(&acc_full[i], 1);
      mbar_init(&acc_empty[i], TC_EPI_WARPS);
    }
    mbar_init(&done_bar, 1);
    abort_sh = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(&tmem_base_sh)),
                 "r"(TC_TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  if (CS > 1) cluster_sync_all();  // every CTA's barriers exist before any multicast reaches them
  tc_fence_after();
  const uint32_t tmem = tmem_base_sh;

  if (warp == 0) {
    // ---------------- TMA producer ----------------
    if (lane == 0) {
      int it = 0;
      bool ok = true;
      for (int dg = 0; dg < s && ok; ++dg)
        for (int p = 0; p <= dg && ok; ++p)
          for (int c = 0; c < nchunk && ok; ++c) {
            const int q = dg - p;
            const int64_t c0 = (int64_t)c * chunk;
            const int nkb = (int)(((Kp - c0) < chunk ? (Kp - c0) : chunk) / TC_KB);
            for (int kb = 0; kb < nkb; ++kb, ++it) {
              const int st = it % TC_STAGES;
              if (!mbar_wait(&empty_bar[st], ((it / TC_STAGES) & 1) ^ 1, limit) || *(volatile int*)&abort_sh) {
                ok = false;
                break;
              }
              unsigned char* a = smem + st * TC_STAGE_BYTES;
              unsigned char* b = a + TC_A_BYTES;
              mbar_expect_tx(&full_bar[st], TC_STAGE_BYTES);  // A and the whole B tile (all CS shares)
              const int kc = (int)(c0 + kb * TC_KB);
              tma_load_3d(a, &mapA, &full_bar[st], kc, (int)m0, p);
              if (CS == 1)
                tma_load_3d(b, &mapB, &full_bar[st], kc, (int)n0, q);
              else
                tma_load_3d_multicast(b + rank * (B_ROWS * 128), &mapB, &full_bar[st], kc,
                                      (int)(n0 + rank * B_ROWS), q, (uint16_t)((1u << CS) - 1u));
            }
          }
      if (CS > 1 && ok) {
        // every peer's last releases of this CTA's stages have arrived: no
        // remote arrive can reach this CTA's barriers after it exits
        for (int j = (it > TC_STAGES ? it - TC_STAGES : 0); j < it && ok; ++j)
          ok = mbar_wait(&empty_bar[j % TC_STAGES], ((j / TC_STAGES) & 1), limit);
      }
      if (!ok) {
        atomicCAS(status, 0, FRACLAP_ERR_TIMEOUT);
        abort_sh = 1;
        // let the copies already issued land before the CTA can exit
        for (int j = (it > TC_STAGES ? it - TC_STAGES : 0); j < it; ++j)
          mbar_wait(&full_bar[j % TC_STAGES], (j / TC_STAGES) & 1, limit);
      }
    }
  } else if (warp == 1) {
    // ---------------- MMA issuer ----------------
    if (lane == 0) {
      int it = 0, chunk_i = 0;
      bool ok = true;
      for (int dg = 0; dg < s && ok; ++dg)
        for (int p = 0; p <= dg && ok; ++p)
          for (int c = 0; c < nchunk && ok; ++c, ++chunk_i) {
            const int buf = chunk_i % NBUF;
            if (!mbar_wait(&acc_empty[buf], ((chunk_i / NBUF) & 1) ^ 1, limit) || *(volatile int*)&abort_sh) {
              ok = false;
              break;
            }
            tc_fence_after();
            const uint32_t d = tmem + (uint32_t)(buf * TC_N);
            const int64_t c0 = (int64_t)c * chunk;
            const int nkb = (int)(((Kp - c0) < chunk ? (Kp - c0) : chunk) / TC_KB);
            for (int kb = 0; kb < nkb; ++kb, ++it) {
              const int st = it % TC_STAGES;
              if (!mbar_wait(&full_bar[st], (it / TC_STAGES) & 1, limit) || *(volatile int*)&abort_sh) {
                ok = false;
                break;
              }
              tc_fence_after();
              const uint32_t a = smem_u32(smem + st * TC_STAGE_BYTES);
              const uint32_t b = a + TC_A_BYTES;
#pragma unroll
              for (int kk = 0; kk < TC_KB / 16; ++kk)  // K = 16 per instruction: 32 bytes
                umma<false>(d, sdesc_k128(a + kk * 32), sdesc_k128(b + kk * 32), TC_IDESC, (kb > 0 || kk > 0) ? 1u : 0u);
              if (CS == 1)
                umma_commit(&empty_bar[st]);  // frees the stage once these MMAs have read it
              else
                umma_commit_multicast(&empty_bar[st], (uint16_t)((1u << CS) - 1u));  // in every CTA of the cluster
            }
            if (!ok) break;
            umma_commit(&acc_full[buf]);  // the chunk's accumulator is complete
          }
      if (!ok) {
        atomicCAS(status, 0, FRACLAP_ERR_TIMEOUT);
        abort_sh = 1;
      }
      umma_commit(&done_bar);  // every MMA issued so far has finished when this fires
      mbar_wait(&done_bar, 0, limit);
    }
  } else {
    // ---------------- epilogue: exact integer sums, FP64 once per diagonal ----------------
    // Pairs are visited by diagonal p + q, which share one scale.  A chunk
    // sum is an integer below 2^24 (exact in FP32), so it converts exactly
    // to int32; up to 127 of them add exactly in an int32 accumulator, which
    // is scaled (exactly, by a power of two) and added into C in FP64 at the
    // end of the diagonal (or after 127 chunks).
    const int lg = warp & 3;                          // TMEM lane quarter of this warp
    const int cbase = ((warp - 2) >> 2) * TC_EPI_COLS;  // this warp's columns of the tile
    const int64_t row = m0 + lg * 32 + lane;          // output row of this thread
    const int er = (row < M) ? ea[row] : 0;
    int acc[TC_EPI_COLS];
#pragma unroll
    for (int j = 0; j < TC_EPI_COLS; ++j) acc[j] = 0;
    bool first = true;
    int chunk_i = 0;
    bool ok = true;
    for (int dg = 0; dg < s && ok; ++dg) {
      int pending = 0;
      for (int p = 0; p <= dg && ok; ++p) {
        for (int c = 0; c < nchunk; ++c, ++chunk_i) {
          const int buf = chunk_i % NBUF;
          if (!mbar_wait(&acc_full[buf], (chunk_i / NBUF) & 1, limit) || *(volatile int*)&abort_sh) {
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t taddr = tmem + ((uint32_t)(lg * 32) << 16) + (uint32_t)(buf * TC_N + cbase);
#pragma unroll
          for (int j0 = 0; j0 < TC_EPI_COLS; j0 += 16) {
            uint32_t r[16];
            tmem_ld16(taddr + j0, r);
            tmem_wait_ld();
#pragma unroll
            for (int j = 0; j < 16; ++j) acc[j0 + j] += __float2int_rz(__uint_as_float(r[j]));
          }
          tc_fence_before();
          __syncwarp();
          if (lane == 0) mbar_arrive(&acc_empty[buf]);
          // one call site (the fold is inlined once): after 127 chunks, and
          // after the last chunk of the diagonal
          if (++pending == 127 || (p == dg && c == nchunk - 1)) {
            // fold: acc 2^(e_i + f_j - bits (dg + 2)) into C in FP64, then restart the sums
            const int sh = bits * (dg + 2);
            if (row < M) {
              // opaque copies of the base pointers: the per-column addresses are
              // formed here, not hoisted out of the diagonal loop into registers
              const int* ebp;
              double* cb;
              asm volatile("mov.b64 %0, %1;" : "=l"(ebp) : "l"(eb + n0 + cbase));
              asm volatile("mov.b64 %0, %1;" : "=l"(cb) : "l"(C + row + (n0 + cbase) * ldc));
#pragma unroll
              for (int j = 0; j < TC_EPI_COLS; ++j) {
                const int64_t col = n0 + cbase + j;
                if (col < N && !(lower && row < col)) {
                  // acc 2^e in two exact power-of-two steps (each factor normal);
                  // beyond |e| = 2044 the result is 0 or infinite either way
                  int e = er + ebp[j] - sh;
                  e = (e < -2044) ? -2044 : (e > 2044 ? 2044 : e);
                  const int e1 = e / 2;
                  const double v = alpha * (((double)acc[j] * pow2i(e1)) * pow2i(e - e1));
                  double* cp = cb + j * ldc;
                  *cp = first ? ((beta == 0.0) ? v : v + beta * *cp) : *cp + v;
                }
              }
            }
#pragma unroll
            for (int j = 0; j < TC_EPI_COLS; ++j) acc[j] = 0;
            first = false;
            pending = 0;
          }
        }
      }
    }
    if (!ok) {
      if (lane == 0) atomicCAS(status, 0, FRACLAP_ERR_TIMEOUT);
      abort_sh = 1;
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TC_TMEM_COLS)
                 : "memory");
  }
  if (CS > 1) cluster_sync_all();  // no CTA leaves while a peer may still signal it
}

// 3-D map over the slices S[s][rows][Kp] (bf16), box 64 (K) x box_rows x 1.
bool slice_map(CUtensorMap* map, const __nv_bfloat16* S, int64_t rows, int64_t Kp, int s, int box_rows) {
  EncodeTiledFn fn = encode_tiled();
  if (!fn) return false;
  const cuuint64_t dims[3] = {(cuuint64_t)Kp, (cuuint64_t)rows, (cuuint64_t)s};
  const cuuint64_t strides[2] = {(cuuint64_t)Kp * 2, (cuuint64_t)rows * Kp * 2};
  const cuuint32_t box[3] = {TC_KB, (cuuint32_t)box_rows, 1};
  const cuuint32_t estr[3] = {1, 1, 1};
  return fn(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, (void*)S, dims, strides, box, estr,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}
template <int TCN, int CS>
int launch_tc(fraclap_ctx* ctx, const __nv_bfloat16* SA, const __nv_bfloat16* SB, const int* ea, const int* eb,
              int64_t M, int64_t N, int64_t Kp, int sl, int bits, int64_t chunk, double alpha, double beta,
              double* C, int64_t ldc, bool lower, cudaStream_t st) {
  CUtensorMap ma, mb;
  FL_CHECK(ctx, slice_map(&ma, SA, M, Kp, sl, TC_M) && slice_map(&mb, SB, N, Kp, sl, TCN / CS), FRACLAP_ERR_CUDA,
           "ozaki_gemm: tensor map encoding failed");
  const size_t smem = (size_t)OzTile<TCN>::STAGES * OzTile<TCN>::STAGE_BYTES + 1024;
  auto kern = ozaki_tc_kernel<TCN, CS>;
  FL_CUDA(ctx, cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  // the raster counts clusters of CS tile rows (a tile of CS * 128 rows)
  const int TM = (int)cdiv(cdiv(M, TC_M), CS), TN = (int)cdiv(N, TCN);
  const int G = std::max(1, std::min(ctx->oz_group > 0 ? ctx->oz_group : TM, TM));
  const int64_t tiles = ozaki_tile_count(TM, TN, G, lower, CS * TC_M, TCN);
  FL_CHECK(ctx, tiles * CS <= INT32_MAX, FRACLAP_ERR_UNSUPPORTED, "ozaki_gemm: too many tiles");
  int lw = lower ? 1 : 0;
  if (CS == 1) {
    kern<<<(unsigned)tiles, TC_THREADS, smem, st>>>(ma, mb, ea, eb, M, N, Kp, sl, bits, chunk, alpha, beta, C, ldc,
                                                    lw, G, ctx->wait_cycles, ctx->d_status);
    return 0;
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(tiles * CS));
  cfg.blockDim = dim3(TC_THREADS);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = (unsigned)CS;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  FL_CUDA(ctx, cudaLaunchKernelEx(&cfg, kern, ma, mb, ea, eb, M, N, Kp, sl, bits, chunk, alpha, beta, C, ldc, lw, G,
                                  ctx->wait_cycles, ctx->d_status));
  return 0;
}

}  // namespace

size_t ozaki_ws(int64_t M, int64_t N, int64_t K, int s) {
  const int64_t Kp = cdiv(std::max<int64_t>(K, 1), OZ_KPAD) * OZ_KPAD;
  s = (8 * s + 6) / 7;  // room for the 7-bit slicing
  Arena ar;
  ar.take<__nv_bfloat16>((int64_t)s * M * Kp);
  ar.take<__nv_bfloat16>((int64_t)s * N * Kp);
  ar.take<int>(M);
  ar.take<int>(N);
  ar.take<unsigned long long>(std::max(M, N));
  return ar.off;
}

// Exponents and digit slices of the rows of op(X) (R rows of length K):
// contiguous rows (trans) one block per row; strided rows through the
// column-parallel maximum and the tiled slicing.
int slice_operand(fraclap_ctx* ctx, const double* X, int64_t ldx, bool trans, int64_t R, int64_t K, int64_t Kp,
                  int sl, int bits, int* ex, __nv_bfloat16* S, unsigned long long* mx, cudaStream_t st) {
  if (trans || Kp / 32 > 65535 || cdiv(K, OZ_MAX_KCH) > 65535) {
    row_exponents<<<(unsigned)R, 256, 0, st>>>(X, ldx, trans, K, ex);
    count_launch(ctx);
    if (trans && sl * bits <= 64) {
      const unsigned gs = (unsigned)std::min<int64_t>(cdiv(R * (Kp / 8), 256), 152 * 16);
      make_slices_rows<<<gs, 256, 0, st>>>(X, ldx, R, K, Kp, ex, sl, bits, S);
    } else {
      const unsigned gs = (unsigned)std::min<int64_t>(cdiv(R * Kp, 256), 152 * 32);
      make_slices<<<gs, 256, 0, st>>>(X, ldx, trans, R, K, Kp, ex, sl, bits, S);
    }
    count_launch(ctx);
  } else {
    FL_CUDA(ctx, cudaMemsetAsync(mx, 0, sizeof(unsigned long long) * (size_t)R, st));
    row_absmax_strided<<<dim3((unsigned)cdiv(R, 256), (unsigned)std::max<int64_t>(cdiv(K, OZ_MAX_KCH), 1)), 256, 0,
                         st>>>(X, ldx, R, K, mx);
    count_launch(ctx);
    exponents_of_max<<<(unsigned)cdiv(R, 256), 256, 0, st>>>(mx, R, ex);
    count_launch(ctx);
    make_slices_strided<<<dim3((unsigned)cdiv(R, 32), (unsigned)(Kp / 32)), dim3(32, 8), 0, st>>>(
        X, ldx, R, K, Kp, ex, sl, bits, S);
    count_launch(ctx);
  }
  FL_CUDA(ctx, cudaGetLastError());
  return 0;
}

// C = alpha op(A) op(B) + beta C, FP64-accurate through s BF16 slices
// (s = 7 for full FP64 accuracy of the products).  lower: only C(i,j), i >= j.
int ozaki_gemm(fraclap_ctx* ctx, bool ta, bool tb, int64_t M, int64_t N, int64_t K, double alpha,
               const double* A, int64_t lda, const double* B, int64_t ldb, double beta, double* C,
               int64_t ldc, int s, bool lower, Arena* ar, cudaStream_t st) {
  if (M <= 0 || N <= 0) return 0;
  FL_CHECK(ctx, s >= 1 && s <= 8, FRACLAP_ERR_INVALID_ARG, "ozaki_gemm: slices must be 1..8");
  FL_CHECK(ctx, cdiv(N, OZ_BN) <= 65535, FRACLAP_ERR_UNSUPPORTED, "ozaki_gemm: N too large");
  const int64_t Kp = cdiv(std::max<int64_t>(K, 1), OZ_KPAD) * OZ_KPAD;
  const int smax = (8 * s + 6) / 7;
  __nv_bfloat16* SA = ar->take<__nv_bfloat16>((int64_t)smax * M * Kp);
  __nv_bfloat16* SB = ar->take<__nv_bfloat16>((int64_t)smax * N * Kp);
  int* ea = ar->take<int>(M);
  int* eb = ar->take<int>(N);
  unsigned long long* mx = ar->take<unsigned long long>(std::max(M, N));
  FL_CHECK(ctx, mx != nullptr, FRACLAP_ERR_ALLOC, "ozaki_gemm: workspace too small");
  // op(A) rows: trans -> A stored K x M; op(B) columns = rows of op(B)^T
  // slice width: 8 bits (exact chunks of 256) for short K, else 7 bits (exact
  // chunks of 1024) with one more slice for the same 8s bits: 3x fewer folds.
  int bits = 8, sl = s;
  if (K > 256 && ctx->oz_bits != 8) {
    bits = 7;
    sl = (8 * s + 6) / 7;
  }
  const int64_t chunk = (int64_t)1 << (24 - 2 * bits);
  // rows of op(A) and columns of op(B): contiguous when trans, else strided
  FL_TRY(slice_operand(ctx, A, lda, ta, M, K, Kp, sl, bits, ea, SA, mx, st));
  FL_TRY(slice_operand(ctx, B, ldb, !tb, N, K, Kp, sl, bits, eb, SB, mx, st));
  StageTimer tm(ctx, kStageSliceProducts, st);
  if (ctx->tensor_route == 1) {
    const int tw = (N <= 128) ? 128 : ctx->oz_tile_n;  // a narrow output takes the 128-column tile
    const int cs = ctx->oz_cluster;
#define FL_OZ_LAUNCH(W, K) \
  launch_tc<W, K>(ctx, SA, SB, ea, eb, M, N, Kp, sl, bits, chunk, alpha, beta, C, ldc, lower, st)
    if (cs == 2) {
      FL_TRY(tw == 256 ? FL_OZ_LAUNCH(256, 2) : tw == 192 ? FL_OZ_LAUNCH(192, 2) : FL_OZ_LAUNCH(128, 2));
    } else {
      FL_TRY(tw == 256 ? FL_OZ_LAUNCH(256, 1) : tw == 192 ? FL_OZ_LAUNCH(192, 1) : FL_OZ_LAUNCH(128, 1));
    }
#undef FL_OZ_LAUNCH
  } else {
    dim3 grid((unsigned)cdiv(M, OZ_BM), (unsigned)cdiv(N, OZ_BN));
    ozaki_kernel<<<grid, OZ_NT, 0, st>>>(SA, SB, ea, eb, M, N, Kp, sl, bits, chunk, alpha, beta, C, ldc, lower);
  }
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

extern "C" int fraclap_set_schedule(fraclap_ctx* ctx, int knob, int value) {
  if (!ctx) return FRACLAP_ERR_INVALID_ARG;
  switch (knob) {
    case FRACLAP_SCHED_OZAKI_GROUP:
      FL_CHECK(ctx, value >= 0 && value <= 4096, FRACLAP_ERR_INVALID_ARG, "set_schedule: group must be 0..4096");
      ctx->oz_group = value;
      return 0;
    case FRACLAP_SCHED_OZAKI_BITS:
      FL_CHECK(ctx, value == 7 || value == 8, FRACLAP_ERR_INVALID_ARG, "set_schedule: digit width must be 7 or 8");
      ctx->oz_bits = value;
      return 0;
    case FRACLAP_SCHED_FP32_STAGES:
      FL_CHECK(ctx, value == 0 || value == 1, FRACLAP_ERR_INVALID_ARG, "set_schedule: FP32 stage route must be 0 or 1");
      ctx->fp32_stages_tc = value;
      return 0;
    case FRACLAP_SCHED_OZAKI_TILE_N:
      FL_CHECK(ctx, value == 128 || value == 192 || value == 256, FRACLAP_ERR_INVALID_ARG,
               "set_schedule: tile width must be 128, 192 or 256");
      ctx->oz_tile_n = value;
      return 0;
    case FRACLAP_SCHED_Q2_PARTS:
      FL_CHECK(ctx, value == 0 || value == 4 || value == 8 || value == 16, FRACLAP_ERR_INVALID_ARG,
               "set_schedule: Q2 parts must be 0, 4, 8 or 16");
      ctx->q2_parts = value;
      return 0;
    case FRACLAP_SCHED_OZAKI_CLUSTER:
      FL_CHECK(ctx, value == 1 || value == 2, FRACLAP_ERR_INVALID_ARG,
               "set_schedule: slice-product cluster must be 1 or 2 CTAs");
      ctx->oz_cluster = value;
      return 0;
    default:
      return set_error(ctx, FRACLAP_ERR_INVALID_ARG, "set_schedule: unknown knob %d", knob);
  }
}

extern "C" int fraclap_get_schedule(const fraclap_ctx* ctx, int knob) {
  if (!ctx) return FRACLAP_ERR_INVALID_ARG;
  switch (knob) {
    case FRACLAP_SCHED_OZAKI_GROUP: return ctx->oz_group;
    case FRACLAP_SCHED_OZAKI_BITS: return ctx->oz_bits;
    case FRACLAP_SCHED_FP32_STAGES: return ctx->fp32_stages_tc;
    case FRACLAP_SCHED_OZAKI_TILE_N: return ctx->oz_tile_n;
    case FRACLAP_SCHED_Q2_PARTS: return ctx->q2_parts;
    case FRACLAP_SCHED_OZAKI_CLUSTER: return ctx->oz_cluster;
    default: return FRACLAP_ERR_INVALID_ARG;
  }
}
