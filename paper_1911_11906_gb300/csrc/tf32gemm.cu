// FP32 GEMM on the tensor cores from three TF32 products.
//
// Every FP32 operand entry x is split into hi = tf32(x) (round to nearest,
// 10 explicit mantissa bits) and lo = tf32(x - hi) (x - hi is exact in
// FP32), and C = alpha (A_hi B_hi + A_hi B_lo + A_lo B_hi) + beta C: the
// dropped lo*lo term and the two roundings leave a relative error of a few
// 2^-22 per product, the level of an FP32 accumulation.  A split pass writes
// op(A) and op(B)^T K-major as [hi | hi | lo] and [hi | lo | hi] (each part
// padded to 32 entries), so that one TF32 GEMM over 3K forms the sum; it also
// reads the symmetric-A form (lower triangle) and concatenates a fused second
// product along K.  The MMA kernel is a plain tcgen05 GEMM: CTA tile 128 x
// 128, warp 0 issues TMA tile loads (128-byte swizzle, three 32 KB stages),
// warp 1 owns the 128-column TMEM accumulator and issues
// tcgen05.mma.kind::tf32 (K = 8 per instruction), warps 2-5 read the
// accumulator back with tcgen05.ld and write alpha acc + beta C.  Every
// mbarrier wait is bounded.
#include "internal.cuh"
#include "tc_common.cuh"

namespace fraclap {
namespace {

using namespace tc;

constexpr int TG_M = 128, TG_N = 128, TG_KB = 32, TG_STAGES = 3;
constexpr int TG_A_BYTES = TG_M * TG_KB * 4, TG_B_BYTES = TG_N * TG_KB * 4;
constexpr int TG_STAGE_BYTES = TG_A_BYTES + TG_B_BYTES;
constexpr int TG_THREADS = 192;
constexpr uint32_t TG_TMEM_COLS = TG_N;
// kind::tf32 instruction descriptor: D F32, A and B TF32, both K-major, M 128, N 128.
constexpr uint32_t TG_IDESC = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(TG_N >> 3) << 17) |
                              ((uint32_t)(TG_M >> 4) << 24);

__device__ __forceinline__ float to_tf32(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}

// Entry (r, k) of a row operand: op(A) row r, or op(B) column r.
// layout 0: P[r + k ld]; 1: P[k + r ld]; 2: symmetric, lower triangle of P.
// k >= K1 reads the second source (same layout) at k - K1.
struct SplitSrc {
  const float* P;
  int64_t ld;
  const float* P2;
  int64_t ld2;
  int64_t K1, K2, rows;
  int layout;
};

__device__ __forceinline__ float split_val(const SplitSrc& s, int64_t r, int64_t k) {
  if (r >= s.rows || k >= s.K1 + s.K2) return 0.0f;
  const float* P = s.P;
  int64_t ld = s.ld;
  if (k >= s.K1) {
    P = s.P2;
    ld = s.ld2;
    k -= s.K1;
  }
  if (s.layout == 0) return P[r + k * ld];
  if (s.layout == 1) return P[k + r * ld];
  return (r >= k) ? P[r + k * ld] : P[k + r * ld];
}

// S[r][part * Kp + k] for the three parts; 32 x 32 tiles through shared
// memory so that both the source and the K-major output are read / written
// along their contiguous index.  Block (32, 8).
__global__ void __launch_bounds__(256) split_tf32(SplitSrc src, int64_t Kp, int b_side, float* S) {
  __shared__ float tile[32][33];  // [k][r]
  const int tx = threadIdx.x, ty = threadIdx.y;
  const int64_t k0 = (int64_t)blockIdx.x * 32, r0 = (int64_t)blockIdx.y * 32;
  if (src.layout == 1) {
#pragma unroll
    for (int q = 0; q < 4; ++q) tile[tx][ty + 8 * q] = split_val(src, r0 + ty + 8 * q, k0 + tx);
  } else {
#pragma unroll
    for (int q = 0; q < 4; ++q) tile[ty + 8 * q][tx] = split_val(src, r0 + tx, k0 + ty + 8 * q);
  }
  __syncthreads();
  const int64_t Kq = 3 * Kp;
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int64_t r = r0 + ty + 8 * q;
    if (r >= src.rows) continue;
    const float x = tile[tx][ty + 8 * q];
    const float hi = to_tf32(x);
    const float lo = to_tf32(x - hi);
    float* row = S + r * Kq + k0 + tx;
    row[0] = hi;
    row[Kp] = b_side ? lo : hi;
    row[2 * Kp] = b_side ? hi : lo;
  }
}

// Split-K: CTA z of gridDim.z takes the K-blocks [z kb_per, (z + 1) kb_per)
// and adds alpha acc into C with atomics (the caller has scaled C by beta).
__global__ void __launch_bounds__(TG_THREADS, 1)
tf32_gemm_kernel(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapB, int64_t M,
                 int64_t N, int64_t Kq, float alpha, float beta, float* C, int64_t ldc, int lower, int kb_per,
                 long long limit, int32_t* status) {
  extern __shared__ __align__(1024) unsigned char tg_smem_raw[];
  unsigned char* smem = (unsigned char*)(((uintptr_t)tg_smem_raw + 1023) & ~(uintptr_t)1023);
  __shared__ __align__(8) uint64_t full_bar[TG_STAGES], empty_bar[TG_STAGES];
  __shared__ __align__(8) uint64_t acc_full, done_bar;
  __shared__ uint32_t tmem_base_sh;
  __shared__ int abort_sh;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t m0 = (int64_t)blockIdx.x * TG_M, n0 = (int64_t)blockIdx.y * TG_N;
  if (lower && m0 + TG_M - 1 < n0) return;  // whole tile above the diagonal
  const int nkb_all = (int)(Kq / TG_KB);
  const int kb0 = (int)blockIdx.z * kb_per;
  const int nkb = (kb0 + kb_per < nkb_all ? kb0 + kb_per : nkb_all) - kb0;  // this CTA's K-blocks
  if (nkb <= 0) return;
  const bool split = gridDim.z > 1;

  if (threadIdx.x == 0) {
    for (int i = 0; i < TG_STAGES; ++i) {
      mbar_init(&full_bar[i], 1);
      mbar_init(&empty_bar[i], 1);
    }
    mbar_init(&acc_full, 1);
    mbar_init(&done_bar, 1);
    abort_sh = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(&tmem_base_sh)),
                 "r"(TG_TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_base_sh;

  if (warp == 0) {
    // ---------------- TMA producer ----------------
    if (lane == 0) {
      int kb = 0;
      bool ok = true;
      for (; kb < nkb; ++kb) {
        const int st = kb % TG_STAGES;
        if (!mbar_wait(&empty_bar[st], ((kb / TG_STAGES) & 1) ^ 1, limit) || *(volatile int*)&abort_sh) {
          ok = false;
          break;
        }
        unsigned char* a = smem + st * TG_STAGE_BYTES;
        unsigned char* b = a + TG_A_BYTES;
        mbar_expect_tx(&full_bar[st], TG_STAGE_BYTES);
        tma_load_2d(a, &mapA, &full_bar[st], (kb0 + kb) * TG_KB, (int)m0);
        tma_load_2d(b, &mapB, &full_bar[st], (kb0 + kb) * TG_KB, (int)n0);
      }
      if (!ok) {
        atomicCAS(status, 0, FRACLAP_ERR_TIMEOUT);
        abort_sh = 1;
        // let the copies already issued land before the CTA can exit
        for (int j = (kb > TG_STAGES ? kb - TG_STAGES : 0); j < kb; ++j)
          mbar_wait(&full_bar[j % TG_STAGES], (j / TG_STAGES) & 1, limit);
      }
    }
  } else if (warp == 1) {
    // ---------------- MMA issuer ----------------
    if (lane == 0) {
      bool ok = true;
      for (int kb = 0; kb < nkb; ++kb) {
        const int st = kb % TG_STAGES;
        if (!mbar_wait(&full_bar[st], (kb / TG_STAGES) & 1, limit) || *(volatile int*)&abort_sh) {
          ok = false;
          break;
        }
        tc_fence_after();
        const uint32_t a = smem_u32(smem + st * TG_STAGE_BYTES);
        const uint32_t b = a + TG_A_BYTES;
#pragma unroll
        for (int kk = 0; kk < TG_KB / 8; ++kk)  // K = 8 TF32 per instruction: 32 bytes
          umma<true>(tmem, sdesc_k128(a + kk * 32), sdesc_k128(b + kk * 32), TG_IDESC,
                     (kb > 0 || kk > 0) ? 1u : 0u);
        umma_commit(&empty_bar[st]);  // frees the stage once these MMAs have read it
      }
      if (ok) {
        umma_commit(&acc_full);  // the accumulator is complete
      } else {
        atomicCAS(status, 0, FRACLAP_ERR_TIMEOUT);
        abort_sh = 1;
      }
      umma_commit(&done_bar);  // every MMA issued so far has finished when this fires
      mbar_wait(&done_bar, 0, limit);
    }
  } else {
    // ---------------- epilogue ----------------
    const int lg = warp & 3;                  // TMEM lane quarter of this warp
    const int64_t row = m0 + lg * 32 + lane;  // output row of this thread
    bool ok = true;
    const long long t0 = clock64();
    while (!mbar_try_wait(&acc_full, 0)) {
      if (*(volatile int*)&abort_sh) {
        ok = false;
        break;
      }
      if (clock64() - t0 > limit) {  // the MMA warp's own waits are bounded too
        if (lane == 0) atomicCAS(status, 0, FRACLAP_ERR_TIMEOUT);
        ok = false;
        break;
      }
    }
    if (ok) {
      tc_fence_after();
      const uint32_t taddr = tmem + ((uint32_t)(lg * 32) << 16);
#pragma unroll
      for (int j0 = 0; j0 < TG_N; j0 += 16) {
        uint32_t r[16];
        tmem_ld16(taddr + j0, r);
        tmem_wait_ld();
        if (row < M) {
#pragma unroll
          for (int j = 0; j < 16; ++j) {
            const int64_t col = n0 + j0 + j;
            if (col >= N || (lower && row < col)) continue;
            float* cp = C + row + col * ldc;
            const float v = alpha * __uint_as_float(r[j]);
            if (split) atomicAdd(cp, v);
            else *cp = (beta == 0.0f) ? v : v + beta * *cp;
          }
        }
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TG_TMEM_COLS)
                 : "memory");
  }
}

// 2-D map over a K-major split operand S[rows][Kq] (FP32), box 32 (K) x 128.
bool split_map(CUtensorMap* map, const float* S, int64_t rows, int64_t Kq) {
  EncodeTiledFn fn = encode_tiled();
  if (!fn) return false;
  const cuuint64_t dims[2] = {(cuuint64_t)Kq, (cuuint64_t)rows};
  const cuuint64_t strides[1] = {(cuuint64_t)Kq * 4};
  const cuuint32_t box[2] = {TG_KB, 128};
  const cuuint32_t estr[2] = {1, 1};
  return fn(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, (void*)S, dims, strides, box, estr,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

int64_t pad32(int64_t k) { return cdiv(std::max<int64_t>(k, 1), 32) * 32; }

}  // namespace

size_t tf32_split_bytes(int64_t M, int64_t N, int64_t K) {
  const int64_t Kq = 3 * pad32(K);
  return (size_t)(align256((size_t)M * Kq * 4) + align256((size_t)N * Kq * 4));
}

bool tf32_route_fits(const fraclap_ctx* ctx, GemmMode mode, const GemmDescT<float>& d, int split_k) {
  if (!ctx->tc_scratch || ctx->tensor_route != 1) return false;
  if (split_k > 1 && d.beta != 1.0) return false;
  if (mode != kGemmPlain && mode != kGemmSymA && mode != kGemmLowerC) return false;
  const int64_t Kt = d.K + (d.K2 > 0 ? d.K2 : 0);
  if (d.M < 128 || d.N < 64 || Kt < 64) return false;
  if (d.M > INT32_MAX || d.N > INT32_MAX) return false;
  return tf32_split_bytes(d.M, d.N, Kt) <= ctx->tc_scratch_bytes;
}

int gemm_tf32x3(fraclap_ctx* ctx, bool ta, bool tb, GemmMode mode, const GemmDescT<float>& d, int split_k,
                cudaStream_t st) {
  const int64_t K2 = (d.K2 > 0) ? d.K2 : 0;
  const int64_t Kt = d.K + K2, Kp = pad32(Kt), Kq = 3 * Kp;
  float* Sa = reinterpret_cast<float*>(ctx->tc_scratch);
  float* Sb = reinterpret_cast<float*>(reinterpret_cast<char*>(ctx->tc_scratch) +
                                       align256((size_t)d.M * Kq * 4));
  SplitSrc sa{d.A, d.lda, d.A2, d.lda2, d.K, K2, d.M, (mode == kGemmSymA) ? 2 : (ta ? 1 : 0)};
  // op(B) column j, entry k: tb ? B[j + k ldb] : B[k + j ldb]
  SplitSrc sb{d.B, d.ldb, d.B2, d.ldb2, d.K, K2, d.N, tb ? 0 : 1};
  const dim3 blk(32, 8);
  split_tf32<<<dim3((unsigned)(Kp / 32), (unsigned)cdiv(d.M, 32)), blk, 0, st>>>(sa, Kp, 0, Sa);
  count_launch(ctx);
  split_tf32<<<dim3((unsigned)(Kp / 32), (unsigned)cdiv(d.N, 32)), blk, 0, st>>>(sb, Kp, 1, Sb);
  count_launch(ctx);
  CUtensorMap ma, mb;
  FL_CHECK(ctx, split_map(&ma, Sa, d.M, Kq) && split_map(&mb, Sb, d.N, Kq), FRACLAP_ERR_CUDA,
           "gemm_tf32x3: tensor map encoding failed");
  const size_t smem = (size_t)TG_STAGES * TG_STAGE_BYTES + 1024;
  FL_CUDA(ctx, cudaFuncSetAttribute(tf32_gemm_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  const int nkb = (int)(Kq / TG_KB);
  const int splits = std::max(1, std::min(split_k, nkb));
  const int kb_per = (int)cdiv(nkb, splits);
  const dim3 grid((unsigned)cdiv(d.M, TG_M), (unsigned)cdiv(d.N, TG_N), (unsigned)cdiv(nkb, kb_per));
  FL_CHECK(ctx, grid.y <= 65535, FRACLAP_ERR_UNSUPPORTED, "gemm_tf32x3: N too large");
  tf32_gemm_kernel<<<grid, TG_THREADS, smem, st>>>(ma, mb, d.M, d.N, Kq, (float)d.alpha, (float)d.beta, d.C,
                                                   d.ldc, mode == kGemmLowerC ? 1 : 0, kb_per, ctx->wait_cycles,
                                                   ctx->d_status);
  count_launch(ctx);
  FL_CUDA(ctx, cudaGetLastError());
  return 0;
}

}  // namespace fraclap
