// Internal declarations of the fraclap CUDA library (sm_103a).
#pragma once

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>
#include <stdint.h>
#include <stdio.h>

#include <algorithm>
#include <string>
#include <vector>

#include "../../include/fraclap.h"

struct fraclap_ctx {
  int device = 0;
  int sm_count = 0;
  int band_width = 32;
  int leaf_size = 32;
  double wait_timeout_s = 10.0;
  int tensor_route = 1;          // slice products: 1 = tcgen05 + TMA, 0 = mma.sync
  double refine_tau = 1e-3;      // first-order coefficient above which a pair is clustered
  int apply_slices = 0;          // frac_apply products: 0 = FP64 engine, s = s BF16 slices (tensor cores)
  int oz_group = 8;              // slice-product kernel: tile rows per raster group (0 = all rows)
  int oz_bits = 7;               // slice-product kernel: digit width for K > 256 (7 or 8)
  int oz_tile_n = 192;           // slice-product kernel: tile columns (128, 192 or 256)
  int oz_cluster = 1;            // slice-product kernel: CTAs per cluster sharing a B tile (1 or 2)
  int q2_parts = 0;              // stage-2 back-transformation at b = 64: lane parts per window (0: default 8)
  int fp32_stages_tc = 0;        // mixed route: FP32 band reduction and Q1 products on the tensor cores (TF32 x 3)
  void* tc_scratch = nullptr;    // split operands of the TF32 tensor-core route of FP32 GEMMs
  size_t tc_scratch_bytes = 0;   // (set by the caller of the FP32 stages, null otherwise)
  long long wait_cycles = 0;     // wait_timeout_s in SM clock cycles (upper bound)
  int32_t* d_status = nullptr;   // device status word (0 = ok, else a FRACLAP_ERR_*)
  unsigned* d_barrier = nullptr; // grid-barrier state for cooperative kernels
  void* ws = nullptr;            // context-owned workspace
  size_t ws_bytes = 0;
  std::string last_error;
  long long launches = 0;        // kernels launched through this context
  bool profiling = false;        // record CUDA events around every stage
  struct StageEvent { int stage; cudaEvent_t start, stop; };
  std::vector<StageEvent> stage_events;
  // per refinement iteration: delta, ||S-D||_2 est, ||R||_2 est, ||S-D||_F,
  // ||R||_F, ||A||_2 bound, clusters, largest cluster
  std::vector<double> refine_stats;
  // workers of the batched solver (created on first use): sub-contexts with
  // a share of the SMs, their streams and completion events
  std::vector<fraclap_ctx*> workers;
  std::vector<cudaStream_t> worker_streams;
  std::vector<cudaEvent_t> worker_events;
  cudaEvent_t batch_start = nullptr;
};

namespace fraclap {

// ---------------------------------------------------------------------------
// error handling
// ---------------------------------------------------------------------------
int set_error(fraclap_ctx* ctx, int code, const char* fmt, ...);

#define FL_CUDA(ctx, call)                                                          \
  do {                                                                              \
    cudaError_t e_ = (call);                                                        \
    if (e_ != cudaSuccess)                                                          \
      return ::fraclap::set_error((ctx), FRACLAP_ERR_CUDA, "%s failed: %s (%s:%d)", #call, \
                                  cudaGetErrorString(e_), __FILE__, __LINE__);     \
  } while (0)

#define FL_CHECK(ctx, cond, code, ...)                                   \
  do {                                                                   \
    if (!(cond)) return ::fraclap::set_error((ctx), (code), __VA_ARGS__); \
  } while (0)

#define FL_TRY(expr)          \
  do {                        \
    int rc_ = (expr);         \
    if (rc_ != 0) return rc_; \
  } while (0)

inline void count_launch(fraclap_ctx* c) { c->launches++; }

// Stages timed by fraclap_stage_times (ids are part of the C ABI).
enum Stage : int {
  kStageAssemble = 0,
  kStageBandReduction = 1,
  kStageBulgeChasing = 2,
  kStageTridiagDC = 3,
  kStageBackQ2 = 4,
  kStageBackQ1 = 5,
  kStageApply = 6,
  kStageRefine = 7,
  kStageResidualGemm = 8,
  kStageRefineNorms = 9,      // A X, power iterations, threshold
  kStageRefineUpdate = 10,    // unsafe pairs, correction, X += X E
  kStageRefineSort = 11,      // ranks and column permutation
  kStageRefineClusters = 12,  // exact diagonalisation of the clusters (up to 64)
  kStageRefineBigClusters = 13,  // clusters above 64 (dense FP64 solver)
  kStageSliceProducts = 14,   // the slice-product kernel of an FP64-accurate product
  kStageCount = 15
};

// NVTX range names of the stages ("fraclap:" + the name the binding reports).
inline const char* stage_range_name(int s) {
  static const char* names[kStageCount] = {
      "fraclap:assemble",      "fraclap:band_reduction", "fraclap:bulge_chasing",  "fraclap:tridiag_dc",
      "fraclap:back_q2",       "fraclap:back_q1",        "fraclap:apply",          "fraclap:refine",
      "fraclap:residual_gemm", "fraclap:refine_norms",   "fraclap:refine_update",  "fraclap:refine_sort",
      "fraclap:refine_clusters", "fraclap:refine_big_clusters", "fraclap:slice_products"};
  return (s >= 0 && s < kStageCount) ? names[s] : "fraclap";
}

// Marks a stage with an NVTX range (host timeline, always; free without a
// tool attached) and, when profiling is on, records CUDA events around it
// on `st`.
struct StageTimer {
  fraclap_ctx* ctx;
  int stage;
  cudaStream_t st;
  cudaEvent_t e0 = nullptr;
  StageTimer(fraclap_ctx* c, int s, cudaStream_t stream) : ctx(c), stage(s), st(stream) {
    nvtxRangePushA(stage_range_name(s));
    if (ctx->profiling && cudaEventCreate(&e0) == cudaSuccess) cudaEventRecord(e0, st);
  }
  ~StageTimer() {
    nvtxRangePop();
    if (!e0) return;
    cudaEvent_t e1;
    if (cudaEventCreate(&e1) == cudaSuccess) {
      cudaEventRecord(e1, st);
      ctx->stage_events.push_back({stage, e0, e1});
    } else {
      cudaEventDestroy(e0);
    }
  }
};

// Consecutive spans on one stream: start(id) closes the previous span.
struct StageSpan {
  fraclap_ctx* ctx;
  cudaStream_t st;
  int stage = -1;
  cudaEvent_t e0 = nullptr;
  bool range_open = false;
  StageSpan(fraclap_ctx* c, cudaStream_t s) : ctx(c), st(s) {}
  void start(int id) {
    stop();
    nvtxRangePushA(stage_range_name(id));
    range_open = true;
    if (!ctx->profiling) return;
    stage = id;
    if (cudaEventCreate(&e0) == cudaSuccess) cudaEventRecord(e0, st);
    else e0 = nullptr;
  }
  void stop() {
    if (range_open) {
      nvtxRangePop();
      range_open = false;
    }
    if (!e0) return;
    cudaEvent_t e1;
    if (cudaEventCreate(&e1) == cudaSuccess) {
      cudaEventRecord(e1, st);
      ctx->stage_events.push_back({stage, e0, e1});
    } else {
      cudaEventDestroy(e0);
    }
    e0 = nullptr;
  }
  ~StageSpan() { stop(); }
};

inline int64_t cdiv(int64_t a, int64_t b) { return (a + b - 1) / b; }
inline size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

// Bump allocator over a workspace buffer.
struct Arena {
  char* base = nullptr;
  size_t cap = 0, off = 0;
  template <class T>
  T* take(int64_t count) {
    size_t bytes = align256(sizeof(T) * (size_t)(count > 0 ? count : 1));
    if (base == nullptr) {  // sizing pass
      off += bytes;
      return nullptr;
    }
    if (off + bytes > cap) return nullptr;
    T* p = reinterpret_cast<T*>(base + off);
    off += bytes;
    return p;
  }
};

// Context workspace: the caller's buffer or the context's own (grown).
int get_workspace(fraclap_ctx* ctx, void* work, size_t work_bytes, size_t need, Arena* arena);

// ---------------------------------------------------------------------------
// GEMM engine (FP64 SIMT; the FP64 pipe of GB300 is the bound, see gemm.cu)
// ---------------------------------------------------------------------------
enum GemmMode : int {
  kGemmPlain = 0,     // C = alpha op(A) op(B) + beta C
  kGemmLowerC = 1,    // only C(i, j) with i >= j is written (tiles above skipped)
  kGemmSymA = 2,      // A is symmetric, only its lower triangle is read (M == K)
};

template <class T>
struct GemmDescT {
  int64_t M, N, K;
  const T* A; int64_t lda;
  const T* B; int64_t ldb;
  T* C; int64_t ldc;
  // optional second product accumulated into the same C (K2 = 0: none):
  // C = alpha (op(A) op(B) + op(A2) op(B2)) + beta C, same transposes.
  const T* A2; int64_t lda2;
  const T* B2; int64_t ldb2;
  int64_t K2;
  double alpha, beta;
};
using GemmDesc = GemmDescT<double>;

// One product (T = double: FP64 FMA; T = float: FP32 FMA with FP32
// accumulation); split_k > 1 accumulates partial sums with atomics (beta must
// be 1 and C pre-scaled/zeroed by the caller).
template <class T>
int gemm(fraclap_ctx* ctx, bool ta, bool tb, GemmMode mode, const GemmDescT<T>& d, int split_k,
         cudaStream_t st);
// FP32 GEMM on the tensor cores (three TF32 products, FP32-level accuracy),
// through the split-operand scratch in ctx->tc_scratch; gemm<float> takes
// this route when tf32_route_fits (modes Plain, SymA, LowerC; M >= 128,
// N >= 64, K + K2 >= 64, tensor route 1, scratch large enough; split-K with
// beta = 1 adds into C with atomics, as the FMA kernels do).
size_t tf32_split_bytes(int64_t M, int64_t N, int64_t K);
bool tf32_route_fits(const fraclap_ctx* ctx, GemmMode mode, const GemmDescT<float>& d, int split_k);
int gemm_tf32x3(fraclap_ctx* ctx, bool ta, bool tb, GemmMode mode, const GemmDescT<float>& d, int split_k,
                cudaStream_t st);
// Batched over a device array of descriptors; grid covers max_m x max_n tiles,
// tiles outside a descriptor's M x N exit.  Descriptors with M, N or K <= 0
// are skipped.
template <class T>
int gemm_batched(fraclap_ctx* ctx, bool ta, bool tb, const GemmDescT<T>* d_descs, int count,
                 int64_t max_m, int64_t max_n, cudaStream_t st);

// ---------------------------------------------------------------------------
// stages
// ---------------------------------------------------------------------------
// Stage 1 (dense -> band) workspace: compact-WY panels kept for the
// back-transformation.
// T is the storage/GEMM type (double, or float on the mixed path); the
// Householder norms, scalings and the T-factor recurrence are FP64 always.
template <class T>
struct Stage1T {
  T* Vstore;         // sum_j m_j * b: explicit V of every panel
  T* Tstore;         // npanel * b * b
  double* tau;       // npanel * b
  T* XT;             // n * b
  T* X;              // n * b
  T* Y;              // b * b
  T* Mm;             // b * b
  double* gram;      // b * b
  T* gramT;          // b * b (cluster panel route)
  double* partials;  // 2 * G * 2b
  int64_t npanel;
  int64_t vtotal;
};
using Stage1 = Stage1T<double>;
int64_t stage1_panels(int64_t n, int b);
template <class T>
int stage1_take(Arena* ar, int64_t n, int b, int G, Stage1T<T>* s);
template <class T>
int sy2sb_run(fraclap_ctx* ctx, T* Aw, int64_t n, int64_t lda, int b, T* band, Stage1T<T>* s,
              cudaStream_t st);
template <class T>
int q1_apply_run(fraclap_ctx* ctx, const Stage1T<T>* s, int64_t n, int b, T* Z, int64_t ldz,
                 int64_t ncols, T* W1, T* W2, cudaStream_t st);

// Stage 2 (band -> tridiagonal) workspace: the bulge-chasing reflectors.
template <class T>
struct Stage2T {
  T* refl;        // (n-1) * kmax * b
  double* rtau;   // (n-1) * kmax
  int* progress;  // 2 (n + 1): completed steps per sweep, then published subdiagonal values
  int64_t kmax;
};
using Stage2 = Stage2T<double>;
template <class T>
int stage2_take(Arena* ar, int64_t n, int b, Stage2T<T>* s);
// Band (T) -> tridiagonal (d, e in FP64).
template <class T>
int sb2st_run(fraclap_ctx* ctx, T* band, int64_t n, int b, double* d, double* e, Stage2T<T>* s,
              cudaStream_t st);
// Z <- Q2 Z through a transposed copy Yt (ncols x n, ld ldy >= ncols).
template <class T>
int q2_apply_run(fraclap_ctx* ctx, const Stage2T<T>* s, int64_t n, int b, T* Z, int64_t ldz,
                 int64_t ncols, T* Yt, int64_t ldy, cudaStream_t st);
template <class T>
int transpose_run(fraclap_ctx* ctx, const T* A, int64_t lda, T* Bm, int64_t ldb, int64_t rows,
                  int64_t cols, cudaStream_t st);

// Tridiagonal divide and conquer: secular equations, deflation and the
// Gu-Eisenstat vectors in FP64; eigenvectors stored and merged in T.
template <class T>
size_t stedc_ws(const fraclap_ctx* ctx, int64_t n);
template <class T>
int stedc_run(fraclap_ctx* ctx, const double* d, const double* e, int64_t n, double* lambda, T* Z,
              int64_t ldz, Arena* arena, cudaStream_t st);

// Dense FP64 eigendecomposition of a small symmetric c x c matrix S (lower
// triangle, ld c; overwritten) into w (ascending) and Q (c x c, ld c), with
// the same stages as eig_full; used for large clusters in the refinement.
size_t cluster_eig_ws(const fraclap_ctx* ctx, int64_t c);
int cluster_eig(fraclap_ctx* ctx, double* S, int64_t c, double* w, double* Q, Arena* ar,
                cudaStream_t st);

// FP64-accurate GEMM through BF16 tensor-core slices (ozaki.cu).
size_t ozaki_ws(int64_t M, int64_t N, int64_t K, int s);
int ozaki_gemm(fraclap_ctx* ctx, bool ta, bool tb, int64_t M, int64_t N, int64_t K, double alpha,
               const double* A, int64_t lda, const double* B, int64_t ldb, double beta, double* C,
               int64_t ldc, int s, bool lower, Arena* ar, cudaStream_t st);

// Banded LDL^T (no pivoting) of the symmetric CSR matrix of half-bandwidth
// b: Lb(t, j) = L(j + t, j), Lr(t, i) = L(i, i - t) (both ld b + 1, n
// columns), D the pivots; a pivot <= 0 raises FRACLAP_ERR_NOT_SPD in the
// device status (slicing.cu).  The half-bandwidth query synchronises st.
size_t band_ldlt_ws(int64_t n, int64_t b);
int band_ldlt(fraclap_ctx* ctx, int64_t n, const int64_t* rowptr, const int32_t* col, const double* val, int64_t b,
              double* Lb, double* Lr, double* D, Arena* ar, cudaStream_t st);
int csr_half_bandwidth(fraclap_ctx* ctx, int64_t n, const int64_t* rowptr, const int32_t* col, int64_t* bw,
                       cudaStream_t st);

// Ogita-Aishima refinement of (X, lambda) against the CSR matrix A.
size_t refine_ws(const fraclap_ctx* ctx, int64_t n);
int refine_run(fraclap_ctx* ctx, int64_t n, const int64_t* rowptr, const int32_t* col,
               const double* val, double* X, int64_t ldx, double* lambda, int iters, Arena* ar,
               cudaStream_t st);

// ---------------------------------------------------------------------------
// device helpers
// ---------------------------------------------------------------------------
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__device__ __forceinline__ int ld_acquire_gpu(const int* p) {
  int v;
  asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release_gpu(int* p, int v) {
  asm volatile("st.release.gpu.global.s32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ unsigned ld_acquire_gpu_u(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// Records the first failure code in the device status word.
__device__ __forceinline__ void raise_status(int32_t* status, int code) {
  atomicCAS(status, 0, code);
}

// Grid-wide barrier for cooperative launches, bounded in time.
// state[0] = arrival count, state[1] = generation.  Returns false (after
// raising FRACLAP_ERR_TIMEOUT) when the wait exceeded `limit` cycles or when
// the status word already holds an error.
__device__ __forceinline__ bool grid_barrier(unsigned* state, unsigned nblocks, long long limit,
                                             int32_t* status) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    int ok = 1;
    unsigned gen = ld_acquire_gpu_u(state + 1);
    __threadfence();
    unsigned arrived = atomicAdd(state, 1u);
    if (arrived == nblocks - 1) {
      atomicExch(state, 0u);
      __threadfence();
      atomicAdd(state + 1, 1u);
    } else {
      long long t0 = clock64();
      while (ld_acquire_gpu_u(state + 1) == gen) {
        if (clock64() - t0 > limit) {
          raise_status(status, FRACLAP_ERR_TIMEOUT);
          ok = 0;
          break;
        }
        __nanosleep(64);
      }
    }
    __threadfence();
    if (*(volatile int32_t*)status != 0) ok = 0;
    s_ok = ok;
  }
  __syncthreads();
  return s_ok != 0;
}

}  // namespace fraclap
