// C ABI of the fraclap library: contexts, errors, workspace, and the
// eigendecomposition entry points (the spectral apply is in apply.cu, the
// stencil assembly in assemble.cu).
#include <stdarg.h>

#include <algorithm>

#include "internal.cuh"

namespace fraclap {

int set_error(fraclap_ctx* ctx, int code, const char* fmt, ...) {
  if (ctx) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    ctx->last_error = buf;
  }
  return code;
}

int get_workspace(fraclap_ctx* ctx, void* work, size_t work_bytes, size_t need, Arena* arena) {
  need = align256(need);
  if (work) {
    FL_CHECK(ctx, ((uintptr_t)work & 255) == 0, FRACLAP_ERR_INVALID_ARG,
             "workspace must be 256-byte aligned");
    FL_CHECK(ctx, work_bytes >= need, FRACLAP_ERR_INVALID_ARG,
             "workspace too small: %zu bytes given, %zu needed", work_bytes, need);
    arena->base = (char*)work;
    arena->cap = work_bytes;
    arena->off = 0;
    return 0;
  }
  if (ctx->ws_bytes < need) {
    if (ctx->ws) {
      FL_CUDA(ctx, cudaDeviceSynchronize());
      FL_CUDA(ctx, cudaFree(ctx->ws));
      ctx->ws = nullptr;
      ctx->ws_bytes = 0;
    }
    cudaError_t e = cudaMalloc(&ctx->ws, need);
    if (e != cudaSuccess) {
      cudaGetLastError();
      ctx->ws = nullptr;
      return set_error(ctx, FRACLAP_ERR_ALLOC, "workspace allocation of %zu bytes failed: %s", need,
                       cudaGetErrorString(e));
    }
    ctx->ws_bytes = need;
  }
  arena->base = (char*)ctx->ws;
  arena->cap = ctx->ws_bytes;
  arena->off = 0;
  return 0;
}

namespace {

__global__ void set_identity(double* Z, int64_t ldz, int64_t n) {
  const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= n * n) return;
  const int64_t i = p % n, j = p / n;
  Z[i + j * ldz] = (i == j) ? 1.0 : 0.0;
}

template <class T>
__global__ void copy_lower(const double* A, int64_t lda, T* B, int64_t ldb, int64_t n) {
  const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= n * n) return;
  const int64_t i = p % n, j = p / n;
  if (i >= j) B[i + j * ldb] = (T)A[i + j * lda];
}

__global__ void widen(const float* Z, int64_t n, double* V, int64_t ldv) {
  const int64_t total = n * n;
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < total;
       p += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = p % n, j = p / n;
    V[i + j * ldv] = (double)Z[p];
  }
}

template <class T>
struct EigWork {
  T* Aw;          // n x n working copy (later the transposed eigenvectors)
  T* band;        // 2b x n
  double* d;      // n
  double* e;      // n
  T* W1;          // b x n
  T* W2;          // b x n
  Stage1T<T> s1;
  Stage2T<T> s2;
};

template <class T>
int eig_take(Arena* ar, const fraclap_ctx* ctx, int64_t n, EigWork<T>* w) {
  const int b = ctx->band_width;
  w->Aw = ar->take<T>(n * n);
  w->band = ar->take<T>(2 * (int64_t)b * n);
  w->d = ar->take<double>(n);
  w->e = ar->take<double>(n);
  w->W1 = ar->take<T>((int64_t)b * n);
  w->W2 = ar->take<T>((int64_t)b * n);
  stage1_take<T>(ar, n, b, ctx->sm_count, &w->s1);
  stage2_take<T>(ar, n, b, &w->s2);
  return 0;
}

}  // namespace

size_t eig_ws_bytes(const fraclap_ctx* ctx, int64_t n, bool with_dc) {
  Arena ar;
  EigWork<double> w;
  eig_take<double>(&ar, ctx, n, &w);
  size_t s = ar.off;
  if (with_dc) s += stedc_ws<double>(ctx, n);
  return s + 4096;
}

namespace {

// Split operands of the refinement's FP32 product X E (n x n x n).
size_t tf32_scratch_bytes(int64_t n) { return tf32_split_bytes(n, n, n); }

// Lends the split-operand scratch to gemm<float> for the lifetime of the guard.
struct TcScratch {
  fraclap_ctx* ctx;
  TcScratch(fraclap_ctx* c, void* p, size_t bytes) : ctx(c) {
    ctx->tc_scratch = p;
    ctx->tc_scratch_bytes = p ? bytes : 0;
  }
  ~TcScratch() {
    ctx->tc_scratch = nullptr;
    ctx->tc_scratch_bytes = 0;
  }
};

size_t mixed_ws_bytes(const fraclap_ctx* ctx, int64_t n) {
  Arena ar;
  EigWork<float> w;
  eig_take<float>(&ar, ctx, n, &w);
  ar.take<float>(n * n);  // Z (FP32 eigenvectors)
  ar.take<char>(tf32_scratch_bytes(n));
  return ar.off + stedc_ws<float>(ctx, n) + refine_ws(ctx, n) + 8192;
}

// Reduction of A to tridiagonal form (d, e) in w.
template <class T>
int reduce(fraclap_ctx* ctx, const double* A, int64_t n, int64_t lda, EigWork<T>* w, cudaStream_t st) {
  const int b = ctx->band_width;
  copy_lower<T><<<(unsigned)cdiv(n * n, 256), 256, 0, st>>>(A, lda, w->Aw, n, n);
  count_launch(ctx);
  FL_CUDA(ctx, cudaGetLastError());
  {
    StageTimer t(ctx, kStageBandReduction, st);
    FL_TRY(sy2sb_run<T>(ctx, w->Aw, n, n, b, w->band, &w->s1, st));
  }
  {
    StageTimer t(ctx, kStageBulgeChasing, st);
    FL_TRY(sb2st_run<T>(ctx, w->band, n, b, w->d, w->e, &w->s2, st));
  }
  return 0;
}

template <class T>
int back_transform(fraclap_ctx* ctx, int64_t n, EigWork<T>* w, T* Z, int64_t ldz, cudaStream_t st) {
  const int b = ctx->band_width;
  {
    StageTimer t(ctx, kStageBackQ2, st);
    FL_TRY(q2_apply_run<T>(ctx, &w->s2, n, b, Z, ldz, n, w->Aw, n, st));
  }
  {
    StageTimer t(ctx, kStageBackQ1, st);
    FL_TRY(q1_apply_run<T>(ctx, &w->s1, n, b, Z, ldz, n, w->W1, w->W2, st));
  }
  return 0;
}

}  // namespace

size_t cluster_eig_ws(const fraclap_ctx* ctx, int64_t c) { return eig_ws_bytes(ctx, c, true); }

int cluster_eig(fraclap_ctx* ctx, double* S, int64_t c, double* w, double* Q, Arena* ar,
                cudaStream_t st) {
  // the band width and SM count of the caller's context; sized like cluster_eig_ws
  EigWork<double> ew;
  eig_take<double>(ar, ctx, c, &ew);
  FL_CHECK(ctx, ew.s2.progress != nullptr, FRACLAP_ERR_ALLOC, "cluster eig: workspace too small");
  FL_TRY(reduce<double>(ctx, S, c, c, &ew, st));
  FL_TRY(stedc_run<double>(ctx, ew.d, ew.e, c, w, Q, c, ar, st));
  FL_TRY(back_transform<double>(ctx, c, &ew, Q, c, st));
  return 0;
}

}  // namespace fraclap

using namespace fraclap;

extern "C" const char* fraclap_strerror(int code) {
  switch (code) {
    case FRACLAP_OK: return "ok";
    case FRACLAP_ERR_INVALID_ARG: return "invalid argument";
    case FRACLAP_ERR_NOT_SPD: return "eigenvalue <= 0 with alpha != 0";
    case FRACLAP_ERR_NO_CONVERGENCE: return "eigen-iteration did not converge";
    case FRACLAP_ERR_TIMEOUT: return "device-side wait timed out";
    case FRACLAP_ERR_ALLOC: return "workspace allocation failed";
    case FRACLAP_ERR_CUDA: return "CUDA runtime error";
    case FRACLAP_ERR_UNSUPPORTED: return "unsupported size or option";
    case FRACLAP_ERR_IO: return "file I/O error or invalid checkpoint";
    default: return "unknown error";
  }
}

extern "C" const char* fraclap_last_error(const fraclap_ctx* ctx) {
  return ctx ? ctx->last_error.c_str() : "null context";
}

extern "C" int fraclap_create(fraclap_ctx** out, const fraclap_opts* opts) {
  if (!out) return FRACLAP_ERR_INVALID_ARG;
  *out = nullptr;
  fraclap_ctx* ctx = new fraclap_ctx();
  if (opts) {
    if (opts->band_width) ctx->band_width = opts->band_width;
    if (opts->leaf_size) ctx->leaf_size = opts->leaf_size;
    if (opts->wait_timeout_s > 0) ctx->wait_timeout_s = opts->wait_timeout_s;
  }
  const int bw = ctx->band_width;
  if ((bw != 4 && bw != 8 && bw != 16 && bw != 32 && bw != 64) || ctx->leaf_size < 2 ||
      ctx->leaf_size > 32) {
    delete ctx;
    return FRACLAP_ERR_INVALID_ARG;
  }
  // the wait limit is counted in SM clock cycles; 2.5 GHz bounds every clock
  ctx->wait_cycles = (long long)(ctx->wait_timeout_s * 2.5e9);
  cudaError_t e = cudaGetDevice(&ctx->device);
  if (e == cudaSuccess)
    e = cudaDeviceGetAttribute(&ctx->sm_count, cudaDevAttrMultiProcessorCount, ctx->device);
  if (e == cudaSuccess) e = cudaMalloc(&ctx->d_status, 4 * sizeof(int32_t));
  if (e == cudaSuccess) e = cudaMalloc(&ctx->d_barrier, 4 * sizeof(unsigned));
  if (e == cudaSuccess) e = cudaMemset(ctx->d_status, 0, 4 * sizeof(int32_t));
  if (e == cudaSuccess) e = cudaMemset(ctx->d_barrier, 0, 4 * sizeof(unsigned));
  if (e != cudaSuccess) {
    cudaGetLastError();
    if (ctx->d_status) cudaFree(ctx->d_status);
    if (ctx->d_barrier) cudaFree(ctx->d_barrier);
    delete ctx;
    return FRACLAP_ERR_CUDA;
  }
  *out = ctx;
  return 0;
}

extern "C" void fraclap_destroy(fraclap_ctx* ctx) {
  if (!ctx) return;
  cudaDeviceSynchronize();
  for (fraclap_ctx* w : ctx->workers) fraclap_destroy(w);
  for (cudaStream_t s : ctx->worker_streams) cudaStreamDestroy(s);
  for (cudaEvent_t e : ctx->worker_events) cudaEventDestroy(e);
  if (ctx->batch_start) cudaEventDestroy(ctx->batch_start);
  if (ctx->ws) cudaFree(ctx->ws);
  if (ctx->d_status) cudaFree(ctx->d_status);
  if (ctx->d_barrier) cudaFree(ctx->d_barrier);
  delete ctx;
}

extern "C" int fraclap_sync(fraclap_ctx* ctx, fraclap_stream_t stream) {
  if (!ctx) return FRACLAP_ERR_INVALID_ARG;
  FL_CUDA(ctx, cudaStreamSynchronize((cudaStream_t)stream));
  int32_t st = 0;
  FL_CUDA(ctx, cudaMemcpy(&st, ctx->d_status, sizeof(st), cudaMemcpyDeviceToHost));
  if (st != 0) {
    FL_CUDA(ctx, cudaMemset(ctx->d_status, 0, sizeof(int32_t)));
    return set_error(ctx, st, "device reported: %s", fraclap_strerror(st));
  }
  return 0;
}

extern "C" size_t fraclap_eig_workspace_bytes(const fraclap_ctx* ctx, int64_t n) {
  if (!ctx || n <= 0) return 0;
  return eig_ws_bytes(ctx, n, true);
}

extern "C" size_t fraclap_tridiag_workspace_bytes(const fraclap_ctx* ctx, int64_t n) {
  if (!ctx || n <= 0) return 0;
  return stedc_ws<double>(ctx, n) + 4096;
}

extern "C" int eig_full(fraclap_ctx* ctx, const double* A_dev, int64_t n, int64_t lda,
                        double* lambda_dev, double* V_dev, int64_t ldv, void* work_dev,
                        size_t work_bytes, int32_t* info_dev, fraclap_stream_t stream) {
  if (!ctx) return FRACLAP_ERR_INVALID_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  FL_CHECK(ctx, n >= 0, FRACLAP_ERR_INVALID_ARG, "eig_full: n < 0");
  if (n == 0) return 0;
  FL_CHECK(ctx, A_dev && lambda_dev && V_dev, FRACLAP_ERR_INVALID_ARG, "eig_full: null pointer");
  FL_CHECK(ctx, lda >= n && ldv >= n, FRACLAP_ERR_INVALID_ARG, "eig_full: leading dimension < n");
  FL_CHECK(ctx, n < (1LL << 31) / 64, FRACLAP_ERR_UNSUPPORTED, "eig_full: n too large");
  Arena ar;
  FL_TRY(get_workspace(ctx, work_dev, work_bytes, eig_ws_bytes(ctx, n, true), &ar));
  EigWork<double> w;
  eig_take<double>(&ar, ctx, n, &w);
  FL_CHECK(ctx, w.s2.progress != nullptr, FRACLAP_ERR_ALLOC, "eig_full: workspace too small");
  FL_TRY(reduce<double>(ctx, A_dev, n, lda, &w, st));
  {
    StageTimer t(ctx, kStageTridiagDC, st);
    FL_TRY(stedc_run<double>(ctx, w.d, w.e, n, lambda_dev, V_dev, ldv, &ar, st));
  }
  FL_TRY(back_transform<double>(ctx, n, &w, V_dev, ldv, st));
  if (info_dev) FL_CUDA(ctx, cudaMemcpyAsync(info_dev, ctx->d_status, sizeof(int32_t), cudaMemcpyDeviceToDevice, st));
  return 0;
}

extern "C" int fraclap_tridiagonalize(fraclap_ctx* ctx, const double* A_dev, int64_t n,
                                      int64_t lda, double* d_dev, double* e_dev, double* Q_dev,
                                      int64_t ldq, void* work_dev, size_t work_bytes,
                                      fraclap_stream_t stream) {
  if (!ctx) return FRACLAP_ERR_INVALID_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  FL_CHECK(ctx, n >= 0, FRACLAP_ERR_INVALID_ARG, "tridiagonalize: n < 0");
  if (n == 0) return 0;
  FL_CHECK(ctx, A_dev && d_dev && (e_dev || n == 1), FRACLAP_ERR_INVALID_ARG, "tridiagonalize: null pointer");
  FL_CHECK(ctx, lda >= n && (!Q_dev || ldq >= n), FRACLAP_ERR_INVALID_ARG, "tridiagonalize: leading dimension < n");
  Arena ar;
  FL_TRY(get_workspace(ctx, work_dev, work_bytes, eig_ws_bytes(ctx, n, false), &ar));
  EigWork<double> w;
  eig_take<double>(&ar, ctx, n, &w);
  FL_CHECK(ctx, w.s2.progress != nullptr, FRACLAP_ERR_ALLOC, "tridiagonalize: workspace too small");
  FL_TRY(reduce<double>(ctx, A_dev, n, lda, &w, st));
  FL_CUDA(ctx, cudaMemcpyAsync(d_dev, w.d, sizeof(double) * n, cudaMemcpyDeviceToDevice, st));
  if (n > 1) FL_CUDA(ctx, cudaMemcpyAsync(e_dev, w.e, sizeof(double) * (n - 1), cudaMemcpyDeviceToDevice, st));
  if (Q_dev) {
    set_identity<<<(unsigned)cdiv(n * n, 256), 256, 0, st>>>(Q_dev, ldq, n);
    count_launch(ctx);
    FL_CUDA(ctx, cudaGetLastError());
    FL_TRY(back_transform<double>(ctx, n, &w, Q_dev, ldq, st));
  }
  return 0;
}

extern "C" int fraclap_tridiag_eig(fraclap_ctx* ctx, const double* d_dev, const double* e_dev,
                                   int64_t n, double* lambda_dev, double* Z_dev, int64_t ldz,
                                   void* work_dev, size_t work_bytes, fraclap_stream_t stream) {
  if (!ctx) return FRACLAP_ERR_INVALID_ARG;
  FL_CHECK(ctx, n >= 0, FRACLAP_ERR_INVALID_ARG, "tridiag_eig: n < 0");
  if (n == 0) return 0;
  FL_CHECK(ctx, d_dev && lambda_dev && Z_dev && (e_dev || n == 1), FRACLAP_ERR_INVALID_ARG,
           "tridiag_eig: null pointer");
  FL_CHECK(ctx, ldz >= n, FRACLAP_ERR_INVALID_ARG, "tridiag_eig: ldz < n");
  Arena ar;
  FL_TRY(get_workspace(ctx, work_dev, work_bytes, stedc_ws<double>(ctx, n) + 4096, &ar));
  StageTimer t(ctx, kStageTridiagDC, (cudaStream_t)stream);
  return stedc_run<double>(ctx, d_dev, e_dev, n, lambda_dev, Z_dev, ldz, &ar, (cudaStream_t)stream);
}

extern "C" int fraclap_dgemm(fraclap_ctx* ctx, int trans_a, int trans_b, int64_t m, int64_t n,
                             int64_t k, double alpha, const double* A_dev, int64_t lda,
                             const double* B_dev, int64_t ldb, double beta, double* C_dev,
                             int64_t ldc, fraclap_stream_t stream) {
  if (!ctx) return FRACLAP_ERR_INVALID_ARG;
  FL_CHECK(ctx, m >= 0 && n >= 0 && k >= 0, FRACLAP_ERR_INVALID_ARG, "dgemm: negative size");
  if (m == 0 || n == 0) return 0;
  FL_CHECK(ctx, C_dev && (k == 0 || (A_dev && B_dev)), FRACLAP_ERR_INVALID_ARG, "dgemm: null pointer");
  FL_CHECK(ctx, ldc >= m && lda >= (trans_a ? k : m) && ldb >= (trans_b ? n : k),
           FRACLAP_ERR_INVALID_ARG, "dgemm: leading dimension too small");
  GemmDesc d{m, n, k, A_dev, lda, B_dev, ldb, C_dev, ldc, nullptr, 0, nullptr, 0, 0, alpha, beta};
  return gemm(ctx, trans_a != 0, trans_b != 0, kGemmPlain, d, 1, (cudaStream_t)stream);
}

extern "C" size_t fraclap_sgemm_workspace_bytes(int64_t m, int64_t n, int64_t k) {
  if (m < 0 || n < 0 || k < 0) return 0;
  return tf32_split_bytes(m, n, k) + 256;
}

extern "C" int fraclap_sgemm(fraclap_ctx* ctx, int trans_a, int trans_b, int form, int64_t m, int64_t n,
                             int64_t k, float alpha, const float* A_dev, int64_t lda, const float* B_dev,
                             int64_t ldb, float beta, float* C_dev, int64_t ldc, int route, void* work_dev,
                             size_t work_bytes, fraclap_stream_t stream) {
  if (!ctx) return FRACLAP_ERR_INVALID_ARG;
  FL_CHECK(ctx, m >= 0 && n >= 0 && k >= 0, FRACLAP_ERR_INVALID_ARG, "sgemm: negative size");
  FL_CHECK(ctx, form >= 0 && form <= 2 && (route == 0 || route == 1), FRACLAP_ERR_INVALID_ARG,
           "sgemm: form must be 0..2 and route 0 or 1");
  FL_CHECK(ctx, form != 1 || (!trans_a && m == k), FRACLAP_ERR_INVALID_ARG,
           "sgemm: a symmetric A must be square and untransposed");
  if (m == 0 || n == 0) return 0;
  FL_CHECK(ctx, C_dev && (k == 0 || (A_dev && B_dev)), FRACLAP_ERR_INVALID_ARG, "sgemm: null pointer");
  FL_CHECK(ctx, ldc >= m && lda >= (trans_a ? k : m) && ldb >= (trans_b ? n : k),
           FRACLAP_ERR_INVALID_ARG, "sgemm: leading dimension too small");
  const GemmMode mode = form == 1 ? kGemmSymA : (form == 2 ? kGemmLowerC : kGemmPlain);
  GemmDescT<float> d{m, n, k, A_dev, lda, B_dev, ldb, C_dev, ldc, nullptr, 0, nullptr, 0, 0, alpha, beta};
  if (route == 0) return gemm<float>(ctx, trans_a != 0, trans_b != 0, mode, d, 1, (cudaStream_t)stream);
  Arena ar;
  FL_TRY(get_workspace(ctx, work_dev, work_bytes, tf32_split_bytes(m, n, k), &ar));
  TcScratch lend(ctx, ar.base, ar.cap);
  return gemm<float>(ctx, trans_a != 0, trans_b != 0, mode, d, 1, (cudaStream_t)stream);
}

extern "C" int fraclap_set_profiling(fraclap_ctx* ctx, int enable) {
  if (!ctx) return FRACLAP_ERR_INVALID_ARG;
  ctx->profiling = enable != 0;
  return 0;
}

extern "C" int fraclap_stage_times(fraclap_ctx* ctx, double* ms_out, int64_t* count_out, int nstages) {
  if (!ctx || nstages < 0 || (nstages > 0 && !ms_out)) return FRACLAP_ERR_INVALID_ARG;
  for (int i = 0; i < nstages; ++i) {
    ms_out[i] = 0.0;
    if (count_out) count_out[i] = 0;
  }
  int rc = 0;
  for (auto& ev : ctx->stage_events) {
    float ms = 0.0f;
    cudaError_t e = cudaEventSynchronize(ev.stop);
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, ev.start, ev.stop);
    if (e != cudaSuccess && rc == 0)
      rc = set_error(ctx, FRACLAP_ERR_CUDA, "stage timing: %s", cudaGetErrorString(e));
    if (ev.stage >= 0 && ev.stage < nstages) {
      ms_out[ev.stage] += ms;
      if (count_out) count_out[ev.stage] += 1;
    }
    cudaEventDestroy(ev.start);
    cudaEventDestroy(ev.stop);
  }
  ctx->stage_events.clear();
  return rc;
}

extern "C" long long fraclap_launch_count(const fraclap_ctx* ctx) { return ctx ? ctx->launches : -1; }

extern "C" size_t fraclap_eig_mixed_workspace_bytes(const fraclap_ctx* ctx, int64_t n) {
  if (!ctx || n <= 0) return 0;
  return mixed_ws_bytes(ctx, n);
}

extern "C" int eig_full_mixed(fraclap_ctx* ctx, const double* A_dev, int64_t n, int64_t lda,
                              const int64_t* rowptr_dev, const int32_t* col_dev,
                              const double* val_dev, int refine_iters, double* lambda_dev,
                              double* V_dev, int64_t ldv, void* work_dev, size_t work_bytes,
                              int32_t* info_dev, fraclap_stream_t stream) {
  if (!ctx) return FRACLAP_ERR_INVALID_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  FL_CHECK(ctx, n >= 0, FRACLAP_ERR_INVALID_ARG, "eig_full_mixed: n < 0");
  if (n == 0) return 0;
  FL_CHECK(ctx, A_dev && rowptr_dev && col_dev && val_dev && lambda_dev && V_dev,
           FRACLAP_ERR_INVALID_ARG, "eig_full_mixed: null pointer");
  FL_CHECK(ctx, lda >= n && ldv >= n, FRACLAP_ERR_INVALID_ARG, "eig_full_mixed: leading dimension < n");
  FL_CHECK(ctx, refine_iters >= 0 && refine_iters <= 8, FRACLAP_ERR_INVALID_ARG,
           "eig_full_mixed: refine_iters must be 0..8");
  FL_CHECK(ctx, n <= 65535, FRACLAP_ERR_UNSUPPORTED, "eig_full_mixed: n > 65535");
  Arena ar;
  FL_TRY(get_workspace(ctx, work_dev, work_bytes, mixed_ws_bytes(ctx, n), &ar));
  EigWork<float> w;
  eig_take<float>(&ar, ctx, n, &w);
  float* Z = ar.take<float>(n * n);
  char* tcs = ar.take<char>(tf32_scratch_bytes(n));
  FL_CHECK(ctx, Z != nullptr && tcs != nullptr, FRACLAP_ERR_ALLOC, "eig_full_mixed: workspace too small");
  {
    // FP32 products of the band reduction on the tensor cores (three TF32
    // products) when the context's schedule asks for it, else the FMA kernel
    TcScratch lend(ctx, ctx->fp32_stages_tc ? tcs : nullptr, tf32_scratch_bytes(n));
    FL_TRY(reduce<float>(ctx, A_dev, n, lda, &w, st));
  }
  {
    StageTimer t(ctx, kStageTridiagDC, st);
    FL_TRY(stedc_run<float>(ctx, w.d, w.e, n, lambda_dev, Z, n, &ar, st));
  }
  {
    TcScratch lend(ctx, ctx->fp32_stages_tc ? tcs : nullptr, tf32_scratch_bytes(n));
    FL_TRY(back_transform<float>(ctx, n, &w, Z, n, st));
  }
  {
    StageTimer t(ctx, kStageRefine, st);
    widen<<<(unsigned)std::min<int64_t>(cdiv(n * n, 256), 152 * 16), 256, 0, st>>>(Z, n, V_dev, ldv);
    count_launch(ctx);
    FL_CUDA(ctx, cudaGetLastError());
    // The refinement's FP32 product X E runs on the tensor cores (three TF32
    // products; its error is removed by the next iteration).
    TcScratch lend(ctx, tcs, tf32_scratch_bytes(n));
    Arena rar = ar;  // the refinement reuses everything after the FP32 stages
    FL_TRY(refine_run(ctx, n, rowptr_dev, col_dev, val_dev, V_dev, ldv, lambda_dev, refine_iters, &rar, st));
  }
  if (info_dev) FL_CUDA(ctx, cudaMemcpyAsync(info_dev, ctx->d_status, sizeof(int32_t), cudaMemcpyDeviceToDevice, st));
  return 0;
}

extern "C" int fraclap_refine_stats(const fraclap_ctx* ctx, double* out, int max_values) {
  if (!ctx || max_values < 0 || (max_values > 0 && !out)) return FRACLAP_ERR_INVALID_ARG;
  const int nv = (int)ctx->refine_stats.size();
  for (int i = 0; i < nv && i < max_values; ++i) out[i] = ctx->refine_stats[i];
  return nv;
}

extern "C" int fraclap_set_tensor_route(fraclap_ctx* ctx, int route) {
  if (!ctx || (route != 0 && route != 1)) return FRACLAP_ERR_INVALID_ARG;
  ctx->tensor_route = route;
  return 0;
}

extern "C" int fraclap_set_refine_tau(fraclap_ctx* ctx, double tau) {
  if (!ctx || !(tau > 0.0) || tau > 1.0) return FRACLAP_ERR_INVALID_ARG;
  ctx->refine_tau = tau;
  return 0;
}
