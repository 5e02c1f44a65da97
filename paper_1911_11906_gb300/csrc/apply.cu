// frac_apply: u_j = V diag(lambda^{-alpha_j/2}) V^T f_{pair_f[j]}
// (Sec. II, eq. poisson_solution; the sum v after eq. discrete_laplace).
// frac_diffusion: u_j = V diag(exp(-mu lambda^{alpha_j/2} t_j)) V^T u0_{pair_f[j]}
// (Sec. II, eq. diffusion_solution).
//
// Two GEMMs (W = V^T F over the m distinct forcings or initial states, then
// U = V C) around an elementwise kernel that forms the spectral coefficients
// C(i, j) = g_j(lambda_i) W(i, pair_f[j]) with g_j the pair's multiplier;
// powers are exp(e log lambda) with CUDA's double-precision log() and exp().  The GEMMs run on
// the FP64 engine, or (context setting apply_slices = s > 0) as products of
// s BF16 slices on the tensor cores, accurate to about 2^-8s relative to
// |row max| |column max| per term (s = 7: FP64 level).  A zero or negative
// eigenvalue met with alpha != 0 raises FRACLAP_ERR_NOT_SPD in the device
// status.
#include <cmath>

#include "internal.cuh"

namespace fraclap {
namespace {

// pair_t == nullptr: the Poisson multiplier lambda^{-alpha/2}; otherwise the
// diffusion multiplier exp(-mu lambda^{alpha/2} t_j).  Each thread takes one
// eigenvalue and kScalePairs pairs: log(lambda_i) is formed once and every
// power is exp(e log lambda_i), one exp per coefficient instead of a pow
// (relative error about |e log lambda| 2^-53 more than pow's, below 2e-15
// for the spectra of these grids).
constexpr int kScalePairs = 8;

__global__ void spectral_scale(const double* lambda, int64_t n, const double* W, int64_t ldw,
                               const int32_t* pair_f, const double* pair_alpha, const double* pair_t,
                               double mu, int64_t k, int64_t m, double* C, int64_t ldc, int32_t* status) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double lam = lambda[i];
  const double L = log(lam);  // used only when lam > 0
  const int64_t j0 = (int64_t)blockIdx.y * kScalePairs;
  const int64_t j1 = (j0 + kScalePairs < k) ? j0 + kScalePairs : k;
  for (int64_t j = j0; j < j1; ++j) {
    const double alpha = pair_alpha[j];
    const int32_t f = pair_f[j];
    if (f < 0 || f >= m) {
      raise_status(status, FRACLAP_ERR_INVALID_ARG);
      C[i + j * ldc] = 0.0;
      continue;
    }
    double p = 1.0;  // lambda^{-alpha/2} (Poisson) or lambda^{alpha/2} (diffusion rate)
    if (alpha != 0.0) {
      if (!(lam > 0.0)) raise_status(status, FRACLAP_ERR_NOT_SPD);
      p = exp((pair_t ? 0.5 : -0.5) * alpha * L);
    }
    const double mult = pair_t ? exp(-mu * p * pair_t[j]) : p;
    C[i + j * ldc] = mult * W[i + (int64_t)f * ldw];
  }
}

// The body shared by frac_apply and frac_diffusion.
int spectral_apply(fraclap_ctx* ctx, const char* name, const double* V_dev, int64_t ldv,
                   const double* lambda_dev, int64_t n, const double* F_dev, int64_t ldf, int64_t m,
                   const int32_t* pair_f_dev, const double* pair_alpha_dev, const double* pair_t_dev,
                   double mu, int64_t k, double* U_dev, int64_t ldu, void* work_dev, size_t work_bytes,
                   cudaStream_t st) {
  FL_CHECK(ctx, n >= 0 && m >= 0 && k >= 0, FRACLAP_ERR_INVALID_ARG, "%s: negative size", name);
  if (n == 0 || k == 0) return 0;
  FL_CHECK(ctx, m >= 1, FRACLAP_ERR_INVALID_ARG, "%s: pairs need at least one input column", name);
  FL_CHECK(ctx, V_dev && lambda_dev && F_dev && pair_f_dev && pair_alpha_dev && U_dev,
           FRACLAP_ERR_INVALID_ARG, "%s: null pointer", name);
  FL_CHECK(ctx, ldv >= n && ldf >= n && ldu >= n, FRACLAP_ERR_INVALID_ARG, "%s: leading dimension < n", name);
  FL_CHECK(ctx, k <= 65535 && m <= 65535 * 64, FRACLAP_ERR_UNSUPPORTED, "%s: at most 65535 pairs per call", name);
  StageTimer timer(ctx, kStageApply, st);
  Arena ar;
  FL_TRY(get_workspace(ctx, work_dev, work_bytes, fraclap_apply_workspace_bytes_ctx(ctx, n, m, k), &ar));
  double* W = ar.take<double>(n * m);
  double* C = ar.take<double>(n * k);
  FL_CHECK(ctx, W && C, FRACLAP_ERR_ALLOC, "%s: workspace too small", name);
  const int ozs = ctx->apply_slices;
  // W = V^T F
  if (ozs > 0) {
    Arena oz = ar;
    FL_TRY(ozaki_gemm(ctx, true, false, n, m, n, 1.0, V_dev, ldv, F_dev, ldf, 0.0, W, n, ozs, false, &oz, st));
  } else {
    GemmDesc d{n, m, n, V_dev, ldv, F_dev, ldf, W, n, nullptr, 0, nullptr, 0, 0, 1.0, 0.0};
    FL_TRY(gemm(ctx, true, false, kGemmPlain, d, 1, st));
  }
  spectral_scale<<<dim3((unsigned)cdiv(n, 256), (unsigned)cdiv(k, kScalePairs)), 256, 0, st>>>(
      lambda_dev, n, W, n, pair_f_dev, pair_alpha_dev, pair_t_dev, mu, k, m, C, n, ctx->d_status);
  count_launch(ctx);
  FL_CUDA(ctx, cudaGetLastError());
  // U = V C
  if (ozs > 0) {
    Arena oz = ar;
    FL_TRY(ozaki_gemm(ctx, false, false, n, k, n, 1.0, V_dev, ldv, C, n, 0.0, U_dev, ldu, ozs, false, &oz, st));
  } else {
    GemmDesc d{n, k, n, V_dev, ldv, C, n, U_dev, ldu, nullptr, 0, nullptr, 0, 0, 1.0, 0.0};
    FL_TRY(gemm(ctx, false, false, kGemmPlain, d, 1, st));
  }
  return 0;
}

}  // namespace
}  // namespace fraclap

using namespace fraclap;

extern "C" size_t fraclap_apply_workspace_bytes(int64_t n, int64_t m, int64_t k) {
  if (n < 0 || m < 0 || k < 0) return 0;
  return align256(sizeof(double) * (size_t)(n > 0 ? n : 1) * (size_t)(m > 0 ? m : 1)) +
         align256(sizeof(double) * (size_t)(n > 0 ? n : 1) * (size_t)(k > 0 ? k : 1)) + 512;
}

extern "C" size_t fraclap_apply_workspace_bytes_ctx(const fraclap_ctx* ctx, int64_t n, int64_t m, int64_t k) {
  const size_t base = fraclap_apply_workspace_bytes(n, m, k);
  if (!ctx || ctx->apply_slices <= 0 || base == 0) return base;
  const int64_t nn = n > 0 ? n : 1;
  return base + std::max(ozaki_ws(nn, m > 0 ? m : 1, nn, ctx->apply_slices),
                         ozaki_ws(nn, k > 0 ? k : 1, nn, ctx->apply_slices)) + 1024;
}

extern "C" int fraclap_set_apply_slices(fraclap_ctx* ctx, int slices) {
  if (!ctx || slices < 0 || slices > 8) return FRACLAP_ERR_INVALID_ARG;
  ctx->apply_slices = slices;
  return 0;
}

extern "C" int frac_apply(fraclap_ctx* ctx, const double* V_dev, int64_t ldv,
                          const double* lambda_dev, int64_t n, const double* F_dev, int64_t ldf,
                          int64_t m, const int32_t* pair_f_dev, const double* pair_alpha_dev,
                          int64_t k, double* U_dev, int64_t ldu, void* work_dev, size_t work_bytes,
                          fraclap_stream_t stream) {
  if (!ctx) return FRACLAP_ERR_INVALID_ARG;
  return spectral_apply(ctx, "frac_apply", V_dev, ldv, lambda_dev, n, F_dev, ldf, m, pair_f_dev,
                        pair_alpha_dev, nullptr, 0.0, k, U_dev, ldu, work_dev, work_bytes,
                        (cudaStream_t)stream);
}

extern "C" int frac_diffusion(fraclap_ctx* ctx, const double* V_dev, int64_t ldv,
                              const double* lambda_dev, int64_t n, const double* U0_dev, int64_t ldu0,
                              int64_t m, const int32_t* pair_f_dev, const double* pair_alpha_dev,
                              const double* pair_t_dev, double mu, int64_t k, double* U_dev,
                              int64_t ldu, void* work_dev, size_t work_bytes, fraclap_stream_t stream) {
  if (!ctx) return FRACLAP_ERR_INVALID_ARG;
  FL_CHECK(ctx, k == 0 || n == 0 || pair_t_dev, FRACLAP_ERR_INVALID_ARG, "frac_diffusion: null pointer");
  FL_CHECK(ctx, std::isfinite(mu), FRACLAP_ERR_INVALID_ARG, "frac_diffusion: mu is not finite");
  return spectral_apply(ctx, "frac_diffusion", V_dev, ldv, lambda_dev, n, U0_dev, ldu0, m, pair_f_dev,
                        pair_alpha_dev, pair_t_dev, mu, k, U_dev, ldu, work_dev, work_bytes,
                        (cudaStream_t)stream);
}

// ----------------------------------------------------------------------------
// frac_apply_noalloc: the same spectral apply for callers that cannot
// allocate device memory.  Its scratch (V^T F and the scaled coefficients)
// lives in a fixed file-scope device array that every device loading this
// library keeps until the process exits.
// ----------------------------------------------------------------------------
#include <mutex>

namespace fraclap {
namespace {

constexpr int64_t kNoAllocDoubles = FRACLAP_NOALLOC_MAX_DOUBLES;
constexpr int kNoAllocMaxDevices = 64;

static __device__ __align__(256) double g_noalloc_scratch[kNoAllocDoubles];
static __device__ __align__(256) int32_t g_noalloc_status[1];

std::mutex g_noalloc_mu;
double* g_noalloc_scratch_ptr[kNoAllocMaxDevices] = {};
int32_t* g_noalloc_status_ptr[kNoAllocMaxDevices] = {};

// Device addresses of the scratch array and the fallback status word on the
// current device, looked up once per device (the symbol names are host-side
// stand-ins and must never be passed to a kernel).
int noalloc_setup(double** scratch, int32_t** status) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess) return FRACLAP_ERR_CUDA;
  if (dev < 0 || dev >= kNoAllocMaxDevices) return FRACLAP_ERR_UNSUPPORTED;
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  if (!g_noalloc_scratch_ptr[dev]) {
    double* p = nullptr;
    int32_t* q = nullptr;
    if (cudaGetSymbolAddress((void**)&p, g_noalloc_scratch) != cudaSuccess || !p) {
      cudaGetLastError();
      return FRACLAP_ERR_CUDA;
    }
    if (cudaGetSymbolAddress((void**)&q, g_noalloc_status) != cudaSuccess || !q) {
      cudaGetLastError();
      return FRACLAP_ERR_CUDA;
    }
    g_noalloc_status_ptr[dev] = q;
    g_noalloc_scratch_ptr[dev] = p;
  }
  *scratch = g_noalloc_scratch_ptr[dev];
  *status = g_noalloc_status_ptr[dev];
  return 0;
}

}  // namespace
}  // namespace fraclap

extern "C" int frac_apply_noalloc(const double* V_dev, int64_t ldv, const double* lambda_dev,
                                  int64_t n, const double* F_dev, int64_t ldf, int64_t m,
                                  const int32_t* pair_f_dev, const double* pair_alpha_dev,
                                  int64_t k, double* U_dev, int64_t ldu, int32_t* status_dev,
                                  fraclap_stream_t stream) {
  if (n < 0 || m < 0 || k < 0) return FRACLAP_ERR_INVALID_ARG;
  if (n == 0 || k == 0) return 0;
  if (m < 1 || !V_dev || !lambda_dev || !F_dev || !pair_f_dev || !pair_alpha_dev || !U_dev)
    return FRACLAP_ERR_INVALID_ARG;
  if (ldv < n || ldf < n || ldu < n) return FRACLAP_ERR_INVALID_ARG;
  // the scratch holds W (n x m) and C (n x k), each starting on a 256-byte
  // boundary; the bounds are checked before any product of sizes is formed
  if (m > kNoAllocDoubles || k > 65535 || n > kNoAllocDoubles / (m + k)) return FRACLAP_ERR_UNSUPPORTED;
  const int64_t wlen = ((n * m + 31) / 32) * 32;
  if (wlen + n * k > kNoAllocDoubles) return FRACLAP_ERR_UNSUPPORTED;
  double* scratch = nullptr;
  int32_t* own_status = nullptr;
  const int rc = noalloc_setup(&scratch, &own_status);
  if (rc != 0) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  int32_t* status = status_dev ? status_dev : own_status;
  double* W = scratch;
  double* C = scratch + wlen;
  fraclap_ctx local;  // host-side bookkeeping only (error text, launch count)
  GemmDesc d{n, m, n, V_dev, ldv, F_dev, ldf, W, n, nullptr, 0, nullptr, 0, 0, 1.0, 0.0};
  int r = gemm(&local, true, false, kGemmPlain, d, 1, st);
  if (r != 0) return r;
  spectral_scale<<<dim3((unsigned)cdiv(n, 256), (unsigned)cdiv(k, kScalePairs)), 256, 0, st>>>(
      lambda_dev, n, W, n, pair_f_dev, pair_alpha_dev, nullptr, 0.0, k, m, C, n, status);
  if (cudaGetLastError() != cudaSuccess) return FRACLAP_ERR_CUDA;
  d = GemmDesc{n, k, n, V_dev, ldv, C, n, U_dev, ldu, nullptr, 0, nullptr, 0, 0, 1.0, 0.0};
  return gemm(&local, false, false, kGemmPlain, d, 1, st);
}

// ----------------------------------------------------------------------------
// The spectral apply captured once into a CUDA graph: every later solve with
// new contents of the same buffers is a single graph launch instead of the
// GEMM, scaling and slicing launches one by one.
// ----------------------------------------------------------------------------
struct fraclap_graph {
  fraclap_ctx* ctx = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  long long kernels = 0;  // kernels in the graph (added to the context's launch count per launch)
};

extern "C" int fraclap_apply_graph_create(fraclap_ctx* ctx, const double* V_dev, int64_t ldv,
                                          const double* lambda_dev, int64_t n, const double* F_dev,
                                          int64_t ldf, int64_t m, const int32_t* pair_f_dev,
                                          const double* pair_alpha_dev, const double* pair_t_dev, double mu,
                                          int64_t k, double* U_dev, int64_t ldu, void* work_dev,
                                          size_t work_bytes, fraclap_graph** out) {
  if (!ctx || !out) return FRACLAP_ERR_INVALID_ARG;
  *out = nullptr;
  FL_CHECK(ctx, work_dev != nullptr, FRACLAP_ERR_INVALID_ARG,
           "apply_graph: a graph needs a caller-owned workspace (the context's may be reallocated)");
  FL_CHECK(ctx, std::isfinite(mu), FRACLAP_ERR_INVALID_ARG, "apply_graph: mu is not finite");
  cudaStream_t s = nullptr;
  FL_CUDA(ctx, cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
  cudaError_t e = cudaStreamBeginCapture(s, cudaStreamCaptureModeRelaxed);
  if (e != cudaSuccess) {
    cudaGetLastError();
    cudaStreamDestroy(s);
    return set_error(ctx, FRACLAP_ERR_CUDA, "apply_graph: begin capture: %s", cudaGetErrorString(e));
  }
  const long long before = ctx->launches;
  // no stage events inside the capture: events recorded there belong to the
  // graph and could not be read back by fraclap_stage_times
  const bool profiling = ctx->profiling;
  ctx->profiling = false;
  const int rc = spectral_apply(ctx, pair_t_dev ? "apply_graph(diffusion)" : "apply_graph", V_dev, ldv,
                                lambda_dev, n, F_dev, ldf, m, pair_f_dev, pair_alpha_dev, pair_t_dev, mu, k,
                                U_dev, ldu, work_dev, work_bytes, s);
  ctx->profiling = profiling;
  cudaGraph_t g = nullptr;
  e = cudaStreamEndCapture(s, &g);
  cudaStreamDestroy(s);
  if (rc != 0 || e != cudaSuccess || !g) {
    if (g) cudaGraphDestroy(g);
    cudaGetLastError();
    ctx->launches = before;
    if (rc != 0) return rc;
    return set_error(ctx, FRACLAP_ERR_CUDA, "apply_graph: end capture: %s", cudaGetErrorString(e));
  }
  cudaGraphExec_t x = nullptr;
  e = cudaGraphInstantiate(&x, g, 0);
  if (e != cudaSuccess) {
    cudaGetLastError();
    cudaGraphDestroy(g);
    ctx->launches = before;
    return set_error(ctx, FRACLAP_ERR_CUDA, "apply_graph: instantiate: %s", cudaGetErrorString(e));
  }
  fraclap_graph* G = new fraclap_graph;
  G->ctx = ctx;
  G->graph = g;
  G->exec = x;
  G->kernels = ctx->launches - before;
  ctx->launches = before;  // counted when launched
  *out = G;
  return 0;
}

extern "C" int fraclap_graph_launch(fraclap_graph* g, fraclap_stream_t stream) {
  if (!g || !g->exec) return FRACLAP_ERR_INVALID_ARG;
  FL_CUDA(g->ctx, cudaGraphLaunch(g->exec, (cudaStream_t)stream));
  g->ctx->launches += g->kernels;
  return 0;
}

extern "C" long long fraclap_graph_kernels(const fraclap_graph* g) { return g ? g->kernels : -1; }

extern "C" void fraclap_graph_destroy(fraclap_graph* g) {
  if (!g) return;
  if (g->exec) cudaGraphExecDestroy(g->exec);
  if (g->graph) cudaGraphDestroy(g->graph);
  delete g;
}
