// Exact eigenvalue counting and spectrum slicing (Sec. III-D): the number of
// eigenvalues below a shift sigma is the number of negative pivots of
// A - sigma I = L D L^T (Sylvester's law of inertia, Sec. III-D-2), or of
// K - sigma M for the generalised problem; the greedy partitioning of
// Sec. III-D ("greedy partitioning") turns such counts into P subintervals
// of [0, rho] holding about n / P eigenvalues each.  For the tridiagonal form
// T = Q^T A Q (congruent to A, so with A's counts) the pivots are the Sturm
// recurrence, and bisection on it gives any index range of eigenvalues
// without the divide and conquer.
//
// Banded LDL^T on the GPU: one CTA per shift.  In the natural dof order the
// Laplacian (and the finite-element pencil) is banded with half-width b (the
// grid row length in 2-D, the plane size in 3-D), and the factorisation
// fills exactly that band.  Step j needs only columns j .. j + b: a window of
// b + 1 band columns, each of b + 1 entries (offsets below the diagonal),
// kept in shared memory when it fits (b <= 167) and in a per-shift global
// ring otherwise; column j + b + 1 enters the slot column j leaves.  The
// operations and their order are those of the plain definition (l = B / d,
// then B(i, k) -= l_i (l_k d) for the trailing triangle), with explicit
// round-to-nearest intrinsics so the compiler fuses nothing: the pivots,
// hence the counts, are the same bits as a sequential factorisation.
#include "internal.cuh"

namespace fraclap {
namespace {

constexpr int SL_NT = 256;
constexpr int kSmemWindowMaxLd = 168;  // (b + 1)^2 doubles + 2 (b + 1) in 227 KB

// Half-bandwidth of the lower triangle: max(i - col) over the entries.
__global__ void csr_bandwidth_kernel(int64_t n, const int64_t* rowptr, const int32_t* col,
                                     unsigned long long* bw) {
  unsigned long long m = 0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    for (int64_t p = rowptr[i]; p < rowptr[i + 1]; ++p) {
      const int64_t c = col[p];
      if (c <= i && (unsigned long long)(i - c) > m) m = (unsigned long long)(i - c);
    }
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long v = __shfl_xor_sync(0xffffffffu, m, o);
    m = v > m ? v : m;
  }
  if ((threadIdx.x & 31) == 0 && m > 0) atomicMax(bw, m);
}

// Lower band of the CSR matrix: Bd[(i - c) + c ld] = 0 + val for c <= i
// (ld = b + 1, zero elsewhere; the caller zeroes Bd).  One thread per row
// (distinct rows write distinct entries).  An entry outside the band sets
// FRACLAP_ERR_INVALID_ARG and is skipped.
__global__ void csr_to_band_kernel(int64_t n, const int64_t* rowptr, const int32_t* col, const double* val,
                                   int b, double* Bd, int32_t* status) {
  const int64_t ld = b + 1;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    for (int64_t p = rowptr[i]; p < rowptr[i + 1]; ++p) {
      const int64_t c = col[p];
      if (c > i) continue;
      if (i - c > b || c < 0) {
        raise_status(status, FRACLAP_ERR_INVALID_ARG);
        continue;
      }
      double* q = Bd + (i - c) + c * ld;
      *q = __dadd_rn(*q, val[p]);
    }
}

// Entry t (row k + t) of band column k of A - sigma I, or of K - sigma M.
__device__ __forceinline__ double band_entry(const double* BK, const double* BM, int64_t ld, int64_t k, int t,
                                             double sg) {
  const double a = BK[t + k * ld];
  if (BM) return __dsub_rn(a, __dmul_rn(sg, BM[t + k * ld]));
  return t == 0 ? __dsub_rn(a, sg) : a;
}

// One CTA per shift: count[s] = negative pivots of LDL^T(A - sigma_s I), or
// -1 when a pivot is exactly zero (sigma_s is then, to rounding, an
// eigenvalue of a leading block and the count is not defined by inertia).
// STORE (one CTA, sigma = 0): the factors themselves, the unit lower band
// Lb(t, j) = L(j + t, j) (ld b + 1), its row-wise copy Lr(t, i) = L(i, i - t)
// and the pivots D; a pivot <= 0 raises FRACLAP_ERR_NOT_SPD in `status`.
template <bool SMEM, bool STORE>
__global__ void __launch_bounds__(SL_NT)
band_inertia_kernel(const double* BK, const double* BM, int64_t n, int b, const double* sigma, int64_t nsig,
                    int64_t* count, double* gwin, double* Lb, double* Lr, double* D, int32_t* status) {
  extern __shared__ __align__(16) double sl_smem[];
  const int64_t s = blockIdx.x;
  if (s >= nsig) return;
  const int ld = b + 1;
  double* W = SMEM ? sl_smem : gwin + (size_t)s * ld * ld;  // slot c holds band column k with k % ld == c
  double* l = SMEM ? sl_smem + (size_t)ld * ld : gwin + (size_t)nsig * ld * ld + (size_t)s * 2 * ld;
  double* lk = l + ld;
  __shared__ int s_zero;
  const double sg = STORE ? 0.0 : sigma[s];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarp = SL_NT / 32;
  for (int64_t p = tid; p < (int64_t)ld * ld; p += SL_NT) {
    const int c = (int)(p / ld), t = (int)(p % ld);
    W[p] = (c < n) ? band_entry(BK, BM, ld, c, t, sg) : 0.0;
  }
  if (tid == 0) s_zero = 0;
  int64_t neg = 0;
  __syncthreads();
  for (int64_t j = 0; j < n; ++j) {
    double* Wj = W + (size_t)(j % ld) * ld;
    const double d = Wj[0];
    const int L = (int)((b < n - 1 - j) ? b : n - 1 - j);
    if (d == 0.0) {
      if (tid == 0) s_zero = 1;
    } else {
      for (int t = 1 + tid; t <= L; t += SL_NT) {
        const double lt = __ddiv_rn(Wj[t], d);
        l[t] = lt;
        lk[t] = __dmul_rn(lt, d);
        if (STORE) {
          Lb[t + j * (int64_t)ld] = lt;
          Lr[t + (j + t) * (int64_t)ld] = lt;
        }
      }
    }
    if (tid == 0) {
      neg += (d < 0.0);
      if (STORE) {
        D[j] = d;
        if (!(d > 0.0)) {
          raise_status(status, FRACLAP_ERR_NOT_SPD);
          s_zero = 1;
        }
      }
    }
    __syncthreads();
    if (s_zero) break;
    // trailing triangle: column j + c, entries t = 0 .. L - c (rows j + c + t)
    for (int c = 1 + warp; c <= L; c += nwarp) {
      double* Wc = W + (size_t)((j + c) % ld) * ld;
      const double f = lk[c];
      for (int t = lane; t <= L - c; t += 32) Wc[t] = __dsub_rn(Wc[t], __dmul_rn(l[c + t], f));
    }
    // the slot of column j takes column j + ld
    if (j + ld < n)
      for (int t = tid; t < ld; t += SL_NT) Wj[t] = band_entry(BK, BM, ld, j + ld, t, sg);
    __syncthreads();
  }
  if (!STORE && tid == 0) count[s] = s_zero ? -1 : neg;
}

// Negative pivots of the Sturm recurrence of T - sigma I:
// q_0 = d_0 - sigma, q_i = (d_i - sigma) - e_{i-1}^2 / q_{i-1}; an exact zero
// pivot becomes -1e-300 (sigma moved up below the resolution of any
// eigenvalue).  Sequential in i; the threads of a warp read the same d_i, e_i.
__device__ __forceinline__ int64_t sturm_count(const double* __restrict__ d, const double* __restrict__ e,
                                               int64_t n, double sg) {
  int64_t neg = 0;
  double q = 0.0;
  for (int64_t i = 0; i < n; ++i) {
    const double ds = __dsub_rn(d[i], sg);
    if (i == 0) {
      q = ds;
    } else {
      const double ee = __dmul_rn(e[i - 1], e[i - 1]);
      q = __dsub_rn(ds, __ddiv_rn(ee, q));
    }
    if (q == 0.0) q = -1e-300;
    neg += (q < 0.0);
  }
  return neg;
}

__global__ void sturm_counts_kernel(const double* d, const double* e, int64_t n, const double* sigma,
                                    int64_t nsig, int64_t* count) {
  const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (s < nsig) count[s] = sturm_count(d, e, n, sigma[s]);
}

// Gershgorin interval of T: lo = min(d_i - r_i), hi = max(d_i + r_i) with
// r_i = |e_{i-1}| + |e_i|; one CTA (min and max are exact in any order).
__global__ void gershgorin_kernel(const double* d, const double* e, int64_t n, double* out) {
  __shared__ double slo[32], shi[32];
  double lo = d[0], hi = d[0];
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
    const double r = __dadd_rn(i > 0 ? fabs(e[i - 1]) : 0.0, i + 1 < n ? fabs(e[i]) : 0.0);
    lo = fmin(lo, __dsub_rn(d[i], r));
    hi = fmax(hi, __dadd_rn(d[i], r));
  }
  for (int o = 16; o > 0; o >>= 1) {
    lo = fmin(lo, __shfl_xor_sync(0xffffffffu, lo, o));
    hi = fmax(hi, __shfl_xor_sync(0xffffffffu, hi, o));
  }
  if ((threadIdx.x & 31) == 0) {
    slo[threadIdx.x >> 5] = lo;
    shi[threadIdx.x >> 5] = hi;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (unsigned w = 1; w < blockDim.x / 32; ++w) {
      lo = fmin(lo, slo[w]);
      hi = fmax(hi, shi[w]);
    }
    const double pad = __dadd_rn(__dmul_rn(2.220446049250313e-16, __dadd_rn(fabs(lo), fabs(hi))), 1e-300);
    out[0] = __dsub_rn(lo, pad);
    out[1] = __dadd_rn(hi, pad);
  }
}

// Eigenvalue k0 + thread of T by bisection on the Sturm count from the
// Gershgorin interval: count(lo) <= k < count(hi) throughout; stops when the
// interval holds no representable midpoint or is within 2 eps of its
// magnitude; the result is the last midpoint of the interval.
__global__ void bisect_kernel(const double* d, const double* e, int64_t n, int64_t k0, int64_t k1,
                              const double* ghl, double* lam) {
  const int64_t k = k0 + (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k > k1) return;
  double lo = ghl[0], hi = ghl[1];
  for (int it = 0; it < 4096; ++it) {
    const double mid = __dmul_rn(0.5, __dadd_rn(lo, hi));
    if (mid <= lo || mid >= hi) break;
    if (__dsub_rn(hi, lo) <= __dmul_rn(2.0 * 2.220446049250313e-16, fmax(fabs(lo), fabs(hi)))) break;
    if (sturm_count(d, e, n, mid) > k) hi = mid;
    else lo = mid;
  }
  lam[k - k0] = __dmul_rn(0.5, __dadd_rn(lo, hi));
}

bool smem_window(int64_t b) { return b + 1 <= kSmemWindowMaxLd; }

struct InertiaWork {
  double* BK;
  double* BM;
  double* gwin;  // global windows (large bandwidths only) + l, lk per shift
};

size_t inertia_ws(int64_t n, int64_t b, int64_t nsig, bool pencil) {
  Arena ar;
  const int64_t ld = b + 1;
  ar.take<double>(n * ld);
  if (pencil) ar.take<double>(n * ld);
  if (!smem_window(b)) ar.take<double>(nsig * (ld * ld + 2 * ld));
  return ar.off;
}

int inertia_take(Arena* ar, int64_t n, int64_t b, int64_t nsig, bool pencil, InertiaWork* w) {
  const int64_t ld = b + 1;
  w->BK = ar->take<double>(n * ld);
  w->BM = pencil ? ar->take<double>(n * ld) : nullptr;
  w->gwin = smem_window(b) ? nullptr : ar->take<double>(nsig * (ld * ld + 2 * ld));
  return 0;
}

// Bands of K (and M) into w (the caller sized it for b).
int build_bands(fraclap_ctx* ctx, int64_t n, const int64_t* rowptr, const int32_t* col, const double* valK,
                const double* valM, int64_t b, const InertiaWork& w, cudaStream_t st) {
  const int64_t ld = b + 1;
  const unsigned g = (unsigned)std::max<int64_t>(1, std::min<int64_t>(cdiv(n, 256), 152 * 8));
  FL_CUDA(ctx, cudaMemsetAsync(w.BK, 0, sizeof(double) * n * ld, st));
  csr_to_band_kernel<<<g, 256, 0, st>>>(n, rowptr, col, valK, (int)b, w.BK, ctx->d_status);
  count_launch(ctx);
  if (valM) {
    FL_CUDA(ctx, cudaMemsetAsync(w.BM, 0, sizeof(double) * n * ld, st));
    csr_to_band_kernel<<<g, 256, 0, st>>>(n, rowptr, col, valM, (int)b, w.BM, ctx->d_status);
    count_launch(ctx);
  }
  FL_CUDA(ctx, cudaGetLastError());
  return 0;
}

int launch_inertia(fraclap_ctx* ctx, int64_t n, int64_t b, const InertiaWork& w, const double* sigma,
                   int64_t nsig, int64_t* count, cudaStream_t st) {
  if (nsig <= 0) return 0;
  FL_CHECK(ctx, nsig <= INT32_MAX, FRACLAP_ERR_UNSUPPORTED, "inertia: too many shifts");
  if (smem_window(b)) {
    const size_t ld = (size_t)b + 1;
    const size_t smem = (ld * ld + 2 * ld) * sizeof(double);
    FL_CUDA(ctx, cudaFuncSetAttribute(band_inertia_kernel<true, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)(kSmemWindowMaxLd * kSmemWindowMaxLd + 2 * kSmemWindowMaxLd) *
                                          (int)sizeof(double)));
    band_inertia_kernel<true, false><<<(unsigned)nsig, SL_NT, smem, st>>>(
        w.BK, w.BM, n, (int)b, sigma, nsig, count, nullptr, nullptr, nullptr, nullptr, nullptr);
  } else {
    band_inertia_kernel<false, false><<<(unsigned)nsig, SL_NT, 0, st>>>(
        w.BK, w.BM, n, (int)b, sigma, nsig, count, w.gwin, nullptr, nullptr, nullptr, nullptr);
  }
  count_launch(ctx);
  FL_CUDA(ctx, cudaGetLastError());
  return 0;
}

int check_csr(fraclap_ctx* ctx, const char* who, int64_t n, const int64_t* rowptr, const int32_t* col,
              const double* valK) {
  FL_CHECK(ctx, n >= 1, FRACLAP_ERR_INVALID_ARG, "%s: n must be positive", who);
  FL_CHECK(ctx, n < INT32_MAX, FRACLAP_ERR_UNSUPPORTED, "%s: n too large", who);
  FL_CHECK(ctx, rowptr && col && valK, FRACLAP_ERR_INVALID_ARG, "%s: null CSR pointer", who);
  return 0;
}

// Counts at the host shifts xs (a few per call of the partitioner), through
// the device buffers sig / cnt of the workspace.  Synchronises `st`.
int counts_at(fraclap_ctx* ctx, int64_t n, int64_t b, const InertiaWork& w, const std::vector<double>& xs,
              double* sig, int64_t* cnt, std::vector<int64_t>* out, cudaStream_t st) {
  out->assign(xs.size(), 0);
  if (xs.empty()) return 0;
  FL_CUDA(ctx, cudaMemcpyAsync(sig, xs.data(), sizeof(double) * xs.size(), cudaMemcpyHostToDevice, st));
  FL_TRY(launch_inertia(ctx, n, b, w, sig, (int64_t)xs.size(), cnt, st));
  FL_CUDA(ctx, cudaMemcpyAsync(out->data(), cnt, sizeof(int64_t) * xs.size(), cudaMemcpyDeviceToHost, st));
  FL_CUDA(ctx, cudaStreamSynchronize(st));
  int32_t status = 0;
  FL_CUDA(ctx, cudaMemcpy(&status, ctx->d_status, sizeof(status), cudaMemcpyDeviceToHost));
  if (status != 0) {
    FL_CUDA(ctx, cudaMemset(ctx->d_status, 0, sizeof(int32_t)));
    return set_error(ctx, status, "partition: device reported %s", fraclap_strerror(status));
  }
  for (size_t i = 0; i < xs.size(); ++i)
    FL_CHECK(ctx, (*out)[i] >= 0, FRACLAP_ERR_NOT_SPD, "partition: zero pivot at the shift %.17g", xs[i]);
  return 0;
}

// New splits for P equal loads under the piecewise-constant density the
// counts describe: the cumulative count is taken as linear between the known
// points, and split j is where it reaches j n / P.
std::vector<double> equal_load_splits(const std::vector<double>& pts, const std::vector<double>& cum, int64_t n,
                                      int P) {
  std::vector<double> out;
  const int64_t L = (int64_t)pts.size();
  for (int j = 1; j < P; ++j) {
    const double target = (double)((int64_t)j * n) / (double)P;
    int64_t i = std::lower_bound(cum.begin(), cum.end(), target) - cum.begin();  // first cum >= target
    i = std::min<int64_t>(std::max<int64_t>(i, 1), L - 1);
    const double c0 = cum[i - 1], c1 = cum[i], x0 = pts[i - 1], x1 = pts[i];
    out.push_back(c1 == c0 ? x0 : x0 + (target - c0) / (c1 - c0) * (x1 - x0));
  }
  return out;
}

}  // namespace

size_t band_ldlt_ws(int64_t n, int64_t b) { return inertia_ws(n, b, 1, false); }

int band_ldlt(fraclap_ctx* ctx, int64_t n, const int64_t* rowptr, const int32_t* col, const double* val, int64_t b,
              double* Lb, double* Lr, double* D, Arena* ar, cudaStream_t st) {
  InertiaWork w;
  inertia_take(ar, n, b, 1, false, &w);
  FL_CHECK(ctx, w.BK && (smem_window(b) || w.gwin), FRACLAP_ERR_ALLOC, "band_ldlt: workspace too small");
  FL_TRY(build_bands(ctx, n, rowptr, col, val, nullptr, b, w, st));
  const int64_t ld = b + 1;
  FL_CUDA(ctx, cudaMemsetAsync(Lb, 0, sizeof(double) * n * ld, st));
  FL_CUDA(ctx, cudaMemsetAsync(Lr, 0, sizeof(double) * n * ld, st));
  if (smem_window(b)) {
    const size_t smem = ((size_t)ld * ld + 2 * ld) * sizeof(double);
    FL_CUDA(ctx, cudaFuncSetAttribute(band_inertia_kernel<true, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)(kSmemWindowMaxLd * kSmemWindowMaxLd + 2 * kSmemWindowMaxLd) *
                                          (int)sizeof(double)));
    band_inertia_kernel<true, true><<<1, SL_NT, smem, st>>>(w.BK, nullptr, n, (int)b, nullptr, 1, nullptr, nullptr,
                                                            Lb, Lr, D, ctx->d_status);
  } else {
    band_inertia_kernel<false, true><<<1, SL_NT, 0, st>>>(w.BK, nullptr, n, (int)b, nullptr, 1, nullptr, w.gwin, Lb,
                                                          Lr, D, ctx->d_status);
  }
  count_launch(ctx);
  FL_CUDA(ctx, cudaGetLastError());
  return 0;
}

int csr_half_bandwidth(fraclap_ctx* ctx, int64_t n, const int64_t* rowptr, const int32_t* col, int64_t* bw,
                       cudaStream_t st) {
  return fraclap_csr_half_bandwidth(ctx, n, rowptr, col, bw, (fraclap_stream_t)st);
}

}  // namespace fraclap

using namespace fraclap;

extern "C" int fraclap_csr_half_bandwidth(fraclap_ctx* ctx, int64_t n, const int64_t* rowptr_dev,
                                          const int32_t* col_dev, int64_t* bw_out, fraclap_stream_t stream) {
  if (!ctx || !bw_out) return FRACLAP_ERR_INVALID_ARG;
  *bw_out = 0;
  FL_CHECK(ctx, n >= 0, FRACLAP_ERR_INVALID_ARG, "csr_half_bandwidth: n < 0");
  if (n == 0) return 0;
  FL_CHECK(ctx, rowptr_dev && col_dev, FRACLAP_ERR_INVALID_ARG, "csr_half_bandwidth: null pointer");
  cudaStream_t st = (cudaStream_t)stream;
  Arena ar;
  FL_TRY(get_workspace(ctx, nullptr, 0, 256, &ar));
  unsigned long long* bw = ar.take<unsigned long long>(1);
  FL_CUDA(ctx, cudaMemsetAsync(bw, 0, sizeof(unsigned long long), st));
  csr_bandwidth_kernel<<<(unsigned)std::min<int64_t>(cdiv(n, 256), 152 * 8), 256, 0, st>>>(n, rowptr_dev, col_dev,
                                                                                           bw);
  count_launch(ctx);
  FL_CUDA(ctx, cudaGetLastError());
  unsigned long long h = 0;
  FL_CUDA(ctx, cudaMemcpyAsync(&h, bw, sizeof(h), cudaMemcpyDeviceToHost, st));
  FL_CUDA(ctx, cudaStreamSynchronize(st));
  *bw_out = (int64_t)h;
  return 0;
}

extern "C" size_t fraclap_inertia_workspace_bytes(int64_t n, int64_t half_bandwidth, int64_t nsig, int pencil) {
  if (n < 0 || half_bandwidth < 0 || nsig < 0) return 0;
  return inertia_ws(std::max<int64_t>(n, 1), half_bandwidth, std::max<int64_t>(nsig, 1), pencil != 0) + 1024;
}

extern "C" int fraclap_inertia_counts(fraclap_ctx* ctx, int64_t n, const int64_t* rowptr_dev, const int32_t* col_dev,
                                      const double* valK_dev, const double* valM_dev, int64_t half_bandwidth,
                                      const double* sigma_dev, int64_t nsig, int64_t* count_dev, void* work_dev,
                                      size_t work_bytes, fraclap_stream_t stream) {
  if (!ctx) return FRACLAP_ERR_INVALID_ARG;
  FL_TRY(check_csr(ctx, "inertia_counts", n, rowptr_dev, col_dev, valK_dev));
  FL_CHECK(ctx, nsig >= 0 && half_bandwidth >= 0 && half_bandwidth < n + 1, FRACLAP_ERR_INVALID_ARG,
           "inertia_counts: bad shift count or bandwidth");
  if (nsig == 0) return 0;
  FL_CHECK(ctx, sigma_dev && count_dev, FRACLAP_ERR_INVALID_ARG, "inertia_counts: null shift/count pointer");
  cudaStream_t st = (cudaStream_t)stream;
  const int64_t b = std::min<int64_t>(half_bandwidth, n - 1);
  Arena ar;
  FL_TRY(get_workspace(ctx, work_dev, work_bytes, inertia_ws(n, b, nsig, valM_dev != nullptr), &ar));
  InertiaWork w;
  inertia_take(&ar, n, b, nsig, valM_dev != nullptr, &w);
  FL_CHECK(ctx, w.BK && (!valM_dev || w.BM) && (smem_window(b) || w.gwin), FRACLAP_ERR_ALLOC,
           "inertia_counts: workspace too small");
  FL_TRY(build_bands(ctx, n, rowptr_dev, col_dev, valK_dev, valM_dev, b, w, st));
  return launch_inertia(ctx, n, b, w, sigma_dev, nsig, count_dev, st);
}

extern "C" int fraclap_sturm_counts(fraclap_ctx* ctx, const double* d_dev, const double* e_dev, int64_t n,
                                    const double* sigma_dev, int64_t nsig, int64_t* count_dev,
                                    fraclap_stream_t stream) {
  if (!ctx) return FRACLAP_ERR_INVALID_ARG;
  FL_CHECK(ctx, n >= 1 && nsig >= 0, FRACLAP_ERR_INVALID_ARG, "sturm_counts: n must be positive");
  if (nsig == 0) return 0;
  FL_CHECK(ctx, d_dev && (e_dev || n == 1) && sigma_dev && count_dev, FRACLAP_ERR_INVALID_ARG,
           "sturm_counts: null pointer");
  FL_CHECK(ctx, cdiv(nsig, 128) <= INT32_MAX, FRACLAP_ERR_UNSUPPORTED, "sturm_counts: too many shifts");
  sturm_counts_kernel<<<(unsigned)cdiv(nsig, 128), 128, 0, (cudaStream_t)stream>>>(d_dev, e_dev, n, sigma_dev, nsig,
                                                                                   count_dev);
  count_launch(ctx);
  FL_CUDA(ctx, cudaGetLastError());
  return 0;
}

extern "C" int fraclap_bisect(fraclap_ctx* ctx, const double* d_dev, const double* e_dev, int64_t n, int64_t k0,
                              int64_t k1, double* lambda_dev, fraclap_stream_t stream) {
  if (!ctx) return FRACLAP_ERR_INVALID_ARG;
  FL_CHECK(ctx, n >= 1 && k0 >= 0 && k1 < n && k0 <= k1, FRACLAP_ERR_INVALID_ARG,
           "bisect: need 0 <= k0 <= k1 < n");
  FL_CHECK(ctx, d_dev && (e_dev || n == 1) && lambda_dev, FRACLAP_ERR_INVALID_ARG, "bisect: null pointer");
  cudaStream_t st = (cudaStream_t)stream;
  Arena ar;
  FL_TRY(get_workspace(ctx, nullptr, 0, 256, &ar));
  double* ghl = ar.take<double>(2);
  // a 1-element e keeps the kernels' reads in bounds for n == 1 (they read no e then)
  gershgorin_kernel<<<1, 256, 0, st>>>(d_dev, e_dev, n, ghl);
  count_launch(ctx);
  const int64_t cnt = k1 - k0 + 1;
  bisect_kernel<<<(unsigned)cdiv(cnt, 64), 64, 0, st>>>(d_dev, e_dev, n, k0, k1, ghl, lambda_dev);
  count_launch(ctx);
  FL_CUDA(ctx, cudaGetLastError());
  return 0;
}

extern "C" int fraclap_partition_spectrum(fraclap_ctx* ctx, int64_t n, const int64_t* rowptr_dev,
                                          const int32_t* col_dev, const double* valK_dev, const double* valM_dev,
                                          int64_t half_bandwidth, double rho, int P, int n_a, int n_b, int n_c,
                                          double imbalance, double* splits_host, int64_t* loads_host,
                                          int64_t* history_host, int history_cap, void* work_dev, size_t work_bytes,
                                          fraclap_stream_t stream) {
  if (!ctx) return FRACLAP_ERR_INVALID_ARG;
  FL_TRY(check_csr(ctx, "partition_spectrum", n, rowptr_dev, col_dev, valK_dev));
  FL_CHECK(ctx, P >= 1 && n_a >= 0 && n_b >= 0 && n_c >= 0 && rho > 0.0 && imbalance >= 0.0,
           FRACLAP_ERR_INVALID_ARG, "partition_spectrum: bad P, rho or pass counts");
  FL_CHECK(ctx, (P == 1 || splits_host) && loads_host && (history_cap == 0 || history_host),
           FRACLAP_ERR_INVALID_ARG, "partition_spectrum: null output");
  FL_CHECK(ctx, half_bandwidth >= 0, FRACLAP_ERR_INVALID_ARG, "partition_spectrum: bad bandwidth");
  cudaStream_t st = (cudaStream_t)stream;
  const int64_t b = std::min<int64_t>(half_bandwidth, n - 1);
  const int64_t nsig = std::max(P - 1, 1);
  Arena ar;
  const size_t need = inertia_ws(n, b, nsig, valM_dev != nullptr) + 2 * align256(sizeof(double) * nsig);
  FL_TRY(get_workspace(ctx, work_dev, work_bytes, need, &ar));
  InertiaWork w;
  inertia_take(&ar, n, b, nsig, valM_dev != nullptr, &w);
  double* sig = ar.take<double>(nsig);
  int64_t* cnt = ar.take<int64_t>(nsig);
  FL_CHECK(ctx, cnt != nullptr, FRACLAP_ERR_ALLOC, "partition_spectrum: workspace too small");
  FL_TRY(build_bands(ctx, n, rowptr_dev, col_dev, valK_dev, valM_dev, b, w, st));

  std::vector<int64_t> hist;
  std::vector<double> splits;
  for (int i = 1; i < P; ++i) splits.push_back(rho * (double)i / (double)P);
  std::vector<int64_t> counts, loads(P);
  auto loads_of = [&](const std::vector<double>& s) -> int {
    FL_TRY(counts_at(ctx, n, b, w, s, sig, cnt, &counts, st));
    int64_t prev = 0;
    for (int i = 0; i < P; ++i) {
      const int64_t c = (i < P - 1) ? counts[i] : n;
      loads[i] = c - prev;
      prev = c;
    }
    return 0;
  };
  auto max_load = [&]() { return *std::max_element(loads.begin(), loads.end()); };
  FL_TRY(loads_of(splits));
  int64_t best_max = max_load();
  std::vector<double> best_splits = splits;
  std::vector<int64_t> best_loads = loads;
  hist.push_back(best_max);
  // global refinement (n_a rounds): every split at once from the density the counts describe
  for (int r = 0; r < n_a; ++r) {
    std::vector<double> pts{0.0}, cum{0.0};
    for (int i = 0; i < P - 1; ++i) {
      pts.push_back(splits[i]);
      cum.push_back((double)counts[i]);
    }
    pts.push_back(rho);
    cum.push_back((double)n);
    splits = equal_load_splits(pts, cum, n, P);
    FL_TRY(loads_of(splits));
    hist.push_back(max_load());
    if (max_load() < best_max) {
      best_max = max_load();
      best_splits = splits;
      best_loads = loads;
    }
  }
  splits = best_splits;
  loads = best_loads;
  // local refinement (n_b passes): unbalanced neighbouring pairs move their
  // shared split by a binary search of n_c counts, all pairs of one parity
  // at once (one launch per search step), even positions first
  const double ideal = (double)n / (double)P;
  for (int pass = 0; pass < n_b; ++pass) {
    bool changed = false;
    for (int parity = 0; parity < 2; ++parity) {
      std::vector<int> pairs;
      for (int a = parity; a < P - 1; a += 2)
        if ((double)std::llabs(loads[a] - loads[a + 1]) > imbalance * ideal) pairs.push_back(a);
      if (pairs.empty()) continue;
      const int np = (int)pairs.size();
      std::vector<double> lo(np), hi(np), want(np), x0(np), x1(np);
      std::vector<int64_t> left(np, 0);
      std::vector<double> lefts_at;
      for (int q = 0; q < np; ++q) {
        const int a = pairs[q];
        lo[q] = (a > 0) ? splits[a - 1] : 0.0;
        hi[q] = (a + 1 < P - 1) ? splits[a + 1] : rho;
        if (a > 0) lefts_at.push_back(lo[q]);
      }
      std::vector<int64_t> lc;
      FL_TRY(counts_at(ctx, n, b, w, lefts_at, sig, cnt, &lc, st));
      for (int q = 0, t = 0; q < np; ++q) {
        const int a = pairs[q];
        left[q] = (a > 0) ? lc[t++] : 0;
        want[q] = (double)left[q] + (double)(loads[a] + loads[a + 1]) / 2.0;
        x0[q] = lo[q];
        x1[q] = hi[q];
      }
      for (int step = 0; step < n_c; ++step) {
        std::vector<double> mids(np);
        for (int q = 0; q < np; ++q) mids[q] = 0.5 * (x0[q] + x1[q]);
        std::vector<int64_t> mc;
        FL_TRY(counts_at(ctx, n, b, w, mids, sig, cnt, &mc, st));
        for (int q = 0; q < np; ++q) {
          if ((double)mc[q] < want[q]) x0[q] = mids[q];
          else x1[q] = mids[q];
        }
      }
      std::vector<double> news(np);
      for (int q = 0; q < np; ++q) news[q] = 0.5 * (x0[q] + x1[q]);
      std::vector<int64_t> nc;
      FL_TRY(counts_at(ctx, n, b, w, news, sig, cnt, &nc, st));
      for (int q = 0; q < np; ++q) {
        const int a = pairs[q];
        splits[a] = news[q];
        const int64_t tot = loads[a] + loads[a + 1];
        loads[a] = nc[q] - left[q];
        loads[a + 1] = tot - loads[a];
      }
      changed = true;
    }
    hist.push_back(max_load());
    if (!changed) break;
  }
  for (int i = 0; i < P - 1; ++i) splits_host[i] = splits[i];
  for (int i = 0; i < P; ++i) loads_host[i] = loads[i];
  const int nh = (int)hist.size();
  for (int i = 0; i < nh && i < history_cap; ++i) history_host[i] = hist[i];
  return nh;
}
