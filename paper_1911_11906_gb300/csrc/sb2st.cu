// Stage 2 of the two-stage reduction: band (half-width b) -> tridiagonal,
// by bulge chasing with Householder reflectors of length <= b, and the
// back-transformation by the stage-2 orthogonal factor.
//
// Sweep s annihilates column s below the subdiagonal (reflector on rows
// s+1..s+b), applies it to the diagonal block and, from the right, to the
// block below, which creates a bulge; step k then annihilates the first
// column of the previous window in rows s+1+kb..s+(k+1)b and pushes the
// bulge one window further.  Only that first column is annihilated; the rest
// of the fill stays within 2b-1 diagonals of storage and is absorbed by the
// later sweeps.  Step k of sweep s touches indices
// [s+1+(k-1)b, s+(k+2)b], so it may run as soon as sweep s-1 has finished
// its step k+3: sweeps run in a pipeline, one CTA per sweep in flight, each
// CTA waiting (bounded in time) on a progress counter of its predecessor.
//
// The reflectors H(s,k) of one sweep act on disjoint rows; H(s,k) and
// H(s',k') with k > k', s > s' or k < k', s < s' act on disjoint rows as
// well, so Q2 = prod_s prod_k H(s,k) = prod_{k descending} prod_{s ascending}
// H(s,k).  For fixed k the reflectors form a staircase shifted by one row per
// sweep; Z <- Q2 Z applies k = 0, 1, ... in turn with s descending, keeping a
// sliding window of b rows of Z in shared memory (one lane per column).
#include "internal.cuh"

namespace fraclap {
namespace {

constexpr int SB_NT = 256;

__device__ __forceinline__ int64_t sb_nsteps(int64_t s, int64_t n, int b) {
  return (n - 2 - s) / b + 1;  // valid for s <= n - 2
}

struct SbArgs {
  double* band;   // ld = 2b, band(i - j, j) = A(i, j)
  int64_t n;
  int b;
  int64_t kmax;   // steps of sweep 0
  double* refl;   // (n-1) * kmax * b
  double* rtau;   // (n-1) * kmax
  int* progress;  // n, completed steps per sweep
  int32_t* status;
  long long limit;
};

__global__ void __launch_bounds__(SB_NT) sb2st_kernel(SbArgs a) {
  extern __shared__ double sm[];
  const int b = a.b, ldb = 2 * b;
  const int64_t n = a.n;
  double* xv = sm;                 // b
  double* F = xv + 64;             // b x b  (F[t + q*b])
  double* D = F + 64 * 64;         // b x b  full symmetric (D[t + u*b])
  double* E = D + 64 * 64;         // b x b  (E[t + u*b])
  double* pw = E + 64 * 64;        // b
  double* wq = pw + 64;            // b
  __shared__ double s_coef[4];
  __shared__ int s_abort;
  const int tid = threadIdx.x;
  double* band = a.band;
#define BAND(i, j) band[((i) - (j)) + (int64_t)(j) * ldb]

  for (int64_t s = blockIdx.x; s < n - 1; s += gridDim.x) {
    const int64_t ns = sb_nsteps(s, n, b);
    const int64_t ns_prev = (s > 0) ? sb_nsteps(s - 1, n, b) : 0;
    for (int64_t k = 0; k < ns; ++k) {
      // ---- wait for sweep s-1 to have completed step k+3 ----
      if (tid == 0) {
        int ok = 1;
        if (s > 0) {
          const int64_t need = (k + 4 < ns_prev) ? k + 4 : ns_prev;
          const long long t0 = clock64();
          while (ld_acquire_gpu(a.progress + (s - 1)) < need) {
            if (*(volatile int32_t*)a.status != 0) { ok = 0; break; }
            if (clock64() - t0 > a.limit) {
              raise_status(a.status, FRACLAP_ERR_TIMEOUT);
              ok = 0;
              break;
            }
            __nanosleep(32);
          }
          __threadfence();
        }
        s_abort = !ok;
      }
      __syncthreads();
      if (s_abort) return;

      const int64_t r0 = s + 1 + k * b;
      const int L = (int)((n - r0 < b) ? n - r0 : b);
      const int64_t r1 = r0 + L - 1;
      const int64_t c = (k == 0) ? s : r0 - b;
      const int nf = (int)(r0 - 1 - c);
      const int Lb = (int)((n - 1 - r1 < b) ? n - 1 - r1 : b);

      // ---- load ----
      for (int t = tid; t < L; t += SB_NT) xv[t] = __ldcg(&BAND(r0 + t, c));
      for (int p = tid; p < L * nf; p += SB_NT) {
        const int t = p % L, q = p / L;
        F[t + q * b] = __ldcg(&BAND(r0 + t, c + 1 + q));
      }
      for (int p = tid; p < L * L; p += SB_NT) {
        const int t = p % L, u = p / L;
        if (t >= u) {
          const double v = __ldcg(&BAND(r0 + t, r0 + u));
          D[t + u * b] = v;
          D[u + t * b] = v;
        }
      }
      for (int p = tid; p < Lb * L; p += SB_NT) {
        const int t = p % Lb, u = p / Lb;
        E[t + u * b] = __ldcg(&BAND(r1 + 1 + t, r0 + u));
      }
      __syncthreads();
      // ---- Householder vector from x (warp 0) ----
      if (tid < 32) {
        double tail = 0.0;
        for (int t = 1 + tid; t < L; t += 32) tail += xv[t] * xv[t];
        tail = warp_sum(tail);
        const double x0 = xv[0];
        double beta = x0, v0 = 1.0, tu = 0.0;
        if (tail > 0.0) {
          const double alpha = sqrt(x0 * x0 + tail);
          beta = (x0 >= 0.0) ? -alpha : alpha;
          v0 = x0 - beta;
          tu = (beta - x0) / beta;
        }
        if (tid == 0) {
          s_coef[0] = beta;
          s_coef[1] = tu;
          s_coef[2] = v0;
        }
        __syncwarp();
        const double inv = 1.0 / v0;
        for (int t = 1 + tid; t < L; t += 32) xv[t] = (tu == 0.0) ? 0.0 : xv[t] * inv;
        if (tid == 0) xv[0] = 1.0;
      }
      __syncthreads();
      const double beta = s_coef[0], tu = s_coef[1];
      double* rv = a.refl + ((int64_t)s * a.kmax + k) * b;
      for (int t = tid; t < b; t += SB_NT) rv[t] = (t < L) ? xv[t] : 0.0;
      if (tid == 0) a.rtau[s * a.kmax + k] = tu;
      if (tu != 0.0) {
        // ---- F <- H F, E <- E H, p = tau D v ----
        for (int q = tid; q < nf; q += SB_NT) {
          double w = 0.0;
          for (int t = 0; t < L; ++t) w += xv[t] * F[t + q * b];
          wq[q] = tu * w;
        }
        for (int t = tid; t < L; t += SB_NT) {
          double p = 0.0;
          for (int u = 0; u < L; ++u) p += D[t + u * b] * xv[u];
          pw[t] = tu * p;
        }
        __syncthreads();
        for (int p = tid; p < L * nf; p += SB_NT) {
          const int t = p % L, q = p / L;
          F[t + q * b] -= xv[t] * wq[q];
        }
        if (tid == 0) {
          double pv = 0.0;
          for (int t = 0; t < L; ++t) pv += pw[t] * xv[t];
          s_coef[3] = 0.5 * tu * pv;
        }
        __syncthreads();
        const double K = s_coef[3];
        for (int t = tid; t < L; t += SB_NT) pw[t] -= K * xv[t];  // w = p - K v
        // E <- E H : y_t = tau E(t,:) v
        for (int t = tid; t < Lb; t += SB_NT) {
          double y = 0.0;
          for (int u = 0; u < L; ++u) y += E[t + u * b] * xv[u];
          y *= tu;
          for (int u = 0; u < L; ++u) E[t + u * b] -= y * xv[u];
        }
        __syncthreads();
        for (int p = tid; p < L * L; p += SB_NT) {
          const int t = p % L, u = p / L;
          if (t >= u) D[t + u * b] -= xv[t] * pw[u] + pw[t] * xv[u];
        }
        __syncthreads();
        // ---- store ----
        for (int t = tid; t < L; t += SB_NT) __stcg(&BAND(r0 + t, c), (t == 0) ? beta : 0.0);
        for (int p = tid; p < L * nf; p += SB_NT) {
          const int t = p % L, q = p / L;
          __stcg(&BAND(r0 + t, c + 1 + q), F[t + q * b]);
        }
        for (int p = tid; p < L * L; p += SB_NT) {
          const int t = p % L, u = p / L;
          if (t >= u) __stcg(&BAND(r0 + t, r0 + u), D[t + u * b]);
        }
        for (int p = tid; p < Lb * L; p += SB_NT) {
          const int t = p % Lb, u = p / Lb;
          __stcg(&BAND(r1 + 1 + t, r0 + u), E[t + u * b]);
        }
      }
      __syncthreads();
      if (tid == 0) {
        __threadfence();
        st_release_gpu(a.progress + s, (int)(k + 1));
      }
    }
  }
#undef BAND
}

__global__ void band_diagonals(const double* band, int ldb, int64_t n, double* d, double* e) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  d[i] = band[i * ldb];
  if (i + 1 < n) e[i] = band[1 + i * ldb];
}

// Z <- Q2 Z.  One warp per 32 columns (lane = column); per warp a window of
// b rows in shared memory, slot of row r = r mod b.
constexpr int Q2_WARPS = 2;

__global__ void __launch_bounds__(Q2_WARPS * 32)
q2_apply_kernel(const double* refl, const double* rtau, int64_t n, int b, int64_t kmax,
                double* Z, int64_t ldz, int64_t ncols) {
  extern __shared__ double win_all[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  double* win = win_all + (size_t)warp * b * 32;
  const int64_t col = ((int64_t)blockIdx.x * Q2_WARPS + warp) * 32 + lane;
  const bool active = col < ncols;
  double* zc = Z + (active ? col : 0) * ldz;
  for (int64_t k = 0; k < kmax; ++k) {
    const int64_t smax = n - 2 - k * b;
    if (smax < 0) break;
    int64_t lo = n, hi = n - 1;  // window rows [lo, hi] (empty)
    for (int64_t s = smax; s >= 0; --s) {
      const int64_t r0 = s + 1 + k * b;
      const int L = (int)((n - r0 < b) ? n - r0 : b);
      const int64_t r1 = r0 + L - 1;
      // slide: drop rows > r1, add row r0
      while (hi > r1) {
        if (active) zc[hi] = win[(hi % b) * 32 + lane];
        --hi;
      }
      if (r0 < lo) {
        lo = r0;
        win[(r0 % b) * 32 + lane] = active ? zc[r0] : 0.0;
      }
      const double tu = __ldg(rtau + s * kmax + k);
      if (tu == 0.0) continue;
      const double* v = refl + (s * kmax + k) * b;
      const double va = (lane < L) ? __ldg(v + lane) : 0.0;
      const double vb = (lane + 32 < L) ? __ldg(v + lane + 32) : 0.0;
      double acc0 = 0.0, acc1 = 0.0;
      int t = 0;
      for (; t + 1 < L; t += 2) {
        const double v0 = __shfl_sync(0xffffffffu, t < 32 ? va : vb, t & 31);
        const double v1 = __shfl_sync(0xffffffffu, (t + 1) < 32 ? va : vb, (t + 1) & 31);
        acc0 = fma(v0, win[((r0 + t) % b) * 32 + lane], acc0);
        acc1 = fma(v1, win[((r0 + t + 1) % b) * 32 + lane], acc1);
      }
      if (t < L) {
        const double v0 = __shfl_sync(0xffffffffu, t < 32 ? va : vb, t & 31);
        acc0 = fma(v0, win[((r0 + t) % b) * 32 + lane], acc0);
      }
      const double w = tu * (acc0 + acc1);
      for (t = 0; t < L; ++t) {
        const double vt = __shfl_sync(0xffffffffu, t < 32 ? va : vb, t & 31);
        double* z = &win[((r0 + t) % b) * 32 + lane];
        *z = fma(-w, vt, *z);
      }
    }
    while (hi >= lo) {  // flush
      if (active) zc[hi] = win[(hi % b) * 32 + lane];
      --hi;
    }
  }
}

}  // namespace

int stage2_take(Arena* ar, int64_t n, int b, Stage2* s) {
  s->kmax = (n >= 2) ? (n - 2) / b + 1 : 0;
  const int64_t nsw = (n >= 2) ? n - 1 : 0;
  s->refl = ar->take<double>(nsw * s->kmax * b);
  s->rtau = ar->take<double>(nsw * s->kmax);
  s->progress = ar->take<int>(n + 1);
  return 0;
}

int sb2st_run(fraclap_ctx* ctx, double* band, int64_t n, int b, double* d, double* e, Stage2* s,
              cudaStream_t st) {
  if (n >= 2) {
    FL_CUDA(ctx, cudaMemsetAsync(s->progress, 0, sizeof(int) * (n + 1), st));
    FL_CUDA(ctx, cudaMemsetAsync(s->rtau, 0, sizeof(double) * (n - 1) * s->kmax, st));
    SbArgs a{band, n, b, s->kmax, s->refl, s->rtau, s->progress, ctx->d_status, ctx->wait_cycles};
    const size_t smem = sizeof(double) * (64 + 3 * 64 * 64 + 2 * 64);
    FL_CUDA(ctx, cudaFuncSetAttribute(sb2st_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int per_sm = 0;
    FL_CUDA(ctx, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, sb2st_kernel, SB_NT, smem));
    FL_CHECK(ctx, per_sm >= 1, FRACLAP_ERR_UNSUPPORTED, "sb2st: kernel does not fit on an SM");
    int64_t G = (int64_t)ctx->sm_count * per_sm;
    if (G > n - 1) G = n - 1;
    void* args[] = {&a};
    count_launch(ctx);
      FL_CUDA(ctx, cudaLaunchCooperativeKernel((void*)sb2st_kernel, dim3((unsigned)G), dim3(SB_NT), args, smem, st));
  }
  if (n >= 1) {
    band_diagonals<<<(unsigned)cdiv(n, 256), 256, 0, st>>>(band, 2 * b, n, d, e);
    count_launch(ctx);
    FL_CUDA(ctx, cudaGetLastError());
  }
  return 0;
}

int q2_apply_run(fraclap_ctx* ctx, const Stage2* s, int64_t n, int b, double* Z, int64_t ldz,
                 int64_t ncols, cudaStream_t st) {
  if (n < 2 || ncols <= 0) return 0;
  const size_t smem = sizeof(double) * (size_t)Q2_WARPS * b * 32;
  FL_CUDA(ctx, cudaFuncSetAttribute(q2_apply_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  const int64_t grid = cdiv(ncols, 32 * Q2_WARPS);
  q2_apply_kernel<<<(unsigned)grid, Q2_WARPS * 32, smem, st>>>(s->refl, s->rtau, n, b, s->kmax, Z, ldz,
                                                               ncols);
  count_launch(ctx);
  FL_CUDA(ctx, cudaGetLastError());
  return 0;
}

}  // namespace fraclap
