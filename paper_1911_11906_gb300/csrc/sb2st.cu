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
// later sweeps.  Step k of sweep s touches only entries in rows
// [s+1+kb, s+(k+2)b]; step k' of sweep s-1 touches rows from s+k'b on, so
// the two are disjoint once k' >= k+3 (at k' = k+2 they share the entry
// (s+(k+2)b, s+(k+1)b)).  Sweep s may therefore run step k as soon as sweep
// s-1 has finished its step k+2: sweeps run in a pipeline, one CTA per sweep
// in flight, each CTA waiting (bounded in time) on a progress counter of its
// predecessor.
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

template <class T>
struct SbArgs {
  T* band;        // ld = 2b, band(i - j, j) = A(i, j)
  int64_t n;
  int b;
  int64_t kmax;   // steps of sweep 0
  T* refl;        // (n-1) * kmax * b
  double* rtau;   // (n-1) * kmax
  int* progress;  // n, completed steps per sweep
  int32_t* status;
  long long limit;
};

template <class T>
__global__ void __launch_bounds__(SB_NT) sb2st_kernel(SbArgs<T> a) {
  extern __shared__ __align__(16) unsigned char sm_raw[];
  T* sm = reinterpret_cast<T*>(sm_raw);
  const int b = a.b, ldb = 2 * b;
  const int64_t n = a.n;
  T* xv = sm;                 // b
  T* F = xv + 64;             // b x b  (F[t + q*b])
  T* D = F + 64 * 64;         // b x b  full symmetric (D[t + u*b])
  T* E = D + 64 * 64;         // b x b  (E[t + u*b])
  T* pw = E + 64 * 64;        // b
  T* wq = pw + 64;            // b
  T* ey = wq + 64;            // b
  __shared__ double s_coef[4];
  __shared__ int s_abort;
  const int tid = threadIdx.x;
  T* band = a.band;
#define BAND(i, j) band[((i) - (j)) + (int64_t)(j) * ldb]

  for (int64_t s = blockIdx.x; s < n - 1; s += gridDim.x) {
    const int64_t ns = sb_nsteps(s, n, b);
    const int64_t ns_prev = (s > 0) ? sb_nsteps(s - 1, n, b) : 0;
    for (int64_t k = 0; k < ns; ++k) {
      // ---- wait for sweep s-1 to have completed step k+2 ----
      if (tid == 0) {
        int ok = 1;
        if (s > 0) {
          const int64_t need = (k + 3 < ns_prev) ? k + 3 : ns_prev;
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
          const T v = __ldcg(&BAND(r0 + t, r0 + u));
          D[t + u * b] = v;
          D[u + t * b] = v;
        }
      }
      for (int p = tid; p < Lb * L; p += SB_NT) {
        const int t = p % Lb, u = p / Lb;
        E[t + u * b] = __ldcg(&BAND(r1 + 1 + t, r0 + u));
      }
      __syncthreads();
      // ---- Householder vector from x (warp 0), norms and scaling in FP64 ----
      if (tid < 32) {
        double tail = 0.0;
        for (int t = 1 + tid; t < L; t += 32) tail += (double)xv[t] * (double)xv[t];
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
        for (int t = 1 + tid; t < L; t += 32) xv[t] = (tu == 0.0) ? T(0) : (T)((double)xv[t] * inv);
        if (tid == 0) xv[0] = T(1);
      }
      __syncthreads();
      const double beta = s_coef[0], tu = s_coef[1];
      const T tuT = (T)tu;
      T* rv = a.refl + ((int64_t)s * a.kmax + k) * b;
      for (int t = tid; t < b; t += SB_NT) rv[t] = (t < L) ? xv[t] : T(0);
      if (tid == 0) a.rtau[s * a.kmax + k] = tu;
      if (tu != 0.0) {
        // ---- wq = tau F^T v, pw = tau D v, y = tau E v: 4 threads per dot ----
        {
          const int part = tid & 3;
          const int ntask = nf + L + Lb;
          // warp-uniform trip count: every lane reaches the shuffles
          for (int base = 0; base < ntask; base += SB_NT / 4) {
            const int task = base + (tid >> 2);
            T acc = T(0);
            if (task >= ntask) {
            } else if (task < nf) {
              const T* col = F + task * b;
              for (int t = part; t < L; t += 4) acc += xv[t] * col[t];
            } else if (task < nf + L) {
              const int t = task - nf;
              for (int u = part; u < L; u += 4) acc += D[t + u * b] * xv[u];
            } else {
              const int t = task - nf - L;
              for (int u = part; u < L; u += 4) acc += E[t + u * b] * xv[u];
            }
            acc += __shfl_xor_sync(0xffffffffu, acc, 1);
            acc += __shfl_xor_sync(0xffffffffu, acc, 2);
            if (part == 0 && task < ntask) {
              if (task < nf) wq[task] = tuT * acc;
              else if (task < nf + L) pw[task - nf] = tuT * acc;
              else ey[task - nf - L] = tuT * acc;
            }
          }
        }
        __syncthreads();
        for (int p = tid; p < L * nf; p += SB_NT) {
          const int t = p % L, q = p / L;
          F[t + q * b] -= xv[t] * wq[q];
        }
        for (int p = tid; p < Lb * L; p += SB_NT) {
          const int t = p % Lb, u = p / Lb;
          E[t + u * b] -= ey[t] * xv[u];
        }
        if (tid < 32) {  // K = tau/2 p^T v
          double pv = 0.0;
          for (int t = tid; t < L; t += 32) pv += (double)pw[t] * (double)xv[t];
          pv = warp_sum(pv);
          if (tid == 0) s_coef[3] = 0.5 * tu * pv;
        }
        __syncthreads();
        const T K = (T)s_coef[3];
        for (int t = tid; t < L; t += SB_NT) pw[t] -= K * xv[t];  // w = p - K v
        __syncthreads();
        for (int p = tid; p < L * L; p += SB_NT) {
          const int t = p % L, u = p / L;
          if (t >= u) D[t + u * b] -= xv[t] * pw[u] + pw[t] * xv[u];
        }
        __syncthreads();
        // ---- store ----
        for (int t = tid; t < L; t += SB_NT) __stcg(&BAND(r0 + t, c), (t == 0) ? (T)beta : T(0));
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

template <class T>
__global__ void band_diagonals(const T* band, int ldb, int64_t n, double* d, double* e) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  d[i] = band[i * ldb];
  if (i + 1 < n) e[i] = band[1 + i * ldb];
}

// Y <- Y Q2^T, i.e. Z <- Q2 Z on the transpose Y = Z^T (ld >= n), so that a
// row of Z is contiguous.  For each step k the reflectors H(s, k), s
// descending, act on a window of B rows of Z that slides up by one row per
// reflector.  A warp owns CPW = 32/P columns of Z; its lanes split the window
// into P parts of R = B/P rows each, held in registers: the dot product of a
// reflector with a column is a partial sum per part plus a butterfly over the
// P parts, and the slide moves one row per part boundary with a shuffle.  The
// CTA stages the reflectors of the next D steps in shared memory (double
// buffered) while it applies the current D; the rows entering the window are
// loaded one batch ahead.  Work: 4 L n flops per reflector of length L.
constexpr int Q2T_WARPS = 8, Q2T_D = 8;

template <class T, int B, int P>
__global__ void __launch_bounds__(Q2T_WARPS * 32, 2)
q2t_apply_kernel(const T* __restrict__ refl, const double* __restrict__ rtau, int64_t n,
                 int64_t kmax, T* Y, int64_t ldy, int64_t ncols) {
  constexpr int R = B / P, CPW = 32 / P, D = Q2T_D, NT = Q2T_WARPS * 32;
  constexpr int PER = (D * B + NT - 1) / NT;  // staged doubles per thread
  __shared__ T vbuf[2][D][B];
  __shared__ T tbuf[2][D];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int part = lane / CPW, cl = lane % CPW;
  const int64_t col = ((int64_t)blockIdx.x * Q2T_WARPS + warp) * CPW + cl;
  const bool active = col < ncols;
  T* yc = Y + (active ? col : 0);
  const unsigned full = 0xffffffffu;

  for (int64_t k = 0; k < kmax; ++k) {
    const int64_t smax = n - 2 - k * B;
    if (smax < 0) break;
    const int64_t nbatch = (smax + D) / D;  // reflectors s = smax .. 0
    // stage a batch of reflectors (q = batch * D + j  <->  s = smax - q)
    auto fetch = [&](int64_t batch, T* vr, T* tr) {
      for (int e = 0; e < PER; ++e) {
        const int t = threadIdx.x + e * NT;
        T v = T(0);
        if (t < D * B) {
          const int j = t / B, c = t % B;
          const int64_t sj = smax - (batch * D + j);
          if (sj >= 0) v = __ldg(refl + (sj * kmax + k) * B + c);
        }
        vr[e] = v;
      }
      T tv = T(0);
      if (threadIdx.x < D) {
        const int64_t sj = smax - (batch * D + threadIdx.x);
        if (sj >= 0) tv = (T)__ldg(rtau + sj * kmax + k);
      }
      *tr = tv;
    };
    auto store = [&](int buf, const T* vr, T tr) {
      for (int e = 0; e < PER; ++e) {
        const int t = threadIdx.x + e * NT;
        if (t < D * B) vbuf[buf][t / B][t % B] = vr[e];
      }
      if (threadIdx.x < D) tbuf[buf][threadIdx.x] = tr;
    };
    T vr[PER], tr;
    fetch(0, vr, &tr);
    __syncthreads();  // previous k's readers are done with the buffers
    store(0, vr, tr);

    int64_t r0 = n - 1;  // window rows r0 .. r0 + B - 1 (rows >= n are zero)
    T w[R];
#pragma unroll
    for (int i = 0; i < R; ++i) {
      const int64_t row = r0 + part * R + i;
      w[i] = (active && row < n) ? yc[row * ldy] : T(0);
    }
    T pf[D];  // rows entering the window during the current batch (part 0)
#pragma unroll
    for (int j = 0; j < D; ++j) {
      const int64_t row = r0 - 1 - j;
      pf[j] = (part == 0 && active && row >= 1 + k * B) ? yc[row * ldy] : T(0);
    }
    __syncthreads();
    for (int64_t batch = 0; batch < nbatch; ++batch) {
      const int buf = (int)(batch & 1);
      const bool more = batch + 1 < nbatch;
      if (more) fetch(batch + 1, vr, &tr);
      T pn[D];  // rows for the next batch
#pragma unroll
      for (int j = 0; j < D; ++j) {
        const int64_t row = r0 - 1 - D - j;
        pn[j] = (more && part == 0 && active && row >= 1 + k * B) ? yc[row * ldy] : T(0);
      }
#pragma unroll
      for (int j = 0; j < D; ++j) {
        const int64_t s = smax - (batch * D + j);
        if (s < 0) break;
        const T* v = &vbuf[buf][j][part * R];
        T d0 = T(0), d1 = T(0);
#pragma unroll
        for (int i = 0; i < R; i += 2) {
          d0 = fma(v[i], w[i], d0);
          if (i + 1 < R) d1 = fma(v[i + 1], w[i + 1], d1);
        }
        T dot = d0 + d1;
#pragma unroll
        for (int o = CPW; o < 32; o <<= 1) dot += __shfl_xor_sync(full, dot, o);
        const T f = tbuf[buf][j] * dot;
#pragma unroll
        for (int i = 0; i < R; ++i) w[i] = fma(-f, v[i], w[i]);
        if (s > 0) {  // slide the window up by one row
          const T out = w[R - 1];
          const int64_t leaving = r0 + B - 1;
          if (part == P - 1 && active && leaving < n) yc[leaving * ldy] = out;
          const T prev = __shfl_up_sync(full, out, CPW);
#pragma unroll
          for (int i = R - 1; i > 0; --i) w[i] = w[i - 1];
          w[0] = (part == 0) ? pf[j] : prev;
          --r0;
        }
      }
#pragma unroll
      for (int j = 0; j < D; ++j) pf[j] = pn[j];
      if (more) {
        store(buf ^ 1, vr, tr);
        __syncthreads();
      }
    }
#pragma unroll
    for (int i = 0; i < R; ++i) {  // flush the final window (rows 1 + kB ..)
      const int64_t row = r0 + part * R + i;
      if (active && row < n) yc[row * ldy] = w[i];
    }
  }
}

// 32 x 32 tiled transpose: B(j, i) = A(i, j), A is rows x cols.
template <class T>
__global__ void transpose_kernel(const T* A, int64_t lda, T* Bm, int64_t ldb, int64_t rows,
                                 int64_t cols) {
  __shared__ T tile[32][33];
  const int64_t i0 = (int64_t)blockIdx.x * 32, j0 = (int64_t)blockIdx.y * 32;
  for (int t = threadIdx.y; t < 32; t += blockDim.y) {
    const int64_t i = i0 + threadIdx.x, j = j0 + t;
    if (i < rows && j < cols) tile[t][threadIdx.x] = A[i + j * lda];
  }
  __syncthreads();
  for (int t = threadIdx.y; t < 32; t += blockDim.y) {
    const int64_t j = j0 + threadIdx.x, i = i0 + t;
    if (i < rows && j < cols) Bm[j + i * ldb] = tile[threadIdx.x][t];
  }
}

}  // namespace

template <class T>
int stage2_take(Arena* ar, int64_t n, int b, Stage2T<T>* s) {
  s->kmax = (n >= 2) ? (n - 2) / b + 1 : 0;
  const int64_t nsw = (n >= 2) ? n - 1 : 0;
  s->refl = ar->take<T>(nsw * s->kmax * b);
  s->rtau = ar->take<double>(nsw * s->kmax);
  s->progress = ar->take<int>(n + 1);
  return 0;
}

template <class T>
int sb2st_run(fraclap_ctx* ctx, T* band, int64_t n, int b, double* d, double* e, Stage2T<T>* s,
              cudaStream_t st) {
  if (n >= 2) {
    FL_CUDA(ctx, cudaMemsetAsync(s->progress, 0, sizeof(int) * (n + 1), st));
    FL_CUDA(ctx, cudaMemsetAsync(s->rtau, 0, sizeof(double) * (n - 1) * s->kmax, st));
    SbArgs<T> a{band, n, b, s->kmax, s->refl, s->rtau, s->progress, ctx->d_status, ctx->wait_cycles};
    const size_t smem = sizeof(T) * (64 + 3 * 64 * 64 + 3 * 64);
    FL_CUDA(ctx, cudaFuncSetAttribute(sb2st_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int per_sm = 0;
    FL_CUDA(ctx, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, sb2st_kernel<T>, SB_NT, smem));
    FL_CHECK(ctx, per_sm >= 1, FRACLAP_ERR_UNSUPPORTED, "sb2st: kernel does not fit on an SM");
    int64_t G = (int64_t)ctx->sm_count * per_sm;
    if (G > n - 1) G = n - 1;
    void* args[] = {&a};
    count_launch(ctx);
    FL_CUDA(ctx, cudaLaunchCooperativeKernel((void*)sb2st_kernel<T>, dim3((unsigned)G), dim3(SB_NT), args, smem, st));
  }
  if (n >= 1) {
    band_diagonals<T><<<(unsigned)cdiv(n, 256), 256, 0, st>>>(band, 2 * b, n, d, e);
    count_launch(ctx);
    FL_CUDA(ctx, cudaGetLastError());
  }
  return 0;
}

template <class T>
int transpose_run(fraclap_ctx* ctx, const T* A, int64_t lda, T* Bm, int64_t ldb, int64_t rows,
                  int64_t cols, cudaStream_t st) {
  if (rows <= 0 || cols <= 0) return 0;
  dim3 grid((unsigned)cdiv(rows, 32), (unsigned)cdiv(cols, 32));
  FL_CHECK(ctx, grid.y <= 65535, FRACLAP_ERR_UNSUPPORTED, "transpose: too many columns");
  transpose_kernel<T><<<grid, dim3(32, 8), 0, st>>>(A, lda, Bm, ldb, rows, cols);
  count_launch(ctx);
  FL_CUDA(ctx, cudaGetLastError());
  return 0;
}

// Z <- Q2 Z (n x ncols, ld ldz), through the transposed copy Yt (ld >= ncols).
template <class T>
int q2_apply_run(fraclap_ctx* ctx, const Stage2T<T>* s, int64_t n, int b, T* Z, int64_t ldz,
                 int64_t ncols, T* Yt, int64_t ldy, cudaStream_t st) {
  if (n < 2 || ncols <= 0) return 0;
  FL_TRY(transpose_run<T>(ctx, Z, ldz, Yt, ldy, n, ncols, st));
  int cpw = 0;
#define FL_Q2T(BB, PP)                                                                        \
  if (b == BB) {                                                                              \
    cpw = 32 / PP;                                                                            \
    const int64_t grid = cdiv(ncols, (int64_t)cpw * Q2T_WARPS);                                \
    q2t_apply_kernel<T, BB, PP><<<(unsigned)grid, Q2T_WARPS * 32, 0, st>>>(s->refl, s->rtau, n, \
                                                                          s->kmax, Yt, ldy, ncols); \
    count_launch(ctx);                                                                        \
  }
  FL_Q2T(4, 1)
  FL_Q2T(8, 2)
  FL_Q2T(16, 4)
  FL_Q2T(32, 8)
  FL_Q2T(64, 8)
#undef FL_Q2T
  FL_CHECK(ctx, cpw != 0, FRACLAP_ERR_UNSUPPORTED, "q2 back-transformation: band width %d not in {4, 8, 16, 32, 64}", b);
  FL_CUDA(ctx, cudaGetLastError());
  return transpose_run<T>(ctx, Yt, ldy, Z, ldz, ncols, n, st);
}

template int stage2_take<double>(Arena*, int64_t, int, Stage2T<double>*);
template int stage2_take<float>(Arena*, int64_t, int, Stage2T<float>*);
template int sb2st_run<double>(fraclap_ctx*, double*, int64_t, int, double*, double*, Stage2T<double>*, cudaStream_t);
template int sb2st_run<float>(fraclap_ctx*, float*, int64_t, int, double*, double*, Stage2T<float>*, cudaStream_t);
template int transpose_run<double>(fraclap_ctx*, const double*, int64_t, double*, int64_t, int64_t, int64_t, cudaStream_t);
template int transpose_run<float>(fraclap_ctx*, const float*, int64_t, float*, int64_t, int64_t, int64_t, cudaStream_t);
template int q2_apply_run<double>(fraclap_ctx*, const Stage2T<double>*, int64_t, int, double*, int64_t, int64_t, double*, int64_t, cudaStream_t);
template int q2_apply_run<float>(fraclap_ctx*, const Stage2T<float>*, int64_t, int, float*, int64_t, int64_t, float*, int64_t, cudaStream_t);

}  // namespace fraclap
