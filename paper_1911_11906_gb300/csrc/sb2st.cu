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
// the two are disjoint once k' >= k+3; at k' = k+2 they share only the
// entry (s+(k+2)b, s+(k+1)b), which step k+2 of sweep s-1 sets to the new
// subdiagonal value beta of its reflector before anything else.  Sweep s may
// therefore run step k as soon as sweep s-1 has finished its step k+1 and
// published the beta of its step k+2 (written to the band right after it is
// computed, with a second counter): sweeps run in a pipeline, one CTA per
// sweep in flight, each CTA waiting (bounded in time) on the counters of its
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
  int* beta_progress;  // n, steps per sweep whose subdiagonal value is in the band
  int32_t* status;
  long long limit;
};

// Step of one sweep: thread (t, g) = (tid % B, tid / B) owns row t of the
// step's blocks and the columns u = g + NG i (i < B / NG) of each: the column
// block [x | F] (u = 0 is x, u >= 1 the block F to its right), the diagonal
// block D (symmetric, both triangles) and the block E below it, all in
// registers.  Sums over t (F^T v) are butterfly reduce-scatters inside a warp,
// plus one shared-memory add when a row range spans two warps; sums over u
// (D v, E v) are per-thread partials added across the NG column groups in
// shared memory.  The block E of step k is [x | F] of step k + 1 (same rows,
// columns shifted by b), so it stays in the same registers and step k + 1
// writes it back.
template <class T, int C, int W>
__device__ __forceinline__ T sb_reduce_scatter(T (&v)[C], int lane, int* idx) {
  constexpr int LOGC = (C >= 16) ? 4 : (C >= 8) ? 3 : (C >= 4) ? 2 : (C >= 2) ? 1 : 0;
  static_assert((1 << LOGC) == C && 2 * C <= W, "column count per thread");
  int base = 0;
#pragma unroll
  for (int j = 0; j < LOGC; ++j) {
    const int half = C >> (j + 1);
    const int o = W >> (j + 1);
    const bool up = (lane & o) != 0;
#pragma unroll
    for (int q = 0; q < C / 2; ++q) {
      if (q < half) {
        const T send = up ? v[q] : v[q + half];
        const T keep = up ? v[q + half] : v[q];
        v[q] = keep + __shfl_xor_sync(0xffffffffu, send, o);
      }
    }
    if (up) base += half;
  }
  T r = v[0];
#pragma unroll
  for (int o = W / (2 * C); o >= 1; o /= 2) r += __shfl_xor_sync(0xffffffffu, r, o);
  *idx = base;
  return r;
}

template <int B, int NG>
struct SbShape {
  static constexpr int C = B / NG;                       // columns per thread
  static constexpr int NT = (B * NG < 32) ? 32 : B * NG;  // threads
  static constexpr int W = (B < 32) ? B : 32;            // lanes of one row range in a warp
  static constexpr int H = B / W;                        // warps one row range spans
  static constexpr int NW = NT / 32;
};

template <class T, int B, int NG>
__global__ void __launch_bounds__(SbShape<B, NG>::NT) sb2st_kernel(SbArgs<T> a) {
  using Sh = SbShape<B, NG>;
  constexpr int C = Sh::C, W = Sh::W, H = Sh::H, NW = Sh::NW, LDS = B + 1;
  __shared__ T Ds[B * LDS];     // transpose of D's lower triangle
  __shared__ T xs[B];           // the column x
  __shared__ T red_p[NG][B], red_e[NG][B];
  __shared__ T wpart[H][B];
  __shared__ T kpart[NW];
  __shared__ T wfull[B], eyfull[B], wqfull[B];  // w = p - K v, tau E v, tau F^T v
  __shared__ double s_hh[3];    // beta, tau, 1 / v0
  __shared__ int s_abort;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const bool active = tid < B * NG;
  const int t = tid % B, g = active ? tid / B : 0;
  const int64_t n = a.n;
  constexpr int ldb = 2 * B;
  T* band = a.band;
#define BAND(i, j) band[((i) - (j)) + (int64_t)(j) * ldb]

  T XF[C];
  for (int64_t s = blockIdx.x; s < n - 1; s += gridDim.x) {
    const int64_t ns = sb_nsteps(s, n, B);
    const int64_t ns_prev = (s > 0) ? sb_nsteps(s - 1, n, B) : 0;
    for (int64_t k = 0; k < ns; ++k) {
      // ---- wait for sweep s-1 to have completed step k+1 and published
      // the beta of step k+2 ----
      if (tid == 0) {
        int ok = 1;
        if (s > 0) {
          const int64_t need = (k + 2 < ns_prev) ? k + 2 : ns_prev;
          const int64_t need_b = (k + 3 < ns_prev) ? k + 3 : ns_prev;
          const long long t0 = clock64();
          while (ld_acquire_gpu(a.progress + (s - 1)) < need || ld_acquire_gpu(a.beta_progress + (s - 1)) < need_b) {
            if (*(volatile int32_t*)a.status != 0) { ok = 0; break; }
            if (clock64() - t0 > a.limit) {
              raise_status(a.status, FRACLAP_ERR_TIMEOUT);
              ok = 0;
              break;
            }
            __nanosleep(32);
          }
        }
        s_abort = !ok;
      }
      __syncthreads();
      if (s_abort) return;

      const int64_t r0 = s + 1 + k * B;
      const int L = (int)((n - r0 < B) ? n - r0 : B);
      const int64_t r1 = r0 + L - 1;
      const int64_t c = (k == 0) ? s : r0 - B;
      const int nf = (int)(r0 - 1 - c);  // 0 at step 0, b - 1 after
      const int Lb = (int)((n - 1 - r1 < B) ? n - 1 - r1 : B);

      // ---- load (all of a thread's loads in flight together) ----
      if (k == 0) {
#pragma unroll
        for (int i = 0; i < C; ++i) XF[i] = T(0);
        if (active && g == 0 && t < L) XF[0] = __ldcg(&BAND(r0 + t, c));
      }
      T Dr[C], Er[C];
#pragma unroll
      for (int i = 0; i < C; ++i) {
        const int u = g + NG * i;
        Dr[i] = (active && t < L && u <= t) ? __ldcg(&BAND(r0 + t, r0 + u)) : T(0);
        Er[i] = (active && t < Lb && u < L) ? __ldcg(&BAND(r1 + 1 + t, r0 + u)) : T(0);
      }
#pragma unroll
      for (int i = 0; i < C; ++i) {
        const int u = g + NG * i;
        if (active && u <= t) Ds[u + t * LDS] = Dr[i];
      }
      if (active && g == 0) xs[t] = XF[0];
      __syncthreads();
      // ---- Householder scalars (warp 0; norms in FP64) ----
      if (warp == 0) {
        double tail = 0.0;
        for (int j = 1 + lane; j < B; j += 32) tail += (double)xs[j] * (double)xs[j];
        tail = warp_sum(tail);
        if (lane == 0) {
          const double x0 = (double)xs[0];
          double beta = x0, v0 = 1.0, tu = 0.0;
          if (tail > 0.0) {
            const double alpha = sqrt(x0 * x0 + tail);
            beta = (x0 >= 0.0) ? -alpha : alpha;
            v0 = x0 - beta;
            tu = (beta - x0) / beta;
          }
          s_hh[0] = beta;
          s_hh[1] = tu;
          s_hh[2] = (tu == 0.0) ? 0.0 : 1.0 / v0;
          // the entry sweep s+1 reads at step k-2: published now, not at the
          // end of the step (the store below writes the same value again)
          __stcg(&BAND(r0, c), (T)beta);
          st_release_gpu(a.beta_progress + s, (int)(k + 1));
        }
      }
#pragma unroll
      for (int i = 0; i < C; ++i) {
        const int u = g + NG * i;
        if (active && u > t) Dr[i] = Ds[t + u * LDS];  // upper triangle from the transpose
      }
      __syncthreads();
      const double tu = s_hh[1];
      const T inv = (T)s_hh[2];
      const T vt = (t == 0) ? T(1) : xs[t] * inv;  // v, with v(0) = 1
      T vu[C];
#pragma unroll
      for (int i = 0; i < C; ++i) {
        const int u = g + NG * i;
        vu[i] = (u == 0) ? T(1) : xs[u] * inv;
      }
      if (active && g == 0) a.refl[((int64_t)s * a.kmax + k) * B + t] = vt;
      if (tid == 0) a.rtau[s * a.kmax + k] = tu;
      // ---- partial sums: F^T v (over rows), D v and E v (over columns), v^T D v ----
      {
        T pv[C];
#pragma unroll
        for (int i = 0; i < C; ++i) pv[i] = vt * XF[i];
        int idx;
        const T cs = sb_reduce_scatter<T, C, W>(pv, lane, &idx);
        if (active && (lane & (W / C - 1)) == 0) wpart[(t / W) % H][g + NG * idx] = cs;
      }
      T pp = T(0), ep = T(0);
#pragma unroll
      for (int i = 0; i < C; ++i) {
        pp += Dr[i] * vu[i];
        ep += Er[i] * vu[i];
      }
      if (active) {
        red_p[g][t] = pp;
        red_e[g][t] = ep;
      }
      {
        T kk = active ? vt * pp : T(0);
#pragma unroll
        for (int o = 16; o >= 1; o /= 2) kk += __shfl_xor_sync(0xffffffffu, kk, o);
        if (lane == 0) kpart[warp] = kk;
      }
      __syncthreads();
      // ---- full sums, once per row / column ----
      if (tid < B) {
        const T tuT = (T)tu;
        T ksum = T(0);
#pragma unroll
        for (int q = 0; q < NW; ++q) ksum += kpart[q];
        const T K = T(0.5) * tuT * tuT * ksum;  // tau/2 p^T v with p = tau D v
        const T vj = (tid == 0) ? T(1) : xs[tid] * inv;
        T ps = T(0), es = T(0), cs = T(0);
#pragma unroll
        for (int q = 0; q < NG; ++q) {
          ps += red_p[q][tid];
          es += red_e[q][tid];
        }
#pragma unroll
        for (int h = 0; h < H; ++h) cs += wpart[h][tid];
        wfull[tid] = tuT * ps - K * vj;
        eyfull[tid] = tuT * es;
        wqfull[tid] = tuT * cs;
      }
      __syncthreads();
      // ---- rank-one and rank-two updates in registers ----
      const T wt = wfull[t], eyt = eyfull[t];
#pragma unroll
      for (int i = 0; i < C; ++i) {
        const int u = g + NG * i;
        XF[i] -= vt * wqfull[u];
        if (u <= t) Dr[i] -= vt * wfull[u] + wt * vu[i];  // only the stored triangle
        Er[i] -= eyt * vu[i];
      }
      // ---- store x (annihilated), F and D's lower triangle; E moves on ----
      if (active && t < L) {
        const T beta = (T)s_hh[0];
#pragma unroll
        for (int i = 0; i < C; ++i) {
          const int u = g + NG * i;
          if (u == 0) __stcg(&BAND(r0 + t, c), (t == 0) ? beta : T(0));
          else if (u <= nf) __stcg(&BAND(r0 + t, c + u), XF[i]);
          if (u <= t) __stcg(&BAND(r0 + t, r0 + u), Dr[i]);
        }
      }
#pragma unroll
      for (int i = 0; i < C; ++i) XF[i] = Er[i];
      __syncthreads();
      if (tid == 0) st_release_gpu(a.progress + s, (int)(k + 1));  // orders the CTA's stores (after the barrier)
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
// Every CTA streams all the reflectors through its shared memory, so the
// CTA's warp count W sets the L2 traffic per column: 16 warps per CTA (one
// CTA per SM) halve it against 8 (two per SM), which matters once the
// columns fill the SMs (at n = 8810 in FP32, 68 against 93 ms for the
// kernel alone); with few columns, 8-warp CTAs spread over more SMs.
template <class T, int B, int P, int W>
__global__ void __launch_bounds__(W * 32, 16 / W)
q2t_apply_kernel(const T* __restrict__ refl, const double* __restrict__ rtau, int64_t n,
                 int64_t kmax, T* Y, int64_t ldy, int64_t ncols) {
  // D = R: a batch of D reflectors slides the window by one full register
  // rotation, and the sweep is padded with zero reflectors (tau = 0) to whole
  // batches, so every slide is unconditional and compiles to renaming.
  constexpr int Q2T_WARPS = W;
  constexpr int R = B / P, CPW = 32 / P, D = R, NT = Q2T_WARPS * 32;
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
        const T* v = &vbuf[buf][j][part * R];  // zero (with tau 0) past s = 0
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
        {  // slide the window up by one row (rows above 1 + kB enter as zeros and are never written)
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
      if (active && row < n && row >= 1 + k * B) yc[row * ldy] = w[i];
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
  s->progress = ar->take<int>(2 * (n + 1));  // completed steps, then published betas
  return 0;
}

template <class T, int B, int NG>
int sb2st_launch(fraclap_ctx* ctx, SbArgs<T> a, cudaStream_t st) {
  constexpr int NT = SbShape<B, NG>::NT;
  int per_sm = 0;
  FL_CUDA(ctx, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, sb2st_kernel<T, B, NG>, NT, 0));
  FL_CHECK(ctx, per_sm >= 1, FRACLAP_ERR_UNSUPPORTED, "sb2st: kernel does not fit on an SM");
  int64_t G = (int64_t)ctx->sm_count * per_sm;
  if (G > a.n - 1) G = a.n - 1;
  void* args[] = {&a};
  count_launch(ctx);
  FL_CUDA(ctx, cudaLaunchCooperativeKernel((void*)sb2st_kernel<T, B, NG>, dim3((unsigned)G), dim3(NT), args, 0, st));
  return 0;
}

template <class T>
int sb2st_run(fraclap_ctx* ctx, T* band, int64_t n, int b, double* d, double* e, Stage2T<T>* s,
              cudaStream_t st) {
  if (n >= 2) {
    FL_CUDA(ctx, cudaMemsetAsync(s->progress, 0, sizeof(int) * 2 * (n + 1), st));
    FL_CUDA(ctx, cudaMemsetAsync(s->rtau, 0, sizeof(double) * (n - 1) * s->kmax, st));
    SbArgs<T> a{band, n, b, s->kmax, s->refl, s->rtau, s->progress, s->progress + (n + 1), ctx->d_status,
                ctx->wait_cycles};
    int rc = 0;
    switch (b) {
      case 4: rc = sb2st_launch<T, 4, 4>(ctx, a, st); break;
      case 8: rc = sb2st_launch<T, 8, 4>(ctx, a, st); break;
      case 16: rc = sb2st_launch<T, 16, 4>(ctx, a, st); break;
      case 32: rc = sb2st_launch<T, 32, 4>(ctx, a, st); break;
      case 64: rc = sb2st_launch<T, 64, 4>(ctx, a, st); break;
      default: FL_CHECK(ctx, false, FRACLAP_ERR_UNSUPPORTED, "sb2st: band width %d", b);
    }
    if (rc) return rc;
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
  // parts per window at b = 64: 4 (16 rows per lane, 8 columns per warp),
  // 8 or 16 (fewer rows per lane, more warps over the same columns: the
  // kernel has ncols / (32 / P) warps in all, so small P leaves SMs idle).
  // Default 8: at n = 8810 in FP32 (8-warp CTAs) 123 ms against 140 (P = 4)
  // and 247 (P = 16, a barrier every four reflectors).
  const int parts64 = (ctx->q2_parts == 4 || ctx->q2_parts == 16) ? ctx->q2_parts : 8;
  // 16-warp CTAs once 8-warp CTAs would already cover every SM
  const auto wide = [&](int pp) { return cdiv(ncols, (int64_t)(32 / pp) * 8) >= ctx->sm_count; };
#define FL_Q2T_W(BB, PP, WW)                                                                         \
  {                                                                                                  \
    cpw = 32 / PP;                                                                                   \
    const int64_t grid = cdiv(ncols, (int64_t)cpw * WW);                                             \
    q2t_apply_kernel<T, BB, PP, WW><<<(unsigned)grid, WW * 32, 0, st>>>(s->refl, s->rtau, n, s->kmax, \
                                                                       Yt, ldy, ncols);              \
    count_launch(ctx);                                                                               \
  }
#define FL_Q2T(BB, PP)                    \
  if (b == BB && cpw == 0) {              \
    if (BB == 64 && wide(PP))             \
      FL_Q2T_W(BB, PP, 16)                \
    else                                  \
      FL_Q2T_W(BB, PP, 8)                 \
  }
  FL_Q2T(4, 1)
  FL_Q2T(8, 2)
  FL_Q2T(16, 4)
  FL_Q2T(32, 8)
  if (b == 64) {
    if constexpr (sizeof(T) == 4) {  // FP64 windows of 16 rows would not fit the registers
      if (parts64 == 4) FL_Q2T(64, 4)
    }
    if (parts64 == 8) FL_Q2T(64, 8)
    if (parts64 == 16) FL_Q2T(64, 16)
    if (parts64 == 4) FL_Q2T(64, 8)  // FP64 asked for 4 parts: 8
  }
#undef FL_Q2T
#undef FL_Q2T_W
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
