// Symmetric tridiagonal eigensolver by divide and conquer (Cuppen's split
// with Gu-Eisenstat eigenvector reconstruction), FP64 throughout.
//
// Tree: 2^L leaves of at most `leaf_size` rows, leaf i = [lb(i), lb(i+1)) with
// lb(i) = i n / 2^L; every leaf boundary is the split point of one merge.
// At split point p the coupling beta = e(p-1) is removed from T:
//   T = diag(T1', T2') + beta w w^T,  w = e_{p-1} + e_p,
// T1' and T2' having beta subtracted from their touching diagonal entries.
// Leaves: one warp each, implicit QR with a Wilkinson shift (lane = row of
// the eigenvector block).  Merge of (Q1, L1), (Q2, L2):
//   D + rho z z^T, D = diag(L1, L2), z = (last row of Q1, first row of Q2),
// solved level by level for all merges of a level at once:
//   prep (one CTA per merge): sign flip for rho < 0, normalisation of z,
//     merge of the two sorted spectra, deflation of small |z_i| and of close
//     pairs (Givens rotations), compaction of the K surviving entries;
//   gather: Q columns in sorted order, rotations applied per row;
//   secular: one thread per root of 1 + rho sum z_j^2/(d_j - x) = 0, solved
//     in shifted coordinates x = d_org + tau (org = nearer pole) by a
//     two-pole rational model with bisection safeguard;
//   Gu-Eisenstat: z recomputed from the roots (orthogonal vectors);
//   vectors: U(j, i) = zhat_j / (d_j - lambda_i), normalised;
//   GEMM: Q_new = Q_sorted(:, kept) U  (batched, device-side descriptors);
//   finalise: deflated and new eigenvalues merged into ascending order.
#include "internal.cuh"

namespace fraclap {
namespace {

constexpr double kEps = 2.220446049250313e-16;

__host__ __device__ __forceinline__ int64_t leaf_bound(int64_t i, int64_t n, int L) {
  return (i * n) >> L;
}

struct MergeInfo {
  int64_t lo, mid, hi;
  double rho;   // > 0 after the sign flip and normalisation
  double sign;  // +1, or -1 when the merge was solved for -(D + rho z z^T)
  int64_t K;    // surviving (non-deflated) count
  int64_t nrot; // rotations recorded
};

template <class T>
struct DcBuf {
  double* D;      // n: working diagonal (beta subtracted at split points)
  double* Dp;     // n: sorted (signed) D of the merge
  double* zp;     // n: z in sorted order
  int* perm;      // n: sorted position -> local column
  int* kept;      // n: [lo, lo+K): sorted positions of survivors; [lo+K, hi): deflated
  double* dd;     // n: survivors' D
  double* zz;     // n: survivors' z
  T* ddt;         // n: survivors' D in the working precision (secular equation)
  T* zzt;         // n: survivors' z in the working precision
  double* tau;    // n: root offsets
  int* org;       // n: root origins (index into dd)
  double* zhat;   // n
  int* rot_i;     // n: rotation pairs (sorted positions)
  int* rot_j;
  double* rot_c;
  double* rot_s;
  int* outsrc;    // n: final column -> source (>= 0: new column i; < 0: -1 - deflated sorted pos)
  double* outval; // n: final eigenvalues
  MergeInfo* info;  // per merge
  GemmDescT<T>* desc;  // per merge
  T* Wq;          // gathered Q, n_m x n_m per merge
  T* Qnd;         // survivors' columns, n_m x K
  T* U;           // K x K (ld n_m)
  T* G;           // n_m x K (ld n_m)
};

// ----------------------------------------------------------------------------
__global__ void dc_setup(const double* d, const double* e, int64_t n, int L, double* D) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  // is index p a split point (a leaf boundary lb(m), 0 < m < 2^L)?
  auto is_split = [&](int64_t p) -> bool {
    if (p <= 0 || p >= n) return false;
    // smallest m with lb(m) >= p
    int64_t m = ((p << L) + n - 1) / n;
    return leaf_bound(m, n, L) == p && m > 0 && m < ((int64_t)1 << L);
  };
  double v = d[i];
  if (is_split(i + 1)) v -= e[i];
  if (is_split(i)) v -= e[i - 1];
  D[i] = v;
}

// One warp per leaf; leaf size <= 32.
template <class T>
__global__ void dc_leaf(const double* D, const double* e, int64_t n, int L, double* lambda,
                        T* Z, int64_t ldz, int32_t* status) {
  __shared__ double sd[4][32], se[4][32], sc[4][32], ss[4][32];
  __shared__ double sz[4][32][33];
  __shared__ int sperm[4][32];
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t leaf = (int64_t)blockIdx.x * 4 + w;
  if (leaf >= ((int64_t)1 << L)) return;
  const int64_t lo = leaf_bound(leaf, n, L), hi = leaf_bound(leaf + 1, n, L);
  const int m = (int)(hi - lo);
  if (m <= 0) return;
  double* d = sd[w];
  double* ee = se[w];
  if (lane < m) {
    d[lane] = D[lo + lane];
    ee[lane] = (lane + 1 < m) ? e[lo + lane] : 0.0;
  }
  for (int c = 0; c < m; ++c) sz[w][lane][c] = (lane == c) ? 1.0 : 0.0;
  __syncwarp();
  // implicit QR sweeps; lane 0 runs the scalar recurrence, all lanes rotate their row
  int steps = 0;
  int hi_i = m - 1;
  while (true) {
    int l = 0, hh = 0, go = 0;
    if (lane == 0) {
      while (hi_i > 0) {
        const double t = fabs(ee[hi_i - 1]);
        if (t <= 0.5 * kEps * (fabs(d[hi_i - 1]) + fabs(d[hi_i])) || t == 0.0) {
          ee[hi_i - 1] = 0.0;
          --hi_i;
        } else {
          break;
        }
      }
      if (hi_i > 0) {
        l = hi_i - 1;
        while (l > 0) {
          const double t = fabs(ee[l - 1]);
          if (t <= 0.5 * kEps * (fabs(d[l - 1]) + fabs(d[l])) || t == 0.0) break;
          --l;
        }
        if (l > 0) ee[l - 1] = 0.0;
        if (++steps > 30 * m + 30) {
          raise_status(status, FRACLAP_ERR_NO_CONVERGENCE);
        } else {
          const double a = d[hi_i - 1], bb = ee[hi_i - 1], c = d[hi_i];
          const double delta = 0.5 * (a - c);
          const double rr = hypot(delta, bb);
          const double mu = c - bb * bb / (delta + (delta >= 0.0 ? rr : -rr));
          double x = d[l] - mu, z = ee[l];
          for (int k = l; k < hi_i; ++k) {
            const double r = hypot(x, z);
            double cc = 1.0, sn = 0.0;
            if (r != 0.0) { cc = x / r; sn = z / r; }
            if (k > l) ee[k - 1] = r;
            const double dk = d[k], dk1 = d[k + 1], ek = ee[k];
            d[k] = cc * cc * dk + 2.0 * cc * sn * ek + sn * sn * dk1;
            d[k + 1] = sn * sn * dk - 2.0 * cc * sn * ek + cc * cc * dk1;
            ee[k] = cc * sn * (dk1 - dk) + (cc * cc - sn * sn) * ek;
            sc[w][k] = cc;
            ss[w][k] = sn;
            if (k + 1 < hi_i) {
              x = ee[k];
              z = sn * ee[k + 1];
              ee[k + 1] = cc * ee[k + 1];
            }
          }
          go = 1;
        }
      }
      hh = hi_i;
    }
    go = __shfl_sync(0xffffffffu, go, 0);
    l = __shfl_sync(0xffffffffu, l, 0);
    hh = __shfl_sync(0xffffffffu, hh, 0);
    __syncwarp();
    if (!go) break;
    if (lane < m)
      for (int k = l; k < hh; ++k) {
        const double cc = sc[w][k], sn = ss[w][k];
        const double za = sz[w][lane][k], zb = sz[w][lane][k + 1];
        sz[w][lane][k] = cc * za + sn * zb;
        sz[w][lane][k + 1] = -sn * za + cc * zb;
      }
    __syncwarp();
  }
  // ascending order
  if (lane == 0) {
    for (int i = 0; i < m; ++i) sperm[w][i] = i;
    for (int i = 0; i + 1 < m; ++i) {
      int kmin = i;
      for (int j = i + 1; j < m; ++j)
        if (d[sperm[w][j]] < d[sperm[w][kmin]]) kmin = j;
      const int t = sperm[w][i];
      sperm[w][i] = sperm[w][kmin];
      sperm[w][kmin] = t;
    }
  }
  __syncwarp();
  if (lane < m) {
    lambda[lo + lane] = d[sperm[w][lane]];
    for (int c = 0; c < m; ++c) Z[(lo + lane) + (lo + c) * ldz] = (T)sz[w][lane][sperm[w][c]];
  }
}

// ----------------------------------------------------------------------------
// Merge preparation: one CTA (128 threads) per merge; only the deflation by
// rotations between consecutive survivors runs on one thread.
template <class T>
__global__ void dc_merge_prep(DcBuf<T> B, const double* e, const double* lambda, const T* Z,
                              int64_t ldz, int64_t n, int L, int level, int64_t nmax) {
  const int64_t j = blockIdx.x;
  const int64_t span = (int64_t)1 << level;
  const int64_t lo = leaf_bound(j * span, n, L), hi = leaf_bound((j + 1) * span, n, L);
  const int64_t mid = leaf_bound(j * span + span / 2, n, L);
  const int64_t nm = hi - lo, n1 = mid - lo;
  MergeInfo* inf = B.info + j;
  __shared__ double s_red[32];
  __shared__ int64_t s_cnt[129];
  __shared__ int64_t s_nrot;
  const int tid = threadIdx.x, nt = blockDim.x;  // nt = 128
  // z and D in original local order (scratch: zhat and outval regions)
  double* zloc = B.zhat + lo;
  double* dloc = B.outval + lo;
  const double beta = e[mid - 1];
  const double sgn = (beta < 0.0) ? -1.0 : 1.0;
  double part = 0.0;
  for (int64_t i = tid; i < nm; i += nt) {
    const double zv = (i < n1) ? (double)Z[(mid - 1) + (lo + i) * ldz] : (double)Z[mid + (lo + i) * ldz];
    zloc[i] = zv;
    dloc[i] = sgn * lambda[lo + i];
    part += zv * zv;
  }
  auto block_sum = [&](double v) -> double {
    v = warp_sum(v);
    __syncthreads();
    if ((tid & 31) == 0) s_red[tid >> 5] = v;
    __syncthreads();
    double t = 0.0;
    for (int w = 0; w < nt / 32; ++w) t += s_red[w];
    return t;
  };
  const double nz2 = block_sum(part);
  const double rho = fabs(beta) * nz2;
  const double inv = 1.0 / sqrt(nz2);
  // merge the two sorted runs (descending when sgn < 0) by merge path: output
  // o takes a elements from run A before it, a the smallest with
  // A(a) > B(o - 1 - a); ties go to A first, as in a sequential merge
  double* Dp = B.Dp + lo;
  double* zp = B.zp + lo;
  int* perm = B.perm + lo;
  const int64_t n2 = nm - n1;
  auto ia = [&](int64_t i) -> int64_t { return (sgn > 0) ? i : n1 - 1 - i; };
  auto ib = [&](int64_t i) -> int64_t { return (sgn > 0) ? n1 + i : nm - 1 - i; };
  for (int64_t o = tid; o < nm; o += nt) {
    int64_t l = (o - n2 > 0) ? o - n2 : 0, h = (o < n1) ? o : n1;
    while (l < h) {
      const int64_t md = (l + h) >> 1;
      // A(md) > B(o - 1 - md)?  (o - 1 - md < n2 holds for md >= o - n2)
      if (dloc[ia(md)] > dloc[ib(o - 1 - md)]) h = md;
      else l = md + 1;
    }
    const int64_t ac = l, bc = o - l;
    const bool take_a = ac < n1 && (bc >= n2 || dloc[ia(ac)] <= dloc[ib(bc)]);
    const int64_t src = take_a ? ia(ac) : ib(bc);
    Dp[o] = dloc[src];
    zp[o] = zloc[src] * inv;
    perm[o] = (int)src;
  }
  __syncthreads();
  // deflation tolerance and flags (1 = deflated)
  double dm = 0.0;
  for (int64_t i = tid; i < nm; i += nt) dm = fmax(dm, fabs(Dp[i]));
  for (int o = 16; o >= 1; o >>= 1) dm = fmax(dm, __shfl_xor_sync(0xffffffffu, dm, o));
  __syncthreads();
  if ((tid & 31) == 0) s_red[tid >> 5] = dm;
  __syncthreads();
  double dmax = 0.0;
  for (int w = 0; w < nt / 32; ++w) dmax = fmax(dmax, s_red[w]);
  // deflation at the working precision's rounding level (FP32 merges
  // deflate at 8 eps_32: their results are only FP32-accurate anyway)
  const double eps_t = (sizeof(T) == 4) ? 1.1920928955078125e-07 : kEps;
  const double tol = 8.0 * eps_t * fmax(dmax, rho);
  int* kept = B.kept + lo;
  int* flag = B.outsrc + lo;  // scratch
  for (int64_t i = tid; i < nm; i += nt) flag[i] = (rho * fabs(zp[i]) <= tol) ? 1 : 0;
  __syncthreads();
  // close poles: Givens rotations between consecutive survivors, in order.
  // Each survivor i is tested against the survivor before it; a rotation
  // deflates that one and changes z_i and D_i, so every later test depends
  // on the earlier ones.  Warp 0 takes 32 positions at a time, tests all
  // their pairs at once with the values as they stand, accepts the pairs
  // before the first rotation, applies that rotation (the same arithmetic
  // as a sequential pass) and restarts after it.
  if (tid < 32) {
    const int lane = tid;
    int64_t nrot = 0, cur = -1;  // cur: the last survivor so far
    double zc = 0.0, dc = 0.0;   // its current z and D
    int64_t base = 0;
    while (base < nm) {
      const int64_t pos = base + lane;
      const bool valid = pos < nm && !flag[pos];
      const double z = valid ? zp[pos] : 0.0, d = valid ? Dp[pos] : 0.0;
      const unsigned mask = __ballot_sync(0xffffffffu, valid);
      // the survivor before this lane's position: a lower lane, or cur
      const unsigned below = mask & ((1u << lane) - 1u);
      const int pl = below ? 31 - __clz(below) : -1;
      const double zq = __shfl_sync(0xffffffffu, z, pl < 0 ? 0 : pl);
      const double dq = __shfl_sync(0xffffffffu, d, pl < 0 ? 0 : pl);
      const bool has_pred = valid && (pl >= 0 || cur >= 0);
      const double zpr = (pl >= 0) ? zq : zc, dpr = (pl >= 0) ? dq : dc;
      bool rot = false;
      double r = 0.0, c = 0.0, sn = 0.0;
      if (has_pred) {
        r = hypot(zpr, z);
        c = z / r;
        sn = -zpr / r;
        rot = fabs((d - dpr) * c * sn) <= tol;
      }
      const unsigned rmask = __ballot_sync(0xffffffffu, rot);
      if (rmask == 0u) {  // no rotation among these pairs
        if (mask) {
          const int hl = 31 - __clz(mask);
          cur = base + hl;
          zc = __shfl_sync(0xffffffffu, z, hl);
          dc = __shfl_sync(0xffffffffu, d, hl);
        }
        base += 32;
        continue;
      }
      const int fl = __ffs(rmask) - 1;  // the first rotation: pair (its predecessor, base + fl)
      if (lane == fl) {
        const int64_t pv = (pl >= 0) ? base + pl : cur;
        zp[pos] = r;
        zp[pv] = 0.0;
        const double dp = dpr, dj = d;
        Dp[pv] = dp * c * c + dj * sn * sn;
        const double dnew = dp * sn * sn + dj * c * c;
        Dp[pos] = dnew;
        B.rot_i[lo + nrot] = (int)pv;
        B.rot_j[lo + nrot] = (int)pos;
        B.rot_c[lo + nrot] = c;
        B.rot_s[lo + nrot] = sn;
        flag[pv] = 1;
        zc = r;
        dc = dnew;
      }
      __syncwarp();
      zc = __shfl_sync(0xffffffffu, zc, fl);
      dc = __shfl_sync(0xffffffffu, dc, fl);
      cur = base + fl;
      ++nrot;
      base = base + fl + 1;
    }
    if (lane == 0) s_nrot = nrot;
  }
  __syncthreads();
  const int64_t nrot = s_nrot;
  // compaction: survivors first, then the deflated, each in order (block scan)
  const int64_t chunk = (nm + nt - 1) / nt;
  const int64_t c0 = tid * chunk, c1 = (c0 + chunk < nm) ? c0 + chunk : nm;
  int64_t mine = 0;
  for (int64_t i = c0; i < c1; ++i) mine += flag[i] ? 0 : 1;
  s_cnt[tid + 1] = mine;
  if (tid == 0) s_cnt[0] = 0;
  __syncthreads();
  if (tid == 0)
    for (int t = 1; t <= nt; ++t) s_cnt[t] += s_cnt[t - 1];
  __syncthreads();
  const int64_t K = s_cnt[nt];
  int64_t kk = s_cnt[tid], kd = K + (c0 - s_cnt[tid]);
  for (int64_t i = c0; i < c1; ++i) {
    if (!flag[i]) {
      kept[kk] = (int)i;
      // the poles and weights as the working precision holds them, so that
      // the roots (found in T) and the Gu-Eisenstat weights and vectors
      // (formed in FP64 from dd, zz) see the same secular equation
      B.ddt[lo + kk] = (T)Dp[i];
      B.zzt[lo + kk] = (T)zp[i];
      B.dd[lo + kk] = (double)(T)Dp[i];
      B.zz[lo + kk] = (double)(T)zp[i];
      ++kk;
    } else {
      kept[kd++] = (int)i;
    }
  }
  if (tid != 0) return;
  inf->lo = lo;
  inf->mid = mid;
  inf->hi = hi;
  inf->rho = rho;
  inf->sign = sgn;
  inf->K = K;
  inf->nrot = nrot;
  // GEMM descriptor: G = Qnd (nm x K) * U (K x K)
  const int64_t off = lo * nmax;
  GemmDescT<T> d{};
  d.M = nm; d.N = K; d.K = K;
  d.A = B.Qnd + off; d.lda = nm;
  d.B = B.U + off; d.ldb = nm;
  d.C = B.G + off; d.ldc = nm;
  d.A2 = nullptr; d.lda2 = 0; d.B2 = nullptr; d.ldb2 = 0; d.K2 = 0;
  d.alpha = 1.0; d.beta = 0.0;
  B.desc[j] = d;
}

// Gather Q columns into sorted order and apply the deflation rotations.
// grid: (ceil(nmax/128), nmerge); thread = row of the merge block.
template <class T>
__global__ void dc_gather(DcBuf<T> B, const T* Z, int64_t ldz, int64_t nmax) {
  const MergeInfo inf = B.info[blockIdx.y];
  const int64_t nm = inf.hi - inf.lo;
  const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= nm) return;
  const int64_t lo = inf.lo, n1 = inf.mid - inf.lo;
  T* Wq = B.Wq + lo * nmax;
  const int* perm = B.perm + lo;
  for (int64_t i = 0; i < nm; ++i) {
    const int64_t c = perm[i];
    // block-diagonal: row r of block 1 pairs with columns of block 1 only
    const bool same = (r < n1) == (c < n1);
    Wq[r + i * nm] = same ? Z[(lo + r) + (lo + c) * ldz] : T(0);
  }
  for (int64_t q = 0; q < inf.nrot; ++q) {
    const int64_t a = B.rot_i[lo + q], b = B.rot_j[lo + q];
    const double c = B.rot_c[lo + q], s = B.rot_s[lo + q];
    const double xa = Wq[r + a * nm], xb = Wq[r + b * nm];
    Wq[r + a * nm] = (T)(c * xa + s * xb);
    Wq[r + b * nm] = (T)(-s * xa + c * xb);
  }
}

// Secular equation 1 + rho sum_j z_j^2 / (d_j - lambda) = 0: one warp per
// root, the lanes splitting the sums over the poles (butterfly sums, so every
// lane holds the same totals and takes the same branches).  Root i lies in
// (d_i, d_{i+1}) (the last one in (d_{K-1}, d_{K-1} + rho |z|^2)); it is kept
// as an offset tau from its nearer pole d_org.  Each step fits the two
// neighbouring poles exactly and the rest by the tangent rational model, and
// a bisection bracket guards it.  The terms are formed in the merge's working
// precision T and summed in FP64.  Stop when |f| is at the rounding level of
// its terms (8 eps_T (1 + |psi| + |phi|): psi and phi are sums of terms of
// one sign), when the bracket has closed to the rounding level of tau, or
// when a step no longer moves tau.
__device__ __forceinline__ double warp_allsum(double v) {
#pragma unroll
  for (int o = 16; o >= 1; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

constexpr int kSecWarps = 4;  // roots per 128-thread block

template <class T>
__global__ void __launch_bounds__(32 * kSecWarps) dc_secular(DcBuf<T> B, int32_t* status) {
  const MergeInfo inf = B.info[blockIdx.y];
  const int64_t K = inf.K;
  const int lane = threadIdx.x & 31;
  const int64_t i = (int64_t)blockIdx.x * kSecWarps + (threadIdx.x >> 5);
  if (i >= K) return;  // warp-uniform
  const double eps = (sizeof(T) == 4) ? 1.1920928955078125e-07 : kEps;
  const T* dd = B.ddt + inf.lo;
  const T* zz = B.zzt + inf.lo;
  const double rho = inf.rho;
  T lo_t, hi_t;
  int64_t orgi;
  if (i < K - 1) {
    const T half = T(0.5) * (dd[i + 1] - dd[i]);
    double f = 0.0;
    for (int64_t j = lane; j < K; j += 32) f += (double)(zz[j] * zz[j] / ((dd[j] - dd[i]) - half));
    f = 1.0 + rho * warp_allsum(f);
    if (f >= 0.0) { orgi = i; lo_t = T(0); hi_t = half; }
    else { orgi = i + 1; lo_t = -half; hi_t = T(0); }
  } else {
    double s2 = 0.0;
    for (int64_t j = lane; j < K; j += 32) s2 += (double)zz[j] * (double)zz[j];
    orgi = i; lo_t = T(0); hi_t = (T)(rho * warp_allsum(s2));
  }
  const T dorg = dd[orgi];
  const T a = dd[i] - dorg;
  const T bpole = (i < K - 1) ? dd[i + 1] - dorg : T(0);
  T tau = T(0.5) * (lo_t + hi_t);
  int it = 0;
  for (; it < 200; ++it) {
    double psi = 0.0, phi = 0.0, dpsi = 0.0, dphi = 0.0;
    for (int64_t j = lane; j < K; j += 32) {
      const T den = (dd[j] - dorg) - tau;
      const T t = zz[j] * zz[j] / den;
      if (j <= i) { psi += (double)t; dpsi += (double)(t / den); }
      else { phi += (double)t; dphi += (double)(t / den); }
    }
    psi = rho * warp_allsum(psi);
    phi = rho * warp_allsum(phi);
    dpsi = rho * warp_allsum(dpsi);
    dphi = rho * warp_allsum(dphi);
    const double f = 1.0 + psi + phi;
    if (f > 0.0) hi_t = tau; else lo_t = tau;
    if (fabs(f) <= 8.0 * eps * (1.0 + fabs(psi) + fabs(phi))) break;
    if ((double)(hi_t - lo_t) <= 4.0 * eps * fmax(fabs((double)lo_t), fabs((double)hi_t))) break;
    double x;
    const double at = (double)a - (double)tau;
    if (i < K - 1) {
      const double bt = (double)bpole - (double)tau;
      const double q1 = dpsi * at * at, p1 = psi - dpsi * at;
      const double q2 = dphi * bt * bt, p2 = phi - dphi * bt;
      const double C = 1.0 + p1 + p2;
      // in x - tau: C (at - y)(bt - y) + q1 (bt - y) + q2 (at - y) = 0, y = x - tau
      const double A2 = C, B2 = -(C * (at + bt) + q1 + q2), C2 = C * at * bt + q1 * bt + q2 * at;
      double y = 0.5 * ((double)lo_t + (double)hi_t) - (double)tau;
      if (A2 == 0.0) {
        if (B2 != 0.0) y = -C2 / B2;
      } else {
        const double disc = fmax(B2 * B2 - 4.0 * A2 * C2, 0.0);
        const double sq = sqrt(disc);
        double r1, r2;
        if (B2 >= 0.0) {
          const double t = -B2 - sq;
          r1 = t / (2.0 * A2);
          r2 = (t != 0.0) ? 2.0 * C2 / t : r1;
        } else {
          const double t = -B2 + sq;
          r1 = 2.0 * C2 / t;
          r2 = t / (2.0 * A2);
        }
        const double lo_y = (double)lo_t - (double)tau, hi_y = (double)hi_t - (double)tau;
        if (r1 > lo_y && r1 < hi_y) y = r1;
        else if (r2 > lo_y && r2 < hi_y) y = r2;
      }
      x = (double)tau + y;
    } else {
      const double q1 = dpsi * at * at, p1 = psi - dpsi * at;
      const double C = 1.0 + p1 + phi;
      x = (C != 0.0) ? (double)tau + (at + q1 / C) : 0.5 * ((double)lo_t + (double)hi_t);
    }
    T xn = (T)x;
    if (!(xn > lo_t && xn < hi_t)) xn = T(0.5) * (lo_t + hi_t);
    const bool stalled = fabs((double)xn - (double)tau) <= 2.0 * eps * fabs((double)tau);
    tau = xn;
    if (stalled) break;
  }
  if (lane == 0) {
    if (it >= 200) raise_status(status, FRACLAP_ERR_NO_CONVERGENCE);
    B.tau[inf.lo + i] = (double)tau;
    B.org[inf.lo + i] = (int)orgi;
  }
}

// Gu-Eisenstat: zhat_i^2 = (lam_{K-1} - d_i)/rho * prod_{j<K-1} (lam_j - d_i)/(d_j' - d_i).
template <class T>
__global__ void dc_zhat(DcBuf<T> B) {
  const MergeInfo inf = B.info[blockIdx.y];
  const int64_t K = inf.K;
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= K) return;
  const double* dd = B.dd + inf.lo;
  const double* tau = B.tau + inf.lo;
  const int* org = B.org + inf.lo;
  double prod = ((dd[org[K - 1]] - dd[i]) + tau[K - 1]) / inf.rho;
  for (int64_t j = 0; j + 1 < K; ++j) {
    const double num = (dd[org[j]] - dd[i]) + tau[j];
    const double den = (j < i) ? dd[j] - dd[i] : dd[j + 1] - dd[i];
    prod *= num / den;
  }
  const double zi = B.zz[inf.lo + i];
  B.zhat[inf.lo + i] = copysign(sqrt(fmax(prod, 0.0)), zi);
}

// U(:, i) = zhat ./ (d - lambda_i), normalised; one CTA per (column, merge).
template <class T>
__global__ void dc_vectors(DcBuf<T> B, int64_t nmax) {
  const MergeInfo inf = B.info[blockIdx.y];
  const int64_t K = inf.K, i = blockIdx.x;
  if (i >= K) return;
  const int64_t nm = inf.hi - inf.lo;
  const double* dd = B.dd + inf.lo;
  const double* zh = B.zhat + inf.lo;
  const double t = B.tau[inf.lo + i];
  const double dorg = dd[B.org[inf.lo + i]];
  T* u = B.U + inf.lo * nmax + i * nm;
  double s = 0.0;
  for (int64_t j = threadIdx.x; j < K; j += blockDim.x) {
    const double v = zh[j] / ((dd[j] - dorg) - t);
    s += v * v;
  }
  __shared__ double red[32];
  s = warp_sum(s);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x < 32) {
    double v = (threadIdx.x < blockDim.x / 32) ? red[threadIdx.x] : 0.0;
    v = warp_sum(v);
    if (threadIdx.x == 0) red[0] = v;
  }
  __syncthreads();
  const double inv = 1.0 / sqrt(red[0]);
  for (int64_t j = threadIdx.x; j < K; j += blockDim.x)
    u[j] = (T)(zh[j] / ((dd[j] - dorg) - t) * inv);
}

// Qnd(:, q) = Wq(:, kept[q]) for survivors; grid (ceil(nmax/128), nmerge).
template <class T>
__global__ void dc_gather_kept(DcBuf<T> B, int64_t nmax) {
  const MergeInfo inf = B.info[blockIdx.y];
  const int64_t nm = inf.hi - inf.lo;
  const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= nm) return;
  const T* Wq = B.Wq + inf.lo * nmax;
  T* Q = B.Qnd + inf.lo * nmax;
  const int* kept = B.kept + inf.lo;
  for (int64_t q = 0; q < inf.K; ++q) Q[r + q * nm] = Wq[r + (int64_t)kept[q] * nm];
}

// Final ascending order of the merged spectrum (thread 0 per merge).
template <class T>
__global__ void dc_order(DcBuf<T> B) {
  if (threadIdx.x != 0) return;
  const MergeInfo inf = B.info[blockIdx.x];
  const int64_t lo = inf.lo, nm = inf.hi - inf.lo, K = inf.K, nd = nm - K;
  const int* kept = B.kept + lo;
  const double* Dp = B.Dp + lo;
  int* defl = B.perm + lo;  // perm no longer needed: sorted deflated positions
  for (int64_t q = 0; q < nd; ++q) defl[q] = kept[K + q];
  for (int64_t q = 1; q < nd; ++q) {  // insertion sort by value (nearly sorted)
    const int v = defl[q];
    int64_t p = q - 1;
    while (p >= 0 && Dp[defl[p]] > Dp[v]) { defl[p + 1] = defl[p]; --p; }
    defl[p + 1] = v;
  }
  const double* dd = B.dd + lo;
  const double* tau = B.tau + lo;
  const int* org = B.org + lo;
  int* out = B.outsrc + lo;
  double* val = B.outval + lo;
  int64_t a = 0, b = 0;
  for (int64_t o = 0; o < nm; ++o) {
    const double va = (a < K) ? dd[org[a]] + tau[a] : 0.0;
    const double vb = (b < nd) ? Dp[defl[b]] : 0.0;
    bool take_a = (b >= nd) || (a < K && va <= vb);
    // ascending in signed space; reversed when the merge was flipped
    const int64_t pos = (inf.sign > 0) ? o : nm - 1 - o;
    if (take_a) { out[pos] = (int)a; val[pos] = inf.sign * va; ++a; }
    else { out[pos] = -1 - defl[b]; val[pos] = inf.sign * vb; ++b; }
  }
}

// Z(lo:hi, lo + p) = chosen column; lambda(lo + p) = value.  grid (nmax, nmerge).
template <class T>
__global__ void dc_scatter(DcBuf<T> B, double* lambda, T* Z, int64_t ldz, int64_t nmax) {
  const MergeInfo inf = B.info[blockIdx.y];
  const int64_t nm = inf.hi - inf.lo, p = blockIdx.x;
  if (p >= nm) return;
  const int src = B.outsrc[inf.lo + p];
  const T* col = (src >= 0) ? B.G + inf.lo * nmax + (int64_t)src * nm
                            : B.Wq + inf.lo * nmax + (int64_t)(-1 - src) * nm;
  T* dst = Z + inf.lo + (inf.lo + p) * ldz;
  for (int64_t r = threadIdx.x; r < nm; r += blockDim.x) dst[r] = col[r];
  if (threadIdx.x == 0) lambda[inf.lo + p] = B.outval[inf.lo + p];
}

int tree_levels(int64_t n, int leaf) {
  int L = 0;
  while (cdiv(n, (int64_t)1 << L) > leaf) ++L;
  return L;
}

int64_t level_nmax(int64_t n, int L, int level) {
  int64_t mx = 0;
  const int64_t span = (int64_t)1 << level;
  for (int64_t j = 0; j < ((int64_t)1 << (L - level)); ++j) {
    const int64_t a = leaf_bound(j * span, n, L), b = leaf_bound((j + 1) * span, n, L);
    if (b - a > mx) mx = b - a;
  }
  return mx;
}

template <class T>
int take_bufs(Arena* ar, int64_t n, int L, DcBuf<T>* B) {
  B->D = ar->take<double>(n);
  B->Dp = ar->take<double>(n);
  B->zp = ar->take<double>(n);
  B->perm = ar->take<int>(n);
  B->kept = ar->take<int>(n);
  B->dd = ar->take<double>(n);
  B->zz = ar->take<double>(n);
  B->ddt = ar->take<T>(n);
  B->zzt = ar->take<T>(n);
  B->tau = ar->take<double>(n);
  B->org = ar->take<int>(n);
  B->zhat = ar->take<double>(n);
  B->rot_i = ar->take<int>(n);
  B->rot_j = ar->take<int>(n);
  B->rot_c = ar->take<double>(n);
  B->rot_s = ar->take<double>(n);
  B->outsrc = ar->take<int>(n);
  B->outval = ar->take<double>(n);
  const int64_t nmerge_max = (L >= 1) ? ((int64_t)1 << (L - 1)) : 1;
  B->info = ar->take<MergeInfo>(nmerge_max);
  B->desc = ar->take<GemmDescT<T>>(nmerge_max);
  // per-merge n_m x n_m blocks at offset lo * nmax (<= n * n in total + slack)
  const int64_t big = (n + 2) * n;
  B->Wq = ar->take<T>(big);
  B->Qnd = ar->take<T>(big);
  B->U = ar->take<T>(big);
  B->G = ar->take<T>(big);
  return 0;
}

}  // namespace

template <class T>
size_t stedc_ws(const fraclap_ctx* ctx, int64_t n) {
  Arena ar;
  DcBuf<T> B;
  take_bufs<T>(&ar, n, tree_levels(n, ctx->leaf_size), &B);
  return ar.off;
}

template <class T>
int stedc_run(fraclap_ctx* ctx, const double* d, const double* e, int64_t n, double* lambda, T* Z,
              int64_t ldz, Arena* ar, cudaStream_t st) {
  if (n <= 0) return 0;
  const int L = tree_levels(n, ctx->leaf_size);
  DcBuf<T> B;
  take_bufs<T>(ar, n, L, &B);
  FL_CHECK(ctx, B.G != nullptr, FRACLAP_ERR_ALLOC, "stedc: workspace too small");
  FL_CUDA(ctx, cudaMemset2DAsync(Z, ldz * sizeof(T), 0, n * sizeof(T), n, st));
  dc_setup<<<(unsigned)cdiv(n, 256), 256, 0, st>>>(d, e, n, L, B.D);
  count_launch(ctx);
  const int64_t nleaf = (int64_t)1 << L;
  dc_leaf<T><<<(unsigned)cdiv(nleaf, 4), 128, 0, st>>>(B.D, e, n, L, lambda, Z, ldz, ctx->d_status);
  count_launch(ctx);
  FL_CUDA(ctx, cudaGetLastError());
  for (int level = 1; level <= L; ++level) {
    const int64_t nmerge = (int64_t)1 << (L - level);
    const int64_t nmax = level_nmax(n, L, level);
    FL_CHECK(ctx, nmerge <= 65535 && nmax < (1LL << 31), FRACLAP_ERR_UNSUPPORTED, "stedc: too large");
    dc_merge_prep<T><<<(unsigned)nmerge, 128, 0, st>>>(B, e, lambda, Z, ldz, n, L, level, nmax);
    count_launch(ctx);
    const dim3 rows((unsigned)cdiv(nmax, 128), (unsigned)nmerge);
    dc_gather<T><<<rows, 128, 0, st>>>(B, Z, ldz, nmax);
    count_launch(ctx);
    dc_secular<T><<<dim3((unsigned)cdiv(nmax, kSecWarps), (unsigned)nmerge), 32 * kSecWarps, 0, st>>>(
        B, ctx->d_status);
    count_launch(ctx);
    dc_zhat<T><<<rows, 128, 0, st>>>(B);
    count_launch(ctx);
    dc_vectors<T><<<dim3((unsigned)nmax, (unsigned)nmerge), 128, 0, st>>>(B, nmax);
    count_launch(ctx);
    dc_gather_kept<T><<<rows, 128, 0, st>>>(B, nmax);
    count_launch(ctx);
    FL_CUDA(ctx, cudaGetLastError());
    FL_TRY(gemm_batched<T>(ctx, false, false, B.desc, (int)nmerge, nmax, nmax, st));
    dc_order<T><<<(unsigned)nmerge, 32, 0, st>>>(B);
    count_launch(ctx);
    dc_scatter<T><<<dim3((unsigned)nmax, (unsigned)nmerge), 128, 0, st>>>(B, lambda, Z, ldz, nmax);
    count_launch(ctx);
    FL_CUDA(ctx, cudaGetLastError());
  }
  return 0;
}

template size_t stedc_ws<double>(const fraclap_ctx*, int64_t);
template size_t stedc_ws<float>(const fraclap_ctx*, int64_t);
template int stedc_run<double>(fraclap_ctx*, const double*, const double*, int64_t, double*, double*, int64_t, Arena*, cudaStream_t);
template int stedc_run<float>(fraclap_ctx*, const double*, const double*, int64_t, double*, float*, int64_t, Arena*, cudaStream_t);

}  // namespace fraclap
