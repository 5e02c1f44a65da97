/*
 * fraclap — GB300 (sm_103a) library for the fractional Poisson problem
 * (-Laplacian)^{alpha/2} u = f with homogeneous Dirichlet conditions on
 * masked 2-D/3-D grids, by the eigenfunction-expansion method of
 * arXiv:1911.11906 (Carlson, Kirby, Sundar).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - All matrices are column-major IEEE double: a(i, j) = a[i + j * ld].
 *  - Pointers named *_dev are device pointers owned by the caller; the
 *    library never frees them and never copies to or from the host unless
 *    the entry point says so.  Outputs may not alias inputs unless stated.
 *  - Every call is asynchronous on the given stream (0 = legacy default
 *    stream) unless stated.  Device-side failures (an iteration cap, a wait
 *    that timed out, lambda <= 0 with alpha != 0) are recorded in a device
 *    status word of the context; fraclap_sync() waits for the stream and
 *    returns that status (and clears it).
 *  - Return values: FRACLAP_OK (0) or a negative FRACLAP_ERR_* code.
 *    fraclap_last_error() gives a message for the last failure of a context.
 *  - Workspace: an entry point that takes (work_dev, work_bytes) uses that
 *    caller-owned device buffer (at least the size the matching
 *    *_workspace_bytes query returns, 256-byte aligned); with work_dev == NULL
 *    it uses a buffer owned by the context, grown with cudaMalloc on demand.
 *  - One context serves one device; calls on one context must not overlap.
 */
#ifndef FRACLAP_H_
#define FRACLAP_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st* fraclap_stream_t; /* = cudaStream_t */
typedef struct fraclap_ctx fraclap_ctx;

enum {
  FRACLAP_OK = 0,
  FRACLAP_ERR_INVALID_ARG = -1,   /* a null pointer, a negative size, ld < rows, ... */
  FRACLAP_ERR_NOT_SPD = -2,       /* lambda_i <= 0 met with alpha != 0 in frac_apply */
  FRACLAP_ERR_NO_CONVERGENCE = -3,/* an eigen-iteration hit its cap */
  FRACLAP_ERR_TIMEOUT = -4,       /* a bounded device-side wait expired */
  FRACLAP_ERR_ALLOC = -5,         /* a context-owned workspace allocation failed */
  FRACLAP_ERR_CUDA = -6,          /* a CUDA runtime call failed (see fraclap_last_error) */
  FRACLAP_ERR_UNSUPPORTED = -7,   /* a size or option outside what this build handles */
  FRACLAP_ERR_IO = -8             /* a file could not be written or read, or is not a valid checkpoint */
};

/* Options; zero fields take the defaults in brackets. */
typedef struct fraclap_opts {
  int band_width;           /* half-bandwidth b of the dense-to-band stage [32]: 4, 8, 16, 32 or 64 */
  int leaf_size;            /* largest leaf of the tridiagonal divide and conquer [32]; 2..32 */
  double wait_timeout_s;    /* limit of every device-side spin wait in seconds [10] */
} fraclap_opts;

/* Creates a context on the current CUDA device.  opts may be NULL. */
int fraclap_create(fraclap_ctx** ctx, const fraclap_opts* opts);
void fraclap_destroy(fraclap_ctx* ctx);
const char* fraclap_strerror(int code);
const char* fraclap_last_error(const fraclap_ctx* ctx);
/* Waits for `stream`, then returns and clears the context's device status. */
int fraclap_sync(fraclap_ctx* ctx, fraclap_stream_t stream);

/* ------------------------------------------------------------------------
 * fd_assemble — the discrete Laplace operator of Sec. II, eq.
 * (discrete_laplace), with a nodal finite-difference basis: the mass matrix
 * is the identity and K is the 5-point (dim = 2) or 7-point (dim = 3)
 * Laplacian scaled by 1/h^2 with homogeneous Dirichlet conditions
 * (eq. continuous_eigenproblem): row i holds 2*dim/h^2 on the diagonal and
 * -1/h^2 for every face neighbour inside the mask, columns ascending.
 *
 *  mask_dev  uint8[ext0*ext1*ext2], x fastest then y then z; nonzero = dof.
 *  ext       host int64[3] = (nx, ny, nz); nz must be 1 when dim = 2.
 *  idx_dev   int32[ext0*ext1*ext2] out: dof number of each node, -1 outside;
 *            dofs are numbered in row-major order over the kept nodes.
 *  n_out, nnz_out  host out: number of dofs and of CSR nonzeros.
 *  rowptr_dev int64[n+1], col_dev int32[nnz], val_dev double[nnz]: CSR out.
 *  A_dense_dev double[lda*n]: optional dense copy of the matrix (zero
 *            elsewhere); lda >= n.
 * Two-call protocol: with rowptr_dev == NULL the call numbers the dofs,
 * writes idx_dev, and returns n and nnz (it synchronises `stream` to read
 * them).  A second call with the CSR buffers (and optionally A_dense_dev)
 * fills them; it reads idx_dev from the first call and is asynchronous.
 * ---------------------------------------------------------------------- */
int fd_assemble(fraclap_ctx* ctx, const uint8_t* mask_dev, int dim, const int64_t ext[3],
                double h, int32_t* idx_dev, int64_t* n_out, int64_t* nnz_out,
                int64_t* rowptr_dev, int32_t* col_dev, double* val_dev,
                double* A_dense_dev, int64_t lda, fraclap_stream_t stream);

/* ------------------------------------------------------------------------
 * eig_full — all n eigenpairs A = V diag(lambda) V^T of a dense symmetric
 * matrix (the "solve for all N eigenpairs once" step of Sec. II and
 * Sec. III-A), FP64 throughout.  Route: Householder reduction to a band of
 * half-width b (compact-WY panels, symmetric rank-2b trailing updates),
 * bulge chasing to tridiagonal form, tridiagonal divide and conquer, and
 * back-transformation by both orthogonal factors.
 *
 *  A_dev      double[lda*n], only the lower triangle is read; not modified.
 *  lambda_dev double[n] out, ascending.
 *  V_dev      double[ldv*n] out, orthonormal eigenvectors in columns (the
 *             sign of each column is unspecified); ldv >= n.
 *  work_dev / work_bytes: see fraclap_eig_workspace_bytes.
 *  info_dev   optional int32 out (device): 0, or a positive count of
 *             failures recorded on the device (also in the context status).
 * ---------------------------------------------------------------------- */
size_t fraclap_eig_workspace_bytes(const fraclap_ctx* ctx, int64_t n);
int eig_full(fraclap_ctx* ctx, const double* A_dev, int64_t n, int64_t lda,
             double* lambda_dev, double* V_dev, int64_t ldv, void* work_dev,
             size_t work_bytes, int32_t* info_dev, fraclap_stream_t stream);

/* ------------------------------------------------------------------------
 * eig_full_mixed — the same decomposition through the mixed-precision route:
 * the reduction to band form, the bulge chasing, the divide-and-conquer
 * eigenvector merges and both back-transformations run in FP32 (the FP32
 * pipe of GB300 is ~58x its FP64 pipe); the Householder norms and scalings,
 * the secular equations and the deflation stay FP64.  FP64 accuracy is then
 * regained by `refine_iters` iterations of Ogita-Aishima refinement
 * (R = I - V^T V and S = V^T A V in FP64 with A applied through its CSR
 * form, products on the tensor cores by error-free BF16 splitting; clusters
 * of close eigenvalues, and pairs whose first-order correction would be
 * large, are diagonalised exactly).  refine_iters is the maximum number of
 * iterations; the loop stops after the first iteration that starts with
 * ||I - V^T V||_2 and ||V^T A V - D||_2 / ||A||_2 below 3e-9.  FP32-accurate
 * starting vectors at n ~ 10^4 take three or four.
 *
 *  A_dev      double[lda*n] dense, lower triangle read (the FP32 stages).
 *  rowptr_dev, col_dev, val_dev: the same matrix in CSR (from fd_assemble).
 *  lambda_dev, V_dev: as eig_full.  n <= 65535.
 *  work: fraclap_eig_mixed_workspace_bytes(ctx, n) bytes.
 * ---------------------------------------------------------------------- */
size_t fraclap_eig_mixed_workspace_bytes(const fraclap_ctx* ctx, int64_t n);
int eig_full_mixed(fraclap_ctx* ctx, const double* A_dev, int64_t n, int64_t lda,
                   const int64_t* rowptr_dev, const int32_t* col_dev, const double* val_dev,
                   int refine_iters, double* lambda_dev, double* V_dev, int64_t ldv,
                   void* work_dev, size_t work_bytes, int32_t* info_dev, fraclap_stream_t stream);

/* ------------------------------------------------------------------------
 * frac_apply — the spectral solution operator of Sec. II,
 * eq. (poisson_solution) and the sum v after eq. (discrete_laplace):
 *   u_j = V diag(lambda^{-alpha_j / 2}) V^T f_{pair_f[j]},  j = 0..k-1.
 * alpha may be any real number; alpha < 0 applies the forward operator of
 * eq. (spectral_definition).  With alpha != 0 every lambda must be > 0, else
 * the device status becomes FRACLAP_ERR_NOT_SPD.
 *
 *  V_dev double[ldv*n], lambda_dev double[n]: a decomposition from eig_full.
 *  F_dev double[ldf*m]: m distinct forcings in columns; ldf >= n.
 *  pair_f_dev int32[k] (each in [0, m)), pair_alpha_dev double[k].
 *  U_dev double[ldu*k] out; ldu >= n.
 *  work: fraclap_apply_workspace_bytes(n, m, k) bytes (V^T F and the scaled
 *  coefficients).
 * ---------------------------------------------------------------------- */
size_t fraclap_apply_workspace_bytes(int64_t n, int64_t m, int64_t k);
/* The same for this context's setting of fraclap_set_apply_slices. */
size_t fraclap_apply_workspace_bytes_ctx(const fraclap_ctx* ctx, int64_t n, int64_t m, int64_t k);
/* Products of frac_apply: 0 (default) on the FP64 GEMM engine; s = 1..8 as
 * products of s BF16 slices on the tensor cores (error about 2^-8s relative
 * to |row max| |column max| per term; s = 7 is FP64-level, s = 5 about 1e-12). */
int fraclap_set_apply_slices(fraclap_ctx* ctx, int slices);
int frac_apply(fraclap_ctx* ctx, const double* V_dev, int64_t ldv, const double* lambda_dev,
               int64_t n, const double* F_dev, int64_t ldf, int64_t m,
               const int32_t* pair_f_dev, const double* pair_alpha_dev, int64_t k,
               double* U_dev, int64_t ldu, void* work_dev, size_t work_bytes,
               fraclap_stream_t stream);

/* ------------------------------------------------------------------------
 * frac_diffusion — the solution of the space-fractional diffusion equation
 * du/dt + mu (-Laplacian)^{alpha/2} u = 0 with homogeneous Dirichlet
 * conditions (Sec. II, eqs. model_diffusion and diffusion_solution): every
 * eigenmode decays at its own rate,
 *   u_j = V diag(exp(-mu lambda^{alpha_j / 2} t_j)) V^T u0_{pair_f[j]},  j = 0..k-1.
 * Pair j evolves initial state pair_f[j] with order pair_alpha[j] to time
 * pair_t[j] (any real t; t = 0 returns the initial state, alpha = 0 decays
 * every mode by exp(-mu t)).  With alpha != 0 every lambda must be > 0, else
 * the device status becomes FRACLAP_ERR_NOT_SPD; a pair index outside [0, m)
 * sets FRACLAP_ERR_INVALID_ARG there (its column is zero).
 *
 *  V_dev double[ldv*n], lambda_dev double[n]: a decomposition from eig_full.
 *  U0_dev double[ldu0*m]: m distinct initial states in columns; ldu0 >= n.
 *  pair_f_dev int32[k], pair_alpha_dev double[k], pair_t_dev double[k].
 *  mu: the diffusion coefficient, finite (else FRACLAP_ERR_INVALID_ARG).
 *  U_dev double[ldu*k] out; ldu >= n.
 *  work: fraclap_apply_workspace_bytes_ctx(ctx, n, m, k) bytes.  The products
 *  follow the context's fraclap_set_apply_slices setting, as in frac_apply.
 *  Returns FRACLAP_ERR_UNSUPPORTED for k > 65535; asynchronous on `stream`.
 * ---------------------------------------------------------------------- */
int frac_diffusion(fraclap_ctx* ctx, const double* V_dev, int64_t ldv, const double* lambda_dev,
                   int64_t n, const double* U0_dev, int64_t ldu0, int64_t m,
                   const int32_t* pair_f_dev, const double* pair_alpha_dev, const double* pair_t_dev,
                   double mu, int64_t k, double* U_dev, int64_t ldu, void* work_dev,
                   size_t work_bytes, fraclap_stream_t stream);

/* ------------------------------------------------------------------------
 * CUDA-graph form of the apply: frac_apply (pair_t_dev == NULL) or
 * frac_diffusion (pair_t_dev given, with mu) captured once, on a private
 * stream, into an instantiated CUDA graph, so that repeated solves with new
 * contents of the SAME buffers (new forcings in F_dev, new orders or times in
 * the pair arrays, a new decomposition in V_dev/lambda_dev) cost one graph
 * launch instead of the GEMM, scaling and slicing launches one by one.
 *
 *  Arguments as for frac_diffusion; the product route (FP64 or BF16 slices)
 *  is the context's setting at creation.  work_dev is REQUIRED (a
 *  caller-owned workspace of fraclap_apply_workspace_bytes_ctx bytes: the
 *  context's own may be reallocated by later calls).  The graph keeps every
 *  pointer it was created with: the buffers, the workspace and the context
 *  (its status word receives NOT_SPD / INVALID_ARG from a launch, read by
 *  fraclap_sync) must outlive it, and launches of one graph must not overlap.
 * fraclap_graph_launch: one replay on `stream` (asynchronous).
 * fraclap_graph_kernels: the number of kernels in the graph (-1 for NULL);
 *  each launch adds it to the context's launch count.
 * fraclap_graph_destroy: frees the graph (NULL is a no-op).
 * ---------------------------------------------------------------------- */
typedef struct fraclap_graph fraclap_graph;
int fraclap_apply_graph_create(fraclap_ctx* ctx, const double* V_dev, int64_t ldv,
                               const double* lambda_dev, int64_t n, const double* F_dev, int64_t ldf,
                               int64_t m, const int32_t* pair_f_dev, const double* pair_alpha_dev,
                               const double* pair_t_dev, double mu, int64_t k, double* U_dev,
                               int64_t ldu, void* work_dev, size_t work_bytes, fraclap_graph** out);
int fraclap_graph_launch(fraclap_graph* g, fraclap_stream_t stream);
long long fraclap_graph_kernels(const fraclap_graph* g);
void fraclap_graph_destroy(fraclap_graph* g);

/* ------------------------------------------------------------------------
 * frac_apply_noalloc —frac_apply for callers that cannot allocate device
 * memory.  The paper has no counterpart; this is a deployment variant.
 * It serves code that runs where cudaMalloc is not available to it: inside a
 * host framework whose memory pool already owns the device (an extra
 * allocation would fail or break its accounting), or in latency-critical
 * loops that cannot pay the implicit device synchronisation of
 * cudaMalloc/cudaFree.  It needs no context and allocates nothing: its
 * scratch (V^T F and the scaled coefficients) is a fixed array of
 * FRACLAP_NOALLOC_MAX_DOUBLES doubles (16 MiB) compiled into the library,
 * which every GPU that loads the library holds until the process exits.
 *
 *  Arguments as for frac_apply, without the context and workspace; the
 *  caller still owns every input and output.  status_dev: optional int32 on
 *  the device that receives FRACLAP_ERR_NOT_SPD (or INVALID_ARG for a pair
 *  index out of range) from the kernels; it is not cleared by the call.
 *  With status_dev == NULL those device-side errors are NOT reported: the
 *  kernels record them in a private word that nothing reads (the affected
 *  columns of U are still zeroed), so pass a status word whenever lambda or
 *  the pair indices are not known to be valid.
 *  Returns FRACLAP_ERR_UNSUPPORTED, launching nothing, when the scratch is
 *  too small: n*m rounded up to a multiple of 32, plus n*k, must not exceed
 *  FRACLAP_NOALLOC_MAX_DOUBLES, and k <= 65535.
 *  The first call on each device looks up the array's device address with
 *  cudaGetSymbolAddress (with that device current); make that first call
 *  before any stream capture.  All calls share the one array and it keeps
 *  the previous call's contents (every element used is rewritten before it
 *  is read): calls whose executions overlap on the GPU (different streams,
 *  or host threads without ordering) race on it.
 * ---------------------------------------------------------------------- */
#define FRACLAP_NOALLOC_MAX_DOUBLES (1 << 21)
int frac_apply_noalloc(const double* V_dev, int64_t ldv, const double* lambda_dev, int64_t n,
                       const double* F_dev, int64_t ldf, int64_t m, const int32_t* pair_f_dev,
                       const double* pair_alpha_dev, int64_t k, double* U_dev, int64_t ldu,
                       int32_t* status_dev, fraclap_stream_t stream);

/* ------------------------------------------------------------------------
 * Checkpoint of a decomposition.  The method computes the eigenpairs once
 * and reuses them for every forcing, order and time (Sec. II), so
 * (n, lambda, V) can be kept in a file, tagged with the grid it belongs to.
 * HOST buffers: these calls do file I/O only; the caller copies V to and from
 * the device.  The file is little-endian whatever the host, ends with an
 * FNV-1a-64 checksum of its contents, and is written to "<path>.partial" and
 * renamed, so a failed save never leaves a truncated checkpoint at `path`.
 *
 * fraclap_mask_hash: FNV-1a-64 of (dim, ext, h, mask bytes read as 0/1);
 *   mask_host uint8[ext0*ext1*(dim == 3 ? ext2 : 1)]; returns 0 for invalid
 *   arguments, never 0 otherwise.
 * fraclap_save_decomposition: lambda_host double[n], V_host double[ldv*n]
 *   (ldv >= n; stored packed); dim 2 or 3 with ext and h describing the grid,
 *   or dim 0 for none; mask_hash 0 = none.  FRACLAP_ERR_IO if the file cannot
 *   be written.
 * fraclap_load_decomposition: two calls.  With lambda_host == NULL it reads
 *   and checks the header (every out pointer may be NULL) and returns n, the
 *   grid and the stored mask hash; with lambda_host double[n] and V_host
 *   double[ldv*n] (ldv >= n) it also reads the payload.  FRACLAP_ERR_IO for a
 *   missing, truncated or corrupted file (bad magic, version, size or
 *   checksum; the buffers' contents are then unspecified);
 *   FRACLAP_ERR_INVALID_ARG if expect_mask_hash is nonzero and differs from
 *   the stored hash (the file belongs to another domain).
 * ---------------------------------------------------------------------- */
uint64_t fraclap_mask_hash(const uint8_t* mask_host, int dim, const int64_t ext[3], double h);
int fraclap_save_decomposition(const char* path, int64_t n, const double* lambda_host,
                               const double* V_host, int64_t ldv, int dim, const int64_t ext[3],
                               double h, uint64_t mask_hash);
int fraclap_load_decomposition(const char* path, int64_t* n_out, int* dim_out, int64_t ext_out[3],
                               double* h_out, uint64_t* mask_hash_out, double* lambda_host,
                               double* V_host, int64_t ldv, uint64_t expect_mask_hash);

/* ------------------------------------------------------------------------
 * Stage entry points (the steps eig_full chains), for stage-level checks.
 * ---------------------------------------------------------------------- */

/* Reduction to symmetric tridiagonal form A = Q T Q^T (dense to band, then
 * bulge chasing).  d_dev double[n], e_dev double[n-1] out (T(i+1, i) = e[i]).
 * Q_dev double[ldq*n]: optional (NULL = skip); when given, Q is formed by
 * back-transforming the identity.  work as for eig_full. */
int fraclap_tridiagonalize(fraclap_ctx* ctx, const double* A_dev, int64_t n, int64_t lda,
                           double* d_dev, double* e_dev, double* Q_dev, int64_t ldq,
                           void* work_dev, size_t work_bytes, fraclap_stream_t stream);

/* Eigen-decomposition of the symmetric tridiagonal (d, e) by divide and
 * conquer: lambda_dev double[n] ascending, Z_dev double[ldz*n] eigenvectors. */
size_t fraclap_tridiag_workspace_bytes(const fraclap_ctx* ctx, int64_t n);
int fraclap_tridiag_eig(fraclap_ctx* ctx, const double* d_dev, const double* e_dev, int64_t n,
                        double* lambda_dev, double* Z_dev, int64_t ldz, void* work_dev,
                        size_t work_bytes, fraclap_stream_t stream);

/* C = alpha * op(A) * op(B) + beta * C in FP64 with op = transpose when
 * trans_* != 0 (the GEMM engine behind every dense step). */
int fraclap_dgemm(fraclap_ctx* ctx, int trans_a, int trans_b, int64_t m, int64_t n, int64_t k,
                  double alpha, const double* A_dev, int64_t lda, const double* B_dev,
                  int64_t ldb, double beta, double* C_dev, int64_t ldc, fraclap_stream_t stream);

/* C = alpha * op(A) * op(B) + beta * C in FP32 (column-major), the engine of
 * the FP32 stages of eig_full_mixed.  route 1: tensor cores, three TF32
 * products A_hi B_hi + A_hi B_lo + A_lo B_hi of the operands split as
 * x = tf32(x) + tf32(x - tf32(x)) (FP32-level accuracy; taken when m >= 128,
 * n >= 64, k >= 64, else the SIMT kernel); route 0: FP32 FMA kernel.
 * form 0: plain; 1: A symmetric, only its lower triangle read (trans_a = 0,
 * m = k); 2: only the lower triangle of C (i >= j) is written.
 * work_dev: device scratch of fraclap_sgemm_workspace_bytes(m, n, k) bytes
 * (256-byte aligned; NULL: the context allocates it). */
size_t fraclap_sgemm_workspace_bytes(int64_t m, int64_t n, int64_t k);
int fraclap_sgemm(fraclap_ctx* ctx, int trans_a, int trans_b, int form, int64_t m, int64_t n, int64_t k,
                  float alpha, const float* A_dev, int64_t lda, const float* B_dev, int64_t ldb,
                  float beta, float* C_dev, int64_t ldc, int route, void* work_dev, size_t work_bytes,
                  fraclap_stream_t stream);

/* ------------------------------------------------------------------------
 * fraclap_solve_batched — many independent problems (masked grids of their
 * own size, forcings and orders) in one call: for each problem the
 * eigendecomposition (as eig_full, or eig_full_mixed when the problem
 * carries its CSR; band width 32) of its dense A into
 * lambda_dev / V_dev and, when k > 0, the spectral apply of its k pairs into
 * U_dev (as frac_apply; Sec. II eq. poisson_solution).  The problems are
 * spread over `workers` concurrent streams (0: 16), each with its own share
 * of the SMs and a context-owned workspace sized for its largest problem;
 * the caller's stream waits for all of them.  probs is a host array; every
 * pointer in it is a device pointer owned by the caller, and distinct
 * problems must not share outputs.  Device errors reach the context's status
 * word (fraclap_sync); argument errors name the problem.
 * ---------------------------------------------------------------------- */
typedef struct fraclap_problem {
  int64_t n;
  const double* A_dev;        /* n x n, column-major, lower triangle read */
  int64_t lda;
  double* lambda_dev;         /* n, ascending */
  double* V_dev;              /* n x n eigenvectors */
  int64_t ldv;
  const double* F_dev;        /* n x m forcings (may be NULL when k = 0) */
  int64_t ldf;
  int64_t m;
  const int32_t* pair_f_dev;  /* k forcing columns */
  const double* pair_alpha_dev; /* k orders */
  int64_t k;
  double* U_dev;              /* n x k solutions */
  int64_t ldu;
  /* optional CSR of the same A (as fd_assemble writes it): when rowptr_dev is
   * not NULL the problem takes the mixed route of eig_full_mixed with
   * refine_iters refinement iterations (1..8) instead of the FP64 route */
  const int64_t* rowptr_dev;
  const int32_t* col_dev;
  const double* val_dev;
  int refine_iters;
} fraclap_problem;
int fraclap_solve_batched(fraclap_ctx* ctx, const fraclap_problem* probs, int count, int workers,
                          fraclap_stream_t stream);

/* ------------------------------------------------------------------------
 * Instrumentation (no counterpart in the paper; it reports per-phase wall
 * times, Table I, and these give the same view of this library).
 * ---------------------------------------------------------------------- */
enum {
  FRACLAP_STAGE_ASSEMBLE = 0,       /* fd_assemble */
  FRACLAP_STAGE_BAND_REDUCTION = 1, /* dense -> band (panels + trailing updates) */
  FRACLAP_STAGE_BULGE_CHASING = 2,  /* band -> tridiagonal */
  FRACLAP_STAGE_TRIDIAG_DC = 3,     /* tridiagonal divide and conquer */
  FRACLAP_STAGE_BACK_Q2 = 4,        /* back-transformation by the bulge-chasing reflectors */
  FRACLAP_STAGE_BACK_Q1 = 5,        /* back-transformation by the panel reflectors */
  FRACLAP_STAGE_APPLY = 6,          /* frac_apply */
  FRACLAP_STAGE_REFINE = 7,         /* Ogita-Aishima refinement (eig_full_mixed) */
  FRACLAP_STAGE_RESIDUAL_GEMM = 8,  /* its tensor-core residual products (inside REFINE) */
  FRACLAP_STAGE_REFINE_NORMS = 9,   /* A V, Ritz values, 2-norm estimates (inside REFINE) */
  FRACLAP_STAGE_REFINE_UPDATE = 10, /* cluster detection, correction, V += V E (inside REFINE) */
  FRACLAP_STAGE_REFINE_SORT = 11,   /* ordering of the columns (inside REFINE) */
  FRACLAP_STAGE_REFINE_CLUSTERS = 12, /* exact diagonalisation of clusters up to 64 (inside REFINE) */
  FRACLAP_STAGE_REFINE_BIG_CLUSTERS = 13, /* larger clusters, dense FP64 solver (inside REFINE) */
  FRACLAP_STAGE_SLICE_PRODUCTS = 14, /* the tensor-core kernel of each FP64-accurate product alone */
  FRACLAP_STAGE_COUNT = 15
};
/* With enable != 0, every later stage records a CUDA event pair on its stream. */
int fraclap_set_profiling(fraclap_ctx* ctx, int enable);
/* Waits for the recorded events, writes the summed milliseconds (and the
 * number of records, count_out may be NULL) per stage id, and forgets them. */
int fraclap_stage_times(fraclap_ctx* ctx, double* ms_out, int64_t* count_out, int nstages);
/* Statistics of the last eig_full_mixed refinement, 8 values per iteration:
 * the cluster threshold delta, the estimates of ||S - D||_2 and ||R||_2 used
 * for it, ||S - D||_F, ||R||_F, the Gershgorin bound of ||A||_2, the number
 * of clusters and the largest cluster.  Copies at most max_values values and
 * returns how many there are. */
int fraclap_refine_stats(const fraclap_ctx* ctx, double* out, int max_values);
/* Number of kernels the context has launched so far. */
long long fraclap_launch_count(const fraclap_ctx* ctx);

/* Refinement safeguard of eig_full_mixed: a pair whose first-order
 * correction coefficient exceeds tau (default 1e-3) is treated as part of a
 * cluster and diagonalised exactly; 0 < tau <= 1. */
int fraclap_set_refine_tau(fraclap_ctx* ctx, double tau);

/* Tensor-core route of the BF16 slice products: 1 (default) = tcgen05.mma
 * with TMA-loaded operands and tensor-memory accumulators; 0 = mma.sync
 * (kept to cross-check the first). */
int fraclap_set_tensor_route(fraclap_ctx* ctx, int route);

/* Failure detection of the bounded device waits, without a fault: one CTA
 * waits, through the library's own primitives, on an event that nothing
 * produces -- which = 0: the grid barrier of the cooperative kernels (one CTA
 * arriving where two are expected); which = 1: an mbarrier of the
 * tensor-core kernels with no arrival.  The wait gives up after the
 * context's limit (fraclap_opts.wait_timeout_s), the kernel records
 * FRACLAP_ERR_TIMEOUT in the device status and returns, so the next
 * fraclap_sync reports -4 and the context stays usable.  Asynchronous on
 * `stream`; returns FRACLAP_ERR_INVALID_ARG for any other `which`. */
int fraclap_wait_selftest(fraclap_ctx* ctx, int which, fraclap_stream_t stream);

/* Sustained throughput of the FMA pipe (precision 64: DFMA, 32: FFMA) in
 * flop/s, measured by independent FMA chains over 8 CTAs of 256 threads per
 * SM (iters steps each: 2^14 FP64 or 2^18 FP32 steps take under a tenth
 * of a second on a GB300), one untimed launch
 * then one timed with CUDA events; synchronises `stream`.  The peaks the
 * SIMT FP64 and FP32 kernels are measured against (no counterpart in the
 * paper). */
int fraclap_fma_throughput(fraclap_ctx* ctx, int precision, int64_t iters, double* flops_per_s,
                           fraclap_stream_t stream);

/* C = alpha op(A) op(B) + beta C with FP64-accurate products formed on the
 * BF16 tensor cores by Ozaki's error-free splitting into `slices` 8-bit slices
 * per row/column (7 slices: full FP64 accuracy; fewer: about 8*slices bits
 * relative to the row and column maxima).  The engine behind the
 * refinement's residual products.  work: fraclap_dgemm_ozaki_workspace_bytes. */
size_t fraclap_dgemm_ozaki_workspace_bytes(int64_t m, int64_t n, int64_t k, int slices);
int fraclap_dgemm_ozaki(fraclap_ctx* ctx, int trans_a, int trans_b, int64_t m, int64_t n,
                        int64_t k, double alpha, const double* A_dev, int64_t lda,
                        const double* B_dev, int64_t ldb, double beta, double* C_dev,
                        int64_t ldc, int slices, void* work_dev, size_t work_bytes,
                        fraclap_stream_t stream);

/* ------------------------------------------------------------------------
 * The generalised problem with a mass matrix (Sec. II eq. discrete_laplace:
 * K phi = theta M phi, K_ij = <grad e_i, grad e_j>, M_ij = <e_i, e_j>) for
 * piecewise bilinear (2-D) / trilinear (3-D) basis functions on the grid
 * cells, homogeneous Dirichlet conditions (nodes outside the mask are
 * zero), and its spectral apply in the M-inner product (the coefficient of
 * a nodal vector f on phi_i is phi_i^T M f, the sum v after the equation).
 *
 * fem_assemble: as fd_assemble (same mask, extents, dof numbering and
 *   two-call protocol), but every row holds the dofs of the 3^dim box of
 *   grid nodes around it (columns ascending) and two value arrays:
 *   valK_dev and valM_dev double[nnz] (each entry the sum, over the cells
 *   holding both nodes, of the cell integrals of the multilinear basis
 *   functions: products of the 1-D hat integrals h/3, h/6 and +-1/h).
 *   K_dense_dev, M_dense_dev: optional dense copies (ld >= n).
 * eig_pencil: K Phi = M Phi diag(theta), Phi^T M Phi = I, theta ascending.
 *   K_dev: dense n x n (ldk >= n), lower triangle read; M in CSR
 *   (rowptr_dev, col_dev, valM_dev, lower triangle read) with
 *   half_bandwidth >= fraclap_csr_half_bandwidth.  M = L D L^T by a banded
 *   factorisation (a pivot <= 0: FRACLAP_ERR_NOT_SPD in the device status),
 *   C = D^-1/2 L^-1 K L^-T D^-1/2 by banded solves, C = Z diag(theta) Z^T as
 *   eig_full, Phi = L^-T D^-1/2 Z.  theta_dev double[n], Phi_dev
 *   double[ldp*n] out.  Work: fraclap_eig_pencil_workspace_bytes; the
 *   half-bandwidth may be at most 6399 (FRACLAP_ERR_UNSUPPORTED beyond).
 * frac_apply_mass: u_j = Phi diag(theta^{-alpha_j/2}) Phi^T M f_{pair_f[j]}
 *   (M f formed from the CSR of M, then as frac_apply, whose products and
 *   context settings it shares).  Work: fraclap_apply_mass_workspace_bytes.
 * ---------------------------------------------------------------------- */
int fem_assemble(fraclap_ctx* ctx, const uint8_t* mask_dev, int dim, const int64_t ext[3], double h,
                 int32_t* idx_dev, int64_t* n_out, int64_t* nnz_out, int64_t* rowptr_dev, int32_t* col_dev,
                 double* valK_dev, double* valM_dev, double* K_dense_dev, double* M_dense_dev, int64_t ld,
                 fraclap_stream_t stream);
size_t fraclap_eig_pencil_workspace_bytes(const fraclap_ctx* ctx, int64_t n, int64_t half_bandwidth);
int eig_pencil(fraclap_ctx* ctx, const double* K_dev, int64_t ldk, int64_t n, const int64_t* rowptr_dev,
               const int32_t* col_dev, const double* valM_dev, int64_t half_bandwidth, double* theta_dev,
               double* Phi_dev, int64_t ldp, void* work_dev, size_t work_bytes, fraclap_stream_t stream);
size_t fraclap_apply_mass_workspace_bytes(const fraclap_ctx* ctx, int64_t n, int64_t m, int64_t k);
int frac_apply_mass(fraclap_ctx* ctx, const double* Phi_dev, int64_t ldp, const double* theta_dev, int64_t n,
                    const int64_t* rowptr_dev, const int32_t* col_dev, const double* valM_dev, const double* F_dev,
                    int64_t ldf, int64_t m, const int32_t* pair_f_dev, const double* pair_alpha_dev, int64_t k,
                    double* U_dev, int64_t ldu, void* work_dev, size_t work_bytes, fraclap_stream_t stream);

/* ------------------------------------------------------------------------
 * Exact eigenvalue counts and spectrum slicing (Sec. III-D).  By Sylvester's
 * law of inertia (Sec. III-D-2) the number of eigenvalues of A below sigma is
 * the number of negative pivots of A - sigma I = L D L^T, and for the
 * generalised problem K phi = theta M phi (Sec. II eq. discrete_laplace) the
 * number of theta below sigma is that of K - sigma M.  No dense matrix is
 * needed: the factorisation runs on the band of the sparse matrix (in the
 * natural dof order of a grid, half-width = the grid row length in 2-D, the
 * plane size in 3-D).
 *
 * fraclap_csr_half_bandwidth: max(i - j) over the entries (i, j), j <= i, of
 *   a CSR matrix (int64 rowptr[n+1], int32 col[nnz], as fd_assemble writes
 *   them); synchronises `stream` to return it in *bw_out.
 * fraclap_inertia_counts: count_dev[s] (int64, device) = #{eigenvalues <
 *   sigma_dev[s]} for s < nsig, of the symmetric CSR matrix K (valK_dev;
 *   only the lower triangle is read) or, when valM_dev is not NULL, of the
 *   pencil (K, M) with M on the same sparsity pattern.  One pivot sequence per
 *   shift, all shifts in parallel; -1 for a shift at which a pivot is exactly
 *   zero (the shift is then, to rounding, an eigenvalue of a leading block).
 *   half_bandwidth >= fraclap_csr_half_bandwidth (an entry outside it sets
 *   FRACLAP_ERR_INVALID_ARG in the device status).  Work:
 *   fraclap_inertia_workspace_bytes(n, half_bandwidth, nsig, valM != NULL);
 *   asynchronous.  The pivots are formed by the same operations in the same
 *   order as a sequential banded LDL^T without pivoting, so the counts do not
 *   depend on the launch.
 * fraclap_sturm_counts: the same counts for a symmetric tridiagonal T
 *   (d_dev[n], e_dev[n-1], e.g. from fraclap_tridiagonalize, whose T is
 *   congruent to A) by the Sturm recurrence q_0 = d_0 - sigma,
 *   q_i = (d_i - sigma) - e_{i-1}^2 / q_{i-1} (a zero pivot counts as
 *   negative); one thread per shift; asynchronous.
 * fraclap_bisect: eigenvalues k0..k1 (0-based, ascending) of T into
 *   lambda_dev[k1 - k0 + 1] by bisection on the Sturm count from the
 *   Gershgorin interval, to no representable midpoint or 2 eps relative;
 *   one thread per eigenvalue; asynchronous.
 * fraclap_partition_spectrum: the greedy partitioning of Sec. III-D: P
 *   subintervals of [0, rho] (rho >= the largest eigenvalue, e.g. the
 *   Gershgorin bound 4 dim / h^2) holding about n / P eigenvalues each.
 *   Starts from P equal lengths; n_a global rounds count at every split at
 *   once, read the counts as a piecewise-constant density of states (the
 *   cumulative count linear between counted points) and move every split to
 *   where that density gives equal loads, keeping the best partition (the
 *   smallest largest load); then up to n_b local passes, in which every pair
 *   of neighbouring subintervals whose loads differ by more than
 *   imbalance * n / P moves its shared split by a binary search of n_c
 *   counts towards an even pair (all pairs starting at even positions at
 *   once, then the odd ones).  Outputs (HOST): splits_host[P-1],
 *   loads_host[P] (exact counts per subinterval), history_host[history_cap]
 *   (the largest load after the start, each round and each pass).  Returns
 *   the number of history entries (>= 0) or an error; synchronises
 *   `stream` after every round of counts.  Work: as fraclap_inertia_counts
 *   with nsig = P - 1, plus 512 + 16 (P - 1) bytes.
 * ---------------------------------------------------------------------- */
int fraclap_csr_half_bandwidth(fraclap_ctx* ctx, int64_t n, const int64_t* rowptr_dev, const int32_t* col_dev,
                               int64_t* bw_out, fraclap_stream_t stream);
size_t fraclap_inertia_workspace_bytes(int64_t n, int64_t half_bandwidth, int64_t nsig, int pencil);
int fraclap_inertia_counts(fraclap_ctx* ctx, int64_t n, const int64_t* rowptr_dev, const int32_t* col_dev,
                           const double* valK_dev, const double* valM_dev, int64_t half_bandwidth,
                           const double* sigma_dev, int64_t nsig, int64_t* count_dev, void* work_dev,
                           size_t work_bytes, fraclap_stream_t stream);
int fraclap_sturm_counts(fraclap_ctx* ctx, const double* d_dev, const double* e_dev, int64_t n,
                         const double* sigma_dev, int64_t nsig, int64_t* count_dev, fraclap_stream_t stream);
int fraclap_bisect(fraclap_ctx* ctx, const double* d_dev, const double* e_dev, int64_t n, int64_t k0, int64_t k1,
                   double* lambda_dev, fraclap_stream_t stream);
int fraclap_partition_spectrum(fraclap_ctx* ctx, int64_t n, const int64_t* rowptr_dev, const int32_t* col_dev,
                               const double* valK_dev, const double* valM_dev, int64_t half_bandwidth, double rho,
                               int P, int n_a, int n_b, int n_c, double imbalance, double* splits_host,
                               int64_t* loads_host, int64_t* history_host, int history_cap, void* work_dev,
                               size_t work_bytes, fraclap_stream_t stream);

/* ------------------------------------------------------------------------
 * Schedule knobs of a context (tile orders and digit widths; the results do
 * not depend on them beyond rounding), measured and picked by the autotuner
 * of the Python package.  fraclap_set_schedule returns FRACLAP_ERR_INVALID_ARG
 * for an unknown knob or a value outside its range; fraclap_get_schedule
 * returns the current value (or FRACLAP_ERR_INVALID_ARG).
 *  FRACLAP_SCHED_OZAKI_GROUP: tile rows per raster group of the slice-product
 *    kernel (fraclap_dgemm_ozaki, the refinement's residual products, the
 *    sliced apply), 0..4096; 0 = every tile row in one group [8].
 *  FRACLAP_SCHED_OZAKI_BITS: digit width of the slices when K > 256: 7
 *    (exact chunks of 1024, ceil(8 s / 7) digits per operand) or 8 (exact
 *    chunks of 256, s digits: fewer slice pairs, more chunk sums) [7].
 *  FRACLAP_SCHED_FP32_STAGES: the FP32 products of eig_full_mixed's band
 *    reduction and first back-transformation: 0 on the FP32 FMA kernel, 1 on
 *    the tensor cores as three TF32 products (FP32-level accuracy, a few
 *    2^-22 per product instead of 2^-24) [0].
 *  FRACLAP_SCHED_OZAKI_TILE_N: columns of the slice-product kernel's output
 *    tile, 128, 192 or 256 (rows are 128; outputs of at most 128 columns
 *    always take 128) [192].
 *  FRACLAP_SCHED_Q2_PARTS: at half-bandwidth 64, the lanes that share one
 *    column's window of the stage-2 back-transformation: 4, 8 or 16 (16, 8 or
 *    4 rows per lane; more parts give more warps over the same columns; FP64
 *    takes 8 when asked for 4), or 0 for the default 8 [0].
 *  FRACLAP_SCHED_OZAKI_CLUSTER: CTAs of the slice-product kernel per thread-
 *    block cluster, 1 or 2: the two CTAs of a cluster take consecutive tile
 *    rows of one tile column and share its B tile through TMA multicast,
 *    each loading half of it (fewer L2-to-SM bytes per flop) [1].
 * ---------------------------------------------------------------------- */
enum { FRACLAP_SCHED_OZAKI_GROUP = 0, FRACLAP_SCHED_OZAKI_BITS = 1, FRACLAP_SCHED_FP32_STAGES = 2,
       FRACLAP_SCHED_OZAKI_TILE_N = 3, FRACLAP_SCHED_Q2_PARTS = 4, FRACLAP_SCHED_OZAKI_CLUSTER = 5 };
int fraclap_set_schedule(fraclap_ctx* ctx, int knob, int value);
int fraclap_get_schedule(const fraclap_ctx* ctx, int knob);

#ifdef __cplusplus
}
#endif
#endif /* FRACLAP_H_ */
