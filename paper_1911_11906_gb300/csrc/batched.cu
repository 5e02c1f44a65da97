// Many independent problems in one call: the batched workload of many small
// masked grids (each with its own n, forcings and orders).
//
// A single small decomposition leaves most of the GPU idle: its cost is the
// latency of the panel factorisation and of the bulge-chasing pipeline, not
// arithmetic.  The problems are therefore spread over W workers, each a
// sub-context that sees 1/W of the SMs (so that the cooperative kernels of
// different problems can be resident at the same time) with its own stream,
// workspace, status word and host thread issuing its launches.  Problems are
// dealt largest first to the least-loaded worker (cost ~ n^3); each runs the
// FP64 route, or the mixed route (FP32 stages + refinement) when the problem
// carries its CSR, with band width 32 (half the bulge-chasing step latency of
// 64 for these sizes), and then the spectral apply of its pairs.  The
// caller's stream waits for every worker; device errors of the workers are
// merged into the context's status word.
#include <algorithm>
#include <thread>
#include <vector>

#include "internal.cuh"

using namespace fraclap;

namespace {

__global__ void merge_status(int32_t* parent, int32_t* child) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    const int32_t v = *child;
    if (v != 0) {
      atomicCAS(parent, 0, v);
      *child = 0;
    }
  }
}

int ensure_workers(fraclap_ctx* ctx, int W) {
  while ((int)ctx->workers.size() < W) {
    fraclap_opts o{32, ctx->leaf_size, ctx->wait_timeout_s};
    fraclap_ctx* w = nullptr;
    int rc = fraclap_create(&w, &o);
    if (rc) return set_error(ctx, rc, "batched: worker context creation failed");
    cudaStream_t s = nullptr;
    cudaEvent_t e = nullptr;
    if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) {
      cudaGetLastError();
      if (s) cudaStreamDestroy(s);
      fraclap_destroy(w);
      return set_error(ctx, FRACLAP_ERR_CUDA, "batched: stream or event creation failed");
    }
    ctx->workers.push_back(w);
    ctx->worker_streams.push_back(s);
    ctx->worker_events.push_back(e);
  }
  if (!ctx->batch_start) FL_CUDA(ctx, cudaEventCreateWithFlags(&ctx->batch_start, cudaEventDisableTiming));
  const int share = std::max(8, ctx->sm_count / W);
  for (int i = 0; i < W; ++i) {
    fraclap_ctx* w = ctx->workers[i];
    w->sm_count = share;
    // the caller's settings of the kernels' routes and schedules hold for its workers
    w->tensor_route = ctx->tensor_route;
    w->refine_tau = ctx->refine_tau;
    w->oz_group = ctx->oz_group;
    w->oz_bits = ctx->oz_bits;
    w->oz_tile_n = ctx->oz_tile_n;
    w->oz_cluster = ctx->oz_cluster;
    w->q2_parts = ctx->q2_parts;
    w->fp32_stages_tc = ctx->fp32_stages_tc;
  }
  return 0;
}

}  // namespace

extern "C" int fraclap_solve_batched(fraclap_ctx* ctx, const fraclap_problem* probs, int count, int workers,
                                     fraclap_stream_t stream) {
  if (!ctx) return FRACLAP_ERR_INVALID_ARG;
  FL_CHECK(ctx, count >= 0 && (count == 0 || probs), FRACLAP_ERR_INVALID_ARG, "solve_batched: bad problem list");
  if (count == 0) return 0;
  for (int i = 0; i < count; ++i) {
    const fraclap_problem& p = probs[i];
    FL_CHECK(ctx, p.n >= 0 && p.m >= 0 && p.k >= 0, FRACLAP_ERR_INVALID_ARG, "solve_batched: problem %d: negative size", i);
    FL_CHECK(ctx, p.n == 0 || (p.A_dev && p.lambda_dev && p.V_dev && p.lda >= p.n && p.ldv >= p.n),
             FRACLAP_ERR_INVALID_ARG, "solve_batched: problem %d: missing matrix or output", i);
    FL_CHECK(ctx, p.k == 0 || p.n == 0 || (p.F_dev && p.pair_f_dev && p.pair_alpha_dev && p.U_dev && p.ldf >= p.n && p.ldu >= p.n),
             FRACLAP_ERR_INVALID_ARG, "solve_batched: problem %d: missing forcings or pairs", i);
    FL_CHECK(ctx, !p.rowptr_dev || (p.col_dev && p.val_dev && p.refine_iters >= 1 && p.refine_iters <= 8),
             FRACLAP_ERR_INVALID_ARG, "solve_batched: problem %d: incomplete CSR or refine_iters outside 1..8", i);
  }
  const int W = std::max(1, std::min({workers > 0 ? workers : 16, count, 64}));
  FL_TRY(ensure_workers(ctx, W));
  // deal the problems largest first to the least-loaded worker
  std::vector<int> order(count);
  for (int i = 0; i < count; ++i) order[i] = i;
  std::sort(order.begin(), order.end(), [&](int a, int b) { return probs[a].n > probs[b].n; });
  std::vector<std::vector<int>> plan(W);
  std::vector<double> load(W, 0.0);
  for (int i : order) {
    const int w = (int)(std::min_element(load.begin(), load.end()) - load.begin());
    plan[w].push_back(i);
    const double n = (double)probs[i].n;
    load[w] += n * n * n + 1.0;
  }
  // size every worker's workspace before any launch (growing it later would synchronise)
  for (int w = 0; w < W; ++w) {
    size_t need = 0;
    for (int i : plan[w]) {
      const fraclap_problem& p = probs[i];
      if (p.n == 0) continue;
      need = std::max(need, p.rowptr_dev ? fraclap_eig_mixed_workspace_bytes(ctx->workers[w], p.n)
                                         : fraclap_eig_workspace_bytes(ctx->workers[w], p.n));
      if (p.k > 0) need = std::max(need, fraclap_apply_workspace_bytes(p.n, p.m, p.k));
    }
    if (need == 0) continue;
    Arena ar;
    fraclap_ctx* wc = ctx->workers[w];
    if (get_workspace(wc, nullptr, 0, need, &ar)) return set_error(ctx, FRACLAP_ERR_ALLOC, "solve_batched: %s", wc->last_error.c_str());
  }
  FL_CUDA(ctx, cudaEventRecord(ctx->batch_start, (cudaStream_t)stream));
  for (int w = 0; w < W; ++w) FL_CUDA(ctx, cudaStreamWaitEvent(ctx->worker_streams[w], ctx->batch_start, 0));
  std::vector<int> rcs(W, 0);
  std::vector<int> failed(W, -1);
  auto run = [&](int w) {
    cudaSetDevice(ctx->device);
    fraclap_ctx* wc = ctx->workers[w];
    cudaStream_t s = ctx->worker_streams[w];
    for (int i : plan[w]) {
      const fraclap_problem& p = probs[i];
      if (p.n == 0) continue;
      int rc = p.rowptr_dev
                   ? eig_full_mixed(wc, p.A_dev, p.n, p.lda, p.rowptr_dev, p.col_dev, p.val_dev, p.refine_iters,
                                    p.lambda_dev, p.V_dev, p.ldv, nullptr, 0, nullptr, s)
                   : eig_full(wc, p.A_dev, p.n, p.lda, p.lambda_dev, p.V_dev, p.ldv, nullptr, 0, nullptr, s);
      if (rc == 0 && p.k > 0)
        rc = frac_apply(wc, p.V_dev, p.ldv, p.lambda_dev, p.n, p.F_dev, p.ldf, p.m, p.pair_f_dev,
                        p.pair_alpha_dev, p.k, p.U_dev, p.ldu, nullptr, 0, s);
      if (rc) {
        rcs[w] = rc;
        failed[w] = i;
        break;
      }
    }
    cudaEventRecord(ctx->worker_events[w], s);
  };
  {
    std::vector<std::thread> threads;
    threads.reserve(W);
    for (int w = 1; w < W; ++w) {
      try {
        threads.emplace_back(run, w);
      } catch (...) {  // no thread to be had: this worker's problems run here
        run(w);
      }
    }
    run(0);
    for (auto& t : threads) t.join();
  }
  for (int w = 0; w < W; ++w) {
    FL_CUDA(ctx, cudaStreamWaitEvent((cudaStream_t)stream, ctx->worker_events[w], 0));
    merge_status<<<1, 32, 0, (cudaStream_t)stream>>>(ctx->d_status, ctx->workers[w]->d_status);
    count_launch(ctx);
  }
  FL_CUDA(ctx, cudaGetLastError());
  for (int w = 0; w < W; ++w) {
    ctx->launches += ctx->workers[w]->launches;
    ctx->workers[w]->launches = 0;
    if (rcs[w])
      return set_error(ctx, rcs[w], "solve_batched: problem %d: %s", failed[w], ctx->workers[w]->last_error.c_str());
  }
  return 0;
}
