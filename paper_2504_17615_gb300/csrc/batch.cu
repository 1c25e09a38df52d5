// batch.cu -- many independent graphs partitioned at once.  Each worker is
// a context of its own (stream, memory pool) driven by its own host thread;
// the level loops of different graphs then overlap on the GPU, which a
// single small graph cannot fill.  Every item runs the same partition_impl
// as gp_partition, so the results do not depend on the batching.
#include "gp_internal.cuh"

#include <algorithm>
#include <atomic>
#include <thread>

extern "C" gp_status gp_partition_batch(gp_ctx *ctx, gp_batch_item *items, int32_t count, int32_t workers,
                                        const gp_config *cfg) {
  if (!ctx) return GP_ERR_INVALID;
  if (count < 0 || (count > 0 && !items) || workers < 1 || workers > 64) {
    ctx->last_error = "gp_partition_batch: bad arguments (count >= 0, items, 1 <= workers <= 64)";
    return GP_ERR_INVALID;
  }
  gp_config c;
  if (cfg) c = *cfg;
  else gp_config_default(&c);
  try {
    GP_CUDA(cudaSetDevice(ctx->device));
    while ((int)ctx->workers.size() < workers) {
      cudaStream_t s = nullptr;
      GP_CUDA(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
      gp_ctx *w = nullptr;
      const gp_status st = gp_create(&w, ctx->device, (void *)s, nullptr);
      if (st != GP_OK) {
        cudaStreamDestroy(s);
        gp::fail(st, "gp_partition_batch: creating a worker failed");
      }
      ctx->workers.push_back(w);
    }
    for (int i = 0; i < workers; i++) ctx->workers[i]->device_share = workers;
    // inputs may still be in flight on the caller's stream
    cudaEvent_t ready;
    GP_CUDA(cudaEventCreateWithFlags(&ready, cudaEventDisableTiming));
    GP_CUDA(cudaEventRecord(ready, ctx->stream));
    for (int i = 0; i < workers; i++) GP_CUDA(cudaStreamWaitEvent(ctx->workers[i]->stream, ready, 0));
    GP_CUDA(cudaEventDestroy(ready));
  } catch (const gp::Error &e) {
    ctx->last_error = e.msg;
    return e.status;
  }
  std::vector<int32_t> order((size_t)count);
  for (int32_t i = 0; i < count; i++) order[(size_t)i] = i;
  std::stable_sort(order.begin(), order.end(), [&](int32_t a, int32_t b) { return items[a].g.m2 > items[b].g.m2; });
  std::atomic<int32_t> next{0};
  auto run = [&](gp_ctx *w) {
    cudaSetDevice(w->device);
    for (;;) {
      const int32_t j = next.fetch_add(1);
      if (j >= count) break;
      gp_batch_item &it = items[order[(size_t)j]];
      it.cut = 0;
      it.status = gp_partition(w, &it.g, it.k, it.eps, it.seed, &c, it.blocks, &it.cut, nullptr);
    }
  };
  std::vector<std::thread> threads;
  for (int i = 1; i < workers; i++) threads.emplace_back(run, ctx->workers[(size_t)i]);
  run(ctx->workers[0]);
  for (auto &t : threads) t.join();
  for (int32_t i = 0; i < count; i++) {
    if (items[i].status != GP_OK) {
      ctx->last_error = "gp_partition_batch: item " + std::to_string(i) + " failed";
      return items[i].status;
    }
  }
  ctx->last_error.clear();
  return GP_OK;
}
