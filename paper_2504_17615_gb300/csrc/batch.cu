// batch.cu -- many independent graphs partitioned at once.
//
// Items the batched engine takes (engine.cu) run there first: one persistent
// launch whose CTAs partition whole graphs.  The rest run on the per-graph
// path: each worker is a context of its own (stream, memory pool) driven by
// its own host thread, so the level loops of different graphs overlap on the
// GPU, which a single small graph cannot fill.  Every item, on either path,
// follows the same method and readings as gp_partition, so the results do not
// depend on the batching.
#include "gp_internal.cuh"

#include <algorithm>
#include <atomic>
#include <cmath>
#include <thread>

namespace gp {

void batch_per_graph(gp_ctx *ctx, gp_batch_item *items, const std::vector<int32_t> &idx, int workers,
                     const gp_config &cfg, int share, cudaEvent_t ready) {
  if (idx.empty()) return;
  GP_CUDA(cudaSetDevice(ctx->device));
  while ((int)ctx->workers.size() < workers) {
    cudaStream_t s = nullptr;
    GP_CUDA(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
    gp_ctx *w = nullptr;
    const gp_status st = gp_create(&w, ctx->device, (void *)s, nullptr);
    if (st != GP_OK) {
      cudaStreamDestroy(s);
      fail(st, "gp_partition_batch: creating a worker failed");
    }
    ctx->workers.push_back(w);
  }
  for (int i = 0; i < workers; i++) {
    ctx->workers[(size_t)i]->device_share = share;
    GP_CUDA(cudaStreamWaitEvent(ctx->workers[(size_t)i]->stream, ready, 0));
  }
  std::vector<int32_t> order(idx);
  std::stable_sort(order.begin(), order.end(), [&](int32_t a, int32_t b) { return items[a].g.m2 > items[b].g.m2; });
  std::atomic<size_t> next{0};
  auto run = [&](gp_ctx *w) {
    cudaSetDevice(w->device);
    for (;;) {
      const size_t j = next.fetch_add(1);
      if (j >= order.size()) break;
      gp_batch_item &it = items[order[j]];
      it.cut = 0;
      it.engine = 0;
      it.status = gp_partition(w, &it.g, it.k, it.eps, it.seed, &cfg, it.blocks, &it.cut, it.stats);
    }
  };
  std::vector<std::thread> threads;
  for (int i = 1; i < workers; i++) threads.emplace_back(run, ctx->workers[(size_t)i]);
  run(ctx->workers[0]);
  for (auto &t : threads) t.join();
}

}  // namespace gp

namespace {

// The argument checks gp_partition makes before any launch.
gp_status item_check(const gp_batch_item &it) {
  const gp_graph &g = it.g;
  if (g.n < 0 || g.m2 < 0 || g.m2 >= ((int64_t)1 << 31)) return GP_ERR_INVALID;
  if (g.n > 0 && (!g.xadj || !g.vwgt)) return GP_ERR_INVALID;
  if (g.m2 > 0 && (!g.adjncy || !g.adjwgt)) return GP_ERR_INVALID;
  if (g.n > 0 && !it.blocks) return GP_ERR_INVALID;
  if (it.k < 1 || !(it.eps > 0 && it.eps < 1000) || llround(it.eps * 1e6) < 1) return GP_ERR_INVALID;
  return GP_OK;
}

}  // namespace

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
  std::vector<int32_t> valid;
  for (int32_t i = 0; i < count; i++) {
    items[i].cut = 0;
    items[i].engine = 0;
    items[i].status = item_check(items[i]);
    if (items[i].status == GP_OK) valid.push_back(i);
  }
  try {
    GP_CUDA(cudaSetDevice(ctx->device));
    gp::batch_run(ctx, items, valid, workers, c, gp::batch_tuning(ctx));
  } catch (const gp::Error &e) {
    ctx->last_error = e.msg;
    return e.status;
  }
  for (int32_t i = 0; i < count; i++) {
    if (items[i].status != GP_OK) {
      ctx->last_error = "gp_partition_batch: item " + std::to_string(i) + " failed";
      return items[i].status;
    }
  }
  ctx->last_error.clear();
  return GP_OK;
}
