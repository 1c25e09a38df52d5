// server.cu -- a request loop for partition requests: a FIFO queue, worker
// threads with their own contexts (stream, memory pool), admission against a
// device-memory budget, per-request timing.
#include "gp_internal.cuh"

#include <chrono>
#include <condition_variable>
#include <deque>
#include <mutex>
#include <thread>
#include <unordered_map>

namespace {

using Clock = std::chrono::steady_clock;

struct Job {
  gp_request req;
  int64_t est = 0;
  Clock::time_point t_submit, t_start, t_end;
  gp_status status = GP_OK;
  int64_t cut = 0;
  int64_t order = 0;     // admission order
  int32_t bypassed = 0;  // younger requests admitted while this one headed the queue
  int64_t peak_reserved = 0, peak_used = 0;
  bool done = false;
};

// Device memory a partition request is admitted with: four times its CSR
// (input copy, contraction segments, coarse graph, sparsified graph), the
// hash tables of high-degree nodes (at most 8 bytes per entry plus 16 MiB),
// 128 bytes per node (LP state, lists, the initial partitioner's trial state)
// and 64 MiB; the served test checks every request's measured peak against it.
int64_t estimate(const gp_request &r) {
  const int64_t csr = 4 * ((int64_t)r.n + 1) + 8 * r.m2 + 4 * (int64_t)r.n;
  return 4 * csr + 8 * r.m2 + 128 * (int64_t)r.n + ((int64_t)80 << 20);
}

double ms(Clock::time_point a, Clock::time_point b) {
  return std::chrono::duration<double, std::milli>(b - a).count();
}

}  // namespace

struct gp_server {
  int device = 0;
  gp_config cfg{};
  int64_t budget = 0, in_use = 0;
  int running = 0;
  std::vector<gp_ctx *> ctxs;
  std::vector<cudaStream_t> streams;
  std::vector<std::thread> threads;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<int64_t> queue;
  std::unordered_map<int64_t, Job> jobs;
  int64_t next_ticket = 1, next_order = 1;
  int32_t max_bypass = 8;
  bool stop = false;

  // The oldest queued job if it fits next to those in flight (any job when none
  // is in flight); else a younger one that fits, as long as the oldest has been
  // passed over fewer than max_bypass times.
  bool pick(int64_t *ticket) {
    if (queue.empty()) return false;
    Job &head = jobs[queue.front()];
    if (running == 0 || in_use + head.est <= budget) {
      *ticket = queue.front();
      queue.pop_front();
      return true;
    }
    if (head.bypassed >= max_bypass) return false;
    for (auto it = queue.begin() + 1; it != queue.end(); ++it) {
      if (in_use + jobs[*it].est <= budget) {
        head.bypassed++;
        *ticket = *it;
        queue.erase(it);
        return true;
      }
    }
    return false;
  }

  void worker(int wi) {
    cudaSetDevice(device);
    gp_ctx *ctx = ctxs[(size_t)wi];
    for (;;) {
      int64_t t = 0;
      gp_request req;
      int64_t est = 0;
      {
        std::unique_lock<std::mutex> lk(mu);
        cv_work.wait(lk, [&] { return (stop && queue.empty()) || (!queue.empty() && pick(&t)); });
        if (t == 0) return;  // stopping and nothing left
        Job &j = jobs[t];
        j.t_start = Clock::now();
        j.order = next_order++;
        req = j.req;
        est = j.est;
        in_use += est;
        running++;
      }
      // the worker's pool starts empty, so its high-water marks are this request's
      if (ctx->pool) {
        cudaMemPoolTrimTo(ctx->pool, 0);
        unsigned long long zero = 0;
        cudaMemPoolSetAttribute(ctx->pool, cudaMemPoolAttrReservedMemHigh, &zero);
        cudaMemPoolSetAttribute(ctx->pool, cudaMemPoolAttrUsedMemHigh, &zero);
      }
      int64_t cut = 0;
      const gp_status st = gp_partition_host(ctx, req.n, req.m2, req.xadj, req.adjncy, req.vwgt, req.adjwgt,
                                             req.k, req.eps, req.seed, &cfg, req.blocks, &cut, nullptr);
      unsigned long long hi_res = 0, hi_used = 0;
      if (ctx->pool) {
        cudaStreamSynchronize(ctx->stream);
        cudaMemPoolGetAttribute(ctx->pool, cudaMemPoolAttrReservedMemHigh, &hi_res);
        cudaMemPoolGetAttribute(ctx->pool, cudaMemPoolAttrUsedMemHigh, &hi_used);
        cudaMemPoolTrimTo(ctx->pool, 0);  // an idle worker holds no memory outside the budget
      }
      {
        std::lock_guard<std::mutex> lk(mu);
        Job &j = jobs[t];
        j.t_end = Clock::now();
        j.status = st;
        j.cut = cut;
        j.peak_reserved = (int64_t)hi_res;
        j.peak_used = (int64_t)hi_used;
        j.done = true;
        in_use -= est;
        running--;
      }
      cv_done.notify_all();
      cv_work.notify_all();
    }
  }
};

extern "C" {

gp_status gp_server_create(gp_server **out, int device, int32_t workers, int64_t hbm_budget_bytes,
                           const gp_config *cfg) {
  if (!out || workers < 1 || workers > 64 || hbm_budget_bytes <= 0) return GP_ERR_INVALID;
  *out = nullptr;
  gp_server *s = new (std::nothrow) gp_server();
  if (!s) return GP_ERR_OOM;
  s->device = device;
  s->budget = hbm_budget_bytes;
  if (cfg) s->cfg = *cfg;
  else gp_config_default(&s->cfg);
  if (cudaSetDevice(device) != cudaSuccess) { delete s; return GP_ERR_CUDA; }
  for (int i = 0; i < workers; i++) {
    cudaStream_t st = nullptr;
    gp_ctx *c = nullptr;
    if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess ||
        gp_create(&c, device, (void *)st, nullptr) != GP_OK) {
      if (st) cudaStreamDestroy(st);
      s->stop = true;
      gp_server_destroy(s);
      return GP_ERR_CUDA;
    }
    c->device_share = workers;
    s->ctxs.push_back(c);
    s->streams.push_back(st);
  }
  for (int i = 0; i < workers; i++) s->threads.emplace_back(&gp_server::worker, s, i);
  *out = s;
  return GP_OK;
}

void gp_server_set_max_bypass(gp_server *s, int32_t max_bypass) {
  if (!s || max_bypass < 0) return;
  std::lock_guard<std::mutex> lk(s->mu);
  s->max_bypass = max_bypass;
}

gp_status gp_server_submit(gp_server *s, const gp_request *req, int64_t *ticket) {
  if (!s || !req || !ticket) return GP_ERR_INVALID;
  if (req->n < 0 || req->m2 < 0 || req->m2 >= ((int64_t)1 << 31) || (req->n > 0 && (!req->xadj || !req->vwgt || !req->blocks)) ||
      (req->m2 > 0 && (!req->adjncy || !req->adjwgt)))
    return GP_ERR_INVALID;
  Job j;
  j.req = *req;
  j.est = estimate(*req);
  if (j.est > s->budget) return GP_ERR_BUDGET;
  j.t_submit = Clock::now();
  {
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->stop) return GP_ERR_INVALID;
    *ticket = s->next_ticket++;
    s->jobs.emplace(*ticket, j);
    s->queue.push_back(*ticket);
  }
  s->cv_work.notify_all();
  return GP_OK;
}

gp_status gp_server_wait(gp_server *s, int64_t ticket, gp_response *out) {
  if (!s || !out) return GP_ERR_INVALID;
  std::unique_lock<std::mutex> lk(s->mu);
  if (s->jobs.find(ticket) == s->jobs.end()) return GP_ERR_INVALID;
  // a ticket is waited for once; a second waiter finds it gone and returns GP_ERR_INVALID
  s->cv_done.wait(lk, [&] {
    auto it = s->jobs.find(ticket);
    return it == s->jobs.end() || it->second.done;
  });
  auto it = s->jobs.find(ticket);
  if (it == s->jobs.end()) return GP_ERR_INVALID;
  const Job &j = it->second;
  out->status = j.status;
  out->cut = j.cut;
  out->queued_ms = ms(j.t_submit, j.t_start);
  out->run_ms = ms(j.t_start, j.t_end);
  out->total_ms = ms(j.t_submit, j.t_end);
  out->start_order = j.order;
  out->estimate_bytes = j.est;
  out->peak_reserved_bytes = j.peak_reserved;
  out->peak_used_bytes = j.peak_used;
  s->jobs.erase(it);
  lk.unlock();
  s->cv_done.notify_all();
  return GP_OK;
}

void gp_server_destroy(gp_server *s) {
  if (!s) return;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
  }
  s->cv_work.notify_all();
  for (auto &t : s->threads) t.join();
  cudaSetDevice(s->device);
  for (size_t i = 0; i < s->ctxs.size(); i++) {
    gp_destroy(s->ctxs[i]);
    cudaStreamDestroy(s->streams[i]);
  }
  delete s;
}

}  // extern "C"
