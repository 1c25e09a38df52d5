// engine.cu -- the batched engine, host side: which items it takes, its
// arenas and queue, the launch, the hand-over of items that outgrow their
// arena, and the autotuner (CTA size and the engine / per-graph split by size
// class).  The kernel itself is in engine_dev.cuh, instantiated once per CTA
// size in engine_k*.cu.
#include "engine_abi.cuh"

#include <algorithm>
#include <chrono>
#include <thread>

namespace gp {

namespace {

// Arena bytes one item needs (hierarchy + scratch of the largest level); an
// estimate -- an item that outgrows it is handed to the per-graph path.
int64_t engine_arena_estimate(int64_t n, int64_t m2, int64_t k) {
  return 160 * n + 40 * m2 + 64 * k + ((int64_t)4 << 20);
}

using namespace eng;

Kernel engine_kernel(int threads) {
  switch (threads) {
    case 256: return kernel_256();
    case 1024: return kernel_1024();
    default: return kernel_512();
  }
}

// Resident CTAs of the engine kernel on the whole device.
int engine_resident(gp_ctx *ctx, const Kernel &K) {
  const size_t smem = smem_bytes(K.threads);
  GP_CUDA(cudaFuncSetAttribute(K.fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  int bps = 0;
  GP_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, K.fn, K.threads, smem));
  return bps * ctx->num_sms;
}

struct EngineJob {
  std::vector<EItem> items;            // engine items (device descriptors)
  std::vector<int32_t> owner;          // batch index of each engine item
  std::vector<gp_partition_stats *> stats;
};

// One engine launch in flight: its buffers, and what the host gets back.
struct EngineRun {
  gp_ctx *ctx = nullptr;
  int32_t cnt = 0;
  int grid = 0, threads = 0;
  int64_t arena = 0;
  bool want_lv = false, timed = false;
  DBuf<EItem> d_items;
  DBuf<EOut> d_out;
  DBuf<int32_t> d_order, d_head;
  DBuf<gp_level_stats> d_lv;
  DBuf<unsigned char> d_arena;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  ~EngineRun() {
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
  }
};

// Starts the engine on job (item j of the job = owner[j] of the batch) on the
// context stream without waiting for it.  `share` > 1: the engine takes
// 1/share of the resident CTAs, so that other work (the per-graph path) can
// run beside it.  run.grid == 0: nothing was launched (no arena fits).
void engine_begin(gp_ctx *ctx, const EngineJob &job, const gp_config &cfg, int threads, int64_t arena_cap,
                  int64_t arena_override, int share, bool want_lv, bool timed, EngineRun &run) {
  run.ctx = ctx;
  run.cnt = (int32_t)job.items.size();
  run.threads = threads;
  run.want_lv = want_lv;
  run.timed = timed;
  if (run.cnt == 0) return;
  const Kernel K = engine_kernel(threads);
  const int resident = engine_resident(ctx, K);
  int64_t arena = 0;
  for (const EItem &it : job.items) arena = std::max(arena, engine_arena_estimate(it.n, it.m2, it.k));
  if (arena_override > 0) arena = arena_override;
  arena = (arena + 4095) & ~(int64_t)4095;
  if (arena_cap <= 0) {
    size_t fr = 0, tot = 0;
    GP_CUDA(cudaMemGetInfo(&fr, &tot));
    arena_cap = (int64_t)(fr / 3);
  }
  const int64_t slots = std::max<int64_t>(1, resident / std::max(1, share));
  const int64_t grid64 = std::min<int64_t>({slots, (int64_t)run.cnt, arena_cap / arena});
  if (grid64 < 1) return;
  run.grid = (int)grid64;
  run.arena = arena;
  // queue: largest first
  std::vector<int32_t> order((size_t)run.cnt);
  for (int32_t j = 0; j < run.cnt; j++) order[(size_t)j] = j;
  std::stable_sort(order.begin(), order.end(),
                   [&](int32_t a, int32_t b) { return job.items[(size_t)a].m2 > job.items[(size_t)b].m2; });
  run.d_items.reset(ctx, (size_t)run.cnt);
  run.d_out.reset(ctx, (size_t)run.cnt);
  run.d_order.reset(ctx, (size_t)run.cnt);
  run.d_head.reset(ctx, 1);
  if (want_lv) run.d_lv.reset(ctx, (size_t)run.cnt * GP_MAX_LEVELS);
  run.d_arena.reset(ctx, (size_t)run.grid * (size_t)arena);
  GP_CUDA(cudaMemcpyAsync(run.d_items.get(), job.items.data(), sizeof(EItem) * run.cnt, cudaMemcpyHostToDevice,
                          ctx->stream));
  GP_CUDA(cudaMemcpyAsync(run.d_order.get(), order.data(), sizeof(int32_t) * run.cnt, cudaMemcpyHostToDevice,
                          ctx->stream));
  run.d_head.zero();
  if (want_lv) run.d_lv.zero();
  EArgs a;
  a.items = run.d_items.get();
  a.out = run.d_out.get();
  a.lv = want_lv ? run.d_lv.get() : nullptr;
  a.order = run.d_order.get();
  a.count = run.cnt;
  a.head = run.d_head.get();
  a.arena = run.d_arena.get();
  a.arena_bytes = arena;
  a.profile = (want_lv || getenv("GP_ENGINE_PROFILE")) ? 1 : 0;
  a.cfg = cfg;
  if (timed) {
    GP_CUDA(cudaEventCreate(&run.e0));
    GP_CUDA(cudaEventCreate(&run.e1));
    GP_CUDA(cudaEventRecord(run.e0, ctx->stream));
  }
  K.launch(run.grid, smem_bytes(K.threads), ctx->stream, a);
  GP_LAUNCH_CHECK();
  if (timed) GP_CUDA(cudaEventRecord(run.e1, ctx->stream));
}

// Waits for the engine launch of `run` and returns, per job item, its result;
// the job indices that need the per-graph path (arena too small, or no
// launch at all) are in `retry`.
void engine_end(EngineRun &run, const EngineJob &job, std::vector<EOut> &out, std::vector<gp_level_stats> *lvs,
                std::vector<int32_t> &retry, double *ms) {
  gp_ctx *ctx = run.ctx;
  out.assign((size_t)run.cnt, EOut{});
  retry.clear();
  if (run.grid == 0) {
    for (int32_t j = 0; j < run.cnt; j++) retry.push_back(j);
    return;
  }
  GP_CUDA(cudaMemcpyAsync(out.data(), run.d_out.get(), sizeof(EOut) * run.cnt, cudaMemcpyDeviceToHost, ctx->stream));
  if (lvs && run.want_lv) {
    lvs->resize((size_t)run.cnt * GP_MAX_LEVELS);
    GP_CUDA(cudaMemcpyAsync(lvs->data(), run.d_lv.get(), sizeof(gp_level_stats) * (size_t)run.cnt * GP_MAX_LEVELS,
                            cudaMemcpyDeviceToHost, ctx->stream));
  }
  GP_CUDA(cudaStreamSynchronize(ctx->stream));
  if (ms && run.timed) {
    float f = 0;
    GP_CUDA(cudaEventElapsedTime(&f, run.e0, run.e1));
    *ms = f;
  }
  for (int32_t j = 0; j < run.cnt; j++)
    if (out[(size_t)j].status == kERetry) retry.push_back(j);
  if (getenv("GP_ENGINE_PROFILE")) {
    // per size class (CSR entries up to 4^(c+5)): items and SM cycles of every phase, on stderr
    static const char *names[EP_COUNT] = {"validate", "cluster", "relabel", "contract", "sparsify", "initial",
                                          "refine", "cut"};
    double cyc[GP_TUNE_CLASSES][EP_COUNT] = {};
    int items[GP_TUNE_CLASSES] = {};
    for (int32_t j = 0; j < run.cnt; j++) {
      if (out[(size_t)j].status != GP_OK) continue;
      int q = 0;
      while (q < GP_TUNE_CLASSES - 1 && job.items[(size_t)j].m2 > ((int64_t)1 << (2 * q + 10))) q++;
      items[q]++;
      for (int p = 0; p < EP_COUNT; p++) cyc[q][p] += (double)out[(size_t)j].cyc[p];
    }
    fprintf(stderr, "[gp engine] threads %d grid %d arena %lld B\n", run.threads, run.grid, (long long)run.arena);
    for (int q = 0; q < GP_TUNE_CLASSES; q++) {
      if (!items[q]) continue;
      fprintf(stderr, "[gp engine] entries <= %lld: %d items, Mcycles per item:", (long long)1 << (2 * q + 10),
              items[q]);
      for (int p = 0; p < EP_COUNT; p++) fprintf(stderr, " %s %.3f", names[p], cyc[q][p] / items[q] / 1e6);
      fprintf(stderr, "\n");
    }
  }
}

// The engine alone on the whole device (autotuner): per job item its result.
void engine_launch(gp_ctx *ctx, const EngineJob &job, const gp_config &cfg, int threads, int64_t arena_cap,
                   std::vector<EOut> &out, double *ms) {
  EngineRun run;
  engine_begin(ctx, job, cfg, threads, arena_cap, 0, 1, false, ms != nullptr, run);
  std::vector<int32_t> retry;
  engine_end(run, job, out, nullptr, retry, ms);
}

bool engine_item_ok(const gp_batch_item &it, const gp_batch_tuning &t) {
  return it.g.m2 <= t.max_entries && (int64_t)it.g.n <= t.max_nodes;
}

EItem to_eitem(const gp_batch_item &it) {
  EItem e;
  e.xadj = it.g.xadj; e.adjncy = it.g.adjncy; e.vwgt = it.g.vwgt; e.adjwgt = it.g.adjwgt;
  e.blocks = it.blocks;
  e.m2 = it.g.m2;
  e.eps_ppm = llround(it.eps * 1e6);
  e.seed = it.seed;
  e.n = it.g.n;
  e.k = it.k;
  return e;
}

double now_ms() {
  return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

}  // namespace

bool engine_config_ok(const gp_config &c) {
  return (c.sparsifier == GP_SPARSIFY_NONE || c.sparsifier == GP_SPARSIFY_TWEIGHT ||
          c.sparsifier == GP_SPARSIFY_UNIFORM) &&
         c.lp_subrounds >= 1 && c.lp_subrounds <= 254 && c.ip_trials >= 1 && c.lp_rounds >= 0 &&
         c.ref_rounds >= 0 && c.max_levels >= 0 && c.max_levels <= GP_MAX_LEVELS && c.shrink_num > 0 &&
         c.shrink_den > 0 && c.min_shrink_num > 0 && c.min_shrink_den > 0 && c.tau_e_num >= 0 && c.tau_e_den > 0 &&
         c.tau_d_num >= 0 && c.tau_d_den > 0 && c.rho_num >= 0 && c.rho_den > 0 && c.cluster_factor > 0 &&
         c.coarsest_factor >= 0;
}

const gp_batch_tuning &batch_tuning(gp_ctx *ctx) {
  if (!ctx->tuning_set) {
    gp_batch_tuning_default(&ctx->tuning);
    ctx->tuning_set = true;
  }
  return ctx->tuning;
}

namespace {

void engine_fill(gp_batch_item *items, const EngineJob &job, const std::vector<EOut> &out,
                 const std::vector<gp_level_stats> &lvs, const std::vector<int32_t> &retry, int clock_khz,
                 std::vector<int32_t> &rest) {
  std::vector<char> again(job.items.size(), 0);
  for (int32_t j : retry) again[(size_t)j] = 1;
  for (size_t j = 0; j < job.items.size(); j++) {
    const int32_t i = job.owner[j];
    if (again[j]) { rest.push_back(i); continue; }
    const EOut &o = out[j];
    gp_batch_item &it = items[i];
    it.status = (gp_status)o.status;
    it.cut = o.status == GP_OK ? o.cut : 0;
    it.engine = 1;
    if (it.stats) {
      gp_partition_stats &S = *it.stats;
      memset(&S, 0, sizeof(S));
      if (o.status == GP_OK) {
        S.levels = o.levels;
        for (int l = 0; l < o.levels && l < GP_MAX_LEVELS; l++) S.lv[l] = lvs[j * GP_MAX_LEVELS + (size_t)l];
        S.U = o.U; S.Lmax = o.Lmax; S.W = o.W; S.ip_cut = o.ip_cut; S.cut = o.cut;
        S.rebalance_moves = o.rebalance_moves; S.n_coarsest = o.n_coarsest;
        // time inside the item's CTA, from its SM cycle counts at the maximum SM clock
        const double k = clock_khz > 0 ? 1.0 / clock_khz : 0.0;
        S.ms_coarsen = k * (double)(o.cyc[EP_VALIDATE] + o.cyc[EP_CLUSTER] + o.cyc[EP_RELABEL] +
                                    o.cyc[EP_CONTRACT] + o.cyc[EP_SPARSIFY]);
        S.ms_initial = k * (double)o.cyc[EP_INITIAL];
        S.ms_uncoarsen = k * (double)(o.cyc[EP_REFINE] + o.cyc[EP_CUT]);
        S.ms_total = S.ms_coarsen + S.ms_initial + S.ms_uncoarsen;
      }
    }
  }
}

}  // namespace

void batch_run(gp_ctx *ctx, gp_batch_item *items, const std::vector<int32_t> &idx, int workers, const gp_config &cfg,
               const gp_batch_tuning &t) {
  const bool use = t.engine && engine_config_ok(cfg);
  EngineJob job;
  std::vector<int32_t> rest;
  bool want_stats = false;
  for (int32_t i : idx) {
    if (!use || !engine_item_ok(items[i], t)) { rest.push_back(i); continue; }
    job.items.push_back(to_eitem(items[i]));
    job.owner.push_back(i);
    job.stats.push_back(items[i].stats);
    want_stats = want_stats || items[i].stats != nullptr;
  }
  // the inputs may still be in flight on the context stream: the workers wait for them first
  cudaEvent_t ready;
  GP_CUDA(cudaEventCreateWithFlags(&ready, cudaEventDisableTiming));
  GP_CUDA(cudaEventRecord(ready, ctx->stream));
  const bool both = !job.items.empty() && !rest.empty();
  EngineRun run;
  try {
    // the engine on the context stream, beside the per-graph path (half of the device each)
    if (!job.items.empty())
      engine_begin(ctx, job, cfg, t.threads, t.arena_cap_bytes, t.arena_bytes, both ? 2 : 1, want_stats, false,
                   run);
    batch_per_graph(ctx, items, rest, workers, cfg, both ? 2 * workers : workers, ready);
  } catch (...) {
    cudaStreamSynchronize(ctx->stream);
    cudaEventDestroy(ready);
    throw;
  }
  std::vector<int32_t> again;
  if (!job.items.empty()) {
    std::vector<EOut> out;
    std::vector<gp_level_stats> lvs;
    std::vector<int32_t> retry;
    engine_end(run, job, out, want_stats ? &lvs : nullptr, retry, nullptr);
    int clock_khz = 0;
    if (want_stats) cudaDeviceGetAttribute(&clock_khz, cudaDevAttrClockRate, ctx->device);
    engine_fill(items, job, out, lvs, retry, clock_khz, again);
  }
  // items whose hierarchy outgrew the engine's arena
  batch_per_graph(ctx, items, again, workers, cfg, workers, ready);
  cudaEventDestroy(ready);
}

}  // namespace gp

// ----------------------------------------------------------------- C-ABI

extern "C" {

void gp_batch_tuning_default(gp_batch_tuning *t) {
  if (!t) return;
  memset(t, 0, sizeof(*t));
  t->engine = 1;
  t->threads = 512;
  t->max_entries = (int64_t)1 << 22;
  t->max_nodes = (int64_t)1 << 20;
  t->arena_cap_bytes = 0;
}

gp_status gp_batch_set_tuning(gp_ctx *ctx, const gp_batch_tuning *t) {
  if (!ctx) return GP_ERR_INVALID;
  gp_batch_tuning x;
  if (t) x = *t;
  else gp_batch_tuning_default(&x);
  if (x.threads != 256 && x.threads != 512 && x.threads != 1024) {
    ctx->last_error = "gp_batch_set_tuning: threads must be 256, 512 or 1024";
    return GP_ERR_INVALID;
  }
  if (x.max_entries < 0 || x.max_nodes < 0 || x.arena_cap_bytes < 0 || x.arena_bytes < 0) {
    ctx->last_error = "gp_batch_set_tuning: negative limit";
    return GP_ERR_INVALID;
  }
  ctx->tuning = x;
  ctx->tuning_set = true;
  return GP_OK;
}

gp_status gp_batch_get_tuning(gp_ctx *ctx, gp_batch_tuning *t) {
  if (!ctx || !t) return GP_ERR_INVALID;
  *t = gp::batch_tuning(ctx);
  return GP_OK;
}

gp_status gp_batch_autotune(gp_ctx *ctx, const gp_batch_item *items, int32_t count, int32_t workers,
                            const gp_config *cfg, gp_batch_tuning *out) {
  using namespace gp;
  if (!ctx) return GP_ERR_INVALID;
  if (count < 0 || (count > 0 && !items) || workers < 1 || workers > 64) {
    ctx->last_error = "gp_batch_autotune: bad arguments (count >= 0, items, 1 <= workers <= 64)";
    return GP_ERR_INVALID;
  }
  gp_config c;
  if (cfg) c = *cfg;
  else gp_config_default(&c);
  const double t0 = now_ms();
  gp_batch_tuning T = batch_tuning(ctx);
  T.classes = 0;
  try {
    GP_CUDA(cudaSetDevice(ctx->device));
    if (!engine_config_ok(c)) {
      T.engine = 0;
    } else {
      // size classes by CSR entries: (4^(c+4), 4^(c+5)], the first from 0
      std::vector<std::vector<int32_t>> cls(GP_TUNE_CLASSES);
      for (int32_t i = 0; i < count; i++) {
        const gp_batch_item &it = items[i];
        if (it.g.n <= 0 || it.k < 2 || !(it.eps > 0 && it.eps < 1000)) continue;
        int q = 0;
        while (q < GP_TUNE_CLASSES - 1 && it.g.m2 > ((int64_t)1 << (2 * q + 10))) q++;
        cls[(size_t)q].push_back(i);
      }
      size_t fr = 0, tot = 0;
      GP_CUDA(cudaMemGetInfo(&fr, &tot));
      const int64_t budget = (int64_t)(fr / 3);
      const int sizes[3] = {256, 512, 1024};
      // per class and CTA size: engine graphs/s with the device full of the class's items, and the
      // time of one item in its CTA; per class: the per-graph path's graphs/s
      double egps[GP_TUNE_CLASSES][3] = {}, eitem[GP_TUNE_CLASSES][3] = {};
      cudaEvent_t ready;
      GP_CUDA(cudaEventCreateWithFlags(&ready, cudaEventDisableTiming));
      int nclass = 0;
      for (int q = 0; q < GP_TUNE_CLASSES; q++) {
        T.class_entries[q] = (int64_t)1 << (2 * q + 10);
        T.class_items[q] = (int32_t)cls[(size_t)q].size();
        T.class_threads[q] = 0;
        T.class_engine_gps[q] = 0;
        T.class_path_gps[q] = 0;
        if (cls[(size_t)q].empty()) continue;
        nclass = q + 1;
        const std::vector<int32_t> &S = cls[(size_t)q];
        const int ns = (int)std::min<size_t>(S.size(), 64);
        int64_t nmax = 1, amax = 0;
        for (int j = 0; j < ns; j++) {
          const gp_batch_item &it = items[S[(size_t)j]];
          nmax = std::max<int64_t>(nmax, it.g.n);
          amax = std::max(amax, engine_arena_estimate(it.g.n, it.g.m2, it.k));
        }
        for (int z = 0; z < 3; z++) {
          const Kernel K = engine_kernel(sizes[z]);
          const int resident = engine_resident(ctx, K);
          // replicas of the sample fill the device once (each with its own output)
          int64_t R = std::max<int64_t>(resident, ns);
          R = std::min<int64_t>(R, std::max<int64_t>(1, budget / 2 / (4 * nmax)));
          R = std::min<int64_t>(R, budget / 2 / std::max<int64_t>(amax, 1));
          if (R < 1) continue;
          DBuf<int32_t> outb(ctx, (size_t)R * (size_t)nmax);
          EngineJob job;
          for (int64_t r = 0; r < R; r++) {
            EItem e = to_eitem(items[S[(size_t)(r % ns)]]);
            e.blocks = outb.get() + r * nmax;
            job.items.push_back(e);
          }
          std::vector<EOut> o;
          double ms = 0;
          engine_launch(ctx, job, c, sizes[z], budget / 2, o, &ms);
          bool ok = true;
          for (const EOut &x : o) ok = ok && x.status == GP_OK;
          if (!ok || ms <= 0) continue;
          const int64_t waves = (R + std::min<int64_t>(R, resident) - 1) / std::min<int64_t>(R, resident);
          egps[q][z] = (double)R / (ms * 1e-3);
          eitem[q][z] = ms / (double)waves;
          if (egps[q][z] > T.class_engine_gps[q]) {
            T.class_engine_gps[q] = egps[q][z];
            T.class_threads[q] = sizes[z];
          }
        }
        // the per-graph path on (a copy of) the sample
        {
          const int np = std::min(ns, std::max(2 * workers, 4));
          std::vector<gp_batch_item> tmp((size_t)np);
          std::vector<DBuf<int32_t>> outs((size_t)np);
          std::vector<int32_t> idx;
          for (int j = 0; j < np; j++) {
            tmp[(size_t)j] = items[S[(size_t)j]];
            outs[(size_t)j].reset(ctx, (size_t)std::max(1, tmp[(size_t)j].g.n));
            tmp[(size_t)j].blocks = outs[(size_t)j].get();
            tmp[(size_t)j].stats = nullptr;
            idx.push_back(j);
          }
          GP_CUDA(cudaEventRecord(ready, ctx->stream));
          GP_CUDA(cudaStreamSynchronize(ctx->stream));
          const double a = now_ms();
          batch_per_graph(ctx, tmp.data(), idx, workers, c, workers, ready);
          for (int w = 0; w < workers && w < (int)ctx->workers.size(); w++)
            GP_CUDA(cudaStreamSynchronize(ctx->workers[(size_t)w]->stream));
          const double b = now_ms();
          T.class_path_gps[q] = b > a ? np / ((b - a) * 1e-3) : 0;
        }
      }
      cudaEventDestroy(ready);
      T.classes = nclass;
      // the split: the engine takes the classes up to p (every one measured), the per-graph path
      // the rest; predicted time of the batch = engine work + path work, and no less than one
      // engine item in its CTA; the CTA size with the smallest prediction
      double best = -1;
      int best_p = -1, best_z = 1;
      for (int z = 0; z < 3; z++) {
        for (int p = -1; p < nclass; p++) {
          double te = 0, tp = 0, tmax = 0;
          bool ok = true;
          for (int q = 0; q < nclass; q++) {
            const double nq = (double)cls[(size_t)q].size();
            if (nq == 0) continue;
            if (q <= p) {
              if (egps[q][z] <= 0) { ok = false; break; }
              te += nq / egps[q][z];
              tmax = std::max(tmax, eitem[q][z] * 1e-3);
            } else {
              tp += T.class_path_gps[q] > 0 ? nq / T.class_path_gps[q] : 1e30;
            }
          }
          if (!ok) break;  // larger prefixes include an unmeasured class too
          const double pred = std::max(te + tp, tmax);
          if (best < 0 || pred < best) { best = pred; best_p = p; best_z = z; }
        }
      }
      T.engine = best_p >= 0 ? 1 : 0;
      T.max_entries = best_p >= 0 ? T.class_entries[best_p] : 0;
      T.threads = sizes[best_z];
    }
  } catch (const gp::Error &e) {
    ctx->last_error = e.msg;
    return e.status;
  }
  T.tune_ms = now_ms() - t0;
  ctx->tuning = T;
  ctx->tuning_set = true;
  if (out) *out = T;
  return GP_OK;
}

}  // extern "C"
