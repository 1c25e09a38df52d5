// api.cu -- the C-ABI of include/gp.h: argument checks, error capture and
// the context.  No exception crosses this boundary.
#include "lp.cuh"

namespace {

using gp::Error;

template <typename F>
gp_status guarded(gp_ctx *ctx, F &&f) {
  if (!ctx) return GP_ERR_INVALID;
  try {
    int cur = -1;
    if (cudaGetDevice(&cur) == cudaSuccess && cur != ctx->device) GP_CUDA(cudaSetDevice(ctx->device));
    f();
    ctx->last_error.clear();
    return GP_OK;
  } catch (const Error &e) {
    ctx->last_error = e.msg;
    return e.status;
  } catch (const std::bad_alloc &) {
    ctx->last_error = "host allocation failed";
    return GP_ERR_OOM;
  } catch (...) {
    ctx->last_error = "unexpected internal error";
    return GP_ERR_CUDA;
  }
}

void check_graph(const gp_graph *g) {
  GP_REQUIRE(g != nullptr, GP_ERR_INVALID, "graph is NULL");
  GP_REQUIRE(g->n >= 0 && g->m2 >= 0 && g->m2 < ((int64_t)1 << 31), GP_ERR_INVALID,
             "graph sizes out of range (n >= 0, 0 <= m2 < 2^31)");
  GP_REQUIRE(g->n == 0 || (g->xadj && g->vwgt), GP_ERR_INVALID, "graph arrays are NULL");
  GP_REQUIRE(g->m2 == 0 || (g->adjncy && g->adjwgt), GP_ERR_INVALID, "graph arrays are NULL");
}

gp_config cfg_or_default(const gp_config *cfg) {
  gp_config c;
  if (cfg) c = *cfg;
  else gp_config_default(&c);
  return c;
}

const char *kProfNames[gp::PROF_COUNT_] = {
    "lp_rate",  "lp_accept", "refine_rate", "refine_accept", "round_setup", "two_hop",
    "relabel",  "contract",  "contract_aux", "sparsify",     "initial",     "project",
    "cut",      "validate",  "sort",         "scan",          "lp_overflow", "lp_apply",
    "refine_overflow", "refine_apply", "rebalance", "lp_small", "refine_small"};

}  // namespace

extern "C" {

void gp_config_default(gp_config *c) {
  if (!c) return;
  memset(c, 0, sizeof(*c));
  c->tau_e_num = 1; c->tau_e_den = 2;
  c->tau_d_num = 1; c->tau_d_den = 2;
  c->rho_num = 4; c->rho_den = 1;
  c->cluster_factor = 160;
  c->coarsest_factor = 160;
  c->shrink_num = 5; c->shrink_den = 2;
  c->min_shrink_num = 21; c->min_shrink_den = 20;
  c->lp_rounds = 5; c->lp_subrounds = 8;
  c->ref_rounds = 5;
  c->ip_trials = 8;
  c->sparsifier = GP_SPARSIFY_TWEIGHT;
  c->two_hop = 1; c->isolated = 1;
  c->max_levels = GP_MAX_LEVELS;
  c->dbg_max_subrounds = -1;
  c->validate = 1;
  c->small_lp_nodes = gp::kLpSmallMaxNodes;
}

void gp_set_wait_limit(gp_ctx *ctx, int64_t spins) {
  if (ctx) ctx->wait_spins = spins;
}

const char *gp_version(void) { return "gp-gb300 1.0 (sm_103a)"; }

int64_t gp_launch_count(void) { return gp::g_launch_count.load(); }

gp_status gp_create(gp_ctx **out, int device, void *stream, const gp_allocator *alloc) {
  if (!out) return GP_ERR_INVALID;
  *out = nullptr;
  gp_ctx *ctx = nullptr;
  try {
    ctx = new gp_ctx();
  } catch (...) {
    return GP_ERR_OOM;
  }
  ctx->device = device;
  ctx->stream = (cudaStream_t)stream;
  if (alloc && alloc->alloc && alloc->free) ctx->alloc = *alloc;
  gp_status st = guarded(ctx, [&] {
    GP_CUDA(cudaSetDevice(device));
    GP_CUDA(cudaDeviceGetAttribute(&ctx->num_sms, cudaDevAttrMultiProcessorCount, device));
    GP_CUDA(cudaMallocHost((void **)&ctx->h_stage, 4096 * sizeof(int64_t)));
    if (!ctx->alloc.alloc) {
      // a private pool that keeps freed memory for reuse: allocations in the level loop
      // then cost no driver call
      cudaMemPoolProps props{};
      props.allocType = cudaMemAllocationTypePinned;
      props.location.type = cudaMemLocationTypeDevice;
      props.location.id = device;
      GP_CUDA(cudaMemPoolCreate(&ctx->pool, &props));
      uint64_t keep = UINT64_MAX;
      GP_CUDA(cudaMemPoolSetAttribute(ctx->pool, cudaMemPoolAttrReleaseThreshold, &keep));
    }
    void *p = nullptr;
    GP_CUDA(cudaMalloc(&p, sizeof(unsigned long long) * gp::PROF_COUNT_ * gp::PROF_UNITS));
    ctx->d_units = (unsigned long long *)p;
    GP_CUDA(cudaMemset(p, 0, sizeof(unsigned long long) * gp::PROF_COUNT_ * gp::PROF_UNITS));
  });
  if (st != GP_OK) {
    gp_destroy(ctx);
    return st;
  }
  *out = ctx;
  return GP_OK;
}

void gp_destroy(gp_ctx *ctx) {
  if (!ctx) return;
  cudaSetDevice(ctx->device);
  for (gp_ctx *w : ctx->workers) {
    cudaStream_t s = w->stream;
    gp_destroy(w);
    cudaStreamDestroy(s);
  }
  ctx->workers.clear();
  cudaStreamSynchronize(ctx->stream);
  for (auto &r : ctx->pending) {
    cudaEventDestroy(r.a);
    cudaEventDestroy(r.b);
  }
  for (auto e : ctx->free_events) cudaEventDestroy(e);
  for (auto st : ctx->copy_streams)
    if (st) cudaStreamDestroy(st);
  for (auto ev : ctx->copy_events)
    if (ev) cudaEventDestroy(ev);
  if (ctx->h_stage) cudaFreeHost(ctx->h_stage);
  if (ctx->d_units) cudaFree(ctx->d_units);
  if (ctx->pool) cudaMemPoolDestroy(ctx->pool);  // released once its last allocation is freed
  delete ctx;
}

const char *gp_last_error(const gp_ctx *ctx) { return ctx ? ctx->last_error.c_str() : "no context"; }

gp_status gp_coarsen(gp_ctx *ctx, const gp_graph *g, int64_t U, int32_t level, uint64_t seed,
                     const gp_config *cfg, int32_t *cmap, int32_t *label, int32_t *n_coarse,
                     gp_level_stats *stats) {
  return guarded(ctx, [&] {
    check_graph(g);
    GP_REQUIRE(cmap && n_coarse, GP_ERR_INVALID, "cmap and n_coarse are required");
    GP_REQUIRE(U >= 1, GP_ERR_INVALID, "U must be >= 1");
    GP_REQUIRE(level >= 0 && level <= 0xFFFF, GP_ERR_INVALID, "level must be in [0, 65535]");
    const gp_config c = cfg_or_default(cfg);
    GP_REQUIRE(c.shrink_num > 0 && c.shrink_den > 0, GP_ERR_INVALID, "bad shrink factor");
    gp::LevelOut lo;
    gp::coarsen_level(ctx, gp::DevGraph::wrap(*g), U, level, seed, c, cmap, label, lo);
    *n_coarse = lo.n_coarse;
    lo.st.m = g->m2 / 2;
    if (stats) *stats = lo.st;
  });
}

gp_status gp_contract(gp_ctx *ctx, const gp_graph *g, const int32_t *cmap, int32_t n_coarse,
                      gp_graph *out) {
  return guarded(ctx, [&] {
    check_graph(g);
    GP_REQUIRE(out, GP_ERR_INVALID, "out is NULL");
    GP_REQUIRE(n_coarse >= 0 && n_coarse <= g->n && (g->n == 0 || (cmap && n_coarse >= 1)),
               GP_ERR_INVALID, "n_coarse must be in [1, n]");
    gp::DevGraph res;
    gp::contract_graph(ctx, gp::DevGraph::wrap(*g), cmap, n_coarse, res);
    gp::export_graph(ctx, std::move(res), out);
  });
}

gp_status gp_sparsify(gp_ctx *ctx, const gp_graph *g, int64_t m_hat, int32_t level, uint64_t seed,
                      int32_t mode, gp_graph *out, gp_level_stats *stats) {
  return guarded(ctx, [&] {
    check_graph(g);
    GP_REQUIRE(out, GP_ERR_INVALID, "out is NULL");
    GP_REQUIRE(level >= 0 && level <= 0xFFFF, GP_ERR_INVALID, "level must be in [0, 65535]");
    gp_level_stats st{};
    gp::DevGraph res;
    gp::sparsify_graph(ctx, gp::DevGraph::wrap(*g), m_hat, level, seed, mode, res, &st);
    st.m = g->m2 / 2;
    st.m_hat = m_hat;
    gp::export_graph(ctx, std::move(res), out);
    if (stats) *stats = st;
  });
}

gp_status gp_partition(gp_ctx *ctx, const gp_graph *g, int32_t k, double eps, uint64_t seed,
                       const gp_config *cfg, int32_t *blocks, int64_t *cut, gp_partition_stats *stats) {
  return guarded(ctx, [&] {
    check_graph(g);
    GP_REQUIRE(blocks || g->n == 0, GP_ERR_INVALID, "blocks is NULL");
    const gp_config c = cfg_or_default(cfg);
    gp::partition_impl(ctx, gp::DevGraph::wrap(*g), k, eps, seed, c, blocks, cut, stats);
  });
}

gp_status gp_partition_host(gp_ctx *ctx, int32_t n, int64_t m2, const int32_t *xadj, const int32_t *adjncy,
                            const int32_t *vwgt, const int32_t *adjwgt, int32_t k, double eps,
                            uint64_t seed, const gp_config *cfg, int32_t *blocks, int64_t *cut,
                            gp_partition_stats *stats) {
  return guarded(ctx, [&] {
    GP_REQUIRE(n >= 0 && m2 >= 0 && m2 < ((int64_t)1 << 31), GP_ERR_INVALID, "sizes out of range");
    GP_REQUIRE(n == 0 || (xadj && vwgt && blocks), GP_ERR_INVALID, "host arrays are NULL");
    GP_REQUIRE(m2 == 0 || (adjncy && adjwgt), GP_ERR_INVALID, "host arrays are NULL");
    const gp_config c = cfg_or_default(cfg);
    gp::DevGraph d;
    d.allocate(ctx, n, m2);
    gp::DBuf<int32_t> b(ctx, (size_t)n);
    gp::copy_to_device(ctx, {{d.xadj, xadj, sizeof(int32_t) * ((size_t)n + 1)},
                             {d.adjncy, adjncy, sizeof(int32_t) * (size_t)m2},
                             {d.adjwgt, adjwgt, sizeof(int32_t) * (size_t)m2},
                             {d.vwgt, vwgt, sizeof(int32_t) * (size_t)n}});
    gp::partition_impl(ctx, d, k, eps, seed, c, b.get(), cut, stats);
    if (n > 0) GP_CUDA(cudaMemcpyAsync(blocks, b.get(), sizeof(int32_t) * n, cudaMemcpyDeviceToHost, ctx->stream));
    GP_CUDA(cudaStreamSynchronize(ctx->stream));
  });
}

gp_status gp_initial_partition(gp_ctx *ctx, const gp_graph *g, int32_t k, double eps, uint64_t seed,
                               const gp_config *cfg, int32_t *blocks) {
  return guarded(ctx, [&] {
    check_graph(g);
    GP_REQUIRE(k >= 1 && eps > 0, GP_ERR_INVALID, "k >= 1 and eps > 0 required");
    GP_REQUIRE(blocks || g->n == 0, GP_ERR_INVALID, "blocks is NULL");
    const gp_config c = cfg_or_default(cfg);
    gp::initial_partition(ctx, gp::DevGraph::wrap(*g), k, llround(eps * 1e6), seed, c.ip_trials, blocks);
    GP_CUDA(cudaStreamSynchronize(ctx->stream));
  });
}

gp_status gp_rebalance(gp_ctx *ctx, const gp_graph *g, int32_t k, int64_t Lmax, int32_t *blocks,
                       int64_t *moves) {
  return guarded(ctx, [&] {
    check_graph(g);
    GP_REQUIRE(k >= 1, GP_ERR_INVALID, "k must be >= 1");
    gp::check_blocks(ctx, blocks, g->n, k);
    const int64_t mv = gp::rebalance_blocks(ctx, gp::DevGraph::wrap(*g), k, Lmax, blocks);
    if (moves) *moves = mv;
  });
}

gp_status gp_refine(gp_ctx *ctx, const gp_graph *g, int32_t k, int64_t Lmax, int32_t level, uint64_t seed,
                    const gp_config *cfg, int32_t *blocks, int64_t *moves) {
  return guarded(ctx, [&] {
    check_graph(g);
    GP_REQUIRE(k >= 1, GP_ERR_INVALID, "k must be >= 1");
    GP_REQUIRE(level >= 0 && level <= 0xFFFF, GP_ERR_INVALID, "level must be in [0, 65535]");
    gp::check_blocks(ctx, blocks, g->n, k);
    const gp_config c = cfg_or_default(cfg);
    const int64_t mv = gp::refine_blocks(ctx, gp::DevGraph::wrap(*g), k, Lmax, level, seed, c, blocks);
    GP_CUDA(cudaStreamSynchronize(ctx->stream));
    if (moves) *moves = mv;
  });
}

gp_status gp_project(gp_ctx *ctx, int32_t n, const int32_t *cmap, const int32_t *coarse, int32_t *fine) {
  return guarded(ctx, [&] {
    GP_REQUIRE(n >= 0 && (n == 0 || (cmap && coarse && fine)), GP_ERR_INVALID, "bad projection arguments");
    gp::project(ctx, n, cmap, coarse, fine);
  });
}

gp_status gp_cut(gp_ctx *ctx, const gp_graph *g, const int32_t *blocks, int32_t k, int64_t *cut,
                 int64_t *block_weights) {
  return guarded(ctx, [&] {
    check_graph(g);
    GP_REQUIRE(k >= 1 && (blocks || g->n == 0), GP_ERR_INVALID, "bad cut arguments");
    gp::check_blocks(ctx, blocks, g->n, k);
    gp::cut_and_weights(ctx, gp::DevGraph::wrap(*g), blocks, k, cut, block_weights);
  });
}

void gp_graph_release(gp_ctx *ctx, gp_graph *g) {
  if (!ctx || !g) return;
  try {
    gp::dev_free(ctx, g->xadj, sizeof(int32_t) * ((size_t)g->n + 1));
    gp::dev_free(ctx, g->adjncy, sizeof(int32_t) * (size_t)(g->m2 ? g->m2 : 1));
    gp::dev_free(ctx, g->vwgt, sizeof(int32_t) * (size_t)(g->n ? g->n : 1));
    gp::dev_free(ctx, g->adjwgt, sizeof(int32_t) * (size_t)(g->m2 ? g->m2 : 1));
  } catch (...) {
  }
  memset(g, 0, sizeof(*g));
}

void gp_profile_enable(gp_ctx *ctx, int on) {
  if (ctx) ctx->profile = on != 0;
}

void gp_profile_reset(gp_ctx *ctx) {
  if (!ctx) return;
  cudaStreamSynchronize(ctx->stream);
  for (auto &r : ctx->pending) {
    ctx->free_events.push_back(r.a);
    ctx->free_events.push_back(r.b);
  }
  ctx->pending.clear();
  for (int i = 0; i < gp::PROF_COUNT_; i++) {
    ctx->prof_ms[i] = 0;
    ctx->prof_launches[i] = 0;
    ctx->prof_host_bytes[i] = 0;
  }
  if (ctx->d_units)
    cudaMemsetAsync(ctx->d_units, 0, sizeof(unsigned long long) * gp::PROF_COUNT_ * gp::PROF_UNITS, ctx->stream);
  cudaStreamSynchronize(ctx->stream);
}

int gp_profile_count(void) { return gp::PROF_COUNT_; }

const char *gp_profile_name(int i) { return (i >= 0 && i < gp::PROF_COUNT_) ? kProfNames[i] : ""; }

gp_status gp_profile_read(gp_ctx *ctx, int i, int64_t *launches, double *ms, double *bytes) {
  return guarded(ctx, [&] {
    GP_REQUIRE(i >= 0 && i < gp::PROF_COUNT_, GP_ERR_INVALID, "profile class out of range");
    GP_CUDA(cudaStreamSynchronize(ctx->stream));
    for (auto &r : ctx->pending) {
      float f = 0;
      GP_CUDA(cudaEventElapsedTime(&f, r.a, r.b));
      ctx->prof_ms[r.cls] += f;
      ctx->prof_launches[r.cls] += 1;
      ctx->free_events.push_back(r.a);
      ctx->free_events.push_back(r.b);
    }
    ctx->pending.clear();
    unsigned long long u[gp::PROF_UNITS] = {};
    if (ctx->d_units)
      gp::read_back(ctx, ctx->d_units + (size_t)i * gp::PROF_UNITS, sizeof(u), u);
    // algorithmic bytes: each unit at its own width, counted once
    double b = 0;
    switch (i) {
      case gp::PROF_LP_RATE:
      case gp::PROF_REF_RATE:
      case gp::PROF_LP_SMALL:
      case gp::PROF_REF_SMALL:
        // per entry: neighbour id, edge weight, neighbour label (12 B, 9 B when the
        // labels are one byte); per candidate label its weight (4 B); per node
        // offsets, weight, own label (16 B); per proposal target write + incoming
        // update (12 B)
        // (the weight is not read on unit-weight inputs)
        b = 12.0 * u[0] - 3.0 * u[4] - 4.0 * u[5] + 4.0 * u[2] + 16.0 * u[1] + 12.0 * u[3];
        break;
      case gp::PROF_CONTRACT:
        // map: per fine entry neighbour id, weight, coarse id of the neighbour read (12 B) and
        // (coarse neighbour, weight) written to the segment (8 B); merge: every segment entry
        // read (8 B), every merged entry written (8 B)
        b = 28.0 * u[0] - 4.0 * u[5] + 8.0 * u[3];
        break;
      default:
        b = ctx->prof_host_bytes[i];
    }
    if (launches) *launches = ctx->prof_launches[i];
    if (ms) *ms = ctx->prof_ms[i];
    if (bytes) *bytes = b;
  });
}

gp_status gp_modularity(gp_ctx *ctx, const gp_graph *g, const int32_t *labels, int32_t nlabels,
                        gp_modularity_stats *out) {
  return guarded(ctx, [&] {
    GP_REQUIRE(g && out, GP_ERR_INVALID, "null argument");
    gp::DevGraph dg = gp::DevGraph::wrap(*g);
    gp::validate_graph(ctx, dg, false);
    gp::modularity(ctx, dg, labels, nlabels, out);
  });
}

gp_status gp_measure_random_reads(gp_ctx *ctx, int64_t array_bytes, int64_t reads, double *reads_per_s) {
  return guarded(ctx, [&] {
    GP_REQUIRE(reads_per_s, GP_ERR_INVALID, "null output");
    *reads_per_s = gp::measure_random_reads(ctx, array_bytes, reads);
  });
}

}  // extern "C"
