// partition.cu -- input validation, projection, cut, LP refinement and the
// multilevel driver (Sec. 2, Alg. 1, Sec. 4.3).
#include "lp.cuh"

#include <memory>

namespace gp {

namespace {

constexpr unsigned FULL = 0xFFFFFFFFu;

enum ValErr : int {
  VE_XADJ = 1, VE_VWGT = 2, VE_RANGE = 4, VE_LOOP = 8, VE_AWGT = 16, VE_ORDER = 32, VE_SYM = 64
};

struct ValOut {
  int err;
  int cmax;
  unsigned long long csum, wsum, hlo, hhi, nlo, nhi;
};

__global__ void k_validate_nodes(const int32_t *xadj, const int32_t *vwgt, int n, int64_t m2, ValOut *o) {
  int err = 0, cm = 0;
  unsigned long long cs = 0;
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n;
       v += (int64_t)gridDim.x * blockDim.x) {
    if (xadj[v + 1] < xadj[v]) err |= VE_XADJ;
    const int c = vwgt[v];
    if (c <= 0) err |= VE_VWGT;
    else { cs += (unsigned long long)c; cm = c > cm ? c : cm; }
  }
  if (blockIdx.x == 0 && threadIdx.x == 0 && (xadj[0] != 0 || (int64_t)xadj[n] != m2)) err |= VE_XADJ;
  cs = warp_sum(cs);
  cm = warp_max(cm);
  err = __reduce_or_sync(FULL, err);
  if (lane_id() == 0) {
    if (err) atomicOr(&o->err, err);
    if (cm) atomicMax(&o->cmax, cm);
    if (cs) atomicAdd(&o->csum, cs);
  }
}

__device__ __forceinline__ unsigned long long pair_hash(uint32_t lo, uint32_t hi, int w) {
  return fmix(((((uint64_t)lo << 32) | hi) + (uint64_t)(uint32_t)w * kGold) ^ kGold);
}

// Entry checks: ids in range, no self-loop, positive weights, strictly
// increasing rows, and symmetry by comparing, over the entries below and
// above the diagonal, their counts and the sums of a 64-bit hash of
// (min, max, weight) (equal sums unless the graph is asymmetric, up to a
// 2^-64 collision).  Runs after the row offsets were checked; a warp walks 32
// consecutive rows (one contiguous range of entries) at a time.
constexpr int kValUnroll = 4;

__global__ void __launch_bounds__(256) k_validate_entries(const int32_t *xadj, const int32_t *adjncy,
                                                          const int32_t *adjwgt, int n, int64_t m2,
                                                          ValOut *o) {
  const int lane = (int)lane_id();
  const int wid = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5);
  const int nw = (int)((gridDim.x * blockDim.x) >> 5);
  int err = 0;
  unsigned long long ws = 0, hlo = 0, hhi = 0, nlo = 0, nhi = 0;
  for (int64_t u0 = (int64_t)wid * 32; u0 < n; u0 += (int64_t)nw * 32) {
    const int64_t u = u0 + lane;
    const bool valid = u < n;
    const int xs = valid ? xadj[u] : 0x7FFFFFFF;
    const int xe = valid ? xadj[u + 1] : 0x7FFFFFFF;
    const int e0 = __shfl_sync(FULL, xs, 0);
    const int last = (int)((n - u0) < 32 ? (n - u0) : 32) - 1;
    const int e1 = __shfl_sync(FULL, xe, last);
    for (int f0 = e0; f0 < e1; f0 += 32 * kValUnroll) {
      int e[kValUnroll], row[kValUnroll], rs[kValUnroll], v[kValUnroll], w[kValUnroll], pv[kValUnroll];
#pragma unroll
      for (int r = 0; r < kValUnroll; r++) {
        e[r] = f0 + r * 32 + lane;
        int q = 0;  // owner: lanes whose row ends at or before e
#pragma unroll
        for (int step = 16; step > 0; step >>= 1) {
          const int val = __shfl_sync(FULL, xe, q + step - 1);
          if (val <= e[r]) q += step;
        }
        row[r] = (int)(u0 + q);
        rs[r] = __shfl_sync(FULL, xs, q);
      }
#pragma unroll
      for (int r = 0; r < kValUnroll; r++) {
        const bool in = e[r] < e1;
        v[r] = in ? adjncy[e[r]] : 0;
        w[r] = in ? adjwgt[e[r]] : 1;
        pv[r] = in && e[r] > rs[r] ? adjncy[e[r] - 1] : -1;
      }
#pragma unroll
      for (int r = 0; r < kValUnroll; r++) {
        if (e[r] >= e1) continue;
        if (v[r] < 0 || v[r] >= n) { err |= VE_RANGE; continue; }
        if (v[r] == row[r]) err |= VE_LOOP;
        if (w[r] <= 0) err |= VE_AWGT;
        ws += (unsigned long long)(w[r] > 0 ? w[r] : 0);
        if (pv[r] >= v[r]) err |= VE_ORDER;
        if (row[r] < v[r]) { hlo += pair_hash((uint32_t)row[r], (uint32_t)v[r], w[r]); nlo++; }
        else { hhi += pair_hash((uint32_t)v[r], (uint32_t)row[r], w[r]); nhi++; }
      }
    }
  }
  ws = warp_sum(ws); hlo = warp_sum(hlo); hhi = warp_sum(hhi); nlo = warp_sum(nlo); nhi = warp_sum(nhi);
  err = __reduce_or_sync(FULL, err);
  if (lane == 0) {
    if (err) atomicOr(&o->err, err);
    atomicAdd(&o->wsum, ws);
    atomicAdd(&o->hlo, hlo);
    atomicAdd(&o->hhi, hhi);
    atomicAdd(&o->nlo, nlo);
    atomicAdd(&o->nhi, nhi);
  }
}

__global__ void k_project(int n, const int32_t *cmap, const int32_t *coarse, int32_t *fine) {
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n;
       v += (int64_t)gridDim.x * blockDim.x)
    fine[v] = coarse[cmap[v]];
}

// cut = 1/2 sum over CSR entries whose endpoints lie in different blocks: a
// warp walks 32 consecutive rows (one contiguous range of entries), finds each
// entry's row among its lanes by a shuffle search, and keeps four entries per
// lane in flight.
template <typename B>
__global__ void __launch_bounds__(256) k_cut(const int32_t *xadj, const int32_t *adjncy,
                                             const int32_t *adjwgt, const B *blk, int n,
                                             unsigned long long *cut) {
  constexpr int R = 4;
  const int lane = (int)lane_id();
  const int wid = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5);
  const int nw = (int)((gridDim.x * blockDim.x) >> 5);
  unsigned long long s = 0;
  for (int64_t u0 = (int64_t)wid * 32; u0 < n; u0 += (int64_t)nw * 32) {
    const int64_t u = u0 + lane;
    const bool valid = u < n;
    const int xe = valid ? xadj[u + 1] : 0x7FFFFFFF;
    const int bu = valid ? (int)blk[u] : -1;
    const int e0 = __shfl_sync(FULL, valid ? xadj[u] : 0, 0);
    const int last = (int)((n - u0) < 32 ? (n - u0) : 32) - 1;
    const int e1 = __shfl_sync(FULL, xe, last);
    for (int f0 = e0; f0 < e1; f0 += 32 * R) {
      int e[R], bo[R], v[R], w[R];
#pragma unroll
      for (int r = 0; r < R; r++) {
        e[r] = f0 + r * 32 + lane;
        int q = 0;  // owner: lanes whose row ends at or before e
#pragma unroll
        for (int step = 16; step > 0; step >>= 1) {
          const int val = __shfl_sync(FULL, xe, q + step - 1);
          if (val <= e[r]) q += step;
        }
        bo[r] = __shfl_sync(FULL, bu, q);
      }
#pragma unroll
      for (int r = 0; r < R; r++) {
        const bool in = e[r] < e1;
        v[r] = in ? __ldcs(adjncy + e[r]) : 0;
        w[r] = in ? (adjwgt ? __ldcs(adjwgt + e[r]) : 1) : 0;
      }
#pragma unroll
      for (int r = 0; r < R; r++)
        if (e[r] < e1 && (int)blk[v[r]] != bo[r]) s += (unsigned long long)w[r];
    }
  }
  s = warp_sum(s);
  if (lane == 0 && s) atomicAdd(cut, s);
}

__global__ void k_bweights(const int32_t *blk, const int32_t *vwgt, int n, int k, unsigned long long *bw) {
  extern __shared__ unsigned long long s_bw[];
  for (int b = threadIdx.x; b < k; b += blockDim.x) s_bw[b] = 0;
  __syncthreads();
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n;
       v += (int64_t)gridDim.x * blockDim.x)
    atomicAdd(&s_bw[blk[v]], (unsigned long long)vwgt[v]);
  __syncthreads();
  for (int b = threadIdx.x; b < k; b += blockDim.x)
    if (s_bw[b]) atomicAdd(&bw[b], s_bw[b]);
}

__global__ void k_bweights_global(const int32_t *blk, const int32_t *vwgt, int n, unsigned long long *bw) {
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n;
       v += (int64_t)gridDim.x * blockDim.x)
    atomicAdd(&bw[blk[v]], (unsigned long long)vwgt[v]);
}

// narrow copy of block ids (fewer than 256 blocks): a quarter of the bytes to gather
__global__ void k_narrow(const int32_t *a, int64_t n, uint8_t *b) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    b[i] = (uint8_t)a[i];
}

__global__ void k_to_i32(const unsigned long long *a, int k, int32_t *b) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < k; i += gridDim.x * blockDim.x) b[i] = (int32_t)a[i];
}

__global__ void k_check_blocks(const int32_t *blk, int n, int k, int *bad) {
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n;
       v += (int64_t)gridDim.x * blockDim.x)
    if (blk[v] < 0 || blk[v] >= k) atomicOr(bad, 1);
}

void block_weights_dev(gp_ctx *ctx, const DevGraph &g, const int32_t *blocks, int32_t k,
                       unsigned long long *bw) {
  GP_CUDA(cudaMemsetAsync(bw, 0, sizeof(unsigned long long) * k, ctx->stream));
  if (g.n == 0) return;
  if (k <= 4096) {
    k_bweights<<<grid_for(g.n, 256, ctx->num_sms * 4), 256, sizeof(unsigned long long) * k, ctx->stream>>>(
        blocks, g.vwgt, g.n, k, bw);
    GP_LAUNCH_CHECK();
  } else {
    k_bweights_global<<<grid_for(g.n, 256, ctx->num_sms * 8), 256, 0, ctx->stream>>>(blocks, g.vwgt, g.n, bw);
    GP_LAUNCH_CHECK();
  }
}

}  // namespace

GraphTotals validate_graph(gp_ctx *ctx, const DevGraph &g, bool full) {
  ProfScope ps(ctx, PROF_VALIDATE);
  GP_REQUIRE(g.n >= 0, GP_ERR_INVALID, "n must be >= 0");
  GP_REQUIRE(g.m2 >= 0 && g.m2 < ((int64_t)1 << 31), GP_ERR_INVALID, "m2 must be in [0, 2^31)");
  GP_REQUIRE(g.n == 0 || (g.xadj && g.vwgt), GP_ERR_INVALID, "null graph arrays");
  GP_REQUIRE(g.m2 == 0 || (g.adjncy && g.adjwgt), GP_ERR_INVALID, "null graph arrays");
  if (g.n == 0) return GraphTotals{0, 0, false};
  DBuf<ValOut> o(ctx, 1);
  o.zero();
  k_validate_nodes<<<grid_for(g.n, 256, ctx->num_sms * 8), 256, 0, ctx->stream>>>(g.xadj, g.vwgt, g.n, g.m2,
                                                                                  o.get());
  GP_LAUNCH_CHECK();
  ValOut h;
  read_back(ctx, o.get(), sizeof(ValOut), &h);
  GP_REQUIRE(!(h.err & VE_XADJ), GP_ERR_INVALID, "xadj is not a valid row-offset array");
  GP_REQUIRE(!(h.err & VE_VWGT), GP_ERR_INVALID, "node weights must be > 0");
  GP_REQUIRE(h.csum <= 0x7FFFFFFFull, GP_ERR_OVERFLOW, "total node weight exceeds 2^31 - 1");
  prof_bytes(ctx, PROF_VALIDATE, 8.0 * g.n + 8.0 * g.m2);  // offsets, node weights, ids, edge weights
  if (g.m2 > 0) {
    k_validate_entries<<<grid_for(g.n, 256, ctx->num_sms * 16), 256, 0, ctx->stream>>>(
        g.xadj, g.adjncy, g.adjwgt, g.n, g.m2, o.get());
    GP_LAUNCH_CHECK();
    read_back(ctx, o.get(), sizeof(ValOut), &h);
    GP_REQUIRE(!(h.err & VE_RANGE), GP_ERR_INVALID, "neighbour id out of range");
    GP_REQUIRE(!(h.err & VE_LOOP), GP_ERR_INVALID, "self-loop");
    GP_REQUIRE(!(h.err & VE_AWGT), GP_ERR_INVALID, "edge weights must be > 0");
    GP_REQUIRE(!(h.err & VE_ORDER), GP_ERR_INVALID, "rows must be strictly increasing (sorted, no duplicates)");
    if (full)
      GP_REQUIRE(h.nlo == h.nhi && h.hlo == h.hhi, GP_ERR_INVALID, "graph is not symmetric");
    GP_REQUIRE(h.wsum / 2 <= 0x7FFFFFFFull, GP_ERR_OVERFLOW, "total edge weight exceeds 2^31 - 1");
  }
  // all weights are >= 1, so a total equal to the entry count means all are 1
  return GraphTotals{(int64_t)h.csum, (int64_t)h.cmax, g.m2 > 0 && (int64_t)h.wsum == g.m2};
}

void project(gp_ctx *ctx, int32_t n, const int32_t *cmap, const int32_t *coarse, int32_t *fine) {
  ProfScope ps(ctx, PROF_PROJECT);
  if (n <= 0) return;
  k_project<<<grid_for(n, 256, ctx->num_sms * 8), 256, 0, ctx->stream>>>(n, cmap, coarse, fine);
  GP_LAUNCH_CHECK();
  prof_bytes(ctx, PROF_PROJECT, 12.0 * n);  // coarse id read, coarse block gathered, fine block written
}

void cut_and_weights(gp_ctx *ctx, const DevGraph &g, const int32_t *blocks, int32_t k, int64_t *cut_host,
                     int64_t *bw_host) {
  ProfScope ps(ctx, PROF_CUT);
  DBuf<unsigned long long> c(ctx, 1);
  c.zero();
  if (g.m2 > 0) {
    const int grid = grid_for(g.n, 256, ctx->num_sms * 16);
    if (k <= 255) {
      DBuf<uint8_t> b8(ctx, (size_t)g.n);
      k_narrow<<<grid_for(g.n, 256, ctx->num_sms * 8), 256, 0, ctx->stream>>>(blocks, g.n, b8.get());
      GP_LAUNCH_CHECK();
      k_cut<uint8_t><<<grid, 256, 0, ctx->stream>>>(g.xadj, g.adjncy, g.unit_w ? nullptr : g.adjwgt, b8.get(),
                                                    g.n, c.get());
      GP_LAUNCH_CHECK();
    } else {
      k_cut<int32_t><<<grid, 256, 0, ctx->stream>>>(g.xadj, g.adjncy, g.unit_w ? nullptr : g.adjwgt, blocks,
                                                    g.n, c.get());
      GP_LAUNCH_CHECK();
    }
  }
  // per entry: neighbour id, weight, neighbour block; per node: row offset, own block
  const double bb = k <= 255 ? 1.0 : 4.0;
  prof_bytes(ctx, PROF_CUT, ((g.unit_w ? 4.0 : 8.0) + bb) * g.m2 + (4.0 + bb) * g.n);
  if (bw_host) {
    DBuf<unsigned long long> bw(ctx, (size_t)k);
    block_weights_dev(ctx, g, blocks, k, bw.get());
    read_back(ctx, bw.get(), sizeof(int64_t) * k, bw_host);
  }
  if (cut_host) *cut_host = (int64_t)(read_scalar(ctx, c.get()) / 2);
}

int64_t refine_blocks(gp_ctx *ctx, const DevGraph &g, int32_t k, int64_t Lmax, int32_t level, uint64_t seed,
                      const gp_config &cfg, int32_t *blocks) {
  if (g.n == 0 || k <= 1 || cfg.ref_rounds <= 0) return 0;
  DBuf<unsigned long long> bw64(ctx, (size_t)k);
  DBuf<int32_t> bw(ctx, (size_t)k);
  block_weights_dev(ctx, g, blocks, k, bw64.get());
  k_to_i32<<<grid_for(k, 256, 64), 256, 0, ctx->stream>>>(bw64.get(), k, bw.get());
  GP_LAUNCH_CHECK();
  LpParams p;
  p.tag_act = TAG_RACT; p.tag_tie = TAG_RTIE; p.tag_prio = TAG_RPRIO;
  p.level = level; p.rounds = cfg.ref_rounds; p.subrounds = cfg.lp_subrounds;
  p.bound = Lmax; p.count_clusters = false; p.n_min = 0; p.dbg_max_subrounds = -1;
  p.prof_rate = PROF_REF_RATE; p.prof_accept = PROF_REF_ACCEPT;
  p.prof_overflow = PROF_REF_OVERFLOW; p.prof_apply = PROF_REF_APPLY; p.prof_small = PROF_REF_SMALL;
  p.small_nodes = cfg.small_lp_nodes;
  DBuf<uint8_t> b8;
  if (k <= 255) {
    b8.reset(ctx, (size_t)g.n);
    k_narrow<<<grid_for(g.n, 256, ctx->num_sms * 8), 256, 0, ctx->stream>>>(blocks, g.n, b8.get());
    GP_LAUNCH_CHECK();
  }
  LpResult r = lp_run(ctx, g, blocks, bw.get(), k, seed, p, nullptr, b8.get());
  return r.moves;
}

int64_t lmax_of(int64_t W, int32_t k, int64_t eps_ppm) {
  const int64_t base = (W + k - 1) / k;
  return (int64_t)(((__int128)base * (1000000 + eps_ppm)) / 1000000);
}

void check_blocks(gp_ctx *ctx, const int32_t *blocks, int n, int k) {
  DBuf<int> bad(ctx, 1);
  bad.zero();
  if (n > 0) {
    k_check_blocks<<<grid_for(n, 256, ctx->num_sms * 8), 256, 0, ctx->stream>>>(blocks, n, k, bad.get());
    GP_LAUNCH_CHECK();
  }
  GP_REQUIRE(read_scalar(ctx, bad.get()) == 0, GP_ERR_INVALID, "block ids must be in [0, k)");
}

// --------------------------------------------------------------- driver

struct Timer {
  gp_ctx *ctx;
  cudaEvent_t ev[4] = {};
  explicit Timer(gp_ctx *c) : ctx(c) {
    for (auto &e : ev) GP_CUDA(cudaEventCreate(&e));
  }
  ~Timer() {
    for (auto &e : ev) if (e) cudaEventDestroy(e);
  }
  void mark(int i) { GP_CUDA(cudaEventRecord(ev[i], ctx->stream)); }
  double ms(int a, int b) {
    float f = 0;
    GP_CUDA(cudaEventElapsedTime(&f, ev[a], ev[b]));
    return f;
  }
};

void partition_impl(gp_ctx *ctx, const DevGraph &input, int32_t k, double eps, uint64_t seed,
                    const gp_config &cfg, int32_t *blocks, int64_t *cut_out, gp_partition_stats *st) {
  GP_REQUIRE(k >= 1, GP_ERR_INVALID, "k must be >= 1");
  GP_REQUIRE(eps > 0 && eps < 1000, GP_ERR_INVALID, "eps must be in (0, 1000)");
  const int64_t eps_ppm = llround(eps * 1e6);
  GP_REQUIRE(eps_ppm >= 1, GP_ERR_INVALID, "eps must be at least 1e-6");
  GP_REQUIRE(cfg.max_levels >= 0 && cfg.max_levels <= GP_MAX_LEVELS, GP_ERR_INVALID, "max_levels out of range");
  GP_REQUIRE(cfg.shrink_num > 0 && cfg.shrink_den > 0 && cfg.min_shrink_num > 0 && cfg.min_shrink_den > 0 &&
                 cfg.tau_e_den > 0 && cfg.tau_d_den > 0 && cfg.rho_den > 0 && cfg.cluster_factor > 0,
             GP_ERR_INVALID, "bad configuration");
  Timer tm(ctx);
  tm.mark(0);
  const GraphTotals tot = validate_graph(ctx, input, cfg.validate != 0);
  const int64_t W = tot.W, cmax = tot.cmax;
  const int64_t Lmax = lmax_of(W, k, eps_ppm);
  GP_REQUIRE(cmax <= Lmax, GP_ERR_INFEASIBLE, "a node is heavier than L_max");
  gp_partition_stats local{};
  gp_partition_stats &S = st ? *st : local;
  memset(&S, 0, sizeof(S));
  S.W = W;
  S.Lmax = Lmax;
  const int n = input.n;
  if (k == 1 || n == 0) {
    if (n > 0) GP_CUDA(cudaMemsetAsync(blocks, 0, sizeof(int32_t) * n, ctx->stream));
    if (cut_out) *cut_out = 0;
    S.n_coarsest = n;
    GP_CUDA(cudaStreamSynchronize(ctx->stream));
    return;
  }
  const int64_t U = std::max<int64_t>(1, W / ((int64_t)cfg.cluster_factor * k));
  S.U = U;
  std::vector<std::unique_ptr<DevGraph>> G;
  std::vector<DBuf<int32_t>> C;
  G.push_back(std::make_unique<DevGraph>(DevGraph::wrap(input.view())));
  G[0]->unit_w = tot.unit_w;
  int L = 0;
  while ((int64_t)G[L]->n > (int64_t)cfg.coarsest_factor * k && L < cfg.max_levels) {
    const DevGraph &cur = *G[L];
    DBuf<int32_t> cmap(ctx, (size_t)cur.n);
    LevelOut lo;
    {
      NvtxRange r("coarsen", L + 1);
      coarsen_level(ctx, cur, U, L + 1, seed, cfg, cmap.get(), nullptr, lo);
    }
    auto Gc = std::make_unique<DevGraph>();
    {
      NvtxRange r("contract", L + 1);
      contract_graph(ctx, cur, cmap.get(), lo.n_coarse, *Gc);
    }
    gp_level_stats ls = lo.st;
    ls.n = cur.n;
    ls.n_next = lo.n_coarse;
    ls.m = cur.m2 / 2;
    ls.m_coarse = Gc->m2 / 2;
    if ((int64_t)lo.n_coarse * cfg.min_shrink_num > (int64_t)cur.n * cfg.min_shrink_den) break;
    const int64_t a = (int64_t)(((__int128)ls.m * cfg.tau_e_num) / cfg.tau_e_den);
    const int64_t b = (int64_t)(((__int128)ls.m * lo.n_coarse * cfg.tau_d_num) / ((__int128)cfg.tau_d_den * cur.n));
    ls.m_hat = a < b ? a : b;
    ls.triggered = cfg.sparsifier != GP_SPARSIFY_NONE &&
                   (__int128)ls.m_coarse * cfg.rho_den > (__int128)cfg.rho_num * ls.m_hat;
    if (ls.triggered) {
      auto Gs = std::make_unique<DevGraph>();
      NvtxRange r("sparsify", L + 2);
      sparsify_graph(ctx, *Gc, ls.m_hat, L + 2, seed, cfg.sparsifier, *Gs, &ls);
      Gc = std::move(Gs);
    }
    ls.m_next = Gc->m2 / 2;
    S.lv[L] = ls;
    C.push_back(std::move(cmap));
    G.push_back(std::move(Gc));
    L++;
  }
  S.levels = L;
  S.n_coarsest = G[L]->n;
  tm.mark(1);
  // initial partition of the coarsest graph
  DBuf<int32_t> blk(ctx, (size_t)G[L]->n);
  {
    NvtxRange r("initial");
    initial_partition(ctx, *G[L], k, eps_ppm, seed, cfg.ip_trials, blk.get());
    cut_and_weights(ctx, *G[L], blk.get(), k, &S.ip_cut, nullptr);
    S.rebalance_moves = rebalance_blocks(ctx, *G[L], k, Lmax, blk.get());
  }
  tm.mark(2);
  {
    NvtxRange r("refine", L + 1);
    refine_blocks(ctx, *G[L], k, Lmax, L + 1, seed, cfg, blk.get());
  }
  for (int i = L - 1; i >= 0; i--) {
    DBuf<int32_t> fine;
    int32_t *dst;
    if (i == 0) {
      dst = blocks;
    } else {
      fine.reset(ctx, (size_t)G[i]->n);
      dst = fine.get();
    }
    NvtxRange r("refine", i + 1);
    project(ctx, G[i]->n, C[i].get(), blk.get(), dst);
    refine_blocks(ctx, *G[i], k, Lmax, i + 1, seed, cfg, dst);
    if (i > 0) blk = std::move(fine);
  }
  if (L == 0)
    GP_CUDA(cudaMemcpyAsync(blocks, blk.get(), sizeof(int32_t) * n, cudaMemcpyDeviceToDevice, ctx->stream));
  int64_t cut = 0;
  cut_and_weights(ctx, *G[0], blocks, k, &cut, nullptr);
  tm.mark(3);
  GP_CUDA(cudaEventSynchronize(tm.ev[3]));
  S.cut = cut;
  S.ms_coarsen = tm.ms(0, 1);
  S.ms_initial = tm.ms(1, 2);
  S.ms_uncoarsen = tm.ms(2, 3);
  S.ms_total = tm.ms(0, 3);
  if (cut_out) *cut_out = cut;
}

}  // namespace gp
