// cluster.cu -- one coarsening clustering (Sec. 3, Sec. 4.1, Sec. 4.3):
// size-constrained LP, 2-hop clustering of light singletons through their
// favourite cluster, clustering of isolated nodes with each other, all
// limited to a 2.5x node reduction, then dense coarse ids.
#include "lp.cuh"

namespace gp {

namespace {

__global__ void k_init_clusters(const int32_t *vwgt, int n, int32_t *label, int32_t *cw) {
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n;
       v += (int64_t)gridDim.x * blockDim.x) {
    label[v] = (int32_t)v;
    cw[v] = vwgt[v];
  }
}

// Members per cluster.
__global__ void k_cluster_sizes(const int32_t *label, int n, int32_t *size) {
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n;
       v += (int64_t)gridDim.x * blockDim.x)
    atomicAdd(&size[label[v]], 1);
}

// heaviest member of every favourite group
__global__ void k_fav_cmax(const uint64_t *keys, int count, const int32_t *vwgt, int32_t *cmax) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < count; i += gridDim.x * blockDim.x) {
    const uint64_t k = keys[i];
    atomicMax(&cmax[(int)(k >> 32)], vwgt[(uint32_t)k]);
  }
}

// Runs of g = floor(U / heaviest) consecutive members per favourite group;
// every non-first member of a run is a merge into the run's first member.
__global__ void k_fav_flags(const uint64_t *keys, int count, const int32_t *cmax, int64_t U,
                            int32_t *merge, int32_t *leader) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < count; i += gridDim.x * blockDim.x) {
    const uint64_t k = keys[i];
    const uint64_t seg = k & 0xFFFFFFFF00000000ull;
    int lo = 0, hi = i;
    while (lo < hi) {
      const int mid = (lo + hi) >> 1;
      if (keys[mid] < seg) lo = mid + 1; else hi = mid;
    }
    const int64_t gsz = U / cmax[(int)(k >> 32)];
    const int64_t p = i - lo;
    merge[i] = (p % gsz) != 0;
    leader[i] = (int32_t)(uint32_t)keys[lo + (p / gsz) * gsz];
  }
}

__global__ void k_fav_apply(const uint64_t *keys, int count, const int32_t *merge,
                            const int32_t *rank, const int32_t *leader, int64_t M, int32_t *label) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < count; i += gridDim.x * blockDim.x) {
    if (!merge[i] || rank[i] >= M) continue;
    const int v = (int)(uint32_t)keys[i];
    label[v] = label[leader[i]];
  }
}

__global__ void k_fav_clear(const uint64_t *keys, int count, int32_t *cmax) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < count; i += gridDim.x * blockDim.x)
    cmax[(int)(keys[i] >> 32)] = 0;
}

__global__ void k_iso_flags(const int32_t *xadj, const int32_t *vwgt, int n, int64_t U, int32_t *flag,
                            int *cmax) {
  int m = 0;
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n;
       v += (int64_t)gridDim.x * blockDim.x) {
    const bool iso = xadj[v + 1] == xadj[v] && 2 * (int64_t)vwgt[v] <= U;
    flag[v] = iso;
    if (iso) m = vwgt[v] > m ? vwgt[v] : m;
  }
  m = warp_max(m);
  if (lane_id() == 0 && m) atomicMax(cmax, m);
}

__global__ void k_iso_list(const int32_t *flag, const int32_t *rank, int n, int32_t *list) {
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n;
       v += (int64_t)gridDim.x * blockDim.x)
    if (flag[v]) list[rank[v]] = (int32_t)v;
}

__global__ void k_iso_apply(const int32_t *flag, const int32_t *rank, const int32_t *list, int n,
                            int64_t gsz, int64_t M, int32_t *label) {
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n;
       v += (int64_t)gridDim.x * blockDim.x) {
    if (!flag[v]) continue;
    const int64_t j = rank[v];
    if (j % gsz == 0) continue;
    const int64_t q = j / gsz;
    if (j - q - 1 >= M) continue;  // merge ordinal beyond the cap
    label[v] = list[q * gsz];
  }
}

__global__ void k_mark_used(const int32_t *label, int n, int32_t *used) {
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n;
       v += (int64_t)gridDim.x * blockDim.x)
    used[label[v]] = 1;
}

__global__ void k_cmap(const int32_t *label, const int32_t *rank, int n, int32_t *cmap) {
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n;
       v += (int64_t)gridDim.x * blockDim.x)
    cmap[v] = rank[label[v]];
}

}  // namespace

void coarsen_level(gp_ctx *ctx, const DevGraph &g, int64_t U, int32_t level, uint64_t seed,
                   const gp_config &cfg, int32_t *cmap, int32_t *label_out, LevelOut &out) {
  TraceTimer trace(ctx);
  const int n = g.n;
  const int grid = grid_for(n, 256, ctx->num_sms * 8);
  DBuf<int32_t> label_own;
  int32_t *label = label_out;
  if (!label) {
    label_own.reset(ctx, (size_t)n);
    label = label_own.get();
  }
  DBuf<int32_t> cw(ctx, (size_t)n);
  DBuf<int64_t> ncl_dev(ctx, 1);
  k_init_clusters<<<grid, 256, 0, ctx->stream>>>(g.vwgt, n, label, cw.get());
  GP_LAUNCH_CHECK();
  int64_t n64 = n;
  GP_CUDA(cudaMemcpyAsync(ncl_dev.get(), &n64, sizeof(int64_t), cudaMemcpyHostToDevice, ctx->stream));
  const int64_t n_min = ((int64_t)n * cfg.shrink_den + cfg.shrink_num - 1) / cfg.shrink_num;

  LpParams p;
  p.tag_act = TAG_ACT; p.tag_tie = TAG_TIE; p.tag_prio = TAG_PRIO;
  p.level = level; p.rounds = cfg.lp_rounds; p.subrounds = cfg.lp_subrounds;
  p.bound = U; p.count_clusters = true; p.n_min = n_min;
  p.dbg_max_subrounds = cfg.dbg_max_subrounds;
  p.prof_rate = PROF_LP_RATE; p.prof_accept = PROF_LP_ACCEPT;
  p.prof_overflow = PROF_LP_OVERFLOW; p.prof_apply = PROF_LP_APPLY; p.prof_small = PROF_LP_SMALL;
  p.small_nodes = cfg.small_lp_nodes;
  LpResult r = lp_run(ctx, g, label, cw.get(), n, seed, p, ncl_dev.get());
  int64_t ncl = n == 0 ? 0 : r.nclusters;
  out.st.n = n;
  out.st.lp_subrounds = r.subrounds;
  out.st.lp_moves = r.moves;
  out.st.clusters_lp = ncl;

  // 2-hop clustering (R9)
  if (cfg.two_hop && 2 * ncl > n && ncl > n_min) {
    ProfScope ps(ctx, PROF_TWOHOP);
    const uint64_t kfav = stream_key(seed, TAG_FAV, (uint32_t)level, 0);
    DBuf<int32_t> size(ctx, (size_t)n);
    size.zero();
    k_cluster_sizes<<<grid, 256, 0, ctx->stream>>>(label, n, size.get());
    GP_LAUNCH_CHECK();
    DBuf<uint64_t> keys;
    int32_t count = 0;
    favourites_bucketed(ctx, g, label, size.get(), U, kfav, keys, count);
    if (count > 0) {
      DBuf<uint32_t> dummy(ctx, (size_t)count);
      radix_sort_pairs(ctx, keys.get(), dummy.get(), count, 32 + bits_for(n));
      DBuf<int32_t> cmax(ctx, (size_t)n), merge(ctx, (size_t)count), rank(ctx, (size_t)count),
          leader(ctx, (size_t)count);
      DBuf<int32_t> total(ctx, 1);
      cmax.zero();
      const int gc = grid_for(count, 256, ctx->num_sms * 8);
      k_fav_cmax<<<gc, 256, 0, ctx->stream>>>(keys.get(), count, g.vwgt, cmax.get());
      GP_LAUNCH_CHECK();
      k_fav_flags<<<gc, 256, 0, ctx->stream>>>(keys.get(), count, cmax.get(), U, merge.get(),
                                               leader.get());
      GP_LAUNCH_CHECK();
      scan_exclusive_i32(ctx, merge.get(), rank.get(), count, total.get());
      const int64_t M = ncl - n_min;
      k_fav_apply<<<gc, 256, 0, ctx->stream>>>(keys.get(), count, merge.get(), rank.get(),
                                               leader.get(), M, label);
      GP_LAUNCH_CHECK();
      const int64_t merges = read_scalar(ctx, total.get());
      ncl -= merges < M ? merges : M;
    }
  }
  out.st.clusters_2hop = ncl;

  // isolated nodes (R10)
  if (cfg.isolated && ncl > n_min) {
    ProfScope ps(ctx, PROF_TWOHOP);
    DBuf<int32_t> flag(ctx, (size_t)n), rank(ctx, (size_t)n), total(ctx, 1);
    DBuf<int> cmax(ctx, 1);
    cmax.zero();
    k_iso_flags<<<grid, 256, 0, ctx->stream>>>(g.xadj, g.vwgt, n, U, flag.get(), cmax.get());
    GP_LAUNCH_CHECK();
    scan_exclusive_i32(ctx, flag.get(), rank.get(), n, total.get());
    int32_t niso = read_scalar(ctx, total.get());
    if (niso >= 2) {
      const int64_t cm = read_scalar(ctx, cmax.get());
      const int64_t gsz = U / cm;
      DBuf<int32_t> list(ctx, (size_t)niso);
      k_iso_list<<<grid, 256, 0, ctx->stream>>>(flag.get(), rank.get(), n, list.get());
      GP_LAUNCH_CHECK();
      const int64_t M = ncl - n_min;
      k_iso_apply<<<grid, 256, 0, ctx->stream>>>(flag.get(), rank.get(), list.get(), n, gsz, M, label);
      GP_LAUNCH_CHECK();
      const int64_t merges = niso - (niso + gsz - 1) / gsz;
      ncl -= merges < M ? merges : M;
    }
  }
  out.st.clusters_final = ncl;

  // dense coarse ids (R11)
  {
    ProfScope ps(ctx, PROF_RELABEL);
    DBuf<int32_t> used(ctx, (size_t)n), total(ctx, 1);
    used.zero();
    k_mark_used<<<grid, 256, 0, ctx->stream>>>(label, n, used.get());
    GP_LAUNCH_CHECK();
    scan_exclusive_i32(ctx, used.get(), used.get(), n, total.get());
    k_cmap<<<grid, 256, 0, ctx->stream>>>(label, used.get(), n, cmap);
    GP_LAUNCH_CHECK();
    out.n_coarse = read_scalar(ctx, total.get());
  }
  out.st.n_next = out.n_coarse;
  if (trace.on())
    fprintf(stderr, "[gp coarsen] level=%d n=%d -> %d (lp %lld, 2hop %lld) ms=%.2f\n", level, n, out.n_coarse,
            (long long)out.st.clusters_lp, (long long)out.st.clusters_2hop, trace.ms());
}

}  // namespace gp
