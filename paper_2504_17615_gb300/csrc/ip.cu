// ip.cu -- initial partitioning of the coarsest graph by recursive
// bisection (Sec. 4.3), plus the greedy rebalancer.
//
// All subproblems of one depth of the bisection tree are split together:
// every (subproblem, trial) pair runs in its own thread block, growing side 1
// greedily one node at a time (largest gain 2 conn(v) - deg'(v) among
// frontier nodes that fit under L1, ties by the smallest id; otherwise the
// node of smallest (h32(key(IP, 0, bid), v, t), v)) until side 1 reaches its
// target weight.  The trial with the smallest cut (ties: lowest trial) wins.
#include "gp_internal.cuh"

#include <algorithm>

namespace gp {

namespace {

constexpr int kIpThreads = 512;
constexpr int kIpWarps = kIpThreads / 32;

struct Sub {
  int32_t start, count;  // node list range
  int32_t bid;           // heap id of the bisection
  int32_t pad;
  int64_t T1, L1;        // side-1 target and limit
};

struct IpArgs {
  const int32_t *xadj, *adjncy, *adjwgt, *vwgt;
  const int32_t *list, *loc, *sp, *dp;
  const Sub *subs;
  int trials;
  int n;
  uint64_t seed;
  int smem_nodes;          // subproblems up to this size keep their state in shared memory
  int32_t *gconn;          // global fallback state, per block: stride entries
  uint32_t *ghv;
  uint8_t *gin;
  int64_t gstride;
  int64_t *trial_cut;      // per block
  uint8_t *flags;          // [trial][n] side-1 flags by list position
};

__device__ void block_best(int64_t &gain, int &vf, uint64_t &pn, int64_t *s_g, int *s_v, uint64_t *s_n) {
  // frontier: max gain, then min v (vf < 0 = none); non-frontier: min packed (hv << 32 | v)
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const int64_t g2 = __shfl_xor_sync(0xFFFFFFFFu, gain, o);
    const int v2 = __shfl_xor_sync(0xFFFFFFFFu, vf, o);
    const uint64_t p2 = __shfl_xor_sync(0xFFFFFFFFu, pn, o);
    if (v2 >= 0 && (vf < 0 || g2 > gain || (g2 == gain && v2 < vf))) { gain = g2; vf = v2; }
    pn = p2 < pn ? p2 : pn;
  }
  const int w = threadIdx.x >> 5;
  if (lane_id() == 0) { s_g[w] = gain; s_v[w] = vf; s_n[w] = pn; }
  __syncthreads();
  gain = s_g[0]; vf = s_v[0]; pn = s_n[0];
  for (int i = 1; i < kIpWarps; i++) {
    if (s_v[i] >= 0 && (vf < 0 || s_g[i] > gain || (s_g[i] == gain && s_v[i] < vf))) {
      gain = s_g[i]; vf = s_v[i];
    }
    pn = s_n[i] < pn ? s_n[i] : pn;
  }
  __syncthreads();
}

__global__ void __launch_bounds__(kIpThreads) k_ip_trial(IpArgs a) {
  extern __shared__ unsigned char dyn[];
  __shared__ int64_t s_g[kIpWarps];
  __shared__ int s_v[kIpWarps];
  __shared__ uint64_t s_n[kIpWarps];
  __shared__ int64_t s_w1;
  __shared__ int s_pick;
  __shared__ unsigned long long s_cut;
  const int si = blockIdx.x / a.trials, t = blockIdx.x % a.trials;
  const Sub S = a.subs[si];
  const int cnt = S.count;
  int32_t *conn;
  uint32_t *hv;
  uint8_t *in1;
  if (cnt <= a.smem_nodes) {
    conn = reinterpret_cast<int32_t *>(dyn);
    hv = reinterpret_cast<uint32_t *>(dyn + sizeof(int32_t) * a.smem_nodes);
    in1 = dyn + 2 * sizeof(int32_t) * a.smem_nodes;
  } else {
    conn = a.gconn + (int64_t)blockIdx.x * a.gstride;
    hv = a.ghv + (int64_t)blockIdx.x * a.gstride;
    in1 = a.gin + (int64_t)blockIdx.x * a.gstride;
  }
  const uint64_t kip = stream_key(a.seed, TAG_IP, 0, (uint32_t)S.bid);
  for (int j = threadIdx.x; j < cnt; j += blockDim.x) {
    conn[j] = 0;
    in1[j] = 0;
    hv[j] = h32(kip, (uint32_t)a.list[S.start + j], (uint32_t)t);
  }
  if (threadIdx.x == 0) { s_w1 = 0; s_cut = 0; }
  __syncthreads();
  while (s_w1 < S.T1) {
    const int64_t w1 = s_w1;
    int64_t gain = 0;
    int vf = -1;
    uint64_t pn = ~0ull;
    for (int j = threadIdx.x; j < cnt; j += blockDim.x) {
      if (in1[j]) continue;
      const int v = a.list[S.start + j];
      if (w1 + a.vwgt[v] > S.L1) continue;
      if (conn[j] > 0) {
        const int64_t gj = 2 * (int64_t)conn[j] - a.dp[v];
        if (vf < 0 || gj > gain || (gj == gain && v < vf)) { gain = gj; vf = v; }
      } else {
        const uint64_t p = ((uint64_t)hv[j] << 32) | (uint32_t)v;
        pn = p < pn ? p : pn;
      }
    }
    block_best(gain, vf, pn, s_g, s_v, s_n);
    const int pick = vf >= 0 ? vf : (pn != ~0ull ? (int)(uint32_t)pn : -1);
    if (pick < 0) break;
    if (threadIdx.x == 0) {
      in1[a.loc[pick]] = 1;
      s_w1 = w1 + a.vwgt[pick];
    }
    for (int e = a.xadj[pick] + threadIdx.x; e < a.xadj[pick + 1]; e += blockDim.x) {
      const int u = a.adjncy[e];
      if (a.sp[u] == si) atomicAdd(&conn[a.loc[u]], a.adjwgt[e]);
    }
    __syncthreads();
  }
  // cut of this trial inside the subproblem
  unsigned long long cut = 0;
  for (int j = threadIdx.x; j < cnt; j += blockDim.x) {
    if (!in1[j]) continue;
    const int v = a.list[S.start + j];
    for (int e = a.xadj[v]; e < a.xadj[v + 1]; e++) {
      const int u = a.adjncy[e];
      if (a.sp[u] == si && !in1[a.loc[u]]) cut += (unsigned long long)a.adjwgt[e];
    }
  }
  cut = warp_sum(cut);
  if (lane_id() == 0 && cut) atomicAdd(&s_cut, cut);
  __syncthreads();
  if (threadIdx.x == 0) a.trial_cut[blockIdx.x] = (int64_t)s_cut;
  uint8_t *fl = a.flags + (int64_t)t * a.n + S.start;
  for (int j = threadIdx.x; j < cnt; j += blockDim.x) fl[j] = in1[j];
}

__global__ void k_sub_count(const int32_t *sp, const int32_t *vwgt, int n, int32_t *cnt, long long *w) {
  for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
    const int s = sp[v];
    if (s < 0) continue;
    atomicAdd(&cnt[s], 1);
    atomicAdd((unsigned long long *)&w[s], (unsigned long long)vwgt[v]);
  }
}

__global__ void k_sub_fill(const int32_t *sp, int n, const int32_t *start, int32_t *cursor,
                           int32_t *list, int32_t *loc) {
  for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
    const int s = sp[v];
    if (s < 0) continue;
    const int p = atomicAdd(&cursor[s], 1);
    list[start[s] + p] = v;
    loc[v] = p;
  }
}

// deg'(v): weight to nodes of the same subproblem
__global__ void k_dp(const int32_t *xadj, const int32_t *adjncy, const int32_t *adjwgt, const int32_t *sp,
                     int n, int32_t *dp) {
  const int lane = (int)lane_id();
  const int wid = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int nw = (gridDim.x * blockDim.x) >> 5;
  for (int v = wid; v < n; v += nw) {
    const int s = sp[v];
    if (s < 0) continue;
    int sum = 0;
    for (int e = xadj[v] + lane; e < xadj[v + 1]; e += 32)
      if (sp[adjncy[e]] == s) sum += adjwgt[e];
    sum = warp_sum(sum);
    if (lane == 0) dp[v] = sum;
  }
}

__global__ void k_ip_select(const int64_t *trial_cut, int nsubs, int trials, int32_t *best) {
  for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < nsubs; s += gridDim.x * blockDim.x) {
    int bt = 0;
    for (int t = 1; t < trials; t++)
      if (trial_cut[s * trials + t] < trial_cut[s * trials + bt]) bt = t;
    best[s] = bt;
  }
}

// children: child[2 s + side] = new subproblem index, or -(1 + block) when final
__global__ void k_ip_assign(int n, const int32_t *loc, const int32_t *best, const uint8_t *flags,
                            const int32_t *start, const int32_t *child, int32_t *sp, int32_t *blocks) {
  for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
    const int s = sp[v];
    if (s < 0) continue;
    const int side1 = flags[(int64_t)best[s] * n + start[s] + loc[v]];
    const int c = child[2 * s + (side1 ? 0 : 1)];
    if (c < 0) {
      blocks[v] = -(c + 1);
      sp[v] = -1;
    } else {
      sp[v] = c;
    }
  }
}

int32_t ceil_log2(int64_t k) {
  int32_t b = 0;
  while (((int64_t)1 << b) < k) b++;
  return b;
}

struct HostSub {
  int32_t kk, b0, bid;
};

}  // namespace

void initial_partition(gp_ctx *ctx, const DevGraph &g, int32_t k, int64_t eps_ppm, uint64_t seed,
                       int32_t trials, int32_t *blocks) {
  ProfScope ps(ctx, PROF_IP);
  const int n = g.n;
  GP_REQUIRE(trials >= 1, GP_ERR_INVALID, "ip_trials must be >= 1");
  GP_CUDA(cudaMemsetAsync(blocks, 0, sizeof(int32_t) * (n > 0 ? n : 1), ctx->stream));
  if (k <= 1 || n == 0) return;
  const int grid = grid_for(n, 256, ctx->num_sms * 8);
  DBuf<int32_t> sp(ctx, (size_t)n), list(ctx, (size_t)n), loc(ctx, (size_t)n), dp(ctx, (size_t)n);
  sp.zero();  // everybody in subproblem 0
  const int64_t eps_l = eps_ppm / ceil_log2(k);
  std::vector<HostSub> subs{{k, 0, 1}};
  int smem_nodes = 12000;
  const size_t smem_bytes = (size_t)smem_nodes * 9;
  GP_CUDA(cudaFuncSetAttribute(k_ip_trial, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_bytes));
  DBuf<uint8_t> flags(ctx, (size_t)trials * n);
  while (!subs.empty()) {
    const int ns = (int)subs.size();
    DBuf<int32_t> cnt(ctx, (size_t)ns), start(ctx, (size_t)ns + 1), cursor(ctx, (size_t)ns);
    DBuf<long long> wsum(ctx, (size_t)ns);
    cnt.zero(); wsum.zero(); cursor.zero();
    k_sub_count<<<grid, 256, 0, ctx->stream>>>(sp.get(), g.vwgt, n, cnt.get(), wsum.get());
    GP_LAUNCH_CHECK();
    std::vector<int32_t> hc(ns);
    std::vector<long long> hw(ns);
    read_back(ctx, cnt.get(), sizeof(int32_t) * ns, hc.data());
    read_back(ctx, wsum.get(), sizeof(long long) * ns, hw.data());
    std::vector<int32_t> hs(ns + 1);
    hs[0] = 0;
    for (int i = 0; i < ns; i++) hs[i + 1] = hs[i] + hc[i];
    GP_CUDA(cudaMemcpyAsync(start.get(), hs.data(), sizeof(int32_t) * (ns + 1), cudaMemcpyHostToDevice,
                            ctx->stream));
    k_sub_fill<<<grid, 256, 0, ctx->stream>>>(sp.get(), n, start.get(), cursor.get(), list.get(), loc.get());
    GP_LAUNCH_CHECK();
    k_dp<<<grid_for((int64_t)n * 32, 256, ctx->num_sms * 8), 256, 0, ctx->stream>>>(
        g.xadj, g.adjncy, g.adjwgt, sp.get(), n, dp.get());
    GP_LAUNCH_CHECK();
    std::vector<Sub> hsub(ns);
    int maxcnt = 0;
    for (int i = 0; i < ns; i++) {
      const int64_t kk = subs[i].kk, k1 = (kk + 1) / 2;
      const int64_t W = hw[i];
      hsub[i].start = hs[i];
      hsub[i].count = hc[i];
      hsub[i].bid = subs[i].bid;
      hsub[i].pad = 0;
      hsub[i].T1 = (W * k1 + kk - 1) / kk;
      hsub[i].L1 = (int64_t)(((__int128)hsub[i].T1 * (1000000 + eps_l)) / 1000000);
      maxcnt = std::max(maxcnt, hc[i]);
    }
    DBuf<Sub> dsub(ctx, (size_t)ns);
    GP_CUDA(cudaMemcpyAsync(dsub.get(), hsub.data(), sizeof(Sub) * ns, cudaMemcpyHostToDevice, ctx->stream));
    const int nblocks = ns * trials;
    DBuf<int64_t> tcut(ctx, (size_t)nblocks);
    DBuf<int32_t> gconn;
    DBuf<uint32_t> ghv;
    DBuf<uint8_t> gin;
    IpArgs a{};
    a.xadj = g.xadj; a.adjncy = g.adjncy; a.adjwgt = g.adjwgt; a.vwgt = g.vwgt;
    a.list = list.get(); a.loc = loc.get(); a.sp = sp.get(); a.dp = dp.get(); a.subs = dsub.get();
    a.trials = trials; a.n = n; a.seed = seed; a.smem_nodes = smem_nodes;
    if (maxcnt > smem_nodes) {
      a.gstride = maxcnt;
      gconn.reset(ctx, (size_t)nblocks * maxcnt);
      ghv.reset(ctx, (size_t)nblocks * maxcnt);
      gin.reset(ctx, (size_t)nblocks * maxcnt);
      a.gconn = gconn.get(); a.ghv = ghv.get(); a.gin = gin.get();
    }
    a.trial_cut = tcut.get();
    a.flags = flags.get();
    k_ip_trial<<<nblocks, kIpThreads, smem_bytes, ctx->stream>>>(a);
    GP_LAUNCH_CHECK();
    DBuf<int32_t> best(ctx, (size_t)ns), child(ctx, (size_t)2 * ns);
    k_ip_select<<<grid_for(ns, 128, 1024), 128, 0, ctx->stream>>>(tcut.get(), ns, trials, best.get());
    GP_LAUNCH_CHECK();
    // children of every subproblem (final when they hold a single block)
    std::vector<int32_t> hchild(2 * ns);
    std::vector<HostSub> next;
    for (int i = 0; i < ns; i++) {
      const int32_t kk = subs[i].kk, k1 = (kk + 1) / 2, k2 = kk - k1;
      const HostSub c1{k1, subs[i].b0, 2 * subs[i].bid}, c2{k2, subs[i].b0 + k1, 2 * subs[i].bid + 1};
      const HostSub cs[2] = {c1, c2};
      for (int side = 0; side < 2; side++) {
        if (cs[side].kk <= 1) {
          hchild[2 * i + side] = -(cs[side].b0 + 1);
        } else {
          hchild[2 * i + side] = (int32_t)next.size();
          next.push_back(cs[side]);
        }
      }
    }
    GP_CUDA(cudaMemcpyAsync(child.get(), hchild.data(), sizeof(int32_t) * 2 * ns, cudaMemcpyHostToDevice,
                            ctx->stream));
    k_ip_assign<<<grid, 256, 0, ctx->stream>>>(n, loc.get(), best.get(), flags.get(), start.get(),
                                                child.get(), sp.get(), blocks);
    GP_LAUNCH_CHECK();
    GP_CUDA(cudaStreamSynchronize(ctx->stream));  // host vectors above must outlive the copies
    subs.swap(next);
  }
}

// --------------------------------------------------------------- rebalance

namespace {

constexpr int kRbThreads = 1024;

__global__ void __launch_bounds__(kRbThreads) k_rebalance(const int32_t *xadj, const int32_t *adjncy,
                                                          const int32_t *adjwgt, const int32_t *vwgt,
                                                          int n, int k, int64_t Lmax, int32_t *blk,
                                                          int64_t *bw, long long *moves_out) {
  __shared__ int64_t s_d[32];
  __shared__ int s_v[32];
  __shared__ int s_A, s_B, s_best;
  long long moves = 0;
  for (int64_t it = 0; it <= (int64_t)n; it++) {
    if (threadIdx.x == 0) {
      int A = 0, B = 0;
      for (int b = 1; b < k; b++) {
        if (bw[b] > bw[A]) A = b;
        if (bw[b] < bw[B]) B = b;
      }
      s_A = A;
      s_B = B;
    }
    __syncthreads();
    const int A = s_A, B = s_B;
    if (bw[A] <= Lmax || A == B) break;
    int64_t bd = 0;
    int bv = -1;
    for (int v = threadIdx.x; v < n; v += blockDim.x) {
      if (blk[v] != A || bw[B] + vwgt[v] > Lmax) continue;
      int64_t ca = 0, cb = 0;
      for (int e = xadj[v]; e < xadj[v + 1]; e++) {
        const int b = blk[adjncy[e]];
        if (b == A) ca += adjwgt[e];
        else if (b == B) cb += adjwgt[e];
      }
      const int64_t d = ca - cb;
      if (bv < 0 || d < bd || (d == bd && v < bv)) { bd = d; bv = v; }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const int64_t d2 = __shfl_xor_sync(0xFFFFFFFFu, bd, o);
      const int v2 = __shfl_xor_sync(0xFFFFFFFFu, bv, o);
      if (v2 >= 0 && (bv < 0 || d2 < bd || (d2 == bd && v2 < bv))) { bd = d2; bv = v2; }
    }
    if (lane_id() == 0) { s_d[threadIdx.x >> 5] = bd; s_v[threadIdx.x >> 5] = bv; }
    __syncthreads();
    if (threadIdx.x == 0) {
      int64_t d = s_d[0];
      int v = s_v[0];
      for (int i = 1; i < kRbThreads / 32; i++)
        if (s_v[i] >= 0 && (v < 0 || s_d[i] < d || (s_d[i] == d && s_v[i] < v))) { d = s_d[i]; v = s_v[i]; }
      s_best = v;
      if (v >= 0) {
        blk[v] = B;
        bw[A] -= vwgt[v];
        bw[B] += vwgt[v];
        moves++;
      }
    }
    __syncthreads();
    if (s_best < 0) break;
  }
  if (threadIdx.x == 0) *moves_out = moves;
}

__global__ void k_block_weights(const int32_t *blk, const int32_t *vwgt, int n, long long *bw) {
  for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x)
    atomicAdd((unsigned long long *)&bw[blk[v]], (unsigned long long)vwgt[v]);
}

}  // namespace

int64_t rebalance_blocks(gp_ctx *ctx, const DevGraph &g, int32_t k, int64_t Lmax, int32_t *blocks) {
  ProfScope ps(ctx, PROF_IP);
  if (g.n == 0 || k <= 1) return 0;
  DBuf<long long> bw(ctx, (size_t)k), moves(ctx, 1);
  bw.zero();
  moves.zero();
  k_block_weights<<<grid_for(g.n, 256, ctx->num_sms * 8), 256, 0, ctx->stream>>>(blocks, g.vwgt, g.n, bw.get());
  GP_LAUNCH_CHECK();
  k_rebalance<<<1, kRbThreads, 0, ctx->stream>>>(g.xadj, g.adjncy, g.adjwgt, g.vwgt, g.n, k, Lmax, blocks,
                                                 reinterpret_cast<int64_t *>(bw.get()), moves.get());
  GP_LAUNCH_CHECK();
  return read_scalar(ctx, moves.get());
}

}  // namespace gp
