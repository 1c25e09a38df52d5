// modularity.cu -- the modularity of a clustering and Lemma 2's bound
// (Sec. 5): the weight inside clusters, the total weight, and the cluster
// volumes (sums of weighted degrees), from which Q_C = sum_i (e_ii - a_i^2)
// and alpha_C = max_i a_i follow.
#include "gp_internal.cuh"

namespace gp {

namespace {

constexpr unsigned FULL = 0xFFFFFFFFu;

struct ModOut {
  unsigned long long w_internal, w_total, vol_max, vol_sq;
  int bad;  // a label outside [0, nlabels)
};

__device__ __forceinline__ bool in_range(int L, int nl) { return L >= 0 && L < nl; }

// Warps walk 32 consecutive rows at a time: the weight of entries whose
// endpoints share a label, the total weight, and every row's weight added to
// its node's cluster volume.
__global__ void __launch_bounds__(256) k_mod_rows(const int32_t *xadj, const int32_t *adjncy,
                                                  const int32_t *adjwgt, const int32_t *label, int n, int nl,
                                                  unsigned long long *vol, ModOut *o) {
  __shared__ unsigned long long s_deg[8][32];
  const int lane = (int)lane_id(), wib = threadIdx.x >> 5;
  const int wid = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5);
  const int nw = (int)((gridDim.x * blockDim.x) >> 5);
  unsigned long long win = 0, wtot = 0;
  int bad = 0;
  for (int64_t u0 = (int64_t)wid * 32; u0 < n; u0 += (int64_t)nw * 32) {
    const int64_t u = u0 + lane;
    const bool valid = u < n;
    const int xe = valid ? xadj[u + 1] : 0x7FFFFFFF;
    const int Lu = valid ? label[u] : -1;
    if (valid && !in_range(Lu, nl)) bad = 1;
    const int e0 = xadj[u0];
    const int last = (int)((n - u0) < 32 ? (n - u0) : 32) - 1;
    const int e1 = __shfl_sync(FULL, xe, last);
    s_deg[wib][lane] = 0;
    __syncwarp();
    for (int f0 = e0; f0 < e1; f0 += 32) {
      const int e = f0 + lane;
      int q = 0;  // owner: lanes whose row ends at or before e
#pragma unroll
      for (int step = 16; step > 0; step >>= 1) {
        const int val = __shfl_sync(FULL, xe, q + step - 1);
        if (val <= e) q += step;
      }
      const int Lq = __shfl_sync(FULL, Lu, q);
      if (e < e1) {
        const int w = __ldcs(adjwgt + e);
        const int Lv = label[__ldcs(adjncy + e)];
        if (!in_range(Lv, nl)) bad = 1;
        wtot += (unsigned long long)w;
        if (Lv == Lq) win += (unsigned long long)w;
        atomicAdd(&s_deg[wib][q], (unsigned long long)w);
      }
    }
    __syncwarp();
    if (valid && in_range(Lu, nl) && s_deg[wib][lane]) atomicAdd(&vol[Lu], s_deg[wib][lane]);
    __syncwarp();
  }
  win = warp_sum(win);
  wtot = warp_sum(wtot);
  bad = __reduce_or_sync(FULL, bad);
  if (lane == 0) {
    if (win) atomicAdd(&o->w_internal, win);
    if (wtot) atomicAdd(&o->w_total, wtot);
    if (bad) atomicOr(&o->bad, 1);
  }
}

__global__ void __launch_bounds__(256) k_mod_volumes(const unsigned long long *vol, int nl, ModOut *o) {
  unsigned long long mx = 0, sq = 0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nl; i += gridDim.x * blockDim.x) {
    const unsigned long long x = vol[i];
    mx = x > mx ? x : mx;
    sq += x * x;
  }
  mx = warp_max(mx);
  sq = warp_sum(sq);
  if (lane_id() == 0) {
    if (mx) atomicMax(&o->vol_max, mx);
    if (sq) atomicAdd(&o->vol_sq, sq);
  }
}

}  // namespace

void modularity(gp_ctx *ctx, const DevGraph &g, const int32_t *labels, int32_t nlabels, gp_modularity_stats *out) {
  GP_REQUIRE(nlabels >= 1, GP_ERR_INVALID, "nlabels must be >= 1");
  GP_REQUIRE(g.n == 0 || labels, GP_ERR_INVALID, "null labels");
  DBuf<unsigned long long> vol(ctx, (size_t)nlabels);
  DBuf<ModOut> o(ctx, 1);
  vol.zero();
  o.zero();
  if (g.n > 0) {
    k_mod_rows<<<grid_for(g.n, 256, ctx->num_sms * 16), 256, 0, ctx->stream>>>(
        g.xadj, g.adjncy, g.adjwgt, labels, g.n, nlabels, vol.get(), o.get());
    GP_LAUNCH_CHECK();
  }
  k_mod_volumes<<<grid_for(nlabels, 256, ctx->num_sms * 8), 256, 0, ctx->stream>>>(vol.get(), nlabels, o.get());
  GP_LAUNCH_CHECK();
  ModOut h;
  read_back(ctx, o.get(), sizeof(ModOut), &h);
  GP_REQUIRE(!h.bad, GP_ERR_INVALID, "a label lies outside [0, nlabels)");
  out->w_internal = (int64_t)h.w_internal;
  out->w_total = (int64_t)h.w_total;
  out->vol_max = (int64_t)h.vol_max;
  out->vol_sq = h.vol_sq;
  const double W = (double)h.w_total;
  out->inside = W > 0 ? (double)h.w_internal / W : 0.0;
  out->q = W > 0 ? out->inside - (double)h.vol_sq / (W * W) : 0.0;
  out->alpha = W > 0 ? (double)h.vol_max / W : 0.0;
  out->bound = 1.0 - out->q - out->alpha;
}

}  // namespace gp
