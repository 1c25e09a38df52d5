// contract.cu -- cluster contraction (Sec. 2): coarse node A weighs the sum
// of its members' weights; coarse edge {A, B}, A != B, weighs the total
// weight of the fine edges between the clusters.
//
// Fine nodes are bucketed by coarse id; each coarse node then aggregates the
// (coarse neighbour, weight) pairs of all its members in a hash table (a
// warp with a 256-slot shared-memory table when the members have at most 128
// entries together, otherwise a block with a 4096-slot shared table or a
// global table), writing its row into a temporary at an upper-bound offset;
// the rows are finally packed into the coarse CSR.  Row order inside a
// coarse row is unspecified.
#include "gp_internal.cuh"

namespace gp {

namespace {

constexpr unsigned FULL = 0xFFFFFFFFu;
constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;
constexpr int kWarpSlots = 256;
constexpr int kWarpMaxUb = 128;
constexpr int kBlockSmemSlots = 4096;

__device__ __forceinline__ unsigned slot_hash(int B, int bits) {
  return ((unsigned)B * 2654435761u) >> (32 - bits);
}

__device__ __forceinline__ void table_add(int *tk, int *tv, int mask, int bits, int B, int w) {
  unsigned s = slot_hash(B, bits);
  for (int probe = 0; probe <= mask; probe++) {  // bounded: the table never fills
    const int prev = atomicCAS(&tk[s], -1, B);
    if (prev == -1 || prev == B) { atomicAdd(&tv[s], w); return; }
    s = (s + 1) & (unsigned)mask;
  }
}

__global__ void k_member_count(const int32_t *xadj, const int32_t *vwgt, const int32_t *cmap, int n,
                               int32_t *cnt, int32_t *ub, int32_t *cw) {
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n;
       v += (int64_t)gridDim.x * blockDim.x) {
    const int A = cmap[v];
    atomicAdd(&cnt[A], 1);
    atomicAdd(&ub[A], xadj[v + 1] - xadj[v]);
    atomicAdd(&cw[A], vwgt[v]);
  }
}

__global__ void k_member_fill(const int32_t *cmap, int n, const int32_t *mstart, int32_t *cursor,
                              int32_t *members) {
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n;
       v += (int64_t)gridDim.x * blockDim.x) {
    const int A = cmap[v];
    members[mstart[A] + atomicAdd(&cursor[A], 1)] = (int32_t)v;
  }
}

struct AggArgs {
  const int32_t *xadj, *adjncy, *adjwgt, *cmap, *mstart, *members, *ub, *tstart;
  int nc;
  int32_t *tkeys, *tvals, *rowcnt;
  int32_t *large, *nlarge;
  int32_t *gkeys, *gvals;
  int64_t gstride;
  unsigned long long *units;
};

// One warp per coarse node whose members hold <= 128 entries.
__global__ void __launch_bounds__(kThreads) k_agg_warp(AggArgs a) {
  __shared__ int s_k[kWarps][kWarpSlots];
  __shared__ int s_v[kWarps][kWarpSlots];
  const int lane = (int)lane_id(), wib = threadIdx.x >> 5;
  int *tk = s_k[wib], *tv = s_v[wib];
  for (int t = lane; t < kWarpSlots; t += 32) { tk[t] = -1; tv[t] = 0; }
  __syncwarp();
  const int wid = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5);
  const int nw = (int)((gridDim.x * blockDim.x) >> 5);
  unsigned long long ue = 0, uout = 0;
  for (int A = wid; A < a.nc; A += nw) {
    if (a.ub[A] > kWarpMaxUb) {
      if (lane == 0) a.large[atomicAdd(a.nlarge, 1)] = A;
      continue;
    }
    const int m0 = a.mstart[A], m1 = a.mstart[A + 1];
    for (int mb = m0; mb < m1; mb += 32) {
      int st = 0, d = 0;
      if (mb + lane < m1) {
        const int v = a.members[mb + lane];
        st = a.xadj[v];
        d = a.xadj[v + 1] - st;
      }
      int incl = d;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(FULL, incl, o);
        if (lane >= o) incl += y;
      }
      const int excl = incl - d;
      const int total = __shfl_sync(FULL, incl, 31);
      ue += total;
      for (int f0 = 0; f0 < total; f0 += 32) {
        const int f = f0 + lane;
        // member j of entry f: number of lanes whose inclusive end is <= f
        int j = 0;
#pragma unroll
        for (int step = 16; step > 0; step >>= 1) {
          const int val = __shfl_sync(FULL, incl, j + step - 1);
          if (val <= f) j += step;
        }
        const int sj = __shfl_sync(FULL, st, j);
        const int ej = __shfl_sync(FULL, excl, j);
        if (f < total) {
          const int e = sj + (f - ej);
          const int B = a.cmap[a.adjncy[e]];
          if (B != A) table_add(tk, tv, kWarpSlots - 1, 8, B, a.adjwgt[e]);
        }
      }
    }
    __syncwarp();
    const int base = a.tstart[A];
    int cnt = 0;
    for (int t0 = 0; t0 < kWarpSlots; t0 += 32) {
      const int key = tk[t0 + lane];
      const bool occ = key >= 0;
      const unsigned m = __ballot_sync(FULL, occ);
      if (occ) {
        const int pos = base + cnt + __popc(m & lanemask_lt());
        a.tkeys[pos] = key;
        a.tvals[pos] = tv[t0 + lane];
      }
      cnt += __popc(m);
      tk[t0 + lane] = -1;
      tv[t0 + lane] = 0;
    }
    if (lane == 0) a.rowcnt[A] = cnt;
    uout += cnt;
    __syncwarp();
  }
  if (a.units && lane == 0) {
    atomicAdd(a.units + 0, ue);
    atomicAdd(a.units + 3, uout);
  }
}

// One block per coarse node of the large list.
__global__ void __launch_bounds__(kThreads) k_agg_block(AggArgs a) {
  __shared__ int s_k[kBlockSmemSlots];
  __shared__ int s_v[kBlockSmemSlots];
  __shared__ int s_cnt;
  for (int t = threadIdx.x; t < kBlockSmemSlots; t += blockDim.x) { s_k[t] = -1; s_v[t] = 0; }
  __syncthreads();
  const int nl = *a.nlarge;
  int *gk = a.gkeys ? a.gkeys + (int64_t)blockIdx.x * a.gstride : nullptr;
  int *gv = a.gvals ? a.gvals + (int64_t)blockIdx.x * a.gstride : nullptr;
  const int lane = (int)lane_id(), wib = threadIdx.x >> 5;
  unsigned long long ue = 0, uout = 0;
  for (int li = blockIdx.x; li < nl; li += gridDim.x) {
    const int A = a.large[li];
    const int ub = a.ub[A];
    int bits = 1;
    while ((1 << bits) < 2 * ub) bits++;
    const int tsize = 1 << bits;
    const bool in_smem = tsize <= kBlockSmemSlots;
    int *tk = in_smem ? s_k : gk;
    int *tv = in_smem ? s_v : gv;
    const int m0 = a.mstart[A], m1 = a.mstart[A + 1];
    for (int mi = m0 + wib; mi < m1; mi += kWarps) {
      const int v = a.members[mi];
      const int st = a.xadj[v], en = a.xadj[v + 1];
      for (int e = st + lane; e < en; e += 32) {
        const int B = a.cmap[a.adjncy[e]];
        if (B != A) table_add(tk, tv, tsize - 1, bits, B, a.adjwgt[e]);
      }
    }
    if (threadIdx.x == 0) s_cnt = 0;
    __syncthreads();
    const int base = a.tstart[A];
    for (int t = threadIdx.x; t < tsize; t += blockDim.x) {
      const int key = tk[t];
      if (key >= 0) {
        const int pos = atomicAdd(&s_cnt, 1);
        a.tkeys[base + pos] = key;
        a.tvals[base + pos] = tv[t];
        tk[t] = -1;
        tv[t] = 0;
      }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      a.rowcnt[A] = s_cnt;
      ue += ub;
      uout += s_cnt;
    }
    __syncthreads();
  }
  if (a.units && threadIdx.x == 0) {
    atomicAdd(a.units + 0, ue);
    atomicAdd(a.units + 3, uout);
  }
}

__global__ void k_max_i32(const int32_t *x, int n, int *out) {
  int m = 0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    m = x[i] > m ? x[i] : m;
  m = warp_max(m);
  if (lane_id() == 0 && m) atomicMax(out, m);
}

// Packs the rows from the upper-bound layout into the final CSR.
__global__ void __launch_bounds__(kThreads) k_pack_rows(const int32_t *tstart, const int32_t *rowcnt,
                                                        const int32_t *xadj_out, int nc,
                                                        const int32_t *tkeys, const int32_t *tvals,
                                                        int32_t *adj, int32_t *w) {
  const int lane = (int)lane_id();
  const int wid = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5);
  const int nw = (int)((gridDim.x * blockDim.x) >> 5);
  for (int A = wid; A < nc; A += nw) {
    const int src = tstart[A], dst = xadj_out[A], c = rowcnt[A];
    for (int j = lane; j < c; j += 32) {
      adj[dst + j] = tkeys[src + j];
      w[dst + j] = tvals[src + j];
    }
  }
}

}  // namespace

void contract_graph(gp_ctx *ctx, const DevGraph &g, const int32_t *cmap, int32_t nc, DevGraph &out) {
  TraceTimer trace(ctx);
  const int n = g.n;
  const int grid = grid_for(n, 256, ctx->num_sms * 8);
  DBuf<int32_t> cnt(ctx, (size_t)nc + 1), ub(ctx, (size_t)nc + 1), cw(ctx, (size_t)nc + 1);
  DBuf<int32_t> mstart(ctx, (size_t)nc + 1), tstart(ctx, (size_t)nc + 1), cursor(ctx, (size_t)nc + 1);
  DBuf<int32_t> members(ctx, (size_t)n);
  {
    ProfScope ps(ctx, PROF_CONTRACT_AUX);
    cnt.zero(); ub.zero(); cw.zero(); cursor.zero();
    k_member_count<<<grid, 256, 0, ctx->stream>>>(g.xadj, g.vwgt, cmap, n, cnt.get(), ub.get(), cw.get());
    GP_LAUNCH_CHECK();
    scan_exclusive_i32(ctx, cnt.get(), mstart.get(), nc + 1, nullptr);
    scan_exclusive_i32(ctx, ub.get(), tstart.get(), nc + 1, nullptr);
    k_member_fill<<<grid, 256, 0, ctx->stream>>>(cmap, n, mstart.get(), cursor.get(), members.get());
    GP_LAUNCH_CHECK();
  }
  DBuf<int32_t> tkeys(ctx, (size_t)(g.m2 > 0 ? g.m2 : 1)), tvals(ctx, (size_t)(g.m2 > 0 ? g.m2 : 1));
  DBuf<int32_t> rowcnt(ctx, (size_t)nc + 1), large(ctx, (size_t)nc + 1), nlarge(ctx, 1);
  rowcnt.zero();
  nlarge.zero();
  AggArgs a{};
  a.xadj = g.xadj; a.adjncy = g.adjncy; a.adjwgt = g.adjwgt; a.cmap = cmap;
  a.mstart = mstart.get(); a.members = members.get(); a.ub = ub.get(); a.tstart = tstart.get();
  a.nc = nc; a.tkeys = tkeys.get(); a.tvals = tvals.get(); a.rowcnt = rowcnt.get();
  a.large = large.get(); a.nlarge = nlarge.get();
  a.units = ctx->d_units ? ctx->d_units + PROF_CONTRACT * PROF_UNITS : nullptr;
  // global tables when some coarse node needs more than the shared table
  DBuf<int> maxub(ctx, 1);
  maxub.zero();
  k_max_i32<<<grid_for(nc, 256, ctx->num_sms * 8), 256, 0, ctx->stream>>>(ub.get(), nc, maxub.get());
  GP_LAUNCH_CHECK();
  const int mub = read_scalar(ctx, maxub.get());
  int bits = 1;
  while ((1 << bits) < 2 * mub) bits++;
  const int lblocks = ctx->num_sms * 4;
  DBuf<int32_t> gk, gv;
  if ((1 << bits) > kBlockSmemSlots) {
    a.gstride = (int64_t)1 << bits;
    gk.reset(ctx, (size_t)(a.gstride * lblocks));
    gv.reset(ctx, (size_t)(a.gstride * lblocks));
    gk.fill_bytes(0xFF);
    gv.zero();
    a.gkeys = gk.get();
    a.gvals = gv.get();
  }
  {
    ProfScope ps(ctx, PROF_CONTRACT);
    k_agg_warp<<<grid_for((int64_t)nc * 32, kThreads, ctx->num_sms * 8), kThreads, 0, ctx->stream>>>(a);
    GP_LAUNCH_CHECK();
    k_agg_block<<<lblocks, kThreads, 0, ctx->stream>>>(a);
    GP_LAUNCH_CHECK();
  }
  DBuf<int32_t> total(ctx, 1);
  out.n = nc;
  out.bx.reset(ctx, (size_t)nc + 1);
  out.xadj = out.bx.get();
  scan_exclusive_i32(ctx, rowcnt.get(), out.xadj, nc + 1, total.get());
  const int32_t m2 = read_scalar(ctx, total.get());
  out.m2 = m2;
  out.ba.reset(ctx, (size_t)m2);
  out.bw.reset(ctx, (size_t)m2);
  out.adjncy = out.ba.get();
  out.adjwgt = out.bw.get();
  {
    ProfScope ps(ctx, PROF_CONTRACT_AUX);
    k_pack_rows<<<grid_for((int64_t)nc * 32, kThreads, ctx->num_sms * 8), kThreads, 0, ctx->stream>>>(
        tstart.get(), rowcnt.get(), out.xadj, nc, tkeys.get(), tvals.get(), out.adjncy, out.adjwgt);
    GP_LAUNCH_CHECK();
  }
  out.bv.reset(ctx, (size_t)nc);
  out.vwgt = out.bv.get();
  if (trace.on())
    fprintf(stderr, "[gp contract] n=%d m2=%lld -> n=%d m2=%lld ms=%.2f\n", n, (long long)g.m2, nc,
            (long long)out.m2, trace.ms());
  if (nc > 0)
    GP_CUDA(cudaMemcpyAsync(out.vwgt, cw.get(), sizeof(int32_t) * nc, cudaMemcpyDeviceToDevice,
                            ctx->stream));
}

}  // namespace gp
