// contract.cu -- cluster contraction (Sec. 2): coarse node A weighs the sum
// of its members' weights; coarse edge {A, B}, A != B, weighs the total
// weight of the fine edges between the clusters.
//
// Three passes over the fine graph, each with coalesced streams:
//  reserve: every fine node reserves room for its row inside its coarse
//           node's segment (an atomic add on the segment length returns the
//           node's offset) and adds its weight to the coarse node;
//  map    : warps walk 32 consecutive fine rows at a time (one contiguous
//           range of entries) and write (coarse id of the neighbour, weight)
//           into the owner's segment; entries inside the cluster are marked;
//  merge  : each segment is summed by coarse neighbour in a hash table (a
//           warp with a shared-memory table up to 256 entries, a block with
//           a 4096-slot shared or a global table above) and written back in
//           place, compacted;
// and the merged rows are finally packed into the coarse CSR.  Row order
// inside a coarse row is unspecified.
#include "gp_internal.cuh"

namespace gp {

namespace {

constexpr unsigned FULL = 0xFFFFFFFFu;
constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;
constexpr int kWarpSlots = 256;
constexpr int kWarpMaxUb = 128;
constexpr int kBlockSmemSlots = 4096;
constexpr int kMapUnroll = 8;

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

__device__ __forceinline__ int table_bits(int entries) {
  int bits = 5;
  while ((1 << bits) < 2 * entries) bits++;
  return bits;
}

// Segment length (the member rows' total length) and weight of every coarse
// node; moff[v] = offset of v's row inside its coarse node's segment.
__global__ void k_reserve(const int32_t *xadj, const int32_t *vwgt, const int32_t *cmap, int n, int32_t *seg,
                          int32_t *cw, int32_t *moff) {
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n;
       v += (int64_t)gridDim.x * blockDim.x) {
    const int A = cmap[v];
    moff[v] = atomicAdd(&seg[A], xadj[v + 1] - xadj[v]);
    atomicAdd(&cw[A], vwgt[v]);
  }
}

// (coarse neighbour, weight) of every fine entry into its owner's segment;
// entries inside the owner's cluster get neighbour -1.
__global__ void __launch_bounds__(kThreads) k_map(const int32_t *xadj, const int32_t *adjncy,
                                                  const int32_t *adjwgt, const int32_t *cmap,
                                                  const int32_t *moff, const int32_t *tstart, int n,
                                                  int2 *temp, unsigned long long *units) {
  const int lane = (int)lane_id();
  const int wid = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5);
  const int nw = (int)((gridDim.x * blockDim.x) >> 5);
  unsigned long long ue = 0;
  for (int64_t u0 = (int64_t)wid * 32; u0 < n; u0 += (int64_t)nw * 32) {
    const int64_t u = u0 + lane;
    const bool valid = u < n;
    int xs = 0, xe = 0x7FFFFFFF, A = -2, base = 0;
    if (valid) {
      xs = xadj[u];
      xe = xadj[u + 1];
      A = cmap[u];
      base = tstart[A] + moff[u] - xs;
    }
    const int e0 = __shfl_sync(FULL, xs, 0);
    const int last = (int)((n - u0) < 32 ? (n - u0) : 32) - 1;
    const int e1 = __shfl_sync(FULL, xe, last);
    if (lane == 0) ue += (unsigned long long)(e1 - e0);
    // kMapUnroll entries per lane in flight: ids, then coarse ids, then the writes
    for (int f0 = e0; f0 < e1; f0 += 32 * kMapUnroll) {
      int e[kMapUnroll], bj[kMapUnroll], Aj[kMapUnroll], nb[kMapUnroll];
#pragma unroll
      for (int r = 0; r < kMapUnroll; r++) {
        e[r] = f0 + r * 32 + lane;
        int j = 0;  // owner: lanes whose row ends at or before e
#pragma unroll
        for (int step = 16; step > 0; step >>= 1) {
          const int val = __shfl_sync(FULL, xe, j + step - 1);
          if (val <= e[r]) j += step;
        }
        bj[r] = __shfl_sync(FULL, base, j);
        Aj[r] = __shfl_sync(FULL, A, j);
      }
#pragma unroll
      for (int r = 0; r < kMapUnroll; r++) nb[r] = e[r] < e1 ? __ldcs(adjncy + e[r]) : 0;  // read once: evict first
#pragma unroll
      for (int r = 0; r < kMapUnroll; r++) nb[r] = e[r] < e1 ? cmap[nb[r]] : 0;
#pragma unroll
      for (int r = 0; r < kMapUnroll; r++)
        if (e[r] < e1) temp[bj[r] + e[r]] = nb[r] == Aj[r] ? make_int2(-1, 0) : make_int2(nb[r], adjwgt ? __ldcs(adjwgt + e[r]) : 1);
    }
  }
  ue = warp_sum(ue);
  if (units && lane == 0) {
    atomicAdd(units + 0, ue);
    if (!adjwgt) atomicAdd(units + 5, ue);
  }
}

struct MergeArgs {
  const int32_t *tstart;
  int nc;
  int2 *temp;
  int32_t *rowcnt;
  int32_t *large, *nlarge;
  int32_t *gkeys, *gvals;
  int64_t gstride;
  unsigned long long *units;
};

// One warp per coarse node whose segment holds at most kWarpMaxUb entries.
__global__ void __launch_bounds__(kThreads) k_merge_warp(MergeArgs a) {
  __shared__ int s_k[kWarps][kWarpSlots];
  __shared__ int s_v[kWarps][kWarpSlots];
  const int lane = (int)lane_id(), wib = threadIdx.x >> 5;
  int *tk = s_k[wib], *tv = s_v[wib];
  for (int t = lane; t < kWarpSlots; t += 32) { tk[t] = -1; tv[t] = 0; }
  __syncwarp();
  const int wid = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5);
  const int nw = (int)((gridDim.x * blockDim.x) >> 5);
  unsigned long long uout = 0;
  for (int A = wid; A < a.nc; A += nw) {
    const int s0 = a.tstart[A], s1 = a.tstart[A + 1];
    const int len = s1 - s0;
    if (len > kWarpMaxUb) {
      if (lane == 0) a.large[atomicAdd(a.nlarge, 1)] = A;
      continue;
    }
    const int bits = table_bits(len), tsize = 1 << bits;
    for (int i0 = s0; i0 < s1; i0 += 64) {  // two entries per lane in flight
      const int i1 = i0 + lane, i2 = i0 + 32 + lane;
      const int2 x1 = i1 < s1 ? __ldcs(a.temp + i1) : make_int2(-1, 0);
      const int2 x2 = i2 < s1 ? __ldcs(a.temp + i2) : make_int2(-1, 0);
      if (x1.x >= 0) table_add(tk, tv, tsize - 1, bits, x1.x, x1.y);
      if (x2.x >= 0) table_add(tk, tv, tsize - 1, bits, x2.x, x2.y);
    }
    __syncwarp();
    // extract in slot order and leave the table clean for the next node
    int cnt = 0;
    for (int t0 = 0; t0 < tsize; t0 += 32) {
      const int key = tk[t0 + lane];
      const bool occ = key >= 0;
      const unsigned m = __ballot_sync(FULL, occ);
      if (occ) {
        a.temp[s0 + cnt + __popc(m & lanemask_lt())] = make_int2(key, tv[t0 + lane]);
        tk[t0 + lane] = -1;
        tv[t0 + lane] = 0;
      }
      cnt += __popc(m);
    }
    if (lane == 0) a.rowcnt[A] = cnt;
    uout += cnt;
    __syncwarp();
  }
  if (a.units && lane == 0) atomicAdd(a.units + 3, uout);
}

// One block per coarse node of the large list.
__global__ void __launch_bounds__(kThreads) k_merge_block(MergeArgs a) {
  __shared__ int s_k[kBlockSmemSlots];
  __shared__ int s_v[kBlockSmemSlots];
  __shared__ int s_cnt;
  const int nl = *a.nlarge;
  int *gk = a.gkeys ? a.gkeys + (int64_t)blockIdx.x * a.gstride : nullptr;
  int *gv = a.gvals ? a.gvals + (int64_t)blockIdx.x * a.gstride : nullptr;
  unsigned long long uout = 0;
  for (int li = blockIdx.x; li < nl; li += gridDim.x) {
    const int A = a.large[li];
    const int s0 = a.tstart[A], s1 = a.tstart[A + 1];
    const int bits = table_bits(s1 - s0), tsize = 1 << bits;
    const bool in_smem = tsize <= kBlockSmemSlots;
    int *tk = in_smem ? s_k : gk;
    int *tv = in_smem ? s_v : gv;
    for (int t = threadIdx.x; t < tsize; t += blockDim.x) { tk[t] = -1; tv[t] = 0; }
    if (threadIdx.x == 0) s_cnt = 0;
    __syncthreads();
    for (int i = s0 + threadIdx.x; i < s1; i += blockDim.x) {
      const int2 x = a.temp[i];
      if (x.x >= 0) table_add(tk, tv, tsize - 1, bits, x.x, x.y);
    }
    __syncthreads();
    for (int t = threadIdx.x; t < tsize; t += blockDim.x) {
      const int key = tk[t];
      if (key >= 0) a.temp[s0 + atomicAdd(&s_cnt, 1)] = make_int2(key, tv[t]);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      a.rowcnt[A] = s_cnt;
      uout += s_cnt;
    }
    __syncthreads();
  }
  if (a.units && threadIdx.x == 0) atomicAdd(a.units + 3, uout);
}

__global__ void k_max_i32(const int32_t *x, int n, int *out) {
  int m = 0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    m = x[i] > m ? x[i] : m;
  m = warp_max(m);
  if (lane_id() == 0 && m) atomicMax(out, m);
}

// Packs the merged rows from the segment layout into the final CSR.
__global__ void __launch_bounds__(kThreads) k_pack_rows(const int32_t *tstart, const int32_t *rowcnt,
                                                        const int32_t *xadj_out, int nc, const int2 *temp,
                                                        int32_t *adj, int32_t *w) {
  const int lane = (int)lane_id();
  const int wid = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5);
  const int nw = (int)((gridDim.x * blockDim.x) >> 5);
  for (int A = wid; A < nc; A += nw) {
    const int src = tstart[A], dst = xadj_out[A], c = rowcnt[A];
    for (int j = lane; j < c; j += 32) {
      const int2 x = temp[src + j];
      adj[dst + j] = x.x;
      w[dst + j] = x.y;
    }
  }
}

}  // namespace

void contract_graph(gp_ctx *ctx, const DevGraph &g, const int32_t *cmap, int32_t nc, DevGraph &out) {
  TraceTimer trace(ctx);
  const int n = g.n;
  const int grid = grid_for(n, 256, ctx->num_sms * 8);
  DBuf<int32_t> seg(ctx, (size_t)nc + 1), cw(ctx, (size_t)nc + 1), tstart(ctx, (size_t)nc + 1);
  DBuf<int32_t> moff(ctx, (size_t)(n > 0 ? n : 1));
  {
    ProfScope ps(ctx, PROF_CONTRACT_AUX);
    seg.zero(); cw.zero();
    k_reserve<<<grid, 256, 0, ctx->stream>>>(g.xadj, g.vwgt, cmap, n, seg.get(), cw.get(), moff.get());
    GP_LAUNCH_CHECK();
    scan_exclusive_i32(ctx, seg.get(), tstart.get(), nc + 1, nullptr);
  }
  DBuf<int2> temp(ctx, (size_t)(g.m2 > 0 ? g.m2 : 1));
  DBuf<int32_t> rowcnt(ctx, (size_t)nc + 1), large(ctx, (size_t)nc + 1), nlarge(ctx, 1);
  rowcnt.zero();
  nlarge.zero();
  MergeArgs a{};
  a.tstart = tstart.get(); a.nc = nc; a.temp = temp.get(); a.rowcnt = rowcnt.get();
  a.large = large.get(); a.nlarge = nlarge.get();
  unsigned long long *units = ctx->d_units ? ctx->d_units + PROF_CONTRACT * PROF_UNITS : nullptr;
  a.units = units;
  // global tables when some coarse node needs more than the shared table
  DBuf<int> maxseg(ctx, 1);
  maxseg.zero();
  k_max_i32<<<grid_for(nc, 256, ctx->num_sms * 8), 256, 0, ctx->stream>>>(seg.get(), nc, maxseg.get());
  GP_LAUNCH_CHECK();
  const int mseg = read_scalar(ctx, maxseg.get());
  int bits = 1;
  while ((1 << bits) < 2 * mseg) bits++;
  int lblocks = ctx->num_sms * 4;
  DBuf<int32_t> gk, gv;
  if ((1 << bits) > kBlockSmemSlots) {
    a.gstride = (int64_t)1 << bits;
    lblocks = table_blocks(g.m2, a.gstride, lblocks);
    gk.reset(ctx, (size_t)(a.gstride * lblocks));
    gv.reset(ctx, (size_t)(a.gstride * lblocks));
    a.gkeys = gk.get();
    a.gvals = gv.get();
  }
  {
    ProfScope ps(ctx, PROF_CONTRACT);
    if (n > 0) {
      k_map<<<grid_for((int64_t)n, kThreads, ctx->num_sms * 16), kThreads, 0, ctx->stream>>>(
          g.xadj, g.adjncy, g.unit_w ? nullptr : g.adjwgt, cmap, moff.get(), tstart.get(), n, temp.get(), units);
      GP_LAUNCH_CHECK();
    }
    k_merge_warp<<<grid_for((int64_t)nc * 32, kThreads, ctx->num_sms * 8), kThreads, 0, ctx->stream>>>(a);
    GP_LAUNCH_CHECK();
    k_merge_block<<<lblocks, kThreads, 0, ctx->stream>>>(a);
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
        tstart.get(), rowcnt.get(), out.xadj, nc, temp.get(), out.adjncy, out.adjwgt);
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
