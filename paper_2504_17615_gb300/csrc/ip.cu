// ip.cu -- initial partitioning of the coarsest graph by recursive
// bisection (Sec. 4.3), plus the greedy rebalancer.
//
// All subproblems of one depth of the bisection tree are split together;
// every (subproblem, trial) pair runs in its own warp.  A trial grows side 1
// greedily: among nodes that still fit under L1, frontier nodes (connected
// to side 1) of largest gain 2 conn(v) - deg'(v), ties by the smallest id;
// when no frontier node fits, the node of smallest (h32(key(IP, 0, bid), v,
// t), v).  It stops once side 1 weighs >= T1.  The trial with the smallest
// cut (ties: lowest trial) wins.
//
// Each growing step takes up to B = 1 + n'/1024 frontier nodes in order of
// their gains at the start of the step, skipping those that no longer fit
// (one node per step below 1024 nodes).
//
// A node costs O(deg + n'/64), not O(n'): node lists are sorted by id, so
// local index order is id order; every 64-node chunk keeps the largest key
// (gain, -index) of its live frontier nodes, raised with a 64-bit atomicMax
// when a neighbour's connection grows and recomputed only for the chunks of
// the nodes just taken.  A picked node that no longer fits is retired for
// good (side 1 only gets heavier), which leaves the choice among the nodes
// that fit unchanged.
//
// Steps of B >= 8 nodes select their nodes together instead of one by one:
// the chunk maxima are sorted, the q-th largest of them (q = nodes still
// wanted) is a threshold that at least q frontier nodes reach, and all of
// those lie in the q leading chunks; they are ranked, and one warp walks them
// in key order with prefix sums of their weights, taking, retiring or
// stopping exactly as the one-by-one walk would.  A round that runs out of
// candidates (retired nodes) selects again.
#include "gp_internal.cuh"

#include <algorithm>

namespace gp {

namespace {

constexpr int kUpdUnroll = 8;
constexpr int kSmemBatch = 64;  // the nodes of a growing step live in shared memory up to this many
constexpr int kChunkNodes = 64;
constexpr int kBatchMinB = 8;    // steps of at least this many nodes select them together
constexpr int kSortCap = 512;    // chunk maxima sorted per selection round
constexpr int kCandCap = 256;    // candidates ranked per round, a quarter per warp; more fall back to
                                 // one-by-one extraction
// dynamic part (static shared variables use the rest: the sort and candidate buffers and a few words)
constexpr int kMaxSmemBytes = 227 * 1024 - (kSortCap + 2 * kCandCap) * 8 - kSmemBatch * 4 - 1024;

struct Sub {
  int32_t start, count;  // node list range
  int32_t bid;           // heap id of the bisection
  int32_t pad;
  int64_t T1, L1;        // side-1 target and limit
};

// Per-node state of a trial: S_FREE not connected to side 1, S_FRONT free and
// connected, S_ONE in side 1, S_OUT retired (can never fit again).
enum : uint8_t { S_FREE = 0, S_ONE = 1, S_OUT = 2, S_FRONT = 3 };

struct IpArgs {
  const int32_t *lxadj;            // local CSR of every subproblem (by list position)
  const int2 *ladj;                // (local index, weight) of internal neighbours
  const int32_t *vtx, *cvl, *dpl;  // by list position: node id, weight, deg'
  const Sub *subs;
  int trials;
  int n;
  uint64_t seed;
  int smem_nodes;                  // subproblems up to this size keep their state in shared memory
  int cv16;                        // node weights fit 16 bits: kept in shared memory too
  int hv_smem;                     // the trial's fallback hashes fit in shared memory too
  int32_t *gg;                     // global fallback state per block
  uint8_t *gst;
  uint16_t *gcv;
  unsigned long long *gbest, *gsup;
  int64_t gnodes, gchunks;
  int32_t *gbatch;                 // per block: the nodes taken in the current step
  int batch_cap;
  unsigned long long *trace;       // optional: [0] growing steps, [1] fallback scans, [2] retired nodes
  int64_t *trial_cut;              // per block
  uint8_t *flags;                  // [trial][n] side-1 flag by list position
};

__device__ __forceinline__ unsigned long long gain_key(int64_t gain, int j) {
  return ((unsigned long long)(gain + 2147483648ll) << 32) | (0xFFFFFFFFu - (unsigned)j);
}

// 64-bit maximum / minimum over the warp with two 32-bit reductions each.
__device__ __forceinline__ unsigned long long wmax_u64(unsigned long long x) {
  const unsigned hi = (unsigned)(x >> 32);
  const unsigned mh = __reduce_max_sync(0xFFFFFFFFu, hi);
  const unsigned ml = __reduce_max_sync(0xFFFFFFFFu, hi == mh ? (unsigned)x : 0u);
  return ((unsigned long long)mh << 32) | ml;
}

__device__ __forceinline__ unsigned long long wmin_u64(unsigned long long x) {
  const unsigned hi = (unsigned)(x >> 32);
  const unsigned mh = __reduce_min_sync(0xFFFFFFFFu, hi);
  const unsigned ml = __reduce_min_sync(0xFFFFFFFFu, hi == mh ? (unsigned)x : 0xFFFFFFFFu);
  return ((unsigned long long)mh << 32) | ml;
}

// chunk best over the live frontier nodes of chunk c (one warp)
__device__ __forceinline__ void rescan_chunk(int c, int cnt, const int32_t *g, const uint8_t *st,
                                             unsigned long long *best) {
  const int lane = (int)lane_id();
  unsigned long long b = 0;
#pragma unroll
  for (int r = 0; r < kChunkNodes / 32; r++) {
    const int j = c * kChunkNodes + r * 32 + lane;
    if (j < cnt && st[j] == S_FRONT) {
      const unsigned long long key = gain_key(g[j], j);
      b = key > b ? key : b;
    }
  }
  b = wmax_u64(b);
  if (lane == 0) best[c] = b;
  __syncwarp();
}

constexpr int kIpWarps = 4;  // warps per (subproblem, trial)

// Bitonic sort of kSortCap = 512 keys into descending order by the block's
// 128 threads, four keys per thread in registers (thread t holds positions
// 4t .. 4t+3): partners at distance 1 and 2 are in the same thread, at 4 .. 64
// in the same warp (shuffles), at 128 and 256 in another warp (through x, the
// only stages with block barriers).  On return x[0, 512) holds the sorted keys
// and the block is synchronised.
static_assert(kSortCap == 4 * 32 * kIpWarps, "four keys per thread");
static_assert(kChunkNodes == 64, "two chunk nodes per lane");
constexpr int kSegCap = kCandCap / kIpWarps;  // candidates per warp and round

__device__ __forceinline__ unsigned long long keep(unsigned long long mine, unsigned long long other, bool take_max) {
  return take_max ? (mine > other ? mine : other) : (mine < other ? mine : other);
}

__device__ __forceinline__ void sort512_desc(unsigned long long (&r)[4], unsigned long long *x) {
  const int t = threadIdx.x;
#pragma unroll
  for (int size = 2; size <= kSortCap; size <<= 1) {
#pragma unroll
    for (int stride = size >> 1; stride > 0; stride >>= 1) {
      if (stride >= 128) {
#pragma unroll
        for (int k = 0; k < 4; k++) x[4 * t + k] = r[k];
        __syncthreads();
#pragma unroll
        for (int k = 0; k < 4; k++) {
          const int i = 4 * t + k;
          const unsigned long long o = x[i ^ stride];
          r[k] = keep(r[k], o, ((i & stride) == 0) == ((i & size) == 0));
        }
        __syncthreads();
      } else if (stride >= 4) {
#pragma unroll
        for (int k = 0; k < 4; k++) {
          const int i = 4 * t + k;
          const unsigned long long o = __shfl_xor_sync(0xFFFFFFFFu, r[k], stride / 4);
          r[k] = keep(r[k], o, ((i & stride) == 0) == ((i & size) == 0));
        }
      } else {
#pragma unroll
        for (int k = 0; k < 4; k++) {
          if (k & stride) continue;
          const int i = 4 * t + k;
          const unsigned long long lo = r[k], hi = r[k | stride];
          const bool desc = (i & size) == 0;
          r[k] = keep(lo, hi, desc);
          r[k | stride] = keep(lo, hi, !desc);
        }
      }
    }
  }
#pragma unroll
  for (int k = 0; k < 4; k++) x[4 * t + k] = r[k];
  __syncthreads();
}

__device__ __forceinline__ int node_of(unsigned long long key) {
  return (int)(0xFFFFFFFFu - (unsigned)(key & 0xFFFFFFFFull));
}

// One block of kIpWarps warps per (subproblem, trial).  Warp 0 takes the
// step's nodes from the chunk tournament; all warps then raise the
// connections of the taken nodes' neighbours, scan for the fallback node and
// add up the trial's cut.
__global__ void __launch_bounds__(32 * kIpWarps) k_ip_grow(IpArgs a) {
  extern __shared__ __align__(16) unsigned char dyn[];
  __shared__ int s_nb, s_nz, s_wc[kIpWarps];
  __shared__ long long s_w1;
  __shared__ unsigned long long s_red[kIpWarps];
  __shared__ unsigned long long s_sort[kSortCap], s_cand[kCandCap], s_rank[kCandCap];
  __shared__ int32_t s_batch[kSmemBatch];
  const int lane = (int)lane_id(), warp = threadIdx.x >> 5;
  const int si = blockIdx.x / a.trials, t = blockIdx.x % a.trials;
  const Sub S = a.subs[si];
  const int cnt = S.count, nch = (cnt + kChunkNodes - 1) / kChunkNodes;
  const int start = S.start;
  const int nsup = (nch + 31) / 32;
  unsigned long long *best, *sup;  // chunk maxima, and maxima over 32 chunks
  int32_t *g;
  uint8_t *st;
  uint16_t *cv = nullptr;
  uint32_t *hv = nullptr;  // fallback hashes of the trial, when shared memory has room for them
  if (cnt <= a.smem_nodes) {
    const int mch = (a.smem_nodes + kChunkNodes - 1) / kChunkNodes;
    const int msup = (mch + 31) / 32;
    best = reinterpret_cast<unsigned long long *>(dyn);
    sup = best + mch;
    g = reinterpret_cast<int32_t *>(dyn + sizeof(unsigned long long) * (mch + msup));
    unsigned char *tail = reinterpret_cast<unsigned char *>(g + a.smem_nodes);
    if (a.hv_smem) {
      hv = reinterpret_cast<uint32_t *>(tail);
      tail += sizeof(uint32_t) * a.smem_nodes;
    }
    if (a.cv16) {
      cv = reinterpret_cast<uint16_t *>(tail);
      tail += sizeof(uint16_t) * a.smem_nodes;
    }
    st = tail;
  } else {
    best = a.gbest + (int64_t)blockIdx.x * a.gchunks;
    sup = a.gsup + (int64_t)blockIdx.x * ((a.gchunks + 31) / 32);
    g = a.gg + (int64_t)blockIdx.x * a.gnodes;
    st = a.gst + (int64_t)blockIdx.x * a.gnodes;
    if (a.cv16) cv = a.gcv + (int64_t)blockIdx.x * a.gnodes;
  }
  const uint64_t kip = stream_key(a.seed, TAG_IP, 0, (uint32_t)S.bid);
  for (int j = threadIdx.x; j < cnt; j += blockDim.x) {
    g[j] = -a.dpl[start + j];
    st[j] = S_FREE;
    if (cv) cv[j] = (uint16_t)a.cvl[start + j];
    if (hv) hv[j] = h32(kip, (uint32_t)a.vtx[start + j], (uint32_t)t);
  }
  for (int c = threadIdx.x; c < nch; c += blockDim.x) best[c] = 0;
  for (int c = threadIdx.x; c < nsup; c += blockDim.x) sup[c] = 0;
  __syncthreads();
  int64_t w1 = 0;  // warp 0's copy is the authoritative one; others read s_w1
  const int B = 1 + cnt / 1024;  // nodes per growing step
  int32_t *batch = B <= kSmemBatch ? s_batch : a.gbatch + (int64_t)blockIdx.x * a.batch_cap;
  const bool batched = B >= kBatchMinB && cnt <= a.smem_nodes && nch <= kSortCap;
  for (;;) {
    if (threadIdx.x == 0) s_w1 = w1;
    __syncthreads();
    w1 = s_w1;
    if (w1 >= S.T1) break;
    // up to B nodes in (gain desc, id asc) order; gains stay frozen until the step ends
    bool seq = !batched;
    if (batched) {
      if (threadIdx.x == 0) {
        s_nb = 0;
        if (a.trace) atomicAdd(a.trace + 0, 1ull);
      }
      for (;;) {  // selection rounds
        __syncthreads();
        const int nb0 = s_nb;
        const long long w10 = s_w1;
        if (nb0 >= B || w10 >= S.T1) break;
        {
          unsigned long long rk[4];
#pragma unroll
          for (int k = 0; k < 4; k++) {
            const int i = 4 * (int)threadIdx.x + k;
            rk[k] = i < nch ? best[i] : 0ull;
          }
          if (threadIdx.x == 0) s_nz = 0;
          sort512_desc(rk, s_sort);
        }
        for (int i = threadIdx.x; i < kSortCap; i += blockDim.x)
          if (s_sort[i] != 0 && (i + 1 == kSortCap || s_sort[i + 1] == 0)) s_nz = i + 1;
        __syncthreads();
        const int nz = s_nz;
        if (nz == 0) break;  // no frontier node left
        const int q = min(B - nb0, nz);
        const unsigned long long tau = s_sort[q - 1];
        // every frontier node with key >= tau sits in one of the q leading chunks; each warp
        // gathers those of its chunks into its own segment of s_cand
        {
          int mine = 0;
          unsigned long long *seg = s_cand + warp * kSegCap;
          for (int r = warp; r < q; r += kIpWarps) {
            const int c = node_of(s_sort[r]) / kChunkNodes;
            const int j0 = c * kChunkNodes + lane, j1 = j0 + 32;
            unsigned long long k0 = 0, k1 = 0;
            if (j0 < cnt && st[j0] == S_FRONT) k0 = gain_key(g[j0], j0);
            if (j1 < cnt && st[j1] == S_FRONT) k1 = gain_key(g[j1], j1);
            const bool in0 = k0 != 0 && k0 >= tau, in1 = k1 != 0 && k1 >= tau;
            const unsigned m0 = __ballot_sync(0xFFFFFFFFu, in0), m1 = __ballot_sync(0xFFFFFFFFu, in1);
            const int p0 = mine + __popc(m0 & lanemask_lt());
            const int p1 = mine + __popc(m0) + __popc(m1 & lanemask_lt());
            if (in0 && p0 < kSegCap) seg[p0] = k0;
            if (in1 && p1 < kSegCap) seg[p1] = k1;
            mine += __popc(m0) + __popc(m1);
          }
          if (lane == 0) s_wc[warp] = mine;
        }
        __syncthreads();
        int wc[kIpWarps], C = 0;
        bool over = false;
#pragma unroll
        for (int w2 = 0; w2 < kIpWarps; w2++) {
          wc[w2] = s_wc[w2];
          C += wc[w2];
          over = over || wc[w2] > kSegCap;
        }
        if (over) { seq = true; break; }
        for (int t = threadIdx.x; t < C; t += blockDim.x) {  // keys are distinct: rank = place
          int at = -1, acc = 0;
#pragma unroll
          for (int w3 = 0; w3 < kIpWarps; w3++) {
            if (at < 0 && t < acc + wc[w3]) at = w3 * kSegCap + (t - acc);
            acc += wc[w3];
          }
          const unsigned long long x = s_cand[at];
          int r = 0;
#pragma unroll
          for (int w3 = 0; w3 < kIpWarps; w3++)
            for (int i2 = 0; i2 < wc[w3]; i2++) r += s_cand[w3 * kSegCap + i2] > x ? 1 : 0;
          s_rank[r] = x;
        }
        __syncthreads();
        if (warp == 0) {
          int nb = nb0;
          long long w = w10;
          int i0 = 0;
          while (i0 < C) {
            const int i = i0 + lane;
            int j = -1;
            long long c = 0;
            if (i < C) {
              j = node_of(s_rank[i]);
              c = cv ? (long long)cv[j] : (long long)a.cvl[start + j];
            }
            long long pre = c;  // weight of lanes i0..i
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
              const long long y = __shfl_up_sync(0xFFFFFFFFu, pre, o);
              if (lane >= o) pre += y;
            }
            // lane i is reached iff every earlier lane of the group was taken
            const bool considered = i < C && nb + (i - i0) < B && w + (pre - c) < S.T1;
            const bool fits = w + pre <= S.L1;
            const unsigned bad = __ballot_sync(0xFFFFFFFFu, !(considered && fits));
            const int f = bad ? __ffs(bad) - 1 : 32;
            if (lane < f) {
              st[j] = S_ONE;
              batch[nb + lane] = j;
            }
            const long long wf = __shfl_sync(0xFFFFFFFFu, pre, f > 0 ? f - 1 : 0);
            const bool cf = __shfl_sync(0xFFFFFFFFu, considered, f < 32 ? f : 0);
            if (f > 0) w += wf;
            nb += f;
            if (f == 32) { i0 += 32; continue; }
            if (i0 + f >= C || !cf) break;  // list used up, or the step is complete
            if (lane == f) {  // reached and does not fit: retired
              st[j] = S_OUT;
              if (a.trace) atomicAdd(a.trace + 2, 1ull);
            }
            i0 += f + 1;
          }
          if (lane == 0) { s_nb = nb; s_w1 = w; }
        }
        __syncthreads();
        // the q leading chunks' maxima again, two chunks per warp at a time
        for (int r = warp; r < q; r += 2 * kIpWarps) {
          const bool two = r + kIpWarps < q;
          const int ca = node_of(s_sort[r]) / kChunkNodes;
          const int cb = two ? node_of(s_sort[r + kIpWarps]) / kChunkNodes : ca;
          unsigned long long ba = 0, bb = 0;
#pragma unroll
          for (int rr = 0; rr < kChunkNodes / 32; rr++) {
            const int ja = ca * kChunkNodes + rr * 32 + lane, jb = cb * kChunkNodes + rr * 32 + lane;
            const bool fa = ja < cnt && st[ja] == S_FRONT, fb = jb < cnt && st[jb] == S_FRONT;
            if (fa) { const unsigned long long k = gain_key(g[ja], ja); ba = k > ba ? k : ba; }
            if (fb) { const unsigned long long k = gain_key(g[jb], jb); bb = k > bb ? k : bb; }
          }
          ba = wmax_u64(ba);
          bb = wmax_u64(bb);
          if (lane == 0) {
            best[ca] = ba;
            if (two) best[cb] = bb;
          }
        }
      }
      __syncthreads();
      if (seq) {  // the chunk groups' maxima again for the one-by-one walk
        for (int sc = warp; sc < nsup; sc += kIpWarps) {
          const int c = sc * 32 + lane;
          const unsigned long long x = wmax_u64(c < nch ? best[c] : 0ull);
          if (lane == 0) sup[sc] = x;
        }
        __syncthreads();
        w1 = s_w1;
      }
    }
    if (seq && warp == 0) {
      int nb = batched ? s_nb : 0;
      while (nb < B && w1 < S.T1) {
        unsigned long long b = 0;
        for (int c = lane; c < nsup; c += 32) b = sup[c] > b ? sup[c] : b;
        b = wmax_u64(b);
        if (b == 0) break;
        const int j = (int)(0xFFFFFFFFu - (unsigned)(b & 0xFFFFFFFFull));
        const int cj = cv ? (int)cv[j] : a.cvl[start + j];
        const bool fit = w1 + cj <= S.L1;
        if (lane == 0) {
          st[j] = fit ? S_ONE : S_OUT;  // S_OUT: cannot fit now, nor later
          if (fit) batch[nb] = j;
          if (a.trace && !fit) atomicAdd(a.trace + 2, 1ull);
        }
        if (fit) { nb++; w1 += cj; }
        __syncwarp();
        const int c = j / kChunkNodes;
        rescan_chunk(c, cnt, g, st, best);
        const int s0 = (c / 32) * 32;  // the maximum over c's 32 chunks again
        unsigned long long x = s0 + lane < nch ? best[s0 + lane] : 0;
        x = wmax_u64(x);
        if (lane == 0) sup[c / 32] = x;
        __syncwarp();
      }
      if (lane == 0) {
        s_nb = nb;
        s_w1 = w1;
        if (a.trace && !batched) atomicAdd(a.trace + 0, 1ull);
      }
    }
    __syncthreads();
    int nb = s_nb;
    w1 = s_w1;
    if (nb == 0) {  // no frontier node fits: the smallest-hash node that fits, found by all warps
      if (a.trace && threadIdx.x == 0) atomicAdd(a.trace + 1, 1ull);
      unsigned long long m = ~0ull;
      for (int jj = threadIdx.x; jj < cnt; jj += blockDim.x) {
        if (st[jj] != S_FREE) continue;
        const int cjj = cv ? (int)cv[jj] : a.cvl[start + jj];
        if (w1 + cjj > S.L1) continue;
        const uint32_t h = hv ? hv[jj] : h32(kip, (uint32_t)a.vtx[start + jj], (uint32_t)t);
        const unsigned long long key = ((unsigned long long)h << 32) | (unsigned)jj;
        m = key < m ? key : m;
      }
      m = wmin_u64(m);
      if (lane == 0) s_red[warp] = m;
      __syncthreads();
      if (threadIdx.x == 0) {
        unsigned long long mm = s_red[0];
        for (int q = 1; q < kIpWarps; q++) mm = s_red[q] < mm ? s_red[q] : mm;
        if (mm == ~0ull) {
          s_nb = -1;
        } else {
          const int j = (int)(unsigned)(mm & 0xFFFFFFFFull);
          s_w1 = w1 + (cv ? (int)cv[j] : a.cvl[start + j]);
          st[j] = S_ONE;
          batch[0] = j;
          s_nb = 1;
        }
      }
      __syncthreads();
      nb = s_nb;
      if (nb < 0) break;
      if (threadIdx.x == 0) w1 = s_w1;
    }
    if (threadIdx.x == 0) w1 = s_w1;
    // neighbours of the step's nodes, over their concatenated local rows (32 nodes at a time),
    // 32 * kUpdUnroll entries per warp and pass
    for (int b0 = 0; b0 < nb; b0 += 32) {
      int rs = 0, d = 0;
      if (b0 + lane < nb) {
        const int p = start + batch[b0 + lane];
        rs = a.lxadj[p];
        d = a.lxadj[p + 1] - rs;
      }
      int incl = d;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xFFFFFFFFu, incl, o);
        if (lane >= o) incl += y;
      }
      const int excl = incl - d, total = __shfl_sync(0xFFFFFFFFu, incl, 31);
      for (int f0 = warp * 32 * kUpdUnroll; f0 < total; f0 += kIpWarps * 32 * kUpdUnroll) {
        int idx[kUpdUnroll];
#pragma unroll
        for (int r = 0; r < kUpdUnroll; r++) {
          const int f = f0 + r * 32 + lane;
          int q = 0;
#pragma unroll
          for (int step = 16; step > 0; step >>= 1) {
            const int val = __shfl_sync(0xFFFFFFFFu, incl, q + step - 1);
            if (val <= f) q += step;
          }
          const int sq = __shfl_sync(0xFFFFFFFFu, rs, q), eq = __shfl_sync(0xFFFFFFFFu, excl, q);
          idx[r] = f < total ? sq + (f - eq) : -1;
        }
        int2 e[kUpdUnroll];
#pragma unroll
        for (int r = 0; r < kUpdUnroll; r++) e[r] = idx[r] >= 0 ? a.ladj[idx[r]] : make_int2(-1, 0);
#pragma unroll
        for (int r = 0; r < kUpdUnroll; r++) {
          if (e[r].x < 0) continue;
          const uint8_t su = st[e[r].x];
          if (su == S_FREE || su == S_FRONT) {
            const int ng = atomicAdd(&g[e[r].x], 2 * e[r].y) + 2 * e[r].y;
            if (su == S_FREE) st[e[r].x] = S_FRONT;
            atomicMax(&best[e[r].x / kChunkNodes], gain_key(ng, e[r].x));
          }
        }
      }
    }
    __syncthreads();
    // the maxima over 32 chunks again, from the raised chunk maxima (one warp per group); the
    // batched selection reads the chunk maxima alone
    for (int sc = warp; sc < (batched ? 0 : nsup); sc += kIpWarps) {
      const int c = sc * 32 + lane;
      const unsigned long long x = wmax_u64(c < nch ? best[c] : 0ull);
      if (lane == 0) sup[sc] = x;
    }
    __syncthreads();
  }
  // cut of this trial inside the subproblem
  unsigned long long cut = 0;
  for (int jj = threadIdx.x; jj < cnt; jj += blockDim.x) {
    if (st[jj] != S_ONE) continue;
    const int p = start + jj;
    for (int e = a.lxadj[p]; e < a.lxadj[p + 1]; e++) {
      const int2 x = a.ladj[e];
      if (st[x.x] != S_ONE) cut += (unsigned long long)x.y;
    }
  }
  cut = warp_sum(cut);
  if (lane == 0) s_red[warp] = cut;
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned long long c = 0;
    for (int q = 0; q < kIpWarps; q++) c += s_red[q];
    a.trial_cut[blockIdx.x] = (int64_t)c;
  }
  uint8_t *fl = a.flags + (int64_t)t * a.n + start;
  for (int jj = threadIdx.x; jj < cnt; jj += blockDim.x) fl[jj] = st[jj] == S_ONE;
}

__global__ void k_sub_count(const int32_t *sp, const int32_t *vwgt, int n, int32_t *cnt, long long *w) {
  for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
    const int s = sp[v];
    if (s < 0) continue;
    atomicAdd(&cnt[s], 1);
    atomicAdd((unsigned long long *)&w[s], (unsigned long long)vwgt[v]);
  }
}

// sort keys: live nodes by (subproblem, id) first, finished nodes after them
__global__ void k_sub_keys(const int32_t *sp, int n, int ns, uint64_t *keys, uint32_t *vals) {
  for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
    const int s = sp[v];
    keys[v] = ((uint64_t)(uint32_t)(s >= 0 ? s : ns) << 32) | (uint32_t)v;
    vals[v] = 0;
  }
}

__global__ void k_sub_lists(const uint64_t *keys, int n, int live, const int32_t *start, const int32_t *vwgt,
                            int32_t *vtx, int32_t *cvl, int2 *splo) {
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < n; p += gridDim.x * blockDim.x) {
    const int v = (int)(uint32_t)keys[p];
    if (p < live) {
      const int s = (int)(keys[p] >> 32);
      vtx[p] = v;
      cvl[p] = vwgt[v];
      splo[v] = make_int2(s, p - start[s]);
    } else {
      splo[v] = make_int2(-1, 0);
    }
  }
}

// deg'(v) (weight to nodes of the same subproblem) and the number of such
// neighbours, one warp per listed node
__global__ void k_sub_dp(const int32_t *xadj, const int32_t *adjncy, const int32_t *adjwgt, const int32_t *vtx,
                         const int2 *splo, int live, int32_t *dpl, int32_t *lcnt) {
  const int lane = (int)lane_id();
  const int wid = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int nw = (gridDim.x * blockDim.x) >> 5;
  for (int p = wid; p < live; p += nw) {
    const int v = vtx[p];
    const int s = splo[v].x;
    int sum = 0, c = 0;
    for (int e = xadj[v] + lane; e < xadj[v + 1]; e += 32)
      if (splo[adjncy[e]].x == s) { sum += adjwgt[e]; c++; }
    sum = warp_sum(sum);
    c = warp_sum(c);
    if (lane == 0) { dpl[p] = sum; lcnt[p] = c; }
  }
}

// local rows: (local index, weight) of the internal neighbours of every listed node
__global__ void k_sub_rows(const int32_t *xadj, const int32_t *adjncy, const int32_t *adjwgt, const int32_t *vtx,
                           const int2 *splo, int live, const int32_t *lxadj, int2 *ladj) {
  const int lane = (int)lane_id();
  const int wid = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int nw = (gridDim.x * blockDim.x) >> 5;
  for (int p = wid; p < live; p += nw) {
    const int v = vtx[p];
    const int s = splo[v].x;
    int pos = lxadj[p];
    for (int e0 = xadj[v]; e0 < xadj[v + 1]; e0 += 32) {
      const int e = e0 + lane;
      int2 sl = make_int2(-1, 0);
      if (e < xadj[v + 1]) sl = splo[adjncy[e]];
      const bool in = sl.x == s;
      const unsigned m = __ballot_sync(0xFFFFFFFFu, in);
      if (in) ladj[pos + __popc(m & lanemask_lt())] = make_int2(sl.y, adjwgt[e]);
      pos += __popc(m);
    }
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
__global__ void k_ip_assign(int n, int live, const int32_t *vtx, const int2 *splo, const int32_t *best,
                            const uint8_t *flags, const int32_t *child, int32_t *sp, int32_t *blocks) {
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < live; p += gridDim.x * blockDim.x) {
    const int v = vtx[p];
    const int s = splo[v].x;
    const int side1 = flags[(int64_t)best[s] * n + p];
    const int c = child[2 * s + (side1 ? 0 : 1)];
    if (c < 0) {
      blocks[v] = -(c + 1);
      sp[v] = -1;
    } else {
      sp[v] = c;
    }
  }
}

__global__ void k_max_weight(const int32_t *w, int n, int *out) {
  int m = 0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) m = w[i] > m ? w[i] : m;
  m = warp_max(m);
  if (lane_id() == 0 && m) atomicMax(out, m);
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
  DBuf<int32_t> sp(ctx, (size_t)n), vtx(ctx, (size_t)n), cvl(ctx, (size_t)n), dpl(ctx, (size_t)n),
      lxadj(ctx, (size_t)n + 1);
  DBuf<int2> ladj(ctx, (size_t)(g.m2 > 0 ? g.m2 : 1));
  DBuf<int> maxc(ctx, 1);
  DBuf<int2> splo(ctx, (size_t)n);
  DBuf<uint64_t> keys(ctx, (size_t)n);
  DBuf<uint32_t> vals(ctx, (size_t)n);
  sp.zero();  // everybody in subproblem 0
  const int64_t eps_l = eps_ppm / ceil_log2(k);
  std::vector<HostSub> subs{{k, 0, 1}};
  GP_CUDA(cudaFuncSetAttribute(k_ip_grow, cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxSmemBytes));
  maxc.zero();
  k_max_weight<<<grid, 256, 0, ctx->stream>>>(g.vwgt, n, maxc.get());
  GP_LAUNCH_CHECK();
  const int cvmax = read_scalar(ctx, maxc.get());
  DBuf<uint8_t> flags(ctx, (size_t)trials * n);
  while (!subs.empty()) {
    const int ns = (int)subs.size();
    DBuf<int32_t> cnt(ctx, (size_t)ns), start(ctx, (size_t)ns + 1);
    DBuf<long long> wsum(ctx, (size_t)ns);
    cnt.zero(); wsum.zero();
    k_sub_count<<<grid, 256, 0, ctx->stream>>>(sp.get(), g.vwgt, n, cnt.get(), wsum.get());
    GP_LAUNCH_CHECK();
    std::vector<int32_t> hc(ns);
    std::vector<long long> hw(ns);
    read_back(ctx, cnt.get(), sizeof(int32_t) * ns, hc.data());
    read_back(ctx, wsum.get(), sizeof(long long) * ns, hw.data());
    std::vector<int32_t> hs(ns + 1);
    hs[0] = 0;
    for (int i = 0; i < ns; i++) hs[i + 1] = hs[i] + hc[i];
    const int live = hs[ns];
    GP_CUDA(cudaMemcpyAsync(start.get(), hs.data(), sizeof(int32_t) * (ns + 1), cudaMemcpyHostToDevice,
                            ctx->stream));
    k_sub_keys<<<grid, 256, 0, ctx->stream>>>(sp.get(), n, ns, keys.get(), vals.get());
    GP_LAUNCH_CHECK();
    radix_sort_pairs(ctx, keys.get(), vals.get(), n, 32 + 1 + ceil_log2(ns + 1));
    k_sub_lists<<<grid, 256, 0, ctx->stream>>>(keys.get(), n, live, start.get(), g.vwgt, vtx.get(), cvl.get(),
                                                splo.get());
    GP_LAUNCH_CHECK();
    k_sub_dp<<<grid_for((int64_t)live * 32, 256, ctx->num_sms * 8), 256, 0, ctx->stream>>>(
        g.xadj, g.adjncy, g.adjwgt, vtx.get(), splo.get(), live, dpl.get(), lxadj.get());
    GP_LAUNCH_CHECK();
    GP_CUDA(cudaMemsetAsync(lxadj.get() + live, 0, sizeof(int32_t), ctx->stream));
    scan_exclusive_i32(ctx, lxadj.get(), lxadj.get(), live + 1, nullptr);
    k_sub_rows<<<grid_for((int64_t)live * 32, 256, ctx->num_sms * 8), 256, 0, ctx->stream>>>(
        g.xadj, g.adjncy, g.adjwgt, vtx.get(), splo.get(), live, lxadj.get(), ladj.get());
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
    IpArgs a{};
    a.lxadj = lxadj.get(); a.ladj = ladj.get();
    a.vtx = vtx.get(); a.cvl = cvl.get(); a.dpl = dpl.get();
    a.subs = dsub.get(); a.trials = trials; a.n = n; a.seed = seed;
    a.cv16 = cvmax <= 65535 ? 1 : 0;
    // shared-memory state: chunk maxima (8 B per 64 nodes) + gain (4 B) + weight (2 B, when it fits) +
    // state (1 B) per node, and the fallback hash (4 B) when that still holds every subproblem of
    // this depth
    int per_node = a.cv16 ? 7 : 5;
    auto cap_for = [&](int pn) { return (kMaxSmemBytes - 128) * kChunkNodes / (9 + pn * kChunkNodes); };
    a.hv_smem = maxcnt <= cap_for(per_node + 4) ? 1 : 0;
    if (a.hv_smem) per_node += 4;
    const int smem_cap = cap_for(per_node);
    a.smem_nodes = std::max(1, std::min(maxcnt, smem_cap));
    const int mch = (a.smem_nodes + kChunkNodes - 1) / kChunkNodes;
    const size_t smem_bytes = (size_t)(mch + (mch + 31) / 32) * 8 + (size_t)a.smem_nodes * per_node;
    DBuf<int32_t> gg;
    DBuf<uint8_t> gst;
    DBuf<uint16_t> gcv;
    DBuf<unsigned long long> gbest, gsup;
    if (maxcnt > a.smem_nodes) {
      a.gnodes = maxcnt;
      a.gchunks = (maxcnt + kChunkNodes - 1) / kChunkNodes;
      gg.reset(ctx, (size_t)nblocks * a.gnodes);
      gst.reset(ctx, (size_t)nblocks * a.gnodes);
      if (a.cv16) gcv.reset(ctx, (size_t)nblocks * a.gnodes);
      gbest.reset(ctx, (size_t)nblocks * a.gchunks);
      gsup.reset(ctx, (size_t)nblocks * ((a.gchunks + 31) / 32));
      a.gg = gg.get(); a.gst = gst.get(); a.gcv = gcv.get(); a.gbest = gbest.get(); a.gsup = gsup.get();
    }
    a.trial_cut = tcut.get();
    a.flags = flags.get();
    a.batch_cap = 1 + maxcnt / 1024;
    DBuf<int32_t> gbatch(ctx, (size_t)nblocks * a.batch_cap);
    a.gbatch = gbatch.get();
    const bool trace = getenv("GP_TRACE") != nullptr;
    DBuf<unsigned long long> tr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (trace) {
      tr.reset(ctx, 3);
      tr.zero();
      a.trace = tr.get();
      GP_CUDA(cudaEventCreate(&e0));
      GP_CUDA(cudaEventCreate(&e1));
      GP_CUDA(cudaEventRecord(e0, ctx->stream));
    }
    k_ip_grow<<<nblocks, 32 * kIpWarps, smem_bytes, ctx->stream>>>(a);
    GP_LAUNCH_CHECK();
    if (trace) {
      GP_CUDA(cudaEventRecord(e1, ctx->stream));
      unsigned long long h[3];
      read_back(ctx, tr.get(), sizeof(h), h);
      float ms = 0;
      GP_CUDA(cudaEventElapsedTime(&ms, e0, e1));
      fprintf(stderr, "[gp ip] subproblems=%d max_nodes=%d grow_ms=%.2f steps=%llu fallbacks=%llu retired=%llu\n",
              ns, maxcnt, ms, h[0], h[1], h[2]);
      cudaEventDestroy(e0);
      cudaEventDestroy(e1);
    }
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
    k_ip_assign<<<grid, 256, 0, ctx->stream>>>(n, live, vtx.get(), splo.get(), best.get(), flags.get(),
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
  ProfScope ps(ctx, PROF_REBALANCE);
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
