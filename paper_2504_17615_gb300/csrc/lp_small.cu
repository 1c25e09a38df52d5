// lp_small.cu -- size-constrained label propagation for small graphs as one
// cooperative persistent kernel.
//
// The schedule is lp.cu's (synchronous sub-rounds with hash priorities: the
// readings R3-R8 of the clustering of Sec. 3 / Sec. 4.1 and the refinement of
// Sec. 4.3); only the execution differs.  On a graph of a few hundred thousand
// nodes a sub-round is a few microseconds of work, and the launch-per-phase
// driver of lp.cu spends most of its time in launch gaps and in the host read
// of the counters after every sub-round.  Here the whole LP run is one launch:
// every block of a co-resident grid walks the same rounds and sub-rounds, the
// phases of a sub-round are separated by grid-wide barriers, and every block
// takes the same stop decisions from the same global counters.
//
// Per round, the nodes with neighbours are listed by (sub-round, degree
// class) in two passes (count, scatter).  Per sub-round:
//   rate    nodes of degree <= 8 are rated by 8-lane groups, <= 32 by a warp
//           with one entry per lane, <= 128 by a warp with four entries per
//           lane (equal labels summed in a small shared table, read back only
//           by the lane that claimed the label's slot), larger ones by a block
//   decide  a target whose snapshot weight plus all incoming weight fits the
//           bound accepts its proposers outright; the others are resolved in
//           (target, h32(PRIO), node) order, longest prefix (R7)
//   cap     clustering only, when the accepted moves could empty more than
//           D = c - n_min clusters: the (D+1)-th smallest emptying key is
//           selected by an MSD radix pass over all blocks (R8)
//   apply   labels and weights; the number of non-empty clusters follows from
//           the weight transitions (a cluster weight reaching zero or leaving
//           zero), every transition an atomic, so the count is exact
//
// Refinement skips nodes that cannot move: a node whose rating found no label
// rated above its own (admissible or not) proposes nothing until a neighbour
// changes its label, so it is not rated again until a move of a neighbour (or
// its own) marks it; the result is unchanged.
//
// Every grid barrier waits with an iteration limit; when it runs out the
// kernel records GP_ERR_TIMEOUT in a status word and every block returns.
#include "lp.cuh"
#include "lp_rate.cuh"

#include <algorithm>

namespace gp {

namespace {

constexpr unsigned FULL = 0xFFFFFFFFu;
constexpr int kPThreads = 256;
constexpr int kPWarps = kPThreads / 32;
constexpr int kPSlots = 256;        // per-warp rating table (nodes of degree <= kPLight)
constexpr int kPLight = 128;
constexpr int kPHeavySlots = 4096;  // per-block shared table (degree <= 2048); larger: global
constexpr int kPSortSmem = 2048;    // overflow sets sorted in shared memory up to this size
constexpr int kPBuckets = 4096;     // few-label overflow: priority buckets (top 12 bits)
constexpr int kPCross = 1024;       // few-label overflow: crossing-bucket entries kept in shared memory
constexpr int kPFewLabels = 256;    // labels up to this count: per-target overflow resolution
constexpr int kPAggLabels = 4096;   // labels up to this count: weight updates aggregated per block
constexpr int kPWeightSmem = 1024;  // refinement with labels up to this count: weights in shared memory
constexpr int kPKeys = 64 * 4;      // (sub-round, degree class) lists of a round
// resident blocks per SM of the persistent grid, and the pause between polls of a grid-wide wait
#ifndef GP_PLP_BLOCKS_PER_SM
#define GP_PLP_BLOCKS_PER_SM 3
#endif
#ifndef GP_PLP_POLL_NS
#define GP_PLP_POLL_NS 128
#endif

// Per sub-round counters (three sets in rotation, so a set can be cleared
// while the previous one is still being read).
struct PCount {
  int nprop, nheavy, nov, ecount;
  long long delta, moved;
  int touched;  // few-label overflow: at least one entry seen (unused otherwise)
  int pad;
};

struct PResult {
  int subrounds, capped;
  long long moves, proposals, ov_total, ov_max, nclusters;
};

struct PArgs {
  const int32_t *xadj, *adjncy, *adjwgt, *vwgt;
  int n;
  int32_t *label, *weight;
  uint8_t *label8;
  uint8_t *dirty;        // refinement: per node, 0 = cannot move until a neighbour moves (may be null)
  int64_t nlabels;
  int64_t bound, n_min;
  int count_clusters, rounds, S, dbg_max, level;
  uint64_t seed;
  uint32_t tag_act, tag_tie, tag_prio;
  int64_t ncl0;
  // scratch
  int4 *prop;            // [n] (node, target, own label, weight)
  int32_t *incoming;     // [nlabels], zero between sub-rounds
  uint8_t *acc;          // [n] per proposal: accepted
  int32_t *blist;        // [n] the round's nodes by (sub-round, degree class)
  int32_t *bcnt, *bfill; // [2][kPKeys] list sizes and fill cursors (by round parity)
  int32_t *boffs;        // [2][kPKeys + 1] list offsets
  uint64_t *ovk;         // [cap2] (target << 32 | priority)
  uint32_t *ovv;         // [cap2] node
  int32_t *ovi;          // [cap2] proposal index
  long long *ovps;       // [cap2] running weights (global sort path)
  int64_t cap2;
  int32_t *depw;         // [nlabels] clustering: weight leaving a cluster, zero between sub-rounds
  unsigned long long *dkey;  // [nlabels] clustering: latest departure key, zero between sub-rounds
  uint64_t *ekeys;       // [n] emptying keys
  unsigned *chist;       // [8][256] cap select histograms
  int32_t *gtk, *gtv;    // per-block global tables for heavy nodes beyond kPHeavySlots
  int64_t gstride;
  int hblocks;           // the first hblocks blocks rate the heavy nodes (one table each)
  PCount *cnt;           // [3]
  unsigned *bar;         // [0] arrivals, [1] generation
  int *status;
  long long spin_cap;
  PResult *out;
  unsigned long long *units;
};

// ------------------------------------------------------------- barrier
//
// Arrival is an acquire-release add on the arrival count; the last block to
// arrive resets it and publishes the next generation with a release add;
// waiting blocks poll the generation with acquire loads.  The barrier's
// thread 0 thereby synchronises with every block's writes before the
// barrier, and the block's __syncthreads extends that to all its threads,
// so plain loads after the barrier see every write made before it.

__device__ __forceinline__ unsigned ld_acquire(const unsigned *p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ unsigned atom_add_acq_rel(unsigned *p, unsigned x) {
  unsigned old;
  asm volatile("atom.add.acq_rel.gpu.global.u32 %0, [%1], %2;" : "=r"(old) : "l"(p), "r"(x) : "memory");
  return old;
}

__device__ __forceinline__ void red_add_release(unsigned *p, unsigned x) {
  asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(p), "r"(x) : "memory");
}

__device__ bool grid_sync(const PArgs &a) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    int ok = 1;
    volatile int *status = a.status;
    const unsigned g0 = ld_acquire(a.bar + 1);
    if (atom_add_acq_rel(a.bar, 1u) == gridDim.x - 1) {
      a.bar[0] = 0;  // ordered before the release below
      red_add_release(a.bar + 1, 1u);
    } else {
      long long spins = 0;
      while (ld_acquire(a.bar + 1) == g0) {
        if (*status != 0) { ok = 0; break; }
        if (++spins > a.spin_cap) {
          atomicCAS(a.status, 0, (int)GP_ERR_TIMEOUT);
          ok = 0;
          break;
        }
        if (GP_PLP_POLL_NS > 0) __nanosleep(GP_PLP_POLL_NS);
      }
    }
    s_ok = ok && *status == 0;
  }
  __syncthreads();
  return s_ok != 0;
}

__device__ __forceinline__ int plabel(const PArgs &a, int u) { return a.label8 ? (int)a.label8[u] : a.label[u]; }

__device__ __forceinline__ uint64_t pkey(uint64_t kprio, int v) {
  return ((uint64_t)h32(kprio, (uint32_t)v, 0) << 32) | (uint32_t)v;
}

// Appends one proposal (lane 0 of the rating warp / thread 0 of the rating block).
__device__ __forceinline__ void propose(const PArgs &a, PCount *c, int v, int K, int own, int cv) {
  const int i = atomicAdd(&c->nprop, 1);
  a.prop[i] = make_int4(v, K, own, cv);
  atomicAdd(&a.incoming[K], cv);
}

// Best candidate over a rating table (keys tk, sums tv, `size` slots) walked by
// `lane` with stride `step`: own rating, then the admissible label of largest
// rating, ties by the smallest h32(ktie, v, L), then the smallest label.
// Returns the packed (hash << 32 | label) of the best candidate, ~0 if none,
// via the reductions red_max / red_min; stable: no label other than own rated
// above own (computed only when the skip flags are kept).
template <typename RMAX, typename RMIN>
__device__ __forceinline__ uint64_t choose(const PArgs &a, const int *tk, const int *tv, int size, int tid,
                                           int step, int v, int own, int cv, uint64_t ktie, RMAX red_max,
                                           RMIN red_min, int &own_r_out, int &rmax_out, bool &stable) {
  int own_loc = 0, rloc = -1, rall = 0;
  for (int t = tid; t < size; t += step) {
    const int L = tk[t];
    if (L < 0) continue;
    const int r = tv[t];
    if (L == own) { own_loc = r; continue; }
    rall = r > rall ? r : rall;
    if ((int64_t)a.weight[L] + cv > a.bound) continue;
    rloc = r > rloc ? r : rloc;
  }
  const int own_r = red_max(own_loc);
  const int rmax = red_max(rloc);
  stable = a.dirty != nullptr && red_max(rall) <= own_r;
  own_r_out = own_r;
  rmax_out = rmax;
  if (rmax < 0 || rmax <= own_r) return ~0ull;
  uint64_t packed = ~0ull;
  for (int t = tid; t < size; t += step) {
    const int L = tk[t];
    if (L < 0 || L == own || tv[t] != rmax) continue;
    if ((int64_t)a.weight[L] + cv > a.bound) continue;
    const uint64_t p = ((uint64_t)h32(ktie, (uint32_t)v, (uint32_t)L) << 32) | (uint32_t)L;
    packed = p < packed ? p : packed;
  }
  return red_min(packed);
}

// ------------------------------------------------------- block helpers

__device__ __forceinline__ int block_max_int(int v, int *s_red) {
  v = warp_max(v);
  const int w = threadIdx.x >> 5;
  __syncthreads();
  if (lane_id() == 0) s_red[w] = v;
  __syncthreads();
  int r = s_red[0];
  for (int i = 1; i < kPWarps; i++) r = s_red[i] > r ? s_red[i] : r;
  return r;
}

__device__ __forceinline__ uint64_t block_min_u64(uint64_t v, uint64_t *s_red) {
  v = warp_min(v);
  const int w = threadIdx.x >> 5;
  __syncthreads();
  if (lane_id() == 0) s_red[w] = v;
  __syncthreads();
  uint64_t r = s_red[0];
  for (int i = 1; i < kPWarps; i++) r = s_red[i] < r ? s_red[i] : r;
  return r;
}

// Inclusive block scan of 64-bit values (256 threads).
__device__ __forceinline__ long long block_incl_scan(long long x, long long *s_w, long long &total) {
  const int lane = (int)lane_id(), w = threadIdx.x >> 5;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const long long y = __shfl_up_sync(FULL, x, o);
    if (lane >= o) x += y;
  }
  __syncthreads();
  if (lane == 31) s_w[w] = x;
  __syncthreads();
  long long before = 0;
  total = 0;
  for (int q = 0; q < kPWarps; q++) {
    if (q < w) before += s_w[q];
    total += s_w[q];
  }
  return before + x;
}

// Bitonic sort by (key, val) of P (a power of two) entries held in k / v / ix
// (shared or global memory), by one block.
__device__ void bitonic(uint64_t *k, uint32_t *v, int32_t *ix, int P) {
  for (int size = 2; size <= P; size <<= 1) {
    for (int stride = size >> 1; stride > 0; stride >>= 1) {
      for (int i = threadIdx.x; i < P / 2; i += blockDim.x) {
        const int lo = 2 * i - (i & (stride - 1));
        const int hi = lo + stride;
        const bool up = (lo & size) == 0;
        const uint64_t ka = k[lo], kb = k[hi];
        const uint32_t va = v[lo], vb = v[hi];
        const bool gt = ka > kb || (ka == kb && va > vb);
        if (gt == up) {
          k[lo] = kb; k[hi] = ka;
          v[lo] = vb; v[hi] = va;
          const int32_t t = ix[lo]; ix[lo] = ix[hi]; ix[hi] = t;
        }
      }
      __syncthreads();
    }
  }
}

// Rates the nodes list[0 .. count), one node per G-lane group with up to E
// entries per lane (rate_group of lp_rate.cuh), and proposes the moves.
template <int G, int E>
__device__ __forceinline__ void rate_list(const PArgs &a, PCount *c, const int32_t *list, int count, int gw,
                                          int nw, int *tk, int *tv, uint64_t ktie, const int *s_wl,
                                          unsigned long long &ue, unsigned long long &uv) {
  constexpr int NV = 32 / G;
  constexpr int TS = GroupTable<G, E>::TS;
  static_assert(NV * TS <= kPSlots, "table size");
  const int lane = (int)lane_id(), grp = lane / G, gl = lane % G;
  const unsigned gmask = G == 32 ? FULL : (((1u << G) - 1u) << (grp * G));
  for (int i0 = gw * NV; i0 < count; i0 += nw * NV) {
    const int i = i0 + grp;
    int v = i < count ? list[i] : -1;
    if (v >= 0 && a.dirty && !a.dirty[v]) v = -1;  // cannot move until a neighbour moves
    int st = 0, deg = 0, own = -2, cv = 0;
    if (v >= 0) {
      st = a.xadj[v];
      deg = a.xadj[v + 1] - st;
      own = plabel(a, v);
      cv = a.vwgt[v];
    }
    int nc = 0;
    bool stable = false;
    const unsigned best = rate_group<G, E, false>(a.adjncy, a.adjwgt, a.label, a.label8, a.weight, s_wl, a.bound,
                                                  ktie, v, st, deg, own, cv, tk + grp * TS, tv + grp * TS, gmask,
                                                  gl, false, nc, stable);
    if (gl == 0 && v >= 0) {
      ue += deg;
      uv += 1;
      if (best != 0xFFFFFFFFu) propose(a, c, v, (int)best, own, cv);
      if (a.dirty && stable) a.dirty[v] = 0;
    }
  }
}

// degree classes of the per-round lists: <= 8 (8 lanes per node), <= 32 (a
// warp, one entry per lane), <= 128 (a warp, four entries per lane), larger
// (a block)
__device__ __forceinline__ int deg_class(int deg) { return deg <= 8 ? 0 : deg <= 32 ? 1 : deg <= kPLight ? 2 : 3; }

// ---------------------------------------------------------- the kernel

__global__ void __launch_bounds__(kPThreads) k_lp_persistent(PArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  // per-warp rating tables, then a phase-shared area
  int *wtk = reinterpret_cast<int *>(smem);                 // [kPWarps][kPSlots]
  int *wtv = wtk + kPWarps * kPSlots;                        // [kPWarps][kPSlots]
  unsigned char *area = reinterpret_cast<unsigned char *>(wtv + kPWarps * kPSlots);
  __shared__ int s_ri[kPWarps];
  __shared__ uint64_t s_ru[kPWarps];
  __shared__ long long s_ll[kPWarps];
  __shared__ unsigned s_h[256];
  __shared__ int s_bc[kPKeys], s_bb[kPKeys], s_bo[kPKeys + 1];
  __shared__ int s_wl[kPWeightSmem];

  const int lane = (int)lane_id(), wib = threadIdx.x >> 5;
  const int gw = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5);
  const int nw = (int)((gridDim.x * blockDim.x) >> 5);
  const int gt = (int)(blockIdx.x * blockDim.x + threadIdx.x);
  const int gthreads = (int)(gridDim.x * blockDim.x);
  int *tk = wtk + wib * kPSlots, *tv = wtv + wib * kPSlots;
  for (int t = lane; t < kPSlots; t += 32) { tk[t] = -1; tv[t] = 0; }
  __syncwarp();

  const int n = a.n;
  long long ncl = a.ncl0;
  long long moves_total = 0, props_total = 0, ov_total = 0, ov_max = 0;
  int subs = 0, capped = 0;
  bool stop = false;
  unsigned long long ue = 0, uv = 0;
  const bool few = a.nlabels <= kPFewLabels;
  const bool agg = !a.count_clusters && a.nlabels <= kPAggLabels;
  const bool few_w = !a.count_clusters && a.nlabels <= kPWeightSmem;  // label weights in shared memory

  for (int r = 0; r < a.rounds && !stop; r++) {
    const uint64_t kact = stream_key(a.seed, a.tag_act, (uint32_t)a.level, (uint32_t)r);
    const uint64_t ktie = stream_key(a.seed, a.tag_tie, (uint32_t)a.level, (uint32_t)r);
    const uint64_t kprio = stream_key(a.seed, a.tag_prio, (uint32_t)a.level, (uint32_t)r);
    long long moved_round = 0;
    if (a.count_clusters && ncl <= a.n_min) break;
    if (a.dbg_max >= 0 && subs >= a.dbg_max) break;
    // the round's lists: nodes with neighbours by (sub-round, degree class), in two passes
    {
      const int nkeys = a.S * 4;
      int32_t *cnt = a.bcnt + (r & 1) * kPKeys;
      int32_t *fill = a.bfill + (r & 1) * kPKeys;
      int32_t *offs = a.boffs + (r & 1) * (kPKeys + 1);
      if (blockIdx.x == 0) {  // the other parity's counters, for the next round
        for (int t = threadIdx.x; t < kPKeys; t += blockDim.x) {
          a.bcnt[((r + 1) & 1) * kPKeys + t] = 0;
          a.bfill[((r + 1) & 1) * kPKeys + t] = 0;
        }
      }
      for (int t = threadIdx.x; t < nkeys; t += blockDim.x) s_bc[t] = 0;
      __syncthreads();
      for (int v = gt; v < n; v += gthreads) {
        const int deg = a.xadj[v + 1] - a.xadj[v];
        if (deg == 0) continue;
        const int sr = (int)(h32(kact, (uint32_t)v, 0) % (uint32_t)a.S);
        atomicAdd(&s_bc[sr * 4 + deg_class(deg)], 1);
      }
      __syncthreads();
      for (int t = threadIdx.x; t < nkeys; t += blockDim.x)
        if (s_bc[t]) atomicAdd(&cnt[t], s_bc[t]);
      if (!grid_sync(a)) return;
      // offsets (every block computes the same prefix), then the scatter in chunks
      if (threadIdx.x == 0) {
        int run = 0;
        for (int t = 0; t < nkeys; t++) { s_bo[t] = run; run += cnt[t]; }
        s_bo[nkeys] = run;
      }
      __syncthreads();
      if (blockIdx.x == 0)
        for (int t = threadIdx.x; t <= nkeys; t += blockDim.x) offs[t] = s_bo[t];
      for (int c0 = blockIdx.x * kPThreads * 4; c0 < n; c0 += gridDim.x * kPThreads * 4) {
        for (int t = threadIdx.x; t < nkeys; t += blockDim.x) s_bc[t] = 0;
        __syncthreads();
        int key[4];
#pragma unroll
        for (int q = 0; q < 4; q++) {
          const int v = c0 + q * kPThreads + (int)threadIdx.x;
          key[q] = -1;
          if (v < n) {
            const int deg = a.xadj[v + 1] - a.xadj[v];
            if (deg > 0) key[q] = (int)(h32(kact, (uint32_t)v, 0) % (uint32_t)a.S) * 4 + deg_class(deg);
          }
          if (key[q] >= 0) atomicAdd(&s_bc[key[q]], 1);
        }
        __syncthreads();
        for (int t = threadIdx.x; t < nkeys; t += blockDim.x) {
          s_bb[t] = s_bc[t] ? s_bo[t] + atomicAdd(&fill[t], s_bc[t]) : 0;
          s_bc[t] = 0;
        }
        __syncthreads();
#pragma unroll
        for (int q = 0; q < 4; q++) {
          if (key[q] < 0) continue;
          const int v = c0 + q * kPThreads + (int)threadIdx.x;
          a.blist[s_bb[key[q]] + atomicAdd(&s_bc[key[q]], 1)] = v;
        }
        __syncthreads();
      }
      if (!grid_sync(a)) return;
    }
    for (int s = 0; s < a.S; s++) {
      if (a.count_clusters && ncl <= a.n_min) { stop = true; break; }
      if (a.dbg_max >= 0 && subs >= a.dbg_max) { stop = true; break; }
      PCount *c = a.cnt + (subs % 3);
      if (blockIdx.x == 0 && threadIdx.x == 0) {
        PCount *nx = a.cnt + ((subs + 1) % 3);
        nx->nprop = 0; nx->nheavy = 0; nx->nov = 0; nx->ecount = 0;
        nx->delta = 0; nx->moved = 0; nx->touched = 0;
      }
      // ---------------------------------------------------------- rate
      const int32_t *lo = a.boffs + (r & 1) * (kPKeys + 1) + s * 4;  // this sub-round's four lists
      if (few_w) {
        for (int t = threadIdx.x; t < (int)a.nlabels; t += blockDim.x) s_wl[t] = a.weight[t];
        __syncthreads();
      }
      // nodes of degree > kPLight: a block each, tables in shared memory (or global beyond)
      {
        int *htk = reinterpret_cast<int *>(area);
        int *htv = htk + kPHeavySlots;
        const int h0 = lo[3], h1 = lo[4];
        if (h1 > h0) {
          for (int t = threadIdx.x; t < kPHeavySlots; t += blockDim.x) { htk[t] = -1; htv[t] = 0; }
          __syncthreads();
        }
        for (int h = h0 + blockIdx.x; h < h1 && (int)blockIdx.x < a.hblocks; h += a.hblocks) {
          const int v = a.blist[h];
          // read by every thread before thread 0 may clear it below (barriers in between)
          if (a.dirty && !a.dirty[v]) continue;
          const int st = a.xadj[v], deg = a.xadj[v + 1] - st;
          int bits = 1;
          while ((1 << bits) < 2 * deg) bits++;
          const int tsize = 1 << bits;
          const bool sm = tsize <= kPHeavySlots;
          int *k2 = sm ? htk : a.gtk + (int64_t)blockIdx.x * a.gstride;
          int *v2 = sm ? htv : a.gtv + (int64_t)blockIdx.x * a.gstride;
          const int own = plabel(a, v), cv = a.vwgt[v];
          for (int j = threadIdx.x; j < deg; j += blockDim.x) {
            const int L = plabel(a, a.adjncy[st + j]);
            const int w = a.adjwgt[st + j];
            unsigned sl = ((unsigned)L * 2654435761u) >> (32 - bits);
            for (int probe = 0; probe < tsize; probe++) {  // bounded: the table never fills
              const int prev = atomicCAS(&k2[sl], -1, L);
              if (prev == -1 || prev == L) { atomicAdd(&v2[sl], w); break; }
              sl = (sl + 1) & (unsigned)(tsize - 1);
            }
          }
          __syncthreads();
          int own_r, rmax;
          bool stable;
          const uint64_t best = choose(a, k2, v2, tsize, threadIdx.x, blockDim.x, v, own, cv, ktie,
                                       [&](int x) { return block_max_int(x, s_ri); },
                                       [&](uint64_t x) { return block_min_u64(x, s_ru); }, own_r, rmax, stable);
          if (threadIdx.x == 0) {
            ue += deg;
            uv += 1;
            if (best != ~0ull) propose(a, c, v, (int)(uint32_t)best, own, cv);
            if (stable) a.dirty[v] = 0;
          }
          __syncthreads();
          for (int t = threadIdx.x; t < tsize; t += blockDim.x) { k2[t] = -1; v2[t] = 0; }
          __syncthreads();
        }
      }
      {
        const int *wl = few_w ? s_wl : nullptr;
        rate_list<32, 4>(a, c, a.blist + lo[2], lo[3] - lo[2], gw, nw, tk, tv, ktie, wl, ue, uv);
        rate_list<32, 1>(a, c, a.blist + lo[1], lo[2] - lo[1], gw, nw, tk, tv, ktie, wl, ue, uv);
        rate_list<8, 1>(a, c, a.blist + lo[0], lo[1] - lo[0], gw, nw, tk, tv, ktie, wl, ue, uv);
      }
      if (!grid_sync(a)) return;
      // -------------------------------------------------------- decide
      const int nprop = *(volatile int *)&c->nprop;
      for (int b0 = blockIdx.x * blockDim.x; b0 < nprop; b0 += gthreads) {
        const int i = b0 + (int)threadIdx.x;
        bool over = false;
        int4 p = make_int4(0, 0, 0, 0);
        if (i < nprop) {
          p = a.prop[i];
          const bool fit = (int64_t)a.weight[p.y] + a.incoming[p.y] <= a.bound;
          a.acc[i] = fit ? 1 : 0;
          over = !fit;
        }
        const int j = warp_append(&c->nov, over);
        if (over) {
          a.ovk[j] = ((uint64_t)(uint32_t)p.y << 32) | h32(kprio, (uint32_t)p.x, 0);
          a.ovv[j] = (uint32_t)p.x;
          a.ovi[j] = i;
        }
      }
      if (!grid_sync(a)) return;
      // ------------------------------------------------------ overflow
      const int nov = *(volatile int *)&c->nov;
      if (nov > 0) {
        if (few) {
          // per target: weighted histogram over the top 12 priority bits finds the
          // bucket where the running weight passes the room; only that bucket's
          // entries are ranked exactly
          long long *hist = reinterpret_cast<long long *>(area);                    // [kPBuckets]
          uint64_t *xk = reinterpret_cast<uint64_t *>(hist + kPBuckets);            // [kPCross]
          int *xc = reinterpret_cast<int *>(xk + kPCross);                           // [kPCross]
          int *xi = xc + kPCross;                                                    // [kPCross]
          __shared__ int s_any, s_cross, s_nx;
          __shared__ long long s_base;
          for (int t = blockIdx.x; t < (int)a.nlabels; t += gridDim.x) {
            for (int q = threadIdx.x; q < kPBuckets; q += blockDim.x) hist[q] = 0;
            if (threadIdx.x == 0) { s_any = 0; s_nx = 0; }
            __syncthreads();
            for (int j = threadIdx.x; j < nov; j += blockDim.x) {
              const uint64_t k = a.ovk[j];
              if ((int)(k >> 32) != t) continue;
              atomicAdd((unsigned long long *)&hist[(uint32_t)k >> 20], (unsigned long long)a.vwgt[a.ovv[j]]);
              s_any = 1;
            }
            __syncthreads();
            if (!s_any) continue;
            const long long room = a.bound - (long long)a.weight[t];
            // crossing bucket: 16 buckets per thread
            long long loc = 0;
            const int b0 = threadIdx.x * (kPBuckets / kPThreads);
            for (int q = 0; q < kPBuckets / kPThreads; q++) loc += hist[b0 + q];
            long long tot;
            const long long incl = block_incl_scan(loc, s_ll, tot);
            if (threadIdx.x == 0) { s_cross = kPBuckets; s_base = 0; }
            __syncthreads();
            long long run = incl - loc;
            for (int q = 0; q < kPBuckets / kPThreads; q++) {
              const long long x = hist[b0 + q];
              if (x > 0 && run + x > room) {
                atomicMin(&s_cross, b0 + q);
                break;
              }
              run += x;
            }
            __syncthreads();
            {
              // base = weight of the buckets before the crossing one
              long long mine = 0;
              for (int q = 0; q < kPBuckets / kPThreads; q++)
                if (b0 + q < s_cross) mine += hist[b0 + q];
              long long t2;
              block_incl_scan(mine, s_ll, t2);
              if (threadIdx.x == 0) s_base = t2;
            }
            __syncthreads();
            const int cross = s_cross;
            for (int j = threadIdx.x; j < nov; j += blockDim.x) {
              const uint64_t k = a.ovk[j];
              if ((int)(k >> 32) != t) continue;
              const int bk = (int)((uint32_t)k >> 20);
              if (bk != cross) {
                a.acc[a.ovi[j]] = bk < cross ? 1 : 0;
                continue;
              }
              const int x = atomicAdd(&s_nx, 1);
              if (x < kPCross) {
                xk[x] = ((uint64_t)(uint32_t)k << 32) | a.ovv[j];
                xc[x] = a.vwgt[a.ovv[j]];
                xi[x] = a.ovi[j];
              }
            }
            __syncthreads();
            const int nx = s_nx;
            if (nx <= kPCross) {
              for (int x = threadIdx.x; x < nx; x += blockDim.x) {
                long long w = s_base;
                for (int y = 0; y < nx; y++)
                  if (xk[y] <= xk[x]) w += xc[y];
                a.acc[xi[x]] = w <= room ? 1 : 0;
              }
            } else {
              // more crossing entries than fit in shared memory: rank each against all entries
              for (int j = threadIdx.x; j < nov; j += blockDim.x) {
                const uint64_t k = a.ovk[j];
                if ((int)(k >> 32) != t || (int)((uint32_t)k >> 20) != cross) continue;
                const uint64_t me = ((uint64_t)(uint32_t)k << 32) | a.ovv[j];
                long long w = s_base;
                for (int y = 0; y < nov; y++) {
                  const uint64_t ky = a.ovk[y];
                  if ((int)(ky >> 32) != t || (int)((uint32_t)ky >> 20) != cross) continue;
                  const uint64_t other = ((uint64_t)(uint32_t)ky << 32) | a.ovv[y];
                  if (other <= me) w += a.vwgt[a.ovv[y]];
                }
                a.acc[a.ovi[j]] = w <= room ? 1 : 0;
              }
            }
            __syncthreads();
          }
        } else if (blockIdx.x == 0) {
          // one block orders the overflow set by (target, priority, node) and accepts the
          // longest fitting prefix per target
          int P = 1;
          while (P < nov) P <<= 1;
          uint64_t *k;
          uint32_t *vv;
          int32_t *ix;
          long long *ps;
          if (P <= kPSortSmem) {
            k = reinterpret_cast<uint64_t *>(area);
            vv = reinterpret_cast<uint32_t *>(k + kPSortSmem);
            ix = reinterpret_cast<int32_t *>(vv + kPSortSmem);
            ps = reinterpret_cast<long long *>(ix + kPSortSmem);
            for (int i = threadIdx.x; i < P; i += blockDim.x) {
              k[i] = i < nov ? a.ovk[i] : ~0ull;
              vv[i] = i < nov ? a.ovv[i] : 0xFFFFFFFFu;
              ix[i] = i < nov ? a.ovi[i] : -1;
            }
          } else {
            k = a.ovk; vv = a.ovv; ix = a.ovi; ps = a.ovps;
            for (int i = nov + threadIdx.x; i < P; i += blockDim.x) { k[i] = ~0ull; vv[i] = 0xFFFFFFFFu; ix[i] = -1; }
          }
          __syncthreads();
          bitonic(k, vv, ix, P);
          long long carry = 0;
          for (int c0 = 0; c0 < nov; c0 += blockDim.x) {
            const int i = c0 + threadIdx.x;
            const long long x = i < nov ? (long long)a.vwgt[vv[i]] : 0;
            long long tot;
            const long long incl = block_incl_scan(x, s_ll, tot);
            if (i < nov) ps[i] = carry + incl;
            carry += tot;
          }
          __syncthreads();
          for (int i = threadIdx.x; i < nov; i += blockDim.x) {
            const uint64_t seg = k[i] & 0xFFFFFFFF00000000ull;
            int lo = 0, hi = i;
            while (lo < hi) {
              const int mid = (lo + hi) >> 1;
              if (k[mid] < seg) lo = mid + 1; else hi = mid;
            }
            const long long w = ps[i] - (lo > 0 ? ps[lo - 1] : 0);
            const int K = (int)(k[i] >> 32);
            a.acc[ix[i]] = (int64_t)a.weight[K] + w <= a.bound ? 1 : 0;
          }
        }
        if (!grid_sync(a)) return;
      }
      // ----------------------------------------------------------- cap
      unsigned long long cutoff = ~0ull;
      if (a.count_clusters && (long long)nprop > ncl - a.n_min) {
        const long long D = ncl - a.n_min;
        for (int i = gt; i < nprop; i += gthreads) {
          if (!a.acc[i]) continue;
          const int4 p = a.prop[i];
          atomicAdd(&a.depw[p.z], p.w);
          atomicMax(&a.dkey[p.z], (unsigned long long)pkey(kprio, p.x));
        }
        if (blockIdx.x == 0)
          for (int q = threadIdx.x; q < 8 * 256; q += blockDim.x) a.chist[q] = 0;
        if (!grid_sync(a)) return;
        for (int b0 = blockIdx.x * blockDim.x; b0 < nprop; b0 += gthreads) {
          const int i = b0 + (int)threadIdx.x;
          bool emit_key = false;
          uint64_t key = 0;
          if (i < nprop && a.acc[i]) {
            const int4 p = a.prop[i];
            key = pkey(kprio, p.x);
            emit_key = a.depw[p.z] == a.weight[p.z] && key == a.dkey[p.z];
          }
          const int pos = warp_append(&c->ecount, emit_key);
          if (emit_key) a.ekeys[pos] = key;
        }
        if (!grid_sync(a)) return;
        const int E = *(volatile int *)&c->ecount;
        // the per-cluster departure state is cleared for the next sub-round
        for (int i = gt; i < nprop; i += gthreads) {
          if (!a.acc[i]) continue;
          const int own = a.prop[i].z;
          a.depw[own] = 0;
          a.dkey[own] = 0;
        }
        if (E > D) {
          // MSD radix select of the (D+1)-th smallest emptying key, 8 bits per pass
          uint64_t prefix = 0, mask = 0;
          long long rank = D;
          for (int pass = 0; pass < 8; pass++) {
            const int shift = 56 - 8 * pass;
            for (int q = threadIdx.x; q < 256; q += blockDim.x) s_h[q] = 0;
            __syncthreads();
            for (int i = gt; i < E; i += gthreads) {
              const uint64_t key = a.ekeys[i];
              if ((key & mask) == prefix) atomicAdd(&s_h[(key >> shift) & 255u], 1u);
            }
            __syncthreads();
            for (int q = threadIdx.x; q < 256; q += blockDim.x)
              if (s_h[q]) atomicAdd(&a.chist[pass * 256 + q], s_h[q]);
            if (!grid_sync(a)) return;
            const volatile unsigned *hh = a.chist + pass * 256;
            int d = 0;
            for (; d < 255; d++) {
              const long long x = hh[d];
              if (rank < x) break;
              rank -= x;
            }
            prefix |= (uint64_t)d << shift;
            mask |= (uint64_t)255 << shift;
          }
          cutoff = prefix;
          capped++;
        }
      }
      // --------------------------------------------------------- apply
      int *s_dw = reinterpret_cast<int *>(area);
      if (agg) {
        for (int q = threadIdx.x; q < (int)a.nlabels; q += blockDim.x) s_dw[q] = 0;
        __syncthreads();
      }
      long long moved = 0, delta = 0;
      for (int i = gt; i < nprop; i += gthreads) {
        const int4 p = a.prop[i];
        a.incoming[p.y] = 0;
        if (!a.acc[i]) continue;
        if (cutoff != ~0ull && pkey(kprio, p.x) >= cutoff) continue;
        a.label[p.x] = p.y;
        if (a.label8) a.label8[p.x] = (uint8_t)p.y;
        if (agg) {
          atomicAdd(&s_dw[p.y], p.w);
          atomicSub(&s_dw[p.z], p.w);
        } else {
          const int oldK = atomicAdd(&a.weight[p.y], p.w);
          const int oldO = atomicSub(&a.weight[p.z], p.w);
          delta += (oldK == 0) - (oldO == p.w);
        }
        moved++;
      }
      if (agg) {
        __syncthreads();
        for (int q = threadIdx.x; q < (int)a.nlabels; q += blockDim.x)
          if (s_dw[q]) atomicAdd(&a.weight[q], s_dw[q]);
      }
      if (a.dirty) {  // every applied move marks its node and the node's neighbours, a warp per move
        for (int i = gw; i < nprop; i += nw) {
          if (!a.acc[i]) continue;
          const int v = a.prop[i].x;
          if (cutoff != ~0ull && pkey(kprio, v) >= cutoff) continue;
          const int e0 = a.xadj[v], e1 = a.xadj[v + 1];
          if (lane == 0) a.dirty[v] = 1;
          for (int e = e0 + lane; e < e1; e += 32) a.dirty[a.adjncy[e]] = 1;
        }
      }
      moved = warp_sum(moved);
      delta = warp_sum(delta);
      if (lane == 0) {
        if (moved) atomicAdd((unsigned long long *)&c->moved, (unsigned long long)moved);
        if (delta) atomicAdd((unsigned long long *)&c->delta, (unsigned long long)delta);
      }
      if (!grid_sync(a)) return;
      const long long mv = *(volatile long long *)&c->moved;
      ncl += *(volatile long long *)&c->delta;
      moved_round += mv;
      moves_total += mv;
      props_total += nprop;
      ov_total += nov;
      ov_max = nov > ov_max ? nov : ov_max;
      subs++;
    }
    if (moved_round == 0) stop = true;
  }
  if (a.units) {
    ue = warp_sum(ue);
    uv = warp_sum(uv);
    if (lane == 0) {
      if (ue) atomicAdd(a.units + 0, ue);
      if (ue && a.label8) atomicAdd(a.units + 4, ue);
      if (uv) atomicAdd(a.units + 1, uv);
    }
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    a.out->subrounds = subs;
    a.out->capped = capped;
    a.out->moves = moves_total;
    a.out->proposals = props_total;
    a.out->ov_total = ov_total;
    a.out->ov_max = ov_max;
    a.out->nclusters = ncl;
  }
}

constexpr size_t kAreaBytes() {
  // the largest phase use of the shared area
  size_t heavy = sizeof(int) * 2 * kPHeavySlots;
  size_t sort = (sizeof(uint64_t) + sizeof(uint32_t) + sizeof(int32_t) + sizeof(long long)) * kPSortSmem;
  size_t fewb = sizeof(long long) * kPBuckets + (sizeof(uint64_t) + 2 * sizeof(int)) * kPCross;
  size_t aggb = sizeof(int) * kPAggLabels;
  size_t m = heavy;
  m = sort > m ? sort : m;
  m = fewb > m ? fewb : m;
  m = aggb > m ? aggb : m;
  return m;
}

constexpr size_t kSmemBytes = sizeof(int) * 2 * kPWarps * kPSlots + kAreaBytes();

__global__ void k_pmax_degree(const int32_t *xadj, int n, int *out) {
  int m = 0;
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
    const int d = xadj[v + 1] - xadj[v];
    m = d > m ? d : m;
  }
  m = warp_max(m);
  if (lane_id() == 0 && m) atomicMax(out, m);
}

}  // namespace

bool lp_small_applicable(const DevGraph &g, const LpParams &p) {
  return g.n > 0 && g.n <= p.small_nodes && g.m2 <= kLpSmallMaxEntries;
}

LpResult lp_run_small(gp_ctx *ctx, const DevGraph &g, int32_t *label, int32_t *weight, int64_t nlabels,
                      uint64_t seed, const LpParams &p, int64_t *nclusters_dev, uint8_t *label8) {
  LpResult res;
  const int n = g.n;
  GP_REQUIRE(p.subrounds >= 1 && p.subrounds <= 64, GP_ERR_INVALID, "lp_subrounds must be in [1, 64]");
  static bool attr_set[64] = {};
  if (ctx->device >= 0 && ctx->device < 64 && !attr_set[ctx->device]) {
    GP_CUDA(cudaFuncSetAttribute(k_lp_persistent, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemBytes));
    attr_set[ctx->device] = true;
  }
  int per_sm = 0;
  GP_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_lp_persistent, kPThreads, kSmemBytes));
  GP_REQUIRE(per_sm >= 1, GP_ERR_CUDA, "persistent LP kernel does not fit on an SM");
  // about one thread per node, at most the resident blocks of the device, divided among the
  // contexts that share it (so that their persistent launches can run side by side)
  const int full = ctx->num_sms * std::min(per_sm, GP_PLP_BLOCKS_PER_SM);
  const int share = std::max(1, full / std::max(1, ctx->device_share));
  const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(share, ((int64_t)n + kPThreads - 1) / kPThreads));

  int64_t ncl0 = 0;
  if (p.count_clusters && nclusters_dev) read_back(ctx, nclusters_dev, sizeof(int64_t), &ncl0);
  int64_t cap2 = 1;
  while (cap2 < n) cap2 <<= 1;
  DBuf<int4> prop(ctx, (size_t)n);
  DBuf<int32_t> incoming(ctx, (size_t)nlabels), blist(ctx, (size_t)n), ovi(ctx, (size_t)cap2);
  DBuf<int32_t> bcnt(ctx, 2 * (size_t)kPKeys), bfill(ctx, 2 * (size_t)kPKeys), boffs(ctx, 2 * ((size_t)kPKeys + 1));
  bcnt.zero();
  bfill.zero();
  DBuf<uint8_t> acc(ctx, (size_t)n);
  DBuf<uint64_t> ovk(ctx, (size_t)cap2);
  DBuf<uint32_t> ovv(ctx, (size_t)cap2);
  DBuf<long long> ovps(ctx, (size_t)cap2);
  DBuf<int32_t> depw;
  DBuf<unsigned long long> dkey;
  DBuf<uint64_t> ekeys;
  DBuf<unsigned> chist(ctx, 8 * 256);
  if (p.count_clusters) {
    depw.reset(ctx, (size_t)nlabels);
    dkey.reset(ctx, (size_t)nlabels);
    ekeys.reset(ctx, (size_t)n);
    depw.zero();
    dkey.zero();
  }
  incoming.zero();
  DBuf<uint8_t> dirty;
  if (!p.count_clusters) {
    dirty.reset(ctx, (size_t)n);
    dirty.fill_bytes(1);
  }
  // global rating tables for nodes whose table exceeds the shared one
  DBuf<int> md(ctx, 1);
  md.zero();
  k_pmax_degree<<<grid_for(n, 256, ctx->num_sms * 8), 256, 0, ctx->stream>>>(g.xadj, n, md.get());
  GP_LAUNCH_CHECK();
  const int maxdeg = read_scalar(ctx, md.get());
  int bits = 1;
  while ((1 << bits) < 2 * maxdeg) bits++;
  DBuf<int32_t> gtk, gtv;
  int64_t gstride = 0;
  int hblocks = grid;  // blocks that rate the nodes of degree > kPLight
  if ((1 << bits) > kPHeavySlots) {
    gstride = (int64_t)1 << bits;
    hblocks = table_blocks(g.m2, gstride, grid);
    gtk.reset(ctx, (size_t)(gstride * hblocks));
    gtv.reset(ctx, (size_t)(gstride * hblocks));
    gtk.fill_bytes(0xFF);
    gtv.zero();
  }
  struct Ctl {
    PCount cnt[3];
    unsigned bar[2];
    int status;
    int pad;
    PResult out;
  };
  DBuf<Ctl> ctl(ctx, 1);
  ctl.zero();
  Ctl *dc = ctl.get();

  PArgs a{};
  a.xadj = g.xadj; a.adjncy = g.adjncy; a.adjwgt = g.adjwgt; a.vwgt = g.vwgt; a.n = n;
  a.label = label; a.weight = weight; a.label8 = label8; a.nlabels = nlabels;
  a.dirty = p.count_clusters ? nullptr : dirty.get();
  a.bound = p.bound; a.n_min = p.n_min; a.count_clusters = p.count_clusters ? 1 : 0;
  a.rounds = p.rounds; a.S = p.subrounds; a.dbg_max = p.dbg_max_subrounds; a.level = p.level;
  a.seed = seed; a.tag_act = p.tag_act; a.tag_tie = p.tag_tie; a.tag_prio = p.tag_prio;
  a.ncl0 = ncl0;
  a.prop = prop.get(); a.incoming = incoming.get(); a.acc = acc.get(); a.blist = blist.get();
  a.bcnt = bcnt.get(); a.bfill = bfill.get(); a.boffs = boffs.get();
  a.ovk = ovk.get(); a.ovv = ovv.get(); a.ovi = ovi.get(); a.ovps = ovps.get(); a.cap2 = cap2;
  a.depw = depw.get(); a.dkey = dkey.get(); a.ekeys = ekeys.get(); a.chist = chist.get();
  a.gtk = gtk.get(); a.gtv = gtv.get(); a.gstride = gstride; a.hblocks = hblocks;
  a.cnt = dc->cnt; a.bar = dc->bar; a.status = &dc->status;
  a.spin_cap = ctx->wait_spins > 0 ? ctx->wait_spins : (ctx->wait_spins == 0 ? kDefaultWaitSpins : -1);
  a.out = &dc->out;
  a.units = ctx->d_units ? ctx->d_units + p.prof_small * PROF_UNITS : nullptr;
  TraceTimer trace(ctx);
  {
    ProfScope ps(ctx, p.prof_small);
    void *args[] = {&a};
    GP_CUDA(cudaLaunchCooperativeKernel((const void *)k_lp_persistent, dim3(grid), dim3(kPThreads), args,
                                        kSmemBytes, ctx->stream));
    GP_LAUNCH_CHECK();
  }
  Ctl h;
  read_back(ctx, dc, sizeof(Ctl), &h);
  GP_REQUIRE(h.status == 0, (gp_status)(h.status == GP_ERR_TIMEOUT ? GP_ERR_TIMEOUT : GP_ERR_CUDA),
             "label propagation: a grid-wide wait ran out (GP_ERR_TIMEOUT)");
  res.subrounds = h.out.subrounds;
  res.moves = h.out.moves;
  res.nclusters = h.out.nclusters;
  res.proposals = h.out.proposals;
  res.overflow_total = h.out.ov_total;
  res.overflow_max = h.out.ov_max;
  res.capped = h.out.capped;
  if (trace.on())
    fprintf(stderr,
            "[gp lp-small] %s level=%d n=%d m2=%lld labels=%lld grid=%d subrounds=%d moves=%lld proposals=%lld "
            "overflow_total=%lld overflow_max=%lld capped=%d ms=%.3f\n",
            p.count_clusters ? "cluster" : "refine", p.level, n, (long long)g.m2, (long long)nlabels, grid,
            res.subrounds, (long long)res.moves, (long long)res.proposals, (long long)res.overflow_total,
            (long long)res.overflow_max, res.capped, trace.ms());
  if (p.count_clusters && nclusters_dev)
    GP_CUDA(cudaMemcpyAsync(nclusters_dev, &dc->out.nclusters, sizeof(int64_t), cudaMemcpyDeviceToDevice,
                            ctx->stream));
  return res;
}

}  // namespace gp
