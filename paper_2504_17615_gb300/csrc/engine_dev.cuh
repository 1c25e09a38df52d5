// engine_dev.cuh -- the batched engine (device side): many small and mid-sized graphs partitioned
// by one persistent launch.
//
// Every CTA of a persistent grid takes whole graphs from a device-side queue
// (an atomic head over the items, largest first) and runs the complete
// multilevel partition of each graph inside the CTA: validation, the
// coarsening loop of Alg. 1 (size-constrained LP clustering with the 2.5x
// cap, 2-hop and isolated-node clustering of Sec. 3 / Sec. 4.1, contraction
// of Sec. 2, the sparsification of Sec. 4.2 when the trigger of Alg. 1
// fires), the recursive-bisection initial partition with the greedy
// rebalance (Sec. 4.3), projection and LP refinement on every level (Sec. 3),
// and the cut.  A graph of a few thousand to a few hundred thousand nodes
// cannot fill the GPU by itself -- every level of the per-graph path is a
// handful of launches and grid-wide barriers around microseconds of work --
// but a CTA per graph turns every barrier into __syncthreads and lets a few
// hundred graphs proceed side by side with no launch between their phases.
//
// The method and its readings are those of the per-graph path (R1-R20): the
// same hash keys, the same synchronous sub-rounds, the same acceptance order,
// cap, packing rules, bipartitioner and rebalance, so every item's blocks and
// cut equal a gp_partition call with the same arguments.  Only the execution
// differs: block-wide scans, an LSD radix sort in global memory, lane-group
// rating (the per-graph path's rate_group) for nodes of degree <= 128 and a
// CTA-wide table for larger ones, and a named barrier per group of four warps
// that runs one bisection trial.
//
// Memory: each CTA owns an arena of fixed size carved out of one allocation.
// The hierarchy of the current graph grows from the bottom of the arena,
// scratch from the top.  A graph whose hierarchy does not fit is abandoned
// with a retry status and the host runs it on the per-graph path.
#pragma once
#include "engine_abi.cuh"
#include "lp.cuh"
#include "lp_rate.cuh"

namespace gp {

namespace {

using namespace eng;
constexpr unsigned FULL = 0xFFFFFFFFu;

// ------------------------------------------------------------------ arena

struct Arena {
  unsigned char *base;
  int64_t lo, hi;  // hierarchy top (grows up), scratch bottom (grows down)
  bool fail;
  __device__ void *hier(int64_t bytes) {
    bytes = (bytes + 255) & ~(int64_t)255;
    if (fail || lo + bytes > hi) { fail = true; return base; }
    void *p = base + lo;
    lo += bytes;
    return p;
  }
  __device__ void *scr(int64_t bytes) {
    bytes = (bytes + 255) & ~(int64_t)255;
    if (fail || hi - bytes < lo) { fail = true; return base; }
    hi -= bytes;
    return base + hi;
  }
  template <typename T>
  __device__ T *h(int64_t count) { return static_cast<T *>(hier(count * (int64_t)sizeof(T))); }
  template <typename T>
  __device__ T *s(int64_t count) { return static_cast<T *>(scr(count * (int64_t)sizeof(T))); }
};

// ------------------------------------------------------- block primitives

struct ESmem {
  long long ll[kEMaxWarps];
  unsigned long long u[kEMaxWarps];
  int i[kEMaxWarps];
  int hist[256], base[256], tcount[256];
  int wc[kEMaxWarps * 5], off[5], tot[5];
  int flag, cnt;
};

__device__ __forceinline__ int nwarps() { return (int)(blockDim.x >> 5); }
__device__ __forceinline__ int warp_idx() { return (int)(threadIdx.x >> 5); }

__device__ long long blk_sum(long long x, ESmem &s) {
  x = warp_sum(x);
  __syncthreads();
  if (lane_id() == 0) s.ll[warp_idx()] = x;
  __syncthreads();
  long long t = 0;
  for (int i = 0; i < nwarps(); i++) t += s.ll[i];
  return t;
}

__device__ long long blk_max(long long x, ESmem &s) {
  x = warp_max(x);
  __syncthreads();
  if (lane_id() == 0) s.ll[warp_idx()] = x;
  __syncthreads();
  long long t = s.ll[0];
  for (int i = 1; i < nwarps(); i++) t = s.ll[i] > t ? s.ll[i] : t;
  return t;
}

__device__ __forceinline__ unsigned long long wmin64(unsigned long long x) {
  const unsigned hi = (unsigned)(x >> 32);
  const unsigned mh = __reduce_min_sync(FULL, hi);
  const unsigned ml = __reduce_min_sync(FULL, hi == mh ? (unsigned)x : 0xFFFFFFFFu);
  return ((unsigned long long)mh << 32) | ml;
}

__device__ __forceinline__ unsigned long long wmax64(unsigned long long x) {
  const unsigned hi = (unsigned)(x >> 32);
  const unsigned mh = __reduce_max_sync(FULL, hi);
  const unsigned ml = __reduce_max_sync(FULL, hi == mh ? (unsigned)x : 0u);
  return ((unsigned long long)mh << 32) | ml;
}

__device__ unsigned long long blk_min_u64(unsigned long long x, ESmem &s) {
  x = wmin64(x);
  __syncthreads();
  if (lane_id() == 0) s.u[warp_idx()] = x;
  __syncthreads();
  unsigned long long t = s.u[0];
  for (int i = 1; i < nwarps(); i++) t = s.u[i] < t ? s.u[i] : t;
  return t;
}

// Exclusive scan over i < n of val(i); out(i, prefix) receives each prefix.
// Returns the total.  Tiles of blockDim values, in index order.
template <typename T, class V, class O>
__device__ T blk_scan(int64_t n, V val, O out, ESmem &s) {
  T carry = 0;
  const int lane = (int)lane_id(), w = warp_idx(), nw = nwarps();
  T *sw = reinterpret_cast<T *>(sizeof(T) == 8 ? (void *)s.ll : (void *)s.i);
  for (int64_t b = 0; b < n; b += blockDim.x) {
    const int64_t i = b + threadIdx.x;
    const T x = i < n ? val(i) : (T)0;
    T incl = x;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const T y = __shfl_up_sync(FULL, incl, o);
      if (lane >= o) incl += y;
    }
    __syncthreads();
    if (lane == 31) sw[w] = incl;
    __syncthreads();
    T before = carry, total = carry;
    for (int q = 0; q < nw; q++) {
      const T t = sw[q];
      if (q < w) before += t;
      total += t;
    }
    if (i < n) out(i, before + incl - x);
    carry = total;
  }
  __syncthreads();
  return carry;
}

// Writes every index i < n of class cls(i) in [0, NC) into out[s.off[c] + rank]
// (ranks in index order); s.off must hold the start of every class and is
// advanced past it.  cls(i) < 0: not listed.
template <int NC, class F>
__device__ void blk_classify(int64_t n, F cls, int32_t *out, ESmem &s) {
  const int lane = (int)lane_id(), w = warp_idx(), nw = nwarps();
  for (int64_t b = 0; b < n; b += blockDim.x) {
    const int64_t i = b + threadIdx.x;
    const int c = i < n ? cls(i) : -1;
    int rank = 0;
#pragma unroll
    for (int q = 0; q < NC; q++) {
      const unsigned m = __ballot_sync(FULL, c == q);
      if (c == q) rank = __popc(m & lanemask_lt());
      if (lane == 0) s.wc[w * NC + q] = __popc(m);
    }
    __syncthreads();
    if (threadIdx.x < NC) {
      int run = 0;
      for (int q = 0; q < nw; q++) {
        const int t = s.wc[q * NC + threadIdx.x];
        s.wc[q * NC + threadIdx.x] = run;
        run += t;
      }
      s.tot[threadIdx.x] = run;
    }
    __syncthreads();
    if (c >= 0) out[s.off[c] + s.wc[w * NC + c] + rank] = (int32_t)i;
    __syncthreads();
    if (threadIdx.x < NC) s.off[threadIdx.x] += s.tot[threadIdx.x];
    __syncthreads();
  }
}

// Counts the indices of every class (s.tot[c]) and sets s.off[c] to the class
// starts (classes in order, from `start`).
template <int NC, class F>
__device__ void blk_count_classes(int64_t n, F cls, int start, ESmem &s) {
  int cnt[NC];
#pragma unroll
  for (int q = 0; q < NC; q++) cnt[q] = 0;
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
    const int c = cls(i);
#pragma unroll
    for (int q = 0; q < NC; q++) cnt[q] += c == q ? 1 : 0;
  }
#pragma unroll
  for (int q = 0; q < NC; q++) {
    const long long t = blk_sum(cnt[q], s);
    if (threadIdx.x == 0) s.tot[q] = (int)t;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    int run = start;
    for (int q = 0; q < NC; q++) { s.off[q] = run; run += s.tot[q]; }
  }
  __syncthreads();
}

// Stable LSD radix sort of (key, val) pairs on key bits [0, nbits), 8 bits a
// pass, in global memory; k/v and tk/tv swap roles every pass that moves
// anything; on return k/v point at the sorted data.  wcnt: nwarps * 256 ints
// of shared memory.
__device__ void blk_sort(uint64_t *&k, uint32_t *&v, uint64_t *&tk, uint32_t *&tv, int n, int nbits, int *wcnt,
                         ESmem &s) {
  bool used = false;
  const int w = warp_idx(), nw = nwarps();
  for (int shift = 0; shift < nbits; shift += 8) {
    for (int t = threadIdx.x; t < 256; t += blockDim.x) s.hist[t] = 0;
    __syncthreads();
    for (int i = threadIdx.x; i < n; i += blockDim.x) atomicAdd(&s.hist[(int)((k[i] >> shift) & 255)], 1);
    __syncthreads();
    if (threadIdx.x == 0) {
      int run = 0, skip = 0;
      for (int d = 0; d < 256; d++) {
        s.base[d] = run;
        run += s.hist[d];
        if (s.hist[d] == n) skip = 1;
      }
      s.flag = skip;
    }
    __syncthreads();
    if (s.flag) continue;
    used = true;
    for (int b = 0; b < n; b += blockDim.x) {
      const int i = b + (int)threadIdx.x;
      const bool in = i < n;
      const uint64_t key = in ? k[i] : 0;
      const uint32_t val = in ? v[i] : 0;
      const int d = (int)((key >> shift) & 255);
      for (int t = threadIdx.x; t < nw * 256; t += blockDim.x) wcnt[t] = 0;
      __syncthreads();
      const unsigned act = __ballot_sync(FULL, in);
      int rank = 0;
      if (in) {
        const unsigned peers = __match_any_sync(act, d);
        rank = __popc(peers & lanemask_lt());
        if (rank == 0) wcnt[w * 256 + d] = __popc(peers);
      }
      __syncthreads();
      for (int dd = threadIdx.x; dd < 256; dd += blockDim.x) {
        int run = 0;
        for (int q = 0; q < nw; q++) {
          const int t = wcnt[q * 256 + dd];
          wcnt[q * 256 + dd] = run;
          run += t;
        }
        s.tcount[dd] = run;
      }
      __syncthreads();
      if (in) {
        const int pos = s.base[d] + wcnt[w * 256 + d] + rank;
        tk[pos] = key;
        tv[pos] = val;
      }
      __syncthreads();
      for (int dd = threadIdx.x; dd < 256; dd += blockDim.x) s.base[dd] += s.tcount[dd];
      __syncthreads();
    }
    uint64_t *x = k; k = tk; tk = x;
    uint32_t *y = v; v = tv; tv = y;
  }
  // wcnt is the CTA-wide hash table (keys, then values) outside sorts: leave it empty
  if (used) {
    for (int t = threadIdx.x; t < kEBlockSlots; t += blockDim.x) { wcnt[t] = -1; wcnt[kEBlockSlots + t] = 0; }
  }
  __syncthreads();
}

// First index of a sorted key array with key >= x.
__device__ __forceinline__ int lower_bound_u64(const uint64_t *a, int n, uint64_t x) {
  int lo = 0, hi = n;
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if (a[mid] < x) lo = mid + 1; else hi = mid;
  }
  return lo;
}

__device__ __forceinline__ int ebits(int64_t x) {  // bits needed for values in [0, x]
  int b = 0;
  while (b < 62 && ((int64_t)1 << b) <= x) b++;
  return b;
}

// Calls f(row, entry) for every CSR entry; each warp walks 32 consecutive rows
// as one entry range (the entry's row found by a shuffle search over the
// lanes' row ends).
template <class F>
__device__ void blk_for_entries(const int32_t *xadj, int n, F f) {
  const int lane = (int)lane_id();
  for (int u0 = warp_idx() * 32; u0 < n; u0 += nwarps() * 32) {
    const int u = u0 + lane;
    const bool valid = u < n;
    const int xe = valid ? xadj[u + 1] : 0x7FFFFFFF;
    const int e0 = __shfl_sync(FULL, valid ? xadj[u] : 0, 0);
    const int last = (n - u0 < 32 ? n - u0 : 32) - 1;
    const int e1 = __shfl_sync(FULL, xe, last);
    for (int f0 = e0; f0 < e1; f0 += 32) {
      const int e = f0 + lane;
      int q = 0;
#pragma unroll
      for (int step = 16; step > 0; step >>= 1) {
        const int val = __shfl_sync(FULL, xe, q + step - 1);
        if (val <= e) q += step;
      }
      if (e < e1) f(u0 + q, e);
    }
  }
}

// floor(a * b / c) for a * b up to 2^128 (c < 2^63); the quotient must fit 64 bits
__device__ uint64_t muldiv_u64(uint64_t a, uint64_t b, uint64_t c) {
  const uint64_t hi = __umul64hi(a, b), lo = a * b;
  if (hi == 0) return lo / c;
  uint64_t q = 0, r = 0;
  for (int i = 127; i >= 0; i--) {
    const uint64_t bit = i >= 64 ? (hi >> (i - 64)) & 1 : (lo >> i) & 1;
    r = (r << 1) | bit;
    q <<= 1;
    if (r >= c) { r -= c; q |= 1; }
  }
  return q;
}

// L_max = floor(ceil(W / k) (10^6 + eps_ppm) / 10^6) (R2)
__device__ __forceinline__ int64_t lmax_of_dev(int64_t W, int k, int64_t eps_ppm) {
  const int64_t base = (W + k - 1) / k;
  return (int64_t)muldiv_u64((uint64_t)base, (uint64_t)(1000000 + eps_ppm), 1000000ull);
}

// ---------------------------------------------------------------- context

struct EGraph {
  const int32_t *xadj, *adjncy, *vwgt, *adjwgt;
  int32_t n;
  int64_t m2;
};

struct ECtx {
  Arena ar;
  ESmem *s;
  bool prof;
  long long t0;
  long long *cyc;  // per-phase SM cycles of the current item (thread 0's count is the one kept)
  int *wtk, *wtv;  // per-warp tables (kEWarpSlots each)
  int *btk, *btv;  // CTA-wide table (kEBlockSlots each); also the sort's warp counters
  const gp_config *cfg;
};

__device__ __forceinline__ void phase(ECtx &c, int p) {
  if (c.prof) {
    const long long t = clock64();
    c.cyc[p] += t - c.t0;
    c.t0 = t;
  }
}

struct ELp {
  uint32_t tag_act, tag_tie, tag_prio;
  int level, rounds, S, dbg;
  int64_t bound, n_min;
  bool count;
};

struct ELpScr {
  uint8_t *sr, *acc;
  int32_t *pk, *list, *incoming, *P, *depw;
  uint64_t *ovk, *ovk2, *dkey, *empt, *empt2;
  uint32_t *ovv, *ovv2, *ev, *ev2;
  int2 *gtab;   // the CTA's table for nodes of degree > kEWarpHeavy
  int gslots;
  int2 *wtab;   // per warp: a table of wbits^2 slots for nodes of degree in (kELight, kEWarpHeavy]
  int wbits;
};

// degree classes: lane groups of 8 / a warp with one or four entries per lane
// (shared tables), a warp with a table in the arena, the CTA
__device__ __forceinline__ int deg_class(int deg) {
  return deg <= 8 ? 0 : deg <= 32 ? 1 : deg <= kELight ? 2 : deg <= kEWarpHeavy ? 3 : 4;
}

__device__ int pow2_at_least(int64_t x) {
  int b = 1;
  while (((int64_t)1 << b) < x) b++;
  return b;
}

__device__ void lp_scratch(ECtx &c, int n, int64_t nlabels, int maxdeg, ELpScr &L) {
  L.sr = c.ar.s<uint8_t>(n);
  L.acc = c.ar.s<uint8_t>(n);
  L.pk = c.ar.s<int32_t>(n);
  L.list = c.ar.s<int32_t>(n);
  L.P = c.ar.s<int32_t>(n);
  L.incoming = c.ar.s<int32_t>(nlabels);
  L.depw = c.ar.s<int32_t>(nlabels);
  L.dkey = c.ar.s<uint64_t>(nlabels);
  L.ovk = c.ar.s<uint64_t>(n);
  L.ovk2 = c.ar.s<uint64_t>(n);
  L.ovv = c.ar.s<uint32_t>(n);
  L.ovv2 = c.ar.s<uint32_t>(n);
  L.empt = c.ar.s<uint64_t>(n);
  L.empt2 = c.ar.s<uint64_t>(n);
  L.ev = c.ar.s<uint32_t>(n);
  L.ev2 = c.ar.s<uint32_t>(n);
  L.gslots = 0;
  L.gtab = nullptr;
  if (2 * (int64_t)maxdeg > kEBlockSlots) {
    L.gslots = 1 << pow2_at_least(2 * (int64_t)maxdeg);
    L.gtab = c.ar.s<int2>(L.gslots);
  }
  L.wbits = 0;
  L.wtab = nullptr;
  if (maxdeg > kELight) {
    L.wbits = pow2_at_least(2 * (int64_t)min(maxdeg, kEWarpHeavy));
    L.wtab = c.ar.s<int2>((int64_t)nwarps() << L.wbits);
  }
}

// Empties the arena tables of an LP scratch (they are left empty after every use).
__device__ void lp_scratch_clear(ELpScr &L) {
  for (int t = threadIdx.x; t < L.gslots; t += blockDim.x) L.gtab[t] = make_int2(-1, 0);
  const int64_t w = L.wtab ? ((int64_t)nwarps() << L.wbits) : 0;
  for (int64_t t = threadIdx.x; t < w; t += blockDim.x) L.wtab[t] = make_int2(-1, 0);
}

// Adds (key, w) into a warp's open-addressing table of 2^bits int pairs
// (key -1: empty slot); the table has room for every key inserted.
__device__ __forceinline__ void wtab_add(int2 *tab, int bits, int key, int w) {
  const unsigned mask = (1u << bits) - 1u;
  unsigned sl = ((unsigned)key * 2654435761u) >> (32 - bits);
  for (int probe = 0; probe <= (int)mask; probe++) {
    const int prev = atomicCAS(&tab[sl].x, -1, key);
    if (prev == -1 || prev == key) {
      atomicAdd(&tab[sl].y, w);
      return;
    }
    sl = (sl + 1) & mask;
  }
}

// Rates one node of degree in (kELight, kEWarpHeavy] with one warp and the
// warp's table in the arena; same choice as rate_heavy.
template <bool FAV>
__device__ int rate_warp_tab(const EGraph &g, const int32_t *label, const int32_t *weight, int64_t bound,
                             uint64_t ktie, int v, int own, int cv, int2 *tab, int bits) {
  const int lane = (int)lane_id();
  const int st = g.xadj[v], deg = g.xadj[v + 1] - st;
  const int tbits = pow2_at_least(2 * (int64_t)deg);
  const int tsize = 1 << tbits;
  for (int j = lane; j < deg; j += 32) wtab_add(tab, tbits, label[g.adjncy[st + j]], g.adjwgt[st + j]);
  __syncwarp();
  int own_loc = 0, rloc = -1;
  for (int t = lane; t < tsize; t += 32) {
    const int2 x = tab[t];
    if (x.x < 0) continue;
    if (x.x == own) { own_loc = x.y; continue; }
    if (!FAV && (int64_t)weight[x.x] + cv > bound) continue;
    rloc = x.y > rloc ? x.y : rloc;
  }
  const int own_r = FAV ? -1 : (int)__reduce_max_sync(FULL, (unsigned)own_loc);
  const int rmax = (int)__reduce_max_sync(FULL, (unsigned)(rloc + 1)) - 1;
  int best = -1;
  if (rmax >= 0 && rmax > own_r) {
    unsigned long long p = ~0ull;
    for (int t = lane; t < tsize; t += 32) {
      const int2 x = tab[t];
      if (x.x < 0 || x.x == own || x.y != rmax) continue;
      if (!FAV && (int64_t)weight[x.x] + cv > bound) continue;
      const unsigned long long q = ((unsigned long long)h32(ktie, (uint32_t)v, (uint32_t)x.x) << 32) | (uint32_t)x.x;
      p = q < p ? q : p;
    }
    best = (int)(uint32_t)wmin64(p);
  }
  __syncwarp();
  for (int t = lane; t < tsize; t += 32) tab[t] = make_int2(-1, 0);
  __syncwarp();
  (void)bits;
  return best;
}


__device__ void fill_i32(int32_t *a, int64_t n, int32_t x) {
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) a[i] = x;
}

// Rates one node of degree > kELight with the whole CTA (table in shared
// memory up to kEBlockSlots slots, else in the arena).  LP mode: returns the
// best admissible label rated above own, or -1.  FAV mode: the best label !=
// own, ignoring the bound and own's rating.
template <bool FAV>
__device__ int rate_heavy(ECtx &c, const EGraph &g, const int32_t *label, const int32_t *weight, int64_t bound,
                          uint64_t ktie, int v, int own, int cv, int2 *gtab) {
  const int st = g.xadj[v], deg = g.xadj[v + 1] - st;
  const int bits = pow2_at_least(2 * (int64_t)deg);
  const int tsize = 1 << bits;
  const bool sm = tsize <= kEBlockSlots;
  int *tk = sm ? c.btk : nullptr;
  int *tv = sm ? c.btv : nullptr;
  for (int j = threadIdx.x; j < deg; j += blockDim.x) {
    const int L = label[g.adjncy[st + j]];
    const int w = g.adjwgt[st + j];
    unsigned sl = ((unsigned)L * 2654435761u) >> (32 - bits);
    for (int probe = 0; probe < tsize; probe++) {  // at most deg labels in 2 deg slots: never full
      const int prev = sm ? atomicCAS(&tk[sl], -1, L) : atomicCAS(&gtab[sl].x, -1, L);
      if (prev == -1 || prev == L) {
        atomicAdd(sm ? &tv[sl] : &gtab[sl].y, w);
        break;
      }
      sl = (sl + 1) & (unsigned)(tsize - 1);
    }
  }
  __syncthreads();
  int own_loc = 0, rloc = -1;
  for (int t = threadIdx.x; t < tsize; t += blockDim.x) {
    const int L = sm ? tk[t] : gtab[t].x;
    if (L < 0) continue;
    const int r = sm ? tv[t] : gtab[t].y;
    if (L == own) { own_loc = r; continue; }
    if (!FAV && (int64_t)weight[L] + cv > bound) continue;
    rloc = r > rloc ? r : rloc;
  }
  const int own_r = FAV ? -1 : (int)blk_max(own_loc, *c.s);
  const int rmax = (int)blk_max(rloc, *c.s);
  int best = -1;
  if (rmax >= 0 && rmax > own_r) {
    unsigned long long p = ~0ull;
    for (int t = threadIdx.x; t < tsize; t += blockDim.x) {
      const int L = sm ? tk[t] : gtab[t].x;
      if (L < 0 || L == own) continue;
      if ((sm ? tv[t] : gtab[t].y) != rmax) continue;
      if (!FAV && (int64_t)weight[L] + cv > bound) continue;
      const unsigned long long q = ((unsigned long long)h32(ktie, (uint32_t)v, (uint32_t)L) << 32) | (uint32_t)L;
      p = q < p ? q : p;
    }
    p = blk_min_u64(p, *c.s);
    best = (int)(uint32_t)p;
  }
  __syncthreads();
  for (int t = threadIdx.x; t < tsize; t += blockDim.x) {
    if (sm) { tk[t] = -1; tv[t] = 0; }
    else gtab[t] = make_int2(-1, 0);
  }
  __syncthreads();
  return best;
}

// Rates the listed nodes (all of one degree class) by lane groups of G lanes,
// E entries per lane; LP mode proposes (pk, incoming), FAV mode writes fav.
template <int G, int E, bool FAV>
__device__ void rate_lanes(ECtx &c, const EGraph &g, const int32_t *list, int cnt, const int32_t *label,
                           const int32_t *weight, int64_t bound, uint64_t ktie, int32_t *pk, int32_t *incoming) {
  constexpr int NV = 32 / G;
  constexpr int TS = GroupTable<G, E>::TS;
  const int lane = (int)lane_id(), grp = lane / G, gl = lane % G;
  const unsigned gmask = G == 32 ? FULL : (((1u << G) - 1u) << (grp * G));
  int *tk = c.wtk + warp_idx() * kEWarpSlots + grp * TS;
  int *tv = c.wtv + warp_idx() * kEWarpSlots + grp * TS;
  for (int i0 = warp_idx() * NV; i0 < cnt; i0 += nwarps() * NV) {
    const int i = i0 + grp;
    const int v = i < cnt ? list[i] : -1;
    int st = 0, deg = 0, own = -2, cv = 0;
    if (v >= 0) {
      st = g.xadj[v];
      deg = g.xadj[v + 1] - st;
      own = label[v];
      cv = g.vwgt[v];
    }
    int nc = 0;
    bool stable = false;
    const unsigned best = rate_group<G, E, FAV>(g.adjncy, g.adjwgt, label, nullptr, weight, nullptr, bound, ktie, v,
                                                st, deg, own, cv, tk, tv, gmask, gl, false, nc, stable);
    if (gl == 0 && v >= 0) {
      if (FAV) {
        pk[v] = best == 0xFFFFFFFFu ? -1 : (int)best;
      } else {
        pk[v] = best == 0xFFFFFFFFu ? -1 : (int)best;
        if (best != 0xFFFFFFFFu) atomicAdd(&incoming[best], cv);
      }
    }
  }
}

// Rates the four degree-class lists list[off[q] .. off[q+1]) (heavy nodes: the
// whole CTA, one node after another).
template <bool FAV>
__device__ void rate_all(ECtx &c, const EGraph &g, const int32_t *list, const int *off, const int32_t *label,
                         const int32_t *weight, int64_t bound, uint64_t ktie, int32_t *pk, int32_t *incoming,
                         const ELpScr &L) {
  int2 *gtab = L.gtab;
  rate_lanes<8, 1, FAV>(c, g, list + off[0], off[1] - off[0], label, weight, bound, ktie, pk, incoming);
  rate_lanes<32, 1, FAV>(c, g, list + off[1], off[2] - off[1], label, weight, bound, ktie, pk, incoming);
  rate_lanes<32, 4, FAV>(c, g, list + off[2], off[3] - off[2], label, weight, bound, ktie, pk, incoming);
  if (off[4] > off[3]) {
    int2 *tab = L.wtab + ((int64_t)warp_idx() << L.wbits);
    for (int i = off[3] + warp_idx(); i < off[4]; i += nwarps()) {
      const int v = list[i];
      const int own = label[v], cv = g.vwgt[v];
      const int best = rate_warp_tab<FAV>(g, label, weight, bound, ktie, v, own, cv, tab, L.wbits);
      if (lane_id() == 0) {
        pk[v] = best;
        if (!FAV && best >= 0) atomicAdd(&incoming[best], cv);
      }
    }
  }
  __syncthreads();
  for (int i = off[4]; i < off[5]; i++) {
    const int v = list[i];
    const int own = label[v], cv = g.vwgt[v];
    const int best = rate_heavy<FAV>(c, g, label, weight, bound, ktie, v, own, cv, gtab);
    if (threadIdx.x == 0) {
      pk[v] = best;
      if (!FAV && best >= 0) atomicAdd(&incoming[best], cv);
    }
  }
  __syncthreads();
}

// Size-constrained LP (Sec. 3; readings R3-R8 for clustering, R20 for
// refinement) on one graph with the CTA: synchronous sub-rounds over the
// snapshot, acceptance of the longest prefix per target in (h32(PRIO), v)
// order, the 2.5x cap by the (D+1)-th smallest emptying key.  label (n) and
// weight (nlabels) are updated in place.
__device__ void e_lp(ECtx &c, const EGraph &g, int32_t *label, int32_t *weight, int64_t nlabels, uint64_t seed,
                     const ELp &P, ELpScr &L, int64_t &ncl, int &subs_out, int64_t &moves_out) {
  ESmem &s = *c.s;
  const int n = g.n;
  fill_i32(L.incoming, nlabels, 0);
  fill_i32(L.depw, nlabels, 0);
  for (int64_t i = threadIdx.x; i < nlabels; i += blockDim.x) L.dkey[i] = 0;
  __syncthreads();
  int subs = 0;
  int64_t total_moves = 0;
  bool stop = false;
  const int kbits = 32 + ebits(nlabels - 1);
  for (int r = 0; r < P.rounds && !stop; r++) {
    const uint64_t kact = stream_key(seed, P.tag_act, (uint32_t)P.level, (uint32_t)r);
    const uint64_t ktie = stream_key(seed, P.tag_tie, (uint32_t)P.level, (uint32_t)r);
    const uint64_t kprio = stream_key(seed, P.tag_prio, (uint32_t)P.level, (uint32_t)r);
    for (int v = threadIdx.x; v < n; v += blockDim.x) {
      const bool has = g.xadj[v + 1] > g.xadj[v];
      L.sr[v] = has ? (uint8_t)(h32(kact, (uint32_t)v, 0) % (uint32_t)P.S) : (uint8_t)0xFF;
    }
    __syncthreads();
    int64_t round_moves = 0;
    for (int sub = 0; sub < P.S; sub++) {
      if (P.count && ncl <= P.n_min) { stop = true; break; }
      if (P.dbg >= 0 && subs >= P.dbg) { stop = true; break; }
      // the sub-round's nodes by degree class, each class in id order
      auto cls = [&](int64_t v) -> int {
        if (L.sr[v] != (uint8_t)sub) return -1;
        return deg_class(g.xadj[v + 1] - g.xadj[v]);
      };
      blk_count_classes<5>(n, cls, 0, s);
      int off[6];
      for (int q = 0; q < 5; q++) off[q] = s.off[q];
      off[5] = s.off[4] + s.tot[4];
      __syncthreads();
      blk_classify<5>(n, cls, L.list, s);
      const int nact = off[5];
      // rate
      rate_all<false>(c, g, L.list, off, label, weight, P.bound, ktie, L.pk, L.incoming, L);
      // decide: targets that take all their proposers
      for (int i = threadIdx.x; i < nact; i += blockDim.x) {
        const int v = L.list[i];
        const int K = L.pk[v];
        if (K < 0) continue;
        L.acc[v] = (int64_t)weight[K] + L.incoming[K] <= P.bound ? 1 : 2;
      }
      __syncthreads();
      // overflowing targets: proposers in (target, h32(PRIO), v) order, longest prefix
      {
        auto ovc = [&](int64_t v) -> int {
          return (L.sr[v] == (uint8_t)sub && L.pk[v] >= 0 && L.acc[v] == 2) ? 0 : -1;
        };
        blk_count_classes<1>(n, ovc, 0, s);
        const int nov = s.tot[0];
        __syncthreads();
        if (nov > 0) {
          blk_classify<1>(n, ovc, reinterpret_cast<int32_t *>(L.ovv), s);
          for (int i = threadIdx.x; i < nov; i += blockDim.x) {
            const int v = (int)L.ovv[i];
            L.ovk[i] = ((uint64_t)(uint32_t)L.pk[v] << 32) | h32(kprio, (uint32_t)v, 0);
          }
          __syncthreads();
          uint64_t *k1 = L.ovk, *k2 = L.ovk2;
          uint32_t *v1 = L.ovv, *v2 = L.ovv2;
          blk_sort(k1, v1, k2, v2, nov, kbits, c.btk, s);
          blk_scan<int>(
              nov, [&](int64_t i) { return g.vwgt[v1[i]]; }, [&](int64_t i, int p) { L.P[i] = p + g.vwgt[v1[i]]; },
              s);
          for (int i = threadIdx.x; i < nov; i += blockDim.x) {
            const int K = (int)(k1[i] >> 32);
            const int st = lower_bound_u64(k1, nov, (uint64_t)(uint32_t)K << 32);
            const int pre = L.P[i] - (st > 0 ? L.P[st - 1] : 0);
            L.acc[v1[i]] = (int64_t)weight[K] + pre <= P.bound ? 1 : 0;
          }
          __syncthreads();
        }
      }
      // the 2.5x cap (R8): at most D = ncl - n_min clusters may be emptied
      if (P.count) {
        for (int i = threadIdx.x; i < nact; i += blockDim.x) {
          const int v = L.list[i];
          if (L.pk[v] < 0 || L.acc[v] != 1) continue;
          const int own = label[v];
          atomicAdd(&L.depw[own], g.vwgt[v]);
          atomicMax((unsigned long long *)&L.dkey[own],
                    ((unsigned long long)h32(kprio, (uint32_t)v, 0) << 32) | (uint32_t)v);
        }
        if (threadIdx.x == 0) s.cnt = 0;
        __syncthreads();
        for (int i0 = 0; i0 < nact; i0 += blockDim.x) {
          const int i = i0 + (int)threadIdx.x;
          bool e = false;
          uint64_t kv = 0;
          if (i < nact) {
            const int v = L.list[i];
            if (L.pk[v] >= 0 && L.acc[v] == 1) {
              const int own = label[v];
              kv = ((uint64_t)h32(kprio, (uint32_t)v, 0) << 32) | (uint32_t)v;
              e = L.depw[own] == weight[own] && kv == L.dkey[own];
            }
          }
          const int j = warp_append(&s.cnt, e);
          if (e) L.empt[j] = kv;
        }
        __syncthreads();
        const int64_t E = s.cnt;
        const int64_t D = ncl - P.n_min;
        __syncthreads();
        if (E > D) {
          for (int i = threadIdx.x; i < E; i += blockDim.x) L.ev[i] = 0;
          __syncthreads();
          uint64_t *k1 = L.empt, *k2 = L.empt2;
          uint32_t *v1 = L.ev, *v2 = L.ev2;
          blk_sort(k1, v1, k2, v2, (int)E, 64, c.btk, s);
          const uint64_t cutoff = k1[D];
          for (int i = threadIdx.x; i < nact; i += blockDim.x) {
            const int v = L.list[i];
            if (L.pk[v] < 0 || L.acc[v] != 1) continue;
            const uint64_t kv = ((uint64_t)h32(kprio, (uint32_t)v, 0) << 32) | (uint32_t)v;
            if (kv >= cutoff) L.acc[v] = 0;
          }
          __syncthreads();
        }
        for (int i = threadIdx.x; i < nact; i += blockDim.x) {
          const int v = L.list[i];
          if (L.pk[v] < 0) continue;
          const int own = label[v];
          L.depw[own] = 0;
          L.dkey[own] = 0;
        }
        __syncthreads();
      }
      // apply; the cluster count follows the weight transitions 0 <-> non-0
      long long moved = 0, delta = 0;
      for (int i = threadIdx.x; i < nact; i += blockDim.x) {
        const int v = L.list[i];
        const int K = L.pk[v];
        if (K < 0) continue;
        if (L.acc[v] == 1) {
          const int own = label[v], cv = g.vwgt[v];
          label[v] = K;
          if (atomicSub(&weight[own], cv) == cv) delta--;
          if (atomicAdd(&weight[K], cv) == 0) delta++;
          moved++;
        }
        L.incoming[K] = 0;
      }
      moved = blk_sum(moved, s);
      delta = blk_sum(delta, s);
      if (P.count) ncl += delta;
      round_moves += moved;
      subs++;
    }
    total_moves += round_moves;
    if (round_moves == 0) break;
  }
  subs_out = subs;
  moves_out = total_moves;
}

// ---------------------------------------------------------- validation

__device__ __forceinline__ unsigned long long epair_hash(uint32_t lo, uint32_t hi, int w) {
  return fmix(((((uint64_t)lo << 32) | hi) + (uint64_t)(uint32_t)w * kGold) ^ kGold);
}

// Problem statement checks (Sec. 2) in the order of the per-graph path;
// returns a gp_status, W and the heaviest node.
__device__ int e_validate(ECtx &c, const EGraph &g, bool full, int64_t &W, int64_t &cmax) {
  ESmem &s = *c.s;
  const int n = g.n;
  W = 0;
  cmax = 0;
  if (n == 0) return GP_OK;
  long long err = 0, cs = 0, cm = 0;
  for (int v = threadIdx.x; v < n; v += blockDim.x) {
    if (g.xadj[v + 1] < g.xadj[v]) err = 1;
    const int cv = g.vwgt[v];
    if (cv <= 0) err = 1;
    else { cs += cv; cm = cv > cm ? cv : cm; }
  }
  if (threadIdx.x == 0 && (g.xadj[0] != 0 || (int64_t)g.xadj[n] != g.m2)) err = 1;
  err = blk_max(err, s);
  cs = blk_sum(cs, s);
  cm = blk_max(cm, s);
  if (err) return GP_ERR_INVALID;
  if (cs > 0x7FFFFFFFll) return GP_ERR_OVERFLOW;
  W = cs;
  cmax = cm;
  if (g.m2 == 0) return GP_OK;
  long long bad = 0, ws = 0;
  unsigned long long hlo = 0, hhi = 0, nlo = 0, nhi = 0;
  blk_for_entries(g.xadj, n, [&](int u, int e) {
    const int v = g.adjncy[e], w = g.adjwgt[e];
    if (v < 0 || v >= n) { bad = 1; return; }
    if (v == u || w <= 0) bad = 1;
    if (e > g.xadj[u] && g.adjncy[e - 1] >= v) bad = 1;
    ws += w > 0 ? w : 0;
    if (u < v) { hlo += epair_hash((uint32_t)u, (uint32_t)v, w); nlo++; }
    else { hhi += epair_hash((uint32_t)v, (uint32_t)u, w); nhi++; }
  });
  bad = blk_max(bad, s);
  ws = blk_sum(ws, s);
  const long long a = blk_sum((long long)hlo, s), b = blk_sum((long long)hhi, s);
  const long long x = blk_sum((long long)nlo, s), y = blk_sum((long long)nhi, s);
  if (bad) return GP_ERR_INVALID;
  if (full && (a != b || x != y)) return GP_ERR_INVALID;
  if (ws / 2 > 0x7FFFFFFFll) return GP_ERR_OVERFLOW;
  return GP_OK;
}

// ------------------------------------------------------------ clustering

struct ECluster {
  int64_t ncl_lp, ncl_2hop, ncl_final, moves;
  int subs;
};

// LP clustering, 2-hop and isolated-node clustering (Sec. 3, Sec. 4.1; R8-R10)
// into label (n); returns the statistics.
__device__ void e_cluster(ECtx &c, const EGraph &g, int64_t U, int level, uint64_t seed, int32_t *label,
                          int maxdeg, ECluster &out) {
  ESmem &s = *c.s;
  const gp_config &cfg = *c.cfg;
  const int n = g.n;
  const int64_t smark = c.ar.hi;
  int32_t *cw = c.ar.s<int32_t>(n);
  ELpScr L;
  lp_scratch(c, n, n, maxdeg, L);
  if (c.ar.fail) return;
  lp_scratch_clear(L);
  for (int v = threadIdx.x; v < n; v += blockDim.x) { label[v] = v; cw[v] = g.vwgt[v]; }
  __syncthreads();
  const int64_t n_min = ((int64_t)n * cfg.shrink_den + cfg.shrink_num - 1) / cfg.shrink_num;
  int64_t ncl = n;
  ELp P;
  P.tag_act = TAG_ACT; P.tag_tie = TAG_TIE; P.tag_prio = TAG_PRIO;
  P.level = level; P.rounds = cfg.lp_rounds; P.S = cfg.lp_subrounds; P.dbg = cfg.dbg_max_subrounds;
  P.bound = U; P.n_min = n_min; P.count = true;
  e_lp(c, g, label, cw, n, seed, P, L, ncl, out.subs, out.moves);
  out.ncl_lp = ncl;
  // 2-hop clustering (R9)
  int32_t *size = L.P;  // reuse: n ints
  int32_t *fav = L.pk;
  if (cfg.two_hop && 2 * ncl > n && ncl > n_min) {
    fill_i32(size, n, 0);
    __syncthreads();
    for (int v = threadIdx.x; v < n; v += blockDim.x) atomicAdd(&size[label[v]], 1);
    __syncthreads();
    auto cand = [&](int64_t v) -> int {
      const int deg = g.xadj[v + 1] - g.xadj[v];
      if (deg == 0 || size[label[v]] != 1 || 2 * (int64_t)g.vwgt[v] > U) return -1;
      return deg_class(deg);
    };
    blk_count_classes<5>(n, cand, 0, s);
    int off[6];
    for (int q = 0; q < 5; q++) off[q] = s.off[q];
    off[5] = s.off[4] + s.tot[4];
    __syncthreads();
    blk_classify<5>(n, cand, L.list, s);
    const uint64_t kfav = stream_key(seed, TAG_FAV, (uint32_t)level, 0);
    rate_all<true>(c, g, L.list, off, label, cw, U, kfav, fav, nullptr, L);
    // (fav, v) keys of the candidates with a favourite (all of them: a singleton's
    // neighbours lie in other clusters), sorted
    auto hasfav = [&](int64_t v) -> int { return (cand(v) >= 0 && fav[v] >= 0) ? 0 : -1; };
    blk_count_classes<1>(n, hasfav, 0, s);
    const int nf = s.tot[0];
    __syncthreads();
    blk_classify<1>(n, hasfav, L.list, s);
    for (int i = threadIdx.x; i < nf; i += blockDim.x) {
      const int v = L.list[i];
      L.ovk[i] = ((uint64_t)(uint32_t)fav[v] << 32) | (uint32_t)v;
      L.ovv[i] = 0;
    }
    int32_t *gmax = L.depw;  // n ints (nlabels = n)
    fill_i32(gmax, n, 0);
    __syncthreads();
    uint64_t *k1 = L.ovk, *k2 = L.ovk2;
    uint32_t *v1 = L.ovv, *v2 = L.ovv2;
    const int ns = nf;
    blk_sort(k1, v1, k2, v2, ns, 32 + ebits(n - 1), c.btk, s);
    for (int i = threadIdx.x; i < ns; i += blockDim.x) {
      const int v = (int)(uint32_t)k1[i];
      atomicMax(&gmax[(int)(k1[i] >> 32)], g.vwgt[v]);
    }
    __syncthreads();
    const int64_t M = ncl - n_min;
    int32_t *rank = reinterpret_cast<int32_t *>(v2);
    auto nonleader = [&](int64_t i) -> int {
      const int f = (int)(k1[i] >> 32);
      const int st = lower_bound_u64(k1, ns, (uint64_t)(uint32_t)f << 32);
      const int64_t gsz = U / gmax[f];
      return ((i - st) % gsz) != 0 ? 1 : 0;
    };
    const int NL = blk_scan<int>(ns, nonleader, [&](int64_t i, int p) { rank[i] = p; }, s);
    for (int i = threadIdx.x; i < ns; i += blockDim.x) {
      const int f = (int)(k1[i] >> 32);
      const int st = lower_bound_u64(k1, ns, (uint64_t)(uint32_t)f << 32);
      const int64_t gsz = U / gmax[f];
      const int64_t p = i - st;
      if (p % gsz == 0 || rank[i] >= M) continue;
      const int leader = (int)(uint32_t)k1[st + (p / gsz) * gsz];
      label[(int)(uint32_t)k1[i]] = label[leader];
    }
    __syncthreads();
    ncl -= NL < M ? NL : M;
  }
  out.ncl_2hop = ncl;
  // isolated nodes (R10)
  if (cfg.isolated && ncl > n_min) {
    auto iso = [&](int64_t v) -> int {
      return (g.xadj[v + 1] == g.xadj[v] && 2 * (int64_t)g.vwgt[v] <= U) ? 0 : -1;
    };
    blk_count_classes<1>(n, iso, 0, s);
    const int niso = s.tot[0];
    __syncthreads();
    if (niso >= 2) {
      blk_classify<1>(n, iso, L.list, s);
      long long cm = 0;
      for (int j = threadIdx.x; j < niso; j += blockDim.x) cm = max(cm, (long long)g.vwgt[L.list[j]]);
      cm = blk_max(cm, s);
      const int64_t gsz = U / cm, M = ncl - n_min;
      for (int j = threadIdx.x; j < niso; j += blockDim.x) {
        if (j % gsz == 0) continue;
        const int64_t before = j - (j + gsz - 1) / gsz;  // non-leaders ahead of j
        if (before >= M) continue;
        label[L.list[j]] = label[L.list[(j / gsz) * gsz]];
      }
      __syncthreads();
      const int64_t NL = niso - (niso + gsz - 1) / gsz;
      ncl -= NL < M ? NL : M;
    }
  }
  out.ncl_final = ncl;
  c.ar.hi = smark;
  __syncthreads();
}

// R11: coarse id = rank of the cluster id among the ids in use.
__device__ int e_relabel(ECtx &c, int n, const int32_t *label, int32_t *cmap) {
  const int64_t smark = c.ar.hi;
  int32_t *rank = c.ar.s<int32_t>(n);
  if (c.ar.fail) return 0;
  fill_i32(rank, n, 0);
  __syncthreads();
  for (int v = threadIdx.x; v < n; v += blockDim.x) rank[label[v]] = 1;
  __syncthreads();
  const int nc = blk_scan<int>(n, [&](int64_t v) { return rank[v]; }, [&](int64_t v, int p) { rank[v] = p; }, *c.s);
  for (int v = threadIdx.x; v < n; v += blockDim.x) cmap[v] = rank[label[v]];
  __syncthreads();
  c.ar.hi = smark;
  return nc;
}

// ------------------------------------------------------------ contraction

// Coarse graph of cmap (Sec. 2): members grouped by coarse node, each coarse
// row aggregated in a hash table (a warp's shared table for rows of at most
// kEWarpSlots / 2 member entries, the CTA's otherwise), rows unordered (R12).
__device__ void e_contract(ECtx &c, const EGraph &g, const int32_t *cmap, int nc, EGraph &out) {
  ESmem &s = *c.s;
  const int n = g.n;
  const int64_t smark = c.ar.hi;
  int32_t *cnt = c.ar.s<int32_t>(nc + 1);
  int32_t *ms = c.ar.s<int32_t>(nc + 1);
  int32_t *dsum = c.ar.s<int32_t>(nc + 1);
  int32_t *es = c.ar.s<int32_t>(nc + 1);
  int32_t *len = c.ar.s<int32_t>(nc + 1);
  int32_t *cvw = c.ar.s<int32_t>(nc + 1);
  int32_t *mem = c.ar.s<int32_t>(n);
  int32_t *heavy = c.ar.s<int32_t>(nc + 1);
  int2 *tmp = c.ar.s<int2>(g.m2 > 0 ? g.m2 : 1);
  if (c.ar.fail) return;
  fill_i32(cnt, nc, 0);
  fill_i32(dsum, nc, 0);
  fill_i32(cvw, nc, 0);
  __syncthreads();
  for (int v = threadIdx.x; v < n; v += blockDim.x) {
    const int A = cmap[v];
    atomicAdd(&cnt[A], 1);
    atomicAdd(&dsum[A], g.xadj[v + 1] - g.xadj[v]);
    atomicAdd(&cvw[A], g.vwgt[v]);
  }
  __syncthreads();
  blk_scan<int>(nc, [&](int64_t A) { return cnt[A]; }, [&](int64_t A, int p) { ms[A] = p; }, s);
  long long dmax = 0;
  for (int A = threadIdx.x; A < nc; A += blockDim.x) dmax = max(dmax, (long long)dsum[A]);
  dmax = blk_max(dmax, s);
  blk_scan<int>(nc, [&](int64_t A) { return dsum[A]; }, [&](int64_t A, int p) { es[A] = p; }, s);
  fill_i32(cnt, nc, 0);
  __syncthreads();
  for (int v = threadIdx.x; v < n; v += blockDim.x) {
    const int A = cmap[v];
    mem[ms[A] + atomicAdd(&cnt[A], 1)] = v;
  }
  __syncthreads();
  int2 *gtab = nullptr;
  int gslots = 0;
  if (2 * dmax > kEBlockSlots) {
    gslots = 1 << pow2_at_least(2 * dmax);
    gtab = c.ar.s<int2>(gslots);
    if (c.ar.fail) return;
    for (int t = threadIdx.x; t < gslots; t += blockDim.x) gtab[t] = make_int2(-1, 0);
    __syncthreads();
  }
  // coarse nodes of at most kEWarpHeavy member entries: a warp each, with its
  // shared table (at most kEWarpSlots / 2 entries) or its table in the arena
  int2 *wtab = nullptr;
  int wbits = 0;
  if (dmax > kEWarpSlots / 2) {
    wbits = pow2_at_least(2 * min(dmax, (long long)kEWarpHeavy));
    wtab = c.ar.s<int2>((int64_t)nwarps() << wbits);
    if (c.ar.fail) return;
    for (int64_t t = threadIdx.x; t < ((int64_t)nwarps() << wbits); t += blockDim.x) wtab[t] = make_int2(-1, 0);
    __syncthreads();
  }
  const int lane = (int)lane_id();
  int *tk = c.wtk + warp_idx() * kEWarpSlots, *tv = c.wtv + warp_idx() * kEWarpSlots;
  int2 *wt = wtab ? wtab + ((int64_t)warp_idx() << wbits) : nullptr;
  constexpr int kBits = 8;  // kEWarpSlots = 256
  for (int A = warp_idx(); A < nc; A += nwarps()) {
    if (dsum[A] > kEWarpHeavy) continue;
    const bool big = dsum[A] > kEWarpSlots / 2;
    const int tbits = big ? pow2_at_least(2 * (int64_t)dsum[A]) : kBits;
    const int m0 = ms[A], nm = cnt[A];
    for (int mb = 0; mb < nm; mb += 32) {
      const int j = mb + lane;
      int st = 0, d = 0;
      if (j < nm) {
        const int v = mem[m0 + j];
        st = g.xadj[v];
        d = g.xadj[v + 1] - st;
      }
      int incl = d;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(FULL, incl, o);
        if (lane >= o) incl += y;
      }
      const int tot = __shfl_sync(FULL, incl, 31);
      for (int t0 = 0; t0 < tot; t0 += 32) {
        const int t = t0 + lane;
        int q = 0;
#pragma unroll
        for (int step = 16; step > 0; step >>= 1) {
          const int val = __shfl_sync(FULL, incl, q + step - 1);
          if (val <= t) q += step;
        }
        const int qs = __shfl_sync(FULL, st, q & 31);
        const int qx = __shfl_sync(FULL, incl - d, q & 31);
        if (t < tot) {
          const int e = qs + (t - qx);
          const int B = cmap[g.adjncy[e]];
          if (B != A) {
            const int w = g.adjwgt[e];
            if (big) {
              wtab_add(wt, tbits, B, w);
            } else {
              unsigned sl = ((unsigned)B * 2654435761u) >> (32 - kBits);
              for (int probe = 0; probe < kEWarpSlots; probe++) {
                const int prev = atomicCAS(&tk[sl], -1, B);
                if (prev == -1 || prev == B) { atomicAdd(&tv[sl], w); break; }
                sl = (sl + 1) & (kEWarpSlots - 1);
              }
            }
          }
        }
      }
    }
    __syncwarp();
    int base = 0;
    for (int t0 = 0; t0 < (1 << tbits); t0 += 32) {
      const int t = t0 + lane;
      int key, val;
      if (big) {
        const int2 x = wt[t];
        key = x.x;
        val = x.y;
      } else {
        key = tk[t];
        val = tv[t];
      }
      const bool has = key >= 0;
      const unsigned m = __ballot_sync(FULL, has);
      if (has) {
        tmp[es[A] + base + __popc(m & lanemask_lt())] = make_int2(key, val);
        if (big) wt[t] = make_int2(-1, 0);
        else { tk[t] = -1; tv[t] = 0; }
      }
      base += __popc(m);
    }
    if (lane == 0) len[A] = base;
    __syncwarp();
  }
  __syncthreads();
  // heavy coarse nodes: the CTA each
  auto hv = [&](int64_t A) -> int { return dsum[A] > kEWarpHeavy ? 0 : -1; };
  blk_count_classes<1>(nc, hv, 0, s);
  const int nh = s.tot[0];
  __syncthreads();
  if (nh > 0) blk_classify<1>(nc, hv, heavy, s);
  for (int h = 0; h < nh; h++) {
    const int A = heavy[h];
    const int bits = pow2_at_least(2 * (int64_t)dsum[A]);
    const int tsize = 1 << bits;
    const bool sm = tsize <= kEBlockSlots;
    const int m0 = ms[A], nm = cnt[A];
    for (int j = warp_idx(); j < nm; j += nwarps()) {
      const int v = mem[m0 + j];
      for (int e = g.xadj[v] + lane; e < g.xadj[v + 1]; e += 32) {
        const int B = cmap[g.adjncy[e]];
        if (B == A) continue;
        const int w = g.adjwgt[e];
        unsigned sl = ((unsigned)B * 2654435761u) >> (32 - bits);
        for (int probe = 0; probe < tsize; probe++) {
          const int prev = sm ? atomicCAS(&c.btk[sl], -1, B) : atomicCAS(&gtab[sl].x, -1, B);
          if (prev == -1 || prev == B) {
            atomicAdd(sm ? &c.btv[sl] : &gtab[sl].y, w);
            break;
          }
          sl = (sl + 1) & (unsigned)(tsize - 1);
        }
      }
    }
    __syncthreads();
    if (threadIdx.x == 0) s.cnt = 0;
    __syncthreads();
    for (int t0 = 0; t0 < tsize; t0 += blockDim.x) {
      const int t = t0 + (int)threadIdx.x;
      int key = -1, val = 0;
      if (t < tsize) {
        key = sm ? c.btk[t] : gtab[t].x;
        val = sm ? c.btv[t] : gtab[t].y;
      }
      const int j = warp_append(&s.cnt, key >= 0);
      if (key >= 0) {
        tmp[es[A] + j] = make_int2(key, val);
        if (sm) { c.btk[t] = -1; c.btv[t] = 0; }
        else gtab[t] = make_int2(-1, 0);
      }
    }
    __syncthreads();
    if (threadIdx.x == 0) len[A] = s.cnt;
    __syncthreads();
  }
  // coarse CSR
  out.n = nc;
  int32_t *ox = c.ar.h<int32_t>(nc + 1);
  if (c.ar.fail) return;
  const int m2c = blk_scan<int>(nc, [&](int64_t A) { return len[A]; }, [&](int64_t A, int p) { ox[A] = p; }, s);
  int32_t *oa = c.ar.h<int32_t>(m2c > 0 ? m2c : 1);
  int32_t *ov = c.ar.h<int32_t>(nc > 0 ? nc : 1);
  int32_t *ow = c.ar.h<int32_t>(m2c > 0 ? m2c : 1);
  if (c.ar.fail) return;
  if (threadIdx.x == 0) ox[nc] = m2c;
  for (int A = threadIdx.x; A < nc; A += blockDim.x) ov[A] = cvw[A];
  for (int A = warp_idx(); A < nc; A += nwarps()) {
    const int o = ox[A], src = es[A], l = len[A];
    for (int t = lane; t < l; t += 32) {
      const int2 x = tmp[src + t];
      oa[o + t] = x.x;
      ow[o + t] = x.y;
    }
  }
  __syncthreads();
  out.xadj = ox; out.adjncy = oa; out.vwgt = ov; out.adjwgt = ow; out.m2 = m2c;
  c.ar.hi = smark;
}

// ---------------------------------------------------------- sparsification

// Sec. 4.2 (R16, R17) in place of the coarse graph G' (the top of the
// hierarchy): T-Weight (mode 1) or UR (mode 2).
__device__ void e_sparsify(ECtx &c, EGraph &gc, int64_t m_hat, int level, uint64_t seed, int mode,
                           gp_level_stats &ls) {
  ESmem &s = *c.s;
  const int n = gc.n;
  const int64_t m = gc.m2 / 2;
  int64_t wt = 0, ng = 0, ne = 0;
  uint64_t T = 0;
  const uint64_t key = stream_key(seed, mode == GP_SPARSIFY_UNIFORM ? TAG_UNIFORM : TAG_SPARSE, (uint32_t)level, 0);
  const bool keep_all = m_hat >= m, keep_none = m_hat <= 0;
  if (!keep_all && !keep_none) {
    if (mode == GP_SPARSIFY_UNIFORM) {
      T = ((uint64_t)m_hat << 32) / (uint64_t)m;
    } else {
      // omega_t: the m_hat-th largest weight over the entries u < v, by digits from the top
      uint32_t prefix = 0, mask = 0;
      int64_t need = m_hat;
      for (int shift = 24; shift >= 0; shift -= 8) {
        for (int t = threadIdx.x; t < 256; t += blockDim.x) s.hist[t] = 0;
        __syncthreads();
        blk_for_entries(gc.xadj, n, [&](int u, int e) {
          const uint32_t w = (uint32_t)gc.adjwgt[e];
          if (u < gc.adjncy[e] && (w & mask) == prefix) atomicAdd(&s.hist[(w >> shift) & 255], 1);
        });
        __syncthreads();
        if (threadIdx.x == 0) {
          int64_t cum = 0;
          int d = 255;
          for (; d > 0; d--) {
            if (cum + s.hist[d] >= need) break;
            cum += s.hist[d];
          }
          s.flag = d;
          s.ll[0] = need - cum;
        }
        __syncthreads();
        prefix |= (uint32_t)s.flag << shift;
        mask |= 255u << shift;
        need = s.ll[0];
        __syncthreads();
      }
      wt = (int64_t)prefix;
      long long a = 0, b = 0;
      blk_for_entries(gc.xadj, n, [&](int u, int e) {
        if (u < gc.adjncy[e]) {
          const int w = gc.adjwgt[e];
          a += w > wt ? 1 : 0;
          b += w == wt ? 1 : 0;
        }
      });
      ng = blk_sum(a, s);
      ne = blk_sum(b, s);
      T = ((uint64_t)(m_hat - ng) << 32) / (uint64_t)ne;
    }
  }
  auto keep = [&](int u, int e) -> bool {
    if (keep_all) return true;
    if (keep_none) return false;
    const int v = gc.adjncy[e], w = gc.adjwgt[e];
    const uint32_t lo = (uint32_t)(u < v ? u : v), hi = (uint32_t)(u < v ? v : u);
    const uint64_t h = h32(key, lo, hi);
    if (mode == GP_SPARSIFY_UNIFORM) return h < T;
    return w > wt || (w == wt && h < T);
  };
  const int64_t smark = c.ar.hi;
  int32_t *klen = c.ar.s<int32_t>(n + 1);
  int32_t *cur = c.ar.s<int32_t>(n + 1);
  if (c.ar.fail) return;
  fill_i32(klen, n, 0);
  fill_i32(cur, n, 0);
  __syncthreads();
  blk_for_entries(gc.xadj, n, [&](int u, int e) {
    if (keep(u, e)) atomicAdd(&klen[u], 1);
  });
  __syncthreads();
  int32_t *sx = c.ar.s<int32_t>(n + 1);
  if (c.ar.fail) return;
  const int m2s = blk_scan<int>(n, [&](int64_t u) { return klen[u]; }, [&](int64_t u, int p) { sx[u] = p; }, s);
  int32_t *sa = c.ar.s<int32_t>(m2s > 0 ? m2s : 1);
  int32_t *sw = c.ar.s<int32_t>(m2s > 0 ? m2s : 1);
  if (c.ar.fail) return;
  if (threadIdx.x == 0) sx[n] = m2s;
  blk_for_entries(gc.xadj, n, [&](int u, int e) {
    if (keep(u, e)) {
      const int p = sx[u] + atomicAdd(&cur[u], 1);
      sa[p] = gc.adjncy[e];
      sw[p] = gc.adjwgt[e];
    }
  });
  __syncthreads();
  // the kept graph replaces G' at the top of the hierarchy (node weights stay)
  int32_t *ox = const_cast<int32_t *>(gc.xadj);
  int32_t *oa = const_cast<int32_t *>(gc.adjncy);
  int32_t *ow = const_cast<int32_t *>(gc.adjwgt);
  for (int u = threadIdx.x; u <= n; u += blockDim.x) ox[u] = sx[u];
  for (int p = threadIdx.x; p < m2s; p += blockDim.x) { oa[p] = sa[p]; ow[p] = sw[p]; }
  __syncthreads();
  gc.m2 = m2s;
  c.ar.hi = smark;
  ls.omega_t = (int32_t)wt;
  ls.n_greater = ng;
  ls.n_equal = ne;
  ls.threshold = T;
}

// --------------------------------------------------- initial partitioning

struct ESub {
  int32_t start, count, kk, b0;
  uint32_t bid;
  int32_t pad;
};

// a subproblem being bisected at the current depth
struct EBis {
  int32_t start, count, kk, b0;
  uint32_t bid;
  int32_t pad;
  int64_t T1, L1, B;
};

__device__ __forceinline__ unsigned long long egain_key(int64_t gain, int j) {
  return ((unsigned long long)(gain + 2147483648ll) << 32) | (0xFFFFFFFFu - (unsigned)j);
}

// States of a node in a growing trial.
enum : uint8_t { T_FREE = 0, T_FRONT = 1, T_ONE = 2, T_OUT = 3 };

// One greedy-growing trial of bisection b (R18) by one warp.  Each step takes,
// in order of their gains at the start of the step, up to B frontier nodes
// that still fit; the node of largest key (gain, -index) comes from per-chunk
// maxima of 64 keys.  A node that no longer fits when it comes up is retired
// for good (side 1 only gets heavier), which leaves the choice among the
// nodes that fit as it is.  The neighbour updates of the nodes a step takes
// are applied after the step, so the step ranks by the gains at its start.
// With no frontier node that fits, the step takes the free node of smallest
// (h32(key(IP, 0, bid), v, t), index) that fits.  Writes the side-1 flags and
// returns the cut.
__device__ long long ip_trial(const EGraph &g, const int32_t *V, const int32_t *cw, const int32_t *Dp,
                              const int32_t *mark, const int32_t *loc, const EBis &b, int t, uint64_t kip,
                              int32_t *conn, uint64_t *key, uint8_t *st, uint64_t *cmax, int32_t *tkn,
                              uint8_t *side) {
  const int lane = (int)lane_id();
  const int nv = b.count, nch = (nv + 63) >> 6;
  const int32_t bid = (int32_t)b.bid;
  for (int j = lane; j < nv; j += 32) { conn[j] = 0; key[j] = 0; st[j] = T_FREE; }
  for (int q = lane; q < nch; q += 32) cmax[q] = 0;
  __syncwarp();
  auto rescan = [&](int ch) {
    const int j0 = ch << 6;
    const uint64_t a0 = j0 + lane < nv ? key[j0 + lane] : 0;
    const uint64_t a1 = j0 + 32 + lane < nv ? key[j0 + 32 + lane] : 0;
    const uint64_t m = wmax64(a0 > a1 ? a0 : a1);
    if (lane == 0) cmax[ch] = m;
    __syncwarp();
  };
  int64_t w1 = 0;
  while (w1 < b.T1) {
    int ntk = 0;
    int64_t taken = 0;
    while (taken < b.B && w1 < b.T1) {
      uint64_t m = 0;
      for (int q = lane; q < nch; q += 32) m = cmax[q] > m ? cmax[q] : m;
      m = wmax64(m);
      if (m == 0) break;
      const int j = (int)(0xFFFFFFFFu - (uint32_t)m);
      const int cj = cw[j];
      const bool fits = w1 + cj <= b.L1;
      if (lane == 0) {
        key[j] = 0;
        st[j] = fits ? T_ONE : T_OUT;
        if (fits) tkn[ntk] = j;
      }
      __syncwarp();
      rescan(j >> 6);
      if (!fits) continue;  // no longer fits (nor ever will)
      ntk++;
      taken++;
      w1 += cj;
    }
    if (taken == 0) {
      unsigned long long fb = ~0ull;
      for (int j = lane; j < nv; j += 32) {
        if (st[j] != T_FREE || w1 + cw[j] > b.L1) continue;
        const unsigned long long h = ((unsigned long long)h32(kip, (uint32_t)V[j], (uint32_t)t) << 32) | (uint32_t)j;
        fb = h < fb ? h : fb;
      }
      fb = wmin64(fb);
      if (fb == ~0ull) break;
      const int j = (int)(uint32_t)fb;
      if (lane == 0) { st[j] = T_ONE; tkn[0] = j; }
      ntk = 1;
      w1 += cw[j];
      __syncwarp();
    }
    // neighbour updates of the nodes taken in this step, then their keys
    for (int q = 0; q < ntk; q++) {
      const int v = V[tkn[q]];
      for (int e = g.xadj[v] + lane; e < g.xadj[v + 1]; e += 32) {
        const int u = g.adjncy[e];
        if (mark[u] == bid) atomicAdd(&conn[loc[u]], g.adjwgt[e]);
      }
    }
    __syncwarp();
    for (int q = 0; q < ntk; q++) {
      const int v = V[tkn[q]];
      for (int e = g.xadj[v] + lane; e < g.xadj[v + 1]; e += 32) {
        const int u = g.adjncy[e];
        if (mark[u] != bid) continue;
        const int lu = loc[u];
        const uint8_t su = st[lu];
        if (su != T_FREE && su != T_FRONT) continue;
        const uint64_t nk = egain_key(2 * (int64_t)conn[lu] - Dp[lu], lu);
        key[lu] = nk;
        st[lu] = T_FRONT;
        atomicMax((unsigned long long *)&cmax[lu >> 6], (unsigned long long)nk);
      }
    }
    __syncwarp();
  }
  long long cut = 0;
  for (int j = lane; j < nv; j += 32) {
    const bool one = st[j] == T_ONE;
    side[j] = one ? 1 : 0;
    if (!one) continue;
    const int v = V[j];
    for (int e = g.xadj[v]; e < g.xadj[v + 1]; e++) {
      const int u = g.adjncy[e];
      if (mark[u] == bid && st[loc[u]] != T_ONE) cut += g.adjwgt[e];
    }
  }
  cut = warp_sum(cut);
  __syncwarp();
  return cut;
}

// Recursive bisection of the coarsest graph (Sec. 4.3, R18), depth by depth:
// the trials of all subproblems of a depth are work items that the warps of
// the CTA take, largest subproblems first; the smallest cut wins (ties:
// lowest trial), and each subproblem splits into side 1 and the rest, in
// list order.
__device__ void e_initial(ECtx &c, const EGraph &g, int k, int64_t eps_ppm, uint64_t seed, int trials,
                          int32_t *blk) {
  ESmem &s = *c.s;
  const int n = g.n;
  const int NW = nwarps();
  const int64_t smark = c.ar.hi;
  int32_t *mark = c.ar.s<int32_t>(n);
  int32_t *loc = c.ar.s<int32_t>(n);
  int32_t *la = c.ar.s<int32_t>(n);
  int32_t *lb = c.ar.s<int32_t>(n);
  int32_t *Dp = c.ar.s<int32_t>(n);
  int32_t *cw = c.ar.s<int32_t>(n);
  ESub *sa = c.ar.s<ESub>(k + 1);
  ESub *sb = c.ar.s<ESub>(k + 1);
  EBis *bis = c.ar.s<EBis>(k + 1);
  int32_t *ord = c.ar.s<int32_t>(k + 1);
  long long *res = c.ar.s<long long>((int64_t)(k + 1) * trials);
  uint8_t *side = c.ar.s<uint8_t>((int64_t)n * trials);
  if (c.ar.fail) return;
  int lg = 0;
  while ((1ll << lg) < k) lg++;
  const int64_t eps_l = eps_ppm / (lg > 0 ? lg : 1);
  for (int v = threadIdx.x; v < n; v += blockDim.x) { la[v] = v; mark[v] = 0; blk[v] = 0; }
  if (threadIdx.x == 0) sa[0] = ESub{0, n, k, 0, 1u, 0};
  __syncthreads();
  int nsubs = 1;
  int32_t *cl = la, *nl = lb;
  ESub *cs = sa, *ns = sb;
  while (nsubs > 0) {
    // leaves take their block; the others are marked and listed for bisection
    if (threadIdx.x == 0) { s.cnt = 0; s.flag = 0; }
    __syncthreads();
    for (int si = 0; si < nsubs; si++) {
      const ESub sub = cs[si];
      const int nv = sub.count;
      const int32_t *V = cl + sub.start;
      if (nv == 0) continue;
      if (sub.kk == 1) {
        for (int j = threadIdx.x; j < nv; j += blockDim.x) blk[V[j]] = sub.b0;
        continue;
      }
      long long Wl = 0;
      for (int j = threadIdx.x; j < nv; j += blockDim.x) {
        const int v = V[j];
        mark[v] = (int32_t)sub.bid;
        loc[v] = j;
        cw[sub.start + j] = g.vwgt[v];
        Wl += g.vwgt[v];
      }
      const int64_t Ws = blk_sum(Wl, s);
      if (threadIdx.x == 0) {
        const int k1 = (sub.kk + 1) / 2;
        EBis x;
        x.start = sub.start; x.count = nv; x.kk = sub.kk; x.b0 = sub.b0; x.bid = sub.bid; x.pad = 0;
        x.T1 = (Ws * k1 + sub.kk - 1) / sub.kk;
        x.L1 = (int64_t)muldiv_u64((uint64_t)x.T1, (uint64_t)(1000000 + eps_l), 1000000ull);
        x.B = 1 + nv / 1024;
        bis[s.cnt] = x;
        s.cnt++;
        s.flag = nv > s.flag ? nv : s.flag;
      }
      __syncthreads();
    }
    const int nb = s.cnt, nvmax = s.flag;
    __syncthreads();
    if (nb == 0) break;
    // deg' inside the subproblem, per list position
    for (int bi = 0; bi < nb; bi++) {
      const EBis b = bis[bi];
      for (int j = warp_idx(); j < b.count; j += NW) {
        const int v = cl[b.start + j];
        long long d = 0;
        for (int e = g.xadj[v] + (int)lane_id(); e < g.xadj[v + 1]; e += 32)
          if (mark[g.adjncy[e]] == (int32_t)b.bid) d += g.adjwgt[e];
        d = warp_sum(d);
        if (lane_id() == 0) Dp[b.start + j] = (int32_t)d;
      }
    }
    // work order: subproblems by size, largest first
    if (threadIdx.x == 0) {
      for (int i = 0; i < nb; i++) {
        int j = i;
        while (j > 0 && bis[ord[j - 1]].count < bis[i].count) { ord[j] = ord[j - 1]; j--; }
        ord[j] = i;
      }
      s.cnt = 0;
    }
    __syncthreads();
    const int items = nb * trials;
    const int slots = items < NW ? items : NW;
    const int64_t dmark = c.ar.hi;
    const int nchmax = (nvmax + 63) >> 6;
    int32_t *conn = c.ar.s<int32_t>((int64_t)slots * nvmax);
    uint64_t *key = c.ar.s<uint64_t>((int64_t)slots * nvmax);
    uint8_t *st = c.ar.s<uint8_t>((int64_t)slots * nvmax);
    uint64_t *cmax = c.ar.s<uint64_t>((int64_t)slots * nchmax);
    int32_t *tkn = c.ar.s<int32_t>((int64_t)slots * (1 + nvmax / 1024));
    if (c.ar.fail) return;
    const int w = warp_idx();
    if (w < slots) {
      for (;;) {
        int it = 0;
        if (lane_id() == 0) it = atomicAdd(&s.cnt, 1);
        it = __shfl_sync(FULL, it, 0);
        if (it >= items) break;
        const int bi = ord[it / trials], t = it % trials;
        const EBis b = bis[bi];
        const uint64_t kip = stream_key(seed, TAG_IP, 0, b.bid);
        const long long cut =
            ip_trial(g, cl + b.start, cw + b.start, Dp + b.start, mark, loc, b, t, kip,
                     conn + (int64_t)w * nvmax, key + (int64_t)w * nvmax, st + (int64_t)w * nvmax,
                     cmax + (int64_t)w * nchmax, tkn + (int64_t)w * (1 + nvmax / 1024),
                     side + (int64_t)t * n + b.start);
        if (lane_id() == 0) res[bi * trials + t] = cut;
      }
    }
    __syncthreads();
    c.ar.hi = dmark;
    // split every subproblem by its best trial: side 1 then the rest, in list order
    if (threadIdx.x == 0) s.cnt = 0;
    __syncthreads();
    for (int bi = 0; bi < nb; bi++) {
      const EBis b = bis[bi];
      int tb = 0;
      for (int t = 1; t < trials; t++)
        if (res[bi * trials + t] < res[bi * trials + tb]) tb = t;
      const uint8_t *win = side + (int64_t)tb * n + b.start;
      auto sidecls = [&](int64_t j) -> int { return win[j] ? 0 : 1; };
      blk_count_classes<2>(b.count, sidecls, 0, s);
      const int n1 = s.tot[0], n2 = s.tot[1];
      __syncthreads();
      if (threadIdx.x == 0) { s.off[0] = 0; s.off[1] = n1; }
      __syncthreads();
      int32_t *tmpl = Dp + b.start;  // list positions; deg' is no longer needed
      blk_classify<2>(b.count, sidecls, tmpl, s);
      for (int j = threadIdx.x; j < b.count; j += blockDim.x) nl[b.start + j] = cl[b.start + tmpl[j]];
      if (threadIdx.x == 0) {
        const int k1 = (b.kk + 1) / 2, k2 = b.kk - k1;
        const int q = s.cnt;
        ns[q] = ESub{b.start, n1, k1, b.b0, 2 * b.bid, 0};
        ns[q + 1] = ESub{b.start + n1, n2, k2, b.b0 + k1, 2 * b.bid + 1, 0};
        s.cnt = q + 2;
      }
      __syncthreads();
    }
    nsubs = s.cnt;
    __syncthreads();
    int32_t *tl = cl; cl = nl; nl = tl;
    ESub *ts = cs; cs = ns; ns = ts;
  }
  c.ar.hi = smark;
  __syncthreads();
}

// R19: while a block exceeds L_max, move from the heaviest block A to the
// lightest block B the node of A that fits and loses the least cut (ties:
// smallest id); stop when nothing fits.
__device__ int64_t e_rebalance(ECtx &c, const EGraph &g, int k, int64_t Lmax, int32_t *blk) {
  ESmem &s = *c.s;
  const int n = g.n;
  const int64_t smark = c.ar.hi;
  long long *bw = c.ar.s<long long>(k);
  if (c.ar.fail) return 0;
  for (int b = threadIdx.x; b < k; b += blockDim.x) bw[b] = 0;
  __syncthreads();
  for (int v = threadIdx.x; v < n; v += blockDim.x) atomicAdd((unsigned long long *)&bw[blk[v]], (unsigned long long)g.vwgt[v]);
  __syncthreads();
  int64_t moves = 0;
  for (int64_t it = 0; it <= (int64_t)n; it++) {
    if (threadIdx.x == 0) {
      int A = 0, Bb = 0;
      for (int b = 1; b < k; b++) {
        if (bw[b] > bw[A]) A = b;
        if (bw[b] < bw[Bb]) Bb = b;
      }
      s.off[0] = A; s.off[1] = Bb;
      s.flag = (bw[A] <= Lmax || A == Bb) ? 1 : 0;
    }
    __syncthreads();
    const int A = s.off[0], Bb = s.off[1];
    if (s.flag) break;
    const long long bwB = bw[Bb];
    unsigned long long best = ~0ull;
    for (int v = threadIdx.x; v < n; v += blockDim.x) {
      if (blk[v] != A || bwB + g.vwgt[v] > Lmax) continue;
      long long ca = 0, cb = 0;
      for (int e = g.xadj[v]; e < g.xadj[v + 1]; e++) {
        const int b = blk[g.adjncy[e]];
        if (b == A) ca += g.adjwgt[e];
        else if (b == Bb) cb += g.adjwgt[e];
      }
      const unsigned long long key = ((unsigned long long)(ca - cb + 2147483648ll) << 32) | (uint32_t)v;
      best = key < best ? key : best;
    }
    best = blk_min_u64(best, s);
    if (best == ~0ull) break;
    if (threadIdx.x == 0) {
      const int v = (int)(uint32_t)best;
      blk[v] = Bb;
      bw[A] -= g.vwgt[v];
      bw[Bb] += g.vwgt[v];
    }
    moves++;
    __syncthreads();
  }
  c.ar.hi = smark;
  __syncthreads();
  return moves;
}

// cut = 1/2 sum over entries whose endpoints lie in different blocks
__device__ int64_t e_cut(ECtx &c, const EGraph &g, const int32_t *blk) {
  long long s = 0;
  blk_for_entries(g.xadj, g.n, [&](int u, int e) {
    if (blk[g.adjncy[e]] != blk[u]) s += g.adjwgt[e];
  });
  return blk_sum(s, *c.s) / 2;
}

// LP refinement of the blocks of g (Sec. 3, Sec. 4.3; R20).
__device__ void e_refine(ECtx &c, const EGraph &g, int k, int64_t Lmax, int level, uint64_t seed, int32_t *blk,
                         int32_t *bw, ELpScr &L) {
  const gp_config &cfg = *c.cfg;
  if (g.n == 0 || k <= 1 || cfg.ref_rounds <= 0) return;
  fill_i32(bw, k, 0);
  __syncthreads();
  for (int v = threadIdx.x; v < g.n; v += blockDim.x) atomicAdd(&bw[blk[v]], g.vwgt[v]);
  __syncthreads();
  ELp P;
  P.tag_act = TAG_RACT; P.tag_tie = TAG_RTIE; P.tag_prio = TAG_RPRIO;
  P.level = level; P.rounds = cfg.ref_rounds; P.S = cfg.lp_subrounds; P.dbg = -1;
  P.bound = Lmax; P.n_min = 0; P.count = false;
  int64_t ncl = 0, moves = 0;
  int subs = 0;
  e_lp(c, g, blk, bw, k, seed, P, L, ncl, subs, moves);
}

__device__ int e_maxdeg(ECtx &c, const EGraph &g) {
  long long d = 0;
  for (int v = threadIdx.x; v < g.n; v += blockDim.x) d = max(d, (long long)(g.xadj[v + 1] - g.xadj[v]));
  return (int)blk_max(d, *c.s);
}

// ------------------------------------------------------------ one item

struct ELevel {
  EGraph g;
  int32_t *cmap;
};

__device__ void e_item(ECtx &c, const EItem &it, EOut &o, gp_level_stats *lvo, ELevel *lv) {
  const gp_config &cfg = *c.cfg;
  const EGraph in{it.xadj, it.adjncy, it.vwgt, it.adjwgt, it.n, it.m2};
  int64_t W, cmax;
  c.cyc = o.cyc;
  c.t0 = clock64();
  int st = e_validate(c, in, cfg.validate != 0, W, cmax);
  phase(c, EP_VALIDATE);
  if (st != GP_OK) { o.status = st; return; }
  const int64_t Lmax = lmax_of_dev(W, it.k, it.eps_ppm);
  if (cmax > Lmax) { o.status = GP_ERR_INFEASIBLE; return; }
  o.W = W;
  o.Lmax = Lmax;
  const int n = it.n;
  const int k = it.k;
  if (k == 1 || n == 0) {
    for (int v = threadIdx.x; v < n; v += blockDim.x) it.blocks[v] = 0;
    o.cut = 0;
    o.n_coarsest = n;
    o.status = GP_OK;
    return;
  }
  const int64_t U = max((int64_t)1, W / ((int64_t)cfg.cluster_factor * k));
  o.U = U;
  if (threadIdx.x == 0) {
    lv[0].g = in;
    lv[0].cmap = nullptr;
  }
  __syncthreads();
  int L = 0;
  const int maxl = cfg.max_levels < GP_MAX_LEVELS ? cfg.max_levels : GP_MAX_LEVELS;
  while ((int64_t)lv[L].g.n > (int64_t)cfg.coarsest_factor * k && L < maxl) {
    const EGraph cur = lv[L].g;
    const int64_t hmark = c.ar.lo;
    int32_t *cmap = c.ar.h<int32_t>(cur.n);
    const int64_t smark = c.ar.hi;
    int32_t *label = c.ar.s<int32_t>(cur.n);
    if (c.ar.fail) { o.status = kERetry; return; }
    const int maxdeg = e_maxdeg(c, cur);
    ECluster cl{};
    e_cluster(c, cur, U, L + 1, it.seed, label, maxdeg, cl);
    phase(c, EP_CLUSTER);
    if (c.ar.fail) { o.status = kERetry; return; }
    const int nc = e_relabel(c, cur.n, label, cmap);
    c.ar.hi = smark;
    phase(c, EP_RELABEL);
    if (c.ar.fail) { o.status = kERetry; return; }
    EGraph gc{};
    e_contract(c, cur, cmap, nc, gc);
    phase(c, EP_CONTRACT);
    if (c.ar.fail) { o.status = kERetry; return; }
    gp_level_stats ls{};
    ls.n = cur.n;
    ls.n_next = nc;
    ls.m = cur.m2 / 2;
    ls.m_coarse = gc.m2 / 2;
    ls.lp_subrounds = cl.subs;
    ls.lp_moves = cl.moves;
    ls.clusters_lp = cl.ncl_lp;
    ls.clusters_2hop = cl.ncl_2hop;
    ls.clusters_final = cl.ncl_final;
    if ((int64_t)nc * cfg.min_shrink_num > (int64_t)cur.n * cfg.min_shrink_den) {
      c.ar.lo = hmark;
      break;
    }
    const int64_t a = (int64_t)muldiv_u64((uint64_t)ls.m, (uint64_t)cfg.tau_e_num, (uint64_t)cfg.tau_e_den);
    const int64_t b = (int64_t)muldiv_u64((uint64_t)ls.m * (uint64_t)nc, (uint64_t)cfg.tau_d_num,
                                          (uint64_t)cfg.tau_d_den * (uint64_t)cur.n);
    ls.m_hat = a < b ? a : b;
    ls.triggered = cfg.sparsifier != GP_SPARSIFY_NONE &&
                   (uint64_t)ls.m_coarse * (uint64_t)cfg.rho_den > (uint64_t)cfg.rho_num * (uint64_t)ls.m_hat;
    if (ls.triggered) {
      e_sparsify(c, gc, ls.m_hat, L + 2, it.seed, cfg.sparsifier, ls);
      phase(c, EP_SPARSIFY);
      if (c.ar.fail) { o.status = kERetry; return; }
    }
    ls.m_next = gc.m2 / 2;
    if (threadIdx.x == 0) {
      if (lvo) lvo[L] = ls;
      lv[L].cmap = cmap;
      lv[L + 1].g = gc;
      lv[L + 1].cmap = nullptr;
    }
    L++;
    __syncthreads();
  }
  o.levels = L;
  o.n_coarsest = lv[L].g.n;
  // buffers of the uncoarsening: block ids per level (two alternating), LP scratch for the largest level
  int nmax = 0, dmax = 0;
  for (int i = 1; i <= L; i++) nmax = lv[i].g.n > nmax ? lv[i].g.n : nmax;
  for (int i = 0; i <= L; i++) {
    const int d = e_maxdeg(c, lv[i].g);
    dmax = d > dmax ? d : dmax;
  }
  int32_t *ba = c.ar.s<int32_t>(nmax > 0 ? nmax : 1);
  int32_t *bb = c.ar.s<int32_t>(nmax > 0 ? nmax : 1);
  int32_t *bw = c.ar.s<int32_t>(k);
  if (c.ar.fail) { o.status = kERetry; return; }
  int32_t *blk = L == 0 ? it.blocks : ba;
  const EGraph &gco = lv[L].g;
  e_initial(c, gco, k, it.eps_ppm, it.seed, cfg.ip_trials, blk);
  if (c.ar.fail) { o.status = kERetry; return; }
  o.ip_cut = e_cut(c, gco, blk);
  o.rebalance_moves = e_rebalance(c, gco, k, Lmax, blk);
  phase(c, EP_INITIAL);
  ELpScr LS;
  lp_scratch(c, n, k, dmax, LS);
  if (c.ar.fail) { o.status = kERetry; return; }
  lp_scratch_clear(LS);
  __syncthreads();
  e_refine(c, gco, k, Lmax, L + 1, it.seed, blk, bw, LS);
  for (int i = L - 1; i >= 0; i--) {
    int32_t *fine = i == 0 ? it.blocks : (blk == ba ? bb : ba);
    const int32_t *cm = lv[i].cmap;
    for (int v = threadIdx.x; v < lv[i].g.n; v += blockDim.x) fine[v] = blk[cm[v]];
    __syncthreads();
    e_refine(c, lv[i].g, k, Lmax, i + 1, it.seed, fine, bw, LS);
    blk = fine;
  }
  phase(c, EP_REFINE);
  o.cut = e_cut(c, in, it.blocks);
  phase(c, EP_CUT);
  o.status = GP_OK;
}

template <int NT>
__global__ void __launch_bounds__(NT) k_engine(EArgs a) {
  extern __shared__ __align__(16) unsigned char esm[];
  __shared__ ESmem s;
  __shared__ ELevel lv[GP_MAX_LEVELS + 1];
  __shared__ int s_item;
  const int nw = nwarps();
  ECtx c;
  c.s = &s;
  c.cfg = &a.cfg;
  c.prof = a.profile != 0;
  c.wtk = reinterpret_cast<int *>(esm);
  c.wtv = c.wtk + nw * kEWarpSlots;
  c.btk = c.wtv + nw * kEWarpSlots;
  c.btv = c.btk + kEBlockSlots;
  for (int t = threadIdx.x; t < nw * kEWarpSlots; t += blockDim.x) { c.wtk[t] = -1; c.wtv[t] = 0; }
  for (int t = threadIdx.x; t < kEBlockSlots; t += blockDim.x) { c.btk[t] = -1; c.btv[t] = 0; }
  __syncthreads();
  for (;;) {
    if (threadIdx.x == 0) s_item = atomicAdd(a.head, 1);
    __syncthreads();
    const int q = s_item;
    __syncthreads();
    if (q >= a.count) break;
    const int idx = a.order[q];
    c.ar.base = a.arena + (int64_t)blockIdx.x * a.arena_bytes;
    c.ar.lo = 0;
    c.ar.hi = a.arena_bytes;
    c.ar.fail = false;
    EOut o{};
    o.status = GP_ERR_CUDA;
    e_item(c, a.items[idx], o, a.lv ? a.lv + (int64_t)idx * GP_MAX_LEVELS : nullptr, lv);
    if (threadIdx.x == 0) a.out[idx] = o;
    // the shared tables are left empty by every phase; the sort's counters reuse them
    for (int t = threadIdx.x; t < kEBlockSlots; t += blockDim.x) { c.btk[t] = -1; c.btv[t] = 0; }
    __syncthreads();
  }
}

}  // namespace
}  // namespace gp

