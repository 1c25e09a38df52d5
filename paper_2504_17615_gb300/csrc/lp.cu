// lp.cu -- size-constrained label propagation (Sec. 3 of the paper; the
// clustering of Sec. 4.1 and the refinement of Sec. 4.3) as synchronous
// sub-rounds with hash priorities:
//
//  per round r: nodes with neighbours are bucketed by (sub-round, degree
//  class); per sub-round s:
//   rate   : every active node sums the edge weight to each neighbouring
//            label on the snapshot and picks the admissible label of largest
//            rating (ties: smallest h32(TIE), then smallest label); it
//            proposes when that beats its own label's rating
//   decide : a target whose snapshot weight plus all incoming weight fits
//            the bound accepts everybody; the proposers of overflowing
//            targets are sorted by (target, h32(PRIO), node) and accepted
//            while the running weight fits (longest prefix)
//   apply  : labels and weights are updated; the non-empty clusters (the
//            labels of positive weight) are counted; the stop flag is raised
//            when that count reaches n_min or a round moved nothing.
#include "lp.cuh"

#include <chrono>

namespace gp {

namespace {

constexpr unsigned FULL = 0xFFFFFFFFu;
constexpr int kMedSlots = 256;
constexpr int kThreads = 256;
constexpr int kWarpsPerBlock = kThreads / 32;
constexpr int kMaxKeys = 64 * kNumBuckets;

struct RateArgs {
  const int32_t *xadj, *adjncy, *adjwgt, *vwgt, *label, *weight;
  const uint8_t *label8;  // optional narrow copy of label (fewer than 256 labels) for gathers
  const int4 *list;     // bucket list: (node, row offset, degree, node weight)
  const int32_t *offs;
  int key;
  int64_t bound;
  uint64_t ktie;
  int2 *prop;           // RATE_LP: per list position (proposed label or -1, own label)
  int32_t *incoming;    // RATE_LP: per label incoming weight
  uint64_t *fav_keys;   // RATE_FAV: per list position (fav << 32 | v)
  const int *stop;
  int32_t *gkeys, *gvals;  // large kernel global tables
  int64_t gstride;
  unsigned long long *units;
  int wlabels;          // labels whose weights a launch may copy to shared memory (<= 256)
  uint8_t *dirty;       // optional: per node, 0 = cannot move until a neighbour moves (rating skipped)
  const int32_t *ccount;  // optional: the list holds ccount[key] records from offs[key] (compacted)
};

__device__ __forceinline__ int list_end(const RateArgs &a) {
  return a.ccount ? a.offs[a.key] + a.ccount[a.key] : a.offs[a.key + 1];
}

__device__ __forceinline__ void add_units(unsigned long long *units, unsigned long long e,
                                          unsigned long long v, unsigned long long c,
                                          unsigned long long p, bool narrow, bool implied) {
  if (!units) return;
  e = warp_sum(e); v = warp_sum(v); c = warp_sum(c); p = warp_sum(p);
  if (lane_id() == 0) {
    if (e) atomicAdd(units + 0, e);
    if (e && narrow) atomicAdd(units + 4, e);
    if (e && implied) atomicAdd(units + 5, e);
    if (v) atomicAdd(units + 1, v);
    if (c) atomicAdd(units + 2, c);
    if (p) atomicAdd(units + 3, p);
  }
}

__device__ __forceinline__ int label_of(const RateArgs &a, int u) {
  return a.label8 ? (int)a.label8[u] : a.label[u];
}

__device__ __forceinline__ unsigned slot_hash(int L, int bits) {
  return ((unsigned)L * 2654435761u) >> (32 - bits);
}

template <int MODE>
__device__ __forceinline__ void emit(const RateArgs &a, int i, int v, int best, int cv, int own) {
  if (MODE == RATE_LP) {
    a.prop[i] = make_int2(best, own);
    atomicAdd(&a.incoming[best], cv);
  } else {
    a.fav_keys[i] = ((uint64_t)(uint32_t)best << 32) | (uint32_t)v;
  }
}

// ------------------------------------- degree <= 32: G lanes per node
//
// A warp rates 32/G nodes side by side (one neighbour per lane of a G-lane
// group) and keeps U such sets in flight, issuing the loads of all U*32/G
// nodes phase by phase (offsets, neighbours, labels) so that independent
// dependency chains overlap.  Equal labels within a group are summed in a
// 2G-slot shared-memory table per group (the first lane to claim a slot is
// the label's leader).  The choice is lazy in the label weights: candidates
// are ranked by (rating, tie hash, label) without the bound, and only the
// leading candidate's weight is fetched; if it does not fit, it is dropped
// and the next one is tried.  This picks exactly the best admissible
// candidate while reading one label weight per node in the usual case, and
// none at all when no neighbouring label beats the node's own label.  With
// one-byte labels (refinement: at most 255 labels) the label weights are
// copied to shared memory once per launch and every candidate is checked
// against the bound up front, so the first pass already picks the best
// admissible label.

// Label kinds: LK_WIDE int32 labels summed in hash tables; LK_NARROW uint8
// labels (fewer than 256) in hash tables; LK_DENSE uint8 labels below
// kDenseLabels summed in a dense per-group array indexed by label.
enum LabelKind { LK_WIDE = 0, LK_NARROW = 1, LK_DENSE = 2 };
constexpr int kDenseLabels = 128;

template <int MODE, int G, int U, int LK>
__global__ void __launch_bounds__(kThreads, G == 32 ? 4 : 5) k_rate_group(RateArgs a) {
  static_assert(G == 8 || G == 16 || G == 32, "group width");
  constexpr int NV = 32 / G;
  constexpr int PER = NV * U;
  constexpr int TS = 2 * G;  // hash-table slots per group
  constexpr int TW = LK == LK_DENSE ? U * NV * kDenseLabels : U * 64;  // table words per warp
  __shared__ int s_tk[LK == LK_DENSE ? 1 : kWarpsPerBlock][LK == LK_DENSE ? 1 : U * 64];
  __shared__ int s_tv[kWarpsPerBlock][TW];
  constexpr bool kSmemW = MODE == RATE_LP && LK != LK_WIDE;
  __shared__ int s_w[kSmemW ? 256 : 1];
  if (a.stop && *a.stop) return;
  if (kSmemW) {
    for (int t = threadIdx.x; t < a.wlabels; t += blockDim.x) s_w[t] = a.weight[t];
    __syncthreads();
  }
  const int lane = (int)lane_id(), wib = threadIdx.x >> 5;
  const int grp = lane / G, gl = lane % G;
  const unsigned gmask = G == 32 ? FULL : (((1u << G) - 1u) << (grp * G));
  for (int t = lane; t < TW; t += 32) {
    if (LK != LK_DENSE) s_tk[wib][t] = -1;
    s_tv[wib][t] = 0;
  }
  __syncwarp();
  const int begin = a.offs[a.key], end = list_end(a);
  const int wid = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5);
  const int nw = (int)((gridDim.x * blockDim.x) >> 5);
  unsigned long long ue = 0, uv = 0, uc = 0, up = 0;
  for (int base = begin + wid * PER; base < end; base += nw * PER) {
    int v[U], st[U], deg[U], own[U], cv[U], L[U], w[U], u[U];
    bool skip[U];
#pragma unroll
    for (int q = 0; q < U; q++) {
      const int i = base + q * NV + grp;
      const int4 rec = i < end ? a.list[i] : make_int4(-1, 0, 0, 0);
      v[q] = rec.x; st[q] = rec.y; deg[q] = rec.z; cv[q] = rec.w;
    }
#pragma unroll
    for (int q = 0; q < U; q++) {
      // a clean node cannot move: neither its neighbours' labels nor its own changed since it
      // last found no label rated above its own
      skip[q] = a.dirty && v[q] >= 0 && !a.dirty[v[q]];
      if (skip[q]) { v[q] = -1; deg[q] = 0; }
    }
#pragma unroll
    for (int q = 0; q < U; q++) {
      const bool ok = v[q] >= 0;
      own[q] = ok ? (LK == LK_WIDE ? a.label[v[q]] : (int)a.label8[v[q]]) : -2;
    }
#pragma unroll
    for (int q = 0; q < U; q++) {
      const bool ok = gl < deg[q];
      u[q] = ok ? __ldcs(a.adjncy + st[q] + gl) : -1;  // rows are read once a round: evict first
      w[q] = ok ? (a.adjwgt ? __ldcs(a.adjwgt + st[q] + gl) : 1) : 0;
    }
#pragma unroll
    for (int q = 0; q < U; q++)
      L[q] = u[q] >= 0 ? (LK == LK_WIDE ? a.label[u[q]] : (int)a.label8[u[q]]) : -1;
    // sum equal labels per group in shared memory
    int slot[U], own_r[U], sum[U];
    bool lead[U];
    if (LK == LK_DENSE) {
#pragma unroll
      for (int q = 0; q < U; q++) {
        slot[q] = (q * NV + grp) * kDenseLabels;
        if (u[q] >= 0) atomicAdd(&s_tv[wib][slot[q] + L[q]], w[q]);
      }
      __syncwarp();
#pragma unroll
      for (int q = 0; q < U; q++) {
        sum[q] = u[q] >= 0 ? s_tv[wib][slot[q] + L[q]] : 0;
        own_r[q] = v[q] >= 0 ? s_tv[wib][slot[q] + own[q]] : 0;
        lead[q] = u[q] >= 0;  // duplicates of a label are harmless below
      }
      __syncwarp();
#pragma unroll
      for (int q = 0; q < U; q++)
        if (u[q] >= 0) s_tv[wib][slot[q] + L[q]] = 0;
      __syncwarp();
    } else {
#pragma unroll
      for (int q = 0; q < U; q++) {
        int *tk = &s_tk[wib][q * 64 + grp * TS];
        slot[q] = -1;
        lead[q] = false;
        if (u[q] >= 0) {
          unsigned sl = ((unsigned)L[q] * 2654435761u) >> (32 - (G == 8 ? 4 : G == 16 ? 5 : 6));
          for (int p = 0; p < TS; p++) {  // bounded: a group has at most G labels in 2G slots
            const int prev = atomicCAS(&tk[sl], -1, L[q]);
            if (prev == -1) { lead[q] = true; break; }
            if (prev == L[q]) break;
            sl = (sl + 1) & (TS - 1);
          }
          slot[q] = q * 64 + grp * TS + (int)sl;
          atomicAdd(&s_tv[wib][slot[q]], w[q]);
        }
      }
      __syncwarp();
#pragma unroll
      for (int q = 0; q < U; q++) sum[q] = slot[q] >= 0 ? s_tv[wib][slot[q]] : 0;
      __syncwarp();
#pragma unroll
      for (int q = 0; q < U; q++)
        if (lead[q]) { s_tk[wib][slot[q]] = -1; s_tv[wib][slot[q]] = 0; }
      __syncwarp();
#pragma unroll
      for (int q = 0; q < U; q++)
        own_r[q] = __reduce_max_sync(gmask, (lead[q] && L[q] == own[q]) ? sum[q] : 0);
    }
    // choose: all U sets advance together, so that the weight reads of their
    // leading candidates are issued side by side.  When a group's leading
    // candidate does not fit, the weights of all its remaining candidates are
    // read at once on the next pass and the inadmissible ones dropped, so a
    // node takes at most three passes.
    bool alive[U], searching[U], eager[U];
    unsigned best[U];
    // no label rated above the own one, admissible or not: the node proposes nothing (so it skips
    // the choice), and in refinement it stays clean until a neighbour moves
    bool stay[U];
#pragma unroll
    for (int q = 0; q < U; q++) {
      const int rall = (int)__reduce_max_sync(gmask, (lead[q] && L[q] != own[q]) ? (unsigned)sum[q] : 0u);
      stay[q] = MODE == RATE_LP && rall <= own_r[q];
      if (a.dirty && gl == 0 && v[q] >= 0 && stay[q]) a.dirty[v[q]] = 0;
    }
#pragma unroll
    for (int q = 0; q < U; q++) {
      alive[q] = lead[q] && L[q] != own[q];
      uc += alive[q];
      if (kSmemW && alive[q]) alive[q] = (int64_t)s_w[L[q]] + cv[q] <= a.bound;
      searching[q] = v[q] >= 0 && !stay[q];
      eager[q] = kSmemW;
      best[q] = 0xFFFFFFFFu;
    }
    for (int it = 0; it <= G; it++) {  // bounded: every pass drops one candidate per searching group
      bool any = false;
#pragma unroll
      for (int q = 0; q < U; q++) any = any || searching[q];
      if (!__any_sync(FULL, any)) break;
      if (MODE == RATE_LP && !kSmemW) {
        int we[U];
#pragma unroll
        for (int q = 0; q < U; q++) we[q] = (eager[q] && searching[q] && alive[q]) ? a.weight[L[q]] : 0;
#pragma unroll
        for (int q = 0; q < U; q++)
          if (eager[q] && searching[q] && alive[q] && (int64_t)we[q] + cv[q] > a.bound) alive[q] = false;
      }
      unsigned c[U];
      bool holder[U];
#pragma unroll
      for (int q = 0; q < U; q++) {
        const int r = __reduce_max_sync(gmask, (searching[q] && alive[q]) ? sum[q] : -1);
        if (r < 0 || (MODE == RATE_LP && r <= own_r[q])) searching[q] = false;
        const bool top = searching[q] && alive[q] && sum[q] == r;
        const unsigned h = top ? h32(a.ktie, (uint32_t)v[q], (uint32_t)L[q]) : 0xFFFFFFFFu;
        const unsigned hmin = __reduce_min_sync(gmask, h);
        c[q] = __reduce_min_sync(gmask, (top && h == hmin) ? (unsigned)L[q] : 0xFFFFFFFFu);
        holder[q] = top && h == hmin && (unsigned)L[q] == c[q];
      }
      if (MODE != RATE_LP || kSmemW) {
#pragma unroll
        for (int q = 0; q < U; q++)
          if (searching[q]) { best[q] = c[q]; searching[q] = false; }
      } else {
        int wc[U];
#pragma unroll
        for (int q = 0; q < U; q++) wc[q] = (holder[q] && !eager[q]) ? a.weight[c[q]] : 0;
#pragma unroll
        for (int q = 0; q < U; q++) {
          // after an eager pass every remaining candidate fits
          const unsigned fits = holder[q] && (eager[q] || (int64_t)wc[q] + cv[q] <= a.bound) ? 1u : 0u;
          if (__reduce_or_sync(gmask, fits) && searching[q]) { best[q] = c[q]; searching[q] = false; }
          alive[q] = alive[q] && (unsigned)L[q] != c[q];
          eager[q] = true;
        }
      }
    }
#pragma unroll
    for (int q = 0; q < U; q++) {
      if (gl == 0 && v[q] >= 0) {
        ue += deg[q];
        uv += 1;
        if (best[q] != 0xFFFFFFFFu) {
          emit<MODE>(a, base + q * NV + grp, v[q], (int)best[q], cv[q], own[q]);
          up += 1;
        } else if (MODE == RATE_LP) {
          a.prop[base + q * NV + grp] = make_int2(-1, 0);
        }
      } else if (gl == 0 && skip[q] && MODE == RATE_LP) {
        a.prop[base + q * NV + grp] = make_int2(-1, 0);
      }
    }
  }
  add_units(a.units, ue, uv, uc, up, a.label8 != nullptr, a.adjwgt == nullptr);
}

// ----------------- degree <= 32 with E entries per lane: G lanes per node
//
// The same rating and choice as k_rate_group, with every lane of a G-lane group
// holding up to E neighbours, so that a warp rates 32/G nodes of degree up to
// G * E side by side and every group-wide reduction of the choice serves 32/G
// nodes at once (nodes of degree 9-32 on 8 or 16 lanes instead of a whole warp).
template <int MODE, int G, int E, int U, int LK>
__global__ void __launch_bounds__(kThreads, 4) k_rate_multi(RateArgs a) {
  static_assert(G == 8 || G == 16, "group width");
  constexpr int NV = 32 / G;
  constexpr int PER = NV * U;
  constexpr int TS = 2 * G * E;  // hash-table slots per (set, group)
  constexpr int TBITS = TS == 32 ? 5 : TS == 64 ? 6 : 7;
  static_assert((1 << TBITS) == TS, "table size");
  constexpr int TW = LK == LK_DENSE ? U * NV * kDenseLabels : U * NV * TS;  // table words per warp
  __shared__ int s_tk[LK == LK_DENSE ? 1 : kWarpsPerBlock][LK == LK_DENSE ? 1 : TW];
  __shared__ int s_tv[kWarpsPerBlock][TW];
  constexpr bool kSmemW = MODE == RATE_LP && LK != LK_WIDE;
  __shared__ int s_w[kSmemW ? 256 : 1];
  if (a.stop && *a.stop) return;
  if (kSmemW) {
    for (int t = threadIdx.x; t < a.wlabels; t += blockDim.x) s_w[t] = a.weight[t];
    __syncthreads();
  }
  const int lane = (int)lane_id(), wib = threadIdx.x >> 5;
  const int grp = lane / G, gl = lane % G;
  const unsigned gmask = ((1u << G) - 1u) << (grp * G);
  for (int t = lane; t < TW; t += 32) {
    if (LK != LK_DENSE) s_tk[wib][t] = -1;
    s_tv[wib][t] = 0;
  }
  __syncwarp();
  const int begin = a.offs[a.key], end = list_end(a);
  const int wid = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5);
  const int nw = (int)((gridDim.x * blockDim.x) >> 5);
  unsigned long long ue = 0, uv = 0, uc = 0, up = 0;
  for (int base = begin + wid * PER; base < end; base += nw * PER) {
    int v[U], st[U], deg[U], own[U], cv[U];
    int L[U][E], w[U][E], u[U][E];
    bool skip[U];
#pragma unroll
    for (int q = 0; q < U; q++) {
      const int i = base + q * NV + grp;
      const int4 rec = i < end ? a.list[i] : make_int4(-1, 0, 0, 0);
      v[q] = rec.x; st[q] = rec.y; deg[q] = rec.z; cv[q] = rec.w;
    }
#pragma unroll
    for (int q = 0; q < U; q++) {
      skip[q] = a.dirty && v[q] >= 0 && !a.dirty[v[q]];
      if (skip[q]) { v[q] = -1; deg[q] = 0; }
    }
#pragma unroll
    for (int q = 0; q < U; q++) {
      const bool ok = v[q] >= 0;
      own[q] = ok ? (LK == LK_WIDE ? a.label[v[q]] : (int)a.label8[v[q]]) : -2;
    }
#pragma unroll
    for (int q = 0; q < U; q++)
#pragma unroll
      for (int e = 0; e < E; e++) {
        const int j = gl + e * G;
        const bool ok = j < deg[q];
        u[q][e] = ok ? __ldcs(a.adjncy + st[q] + j) : -1;  // rows are read once a round: evict first
        w[q][e] = ok ? (a.adjwgt ? __ldcs(a.adjwgt + st[q] + j) : 1) : 0;
      }
#pragma unroll
    for (int q = 0; q < U; q++)
#pragma unroll
      for (int e = 0; e < E; e++)
        L[q][e] = u[q][e] >= 0 ? (LK == LK_WIDE ? a.label[u[q][e]] : (int)a.label8[u[q][e]]) : -1;
    int own_r[U], sum[U][E];
    bool lead[U][E];
    if (LK == LK_DENSE) {
#pragma unroll
      for (int q = 0; q < U; q++) {
        const int sb = (q * NV + grp) * kDenseLabels;
#pragma unroll
        for (int e = 0; e < E; e++)
          if (u[q][e] >= 0) atomicAdd(&s_tv[wib][sb + L[q][e]], w[q][e]);
      }
      __syncwarp();
#pragma unroll
      for (int q = 0; q < U; q++) {
        const int sb = (q * NV + grp) * kDenseLabels;
        own_r[q] = v[q] >= 0 ? s_tv[wib][sb + own[q]] : 0;
#pragma unroll
        for (int e = 0; e < E; e++) {
          sum[q][e] = u[q][e] >= 0 ? s_tv[wib][sb + L[q][e]] : 0;
          lead[q][e] = u[q][e] >= 0;  // duplicates of a label are harmless below
        }
      }
      __syncwarp();
#pragma unroll
      for (int q = 0; q < U; q++) {
        const int sb = (q * NV + grp) * kDenseLabels;
#pragma unroll
        for (int e = 0; e < E; e++)
          if (u[q][e] >= 0) s_tv[wib][sb + L[q][e]] = 0;
      }
      __syncwarp();
    } else {
      int slot[U][E];
#pragma unroll
      for (int q = 0; q < U; q++) {
        const int sb = (q * NV + grp) * TS;
        int *tk = &s_tk[wib][sb];
#pragma unroll
        for (int e = 0; e < E; e++) {
          slot[q][e] = -1;
          lead[q][e] = false;
          if (u[q][e] < 0) continue;
          unsigned sl = ((unsigned)L[q][e] * 2654435761u) >> (32 - TBITS);
          for (int p = 0; p < TS; p++) {  // bounded: a group holds at most G E labels in 2 G E slots
            const int prev = atomicCAS(&tk[sl], -1, L[q][e]);
            if (prev == -1) { lead[q][e] = true; break; }
            if (prev == L[q][e]) break;
            sl = (sl + 1) & (TS - 1);
          }
          slot[q][e] = sb + (int)sl;
          atomicAdd(&s_tv[wib][slot[q][e]], w[q][e]);
        }
      }
      __syncwarp();
#pragma unroll
      for (int q = 0; q < U; q++)
#pragma unroll
        for (int e = 0; e < E; e++) sum[q][e] = slot[q][e] >= 0 ? s_tv[wib][slot[q][e]] : 0;
      __syncwarp();
#pragma unroll
      for (int q = 0; q < U; q++)
#pragma unroll
        for (int e = 0; e < E; e++)
          if (lead[q][e]) { s_tk[wib][slot[q][e]] = -1; s_tv[wib][slot[q][e]] = 0; }
      __syncwarp();
#pragma unroll
      for (int q = 0; q < U; q++) {
        unsigned o = 0;
#pragma unroll
        for (int e = 0; e < E; e++)
          if (lead[q][e] && L[q][e] == own[q]) o = max(o, (unsigned)sum[q][e]);
        own_r[q] = (int)__reduce_max_sync(gmask, o);
      }
    }
    // choose (as k_rate_group): all U sets advance together; a group whose leading candidate does
    // not fit reads the weights of all its remaining candidates on the next pass
    bool alive[U][E], searching[U], eager[U];
    unsigned best[U];
    // no label rated above the own one, admissible or not: the node proposes nothing (so it skips
    // the choice), and in refinement it stays clean until a neighbour moves
    bool stay[U];
#pragma unroll
    for (int q = 0; q < U; q++) {
      unsigned ra = 0;
#pragma unroll
      for (int e = 0; e < E; e++)
        if (lead[q][e] && L[q][e] != own[q]) ra = max(ra, (unsigned)sum[q][e]);
      const int rall = (int)__reduce_max_sync(gmask, ra);
      stay[q] = MODE == RATE_LP && rall <= own_r[q];
      if (a.dirty && gl == 0 && v[q] >= 0 && stay[q]) a.dirty[v[q]] = 0;
    }
#pragma unroll
    for (int q = 0; q < U; q++) {
#pragma unroll
      for (int e = 0; e < E; e++) {
        alive[q][e] = lead[q][e] && L[q][e] != own[q];
        uc += alive[q][e];
        if (kSmemW && alive[q][e]) alive[q][e] = (int64_t)s_w[L[q][e]] + cv[q] <= a.bound;
      }
      searching[q] = v[q] >= 0 && !stay[q];
      eager[q] = kSmemW;
      best[q] = 0xFFFFFFFFu;
    }
    for (int it = 0; it <= G * E; it++) {  // bounded: every pass drops one candidate per searching group
      bool any = false;
#pragma unroll
      for (int q = 0; q < U; q++) any = any || searching[q];
      if (!__any_sync(FULL, any)) break;
      if (MODE == RATE_LP && !kSmemW) {
#pragma unroll
        for (int q = 0; q < U; q++)
#pragma unroll
          for (int e = 0; e < E; e++)
            if (eager[q] && searching[q] && alive[q][e] && (int64_t)a.weight[L[q][e]] + cv[q] > a.bound)
              alive[q][e] = false;
      }
      unsigned c[U];
      bool holder[U];
#pragma unroll
      for (int q = 0; q < U; q++) {
        int rl = -1;
#pragma unroll
        for (int e = 0; e < E; e++)
          if (searching[q] && alive[q][e]) rl = max(rl, sum[q][e]);
        const int r = __reduce_max_sync(gmask, rl);
        if (r < 0 || (MODE == RATE_LP && r <= own_r[q])) searching[q] = false;
        unsigned h[E], hl = 0xFFFFFFFFu;
#pragma unroll
        for (int e = 0; e < E; e++) {
          const bool top = searching[q] && alive[q][e] && sum[q][e] == r;
          h[e] = top ? h32(a.ktie, (uint32_t)v[q], (uint32_t)L[q][e]) : 0xFFFFFFFFu;
          hl = min(hl, h[e]);
        }
        const unsigned hmin = __reduce_min_sync(gmask, hl);
        unsigned cl = 0xFFFFFFFFu;
#pragma unroll
        for (int e = 0; e < E; e++)
          if (searching[q] && alive[q][e] && sum[q][e] == r && h[e] == hmin) cl = min(cl, (unsigned)L[q][e]);
        c[q] = __reduce_min_sync(gmask, cl);
        holder[q] = false;
#pragma unroll
        for (int e = 0; e < E; e++)
          holder[q] = holder[q] || (searching[q] && alive[q][e] && sum[q][e] == r && h[e] == hmin &&
                                    (unsigned)L[q][e] == c[q]);
      }
      if (MODE != RATE_LP || kSmemW) {
#pragma unroll
        for (int q = 0; q < U; q++)
          if (searching[q]) { best[q] = c[q]; searching[q] = false; }
      } else {
        int wc[U];
#pragma unroll
        for (int q = 0; q < U; q++) wc[q] = (holder[q] && !eager[q]) ? a.weight[c[q]] : 0;
#pragma unroll
        for (int q = 0; q < U; q++) {
          // after an eager pass every remaining candidate fits
          const unsigned fits = holder[q] && (eager[q] || (int64_t)wc[q] + cv[q] <= a.bound) ? 1u : 0u;
          if (__reduce_or_sync(gmask, fits) && searching[q]) { best[q] = c[q]; searching[q] = false; }
#pragma unroll
          for (int e = 0; e < E; e++) alive[q][e] = alive[q][e] && (unsigned)L[q][e] != c[q];
          eager[q] = true;
        }
      }
    }
#pragma unroll
    for (int q = 0; q < U; q++) {
      if (gl == 0 && v[q] >= 0) {
        ue += deg[q];
        uv += 1;
        if (best[q] != 0xFFFFFFFFu) {
          emit<MODE>(a, base + q * NV + grp, v[q], (int)best[q], cv[q], own[q]);
          up += 1;
        } else if (MODE == RATE_LP) {
          a.prop[base + q * NV + grp] = make_int2(-1, 0);
        }
      } else if (gl == 0 && skip[q] && MODE == RATE_LP) {
        a.prop[base + q * NV + grp] = make_int2(-1, 0);
      }
    }
  }
  add_units(a.units, ue, uv, uc, up, a.label8 != nullptr, a.adjwgt == nullptr);
}

// --------------------------------------- degree <= 128: warp/node + table

template <int MODE>
__global__ void __launch_bounds__(kThreads) k_rate_medium(RateArgs a) {
  __shared__ int s_k[kWarpsPerBlock][kMedSlots];
  __shared__ int s_v[kWarpsPerBlock][kMedSlots];
  const int lane = (int)lane_id(), wib = threadIdx.x >> 5;
  int *tk = s_k[wib], *tv = s_v[wib];
  for (int t = lane; t < kMedSlots; t += 32) { tk[t] = -1; tv[t] = 0; }
  __syncwarp();
  if (a.stop && *a.stop) return;
  const int begin = a.offs[a.key], end = list_end(a);
  const int wid = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5);
  const int nw = (int)((gridDim.x * blockDim.x) >> 5);
  unsigned long long ue = 0, uv = 0, uc = 0, up = 0;
  for (int i = begin + wid; i < end; i += nw) {
    const int4 rec = a.list[i];
    const int v = rec.x, start = rec.y, deg = rec.z, cv = rec.w;
    if (a.dirty && !a.dirty[v]) {  // clean: cannot move
      if (MODE == RATE_LP && lane == 0) a.prop[i] = make_int2(-1, 0);
      continue;
    }
    const int own = label_of(a, v);
    for (int j = lane; j < deg; j += 32) {
      const int L = label_of(a, __ldcs(a.adjncy + start + j));
      const int w = a.adjwgt ? __ldcs(a.adjwgt + start + j) : 1;
      unsigned s = slot_hash(L, 8);
      for (int probe = 0; probe < kMedSlots; probe++) {  // bounded: the table never fills
        const int prev = atomicCAS(&tk[s], -1, L);
        if (prev == -1 || prev == L) { atomicAdd(&tv[s], w); break; }
        s = (s + 1) & (kMedSlots - 1);
      }
    }
    __syncwarp();
    int own_loc = 0, rloc = -1, nc = 0, rall = 0;
    for (int t = lane; t < kMedSlots; t += 32) {
      const int L = tk[t];
      if (L < 0) continue;
      const int r = tv[t];
      if (L == own) { own_loc = r; continue; }
      nc++;
      rall = r > rall ? r : rall;
      if (MODE == RATE_LP && (int64_t)a.weight[L] + cv > a.bound) continue;
      rloc = r > rloc ? r : rloc;
    }
    const int own_r = warp_max(own_loc);
    const int rmax = warp_max(rloc);
    if (a.dirty && warp_max(rall) <= own_r && lane == 0) a.dirty[v] = 0;
    ue += deg; uv += 1; uc += nc;
    if (!(rmax < 0 || (MODE == RATE_LP && rmax <= own_r))) {
      uint64_t packed = ~0ull;
      for (int t = lane; t < kMedSlots; t += 32) {
        const int L = tk[t];
        if (L < 0 || L == own || tv[t] != rmax) continue;
        if (MODE == RATE_LP && (int64_t)a.weight[L] + cv > a.bound) continue;
        const uint64_t p = ((uint64_t)h32(a.ktie, (uint32_t)v, (uint32_t)L) << 32) | (uint32_t)L;
        packed = p < packed ? p : packed;
      }
      packed = warp_min(packed);
      if (lane == 0) { emit<MODE>(a, i, v, (int)(uint32_t)packed, cv, own); up += 1; }
    } else if (MODE == RATE_LP && lane == 0) {
      a.prop[i] = make_int2(-1, 0);
    }
    for (int t = lane; t < kMedSlots; t += 32) { tk[t] = -1; tv[t] = 0; }
    __syncwarp();
  }
  add_units(a.units, ue * (lane == 0), uv * (lane == 0), uc, up, a.label8 != nullptr, a.adjwgt == nullptr);
}

// --------------------------------------------- degree > 128: block/node

__device__ __forceinline__ int block_max_i32(int v, int *s_red) {
  v = warp_max(v);
  const int w = threadIdx.x >> 5;
  __syncthreads();
  if (lane_id() == 0) s_red[w] = v;
  __syncthreads();
  int r = s_red[0];
  for (int i = 1; i < kWarpsPerBlock; i++) r = s_red[i] > r ? s_red[i] : r;
  return r;
}

__device__ __forceinline__ uint64_t block_min_u64(uint64_t v, uint64_t *s_red) {
  v = warp_min(v);
  const int w = threadIdx.x >> 5;
  __syncthreads();
  if (lane_id() == 0) s_red[w] = v;
  __syncthreads();
  uint64_t r = s_red[0];
  for (int i = 1; i < kWarpsPerBlock; i++) r = s_red[i] < r ? s_red[i] : r;
  return r;
}

template <int MODE>
__global__ void __launch_bounds__(kThreads) k_rate_large(RateArgs a) {
  __shared__ int s_k[kLargeSmemSlots];
  __shared__ int s_v[kLargeSmemSlots];
  __shared__ int s_ri[kWarpsPerBlock];
  __shared__ uint64_t s_ru[kWarpsPerBlock];
  if (a.stop && *a.stop) return;
  for (int t = threadIdx.x; t < kLargeSmemSlots; t += blockDim.x) { s_k[t] = -1; s_v[t] = 0; }
  __syncthreads();
  const int begin = a.offs[a.key], end = list_end(a);
  int *gk = a.gkeys ? a.gkeys + (int64_t)blockIdx.x * a.gstride : nullptr;
  int *gv = a.gvals ? a.gvals + (int64_t)blockIdx.x * a.gstride : nullptr;
  unsigned long long ue = 0, uv = 0, uc = 0, up = 0;
  for (int i = begin + (int)blockIdx.x; i < end; i += (int)gridDim.x) {
    const int4 rec = a.list[i];
    const int v = rec.x, start = rec.y, deg = rec.z, cv = rec.w;
    if (a.dirty && !a.dirty[v]) {  // clean: cannot move (uniform in the block)
      if (MODE == RATE_LP && threadIdx.x == 0) a.prop[i] = make_int2(-1, 0);
      continue;
    }
    const int own = label_of(a, v);
    int bits = 1;
    while ((1 << bits) < 2 * deg) bits++;
    const int tsize = 1 << bits;
    const bool in_smem = tsize <= kLargeSmemSlots;
    int *tk = in_smem ? s_k : gk;
    int *tv = in_smem ? s_v : gv;
    for (int j = threadIdx.x; j < deg; j += blockDim.x) {
      const int L = label_of(a, __ldcs(a.adjncy + start + j));
      const int w = a.adjwgt ? __ldcs(a.adjwgt + start + j) : 1;
      unsigned s = slot_hash(L, bits);
      for (int probe = 0; probe < tsize; probe++) {  // bounded: the table never fills
        const int prev = atomicCAS(&tk[s], -1, L);
        if (prev == -1 || prev == L) { atomicAdd(&tv[s], w); break; }
        s = (s + 1) & (unsigned)(tsize - 1);
      }
    }
    __syncthreads();
    int own_loc = 0, rloc = -1, nc = 0, rall = 0;
    for (int t = threadIdx.x; t < tsize; t += blockDim.x) {
      const int L = tk[t];
      if (L < 0) continue;
      const int r = tv[t];
      if (L == own) { own_loc = r; continue; }
      nc++;
      rall = r > rall ? r : rall;
      if (MODE == RATE_LP && (int64_t)a.weight[L] + cv > a.bound) continue;
      rloc = r > rloc ? r : rloc;
    }
    const int own_r = block_max_i32(own_loc, s_ri);
    const int rmax = block_max_i32(rloc, s_ri);
    if (a.dirty) {
      const int ra = block_max_i32(rall, s_ri);
      if (ra <= own_r && threadIdx.x == 0) a.dirty[v] = 0;
    }
    uc += nc;
    if (threadIdx.x == 0) { ue += deg; uv += 1; }
    if (!(rmax < 0 || (MODE == RATE_LP && rmax <= own_r))) {
      uint64_t packed = ~0ull;
      for (int t = threadIdx.x; t < tsize; t += blockDim.x) {
        const int L = tk[t];
        if (L < 0 || L == own || tv[t] != rmax) continue;
        if (MODE == RATE_LP && (int64_t)a.weight[L] + cv > a.bound) continue;
        const uint64_t p = ((uint64_t)h32(a.ktie, (uint32_t)v, (uint32_t)L) << 32) | (uint32_t)L;
        packed = p < packed ? p : packed;
      }
      packed = block_min_u64(packed, s_ru);
      if (threadIdx.x == 0) { emit<MODE>(a, i, v, (int)(uint32_t)packed, cv, own); up += 1; }
    } else if (MODE == RATE_LP && threadIdx.x == 0) {
      a.prop[i] = make_int2(-1, 0);
    }
    __syncthreads();
    for (int t = threadIdx.x; t < tsize; t += blockDim.x) { tk[t] = -1; tv[t] = 0; }
    __syncthreads();
  }
  add_units(a.units, ue, uv, uc, up, a.label8 != nullptr, a.adjwgt == nullptr);
}

// ----------------------------------------------------- per-round buckets

struct BucketArgs {
  const int32_t *xadj, *label, *size, *vwgt;
  int n;
  uint64_t kact;
  int S;           // sub-rounds (1 for the favourite lists)
  int fav_mode;    // 0: all nodes with neighbours; 1: light singletons
  int64_t U;       // fav_mode: light means 2 c <= U
  const int *stop;
};

__device__ __forceinline__ int bucket_key(const BucketArgs &b, int v) {
  const int deg = b.xadj[v + 1] - b.xadj[v];
  if (deg == 0) return -1;
  if (b.fav_mode) {
    if (b.size[b.label[v]] != 1 || 2 * (int64_t)b.vwgt[v] > b.U) return -1;
    return degree_bucket(deg);
  }
  const int s = (int)(h32(b.kact, (uint32_t)v, 0) % (uint32_t)b.S);
  return s * kNumBuckets + degree_bucket(deg);
}

constexpr int kChunk = kThreads * 16;

__global__ void __launch_bounds__(kThreads) k_bucket_count(BucketArgs b, int nkeys, int *cnt) {
  __shared__ int s_c[kMaxKeys];
  if (b.stop && *b.stop) return;
  for (int t = threadIdx.x; t < nkeys; t += blockDim.x) s_c[t] = 0;
  __syncthreads();
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < b.n;
       v += (int64_t)gridDim.x * blockDim.x) {
    const int k = bucket_key(b, (int)v);
    if (k >= 0) atomicAdd(&s_c[k], 1);
  }
  __syncthreads();
  for (int t = threadIdx.x; t < nkeys; t += blockDim.x)
    if (s_c[t]) atomicAdd(&cnt[t], s_c[t]);
}

__global__ void k_bucket_offsets(const int *cnt, int nkeys, int *offs, int *cursor, const int *stop) {
  if (stop && *stop) return;
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    int run = 0;
    for (int k = 0; k < nkeys; k++) {
      offs[k] = run;
      cursor[k] = run;
      run += cnt[k];
    }
    offs[nkeys] = run;
  }
}

__global__ void __launch_bounds__(kThreads) k_bucket_scatter(BucketArgs b, int nkeys, int *cursor,
                                                             int4 *list) {
  __shared__ int s_c[kMaxKeys];
  __shared__ int s_base[kMaxKeys];
  if (b.stop && *b.stop) return;
  for (int64_t c0 = (int64_t)blockIdx.x * kChunk; c0 < b.n; c0 += (int64_t)gridDim.x * kChunk) {
    for (int t = threadIdx.x; t < nkeys; t += blockDim.x) s_c[t] = 0;
    __syncthreads();
    int keys[16];
#pragma unroll
    for (int j = 0; j < 16; j++) {
      const int64_t v = c0 + j * kThreads + threadIdx.x;
      keys[j] = v < b.n ? bucket_key(b, (int)v) : -1;
      if (keys[j] >= 0) atomicAdd(&s_c[keys[j]], 1);
    }
    __syncthreads();
    for (int t = threadIdx.x; t < nkeys; t += blockDim.x) {
      s_base[t] = s_c[t] ? atomicAdd(&cursor[t], s_c[t]) : 0;
      s_c[t] = 0;
    }
    __syncthreads();
#pragma unroll
    for (int j = 0; j < 16; j++) {
      if (keys[j] < 0) continue;
      const int64_t v = c0 + j * kThreads + threadIdx.x;
      const int pos = s_base[keys[j]] + atomicAdd(&s_c[keys[j]], 1);
      const int st = b.xadj[v];
      list[pos] = make_int4((int)v, st, b.xadj[v + 1] - st, b.vwgt[v]);
    }
    __syncthreads();
  }
}

// ------------------------------------------------------ clean nodes
//
// Refinement keeps a flag per node: a node whose rating found no label rated
// above its own (admissible or not) cannot propose until one of its
// neighbours moves, so it is left out of the rating lists until then.

// The dirty records of the sub-round's buckets k0 .. k1-1, packed from the
// start of each bucket's range; ccount[key] receives the bucket's count.
__global__ void __launch_bounds__(kThreads) k_compact_dirty(const int4 *list, const int32_t *offs, int k0, int k1,
                                                            const uint8_t *dirty, int4 *clist, int32_t *ccount,
                                                            const int *stop) {
  if (stop && *stop) return;
  __shared__ int s_cnt[kNumBuckets], s_base[kNumBuckets];
  const int begin = offs[k0], end = offs[k1];
  const int lane = (int)lane_id();
  for (int base = begin + (int)(blockIdx.x * blockDim.x); base < end; base += gridDim.x * blockDim.x) {
    if (threadIdx.x < kNumBuckets) s_cnt[threadIdx.x] = 0;
    __syncthreads();
    const int i = base + (int)threadIdx.x;
    int bk = k1;  // bucket of the position (k1 past the end)
    int b = -1;   // bucket if the record is kept
    int4 rec = make_int4(0, 0, 0, 0);
    if (i < end) {
      bk = k0;
      while (bk + 1 < k1 && offs[bk + 1] <= i) bk++;
      rec = list[i];
      if (dirty[rec.x]) b = bk;
    }
    // consecutive lanes hold consecutive list positions, so a bucket's lanes form one run:
    // its kept lanes are the peers (no match over arbitrary keys needed)
    const int prev = __shfl_up_sync(FULL, bk, 1);
    const unsigned starts = __ballot_sync(FULL, lane == 0 || prev != bk);
    const unsigned kept = __ballot_sync(FULL, b >= 0);
    const unsigned le = lanemask_lt() | (1u << lane);
    const unsigned after = starts & ~le;  // run starts after this lane
    const unsigned run_lo = 31 - __clz(starts & le);
    const unsigned run_hi = after ? (unsigned)__ffs(after) - 1 : 32u;  // one past the run
    const unsigned run = (run_hi == 32 ? FULL : ((1u << run_hi) - 1u)) & ~((1u << run_lo) - 1u);
    const unsigned peers = kept & run;
    int pos = 0;
    if (b >= 0) {
      // the block's kept records of each bucket are counted in shared memory, and the bucket's
      // global cursor advances once per block and bucket
      const int leader = __ffs(peers) - 1;
      if (lane == leader) pos = atomicAdd(&s_cnt[b - k0], __popc(peers));
      pos = __shfl_sync(peers, pos, leader) + __popc(peers & lanemask_lt());
    }
    __syncthreads();
    if (threadIdx.x < kNumBuckets && s_cnt[threadIdx.x] > 0)
      s_base[threadIdx.x] = atomicAdd(&ccount[k0 + threadIdx.x], s_cnt[threadIdx.x]);
    __syncthreads();
    if (b >= 0) clist[offs[b] + s_base[b - k0] + pos] = rec;
  }
}
__global__ void __launch_bounds__(kThreads) k_mark_dirty(const int4 *mov, int nmov, const uint64_t *ov_key,
                                                         const uint32_t *ov_val, const uint8_t *ov_acc, int nov,
                                                         const uint64_t *cutoff, uint64_t kprio,
                                                         const int32_t *xadj, const int32_t *adjncy,
                                                         uint8_t *dirty) {
  const int lane = (int)lane_id();
  const int wid = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5);
  const int nw = (int)((gridDim.x * blockDim.x) >> 5);
  const int total = nmov + nov;
  for (int t0 = 2 * wid; t0 < total; t0 += 2 * nw) {
    int v[2], e0[2], e1[2];
#pragma unroll
    for (int q = 0; q < 2; q++) {
      const int t = t0 + q;
      v[q] = -1;
      if (t < nmov) v[q] = mov[t].x;
      else if (t < total && ov_acc[t - nmov]) v[q] = (int)ov_val[t - nmov];
      if (v[q] >= 0 && cutoff &&
          ((((uint64_t)h32(kprio, (uint32_t)v[q], 0)) << 32) | (uint32_t)v[q]) >= *cutoff)
        v[q] = -1;
      e0[q] = v[q] >= 0 ? xadj[v[q]] : 0;
      e1[q] = v[q] >= 0 ? xadj[v[q] + 1] : 0;
    }
#pragma unroll
    for (int q = 0; q < 2; q++)
      if (lane == 0 && v[q] >= 0) dirty[v[q]] = 1;
    const int len = max(e1[0] - e0[0], e1[1] - e0[1]);
    for (int o = lane; o < len; o += 32) {
      const int a0 = e0[0] + o, a1 = e0[1] + o;
      const int u0 = a0 < e1[0] ? adjncy[a0] : -1, u1 = a1 < e1[1] ? adjncy[a1] : -1;
      if (u0 >= 0) dirty[u0] = 1;
      if (u1 >= 0) dirty[u1] = 1;
    }
  }
}

// ------------------------------------------------------------- acceptance

struct Counters {
  int stop;
  int nov;   // proposers of overflowing targets this sub-round
  int nmov;  // proposers accepted outright this sub-round
  int pad0;
  long long moved_sub;
  long long moved_round;
  long long moved_total;
  long long nonempty;   // clustering: change of the number of labels of positive weight in the sub-round
  long long nclusters;
};

// Every active node's proposal (written by the rating kernels at its list
// position) goes to the list of outright acceptances (the target's snapshot
// weight plus all incoming weight fits), as a (node, target, own label,
// weight) record, or to the list of proposers of overflowing targets.  Slots
// in both lists are reserved once per block and iteration.
__global__ void __launch_bounds__(kThreads) k_decide(const int4 *list, const int32_t *offs,
                                                     int k0, int k1, const int2 *prop,
                                                     const int32_t *weight, const int32_t *incoming,
                                                     int64_t bound, int4 *mov,
                                                     uint64_t *ov_key, uint32_t *ov_val, Counters *cnt,
                                                     uint64_t kprio, const int32_t *ccount) {
  __shared__ int s_a[kWarpsPerBlock + 1], s_o[kWarpsPerBlock + 1];
  if (cnt->stop) return;
  const int begin = offs[k0], end = offs[k1];
  const int stride = gridDim.x * blockDim.x;
  const int lane = (int)lane_id(), w = threadIdx.x >> 5;
  for (int base = begin + (int)(blockIdx.x * blockDim.x); base < end; base += stride) {
    const int i = base + (int)threadIdx.x;
    bool acc = false, over = false;
    int v = 0, K = -1, own = 0, c = 0;
    bool live = i < end;
    if (live && ccount) {  // compacted lists: positions past a bucket's count hold nothing
      int b = k0;
      while (b + 1 < k1 && offs[b + 1] <= i) b++;
      live = i < offs[b] + ccount[b];
    }
    if (live) {
      const int2 pr = prop[i];
      K = pr.x;
      if (K >= 0) {
        const int4 rec = list[i];
        v = rec.x; c = rec.w; own = pr.y;
        if ((int64_t)weight[K] + incoming[K] <= bound) acc = true;
        else over = true;
      }
    }
    const unsigned ma = __ballot_sync(0xFFFFFFFFu, acc), mo = __ballot_sync(0xFFFFFFFFu, over);
    if (lane == 0) { s_a[w] = __popc(ma); s_o[w] = __popc(mo); }
    __syncthreads();
    if (threadIdx.x == 0) {
      int ra = 0, ro = 0;
      for (int j = 0; j < kWarpsPerBlock; j++) {
        const int ca = s_a[j], co = s_o[j];
        s_a[j] = ra; s_o[j] = ro;
        ra += ca; ro += co;
      }
      s_a[kWarpsPerBlock] = ra ? atomicAdd(&cnt->nmov, ra) : 0;
      s_o[kWarpsPerBlock] = ro ? atomicAdd(&cnt->nov, ro) : 0;
    }
    __syncthreads();
    if (acc) {
      const int pos = s_a[kWarpsPerBlock] + s_a[w] + __popc(ma & lanemask_lt());
      mov[pos] = make_int4(v, K, own, c);
    }
    if (over) {
      const int pos = s_o[kWarpsPerBlock] + s_o[w] + __popc(mo & lanemask_lt());
      ov_key[pos] = ((uint64_t)(uint32_t)K << 32) | h32(kprio, (uint32_t)v, 0);
      ov_val[pos] = (uint32_t)v;
    }
    __syncthreads();
  }
}

// Runs of equal keys are ordered by node id (the last tie-break of R7).
__global__ void k_fix_runs(const uint64_t *keys, uint32_t *vals, int n) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    if (i > 0 && keys[i - 1] == keys[i]) continue;
    if (i + 1 >= n || keys[i + 1] != keys[i]) continue;
    int e = i + 1;
    while (e < n && keys[e] == keys[i]) e++;
    for (int a = i + 1; a < e; a++) {
      uint32_t x = vals[a];
      int b = a - 1;
      while (b >= i && vals[b] > x) { vals[b + 1] = vals[b]; b--; }
      vals[b + 1] = x;
    }
  }
}

__global__ void k_ov_weights(const uint32_t *vals, int n, const int32_t *vwgt, int64_t *cs) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    cs[i] = vwgt[vals[i]];
}

// Sorted by (target, prio, node): accept while the running weight within the
// target's segment fits (ps = exclusive prefix sum of the weights).
__global__ void k_ov_accept(const uint64_t *keys, const uint32_t *vals, int n, const int64_t *ps,
                            const int32_t *vwgt, const int32_t *weight, int64_t bound, uint8_t *ov_acc) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const uint64_t k = keys[i];
    const uint64_t seg = k & 0xFFFFFFFF00000000ull;
    int lo = 0, hi = i;  // first index with key >= seg
    while (lo < hi) {
      int mid = (lo + hi) >> 1;
      if (keys[mid] < seg) lo = mid + 1; else hi = mid;
    }
    const int K = (int)(k >> 32);
    const int64_t incl = ps[i] - ps[lo] + vwgt[vals[i]];
    ov_acc[i] = (int64_t)weight[K] + incl <= bound ? 1 : 0;
  }
}

// ------------------------------------------ small overflow sets
//
// Up to kOvSmall proposers of overflowing targets are ordered by (target,
// priority, node) with a bitonic sort in one block's shared memory; a block
// scan of their weights gives every proposer its running weight within its
// target, and it is accepted iff the target's weight plus that fits.

constexpr int kOvSmall = 2048;
constexpr int kOvSmallThreads = 1024;

__global__ void __launch_bounds__(kOvSmallThreads) k_ov_small(uint64_t *key, uint32_t *val, int nov,
                                                              const int32_t *vwgt, const int32_t *weight,
                                                              int64_t bound, uint8_t *acc) {
  __shared__ uint64_t s_k[kOvSmall];
  __shared__ uint32_t s_v[kOvSmall];
  __shared__ long long s_w[kOvSmallThreads / 32];
  int P = 1;
  while (P < nov) P <<= 1;
  const int t = threadIdx.x;
  for (int i = t; i < P; i += blockDim.x) {
    s_k[i] = i < nov ? key[i] : ~0ull;
    s_v[i] = i < nov ? val[i] : 0xFFFFFFFFu;
  }
  __syncthreads();
  for (int size = 2; size <= P; size <<= 1) {
    for (int stride = size >> 1; stride > 0; stride >>= 1) {
      for (int i = t; i < P / 2; i += blockDim.x) {
        const int lo = 2 * i - (i & (stride - 1));  // pairs (lo, lo + stride)
        const int hi = lo + stride;
        const bool up = (lo & size) == 0;
        const uint64_t ka = s_k[lo], kb = s_k[hi];
        const uint32_t va = s_v[lo], vb = s_v[hi];
        const bool gt = ka > kb || (ka == kb && va > vb);
        if (gt == up) { s_k[lo] = kb; s_k[hi] = ka; s_v[lo] = vb; s_v[hi] = va; }
      }
      __syncthreads();
    }
  }
  // sorted order written back; inclusive running weights (their total is at most
  // the graph's node weight, below 2^31) replace the node ids in shared memory
  long long carry = 0;
  const int lane = (int)lane_id(), wp = t >> 5, nwp = blockDim.x >> 5;
  for (int c0 = 0; c0 < nov; c0 += blockDim.x) {
    const int i = c0 + t;
    long long x = 0;
    if (i < nov) {
      const uint32_t v = s_v[i];
      key[i] = s_k[i];
      val[i] = v;
      x = vwgt[v];
    }
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const long long y = __shfl_up_sync(FULL, x, o);
      if (lane >= o) x += y;
    }
    if (lane == 31) s_w[wp] = x;
    __syncthreads();
    long long before = carry, chunk = 0;
    for (int q = 0; q < nwp; q++) {
      if (q < wp) before += s_w[q];
      chunk += s_w[q];
    }
    if (i < nov) s_v[i] = (uint32_t)(before + x);
    carry += chunk;
    __syncthreads();
  }
  for (int i = t; i < nov; i += blockDim.x) {
    // first proposer of i's target: lower bound of (target << 32) in the sorted keys
    const uint64_t seg = s_k[i] & 0xFFFFFFFF00000000ull;
    int a = 0, b = i;
    while (a < b) {
      const int mid = (a + b) >> 1;
      if (s_k[mid] < seg) a = mid + 1; else b = mid;
    }
    const long long incl = (long long)s_v[i] - (a > 0 ? (long long)s_v[a - 1] : 0);
    const int K = (int)(s_k[i] >> 32);
    acc[i] = (int64_t)weight[K] + incl <= bound ? 1 : 0;
  }
}

// ------------------------------------------ overflow with few labels
//
// The proposers of overflowing targets are not sorted.  Per target, a
// histogram of their weights over the top bits of the priority locates the
// bucket in which the running weight (in priority order) crosses the
// target's free room: proposers in earlier buckets fit (the accepted prefix
// contains them), proposers in later ones do not, and only the crossing
// bucket's proposers are ranked exactly by (priority, node), in one block per
// target.  The result equals the longest-prefix rule of the sorted order.

constexpr int kOvBuckets = 4096;   // priority buckets per label (top 12 bits)
constexpr int kOvMaxLabels = 256;  // labels handled this way
constexpr int kOvSmem = 2048;      // crossing-bucket proposers ranked in shared memory

__global__ void k_ovb_hist(const uint64_t *key, const uint32_t *val, int nov, const int32_t *vwgt,
                           unsigned long long *hw, int32_t *hc) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nov; i += gridDim.x * blockDim.x) {
    const uint64_t k = key[i];
    const int64_t slot = (int64_t)(k >> 32) * kOvBuckets + (int)((uint32_t)k >> 20);
    atomicAdd(&hw[slot], (unsigned long long)vwgt[val[i]]);
    atomicAdd(&hc[slot], 1);
  }
}

// One block per label: the crossing bucket, the weight before it and the
// number of proposers in it.
__global__ void __launch_bounds__(256) k_ovb_cut(const unsigned long long *hw, const int32_t *hc,
                                                 const int32_t *weight, int64_t bound, int32_t *cut,
                                                 long long *base, int32_t *mcnt) {
  constexpr int PER = kOvBuckets / 256;
  __shared__ long long s_w[8];
  __shared__ int s_cut;
  const int K = blockIdx.x;
  const unsigned long long *h = hw + (int64_t)K * kOvBuckets;
  const int t = threadIdx.x, lane = (int)lane_id(), wp = t >> 5;
  long long loc = 0;
#pragma unroll
  for (int q = 0; q < PER; q++) loc += (long long)h[t * PER + q];
  long long incl = loc;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const long long y = __shfl_up_sync(FULL, incl, o);
    if (lane >= o) incl += y;
  }
  if (lane == 31) s_w[wp] = incl;
  if (t == 0) s_cut = kOvBuckets;
  __syncthreads();
  long long excl = incl - loc;
  for (int q = 0; q < wp; q++) excl += s_w[q];
  const long long room = bound - (long long)weight[K];
  long long run = excl;
  int mine = kOvBuckets;
  long long before = 0;
  for (int q = 0; q < PER; q++) {
    const long long x = (long long)h[t * PER + q];
    if (x > 0 && run + x > room) { mine = t * PER + q; before = run; break; }
    run += x;
  }
  if (mine < kOvBuckets) atomicMin(&s_cut, mine);
  __syncthreads();
  if (mine == s_cut && mine < kOvBuckets) {
    cut[K] = mine;
    base[K] = before;
    mcnt[K] = hc[(int64_t)K * kOvBuckets + mine];
  }
  if (t == 0 && s_cut == kOvBuckets) { cut[K] = kOvBuckets; base[K] = 0; mcnt[K] = 0; }
}

__global__ void __launch_bounds__(1024) k_ovb_offsets(const int32_t *mcnt, int nlabels, int32_t *roff,
                                                      int32_t *cursor) {
  if (threadIdx.x == 0) {
    int run = 0;
    for (int K = 0; K < nlabels; K++) { roff[K] = run; cursor[K] = run; run += mcnt[K]; }
    roff[nlabels] = run;
  }
}

// Earlier buckets accepted, later ones rejected, the crossing bucket's
// proposers listed per label.
__global__ void k_ovb_class(const uint64_t *key, const uint32_t *val, int nov, const int32_t *cut,
                            int32_t *cursor, uint8_t *acc, uint64_t *bkey, int32_t *bidx) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nov; i += gridDim.x * blockDim.x) {
    const uint64_t k = key[i];
    const int K = (int)(k >> 32), b = (int)((uint32_t)k >> 20), c = cut[K];
    acc[i] = b < c ? 1 : 0;
    if (b == c) {
      const int j = atomicAdd(&cursor[K], 1);
      bkey[j] = ((uint64_t)(uint32_t)k << 32) | val[i];  // (priority, node)
      bidx[j] = i;
    }
  }
}

// One block per label: ranks the crossing bucket's proposers by (priority,
// node) and accepts those whose running weight still fits.
__global__ void __launch_bounds__(256) k_ovb_resolve(const uint64_t *bkey, const int32_t *bidx,
                                                     const int32_t *roff, const int32_t *vwgt,
                                                     const int32_t *weight, const long long *base,
                                                     int64_t bound, uint8_t *acc) {
  __shared__ uint64_t s_k[kOvSmem];
  __shared__ int s_c[kOvSmem];
  const int K = blockIdx.x;
  const int r0 = roff[K], m = roff[K + 1] - r0;
  if (m == 0) return;
  const bool in_smem = m <= kOvSmem;
  if (in_smem) {
    for (int j = threadIdx.x; j < m; j += blockDim.x) {
      s_k[j] = bkey[r0 + j];
      s_c[j] = vwgt[(uint32_t)bkey[r0 + j]];
    }
    __syncthreads();
  }
  const long long room = bound - (long long)weight[K] - base[K];
  for (int i = threadIdx.x; i < m; i += blockDim.x) {
    const uint64_t ki = in_smem ? s_k[i] : bkey[r0 + i];
    long long incl = 0;
    for (int j = 0; j < m; j++) {  // weight of the proposers up to and including i
      const uint64_t kj = in_smem ? s_k[j] : bkey[r0 + j];
      if (kj <= ki) incl += in_smem ? s_c[j] : vwgt[(uint32_t)kj];
    }
    acc[bidx[r0 + i]] = incl <= room ? 1 : 0;
  }
}

struct ApplyArgs {
  const int4 *mov;  // outright moves: (node, target, own label, node weight)
  const uint64_t *ov_key;
  const uint32_t *ov_val;
  const uint8_t *ov_acc;
  int nmov, nov;
  const int32_t *vwgt;
  int32_t *label, *weight, *incoming;
  uint8_t *label8;
  int nshared;       // > 0: few labels; weight changes summed per block in shared memory
  Counters *cnt;
  const uint64_t *cutoff;  // 2.5x cap: only moves with key (h32(PRIO), v) below *cutoff apply (null: all)
  uint64_t kprio;
  int track;  // clustering: count the labels whose weight reaches or leaves 0
};

__device__ __forceinline__ uint64_t move_key(uint64_t kprio, int v) {
  return ((uint64_t)h32(kprio, (uint32_t)v, 0) << 32) | (uint32_t)v;
}

__device__ __forceinline__ void proposal(const ApplyArgs &a, int t, int &v, int &K, int &own, int &c,
                                         bool &mv) {
  if (t < a.nmov) {
    const int4 r = a.mov[t];
    v = r.x; K = r.y; own = r.z; c = r.w; mv = true;
  } else {
    const int j = t - a.nmov;
    v = (int)a.ov_val[j]; K = (int)(a.ov_key[j] >> 32); mv = a.ov_acc[j] != 0;
    own = mv ? a.label[v] : 0;
    c = mv ? a.vwgt[v] : 0;
  }
}

// Moves every accepted proposer (outright or through the overflow order).
__global__ void __launch_bounds__(kThreads) k_apply(ApplyArgs a) {
  extern __shared__ int s_dw[];
  for (int t = threadIdx.x; t < a.nshared; t += blockDim.x) s_dw[t] = 0;
  if (a.nshared) __syncthreads();
  const int total = a.nmov + a.nov;
  long long moved = 0, dne = 0;  // dne: labels whose weight left 0 minus labels whose weight reached 0
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < total; t += gridDim.x * blockDim.x) {
    int v, K, own, c;
    bool mv;
    proposal(a, t, v, K, own, c, mv);
    if (mv && a.cutoff && move_key(a.kprio, v) >= *a.cutoff) mv = false;
    if (mv) {
      a.label[v] = K;
      if (a.label8) a.label8[v] = (uint8_t)K;

      if (a.nshared) {
        atomicAdd(&s_dw[K], c);
        atomicSub(&s_dw[own], c);
      } else {
        // every update's transition 0 <-> non-0 counted: their sum is the net change
        const int ok = atomicAdd(&a.weight[K], c);
        const int oo = atomicSub(&a.weight[own], c);
        if (a.track) dne += (ok == 0 ? 1 : 0) - (oo == c ? 1 : 0);
      }
      moved++;
    }
  }
  if (a.nshared) {
    __syncthreads();
    for (int t = threadIdx.x; t < a.nshared; t += blockDim.x)
      if (s_dw[t]) {
        const int o = atomicAdd(&a.weight[t], s_dw[t]);
        if (a.track) dne += ((o + s_dw[t] > 0) ? 1 : 0) - ((o > 0) ? 1 : 0);
      }
  }
  moved = warp_sum(moved);
  dne = warp_sum(dne);
  if (lane_id() == 0 && moved)
    atomicAdd((unsigned long long *)&a.cnt->moved_sub, (unsigned long long)moved);
  if (lane_id() == 0 && dne) atomicAdd((unsigned long long *)&a.cnt->nonempty, (unsigned long long)dne);
}

// ------------------------------------------------------- the 2.5x cap
//
// The node reduction of a clustering is at most 2.5x (Sec. 4.3): with c
// clusters at the start of a sub-round, its moves may empty at most D =
// c - n_min of them.  A cluster all of whose weight leaves is emptied at the
// largest move key (h32(PRIO), node) among its departures (arrivals are not
// counted); if more than D clusters are emptied, only the moves below the
// (D+1)-th smallest emptying key apply.  These kernels run before k_apply, on
// the snapshot labels and weights, and only in sub-rounds whose accepted moves
// could exceed D.

// Departure weight and latest departure key per source cluster.
__global__ void __launch_bounds__(kThreads) k_cap_depart(ApplyArgs a, int32_t *depw,
                                                         unsigned long long *dkey) {
  const int total = a.nmov + a.nov;
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < total; t += gridDim.x * blockDim.x) {
    int v, K, own, c;
    bool mv;
    proposal(a, t, v, K, own, c, mv);
    if (!mv) continue;
    atomicAdd(&depw[own], c);
    atomicMax(&dkey[own], (unsigned long long)move_key(a.kprio, v));
  }
}

// The emptying key of every emptied cluster (listed once, by its latest mover);
// then clears the per-cluster state of the sources.
__global__ void __launch_bounds__(kThreads) k_cap_collect(ApplyArgs a, const int32_t *depw,
                                                          const unsigned long long *dkey,
                                                          uint64_t *ekeys, int *ecount) {
  const int total = a.nmov + a.nov;
  for (int base = blockIdx.x * blockDim.x; base < total; base += gridDim.x * blockDim.x) {
    const int t = base + (int)threadIdx.x;
    bool emit_key = false;
    uint64_t key = 0;
    if (t < total) {
      int v, K, own, c;
      bool mv;
      proposal(a, t, v, K, own, c, mv);
      if (mv) {
        key = move_key(a.kprio, v);
        emit_key = depw[own] == a.weight[own] && key == dkey[own];
      }
    }
    const int pos = warp_append(ecount, emit_key);
    if (emit_key) ekeys[pos] = key;
  }
}

__global__ void __launch_bounds__(kThreads) k_cap_clear(ApplyArgs a, int32_t *depw, unsigned long long *dkey) {
  const int total = a.nmov + a.nov;
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < total; t += gridDim.x * blockDim.x) {
    int v, K, own, c;
    bool mv;
    proposal(a, t, v, K, own, c, mv);
    if (!mv) continue;
    depw[own] = 0;
    dkey[own] = 0;
  }
}

// Closes a sub-round in one launch: clears the incoming weights of its
// targets, counts the non-empty clusters (node weights are positive, so a
// label is in use iff its weight is), and the last block to finish updates
// the counters: cluster count, moves, the stop flag (cluster count at n_min;
// at the end of a round, a round without moves), and clears the proposal
// list sizes for the next sub-round.
__global__ void __launch_bounds__(kThreads) k_close(ApplyArgs a, int64_t count_labels, long long n_min,
                                                    int round_end, unsigned *done) {
  Counters *cnt = a.cnt;
  if (cnt->stop) return;
  const int total = a.nmov + a.nov;
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < total; t += gridDim.x * blockDim.x) {
    const int K = t < a.nmov ? a.mov[t].y : (int)(a.ov_key[t - a.nmov] >> 32);
    a.incoming[K] = 0;
  }
  __syncthreads();
  __shared__ bool s_last;
  if (threadIdx.x == 0) {
    __threadfence();
    s_last = atomicAdd(done, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (!s_last || threadIdx.x != 0) return;
  __threadfence();
  volatile Counters *vc = cnt;
  if (count_labels > 0) vc->nclusters = vc->nclusters + vc->nonempty;  // k_apply's net change
  vc->nonempty = 0;
  const long long moved = vc->moved_sub;
  vc->moved_round = vc->moved_round + moved;
  vc->moved_total = vc->moved_total + moved;
  vc->moved_sub = 0;
  vc->nov = 0;
  vc->nmov = 0;
  if (count_labels > 0 && vc->nclusters <= n_min) vc->stop = 1;
  if (round_end) {
    if (!vc->stop && vc->moved_round == 0) vc->stop = 1;
    vc->moved_round = 0;
  }
  *done = 0;
}

__global__ void k_counters_init(Counters *cnt, long long nclusters) {
  cnt->stop = 0; cnt->nov = 0; cnt->nmov = 0; cnt->pad0 = 0; cnt->moved_sub = 0; cnt->moved_round = 0;
  cnt->moved_total = 0; cnt->nonempty = 0; cnt->nclusters = nclusters;
}


__global__ void k_fill_i32(int32_t *a, int64_t n, int32_t v) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    a[i] = v;
}

// Largest degree among nodes with more than kMediumMaxDeg neighbours.
__global__ void k_max_degree(const int32_t *xadj, int n, int *out) {
  int m = 0;
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n;
       v += (int64_t)gridDim.x * blockDim.x) {
    const int d = xadj[v + 1] - xadj[v];
    m = d > m ? d : m;
  }
  m = warp_max(m);
  if (lane_id() == 0 && m) atomicMax(out, m);
}

struct RateTables {
  DBuf<int32_t> gkeys, gvals;
  int64_t stride = 0;
  int blocks = 0;
};

// Global hash tables for the block-per-node kernel when some node needs more
// than kLargeSmemSlots slots.
void make_tables(gp_ctx *ctx, const DevGraph &g, RateTables &t) {
  DBuf<int> md(ctx, 1);
  md.zero();
  k_max_degree<<<grid_for(g.n, 256, ctx->num_sms * 8), 256, 0, ctx->stream>>>(g.xadj, g.n, md.get());
  GP_LAUNCH_CHECK();
  const int maxdeg = read_scalar(ctx, md.get());
  int bits = 1;
  while ((1 << bits) < 2 * maxdeg) bits++;
  t.blocks = ctx->num_sms * 4;
  if ((1 << bits) > kLargeSmemSlots) {
    t.stride = (int64_t)1 << bits;
    t.blocks = table_blocks(g.m2, t.stride, t.blocks);
    t.gkeys.reset(ctx, (size_t)(t.stride * t.blocks));
    t.gvals.reset(ctx, (size_t)(t.stride * t.blocks));
    t.gkeys.fill_bytes(0xFF);
    t.gvals.zero();
  }
}

// Grid for `count` listed nodes, `per_block` nodes per block and iteration
// (count < 0: unknown, the full grid).
inline int rate_grid(gp_ctx *ctx, int64_t count, int per_block, int cap) {
  if (count < 0) return cap;
  return grid_for(count, per_block, cap);
}

template <int G, int U>
constexpr int group_nodes_per_block() { return kWarpsPerBlock * (32 / G) * U; }

// hcnt: the five bucket sizes of this sub-round when the host knows them (empty
// buckets are then not launched), else nullptr
template <int MODE, int LK>
void launch_groups(gp_ctx *ctx, const RateArgs &a0, int bucket_key_base, const int *hcnt) {
  const int cap = ctx->num_sms * 8;
  RateArgs a = a0;
  if (!hcnt || hcnt[0] > 0) {
    a.key = bucket_key_base + 0;
    k_rate_group<MODE, 8, 2, LK><<<rate_grid(ctx, hcnt ? hcnt[0] : -1, group_nodes_per_block<8, 2>(), cap),
                                   kThreads, 0, ctx->stream>>>(a);
    GP_LAUNCH_CHECK();
  }
  if (!hcnt || hcnt[1] > 0) {
    a.key = bucket_key_base + 1;
    k_rate_multi<MODE, 8, 2, 2, LK><<<rate_grid(ctx, hcnt ? hcnt[1] : -1, group_nodes_per_block<8, 2>(), cap),
                                      kThreads, 0, ctx->stream>>>(a);
    GP_LAUNCH_CHECK();
  }
  if (!hcnt || hcnt[2] > 0) {
    a.key = bucket_key_base + 2;
    k_rate_multi<MODE, 16, 2, 3, LK><<<rate_grid(ctx, hcnt ? hcnt[2] : -1, group_nodes_per_block<16, 3>(), cap),
                                       kThreads, 0, ctx->stream>>>(a);
    GP_LAUNCH_CHECK();
  }
}

// nlabels: number of labels (chooses the narrow / dense group kernels when
// a uint8 copy of the labels is present)
template <int MODE>
void launch_rate(gp_ctx *ctx, RateArgs a, int bucket_key_base, const RateTables &t, int64_t nlabels,
                 const int *hcnt) {
  const int cap = ctx->num_sms * 8;
  if (MODE == RATE_LP && a.label8 && nlabels <= kDenseLabels) launch_groups<MODE, LK_DENSE>(ctx, a, bucket_key_base, hcnt);
  else if (MODE == RATE_LP && a.label8) launch_groups<MODE, LK_NARROW>(ctx, a, bucket_key_base, hcnt);
  else launch_groups<MODE, LK_WIDE>(ctx, a, bucket_key_base, hcnt);
  if (!hcnt || hcnt[3] > 0) {
    a.key = bucket_key_base + 3;
    k_rate_medium<MODE><<<rate_grid(ctx, hcnt ? hcnt[3] : -1, kWarpsPerBlock, cap), kThreads, 0, ctx->stream>>>(a);
    GP_LAUNCH_CHECK();
  }
  if (!hcnt || hcnt[4] > 0) {
    a.key = bucket_key_base + 4;
    a.gkeys = t.gkeys.get();
    a.gvals = t.gvals.get();
    a.gstride = t.stride;
    k_rate_large<MODE><<<rate_grid(ctx, hcnt ? hcnt[4] : -1, 1, t.blocks), kThreads, 0, ctx->stream>>>(a);
    GP_LAUNCH_CHECK();
  }
}

}  // namespace

int bits_for(int64_t x) {
  int b = 0;
  while (((int64_t)1 << b) <= x) b++;
  return b < 1 ? 1 : b;
}

LpResult lp_run(gp_ctx *ctx, const DevGraph &g, int32_t *label, int32_t *weight, int64_t nlabels, uint64_t seed, const LpParams &p, int64_t *nclusters_dev,
                uint8_t *label8) {
  if (lp_small_applicable(g, p)) return lp_run_small(ctx, g, label, weight, nlabels, seed, p, nclusters_dev, label8);
  LpResult res;
  const int n = g.n;
  const int S = p.subrounds;
  GP_REQUIRE(S >= 1 && S <= 64, GP_ERR_INVALID, "lp_subrounds must be in [1, 64]");
  const int nkeys = S * kNumBuckets;
  DBuf<int4> list(ctx, (size_t)n);
  DBuf<int2> prop(ctx, (size_t)n);
  DBuf<int32_t> incoming(ctx, (size_t)nlabels);
  DBuf<int32_t> cnt(ctx, (size_t)nkeys), offs(ctx, (size_t)nkeys + 1), cursor(ctx, (size_t)nkeys);
  DBuf<int4> mov(ctx, (size_t)n);
  DBuf<uint64_t> ov_key(ctx, (size_t)n);
  DBuf<uint32_t> ov_val(ctx, (size_t)n);
  DBuf<uint8_t> ov_acc(ctx, (size_t)n);
  // few labels (refinement): bucketed overflow resolution, no sort
  const bool few = nlabels <= kOvMaxLabels;
  DBuf<unsigned long long> ovb_hw;
  DBuf<int32_t> ovb_hc, ovb_cut, ovb_m, ovb_roff, ovb_cursor, ovb_idx;
  DBuf<long long> ovb_base;
  DBuf<uint64_t> ovb_key;
  if (few) {
    ovb_hw.reset(ctx, (size_t)nlabels * kOvBuckets);
    ovb_hc.reset(ctx, (size_t)nlabels * kOvBuckets);
    ovb_cut.reset(ctx, (size_t)nlabels);
    ovb_m.reset(ctx, (size_t)nlabels);
    ovb_roff.reset(ctx, (size_t)nlabels + 1);
    ovb_cursor.reset(ctx, (size_t)nlabels);
    ovb_base.reset(ctx, (size_t)nlabels);
    ovb_key.reset(ctx, (size_t)n);
    ovb_idx.reset(ctx, (size_t)n);
  }
  DBuf<Counters> counters(ctx, 1);
  Counters *C = counters.get();
  // refinement: nodes that must be rated (all at first; a node with no label rated above its
  // own is left out until a neighbour moves: it cannot propose, so results are unchanged)
  const bool use_dirty = !p.count_clusters;
  DBuf<uint8_t> dirty;
  DBuf<int4> clist;
  DBuf<int32_t> ccount;
  if (use_dirty) {
    dirty.reset(ctx, (size_t)n);
    dirty.fill_bytes(1);
    clist.reset(ctx, (size_t)n);
    ccount.reset(ctx, (size_t)nkeys);
  }
  // the 2.5x cap (clustering): departure weight and latest key per cluster, emptying keys
  DBuf<int32_t> cap_w;
  DBuf<unsigned long long> cap_k;
  DBuf<uint64_t> cap_e;
  DBuf<int> cap_n;
  DBuf<unsigned> done(ctx, 1);
  done.zero();
  incoming.zero();
  int64_t ncl0 = 0;
  if (p.count_clusters && nclusters_dev) read_back(ctx, nclusters_dev, sizeof(int64_t), &ncl0);
  k_counters_init<<<1, 1, 0, ctx->stream>>>(C, ncl0);
  GP_LAUNCH_CHECK();
  RateTables tables;
  make_tables(ctx, g, tables);
  unsigned long long *units_rate = ctx->d_units ? ctx->d_units + p.prof_rate * PROF_UNITS : nullptr;

  TraceTimer trace(ctx);
  const int grid = ctx->num_sms * 8;
  std::vector<int32_t> hoffs((size_t)nkeys + 1);
  double sync_s = 0;  // host time blocked in the per-sub-round read of the counters (tracing)
  const auto t_host0 = std::chrono::steady_clock::now();
  const bool agg = nlabels <= 4096;  // refinement: few labels, aggregate weight updates
  bool stop = n == 0 || (p.count_clusters && ncl0 <= p.n_min);
  int32_t subs = 0;
  for (int r = 0; r < p.rounds && !stop; r++) {
    const uint64_t kact = stream_key(seed, p.tag_act, (uint32_t)p.level, (uint32_t)r);
    const uint64_t ktie = stream_key(seed, p.tag_tie, (uint32_t)p.level, (uint32_t)r);
    const uint64_t kprio = stream_key(seed, p.tag_prio, (uint32_t)p.level, (uint32_t)r);
    {
      ProfScope ps(ctx, PROF_ROUND_SETUP);
      BucketArgs b{g.xadj, label, nullptr, g.vwgt, n, kact, S, 0, 0, &C->stop};
      cnt.zero();
      k_bucket_count<<<grid_for(n, kThreads, grid), kThreads, 0, ctx->stream>>>(b, nkeys, cnt.get());
      GP_LAUNCH_CHECK();
      k_bucket_offsets<<<1, 1, 0, ctx->stream>>>(cnt.get(), nkeys, offs.get(), cursor.get(), &C->stop);
      GP_LAUNCH_CHECK();
      k_bucket_scatter<<<grid_for(n, kChunk, grid), kThreads, 0, ctx->stream>>>(b, nkeys, cursor.get(),
                                                                               list.get());
      GP_LAUNCH_CHECK();
    }
    // bucket sizes of the round (launch shapes, empty buckets skipped) and the stop flag
    int stop_now = 0;
    read_back(ctx, &C->stop, sizeof(int), &stop_now);
    if (stop_now) { stop = true; break; }
    read_back(ctx, offs.get(), sizeof(int32_t) * (nkeys + 1), hoffs.data());
    for (int s = 0; s < S; s++) {
      if (p.dbg_max_subrounds >= 0 && subs >= p.dbg_max_subrounds) { stop = true; break; }
      RateArgs a{};
      a.xadj = g.xadj; a.adjncy = g.adjncy; a.adjwgt = g.unit_w ? nullptr : g.adjwgt; a.vwgt = g.vwgt;
      a.label = label; a.weight = weight; a.list = list.get(); a.offs = offs.get();
      a.bound = p.bound; a.ktie = ktie; a.prop = prop.get(); a.incoming = incoming.get();
      a.stop = &C->stop; a.units = units_rate; a.label8 = label8;
      a.wlabels = label8 ? (int)nlabels : 0;
      a.dirty = dirty.get();
      if (use_dirty && r > 0) {  // in round 0 every node is still marked: the lists stay as they are
        const int k0c = s * kNumBuckets;
        GP_CUDA(cudaMemsetAsync(ccount.get() + k0c, 0, sizeof(int32_t) * kNumBuckets, ctx->stream));
        const int act = hoffs[k0c + kNumBuckets] - hoffs[k0c];
        if (act > 0) {
          k_compact_dirty<<<grid_for(act, kThreads, grid), kThreads, 0, ctx->stream>>>(
              list.get(), offs.get(), k0c, k0c + kNumBuckets, dirty.get(), clist.get(), ccount.get(), &C->stop);
          GP_LAUNCH_CHECK();
        }
        a.list = clist.get();
        a.ccount = ccount.get();
      }
      {
        ProfScope ps(ctx, p.prof_rate);
        int hcnt[kNumBuckets];
        for (int b = 0; b < kNumBuckets; b++) hcnt[b] = hoffs[s * kNumBuckets + b + 1] - hoffs[s * kNumBuckets + b];
        launch_rate<RATE_LP>(ctx, a, s * kNumBuckets, tables, nlabels, hcnt);
      }
      const int k0 = s * kNumBuckets, k1 = s * kNumBuckets + kNumBuckets;
      const int active = hoffs[k1] - hoffs[k0];
      {
        ProfScope ps(ctx, p.prof_accept);
        k_decide<<<grid_for(active, kThreads, grid), kThreads, 0, ctx->stream>>>(
            use_dirty && r > 0 ? clist.get() : list.get(), offs.get(), k0, k1, prop.get(), weight, incoming.get(),
            p.bound, mov.get(), ov_key.get(), ov_val.get(), C, kprio, use_dirty && r > 0 ? ccount.get() : nullptr);
        GP_LAUNCH_CHECK();
      }
      Counters hdr;
      const auto t_sync0 = std::chrono::steady_clock::now();
      read_back(ctx, C, sizeof(hdr), &hdr);
      sync_s += std::chrono::duration<double>(std::chrono::steady_clock::now() - t_sync0).count();
      if (hdr.stop) { stop = true; break; }
      const int nov = hdr.nov, nmov = hdr.nmov;
      subs++;
      res.overflow_total += nov;
      if (nov > res.overflow_max) res.overflow_max = nov;
      res.proposals += nov + nmov;
      if (nov > 0 && few) {
        ProfScope ps(ctx, p.prof_overflow);
        const int gsmall = grid_for(nov, 256, grid);
        GP_CUDA(cudaMemsetAsync(ovb_hw.get(), 0, sizeof(unsigned long long) * ovb_hw.count, ctx->stream));
        GP_CUDA(cudaMemsetAsync(ovb_hc.get(), 0, sizeof(int32_t) * ovb_hc.count, ctx->stream));
        k_ovb_hist<<<gsmall, 256, 0, ctx->stream>>>(ov_key.get(), ov_val.get(), nov, g.vwgt, ovb_hw.get(),
                                                    ovb_hc.get());
        GP_LAUNCH_CHECK();
        k_ovb_cut<<<(int)nlabels, 256, 0, ctx->stream>>>(ovb_hw.get(), ovb_hc.get(), weight, p.bound,
                                                        ovb_cut.get(), ovb_base.get(), ovb_m.get());
        GP_LAUNCH_CHECK();
        k_ovb_offsets<<<1, 32, 0, ctx->stream>>>(ovb_m.get(), (int)nlabels, ovb_roff.get(), ovb_cursor.get());
        GP_LAUNCH_CHECK();
        k_ovb_class<<<gsmall, 256, 0, ctx->stream>>>(ov_key.get(), ov_val.get(), nov, ovb_cut.get(),
                                                     ovb_cursor.get(), ov_acc.get(), ovb_key.get(),
                                                     ovb_idx.get());
        GP_LAUNCH_CHECK();
        k_ovb_resolve<<<(int)nlabels, 256, 0, ctx->stream>>>(ovb_key.get(), ovb_idx.get(), ovb_roff.get(),
                                                            g.vwgt, weight, ovb_base.get(), p.bound,
                                                            ov_acc.get());
        GP_LAUNCH_CHECK();
      } else if (nov > 0 && nov <= kOvSmall) {
        ProfScope ps(ctx, p.prof_overflow);
        k_ov_small<<<1, kOvSmallThreads, 0, ctx->stream>>>(ov_key.get(), ov_val.get(), nov, g.vwgt, weight,
                                                           p.bound, ov_acc.get());
        GP_LAUNCH_CHECK();
      } else if (nov > 0) {
        ProfScope ps(ctx, p.prof_overflow);
        const int kbits = bits_for(nlabels) + 32;
        radix_sort_pairs(ctx, ov_key.get(), ov_val.get(), nov, kbits);
        const int gsmall = grid_for(nov, 256, grid);
        k_fix_runs<<<gsmall, 256, 0, ctx->stream>>>(ov_key.get(), ov_val.get(), nov);
        GP_LAUNCH_CHECK();
        DBuf<int64_t> cs(ctx, (size_t)nov);
        k_ov_weights<<<gsmall, 256, 0, ctx->stream>>>(ov_val.get(), nov, g.vwgt, cs.get());
        GP_LAUNCH_CHECK();
        scan_exclusive_i64(ctx, cs.get(), cs.get(), nov, nullptr);
        k_ov_accept<<<gsmall, 256, 0, ctx->stream>>>(ov_key.get(), ov_val.get(), nov, cs.get(), g.vwgt,
                                                     weight, p.bound, ov_acc.get());
        GP_LAUNCH_CHECK();
      }
      {
        ProfScope ps(ctx, p.prof_apply);
        ApplyArgs aa{};
        aa.mov = mov.get(); aa.ov_key = ov_key.get(); aa.ov_val = ov_val.get();
        aa.ov_acc = ov_acc.get(); aa.nmov = nmov; aa.nov = nov; aa.vwgt = g.vwgt; aa.label = label;
        aa.weight = weight; aa.incoming = incoming.get(); aa.label8 = label8;
        aa.nshared = agg ? (int)nlabels : 0; aa.cnt = C;
        aa.kprio = kprio;
        aa.track = p.count_clusters ? 1 : 0;

        const int ga = grid_for((int64_t)nmov + nov, kThreads, grid);
        // the 2.5x cap: only when the accepted moves could empty more than D clusters
        const int64_t D = hdr.nclusters - p.n_min;
        if (p.count_clusters && (int64_t)nmov + nov > D) {
          if (!cap_w.get()) {
            cap_w.reset(ctx, (size_t)nlabels);
            cap_k.reset(ctx, (size_t)nlabels);
            cap_w.zero();
            cap_k.zero();
            cap_e.reset(ctx, (size_t)n);
            cap_n.reset(ctx, 1);
          }
          cap_n.zero();
          k_cap_depart<<<ga, kThreads, 0, ctx->stream>>>(aa, cap_w.get(), cap_k.get());
          GP_LAUNCH_CHECK();
          k_cap_collect<<<ga, kThreads, 0, ctx->stream>>>(aa, cap_w.get(), cap_k.get(), cap_e.get(), cap_n.get());
          GP_LAUNCH_CHECK();
          k_cap_clear<<<ga, kThreads, 0, ctx->stream>>>(aa, cap_w.get(), cap_k.get());
          GP_LAUNCH_CHECK();
          const int E = read_scalar(ctx, cap_n.get());
          if (E > D) {
            DBuf<uint32_t> dummy(ctx, (size_t)E);
            radix_sort_pairs(ctx, cap_e.get(), dummy.get(), E, 64);
            aa.cutoff = cap_e.get() + D;
            res.capped++;
          }
        }
        if (nmov + nov > 0) {
          k_apply<<<ga, kThreads, sizeof(int) * aa.nshared, ctx->stream>>>(aa);
          GP_LAUNCH_CHECK();
          if (use_dirty) {
            k_mark_dirty<<<grid_for((int64_t)(nmov + nov) * 16, kThreads, grid), kThreads, 0, ctx->stream>>>(
                mov.get(), nmov, ov_key.get(), ov_val.get(), ov_acc.get(), nov, aa.cutoff, kprio, g.xadj, g.adjncy,
                dirty.get());
            GP_LAUNCH_CHECK();
          }
        }
        const int64_t count_labels = p.count_clusters ? nlabels : 0;
        const int gc = grid_for((int64_t)nmov + nov, kThreads, grid);
        k_close<<<gc, kThreads, 0, ctx->stream>>>(aa, count_labels, (long long)p.n_min, s == S - 1 ? 1 : 0,
                                                  done.get());
        GP_LAUNCH_CHECK();
      }
    }
    if (stop) break;
  }
  Counters hc;
  read_back(ctx, C, sizeof(Counters), &hc);
  res.subrounds = subs;
  res.moves = hc.moved_total;
  res.nclusters = hc.nclusters;
  if (trace.on()) {
    const double host_s = std::chrono::duration<double>(std::chrono::steady_clock::now() - t_host0).count();
    fprintf(stderr,
            "[gp lp] %s level=%d n=%d m2=%lld labels=%lld subrounds=%d moves=%lld proposals=%lld "
            "overflow_total=%lld overflow_max=%lld capped=%d host_ms=%.2f sync_ms=%.2f ms=%.2f\n",
            p.count_clusters ? "cluster" : "refine", p.level, n, (long long)g.m2, (long long)nlabels, subs,
            (long long)res.moves, (long long)res.proposals, (long long)res.overflow_total,
            (long long)res.overflow_max, res.capped, 1000 * host_s, 1000 * sync_s, trace.ms());
  }
  if (p.count_clusters && nclusters_dev)
    GP_CUDA(cudaMemcpyAsync(nclusters_dev, &C->nclusters, sizeof(int64_t), cudaMemcpyDeviceToDevice,
                            ctx->stream));
  return res;
}

// ------------------------------------------------------- 2-hop favourites

namespace {
__global__ void k_fill_u64(uint64_t *a, int64_t n, uint64_t v) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    a[i] = v;
}
}  // namespace

void favourites_bucketed(gp_ctx *ctx, const DevGraph &g, const int32_t *label, const int32_t *size,
                         int64_t U, uint64_t kfav, DBuf<uint64_t> &keys, int32_t &count) {
  const int n = g.n;
  const int nkeys = kNumBuckets;
  const int grid = ctx->num_sms * 8;
  DBuf<int4> list(ctx, (size_t)n);
  DBuf<int32_t> cnt(ctx, (size_t)nkeys), offs(ctx, (size_t)nkeys + 1),
      cursor(ctx, (size_t)nkeys);
  BucketArgs b{g.xadj, label, size, g.vwgt, n, 0, 1, 1, U, nullptr};
  cnt.zero();
  k_bucket_count<<<grid_for(n, kThreads, grid), kThreads, 0, ctx->stream>>>(b, nkeys, cnt.get());
  GP_LAUNCH_CHECK();
  k_bucket_offsets<<<1, 1, 0, ctx->stream>>>(cnt.get(), nkeys, offs.get(), cursor.get(), nullptr);
  GP_LAUNCH_CHECK();
  k_bucket_scatter<<<grid_for(n, kChunk, grid), kThreads, 0, ctx->stream>>>(b, nkeys, cursor.get(),
                                                                           list.get());
  GP_LAUNCH_CHECK();
  int32_t total = 0;
  read_back(ctx, offs.get() + nkeys, sizeof(int32_t), &total);
  count = total;
  keys.reset(ctx, (size_t)(total > 0 ? total : 1));
  if (total == 0) return;
  k_fill_u64<<<grid_for(total, 256, grid), 256, 0, ctx->stream>>>(keys.get(), total, ~0ull);
  GP_LAUNCH_CHECK();
  RateTables tables;
  make_tables(ctx, g, tables);
  RateArgs a{};
  a.xadj = g.xadj; a.adjncy = g.adjncy; a.adjwgt = g.unit_w ? nullptr : g.adjwgt; a.vwgt = g.vwgt;
  a.label = label; a.weight = nullptr; a.list = list.get(); a.offs = offs.get();
  a.bound = U; a.ktie = kfav; a.fav_keys = keys.get(); a.stop = nullptr;
  launch_rate<RATE_FAV>(ctx, a, 0, tables, 0, nullptr);
}

}  // namespace gp
