// lp_rate.cuh -- rating one node per lane group (Sec. 3: a node rates the
// labels of its neighbours by the summed edge weight; readings R5, R6).
//
// A group of G lanes rates one node of degree <= G * E, each lane holding up
// to E neighbours; the groups of a warp rate 32/G nodes side by side.  Equal
// labels are summed in a 2 G E slot table per group in shared memory; the
// lane that claims a label's slot speaks for the label.  The best candidate
// is the label != own of largest rating (admissible: its weight plus the
// node's weight within the bound), ties by the smallest h32(ktie, v, L), then
// the smallest label; the node proposes iff that rating beats its own
// label's (own wins ties).  With the label weights in shared memory every
// candidate is checked up front; otherwise only the leading candidate's
// weight is read, and the remaining candidates' weights only when it does not
// fit.  In favourite mode (2-hop clustering, Sec. 4.1) the bound and the own
// label's rating play no part.
#pragma once
#include "gp_internal.cuh"

namespace gp {

template <int G, int E>
struct GroupTable {
  static constexpr int TS = 2 * G * E;
  static constexpr int BITS = TS == 16 ? 4 : TS == 32 ? 5 : TS == 64 ? 6 : TS == 128 ? 7 : 8;
  static_assert((1 << BITS) == TS, "table size");
};

// Returns the chosen label (0xFFFFFFFF: none).  All lanes of the warp call it
// together (gmask: the caller's group); tk / tv: the group's TS slots, empty
// (-1 / 0) on entry and left empty.  label8 (may be null) replaces label for
// the gathers.  weight: global label weights (unused with s_wl or FAV).
// stable: no label other than own is rated above own, admissible or not, so
// the node cannot propose until a neighbour's label changes (not FAV).
template <int G, int E, bool FAV>
__device__ __forceinline__ unsigned rate_group(const int32_t *__restrict__ adjncy, const int32_t *__restrict__ adjwgt,
                                               const int32_t *label, const uint8_t *label8, const int32_t *weight,
                                               const int *s_wl, int64_t bound, uint64_t ktie, int v, int st,
                                               int deg, int own, int cv, int *tk, int *tv, unsigned gmask, int gl,
                                               bool stream_rows, int &ncand, bool &stable) {
  constexpr int TS = GroupTable<G, E>::TS;
  constexpr int BITS = GroupTable<G, E>::BITS;
  int L[E], w[E], slot[E], sum[E];
  bool lead[E];
#pragma unroll
  for (int e = 0; e < E; e++) {
    const int j = gl + e * G;
    const bool ok = j < deg;
    int u = 0;
    if (ok) {
      u = stream_rows ? __ldcs(adjncy + st + j) : adjncy[st + j];
      w[e] = stream_rows ? __ldcs(adjwgt + st + j) : adjwgt[st + j];
    } else {
      w[e] = 0;
    }
    L[e] = u;
    if (!ok) L[e] = -1;
  }
#pragma unroll
  for (int e = 0; e < E; e++)
    if (L[e] >= 0) L[e] = label8 ? (int)label8[L[e]] : label[L[e]];
#pragma unroll
  for (int e = 0; e < E; e++) {
    slot[e] = -1;
    lead[e] = false;
    if (L[e] < 0) continue;
    unsigned sl = ((unsigned)L[e] * 2654435761u) >> (32 - BITS);
    for (int probe = 0; probe < TS; probe++) {  // bounded: at most G E labels in 2 G E slots
      const int prev = atomicCAS(&tk[sl], -1, L[e]);
      if (prev == -1) { lead[e] = true; break; }
      if (prev == L[e]) break;
      sl = (sl + 1) & (TS - 1);
    }
    slot[e] = (int)sl;
    atomicAdd(&tv[sl], w[e]);
  }
  __syncwarp();
  unsigned own_loc = 0;
#pragma unroll
  for (int e = 0; e < E; e++) {
    sum[e] = lead[e] ? tv[slot[e]] : 0;
    if (lead[e] && L[e] == own) own_loc = (unsigned)sum[e];
  }
  __syncwarp();
#pragma unroll
  for (int e = 0; e < E; e++)
    if (lead[e]) { tk[slot[e]] = -1; tv[slot[e]] = 0; }
  const int own_r = FAV ? -1 : (int)__reduce_max_sync(gmask, own_loc);
  stable = false;
  if (!FAV) {
    unsigned rl_all = 0;
#pragma unroll
    for (int e = 0; e < E; e++)
      if (lead[e] && L[e] != own) rl_all = max(rl_all, (unsigned)sum[e]);
    stable = (int)__reduce_max_sync(gmask, rl_all) <= own_r;
  }
  bool alive[E];
  ncand = 0;
#pragma unroll
  for (int e = 0; e < E; e++) {
    alive[e] = lead[e] && L[e] != own;
    ncand += alive[e] ? 1 : 0;
    if (!FAV && s_wl && alive[e]) alive[e] = (int64_t)s_wl[L[e]] + cv <= bound;
  }
  // no label rated above own (admissible or not): nothing to propose, the choice is skipped
  bool eager = FAV || s_wl != nullptr, searching = v >= 0 && (FAV || !stable);
  unsigned best = 0xFFFFFFFFu;
  for (int it = 0; it < 3; it++) {  // lazy pass, eager pass, one to find nothing left
    if (!__any_sync(0xFFFFFFFFu, searching)) break;
    if (!FAV && eager && !s_wl) {
#pragma unroll
      for (int e = 0; e < E; e++)
        if (searching && alive[e] && (int64_t)weight[L[e]] + cv > bound) alive[e] = false;
    }
    unsigned rl = 0;
#pragma unroll
    for (int e = 0; e < E; e++)
      if (searching && alive[e]) rl = max(rl, (unsigned)sum[e] + 1u);
    const int r = (int)__reduce_max_sync(gmask, rl) - 1;
    if (r < 0 || r <= own_r) searching = false;
    unsigned hl = 0xFFFFFFFFu, hv[E];
#pragma unroll
    for (int e = 0; e < E; e++) {
      hv[e] = (searching && alive[e] && sum[e] == r) ? h32(ktie, (uint32_t)v, (uint32_t)L[e]) : 0xFFFFFFFFu;
      hl = min(hl, hv[e]);
    }
    const unsigned hmin = __reduce_min_sync(gmask, hl);
    unsigned cl = 0xFFFFFFFFu;
#pragma unroll
    for (int e = 0; e < E; e++)
      if (searching && alive[e] && sum[e] == r && hv[e] == hmin) cl = min(cl, (unsigned)L[e]);
    const unsigned cL = __reduce_min_sync(gmask, cl);
    if (eager) {
      if (searching) { best = cL; searching = false; }
    } else {
      bool holder = false;
#pragma unroll
      for (int e = 0; e < E; e++) holder = holder || (searching && alive[e] && (unsigned)L[e] == cL);
      const unsigned fits = holder && (int64_t)weight[cL] + cv <= bound ? 1u : 0u;
      if (__reduce_or_sync(gmask, fits) && searching) { best = cL; searching = false; }
#pragma unroll
      for (int e = 0; e < E; e++) alive[e] = alive[e] && (unsigned)L[e] != cL;
      eager = true;
    }
  }
  return best;
}

}  // namespace gp
