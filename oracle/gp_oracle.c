/*
 * gp_oracle.c -- CPU oracle of the deterministic linear-time multilevel
 * partitioner of "Linear-Time Multilevel Graph Partitioning via Edge
 * Sparsification" (Gottesbueren, Maas, Rosch, Sanders, Seemaier).
 *
 * TEST INFRASTRUCTURE ONLY: the yardstick for the GPU library.  Plain,
 * slow, single-threaded, integer-only C that takes the method's steps in the
 * paper's order.  It shares no code with the GPU library.  Where the paper
 * leaves a choice open (visit order, tie-breaking, round counts, the
 * bipartitioner, ...), the reading taken is named R1..R20 below; the GPU
 * library implements the same readings independently.
 *
 * Pinned by the CPU tests against closed forms, brute force and invariants;
 * the initial partitioner and the LP heuristics themselves have no published
 * reference values (parity unpinned beyond invariants and brute-force bounds).
 *
 * Hash (a keyed counter hash built on the SplitMix64 finaliser of Steele,
 * Lea and Flood, OOPSLA 2014):
 *   mix(z)            = SplitMix64 output finaliser
 *   key(s, t, l, r)   = mix(mix(s ^ GOLD) + (t << 48 | (l & 0xFFFF) << 32 | r))
 *   h32(key, x, y)    = top 32 bits of mix(key ^ (x << 32 | y))
 */
#include "gp_oracle.h"

#include <stdlib.h>
#include <string.h>

#define GOLD 0x9E3779B97F4A7C15ULL

/* ------------------------------------------------------------------ hash */

static uint64_t mix(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

uint64_t or_key(uint64_t seed, uint32_t tag, uint32_t level, uint32_t round) {
  uint64_t w = ((uint64_t)tag << 48) | ((uint64_t)(level & 0xFFFFu) << 32) | (uint64_t)round;
  return mix(mix(seed ^ GOLD) + w);
}

uint32_t or_h32(uint64_t key, uint32_t x, uint32_t y) {
  return (uint32_t)(mix(key ^ (((uint64_t)x << 32) | (uint64_t)y)) >> 32);
}

/* all 64 bits of the same mix: the order of the exact-count sampler */
uint64_t or_h64(uint64_t key, uint32_t x, uint32_t y) {
  return mix(key ^ (((uint64_t)x << 32) | (uint64_t)y));
}

/* ----------------------------------------------------------------- graph */

typedef struct {
  int32_t n;
  int64_t m2;
  int64_t *xadj;
  int32_t *adjncy, *vwgt, *adjwgt;
  int owns;
} og;

static og view(int32_t n, const int64_t *xadj, const int32_t *adjncy, const int32_t *vwgt,
               const int32_t *adjwgt) {
  og g;
  g.n = n;
  g.m2 = xadj[n];
  g.xadj = (int64_t *)xadj;
  g.adjncy = (int32_t *)adjncy;
  g.vwgt = (int32_t *)vwgt;
  g.adjwgt = (int32_t *)adjwgt;
  g.owns = 0;
  return g;
}

static void og_free(og *g) {
  if (g->owns) { free(g->xadj); free(g->adjncy); free(g->vwgt); free(g->adjwgt); }
  memset(g, 0, sizeof *g);
}

static int og_alloc(og *g, int32_t n, int64_t m2) {
  g->n = n;
  g->m2 = m2;
  g->owns = 1;
  g->xadj = (int64_t *)calloc((size_t)n + 1, sizeof(int64_t));
  g->adjncy = (int32_t *)malloc(sizeof(int32_t) * ((size_t)m2 + 1));
  g->vwgt = (int32_t *)malloc(sizeof(int32_t) * ((size_t)n + 1));
  g->adjwgt = (int32_t *)malloc(sizeof(int32_t) * ((size_t)m2 + 1));
  return (g->xadj && g->adjncy && g->vwgt && g->adjwgt) ? 0 : -1;
}

void or_free(void *p) { free(p); }

/* ------------------------------------------------------------ validation */

/*
 * Problem statement (Sec. 2): c(v) > 0, w(e) > 0, undirected (symmetric CSR
 * with equal weights both ways), no self-loops, rows strictly increasing.
 * Totals must fit int32: sum of c and sum of w over undirected edges.
 */
int or_validate(int32_t n, const int64_t *xadj, const int32_t *adjncy, const int32_t *vwgt,
                const int32_t *adjwgt, int64_t *W_out) {
  if (n < 0 || xadj[0] != 0) return OR_INVALID;
  int64_t W = 0, wsum = 0;
  for (int32_t v = 0; v < n; v++) {
    if (xadj[v + 1] < xadj[v]) return OR_INVALID;
    if (vwgt[v] <= 0) return OR_INVALID;
    W += vwgt[v];
    for (int64_t j = xadj[v]; j < xadj[v + 1]; j++) {
      int32_t u = adjncy[j];
      if (u < 0 || u >= n || u == v || adjwgt[j] <= 0) return OR_INVALID;
      if (j > xadj[v] && adjncy[j - 1] >= u) return OR_INVALID;
      /* the reverse entry must exist with the same weight */
      int64_t lo = xadj[u], hi = xadj[u + 1];
      while (lo < hi) {
        int64_t mid = (lo + hi) / 2;
        if (adjncy[mid] < v) lo = mid + 1; else hi = mid;
      }
      if (lo >= xadj[u + 1] || adjncy[lo] != v || adjwgt[lo] != adjwgt[j]) return OR_INVALID;
      wsum += adjwgt[j];
    }
  }
  if (W > INT32_MAX || wsum / 2 > INT32_MAX) return OR_OVERFLOW;
  if (W_out) *W_out = W;
  return OR_OK;
}

/* L_max = (1 + eps) * ceil(W / k), R2: floor of the exact value with eps in ppm. */
int64_t or_lmax(int64_t W, int32_t k, int64_t eps_ppm) {
  int64_t base = (W + k - 1) / k;
  return (int64_t)(((__int128)base * (1000000 + eps_ppm)) / 1000000);
}

/* U = c(V) / (160 k), R1: floor, at least 1 (Sec. 4.3). */
int64_t or_cluster_bound(int64_t W, int32_t k, int32_t cluster_factor) {
  int64_t U = W / ((int64_t)cluster_factor * k);
  return U < 1 ? 1 : U;
}

/* ---------------------------------------------- size-constrained LP core */

typedef struct {
  int32_t k;     /* target label */
  uint32_t prio; /* acceptance priority hash */
  int32_t v;
} prop_t;

static int cmp_u64(const void *a, const void *b) {
  uint64_t x = *(const uint64_t *)a, y = *(const uint64_t *)b;
  return (x > y) - (x < y);
}

static int prop_cmp(const void *a, const void *b) {
  const prop_t *x = (const prop_t *)a, *y = (const prop_t *)b;
  if (x->k != y->k) return x->k < y->k ? -1 : 1;
  if (x->prio != y->prio) return x->prio < y->prio ? -1 : 1;
  return (x->v > y->v) - (x->v < y->v);
}

typedef struct {
  uint32_t tag_act, tag_tie, tag_prio;
  int32_t level, rounds, subrounds;
  int64_t bound;      /* U (clustering) or L_max (refinement) */
  int count_clusters; /* clustering: track non-empty clusters and stop at n_min */
  int64_t n_min;
  int32_t dbg_max_subrounds;
  uint64_t *digests;   /* optional: label digest after each sub-round (tests) */
  int32_t max_digests;
} lp_params;

/* Digest of a labelling: sum over v of mix(v << 32 | label[v]), modulo 2^64.
 * Equal labellings give equal digests; any difference changes the digest
 * unless a 2^-64 coincidence.  Test instrumentation only. */
static uint64_t label_digest(int32_t n, const int32_t *label) {
  uint64_t d = 0;
  for (int32_t v = 0; v < n; v++) d += mix(((uint64_t)(uint32_t)v << 32) | (uint32_t)label[v]);
  return d;
}

/*
 * Size-constrained label propagation (Sec. 3, KaMinPar's LP; Sec. 4.1).
 * Synchronous sub-rounds (R4): in round r, node v is active in sub-round
 * h32(key(ACT, level, r), v, 0) mod S.  Every active node with neighbours
 * rates the labels of its neighbours on the snapshot taken at the start of
 * the sub-round: rating[K] = sum of w(v,u) over neighbours u with label K
 * (R5).  Candidates are K != own with weight[K] + c(v) <= bound.  The best
 * candidate has the largest rating, then the smallest h32(key(TIE), v, K),
 * then the smallest K (R6); v proposes to move iff its rating beats the
 * rating of its own label (own wins ties).  Per target, proposers ordered
 * by (h32(key(PRIO), v, 0), v) are accepted while the snapshot weight plus
 * the accepted weight stays within the bound (longest prefix, R7).  Stops
 * after a round without moves (R3) and, when clustering, as soon as the
 * number of non-empty clusters reaches n_min.
 *
 * The node reduction of a level is at most 2.5x (Sec. 4.3), so the clustering
 * never goes below n_min clusters (R8): with c clusters at the start of a
 * sub-round, at most D = c - n_min of them may be emptied by its moves.  All
 * accepted moves carry the key (h32(key(PRIO), v, 0), v).  A cluster all of
 * whose members leave in the sub-round is emptied at the largest key among its
 * departures (arrivals are not counted, so a refilled cluster still counts as
 * emptied).  If more than D clusters are emptied, only the moves whose key is
 * below the (D+1)-th smallest emptying key are applied: the D clusters emptied
 * first lose all their members, every other cluster keeps at least one, and
 * at least n_min clusters remain.
 */
static void lp_run(const og *g, int32_t *label, int64_t *weight, int64_t nlabels, uint64_t seed,
                   const lp_params *P, int64_t *nclusters, int32_t *subrounds_run,
                   int64_t *moves_out) {
  int32_t n = g->n;
  int64_t *rating = (int64_t *)calloc((size_t)nlabels + 1, sizeof(int64_t));
  int32_t *touched = (int32_t *)malloc(sizeof(int32_t) * ((size_t)n + 1));
  prop_t *props = (prop_t *)malloc(sizeof(prop_t) * ((size_t)n + 1));
  char *accept = (char *)malloc((size_t)n + 1);
  int32_t *size = NULL;
  int64_t *dep_w = NULL;  /* R8: weight leaving each cluster in the sub-round */
  uint64_t *dep_key = NULL, *empt = NULL;  /* R8: latest departure key; emptying keys */
  if (P->count_clusters) {
    size = (int32_t *)calloc((size_t)nlabels + 1, sizeof(int32_t));
    for (int32_t v = 0; v < n; v++) size[label[v]]++;
    dep_w = (int64_t *)calloc((size_t)nlabels + 1, sizeof(int64_t));
    dep_key = (uint64_t *)calloc((size_t)nlabels + 1, sizeof(uint64_t));
    empt = (uint64_t *)malloc(sizeof(uint64_t) * ((size_t)n + 1));
  }
  int32_t sub_done = 0;
  int64_t total_moves = 0;
  int stop = 0;
  for (int32_t r = 0; r < P->rounds && !stop; r++) {
    uint64_t kact = or_key(seed, P->tag_act, (uint32_t)P->level, (uint32_t)r);
    uint64_t ktie = or_key(seed, P->tag_tie, (uint32_t)P->level, (uint32_t)r);
    uint64_t kprio = or_key(seed, P->tag_prio, (uint32_t)P->level, (uint32_t)r);
    int64_t round_moves = 0;
    for (int32_t s = 0; s < P->subrounds; s++) {
      if (P->count_clusters && *nclusters <= P->n_min) { stop = 1; break; }
      if (P->dbg_max_subrounds >= 0 && sub_done >= P->dbg_max_subrounds) { stop = 1; break; }
      /* 1. proposals, all computed on the snapshot */
      int64_t np = 0;
      for (int32_t v = 0; v < n; v++) {
        if (g->xadj[v + 1] == g->xadj[v]) continue;
        if (or_h32(kact, (uint32_t)v, 0) % (uint32_t)P->subrounds != (uint32_t)s) continue;
        int32_t own = label[v];
        int64_t nt = 0;
        for (int64_t j = g->xadj[v]; j < g->xadj[v + 1]; j++) {
          int32_t K = label[g->adjncy[j]];
          if (rating[K] == 0) touched[nt++] = K;
          rating[K] += g->adjwgt[j];
        }
        int64_t r_own = rating[own];
        int32_t best = -1;
        int64_t best_r = 0;
        uint32_t best_h = 0;
        for (int64_t t = 0; t < nt; t++) {
          int32_t K = touched[t];
          if (K == own) continue;
          if (weight[K] + g->vwgt[v] > P->bound) continue;
          int64_t rk = rating[K];
          uint32_t hk = or_h32(ktie, (uint32_t)v, (uint32_t)K);
          if (best < 0 || rk > best_r || (rk == best_r && (hk < best_h || (hk == best_h && K < best)))) {
            best = K; best_r = rk; best_h = hk;
          }
        }
        for (int64_t t = 0; t < nt; t++) rating[touched[t]] = 0;
        if (best >= 0 && best_r > r_own) {
          props[np].k = best;
          props[np].prio = or_h32(kprio, (uint32_t)v, 0);
          props[np].v = v;
          np++;
        }
      }
      /* 2. acceptance per target: longest prefix in (prio, v) order */
      qsort(props, (size_t)np, sizeof(prop_t), prop_cmp);
      int64_t i = 0;
      while (i < np) {
        int64_t j = i;
        int32_t K = props[i].k;
        int64_t acc = weight[K];
        int blocked = 0;
        for (; j < np && props[j].k == K; j++) {
          int64_t c = g->vwgt[props[j].v];
          if (!blocked && acc + c <= P->bound) { acc += c; accept[j] = 1; }
          else { blocked = 1; accept[j] = 0; }
        }
        i = j;
      }
      /* 3. the 2.5x cap (R8): at most D = c - n_min clusters may be emptied */
      if (P->count_clusters) {
        int64_t D = *nclusters - P->n_min;
        for (int64_t t = 0; t < np; t++) {
          if (!accept[t]) continue;
          int32_t own = label[props[t].v];
          uint64_t kv = ((uint64_t)props[t].prio << 32) | (uint32_t)props[t].v;
          dep_w[own] += g->vwgt[props[t].v];
          if (kv > dep_key[own]) dep_key[own] = kv;
        }
        int64_t E = 0;
        for (int64_t t = 0; t < np; t++) {
          if (!accept[t]) continue;
          int32_t own = label[props[t].v];
          uint64_t kv = ((uint64_t)props[t].prio << 32) | (uint32_t)props[t].v;
          /* a cluster is emptied iff all of its weight leaves; count it once, at its latest key */
          if (dep_w[own] == weight[own] && kv == dep_key[own]) empt[E++] = kv;
        }
        if (E > D) {
          qsort(empt, (size_t)E, sizeof(uint64_t), cmp_u64);
          uint64_t cutoff = empt[D];
          for (int64_t t = 0; t < np; t++) {
            uint64_t kv = ((uint64_t)props[t].prio << 32) | (uint32_t)props[t].v;
            if (accept[t] && kv >= cutoff) accept[t] = 0;
          }
        }
        for (int64_t t = 0; t < np; t++) {
          int32_t own = label[props[t].v];
          dep_w[own] = 0;
          dep_key[own] = 0;
        }
      }
      /* 4. apply */
      int64_t moved = 0;
      for (int64_t t = 0; t < np; t++) {
        if (!accept[t]) continue;
        int32_t v = props[t].v, K = props[t].k, own = label[v];
        label[v] = K;
        weight[own] -= g->vwgt[v];
        weight[K] += g->vwgt[v];
        if (size) { size[own]--; size[K]++; }
        moved++;
      }
      if (size) {
        int64_t cnt = 0;
        for (int64_t K = 0; K < nlabels; K++) cnt += size[K] > 0;
        *nclusters = cnt;
      }
      round_moves += moved;
      if (P->digests && sub_done < P->max_digests) P->digests[sub_done] = label_digest(n, label);
      sub_done++;
    }
    total_moves += round_moves;
    if (round_moves == 0) break;
  }
  if (subrounds_run) *subrounds_run = sub_done;
  if (moves_out) *moves_out = total_moves;
  free(rating); free(touched); free(props); free(accept); free(size);
  free(dep_w); free(dep_key); free(empt);
}

/* ------------------------------------------------------------ clustering */

typedef struct { int32_t fav; int32_t v; } fav_t;

static int fav_cmp(const void *a, const void *b) {
  const fav_t *x = (const fav_t *)a, *y = (const fav_t *)b;
  if (x->fav != y->fav) return x->fav < y->fav ? -1 : 1;
  return (x->v > y->v) - (x->v < y->v);
}

/*
 * One clustering of G_level: LP (Sec. 3), then 2-hop clustering (Sec. 4.1,
 * only when LP shrank n by less than 2x) and isolated-node clustering
 * (Sec. 4.1, last paragraph).  label[v] = cluster id (a node id).
 *
 * 2-hop (R9): light singletons (deg > 0, alone in their cluster, 2c <= U)
 * get a favourite cluster = argmax rating over adjacent clusters ignoring U
 * (ties: smallest h32(key(FAV, level, 0), v, K), then smallest K).  Sorted by
 * (favourite, v), each favourite group is cut into runs of g = floor(U /
 * heaviest member) consecutive members; every run joins the cluster of its
 * first member.  Merges are taken in (favourite, v) order and stop once the
 * cluster count reaches n_min.
 * Isolated nodes (R10): light degree-0 nodes in id order, runs of g =
 * floor(U / heaviest light isolated node), same stop rule.
 */
/* set only for the duration of or_coarsen_traced (single-threaded use per call) */
static __thread uint64_t *g_digests = NULL;
static __thread int32_t g_max_digests = 0;

int or_cluster(int32_t n, const int64_t *xadj, const int32_t *adjncy, const int32_t *vwgt,
               const int32_t *adjwgt, int64_t U, int32_t level, uint64_t seed,
               const or_config *cfg, int32_t *label, int64_t *nclusters_out, or_level *st) {
  og g = view(n, xadj, adjncy, vwgt, adjwgt);
  int64_t *cw = (int64_t *)malloc(sizeof(int64_t) * ((size_t)n + 1));
  if (!cw) return OR_NOMEM;
  for (int32_t v = 0; v < n; v++) { label[v] = v; cw[v] = vwgt[v]; }
  int64_t nclusters = n;
  /* n_min = ceil(n * den / num): at most num/den node reduction (R8) */
  int64_t n_min = ((int64_t)n * cfg->shrink_den + cfg->shrink_num - 1) / cfg->shrink_num;
  lp_params P;
  P.tag_act = OR_TAG_ACT; P.tag_tie = OR_TAG_TIE; P.tag_prio = OR_TAG_PRIO;
  P.level = level; P.rounds = cfg->lp_rounds; P.subrounds = cfg->lp_subrounds;
  P.bound = U; P.count_clusters = 1; P.n_min = n_min;
  P.dbg_max_subrounds = cfg->dbg_max_subrounds;
  P.digests = g_digests; P.max_digests = g_max_digests;
  int32_t subs = 0;
  int64_t moves = 0;
  lp_run(&g, label, cw, n, seed, &P, &nclusters, &subs, &moves);
  if (st) { st->lp_subrounds = subs; st->lp_moves = moves; st->clusters_lp = nclusters; }

  int32_t *size = (int32_t *)calloc((size_t)n + 1, sizeof(int32_t));
  for (int32_t v = 0; v < n; v++) size[label[v]]++;

  /* 2-hop clustering */
  if (cfg->two_hop && 2 * nclusters > n && nclusters > n_min) {
    uint64_t kfav = or_key(seed, OR_TAG_FAV, (uint32_t)level, 0);
    fav_t *S = (fav_t *)malloc(sizeof(fav_t) * ((size_t)n + 1));
    int64_t *rating = (int64_t *)calloc((size_t)n + 1, sizeof(int64_t));
    int32_t *touched = (int32_t *)malloc(sizeof(int32_t) * ((size_t)n + 1));
    int64_t ns = 0;
    for (int32_t v = 0; v < n; v++) {
      if (xadj[v + 1] == xadj[v] || size[label[v]] != 1 || 2 * (int64_t)vwgt[v] > U) continue;
      int64_t nt = 0;
      for (int64_t j = xadj[v]; j < xadj[v + 1]; j++) {
        int32_t K = label[adjncy[j]];
        if (rating[K] == 0) touched[nt++] = K;
        rating[K] += adjwgt[j];
      }
      int32_t best = -1;
      int64_t best_r = 0;
      uint32_t best_h = 0;
      for (int64_t t = 0; t < nt; t++) {
        int32_t K = touched[t];
        if (K == label[v]) continue;
        int64_t rk = rating[K];
        uint32_t hk = or_h32(kfav, (uint32_t)v, (uint32_t)K);
        if (best < 0 || rk > best_r || (rk == best_r && (hk < best_h || (hk == best_h && K < best)))) {
          best = K; best_r = rk; best_h = hk;
        }
      }
      for (int64_t t = 0; t < nt; t++) rating[touched[t]] = 0;
      if (best >= 0) { S[ns].fav = best; S[ns].v = v; ns++; }
    }
    qsort(S, (size_t)ns, sizeof(fav_t), fav_cmp);
    int64_t M = nclusters - n_min, merges = 0;
    int64_t a = 0;
    while (a < ns) {
      int64_t b = a;
      int64_t cmax = 0;
      while (b < ns && S[b].fav == S[a].fav) { if (vwgt[S[b].v] > cmax) cmax = vwgt[S[b].v]; b++; }
      int64_t gsz = U / cmax; /* >= 2 since every member is light */
      for (int64_t p = 0; p < b - a; p++) {
        if (p % gsz == 0) continue;
        if (merges >= M) break;
        int32_t leader = S[a + (p / gsz) * gsz].v;
        label[S[a + p].v] = label[leader];
        merges++;
      }
      a = b;
    }
    nclusters -= merges;
    free(S); free(rating); free(touched);
  }
  if (st) st->clusters_2hop = nclusters;

  /* isolated nodes */
  if (cfg->isolated && nclusters > n_min) {
    int64_t cmax = 0, niso = 0;
    for (int32_t v = 0; v < n; v++)
      if (xadj[v + 1] == xadj[v] && 2 * (int64_t)vwgt[v] <= U) {
        niso++;
        if (vwgt[v] > cmax) cmax = vwgt[v];
      }
    if (niso >= 2) {
      int64_t gsz = U / cmax, M = nclusters - n_min, merges = 0, j = 0;
      int32_t leader = -1;
      for (int32_t v = 0; v < n && merges < M; v++) {
        if (!(xadj[v + 1] == xadj[v] && 2 * (int64_t)vwgt[v] <= U)) continue;
        if (j % gsz == 0) leader = v;
        else { label[v] = label[leader]; merges++; }
        j++;
      }
      nclusters -= merges;
    }
  }
  if (st) st->clusters_final = nclusters;
  if (nclusters_out) *nclusters_out = nclusters;
  free(cw); free(size);
  return OR_OK;
}

/* R11: coarse id = rank of the cluster id among the ids in use. */
static int32_t relabel(int32_t n, const int32_t *label, int32_t *cmap) {
  int32_t *rank = (int32_t *)malloc(sizeof(int32_t) * ((size_t)n + 1));
  for (int32_t v = 0; v < n; v++) rank[v] = 0;
  for (int32_t v = 0; v < n; v++) rank[label[v]] = 1;
  int32_t nc = 0;
  for (int32_t v = 0; v < n; v++) { int32_t used = rank[v]; rank[v] = nc; nc += used; }
  for (int32_t v = 0; v < n; v++) cmap[v] = rank[label[v]];
  free(rank);
  return nc;
}

int or_coarsen(int32_t n, const int64_t *xadj, const int32_t *adjncy, const int32_t *vwgt,
               const int32_t *adjwgt, int64_t U, int32_t level, uint64_t seed,
               const or_config *cfg, int32_t *cmap, int32_t *n_coarse, or_level *st) {
  int32_t *label = (int32_t *)malloc(sizeof(int32_t) * ((size_t)n + 1));
  if (!label) return OR_NOMEM;
  int rc = or_cluster(n, xadj, adjncy, vwgt, adjwgt, U, level, seed, cfg, label, NULL, st);
  if (rc == OR_OK) *n_coarse = relabel(n, label, cmap);
  free(label);
  return rc;
}

/*
 * or_coarsen plus the labels (cluster ids before relabelling) and, for tests,
 * the label digest after every clustering LP sub-round (at most max_digests).
 */
int or_coarsen_traced(int32_t n, const int64_t *xadj, const int32_t *adjncy, const int32_t *vwgt,
                      const int32_t *adjwgt, int64_t U, int32_t level, uint64_t seed,
                      const or_config *cfg, int32_t *label, int32_t *cmap, int32_t *n_coarse,
                      or_level *st, uint64_t *digests, int32_t max_digests) {
  g_digests = digests;
  g_max_digests = max_digests;
  int rc = or_cluster(n, xadj, adjncy, vwgt, adjwgt, U, level, seed, cfg, label, NULL, st);
  g_digests = NULL;
  g_max_digests = 0;
  if (rc == OR_OK) *n_coarse = relabel(n, label, cmap);
  return rc;
}

/* ----------------------------------------------------------- contraction */

/*
 * Cluster contraction (Sec. 2): coarse node A weighs the sum of its members'
 * weights; coarse edge {A, B}, A != B, weighs the total weight of the fine
 * edges between the clusters.  R12: rows sorted by ascending neighbour.
 */
static int contract(const og *g, const int32_t *cmap, int32_t nc, og *out) {
  int32_t n = g->n;
  int64_t *mstart = (int64_t *)calloc((size_t)nc + 1, sizeof(int64_t));
  int32_t *members = (int32_t *)malloc(sizeof(int32_t) * ((size_t)n + 1));
  int64_t *acc = (int64_t *)calloc((size_t)nc + 1, sizeof(int64_t));
  int32_t *touched = (int32_t *)malloc(sizeof(int32_t) * ((size_t)nc + 1));
  int64_t *cur = (int64_t *)calloc((size_t)nc + 1, sizeof(int64_t));
  if (!mstart || !members || !acc || !touched || !cur) return OR_NOMEM;
  for (int32_t v = 0; v < n; v++) mstart[cmap[v] + 1]++;
  for (int32_t A = 0; A < nc; A++) mstart[A + 1] += mstart[A];
  for (int32_t v = 0; v < n; v++) members[mstart[cmap[v]] + cur[cmap[v]]++] = v;
  /* upper bound on coarse entries: the fine entry count */
  int64_t cap = g->m2;
  if (og_alloc(out, nc, cap)) return OR_NOMEM;
  int64_t w = 0;
  for (int32_t A = 0; A < nc; A++) {
    out->xadj[A] = w;
    int64_t cw = 0, nt = 0;
    for (int64_t i = mstart[A]; i < mstart[A + 1]; i++) {
      int32_t v = members[i];
      cw += g->vwgt[v];
      for (int64_t j = g->xadj[v]; j < g->xadj[v + 1]; j++) {
        int32_t B = cmap[g->adjncy[j]];
        if (B == A) continue;
        if (acc[B] == 0) touched[nt++] = B;
        acc[B] += g->adjwgt[j];
      }
    }
    out->vwgt[A] = (int32_t)cw;
    /* sort the touched neighbours ascending (insertion sort: plain) */
    for (int64_t i = 1; i < nt; i++) {
      int32_t x = touched[i];
      int64_t j = i - 1;
      while (j >= 0 && touched[j] > x) { touched[j + 1] = touched[j]; j--; }
      touched[j + 1] = x;
    }
    for (int64_t t = 0; t < nt; t++) {
      out->adjncy[w] = touched[t];
      out->adjwgt[w] = (int32_t)acc[touched[t]];
      acc[touched[t]] = 0;
      w++;
    }
  }
  out->xadj[nc] = w;
  out->m2 = w;
  free(mstart); free(members); free(acc); free(touched); free(cur);
  return OR_OK;
}

/* --------------------------------------------------------- sparsification */

static int cmp_desc_i32(const void *a, const void *b) {
  int32_t x = *(const int32_t *)a, y = *(const int32_t *)b;
  return (x < y) - (x > y);
}

/*
 * Edge sparsification to m_hat edges in expectation (Sec. 4.2).
 * Weighted threshold sampling (mode 1): w_t = weight of the m_hat-th
 * heaviest undirected edge; heavier edges are kept, lighter ones dropped,
 * and an edge of weight w_t is kept iff h32(key(SPARSE, level, 0), min, max)
 * < T with T = floor((m_hat - |E>|) * 2^32 / |E=|) (R16: one Bernoulli draw
 * per edge, keyed on its endpoints so both CSR directions agree).
 * Uniform sampling (mode 2): keep iff h32(key(UNIFORM, level, 0), min, max)
 * < floor(m_hat * 2^32 / m).  Weights are kept unchanged (R17).
 */
typedef struct {
  uint64_t h;
  uint32_t lo, hi;
} heq_t;

static int heq_cmp(const void *a, const void *b) {
  const heq_t *x = (const heq_t *)a, *y = (const heq_t *)b;
  if (x->h != y->h) return x->h < y->h ? -1 : 1;
  if (x->lo != y->lo) return x->lo < y->lo ? -1 : 1;
  if (x->hi != y->hi) return x->hi < y->hi ? -1 : 1;
  return 0;
}

/*
 * Sec. 4.2 sampling of the edges of weight omega_t.  Modes: 1 T-Weight (each
 * such edge kept with probability (m_hat - |E>|) / |E=| by a hash draw), 2 UR
 * (every edge with probability m_hat / m), 3 exact-count T-Weight: of the edges
 * of weight omega_t exactly m_hat - |E>| are kept, those first in the order of
 * (64-bit hash of the endpoints, min, max), so the level keeps exactly m_hat
 * edges.
 */
static int sparsify(const og *g, int64_t m_hat, int32_t level, uint64_t seed, int mode, og *out,
                    or_sparse_stats *st) {
  int32_t n = g->n;
  int64_t m = g->m2 / 2;
  int64_t wt = 0, ng = 0, ne = 0;
  uint64_t T = 0;
  uint64_t key = or_key(seed, mode == 2 ? OR_TAG_UNIFORM : OR_TAG_SPARSE, (uint32_t)level, 0);
  int keep_all = m_hat >= m, keep_none = m_hat <= 0;
  if (!keep_all && !keep_none) {
    if (mode == 2) {
      T = (uint64_t)(((unsigned __int128)m_hat << 32) / (uint64_t)m);
    } else {
      int32_t *ws = (int32_t *)malloc(sizeof(int32_t) * ((size_t)m + 1));
      if (!ws) return OR_NOMEM;
      int64_t c = 0;
      for (int32_t u = 0; u < n; u++)
        for (int64_t j = g->xadj[u]; j < g->xadj[u + 1]; j++)
          if (u < g->adjncy[j]) ws[c++] = g->adjwgt[j];
      qsort(ws, (size_t)m, sizeof(int32_t), cmp_desc_i32);
      wt = ws[m_hat - 1];
      for (int64_t i = 0; i < m; i++) { ng += ws[i] > wt; ne += ws[i] == wt; }
      T = (uint64_t)(((unsigned __int128)(m_hat - ng) << 32) / (uint64_t)ne);
      free(ws);
    }
  }
  heq_t bound = {0, 0, 0};  /* mode 3: the last kept edge of weight omega_t in the hash order */
  if (mode == 3 && !keep_all && !keep_none) {
    heq_t *eq = (heq_t *)malloc(sizeof(heq_t) * ((size_t)ne + 1));
    if (!eq) return OR_NOMEM;
    int64_t c = 0;
    for (int32_t u = 0; u < n; u++)
      for (int64_t j = g->xadj[u]; j < g->xadj[u + 1]; j++) {
        int32_t v = g->adjncy[j];
        if (u < v && g->adjwgt[j] == wt) {
          eq[c].h = or_h64(key, (uint32_t)u, (uint32_t)v);
          eq[c].lo = (uint32_t)u;
          eq[c].hi = (uint32_t)v;
          c++;
        }
      }
    qsort(eq, (size_t)c, sizeof(heq_t), heq_cmp);
    bound = eq[m_hat - ng - 1];
    T = bound.h;
    free(eq);
  }
  if (og_alloc(out, n, g->m2)) return OR_NOMEM;
  int64_t w = 0;
  for (int32_t u = 0; u < n; u++) {
    out->vwgt[u] = g->vwgt[u];
    out->xadj[u] = w;
    for (int64_t j = g->xadj[u]; j < g->xadj[u + 1]; j++) {
      int32_t v = g->adjncy[j], ew = g->adjwgt[j];
      int keep;
      if (keep_all) keep = 1;
      else if (keep_none) keep = 0;
      else {
        uint32_t lo = (uint32_t)(u < v ? u : v), hi = (uint32_t)(u < v ? v : u);
        uint64_t h = or_h32(key, lo, hi);
        if (mode == 2) keep = h < T;
        else if (mode == 3) {
          heq_t x = {or_h64(key, lo, hi), lo, hi};
          keep = ew > wt || (ew == wt && heq_cmp(&x, &bound) <= 0);
        } else keep = ew > wt || (ew == wt && h < T);
      }
      if (keep) { out->adjncy[w] = v; out->adjwgt[w] = ew; w++; }
    }
  }
  out->xadj[n] = w;
  out->m2 = w;
  if (st) {
    st->omega_t = wt; st->n_greater = ng; st->n_equal = ne; st->threshold = T;
    st->m_in = m; st->m_out = w / 2;
  }
  return OR_OK;
}

/* ------------------------------------------------- initial partitioning */

static int32_t ceil_log2(int64_t k) {
  int32_t b = 0;
  while (((int64_t)1 << b) < k) b++;
  return b;
}

typedef struct {
  const og *g;
  int32_t k;
  int64_t eps_ppm;
  uint64_t seed;
  int32_t trials;
  int32_t *blk;
  int32_t *mark; /* subproblem id of each node while it is being split */
  int32_t *loc;  /* position of each node in its subproblem's node list */
} ip_ctx;

typedef struct { int64_t gain; int32_t j; } gain_t;

static int gain_cmp(const void *a, const void *b) {
  const gain_t *x = (const gain_t *)a, *y = (const gain_t *)b;
  if (x->gain != y->gain) return x->gain > y->gain ? -1 : 1;
  return (x->j > y->j) - (x->j < y->j);
}

/*
 * Recursive bisection of the coarsest graph (Sec. 4.3; the bipartitioner
 * is not specified in the paper, R18).  Subproblem (nodes V', k' blocks
 * starting at b0, heap id bid): k1 = ceil(k'/2) blocks go to side 1 with
 * target T1 = ceil(c(V') k1 / k') and limit L1 = floor(T1 (1e6 + eps') / 1e6),
 * eps' = eps_ppm / ceil(log2 k).  Each of the trials grows side 1 greedily
 * from empty in steps: the frontier nodes (connected to side 1) that fit
 * under L1 at the start of a step are ranked by gain 2 conn(v) - deg'(v)
 * (desc, ties: smallest id) and taken in that order while they still fit,
 * at most B = 1 + |V'| / 1024 of them per step (one at a time below 1024
 * nodes); with no such frontier node the step takes the node of smallest
 * (h32(key(IP, 0, bid), v, t), v) that fits.  Growing stops once side 1
 * weighs >= T1 or nothing fits.  The trial with the
 * smallest cut (ties: lowest t) wins; recurse on both sides.
 */
/* moves local node j to side 1 and raises its neighbours' connection */
static void add_to_side1(ip_ctx *C, uint32_t bid, int32_t j, const int32_t *V, char *in1, int64_t *conn,
                         int64_t *w1) {
  const og *g = C->g;
  int32_t v = V[j];
  in1[j] = 1;
  *w1 += g->vwgt[v];
  for (int64_t e = g->xadj[v]; e < g->xadj[v + 1]; e++) {
    int32_t u = g->adjncy[e];
    if (C->mark[u] == (int32_t)bid) conn[C->loc[u]] += g->adjwgt[e];
  }
}

static void ip_bisect(ip_ctx *C, int32_t *V, int32_t nv, int32_t kk, int32_t b0, uint32_t bid) {
  const og *g = C->g;
  if (nv == 0) return;
  if (kk == 1) {
    for (int32_t j = 0; j < nv; j++) C->blk[V[j]] = b0;
    return;
  }
  int32_t k1 = (kk + 1) / 2, k2 = kk - k1;
  int64_t W = 0;
  for (int32_t j = 0; j < nv; j++) {
    C->mark[V[j]] = (int32_t)bid;
    C->loc[V[j]] = j;
    W += g->vwgt[V[j]];
  }
  int64_t T1 = (W * k1 + kk - 1) / kk;
  int64_t eps_l = C->eps_ppm / ceil_log2(C->k);
  int64_t L1 = (int64_t)(((__int128)T1 * (1000000 + eps_l)) / 1000000);
  int64_t *Dp = (int64_t *)calloc((size_t)nv, sizeof(int64_t));
  int64_t *conn = (int64_t *)malloc(sizeof(int64_t) * (size_t)nv);
  uint32_t *hv = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)nv);
  char *in1 = (char *)malloc((size_t)nv);
  char *best_in1 = (char *)malloc((size_t)nv);
  gain_t *F = (gain_t *)malloc(sizeof(gain_t) * ((size_t)nv + 1));
  const int64_t B = 1 + nv / 1024; /* nodes taken per growing step */
  for (int32_t j = 0; j < nv; j++) {
    int32_t v = V[j];
    for (int64_t e = g->xadj[v]; e < g->xadj[v + 1]; e++)
      if (C->mark[g->adjncy[e]] == (int32_t)bid) Dp[j] += g->adjwgt[e];
  }
  uint64_t kip = or_key(C->seed, OR_TAG_IP, 0, bid);
  int64_t best_cut = -1;
  for (int32_t t = 0; t < C->trials; t++) {
    for (int32_t j = 0; j < nv; j++) {
      conn[j] = 0;
      in1[j] = 0;
      hv[j] = or_h32(kip, (uint32_t)V[j], (uint32_t)t);
    }
    int64_t w1 = 0;
    while (w1 < T1) {
      /* the admissible frontier at the start of the step, by (gain desc, id asc) */
      int32_t nf = 0, bn = -1;
      for (int32_t j = 0; j < nv; j++) {
        if (in1[j] || w1 + g->vwgt[V[j]] > L1) continue;
        if (conn[j] > 0) {
          F[nf].gain = 2 * conn[j] - Dp[j];
          F[nf].j = j;
          nf++;
        } else if (bn < 0 || hv[j] < hv[bn]) {
          bn = j;
        }
      }
      if (nf > 0) {
        qsort(F, (size_t)nf, sizeof(gain_t), gain_cmp);
        int64_t taken = 0;
        for (int32_t f = 0; f < nf && taken < B && w1 < T1; f++) {
          int32_t j = F[f].j;
          if (w1 + g->vwgt[V[j]] > L1) continue; /* no longer fits (nor ever will) */
          add_to_side1(C, bid, j, V, in1, conn, &w1);
          taken++;
        }
      } else if (bn >= 0) {
        add_to_side1(C, bid, bn, V, in1, conn, &w1);
      } else {
        break;
      }
    }
    int64_t cut = 0;
    for (int32_t j = 0; j < nv; j++) {
      if (!in1[j]) continue;
      int32_t v = V[j];
      for (int64_t e = g->xadj[v]; e < g->xadj[v + 1]; e++) {
        int32_t u = g->adjncy[e];
        if (C->mark[u] == (int32_t)bid && !in1[C->loc[u]]) cut += g->adjwgt[e];
      }
    }
    if (best_cut < 0 || cut < best_cut) {
      best_cut = cut;
      memcpy(best_in1, in1, (size_t)nv);
    }
  }
  int32_t *V1 = (int32_t *)malloc(sizeof(int32_t) * (size_t)nv);
  int32_t *V2 = (int32_t *)malloc(sizeof(int32_t) * (size_t)nv);
  int32_t n1 = 0, n2 = 0;
  for (int32_t j = 0; j < nv; j++) {
    if (best_in1[j]) V1[n1++] = V[j]; else V2[n2++] = V[j];
  }
  free(Dp); free(conn); free(hv); free(in1); free(best_in1); free(F);
  ip_bisect(C, V1, n1, k1, b0, 2 * bid);
  ip_bisect(C, V2, n2, k2, b0 + k1, 2 * bid + 1);
  free(V1); free(V2);
}

/*
 * R19: while some block exceeds L_max, move from the heaviest block A
 * (ties: smallest id) to the lightest block B (ties: smallest id) the node
 * of A that fits into B and loses the least cut, conn(v, A) - conn(v, B)
 * (ties: smallest id); stop when nothing fits.
 */
static int64_t rebalance(const og *g, int32_t k, int64_t Lmax, int32_t *blk) {
  int64_t *bw = (int64_t *)calloc((size_t)k, sizeof(int64_t));
  for (int32_t v = 0; v < g->n; v++) bw[blk[v]] += g->vwgt[v];
  int64_t moves = 0;
  for (int64_t it = 0; it <= (int64_t)g->n; it++) {
    int32_t A = 0, B = 0;
    for (int32_t b = 1; b < k; b++) {
      if (bw[b] > bw[A]) A = b;
      if (bw[b] < bw[B]) B = b;
    }
    if (bw[A] <= Lmax || A == B) break;
    int32_t best = -1;
    int64_t best_d = 0;
    for (int32_t v = 0; v < g->n; v++) {
      if (blk[v] != A || bw[B] + g->vwgt[v] > Lmax) continue;
      int64_t ca = 0, cb = 0;
      for (int64_t e = g->xadj[v]; e < g->xadj[v + 1]; e++) {
        int32_t b = blk[g->adjncy[e]];
        if (b == A) ca += g->adjwgt[e];
        else if (b == B) cb += g->adjwgt[e];
      }
      if (best < 0 || ca - cb < best_d) { best = v; best_d = ca - cb; }
    }
    if (best < 0) break;
    blk[best] = B;
    bw[A] -= g->vwgt[best];
    bw[B] += g->vwgt[best];
    moves++;
  }
  free(bw);
  return moves;
}

int or_initial_partition(int32_t n, const int64_t *xadj, const int32_t *adjncy,
                         const int32_t *vwgt, const int32_t *adjwgt, int32_t k, int64_t eps_ppm,
                         uint64_t seed, int32_t trials, int32_t *blk) {
  og g = view(n, xadj, adjncy, vwgt, adjwgt);
  ip_ctx C;
  C.g = &g; C.k = k; C.eps_ppm = eps_ppm; C.seed = seed; C.trials = trials; C.blk = blk;
  C.mark = (int32_t *)malloc(sizeof(int32_t) * ((size_t)n + 1));
  C.loc = (int32_t *)malloc(sizeof(int32_t) * ((size_t)n + 1));
  int32_t *V = (int32_t *)malloc(sizeof(int32_t) * ((size_t)n + 1));
  if (!C.mark || !C.loc || !V) return OR_NOMEM;
  for (int32_t v = 0; v < n; v++) { V[v] = v; C.mark[v] = 0; blk[v] = 0; }
  ip_bisect(&C, V, n, k, 0, 1);
  free(C.mark); free(C.loc); free(V);
  return OR_OK;
}

int64_t or_rebalance(int32_t n, const int64_t *xadj, const int32_t *adjncy, const int32_t *vwgt,
                     const int32_t *adjwgt, int32_t k, int64_t Lmax, int32_t *blk) {
  og g = view(n, xadj, adjncy, vwgt, adjwgt);
  return rebalance(&g, k, Lmax, blk);
}

/* -------------------------------------------------------------- refinement */

/*
 * Size-constrained LP refinement (Sec. 3 uncoarsening, Sec. 4.3): labels are
 * the k blocks, the bound is L_max, the own rating is the connection to the
 * current block, and only strictly improving moves are proposed (R20).
 */
int or_refine(int32_t n, const int64_t *xadj, const int32_t *adjncy, const int32_t *vwgt,
              const int32_t *adjwgt, int32_t k, int64_t Lmax, int32_t level, uint64_t seed,
              const or_config *cfg, int32_t *blk, int64_t *moves_out) {
  og g = view(n, xadj, adjncy, vwgt, adjwgt);
  int64_t *bw = (int64_t *)calloc((size_t)k + 1, sizeof(int64_t));
  if (!bw) return OR_NOMEM;
  for (int32_t v = 0; v < n; v++) bw[blk[v]] += vwgt[v];
  lp_params P;
  P.tag_act = OR_TAG_RACT; P.tag_tie = OR_TAG_RTIE; P.tag_prio = OR_TAG_RPRIO;
  P.level = level; P.rounds = cfg->ref_rounds; P.subrounds = cfg->lp_subrounds;
  P.bound = Lmax; P.count_clusters = 0; P.n_min = 0;
  P.dbg_max_subrounds = -1;
  P.digests = NULL; P.max_digests = 0;
  int64_t moves = 0;
  lp_run(&g, blk, bw, k, seed, &P, NULL, NULL, &moves);
  if (moves_out) *moves_out = moves;
  free(bw);
  return OR_OK;
}

/* cut = sum over i < j of w(E_ij) (Sec. 2) = half the CSR entries across blocks */
int64_t or_cut(int32_t n, const int64_t *xadj, const int32_t *adjncy, const int32_t *adjwgt,
               const int32_t *blk) {
  int64_t cut = 0;
  for (int32_t v = 0; v < n; v++)
    for (int64_t e = xadj[v]; e < xadj[v + 1]; e++)
      if (blk[adjncy[e]] != blk[v]) cut += adjwgt[e];
  return cut / 2;
}

/* ------------------------------------------------- exported graph steps */

/* Output graphs are malloc'ed here; free each array with or_free. */
int or_contract(int32_t n, const int64_t *xadj, const int32_t *adjncy, const int32_t *vwgt,
                const int32_t *adjwgt, const int32_t *cmap, int32_t nc, int64_t **oxadj,
                int32_t **oadjncy, int32_t **ovwgt, int32_t **oadjwgt) {
  og g = view(n, xadj, adjncy, vwgt, adjwgt), out;
  memset(&out, 0, sizeof out);
  int rc = contract(&g, cmap, nc, &out);
  *oxadj = out.xadj; *oadjncy = out.adjncy; *ovwgt = out.vwgt; *oadjwgt = out.adjwgt;
  return rc;
}

/*
 * Modularity of a clustering (Sec. 5): with e_ij the fraction of the edge
 * weight running from cluster i to cluster j (each direction counted, so the
 * fractions sum to one), a_i = sum_j e_ij, Q_C = sum_i (e_ii - a_i^2) and
 * alpha_C = max_i a_i; Lemma 2 bounds the weight fraction inside clusters by
 * Q_C <= sum_i e_ii <= Q_C + alpha_C, so 1 - Q_C - alpha_C bounds the fraction
 * between clusters from below.  Returned as exact integers over the CSR
 * entries: out[0] weight inside clusters, out[1] total weight (both
 * directions), out[2] largest cluster volume, out[3] sum of squared volumes
 * (unsigned).  label[v] must lie in [0, nlabels).
 */
int or_modularity(int32_t n, const int64_t *xadj, const int32_t *adjncy, const int32_t *adjwgt,
                  const int32_t *label, int32_t nlabels, int64_t *out) {
  uint64_t *vol = (uint64_t *)calloc((size_t)nlabels + 1, sizeof(uint64_t));
  if (!vol) return OR_NOMEM;
  int64_t win = 0, wtot = 0;
  for (int32_t u = 0; u < n; u++) {
    if (label[u] < 0 || label[u] >= nlabels) { free(vol); return OR_INVALID; }
    for (int64_t j = xadj[u]; j < xadj[u + 1]; j++) {
      int32_t v = adjncy[j];
      if (label[v] < 0 || label[v] >= nlabels) { free(vol); return OR_INVALID; }
      wtot += adjwgt[j];
      vol[label[u]] += (uint64_t)adjwgt[j];
      if (label[u] == label[v]) win += adjwgt[j];
    }
  }
  uint64_t vmax = 0, sq = 0;
  for (int32_t i = 0; i < nlabels; i++) {
    if (vol[i] > vmax) vmax = vol[i];
    sq += vol[i] * vol[i];
  }
  free(vol);
  out[0] = win;
  out[1] = wtot;
  out[2] = (int64_t)vmax;
  out[3] = (int64_t)sq;
  return OR_OK;
}

int or_sparsify(int32_t n, const int64_t *xadj, const int32_t *adjncy, const int32_t *vwgt,
                const int32_t *adjwgt, int64_t m_hat, int32_t level, uint64_t seed, int32_t mode,
                int64_t **oxadj, int32_t **oadjncy, int32_t **ovwgt, int32_t **oadjwgt,
                or_sparse_stats *st) {
  og g = view(n, xadj, adjncy, vwgt, adjwgt), out;
  memset(&out, 0, sizeof out);
  int rc = sparsify(&g, m_hat, level, seed, mode, &out, st);
  *oxadj = out.xadj; *oadjncy = out.adjncy; *ovwgt = out.vwgt; *oadjwgt = out.adjwgt;
  return rc;
}

/* m_hat = min(tau_e |E_i|, tau_d |E_i| / |V_i| * |V_i+1|), R14: floor (Alg. 1). */
int64_t or_m_hat(int64_t m, int64_t n, int64_t n_next, const or_config *cfg) {
  int64_t a = (int64_t)(((__int128)m * cfg->tau_e_num) / cfg->tau_e_den);
  if (n <= 0) return a;
  int64_t b = (int64_t)(((__int128)m * n_next * cfg->tau_d_num) / ((__int128)cfg->tau_d_den * n));
  return a < b ? a : b;
}

/* R15: sparsify iff |E'| > rho * m_hat (strict, Alg. 1). */
int or_trigger(int64_t m_coarse, int64_t m_hat, const or_config *cfg) {
  return (__int128)m_coarse * cfg->rho_den > (__int128)cfg->rho_num * m_hat;
}

/* ------------------------------------------------------- full partitioner */

/*
 * The coarsening loop of Alg. 1: G[0] is the input; fills G[1..L] and the
 * coarse-id maps C[0..L-1] (owned: free with free / og_free); returns L.
 */
static int32_t coarsen_hierarchy(og *G, int32_t **C, int32_t k, int64_t U, uint64_t seed,
                                 const or_config *cfg, or_stats *st) {
  int32_t L = 0;
  int32_t maxl = cfg->max_levels < OR_MAX_LEVELS ? cfg->max_levels : OR_MAX_LEVELS;
  while ((int64_t)G[L].n > (int64_t)cfg->coarsest_factor * k && L < maxl) {
    og *g = &G[L];
    or_level lv;
    memset(&lv, 0, sizeof lv);
    int32_t *cmap = (int32_t *)malloc(sizeof(int32_t) * ((size_t)g->n + 1));
    int32_t nc = 0;
    or_coarsen(g->n, g->xadj, g->adjncy, g->vwgt, g->adjwgt, U, L + 1, seed, cfg, cmap, &nc, &lv);
    og Gc;
    memset(&Gc, 0, sizeof Gc);
    contract(g, cmap, nc, &Gc);
    lv.n = g->n;
    lv.n_next = nc;
    lv.m = g->m2 / 2;
    lv.m_coarse = Gc.m2 / 2;
    if ((int64_t)nc * cfg->min_shrink_num > (int64_t)g->n * cfg->min_shrink_den) {
      og_free(&Gc);
      free(cmap);
      break;
    }
    lv.m_hat = or_m_hat(lv.m, g->n, nc, cfg);
    lv.triggered = cfg->sparsifier != 0 && or_trigger(lv.m_coarse, lv.m_hat, cfg);
    if (lv.triggered) {
      og Gs;
      memset(&Gs, 0, sizeof Gs);
      or_sparse_stats ss;
      sparsify(&Gc, lv.m_hat, L + 2, seed, cfg->sparsifier, &Gs, &ss);
      lv.omega_t = (int32_t)ss.omega_t;
      lv.n_greater = ss.n_greater;
      lv.n_equal = ss.n_equal;
      lv.threshold = ss.threshold;
      og_free(&Gc);
      Gc = Gs;
    }
    lv.m_next = Gc.m2 / 2;
    if (st) st->lv[L] = lv;
    C[L] = cmap;
    G[L + 1] = Gc;
    L++;
  }
  return L;
}

/*
 * Multilevel partitioning (Sec. 2, Alg. 1, Sec. 4.3): coarsen until
 * n <= coarsest_factor * k or the shrink is too small (R13: n' * 21 > n * 20),
 * sparsifying each coarse graph that exceeds rho * m_hat; recursive
 * bisection of the coarsest graph plus R19; then project and refine level
 * by level.  Hash levels: coarsening G_i uses level i (G_1 = input), the
 * sparsifier producing G_{i+1} uses level i+1, refining G_i uses level i.
 */
int or_partition(int32_t n, const int64_t *xadj, const int32_t *adjncy, const int32_t *vwgt,
                 const int32_t *adjwgt, int32_t k, int64_t eps_ppm, uint64_t seed,
                 const or_config *cfg, int32_t *blocks, int64_t *cut_out, or_stats *st) {
  if (k < 1 || eps_ppm < 1) return OR_INVALID;
  int64_t W = 0;
  int rc = or_validate(n, xadj, adjncy, vwgt, adjwgt, &W);
  if (rc != OR_OK) return rc;
  int64_t Lmax = or_lmax(W, k, eps_ppm);
  for (int32_t v = 0; v < n; v++)
    if (vwgt[v] > Lmax) return OR_INFEASIBLE;
  if (st) { memset(st, 0, sizeof *st); st->W = W; st->Lmax = Lmax; }
  if (k == 1 || n == 0) {
    for (int32_t v = 0; v < n; v++) blocks[v] = 0;
    if (cut_out) *cut_out = 0;
    if (st) st->n_coarsest = n;
    return OR_OK;
  }
  int64_t U = or_cluster_bound(W, k, cfg->cluster_factor);
  if (st) st->U = U;
  og G[OR_MAX_LEVELS + 1];
  int32_t *C[OR_MAX_LEVELS + 1];
  G[0] = view(n, xadj, adjncy, vwgt, adjwgt);
  int32_t L = coarsen_hierarchy(G, C, k, U, seed, cfg, st);
  if (st) { st->levels = L; st->n_coarsest = G[L].n; }
  /* initial partition of the coarsest graph */
  og *gc = &G[L];
  int32_t *blk = (int32_t *)malloc(sizeof(int32_t) * ((size_t)gc->n + 1));
  or_initial_partition(gc->n, gc->xadj, gc->adjncy, gc->vwgt, gc->adjwgt, k, eps_ppm, seed,
                       cfg->ip_trials, blk);
  if (st) st->ip_cut = or_cut(gc->n, gc->xadj, gc->adjncy, gc->adjwgt, blk);
  int64_t rb = rebalance(gc, k, Lmax, blk);
  if (st) st->rebalance_moves = rb;
  or_refine(gc->n, gc->xadj, gc->adjncy, gc->vwgt, gc->adjwgt, k, Lmax, L + 1, seed, cfg, blk, NULL);
  for (int32_t i = L - 1; i >= 0; i--) {
    og *g = &G[i];
    int32_t *fine = (int32_t *)malloc(sizeof(int32_t) * ((size_t)g->n + 1));
    for (int32_t v = 0; v < g->n; v++) fine[v] = blk[C[i][v]];
    free(blk);
    blk = fine;
    or_refine(g->n, g->xadj, g->adjncy, g->vwgt, g->adjwgt, k, Lmax, i + 1, seed, cfg, blk, NULL);
  }
  memcpy(blocks, blk, sizeof(int32_t) * (size_t)n);
  free(blk);
  int64_t cut = or_cut(n, xadj, adjncy, adjwgt, blocks);
  if (cut_out) *cut_out = cut;
  if (st) st->cut = cut;
  for (int32_t i = 0; i < L; i++) { free(C[i]); og_free(&G[i + 1]); }
  return OR_OK;
}

/*
 * The coarsening phase alone (Alg. 1 with the clustering of Sec. 4.1 and the
 * sparsifier of Sec. 4.2) on a validated graph; fills the per-level records
 * of st and frees the hierarchy.  Used to time the method's coarsening.
 */
int or_coarsen_only(int32_t n, const int64_t *xadj, const int32_t *adjncy, const int32_t *vwgt,
                    const int32_t *adjwgt, int32_t k, uint64_t seed, const or_config *cfg,
                    or_stats *st) {
  if (k < 1) return OR_INVALID;
  int64_t W = 0;
  for (int32_t v = 0; v < n; v++) W += vwgt[v];
  if (st) { memset(st, 0, sizeof *st); st->W = W; }
  int64_t U = or_cluster_bound(W, k, cfg->cluster_factor);
  if (st) st->U = U;
  og G[OR_MAX_LEVELS + 1];
  int32_t *C[OR_MAX_LEVELS + 1];
  G[0] = view(n, xadj, adjncy, vwgt, adjwgt);
  int32_t L = coarsen_hierarchy(G, C, k, U, seed, cfg, st);
  if (st) { st->levels = L; st->n_coarsest = G[L].n; }
  for (int32_t i = 0; i < L; i++) { free(C[i]); og_free(&G[i + 1]); }
  return OR_OK;
}
