/*
 * graphgen.c -- seeded synthetic graph generators shared by the CPU oracle
 * tests and the GPU path (tests and bench).
 *
 * This module holds no arithmetic of the partitioning method: it only draws
 * graphs.  Every graph is a simple undirected graph returned as a symmetric
 * CSR (each undirected edge stored in both rows) with rows sorted ascending,
 * no self-loops and no duplicates.  Output is identical for any thread count
 * and on any host (integer arithmetic only; no char signedness, no x86-only
 * code).
 *
 * Random words come from SplitMix64 (Steele, Lea and Flood, "Fast splittable
 * pseudorandom number generators", OOPSLA 2014): word t of stream `seed` is
 * fin(fin(seed + SALT) + (t + 1) * GAMMA), fin being the SplitMix64 output
 * finaliser.
 *
 * Generators (the input families the paper evaluates on, Table 1: the
 * Erdos-Renyi, R-MAT classes; plus grids and hand graphs for tests):
 *   gg_er     G(n, m): the first m distinct non-loop pairs in counter order,
 *             pair t = (hi32(word t) * n >> 32, lo32(word t) * n >> 32).
 *   gg_rmat   R-MAT: 2^scale nodes, ef * 2^scale sampled edges; per level a
 *             16-bit digit picks a quadrant against integer thresholds
 *             qa < qab < qabc (of 65536); symmetrised, loops and duplicate
 *             pairs removed.
 *   gg_grid2d / gg_grid3d   4- / 6-neighbour lattices, row-major ids.
 *   gg_from_pairs           any pair list, symmetrised and deduplicated.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <pthread.h>
#include <unistd.h>

#define GG_GAMMA 0x9E3779B97F4A7C15ULL
#define GG_SALT 0x632BE59BD9B4E019ULL

static inline uint64_t gg_fin(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

uint64_t gg_word(uint64_t seed, uint64_t t) {
  return gg_fin(gg_fin(seed + GG_SALT) + (t + 1) * GG_GAMMA);
}

typedef struct gg_graph {
  int32_t n;
  int64_t m2;
  int64_t *xadj; /* n+1 (int64 so that any size can be described) */
  int32_t *adjncy;
} gg_graph;

void gg_free(gg_graph *g);

/* ---------------------------------------------------------------- threads */

typedef void (*gg_body)(int64_t lo, int64_t hi, void *arg);
typedef struct { gg_body f; void *arg; int64_t lo, hi; } gg_job;

static void *gg_run(void *p) {
  gg_job *j = (gg_job *)p;
  j->f(j->lo, j->hi, j->arg);
  return NULL;
}

static int gg_threads(int want) {
  if (want > 0) return want > 256 ? 256 : want;
  long c = sysconf(_SC_NPROCESSORS_ONLN);
  if (c < 1) c = 1;
  return c > 256 ? 256 : (int)c;
}

/* Runs f over [0, total) split into nthreads contiguous ranges. */
static void gg_parallel(int64_t total, int nthreads, gg_body f, void *arg) {
  if (total <= 0) return;
  if (nthreads <= 1 || total < 4096) { f(0, total, arg); return; }
  pthread_t th[256];
  gg_job jobs[256];
  int64_t chunk = (total + nthreads - 1) / nthreads;
  int used = 0;
  for (int i = 0; i < nthreads; i++) {
    int64_t lo = (int64_t)i * chunk, hi = lo + chunk;
    if (lo >= total) break;
    if (hi > total) hi = total;
    jobs[i].f = f; jobs[i].arg = arg; jobs[i].lo = lo; jobs[i].hi = hi;
    used++;
  }
  for (int i = 1; i < used; i++) pthread_create(&th[i], NULL, gg_run, &jobs[i]);
  gg_run(&jobs[0]);
  for (int i = 1; i < used; i++) pthread_join(th[i], NULL);
}

/* ------------------------------------------------ key list -> sorted CSR */

static int cmp_i32(const void *a, const void *b) {
  int32_t x = *(const int32_t *)a, y = *(const int32_t *)b;
  return (x > y) - (x < y);
}

static void sort_i32(int32_t *a, int64_t len) {
  if (len < 2) return;
  if (len <= 24) { /* insertion sort for the common short rows */
    for (int64_t i = 1; i < len; i++) {
      int32_t x = a[i];
      int64_t j = i - 1;
      while (j >= 0 && a[j] > x) { a[j + 1] = a[j]; j--; }
      a[j + 1] = x;
    }
    return;
  }
  qsort(a, (size_t)len, sizeof(int32_t), cmp_i32);
}

/* Dynamic task pool: f(task, arg) for task in [0, ntasks). */
typedef void (*gg_task)(int64_t task, void *arg);
typedef struct { gg_task f; void *arg; int64_t ntasks; int64_t next; } gg_pool;

static void gg_pool_body(int64_t lo, int64_t hi, void *a) {
  (void)lo; (void)hi;
  gg_pool *p = (gg_pool *)a;
  for (;;) {
    int64_t t = __atomic_fetch_add(&p->next, 1, __ATOMIC_RELAXED);
    if (t >= p->ntasks) break;
    p->f(t, p->arg);
  }
}

static void gg_tasks(int64_t ntasks, int nth, gg_task f, void *arg) {
  gg_pool p = {f, arg, ntasks, 0};
  if (nth > ntasks) nth = (int)(ntasks > 0 ? ntasks : 1);
  if (nth <= 1) { gg_pool_body(0, 0, &p); return; }
  pthread_t th[256];
  gg_job jobs[256];
  for (int i = 0; i < nth; i++) { jobs[i].f = gg_pool_body; jobs[i].arg = &p; jobs[i].lo = 0; jobs[i].hi = 0; }
  for (int i = 1; i < nth; i++) pthread_create(&th[i], NULL, gg_run, &jobs[i]);
  gg_run(&jobs[0]);
  for (int i = 1; i < nth; i++) pthread_join(th[i], NULL);
}

/*
 * Directed keys (row << 32 | col, UINT64_MAX = skip) -> CSR with sorted,
 * deduplicated rows.  Keys are scattered into row-range buckets (per-thread
 * histograms, no atomics), then every bucket is counted, placed, sorted and
 * deduplicated on its own, in cache.
 */
typedef struct {
  int32_t n;
  int shift, nb, nparts;
  const uint64_t *keys;
  int64_t nkeys, chunk;
  uint64_t *bkeys;  /* keys grouped by bucket */
  int64_t *hist;    /* nparts x nb, then scatter cursors */
  int64_t *bstart;  /* nb+1 */
  int32_t *tmp;     /* cols placed by row inside each bucket */
  int64_t *rstart;  /* n+1: start of each row inside tmp */
  int64_t *deg;     /* n: deduplicated degree */
  int64_t *xadj;
  int32_t *adj;
} csr_ctx;

static void ck_hist(int64_t part, void *a) {
  csr_ctx *c = (csr_ctx *)a;
  int64_t *h = c->hist + part * c->nb;
  int64_t lo = part * c->chunk, hi = lo + c->chunk;
  if (hi > c->nkeys) hi = c->nkeys;
  for (int64_t i = lo; i < hi; i++) {
    uint64_t k = c->keys[i];
    if (k != UINT64_MAX) h[(k >> 32) >> c->shift]++;
  }
}

static void ck_scatter(int64_t part, void *a) {
  csr_ctx *c = (csr_ctx *)a;
  int64_t *h = c->hist + part * c->nb;
  int64_t lo = part * c->chunk, hi = lo + c->chunk;
  if (hi > c->nkeys) hi = c->nkeys;
  for (int64_t i = lo; i < hi; i++) {
    uint64_t k = c->keys[i];
    if (k != UINT64_MAX) c->bkeys[h[(k >> 32) >> c->shift]++] = k;
  }
}

static void ck_bucket(int64_t b, void *a) {
  csr_ctx *c = (csr_ctx *)a;
  int64_t r0 = b << c->shift, r1 = (b + 1) << c->shift;
  if (r1 > c->n) r1 = c->n;
  if (r0 >= r1) return;
  int64_t lo = c->bstart[b], hi = c->bstart[b + 1];
  /* only rows [r0, r1) are touched: buckets never share an entry */
  for (int64_t r = r0; r < r1; r++) c->deg[r] = 0;
  for (int64_t i = lo; i < hi; i++) c->deg[(int64_t)(c->bkeys[i] >> 32)]++;
  int64_t run = lo;
  for (int64_t r = r0; r < r1; r++) { c->rstart[r] = run; run += c->deg[r]; c->deg[r] = 0; }
  for (int64_t i = lo; i < hi; i++) {
    int64_t r = (int64_t)(c->bkeys[i] >> 32);
    c->tmp[c->rstart[r] + c->deg[r]++] = (int32_t)(c->bkeys[i] & 0xFFFFFFFFu);
  }
  for (int64_t r = r0; r < r1; r++) {
    int32_t *row = c->tmp + c->rstart[r];
    int64_t len = c->deg[r];
    sort_i32(row, len);
    int64_t w = 0;
    for (int64_t i = 0; i < len; i++)
      if (w == 0 || row[w - 1] != row[i]) row[w++] = row[i];
    c->deg[r] = w;
  }
}

static void ck_copy(int64_t b, void *a) {
  csr_ctx *c = (csr_ctx *)a;
  int64_t r0 = b << c->shift, r1 = (b + 1) << c->shift;
  if (r1 > c->n) r1 = c->n;
  for (int64_t r = r0; r < r1; r++)
    memcpy(c->adj + c->xadj[r], c->tmp + c->rstart[r], sizeof(int32_t) * (size_t)c->deg[r]);
}

static gg_graph *csr_from_keys(int32_t n, const uint64_t *keys, int64_t nkeys, int nth) {
  csr_ctx c;
  memset(&c, 0, sizeof c);
  c.n = n; c.keys = keys; c.nkeys = nkeys;
  int bits = 0;
  while ((1ll << bits) < (int64_t)n) bits++;
  c.shift = bits > 12 ? bits - 12 : 0;
  c.nb = (int)(((int64_t)n + (1ll << c.shift) - 1) >> c.shift);
  if (c.nb < 1) c.nb = 1;
  c.nparts = nth < 1 ? 1 : nth;
  c.chunk = (nkeys + c.nparts - 1) / c.nparts;
  if (c.chunk < 1) c.chunk = 1;
  gg_graph *g = (gg_graph *)calloc(1, sizeof(gg_graph));
  c.hist = (int64_t *)calloc((size_t)c.nparts * (size_t)c.nb, sizeof(int64_t));
  c.bstart = (int64_t *)calloc((size_t)c.nb + 1, sizeof(int64_t));
  c.bkeys = (uint64_t *)malloc(sizeof(uint64_t) * ((size_t)nkeys + 1));
  c.tmp = (int32_t *)malloc(sizeof(int32_t) * ((size_t)nkeys + 1));
  c.rstart = (int64_t *)malloc(sizeof(int64_t) * ((size_t)n + 1));
  c.deg = (int64_t *)malloc(sizeof(int64_t) * ((size_t)n + 1));
  c.xadj = (int64_t *)malloc(sizeof(int64_t) * ((size_t)n + 1));
  if (!g || !c.hist || !c.bstart || !c.bkeys || !c.tmp || !c.rstart || !c.deg || !c.xadj) goto fail;
  gg_tasks(c.nparts, nth, ck_hist, &c);
  {
    int64_t run = 0;
    for (int b = 0; b < c.nb; b++) {
      c.bstart[b] = run;
      for (int p = 0; p < c.nparts; p++) {
        int64_t t = c.hist[(int64_t)p * c.nb + b];
        c.hist[(int64_t)p * c.nb + b] = run;
        run += t;
      }
    }
    c.bstart[c.nb] = run;
  }
  gg_tasks(c.nparts, nth, ck_scatter, &c);
  gg_tasks(c.nb, nth, ck_bucket, &c);
  c.xadj[0] = 0;
  for (int32_t r = 0; r < n; r++) c.xadj[r + 1] = c.xadj[r] + c.deg[r];
  c.adj = (int32_t *)malloc(sizeof(int32_t) * ((size_t)c.xadj[n] + 1));
  if (!c.adj) goto fail;
  gg_tasks(c.nb, nth, ck_copy, &c);
  g->n = n; g->m2 = c.xadj[n]; g->xadj = c.xadj; g->adjncy = c.adj;
  free(c.hist); free(c.bstart); free(c.bkeys); free(c.tmp); free(c.rstart); free(c.deg);
  return g;
fail:
  free(g); free(c.hist); free(c.bstart); free(c.bkeys); free(c.tmp); free(c.rstart); free(c.deg);
  free(c.xadj); free(c.adj);
  return NULL;
}

/* Both directions of every pair (u << 32 | v, u < v) in `pairs`. */
typedef struct { const uint64_t *pairs; uint64_t *keys; } both_ctx;

static void both_body(int64_t lo, int64_t hi, void *a) {
  both_ctx *c = (both_ctx *)a;
  for (int64_t t = lo; t < hi; t++) {
    uint64_t p = c->pairs[t];
    if (p == UINT64_MAX) { c->keys[2 * t] = c->keys[2 * t + 1] = UINT64_MAX; continue; }
    c->keys[2 * t] = p;
    c->keys[2 * t + 1] = (p << 32) | (p >> 32);
  }
}

static gg_graph *sym_from_pairs(int32_t n, const uint64_t *pairs, int64_t npairs, int nth) {
  uint64_t *keys = (uint64_t *)malloc(sizeof(uint64_t) * (2 * (size_t)npairs + 1));
  if (!keys) return NULL;
  both_ctx c = {pairs, keys};
  gg_parallel(npairs, nth, both_body, &c);
  gg_graph *g = csr_from_keys(n, keys, 2 * npairs, nth);
  free(keys);
  return g;
}

/* ---------------------------------------------------------- Erdos-Renyi */

typedef struct { int32_t n; uint64_t seed; uint64_t *pairs; } er_ctx;

static inline uint64_t er_pair(uint64_t seed, int32_t n, uint64_t t) {
  uint64_t x = gg_word(seed, t);
  uint64_t a = ((x >> 32) * (uint64_t)n) >> 32;
  uint64_t b = ((x & 0xFFFFFFFFull) * (uint64_t)n) >> 32;
  if (a == b) return UINT64_MAX;
  return a < b ? (a << 32 | b) : (b << 32 | a);
}

static void er_draw(int64_t lo, int64_t hi, void *a) {
  er_ctx *c = (er_ctx *)a;
  for (int64_t t = lo; t < hi; t++) c->pairs[t] = er_pair(c->seed, c->n, (uint64_t)t);
}

static int in_sorted(const int32_t *row, int64_t len, int32_t v) {
  int64_t lo = 0, hi = len;
  while (lo < hi) {
    int64_t mid = (lo + hi) / 2;
    if (row[mid] < v) lo = mid + 1; else hi = mid;
  }
  return lo < len && row[lo] == v;
}

typedef struct { const gg_graph *up; uint64_t *out; } flat_ctx;

static void flat_body(int64_t lo, int64_t hi, void *a) {
  flat_ctx *c = (flat_ctx *)a;
  for (int64_t u = lo; u < hi; u++)
    for (int64_t j = c->up->xadj[u]; j < c->up->xadj[u + 1]; j++)
      c->out[j] = ((uint64_t)u << 32) | (uint32_t)c->up->adjncy[j];
}

gg_graph *gg_er(int32_t n, int64_t m, uint64_t seed, int nthreads) {
  int nth = gg_threads(nthreads);
  if (n < 2 || m < 0 || m > (int64_t)n * (n - 1) / 2) return NULL;
  er_ctx c = {n, seed, NULL};
  c.pairs = (uint64_t *)malloc(sizeof(uint64_t) * ((size_t)m + 1));
  if (!c.pairs) return NULL;
  gg_parallel(m, nth, er_draw, &c);
  /* distinct pairs among the first m counters, as upper lists (row = min) */
  gg_graph *up = csr_from_keys(n, c.pairs, m, nth);
  free(c.pairs);
  if (!up) return NULL;
  int64_t have = up->m2;
  /* top up with later counters, in order, until m distinct pairs */
  uint64_t *extra = NULL;
  int64_t nextra = 0, cap = 0;
  uint64_t t = (uint64_t)m;
  while (have < m) {
    uint64_t p = er_pair(seed, n, t++);
    if (p == UINT64_MAX) continue;
    int32_t a = (int32_t)(p >> 32), b = (int32_t)(p & 0xFFFFFFFFu);
    if (in_sorted(up->adjncy + up->xadj[a], up->xadj[a + 1] - up->xadj[a], b)) continue;
    int dup = 0;
    for (int64_t i = 0; i < nextra; i++) if (extra[i] == p) { dup = 1; break; }
    if (dup) continue;
    if (nextra == cap) {
      cap = cap ? cap * 2 : 64;
      uint64_t *ne = (uint64_t *)realloc(extra, sizeof(uint64_t) * (size_t)cap);
      if (!ne) { free(extra); gg_free(up); return NULL; }
      extra = ne;
    }
    extra[nextra++] = p;
    have++;
  }
  uint64_t *all = (uint64_t *)malloc(sizeof(uint64_t) * ((size_t)have + 1));
  if (!all) { free(extra); gg_free(up); return NULL; }
  flat_ctx fc = {up, all};
  gg_parallel(n, nth, flat_body, &fc);
  for (int64_t i = 0; i < nextra; i++) all[up->m2 + i] = extra[i];
  free(extra);
  gg_free(up);
  gg_graph *g = sym_from_pairs(n, all, have, nth);
  free(all);
  return g;
}

/* ---------------------------------------------------------------- R-MAT */

typedef struct {
  int scale;
  uint32_t qa, qab, qabc;
  uint64_t seed;
  uint64_t *pairs;
} rmat_ctx;

static void rmat_draw(int64_t lo, int64_t hi, void *a) {
  rmat_ctx *c = (rmat_ctx *)a;
  for (int64_t t = lo; t < hi; t++) {
    uint64_t r = 0, col = 0, w = 0;
    for (int l = 0; l < c->scale; l++) {
      if ((l & 3) == 0) w = gg_word(c->seed, (uint64_t)t * 8u + (uint64_t)(l >> 2));
      uint32_t d = (uint32_t)((w >> (16 * (l & 3))) & 0xFFFFu);
      uint64_t bit = 1ull << (c->scale - 1 - l);
      if (d < c->qa) {
      } else if (d < c->qab) {
        col |= bit;
      } else if (d < c->qabc) {
        r |= bit;
      } else {
        r |= bit;
        col |= bit;
      }
    }
    if (r == col) c->pairs[t] = UINT64_MAX;
    else c->pairs[t] = r < col ? (r << 32 | col) : (col << 32 | r);
  }
}

gg_graph *gg_rmat(int scale, int64_t nedges, uint32_t qa, uint32_t qab, uint32_t qabc,
                  uint64_t seed, int nthreads) {
  int nth = gg_threads(nthreads);
  if (scale < 1 || scale > 30 || nedges < 0 || !(qa <= qab && qab <= qabc && qabc <= 65536u))
    return NULL;
  rmat_ctx c = {scale, qa, qab, qabc, seed, NULL};
  c.pairs = (uint64_t *)malloc(sizeof(uint64_t) * ((size_t)nedges + 1));
  if (!c.pairs) return NULL;
  gg_parallel(nedges, nth, rmat_draw, &c);
  gg_graph *g = sym_from_pairs((int32_t)(1 << scale), c.pairs, nedges, nth);
  free(c.pairs);
  return g;
}

/* ---------------------------------------------------------------- others */

gg_graph *gg_from_pairs(int32_t n, int64_t npairs, const int32_t *a, const int32_t *b,
                        int nthreads) {
  int nth = gg_threads(nthreads);
  if (n < 1 || npairs < 0) return NULL;
  uint64_t *pairs = (uint64_t *)malloc(sizeof(uint64_t) * ((size_t)npairs + 1));
  if (!pairs) return NULL;
  for (int64_t t = 0; t < npairs; t++) {
    uint64_t x = (uint64_t)(uint32_t)a[t], y = (uint64_t)(uint32_t)b[t];
    if (x >= (uint64_t)n || y >= (uint64_t)n) { free(pairs); return NULL; }
    pairs[t] = x == y ? UINT64_MAX : (x < y ? (x << 32 | y) : (y << 32 | x));
  }
  gg_graph *g = sym_from_pairs(n, pairs, npairs, nth);
  free(pairs);
  return g;
}

gg_graph *gg_grid3d(int32_t nx, int32_t ny, int32_t nz, int nthreads) {
  int64_t n = (int64_t)nx * ny * nz;
  if (nx < 1 || ny < 1 || nz < 1 || n > INT32_MAX) return NULL;
  int64_t np = (int64_t)(nx - 1) * ny * nz + (int64_t)nx * (ny - 1) * nz + (int64_t)nx * ny * (nz - 1);
  int32_t *a = (int32_t *)malloc(sizeof(int32_t) * ((size_t)np + 1));
  int32_t *b = (int32_t *)malloc(sizeof(int32_t) * ((size_t)np + 1));
  if (!a || !b) { free(a); free(b); return NULL; }
  int64_t w = 0;
  for (int32_t z = 0; z < nz; z++)
    for (int32_t y = 0; y < ny; y++)
      for (int32_t x = 0; x < nx; x++) {
        int32_t id = (int32_t)(((int64_t)z * ny + y) * nx + x);
        if (x + 1 < nx) { a[w] = id; b[w++] = id + 1; }
        if (y + 1 < ny) { a[w] = id; b[w++] = id + nx; }
        if (z + 1 < nz) { a[w] = id; b[w++] = id + nx * ny; }
      }
  gg_graph *g = gg_from_pairs((int32_t)n, w, a, b, nthreads);
  free(a); free(b);
  return g;
}

gg_graph *gg_grid2d(int32_t nx, int32_t ny, int nthreads) { return gg_grid3d(nx, ny, 1, nthreads); }

int32_t gg_n(const gg_graph *g) { return g->n; }
int64_t gg_m2(const gg_graph *g) { return g->m2; }

/* Copies the CSR out; xadj must hold n+1 entries, adjncy m2 entries. */
void gg_copy(const gg_graph *g, int64_t *xadj, int32_t *adjncy) {
  memcpy(xadj, g->xadj, sizeof(int64_t) * ((size_t)g->n + 1));
  memcpy(adjncy, g->adjncy, sizeof(int32_t) * (size_t)g->m2);
}

void gg_free(gg_graph *g) {
  if (!g) return;
  free(g->xadj); free(g->adjncy); free(g);
}
