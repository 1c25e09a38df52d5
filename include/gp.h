/*
 * gp.h -- C-ABI of the GB300 library for linear-time multilevel graph
 * partitioning via edge sparsification (Gottesbueren, Maas, Rosch, Sanders,
 * Seemaier, "Linear-Time Multilevel Graph Partitioning via Edge
 * Sparsification").
 *
 * Problem (Sec. 2): an undirected graph G = (V, E, c, w) with node weights
 * c > 0 and edge weights w > 0 is split into k blocks of weight at most
 * L_max = (1 + eps) * ceil(c(V) / k), minimising the cut, the total weight
 * of edges between blocks.
 *
 * Graphs are symmetric CSR arrays in DEVICE memory: every undirected edge is
 * stored in both rows, rows hold no self-loops and no duplicates.  Ids and
 * weights are int32; xadj is int32 (at most 2^31 - 1 entries).  All work is
 * ordered on the context's stream; functions that return a host scalar
 * synchronise that stream before returning.  No function throws; every
 * function returns a gp_status, and on error the outputs are undefined and
 * gp_last_error() describes the failure.  Results are deterministic: a call
 * with the same inputs, parameters and seed returns the same bits, and equal
 * those of the CPU oracle of the same method.
 */
#ifndef GP_H
#define GP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  GP_OK = 0,
  GP_ERR_INVALID = 1,    /* malformed graph or argument */
  GP_ERR_INFEASIBLE = 2, /* a node is heavier than L_max */
  GP_ERR_OVERFLOW = 3,   /* total node or edge weight exceeds 2^31 - 1 */
  GP_ERR_OOM = 4,        /* the allocator returned NULL */
  GP_ERR_CUDA = 5,       /* a CUDA runtime call failed */
  GP_ERR_TIMEOUT = 6,    /* a bounded device wait ran out */
  GP_ERR_BUDGET = 7      /* a request does not fit the memory budget */
} gp_status;

/* A graph in device memory.  m2 = number of CSR entries = 2 |E|. */
typedef struct gp_graph {
  int32_t n;
  int64_t m2;
  int32_t *xadj;   /* n + 1 row offsets */
  int32_t *adjncy; /* m2 neighbour ids */
  int32_t *vwgt;   /* n node weights c(v) > 0 */
  int32_t *adjwgt; /* m2 edge weights w(e) > 0, equal in both directions */
} gp_graph;

/*
 * Device-memory allocator.  alloc returns `bytes` of device memory usable in
 * stream order on `stream` (NULL on failure); free returns memory allocated
 * by alloc.  When no allocator is given the library allocates from a private
 * stream-ordered memory pool of the context (cudaMallocFromPoolAsync on the
 * context stream) that keeps freed memory for reuse until gp_destroy.
 */
typedef struct gp_allocator {
  void *(*alloc)(size_t bytes, void *user, void *stream);
  void (*free)(void *ptr, size_t bytes, void *user, void *stream);
  void *user;
} gp_allocator;

/* Sparsifier choice (Sec. 4.2; the exact-count variant keeps exactly m_hat edges). */
enum { GP_SPARSIFY_NONE = 0, GP_SPARSIFY_TWEIGHT = 1, GP_SPARSIFY_UNIFORM = 2, GP_SPARSIFY_TWEIGHT_EXACT = 3 };

/*
 * Method parameters.  gp_config_default() gives the paper's values:
 * tau_e = tau_d = 1/2 and rho = 4 (Sec. 6.1), U = c(V) / (160 k), at most
 * 2.5x node reduction per level and a coarsest size of 160 k (Sec. 4.3),
 * weighted threshold sampling (Sec. 6.2), and this library's fixed LP
 * schedule (5 rounds of 8 synchronous sub-rounds, 8 bisection trials).
 */
typedef struct gp_config {
  int32_t tau_e_num, tau_e_den;       /* edge bound tau_e */
  int32_t tau_d_num, tau_d_den;       /* density bound tau_d */
  int32_t rho_num, rho_den;           /* trigger factor rho */
  int32_t cluster_factor;             /* U = W / (cluster_factor * k) */
  int32_t coarsest_factor;            /* coarsen while n > coarsest_factor * k */
  int32_t shrink_num, shrink_den;     /* at most num/den node reduction per level */
  int32_t min_shrink_num, min_shrink_den; /* stop when n' * num > n * den */
  int32_t lp_rounds, lp_subrounds;    /* clustering LP schedule */
  int32_t ref_rounds;                 /* refinement LP rounds */
  int32_t ip_trials;                  /* greedy-growing trials per bisection */
  int32_t sparsifier;                 /* GP_SPARSIFY_* */
  int32_t two_hop, isolated;          /* enable 2-hop / isolated-node clustering */
  int32_t max_levels;                 /* cap on the hierarchy depth (<= 64) */
  int32_t dbg_max_subrounds;          /* < 0: no limit; else stop clustering LP early (tests) */
  int32_t validate;                   /* gp_partition: 1 = full input validation */
  int32_t small_lp_nodes;             /* LP runs on graphs of at most this many nodes use one
                                         persistent launch (0: never); same results either way */
} gp_config;

/* Per-level record of one coarsening step (Alg. 1 quantities). */
typedef struct gp_level_stats {
  int32_t n, n_next;
  int64_t m, m_coarse, m_hat, m_next;
  int32_t triggered, omega_t;
  int64_t n_greater, n_equal;
  uint64_t threshold;
  int32_t lp_subrounds;
  int64_t lp_moves, clusters_lp, clusters_2hop, clusters_final;
} gp_level_stats;

#define GP_MAX_LEVELS 64
typedef struct gp_partition_stats {
  int32_t levels;
  gp_level_stats lv[GP_MAX_LEVELS];
  int64_t U, Lmax, W, ip_cut, cut, rebalance_moves;
  int32_t n_coarsest;
  double ms_coarsen, ms_initial, ms_uncoarsen, ms_total; /* device time per phase */
} gp_partition_stats;

typedef struct gp_ctx gp_ctx;

/* Default parameters (see gp_config). */
void gp_config_default(gp_config *cfg);

/*
 * Creates a context on CUDA device `device` whose work is ordered on
 * `stream` (a cudaStream_t; NULL = the legacy default stream).  `alloc` may
 * be NULL.  The context keeps no graph between calls.
 */
gp_status gp_create(gp_ctx **ctx, int device, void *stream, const gp_allocator *alloc);
void gp_destroy(gp_ctx *ctx);
/*
 * Upper bound on the iterations of every grid-wide wait inside the library's
 * persistent kernels (the small-graph label propagation).  A wait that runs
 * out makes the call return GP_ERR_TIMEOUT; the context stays usable and the
 * call's outputs are undefined.  spins = 0 restores the default (several
 * seconds of waiting); spins < 0 makes every wait give up at once (tests).
 * Not an algorithm parameter: no counterpart in the paper.
 */
void gp_set_wait_limit(gp_ctx *ctx, int64_t spins);

/* Text of the last error on this context ("" if none).  Owned by ctx. */
const char *gp_last_error(const gp_ctx *ctx);
/* Library build string (version, compute capability compiled for). */
const char *gp_version(void);
/* Number of kernels this library has launched in this process (all contexts). */
int64_t gp_launch_count(void);

/*
 * One coarsening clustering of G_level (Sec. 3, Sec. 4.1): size-constrained
 * label propagation under the cluster bound U, then 2-hop clustering and
 * isolated-node clustering, limited to a 2.5x node reduction (Sec. 4.3).
 * cmap (device, n entries, caller-owned) receives dense coarse ids in
 * [0, *n_coarse), numbered by the rank of each cluster's id.  `label`
 * (device, n entries, may be NULL) receives the cluster id of every node.
 * `stats` (host, may be NULL) receives the step's counters.  Synchronises.
 */
gp_status gp_coarsen(gp_ctx *ctx, const gp_graph *g, int64_t U, int32_t level, uint64_t seed,
                     const gp_config *cfg, int32_t *cmap, int32_t *label, int32_t *n_coarse,
                     gp_level_stats *stats);

/*
 * Cluster contraction (Sec. 2): coarse node A weighs the total weight of
 * its members; coarse edge {A, B}, A != B, weighs the total weight of the
 * fine edges between the two clusters.  cmap (device, g->n entries) maps to
 * [0, n_coarse).  *out receives a new graph allocated through the context
 * allocator (release with gp_graph_release).  Row order inside a coarse row
 * is unspecified.  Synchronises.
 */
gp_status gp_contract(gp_ctx *ctx, const gp_graph *g, const int32_t *cmap, int32_t n_coarse,
                      gp_graph *out);

/*
 * Edge sparsification to m_hat edges in expectation (Sec. 4.2).  mode
 * GP_SPARSIFY_TWEIGHT (weighted threshold sampling): the m_hat-th heaviest
 * undirected edge weight w_t is found; heavier edges are kept, lighter ones
 * dropped and edges of weight w_t kept with probability
 * (m_hat - |E>|) / |E=| by a counter-based hash of their endpoints.
 * GP_SPARSIFY_UNIFORM keeps every edge with probability m_hat / |E|.
 * GP_SPARSIFY_TWEIGHT_EXACT selects w_t in the same way but keeps, of the
 * edges of weight w_t, exactly m_hat - |E>|: those first in the order of
 * (64-bit hash of the endpoints, smaller endpoint, larger endpoint), so the
 * result has exactly min(m_hat, |E|) edges.  Kept edges keep their weights;
 * node weights are copied.  *out is allocated through the context allocator.
 * `stats` (host, may be NULL) gets w_t, |E>|, |E=| and the hash threshold
 * (the last kept hash in the exact mode) in its omega_t / n_greater /
 * n_equal / threshold fields.  Synchronises.
 */
gp_status gp_sparsify(gp_ctx *ctx, const gp_graph *g, int64_t m_hat, int32_t level,
                      uint64_t seed, int32_t mode, gp_graph *out, gp_level_stats *stats);

/*
 * Full multilevel partition (Sec. 2, Alg. 1, Sec. 4.3): coarsening with
 * sparsification, recursive-bisection initial partitioning of the coarsest
 * graph on the device, and label-propagation refinement on every level.
 * blocks (device, g->n entries, caller-owned) receives block ids in [0, k);
 * *cut (host) the cut weight.  eps > 0 is used as round(eps * 1e6) parts
 * per million.  `stats` (host, may be NULL).  Synchronises.
 */
gp_status gp_partition(gp_ctx *ctx, const gp_graph *g, int32_t k, double eps, uint64_t seed,
                       const gp_config *cfg, int32_t *blocks, int64_t *cut,
                       gp_partition_stats *stats);

/*
 * gp_partition on HOST arrays: copies the graph (n + 1 + 2 m2 + n int32
 * values) to the device, partitions, and copies the n block ids back into
 * `blocks` (host).  Page-locked host memory makes the copies faster.
 */
gp_status gp_partition_host(gp_ctx *ctx, int32_t n, int64_t m2, const int32_t *xadj,
                            const int32_t *adjncy, const int32_t *vwgt, const int32_t *adjwgt,
                            int32_t k, double eps, uint64_t seed, const gp_config *cfg,
                            int32_t *blocks, int64_t *cut, gp_partition_stats *stats);

/* ---- the steps gp_partition is made of (also used by the tests) ---- */

/*
 * Recursive-bisection initial partition of a small graph (Sec. 4.3): each
 * bisection runs cfg->ip_trials seeded greedy-growing trials, one thread
 * block per trial, and keeps the smallest cut.  blocks: device, n entries.
 */
gp_status gp_initial_partition(gp_ctx *ctx, const gp_graph *g, int32_t k, double eps,
                               uint64_t seed, const gp_config *cfg, int32_t *blocks);

/* Moves nodes out of blocks heavier than Lmax (greedy, least cut loss). */
gp_status gp_rebalance(gp_ctx *ctx, const gp_graph *g, int32_t k, int64_t Lmax,
                       int32_t *blocks, int64_t *moves);

/*
 * Size-constrained label-propagation refinement (Sec. 3): blocks are the
 * labels, Lmax the bound; cfg->ref_rounds rounds of strictly improving
 * moves.  blocks: device, in/out.  *moves (host, may be NULL).
 */
gp_status gp_refine(gp_ctx *ctx, const gp_graph *g, int32_t k, int64_t Lmax, int32_t level,
                    uint64_t seed, const gp_config *cfg, int32_t *blocks, int64_t *moves);

/* Projection (uncoarsening): fine[v] = coarse[cmap[v]] for v < n. Device arrays. */
gp_status gp_project(gp_ctx *ctx, int32_t n, const int32_t *cmap, const int32_t *coarse,
                     int32_t *fine);

/*
 * Cut weight and block weights of a partition (Sec. 2).  block_weights:
 * host array of k entries, may be NULL.  Synchronises.
 */
gp_status gp_cut(gp_ctx *ctx, const gp_graph *g, const int32_t *blocks, int32_t k, int64_t *cut,
                 int64_t *block_weights);

/*
 * gp_cut without any allocation.  The paper has no counterpart: this entry
 * point exists for callers that must not allocate device memory while they
 * run -- a serving loop that reserved the whole device for its own arena up
 * front, or a latency-critical path that cannot accept cudaMalloc's implicit
 * device-wide synchronisation.  It needs no context and performs no
 * cudaMalloc, cudaFree or other allocation: its only scratch is one fixed
 * device array inside the library, present on every device that loads the
 * library until the process exits.
 *   g        graph in device memory (as for gp_cut); entries need rows:
 *            m2 > 0 with n == 0 is GP_ERR_INVALID
 *   blocks   device, g->n block ids in [0, k)
 *   k        1 <= k <= GP_CUT_NOALLOC_MAX_K, else GP_ERR_INVALID
 *   stream   cudaStream_t the work is ordered on; the call synchronises it
 *   cut      host, receives the cut weight
 *   block_weights  host array of k entries, or NULL
 * Returns GP_ERR_INVALID for bad arguments or a block id outside [0, k),
 * GP_ERR_CUDA when a CUDA call fails.  The first call on each device (with
 * that device current) looks up the scratch array's device address once;
 * make that first call before any stream capture on the device.  All calls
 * share the scratch array: calls that overlap on the GPU race on it.
 */
#define GP_CUT_NOALLOC_MAX_K 4096
gp_status gp_cut_noalloc(const gp_graph *g, const int32_t *blocks, int32_t k, void *stream,
                         int64_t *cut, int64_t *block_weights);

/* Frees a graph returned by gp_contract / gp_sparsify. */
void gp_graph_release(gp_ctx *ctx, gp_graph *g);

/*
 * Profiling: when enabled, every major kernel launch is bracketed by CUDA
 * events on the context stream, and gp_profile_read returns, per kernel
 * class, the number of bracketed launch groups, the summed device time (ms)
 * and the algorithmic bytes moved: the bytes the step must read and write
 * at least (each CSR entry, label, weight and output word counted once, at
 * its own width), from unit counts the kernels record.  Classes are named by
 * gp_profile_name(i) for i < gp_profile_count().
 */
void gp_profile_enable(gp_ctx *ctx, int on);
void gp_profile_reset(gp_ctx *ctx);
int gp_profile_count(void);
const char *gp_profile_name(int i);
gp_status gp_profile_read(gp_ctx *ctx, int i, int64_t *launches, double *ms, double *bytes);

/*
 * Many independent graphs partitioned at once (no counterpart in the paper:
 * a throughput form of gp_partition for batches of small or mid-sized
 * graphs, whose levels are too small to fill the GPU one graph at a time).
 * Items the batched engine takes (gp_batch_tuning below) are partitioned by
 * its persistent kernel; for the others `workers` host threads (1..64), each
 * with its own stream and memory pool kept in the context, take the items
 * largest first and run gp_partition on each.  Every item's blocks and cut
 * equal those of a gp_partition call with the same arguments.  Work already queued
 * on the context stream is waited for first.  Per item: `blocks` (device,
 * g.n entries, caller-owned) and, on return, `cut` and `status` (the item's
 * own result; its message is lost).  Returns GP_OK when every item succeeded,
 * else the first failing item's status (gp_last_error names the item).
 * Synchronises.
 */
typedef struct gp_batch_item {
  gp_graph g;
  int32_t k;
  double eps;
  uint64_t seed;
  int32_t *blocks;
  int64_t cut;
  gp_status status;
  int32_t engine;              /* out: 1 if the item ran on the batched engine, 0 on the per-graph path */
  gp_partition_stats *stats;   /* host, may be NULL: the item's per-level records; on the engine the
                                  phase times are the item's CTA time (SM cycles at the peak clock) */
} gp_batch_item;
gp_status gp_partition_batch(gp_ctx *ctx, gp_batch_item *items, int32_t count, int32_t workers,
                             const gp_config *cfg);

/*
 * The batched engine of gp_partition_batch (no counterpart in the paper).
 * Items of at most max_entries CSR entries and max_nodes nodes run on one
 * persistent kernel: each CTA takes whole graphs from a device-side queue
 * (largest first) and partitions each inside the CTA -- the same method and
 * readings as gp_partition, so the results are identical -- with its hierarchy
 * and scratch in a per-CTA arena.  The other items, and engine items whose
 * hierarchy outgrows the arena, run on the per-graph path (the worker
 * contexts above), after the engine.  The configuration must use a sparsifier
 * other than GP_SPARSIFY_TWEIGHT_EXACT, at most 254 sub-rounds and at least one
 * bisection trial; otherwise every item takes the per-graph path.
 *
 * gp_batch_autotune measures, on the items given (grouped into size classes
 * by their CSR entries, class c holding (class_entries[c-1],
 * class_entries[c]]), the engine's graphs/s with each CTA size and the
 * per-graph path's graphs/s with `workers` workers, and picks the CTA size
 * and the largest class up to which the engine wins; the items' outputs are
 * not written.  The result is installed in the context (gp_batch_set_tuning)
 * and returned in *out (may be NULL).  Synchronises.
 */
#define GP_TUNE_CLASSES 12
typedef struct gp_batch_tuning {
  int32_t engine;             /* 1: use the engine; 0: per-graph path only */
  int32_t threads;            /* engine CTA size: 256, 512 or 1024 */
  int64_t max_entries;        /* engine items have at most this many CSR entries ... */
  int64_t max_nodes;          /* ... and at most this many nodes */
  int64_t arena_cap_bytes;    /* device memory all arenas may take (0: a third of the free memory) */
  int64_t arena_bytes;        /* arena per CTA (0: estimated from the largest engine item) */
  int32_t classes;            /* autotuner: size classes it measured */
  int32_t pad;
  int64_t class_entries[GP_TUNE_CLASSES];    /* upper end of each class (CSR entries) */
  int32_t class_items[GP_TUNE_CLASSES];      /* items of the class in the tuning set */
  int32_t class_threads[GP_TUNE_CLASSES];    /* fastest engine CTA size on the class */
  double class_engine_gps[GP_TUNE_CLASSES];  /* engine graphs/s on the class with that CTA size */
  double class_path_gps[GP_TUNE_CLASSES];    /* per-graph path graphs/s on the class (0: not measured) */
  double tune_ms;                            /* wall time of the tuning */
} gp_batch_tuning;
void gp_batch_tuning_default(gp_batch_tuning *t);
gp_status gp_batch_set_tuning(gp_ctx *ctx, const gp_batch_tuning *t);
gp_status gp_batch_get_tuning(gp_ctx *ctx, gp_batch_tuning *t);
gp_status gp_batch_autotune(gp_ctx *ctx, const gp_batch_item *items, int32_t count, int32_t workers,
                            const gp_config *cfg, gp_batch_tuning *out);

/*
 * Serving (no counterpart in the paper): a request loop for partition
 * requests that arrive over time.  `workers` host threads (1..64), each with
 * its own context, stream and memory pool, take queued requests in arrival
 * order as soon as a worker is free and the request's estimated device
 * memory fits the budget next to the requests in flight (the first queued
 * request that fits goes first; a request alone in the server is always
 * admitted).  Requests in flight overlap on the GPU.  Each request is the
 * host-array partition of gp_partition_host, so its blocks and cut equal a
 * gp_partition_host call with the same arguments, alone or in any mix.
 * The estimate is 4x the request's CSR bytes plus 64 bytes per node plus
 * 64 MiB; a request whose estimate exceeds the budget is refused at submit
 * with GP_ERR_BUDGET.  A worker's pool is trimmed back to 1/workers of the
 * budget after each request.
 */
typedef struct gp_server gp_server;
typedef struct gp_request {
  int32_t n;
  int64_t m2;
  const int32_t *xadj, *adjncy, *vwgt, *adjwgt; /* host arrays, untouched until the request completes */
  int32_t k;
  double eps;
  uint64_t seed;
  int32_t *blocks;                              /* host output, n entries */
} gp_request;
typedef struct gp_response {
  gp_status status;
  int64_t cut;
  double queued_ms, run_ms, total_ms; /* submit to start, start to end, submit to end */
  int64_t start_order;                /* 1 for the first request a worker took, 2 for the next, ... */
  int64_t estimate_bytes;             /* the admission estimate of the request */
  int64_t peak_reserved_bytes;        /* device memory its worker's pool held at most while it ran */
  int64_t peak_used_bytes;            /* device memory it had allocated at most */
} gp_response;
gp_status gp_server_create(gp_server **out, int device, int32_t workers, int64_t hbm_budget_bytes,
                           const gp_config *cfg);
/*
 * Head-of-line bound: while the oldest queued request does not fit next to the
 * requests in flight, younger requests that do fit may start ahead of it, but
 * at most max_bypass of them (default 8); after that nothing else starts until
 * the oldest one does.  A request therefore waits for at most max_bypass
 * requests submitted after it.  Not an algorithm parameter.
 */
void gp_server_set_max_bypass(gp_server *srv, int32_t max_bypass);
/* Queues a request; *ticket identifies it for gp_server_wait. */
gp_status gp_server_submit(gp_server *srv, const gp_request *req, int64_t *ticket);
/* Blocks until the request is done, fills *out and forgets the ticket (wait once per ticket). */
gp_status gp_server_wait(gp_server *srv, int64_t ticket, gp_response *out);
/* Finishes the queued and running requests, then stops the workers. */
void gp_server_destroy(gp_server *srv);

/*
 * Modularity of a clustering (Sec. 5).  With e_ij the fraction of the edge
 * weight running from cluster i to cluster j (both directions of an edge
 * counted, so the fractions sum to one), a_i = sum_j e_ij, Q_C = sum_i (e_ii -
 * a_i^2) and alpha_C = max_i a_i, Lemma 2 bounds the weight fraction inside
 * the clusters by Q_C <= sum_i e_ii <= Q_C + alpha_C: 1 - Q_C - alpha_C is a
 * lower bound of the fraction of the weight that a contraction of the
 * clustering keeps (before parallel edges merge), the paper's criterion for
 * whether sparsification will be needed.  labels (device, g->n entries) must
 * lie in [0, nlabels) (else GP_ERR_INVALID).  The integer totals are exact;
 * the fractions are computed from them in double precision.  Synchronises.
 */
typedef struct gp_modularity_stats {
  int64_t w_internal;  /* sum over CSR entries whose endpoints share a cluster */
  int64_t w_total;     /* sum over all CSR entries (twice the edge weight) */
  int64_t vol_max;     /* largest cluster volume (sum of its nodes' weighted degrees) */
  uint64_t vol_sq;     /* sum of squared cluster volumes */
  double inside;       /* sum_i e_ii = w_internal / w_total */
  double q;            /* Q_C */
  double alpha;        /* alpha_C */
  double bound;        /* 1 - Q_C - alpha_C */
} gp_modularity_stats;
gp_status gp_modularity(gp_ctx *ctx, const gp_graph *g, const int32_t *labels, int32_t nlabels,
                        gp_modularity_stats *out);

/*
 * Measurement helper with no counterpart in the paper: the device's rate of
 * random 4-byte reads from an array of `array_bytes` bytes (`reads` reads,
 * indices from a counter hash, timed with CUDA events after two warm-up
 * passes).  The label and coarse-id reads of the rating and contraction
 * kernels are such reads, so this rate bounds them.  Allocates the array
 * through the context allocator; returns reads per second in *reads_per_s.
 */
gp_status gp_measure_random_reads(gp_ctx *ctx, int64_t array_bytes, int64_t reads, double *reads_per_s);

#ifdef __cplusplus
}
#endif
#endif /* GP_H */
