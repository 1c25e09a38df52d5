/*
 * gp_oracle.h -- CPU oracle of the deterministic linear-time multilevel
 * partitioner (Gottesbueren, Maas, Rosch, Sanders, Seemaier: "Linear-Time
 * Multilevel Graph Partitioning via Edge Sparsification").
 *
 * TEST INFRASTRUCTURE ONLY.  This plain, slow, single-threaded C program is
 * the yardstick the GPU library is checked against.  It shares no code,
 * header, table or helper with the GPU library; only tests, the smoke check
 * and the benchmark's CPU-baseline leg may load it.
 *
 * Graphs are symmetric CSR with int64 row offsets; every array is host
 * memory owned by the caller unless stated otherwise.
 */
#ifndef GP_ORACLE_H
#define GP_ORACLE_H
#include <stdint.h>

enum { OR_OK = 0, OR_INVALID = 1, OR_INFEASIBLE = 2, OR_OVERFLOW = 3, OR_NOMEM = 4 };

/* hash stream tags */
enum {
  OR_TAG_ACT = 1, OR_TAG_TIE = 2, OR_TAG_PRIO = 3, OR_TAG_FAV = 4, OR_TAG_SPARSE = 5,
  OR_TAG_UNIFORM = 6, OR_TAG_RACT = 7, OR_TAG_RTIE = 8, OR_TAG_RPRIO = 9, OR_TAG_IP = 10
};

typedef struct {
  int32_t tau_e_num, tau_e_den;     /* edge bound tau_e (Sec. 4.2), 1/2 */
  int32_t tau_d_num, tau_d_den;     /* density bound tau_d, 1/2 */
  int32_t rho_num, rho_den;         /* trigger factor rho, 4 */
  int32_t cluster_factor;           /* U = W / (cluster_factor * k), 160 (Sec. 4.3) */
  int32_t coarsest_factor;          /* stop once n <= coarsest_factor * k, 160 */
  int32_t shrink_num, shrink_den;   /* node reduction per level at most num/den = 5/2 */
  int32_t min_shrink_num, min_shrink_den; /* stop if n' * num > n * den (21/20) */
  int32_t lp_rounds, lp_subrounds;  /* clustering LP: 5 rounds x 8 sub-rounds */
  int32_t ref_rounds;               /* refinement LP rounds, 5 */
  int32_t ip_trials;                /* greedy growing trials per bisection, 8 */
  int32_t sparsifier;               /* 0 none, 1 weighted threshold, 2 uniform, 3 exact-count threshold */
  int32_t two_hop, isolated;        /* enable 2-hop / isolated-node clustering */
  int32_t max_levels;               /* hard cap on hierarchy depth */
  int32_t dbg_max_subrounds;        /* <0: unlimited; else stop LP after that many sub-rounds */
} or_config;

typedef struct {
  int32_t n, n_next;
  int64_t m, m_coarse, m_hat, m_next;
  int32_t triggered;
  int32_t omega_t;
  int64_t n_greater, n_equal;
  uint64_t threshold;
  int32_t lp_subrounds;
  int64_t lp_moves;
  int64_t clusters_lp, clusters_2hop, clusters_final;
} or_level;

#define OR_MAX_LEVELS 64
typedef struct {
  int32_t levels;                   /* coarsening steps taken */
  or_level lv[OR_MAX_LEVELS];
  int64_t U, Lmax, W;
  int64_t ip_cut, cut;
  int64_t rebalance_moves;
  int32_t n_coarsest;
} or_stats;

typedef struct {
  int64_t omega_t, n_greater, n_equal, m_in, m_out;
  uint64_t threshold;
} or_sparse_stats;

#endif
