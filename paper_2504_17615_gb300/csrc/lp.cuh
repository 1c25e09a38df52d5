// lp.cuh -- size-constrained label propagation on the GPU (shared by
// clustering, refinement and the 2-hop favourite search).
#pragma once
#include "gp_internal.cuh"

namespace gp {

// Degree classes of the rating kernels: <= 8, <= 16, <= 32 (8/16/32 lanes per
// node, one neighbour per lane), <= 128 (a warp with a 256-slot shared table),
// larger (a block with a shared table, or a global one beyond 2048).
constexpr int kNumBuckets = 5;
constexpr int kMediumMaxDeg = 128;
constexpr int kLargeSmemSlots = 4096;

__host__ __device__ __forceinline__ int degree_bucket(int deg) {
  return deg <= 8 ? 0 : deg <= 16 ? 1 : deg <= 32 ? 2 : deg <= kMediumMaxDeg ? 3 : 4;
}

enum RateMode { RATE_LP = 0, RATE_FAV = 1 };

// LP runs on graphs up to this size use the persistent kernel of lp_small.cu
// (gp_config.small_lp_nodes, default) and at most this many CSR entries.
constexpr int32_t kLpSmallMaxNodes = 5 << 20;
constexpr int64_t kLpSmallMaxEntries = (int64_t)1 << 26;
// iterations of a device-side wait before it gives up (about seconds)
constexpr long long kDefaultWaitSpins = 1ll << 25;

struct LpParams {
  uint32_t tag_act, tag_tie, tag_prio;
  int32_t level, rounds, subrounds;
  int64_t bound;
  bool count_clusters;
  int64_t n_min;
  int32_t dbg_max_subrounds;
  int32_t small_nodes;  // graphs up to this many nodes: one persistent launch (0: never)
  int prof_rate, prof_accept, prof_overflow, prof_apply, prof_small;
};

struct LpResult {
  int32_t subrounds = 0;
  int64_t moves = 0;
  int64_t nclusters = 0;
  int64_t proposals = 0;       // over all sub-rounds
  int64_t overflow_total = 0;  // proposers of overflowing targets, over all sub-rounds
  int64_t overflow_max = 0;    // largest such set in one sub-round
  int32_t capped = 0;          // sub-rounds cut short by the 2.5x cap
};

// Runs LP on g.  label (n) and weight (nlabels) are updated in place; size
// (nlabels) is maintained when p.count_clusters (may be null otherwise).
// nclusters_dev: device int64 with the current number of non-empty clusters
// (clustering only).
// label8 (may be null): a uint8 copy of label, used for the gathers and kept
// in step (fewer than 256 labels).
LpResult lp_run(gp_ctx *ctx, const DevGraph &g, int32_t *label, int32_t *weight,
                int64_t nlabels, uint64_t seed, const LpParams &p, int64_t *nclusters_dev,
                uint8_t *label8 = nullptr);

// 2-hop favourites (Sec. 4.1): for every light singleton (deg > 0, alone in
// its cluster, 2 c <= U), the adjacent cluster K != label(v) of largest
// rating, ties by the smallest h32(kfav, v, K) then the smallest K, ignoring
// U.  keys receives (fav << 32 | v) per singleton; count their number.
void favourites_bucketed(gp_ctx *ctx, const DevGraph &g, const int32_t *label, const int32_t *size,
                         int64_t U, uint64_t kfav, DBuf<uint64_t> &keys, int32_t &count);

int bits_for(int64_t x);

// The same LP run as lp_run as one cooperative persistent launch (lp_small.cu);
// for graphs of at most p.small_nodes nodes and kLpSmallMaxEntries entries.
bool lp_small_applicable(const DevGraph &g, const LpParams &p);
LpResult lp_run_small(gp_ctx *ctx, const DevGraph &g, int32_t *label, int32_t *weight, int64_t nlabels,
                      uint64_t seed, const LpParams &p, int64_t *nclusters_dev, uint8_t *label8);

}  // namespace gp
