// engine_abi.cuh -- what the host side of the batched engine shares with the
// kernel instantiations (engine_k*.cu): the item / result / argument records,
// the arena-retry status and the launch entry points.
#pragma once
#include "gp_internal.cuh"

namespace gp {
namespace eng {

constexpr int kEMaxWarps = 32;
constexpr int kEWarpSlots = 256;   // per-warp rating / aggregation table (int pairs)
constexpr int kELight = 128;       // nodes up to this degree are rated by a lane group or a warp
constexpr int kEBlockSlots = 4096; // CTA-wide shared table; larger tables live in the arena
constexpr int kEWarpHeavy = 4096;  // degree (member entries) up to which a warp rates (merges) with a
                                   // table of its own in the arena; larger ones: the whole CTA
constexpr int kERetry = 1000;      // item status: the arena was too small

struct EItem {
  const int32_t *xadj, *adjncy, *vwgt, *adjwgt;
  int32_t *blocks;
  int64_t m2, eps_ppm;
  uint64_t seed;
  int32_t n, k;
};

// Phases whose SM cycles the engine adds up per item when profiling.
enum EPhase { EP_VALIDATE = 0, EP_CLUSTER, EP_RELABEL, EP_CONTRACT, EP_SPARSIFY, EP_INITIAL, EP_REFINE, EP_CUT,
              EP_COUNT };

struct EOut {
  int32_t status, levels, n_coarsest, pad;
  int64_t U, Lmax, W, ip_cut, cut, rebalance_moves;
  long long cyc[EP_COUNT];
};

struct EArgs {
  const EItem *items;
  EOut *out;
  gp_level_stats *lv;   // [count][GP_MAX_LEVELS], may be null
  const int32_t *order; // queue: item indices, largest first
  int32_t count;
  int32_t *head;        // queue head
  unsigned char *arena;
  int64_t arena_bytes;  // per CTA
  int profile;          // add up the SM cycles of every phase per item
  gp_config cfg;
};


// Launch entry points of the kernel instantiations (one translation unit each).
struct Kernel {
  void (*launch)(int grid, size_t smem, cudaStream_t stream, const EArgs &a);
  const void *fn;  // for the attribute / occupancy queries
  int threads;
};
Kernel kernel_256();
Kernel kernel_512();
Kernel kernel_1024();

// dynamic shared memory of the kernel with `threads` threads per CTA
inline size_t smem_bytes(int threads) {
  return (size_t)(2 * kEBlockSlots + 2 * (threads / 32) * kEWarpSlots) * sizeof(int);
}

}  // namespace eng
}  // namespace gp
