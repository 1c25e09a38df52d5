// gp_internal.cuh -- shared internals of the GB300 partitioning library:
// error handling, the context, stream-ordered device buffers, the keyed
// counter hash, and warp-level helpers.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <initializer_list>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "gp.h"

namespace gp {

// ------------------------------------------------------------------ errors

struct Error {
  gp_status status;
  std::string msg;
};

[[noreturn]] inline void fail(gp_status st, const std::string &msg) { throw Error{st, msg}; }

#define GP_CUDA(call)                                                                   \
  do {                                                                                  \
    cudaError_t e_ = (call);                                                            \
    if (e_ != cudaSuccess)                                                              \
      ::gp::fail(GP_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_) +      \
                                  " (" + __FILE__ + ":" + std::to_string(__LINE__) + ")"); \
  } while (0)

// Every kernel launch of the library is followed by GP_LAUNCH_CHECK(), which
// also counts it (gp_launch_count).
extern std::atomic<long long> g_launch_count;
#define GP_LAUNCH_CHECK()                                           \
  do {                                                              \
    ::gp::g_launch_count.fetch_add(1, std::memory_order_relaxed);   \
    GP_CUDA(cudaGetLastError());                                    \
  } while (0)

#define GP_REQUIRE(cond, st, msg) \
  do {                            \
    if (!(cond)) ::gp::fail((st), (msg)); \
  } while (0)

// ------------------------------------------------------------- profiling

enum ProfClass {
  PROF_LP_RATE = 0,   // clustering LP: rate + choose (the dominant kernel)
  PROF_LP_ACCEPT,     // clustering LP: acceptance decision
  PROF_REF_RATE,      // refinement LP: rate + choose
  PROF_REF_ACCEPT,    // refinement LP: acceptance decision
  PROF_ROUND_SETUP,   // per-round activity bucketing
  PROF_TWOHOP,        // 2-hop favourites + packing, isolated packing
  PROF_RELABEL,
  PROF_CONTRACT,      // contraction aggregation
  PROF_CONTRACT_AUX,  // contraction bucketing / copy
  PROF_SPARSIFY,
  PROF_IP,
  PROF_PROJECT,
  PROF_CUT,
  PROF_VALIDATE,
  PROF_SORT,
  PROF_SCAN,
  PROF_LP_OVERFLOW,   // clustering LP: ordering the proposers of overflowing targets
  PROF_LP_APPLY,      // clustering LP: apply moves, count emptied clusters
  PROF_REF_OVERFLOW,
  PROF_REF_APPLY,
  PROF_REBALANCE,     // greedy rebalance after the initial partition
  PROF_LP_SMALL,      // clustering LP of a small graph in one persistent launch
  PROF_REF_SMALL,     // refinement LP of a small graph in one persistent launch
  PROF_COUNT_
};

// device-side unit counters, per class: [0] entries, [1] vertices, [2] candidates, [3] proposals,
// [4] entries whose neighbour label was read as one byte, [5] entries whose weight was not read
// (unit edge weights)
constexpr int PROF_UNITS = 6;

struct ProfRecord {
  int cls;
  cudaEvent_t a, b;
};

}  // namespace gp

// ------------------------------------------------------------------ context

struct gp_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  gp_allocator alloc{};
  bool own_alloc = false;
  cudaMemPool_t pool = nullptr;  // the library's own stream-ordered pool (no external allocator)
  int num_sms = 0;
  std::string last_error;
  // small pinned host staging area and device scratch for counters
  int64_t *h_stage = nullptr;  // 4096 int64
  int64_t *d_stage = nullptr;  // 4096 int64
  // profiling
  bool profile = false;
  std::vector<gp::ProfRecord> pending;
  std::vector<cudaEvent_t> free_events;
  double prof_ms[gp::PROF_COUNT_] = {};
  int64_t prof_launches[gp::PROF_COUNT_] = {};
  unsigned long long *d_units = nullptr;  // PROF_COUNT_ x PROF_UNITS
  double prof_host_bytes[gp::PROF_COUNT_] = {};  // algorithmic bytes of classes sized on the host
  std::vector<gp_ctx *> workers;                 // batch workers (own streams and pools)
  int64_t wait_spins = 0;                        // limit of device-side waits (0: default)
  int device_share = 1;  // contexts sharing the device (batch / server workers): persistent grids shrink
  gp_batch_tuning tuning{};        // batched engine settings (gp_batch_set_tuning / gp_batch_autotune)
  bool tuning_set = false;
  cudaStream_t copy_streams[4] = {};  // host-to-device copies of large inputs
  cudaEvent_t copy_events[5] = {};
};

namespace gp {

// ------------------------------------------------------ device memory RAII

void *dev_alloc(gp_ctx *ctx, size_t bytes);
void dev_free(gp_ctx *ctx, void *p, size_t bytes);

template <typename T>
struct DBuf {
  gp_ctx *ctx = nullptr;
  T *p = nullptr;
  size_t count = 0;
  DBuf() = default;
  DBuf(gp_ctx *c, size_t n) { reset(c, n); }
  DBuf(const DBuf &) = delete;
  DBuf &operator=(const DBuf &) = delete;
  DBuf(DBuf &&o) noexcept : ctx(o.ctx), p(o.p), count(o.count) { o.p = nullptr; o.count = 0; }
  DBuf &operator=(DBuf &&o) noexcept {
    if (this != &o) {
      release();
      ctx = o.ctx; p = o.p; count = o.count;
      o.p = nullptr; o.count = 0;
    }
    return *this;
  }
  ~DBuf() { release(); }
  void reset(gp_ctx *c, size_t n) {
    release();
    ctx = c;
    count = n;
    p = static_cast<T *>(dev_alloc(c, (n ? n : 1) * sizeof(T)));
  }
  void release() {
    if (p) dev_free(ctx, p, (count ? count : 1) * sizeof(T));
    p = nullptr;
    count = 0;
  }
  T *get() const { return p; }
  void zero() {
    if (p) GP_CUDA(cudaMemsetAsync(p, 0, (count ? count : 1) * sizeof(T), ctx->stream));
  }
  void fill_bytes(int byte) {
    if (p) GP_CUDA(cudaMemsetAsync(p, byte, (count ? count : 1) * sizeof(T), ctx->stream));
  }
};

// One host-to-device copy of copy_to_device.
struct HostCopy {
  void *dst;
  const void *src;
  size_t bytes;
};
void copy_to_device(gp_ctx *ctx, std::initializer_list<HostCopy> parts);

// Copies `n` device int64 values to the host (synchronises the stream).
void read_back(gp_ctx *ctx, const void *dev, size_t bytes, void *host);
template <typename T>
T read_scalar(gp_ctx *ctx, const T *dev) {
  T v;
  read_back(ctx, dev, sizeof(T), &v);
  return v;
}

// ------------------------------------------------------------- profiling

// Adds algorithmic bytes to a class whose sizes the host knows (profiling only).
inline void prof_bytes(gp_ctx *ctx, int cls, double bytes) {
  if (ctx->profile) ctx->prof_host_bytes[cls] += bytes;
}

struct ProfScope {
  gp_ctx *ctx;
  int cls;
  cudaEvent_t a = nullptr;
  ProfScope(gp_ctx *c, int k);
  ~ProfScope();
};

// A named NVTX range around a phase of the method (visible to profilers such
// as ncu --nvtx; costs nothing without one attached).
struct NvtxRange {
  explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
  NvtxRange(const char *what, int level) {
    char buf[48];
    snprintf(buf, sizeof buf, "%s_L%d", what, level);
    nvtxRangePushA(buf);
  }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange &) = delete;
  NvtxRange &operator=(const NvtxRange &) = delete;
};

// Wall time of a stretch of stream work, measured only when the GP_TRACE
// environment variable is set (diagnostic output on stderr).
struct TraceTimer {
  gp_ctx *ctx;
  cudaEvent_t a = nullptr, b = nullptr;
  explicit TraceTimer(gp_ctx *c) : ctx(c) {
    if (!getenv("GP_TRACE")) return;
    if (cudaEventCreate(&a) != cudaSuccess || cudaEventCreate(&b) != cudaSuccess) { a = b = nullptr; return; }
    cudaEventRecord(a, ctx->stream);
  }
  bool on() const { return a != nullptr; }
  double ms() {
    if (!a) return 0;
    float f = 0;
    cudaEventRecord(b, ctx->stream);
    cudaEventSynchronize(b);
    cudaEventElapsedTime(&f, a, b);
    return f;
  }
  ~TraceTimer() {
    if (a) cudaEventDestroy(a);
    if (b) cudaEventDestroy(b);
  }
};

// ---------------------------------------------------------------- launch

constexpr int kWarp = 32;

// Blocks that get a private global hash table of `slots` int pairs, at most
// `want`: the tables together stay within 8 bytes per CSR entry plus 16 MiB,
// so scratch memory grows with the graph, not with its largest degree.
inline int table_blocks(int64_t m2, int64_t slots, int want) {
  const int64_t cap = 8 * m2 + ((int64_t)16 << 20);
  int64_t b = cap / (slots * 8);
  if (b > want) b = want;
  return b < 1 ? 1 : (int)b;
}

inline int grid_for(int64_t items, int per_block, int cap) {
  int64_t g = (items + per_block - 1) / per_block;
  if (g < 1) g = 1;
  if (g > cap) g = cap;
  return (int)g;
}

// ------------------------------------------------------------------ hash

// Keyed counter hash of the method (SplitMix64 output finaliser of Steele,
// Lea and Flood, OOPSLA 2014):
//   key(s, t, l, r) = mix(mix(s ^ GOLD) + (t << 48 | (l & 0xFFFF) << 32 | r))
//   h32(key, x, y)  = top 32 bits of mix(key ^ (x << 32 | y))
constexpr uint64_t kGold = 0x9E3779B97F4A7C15ull;

__host__ __device__ __forceinline__ uint64_t fmix(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

__host__ __device__ __forceinline__ uint64_t stream_key(uint64_t seed, uint32_t tag, uint32_t level,
                                                        uint32_t round) {
  uint64_t w = ((uint64_t)tag << 48) | ((uint64_t)(level & 0xFFFFu) << 32) | (uint64_t)round;
  return fmix(fmix(seed ^ kGold) + w);
}

__host__ __device__ __forceinline__ uint64_t h64(uint64_t key, uint32_t x, uint32_t y) {
  return fmix(key ^ (((uint64_t)x << 32) | (uint64_t)y));
}
__host__ __device__ __forceinline__ uint32_t h32(uint64_t key, uint32_t x, uint32_t y) {
  return (uint32_t)(fmix(key ^ (((uint64_t)x << 32) | (uint64_t)y)) >> 32);
}

enum Tag : uint32_t {
  TAG_ACT = 1, TAG_TIE = 2, TAG_PRIO = 3, TAG_FAV = 4, TAG_SPARSE = 5, TAG_UNIFORM = 6,
  TAG_RACT = 7, TAG_RTIE = 8, TAG_RPRIO = 9, TAG_IP = 10
};

// ------------------------------------------------------------ warp utils

__device__ __forceinline__ unsigned lane_id() { return threadIdx.x & 31u; }
__device__ __forceinline__ unsigned lanemask_lt() {
  unsigned m;
  asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
  return m;
}

// Warp-aggregated atomicAdd of `val` to counter[0] by the lanes in `active`
// (all lanes of the warp call it); returns each lane's exclusive offset.
__device__ __forceinline__ int warp_append(int *counter, bool pred) {
  unsigned m = __ballot_sync(0xFFFFFFFFu, pred);
  int base = 0;
  if (m) {
    int leader = __ffs(m) - 1;
    if ((int)lane_id() == leader) base = atomicAdd(counter, __popc(m));
    base = __shfl_sync(0xFFFFFFFFu, base, leader);
  }
  return base + __popc(m & lanemask_lt());
}

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xFFFFFFFFu, v, o);
  return v;
}

template <typename T>
__device__ __forceinline__ T warp_max(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    T x = __shfl_xor_sync(0xFFFFFFFFu, v, o);
    v = x > v ? x : v;
  }
  return v;
}

template <typename T>
__device__ __forceinline__ T warp_min(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    T x = __shfl_xor_sync(0xFFFFFFFFu, v, o);
    v = x < v ? x : v;
  }
  return v;
}

// Adds `val` into *addr, aggregating lanes that target the same address.
__device__ __forceinline__ void warp_agg_add(int *base, int idx, int val, bool pred) {
  unsigned act = __ballot_sync(0xFFFFFFFFu, pred);
  if (!pred) return;
  unsigned peers = __match_any_sync(act, idx);
  int sum = __reduce_add_sync(peers, val);
  if ((int)lane_id() == __ffs(peers) - 1) atomicAdd(base + idx, sum);
}

// Row of CSR entry e: the largest r < n with xadj[r] <= e.
__device__ __forceinline__ int row_of(const int32_t *xadj, int n, int64_t e) {
  int lo = 0, hi = n;  // invariant: xadj[lo] <= e < xadj[hi] (xadj[n] = m2 > e)
  while (hi - lo > 1) {
    int mid = (lo + hi) >> 1;
    if ((int64_t)xadj[mid] <= e) lo = mid; else hi = mid;
  }
  return lo;
}

// ---------------------------------------------------------- primitives

// Exclusive prefix sum of n values; total (device pointer, may be null)
// receives the sum.  in and out may alias.
void scan_exclusive_i32(gp_ctx *ctx, const int32_t *in, int32_t *out, int64_t n, int32_t *total);
void scan_exclusive_i64(gp_ctx *ctx, const int64_t *in, int64_t *out, int64_t n, int64_t *total);
// Exclusive prefix sum of int32 inputs into int64 outputs.
void scan_exclusive_i32_i64(gp_ctx *ctx, const int32_t *in, int64_t *out, int64_t n,
                            int64_t *total);

// Stable LSD radix sort of (key, value) pairs on key bits [0, bits), in place
// (uses scratch of the same size).  n is a host count.
void radix_sort_pairs(gp_ctx *ctx, uint64_t *keys, uint32_t *vals, int64_t n, int bits);

// Reductions into device scalars.
void reduce_sum_i32_to_i64(gp_ctx *ctx, const int32_t *in, int64_t n, int64_t *out);

// --------------------------------------------------------------- graphs

struct DevGraph {
  int32_t n = 0;
  int64_t m2 = 0;
  int32_t *xadj = nullptr, *adjncy = nullptr, *vwgt = nullptr, *adjwgt = nullptr;
  // every edge weight is 1 (found by the input validation: positive weights summing to the
  // entry count); kernels that honour it use 1 instead of reading adjwgt
  bool unit_w = false;
  // ownership (when created by the library)
  DBuf<int32_t> bx, ba, bv, bw;
  gp_graph view() const {
    gp_graph g;
    g.n = n; g.m2 = m2; g.xadj = xadj; g.adjncy = adjncy; g.vwgt = vwgt; g.adjwgt = adjwgt;
    return g;
  }
  static DevGraph wrap(const gp_graph &g) {
    DevGraph d;
    d.n = g.n; d.m2 = g.m2; d.xadj = g.xadj; d.adjncy = g.adjncy; d.vwgt = g.vwgt; d.adjwgt = g.adjwgt;
    return d;
  }
  void allocate(gp_ctx *ctx, int32_t nn, int64_t mm2) {
    n = nn; m2 = mm2;
    bx.reset(ctx, (size_t)nn + 1); ba.reset(ctx, (size_t)mm2); bv.reset(ctx, (size_t)nn);
    bw.reset(ctx, (size_t)mm2);
    xadj = bx.get(); adjncy = ba.get(); vwgt = bv.get(); adjwgt = bw.get();
  }
};

// Moves an owned DevGraph into a heap object handed out through gp_graph
// (gp_graph_release frees it).
void export_graph(gp_ctx *ctx, DevGraph &&g, gp_graph *out);

// ------------------------------------------------------ method internals

struct LevelOut {
  int32_t n_coarse = 0;
  gp_level_stats st{};
};

// Clustering of one level (LP + 2-hop + isolated) and relabel into cmap.
void coarsen_level(gp_ctx *ctx, const DevGraph &g, int64_t U, int32_t level, uint64_t seed,
                   const gp_config &cfg, int32_t *cmap, int32_t *label_out, LevelOut &out);

// Contraction into a new owned graph.
void contract_graph(gp_ctx *ctx, const DevGraph &g, const int32_t *cmap, int32_t nc, DevGraph &out);

// Sparsification into a new owned graph; fills omega_t etc. in st.
void sparsify_graph(gp_ctx *ctx, const DevGraph &g, int64_t m_hat, int32_t level, uint64_t seed,
                    int mode, DevGraph &out, gp_level_stats *st);

// Refinement LP on blocks (k labels).
int64_t refine_blocks(gp_ctx *ctx, const DevGraph &g, int32_t k, int64_t Lmax, int32_t level,
                      uint64_t seed, const gp_config &cfg, int32_t *blocks);

void initial_partition(gp_ctx *ctx, const DevGraph &g, int32_t k, int64_t eps_ppm, uint64_t seed,
                       int32_t trials, int32_t *blocks);
int64_t rebalance_blocks(gp_ctx *ctx, const DevGraph &g, int32_t k, int64_t Lmax, int32_t *blocks);
void project(gp_ctx *ctx, int32_t n, const int32_t *cmap, const int32_t *coarse, int32_t *fine);
void cut_and_weights(gp_ctx *ctx, const DevGraph &g, const int32_t *blocks, int32_t k,
                     int64_t *cut_host, int64_t *bw_host);
// Validates the input graph (throws on a malformed one); returns the total
// node weight W and the heaviest node weight.
struct GraphTotals {
  int64_t W;
  int64_t cmax;
  bool unit_w;  // every edge weight is 1
};
GraphTotals validate_graph(gp_ctx *ctx, const DevGraph &g, bool full);
int64_t lmax_of(int64_t W, int32_t k, int64_t eps_ppm);
double measure_random_reads(gp_ctx *ctx, int64_t array_bytes, int64_t reads);
void modularity(gp_ctx *ctx, const DevGraph &g, const int32_t *labels, int32_t nlabels, gp_modularity_stats *out);
void check_blocks(gp_ctx *ctx, const int32_t *blocks, int n, int k);
void partition_impl(gp_ctx *ctx, const DevGraph &input, int32_t k, double eps, uint64_t seed,
                    const gp_config &cfg, int32_t *blocks, int64_t *cut_out, gp_partition_stats *st);

// Batched form (batch.cu, engine.cu).  batch_per_graph: the listed items on
// `workers` worker contexts (created on first use), each worker's persistent
// grids limited to 1/share of the device, after `ready` (an event on the
// caller's stream).  batch_run: the engine for the items it takes, beside the
// per-graph path for the rest, then the per-graph path for engine items that
// outgrew their arena.
void batch_per_graph(gp_ctx *ctx, gp_batch_item *items, const std::vector<int32_t> &idx, int workers,
                     const gp_config &cfg, int share, cudaEvent_t ready);
void batch_run(gp_ctx *ctx, gp_batch_item *items, const std::vector<int32_t> &idx, int workers,
               const gp_config &cfg, const gp_batch_tuning &t);
bool engine_config_ok(const gp_config &cfg);
const gp_batch_tuning &batch_tuning(gp_ctx *ctx);

}  // namespace gp
