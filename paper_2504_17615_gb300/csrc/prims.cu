// prims.cu -- device memory plumbing, profiling scopes, prefix sums and a
// stable LSD radix sort used by the partitioner's steps.
#include "gp_internal.cuh"

namespace gp {

std::atomic<long long> g_launch_count{0};

// ------------------------------------------------------------------ memory

void *dev_alloc(gp_ctx *ctx, size_t bytes) {
  void *p = nullptr;
  if (ctx->alloc.alloc) {
    p = ctx->alloc.alloc(bytes, ctx->alloc.user, (void *)ctx->stream);
  } else {
    cudaError_t e = ctx->pool ? cudaMallocFromPoolAsync(&p, bytes, ctx->pool, ctx->stream)
                              : cudaMallocAsync(&p, bytes, ctx->stream);
    if (e != cudaSuccess) {
      (void)cudaGetLastError();
      p = nullptr;
    }
  }
  if (!p) fail(GP_ERR_OOM, "device allocation of " + std::to_string(bytes) + " bytes failed");
  return p;
}

void dev_free(gp_ctx *ctx, void *p, size_t bytes) {
  if (!p) return;
  if (ctx->alloc.free) ctx->alloc.free(p, bytes, ctx->alloc.user, (void *)ctx->stream);
  else cudaFreeAsync(p, ctx->stream);
}

void read_back(gp_ctx *ctx, const void *dev, size_t bytes, void *host) {
  if (bytes <= 4096 * sizeof(int64_t)) {
    GP_CUDA(cudaMemcpyAsync(ctx->h_stage, dev, bytes, cudaMemcpyDeviceToHost, ctx->stream));
    GP_CUDA(cudaStreamSynchronize(ctx->stream));
    memcpy(host, ctx->h_stage, bytes);
  } else {
    GP_CUDA(cudaMemcpyAsync(host, dev, bytes, cudaMemcpyDeviceToHost, ctx->stream));
    GP_CUDA(cudaStreamSynchronize(ctx->stream));
  }
}

// Host-to-device copies of large arrays: 256 MiB chunks spread round-robin
// over four streams of the context (several copy engines in flight), ordered
// after the context stream's earlier work and joined back into it.
void copy_to_device(gp_ctx *ctx, std::initializer_list<HostCopy> parts) {
  constexpr size_t kChunk = (size_t)256 << 20;
  constexpr int kStreams = 4;
  size_t total = 0;
  for (const HostCopy &h : parts) total += h.bytes;
  if (total <= kChunk) {
    for (const HostCopy &h : parts)
      if (h.bytes) GP_CUDA(cudaMemcpyAsync(h.dst, h.src, h.bytes, cudaMemcpyHostToDevice, ctx->stream));
    return;
  }
  if (!ctx->copy_streams[0]) {
    for (int i = 0; i < kStreams; i++) {
      GP_CUDA(cudaStreamCreateWithFlags(&ctx->copy_streams[i], cudaStreamNonBlocking));
      GP_CUDA(cudaEventCreateWithFlags(&ctx->copy_events[i], cudaEventDisableTiming));
    }
    GP_CUDA(cudaEventCreateWithFlags(&ctx->copy_events[kStreams], cudaEventDisableTiming));
  }
  GP_CUDA(cudaEventRecord(ctx->copy_events[kStreams], ctx->stream));
  for (int i = 0; i < kStreams; i++) GP_CUDA(cudaStreamWaitEvent(ctx->copy_streams[i], ctx->copy_events[kStreams], 0));
  int next = 0;
  for (const HostCopy &h : parts) {
    for (size_t off = 0; off < h.bytes; off += kChunk) {
      const size_t len = h.bytes - off < kChunk ? h.bytes - off : kChunk;
      GP_CUDA(cudaMemcpyAsync(static_cast<char *>(h.dst) + off, static_cast<const char *>(h.src) + off, len,
                              cudaMemcpyHostToDevice, ctx->copy_streams[next]));
      next = (next + 1) % kStreams;
    }
  }
  for (int i = 0; i < kStreams; i++) {
    GP_CUDA(cudaEventRecord(ctx->copy_events[i], ctx->copy_streams[i]));
    GP_CUDA(cudaStreamWaitEvent(ctx->stream, ctx->copy_events[i], 0));
  }
}

// --------------------------------------------------------------- profiling

static cudaEvent_t take_event(gp_ctx *ctx) {
  if (!ctx->free_events.empty()) {
    cudaEvent_t e = ctx->free_events.back();
    ctx->free_events.pop_back();
    return e;
  }
  cudaEvent_t e;
  GP_CUDA(cudaEventCreate(&e));
  return e;
}

ProfScope::ProfScope(gp_ctx *c, int k) : ctx(c), cls(k) {
  if (!ctx->profile) return;
  a = take_event(ctx);
  GP_CUDA(cudaEventRecord(a, ctx->stream));
}

ProfScope::~ProfScope() {
  if (!ctx->profile || !a) return;
  cudaEvent_t b = nullptr;
  if (!ctx->free_events.empty()) {
    b = ctx->free_events.back();
    ctx->free_events.pop_back();
  } else if (cudaEventCreate(&b) != cudaSuccess) {
    return;
  }
  cudaEventRecord(b, ctx->stream);
  ctx->pending.push_back(ProfRecord{cls, a, b});
}

// ------------------------------------------------------------------- scans

constexpr int kScanThreads = 256;
constexpr int kScanItems = 16;
constexpr int kScanTile = kScanThreads * kScanItems;

template <typename T>
__device__ __forceinline__ T block_exclusive_scan(T v, T *s_warp, T *total) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  T x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    T y = __shfl_up_sync(0xFFFFFFFFu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) s_warp[warp] = x;
  __syncthreads();
  if (warp == 0) {
    T w = lane < (kScanThreads / 32) ? s_warp[lane] : T(0);
    T wx = w;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      T y = __shfl_up_sync(0xFFFFFFFFu, wx, o);
      if (lane >= o) wx += y;
    }
    if (lane < (kScanThreads / 32)) s_warp[lane] = wx - w;
    if (lane == (kScanThreads / 32) - 1) s_warp[kScanThreads / 32] = wx;
  }
  __syncthreads();
  T r = s_warp[warp] + x - v;
  if (total) *total = s_warp[kScanThreads / 32];
  return r;
}

template <typename TIn, typename TOut>
__global__ void k_tile_reduce(const TIn *__restrict__ in, int64_t n, TOut *__restrict__ sums) {
  __shared__ TOut s_warp[kScanThreads / 32 + 1];
  int64_t start = (int64_t)blockIdx.x * kScanTile;
  int64_t end = start + kScanTile < n ? start + kScanTile : n;
  TOut s = 0;
  for (int64_t i = start + threadIdx.x; i < end; i += kScanThreads) s += (TOut)in[i];
  TOut tot;
  block_exclusive_scan<TOut>(s, s_warp, &tot);
  if (threadIdx.x == 0) sums[blockIdx.x] = tot;
}

// Exclusive scan of one tile per block, plus the block's offset.
template <typename TIn, typename TOut>
__global__ void k_tile_scan(const TIn *in, TOut *out, int64_t n, const TOut *__restrict__ offsets,
                            TOut *total) {
  __shared__ TOut s_data[kScanTile];
  __shared__ TOut s_warp[kScanThreads / 32 + 1];
  int64_t start = (int64_t)blockIdx.x * kScanTile;
  for (int i = threadIdx.x; i < kScanTile; i += kScanThreads) {
    int64_t g = start + i;
    s_data[i] = g < n ? (TOut)in[g] : TOut(0);
  }
  __syncthreads();
  TOut local[kScanItems];
  TOut sum = 0;
#pragma unroll
  for (int j = 0; j < kScanItems; j++) {
    local[j] = sum;
    sum += s_data[threadIdx.x * kScanItems + j];
  }
  TOut tile_total;
  TOut excl = block_exclusive_scan<TOut>(sum, s_warp, &tile_total);
  TOut base = offsets ? offsets[blockIdx.x] : TOut(0);
#pragma unroll
  for (int j = 0; j < kScanItems; j++) s_data[threadIdx.x * kScanItems + j] = local[j] + excl + base;
  __syncthreads();
  for (int i = threadIdx.x; i < kScanTile; i += kScanThreads) {
    int64_t g = start + i;
    if (g < n) out[g] = s_data[i];
  }
  if (total && threadIdx.x == 0 && blockIdx.x == gridDim.x - 1) *total = base + tile_total;
}

template <typename TIn, typename TOut>
static void scan_impl(gp_ctx *ctx, const TIn *in, TOut *out, int64_t n, TOut *total) {
  if (n <= 0) {
    if (total) GP_CUDA(cudaMemsetAsync(total, 0, sizeof(TOut), ctx->stream));
    return;
  }
  int64_t tiles = (n + kScanTile - 1) / kScanTile;
  if (tiles == 1) {
    k_tile_scan<TIn, TOut><<<1, kScanThreads, 0, ctx->stream>>>(in, out, n, nullptr, total);
    GP_LAUNCH_CHECK();
    return;
  }
  DBuf<TOut> sums(ctx, (size_t)tiles);
  k_tile_reduce<TIn, TOut><<<(unsigned)tiles, kScanThreads, 0, ctx->stream>>>(in, n, sums.get());
  GP_LAUNCH_CHECK();
  scan_impl<TOut, TOut>(ctx, sums.get(), sums.get(), tiles, total);
  k_tile_scan<TIn, TOut><<<(unsigned)tiles, kScanThreads, 0, ctx->stream>>>(in, out, n, sums.get(),
                                                                           nullptr);
  GP_LAUNCH_CHECK();
}

void scan_exclusive_i32(gp_ctx *ctx, const int32_t *in, int32_t *out, int64_t n, int32_t *total) {
  ProfScope ps(ctx, PROF_SCAN);
  scan_impl<int32_t, int32_t>(ctx, in, out, n, total);
}
void scan_exclusive_i64(gp_ctx *ctx, const int64_t *in, int64_t *out, int64_t n, int64_t *total) {
  ProfScope ps(ctx, PROF_SCAN);
  scan_impl<int64_t, int64_t>(ctx, in, out, n, total);
}
void scan_exclusive_i32_i64(gp_ctx *ctx, const int32_t *in, int64_t *out, int64_t n,
                            int64_t *total) {
  ProfScope ps(ctx, PROF_SCAN);
  scan_impl<int32_t, int64_t>(ctx, in, out, n, total);
}

// -------------------------------------------------------------- reductions

__global__ void k_reduce_sum(const int32_t *__restrict__ in, int64_t n,
                             unsigned long long *__restrict__ out) {
  long long s = 0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    s += in[i];
  s = warp_sum(s);
  if (lane_id() == 0 && s) atomicAdd(out, (unsigned long long)s);
}

void reduce_sum_i32_to_i64(gp_ctx *ctx, const int32_t *in, int64_t n, int64_t *out) {
  GP_CUDA(cudaMemsetAsync(out, 0, sizeof(int64_t), ctx->stream));
  if (n <= 0) return;
  k_reduce_sum<<<grid_for(n, 256, ctx->num_sms * 8), 256, 0, ctx->stream>>>(
      in, n, reinterpret_cast<unsigned long long *>(out));
  GP_LAUNCH_CHECK();
}

// -------------------------------------------------------------- radix sort

constexpr int kSortThreads = 256;
constexpr int kSortChunks = 16;
constexpr int kSortTile = kSortThreads * kSortChunks;

__global__ void k_radix_hist(const uint64_t *__restrict__ keys, int64_t n, int shift,
                             int32_t *__restrict__ hist, int64_t tiles) {
  __shared__ int32_t s_h[256];
  s_h[threadIdx.x] = 0;
  __syncthreads();
  int64_t start = (int64_t)blockIdx.x * kSortTile;
  for (int c = 0; c < kSortChunks; c++) {
    int64_t i = start + c * kSortThreads + threadIdx.x;
    bool valid = i < n;
    unsigned d = valid ? (unsigned)((keys[i] >> shift) & 255u) : 256u;
    unsigned peers = __match_any_sync(0xFFFFFFFFu, d);
    if (valid && (int)lane_id() == __ffs(peers) - 1) atomicAdd(&s_h[d], __popc(peers));
  }
  __syncthreads();
  hist[(int64_t)threadIdx.x * tiles + blockIdx.x] = s_h[threadIdx.x];
}

__global__ void k_radix_scatter(const uint64_t *__restrict__ kin, const uint32_t *__restrict__ vin,
                                uint64_t *__restrict__ kout, uint32_t *__restrict__ vout, int64_t n,
                                int shift, const int32_t *__restrict__ offs, int64_t tiles) {
  __shared__ int32_t s_wh[kSortThreads / 32][256];
  __shared__ int32_t s_base[256];
  const int warp = threadIdx.x >> 5;
  s_base[threadIdx.x] = offs[(int64_t)threadIdx.x * tiles + blockIdx.x];
  int64_t start = (int64_t)blockIdx.x * kSortTile;
  for (int c = 0; c < kSortChunks; c++) {
    for (int w = 0; w < kSortThreads / 32; w++) s_wh[w][threadIdx.x] = 0;
    __syncthreads();
    int64_t i = start + c * kSortThreads + threadIdx.x;
    bool valid = i < n;
    uint64_t key = valid ? kin[i] : 0;
    unsigned d = valid ? (unsigned)((key >> shift) & 255u) : 256u;
    unsigned peers = __match_any_sync(0xFFFFFFFFu, d);
    int rank = __popc(peers & lanemask_lt());
    if (valid && (int)lane_id() == __ffs(peers) - 1) s_wh[warp][d] = __popc(peers);
    __syncthreads();
    {
      int dd = threadIdx.x;
      int run = s_base[dd];
#pragma unroll
      for (int w = 0; w < kSortThreads / 32; w++) {
        int t = s_wh[w][dd];
        s_wh[w][dd] = run;
        run += t;
      }
      s_base[dd] = run;
    }
    __syncthreads();
    if (valid) {
      int pos = s_wh[warp][d] + rank;
      kout[pos] = key;
      vout[pos] = vin[i];
    }
    __syncthreads();
  }
}

void radix_sort_pairs(gp_ctx *ctx, uint64_t *keys, uint32_t *vals, int64_t n, int bits) {
  if (n <= 1 || bits <= 0) return;
  ProfScope ps(ctx, PROF_SORT);
  GP_REQUIRE(n < ((int64_t)1 << 31), GP_ERR_INVALID, "radix sort: too many keys");
  int64_t tiles = (n + kSortTile - 1) / kSortTile;
  DBuf<uint64_t> k2(ctx, (size_t)n);
  DBuf<uint32_t> v2(ctx, (size_t)n);
  DBuf<int32_t> hist(ctx, (size_t)(256 * tiles));
  uint64_t *ka = keys, *kb = k2.get();
  uint32_t *va = vals, *vb = v2.get();
  int passes = (bits + 7) / 8;
  for (int p = 0; p < passes; p++) {
    int shift = p * 8;
    k_radix_hist<<<(unsigned)tiles, kSortThreads, 0, ctx->stream>>>(ka, n, shift, hist.get(), tiles);
    GP_LAUNCH_CHECK();
    scan_impl<int32_t, int32_t>(ctx, hist.get(), hist.get(), 256 * tiles, nullptr);
    k_radix_scatter<<<(unsigned)tiles, kSortThreads, 0, ctx->stream>>>(ka, va, kb, vb, n, shift,
                                                                       hist.get(), tiles);
    GP_LAUNCH_CHECK();
    std::swap(ka, kb);
    std::swap(va, vb);
  }
  if (ka != keys) {
    GP_CUDA(cudaMemcpyAsync(keys, ka, sizeof(uint64_t) * n, cudaMemcpyDeviceToDevice, ctx->stream));
    GP_CUDA(cudaMemcpyAsync(vals, va, sizeof(uint32_t) * n, cudaMemcpyDeviceToDevice, ctx->stream));
  }
}

// ------------------------------------------------------------ graph export

struct ExportedGraph {
  DevGraph g;
};

void export_graph(gp_ctx *ctx, DevGraph &&g, gp_graph *out) {
  (void)ctx;
  *out = g.view();
  // ownership passes to the caller: the buffers are freed by gp_graph_release
  g.bx.p = nullptr; g.ba.p = nullptr; g.bv.p = nullptr; g.bw.p = nullptr;
}

}  // namespace gp
