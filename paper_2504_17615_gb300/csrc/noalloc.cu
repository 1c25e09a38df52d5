// noalloc.cu -- gp_cut_noalloc: cut weight and block weights of a partition
// computed without allocating any memory.
//
// Some callers cannot allocate device memory while they run: a serving loop
// that has reserved the whole device for its own memory arena up front, or a
// latency-critical path where cudaMalloc's implicit device-wide
// synchronisation is not acceptable.  This entry point serves them: its only
// scratch is the file-scope device array below, of fixed size, so a call
// performs no cudaMalloc, cudaFree or other allocation (the caller passes the
// graph, the block ids and the host outputs).
//
// The array lives in every device that loads the library, until the process
// exits.  Host code cannot use its name as a device address (the host-side
// symbol is only a stand-in), so the first call on each device, with that
// device current, looks the address up with cudaGetSymbolAddress and caches
// it; that first call on a device should therefore come before any stream
// capture on it.  All calls share the array and it keeps the previous call's
// contents, so every call clears the part it uses first; calls that overlap
// on the GPU (for example on two streams at once) race on the array and give
// wrong results.
#include "gp_internal.cuh"

#include <mutex>

namespace {

constexpr int kMaxK = GP_CUT_NOALLOC_MAX_K;
constexpr int kMaxDevices = 64;

// [0] twice the cut, [1] error flag (block id out of range), [2 .. 2 + k) block weights
static __device__ __align__(256) unsigned long long g_cut_scratch[2 + kMaxK];

unsigned long long *g_scratch_addr[kMaxDevices] = {};
std::mutex g_scratch_mutex;

__global__ void k_na_clear(unsigned long long *s, int count) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < count; i += gridDim.x * blockDim.x) s[i] = 0;
}

__global__ void __launch_bounds__(256) k_na_cut(const int32_t *xadj, const int32_t *adjncy,
                                                const int32_t *adjwgt, const int32_t *blk, int n,
                                                int64_t m2, unsigned long long *s) {
  const int lane = (int)gp::lane_id();
  const int64_t chunk = 1024;
  const int64_t nchunks = (m2 + chunk - 1) / chunk;
  const int64_t wid = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  unsigned long long sum = 0;
  for (int64_t c = wid; c < nchunks; c += nw) {
    const int64_t e0 = c * chunk;
    const int64_t e1 = e0 + chunk < m2 ? e0 + chunk : m2;
    int row = 0;
    if (lane == 0) row = gp::row_of(xadj, n, e0);
    row = __shfl_sync(0xFFFFFFFFu, row, 0);
    for (int64_t e = e0 + lane; e < e1; e += 32) {
      while (row < n - 1 && (int64_t)xadj[row + 1] <= e) row++;
      if (blk[adjncy[e]] != blk[row]) sum += (unsigned long long)adjwgt[e];
    }
  }
  sum = gp::warp_sum(sum);
  if (lane == 0 && sum) atomicAdd(&s[0], sum);
}

__global__ void __launch_bounds__(256) k_na_weights(const int32_t *blk, const int32_t *vwgt, int n, int k,
                                                    unsigned long long *s) {
  __shared__ unsigned long long s_bw[kMaxK];
  for (int b = threadIdx.x; b < k; b += blockDim.x) s_bw[b] = 0;
  __syncthreads();
  bool bad = false;
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n;
       v += (int64_t)gridDim.x * blockDim.x) {
    const int b = blk[v];
    if (b < 0 || b >= k) { bad = true; continue; }
    atomicAdd(&s_bw[b], (unsigned long long)vwgt[v]);
  }
  __syncthreads();
  for (int b = threadIdx.x; b < k; b += blockDim.x)
    if (s_bw[b]) atomicAdd(&s[2 + b], s_bw[b]);
  if (bad) s[1] = 1;
}

// Device address of the scratch array on the current device (looked up once).
unsigned long long *scratch_on_current_device(gp_status *st) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    *st = GP_ERR_CUDA;
    return nullptr;
  }
  std::lock_guard<std::mutex> lock(g_scratch_mutex);
  if (!g_scratch_addr[dev]) {
    void *p = nullptr;
    if (cudaGetSymbolAddress(&p, g_cut_scratch) != cudaSuccess || !p) {
      (void)cudaGetLastError();
      *st = GP_ERR_CUDA;
      return nullptr;
    }
    g_scratch_addr[dev] = static_cast<unsigned long long *>(p);
  }
  return g_scratch_addr[dev];
}

}  // namespace

extern "C" gp_status gp_cut_noalloc(const gp_graph *g, const int32_t *blocks, int32_t k, void *stream,
                                    int64_t *cut, int64_t *block_weights) {
  if (!g || !cut || k < 1 || g->n < 0 || g->m2 < 0 || g->m2 >= ((int64_t)1 << 31)) return GP_ERR_INVALID;
  if (k > kMaxK) return GP_ERR_INVALID;  // the fixed scratch holds at most GP_CUT_NOALLOC_MAX_K blocks
  if (g->n > 0 && (!g->xadj || !g->vwgt || !blocks)) return GP_ERR_INVALID;
  if (g->m2 > 0 && (g->n == 0 || !g->adjncy || !g->adjwgt)) return GP_ERR_INVALID;  // entries need rows
  gp_status st = GP_OK;
  unsigned long long *s = scratch_on_current_device(&st);
  if (!s) return st;
  cudaStream_t sm = (cudaStream_t)stream;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return GP_ERR_CUDA;
  k_na_clear<<<gp::grid_for(2 + k, 256, 64), 256, 0, sm>>>(s, 2 + k);
  int launched = 1;
  if (g->m2 > 0) {
    k_na_cut<<<gp::grid_for((g->m2 + 1023) / 1024 * 32, 256, sms * 16), 256, 0, sm>>>(
        g->xadj, g->adjncy, g->adjwgt, blocks, g->n, g->m2, s);
    launched++;
  }
  if (g->n > 0) {
    k_na_weights<<<gp::grid_for(g->n, 256, sms * 4), 256, 0, sm>>>(blocks, g->vwgt, g->n, k, s);
    launched++;
  }
  gp::g_launch_count.fetch_add(launched, std::memory_order_relaxed);
  if (cudaGetLastError() != cudaSuccess) return GP_ERR_CUDA;
  unsigned long long hdr[2] = {0, 0};
  if (cudaMemcpyAsync(hdr, s, sizeof(hdr), cudaMemcpyDeviceToHost, sm) != cudaSuccess) return GP_ERR_CUDA;
  if (block_weights &&
      cudaMemcpyAsync(block_weights, s + 2, sizeof(int64_t) * k, cudaMemcpyDeviceToHost, sm) != cudaSuccess)
    return GP_ERR_CUDA;
  if (cudaStreamSynchronize(sm) != cudaSuccess) return GP_ERR_CUDA;
  if (hdr[1]) return GP_ERR_INVALID;  // a block id outside [0, k)
  *cut = (int64_t)(hdr[0] / 2);
  return GP_OK;
}
