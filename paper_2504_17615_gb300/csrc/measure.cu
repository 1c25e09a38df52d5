// measure.cu -- rate of random 4-byte reads (a bound of the gather-heavy
// kernels; no counterpart in the paper).
#include "gp_internal.cuh"

namespace gp {

namespace {

constexpr int kReadUnroll = 4;

__global__ void __launch_bounds__(256) k_random_reads(const int32_t *a, uint32_t len, int64_t reads,
                                                      uint64_t key, int32_t *sink) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  int acc = 0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < reads; i += stride * kReadUnroll) {
    int x[kReadUnroll];
#pragma unroll
    for (int r = 0; r < kReadUnroll; r++) {
      const int64_t j = i + r * stride;
      // index in [0, len): the top 32 bits of a hash scaled by len
      const uint32_t idx = (uint32_t)(((uint64_t)h32(key, (uint32_t)j, (uint32_t)(j >> 32)) * len) >> 32);
      x[r] = j < reads ? a[idx] : 0;
    }
#pragma unroll
    for (int r = 0; r < kReadUnroll; r++) acc += x[r];
  }
  if (acc == 0x7FFFFFFF) *sink = acc;  // keeps the reads alive
}

}  // namespace

double measure_random_reads(gp_ctx *ctx, int64_t array_bytes, int64_t reads) {
  GP_REQUIRE(array_bytes >= 4 && array_bytes / 4 <= 0xFFFFFFFFll, GP_ERR_INVALID, "array size out of range");
  GP_REQUIRE(reads > 0, GP_ERR_INVALID, "reads must be positive");
  const uint32_t len = (uint32_t)(array_bytes / 4);
  DBuf<int32_t> a(ctx, len), sink(ctx, 1);
  GP_CUDA(cudaMemsetAsync(a.get(), 1, sizeof(int32_t) * (size_t)len, ctx->stream));
  cudaEvent_t e0, e1;
  GP_CUDA(cudaEventCreate(&e0));
  GP_CUDA(cudaEventCreate(&e1));
  const int grid = ctx->num_sms * 8;
  float ms = 0;
  for (int it = 0; it < 3; it++) {
    GP_CUDA(cudaEventRecord(e0, ctx->stream));
    k_random_reads<<<grid, 256, 0, ctx->stream>>>(a.get(), len, reads, stream_key(0x5EEDull, 0, 0, it),
                                                  sink.get());
    GP_LAUNCH_CHECK();
    GP_CUDA(cudaEventRecord(e1, ctx->stream));
    GP_CUDA(cudaEventSynchronize(e1));
    GP_CUDA(cudaEventElapsedTime(&ms, e0, e1));
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return ms > 0 ? (double)reads / (ms * 1e-3) : 0.0;
}

}  // namespace gp
