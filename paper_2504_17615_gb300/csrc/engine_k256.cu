// engine_k256.cu -- the batched engine kernel with 256 threads per CTA.
#include "engine_dev.cuh"

namespace gp {
namespace eng {

namespace {
void launch256(int grid, size_t smem, cudaStream_t stream, const EArgs &a) {
  k_engine<256><<<grid, 256, smem, stream>>>(a);
}
}  // namespace

Kernel kernel_256() { return Kernel{launch256, (const void *)k_engine<256>, 256}; }

}  // namespace eng
}  // namespace gp
