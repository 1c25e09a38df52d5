// engine_k1024.cu -- the batched engine kernel with 1024 threads per CTA.
#include "engine_dev.cuh"

namespace gp {
namespace eng {

namespace {
void launch1024(int grid, size_t smem, cudaStream_t stream, const EArgs &a) {
  k_engine<1024><<<grid, 1024, smem, stream>>>(a);
}
}  // namespace

Kernel kernel_1024() { return Kernel{launch1024, (const void *)k_engine<1024>, 1024}; }

}  // namespace eng
}  // namespace gp
