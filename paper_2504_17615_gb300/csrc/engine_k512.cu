// engine_k512.cu -- the batched engine kernel with 512 threads per CTA.
#include "engine_dev.cuh"

namespace gp {
namespace eng {

namespace {
void launch512(int grid, size_t smem, cudaStream_t stream, const EArgs &a) {
  k_engine<512><<<grid, 512, smem, stream>>>(a);
}
}  // namespace

Kernel kernel_512() { return Kernel{launch512, (const void *)k_engine<512>, 512}; }

}  // namespace eng
}  // namespace gp
