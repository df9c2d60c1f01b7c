// selftest.cu -- failure detection without a GPU fault.  One CTA enters the
// library's bounded grid barrier (the one the cooperative panel QR uses)
// expecting a second CTA that is never launched; the wait expires after
// GBHE_WAIT_NS of %globaltimer, records GBHE_ETIMEOUT in the handle's status
// word and the kernel returns normally, so the context stays usable.
#include "internal.cuh"

namespace gbhe {
namespace {

__global__ void k_wait_expire(unsigned* bar, int* st) { grid_barrier(bar, 2u, st); }

}  // namespace
}  // namespace gbhe

extern "C" int gbhe_wait_selftest(gbhe_handle h, void* stream) {
  using namespace gbhe;
  if (!h) return -1;
  if (cudaSetDevice(h->device) != cudaSuccess) return GBHE_ECUDA;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  GBHE_CUDA(cudaMemsetAsync(h->status + ST_SELF, 0, 2 * sizeof(int), st));
  k_wait_expire<<<1, 32, 0, st>>>(reinterpret_cast<unsigned*>(h->status + ST_SELF), h->status);
  count_launch();
  GBHE_CUDA(cudaGetLastError());
  return 0;
}
