// noalloc.cu -- the complex DMMA GEMM with its split-K partial sums in a
// statically sized device array instead of caller-provided workspace.
//
// The ordinary entry points take their scratch from the workspace a caller
// attaches to a handle.  Some callers cannot do that: code that must not
// allocate device memory after start-up (a serving loop whose memory is fixed
// once, or an allocator-frozen phase of a larger program) and code that holds
// no handle at all.  gbhe_zgemm_static serves them: it needs no handle and
// allocates nothing; the only device memory it touches besides the operands
// is the file-scope array below, which the CUDA module provides when the
// library is loaded.
#include <mutex>

#include "internal.cuh"

// Split-K partial sums: GBHE_ZGEMM_STATIC_SCRATCH complex128 values (16 MiB).
// Every split writes all of its partial sums before the reduction reads them,
// so nothing here has to start at zero.
static __device__ __align__(256) double2 g_static_partial[GBHE_ZGEMM_STATIC_SCRATCH];

namespace {

constexpr int kMaxDevices = 64;
std::once_flag g_once[kMaxDevices];
void* g_addr[kMaxDevices];
cudaError_t g_setup_err[kMaxDevices];

// Address of the array on the current device, looked up once per device.
int static_scratch(int dev, void** out) {
  std::call_once(g_once[dev], [dev] {
    void* p = nullptr;
    g_setup_err[dev] = cudaGetSymbolAddress(&p, g_static_partial);
    g_addr[dev] = p;
  });
  if (g_setup_err[dev] != cudaSuccess || !g_addr[dev]) return GBHE_ECUDA;
  *out = g_addr[dev];
  return 0;
}

}  // namespace

extern "C" int gbhe_zgemm_static(int opA, int opB, int m, int n, int k, gbhe_cplx alpha, const gbhe_cplx* A,
                                 int lda, const gbhe_cplx* B, int ldb, gbhe_cplx beta, gbhe_cplx* C, int ldc,
                                 int lower, void* stream) {
  using namespace gbhe;
  if (opA < 0 || opA > 3) return -1;
  if (opB < 0 || opB > 2) return -2;
  if (m < 0) return -3;
  if (n < 0) return -4;
  if (k < 0) return -5;
  const int ra = (opA == OP_N || opA == OP_H) ? m : k;
  if (m > 0 && k > 0 && !A) return -7;
  if (lda < std::max(1, ra)) return -8;
  const int rb = (opB == OP_N) ? k : n;
  if (n > 0 && k > 0 && !B) return -9;
  if (ldb < std::max(1, rb)) return -10;
  if (m > 0 && n > 0 && !C) return -12;
  if (ldc < std::max(1, m)) return -13;
  if (opA == OP_H && m != k) return -1;
  if ((long long)m * n > GBHE_ZGEMM_STATIC_MAX_MN) return GBHE_ETOOLARGE;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return GBHE_ECUDA;
  if (dev < 0 || dev >= kMaxDevices) return GBHE_ECUDA;
  void* scratch = nullptr;
  int rc = static_scratch(dev, &scratch);
  if (rc) return rc;
  const GemmArgs g = gemm_args(opA, opB, m, n, k, mk(alpha.re, alpha.im), A, lda, B, ldb, mk(beta.re, beta.im), C,
                               ldc, lower);
  return zgemm(static_cast<cudaStream_t>(stream), g, scratch, sizeof(double2) * (size_t)GBHE_ZGEMM_STATIC_SCRATCH);
}
