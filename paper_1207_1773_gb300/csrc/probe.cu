// probe.cu -- live FP64 peak measurement (DFMA and DMMA m16n8k4) for the
// benchmark's roofline denominators.
#include "common.cuh"
#include "../../include/gbhegv_probe.h"

namespace {

constexpr int ITERS = 2048;

__global__ void k_probe_dfma(double* out, double s) {
  double a0 = threadIdx.x * 1e-9, a1 = a0 + 1, a2 = a0 + 2, a3 = a0 + 3, a4 = a0 + 4, a5 = a0 + 5,
         a6 = a0 + 6, a7 = a0 + 7;
  const double m = 1.0000001 + s;
  for (int i = 0; i < ITERS; ++i) {
    a0 = fma(a0, m, s); a1 = fma(a1, m, s); a2 = fma(a2, m, s); a3 = fma(a3, m, s);
    a4 = fma(a4, m, s); a5 = fma(a5, m, s); a6 = fma(a6, m, s); a7 = fma(a7, m, s);
  }
  out[blockIdx.x * blockDim.x + threadIdx.x] = a0 + a1 + a2 + a3 + a4 + a5 + a6 + a7;
}

// The operands change every iteration and the accumulators start distinct:
// with loop-invariant operands the measured rate comes out twice the real one.
__global__ void k_probe_dmma(double* out) {
  double a0 = threadIdx.x * 1e-3 + blockIdx.x, a1 = a0 + 1, b = 1.0 + threadIdx.x * 1e-4;
  double c[4][4];
  for (int j = 0; j < 4; ++j)
    for (int q = 0; q < 4; ++q) c[j][q] = 0.5 * j + q;
  for (int i = 0; i < ITERS; ++i) {
#pragma unroll
    for (int j = 0; j < 4; ++j)
      asm volatile(
          "mma.sync.aligned.m16n8k4.row.col.f64.f64.f64.f64 {%0,%1,%2,%3}, {%4,%5}, {%6}, "
          "{%0,%1,%2,%3};"
          : "+d"(c[j][0]), "+d"(c[j][1]), "+d"(c[j][2]), "+d"(c[j][3])
          : "d"(a0), "d"(a1), "d"(b));
    a0 += 1e-9;
  }
  // every accumulator value is consumed: dead output rows let the compiler
  // drop half of an m16n8k4 product and the rate would read twice too high
  double s = 0.0;
  for (int j = 0; j < 4; ++j) s += c[j][0] + c[j][1] + c[j][2] + c[j][3];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

}  // namespace

extern "C" int gbhe_probe_fp64_peaks(int device, double* dfma_tflops, double* dmma_tflops) {
  if (cudaSetDevice(device) != cudaSuccess) return GBHE_ECUDA;
  cudaDeviceProp p;
  if (cudaGetDeviceProperties(&p, device) != cudaSuccess) return GBHE_ECUDA;
  const int threads = 256, blocks = p.multiProcessorCount * 8;
  const size_t nout = (size_t)blocks * threads;
  double* out = nullptr;
  if (cudaMalloc(&out, nout * sizeof(double)) != cudaSuccess) return GBHE_ECUDA;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  float best_f = 1e30f, best_m = 1e30f;
  for (int rep = 0; rep < 3; ++rep) {
    float ms;
    cudaEventRecord(e0);
    k_probe_dfma<<<blocks, threads>>>(out, 1e-12);
    gbhe::count_launch();
    cudaEventRecord(e1);
    cudaEventSynchronize(e1);
    cudaEventElapsedTime(&ms, e0, e1);
    if (rep > 0 && ms < best_f) best_f = ms;
    cudaEventRecord(e0);
    k_probe_dmma<<<blocks, threads>>>(out);
    gbhe::count_launch();
    cudaEventRecord(e1);
    cudaEventSynchronize(e1);
    cudaEventElapsedTime(&ms, e0, e1);
    if (rep > 0 && ms < best_m) best_m = ms;
  }
  const cudaError_t err = cudaGetLastError();
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(out);
  if (err != cudaSuccess) return GBHE_ECUDA;
  const double warps = (double)blocks * threads / 32.0;
  if (dfma_tflops) *dfma_tflops = 2.0 * 8 * ITERS * (double)nout / (best_f * 1e-3) / 1e12;
  if (dmma_tflops) *dmma_tflops = 2.0 * 16 * 8 * 4 * 4 * ITERS * warps / (best_m * 1e-3) / 1e12;
  return 0;
}
