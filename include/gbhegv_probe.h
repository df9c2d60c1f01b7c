/*
 * gbhegv_probe.h -- FP64 throughput probe of libgbhegv, used to report the
 * roofline of the FP64 kernels against a peak measured live on the same GPU.
 * The paper has no counterpart (it names no peak); this is measurement
 * infrastructure for the benchmark.
 */
#ifndef GBHEGV_PROBE_H_
#define GBHEGV_PROBE_H_

#ifdef __cplusplus
extern "C" {
#endif

/* Run two short saturating kernels on `device` and return their FP64 rates
 * in TFLOP/s (2 flops per fused multiply-add):
 *   dfma_tflops  scalar FP64 FMA pipe (8 independent chains per thread);
 *   dmma_tflops  FP64 tensor pipe, mma.sync.aligned.m16n8k4 .f64 (the
 *                instruction the library's GEMM uses).
 * Allocates and frees a small output buffer; synchronous.  Returns 0 or a
 * negative GBHE_* code. */
int gbhe_probe_fp64_peaks(int device, double* dfma_tflops, double* dmma_tflops);

#ifdef __cplusplus
}
#endif

#endif /* GBHEGV_PROBE_H_ */
