// gemm.cuh -- FP64 tensor-core (DMMA, mma.sync m16n8k4 f64) GEMM used by every
// level-3 step of the solver: C = alpha op(A) op(B) + beta C, complex128 or
// real FP64, column-major.
#pragma once
#include "common.cuh"

namespace gbhe {

enum Op { OP_N = 0, OP_T = 1, OP_C = 2, OP_H = 3 /* Hermitian, lower-stored square */ };

struct GemmArgs {
  int opA, opB, m, n, k;
  cplx alpha, beta;
  const void* A;
  int lda;
  const void* B;
  int ldb;
  void* C;
  int ldc;
  int lower_only;  // write only C(i,j) with i >= j (tiles above the diagonal skipped)
};

// Complex GEMM.  `scratch`/`scratch_bytes` is device memory used for split-K
// partial sums when m*n is small and k large (may be null: no split).
int zgemm(cudaStream_t st, const GemmArgs& g, void* scratch, size_t scratch_bytes);
// Real FP64 GEMM (A, B, C double; alpha.x/beta.x used).
int dgemm(cudaStream_t st, const GemmArgs& g, void* scratch, size_t scratch_bytes);

// Grouped real GEMM whose sizes live in device memory (used where sizes are
// only known on the device).  desc[i] = {m, n, k, lda, ldb, ldc} with
// pointers A[i], B[i], C[i]; C = alpha A B + beta C (no transposes).
struct DGroupDesc {
  const double* A;
  const double* B;
  double* C;
  const int* cmap;  // optional: column j of the product goes to column cmap[j] of C
  int m, n, k, lda, ldb, ldc;
};
int dgemm_grouped(cudaStream_t st, const DGroupDesc* d_desc, int ngroups, int max_m, int max_n,
                  double alpha, double beta);

inline GemmArgs gemm_args(int opA, int opB, int m, int n, int k, cplx alpha, const void* A, int lda,
                          const void* B, int ldb, cplx beta, void* C, int ldc, int lower = 0) {
  GemmArgs g;
  g.opA = opA; g.opB = opB; g.m = m; g.n = n; g.k = k; g.alpha = alpha; g.beta = beta;
  g.A = A; g.lda = lda; g.B = B; g.ldb = ldb; g.C = C; g.ldc = ldc; g.lower_only = lower;
  return g;
}

}  // namespace gbhe
