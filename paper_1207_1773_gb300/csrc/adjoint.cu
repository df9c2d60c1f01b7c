// adjoint.cu -- reverse-mode derivative of the selected eigenpairs of the
// Hermitian-definite problem A x = lambda B x (X^H B X = I), from first-order
// perturbation theory (the paper has no counterpart):
//
//   d lambda_i = x_i^H (dA - lambda_i dB) x_i
//   d x_i      = sum_{j != i} x_j x_j^H (dA - lambda_i dB) x_i / (lambda_i - lambda_j)
//                - 1/2 x_i (x_i^H dB x_i)            (phase of x_i left free)
//
// with j over the whole spectrum.  For a real loss L with cotangents
// g_i = dL/dlambda_i and G_i (dL = sum g_i dlambda_i + Re sum G_i^H dx_i):
//
//   K = X_all^H G,  K'_ji = K_ji / (lambda_i - lambda_j)  (0 for j = i and for
//                   |lambda_i - lambda_j| < delta: degenerate-gap masking)
//   U = X_all K',   c_i = Re(x_i^H G_i)
//   W_A = X_S diag(g) + U,   W_B = X_S diag(lambda g + c/2) + U diag(lambda)
//   dL/dA = herm(X_S W_A^H),  dL/dB = -herm(X_S W_B^H),  herm(M) = (M + M^H)/2
//
// so that dL = Re tr(dL/dA^H dA) + Re tr(dL/dB^H dB) for Hermitian dA, dB.
#include <algorithm>

#include "internal.cuh"

namespace gbhe {
namespace {

// K (n x m) -> K' in place; c_i = Re K(il-1+i, i) first.
__global__ void k_adj_scale(int n, int m, int il, const double* w_all, double delta, cplx* K, int ldk, double* c) {
  const size_t total = (size_t)n * m;
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < total; t += (size_t)gridDim.x * blockDim.x) {
    const int j = (int)(t % n), i = (int)(t / n), gi = il - 1 + i;
    cplx v = K[(size_t)j + (size_t)i * ldk];
    if (j == gi) {
      c[i] = v.x;
      v = mk(0.0, 0.0);
    } else {
      const double gap = w_all[gi] - w_all[j];
      v = fabs(gap) < delta ? mk(0.0, 0.0) : cscal(1.0 / gap, v);
    }
    K[(size_t)j + (size_t)i * ldk] = v;
  }
}

// W_A = X_S diag(g) + U,  W_B = X_S diag(lambda g + c/2) + U diag(lambda)
__global__ void k_adj_w(int n, int m, int il, const double* w_all, const double* g, const double* c, const cplx* X,
                        int ldx, const cplx* U, int ldu, cplx* WA, cplx* WB, int ldw) {
  const size_t total = (size_t)n * m;
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < total; t += (size_t)gridDim.x * blockDim.x) {
    const int r = (int)(t % n), i = (int)(t / n);
    const double lam = w_all[il - 1 + i];
    const cplx x = X[(size_t)r + (size_t)(il - 1 + i) * ldx];
    const cplx u = U[(size_t)r + (size_t)i * ldu];
    WA[(size_t)r + (size_t)i * ldw] = cadd(cscal(g[i], x), u);
    WB[(size_t)r + (size_t)i * ldw] = cadd(cscal(lam * g[i] + 0.5 * c[i], x), cscal(lam, u));
  }
}

}  // namespace

size_t adjoint_ws_bytes(int n, int m) {
  const size_t nn = (size_t)std::max(n, 1), mm = (size_t)std::max(m, 1);
  return 4 * nn * mm * sizeof(cplx) + mm * sizeof(double) + 5 * 256;
}

int adjoint_run(Ctx& c, int n, int il, int iu, const double* w_all, const cplx* X, int ldx, const double* g,
                const cplx* G, int ldg, double delta, cplx* dA, int ldda, cplx* dB, int lddb) {
  const int m = iu - il + 1;
  if (n <= 0 || m <= 0) return 0;
  Arena& ar = c.arena;
  const size_t save = ar.off;
  cplx* K = ar.take<cplx>((size_t)n * m);
  cplx* U = ar.take<cplx>((size_t)n * m);
  cplx* WA = ar.take<cplx>((size_t)n * m);
  cplx* WB = ar.take<cplx>((size_t)n * m);
  double* cv = ar.take<double>((size_t)m);
  if (!ar.ok() || !cv) { ar.off = save; return GBHE_EWORKSPACE; }
  const cplx one = mk(1, 0), zero = mk(0, 0), half = mk(0.5, 0), mhalf = mk(-0.5, 0);
  const cplx* XS = X + (size_t)(il - 1) * ldx;
  const int blocks = (int)std::min<size_t>(((size_t)n * m + 255) / 256, 4096);
  int rc;
  // K = X_all^H G
  if ((rc = gemm(c, gemm_args(OP_C, OP_N, n, m, n, one, X, ldx, G, ldg, zero, K, n), 1))) { ar.off = save; return rc; }
  k_adj_scale<<<blocks, 256, 0, c.st>>>(n, m, il, w_all, delta, K, n, cv);
  count_launch();
  // U = X_all K'
  if ((rc = gemm(c, gemm_args(OP_N, OP_N, n, m, n, one, X, ldx, K, n, zero, U, n), 1))) { ar.off = save; return rc; }
  k_adj_w<<<blocks, 256, 0, c.st>>>(n, m, il, w_all, g, cv, X, ldx, U, n, WA, WB, n);
  count_launch();
  GBHE_CUDA(cudaGetLastError());
  // dA = (X_S W_A^H + W_A X_S^H) / 2,  dB = -(X_S W_B^H + W_B X_S^H) / 2
  if ((rc = gemm(c, gemm_args(OP_N, OP_C, n, n, m, half, XS, ldx, WA, n, zero, dA, ldda), 1)) ||
      (rc = gemm(c, gemm_args(OP_N, OP_C, n, n, m, half, WA, n, XS, ldx, one, dA, ldda), 1)) ||
      (rc = gemm(c, gemm_args(OP_N, OP_C, n, n, m, mhalf, XS, ldx, WB, n, zero, dB, lddb), 1)) ||
      (rc = gemm(c, gemm_args(OP_N, OP_C, n, n, m, mhalf, WB, n, XS, ldx, one, dB, lddb), 1))) {
    ar.off = save;
    return rc;
  }
  ar.off = save;
  return 0;
}

}  // namespace gbhe
