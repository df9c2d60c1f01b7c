// backtransform.cu -- Algorithm 2 step 3 for two stages (paper Section 4.2):
// X = Q1 Q2 Z.  Because the reduction ran in two steps, the back-transform
// does too.
//
// Q2 (bulge-chasing reflectors).  Q2 = prod over sweeps s (ascending) and
// steps j of H(s, j); H(s, j) acts on rows s+1+j*nb .. s+(j+1)*nb.  Within a
// sweep the steps act on disjoint rows (they commute); H(s+1, .) overlaps
// H(s, .) only for equal or neighbouring steps.  Grouping nb consecutive
// sweeps, the valid order is: groups from last to first; inside a group step
// j ascending; inside (group, j) sweeps descending.  Each CTA owns a slab of
// SLAB columns of X and walks all reflectors in that order, keeping the
// (2nb-1)-row window of the current (group, j) in shared memory.
//
// Q1 (panel block reflectors of stage 1).  Q1 = Q_0 Q_1 ... with
// Q_p = I - V_p T_p V_p^H on rows p*nb+nb .. n-1, applied last panel first
// as three DMMA GEMMs: W = V^H X, W = T W, X -= V W.
#include <algorithm>
#include "internal.cuh"

namespace gbhe {
namespace {

constexpr int SLAB = 16;
constexpr int QT = 128;  // 16 columns x 8 lanes

__global__ void k_promote(const double* Z, int ldz, int n, int m, cplx* X, int ldx) {
  const size_t total = (size_t)n * m;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total;
       i += (size_t)gridDim.x * blockDim.x) {
    const int r = (int)(i % n), c = (int)(i / n);
    X[(size_t)r + (size_t)c * ldx] = mk(Z[(size_t)r + (size_t)c * ldz], 0.0);
  }
}

__global__ void __launch_bounds__(QT) k_apply_q2(int n, int nb, int m, int J, const cplx* V2,
                                                 const cplx* tau2, cplx* X, int ldx) {
  extern __shared__ cplx sm[];
  cplx* Ys = sm;                      // (2nb) x SLAB, ld 2nb
  cplx* vs = sm + 2 * nb * SLAB;      // 2 x nb
  const int t = threadIdx.x, col = t >> 3, sub = t & 7;
  const int c0 = blockIdx.x * SLAB;
  const int gc = c0 + col;
  const int W = 2 * nb;
  const int ngroups = (n - 1 + nb - 1) / nb;  // sweeps 0..n-2
  for (int b = ngroups - 1; b >= 0; --b) {
    const int s0 = b * nb;
    const int s_last = std::min(s0 + nb - 1, n - 2);
    const int jmax = (n - 1 - s0 + nb - 1) / nb;  // steps of the first sweep of the group
    for (int j = 0; j < jmax; ++j) {
      const int lo_w = s0 + 1 + j * nb;
      if (lo_w >= n) break;
      const int hi_w = std::min(n, s0 + nb + (j + 1) * nb);
      const int rows = hi_w - lo_w;
      __syncthreads();
      for (int i = t; i < rows * SLAB; i += QT) {
        const int r = i % rows, c = i / rows;
        Ys[r + c * W] = (c0 + c < m) ? X[(size_t)(lo_w + r) + (size_t)(c0 + c) * ldx] : mk(0.0, 0.0);
      }
      int buf = 0;
      for (int s = s_last; s >= s0; --s) {
        const int ntask = (n - 1 - s + nb - 1) / nb;
        if (j >= ntask) continue;
        const int a = s + 1 + j * nb;
        const int L = std::min(nb, n - a);
        const cplx* v = V2 + ((size_t)s * J + j) * nb;
        cplx* vb = vs + buf * nb;
        for (int i = t; i < L; i += QT) vb[i] = v[i];
        const cplx tau = tau2[(size_t)s * J + j];
        __syncthreads();
        if (tau.x != 0.0 || tau.y != 0.0) {
          cplx* y = Ys + (a - lo_w) + col * W;
          cplx acc = mk(0.0, 0.0);
          for (int r = sub; r < L; r += 8) ccfma(acc, vb[r], y[r]);
#pragma unroll
          for (int o = 4; o > 0; o >>= 1) {
            acc.x += __shfl_xor_sync(0xffffffffu, acc.x, o);
            acc.y += __shfl_xor_sync(0xffffffffu, acc.y, o);
          }
          const cplx tw = cmul(tau, acc);
          for (int r = sub; r < L; r += 8) y[r] = csub(y[r], cmul(vb[r], tw));
        }
        buf ^= 1;
      }
      __syncthreads();
      if (gc < m)
        for (int r = sub; r < rows; r += 8) X[(size_t)(lo_w + r) + (size_t)gc * ldx] = Ys[r + col * W];
    }
  }
}

// Explicit V of panel p (mp x kr, ld ldv): unit diagonal, zeros above, the
// stored reflectors below.
__global__ void k_panel_v(const cplx* A, int lda, int k, int nb, int mp, int kr, cplx* V, int ldv) {
  const size_t total = (size_t)mp * nb;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total;
       i += (size_t)gridDim.x * blockDim.x) {
    const int r = (int)(i % mp), c = (int)(i / mp);
    cplx e = mk(0.0, 0.0);
    if (c < kr) {
      if (r == c) e = mk(1.0, 0.0);
      else if (r > c) e = A[(size_t)(k + nb + r) + (size_t)(k + c) * lda];
    }
    V[(size_t)r + (size_t)c * ldv] = e;
  }
}

}  // namespace

size_t unmtr_ws_bytes(int n, int nb, int m) {
  const size_t nn = (size_t)std::max(n, 1), mm = (size_t)std::max(m, 1);
  return nn * nb * sizeof(cplx) + 2 * (size_t)nb * mm * sizeof(cplx) + 3 * 256;
}

int unmtr2_run(Ctx& c, int n, int nb, int m, const cplx* A, int lda, const cplx* T1, const cplx* V2,
               const cplx* tau2, const double* Z, int ldz, cplx* X, int ldx) {
  if (n <= 0 || m <= 0) return 0;
  Arena& ar = c.arena;
  const size_t save = ar.off;
  cplx* V = ar.take<cplx>((size_t)n * nb);
  cplx* W1 = ar.take<cplx>((size_t)nb * m);
  cplx* W2 = ar.take<cplx>((size_t)nb * m);
  if (!ar.ok() || !V) { ar.off = save; return GBHE_EWORKSPACE; }
  const size_t total = (size_t)n * m;
  k_promote<<<(int)std::min<size_t>((total + 255) / 256, 4096), 256, 0, c.st>>>(Z, ldz, n, m, X, ldx);
  count_launch();
  GBHE_CUDA(cudaGetLastError());
  // ---- Q2
  if (n >= 2) {
    const int J = hb2st_J(n, nb);
    const size_t smem = (size_t)(2 * nb * SLAB + 2 * nb) * sizeof(cplx);
    if (smem > 48 * 1024)
      GBHE_CUDA(cudaFuncSetAttribute(k_apply_q2, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    double fl = 0.0;
    if (prof_on())
      for (int s = 0; s <= n - 2; ++s)
        for (int a0 = s + 1; a0 < n; a0 += nb) fl += 16.0 * std::min(nb, n - a0) * (double)m;
    ProfScope prof(c.st, GBHE_PROF_Q2, fl, 16.0 * ((double)n * J * nb + 2.0 * (double)n * m));
    k_apply_q2<<<(m + SLAB - 1) / SLAB, QT, smem, c.st>>>(n, nb, m, J, V2, tau2, X, ldx);
    count_launch();
    GBHE_CUDA(cudaGetLastError());
  }
  // ---- Q1
  int npan = 0;
  for (int k = 0; k + nb < n; k += nb) ++npan;
  const cplx one = mk(1, 0), zero = mk(0, 0), mone = mk(-1, 0);
  for (int p = npan - 1; p >= 0; --p) {
    const int k = p * nb, mp = n - k - nb, kr = std::min(nb, mp);
    k_panel_v<<<(int)std::min<size_t>(((size_t)mp * nb + 255) / 256, 4096), 256, 0, c.st>>>(A, lda, k, nb, mp, kr, V, n);
    count_launch();
    GBHE_CUDA(cudaGetLastError());
    cplx* Xr = X + (k + nb);
    const cplx* T = T1 + (size_t)p * nb * nb;
    int rc;
    if ((rc = zgemm(c, gemm_args(OP_C, OP_N, kr, m, mp, one, V, n, Xr, ldx, zero, W1, nb), c.gemm_scratch,
                    c.gemm_scratch_bytes))) { ar.off = save; return rc; }
    if ((rc = zgemm(c, gemm_args(OP_N, OP_N, kr, m, kr, one, T, nb, W1, nb, zero, W2, nb), nullptr, 0))) {
      ar.off = save; return rc;
    }
    if ((rc = zgemm(c, gemm_args(OP_N, OP_N, mp, m, kr, mone, V, n, W2, nb, one, Xr, ldx), nullptr, 0))) {
      ar.off = save; return rc;
    }
  }
  ar.off = save;
  return 0;
}

}  // namespace gbhe
