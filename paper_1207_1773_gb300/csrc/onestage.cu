// onestage.cu -- one-stage comparator (paper Section 4.1): the LAPACK-style
// blocked Householder tridiagonalisation, where half of the flops are
// Hermitian matrix-vector products (level 2), followed by the same divide and
// conquer and a single blocked back-transformation.
//
// Panel of NBT columns starting at k; for column i = k + j:
//   a_i  -= V(:,0:j) conj(W(i,0:j))^T + W(:,0:j) conj(V(i,0:j))^T  (delayed update)
//   H_i from a_i(i+1:n);  v stored in A below the sub-diagonal and in V(:,j)
//   y = A22 v              (A22 = A(i+1:n, i+1:n), not yet updated by this panel)
//   y = tau (y - V (W^H v) - W (V^H v));  w = y - tau/2 (y^H v) v  -> W(:,j)
// after the panel:  A(k+NBT:, k+NBT:) -= V W^H + W V^H   (DMMA GEMMs).
#include <algorithm>
#include <cmath>
#include "internal.cuh"

namespace gbhe {
namespace {

constexpr int NBT = 32;
constexpr int HT = 32;  // hemv tile

__device__ __forceinline__ cplx warp_sum(cplx v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    v.x += __shfl_xor_sync(0xffffffffu, v.x, o);
    v.y += __shfl_xor_sync(0xffffffffu, v.y, o);
  }
  return v;
}

// Block-wide sum (blockDim.x multiple of 32, <= 1024).
__device__ cplx block_sum(cplx v) {
  __shared__ cplx red[32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  v = warp_sum(v);
  __syncthreads();
  if (lane == 0) red[warp] = v;
  __syncthreads();
  cplx s = mk(0.0, 0.0);
  if (warp == 0) {
    s = (lane < (int)(blockDim.x >> 5)) ? red[lane] : mk(0.0, 0.0);
    s = warp_sum(s);
  }
  __syncthreads();
  if (threadIdx.x == 0) red[0] = s;
  __syncthreads();
  return red[0];
}

// column update of a_i with the panel's earlier reflectors
__global__ void k_col_update(cplx* A, int lda, int n, int i, int j, const cplx* V, const cplx* W) {
  const int r = i + blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= n) return;
  cplx acc = A[(size_t)r + (size_t)i * lda];
  for (int q = 0; q < j; ++q) {
    const cplx vr = V[(size_t)r + (size_t)q * n], wr = W[(size_t)r + (size_t)q * n];
    const cplx vi = V[(size_t)i + (size_t)q * n], wi = W[(size_t)i + (size_t)q * n];
    acc = csub(acc, cadd(cmulc(vr, wi), cmulc(wr, vi)));
  }
  if (r == i) acc.y = 0.0;
  A[(size_t)r + (size_t)i * lda] = acc;
}

// reflector of column i (one CTA): V(:,j), A below the sub-diagonal, d, e, tau
__global__ void __launch_bounds__(1024) k_col_reflector(cplx* A, int lda, int n, int i, int j, cplx* V,
                                                        cplx* W, double* d, double* e, cplx* tau) {
  const int t = threadIdx.x;
  double s = 0.0;
  for (int r = i + 2 + t; r < n; r += blockDim.x) s += cabs2(A[(size_t)r + (size_t)i * lda]);
  const double xn2 = block_sum(mk(s, 0.0)).x;
  __shared__ cplx sh_tau, sh_scal;
  __shared__ double sh_beta;
  if (t == 0) {
    const cplx al = A[(size_t)(i + 1) + (size_t)i * lda];
    if (xn2 == 0.0 && al.y == 0.0) {
      sh_tau = mk(0.0, 0.0); sh_beta = al.x; sh_scal = mk(0.0, 0.0);
    } else {
      const double nrm = sqrt(al.x * al.x + al.y * al.y + xn2);
      const double beta = (al.x >= 0.0) ? -nrm : nrm;
      sh_beta = beta;
      sh_tau = mk((beta - al.x) / beta, -al.y / beta);
      sh_scal = cinv(mk(al.x - beta, al.y));
    }
    d[i] = A[(size_t)i + (size_t)i * lda].x;
    e[i] = sh_beta;
    tau[i] = sh_tau;
    A[(size_t)(i + 1) + (size_t)i * lda] = mk(sh_beta, 0.0);
  }
  __syncthreads();
  const cplx sc = sh_scal;
  for (int r = t; r < n; r += blockDim.x) {
    cplx v = mk(0.0, 0.0);
    if (r == i + 1) {
      v = mk(1.0, 0.0);
    } else if (r > i + 1) {
      v = cmul(A[(size_t)r + (size_t)i * lda], sc);
      A[(size_t)r + (size_t)i * lda] = v;
    }
    V[(size_t)r + (size_t)j * n] = v;
    if (r <= i) W[(size_t)r + (size_t)j * n] = mk(0.0, 0.0);
  }
}

// y += A22 v with A22 Hermitian, lower-stored, order L; 32 x 32 tiles of the
// lower triangle, each contributing A_t v and (off-diagonal) A_t^H v.
__global__ void __launch_bounds__(128) k_hemv(const cplx* A22, int lda, int L, const cplx* v, cplx* y) {
  __shared__ cplx T[HT][HT + 1];
  __shared__ cplx vr[HT], vc[HT];
  __shared__ cplx part[4][HT];
  const long t = blockIdx.x;
  int bi = (int)((sqrt(8.0 * (double)t + 1.0) - 1.0) * 0.5);
  while ((long)bi * (bi + 1) / 2 > t) --bi;
  while ((long)(bi + 1) * (bi + 2) / 2 <= t) ++bi;
  const int bj = (int)(t - (long)bi * (bi + 1) / 2);
  const int r0 = bi * HT, c0 = bj * HT;
  const int tid = threadIdx.x;
  for (int q = tid; q < HT * HT; q += blockDim.x) {
    const int r = q % HT, c = q / HT, gr = r0 + r, gc = c0 + c;
    cplx a = mk(0.0, 0.0);
    if (gr < L && gc < L && gr >= gc) a = A22[(size_t)gr + (size_t)gc * lda];
    if (gr == gc) a.y = 0.0;
    T[r][c] = a;
  }
  if (tid < HT) {
    vr[tid] = (r0 + tid < L) ? v[r0 + tid] : mk(0.0, 0.0);
    vc[tid] = (c0 + tid < L) ? v[c0 + tid] : mk(0.0, 0.0);
  }
  __syncthreads();
  // rows: y[r0+r] += sum_c T[r][c] vc[c]     (threads: r = tid % 32, quarter = tid / 32)
  const int r = tid & 31, qt = tid >> 5;
  cplx acc = mk(0.0, 0.0);
  for (int c = qt * 8; c < qt * 8 + 8; ++c) cfma(acc, T[r][c], vc[c]);
  part[qt][r] = acc;
  __syncthreads();
  if (tid < HT && r0 + tid < L) {
    cplx s = cadd(cadd(part[0][tid], part[1][tid]), cadd(part[2][tid], part[3][tid]));
    atomicAdd(&y[r0 + tid].x, s.x);
    atomicAdd(&y[r0 + tid].y, s.y);
  }
  __syncthreads();
  // columns (the mirrored upper triangle): y[c0+c] += sum_r conj(T[r][c]) vr[r],
  // over the strictly lower elements only in a diagonal tile
  const int c = tid & 31;
  acc = mk(0.0, 0.0);
  for (int rr = qt * 8; rr < qt * 8 + 8; ++rr)
    if (bi != bj || rr > c) ccfma(acc, T[rr][c], vr[rr]);
  part[qt][c] = acc;
  __syncthreads();
  if (tid < HT && c0 + tid < L) {
    cplx s = cadd(cadd(part[0][tid], part[1][tid]), cadd(part[2][tid], part[3][tid]));
    atomicAdd(&y[c0 + tid].x, s.x);
    atomicAdd(&y[c0 + tid].y, s.y);
  }
}

// u[q] = W(:,q)^H v (q < j) and u[j+q] = V(:,q)^H v over rows i+1..n-1; one CTA per dot.
__global__ void __launch_bounds__(256) k_corr_dots(int n, int i, int j, const cplx* V, const cplx* W, cplx* u) {
  const int q = blockIdx.x % j;
  const cplx* M = (blockIdx.x < j) ? W : V;
  const cplx* v = V + (size_t)j * n;
  cplx acc = mk(0.0, 0.0);
  for (int r = i + 1 + threadIdx.x; r < n; r += blockDim.x) ccfma(acc, M[(size_t)r + (size_t)q * n], v[r]);
  acc = block_sum(acc);
  if (threadIdx.x == 0) u[blockIdx.x] = acc;
}

// y := tau (y - V u2 - W u1) for rows i+1..n-1, stored in W(:,j); partial y^H v in sum.
__global__ void k_finish_y(int n, int i, int j, const cplx* V, cplx* W, const cplx* y, const cplx* u,
                           const cplx* tau, cplx* sum) {
  const int r = i + 1 + blockIdx.x * blockDim.x + threadIdx.x;
  cplx val = mk(0.0, 0.0);
  if (r < n) {
    cplx acc = y[r - i - 1];
    for (int q = 0; q < j; ++q) {
      acc = csub(acc, cmul(V[(size_t)r + (size_t)q * n], u[q]));      // V (W^H v)
      acc = csub(acc, cmul(W[(size_t)r + (size_t)q * n], u[j + q]));  // W (V^H v)
    }
    acc = cmul(tau[i], acc);
    W[(size_t)r + (size_t)j * n] = acc;
    val = cmulc(V[(size_t)r + (size_t)j * n], acc);  // v_r conj(y_r): summed, y^H v
  }
  val = block_sum(val);
  if (threadIdx.x == 0) {
    atomicAdd(&sum->x, val.x);
    atomicAdd(&sum->y, val.y);
  }
}

__global__ void k_finish_w(int n, int i, int j, const cplx* V, cplx* W, const cplx* tau, const cplx* sum) {
  const int r = i + 1 + blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= n) return;
  const cplx al = cscal(-0.5, cmul(tau[i], *sum));
  W[(size_t)r + (size_t)j * n] = cadd(W[(size_t)r + (size_t)j * n], cmul(al, V[(size_t)r + (size_t)j * n]));
}

__global__ void k_last_diag(const cplx* A, int lda, int n, double* d) { d[n - 1] = A[(size_t)(n - 1) * (lda + 1)].x; }

// T (jn x jn, ld NBT) from G = V^H V and tau: T(j,j) = tau_j,
// T(0:j, j) = -tau_j T(0:j, 0:j) G(0:j, j).
__global__ void k_larft(const cplx* G, int ldg, const cplx* tau, int jn, cplx* T) {
  for (int q = threadIdx.x; q < NBT * NBT; q += blockDim.x) T[q] = mk(0.0, 0.0);
  __syncthreads();
  for (int j = 0; j < jn; ++j) {
    const cplx tj = tau[j];
    for (int r = threadIdx.x; r < j; r += blockDim.x) {
      cplx acc = mk(0.0, 0.0);
      for (int q = r; q < j; ++q) cfma(acc, T[r + q * NBT], G[q + (size_t)j * ldg]);
      T[r + j * NBT] = cscal(-1.0, cmul(tj, acc));
    }
    if (threadIdx.x == 0) T[j + j * NBT] = tj;
    __syncthreads();
  }
}

// explicit V of one-stage panel (reflectors k..k+jn-1; rows k+1..n-1)
__global__ void k_os_panel_v(const cplx* A, int lda, int n, int k, int jn, cplx* V, int ldv) {
  const int mp = n - k - 1;
  const size_t total = (size_t)mp * jn;
  for (size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x; q < total; q += (size_t)gridDim.x * blockDim.x) {
    const int r = (int)(q % mp), c = (int)(q / mp);
    cplx e = mk(0.0, 0.0);
    if (r == c) e = mk(1.0, 0.0);
    else if (r > c) e = A[(size_t)(k + 1 + r) + (size_t)(k + c) * lda];
    V[(size_t)r + (size_t)c * ldv] = e;
  }
}

}  // namespace

size_t onestage_ws_bytes(int n, int m) {
  const size_t nn = (size_t)std::max(n, 1), mm = (size_t)std::max(m, 1);
  size_t b = 0;
  b += 2 * nn * NBT * sizeof(cplx) + 512;        // V, W
  b += nn * sizeof(cplx) * 2 + 512;              // y, tau
  b += 2 * nn * sizeof(double) + 512;            // d, e
  b += (2 * NBT + 8) * sizeof(cplx) + 512;       // u, sum
  b += nn * mm * sizeof(double) + 256;           // Z
  b += 2 * (size_t)NBT * mm * sizeof(cplx) + 512; // W1, W2 (back-transform)
  b += 2 * NBT * NBT * sizeof(cplx) + 512;       // G, T
  b += stedc_ws_bytes(n);
  return b;
}

static int hetrd_onestage(Ctx& c, int n, cplx* A, int lda, cplx* V, cplx* W, cplx* y, cplx* u, cplx* sum,
                          double* d, double* e, cplx* tau) {
  const cplx one = mk(1, 0), mone = mk(-1, 0);
  for (int k = 0; k < n - 1; k += NBT) {
    const int jn = std::min(NBT, n - 1 - k);
    for (int j = 0; j < jn; ++j) {
      const int i = k + j;
      const int rows = n - i;
      k_col_update<<<(rows + 255) / 256, 256, 0, c.st>>>(A, lda, n, i, j, V, W);
      count_launch();
      k_col_reflector<<<1, 1024, 0, c.st>>>(A, lda, n, i, j, V, W, d, e, tau);
      count_launch();
      const int L = n - i - 1;
      GBHE_CUDA(cudaMemsetAsync(y, 0, sizeof(cplx) * L, c.st));
      {
        const long nt = (L + HT - 1) / HT;
        ProfScope prof(c.st, GBHE_PROF_HEMV, 8.0 * (double)L * L, 16.0 * (double)L * L / 2);
        k_hemv<<<(unsigned)(nt * (nt + 1) / 2), 128, 0, c.st>>>(A + (size_t)(i + 1) + (size_t)(i + 1) * lda, lda, L,
                                                                V + (size_t)(i + 1) + (size_t)j * n, y);
        count_launch();
      }
      GBHE_CUDA(cudaMemsetAsync(sum, 0, sizeof(cplx), c.st));
      if (j > 0) {
        k_corr_dots<<<2 * j, 256, 0, c.st>>>(n, i, j, V, W, u);
        count_launch();
      }
      k_finish_y<<<(L + 255) / 256, 256, 0, c.st>>>(n, i, j, V, W, y, u, tau, sum);
      count_launch();
      k_finish_w<<<(L + 255) / 256, 256, 0, c.st>>>(n, i, j, V, W, tau, sum);
      count_launch();
      GBHE_CUDA(cudaGetLastError());
    }
    const int k2 = k + jn;
    if (k2 < n) {
      cplx* A22 = A + (size_t)k2 + (size_t)k2 * lda;
      const int m2 = n - k2;
      int rc;
      if ((rc = zgemm(c, gemm_args(OP_N, OP_C, m2, m2, jn, mone, V + k2, n, W + k2, n, one, A22, lda, 1),
                      nullptr, 0))) return rc;
      if ((rc = zgemm(c, gemm_args(OP_N, OP_C, m2, m2, jn, mone, W + k2, n, V + k2, n, one, A22, lda, 1),
                      nullptr, 0))) return rc;
    }
  }
  k_last_diag<<<1, 1, 0, c.st>>>(A, lda, n, d);
  count_launch();
  GBHE_CUDA(cudaGetLastError());
  return 0;
}

// X := Q X, Q = H_0 ... H_{n-2} (reflectors of hetrd_onestage), blocked by NBT.
static int unmtr_onestage(Ctx& c, int n, int m, const cplx* A, int lda, const cplx* tau, cplx* X, int ldx,
                          cplx* V, cplx* G, cplx* T, cplx* W1, cplx* W2) {
  const cplx one = mk(1, 0), zero = mk(0, 0), mone = mk(-1, 0);
  int npan = 0;
  for (int k = 0; k < n - 1; k += NBT) ++npan;
  for (int p = npan - 1; p >= 0; --p) {
    const int k = p * NBT, jn = std::min(NBT, n - 1 - k), mp = n - k - 1;
    k_os_panel_v<<<(int)std::min<size_t>(((size_t)mp * jn + 255) / 256, 4096), 256, 0, c.st>>>(A, lda, n, k, jn, V, n);
    count_launch();
    int rc;
    if ((rc = zgemm(c, gemm_args(OP_C, OP_N, jn, jn, mp, one, V, n, V, n, zero, G, NBT), c.gemm_scratch,
                    c.gemm_scratch_bytes))) return rc;
    k_larft<<<1, 128, 0, c.st>>>(G, NBT, tau + k, jn, T);
    count_launch();
    cplx* Xr = X + (k + 1);
    if ((rc = zgemm(c, gemm_args(OP_C, OP_N, jn, m, mp, one, V, n, Xr, ldx, zero, W1, NBT), c.gemm_scratch,
                    c.gemm_scratch_bytes))) return rc;
    if ((rc = zgemm(c, gemm_args(OP_N, OP_N, jn, m, jn, one, T, NBT, W1, NBT, zero, W2, NBT), nullptr, 0)))
      return rc;
    if ((rc = zgemm(c, gemm_args(OP_N, OP_N, mp, m, jn, mone, V, n, W2, NBT, one, Xr, ldx), nullptr, 0)))
      return rc;
  }
  return 0;
}

__global__ void k_promote_os(const double* Z, int ldz, int n, int m, cplx* X, int ldx) {
  const size_t total = (size_t)n * m;
  for (size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x; q < total; q += (size_t)gridDim.x * blockDim.x) {
    const int r = (int)(q % n), cc = (int)(q / n);
    X[(size_t)r + (size_t)cc * ldx] = mk(Z[(size_t)r + (size_t)cc * ldz], 0.0);
  }
}

int hegv_onestage_run(Ctx& c, int n, cplx* A, int lda, cplx* B, int ldb, int il, int iu, double* w,
                      cplx* X, int ldx) {
  const int m = iu - il + 1;
  Arena& ar = c.arena;
  const size_t save = ar.off;
  cplx* V = ar.take<cplx>((size_t)n * NBT);
  cplx* W = ar.take<cplx>((size_t)n * NBT);
  cplx* y = ar.take<cplx>((size_t)n);
  cplx* tau = ar.take<cplx>((size_t)n);
  double* d = ar.take<double>((size_t)n);
  double* e = ar.take<double>((size_t)n);
  cplx* u = ar.take<cplx>(2 * NBT + 4);
  cplx* sum = ar.take<cplx>(4);
  double* Z = ar.take<double>((size_t)n * m);
  cplx* W1 = ar.take<cplx>((size_t)NBT * m);
  cplx* W2 = ar.take<cplx>((size_t)NBT * m);
  cplx* G = ar.take<cplx>(NBT * NBT);
  cplx* T = ar.take<cplx>(NBT * NBT);
  if (!ar.ok() || !T) { ar.off = save; return GBHE_EWORKSPACE; }
  int rc;
  if ((rc = potrf_run(c, n, B, ldb))) { ar.off = save; return rc; }
  if ((rc = hegst_run(c, n, A, lda, B, ldb))) { ar.off = save; return rc; }
  GBHE_CUDA(cudaMemsetAsync(tau, 0, sizeof(cplx) * n, c.st));
  if (n >= 2) {
    if ((rc = hetrd_onestage(c, n, A, lda, V, W, y, u, sum, d, e, tau))) { ar.off = save; return rc; }
  } else {
    k_last_diag<<<1, 1, 0, c.st>>>(A, lda, n, d);
    count_launch();
  }
  if ((rc = stedc_run(c, n, d, e, il, iu, w, Z, n))) { ar.off = save; return rc; }
  k_promote_os<<<(int)std::min<size_t>(((size_t)n * m + 255) / 256, 4096), 256, 0, c.st>>>(Z, n, n, m, X, ldx);
  count_launch();
  if (n >= 2)
    if ((rc = unmtr_onestage(c, n, m, A, lda, tau, X, ldx, V, G, T, W1, W2))) { ar.off = save; return rc; }
  rc = trsm_run(c, 1, n, m, B, ldb, X, ldx);
  ar.off = save;
  return rc;
}

}  // namespace gbhe
