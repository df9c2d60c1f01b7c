// dense.cu -- Algorithm 1 steps 1, 2 and 4 of the paper (Section 3):
//   potrf  B = L L^H                (blocked right-looking Cholesky)
//   hegst  A' = L^{-1} A L^{-H}     (blocked two-sided reduction: per block
//                                    column a rank-2 trailing update and a
//                                    thin forward solve, about 4 n^3 flops)
//   trsm   X = L^{-1} X  or  X = L^{-H} X
// The diagonal blocks (DB x DB) are factored / inverted by one CTA each in
// shared memory; everything else is DMMA GEMM (gemm.cu).
#include <algorithm>
#include "internal.cuh"

namespace gbhe {
namespace {

constexpr int DB = 64;      // diagonal block order
constexpr int DT = 256;     // threads of the diagonal-block kernels

// Factor the diagonal block A[k0:k0+bs, k0:k0+bs] (lower) in place and write
// the inverse of its Cholesky factor to Linv (bs x bs, ld DB).
__global__ void __launch_bounds__(DT) k_potrf_diag(cplx* A, int lda, int k0, int bs, cplx* Linv,
                                                   int* st, int info_off) {
  extern __shared__ cplx sm[];
  cplx* L = sm;              // DB x DB, ld DB
  cplx* X = sm + DB * DB;    // inverse
  const int t = threadIdx.x;
  for (int i = t; i < bs * bs; i += DT) {
    int r = i % bs, c = i / bs;
    L[r + c * DB] = (r >= c) ? A[(size_t)(k0 + r) + (size_t)(k0 + c) * lda] : mk(0.0, 0.0);
  }
  __syncthreads();
  __shared__ double piv;
  __shared__ int bad;
  if (t == 0) bad = 0;
  for (int j = 0; j < bs; ++j) {
    if (t == 0) {
      double d = L[j + j * DB].x;
      if (!(d > 0.0) || !isfinite(d)) {
        if (!bad) set_info_once(st, info_off + k0 + j + 1);
        bad = 1;
        d = 1.0;  // keep going on a harmless value; the status word carries the failure
      }
      piv = sqrt(d);
      L[j + j * DB] = mk(piv, 0.0);
    }
    __syncthreads();
    const double inv = 1.0 / piv;
    for (int r = j + 1 + t; r < bs; r += DT) L[r + j * DB] = cscal(inv, L[r + j * DB]);
    __syncthreads();
    // trailing lower update: L[r, c] -= L[r, j] conj(L[c, j]),  j < c <= r
    const int rem = bs - j - 1;
    for (int i = t; i < rem * rem; i += DT) {
      int r = j + 1 + i % rem, c = j + 1 + i / rem;
      if (r >= c) {
        cplx a = L[r + c * DB];
        cplx p = cmulc(L[r + j * DB], L[c + j * DB]);
        L[r + c * DB] = csub(a, p);
      }
    }
    __syncthreads();
  }
  // inverse of the lower-triangular L: column c solved by thread c
  if (t < bs) {
    const int c = t;
    for (int r = 0; r < bs; ++r) {
      if (r < c) { X[r + c * DB] = mk(0.0, 0.0); continue; }
      cplx s = mk(r == c ? 1.0 : 0.0, 0.0);
      for (int q = c; q < r; ++q) s = csub(s, cmul(L[r + q * DB], X[q + c * DB]));
      X[r + c * DB] = cdiv(s, L[r + r * DB]);
    }
  }
  __syncthreads();
  for (int i = t; i < bs * bs; i += DT) {
    int r = i % bs, c = i / bs;
    if (r >= c) A[(size_t)(k0 + r) + (size_t)(k0 + c) * lda] = L[r + c * DB];
    Linv[r + c * DB] = X[r + c * DB];
  }
}

// Inverse of every diagonal block of the lower-triangular L (block b of order
// bs_b = min(DB, n - b*DB)) into Linv + b*DB*DB (ld DB).  One CTA per block.
__global__ void __launch_bounds__(DT) k_trtri_diag(const cplx* Lg, int ldl, int n, cplx* Linv) {
  extern __shared__ cplx sm[];
  cplx* L = sm;
  cplx* X = sm + DB * DB;
  const int b = blockIdx.x, k0 = b * DB, bs = min(DB, n - k0), t = threadIdx.x;
  for (int i = t; i < bs * bs; i += DT) {
    int r = i % bs, c = i / bs;
    L[r + c * DB] = (r >= c) ? Lg[(size_t)(k0 + r) + (size_t)(k0 + c) * ldl] : mk(0.0, 0.0);
  }
  __syncthreads();
  if (t < bs) {
    const int c = t;
    for (int r = 0; r < bs; ++r) {
      if (r < c) { X[r + c * DB] = mk(0.0, 0.0); continue; }
      cplx s = mk(r == c ? 1.0 : 0.0, 0.0);
      for (int q = c; q < r; ++q) s = csub(s, cmul(L[r + q * DB], X[q + c * DB]));
      X[r + c * DB] = cdiv(s, L[r + r * DB]);
    }
  }
  __syncthreads();
  cplx* out = Linv + (size_t)b * DB * DB;
  for (int i = t; i < DB * DB; i += DT) {
    int r = i % DB, c = i / DB;
    out[i] = (r < bs && c < bs) ? X[r + c * DB] : mk(0.0, 0.0);
  }
}

// Mirror the lower triangle into the upper one (A Hermitian, real diagonal).
__global__ void k_fill_upper(cplx* A, int lda, int n) {
  const size_t total = (size_t)n * n;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total;
       i += (size_t)gridDim.x * blockDim.x) {
    int r = (int)(i % n), c = (int)(i / n);
    if (r < c) A[(size_t)r + (size_t)c * lda] = cconj(A[(size_t)c + (size_t)r * lda]);
    else if (r == c) A[(size_t)r + (size_t)c * lda].y = 0.0;
  }
}

int diag_smem() { return 2 * DB * DB * (int)sizeof(cplx); }

int ensure_attrs() {
  static bool done[MAX_DEVICES] = {};
  const int dev = device_slot();
  if (dev < 0) return GBHE_ECUDA;
  if (done[dev]) return 0;
  GBHE_CUDA(cudaFuncSetAttribute(k_potrf_diag, cudaFuncAttributeMaxDynamicSharedMemorySize, diag_smem()));
  GBHE_CUDA(cudaFuncSetAttribute(k_trtri_diag, cudaFuncAttributeMaxDynamicSharedMemorySize, diag_smem()));
  done[dev] = true;
  return 0;
}

inline int grid1d(size_t total, int threads = 256) {
  return (int)std::min<size_t>((total + threads - 1) / threads, 152 * 16);
}

}  // namespace

// Outer blocking: the level-3 updates use TB = 256 columns (the tensor-core
// GEMM is several times faster at K = 256 than at K = 64); the TB x TB
// diagonal blocks are factored / inverted with the 64-wide kernels above.
constexpr int TB = 256;

// Layout of the dense scratch: 64-block inverses | TB-block inverses | temp
// (n x TB) | the hegst panel buffer [A21 L21 A21] (n x 3 TB).
size_t inv64_elems(int n) { return (size_t)((n + DB - 1) / DB) * DB * DB; }
size_t invtb_elems(int n) { return (size_t)((n + TB - 1) / TB) * TB * TB; }

size_t dense_ws_bytes(int n) {
  const size_t nn = (size_t)std::max(n, 1);
  return (inv64_elems(n) + invtb_elems(n) + nn * TB + nn * 3 * TB) * sizeof(cplx) + 4 * 256;
}

namespace {

cplx* inv64_buf(Ctx& c) { return c.dense_scratch; }
cplx* invtb_buf(Ctx& c, int n) { return c.dense_scratch + inv64_elems(n); }
cplx* temp_buf(Ctx& c, int n) { return c.dense_scratch + inv64_elems(n) + invtb_elems(n); }
cplx* panel3_buf(Ctx& c, int n) {
  return c.dense_scratch + inv64_elems(n) + invtb_elems(n) + (size_t)std::max(n, 1) * TB;
}

__global__ void k_set_identity(cplx* X, int ldx, int bs) {
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < bs * bs; q += gridDim.x * blockDim.x) {
    const int r = q % bs, cc = q / bs;
    X[(size_t)r + (size_t)cc * ldx] = mk(r == cc ? 1.0 : 0.0, 0.0);
  }
}

__global__ void k_copy_block(const cplx* S, int lds, cplx* D, int ldd, int rows, int cols) {
  const size_t total = (size_t)rows * cols;
  for (size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x; q < total; q += (size_t)gridDim.x * blockDim.x) {
    const int r = (int)(q % rows), cc = (int)(q / rows);
    D[(size_t)r + (size_t)cc * ldd] = S[(size_t)r + (size_t)cc * lds];
  }
}

// 64-blocked Cholesky of the n x n block B (info reported at offset info_off).
int potrf64(Ctx& c, int n, cplx* B, int ldb, int info_off) {
  cplx* Linv = inv64_buf(c);
  for (int k0 = 0; k0 < n; k0 += DB) {
    const int bs = std::min(DB, n - k0);
    k_potrf_diag<<<1, DT, diag_smem(), c.st>>>(B, ldb, k0, bs, Linv, c.status, info_off);
    count_launch();
    GBHE_CUDA(cudaGetLastError());
    const int rest = n - k0 - bs;
    if (rest <= 0) break;
    cplx* A21 = B + (size_t)(k0 + bs) + (size_t)k0 * ldb;
    // L21 = A21 * Linv^H   (in place: N = 64 is one column tile of every engine)
    int rc = zgemm(c, gemm_args(OP_N, OP_C, rest, bs, bs, mk(1, 0), A21, ldb, Linv, DB, mk(0, 0), A21, ldb), nullptr, 0);
    if (rc) return rc;
    cplx* A22 = B + (size_t)(k0 + bs) + (size_t)(k0 + bs) * ldb;
    rc = zgemm(c, gemm_args(OP_N, OP_C, rest, rest, bs, mk(-1, 0), A21, ldb, A21, ldb, mk(1, 0), A22, ldb, 1),
               nullptr, 0);
    if (rc) return rc;
  }
  return 0;
}

// Inverse of the lower-triangular bs x bs block L (bs <= TB) into Linv (ld TB),
// by the 64-blocked forward solve L X = I.
int trtri_block(Ctx& c, int bs, const cplx* L, int ldl, cplx* Linv) {
  k_set_identity<<<64, 256, 0, c.st>>>(Linv, TB, bs);
  count_launch();
  const int nb64 = (bs + DB - 1) / DB;
  cplx* I64 = inv64_buf(c);
  k_trtri_diag<<<nb64, DT, diag_smem(), c.st>>>(L, ldl, bs, I64);
  count_launch();
  GBHE_CUDA(cudaGetLastError());
  for (int b = 0; b < nb64; ++b) {
    const int k0 = b * DB, b64 = std::min(DB, bs - k0);
    cplx* Xb = Linv + k0;
    // rows k0.. of X: X_b = inv64 * X_b (M = 64 <= one row tile: in place is safe)
    int rc = zgemm(c, gemm_args(OP_N, OP_N, b64, bs, b64, mk(1, 0), I64 + (size_t)b * DB * DB, DB, Xb, TB, mk(0, 0),
                                Xb, TB), nullptr, 0);
    if (rc) return rc;
    const int rest = bs - k0 - b64;
    if (rest > 0) {
      rc = zgemm(c, gemm_args(OP_N, OP_N, rest, bs, b64, mk(-1, 0), L + (size_t)(k0 + b64) + (size_t)k0 * ldl, ldl, Xb,
                              TB, mk(1, 0), Linv + k0 + b64, TB), nullptr, 0);
      if (rc) return rc;
    }
  }
  return 0;
}

}  // namespace

int potrf_run(Ctx& c, int n, cplx* B, int ldb) {
  if (n <= 0) return 0;
  int rc = ensure_attrs();
  if (rc) return rc;
  cplx* Linv = invtb_buf(c, n);
  cplx* T = temp_buf(c, n);
  for (int k0 = 0; k0 < n; k0 += TB) {
    const int bs = std::min(TB, n - k0);
    cplx* Bkk = B + (size_t)k0 + (size_t)k0 * ldb;
    if ((rc = potrf64(c, bs, Bkk, ldb, k0))) return rc;
    const int rest = n - k0 - bs;
    if (rest <= 0) break;
    if ((rc = trtri_block(c, bs, Bkk, ldb, Linv))) return rc;
    cplx* A21 = B + (size_t)(k0 + bs) + (size_t)k0 * ldb;
    // L21 = A21 Linv^H  (through a temporary: N = TB spans several column tiles)
    if ((rc = zgemm(c, gemm_args(OP_N, OP_C, rest, bs, bs, mk(1, 0), A21, ldb, Linv, TB, mk(0, 0), T, rest), nullptr,
                    0)))
      return rc;
    k_copy_block<<<1024, 256, 0, c.st>>>(T, rest, A21, ldb, rest, bs);
    count_launch();
    // A22 -= L21 L21^H (lower)
    cplx* A22 = B + (size_t)(k0 + bs) + (size_t)(k0 + bs) * ldb;
    if ((rc = zgemm(c, gemm_args(OP_N, OP_C, rest, rest, bs, mk(-1, 0), A21, ldb, A21, ldb, mk(1, 0), A22, ldb, 1),
                    nullptr, 0)))
      return rc;
  }
  return 0;
}

// X (n x m) := L^{-1} X (trans = 0) or L^{-H} X (trans = 1), TB-blocked.
int trsm_run(Ctx& c, int trans, int n, int m, const cplx* L, int ldl, cplx* X, int ldx) {
  if (n <= 0 || m <= 0) return 0;
  int rc = ensure_attrs();
  if (rc) return rc;
  const int nblk = (n + TB - 1) / TB;
  cplx* Linv = invtb_buf(c, n);
  for (int b = 0; b < nblk; ++b) {
    const int k0 = b * TB, bs = std::min(TB, n - k0);
    if ((rc = trtri_block(c, bs, L + (size_t)k0 + (size_t)k0 * ldl, ldl, Linv + (size_t)b * TB * TB))) return rc;
  }
  cplx* T = temp_buf(c, n);
  // the temporary holds TB x mc; process the columns in chunks of mc
  const int mc = std::max(1, std::min(m, (int)(((size_t)std::max(n, 1) * TB) / TB)));
  for (int c0 = 0; c0 < m; c0 += mc) {
    const int mm = std::min(mc, m - c0);
    cplx* Xc = X + (size_t)c0 * ldx;
    if (trans == 0) {
      for (int b = 0; b < nblk; ++b) {
        const int k0 = b * TB, bs = std::min(TB, n - k0);
        cplx* Xb = Xc + k0;
        if ((rc = zgemm(c, gemm_args(OP_N, OP_N, bs, mm, bs, mk(1, 0), Linv + (size_t)b * TB * TB, TB, Xb, ldx,
                                     mk(0, 0), T, TB), nullptr, 0)))
          return rc;
        k_copy_block<<<1024, 256, 0, c.st>>>(T, TB, Xb, ldx, bs, mm);
        count_launch();
        const int rest = n - k0 - bs;
        if (rest > 0)
          if ((rc = zgemm(c, gemm_args(OP_N, OP_N, rest, mm, bs, mk(-1, 0), L + (size_t)(k0 + bs) + (size_t)k0 * ldl,
                                       ldl, Xb, ldx, mk(1, 0), Xb + bs, ldx), nullptr, 0)))
            return rc;
      }
    } else {
      for (int b = nblk - 1; b >= 0; --b) {
        const int k0 = b * TB, bs = std::min(TB, n - k0);
        cplx* Xb = Xc + k0;
        if ((rc = zgemm(c, gemm_args(OP_C, OP_N, bs, mm, bs, mk(1, 0), Linv + (size_t)b * TB * TB, TB, Xb, ldx,
                                     mk(0, 0), T, TB), nullptr, 0)))
          return rc;
        k_copy_block<<<1024, 256, 0, c.st>>>(T, TB, Xb, ldx, bs, mm);
        count_launch();
        if (k0 > 0)
          if ((rc = zgemm(c, gemm_args(OP_C, OP_N, k0, mm, bs, mk(-1, 0), L + k0, ldl, Xb, ldx, mk(1, 0), Xc, ldx),
                          nullptr, 0)))
            return rc;
      }
    }
  }
  return 0;
}

// Blocked two-sided reduction A' = L^{-1} A L^{-H} (lower storage), block
// column b of order bs at k0 (the standard right-looking scheme):
//   A11 <- L11^{-1} A11 L11^{-H}
//   A21 <- A21 L11^{-H};  A21 -= 1/2 L21 A11
//   A22 -= A21 L21^H + L21 A21^H          (lower; one product [A21 L21][L21 A21]^H)
//   A21 -= 1/2 L21 A11;   A21 <- L22^{-1} A21
// with every TB x TB diagonal block of L inverted once up front.  The upper
// triangle of A is never read; on return it holds the mirror of the lower.
int hegst_run(Ctx& c, int n, cplx* A, int lda, const cplx* L, int ldl) {
  if (n <= 0) return 0;
  int rc = ensure_attrs();
  if (rc) return rc;
  const int nblk = (n + TB - 1) / TB;
  cplx* Linv = invtb_buf(c, n);
  for (int b = 0; b < nblk; ++b) {
    const int k0 = b * TB, bs = std::min(TB, n - k0);
    if ((rc = trtri_block(c, bs, L + (size_t)k0 + (size_t)k0 * ldl, ldl, Linv + (size_t)b * TB * TB))) return rc;
  }
  cplx* T = temp_buf(c, n);
  cplx* P3 = panel3_buf(c, n);
  const cplx one = mk(1, 0), zero = mk(0, 0), mone = mk(-1, 0), mhalf = mk(-0.5, 0);
  for (int b = 0; b < nblk; ++b) {
    const int k0 = b * TB, bs = std::min(TB, n - k0), rest = n - k0 - bs;
    cplx* A11 = A + (size_t)k0 + (size_t)k0 * lda;
    const cplx* Lb = Linv + (size_t)b * TB * TB;
    // A11 <- Lb A11 Lb^H (A11 read Hermitian from its lower triangle, written as a full square)
    if ((rc = zgemm(c, gemm_args(OP_H, OP_C, bs, bs, bs, one, A11, lda, Lb, TB, zero, T, bs), nullptr, 0))) return rc;
    if ((rc = zgemm(c, gemm_args(OP_N, OP_N, bs, bs, bs, one, Lb, TB, T, bs, zero, A11, lda), nullptr, 0))) return rc;
    if (rest <= 0) break;
    cplx* A21 = A + (size_t)(k0 + bs) + (size_t)k0 * lda;
    const cplx* L21 = L + (size_t)(k0 + bs) + (size_t)k0 * ldl;
    cplx* A22 = A + (size_t)(k0 + bs) + (size_t)(k0 + bs) * lda;
    // A21 <- A21 Lb^H (through the temporary), then A21 -= 1/2 L21 A11
    if ((rc = zgemm(c, gemm_args(OP_N, OP_C, rest, bs, bs, one, A21, lda, Lb, TB, zero, T, rest), nullptr, 0)))
      return rc;
    k_copy_block<<<1024, 256, 0, c.st>>>(T, rest, A21, lda, rest, bs);
    count_launch();
    if ((rc = zgemm(c, gemm_args(OP_N, OP_N, rest, bs, bs, mhalf, L21, ldl, A11, lda, one, A21, lda), nullptr, 0)))
      return rc;
    // A22 -= [A21 L21] [L21 A21]^H (lower), from the buffer [A21 L21 A21] (ld rest)
    k_copy_block<<<1024, 256, 0, c.st>>>(A21, lda, P3, rest, rest, bs);
    k_copy_block<<<1024, 256, 0, c.st>>>(L21, ldl, P3 + (size_t)bs * rest, rest, rest, bs);
    k_copy_block<<<1024, 256, 0, c.st>>>(A21, lda, P3 + (size_t)2 * bs * rest, rest, rest, bs);
    count_launch(3);
    if ((rc = zgemm(c, gemm_args(OP_N, OP_C, rest, rest, 2 * bs, mone, P3, rest, P3 + (size_t)bs * rest, rest, one,
                                 A22, lda, 1), nullptr, 0)))
      return rc;
    if ((rc = zgemm(c, gemm_args(OP_N, OP_N, rest, bs, bs, mhalf, L21, ldl, A11, lda, one, A21, lda), nullptr, 0)))
      return rc;
    // A21 <- L22^{-1} A21: forward solve over the following diagonal blocks
    for (int bb = b + 1; bb < nblk; ++bb) {
      const int off = bb * TB - (k0 + bs), bsb = std::min(TB, n - bb * TB), rest2 = rest - off - bsb;
      cplx* Xb = A21 + off;
      if ((rc = zgemm(c, gemm_args(OP_N, OP_N, bsb, bs, bsb, one, Linv + (size_t)bb * TB * TB, TB, Xb, lda, zero, T,
                                   TB), nullptr, 0)))
        return rc;
      k_copy_block<<<1024, 256, 0, c.st>>>(T, TB, Xb, lda, bsb, bs);
      count_launch();
      if (rest2 > 0)
        if ((rc = zgemm(c, gemm_args(OP_N, OP_N, rest2, bs, bsb, mone, L + (size_t)(bb * TB + bsb) + (size_t)(bb * TB) * ldl,
                                     ldl, Xb, lda, one, Xb + bsb, lda), nullptr, 0)))
          return rc;
    }
  }
  const size_t total = (size_t)n * n;
  k_fill_upper<<<grid1d(total), 256, 0, c.st>>>(A, lda, n);
  count_launch();
  GBHE_CUDA(cudaGetLastError());
  return 0;
}

}  // namespace gbhe
