// backtransform.cu -- Algorithm 2 step 3 for two stages (paper Section 4.2):
// X = Q1 Q2 Z.  Because the reduction ran in two steps, the back-transform
// does too.
//
// Q2 (bulge-chasing reflectors).  Q2 = prod over sweeps s (ascending) and
// steps j of H(s, j); H(s, j) acts on rows s+1+j*nb .. s+(j+1)*nb.  Within a
// sweep the steps act on disjoint rows (they commute); H(s+1, .) overlaps
// H(s, .) only for equal or neighbouring steps.  Grouping nb consecutive
// sweeps, the valid order is: groups from last to first; inside a group step
// j ascending; inside (group, j) sweeps descending.  With the tensor-core
// engine the reflectors of one (group, j) form a block reflector, two groups'
// blocks are merged, and the merged blocks are applied in wavefront steps as
// batched products (apply_q2_blocks); when most eigenvectors are wanted the
// same blocks are applied to the identity instead, each only to the columns
// it can reach, and X = Q2 Z follows as one product.  Otherwise (the FP64
// engine, or nb beyond the block path) each CTA owns a slab of SLAB columns
// of X and walks all reflectors in that order, keeping the (2nb-1)-row window
// of the current (group, j) in shared memory (k_apply_q2).
//
// Q1 (panel block reflectors of stage 1).  Q1 = Q_0 Q_1 ... with
// Q_p = I - V_p T_p V_p^H on rows p*nb+nb .. n-1, applied last panel first,
// two panels at a time: Q_{p-1} Q_p = I - [V_{p-1} V_p] Tm [V_{p-1} V_p]^H with
// Tm = [[T_{p-1}, -T_{p-1} (V_{p-1}^H V_p) T_p], [0, T_p]] (V_p starts nb rows
// lower), as three products formed transposed so that the 2nb-wide side is
// the column dimension: Wt = X^H V, Wt = Wt Tm^H, X -= V Wt^H.  Pairing halves
// the passes over X and doubles the contraction of the last product.
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

// ---------------------------------------------------------------- Q2 as block reflectors
// Diamond (b, j): the step-j reflectors of sweeps b*nb .. b*nb+nb-1.  Their
// rows start at r0 = (b + j) nb + 1 (the reflector of sweep b*nb + c starts at
// local row c), so the diamond is one block reflector on a (2nb-1)-row window:
//   H(s0, j) H(s0+1, j) ... H(s0+nb-1, j) = I - V T V^H = I - U V^H,  U = V T,
// T upper triangular from the forward recurrence.  Diamonds are numbered
// gid = b J - b (b - 1) / 2 + j.  Applied in wavefront order
// t = 2 (J - 1 - b) + j: diamonds of one step touch disjoint rows, and every
// pair of overlapping diamonds is ordered as the sequential order requires
// (later sweeps first; within a sweep group, step j ascending).
__host__ __device__ inline long q2_gid(int b, int j, int J) { return (long)b * J - (long)b * (b - 1) / 2 + j; }

__global__ void __launch_bounds__(256) k_q2_build(int n, int nb, int J, const cplx* V2, const cplx* tau2, cplx* Vg,
                                                  cplx* Ug, cplx* Tg) {
  extern __shared__ cplx sm[];
  cplx* T = sm;            // nb x nb
  cplx* G = sm + nb * nb;  // nb x nb (Gram V^H V)
  __shared__ cplx tau_s[128];
  const long gid = blockIdx.x;
  int b = 0;
  while (b + 1 < J && q2_gid(b + 1, 0, J) <= gid) ++b;
  const int j = (int)(gid - q2_gid(b, 0, J));
  const int s0 = b * nb, r0 = (b + j) * nb + 1, W2 = 2 * nb;
  cplx* V = Vg + (size_t)gid * W2 * nb;
  cplx* U = Ug + (size_t)gid * W2 * nb;
  const int t = threadIdx.x;
  // V (window rows x nb, ld 2nb): column c holds the reflector of sweep s0 + c at rows c.. c+L-1
  for (int q = t; q < W2 * nb; q += blockDim.x) {
    const int i = q % W2, c = q / W2, s = s0 + c;
    cplx v = mk(0.0, 0.0);
    if (s <= n - 2 && j < (n - 1 - s + nb - 1) / nb) {
      const int a = s + 1 + j * nb, L = min(nb, n - a);
      if (i >= c && i < c + L && r0 + i < n) v = V2[((size_t)s * J + j) * nb + (i - c)];
    }
    V[q] = v;
  }
  for (int c = t; c < nb; c += blockDim.x) {
    const int s = s0 + c;
    tau_s[c] = (s <= n - 2 && j < (n - 1 - s + nb - 1) / nb) ? tau2[(size_t)s * J + j] : mk(0.0, 0.0);
  }
  __syncthreads();
  // Gram: G[q][c] = V(:,q)^H V(:,c) for q < c (overlap rows c .. q+nb-1)
  for (int e = t; e < nb * nb; e += blockDim.x) {
    const int q = e % nb, c = e / nb;
    cplx acc = mk(0.0, 0.0);
    if (q < c)
      for (int i = c; i < min(q + nb, W2); ++i) ccfma(acc, V[i + (size_t)q * W2], V[i + (size_t)c * W2]);
    G[q + c * nb] = acc;
    T[q + c * nb] = mk(0.0, 0.0);
  }
  __syncthreads();
  for (int c = 0; c < nb; ++c) {
    const cplx tc = tau_s[c];
    // T(0:c, c) = -tau_c T(0:c, 0:c) G(0:c, c)
    for (int r = t; r < c; r += blockDim.x) {
      cplx acc = mk(0.0, 0.0);
      for (int q = r; q < c; ++q) cfma(acc, T[r + q * nb], G[q + c * nb]);
      T[r + c * nb] = cscal(-1.0, cmul(tc, acc));
    }
    if (t == 0) T[c + c * nb] = tc;
    __syncthreads();
  }
  // U = V T
  for (int q = t; q < W2 * nb; q += blockDim.x) {
    const int i = q % W2, c = q / W2;
    cplx acc = mk(0.0, 0.0);
    for (int k = max(0, i - nb + 1); k <= min(c, i); ++k) cfma(acc, V[i + (size_t)k * W2], T[k + c * nb]);
    U[q] = acc;
  }
  cplx* Tout = Tg + (size_t)gid * nb * nb;
  for (int q = t; q < nb * nb; q += blockDim.x) Tout[q] = T[q];
}

// ---------------------------------------------------------------- merged blocks
// The diamonds of sweep groups 2c and 2c+1 at the same step j cover rows
// r0 .. r0+3nb-2 (r0 = (2c + j) nb + 1; the second one starts nb rows lower)
// and are applied as one block reflector of 2nb columns,
//   D(2c, j) D(2c+1, j) = I - [V1 V2] [[T1, T12], [0, T2]] [V1 V2]^H,
//   T12 = -T1 (V1^H V2) T2,   U = V T = [U1, V1 T12 + U2],
// the group 2c+1 diamond acting first (later sweeps first).  Merged blocks
// (c, j), j < J - 2c, are numbered mid = c J - c (c - 1) + j and applied in
// wavefront order w = (C - 1 - c) + j, C = ceil(J / 2): blocks of one step
// touch disjoint rows, and every block comes after the blocks it overlaps
// that the sequential order puts first ((c+1, j-2 .. j) and (c, j-1)).  This
// halves the number of wavefront steps (about 1.5 J instead of 3 J) and
// doubles the contraction of both products.
__host__ __device__ inline long q2m_mid(int c, int j, int J) { return (long)c * J - (long)c * (c - 1) + j; }
inline int q2_pairs(int J) { return (J + 1) / 2; }
inline long q2m_count(int J) {
  const int C = q2_pairs(J);
  return (long)C * J - (long)C * (C - 1);
}

__global__ void __launch_bounds__(256) k_q2_merge(int n, int nb, int J, const cplx* Vg, const cplx* Ug,
                                                  const cplx* Tg, cplx* Vm, cplx* Um) {
  extern __shared__ cplx sm[];
  cplx* X1 = sm;            // nb x nb: V1^H V2, then T12
  cplx* X2 = sm + nb * nb;  // nb x nb: V1^H V2 T2
  const long mid = blockIdx.x;
  const int C = (J + 1) / 2;
  int c = 0;
  while (c + 1 < C && q2m_mid(c + 1, 0, J) <= mid) ++c;
  const int j = (int)(mid - q2m_mid(c, 0, J));
  const int b = 2 * c, b2 = b + 1;
  const bool has2 = b2 < J && j < J - b2;
  const int W2 = 2 * nb, W3 = 3 * nb;
  const long g1 = q2_gid(b, j, J), g2 = has2 ? q2_gid(b2, j, J) : 0;
  const cplx* V1 = Vg + (size_t)g1 * W2 * nb;  // W2 x nb, ld W2
  const cplx* U1 = Ug + (size_t)g1 * W2 * nb;
  const cplx* T1 = Tg + (size_t)g1 * nb * nb;  // upper triangular, ld nb
  const cplx* V2b = Vg + (size_t)g2 * W2 * nb;
  const cplx* U2 = Ug + (size_t)g2 * W2 * nb;
  const cplx* T2 = Tg + (size_t)g2 * nb * nb;
  cplx* V = Vm + (size_t)mid * W3 * W2;  // W3 x 2nb, ld W3
  cplx* U = Um + (size_t)mid * W3 * W2;
  const int t = threadIdx.x;
  // V = [V1 on rows 0..2nb-1 | V2 on rows nb..3nb-1],  U(:, 0:nb) = U1 on rows 0..2nb-1
  for (int q = t; q < W3 * nb; q += blockDim.x) {
    const int i = q % W3, k = q / W3;
    V[i + (size_t)k * W3] = (i < W2) ? V1[i + (size_t)k * W2] : mk(0.0, 0.0);
    U[i + (size_t)k * W3] = (i < W2) ? U1[i + (size_t)k * W2] : mk(0.0, 0.0);
    V[i + (size_t)(nb + k) * W3] = (has2 && i >= nb) ? V2b[(i - nb) + (size_t)k * W2] : mk(0.0, 0.0);
  }
  if (!has2) {
    for (int q = t; q < W3 * nb; q += blockDim.x) U[(q % W3) + (size_t)(nb + q / W3) * W3] = mk(0.0, 0.0);
    return;
  }
  // X1 = V1^H V2 (the overlap: rows nb..2nb-1 of V1, rows 0..nb-1 of V2)
  for (int e = t; e < nb * nb; e += blockDim.x) {
    const int r = e % nb, k = e / nb;
    cplx acc = mk(0.0, 0.0);
    for (int i = 0; i < nb; ++i) ccfma(acc, V1[(nb + i) + (size_t)r * W2], V2b[i + (size_t)k * W2]);
    X1[r + k * nb] = acc;
  }
  __syncthreads();
  // X2 = X1 T2
  for (int e = t; e < nb * nb; e += blockDim.x) {
    const int r = e % nb, k = e / nb;
    cplx acc = mk(0.0, 0.0);
    for (int q = 0; q <= k; ++q) cfma(acc, X1[r + q * nb], T2[q + (size_t)k * nb]);
    X2[r + k * nb] = acc;
  }
  __syncthreads();
  // X1 = T12 = -T1 X2
  for (int e = t; e < nb * nb; e += blockDim.x) {
    const int r = e % nb, k = e / nb;
    cplx acc = mk(0.0, 0.0);
    for (int q = r; q < nb; ++q) cfma(acc, T1[r + (size_t)q * nb], X2[q + k * nb]);
    X1[r + k * nb] = cscal(-1.0, acc);
  }
  __syncthreads();
  // U(:, nb:2nb) = V1 T12 on rows 0..2nb-1, plus U2 on rows nb..3nb-1
  for (int q = t; q < W3 * nb; q += blockDim.x) {
    const int i = q % W3, k = q / W3;
    cplx acc = (i >= nb) ? U2[(i - nb) + (size_t)k * W2] : mk(0.0, 0.0);
    if (i < W2)
      for (int r = 0; r < nb; ++r) cfma(acc, V1[i + (size_t)r * W2], X1[r + k * nb]);
    U[i + (size_t)(nb + k) * W3] = acc;
  }
}

// First column that a merged block of pair c can find nonzero when the blocks
// are applied, in wavefront order, to the identity: every block applied
// before it mixes only rows >= 2c nb + 1 with each other, and those rows of
// the identity are zero left of that column.
__host__ __device__ inline int q2_first_col(int c, int nb) { return 2 * c * nb + 1; }

// Descriptors of merged wavefront step w for the batched products
//   Wt_z = X[r0 : r0+Wh, lo : c0+mc]^H V_z          (GEMM 1, W_z^H)
//   X[r0 : r0+Wh, lo : c0+mc] -= U_z Wt_z^H         (GEMM 2)
// with lo = c0, or, when Q2 itself is being formed (X starts as the
// identity), lo = max(c0, first column the block can reach).  GEMM 1 is
// formed transposed so that its long dimension (the columns of X) is the row
// dimension of the product.
__global__ void k_q2_desc(int n, int nb, int J, int w, int c_lo, int cnt, const cplx* Vm, const cplx* Um, cplx* X,
                          int ldx, int c0, int mc, int form_q, cplx* Wbuf, CrtDesc* D1, CrtDesc* D2) {
  const int z = blockIdx.x * blockDim.x + threadIdx.x;
  if (z >= cnt) return;
  const int C = (J + 1) / 2;
  const int c = c_lo + z, j = w - (C - 1 - c);
  const long mid = q2m_mid(c, j, J);
  const int r0 = (2 * c + j) * nb + 1, Wh = min(3 * nb - 1, n - r0), W3 = 3 * nb, NB2 = 2 * nb;
  const int lo = form_q ? max(c0, q2_first_col(c, nb)) : c0;
  const int cols = max(0, c0 + mc - lo);
  cplx* Wz = Wbuf + (size_t)z * NB2 * mc + (lo - c0);  // cols x 2nb, ld mc
  CrtDesc d;
  d.cmap = nullptr;
  d.A = X + (size_t)r0 + (size_t)lo * ldx; d.lda = ldx;  // op C: X window^H
  d.B = Vm + (size_t)mid * W3 * NB2; d.ldb = W3;         // op N
  d.C = Wz; d.ldc = mc;
  d.M = cols; d.N = NB2; d.K = Wh;
  D1[z] = d;
  d.A = Um + (size_t)mid * W3 * NB2; d.lda = W3;         // op N
  d.B = Wz; d.ldb = mc;                                   // op C: Wt^H = W
  d.C = X + (size_t)r0 + (size_t)lo * ldx; d.ldc = ldx;
  d.M = Wh; d.N = cols; d.K = NB2;
  D2[z] = d;
}

__global__ void k_eye(cplx* Q, int n, int ldq) {
  const size_t total = (size_t)n * n;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
    const int r = (int)(i % n), c = (int)(i / n);
    Q[(size_t)r + (size_t)c * ldq] = mk(r == c ? 1.0 : 0.0, 0.0);
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

namespace {

// Merged blocks of wavefront step w: pairs c_lo .. c_lo + cnt - 1.
void q2_step_range(int J, int w, int* c_lo, int* cnt) {
  const int C = q2_pairs(J);
  *c_lo = -1;
  *cnt = 0;
  for (int c = std::max(0, C - 1 - w); c < C; ++c) {
    const int j = w - (C - 1 - c);
    if (j < 0 || j >= J - 2 * c) break;
    if (*c_lo < 0) *c_lo = c;
    ++*cnt;
  }
}

// Largest number of merged blocks in one wavefront step.
int q2_max_step(int J) {
  int best = 0;
  for (int w = 0; w <= q2_pairs(J) + J - 2; ++w) {
    int lo, cnt;
    q2_step_range(J, w, &lo, &cnt);
    best = std::max(best, cnt);
  }
  return best;
}

bool q2_use_blocks(const Ctx& c, int n, int nb) {
  return c.engine == GBHE_ENGINE_CRT && c.crt_ws != nullptr && nb >= 2 && nb <= 64 && n > 2 * nb;
}

size_t q2_block_bytes(int n, int nb, int m) {
  const int J = hb2st_J(n, nb);
  const size_t ng = (size_t)J * (J + 1) / 2;
  const size_t nm = (size_t)q2m_count(J);
  const size_t cm = (size_t)q2_max_step(J) + 1;
  return 2 * ng * 2 * nb * nb * sizeof(cplx) + ng * nb * nb * sizeof(cplx) + 2 * nm * 6 * nb * nb * sizeof(cplx) +
         cm * 2 * nb * (size_t)std::max(m, 1) * sizeof(cplx) + 2 * cm * sizeof(CrtDesc) + 8 * 256;
}

}  // namespace

// Q2 is formed explicitly (the blocks applied to the identity, each only to
// the columns it can reach: about 2/3 of the work of applying them to n
// columns) and then applied as one n x n x m product when at least 4/5 of
// the eigenvectors are wanted; below that, the blocks go straight to X.
inline bool q2_form_explicit(int n, int m) { return 5 * (long)m >= 4 * (long)n; }

size_t unmtr_ws_bytes(int n, int nb, int m) {
  const size_t nn = (size_t)std::max(n, 1), mm = (size_t)std::max(m, 1);
  size_t b = 2 * nn * nb * sizeof(cplx) + 4 * (size_t)nb * mm * sizeof(cplx) + 6 * (size_t)nb * nb * sizeof(cplx) +
             6 * 256;
  if (nb >= 2 && nb <= 64 && n > 2 * nb) {
    if (q2_form_explicit(n, m))
      b += (nn * nn + nn * mm) * sizeof(cplx) + 2 * 256 + q2_block_bytes(n, nb, std::max(n, m));
    else
      b += q2_block_bytes(n, nb, m);
  }
  return b;
}

// Q2 applied as wavefront-batched merged block reflectors on the tensor-core
// GEMM to the m columns of X; with form_q, X is the identity (m = n) and each
// block touches only the columns it can reach.
static int apply_q2_blocks(Ctx& c, int n, int nb, int m, const cplx* V2, const cplx* tau2, cplx* X, int ldx,
                           bool form_q) {
  Arena& ar = c.arena;
  const size_t save = ar.off;
  const int J = hb2st_J(n, nb);
  const long ng = (long)J * (J + 1) / 2;
  const long nm = q2m_count(J);
  const int C = q2_pairs(J);
  const int cm = q2_max_step(J);
  const int W2 = 2 * nb, W3 = 3 * nb;
  cplx* Vg = ar.take<cplx>((size_t)ng * W2 * nb);
  cplx* Ug = ar.take<cplx>((size_t)ng * W2 * nb);
  cplx* Tg = ar.take<cplx>((size_t)ng * nb * nb);
  cplx* Vm = ar.take<cplx>((size_t)nm * W3 * W2);
  cplx* Um = ar.take<cplx>((size_t)nm * W3 * W2);
  // column chunk so that one batched product fits the tensor-core workspace
  int mc = std::min(m, 64 * ((m + 63) / 64));
  auto need = [&](int w) {
    return std::max(crt_batched_ws_bytes(cm, w, W2, W3 - 1, 1), crt_batched_ws_bytes(cm, W3 - 1, w, W2, 1));
  };
  while (mc > 64 && need(mc) > c.crt_ws_bytes) mc -= 64;
  mc = std::min(mc, m);
  cplx* Wbuf = ar.take<cplx>((size_t)std::max(cm, 1) * W2 * mc);
  CrtDesc* D1 = ar.take<CrtDesc>((size_t)std::max(cm, 1));
  CrtDesc* D2 = ar.take<CrtDesc>((size_t)std::max(cm, 1));
  if (!ar.ok() || !D2) { ar.off = save; return GBHE_EWORKSPACE; }
  const size_t smem = (size_t)2 * nb * nb * sizeof(cplx);
  GBHE_CUDA(cudaFuncSetAttribute(k_q2_build, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  GBHE_CUDA(cudaFuncSetAttribute(k_q2_merge, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  double fl = 0.0;
  if (prof_on())
    for (int s = 0; s <= n - 2; ++s)
      for (int a0 = s + 1; a0 < n; a0 += nb) fl += 16.0 * std::min(nb, n - a0) * (double)m;
  ProfScope prof(c.st, GBHE_PROF_Q2, fl, 16.0 * ((double)n * J * nb + 2.0 * (double)n * m));
  k_q2_build<<<(unsigned)ng, 256, smem, c.st>>>(n, nb, J, V2, tau2, Vg, Ug, Tg);
  count_launch();
  GBHE_CUDA(cudaGetLastError());
  k_q2_merge<<<(unsigned)nm, 256, smem, c.st>>>(n, nb, J, Vg, Ug, Tg, Vm, Um);
  count_launch();
  GBHE_CUDA(cudaGetLastError());
  int rc = 0;
  for (int c0 = 0; c0 < m && !rc; c0 += mc) {
    const int mcc = std::min(mc, m - c0);
    for (int w = 0; w <= C + J - 2 && !rc; ++w) {
      int c_lo, cnt;
      q2_step_range(J, w, &c_lo, &cnt);
      if (cnt == 0) continue;
      k_q2_desc<<<(cnt + 127) / 128, 128, 0, c.st>>>(n, nb, J, w, c_lo, cnt, Vm, Um, X, ldx, c0, mcc, form_q ? 1 : 0,
                                                      Wbuf, D1, D2);
      count_launch();
      double gfl = 0.0;  // each of the two products: 8 (2 nb) cols Wh per merged block
      if (prof_on())
        for (int z = 0; z < cnt; ++z) {
          const int cc = c_lo + z, j = w - (C - 1 - cc);
          const int lo = form_q ? std::max(c0, q2_first_col(cc, nb)) : c0;
          gfl += 8.0 * W2 * std::max(0, c0 + mcc - lo) * std::min(W3 - 1, n - ((2 * cc + j) * nb + 1));
        }
      rc = crt_gemm_batched(c.st, OP_C, OP_N, mk(1, 0), mk(0, 0), 1, D1, cnt, mcc, W2, W3 - 1, c.crt_ws,
                            c.crt_ws_bytes, c.status, gfl);
      if (!rc)
        rc = crt_gemm_batched(c.st, OP_N, OP_C, mk(-1, 0), mk(1, 0), 1, D2, cnt, W3 - 1, mcc, W2, c.crt_ws,
                              c.crt_ws_bytes, c.status, gfl);
    }
  }
  ar.off = save;
  return rc;
}

int unmtr2_run(Ctx& c, int n, int nb, int m, const cplx* A, int lda, const cplx* T1, const cplx* V2,
               const cplx* tau2, const double* Z, int ldz, cplx* X, int ldx) {
  if (n <= 0 || m <= 0) return 0;
  Arena& ar = c.arena;
  const size_t save = ar.off;
  cplx* V = ar.take<cplx>((size_t)n * 2 * nb);      // [V_{p-1} V_p], ld n
  cplx* W1 = ar.take<cplx>((size_t)2 * nb * m);     // m x 2nb, ld m
  cplx* W2 = ar.take<cplx>((size_t)2 * nb * m);
  cplx* Tm = ar.take<cplx>((size_t)4 * nb * nb);    // 2nb x 2nb, ld 2nb
  cplx* Gs = ar.take<cplx>((size_t)nb * nb);        // nb x nb
  cplx* Ss = ar.take<cplx>((size_t)nb * nb);
  if (!ar.ok() || !Ss) { ar.off = save; return GBHE_EWORKSPACE; }
  const size_t total = (size_t)n * m;
  const bool form_q = q2_use_blocks(c, n, nb) && q2_form_explicit(n, m);
  if (form_q) {
    // ---- Q2 formed explicitly, then X = Q2 Z in one product
    cplx* Qe = ar.take<cplx>((size_t)n * n);
    cplx* Zc = ar.take<cplx>(total);
    if (!ar.ok() || !Zc) { ar.off = save; return GBHE_EWORKSPACE; }
    k_eye<<<(int)std::min<size_t>(((size_t)n * n + 255) / 256, 4096), 256, 0, c.st>>>(Qe, n, n);
    count_launch();
    k_promote<<<(int)std::min<size_t>((total + 255) / 256, 4096), 256, 0, c.st>>>(Z, ldz, n, m, Zc, n);
    count_launch();
    GBHE_CUDA(cudaGetLastError());
    int rc = apply_q2_blocks(c, n, nb, n, V2, tau2, Qe, n, true);
    if (!rc) {
      ProfScope prof(c.st, GBHE_PROF_Q2, 0.0, 0.0);
      rc = zgemm(c, gemm_args(OP_N, OP_N, n, m, n, mk(1, 0), Qe, n, Zc, n, mk(0, 0), X, ldx), nullptr, 0);
    }
    if (rc) { ar.off = save; return rc; }
  } else {
    k_promote<<<(int)std::min<size_t>((total + 255) / 256, 4096), 256, 0, c.st>>>(Z, ldz, n, m, X, ldx);
    count_launch();
    GBHE_CUDA(cudaGetLastError());
  }
  // ---- Q2 applied to X (unless it was formed above)
  if (form_q) {
    // done
  } else if (q2_use_blocks(c, n, nb)) {
    int rc = apply_q2_blocks(c, n, nb, m, V2, tau2, X, ldx, false);
    if (rc) { ar.off = save; return rc; }
  } else if (n >= 2) {
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
  // ---- Q1, last panel first, in pairs (p-1, p)
  int npan = 0;
  for (int k = 0; k + nb < n; k += nb) ++npan;
  const cplx one = mk(1, 0), zero = mk(0, 0), mone = mk(-1, 0);
  const size_t es = sizeof(cplx);
  // explicit V of panel p (its mp rows, nb columns, ld n) at dst
  auto vpanel = [&](int p, cplx* dst) {
    const int k = p * nb, mp = n - k - nb, kr = std::min(nb, mp);
    k_panel_v<<<(int)std::min<size_t>(((size_t)mp * nb + 255) / 256, 4096), 256, 0, c.st>>>(A, lda, k, nb, mp, kr, dst,
                                                                                           n);
    count_launch();
    return cudaGetLastError() == cudaSuccess ? 0 : GBHE_ECUDA;
  };
  int rc = 0;
  for (int p = npan - 1; p >= 0 && !rc; p -= 2) {
    const int q = p - 1;                       // the pair (q, p), or p alone when q < 0
    const int k = (q >= 0 ? q : p) * nb, mp = n - k - nb;
    cplx* Xr = X + (k + nb);
    int w;                                     // block width
    const cplx* Tb;                            // its T, ld ldt
    int ldt;
    if (q >= 0) {
      w = 2 * nb;
      if ((rc = vpanel(q, V))) break;
      // V_p, nb rows lower in the second column block; its first nb rows are zero
      GBHE_CUDA(cudaMemset2DAsync(V + (size_t)nb * n, es * n, 0, es * nb, nb, c.st));
      if ((rc = vpanel(p, V + (size_t)nb * n + nb))) break;
      const cplx* Tq = T1 + (size_t)q * nb * nb;
      const cplx* Tp = T1 + (size_t)p * nb * nb;
      // Tm = [[Tq, -Tq (Vq^H Vp) Tp], [0, Tp]]
      if ((rc = zgemm(c, gemm_args(OP_C, OP_N, nb, nb, mp, one, V, n, V + (size_t)nb * n, n, zero, Gs, nb),
                      c.gemm_scratch, c.gemm_scratch_bytes))) break;
      if ((rc = zgemm(c, gemm_args(OP_N, OP_N, nb, nb, nb, one, Gs, nb, Tp, nb, zero, Ss, nb), nullptr, 0))) break;
      if ((rc = zgemm(c, gemm_args(OP_N, OP_N, nb, nb, nb, mone, Tq, nb, Ss, nb, zero, Tm + (size_t)nb * 2 * nb,
                                   2 * nb), nullptr, 0))) break;
      GBHE_CUDA(cudaMemcpy2DAsync(Tm, es * 2 * nb, Tq, es * nb, es * nb, nb, cudaMemcpyDeviceToDevice, c.st));
      GBHE_CUDA(cudaMemcpy2DAsync(Tm + (size_t)nb * 2 * nb + nb, es * 2 * nb, Tp, es * nb, es * nb, nb,
                                  cudaMemcpyDeviceToDevice, c.st));
      GBHE_CUDA(cudaMemset2DAsync(Tm + nb, es * 2 * nb, 0, es * nb, nb, c.st));
      Tb = Tm;
      ldt = 2 * nb;
    } else {
      w = std::min(nb, mp);
      if ((rc = vpanel(p, V))) break;
      Tb = T1 + (size_t)p * nb * nb;
      ldt = nb;
    }
    if ((rc = zgemm(c, gemm_args(OP_C, OP_N, m, w, mp, one, Xr, ldx, V, n, zero, W1, m), c.gemm_scratch,
                    c.gemm_scratch_bytes))) break;
    if ((rc = zgemm(c, gemm_args(OP_N, OP_C, m, w, w, one, W1, m, Tb, ldt, zero, W2, m), nullptr, 0))) break;
    if ((rc = zgemm(c, gemm_args(OP_N, OP_C, mp, m, w, mone, V, n, W2, m, one, Xr, ldx), nullptr, 0))) break;
  }
  if (rc) { ar.off = save; return rc; }
  ar.off = save;
  return 0;
}

}  // namespace gbhe
