// he2hb.cu -- first stage of the two-stage tridiagonalisation (paper Section
// 4.2, Figure 1): Hermitian dense -> Hermitian band of half-bandwidth nb by
// block Householder transformations.
//
// For each panel (columns k..k+nb-1):
//   (a) QR of the panel P = A[k+nb:n, k:k+nb] = Q R,  Q = I - V T V^H
//       (one cooperative kernel: rows split over the CTAs, each CTA keeps its
//       rows in shared memory; one bounded grid barrier per column);
//   (c) two-sided update of the trailing matrix A22 <- Q^H A22 Q as
//       X = A22 V T,  W = X - 1/2 V (T^H V^H X),  A22 -= V W^H + W V^H
//       (A22 read as Hermitian from its lower triangle and only the lower
//       triangle written).  The rank-2nb update is one product,
//       A22 -= [V W] [W V]^H, so the trailing matrix is read and written once
//       per panel with a contraction of 2nb: V, W and a second copy of V sit
//       side by side in one buffer, [V W] and [W V] are two overlapping
//       column ranges of it.
// Lookahead (the panel/update overlap of the paper's Figure 1): the update
// first brings the next panel's nb columns up to date, then the next panel is
// factored on the handle's panel stream while the rest of the trailing matrix
// is updated on the caller's stream; the two meet again before the next
// update.  Panels alternate between two [V X V] buffers so that the next
// panel never overwrites the V that the running update still reads.
#include <algorithm>
#include "internal.cuh"

namespace gbhe {
namespace {

constexpr int PT = 256;

struct PanelArgs {
  cplx* A;
  int lda, n, k, nb, kr, mp, chunk;
  cplx* V;     // explicit V (mp x nb, ld ldv): unit diagonal, zeros above
  int ldv;
  cplx* tau;   // tau1 + k
  cplx* T;     // nb x nb, ld nb
  cplx* part;  // 2 x G x (nb + 1) partial sums (double-buffered by column parity)
  cplx* row;   // 2 x nb: the pivot row of the next column (double-buffered)
  unsigned* bar;
  int* st;
};

__device__ __forceinline__ cplx warp_sum(cplx v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    v.x += __shfl_xor_sync(0xffffffffu, v.x, o);
    v.y += __shfl_xor_sync(0xffffffffu, v.y, o);
  }
  return v;
}

// Householder QR of the panel with one grid barrier per column.  The
// reflector of column j is v = (x - beta e_j) / (alpha - beta) (x the column,
// alpha = x_j), so everything the update needs can be summed over the CTAs
// from the UNSCALED column in one round:
//   |x(j+1:)|^2,  x^H P(:, c) (c > j),  V(:, c)^H x (c < j; for T),
// plus the pivot row P(j, :) published by its owner; then
//   w_c = v^H P(:, c) = conj(s) (x^H P(:, c) - beta P(j, c)),
//   V(:, c)^H v = s (V(:, c)^H x - beta conj(V(j, c))),  s = 1 / (alpha - beta),
// and after the update each CTA forms its parts of the next column's sums
// before the barrier.  Partial sums and the pivot row alternate between two
// buffers, so a CTA that runs ahead never overwrites what a slower one still
// reads (it cannot pass the next barrier before the slower one arrives).
__global__ void __launch_bounds__(PT) k_panel_qr(PanelArgs p) {
  extern __shared__ cplx S[];  // chunk x nb, ld chunk
  __shared__ cplx wsum[128], cw[128], vv[128];
  __shared__ double rednrm[PT / 32];
  __shared__ cplx sh_tau, sh_scal;
  __shared__ double sh_beta;
  const int G = gridDim.x, b = blockIdx.x, t = threadIdx.x, lane = t & 31, warp = t >> 5;
  const int r0 = b * p.chunk, r1 = min(p.mp, r0 + p.chunk), rows = max(0, r1 - r0);
  const int nb = p.nb, PS = nb + 1;
  for (int i = t; i < rows * nb; i += PT) {
    int r = i % rows, c = i / rows;
    S[r + c * p.chunk] = p.A[(size_t)(p.k + nb + r0 + r) + (size_t)(p.k + c) * p.lda];
  }
  if (b == 0)
    for (int i = t; i < nb * nb; i += PT) p.T[i] = mk(0.0, 0.0);
  __syncthreads();

  // this CTA's parts of the sums of column j (rows gi >= j) into buffer j & 1,
  // and the pivot row j if this CTA holds it
  auto sums = [&](int j) {
    cplx* pb = p.part + ((size_t)(j & 1) * G + b) * PS;
    double s = 0.0;
    for (int r = t; r < rows; r += PT)
      if (r0 + r > j) s += cabs2(S[r + j * p.chunk]);
    s = warp_sum(mk(s, 0.0)).x;
    if (lane == 0) rednrm[warp] = s;
    for (int c = warp; c < nb; c += PT / 32) {
      if (c == j) continue;
      cplx acc = mk(0.0, 0.0);
      for (int r = lane; r < rows; r += 32) {
        if (r0 + r < j) continue;
        const cplx x = S[r + j * p.chunk];
        if (c > j) ccfma(acc, x, S[r + c * p.chunk]);  // conj(x_i) P(i, c)
        else ccfma(acc, S[r + c * p.chunk], x);        // conj(V(i, c)) x_i
      }
      acc = warp_sum(acc);
      if (lane == 0) pb[1 + c] = acc;
    }
    if (j >= r0 && j < r1) {
      cplx* rw = p.row + (size_t)(j & 1) * nb;
      for (int c = t; c < nb; c += PT) rw[c] = S[(j - r0) + c * p.chunk];
    }
    __syncthreads();
    if (t == 0) {
      double tot = 0.0;
      for (int w = 0; w < PT / 32; ++w) tot += rednrm[w];
      pb[0] = mk(tot, 0.0);
    }
  };

  if (p.kr > 0) sums(0);
  for (int j = 0; j < p.kr; ++j) {
    if (!grid_barrier(p.bar, G, p.st)) return;
    const cplx* pbuf = p.part + (size_t)(j & 1) * G * PS;
    const cplx* rw = p.row + (size_t)(j & 1) * nb;
    // ---- totals over the CTAs
    if (warp == 0) {
      double x2 = 0.0;
      for (int q = lane; q < G; q += 32) x2 += __ldcg(&pbuf[(size_t)q * PS]).x;
      x2 = warp_sum(mk(x2, 0.0)).x;
      if (lane == 0) {
        const cplx al = __ldcg(&rw[j]);
        if (x2 == 0.0 && al.y == 0.0) {
          sh_tau = mk(0.0, 0.0); sh_beta = al.x; sh_scal = mk(0.0, 0.0);
        } else {
          const double nrm = sqrt(al.x * al.x + al.y * al.y + x2);
          const double beta = (al.x >= 0.0) ? -nrm : nrm;
          sh_beta = beta;
          sh_tau = mk((beta - al.x) / beta, -al.y / beta);
          sh_scal = cinv(mk(al.x - beta, al.y));
        }
      }
    }
    for (int c = warp; c < nb; c += PT / 32) {
      cplx acc = mk(0.0, 0.0);
      if (c != j)
        for (int q = lane; q < G; q += 32) acc = cadd(acc, __ldcg(&pbuf[(size_t)q * PS + 1 + c]));
      acc = warp_sum(acc);
      if (lane == 0) wsum[c] = acc;
    }
    __syncthreads();
    const cplx tau = sh_tau, scal = sh_scal;
    const double beta = sh_beta;
    if (t < nb) {
      const cplx rc = __ldcg(&rw[t]);
      if (t > j) {  // conj(tau) w_c
        const cplx wc = cmul(cconj(scal), csub(wsum[t], cscal(beta, rc)));
        cw[t] = cmul(cconj(tau), wc);
      } else if (t < j) {  // V(:, t)^H v
        vv[t] = cmul(scal, csub(wsum[t], cscal(beta, cconj(rc))));
      }
    }
    // ---- the reflector in column j
    for (int r = t; r < rows; r += PT) {
      const int gi = r0 + r;
      if (gi > j) S[r + j * p.chunk] = cmul(S[r + j * p.chunk], scal);
      else if (gi == j) S[r + j * p.chunk] = mk(beta, 0.0);
    }
    if (b == 0 && t == 0) p.tau[j] = tau;
    __syncthreads();
    // ---- P(i, c) -= conj(tau) v_i w_c  (c > j, i >= j, v_j = 1)
    for (int i = t; i < rows * nb; i += PT) {
      const int r = i % rows, c = i / rows, gi = r0 + r;
      if (c <= j || gi < j) continue;
      const cplx vi = (gi == j) ? mk(1.0, 0.0) : S[r + j * p.chunk];
      S[r + c * p.chunk] = csub(S[r + c * p.chunk], cmul(vi, cw[c]));
    }
    if (b == 0) {
      // T(0:j, j) = -tau T(0:j, 0:j) (V^H v_j);  T(j, j) = tau
      for (int r = t; r < j; r += PT) {
        cplx acc = mk(0.0, 0.0);
        for (int q = r; q < j; ++q) cfma(acc, p.T[r + q * nb], vv[q]);
        p.T[r + j * nb] = cscal(-1.0, cmul(tau, acc));
      }
      if (t == 0) p.T[j + j * nb] = tau;
    }
    __syncthreads();
    if (j + 1 < p.kr) sums(j + 1);
  }
  // write back the panel (R above/on the diagonal, V below) and explicit V
  for (int i = t; i < rows * nb; i += PT) {
    int r = i % rows, c = i / rows, gi = r0 + r;
    cplx v = S[r + c * p.chunk];
    p.A[(size_t)(p.k + nb + gi) + (size_t)(p.k + c) * p.lda] = v;
    cplx e = mk(0.0, 0.0);
    if (c < p.kr) {
      if (gi == c) e = mk(1.0, 0.0);
      else if (gi > c) e = v;
    }
    p.V[(size_t)gi + (size_t)c * p.ldv] = e;
  }
}

}  // namespace

size_t he2hb_ws_bytes(int n, int nb, int num_sms) {
  size_t nn = (size_t)std::max(n, 1);
  size_t b = 0;
  b += nn * nb * sizeof(cplx) * 7 + 3 * 256;          // two [V X V], VT
  b += (size_t)nb * nb * sizeof(cplx) * 2 + 2 * 256;  // Y, Z
  b += 2 * (size_t)(num_sms + 1) * (nb + 1) * sizeof(cplx) + 256;  // partial sums, two buffers
  b += 2 * (size_t)nb * sizeof(cplx) + 256;                         // pivot rows, two buffers
  b += 256 * 2;
  return b;
}

int he2hb_run(Ctx& c, int n, int nb, cplx* A, int lda, cplx* T1, cplx* tau1) {
  if (n <= 0) return 0;
  Arena& a = c.arena;
  const size_t save = a.off;
  // VXV: V (explicit, from the panel kernel), then X, then a copy of V, each
  // kr columns wide with leading dimension n; nb + 2 nb columns are reserved
  // (the panel kernel writes nb columns of V, zero beyond kr)
  cplx* VXVb[2];
  VXVb[0] = a.take<cplx>((size_t)n * 3 * nb);
  VXVb[1] = a.take<cplx>((size_t)n * 3 * nb);
  cplx* VT = a.take<cplx>((size_t)n * nb);
  cplx* Ys = a.take<cplx>((size_t)nb * nb);
  cplx* Zs = a.take<cplx>((size_t)nb * nb);
  cplx* part = a.take<cplx>(2 * (size_t)(c.num_sms + 1) * (nb + 1));
  cplx* prow = a.take<cplx>(2 * (size_t)nb);
  if (!a.ok() || !prow) { a.off = save; return GBHE_EWORKSPACE; }
  GBHE_CUDA(cudaMemsetAsync(tau1, 0, sizeof(cplx) * n, c.st));
  const int npan = (n + nb - 1) / nb;
  GBHE_CUDA(cudaMemsetAsync(T1, 0, sizeof(cplx) * (size_t)npan * nb * nb, c.st));
  int rc = 0;
  static size_t attr_set[MAX_DEVICES] = {};
  const int dev = device_slot();
  if (dev < 0) { a.off = save; return GBHE_ECUDA; }
  bool pending = false;  // a panel recorded on ev_b that the caller's stream has not joined yet
  // QR of panel k (columns k .. k+nb-1, rows k+nb .. n-1) on the panel
  // stream, after the work already queued on the caller's stream, into the
  // [V X V] buffer `buf`; the caller's stream waits for it before the update.
  auto panel = [&](int k, cplx* buf) -> int {
    const int mp = n - k - nb, kr = std::min(nb, mp);
    const int G = std::min(c.num_sms, std::max(1, (mp + 7) / 8));
    const int chunk = (mp + G - 1) / G;
    const size_t smem = (size_t)chunk * nb * sizeof(cplx);
    if (smem > 200 * 1024) return -3;
    if (smem > 48 * 1024 && smem > attr_set[dev]) {
      GBHE_CUDA(cudaFuncSetAttribute(k_panel_qr, cudaFuncAttributeMaxDynamicSharedMemorySize, 210 * 1024));
      attr_set[dev] = 210 * 1024;
    }
    PanelArgs pa;
    pa.A = A; pa.lda = lda; pa.n = n; pa.k = k; pa.nb = nb; pa.kr = kr; pa.mp = mp; pa.chunk = chunk;
    pa.V = buf; pa.ldv = n; pa.tau = tau1 + k; pa.T = T1 + (size_t)(k / nb) * nb * nb;
    pa.part = part; pa.row = prow; pa.bar = reinterpret_cast<unsigned*>(c.status + ST_BAR);
    pa.st = c.status;
    void* args[] = {&pa};
    GBHE_CUDA(cudaEventRecord(c.ev_a, c.st));
    GBHE_CUDA(cudaStreamWaitEvent(c.aux, c.ev_a, 0));
    count_launch();
    {
      const double fl = 4.0 * (2.0 * mp * (double)kr * kr - 2.0 * (double)kr * kr * kr / 3.0);
      ProfScope prof(c.aux, GBHE_PROF_PANEL, fl, 2.0 * 16.0 * mp * nb);
      GBHE_CUDA(cudaLaunchCooperativeKernel((const void*)k_panel_qr, dim3(G), dim3(PT), args, smem, c.aux));
    }
    GBHE_CUDA(cudaEventRecord(c.ev_b, c.aux));
    pending = true;
    return 0;
  };
  if (nb < n && (rc = panel(0, VXVb[0]))) { a.off = save; return rc; }
  for (int k = 0, p = 0; k + nb < n; k += nb, ++p) {
    const int mp = n - k - nb;
    const int kr = std::min(nb, mp);
    cplx* VXV = VXVb[p & 1];
    cplx* V = VXV;
    cplx* X = VXV + (size_t)kr * n;
    cplx* V2c = VXV + (size_t)2 * kr * n;
    GBHE_CUDA(cudaStreamWaitEvent(c.st, c.ev_b, 0));  // panel k factored
    pending = false;
    // ---- trailing update
    cplx* A22 = A + (size_t)(k + nb) + (size_t)(k + nb) * lda;
    const cplx* T = T1 + (size_t)(k / nb) * nb * nb;
    const cplx one = mk(1, 0), zero = mk(0, 0), mone = mk(-1, 0);
    if ((rc = zgemm(c, gemm_args(OP_N, OP_N, mp, kr, kr, one, V, n, T, nb, zero, VT, n), nullptr, 0))) break;
    if ((rc = zgemm(c, gemm_args(OP_H, OP_N, mp, kr, mp, one, A22, lda, VT, n, zero, X, n), nullptr, 0))) break;
    if ((rc = zgemm(c, gemm_args(OP_C, OP_N, kr, kr, mp, one, V, n, X, n, zero, Ys, nb), c.gemm_scratch,
                    c.gemm_scratch_bytes))) break;
    if ((rc = zgemm(c, gemm_args(OP_C, OP_N, kr, kr, kr, one, T, nb, Ys, nb, zero, Zs, nb), nullptr, 0))) break;
    if ((rc = zgemm(c, gemm_args(OP_N, OP_N, mp, kr, kr, mk(-0.5, 0), V, n, Zs, nb, one, X, n), nullptr, 0))) break;
    // A22 -= [V X] [X V]^H (lower triangle), one contraction of 2 kr
    GBHE_CUDA(cudaMemcpy2DAsync(V2c, sizeof(cplx) * n, V, sizeof(cplx) * n, sizeof(cplx) * mp, kr,
                                cudaMemcpyDeviceToDevice, c.st));
    if (k + 2 * nb < n) {
      // the next panel's nb columns first, then its QR on the panel stream
      // beside the update of the remaining columns
      if ((rc = zgemm(c, gemm_args(OP_N, OP_C, mp, nb, 2 * kr, mone, V, n, X, n, one, A22, lda, 1), nullptr, 0)))
        break;
      if ((rc = panel(k + nb, VXVb[(p + 1) & 1]))) break;
      if ((rc = zgemm(c, gemm_args(OP_N, OP_C, mp - nb, mp - nb, 2 * kr, mone, V + nb, n, X + nb, n, one,
                                   A22 + nb + (size_t)nb * lda, lda, 1), nullptr, 0)))
        break;
    } else {
      if ((rc = zgemm(c, gemm_args(OP_N, OP_C, mp, mp, 2 * kr, mone, V, n, X, n, one, A22, lda, 1), nullptr, 0)))
        break;
    }
  }
  // the caller's stream joins every panel it started (also on an early return)
  if (pending) cudaStreamWaitEvent(c.st, c.ev_b, 0);
  a.off = save;
  return rc;
}

}  // namespace gbhe
