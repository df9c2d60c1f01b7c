// hb2st.cu -- second stage of the two-stage tridiagonalisation (paper Section
// 4.2): Hermitian band (half-bandwidth nb) -> real symmetric tridiagonal by
// bulge chasing with column-wise elimination.
//
// Sweep s (s = 0..n-2) annihilates column s below the sub-diagonal and chases
// the resulting bulge down the band in steps j = 0, 1, ...  With
// R_j = [s+1+j*nb, s+1+(j+1)*nb) ∩ [0, n):
//   step 0: reflector H_0 from A[R_0, s] (H_0^H x = beta e_1, beta real);
//           A[R_0, R_0] <- H_0^H A[R_0, R_0] H_0.
//   step j: E = A[R_j, R_{j-1}] <- E H_{j-1}          (creates the bulge)
//           H_j from the first column of E; E <- H_j^H E (column 0 -> beta e_1)
//           A[R_j, R_j] <- H_j^H A[R_j, R_j] H_j.
// Only the first column of each bulge is annihilated; what is left of it lies
// inside the columns that the next sweeps eliminate, so the working band needs
// 2*nb sub-diagonals.  Step (s, j) overlaps step (s-1, j+1) and nothing later
// of sweep s-1, so sweep s may run step j once sweep s-1 has finished step
// j+1: the sweeps are pipelined over persistent CTAs (sweep s on CTA s mod G),
// handed over through per-sweep progress counters with bounded waits.
#include <algorithm>
#include "internal.cuh"

namespace gbhe {
namespace {

constexpr int HT = 128;
constexpr int MAXNB = 128;

struct ChaseArgs {
  cplx* WB;       // working band, ld = ldb = 2*nb+1:  WB[(r-c) + c*ldb], 0 <= r-c <= 2nb
  int ldb, n, nb, J;
  cplx* V2;       // (s*J + j)*nb
  cplx* tau2;     // s*J + j
  int* progress;  // n
  int* st;
};

__device__ __forceinline__ cplx* bat(const ChaseArgs& a, int r, int c) {
  return a.WB + (size_t)(r - c) + (size_t)c * a.ldb;
}
__device__ __forceinline__ cplx ldb_(const cplx* p) { return __ldcg(p); }
__device__ __forceinline__ void stb_(cplx* p, cplx v) { __stcg(p, v); }

__device__ __forceinline__ cplx warp_sum(cplx v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    v.x += __shfl_xor_sync(0xffffffffu, v.x, o);
    v.y += __shfl_xor_sync(0xffffffffu, v.y, o);
  }
  return v;
}

// Reflector from x[0..len) held in smem `x`: on return x = v (v[0] = 1),
// returns tau, writes beta to *beta.
__device__ void make_reflector(cplx* x, int len, cplx* tau_out, double* beta_out, cplx* red) {
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  double s = 0.0;
  for (int i = 1 + t; i < len; i += HT) s += cabs2(x[i]);
  cplx sv = warp_sum(mk(s, 0.0));
  __syncthreads();
  if (lane == 0) red[warp] = sv;
  __syncthreads();
  __shared__ cplx sh_scal;
  if (t == 0) {
    double xn2 = 0.0;
    for (int w = 0; w < HT / 32; ++w) xn2 += red[w].x;
    cplx al = x[0];
    if (xn2 == 0.0 && al.y == 0.0) {
      *tau_out = mk(0.0, 0.0); *beta_out = al.x; sh_scal = mk(0.0, 0.0);
    } else {
      double nrm = sqrt(al.x * al.x + al.y * al.y + xn2);
      double beta = (al.x >= 0.0) ? -nrm : nrm;
      *beta_out = beta;
      *tau_out = mk((beta - al.x) / beta, -al.y / beta);
      sh_scal = cinv(mk(al.x - beta, al.y));
    }
  }
  __syncthreads();
  const cplx sc = sh_scal;
  for (int i = 1 + t; i < len; i += HT) x[i] = cmul(x[i], sc);
  __syncthreads();
  if (t == 0) x[0] = mk(1.0, 0.0);
  __syncthreads();
}

// D <- H^H D H for the Hermitian block D = A[a0:a0+L, a0:a0+L] (lower stored).
__device__ void two_sided(const ChaseArgs& A, int a0, int L, const cplx* v, cplx tau, cplx* p,
                          cplx* red) {
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  // p = tau * D v
  for (int r = t; r < L; r += HT) {
    cplx acc = mk(0.0, 0.0);
    for (int c = 0; c < L; ++c) {
      cplx d = (r >= c) ? ldb_(bat(A, a0 + r, a0 + c)) : cconj(ldb_(bat(A, a0 + c, a0 + r)));
      if (r == c) d.y = 0.0;
      cfma(acc, d, v[c]);
    }
    p[r] = cmul(tau, acc);
  }
  __syncthreads();
  // alpha = -1/2 tau (p^H v);  w = p + alpha v
  cplx pv = mk(0.0, 0.0);
  for (int r = t; r < L; r += HT) ccfma(pv, p[r], v[r]);
  pv = warp_sum(pv);
  if (lane == 0) red[warp] = pv;
  __syncthreads();
  __shared__ cplx sh_alpha;
  if (t == 0) {
    cplx s = mk(0.0, 0.0);
    for (int w = 0; w < HT / 32; ++w) s = cadd(s, red[w]);
    sh_alpha = cscal(-0.5, cmul(tau, s));
  }
  __syncthreads();
  for (int r = t; r < L; r += HT) p[r] = cadd(p[r], cmul(sh_alpha, v[r]));
  __syncthreads();
  // D -= v w^H + w v^H (lower)
  for (int i = t; i < L * L; i += HT) {
    int r = i % L, c = i / L;
    if (r < c) continue;
    cplx* q = bat(A, a0 + r, a0 + c);
    cplx d = ldb_(q);
    cplx u = cadd(cmulc(v[r], p[c]), cmulc(p[r], v[c]));
    d = csub(d, u);
    if (r == c) d.y = 0.0;
    stb_(q, d);
  }
  __syncthreads();
}

__global__ void __launch_bounds__(HT) k_chase(ChaseArgs A) {
  __shared__ cplx vprev[MAXNB], vcur[MAXNB], y[MAXNB], p[MAXNB];
  __shared__ cplx red[HT / 32];
  __shared__ cplx sh_tau;
  __shared__ double sh_beta;
  __shared__ int sh_ok;
  const int t = threadIdx.x, n = A.n, nb = A.nb;
  for (int s = blockIdx.x; s <= n - 2; s += gridDim.x) {
    const int ntask = (n - 1 - s + nb - 1) / nb;
    const int ntask_prev = (s > 0) ? (n - 1 - (s - 1) + nb - 1) / nb : 0;
    cplx tprev = mk(0.0, 0.0);
    int Lprev = 0;
    for (int j = 0; j < ntask; ++j) {
      // wait for sweep s-1 to finish step j+1
      if (s > 0) {
        if (t == 0) {
          const int need = min(j + 2, ntask_prev);
          const unsigned long long t0 = gtimer();
          int ok = 1;
          while (ld_acquire_i(&A.progress[s - 1]) < need) {
            if (gtimer() - t0 > GBHE_WAIT_NS || ld_acquire_i(&A.st[ST_ERR]) != 0) {
              set_err_once(A.st, GBHE_ETIMEOUT);
              ok = 0;
              break;
            }
            __nanosleep(32);
          }
          sh_ok = ok;
        }
        __syncthreads();
        if (!sh_ok) return;
      }
      const int a0 = s + 1 + j * nb;
      const int L = min(nb, n - a0);
      if (j == 0) {
        for (int i = t; i < L; i += HT) vcur[i] = ldb_(bat(A, a0 + i, s));
        __syncthreads();
        make_reflector(vcur, L, &sh_tau, &sh_beta, red);
        for (int i = t; i < L; i += HT) stb_(bat(A, a0 + i, s), i == 0 ? mk(sh_beta, 0.0) : mk(0.0, 0.0));
      } else {
        const int c0 = a0 - nb;  // first column of R_{j-1}
        // E <- E H_{j-1}:  y = E vprev;  E -= tau_prev y vprev^H
        for (int r = t; r < L; r += HT) {
          cplx acc = mk(0.0, 0.0);
          for (int c = 0; c < Lprev; ++c) cfma(acc, ldb_(bat(A, a0 + r, c0 + c)), vprev[c]);
          y[r] = cmul(tprev, acc);
        }
        __syncthreads();
        for (int i = t; i < L * Lprev; i += HT) {
          int r = i % L, c = i / L;
          cplx* q = bat(A, a0 + r, c0 + c);
          stb_(q, csub(ldb_(q), cmulc(y[r], vprev[c])));
        }
        __syncthreads();
        // new reflector from column 0 of E
        for (int i = t; i < L; i += HT) vcur[i] = ldb_(bat(A, a0 + i, c0));
        __syncthreads();
        make_reflector(vcur, L, &sh_tau, &sh_beta, red);
        for (int i = t; i < L; i += HT) stb_(bat(A, a0 + i, c0), i == 0 ? mk(sh_beta, 0.0) : mk(0.0, 0.0));
        // E[:, 1:] <- H^H E[:, 1:]:  z_c = v^H E[:, c];  E[:, c] -= conj(tau) v z_c
        const cplx ct = cconj(sh_tau);
        for (int c = 1 + t; c < Lprev; c += HT) {
          cplx acc = mk(0.0, 0.0);
          for (int r = 0; r < L; ++r) ccfma(acc, vcur[r], ldb_(bat(A, a0 + r, c0 + c)));
          y[c] = cmul(ct, acc);
        }
        __syncthreads();
        for (int i = t; i < L * Lprev; i += HT) {
          int r = i % L, c = i / L;
          if (c == 0) continue;
          cplx* q = bat(A, a0 + r, c0 + c);
          stb_(q, csub(ldb_(q), cmul(vcur[r], y[c])));
        }
        __syncthreads();
      }
      // store the reflector
      cplx* vout = A.V2 + ((size_t)s * A.J + j) * nb;
      for (int i = t; i < nb; i += HT) vout[i] = (i < L) ? vcur[i] : mk(0.0, 0.0);
      if (t == 0) A.tau2[(size_t)s * A.J + j] = sh_tau;
      // two-sided update of the diagonal block
      two_sided(A, a0, L, vcur, sh_tau, p, red);
      // publish progress, keep H_j for the next step
      if (t == 0) {
        __threadfence();
        st_release_i(&A.progress[s], j + 1);
      }
      for (int i = t; i < L; i += HT) vprev[i] = vcur[i];
      tprev = sh_tau;
      Lprev = L;
      __syncthreads();
    }
  }
}

// Copy the lower band of A into the working band (2nb extra sub-diagonals zeroed).
__global__ void k_band_in(const cplx* A, int lda, int n, int nb, cplx* WB, int ldb) {
  const size_t total = (size_t)ldb * n;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total;
       i += (size_t)gridDim.x * blockDim.x) {
    int dr = (int)(i % ldb), c = (int)(i / ldb), r = c + dr;
    cplx v = mk(0.0, 0.0);
    if (dr <= nb && r < n) v = A[(size_t)r + (size_t)c * lda];
    if (dr == 0) v.y = 0.0;
    WB[i] = v;
  }
}

__global__ void k_band_out(const cplx* WB, int ldb, int n, double* d, double* e) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    d[i] = WB[(size_t)i * ldb].x;
    if (i + 1 < n) e[i] = WB[1 + (size_t)i * ldb].x;
  }
}

}  // namespace

size_t hb2st_ws_bytes(int n, int nb) {
  return (size_t)(2 * nb + 1) * std::max(n, 1) * sizeof(cplx) + (size_t)std::max(n, 1) * sizeof(int) + 512;
}

int hb2st_run(Ctx& c, int n, int nb, const cplx* A, int lda, double* d, double* e, cplx* V2, cplx* tau2) {
  if (n <= 0) return 0;
  if (nb < 1 || nb > MAXNB) return -3;
  Arena& a = c.arena;
  const size_t save = a.off;
  const int ldb = 2 * nb + 1;
  cplx* WB = a.take<cplx>((size_t)ldb * n);
  int* prog = a.take<int>(n);
  if (!a.ok() || !WB) { a.off = save; return GBHE_EWORKSPACE; }
  const int J = hb2st_J(n, nb);
  k_band_in<<<std::min<size_t>(((size_t)ldb * n + 255) / 256, 4096), 256, 0, c.st>>>(A, lda, n, nb, WB, ldb);
  count_launch();
  GBHE_CUDA(cudaGetLastError());
  GBHE_CUDA(cudaMemsetAsync(prog, 0, sizeof(int) * n, c.st));
  if (n >= 2) {
    ChaseArgs ca;
    ca.WB = WB; ca.ldb = ldb; ca.n = n; ca.nb = nb; ca.J = J; ca.V2 = V2; ca.tau2 = tau2;
    ca.progress = prog; ca.st = c.status;
    const int G = std::min(c.num_sms, n - 1);
    void* args[] = {&ca};
    count_launch();
    double fl = 0.0;
    if (prof_on()) {
      // per step: E H (2 L Lp), H^H E (2 L (Lp-1)), two-sided (2 L^2) complex multiply-adds
      for (int s = 0; s <= n - 2; ++s) {
        int Lp = 0;
        for (int a0 = s + 1; a0 < n; a0 += nb) {
          const int L = std::min(nb, n - a0);
          fl += 8.0 * (2.0 * L * Lp + 2.0 * L * std::max(Lp - 1, 0) + 2.0 * L * L);
          Lp = L;
        }
      }
    }
    const double by = 16.0 * ((double)n * J * nb + 2.0 * ldb * n);
    ProfScope prof(c.st, GBHE_PROF_CHASE, fl, by);
    GBHE_CUDA(cudaLaunchCooperativeKernel((const void*)k_chase, dim3(G), dim3(HT), args, 0, c.st));
  }
  k_band_out<<<std::min((n + 255) / 256, 1024), 256, 0, c.st>>>(WB, ldb, n, d, e);
  count_launch();
  GBHE_CUDA(cudaGetLastError());
  a.off = save;
  return 0;
}

}  // namespace gbhe
