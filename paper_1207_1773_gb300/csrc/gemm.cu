// gemm.cu -- FP64 tensor-core GEMM (DMMA: mma.sync.aligned.m16n8k4 .f64).
//
// One CTA of 128 threads computes a 64x64 tile of C; each of its 4 warps a
// 32x32 sub-tile as 2 x 4 MMA tiles of 16x8.  A complex product is 4 real
// MMAs on de-interleaved (re, im) planes staged in shared memory:
//   Cre += Are Bre - Aim Bim,   Cim += Are Bim + Aim Bre.
// The next K-tile is fetched into registers while the current one is
// multiplied (register double buffering).  Shared-memory rows are padded to
// 68 doubles so that the fragment loads of a half-warp hit 16 distinct banks.
#include <algorithm>
#include "internal.cuh"

namespace gbhe {
namespace {

constexpr int BM = 64, BN = 64, BK = 16, LDS = BM + 4, NT = 128;

__device__ __forceinline__ void dmma(double (&c)[4], double a0, double a1, double b0) {
  asm volatile(
      "mma.sync.aligned.m16n8k4.row.col.f64.f64.f64.f64 {%0,%1,%2,%3}, {%4,%5}, {%6}, "
      "{%0,%1,%2,%3};"
      : "+d"(c[0]), "+d"(c[1]), "+d"(c[2]), "+d"(c[3])
      : "d"(a0), "d"(a1), "d"(b0));
}

template <bool CPLX>
__device__ __forceinline__ cplx ldv(const void* p, size_t idx) {
  if (CPLX) return reinterpret_cast<const cplx*>(p)[idx];
  return mk(reinterpret_cast<const double*>(p)[idx], 0.0);
}

// Fetch this thread's 8 elements of op(A)(m0:m0+64, k0:k0+16) into regs and
// record their (row, k) positions in the tile.
template <bool CPLX>
__device__ __forceinline__ void fetch_A(const GemmArgs& g, int m0, int k0, int kend, cplx (&v)[8],
                                        unsigned char (&pr)[8], unsigned char (&pk)[8]) {
  const int t = threadIdx.x;
  if (g.opA == OP_T || g.opA == OP_C) {
    const int kk = t & 15, rb = t >> 4;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      int r = rb + 8 * i, gr = m0 + r, gk = k0 + kk;
      cplx x = mk(0.0, 0.0);
      if (gr < g.m && gk < kend) x = ldv<CPLX>(g.A, (size_t)gk + (size_t)gr * g.lda);
      if (g.opA == OP_C) x.y = -x.y;
      v[i] = x; pr[i] = (unsigned char)r; pk[i] = (unsigned char)kk;
    }
  } else {
    const int r = t & 63, kb = t >> 6;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      int kk = kb + 2 * i, gr = m0 + r, gk = k0 + kk;
      cplx x = mk(0.0, 0.0);
      if (gr < g.m && gk < kend) {
        if (g.opA == OP_N || gr > gk) {
          x = ldv<CPLX>(g.A, (size_t)gr + (size_t)gk * g.lda);
        } else if (gr == gk) {
          x = ldv<CPLX>(g.A, (size_t)gr + (size_t)gk * g.lda);
          x.y = 0.0;
        } else {
          x = ldv<CPLX>(g.A, (size_t)gk + (size_t)gr * g.lda);
          x.y = -x.y;
        }
      }
      v[i] = x; pr[i] = (unsigned char)r; pk[i] = (unsigned char)kk;
    }
  }
}

template <bool CPLX>
__device__ __forceinline__ void fetch_B(const GemmArgs& g, int n0, int k0, int kend, cplx (&v)[8],
                                        unsigned char (&pc)[8], unsigned char (&pk)[8]) {
  const int t = threadIdx.x;
  if (g.opB == OP_N) {
    const int kk = t & 15, cb = t >> 4;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      int c = cb + 8 * i, gc = n0 + c, gk = k0 + kk;
      cplx x = mk(0.0, 0.0);
      if (gc < g.n && gk < kend) x = ldv<CPLX>(g.B, (size_t)gk + (size_t)gc * g.ldb);
      v[i] = x; pc[i] = (unsigned char)c; pk[i] = (unsigned char)kk;
    }
  } else {
    const int c = t & 63, kb = t >> 6;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      int kk = kb + 2 * i, gc = n0 + c, gk = k0 + kk;
      cplx x = mk(0.0, 0.0);
      if (gc < g.n && gk < kend) x = ldv<CPLX>(g.B, (size_t)gc + (size_t)gk * g.ldb);
      if (g.opB == OP_C) x.y = -x.y;
      v[i] = x; pc[i] = (unsigned char)c; pk[i] = (unsigned char)kk;
    }
  }
}

// Computes the 64x64 tile (m0, n0) of alpha*op(A)op(B) over k in [kbeg, kend)
// and either stores alpha*acc + beta*C into C (partial == nullptr) or the raw
// sum into `partial` (ld = g.m).
template <bool CPLX>
__device__ __forceinline__ void gemm_tile(const GemmArgs& g, int m0, int n0, int kbeg, int kend,
                                          cplx* partial, const int* cmap = nullptr) {
  constexpr int NP = CPLX ? 2 : 1;
  __shared__ double As[NP][BK][LDS];
  __shared__ double Bs[NP][BK][LDS];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int gq = lane >> 2, tq = lane & 3;
  const int wm = (w & 1) * 32, wn = (w >> 1) * 32;

  double accr[2][4][4], acci[2][4][4];
#pragma unroll
  for (int a = 0; a < 2; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b)
#pragma unroll
      for (int c = 0; c < 4; ++c) { accr[a][b][c] = 0.0; acci[a][b][c] = 0.0; }

  cplx va[8], vb[8];
  unsigned char ar[8], ak[8], bc[8], bk[8];
  if (kbeg < kend) {
    fetch_A<CPLX>(g, m0, kbeg, kend, va, ar, ak);
    fetch_B<CPLX>(g, n0, kbeg, kend, vb, bc, bk);
  }
  for (int k0 = kbeg; k0 < kend; k0 += BK) {
    __syncthreads();
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      As[0][ak[i]][ar[i]] = va[i].x;
      Bs[0][bk[i]][bc[i]] = vb[i].x;
      if (CPLX) {
        As[NP - 1][ak[i]][ar[i]] = va[i].y;
        Bs[NP - 1][bk[i]][bc[i]] = vb[i].y;
      }
    }
    __syncthreads();
    if (k0 + BK < kend) {
      fetch_A<CPLX>(g, m0, k0 + BK, kend, va, ar, ak);
      fetch_B<CPLX>(g, n0, k0 + BK, kend, vb, bc, bk);
    }
#pragma unroll
    for (int ks = 0; ks < BK / 4; ++ks) {
      const int kk = ks * 4 + tq;
      double fr[2][2], fi[2][2], gr_[4], gi[4];
#pragma unroll
      for (int mt = 0; mt < 2; ++mt) {
        const int r = wm + mt * 16 + gq;
        fr[mt][0] = As[0][kk][r];
        fr[mt][1] = As[0][kk][r + 8];
        if (CPLX) { fi[mt][0] = As[NP - 1][kk][r]; fi[mt][1] = As[NP - 1][kk][r + 8]; }
      }
#pragma unroll
      for (int nt = 0; nt < 4; ++nt) {
        const int c = wn + nt * 8 + gq;
        gr_[nt] = Bs[0][kk][c];
        if (CPLX) gi[nt] = Bs[NP - 1][kk][c];
      }
#pragma unroll
      for (int mt = 0; mt < 2; ++mt)
#pragma unroll
        for (int nt = 0; nt < 4; ++nt) {
          dmma(accr[mt][nt], fr[mt][0], fr[mt][1], gr_[nt]);
          if (CPLX) {
            dmma(accr[mt][nt], -fi[mt][0], -fi[mt][1], gi[nt]);
            dmma(acci[mt][nt], fr[mt][0], fr[mt][1], gi[nt]);
            dmma(acci[mt][nt], fi[mt][0], fi[mt][1], gr_[nt]);
          }
        }
    }
  }

  // epilogue
  const bool beta0 = (g.beta.x == 0.0 && g.beta.y == 0.0);
#pragma unroll
  for (int mt = 0; mt < 2; ++mt)
#pragma unroll
    for (int nt = 0; nt < 4; ++nt)
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int r = m0 + wm + mt * 16 + gq + (q >> 1) * 8;
        const int c = n0 + wn + nt * 8 + 2 * tq + (q & 1);
        if (r >= g.m || c >= g.n) continue;
        cplx acc = mk(accr[mt][nt][q], CPLX ? acci[mt][nt][q] : 0.0);
        if (partial) {
          partial[(size_t)r + (size_t)c * g.m] = acc;
          continue;
        }
        if (g.lower_only && r < c) continue;
        const size_t idx = (size_t)r + (size_t)(cmap ? cmap[c] : c) * g.ldc;
        if (CPLX) {
          cplx* C = reinterpret_cast<cplx*>(g.C);
          cplx out = cmul(g.alpha, acc);
          if (!beta0) out = cadd(out, cmul(g.beta, C[idx]));
          C[idx] = out;
        } else {
          double* C = reinterpret_cast<double*>(g.C);
          double out = g.alpha.x * acc.x;
          if (!beta0) out += g.beta.x * C[idx];
          C[idx] = out;
        }
      }
}

template <bool CPLX>
__global__ void __launch_bounds__(NT) k_gemm(GemmArgs g, int kchunk, cplx* partial) {
  const int m0 = blockIdx.x * BM, n0 = blockIdx.y * BN;
  if (g.lower_only && m0 + BM - 1 < n0) return;  // tile strictly above the diagonal
  const int kbeg = blockIdx.z * kchunk;
  const int kend = min(g.k, kbeg + kchunk);
  cplx* p = partial ? partial + (size_t)blockIdx.z * g.m * g.n : nullptr;
  gemm_tile<CPLX>(g, m0, n0, kbeg, kend, p);
}

template <bool CPLX>
__global__ void k_splitk_reduce(GemmArgs g, int nsplit, const cplx* partial) {
  const size_t total = (size_t)g.m * g.n;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total;
       i += (size_t)gridDim.x * blockDim.x) {
    const int r = (int)(i % g.m), c = (int)(i / g.m);
    if (g.lower_only && r < c) continue;
    cplx s = mk(0.0, 0.0);
    for (int z = 0; z < nsplit; ++z) s = cadd(s, partial[(size_t)z * total + i]);
    const size_t idx = (size_t)r + (size_t)c * g.ldc;
    const bool beta0 = (g.beta.x == 0.0 && g.beta.y == 0.0);
    if (CPLX) {
      cplx* C = reinterpret_cast<cplx*>(g.C);
      cplx out = cmul(g.alpha, s);
      if (!beta0) out = cadd(out, cmul(g.beta, C[idx]));
      C[idx] = out;
    } else {
      double* C = reinterpret_cast<double*>(g.C);
      double out = g.alpha.x * s.x;
      if (!beta0) out += g.beta.x * C[idx];
      C[idx] = out;
    }
  }
}

__global__ void __launch_bounds__(NT) k_dgemm_grouped(const DGroupDesc* desc, double alpha,
                                                      double beta) {
  const DGroupDesc d = desc[blockIdx.z];
  const int m0 = blockIdx.x * BM, n0 = blockIdx.y * BN;
  if (m0 >= d.m || n0 >= d.n) return;
  GemmArgs g;
  g.opA = OP_N; g.opB = OP_N; g.m = d.m; g.n = d.n; g.k = d.k;
  g.alpha = mk(alpha, 0.0); g.beta = mk(beta, 0.0);
  g.A = d.A; g.lda = d.lda; g.B = d.B; g.ldb = d.ldb; g.C = d.C; g.ldc = d.ldc;
  g.lower_only = 0;
  gemm_tile<false>(g, m0, n0, 0, d.k, nullptr, d.cmap);
}

template <bool CPLX>
int gemm_launch(cudaStream_t st, const GemmArgs& g, void* scratch, size_t scratch_bytes) {
  if (g.m <= 0 || g.n <= 0) return 0;
  if (g.k <= 0) {
    // C = beta C: run one pass with an empty K loop
    GemmArgs h = g;
    h.k = 0;
    dim3 grid((g.m + BM - 1) / BM, (g.n + BN - 1) / BN, 1);
    k_gemm<CPLX><<<grid, NT, 0, st>>>(h, 1, nullptr);
    count_launch();
    return cudaGetLastError() == cudaSuccess ? 0 : GBHE_ECUDA;
  }
  const int tm = (g.m + BM - 1) / BM, tn = (g.n + BN - 1) / BN;
  // algorithmic flops of this call (lower-only: the lower triangle of a square C)
  const double outs = g.lower_only ? (double)g.n * (g.n + 1) / 2 + (double)(g.m - g.n) * g.n : (double)g.m * g.n;
  const double flops = (CPLX ? 8.0 : 2.0) * outs * g.k;
  const double esz = CPLX ? 16.0 : 8.0;
  const double bytes = esz * ((double)g.m * g.k + (double)g.k * g.n + outs * (g.beta.x != 0.0 || g.beta.y != 0.0 ? 2 : 1));
  ProfScope prof(st, CPLX ? GBHE_PROF_ZGEMM : GBHE_PROF_DGEMM, flops, bytes);
  int nsplit = 1;
  const long tiles = (long)tm * tn;
  if (scratch && tiles < 96 && g.k >= 1024) {
    nsplit = (int)std::min<long>((g.k + 255) / 256, (304 + tiles - 1) / tiles);
    const size_t need = (size_t)nsplit * g.m * g.n * sizeof(cplx);
    if (need > scratch_bytes) nsplit = (int)std::max<size_t>(1, scratch_bytes / ((size_t)g.m * g.n * sizeof(cplx)));
  }
  if (nsplit <= 1) {
    dim3 grid(tm, tn, 1);
    k_gemm<CPLX><<<grid, NT, 0, st>>>(g, g.k, nullptr);
    count_launch();
  } else {
    int kchunk = (g.k + nsplit - 1) / nsplit;
    kchunk = (kchunk + BK - 1) / BK * BK;
    nsplit = (g.k + kchunk - 1) / kchunk;
    dim3 grid(tm, tn, nsplit);
    GemmArgs h = g;
    h.lower_only = 0;
    k_gemm<CPLX><<<grid, NT, 0, st>>>(h, kchunk, reinterpret_cast<cplx*>(scratch));
    count_launch();
    const size_t total = (size_t)g.m * g.n;
    int blocks = (int)std::min<size_t>((total + 255) / 256, 1024);
    k_splitk_reduce<CPLX><<<blocks, 256, 0, st>>>(g, nsplit, reinterpret_cast<const cplx*>(scratch));
    count_launch();
  }
  return cudaGetLastError() == cudaSuccess ? 0 : GBHE_ECUDA;
}

}  // namespace

int zgemm(cudaStream_t st, const GemmArgs& g, void* scratch, size_t scratch_bytes) {
  return gemm_launch<true>(st, g, scratch, scratch_bytes);
}
int dgemm(cudaStream_t st, const GemmArgs& g, void* scratch, size_t scratch_bytes) {
  return gemm_launch<false>(st, g, scratch, scratch_bytes);
}
int dgemm_grouped(cudaStream_t st, const DGroupDesc* d_desc, int ngroups, int max_m, int max_n,
                  double alpha, double beta) {
  if (ngroups <= 0 || max_m <= 0 || max_n <= 0) return 0;
  dim3 grid((max_m + BM - 1) / BM, (max_n + BN - 1) / BN, ngroups);
  ProfScope prof(st, GBHE_PROF_DGEMM, 0.0, 0.0);  // sizes live on the device
  k_dgemm_grouped<<<grid, NT, 0, st>>>(d_desc, alpha, beta);
  count_launch();
  return cudaGetLastError() == cudaSuccess ? 0 : GBHE_ECUDA;
}

}  // namespace gbhe
