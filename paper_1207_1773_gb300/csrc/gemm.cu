// gemm.cu -- FP64 tensor-core GEMM (DMMA: mma.sync.aligned.m16n8k4 .f64).
//
// One CTA of 128 threads computes a 64x64 tile of C; each of its 4 warps a
// 32x32 sub-tile as 2 x 4 MMA tiles of 16x8.  Operand tiles (64 x 16) are
// staged into shared memory with cp.async in a 3-stage pipeline; the copy
// addressing absorbs the operand mode (N, T, conjugate-transpose, Hermitian
// read from its lower triangle), so shared memory always holds op(A) as
// [k][row] and op(B) as [k][col] (complex elements interleaved), and the
// conjugations are applied as sign flips (integer ops, off the FP64 pipe)
// when fragments are read.  A complex product is 4 real MMAs,
//   Cre += Are Bre - Aim Bim,   Cim += Are Bim + Aim Bre,
// issued phase by phase so that consecutive MMAs never depend on each other.
// Row pitch 66 (complex) / 68 (real) makes the fragment loads of every
// quarter-warp (16-byte) or half-warp (8-byte) hit distinct banks.
#include <algorithm>
#include "internal.cuh"

namespace gbhe {
namespace {

constexpr int BM = 64, BN = 64, BK = 16, NT = 128, NSTAGE = 3;

template <bool CPLX> struct Elem { typedef double2 T; static constexpr int LDS = BM + 2; };
template <> struct Elem<false> { typedef double T; static constexpr int LDS = BM + 4; };

template <bool CPLX>
__host__ __device__ constexpr int stage_elems() { return 2 * BK * Elem<CPLX>::LDS; }
template <bool CPLX>
__host__ __device__ constexpr size_t smem_bytes() { return (size_t)NSTAGE * stage_elems<CPLX>() * sizeof(typename Elem<CPLX>::T); }

__device__ __forceinline__ void dmma(double (&c)[4], double a0, double a1, double b0) {
  asm("mma.sync.aligned.m16n8k4.row.col.f64.f64.f64.f64 {%0,%1,%2,%3}, {%4,%5}, {%6}, {%0,%1,%2,%3};"
      : "+d"(c[0]), "+d"(c[1]), "+d"(c[2]), "+d"(c[3])
      : "d"(a0), "d"(a1), "d"(b0));
}

__device__ __forceinline__ double neg(double x) {
  return __longlong_as_double(__double_as_longlong(x) ^ (long long)0x8000000000000000ull);
}

template <int BYTES>
__device__ __forceinline__ void cp_async(void* smem, const void* gmem, bool pred) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  const int sz = pred ? BYTES : 0;
  if (BYTES == 16)
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(s), "l"(gmem), "r"(sz) : "memory");
  else
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;" ::"r"(s), "l"(gmem), "r"(sz) : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

// Issue the copies of op(A)(m0:m0+64, k0:k0+16) and op(B)(k0:k0+16, n0:n0+64)
// into one stage: As[kk][r], Bs[kk][c].
template <bool CPLX, int OPA, int OPB>
__device__ __forceinline__ void load_stage(const GemmArgs& g, int m0, int n0, int k0, int kend,
                                           typename Elem<CPLX>::T* As, typename Elem<CPLX>::T* Bs) {
  typedef typename Elem<CPLX>::T T;
  constexpr int LDS = Elem<CPLX>::LDS;
  constexpr int BYTES = sizeof(T);
  const T* A = reinterpret_cast<const T*>(g.A);
  const T* B = reinterpret_cast<const T*>(g.B);
  const int t = threadIdx.x;
  // ---- A
  int modeA = OPA;  // OP_H: decide per tile which stored triangle to read
  if (OPA == OP_H) {
    if (m0 >= k0 + BK - 1) modeA = OP_N;
    else if (m0 + BM - 1 < k0) modeA = OP_T;
  }
  if (modeA == OP_N) {
    const int r = t & 63, kb = t >> 6;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const int kk = kb + 2 * i, gr = m0 + r, gk = k0 + kk;
      const bool p = gr < g.m && gk < kend;
      cp_async<BYTES>(As + kk * LDS + r, p ? A + (size_t)gr + (size_t)gk * g.lda : A, p);
    }
  } else if (modeA == OP_T || modeA == OP_C) {
    const int kk = t & 15, rb = t >> 4;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const int r = rb + 8 * i, gr = m0 + r, gk = k0 + kk;
      const bool p = gr < g.m && gk < kend;
      cp_async<BYTES>(As + kk * LDS + r, p ? A + (size_t)gk + (size_t)gr * g.lda : A, p);
    }
  } else {  // Hermitian tile crossing the diagonal: per element
    const int r = t & 63, kb = t >> 6;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const int kk = kb + 2 * i, gr = m0 + r, gk = k0 + kk;
      const bool p = gr < g.m && gk < kend;
      const T* src = (gr >= gk) ? A + (size_t)gr + (size_t)gk * g.lda : A + (size_t)gk + (size_t)gr * g.lda;
      cp_async<BYTES>(As + kk * LDS + r, p ? src : A, p);
    }
  }
  // ---- B
  if (OPB == OP_N) {
    const int kk = t & 15, cb = t >> 4;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const int c = cb + 8 * i, gc = n0 + c, gk = k0 + kk;
      const bool p = gc < g.n && gk < kend;
      cp_async<BYTES>(Bs + kk * LDS + c, p ? B + (size_t)gk + (size_t)gc * g.ldb : B, p);
    }
  } else {
    const int c = t & 63, kb = t >> 6;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const int kk = kb + 2 * i, gc = n0 + c, gk = k0 + kk;
      const bool p = gc < g.n && gk < kend;
      cp_async<BYTES>(Bs + kk * LDS + c, p ? B + (size_t)gc + (size_t)gk * g.ldb : B, p);
    }
  }
}

// 64x64 tile (m0, n0) of op(A) op(B) over k in [kbeg, kend); epilogue into C
// (alpha acc + beta C, optional column map / lower-only) or raw partial sums.
template <bool CPLX, int OPA, int OPB>
__device__ __forceinline__ void gemm_tile(const GemmArgs& g, int m0, int n0, int kbeg, int kend, cplx* partial,
                                          const int* cmap) {
  typedef typename Elem<CPLX>::T T;
  constexpr int LDS = Elem<CPLX>::LDS;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* sm = reinterpret_cast<T*>(smem_raw);
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

  const int ktiles = (kend > kbeg) ? (kend - kbeg + BK - 1) / BK : 0;
#pragma unroll
  for (int s = 0; s < NSTAGE - 1; ++s) {
    if (s < ktiles)
      load_stage<CPLX, OPA, OPB>(g, m0, n0, kbeg + s * BK, kend, sm + s * stage_elems<CPLX>(),
                                 sm + s * stage_elems<CPLX>() + BK * LDS);
    cp_commit();
  }
  for (int kt = 0; kt < ktiles; ++kt) {
    cp_wait<NSTAGE - 2>();
    __syncthreads();
    {
      const int ks = kt + NSTAGE - 1;
      const int st = ks % NSTAGE;
      if (ks < ktiles)
        load_stage<CPLX, OPA, OPB>(g, m0, n0, kbeg + ks * BK, kend, sm + st * stage_elems<CPLX>(),
                                   sm + st * stage_elems<CPLX>() + BK * LDS);
      cp_commit();
    }
    const T* As = sm + (kt % NSTAGE) * stage_elems<CPLX>();
    const T* Bs = As + BK * LDS;
    const int k0 = kbeg + kt * BK;
#pragma unroll
    for (int ks = 0; ks < BK / 4; ++ks) {
      const int kk = ks * 4 + tq;
      double ar[2][2], ai[2][2], br[4], bi[4];
#pragma unroll
      for (int mt = 0; mt < 2; ++mt)
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const int r = wm + mt * 16 + gq + 8 * h;
          if (CPLX) {
            const double2 v = *reinterpret_cast<const double2*>(As + kk * LDS + r);
            double im = v.y;
            if (OPA == OP_C) im = neg(im);
            if (OPA == OP_H) {
              const int gr = m0 + r, gk = k0 + kk;
              if (gr < gk) im = neg(im);
              if (gr == gk) im = 0.0;
            }
            ar[mt][h] = v.x;
            ai[mt][h] = im;
          } else {
            ar[mt][h] = *reinterpret_cast<const double*>(As + kk * LDS + r);
            ai[mt][h] = 0.0;
          }
        }
#pragma unroll
      for (int nt = 0; nt < 4; ++nt) {
        const int c = wn + nt * 8 + gq;
        if (CPLX) {
          const double2 v = *reinterpret_cast<const double2*>(Bs + kk * LDS + c);
          br[nt] = v.x;
          bi[nt] = (OPB == OP_C) ? neg(v.y) : v.y;
        } else {
          br[nt] = *reinterpret_cast<const double*>(Bs + kk * LDS + c);
          bi[nt] = 0.0;
        }
      }
#pragma unroll
      for (int mt = 0; mt < 2; ++mt)
#pragma unroll
        for (int nt = 0; nt < 4; ++nt) dmma(accr[mt][nt], ar[mt][0], ar[mt][1], br[nt]);
      if (CPLX) {
#pragma unroll
        for (int mt = 0; mt < 2; ++mt)
#pragma unroll
          for (int nt = 0; nt < 4; ++nt) dmma(acci[mt][nt], ar[mt][0], ar[mt][1], bi[nt]);
        double nai[2][2];
#pragma unroll
        for (int mt = 0; mt < 2; ++mt) { nai[mt][0] = neg(ai[mt][0]); nai[mt][1] = neg(ai[mt][1]); }
#pragma unroll
        for (int mt = 0; mt < 2; ++mt)
#pragma unroll
          for (int nt = 0; nt < 4; ++nt) dmma(accr[mt][nt], nai[mt][0], nai[mt][1], bi[nt]);
#pragma unroll
        for (int mt = 0; mt < 2; ++mt)
#pragma unroll
          for (int nt = 0; nt < 4; ++nt) dmma(acci[mt][nt], ai[mt][0], ai[mt][1], br[nt]);
      }
    }
  }
  cp_wait<0>();

  // ---- epilogue
  const bool beta0 = (g.beta.x == 0.0 && g.beta.y == 0.0);
  const bool beta1 = (g.beta.x == 1.0 && g.beta.y == 0.0);
  const bool alpha1 = (g.alpha.x == 1.0 && g.alpha.y == 0.0);
  const bool alpham1 = (g.alpha.x == -1.0 && g.alpha.y == 0.0);
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
        cplx out;
        if (alpha1) out = acc;
        else if (alpham1) out = mk(neg(acc.x), neg(acc.y));
        else out = cmul(g.alpha, acc);
        if (CPLX) {
          cplx* C = reinterpret_cast<cplx*>(g.C);
          if (beta1) out = cadd(out, C[idx]);
          else if (!beta0) out = cadd(out, cmul(g.beta, C[idx]));
          C[idx] = out;
        } else {
          double* C = reinterpret_cast<double*>(g.C);
          double o = out.x;
          if (beta1) o += C[idx];
          else if (!beta0) o += g.beta.x * C[idx];
          C[idx] = o;
        }
      }
}

template <bool CPLX, int OPA, int OPB>
__global__ void __launch_bounds__(NT, 2) k_gemm(GemmArgs g, int kchunk, cplx* partial) {
  const int m0 = blockIdx.x * BM, n0 = blockIdx.y * BN;
  if (g.lower_only && m0 + BM - 1 < n0) return;  // tile strictly above the diagonal
  const int kbeg = blockIdx.z * kchunk;
  const int kend = min(g.k, kbeg + kchunk);
  cplx* p = partial ? partial + (size_t)blockIdx.z * g.m * g.n : nullptr;
  gemm_tile<CPLX, OPA, OPB>(g, m0, n0, kbeg, kend, p, nullptr);
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

__global__ void __launch_bounds__(NT, 2) k_dgemm_grouped(const DGroupDesc* desc, double alpha, double beta) {
  const DGroupDesc d = desc[blockIdx.z];
  const int m0 = blockIdx.x * BM, n0 = blockIdx.y * BN;
  if (m0 >= d.m || n0 >= d.n) return;
  GemmArgs g;
  g.opA = OP_N; g.opB = OP_N; g.m = d.m; g.n = d.n; g.k = d.k;
  g.alpha = mk(alpha, 0.0); g.beta = mk(beta, 0.0);
  g.A = d.A; g.lda = d.lda; g.B = d.B; g.ldb = d.ldb; g.C = d.C; g.ldc = d.ldc;
  g.lower_only = 0;
  gemm_tile<false, OP_N, OP_N>(g, m0, n0, 0, d.k, nullptr, d.cmap);
}

template <bool CPLX, int OPA, int OPB>
int launch_mode(cudaStream_t st, dim3 grid, const GemmArgs& g, int kchunk, cplx* partial) {
  static bool attr[MAX_DEVICES] = {};
  const int dev = device_slot();
  if (dev < 0) return GBHE_ECUDA;
  if (!attr[dev]) {
    if (cudaFuncSetAttribute(k_gemm<CPLX, OPA, OPB>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem_bytes<CPLX>()) != cudaSuccess)
      return GBHE_ECUDA;
    attr[dev] = true;
  }
  k_gemm<CPLX, OPA, OPB><<<grid, NT, smem_bytes<CPLX>(), st>>>(g, kchunk, partial);
  count_launch();
  return 0;
}

template <bool CPLX, int OPA>
int dispatch_b(cudaStream_t st, dim3 grid, const GemmArgs& g, int kchunk, cplx* partial) {
  switch (g.opB) {
    case OP_N: return launch_mode<CPLX, OPA, OP_N>(st, grid, g, kchunk, partial);
    case OP_T: return launch_mode<CPLX, OPA, OP_T>(st, grid, g, kchunk, partial);
    default: return launch_mode<CPLX, OPA, OP_C>(st, grid, g, kchunk, partial);
  }
}

template <bool CPLX>
int dispatch(cudaStream_t st, dim3 grid, const GemmArgs& g, int kchunk, cplx* partial) {
  switch (g.opA) {
    case OP_N: return dispatch_b<CPLX, OP_N>(st, grid, g, kchunk, partial);
    case OP_T: return dispatch_b<CPLX, OP_T>(st, grid, g, kchunk, partial);
    case OP_C: return dispatch_b<CPLX, OP_C>(st, grid, g, kchunk, partial);
    default: return dispatch_b<CPLX, OP_H>(st, grid, g, kchunk, partial);
  }
}

template <bool CPLX>
int gemm_launch(cudaStream_t st, const GemmArgs& g, void* scratch, size_t scratch_bytes) {
  if (g.m <= 0 || g.n <= 0) return 0;
  int rc;
  if (g.k <= 0) {  // C = beta C: one pass with an empty K loop
    GemmArgs h = g;
    h.k = 0;
    dim3 grid((g.m + BM - 1) / BM, (g.n + BN - 1) / BN, 1);
    if ((rc = dispatch<CPLX>(st, grid, h, 1, nullptr))) return rc;
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
    if ((rc = dispatch<CPLX>(st, dim3(tm, tn, 1), g, g.k, nullptr))) return rc;
  } else {
    int kchunk = (g.k + nsplit - 1) / nsplit;
    kchunk = (kchunk + BK - 1) / BK * BK;
    nsplit = (g.k + kchunk - 1) / kchunk;
    GemmArgs h = g;
    h.lower_only = 0;
    if ((rc = dispatch<CPLX>(st, dim3(tm, tn, nsplit), h, kchunk, reinterpret_cast<cplx*>(scratch)))) return rc;
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
  static bool attr[MAX_DEVICES] = {};
  const int dev = device_slot();
  if (dev < 0) return GBHE_ECUDA;
  if (!attr[dev]) {
    if (cudaFuncSetAttribute(k_dgemm_grouped, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem_bytes<false>()) != cudaSuccess)
      return GBHE_ECUDA;
    attr[dev] = true;
  }
  dim3 grid((max_m + BM - 1) / BM, (max_n + BN - 1) / BN, ngroups);
  ProfScope prof(st, GBHE_PROF_DGEMM, 0.0, 0.0);  // sizes live on the device
  k_dgemm_grouped<<<grid, NT, smem_bytes<false>(), st>>>(d_desc, alpha, beta);
  count_launch();
  return cudaGetLastError() == cudaSuccess ? 0 : GBHE_ECUDA;
}

}  // namespace gbhe
