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
// j+1: the sweeps are pipelined over persistent CTAs (or CTA clusters),
// handed over through per-sweep progress counters with bounded waits.
//
// Forward progress does not rest on all CTAs being resident at once: a CTA
// (cluster) takes its next sweep from a global ticket counter when it is
// ready, so sweeps are handed out in the order in which running CTAs ask for
// them.  The holder of sweep s-1 took its ticket earlier and is therefore
// already running; it waits only on sweep s-2, and sweep 0 waits on nothing,
// so the chain always advances whatever the number of co-resident CTAs (an
// ordinary launch: no cooperative or co-scheduling guarantee is needed).
#include <algorithm>
#include <cooperative_groups.h>
#include "internal.cuh"

namespace cg = cooperative_groups;

namespace gbhe {
namespace {

constexpr int HT = 256;     // threads per CTA
constexpr int MAXNB = 64;   // largest band width of the shared-memory chase
constexpr int LDS = MAXNB + 1;  // smem column pitch (complex elements)

struct ChaseArgs {
  cplx* WB;       // working band, ld = ldb = 2*nb+1:  WB[(r-c) + c*ldb], 0 <= r-c <= 2nb
  int ldb, n, nb, J;
  cplx* V2;       // (s*J + j)*nb
  cplx* tau2;     // s*J + j
  int* progress;  // n counters, PSTRIDE ints apart (one 128-byte line each), then the sweep ticket;
                  // k_chase counts finished steps, k_chase_cl finished (CTA, step) pairs
  int* st;
};
constexpr int PSTRIDE = 32;

// The sweep-ticket counter: one line after the n progress counters (zeroed
// with them before the launch).
__device__ __forceinline__ int* ticket_ptr(const ChaseArgs& a) { return a.progress + (size_t)a.n * PSTRIDE; }

__device__ __forceinline__ cplx* bat(const ChaseArgs& a, int r, int c) {
  return a.WB + (size_t)(r - c) + (size_t)c * a.ldb;
}

__device__ __forceinline__ cplx warp_sum(cplx v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    v.x += __shfl_xor_sync(0xffffffffu, v.x, o);
    v.y += __shfl_xor_sync(0xffffffffu, v.y, o);
  }
  return v;
}

// Shared-memory state of one CTA: the step's diagonal block D (full square),
// its sub-diagonal block E (rows R_j, columns R_{j-1}), the reflectors and
// reduction scratch.
struct ChaseSmem {
  cplx D[MAXNB * LDS];
  cplx E[MAXNB * LDS];
  cplx vprev[MAXNB], vcur[MAXNB], y[MAXNB];
  cplx part[4][MAXNB];
  cplx red[HT / 32];
  cplx scal;
  cplx tau;
  double beta;
  int ok;
  int sweep;
};

// Reflector from x[0..len) (in smem): on return x = v (v[0] = 1), S.tau and
// S.beta set (H^H x = beta e_1, beta real).
__device__ void make_reflector(ChaseSmem& S, cplx* x, int len) {
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  double s = 0.0;
  for (int i = 1 + t; i < len; i += HT) s += cabs2(x[i]);
  const cplx sv = warp_sum(mk(s, 0.0));
  if (lane == 0) S.red[warp] = sv;
  __syncthreads();
  if (t == 0) {
    double xn2 = 0.0;
    for (int w = 0; w < HT / 32; ++w) xn2 += S.red[w].x;
    const cplx al = x[0];
    if (xn2 == 0.0 && al.y == 0.0) {
      S.tau = mk(0.0, 0.0);
      S.beta = al.x;
      S.scal = mk(0.0, 0.0);
    } else {
      const double nrm = sqrt(al.x * al.x + al.y * al.y + xn2);
      const double beta = (al.x >= 0.0) ? -nrm : nrm;
      S.beta = beta;
      S.tau = mk((beta - al.x) / beta, -al.y / beta);
      S.scal = cinv(mk(al.x - beta, al.y));
    }
  }
  __syncthreads();
  const cplx sc = S.scal;
  for (int i = 1 + t; i < len; i += HT) x[i] = cmul(x[i], sc);
  if (t == 0) x[0] = mk(1.0, 0.0);
  __syncthreads();
}

// out[r] = sum_c M(r, c) x[c], r < R, c < Cn (M column-major, pitch LDS):
// four threads per row, partial sums combined through S.part.
__device__ __forceinline__ void smem_gemv(ChaseSmem& S, const cplx* M, int R, int Cn, const cplx* x, cplx* out,
                                          cplx scale) {
  const int t = threadIdx.x, r = t & 63, q = t >> 6;
  if (r < R) {
    cplx acc = mk(0.0, 0.0);
    for (int c = q; c < Cn; c += 4) cfma(acc, M[c * LDS + r], x[c]);
    S.part[q][r] = acc;
  }
  __syncthreads();
  if (t < R) out[t] = cmul(scale, cadd(cadd(S.part[0][t], S.part[1][t]), cadd(S.part[2][t], S.part[3][t])));
  __syncthreads();
}

// out[c] = sum_r conj(x[r]) M(r, c), c in [c0, Cn), r < R.
__device__ __forceinline__ void smem_gemv_h(ChaseSmem& S, const cplx* M, int R, int c0, int Cn, const cplx* x,
                                            cplx* out, cplx scale) {
  const int t = threadIdx.x, c = t & 63, q = t >> 6;
  if (c >= c0 && c < Cn) {
    cplx acc = mk(0.0, 0.0);
    for (int r = q; r < R; r += 4) ccfma(acc, x[r], M[c * LDS + r]);
    S.part[q][c] = acc;
  }
  __syncthreads();
  if (t >= c0 && t < Cn) out[t] = cmul(scale, cadd(cadd(S.part[0][t], S.part[1][t]), cadd(S.part[2][t], S.part[3][t])));
  __syncthreads();
}

// D <- H^H D H for the Hermitian L x L block in S.D (full square).
__device__ void two_sided(ChaseSmem& S, int L, const cplx* v, cplx tau) {
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  cplx* p = S.y;
  smem_gemv(S, S.D, L, L, v, p, tau);  // p = tau D v
  // alpha = -1/2 tau (p^H v);  w = p + alpha v
  cplx pv = mk(0.0, 0.0);
  for (int r = t; r < L; r += HT) ccfma(pv, p[r], v[r]);
  pv = warp_sum(pv);
  if (lane == 0) S.red[warp] = pv;
  __syncthreads();
  if (t == 0) {
    cplx s = mk(0.0, 0.0);
    for (int w = 0; w < HT / 32; ++w) s = cadd(s, S.red[w]);
    S.scal = cscal(-0.5, cmul(tau, s));
  }
  __syncthreads();
  const cplx al = S.scal;
  for (int r = t; r < L; r += HT) p[r] = cadd(p[r], cmul(al, v[r]));
  __syncthreads();
  // D -= v w^H + w v^H
  for (int i = t; i < L * L; i += HT) {
    const int r = i % L, c = i / L;
    cplx d = csub(S.D[c * LDS + r], cadd(cmulc(v[r], p[c]), cmulc(p[r], v[c])));
    if (r == c) d.y = 0.0;
    S.D[c * LDS + r] = d;
  }
  __syncthreads();
}

// One CTA per sweep at a time (sweeps taken from the ticket counter).  Each
// step stages its blocks in shared memory: one coalesced read of D (lower,
// mirrored) and E from the working band, the step's arithmetic on chip, one
// write back.
__global__ void __launch_bounds__(HT, 1) k_chase(ChaseArgs A) {
  extern __shared__ __align__(16) unsigned char chase_smem_raw[];
  ChaseSmem& S = *reinterpret_cast<ChaseSmem*>(chase_smem_raw);
  const int t = threadIdx.x, n = A.n, nb = A.nb;
  for (;;) {
    if (t == 0) S.sweep = atomicAdd(ticket_ptr(A), 1);
    __syncthreads();
    const int s = S.sweep;
    __syncthreads();  // every thread has read the ticket before thread 0 may take the next
    if (s > n - 2) return;
    const int ntask = (n - 1 - s + nb - 1) / nb;
    const int ntask_prev = (s > 0) ? (n - 1 - (s - 1) + nb - 1) / nb : 0;
    cplx tprev = mk(0.0, 0.0);
    int Lprev = 0;
    for (int j = 0; j < ntask; ++j) {
      // wait for sweep s-1 to finish step j+1
      if (s > 0) {
        if (t == 0) {
          // poll sweep s-1's counter (its own cache line) with a growing pause;
          // the shared status word is looked at only every 64 polls
          const int need = min(j + 2, ntask_prev);
          const unsigned long long t0 = gtimer();
          int ok = 1;
          unsigned pause = 16, polls = 0;
          while (ld_acquire_i(&A.progress[(size_t)(s - 1) * PSTRIDE]) < need) {
            if ((++polls & 63) == 0 && (gtimer() - t0 > GBHE_WAIT_NS || ld_acquire_i(&A.st[ST_ERR]) != 0)) {
              set_err_once(A.st, GBHE_ETIMEOUT);
              ok = 0;
              break;
            }
            __nanosleep(pause);
            if (pause < 256) pause <<= 1;
          }
          S.ok = ok;
        }
        __syncthreads();
        if (!S.ok) return;
      }
      const int a0 = s + 1 + j * nb;
      const int L = min(nb, n - a0);
      const int c0 = a0 - nb;  // first column of R_{j-1}
      // stage D = A[R_j, R_j] (lower read, mirrored) and, for j > 0, E = A[R_j, R_{j-1}]:
      // every load of a thread is issued before the first shared-memory store
      {
        constexpr int PER = MAXNB * MAXNB / HT;
        cplx dv[PER], ev[PER];
#pragma unroll
        for (int k = 0; k < PER; ++k) {
          const int i = t + k * HT, r = i % MAXNB, c = i / MAXNB;
          dv[k] = (r < L && c <= r) ? __ldcg(bat(A, a0 + r, a0 + c)) : mk(0.0, 0.0);
          ev[k] = (j > 0 && r < L && c < Lprev) ? __ldcg(bat(A, a0 + r, c0 + c)) : mk(0.0, 0.0);
        }
        if (j == 0)
          for (int i = t; i < L; i += HT) S.vcur[i] = __ldcg(bat(A, a0 + i, s));
#pragma unroll
        for (int k = 0; k < PER; ++k) {
          const int i = t + k * HT, r = i % MAXNB, c = i / MAXNB;
          if (r < L && c <= r) {
            cplx d = dv[k];
            if (r == c) d.y = 0.0;
            S.D[c * LDS + r] = d;
            S.D[r * LDS + c] = cconj(d);
          }
          if (j > 0 && r < L && c < Lprev) S.E[c * LDS + r] = ev[k];
        }
      }
      __syncthreads();
      if (j == 0) {
        make_reflector(S, S.vcur, L);
        for (int i = t; i < L; i += HT) __stcg(bat(A, a0 + i, s), i == 0 ? mk(S.beta, 0.0) : mk(0.0, 0.0));
      } else {
        // E <- E H_{j-1}:  y = tau_prev E vprev;  E -= y vprev^H
        smem_gemv(S, S.E, L, Lprev, S.vprev, S.y, tprev);
        for (int i = t; i < L * Lprev; i += HT) {
          const int r = i % L, c = i / L;
          S.E[c * LDS + r] = csub(S.E[c * LDS + r], cmulc(S.y[r], S.vprev[c]));
        }
        __syncthreads();
        // new reflector from column 0 of E
        for (int i = t; i < L; i += HT) S.vcur[i] = S.E[i];
        __syncthreads();
        make_reflector(S, S.vcur, L);
        // E[:, 1:] <- H^H E[:, 1:]:  z_c = conj(tau) v^H E[:, c];  E[:, c] -= v z_c;  E[:, 0] = beta e_1
        smem_gemv_h(S, S.E, L, 1, Lprev, S.vcur, S.y, cconj(S.tau));
        for (int i = t; i < L * Lprev; i += HT) {
          const int r = i % L, c = i / L;
          cplx e;
          if (c == 0) e = (r == 0) ? mk(S.beta, 0.0) : mk(0.0, 0.0);
          else e = csub(S.E[c * LDS + r], cmul(S.vcur[r], S.y[c]));
          __stcg(bat(A, a0 + r, c0 + c), e);
        }
      }
      // store the reflector
      cplx* vout = A.V2 + ((size_t)s * A.J + j) * nb;
      for (int i = t; i < nb; i += HT) vout[i] = (i < L) ? S.vcur[i] : mk(0.0, 0.0);
      if (t == 0) A.tau2[(size_t)s * A.J + j] = S.tau;
      const cplx tau = S.tau;
      // two-sided update of the diagonal block, written back (lower)
      two_sided(S, L, S.vcur, tau);
      for (int i = t; i < L * L; i += HT) {
        const int r = i % L, c = i / L;
        if (r >= c) __stcg(bat(A, a0 + r, a0 + c), S.D[c * LDS + r]);
      }
      // keep H_j for the next step
      for (int i = t; i < L; i += HT) S.vprev[i] = S.vcur[i];
      tprev = tau;
      Lprev = L;
      __syncthreads();
      // publish progress
      if (t == 0) {
        __threadfence();
        st_release_i(&A.progress[(size_t)s * PSTRIDE], j + 1);
      }
    }
  }
}

// ---------------------------------------------------------------- cluster form
// The same chase with one step split over a cluster of CS CTAs: CTA `rank`
// owns rows rank*RS .. rank*RS+RS-1 of the step's blocks (D and E).  Every
// row-local operation (E H_{j-1}, H^H E, D v, the two-sided update) runs on
// the owning CTA; the data the CTAs exchange go through distributed shared
// memory with two cluster barriers per step:
//   A: the rows of x (the column the reflector is made from), the parts of
//      |x(1:)|^2 and every CTA's verdict on its wait for the previous sweep;
//   B: the parts of z = v^H E, the rows of p = tau D v and the parts of p^H v
//      (D v needs only v, so p is formed beside z and both cross one barrier).
// Every CTA waits for the previous sweep itself and reports its own step
// through an atomic count (CS per finished step), so no barrier is spent on
// the hand-over.  A wait that expires is reported at A and the whole cluster
// returns together (nobody leaves while a peer may still read its shared
// memory, and nobody is left waiting at a barrier).  The published arrays of
// A and B are distinct, and a CTA cannot pass barrier A (B) of the next step
// before every peer has arrived there, i.e. has finished reading this step's
// data: no data of a step is overwritten while a peer reads it.
constexpr int CS = 4, CT = 128, RS = MAXNB / CS;
static_assert(RS * CS == MAXNB && CT % 8 == 0, "row split");

struct ClSmem {
  cplx D[RS * LDS];  // my rows of the diagonal block, all columns (row-major, pitch LDS)
  cplx E[RS * LDS];  // my rows of the sub-diagonal block
  cplx vprev[MAXNB], v[MAXNB], w[MAXNB], z[MAXNB];
  cplx half[2][MAXNB];
  cplx pub_x[RS];     // A: my rows of x
  double pub_nrm;     // A: my rows' part of |x(1:)|^2
  int pub_ok;         // A: my wait for the previous sweep succeeded
  cplx pub_z[MAXNB];  // B: my rows' part of v^H E
  cplx pub_p[RS];     // B: my rows of p = tau D v
  cplx pub_pv;        // B: my rows' part of p^H v
  double red[CT / 32];
  cplx redc[CT / 32];
  cplx tau, scal;
  double beta;
  int ok;
  int sweep;
};

__device__ __forceinline__ cplx warp_sum8(cplx v) {  // sum over aligned groups of 8 lanes
#pragma unroll
  for (int o = 4; o > 0; o >>= 1) {
    v.x += __shfl_xor_sync(0xffffffffu, v.x, o);
    v.y += __shfl_xor_sync(0xffffffffu, v.y, o);
  }
  return v;
}

__global__ void __launch_bounds__(CT) k_chase_cl(ChaseArgs A) {
  extern __shared__ __align__(16) unsigned char cl_smem_raw[];
  ClSmem& S = *reinterpret_cast<ClSmem*>(cl_smem_raw);
  cg::cluster_group cl = cg::this_cluster();
  const int rank = (int)cl.block_rank();
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  const int n = A.n, nb = A.nb;
  const int R0 = rank * RS;
  const int row8 = t >> 3, sub = t & 7;  // 8 threads per local row
  ClSmem* peer[CS];
#pragma unroll
  for (int q = 0; q < CS; ++q) peer[q] = cl.map_shared_rank(&S, q);

  for (;;) {
    // ---- next sweep: rank 0 takes a ticket and publishes it to the cluster
    if (rank == 0 && t == 0) S.sweep = atomicAdd(ticket_ptr(A), 1);
    cl.sync();
    const int s = peer[0]->sweep;
    if (s > n - 2) {
      cl.sync();  // nobody leaves while another CTA may still read its shared memory
      return;
    }
    const int ntask = (n - 1 - s + nb - 1) / nb;
    const int ntask_prev = (s > 0) ? (n - 1 - (s - 1) + nb - 1) / nb : 0;
    cplx tprev = mk(0.0, 0.0);
    int Lprev = 0;
    for (int j = 0; j < ntask; ++j) {
      // ---- wait (every CTA) for all CS CTAs of sweep s-1 to finish step j+1
      if (t == 0) {
        int ok = 1;
        if (s > 0) {
          const int need = CS * min(j + 2, ntask_prev);
          const unsigned long long t0 = gtimer();
          unsigned pause = 16, polls = 0;
          while (ld_acquire_i(&A.progress[(size_t)(s - 1) * PSTRIDE]) < need) {
            if ((++polls & 63) == 0 && (gtimer() - t0 > GBHE_WAIT_NS || ld_acquire_i(&A.st[ST_ERR]) != 0)) {
              set_err_once(A.st, GBHE_ETIMEOUT);
              ok = 0;
              break;
            }
            __nanosleep(pause);
            if (pause < 256) pause <<= 1;
          }
        }
        S.ok = ok;
      }
      __syncthreads();
      const int a0 = s + 1 + j * nb;
      const int L = min(nb, n - a0);
      const int c0 = a0 - nb;
      const int R1 = min(L, R0 + RS), nloc = max(0, R1 - R0);
      // ---- stage my rows of D (lower read, mirrored) and of E (only after a wait that succeeded):
      // every load of a thread is issued before the first shared-memory store,
      // so the step pays one round trip to L2 instead of one per element group
      if (S.ok) {
        constexpr int PER = RS * MAXNB / CT;
        cplx dv[PER], ev[PER], uv[PER], xv = mk(0.0, 0.0);
#pragma unroll
        for (int k = 0; k < PER; ++k) {
          const int idx = t + k * CT;
          const int r = idx % RS, c = idx / RS, i = R0 + r;  // consecutive threads: consecutive rows
          dv[k] = (r < nloc && c < L && c <= i) ? __ldcg(bat(A, a0 + i, a0 + c)) : mk(0.0, 0.0);
          ev[k] = (j > 0 && r < nloc && c < Lprev) ? __ldcg(bat(A, a0 + i, c0 + c)) : mk(0.0, 0.0);
        }
#pragma unroll
        for (int k = 0; k < PER; ++k) {
          const int idx = t + k * CT;
          const int r = idx / MAXNB, c = idx % MAXNB, i = R0 + r;  // consecutive threads: consecutive columns
          uv[k] = (r < nloc && c < L && c > i) ? __ldcg(bat(A, a0 + c, a0 + i)) : mk(0.0, 0.0);
        }
        if (j == 0 && t < nloc) xv = __ldcg(bat(A, a0 + R0 + t, s));  // x in column 0
#pragma unroll
        for (int k = 0; k < PER; ++k) {
          const int idx = t + k * CT;
          const int r = idx % RS, c = idx / RS, i = R0 + r;
          if (r < nloc && c < L && c <= i) {
            cplx d = dv[k];
            if (c == i) d.y = 0.0;
            S.D[r * LDS + c] = d;
          }
          if (j > 0 && r < nloc && c < Lprev) S.E[r * LDS + c] = ev[k];
        }
#pragma unroll
        for (int k = 0; k < PER; ++k) {
          const int idx = t + k * CT;
          const int r = idx / MAXNB, c = idx % MAXNB, i = R0 + r;
          if (r < nloc && c < L && c > i) S.D[r * LDS + c] = cconj(uv[k]);
        }
        if (j == 0 && t < nloc) S.E[t * LDS] = xv;
      }
      __syncthreads();
      // ---- E <- E H_{j-1}:  y = tau_prev E vprev;  E -= y vprev^H   (row-local)
      if (j > 0) {  // j is uniform: every lane reaches the shuffle of warp_sum8
        const bool mine = row8 < nloc;
        cplx acc = mk(0.0, 0.0);
        if (mine)
          for (int c = sub; c < Lprev; c += 8) cfma(acc, S.E[row8 * LDS + c], S.vprev[c]);
        const cplx y = cmul(tprev, warp_sum8(acc));
        if (mine)
          for (int c = sub; c < Lprev; c += 8) S.E[row8 * LDS + c] = csub(S.E[row8 * LDS + c], cmulc(y, S.vprev[c]));
      }
      __syncthreads();
      // ---- publish x (my rows of column 0), my part of |x(1:)|^2 and my wait's verdict
      double nrm = 0.0;
      for (int r = t; r < nloc; r += CT) {
        const cplx x = S.E[r * LDS];
        S.pub_x[r] = x;
        if (R0 + r >= 1) nrm += cabs2(x);
      }
      for (int o = 16; o > 0; o >>= 1) nrm += __shfl_xor_sync(0xffffffffu, nrm, o);
      if (lane == 0) S.red[warp] = nrm;
      __syncthreads();
      if (t == 0) {
        double sum = 0.0;
        for (int q = 0; q < CT / 32; ++q) sum += S.red[q];
        S.pub_nrm = sum;
        S.pub_ok = S.ok;
      }
      cl.sync();  // A
      {
        int all_ok = 1;
#pragma unroll
        for (int q = 0; q < CS; ++q) all_ok &= peer[q]->pub_ok;
        if (!all_ok) {  // the same verdict in every CTA: the cluster returns together
          cl.sync();
          return;
        }
      }
      // ---- reflector, identical in every CTA: gather x, then scale
      if (t < L) S.v[t] = peer[t / RS]->pub_x[t % RS];
      if (t == 0) {
        double xn2 = 0.0;
        for (int q = 0; q < CS; ++q) xn2 += peer[q]->pub_nrm;
        const cplx al = peer[0]->pub_x[0];
        if (xn2 == 0.0 && al.y == 0.0) {
          S.tau = mk(0.0, 0.0); S.beta = al.x; S.scal = mk(0.0, 0.0);
        } else {
          const double nrmx = sqrt(al.x * al.x + al.y * al.y + xn2);
          const double beta = (al.x >= 0.0) ? -nrmx : nrmx;
          S.beta = beta;
          S.tau = mk((beta - al.x) / beta, -al.y / beta);
          S.scal = cinv(mk(al.x - beta, al.y));
        }
      }
      __syncthreads();
      const cplx tau = S.tau;
      if (t >= 1 && t < L) S.v[t] = cmul(S.v[t], S.scal);
      if (t == 0) S.v[0] = mk(1.0, 0.0);
      for (int r = t; r < nloc; r += CT) S.E[r * LDS] = (R0 + r == 0) ? mk(S.beta, 0.0) : mk(0.0, 0.0);
      __syncthreads();
      // ---- my parts of z = conj(tau) v^H E[:, 1:] (j > 0) and of p = tau D v, p^H v
      if (j > 0) {
        const int c = t % MAXNB, h = t / MAXNB;
        cplx acc = mk(0.0, 0.0);
        if (c >= 1 && c < Lprev)
          for (int r = h; r < nloc; r += 2) ccfma(acc, S.v[R0 + r], S.E[r * LDS + c]);
        S.half[h][c] = acc;
      }
      {
        const bool mine = row8 < nloc;
        cplx acc = mk(0.0, 0.0);
        if (mine)
          for (int c = sub; c < L; c += 8) cfma(acc, S.D[row8 * LDS + c], S.v[c]);
        const cplx pr = cmul(tau, warp_sum8(acc));  // every lane reaches the shuffle
        if (mine && sub == 0) S.pub_p[row8] = pr;
        // my part of p^H v: one contribution per row (the sub == 0 lane)
        cplx pv = (mine && sub == 0) ? cmulc(S.v[R0 + row8], pr) : mk(0.0, 0.0);  // v conj(p) = conj(p) v
        pv = warp_sum(pv);
        if (lane == 0) S.redc[warp] = pv;
      }
      __syncthreads();
      if (j > 0 && t < MAXNB) S.pub_z[t] = cadd(S.half[0][t], S.half[1][t]);
      if (t == 0) {
        cplx sum = mk(0.0, 0.0);
        for (int q = 0; q < CT / 32; ++q) sum = cadd(sum, S.redc[q]);
        S.pub_pv = sum;
      }
      cl.sync();  // B
      // ---- totals: z (j > 0) and w = p + alpha v, alpha = -1/2 tau p^H v (every thread sums the parts)
      if (j > 0 && t >= 1 && t < Lprev) {
        cplx zz = mk(0.0, 0.0);
        for (int q = 0; q < CS; ++q) zz = cadd(zz, peer[q]->pub_z[t]);
        S.z[t] = cmul(cconj(tau), zz);
      }
      if (t < L) {
        cplx pvt = mk(0.0, 0.0);
        for (int q = 0; q < CS; ++q) pvt = cadd(pvt, peer[q]->pub_pv);
        const cplx al = cscal(-0.5, cmul(tau, pvt));
        S.w[t] = cadd(peer[t / RS]->pub_p[t % RS], cmul(al, S.v[t]));
      }
      __syncthreads();
      if (j == 0) {
        for (int r = t; r < nloc; r += CT) __stcg(bat(A, a0 + R0 + r, s), S.E[r * LDS]);
      } else {
        // E[:, c] -= v z_c (c >= 1), then write my rows of E back
        for (int idx = t; idx < RS * MAXNB; idx += CT) {
          const int r = idx % RS, c = idx / RS;
          if (r < nloc && c < Lprev) {
            cplx e = S.E[r * LDS + c];
            if (c >= 1) e = csub(e, cmul(S.v[R0 + r], S.z[c]));
            __stcg(bat(A, a0 + R0 + r, c0 + c), e);
          }
        }
      }
      // ---- store the reflector (rank 0)
      if (rank == 0) {
        cplx* vout = A.V2 + ((size_t)s * A.J + j) * nb;
        for (int i = t; i < nb; i += CT) vout[i] = (i < L) ? S.v[i] : mk(0.0, 0.0);
        if (t == 0) A.tau2[(size_t)s * A.J + j] = tau;
      }
      // ---- D -= v w^H + w v^H on my rows; write back the lower part
      for (int idx = t; idx < RS * MAXNB; idx += CT) {
        const int r = idx % RS, c = idx / RS, i = R0 + r;
        if (r < nloc && c < L && c <= i) {
          cplx d = csub(S.D[r * LDS + c], cadd(cmulc(S.v[i], S.w[c]), cmulc(S.w[i], S.v[c])));
          if (c == i) d.y = 0.0;
          __stcg(bat(A, a0 + i, a0 + c), d);
        }
      }
      // keep H_j for the next step
      for (int i = t; i < L; i += CT) S.vprev[i] = S.v[i];
      tprev = tau;
      Lprev = L;
      __syncthreads();
      // ---- report my part of the step (every store of this CTA is done)
      if (t == 0) {
        __threadfence();
        atomicAdd(&A.progress[(size_t)s * PSTRIDE], 1);
      }
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
  return (size_t)(2 * nb + 1) * std::max(n, 1) * sizeof(cplx) + (size_t)(std::max(n, 1) + 1) * PSTRIDE * sizeof(int) +
         512;
}

int hb2st_run(Ctx& c, int n, int nb, const cplx* A, int lda, double* d, double* e, cplx* V2, cplx* tau2) {
  if (n <= 0) return 0;
  if (nb < 1 || nb > MAXNB) return -3;
  Arena& a = c.arena;
  const size_t save = a.off;
  const int ldb = 2 * nb + 1;
  cplx* WB = a.take<cplx>((size_t)ldb * n);
  int* prog = a.take<int>((size_t)(n + 1) * PSTRIDE);  // progress counters, then the sweep ticket
  if (!a.ok() || !WB) { a.off = save; return GBHE_EWORKSPACE; }
  const int J = hb2st_J(n, nb);
  k_band_in<<<std::min<size_t>(((size_t)ldb * n + 255) / 256, 4096), 256, 0, c.st>>>(A, lda, n, nb, WB, ldb);
  count_launch();
  GBHE_CUDA(cudaGetLastError());
  GBHE_CUDA(cudaMemsetAsync(prog, 0, sizeof(int) * (size_t)(n + 1) * PSTRIDE, c.st));
  if (n >= 2) {
    ChaseArgs ca;
    ca.WB = WB; ca.ldb = ldb; ca.n = n; ca.nb = nb; ca.J = J; ca.V2 = V2; ca.tau2 = tau2;
    ca.progress = prog; ca.st = c.status;
    // sweep s starts about 2 steps after sweep s-1 and lasts at most J steps, so
    // at most ceil(J/2) + 1 sweeps are ever active: more CTAs would only wait
    // (and would keep other streams' kernels off their SMs)
    int G = std::min(std::min(c.num_sms, n - 1), (J + 1) / 2 + 2);
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
    // Cluster form (CS CTAs per sweep) when the device runs cluster launches of
    // this kernel, else the one-CTA form; decided once per device, outside
    // stream capture.  Both are ordinary launches: the ticket order, not
    // co-residency, guarantees progress, so the grid is only capped at the
    // clusters that fit at once (more would only wait for a free slot).
    static int cl_states[MAX_DEVICES] = {};  // 0 unknown, 1 usable, -1 not usable
    static int cl_max[MAX_DEVICES] = {};     // clusters resident at once
    const int dev = device_slot();
    if (dev < 0) { a.off = save; return GBHE_ECUDA; }
    int& cl_state = cl_states[dev];
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    GBHE_CUDA(cudaStreamIsCapturing(c.st, &cap));
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = CS;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.blockDim = dim3(CT);
    cfg.dynamicSmemBytes = sizeof(ClSmem);
    cfg.stream = c.st;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    if (cl_state == 0 && cap == cudaStreamCaptureStatusNone) {
      cfg.gridDim = dim3(CS);
      int maxc = 0;
      if (cudaOccupancyMaxActiveClusters(&maxc, (void*)k_chase_cl, &cfg) == cudaSuccess && maxc >= 1) {
        cl_state = 1;
        cl_max[dev] = maxc;
      } else {
        (void)cudaGetLastError();
        cl_state = -1;
      }
    }
    bool launched = false;
    if (cl_state == 1) {
      const int Gc = std::max(1, std::min(G, cl_max[dev]));
      cfg.gridDim = dim3(Gc * CS);
      if (cudaLaunchKernelEx(&cfg, k_chase_cl, ca) == cudaSuccess) launched = true;
      else (void)cudaGetLastError();
    }
    if (!launched) {
      GBHE_CUDA(cudaFuncSetAttribute(k_chase, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(ChaseSmem)));
      k_chase<<<G, HT, sizeof(ChaseSmem), c.st>>>(ca);
      GBHE_CUDA(cudaGetLastError());
    }
  }
  k_band_out<<<std::min((n + 255) / 256, 1024), 256, 0, c.st>>>(WB, ldb, n, d, e);
  count_launch();
  GBHE_CUDA(cudaGetLastError());
  a.off = save;
  return 0;
}

}  // namespace gbhe
