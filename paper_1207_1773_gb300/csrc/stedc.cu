// stedc.cu -- divide and conquer eigensolver for a real symmetric tridiagonal
// T (paper Section 4.3), entirely on the GPU.
//
// Tearing: T is cut into leaves of LS = 32 rows.  At a cut between rows p-1
// and p with coupling beta = e[p-1]:
//   T = diag(T1', T2') + |beta| v v^T,  v = e_{p-1} + sign(beta) e_p,
// where T1', T2' have |beta| subtracted from their touching diagonal entries.
// Leaves: one warp each, implicit symmetric QR with Wilkinson shift; every
// lane owns one row of the 32 x 32 eigenvector block.
// Merge of two children (eigenpairs (Lambda1, Z1), (Lambda2, Z2)) -- the
// rank-one update of the paper's merge equation:
//   T = diag(Z1, Z2) (diag(Lambda1, Lambda2) + rho u u^T) diag(Z1, Z2)^T,
//   u = [last row of Z1, sign(beta) * first row of Z2] / sqrt(2), rho = 2|beta|;
//   D + rho u u^T = Q Lambda Q^T;  Z = diag(Z1, Z2) Q   (GEMM).
// Steps per tree level (all nodes of the level in each launch):
//   deflate   merge-sort of D, deflation of tiny u_j and of close pairs (a
//             plane rotation zeroes one u component), column classification
//             (upper-only / mixed / lower-only) so the GEMM skips zero blocks;
//   rotate    apply the recorded rotations to the eigenvector columns;
//   gather    pack the non-deflated columns in GEMM order, then the deflated;
//   secular   one thread per root of 1 + rho sum u_j^2/(d_j - lambda) = 0,
//             bracketed iteration on a two-pole rational model, lambda kept as
//             (origin pole) + tau for accurate differences d_j - lambda;
//   zhat      Gu-Eisenstat recomputation of u from the computed roots, so the
//             eigenvectors q_i(j) = zhat_j/(d_j - lambda_i) are orthogonal;
//   qbuild    normalised Q columns;
//   positions final ascending order of roots and deflated values;
//   gemm      grouped DMMA GEMMs (upper rows, lower rows) straight into the
//             final column positions; deflated columns copied.
// In the last merge only the columns il..iu are formed (Section 4.3, end).
#include <algorithm>
#include "internal.cuh"

namespace gbhe {
namespace {

constexpr int LS = 32;
constexpr double EPS = 2.220446049250313e-16;

struct DC {
  int n, nleaf;
  double* scale;   // [0] = max |T| used to normalise
  double* dd;      // torn, scaled diagonal
  double* ee;      // scaled off-diagonal
  double* lam;     // eigenvalues per node (ascending within the node)
  double* Z;       // n x n block-diagonal eigenvectors, ld n
  double* Zt;      // gathered columns, ld n
  double* Q;       // secular eigenvectors, ld n
  // per node arrays, indexed by node.lo + local index
  double *sD, *sz;
  int *stype, *scol;
  int *ndq, *ndtype, *ndgrp;
  double *ndD, *ndz;
  int* dfq;
  double* dfv;
  int *rota, *rotb;
  double *rotc, *rots;
  int *cnt;        // 8 ints per node, at 8 * (node.lo / LS)
  int *rorg;
  double *rtau, *rlam, *zhat;
  int *dfrank, *cpos, *dfpos;
  DGroupDesc* desc;
  CrtDesc* cdesc;  // the same products for the tensor-core GEMM
  int* st;
};

struct NodeR {
  int lo, mid, hi, merge;
};

__host__ __device__ inline NodeR node_range(int n, int nleaf, int lev, int i) {
  NodeR r;
  const int l0 = i << lev, l1 = min((i + 1) << lev, nleaf);
  r.lo = l0 * LS;
  r.hi = min(l1 * LS, n);
  const int lm = l0 + (lev > 0 ? (1 << (lev - 1)) : 1);
  r.merge = (lev > 0 && lm < l1) ? 1 : 0;
  r.mid = r.merge ? lm * LS : r.hi;
  return r;
}

__device__ inline int* node_cnt(const DC& a, int lo) { return a.cnt + 8 * (lo / LS); }

// A recorded error (non-finite input, a leaf that did not converge) stops the
// divide and conquer: later kernels return at once, so that no index derived
// from NaN data is ever used.
__device__ __forceinline__ bool dc_failed(const DC& a) { return *(volatile int*)&a.st[ST_ERR] != 0; }
enum { C_K = 0, C_ND = 1, C_ROT = 2, C_K1 = 3, C_K2 = 4, C_K3 = 5 };

// ---------------------------------------------------------------- scaling
__global__ void k_scale_tear(DC a, const double* d, const double* e) {
  __shared__ double red[1024];
  __shared__ int bad;
  const int t = threadIdx.x, n = a.n;
  if (t == 0) bad = 0;
  __syncthreads();
  double m = 0.0;
  bool nf = false;  // fmax drops NaN, so non-finite entries are flagged separately
  for (int i = t; i < n; i += blockDim.x) { m = fmax(m, fabs(d[i])); nf |= !isfinite(d[i]); }
  for (int i = t; i + 1 < n; i += blockDim.x) { m = fmax(m, fabs(e[i])); nf |= !isfinite(e[i]); }
  if (nf) atomicOr(&bad, 1);
  red[t] = m;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (t < s) red[t] = fmax(red[t], red[t + s]);
    __syncthreads();
  }
  double sc = red[0];
  if (t == 0 && bad) set_err_once(a.st, GBHE_ENONFINITE);  // NaN or Inf in (d, e)
  if (!(sc > 0.0) || !isfinite(sc)) sc = 1.0;
  if (t == 0) a.scale[0] = sc;
  const double inv = 1.0 / sc;
  for (int i = t; i < n; i += blockDim.x) a.dd[i] = d[i] * inv;
  for (int i = t; i + 1 < n; i += blockDim.x) a.ee[i] = e[i] * inv;
  if (t == 0 && n > 0) a.ee[n - 1] = 0.0;
  __syncthreads();
  for (int q = 1 + t; q < a.nleaf; q += blockDim.x) {
    const int p = q * LS;
    const double rho = fabs(a.ee[p - 1]);
    a.dd[p - 1] -= rho;
    a.dd[p] -= rho;
  }
}

// ---------------------------------------------------------------- leaves
// One warp per leaf; lane r owns row r of the leaf's eigenvector block.
__global__ void __launch_bounds__(128) k_leaf(DC a) {
  if (dc_failed(a)) return;
  __shared__ double Zs[4][LS][LS + 1];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int leaf = blockIdx.x * 4 + warp;
  if (leaf >= a.nleaf) return;
  const int lo = leaf * LS, sz = min(LS, a.n - lo);
  double dl[LS], el[LS];
  for (int i = 0; i < LS; ++i) {
    dl[i] = (i < sz) ? a.dd[lo + i] : 0.0;
    el[i] = (i + 1 < sz) ? a.ee[lo + i] : 0.0;
  }
  for (int c = 0; c < LS; ++c) Zs[warp][lane][c] = (lane == c) ? 1.0 : 0.0;
  __syncwarp();
  int hi = sz - 1, iter = 0;
  while (hi > 0) {
    for (int i = 0; i < hi; ++i)
      if (fabs(el[i]) <= EPS * (fabs(dl[i]) + fabs(dl[i + 1]))) el[i] = 0.0;
    if (el[hi - 1] == 0.0) { --hi; continue; }
    int lo2 = hi - 1;
    while (lo2 > 0 && el[lo2 - 1] != 0.0) --lo2;
    if (++iter > 60 * LS) {
      if (lane == 0) set_err_once(a.st, GBHE_ENOTCONV);
      break;
    }
    const double dd_ = 0.5 * (dl[hi - 1] - dl[hi]);
    const double bb = el[hi - 1];
    const double h = hypot(dd_, bb);
    const double mu = dl[hi] - bb * bb / (dd_ + (dd_ >= 0.0 ? h : -h));
    double x = dl[lo2] - mu, z = el[lo2];
    for (int k = lo2; k < hi; ++k) {
      double r = hypot(x, z), c = 1.0, s = 0.0;
      if (r != 0.0) { c = x / r; s = z / r; }
      if (k > lo2) el[k - 1] = r;
      const double p0 = dl[k], q0 = el[k], r0 = dl[k + 1];
      dl[k] = c * c * p0 + 2.0 * c * s * q0 + s * s * r0;
      dl[k + 1] = s * s * p0 - 2.0 * c * s * q0 + c * c * r0;
      el[k] = c * s * (r0 - p0) + (c * c - s * s) * q0;
      if (k + 1 < hi) {
        z = s * el[k + 1];
        el[k + 1] = c * el[k + 1];
        x = el[k];
      }
      const double zk = Zs[warp][lane][k], zk1 = Zs[warp][lane][k + 1];
      Zs[warp][lane][k] = c * zk + s * zk1;
      Zs[warp][lane][k + 1] = -s * zk + c * zk1;
    }
  }
  // ascending order (stable), identical in every lane
  int perm[LS];
  for (int i = 0; i < LS; ++i) perm[i] = i;
  for (int i = 1; i < sz; ++i) {
    int t = perm[i], j = i - 1;
    while (j >= 0 && dl[perm[j]] > dl[t]) { perm[j + 1] = perm[j]; --j; }
    perm[j + 1] = t;
  }
  __syncwarp();
  if (lane < sz) {
    for (int c = 0; c < sz; ++c) a.Z[(size_t)(lo + lane) + (size_t)(lo + c) * a.n] = Zs[warp][lane][perm[c]];
    a.lam[lo + lane] = dl[perm[lane]];
  }
}

// ---------------------------------------------------------------- deflate
// One CTA per merging node.
__global__ void __launch_bounds__(256) k_deflate(DC a, int lev) {
  if (dc_failed(a)) return;
  const NodeR nd = node_range(a.n, a.nleaf, lev, blockIdx.x);
  if (!nd.merge) return;
  const int lo = nd.lo, mid = nd.mid, hi = nd.hi, n0 = hi - lo, n1 = mid - lo;
  const int t = threadIdx.x;
  const double beta = a.ee[mid - 1];
  const double rho = 2.0 * fabs(beta);
  const double sgn = (beta >= 0.0) ? 1.0 : -1.0;
  const double isq2 = 0.70710678118654752440;
  __shared__ double red[256], redz[256];
  double dmax = 0.0, zmax = 0.0;
  for (int i = t; i < n0; i += blockDim.x) {
    const double Di = a.lam[lo + i];
    double zi;
    int pos;
    if (i < n1) {
      zi = a.Z[(size_t)(mid - 1) + (size_t)(lo + i) * a.n] * isq2;
      // number of right-child values strictly below Di
      int l = 0, h = hi - mid;
      while (l < h) { int m = (l + h) >> 1; if (a.lam[mid + m] < Di) l = m + 1; else h = m; }
      pos = i + l;
    } else {
      zi = sgn * a.Z[(size_t)mid + (size_t)(lo + i) * a.n] * isq2;
      int l = 0, h = n1;
      while (l < h) { int m = (l + h) >> 1; if (a.lam[lo + m] <= Di) l = m + 1; else h = m; }
      pos = (i - n1) + l;
    }
    pos = min(max(pos, 0), n0 - 1);
    a.sD[lo + pos] = Di;
    a.sz[lo + pos] = zi;
    a.scol[lo + pos] = lo + i;
    a.stype[lo + pos] = (i < n1) ? 1 : 3;
    dmax = fmax(dmax, fabs(Di));
    zmax = fmax(zmax, fabs(zi));
  }
  red[t] = dmax;
  redz[t] = zmax;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (t < s) { red[t] = fmax(red[t], red[t + s]); redz[t] = fmax(redz[t], redz[t + s]); }
    __syncthreads();
  }
  if (t != 0) return;
  dmax = red[0];
  zmax = redz[0];
  const double tol = 8.0 * EPS * fmax(dmax, rho);
  int k = 0, ndf = 0, nrot = 0, grp[4] = {0, 0, 0, 0};
  const bool all = !(rho * zmax > tol);
  int pq = -1, ptype = 0;
  double pD = 0.0, pz = 0.0;
  for (int q = 0; q < n0; ++q) {
    const double Dq = a.sD[lo + q], zq = a.sz[lo + q];
    const int tq = a.stype[lo + q];
    if (all || rho * fabs(zq) <= tol) {
      a.dfq[lo + ndf] = q;
      a.dfv[lo + ndf] = Dq;
      ++ndf;
      continue;
    }
    if (pq < 0) { pq = q; pD = Dq; pz = zq; ptype = tq; continue; }
    const double tau = hypot(zq, pz);
    const double c = zq / tau, s = pz / tau;
    const double tt = Dq - pD;
    if (fabs(tt * c * s) <= tol) {
      // [col_p, col_q] <- [c col_p - s col_q, s col_p + c col_q]; col_p deflated
      a.rota[lo + nrot] = pq;
      a.rotb[lo + nrot] = q;
      a.rotc[lo + nrot] = c;
      a.rots[lo + nrot] = s;
      ++nrot;
      a.dfq[lo + ndf] = pq;
      a.dfv[lo + ndf] = c * c * pD + s * s * Dq;
      ++ndf;
      const double Dn = s * s * pD + c * c * Dq;
      ptype = (ptype == tq) ? tq : 2;
      pq = q; pD = Dn; pz = tau;
    } else {
      a.ndq[lo + k] = pq; a.ndD[lo + k] = pD; a.ndz[lo + k] = pz; a.ndtype[lo + k] = ptype;
      a.ndgrp[lo + k] = grp[ptype]++;
      ++k;
      pq = q; pD = Dq; pz = zq; ptype = tq;
    }
  }
  if (pq >= 0) {
    a.ndq[lo + k] = pq; a.ndD[lo + k] = pD; a.ndz[lo + k] = pz; a.ndtype[lo + k] = ptype;
    a.ndgrp[lo + k] = grp[ptype]++;
    ++k;
  }
  int* cn = node_cnt(a, lo);
  cn[C_K] = k; cn[C_ND] = ndf; cn[C_ROT] = nrot;
  cn[C_K1] = grp[1]; cn[C_K2] = grp[2]; cn[C_K3] = grp[3];
}

// ---------------------------------------------------------------- rotate
__global__ void __launch_bounds__(256) k_rotate(DC a, int lev) {
  if (dc_failed(a)) return;
  const NodeR nd = node_range(a.n, a.nleaf, lev, blockIdx.x);
  if (!nd.merge) return;
  const int lo = nd.lo, hi = nd.hi;
  const int nrot = node_cnt(a, lo)[C_ROT];
  for (int r = 0; r < nrot; ++r) {
    const int ca = a.scol[lo + a.rota[lo + r]], cb = a.scol[lo + a.rotb[lo + r]];
    if (ca < lo || ca >= hi || cb < lo || cb >= hi) continue;  // never for finite data
    const double c = a.rotc[lo + r], s = a.rots[lo + r];
    for (int row = lo + threadIdx.x; row < hi; row += blockDim.x) {
      double* pa = a.Z + (size_t)row + (size_t)ca * a.n;
      double* pb = a.Z + (size_t)row + (size_t)cb * a.n;
      const double x = *pa, y = *pb;
      *pa = c * x - s * y;
      *pb = s * x + c * y;
    }
    __syncthreads();
  }
}

__device__ inline int node_of(const DC& a, int lev, int g, NodeR& nd) {
  const int idx = (g / LS) >> lev;
  nd = node_range(a.n, a.nleaf, lev, idx);
  return idx;
}

__device__ inline int gemm_pos(const int* cn, int type, int grp) {
  return type == 1 ? grp : (type == 2 ? cn[C_K1] + grp : cn[C_K1] + cn[C_K2] + grp);
}

// ---------------------------------------------------------------- gather
// One CTA per (node-local) column slot: slot j < k -> non-deflated column in
// GEMM order; slot k + r -> deflated column r.
__global__ void __launch_bounds__(128) k_gather(DC a, int lev) {
  if (dc_failed(a)) return;
  NodeR nd;
  node_of(a, lev, blockIdx.x, nd);
  if (!nd.merge) return;
  const int lo = nd.lo, n0 = nd.hi - nd.lo, j = blockIdx.x - lo;
  if (j >= n0) return;
  const int* cn = node_cnt(a, lo);
  const int k = cn[C_K];
  int src, dst;
  if (j < k) {
    src = a.scol[lo + a.ndq[lo + j]];
    dst = lo + gemm_pos(cn, a.ndtype[lo + j], a.ndgrp[lo + j]);
  } else {
    src = a.scol[lo + a.dfq[lo + (j - k)]];
    dst = lo + j;
  }
  if (src < lo || src >= nd.hi || dst < lo || dst >= nd.hi) return;  // never for finite data
  const double* s = a.Z + (size_t)src * a.n;
  double* d = a.Zt + (size_t)dst * a.n;
  for (int row = lo + threadIdx.x; row < nd.hi; row += blockDim.x) d[row] = s[row];
}

// ---------------------------------------------------------------- secular
// Sums over the k poles, split across the 32 lanes of a warp; every lane ends
// with the totals (butterfly reductions), so the whole warp takes the same
// iteration decisions.
__device__ __forceinline__ double warp_allsum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__device__ void secular_eval(const double* D, const double* z, int k, int org, double rho, double tau,
                             int split, int lane, double& g, double& psi, double& dpsi, double& phi, double& dphi,
                             double& erretm) {
  psi = dpsi = phi = dphi = 0.0;
  erretm = 0.0;
  const double Do = D[org];
  for (int j = lane; j < k; j += 32) {
    const double del = (D[j] - Do) - tau;
    const double tmp = z[j] / del;
    const double term = rho * z[j] * tmp;
    if (j <= split) { psi += term; dpsi += rho * tmp * tmp; }
    else { phi += term; dphi += rho * tmp * tmp; }
    erretm += fabs(term);
  }
  psi = warp_allsum(psi);
  dpsi = warp_allsum(dpsi);
  phi = warp_allsum(phi);
  dphi = warp_allsum(dphi);
  erretm = warp_allsum(erretm);
  g = 1.0 + psi + phi;
}

// One warp per root.  Root i lies in (D_i, D_{i+1}) (i < k-1) or
// (D_{k-1}, D_{k-1} + rho |z|^2] (i = k-1).
__global__ void __launch_bounds__(128) k_secular(DC a, int lev) {
  if (dc_failed(a)) return;
  const int g = blockIdx.x * 4 + (threadIdx.x >> 5), lane = threadIdx.x & 31;
  if (g >= a.n) return;
  NodeR nd;
  node_of(a, lev, g, nd);
  if (!nd.merge) return;
  const int lo = nd.lo, i = g - lo;
  const int* cn = node_cnt(a, lo);
  const int k = cn[C_K];
  if (i >= k) return;
  const double* D = a.ndD + lo;
  const double* z = a.ndz + lo;
  const double rho = 2.0 * fabs(a.ee[nd.mid - 1]);
  if (k == 1) {
    if (lane == 0) {
      a.rorg[lo] = 0;
      a.rtau[lo] = rho * z[0] * z[0];
      a.rlam[lo] = D[0] + rho * z[0] * z[0];
    }
    return;
  }
  int org, split;
  double lo_t, hi_t;  // bracket for tau (relative to D[org])
  if (i < k - 1) {
    const double del = D[i + 1] - D[i];
    const double mid = 0.5 * del;
    // f(D_i + del/2) > 0  <=>  root below the midpoint
    double fm = 0.0;
    for (int j = lane; j < k; j += 32) fm += rho * z[j] * z[j] / ((D[j] - D[i]) - mid);
    fm = 1.0 + warp_allsum(fm);
    if (fm >= 0.0) { org = i; lo_t = 0.0; hi_t = mid; }
    else { org = i + 1; lo_t = -mid; hi_t = 0.0; }
    split = i;
  } else {
    double zz = 0.0;
    for (int j = lane; j < k; j += 32) zz += z[j] * z[j];
    zz = warp_allsum(zz);
    org = k - 1; lo_t = 0.0; hi_t = rho * zz; split = k - 1;
  }
  const double dl = D[i] - D[org];                       // left pole (relative)
  const double dr = (i < k - 1) ? D[i + 1] - D[org] : 0.0;  // right pole (relative)
  double x = 0.5 * (lo_t + hi_t);
  int it;
  for (it = 0; it < 200; ++it) {
    double gv, psi, dpsi, phi, dphi, erretm;
    secular_eval(D, z, k, org, rho, x, split, lane, gv, psi, dpsi, phi, dphi, erretm);
    if (fabs(gv) <= 8.0 * EPS * (1.0 + erretm) * (double)k) break;
    if (gv > 0.0) hi_t = x; else lo_t = x;
    if (hi_t - lo_t <= 2.0 * EPS * fmax(fabs(lo_t), fabs(hi_t))) break;
    // two-pole rational model: psi ~ A1 + B1/(dl - y), phi ~ A2 + B2/(dr - y)
    double y;
    const double B1 = dpsi * (dl - x) * (dl - x);
    const double A1 = psi - B1 / (dl - x);
    if (i < k - 1) {
      const double B2 = dphi * (dr - x) * (dr - x);
      const double A2 = phi - B2 / (dr - x);
      const double C = 1.0 + A1 + A2;
      // C (dl - y)(dr - y) + B1 (dr - y) + B2 (dl - y) = 0
      const double qa = C;
      const double qb = -(C * (dl + dr) + B1 + B2);
      const double qc = C * dl * dr + B1 * dr + B2 * dl;
      double r1, r2;
      if (qa == 0.0) {
        r1 = r2 = -qc / qb;
      } else {
        double disc = qb * qb - 4.0 * qa * qc;
        disc = sqrt(fmax(disc, 0.0));
        const double qq = -0.5 * (qb + (qb >= 0.0 ? disc : -disc));
        r1 = qq / qa;
        r2 = (qq != 0.0) ? qc / qq : r1;
      }
      y = (r1 > lo_t && r1 < hi_t) ? r1 : r2;
    } else {
      // 1 + A1 + phi + B1/(dl - y) = 0,  dl = 0 for the last root
      const double C = 1.0 + A1 + phi;
      y = (C != 0.0) ? dl + B1 / C : 0.5 * (lo_t + hi_t);
    }
    if (!(y > lo_t && y < hi_t)) y = 0.5 * (lo_t + hi_t);
    x = y;
  }
  if (lane != 0) return;
  if (it >= 200) set_err_once(a.st, GBHE_ENOTCONV);
  a.rorg[lo + i] = org;
  a.rtau[lo + i] = x;
  a.rlam[lo + i] = D[org] + x;
}

// ---------------------------------------------------------------- zhat
// One warp per pole j; the product over i != j is split across the lanes.
__global__ void __launch_bounds__(128) k_zhat(DC a, int lev) {
  if (dc_failed(a)) return;
  const int g = blockIdx.x * 4 + (threadIdx.x >> 5), lane = threadIdx.x & 31;
  if (g >= a.n) return;
  NodeR nd;
  node_of(a, lev, g, nd);
  if (!nd.merge) return;
  const int lo = nd.lo, j = g - lo;
  const int k = node_cnt(a, lo)[C_K];
  if (j >= k) return;
  const double* D = a.ndD + lo;
  const double rho = 2.0 * fabs(a.ee[nd.mid - 1]);
  // zhat_j^2 = (lambda_j - d_j)/rho * prod_{i != j} (lambda_i - d_j)/(d_i - d_j)
  const double dj = D[j];
  double p = 1.0;
  for (int i = lane; i < k; i += 32) {
    if (i == j) continue;
    const double lmd = -((dj - D[a.rorg[lo + i]]) - a.rtau[lo + i]);  // lambda_i - d_j
    p *= lmd / (D[i] - dj);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) p *= __shfl_xor_sync(0xffffffffu, p, o);
  if (lane != 0) return;
  p *= -((dj - D[a.rorg[lo + j]]) - a.rtau[lo + j]) / rho;
  const double zj = a.ndz[lo + j];
  const double v = sqrt(fabs(p));
  a.zhat[lo + j] = (zj >= 0.0) ? v : -v;
}

__global__ void __launch_bounds__(128) k_qbuild(DC a, int lev) {
  if (dc_failed(a)) return;
  const int g = blockIdx.x * 4 + (threadIdx.x >> 5), lane = threadIdx.x & 31;
  if (g >= a.n) return;
  NodeR nd;
  node_of(a, lev, g, nd);
  if (!nd.merge) return;
  const int lo = nd.lo, i = g - lo;
  const int* cn = node_cnt(a, lo);
  const int k = cn[C_K];
  if (i >= k) return;
  const double* D = a.ndD + lo;
  const double Dorg = D[a.rorg[lo + i]], tau = a.rtau[lo + i];
  double s = 0.0;
  for (int j = lane; j < k; j += 32) {
    const double v = a.zhat[lo + j] / ((D[j] - Dorg) - tau);
    s += v * v;
  }
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  const double inv = 1.0 / sqrt(s);
  double* col = a.Q + (size_t)(lo + i) * a.n + lo;
  for (int j = lane; j < k; j += 32) {
    const double v = a.zhat[lo + j] / ((D[j] - Dorg) - tau);
    col[gemm_pos(cn, a.ndtype[lo + j], a.ndgrp[lo + j])] = v * inv;
  }
}

// ---------------------------------------------------------------- positions
// Ranks of the deflated values, final positions of roots and deflated values,
// new eigenvalues of the node.  One CTA per node.
__global__ void __launch_bounds__(256) k_positions(DC a, int lev, int last, int il, int iu,
                                                   double* w_out) {
  if (dc_failed(a)) return;
  const NodeR nd = node_range(a.n, a.nleaf, lev, blockIdx.x);
  if (!nd.merge) return;
  const int lo = nd.lo;
  const int* cn = node_cnt(a, lo);
  const int k = cn[C_K], ndf = cn[C_ND];
  const double* dv = a.dfv + lo;
  const double* rl = a.rlam + lo;
  // rank of each deflated value (ties by index)
  for (int r = threadIdx.x; r < ndf; r += blockDim.x) {
    const double v = dv[r];
    int rank = 0;
    for (int q = 0; q < ndf; ++q) rank += (dv[q] < v || (dv[q] == v && q < r)) ? 1 : 0;
    a.dfrank[lo + r] = rank;
  }
  __syncthreads();
  // roots: pos = i + #{deflated <= lambda_i}
  for (int i = threadIdx.x; i < k; i += blockDim.x) {
    const double v = rl[i];
    int c = 0;
    for (int q = 0; q < ndf; ++q) c += (dv[q] <= v) ? 1 : 0;
    a.cpos[lo + i] = min(i + c, nd.hi - lo - 1);
  }
  for (int r = threadIdx.x; r < ndf; r += blockDim.x) {
    const double v = dv[r];
    int l = 0, h = k;
    while (l < h) { int m = (l + h) >> 1; if (rl[m] < v) l = m + 1; else h = m; }
    a.dfpos[lo + r] = min(a.dfrank[lo + r] + l, nd.hi - lo - 1);
  }
  __syncthreads();
  if (!last) {
    for (int i = threadIdx.x; i < k; i += blockDim.x) a.lam[lo + a.cpos[lo + i]] = rl[i];
    for (int r = threadIdx.x; r < ndf; r += blockDim.x) a.lam[lo + a.dfpos[lo + r]] = dv[r];
  } else {
    const double sc = a.scale[0];
    for (int i = threadIdx.x; i < k; i += blockDim.x) {
      const int p = a.cpos[lo + i];
      if (p >= il - 1 && p <= iu - 1) w_out[p - (il - 1)] = rl[i] * sc;
    }
    for (int r = threadIdx.x; r < ndf; r += blockDim.x) {
      const int p = a.dfpos[lo + r];
      if (p >= il - 1 && p <= iu - 1) w_out[p - (il - 1)] = dv[r] * sc;
    }
  }
}

// Build the grouped-GEMM descriptors: two per node (upper rows, lower rows).
// For the last merge only roots whose final position is in [il-1, iu-1] are
// formed; they are a contiguous range of roots because positions increase.
__global__ void k_descs(DC a, int lev, int nnodes, int last, int il, int iu, double* Zout, int ldz,
                        int* cmap_last) {
  const int node = blockIdx.x * blockDim.x + threadIdx.x;
  if (node >= nnodes) return;
  const NodeR nd = node_range(a.n, a.nleaf, lev, node);
  DGroupDesc* d0 = a.desc + 2 * node;
  DGroupDesc* d1 = d0 + 1;
  d0->m = d1->m = 0; d0->n = d1->n = 0; d0->k = d1->k = 0;
  d0->cmap = d1->cmap = nullptr;
  if (!nd.merge || dc_failed(a)) return;
  const int lo = nd.lo, mid = nd.mid, hi = nd.hi, n = a.n;
  const int* cn = node_cnt(a, lo);
  const int k = cn[C_K], k1 = cn[C_K1], k2 = cn[C_K2];
  int r0 = 0, r1 = k;
  double* C;
  int ldc;
  const int* cmap;
  if (!last) {
    C = a.Z; ldc = n;
    for (int i = 0; i < k; ++i) a.cpos[lo + i] += lo;  // absolute column index in Z
    cmap = a.cpos + lo;
  } else {
    // contiguous range of selected roots
    r0 = k; r1 = k;
    for (int i = 0; i < k; ++i) {
      const int p = a.cpos[lo + i];
      if (p >= il - 1 && p <= iu - 1) { if (r0 == k) r0 = i; r1 = i + 1; }
    }
    for (int i = r0; i < r1; ++i) cmap_last[i - r0] = a.cpos[lo + i] - (il - 1);
    C = Zout; ldc = ldz; cmap = cmap_last;
  }
  const int nn = r1 - r0;
  // upper rows [lo, mid): columns of types 1 and 2
  d0->A = a.Zt + (size_t)lo + (size_t)lo * n;  d0->lda = n;
  d0->B = a.Q + (size_t)lo + (size_t)(lo + r0) * n;  d0->ldb = n;
  d0->C = C + (last ? 0 : lo);  d0->ldc = ldc;
  d0->m = mid - lo; d0->n = nn; d0->k = k1 + k2; d0->cmap = cmap;
  // lower rows [mid, hi): columns of types 2 and 3
  d1->A = a.Zt + (size_t)mid + (size_t)(lo + k1) * n;  d1->lda = n;
  d1->B = a.Q + (size_t)(lo + k1) + (size_t)(lo + r0) * n;  d1->ldb = n;
  d1->C = C + (last ? (mid - lo) : mid);  d1->ldc = ldc;
  d1->m = hi - mid; d1->n = nn; d1->k = k - k1; d1->cmap = cmap;
}

// Descriptors of the tensor-core batched GEMM from the grouped-GEMM ones.
__global__ void k_crt_descs(const DGroupDesc* in, CrtDesc* out, int cnt) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= cnt) return;
  const DGroupDesc g = in[i];
  CrtDesc d;
  d.A = g.A; d.B = g.B; d.C = g.C; d.cmap = g.cmap;
  d.M = g.m; d.N = g.n; d.K = g.k; d.lda = g.lda; d.ldb = g.ldb; d.ldc = g.ldc;
  out[i] = d;
}

// Copy the deflated columns to their final positions.
__global__ void __launch_bounds__(128) k_copy_defl(DC a, int lev, int last, int il, int iu, double* Zout,
                                                   int ldz) {
  if (dc_failed(a)) return;
  NodeR nd;
  node_of(a, lev, blockIdx.x, nd);
  if (!nd.merge) return;
  const int lo = nd.lo, r = blockIdx.x - lo;
  const int* cn = node_cnt(a, lo);
  const int k = cn[C_K], ndf = cn[C_ND];
  if (r >= ndf) return;
  const int p = a.dfpos[lo + r];
  const double* s = a.Zt + (size_t)(lo + k + r) * a.n;
  if (!last) {
    double* d = a.Z + (size_t)(lo + p) * a.n;
    for (int row = lo + threadIdx.x; row < nd.hi; row += blockDim.x) d[row] = s[row];
  } else {
    if (p < il - 1 || p > iu - 1) return;
    double* d = Zout + (size_t)(p - (il - 1)) * ldz;
    for (int row = threadIdx.x; row < a.n; row += blockDim.x) d[row] = s[row];
  }
}

// Single-leaf problem (n <= LS): copy the selected columns out.
__global__ void k_single_out(DC a, int il, int iu, double* w, double* Zout, int ldz) {
  if (dc_failed(a)) return;
  const int m = iu - il + 1;
  for (int i = threadIdx.x; i < m * a.n; i += blockDim.x) {
    const int r = i % a.n, c = i / a.n;
    Zout[(size_t)r + (size_t)c * ldz] = a.Z[(size_t)r + (size_t)(il - 1 + c) * a.n];
  }
  for (int c = threadIdx.x; c < m; c += blockDim.x) w[c] = a.lam[il - 1 + c] * a.scale[0];
}

}  // namespace

size_t stedc_ws_bytes(int n) {
  const size_t nn = (size_t)std::max(n, 1);
  size_t b = 0;
  b += 3 * nn * nn * sizeof(double);               // Z, Zt, Q
  b += 16 * nn * sizeof(double);                   // per-index doubles
  b += 20 * nn * sizeof(int);                      // per-index ints
  b += (nn / LS + 2) * 8 * sizeof(int);            // counters
  b += (nn / LS + 2) * 2 * sizeof(DGroupDesc);     // descriptors
  b += (nn / LS + 2) * 2 * sizeof(CrtDesc);
  b += 64 * 256;
  return b;
}

int stedc_run(Ctx& c, int n, const double* d, const double* e, int il, int iu, double* w, double* Zout,
              int ldz) {
  if (n <= 0 || iu < il) return 0;
  Arena& ar = c.arena;
  const size_t save = ar.off;
  DC a;
  a.n = n;
  a.nleaf = (n + LS - 1) / LS;
  const size_t nn = (size_t)n;
  a.scale = ar.take<double>(1);
  a.dd = ar.take<double>(nn); a.ee = ar.take<double>(nn); a.lam = ar.take<double>(nn);
  a.Z = ar.take<double>(nn * nn); a.Zt = ar.take<double>(nn * nn); a.Q = ar.take<double>(nn * nn);
  a.sD = ar.take<double>(nn); a.sz = ar.take<double>(nn);
  a.stype = ar.take<int>(nn); a.scol = ar.take<int>(nn);
  a.ndq = ar.take<int>(nn); a.ndtype = ar.take<int>(nn); a.ndgrp = ar.take<int>(nn);
  a.ndD = ar.take<double>(nn); a.ndz = ar.take<double>(nn);
  a.dfq = ar.take<int>(nn); a.dfv = ar.take<double>(nn);
  a.rota = ar.take<int>(nn); a.rotb = ar.take<int>(nn);
  a.rotc = ar.take<double>(nn); a.rots = ar.take<double>(nn);
  a.cnt = ar.take<int>((size_t)(a.nleaf + 1) * 8);
  a.rorg = ar.take<int>(nn);
  a.rtau = ar.take<double>(nn); a.rlam = ar.take<double>(nn); a.zhat = ar.take<double>(nn);
  a.dfrank = ar.take<int>(nn); a.cpos = ar.take<int>(nn); a.dfpos = ar.take<int>(nn);
  int* cmap_last = ar.take<int>(nn);
  a.desc = ar.take<DGroupDesc>((size_t)(a.nleaf + 1) * 2);
  a.cdesc = ar.take<CrtDesc>((size_t)(a.nleaf + 1) * 2);
  a.st = c.status;
  if (!ar.ok() || !a.desc) { ar.off = save; return GBHE_EWORKSPACE; }

  ProfScope prof(c.st, GBHE_PROF_STEDC, 0.0, 0.0);
  k_scale_tear<<<1, 1024, 0, c.st>>>(a, d, e);
  count_launch();
  GBHE_CUDA(cudaMemsetAsync(a.Z, 0, nn * nn * sizeof(double), c.st));
  k_leaf<<<(a.nleaf + 3) / 4, 128, 0, c.st>>>(a);
  count_launch();
  GBHE_CUDA(cudaGetLastError());
  if (a.nleaf == 1) {
    k_single_out<<<1, 256, 0, c.st>>>(a, il, iu, w, Zout, ldz);
    count_launch();
    ar.off = save;
    return cudaGetLastError() == cudaSuccess ? 0 : GBHE_ECUDA;
  }
  int levels = 0;
  while ((1 << levels) < a.nleaf) ++levels;
  for (int lev = 1; lev <= levels; ++lev) {
    const int nnodes = (a.nleaf + (1 << lev) - 1) >> lev;
    const int last = (lev == levels);
    // largest node (rows) at this level, for the GEMM grid
    const int span = std::min(n, (1 << lev) * LS);
    k_deflate<<<nnodes, 256, 0, c.st>>>(a, lev);
    count_launch();
    k_rotate<<<nnodes, 256, 0, c.st>>>(a, lev);
    count_launch();
    k_gather<<<n, 128, 0, c.st>>>(a, lev);
    count_launch();
    k_secular<<<(n + 3) / 4, 128, 0, c.st>>>(a, lev);
    count_launch();
    k_zhat<<<(n + 3) / 4, 128, 0, c.st>>>(a, lev);
    count_launch();
    k_qbuild<<<(n + 3) / 4, 128, 0, c.st>>>(a, lev);
    count_launch();
    k_positions<<<nnodes, 256, 0, c.st>>>(a, lev, last, il, iu, w);
    count_launch();
    k_descs<<<(nnodes + 127) / 128, 128, 0, c.st>>>(a, lev, nnodes, last, il, iu, Zout, ldz, cmap_last);
    count_launch();
    GBHE_CUDA(cudaGetLastError());
    // merge products: Z(rows of the node) = Zt Q on the tensor-core engine
    // when its workspace holds the level's batch, else on the FP64 pipe
    const int maxm = std::min(span, (1 << (lev - 1)) * LS);
    int rc;
    if (c.engine == GBHE_ENGINE_CRT && c.crt_ws && span >= 256 &&
        crt_batched_ws_bytes(2 * nnodes, maxm, span, span, 0) <= c.crt_ws_bytes) {
      k_crt_descs<<<(2 * nnodes + 127) / 128, 128, 0, c.st>>>(a.desc, a.cdesc, 2 * nnodes);
      count_launch();
      rc = crt_gemm_batched(c.st, OP_N, OP_N, mk(1.0, 0.0), mk(0.0, 0.0), 0, a.cdesc, 2 * nnodes, maxm, span, span,
                            c.crt_ws, c.crt_ws_bytes, c.status);
    } else {
      rc = dgemm_grouped(c.st, a.desc, 2 * nnodes, span, span, 1.0, 0.0);
    }
    if (rc) { ar.off = save; return rc; }
    k_copy_defl<<<n, 128, 0, c.st>>>(a, lev, last, il, iu, Zout, ldz);
    count_launch();
    GBHE_CUDA(cudaGetLastError());
  }
  ar.off = save;
  return 0;
}

}  // namespace gbhe
