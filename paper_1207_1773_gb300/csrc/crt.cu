// crt.cu -- FP64-accurate GEMM on the FP16 tensor cores by exact modular
// arithmetic (a GB300-specific replacement for FP64 level-3 products: this
// GPU's FP64 pipes, scalar and tensor alike, deliver about 1 TFLOP/s while
// its FP16 tensor cores deliver hundreds).
//
//   1. Scaling.  Every row i of op(A) is scaled by 2^(52 - ea_i) and every
//      column j of op(B) by 2^(52 - eb_j), ea/eb the smallest exponents with
//      |x| < 2^e over the row/column, and rounded to integers |v| <= 2^52
//      (integer bit manipulation, exact apart from that rounding, which is at
//      the level of the last bit of the largest element of the row/column).
//   2. Residues.  The integers are reduced modulo NMOD = 16 pairwise coprime
//      moduli p_l <= 256 (product M ~ 2^125) to symmetric residues
//      -128 <= r <= 127, stored as signed bytes (the one even modulus, 256,
//      takes -128 for its residue 128).  Complex operands give two planes
//      (Re, Im) per modulus.  The reduction runs in FP32 on exact integers:
//      four signed 13-bit limbs of v, t = l0 + l1 w1 + l2 w2 + l3 w3 with w_i
//      the symmetric residues of 2^(13 i) (|t| < 2^23), r = t - p rint(t / p)
//      (|r| <= p/2 + 1 <= 128).
//   3. Products.  For each modulus the residue products run on tcgen05.mma
//      kind::f16 (f16 -> f32 accumulators in tensor memory; the producer
//      warps widen each staged byte tile to FP16, exactly): real operands
//      one product, complex operands Re C = Ar Br - Ai Bi and
//      Im C = Ar Bi + Ai Br (the subtraction by the MMA's negate-A bit).
//      Every partial sum of at most 2^23 / 128^2 = 512 products of
//      |r| <= 128 (chunks of 512 contraction terms real, 256 complex, which add
//      two products per term) is an integer below 2^23, so the FP32
//      accumulation is exact; after each chunk the sums are reduced mod p_l
//      and the residues of Re C and Im C are stored as bytes.
//   4. Reconstruction.  C_int = sum_l c_l W_l - q M (CRT, W_l = M_l (M_l^-1
//      mod p_l)) in 160-bit integer arithmetic, q = round(sum_l c_l y_l/p_l)
//      (the true value is far inside (-M/2, M/2): |C_int| <= K 2^105 < M/8
//      for K <= 2^16, and the FP32 estimate of q errs by less than 2^-8),
//      then converted to the nearest double and scaled by
//      2^(ea_i + eb_j - 104) -- all with integer instructions.
// The result equals the exact product of the rounded operands, rounded once
// to double: as accurate as an FP64 GEMM for operands whose rows/columns are
// not strongly graded.
#include <algorithm>
#include <cstdint>
#include <cstring>
#include <cuda_fp16.h>
#include "internal.cuh"

namespace gbhe {
namespace {

constexpr int NMOD = 16;
constexpr int CBM = 128, CBN = 64, CBK = 32;  // output tile of the residue products; K padding
constexpr int KMAX = 65536;          // contraction bound of the margin argument above

const int h_mod[NMOD] = {256, 255, 253, 251, 247, 241, 239, 233, 229, 227, 223, 211, 199, 197, 193, 191};

__constant__ int c_p[NMOD];
__constant__ float c_pinv[NMOD];
__constant__ float c_frac[NMOD];         // y_l / p_l
__constant__ unsigned c_W[NMOD][4];      // W_l (128-bit, little-endian words)
__constant__ unsigned c_M[4];            // M
__constant__ float c_kw[NMOD][3];        // symmetric residues of 2^13, 2^26, 2^39 mod p (limb weights)

bool g_const_ready[MAX_DEVICES] = {};

// The number-theory tables of the engine, computed on the host (the one
// source of what init_constants copies to the device and gbhe_crt_tables
// returns).
struct HostTables {
  int p[NMOD];
  float pinv[NMOD], frac[NMOD];
  unsigned W[NMOD][4], M[4];
  int kw[NMOD][3];  // symmetric residues of 2^13, 2^26, 2^39 modulo p_l
};

void crt_tables(HostTables& t) {
  typedef unsigned __int128 u128;
  u128 M = 1;
  for (int l = 0; l < NMOD; ++l) M *= (u128)h_mod[l];
  for (int l = 0; l < NMOD; ++l) {
    const int pl = h_mod[l];
    const u128 Ml = M / (u128)pl;
    const int mr = (int)(Ml % (u128)pl);
    int y = 0;
    for (int v = 1; v < pl; ++v)
      if ((mr * v) % pl == 1) { y = v; break; }
    const u128 Wl = (Ml * (u128)y) % M;
    for (int w = 0; w < 4; ++w) t.W[l][w] = (unsigned)(Wl >> (32 * w));
    t.p[l] = pl;
    t.pinv[l] = 1.0f / (float)pl;
    t.frac[l] = (float)((double)y / (double)pl);
    for (int i = 0; i < 3; ++i) {
      const int r = (int)(((u128)1 << (13 * (i + 1))) % (u128)pl);
      t.kw[l][i] = r > pl / 2 ? r - pl : r;
    }
  }
  for (int w = 0; w < 4; ++w) t.M[w] = (unsigned)(M >> (32 * w));
}

int init_constants() {
  const int dev = device_slot();
  if (dev < 0) return GBHE_ECUDA;
  if (g_const_ready[dev]) return 0;
  HostTables t;
  crt_tables(t);
  GBHE_CUDA(cudaMemcpyToSymbol(c_p, t.p, sizeof(t.p)));
  GBHE_CUDA(cudaMemcpyToSymbol(c_pinv, t.pinv, sizeof(t.pinv)));
  GBHE_CUDA(cudaMemcpyToSymbol(c_frac, t.frac, sizeof(t.frac)));
  GBHE_CUDA(cudaMemcpyToSymbol(c_W, t.W, sizeof(t.W)));
  GBHE_CUDA(cudaMemcpyToSymbol(c_M, t.M, sizeof(t.M)));
  float kw[NMOD][3];
  for (int l = 0; l < NMOD; ++l)
    for (int i = 0; i < 3; ++i) kw[l][i] = (float)t.kw[l][i];
  GBHE_CUDA(cudaMemcpyToSymbol(c_kw, kw, sizeof(kw)));
  g_const_ready[dev] = true;
  return 0;
}

// ------------------------------------------------------------------ operand access
// Element (r, k) of the operand: for op(A) r is the row, for op(B) r is the
// column of op(B); k runs along the contraction.  `mode` encodes the storage:
//   0: X[r + k ld]            (A with N;  B with T or C)
//   1: X[k + r ld]            (A with T or C;  B with N)
//   2: Hermitian, lower stored: r >= k ? X[r + k ld] : conj X[k + r ld]
// `cj` conjugates every element (A with C, B with C).
struct Operand {
  const void* X;
  int ld, R, K, mode, cj, cplx;
};

__device__ __forceinline__ double2 op_elem(const Operand& o, int r, int k) {
  double2 v;
  if (o.cplx) {
    const double2* X = reinterpret_cast<const double2*>(o.X);
    if (o.mode == 0) v = X[(size_t)r + (size_t)k * o.ld];
    else if (o.mode == 1) v = X[(size_t)k + (size_t)r * o.ld];
    else if (r >= k) { v = X[(size_t)r + (size_t)k * o.ld]; if (r == k) v.y = 0.0; }
    else { v = X[(size_t)k + (size_t)r * o.ld]; v.y = -v.y; }
    if (o.cj) v.y = -v.y;
  } else {
    const double* X = reinterpret_cast<const double*>(o.X);
    v.x = (o.mode == 0) ? X[(size_t)r + (size_t)k * o.ld] : X[(size_t)k + (size_t)r * o.ld];
    v.y = 0.0;
  }
  return v;
}

__device__ __forceinline__ int exp_bound(double x) {
  // smallest e with |x| < 2^e for normal x; zero/denormal -> -1100
  const long long b = __double_as_longlong(x);
  const int E = (int)((b >> 52) & 0x7FF);
  return E == 0 ? -1100 : E - 1022;
}

// Max exponent per r over k.  Tile 32 (r) x 32 (k) per block of 32 x 8
// threads; the contiguous storage direction maps to threadIdx.x.
__device__ __forceinline__ void op_exponents_tile(const Operand& o, int* e, int bx, int by) {
  __shared__ int tile[32][33];
  const int r0 = bx * 32, k0 = by * 32;
  if (r0 >= o.R || k0 >= o.K) return;
  const int tx = threadIdx.x, ty = threadIdx.y;
  const bool r_contig = (o.mode == 0) || (o.mode == 2 && r0 >= k0 + 31);
  for (int q = ty; q < 32; q += 8) {
    const int r = r_contig ? r0 + tx : r0 + q;
    const int k = r_contig ? k0 + q : k0 + tx;
    int ev = -1100;
    if (r < o.R && k < o.K) {
      const double2 v = op_elem(o, r, k);
      ev = max(exp_bound(v.x), exp_bound(v.y));
    }
    if (r_contig) tile[tx][q] = ev; else tile[q][tx] = ev;
  }
  __syncthreads();
  if (ty == 0 && r0 + tx < o.R) {
    int m = -1100;
    for (int q = 0; q < 32; ++q) m = max(m, tile[tx][q]);
    atomicMax(&e[r0 + tx], m);
  }
}

// Both operands in one launch: blocks x < gA take op(A), the rest op(B).
__global__ void k_op_exponents(Operand oa, int* ea, Operand ob, int* eb, int gA) {
  const bool isA = blockIdx.x < (unsigned)gA;
  op_exponents_tile(isA ? oa : ob, isA ? ea : eb, isA ? blockIdx.x : blockIdx.x - gA, blockIdx.y);
}

__global__ void k_fill_int(int* p, int n, int v) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) p[i] = v;
}

// Residue planes: P[(l * ncomp + c) * R * Kp + r * Kp + k] (signed bytes),
// symmetric residues of the scaled integer of element (r, k); zero for k >= K.
__device__ __forceinline__ void op_residues_tile(const Operand& o, const int* e, int Kp, int8_t* P, int bx, int by) {
  __shared__ double2 tile[32][33];
  const int r0 = bx * 32, k0 = by * 32;
  if (r0 >= o.R || k0 >= Kp) return;
  const int tx = threadIdx.x, ty = threadIdx.y;
  const bool r_contig = (o.mode == 0) || (o.mode == 2 && r0 >= k0 + 31);
  for (int q = ty; q < 32; q += 8) {
    const int r = r_contig ? r0 + tx : r0 + q;
    const int k = r_contig ? k0 + q : k0 + tx;
    double2 v = make_double2(0.0, 0.0);
    if (r < o.R && k < o.K) v = op_elem(o, r, k);
    if (r_contig) tile[tx][q] = v; else tile[q][tx] = v;
  }
  __syncthreads();
  const int ncomp = o.cplx ? 2 : 1;
  const size_t plane = (size_t)o.R * Kp;
  // each thread: one row, four consecutive k (one 4-byte store per plane)
  const int t = ty * 32 + tx, q = t >> 3, kq = (t & 7) * 4;
  const int r = r0 + q, k = k0 + kq;
  if (r >= o.R) return;
  const int er = e[r];
  // scaled integers (|v| <= 2^52) as four signed 13-bit limbs, exact in FP32
  float lim[4][2][4];
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    const double2 v = tile[q][kq + u];
#pragma unroll
    for (int part = 0; part < 2; ++part) {
      const double x = part ? v.y : v.x;
      const long long bits = __double_as_longlong(x);
      const int E = (int)((bits >> 52) & 0x7FF);
      unsigned long long mag = 0;
      if (E != 0 && k + u < o.K) {
        const unsigned long long mant = ((unsigned long long)bits & 0xFFFFFFFFFFFFFull) | (1ull << 52);
        const int sh = er - (E - 1023);  // right shift (>= 1)
        if (sh <= 60) mag = (mant + (1ull << (sh - 1))) >> sh;
      }
      const float sg = bits < 0 ? -1.f : 1.f;
      lim[u][part][0] = sg * (float)(unsigned)(mag & 0x1FFFu);
      lim[u][part][1] = sg * (float)(unsigned)((mag >> 13) & 0x1FFFu);
      lim[u][part][2] = sg * (float)(unsigned)((mag >> 26) & 0x1FFFu);
      lim[u][part][3] = sg * (float)(unsigned)(mag >> 39);  // <= 2^13
    }
  }
#pragma unroll
  for (int l = 0; l < NMOD; ++l) {
    const float p = (float)c_p[l], pinv = c_pinv[l], w1 = c_kw[l][0], w2 = c_kw[l][1], w3 = c_kw[l][2];
#pragma unroll
    for (int part = 0; part < 2; ++part) {
      if (part == 1 && !o.cplx) break;
      unsigned pk = 0;
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        // t = v mod-equivalent, an integer below 2^23 (every partial sum exact)
        const float t = fmaf(lim[u][part][3], w3, fmaf(lim[u][part][2], w2, fmaf(lim[u][part][1], w1,
                                                                                   lim[u][part][0])));
        float rv = fmaf(-rintf(t * pinv), p, t);  // symmetric, |r| <= 128
        if (rv > 127.f) rv -= p;                  // 128 only for p = 256: -128 is the same residue
        pk |= ((unsigned)(int)rv & 0xFFu) << (8 * u);
      }
      // Kp is a multiple of 32 and k of 4: the 4-byte store is aligned and in the row
      int8_t* dst = P + (size_t)(l * ncomp + part) * plane + (size_t)r * Kp + k;
      *reinterpret_cast<unsigned*>(dst) = pk;
    }
  }
}

__global__ void k_op_residues(Operand oa, const int* ea, int8_t* PA, Operand ob, const int* eb, int8_t* PB, int gA,
                              int Kp) {
  const bool isA = blockIdx.x < (unsigned)gA;
  op_residues_tile(isA ? oa : ob, isA ? ea : eb, Kp, isA ? PA : PB, isA ? blockIdx.x : blockIdx.x - gA, blockIdx.y);
}

// ---- batched forms: entry z of a device descriptor array per blockIdx.z
__device__ __forceinline__ Operand desc_operand(const CrtDesc& d, int isA, int op, int cplx) {
  Operand o;
  o.cplx = cplx;
  o.cj = (op == OP_C) ? 1 : 0;
  if (isA) {
    o.X = d.A; o.ld = d.lda; o.R = d.M; o.K = d.K;
    o.mode = (op == OP_N) ? 0 : (op == OP_H ? 2 : 1);
  } else {
    o.X = d.B; o.ld = d.ldb; o.R = d.N; o.K = d.K;
    o.mode = (op == OP_N) ? 1 : 0;
  }
  return o;
}

// Both operands of every entry in one launch: blocks x < gA = ceil(maxM/32)
// take op(A_z), the rest op(B_z).
__global__ void k_bop_exponents(const CrtDesc* D, int opA, int opB, int cplx, int maxM, int maxN, int* ea, int* eb,
                                int gA) {
  const bool isA = blockIdx.x < (unsigned)gA;
  const Operand o = desc_operand(D[blockIdx.z], isA ? 1 : 0, isA ? opA : opB, cplx);
  int* e = isA ? ea + (size_t)blockIdx.z * maxM : eb + (size_t)blockIdx.z * maxN;
  op_exponents_tile(o, e, isA ? blockIdx.x : blockIdx.x - gA, blockIdx.y);
}

__global__ void k_bop_residues(const CrtDesc* D, int opA, int opB, int cplx, int maxM, int maxN, const int* ea,
                               const int* eb, int Kp, int8_t* PA, int8_t* PB, int gA) {
  const bool isA = blockIdx.x < (unsigned)gA;
  const Operand o = desc_operand(D[blockIdx.z], isA ? 1 : 0, isA ? opA : opB, cplx);
  const int maxR = isA ? maxM : maxN;
  const size_t entry = (size_t)NMOD * (cplx ? 2 : 1) * maxR * Kp;
  op_residues_tile(o, (isA ? ea : eb) + (size_t)blockIdx.z * maxR, Kp, (isA ? PA : PB) + blockIdx.z * entry,
                   isA ? blockIdx.x : blockIdx.x - gA, blockIdx.y);
}

__global__ void k_fill_int_batched(int* p, size_t n, int v) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) p[i] = v;
}

// ------------------------------------------------------------------ residue products
__device__ __forceinline__ void cp16(void* smem, const void* g, bool pred) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(s), "l"(g), "r"(pred ? 16 : 0) : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

// x - p rint(x / p) for an integer-valued x with |x| <= 2^24: an integer of
// magnitude at most p/2 + 1, exact in FP32 (the FMA rounds nothing away).
__device__ __forceinline__ float red_sym(float x, float p, float pinv) { return fmaf(-rintf(x * pinv), p, x); }

// Residues of one output tile in the tile-major layout shared with the
// reconstruction: tile t = by * TM + bx (TM = ceil(maxM / CBM)), and for
// modulus l and component c a CBM x CBN byte block, column-major, at
// Out + ((t * NMOD + l) * ncout + c) * CBM * CBN.
constexpr int OTILE = CBM * CBN;
constexpr int OPITCH = CBM + 16;  // smem column pitch of the staged tile (bank-spread, 16 B aligned)

// ------------------------------------------------------------------ residue products on tcgen05
// tcgen05.mma kind::f16 (FP16 operands from shared memory, FP32 accumulators
// in tensor memory), issued by one thread; operands staged by cp.async in the
// no-swizzle K-major core-matrix layout (8 rows x 16 bytes per core matrix,
// K-adjacent core matrices 128 B apart, 8-row groups 512 B apart).
//
// One CTA computes a UBM x BN output tile (BN = 128, or 64 for products with
// at most 64 columns, where a wider tile would leave half of every MMA idle)
// for `mpc` consecutive moduli.  Its
// work is a flat sequence of K tiles over those moduli, cut into units (one
// exact chunk of one modulus).  Each unit accumulates Re and Im (one
// accumulator for real operands) in one of two TMEM buffers; while the
// tensor cores run unit u, the threads fold unit u - 1 into the running
// residues and, at the end of a modulus, write its bytes in the tile-major
// layout read by the reconstruction (two CBN-wide tiles per CTA).
constexpr int UBM = 128, UBN = 128, UBK = 32;
constexpr int UTHREADS = 256;
constexpr int U_APL = UBM * UBK * 2;  // bytes of one plane tile of op(A)
static_assert(UBM == CBM && UBN == 2 * CBN, "a wide CTA tile covers two tiles of the residue layout");
// Operands travel as signed bytes (half the bytes of FP16 through L2 and
// HBM): each K tile is copied by cp.async into a byte staging slot, and the
// thread that copied a 16-byte chunk widens it to FP16 into the stage the
// tensor cores read (so no barrier is needed between copy and widening).
template <bool CPLX, int BN>
struct UCfg {
  static_assert(BN == UBN || BN == CBN, "tile width 128 or 64");
  static constexpr int NC = CPLX ? 2 : 1;         // planes per operand = accumulators
  static constexpr int F = 3;                     // FP16 stages read by the tensor cores
  static constexpr int S8 = 5;                    // byte staging slots (copies run S8 - 1 K tiles ahead)
  static constexpr int KC_TERMS = CPLX ? 256 : 512;  // exact chunk (contraction terms)
  static constexpr int BPL = BN * UBK * 2;           // bytes of one plane tile of op(B)
  static constexpr unsigned BUFC = NC * BN;          // TMEM columns of one buffer
  static constexpr unsigned COLS = 2 * BUFC;         // allocation (two buffers; a power of 2 >= 32)
  static constexpr int NRES = BN / 2;                // columns per epilogue thread
  static constexpr int STB = NC * (U_APL + BPL);     // bytes per FP16 stage
  static constexpr int ST8 = NC * (UBM + BN) * UBK;  // bytes per byte staging slot
  static constexpr int NCH_A = NC * UBM * 2;         // 16-byte chunks of op(A) per K tile (two per row)
  static constexpr int NCH = NC * (UBM + BN) * 2;    // 16-byte chunks per K tile
  static constexpr size_t SMEM =
      (size_t)F * STB + (size_t)S8 * ST8 + (size_t)NC * BN * OPITCH + 8 * (F + 3) + 16;
};

// Two signed bytes of `ub` (already biased by +128 per byte), selected by
// `sel`, to an FP16 pair: the byte placed under the exponent bits of 1024
// (0x64uu = 1024 + u) minus 1152 gives u - 128 exactly.
__device__ __forceinline__ unsigned h2_of_bytes(unsigned ub, unsigned sel) {
  unsigned out;
  asm("{\n\t.reg .b32 t;\n\tprmt.b32 t, %1, %2, %3;\n\tsub.rn.f16x2 %0, t, %4;\n\t}"
      : "=r"(out)
      : "r"(ub), "r"(0x64646464u), "r"(sel), "r"(0x64806480u));
  return out;
}
// 16 signed bytes (contraction index k .. k+15 of one row) to the two FP16
// core-matrix rows k .. k+7 (lo) and k+8 .. k+15 (hi).
__device__ __forceinline__ void widen16(const uint4 v, uint4& lo, uint4& hi) {
  const unsigned a = v.x ^ 0x80808080u, b = v.y ^ 0x80808080u, c = v.z ^ 0x80808080u, d = v.w ^ 0x80808080u;
  lo = make_uint4(h2_of_bytes(a, 0x4140u), h2_of_bytes(a, 0x4342u), h2_of_bytes(b, 0x4140u), h2_of_bytes(b, 0x4342u));
  hi = make_uint4(h2_of_bytes(c, 0x4140u), h2_of_bytes(c, 0x4342u), h2_of_bytes(d, 0x4140u), h2_of_bytes(d, 0x4342u));
}

// Copy (issue) and widening of K tile `it` by the `nthr` threads t = 0 ..
// nthr - 1 of a CTA: chunk i < NCH_A is row r = (i % (2 UBM)) / 2, half hk =
// i % 2 of plane c = i / (2 UBM) of op(A); the rest likewise of op(B).  Rows
// beyond the matrix are zero-filled by the copy (source size 0).
template <bool CPLX, int BN, int NTHR>
__device__ __forceinline__ void stage_issue(unsigned char* s8, const int8_t* PA, const int8_t* PB, size_t planeA,
                                            size_t planeB, int l, int k0, int Kp, int m0, int n0, int M, int N,
                                            int t) {
  using CF = UCfg<CPLX, BN>;
  const int8_t* Al = PA + (size_t)l * CF::NC * planeA;
  const int8_t* Bl = PB + (size_t)l * CF::NC * planeB;
#pragma unroll
  for (int i = t; i < CF::NCH_A; i += NTHR) {
    const int c = i / (UBM * 2), rem = i % (UBM * 2), r = rem >> 1, hk = rem & 1;
    const bool ok = (m0 + r) < M;
    cp16(s8 + i * 16, Al + (size_t)c * planeA + (size_t)(ok ? m0 + r : 0) * Kp + k0 + hk * 16, ok);
  }
#pragma unroll
  for (int i = CF::NCH_A + t; i < CF::NCH; i += NTHR) {
    const int j = i - CF::NCH_A, c = j / (BN * 2), rem = j % (BN * 2), r = rem >> 1, hk = rem & 1;
    const bool ok = (n0 + r) < N;
    cp16(s8 + i * 16, Bl + (size_t)c * planeB + (size_t)(ok ? n0 + r : 0) * Kp + k0 + hk * 16, ok);
  }
}
template <bool CPLX, int BN, int NTHR>
__device__ __forceinline__ void stage_widen(const unsigned char* s8, unsigned char* sA, int t) {
  using CF = UCfg<CPLX, BN>;
  unsigned char* sB = sA + CF::NC * U_APL;
#pragma unroll
  for (int i = t; i < CF::NCH_A; i += NTHR) {
    const int c = i / (UBM * 2), rem = i % (UBM * 2), r = rem >> 1, hk = rem & 1;
    uint4 lo, hi;
    widen16(*reinterpret_cast<const uint4*>(s8 + i * 16), lo, hi);
    unsigned char* d = sA + c * U_APL + ((r >> 3) * 4 + 2 * hk) * 128 + (r & 7) * 16;
    *reinterpret_cast<uint4*>(d) = lo;
    *reinterpret_cast<uint4*>(d + 128) = hi;
  }
#pragma unroll
  for (int i = CF::NCH_A + t; i < CF::NCH; i += NTHR) {
    const int j = i - CF::NCH_A, c = j / (BN * 2), rem = j % (BN * 2), r = rem >> 1, hk = rem & 1;
    uint4 lo, hi;
    widen16(*reinterpret_cast<const uint4*>(s8 + i * 16), lo, hi);
    unsigned char* d = sB + c * CF::BPL + ((r >> 3) * 4 + 2 * hk) * 128 + (r & 7) * 16;
    *reinterpret_cast<uint4*>(d) = lo;
    *reinterpret_cast<uint4*>(d + 128) = hi;
  }
}

__device__ __forceinline__ unsigned smem_addr(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

// shared-memory matrix descriptor: start address, leading (K) and stride (M/N)
// byte offsets between core matrices, descriptor version 1, no swizzle
__device__ __forceinline__ unsigned long long umma_sdesc(unsigned addr, unsigned lbo, unsigned sbo) {
  unsigned long long d = (unsigned long long)((addr & 0x3FFFFu) >> 4);
  d |= (unsigned long long)((lbo >> 4) & 0x3FFFu) << 16;
  d |= (unsigned long long)((sbo >> 4) & 0x3FFFu) << 32;
  d |= 1ull << 46;
  return d;
}

__device__ __forceinline__ void umma_f16(unsigned tmem_d, unsigned long long da, unsigned long long db, unsigned idesc,
                                         unsigned accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
      "l"(da), "l"(db), "r"(idesc), "r"(accumulate));
}

__device__ __forceinline__ void umma_commit(unsigned bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}

// Wait until the phase of parity `parity` of the mbarrier has completed, for
// at most GBHE_WAIT_NS of %globaltimer; false on expiry.
__device__ __forceinline__ bool mbar_wait(unsigned bar, unsigned parity) {
  const unsigned long long t0 = gtimer();
  while (true) {
    unsigned done;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(bar), "r"(parity)
        : "memory");
    if (done) return true;
    if (gtimer() - t0 > GBHE_WAIT_NS) return false;
  }
}

__device__ __forceinline__ void tmem_ld16(unsigned addr, float (&v)[16]) {
  unsigned r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(addr));
#pragma unroll
  for (int x = 0; x < 16; ++x) v[x] = __uint_as_float(r[x]);
}

// grid (TM * TN2 tiles in grouped order, 1, (NMOD/mpc) * nbatch), 256 threads;
// TM = ceil(maxM/UBM), TN2 = ceil(maxN/BN).  PA: residue planes of op(A)
// (R = M), PB: of op(B) (R = N); both K-padded to Kp.  Batched form
// (D != nullptr): blockIdx.z / (NMOD/mpc) is the entry; entry regions of the
// planes and outputs are sized for maxM / maxN, the layout inside an entry's
// planes uses the entry's own M, N.  lower != 0 skips tiles strictly above the
// diagonal (their outputs are never read).  Timeouts of the bounded waits
// record GBHE_ETIMEOUT in status[ST_ERR].  Used for products whose moduli span
// several exact chunks (Kp > KC_TERMS); single-chunk products use
// k_crt_umma_ws below.
template <bool CPLX, int BN>
__global__ void __launch_bounds__(UTHREADS, 1) k_crt_umma(const int8_t* PA, const int8_t* PB, int M, int N, int Kp,
                                                         unsigned char* Out, const CrtDesc* D, int maxM, int maxN,
                                                         int lower, int mpc, int* status) {
  using CF = UCfg<CPLX, BN>;
  constexpr int NC = CF::NC;
  constexpr int F = CF::F, S8 = CF::S8, LAG = S8 - 1;
  constexpr int STB = CF::STB;
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* stage8 = smem_raw + F * STB;
  unsigned char* stile = stage8 + S8 * CF::ST8;
  // bars: [0, F) FP16 stage empty, F + b accumulator b full, F + 2 drain (before TMEM is freed)
  unsigned long long* bars = reinterpret_cast<unsigned long long*>(stile + NC * BN * OPITCH);
  unsigned* tslot = reinterpret_cast<unsigned*>(bars + F + 3);
  volatile int* sabort = reinterpret_cast<volatile int*>(tslot + 1);

  const int TM = (maxM + UBM - 1) / UBM, TN2 = (maxN + BN - 1) / BN;
  const int TN = (maxN + CBN - 1) / CBN;  // tiles of the residue layout
  const int ngrp = NMOD / mpc;
  const int entry = blockIdx.z / ngrp, grp = blockIdx.z % ngrp;
  // grouped order: eight tile rows at a time, so that concurrent CTAs share operand tiles in L2
  int bx, by;
  {
    const int pid = blockIdx.x, GM = 8;
    const int first = (pid / (GM * TN2)) * GM, gm = min(TM - first, GM);
    bx = first + (pid % (GM * TN2)) % gm;
    by = (pid % (GM * TN2)) / gm;
  }
  if (D) {
    M = D[entry].M;
    N = D[entry].N;
    PA += (size_t)entry * NMOD * NC * maxM * Kp;
    PB += (size_t)entry * NMOD * NC * maxN * Kp;
    Out += (size_t)entry * TM * TN * NMOD * NC * OTILE;
  }
  const int m0 = bx * UBM, n0 = by * BN;
  if (m0 >= M || n0 >= N) return;
  if (lower && m0 + UBM - 1 < n0) return;
  const int t = threadIdx.x, lane = t & 31, w = t >> 5;
  const int q = w & 3, h = w >> 2;  // TMEM lane quarter and column half of this warp
  const int l0 = grp * mpc;
  const size_t planeA = (size_t)M * Kp, planeB = (size_t)N * Kp;

  if (t == 0) {
    for (int i = 0; i < F + 3; ++i) asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(bars + i)));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    *sabort = 0;
  }
  if (w == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(tslot)),
                 "r"(CF::COLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const unsigned tmem = *tslot;

  const int ktiles = Kp / UBK;
  constexpr int KTC = CF::KC_TERMS / UBK;  // K tiles per exact chunk
  const int nch = (ktiles + KTC - 1) / KTC;
  const int iters = mpc * ktiles;
  // instruction descriptor: f32 accumulator, f16 A and B, both K-major, N, M
  const unsigned idesc = (1u << 4) | ((unsigned)(BN >> 3) << 17) | ((unsigned)(UBM >> 4) << 24);
  const unsigned idesc_negA = idesc | (1u << 13);

  // copies of K tile `it` into its byte slot; widening into its FP16 stage
  auto issue = [&](int it) {
    stage_issue<CPLX, BN, UTHREADS>(stage8 + (it % S8) * CF::ST8, PA, PB, planeA, planeB, l0 + it / ktiles,
                                    (it % ktiles) * UBK, Kp, m0, n0, M, N, t);
  };
  auto widen = [&](int it) {
    stage_widen<CPLX, BN, UTHREADS>(stage8 + (it % S8) * CF::ST8, smem_raw + (it % F) * STB, t);
  };

  // running residues of this thread's row (32 q + lane) and NRES columns (NRES h + x)
  constexpr int NRES = CF::NRES;
  float res[NC][NRES];
#pragma unroll
  for (int c = 0; c < NC; ++c)
#pragma unroll
    for (int x = 0; x < NRES; ++x) res[c][x] = 0.f;

  auto epilogue = [&](int u) {
    const int b = u & 1;
    if (!mbar_wait(smem_addr(bars + F + b), (unsigned)(u >> 1) & 1u)) {
      *sabort = 1;
      if (status) set_err_once(status, GBHE_ETIMEOUT);
    }
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const int l = l0 + u / nch;
    const float p = (float)c_p[l], pinv = c_pinv[l];
    const unsigned tb = tmem + ((unsigned)(32 * q) << 16) + (unsigned)b * CF::BUFC + (unsigned)(NRES * h);
    const int il = 32 * q + lane;
#pragma unroll
    for (int sl = 0; sl < NRES / 16; ++sl) {
      float P[NC][16];
#pragma unroll
      for (int c = 0; c < NC; ++c) tmem_ld16(tb + c * BN + sl * 16, P[c]);
      asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
      for (int c = 0; c < NC; ++c)
#pragma unroll
        for (int x = 0; x < 16; ++x) res[c][sl * 16 + x] += red_sym(P[c][x], p, pinv);
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    if ((u % nch) == nch - 1) {
#pragma unroll
      for (int x = 0; x < NRES; ++x) {
#pragma unroll
        for (int c = 0; c < NC; ++c) {
          float v = red_sym(res[c][x], p, pinv);
          if (v < 0.f) v += p;  // [0, p)
          stile[(c * BN + NRES * h + x) * OPITCH + il] = (unsigned char)(int)v;
          res[c][x] = 0.f;
        }
      }
      __syncthreads();
      // the BN / CBN layout tiles of this CTA
      const int nu = (min(UBM, M - m0) + 15) / 16, ncol = min(BN, N - n0);
      for (int i = t; i < NC * ncol * nu; i += UTHREADS) {
        const int c = i / (ncol * nu), rem = i % (ncol * nu), jl = rem / nu, uu = rem % nu;
        const int tile = ((BN / CBN) * by + jl / CBN) * TM + bx;
        unsigned char* dst = Out + ((size_t)tile * NMOD + l) * NC * OTILE;
        const uint4 v = *reinterpret_cast<const uint4*>(stile + (c * BN + jl) * OPITCH + uu * 16);
        *reinterpret_cast<uint4*>(dst + ((size_t)c * CBN + (jl % CBN)) * CBM + uu * 16) = v;
      }
    }
  };

  for (int s = 0; s < LAG; ++s) {
    if (s < iters) issue(s);
    cp_commit();
  }
  bool aborted = false;
  for (int it = 0; it < iters; ++it) {
    const int f = it % F;
    const int kt = it % ktiles;
    const int u = (it / ktiles) * nch + kt / KTC;
    const bool unit_start = (kt % KTC) == 0;
    cp_wait<LAG - 1>();  // this thread's copies of K tile `it` have landed
    // FP16 stage f is free once the products of K tile it - F have completed
    if (it >= F && !mbar_wait(smem_addr(bars + f), (unsigned)((it / F) - 1) & 1u)) {
      *sabort = 1;
      if (status) set_err_once(status, GBHE_ETIMEOUT);
    }
    widen(it);
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    // one decision for the whole CTA: a timeout recorded by any thread before
    // this barrier stops every thread at the same iteration
    const int stop = __syncthreads_or(*sabort);
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (stop) { aborted = true; break; }
    if (t == 0) {
      const unsigned dbuf = tmem + (unsigned)(u & 1) * CF::BUFC;
      const unsigned sA = smem_addr(smem_raw + f * STB), sB = sA + NC * U_APL;
#pragma unroll
      for (int kk = 0; kk < UBK / 16; ++kk) {
        const unsigned first = (unit_start && kk == 0) ? 0u : 1u;
        const unsigned long long ar = umma_sdesc(sA + kk * 256, 128, 512);
        const unsigned long long br = umma_sdesc(sB + kk * 256, 128, 512);
        umma_f16(dbuf, ar, br, idesc, first);  // Re (or the real product) += Ar Br
        if constexpr (CPLX) {
          const unsigned long long ai = umma_sdesc(sA + U_APL + kk * 256, 128, 512);
          const unsigned long long bi = umma_sdesc(sB + CF::BPL + kk * 256, 128, 512);
          umma_f16(dbuf, ai, bi, idesc_negA, 1u);     // Re -= Ai Bi
          umma_f16(dbuf + BN, ar, bi, idesc, first);  // Im += Ar Bi
          umma_f16(dbuf + BN, ai, br, idesc, 1u);     // Im += Ai Br
        }
      }
      umma_commit(smem_addr(bars + f));
      if ((kt % KTC) == KTC - 1 || kt == ktiles - 1) umma_commit(smem_addr(bars + F + (u & 1)));
    }
    // the byte slot of K tile it + LAG is the one this thread widened at it - 1
    if (it + LAG < iters) issue(it + LAG);
    cp_commit();
    if (unit_start && u > 0) epilogue(u - 1);
  }
  if (!aborted) epilogue(mpc * nch - 1);
  cp_wait<0>();
  // TMEM is freed only after every MMA this CTA issued has completed: the
  // issuing thread commits once more and waits for that commit (bounded), also
  // on the path that gave up early
  if (t == 0) {
    umma_commit(smem_addr(bars + F + 2));
    if (!mbar_wait(smem_addr(bars + F + 2), 0u) && status) set_err_once(status, GBHE_ETIMEOUT);
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (w == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(CF::COLS));
}

// Warp-specialised form for products whose moduli are each one exact chunk
// (Kp <= KC_TERMS: the K <= 256 updates of the blocked factorisations, the
// panel updates and the back-transform's block reflectors).  Warps 0-3 stage
// operands with cp.async, warp 4 issues the MMAs (one lane), warps 5-12 (two
// per TMEM lane quarter) drain the TMEM buffer of the previous modulus while
// the tensor cores work on the next one.  Handshakes: per stage "ready" (the
// 128 producers, each after its own copies of the stage completed and were
// fenced for the tensor cores) and "empty" (MMA completion), per TMEM buffer
// "full" (MMA completion) and "drained" (the 256 epilogue threads).  The
// producers copy byte tiles WS_LAG K tiles ahead of the tile they widen and
// report ready, so the MMA warp never waits on the copies of the stage it
// just read.
// The epilogue stores each residue byte straight from its register to the
// tile-major output layout (a warp covers 32 consecutive rows of one column:
// one 32-byte segment per store), so no shared-memory staging tile is needed
// and the shared memory goes to a deeper operand pipeline.
// Grid and arguments as for k_crt_umma, 384 threads.
constexpr int WS_F = 4, WS_S8 = 4, WS_LAG = WS_S8 - 1;  // FP16 stages, byte slots, copy lead
constexpr int WS_THREADS = 416, WS_EPI = 256;

__device__ __forceinline__ void mbar_arrive(unsigned bar) {
  asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.shared::cta.b64 st, [%0];\n\t}" ::"r"(bar) : "memory");
}
__device__ __forceinline__ void named_sync(int id, int nthreads) {
  asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(nthreads) : "memory");
}
// Bounded wait that gives up at once after any thread of the CTA recorded a timeout.
__device__ __forceinline__ void mbar_wait_cta(unsigned bar, unsigned parity, volatile int* sabort, int* status) {
  if (*sabort) return;
  if (!mbar_wait(bar, parity)) {
    *sabort = 1;
    if (status) set_err_once(status, GBHE_ETIMEOUT);
  }
}

template <bool CPLX, int BN>
struct WsCfg {
  static constexpr int NC = UCfg<CPLX, BN>::NC;
  static constexpr int STB = UCfg<CPLX, BN>::STB;
  static constexpr int ST8 = UCfg<CPLX, BN>::ST8;
  static constexpr size_t SMEM = (size_t)WS_F * STB + (size_t)WS_S8 * ST8 + 8 * (2 * WS_F + 5) + 16;
};

template <bool CPLX, int BN>
__global__ void __launch_bounds__(WS_THREADS, 1) k_crt_umma_ws(const int8_t* PA, const int8_t* PB, int M, int N,
                                                            int Kp, unsigned char* Out, const CrtDesc* D, int maxM,
                                                            int maxN, int lower, int mpc, int* status) {
  using CF = UCfg<CPLX, BN>;
  constexpr int NC = CF::NC;
  constexpr int STB = CF::STB;
  constexpr int S = WS_F;
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* stage8 = smem_raw + S * STB;
  unsigned long long* bars = reinterpret_cast<unsigned long long*>(stage8 + WS_S8 * CF::ST8);
  // bars: [0, S) FP16 stage empty, S + b accumulator full, S + 2 + b accumulator drained,
  // S + 4 drain of every issued MMA (before TMEM is freed), S + 5 + s FP16 stage ready
  unsigned* tslot = reinterpret_cast<unsigned*>(bars + 2 * S + 5);
  volatile int* sabort = reinterpret_cast<volatile int*>(tslot + 1);

  const int TM = (maxM + UBM - 1) / UBM, TN2 = (maxN + BN - 1) / BN;
  const int TN = (maxN + CBN - 1) / CBN;
  const int ngrp = NMOD / mpc;
  const int entry = blockIdx.z / ngrp, grp = blockIdx.z % ngrp;
  int bx, by;
  {
    const int pid = blockIdx.x, GM = 8;
    const int first = (pid / (GM * TN2)) * GM, gm = min(TM - first, GM);
    bx = first + (pid % (GM * TN2)) % gm;
    by = (pid % (GM * TN2)) / gm;
  }
  if (D) {
    M = D[entry].M;
    N = D[entry].N;
    PA += (size_t)entry * NMOD * NC * maxM * Kp;
    PB += (size_t)entry * NMOD * NC * maxN * Kp;
    Out += (size_t)entry * TM * TN * NMOD * NC * OTILE;
  }
  const int m0 = bx * UBM, n0 = by * BN;
  if (m0 >= M || n0 >= N) return;
  if (lower && m0 + UBM - 1 < n0) return;
  const int t = threadIdx.x, lane = t & 31, w = t >> 5;
  const int l0 = grp * mpc;
  const size_t planeA = (size_t)M * Kp, planeB = (size_t)N * Kp;

  if (t == 0) {
    for (int i = 0; i < S + 2; ++i)
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(bars + i)));
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(bars + S + 4)));
    for (int i = 0; i < 2; ++i)
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bars + S + 2 + i)), "r"(WS_EPI));
    for (int i = 0; i < S; ++i)
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bars + S + 5 + i)), "r"(128));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    *sabort = 0;
  }
  if (w == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(tslot)),
                 "r"(CF::COLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const unsigned tmem = *tslot;
  const int ktiles = Kp / UBK;
  const int iters = mpc * ktiles;

  if (w < 4) {
    // ---------------- producers (128 threads): copy byte tiles, widen them to FP16
    auto issue = [&](int it) {
      stage_issue<CPLX, BN, 128>(stage8 + (it % WS_S8) * CF::ST8, PA, PB, planeA, planeB, l0 + it / ktiles,
                                 (it % ktiles) * UBK, Kp, m0, n0, M, N, t);
    };
    for (int it = 0; it < WS_LAG; ++it) {
      if (it < iters) issue(it);
      cp_commit();
    }
    for (int it = 0; it < iters; ++it) {
      const int s = it % S;
      // the byte slot of K tile it + WS_LAG is the one this thread widened at it - 1
      if (it + WS_LAG < iters) issue(it + WS_LAG);
      cp_commit();
      cp_wait<WS_LAG>();  // this thread's copies of K tile `it` have landed
      if (it >= S)        // the MMAs of K tile it - S have read the FP16 stage
        mbar_wait_cta(smem_addr(bars + s), (unsigned)((it / S) - 1) & 1u, sabort, status);
      stage_widen<CPLX, BN, 128>(stage8 + (it % WS_S8) * CF::ST8, smem_raw + s * STB, t);
      // my part of the stage is written: fence it for the tensor cores and report
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      mbar_arrive(smem_addr(bars + S + 5 + s));
    }
    cp_wait<0>();
  } else if (w == 4) {
    // ---------------- MMA issue (one lane of warp 4)
    const unsigned idesc = (1u << 4) | ((unsigned)(BN >> 3) << 17) | ((unsigned)(UBM >> 4) << 24);
    const unsigned idesc_negA = idesc | (1u << 13);
    for (int it = 0; it < iters; ++it) {
      const int s = it % S;
      const int li = it / ktiles, kt = it % ktiles, b = li & 1;
      // buffer b must have been drained by the epilogue of modulus li - 2
      if (kt == 0 && li >= 2)
        mbar_wait_cta(smem_addr(bars + S + 2 + b), (unsigned)((li - 2) >> 1) & 1u, sabort, status);
      mbar_wait_cta(smem_addr(bars + S + 5 + s), (unsigned)(it / S) & 1u, sabort, status);
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      if (lane == 0) {
        const unsigned dbuf = tmem + (unsigned)b * CF::BUFC;
        const unsigned sA = smem_addr(smem_raw + s * STB), sB = sA + NC * U_APL;
#pragma unroll
        for (int kk = 0; kk < UBK / 16; ++kk) {
          const unsigned first = (kt == 0 && kk == 0) ? 0u : 1u;
          const unsigned long long ar = umma_sdesc(sA + kk * 256, 128, 512);
          const unsigned long long br = umma_sdesc(sB + kk * 256, 128, 512);
          umma_f16(dbuf, ar, br, idesc, first);
          if constexpr (CPLX) {
            const unsigned long long ai = umma_sdesc(sA + U_APL + kk * 256, 128, 512);
            const unsigned long long bi = umma_sdesc(sB + CF::BPL + kk * 256, 128, 512);
            umma_f16(dbuf, ai, bi, idesc_negA, 1u);
            umma_f16(dbuf + BN, ar, bi, idesc, first);
            umma_f16(dbuf + BN, ai, br, idesc, 1u);
          }
        }
        umma_commit(smem_addr(bars + s));
        if (kt == ktiles - 1) umma_commit(smem_addr(bars + S + b));
      }
      __syncwarp();
    }
    // every MMA issued here has completed before TMEM is freed (bounded wait;
    // also when a timeout made the other waits give up)
    if (lane == 0) {
      umma_commit(smem_addr(bars + S + 4));
      if (!mbar_wait(smem_addr(bars + S + 4), 0u) && status) set_err_once(status, GBHE_ETIMEOUT);
    }
    __syncwarp();
  } else {
    // ---------------- epilogue (warps 5-12): row 32 q + lane, columns NRES hh .. NRES hh + NRES - 1
    constexpr int NRES = CF::NRES;
    const int q = w & 3, hh = (w - 5) >> 2, il = 32 * q + lane;
    const bool row_ok = m0 + il < M;
    // this thread's columns lie in one CBN-wide tile of the output layout
    const int tile = ((BN / CBN) * by + (NRES * hh) / CBN) * TM + bx;
    const int ct0 = (NRES * hh) % CBN;      // first column inside that tile
    const int cv = N - n0 - NRES * hh;      // columns of this thread that exist
    for (int li = 0; li < mpc; ++li) {
      const int b = li & 1, l = l0 + li;
      unsigned char* obase = Out + ((size_t)tile * NMOD + l) * NC * OTILE + (size_t)ct0 * CBM + il;
      mbar_wait_cta(smem_addr(bars + S + b), (unsigned)(li >> 1) & 1u, sabort, status);
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const float p = (float)c_p[l], pinv = c_pinv[l];
      const unsigned tb = tmem + ((unsigned)(32 * q) << 16) + (unsigned)b * CF::BUFC + (unsigned)(NRES * hh);
#pragma unroll 1
      for (int sl = 0; sl < NRES / 16; ++sl) {
        float P[NC][16];
#pragma unroll
        for (int c = 0; c < NC; ++c) tmem_ld16(tb + c * BN + sl * 16, P[c]);
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
        for (int c = 0; c < NC; ++c)
#pragma unroll
          for (int x = 0; x < 16; ++x) {
            float v = red_sym(P[c][x], p, pinv);  // |v| <= p/2 + 1
            if (v < 0.f) v += p;                  // [0, p)
            if (row_ok && sl * 16 + x < cv)
              obase[(size_t)c * OTILE + (size_t)(sl * 16 + x) * CBM] = (unsigned char)(int)v;
          }
      }
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      mbar_arrive(smem_addr(bars + S + 2 + b));  // buffer b may be overwritten
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (w == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(CF::COLS));
}

// ------------------------------------------------------------------ reconstruction
// value of the 160-bit two's complement integer D times 2^sc, rounded to double
__device__ __forceinline__ double int160_to_double(unsigned (&D)[5], int sc) {
  const bool negv = (int)D[4] < 0;
  if (negv) {  // D = -D
    unsigned c = 1;
    for (int i = 0; i < 5; ++i) {
      const unsigned x = ~D[i];
      D[i] = x + c;
      c = (c && D[i] == 0) ? 1 : 0;
    }
  }
  // the leading nonzero word (t2), the two below it and a sticky bit for the rest,
  // chosen by comparisons so that D stays in registers
  int top;
  unsigned t2, t1, t0;
  bool sticky;
  if (D[4]) { top = 4; t2 = D[4]; t1 = D[3]; t0 = D[2]; sticky = (D[1] | D[0]) != 0; }
  else if (D[3]) { top = 3; t2 = D[3]; t1 = D[2]; t0 = D[1]; sticky = D[0] != 0; }
  else if (D[2]) { top = 2; t2 = D[2]; t1 = D[1]; t0 = D[0]; sticky = false; }
  else if (D[1]) { top = 1; t2 = D[1]; t1 = D[0]; t0 = 0; sticky = false; }
  else if (D[0]) { top = 0; t2 = D[0]; t1 = 0; t0 = 0; sticky = false; }
  else return 0.0;
  // take 64 bits starting at the top word
  const int lz = __clz(t2);
  unsigned long long hi = ((unsigned long long)t2 << 32) | t1;
  unsigned long long lo = (unsigned long long)t0 << 32;
  // normalise: shift left by lz so bit 63 of hi is set
  if (lz) { hi = (hi << lz) | (lo >> (64 - lz)); lo <<= lz; }
  sticky |= (lo != 0);
  // hi holds the top 64 bits; keep 53, round to nearest even
  unsigned long long mant = hi >> 11;
  const unsigned long long rem = hi & 0x7FFull;
  const bool round_up = (rem > 0x400) || (rem == 0x400 && (sticky || (mant & 1)));
  if (round_up) {
    ++mant;
    if (mant == (1ull << 53)) { mant >>= 1; ++sc; }  // carried into a new bit
  }
  // value = mant * 2^(e2), e2 = (bit index of hi's MSB) - 52 + sc
  const int msb = 32 * top + 31 - lz;  // bit index of the leading one of D
  int e2 = msb - 52 + sc;
  const int expo = e2 + 52 + 1023;  // biased exponent of mant * 2^e2 (mant in [2^52, 2^53))
  if (expo <= 0) return 0.0;       // underflow to zero (results this small are below FP64 noise)
  if (expo >= 2047) return negv ? -INFINITY : INFINITY;
  const unsigned long long bits = ((unsigned long long)expo << 52) | (mant & 0xFFFFFFFFFFFFFull) |
                                  (negv ? 0x8000000000000000ull : 0ull);
  return __longlong_as_double((long long)bits);
}

// 160-bit value of sum_w X_w 2^(32 w) for four 64-bit column sums X_w < 2^63
__device__ __forceinline__ void combine160(unsigned (&D)[5], unsigned long long X0, unsigned long long X1,
                                           unsigned long long X2, unsigned long long X3) {
  D[0] = (unsigned)X0;
  unsigned long long t = (X0 >> 32) + X1;
  D[1] = (unsigned)t;
  t = (t >> 32) + X2;
  D[2] = (unsigned)t;
  t = (t >> 32) + X3;
  D[3] = (unsigned)t;
  D[4] = (unsigned)(t >> 32);
}

// Double value of (S - q M) 2^sc for the CRT sum held as four 64-bit word sums.
__device__ __forceinline__ double crt_finish(const unsigned long long (&X)[4], float F, const unsigned (&Mw)[4], int sc) {
  unsigned S[5], qM[5];
  combine160(S, X[0], X[1], X[2], X[3]);
  const unsigned q = (unsigned)rintf(F);  // < 2^12
  combine160(qM, (unsigned long long)q * Mw[0], (unsigned long long)q * Mw[1], (unsigned long long)q * Mw[2],
             (unsigned long long)q * Mw[3]);
  unsigned D[5];
  unsigned borrow = 0;
#pragma unroll
  for (int i = 0; i < 5; ++i) {
    const unsigned long long d = (unsigned long long)S[i] - qM[i] - borrow;
    D[i] = (unsigned)d;
    borrow = (unsigned)((d >> 63) & 1);
  }
  return int160_to_double(D, sc);
}

// Reconstruct four consecutive rows i0..i0+3 of column j of one output tile
// (tile base `T` in the tile-major residue layout, offset `loc` inside it)
// and update C.  One component (Re, then Im) at a time: its CRT sums are
// kept as four independent 64-bit word sums per value (each term < 2^40,
// sixteen terms < 2^44), carries propagated once at the end.  The loops over
// the moduli and the words are unrolled, so the table words W_l and y_l / p_l
// are constant-bank operands of the multiply-adds (no registers, no shared
// memory), and only one component's sums are live at a time.
// CRT values of one component (c) of four consecutive rows.
template <int NCOUT>
__device__ __noinline__ void crt_component4(const unsigned char* T, int loc, int c, const int (&sc)[4],
                                            double (&v)[4]) {
  const unsigned Mw[4] = {c_M[0], c_M[1], c_M[2], c_M[3]};
  unsigned w[NMOD];
#pragma unroll
  for (int l = 0; l < NMOD; ++l) w[l] = __ldcs(reinterpret_cast<const unsigned*>(T + (size_t)(l * NCOUT + c) * OTILE + loc));
  unsigned long long X[4][4];
  float F[4];
#pragma unroll
  for (int r = 0; r < 4; ++r) {
    F[r] = 0.f;
#pragma unroll
    for (int k = 0; k < 4; ++k) X[r][k] = 0ull;
  }
#pragma unroll
  for (int l = 0; l < NMOD; ++l) {
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      const unsigned cv = (w[l] >> (8 * r)) & 0xFFu;
#pragma unroll
      for (int k = 0; k < 4; ++k) X[r][k] += (unsigned long long)cv * c_W[l][k];
      F[r] = fmaf((float)cv, c_frac[l], F[r]);
    }
  }
#pragma unroll
  for (int r = 0; r < 4; ++r) v[r] = crt_finish(X[r], F[r], Mw, sc[r]);
}

template <bool CPLX>
__device__ __forceinline__ void crt_store4(const unsigned char* T, int loc, int i0, int j, int M, int lower,
                                           const int* ea, int ebj, double2 alpha, double2 beta, void* Cv, int ldc) {
  constexpr int NCOUT = CPLX ? 2 : 1;
  const bool beta0 = (beta.x == 0.0 && beta.y == 0.0);
  const bool beta1 = (beta.x == 1.0 && beta.y == 0.0);
  const bool alpha1 = (alpha.x == 1.0 && alpha.y == 0.0);
  const bool alpham1 = (alpha.x == -1.0 && alpha.y == 0.0);
  int sc[4];
#pragma unroll
  for (int r = 0; r < 4; ++r) sc[r] = (i0 + r < M) ? ea[i0 + r] + ebj - 104 : 0;
  double v[NCOUT][4];
  crt_component4<NCOUT>(T, loc, 0, sc, v[0]);
  if (CPLX) crt_component4<NCOUT>(T, loc, 1, sc, v[NCOUT - 1]);
#pragma unroll
  for (int r = 0; r < 4; ++r) {
    const int i = i0 + r;
    if (i >= M || (lower && i < j)) continue;
    const double vr = v[0][r];
    const double vi = CPLX ? v[NCOUT - 1][r] : 0.0;
    double2 out;
    if (alpha1) out = make_double2(vr, vi);
    else if (alpham1) out = make_double2(-vr, -vi);
    else out = cmul(alpha, make_double2(vr, vi));
    const size_t ci = (size_t)i + (size_t)j * ldc;
    if (CPLX) {
      double2* C = reinterpret_cast<double2*>(Cv);
      if (beta1) out = cadd(out, C[ci]);
      else if (!beta0) out = cadd(out, cmul(beta, C[ci]));
      C[ci] = out;
    } else {
      double* C = reinterpret_cast<double*>(Cv);
      double o = out.x;
      if (beta1) o += C[ci];
      else if (!beta0) o += beta.x * C[ci];
      C[ci] = o;
    }
  }
}

// C = alpha * (A B) + beta * C from the residues; one thread per four
// consecutive rows of a tile column (4-byte loads of every residue block).
// Both reconstruction kernels are held to 64 registers (four 256-thread CTAs
// per SM): the integer multiply-add chains are latency-bound, and the extra
// resident warps hide more of it than the 80-register form does, a few
// spilled words included (about 5 % less reconstruction time in the
// n = 10000 solve).
__global__ void __launch_bounds__(256, 4) k_crt_reconstruct(const unsigned char* Out, int M, int N, const int* ea, const int* eb, GemmArgs g,
                                  int cplx) {
  const int TM = (M + CBM - 1) / CBM, TN = (N + CBN - 1) / CBN;
  const int ncout = cplx ? 2 : 1;
  const size_t per_tile = OTILE / 4;
  const size_t groups = (size_t)TM * TN * per_tile;
  for (size_t gi = blockIdx.x * (size_t)blockDim.x + threadIdx.x; gi < groups;
       gi += (size_t)gridDim.x * blockDim.x) {
    const size_t tile = gi / per_tile;
    const int loc = (int)(gi % per_tile) * 4;
    const int bx = (int)(tile % TM), by = (int)(tile / TM);
    const int i0 = bx * CBM + loc % CBM, j = by * CBN + loc / CBM;
    if (i0 >= M || j >= N) continue;
    if (g.lower_only && i0 + 3 < j) continue;
    const unsigned char* T = Out + tile * NMOD * ncout * OTILE;
    if (cplx) crt_store4<true>(T, loc, i0, j, M, g.lower_only, ea, eb[j], g.alpha, g.beta, g.C, g.ldc);
    else crt_store4<false>(T, loc, i0, j, M, g.lower_only, ea, eb[j], g.alpha, g.beta, g.C, g.ldc);
  }
}

// Batched reconstruction: C_z = alpha (A_z B_z) + beta C_z for every entry z
// (tiles laid out for maxM x maxN per entry).
__global__ void __launch_bounds__(256, 4) k_bcrt_reconstruct(const unsigned char* Out, const CrtDesc* D, int nbatch, int maxM, int maxN,
                                   const int* ea, const int* eb, double2 alpha, double2 beta, int cplx) {
  const int TM = (maxM + CBM - 1) / CBM, TN = (maxN + CBN - 1) / CBN;
  const int ncout = cplx ? 2 : 1;
  const size_t per_tile = OTILE / 4;
  const size_t tiles = (size_t)TM * TN;
  const size_t groups = (size_t)nbatch * tiles * per_tile;
  for (size_t gi = blockIdx.x * (size_t)blockDim.x + threadIdx.x; gi < groups;
       gi += (size_t)gridDim.x * blockDim.x) {
    const size_t tile = gi / per_tile;  // global tile index over entries
    const int z = (int)(tile / tiles);
    const size_t tz = tile % tiles;
    const int loc = (int)(gi % per_tile) * 4;
    const int bx = (int)(tz % TM), by = (int)(tz / TM);
    const int i0 = bx * CBM + loc % CBM, j = by * CBN + loc / CBM;
    const CrtDesc d = D[z];
    if (i0 >= d.M || j >= d.N) continue;
    // a column map sends product column j to column cmap[j] of C
    char* Cj = reinterpret_cast<char*>(d.C) +
               (d.cmap ? (ptrdiff_t)(d.cmap[j] - j) * d.ldc * (ptrdiff_t)(cplx ? sizeof(double2) : sizeof(double)) : 0);
    const unsigned char* T = Out + tile * NMOD * ncout * OTILE;
    if (cplx)
      crt_store4<true>(T, loc, i0, j, d.M, 0, ea + (size_t)z * maxM, eb[(size_t)z * maxN + j], alpha, beta, Cj,
                       d.ldc);
    else
      crt_store4<false>(T, loc, i0, j, d.M, 0, ea + (size_t)z * maxM, eb[(size_t)z * maxN + j], alpha, beta, Cj,
                        d.ldc);
  }
}

inline size_t out_bytes(int M, int N, int cplx) {
  return (size_t)((M + CBM - 1) / CBM) * ((N + CBN - 1) / CBN) * NMOD * (cplx ? 2 : 1) * OTILE;
}

// Launch of the tcgen05 residue products: 64-column tiles when every product
// has at most 64 columns, else 128; moduli per CTA chosen so that the grid
// covers the GPU at least twice.
template <bool CPLX, bool ONE, int BN>
int umma_prepare(int* nsm_out) {
  static bool ready[MAX_DEVICES] = {};
  static int nsm[MAX_DEVICES] = {};
  const int dev = device_slot();
  if (dev < 0) return GBHE_ECUDA;
  if (!ready[dev]) {
    if (ONE)
      GBHE_CUDA(cudaFuncSetAttribute(k_crt_umma_ws<CPLX, BN>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)WsCfg<CPLX, BN>::SMEM));
    else
      GBHE_CUDA(cudaFuncSetAttribute(k_crt_umma<CPLX, BN>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)UCfg<CPLX, BN>::SMEM));
    GBHE_CUDA(cudaDeviceGetAttribute(&nsm[dev], cudaDevAttrMultiProcessorCount, dev));
    ready[dev] = true;
  }
  *nsm_out = nsm[dev];
  return 0;
}

template <bool CPLX, int BN>
int launch_umma_bn(cudaStream_t st, const int8_t* PA, const int8_t* PB, int M, int N, int Kp, unsigned char* Out,
                   const CrtDesc* D, int maxM, int maxN, int lower, int nbatch, int* status) {
  const bool one = Kp <= UCfg<CPLX, BN>::KC_TERMS;
  int nsm = 0;
  int rc = one ? umma_prepare<CPLX, true, BN>(&nsm) : umma_prepare<CPLX, false, BN>(&nsm);
  if (rc) return rc;
  const int TM = (maxM + UBM - 1) / UBM, TN2 = (maxN + BN - 1) / BN;
  const long tiles = (long)TM * TN2 * nbatch;
  // moduli per CTA: as many as keep at least two CTAs per SM
  int mpc = NMOD;
  while (mpc > 1 && tiles * (NMOD / mpc) < 2L * nsm) mpc /= 2;
  dim3 grid(TM * TN2, 1, (NMOD / mpc) * nbatch);
  if (one)
    k_crt_umma_ws<CPLX, BN><<<grid, WS_THREADS, WsCfg<CPLX, BN>::SMEM, st>>>(PA, PB, M, N, Kp, Out, D, maxM, maxN,
                                                                             lower, mpc, status);
  else
    k_crt_umma<CPLX, BN><<<grid, UTHREADS, UCfg<CPLX, BN>::SMEM, st>>>(PA, PB, M, N, Kp, Out, D, maxM, maxN, lower,
                                                                       mpc, status);
  count_launch();
  return 0;
}

template <bool CPLX>
int launch_umma(cudaStream_t st, const int8_t* PA, const int8_t* PB, int M, int N, int Kp, unsigned char* Out,
                const CrtDesc* D, int maxM, int maxN, int lower, int nbatch, int* status) {
  if (maxN <= CBN)
    return launch_umma_bn<CPLX, CBN>(st, PA, PB, M, N, Kp, Out, D, maxM, maxN, lower, nbatch, status);
  return launch_umma_bn<CPLX, UBN>(st, PA, PB, M, N, Kp, Out, D, maxM, maxN, lower, nbatch, status);
}

size_t crt_bytes(int M, int N, int K, int cplx) {
  const size_t Kp = (size_t)(K + CBK - 1) / CBK * CBK;
  const int nc = cplx ? 2 : 1;
  size_t b = 0;
  b += (size_t)NMOD * nc * (size_t)M * Kp + 256;
  b += (size_t)NMOD * nc * (size_t)N * Kp + 256;
  b += out_bytes(M, N, cplx) + 256;
  b += ((size_t)M + N) * sizeof(int) + 256;
  return b;
}

Operand make_operand(const void* X, int ld, int R, int K, int op, bool isA, int cplx) {
  Operand o;
  o.X = X; o.ld = ld; o.R = R; o.K = K; o.cplx = cplx; o.cj = (op == OP_C) ? 1 : 0;
  if (isA) o.mode = (op == OP_N) ? 0 : (op == OP_H ? 2 : 1);
  else o.mode = (op == OP_N) ? 1 : 0;
  return o;
}

}  // namespace

size_t crt_gemm_ws_bytes(int M, int N, int K, int cplx) { return crt_bytes(M, N, K, cplx); }

size_t crt_batched_ws_bytes(int nbatch, int maxM, int maxN, int maxK, int cplx) {
  const size_t Kp = (size_t)(maxK + CBK - 1) / CBK * CBK;
  const int nc = cplx ? 2 : 1;
  const size_t nbt = (size_t)std::max(nbatch, 1);
  size_t b = 0;
  b += nbt * NMOD * nc * (size_t)maxM * Kp + 256;
  b += nbt * NMOD * nc * (size_t)maxN * Kp + 256;
  b += nbt * out_bytes(maxM, maxN, cplx) + 256;
  b += nbt * ((size_t)maxM + maxN) * sizeof(int) + 256;
  return b;
}

int crt_gemm_batched(cudaStream_t st, int opA, int opB, cplx alpha, cplx beta, int cplx_flag, const CrtDesc* D,
                     int nbatch, int maxM, int maxN, int maxK, void* ws, size_t ws_bytes, int* status, double flops) {
  if (nbatch <= 0 || maxM <= 0 || maxN <= 0 || maxK <= 0) return 0;
  if (maxK > KMAX || nbatch > 65535 / NMOD) return GBHE_EWORKSPACE;
  if (crt_batched_ws_bytes(nbatch, maxM, maxN, maxK, cplx_flag) > ws_bytes) return GBHE_EWORKSPACE;
  int rc = init_constants();
  if (rc) return rc;
  const int Kp = (maxK + CBK - 1) / CBK * CBK;
  const int nc = cplx_flag ? 2 : 1;
  char* p = reinterpret_cast<char*>(ws);
  auto take = [&](size_t bytes) { char* q = p; p += (bytes + 255) & ~size_t(255); return q; };
  int8_t* PA = reinterpret_cast<int8_t*>(take((size_t)nbatch * NMOD * nc * maxM * Kp));
  int8_t* PB = reinterpret_cast<int8_t*>(take((size_t)nbatch * NMOD * nc * maxN * Kp));
  unsigned char* Out = reinterpret_cast<unsigned char*>(take((size_t)nbatch * out_bytes(maxM, maxN, cplx_flag)));
  int* ea = reinterpret_cast<int*>(take((size_t)nbatch * (maxM + maxN) * sizeof(int)));
  int* eb = ea + (size_t)nbatch * maxM;
  ProfScope prof(st, GBHE_PROF_CRT, flops, 0.0);
  {
    ProfScope pp(st, GBHE_PROF_CRT_PREP, 0.0, 0.0);
    k_fill_int_batched<<<256, 256, 0, st>>>(ea, (size_t)nbatch * (maxM + maxN), -1100);
    count_launch();
    const int gA = (maxM + 31) / 32, gB = (maxN + 31) / 32;
    k_bop_exponents<<<dim3(gA + gB, (maxK + 31) / 32, nbatch), dim3(32, 8), 0, st>>>(D, opA, opB, cplx_flag, maxM, maxN,
                                                                                     ea, eb, gA);
    count_launch();
    k_bop_residues<<<dim3(gA + gB, Kp / 32, nbatch), dim3(32, 8), 0, st>>>(D, opA, opB, cplx_flag, maxM, maxN, ea, eb,
                                                                           Kp, PA, PB, gA);
    count_launch();
  }
  {
    ProfScope pm(st, GBHE_PROF_CRT_MMA, flops, 0.0);
    rc = cplx_flag ? launch_umma<true>(st, PA, PB, maxM, maxN, Kp, Out, D, maxM, maxN, 0, nbatch, status)
                   : launch_umma<false>(st, PA, PB, maxM, maxN, Kp, Out, D, maxM, maxN, 0, nbatch, status);
    if (rc) return rc;
  }
  ProfScope pr(st, GBHE_PROF_CRT_REC, 0.0, 0.0);
  const size_t total = (size_t)nbatch * out_bytes(maxM, maxN, 0) / NMOD / 4;  // four outputs per thread
  k_bcrt_reconstruct<<<(int)std::min<size_t>((total + 255) / 256, 152 * 64), 256, 0, st>>>(Out, D, nbatch, maxM, maxN,
                                                                                           ea, eb, alpha, beta,
                                                                                           cplx_flag);
  count_launch();
  return cudaGetLastError() == cudaSuccess ? 0 : GBHE_ECUDA;
}

size_t crt_budget_bytes(int n, int block) {
  const int b = std::max(1, std::min(n, block));
  // at least 64 MiB: the batched products of small problems (one padded
  // 128 x 64 output tile per entry) need more than an n x n x n product
  return std::max(crt_bytes(b, b, b, 1), size_t(64) << 20);
}

int gemm(Ctx& c, const GemmArgs& g, int cplx) {
  if (g.m <= 0 || g.n <= 0) return 0;
  // The FP64 tensor pipe delivers about 7 GFLOP/s per SM, so a DMMA product
  // that covers only a few 64 x 64 output tiles runs for hundreds of
  // microseconds; the tensor-core engine costs a few short launches instead.
  // Engine products for everything with k >= 16 except products so small
  // that each DMMA tile holds less than ~5e4 multiply-adds.
  const double work = (double)g.m * g.n * std::max(g.k, 0);
  const double tiles = std::ceil(g.m / 64.0) * std::ceil(g.n / 64.0);
  const bool use_crt = c.engine == GBHE_ENGINE_CRT && c.crt_ws != nullptr && g.k >= 16 &&
                       (work >= 2.0e6 || work > 5.0e4 * std::min(tiles, 152.0));
  if (!use_crt) return cplx ? zgemm(c.st, g, c.gemm_scratch, c.gemm_scratch_bytes)
                            : dgemm(c.st, g, c.gemm_scratch, c.gemm_scratch_bytes);
  // blocks of at most CRT_BLOCK in every dimension; K blocks accumulate in C
  const int bm = std::min(g.m, c.crt_block), bn = std::min(g.n, c.crt_block), bk = std::min(g.k, c.crt_block);
  // element size in bytes (the int parameter `cplx` shadows the type name here)
  const size_t es = cplx ? sizeof(double2) : sizeof(double);
  const bool herm = (g.opA == OP_H);
  for (int k0 = 0; k0 < g.k; k0 += bk) {
    const int kk = std::min(bk, g.k - k0);
    for (int j0 = 0; j0 < g.n; j0 += bn) {
      const int nn = std::min(bn, g.n - j0);
      for (int i0 = 0; i0 < g.m; i0 += bm) {
        const int mm = std::min(bm, g.m - i0);
        if (g.lower_only && i0 + mm <= j0) continue;  // block strictly above the diagonal
        GemmArgs s = g;
        s.m = mm; s.n = nn; s.k = kk;
        s.lower_only = (g.lower_only && i0 < j0 + nn) ? 1 : 0;
        if (s.lower_only && i0 != j0) return GBHE_EWORKSPACE;  // the block's corner lies on the diagonal
        if (k0 > 0) s.beta = mk(1.0, 0.0);
        // operand sub-blocks
        const char* A = reinterpret_cast<const char*>(g.A);
        const char* B = reinterpret_cast<const char*>(g.B);
        if (herm) {
          if (g.k != g.m) return GBHE_EWORKSPACE;
          // op(A)(i0:i0+mm, k0:k0+kk) of a Hermitian matrix: Hermitian only on diagonal blocks
          if (i0 == k0 && mm == kk) {
            s.opA = OP_H;
            s.A = A + ((size_t)i0 + (size_t)k0 * g.lda) * es;
          } else if (i0 > k0) {
            s.opA = OP_N;
            s.A = A + ((size_t)i0 + (size_t)k0 * g.lda) * es;
          } else {
            s.opA = OP_C;  // stored lower block (k0.., i0..), conjugate-transposed
            s.A = A + ((size_t)k0 + (size_t)i0 * g.lda) * es;
          }
        } else if (g.opA == OP_N) {
          s.A = A + ((size_t)i0 + (size_t)k0 * g.lda) * es;
        } else {
          s.A = A + ((size_t)k0 + (size_t)i0 * g.lda) * es;
        }
        if (g.opB == OP_N) s.B = B + ((size_t)k0 + (size_t)j0 * g.ldb) * es;
        else s.B = B + ((size_t)j0 + (size_t)k0 * g.ldb) * es;
        s.C = reinterpret_cast<char*>(g.C) + ((size_t)i0 + (size_t)j0 * g.ldc) * es;
        int rc = crt_gemm(c.st, s, cplx, c.crt_ws, c.crt_ws_bytes, c.status);
        if (rc) return rc;
      }
    }
  }
  return 0;
}

int crt_gemm(cudaStream_t st, const GemmArgs& g, int cplx, void* ws, size_t ws_bytes, int* status) {
  if (g.m <= 0 || g.n <= 0) return 0;
  if (g.k <= 0 || g.k > KMAX) return GBHE_EWORKSPACE;
  int rc = init_constants();
  if (rc) return rc;
  const int M = g.m, N = g.n, K = g.k;
  const int Kp = (K + CBK - 1) / CBK * CBK;
  const int nc = cplx ? 2 : 1;
  if (crt_bytes(M, N, K, cplx) > ws_bytes) return GBHE_EWORKSPACE;
  char* p = reinterpret_cast<char*>(ws);
  auto take = [&](size_t bytes) { char* q = p; p += (bytes + 255) & ~size_t(255); return q; };
  int8_t* PA = reinterpret_cast<int8_t*>(take((size_t)NMOD * nc * M * Kp));
  int8_t* PB = reinterpret_cast<int8_t*>(take((size_t)NMOD * nc * N * Kp));
  unsigned char* Out = reinterpret_cast<unsigned char*>(take(out_bytes(M, N, cplx)));
  int* ea = reinterpret_cast<int*>(take((size_t)(M + N) * sizeof(int)));
  int* eb = ea + M;
  const Operand oa = make_operand(g.A, g.lda, M, K, g.opA, true, cplx);
  const Operand ob = make_operand(g.B, g.ldb, N, K, g.opB, false, cplx);
  // executed FP64-equivalent flops of this call: lower-only products count the
  // outputs on and below the diagonal only (the tiles above it are skipped)
  const double mn = std::min(M, N);
  const double outs = g.lower_only ? mn * M - mn * (mn - 1.0) / 2.0 : (double)M * N;
  const double flops = (cplx ? 8.0 : 2.0) * outs * K;
  ProfScope prof(st, GBHE_PROF_CRT, flops, 0.0);
  {
    ProfScope pp(st, GBHE_PROF_CRT_PREP, 0.0, 0.0);
    k_fill_int<<<64, 256, 0, st>>>(ea, M + N, -1100);
    count_launch();
    const int gA = (M + 31) / 32, gB = (N + 31) / 32;
    k_op_exponents<<<dim3(gA + gB, (K + 31) / 32), dim3(32, 8), 0, st>>>(oa, ea, ob, eb, gA);
    count_launch();
    k_op_residues<<<dim3(gA + gB, Kp / 32), dim3(32, 8), 0, st>>>(oa, ea, PA, ob, eb, PB, gA, Kp);
    count_launch();
  }
  {
    ProfScope pm(st, GBHE_PROF_CRT_MMA, flops, 0.0);
    rc = cplx ? launch_umma<true>(st, PA, PB, M, N, Kp, Out, nullptr, M, N, g.lower_only, 1, status)
              : launch_umma<false>(st, PA, PB, M, N, Kp, Out, nullptr, M, N, g.lower_only, 1, status);
    if (rc) return rc;
  }
  ProfScope pr(st, GBHE_PROF_CRT_REC, 0.0, 0.0);
  const size_t total = out_bytes(M, N, 0) / NMOD / 4;  // four outputs per thread
  k_crt_reconstruct<<<(int)std::min<size_t>((total + 255) / 256, 152 * 64), 256, 0, st>>>(Out, M, N, ea, eb, g, cplx);
  count_launch();
  return cudaGetLastError() == cudaSuccess ? 0 : GBHE_ECUDA;
}

}  // namespace gbhe

extern "C" int gbhe_crt_tables(int* p, unsigned* W, unsigned* M, int* k13, int* k26, int* k39, float* frac) {
  gbhe::HostTables t;
  gbhe::crt_tables(t);
  for (int l = 0; l < gbhe::NMOD; ++l) {
    if (p) p[l] = t.p[l];
    if (frac) frac[l] = t.frac[l];
    if (k13) k13[l] = t.kw[l][0];
    if (k26) k26[l] = t.kw[l][1];
    if (k39) k39[l] = t.kw[l][2];
    for (int w = 0; w < 4; ++w)
      if (W) W[4 * l + w] = t.W[l][w];
  }
  for (int w = 0; w < 4; ++w)
    if (M) M[w] = t.M[w];
  return gbhe::NMOD;
}
