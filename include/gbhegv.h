/*
 * gbhegv.h -- C-ABI of libgbhegv: a GB300 (sm_103a) solver for the
 * Hermitian-definite generalized eigenproblem  A x = lambda B x  in complex128,
 * following the paper's Algorithm 1 (Cholesky B = L L^H, reduction
 * A' = L^{-1} A L^{-H}, standard eigensolver, x = L^{-H} y) with Algorithm 2 in
 * its two-stage form (Section 4.2: dense -> band -> tridiagonal, tridiagonal
 * divide and conquer of Section 4.3, back-transformation y = Q1 Q2 y').
 *
 * Common conventions
 *   - complex numbers are gbhe_cplx {re, im} (layout of double2,
 *     cuDoubleComplex, C99 double complex, torch.complex128);
 *   - matrices are column-major with a leading dimension (ld >= max(1, rows));
 *     Hermitian inputs are read from their LOWER triangle only;
 *   - every matrix/vector pointer is DEVICE memory owned by the caller; the
 *     library never allocates inside a stream-ordered call: temporaries come
 *     from the workspace the caller attaches with gbhe_set_workspace;
 *   - `stream` is a cudaStream_t passed as void*; calls are asynchronous on it;
 *   - return value: 0 = enqueued (or done), -i = argument i is invalid
 *     (LAPACK convention, 1-based over the C argument list), GBHE_E* for
 *     library errors detected on the host.  Numerical failures found on the
 *     device (B not positive definite, non-convergence, a bounded device wait
 *     that expired) are recorded in the handle's status word and returned by
 *     gbhe_get_status, which synchronises the stream.
 */
#ifndef GBHEGV_H_
#define GBHEGV_H_

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
  double re, im;
} gbhe_cplx;

typedef struct gbhe_ctx* gbhe_handle;

/* Library error codes (negative values below -100 so they never collide with
 * the -i argument codes). */
#define GBHE_EWORKSPACE (-101) /* workspace missing or smaller than gbhe_workspace_size */
#define GBHE_ECUDA (-102)      /* a CUDA runtime call failed */
#define GBHE_ETIMEOUT (-103)   /* a bounded device-side wait expired (status word) */
#define GBHE_ENONFINITE (-104) /* NaN/Inf met where a finite value is required */
#define GBHE_ENOTCONV (-105)   /* an iteration did not converge (status word) */

/* Create a handle on CUDA device `device` (made current).  Allocates only the
 * handle's small status buffer.  Returns 0 or GBHE_ECUDA. */
int gbhe_create(gbhe_handle* handle, int device);

/* Release the handle (does not touch the caller's workspace). */
int gbhe_destroy(gbhe_handle handle);

/* Bytes of device workspace that every entry point below needs for a
 * problem of order n, band width nb and m = iu-il+1 wanted eigenvectors
 * (an upper bound over all stages).  nb = 0 means the band width the
 * handle's rule gives for (n, m) (gbhe_resolve_nb). */
int gbhe_workspace_size(gbhe_handle handle, int n, int nb, int m, size_t* bytes);

/* Attach caller-owned device workspace (256-byte aligned). */
int gbhe_set_workspace(gbhe_handle handle, void* dwork, size_t bytes);

/* Synchronise `stream` and return the device status: 0 = success,
 * k > 0 = the leading minor of order k of B is not positive definite
 * (potrf), or GBHE_ETIMEOUT / GBHE_ENOTCONV.  Clears the status. */
int gbhe_get_status(gbhe_handle handle, void* stream);
/* The same call under the name of the boundary's status query. */
int gbhe_sync_status(gbhe_handle handle, void* stream);

/* Default band width used when nb = 0 is passed and the handle has no
 * band-width rule (16 up to n = 128, 32 up to n = 1024, 64 beyond). */
int gbhe_default_nb(int n);

/* Band-width rule: the handle's tuning cache, filled by an autotuner that
 * times the solve for several nb (the paper leaves nb open; it trades the
 * stage-1 panel width against the stage-2 chase and the Q2 back-transform,
 * both O(n^2 nb) work, Section 4.2).  `count` entries
 * (n_max[i], frac_max[i], nb[i]); for a problem of order n with m selected
 * pairs the rule picks the entries with the smallest n_max[i] >= n (the
 * largest n_max when none is >= n), among those the entry with the smallest
 * frac_max[i] >= m/n (the largest frac_max when none is; the first of equal
 * entries), and gives its nb -- unless that nb is >= n, when the default
 * (gbhe_default_nb) is given.  count = 0 is the default everywhere.
 * Requirements: 0 <= count <= GBHE_NB_RULE_MAX, n_max[i] >= 1,
 * 0 < frac_max[i] <= 1, 1 <= nb[i] <= 64; the arrays are host memory, read
 * only during the call.  gbhe_nb_rule_pick evaluates a rule without a handle
 * (no CUDA call) and writes the band width to *nb_out: 0, or -1 count, -2
 * n_max, -3 frac_max, -4 nb, -5 n < 0 or m outside [0, n], -6 nb_out NULL. */
#define GBHE_NB_RULE_MAX 64
int gbhe_nb_rule_pick(int count, const int* n_max, const double* frac_max, const int* nb, int n, int m,
                      int* nb_out);
/* Install a rule on the handle (copied; replaces the previous one).  Returns
 * 0, -1 (handle NULL) or the codes of gbhe_nb_rule_pick shifted by one
 * (-2 count, -3 n_max, -4 frac_max, -5 nb). */
int gbhe_set_nb_rule(gbhe_handle h, int count, const int* n_max, const double* frac_max, const int* nb);
/* The band width that nb = 0 selects on this handle for order n and m
 * selected pairs: 0, -1 handle NULL, -2 n < 0 or m outside [0, n], -3 nb NULL. */
int gbhe_resolve_nb(gbhe_handle h, int n, int m, int* nb);

/* Engine of the FP64 level-3 products of every stage:
 *   GBHE_ENGINE_CRT  (default) exact modular products on the FP16 tensor
 *                    cores for large products (see gbhe_gemm_crt), the FP64
 *                    tensor pipe (DMMA) for small ones;
 *   GBHE_ENGINE_DMMA FP64 tensor pipe only.
 * The paper's level-3 BLAS on the GPU (Section 3) has one engine; the choice
 * exists because this GPU's FP64 pipes are about 1 TFLOP/s. */
#define GBHE_ENGINE_DMMA 0
#define GBHE_ENGINE_CRT 1
int gbhe_set_gemm_engine(gbhe_handle h, int engine);

/* Largest block (in every dimension) of one tensor-core GEMM call, 128 ..
 * 16384 (the default).  Larger products are cut into blocks of this size.
 * The workspace reported by gbhe_workspace_size grows with the square of
 * min(n, block) (about 16 GB at n = 10000 with the default); a smaller block
 * trades speed for memory.  Set it before gbhe_workspace_size.  No
 * counterpart in the paper.  Returns 0, -1 (no handle) or -2 (out of range). */
int gbhe_set_crt_block(gbhe_handle h, int block);

/* Algorithm 1, step 1 (paper Section 3): Cholesky factorisation B = L L^H.
 * B (n x n, ldb) lower triangle read; L overwrites it (upper untouched).
 * A non-positive pivot at order k sets status k (first failure wins). */
int gbhe_potrf(gbhe_handle h, int n, gbhe_cplx* B, int ldb, void* stream);

/* Algorithm 1, step 2: A' = L^{-1} A L^{-H}.  A (n x n, lda) lower triangle
 * read; on return A holds the full Hermitian A' (both triangles).  L is the
 * lower factor from gbhe_potrf (n x n, ldl, lower read). */
int gbhe_hegst(gbhe_handle h, int n, gbhe_cplx* A, int lda, const gbhe_cplx* L, int ldl,
               void* stream);

/* Algorithm 2, step 1, first stage (Section 4.2, Figure 1): reduction of the
 * Hermitian A (lower read) to Hermitian band form of half-bandwidth nb,
 * A = Q1 Band Q1^H.  Block reflectors: panel p (columns p*nb .. p*nb+nb-1)
 * contributes Q1_p = I - V_p T_p V_p^H acting on rows p*nb+nb .. n-1.
 * On return the lower band (rows i..i+nb of column i) of A holds the band;
 * V_p is stored below the band (unit diagonal implicit); T1 receives the
 * nb x nb upper-triangular T_p of each panel (T1 + p*nb*nb, ld nb; size
 * ceil(n/nb)*nb*nb); tau1 (n) the reflector scalars.  1 <= nb <= 128. */
int gbhe_he2hb(gbhe_handle h, int n, int nb, gbhe_cplx* A, int lda, gbhe_cplx* T1,
               gbhe_cplx* tau1, void* stream);

/* Size (elements) of the V2 and tau2 arrays of gbhe_hb2st:
 * V2: n * ceil((n-1)/nb) * nb complex,  tau2: n * ceil((n-1)/nb) complex. */
int gbhe_hb2st_sizes(int n, int nb, size_t* v2_elems, size_t* tau2_elems);

/* Algorithm 2, step 1, second stage (Section 4.2): bulge chasing with
 * column-wise elimination from band (lower band of A, half-bandwidth nb) to
 * real symmetric tridiagonal T = Q2^H Band Q2.  d (n) and e (n-1) receive
 * the diagonal and sub-diagonal.  Reflector (s, j) -- sweep s = 0..n-2, step
 * j -- is H = I - tau v v^H acting on rows s+1+j*nb .. s+nb+j*nb (clipped to
 * n); v (v[0] = 1) is stored at V2 + (s*J + j)*nb and tau at tau2[s*J + j],
 * J = ceil((n-1)/nb).  Q2 is the product of all H in generation order
 * (s major, j minor).  A is not modified.  1 <= nb <= 64 (one step's blocks
 * are held in shared memory). */
int gbhe_hb2st(gbhe_handle h, int n, int nb, const gbhe_cplx* A, int lda, double* d, double* e,
               gbhe_cplx* V2, gbhe_cplx* tau2, void* stream);

/* Algorithm 2, step 2 (Section 4.3): divide and conquer eigensolver of the
 * real symmetric tridiagonal (d, e).  w receives the eigenvalues il..iu
 * (1-based, inclusive, ascending; m = iu-il+1 values) and Z (n x m, ldz) the
 * orthonormal eigenvectors; in the last merge only these m vectors are
 * formed (Section 4.3, last paragraph).  d and e are not modified. */
int gbhe_stedc(gbhe_handle h, int n, const double* d, const double* e, int il, int iu,
               double* w, double* Z, int ldz, void* stream);

/* Algorithm 2, step 3 for two stages (Section 4.2): X = Q1 Q2 Z for the m
 * real columns of Z (n x m, ldz); X (n x m, ldx) complex output.  A, T1
 * from gbhe_he2hb; V2, tau2 from gbhe_hb2st. */
int gbhe_unmtr_2stage(gbhe_handle h, int n, int nb, int m, const gbhe_cplx* A, int lda,
                      const gbhe_cplx* T1, const gbhe_cplx* V2, const gbhe_cplx* tau2,
                      const double* Z, int ldz, gbhe_cplx* X, int ldx, void* stream);

/* Algorithm 1, step 4: X := L^{-H} X for the m columns of X (n x m, ldx);
 * L lower (n x n, ldl) from gbhe_potrf. */
int gbhe_trsm_lh(gbhe_handle h, int n, int m, const gbhe_cplx* L, int ldl, gbhe_cplx* X,
                 int ldx, void* stream);

/* Full two-stage driver (Algorithm 1 around two-stage Algorithm 2):
 * eigenpairs il..iu (1-based, inclusive) of A x = lambda B x.  A (lower
 * read) and B (lower read) are overwritten (A by band/V1 data, B by L);
 * w (m) ascending eigenvalues, X (n x m, ldx) B-orthonormal eigenvectors.
 * nb = 0 selects the handle's band width for (n, m = iu-il+1)
 * (gbhe_resolve_nb); 1 <= nb <= 64. */
int gbhe_hegv(gbhe_handle h, int n, int nb, gbhe_cplx* A, int lda, gbhe_cplx* B, int ldb, int il,
              int iu, double* w, gbhe_cplx* X, int ldx, void* stream);

/* One-stage comparator (Section 4.1): same contract as gbhe_hegv with the
 * reduction done by one-stage Householder tridiagonalisation (half of its
 * flops in Hermitian matrix-vector products) and a single back-transform. */
int gbhe_hegv_onestage(gbhe_handle h, int n, gbhe_cplx* A, int lda, gbhe_cplx* B, int ldb, int il,
                       int iu, double* w, gbhe_cplx* X, int ldx, void* stream);

/* Many independent problems of uneven sizes (the repeated solves that
 * motivate the paper, Section 1): problem i is gbhe_hegv(n[i], nb[i], A[i],
 * lda[i], B[i], ldb[i], il[i], iu[i], w[i], X[i], ldx[i]) on worker stream
 * workers[k] with handle hs[k], k = assign[i] from gbhe_batched_plan (largest
 * problems first, each to the worker with the least n^3 work so far;
 * deterministic).  Each hs[k] needs the workspace of the largest problem it
 * is assigned (gbhe_workspace_size with that n, nb and m = iu - il + 1).  The
 * workers are forked from `stream` (they wait for the work already on it) and
 * joined back with the handles' events, so the batch is ordered on `stream`:
 * capturing `stream` into a CUDA graph captures every solve, and later
 * launches of that graph repeat them.  Before the first capture, solve once
 * outside capture (first use sets up device constants), and pass no status
 * checks during capture (gbhe_get_status synchronises).  Returns 0, a negative
 * argument index (-5: an argument of some problem) or a GBHE_E* code; the
 * join is enqueued in every case.  The paper has no counterpart. */
int gbhe_batched_plan(int nworkers, int count, const int* n, int* assign);
int gbhe_hegv_batched(gbhe_handle* hs, void* const* workers, int nworkers, int count, const int* n, const int* nb,
                      gbhe_cplx* const* A, const int* lda, gbhe_cplx* const* B, const int* ldb, const int* il,
                      const int* iu, double* const* w, gbhe_cplx* const* X, const int* ldx, void* stream);

/* Reverse-mode derivative of the selected eigenpairs il..iu of gbhe_hegv
 * (first-order perturbation theory; the paper has no counterpart).  Inputs:
 * the whole decomposition of the same pair -- w_all (n, ascending) and the
 * B-orthonormal X_all (n x n, ldx), e.g. gbhe_hegv with il = 1, iu = n -- and
 * the cotangents of the selected pairs: gw (m = iu-il+1 real) and gX (n x m,
 * ldg), meaning dL = sum_i gw_i dlambda_i + Re sum_i gX_i^H dx_i.  Outputs
 * (n x n, full storage, Hermitian): dA and dB with
 * dL = Re tr(dA^H dA') + Re tr(dB^H dB') for Hermitian perturbations dA', dB'.
 * Terms 1/(lambda_i - lambda_j) with |lambda_i - lambda_j| < delta are dropped
 * (degenerate-gap masking; the eigenvector phase is free, so a loss must not
 * depend on it).  Four n x n x m products on the library's GEMM engine. */
int gbhe_hegv_adjoint(gbhe_handle h, int n, int il, int iu, const double* w_all, const gbhe_cplx* X_all, int ldx,
                      const double* gw, const gbhe_cplx* gX, int ldg, double delta, gbhe_cplx* dA, int ldda,
                      gbhe_cplx* dB, int lddb, void* stream);

/* The complex GEMM that every level-3 step above uses, through the engine
 * selected on the handle (gbhe_set_gemm_engine: the tensor-core CRT GEMM for
 * every product with k >= 16 except the tiniest -- those whose DMMA grid
 * would hold fewer than about 5e4 multiply-adds per 64 x 64 tile -- cut into
 * blocks of gbhe_set_crt_block, and the FP64 DMMA GEMM for the rest),
 * exposed for testing and profiling:
 * C = alpha op(A) op(B) + beta C, complex128 column-major.  opA in {0: N,
 * 1: T, 2: C (conjugate transpose), 3: Hermitian matrix read from its lower
 * triangle}; opB in {0: N, 1: T, 2: C}.  lower != 0 writes only C(i,j) with
 * i >= j.  Not part of Algorithms 1-2; the paper has no counterpart beyond
 * "level 3 BLAS on the GPU" (Section 3). */
int gbhe_zgemm(gbhe_handle h, int opA, int opB, int m, int n, int k, gbhe_cplx alpha, const gbhe_cplx* A,
               int lda, const gbhe_cplx* B, int ldb, gbhe_cplx beta, gbhe_cplx* C, int ldc, int lower,
               void* stream);

/* The same product computed on the FP16 tensor cores with exact modular
 * arithmetic (16 moduli <= 256, Chinese remainder reconstruction, one final
 * rounding to double).  Each row of op(A) and column of op(B) is rounded to
 * 53-bit integers relative to its largest entry, and the products of those
 * integers are exact, so the error is normwise per row and column:
 *   |err_ij| <= 4 eps (max_k |a_ik| sum_k |b_kj| + sum_k |a_ik| max_k |b_kj|)
 *               + eps |c_ij|   (complex; independent of k),
 * which matches an FP64 GEMM for rows/columns of even magnitude and is weaker
 * than its componentwise bound for entries far below their row/column
 * maximum.  Complex (cplx != 0, gbhe_cplx
 * operands) or real (cplx = 0, double operands).  opA in {0,1,2,3} as for
 * gbhe_zgemm, opB in {0,1,2}; k <= 65536.  Needs gbhe_crt_workspace_size bytes
 * of workspace beyond the common part (see gbhe_workspace_size); returns
 * GBHE_EWORKSPACE otherwise.  No counterpart in the paper (a GB300-specific
 * way of doing its level-3 products). */
int gbhe_crt_workspace_size(int m, int n, int k, int cplx, size_t* bytes);
int gbhe_gemm_crt(gbhe_handle h, int cplx, int opA, int opB, int m, int n, int k, gbhe_cplx alpha, const void* A,
                  int lda, const void* B, int ldb, gbhe_cplx beta, void* C, int ldc, int lower, void* stream);

/* The number-theory tables of that engine, exactly as copied to the device
 * (host-only, no CUDA call): moduli p[16]; CRT weights W[16][4], W_l =
 * (M/p_l) * ((M/p_l)^-1 mod p_l) mod M as 128-bit little-endian 32-bit words;
 * M[4] = prod p_l, likewise; k13[16], k26[16], k39[16] = the symmetric
 * residues (in [-p/2, p/2]) of 2^13, 2^26, 2^39 modulo p_l (the limb weights
 * of the FP32 residue split); frac[16] = y_l / p_l rounded to float, y_l =
 * (M/p_l)^-1 mod p_l (the FP32 estimate of the reconstruction's multiple of
 * M).  Any pointer may be NULL.  Returns the number of moduli. */
int gbhe_crt_tables(int* p, unsigned* W, unsigned* M, int* k13, int* k26, int* k39, float* frac);

/* The complex DMMA GEMM of gbhe_zgemm (same operand modes and arguments, no
 * handle) for callers that cannot allocate: code that must not take device
 * memory after start-up, or that holds no handle and so has no workspace to
 * hand over.  It allocates nothing.  Its split-K partial sums live in a
 * statically sized array inside the library (GBHE_ZGEMM_STATIC_SCRATCH
 * complex values, 16 MiB), which the CUDA module provides on load; no part of
 * that array has to start at zero.
 *   - m * n may be at most GBHE_ZGEMM_STATIC_MAX_MN; larger products return
 *     GBHE_ETOOLARGE and leave C untouched.  k is not limited.
 *   - The first call on each device (the device current at the call) looks up
 *     the array's address on that device; make that first call before any
 *     stream capture on the device.
 *   - The array is shared by every call on a device: two calls whose work
 *     overlaps in time (different streams, or different host threads) race on
 *     it and give wrong results.  Calls issued in order on one stream are safe.
 * Returns 0, a negative argument index, GBHE_ETOOLARGE or GBHE_ECUDA.  Not
 * part of the paper's method: the paper has no counterpart. */
#define GBHE_ETOOLARGE (-106)                   /* product larger than the static scratch allows */
#define GBHE_ZGEMM_STATIC_SCRATCH (1 << 20)     /* complex128 values of split-K scratch */
#define GBHE_ZGEMM_STATIC_MAX_MN (1 << 18)      /* largest m * n accepted */
int gbhe_zgemm_static(int opA, int opB, int m, int n, int k, gbhe_cplx alpha, const gbhe_cplx* A, int lda,
                      const gbhe_cplx* B, int ldb, gbhe_cplx beta, gbhe_cplx* C, int ldc, int lower, void* stream);

/* Number of CUDA kernels this library has launched in this process so far
 * (host-side counter; benchmarks difference it around a timed region). */
unsigned long long gbhe_launch_count(void);

/* Kernel-class profiler (process-wide; for benchmarks).  While enabled, the
 * library records a pair of CUDA events on the launching stream around each
 * launch of the classes below and accumulates the algorithmic flop and byte
 * counts that launch performs.  gbhe_profile_enable(1) resets and starts,
 * gbhe_profile_enable(0) stops; gbhe_profile_read synchronises the recorded
 * events and returns, for one class, the launch count, total flops, total
 * bytes and total device milliseconds.  No counterpart in the paper. */
#define GBHE_PROF_ZGEMM 0  /* complex DMMA GEMM (all level-3 steps)        */
#define GBHE_PROF_DGEMM 1  /* real DMMA GEMM (divide-and-conquer merges)   */
#define GBHE_PROF_PANEL 2  /* stage-1 panel QR                             */
#define GBHE_PROF_CHASE 3  /* stage-2 bulge chasing                        */
#define GBHE_PROF_Q2 4     /* Q2 back-transform (bulge reflectors)         */
#define GBHE_PROF_STEDC 5  /* tridiagonal divide and conquer (whole call)  */
#define GBHE_PROF_HEMV 6   /* one-stage Hermitian matrix-vector products   */
#define GBHE_PROF_CRT 7    /* FP64-exact GEMM on FP16 tensor cores (CRT)   */
#define GBHE_PROF_CRT_PREP 8  /* CRT: exponents and residues of the operands */
#define GBHE_PROF_CRT_MMA 9   /* CRT: residue products (tcgen05)             */
#define GBHE_PROF_CRT_REC 10  /* CRT: reconstruction and update of C         */
#define GBHE_PROF_NCLASS 11
int gbhe_profile_enable(int on);
int gbhe_profile_read(int cls, unsigned long long* launches, double* flops, double* bytes, double* ms);

/* Human-readable text for a return/status code. */
const char* gbhe_status_string(int code);

/* Failure-detection self-test (no GPU fault): enqueues on `stream` one kernel
 * that enters the library's bounded device wait (the grid barrier of the
 * cooperative kernels) for a partner that never arrives.  The wait gives up
 * after its time limit (2 s of %globaltimer), records GBHE_ETIMEOUT in the
 * handle's status word and returns normally; the next gbhe_get_status
 * returns GBHE_ETIMEOUT and clears the status, after which the handle and
 * the context are usable as before.  Returns 0, -1 (handle NULL) or
 * GBHE_ECUDA. */
int gbhe_wait_selftest(gbhe_handle h, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* GBHEGV_H_ */
