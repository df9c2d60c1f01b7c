// internal.cuh -- per-call context and the stage functions shared by the C-ABI.
#pragma once
#include "common.cuh"
#include "gemm.cuh"
#if defined(__has_include)
#if __has_include(<nvtx3/nvToolsExt.h>)
#include <nvtx3/nvToolsExt.h>
#define GBHE_HAVE_NVTX 1
#endif
#endif

namespace gbhe {

// NVTX range around a host-side stage, for Nsight timelines; a no-op when no
// tool is attached (or when the NVTX headers are absent at build time).
class NvtxRange {
 public:
  explicit NvtxRange(const char* name) {
#ifdef GBHE_HAVE_NVTX
    nvtxRangePushA(name);
#else
    (void)name;
#endif
  }
  ~NvtxRange() {
#ifdef GBHE_HAVE_NVTX
    nvtxRangePop();
#endif
  }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};

// Everything a stage needs for one call: the stream, the device status words
// and carved pieces of the caller's workspace.
struct Ctx {
  cudaStream_t st;
  int* status;
  int num_sms;
  cplx* dense_scratch;        // diagonal-block inverses, ceil(n/64)*64*64
  void* gemm_scratch;         // split-K partial sums
  size_t gemm_scratch_bytes;
  void* crt_ws;               // residue planes of the tensor-core FP64 GEMM
  size_t crt_ws_bytes;
  int engine;                 // GBHE_ENGINE_DMMA or GBHE_ENGINE_CRT
  int crt_block;              // largest block of the tensor-core GEMM
  cudaStream_t aux;           // the handle's panel stream and its two events (stage 1 lookahead)
  cudaEvent_t ev_a, ev_b;
  Arena arena;                // the rest, for stage temporaries
};

// One-time set-ups (kernel attributes, __constant__ tables, launch-form
// decisions) belong to a device, not to the process: they are kept in arrays
// indexed by the current device.  Returns that index, or -1 when it cannot be
// read or lies beyond MAX_DEVICES.
constexpr int MAX_DEVICES = 64;
inline int device_slot() {
  int d = -1;
  if (cudaGetDevice(&d) != cudaSuccess || d < 0 || d >= MAX_DEVICES) return -1;
  return d;
}

constexpr size_t GEMM_SCRATCH_BYTES = size_t(32) << 20;
// Workspace of the tensor-core FP64 GEMM: enough for one complex product of
// min(n, block) in every dimension (about 16 GB at n = 10000 with the default
// block); larger products are cut into blocks of that size.
constexpr int CRT_BLOCK = 16384;
size_t crt_budget_bytes(int n, int block);

// FP64 GEMM through the engine selected on the handle: exact modular products
// on the FP16 tensor cores for large products, DMMA otherwise.
int gemm(Ctx& c, const GemmArgs& g, int cplx);
// Complex product through the engine selected on the handle (the scratch
// arguments are kept for the DMMA split-K path, which uses the context's).
inline int zgemm(Ctx& c, const GemmArgs& g, void*, size_t) { return gemm(c, g, 1); }

// RAII marker for the optional profiler: records CUDA events around the
// enclosed launches of class `cls` when profiling is on (prof.cu).
bool prof_on();
class ProfScope {
 public:
  ProfScope(cudaStream_t st, int cls, double flops, double bytes);
  ~ProfScope();
  ProfScope(const ProfScope&) = delete;
  ProfScope& operator=(const ProfScope&) = delete;

 private:
  cudaStream_t st_;
  int cls_;
  void* ev_;
};

// FP64-exact GEMM on the FP16 tensor cores (crt.cu); workspace passed
// explicitly; an expired bounded wait records GBHE_ETIMEOUT in status[ST_ERR].
size_t crt_gemm_ws_bytes(int M, int N, int K, int cplx);
int crt_gemm(cudaStream_t st, const GemmArgs& g, int cplx, void* ws, size_t ws_bytes, int* status);

// Batched form: entry z computes C_z = alpha op(A_z) op(B_z) + beta C_z with
// its own sizes (M_z <= maxM, N_z <= maxN, K_z <= maxK) and pointers; the
// descriptor array lives in device memory.  Operand modes, alpha and beta are
// shared by all entries.
struct CrtDesc {
  const void* A;
  const void* B;
  void* C;
  const int* cmap;  // optional: column j of the product goes to column cmap[j] of C
  int M, N, K, lda, ldb, ldc;
};
size_t crt_batched_ws_bytes(int nbatch, int maxM, int maxN, int maxK, int cplx);
// `flops` (FP64-equivalent, for the profiler only) is the caller's count of
// the batch's work; the entries' sizes live on the device.
int crt_gemm_batched(cudaStream_t st, int opA, int opB, cplx alpha, cplx beta, int cplx_flag, const CrtDesc* d_desc,
                     int nbatch, int maxM, int maxN, int maxK, void* ws, size_t ws_bytes, int* status,
                     double flops = 0.0);

size_t dense_ws_bytes(int n);
int potrf_run(Ctx& c, int n, cplx* B, int ldb);
int trsm_run(Ctx& c, int trans, int n, int m, const cplx* L, int ldl, cplx* X, int ldx);
int hegst_run(Ctx& c, int n, cplx* A, int lda, const cplx* L, int ldl);

size_t he2hb_ws_bytes(int n, int nb, int num_sms);
int he2hb_run(Ctx& c, int n, int nb, cplx* A, int lda, cplx* T1, cplx* tau1);

inline int hb2st_J(int n, int nb) { return n > 1 ? (n - 1 + nb - 1) / nb : 0; }
size_t hb2st_ws_bytes(int n, int nb);
int hb2st_run(Ctx& c, int n, int nb, const cplx* A, int lda, double* d, double* e, cplx* V2, cplx* tau2);

size_t stedc_ws_bytes(int n);
int stedc_run(Ctx& c, int n, const double* d, const double* e, int il, int iu, double* w, double* Z,
              int ldz);

size_t unmtr_ws_bytes(int n, int nb, int m);
int unmtr2_run(Ctx& c, int n, int nb, int m, const cplx* A, int lda, const cplx* T1, const cplx* V2,
               const cplx* tau2, const double* Z, int ldz, cplx* X, int ldx);

size_t onestage_ws_bytes(int n, int m);
size_t adjoint_ws_bytes(int n, int m);
int adjoint_run(Ctx& c, int n, int il, int iu, const double* w_all, const cplx* X, int ldx, const double* g,
                const cplx* G, int ldg, double delta, cplx* dA, int ldda, cplx* dB, int lddb);
int hegv_onestage_run(Ctx& c, int n, cplx* A, int lda, cplx* B, int ldb, int il, int iu, double* w,
                      cplx* X, int ldx);

}  // namespace gbhe
