// api.cu -- the C-ABI of libgbhegv (declared in include/gbhegv.h): handle,
// workspace, argument checks, per-stage entry points and the drivers.
#include <algorithm>
#include <cstdlib>
#include <cstring>
#include "internal.cuh"

using namespace gbhe;

namespace gbhe {
static unsigned long long g_launches = 0;
void count_launch(unsigned k) { __atomic_fetch_add(&g_launches, (unsigned long long)k, __ATOMIC_RELAXED); }
}  // namespace gbhe

namespace {

int default_nb(int n) {
  if (n <= 128) return 16;
  if (n <= 1024) return 32;
  return 64;
}

int nb_rule_check(int count, const int* n_max, const double* frac_max, const int* nb) {
  if (count < 0 || count > GBHE_NB_RULE_MAX) return -1;
  if (count > 0 && !n_max) return -2;
  if (count > 0 && !frac_max) return -3;
  if (count > 0 && !nb) return -4;
  for (int i = 0; i < count; ++i) {
    if (n_max[i] < 1) return -2;
    if (!(frac_max[i] > 0.0 && frac_max[i] <= 1.0)) return -3;
    if (nb[i] < 1 || nb[i] > 64) return -4;
  }
  return 0;
}

// The entries of the smallest n_max >= n (else of the largest n_max); among
// them the smallest frac_max >= m/n (else the largest frac_max); the first of
// equal entries.  An nb that is not below n gives way to the default.
int nb_rule_eval(int count, const int* n_max, const double* frac_max, const int* nb, int n, int m) {
  if (count == 0) return default_nb(n);
  int nsel = -1, nbig = n_max[0];
  for (int i = 0; i < count; ++i) {
    nbig = std::max(nbig, n_max[i]);
    if (n_max[i] >= n && (nsel < 0 || n_max[i] < nsel)) nsel = n_max[i];
  }
  if (nsel < 0) nsel = nbig;
  const double f = n > 0 ? (double)m / n : 1.0;
  int fit = -1, big = -1;
  for (int i = 0; i < count; ++i) {
    if (n_max[i] != nsel) continue;
    if (big < 0 || frac_max[i] > frac_max[big]) big = i;
    if (frac_max[i] >= f && (fit < 0 || frac_max[i] < frac_max[fit])) fit = i;
  }
  const int v = nb[fit >= 0 ? fit : big];
  return v < n ? v : default_nb(n);
}

int resolve_nb(gbhe_handle h, int n, int m) {
  return nb_rule_eval(h->nbr_count, h->nbr_n, h->nbr_f, h->nbr_nb, n, m);
}

// Workspace every call carves first: split-K scratch and the diagonal-block
// inverses.
size_t common_bytes(gbhe_handle h, int n) {
  return GEMM_SCRATCH_BYTES + dense_ws_bytes(n) + crt_budget_bytes(n, h->crt_block) + 1024;
}

size_t stage_bytes(gbhe_handle h, int n, int nb, int m) {
  size_t s = 0;
  s = std::max(s, he2hb_ws_bytes(n, nb, h->num_sms));
  s = std::max(s, hb2st_ws_bytes(n, nb));
  s = std::max(s, stedc_ws_bytes(n));
  s = std::max(s, unmtr_ws_bytes(n, nb, m));
  s = std::max(s, onestage_ws_bytes(n, m));
  s = std::max(s, adjoint_ws_bytes(n, m));
  return s;
}

// Outputs of the intermediate stages that gbhe_hegv keeps in the workspace.
size_t driver_bytes(int n, int nb, int m) {
  const size_t nn = (size_t)std::max(n, 1), mm = (size_t)std::max(m, 1);
  const size_t npan = (nn + nb - 1) / nb;
  const size_t J = (size_t)std::max(hb2st_J(n, nb), 1);
  size_t b = 0;
  b += npan * nb * nb * sizeof(cplx) + 256;  // T1
  b += nn * sizeof(cplx) + 256;              // tau1
  b += nn * J * nb * sizeof(cplx) + 256;     // V2
  b += nn * J * sizeof(cplx) + 256;          // tau2
  b += 2 * nn * sizeof(double) + 512;        // d, e
  b += nn * mm * sizeof(double) + 256;       // Z
  return b;
}

int make_ctx(gbhe_handle h, int n, void* stream, Ctx* c) {
  if (!h) return GBHE_EWORKSPACE;
  if (!h->work) return GBHE_EWORKSPACE;
  c->st = reinterpret_cast<cudaStream_t>(stream);
  c->status = h->status;
  c->num_sms = h->num_sms;
  c->arena.base = reinterpret_cast<char*>(h->work);
  c->arena.cap = h->work_bytes;
  c->arena.off = 0;
  c->arena.measure = false;
  c->gemm_scratch = c->arena.take<char>(GEMM_SCRATCH_BYTES);
  c->gemm_scratch_bytes = GEMM_SCRATCH_BYTES;
  c->dense_scratch = c->arena.take<cplx>(dense_ws_bytes(n) / sizeof(cplx));
  if (!c->arena.ok() || !c->gemm_scratch) return GBHE_EWORKSPACE;
  c->engine = h->engine;
  c->crt_block = h->crt_block;
  c->aux = h->aux;
  c->ev_a = h->ev_a;
  c->ev_b = h->ev_b;
  c->crt_ws = nullptr;
  c->crt_ws_bytes = 0;
  if (h->engine == GBHE_ENGINE_CRT) {
    const size_t cb = crt_budget_bytes(n, h->crt_block);
    const size_t save = c->arena.off;
    char* ws = c->arena.take<char>(cb);
    if (c->arena.ok() && ws) {
      c->crt_ws = ws;
      c->crt_ws_bytes = cb;
    } else {
      c->arena.off = save;  // workspace too small for the tensor-core engine: DMMA only
    }
  }
  if (cudaSetDevice(h->device) != cudaSuccess) return GBHE_ECUDA;
  return 0;
}

inline cplx* Z_(gbhe_cplx* p) { return reinterpret_cast<cplx*>(p); }
inline const cplx* Z_(const gbhe_cplx* p) { return reinterpret_cast<const cplx*>(p); }

}  // namespace

extern "C" {

int gbhe_default_nb(int n) { return default_nb(n); }

int gbhe_nb_rule_pick(int count, const int* n_max, const double* frac_max, const int* nb, int n, int m,
                      int* nb_out) {
  const int rc = nb_rule_check(count, n_max, frac_max, nb);
  if (rc) return rc;
  if (n < 0 || m < 0 || m > n) return -5;
  if (!nb_out) return -6;
  *nb_out = nb_rule_eval(count, n_max, frac_max, nb, n, m);
  return 0;
}

int gbhe_set_nb_rule(gbhe_handle h, int count, const int* n_max, const double* frac_max, const int* nb) {
  if (!h) return -1;
  const int rc = nb_rule_check(count, n_max, frac_max, nb);
  if (rc) return rc - 1;
  for (int i = 0; i < count; ++i) {
    h->nbr_n[i] = n_max[i];
    h->nbr_f[i] = frac_max[i];
    h->nbr_nb[i] = nb[i];
  }
  h->nbr_count = count;
  return 0;
}

int gbhe_resolve_nb(gbhe_handle h, int n, int m, int* nb) {
  if (!h) return -1;
  if (n < 0 || m < 0 || m > n) return -2;
  if (!nb) return -3;
  *nb = resolve_nb(h, n, m);
  return 0;
}

int gbhe_set_gemm_engine(gbhe_handle h, int engine) {
  if (!h) return -1;
  if (engine != GBHE_ENGINE_DMMA && engine != GBHE_ENGINE_CRT) return -2;
  h->engine = engine;
  return 0;
}

int gbhe_hegv_adjoint(gbhe_handle h, int n, int il, int iu, const double* w_all, const gbhe_cplx* X_all, int ldx,
                      const double* gw, const gbhe_cplx* gX, int ldg, double delta, gbhe_cplx* dA, int ldda,
                      gbhe_cplx* dB, int lddb, void* stream) {
  if (!h) return -1;
  if (n < 0) return -2;
  if (n > 0 && (il < 1 || il > n)) return -3;
  if (n > 0 && (iu < il || iu > n)) return -4;
  if (n > 0 && !w_all) return -5;
  if (n > 0 && !X_all) return -6;
  if (ldx < std::max(1, n)) return -7;
  if (n > 0 && !gw) return -8;
  if (n > 0 && !gX) return -9;
  if (ldg < std::max(1, n)) return -10;
  if (!(delta >= 0.0)) return -11;
  if (n > 0 && !dA) return -12;
  if (ldda < std::max(1, n)) return -13;
  if (n > 0 && !dB) return -14;
  if (lddb < std::max(1, n)) return -15;
  if (n == 0) return 0;
  Ctx c;
  int rc = make_ctx(h, n, stream, &c);
  if (rc) return rc;
  return adjoint_run(c, n, il, iu, w_all, Z_(X_all), ldx, gw, Z_(gX), ldg, delta, Z_(dA), ldda, Z_(dB), lddb);
}

int gbhe_set_crt_block(gbhe_handle h, int block) {
  if (!h) return -1;
  if (block < 128 || block > CRT_BLOCK) return -2;
  h->crt_block = block;
  return 0;
}

unsigned long long gbhe_launch_count(void) { return __atomic_load_n(&g_launches, __ATOMIC_RELAXED); }

int gbhe_create(gbhe_handle* handle, int device) {
  if (!handle) return -1;
  *handle = nullptr;
  if (cudaSetDevice(device) != cudaSuccess) return GBHE_ECUDA;
  gbhe_ctx* h = new gbhe_ctx();
  h->device = device;
  cudaDeviceProp p;
  if (cudaGetDeviceProperties(&p, device) != cudaSuccess) { delete h; return GBHE_ECUDA; }
  h->num_sms = p.multiProcessorCount;
  h->smem_optin = p.sharedMemPerBlockOptin;
  if (cudaMalloc(&h->status, ST_WORDS * sizeof(int)) != cudaSuccess) { delete h; return GBHE_ECUDA; }
  if (cudaMemset(h->status, 0, ST_WORDS * sizeof(int)) != cudaSuccess) { cudaFree(h->status); delete h; return GBHE_ECUDA; }
  if (cudaMallocHost(&h->status_host, ST_WORDS * sizeof(int)) != cudaSuccess) {
    cudaFree(h->status); delete h; return GBHE_ECUDA;
  }
  h->work = nullptr;
  h->work_bytes = 0;
  h->engine = GBHE_ENGINE_CRT;
  h->crt_block = CRT_BLOCK;
  h->nbr_count = 0;
  int prio_lo = 0, prio_hi = 0;
  if (cudaDeviceGetStreamPriorityRange(&prio_lo, &prio_hi) != cudaSuccess) prio_hi = 0;
  if (cudaEventCreateWithFlags(&h->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&h->ev_join, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&h->ev_a, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&h->ev_b, cudaEventDisableTiming) != cudaSuccess ||
      cudaStreamCreateWithPriority(&h->aux, cudaStreamNonBlocking, prio_hi) != cudaSuccess) {
    cudaFree(h->status); cudaFreeHost(h->status_host); delete h; return GBHE_ECUDA;
  }
  *handle = h;
  return 0;
}

int gbhe_destroy(gbhe_handle h) {
  if (!h) return 0;
  cudaSetDevice(h->device);
  cudaStreamSynchronize(h->aux);
  cudaStreamDestroy(h->aux);
  cudaEventDestroy(h->ev_fork);
  cudaEventDestroy(h->ev_join);
  cudaEventDestroy(h->ev_a);
  cudaEventDestroy(h->ev_b);
  cudaFree(h->status);
  cudaFreeHost(h->status_host);
  delete h;
  return 0;
}

int gbhe_workspace_size(gbhe_handle h, int n, int nb, int m, size_t* bytes) {
  if (!h) return -1;
  if (n < 0) return -2;
  if (m < 0 || m > n) return -4;
  if (nb == 0) nb = resolve_nb(h, n, m);
  if (nb < 1 || nb > 128) return -3;
  if (!bytes) return -5;
  *bytes = common_bytes(h, n) + driver_bytes(n, nb, m) + stage_bytes(h, n, nb, m) + 4096;
  return 0;
}

int gbhe_set_workspace(gbhe_handle h, void* dwork, size_t bytes) {
  if (!h) return -1;
  if (dwork && (reinterpret_cast<uintptr_t>(dwork) & 255)) return -2;
  h->work = dwork;
  h->work_bytes = dwork ? bytes : 0;
  return 0;
}

int gbhe_get_status(gbhe_handle h, void* stream) {
  if (!h) return -1;
  cudaSetDevice(h->device);
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  if (cudaStreamSynchronize(st) != cudaSuccess) return GBHE_ECUDA;
  if (cudaMemcpy(h->status_host, h->status, ST_WORDS * sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess)
    return GBHE_ECUDA;
  int info = h->status_host[ST_INFO], err = h->status_host[ST_ERR];
  if (info != 0 || err != 0)
    if (cudaMemset(h->status, 0, ST_WORDS * sizeof(int)) != cudaSuccess) return GBHE_ECUDA;
  if (info > 0) return info;
  return err;
}

int gbhe_sync_status(gbhe_handle h, void* stream) { return gbhe_get_status(h, stream); }

const char* gbhe_status_string(int code) {
  switch (code) {
    case 0: return "success";
    case GBHE_EWORKSPACE: return "workspace missing or too small";
    case GBHE_ECUDA: return "CUDA runtime error";
    case GBHE_ETIMEOUT: return "bounded device wait expired";
    case GBHE_ENONFINITE: return "non-finite value";
    case GBHE_ENOTCONV: return "iteration did not converge";
    default: break;
  }
  if (code > 0) return "leading minor of B not positive definite";
  return "invalid argument";
}

int gbhe_potrf(gbhe_handle h, int n, gbhe_cplx* B, int ldb, void* stream) {
  if (!h) return -1;
  if (n < 0) return -2;
  if (n > 0 && !B) return -3;
  if (ldb < std::max(1, n)) return -4;
  Ctx c;
  int rc = make_ctx(h, n, stream, &c);
  if (rc) return rc;
  return potrf_run(c, n, Z_(B), ldb);
}

int gbhe_hegst(gbhe_handle h, int n, gbhe_cplx* A, int lda, const gbhe_cplx* L, int ldl, void* stream) {
  if (!h) return -1;
  if (n < 0) return -2;
  if (n > 0 && !A) return -3;
  if (lda < std::max(1, n)) return -4;
  if (n > 0 && !L) return -5;
  if (ldl < std::max(1, n)) return -6;
  Ctx c;
  int rc = make_ctx(h, n, stream, &c);
  if (rc) return rc;
  return hegst_run(c, n, Z_(A), lda, Z_(L), ldl);
}

int gbhe_he2hb(gbhe_handle h, int n, int nb, gbhe_cplx* A, int lda, gbhe_cplx* T1, gbhe_cplx* tau1,
               void* stream) {
  if (!h) return -1;
  if (n < 0) return -2;
  if (nb < 1 || nb > 128) return -3;
  if (n > 0 && !A) return -4;
  if (lda < std::max(1, n)) return -5;
  if (n > 0 && !T1) return -6;
  if (n > 0 && !tau1) return -7;
  Ctx c;
  int rc = make_ctx(h, n, stream, &c);
  if (rc) return rc;
  return he2hb_run(c, n, nb, Z_(A), lda, Z_(T1), Z_(tau1));
}

int gbhe_hb2st_sizes(int n, int nb, size_t* v2_elems, size_t* tau2_elems) {
  if (n < 0) return -1;
  if (nb < 1 || nb > 128) return -2;
  const size_t J = (size_t)hb2st_J(n, nb);
  if (v2_elems) *v2_elems = (size_t)n * J * nb;
  if (tau2_elems) *tau2_elems = (size_t)n * J;
  return 0;
}

int gbhe_hb2st(gbhe_handle h, int n, int nb, const gbhe_cplx* A, int lda, double* d, double* e, gbhe_cplx* V2,
               gbhe_cplx* tau2, void* stream) {
  if (!h) return -1;
  if (n < 0) return -2;
  if (nb < 1 || nb > 64) return -3;
  if (n > 0 && !A) return -4;
  if (lda < std::max(1, n)) return -5;
  if (n > 0 && !d) return -6;
  if (n > 1 && !e) return -7;
  if (n > 1 && (!V2 || !tau2)) return -8;
  Ctx c;
  int rc = make_ctx(h, n, stream, &c);
  if (rc) return rc;
  return hb2st_run(c, n, nb, Z_(A), lda, d, e, Z_(V2), Z_(tau2));
}

int gbhe_stedc(gbhe_handle h, int n, const double* d, const double* e, int il, int iu, double* w, double* Z,
               int ldz, void* stream) {
  if (!h) return -1;
  if (n < 0) return -2;
  if (n > 0 && !d) return -3;
  if (n > 1 && !e) return -4;
  if (n > 0 && (il < 1 || il > n)) return -5;
  if (n > 0 && (iu < il || iu > n)) return -6;
  if (n > 0 && !w) return -7;
  if (n > 0 && !Z) return -8;
  if (ldz < std::max(1, n)) return -9;
  Ctx c;
  int rc = make_ctx(h, n, stream, &c);
  if (rc) return rc;
  return stedc_run(c, n, d, e, il, iu, w, Z, ldz);
}

int gbhe_unmtr_2stage(gbhe_handle h, int n, int nb, int m, const gbhe_cplx* A, int lda, const gbhe_cplx* T1,
                      const gbhe_cplx* V2, const gbhe_cplx* tau2, const double* Z, int ldz, gbhe_cplx* X, int ldx,
                      void* stream) {
  if (!h) return -1;
  if (n < 0) return -2;
  if (nb < 1 || nb > 128) return -3;
  if (m < 0) return -4;
  if (n > 0 && !A) return -5;
  if (lda < std::max(1, n)) return -6;
  if (n > 0 && !T1) return -7;
  if (n > 1 && !V2) return -8;
  if (n > 1 && !tau2) return -9;
  if (n > 0 && m > 0 && !Z) return -10;
  if (ldz < std::max(1, n)) return -11;
  if (n > 0 && m > 0 && !X) return -12;
  if (ldx < std::max(1, n)) return -13;
  Ctx c;
  int rc = make_ctx(h, n, stream, &c);
  if (rc) return rc;
  return unmtr2_run(c, n, nb, m, Z_(A), lda, Z_(T1), Z_(V2), Z_(tau2), Z, ldz, Z_(X), ldx);
}

int gbhe_trsm_lh(gbhe_handle h, int n, int m, const gbhe_cplx* L, int ldl, gbhe_cplx* X, int ldx, void* stream) {
  if (!h) return -1;
  if (n < 0) return -2;
  if (m < 0) return -3;
  if (n > 0 && !L) return -4;
  if (ldl < std::max(1, n)) return -5;
  if (n > 0 && m > 0 && !X) return -6;
  if (ldx < std::max(1, n)) return -7;
  Ctx c;
  int rc = make_ctx(h, n, stream, &c);
  if (rc) return rc;
  return trsm_run(c, 1, n, m, Z_(L), ldl, Z_(X), ldx);
}

int gbhe_hegv(gbhe_handle h, int n, int nb, gbhe_cplx* A, int lda, gbhe_cplx* B, int ldb, int il, int iu,
              double* w, gbhe_cplx* X, int ldx, void* stream) {
  if (!h) return -1;
  if (n < 0) return -2;
  if (nb == 0) nb = (n > 0 && il >= 1 && iu >= il && iu <= n) ? resolve_nb(h, n, iu - il + 1) : default_nb(n);
  if (nb < 1 || nb > 64) return -3;
  if (n > 0 && !A) return -4;
  if (lda < std::max(1, n)) return -5;
  if (n > 0 && !B) return -6;
  if (ldb < std::max(1, n)) return -7;
  if (n > 0 && (il < 1 || il > n)) return -8;
  if (n > 0 && (iu < il || iu > n)) return -9;
  if (n > 0 && !w) return -10;
  if (n > 0 && !X) return -11;
  if (ldx < std::max(1, n)) return -12;
  if (n == 0) return 0;
  const int m = iu - il + 1;
  Ctx c;
  int rc = make_ctx(h, n, stream, &c);
  if (rc) return rc;
  Arena& ar = c.arena;
  const int npan = (n + nb - 1) / nb;
  const int J = std::max(hb2st_J(n, nb), 1);
  cplx* T1 = ar.take<cplx>((size_t)npan * nb * nb);
  cplx* tau1 = ar.take<cplx>((size_t)n);
  cplx* V2 = ar.take<cplx>((size_t)n * J * nb);
  cplx* tau2 = ar.take<cplx>((size_t)n * J);
  double* d = ar.take<double>((size_t)n);
  double* e = ar.take<double>((size_t)n);
  double* Z = ar.take<double>((size_t)n * m);
  if (!ar.ok() || !Z) return GBHE_EWORKSPACE;
  cplx* Ac = Z_(A);
  cplx* L = Z_(B);
  NvtxRange all("gbhe_hegv");
#define GBHE_STAGE(name, call)   \
  do {                           \
    NvtxRange r_(name);          \
    if ((rc = (call))) return rc; \
  } while (0)
  GBHE_STAGE("potrf", potrf_run(c, n, L, ldb));
  GBHE_STAGE("hegst", hegst_run(c, n, Ac, lda, L, ldb));
  GBHE_STAGE("he2hb", he2hb_run(c, n, nb, Ac, lda, T1, tau1));
  GBHE_STAGE("hb2st", hb2st_run(c, n, nb, Ac, lda, d, e, V2, tau2));
  GBHE_STAGE("stedc", stedc_run(c, n, d, e, il, iu, w, Z, n));
  GBHE_STAGE("unmtr_2stage", unmtr2_run(c, n, nb, m, Ac, lda, T1, V2, tau2, Z, n, Z_(X), ldx));
  GBHE_STAGE("trsm_lh", trsm_run(c, 1, n, m, L, ldb, Z_(X), ldx));
#undef GBHE_STAGE
  return 0;
}

int gbhe_hegv_onestage(gbhe_handle h, int n, gbhe_cplx* A, int lda, gbhe_cplx* B, int ldb, int il, int iu,
                       double* w, gbhe_cplx* X, int ldx, void* stream) {
  if (!h) return -1;
  if (n < 0) return -2;
  if (n > 0 && !A) return -3;
  if (lda < std::max(1, n)) return -4;
  if (n > 0 && !B) return -5;
  if (ldb < std::max(1, n)) return -6;
  if (n > 0 && (il < 1 || il > n)) return -7;
  if (n > 0 && (iu < il || iu > n)) return -8;
  if (n > 0 && !w) return -9;
  if (n > 0 && !X) return -10;
  if (ldx < std::max(1, n)) return -11;
  if (n == 0) return 0;
  Ctx c;
  int rc = make_ctx(h, n, stream, &c);
  if (rc) return rc;
  return hegv_onestage_run(c, n, Z_(A), lda, Z_(B), ldb, il, iu, w, Z_(X), ldx);
}

int gbhe_zgemm(gbhe_handle h, int opA, int opB, int m, int n, int k, gbhe_cplx alpha, const gbhe_cplx* A,
               int lda, const gbhe_cplx* B, int ldb, gbhe_cplx beta, gbhe_cplx* C, int ldc, int lower,
               void* stream) {
  if (!h) return -1;
  if (opA < 0 || opA > 3) return -2;
  if (opB < 0 || opB > 2) return -3;
  if (m < 0) return -4;
  if (n < 0) return -5;
  if (k < 0) return -6;
  const int ra = (opA == OP_N || opA == OP_H) ? m : k;
  if (m > 0 && k > 0 && !A) return -8;
  if (lda < std::max(1, ra)) return -9;
  const int rb = (opB == OP_N) ? k : n;
  if (n > 0 && k > 0 && !B) return -10;
  if (ldb < std::max(1, rb)) return -11;
  if (m > 0 && n > 0 && !C) return -13;
  if (ldc < std::max(1, m)) return -14;
  if (opA == OP_H && m != k) return -2;
  Ctx c;
  int rc = make_ctx(h, std::max(std::max(m, n), k), stream, &c);
  if (rc) return rc;
  // through the engine selected on the handle (large products cut into blocks)
  return gemm(c, gemm_args(opA, opB, m, n, k, mk(alpha.re, alpha.im), A, lda, B, ldb, mk(beta.re, beta.im), C, ldc,
                           lower),
              1);
}

int gbhe_crt_workspace_size(int m, int n, int k, int cplx, size_t* bytes) {
  if (m < 0) return -1;
  if (n < 0) return -2;
  if (k < 0 || k > 65536) return -3;
  if (!bytes) return -5;
  *bytes = crt_gemm_ws_bytes(std::max(m, 1), std::max(n, 1), std::max(k, 1), cplx ? 1 : 0);
  return 0;
}

int gbhe_gemm_crt(gbhe_handle h, int cplx, int opA, int opB, int m, int n, int k, gbhe_cplx alpha, const void* A,
                  int lda, const void* B, int ldb, gbhe_cplx beta, void* C, int ldc, int lower, void* stream) {
  if (!h) return -1;
  if (opA < 0 || opA > 3 || (!cplx && opA == OP_H)) return -3;
  if (opB < 0 || opB > 2) return -4;
  if (m < 0) return -5;
  if (n < 0) return -6;
  if (k < 0 || k > 65536) return -7;
  const int ra = (opA == OP_N || opA == OP_H) ? m : k;
  if (m > 0 && k > 0 && !A) return -9;
  if (lda < std::max(1, ra)) return -10;
  const int rb = (opB == OP_N) ? k : n;
  if (n > 0 && k > 0 && !B) return -11;
  if (ldb < std::max(1, rb)) return -12;
  if (m > 0 && n > 0 && !C) return -14;
  if (ldc < std::max(1, m)) return -15;
  if (opA == OP_H && m != k) return -3;
  Ctx c;
  int rc = make_ctx(h, 1, stream, &c);
  if (rc) return rc;
  if (m == 0 || n == 0) return 0;
  GemmArgs g = gemm_args(opA, opB, m, n, k, mk(alpha.re, alpha.im), A, lda, B, ldb, mk(beta.re, beta.im), C, ldc,
                         lower);
  if (k == 0) return cplx ? zgemm(c.st, g, nullptr, 0) : dgemm(c.st, g, nullptr, 0);
  const size_t need = crt_gemm_ws_bytes(m, n, k, cplx ? 1 : 0);
  char* ws = c.arena.take<char>(need);
  if (!c.arena.ok() || !ws) return GBHE_EWORKSPACE;
  return crt_gemm(c.st, g, cplx ? 1 : 0, ws, need, c.status);
}

}  // extern "C"
