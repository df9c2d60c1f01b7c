// common.cuh -- shared device/host helpers of libgbhegv (complex128 arithmetic,
// status words, bounded grid barrier, workspace carving).
#pragma once
#include <cuda_runtime.h>
#include <cstdint>
#include <cstddef>
#include <cmath>
#include "../../include/gbhegv.h"

namespace gbhe {

typedef double2 cplx;

__host__ __device__ __forceinline__ cplx mk(double r, double i) { return make_double2(r, i); }
__host__ __device__ __forceinline__ cplx cadd(cplx a, cplx b) { return mk(a.x + b.x, a.y + b.y); }
__host__ __device__ __forceinline__ cplx csub(cplx a, cplx b) { return mk(a.x - b.x, a.y - b.y); }
__host__ __device__ __forceinline__ cplx cmul(cplx a, cplx b) { return mk(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x); }
// a * conj(b)
__host__ __device__ __forceinline__ cplx cmulc(cplx a, cplx b) { return mk(a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y); }
// conj(a) * b
__host__ __device__ __forceinline__ cplx ccmul(cplx a, cplx b) { return mk(a.x * b.x + a.y * b.y, a.x * b.y - a.y * b.x); }
__host__ __device__ __forceinline__ cplx cconj(cplx a) { return mk(a.x, -a.y); }
__host__ __device__ __forceinline__ cplx cscal(double s, cplx a) { return mk(s * a.x, s * a.y); }
__host__ __device__ __forceinline__ double cabs2(cplx a) { return a.x * a.x + a.y * a.y; }
// acc += a * b
__device__ __forceinline__ void cfma(cplx& acc, cplx a, cplx b) {
  acc.x = fma(a.x, b.x, fma(-a.y, b.y, acc.x));
  acc.y = fma(a.x, b.y, fma(a.y, b.x, acc.y));
}
// acc += conj(a) * b
__device__ __forceinline__ void ccfma(cplx& acc, cplx a, cplx b) {
  acc.x = fma(a.x, b.x, fma(a.y, b.y, acc.x));
  acc.y = fma(a.x, b.y, fma(-a.y, b.x, acc.y));
}
// 1 / z
__host__ __device__ __forceinline__ cplx cinv(cplx z) {
  double s = 1.0 / (z.x * z.x + z.y * z.y);
  return mk(z.x * s, -z.y * s);
}
__host__ __device__ __forceinline__ cplx cdiv(cplx a, cplx b) { return cmul(a, cinv(b)); }

// Device status words (one per handle).  word[0] = info (first numerical
// failure), word[1] = error code (GBHE_ETIMEOUT ...), words[4..5] the grid
// barrier of the panel QR, words[8..9] the barrier of the wait self-test.
enum { ST_INFO = 0, ST_ERR = 1, ST_BAR = 4, ST_SELF = 8, ST_WORDS = 64 };

__device__ __forceinline__ void set_info_once(int* st, int info) { atomicCAS(&st[ST_INFO], 0, info); }
__device__ __forceinline__ void set_err_once(int* st, int err) { atomicCAS(&st[ST_ERR], 0, err); }

// Time limit for every device-side wait, in nanoseconds of %globaltimer; on
// expiry the waiter records GBHE_ETIMEOUT and gives up.
#ifndef GBHE_WAIT_NS
#define GBHE_WAIT_NS 2000000000ull
#endif

__device__ __forceinline__ unsigned long long gtimer() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ unsigned ld_acquire(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ int ld_acquire_i(const int* p) {
  int v;
  asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release_i(int* p, int v) {
  asm volatile("st.release.gpu.global.s32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Grid-wide barrier for a cooperatively launched kernel (all CTAs resident).
// bar[0] = arrival count, bar[1] = generation.  Bounded: returns false (and
// records GBHE_ETIMEOUT) if the generation does not advance in time or if
// another CTA already recorded an error.
__device__ __forceinline__ bool grid_barrier(unsigned* bar, unsigned nblocks, int* st) {
  __shared__ int ok_s;
  __syncthreads();
  if (threadIdx.x == 0) {
    int ok = 1;
    unsigned gen = ld_acquire(&bar[1]);
    __threadfence();
    unsigned arrived = atomicAdd(&bar[0], 1u);
    if (arrived == nblocks - 1) {
      atomicExch(&bar[0], 0u);
      __threadfence();
      atomicAdd(&bar[1], 1u);
    } else {
      // the shared status word is looked at only every 64 polls, so that the
      // waiting CTAs do not crowd the L2 slice that holds it
      const unsigned long long t0 = gtimer();
      unsigned polls = 0;
      while (ld_acquire(&bar[1]) == gen) {
        if ((++polls & 63) == 0 && (gtimer() - t0 > GBHE_WAIT_NS || ld_acquire_i(&st[ST_ERR]) != 0)) {
          set_err_once(st, GBHE_ETIMEOUT);
          ok = 0;
          break;
        }
        __nanosleep(64);
      }
    }
    __threadfence();
    ok_s = ok;
  }
  __syncthreads();
  return ok_s != 0;
}

// Host-side count of kernel launches made by this library (benchmark claim).
void count_launch(unsigned k = 1);

// Host-side bump allocator over the caller's workspace.
struct Arena {
  char* base;
  size_t cap;
  size_t off;
  bool measure;  // when true only sizes are accumulated
  template <typename T>
  T* take(size_t count) {
    size_t bytes = (count * sizeof(T) + 255) & ~size_t(255);
    size_t at = off;
    off += bytes;
    if (measure || base == nullptr) return nullptr;
    if (off > cap) return nullptr;
    return reinterpret_cast<T*>(base + at);
  }
  bool ok() const { return measure || off <= cap; }
};

}  // namespace gbhe

// Opaque handle (declared in the public header).
struct gbhe_ctx {
  int device;
  int num_sms;
  size_t smem_optin;
  int* status;          // device, ST_WORDS ints
  int* status_host;     // pinned host mirror
  void* work;           // caller-owned device workspace
  size_t work_bytes;
  int engine;           // GBHE_ENGINE_CRT (default) or GBHE_ENGINE_DMMA
  int crt_block;        // largest tensor-core GEMM block (workspace vs speed)
  cudaEvent_t ev_fork;  // fork / join events of gbhe_hegv_batched
  cudaEvent_t ev_join;
  cudaStream_t aux;     // stage 1's panel stream (lookahead), high priority
  cudaEvent_t ev_a;     // main -> aux: the next panel's columns are updated
  cudaEvent_t ev_b;     // aux -> main: the panel is factored
  int nbr_count;        // band-width rule (gbhe_set_nb_rule); 0 = default
  int nbr_n[GBHE_NB_RULE_MAX];
  double nbr_f[GBHE_NB_RULE_MAX];
  int nbr_nb[GBHE_NB_RULE_MAX];
};

#define GBHE_CUDA(call)                                      \
  do {                                                       \
    cudaError_t e_ = (call);                                 \
    if (e_ != cudaSuccess) return GBHE_ECUDA;                \
  } while (0)
