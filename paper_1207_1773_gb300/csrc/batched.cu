// batched.cu -- many independent generalized eigenproblems of uneven sizes
// (the "solved many times" use case of the paper's introduction): a host-side
// scheduler that spreads the problems over worker streams, each with its own
// handle, forked from and joined back to the caller's stream with events, so
// that capturing the caller's stream captures the whole batch as one graph.
#include <algorithm>
#include <numeric>
#include <vector>

#include "internal.cuh"

namespace {

// Largest problems first, each to the worker with the least n^3 work so far
// (ties to the lower index): deterministic, so that gbhe_batched_plan and
// gbhe_hegv_batched agree.
void make_plan(int nworkers, int count, const int* n, int* assign) {
  std::vector<int> order(count);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return n[a] > n[b]; });
  std::vector<double> load(nworkers, 0.0);
  for (int i : order) {
    int best = 0;
    for (int k = 1; k < nworkers; ++k)
      if (load[k] < load[best]) best = k;
    assign[i] = best;
    load[best] += (double)n[i] * n[i] * n[i];
  }
}

}  // namespace

extern "C" int gbhe_batched_plan(int nworkers, int count, const int* n, int* assign) {
  if (nworkers < 1) return -1;
  if (count < 0) return -2;
  if (count > 0 && !n) return -3;
  if (count > 0 && !assign) return -4;
  for (int i = 0; i < count; ++i)
    if (n[i] < 0) return -3;
  make_plan(nworkers, count, n, assign);
  return 0;
}

extern "C" int gbhe_hegv_batched(gbhe_handle* hs, void* const* workers, int nworkers, int count, const int* n,
                                 const int* nb, gbhe_cplx* const* A, const int* lda, gbhe_cplx* const* B,
                                 const int* ldb, const int* il, const int* iu, double* const* w,
                                 gbhe_cplx* const* X, const int* ldx, void* stream) {
  using namespace gbhe;
  if (!hs) return -1;
  if (!workers) return -2;
  if (nworkers < 1) return -3;
  if (count < 0) return -4;
  if (count > 0 && (!n || !nb || !A || !lda || !B || !ldb || !il || !iu || !w || !X || !ldx)) return -5;
  for (int k = 0; k < nworkers; ++k)
    if (!hs[k] || !workers[k]) return -1;
  if (count == 0) return 0;
  std::vector<int> assign(count);
  make_plan(nworkers, count, n, assign.data());
  cudaStream_t origin = reinterpret_cast<cudaStream_t>(stream);
  // fork: every worker waits for the work already on the caller's stream
  GBHE_CUDA(cudaEventRecord(hs[0]->ev_fork, origin));
  for (int k = 0; k < nworkers; ++k)
    GBHE_CUDA(cudaStreamWaitEvent(reinterpret_cast<cudaStream_t>(workers[k]), hs[0]->ev_fork, 0));
  int rc = 0;
  for (int i = 0; i < count && !rc; ++i) {
    const int k = assign[i];
    rc = gbhe_hegv(hs[k], n[i], nb[i], A[i], lda[i], B[i], ldb[i], il[i], iu[i], w[i], X[i], ldx[i], workers[k]);
    if (rc > 0 || rc < -100) break;
    if (rc < 0) rc = -5;  // an argument of problem i
  }
  // join: the caller's stream waits for every worker, also after an error
  for (int k = 0; k < nworkers; ++k) {
    cudaEventRecord(hs[k]->ev_join, reinterpret_cast<cudaStream_t>(workers[k]));
    cudaStreamWaitEvent(origin, hs[k]->ev_join, 0);
  }
  return rc;
}
