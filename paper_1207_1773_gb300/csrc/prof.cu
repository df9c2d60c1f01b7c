// prof.cu -- optional kernel-class profiler: CUDA events recorded on the
// launching stream around each instrumented launch, summed on read-out.
#include <vector>
#include "internal.cuh"

namespace gbhe {
namespace {

struct Rec {
  cudaEvent_t a, b;
};

struct ClassAcc {
  std::vector<Rec> pool;
  size_t used = 0;
  unsigned long long launches = 0;
  double flops = 0.0;
  double bytes = 0.0;
};

bool g_on = false;
ClassAcc g_cls[GBHE_PROF_NCLASS];

}  // namespace

bool prof_on() { return g_on; }

ProfScope::ProfScope(cudaStream_t st, int cls, double flops, double bytes) : st_(st), cls_(cls), ev_(nullptr) {
  if (!g_on || cls < 0 || cls >= GBHE_PROF_NCLASS) return;
  ClassAcc& c = g_cls[cls];
  if (c.used == c.pool.size()) {
    Rec r;
    if (cudaEventCreate(&r.a) != cudaSuccess) return;
    if (cudaEventCreate(&r.b) != cudaSuccess) { cudaEventDestroy(r.a); return; }
    c.pool.push_back(r);
  }
  Rec* r = &c.pool[c.used++];
  cudaEventRecord(r->a, st);
  ev_ = r;
  c.launches += 1;
  c.flops += flops;
  c.bytes += bytes;
}

ProfScope::~ProfScope() {
  if (ev_) cudaEventRecord(static_cast<Rec*>(ev_)->b, st_);
}

}  // namespace gbhe

using namespace gbhe;

extern "C" int gbhe_profile_enable(int on) {
  g_on = (on != 0);
  for (int i = 0; i < GBHE_PROF_NCLASS; ++i) {
    g_cls[i].used = 0;
    g_cls[i].launches = 0;
    g_cls[i].flops = 0.0;
    g_cls[i].bytes = 0.0;
  }
  return 0;
}

extern "C" int gbhe_profile_read(int cls, unsigned long long* launches, double* flops, double* bytes, double* ms) {
  if (cls < 0 || cls >= GBHE_PROF_NCLASS) return -1;
  ClassAcc& c = g_cls[cls];
  double tot = 0.0;
  for (size_t i = 0; i < c.used; ++i) {
    if (cudaEventSynchronize(c.pool[i].b) != cudaSuccess) return GBHE_ECUDA;
    float t = 0.f;
    if (cudaEventElapsedTime(&t, c.pool[i].a, c.pool[i].b) != cudaSuccess) return GBHE_ECUDA;
    tot += t;
  }
  if (launches) *launches = c.launches;
  if (flops) *flops = c.flops;
  if (bytes) *bytes = c.bytes;
  if (ms) *ms = tot;
  return 0;
}
