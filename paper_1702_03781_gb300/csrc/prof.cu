// prof.cu -- per-kernel-class device timing behind harp_profile_begin/end.
#include <vector>

#include "prof.cuh"

namespace harp {

namespace {
struct Rec {
  int kind;
  double flops;
  cudaEvent_t e0, e1;
};
struct Profiler {
  unsigned mask = 0;
  std::vector<cudaEvent_t> pool;
  size_t next = 0;
  std::vector<Rec> recs;
  int device = -1;
};
Profiler g_prof;

cudaEvent_t take_event() {
  if (g_prof.next < g_prof.pool.size()) return g_prof.pool[g_prof.next++];
  cudaEvent_t e = nullptr;
  if (cudaEventCreate(&e) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  g_prof.pool.push_back(e);
  ++g_prof.next;
  return e;
}
}  // namespace

ProfScope::ProfScope(int k, double f, cudaStream_t s) : kind(k), flops(f), st(s), slot(-1) {
  if (k < 0 || k >= 32 || !(g_prof.mask & (1u << k))) return;  // k < 0: not recorded
  cudaEvent_t e0 = take_event(), e1 = take_event();
  if (!e0 || !e1) return;
  if (cudaEventRecord(e0, st) != cudaSuccess) {
    cudaGetLastError();
    return;
  }
  g_prof.recs.push_back(Rec{k, f, e0, e1});
  slot = (int)g_prof.recs.size() - 1;
}

ProfScope::~ProfScope() {
  if (slot < 0) return;
  if (cudaEventRecord(g_prof.recs[slot].e1, st) != cudaSuccess) {
    cudaGetLastError();
    g_prof.recs[slot].kind = -1;
  }
}

// Whether any kernel class is being recorded: the refinement's captured
// graphs (the triangular solves, the correction and residual-update
// segments) would hide their launches from the recorder, so they run
// uncaptured meanwhile.
bool profiling_active() { return g_prof.mask != 0; }

}  // namespace harp

using namespace harp;

extern "C" int harp_profile_begin(harp_ctx* ctx, unsigned mask) {
  if (!ctx) return -1;
  g_prof.mask = mask;
  g_prof.recs.clear();
  g_prof.next = 0;
  g_prof.device = ctx->device;
  return HARP_OK;
}

extern "C" int harp_profile_end(harp_ctx* ctx, double* ms, double* flops, long long* launches) {
  if (!ctx) return -1;
  if (!ms) return -2;
  if (!flops) return -3;
  if (!launches) return -4;
  DeviceGuard g(ctx->device);
  for (int k = 0; k < HARP_PROF_KINDS; ++k) {
    ms[k] = 0.0;
    flops[k] = 0.0;
    launches[k] = 0;
  }
  int status = HARP_OK;
  for (const Rec& r : g_prof.recs) {
    if (r.kind < 0) continue;
    if (cudaEventSynchronize(r.e1) != cudaSuccess) {
      status = cuda_status(cudaGetLastError());
      break;
    }
    float t = 0.f;
    if (cudaEventElapsedTime(&t, r.e0, r.e1) != cudaSuccess) {
      status = cuda_status(cudaGetLastError());
      break;
    }
    ms[r.kind] += t;
    flops[r.kind] += r.flops;
    launches[r.kind] += 1;
  }
  g_prof.mask = 0;
  g_prof.recs.clear();
  g_prof.next = 0;
  return status;
}
