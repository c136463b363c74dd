// Kernel launch counting and optional per-kind CUDA-event timing.
#include <atomic>
#include <vector>

#include "../../include/zolo_csd.h"
#include "profile.h"

namespace zcsd {

static std::atomic<long long> g_launches{0};
thread_local Profiler* t_prof = nullptr;

void count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }

long long launch_count() { return g_launches.load(); }

int Profiler::event() {
  if (used == (int)pool.size()) {
    cudaEvent_t e;
    ZCSD_CUDA(cudaEventCreate(&e));
    pool.push_back(e);
  }
  return used++;
}

void Profiler::flush() {
  if (recs.empty()) {
    used = 0;
    return;
  }
  ZCSD_CUDA(cudaEventSynchronize(pool[recs.back().b]));
  for (const Rec& r : recs) {
    float ms_ = 0.f;
    ZCSD_CUDA(cudaEventElapsedTime(&ms_, pool[r.a], pool[r.b]));
    ms[r.kind] += ms_;
    flops[r.kind] += r.flops;
    count[r.kind] += 1;
    if ((r.kind == PK_GEMM || r.kind == PK_TC) && r.site >= 0 && r.site < PROF_SITES) {
      site_ms[r.site] += ms_;
      site_flops[r.site] += r.flops;
      site_count[r.site] += 1;
    }
  }
  recs.clear();
  used = 0;
}

void Profiler::reset() {
  recs.clear();
  used = 0;
  for (int k = 0; k < PK_KINDS; ++k) { ms[k] = 0; flops[k] = 0; count[k] = 0; }
  for (int k = 0; k < PROF_SITES; ++k) { site_ms[k] = 0; site_flops[k] = 0; site_count[k] = 0; }
}

Profiler::~Profiler() {
  for (cudaEvent_t e : pool) cudaEventDestroy(e);
}

ProfToken prof_begin(cudaStream_t st) {
  ProfToken t;
  Profiler* p = t_prof;
  if (!p || !p->enabled) return t;
  if ((int)p->recs.size() >= 8192) p->flush();
  t.slot = p->event();
  ZCSD_CUDA(cudaEventRecord(p->pool[t.slot], st));
  return t;
}

void prof_end(ProfToken t, cudaStream_t st, int kind, double flops, int site) {
  Profiler* p = t_prof;
  if (!p || !p->enabled || t.slot < 0) return;
  const int b = p->event();
  ZCSD_CUDA(cudaEventRecord(p->pool[b], st));
  p->recs.push_back({t.slot, b, kind, site, flops});
}

}  // namespace zcsd
