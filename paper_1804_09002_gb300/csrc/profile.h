// Per-context kernel timing used by csd_profile_* (see profile.cu).
#pragma once
#include <vector>

#include "common.cuh"

namespace zcsd {

struct Profiler {
  bool enabled = false;
  struct Rec {
    int a, b, kind, site;
    double flops;
  };
  std::vector<cudaEvent_t> pool;
  std::vector<Rec> recs;
  int used = 0;
  double ms[PK_KINDS] = {};
  double flops[PK_KINDS] = {};
  long long count[PK_KINDS] = {};
  double site_ms[PROF_SITES] = {};
  double site_flops[PROF_SITES] = {};
  long long site_count[PROF_SITES] = {};
  int event();
  void flush();
  void reset();
  ~Profiler();
};

// Profiler of the context whose entry point is running on this thread.
extern thread_local Profiler* t_prof;
long long launch_count();

}  // namespace zcsd
