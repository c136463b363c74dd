// Shared state of the solver entry points (solver.cu) and their Zolo-pd core.
#pragma once
#include "linalg.h"
#include "profile.h"

namespace zcsd {

constexpr double U_ROUND = 0x1p-53;
constexpr double EPS_ZOLO = 1e-15;  // interval [eps, 1] of the modified Zolo-pd (Section 5.1)
constexpr int R_MAX = 8;            // p <= 8 (Section 5)

// Zolo-pd iteration plan (coefficients of every iteration) and the per-call
// context: device, stream, workspace, pinned host scalars, profiler.
struct Plan {
  int steps = 0;
  int r[4];
  double ell[4];
  double c[4][2 * R_MAX], a[4][R_MAX], mhat[4], sqrtc[4][R_MAX], w[4][R_MAX];
};

struct Ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  char* ws = nullptr;
  size_t ws_bytes = 0;
  HostScalars hs;
  Plan plan;
  bool plan_ready = false;
  unsigned long long seed = 0x5EEDull;
  Profiler prof;
  bool tensor_cores = false;
  unsigned tc_sites = 0;
  int theta_mode = 0;  // 0: atan2(S, C) (remark (iii)); 1: from Lambda (remark (iv))
};

struct PolarDiag {
  int chol_fallback = 0;
};

const Plan& get_plan(Ctx& cx);
// device -> host copy on the context stream, then wait for it
void d2h(Ctx& cx, void* dst, const void* src, size_t bytes);

// W_p = polar factor of X0_p for p < P (Zolo-pd, Section 5); X0 and W are
// P consecutive n x n matrices (ld n).  Workspace comes from `ar`.
template <class T>
void zolo_pd(Ctx& cx, Arena& ar, int n, int P, const T* X0, T* W, PolarDiag* pd);

}  // namespace zcsd
