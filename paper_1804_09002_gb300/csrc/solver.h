// Shared state of the solver entry points (solver.cu) and their Zolo-pd core.
#pragma once
#include <vector>

#include "linalg.h"
#include "profile.h"
#include "../../include/zolo_csd.h"

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
  int zolo_extra_passes = 1;  // polar(): further passes of the plan when the iterate has not converged
  int zolo_stop_after = 0;    // polar(): > 0 returns the iterate X_k after k iterations (k <= plan steps)
  unsigned test_flags = 0;    // TEST_* below (fault injection on the host; default off)
  long long tc_probe_wait = 0;  // tensor-core kernel: polls of a barrier nothing signals (0 = none)
  int tc_flush_every = 0;       // tensor-core kernel: drains between int64 write-outs (0 = default)
  bool force_tc_err = false;    // the running call needs the tensor-core error flag (csd_gemm)
  int sign_mode = 0;            // 1: canonical column signs of U1, U2, V1 (csd_set_sign_convention)
  double alg2_svd_factor = 1e3;  // SVD polar fallback when ||R~ - R|| / ||R|| > factor n u (< 0: never)
  int eig_leaf = LEAF;           // Zolo-eig blocks of at most this size go to the Jacobi leaf solver
  int mixed_slices = 7;          // BF16 slices of the Cholesky-iteration products (5, 6 or 7)
  unsigned mixed_scope = 0;      // bit 0: the CSD's / polar()'s Zolo-pd, bit 1: Zolo-eig's Zolo-pd
};

// Host-side fault injection for the failure-path tests.
enum TestFlags : unsigned {
  TEST_REJECT_EIG_SPLITS = CSD_TEST_REJECT_EIG_SPLITS,  // Zolo-eig treats every split attempt as rejected
};

struct PolarDiag {
  int chol_fallback = 0;
  int iters = 0;  // Zolo-pd iterations run
};

// A Zolo-eig block that could not be split after every retry; thrown by
// value so the entry point can report the counts.
struct EigFail {
  int splits, retries;
};

const Plan& get_plan(Ctx& cx);
// device -> host copy on the context stream, then wait for it
void d2h(Ctx& cx, void* dst, const void* src, size_t bytes);

// W_p = polar factor of X0_p for p < P (Zolo-pd, Section 5); X0 and W are
// P consecutive n x n matrices (ld n).  Workspace comes from `ar`.
// stop_after > 0 stops after that many iterations (the iterate X_k).
// reduced_slices = 5 or 6 runs the Gram and triangular-solve products of the
// Cholesky-form iterations with that many BF16 slices (tensor-core path).
// sync_free: no device-to-host read (the Cholesky pivot check is skipped:
// a non-positive pivot leaves NaN, which the caller's checks catch), so the
// call can be captured in a CUDA graph.
template <class T>
void zolo_pd(Ctx& cx, Arena& ar, int n, int P, const T* X0, T* W, PolarDiag* pd, int stop_after = 0,
             int reduced_slices = 0, bool sync_free = false);

// Counters of one Zolo-eig call.
struct EigDiag {
  int splits = 0, retries = 0, leaves = 0;
  double offblock = 0.0;
  int status = 0;
};

// Eigendecomposition of the Hermitian n x n matrix Bin (device, ld ldb) by
// spectral divide and conquer (Section 5, eig.cu).  Writes lam (device,
// length n) and V (device, ld n).  If split_at is finite, only eigenpairs
// below it are computed (Section 5.2: split at 1.1 for Algorithm 3); they
// occupy columns [*lo, n) on return.  Eigenvalues in [*lo, n) are sorted
// ascending with V.  Throws EigFail when a block cannot be split.
template <class T>
void heig_impl(Ctx& cx, Arena& ar, int n, const T* Bin, int ldb, double* lam, T* V, double split_at, int* lo_out,
               EigDiag* ed);

// Columns of V (and of U1, U2) scaled by the inverse phase of V's entry of
// largest magnitude (real: made positive), columns 0..ncols-1.
template <class T>
void canonical_signs(cudaStream_t st, int m1, int m2, int n, int ncols, T* V, int ldv, T* U1, int ldu1, T* U2,
                     int ldu2);

// W = U V^* from the one-sided Jacobi SVD A = U Sigma V^* (svd.cu): the
// SVD-based polar factor of Section 5.1's fallback.  A and W n x n.
template <class T>
void svd_polar(Ctx& cx, Arena& ar, int n, const T* A, int lda, T* W, int ldw);

// Leaf tables of the batched one-sided Jacobi eigensolver (device arrays in
// the arena): leaf l is the sz x sz Hermitian block at element offset boff
// of the B buffer (leading dimension ldb); its eigenvalues go to lam[loff ..]
// and its G_l, V_l (leading dimension sz) sit at goff in packed buffers of
// vtot elements.
struct LeafTable {
  const long long* boff = nullptr;
  const int* ldb = nullptr;
  const int* loff = nullptr;
  const int* sz = nullptr;
  const int* pre = nullptr;  // column pairs before leaf l (pre[nl] = total)
  const long long* goff = nullptr;
  const long long* roff = nullptr;  // per-row rotation records of leaf l at roff[l]
  char* rows = nullptr;             // rotation records (rtot of them)
  double* c = nullptr;       // ||B_l||_F (rotation threshold u ||B_l||_F)
  int* rot = nullptr;        // rotations of leaf l in the current sweep
  int* done = nullptr;       // leaf l converged
  int nl = 0, maxsz = 0, maxpad = 0, total_pairs = 0;
  long long vtot = 0, rtot = 0;
  double sweep_flops = 0.0;  // three dot products and two column-pair rotations per pair, all leaves
};
LeafTable leaf_table_build(Ctx& cx, Arena& ar, const std::vector<long long>& boff, const std::vector<int>& ldb,
                           const std::vector<int>& loff, const std::vector<int>& sz);
// fixed_sweeps > 0: that many sweeps with no device-to-host read (leaves
// that stop rotating are skipped), for graph capture; 0: until converged.
template <class T>
void leaf_solve(Ctx& cx, const LeafTable& L, const T* B, double* lam, T* G, T* V, int fixed_sweeps);

// Eigendecomposition of the diagonal blocks (off[l], sz[l]) of B by
// one-sided Jacobi, all leaves batched (svd.cu): eigenvalues to
// lam[off[l] ..], eigenvectors of leaf l to Vl + voff[l] (ld sz[l]).
template <class T>
void jacobi_eig_leaves(Ctx& cx, Arena& ar, const std::vector<int>& off, const std::vector<int>& sz, const T* B,
                       int ldb, double* lam, T* Vl, std::vector<long long>& voff);

// Reverse-mode derivative of the full-rank real CSD from its outputs
// (grad.cu); gradient inputs may be null (zero).
int csd_backward_impl(Ctx& cx, Arena& ar, int n, const double* U1, int ldu1, const double* U2, int ldu2,
                      const double* V, int ldv, const double* theta, const double* gU1, int ldgu1, const double* gU2,
                      int ldgu2, const double* gV, int ldgv, const double* gtheta, double* gA1, int ldga1, double* gA2,
                      int ldga2);

// The polar() entry point on an arena the caller provides (also used by the
// allocation-free entry point).  Returns a CSD_* status.
template <class T>
int polar_impl(Ctx& cx, Arena& ar, int n, const T* A, int lda, T* Wo, int ldw, T* Ho, int ldh, csd_info* info);

}  // namespace zcsd
