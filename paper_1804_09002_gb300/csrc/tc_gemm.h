// FP64-accurate GEMM on the tcgen05 tensor cores by error-free BF16 slicing
// (tc_gemm.cu).  Real FP64 only; op(A), op(B) in {N, T}.
#pragma once
#include "linalg.h"

namespace zcsd {

bool tc_gemm_supported(const GemmArgs<double>& g);

// Per-call tensor-core state of the running entry point (thread-local): when
// `enabled`, gemm<double>() sends eligible products to tc_gemm() using this
// arena and error flag.
struct TcState {
  bool enabled = false;
  unsigned sites = 0;  // bit s: GEMM call site s (GemmSite) may run on the tensor cores
  Arena* ar = nullptr;
  int* err = nullptr;
  long long probe_wait = 0;  // > 0: each launch first polls a barrier nothing signals (timeout-path tests)
  int flush_every = 0;       // > 0: drains between write-outs of the int64 sum (flush-path tests)
  unsigned reduced_sites = 0;  // bit s: call site s uses reduced_slices BF16 slices instead of 7
  int reduced_slices = 7;      // 5 (40 bits) or 6 (48 bits)
};
extern thread_local TcState t_tc;
// true when gemm<double>(g) will run on the tensor cores
bool tc_will_handle(const GemmArgs<double>& g);
// split-K factor (<= cap) for a product the tensor cores take
int tc_pick_ksplit(const GemmArgs<double>& g, int cap);
// C = alpha sum_j w_j op(A_j) op(B_j) + beta Cin, as gemm(); workspace for the
// slices comes from `ar`; *err is set to 1 if a tensor-core wait timed out.
void tc_gemm(const GemmArgs<double>& g, cudaStream_t st, Arena& ar, int* err);

// Complex FP64 products with real alpha and beta as two real grouped sums
// over the interleaved real and imaginary parts (element stride 2):
// Re C = Re A Re B - Im A Im B, Im C = Re A Im B + Im A Re B (signs of the
// conjugate transposes folded into the term weights).
bool tc_will_handle_complex(const GemmArgs<z64>& g);
void tc_gemm_complex(const GemmArgs<z64>& g, cudaStream_t st, Arena& ar, int* err);

}  // namespace zcsd
