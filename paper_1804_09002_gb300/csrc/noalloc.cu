// polar_noalloc: the Zolo-pd polar decomposition for small matrices with all
// of its scratch memory in one static device array, for callers that cannot
// allocate device memory (see include/zolo_csd.h).
//
// The scratch below is a file-scope __device__ array.  Host code must not use
// its name as a device address: on the host the symbol is only a stand-in, and
// handing it to a kernel would fault (or, where the GPU can reach host memory,
// silently use the wrong memory).  The real device address is fetched once per
// device with cudaGetSymbolAddress, with that device current, and cached.
#include <mutex>

#include "../../include/zolo_csd.h"
#include "solver.h"
#include "tc_gemm.h"

namespace zcsd {

// Workspace of one Zolo-pd call (P = 1) for n <= CSD_NOALLOC_MAX_N, complex
// FP64 (the larger element type), plus the input/output staging of polar():
// about 4 MiB at n = 64 (panels of at most 96 rows take no split-K
// partial products); 6 MiB leaves headroom.
constexpr size_t NOALLOC_BYTES = (size_t)6 << 20;

static __device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_BYTES];

namespace {

constexpr int MAX_DEVICES = 64;
std::mutex g_setup_mu;
void* g_scratch_ptr[MAX_DEVICES] = {};

// Device address of g_noalloc_scratch on the current device (set-up on the
// first call per device).  Returns nullptr on failure.
void* scratch_for_current_device(int dev) {
  std::lock_guard<std::mutex> lk(g_setup_mu);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || p == nullptr) {
      cudaGetLastError();
      return nullptr;
    }
    g_scratch_ptr[dev] = p;
  }
  return g_scratch_ptr[dev];
}

bool on_device(const void* p) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

// Host-side scalar buffers of this thread (device-to-host reads of one call).
thread_local double t_hd[64];
thread_local int t_hi[4096];

// The call runs polar_impl (the polar() entry point's body) on an arena over
// the static scratch.  The thread's tensor-core dispatch state and profiler
// are switched off for the call and restored afterwards, so a product can
// never draw slices from another call's arena (n <= 64 is also below the
// tensor-core kernel's smallest tile).
template <class T>
int polar_noalloc_impl(int n, const T* A, int lda, T* Wo, int ldw, T* Ho, int ldh, cudaStream_t st, void* base) {
  struct StateScope {
    TcState tc;
    Profiler* prof;
    StateScope() : tc(t_tc), prof(t_prof) {
      t_tc = TcState{};
      t_prof = nullptr;
    }
    ~StateScope() {
      t_tc = tc;
      t_prof = prof;
    }
  } scope;
  Ctx cx;
  cx.stream = st;
  cx.hs.d = t_hd;
  cx.hs.i = t_hi;
  Arena ar;
  ar.base = static_cast<char*>(base);
  ar.cap = NOALLOC_BYTES;
  return polar_impl<T>(cx, ar, n, A, lda, Wo, ldw, Ho, ldh, nullptr);
}

}  // namespace
}  // namespace zcsd

extern "C" int polar_noalloc(int dtype, int n, const void* A, int lda, void* W, int ldw, void* H, int ldh,
                             void* stream) {
  using namespace zcsd;
  if (dtype != CSD_F64 && dtype != CSD_C128) return -1;
  if (n < 1 || n > CSD_NOALLOC_MAX_N) return -2;
  if (!A || !on_device(A)) return -3;
  if (lda < n) return -4;
  if (!W || !on_device(W)) return -5;
  if (ldw < n) return -6;
  if (H && !on_device(H)) return -7;
  if (H && ldh < n) return -8;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= MAX_DEVICES) {
    cudaGetLastError();
    return CSD_ERR_NO_DEVICE;
  }
  void* base = scratch_for_current_device(dev);
  if (!base) return CSD_ERR_CUDA;
  cudaStream_t st = (cudaStream_t)stream;
  try {
    if (dtype == CSD_F64)
      return polar_noalloc_impl<double>(n, (const double*)A, lda, (double*)W, ldw, (double*)H, ldh, st, base);
    return polar_noalloc_impl<z64>(n, (const z64*)A, lda, (z64*)W, ldw, (z64*)H, ldh, st, base);
  } catch (ArenaOverflow&) {
    return CSD_ERR_INTERNAL;  // the static scratch is sized for n <= CSD_NOALLOC_MAX_N
  } catch (CudaFail& f) {
    fprintf(stderr, "zolo_csd: CUDA error %s at %s:%d\n", cudaGetErrorString(f.err), f.file, f.line);
    return CSD_ERR_CUDA;
  }
}
