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

template <class T>
int polar_noalloc_impl(int n, const T* A, int lda, T* Wo, int ldw, T* Ho, int ldh, cudaStream_t st, void* base) {
  Ctx cx;
  cx.stream = st;
  cx.hs.d = t_hd;
  cx.hs.i = t_hi;
  Arena ar;
  ar.base = static_cast<char*>(base);
  ar.cap = NOALLOC_BYTES;
  const long long nn = (long long)n * n;
  T* X = ar.get<T>(nn);
  T* W = ar.get<T>(nn);
  double* sc = ar.get<double>(64);
  double* scratch = ar.get<double>(304 * 4);
  axpby<T>(st, n, n, 1.0, A, lda, 0, 0.0, X, n, 0, 1);
  count_nonfinite<T>(st, n, n, X, n, sc, scratch);
  fro2<T>(st, n, n, X, n, 0, 0.0, sc + 1, 1, scratch);
  d2h(cx, cx.hs.d, sc, 2 * sizeof(double));
  if (cx.hs.d[0] != 0.0) return CSD_ERR_NONFINITE;
  const double fn = std::sqrt(cx.hs.d[1]);
  const double alpha = (fn > 1.0) ? 1.0 / fn : 1.0;
  if (alpha != 1.0) axpby<T>(st, n, n, alpha, X, n, 0, 0.0, X, n, 0, 1);
  zolo_pd<T>(cx, ar, n, 1, X, W, nullptr);
  axpby<T>(st, n, n, 1.0, W, n, 0, 0.0, Wo, ldw, 0, 1);
  if (Ho) {
    gemm1<T>(st, OP_C, OP_N, n, n, n, from_re<T>(1.0), W, n, A, lda, zero<T>(), X, n);
    symmetrize<T>(st, n, X, n, 0, Ho, ldh, 0, 1);
  }
  ZCSD_CUDA(cudaStreamSynchronize(st));
  return CSD_OK;
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
