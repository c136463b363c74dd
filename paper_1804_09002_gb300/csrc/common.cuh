// Shared device/host definitions of the Zolo-csd CUDA library.
//
// Matrices are column-major with an explicit leading dimension, FP64 real
// (double) or complex (z64 = {re, im}).  All kernels are templated on the
// scalar type T through the small set of helpers below.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <cmath>
#include <cstdio>

namespace zcsd {

struct z64 {
  double x, y;
};

// ---------------------------------------------------------------- scalars
__host__ __device__ inline double re(double a) { return a; }
__host__ __device__ inline double re(z64 a) { return a.x; }
__host__ __device__ inline double im(double) { return 0.0; }
__host__ __device__ inline double im(z64 a) { return a.y; }
__host__ __device__ inline double conj_(double a) { return a; }
__host__ __device__ inline z64 conj_(z64 a) { return {a.x, -a.y}; }
__host__ __device__ inline double abs2(double a) { return a * a; }
__host__ __device__ inline double abs2(z64 a) { return a.x * a.x + a.y * a.y; }
template <class T> __host__ __device__ inline T from_re(double a);
template <> __host__ __device__ inline double from_re<double>(double a) { return a; }
template <> __host__ __device__ inline z64 from_re<z64>(double a) { return {a, 0.0}; }
template <class T> __host__ __device__ inline T zero() { return from_re<T>(0.0); }
__host__ __device__ inline double add(double a, double b) { return a + b; }
__host__ __device__ inline z64 add(z64 a, z64 b) { return {a.x + b.x, a.y + b.y}; }
__host__ __device__ inline double sub(double a, double b) { return a - b; }
__host__ __device__ inline z64 sub(z64 a, z64 b) { return {a.x - b.x, a.y - b.y}; }
__host__ __device__ inline double mul(double a, double b) { return a * b; }
__host__ __device__ inline z64 mul(z64 a, z64 b) {
  return {a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x};
}
__host__ __device__ inline double scal(double s, double a) { return s * a; }
__host__ __device__ inline z64 scal(double s, z64 a) { return {s * a.x, s * a.y}; }
// c + a*b
__host__ __device__ inline double fmac(double a, double b, double c) { return fma(a, b, c); }
__host__ __device__ inline z64 fmac(z64 a, z64 b, z64 c) {
  return {fma(a.x, b.x, fma(-a.y, b.y, c.x)), fma(a.x, b.y, fma(a.y, b.x, c.y))};
}
// conj(a)*b
__host__ __device__ inline double cmul(double a, double b) { return a * b; }
__host__ __device__ inline z64 cmul(z64 a, z64 b) {
  return {a.x * b.x + a.y * b.y, a.x * b.y - a.y * b.x};
}
__host__ __device__ inline double div_(double a, double b) { return a / b; }
__host__ __device__ inline z64 div_(z64 a, z64 b) {
  double d = b.x * b.x + b.y * b.y;
  return {(a.x * b.x + a.y * b.y) / d, (a.y * b.x - a.x * b.y) / d};
}

template <class T> struct dtype_id;
template <> struct dtype_id<double> { static constexpr int value = 0; };
template <> struct dtype_id<z64> { static constexpr int value = 1; };

// ---------------------------------------------------------------- errors
// Library-internal error carrier: a CUDA error is turned into a status code
// at the C-ABI boundary.
struct CudaFail {
  cudaError_t err;
  const char* file;
  int line;
};

#define ZCSD_CUDA(call)                                     \
  do {                                                      \
    cudaError_t e_ = (call);                                \
    if (e_ != cudaSuccess) throw ::zcsd::CudaFail{e_, __FILE__, __LINE__}; \
  } while (0)

// Every kernel launch goes through ZCSD_LAUNCH(), which also counts it.
void count_launch();
#define ZCSD_LAUNCH()                  \
  do {                                 \
    ::zcsd::count_launch();            \
    ZCSD_CUDA(cudaGetLastError());     \
  } while (0)

// Optional per-kind kernel timing (CUDA events on the launch stream), used
// for roofline reports.  prof_begin/prof_end bracket one launch; both are
// no-ops unless a profiler is active on the calling thread.
enum ProfKind { PK_GEMM = 0, PK_QR_PANEL = 1, PK_POTRF = 2, PK_JACOBI = 3, PK_TC = 4, PK_KINDS = 5 };
struct ProfToken {
  int slot = -1;
};
ProfToken prof_begin(cudaStream_t st);
void prof_end(ProfToken t, cudaStream_t st, int kind, double flops, int site = 0);
constexpr int PROF_SITES = 24;

inline int ceil_div(long long a, long long b) { return (int)((a + b - 1) / b); }

}  // namespace zcsd
