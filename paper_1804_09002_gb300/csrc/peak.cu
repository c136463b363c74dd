// FP64 peak microbenchmarks: the denominators of the FP64 roofline.  GB300
// runs FP64 on the FMA pipe (DFMA) and, for matrix shapes, on the legacy
// warp-level mma.sync f64 path; tcgen05 has no FP64 kind.  Each kernel keeps
// many independent accumulator chains per thread in flight and writes one
// value per thread, so the compiler keeps every operation.
#include "../../include/zolo_csd.h"
#include "common.cuh"

namespace zcsd {
namespace {

constexpr int PK_CHAINS = 8;

__global__ void __launch_bounds__(256) dfma_loop_kernel(int iters, double a, double b, double* out) {
  double x[PK_CHAINS];
#pragma unroll
  for (int c = 0; c < PK_CHAINS; ++c) x[c] = (double)(threadIdx.x + c) * 1e-3;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int c = 0; c < PK_CHAINS; ++c) x[c] = fma(x[c], a, b);
  }
  double s = 0.0;
#pragma unroll
  for (int c = 0; c < PK_CHAINS; ++c) s += x[c];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

// one m8n8k4 f64 MMA per chain per iteration: 8 x 8 x 4 FMAs per warp
__global__ void __launch_bounds__(256) dmma_loop_kernel(int iters, double a, double b, double* out) {
  double acc[PK_CHAINS][2];
#pragma unroll
  for (int c = 0; c < PK_CHAINS; ++c) { acc[c][0] = 0.0; acc[c][1] = 0.0; }
  const double av = a * (double)(threadIdx.x & 7), bv = b;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int c = 0; c < PK_CHAINS; ++c)
      asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0,%1}, {%2}, {%3}, {%0,%1};\n"
                   : "+d"(acc[c][0]), "+d"(acc[c][1])
                   : "d"(av), "d"(bv));
  }
  double s = 0.0;
#pragma unroll
  for (int c = 0; c < PK_CHAINS; ++c) s += acc[c][0] + acc[c][1];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

}  // namespace
}  // namespace zcsd

extern "C" int csd_fp64_peak(int device, int kind, double* tflops, double* ms_out) {
  using namespace zcsd;
  if (device < 0) return -1;
  if (kind != 0 && kind != 1) return -2;
  if (!tflops) return -3;
  if (cudaSetDevice(device) != cudaSuccess) { cudaGetLastError(); return CSD_ERR_CUDA; }
  int sms = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
  const int blocks = sms * 8, threads = 256;
  double* out = nullptr;
  if (cudaMalloc((void**)&out, sizeof(double) * blocks * threads) != cudaSuccess) {
    cudaGetLastError();
    return CSD_ERR_ALLOC;
  }
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  const int iters = kind == 0 ? 20000 : 4000;
  float best = 1e30f;
  int status = CSD_OK;
  for (int rep = 0; rep < 11 && status == CSD_OK; ++rep) {  // first launch warms up
    cudaEventRecord(e0);
    if (kind == 0) dfma_loop_kernel<<<blocks, threads>>>(iters, 0.999999, 1e-7, out);
    else dmma_loop_kernel<<<blocks, threads>>>(iters, 0.999999, 1e-7, out);
    cudaEventRecord(e1);
    if (cudaEventSynchronize(e1) != cudaSuccess || cudaGetLastError() != cudaSuccess) status = CSD_ERR_CUDA;
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (rep > 0 && ms < best) best = ms;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(out);
  if (status != CSD_OK) return status;
  // DFMA: 2 flops per FMA; DMMA: 8 x 8 x 4 FMAs per warp instruction
  const double fl = kind == 0 ? 2.0 * PK_CHAINS * (double)iters * blocks * threads
                              : 2.0 * 256.0 * PK_CHAINS * (double)iters * blocks * (threads / 32);
  *tflops = fl / (best * 1e-3) / 1e12;
  if (ms_out) *ms_out = best;
  return CSD_OK;
}
