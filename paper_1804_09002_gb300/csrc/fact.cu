// Factorization kernels: Householder QR panel (with the compact-WY T factor),
// Cholesky of a diagonal block with its triangular inverse, and the cyclic
// Jacobi eigensolver for the small leaf blocks of Zolo-eig.
//
// The panel and diagonal-block kernels run one CTA per problem of a batch;
// everything with O(n^3) work around them is a GEMM (blas.cu).
#include <algorithm>

#include <cooperative_groups.h>

#include "ops.h"

namespace zcsd {

namespace {

constexpr int PANEL_THREADS = 512;
constexpr int PANEL_MAXNB = 32;

// Sum the PANEL_MAXNB per-thread values across the CTA; the total of value c
// lands in red[nwarps * PANEL_MAXNB + c] for c < cnt.  Inside a warp this is a
// butterfly reduce-scatter: at each of the 5 xor-shuffle steps a lane keeps
// half of its remaining values and adds the partner's copy of that half
// (31 shuffles per component instead of 5 per value), after which lane l
// holds the warp total of value l.
__device__ inline void warp_reduce_scatter32(double (&v)[PANEL_MAXNB]) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int o = 16, cnt = 32; o > 0; o >>= 1, cnt >>= 1) {
    const bool up = (lane & o) != 0;
#pragma unroll
    for (int t = 0; t < 16; ++t) {
      if (t < cnt / 2) {
        const double send = up ? v[t] : v[t + cnt / 2];
        const double keep = up ? v[t + cnt / 2] : v[t];
        v[t] = keep + __shfl_xor_sync(0xffffffffu, send, o);
      }
    }
  }
}

template <class T>
__device__ void block_reduce_vec(T (&vals)[PANEL_MAXNB], int cnt, T* red /* [nwarps+1][PANEL_MAXNB] */) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  double x[PANEL_MAXNB];
#pragma unroll
  for (int c = 0; c < PANEL_MAXNB; ++c) x[c] = re(vals[c]);
  warp_reduce_scatter32(x);
  if constexpr (sizeof(T) == sizeof(double)) {
    red[w * PANEL_MAXNB + lane] = from_re<T>(x[0]);
  } else {
    double y[PANEL_MAXNB];
#pragma unroll
    for (int c = 0; c < PANEL_MAXNB; ++c) y[c] = im(vals[c]);
    warp_reduce_scatter32(y);
    z64 z{x[0], y[0]};
    red[w * PANEL_MAXNB + lane] = *reinterpret_cast<T*>(&z);
  }
  __syncthreads();
  if ((int)threadIdx.x < cnt) {
    T s = zero<T>();
    for (int i = 0; i < nw; ++i) s = add(s, red[i * PANEL_MAXNB + threadIdx.x]);
    red[(nw)*PANEL_MAXNB + threadIdx.x] = s;
  }
  __syncthreads();
}

template <class T>
__device__ inline T make_c(double x, double y) {
  if constexpr (sizeof(T) == sizeof(double)) return from_re<T>(x);
  else { z64 z{x, y}; return *reinterpret_cast<T*>(&z); }
}

// Householder QR of columns [k0, k0+nb) of M (LAPACK geqr2 + larft semantics):
// H_k = I - tau_k v_k v_k^*, beta real, A = Q R with Q = H_k0 ... H_k0+nb-1,
// and Q = I - V T V^* with T upper triangular.
template <class T>
__global__ void __launch_bounds__(PANEL_THREADS) qr_panel_kernel(int m, int n, int band, T* Mall, int ldm,
                                                                 long long sM, int k0, int nb, T* Yall, int ldy,
                                                                 long long sY, T* Tall, long long sT) {
  __shared__ T red[(PANEL_THREADS / 32 + 1) * PANEL_MAXNB];
  __shared__ T wv[PANEL_MAXNB];
  __shared__ T Ts[PANEL_MAXNB * PANEL_MAXNB];
  __shared__ T sh_scale, sh_tau, sh_beta;
  const int b = blockIdx.x;
  T* M = Mall + b * sM;
  T* Y = Yall + b * sY;
  T* Tf = Tall + b * sT;
  const int tid = threadIdx.x, nt = blockDim.x;
  const int hrows = min(m, k0 + nb - 1 + band) - k0;  // rows of the Y panel
  for (int i = tid; i < PANEL_MAXNB * PANEL_MAXNB; i += nt) Ts[i] = zero<T>();
  __syncthreads();

  for (int j = 0; j < nb; ++j) {
    const int k = k0 + j;
    const int rend = min(m, k + band);
    // ---- pass 1: d_c = sum_{i>k} conj(M[i,k]) M[i,k0+c] for every panel column c
    T d[PANEL_MAXNB];
#pragma unroll
    for (int c = 0; c < PANEL_MAXNB; ++c) d[c] = zero<T>();
    for (int i = k + 1 + tid; i < rend; i += nt) {
      const T x = M[i + (long long)k * ldm];
#pragma unroll
      for (int c = 0; c < PANEL_MAXNB; ++c)
        if (c < nb) d[c] = add(d[c], cmul(x, M[i + (long long)(k0 + c) * ldm]));
    }
    block_reduce_vec(d, nb, red);
    const T* dsum = red + (nt / 32) * PANEL_MAXNB;
    // ---- reflector (LAPACK larfg) and the dot products it needs
    if (tid == 0) {
      const T alpha = M[k + (long long)k * ldm];
      const double xnorm2 = re(dsum[j]);
      T tau, scale, beta;
      if (xnorm2 == 0.0 && im(alpha) == 0.0) {
        tau = zero<T>();
        scale = zero<T>();
        beta = alpha;
      } else {
        const double nrm = sqrt(abs2(alpha) + xnorm2);
        const double bt = re(alpha) >= 0.0 ? -nrm : nrm;
        beta = from_re<T>(bt);
        tau = make_c<T>((bt - re(alpha)) / bt, -im(alpha) / bt);
        scale = div_(from_re<T>(1.0), sub(alpha, beta));
      }
      sh_tau = tau;
      sh_scale = scale;
      sh_beta = beta;
    }
    __syncthreads();
    const T tau = sh_tau, scale = sh_scale;
    if (tid < nb) {
      const int c = tid;
      const T mk = M[k + (long long)(k0 + c) * ldm];
      if (c > j) {
        // w_c = v^* M[:, c] = M[k, c] + conj(scale) d_c
        wv[c] = add(mk, mul(conj_(scale), dsum[c]));
      } else if (c < j) {
        // y_c = V[:, c]^* v = conj(M[k, c]) + scale conj(d_c)
        wv[c] = add(conj_(mk), mul(scale, conj_(dsum[c])));
      }
    }
    __syncthreads();
    // T[0:j, j] = -tau T[0:j, 0:j] y[0:j];  T[j, j] = tau
    if (tid < j) {
      const int r = tid;
      T s = zero<T>();
      for (int c = r; c < j; ++c) s = fmac(Ts[r + c * PANEL_MAXNB], wv[c], s);
      red[r] = mul(from_re<T>(-1.0), mul(tau, s));  // scratch (red no longer needed)
    }
    __syncthreads();
    if (tid < j) Ts[tid + j * PANEL_MAXNB] = red[tid];
    if (tid == 0) Ts[j + j * PANEL_MAXNB] = tau;
    // ---- pass 2: v, Y and the update of the remaining panel columns
    const T ctau = conj_(tau);
    for (int i = k + tid; i < rend; i += nt) {
      T v;
      if (i == k) v = from_re<T>(1.0);
      else {
        v = mul(scale, M[i + (long long)k * ldm]);
        M[i + (long long)k * ldm] = v;
      }
      Y[(i - k0) + (long long)j * ldy] = v;
      const T cv = mul(ctau, v);
      for (int c = j + 1; c < nb; ++c) {
        T* p = M + i + (long long)(k0 + c) * ldm;
        *p = sub(*p, mul(cv, wv[c]));
      }
    }
    // zeros of the explicit V panel outside [k, rend)
    for (int i = tid; i < hrows; i += nt) {
      const int gi = k0 + i;
      if (gi < k || gi >= rend) Y[i + (long long)j * ldy] = zero<T>();
    }
    __syncthreads();
    if (tid == 0) M[k + (long long)k * ldm] = sh_beta;
    __syncthreads();
  }
  for (int i = tid; i < nb * nb; i += nt) {
    const int r = i % nb, c = i / nb;
    Tf[r + c * nb] = Ts[r + c * PANEL_MAXNB];
  }
}

// Cluster version of the panel: the CL CTAs of a thread-block cluster split
// the panel rows; per column each CTA reduces its partial dot products, the
// partials are exchanged through distributed shared memory after one cluster
// barrier, and every CTA derives the same reflector (fixed summation order).
// Double-buffered exchange slots make one barrier per column sufficient: a
// slot is rewritten two columns later, after every CTA has passed the
// barrier that follows its last read of it.
constexpr int PANEL_CL = 8;
constexpr int PANEL_CL_THREADS = 256;

template <class T>
__global__ void __launch_bounds__(PANEL_CL_THREADS) qr_panel_cluster_kernel(int m, int n, int band, T* Mall, int ldm,
                                                                            long long sM, int k0, int nb, T* Yall,
                                                                            int ldy, long long sY, T* Tall,
                                                                            long long sT) {
  namespace cg = cooperative_groups;
  cg::cluster_group cluster = cg::this_cluster();
  __shared__ T red[(PANEL_CL_THREADS / 32 + 1) * PANEL_MAXNB];
  __shared__ T part[2][2 * PANEL_MAXNB];  // [slot][partial dots | pivot row]
  __shared__ T dtot[PANEL_MAXNB], prow[PANEL_MAXNB];
  __shared__ T wv[PANEL_MAXNB];
  __shared__ T Ts[PANEL_MAXNB * PANEL_MAXNB];
  __shared__ T sh_scale, sh_tau, sh_beta;
  const int rank = (int)cluster.block_rank();
  const int b = blockIdx.x / PANEL_CL;
  T* M = Mall + b * sM;
  T* Y = Yall + b * sY;
  T* Tf = Tall + b * sT;
  const int tid = threadIdx.x, nt = blockDim.x;
  const int hrows = min(m, k0 + nb - 1 + band) - k0;
  const int chunk = (hrows + PANEL_CL - 1) / PANEL_CL;
  const int rlo = k0 + rank * chunk, rhi = k0 + min(hrows, (rank + 1) * chunk);
  for (int i = tid; i < PANEL_MAXNB * PANEL_MAXNB; i += nt) Ts[i] = zero<T>();
  __syncthreads();

  for (int j = 0; j < nb; ++j) {
    const int k = k0 + j;
    const int rend = min(m, k + band);
    const int slot = j & 1;
    // ---- pass 1 over this CTA's rows: d_c = sum_{i>k} conj(M[i,k]) M[i,k0+c]
    T d[PANEL_MAXNB];
#pragma unroll
    for (int c = 0; c < PANEL_MAXNB; ++c) d[c] = zero<T>();
    const int i0 = max(k + 1, rlo), i1 = min(rend, rhi);
    for (int i = i0 + tid; i < i1; i += nt) {
      const T x = M[i + (long long)k * ldm];
#pragma unroll
      for (int c = 0; c < PANEL_MAXNB; ++c)
        if (c < nb) d[c] = add(d[c], cmul(x, M[i + (long long)(k0 + c) * ldm]));
    }
    block_reduce_vec(d, nb, red);
    const T* dloc = red + (nt / 32) * PANEL_MAXNB;
    const bool owner = (k >= rlo && k < rhi);
    if (tid < nb) {
      part[slot][tid] = dloc[tid];
      part[slot][PANEL_MAXNB + tid] = owner ? M[k + (long long)(k0 + tid) * ldm] : zero<T>();
    }
    cluster.sync();
    // ---- combine the partials of all CTAs (same order everywhere)
    if (tid < nb) {
      T sum = zero<T>(), pr = zero<T>();
      for (int r = 0; r < PANEL_CL; ++r) {
        const T* rp = cluster.map_shared_rank(&part[slot][0], r);
        sum = add(sum, rp[tid]);
        pr = add(pr, rp[PANEL_MAXNB + tid]);  // only the owner's entry is nonzero
      }
      dtot[tid] = sum;
      prow[tid] = pr;
    }
    __syncthreads();
    if (tid == 0) {
      const T alpha = prow[j];
      const double xnorm2 = re(dtot[j]);
      T tau, scale, beta;
      if (xnorm2 == 0.0 && im(alpha) == 0.0) {
        tau = zero<T>();
        scale = zero<T>();
        beta = alpha;
      } else {
        const double nrm = sqrt(abs2(alpha) + xnorm2);
        const double bt = re(alpha) >= 0.0 ? -nrm : nrm;
        beta = from_re<T>(bt);
        tau = make_c<T>((bt - re(alpha)) / bt, -im(alpha) / bt);
        scale = div_(from_re<T>(1.0), sub(alpha, beta));
      }
      sh_tau = tau;
      sh_scale = scale;
      sh_beta = beta;
    }
    __syncthreads();
    const T tau = sh_tau, scale = sh_scale;
    if (tid < nb) {
      const int c = tid;
      const T mk = prow[c];
      if (c > j) wv[c] = add(mk, mul(conj_(scale), dtot[c]));
      else if (c < j) wv[c] = add(conj_(mk), mul(scale, conj_(dtot[c])));
    }
    __syncthreads();
    if (tid < j) {
      const int r = tid;
      T s = zero<T>();
      for (int c = r; c < j; ++c) s = fmac(Ts[r + c * PANEL_MAXNB], wv[c], s);
      red[r] = mul(from_re<T>(-1.0), mul(tau, s));
    }
    __syncthreads();
    if (tid < j) Ts[tid + j * PANEL_MAXNB] = red[tid];
    if (tid == 0) Ts[j + j * PANEL_MAXNB] = tau;
    // ---- pass 2 over this CTA's rows
    const T ctau = conj_(tau);
    const int u0 = max(k, rlo);
    for (int i = u0 + tid; i < i1; i += nt) {
      T v;
      if (i == k) v = from_re<T>(1.0);
      else {
        v = mul(scale, M[i + (long long)k * ldm]);
        M[i + (long long)k * ldm] = v;
      }
      Y[(i - k0) + (long long)j * ldy] = v;
      const T cv = mul(ctau, v);
      for (int c = j + 1; c < nb; ++c) {
        T* q = M + i + (long long)(k0 + c) * ldm;
        *q = sub(*q, mul(cv, wv[c]));
      }
    }
    for (int i = rlo + tid; i < rhi; i += nt)
      if (i < k || i >= rend) Y[(i - k0) + (long long)j * ldy] = zero<T>();
    __syncthreads();
    if (tid == 0 && owner) M[k + (long long)k * ldm] = sh_beta;
  }
  if (rank == 0)
    for (int i = tid; i < nb * nb; i += nt) {
      const int r = i % nb, c = i / nb;
      Tf[r + c * nb] = Ts[r + c * PANEL_MAXNB];
    }
  // no CTA may exit while another can still read its shared memory
  cluster.sync();
}

// Shared-memory-resident cluster panel: as qr_panel_cluster_kernel, but each
// CTA first copies its block of panel rows (all nb columns) into shared
// memory, runs every column there, and writes R/V and the explicit V panel
// back once.  Per column only the cluster exchange touches anything but
// shared memory.  S holds column c of the CTA's rows at S[c * lds + (i - rlo)].
template <class T, int CL>
__global__ void __launch_bounds__(PANEL_CL_THREADS) qr_panel_smem_kernel(int m, int n, int band, T* Mall, int ldm,
                                                                         long long sM, int k0, int nb, T* Yall,
                                                                         int ldy, long long sY, T* Tall, long long sT,
                                                                         int chunk) {
  namespace cg = cooperative_groups;
  cg::cluster_group cluster = cg::this_cluster();
  extern __shared__ __align__(16) unsigned char dyn_smem[];
  T* S = reinterpret_cast<T*>(dyn_smem);
  const int lds = chunk;
  __shared__ T red[(PANEL_CL_THREADS / 32 + 1) * PANEL_MAXNB];
  __shared__ T part[2][2 * PANEL_MAXNB];
  __shared__ T dtot[PANEL_MAXNB], prow[PANEL_MAXNB];
  __shared__ T wv[PANEL_MAXNB];
  __shared__ T Ts[PANEL_MAXNB * PANEL_MAXNB];
  __shared__ T sh_scale, sh_tau, sh_beta;
  const int rank = (int)cluster.block_rank();
  const int b = blockIdx.x / CL;
  T* M = Mall + b * sM;
  T* Y = Yall + b * sY;
  T* Tf = Tall + b * sT;
  const int tid = threadIdx.x, nt = blockDim.x;
  const int hrows = min(m, k0 + nb - 1 + band) - k0;
  const int rlo = k0 + rank * chunk, rhi = k0 + min(hrows, (rank + 1) * chunk);
  for (int i = tid; i < PANEL_MAXNB * PANEL_MAXNB; i += nt) Ts[i] = zero<T>();
  for (int c = 0; c < nb; ++c)
    for (int i = rlo + tid; i < rhi; i += nt) S[c * lds + (i - rlo)] = M[i + (long long)(k0 + c) * ldm];
  __syncthreads();

  for (int j = 0; j < nb; ++j) {
    const int k = k0 + j;
    const int rend = min(m, k + band);
    const int slot = j & 1;
    T d[PANEL_MAXNB];
#pragma unroll
    for (int c = 0; c < PANEL_MAXNB; ++c) d[c] = zero<T>();
    const int i0 = max(k + 1, rlo), i1 = min(rend, rhi);
    for (int i = i0 + tid; i < i1; i += nt) {
      const T x = S[j * lds + (i - rlo)];
#pragma unroll
      for (int c = 0; c < PANEL_MAXNB; ++c)
        if (c < nb) d[c] = add(d[c], cmul(x, S[c * lds + (i - rlo)]));
    }
    block_reduce_vec(d, nb, red);
    const T* dloc = red + (nt / 32) * PANEL_MAXNB;
    const bool owner = (k >= rlo && k < rhi);
    if (tid < nb) {
      part[slot][tid] = dloc[tid];
      part[slot][PANEL_MAXNB + tid] = owner ? S[tid * lds + (k - rlo)] : zero<T>();
    }
    cluster.sync();
    if (tid < nb) {
      T vals[CL], prs[CL];
#pragma unroll
      for (int r = 0; r < CL; ++r) {  // independent remote loads, summed in rank order
        const T* rp = cluster.map_shared_rank(&part[slot][0], r);
        vals[r] = rp[tid];
        prs[r] = rp[PANEL_MAXNB + tid];
      }
      T sum = zero<T>(), pr = zero<T>();
#pragma unroll
      for (int r = 0; r < CL; ++r) {
        sum = add(sum, vals[r]);
        pr = add(pr, prs[r]);
      }
      dtot[tid] = sum;
      prow[tid] = pr;
    }
    __syncthreads();
    if (tid == 0) {
      const T alpha = prow[j];
      const double xnorm2 = re(dtot[j]);
      T tau, scale, beta;
      if (xnorm2 == 0.0 && im(alpha) == 0.0) {
        tau = zero<T>();
        scale = zero<T>();
        beta = alpha;
      } else {
        const double nrm = sqrt(abs2(alpha) + xnorm2);
        const double bt = re(alpha) >= 0.0 ? -nrm : nrm;
        beta = from_re<T>(bt);
        tau = make_c<T>((bt - re(alpha)) / bt, -im(alpha) / bt);
        scale = div_(from_re<T>(1.0), sub(alpha, beta));
      }
      sh_tau = tau;
      sh_scale = scale;
      sh_beta = beta;
    }
    __syncthreads();
    const T tau = sh_tau, scale = sh_scale;
    if (tid < nb) {
      const int c = tid;
      const T mk = prow[c];
      if (c > j) wv[c] = add(mk, mul(conj_(scale), dtot[c]));
      else if (c < j) wv[c] = add(conj_(mk), mul(scale, conj_(dtot[c])));
    }
    __syncthreads();
    if (tid < j) {
      const int r = tid;
      T sacc = zero<T>();
      for (int c = r; c < j; ++c) sacc = fmac(Ts[r + c * PANEL_MAXNB], wv[c], sacc);
      red[r] = mul(from_re<T>(-1.0), mul(tau, sacc));
    }
    __syncthreads();
    if (tid < j) Ts[tid + j * PANEL_MAXNB] = red[tid];
    if (tid == 0) Ts[j + j * PANEL_MAXNB] = tau;
    const T ctau = conj_(tau);
    const int u0 = max(k, rlo);
    for (int i = u0 + tid; i < i1; i += nt) {
      T v;
      if (i == k) v = from_re<T>(1.0);
      else {
        v = mul(scale, S[j * lds + (i - rlo)]);
        S[j * lds + (i - rlo)] = v;
      }
      const T cv = mul(ctau, v);
      for (int c = j + 1; c < nb; ++c) {
        T* q = S + c * lds + (i - rlo);
        *q = sub(*q, mul(cv, wv[c]));
      }
    }
    __syncthreads();
    if (tid == 0 && owner) S[j * lds + (k - rlo)] = sh_beta;
    __syncthreads();
  }
  // write back R / V and the explicit unit-lower V panel
  for (int c = 0; c < nb; ++c) {
    const int kc = k0 + c, rendc = min(m, kc + band);
    for (int i = rlo + tid; i < rhi; i += nt) {
      const T x = S[c * lds + (i - rlo)];
      M[i + (long long)kc * ldm] = x;
      T yv;
      if (i < kc || i >= rendc) yv = zero<T>();
      else if (i == kc) yv = from_re<T>(1.0);
      else yv = x;
      Y[(i - k0) + (long long)c * ldy] = yv;
    }
  }
  if (rank == 0)
    for (int i = tid; i < nb * nb; i += nt) {
      const int r = i % nb, c = i / nb;
      Tf[r + c * nb] = Ts[r + c * PANEL_MAXNB];
    }
  cluster.sync();
}

constexpr int PANEL_SMEM_MAX = 200 * 1024;

template <class T, int CL>
void launch_panel_smem(cudaStream_t st, int m, int n, int band, T* M, int ldm, long long sM, int k0, int nb, T* Y,
                       int ldy, long long sY, T* Tf, long long sT, int batch, int chunk) {
  const int smem = PANEL_MAXNB * chunk * (int)sizeof(T);
  // the attribute is set once per kernel (to the largest dynamic shared
  // memory its launches use, PANEL_SMEM_MAX), not per launch: launches may
  // be graph-captured
  static const bool attr_set = [] {
    ZCSD_CUDA(cudaFuncSetAttribute(qr_panel_smem_kernel<T, CL>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   PANEL_SMEM_MAX));
    return true;
  }();
  (void)attr_set;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(batch * CL, 1, 1);
  cfg.blockDim = dim3(PANEL_CL_THREADS, 1, 1);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = CL;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  ZCSD_CUDA(cudaLaunchKernelEx(&cfg, qr_panel_smem_kernel<T, CL>, m, n, band, M, ldm, sM, k0, nb, Y, ldy, sY, Tf, sT,
                               chunk));
}

constexpr int CHOL_MAXNB = 64;

template <class T>
__global__ void __launch_bounds__(256) potrf_inv_kernel(int n, T* Aall, int lda, long long sA, int k0, int nb,
                                                        T* Rall, int ldr, long long sR, int* info) {
  extern __shared__ __align__(16) unsigned char dyn_smem[];
  T(*S)[CHOL_MAXNB + 1] = reinterpret_cast<T(*)[CHOL_MAXNB + 1]>(dyn_smem);
  T(*X)[CHOL_MAXNB + 1] = S + CHOL_MAXNB;
  __shared__ int bad;
  const int b = blockIdx.x;
  T* A = Aall + b * sA;
  T* Rinv = Rall + b * sR;
  const int tid = threadIdx.x;
  if (tid == 0) bad = 0;
  for (int t = tid; t < nb * nb; t += blockDim.x) {
    const int i = t % nb, j = t / nb;
    S[i][j] = (i <= j) ? A[(k0 + i) + (long long)(k0 + j) * lda] : zero<T>();
    X[i][j] = zero<T>();
  }
  __syncthreads();
  // upper Cholesky, row by row: R[j, j:] from S[j, j:] - sum_{p<j} conj(R[p, j]) R[p, j:]
  for (int j = 0; j < nb; ++j) {
    if (tid == 0) {
      double dd = re(S[j][j]);
      for (int p = 0; p < j; ++p) dd -= abs2(S[p][j]);
      if (!(dd > 0.0) || !isfinite(dd)) {
        if (!bad) bad = k0 + j + 1;
        dd = 1.0;
      }
      S[j][j] = from_re<T>(sqrt(dd));
    }
    __syncthreads();
    const double rjj = re(S[j][j]);
    for (int c = j + 1 + tid; c < nb; c += blockDim.x) {
      T s = S[j][c];
      for (int p = 0; p < j; ++p) s = sub(s, cmul(S[p][j], S[p][c]));
      S[j][c] = scal(1.0 / rjj, s);
    }
    __syncthreads();
  }
  // R^{-1}: column c by back substitution (one thread per column)
  for (int c = tid; c < nb; c += blockDim.x) {
    X[c][c] = from_re<T>(1.0 / re(S[c][c]));
    for (int i = c - 1; i >= 0; --i) {
      T s = zero<T>();
      for (int p = i + 1; p <= c; ++p) s = fmac(S[i][p], X[p][c], s);
      X[i][c] = scal(-1.0 / re(S[i][i]), s);
    }
  }
  __syncthreads();
  for (int t = tid; t < nb * nb; t += blockDim.x) {
    const int i = t % nb, j = t / nb;
    if (i <= j) A[(k0 + i) + (long long)(k0 + j) * lda] = S[i][j];
    Rinv[i + (long long)j * ldr] = (i <= j) ? X[i][j] : zero<T>();
  }
  if (tid == 0 && bad && info[b] == 0) info[b] = bad;
}

}  // namespace

template <class T>
void qr_panel(cudaStream_t st, int m, int n, int band, T* M, int ldm, long long sM, int k0, int nb, T* Y, int ldy,
              long long sY, T* Tf, long long sT, int batch) {
  if (nb > PANEL_MAXNB) throw CudaFail{cudaErrorInvalidValue, __FILE__, __LINE__};
  ProfToken tok = prof_begin(st);
  const int hrows = std::min(m, k0 + nb - 1 + band) - k0;
  const int chunk8 = (hrows + 7) / 8, chunk4 = (hrows + 3) / 4;
  if (hrows >= 1024 && PANEL_MAXNB * chunk8 * (int)sizeof(T) <= PANEL_SMEM_MAX) {
    launch_panel_smem<T, 8>(st, m, n, band, M, ldm, sM, k0, nb, Y, ldy, sY, Tf, sT, batch, chunk8);
  } else if (hrows >= 256 && hrows < 1024) {
    launch_panel_smem<T, 4>(st, m, n, band, M, ldm, sM, k0, nb, Y, ldy, sY, Tf, sT, batch, chunk4);
  } else if (hrows >= 1024) {
    // tall panel: a cluster of PANEL_CL CTAs per problem
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(batch * PANEL_CL, 1, 1);
    cfg.blockDim = dim3(PANEL_CL_THREADS, 1, 1);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = PANEL_CL;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    ZCSD_CUDA(cudaLaunchKernelEx(&cfg, qr_panel_cluster_kernel<T>, m, n, band, M, ldm, sM, k0, nb, Y, ldy, sY, Tf,
                                 sT));
  } else {
    qr_panel_kernel<T><<<batch, PANEL_THREADS, 0, st>>>(m, n, band, M, ldm, sM, k0, nb, Y, ldy, sY, Tf, sT);
  }
  ZCSD_LAUNCH();
  if (tok.slot >= 0) {
    // Householder panel: about 4 h nb^2 real flops (dots + rank-1 updates)
    const double h = std::min(m, k0 + nb - 1 + band) - k0;
    prof_end(tok, st, PK_QR_PANEL, 4.0 * h * nb * nb * batch * (sizeof(T) == sizeof(double) ? 1.0 : 4.0));
  }
}

template <class T>
void potrf_inv(cudaStream_t st, int n, T* A, int lda, long long sA, int k0, int nb, T* Rinv, int ldr,
               long long sR, int* info, int batch) {
  if (nb > CHOL_MAXNB) throw CudaFail{cudaErrorInvalidValue, __FILE__, __LINE__};
  const int smem = 2 * CHOL_MAXNB * (CHOL_MAXNB + 1) * (int)sizeof(T);
  static const bool attr_set = [smem] {
    ZCSD_CUDA(cudaFuncSetAttribute(potrf_inv_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    return true;
  }();
  (void)attr_set;
  ProfToken tok = prof_begin(st);
  potrf_inv_kernel<T><<<batch, 256, smem, st>>>(n, A, lda, sA, k0, nb, Rinv, ldr, sR, info);
  ZCSD_LAUNCH();
  if (tok.slot >= 0) prof_end(tok, st, PK_POTRF, (2.0 / 3.0) * nb * nb * nb * batch);
}

#define ZCSD_INST_F(T)                                                                                        \
  template void qr_panel<T>(cudaStream_t, int, int, int, T*, int, long long, int, int, T*, int, long long, T*, \
                            long long, int);                                                                 \
  template void potrf_inv<T>(cudaStream_t, int, T*, int, long long, int, int, T*, int, long long, int*, int);

ZCSD_INST_F(double)
ZCSD_INST_F(z64)

}  // namespace zcsd
