// Dense FP64 building blocks: batched/grouped GEMM on the FP64 FMA pipe,
// elementwise kernels and deterministic reductions.
//
// GB300 executes FP64 at about 2 DFMA per clock per SM (the f64 mma.sync path
// is slower still), so these kernels are bound by the DFMA pipe, not by HBM:
// the GEMM keeps a 4x4 register tile per thread fed from shared memory, which
// needs one shared-memory load per two FMAs, and relies on several resident
// CTAs per SM to cover global-load latency.  Grids are sized by the output
// tiles of all problems of a batch together.
#include <type_traits>

#include "ops.h"
#include "tc_gemm.h"

namespace zcsd {

namespace {

constexpr int BK = 16, NT = 256;

// Output tile BM x BN (BM * BN = 4096: 16 outputs per thread as a 4 x 4
// register tile), k-step BK.  BM = 64 (64 x 64 tiles) is the default; BM = 32
// (32 x 128 tiles) serves the m <= 32 products of the compact-WY updates.
template <class T, int OPA, int OPB, int BM>
__global__ void __launch_bounds__(NT, 2) gemm_kernel(GemmArgs<T> g) {
  constexpr int BN = 4096 / BM;
  constexpr int TX = BM / 4, TY = BN / 4;  // thread grid over the tile
  const int z = blockIdx.z;
  const int b = z / g.ksplit, ks = z % g.ksplit;
  const int m0 = blockIdx.x * BM, n0 = blockIdx.y * BN;
  if (g.uplo == 1 && m0 > n0 + BN - 1) return;
  if (g.uplo == 2 && n0 > m0 + BM - 1) return;
  int kb = 0, ke = g.k;
  if (g.ksplit > 1) {
    const int kc = ((g.k + g.ksplit - 1) / g.ksplit + BK - 1) / BK * BK;
    kb = ks * kc;
    ke = min(g.k, kb + kc);
  }
  if (g.kflags & K_FROM_COL) kb = max(kb, n0);
  if (g.kflags & K_FROM_ROW) kb = max(kb, m0);
  if (g.kflags & K_TO_COL) ke = min(ke, n0 + BN);
  if (g.kflags & K_TO_ROW) ke = min(ke, m0 + BM);

  __shared__ T As[BK][BM + 1];
  __shared__ T Bs[BK][BN + 1];
  const int tid = threadIdx.x;
  const int tx = tid % TX, ty = tid / TX;
  T acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = zero<T>();

  for (int js = 0; js < g.nsum; ++js) {
    const T* A = g.A + (b / g.bdivA) * g.sA + js * g.sAj;
    const T* B = g.B + (b / g.bdivB) * g.sB + js * g.sBj;
    const double wj = g.w[js];
    for (int kt = (kb / BK) * BK; kt < ke; kt += BK) {
      // ---- op(A)[m0:m0+BM, kt:kt+BK] -> As[k][i], coalesced along memory
#pragma unroll
      for (int s = 0; s < (BM * BK) / NT; ++s) {
        const int e = tid + NT * s;
        const int i = (OPA == OP_N) ? (e % BM) : (e / BK);
        const int k = (OPA == OP_N) ? (e / BM) : (e % BK);
        const int gi = m0 + i, gk = kt + k;
        T v = zero<T>();
        if (gi < g.m && gk >= kb && gk < ke) {
          if (OPA == OP_N) v = A[gi + (long long)gk * g.lda];
          else {
            v = A[gk + (long long)gi * g.lda];
            if (OPA == OP_C) v = conj_(v);
          }
        }
        As[k][i] = scal(wj, v);
      }
      // ---- op(B)[kt:kt+BK, n0:n0+BN] -> Bs[k][j]
#pragma unroll
      for (int s = 0; s < (BN * BK) / NT; ++s) {
        const int e = tid + NT * s;
        const int k = (OPB == OP_N) ? (e % BK) : (e / BN);
        const int j = (OPB == OP_N) ? (e / BK) : (e % BN);
        const int gj = n0 + j, gk = kt + k;
        T v = zero<T>();
        if (gj < g.n && gk >= kb && gk < ke) {
          if (OPB == OP_N) v = B[gk + (long long)gj * g.ldb];
          else {
            v = B[gj + (long long)gk * g.ldb];
            if (OPB == OP_C) v = conj_(v);
          }
        }
        Bs[k][j] = v;
      }
      __syncthreads();
#pragma unroll
      for (int k = 0; k < BK; ++k) {
        T a[4], bb[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) a[i] = As[k][tx + TX * i];
#pragma unroll
        for (int j = 0; j < 4; ++j) bb[j] = Bs[k][ty + TY * j];
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
          for (int j = 0; j < 4; ++j) acc[i][j] = fmac(a[i], bb[j], acc[i][j]);
      }
      __syncthreads();
    }
  }
  // ---- epilogue
  T* C = g.C + z * g.sC;
  const T* Cin = g.Cin ? g.Cin + (b / g.bdivC) * g.sCin : nullptr;
  const bool use_beta = Cin && ks == 0 && (re(g.beta) != 0.0 || im(g.beta) != 0.0);
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const int gj = n0 + ty + TY * j;
    if (gj >= g.n) continue;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int gi = m0 + tx + TX * i;
      if (gi >= g.m) continue;
      T v = mul(g.alpha, acc[i][j]);
      if (use_beta) v = fmac(g.beta, Cin[gi + (long long)gj * g.ldcin], v);
      C[gi + (long long)gj * g.ldc] = v;
    }
  }
}

template <class T, int OPA, int BM>
void gemm_dispatch_b(const GemmArgs<T>& g, cudaStream_t st) {
  constexpr int BN = 4096 / BM;
  dim3 grid(ceil_div(g.m, BM), ceil_div(g.n, BN), g.batch * g.ksplit);
  switch (g.opB) {
    case OP_N: gemm_kernel<T, OPA, OP_N, BM><<<grid, NT, 0, st>>>(g); break;
    case OP_T: gemm_kernel<T, OPA, OP_T, BM><<<grid, NT, 0, st>>>(g); break;
    default: gemm_kernel<T, OPA, OP_C, BM><<<grid, NT, 0, st>>>(g); break;
  }
}

template <class T, int BM>
void gemm_dispatch(const GemmArgs<T>& g, cudaStream_t st) {
  switch (g.opA) {
    case OP_N: gemm_dispatch_b<T, OP_N, BM>(g, st); break;
    case OP_T: gemm_dispatch_b<T, OP_T, BM>(g, st); break;
    default: gemm_dispatch_b<T, OP_C, BM>(g, st); break;
  }
}

// Multiply-add work the kernel executes for g, counted per output tile over
// the k range it traverses (2 flops per real FMA, 8 per complex FMA).
template <class T>
double gemm_flops(const GemmArgs<T>& g, int BM, int BN) {
  double fma = 0.0;
  const int tm = ceil_div(g.m, BM), tn = ceil_div(g.n, BN);
  for (int bx = 0; bx < tm; ++bx) {
    const int m0 = bx * BM, rows = std::min(BM, g.m - m0);
    for (int by = 0; by < tn; ++by) {
      const int n0 = by * BN, cols = std::min(BN, g.n - n0);
      if (g.uplo == 1 && m0 > n0 + BN - 1) continue;
      if (g.uplo == 2 && n0 > m0 + BM - 1) continue;
      int kb = 0, ke = g.k;
      if (g.kflags & K_FROM_COL) kb = std::max(kb, n0);
      if (g.kflags & K_FROM_ROW) kb = std::max(kb, m0);
      if (g.kflags & K_TO_COL) ke = std::min(ke, n0 + BN);
      if (g.kflags & K_TO_ROW) ke = std::min(ke, m0 + BM);
      if (ke > kb) fma += (double)rows * cols * (ke - kb);
    }
  }
  return fma * g.nsum * g.batch * (sizeof(T) == sizeof(double) ? 2.0 : 8.0);
}

}  // namespace

template <class T>
void gemm(const GemmArgs<T>& g, cudaStream_t st) {
  if (g.m <= 0 || g.n <= 0 || g.batch <= 0) return;
  if constexpr (std::is_same<T, double>::value) {
    if (tc_will_handle(g)) {
      tc_gemm(g, st, *t_tc.ar, t_tc.err);
      return;
    }
  } else {
    if (tc_will_handle_complex(g)) {
      tc_gemm_complex(g, st, *t_tc.ar, t_tc.err);
      return;
    }
  }
  const bool narrow = g.m <= 32;
  ProfToken tok = prof_begin(st);
  if (narrow) gemm_dispatch<T, 32>(g, st);
  else gemm_dispatch<T, 64>(g, st);
  ZCSD_LAUNCH();
  if (tok.slot >= 0) prof_end(tok, st, PK_GEMM, narrow ? gemm_flops(g, 32, 128) : gemm_flops(g, 64, 64), g.site);
}

template <class T>
void gemm1(cudaStream_t st, int opA, int opB, int m, int n, int k, T alpha, const T* A, int lda,
           const T* B, int ldb, T beta, T* C, int ldc, int uplo, int kflags, int site) {
  GemmArgs<T> g;
  g.site = site;
  g.m = m; g.n = n; g.k = k; g.opA = opA; g.opB = opB;
  g.A = A; g.lda = lda; g.B = B; g.ldb = ldb;
  g.Cin = C; g.ldcin = ldc; g.C = C; g.ldc = ldc;
  g.alpha = alpha; g.beta = beta; g.uplo = uplo; g.kflags = kflags;
  gemm(g, st);
}

// ------------------------------------------------------------------ elementwise
namespace {

struct Vec16 {
  double v[MAX_SUM];
};

template <class F>
__global__ void ew2d_kernel(int m, int n, int batch, F f) {
  const long long total = (long long)m * n;
  const int b = blockIdx.y;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(t % m), j = (int)(t / m);
    f(i, j, b);
  }
  (void)batch;
}

template <class F>
void ew2d(cudaStream_t st, int m, int n, int batch, F f) {
  if (m <= 0 || n <= 0 || batch <= 0) return;
  long long total = (long long)m * n;
  int blocks = (int)std::min<long long>((total + 255) / 256, 152 * 8);
  ew2d_kernel<<<dim3(blocks, batch), 256, 0, st>>>(m, n, batch, f);
  ZCSD_LAUNCH();
}

}  // namespace

template <class T>
void axpby(cudaStream_t st, int m, int n, double alpha, const T* X, int ldx, long long sX, double beta, T* Y,
           int ldy, long long sY, int batch) {
  ew2d(st, m, n, batch, [=] __device__(int i, int j, int b) {
    T x = scal(alpha, X[b * sX + i + (long long)j * ldx]);
    T* y = Y + b * sY + i + (long long)j * ldy;
    *y = (beta != 0.0) ? add(x, scal(beta, *y)) : x;
  });
}

template <class T>
void sum_parts(cudaStream_t st, int m, int n, T* X, int ldx, long long sPart, int parts, int batch) {
  if (parts <= 1) return;
  ew2d(st, m, n, batch, [=] __device__(int i, int j, int b) {
    T* x = X + (long long)b * parts * sPart + i + (long long)j * ldx;
    T acc = *x;
    for (int s = 1; s < parts; ++s) acc = add(acc, x[s * sPart]);
    *x = acc;
  });
}

template <class T>
void shift_terms(cudaStream_t st, int n, const T* X, int ldx, long long sXb, const double* shifts, int nterms,
                 T* Y, int ldy, long long sY, int batch) {
  Vec16 s;
  for (int j = 0; j < MAX_SUM; ++j) s.v[j] = j < nterms ? shifts[j] : 0.0;
  // problem index p = b * nterms + jterm
  ew2d(st, n, n, batch * nterms, [=] __device__(int i, int j, int p) {
    const int bb = p / nterms, jt = p % nterms;
    T x = X[bb * sXb + i + (long long)j * ldx];
    if (i == j) x = add(x, from_re<T>(s.v[jt]));
    Y[p * sY + i + (long long)j * ldy] = x;
  });
}

template <class T>
void stack_terms(cudaStream_t st, int n, const T* X, int ldx, long long sXb, const double* sqrtc, int nterms,
                 T* M, int ldm, long long sM, int batch) {
  Vec16 s;
  for (int j = 0; j < MAX_SUM; ++j) s.v[j] = j < nterms ? sqrtc[j] : 0.0;
  ew2d(st, 2 * n, n, batch * nterms, [=] __device__(int i, int j, int p) {
    const int bb = p / nterms, jt = p % nterms;
    T v;
    if (i < n) v = X[bb * sXb + i + (long long)j * ldx];
    else v = (i - n == j) ? from_re<T>(s.v[jt]) : zero<T>();
    M[p * sM + i + (long long)j * ldm] = v;
  });
}

template <class T>
void sum_terms(cudaStream_t st, int n, double mhat, const T* X1, int ldx, long long sXb, const double* a,
               int nterms, const T* Tm, int ldt, long long sT, T* X2, int ldx2, long long sX2b, int batch) {
  Vec16 s;
  for (int j = 0; j < MAX_SUM; ++j) s.v[j] = j < nterms ? a[j] : 0.0;
  ew2d(st, n, n, batch, [=] __device__(int i, int j, int b) {
    T acc = X1[b * sXb + i + (long long)j * ldx];
    for (int t = 0; t < nterms; ++t) {
      const T v = Tm[(long long)(b * nterms + t) * sT + i + (long long)j * ldt];
      acc = add(acc, scal(s.v[t], v));
    }
    X2[b * sX2b + i + (long long)j * ldx2] = scal(mhat, acc);
  });
}

template <class T>
void symmetrize(cudaStream_t st, int n, const T* Y, int ldy, long long sY, T* H, int ldh, long long sH, int batch) {
  // each (i, j) with i <= j handled once, so in-place use is race-free
  ew2d(st, n, n, batch, [=] __device__(int i, int j, int b) {
    if (i > j) return;
    const T a = Y[b * sY + i + (long long)j * ldy];
    const T c = Y[b * sY + j + (long long)i * ldy];
    const T h = scal(0.5, add(a, conj_(c)));
    H[b * sH + i + (long long)j * ldh] = h;
    H[b * sH + j + (long long)i * ldh] = conj_(h);
    if (i == j) H[b * sH + i + (long long)i * ldh] = from_re<T>(re(h));
  });
}

template <class T>
void set_eye(cudaStream_t st, int m, int n, T* E, int lde, long long sE, int batch) {
  ew2d(st, m, n, batch, [=] __device__(int i, int j, int b) {
    E[b * sE + i + (long long)j * lde] = (i == j) ? from_re<T>(1.0) : zero<T>();
  });
}

// ------------------------------------------------------------------ reductions
namespace {

constexpr int RED_BLOCKS = 304;  // 2 per SM; partial sums are combined in fixed order

__device__ inline double block_sum(double v, double* sh) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (lane == 0) sh[w] = v;
  __syncthreads();
  double r = 0.0;
  if (threadIdx.x == 0) {
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) r += sh[i];
  }
  __syncthreads();
  return r;
}

template <class T>
__global__ void fro2_partial(int m, int n, const T* X, int ldx, long long sX, double shift, double* part) {
  __shared__ double sh[32];
  const int b = blockIdx.y;
  const long long total = (long long)m * n;
  double acc = 0.0;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(t % m), j = (int)(t / m);
    T x = X[b * sX + i + (long long)j * ldx];
    if (i == j) x = sub(x, from_re<T>(shift));
    acc += abs2(x);
  }
  const double r = block_sum(acc, sh);
  if (threadIdx.x == 0) part[b * gridDim.x + blockIdx.x] = r;
}

__global__ void finish_sum(const double* part, int nparts, int batch, double* out) {
  __shared__ double sh[32];
  for (int b = 0; b < batch; ++b) {
    double acc = 0.0;
    for (int i = threadIdx.x; i < nparts; i += blockDim.x) acc += part[b * nparts + i];
    const double r = block_sum(acc, sh);
    if (threadIdx.x == 0) out[b] = r;
  }
}

template <class T>
__global__ void nonfinite_partial(int m, int n, const T* X, int ldx, double* part) {
  __shared__ double sh[32];
  const long long total = (long long)m * n;
  double acc = 0.0;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(t % m), j = (int)(t / m);
    const T x = X[i + (long long)j * ldx];
    if (!isfinite(re(x)) || !isfinite(im(x))) acc += 1.0;
  }
  const double r = block_sum(acc, sh);
  if (threadIdx.x == 0) part[blockIdx.x] = r;
}

template <class T>
__global__ void col_dots_kernel(int m, int n, const T* V, int ldv, const T* Y, int ldy, double* d) {
  __shared__ double sh[32];
  const int j = blockIdx.x;
  double acc = 0.0;
  for (int i = threadIdx.x; i < m; i += blockDim.x)
    acc += re(cmul(V[i + (long long)j * ldv], Y[i + (long long)j * ldy]));
  const double r = block_sum(acc, sh);
  if (threadIdx.x == 0) d[j] = r;
}

template <class T>
__global__ void diag_real_kernel(int n, const T* X, int ldx, double* d) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    d[i] = re(X[i + (long long)i * ldx]);
}

// theta = atan2(S, C) clamped to [0, pi/2], the range of the principal
// angles (Section 1); rounding can otherwise leave S or C a few ulps below 0.
__global__ void theta_kernel(int n, const double* C, const double* S, double* th) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    th[i] = fmin(fmax(atan2(S[i], C[i]), 0.0), 1.5707963267948966);
}

// remark (iv): theta solves sin(theta) - cos(theta) = Lambda, i.e.
// sqrt(2) sin(theta - pi/4) = Lambda, theta = pi/4 + asin(Lambda / sqrt(2)),
// with Lambda / sqrt(2) clamped to [-1, 1] and theta to [0, pi/2].
__global__ void theta_lambda_kernel(int n, const double* lam, double* th) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const double x = fmin(fmax(lam[i] * 0.70710678118654752, -1.0), 1.0);
    th[i] = fmin(fmax(0.78539816339744831 + asin(x), 0.0), 1.5707963267948966);
  }
}

// rank of each key among all keys (ties by index): perm[rank] = index.
// NaN keys order after +inf, so the ranks always form a permutation.
__device__ inline double sort_key(double v) { return isnan(v) ? INFINITY : v; }

__global__ void sort_perm_kernel(int n, const double* key, int* perm) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const double v = sort_key(key[i]);
    const bool vnan = isnan(key[i]);
    int rank = 0;
    for (int k = 0; k < n; ++k) {
      const double w = sort_key(key[k]);
      const bool wnan = isnan(key[k]);
      const bool before = (w < v) || (w == v && (wnan == vnan ? k < i : !wnan));
      rank += before;
    }
    perm[rank] = i;
  }
}

template <class T>
__global__ void gather_cols_kernel(int m, int ncols, const T* X, int ldx, const int* perm, T* Y, int ldy) {
  const long long total = (long long)m * ncols;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(t % m), j = (int)(t / m);
    const int pj = perm[j];
    // perm is a permutation of [0, ncols); the guard only keeps a corrupted
    // index from reading outside X
    Y[i + (long long)j * ldy] = (pj >= 0 && pj < ncols) ? X[i + (long long)pj * ldx] : from_re<T>(NAN);
  }
}

__global__ void gather_vec_kernel(int n, const double* x, const int* perm, double* y) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const int p = perm[i];
    y[i] = (p >= 0 && p < n) ? x[p] : NAN;
  }
}

// splitmix64 (Steele, Lea and Flood 2014): a bijective 64-bit mixer used as a
// counter-based generator, stream position = element index.
__device__ inline unsigned long long splitmix64(unsigned long long z) {
  z += 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

__device__ inline double unit_open(unsigned long long r) {  // (0, 1)
  return ((double)(r >> 11) + 0.5) * 0x1p-53;
}

template <class T>
__global__ void randn_kernel(int m, int n, T* X, int ldx, unsigned long long seed) {
  const long long total = (long long)m * n;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(t % m), j = (int)(t / m);
    const unsigned long long base = seed * 0x100000001B3ull + (unsigned long long)t * 2ull;
    const double u1 = unit_open(splitmix64(base)), u2 = unit_open(splitmix64(base + 1));
    const double rad = sqrt(-2.0 * log(u1));
    double s, c;
    sincospi(2.0 * u2, &s, &c);
    T v;
    if constexpr (sizeof(T) == sizeof(double)) v = from_re<T>(rad * c);
    else { z64 z{rad * c * 0.7071067811865476, rad * s * 0.7071067811865476}; v = *reinterpret_cast<T*>(&z); }
    X[i + (long long)j * ldx] = v;
  }
}

}  // namespace

template <class T>
void fro2(cudaStream_t st, int m, int n, const T* X, int ldx, long long sX, double shift, double* out, int batch,
          double* scratch) {
  if (m <= 0 || n <= 0) {
    ZCSD_CUDA(cudaMemsetAsync(out, 0, sizeof(double) * batch, st));
    return;
  }
  fro2_partial<T><<<dim3(RED_BLOCKS, batch), 256, 0, st>>>(m, n, X, ldx, sX, shift, scratch);
  ZCSD_LAUNCH();
  finish_sum<<<1, 256, 0, st>>>(scratch, RED_BLOCKS, batch, out);
  ZCSD_LAUNCH();
}

template <class T>
void count_nonfinite(cudaStream_t st, int m, int n, const T* X, int ldx, double* out, double* scratch) {
  nonfinite_partial<T><<<RED_BLOCKS, 256, 0, st>>>(m, n, X, ldx, scratch);
  ZCSD_LAUNCH();
  finish_sum<<<1, 256, 0, st>>>(scratch, RED_BLOCKS, 1, out);
  ZCSD_LAUNCH();
}

template <class T>
void col_dots(cudaStream_t st, int m, int n, const T* V, int ldv, const T* Y, int ldy, double* d) {
  if (n <= 0) return;
  col_dots_kernel<T><<<n, 256, 0, st>>>(m, n, V, ldv, Y, ldy, d);
  ZCSD_LAUNCH();
}

template <class T>
void diag_real(cudaStream_t st, int n, const T* X, int ldx, double* d) {
  if (n <= 0) return;
  diag_real_kernel<T><<<ceil_div(n, 256), 256, 0, st>>>(n, X, ldx, d);
  ZCSD_LAUNCH();
}

void theta_from_cs(cudaStream_t st, int n, const double* C, const double* S, double* theta) {
  if (n <= 0) return;
  theta_kernel<<<ceil_div(n, 256), 256, 0, st>>>(n, C, S, theta);
  ZCSD_LAUNCH();
}

void theta_from_lambda(cudaStream_t st, int n, const double* lam, double* theta) {
  if (n <= 0) return;
  theta_lambda_kernel<<<ceil_div(n, 256), 256, 0, st>>>(n, lam, theta);
  ZCSD_LAUNCH();
}

void sort_perm(cudaStream_t st, int n, const double* key, int* perm) {
  if (n <= 0) return;
  sort_perm_kernel<<<ceil_div(n, 256), 256, 0, st>>>(n, key, perm);
  ZCSD_LAUNCH();
}

template <class T>
void gather_cols(cudaStream_t st, int m, int ncols, const T* X, int ldx, const int* perm, T* Y, int ldy) {
  if (m <= 0 || ncols <= 0) return;
  long long total = (long long)m * ncols;
  gather_cols_kernel<T><<<(int)std::min<long long>((total + 255) / 256, 152 * 8), 256, 0, st>>>(m, ncols, X, ldx,
                                                                                              perm, Y, ldy);
  ZCSD_LAUNCH();
}

void gather_vec(cudaStream_t st, int n, const double* x, const int* perm, double* y) {
  if (n <= 0) return;
  gather_vec_kernel<<<ceil_div(n, 256), 256, 0, st>>>(n, x, perm, y);
  ZCSD_LAUNCH();
}

template <class T>
void randn(cudaStream_t st, int m, int n, T* X, int ldx, unsigned long long seed) {
  long long total = (long long)m * n;
  if (total <= 0) return;
  randn_kernel<T><<<(int)std::min<long long>((total + 255) / 256, 152 * 8), 256, 0, st>>>(m, n, X, ldx, seed);
  ZCSD_LAUNCH();
}

// ------------------------------------------------------------------ instantiations
#define ZCSD_INST(T)                                                                                             \
  template void gemm<T>(const GemmArgs<T>&, cudaStream_t);                                                      \
  template void gemm1<T>(cudaStream_t, int, int, int, int, int, T, const T*, int, const T*, int, T, T*, int, int, \
                         int, int);                                                                                \
  template void axpby<T>(cudaStream_t, int, int, double, const T*, int, long long, double, T*, int, long long, int); \
  template void sum_parts<T>(cudaStream_t, int, int, T*, int, long long, int, int);                                  \
  template void shift_terms<T>(cudaStream_t, int, const T*, int, long long, const double*, int, T*, int, long long, \
                               int);                                                                            \
  template void stack_terms<T>(cudaStream_t, int, const T*, int, long long, const double*, int, T*, int, long long, \
                               int);                                                                            \
  template void sum_terms<T>(cudaStream_t, int, double, const T*, int, long long, const double*, int, const T*, int, \
                             long long, T*, int, long long, int);                                               \
  template void symmetrize<T>(cudaStream_t, int, const T*, int, long long, T*, int, long long, int);            \
  template void set_eye<T>(cudaStream_t, int, int, T*, int, long long, int);                                    \
  template void fro2<T>(cudaStream_t, int, int, const T*, int, long long, double, double*, int, double*);       \
  template void count_nonfinite<T>(cudaStream_t, int, int, const T*, int, double*, double*);                    \
  template void col_dots<T>(cudaStream_t, int, int, const T*, int, const T*, int, double*);                     \
  template void diag_real<T>(cudaStream_t, int, const T*, int, double*);                                        \
  template void gather_cols<T>(cudaStream_t, int, int, const T*, int, const int*, T*, int);                     \
  template void randn<T>(cudaStream_t, int, int, T*, int, unsigned long long);

ZCSD_INST(double)
ZCSD_INST(z64)

}  // namespace zcsd
