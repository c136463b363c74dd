// Polar decomposition through the SVD, the paper's robust fallback: "In the
// rare event that ||R~_i - R_i|| is unacceptably large ... compute the polar
// decompositions via the SVD, which is unconditionally backward stable"
// (Section 5.1, after Algorithm 2).
//
// The SVD is the one-sided (Hestenes) Jacobi method: G = A is rotated from
// the right by plane rotations J_pq until its columns are mutually
// orthogonal, G = A V, V = prod J_pq; then sigma_j = ||g_j||, u_j = g_j /
// sigma_j and W = U V^*.  Each rotation orthogonalises one column pair
// exactly (Rutishauser's form: zeta = (beta - alpha) / (2 |gamma|),
// t = sign(zeta) / (|zeta| + sqrt(1 + zeta^2)), c = 1 / sqrt(1 + t^2),
// s = c t, with alpha = |g_p|^2, beta = |g_q|^2, gamma = g_p^* g_q; for
// complex data the phase of gamma is moved into column q first).  The
// column pairs of a sweep follow the round-robin (tournament) order: n/2
// disjoint pairs per round, one CTA per pair, n - 1 rounds per sweep; a
// pair is rotated only while |gamma| > tol sqrt(alpha beta), and the sweeps
// stop when a whole sweep rotates nothing.  Columns of G that are exactly
// zero (exactly singular A) get an orthonormal completion by Gram-Schmidt.
#include "solver.h"

namespace zcsd {

namespace {

constexpr int SVD_THREADS = 256;

template <class T>
__device__ __forceinline__ void block_sum3(double& a, double& b, T& c, double* sh) {
  // sh: 4 * SVD_THREADS doubles
  const int t = threadIdx.x;
  sh[t] = a;
  sh[SVD_THREADS + t] = b;
  sh[2 * SVD_THREADS + t] = re(c);
  sh[3 * SVD_THREADS + t] = im(c);
  __syncthreads();
  for (int s = SVD_THREADS / 2; s > 0; s >>= 1) {
    if (t < s)
      for (int q = 0; q < 4; ++q) sh[q * SVD_THREADS + t] += sh[q * SVD_THREADS + t + s];
    __syncthreads();
  }
  a = sh[0];
  b = sh[SVD_THREADS];
  if constexpr (sizeof(T) == sizeof(double)) c = from_re<T>(sh[2 * SVD_THREADS]);
  else c = T{sh[2 * SVD_THREADS], sh[3 * SVD_THREADS]};
}

// One round of the tournament: pair k of round `round` (npad even >= n).
template <class T>
__global__ void __launch_bounds__(SVD_THREADS) jacobi_round_kernel(int m, int n, int npad, int round, T* G, int ldg,
                                                                   T* V, int ldv, double tol, int* rotated) {
  __shared__ double sh[4 * SVD_THREADS];
  const int k = blockIdx.x;
  int p, q;
  if (k == 0) {
    p = npad - 1;
    q = round;
  } else {
    p = (round + k) % (npad - 1);
    q = (round - k + (npad - 1)) % (npad - 1);
  }
  if (p > q) { const int x = p; p = q; q = x; }
  if (q >= n) return;  // a dummy column (odd n)
  T* gp = G + (long long)p * ldg;
  T* gq = G + (long long)q * ldg;
  double a = 0.0, b = 0.0;
  T c = zero<T>();
  for (int i = threadIdx.x; i < m; i += SVD_THREADS) {
    const T x = gp[i], y = gq[i];
    a += abs2(x);
    b += abs2(y);
    c = add(c, cmul(x, y));  // conj(x) y
  }
  block_sum3<T>(a, b, c, sh);
  const double g = sqrt(abs2(c));
  if (!(g > tol * sqrt(a * b))) return;  // already orthogonal (or a zero column)
  const T ph = scal(1.0 / g, c);          // gamma / |gamma|
  const double zeta = (b - a) / (2.0 * g);
  const double t = (zeta >= 0.0 ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
  const double cs = 1.0 / sqrt(1.0 + t * t), sn = cs * t;
  // [g_p, g_q ph^*] rotated: g_p' = c g_p - s g_q ph^*, g_q' = (s g_p + c g_q ph^*) ph
  for (int i = threadIdx.x; i < m; i += SVD_THREADS) {
    const T x = gp[i], y = mul(gq[i], conj_(ph));
    gp[i] = sub(scal(cs, x), scal(sn, y));
    gq[i] = mul(add(scal(sn, x), scal(cs, y)), ph);
  }
  T* vp = V + (long long)p * ldv;
  T* vq = V + (long long)q * ldv;
  for (int i = threadIdx.x; i < n; i += SVD_THREADS) {
    const T x = vp[i], y = mul(vq[i], conj_(ph));
    vp[i] = sub(scal(cs, x), scal(sn, y));
    vq[i] = mul(add(scal(sn, x), scal(cs, y)), ph);
  }
  if (threadIdx.x == 0) atomicAdd(rotated, 1);
}

// u_j = g_j / ||g_j||; nrm[j] = ||g_j|| (one CTA per column)
template <class T>
__global__ void __launch_bounds__(SVD_THREADS) normalize_cols_kernel(int m, T* G, int ldg, double* nrm) {
  __shared__ double sh[4 * SVD_THREADS];
  T* g = G + (long long)blockIdx.x * ldg;
  double a = 0.0, b = 0.0;
  T c = zero<T>();
  for (int i = threadIdx.x; i < m; i += SVD_THREADS) a += abs2(g[i]);
  block_sum3<T>(a, b, c, sh);
  const double s = sqrt(a);
  if (threadIdx.x == 0) nrm[blockIdx.x] = s;
  if (s > 0.0)
    for (int i = threadIdx.x; i < m; i += SVD_THREADS) g[i] = scal(1.0 / s, g[i]);
}

template <class T>
__global__ void unit_col_kernel(int m, T* x, int k) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < m; i += gridDim.x * blockDim.x)
    x[i] = from_re<T>(i == k ? 1.0 : 0.0);
}

}  // namespace

template <class T>
void svd_polar(Ctx& cx, Arena& ar, int n, const T* A, int lda, T* W, int ldw) {
  cudaStream_t st = cx.stream;
  const long long nn = (long long)n * n;
  const size_t mk = ar.mark();
  T* G = ar.get<T>(nn);
  T* V = ar.get<T>(nn);
  T* y = ar.get<T>(n);
  double* nrm = ar.get<double>(n);
  int* rot = ar.get<int>(1);
  axpby<T>(st, n, n, 1.0, A, lda, 0, 0.0, G, n, 0, 1);
  set_eye<T>(st, n, n, V, n, 0, 1);
  const int npad = n + (n & 1);
  const double tol = std::sqrt((double)n) * U_ROUND;  // the level a plain dot product can resolve
  for (int sweep = 0; sweep < 40 && n > 1; ++sweep) {
    ZCSD_CUDA(cudaMemsetAsync(rot, 0, sizeof(int), st));
    for (int r = 0; r < npad - 1; ++r) {
      jacobi_round_kernel<T><<<npad / 2, SVD_THREADS, 0, st>>>(n, n, npad, r, G, n, V, n, tol, rot);
      ZCSD_LAUNCH();
    }
    d2h(cx, cx.hs.i, rot, sizeof(int));
    if (cx.hs.i[0] == 0) break;
  }
  normalize_cols_kernel<T><<<n, SVD_THREADS, 0, st>>>(n, G, n, nrm);
  ZCSD_LAUNCH();
  // exactly zero columns (sigma_j = 0): orthonormal completion against the
  // other columns, x = e_k - U (U^* e_k), twice, normalised
  std::vector<double> hn(n);
  ZCSD_CUDA(cudaMemcpyAsync(hn.data(), nrm, sizeof(double) * n, cudaMemcpyDeviceToHost, st));
  ZCSD_CUDA(cudaStreamSynchronize(st));
  const T one = from_re<T>(1.0), mone = from_re<T>(-1.0), zer = zero<T>();
  int kpick = 0;
  for (int j = 0; j < n; ++j) {
    if (hn[j] > 0.0) continue;
    T* x = G + (long long)j * n;
    for (int attempt = 0; attempt < n; ++attempt, kpick = (kpick + 1) % n) {
      unit_col_kernel<T><<<ceil_div(n, 256), 256, 0, st>>>(n, x, kpick);
      ZCSD_LAUNCH();
      for (int rep = 0; rep < 2; ++rep) {
        // the zero column itself contributes nothing (it is x, orthogonal to the rest)
        gemm1<T>(st, OP_C, OP_N, n, 1, n, one, G, n, x, n, zer, y, n, 0, 0, GS_ALG2);
        unit_col_kernel<T><<<1, 32, 0, st>>>(1, y + j, -1);  // y_j = 0: leave x's own coefficient out
        ZCSD_LAUNCH();
        gemm1<T>(st, OP_N, OP_N, n, 1, n, mone, G, n, y, n, one, x, n, 0, 0, GS_ALG2);
      }
      normalize_cols_kernel<T><<<1, SVD_THREADS, 0, st>>>(n, x, n, nrm + j);
      ZCSD_LAUNCH();
      double hx = 0.0;
      ZCSD_CUDA(cudaMemcpyAsync(&hx, nrm + j, sizeof(double), cudaMemcpyDeviceToHost, st));
      ZCSD_CUDA(cudaStreamSynchronize(st));
      if (hx > 0.5) {  // e_k had a component of at least 1/2 outside the kept span
        kpick = (kpick + 1) % n;
        break;
      }
    }
  }
  // W = U V^*
  gemm1<T>(st, OP_N, OP_C, n, n, n, one, G, n, V, n, zer, W, ldw, 0, 0, GS_ALG2);
  ar.release(mk);
}

template void svd_polar<double>(Ctx&, Arena&, int, const double*, int, double*, int);
template void svd_polar<z64>(Ctx&, Arena&, int, const z64*, int, z64*, int);

}  // namespace zcsd
