// Reverse-mode derivative of the full-rank real CS decomposition computed by
// Algorithm 1 (the paper has no derivatives; this is the adjoint of its
// steps).  At a partial isometry the two Hermitian polar factors share the
// eigenvectors V1 of B = H2 - H1 (Section 3: H1 = V1 C V1^*, H2 = V1 S V1^*)
// and W_i = U_i V1^*, so the whole adjoint can be written in the basis V1
// from the outputs (U1, U2, V1, theta) alone:
//
//   X  = V1^T V1_bar + U1^T U1_bar + U2^T U2_bar           (three products)
//   lam_k = s_k - c_k (eigenvalues of B), c = cos theta, s = sin theta
//   c_bar = -s theta_bar, s_bar = c theta_bar              (theta = atan2(s, c))
//   Bb_kl = skew(X)_kl / (lam_l - lam_k), k != l           (eig of B)
//   H1b = diag(c_bar) - Bb,  H2b = diag(s_bar) + Bb        (B = H2 - H1)
//   G_i  = skew(U_i^T U_i_bar) - (H_ib Sig_i - Sig_i H_ib) / 2
//   K_i  = 2 G_i / (sig_k + sig_l) + H_ib                  (Lyapunov solve of the
//          polar factor, Sig_1 = diag(c), Sig_2 = diag(s))
//   A_i_bar = U_i K_i V1^T                                  (four products)
#include "solver.h"

namespace zcsd {

namespace {

__global__ void csd_grad_core_kernel(int n, const double* theta, const double* gtheta, const double* M0,
                                     const double* M1, const double* M2, double* K1, double* K2) {
  const long long total = (long long)n * n;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    const int k = (int)(t % n), l = (int)(t / n);
    const long long kl = t, lk = l + (long long)k * n;
    double ck, sk, cl, sl;
    sincos(theta[k], &sk, &ck);
    sincos(theta[l], &sl, &cl);
    const double xkl = M0[kl] + M1[kl] + M2[kl], xlk = M0[lk] + M1[lk] + M2[lk];
    const double dl = (sl - cl) - (sk - ck);  // lam_l - lam_k
    const double bb = (k != l && dl != 0.0) ? 0.5 * (xkl - xlk) / dl : 0.0;
    double h1 = -bb, h2 = bb;
    if (k == l) {
      const double tb = gtheta ? gtheta[k] : 0.0;
      h1 += -sk * tb;
      h2 += ck * tb;
    }
    const double g1 = 0.5 * (M1[kl] - M1[lk]) - 0.5 * h1 * (cl - ck);
    const double g2 = 0.5 * (M2[kl] - M2[lk]) - 0.5 * h2 * (sl - sk);
    const double d1 = ck + cl, d2 = sk + sl;
    K1[t] = (d1 != 0.0 ? 2.0 * g1 / d1 : 0.0) + h1;
    K2[t] = (d2 != 0.0 ? 2.0 * g2 / d2 : 0.0) + h2;
  }
}

// Column j of V1 (and of U1, U2) times the sign (or, complex, the inverse
// phase) of V1's entry of largest magnitude (first such index): one CTA per
// column.
template <class T>
__global__ void canon_signs_kernel(int m1, int m2, int n, int ncols, T* V, int ldv, T* U1, int ldu1, T* U2, int ldu2) {
  const int j = blockIdx.x;
  if (j >= ncols) return;
  __shared__ double best[256];
  __shared__ int bidx[256];
  double bv = -1.0;
  int bi = 0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const double a = abs2(V[i + (long long)j * ldv]);
    if (a > bv) { bv = a; bi = i; }
  }
  best[threadIdx.x] = bv;
  bidx[threadIdx.x] = bi;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) {
      const double o = best[threadIdx.x + s];
      const int oi = bidx[threadIdx.x + s];
      if (o > best[threadIdx.x] || (o == best[threadIdx.x] && oi < bidx[threadIdx.x])) {
        best[threadIdx.x] = o;
        bidx[threadIdx.x] = oi;
      }
    }
    __syncthreads();
  }
  const T p = V[bidx[0] + (long long)j * ldv];
  const double a = sqrt(abs2(p));
  const T ph = a > 0.0 ? scal(1.0 / a, conj_(p)) : from_re<T>(1.0);  // |ph| = 1
  __syncthreads();
  for (int i = threadIdx.x; i < n; i += blockDim.x) V[i + (long long)j * ldv] = mul(V[i + (long long)j * ldv], ph);
  for (int i = threadIdx.x; i < m1; i += blockDim.x) U1[i + (long long)j * ldu1] = mul(U1[i + (long long)j * ldu1], ph);
  for (int i = threadIdx.x; i < m2; i += blockDim.x) U2[i + (long long)j * ldu2] = mul(U2[i + (long long)j * ldu2], ph);
}

int grid_for_n2(long long total) { return (int)std::min<long long>((total + 255) / 256, 152 * 8); }

}  // namespace

template <class T>
void canonical_signs(cudaStream_t st, int m1, int m2, int n, int ncols, T* V, int ldv, T* U1, int ldu1, T* U2,
                     int ldu2) {
  if (ncols <= 0) return;
  canon_signs_kernel<T><<<ncols, 256, 0, st>>>(m1, m2, n, ncols, V, ldv, U1, ldu1, U2, ldu2);
  ZCSD_LAUNCH();
}

template void canonical_signs<double>(cudaStream_t, int, int, int, int, double*, int, double*, int, double*, int);
template void canonical_signs<z64>(cudaStream_t, int, int, int, int, z64*, int, z64*, int, z64*, int);

int csd_backward_impl(Ctx& cx, Arena& ar, int n, const double* U1, int ldu1, const double* U2, int ldu2,
                      const double* V, int ldv, const double* theta, const double* gU1, int ldgu1, const double* gU2,
                      int ldgu2, const double* gV, int ldgv, const double* gtheta, double* gA1, int ldga1, double* gA2,
                      int ldga2) {
  cudaStream_t st = cx.stream;
  const long long nn = (long long)n * n;
  double* M = ar.get<double>(3 * nn);  // V^T gV, U1^T gU1, U2^T gU2
  double* K = ar.get<double>(2 * nn);
  double* Tm = ar.get<double>(nn);
  const double* G[3] = {gV, gU1, gU2};
  const double* F[3] = {V, U1, U2};
  const int ldf[3] = {ldv, ldu1, ldu2}, ldg[3] = {ldgv, ldgu1, ldgu2};
  for (int q = 0; q < 3; ++q) {
    if (G[q]) gemm1<double>(st, OP_T, OP_N, n, n, n, 1.0, F[q], ldf[q], G[q], ldg[q], 0.0, M + q * nn, n, 0, 0, GS_GRAD);
    else ZCSD_CUDA(cudaMemsetAsync(M + q * nn, 0, sizeof(double) * nn, st));
  }
  csd_grad_core_kernel<<<grid_for_n2(nn), 256, 0, st>>>(n, theta, gtheta, M, M + nn, M + 2 * nn, K, K + nn);
  ZCSD_LAUNCH();
  double* out[2] = {gA1, gA2};
  const int ldo[2] = {ldga1, ldga2};
  for (int i = 0; i < 2; ++i) {
    // A_i_bar = U_i K_i V^T
    gemm1<double>(st, OP_N, OP_N, n, n, n, 1.0, F[1 + i], ldf[1 + i], K + i * nn, n, 0.0, Tm, n, 0, 0, GS_GRAD);
    gemm1<double>(st, OP_N, OP_T, n, n, n, 1.0, Tm, n, V, ldv, 0.0, out[i], ldo[i], 0, 0, GS_GRAD);
  }
  return CSD_OK;
}

}  // namespace zcsd
