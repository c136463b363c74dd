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
#include <vector>

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

// ---------------------------------------------------------------- leaves
// Eigendecomposition of the leaf blocks of Zolo-eig by the same one-sided
// Jacobi method, batched over all leaves of any sizes: for leaf l (the
// sz_l x sz_l diagonal block of B at offset off_l) G_l = B_l + c_l I with
// c_l = ||B_l||_F, which is positive definite, so its one-sided Jacobi
// factorization G_l V_l = U_l Sigma_l has U_l = V_l and
// lambda_j = sigma_j - c_l (eigenvalues of distinct sigma stay distinct).
// Every CTA of a round rotates one column pair of one leaf; leaves are packed
// one after another (G_l and V_l with leading dimension sz_l at goff_l).
namespace {

struct LeafDev {
  const int* off;   // offset of the block in B
  const int* sz;    // block size
  const int* pre;   // pairs before leaf l (exclusive prefix of npad_l / 2), pre[nl] = total
  const long long* goff;  // element offset of G_l and V_l in the packed buffers
  const double* c;  // shift c_l
  int* rot;         // rotations of leaf l in the current sweep
  const int* done;  // leaf l converged
  int nl;
};

__device__ __forceinline__ int leaf_of(const LeafDev& L, int b) {
  int lo = 0, hi = L.nl - 1;  // last l with pre[l] <= b
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (L.pre[mid] <= b) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

template <class T>
__global__ void __launch_bounds__(SVD_THREADS) leaf_round_kernel(LeafDev L, int round, T* G, T* V, double tol) {
  __shared__ double sh[4 * SVD_THREADS];
  const int l = leaf_of(L, blockIdx.x);
  if (L.done[l]) return;
  const int n = L.sz[l], npad = n + (n & 1);
  if (round >= npad - 1) return;
  const int k = blockIdx.x - L.pre[l];
  int p, q;
  if (k == 0) {
    p = npad - 1;
    q = round;
  } else {
    p = (round + k) % (npad - 1);
    q = (round - k + (npad - 1)) % (npad - 1);
  }
  if (p > q) { const int x = p; p = q; q = x; }
  if (q >= n) return;
  T* gp = G + L.goff[l] + (long long)p * n;
  T* gq = G + L.goff[l] + (long long)q * n;
  double a = 0.0, b = 0.0;
  T c = zero<T>();
  for (int i = threadIdx.x; i < n; i += SVD_THREADS) {
    const T x = gp[i], y = gq[i];
    a += abs2(x);
    b += abs2(y);
    c = add(c, cmul(x, y));
  }
  block_sum3<T>(a, b, c, sh);
  const double g = sqrt(abs2(c));
  if (!(g > tol * sqrt(a * b))) return;
  const T ph = scal(1.0 / g, c);
  const double zeta = (b - a) / (2.0 * g);
  const double t = (zeta >= 0.0 ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
  const double cs = 1.0 / sqrt(1.0 + t * t), sn = cs * t;
  for (int i = threadIdx.x; i < n; i += SVD_THREADS) {
    const T x = gp[i], y = mul(gq[i], conj_(ph));
    gp[i] = sub(scal(cs, x), scal(sn, y));
    gq[i] = mul(add(scal(sn, x), scal(cs, y)), ph);
  }
  T* vp = V + L.goff[l] + (long long)p * n;
  T* vq = V + L.goff[l] + (long long)q * n;
  for (int i = threadIdx.x; i < n; i += SVD_THREADS) {
    const T x = vp[i], y = mul(vq[i], conj_(ph));
    vp[i] = sub(scal(cs, x), scal(sn, y));
    vq[i] = mul(add(scal(sn, x), scal(cs, y)), ph);
  }
  if (threadIdx.x == 0) atomicAdd(&L.rot[l], 1);
}

// c_l = ||B_l||_F (one CTA per leaf)
template <class T>
__global__ void __launch_bounds__(SVD_THREADS) leaf_norm_kernel(LeafDev L, const T* B, int ldb, double* c) {
  __shared__ double sh[4 * SVD_THREADS];
  const int l = blockIdx.x, n = L.sz[l], o = L.off[l];
  double a = 0.0, b = 0.0;
  T z = zero<T>();
  for (long long t = threadIdx.x; t < (long long)n * n; t += SVD_THREADS) {
    const int i = (int)(t % n), j = (int)(t / n);
    a += abs2(B[o + i + (long long)(o + j) * ldb]);
  }
  block_sum3<T>(a, b, z, sh);
  if (threadIdx.x == 0) c[l] = sqrt(a) > 0.0 ? sqrt(a) : 1.0;
}

// G_l = B_l + c_l I, V_l = I (blockIdx.y = leaf)
template <class T>
__global__ void leaf_setup_kernel(LeafDev L, const T* B, int ldb, T* G, T* V) {
  const int l = blockIdx.y, n = L.sz[l], o = L.off[l];
  const double c = L.c[l];
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < (long long)n * n;
       t += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(t % n), j = (int)(t / n);
    T v = B[o + i + (long long)(o + j) * ldb];
    if (i == j) v = add(v, from_re<T>(c));
    G[L.goff[l] + t] = v;
    V[L.goff[l] + t] = from_re<T>(i == j ? 1.0 : 0.0);
  }
}

// lambda[off_l + j] = ||g_j|| - c_l (blockIdx.y = leaf, one CTA per column)
template <class T>
__global__ void __launch_bounds__(SVD_THREADS) leaf_values_kernel(LeafDev L, const T* G, double* lam) {
  __shared__ double sh[4 * SVD_THREADS];
  const int l = blockIdx.y, n = L.sz[l], j = blockIdx.x;
  if (j >= n) return;
  const T* g = G + L.goff[l] + (long long)j * n;
  double a = 0.0, b = 0.0;
  T z = zero<T>();
  for (int i = threadIdx.x; i < n; i += SVD_THREADS) a += abs2(g[i]);
  block_sum3<T>(a, b, z, sh);
  if (threadIdx.x == 0) lam[L.off[l] + j] = sqrt(a) - L.c[l];
}

}  // namespace

template <class T>
void jacobi_eig_leaves(Ctx& cx, Arena& ar, const std::vector<int>& off, const std::vector<int>& sz, const T* B,
                       int ldb, double* lam, T* Vl, std::vector<long long>& voff) {
  cudaStream_t st = cx.stream;
  const int nl = (int)off.size();
  if (nl == 0) return;
  const size_t mk = ar.mark();
  std::vector<int> hi(3 * nl + 1);
  voff.assign(nl + 1, 0);
  int maxsz = 0, maxpad = 0;
  hi[2 * nl] = 0;
  for (int l = 0; l < nl; ++l) {
    hi[l] = off[l];
    hi[nl + l] = sz[l];
    const int npad = sz[l] + (sz[l] & 1);
    hi[2 * nl + l + 1] = hi[2 * nl + l] + npad / 2;
    voff[l + 1] = voff[l] + (long long)sz[l] * sz[l];
    maxsz = std::max(maxsz, sz[l]);
    maxpad = std::max(maxpad, npad);
  }
  const int total_pairs = hi[3 * nl];
  ProfToken tok = prof_begin(st);
  int* di = ar.get<int>(3 * nl + 1 + 2 * nl);
  long long* dgo = ar.get<long long>(nl + 1);
  double* dc = ar.get<double>(nl);
  T* G = ar.get<T>((size_t)voff[nl]);
  ZCSD_CUDA(cudaMemcpyAsync(di, hi.data(), sizeof(int) * (3 * nl + 1), cudaMemcpyHostToDevice, st));
  ZCSD_CUDA(cudaMemcpyAsync(dgo, voff.data(), sizeof(long long) * (nl + 1), cudaMemcpyHostToDevice, st));
  ZCSD_CUDA(cudaMemsetAsync(di + 3 * nl + 1, 0, sizeof(int) * 2 * nl, st));
  LeafDev L;
  L.off = di;
  L.sz = di + nl;
  L.pre = di + 2 * nl;
  L.goff = dgo;
  L.c = dc;
  L.rot = di + 3 * nl + 1;
  L.done = di + 4 * nl + 1;
  L.nl = nl;
  leaf_norm_kernel<T><<<nl, SVD_THREADS, 0, st>>>(L, B, ldb, dc);
  ZCSD_LAUNCH();
  leaf_setup_kernel<T><<<dim3(ceil_div((long long)maxsz * maxsz, 256 * 4) + 1, nl), 256, 0, st>>>(L, B, ldb, G, Vl);
  ZCSD_LAUNCH();
  const double tol = std::sqrt((double)std::max(maxsz, 1)) * U_ROUND;
  std::vector<int> hrot(nl), hdone(nl, 0);
  double flops = 0.0;  // per pair and sweep: three dot products and two column-pair rotations (G and V)
  for (int sweep = 0; sweep < 40 && maxsz > 1; ++sweep) {
    for (int l = 0; l < nl; ++l)
      if (!hdone[l]) flops += (double)sz[l] * (sz[l] - 1) / 2 * (sizeof(T) == 8 ? 30.0 : 120.0) * sz[l];
    ZCSD_CUDA(cudaMemsetAsync(L.rot, 0, sizeof(int) * nl, st));
    for (int r = 0; r < maxpad - 1; ++r) {
      leaf_round_kernel<T><<<total_pairs, SVD_THREADS, 0, st>>>(L, r, G, Vl, tol);
      ZCSD_LAUNCH();
    }
    ZCSD_CUDA(cudaMemcpyAsync(hrot.data(), L.rot, sizeof(int) * nl, cudaMemcpyDeviceToHost, st));
    ZCSD_CUDA(cudaStreamSynchronize(st));
    bool all = true;
    for (int l = 0; l < nl; ++l) {
      if (hrot[l] == 0) hdone[l] = 1;
      all = all && hdone[l];
    }
    if (all) break;
    ZCSD_CUDA(cudaMemcpyAsync((int*)L.done, hdone.data(), sizeof(int) * nl, cudaMemcpyHostToDevice, st));
  }
  leaf_values_kernel<T><<<dim3(maxsz, nl), SVD_THREADS, 0, st>>>(L, G, lam);
  ZCSD_LAUNCH();
  if (tok.slot >= 0) prof_end(tok, st, PK_JACOBI, flops);
  ZCSD_CUDA(cudaStreamSynchronize(st));  // host vectors above go out of scope
  ar.release(mk);
}

template void jacobi_eig_leaves<double>(Ctx&, Arena&, const std::vector<int>&, const std::vector<int>&, const double*,
                                        int, double*, double*, std::vector<long long>&);
template void jacobi_eig_leaves<z64>(Ctx&, Arena&, const std::vector<int>&, const std::vector<int>&, const z64*, int,
                                     double*, z64*, std::vector<long long>&);

}  // namespace zcsd
