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
#include <algorithm>
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
// Eigendecomposition of the leaf blocks of Zolo-eig by two-sided cyclic
// Jacobi, batched over all leaves of any sizes.  Leaf l is an sz_l x sz_l
// Hermitian block B_l (element offset boff_l, leading dimension ldb_l),
// copied to G_l (leading dimension sz_l, packed at goff_l).  A round of the
// tournament order rotates n/2 disjoint pairs (p, q); each rotation zeroes
// g_pq (tan 2 phi = 2 |g_pq| / (g_qq - g_pp), the phase of g_pq moved into
// column q first) and G <- J^* G J is applied in column-only form, so every
// access is to a CTA's own two columns:
//   kernel 1 (one CTA per pair): the angle from g_pp, g_qq, g_pq (entries of
//     its own columns), the column rotation of G and V, and the rotation
//     recorded for rows p and q;
//   kernel 2 (one CTA per pair, the idle column of an odd size included):
//     the row rotations of every pair applied to the CTA's own columns.
// Pairs with |g_pq| <= u ||B_l||_F are not rotated; a sweep with no
// rotation ends the leaf.  The eigenvalues are the diagonal of G.  Unlike
// one-sided Jacobi on a shifted matrix, every step is a similarity
// transform of B_l itself, so the eigenvectors carry no shift-dependent
// error.
namespace {

__device__ __forceinline__ int leaf_of(const LeafTable& L, int b) {
  int lo = 0, hi = L.nl - 1;  // last l with pre[l] <= b
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (L.pre[mid] <= b) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

// rotation recorded for row i of a leaf in the current round
struct JRow {
  int partner;  // the other index of i's pair (-1: i is idle this round)
  int first;    // i is the smaller index of its pair
  double c, s, phr, phi;  // rotation and the phase of g_pq (moved into q)
};

__device__ __forceinline__ void leaf_pair(const LeafTable& L, int round, int& l, int& p, int& q, int& n) {
  l = leaf_of(L, blockIdx.x);
  n = L.sz[l];
  const int npad = n + (n & 1);
  const int k = blockIdx.x - L.pre[l];
  if (k == 0) {
    p = npad - 1;
    q = round;
  } else {
    p = (round + k) % (npad - 1);
    q = (round - k + (npad - 1)) % (npad - 1);
  }
  if (p > q) { const int x = p; p = q; q = x; }
}

template <class T>
__device__ __forceinline__ T phase_of(double r, double i);
template <>
__device__ __forceinline__ double phase_of<double>(double r, double) { return r; }
template <>
__device__ __forceinline__ z64 phase_of<z64>(double r, double i) { return z64{r, i}; }

template <class T>
__global__ void __launch_bounds__(SVD_THREADS) leaf_col_kernel(LeafTable L, int round, T* G, T* V, JRow* rows) {
  int l, p, q, n;
  leaf_pair(L, round, l, p, q, n);
  if (L.done[l]) return;
  const int npad = n + (n & 1);
  if (round >= npad - 1) return;
  JRow* R = rows + L.roff[l];
  if (q >= n) {  // p is idle this round
    if (threadIdx.x == 0 && p < n) R[p] = JRow{-1, 0, 1.0, 0.0, 1.0, 0.0};
    return;
  }
  T* gp = G + L.goff[l] + (long long)p * n;
  T* gq = G + L.goff[l] + (long long)q * n;
  const double gpp = re(gp[p]), gqq = re(gq[q]);
  const T gpq = gq[p];
  // every thread has its copy of the pivot entries before any thread
  // rotates rows p and q of these columns (all threads reach this barrier:
  // the early returns above are uniform over the CTA)
  __syncthreads();
  const double g = sqrt(abs2(gpq));
  double cs = 1.0, sn = 0.0;
  T ph = from_re<T>(1.0);
  const bool rot = g > U_ROUND * L.c[l];
  if (rot) {
    ph = scal(1.0 / g, gpq);
    const double zeta = (gqq - gpp) / (2.0 * g);
    const double t = (zeta >= 0.0 ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
    cs = 1.0 / sqrt(1.0 + t * t);
    sn = cs * t;
    for (int i = threadIdx.x; i < n; i += SVD_THREADS) {
      const T x = gp[i], y = mul(gq[i], conj_(ph));
      gp[i] = sub(scal(cs, x), scal(sn, y));
      gq[i] = add(scal(sn, x), scal(cs, y));
    }
    T* vp = V + L.goff[l] + (long long)p * n;
    T* vq = V + L.goff[l] + (long long)q * n;
    for (int i = threadIdx.x; i < n; i += SVD_THREADS) {
      const T x = vp[i], y = mul(vq[i], conj_(ph));
      vp[i] = sub(scal(cs, x), scal(sn, y));
      vq[i] = add(scal(sn, x), scal(cs, y));
    }
  }
  if (threadIdx.x == 0) {
    R[p] = JRow{q, 1, cs, sn, re(ph), im(ph)};
    R[q] = JRow{p, 0, cs, sn, re(ph), im(ph)};
    if (rot) atomicAdd(&L.rot[l], 1);
  }
}

template <class T>
__global__ void __launch_bounds__(SVD_THREADS) leaf_row_kernel(LeafTable L, int round, T* G, const JRow* rows) {
  int l, p, q, n;
  leaf_pair(L, round, l, p, q, n);
  if (L.done[l]) return;
  const int npad = n + (n & 1);
  if (round >= npad - 1) return;
  const JRow* R = rows + L.roff[l];
  for (int w = 0; w < 2; ++w) {
    const int col = w == 0 ? p : q;
    if (col >= n) continue;
    T* gc = G + L.goff[l] + (long long)col * n;
    for (int i = threadIdx.x; i < n; i += SVD_THREADS) {
      const JRow r = R[i];
      if (!r.first || r.partner < 0) continue;
      if (r.s == 0.0 && r.phr == 1.0 && r.phi == 0.0) continue;  // not rotated
      const int j = r.partner;
      const T ph = phase_of<T>(r.phr, r.phi);
      const T x = gc[i], y = mul(gc[j], ph);
      gc[i] = sub(scal(r.c, x), scal(r.s, y));
      gc[j] = add(scal(r.s, x), scal(r.c, y));
    }
  }
}

// c_l = ||B_l||_F (one CTA per leaf)
template <class T>
__global__ void __launch_bounds__(SVD_THREADS) leaf_norm_kernel(LeafTable L, const T* B) {
  __shared__ double sh[4 * SVD_THREADS];
  const int l = blockIdx.x, n = L.sz[l], ld = L.ldb[l];
  const T* Bl = B + L.boff[l];
  double a = 0.0, b = 0.0;
  T z = zero<T>();
  for (long long t = threadIdx.x; t < (long long)n * n; t += SVD_THREADS) {
    const int i = (int)(t % n), j = (int)(t / n);
    a += abs2(Bl[i + (long long)j * ld]);
  }
  block_sum3<T>(a, b, z, sh);
  if (threadIdx.x == 0) {
    L.c[l] = sqrt(a) > 0.0 ? sqrt(a) : 1.0;
    L.rot[l] = 0;
    L.done[l] = 0;
  }
}

// G_l = B_l, V_l = I (blockIdx.y = leaf)
template <class T>
__global__ void leaf_setup_kernel(LeafTable L, const T* B, T* G, T* V) {
  const int l = blockIdx.y, n = L.sz[l], ld = L.ldb[l];
  const T* Bl = B + L.boff[l];
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < (long long)n * n;
       t += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(t % n), j = (int)(t / n);
    G[L.goff[l] + t] = Bl[i + (long long)j * ld];
    V[L.goff[l] + t] = from_re<T>(i == j ? 1.0 : 0.0);
  }
}

// after a sweep: a leaf that rotated nothing is done
__global__ void leaf_sweep_end_kernel(LeafTable L) {
  for (int l = blockIdx.x * blockDim.x + threadIdx.x; l < L.nl; l += gridDim.x * blockDim.x) {
    if (L.rot[l] == 0) L.done[l] = 1;
    L.rot[l] = 0;
  }
}

// lambda[loff_l + j] = Re g_jj (blockIdx.y = leaf)
template <class T>
__global__ void leaf_values_kernel(LeafTable L, const T* G, double* lam) {
  const int l = blockIdx.y, n = L.sz[l];
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x)
    lam[L.loff[l] + j] = re(G[L.goff[l] + j + (long long)j * n]);
}

// Leaves of at most SMALL_LEAF rows: one CTA per leaf runs the whole
// iteration in shared memory (G and V of a 64-row complex leaf take 128 KiB).
// Every round: the rotations of its disjoint pairs from G (one thread per
// pair, the same formulas as leaf_col_kernel), then the column rotations of
// G and V, then the row rotations of G, each phase closed by a barrier; a
// sweep with no rotation ends the iteration (at most 40 sweeps).  No launch
// per round and no host read per sweep.
constexpr int SMALL_LEAF = 64;

template <class T>
__global__ void __launch_bounds__(SVD_THREADS) leaf_smem_kernel(const T* B, int ldb, const int* off, const int* sz,
                                                                 const long long* voff, double* lam, T* Vl) {
  extern __shared__ __align__(16) unsigned char leaf_smem[];
  __shared__ int pp[SMALL_LEAF / 2], pq[SMALL_LEAF / 2], act[SMALL_LEAF / 2];
  __shared__ double pc[SMALL_LEAF / 2], ps[SMALL_LEAF / 2], phr[SMALL_LEAF / 2], phi[SMALL_LEAF / 2];
  __shared__ int nrot;
  __shared__ double sh[4 * SVD_THREADS];
  const int l = blockIdx.x, o = off[l], n = sz[l];
  const int tid = threadIdx.x;
  T* G = reinterpret_cast<T*>(leaf_smem);  // n x n, column-major, ld n
  T* W = G + n * n;                        // eigenvectors
  double a = 0.0, b2 = 0.0;
  T z = zero<T>();
  for (int t = tid; t < n * n; t += SVD_THREADS) {
    const int i = t % n, j = t / n;
    const T x = B[(o + i) + (long long)(o + j) * ldb];
    G[t] = x;
    W[t] = from_re<T>(i == j ? 1.0 : 0.0);
    a += abs2(x);
  }
  block_sum3<T>(a, b2, z, sh);  // a = ||B_l||_F^2 for every thread
  const double thr = U_ROUND * (a > 0.0 ? sqrt(a) : 1.0);
  const int npad = n + (n & 1), npairs = npad / 2;
  for (int sweep = 0; sweep < 40 && n > 1; ++sweep) {
    if (tid == 0) nrot = 0;
    __syncthreads();
    for (int r = 0; r < npad - 1; ++r) {
      if (tid < npairs) {
        const int k = tid;
        int p, q;
        if (k == 0) {
          p = npad - 1;
          q = r;
        } else {
          p = (r + k) % (npad - 1);
          q = (r - k + (npad - 1)) % (npad - 1);
        }
        if (p > q) { const int x = p; p = q; q = x; }
        int on = 0;
        if (q < n) {
          const double gpp = re(G[p + p * n]), gqq = re(G[q + q * n]);
          const T gpq = G[p + q * n];
          const double g = sqrt(abs2(gpq));
          if (g > thr) {
            const T ph = scal(1.0 / g, gpq);
            const double zeta = (gqq - gpp) / (2.0 * g);
            const double t = (zeta >= 0.0 ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
            const double c = 1.0 / sqrt(1.0 + t * t);
            pc[k] = c;
            ps[k] = c * t;
            phr[k] = re(ph);
            phi[k] = im(ph);
            on = 1;
            atomicAdd(&nrot, 1);
          }
        }
        pp[k] = p;
        pq[k] = q;
        act[k] = on;
      }
      __syncthreads();
      // columns p, q of G and V
      for (int it = tid; it < npairs * n; it += SVD_THREADS) {
        const int k = it / n, i = it % n;
        if (!act[k]) continue;
        const int p = pp[k], q = pq[k];
        const double c = pc[k], s = ps[k];
        const T phc = conj_(phase_of<T>(phr[k], phi[k]));
        {
          const T x = G[i + p * n], y = mul(G[i + q * n], phc);
          G[i + p * n] = sub(scal(c, x), scal(s, y));
          G[i + q * n] = add(scal(s, x), scal(c, y));
        }
        {
          const T x = W[i + p * n], y = mul(W[i + q * n], phc);
          W[i + p * n] = sub(scal(c, x), scal(s, y));
          W[i + q * n] = add(scal(s, x), scal(c, y));
        }
      }
      __syncthreads();
      // rows p, q of G
      for (int it = tid; it < npairs * n; it += SVD_THREADS) {
        const int k = it / n, j = it % n;
        if (!act[k]) continue;
        const int p = pp[k], q = pq[k];
        const double c = pc[k], s = ps[k];
        const T ph = phase_of<T>(phr[k], phi[k]);
        const T x = G[p + j * n], y = mul(G[q + j * n], ph);
        G[p + j * n] = sub(scal(c, x), scal(s, y));
        G[q + j * n] = add(scal(s, x), scal(c, y));
      }
      __syncthreads();
    }
    // every thread reads the count before thread 0 may reset it for the
    // next sweep, so the exit is uniform over the CTA
    const int rotated = nrot;
    __syncthreads();
    if (rotated == 0) break;
  }
  for (int j = tid; j < n; j += SVD_THREADS) lam[o + j] = re(G[j + j * n]);
  T* Vo = Vl + voff[l];
  for (int t = tid; t < n * n; t += SVD_THREADS) Vo[t] = W[t];
}

}  // namespace

LeafTable leaf_table_build(Ctx& cx, Arena& ar, const std::vector<long long>& boff, const std::vector<int>& ldb,
                           const std::vector<int>& loff, const std::vector<int>& sz) {
  LeafTable L;
  const int nl = (int)sz.size();
  L.nl = nl;
  std::vector<int> hi(5 * nl + 1, 0);
  std::vector<long long> hl(3 * nl + 2, 0);
  for (int l = 0; l < nl; ++l) {
    hi[l] = ldb[l];
    hi[nl + l] = loff[l];
    hi[2 * nl + l] = sz[l];
    const int npad = sz[l] + (sz[l] & 1);
    hi[3 * nl + l + 1] = hi[3 * nl + l] + npad / 2;
    hl[l] = boff[l];
    hl[nl + l + 1] = hl[nl + l] + (long long)sz[l] * sz[l];
    hl[2 * nl + 1 + l + 1] = hl[2 * nl + 1 + l] + sz[l];
    L.maxsz = std::max(L.maxsz, sz[l]);
    L.maxpad = std::max(L.maxpad, npad);
    L.sweep_flops += (double)sz[l] * (sz[l] - 1) / 2 * 30.0 * sz[l];
  }
  L.total_pairs = hi[4 * nl];
  L.vtot = hl[2 * nl];
  L.rtot = hl[3 * nl + 1];
  int* di = ar.get<int>(7 * nl + 1);
  long long* dl = ar.get<long long>(3 * nl + 2);
  L.c = ar.get<double>(nl);
  ZCSD_CUDA(cudaMemcpyAsync(di, hi.data(), sizeof(int) * (4 * nl + 1), cudaMemcpyHostToDevice, cx.stream));
  ZCSD_CUDA(cudaMemcpyAsync(dl, hl.data(), sizeof(long long) * (3 * nl + 2), cudaMemcpyHostToDevice, cx.stream));
  ZCSD_CUDA(cudaStreamSynchronize(cx.stream));  // host tables go out of scope
  L.ldb = di;
  L.loff = di + nl;
  L.sz = di + 2 * nl;
  L.pre = di + 3 * nl;
  L.rot = di + 4 * nl + 1;
  L.done = di + 5 * nl + 1;
  L.boff = dl;
  L.goff = dl + nl;
  L.roff = dl + 2 * nl + 1;
  L.rows = ar.get<char>((size_t)L.rtot * sizeof(JRow));
  return L;
}

template <class T>
void leaf_solve(Ctx& cx, const LeafTable& L, const T* B, double* lam, T* G, T* V, int fixed_sweeps) {
  cudaStream_t st = cx.stream;
  if (L.nl == 0) return;
  ProfToken tok = prof_begin(st);
  JRow* rows = reinterpret_cast<JRow*>(L.rows);
  leaf_norm_kernel<T><<<L.nl, SVD_THREADS, 0, st>>>(L, B);
  ZCSD_LAUNCH();
  leaf_setup_kernel<T><<<dim3(ceil_div((long long)L.maxsz * L.maxsz, 1024) + 1, L.nl), 256, 0, st>>>(L, B, G, V);
  ZCSD_LAUNCH();
  const int nsweeps = fixed_sweeps > 0 ? fixed_sweeps : 40;
  std::vector<int> hrot(L.nl);
  double flops = 0.0;
  for (int sweep = 0; sweep < nsweeps && L.maxsz > 1; ++sweep) {
    flops += L.sweep_flops * (sizeof(T) == 8 ? 1.0 : 4.0);
    for (int r = 0; r < L.maxpad - 1; ++r) {
      leaf_col_kernel<T><<<L.total_pairs, SVD_THREADS, 0, st>>>(L, r, G, V, rows);
      ZCSD_LAUNCH();
      leaf_row_kernel<T><<<L.total_pairs, SVD_THREADS, 0, st>>>(L, r, G, rows);
      ZCSD_LAUNCH();
    }
    if (fixed_sweeps <= 0) {  // read the rotation counts: stop once no leaf rotated
      ZCSD_CUDA(cudaMemcpyAsync(hrot.data(), L.rot, sizeof(int) * L.nl, cudaMemcpyDeviceToHost, st));
      ZCSD_CUDA(cudaStreamSynchronize(st));
      bool any = false;
      for (int l = 0; l < L.nl; ++l) any = any || hrot[l] != 0;
      if (!any) break;
    }
    leaf_sweep_end_kernel<<<ceil_div(L.nl, 256), 256, 0, st>>>(L);
    ZCSD_LAUNCH();
  }
  leaf_values_kernel<T><<<dim3(ceil_div(L.maxsz, 256), L.nl), 256, 0, st>>>(L, G, lam);
  ZCSD_LAUNCH();
  if (tok.slot >= 0) prof_end(tok, st, PK_JACOBI, flops);
}

template void leaf_solve<double>(Ctx&, const LeafTable&, const double*, double*, double*, double*, int);
template void leaf_solve<z64>(Ctx&, const LeafTable&, const z64*, double*, z64*, z64*, int);

template <class T>
void jacobi_eig_leaves(Ctx& cx, Arena& ar, const std::vector<int>& off, const std::vector<int>& sz, const T* B,
                       int ldb, double* lam, T* Vl, std::vector<long long>& voff) {
  const int nl = (int)off.size();
  if (nl == 0) return;
  const size_t mk = ar.mark();
  std::vector<long long> boff(nl);
  std::vector<int> lds(nl, ldb);
  voff.assign(nl + 1, 0);
  for (int l = 0; l < nl; ++l) {
    boff[l] = off[l] + (long long)off[l] * ldb;
    voff[l + 1] = voff[l] + (long long)sz[l] * sz[l];
  }
  const int maxsz = *std::max_element(sz.begin(), sz.end());
  if (maxsz <= SMALL_LEAF) {
    // every leaf in one CTA of shared memory, all leaves in one launch
    const size_t smem = 2 * (size_t)SMALL_LEAF * SMALL_LEAF * sizeof(T);
    static const bool attr = [smem] {
      ZCSD_CUDA(cudaFuncSetAttribute(leaf_smem_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
      return true;
    }();
    (void)attr;
    int* doff = ar.get<int>(nl);
    int* dsz = ar.get<int>(nl);
    long long* dvoff = ar.get<long long>(nl);
    ZCSD_CUDA(cudaMemcpyAsync(doff, off.data(), sizeof(int) * nl, cudaMemcpyHostToDevice, cx.stream));
    ZCSD_CUDA(cudaMemcpyAsync(dsz, sz.data(), sizeof(int) * nl, cudaMemcpyHostToDevice, cx.stream));
    ZCSD_CUDA(cudaMemcpyAsync(dvoff, voff.data(), sizeof(long long) * nl, cudaMemcpyHostToDevice, cx.stream));
    ProfToken tok = prof_begin(cx.stream);
    leaf_smem_kernel<T><<<nl, SVD_THREADS, 2 * (size_t)maxsz * maxsz * sizeof(T), cx.stream>>>(B, ldb, doff, dsz, dvoff,
                                                                                               lam, Vl);
    ZCSD_LAUNCH();
    if (tok.slot >= 0) prof_end(tok, cx.stream, PK_JACOBI, 0.0);
    ar.release(mk);
    return;
  }
  LeafTable L = leaf_table_build(cx, ar, boff, lds, off, sz);
  T* G = ar.get<T>((size_t)L.vtot);
  leaf_solve<T>(cx, L, B, lam, G, Vl, 0);
  ar.release(mk);
}

template void jacobi_eig_leaves<double>(Ctx&, Arena&, const std::vector<int>&, const std::vector<int>&, const double*,
                                        int, double*, double*, std::vector<long long>&);
template void jacobi_eig_leaves<z64>(Ctx&, Arena&, const std::vector<int>&, const std::vector<int>&, const z64*, int,
                                     double*, z64*, std::vector<long long>&);

}  // namespace zcsd
