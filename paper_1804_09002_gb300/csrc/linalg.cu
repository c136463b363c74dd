// Blocked Householder QR (compact WY), blocked Cholesky and the paired
// triangular solves, as sequences of panel kernels and batched GEMMs.
#include <type_traits>

#include "linalg.h"
#include "tc_gemm.h"

namespace zcsd {

// Split-K factor for a product whose output alone gives too few tiles, or a
// tile count that fills its last wave poorly: the GEMM keeps two CTAs per SM
// resident (304 slots on 152 SMs), so a launch of C CTAs runs ceil(C / 304)
// waves; pick the split s (K chunks of at least kmin) that maximises the
// filled fraction C s / (304 ceil(C s / 304)), smaller s on ties.
static int pick_ksplit(int m, int n, int k, int batch, int bm, int kmin = 256) {
  const long long tiles = (long long)ceil_div(m, bm) * ceil_div(n, 4096 / bm) * batch;
  const int smax = std::min(MAX_SUM, std::max(1, k / kmin));
  constexpr long long slots = 2 * 152;
  int best = 1;
  double best_eff = -1.0;
  for (int s = 1; s <= smax; ++s) {
    const long long c = tiles * s;
    const double eff = (double)c / (double)(slots * ((c + slots - 1) / slots));
    if (eff > best_eff + 0.02) {
      best_eff = eff;
      best = s;
    }
  }
  return best;
}

// Products the tensor-core path takes run unsplit (it takes the whole K range).
template <class T>
static int resolve_ksplit(GemmArgs<T>& g, int ks) {
  g.ksplit = ks;
  if constexpr (std::is_same<T, double>::value) {
    if (ks > 1) {
      GemmArgs<T> probe = g;
      probe.ksplit = 1;
      if (tc_will_handle(probe)) g.ksplit = 1;
    }
  }
  return g.ksplit;
}

template <class T>
QRStore<T> qr_alloc(Arena& ar, int m, int n, int band, int batch) {
  QRStore<T> q;
  q.m = m; q.n = n; q.band = band; q.batch = batch;
  q.npan = ceil_div(n, NB_QR);
  q.ldy = std::max(1, std::min(m, NB_QR - 1 + band));
  q.sY = (long long)q.npan * q.ldy * NB_QR;
  q.sT = (long long)q.npan * NB_QR * NB_QR;
  q.Y = ar.get<T>((size_t)q.sY * batch);
  q.Tf = ar.get<T>((size_t)q.sT * batch);
  return q;
}

template <class T>
void qr_factor(cudaStream_t st, Arena& ar, QRStore<T>& q, T* M, int ldm, long long sM) {
  const int m = q.m, n = q.n;
  const size_t mk = ar.mark();
  const int kmax = std::min(MAX_SUM, std::max(1, q.ldy / 256));  // largest split pick_ksplit can return
  T* W = ar.get<T>((size_t)NB_QR * n * q.batch * kmax);
  T* W2 = ar.get<T>((size_t)NB_QR * n * q.batch);
  const T one = from_re<T>(1.0), mone = from_re<T>(-1.0), zer = zero<T>();
  const long long sW = (long long)NB_QR * n;  // one partial W
  for (int p = 0; p < q.npan; ++p) {
    const int k0 = p * NB_QR;
    if (k0 >= m) break;
    const int nb = std::min(NB_QR, n - k0);
    const int h = std::min(m, k0 + nb - 1 + q.band) - k0;
    T* Yp = q.Y + (long long)p * q.ldy * NB_QR;
    T* Tp = q.Tf + (long long)p * NB_QR * NB_QR;
    qr_panel<T>(st, m, n, q.band, M, ldm, sM, k0, nb, Yp, q.ldy, q.sY, Tp, q.sT, q.batch);
    const int nc = n - (k0 + nb);
    if (nc <= 0) continue;
    // W = Y^* C, split along K into ks partial products W_s
    GemmArgs<T> g;
    g.batch = q.batch;
    g.m = nb; g.n = nc; g.k = h; g.opA = OP_C; g.opB = OP_N;
    g.A = Yp; g.lda = q.ldy; g.sA = q.sY;
    g.B = M + k0 + (long long)(k0 + nb) * ldm; g.ldb = ldm; g.sB = sM;
    g.C = W; g.ldc = NB_QR; g.sC = sW;
    g.site = GS_QR_W;
    const int ks = resolve_ksplit(g, pick_ksplit(nb, nc, h, q.batch, 32));
    g.alpha = one; g.beta = zer;
    gemm(g, st);
    // W2 = T^* sum_s W_s   (T upper triangular: op(A)[i,k] = conj(T[k,i]) = 0 for k > i)
    GemmArgs<T> g2;
    g2.batch = q.batch;
    g2.nsum = ks;
    g2.m = nb; g2.n = nc; g2.k = nb; g2.opA = OP_C; g2.opB = OP_N;
    g2.A = Tp; g2.lda = nb; g2.sA = q.sT; g2.sAj = 0;
    g2.B = W; g2.ldb = NB_QR; g2.sB = sW * ks; g2.sBj = sW;
    g2.C = W2; g2.ldc = NB_QR; g2.sC = sW;
    g2.site = GS_QR_W2;
    g2.alpha = one; g2.beta = zer; g2.kflags = K_TO_ROW;
    gemm(g2, st);
    // C -= Y W2
    GemmArgs<T> g3;
    g3.batch = q.batch;
    g3.m = h; g3.n = nc; g3.k = nb; g3.opA = OP_N; g3.opB = OP_N;
    g3.A = Yp; g3.lda = q.ldy; g3.sA = q.sY;
    g3.B = W2; g3.ldb = NB_QR; g3.sB = (long long)NB_QR * n;
    g3.Cin = M + k0 + (long long)(k0 + nb) * ldm; g3.ldcin = ldm; g3.sCin = sM;
    g3.C = M + k0 + (long long)(k0 + nb) * ldm; g3.ldc = ldm; g3.sC = sM;
    g3.site = GS_QR_UPD;
    g3.alpha = mone; g3.beta = one;
    gemm(g3, st);
  }
  ar.release(mk);
}

template <class T>
void qr_form_q(cudaStream_t st, Arena& ar, const QRStore<T>& q, T* E, int lde, long long sE) {
  const int m = q.m, n = q.n;
  set_eye<T>(st, m, n, E, lde, sE, q.batch);
  const size_t mk = ar.mark();
  const int kmax = std::min(MAX_SUM, std::max(1, q.ldy / 256));
  T* W = ar.get<T>((size_t)NB_QR * n * q.batch * kmax);
  T* W2 = ar.get<T>((size_t)NB_QR * n * q.batch);
  const T one = from_re<T>(1.0), mone = from_re<T>(-1.0), zer = zero<T>();
  const long long sW = (long long)NB_QR * n;
  for (int p = q.npan - 1; p >= 0; --p) {
    const int k0 = p * NB_QR;
    if (k0 >= m) continue;
    const int nb = std::min(NB_QR, n - k0);
    const int h = std::min(m, k0 + nb - 1 + q.band) - k0;
    const int nc = n - k0;
    const T* Yp = q.Y + (long long)p * q.ldy * NB_QR;
    const T* Tp = q.Tf + (long long)p * NB_QR * NB_QR;
    T* Es = E + k0 + (long long)k0 * lde;
    GemmArgs<T> g;  // W = Y^* E_sub, split along K
    g.batch = q.batch;
    g.m = nb; g.n = nc; g.k = h; g.opA = OP_C; g.opB = OP_N;
    g.A = Yp; g.lda = q.ldy; g.sA = q.sY;
    g.B = Es; g.ldb = lde; g.sB = sE;
    g.C = W; g.ldc = NB_QR; g.sC = sW;
    g.site = GS_FQ_W;
    const int ks = resolve_ksplit(g, pick_ksplit(nb, nc, h, q.batch, 32));
    g.alpha = one; g.beta = zer;
    gemm(g, st);
    GemmArgs<T> g2;  // W2 = T sum_s W_s
    g2.batch = q.batch;
    g2.nsum = ks;
    g2.m = nb; g2.n = nc; g2.k = nb; g2.opA = OP_N; g2.opB = OP_N;
    g2.A = Tp; g2.lda = nb; g2.sA = q.sT; g2.sAj = 0;
    g2.B = W; g2.ldb = NB_QR; g2.sB = sW * ks; g2.sBj = sW;
    g2.C = W2; g2.ldc = NB_QR; g2.sC = sW;
    g2.site = GS_FQ_W2;
    g2.alpha = one; g2.beta = zer; g2.kflags = K_FROM_ROW;
    gemm(g2, st);
    GemmArgs<T> g3;  // E_sub -= Y W2
    g3.batch = q.batch;
    g3.m = h; g3.n = nc; g3.k = nb; g3.opA = OP_N; g3.opB = OP_N;
    g3.A = Yp; g3.lda = q.ldy; g3.sA = q.sY;
    g3.B = W2; g3.ldb = NB_QR; g3.sB = (long long)NB_QR * n;
    g3.Cin = Es; g3.ldcin = lde; g3.sCin = sE;
    g3.C = Es; g3.ldc = lde; g3.sC = sE;
    g3.site = GS_FQ_UPD;
    g3.alpha = mone; g3.beta = one;
    gemm(g3, st);
  }
  ar.release(mk);
}

template <class T>
void cholesky(cudaStream_t st, int n, T* Z, int ldz, long long sZ, T* Rinv, long long sR, int* info, int batch) {
  ZCSD_CUDA(cudaMemsetAsync(info, 0, sizeof(int) * batch, st));
  const T one = from_re<T>(1.0), mone = from_re<T>(-1.0), zer = zero<T>();
  for (int k0 = 0; k0 < n; k0 += NB_CHOL) {
    const int nb = std::min(NB_CHOL, n - k0);
    T* Rk = Rinv + (long long)k0 * NB_CHOL;
    potrf_inv<T>(st, n, Z, ldz, sZ, k0, nb, Rk, NB_CHOL, sR, info, batch);
    const int nc = n - (k0 + nb);
    if (nc <= 0) break;
    T* Zkr = Z + k0 + (long long)(k0 + nb) * ldz;
    // R[k, >k] = R_kk^{-*} Z[k, >k]   (in place: one row tile covers the block)
    GemmArgs<T> g;
    g.batch = batch;
    g.m = nb; g.n = nc; g.k = nb; g.opA = OP_C; g.opB = OP_N;
    g.A = Rk; g.lda = NB_CHOL; g.sA = sR;
    g.B = Zkr; g.ldb = ldz; g.sB = sZ;
    g.C = Zkr; g.ldc = ldz; g.sC = sZ;
    g.site = GS_CHOL_ROW;
    g.alpha = one; g.beta = zer; g.kflags = K_TO_ROW;
    gemm(g, st);
    // Z[>k, >k] -= R[k, >k]^* R[k, >k]  (tiles touching the upper triangle)
    GemmArgs<T> g2;
    g2.batch = batch;
    g2.m = nc; g2.n = nc; g2.k = nb; g2.opA = OP_C; g2.opB = OP_N;
    g2.A = Zkr; g2.lda = ldz; g2.sA = sZ;
    g2.B = Zkr; g2.ldb = ldz; g2.sB = sZ;
    T* Ztr = Z + (k0 + nb) + (long long)(k0 + nb) * ldz;
    g2.Cin = Ztr; g2.ldcin = ldz; g2.sCin = sZ;
    g2.C = Ztr; g2.ldc = ldz; g2.sC = sZ;
    g2.site = GS_CHOL_TRAIL;
    g2.alpha = mone; g2.beta = one; g2.uplo = 1;
    gemm(g2, st);
  }
}

template <class T>
void trsm_pair(cudaStream_t st, Arena& ar, int n, const T* X, int ldx, long long sX, int xdiv, const T* Z, int ldz,
               long long sZ, const T* Rinv, long long sR, T* Yt, T* Tt, int ldt, long long sT, int batch) {
  const size_t mk = ar.mark();
  const int kmax = std::min(MAX_SUM, std::max(1, n / 256));
  T* Tmp = ar.get<T>((size_t)n * NB_CHOL * batch * kmax);
  const long long sTmp = (long long)n * NB_CHOL;  // one partial
  const T one = from_re<T>(1.0), mone = from_re<T>(-1.0), zer = zero<T>();
  // forward: Yt[:, k] = (X[:, k] - Yt[:, <k] R[<k, k]) R_kk^{-1}
  for (int k0 = 0; k0 < n; k0 += NB_CHOL) {
    const int nb = std::min(NB_CHOL, n - k0);
    // Tmp_s = [s == 0] X[:, k] - Yt[:, K_s] R[K_s, k] over K chunks K_s of [0, k0)
    GemmArgs<T> g;
    g.batch = batch;
    g.m = n; g.n = nb; g.k = k0; g.opA = OP_N; g.opB = OP_N;
    g.A = Yt; g.lda = ldt; g.sA = sT;
    g.B = Z + (long long)k0 * ldz; g.ldb = ldz; g.sB = sZ;
    g.Cin = X + (long long)k0 * ldx; g.ldcin = ldx; g.sCin = sX; g.bdivC = xdiv;
    g.C = Tmp; g.ldc = n; g.sC = sTmp;
    g.site = GS_TRSM_F_UPD;
    g.alpha = mone; g.beta = one;
    if (k0 == 0) { g.k = 0; g.nsum = 0; }
    const int ks = resolve_ksplit(g, k0 > 0 ? pick_ksplit(n, nb, k0, batch, 64) : 1);
    gemm(g, st);
    // Yt[:, k] = (sum_s Tmp_s) R_kk^{-1}
    GemmArgs<T> g2;
    g2.batch = batch;
    g2.nsum = ks;
    g2.m = n; g2.n = nb; g2.k = nb; g2.opA = OP_N; g2.opB = OP_N;
    g2.A = Tmp; g2.lda = n; g2.sA = sTmp * ks; g2.sAj = sTmp;
    g2.B = Rinv + (long long)k0 * NB_CHOL; g2.ldb = NB_CHOL; g2.sB = sR;
    g2.C = Yt + (long long)k0 * ldt; g2.ldc = ldt; g2.sC = sT;
    g2.site = GS_TRSM_F_DIAG;
    g2.alpha = one; g2.beta = zer; g2.kflags = K_TO_COL;
    gemm(g2, st);
  }
  // backward: Tt[:, k] = (Yt[:, k] - Tt[:, >k] R[k, >k]^*) R_kk^{-*}
  const int nblk = ceil_div(n, NB_CHOL);
  for (int bk = nblk - 1; bk >= 0; --bk) {
    const int k0 = bk * NB_CHOL;
    const int nb = std::min(NB_CHOL, n - k0);
    const int ke = k0 + nb;
    GemmArgs<T> g;
    g.batch = batch;
    g.m = n; g.n = nb; g.k = n - ke; g.opA = OP_N; g.opB = OP_C;
    g.A = Tt + (long long)ke * ldt; g.lda = ldt; g.sA = sT;
    g.B = Z + k0 + (long long)ke * ldz; g.ldb = ldz; g.sB = sZ;
    g.Cin = Yt + (long long)k0 * ldt; g.ldcin = ldt; g.sCin = sT;
    g.C = Tmp; g.ldc = n; g.sC = sTmp;
    g.site = GS_TRSM_B_UPD;
    g.alpha = mone; g.beta = one;
    if (ke >= n) { g.k = 0; g.nsum = 0; }
    const int ks = resolve_ksplit(g, ke < n ? pick_ksplit(n, nb, n - ke, batch, 64) : 1);
    gemm(g, st);
    GemmArgs<T> g2;
    g2.batch = batch;
    g2.nsum = ks;
    g2.m = n; g2.n = nb; g2.k = nb; g2.opA = OP_N; g2.opB = OP_C;
    g2.A = Tmp; g2.lda = n; g2.sA = sTmp * ks; g2.sAj = sTmp;
    g2.B = Rinv + (long long)k0 * NB_CHOL; g2.ldb = NB_CHOL; g2.sB = sR;
    g2.C = Tt + (long long)k0 * ldt; g2.ldc = ldt; g2.sC = sT;
    g2.site = GS_TRSM_B_DIAG;
    g2.alpha = one; g2.beta = zer; g2.kflags = K_FROM_COL;
    gemm(g2, st);
  }
  ar.release(mk);
}

#define ZCSD_INST_L(T)                                                                                          \
  template QRStore<T> qr_alloc<T>(Arena&, int, int, int, int);                                                  \
  template void qr_factor<T>(cudaStream_t, Arena&, QRStore<T>&, T*, int, long long);                            \
  template void qr_form_q<T>(cudaStream_t, Arena&, const QRStore<T>&, T*, int, long long);                      \
  template void cholesky<T>(cudaStream_t, int, T*, int, long long, T*, long long, int*, int);                   \
  template void trsm_pair<T>(cudaStream_t, Arena&, int, const T*, int, long long, int, const T*, int, long long, \
                             const T*, long long, T*, T*, int, long long, int);

ZCSD_INST_L(double)
ZCSD_INST_L(z64)

}  // namespace zcsd
