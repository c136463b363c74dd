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

// Split-K factor of a product: the FP64-pipe choice `ks`, or, when the
// tensor-core path takes the product, its own choice (one CTA per SM there);
// both at most `cap`, the partial buffers the caller holds.
template <class T>
static int resolve_ksplit(GemmArgs<T>& g, int ks, int cap) {
  g.ksplit = std::max(1, std::min(ks, cap));
  GemmArgs<T> probe = g;
  probe.ksplit = 1;
  if constexpr (std::is_same<T, double>::value) {
    if (tc_will_handle(probe)) g.ksplit = tc_pick_ksplit(probe, cap);
  } else {
    if (tc_will_handle_complex(probe)) {
      GemmArgs<double> r;  // the real products it becomes: same tiles
      r.m = g.m; r.n = g.n; r.k = g.k; r.batch = g.batch;
      g.ksplit = tc_pick_ksplit(r, cap);
    }
  }
  return g.ksplit;
}

template <class T>
QRStore<T> qr_alloc(Arena& ar, int m, int n, int band, int batch) {
  QRStore<T> q;
  q.m = m; q.n = n; q.band = band; q.batch = batch;
  q.nbo = std::min(NB_OUT, ceil_div(n, NB_QR) * NB_QR);  // outer block width (small n: the whole matrix)
  q.npan = ceil_div(n, q.nbo);
  q.ldy = std::max(1, std::min(m, q.nbo - 1 + band));
  q.sY = (long long)q.npan * q.ldy * q.nbo;
  q.sT = (long long)q.npan * q.nbo * q.nbo;
  q.Y = ar.get<T>((size_t)q.sY * batch);
  q.Tf = ar.get<T>((size_t)q.sT * batch);
  return q;
}

// C <- (I - Y op(T) Y^*) C for `batch` problems: op(T) = T^* applies Q^* (the
// factorization sweep), op(T) = T applies Q (forming Q).  Y is h x nb with
// explicit zeros / unit diagonal, T is nb x nb upper triangular, C is h x nc.
// W = Y^* C is split along its long K = h range when its output is small.
template <class T>
static void wy_apply(cudaStream_t st, Arena& ar, int h, int nc, int nb, const T* Y, int ldy, long long sY,
                     const T* Tm, int ldt, long long sT, bool adjoint, T* C, int ldc, long long sC, int batch,
                     int site_w, int site_w2, int site_upd, int xrows = 0) {
  if (nc <= 0 || nb <= 0 || h <= 0) return;
  const int kcap = std::min(nb > NB_QR ? 4 : MAX_SUM, std::max(1, h / 256));
  const size_t mk = ar.mark();
  const long long sW = (long long)nb * nc;
  T* W = ar.get<T>((size_t)sW * batch * kcap);
  T* W2 = ar.get<T>((size_t)sW * batch);
  const T one = from_re<T>(1.0), mone = from_re<T>(-1.0), zer = zero<T>();
  GemmArgs<T> g;  // W_s = Y^* C over K chunk s
  g.batch = batch;
  g.m = nb; g.n = nc; g.k = h; g.opA = OP_C; g.opB = OP_N;
  g.A = Y; g.lda = ldy; g.sA = sY;
  g.B = C; g.ldb = ldc; g.sB = sC;
  g.C = W; g.ldc = nb; g.sC = sW;
  g.site = site_w;
  g.alpha = one; g.beta = zer;
  const int ks = resolve_ksplit(g, pick_ksplit(nb, nc, h, batch, nb <= 32 ? 32 : 64), kcap);
  gemm(g, st);
  sum_parts<T>(st, nb, nc, W, nb, sW, ks, batch);  // W_0 = sum_s W_s
  GemmArgs<T> g2;  // W2 = op(T) W_0
  g2.batch = batch;
  g2.m = nb; g2.n = nc; g2.k = nb;
  g2.opA = adjoint ? OP_C : OP_N;
  g2.kflags = adjoint ? K_TO_ROW : K_FROM_ROW;  // T upper triangular
  g2.A = Tm; g2.lda = ldt; g2.sA = sT;
  g2.B = W; g2.ldb = nb; g2.sB = sW * ks;
  g2.C = W2; g2.ldc = nb; g2.sC = sW;
  g2.site = site_w2;
  g2.alpha = one; g2.beta = zer;
  gemm(g2, st);
  // C -= Y W2; for a stacked [X; sqrt(c) I] the rows of the X block and the
  // rows below it are separate products (sites GS_QR_UPD_X and site_upd)
  const int hx = std::min(std::max(xrows, 0), h);
  for (int part = 0; part < 2; ++part) {
    const int r0 = part == 0 ? 0 : hx, r1 = part == 0 ? hx : h;
    if (r1 <= r0) continue;
    GemmArgs<T> g3;
    g3.batch = batch;
    g3.m = r1 - r0; g3.n = nc; g3.k = nb; g3.opA = OP_N; g3.opB = OP_N;
    g3.A = Y + r0; g3.lda = ldy; g3.sA = sY;
    g3.B = W2; g3.ldb = nb; g3.sB = sW;
    g3.Cin = C + r0; g3.ldcin = ldc; g3.sCin = sC;
    g3.C = C + r0; g3.ldc = ldc; g3.sC = sC;
    g3.site = part == 0 ? GS_QR_UPD_X : site_upd;
    g3.kbal = part == 0 ? 0 : 1;  // rows of the size of sqrt(c): balance k on the tensor cores
    g3.alpha = mone; g3.beta = one;
    gemm(g3, st);
  }
  ar.release(mk);
}

// Two-level blocked Householder QR: outer blocks of NB_OUT columns, each
// factored as NB_QR-wide panels (panel kernel + updates inside the block);
// the block's compact-WY factor T (NB_OUT x NB_OUT) is merged from the panel
// factors, T_{<i, i} = -T_{<i} (Y_{<i}^* Y_i) T_i (Q = Q_{<i} Q_i), and the
// trailing matrix is updated once per outer block.
template <class T>
void qr_factor(cudaStream_t st, Arena& ar, QRStore<T>& q, T* M, int ldm, long long sM) {
  const int m = q.m, n = q.n;
  const size_t mk = ar.mark();
  T* Tin = ar.get<T>((size_t)NB_QR * NB_QR * q.batch);
  const int NBO = q.nbo;
  const int scap = std::min(MAX_SUM, std::max(1, q.ldy / 256));
  T* S = ar.get<T>((size_t)NBO * NBO * q.batch * scap);  // split-K parts of the Gram matrix Y_b^* Y_b
  T* S2 = ar.get<T>((size_t)NBO * NB_QR * q.batch);
  const long long sS = (long long)NBO * NBO, sS2 = (long long)NBO * NB_QR;
  const T one = from_re<T>(1.0), mone = from_re<T>(-1.0), zer = zero<T>();
  for (int ob = 0; ob < q.npan; ++ob) {
    const int K0 = ob * NBO;
    if (K0 >= m) break;
    const int nbo = std::min(NBO, n - K0);
    const int hb = std::min(m, K0 + nbo - 1 + q.band) - K0;
    T* Yb = q.Y + (long long)ob * q.ldy * NBO;
    T* Tb = q.Tf + (long long)ob * NBO * NBO;
    ZCSD_CUDA(cudaMemset2DAsync(Yb, sizeof(T) * q.sY, 0, sizeof(T) * (size_t)q.ldy * NBO, q.batch, st));
    ZCSD_CUDA(cudaMemset2DAsync(Tb, sizeof(T) * q.sT, 0, sizeof(T) * (size_t)NBO * NBO, q.batch, st));
    for (int c0 = 0; c0 < nbo; c0 += NB_QR) {
      const int k0 = K0 + c0;
      if (k0 >= m) break;
      const int nb = std::min(NB_QR, nbo - c0);
      T* Yi = Yb + c0 + (long long)c0 * q.ldy;
      T* Ti = Tb + c0 + (long long)c0 * NBO;
      qr_panel<T>(st, m, n, q.band, M, ldm, sM, k0, nb, Yi, q.ldy, q.sY, Tin, (long long)NB_QR * NB_QR, q.batch);
      axpby<T>(st, nb, nb, 1.0, Tin, nb, (long long)NB_QR * NB_QR, 0.0, Ti, NBO, q.sT, q.batch);
      // update the rest of this outer block with panel i
      const int nc_in = K0 + nbo - (k0 + nb);
      if (nc_in > 0) {
        const int hi = std::min(m, k0 + nb - 1 + q.band) - k0;
        wy_apply<T>(st, ar, hi, nc_in, nb, Yi, q.ldy, q.sY, Ti, NBO, q.sT, true, M + k0 + (long long)(k0 + nb) * ldm,
                    ldm, sM, q.batch, GS_QR_W, GS_QR_W2, GS_QR_UPD, q.xrows - k0);
      }
    }
    // merge the panel factors into the block's T: one Gram matrix
    // S = Y_b^* Y_b (split along its long K), then for each panel i,
    // T_{<i, i} = -T_{<i} S[<i, i] T_i  (Q = Q_{<i} Q_i)
    if (nbo > NB_QR) {
      GemmArgs<T> g;
      g.batch = q.batch;
      g.m = nbo; g.n = nbo; g.k = hb; g.opA = OP_C; g.opB = OP_N;
      g.A = Yb; g.lda = q.ldy; g.sA = q.sY;
      g.B = Yb; g.ldb = q.ldy; g.sB = q.sY;
      g.C = S; g.ldc = NBO; g.sC = sS;
      g.alpha = one; g.beta = zer; g.site = GS_TMERGE;
      const int ks = resolve_ksplit(g, pick_ksplit(nbo, nbo, hb, q.batch, 64), scap);
      gemm(g, st);
      sum_parts<T>(st, nbo, nbo, S, NBO, sS, ks, q.batch);  // S_0 = sum_s S_s
      for (int c0 = NB_QR; c0 < nbo; c0 += NB_QR) {
        const int nb = std::min(NB_QR, nbo - c0);
        T* Ti = Tb + c0 + (long long)c0 * NBO;
        GemmArgs<T> g2;  // S2 = T_{<i} S_0[<i, i]
        g2.batch = q.batch;
        g2.m = c0; g2.n = nb; g2.k = c0; g2.opA = OP_N; g2.opB = OP_N;
        g2.A = Tb; g2.lda = NBO; g2.sA = q.sT;
        g2.B = S + (long long)c0 * NBO; g2.ldb = NBO; g2.sB = sS * ks;
        g2.C = S2; g2.ldc = NBO; g2.sC = sS2;
        g2.alpha = one; g2.beta = zer; g2.kflags = K_FROM_ROW; g2.site = GS_TMERGE;
        gemm(g2, st);
        GemmArgs<T> g3;  // T_{<i, i} = -S2 T_i
        g3.batch = q.batch;
        g3.m = c0; g3.n = nb; g3.k = nb; g3.opA = OP_N; g3.opB = OP_N;
        g3.A = S2; g3.lda = NBO; g3.sA = sS2;
        g3.B = Ti; g3.ldb = NBO; g3.sB = q.sT;
        g3.C = Tb + (long long)c0 * NBO; g3.ldc = NBO; g3.sC = q.sT;
        g3.alpha = mone; g3.beta = zer; g3.kflags = K_TO_COL; g3.site = GS_TMERGE;
        gemm(g3, st);
      }
    }
    const int nc = n - (K0 + nbo);
    if (nc > 0)
      wy_apply<T>(st, ar, hb, nc, nbo, Yb, q.ldy, q.sY, Tb, NBO, q.sT, true, M + K0 + (long long)(K0 + nbo) * ldm,
                  ldm, sM, q.batch, GS_QR_W, GS_QR_W2, GS_QR_UPD, q.xrows - K0);
  }
  ar.release(mk);
}

template <class T>
void qr_form_q(cudaStream_t st, Arena& ar, const QRStore<T>& q, T* E, int lde, long long sE) {
  const int m = q.m, n = q.n;
  set_eye<T>(st, m, n, E, lde, sE, q.batch);
  const int NBO = q.nbo;
  for (int ob = q.npan - 1; ob >= 0; --ob) {
    const int K0 = ob * NBO;
    if (K0 >= m) continue;
    const int nbo = std::min(NBO, n - K0);
    const int hb = std::min(m, K0 + nbo - 1 + q.band) - K0;
    const T* Yb = q.Y + (long long)ob * q.ldy * NBO;
    const T* Tb = q.Tf + (long long)ob * NBO * NBO;
    wy_apply<T>(st, ar, hb, n - K0, nbo, Yb, q.ldy, q.sY, Tb, NBO, q.sT, false, E + K0 + (long long)K0 * lde, lde,
                sE, q.batch, GS_FQ_W, GS_FQ_W2, GS_FQ_UPD);
  }
}

// Rows [r0, r1) of R times columns [j0, j1): Z[r0:r1, j0:j1] <- R11^{-*}
// Z[r0:r1, j0:j1] with R11 = R[r0:r1, r0:r1] (its lower-triangular adjoint
// solved recursively: X1 = Ra^{-*} Z1, Z2 -= Rb^* X1, X2 = Rc^{-*} Z2); leaves
// multiply in place by the inverted diagonal block (one row tile covers it).
template <class T>
static void chol_row_rec(cudaStream_t st, int r0, int r1, int j0, int j1, T* Z, int ldz, long long sZ, const T* Rinv,
                         long long sR, int batch) {
  const int w = r1 - r0;
  const T one = from_re<T>(1.0), mone = from_re<T>(-1.0), zer = zero<T>();
  T* Zr = Z + r0 + (long long)j0 * ldz;
  if (w <= NB_CHOL) {
    GemmArgs<T> g;
    g.batch = batch;
    g.m = w; g.n = j1 - j0; g.k = w; g.opA = OP_C; g.opB = OP_N;
    g.A = Rinv + (long long)r0 * NB_CHOL; g.lda = NB_CHOL; g.sA = sR;
    g.B = Zr; g.ldb = ldz; g.sB = sZ;
    g.C = Zr; g.ldc = ldz; g.sC = sZ;
    g.site = GS_CHOL_ROW;
    g.alpha = one; g.beta = zer; g.kflags = K_TO_ROW;
    gemm(g, st);
    return;
  }
  const int rm = r0 + ceil_div(w / 2, NB_CHOL) * NB_CHOL;
  chol_row_rec(st, r0, rm, j0, j1, Z, ldz, sZ, Rinv, sR, batch);
  GemmArgs<T> g;  // Z[rm:r1, j0:j1] -= R[r0:rm, rm:r1]^* X[r0:rm, j0:j1]
  g.batch = batch;
  g.m = r1 - rm; g.n = j1 - j0; g.k = rm - r0; g.opA = OP_C; g.opB = OP_N;
  g.A = Z + r0 + (long long)rm * ldz; g.lda = ldz; g.sA = sZ;
  g.B = Zr; g.ldb = ldz; g.sB = sZ;
  T* Z2 = Z + rm + (long long)j0 * ldz;
  g.Cin = Z2; g.ldcin = ldz; g.sCin = sZ;
  g.C = Z2; g.ldc = ldz; g.sC = sZ;
  g.site = GS_CHOL_ROW;
  g.alpha = mone; g.beta = one;
  gemm(g, st);
  chol_row_rec(st, rm, r1, j0, j1, Z, ldz, sZ, Rinv, sR, batch);
}

// Recursive Cholesky Z = R^* R on [c0, c1): factor the leading half, solve
// its rows R12 = R11^{-*} Z12, update Z22 -= R12^* R12 (one product with K =
// half the width), factor Z22.  Leaves of NB_CHOL columns factor and invert
// the diagonal block.
template <class T>
static void chol_rec(cudaStream_t st, int n, int c0, int c1, T* Z, int ldz, long long sZ, T* Rinv, long long sR,
                     int* info, int batch) {
  const int w = c1 - c0;
  if (w <= NB_CHOL) {
    potrf_inv<T>(st, n, Z, ldz, sZ, c0, w, Rinv + (long long)c0 * NB_CHOL, NB_CHOL, sR, info, batch);
    return;
  }
  const int mid = c0 + ceil_div(w / 2, NB_CHOL) * NB_CHOL;
  chol_rec(st, n, c0, mid, Z, ldz, sZ, Rinv, sR, info, batch);
  chol_row_rec(st, c0, mid, mid, c1, Z, ldz, sZ, Rinv, sR, batch);
  GemmArgs<T> g;  // Z22 -= R12^* R12  (tiles touching the upper triangle)
  g.batch = batch;
  g.m = c1 - mid; g.n = c1 - mid; g.k = mid - c0; g.opA = OP_C; g.opB = OP_N;
  T* R12 = Z + c0 + (long long)mid * ldz;
  g.A = R12; g.lda = ldz; g.sA = sZ;
  g.B = R12; g.ldb = ldz; g.sB = sZ;
  T* Z22 = Z + mid + (long long)mid * ldz;
  g.Cin = Z22; g.ldcin = ldz; g.sCin = sZ;
  g.C = Z22; g.ldc = ldz; g.sC = sZ;
  g.site = GS_CHOL_TRAIL;
  g.alpha = from_re<T>(-1.0); g.beta = from_re<T>(1.0); g.uplo = 1;
  gemm(g, st);
  chol_rec(st, n, mid, c1, Z, ldz, sZ, Rinv, sR, info, batch);
}

template <class T>
void cholesky(cudaStream_t st, int n, T* Z, int ldz, long long sZ, T* Rinv, long long sR, int* info, int batch) {
  ZCSD_CUDA(cudaMemsetAsync(info, 0, sizeof(int) * batch, st));
  chol_rec(st, n, 0, n, Z, ldz, sZ, Rinv, sR, info, batch);
}

// Recursive right-side triangular solves on column ranges [c0, c1) aligned to
// NB_CHOL: Y R = X splits R = [R11 R12; 0 R22] into Y1 = X1 R11^{-1},
// X2 -= Y1 R12, Y2 = X2 R22^{-1}; leaves multiply by the inverted diagonal
// blocks.  The off-diagonal updates are n x (w/2) x (w/2) products.
template <class T>
static void trsm_fwd_rec(cudaStream_t st, int n, int c0, int c1, T* Yt, int ldt, long long sT, const T* Z, int ldz,
                         long long sZ, const T* Rinv, long long sR, T* Tmp, int batch) {
  const int w = c1 - c0;
  const T one = from_re<T>(1.0), mone = from_re<T>(-1.0), zer = zero<T>();
  if (w <= NB_CHOL) {
    axpby<T>(st, n, w, 1.0, Yt + (long long)c0 * ldt, ldt, sT, 0.0, Tmp, n, (long long)n * NB_CHOL, batch);
    GemmArgs<T> g;  // Y[:, c0:c1] = X[:, c0:c1] R_kk^{-1}
    g.batch = batch;
    g.m = n; g.n = w; g.k = w; g.opA = OP_N; g.opB = OP_N;
    g.A = Tmp; g.lda = n; g.sA = (long long)n * NB_CHOL;
    g.B = Rinv + (long long)c0 * NB_CHOL; g.ldb = NB_CHOL; g.sB = sR;
    g.C = Yt + (long long)c0 * ldt; g.ldc = ldt; g.sC = sT;
    g.alpha = one; g.beta = zer; g.kflags = K_TO_COL; g.site = GS_TRSM_F_DIAG;
    gemm(g, st);
    return;
  }
  const int mid = c0 + ceil_div(w / 2, NB_CHOL) * NB_CHOL;
  trsm_fwd_rec(st, n, c0, mid, Yt, ldt, sT, Z, ldz, sZ, Rinv, sR, Tmp, batch);
  GemmArgs<T> g;  // X2 -= Y1 R12
  g.batch = batch;
  g.m = n; g.n = c1 - mid; g.k = mid - c0; g.opA = OP_N; g.opB = OP_N;
  g.A = Yt + (long long)c0 * ldt; g.lda = ldt; g.sA = sT;
  g.B = Z + c0 + (long long)mid * ldz; g.ldb = ldz; g.sB = sZ;
  g.Cin = Yt + (long long)mid * ldt; g.ldcin = ldt; g.sCin = sT;
  g.C = Yt + (long long)mid * ldt; g.ldc = ldt; g.sC = sT;
  g.alpha = mone; g.beta = one; g.site = GS_TRSM_F_UPD;
  gemm(g, st);
  trsm_fwd_rec(st, n, mid, c1, Yt, ldt, sT, Z, ldz, sZ, Rinv, sR, Tmp, batch);
}

// T R^* = Y with R^* lower triangular: T2 = Y2 R22^{-*}, Y1 -= T2 R12^*, T1 = Y1 R11^{-*}.
template <class T>
static void trsm_bwd_rec(cudaStream_t st, int n, int c0, int c1, T* Tt, int ldt, long long sT, const T* Z, int ldz,
                         long long sZ, const T* Rinv, long long sR, T* Tmp, int batch) {
  const int w = c1 - c0;
  const T one = from_re<T>(1.0), mone = from_re<T>(-1.0), zer = zero<T>();
  if (w <= NB_CHOL) {
    axpby<T>(st, n, w, 1.0, Tt + (long long)c0 * ldt, ldt, sT, 0.0, Tmp, n, (long long)n * NB_CHOL, batch);
    GemmArgs<T> g;  // T[:, c0:c1] = Y[:, c0:c1] R_kk^{-*}
    g.batch = batch;
    g.m = n; g.n = w; g.k = w; g.opA = OP_N; g.opB = OP_C;
    g.A = Tmp; g.lda = n; g.sA = (long long)n * NB_CHOL;
    g.B = Rinv + (long long)c0 * NB_CHOL; g.ldb = NB_CHOL; g.sB = sR;
    g.C = Tt + (long long)c0 * ldt; g.ldc = ldt; g.sC = sT;
    g.alpha = one; g.beta = zer; g.kflags = K_FROM_COL; g.site = GS_TRSM_B_DIAG;
    gemm(g, st);
    return;
  }
  const int mid = c0 + ceil_div(w / 2, NB_CHOL) * NB_CHOL;
  trsm_bwd_rec(st, n, mid, c1, Tt, ldt, sT, Z, ldz, sZ, Rinv, sR, Tmp, batch);
  GemmArgs<T> g;  // Y1 -= T2 R12^*
  g.batch = batch;
  g.m = n; g.n = mid - c0; g.k = c1 - mid; g.opA = OP_N; g.opB = OP_C;
  g.A = Tt + (long long)mid * ldt; g.lda = ldt; g.sA = sT;
  g.B = Z + c0 + (long long)mid * ldz; g.ldb = ldz; g.sB = sZ;
  g.Cin = Tt + (long long)c0 * ldt; g.ldcin = ldt; g.sCin = sT;
  g.C = Tt + (long long)c0 * ldt; g.ldc = ldt; g.sC = sT;
  g.alpha = mone; g.beta = one; g.site = GS_TRSM_B_UPD;
  gemm(g, st);
  trsm_bwd_rec(st, n, c0, mid, Tt, ldt, sT, Z, ldz, sZ, Rinv, sR, Tmp, batch);
}

template <class T>
void trsm_pair(cudaStream_t st, Arena& ar, int n, const T* X, int ldx, long long sX, int xdiv, const T* Z, int ldz,
               long long sZ, const T* Rinv, long long sR, T* Yt, T* Tt, int ldt, long long sT, int batch) {
  const size_t mk = ar.mark();
  T* Tmp = ar.get<T>((size_t)n * NB_CHOL * batch);
  // Yt = X (problem b reads X_{b / xdiv}), then solve in place
  const int P = batch / xdiv;
  for (int j = 0; j < xdiv; ++j)
    axpby<T>(st, n, n, 1.0, X, ldx, sX, 0.0, Yt + (long long)j * sT, ldt, sT * xdiv, P);
  trsm_fwd_rec(st, n, 0, n, Yt, ldt, sT, Z, ldz, sZ, Rinv, sR, Tmp, batch);
  axpby<T>(st, n, n, 1.0, Yt, ldt, sT, 0.0, Tt, ldt, sT, batch);
  trsm_bwd_rec(st, n, 0, n, Tt, ldt, sT, Z, ldz, sZ, Rinv, sR, Tmp, batch);
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
