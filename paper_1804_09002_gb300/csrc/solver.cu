// Zolo-pd (Section 5), Zolo-eig (Section 5) and the CS decomposition driver
// (Algorithms 1-3), plus the C ABI declared in include/zolo_csd.h.
#include <chrono>
#include <cstdlib>
#include <cstring>
#include <new>
#include <vector>

#include "../../include/zolo_csd.h"
#include "solver.h"
#include "tc_gemm.h"

namespace zcsd {


// ---------------------------------------------------------------- small kernels
namespace {

template <class T>
__global__ void diag_phase_kernel(int n, const T* R, int ldr, T* d) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const T r = R[i + (long long)i * ldr];
    const double a = sqrt(abs2(r));
    d[i] = (a > 0.0) ? scal(1.0 / a, r) : from_re<T>(1.0);
  }
}

// Y[:, j] = X[:, j] * d1[j] * conj(d2[j])
template <class T>
__global__ void scale_cols_phase_kernel(int m, int n, const T* X, int ldx, const T* d1, const T* d2, T* Y, int ldy) {
  const long long total = (long long)m * n;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(t % m), j = (int)(t / m);
    Y[i + (long long)j * ldy] = mul(X[i + (long long)j * ldx], mul(d1[j], conj_(d2[j])));
  }
}

// D = conj(d1_i) R1[i,j] - conj(d2_i) R2[i,j] on the upper triangle, 0 below
template <class T>
__global__ void rdiff_kernel(int n, const T* R1, int ld1, const T* d1, const T* R2, int ld2, const T* d2, T* D) {
  const long long total = (long long)n * n;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(t % n), j = (int)(t / n);
    T v = zero<T>();
    if (i <= j) v = sub(cmul(d1[i], R1[i + (long long)j * ld1]), cmul(d2[i], R2[i + (long long)j * ld2]));
    D[t] = v;
  }
}

// B = H2 - H1 + mu (I - G), G = A1^* A1 + A2^* A2 (G may be null when mu = 0)
template <class T>
__global__ void form_b_kernel(int n, const T* H, long long sH, const T* G, double mu, T* B) {
  const long long total = (long long)n * n;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(t % n), j = (int)(t / n);
    T v = sub(H[sH + t], H[t]);
    if (mu != 0.0) {
      T im = scal(-1.0, G[t]);
      if (i == j) im = add(im, from_re<T>(1.0));
      v = add(v, scal(mu, im));
    }
    B[t] = v;
  }
}

__global__ void zero_tail_kernel(int n, int r, double* theta) {
  for (int i = r + blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) theta[i] = 0.0;
}

int grid_for(long long total) { return (int)std::min<long long>((total + 255) / 256, 152 * 8); }

}  // namespace

const Plan& get_plan(Ctx& cx) {
  if (!cx.plan_ready) {
    Plan& p = cx.plan;
    p.steps = zolo_plan(EPS_ZOLO, R_MAX, 4, p.r, p.ell);
    for (int s = 0; s < p.steps; ++s) {
      double next;
      zolo_coeffs(p.ell[s], p.r[s], p.c[s], p.a[s], &p.mhat[s], &next);
      for (int j = 0; j < p.r[s]; ++j) {
        p.sqrtc[s][j] = std::sqrt(p.c[s][2 * j]);
        p.w[s][j] = p.mhat[s] * p.a[s][j] / p.sqrtc[s][j];
      }
    }
    cx.plan_ready = true;
  }
  return cx.plan;
}

void d2h(Ctx& cx, void* dst, const void* src, size_t bytes) {
  ZCSD_CUDA(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToHost, cx.stream));
  ZCSD_CUDA(cudaStreamSynchronize(cx.stream));
}

// ---------------------------------------------------------------- Zolo-pd

// W_p = Zolo-pd polar factor of X0_p (p < P), X0 with ||X0_p||_2 <= 1 (ld n,
// stride n*n).  W may alias nothing else.  Section 5: iterates
// X_{k+1} = M (X_k + sum_j a_j X_k (X_k^* X_k + c_{2j-1} I)^{-1}); the first
// iteration in QR form (X (X^*X + cI)^{-1} = Q1 Q2^* / sqrt(c) for
// [X; sqrt(c) I] = [Q1; Q2] R), later ones in Cholesky form.
template <class T>
void zolo_pd(Ctx& cx, Arena& ar, int n, int P, const T* X0, T* W, PolarDiag* pd, int stop_after,
             int reduced_slices, bool sync_free) {
  cudaStream_t st = cx.stream;
  const Plan& pl = get_plan(cx);
  const int steps = (stop_after > 0) ? std::min(stop_after, pl.steps) : pl.steps;
  const long long nn = (long long)n * n;
  const size_t mk = ar.mark();
  T* Xa = ar.get<T>(nn * P);
  T* Xb = ar.get<T>(nn * P);
  axpby<T>(st, n, n, 1.0, X0, n, nn, 0.0, Xa, n, nn, P);
  T* X = Xa;
  T* Xn = Xb;
  const T one = from_re<T>(1.0), mone = from_re<T>(-1.0), zer = zero<T>();
  for (int s = 0; s < steps; ++s) {
    const int r = pl.r[s];
    bool use_qr = (s == 0);
    if (pd) pd->iters += 1;
    for (int attempt = 0; attempt < 2; ++attempt) {
      const size_t mk2 = ar.mark();
      if (use_qr) {
        // ---- QR form on the stacked [X; sqrt(c_{2j-1}) I], 2n x n, P*r problems
        const int m2 = 2 * n;
        const long long sM = (long long)m2 * n;
        T* M = ar.get<T>(sM * P * r);
        T* E = ar.get<T>(sM * P * r);
        stack_terms<T>(st, n, X, n, nn, pl.sqrtc[s], r, M, m2, sM, P);
        QRStore<T> q = qr_alloc<T>(ar, m2, n, n + 1, P * r);
        q.xrows = n;
        qr_factor<T>(st, ar, q, M, m2, sM);
        qr_form_q<T>(st, ar, q, E, m2, sM);
        // X_new = mhat X + sum_j (mhat a_j / sqrt(c_j)) Q1_j Q2_j^*   (Q2 upper triangular)
        GemmArgs<T> g;
        g.batch = P;
        g.m = n; g.n = n; g.k = n; g.opA = OP_N; g.opB = OP_C;
        g.A = E; g.lda = m2; g.sA = sM * r; g.sAj = sM;
        g.B = E + n; g.ldb = m2; g.sB = sM * r; g.sBj = sM;
        g.nsum = r;
        for (int j = 0; j < r; ++j) g.w[j] = pl.w[s][j];
        g.Cin = X; g.ldcin = n; g.sCin = nn;
        g.C = Xn; g.ldc = n; g.sC = nn;
        g.alpha = one; g.beta = from_re<T>(pl.mhat[s]);
        g.kflags = K_FROM_COL;
        g.site = GS_ZOLO_COMBINE;
        gemm(g, st);
        ar.release(mk2);
        break;
      }
      // ---- Cholesky form: Z_j = X^* X + c_{2j-1} I = R^* R, T_j = X R^{-1} R^{-*}
      // X is well conditioned here (its singular values lie in [l_s, 1]);
      // with reduced_slices the Gram and triangular-solve products run with
      // fewer BF16 slices, the Cholesky factorizations themselves do not
      struct ReducedScope {
        unsigned sites;
        int slices;
        ReducedScope(int rs) : sites(t_tc.reduced_sites), slices(t_tc.reduced_slices) {
          if (rs == 5 || rs == 6) {
            t_tc.reduced_sites = (1u << GS_GRAM) | (1u << GS_TRSM_F_UPD) | (1u << GS_TRSM_F_DIAG) |
                                 (1u << GS_TRSM_B_UPD) | (1u << GS_TRSM_B_DIAG);
            t_tc.reduced_slices = rs;
          }
        }
        ~ReducedScope() {
          t_tc.reduced_sites = sites;
          t_tc.reduced_slices = slices;
        }
      } reduced_scope(reduced_slices);
      T* G = ar.get<T>(nn * P);
      T* Z = ar.get<T>(nn * P * r);
      T* Rinv = ar.get<T>((size_t)NB_CHOL * n * P * r);
      T* Yt = ar.get<T>(nn * P * r);
      T* Tt = ar.get<T>(nn * P * r);
      int* info = ar.get<int>(P * r);
      GemmArgs<T> g;
      g.batch = P;
      g.m = n; g.n = n; g.k = n; g.opA = OP_C; g.opB = OP_N;
      g.A = X; g.lda = n; g.sA = nn;
      g.B = X; g.ldb = n; g.sB = nn;
      g.C = G; g.ldc = n; g.sC = nn;
      g.alpha = one; g.beta = zer; g.uplo = 1;
      g.site = GS_GRAM;
      gemm(g, st);
      double shifts[R_MAX];
      for (int j = 0; j < r; ++j) shifts[j] = pl.c[s][2 * j];
      shift_terms<T>(st, n, G, n, nn, shifts, r, Z, n, nn, P);
      cholesky<T>(st, n, Z, n, nn, Rinv, (long long)NB_CHOL * n, info, P * r);
      bool ok = true;
      if (!sync_free) {
        d2h(cx, cx.hs.i, info, sizeof(int) * P * r);
        for (int q = 0; q < P * r; ++q) ok = ok && (cx.hs.i[q] == 0);
      }
      if (!ok) {
        // non-positive pivot: redo this iteration in QR form
        ar.release(mk2);
        use_qr = true;
        if (pd) pd->chol_fallback += 1;
        continue;
      }
      trsm_pair<T>(st, ar, n, X, n, nn, r, Z, n, nn, Rinv, (long long)NB_CHOL * n, Yt, Tt, n, nn, P * r);
      double aa[R_MAX];
      for (int j = 0; j < r; ++j) aa[j] = pl.a[s][j];
      sum_terms<T>(st, n, pl.mhat[s], X, n, nn, aa, r, Tt, n, nn, Xn, n, nn, P);
      ar.release(mk2);
      break;
    }
    std::swap(X, Xn);
    (void)mone;
  }
  axpby<T>(st, n, n, 1.0, X, n, nn, 0.0, W, n, nn, P);
  ar.release(mk);
}

template void zolo_pd<double>(Ctx&, Arena&, int, int, const double*, double*, PolarDiag*, int, int, bool);
template void zolo_pd<z64>(Ctx&, Arena&, int, int, const z64*, z64*, PolarDiag*, int, int, bool);

// ---------------------------------------------------------------- CSD
template <class T>
int csd_impl(Ctx& cx, Arena& ar, int n, const T* A1, int lda1, const T* A2, int lda2, T* U1, int ldu1, T* U2,
             int ldu2, T* V1, int ldv1, double* theta, int* rank_out, csd_info* info) {
  cudaStream_t st = cx.stream;
  const long long nn = (long long)n * n;
  const Plan& pl = get_plan(cx);
  T* Apk = ar.get<T>(2 * nn);   // [A1 | A2] packed, ld n
  T* W = ar.get<T>(2 * nn);
  T* H = ar.get<T>(2 * nn);
  T* Bm = ar.get<T>(nn);
  T* V = ar.get<T>(nn);
  T* Ut = ar.get<T>(2 * nn);
  double* lam = ar.get<double>(n);
  double* dv = ar.get<double>(4 * n + 64);
  double* scratch = ar.get<double>(304 * 4);
  int* perm = ar.get<int>(n);
  double* sc = dv + 4 * n;
  axpby<T>(st, n, n, 1.0, A1, lda1, 0, 0.0, Apk, n, 0, 1);
  axpby<T>(st, n, n, 1.0, A2, lda2, 0, 0.0, Apk + nn, n, 0, 1);
  // ---- input checks and rank (remark (vi): ||A||_F^2 ~ rank)
  count_nonfinite<T>(st, n, 2 * n, Apk, n, sc, scratch);
  fro2<T>(st, n, n, Apk, n, nn, 0.0, sc + 1, 2, scratch);
  d2h(cx, cx.hs.d, sc, 3 * sizeof(double));
  if (cx.hs.d[0] != 0.0) return CSD_ERR_NONFINITE;
  const double fro = cx.hs.d[1] + cx.hs.d[2];
  int r = (int)std::floor(fro + 0.5);
  r = std::max(0, std::min(n, r));
  const double mu = (r == n) ? 0.0 : 2.0;
  if (info) {
    info->rank = r;
    info->mu = mu;
    info->zolo_iters = pl.steps;
    for (int s = 0; s < 4; ++s) {
      info->r_terms[s] = s < pl.steps ? pl.r[s] : 0;
      info->ell[s] = s < pl.steps ? pl.ell[s] : 0.0;
    }
  }
  // ---- lines 1-2: W_i H_i = A_i (both polar decompositions in one batch)
  PolarDiag pd;
  zolo_pd<T>(cx, ar, n, 2, Apk, W, &pd, 0, (cx.mixed_scope & 1u) ? cx.mixed_slices : 0);
  const T one = from_re<T>(1.0), zer = zero<T>();
  {
    GemmArgs<T> g;  // H_i = sym(W_i^* A_i)
    g.batch = 2;
    g.m = n; g.n = n; g.k = n; g.opA = OP_C; g.opB = OP_N;
    g.A = W; g.lda = n; g.sA = nn;
    g.B = Apk; g.ldb = n; g.sB = nn;
    g.C = H; g.ldc = n; g.sC = nn;
    g.alpha = one; g.beta = zer;
    g.site = GS_H;
    gemm(g, st);
    symmetrize<T>(st, n, H, n, nn, H, n, nn, 2);
  }
  // ---- orthogonality of W_i; Algorithm 2 where W_i is not orthonormal
  {
    const size_t mk = ar.mark();
    T* Gw = ar.get<T>(2 * nn);
    GemmArgs<T> g;
    g.batch = 2;
    g.m = n; g.n = n; g.k = n; g.opA = OP_C; g.opB = OP_N;
    g.A = W; g.lda = n; g.sA = nn;
    g.B = W; g.ldb = n; g.sB = nn;
    g.C = Gw; g.ldc = n; g.sC = nn;
    g.alpha = one; g.beta = zer;
    g.site = GS_ORTH;
    gemm(g, st);
    fro2<T>(st, n, n, Gw, n, nn, 1.0, sc + 4, 2, scratch);
    d2h(cx, cx.hs.d, sc + 4, 2 * sizeof(double));
    ar.release(mk);
  }
  const double orth[2] = {std::sqrt(cx.hs.d[0]), std::sqrt(cx.hs.d[1])};
  int status = CSD_OK;
  if (info) {
    info->orth_err[0] = orth[0];
    info->orth_err[1] = orth[1];
    info->chol_fallback = pd.chol_fallback;
  }
  // Algorithm 2, lines 2-3, for block i: A_i = Q_i R_i, H_i = Q~ R~,
  // W_i = Q_i Q~^* (diag(R) >= 0); H_i is kept
  auto alg2 = [&](int i) {
    const size_t mk = ar.mark();
    T* Ma = ar.get<T>(nn);
    T* Mh = ar.get<T>(nn);
    T* Qa = ar.get<T>(nn);
    T* Qh = ar.get<T>(nn);
    T* d1 = ar.get<T>(n);
    T* d2 = ar.get<T>(n);
    T* D = ar.get<T>(nn);
    axpby<T>(st, n, n, 1.0, Apk + i * nn, n, 0, 0.0, Ma, n, 0, 1);
    axpby<T>(st, n, n, 1.0, H + i * nn, n, 0, 0.0, Mh, n, 0, 1);
    {
      const size_t mq = ar.mark();
      QRStore<T> qa = qr_alloc<T>(ar, n, n, n, 1);
      qr_factor<T>(st, ar, qa, Ma, n, 0);
      qr_form_q<T>(st, ar, qa, Qa, n, 0);
      ar.release(mq);
      QRStore<T> qh = qr_alloc<T>(ar, n, n, n, 1);
      qr_factor<T>(st, ar, qh, Mh, n, 0);
      qr_form_q<T>(st, ar, qh, Qh, n, 0);
      ar.release(mq);
    }
    diag_phase_kernel<T><<<ceil_div(n, 256), 256, 0, st>>>(n, Ma, n, d1);
    diag_phase_kernel<T><<<ceil_div(n, 256), 256, 0, st>>>(n, Mh, n, d2);
    ZCSD_LAUNCH();
    scale_cols_phase_kernel<T><<<grid_for(nn), 256, 0, st>>>(n, n, Qa, n, d1, d2, Qa, n);
    ZCSD_LAUNCH();
    gemm1<T>(st, OP_N, OP_C, n, n, n, one, Qa, n, Qh, n, zer, W + i * nn, n, 0, 0, GS_ALG2);
    rdiff_kernel<T><<<grid_for(nn), 256, 0, st>>>(n, Ma, n, d1, Mh, n, d2, D);
    ZCSD_LAUNCH();
    fro2<T>(st, n, n, D, n, 0, 0.0, sc + 8, 1, scratch);
    d2h(cx, cx.hs.d, sc + 8, sizeof(double));
    const double rd = std::sqrt(cx.hs.d[0]) / std::max(std::sqrt(fro / 2.0), 1e-300);
    if (info) { info->alg2_used[i] = 1; info->rdiff[i] = rd; }
    ar.release(mk);
    if (rd > 1e3 * n * U_ROUND || (cx.alg2_svd_factor >= 0.0 && rd >= cx.alg2_svd_factor * n * U_ROUND)) {
      if (cx.alg2_svd_factor < 0.0) {
        status = CSD_WARN_ALG2_RCHECK;
      } else {
        // Section 5.1: ||R~ - R|| not O(u), so W_i H_i is not a backward
        // stable polar decomposition of A_i; take the polar decomposition
        // from the SVD instead (W_i = U V^*, H_i = sym(W_i^* A_i))
        svd_polar<T>(cx, ar, n, Apk + i * nn, n, W + i * nn, n);
        gemm1<T>(st, OP_C, OP_N, n, n, n, one, W + i * nn, n, Apk + i * nn, n, zer, H + i * nn, n, 0, 0, GS_H);
        symmetrize<T>(st, n, H + i * nn, n, 0, H + i * nn, n, 0, 1);
        if (info) info->alg2_used[i] = 2;
      }
    }
  };
  // full rank: Algorithm 2 where W_i is not orthonormal
  const double orth_tol = 50.0 * n * U_ROUND;
  for (int i = 0; i < 2 && mu == 0.0; ++i)
    if (orth[i] > orth_tol) alg2(i);
  // ---- line 4: B = H2 - H1 + mu (I - A^* A)
  {
    const size_t mk = ar.mark();
    T* G = nullptr;
    if (mu != 0.0) {
      G = ar.get<T>(nn);
      GemmArgs<T> g;  // A^* A = A1^* A1 + A2^* A2 (two-term grouped sum)
      g.batch = 1;
      g.m = n; g.n = n; g.k = n; g.opA = OP_C; g.opB = OP_N;
      g.A = Apk; g.lda = n; g.sAj = nn;
      g.B = Apk; g.ldb = n; g.sBj = nn;
      g.nsum = 2;
      g.C = G; g.ldc = n;
      g.alpha = one; g.beta = zer;
      gemm(g, st);
    }
    form_b_kernel<T><<<grid_for(nn), 256, 0, st>>>(n, H, nn, G, mu, Bm);
    ZCSD_LAUNCH();
    symmetrize<T>(st, n, Bm, n, 0, Bm, n, 0, 1);
    ar.release(mk);
  }
  // ---- line 5: V1 Lambda V1^* = B (Zolo-eig; Algorithm 3 keeps Lambda < 1.1)
  EigDiag ed;
  int lo = 0;
  heig_impl<T>(cx, ar, n, Bm, n, lam, V, mu != 0.0 ? 1.1 : INFINITY, &lo, &ed);
  const int rk = n - lo;
  if (info) {
    info->eig_splits = ed.splits;
    info->eig_retries = ed.retries;
    info->eig_leaves = ed.leaves;
    info->eig_offblock = ed.offblock;
  }
  // ---- lines 6-9: C/S = diag(V1^* H_i V1), U_i = W_i V1, theta = atan2(S, C)
  // (remark (iii)); or theta from Lambda (remark (iv)), which needs no C, S
  T* Vr = V + (long long)lo * n;
  if (rk > 0) {
    GemmArgs<T> g;
    g.batch = 2;
    g.m = n; g.n = rk; g.k = n; g.opA = OP_N; g.opB = OP_N;
    g.lda = n; g.sA = nn;
    g.B = Vr; g.ldb = n; g.sB = 0;
    g.C = Ut; g.ldc = n; g.sC = nn;
    g.alpha = one; g.beta = zer;
    g.site = GS_ASSEMBLY;
    double* Cd = dv;
    double* Sd = dv + n;
    double* th = dv + 2 * n;
    if (cx.theta_mode == 0) {
      g.A = H;  // H_i V1 (into Ut, overwritten by U_i below)
      gemm(g, st);
      col_dots<T>(st, n, rk, Vr, n, Ut, n, Cd);
      col_dots<T>(st, n, rk, Vr, n, Ut + nn, n, Sd);
    }
    g.A = W;  // U_i = W_i V1
    gemm(g, st);
    if (mu != 0.0) {
      // rank-deficient and C or S ill conditioned (Section 5.2, last
      // paragraph): the modified Zolo-pd's W_i is not orthonormal, and where
      // a kept angle's cosine / sine is small W_i V1 loses orthonormality
      // too.  Check U_i^* U_i = I (the tolerance of the full-rank W_i check);
      // a block that fails takes W_i from Algorithm 2, lines 2-3.
      const size_t mk = ar.mark();
      T* Gu = ar.get<T>(2 * (size_t)rk * rk);
      GemmArgs<T> gg;
      gg.batch = 2;
      gg.m = rk; gg.n = rk; gg.k = n; gg.opA = OP_C; gg.opB = OP_N;
      gg.A = Ut; gg.lda = n; gg.sA = nn;
      gg.B = Ut; gg.ldb = n; gg.sB = nn;
      gg.C = Gu; gg.ldc = rk; gg.sC = (long long)rk * rk;
      gg.alpha = one; gg.beta = zer;
      gg.site = GS_ORTH;
      gemm(gg, st);
      fro2<T>(st, rk, rk, Gu, rk, (long long)rk * rk, 1.0, sc + 12, 2, scratch);
      d2h(cx, cx.hs.d, sc + 12, 2 * sizeof(double));
      ar.release(mk);
      const double ou[2] = {std::sqrt(cx.hs.d[0]), std::sqrt(cx.hs.d[1])};
      for (int i = 0; i < 2; ++i) {
        if (ou[i] <= orth_tol) continue;
        alg2(i);
        GemmArgs<T> gi = g;
        gi.batch = 1;
        gi.A = W + i * nn;
        gi.C = Ut + i * nn;
        gemm(gi, st);
      }
    }
    if (cx.theta_mode == 0) theta_from_cs(st, rk, Cd, Sd, th);
    else theta_from_lambda(st, rk, lam + lo, th);
    sort_perm(st, rk, th, perm);
    gather_vec(st, rk, th, perm, theta);
    gather_cols<T>(st, n, rk, Ut, n, perm, U1, ldu1);
    gather_cols<T>(st, n, rk, Ut + nn, n, perm, U2, ldu2);
    gather_cols<T>(st, n, rk, Vr, n, perm, V1, ldv1);
    if (cx.sign_mode == 1) canonical_signs<T>(st, n, n, n, rk, V1, ldv1, U1, ldu1, U2, ldu2);
  }
  if (rk < n) {
    zero_tail_kernel<<<ceil_div(n, 256), 256, 0, st>>>(n, rk, theta);
    ZCSD_LAUNCH();
  }
  ZCSD_CUDA(cudaStreamSynchronize(st));
  if (rank_out) *rank_out = rk;
  if (info) info->rank = rk;
  return status;
}

// Remark (viii): V2 of the complete 2 x 2 CS decomposition of a unitary
// [A1 A3; A2 A4], given U1, U2, theta of [A1; A2]: X = -A3^* U1 S + A4^* U2 C,
// X = Q R with diag(R) >= 0, V2 = Q.
template <class T>
__global__ void scale_cs_kernel(int n, const T* U1, int ldu1, const T* U2, int ldu2, const double* theta, T* P) {
  const long long nn = (long long)n * n;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < nn; t += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(t % n), j = (int)(t / n);
    P[t] = scal(sin(theta[j]), U1[i + (long long)j * ldu1]);       // U1 S
    P[nn + t] = scal(cos(theta[j]), U2[i + (long long)j * ldu2]);  // U2 C
  }
}

template <class T>
__global__ void scale_cols_kernel(int n, const T* Q, const T* d, T* V, int ldv) {
  const long long nn = (long long)n * n;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < nn; t += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(t % n), j = (int)(t / n);
    V[i + (long long)j * ldv] = mul(Q[t], d[j]);
  }
}

template <class T>
int complete_v2_impl(Ctx& cx, Arena& ar, int n, const T* A3, int lda3, const T* A4, int lda4, const T* U1, int ldu1,
                     const T* U2, int ldu2, const double* theta, T* V2, int ldv2) {
  cudaStream_t st = cx.stream;
  const long long nn = (long long)n * n;
  T* P = ar.get<T>(2 * nn);
  T* X = ar.get<T>(nn);
  T* Q = ar.get<T>(nn);
  T* d = ar.get<T>(n);
  const T one = from_re<T>(1.0), mone = from_re<T>(-1.0), zer = zero<T>();
  scale_cs_kernel<T><<<grid_for(nn), 256, 0, st>>>(n, U1, ldu1, U2, ldu2, theta, P);
  ZCSD_LAUNCH();
  gemm1<T>(st, OP_C, OP_N, n, n, n, mone, A3, lda3, P, n, zer, X, n, 0, 0, GS_OTHER);      // -A3^* U1 S
  gemm1<T>(st, OP_C, OP_N, n, n, n, one, A4, lda4, P + nn, n, one, X, n, 0, 0, GS_OTHER);  // + A4^* U2 C
  const size_t mq = ar.mark();
  QRStore<T> q = qr_alloc<T>(ar, n, n, n, 1);
  qr_factor<T>(st, ar, q, X, n, 0);
  qr_form_q<T>(st, ar, q, Q, n, 0);
  ar.release(mq);
  diag_phase_kernel<T><<<ceil_div(n, 256), 256, 0, st>>>(n, X, n, d);
  ZCSD_LAUNCH();
  scale_cols_kernel<T><<<grid_for(nn), 256, 0, st>>>(n, Q, d, V2, ldv2);
  ZCSD_LAUNCH();
  return CSD_OK;
}

// Rectangular blocks A_i (m_i x n, m_i >= n; the partial isometries of
// Section 2): A_i = Q_i R_i by Householder QR (Q_i with orthonormal columns),
// the square CSD of [R1; R2] (its columns are orthonormal as well, since
// R1^* R1 + R2^* R2 = A^* A), and U_i = Q_i U_i'.
template <class T>
__global__ void upper_tri_kernel(int n, const T* M, int ldm, T* R) {
  const long long nn = (long long)n * n;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < nn; t += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(t % n), j = (int)(t / n);
    R[t] = (i <= j) ? M[i + (long long)j * ldm] : zero<T>();
  }
}

template <class T>
int csd_rect_impl(Ctx& cx, Arena& ar, int m1, int m2, int n, const T* A1, int lda1, const T* A2, int lda2, T* U1,
                  int ldu1, T* U2, int ldu2, T* V1, int ldv1, double* theta, int* rank_out, csd_info* info) {
  cudaStream_t st = cx.stream;
  const long long nn = (long long)n * n;
  T* R = ar.get<T>(2 * nn);  // R1 | R2, n x n each
  T* Q1 = ar.get<T>((size_t)m1 * n);
  T* Q2 = ar.get<T>((size_t)m2 * n);
  T* Us = ar.get<T>(2 * nn);  // U1', U2' of the square CSD
  const T one = from_re<T>(1.0), zer = zero<T>();
  for (int i = 0; i < 2; ++i) {
    const int m = i == 0 ? m1 : m2;
    const T* A = i == 0 ? A1 : A2;
    const int lda = i == 0 ? lda1 : lda2;
    T* Q = i == 0 ? Q1 : Q2;
    const size_t mk = ar.mark();
    T* M = ar.get<T>((size_t)m * n);
    axpby<T>(st, m, n, 1.0, A, lda, 0, 0.0, M, m, 0, 1);
    QRStore<T> q = qr_alloc<T>(ar, m, n, m, 1);
    qr_factor<T>(st, ar, q, M, m, 0);
    qr_form_q<T>(st, ar, q, Q, m, 0);
    upper_tri_kernel<T><<<grid_for(nn), 256, 0, st>>>(n, M, m, R + i * nn);
    ZCSD_LAUNCH();
    ar.release(mk);
  }
  int rk = 0;
  const int stt = csd_impl<T>(cx, ar, n, R, n, R + nn, n, Us, n, Us + nn, n, V1, ldv1, theta, &rk, info);
  if (stt != CSD_OK && stt != CSD_WARN_ALG2_RCHECK) return stt;
  if (rk > 0) {
    gemm1<T>(st, OP_N, OP_N, m1, rk, n, one, Q1, m1, Us, n, zer, U1, ldu1, 0, 0, GS_ASSEMBLY);
    gemm1<T>(st, OP_N, OP_N, m2, rk, n, one, Q2, m2, Us + nn, n, zer, U2, ldu2, 0, 0, GS_ASSEMBLY);
  }
  ZCSD_CUDA(cudaStreamSynchronize(st));
  if (rank_out) *rank_out = rk;
  return stt;
}

// ||W^* W - I||_F of the n x n W (device) read back to the host.
template <class T>
static double orth_error(Ctx& cx, Arena& ar, int n, const T* W, double* sc, double* scratch) {
  const size_t mk = ar.mark();
  T* G = ar.get<T>((size_t)n * n);
  gemm1<T>(cx.stream, OP_C, OP_N, n, n, n, from_re<T>(1.0), W, n, W, n, zero<T>(), G, n, 0, 0, GS_ORTH);
  fro2<T>(cx.stream, n, n, G, n, 0, 1.0, sc, 1, scratch);
  d2h(cx, cx.hs.d, sc, sizeof(double));
  ar.release(mk);
  return std::sqrt(cx.hs.d[0]);
}

// polar(): Zolo-pd on [eps, 1] (Section 5.1), then the convergence test.
// Section 5 runs two iterations; with the interval fixed in advance they
// converge exactly when every singular value of the scaled A is at least
// eps, and otherwise the iterate is not unitary.  The test is therefore
// ||X^* X - I||_F <= 50 n u after the planned iterations.  A failing iterate
// goes through the plan again (its smallest singular values have grown by
// the slope of the composed map near zero, so one more pass converges
// unless A is singular to working precision), up to cx.zolo_extra_passes
// times; if it still fails, the call returns CSD_ERR_NOT_CONVERGED with the
// last iterate written.  cx.zolo_stop_after > 0 returns the iterate X_k
// itself (no test), for checking the iterates against U Z_k(Sigma) V^*.
template <class T>
int polar_impl(Ctx& cx, Arena& ar, int n, const T* A, int lda, T* Wo, int ldw, T* Ho, int ldh, csd_info* info) {
  cudaStream_t st = cx.stream;
  const long long nn = (long long)n * n;
  T* X = ar.get<T>(nn);
  T* W = ar.get<T>(nn);
  double* sc = ar.get<double>(64);
  double* scratch = ar.get<double>(304 * 4);
  axpby<T>(st, n, n, 1.0, A, lda, 0, 0.0, X, n, 0, 1);
  count_nonfinite<T>(st, n, n, X, n, sc, scratch);
  fro2<T>(st, n, n, X, n, 0, 0.0, sc + 1, 1, scratch);
  d2h(cx, cx.hs.d, sc, 2 * sizeof(double));
  if (cx.hs.d[0] != 0.0) return CSD_ERR_NONFINITE;
  const double fn = std::sqrt(cx.hs.d[1]);
  // ||A||_2 <= 1 is needed; rescale by ||A||_F only when it could be violated
  const double alpha = (fn > 1.0) ? 1.0 / fn : 1.0;
  if (alpha != 1.0) axpby<T>(st, n, n, alpha, X, n, 0, 0.0, X, n, 0, 1);
  PolarDiag pd;
  int status = CSD_OK;
  double orth = 0.0;
  if (cx.zolo_stop_after > 0) {
    zolo_pd<T>(cx, ar, n, 1, X, W, &pd, cx.zolo_stop_after);
  } else {
    zolo_pd<T>(cx, ar, n, 1, X, W, &pd, 0, (cx.mixed_scope & 1u) ? cx.mixed_slices : 0);
    const double tol = 50.0 * n * U_ROUND;
    orth = orth_error<T>(cx, ar, n, W, sc + 2, scratch);
    for (int pass = 0; pass < cx.zolo_extra_passes && !(orth <= tol); ++pass) {
      zolo_pd<T>(cx, ar, n, 1, W, W, &pd);
      orth = orth_error<T>(cx, ar, n, W, sc + 2, scratch);
    }
    if (!(orth <= tol)) status = CSD_ERR_NOT_CONVERGED;
  }
  axpby<T>(st, n, n, 1.0, W, n, 0, 0.0, Wo, ldw, 0, 1);
  if (Ho) {
    T* Hm = X;
    gemm1<T>(st, OP_C, OP_N, n, n, n, from_re<T>(1.0), W, n, A, lda, zero<T>(), Hm, n, 0, 0, GS_H);
    symmetrize<T>(st, n, Hm, n, 0, Ho, ldh, 0, 1);
  }
  if (info) {
    const Plan& pl = get_plan(cx);
    info->zolo_iters = pd.iters;
    for (int s = 0; s < 4; ++s) {
      info->r_terms[s] = s < pl.steps ? pl.r[s] : 0;
      info->ell[s] = s < pl.steps ? pl.ell[s] : 0.0;
    }
    info->chol_fallback = pd.chol_fallback;
    info->orth_err[0] = orth;
  }
  ZCSD_CUDA(cudaStreamSynchronize(st));
  return status;
}

template int polar_impl<double>(Ctx&, Arena&, int, const double*, int, double*, int, double*, int, csd_info*);
template int polar_impl<z64>(Ctx&, Arena&, int, const z64*, int, z64*, int, z64*, int, csd_info*);

template <class T>
int heig_entry(Ctx& cx, Arena& ar, int n, const T* B, int ldb, double* lam, T* Vo, int ldv, csd_info* info) {
  cudaStream_t st = cx.stream;
  const long long nn = (long long)n * n;
  T* V = ar.get<T>(nn);
  double* sc = ar.get<double>(64);
  double* scratch = ar.get<double>(304 * 4);
  count_nonfinite<T>(st, n, n, B, ldb, sc, scratch);
  d2h(cx, cx.hs.d, sc, sizeof(double));
  if (cx.hs.d[0] != 0.0) return CSD_ERR_NONFINITE;
  EigDiag ed;
  int lo = 0;
  heig_impl<T>(cx, ar, n, B, ldb, lam, V, INFINITY, &lo, &ed);
  axpby<T>(st, n, n, 1.0, V, n, 0, 0.0, Vo, ldv, 0, 1);
  if (info) {
    info->eig_splits = ed.splits;
    info->eig_retries = ed.retries;
    info->eig_leaves = ed.leaves;
    info->eig_offblock = ed.offblock;
  }
  ZCSD_CUDA(cudaStreamSynchronize(st));
  return CSD_OK;
}

}  // namespace zcsd

// ====================================================================== C ABI
using namespace zcsd;

struct csd_ctx {
  Ctx cx;
};

zcsd::Ctx* ctx_internal(csd_ctx* ctx) { return &ctx->cx; }

namespace {

bool is_device_ptr(const void* p) {
  if (!p) return false;
  cudaPointerAttributes at;
  cudaError_t e = cudaPointerGetAttributes(&at, p);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

// Upper bound of the workspace (bytes) needed by a call; run_with_ws also
// grows the arena and retries if a bound turns out short.
size_t polar_bytes(long long n, int P, size_t es) {
  const long long nn = n * n;
  const long long r = R_MAX;
  long long qr = 2 * (2 * nn) * P * r                                         // M, E
                 + (long long)ceil_div(n, NB_OUT) * (n + 1 + NB_OUT) * NB_OUT * P * r  // Y
                 + (long long)ceil_div(n, NB_OUT) * NB_OUT * NB_OUT * P * r           // T
                 + (long long)(5 * NB_OUT + (MAX_SUM + 1) * NB_QR) * n * P * r;         // W parts, W2
  long long ch = nn * P + 3 * nn * P * r + (long long)NB_CHOL * n * P * r * (2 + MAX_SUM);
  return (size_t)((2 * nn * P + std::max(qr, ch)) * es) + 64 * 256;
}

size_t heig_bytes(long long n, size_t es) {
  const long long nn = n * n;
  long long qr = (long long)ceil_div(n, NB_OUT) * (n + NB_OUT) * NB_OUT +
                 (long long)ceil_div(n, NB_OUT) * NB_OUT * NB_OUT + (long long)(5 * NB_OUT + (MAX_SUM + 1) * NB_QR) * n;
  long long leaves = 2 * (long long)LEAF_MAX * n + 8 * n;  // packed G_l and V_l: sum sz_l^2 <= n * leaf
  return (size_t)((7 * nn + std::max(qr, leaves)) * es) + polar_bytes(n, 1, es) + (size_t)(3 * n + 2048) * 8 + 64 * 256;
}

size_t csd_bytes(long long n, size_t es) {
  const long long nn = n * n;
  size_t fixed = (size_t)(11 * nn * es) + (size_t)(6 * n + 2048) * 8 + 64 * 256;
  size_t alg2 = (size_t)(7 * nn * es) + polar_bytes(1, 1, es);
  return fixed + std::max({polar_bytes(n, 2, es), heig_bytes(n, es), alg2 + (size_t)(2 * nn * es)});
}

int ensure_ws(Ctx& cx, size_t bytes) {
  if (cx.ws_bytes >= bytes) return 0;
  if (cx.ws) {
    cudaStreamSynchronize(cx.stream);
    cudaFree(cx.ws);
    cx.ws = nullptr;
    cx.ws_bytes = 0;
  }
  if (cudaMalloc((void**)&cx.ws, bytes) != cudaSuccess) {
    cudaGetLastError();
    cx.ws = nullptr;
    return CSD_ERR_ALLOC;
  }
  cx.ws_bytes = bytes;
  return 0;
}

// Run `body(arena)` with a workspace of at least `need` bytes, growing it on
// an arena overflow; translates exceptions to status codes.
template <class F>
int run_with_ws(Ctx& cx, size_t need, csd_info* info, F body) {
  const auto t0 = std::chrono::steady_clock::now();
  int status = CSD_OK;
  if (cudaSetDevice(cx.device) != cudaSuccess) { cudaGetLastError(); return CSD_ERR_CUDA; }
  struct ProfScope {  // make this context's profiler the thread's active one
    Profiler* prev;
    explicit ProfScope(Profiler* p) : prev(t_prof) { t_prof = p; }
    ~ProfScope() { t_prof = prev; }
  } scope(&cx.prof);
  struct TcScope {  // tensor-core dispatch state for this call
    TcState prev;
    TcScope() : prev(t_tc) {}
    ~TcScope() { t_tc = prev; }
  } tc_scope;
  for (int attempt = 0; attempt < 4; ++attempt) {
    status = ensure_ws(cx, need);
    if (status) break;
    Arena ar;
    ar.base = cx.ws;
    ar.cap = cx.ws_bytes;
    try {
      int* tc_err = nullptr;
      if (cx.tensor_cores || cx.force_tc_err) {
        tc_err = ar.get<int>(1);
        ZCSD_CUDA(cudaMemsetAsync(tc_err, 0, sizeof(int), cx.stream));
      }
      t_tc.enabled = cx.tensor_cores;
      t_tc.sites = cx.tc_sites;
      t_tc.ar = &ar;
      t_tc.err = tc_err;
      t_tc.probe_wait = cx.tc_probe_wait;
      t_tc.flush_every = cx.tc_flush_every;
      status = body(ar);
      if (tc_err) {
        int h = 0;
        ZCSD_CUDA(cudaMemcpyAsync(&h, tc_err, sizeof(int), cudaMemcpyDeviceToHost, cx.stream));
        ZCSD_CUDA(cudaStreamSynchronize(cx.stream));
        // a timed-out product leaves NaN behind, which later steps may report
        // in their own way; the timeout is the cause
        if (h && status != CSD_ERR_CUDA) status = CSD_ERR_DEVICE_TIMEOUT;
      }
      break;
    } catch (ArenaOverflow& o) {
      cudaStreamSynchronize(cx.stream);
      need = std::max(need * 2, o.needed + need / 2);
      status = CSD_ERR_INTERNAL;
    } catch (CudaFail& f) {
      fprintf(stderr, "zolo_csd: CUDA error %s at %s:%d\n", cudaGetErrorString(f.err), f.file, f.line);
      status = CSD_ERR_CUDA;
      break;
    } catch (EigFail& e) {
      status = CSD_ERR_EIG_SPLIT;
      if (info) {
        info->eig_splits = e.splits;
        info->eig_retries = e.retries;
      }
      break;
    } catch (std::bad_alloc&) {
      status = CSD_ERR_ALLOC;
      break;
    }
  }
  const auto t1 = std::chrono::steady_clock::now();
  if (info) {
    info->status = status;
    info->ms_total = std::chrono::duration<double, std::milli>(t1 - t0).count();
  }
  return status;
}

// Device view of a caller matrix: the pointer itself when it is device
// memory, else a staging copy in the arena (copied in when `in`).
template <class T>
struct Mat {
  T* d = nullptr;
  int ld = 0;
  const void* host = nullptr;
  void* host_out = nullptr;
  int host_ld = 0;
};

template <class T>
Mat<T> view_in(Ctx& cx, Arena& ar, const void* p, int ld, int m, int n) {
  Mat<T> v;
  if (is_device_ptr(p)) {
    v.d = (T*)p;
    v.ld = ld;
    return v;
  }
  v.d = ar.get<T>((size_t)m * n);
  v.ld = m;
  ZCSD_CUDA(cudaMemcpy2DAsync(v.d, sizeof(T) * m, p, sizeof(T) * ld, sizeof(T) * m, n, cudaMemcpyHostToDevice,
                              cx.stream));
  return v;
}

template <class T>
Mat<T> view_out(Arena& ar, void* p, int ld, int m, int n) {
  Mat<T> v;
  if (is_device_ptr(p)) {
    v.d = (T*)p;
    v.ld = ld;
    return v;
  }
  v.d = ar.get<T>((size_t)m * n);
  v.ld = m;
  v.host_out = p;
  v.host_ld = ld;
  return v;
}

template <class T>
void copy_out(Ctx& cx, const Mat<T>& v, int m, int n) {
  if (!v.host_out) return;
  ZCSD_CUDA(cudaMemcpy2DAsync(v.host_out, sizeof(T) * v.host_ld, v.d, sizeof(T) * m, sizeof(T) * m, n,
                              cudaMemcpyDeviceToHost, cx.stream));
}

template <class T>
int csd_typed(csd_ctx* ctx, int n, const void* A1, int lda1, const void* A2, int lda2, void* U1, int ldu1, void* U2,
              int ldu2, void* V1, int ldv1, double* theta, int* rank, csd_info* info) {
  Ctx& cx = ctx->cx;
  const size_t need = csd_bytes(n, sizeof(T)) + (size_t)8 * n * n * sizeof(T);
  return run_with_ws(cx, need, info, [&](Arena& ar) -> int {
    Mat<T> a1 = view_in<T>(cx, ar, A1, lda1, n, n);
    Mat<T> a2 = view_in<T>(cx, ar, A2, lda2, n, n);
    Mat<T> u1 = view_out<T>(ar, U1, ldu1, n, n);
    Mat<T> u2 = view_out<T>(ar, U2, ldu2, n, n);
    Mat<T> v1 = view_out<T>(ar, V1, ldv1, n, n);
    Mat<double> th = view_out<double>(ar, theta, n, n, 1);
    int rk = 0;
    int st = csd_impl<T>(cx, ar, n, a1.d, a1.ld, a2.d, a2.ld, u1.d, u1.ld, u2.d, u2.ld, v1.d, v1.ld, th.d, &rk, info);
    if (st == CSD_OK || st == CSD_WARN_ALG2_RCHECK) {
      copy_out(cx, u1, n, n);
      copy_out(cx, u2, n, n);
      copy_out(cx, v1, n, n);
      copy_out(cx, th, n, 1);
      ZCSD_CUDA(cudaStreamSynchronize(cx.stream));
      if (rank) *rank = rk;
    }
    return st;
  });
}

template <class T>
int polar_typed(csd_ctx* ctx, int n, const void* A, int lda, void* W, int ldw, void* H, int ldh, csd_info* info) {
  Ctx& cx = ctx->cx;
  const size_t need = polar_bytes(n, 1, sizeof(T)) + (size_t)8 * n * n * sizeof(T);
  return run_with_ws(cx, need, info, [&](Arena& ar) -> int {
    Mat<T> a = view_in<T>(cx, ar, A, lda, n, n);
    Mat<T> w = view_out<T>(ar, W, ldw, n, n);
    Mat<T> h;
    if (H) h = view_out<T>(ar, H, ldh, n, n);
    int st = polar_impl<T>(cx, ar, n, a.d, a.ld, w.d, w.ld, H ? h.d : nullptr, h.ld, info);
    if (st == CSD_OK || st == CSD_ERR_NOT_CONVERGED) {
      copy_out(cx, w, n, n);
      if (H) copy_out(cx, h, n, n);
      ZCSD_CUDA(cudaStreamSynchronize(cx.stream));
    }
    return st;
  });
}

template <class T>
int heig_typed(csd_ctx* ctx, int n, const void* B, int ldb, double* lam, void* V, int ldv, csd_info* info) {
  Ctx& cx = ctx->cx;
  const size_t need = heig_bytes(n, sizeof(T)) + (size_t)4 * n * n * sizeof(T);
  return run_with_ws(cx, need, info, [&](Arena& ar) -> int {
    Mat<T> b = view_in<T>(cx, ar, B, ldb, n, n);
    Mat<T> v = view_out<T>(ar, V, ldv, n, n);
    Mat<double> l = view_out<double>(ar, lam, n, n, 1);
    int st = heig_entry<T>(cx, ar, n, b.d, b.ld, l.d, v.d, v.ld, info);
    if (st == CSD_OK) {
      copy_out(cx, v, n, n);
      copy_out(cx, l, n, 1);
      ZCSD_CUDA(cudaStreamSynchronize(cx.stream));
    }
    return st;
  });
}

template <class T>
int csd_rect_typed(csd_ctx* ctx, int m1, int m2, int n, const void* A1, int lda1, const void* A2, int lda2, void* U1,
                   int ldu1, void* U2, int ldu2, void* V1, int ldv1, double* theta, int* rank, csd_info* info) {
  Ctx& cx = ctx->cx;
  const size_t need = csd_bytes(n, sizeof(T)) + (size_t)(4 * (long long)(m1 + m2) * n + 8LL * n * n) * sizeof(T) +
                      heig_bytes(std::max(m1, m2), sizeof(T)) / 4;
  return run_with_ws(cx, need, info, [&](Arena& ar) -> int {
    Mat<T> a1 = view_in<T>(cx, ar, A1, lda1, m1, n);
    Mat<T> a2 = view_in<T>(cx, ar, A2, lda2, m2, n);
    Mat<T> u1 = view_out<T>(ar, U1, ldu1, m1, n);
    Mat<T> u2 = view_out<T>(ar, U2, ldu2, m2, n);
    Mat<T> v1 = view_out<T>(ar, V1, ldv1, n, n);
    Mat<double> th = view_out<double>(ar, theta, n, n, 1);
    int rk = 0;
    int st = csd_rect_impl<T>(cx, ar, m1, m2, n, a1.d, a1.ld, a2.d, a2.ld, u1.d, u1.ld, u2.d, u2.ld, v1.d, v1.ld, th.d,
                              &rk, info);
    if (st == CSD_OK || st == CSD_WARN_ALG2_RCHECK) {
      copy_out(cx, u1, m1, n);
      copy_out(cx, u2, m2, n);
      copy_out(cx, v1, n, n);
      copy_out(cx, th, n, 1);
      ZCSD_CUDA(cudaStreamSynchronize(cx.stream));
      if (rank) *rank = rk;
    }
    return st;
  });
}

template <class T>
int complete_v2_typed(csd_ctx* ctx, int n, const void* A3, int lda3, const void* A4, int lda4, const void* U1,
                      int ldu1, const void* U2, int ldu2, const double* theta, void* V2, int ldv2, csd_info* info) {
  Ctx& cx = ctx->cx;
  const size_t need = heig_bytes(n, sizeof(T)) + (size_t)8 * n * n * sizeof(T);
  return run_with_ws(cx, need, info, [&](Arena& ar) -> int {
    Mat<T> a3 = view_in<T>(cx, ar, A3, lda3, n, n);
    Mat<T> a4 = view_in<T>(cx, ar, A4, lda4, n, n);
    Mat<T> u1 = view_in<T>(cx, ar, U1, ldu1, n, n);
    Mat<T> u2 = view_in<T>(cx, ar, U2, ldu2, n, n);
    Mat<double> th = view_in<double>(cx, ar, theta, n, n, 1);
    Mat<T> v2 = view_out<T>(ar, V2, ldv2, n, n);
    int st = complete_v2_impl<T>(cx, ar, n, a3.d, a3.ld, a4.d, a4.ld, u1.d, u1.ld, u2.d, u2.ld, th.d, v2.d, v2.ld);
    if (st == CSD_OK) copy_out(cx, v2, n, n);
    ZCSD_CUDA(cudaStreamSynchronize(cx.stream));
    return st;
  });
}

int backward_typed(csd_ctx* ctx, int n, const void* U1, int ldu1, const void* U2, int ldu2, const void* V1, int ldv1,
                   const double* theta, const void* gU1, int ldgu1, const void* gU2, int ldgu2, const void* gV1,
                   int ldgv1, const double* gtheta, void* gA1, int ldga1, void* gA2, int ldga2, csd_info* info) {
  Ctx& cx = ctx->cx;
  const size_t need = (size_t)16 * n * n * sizeof(double) + ((size_t)1 << 20);
  return run_with_ws(cx, need, info, [&](Arena& ar) -> int {
    Mat<double> u1 = view_in<double>(cx, ar, U1, ldu1, n, n);
    Mat<double> u2 = view_in<double>(cx, ar, U2, ldu2, n, n);
    Mat<double> v1 = view_in<double>(cx, ar, V1, ldv1, n, n);
    Mat<double> th = view_in<double>(cx, ar, theta, n, n, 1);
    Mat<double> gu1, gu2, gv1, gth;
    if (gU1) gu1 = view_in<double>(cx, ar, gU1, ldgu1, n, n);
    if (gU2) gu2 = view_in<double>(cx, ar, gU2, ldgu2, n, n);
    if (gV1) gv1 = view_in<double>(cx, ar, gV1, ldgv1, n, n);
    if (gtheta) gth = view_in<double>(cx, ar, gtheta, n, n, 1);
    Mat<double> ga1 = view_out<double>(ar, gA1, ldga1, n, n);
    Mat<double> ga2 = view_out<double>(ar, gA2, ldga2, n, n);
    int st = csd_backward_impl(cx, ar, n, u1.d, u1.ld, u2.d, u2.ld, v1.d, v1.ld, th.d, gu1.d, gu1.ld, gu2.d, gu2.ld,
                               gv1.d, gv1.ld, gth.d, ga1.d, ga1.ld, ga2.d, ga2.ld);
    copy_out(cx, ga1, n, n);
    copy_out(cx, ga2, n, n);
    ZCSD_CUDA(cudaStreamSynchronize(cx.stream));
    return st;
  });
}

// C = alpha op(A) op(B) + beta C on the FP64 pipe (engine 0) or the
// tensor-core kernel (engine 1, any shape).
int gemm_typed(csd_ctx* ctx, int opA, int opB, int m, int n, int k, double alpha, const double* A, int lda,
               const double* B, int ldb, double beta, double* C, int ldc, int engine) {
  Ctx& cx = ctx->cx;
  const size_t need = (size_t)16 * ((size_t)(m + 128) * (k + 64) + (size_t)(n + 128) * (k + 64)) + (1 << 20);
  cx.force_tc_err = engine == 1;
  const int st = run_with_ws(cx, need, nullptr, [&](Arena& ar) -> int {
    GemmArgs<double> g;
    g.m = m; g.n = n; g.k = k; g.opA = opA; g.opB = opB;
    g.A = A; g.lda = lda; g.B = B; g.ldb = ldb;
    g.Cin = C; g.ldcin = ldc; g.C = C; g.ldc = ldc;
    g.alpha = alpha; g.beta = beta;
    if (engine == 1) {
      tc_gemm(g, cx.stream, ar, t_tc.err);
    } else {
      t_tc.enabled = false;
      gemm(g, cx.stream);
    }
    ZCSD_CUDA(cudaStreamSynchronize(cx.stream));
    return CSD_OK;
  });
  cx.force_tc_err = false;
  return st;
}

}  // namespace

extern "C" {

int csd_set_eig_leaf(csd_ctx* ctx, int leaf) {
  if (!ctx) return -1;
  if (leaf < 1 || leaf > LEAF_MAX) return -2;
  ctx->cx.eig_leaf = leaf;
  return CSD_OK;
}

int csd_set_mixed_precision(csd_ctx* ctx, int slices, unsigned scope) {
  if (!ctx) return -1;
  if (slices < 5 || slices > 7) return -2;
  if (scope & ~3u) return -3;
  ctx->cx.mixed_slices = slices;
  ctx->cx.mixed_scope = scope;
  return CSD_OK;
}

int csd_set_alg2_fallback(csd_ctx* ctx, double factor) {
  if (!ctx) return -1;
  if (!(factor == factor)) return -2;
  ctx->cx.alg2_svd_factor = factor;
  return CSD_OK;
}

int csd_set_sign_convention(csd_ctx* ctx, int mode) {
  if (!ctx) return -1;
  if (mode != 0 && mode != 1) return -2;
  ctx->cx.sign_mode = mode;
  return CSD_OK;
}

int csd_polar_backward(csd_ctx* ctx, int dtype, int n, const void* U1, int ldu1, const void* U2, int ldu2,
                       const void* V1, int ldv1, const double* theta, const void* gU1, int ldgu1, const void* gU2,
                       int ldgu2, const void* gV1, int ldgv1, const double* gtheta, void* gA1, int ldga1, void* gA2,
                       int ldga2, csd_info* info) {
  if (!ctx) return -1;
  if (dtype != CSD_F64) return -2;
  if (n < 1) return -3;
  if (!U1) return -4;
  if (ldu1 < n) return -5;
  if (!U2) return -6;
  if (ldu2 < n) return -7;
  if (!V1) return -8;
  if (ldv1 < n) return -9;
  if (!theta) return -10;
  if (gU1 && ldgu1 < n) return -12;
  if (gU2 && ldgu2 < n) return -14;
  if (gV1 && ldgv1 < n) return -16;
  if (!gA1) return -18;
  if (ldga1 < n) return -19;
  if (!gA2) return -20;
  if (ldga2 < n) return -21;
  if (info) std::memset(info, 0, sizeof(csd_info));
  return backward_typed(ctx, n, U1, ldu1, U2, ldu2, V1, ldv1, theta, gU1, ldgu1, gU2, ldgu2, gV1, ldgv1, gtheta, gA1,
                        ldga1, gA2, ldga2, info);
}

int csd_set_zolo_control(csd_ctx* ctx, int max_extra_passes, int stop_after) {
  if (!ctx) return -1;
  if (max_extra_passes < 0 || max_extra_passes > 4) return -2;
  if (stop_after < 0) return -3;
  ctx->cx.zolo_extra_passes = max_extra_passes;
  ctx->cx.zolo_stop_after = stop_after;
  return CSD_OK;
}

int csd_set_test_hooks(csd_ctx* ctx, unsigned flags, long long tc_probe_wait, int tc_flush_every) {
  if (!ctx) return -1;
  if (flags & ~(unsigned)CSD_TEST_REJECT_EIG_SPLITS) return -2;
  if (tc_probe_wait < 0) return -3;
  if (tc_flush_every < 0) return -4;
  ctx->cx.test_flags = flags;
  ctx->cx.tc_probe_wait = tc_probe_wait;
  ctx->cx.tc_flush_every = tc_flush_every;
  return CSD_OK;
}

int csd_gemm(csd_ctx* ctx, int opA, int opB, int m, int n, int k, double alpha, const double* A, int lda,
             const double* B, int ldb, double beta, double* C, int ldc, int engine) {
  if (!ctx) return -1;
  if (opA != 0 && opA != 1) return -2;
  if (opB != 0 && opB != 1) return -3;
  if (m < 0) return -4;
  if (n < 0) return -5;
  if (k < 0) return -6;
  const int ra = opA == 0 ? m : k, rb = opB == 0 ? k : n;
  if (k > 0 && m > 0 && !is_device_ptr(A)) return -8;
  if (lda < std::max(1, ra)) return -9;
  if (k > 0 && n > 0 && !is_device_ptr(B)) return -10;
  if (ldb < std::max(1, rb)) return -11;
  if (m > 0 && n > 0 && !is_device_ptr(C)) return -13;
  if (ldc < std::max(1, m)) return -14;
  if (engine != 0 && engine != 1) return -15;
  if (m == 0 || n == 0) return CSD_OK;
  if (k == 0) {
    if (beta == 1.0) return CSD_OK;
    return gemm_typed(ctx, opA, opB, m, n, 0, alpha, A, lda, B, ldb, beta, C, ldc, 0);
  }
  return gemm_typed(ctx, opA, opB, m, n, k, alpha, A, lda, B, ldb, beta, C, ldc, engine);
}

int csd_create(csd_ctx** ctx, int device, void* stream) {
  if (!ctx) return -1;
  int cnt = 0;
  if (cudaGetDeviceCount(&cnt) != cudaSuccess || cnt <= 0) {
    cudaGetLastError();
    return CSD_ERR_NO_DEVICE;
  }
  if (device < 0 || device >= cnt) return -2;
  if (cudaSetDevice(device) != cudaSuccess) { cudaGetLastError(); return CSD_ERR_CUDA; }
  csd_ctx* c = new (std::nothrow) csd_ctx();
  if (!c) return CSD_ERR_ALLOC;
  c->cx.device = device;
  c->cx.stream = (cudaStream_t)stream;
  if (cudaMallocHost((void**)&c->cx.hs.d, 64 * sizeof(double)) != cudaSuccess ||
      cudaMallocHost((void**)&c->cx.hs.i, 4096 * sizeof(int)) != cudaSuccess) {
    cudaGetLastError();
    delete c;
    return CSD_ERR_ALLOC;
  }
  *ctx = c;
  return CSD_OK;
}

int csd_set_stream(csd_ctx* ctx, void* stream) {
  if (!ctx) return -1;
  ctx->cx.stream = (cudaStream_t)stream;
  return CSD_OK;
}

int csd_destroy(csd_ctx* ctx) {
  if (!ctx) return CSD_OK;
  cudaSetDevice(ctx->cx.device);
  cudaStreamSynchronize(ctx->cx.stream);
  if (ctx->cx.ws) cudaFree(ctx->cx.ws);
  if (ctx->cx.hs.d) cudaFreeHost(ctx->cx.hs.d);
  if (ctx->cx.hs.i) cudaFreeHost(ctx->cx.hs.i);
  delete ctx;
  return CSD_OK;
}

long long csd_workspace_bytes(const csd_ctx* ctx) { return ctx ? (long long)ctx->cx.ws_bytes : 0; }

long long csd_launch_count(void) { return launch_count(); }

int csd_set_tensor_cores(csd_ctx* ctx, int enable) {
  if (!ctx) return -1;
  ctx->cx.tensor_cores = enable != 0;
  ctx->cx.tc_sites = (unsigned)enable;  // bit s: call site s; -1: every site
  return CSD_OK;
}

int csd_profile_enable(csd_ctx* ctx, int enable) {
  if (!ctx) return -1;
  try {
    cudaSetDevice(ctx->cx.device);
    ctx->cx.prof.flush();
    ctx->cx.prof.reset();
  } catch (CudaFail&) {
    return CSD_ERR_CUDA;
  }
  ctx->cx.prof.enabled = enable != 0;
  return CSD_OK;
}

int csd_profile_read(csd_ctx* ctx, csd_profile* out) {
  if (!ctx) return -1;
  if (!out) return -2;
  try {
    cudaSetDevice(ctx->cx.device);
    ctx->cx.prof.flush();
  } catch (CudaFail&) {
    return CSD_ERR_CUDA;
  }
  for (int k = 0; k < PK_KINDS; ++k) {
    out->count[k] = ctx->cx.prof.count[k];
    out->ms[k] = ctx->cx.prof.ms[k];
    out->flops[k] = ctx->cx.prof.flops[k];
  }
  for (int k = 0; k < PROF_SITES; ++k) {
    out->site_count[k] = ctx->cx.prof.site_count[k];
    out->site_ms[k] = ctx->cx.prof.site_ms[k];
    out->site_flops[k] = ctx->cx.prof.site_flops[k];
  }
  return CSD_OK;
}

int csd_polar(csd_ctx* ctx, int dtype, int n, const void* A1, int lda1, const void* A2, int lda2, void* U1, int ldu1,
              void* U2, int ldu2, void* V1, int ldv1, double* theta, int* rank, csd_info* info) {
  if (!ctx) return -1;
  if (dtype != CSD_F64 && dtype != CSD_C128) return -2;
  if (n < 1) return -3;
  if (!A1) return -4;
  if (lda1 < n) return -5;
  if (!A2) return -6;
  if (lda2 < n) return -7;
  if (!U1) return -8;
  if (ldu1 < n) return -9;
  if (!U2) return -10;
  if (ldu2 < n) return -11;
  if (!V1) return -12;
  if (ldv1 < n) return -13;
  if (!theta) return -14;
  if (info) std::memset(info, 0, sizeof(csd_info));
  if (dtype == CSD_F64)
    return csd_typed<double>(ctx, n, A1, lda1, A2, lda2, U1, ldu1, U2, ldu2, V1, ldv1, theta, rank, info);
  return csd_typed<z64>(ctx, n, A1, lda1, A2, lda2, U1, ldu1, U2, ldu2, V1, ldv1, theta, rank, info);
}

int csd_polar_rect(csd_ctx* ctx, int dtype, int m1, int m2, int n, const void* A1, int lda1, const void* A2,
                   int lda2, void* U1, int ldu1, void* U2, int ldu2, void* V1, int ldv1, double* theta, int* rank,
                   csd_info* info) {
  if (!ctx) return -1;
  if (dtype != CSD_F64 && dtype != CSD_C128) return -2;
  if (n < 1) return -5;
  if (m1 < n) return -3;
  if (m2 < n) return -4;
  if (!A1) return -6;
  if (lda1 < m1) return -7;
  if (!A2) return -8;
  if (lda2 < m2) return -9;
  if (!U1) return -10;
  if (ldu1 < m1) return -11;
  if (!U2) return -12;
  if (ldu2 < m2) return -13;
  if (!V1) return -14;
  if (ldv1 < n) return -15;
  if (!theta) return -16;
  if (info) std::memset(info, 0, sizeof(csd_info));
  if (dtype == CSD_F64)
    return csd_rect_typed<double>(ctx, m1, m2, n, A1, lda1, A2, lda2, U1, ldu1, U2, ldu2, V1, ldv1, theta, rank,
                                  info);
  return csd_rect_typed<z64>(ctx, m1, m2, n, A1, lda1, A2, lda2, U1, ldu1, U2, ldu2, V1, ldv1, theta, rank, info);
}

int csd_complete_v2(csd_ctx* ctx, int dtype, int n, const void* A3, int lda3, const void* A4, int lda4,
                    const void* U1, int ldu1, const void* U2, int ldu2, const double* theta, void* V2, int ldv2,
                    csd_info* info) {
  if (!ctx) return -1;
  if (dtype != CSD_F64 && dtype != CSD_C128) return -2;
  if (n < 1) return -3;
  if (!A3) return -4;
  if (lda3 < n) return -5;
  if (!A4) return -6;
  if (lda4 < n) return -7;
  if (!U1) return -8;
  if (ldu1 < n) return -9;
  if (!U2) return -10;
  if (ldu2 < n) return -11;
  if (!theta) return -12;
  if (!V2) return -13;
  if (ldv2 < n) return -14;
  if (info) std::memset(info, 0, sizeof(csd_info));
  if (dtype == CSD_F64)
    return complete_v2_typed<double>(ctx, n, A3, lda3, A4, lda4, U1, ldu1, U2, ldu2, theta, V2, ldv2, info);
  return complete_v2_typed<z64>(ctx, n, A3, lda3, A4, lda4, U1, ldu1, U2, ldu2, theta, V2, ldv2, info);
}

int csd_set_theta_mode(csd_ctx* ctx, int mode) {
  if (!ctx) return -1;
  if (mode != 0 && mode != 1) return -2;
  ctx->cx.theta_mode = mode;
  return CSD_OK;
}

int polar(csd_ctx* ctx, int dtype, int n, const void* A, int lda, void* W, int ldw, void* H, int ldh,
          csd_info* info) {
  if (!ctx) return -1;
  if (dtype != CSD_F64 && dtype != CSD_C128) return -2;
  if (n < 1) return -3;
  if (!A) return -4;
  if (lda < n) return -5;
  if (!W) return -6;
  if (ldw < n) return -7;
  if (H && ldh < n) return -9;
  if (info) std::memset(info, 0, sizeof(csd_info));
  if (dtype == CSD_F64) return polar_typed<double>(ctx, n, A, lda, W, ldw, H, ldh, info);
  return polar_typed<z64>(ctx, n, A, lda, W, ldw, H, ldh, info);
}

int heig(csd_ctx* ctx, int dtype, int n, const void* B, int ldb, double* lambda, void* V, int ldv, csd_info* info) {
  if (!ctx) return -1;
  if (dtype != CSD_F64 && dtype != CSD_C128) return -2;
  if (n < 1) return -3;
  if (!B) return -4;
  if (ldb < n) return -5;
  if (!lambda) return -6;
  if (!V) return -7;
  if (ldv < n) return -8;
  if (info) std::memset(info, 0, sizeof(csd_info));
  if (dtype == CSD_F64) return heig_typed<double>(ctx, n, B, ldb, lambda, V, ldv, info);
  return heig_typed<z64>(ctx, n, B, ldb, lambda, V, ldv, info);
}

const char* csd_status_str(int s) {
  if (s < 0) return "invalid argument";
  switch (s) {
    case CSD_OK: return "ok";
    case CSD_ERR_CUDA: return "CUDA error";
    case CSD_ERR_NOT_CONVERGED: return "Zolo-pd did not converge";
    case CSD_WARN_ALG2_RCHECK: return "Algorithm 2 check ||R~ - R|| above tolerance (outputs written)";
    case CSD_ERR_EIG_SPLIT: return "Zolo-eig could not split a block";
    case CSD_ERR_NONFINITE: return "input holds NaN or Inf";
    case CSD_ERR_ALLOC: return "device workspace allocation failed";
    case CSD_ERR_INTERNAL: return "internal error";
    case CSD_ERR_NO_DEVICE: return "no CUDA device";
    case CSD_ERR_DEVICE_TIMEOUT: return "a tensor-core wait on the device timed out";
    default: return "unknown status";
  }
}

}  // extern "C"
