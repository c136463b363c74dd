// Host launchers of the library's CUDA kernels (all asynchronous on `st`).
// Every matrix argument is a device pointer to column-major data with the
// given leading dimension; batched launchers take element strides between
// consecutive problems.
#pragma once
#include "common.cuh"

namespace zcsd {

enum Op { OP_N = 0, OP_T = 1, OP_C = 2 };

// Structural k-range restrictions of a GEMM tile (bit flags): the product
// skips k outside [kb, ke) where kb/ke follow the output tile position.
enum KFlags {
  K_FROM_COL = 1,  // k >= first column of the tile (op(B)[k,j] = 0 for k < j)
  K_FROM_ROW = 2,  // k >= first row of the tile    (op(A)[i,k] = 0 for k < i)
  K_TO_COL = 4,    // k <  last column + 1           (op(B)[k,j] = 0 for k > j)
  K_TO_ROW = 8,    // k <  last row + 1              (op(A)[i,k] = 0 for k > i)
};

constexpr int MAX_SUM = 16;

// Call sites of the GEMM, for per-site kernel accounting.
enum GemmSite {
  GS_OTHER = 0, GS_QR_W, GS_QR_W2, GS_QR_UPD, GS_FQ_W, GS_FQ_W2, GS_FQ_UPD, GS_ZOLO_COMBINE, GS_GRAM,
  GS_CHOL_ROW, GS_CHOL_TRAIL, GS_TRSM_F_UPD, GS_TRSM_F_DIAG, GS_TRSM_B_UPD, GS_TRSM_B_DIAG, GS_H, GS_ORTH,
  GS_EIG, GS_ASSEMBLY, GS_ALG2, GS_TMERGE, GS_QR_UPD_X, GS_GRAD, GS_SITES
};

template <class T>
struct GemmArgs {
  int m = 0, n = 0, k = 0;
  int opA = OP_N, opB = OP_N;
  const T* A = nullptr; int lda = 1; long long sA = 0, sAj = 0;
  const T* B = nullptr; int ldb = 1; long long sB = 0, sBj = 0;
  const T* Cin = nullptr; int ldcin = 1; long long sCin = 0;
  T* C = nullptr; int ldc = 1; long long sC = 0;
  T alpha{}; T beta{};
  int nsum = 1;                 // C = alpha * sum_j w_j op(A_j) op(B_j) + beta * Cin
  double w[MAX_SUM];            // per-term real weights (w_j = 1 when unset)
  int batch = 1;
  int bdivA = 1, bdivB = 1, bdivC = 1;  // problem b uses A_{b / bdivA}, B_{b / bdivB}, Cin_{b / bdivC}
  int uplo = 0;                 // 0 all tiles, 1 only tiles touching the upper triangle, 2 lower
  int kflags = 0;
  int site = 0;                 // call-site label for kernel accounting (GemmSite)
  int ksplit = 1;               // split-K: problem b, part s writes C_{b*ksplit+s} (Cin/beta only in part 0)
  int kbal = 0;                 // tensor-core path: balance the inner dimension by the row maxima of op(B)
  int es = 1;                   // tensor-core path: element stride in doubles of A, B, Cin, C (2: one part of
                                // interleaved complex data; ld and problem strides stay in elements)
  GemmArgs() { for (int i = 0; i < MAX_SUM; ++i) w[i] = 1.0; }
};

template <class T> void gemm(const GemmArgs<T>& g, cudaStream_t st);

// Convenience wrapper: C = alpha op(A) op(B) + beta C (single problem).
template <class T>
void gemm1(cudaStream_t st, int opA, int opB, int m, int n, int k, T alpha, const T* A, int lda,
           const T* B, int ldb, T beta, T* C, int ldc, int uplo = 0, int kflags = 0, int site = 0);

// ---- elementwise (batched; `batch` problems at strides s*)
// Y = alpha X (+ beta Y when beta != 0)
template <class T> void axpby(cudaStream_t st, int m, int n, double alpha, const T* X, int ldx, long long sX,
                              double beta, T* Y, int ldy, long long sY, int batch);
// X_{b parts} += sum_{s=1}^{parts-1} X_{b parts + s}: fold split-K partial
// products (part s of problem b at X + (b parts + s) sPart) into part 0
template <class T> void sum_parts(cudaStream_t st, int m, int n, T* X, int ldx, long long sPart, int parts, int batch);
// Y_j = X + shift_j I for j < nterms (shifts on device or by value), Y_j at stride sY
template <class T> void shift_terms(cudaStream_t st, int n, const T* X, int ldx, long long sXb,
                                    const double* shifts, int nterms, T* Y, int ldy, long long sY, int batch);
// M_j = [X; sqrt(c_j) I] (2n x n, ld = ldm), for j < nterms of each of `batch` X's
template <class T> void stack_terms(cudaStream_t st, int n, const T* X, int ldx, long long sXb,
                                    const double* sqrtc, int nterms, T* M, int ldm, long long sM, int batch);
// X2 = mhat (X1 + sum_j a_j T_j)
template <class T> void sum_terms(cudaStream_t st, int n, double mhat, const T* X1, int ldx, long long sXb,
                                  const double* a, int nterms, const T* Tm, int ldt, long long sT,
                                  T* X2, int ldx2, long long sX2b, int batch);
// H = (Y + Y^*)/2 (in place allowed)
template <class T> void symmetrize(cudaStream_t st, int n, const T* Y, int ldy, long long sY, T* H, int ldh,
                                   long long sH, int batch);
// E = [I; 0] (m x n)
template <class T> void set_eye(cudaStream_t st, int m, int n, T* E, int lde, long long sE, int batch);

// ---- reductions (deterministic fixed-order; result written to device `out`)
// out[b] = sum |X_b - shift I|^2 over the m x n block (shift subtracted on the diagonal)
template <class T> void fro2(cudaStream_t st, int m, int n, const T* X, int ldx, long long sX, double shift,
                             double* out, int batch, double* scratch);
// out[0] = number of non-finite entries (as double)
template <class T> void count_nonfinite(cudaStream_t st, int m, int n, const T* X, int ldx, double* out,
                                        double* scratch);
// d[j] = Re sum_i conj(V_ij) Y_ij
template <class T> void col_dots(cudaStream_t st, int m, int n, const T* V, int ldv, const T* Y, int ldy, double* d);
// trace of the real part, diag copy
template <class T> void diag_real(cudaStream_t st, int n, const T* X, int ldx, double* d);
// theta_j = atan2(S_j, C_j); perm = ascending order of key (ties by index)
void theta_from_cs(cudaStream_t st, int n, const double* C, const double* S, double* theta);
// theta = pi/4 + asin(Lambda / sqrt(2)) (remark (iv)), clamped to [0, pi/2]
void theta_from_lambda(cudaStream_t st, int n, const double* lam, double* theta);
void sort_perm(cudaStream_t st, int n, const double* key, int* perm);
// Y[:, j] = X[:, perm[j]] for j < ncols
template <class T> void gather_cols(cudaStream_t st, int m, int ncols, const T* X, int ldx, const int* perm,
                                    T* Y, int ldy);
void gather_vec(cudaStream_t st, int n, const double* x, const int* perm, double* y);
// Gaussian N(0,1) entries from a counter-based generator (splitmix64 + Box-Muller)
template <class T> void randn(cudaStream_t st, int m, int n, T* X, int ldx, unsigned long long seed);

// ---- factorizations
// Householder QR panel (one CTA per problem): columns [k0, k0+nb) of M_b; column
// k's reflector spans rows [k, min(m, k + band)).  Writes R/V into M, the
// explicit unit-lower V panel into Y (rows [k0, k0+h), ld = ldy, stride sY),
// tau, and the nb x nb upper triangular T of Q = I - V T V^* (ld = nbmax).
template <class T> void qr_panel(cudaStream_t st, int m, int n, int band, T* M, int ldm, long long sM,
                                 int k0, int nb, T* Y, int ldy, long long sY, T* Tf, long long sT, int batch);
// Upper Cholesky R^* R = A_kk of the nb x nb diagonal block at (k0, k0) and
// its inverse R^{-1} (written to Rinv, ld = nb_ld, zeros below the diagonal).
// info[b] is set to (k0 + j + 1) at the first non-positive pivot.
template <class T> void potrf_inv(cudaStream_t st, int n, T* A, int lda, long long sA, int k0, int nb,
                                  T* Rinv, int ldr, long long sR, int* info, int batch);
}  // namespace zcsd
