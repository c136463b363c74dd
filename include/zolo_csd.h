/*
 * zolo_csd.h -- C ABI of the GB300 (sm_103a) Zolo-csd library.
 *
 * The library computes the CS decomposition of a 2n x n partial isometry
 * A = [A1; A2] (Section 1; Theorem 2.1 for the rank-deficient case) by the
 * method of Algorithm 1: two polar decompositions A_i = W_i H_i by Zolo-pd
 * (Section 5), the eigendecomposition of B = H2 - H1 + mu (I - A^*A)
 * (Section 3, line 4 of Algorithm 1) by the spectral divide-and-conquer
 * Zolo-eig (Section 5), and U_i = W_i V1, C/S = diag(V1^* H_i V1),
 * theta = atan2(S, C) (Algorithm 1 lines 6-9, remark (iii)).  Ill-conditioned
 * blocks use the eps-modified Zolo-pd with eps = 1e-15 and, when W_i is not
 * orthonormal, Algorithm 2; rank-deficient inputs use Algorithm 3, with
 * Algorithm 2's W_i for a block whose U_i = W_i V1 is not orthonormal (C or S
 * ill conditioned, Section 5.2).
 *
 * Conventions for every entry point
 *   - Matrices are column-major with leading dimension ld >= n.
 *   - dtype 0 = real FP64 (double), dtype 1 = complex FP64 (two doubles,
 *     real part first, C99 double complex layout).
 *   - Matrix and vector pointers may point to device memory or to host
 *     memory (pageable or pinned); the library inspects each pointer, stages
 *     host data through its own device buffers and copies results back.
 *   - The caller owns all input and output buffers; inputs are never
 *     modified.  The library owns its device workspace, which lives in the
 *     context, grows on demand and is released by csd_destroy.
 *   - Work is issued on the context's CUDA stream; on return all outputs are
 *     complete (the call synchronises the stream).
 *   - Return value: 0 on success; -k when argument k (1-based) is invalid;
 *     a positive CSD_ERR_* / CSD_WARN_* code otherwise (csd_status_str).
 *     A warning still writes every output.
 */
#ifndef ZOLO_CSD_H
#define ZOLO_CSD_H

#ifdef __cplusplus
extern "C" {
#endif

#define CSD_OK 0
#define CSD_ERR_CUDA 1            /* a CUDA call failed (context may be lost) */
#define CSD_ERR_NOT_CONVERGED 2   /* polar(): the Zolo-pd iterate did not converge (last iterate written) */
#define CSD_WARN_ALG2_RCHECK 3    /* Algorithm 2: ||R~ - R|| above tolerance (Section 5.1) */
#define CSD_ERR_EIG_SPLIT 4       /* Zolo-eig could not split a block after retries */
#define CSD_ERR_NONFINITE 5       /* input holds NaN or Inf */
#define CSD_ERR_ALLOC 6           /* device workspace allocation failed */
#define CSD_ERR_INTERNAL 7        /* internal consistency check failed */
#define CSD_ERR_NO_DEVICE 8       /* no usable CUDA device for the context */
#define CSD_ERR_DEVICE_TIMEOUT 9  /* a bounded wait inside a tensor-core kernel gave up */

#define CSD_F64 0
#define CSD_C128 1

typedef struct csd_ctx csd_ctx;

/* Diagnostics filled by every entry point (may be NULL). */
typedef struct {
  int status;             /* same as the return value */
  int rank;               /* detected rank r = round(||A||_F^2) (remark (vi)) */
  double mu;              /* 0 (full rank) or 2 (Algorithm 3) */
  int zolo_iters;         /* Zolo-pd iterations per polar decomposition (polar(): all passes) */
  int r_terms[4];         /* partial-fraction terms r of each iteration */
  double ell[4];          /* lower end l of [l, 1] entering each iteration */
  int chol_fallback;      /* Cholesky iterations redone in QR form */
  int alg2_used[2];       /* Algorithm 2 applied to block i (2: then the SVD polar fallback) */
  double orth_err[2];     /* ||W_i^* W_i - I||_F of the Zolo-pd factor (polar(): entry 0) */
  double rdiff[2];        /* ||R~_i - R_i||_F / ||R_i||_F (Algorithm 2 check) */
  int eig_splits;         /* Zolo-eig splits performed */
  int eig_retries;        /* splits redone with a perturbed shift */
  int eig_leaves;         /* leaf blocks solved by Jacobi */
  double eig_offblock;    /* largest ||B21||_F / ||B||_F accepted at a split */
  double ms_total;        /* wall time of the call, milliseconds */
} csd_info;

/* Create a context on CUDA device `device` bound to the CUDA stream
 * `stream` (a cudaStream_t; NULL = the legacy default stream).  *ctx
 * receives the handle.  Returns 0, -1/-2 on bad arguments, or
 * CSD_ERR_NO_DEVICE / CSD_ERR_CUDA. */
int csd_create(csd_ctx** ctx, int device, void* stream);

/* Rebind the context to another stream of the same device. */
int csd_set_stream(csd_ctx* ctx, void* stream);

/* Release the context and its device workspace.  NULL is accepted. */
int csd_destroy(csd_ctx* ctx);

/* Bytes of device workspace currently held by the context. */
long long csd_workspace_bytes(const csd_ctx* ctx);

/* CS decomposition (Algorithm 1; Algorithms 2 and 3 as needed).
 *   A1, A2   n x n blocks of A (lda1, lda2 >= n), read only.
 *   U1, U2   n x n outputs (ldu1, ldu2 >= n): columns 0..rank-1 hold the
 *            economical factors of Algorithm 3, the rest are unspecified.
 *   V1       n x n output (ldv1 >= n), same column convention.
 *   theta    length-n output: theta[0..rank-1] ascending in [0, pi/2]
 *            (remark (iii)); entries rank..n-1 are set to 0.
 *   rank     host int, receives r (may be NULL).
 * A1 = U1 diag(cos theta) V1^*, A2 = U2 diag(sin theta) V1^* up to the
 * backward error of Theorem 3.1. */
int csd_polar(csd_ctx* ctx, int dtype, int n,
              const void* A1, int lda1, const void* A2, int lda2,
              void* U1, int ldu1, void* U2, int ldu2, void* V1, int ldv1,
              double* theta, int* rank, csd_info* info);

/* CS decomposition with rectangular blocks: A1 is m1 x n, A2 is m2 x n,
 * m1, m2 >= n (a 2-block partial isometry, Section 2).  Each block is first
 * reduced by its Householder QR, A_i = Q_i R_i; [R1; R2] has orthonormal
 * columns (or is the same partial isometry) and goes through csd_polar's
 * path; U_i = Q_i U_i'.
 *   U1 (m1 x n, ldu1 >= m1), U2 (m2 x n, ldu2 >= m2): columns 0..rank-1
 *   hold the factors; V1 (n x n), theta (length n) and rank as in csd_polar.
 * Returns as csd_polar; -3 / -4 when m1 / m2 < n, -5 when n < 1. */
int csd_polar_rect(csd_ctx* ctx, int dtype, int m1, int m2, int n, const void* A1, int lda1, const void* A2,
                   int lda2, void* U1, int ldu1, void* U2, int ldu2, void* V1, int ldv1, double* theta, int* rank,
                   csd_info* info);

/* How csd_polar obtains theta (and C = cos theta, S = sin theta):
 *   mode 0 (default): theta = atan2(S, C) with C, S = diag(V1^* H_i V1)
 *                     (Algorithm 1 lines 8-9 and remark (iii));
 *   mode 1:           theta solves sin(theta) - cos(theta) = Lambda, i.e.
 *                     theta = pi/4 + asin(Lambda / sqrt(2)) (remark (iv)):
 *                     cheaper (no V1^* H_i V1), still backward stable, and
 *                     per the paper generally less accurate.
 * Returns 0, -1 (NULL context) or -2 (other mode). */
int csd_set_theta_mode(csd_ctx* ctx, int mode);

/* V2 of the complete 2 x 2 CS decomposition (remark (viii)): for a unitary
 * [A1 A3; A2 A4] (2n x 2n) whose first block column has the full-rank CSD
 * A1 = U1 C V1^*, A2 = U2 S V1^* (from csd_polar), computes
 * X = -A3^* U1 S + A4^* U2 C and its QR factorization X = Q R with
 * diag(R) >= 0, and writes V2 = Q, so that A3 = -U1 S V2^* and
 * A4 = U2 C V2^* up to the backward error.
 *   A3, A4   n x n blocks (lda3, lda4 >= n), read only.
 *   U1, U2   n x n factors from csd_polar (ldu1, ldu2 >= n), read only.
 *   theta    length n (host or device), C = cos theta, S = sin theta.
 *   V2       n x n output (ldv2 >= n), unitary.
 * Returns 0, -k for invalid argument k, or a CSD_ERR_* code. */
int csd_complete_v2(csd_ctx* ctx, int dtype, int n, const void* A3, int lda3, const void* A4, int lda4,
                    const void* U1, int ldu1, const void* U2, int ldu2, const double* theta, void* V2, int ldv2,
                    csd_info* info);

/* Polar decomposition A = W H by Zolo-pd (Section 5) on [eps, 1],
 * eps = 1e-15 (Section 5.1), for an n x n A with ||A||_2 <= 1 (as for the
 * blocks of a partial isometry; larger inputs are scaled by 1/||A||_F first).
 * W (ldw >= n) receives the unitary factor, H (ldh >= n) the Hermitian
 * factor sym(W^* A) (H may be NULL). */
int polar(csd_ctx* ctx, int dtype, int n, const void* A, int lda,
          void* W, int ldw, void* H, int ldh, csd_info* info);

/* Hermitian eigendecomposition B = V diag(lambda) V^* by Zolo-eig
 * (Section 5: spectral divide and conquer on the polar factor of B - sI).
 * The recursion runs level by level: the blocks of one level are split
 * together (batched Zolo-pd, QR and products, each block padded to its
 * group's size with an identity block).  Only the Hermitian part
 * (B + B^*)/2 is used.  lambda (length n) receives the eigenvalues
 * ascending, V (ldv >= n) the eigenvectors.  CSD_ERR_EIG_SPLIT when a block
 * cannot be split after its shifted retries. */
int heig(csd_ctx* ctx, int dtype, int n, const void* B, int ldb,
         double* lambda, void* V, int ldv, csd_info* info);

/* polar() without any allocation, for callers that cannot allocate device
 * memory: code running where cudaMalloc is unavailable or forbidden (for
 * instance inside a host callback or a memory-budgeted plug-in whose
 * allocations must all be made up front), or that must not add memory while
 * another component owns the device.  The paper has no counterpart: it is a
 * deployment variant of the Zolo-pd entry point.
 *   - n <= CSD_NOALLOC_MAX_N (64); a larger n returns -2.
 *   - A, W and H (H may be NULL) must be device pointers; a host pointer
 *     returns -3 / -5 / -7.  `stream` is a cudaStream_t (NULL = legacy default
 *     stream).  The call synchronises that stream before returning.
 *   - Scratch memory is one static device array of 6 MiB inside this library,
 *     which every GPU that loads the library holds until the process exits.
 *     The first call on a device looks up that array's device address (no
 *     allocation); make that first call before any stream capture.
 *   - The call calls no cudaMalloc, cudaFree or allocating library routine.
 *   - Every call shares the one scratch array and starts by writing all the
 *     scratch it reads, so nothing is carried over from the previous call;
 *     calls that overlap on the GPU (other threads or streams, same device)
 *     race on it and must be serialised by the caller.
 * Same results and status codes as polar() otherwise. */
#define CSD_NOALLOC_MAX_N 64
int polar_noalloc(int dtype, int n, const void* A, int lda, void* W, int ldw, void* H, int ldh, void* stream);

/* Zolotarev coefficients for [ell, 1] and r terms (host only, no GPU):
 * c[0..2r-1] = c_1..c_2r, a[0..r-1] = a_1..a_r, *mhat (Z(1) = 1) and
 * *ell_next = Z(ell).  0 < ell < 1, 1 <= r <= 16.  Returns 0 or -k. */
int zolo_coeffs(double ell, int r, double* c, double* a, double* mhat, double* ell_next);

/* Iteration plan of Zolo-pd from ell0 (host only): at each step the
 * smallest r <= rmax with 1 - ell_next <= 4u, else rmax; stops once
 * 1 - ell <= 4u.  r_out/ell_out (length max_iter) receive r and the entering
 * ell of each step; returns the number of steps (or -k). */
int zolo_plan(double ell0, int rmax, int max_iter, int* r_out, double* ell_out);

/* Kernel accounting, for roofline reports (not needed for computing).
 * Kinds: 0 = GEMM (FP64 FMA tiles), 1 = Householder QR panel, 2 = Cholesky
 * diagonal block, 3 = Jacobi leaves, 4 = tensor-core FP64 GEMM (sliced BF16
 * products on tcgen05; `flops` counts the FP64-equivalent 2mnk).  While enabled, each launch of these
 * kernels is bracketed by CUDA events on the context stream; `flops` sums
 * the multiply-add work each launch executes (2 per real FMA, 8 per complex
 * FMA; QR panel and Cholesky block use their textbook counts).
 * csd_profile_enable resets the counters; csd_profile_read synchronises the
 * stream and returns the totals since then. */
typedef struct {
  long long count[5];
  double ms[5];
  double flops[5];
  /* GEMM launches split by call site (0 other, 1-3 QR panel update, 4-6 Q
   * formation, 7 Zolotarev term sum, 8 Gram matrix, 9-10 Cholesky, 11-14
   * triangular solves, 15 H, 16 orthogonality check, 17 Zolo-eig,
   * 18 assembly, 19 Algorithm 2, 20 merging of the blocked QR's WY factors,
   * 21 rows of the dense block X in the trailing update of the stacked
   * [X; sqrt(c) I] QR factorization; site 3 holds the rows below it;
   * 22 csd_polar_backward) */
  long long site_count[24];
  double site_ms[24];
  double site_flops[24];
} csd_profile;

int csd_profile_enable(csd_ctx* ctx, int enable);

/* Run the real FP64 matrix products of this context on the tcgen05 tensor
 * cores instead of the FP64 FMA pipe.  enable = 0 (the default) keeps every
 * product on the FP64 pipe; otherwise bit s of `enable` selects the products
 * of call site s (the site numbering of csd_profile); enable = -1 selects
 * every site.
 * The products stay FP64-accurate: each operand is split exactly into seven
 * BF16 slices with per-row / per-column power-of-two scaling, the slice
 * products are accumulated exactly (FP32 over 128 k, then a 64-bit integer)
 * except the smallest ones (error of the same order as an FP64 product).
 * The rows below X in the trailing update of the stacked [X; sqrt(c) I]
 * factorization (site 3) are of the size of sqrt(c) and need accuracy
 * relative to themselves: that product is also balanced along its inner
 * dimension by powers of two (A D, D^-1 B, D = diag of the row maxima of B).
 * Complex products with real alpha and beta run as two real grouped sums
 * over the interleaved parts (Re C = Re A Re B - Im A Im B,
 * Im C = Re A Im B + Im A Re B); grouped complex sums and the balanced
 * product stay on the FP64 pipe.  Returns 0 or -1 (NULL context). */
int csd_set_tensor_cores(csd_ctx* ctx, int enable);
int csd_profile_read(csd_ctx* ctx, csd_profile* out);

/* Leaf size of Zolo-eig's spectral divide and conquer (Section 5): blocks of
 * at most `leaf` rows (1..1024, default 256) are not split further but
 * diagonalised by two-sided cyclic Jacobi (parallel tournament order), all
 * leaves of a call batched into the same launches, one CTA per column pair
 * and round; when every leaf has at most 64 rows, one CTA per leaf runs the
 * whole iteration in shared memory.  The paper leaves the recursion's
 * stopping size open.
 * Returns 0, -1 (NULL context) or -2 (out of range). */
int csd_set_eig_leaf(csd_ctx* ctx, int leaf);

/* Mixed precision on the tensor-core path (csd_set_tensor_cores): once the
 * first, QR-form iteration has mapped the singular values into
 * [l_1, 1] = [0.4565, 1], the Cholesky-form iteration works on a well
 * conditioned X, and its Gram product X^* X and the products of its paired
 * triangular solves may run with `slices` = 5 or 6 BF16 slices per operand
 * (40 or 48 bits, 15 or 21 slice products instead of 28) while the QR
 * iteration, the Cholesky factorizations, H_i, B, Zolo-eig's subspace
 * products and the assembly keep 7 (FP64-accurate).  scope bit 0: the two
 * polar decompositions of csd_polar (and polar()); bit 1: the polar
 * decompositions inside Zolo-eig.  slices = 7 or scope = 0 is the default
 * FP64-accurate path.  The result is checked like any other: angles,
 * backward error and orthogonality against the 50 n u bar.
 * Returns 0, -1 (NULL context), -2 (slices not 5..7), -3 (unknown scope bit). */
int csd_set_mixed_precision(csd_ctx* ctx, int slices, unsigned scope);

/* Fallback of Algorithm 2 (Section 5.1): when ||R~_i - R_i||_F / ||R_i||_F
 * (the backward error of W_i H~_i, info->rdiff) reaches factor * n * u, the
 * polar decomposition of A_i is recomputed through the SVD (one-sided
 * Jacobi, W_i = U V^*, H_i = sym(W_i^* A_i)), which is unconditionally
 * backward stable, and info->alg2_used[i] = 2.  Default factor 1e3; 0 makes
 * every block that takes Algorithm 2 use the SVD; a negative factor
 * disables the fallback, and a block above 1e3 n u then returns
 * CSD_WARN_ALG2_RCHECK as a warning.  The SVD costs O(n^3) per sweep and
 * some ten sweeps.  Returns 0, -1 (NULL context) or -2 (NaN). */
int csd_set_alg2_fallback(csd_ctx* ctx, double factor);

/* Column convention of csd_polar's factors.  The CSD leaves each column
 * pair (U1, U2, V1)[:, j] free up to a common sign (a common phase when
 * complex) for distinct angles.  mode 0 (default) keeps what the
 * algorithm produces; mode 1 scales column j so that the entry of V1[:, j]
 * of largest magnitude (first such index) is real and positive, which makes
 * the factors unique for distinct angles and hence differentiable functions
 * of A (needed by csd_polar_backward's callers that put a loss on U1, U2 or
 * V1).  Returns 0, -1 (NULL context) or -2. */
int csd_set_sign_convention(csd_ctx* ctx, int mode);

/* Reverse-mode derivative of csd_polar for a real, full-rank input (the
 * paper has no derivatives: this is the adjoint of Algorithm 1's steps).
 * Given the forward's outputs U1, U2, V1 (n x n), theta (length n) and the
 * gradients gU1, gU2, gV1 (n x n), gtheta (length n) of a scalar loss --
 * any of them NULL for zero -- writes gA1, gA2 (n x n) = dLoss/dA1, dA2.
 * It uses that at a partial isometry H1 = V1 diag(cos theta) V1^T and
 * H2 = V1 diag(sin theta) V1^T (Section 3) and W_i = U_i V1^T, so both polar
 * adjoints (the Lyapunov equations H dX + dX H = ..., solved by division by
 * sigma_k + sigma_l) and the eigenvector adjoint of B = H2 - H1 (division by
 * lambda_l - lambda_k, lambda = sin theta - cos theta) are elementwise in
 * the basis V1: seven n x n x n products and one elementwise kernel; the
 * forward's iterates are not needed.  Defined for distinct angles in
 * (0, pi/2); a repeated angle contributes no eigenvector term (the
 * eigenvectors are not unique there), an angle at 0 or pi/2 no polar term.
 * For a loss on U1, U2 or V1, run the forward with csd_set_sign_convention
 * mode 1.  Pointers may be device or host memory.  dtype must be CSD_F64
 * (else -2).  Returns 0, -k for invalid argument k, or a CSD_ERR_* code. */
int csd_polar_backward(csd_ctx* ctx, int dtype, int n, const void* U1, int ldu1, const void* U2, int ldu2,
                       const void* V1, int ldv1, const double* theta, const void* gU1, int ldgu1, const void* gU2,
                       int ldgu2, const void* gV1, int ldgv1, const double* gtheta, void* gA1, int ldga1, void* gA2,
                       int ldga2, csd_info* info);

/* Zolo-pd iteration control of polar() (Section 5).
 *   max_extra_passes (0..4, default 1): Section 5's two iterations on
 *     [eps, 1] converge exactly when every singular value of the (scaled)
 *     input is at least eps = 1e-15; polar() tests ||W^* W - I||_F <= 50 n u
 *     afterwards and, when that fails, runs the iteration plan again on the
 *     current iterate, up to this many times.  If the test still fails the
 *     call returns CSD_ERR_NOT_CONVERGED with the last iterate in W (and the
 *     matching H): A is then singular to working precision and has no
 *     unitary polar factor that the iteration can reach.
 *   stop_after (default 0): k > 0 makes polar() return the iterate X_k
 *     after k iterations instead of the polar factor (no convergence test),
 *     so that callers can check X_k = U Z_k(Sigma) V^*: Zolo-pd's iterates
 *     share the singular vectors of A (Section 5).
 * csd_polar, heig and csd_polar_rect are unaffected: in the CS
 * decomposition an unconverged factor takes Algorithm 2 (Section 5.1).
 * Returns 0, -1 (NULL context), -2 / -3 (out of range). */
int csd_set_zolo_control(csd_ctx* ctx, int max_extra_passes, int stop_after);

/* Test hooks (all off by default; none changes results when off).
 *   flags & CSD_TEST_REJECT_EIG_SPLITS: Zolo-eig rejects every split
 *     attempt, so a call that needs one retries with every shifted split
 *     (Section 5's spectral divide and conquer) and then returns
 *     CSD_ERR_EIG_SPLIT with info->eig_retries filled in.
 *   tc_probe_wait > 0: every tensor-core kernel launch first polls, this
 *     many times, an mbarrier that nothing signals, before it issues any
 *     copy or MMA; the wait runs out, the launch writes NaN outputs, sets
 *     the device error flag and the call returns CSD_ERR_DEVICE_TIMEOUT.
 *     The context stays usable.
 *   tc_flush_every > 0: the tensor-core kernel writes its 64-bit integer
 *     partial sum out to C every this many 128-k drains (default: every
 *     120 drains, i.e. only for K > 15 360).
 * Returns 0, -1 (NULL context), -2 (unknown flag), -3 / -4 (negative). */
#define CSD_TEST_REJECT_EIG_SPLITS 1u
int csd_set_test_hooks(csd_ctx* ctx, unsigned flags, long long tc_probe_wait, int tc_flush_every);

/* C = alpha op(A) op(B) + beta C in real FP64 on this library's product
 * kernels: engine 0 = the FP64-pipe tiles, engine 1 = the tensor-core kernel
 * (exact BF16 slicing, FP64-accurate; any m, n, k).  The building block of
 * every step of Zolo-pd and Zolo-eig; it is not itself a step of the paper.
 *   opA, opB: 0 = N, 1 = T.  A (lda >= rows of A), B (ldb), C (ldc >= m)
 *   are column-major DEVICE pointers (a host pointer returns -8/-10/-13).
 * Returns 0, -k for invalid argument k, or CSD_ERR_DEVICE_TIMEOUT /
 * CSD_ERR_CUDA / CSD_ERR_ALLOC. */
int csd_gemm(csd_ctx* ctx, int opA, int opB, int m, int n, int k, double alpha, const double* A, int lda,
             const double* B, int ldb, double beta, double* C, int ldc, int engine);

/* FP64 peak microbenchmark (the FP64 roofline's denominator; not a step of
 * the paper): kind 0 = DFMA loop on the FMA pipe, kind 1 = mma.sync
 * m8n8k4 f64 loop, 8 CTAs of 256 threads per SM, 8 independent chains per
 * thread; best of 10 timed launches (CUDA events) after one warm-up.
 * *tflops receives the rate, *ms (may be NULL) the best launch time.
 * Allocates and frees a small device buffer.  Returns 0, -k for invalid
 * argument k, or CSD_ERR_CUDA / CSD_ERR_ALLOC. */
int csd_fp64_peak(int device, int kind, double* tflops, double* ms);

/* Batched CS decompositions: many real FP64 CSDs of different sizes
 * (n_i <= 1024, full rank) in one CUDA-graph launch.  Independent problems
 * batched on one GPU, as the paper batches the two polar decompositions and
 * the r partial-fraction terms of Zolo-pd (Section 3, remark (ii)).
 * Per instance: Zolo-pd for both blocks (identity-padded to the instance's
 * size bucket; the padding stays exactly decoupled), B = H2 - H1, its
 * eigendecomposition by the batched Jacobi leaf solver (one leaf per
 * instance, at its own size), C, S, theta = atan2(S, C), U_i = W_i V1 and
 * the ascending order (Algorithm 1).  No Algorithm 2 or 3 branch: an
 * instance whose angles come out non-finite reports CSD_ERR_INTERNAL in
 * status[i], one whose Jacobi leaf still rotated in its last sweep (30
 * sweeps, a converged leaf stops rotating) CSD_ERR_NOT_CONVERGED; callers
 * with rank-deficient or ill-conditioned blocks use csd_polar.
 *
 * Packed layout (all device pointers): instance i's n_i x n_i matrices are
 * column-major with leading dimension n_i at element offset
 * sum_{j<i} n_j^2 of A1, A2, U1, U2 and V1; its angles at sum_{j<i} n_j of
 * theta.  The plan keeps the sizes; the first csd_batch_run autotunes the
 * bucket granularity (16, 32 or 64) and, per bucket, the product engine
 * (FP64-pipe tiles or tensor-core tiles) by timing each on the caller's
 * data, runs once outside a capture, then captures the whole batch into a
 * CUDA graph; later runs on the same buffers only launch the graph (new
 * buffers are captured again).  status (host, count ints, may be NULL)
 * receives 0, CSD_ERR_NOT_CONVERGED or CSD_ERR_INTERNAL per instance.  The plan owns its device
 * workspace (grown on demand) and uses the context's stream; destroy the
 * plan before the context.
 * create returns 0, -1 (NULL context), -2 (count < 1), -3 (bad sizes),
 * -4 (NULL plan pointer) or CSD_ERR_ALLOC; run returns 0, -k, or a
 * CSD_ERR_* code. */
typedef struct csd_batch csd_batch;
int csd_batch_create(csd_ctx* ctx, int count, const int* n, csd_batch** plan);
int csd_batch_run(csd_batch* plan, const double* A1, const double* A2, double* U1, double* U2, double* V1,
                  double* theta, int* status);
int csd_batch_destroy(csd_batch* plan);
/* Autotuner outcome: bucket granularity, number of buckets, buckets on the
 * tensor cores, and the timed batch (ms) for granularity 16, 32, 64. */
int csd_batch_stats(const csd_batch* plan, int* granularity, int* buckets, int* tc_buckets, double* tune_ms);

/* Process-wide number of kernels this library has launched so far. */
long long csd_launch_count(void);

/* Human-readable text of a status code. */
const char* csd_status_str(int status);

#ifdef __cplusplus
}
#endif
#endif /* ZOLO_CSD_H */
