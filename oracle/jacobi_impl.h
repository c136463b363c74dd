/*
 * Oracle (test infrastructure only; never on the product path).
 *
 * Scalar-generic body of the two Jacobi sub-solvers the oracle uses in place
 * of Zolo-pd and Zolo-eig.  Included twice by jacobi.c: once with SCALAR =
 * double (suffix _d) and once with SCALAR = double complex (suffix _z).
 *
 *  - one-sided (Hestenes) Jacobi SVD: the columns of G are rotated pairwise
 *    until every pair is orthogonal to working precision; the accumulated
 *    rotations form V, the column norms are the singular values and the
 *    normalised columns are U.  This gives the polar factors W = U V^*,
 *    H = V Sigma V^* of Section 1 (the decompositions A_i = W_i H_i).
 *  - cyclic two-sided Jacobi for a Hermitian B: plane rotations J^* B J that
 *    annihilate one off-diagonal pair at a time until off(B) <= u ||B||_F.
 *
 * Both sweep over column pairs in round-robin (tournament) order, so the
 * n/2 rotations of one round act on disjoint index pairs; they commute and
 * each one's 2x2 data is untouched by the others, which makes the parallel
 * round exactly equal to applying the same rotations one after another.
 */
#define CAT2(a, b) a##b
#define CAT(a, b) CAT2(a, b)
#define FN(name) CAT(name, SUFFIX)

/* pair (p,q) of round `rd` in a round-robin schedule on nn (even) players */
static void FN(rr_pair)(int nn, int rd, int k, int* p, int* q) {
  /* player nn-1 is fixed; the others rotate */
  int a, b;
  if (k == 0) { a = nn - 1; b = rd % (nn - 1); }
  else { a = (rd + k) % (nn - 1); b = (rd - k + (nn - 1)) % (nn - 1); }
  if (a < b) { *p = a; *q = b; } else { *p = b; *q = a; }
}

/* x^* y in twice the working precision (Dot2 of Ogita, Rump and Oishi,
 * "Accurate sum and dot product", SIAM J. Sci. Comput. 26, 2005: error-free
 * TwoProduct by fma and TwoSum, with the error terms summed separately),
 * so the orthogonality test below sees the true inner product to ~u. */
static SCALAR FN(dot2)(int m, const SCALAR* x, const SCALAR* y) {
  double s[2] = {0, 0}, c[2] = {0, 0};
  for (int i = 0; i < m; ++i) {
    double xr = CREAL(x[i]), xi = CIMAG(x[i]), yr = CREAL(y[i]), yi = CIMAG(y[i]);
    /* real part: xr yr + xi yi;  imaginary part: xr yi - xi yr */
    double a[4] = {xr, xi, xr, -xi}, b[4] = {yr, yi, yi, yr};
    for (int t = 0; t < (IS_COMPLEX ? 4 : 1); ++t) {
      int k = t >> 1;
      double p = a[t] * b[t];
      double e = fma(a[t], b[t], -p);
      double s1 = s[k] + p;
      double z = s1 - s[k];
      double q = (s[k] - (s1 - z)) + (p - z);
      s[k] = s1;
      c[k] += q + e;
    }
  }
  return MAKE(s[0] + c[0], s[1] + c[1]);
}

/* One-sided Jacobi SVD of the m x n matrix G (overwritten by U Sigma).
 * V (n x n) receives the right singular vectors, sigma the column norms.
 * Returns the number of sweeps used, or -1 if max_sweeps was reached. */
int FN(oracle_jacobi_svd)(int m, int n, SCALAR* G, int ldg, SCALAR* V, int ldv,
                          double* sigma, int max_sweeps, int nthreads) {
  const double u = 0x1p-53;
  /* rotation threshold: pairs whose cosine is below max(JTOL, sqrt(m)) u
   * are left alone; a sweep without rotations ends the iteration.  The
   * inner product itself is accurate to ~u (dot2), but every rotation of a
   * sweep rounds its two columns, which leaves cosines of order sqrt(m) u
   * between columns; a fixed threshold of a few u is then never met for
   * large m (the sweeps cycle).  sqrt(m) u is the threshold of LAPACK's
   * one-sided Jacobi SVD (xGESVJ, Drmac and Veselic 2008). */
  const double tol = (JTOL > sqrt((double)m) ? JTOL : sqrt((double)m)) * u;
  for (int j = 0; j < n; ++j)
    for (int i = 0; i < n; ++i) V[i + (size_t)j * ldv] = (i == j) ? 1.0 : 0.0;
  int nn = n + (n & 1); /* add a phantom column when n is odd */
  int sweeps = 0, converged = (n <= 1);
  while (!converged && sweeps < max_sweeps) {
    long rotations = 0;
    for (int rd = 0; rd < nn - 1; ++rd) {
#pragma omp parallel for num_threads(nthreads) reduction(+ : rotations) schedule(static)
      for (int k = 0; k < nn / 2; ++k) {
        int p, q;
        FN(rr_pair)(nn, rd, k, &p, &q);
        if (q >= n) continue; /* paired with the phantom column */
        SCALAR* gp = G + (size_t)p * ldg;
        SCALAR* gq = G + (size_t)q * ldg;
        double alpha = 0, beta = 0;
        for (int i = 0; i < m; ++i) {
          alpha += ABS2(gp[i]);
          beta += ABS2(gq[i]);
        }
        SCALAR gamma = FN(dot2)(m, gp, gq);
        double ag = CABS(gamma);
        if (ag == 0.0 || ag <= tol * sqrt(alpha) * sqrt(beta)) continue;
        SCALAR ph = gamma / ag; /* e^{i phi} */
        double zeta = (beta - alpha) / (2.0 * ag);
        double t = (zeta >= 0 ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
        double c = 1.0 / sqrt(1.0 + t * t), s = c * t;
        /* Rutishauser's form of the rotation, c a - s b = a - s (b + tau a)
         * with tau = s / (1 + c), keeps the O(s^2) part of c - 1 that is lost
         * when c rounds to 1, so norms do not drift over many rotations. */
        double tau = s / (1.0 + c);
        SCALAR phc = CONJ(ph);
        for (int i = 0; i < m; ++i) {
          SCALAR a = gp[i], b = phc * gq[i];
          gp[i] = a - s * (b + tau * a);
          gq[i] = b + s * (a - tau * b);
        }
        SCALAR* vp = V + (size_t)p * ldv;
        SCALAR* vq = V + (size_t)q * ldv;
        for (int i = 0; i < n; ++i) {
          SCALAR a = vp[i], b = phc * vq[i];
          vp[i] = a - s * (b + tau * a);
          vq[i] = b + s * (a - tau * b);
        }
        rotations += 1;
      }
    }
    ++sweeps;
    converged = (rotations == 0);
  }
  for (int j = 0; j < n; ++j) {
    double s2 = 0;
    for (int i = 0; i < m; ++i) s2 += ABS2(G[i + (size_t)j * ldg]);
    sigma[j] = sqrt(s2);
  }
  return converged ? sweeps : -1;
}

/* Cyclic Jacobi eigendecomposition of the Hermitian n x n matrix B
 * (overwritten; its diagonal ends up holding the eigenvalues).
 * V receives the eigenvectors.  Returns sweeps used, or -1. */
int FN(oracle_jacobi_eig)(int n, SCALAR* B, int ldb, SCALAR* V, int ldv,
                          double* lambda, int max_sweeps, int nthreads) {
  const double u = 0x1p-53;
  for (int j = 0; j < n; ++j)
    for (int i = 0; i < n; ++i) V[i + (size_t)j * ldv] = (i == j) ? 1.0 : 0.0;
  /* make the input exactly Hermitian: average with its conjugate transpose */
  for (int j = 0; j < n; ++j) {
    B[j + (size_t)j * ldb] = CREAL(B[j + (size_t)j * ldb]);
    for (int i = j + 1; i < n; ++i) {
      SCALAR x = 0.5 * (B[i + (size_t)j * ldb] + CONJ(B[j + (size_t)i * ldb]));
      B[i + (size_t)j * ldb] = x;
      B[j + (size_t)i * ldb] = CONJ(x);
    }
  }
  double fro2 = 0;
  for (int j = 0; j < n; ++j)
    for (int i = 0; i < n; ++i) fro2 += ABS2(B[i + (size_t)j * ldb]);
  double tol = u * sqrt(fro2);
  int nn = n + (n & 1);
  int sweeps = 0, converged = (n <= 1);
  double prev_off = INFINITY;
  double* cs = (double*)malloc(sizeof(double) * 2 * (nn / 2 + 1));
  SCALAR* ph = (SCALAR*)malloc(sizeof(SCALAR) * (nn / 2 + 1));
  int* pp = (int*)malloc(sizeof(int) * 2 * (nn / 2 + 1));
  while (!converged && sweeps < max_sweeps) {
    for (int rd = 0; rd < nn - 1; ++rd) {
      /* 1. rotation parameters for every pair of this round, from the current B */
      for (int k = 0; k < nn / 2; ++k) {
        int p, q;
        FN(rr_pair)(nn, rd, k, &p, &q);
        pp[2 * k] = p; pp[2 * k + 1] = q;
        cs[2 * k] = 1.0; cs[2 * k + 1] = 0.0; ph[k] = 1.0;
        if (q >= n) continue;
        SCALAR bpq = B[p + (size_t)q * ldb];
        double abpq = CABS(bpq);
        if (abpq == 0.0) continue;
        double bpp = CREAL(B[p + (size_t)p * ldb]), bqq = CREAL(B[q + (size_t)q * ldb]);
        double tau = (bqq - bpp) / (2.0 * abpq);
        double t = (tau >= 0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
        double c = 1.0 / sqrt(1.0 + t * t);
        cs[2 * k] = c; cs[2 * k + 1] = t * c; ph[k] = bpq / abpq;
      }
      /* 2. columns:  B <- B J,  V <- V J  with J = [[c, s], [-s e^{-i phi}, c e^{-i phi}]]
       * (Rutishauser's form, see the one-sided solver) */
#pragma omp parallel for num_threads(nthreads) schedule(static)
      for (int k = 0; k < nn / 2; ++k) {
        int p = pp[2 * k], q = pp[2 * k + 1];
        if (q >= n || cs[2 * k + 1] == 0.0) continue;
        double c = cs[2 * k], s = cs[2 * k + 1], tau = s / (1.0 + c);
        SCALAR phc = CONJ(ph[k]);
        SCALAR* bp = B + (size_t)p * ldb; SCALAR* bq = B + (size_t)q * ldb;
        for (int i = 0; i < n; ++i) {
          SCALAR a = bp[i], b = phc * bq[i];
          bp[i] = a - s * (b + tau * a);
          bq[i] = b + s * (a - tau * b);
        }
        SCALAR* vp = V + (size_t)p * ldv; SCALAR* vq = V + (size_t)q * ldv;
        for (int i = 0; i < n; ++i) {
          SCALAR a = vp[i], b = phc * vq[i];
          vp[i] = a - s * (b + tau * a);
          vq[i] = b + s * (a - tau * b);
        }
      }
      /* 3. rows:  B <- J^* B  (row p <- c row_p - s e^{i phi} row_q, row q <- s row_p + c e^{i phi} row_q) */
#pragma omp parallel for num_threads(nthreads) schedule(static)
      for (int k = 0; k < nn / 2; ++k) {
        int p = pp[2 * k], q = pp[2 * k + 1];
        if (q >= n || cs[2 * k + 1] == 0.0) continue;
        double c = cs[2 * k], s = cs[2 * k + 1], tau = s / (1.0 + c);
        SCALAR phk = ph[k];
        for (int j = 0; j < n; ++j) {
          SCALAR a = B[p + (size_t)j * ldb], b = phk * B[q + (size_t)j * ldb];
          B[p + (size_t)j * ldb] = a - s * (b + tau * a);
          B[q + (size_t)j * ldb] = b + s * (a - tau * b);
        }
        /* the annihilated pair is zero in exact arithmetic; keep B Hermitian */
        B[p + (size_t)q * ldb] = 0.0;
        B[q + (size_t)p * ldb] = 0.0;
        B[p + (size_t)p * ldb] = CREAL(B[p + (size_t)p * ldb]);
        B[q + (size_t)q * ldb] = CREAL(B[q + (size_t)q * ldb]);
      }
    }
    ++sweeps;
    double off2 = 0;
    for (int j = 0; j < n; ++j)
      for (int i = 0; i < n; ++i)
        if (i != j) off2 += ABS2(B[i + (size_t)j * ldb]);
    /* converged at off(B) <= u ||B||_F, or once off(B) has stalled at the
     * rounding level n u ||B||_F of the rotations themselves */
    double off = sqrt(off2);
    converged = (off <= tol) || (off <= n * tol && off >= 0.5 * prev_off);
    prev_off = off;
  }
  for (int j = 0; j < n; ++j) lambda[j] = CREAL(B[j + (size_t)j * ldb]);
  free(cs); free(ph); free(pp);
  return converged ? sweeps : -1;
}

#undef FN
#undef CAT
#undef CAT2
