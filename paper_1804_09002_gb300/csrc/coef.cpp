// Host computation of Zolotarev's rational approximation of sign(x) on
// [-1, -l] u [l, 1] (Section 5, Zolo-pd; formulas of Zolotarev 1877 as used by
// Nakatsukasa and Freund 2016, which the paper cites):
//   c_i = l^2 sn^2(i K'/(2r+1); l') / cn^2(i K'/(2r+1); l'),  i = 1..2r,
//   Z(x) = M x prod_j (x^2 + c_2j) / (x^2 + c_2j-1) = M x (1 + sum_j a_j / (x^2 + c_2j-1)),
// with l' = sqrt(1 - l^2) and K' = K(l').
//
// For small l the modulus l' is within l^2/2 of 1, where evaluating sn and cn
// directly loses most digits of cn.  Instead sn/cn = sc(u; l') is evaluated
// through Jacobi's imaginary transformation sc(u; k) = -i sn(iu; k') and the
// theta-function form of sn with the nome of the small modulus l,
//   q = exp(-pi K(l') / K(l)),   y = pi u / (2 K(l)),
//   sc(u; l') = theta3(0) * S(y) / (T2 * D(y)),
//   S(y) = sum_n (-1)^n q^(n(n+1)) sinh((2n+1) y),  D(y) = 1 + 2 sum_n>=1 (-1)^n q^(n^2) cosh(2ny),
//   T2 = sum_n q^(n(n+1)),  theta3(0) = 1 + 2 sum_n>=1 q^(n^2),
// whose series converge after a few terms for every l in (0, 1).  K is taken
// from the arithmetic-geometric mean, K(k) = pi / (2 AGM(1, sqrt(1 - k^2)))
// (Abramowitz and Stegun 17.6), so K(l')/K(l) = AGM(1, l') / AGM(1, l).
#include <cmath>

#include "../../include/zolo_csd.h"

namespace {

double agm(double a, double b) {
  for (int it = 0; it < 200; ++it) {
    double an = 0.5 * (a + b), bn = std::sqrt(a * b);
    a = an;
    b = bn;
    if (std::fabs(a - b) <= 1e-17 * a) break;
  }
  return 0.5 * (a + b);
}

// sc(u; l') at u = i K(l') / (2r+1) for i = 1..2r, via the series above.
void zolo_c(double ell, int r, double* c) {
  const double lp = std::sqrt((1.0 - ell) * (1.0 + ell));
  const double lnq = -M_PI * agm(1.0, lp) / agm(1.0, ell);  // ln q
  const double q = std::exp(lnq);
  double theta3 = 1.0, t2 = 0.0;
  for (int n = 0; n < 64; ++n) {
    double e = std::exp(lnq * (double)n * (double)(n + 1));
    t2 += e;
    if (n >= 1) theta3 += 2.0 * std::exp(lnq * (double)n * (double)n);
    if (e < 1e-40) break;
  }
  (void)q;
  for (int i = 1; i <= 2 * r; ++i) {
    const double y = -(double)i * lnq / (2.0 * (2 * r + 1));
    double S = 0.0, D = 1.0;
    for (int n = 0; n < 64; ++n) {
      // q^(n(n+1)) sinh((2n+1) y) and q^(n^2) cosh(2 n y), in log space
      double ls = lnq * (double)n * (double)(n + 1);
      double ts = std::exp(ls) * std::sinh((2.0 * n + 1.0) * y);
      S += (n & 1) ? -ts : ts;
      double td = 0.0;
      if (n >= 1) {
        td = 2.0 * std::exp(lnq * (double)n * (double)n) * std::cosh(2.0 * n * y);
        D += (n & 1) ? -td : td;
      }
      if (n >= 2 && std::fabs(ts) <= 1e-19 * std::fabs(S) && td <= 1e-19 * std::fabs(D)) break;
    }
    const double sc = theta3 * S / (t2 * D);
    c[i - 1] = ell * ell * sc * sc;
  }
}

double zprod(double x, const double* c, int r) {
  double p = x;
  for (int j = 0; j < r; ++j) p *= (x * x + c[2 * j + 1]) / (x * x + c[2 * j]);
  return p;
}

}  // namespace

extern "C" int zolo_coeffs(double ell, int r, double* c, double* a, double* mhat, double* ell_next) {
  if (!(ell > 0.0 && ell < 1.0)) return -1;
  if (r < 1 || r > 16) return -2;
  if (!c) return -3;
  zolo_c(ell, r, c);
  if (a) {
    // residue of prod_k (y + c_2k)/(y + c_2k-1) at y = -c_2j-1
    for (int j = 0; j < r; ++j) {
      const double y = -c[2 * j];
      double num = 1.0, den = 1.0;
      for (int k = 0; k < r; ++k) {
        num *= (y + c[2 * k + 1]);
        if (k != j) den *= (y + c[2 * k]);
      }
      a[j] = num / den;
    }
  }
  const double m = 1.0 / zprod(1.0, c, r);
  if (mhat) *mhat = m;
  if (ell_next) *ell_next = std::fmin(1.0, m * zprod(ell, c, r));
  return 0;
}

extern "C" int zolo_plan(double ell0, int rmax, int max_iter, int* r_out, double* ell_out) {
  if (!(ell0 > 0.0 && ell0 <= 1.0)) return -1;
  if (rmax < 1 || rmax > 16) return -2;
  if (max_iter < 1) return -3;
  const double tol = 4.0 * 0x1p-53;
  double ell = ell0, c[32];
  int k = 0;
  while (k < max_iter && 1.0 - ell > tol) {
    int rc = rmax;
    double next = 0.0;
    for (int r = 1; r <= rmax; ++r) {
      zolo_coeffs(ell, r, c, nullptr, nullptr, &next);
      if (1.0 - next <= tol) { rc = r; break; }
    }
    zolo_coeffs(ell, rc, c, nullptr, nullptr, &next);
    if (r_out) r_out[k] = rc;
    if (ell_out) ell_out[k] = ell;
    ell = next;
    ++k;
  }
  return k;
}
