"""Oracle (test infrastructure only; never on the product path).

Zolotarev's best rational approximation of the sign function, as used by
Zolo-pd (Section 5: type (2r+1, 2r) functions, composed over two iterations,
with the interval [-1, -eps] u [eps, 1], eps = 1e-15, of Section 5.1).
The paper cites the formulas (Nakatsukasa and Freund 2016) without printing
them; the published definitions restated here are

    l' = sqrt(1 - l^2),   K' = K(l')            (complete elliptic integral,
                                                 modulus l')
    c_i = l^2 sn^2(i K'/(2r+1); l') / cn^2(i K'/(2r+1); l'),   i = 1..2r
    Z(x) = M x prod_{j=1..r} (x^2 + c_{2j}) / (x^2 + c_{2j-1})
         = M x (1 + sum_j a_j / (x^2 + c_{2j-1}))      (partial fractions)
    a_j  = residue of prod_k (y + c_{2k}) / (y + c_{2k-1}) at y = -c_{2j-1}.

M normalises Z(1) = 1 (so that [l, 1] maps into [Z(l), 1] and the next
iteration works on l_next = Z(l)).  The matrix iteration is
    X_{k+1} = M (X_k + sum_j a_j X_k (X_k^* X_k + c_{2j-1} I)^{-1}),
so X_k = U r_k(Sigma) V^* with r_k the composition of the scalar maps
(Section 5: iterates share the singular vectors of A).

Everything is evaluated with mpmath at 50 significant digits: the Jacobi
elliptic functions sn, cn and K come from mpmath (a library primitive).
"""
import mpmath as mp
import numpy as np

DPS = 50
EPS = 1e-15
U_ROUND = 2.0 ** -53


def coeffs(ell, r):
    """Zolotarev coefficients for the interval [ell, 1] and degree r.

    Returns dict(c=[c_1..c_2r], a=[a_1..a_r], mhat, ell_next) as mpf."""
    with mp.workdps(DPS):
        ell = mp.mpf(ell)
        m = 1 - ell ** 2                      # parameter m = (modulus l')^2
        Kp = mp.ellipk(m)
        c = []
        for i in range(1, 2 * r + 1):
            uu = i * Kp / (2 * r + 1)
            sn = mp.ellipfun("sn", uu, m=m)
            cn = mp.ellipfun("cn", uu, m=m)
            c.append(ell ** 2 * sn ** 2 / cn ** 2)
        a = []
        for j in range(r):
            y = -c[2 * j]                     # pole at y = -c_{2j-1} (1-based)
            num = mp.mpf(1)
            for k in range(r):
                num *= (y + c[2 * k + 1])
            den = mp.mpf(1)
            for k in range(r):
                if k != j:
                    den *= (y + c[2 * k])
            a.append(num / den)
        unnorm_1 = _prod_form(mp.mpf(1), c, r)
        mhat = 1 / unnorm_1
        ell_next = mhat * _prod_form(ell, c, r)
        return dict(c=c, a=a, mhat=mhat, ell_next=ell_next, ell=ell, r=r)


def _prod_form(x, c, r):
    p = x
    for j in range(r):
        p *= (x * x + c[2 * j + 1]) / (x * x + c[2 * j])
    return p


def zhat(x, co):
    """Z(x) in product form (mpf)."""
    with mp.workdps(DPS):
        return co["mhat"] * _prod_form(mp.mpf(x), co["c"], co["r"])


def zhat_pf(x, co):
    """Z(x) in partial-fraction form (mpf)."""
    with mp.workdps(DPS):
        x = mp.mpf(x)
        s = mp.mpf(1)
        for j in range(co["r"]):
            s += co["a"][j] / (x * x + co["c"][2 * j])
        return co["mhat"] * x * s


def plan(ell0=EPS, rmax=8, tol=4 * U_ROUND, max_iter=6):
    """Iteration plan: at each step the smallest r <= rmax whose output
    interval [l_next, 1] satisfies 1 - l_next <= tol; if none does, r = rmax.
    Returns the list of coefficient dicts, one per iteration."""
    out = []
    ell = mp.mpf(ell0)
    for _ in range(max_iter):
        if 1 - ell <= tol:
            break
        chosen = None
        for r in range(1, rmax + 1):
            co = coeffs(ell, r)
            if 1 - co["ell_next"] <= tol:
                chosen = co
                break
        if chosen is None:
            chosen = coeffs(ell, rmax)
        out.append(chosen)
        ell = chosen["ell_next"]
    return out


def compose(x, steps):
    """r_k(x): the scalar map of the whole iteration (composition)."""
    with mp.workdps(DPS):
        y = mp.mpf(x)
        for co in steps:
            y = zhat(y, co)
        return y


def expected_iterates(A, steps, svd):
    """X_k = U r_k(Sigma) V^* for k = 1..len(steps), from an SVD of A given
    as svd = (U, sigma, V) (A = U diag(sigma) V^*)."""
    U, sigma, V = svd
    outs = []
    vals = [mp.mpf(float(s)) for s in sigma]
    with mp.workdps(DPS):
        for co in steps:
            vals = [zhat(v, co) for v in vals]
            f = np.array([float(v) for v in vals])
            outs.append((U * f[None, :]) @ V.conj().T)
    return outs


def as_float(co):
    """Coefficients as float64 numpy arrays (c, a, mhat, ell_next)."""
    return (np.array([float(v) for v in co["c"]]), np.array([float(v) for v in co["a"]]),
            float(co["mhat"]), float(co["ell_next"]))
