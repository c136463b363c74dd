"""Pins for the oracle's Zolotarev functions (no GPU).

Section 5 (Zolo-pd) uses Zolotarev's best rational approximations of the
sign function but defers their formulas to the literature; the oracle
restates them (oracle/zolo.py).  These tests pin that restatement to facts
that do not depend on it: the r = 1 case is QDWH's dynamically weighted
Halley map, whose weights have a closed form; best approximations
equioscillate; two type-(17, 16) steps from eps = 1e-15 reach 1 - O(u)
(Section 5 and 5.1); and the matrix iteration reproduces U r(Sigma) V^*
(Section 5: iterates share the singular vectors of A).
"""
import mpmath as mp
import numpy as np
import pytest

zolo = pytest.importorskip("oracle.zolo")
mp.mp.dps = 50

u = 2.0 ** -53


def qdwh_weights(ell):
    """QDWH (Nakatsukasa, Bai and Gygi 2010): a = h(l), b = (a-1)^2/4,
    c = a + b - 1, f(x) = x (a + b x^2) / (1 + c x^2)."""
    mp.mp.dps = 50
    ell = mp.mpf(ell)
    d = mp.cbrt(4 * (1 - ell ** 2) / ell ** 4)
    a = mp.sqrt(1 + d) + mp.sqrt(8 - 4 * d + 8 * (2 - ell ** 2) / (ell ** 2 * mp.sqrt(1 + d))) / 2
    b = (a - 1) ** 2 / 4
    c = a + b - 1
    return a, b, c


@pytest.mark.parametrize("ell", [1e-15, 1e-6, 0.01, 0.3, 0.9])
def test_r1_is_qdwh(ell):
    co = zolo.coeffs(ell, 1)
    a, b, c = qdwh_weights(ell)
    with mp.workdps(40):
        for x in [ell, 2 * ell, 0.1, 0.5, 0.77, 1.0]:
            f = mp.mpf(x) * (a + b * mp.mpf(x) ** 2) / (1 + c * mp.mpf(x) ** 2)
            assert abs(zolo.zhat(x, co) - f) <= mp.mpf("1e-20") * abs(f)


def _extrema(co, ell):
    """Values of Z at the end points and at its interior critical points on
    [ell, 1] (located on a log grid, refined by mpmath's root finder)."""
    with mp.workdps(40):
        f = lambda x: zolo.zhat(x, co)
        c = co["c"]

        def df(x):  # Z'(x) = Z(x) (1/x + sum_j 2x/(x^2+c_2j) - 2x/(x^2+c_2j-1))
            x = mp.mpf(x)
            g = 1 / x
            for j in range(co["r"]):
                g += 2 * x / (x * x + c[2 * j + 1]) - 2 * x / (x * x + c[2 * j])
            return f(x) * g
        xs = [mp.mpf(ell) * (1 / mp.mpf(ell)) ** (mp.mpf(k) / 2000) for k in range(2001)]
        ds = [df(x) for x in xs]
        pts = [mp.mpf(ell)]
        for i in range(len(xs) - 1):
            if ds[i] * ds[i + 1] < 0:
                lo, hi, dlo = xs[i], xs[i + 1], ds[i]
                for _ in range(120):          # plain bisection on Z'
                    mid = (lo + hi) / 2
                    dm = df(mid)
                    if dm * dlo > 0:
                        lo, dlo = mid, dm
                    else:
                        hi = mid
                pts.append((lo + hi) / 2)
        pts.append(mp.mpf(1))
        return [f(x) for x in pts]


@pytest.mark.parametrize("ell,r", [(0.05, 2), (1e-3, 3), (0.2, 4)])
def test_equioscillation(ell, r):
    """A best type (2r+1, 2r) approximation of sign on [ell, 1] equioscillates
    at 2r + 2 points: r + 1 equal minima and r + 1 equal maxima (= 1 with
    the normalisation Z(1) = 1), alternating."""
    co = zolo.coeffs(ell, r)
    vals = _extrema(co, ell)
    assert len(vals) == 2 * r + 2
    lo = [v for i, v in enumerate(vals) if i % 2 == 0]
    hi = [v for i, v in enumerate(vals) if i % 2 == 1]
    assert max(hi) - min(hi) <= mp.mpf("1e-25")
    assert max(lo) - min(lo) <= mp.mpf("1e-25")
    assert abs(hi[-1] - 1) <= mp.mpf("1e-30")
    assert all(h > l for h, l in zip(hi, lo))


def test_two_steps_reach_unit_roundoff():
    """Section 5.1: with eps = 1e-15 and p = 8, two iterations map [eps, 1]
    to 1 - O(u); and p = 7 would not suffice for the second step."""
    steps = zolo.plan(1e-15)
    assert [co["r"] for co in steps] == [8, 8]
    assert 1 - steps[-1]["ell_next"] <= u
    co7 = zolo.coeffs(steps[0]["ell_next"], 7)
    assert 1 - co7["ell_next"] > 4 * u
    # r_2(x) in [0, 1] on [0, 1] (Section 5.1), increasing below eps and
    # within u of 1 on [eps, 1]
    lo = [zolo.compose(x, steps) for x in [0.0, 1e-17, 1e-16, 5e-16, 1e-15]]
    assert all(lo[i] <= lo[i + 1] for i in range(len(lo) - 1))
    assert lo[0] == 0
    hi = [zolo.compose(x, steps) for x in [1e-15, 3e-15, 1e-12, 1e-9, 1e-4, 0.1, 0.5, 0.9, 1.0]]
    assert all(1 - u <= y <= 1 + mp.mpf("1e-30") for y in hi)


def test_coefficient_structure():
    for ell, r in [(1e-15, 8), (0.4565, 8), (0.1, 3)]:
        co = zolo.coeffs(ell, r)
        c = co["c"]
        assert all(x > 0 for x in c)
        assert all(c[i] < c[i + 1] for i in range(len(c) - 1))
        assert all(a > 0 for a in co["a"])
        for x in [ell, 0.3, 1.0]:
            assert abs(zolo.zhat(x, co) - zolo.zhat_pf(x, co)) <= mp.mpf("1e-35")


def test_matrix_iteration_matches_scalar_map():
    """X_{k+1} = M (X_k + sum_j a_j X_k (X_k^T X_k + c_{2j-1} I)^{-1}) applied
    to a matrix equals U r_k(Sigma) V^T (Section 5)."""
    rng = np.random.default_rng(3)
    n = 12
    U = np.linalg.qr(rng.standard_normal((n, n)))[0]
    V = np.linalg.qr(rng.standard_normal((n, n)))[0]
    sig = np.geomspace(0.05, 1.0, n)
    A = (U * sig) @ V.T
    steps = zolo.plan(0.05)
    X = A.copy()
    for co in steps:
        c, a, mhat, _ = zolo.as_float(co)
        acc = X.copy()
        for j in range(co["r"]):
            acc += a[j] * np.linalg.solve((X.T @ X + c[2 * j] * np.eye(n)).T, X.T).T
        X = mhat * acc
    want = zolo.expected_iterates(A, steps, (U, sig, V))[-1]
    assert np.max(np.abs(X - want)) <= 1e-13
    assert np.linalg.norm(X.T @ X - np.eye(n)) <= 1e-13
