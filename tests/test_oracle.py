"""Pins for the CPU FP64 oracle (no GPU).

The oracle is checked against what the paper and the mathematics fix, not
against itself: closed forms (n = 1), the Section 3 MATLAB example, known
angles of synthetic inputs, singular values from LAPACK (numpy), LAPACK's
CS decomposition (scipy.linalg.cossin), invariants of the CSD (Section 1,
Theorem 2.1), the swap symmetry of remark (i) and the accuracy magnitudes of
Tables 1-2.  A few tests plant a mistake in the oracle (on the CPU) and
check that a pin catches it.
"""
import numpy as np
import pytest

from oracle import csd as O
from oracle import jacobi as J
from oracle import metrics as M
from paper_1804_09002_gb300 import inputs as I

u = M.U_ROUND


def _golden(name):
    vals = {}
    import os
    with open(os.path.join(os.path.dirname(__file__), "golden", name)) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                k, v = line.split()
                vals[k] = float(v)
    return vals


# ---------------------------------------------------------------- sub-solvers
@pytest.mark.parametrize("m,n,cplx", [(40, 40, False), (57, 31, False), (33, 33, True), (20, 7, True)])
def test_jacobi_svd_matches_lapack(m, n, cplx):
    rng = np.random.default_rng(m * 100 + n)
    A = rng.standard_normal((m, n)) + (1j * rng.standard_normal((m, n)) if cplx else 0)
    G, V, s, _ = J.svd_onesided(A)
    ref = np.linalg.svd(A, compute_uv=False)
    assert np.max(np.abs(np.sort(s)[::-1] - ref)) <= 50 * n * u * ref[0]
    assert np.max(np.abs(A @ V - G)) <= 50 * n * u * ref[0]
    assert np.linalg.norm(V.conj().T @ V - np.eye(n), 2) <= 20 * n * u


@pytest.mark.parametrize("n,cplx", [(1, False), (2, True), (37, False), (64, True)])
def test_jacobi_eig_matches_lapack(n, cplx):
    rng = np.random.default_rng(n)
    X = rng.standard_normal((n, n)) + (1j * rng.standard_normal((n, n)) if cplx else 0)
    B = X + X.conj().T
    lam, V = O.heig(B)
    ref = np.linalg.eigvalsh(B)
    nb = np.linalg.norm(B, 2)
    assert np.all(np.diff(lam) >= 0)
    assert np.max(np.abs(lam - ref)) <= 20 * n * u * nb
    assert np.linalg.norm(B @ V - V * lam[None, :], 2) <= 20 * n * u * nb
    assert np.linalg.norm(V.conj().T @ V - np.eye(n), 2) <= 20 * n * u


def test_polar_is_polar():
    rng = np.random.default_rng(7)
    A = rng.standard_normal((50, 50))
    W, H = O.polar(A)
    assert np.linalg.norm(W @ H - A) <= 100 * u * np.linalg.norm(A)
    assert np.linalg.norm(W.T @ W - np.eye(50), 2) <= 1000 * u
    assert np.min(np.linalg.eigvalsh(H)) >= -1e-13
    # H = (A^* A)^{1/2}: H^2 = A^* A (Section 2)
    assert np.linalg.norm(H @ H - A.T @ A) <= 1e3 * u * np.linalg.norm(A) ** 2


def test_polar_zero_columns_completed():
    """Rank-deficient input: W must still have orthonormal columns."""
    rng = np.random.default_rng(8)
    X = rng.standard_normal((20, 12))
    A = X @ rng.standard_normal((12, 20))  # rank 12
    A[:, 3] = 0.0
    W, H = O.polar(A)
    assert np.linalg.norm(W.T @ W - np.eye(20), 2) <= 1e-12
    assert np.linalg.norm(W @ H - A) <= 1e-12 * np.linalg.norm(A)


# ---------------------------------------------------------------- closed forms
@pytest.mark.parametrize("a1,a2", [(0.6, 0.8), (-0.28, 0.96), (1.0, 0.0), (0.0, -1.0),
                                   (0.6j, 0.8), ((0.6 + 0.0j) * np.exp(0.3j), -0.8j)])
def test_n1_closed_form(a1, a2):
    """n = 1: A = [a1; a2], |a1|^2 + |a2|^2 = 1 has theta = atan2(|a2|, |a1|),
    U_i = a_i/|a_i| (any unit scalar if a_i = 0), V1 a unit scalar (Section 1)."""
    A1 = np.array([[a1]])
    A2 = np.array([[a2]])
    R = O.csd(A1, A2)
    assert R["rank"] == 1 and R["mu"] == 0.0
    assert abs(R["theta"][0] - np.arctan2(abs(a2), abs(a1))) <= 4 * u
    v = R["V1"][0, 0]
    assert abs(abs(v) - 1) <= 4 * u
    for a, Ui, f in ((a1, R["U1"], np.cos), (a2, R["U2"], np.sin)):
        assert abs(abs(Ui[0, 0]) - 1) <= 4 * u
        # A_i = U_i f(theta) V1^*
        assert abs(Ui[0, 0] * f(R["theta"][0]) * np.conj(v) - a) <= 8 * u


def test_matlab_example_section3():
    """Section 3: V from eig(H2 - H1) diagonalises H2 to O(u); V from eig(H1)
    leaves off-diagonal entries of order 1e-9.  The paper prints
    1.7806e-17 and 2.8187e-09; a different eigensolver gives other digits but
    the same orders of magnitude."""
    g = _golden("matlab_example.txt")
    H1, H2, V1, th = I.matlab_example()

    def offdiag(Vh):
        S = Vh.T @ H2 @ Vh
        return np.max(np.abs(S - np.diag(np.diag(S))))

    good = offdiag(O.heig(H2 - H1)[1])
    bad = offdiag(O.heig(H1)[1])
    assert good <= 100 * g["eig_H2_minus_H1"]
    assert bad >= 0.01 * g["eig_H1"]
    assert bad / good > 1e5


# ---------------------------------------------------------------- known angles
def _check_full(A1, A2, th, R, tol_theta):
    n = A1.shape[1]
    assert R["rank"] == n and R["mu"] == 0.0
    assert np.max(np.abs(R["theta"] - th)) <= tol_theta
    be = M.backward_error_fro(A1, A2, R["U1"], R["U2"], R["theta"], R["V1"])
    assert be <= 50 * n * u
    for X in (R["U1"], R["U2"], R["V1"]):
        assert M.orthogonality(X) <= 10 * n * u + 100 * u


@pytest.mark.parametrize("n,cplx", [(2, False), (17, False), (64, False), (33, True)])
def test_known_theta_haar(n, cplx):
    A1, A2, th = I.haar_csd(n, seed=1 + n, cplx=cplx)
    R = O.csd(A1, A2)
    _check_full(A1, A2, th, R, 1e-12 * n)


def test_known_theta_clustered():
    n = 96
    A1, A2, th = I.clustered_csd(n, seed=2)
    R = O.csd(A1, A2)
    # the 1e-14 perturbation moves each angle by O(1e-14)
    _check_full(A1, A2, th, R, 1e-12 * n)
    # clustered angles are still resolved to O(u) absolute
    assert np.max(np.abs(R["theta"][: n // 4] - th[: n // 4])) <= 1e-13


def test_singular_values_are_cos_sin():
    """sigma(A1) = cos(theta), sigma(A2) = sin(theta) (Section 1), with the
    singular values from LAPACK."""
    A1, A2, _ = I.haar_csd(48, seed=11)
    R = O.csd(A1, A2)
    s1 = np.sort(np.linalg.svd(A1, compute_uv=False))
    s2 = np.sort(np.linalg.svd(A2, compute_uv=False))
    assert np.max(np.abs(np.sort(np.cos(R["theta"])) - s1)) <= 1e-13
    assert np.max(np.abs(np.sort(np.sin(R["theta"])) - s2)) <= 1e-13
    assert np.max(np.abs(R["C"] ** 2 + R["S"] ** 2 - 1)) <= 4 * u


def test_swap_symmetry_remark_i():
    """Exchanging A1 and A2 negates B and maps theta to pi/2 - theta
    (remark (i) prints pi/4; swapping C and S gives pi/2)."""
    A1, A2, _ = I.haar_csd(40, seed=12)
    R = O.csd(A1, A2)
    Rs = O.csd(A2, A1)
    assert np.max(np.abs(Rs["theta"] - (np.pi / 2 - R["theta"][::-1]))) <= 1e-13
    assert np.max(np.abs(Rs["B"] + R["B"])) <= 1e-15


def test_lapack_cossin_crosscheck():
    """Angles agree with LAPACK's CS decomposition (scipy.linalg.cossin) of
    the orthogonal completion [A, A_perp]."""
    linalg = pytest.importorskip("scipy.linalg")
    n = 24
    A1, A2, _ = I.haar_csd(n, seed=13)
    A = np.vstack([A1, A2])
    Q, _ = np.linalg.qr(A, mode="complete")
    X = np.hstack([A, Q[:, n:]])
    u_, cs, vdh = linalg.cossin(X, p=n, q=n)
    th_lapack = np.sort(np.arctan2(np.diag(cs[n:, :n]), np.diag(cs[:n, :n])))
    R = O.csd(A1, A2)
    assert np.max(np.abs(R["theta"] - th_lapack)) <= 1e-13


# ---------------------------------------------------------------- rank deficient
@pytest.mark.parametrize("n,k,cplx", [(32, 24, True), (40, 30, False)])
def test_rank_deficient(n, k, cplx):
    """Theorem 2.1 / Algorithm 3: rank k partial isometry; ||A||_F^2 = k,
    mu = 2, exactly n - k eigenvalues of B at 2, economical U1, U2, V1."""
    A1, A2, th = I.rankdef_csd(n, k, seed=5, cplx=cplx, n_repeat=4)
    R = O.csd(A1, A2)
    assert R["rank"] == k and R["mu"] == 2.0
    lam = R["Lambda"]
    assert np.sum(lam > 1.5) == n - k
    assert np.max(np.abs(lam[lam > 1.5] - 2.0)) <= 1e-13
    assert np.max(np.abs(R["theta"] - th)) <= 1e-12 * n
    be = M.backward_error_fro(A1, A2, R["U1"], R["U2"], R["theta"], R["V1"])
    assert be <= 50 * n * u
    for X in (R["U1"], R["U2"], R["V1"]):
        assert X.shape == (n, k)
        assert M.orthogonality(X) <= 10 * n * u + 100 * u


# ---------------------------------------------------------------- paper families
@pytest.mark.parametrize("kind", [1, 2, 3, 4])
@pytest.mark.parametrize("noisy", [False, True])
def test_paper_families_tables(kind, noisy):
    """Section 6 families at n = 30, 42: the scaled residual ||A_hat - A||_2
    / d(A) stays at the magnitudes of Tables 1-2 (all below 85 there)."""
    for n in (30, 42):
        A1, A2 = I.paper_test(kind, n, seed=100 + kind, noisy=noisy)
        R = O.csd(A1, A2)
        d = M.dist_partial_isometry(A1, A2)
        r2 = M.residual_2(A1, A2, R["U1"], R["U2"], R["theta"], R["V1"])
        assert r2 / max(d, u) <= 100.0
        expect_rank = n if kind in (1, 2) else int(np.floor(3 * n / 4 + 0.5))
        assert R["rank"] == expect_rank
        for X in (R["U1"], R["U2"], R["V1"]):
            assert M.orthogonality(X) <= 10 * n * u + 100 * u


# ---------------------------------------------------------------- planted mistakes
def test_planted_wrong_B_is_caught(monkeypatch):
    """Eigendecomposing H1 instead of B = H2 - H1 (the unstable choice of
    Section 3) on angles clustered near 0: the backward-error pin must fail."""
    rng = np.random.default_rng(21)
    n = 12
    th = np.sort(rng.uniform(0, 5e-8, n))
    A1, A2 = I.from_angles(th, rng)
    seen = []
    real_polar, real_heig = O.polar, O.heig

    def spy_polar(A):
        W, H = real_polar(A)
        seen.append(H)
        return W, H

    monkeypatch.setattr(O, "polar", spy_polar)
    monkeypatch.setattr(O, "heig", lambda B: real_heig(seen[0]))
    R = O.csd(A1, A2)
    assert M.backward_error_fro(A1, A2, R["U1"], R["U2"], R["theta"], R["V1"]) > 50 * n * u


def test_planted_transpose_is_caught(monkeypatch):
    """Polar factor returned transposed: the backward-error pin must fail."""
    A1, A2, _ = I.haar_csd(16, seed=22)
    real_polar = O.polar
    monkeypatch.setattr(O, "polar", lambda A: (lambda W, H: (W.T, H))(*real_polar(A)))
    R = O.csd(A1, A2)
    assert M.backward_error_fro(A1, A2, R["U1"], R["U2"], R["theta"], R["V1"]) > 1e-3


def test_planted_missing_shift_is_caught(monkeypatch):
    """mu forced to 0 on a rank-deficient input: the count of kept angles
    (the rank pin) must fail."""
    A1, A2, th = I.rankdef_csd(24, 18, seed=23, cplx=False, n_repeat=2)
    R = O.csd(A1, A2, mu=0.0)
    assert R["V1"].shape[1] != 18


# ------------------------------------------------ remarks (iv) and (viii)
@pytest.mark.parametrize("n,cplx", [(40, False), (24, True)])
def test_theta_from_lambda_remark_iv(n, cplx):
    """theta from sin(theta) - cos(theta) = Lambda: the known angles within
    O(u) (d theta / d Lambda = 1 / (cos + sin) <= 1 on [0, pi/2]), the
    defining equation on the kept eigenvalues, and a backward-stable CSD."""
    A1, A2, th = I.haar_csd(n, seed=70 + n, cplx=cplx)
    R = O.csd(A1, A2, theta_from="lambda")
    assert np.max(np.abs(R["theta"] - th)) <= 1e-12 * n
    lam = np.sort(R["Lambda_r"])
    assert np.max(np.abs(np.sin(R["theta"]) - np.cos(R["theta"]) - lam)) <= 1e-14 * n
    be = M.backward_error_fro(A1, A2, R["U1"], R["U2"], R["theta"], R["V1"])
    assert be <= 50 * n * u


def test_theta_from_lambda_rank_deficient():
    n, k = 32, 24
    A1, A2, th = I.rankdef_csd(n, k, seed=71, cplx=False, n_repeat=4)
    R = O.csd(A1, A2, theta_from="lambda")
    assert R["rank"] == k
    assert np.max(np.abs(R["theta"] - th)) <= 1e-12 * n


def _complete_blocks(n, cplx, seed):
    rng = np.random.default_rng(seed)
    Q = I.haar(2 * n, rng, cplx)
    return Q[:n, :n], Q[n:, :n], Q[:n, n:], Q[n:, n:]


@pytest.mark.parametrize("n,cplx", [(24, False), (16, True)])
def test_complete_2x2_csd_remark_viii(n, cplx):
    """For a unitary [A1 A3; A2 A4], V2 from X = -A3^* U1 S + A4^* U2 C
    completes the 2 x 2 CSD: A3 = -U1 S V2^*, A4 = U2 C V2^*, V2 unitary
    (the defining identities of remark (viii), checked to O(u))."""
    A1, A2, A3, A4 = _complete_blocks(n, cplx, 80 + n)
    R = O.csd(A1, A2)
    V2 = O.complete_v2(A3, A4, R["U1"], R["U2"], R["theta"])
    C, S = np.cos(R["theta"]), np.sin(R["theta"])
    r3 = np.linalg.norm(A3 + (R["U1"] * S[None, :]) @ V2.conj().T)
    r4 = np.linalg.norm(A4 - (R["U2"] * C[None, :]) @ V2.conj().T)
    assert max(r3, r4) <= 50 * n * u
    assert M.orthogonality(V2) <= 10 * n * u
    # a sign slip in X (+A3 instead of -A3) breaks the identity
    X = (A3.conj().T @ (R["U1"] * S[None, :])) + A4.conj().T @ (R["U2"] * C[None, :])
    Qw = np.linalg.qr(X)[0]
    assert np.linalg.norm(A3 + (R["U1"] * S[None, :]) @ Qw.conj().T) > 1e-3


# ------------------------------------------------ rectangular blocks (Section 2)
@pytest.mark.parametrize("m1,m2,n,cplx,k", [(31, 26, 20, False, None), (24, 30, 18, True, None),
                                           (28, 22, 20, False, 14)])
def test_rectangular_blocks(m1, m2, n, cplx, k):
    """A_i of size m_i x n (m_i >= n): the oracle's polar factors are m_i x n,
    B stays n x n; the known angles, sigma(A1) = cos(theta), the backward
    error and orthogonality of U_i (m_i x r) hold as in the square case."""
    A1, A2, th = I.rect_csd(m1, m2, n, seed=m1 + n, cplx=cplx, k=k)
    R = O.csd(A1, A2)
    r = n if k is None else k
    assert R["rank"] == r and R["U1"].shape == (m1, r) and R["U2"].shape == (m2, r)
    assert np.max(np.abs(R["theta"] - th)) <= 1e-12 * n
    s1 = np.sort(np.linalg.svd(A1, compute_uv=False))[::-1][:r]
    assert np.max(np.abs(np.sort(np.cos(R["theta"]))[::-1] - s1)) <= 1e-13
    be = M.backward_error_fro(A1, A2, R["U1"], R["U2"], R["theta"], R["V1"])
    assert be <= 50 * n * u
    for X in (R["U1"], R["U2"], R["V1"]):
        assert M.orthogonality(X) <= 10 * n * u + 100 * u
