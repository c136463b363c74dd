"""Parity of the CUDA path (through the C ABI) with the CPU FP64 oracle.

Tolerances: angles within 1e-12 * n of the oracle, backward error
||A - A_hat||_F / ||A||_F <= 50 n u, and orthogonality ||X^* X - I||_2 <= 50 n u
for U1, U2, V1 (FP64, u = 2^-53).  Factors inside clusters of equal angles
are not unique, so U1, U2, V1 are compared through these invariants, never
column by column.
"""
import numpy as np
import pytest

from oracle import csd as O
from oracle import metrics as M
from paper_1804_09002_gb300 import inputs as I
from tests.gpu_util import U, to_dev, to_host

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def B():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1804_09002_gb300 import binding
    return binding


def _check_csd(A1, A2, R, n, theta_ref=None, rank=None):
    th = to_host(R["theta"])
    rk = R["rank"]
    if rank is not None:
        assert rk == rank
    U1, U2, V1 = (to_host(R[k])[:, :rk] for k in ("U1", "U2", "V1"))
    th = th[:rk]
    assert np.all(np.diff(th) >= 0)
    assert np.all(th >= 0) and np.all(th <= np.pi / 2 + 1e-15)
    if theta_ref is not None:
        assert np.max(np.abs(th - theta_ref)) <= 1e-12 * n
    be = M.backward_error_fro(A1, A2, U1, U2, th, V1)
    assert be <= 50 * n * U, be
    for X in (U1, U2, V1):
        assert M.orthogonality(X) <= 50 * n * U
    return th


# ------------------------------------------------------------------ Zolo-pd
@pytest.mark.parametrize("n", [1, 2, 31, 64, 100])
def test_polar_matches_oracle(B, n):
    rng = np.random.default_rng(n)
    A = rng.standard_normal((n, n))
    A /= np.linalg.norm(A, 2)
    W, H, info = B.polar(to_dev(A))
    W, H = to_host(W), to_host(H)
    Wo, Ho = O.polar(A)
    kappa = np.linalg.cond(A)
    assert info["r_terms"][:2] == [8, 8]
    assert np.linalg.norm(W - Wo) <= 1e-13 * n * max(kappa, 1)
    assert np.linalg.norm(H - Ho) <= 50 * n * U
    assert np.linalg.norm(W.T @ W - np.eye(n), 2) <= 50 * n * U
    assert np.linalg.norm(W @ H - A) <= 50 * n * U


def test_polar_ill_conditioned_and_host_pointers(B):
    """kappa = 1e12 (Section 5.1: [eps, 1] with eps = 1e-15 still maps every
    singular value to 1); numpy inputs exercise the host-pointer path."""
    n = 80
    rng = np.random.default_rng(5)
    Uo = np.linalg.qr(rng.standard_normal((n, n)))[0]
    Vo = np.linalg.qr(rng.standard_normal((n, n)))[0]
    s = np.geomspace(1e-12, 1.0, n)
    A = np.asfortranarray((Uo * s) @ Vo.T)
    W, H, _ = B.polar(A)
    assert isinstance(W, np.ndarray)
    assert np.linalg.norm(W - Uo @ Vo.T) <= 1e-3   # unique polar factor, error ~ u / sigma_min
    assert np.linalg.norm(W.T @ W - np.eye(n), 2) <= 50 * n * U
    assert np.linalg.norm(W @ H - A) <= 50 * n * U


def test_polar_complex(B):
    n = 40
    rng = np.random.default_rng(9)
    A = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
    A /= np.linalg.norm(A, 2)
    W, H, _ = B.polar(to_dev(A))
    W, H = to_host(W), to_host(H)
    Wo, Ho = O.polar(A)
    assert np.linalg.norm(W - Wo) <= 1e-10
    assert np.linalg.norm(H - Ho) <= 50 * n * U
    assert np.linalg.norm(W.conj().T @ W - np.eye(n), 2) <= 50 * n * U


# ------------------------------------------------------------------ Zolo-eig
@pytest.mark.parametrize("n", [1, 5, 64, 65, 150])
def test_heig_matches_oracle(B, n):
    rng = np.random.default_rng(100 + n)
    X = rng.standard_normal((n, n))
    Bm = X + X.T
    lam, V, info = B.heig(to_dev(Bm))
    lam, V = to_host(lam), to_host(V)
    lo, _ = O.heig(Bm)
    nb = np.linalg.norm(Bm, 2)
    assert np.all(np.diff(lam) >= 0)
    assert np.max(np.abs(lam - lo)) <= 50 * n * U * nb
    assert np.linalg.norm(Bm @ V - V * lam) <= 50 * n * U * nb
    assert np.linalg.norm(V.T @ V - np.eye(n), 2) <= 50 * n * U


def test_heig_repeated_eigenvalues(B):
    """Exactly repeated eigenvalues (a scalar block after a split)."""
    n = 160
    rng = np.random.default_rng(3)
    Q = np.linalg.qr(rng.standard_normal((n, n)))[0]
    ev = np.concatenate([np.full(70, 0.25), np.full(50, -0.5), rng.uniform(-1, 1, 40)])
    Bm = (Q * ev) @ Q.T
    lam, V, _ = B.heig(to_dev(Bm))
    lam, V = to_host(lam), to_host(V)
    assert np.max(np.abs(lam - np.sort(ev))) <= 50 * n * U
    assert np.linalg.norm(Bm @ V - V * lam) <= 50 * n * U
    assert np.linalg.norm(V.T @ V - np.eye(n), 2) <= 50 * n * U


# ------------------------------------------------------------------ CSD
def test_csd_config_n64(B):
    """n = 64, Haar U1, U2, V, theta ~ U[0, pi/2] (the small parity case)."""
    n = 64
    A1, A2, th = I.haar_csd(n, seed=1)
    R = B.csd_polar(to_dev(A1), to_dev(A2))
    ref = O.csd(A1, A2)
    got = _check_csd(A1, A2, R, n, theta_ref=ref["theta"], rank=n)
    assert np.max(np.abs(got - th)) <= 1e-12 * n


@pytest.mark.parametrize("n", [1, 2, 3, 33, 97, 130])
def test_csd_ragged_sizes(B, n):
    A1, A2, th = I.haar_csd(n, seed=40 + n)
    R = B.csd_polar(to_dev(A1), to_dev(A2))
    ref = O.csd(A1, A2)
    _check_csd(A1, A2, R, n, theta_ref=ref["theta"], rank=n)


def test_csd_clustered(B):
    """Angles clustered within 1e-8 of 0 and pi/2 (kappa(A_i) ~ 1e8+), 1e-14
    noise and re-orthonormalisation: the ill-conditioned workload family."""
    n = 192
    A1, A2, th = I.clustered_csd(n, seed=2)
    R = B.csd_polar(to_dev(A1), to_dev(A2))
    ref = O.csd(A1, A2)
    _check_csd(A1, A2, R, n, theta_ref=ref["theta"], rank=n)


def test_csd_host_pointers(B):
    n = 48
    A1, A2, th = I.haar_csd(n, seed=7)
    R = B.csd_polar(A1, A2)   # numpy in, numpy out
    assert isinstance(R["U1"], np.ndarray)
    ref = O.csd(A1, A2)
    _check_csd(A1, A2, R, n, theta_ref=ref["theta"], rank=n)


@pytest.mark.parametrize("n,k,cplx", [(64, 48, False), (48, 36, True)])
def test_csd_rank_deficient(B, n, k, cplx):
    """Algorithm 3: rank-k partial isometry, mu = 2, economical output."""
    A1, A2, th = I.rankdef_csd(n, k, seed=3, cplx=cplx, n_repeat=n // 8)
    to = (lambda a: to_dev(a))
    R = B.csd_polar(to(A1), to(A2))
    ref = O.csd(A1, A2)
    assert R["info"]["mu"] == 2.0
    _check_csd(A1, A2, R, n, theta_ref=ref["theta"], rank=k)


def test_csd_complex_full_rank(B):
    n = 40
    A1, A2, th = I.haar_csd(n, seed=11, cplx=True)
    R = B.csd_polar(to_dev(A1), to_dev(A2))
    ref = O.csd(A1, A2)
    _check_csd(A1, A2, R, n, theta_ref=ref["theta"], rank=n)


def test_csd_nonfinite_input_is_rejected(B):
    n = 8
    A1, A2, _ = I.haar_csd(n, seed=12)
    A1 = A1.copy()
    A1[2, 3] = np.nan
    with pytest.raises(B.CSDError) as e:
        B.csd_polar(to_dev(A1), to_dev(A2))
    assert e.value.status == 5
