"""The tensor-core path: real FP64 products run as exact BF16 slice products
on tcgen05 (csd_set_tensor_cores).  The same parity bars as the FP64-pipe
path: against the CPU oracle, known angles, backward error <= 50 n u and
orthogonality <= 50 n u."""
import numpy as np
import pytest

from oracle import csd as O
from oracle import metrics as M
from paper_1804_09002_gb300 import inputs as I
from tests.gpu_util import U, to_dev, to_host
from tests.test_gpu_parity import _check_csd, _dev_metrics

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def C():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1804_09002_gb300 import binding
    ctx = binding.Context(0)
    ctx.set_tensor_cores(True)
    yield ctx
    ctx.close()


@pytest.mark.parametrize("n", [64, 100, 257])
def test_tc_polar_matches_oracle(C, n):
    rng = np.random.default_rng(300 + n)
    A = rng.standard_normal((n, n))
    A /= np.linalg.norm(A, 2)
    W, H, info = C.polar(to_dev(A))
    W, H = to_host(W), to_host(H)
    Wo, Ho = O.polar(A)
    kappa = np.linalg.cond(A)
    assert np.linalg.norm(W - Wo) <= 1e-13 * n * max(kappa, 1)
    assert np.linalg.norm(H - Ho) <= 50 * n * U
    assert np.linalg.norm(W.T @ W - np.eye(n), 2) <= 50 * n * U
    assert np.linalg.norm(W @ H - A) <= 50 * n * U


def test_tc_polar_ill_conditioned(C):
    n = 200
    rng = np.random.default_rng(5)
    Uo = np.linalg.qr(rng.standard_normal((n, n)))[0]
    Vo = np.linalg.qr(rng.standard_normal((n, n)))[0]
    s = np.geomspace(1e-13, 1.0, n)
    A = (Uo * s) @ Vo.T
    W, H, _ = C.polar(to_dev(A))
    W, H = to_host(W), to_host(H)
    assert np.linalg.norm(W.T @ W - np.eye(n), 2) <= 50 * n * U
    assert np.linalg.norm(W @ H - A) <= 50 * n * U


@pytest.mark.parametrize("n", [64, 130, 192])
def test_tc_heig(C, n):
    rng = np.random.default_rng(n)
    X = rng.standard_normal((n, n))
    Bm = X + X.T
    lam, V, _ = C.heig(to_dev(Bm))
    lam, V = to_host(lam), to_host(V)
    lo, _ = O.heig(Bm)
    nb = np.linalg.norm(Bm, 2)
    assert np.max(np.abs(lam - lo)) <= 50 * n * U * nb
    assert np.linalg.norm(Bm @ V - V * lam) <= 50 * n * U * nb
    assert np.linalg.norm(V.T @ V - np.eye(n), 2) <= 50 * n * U


@pytest.mark.parametrize("n", [64, 97, 256])
def test_tc_csd_haar(C, n):
    A1, A2, th = I.haar_csd(n, seed=500 + n)
    R = C.csd_polar(to_dev(A1), to_dev(A2))
    ref = O.csd(A1, A2)
    _check_csd(A1, A2, R, n, theta_ref=ref["theta"], rank=n)


def test_tc_csd_clustered(C):
    n = 320
    A1, A2, th = I.clustered_csd(n, seed=2)
    R = C.csd_polar(to_dev(A1), to_dev(A2))
    ref = O.csd(A1, A2)
    _check_csd(A1, A2, R, n, theta_ref=ref["theta"], rank=n)


def test_tc_csd_rank_deficient_real(C):
    n, k = 128, 96
    A1, A2, th = I.rankdef_csd(n, k, seed=3, cplx=False, n_repeat=16)
    R = C.csd_polar(to_dev(A1), to_dev(A2))
    ref = O.csd(A1, A2)
    _check_csd(A1, A2, R, n, theta_ref=ref["theta"], rank=k)


def test_tc_csd_full_size_n4096(C):
    n = 4096
    A1h, A2h, th = I.clustered_csd(n, seed=2)
    A1, A2 = to_dev(A1h), to_dev(A2h)
    R = C.csd_polar(A1, A2)
    assert R["rank"] == n
    got, be, orth = _dev_metrics(A1, A2, R)
    assert np.max(np.abs(got - th)) <= 1e-12 * n
    assert be <= 50 * n * U
    assert orth <= 50 * n * U


@pytest.mark.parametrize("kind,n,seed", [(2, 339, 2), (4, 480, 4), (4, 480, 5), (4, 339, 4)])
def test_tc_csd_section6_families(C, kind, n, seed):
    # family 2: angles spread over 18 orders of magnitude; family 4: the same
    # with a quarter of the indices rank-deficient.  The stacked-QR rows below
    # X need the inner-dimension balance on the tensor cores (without it,
    # family 4 at n = 480 lost all accuracy); kept sines below eps need
    # Algorithm 2's W_2 in the rank-deficient case
    A1, A2 = I.paper_test(kind, n, seed=seed, cplx=False)
    R = C.csd_polar(to_dev(A1), to_dev(A2))
    ref = O.csd(A1, A2)
    _check_csd(A1, A2, R, n, theta_ref=ref["theta"], rank=ref["rank"])


def test_tc_csd_full_size_n8192(C):
    """n = 8192, the same construction as the n = 4096 workload (config 4's
    matrix): the stacked [X; sqrt(c) I] products have K > 15 360, so the
    tensor-core kernel writes its 64-bit integer sum out to C every 120
    drains (the default schedule).  Angles against the generator's (1e-12 n),
    backward error and orthogonality <= 50 n u."""
    n = 8192
    A1h, A2h, th = I.clustered_csd(n, seed=4)
    A1, A2 = to_dev(A1h), to_dev(A2h)
    del A1h, A2h
    R = C.csd_polar(A1, A2)
    assert R["rank"] == n
    got, be, orth = _dev_metrics(A1, A2, R)
    assert np.max(np.abs(got - th)) <= 1e-12 * n
    assert be <= 50 * n * U
    assert orth <= 50 * n * U


@pytest.mark.parametrize("n,k", [(160, 120), (300, 300)])
def test_tc_csd_complex(C, n, k):
    """Complex128 on the tensor-core path: every complex product with real
    alpha, beta as two real grouped sums over the interleaved parts;
    against the oracle (rank-deficient and full rank)."""
    A1, A2, th = I.rankdef_csd(n, k, seed=60 + n, cplx=True, n_repeat=n // 8)
    R = C.csd_polar(to_dev(A1), to_dev(A2))
    ref = O.csd(A1, A2)
    _check_csd(A1, A2, R, n, theta_ref=ref["theta"], rank=k)


def test_tc_complex_products_match_definition(C):
    """A complex product through the tensor-core split (polar of a complex
    matrix, whose Cholesky iteration, Gram and triangular solves all run as
    complex products) against the oracle's polar factor."""
    n = 200
    rng = np.random.default_rng(71)
    A = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
    A /= np.linalg.norm(A, 2)
    W, H, _ = C.polar(to_dev(A))
    W, H = to_host(W), to_host(H)
    Wo, Ho = O.polar(A)
    kappa = np.linalg.cond(A)
    assert np.linalg.norm(W - Wo) <= 1e-13 * n * max(kappa, 1)
    assert np.linalg.norm(W.conj().T @ W - np.eye(n), 2) <= 50 * n * U
    assert np.linalg.norm(W @ H - A) <= 50 * n * U
