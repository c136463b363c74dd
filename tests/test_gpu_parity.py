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


# ------------------------------------------------------------------ tall panels
@pytest.mark.parametrize("n", [1000, 1100])
def test_polar_large_properties(B, n):
    """n >= 1000 exercises the cluster (multi-CTA) Householder panel of the
    stacked [X; sqrt(c) I] QR (panel height n + 32 >= 1024).  Properties that
    hold at any size: W orthonormal, W H = A, H Hermitian positive
    semidefinite; W equals U V^T of the matrix built from a known SVD."""
    rng = np.random.default_rng(n)
    Uo = np.linalg.qr(rng.standard_normal((n, n)))[0]
    Vo = np.linalg.qr(rng.standard_normal((n, n)))[0]
    s = np.geomspace(1e-6, 1.0, n)
    A = (Uo * s) @ Vo.T
    W, H, info = B.polar(to_dev(A))
    W, H = to_host(W), to_host(H)
    assert np.linalg.norm(W.T @ W - np.eye(n), 2) <= 50 * n * U
    assert np.linalg.norm(W @ H - A) <= 50 * n * U * np.linalg.norm(A)
    assert np.linalg.norm(H - H.T) == 0.0
    assert np.min(np.linalg.eigvalsh(H)) >= -50 * n * U
    assert np.linalg.norm(W - Uo @ Vo.T) <= 1e-8


def test_csd_large_clustered_known_angles(B):
    """n = 1024 clustered workload: angles against the generator's known
    angles (the 1e-14 perturbation moves them by O(1e-14)), backward error
    and orthogonality; the oracle is too slow at this size, so the checks
    are the properties that hold at any size."""
    n = 1024
    A1, A2, th = I.clustered_csd(n, seed=2)
    R = B.csd_polar(to_dev(A1), to_dev(A2))
    _check_csd(A1, A2, R, n, theta_ref=th, rank=n)


# ------------------------------------------------------------------ full-size workloads
def _dev_metrics(A1, A2, R):
    """Angles, backward error and orthogonality computed with torch on the
    GPU (the matrices are too large for a quick host check)."""
    rk = R["rank"]
    th = R["theta"][:rk]
    U1, U2, V1 = (R[k][:, :rk] for k in ("U1", "U2", "V1"))
    c = torch.cos(th).to(U1.dtype)
    s = torch.sin(th).to(U1.dtype)
    Vh = V1.conj().T
    r1 = A1 - (U1 * c) @ Vh
    r2 = A2 - (U2 * s) @ Vh
    num = torch.sqrt(torch.linalg.norm(r1) ** 2 + torch.linalg.norm(r2) ** 2)
    den = torch.sqrt(torch.linalg.norm(A1) ** 2 + torch.linalg.norm(A2) ** 2)
    eye = torch.eye(rk, dtype=U1.dtype, device=U1.device)
    orth = max(float(torch.linalg.norm(X.conj().T @ X - eye)) for X in (U1, U2, V1))
    return th.cpu().numpy(), float(num / den), orth


def test_csd_full_size_n4096_clustered(B):
    """The n = 4096 workload (theta half uniform, quarters within 1e-8 of 0
    and pi/2, 1e-14 noise, re-orthonormalised): angles within 1e-12 n of the
    generator's, backward error <= 50 n u, ||X^* X - I||_F <= 50 n u."""
    n = 4096
    A1h, A2h, th = I.clustered_csd(n, seed=2)
    A1, A2 = to_dev(A1h), to_dev(A2h)
    R = B.csd_polar(A1, A2)
    assert R["rank"] == n
    got, be, orth = _dev_metrics(A1, A2, R)
    assert np.all(np.diff(got) >= 0)
    assert np.max(np.abs(got - th)) <= 1e-12 * n
    assert be <= 50 * n * U
    assert orth <= 50 * n * U


def test_csd_full_size_n2048_complex_rank_deficient(B):
    """Complex128 partial isometry, n = 2048, rank 1536 with 512 zero (C, S)
    pairs and 256 exactly repeated angles (Algorithm 3, mu = 2)."""
    n, k = 2048, 1536
    A1h, A2h, th = I.rankdef_csd(n, k, seed=3, cplx=True, n_repeat=256)
    A1, A2 = to_dev(A1h), to_dev(A2h)
    R = B.csd_polar(A1, A2)
    assert R["rank"] == k and R["info"]["mu"] == 2.0
    got, be, orth = _dev_metrics(A1, A2, R)
    assert np.max(np.abs(got - th)) <= 1e-12 * n
    assert be <= 50 * n * U
    assert orth <= 50 * n * U


def test_csd_algorithm2_exact_zero_angles(B):
    """theta containing exactly 0 and pi/2: A2 (resp. A1) has a zero singular
    value below eps = 1e-15, so the eps-modified Zolo-pd factor is not
    orthonormal and Algorithm 2 (QR of A_i and H_i, W_i = Q_i Q~_i^*) must
    restore it; the rank is still n (mu = 0)."""
    n = 64
    rng = np.random.default_rng(77)
    theta = rng.uniform(0, np.pi / 2, n)
    theta[:3] = 0.0
    theta[3:5] = np.pi / 2
    A1, A2 = I.from_angles(theta, rng)
    R = B.csd_polar(to_dev(A1), to_dev(A2))
    info = R["info"]
    assert R["rank"] == n and info["mu"] == 0.0
    assert info["alg2_used"][0] == 1 and info["alg2_used"][1] == 1
    assert max(info["rdiff"]) <= 1e3 * n * U
    ref = O.csd(A1, A2)
    _check_csd(A1, A2, R, n, theta_ref=ref["theta"], rank=n)
    assert np.max(np.abs(to_host(R["theta"]) - np.sort(theta))) <= 1e-12 * n


@pytest.mark.parametrize("kind,n,seed", [(2, 339, 2), (4, 339, 4), (4, 480, 5)])
def test_csd_section6_families(B, kind, n, seed):
    """Section 6 families 2 and 4 (angles over 18 orders of magnitude; family
    4 rank-deficient).  A kept angle with sine (or cosine) below eps in the
    rank-deficient case needs Algorithm 2's W_i (Section 5.2, last
    paragraph): without it U_2 lost orthogonality (|U_2^* U_2 - I| ~ 0.3)."""
    A1, A2 = I.paper_test(kind, n, seed=seed, cplx=False)
    R = B.csd_polar(to_dev(A1), to_dev(A2))
    ref = O.csd(A1, A2)
    if kind == 4:
        assert R["info"]["mu"] == 2.0 and max(R["info"]["alg2_used"]) == 1
    _check_csd(A1, A2, R, n, theta_ref=ref["theta"], rank=ref["rank"])


def test_csd_rank_deficient_kept_zero_sine(B):
    """Rank-deficient input whose kept angles include sines below eps: W_2
    from Algorithm 2 keeps U_2 orthonormal."""
    n, k = 96, 72
    rng = np.random.default_rng(91)
    theta = rng.uniform(0, np.pi / 2, n)
    theta[:4] = 10.0 ** rng.uniform(-19, -16, 4)
    mask = np.ones(n, bool)
    mask[rng.permutation(np.arange(4, n))[: n - k]] = False
    A1, A2 = I.from_angles(theta, rng, mask=mask)
    R = B.csd_polar(to_dev(A1), to_dev(A2))
    assert R["info"]["mu"] == 2.0 and R["info"]["alg2_used"][1] == 1
    ref = O.csd(A1, A2)
    _check_csd(A1, A2, R, n, theta_ref=ref["theta"], rank=k)


# ------------------------------------------------ remarks (iv) and (viii)
@pytest.mark.parametrize("case", ["haar", "rankdef"])
def test_csd_theta_from_lambda(B, case):
    """Remark (iv): theta from sin(theta) - cos(theta) = Lambda (context mode
    1) against the oracle's same reading, plus the CSD bars."""
    if case == "haar":
        n, k = 100, 100
        A1, A2, th = I.haar_csd(n, seed=73)
    else:
        n, k = 64, 48
        A1, A2, th = I.rankdef_csd(n, k, seed=74, cplx=False, n_repeat=8)
    ctx = B.Context(0)
    try:
        ctx.set_theta_mode(1)
        R = ctx.csd_polar(to_dev(A1), to_dev(A2))
    finally:
        ctx.close()
    ref = O.csd(A1, A2, theta_from="lambda")
    _check_csd(A1, A2, R, n, theta_ref=ref["theta"], rank=k)
    assert np.max(np.abs(to_host(R["theta"])[:k] - th)) <= 1e-12 * n


@pytest.mark.parametrize("n,cplx", [(64, False), (130, False), (40, True)])
def test_complete_v2(B, n, cplx):
    """Remark (viii): V2 of the complete 2 x 2 CSD of a unitary 2n x 2n.
    (a) From the oracle's U1, U2, theta, the GPU V2 equals the oracle's
    (X is unitary up to O(u), so its QR with diag(R) >= 0 is well
    conditioned); (b) from the GPU's own csd_polar outputs,
    A3 = -U1 S V2^* and A4 = U2 C V2^* to 50 n u, V2 unitary."""
    rng = np.random.default_rng(90 + n)
    Q = I.haar(2 * n, rng, cplx)
    A1, A2, A3, A4 = Q[:n, :n], Q[n:, :n], Q[:n, n:], Q[n:, n:]
    ref = O.csd(A1, A2)
    V2o = O.complete_v2(A3, A4, ref["U1"], ref["U2"], ref["theta"])
    V2 = to_host(B.default_context(0).complete_v2(to_dev(A3), to_dev(A4), to_dev(ref["U1"]), to_dev(ref["U2"]),
                                                  torch.from_numpy(ref["theta"]).cuda()))
    assert np.max(np.abs(V2 - V2o)) <= 1e-12 * n
    R = B.csd_polar(to_dev(A1), to_dev(A2))
    U1, U2, th = to_host(R["U1"]), to_host(R["U2"]), to_host(R["theta"])
    V2g = to_host(B.default_context(0).complete_v2(to_dev(A3), to_dev(A4), R["U1"], R["U2"], R["theta"]))
    C, S = np.cos(th), np.sin(th)
    r3 = np.linalg.norm(A3 + (U1 * S[None, :]) @ V2g.conj().T) / np.sqrt(n)
    r4 = np.linalg.norm(A4 - (U2 * C[None, :]) @ V2g.conj().T) / np.sqrt(n)
    assert max(r3, r4) <= 50 * n * U
    assert M.orthogonality(V2g) <= 50 * n * U


def test_complete_v2_host_pointers(B):
    n = 33
    rng = np.random.default_rng(95)
    Q = I.haar(2 * n, rng, False)
    A1, A2, A3, A4 = Q[:n, :n], Q[n:, :n], Q[:n, n:], Q[n:, n:]
    ref = O.csd(A1, A2)
    V2o = O.complete_v2(A3, A4, ref["U1"], ref["U2"], ref["theta"])
    V2 = B.default_context(0).complete_v2(np.asfortranarray(A3), np.asfortranarray(A4), ref["U1"], ref["U2"],
                                          ref["theta"])
    assert isinstance(V2, np.ndarray)
    assert np.max(np.abs(V2 - V2o)) <= 1e-12 * n


@pytest.mark.parametrize("m1,m2,n,cplx,k", [(80, 70, 48, False, None), (130, 100, 100, False, None),
                                           (60, 50, 40, True, None), (72, 64, 48, False, 36)])
def test_csd_rectangular(B, m1, m2, n, cplx, k):
    """Rectangular blocks (csd_polar_rect): QR of each block, square CSD of
    [R1; R2], U_i = Q_i U_i'; against the oracle, which takes the
    rectangular polar decompositions directly."""
    A1, A2, th = I.rect_csd(m1, m2, n, seed=m1 + n, cplx=cplx, k=k)
    R = B.default_context(0).csd_polar_rect(to_dev(A1), to_dev(A2))
    ref = O.csd(A1, A2)
    r = ref["rank"]
    assert R["rank"] == r
    got = to_host(R["theta"])[:r]
    assert np.all(np.diff(got) >= 0) and np.all(got >= 0) and np.all(got <= np.pi / 2 + 1e-15)
    assert np.max(np.abs(got - ref["theta"])) <= 1e-12 * n
    assert np.max(np.abs(got - th)) <= 1e-12 * n
    U1, U2, V1 = (to_host(R[key])[:, :r] for key in ("U1", "U2", "V1"))
    assert U1.shape == (m1, r) and U2.shape == (m2, r)
    be = M.backward_error_fro(A1, A2, U1, U2, got, V1)
    assert be <= 50 * n * U, be
    for X in (U1, U2, V1):
        assert M.orthogonality(X) <= 50 * n * U


@pytest.mark.parametrize("m1,m2,n", [(1, 3, 1), (33, 33, 33), (65, 64, 64), (200, 40, 40)])
def test_csd_rectangular_edges(B, m1, m2, n):
    """Edge shapes of csd_polar_rect: n = 1, square blocks through the
    rectangular entry point, one extra row, a block five times taller."""
    A1, A2, th = I.rect_csd(m1, m2, n, seed=7 + m1 + m2, cplx=False)
    R = B.default_context(0).csd_polar_rect(A1, A2)  # host arrays: staged by the library
    ref = O.csd(A1, A2)
    assert R["rank"] == n and isinstance(R["U1"], np.ndarray)
    got = R["theta"][:n]
    assert np.max(np.abs(got - ref["theta"])) <= 1e-12 * max(n, 1)
    be = M.backward_error_fro(A1, A2, R["U1"], R["U2"], got, R["V1"])
    assert be <= 50 * max(n, 2) * U, be
    for X in (R["U1"], R["U2"], R["V1"]):
        assert M.orthogonality(X) <= 50 * max(n, 2) * U


# ------------------------------------------------ Section 5.1: SVD fallback
@pytest.mark.parametrize("case,cplx", [("exact_zero", False), ("clustered", False), ("exact_zero", True)])
def test_csd_svd_polar_fallback(B, case, cplx):
    """Algorithm 2's check ||R~ - R|| (Section 5.1): with the fallback
    threshold forced to 0 every block that takes Algorithm 2 recomputes its
    polar decomposition through the SVD (one-sided Jacobi); the CSD still
    matches the oracle and the bars hold.  Exactly zero angles make both
    blocks singular (zero columns of G get the orthonormal completion)."""
    rng = np.random.default_rng(88 + cplx)
    if case == "exact_zero":
        n = 64
        theta = rng.uniform(0, np.pi / 2, n)
        theta[:3] = 0.0
        theta[3:5] = np.pi / 2
        A1, A2 = I.from_angles(theta, rng, cplx)
    else:
        n = 96
        A1, A2, _ = I.clustered_csd(n, seed=9, noise=0.0, cluster=1e-17)
    ctx = B.Context(0)
    try:
        ctx.set_alg2_fallback(0.0)
        R = ctx.csd_polar(to_dev(A1), to_dev(A2))
    finally:
        ctx.close()
    info = R["info"]
    assert max(info["alg2_used"]) == 2
    ref = O.csd(A1, A2)
    _check_csd(A1, A2, R, n, theta_ref=ref["theta"], rank=n)


def test_svd_fallback_default_threshold_keeps_algorithm2(B):
    """At the default threshold the exact-zero case keeps Algorithm 2's W_i
    (||R~ - R|| is a small multiple of u, as the paper observed)."""
    n = 64
    rng = np.random.default_rng(77)
    theta = rng.uniform(0, np.pi / 2, n)
    theta[:3] = 0.0
    A1, A2 = I.from_angles(theta, rng)
    R = B.csd_polar(to_dev(A1), to_dev(A2))
    assert 1 in R["info"]["alg2_used"] and 2 not in R["info"]["alg2_used"]
