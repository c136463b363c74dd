"""Oracle parity at the sizes where the kernels change shape: the 8-CTA
cluster Householder panels (panel height >= 1024), split-K products, several
levels of Zolo-eig splits.  Angles are compared with the CPU oracle element
by element (1e-12 n), plus the backward error and the 2-norm orthogonality
(50 n u), on both product engines (FP64 pipe and tensor cores)."""
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


@pytest.fixture(scope="module")
def clustered_1024():
    n = 1024
    A1, A2, th = I.clustered_csd(n, seed=2)
    return n, A1, A2, th, O.csd(A1, A2)


def _check(A1, A2, R, n, ref, rank):
    rk = R["rank"]
    assert rk == rank == ref["rank"]
    th = to_host(R["theta"])[:rk]
    assert np.all(np.diff(th) >= 0)
    err = np.max(np.abs(th - ref["theta"]))
    assert err <= 1e-12 * n, err
    U1, U2, V1 = (to_host(R[k])[:, :rk] for k in ("U1", "U2", "V1"))
    be = M.backward_error_fro(A1, A2, U1, U2, th, V1)
    assert be <= 50 * n * U, be / U
    orth = max(M.orthogonality(X) for X in (U1, U2, V1))
    assert orth <= 50 * n * U, orth / U
    return err, be, orth


@pytest.mark.parametrize("tc", [False, True])
def test_csd_n1024_clustered_matches_oracle(B, clustered_1024, tc):
    n, A1, A2, th, ref = clustered_1024
    ctx = B.Context(0)
    try:
        ctx.set_tensor_cores(tc)
        R = ctx.csd_polar(to_dev(A1), to_dev(A2))
    finally:
        ctx.close()
    _check(A1, A2, R, n, ref, n)
    # the oracle itself sits on the generator's angles (moved by the 1e-14 noise)
    assert np.max(np.abs(ref["theta"] - th)) <= 1e-12 * n


def test_csd_n512_complex_rank_deficient_matches_oracle(B):
    """Complex128, rank 384 (128 zero (C, S) pairs), 64 exactly repeated
    angles: Algorithm 3 with the split at 1.1."""
    n, k = 512, 384
    A1, A2, th = I.rankdef_csd(n, k, seed=31, cplx=True, n_repeat=64)
    ref = O.csd(A1, A2)
    R = B.csd_polar(to_dev(A1), to_dev(A2))
    assert R["info"]["mu"] == 2.0
    _check(A1, A2, R, n, ref, k)
    assert np.max(np.abs(ref["theta"] - th)) <= 1e-12 * n


@pytest.mark.parametrize("slices,scope", [(6, 1), (5, 1), (6, 3)])
def test_csd_n1024_mixed_precision_matches_oracle(B, clustered_1024, slices, scope):
    """The mixed-precision path (Cholesky-iteration products of Zolo-pd with
    5 or 6 BF16 slices; scope 3 also inside Zolo-eig) meets the same bars:
    angles within 1e-12 n of the oracle, backward error and orthogonality
    <= 50 n u."""
    n, A1, A2, th, ref = clustered_1024
    ctx = B.Context(0)
    try:
        ctx.set_tensor_cores(True)
        ctx.set_mixed_precision(slices, scope)
        R = ctx.csd_polar(to_dev(A1), to_dev(A2))
    finally:
        ctx.close()
    _check(A1, A2, R, n, ref, n)
