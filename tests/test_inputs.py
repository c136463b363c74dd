"""The seeded input generators follow the stated recipes: [A1; A2] has
orthonormal columns (or is the stated partial isometry), the singular values
of the blocks are the cosines / sines of the angles the generator reports,
the clustered recipe has its half / quarter / quarter split, and the same
seed gives the same matrices."""
import numpy as np
import pytest

from paper_1804_09002_gb300 import inputs as I

U = 2.0 ** -53


def _orth_err(A1, A2):
    A = np.vstack([A1, A2])
    return np.linalg.norm(A.conj().T @ A - np.eye(A.shape[1]), 2)


@pytest.mark.parametrize("cplx", [False, True])
def test_haar_csd_orthonormal_and_angles(cplx):
    n = 48
    A1, A2, th = I.haar_csd(n, seed=3, cplx=cplx)
    assert A1.dtype == (np.complex128 if cplx else np.float64)
    assert _orth_err(A1, A2) <= 50 * n * U
    assert np.all((th >= 0) & (th <= np.pi / 2)) and np.all(np.diff(th) >= 0)
    s1 = np.sort(np.linalg.svd(A1, compute_uv=False))
    assert np.max(np.abs(s1 - np.sort(np.cos(th)))) <= 1e-13


def test_clustered_recipe():
    n = 200
    A1, A2, th = I.clustered_csd(n, seed=2)
    assert _orth_err(A1, A2) <= 50 * n * U
    near0 = np.sum(th <= 1e-8)
    nearpi2 = np.sum(th >= np.pi / 2 - 1e-8)
    assert near0 >= n // 4 and nearpi2 >= n - n // 2 - n // 4
    # the 1e-14 perturbation moves the singular values by O(1e-14)
    s2 = np.sort(np.linalg.svd(A2, compute_uv=False))
    assert np.max(np.abs(s2 - np.sort(np.sin(th)))) <= 1e-12


def test_rankdef_partial_isometry():
    n, k = 40, 30
    A1, A2, th = I.rankdef_csd(n, k, seed=4, cplx=True, n_repeat=5)
    A = np.vstack([A1, A2])
    s = np.linalg.svd(A, compute_uv=False)
    assert np.sum(s > 0.5) == k and np.max(np.abs(s[:k] - 1)) <= 1e-13 and np.max(s[k:]) <= 1e-13
    assert len(th) == k and np.max(np.unique(th, return_counts=True)[1]) >= 5  # n_repeat equal angles
    # ||A||_F^2 = rank (remark (vi))
    assert abs(np.linalg.norm(A) ** 2 - k) <= 1e-12


@pytest.mark.parametrize("kind", [1, 2, 3, 4])
def test_section6_families(kind):
    n = 30
    A1, A2 = I.paper_test(kind, n, seed=kind, cplx=True)
    A = np.vstack([A1, A2])
    s = np.linalg.svd(A, compute_uv=False)
    r = n if kind in (1, 2) else int(np.floor(3 * n / 4 + 0.5))
    assert np.max(np.abs(s[:r] - 1)) <= 1e-13
    assert r == n or np.max(s[r:]) <= 1e-13


def test_paper_sizes():
    assert I.paper_sizes() == [30, 42, 60, 85, 120, 170, 240, 339, 480, 679]


def test_seeded():
    a = I.clustered_csd(32, seed=9)
    b = I.clustered_csd(32, seed=9)
    assert all(np.array_equal(x, y) for x, y in zip(a, b))
    c = I.clustered_csd(32, seed=10)
    assert not np.array_equal(a[0], c[0])
