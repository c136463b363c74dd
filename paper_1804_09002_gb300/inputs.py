"""Seeded synthetic inputs for the CS decomposition (shared by tests and bench).

This module only *builds* matrices with a prescribed CS structure; it holds
none of the decomposition's arithmetic.  Every generator takes an explicit
seed (numpy PCG64) and returns FP64 (or complex128) column-major arrays.

Construction (Section 1): A = [A1; A2] with A1 = U1 C V^*, A2 = U2 S V^*,
C = diag(cos theta), S = diag(sin theta), U1, U2, V Haar-distributed.  Haar
factors are the Q of a QR factorisation of a Gaussian matrix with the
phases of diag(R) moved into Q (so the distribution is exactly Haar).

Workload families
  * ``haar_csd``        -- theta i.i.d. uniform on [0, pi/2] (n=64 parity case).
  * ``clustered_csd``   -- half uniform, a quarter within 1e-8 of 0 and a
                           quarter within 1e-8 of pi/2, then an additive 1e-14
                           Gaussian perturbation and re-orthonormalisation
                           (the n=4096 headline workload; kappa(A_i) ~ 1e8+).
  * ``rankdef_csd``     -- partial isometry of rank k with zero (C,S) pairs
                           and a block of exactly repeated angles.
  * ``paper_test``      -- the four families of Section 6 (Haar Stiefel,
                           clustered via cumulative sums of 10^(-18 rand),
                           rank-deficient X Y^*, rank-deficient clustered),
                           optionally with 1e-10 complex noise (tests 1'-4').
  * ``matlab_example``  -- the 3x3 example of Section 3.
"""
import numpy as np

HALF_PI = np.pi / 2


def _rng(seed):
    return np.random.default_rng(np.random.PCG64(seed))


def _gauss(rng, shape, cplx):
    if cplx:
        return (rng.standard_normal(shape) + 1j * rng.standard_normal(shape)) / np.sqrt(2.0)
    return rng.standard_normal(shape)


def _phase_fixed_qr(M):
    """Q of the QR factorisation with the diagonal of R made real >= 0."""
    Q, R = np.linalg.qr(M)
    d = np.diag(R).copy()
    ph = np.where(np.abs(d) > 0, d / np.where(np.abs(d) > 0, np.abs(d), 1), 1)
    return Q * ph[None, :]


def haar(n, rng, cplx=False, m=None):
    """m x n matrix with orthonormal columns, Haar distributed (m defaults to n)."""
    m = n if m is None else m
    return np.asfortranarray(_phase_fixed_qr(_gauss(rng, (m, n), cplx)))


def from_angles(theta, rng, cplx=False, mask=None):
    """A1 = U1 C V^*, A2 = U2 S V^* with Haar U1, U2, V.

    ``mask`` (bool, length n) marks the indices whose (C, S) pair is kept; the
    others are set to zero (rank deficiency, Theorem 2.1)."""
    n = len(theta)
    U1 = haar(n, rng, cplx)
    U2 = haar(n, rng, cplx)
    V = haar(n, rng, cplx)
    c = np.cos(theta)
    s = np.sin(theta)
    if mask is not None:
        c = np.where(mask, c, 0.0)
        s = np.where(mask, s, 0.0)
    A1 = (U1 * c[None, :]) @ V.conj().T
    A2 = (U2 * s[None, :]) @ V.conj().T
    return np.asfortranarray(A1), np.asfortranarray(A2)


def _reorthonormalise(A1, A2):
    n = A1.shape[1]
    Q = _phase_fixed_qr(np.vstack([A1, A2]))
    return np.asfortranarray(Q[:n]), np.asfortranarray(Q[n:])


def rect_csd(m1, m2, n, seed=6, cplx=False, k=None):
    """Partial isometry with rectangular blocks A_i (m_i x n, m_i >= n):
    A1 = U1[:, :n] diag(cos theta) V^*, A2 = U2[:, :n] diag(sin theta) V^*
    with Haar U1 (m1 x m1), U2 (m2 x m2), V; theta i.i.d. U[0, pi/2]; with k
    given, n - k indices get C = S = 0.  Returns (A1, A2, theta_sorted of the
    kept indices)."""
    rng = _rng(seed)
    theta = rng.uniform(0.0, HALF_PI, n)
    mask = np.ones(n, bool)
    if k is not None:
        mask[rng.permutation(n)[: n - k]] = False
    U1 = haar(m1, rng, cplx)
    U2 = haar(m2, rng, cplx)
    V = haar(n, rng, cplx)
    c = np.where(mask, np.cos(theta), 0.0)
    s = np.where(mask, np.sin(theta), 0.0)
    A1 = (U1[:, :n] * c[None, :]) @ V.conj().T
    A2 = (U2[:, :n] * s[None, :]) @ V.conj().T
    return np.asfortranarray(A1), np.asfortranarray(A2), np.sort(theta[mask])


def haar_csd(n, seed=1, cplx=False):
    """theta i.i.d. U[0, pi/2]; returns (A1, A2, theta_sorted)."""
    rng = _rng(seed)
    theta = rng.uniform(0.0, HALF_PI, n)
    A1, A2 = from_angles(theta, rng, cplx)
    return A1, A2, np.sort(theta)


def clustered_csd(n, seed=2, cplx=False, noise=1e-14, cluster=1e-8):
    """Half of theta U[0, pi/2], a quarter U[0, cluster], a quarter
    pi/2 - U[0, cluster] (shuffled); then A += noise * N(0,1) and the 2n x n
    matrix is re-orthonormalised (QR with diag(R) >= 0).  Returns
    (A1, A2, theta_sorted) where theta are the pre-perturbation angles (the
    true angles move by O(noise))."""
    rng = _rng(seed)
    h = n // 2
    q = (n - h) // 2
    theta = np.concatenate([
        rng.uniform(0.0, HALF_PI, h),
        rng.uniform(0.0, cluster, q),
        HALF_PI - rng.uniform(0.0, cluster, n - h - q),
    ])
    rng.shuffle(theta)
    A1, A2 = from_angles(theta, rng, cplx)
    if noise:
        A1 = A1 + noise * _gauss(rng, A1.shape, cplx)
        A2 = A2 + noise * _gauss(rng, A2.shape, cplx)
        A1, A2 = _reorthonormalise(A1, A2)
    return A1, A2, np.sort(theta)


def rankdef_csd(n, k, seed=3, cplx=True, n_repeat=None):
    """Partial isometry of rank k: n-k indices get C = S = 0; n_repeat of the
    remaining indices share one angle; the rest are U[0, pi/2].  Returns
    (A1, A2, theta_sorted_of_rank_part)."""
    rng = _rng(seed)
    n_repeat = (n // 8) if n_repeat is None else n_repeat
    t0 = rng.uniform(0.0, HALF_PI)
    theta_r = np.concatenate([np.full(n_repeat, t0), rng.uniform(0.0, HALF_PI, k - n_repeat)])
    theta = np.concatenate([theta_r, np.zeros(n - k)])
    mask = np.concatenate([np.ones(k, bool), np.zeros(n - k, bool)])
    perm = rng.permutation(n)
    theta, mask = theta[perm], mask[perm]
    A1, A2 = from_angles(theta, rng, cplx, mask=mask)
    return A1, A2, np.sort(theta_r)


def paper_test(kind, n, seed=0, cplx=True, noisy=False):
    """The test families of Section 6.  kind in {1, 2, 3, 4}.  Returns (A1, A2)."""
    rng = _rng(seed)
    if kind == 1:
        A = haar(n, rng, cplx, m=2 * n)
        A1, A2 = A[:n], A[n:]
    elif kind in (2, 4):
        delta = 10.0 ** (-18.0 * rng.uniform(size=n + 1))
        theta = HALF_PI * np.cumsum(delta[:n]) / np.sum(delta)
        mask = None
        if kind == 4:
            r = int(np.floor(3 * n / 4 + 0.5))
            mask = np.ones(n, bool)
            mask[rng.permutation(n)[: n - r]] = False
        A1, A2 = from_angles(theta, rng, cplx, mask=mask)
    elif kind == 3:
        r = int(np.floor(3 * n / 4 + 0.5))
        X = haar(r, rng, cplx, m=2 * n)
        Y = haar(r, rng, cplx, m=n)
        A = X @ Y.conj().T
        A1, A2 = A[:n], A[n:]
    else:
        raise ValueError("kind must be 1..4")
    if noisy:
        A1 = A1 + 1e-10 * (rng.standard_normal(A1.shape) + (1j * rng.standard_normal(A1.shape) if cplx else 0))
        A2 = A2 + 1e-10 * (rng.standard_normal(A2.shape) + (1j * rng.standard_normal(A2.shape) if cplx else 0))
    return np.asfortranarray(A1), np.asfortranarray(A2)


def paper_sizes():
    """n = nint(30 * 2^(j/2)), j = 0..9 (Section 6)."""
    return [int(np.floor(30 * 2 ** (j / 2) + 0.5)) for j in range(10)]


def matlab_example():
    """The 3x3 example of Section 3: theta = [1, 2, 3] * 1e-8 and a fixed V1.
    Returns (H1, H2, V1, theta)."""
    theta = np.array([1e-8, 2e-8, 3e-8])
    V1 = np.array([[2.0, -1.0, 2.0], [2.0, 2.0, -1.0], [1.0, -2.0, -2.0]]) / 3.0
    H1 = V1 @ np.diag(np.cos(theta)) @ V1.T
    H2 = V1 @ np.diag(np.sin(theta)) @ V1.T
    return H1, H2, V1, theta


def batch_sizes(count, lo=16, hi=256, seed=5):
    """Sizes n_i ~ U{lo..hi} for the batched workload."""
    return _rng(seed).integers(lo, hi + 1, size=count).tolist()
