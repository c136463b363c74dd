"""CPU models of two facts the level-batched Zolo-eig relies on (Section 5,
the spectral divide-and-conquer paragraph):

* padding a block with an identity block is exactly decoupled: the polar
  factor of diag(X, I) is diag(polar(X), I), and the Householder QR of a
  matrix whose rows below the block are zero (with unit columns on the
  padding) has Q = diag(Q_block, I) with exact zeros, because every
  reflector of a zero sub-column is the identity (tau = 0, the convention
  of the panel kernels);
* the basis from qr(P Omega) with a square Gaussian Omega can miss range(P)
  by about cond(P Omega_1) u, and one step of subspace iteration,
  Q <- qr(P Q), brings the off-diagonal block of Q^* B Q down to rounding.
"""
import numpy as np


def householder_qr(M):
    """Unblocked Householder QR with the larfg convention: a column whose
    entries below the diagonal are exactly zero (and real diagonal) gets
    tau = 0.  Returns the explicit Q."""
    A = np.array(M, dtype=np.float64, copy=True)
    m, n = A.shape
    vs, taus = [], []
    for k in range(min(m, n)):
        x = A[k:, k].copy()
        alpha, rest = x[0], x[1:]
        xnorm2 = float(rest @ rest)
        if xnorm2 == 0.0:
            tau, v = 0.0, np.zeros_like(x)
            v[0] = 1.0
        else:
            beta = -np.copysign(np.sqrt(alpha * alpha + xnorm2), alpha)
            tau = (beta - alpha) / beta
            v = x / (alpha - beta)
            v[0] = 1.0
        A[k:, k:] -= tau * np.outer(v, v @ A[k:, k:])
        vs.append(v)
        taus.append(tau)
    Q = np.eye(m)
    for k in reversed(range(len(vs))):
        Q[k:, :] -= taus[k] * np.outer(vs[k], vs[k] @ Q[k:, :])
    return Q


def sign_polar(X):
    """Unitary polar factor of a symmetric X (its matrix sign)."""
    lam, V = np.linalg.eigh(X)
    return (V * np.sign(lam)) @ V.T


def test_padded_polar_is_block_diagonal():
    rng = np.random.default_rng(3)
    sz, nb = 37, 50
    G = rng.standard_normal((sz, sz))
    X = (G + G.T) / np.linalg.norm(G + G.T)
    Xp = np.eye(nb)
    Xp[:sz, :sz] = X
    U, _, Vt = np.linalg.svd(Xp)
    Wp = U @ Vt
    W = sign_polar(X)
    assert np.max(np.abs(Wp[:sz, :sz] - W)) < 1e-12
    assert np.max(np.abs(Wp[sz:, :sz])) < 1e-13 and np.max(np.abs(Wp[:sz, sz:])) < 1e-13
    assert np.max(np.abs(Wp[sz:, sz:] - np.eye(nb - sz))) < 1e-13


def test_householder_of_padded_basis_is_exactly_block_diagonal():
    rng = np.random.default_rng(4)
    sz, nb = 23, 32
    Mp = np.zeros((nb, nb))
    Mp[:sz, :] = rng.standard_normal((sz, nb))  # P Omega: zero rows below the block
    Mp[sz:, sz:] = np.eye(nb - sz)  # identity columns on the padding
    Mp[:sz, sz:] = rng.standard_normal((sz, nb - sz))  # junk above them: must not matter
    Q = householder_qr(Mp)
    # exact zeros, not small numbers: the padding never mixes with the block
    assert np.all(Q[sz:, :sz] == 0.0) and np.all(Q[:sz, sz:] == 0.0)
    assert np.array_equal(Q[sz:, sz:], np.eye(nb - sz))
    Qb = householder_qr(Mp[:sz, :sz])
    assert np.max(np.abs(Q[:sz, :sz] - Qb)) < 1e-14


def test_one_subspace_step_repairs_the_basis():
    rng = np.random.default_rng(7)
    n, k = 300, 140
    V, _ = np.linalg.qr(rng.standard_normal((n, n)))
    lam = np.concatenate([rng.uniform(0.1, 1.0, k), rng.uniform(-1.0, -0.1, n - k)])
    B = (V * lam) @ V.T
    B = (B + B.T) / 2
    P = (sign_polar(B) + np.eye(n)) / 2
    u = 2.0 ** -53
    off = lambda Q: np.linalg.norm((Q.T @ B @ Q)[k:, :k])
    Om = rng.standard_normal((n, n))
    Q0 = householder_qr(P @ Om)
    Q1 = householder_qr(P @ Q0)
    e0, e1 = off(Q0), off(Q1)
    bound = 10 * np.sqrt(n) * u * np.linalg.norm(B)
    assert e1 <= bound, (e1, bound)
    assert e1 < e0 / 5  # the refined basis is much better than the Gaussian one
    # a planted mistake: refining with the complement projector loses range(P)
    Qbad = householder_qr((np.eye(n) - P) @ Q0)
    assert off(Qbad) > 1e-3
