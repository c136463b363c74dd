"""Oracle (test infrastructure only; never on the product path).

Algorithm 1 (CS decomposition via two polar decompositions), with the
rank-deficient modification of Algorithm 3 and the post-processing of
remark (iii), written out step by step in FP64 with *independent* sub-solvers:

  * polar decomposition A_i = W_i H_i by one-sided Jacobi SVD
    (A V = U Sigma, W = U V^*, H = V Sigma V^*; Section 1, eqs. for A1/A2),
  * Hermitian eigendecomposition of B by cyclic Jacobi.

Readings taken where the paper leaves a choice:
  * rank r = round(||A||_F^2) and mu = 0 if r = n else 2 (remark (vi), line 3);
  * H_i symmetrised as (H + H^*)/2 (Theorem 3.1 assumes H Hermitian);
  * theta = atan2(S, C) (remark (iii), arctan(S/C) read with quadrant),
    clamped to [0, pi/2], the range of the principal angles (Section 1);
  * angles returned ascending (Section 1 orders 0 <= theta_1 <= ... );
  * for mu = 2 the eigenvalues with Lambda <= 1.5 are kept (Algorithm 3,
    line 5 keeps those in [-1, 1]; the others sit at mu = 2).
"""
import numpy as np

from . import jacobi


def _ct(X):
    return X.conj().T


def _complete_columns(U, ok):
    """Replace the columns of U flagged not ok by an orthonormal completion:
    for each, project every unit vector e_k off the columns kept so far
    (Gram-Schmidt, twice) and take the longest residual, normalised (its
    length is at least 1/sqrt(m) when the kept columns are orthonormal)."""
    m, n = U.shape
    U = U.copy()
    basis = np.array([U[:, j] for j in range(n) if ok[j]]).T.reshape(m, -1)
    for j in range(n):
        if ok[j]:
            continue
        E = np.eye(m, dtype=U.dtype)
        for _ in range(2):
            E = E - basis @ (basis.conj().T @ E)
        norms = np.linalg.norm(E, axis=0)
        k = int(np.argmax(norms))
        v = E[:, k] / norms[k]
        U[:, j] = v
        basis = np.hstack([basis, v[:, None]])
    return U


def polar(A):
    """Polar decomposition A = W H (W with orthonormal columns, H Hermitian
    PSD) from the one-sided Jacobi SVD.  Columns of A V that are exactly zero
    (sigma = 0) get an orthonormal completion, so W is always orthonormal."""
    G, V, sigma, _ = jacobi.svd_onesided(A)
    ok = sigma > 1e-290
    U = G / np.where(ok, sigma, 1.0)[None, :]
    if not np.all(ok):
        U = _complete_columns(U, ok)
    W = U @ _ct(V)
    H = (V * sigma[None, :]) @ _ct(V)
    H = 0.5 * (H + _ct(H))
    return W, H


def heig(B):
    """Eigendecomposition B = V diag(lam) V^* of a Hermitian B by cyclic
    Jacobi, eigenvalues ascending (stable order for ties)."""
    lam, V, _ = jacobi.eig_cyclic(B)
    order = np.argsort(lam, kind="stable")
    return lam[order], V[:, order]


def rank_and_mu(A1, A2):
    """Remark (vi): ||A||_F ~ sqrt(rank(A)) for a near partial isometry."""
    n = A1.shape[1]
    fro2 = float(np.sum(np.abs(A1) ** 2) + np.sum(np.abs(A2) ** 2))
    r = int(np.floor(fro2 + 0.5))
    r = max(0, min(n, r))
    return r, (0.0 if r == n else 2.0)


def csd(A1, A2, mu=None, theta_from="cs"):
    """CS decomposition of the 2n x n partial isometry [A1; A2].

    theta_from = "cs": theta = atan2(S, C) with C, S = diag(V^* H_i V)
    (lines 8-9, remark (iii)); "lambda": theta solves
    sin(theta) - cos(theta) = Lambda (remark (iv)).

    Returns a dict with theta (ascending, length r), U1, U2 (n x r),
    V1 (n x r), C, S (length r), Lambda (eigenvalues of B, ascending), rank,
    mu, W1, W2, H1, H2, B."""
    A1 = np.asarray(A1)
    A2 = np.asarray(A2)
    n = A1.shape[1]
    r, mu_auto = rank_and_mu(A1, A2)
    mu = mu_auto if mu is None else float(mu)
    # lines 1-2: two polar decompositions
    W1, H1 = polar(A1)
    W2, H2 = polar(A2)
    # line 4: B = H2 - H1 + mu (I - A^* A)
    B = H2 - H1
    if mu != 0.0:
        AtA = _ct(A1) @ A1 + _ct(A2) @ A2
        B = B + mu * (np.eye(n) - AtA)
    B = 0.5 * (B + _ct(B))
    # line 5: symmetric eigendecomposition
    lam, V = heig(B)
    if mu != 0.0:
        keep = lam <= 1.5          # Algorithm 3, line 5
        V = V[:, keep]
        lam_r = lam[keep]
    else:
        lam_r = lam
    # lines 6-9
    U1 = W1 @ V
    U2 = W2 @ V
    C = np.real(np.einsum("ij,ij->j", V.conj(), H1 @ V))
    S = np.real(np.einsum("ij,ij->j", V.conj(), H2 @ V))
    # remark (iii): theta = arctan(S/C), then C = cos(theta), S = sin(theta);
    # the principal angles lie in [0, pi/2] (Section 1), so rounding below 0
    # or above pi/2 is clamped
    theta = np.clip(np.arctan2(S, C), 0.0, np.pi / 2)
    if theta_from == "lambda":
        # sin(t) - cos(t) = sqrt(2) sin(t - pi/4) = Lambda
        theta = np.clip(np.pi / 4 + np.arcsin(np.clip(lam_r / np.sqrt(2.0), -1.0, 1.0)), 0.0, np.pi / 2)
    elif theta_from != "cs":
        raise ValueError("theta_from must be 'cs' or 'lambda'")
    order = np.argsort(theta, kind="stable")
    theta = theta[order]
    U1, U2, V = U1[:, order], U2[:, order], V[:, order]
    return dict(theta=theta, C=np.cos(theta), S=np.sin(theta), U1=U1, U2=U2, V1=V,
                Lambda=lam, Lambda_r=lam_r[order], rank=V.shape[1], mu=mu,
                W1=W1, W2=W2, H1=H1, H2=H2, B=B)


def complete_v2(A3, A4, U1, U2, theta):
    """Remark (viii): V2 of the complete 2 x 2 CS decomposition of a unitary
    [A1 A3; A2 A4], given U1, U2, theta of [A1; A2]:
    X = -A3^* U1 S + A4^* U2 C, X = Q R with diag(R) >= 0, V2 = Q."""
    C = np.cos(theta)
    S = np.sin(theta)
    X = -_ct(A3) @ (U1 * S[None, :]) + _ct(A4) @ (U2 * C[None, :])
    Q, R = np.linalg.qr(X)
    d = np.diag(R)
    ph = np.where(np.abs(d) > 0, d / np.where(np.abs(d) > 0, np.abs(d), 1.0), 1.0)
    return Q * ph[None, :]
