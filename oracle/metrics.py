"""Oracle (test infrastructure only; never on the product path).

Accuracy measures of Section 6 and Theorem 3.1, in FP64 with numpy.
"""
import numpy as np

U_ROUND = 2.0 ** -53


def reconstruct(U1, U2, theta, V1):
    """A_hat = [U1 diag(cos theta) V1^*; U2 diag(sin theta) V1^*]."""
    c, s = np.cos(theta), np.sin(theta)
    return (U1 * c[None, :]) @ V1.conj().T, (U2 * s[None, :]) @ V1.conj().T


def backward_error_fro(A1, A2, U1, U2, theta, V1):
    """||A - A_hat||_F / ||A||_F."""
    B1, B2 = reconstruct(U1, U2, theta, V1)
    num = np.sqrt(np.linalg.norm(A1 - B1) ** 2 + np.linalg.norm(A2 - B2) ** 2)
    den = np.sqrt(np.linalg.norm(A1) ** 2 + np.linalg.norm(A2) ** 2)
    return num / den


def residual_2(A1, A2, U1, U2, theta, V1):
    """||A_hat - A||_2 (the numerator of the scaled residual of Section 6)."""
    B1, B2 = reconstruct(U1, U2, theta, V1)
    return np.linalg.norm(np.vstack([A1 - B1, A2 - B2]), 2)


def orthogonality(U):
    """||U^* U - I||_2."""
    k = U.shape[1]
    return np.linalg.norm(U.conj().T @ U - np.eye(k), 2)


def dist_partial_isometry(A1, A2):
    """d(A) = max_i min(sigma_i, |1 - sigma_i|) (distance to the nearest
    partial isometry, Section 2)."""
    s = np.linalg.svd(np.vstack([A1, A2]), compute_uv=False)
    return float(np.max(np.minimum(s, np.abs(1.0 - s))))
