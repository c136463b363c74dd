"""Oracle (test infrastructure only; never on the product path).

Reverse-mode derivative of the full-rank real CS decomposition as Algorithm 1
computes it (the paper itself has no derivatives):

    A_i = W_i H_i                      polar decompositions (lines 1-2)
    B   = H_2 - H_1                    line 4 (mu = 0)
    B   = V diag(lam) V^T              line 5, lam ascending
    U_i = W_i V                        line 6
    c   = diag(V^T H_1 V), s = diag(V^T H_2 V),  theta = atan2(s, c)   lines 8-9

Given gradients (theta_bar, U1_bar, U2_bar, V_bar) of a scalar loss, returns
(A1_bar, A2_bar).  Every step is differentiated where it stands, in the
original basis, with the oracle's own sub-solvers:

  * theta = atan2(s, c):        c_bar = -s / (c^2 + s^2) theta_bar,
                                s_bar =  c / (c^2 + s^2) theta_bar;
  * c_j = v_j^T H_1 v_j:         H1_bar += V diag(c_bar) V^T,  V_bar += 2 H_1 V diag(c_bar)
    (likewise s with H_2);
  * U_i = W_i V:                 W_i_bar += U_i_bar V^T,       V_bar += W_i^T U_i_bar;
  * B = V diag(lam) V^T:         B_bar = V (F o skew(V^T V_bar)) V^T,
                                F_kl = 1 / (lam_l - lam_k) (k != l), 0 on the diagonal;
  * B = H_2 - H_1:               H2_bar += B_bar, H1_bar -= B_bar;
  * A = W H (polar):             with Hs = sym(H_bar), M = W^T W_bar and
                                G = skew(M) - (Hs H - H Hs) / 2,
                                A_bar = W (2 L^{-1}(G) + Hs), where L(X) = X H + H X
                                is solved in the eigenbasis of H (H = Q diag(sig) Q^T,
                                its own Jacobi eigendecomposition):
                                L^{-1}(G) = Q [(Q^T G Q)_kl / (sig_k + sig_l)] Q^T.

The polar step follows from W^T dA = Omega H + dH with Omega = W^T dW skew:
Omega solves Omega H + H Omega = W^T dA - dA^T W (a Lyapunov equation) and
dH = sym(W^T dA) - (Omega H - H Omega) / 2.
"""
import numpy as np

from . import csd as O
from . import jacobi


def _skew(X):
    return 0.5 * (X - X.T)


def _sym(X):
    return 0.5 * (X + X.T)


def polar_adjoint(W, H, W_bar, H_bar):
    """A_bar of A = W H (W orthogonal, H symmetric positive definite)."""
    sig, Q, _ = jacobi.eig_cyclic(H)
    Hs = _sym(H_bar)
    G = _skew(W.T @ W_bar) - 0.5 * (Hs @ H - H @ Hs)
    Gq = Q.T @ G @ Q
    Linv = Q @ (Gq / (sig[:, None] + sig[None, :])) @ Q.T
    return W @ (2.0 * Linv + Hs)


def eig_adjoint(lam, V, V_bar):
    """B_bar of B = V diag(lam) V^T (distinct eigenvalues, lam not used by the loss)."""
    d = lam[None, :] - lam[:, None]          # lam_l - lam_k at (k, l)
    F = np.zeros_like(d)
    off = d != 0.0
    F[off] = 1.0 / d[off]
    return V @ (F * _skew(V.T @ V_bar)) @ V.T


def csd_backward(A1, A2, theta_bar=None, U1_bar=None, U2_bar=None, V_bar=None, res=None):
    """(A1_bar, A2_bar) for the outputs of oracle.csd (full rank, real)."""
    r = O.csd(A1, A2) if res is None else res
    n = A1.shape[1]
    if r["rank"] != n or np.iscomplexobj(A1):
        raise ValueError("the derivative is defined here for real full-rank inputs")
    z = np.zeros((n, n))
    theta_bar = np.zeros(n) if theta_bar is None else theta_bar
    U1_bar = z if U1_bar is None else U1_bar
    U2_bar = z if U2_bar is None else U2_bar
    V_bar = z if V_bar is None else V_bar
    V, U1, U2 = r["V1"], r["U1"], r["U2"]
    W1, W2, H1, H2 = r["W1"], r["W2"], r["H1"], r["H2"]
    theta = r["theta"]
    c = np.einsum("ij,ij->j", V, H1 @ V)
    s = np.einsum("ij,ij->j", V, H2 @ V)
    rr = c * c + s * s
    c_bar = -s / rr * theta_bar
    s_bar = c / rr * theta_bar
    H1_bar = V @ np.diag(c_bar) @ V.T
    H2_bar = V @ np.diag(s_bar) @ V.T
    Vt_bar = V_bar + 2.0 * H1 @ V @ np.diag(c_bar) + 2.0 * H2 @ V @ np.diag(s_bar)
    W1_bar = U1_bar @ V.T
    W2_bar = U2_bar @ V.T
    Vt_bar = Vt_bar + W1.T @ U1_bar + W2.T @ U2_bar
    # eigenvalues of B in the same (theta-sorted) column order as V
    lam = np.einsum("ij,ij->j", V, r["B"] @ V)
    B_bar = eig_adjoint(lam, V, Vt_bar)
    H1_bar = H1_bar - B_bar
    H2_bar = H2_bar + B_bar
    del theta
    return polar_adjoint(W1, H1, W1_bar, H1_bar), polar_adjoint(W2, H2, W2_bar, H2_bar)


def canonical_signs(res):
    """Flip each column of V1 (and of U1, U2 with it) so that its entry of
    largest magnitude is positive: the factors are unique for distinct
    angles, so a loss on U1 or V1 is a differentiable function of A."""
    V = res["V1"]
    idx = np.argmax(np.abs(V), axis=0)
    sg = np.sign(V[idx, np.arange(V.shape[1])])
    sg[sg == 0] = 1.0
    out = dict(res)
    for k in ("U1", "U2", "V1"):
        out[k] = res[k] * sg[None, :]
    return out
