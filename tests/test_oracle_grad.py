"""Pins of the oracle's reverse-mode CSD derivative (oracle/grad.py), on the
CPU: (1) a closed form for losses on the angles alone (singular-value
perturbation: dc_j = u1_j^T dA1 v_j, ds_j = u2_j^T dA2 v_j, so
d theta_j = c_j ds_j - s_j dc_j); (2) central finite differences of the
oracle's own forward (Algorithm 1) for a loss on theta, U1, U2 and V1 with
canonical column signs; (3) a planted mistake in the eig adjoint (the sign
of F) is caught by (2)."""
import numpy as np
import pytest

from oracle import csd as O
from oracle import grad as G
from paper_1804_09002_gb300 import inputs as I


def _loss_and_bars(res, w):
    wt, R1, R2, R0 = w
    L = float(wt @ res["theta"] + np.sum(R1 * res["U1"]) + np.sum(R2 * res["U2"]) + np.sum(R0 * res["V1"]))
    return L, (wt, R1, R2, R0)


def _fd(A1, A2, E1, E2, w, h=1e-6):
    def L(a1, a2):
        r = G.canonical_signs(O.csd(a1, a2))
        return _loss_and_bars(r, w)[0]
    return (L(A1 + h * E1, A2 + h * E2) - L(A1 - h * E1, A2 - h * E2)) / (2 * h)


@pytest.mark.parametrize("n,seed", [(5, 1), (8, 2)])
def test_theta_gradient_closed_form(n, seed):
    A1, A2, _ = I.haar_csd(n, seed=seed)
    r = O.csd(A1, A2)
    wt = np.random.default_rng(seed).standard_normal(n)
    g1, g2 = G.csd_backward(A1, A2, theta_bar=wt, res=r)
    c, s = np.cos(r["theta"]), np.sin(r["theta"])
    V, U1, U2 = r["V1"], r["U1"], r["U2"]
    want1 = (U1 * (-s * wt)[None, :]) @ V.T
    want2 = (U2 * (c * wt)[None, :]) @ V.T
    assert np.max(np.abs(g1 - want1)) <= 1e-12
    assert np.max(np.abs(g2 - want2)) <= 1e-12


@pytest.mark.parametrize("n,seed", [(5, 3), (9, 4)])
def test_full_gradient_matches_central_differences(n, seed):
    A1, A2, _ = I.haar_csd(n, seed=seed)
    rng = np.random.default_rng(100 + seed)
    w = (rng.standard_normal(n), rng.standard_normal((n, n)), rng.standard_normal((n, n)),
         rng.standard_normal((n, n)))
    r = G.canonical_signs(O.csd(A1, A2))
    g1, g2 = G.csd_backward(A1, A2, *w, res=r)
    for _ in range(3):
        E1, E2 = rng.standard_normal((n, n)), rng.standard_normal((n, n))
        fd = _fd(A1, A2, E1, E2, w)
        an = float(np.sum(g1 * E1) + np.sum(g2 * E2))
        assert abs(fd - an) <= 1e-6 * max(1.0, abs(an)), (fd, an)


def test_planted_sign_error_in_eig_adjoint_is_caught(monkeypatch):
    n = 6
    A1, A2, _ = I.haar_csd(n, seed=7)
    rng = np.random.default_rng(7)
    w = (rng.standard_normal(n), rng.standard_normal((n, n)), rng.standard_normal((n, n)),
         rng.standard_normal((n, n)))
    good = G.eig_adjoint
    monkeypatch.setattr(G, "eig_adjoint", lambda lam, V, Vb: -good(lam, V, Vb))
    r = G.canonical_signs(O.csd(A1, A2))
    g1, g2 = G.csd_backward(A1, A2, *w, res=r)
    E1, E2 = rng.standard_normal((n, n)), rng.standard_normal((n, n))
    fd = _fd(A1, A2, E1, E2, w)
    an = float(np.sum(g1 * E1) + np.sum(g2 * E2))
    assert abs(fd - an) > 1e-3 * max(1.0, abs(fd))
