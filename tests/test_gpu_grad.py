"""The differentiable path (csd_polar_backward and the torch.autograd
bridge): against the oracle's FP64 reverse-mode derivative (pinned on the CPU
by a closed form and central differences), against the closed form for
losses on the angles, and against central differences (h = 1e-6) of the GPU
forward itself on instances with n ~ U{16..256} and the loss
sum(theta^2) + ||U1 - U1_ref||^2."""
import numpy as np
import pytest

from oracle import csd as O
from oracle import grad as G
from paper_1804_09002_gb300 import inputs as I
from tests.gpu_util import to_dev, to_host

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def B():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1804_09002_gb300 import binding
    return binding


@pytest.fixture(scope="module")
def AG(B):
    from paper_1804_09002_gb300 import autograd
    return autograd


def _weights(n, rng):
    return (rng.standard_normal(n), rng.standard_normal((n, n)), rng.standard_normal((n, n)),
            rng.standard_normal((n, n)))


@pytest.mark.parametrize("n,tc", [(16, False), (37, False), (64, False), (130, False), (256, True)])
def test_backward_matches_oracle_gradient(B, n, tc):
    A1, A2, _ = I.haar_csd(n, seed=600 + n)
    rng = np.random.default_rng(n)
    w = _weights(n, rng)
    ref = G.canonical_signs(O.csd(A1, A2))
    g1o, g2o = G.csd_backward(A1, A2, *w, res=ref)
    ctx = B.Context(0)
    try:
        ctx.set_tensor_cores(tc)
        ctx.set_sign_convention(1)
        R = ctx.csd_polar(to_dev(A1), to_dev(A2))
        # the same canonical factors as the oracle's (distinct angles)
        assert np.max(np.abs(to_host(R["V1"]) - ref["V1"])) <= 1e-9
        g1, g2 = ctx.csd_backward(R["U1"], R["U2"], R["V1"], R["theta"], to_dev(w[1]), to_dev(w[2]), to_dev(w[3]),
                                  torch.from_numpy(w[0]).cuda())
    finally:
        ctx.close()
    g1, g2 = to_host(g1), to_host(g2)
    den = np.sqrt(np.linalg.norm(g1o) ** 2 + np.linalg.norm(g2o) ** 2)
    err = np.sqrt(np.linalg.norm(g1 - g1o) ** 2 + np.linalg.norm(g2 - g2o) ** 2) / den
    assert err <= 1e-8, err


def test_theta_loss_closed_form(B):
    """Loss on the angles only: A1_bar = U1 diag(-s w) V1^T, A2_bar =
    U2 diag(c w) V1^T (singular-value perturbation)."""
    n = 100
    A1, A2, _ = I.haar_csd(n, seed=77)
    w = np.random.default_rng(1).standard_normal(n)
    R = B.csd_polar(to_dev(A1), to_dev(A2))
    g1, g2 = B.default_context(0).csd_backward(R["U1"], R["U2"], R["V1"], R["theta"],
                                               gtheta=torch.from_numpy(w).cuda())
    U1, U2, V1, th = (to_host(R[k]) for k in ("U1", "U2", "V1", "theta"))
    c, s = np.cos(th), np.sin(th)
    assert np.max(np.abs(to_host(g1) - (U1 * (-s * w)[None, :]) @ V1.T)) <= 1e-13 * n
    assert np.max(np.abs(to_host(g2) - (U2 * (c * w)[None, :]) @ V1.T)) <= 1e-13 * n


def _loss(AG, A1, A2, U1_ref):
    U1, U2, V1, th = AG.csd(A1, A2)
    return (th ** 2).sum() + ((U1 - U1_ref) ** 2).sum()


def _separated_instance(n, seed, min_gap=1e-4, attempts=200):
    """Haar CSD with theta ~ U[0, pi/2] redrawn until every pair of angles is
    at least min_gap apart: where two angles cross, the sorted column order
    of U1 (hence the loss on U1) is not differentiable."""
    rng = np.random.default_rng(seed)
    for _ in range(attempts):
        theta = rng.uniform(0.0, np.pi / 2, n)
        if np.min(np.diff(np.sort(theta))) >= min_gap:
            break
    A1, A2 = I.from_angles(theta, rng)
    return A1, A2


def test_autograd_central_differences_sampled_sizes(AG):
    """16 instances with n drawn from U{16..256}: the directional derivative
    <grad, E> (E a random direction of Frobenius norm sqrt(n)) of
    sum(theta^2) + ||U1 - U1_ref||^2, U1_ref = U1(A) + 0.1 N(0, 1), against
    the central difference with step h = 1e-6 (fourth-order stencil), to
    1e-6 relative."""
    rng = np.random.default_rng(2025)
    sizes = rng.integers(16, 257, 16)
    worst = 0.0
    for i, n in enumerate(sizes):
        n = int(n)
        A1h, A2h = _separated_instance(n, 5000 + i)
        A1 = to_dev(A1h).clone().requires_grad_(True)
        A2 = to_dev(A2h).clone().requires_grad_(True)
        with torch.no_grad():
            U1_0 = AG.csd(A1, A2)[0].clone()
        U1_ref = U1_0 + 0.1 * torch.from_numpy(rng.standard_normal((n, n))).cuda()
        L = _loss(AG, A1, A2, U1_ref)
        L.backward()
        E1 = torch.from_numpy(rng.standard_normal((n, n))).cuda()
        E2 = torch.from_numpy(rng.standard_normal((n, n))).cuda()
        # ||E||_F = sqrt(n): h ||E||_2 stays near 2h, far below the 1e-4 angle
        # gap, while the directional derivative stays well above the rounding
        # noise of the loss (about n u |L| / h)
        nrm = float(torch.sqrt((E1 ** 2).sum() + (E2 ** 2).sum())) / np.sqrt(n)
        E1, E2 = E1 / nrm, E2 / nrm
        an = float((A1.grad * E1).sum() + (A2.grad * E2).sum())
        h = 1e-6
        with torch.no_grad():
            f = {j: float(_loss(AG, A1 + j * h * E1, A2 + j * h * E2, U1_ref)) for j in (-2, -1, 1, 2)}
        fd = (-f[2] + 8 * f[1] - 8 * f[-1] + f[-2]) / (12 * h)
        rel = abs(fd - an) / max(1.0, abs(an))
        worst = max(worst, rel)
        assert rel <= 1e-6, (n, fd, an)
    print(f"worst relative FD mismatch over {len(sizes)} instances: {worst:.2e}")
