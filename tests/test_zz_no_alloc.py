"""polar_noalloc: the polar decomposition for callers that cannot allocate
device memory (code that may not call cudaMalloc, e.g. inside callbacks or
under a fixed memory budget owned by someone else).  It must give the same
factors as the regular polar() entry point, call after call, while keeping
the device's free memory unchanged.  Collected last so that a failure here
does not hide any other test.
"""
import ctypes

import numpy as np
import pytest

from tests.gpu_util import U, to_dev, to_host

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def B():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1804_09002_gb300 import binding
    return binding


def _outputs(A):
    n = A.shape[0]
    return (torch.empty((n, n), dtype=A.dtype, device=A.device).t(),
            torch.empty((n, n), dtype=A.dtype, device=A.device).t())


def _noalloc(B, A, dtype_code, W, H):
    n = A.shape[0]
    return B.lib.polar_noalloc(dtype_code, n, A.data_ptr(), A.stride(1), W.data_ptr(), n, H.data_ptr(), n,
                               ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))


def test_polar_noalloc_matches_polar_on_consecutive_calls(B):
    rng = np.random.default_rng(2024)
    # the free-memory check is on the second call, whose kernels the first
    # call has already loaded (lazy module loading maps code on first use)
    cases = [(64, False), (50, False), (37, True), (64, True)]
    free_before = None
    for call, (n, cplx) in enumerate(cases):
        A = rng.standard_normal((n, n)) + (1j * rng.standard_normal((n, n)) if cplx else 0)
        A = A / np.linalg.norm(A, 2)
        Ad = to_dev(A)
        W, H = _outputs(Ad)
        torch.cuda.synchronize()
        if call == 1:
            free_before = torch.cuda.mem_get_info()[0]
        st = _noalloc(B, Ad, 1 if cplx else 0, W, H)
        torch.cuda.synchronize()
        if call == 1:
            assert torch.cuda.mem_get_info()[0] == free_before
        assert st == 0
        Wr, Hr, _ = B.polar(Ad)
        W, H, Wr, Hr = (to_host(x) for x in (W, H, Wr, Hr))
        kappa = np.linalg.cond(A)
        assert np.linalg.norm(W - Wr) <= 1e-13 * n * max(kappa, 1)
        assert np.linalg.norm(H - Hr) <= 50 * n * U
        assert np.linalg.norm(W.conj().T @ W - np.eye(n), 2) <= 50 * n * U
        assert np.linalg.norm(W @ H - A) <= 50 * n * U


def test_polar_noalloc_rejects_large_and_host_inputs(B):
    n = 65
    A = to_dev(np.eye(n))
    W, H = _outputs(A)
    assert _noalloc(B, A, 0, W, H) == -2
    Ah = np.asfortranarray(np.eye(8))
    W = torch.empty((8, 8), dtype=torch.float64, device="cuda:0")
    st = B.lib.polar_noalloc(0, 8, Ah.ctypes.data, 8, W.data_ptr(), 8, None, 8, None)
    assert st == -3
