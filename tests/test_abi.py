"""C-ABI library checks that need no GPU: it loads, exports every function
include/zolo_csd.h declares, rejects bad arguments before touching a device,
and its host-side Zolotarev coefficients and iteration plan agree with the
oracle (Section 5, Zolo-pd)."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def B():
    from paper_1804_09002_gb300 import build
    build.build()
    from paper_1804_09002_gb300 import binding
    return binding


def header_functions():
    src = open(os.path.join(ROOT, "include", "zolo_csd.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    decl = r"^(?:const\s+)?(?:int|long long|void|double|const char)\s*\**\s*([A-Za-z_][A-Za-z0-9_]*)\s*\("
    return sorted(set(re.findall(decl, src, flags=re.M)))


def test_exports_every_declared_function(B):
    names = header_functions()
    assert {"csd_polar", "polar", "heig", "csd_create", "csd_destroy"} <= set(names)
    lib = ctypes.CDLL(B.LIB_PATH)
    for nm in names:
        assert hasattr(lib, nm), nm
    assert set(names) <= set(B.EXPORTED)


def test_bad_arguments_are_rejected_without_a_device(B):
    lib = B.lib
    # NULL context is argument 1
    assert lib.csd_polar(None, 0, 4, None, 4, None, 4, None, 4, None, 4, None, 4, None, None, None) == -1
    assert lib.polar(None, 0, 4, None, 4, None, 4, None, 4, None) == -1
    assert lib.heig(None, 0, 4, None, 4, None, None, 4, None) == -1
    assert lib.csd_create(None, 0, None) == -1
    assert lib.csd_destroy(None) == 0
    assert lib.csd_complete_v2(None, 0, 4, None, 4, None, 4, None, 4, None, 4, None, None, 4, None) == -1
    assert lib.csd_set_theta_mode(None, 1) == -1
    assert lib.csd_polar_rect(None, 0, 8, 8, 4, None, 8, None, 8, None, 8, None, 8, None, 4, None, None, None) == -1
    assert lib.zolo_coeffs(0.0, 8, None, None, None, None) == -1
    assert lib.zolo_coeffs(0.5, 0, None, None, None, None) == -2
    assert lib.csd_set_zolo_control(None, 1, 0) == -1
    assert lib.csd_set_test_hooks(None, 0, 0, 0) == -1
    assert lib.csd_gemm(None, 0, 0, 4, 4, 4, 1.0, None, 4, None, 4, 0.0, None, 4, 1) == -1
    assert B.lib.csd_status_str(-3) == b"invalid argument"
    # entry points of the batched, differentiable and mixed-precision paths
    assert lib.csd_set_eig_leaf(None, 64) == -1
    assert lib.csd_set_mixed_precision(None, 6, 1) == -1
    assert lib.csd_set_alg2_fallback(None, 1e3) == -1
    assert lib.csd_set_sign_convention(None, 1) == -1
    assert lib.csd_polar_backward(None, 0, 4, None, 4, None, 4, None, 4, None, None, 4, None, 4, None, 4, None,
                                  None, 4, None, 4, None) == -1
    assert lib.csd_batch_create(None, 4, None, None) == -1
    assert lib.csd_batch_run(None, None, None, None, None, None, None, None) == -1
    assert lib.csd_batch_stats(None, None, None, None, None) == -1
    assert lib.csd_batch_destroy(None) == 0
    assert lib.csd_fp64_peak(-1, 0, None, None) == -1
    assert lib.csd_fp64_peak(0, 2, None, None) == -2
    assert lib.csd_fp64_peak(0, 0, None, None) == -3


def test_host_zolotarev_coefficients_match_oracle(B):
    zolo = pytest.importorskip("oracle.zolo")
    for ell, r in [(1e-15, 8), (0.4565318346870844, 8), (1e-3, 3), (0.5, 1), (0.9, 4)]:
        c, a, m, en = B.zolo_coeffs(ell, r)
        c0, a0, m0, en0 = zolo.as_float(zolo.coeffs(ell, r))
        assert np.max(np.abs(c / c0 - 1)) <= 1e-13
        assert np.max(np.abs(a / a0 - 1)) <= 1e-13
        assert abs(m / m0 - 1) <= 1e-14
        assert abs(en - en0) <= 1e-14


def test_host_plan_matches_oracle(B):
    zolo = pytest.importorskip("oracle.zolo")
    r, ell = B.zolo_plan(1e-15, 8, 4)
    steps = zolo.plan(1e-15)
    assert r == [co["r"] for co in steps]
    assert np.allclose(ell, [float(co["ell"]) for co in steps], rtol=1e-13, atol=0)
